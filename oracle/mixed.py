"""Mixed-state qutrit mana, FP64 NumPy.  TEST INFRASTRUCTURE ONLY.

Only `tests/` may import this module.  It is the reference for a mixed-state mana kernel:
a plain restatement of the fast tensor-product transform of Sec. 3.3.3 (Algorithm 6), pinned
in `tests/test_oracle_mana_mixed.py` to the dense definition W_u = tr(rho A_u) / 3^N
(Eq. mana, phase-space operators of Eq. phase-space; `brute.wigner_mixed_brute`), to the
pure-state oracle (Algorithm 5) on rho = |psi><psi|, and to closed forms and invariants.

Conventions and readings (the paper is inconsistent or silent here):
  * Sites: site k is base-3 digit k of a row or column index of rho (least significant
    first), as for state vectors everywhere in this package.
  * Vec_N (Sec. 3.3.3): v[p] = rho[r, c] with mu_k = 3 i_k + j_k, i_k / j_k the digit k of
    the row r / column c, and p = sum_k mu_k 9^(N-1-k) (site 0 is the most significant base-9
    digit, as printed).  The printed single-qutrit vec is column-stacked (alpha = i + 3j)
    while mu_k is row-stacked; the single-qutrit matrix must use the convention of Vec_N:
    w_u = tr(rho A_u) = sum_{i,j} rho_ij (A_u)_ji, so M[u, 3i + j] = (A_u)[j, i].
  * Phase-space labels: u = 3a + b for the single-qutrit operator built from
    T_ab = w^(-2^-1 ab) Z^a X^b, the labelling of `brute.phase_point_operators`.
  * Normalisation: Algorithm 6 returns log2 sum_u |w_u|; the Wigner function of Eq. (mana)
    carries 1 / 3^N, so mana = log2(sum_u |w_u| / 3^N) (zero on |0><0|).
"""
from __future__ import annotations

import numpy as np

from . import brute


def _n_sites(dim: int, d: int = 3) -> int:
    N = 0
    while d ** N < dim:
        N += 1
    if d ** N != dim:
        raise ValueError(f"dimension must be {d}^N")
    return N


def reduced_density_matrix(psi, keep, d: int = 3) -> np.ndarray:
    """rho_A = tr_B |psi><psi| for the sites in `keep` (site keep[m] becomes digit m of rho_A),
    for sites of dimension d (qutrits by default).

    The partial trace of Sec. 4.3's mixed-state example, written out: rho_A[r, c] =
    sum_x psi[(r, x)] conj(psi[(c, x)]) over the digits x of the traced-out sites."""
    psi = np.asarray(psi, dtype=np.complex128).ravel()
    N = _n_sites(psi.size, d)
    keep = list(keep)
    if len(set(keep)) != len(keep) or any(k < 0 or k >= N for k in keep):
        raise ValueError("keep must list distinct sites in [0, N)")
    rest = [k for k in range(N) if k not in keep]
    # axis t of the reshaped tensor is site N-1-t (the most significant digit comes first)
    t = psi.reshape((d,) * N) if N else psi.reshape(())
    order = [N - 1 - k for k in reversed(keep)] + [N - 1 - k for k in reversed(rest)]
    m = np.transpose(t, order).reshape(d ** len(keep), d ** len(rest))
    return m @ m.conj().T


def single_qutrit_M() -> np.ndarray:
    """M[u, mu] with w_u = sum_mu M[u, mu] v_mu for one qutrit, v_mu = rho[i, j], mu = 3i + j."""
    As, _ = brute.phase_point_operators(1)  # As[u], u = 3a + b
    M = np.zeros((9, 9), dtype=np.complex128)
    for u in range(9):
        for i in range(3):
            for j in range(3):
                M[u, 3 * i + j] = As[u][j, i]
    return M


def vec_n(rho) -> np.ndarray:
    """Vec_N(rho) of Sec. 3.3.3: v[p(i, j)] = rho[r, c], p = sum_k (3 i_k + j_k) 9^(N-1-k)."""
    rho = np.asarray(rho, dtype=np.complex128)
    D = rho.shape[0]
    N = _n_sites(D)
    v = np.zeros(9 ** N, dtype=np.complex128)
    for c in range(D):
        jd = [(c // 3 ** k) % 3 for k in range(N)]
        for r in range(D):
            idg = [(r // 3 ** k) % 3 for k in range(N)]
            p = 0
            for k in range(N):
                p = 9 * p + 3 * idg[k] + jd[k]
            v[p] = rho[r, c]
    return v


def wigner_mixed(rho) -> np.ndarray:
    """W_u = tr(rho A_u) / 3^N for all u by Algorithm 6: v = Vec_N(rho), then M applied to
    every fiber along every leg (leg l: fibers of 9 elements n_s = 9^(N-1-l) apart).  Entry p
    of the result belongs to u with base-9 digit (site k) u_k = 3a + b, k = 0 most
    significant."""
    rho = np.asarray(rho, dtype=np.complex128)
    N = _n_sites(rho.shape[0])
    M = single_qutrit_M()
    v = vec_n(rho)
    for leg in range(N):
        n_s = 9 ** (N - 1 - leg)
        blocks = v.reshape(-1, 9, n_s)  # [block][a][m]: fiber (block, m) is blocks[b, :, m]
        v = np.einsum("ua,bam->bum", M, blocks).reshape(-1)
    return v / 3 ** N


def mana_mixed(rho):
    """(mana in bits, sum_u |W_u|) of a qutrit density matrix (Eq. mana via Algorithm 6)."""
    W = wigner_mixed(rho)
    s = float(np.abs(W).sum())
    return float(np.log2(s)), s
