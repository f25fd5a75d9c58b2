"""Thermodynamic-integration estimate of M_2 (Sec. 3.2, Eqs. Boltz to M2_TI, Algorithm 3),
FP64 NumPy.  TEST INFRASTRUCTURE ONLY: only `tests/` may import this module.

The X-strings a are sampled from Pi_beta(a) = exp(-beta f(a)) / Z_beta with the "energy"
f(a) = -ln(S(a) + eps), S(a) = sum_b |<psi|X_a Z_b|psi>|^4 (the per-X-string sum of
Algorithm 2, taken from the FP64 oracle), and
    <f>_beta = -d ln Z_beta / d beta,  Z_0 = 2^N,  Z_1 = S_2 + 2^N eps.

Readings (the printed text is inconsistent here):
  * Sign.  Integrating <f>_beta = -d ln Z / d beta over [0, 1] gives ln Z_0 - ln Z_1, so
    I = int_0^1 <f>_beta d beta = -ln((S_2 + 2^N eps) / 2^N) and
    M_2 = -log2(exp(-I) - eps)  (eps = 0: M_2 = I / ln 2).
    The printed identity (ln Z_1 - ln Z_0) and Algorithm 3's return value (-1/ln 2 times the
    quadrature) carry the opposite sign; as printed they give M_2 <= 0.
  * Natural log in f: Z_1 = sum_a exp(-f(a)) = S_2 requires f = -ln S, not -log2 S.
  * Quadrature: composite Simpson on L points beta_l = l / (L - 1).  Algorithm 3 asks for an
    even L, which gives an odd number of intervals; for even L the last three intervals use
    Simpson's 3/8 rule.
  * Random numbers: each chain l draws from SplitMix64 (the generator of the uniform-X
    estimator) seeded with seed + l; per step one output picks the bit to flip (the local,
    symmetric proposal: one uniformly chosen bit of a) and one output, as a double in [0, 1)
    from its top 53 bits, decides acceptance; the start pattern is the top N bits of the
    chain's first output.
  * Even sector (sector="even", Sec. 3.2's restriction of the chain for U(1) or Z_2^Z symmetric
    states, whose odd-weight X-strings have S(a) = 0): the chains stay on even-weight a.  The
    start pattern gets its bit 0 flipped when its weight is odd; each step flips two distinct
    bits drawn from the step's first output r as b1 = r mod N, b2 = (r div N) mod (N-1),
    b2 += 1 if b2 >= b1 (a symmetric move that spans the sector).  Then Z_0 = 2^(N-1),
    Z_1 = S_2 + 2^(N-1) eps and M_2 = 1 - log2(exp(-I) - eps).
  * Statistical error (Eqs. Var_I_eps, m2error): Var[I] ~ sum_l w_l^2 2 tau_int sigma_f^2 / n_l,
    delta M_2 = (d M_2 / d I) sqrt(Var[I]).  The paper does not say how 2 tau_int sigma_f^2 / n_l
    is estimated; here by non-overlapping batch means (the variance of the mean of a correlated
    series is the spread of means of batches much longer than tau_int): the n_s recorded
    samples of a chain are cut into B = min(32, n_s) batches of K = n_s div B consecutive
    samples (the last n_s - B K samples enter the mean only), and
    Var_l = sum_b (m_b - mbar)^2 / (B (B - 1)).  d M_2 / d I = exp(-I) / ((exp(-I) - eps) ln 2).
    With B < 2 the error is reported as 0.
"""
from __future__ import annotations

import math

import numpy as np


def energies(psi, eps: float = 0.0) -> np.ndarray:
    """f(a) = -ln(S(a) + eps) for every X-string a (S(a) from the FP64 oracle)."""
    import oracle
    Sq, _, _ = oracle.sre_terms(psi, 2.0)
    S = Sq + eps
    if np.any(S <= 0.0):
        raise ValueError("S(a) + eps must be positive for every a (use eps > 0)")
    return -np.log(S)


def energy_fn(psi, eps: float = 0.0):
    """f(a) = -ln(S(a) + eps) evaluated on demand, one X-string at a time, and cached: the
    chains visit a small part of the 2^N X-strings, so this is what makes N >= 14 cheap.
    Raises ValueError when an evaluated S(a) + eps is not positive."""
    import oracle
    cache = {}

    def f(a: int) -> float:
        v = cache.get(a)
        if v is None:
            S = float(oracle.sre_terms_list(psi, [a])[0]) + eps
            if S <= 0.0:
                raise ValueError("S(a) + eps must be positive for every visited a (use eps > 0)")
            v = cache[a] = -math.log(S)
        return v
    return f


def even_mask(N: int) -> np.ndarray:
    """True at the even-weight X-strings a in [0, 2^N)."""
    a = np.arange(1 << N)
    w = np.zeros_like(a)
    for j in range(N):
        w += (a >> j) & 1
    return (w & 1) == 0


def boltzmann_mean(f: np.ndarray, beta: float) -> float:
    """<f>_beta = sum_a Pi_beta(a) f(a), Eq. f_expect_beta_reg, by enumeration over the given
    energies (all a, or the sector's)."""
    x = -beta * f
    w = np.exp(x - x.max())
    return float(np.sum(w * f) / np.sum(w))


def simpson_weights(L: int) -> np.ndarray:
    """Weights of composite Simpson's rule on L equally spaced points of [0, 1] (L >= 3); for
    even L the last three intervals use the 3/8 rule."""
    if L < 3:
        raise ValueError("L >= 3")
    h = 1.0 / (L - 1)
    w = np.zeros(L)
    n13 = L - 1 if L % 2 == 1 else L - 4  # intervals covered by the 1/3 rule
    for i in range(0, n13, 2):
        w[i] += h / 3.0
        w[i + 1] += 4.0 * h / 3.0
        w[i + 2] += h / 3.0
    if L % 2 == 0:
        i = L - 4
        w[i] += 3.0 * h / 8.0
        w[i + 1] += 9.0 * h / 8.0
        w[i + 2] += 9.0 * h / 8.0
        w[i + 3] += 3.0 * h / 8.0
    return w


def m2_from_integral(I: float, eps: float = 0.0, sector: str | None = None) -> float:
    """M_2 = -log2(exp(-I) - eps) (Eq. M2_TI_reg_explicit_correct with the sign reading); in
    the even sector Z_0 = 2^(N-1), so M_2 = 1 - log2(exp(-I) - eps)."""
    return -math.log2(math.exp(-I) - eps) + (1.0 if sector == "even" else 0.0)


def m2_ti_exact(psi, L: int, eps: float = 0.0, sector: str | None = None) -> float:
    """Thermodynamic integration with the exact integrand <f>_beta (quadrature error only)."""
    f = energies(psi, eps) if sector is None else energies_sector(psi, eps, sector)
    betas = np.linspace(0.0, 1.0, L)
    I = float(np.dot(simpson_weights(L), [boltzmann_mean(f, b) for b in betas]))
    return m2_from_integral(I, eps, sector)


def energy_table(psi, eps: float = 0.0, sector: str | None = None) -> np.ndarray:
    """f[a] for every a; with sector="even" only the even-weight entries are evaluated (and must
    be finite), the others are +inf, which a chain kept in the sector never reads."""
    if sector is None:
        return energies(psi, eps)
    fs = energies_sector(psi, eps, sector)
    N = int(round(math.log2(np.asarray(psi).size)))
    f = np.full(1 << N, np.inf)
    f[even_mask(N)] = fs
    return f


def energies_sector(psi, eps: float, sector: str) -> np.ndarray:
    """Energies of the sector's X-strings only (sector = "even")."""
    import oracle
    if sector != "even":
        raise ValueError("sector must be 'even'")
    Sq, _, _ = oracle.sre_terms(psi, 2.0)
    N = int(round(math.log2(Sq.size)))
    S = Sq[even_mask(N)] + eps
    if np.any(S <= 0.0):
        raise ValueError("S(a) + eps must be positive for every a of the sector (use eps > 0)")
    return -np.log(S)


def n_batches(n_s: int) -> int:
    """Batches of the batch-means error estimate: B = min(32, n_s)."""
    return min(32, n_s)


def metropolis_means(f, N: int, L: int, n_s: int, seed: int, burn_in: int = 0, record: dict | None = None,
                     sector: str | None = None):
    """Algorithm 3's chains: per beta_l, n_s Metropolis steps (one-bit flips, acceptance
    min(1, exp(-beta (f' - f)))) after `burn_in` unrecorded ones; returns (means, visits)
    with visits[l][a] = how often the recorded chain state was a.

    f is the energy table (f[a] for every a) or a callable a -> f(a).  With `record` given,
    record["traj"][l, t] is the chain state after step t (burn-in included) and
    record["margin"][l, t] = |u - p_acc| of that step's decision (how far the decision was
    from going the other way), and record["batch_sums"][l, b] the sum of the recorded energies
    of batch b (batches of n_s div B consecutive recorded steps, B = n_batches(n_s)).
    sector="even" keeps the chains on even-weight X-strings."""
    import oracle
    energy = f if callable(f) else f.__getitem__
    betas = np.linspace(0.0, 1.0, L)
    means = np.zeros(L)
    visits = np.zeros((L, 1 << N), dtype=np.int64) if not callable(f) else None
    steps = burn_in + n_s
    B = n_batches(n_s)
    K = n_s // B
    if record is not None:
        record["traj"] = np.zeros((L, steps), dtype=np.int64)
        record["margin"] = np.zeros((L, steps))
        record["batch_sums"] = np.zeros((L, B))
    for l, beta in enumerate(betas):
        r = oracle.splitmix64(seed + l, 1 + 2 * steps)
        a = int(r[0] >> np.uint64(64 - N)) if N > 0 else 0
        if sector == "even" and bin(a).count("1") % 2 == 1:
            a ^= 1
        fa = energy(a)
        acc = 0.0
        for t in range(steps):
            u = float(r[2 + 2 * t] >> np.uint64(11)) * 2.0 ** -53
            if sector == "even":
                b1 = int(r[1 + 2 * t] % np.uint64(N))
                b2 = int((r[1 + 2 * t] // np.uint64(N)) % np.uint64(N - 1))
                if b2 >= b1:
                    b2 += 1
                a2 = a ^ (1 << b1) ^ (1 << b2)
            else:
                a2 = a ^ (1 << int(r[1 + 2 * t] % np.uint64(N)))
            f2 = energy(a2)
            p_acc = math.exp(min(0.0, -beta * (f2 - fa)))
            if u < p_acc:
                a, fa = a2, f2
            if record is not None:
                record["traj"][l, t] = a
                record["margin"][l, t] = abs(u - p_acc)
            if t >= burn_in:
                acc += fa
                if visits is not None:
                    visits[l, a] += 1
                b = (t - burn_in) // K
                if record is not None and b < B:
                    record["batch_sums"][l, b] += fa
        means[l] = acc / n_s
    return means, visits


def m2_stderr(batch_sums: np.ndarray, n_s: int, I: float, eps: float = 0.0) -> float:
    """delta M_2 of Eq. m2error from the chains' batch sums (batch-means reading above)."""
    L, B = batch_sums.shape
    if B < 2:
        return 0.0
    K = n_s // B
    w = simpson_weights(L)
    var_I = 0.0
    for l in range(L):
        m = batch_sums[l] / K
        var_I += w[l] ** 2 * float(np.sum((m - m.mean()) ** 2)) / (B * (B - 1))
    slope = math.exp(-I) / ((math.exp(-I) - eps) * math.log(2.0))
    return slope * math.sqrt(var_I)


def m2_metropolis(psi, L: int, n_s: int, seed: int, burn_in: int = 0, eps: float = 0.0,
                  record: dict | None = None, sector: str | None = None) -> float:
    """Algorithm 3 (with the sign reading): M_2 estimate from L chains of n_s samples.  Up to
    12 qubits the energy table is built for every a; beyond, energies are evaluated on demand."""
    psi = np.asarray(psi)
    N = int(round(math.log2(psi.size)))
    f = energy_table(psi, eps, sector) if N <= 12 else energy_fn(psi, eps)
    means, _ = metropolis_means(f, N, L, n_s, seed, burn_in, record, sector)
    return m2_from_integral(float(np.dot(simpson_weights(L), means)), eps, sector)
