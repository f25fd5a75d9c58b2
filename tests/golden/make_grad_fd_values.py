"""Writes tests/golden/grad_large.json: FP64 oracle values that pin the GPU adjoint
dM_2/dpsi* at N = 17 and 18, where the oracle is too slow to run inside a GPU test.

For each state: the oracle's M_2, the norm of its gradient g, the projections 2 Re <g, d_k> on
16 seeded random unit directions d_k (a JL-style element-wise check: an error vector of norm
eps |g| shows in the projections), and for some states central finite differences of the
oracle's forward M_2 along d_0 (and d_1) with step h = 1e-4, which pin the oracle's gradient
itself at this size.

States (complex64 amplitudes, as the GPU reads them):
  * gauss17: inputs.gaussian_state(17, 717)  (the single-state adjoint test's N = 17 state);
  * ladder17, ladder18: the first N = 17 and N = 18 states of
    inputs.batched_ladder_states(64, 10, 18, 8, seed=4001) (the batched configuration).
Directions: d_k = (x + i y) / |x + i y| with x, y standard normal from PCG64(91000 + k).

Calls only `oracle/` (and the seeded input generators); about an hour of CPU:
    nice -n 10 python tests/golden/make_grad_fd_values.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2601_07824_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "grad_large.json")
H = 1e-4
K = 16


def direction(k: int, dim: int) -> np.ndarray:
    rng = np.random.default_rng(91000 + k)
    d = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    return d / np.linalg.norm(d)


def states():
    Ns, st = inputs.batched_ladder_states(64, 10, 18, 8, seed=4001)
    i17 = next(i for i, n in enumerate(Ns) if n == 17)
    i18 = next(i for i, n in enumerate(Ns) if n == 18)
    return {"gauss17": (inputs.gaussian_state(17, 717, dtype=np.complex64), 2),
            "ladder17": (st[i17], 1),
            "ladder18": (st[i18], 0)}, {"ladder17": i17, "ladder18": i18}


def main():
    d = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            d = json.load(f)
    d["_comment"] = ("FP64 oracle gradient projections and finite differences at N = 17, 18, written by "
                     "tests/golden/make_grad_fd_values.py (see its docstring for states, directions and h).")
    sts, idx = states()
    for name, (psi32, n_fd) in sts.items():
        if name in d:
            continue
        psi = psi32.astype(np.complex128)
        t = time.time()
        M2, g = oracle.sre_grad(psi)
        e = {"N": int(psi.size).bit_length() - 1, "M2": M2, "grad_norm": float(np.linalg.norm(g)),
             "proj": [float(2 * np.real(np.vdot(g, direction(k, psi.size)))) for k in range(K)]}
        if name in idx:
            e["batch_index"] = idx[name]
        e["fd"] = []
        for k in range(n_fd):
            dk = direction(k, psi.size)
            fp = oracle.sre(psi + H * dk, 2.0)[0]
            fm = oracle.sre(psi - H * dk, 2.0)[0]
            e["fd"].append((fp - fm) / (2 * H))
        e["oracle_s"] = round(time.time() - t, 1)
        d[name] = e
        with open(OUT, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
            f.write("\n")
        print(name, e["oracle_s"], flush=True)


if __name__ == "__main__":
    main()
