"""Writes tests/golden/oracle_full_size.json: the FP64 oracle's values for the full-size bench
workloads, so that the GPU results at full size have an independent reference.

  * exact M_2 (Eq. sre, Algorithm 2) and lost_norm of the N = 20 brick-wall Haar state (depth 10,
    open chain, seed 2001, complex64 amplitudes as the GPU reads them);
  * mana (Eq. mana2, Algorithm 5) and sum |W| of the N = 11 qutrit Gaussian state (seed 1101,
    complex64).

Calls only `oracle/` (and the seeded input generators).  Several CPU hours at N = 20:
    nice -n 19 python tests/golden/make_full_size_values.py [mana|sre|all]
Each value is written as soon as it is computed.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2601_07824_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "oracle_full_size.json")


def _save(key, value):
    d = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            d = json.load(f)
    d["_comment"] = ("FP64 oracle (oracle/hadamag_oracle.c) on the full-size bench inputs, written by "
                     "tests/golden/make_full_size_values.py; inputs are the complex64 amplitudes the GPU reads.")
    d[key] = value
    with open(OUT, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
        f.write("\n")


def mana11():
    q = inputs.gaussian_state(11, 1101, d=3, dtype=np.complex64)
    t = time.time()
    m, sw = oracle.mana(q)
    _save("mana_gaussian_N11_seed1101", {"cite": "Eq. (mana2), Algorithm 5 (log2 convention, 1/3^N factor)",
                                         "mana": m, "sum_abs_w": sw, "oracle_s": round(time.time() - t, 1)})


def sre20():
    psi = inputs.brickwork_haar(20, 10, seed=2001, dtype=np.complex64)
    t = time.time()
    M2, ln = oracle.sre(psi, 2.0)
    _save("sre_brickwork_N20_depth10_seed2001", {"cite": "Eq. (sre), Algorithm 2, lost_norm of Sec. 4.1",
                                                  "M2": M2, "lost_norm": ln, "oracle_s": round(time.time() - t, 1)})


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("mana", "all"):
        mana11()
    if what in ("sre", "all"):
        sre20()
