"""Write the oracle's energies of the CAS(6,6), 10 core, 100 virtual, 400
auxiliary workload to tests/golden/oracle_cas66_c10_v100_q400.json.

Calls only the CPU oracle (oracle.dsrg_df, the block-restricted
density-fitted FP64 evaluation of Eqs. T2_1st .. E(3)) on the seeded input
from synth/.  Besides the energies it records, for each input array, its
SHA-256 on the machine that ran this script and float fingerprints (sum,
sum of squares, sum with alternating signs) that a test can check on other
machines, where libm or BLAS rounding may change the last bits of the
generated cumulants (the energies move by ~1e-13 Eh then, far below the
1e-9 Eh the tests ask).

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import dsrg_df  # noqa: E402

WORKLOAD = "cas66_c10_v100_q400"
ARRAYS = ("eps", "B", "g1a", "g1b", "l2aa", "l2ab", "l2bb", "l3aaa", "l3aab", "l3abb", "l3bbb")


def fingerprints(inst):
    out = {}
    for k in ARRAYS:
        a = np.ascontiguousarray(inst[k], dtype=np.float64).ravel()
        alt = np.where(np.arange(a.size) % 2 == 0, 1.0, -1.0)
        out[k] = {"sha256": hashlib.sha256(a.tobytes()).hexdigest(), "size": int(a.size),
                  "sum": float(np.sum(a)), "sumsq": float(np.dot(a, a)), "altsum": float(np.dot(a, alt))}
    return out


def main():
    inst = synth.config_instance(WORKLOAD)
    t0 = time.time()
    e = dsrg_df.dsrg_pt3(inst)
    secs = time.time() - t0
    rec = {
        "workload": WORKLOAD,
        "sizes": {k: inst[k] for k in ("nc", "na", "nv", "naux")}, "s": inst["s"],
        "energies_Eh": {k: e[k] for k in ("e2", "e3a", "e3b", "e3")},
        "oracle": "oracle.dsrg_df.dsrg_pt3 (FP64, block-restricted, density-fitted)",
        "oracle_seconds": round(secs, 1), "machine": f"{platform.machine()}, {os.cpu_count()} cores",
        "inputs": fingerprints(inst),
        "script": "tests/golden/make_golden.py",
    }
    path = os.path.join(HERE, f"oracle_{WORKLOAD}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(path, rec["energies_Eh"], f"{secs:.1f} s")


if __name__ == "__main__":
    main()
