"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

Run from the repository root: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from workloads import chain_hamiltonian  # noqa: E402


def chain512():
    # Dimerized chain t1 = -1.0, t2 = -0.6, N = 512, Nocc = 256, tol 1e-12:
    # the SP2 recursion of §IV.A on the Gershgorin-bounded X0 map.
    H, nocc = chain_hamiltonian(512, -1.0, -0.6)
    emin, emax = oracle.gershgorin_bounds(H)
    out = {"n": 512, "nocc": nocc, "tol": 1e-12, "emin": emin, "emax": emax}
    for name, rule in (("nearer", oracle.NEARER), ("paper", oracle.PAPER)):
        r = oracle.sp2_plain(H, nocc, 1e-12, rule=rule)
        out[name] = {"iters": r["iters"], "bits": "".join(map(str, r["bits"])),
                     "trace_x0": r["t1"][0], "trace_x0_sq": r["t2"][0]}
    return out


if __name__ == "__main__":
    path = os.path.join(HERE, "chain512_sp2.json")
    with open(path, "w") as f:
        json.dump(chain512(), f, indent=1, sort_keys=True)
        f.write("\n")
    print("wrote", path)
