"""Writes tests/golden/oracle_config1.txt: a regression fixture of the FP64
oracle on the 64x128 five-region cell (seed 0), 200 steps at dt = 50 tau_exp.

Calls only ``oracle`` and ``workloads``.  Rerun only when the oracle's
arithmetic changes for a reason that names the paper passage behind it.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle  # noqa: E402
from workloads import heat as H  # noqa: E402


def main():
    p = H.config1()
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    E0, F0, Q = o.energy()
    o.step(tau, H.STEPS["config1"])
    T = o.field()
    E1, F1, _ = o.energy()
    rng = np.random.default_rng(123)
    idx = rng.choice(T.size, 24, replace=False)
    with open(os.path.join(HERE, "oracle_config1.txt"), "w") as f:
        f.write("# oracle regression fixture: config1 64x128 seed 0, 200 steps, dt = 50 tau_exp\n")
        f.write("# written by tests/golden/make_golden.py (calls only oracle/ and workloads/)\n")
        f.write(f"tau {tau:.17g}\nE0 {E0:.17g}\nE1 {E1:.17g}\nPhi1 {F1:.17g}\nQ {Q:.17g}\n")
        f.write(f"Tmax {T.max():.17g}\nTmin {T.min():.17g}\n")
        for k in idx:
            f.write(f"T {k} {T.flat[k]:.17g}\n")


if __name__ == "__main__":
    main()
