"""Writes tgv128_500_oracle_u.txt: the FP64 oracle's velocity after 500
steps of the 16-bit storage workload's flow at 128^3 (D3Q27 Taylor-Green +
uniform +-1e-3 velocity noise, seed 20120206, rho = 1, u0 = 0.02,
tau = 0.6, other rates 1, periodic, no force), at 1024 cells drawn by
workloads.sample_cells (seed 20120208).  Calls only the oracle; the run
takes about 10 minutes on 16 cores.

    python tests/golden/make_tgv128_oracle.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

SHAPE = (128, 128, 128)
STEPS = 500
COUNT = 1024
OUT = os.path.join(HERE, "tgv128_500_oracle_u.txt")


def main():
    oracle.build()
    Q = 27
    om = W.omegas(Q, 1 / 0.6)
    rho, u = W.taylor_green(SHAPE, u0=0.02, noise=1e-3)
    f = oracle.run(Q, SHAPE, oracle.equilibrium(Q, rho, u, np.zeros(3)), np.zeros(3), om, STEPS)
    _, vel = oracle.macroscopic(Q, f, np.zeros(3))
    cells = W.sample_cells(SHAPE, COUNT)
    v = vel.reshape(3, -1)[:, cells]
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle, D3Q27 Taylor-Green + noise 128^3, tau 0.6, %d steps: "
                 "cell u_x u_y u_z at %d cells of workloads.sample_cells(seed 20120208); "
                 "written by make_tgv128_oracle.py\n" % (STEPS, COUNT))
        for n, c in enumerate(cells):
            fh.write("%d %.17g %.17g %.17g\n" % (c, v[0, n], v[1, n], v[2, n]))


if __name__ == "__main__":
    main()
