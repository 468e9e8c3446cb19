"""Write the stored per-step sweep energies of the FP64 oracle DMRG (oracle/dmrg.py).

Two-site sweeps of Sec. 2.1 from the Aufbau product state, the same schedule
as dmrg_sweep: forward over positions 0..L-3, backward over L-2..1, each step
the lowest eigenpair of Eq. h_mat followed by the density-matrix truncation
to M states and the renormalization of Eq. renorm_mat.  Integrals from the
seeded synthetic generator (seed 0).  Only oracle/ computes; the GPU library
is not imported.  Run from the repository root:

    python tests/golden/make_oracle_sweeps.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dmrg as od  # noqa: E402
from paper_2001_04890_gb300 import workloads  # noqa: E402

CASES = [(12, 12, 0, 128, 4), (24, 24, 0, 32, 2)]  # L, N, 2Sz, M, sweeps
TOL = 1e-11


def path(L, N, two_sz, M, nsw):
    return os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        f"oracle_sweeps_L{L}_N{N}_2Sz{two_sz}_M{M}_S{nsw}.txt")


def main():
    for L, N, two_sz, M, nsw in CASES:
        h, v = workloads.integrals(L, seed=0)
        E = od.OracleDMRG(h, v, N, two_sz, M).sweep(nsw, tol=TOL)
        with open(path(L, N, two_sz, M, nsw), "w") as f:
            f.write(f"# FP64 oracle two-site DMRG energies (Eh), one per step: L={L} N={N} 2Sz={two_sz} M={M},\n"
                    f"# {nsw} sweeps from the Aufbau start, integrals seed 0, eigen-tolerance {TOL}.\n"
                    f"# Sweep schedule and truncation of Sec. 2.1; written by make_oracle_sweeps.py.\n")
            for e in E:
                f.write(f"{e:.15f}\n")
        print(L, M, nsw, "min", E.min(), flush=True)


if __name__ == "__main__":
    main()
