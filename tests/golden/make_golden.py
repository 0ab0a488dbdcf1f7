"""Writes the stored oracle values under tests/golden/ (calls only the oracle
and the seeded input generators):

  rhs_samples_o8.txt  BSSN right-hand side with Kreiss-Oliger dissipation
                      (Sec. 3.3; 8th-order stencils, 1+log lapse, Gamma-driver
                      shift) at 24 seeded interior points of a perturbed
                      Brill-Lindquist block
  rhs_samples_o4.txt  the same at 4th order with harmonic lapse and frozen
                      shift

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1307_6488_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    "o8": dict(fd_order=8, lapse=0, shift=0, ko_eps=0.1),
    "o4": dict(fd_order=4, lapse=1, shift=1, ko_eps=0.05),
}
NX, NY, NZ, H = 20, 18, 16, 0.125
NPTS = 24


def block(g):
    """Perturbed Brill-Lindquist block (20 x 18 x 16 interior, h = 1/8,
    punctures off-grid, seeded plane-wave perturbation 1e-2, seed 6488)."""
    n = max(NX, NY, NZ)
    u, _ = inputs.brill_lindquist(n, g, lo=-n * H / 2, hi=n * H / 2, masses=(0.3, 0.25),
                                  centers=((-0.37 * n * H / 2, 0.11, 0.05), (0.41 * n * H / 2, -0.07, 0.13)))
    u = np.ascontiguousarray(u[:, :NZ + 2 * g, :NY + 2 * g, :NX + 2 * g])
    inputs.smooth_perturbation(u, g, 1e-2, 6488, H)
    return u


def points():
    rng = np.random.default_rng(1307)
    return np.sort(rng.choice(NX * NY * NZ, NPTS, replace=False)).astype(np.int64)


def compute(case):
    kw = CASES[case]
    g = oracle.required_ghost(kw["fd_order"])
    u = block(g)
    lin = points()
    out = oracle.rhs_points(u, g, H, oracle.Params(**kw), lin, ko=True)
    return g, lin, out


def path(case):
    return os.path.join(HERE, f"rhs_samples_{case}.txt")


def load(case):
    a = np.loadtxt(path(case), comments="#")
    return a[:, 0].astype(np.int64), a[:, 1:]


def main():
    for case, kw in CASES.items():
        g, lin, out = compute(case)
        with open(path(case), "w") as f:
            f.write(f"# BSSN RHS + KO (Sec. 3.3) from the FP64 oracle, params {kw}, ghost {g}\n")
            f.write(f"# block: {NX}x{NY}x{NZ} interior, h = {H}, perturbed Brill-Lindquist (make_golden.block)\n")
            f.write("# columns: linear interior index i + nx (j + ny k), then the 24 variables in state order\n")
            for p, row in zip(lin, out):
                f.write(str(int(p)) + " " + " ".join(repr(float(v)) for v in row) + "\n")


if __name__ == "__main__":
    main()
