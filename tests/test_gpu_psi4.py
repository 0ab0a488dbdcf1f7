"""Weyl diagnostics through the C ABI (bssn_psi4) against the oracle:
E_ij, B_ij, Psi_4 and the invariant I on perturbed Brill-Lindquist data
(every variable non-zero, ragged anisotropic grid) at both orders, and on
Kerr in Kerr-Schild coordinates. Tolerance: 1e-11 of each output's largest
magnitude (these are products of second derivatives, one order of rounding
growth beyond the right-hand side's 1e-12)."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B

from gpu_common import grid_for, need_gpu, perturbed_bl

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import exact  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-11


def gpu_psi4(u, g, h, order, origin):
    torch = need_gpu()
    grid = grid_for(u, g, h)
    p = B.make_params(fd_order=order)
    d = B.upload(u, grid)
    outs = [B.alloc_state(grid) for _ in range(2)]  # 24 arrays each: room for E (6) and B (6), psi, inv
    work = B.alloc_work(grid, p)
    vs = grid.var_stride
    v0, v1 = outs[0], outs[1]
    B.psi4(grid, p, d, origin, work, psi_re=v0[0:vs], psi_im=v0[vs:2 * vs], inv_re=v0[2 * vs:3 * vs],
           inv_im=v0[3 * vs:4 * vs], E=v1[0:6 * vs], B=v1[6 * vs:12 * vs])
    torch.cuda.synchronize()
    a0, a1 = B.download(v0, grid), B.download(v1, grid)
    return dict(psi4=a0[0] + 1j * a0[1], inv=a0[2] + 1j * a0[3], E=a1[0:6], B=a1[6:12])


def compare(got, want, g):
    I = (Ellipsis, slice(g, -g), slice(g, -g), slice(g, -g))
    for k in ("psi4", "inv", "E", "B"):
        scale = np.max(np.abs(want[k][I]))
        assert scale > 0, k
        err = np.max(np.abs(got[k][I] - want[k][I])) / scale
        assert err < TOL, (k, err)


@pytest.mark.parametrize("order", [4, 8])
def test_psi4_perturbed(order):
    g = order // 2 + 1
    h = (0.11, 0.13, 0.12)
    u = perturbed_bl(19, 13, 11, g, 0.12, seed=41 + order)
    origin = (-1.03, 0.21, -0.57)
    compare(gpu_psi4(u, g, h, order, origin), oracle.psi4(u, g, h, order, origin), g)


def test_psi4_kerr():
    order, g, n, h = 4, 3, 16, 0.1
    lo = (0.9, 1.3, -0.8)
    X, Y, Z = exact.box(n, n, n, g, lo, h)
    u = exact.kerr_schild(X, Y, Z, 1.0, 0.6)
    origin = tuple(l + 0.5 * h for l in lo)
    compare(gpu_psi4(u, g, h, order, origin), oracle.psi4(u, g, h, order, origin), g)
