"""Helpers shared by the GPU parity tests: building the library, moving
seeded inputs to the device and the per-variable error norm.

Error norm (per variable v, over interior points):
    err_v = max |gpu - oracle| / max(max |oracle_v|, 1e-300)
"""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs

RHS_TOL = 1e-12     # right-hand side, double precision
STEPS_TOL = 1e-10   # state after 10 RK4 steps, double precision


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_1307_6488_gb300 import build as _b
    _b.build(bounds_check=os.environ.get("BSSN_BOUNDS_CHECK") == "1")
    return torch


def interior(a, g):
    return a[..., g:a.shape[-3] - g, g:a.shape[-2] - g, g:a.shape[-1] - g]


def rel_err(got, want, g):
    gi = interior(got, g).reshape(got.shape[0], -1)
    wi = interior(want, g).reshape(want.shape[0], -1)
    scale = np.maximum(np.max(np.abs(wi), axis=1), 1e-300)
    return np.max(np.abs(gi - wi), axis=1) / scale


TENSORS = [[0], list(range(1, 7)), [7], list(range(8, 14)), list(range(14, 17)), [17], list(range(18, 21)),
           list(range(21, 24))]


def rel_err_tensor(got, want, g):
    """Per-variable error normalised by the largest magnitude of any
    component of the same tensor field (W, gt_ij, K, At_ij, Gt^i, alpha,
    beta^i, B^i). Used for states after several steps: rounding differences
    of order eps_mach |u| in the O(1) components, differentiated twice
    (1/h^2), feed components that are themselves only 1e-10 (seeded noise);
    their size relative to themselves then reflects rounding order, in the
    oracle as much as in the GPU path, while relative to the tensor's norm
    it does not."""
    gi = interior(got, g).reshape(got.shape[0], -1)
    wi = interior(want, g).reshape(want.shape[0], -1)
    mag = np.max(np.abs(wi), axis=1)
    scale = np.zeros_like(mag)
    for grp in TENSORS:
        scale[grp] = np.max(mag[grp])
    return np.max(np.abs(gi - wi), axis=1) / np.maximum(scale, 1e-300)


def oracle_params(p):
    return oracle.Params(fd_order=p.fd_order, ko_eps=p.ko_eps, lapse=p.lapse, shift=p.shift,
                         shift_coeff=p.shift_coeff, eta=p.eta, advect_gauge=p.advect_gauge)


def grid_for(u, g, h):
    nz, ny, nx = (s - 2 * g for s in u.shape[1:])
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    return B.make_grid(nx, ny, nz, ghost=g, dx=hx, dy=hy, dz=hz)


def perturbed_bl(nx, ny, nz, g, h, seed=7, amp=1e-2):
    """Brill-Lindquist-like data with off-grid punctures plus a seeded smooth
    perturbation of every variable (so every term of the right-hand side,
    both shift signs and the off-diagonal metric are exercised)."""
    n = max(nx, ny, nz)
    u, _ = inputs.brill_lindquist(n, g, lo=-n * h / 2, hi=n * h / 2, masses=(0.3, 0.25),
                                  centers=((-0.37 * n * h / 2, 0.11, 0.05), (0.41 * n * h / 2, -0.07, 0.13)))
    u = np.ascontiguousarray(u[:, :nz + 2 * g, :ny + 2 * g, :nx + 2 * g])
    inputs.smooth_perturbation(u, g, amp, seed, h)
    return u


def gauge_wave_c1(n=24, g=3):
    """Gauge wave A = 0.01 along x on [-0.5, 0.5]^3, seeded noise 1e-10 (seed 1307)."""
    return inputs.gauge_wave(n, g, amplitude=0.01, noise=1e-10, seed=1307)
