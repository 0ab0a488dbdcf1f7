"""Pins for the oracle's SOLA Navier-Stokes kernels (oracle/cfd.py), the
paper's three-kernel CFD benchmark (Sec. 3.2), not GPU:
  * a uniform flow with periodic boundaries is an exact fixed point;
  * fluid at rest under gravity with the hydrostatic pressure stays at rest;
  * total momentum is conserved with periodic boundaries by the velocity
    kernel (flux form) and by the mass-conservation kernel;
  * a red-black half-sweep over all cells of one colour at once equals the
    sequential sweep over them (brute force, one cell at a time), and every
    cell's own divergence becomes (1 - omega) D;
  * the mass-conservation iteration drives the divergence to zero;
  * the 2D Taylor-Green vortex (an exact Navier-Stokes solution) is
    reproduced at second order.
"""
import math

import numpy as np
import pytest

from oracle import cfd
from paper_1307_6488_gb300 import inputs


def _rand(shape, seed, amp=1.0):
    return amp * inputs.uniform_noise(seed, 3, shape)


def test_uniform_flow_periodic_is_exact():
    F = cfd.Flow((8, 6, 4), (0.1, 0.2, 0.15), (True, True, True), nu=0.02, dt=0.01)
    F.u[...] = 0.3
    F.v[...] = -0.2
    F.w[...] = 0.1
    F.p[...] = 1.7
    for _ in range(3):
        F.step()
    assert np.all(F.u == 0.3) and np.all(F.v == -0.2) and np.all(F.w == 0.1) and np.all(F.p == 1.7)


def test_hydrostatic_rest_stays_at_rest():
    n, h = (6, 5, 7), (0.2, 0.25, 0.1)
    gz = -9.8
    F = cfd.Flow(n, h, (False, False, False), nu=0.01, dt=0.002, g=(0.0, 0.0, gz))
    z = (np.arange(-1, n[2] + 1) + 0.5) * h[2]
    F.p[...] = (2.0 + gz * z)[:, None, None]
    p0 = F.p.copy()
    for _ in range(5):
        F.step()
    assert np.max(np.abs(F.u)) < 1e-13 and np.max(np.abs(F.v)) < 1e-13 and np.max(np.abs(F.w)) < 1e-13
    assert np.max(np.abs(F.interior(F.p) - F.interior(p0))) < 1e-12


def test_momentum_conserved_periodic():
    F = cfd.Flow((8, 6, 6), (0.1, 0.1, 0.1), (True, True, True), nu=0.05, dt=0.005, alpha=0.4)
    sh = F.u.shape
    F.u[...] = _rand(sh, 1)
    F.v[...] = _rand(sh, 2)
    F.w[...] = _rand(sh, 3)
    F.p[...] = _rand(sh, 4)
    F.boundary()
    tot = [F.interior(f).sum() for f in (F.u, F.v, F.w)]
    F.velocity()
    F.boundary()
    for t, f in zip(tot, (F.u, F.v, F.w)):
        assert abs(F.interior(f).sum() - t) < 1e-11
    tot = [F.interior(f).sum() for f in (F.u, F.v, F.w)]
    for _ in range(3):
        F.mass_iteration()
        F.boundary()
    for t, f in zip(tot, (F.u, F.v, F.w)):
        assert abs(F.interior(f).sum() - t) < 1e-11


def test_half_sweep_equals_sequential_sweep():
    """Periodic in x and y, walls in z: the vectorised red-black half-sweeps
    against a one-cell-at-a-time sweep in the same order; each visited cell's
    own divergence becomes (1 - omega) times its value before the visit."""
    n, h = (4, 4, 3), (0.3, 0.2, 0.25)
    F = cfd.Flow(n, h, (True, True, False), nu=0.01, dt=0.02, omega=1.6)
    sh = F.u.shape
    F.u[...] = _rand(sh, 11)
    F.v[...] = _rand(sh, 12)
    F.w[...] = _rand(sh, 13)
    F.boundary()
    G = cfd.Flow(n, h, (True, True, False), nu=0.01, dt=0.02, omega=1.6)
    for a, b in ((G.u, F.u), (G.v, F.v), (G.w, F.w), (G.p, F.p)):
        a[...] = b
    F.mass_iteration()

    nx, ny, nz = n
    dt, om = 0.02, 1.6

    def face(f, idx):
        # periodic wrap of the x and y face indices into the padded array
        k, j, i = idx
        return f, (k + 1, (j % ny) + 1, (i % nx) + 1)

    for colour in (0, 1):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    if (i + j + k) % 2 != colour:
                        continue
                    faces = [(G.u, (k, j, i), (k, j, i - 1), h[0], True, True),
                             (G.v, (k, j, i), (k, j - 1, i), h[1], True, True),
                             (G.w, (k, j, i), (k - 1, j, i), h[2], k < nz - 1, k > 0)]

                    def div():
                        d = 0.0
                        for f, hi, lo, hh, _, _ in faces:
                            fa, ia = face(f, hi)
                            fb, ib = face(f, lo)
                            d += (fa[ia] - fb[ib]) / hh
                        return d

                    d0 = div()
                    s = sum((mh + ml) / (hh * hh) for _, _, _, hh, mh, ml in faces)
                    dp = -(om / (dt * s)) * d0
                    G.p[k + 1, j + 1, i + 1] += dp
                    for f, hi, lo, hh, mh, ml in faces:
                        if mh:
                            fa, ia = face(f, hi)
                            fa[ia] += dt * dp / hh
                        if ml:
                            fb, ib = face(f, lo)
                            fb[ib] -= dt * dp / hh
                    assert abs(div() - (1 - om) * d0) < 1e-12 * (1 + abs(d0))
        # periodic ghosts of the sequential copy for the next colour
        G.boundary()
    G.boundary()
    F.boundary()
    for a, b in ((G.u, F.u), (G.v, F.v), (G.w, F.w), (G.p, F.p)):
        np.testing.assert_allclose(F.interior(b), G.interior(a), rtol=0, atol=1e-13)


def test_mass_iterations_remove_divergence():
    n = (8, 6, 7)
    F = cfd.Flow(n, (0.1, 0.1, 0.1), (False, True, False), nu=0.01, dt=0.01, omega=1.7)
    sh = F.u.shape
    F.u[...] = _rand(sh, 21)
    F.v[...] = _rand(sh, 22)
    F.w[...] = _rand(sh, 23)
    F.boundary()
    d0 = np.max(np.abs(F.divergence()))
    for _ in range(150):
        F.mass_iteration()
        F.boundary()
    assert np.max(np.abs(F.divergence())) < 1e-9 * d0


def _taylor_green_error(N, T=0.5, nu=0.1):
    L = 2 * math.pi
    h = L / N
    dt = 0.1 * h * h / nu  # forward Euler in time: dt ~ h^2 keeps its error second order in h
    steps = max(1, int(round(T / dt)))
    dt = T / steps
    F = cfd.Flow((N, N, 2), (h, h, h), (True, True, True), nu=nu, dt=dt, omega=1.8, alpha=0.0)
    xc = (np.arange(-1, N + 1) + 0.5) * h   # cell centres
    xf = (np.arange(-1, N + 1) + 1.0) * h   # faces i + 1/2

    def exact(t):
        Fd = math.exp(-2 * nu * t)
        u = np.sin(xf)[None, None, :] * np.cos(xc)[None, :, None] * Fd
        v = -np.cos(xc)[None, None, :] * np.sin(xf)[None, :, None] * Fd
        p = (np.cos(2 * xc)[None, None, :] + np.cos(2 * xc)[None, :, None]) / 4 * Fd * Fd
        sh = F.u.shape
        return np.broadcast_to(u, sh), np.broadcast_to(v, sh), np.broadcast_to(p, sh)

    u, v, p = exact(0.0)
    F.u[...] = u
    F.v[...] = v
    F.p[...] = p
    for _ in range(steps):
        F.step(iterations=100)  # converged pressure: the error is the discretisation's
    u, v, p = exact(T)
    return max(np.max(np.abs(F.interior(F.u) - F.interior(np.ascontiguousarray(u)))),
               np.max(np.abs(F.interior(F.v) - F.interior(np.ascontiguousarray(v)))))


@pytest.mark.slow
def test_taylor_green_second_order():
    e = [_taylor_green_error(N) for N in (16, 32, 64)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert e[0] < 1e-3 and min(orders) > 1.8 and 1.8 < orders[-1] < 2.3, (e, orders)
