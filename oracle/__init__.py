"""Plain FP64 CPU oracle for the BSSN right-hand side, Kreiss-Oliger
dissipation, RK4 step, ghost filling and constraints.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this package. It shares no code with the CUDA library
and never imports it.

Arrays are numpy float64 of shape (24, nz+2g, ny+2g, nx+2g) (variable,
z, y, x; x fastest) unless stated otherwise.
"""
import ctypes
import os

import numpy as np

from .build import build as _build

_L = None

_i = ctypes.c_int
_d = ctypes.c_double
_ll = ctypes.c_longlong
_p = ctypes.c_void_p


def lib():
    global _L
    if _L is None:
        path = _build()
        L = ctypes.CDLL(path)
        L.oracle_fd_weight.argtypes = [ctypes.POINTER(_i), _i, _i, _i, ctypes.POINTER(_ll), ctypes.POINTER(_ll)]
        L.oracle_stencils.argtypes = [_i, _p, _p, ctypes.POINTER(_i), ctypes.POINTER(_i), _p, ctypes.POINTER(_i), _p]
        L.oracle_required_ghost.argtypes = [_i]
        L.oracle_required_ghost.restype = _i
        L.oracle_apply_op.argtypes = [_i, _i, _i, _i, _d, _d, _d, _i, _i, _i, _i, _d, _p, _p]
        L.oracle_rhs.argtypes = [_i, _i, _i, _i, _d, _d, _d, _ll, _i, _d, _i, _i, _d, _d, _i, _p, _p]
        L.oracle_rhs.restype = _i
        L.oracle_rhs_points.argtypes = [_i, _i, _i, _i, _d, _d, _d, _ll, _i, _d, _i, _i, _d, _d, _i, _i, _ll, _p, _p,
                                         _p]
        L.oracle_rhs_points.restype = _i
        L.oracle_ko.argtypes = [_i, _i, _i, _i, _d, _d, _d, _ll, _i, _d, _p, _p]
        L.oracle_ko.restype = _i
        L.oracle_fill_ghosts.argtypes = [_i, _i, _i, _i, _ll, _i, _p, _p]
        L.oracle_fill_ghosts.restype = _i
        L.oracle_rk4_step.argtypes = [_i, _i, _i, _i, _d, _d, _d, _ll, _i, _d, _i, _i, _d, _d, _i, _i, _p, _d, _p]
        L.oracle_rk4_step.restype = _i
        L.oracle_rk3_step.argtypes = L.oracle_rk4_step.argtypes
        L.oracle_rk3_step.restype = _i
        L.oracle_constraints.argtypes = [_i, _i, _i, _i, _d, _d, _d, _ll, _i, _p, _p, _p, _p, _p, _p]
        L.oracle_constraints.restype = _i
        L.oracle_psi4.argtypes = [_i, _i, _i, _i, _d, _d, _d, _ll, _i, _d, _d, _d, _p, _p, _p, _p, _p, _p, _p]
        L.oracle_psi4.restype = _i
        L.oracle_flop_counts.argtypes = [_i, _p]
        L.oracle_flop_counts.restype = _i
        L.oracle_restrict.argtypes = [_i, _i, _i, _i, _ll, _i, _i, _i, _i, _ll, _i, _p, _p]
        L.oracle_restrict.restype = _i
        L.oracle_prolong.argtypes = [_i, _i, _i, _i, _ll, _i, _i, _i, _i, _ll, _p, _p]
        L.oracle_prolong.restype = _i
        L.oracle_conv3d_fwd.argtypes = [_i, _i, _i, _i, _i, _i, _p, _p, _p, _p]
        L.oracle_conv3d_bwd.argtypes = [_i, _i, _i, _i, _i, _i, _p, _p, _p, _p, _p, _p]
        L.oracle_gelu.argtypes = [_ll, _p, _p]
        L.oracle_gelu_grad.argtypes = [_ll, _p, _p]
        L.oracle_corrector_loss.argtypes = [_i, _i, _i, _i, _i, _p, _p, _p, _p, _p, _p]
        L.oracle_corrector_loss.restype = _d
        _L = L
    return _L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check_state(u, g):
    assert u.dtype == np.float64 and u.flags.c_contiguous and u.ndim == 4 and u.shape[0] == 24
    nz, ny, nx = (s - 2 * g for s in u.shape[1:])
    return nx, ny, nz, int(np.prod(u.shape[1:]))


class Params:
    """Evolution parameters: fd_order 4|8, ko_eps, lapse (0 1+log, 1 harmonic,
    2 frozen), shift (0 Gamma-driver, 1 frozen), shift_coeff, eta,
    advect_gauge (1: beta^k d_k on alpha, beta, B)."""

    def __init__(self, fd_order=4, ko_eps=0.1, lapse=0, shift=0, shift_coeff=0.75, eta=2.0, advect_gauge=1):
        self.fd_order = fd_order
        self.ko_eps = ko_eps
        self.lapse = lapse
        self.shift = shift
        self.shift_coeff = shift_coeff
        self.eta = eta
        self.advect_gauge = advect_gauge


def required_ghost(order):
    return lib().oracle_required_ghost(order)


def fd_weight(offsets, m, j):
    o = (ctypes.c_int * len(offsets))(*offsets)
    num, den = _ll(), _ll()
    lib().oracle_fd_weight(o, len(offsets), m, j, ctypes.byref(num), ctypes.byref(den))
    return num.value, den.value


def stencils(order):
    c1 = np.zeros(8)
    c2 = np.zeros(8)
    up = np.zeros(12)
    ko = np.zeros(12)
    lo, n, r = _i(), _i(), _i()
    lib().oracle_stencils(order, _ptr(c1), _ptr(c2), ctypes.byref(lo), ctypes.byref(n), _ptr(up), ctypes.byref(r), _ptr(ko))
    h = order // 2
    return dict(c1=c1[:h].copy(), c2=c2[:h].copy(), up_lo=lo.value, up=up[:n.value].copy(), r=r.value,
                ko=ko[:2 * r.value + 1].copy())


def apply_op(u, g, h, order, kind, a=0, b=0, beta=0.0):
    """One operator on a single padded grid function u (nz+2g, ny+2g, nx+2g):
    kind 0 first derivative along a, 1 second along a, 2 mixed a,b,
    3 upwinded advection beta*d_a (beta constant), 4 Kreiss-Oliger with eps=beta."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    nz, ny, nx = (s - 2 * g for s in u.shape)
    out = np.zeros_like(u)
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    lib().oracle_apply_op(nx, ny, nz, g, hx, hy, hz, order, kind, a, b, beta, _ptr(u), _ptr(out))
    return out


def rhs(u, g, h, p: Params, ko=False):
    """BSSN RHS at interior points (ghosts of u must be filled); with ko=True
    the Kreiss-Oliger term is added."""
    nx, ny, nz, vs = _check_state(u, g)
    out = np.zeros_like(u)
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    rc = lib().oracle_rhs(nx, ny, nz, g, hx, hy, hz, vs, p.fd_order, p.ko_eps, p.lapse, p.shift, p.shift_coeff,
                          p.eta, p.advect_gauge, _ptr(u), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_rhs: invalid arguments")
    if ko:
        rc = lib().oracle_ko(nx, ny, nz, g, hx, hy, hz, vs, p.fd_order, p.ko_eps, _ptr(u), _ptr(out))
        if rc != 0:
            raise ValueError("oracle_ko: invalid arguments")
    return out


def rhs_points(u, g, h, p: Params, lin, ko=False):
    """RHS (+KO) at interior points lin = i + nx (j + ny k); returns (len(lin), 24)."""
    nx, ny, nz, vs = _check_state(u, g)
    lin = np.ascontiguousarray(lin, dtype=np.int64)
    out = np.zeros((len(lin), 24))
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    rc = lib().oracle_rhs_points(nx, ny, nz, g, hx, hy, hz, vs, p.fd_order, p.ko_eps, p.lapse, p.shift,
                                 p.shift_coeff, p.eta, p.advect_gauge, int(ko), len(lin), _ptr(lin), _ptr(u), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_rhs_points: invalid arguments")
    return out


def algebraic_constraints(u, g):
    """The algebraic constraints of the conformal decomposition at interior
    points (the BSSN variables of Sec. 1.1 satisfy det(gt_ij) = 1 and
    gt^ij At_ij = 0 for exact data): returns (det(gt) - 1, gt^ij At_ij),
    each (nz, ny, nx). The determinant is the cofactor expansion along the
    first row written out; the trace contracts At with numpy's inverse of
    gt."""
    _check_state(u, g)
    ui = u[:, g:-g, g:-g, g:-g]
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    G = np.zeros(ui.shape[1:] + (3, 3))
    A = np.zeros(ui.shape[1:] + (3, 3))
    for s, (i, j) in enumerate(pairs):
        G[..., i, j] = G[..., j, i] = ui[1 + s]
        A[..., i, j] = A[..., j, i] = ui[8 + s]
    det = (G[..., 0, 0] * (G[..., 1, 1] * G[..., 2, 2] - G[..., 1, 2] * G[..., 2, 1])
           - G[..., 0, 1] * (G[..., 1, 0] * G[..., 2, 2] - G[..., 1, 2] * G[..., 2, 0])
           + G[..., 0, 2] * (G[..., 1, 0] * G[..., 2, 1] - G[..., 1, 1] * G[..., 2, 0]))
    tr = np.einsum("...ij,...ij->...", np.linalg.inv(G), A)
    return det - 1.0, tr


def ko(u, g, h, p: Params):
    nx, ny, nz, vs = _check_state(u, g)
    out = np.zeros_like(u)
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    rc = lib().oracle_ko(nx, ny, nz, g, hx, hy, hz, vs, p.fd_order, p.ko_eps, _ptr(u), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_ko: invalid arguments")
    return out


def fill_ghosts(u, g, mode=0, src=None):
    """In place: mode 0 periodic, mode 1 static (ghosts copied from src)."""
    nx, ny, nz, vs = _check_state(u, g)
    if src is not None:
        src = np.ascontiguousarray(src, dtype=np.float64)
        assert src.shape == u.shape
    rc = lib().oracle_fill_ghosts(nx, ny, nz, g, vs, mode, _ptr(src), _ptr(u))
    if rc != 0:
        raise ValueError("oracle_fill_ghosts: invalid arguments")
    return u


def rk4_step(u, g, h, dt, p: Params, bc=0, ghost_src=None):
    """One RK4 step (RHS + KO), returns a new array."""
    nx, ny, nz, vs = _check_state(u, g)
    y = u.copy()
    if ghost_src is not None:
        ghost_src = np.ascontiguousarray(ghost_src, dtype=np.float64)
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    rc = lib().oracle_rk4_step(nx, ny, nz, g, hx, hy, hz, vs, p.fd_order, p.ko_eps, p.lapse, p.shift,
                               p.shift_coeff, p.eta, p.advect_gauge, bc, _ptr(ghost_src), dt, _ptr(y))
    if rc != 0:
        raise ValueError("oracle_rk4_step: invalid arguments")
    return y


def rk3_step(u, g, h, dt, p: Params, bc=0, ghost_src=None):
    """One SSP-RK3 (Shu-Osher) step (RHS + KO), returns a new array."""
    nx, ny, nz, vs = _check_state(u, g)
    y = u.copy()
    if ghost_src is not None:
        ghost_src = np.ascontiguousarray(ghost_src, dtype=np.float64)
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    rc = lib().oracle_rk3_step(nx, ny, nz, g, hx, hy, hz, vs, p.fd_order, p.ko_eps, p.lapse, p.shift,
                               p.shift_coeff, p.eta, p.advect_gauge, bc, _ptr(ghost_src), dt, _ptr(y))
    if rc != 0:
        raise ValueError("oracle_rk3_step: invalid arguments")
    return y


def constraints(u, g, h, fd_order, fields=False):
    """Returns (l2[7], max[7], status) for H, M1..3, G1..3 and, with
    fields=True, also (ham, mom[3], gcon[3]) arrays in padded layout."""
    nx, ny, nz, vs = _check_state(u, g)
    l2 = np.zeros(7)
    mx = np.zeros(7)
    ham = mom = gcon = None
    if fields:
        ham = np.zeros(u.shape[1:])
        mom = np.zeros((3,) + u.shape[1:])
        gcon = np.zeros((3,) + u.shape[1:])
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    rc = lib().oracle_constraints(nx, ny, nz, g, hx, hy, hz, vs, fd_order, _ptr(u), _ptr(ham), _ptr(mom),
                                  _ptr(gcon), _ptr(l2), _ptr(mx))
    if rc < 0:
        raise ValueError("oracle_constraints: invalid arguments")
    if fields:
        return l2, mx, rc, (ham, mom, gcon)
    return l2, mx, rc


def psi4(u, g, h, fd_order, origin):
    """Weyl diagnostics at interior points: returns dict with psi4 (complex),
    inv (complex, I = Q_ij Q^ij / 2), E and B (6 packed components each),
    all padded-layout arrays; origin = coordinates of interior point (0,0,0)."""
    nx, ny, nz, vs = _check_state(u, g)
    shape = u.shape[1:]
    pr, pi, ir, ii = (np.zeros(shape) for _ in range(4))
    E = np.zeros((6,) + shape)
    B = np.zeros((6,) + shape)
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    rc = lib().oracle_psi4(nx, ny, nz, g, hx, hy, hz, vs, fd_order, float(origin[0]), float(origin[1]),
                           float(origin[2]), _ptr(u), _ptr(pr), _ptr(pi), _ptr(ir), _ptr(ii), _ptr(E), _ptr(B))
    if rc < 0:
        raise ValueError("oracle_psi4: invalid arguments")
    return dict(psi4=pr + 1j * pi, inv=ir + 1j * ii, E=E, B=B, finite=(rc == 0))


def flop_counts(fd_order):
    out = np.zeros(8, dtype=np.int64)
    rc = lib().oracle_flop_counts(fd_order, _ptr(out))
    if rc != 0:
        raise ValueError("bad order")
    keys = ["first", "second", "mixed_tensor", "upwind_dir", "ko_var", "rhs_algebra", "gather_rhs",
            "constraints_algebra"]
    return dict(zip(keys, (int(x) for x in out)))


# ------------------------------------------------------------------ 2:1 transfer
def restrict(f, fg, cg, order=4):
    """Fine state (24, 2nz+2fg, 2ny+2fg, 2nx+2fg) -> coarse (24, nz+2cg, ...),
    interior only (coarse ghosts zero). order 2: mean of the 8 fine children;
    order 4: tricubic interpolation at the coarse centre (fine ghosts >= 1,
    filled)."""
    fnx, fny, fnz, fvs = _check_state(f, fg)
    cnx, cny, cnz = fnx // 2, fny // 2, fnz // 2
    c = np.zeros((24, cnz + 2 * cg, cny + 2 * cg, cnx + 2 * cg))
    rc = lib().oracle_restrict(fnx, fny, fnz, fg, fvs, cnx, cny, cnz, cg, int(np.prod(c.shape[1:])), order, _ptr(f),
                               _ptr(c))
    if rc != 0:
        raise ValueError("oracle_restrict: invalid arguments")
    return c


def prolong(c, cg, fg):
    """Coarse state (ghosts >= 2 filled) -> fine interior (fine ghosts zero)."""
    cnx, cny, cnz, cvs = _check_state(c, cg)
    f = np.zeros((24, 2 * cnz + 2 * fg, 2 * cny + 2 * fg, 2 * cnx + 2 * fg))
    rc = lib().oracle_prolong(cnx, cny, cnz, cg, cvs, 2 * cnx, 2 * cny, 2 * cnz, fg, int(np.prod(f.shape[1:])),
                              _ptr(c), _ptr(f))
    if rc != 0:
        raise ValueError("oracle_prolong: invalid arguments")
    return f


# ------------------------------------------------------------------ corrector network (corrector_oracle.cpp)
def conv3d_fwd(x, W, b):
    """x: (S, Z, Y, X, Ci); W: (27, Co, Ci), tap (dz+1)*9+(dy+1)*3+(dx+1); b: (Co,).
    Zero padding. Returns (S, Z, Y, X, Co)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    b = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    S, Z, Y, X, Ci = x.shape
    Co = W.shape[1]
    out = np.zeros((S, Z, Y, X, Co))
    lib().oracle_conv3d_fwd(S, Z, Y, X, Ci, Co, _ptr(x), _ptr(W), _ptr(b), _ptr(out))
    return out


def conv3d_bwd(x, W, dout):
    """Gradients (dx, dW, db) of conv3d_fwd for upstream gradient dout."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    dout = np.ascontiguousarray(dout, dtype=np.float64)
    S, Z, Y, X, Ci = x.shape
    Co = W.shape[1]
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    db = np.zeros(Co)
    lib().oracle_conv3d_bwd(S, Z, Y, X, Ci, Co, _ptr(x), _ptr(W), _ptr(dout), _ptr(dx), _ptr(dW), _ptr(db))
    return dx, dW, db


def gelu(x, grad=False):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    (lib().oracle_gelu_grad if grad else lib().oracle_gelu)(x.size, _ptr(x), _ptr(y))
    return y


def corrector_loss(params, channels, x, target, want_grad=True):
    """Loss (and gradient, packed like params, and output) of the conv+GELU
    network with the given channel list on x (S, Z, Y, X, ch[0])."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    target = np.ascontiguousarray(target, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    ch = np.ascontiguousarray(channels, dtype=np.int32)
    S, Z, Y, X, _ = x.shape
    out = np.zeros((S, Z, Y, X, channels[-1]))
    grad = np.zeros_like(params) if want_grad else None
    loss = lib().oracle_corrector_loss(S, Z, Y, X, len(channels) - 1, ch.ctypes.data_as(ctypes.c_void_p),
                                       _ptr(params), _ptr(x), _ptr(target), _ptr(out), _ptr(grad))
    return loss, grad, out


def corrector_param_count(channels):
    return sum(27 * channels[l + 1] * channels[l] + channels[l + 1] for l in range(len(channels) - 1))
