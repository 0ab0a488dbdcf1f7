"""Closed-form solutions of the Einstein equations in BSSN variables, used
as pins for the oracle. Everything here comes from each solution's metric
and the ADM definitions; none of it re-types the oracle's evolution
equations. First derivatives that the definitions need (extrinsic curvature
from the shift and metric, contracted conformal Christoffels from the inverse
conformal metric, time derivatives) are taken by complex-step
differentiation, f'(x) = Im f(x + i e)/e with e = 1e-30, which is exact to
rounding for analytic f.

Conformal decomposition used to map (gamma_ij, K_ij) to BSSN variables:
  W = det(gamma)^(-1/6),  gt_ij = W^2 gamma_ij,  K = gamma^ij K_ij,
  At_ij = W^2 (K_ij - K gamma_ij / 3),  Gt^i = -d_j gt^ij  (det gt = 1).
"""
import numpy as np

from paper_1307_6488_gb300.inputs import IDX, NVAR, SYM

PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
CS = 1e-30


def box(nx, ny, nz, g, lo, h):
    """Cell-centred padded coordinate arrays (z, y, x ordering)."""
    xs = [lo[a] + (np.arange(-g, n + g) + 0.5) * h for a, n in enumerate((nx, ny, nz))]
    Zm, Ym, Xm = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return Xm, Ym, Zm


def _cstep(f, xyz, axis):
    """d f / d x_axis by complex step; f takes a list [x, y, z] of arrays."""
    p = [np.asarray(c, dtype=np.complex128) for c in xyz]
    p[axis] = p[axis] + 1j * CS
    return np.imag(f(p)) / CS


def _pack(W, gt, trK, At, Gt, alpha, beta_up, B=None):
    shape = np.shape(W)
    u = np.zeros((NVAR,) + shape)
    u[IDX["W"]] = W
    for (i, j) in PAIRS:
        u[IDX["gt11"] + SYM[i][j]] = gt[i][j]
        u[IDX["At11"] + SYM[i][j]] = At[i][j]
    u[IDX["trK"]] = trK
    for i in range(3):
        u[IDX["Gt1"] + i] = Gt[i]
        u[IDX["beta1"] + i] = beta_up[i]
        if B is not None:
            u[IDX["B1"] + i] = B[i]
    u[IDX["alpha"]] = alpha
    return u


# ---------------------------------------------------------------- Kerr-Schild
def ks_radius(xyz, a):
    """Kerr-Schild (= Boyer-Lindquist) r: the root of
    (x^2 + y^2) / (r^2 + a^2) + z^2 / r^2 = 1."""
    x, y, z = xyz
    rho2 = x * x + y * y + z * z
    q = rho2 - a * a
    return np.sqrt(0.5 * q + np.sqrt(0.25 * q * q + a * a * z * z))


def _ks_parts(xyz, M, a=0.0):
    x, y, z = xyz
    r = ks_radius(xyz, a)
    H = M * r ** 3 / (r ** 4 + a * a * z * z)
    l = [(r * x + a * y) / (r * r + a * a), (r * y - a * x) / (r * r + a * a), z / r]
    gam = [[(1.0 if i == j else 0.0) + 2 * H * l[i] * l[j] for j in range(3)] for i in range(3)]
    gamu = [[(1.0 if i == j else 0.0) - 2 * H * l[i] * l[j] / (1 + 2 * H) for j in range(3)] for i in range(3)]
    det = 1 + 2 * H
    alpha = 1 / np.sqrt(1 + 2 * H)
    beta_dn = [2 * H * l[i] for i in range(3)]
    beta_up = [2 * H * l[i] / (1 + 2 * H) for i in range(3)]
    return gam, gamu, det, alpha, beta_dn, beta_up


def kerr_schild(Xm, Ym, Zm, M=1.0, a=0.0):
    """Kerr (spin a along z; a = 0: Schwarzschild) in Kerr-Schild coordinates
    with its own (stationary) lapse and shift: gamma_ij = delta_ij + 2 H l_i
    l_j, H = M r^3 / (r^4 + a^2 z^2), l = ((r x + a y), (r y - a x)) / (r^2 +
    a^2), z / r), alpha = (1+2H)^(-1/2), beta_i = 2 H l_i. The extrinsic
    curvature follows from d_t gamma_ij = 0 = -2 alpha K_ij + D_i beta_j +
    D_j beta_i. Returns the 24-variable state (B = 0)."""
    xyz = [Xm, Ym, Zm]
    gam, gamu, det, alpha, beta_dn, beta_up = _ks_parts(xyz, M, a)
    dgam = [[[_cstep(lambda p, i=i, j=j: _ks_parts(p, M, a)[0][i][j], xyz, k) for j in range(3)] for i in range(3)]
            for k in range(3)]  # dgam[k][i][j] = d_k gamma_ij
    dbeta = [[_cstep(lambda p, j=j: _ks_parts(p, M, a)[4][j], xyz, i) for j in range(3)] for i in range(3)]
    Kdn = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            s = dbeta[i][j] + dbeta[j][i]
            for l_ in range(3):
                G_lij = 0.5 * (dgam[i][l_][j] + dgam[j][l_][i] - dgam[l_][i][j])
                s = s - 2 * G_lij * beta_up[l_]
            Kdn[i][j] = s / (2 * alpha)
    W = det ** (-1.0 / 6.0)
    gt = [[W * W * gam[i][j] for j in range(3)] for i in range(3)]
    trK = sum(gamu[i][j] * Kdn[i][j] for i in range(3) for j in range(3))
    At = [[W * W * (Kdn[i][j] - trK * gam[i][j] / 3) for j in range(3)] for i in range(3)]

    def gtu(p, i, j):
        _, gu, dt_, _, _, _ = _ks_parts(p, M, a)
        return dt_ ** (1.0 / 3.0) * gu[i][j]

    Gt = [-sum(_cstep(lambda p, i=i, j=j: gtu(p, i, j), xyz, j) for j in range(3)) for i in range(3)]
    return _pack(W, gt, trK, At, Gt, alpha, beta_up)


def kerr_schild_check(Xm, Ym, Zm, M=1.0, a=0.0):
    """Max |gamma gamma^-1 - I| and |det gamma - (1+2H)|: checks the closed
    forms used above."""
    gam, gamu, det, *_ = _ks_parts([Xm, Ym, Zm], M, a)
    g = np.array(gam)
    gu = np.array(gamu)
    prod = np.einsum("ij...,jk...->ik...", g, gu)
    err_inv = np.max(np.abs(prod - np.eye(3)[:, :, None, None, None]))
    err_det = np.max(np.abs(np.moveaxis(np.linalg.det(np.moveaxis(g, (0, 1), (-2, -1))), 0, 0) - det))
    return err_inv, err_det


# ---------------------------------------------------------------- isotropic Schwarzschild
def isotropic_schwarzschild(Xm, Ym, Zm, M=1.0):
    """Static Schwarzschild in isotropic coordinates: psi = 1 + M/(2r),
    metric psi^4 delta, lapse (1 - M/2r)/(1 + M/2r), zero shift, K_ij = 0."""
    r = np.sqrt(Xm ** 2 + Ym ** 2 + Zm ** 2)
    psi = 1 + M / (2 * r)
    alpha = (1 - M / (2 * r)) / (1 + M / (2 * r))
    one, zero = np.ones_like(r), np.zeros_like(r)
    gt = [[one if i == j else zero for j in range(3)] for i in range(3)]
    At = [[zero] * 3 for _ in range(3)]
    return _pack(psi ** -2, gt, zero, At, [zero] * 3, alpha, [zero] * 3)


# ---------------------------------------------------------------- gauge wave
def _gauge_wave_bssn(x, t, A, d):
    """BSSN variables of the gauge wave as explicit functions of (x, t)
    (complex-safe): H = 1 - A sin(2 pi (x - t)/d), gamma = diag(H, 1, 1),
    alpha = sqrt(H), K_xx = -d_t gamma_xx/(2 alpha), W = H^(-1/6)."""
    th = 2 * np.pi * (x - t) / d
    H = 1 - A * np.sin(th)
    dtH = (2 * np.pi * A / d) * np.cos(th)
    dxH = -dtH
    Kxx = -dtH / (2 * np.sqrt(H))
    W = H ** (-1.0 / 6.0)
    trK = Kxx / H
    gt = [H ** (2.0 / 3.0), H ** (-1.0 / 3.0), H ** (-1.0 / 3.0)]
    At = [W * W * (Kxx - trK * H / 3), W * W * (0 - trK / 3), W * W * (0 - trK / 3)]
    Gt1 = -(-(2.0 / 3.0) * H ** (-5.0 / 3.0) * dxH)  # -d_x gt^xx, gt^xx = H^(-2/3)
    return W, gt, trK, At, Gt1, np.sqrt(H)


def gauge_wave(Xm, t=0.0, A=0.01, d=1.0):
    W, gt, trK, At, Gt1, alpha = _gauge_wave_bssn(Xm, t, A, d)
    zero = np.zeros_like(Xm)
    gtm = [[zero] * 3 for _ in range(3)]
    Atm = [[zero] * 3 for _ in range(3)]
    for i in range(3):
        gtm[i][i] = gt[i]
        Atm[i][i] = At[i]
    return _pack(W, gtm, trK, Atm, [Gt1, zero, zero], alpha, [zero] * 3)


def gauge_wave_dt(Xm, t=0.0, A=0.01, d=1.0):
    """d/dt of the gauge-wave BSSN variables (complex step in t)."""
    tc = t + 1j * CS
    W, gt, trK, At, Gt1, alpha = _gauge_wave_bssn(np.asarray(Xm, dtype=np.complex128), tc, A, d)
    im = lambda a: np.imag(a) / CS
    zero = np.zeros(np.shape(Xm))
    gtm = [[zero] * 3 for _ in range(3)]
    Atm = [[zero] * 3 for _ in range(3)]
    for i in range(3):
        gtm[i][i] = im(gt[i])
        Atm[i][i] = im(At[i])
    return _pack(im(W), gtm, im(trK), Atm, [im(Gt1), zero, zero], im(alpha), [zero] * 3)


# ---------------------------------------------------------------- Kasner
def _kasner_adm(t, p, R):
    D = np.diag([t ** (2 * pi) for pi in p])
    dD = np.diag([2 * pi * t ** (2 * pi - 1) for pi in p])
    gam = R @ D @ R.T
    K = -(R @ dD @ R.T) / 2  # geodesic slicing: K_ij = -d_t gamma_ij / 2
    return gam, K


def _kasner_bssn(t, p, R):
    gam, K = _kasner_adm(t, p, R)
    W = np.linalg.det(gam) ** (-1.0 / 6.0)
    gamu = np.linalg.inv(gam)
    trK = np.sum(gamu * K)
    gt = W * W * gam
    At = W * W * (K - trK * gam / 3)
    v = np.zeros(NVAR, dtype=np.result_type(t, 1.0))
    v[IDX["W"]] = W
    for (i, j) in PAIRS:
        v[IDX["gt11"] + SYM[i][j]] = gt[i, j]
        v[IDX["At11"] + SYM[i][j]] = At[i, j]
    v[IDX["trK"]] = trK
    v[IDX["alpha"]] = 1.0
    return v


def kasner(p_u=1.5, t0=1.3, angles=(0.3, -0.7, 1.1)):
    """Kasner vacuum solution ds^2 = -dt^2 + sum_i t^(2 p_i) dx_i^2 with
    p(u) = (-u, 1+u, u(1+u))/(1+u+u^2) (sum p = sum p^2 = 1), in spatial
    coordinates rotated by a constant rotation (still homogeneous).
    Geodesic slicing: alpha = 1, beta = 0. Returns (u0, du/dt) as 24-vectors
    at t = t0."""
    u = p_u
    den = 1 + u + u * u
    p = [-u / den, (1 + u) / den, u * (1 + u) / den]
    a, b, c = angles
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Ry = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, np.cos(c), -np.sin(c)], [0, np.sin(c), np.cos(c)]])
    R = Rz @ Ry @ Rx
    u0 = _kasner_bssn(t0, p, R).real
    du = np.imag(_kasner_bssn(t0 + 1j * CS, p, R.astype(np.complex128))) / CS
    return u0, du, p


# ---------------------------------------------------------------- momentum data
def momentum_data(Xm, Ym, Zm, amp=0.3, width=0.8, c=(0.2, -0.1, 0.15)):
    """Conformally flat data with K_ij = psi^-2 Ahat_ij, Ahat_ij = d_i d_j f,
    f = x y z + (x^3 - 3 x y^2)/3 (harmonic), so Ahat is traceless and
    divergence free and the momentum constraint holds for any psi (York's
    conformal transverse-traceless construction); psi = 1 + a exp(-r^2/w^2).
    Returns (state, H_exact) with H_exact = -8 psi^-5 lap(psi) -
    psi^-12 Ahat_ij Ahat_ij (the Hamiltonian constraint of this data)."""
    dx, dy, dz = Xm - c[0], Ym - c[1], Zm - c[2]
    r2 = dx * dx + dy * dy + dz * dz
    e = np.exp(-r2 / width ** 2)
    psi = 1 + amp * e
    lap = amp * e * (4 * r2 / width ** 4 - 6 / width ** 2)
    Ahat = [[2 * Xm, Zm - 2 * Ym, Ym], [Zm - 2 * Ym, -2 * Xm, Xm], [Ym, Xm, np.zeros_like(Xm)]]
    one, zero = np.ones_like(Xm), np.zeros_like(Xm)
    gt = [[one if i == j else zero for j in range(3)] for i in range(3)]
    At = [[psi ** -6 * Ahat[i][j] for j in range(3)] for i in range(3)]
    u = _pack(psi ** -2, gt, zero, At, [zero] * 3, one, [zero] * 3)
    AA = sum(Ahat[i][j] ** 2 for i in range(3) for j in range(3))
    Hex = -8 * psi ** -5 * lap - psi ** -12 * AA
    return u, Hex
