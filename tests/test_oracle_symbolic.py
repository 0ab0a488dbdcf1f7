"""A second, independent transcription of the BSSN right-hand side, fed with
exact derivatives, as a pin for the oracle's finite-difference one (not GPU).

The paper cites the BSSN system (Sec. 1.1) without writing it out. The
exact-solution pins elsewhere (flat space, Kasner, gauge wave, Kerr-Schild,
Schwarzschild, York data) each leave some terms at zero: homogeneous data
has no spatial derivatives, stationary data is tested with its own frozen
gauge. Here every one of the 24 variables is a generic smooth analytic
field (sums of sines with seeded wave vectors and phases, the conformal
metric a perturbation of the identity), so every term of every equation is
alive. Their first and second derivatives are taken exactly by sympy; the
right-hand side is then assembled from those values by a plain numpy
transcription written with full 3x3 tensors and einsum (inverse metric by
numpy.linalg.inv), sharing nothing with the oracle's packed, point-by-point
C++. The oracle's right-hand side at a grid point must converge to it at
the stencil order (4 or 8) as the spacing halves; a wrong sign, index or
dropped term in either transcription leaves an h-independent difference and
stops the convergence. The Hamiltonian, momentum and Gamma constraints and
the electric and magnetic parts of the Weyl tensor are checked the same way.
"""
import numpy as np
import pytest

import oracle

sp = pytest.importorskip("sympy")

NV = 24
W_, GT, K_, AT, GAM, AL, BE, BB = 0, 1, 7, 8, 14, 17, 18, 21
PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
X = sp.symbols("x y z", real=True)


def fields(seed):
    """24 smooth analytic fields: base value + two seeded sine waves each."""
    rng = np.random.default_rng(seed)
    base = np.zeros(NV)
    base[W_] = 1.0
    base[AL] = 1.0
    base[K_] = 0.1
    for s, (i, j) in enumerate(PAIRS):
        base[GT + s] = 1.0 if i == j else 0.0
    amp = np.full(NV, 0.08)
    amp[GT:GT + 6] = 0.05
    exprs = []
    for v in range(NV):
        e = sp.Float(base[v])
        for _ in range(2):
            k = rng.uniform(-1.6, 1.6, 3)
            ph = rng.uniform(0, 2 * np.pi)
            a = amp[v] * rng.uniform(0.5, 1.0)
            e = e + sp.Float(a) * sp.sin(sum(sp.Float(k[d]) * X[d] for d in range(3)) + sp.Float(ph))
        exprs.append(e)
    return exprs


def exact_derivatives(exprs, pt):
    """Values, first and second derivatives of every field at pt."""
    val = np.zeros(NV)
    d1 = np.zeros((NV, 3))
    d2 = np.zeros((NV, 3, 3))
    sub = dict(zip(X, pt))
    for v, e in enumerate(exprs):
        val[v] = float(e.evalf(subs=sub))
        for a in range(3):
            da = sp.diff(e, X[a])
            d1[v, a] = float(da.evalf(subs=sub))
            for b in range(a, 3):
                d2[v, a, b] = d2[v, b, a] = float(sp.diff(da, X[b]).evalf(subs=sub))
    return val, d1, d2


def sym33(vec6):
    m = np.zeros(vec6.shape[1:] + (3, 3)) if vec6.ndim > 1 else np.zeros((3, 3))
    for s, (i, j) in enumerate(PAIRS):
        m[..., i, j] = m[..., j, i] = vec6[s]
    return m


def rhs_transcribed(val, d1, d2, lapse, shift, shift_coeff, eta, advect_gauge):
    """The BSSN right-hand side (W form, vacuum) from exact point values.
    Conventions: dX[k, ...] = d_k X; ddX[k, l, ...] = d_k d_l X."""
    W, K, al = val[W_], val[K_], val[AL]
    gt = sym33(val[GT:GT + 6])
    At = sym33(val[AT:AT + 6])
    beta, B = val[BE:BE + 3], val[BB:BB + 3]
    dW, dK, dal = d1[W_], d1[K_], d1[AL]
    dgt = np.stack([sym33(d1[GT:GT + 6, k]) for k in range(3)])            # [k, i, j]
    ddgt = np.array([[sym33(d2[GT:GT + 6, k, l]) for l in range(3)] for k in range(3)])  # [k, l, i, j]
    dGam = d1[GAM:GAM + 3].T                                                # [k, i] = d_k Gt^i
    dbeta = d1[BE:BE + 3].T                                                 # [k, i] = d_k beta^i
    ddbeta = np.moveaxis(d2[BE:BE + 3], 0, -1)                              # [k, l, i]
    ddW, ddal = d2[W_], d2[AL]
    adv = d1 @ beta                                                         # beta^k d_k u, every variable

    gu = np.linalg.inv(gt)
    Gl = 0.5 * (np.einsum("ikj->kij", dgt) + np.einsum("jki->kij", dgt) - dgt)  # Gt_{k ij}
    Gu = np.einsum("kl,lij->kij", gu, Gl)                                   # Gt^k_ij
    Gd = np.einsum("ij,kij->k", gu, Gu)
    # conformal Ricci tensor
    R = -0.5 * np.einsum("lm,lmij->ij", gu, ddgt)
    R += 0.5 * (np.einsum("ki,jk->ij", gt, dGam) + np.einsum("kj,ik->ij", gt, dGam))
    R += 0.5 * np.einsum("k,ijk->ij", Gd, Gl + np.einsum("jik->ijk", Gl))
    R += np.einsum("lm,kli,jkm->ij", gu, Gu, Gl)
    R += np.einsum("lm,klj,ikm->ij", gu, Gu, Gl)
    R += np.einsum("lm,kim,klj->ij", gu, Gu, Gl)
    # conformal-factor part
    DDW = ddW - np.einsum("kij,k->ij", Gu, dW)
    R += (DDW + gt * np.einsum("kl,kl", gu, DDW)) / W - 2 * gt * np.einsum("kl,k,l", gu, dW, dW) / W ** 2
    # second covariant derivative of the lapse
    DDa = ddal - np.einsum("kij,k->ij", Gu, dal)
    DDa += (np.outer(dW, dal) + np.outer(dal, dW) - gt * np.einsum("kl,k,l", gu, dW, dal)) / W
    D2a = W ** 2 * np.einsum("ij,ij", gu, DDa)
    Am = gu @ At                                                            # At^i_j
    Au = gu @ At @ gu                                                       # At^ij
    divb = np.trace(dbeta)
    out = np.zeros(NV)
    out[W_] = adv[W_] + W * (al * K - divb) / 3
    dgt_t = -2 * al * At + np.einsum("ik,jk->ij", gt, dbeta) + np.einsum("jk,ik->ij", gt, dbeta) - 2 / 3 * gt * divb
    out[K_] = adv[K_] - D2a + al * (np.einsum("ij,ij", At, Au) + K ** 2 / 3)
    X_ = -DDa + al * R
    XTF = X_ - gt * np.einsum("kl,kl", gu, X_) / 3
    dAt_t = (W ** 2 * XTF + al * (K * At - 2 * At @ Am) + np.einsum("ik,jk->ij", At, dbeta)
             + np.einsum("jk,ik->ij", At, dbeta) - 2 / 3 * At * divb)
    for s, (i, j) in enumerate(PAIRS):
        out[GT + s] = adv[GT + s] + dgt_t[i, j]
        out[AT + s] = adv[AT + s] + dAt_t[i, j]
    gam_na = (-np.einsum("j,ji->i", Gd, dbeta) + 2 / 3 * Gd * divb + np.einsum("jk,jki->i", gu, ddbeta)
              + gu @ np.einsum("jkk->j", ddbeta) / 3 - 2 * Au @ dal
              + 2 * al * (np.einsum("ijk,jk->i", Gu, Au) - 3 / W * Au @ dW - 2 / 3 * gu @ dK))
    out[GAM:GAM + 3] = adv[GAM:GAM + 3] + gam_na
    ag = 1.0 if advect_gauge else 0.0
    if lapse == 0:
        out[AL] = ag * adv[AL] - 2 * al * K
    elif lapse == 1:
        out[AL] = ag * adv[AL] - al * al * K
    if shift == 0:
        out[BE:BE + 3] = ag * adv[BE:BE + 3] + shift_coeff * B
        out[BB:BB + 3] = ag * adv[BB:BB + 3] + gam_na - eta * B
    return out


def constraints_transcribed(val, d1, d2):
    """Hamiltonian, momentum and Gamma constraints from exact point values:
    H = R + 2/3 K^2 - At_ij At^ij with R = W^2 gt^ij R_ij,
    M_i = gt^jk (d_k At_ij - Gt^l_ki At_lj - Gt^l_kj At_il) - 3/W At^j_i d_j W - 2/3 d_i K,
    G^i = Gt^i - gt^jk Gt^i_jk."""
    W, K = val[W_], val[K_]
    gt = sym33(val[GT:GT + 6])
    At = sym33(val[AT:AT + 6])
    dW, dK = d1[W_], d1[K_]
    dgt = np.stack([sym33(d1[GT:GT + 6, k]) for k in range(3)])
    ddgt = np.array([[sym33(d2[GT:GT + 6, k, l]) for l in range(3)] for k in range(3)])
    dAt = np.stack([sym33(d1[AT:AT + 6, k]) for k in range(3)])             # [k, i, j] = d_k At_ij
    dGam = d1[GAM:GAM + 3].T
    ddW = d2[W_]
    gu = np.linalg.inv(gt)
    Gl = 0.5 * (np.einsum("ikj->kij", dgt) + np.einsum("jki->kij", dgt) - dgt)
    Gu = np.einsum("kl,lij->kij", gu, Gl)
    Gd = np.einsum("ij,kij->k", gu, Gu)
    R = -0.5 * np.einsum("lm,lmij->ij", gu, ddgt)
    R += 0.5 * (np.einsum("ki,jk->ij", gt, dGam) + np.einsum("kj,ik->ij", gt, dGam))
    R += 0.5 * np.einsum("k,ijk->ij", Gd, Gl + np.einsum("jik->ijk", Gl))
    R += np.einsum("lm,kli,jkm->ij", gu, Gu, Gl)
    R += np.einsum("lm,klj,ikm->ij", gu, Gu, Gl)
    R += np.einsum("lm,kim,klj->ij", gu, Gu, Gl)
    DDW = ddW - np.einsum("kij,k->ij", Gu, dW)
    R += (DDW + gt * np.einsum("kl,kl", gu, DDW)) / W - 2 * gt * np.einsum("kl,k,l", gu, dW, dW) / W ** 2
    Au = gu @ At @ gu
    H = W ** 2 * np.einsum("ij,ij", gu, R) + 2 / 3 * K ** 2 - np.einsum("ij,ij", At, Au)
    DAt = np.einsum("kij->ijk", dAt) - np.einsum("lki,lj->ijk", Gu, At) - np.einsum("lkj,il->ijk", Gu, At)  # [i,j,k]
    Amix = np.einsum("jk,ik->ij", gu, At)                                   # [i, j] = At^j_i
    M = np.einsum("jk,ijk->i", gu, DAt) - 3 / W * Amix @ dW - 2 / 3 * dK
    G = val[GAM:GAM + 3] - Gd
    return np.concatenate([[H], M, G])


def weyl_transcribed(val, d1, d2):
    """Electric and magnetic parts of the Weyl tensor from exact point values,
    with the physical metric's own Christoffel symbols (not the conformal
    split): gamma = gt / W^2, K_ij = (At_ij + gt_ij K / 3) / W^2,
    E_ij = R_ij + K K_ij - K_ik K^k_j (K the evolved trace variable),
    B_ij = 1/2 (eps_i^kl D_k K_lj + eps_j^kl D_k K_li), eps^mkl = [mkl] / sqrt(det gamma).
    Returns E and B packed (11 12 13 22 23 33)."""
    W, K = val[W_], val[K_]
    gt = sym33(val[GT:GT + 6])
    At = sym33(val[AT:AT + 6])
    dW, dK = d1[W_], d1[K_]
    dgt = np.stack([sym33(d1[GT:GT + 6, k]) for k in range(3)])
    dAt = np.stack([sym33(d1[AT:AT + 6, k]) for k in range(3)])
    R = _physical_ricci(val, d1, d2)  # through the conformal decomposition
    gam = gt / W ** 2
    Kd = (At + gt * K / 3) / W ** 2
    dgam = dgt / W ** 2 - 2 * gt[None] * dW[:, None, None] / W ** 3
    dKd = ((dAt + dgt * K / 3 + gt[None] * dK[:, None, None] / 3) / W ** 2
           - 2 * (At + gt * K / 3)[None] * dW[:, None, None] / W ** 3)
    gamu = np.linalg.inv(gam)
    chr_ = 0.5 * np.einsum("pq,kql->pkl", gamu, dgam) + 0.5 * np.einsum("pq,lqk->pkl", gamu, dgam) \
        - 0.5 * np.einsum("pq,qkl->pkl", gamu, dgam)                         # Gamma^p_kl
    DK = dKd - np.einsum("pkl,pj->klj", chr_, Kd) - np.einsum("pkj,lp->klj", chr_, Kd)  # [k, l, j]
    E = R + K * Kd - Kd @ gamu @ Kd
    lc = np.zeros((3, 3, 3))
    for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        lc[a, b, c] = 1.0
        lc[a, c, b] = -1.0
    eps_u = lc / np.sqrt(np.linalg.det(gam))                                  # eps^mkl
    eps_m = np.einsum("im,mkl->ikl", gam, eps_u)                              # eps_i^kl
    X = np.einsum("ikl,klj->ij", eps_m, DK)
    Bm = 0.5 * (X + X.T)
    pack = lambda M: np.array([M[i, j] for (i, j) in PAIRS])
    return pack(E), pack(Bm)


def _physical_ricci(val, d1, d2):
    """R_ij of gamma = gt / W^2 through the conformal decomposition
    (conformal Ricci with the evolved Gt^i in its derivative term, plus the
    conformal-factor part), as the right-hand side uses it."""
    W = val[W_]
    gt = sym33(val[GT:GT + 6])
    dW = d1[W_]
    dgt = np.stack([sym33(d1[GT:GT + 6, k]) for k in range(3)])
    ddgt = np.array([[sym33(d2[GT:GT + 6, k, l]) for l in range(3)] for k in range(3)])
    dGam = d1[GAM:GAM + 3].T
    ddW = d2[W_]
    gu = np.linalg.inv(gt)
    Gl = 0.5 * (np.einsum("ikj->kij", dgt) + np.einsum("jki->kij", dgt) - dgt)
    Gu = np.einsum("kl,lij->kij", gu, Gl)
    Gd = np.einsum("ij,kij->k", gu, Gu)
    R = -0.5 * np.einsum("lm,lmij->ij", gu, ddgt)
    R += 0.5 * (np.einsum("ki,jk->ij", gt, dGam) + np.einsum("kj,ik->ij", gt, dGam))
    R += 0.5 * np.einsum("k,ijk->ij", Gd, Gl + np.einsum("jik->ijk", Gl))
    R += np.einsum("lm,kli,jkm->ij", gu, Gu, Gl)
    R += np.einsum("lm,klj,ikm->ij", gu, Gu, Gl)
    R += np.einsum("lm,kim,klj->ij", gu, Gu, Gl)
    DDW = ddW - np.einsum("kij,k->ij", Gu, dW)
    R += (DDW + gt * np.einsum("kl,kl", gu, DDW)) / W - 2 * gt * np.einsum("kl,k,l", gu, dW, dW) / W ** 2
    return R


def oracle_weyl_at(exprs, pt, h, order):
    g = oracle.required_ghost(order)
    off = (np.arange(2 * g + 1) - g) * h
    zz, yy, xx = np.meshgrid(pt[2] + off, pt[1] + off, pt[0] + off, indexing="ij")
    u = np.zeros((NV,) + xx.shape)
    for v, e in enumerate(exprs):
        u[v] = np.broadcast_to(sp.lambdify(X, e, "numpy")(xx, yy, zz), xx.shape)
    out = oracle.psi4(np.ascontiguousarray(u), g, h, order, pt)  # the one interior point is pt
    return out["E"][:, g, g, g], out["B"][:, g, g, g]


def oracle_at(exprs, pt, h, order, p):
    """The oracle's right-hand side at pt: one interior point, its ghosts
    filled with the exact fields."""
    g = oracle.required_ghost(order)
    off = (np.arange(2 * g + 1) - g) * h
    zz, yy, xx = np.meshgrid(pt[2] + off, pt[1] + off, pt[0] + off, indexing="ij")
    u = np.zeros((NV,) + xx.shape)
    for v, e in enumerate(exprs):
        f = sp.lambdify(X, e, "numpy")
        u[v] = np.broadcast_to(f(xx, yy, zz), xx.shape)
    u = np.ascontiguousarray(u)
    if p is None:
        _, _, _, (ham, mom, gcon) = oracle.constraints(u, g, h, order, fields=True)
        return np.concatenate([[ham[g, g, g]], mom[:, g, g, g], gcon[:, g, g, g]])
    return oracle.rhs(u, g, h, p)[:, g, g, g]


GAUGES = [dict(lapse=0, shift=0, advect_gauge=1), dict(lapse=1, shift=0, advect_gauge=0)]


@pytest.mark.parametrize("order,hs", [(4, (0.08, 0.04, 0.02)), (8, (0.3, 0.15, 0.075))])
@pytest.mark.parametrize("gauge", GAUGES)
@pytest.mark.parametrize("seed", [11, 29])
def test_rhs_converges_to_second_transcription(order, hs, gauge, seed):
    exprs = fields(seed)
    pt = np.random.default_rng(seed + 1).uniform(-1, 1, 3)
    pars = dict(shift_coeff=0.75, eta=1.7, **gauge)
    val, d1, d2 = exact_derivatives(exprs, pt)
    want = rhs_transcribed(val, d1, d2, **pars)
    p = oracle.Params(fd_order=order, ko_eps=0.0, **pars)
    scale = np.max(np.abs(want))
    errs = [np.max(np.abs(oracle_at(exprs, pt, h, order, p) - want)) / scale for h in hs]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # every variable is alive: a dropped term would show at O(1)
    assert np.min(np.abs(want)) > 1e-4 * scale
    assert errs[-1] < (1e-5 if order == 4 else 1e-7), errs
    assert order - 0.6 < rates[-1] < order + 1.5, (errs, rates)


@pytest.mark.parametrize("order,hs", [(4, (0.08, 0.04, 0.02)), (8, (0.3, 0.15, 0.075))])
@pytest.mark.parametrize("seed", [11, 29])
def test_constraints_converge_to_second_transcription(order, hs, seed):
    """The same for the Hamiltonian, momentum and Gamma constraints."""
    exprs = fields(seed)
    pt = np.random.default_rng(seed + 2).uniform(-1, 1, 3)
    val, d1, d2 = exact_derivatives(exprs, pt)
    want = constraints_transcribed(val, d1, d2)
    scale = np.max(np.abs(want))
    errs = [np.max(np.abs(oracle_at(exprs, pt, h, order, None) - want)) / scale for h in hs]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.min(np.abs(want)) > 1e-4 * scale
    assert errs[-1] < (1e-5 if order == 4 else 1e-7), errs
    assert order - 0.6 < rates[-1] < order + 1.5, (errs, rates)


@pytest.mark.parametrize("order,hs", [(4, (0.08, 0.04, 0.02)), (8, (0.3, 0.15, 0.075))])
def test_weyl_parts_converge_to_second_transcription(order, hs):
    """E_ij and B_ij of the Weyl diagnostics (the inputs of Psi_4), against a
    transcription that takes the physical metric's Christoffels directly."""
    exprs = fields(11)
    pt = np.array([0.37, -0.21, 0.44])
    val, d1, d2 = exact_derivatives(exprs, pt)
    wE, wB = weyl_transcribed(val, d1, d2)
    for name, want, k in (("E", wE, 0), ("B", wB, 1)):
        scale = np.max(np.abs(want))
        errs = [np.max(np.abs(oracle_weyl_at(exprs, pt, h, order)[k] - want)) / scale for h in hs]
        rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert errs[-1] < (1e-5 if order == 4 else 1e-7), (name, errs)
        assert order - 0.6 < rates[-1] < order + 1.5, (name, errs, rates)


def test_psi4_from_transcribed_weyl_parts():
    """Psi_4 and the invariant I assembled from the transcribed E and B at
    the point: the gamma-orthonormal triad by Gram-Schmidt of the radial,
    theta and phi coordinate directions about the coordinate origin,
    m = (e_theta + i e_phi) / sqrt(2), Psi_4 = (E - i B)_ij mbar^i mbar^j,
    I = (E - i B)_ij (E - i B)^ij / 2. The oracle's values converge to them
    at the stencil order."""
    exprs = fields(29)
    pt = np.array([0.61, -0.48, 0.33])
    val, d1, d2 = exact_derivatives(exprs, pt)
    wE, wB = weyl_transcribed(val, d1, d2)
    Q = sym33(wE) - 1j * sym33(wB)
    gam = sym33(val[GT:GT + 6]) / val[W_] ** 2
    dot = lambda a, b: a @ gam @ b
    x, y, z = pt
    basis = [np.array([x, y, z]), np.array([x * z, y * z, -(x * x + y * y)]), np.array([-y, x, 0.0])]
    tri = []
    for v in basis:
        for e in tri:
            v = v - dot(v, e) * e
        tri.append(v / np.sqrt(dot(v, v)))
    m = (tri[1] + 1j * tri[2]) / np.sqrt(2)
    want_psi4 = np.einsum("ij,i,j", Q, np.conj(m), np.conj(m))
    gamu = np.linalg.inv(gam)
    want_inv = 0.5 * np.einsum("ij,ik,jl,kl", Q, gamu, gamu, Q)
    errs = []
    for h in (0.3, 0.15, 0.075):
        g = oracle.required_ghost(8)
        off = (np.arange(2 * g + 1) - g) * h
        zz, yy, xx = np.meshgrid(pt[2] + off, pt[1] + off, pt[0] + off, indexing="ij")
        u = np.zeros((NV,) + xx.shape)
        for v, e in enumerate(exprs):
            u[v] = np.broadcast_to(sp.lambdify(X, e, "numpy")(xx, yy, zz), xx.shape)
        out = oracle.psi4(np.ascontiguousarray(u), g, h, 8, pt)
        errs.append(max(abs(out["psi4"][g, g, g] - want_psi4) / abs(want_psi4),
                        abs(out["inv"][g, g, g] - want_inv) / abs(want_inv)))
    rate = np.log2(errs[1] / errs[2])
    assert errs[-1] < 1e-7 and 7.4 < rate < 9.5, (errs, rate)


def test_transcription_sees_each_term():
    """The comparison is sensitive: perturbing the oracle's input by a
    planted mistake of the size of one term (the sign of the shift's
    B-coupling, eta) moves the right-hand side far outside the FD error."""
    exprs = fields(11)
    pt = np.array([0.3, -0.2, 0.5])
    val, d1, d2 = exact_derivatives(exprs, pt)
    good = rhs_transcribed(val, d1, d2, 0, 0, 0.75, 1.7, 1)
    bad = rhs_transcribed(val, d1, d2, 0, 0, 0.75, -1.7, 1)
    p = oracle.Params(fd_order=8, ko_eps=0.0, lapse=0, shift=0, shift_coeff=0.75, eta=1.7, advect_gauge=1)
    got = oracle_at(exprs, pt, 0.05, 8, p)
    scale = np.max(np.abs(good))
    assert np.max(np.abs(got - good)) / scale < 1e-7
    assert np.max(np.abs(got - bad)) / scale > 1e-3
