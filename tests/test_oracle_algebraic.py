"""Pins for the oracle's algebraic constraints, det(gt_ij) - 1 and
gt^ij At_ij (not GPU). The conformal decomposition of the BSSN variables
(Sec. 1.1) makes both vanish for exact data; the evolution does not enforce
them, so they are diagnostics of its error."""
import numpy as np

import oracle
from paper_1307_6488_gb300 import inputs
from paper_1307_6488_gb300.inputs import IDX


def test_flat_and_brill_lindquist_exact_zero():
    for u, g in ((inputs.flat_space(6, 5, 4, 3), 3), (inputs.brill_lindquist(12, 5)[0], 5)):
        d, t = oracle.algebraic_constraints(u, g)
        assert np.all(d == 0.0) and np.all(t == 0.0)


def test_gauge_wave_conformal_variables():
    """gt = diag(H^(2/3), H^(-1/3), H^(-1/3)) has determinant 1 and
    At = K_xx diag(2/3 H^(-1/3), -1/3 H^(-4/3), -1/3 H^(-4/3)) is trace-free
    in it, for every phase: both to rounding."""
    u, _ = inputs.gauge_wave(16, 3, amplitude=0.2, noise=0.0)
    d, t = oracle.algebraic_constraints(u, 3)
    assert np.max(np.abs(d)) < 1e-14
    assert np.max(np.abs(t)) < 1e-14
    assert np.max(np.abs(u[IDX["At11"]])) > 0.1  # At really is nonzero


def _random_state(seed, n=5, g=2):
    rng = np.random.default_rng(seed)
    u = np.zeros((24, n + 2 * g, n + 2 * g, n + 2 * g))
    M = rng.normal(size=u.shape[1:] + (3, 3))
    G = np.einsum("...ik,...jk->...ij", M, M) + 0.5 * np.eye(3)  # symmetric positive definite
    S = rng.normal(size=u.shape[1:] + (3, 3))
    A = S + np.swapaxes(S, -1, -2)
    for s, (i, j) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        u[1 + s] = G[..., i, j]
        u[8 + s] = A[..., i, j]
    return u, G[g:-g, g:-g, g:-g], A[g:-g, g:-g, g:-g], g


def test_against_library_routines():
    """Generic symmetric matrices: the determinant against numpy's LU-based
    det, the trace against tr(solve(gt, At))."""
    u, G, A, g = _random_state(3)
    d, t = oracle.algebraic_constraints(u, g)
    want_d = np.linalg.det(G) - 1.0
    want_t = np.trace(np.linalg.solve(G, A), axis1=-2, axis2=-1)
    assert np.max(np.abs(d - want_d) / (np.abs(want_d) + 1.0)) < 1e-13
    assert np.max(np.abs(t - want_t) / (np.abs(want_t) + 1.0)) < 1e-11


def test_scaled_identity():
    """gt = s I: det - 1 = s^3 - 1 and the trace is tr(At) / s."""
    u = inputs.flat_space(4, 4, 4, 2)
    s = 1.25
    for q in (0, 3, 5):
        u[1 + q] = s
    u[8:14] = np.arange(1, 7)[:, None, None, None]
    d, t = oracle.algebraic_constraints(u, 2)
    assert np.allclose(d, s ** 3 - 1.0, rtol=0, atol=1e-15)
    assert np.allclose(t, (1 + 4 + 6) / s, rtol=1e-15, atol=0)
