"""FP32-RHS form: derivatives, right-hand side and dissipation in single
precision on the double-precision state, 1/W and the RK4 update in double
precision. Its error against the FP64 oracle is stated and bounded here.

Single precision represents the state to 6e-8 relative; a second
difference of it over L/h points carries ~ 6e-8 * 4 (L/h)^2 relative error,
so on the smooth data below (L/h ~ 16) the bound is ~1e-4 per tensor field.
Data with 1e-10 noise on O(1) fields (the 24^3 gauge wave) is below single
precision resolution and is a double-precision-only case."""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs

from gpu_common import TENSORS, grid_for, interior, need_gpu, oracle_params, perturbed_bl, rel_err_tensor

pytestmark = pytest.mark.gpu

FP32_RHS_TOL = 3e-4
FP32_STEP_TOL = 1e-3


@pytest.mark.parametrize("order", [4, 8])
def test_fp32_flat_space_exact_zero(order):
    torch = need_gpu()
    g = order // 2 + 1
    u = inputs.flat_space(9, 8, 7, g)
    p = B.make_params(fd_order=order)
    grid = grid_for(u, g, 0.1)
    d = B.upload(u, grid)
    out = B.alloc_state(grid)
    work = B.alloc_work(grid, p, B.FP32_RHS)
    B.rhs(grid, p, B.FP32_RHS, d, out, work)
    B.ko_dissipation(grid, p, B.FP32_RHS, d, out)
    torch.cuda.synchronize()
    assert np.all(interior(B.download(out, grid), g) == 0.0)


def smooth_bl(nx, ny, nz, g, h, seed):
    """Brill-Lindquist-like data (off-grid punctures, kept away from the box)
    plus a seeded smooth perturbation: every variable nonzero and smooth."""
    return perturbed_bl(nx, ny, nz, g, h, seed=seed, amp=1e-2)


@pytest.mark.parametrize("order", [4, 8])
def test_fp32_rhs_vs_oracle(order):
    torch = need_gpu()
    g = order // 2 + 1
    h = 0.12
    u = smooth_bl(17, 13, 11, g, h, seed=40 + order)
    p = B.make_params(fd_order=order)
    grid = grid_for(u, g, h)
    d = B.upload(u, grid)
    work = B.alloc_work(grid, p, B.FP32_RHS)
    for ko in (False, True):
        out = B.alloc_state(grid)
        B.rhs(grid, p, B.FP32_RHS, d, out, work)
        if ko:
            B.ko_dissipation(grid, p, B.FP32_RHS, d, out)
        torch.cuda.synchronize()
        want = oracle.rhs(u, g, h, oracle_params(p), ko=ko)
        err = rel_err_tensor(B.download(out, grid), want, g)
        assert np.max(err) < FP32_RHS_TOL, dict(zip(inputs.VARS, err))
        assert np.max(err) > 1e-9  # it really is single precision


@pytest.mark.parametrize("order", [4, 8])
def test_fp32_steps_vs_oracle(order):
    """Three RK4 steps with static ghosts: change of the state against the
    oracle's change, per tensor field."""
    torch = need_gpu()
    g = order // 2 + 1
    h = 0.15
    u = smooth_bl(14, 12, 10, g, h, seed=60 + order)
    p = B.make_params(fd_order=order)
    grid = grid_for(u, g, h)
    state = B.upload(u, grid)
    src = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p, B.FP32_RHS)
    want = u.copy()
    dt = 0.25 * h
    for _ in range(3):
        B.rk4_step(grid, p, B.FP32_RHS, dt, 1, src, state, bufs, work)
        want = oracle.rk4_step(want, g, h, dt, oracle_params(p), bc=1, ghost_src=u)
    torch.cuda.synchronize()
    got = B.download(state, grid)
    err = rel_err_tensor(got - u, want - u, g)
    assert np.max(err) < FP32_STEP_TOL, dict(zip(inputs.VARS, err))


# alpha, beta^i, B^i
_LAPSE = [17]
_SHIFT = list(range(18, 24))


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("gauge", [dict(lapse=0, shift=0, advect_gauge=1), dict(lapse=1, shift=0, advect_gauge=0),
                                   dict(lapse=2, shift=1, advect_gauge=1), dict(lapse=0, shift=1, advect_gauge=0)])
def test_fp32_gauge_switches(order, gauge):
    """The FP32 form carries each variable's advection beside its dissipation
    and weights it as the gauge's right-hand side takes it: advected lapse
    and shift only with advect_gauge, nothing for a frozen lapse or shift.
    Each gauge choice against the oracle: the right-hand side alone (frozen
    variables exactly zero) and the fused stage with dissipation (frozen
    variables: the dissipation alone, against the operator's norm bound)."""
    torch = need_gpu()
    g = order // 2 + 1
    h = 0.12
    u = smooth_bl(15, 12, 10, g, h, seed=80 + order + 5 * gauge["lapse"] + gauge["advect_gauge"])
    eps = 0.07
    p = B.make_params(fd_order=order, ko_eps=eps, eta=1.7, shift_coeff=0.7, **gauge)
    frozen = (_LAPSE if gauge["lapse"] == 2 else []) + (_SHIFT if gauge["shift"] == 1 else [])
    live = [v for v in range(24) if v not in frozen]
    grid = grid_for(u, g, h)
    d = B.upload(u, grid)
    work = B.alloc_work(grid, p, B.FP32_RHS)
    out = B.alloc_state(grid)
    B.rhs(grid, p, B.FP32_RHS, d, out, work)
    acc = B.alloc_state(grid)
    ynext = B.alloc_state(grid)
    dt = 0.25 * h
    B.rk4_stage(grid, p, B.FP32_RHS, 0, dt, d, d, acc, ynext, work)
    torch.cuda.synchronize()

    got = B.download(out, grid)
    want = oracle.rhs(u, g, h, oracle_params(p), ko=False)
    err = rel_err_tensor(got, want, g)
    assert np.max(err[live]) < FP32_RHS_TOL, dict(zip(inputs.VARS, err))
    for v in frozen:
        assert np.all(interior(got, g)[v] == 0.0), inputs.VARS[v]

    k = B.download(acc, grid) / (dt / 6)
    want_k = oracle.rhs(u, g, h, oracle_params(p), ko=True)
    err = rel_err_tensor(k, want_k, g)
    assert np.max(err[live]) < FP32_RHS_TOL, dict(zip(inputs.VARS, err))
    if frozen:
        scale = eps * 3 / h * np.max(np.abs(u[frozen].reshape(len(frozen), -1)), axis=1)
        gi = interior(k, g)[frozen].reshape(len(frozen), -1)
        wi = interior(want_k, g)[frozen].reshape(len(frozen), -1)
        assert np.max(np.abs(wi), axis=1).min() > 0  # the dissipation is really there
        assert np.max(np.max(np.abs(gi - wi), axis=1) / scale) < 1e-5


@pytest.mark.parametrize("order,bc", [(8, 1), (4, 0)])
@pytest.mark.parametrize("method", [4, 3])
def test_fp32_whole_step_equals_its_stages(order, bc, method):
    """bssn_rk4_step and bssn_rk3_step convert the state to single precision
    once per step: each stage writes the single-precision copy of its output
    beside it and the ghost fill completes it. Two steps must equal, bit for
    bit, the stages called one at a time (ghost fill, then the stage with its
    own fresh conversion), static and periodic ghosts."""
    torch = need_gpu()
    g = order // 2 + 1
    h = 0.12
    u = smooth_bl(14, 11, 9, g, h, seed=70 + order + method)
    p = B.make_params(fd_order=order)
    grid = grid_for(u, g, h)
    src = B.upload(u, grid)
    a = src.clone()
    b = src.clone()
    work = B.alloc_work(grid, p, B.FP32_RHS)
    bufs = B.alloc_state(grid, n=3)
    mine = B.alloc_state(grid, n=3)
    n = 24 * grid.var_stride
    ya, yb, acc = mine[:n], mine[n:2 * n], mine[2 * n:]
    dt = 0.25 * h
    gsrc = src if bc == 1 else None
    for _ in range(2):
        if method == 4:
            B.rk4_step(grid, p, B.FP32_RHS, dt, bc, gsrc, a, bufs, work)
            ys, outs = b, [ya, yb, ya, b]
            for st in range(4):
                B.fill_ghosts(grid, bc, gsrc, ys)
                B.rk4_stage(grid, p, B.FP32_RHS, st, dt, b, ys, acc, outs[st], work)
                ys = outs[st]
        else:
            B.rk3_step(grid, p, B.FP32_RHS, dt, bc, gsrc, a, bufs, work)
            ys, outs = b, [ya, yb, b]
            for st in range(3):
                B.fill_ghosts(grid, bc, gsrc, ys)
                B.rk3_stage(grid, p, B.FP32_RHS, st, dt, b, ys, outs[st], work)
                ys = outs[st]
        B.fill_ghosts(grid, bc, gsrc, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b), float(torch.max(torch.abs(a - b)))
    assert not torch.equal(a, src)


def test_fp32_stage_split_matches_fused_call():
    """bssn_diff_tables + bssn_rk4_stage_fused == bssn_rk4_stage, both forms."""
    torch = need_gpu()
    g = 5
    u = smooth_bl(12, 12, 12, g, 0.1, seed=77)
    inputs.periodic_wrap(u, g)
    p = B.make_params(fd_order=8)
    grid = grid_for(u, g, 0.1)
    y0 = B.upload(u, grid)
    for prec in (B.FP64, B.FP32_RHS):
        work = B.alloc_work(grid, p, prec)
        a1, n1 = B.alloc_state(grid), B.alloc_state(grid)
        a2, n2 = B.alloc_state(grid), B.alloc_state(grid)
        B.rk4_stage(grid, p, prec, 0, 0.02, y0, y0, a1, n1, work)
        B.diff_tables(grid, p, prec, y0, work)
        B.rk4_stage_fused(grid, p, prec, 0, 0.02, y0, y0, a2, n2, work)
        torch.cuda.synchronize()
        assert torch.equal(n1, n2) and torch.equal(a1, a2)


@pytest.mark.slow
@pytest.mark.parametrize("n,prec", [(128, B.FP32_RHS), (256, B.FP32_RHS), (256, B.FP64)])
def test_full_size_sampled(n, prec):
    """The throughput grids of the precision comparison - 128^3 and 256^3
    Brill-Lindquist (bare masses 0.5 at x = +-1.5) with the 8th-order stencil
    and 5 ghosts, plus a seeded 1e-3 perturbation - one fused RK4 stage 0 in
    the benchmark's launch configuration, checked at 4096 sampled points
    against the oracle's right-hand side: FP64 per variable at 1e-12; the
    FP32-RHS form per tensor field at 2e-3. That bound is wider than the
    3e-4 of the smooth-data tests above because at t = 0 the right-hand
    sides of trK and At_ij are small (the Laplacian and trace-free Hessian
    of a nearly flat lapse) next to the single-precision rounding of O(1)
    fields differenced twice, which is absolute, ~eps32/h^2: relative to
    those small tensors it reaches ~1e-3 (measured 8.8e-4 at 128^3, for
    trK at a point with W = 0.91, far from the punctures; 5.8e-4 at 256^3).
    test_full_size_error_is_rounding_of_second_differences checks that
    reading against an absolute bound."""
    torch = need_gpu()
    g = 5
    u, h = inputs.brill_lindquist(n, g, lo=-8.0, hi=8.0)
    inputs.smooth_perturbation(u, g, 1e-3, 4243 + n, h)
    p = B.make_params(fd_order=8)
    grid = grid_for(u, g, h)
    y0 = B.upload(u, grid)
    acc = B.alloc_state(grid)
    ynext = B.alloc_state(grid)
    work = B.alloc_work(grid, p, prec)
    dt = 0.25 * h
    B.rk4_stage(grid, p, prec, 0, dt, y0, y0, acc, ynext, work)
    torch.cuda.synchronize()
    del ynext, work
    rng = np.random.default_rng(n + prec)
    lin = np.unique(rng.integers(0, n ** 3, 4096))
    k = oracle.rhs_points(u, g, h, oracle_params(p), lin, ko=True)  # (npts, 24)
    gi = interior(B.download(acc, grid), g).reshape(24, -1)[:, lin].T
    want = dt / 6 * k
    if prec == B.FP64:
        scale = np.max(np.abs(want), axis=0) + 1e-300
        err = np.max(np.abs(gi - want), axis=0) / scale
        assert np.max(err) < 1e-12, dict(zip(inputs.VARS, err))
    else:
        mag = np.max(np.abs(want), axis=0)
        scale = np.zeros_like(mag)
        for grp in TENSORS:
            scale[grp] = np.max(mag[grp])
        err = np.max(np.abs(gi - want), axis=0) / np.maximum(scale, 1e-300)
        worst = sorted(zip(err, inputs.VARS), reverse=True)[:6]
        assert np.max(err) < 2e-3, worst


@pytest.mark.slow
def test_full_size_error_is_rounding_of_second_differences():
    """The reading behind the 2e-3 bound of test_full_size_sampled, made
    checkable. A second difference of an O(1) field whose values are rounded
    to single precision, formed with single-precision sums, carries an
    absolute error of about eps32 * (sum of |weights| ~ 6.5) / h^2 per axis
    (the input rounding and that of the paired sums, each of that size);
    over three axes and the few O(1) factors of the algebra this stays below
    64 eps32 / h^2. That is an absolute bound on every right-hand side
    (times dt/6, its weight in the stage-0 accumulator). Relative to a
    tensor's largest right-hand side it is large only where that right-hand
    side is small: at t = 0 (K = 0, At = 0) those of trK and At_ij are the
    Laplacian and trace-free Hessian of a nearly flat lapse, ~1e-4..4e-4 of
    dt/6 at 128^3, so the relative error there reaches ~1e-3 far from the
    punctures. The oracle's right-hand side of the state rounded to single
    precision sits about halfway (the input rounding is half of it)."""
    torch = need_gpu()
    n, g = 128, 5
    u, h = inputs.brill_lindquist(n, g, lo=-8.0, hi=8.0)
    inputs.smooth_perturbation(u, g, 1e-3, 4243 + n, h)
    assert np.max(np.abs(u)) < 1.5  # O(1) fields: the bound below is in these units
    p = B.make_params(fd_order=8)
    grid = grid_for(u, g, h)
    y0 = B.upload(u, grid)
    acc = B.alloc_state(grid)
    ynext = B.alloc_state(grid)
    work = B.alloc_work(grid, p, B.FP32_RHS)
    dt = 0.25 * h
    B.rk4_stage(grid, p, B.FP32_RHS, 0, dt, y0, y0, acc, ynext, work)
    torch.cuda.synchronize()
    del ynext, work
    rng = np.random.default_rng(n + B.FP32_RHS)
    lin = np.unique(rng.integers(0, n ** 3, 4096))
    gi = interior(B.download(acc, grid), g).reshape(24, -1)[:, lin].T
    eps32 = 2.0 ** -24
    bound = dt / 6 * 64 * eps32 / h ** 2
    errs = []
    for state in (u, u.astype(np.float32).astype(np.float64)):
        want = dt / 6 * oracle.rhs_points(state, g, h, oracle_params(p), lin, ko=True)
        errs.append(np.max(np.abs(gi - want), axis=0))  # per variable
    exact, rounded = errs
    assert np.all(exact < bound), dict(zip(inputs.VARS, exact / bound))
    k = inputs.VARS.index("trK")
    assert rounded[k] < 0.8 * exact[k], (exact[k], rounded[k])
