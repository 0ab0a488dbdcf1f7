"""The learned corrector's glue through the C ABI: packing of training pairs
(normalisation and BF16 rounding, bit-exact against host arithmetic), the
applied correction (bit-exact against the raw forward pass, which
test_gpu_corrector.py checks against the oracle), the fallback to the fine
method, and the accuracy gain of a trained corrector over the plain coarse
method on held-out Brill-Lindquist data."""
import numpy as np
import pytest

from paper_1307_6488_gb300 import binding as B

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

N = 32
G = 4


def bf16_bits(torch, a):
    """float64 array -> float32 (round to nearest) -> BF16 (round to nearest
    even) bit patterns."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).view(torch.int16).numpy()


def interior_points(u):
    return u[:, G:-G, G:-G, G:-G].reshape(24, -1).T


@pytest.fixture(scope="module")
def setup():
    torch = need_gpu()
    rng = np.random.default_rng(11)
    grid = B.make_grid(N, ghost=G, dx=0.1)
    u = rng.standard_normal((24, N + 2 * G, N + 2 * G, N + 2 * G))
    tgt = u + 0.01 * rng.standard_normal(u.shape)
    off = rng.standard_normal(24)
    isc = rng.uniform(0.5, 2.0, 24)
    osc = rng.uniform(10.0, 100.0, 24)
    c = B.corrector_create(N, 1, seed=3)
    B.corrector_set_scales(c, off, isc, osc)
    yield torch, grid, u, tgt, off, isc, osc, c
    B.corrector_destroy(c)


def test_pack_normalises_and_rounds(setup):
    torch, grid, u, tgt, off, isc, osc, c = setup
    xb = torch.empty((N ** 3, 32), dtype=torch.bfloat16, device="cuda")
    tb = torch.empty_like(xb)
    B.corrector_pack(c, grid, B.upload(u, grid), B.upload(tgt, grid), xb, tb)
    torch.cuda.synchronize()
    I, T = interior_points(u), interior_points(tgt)
    x = xb.cpu().view(torch.int16).numpy()
    t = tb.cpu().view(torch.int16).numpy()
    np.testing.assert_array_equal(x[:, :24], bf16_bits(torch, (I - off) * isc))
    np.testing.assert_array_equal(t[:, :24], bf16_bits(torch, (T - I) * osc))
    assert not x[:, 24:].any() and not t[:, 24:].any()


def test_apply_adds_unscaled_network_output(setup):
    torch, grid, u, tgt, off, isc, osc, c = setup
    xb = torch.empty((N ** 3, 32), dtype=torch.bfloat16, device="cuda")
    tb = torch.empty_like(xb)
    state = B.upload(u, grid)
    B.corrector_pack(c, grid, state, state, xb, tb)
    out = torch.empty((N ** 3, 32), dtype=torch.float32, device="cuda")
    B.corrector_forward_raw(c, 1, xb, out)
    B.corrector_apply(c, grid, state)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    assert np.abs(o[:, :24]).max() > 0
    want = u.copy()
    want[:, G:-G, G:-G, G:-G] += (o[:, :24] / osc).T.reshape(24, N, N, N)
    got = B.download(state, grid)
    np.testing.assert_array_equal(got, want)


def test_step_scale_divides_targets_and_multiplies_corrections(setup):
    torch, grid, u, tgt, off, isc, osc, c = setup
    sc = np.random.default_rng(5).uniform(0.25, 4.0, 24)
    B.corrector_set_step_scale(c, sc)
    try:
        xb = torch.empty((N ** 3, 32), dtype=torch.bfloat16, device="cuda")
        tb = torch.empty_like(xb)
        state = B.upload(u, grid)
        B.corrector_pack(c, grid, state, B.upload(tgt, grid), xb, tb)
        I, T = interior_points(u), interior_points(tgt)
        t = tb.cpu().view(torch.int16).numpy()
        np.testing.assert_array_equal(t[:, :24], bf16_bits(torch, (T - I) * osc / sc))
        out = torch.empty((N ** 3, 32), dtype=torch.float32, device="cuda")
        B.corrector_forward_raw(c, 1, xb, out)
        B.corrector_apply(c, grid, state)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        want = u.copy()
        want[:, G:-G, G:-G, G:-G] += (o[:, :24] * sc / osc).T.reshape(24, N, N, N)
        np.testing.assert_array_equal(B.download(state, grid), want)
        with pytest.raises(B.BssnError):
            B.corrector_set_step_scale(c, np.where(np.arange(24) == 3, 0.0, 1.0))
    finally:
        B.corrector_set_step_scale(c, np.ones(24))


def test_rms_diff_and_roughness(setup):
    torch, grid, u, tgt, off, isc, osc, c = setup
    from paper_1307_6488_gb300 import learned as LR
    params = B.make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    work = B.alloc_work(grid, params, B.FP64)
    a, b = B.upload(u, grid), B.upload(tgt, grid)
    got = B.rms_diff(grid, a, b, work)
    want = np.sqrt(((interior_points(u) - interior_points(tgt)) ** 2).mean(axis=0))
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
    assert np.all(B.rms_diff(grid, a, a, work) == 0)
    # roughness: the RMS of the Kreiss-Oliger operator's output over the interior
    st = LR.Stepper.__new__(LR.Stepper)
    st.p = type("P", (), {"gc": grid, "params": params})()
    st.work_con, st.ko_buf, st.zero = work, None, None
    r = st.roughness(a)
    ko = B.alloc_state(grid)
    B.ko_dissipation(grid, params, B.FP64, a, ko)
    k = interior_points(B.download(ko, grid))
    np.testing.assert_allclose(r, np.sqrt((k ** 2).mean(axis=0)), rtol=1e-12, atol=0)
    assert np.all(r > 0)


def _bl_stepper(masses=(0.45, 0.55), separation=2.7):
    from paper_1307_6488_gb300 import learned as LR
    return LR, LR.Stepper(LR.Problem("bl", N, masses=masses, separation=separation))


def test_fallback_is_the_fine_method(setup):
    torch, _, _, _, _, _, _, c = setup
    LR, st = _bl_stepper()
    B.corrector_set_scales(c, np.zeros(24), np.ones(24), np.ones(24))
    y = st.src_c.clone()
    before = y.clone()
    # factor 0: the learned step is never accepted
    used, h_learned, h_plain = LR.learned_step(st, c, y, fallback_factor=0.0)
    assert used and h_plain > 0
    # y + R(F F P y) - R(P y), formed here on the host from the same kernels
    fine = B.alloc_state(st.p.gf)
    st.prolong(before, fine)
    base = B.alloc_state(st.p.gc)
    st.restrict(fine, base)
    st.fine_step(fine)
    st.fine_step(fine)
    ref = B.alloc_state(st.p.gc)
    st.restrict(fine, ref)
    torch.cuda.synchronize()
    g = st.p.g
    I = (slice(None),) + (slice(g, -g),) * 3
    y0, r0, r2 = (B.download(t, st.p.gc) for t in (before, base, ref))
    want = y0[I] + (r2[I] - r0[I])
    np.testing.assert_array_equal(B.download(y, st.p.gc)[I], want)


def test_add_difference_is_elementwise(setup):
    torch, grid, u, tgt, off, isc, osc, c = setup
    rng = np.random.default_rng(9)
    w = rng.standard_normal(u.shape)
    y, a, b = B.upload(u, grid), B.upload(tgt, grid), B.upload(w, grid)
    out = B.upload(np.full(u.shape, 7.0), grid)
    B.add_difference(grid, y, a, b, out)
    got = B.download(out, grid)
    I = (slice(None),) + (slice(G, -G),) * 3
    np.testing.assert_array_equal(got[I], u[I] + (tgt[I] - w[I]))
    ghost = np.ones(u.shape, bool)
    ghost[I] = False
    assert np.all(got[ghost] == 7.0)
    # in place on an input
    B.add_difference(grid, y, a, b, y)
    np.testing.assert_array_equal(B.download(y, grid)[I], u[I] + (tgt[I] - w[I]))


def test_fallback_is_closer_to_the_fine_method_than_a_plain_step():
    """On the smooth gauge wave the fallback step must land closer to the
    restricted fine solution than the plain coarse step does (errors are
    measured against the plain fine method), and closer than restricting the
    fine steps of the prolonged state outright. It cannot reach the fine
    method itself: the fine steps start from an interpolated state whose
    interpolation error their second derivatives amplify."""
    need_gpu()
    from paper_1307_6488_gb300 import learned as LR
    st = LR.Stepper(LR.Problem("gw", N, amplitude=0.07))
    fine = st.src_f.clone()
    start = B.alloc_state(st.p.gc)
    st.restrict(fine, start)
    plain = start.clone()
    st.coarse_step(plain)
    fb = B.alloc_state(st.p.gc)
    LR.fallback_step(st, start, fb)
    st.fine_step(fine)
    st.fine_step(fine)
    ref = B.alloc_state(st.p.gc)
    st.restrict(fine, ref)
    g = st.p.g
    I = (slice(None),) + (slice(g, -g),) * 3
    r = B.download(ref, st.p.gc)[I]
    e_plain = np.abs(B.download(plain, st.p.gc)[I] - r).max()
    e_fb = np.abs(B.download(fb, st.p.gc)[I] - r).max()
    direct = B.alloc_state(st.p.gf)
    st.prolong(start, direct)
    st.fine_step(direct)
    st.fine_step(direct)
    old = B.alloc_state(st.p.gc)
    st.restrict(direct, old)
    e_old = np.abs(B.download(old, st.p.gc)[I] - r).max()
    assert e_fb < 0.8 * e_plain and e_fb < e_old, (e_fb, e_plain, e_old)


def test_fallback_triggers_on_a_harmful_correction(setup):
    torch, _, _, _, _, _, _, c = setup
    LR, st = _bl_stepper()
    # tiny output scale: the correction is the raw network output x 1e6
    B.corrector_set_scales(c, np.zeros(24), np.ones(24), np.full(24, 1e-6))
    y = st.src_c.clone()
    used, h_learned, h_plain = LR.learned_step(st, c, y, fallback_factor=2.0)
    assert used and not (h_learned <= 2.0 * h_plain)
    # accepted when the bound is loose enough
    B.corrector_set_scales(c, np.zeros(24), np.ones(24), np.full(24, 1e12))
    y = st.src_c.clone()
    used, h_learned, h_plain = LR.learned_step(st, c, y, fallback_factor=2.0)
    assert not used


def test_trained_corrector_beats_the_plain_coarse_method():
    """Train on pairs the plain method generates (16 fine trajectories at
    64^3 -> 32^3 coarse, 10 pairs each: Brill-Lindquist pairs with masses
    0.3-0.7 and separations 2-4, every fifth a gauge wave), then evolve two
    held-out Brill-Lindquist problems 8 coarse steps: the learned error
    against the restricted fine solution must be under half the plain
    coarse error, with no fallback, and the Hamiltonian-constraint L2 must
    stay within 10% of the fine method's."""
    torch = need_gpu()
    from paper_1307_6488_gb300 import learned as LR
    rng = np.random.default_rng(0)
    probs = []
    for i in range(16):
        if i % 5 == 4:
            probs.append(LR.Problem("gw", N, amplitude=float(rng.uniform(0.02, 0.1))))
        else:
            m = rng.uniform(0.3, 0.7, 2)
            probs.append(LR.Problem("bl", N, masses=tuple(m), separation=float(rng.uniform(2, 4))))
    c = B.corrector_create(N, 4, seed=1)
    try:
        pairs = [(pr, LR.trajectory_pairs(LR.Stepper(pr), 10)) for pr in probs]
        sample = [pp for (_, ps) in pairs for pp in ps[::3]]
        B.corrector_set_scales(c, *LR.default_scales(sample, probs[0].gc))
        data = LR.Dataset(c, N)
        for pr, ps in pairs:
            data.add(ps, pr.gc)
        del pairs, sample
        losses = LR.train(c, data, epochs=30, batch=4, lr=1e-3, lr_final=5e-5)
        assert np.mean(losses[-10:]) < 0.2 * losses[0]
        for kw in (dict(masses=(0.45, 0.55), separation=2.7), dict(masses=(0.35, 0.65), separation=3.5)):
            st = LR.Stepper(LR.Problem("bl", N, **kw))
            r = LR.evaluate(st, c, 8)
            assert r["fallbacks"] == 0, r
            assert r["err_learned"] < 0.5 * r["err_plain"], r
            assert abs(r["ham_learned"] - r["ham_fine"]) < 0.1 * r["ham_fine"], r
            # the same network after coarse steps in the FP32-RHS form (FP64
            # state, check and fine reference): the FP32 right-hand side's
            # error is far below the coarse truncation error it corrects
            st32 = LR.Stepper(LR.Problem("bl", N, **kw), prec=B.FP32_RHS, fine_prec=B.FP64)
            r32 = LR.evaluate(st32, c, 8)
            assert r32["fallbacks"] == 0, r32
            assert abs(r32["err_learned"] - r["err_learned"]) < 0.02 * r["err_learned"], (r, r32)
            assert abs(r32["err_plain"] - r["err_plain"]) < 0.02 * r["err_plain"], (r, r32)
    finally:
        B.corrector_destroy(c)
