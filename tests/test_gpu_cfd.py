"""The CFD benchmark's three kernels (SOLA Navier-Stokes, single precision)
on the GPU, through the C ABI, against the oracle (oracle/cfd.py) on the
same seeded inputs.

Tolerance: the GPU and the float32 oracle evaluate the same formulas in
float32; they differ by rounding order (fused multiply-adds on the GPU), a
few units of 2^-24 per operation. Per field, the difference after each
kernel must stay below 1e-5 of the field's largest magnitude (at least 1),
and after several full steps below 1e-4. Against the float64 oracle the bound
is the single-precision error, 1e-3 after several steps."""
import numpy as np
import pytest

from oracle import cfd
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _fields(n, seed, amp=0.5):
    shape = (n[2] + 2, n[1] + 2, n[0] + 2)
    return [amp * inputs.uniform_noise(seed + c, 5, shape) for c in range(4)]


def _flow(n, h, per, dtype, **kw):
    return cfd.Flow(n, h, per, dtype=dtype, **kw)


def _desc(F):
    return B.make_cfd(F.n, F.h, F.per, float(F.nu), float(F.dt), float(F.omega), float(F.alpha), float(F.lid),
                      tuple(float(x) for x in F.g))


def _to_dev(torch, arrays):
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in arrays]


def _err(got, want):
    return float(np.max(np.abs(got - want)) / max(1.0, float(np.max(np.abs(want)))))


CASES = [
    ((12, 10, 8), (0.1, 0.12, 0.09), (False, False, False), dict(nu=0.01, dt=0.004, lid=1.0, alpha=0.3)),
    ((8, 6, 10), (0.2, 0.2, 0.1), (True, True, False), dict(nu=0.05, dt=0.003, alpha=0.0, g=(0.0, 0.0, -1.0))),
    ((9, 8, 6), (0.1, 0.1, 0.1), (False, True, True), dict(nu=0.02, dt=0.004, alpha=1.0, omega=1.4)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_kernels_match_oracle(case):
    torch = need_gpu()
    n, h, per, kw = CASES[case]
    F = _flow(n, h, per, np.float32, **kw)
    F.u[...], F.v[...], F.w[...], F.p[...] = [a.astype(np.float32) for a in _fields(n, 100 + 10 * case)]
    d = _desc(F)
    assert B.cfd_points(d) == F.u.size
    u, v, w, p = _to_dev(torch, (F.u, F.v, F.w, F.p))
    # boundary
    F.boundary()
    B.cfd_boundary(d, u, v, w, p)
    torch.cuda.synchronize()
    for a, b in zip((u, v, w, p), (F.u, F.v, F.w, F.p)):
        assert np.array_equal(a.cpu().numpy(), b)
    # velocity
    un, vn, wn = (x.clone() for x in (u, v, w))
    F.velocity()
    B.cfd_velocity(d, u, v, w, p, un, vn, wn)
    torch.cuda.synchronize()
    for a, b in zip((un, vn, wn), (F.u, F.v, F.w)):
        assert _err(a.cpu().numpy(), b) < 1e-5
    # one mass-conservation half-sweep of each colour, on the oracle's state
    u, v, w, p = _to_dev(torch, (F.u, F.v, F.w, F.p))
    for colour in (0, 1):
        F.half_sweep(colour)
        B.cfd_mass(d, colour, u, v, w, p)
        torch.cuda.synchronize()
        for a, b in zip((u, v, w, p), (F.u, F.v, F.w, F.p)):
            assert _err(a.cpu().numpy(), b) < 1e-5


@pytest.mark.parametrize("case", range(len(CASES)))
def test_steps_match_oracle(case):
    torch = need_gpu()
    n, h, per, kw = CASES[case]
    init = _fields(n, 200 + 10 * case, amp=0.2)
    F32 = _flow(n, h, per, np.float32, **kw)
    F64 = _flow(n, h, per, np.float64, **kw)
    for F in (F32, F64):
        F.u[...], F.v[...], F.w[...], F.p[...] = [a.astype(F.dtype) for a in init]
    d = _desc(F32)
    u, v, w, p = _to_dev(torch, (F32.u, F32.v, F32.w, F32.p))
    npts = B.cfd_points(d)
    scratch = torch.zeros(3 * ((npts + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    for _ in range(4):
        F32.step(4)
        F64.step(4)
        B.cfd_step(d, 4, u, v, w, p, scratch)
    torch.cuda.synchronize()
    for a, b32, b64 in zip((u, v, w, p), (F32.u, F32.v, F32.w, F32.p), (F64.u, F64.v, F64.w, F64.p)):
        g = a.cpu().numpy()
        assert _err(g, b32) < 1e-4
        assert _err(g, b64) < 1e-3


def test_lid_cavity_full_size_sampled():
    """The benchmark's 256^3 lid-driven cavity in the launch configuration
    it times: the velocity kernel at 4096 sampled faces against the oracle
    evaluated on the 3^3-cell neighbourhood of each, and the mass kernel's
    defining property at every cell of the half-sweep (its divergence
    becomes (1 - omega) D)."""
    torch = need_gpu()
    N = 256
    h = 1.0 / N
    d = B.make_cfd((N, N, N), h, (0, 0, 0), nu=1e-3, dt=0.25 * h, omega=1.7, alpha=0.3, lid=1.0)
    npts = B.cfd_points(d)
    shape = (N + 2, N + 2, N + 2)
    gen = torch.Generator(device="cuda").manual_seed(7)
    u, v, w, p = (0.1 * torch.rand(shape, generator=gen, device="cuda", dtype=torch.float32) for _ in range(4))
    scratch = torch.zeros(3 * ((npts + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    B.cfd_step(d, 4, u, v, w, p, scratch)  # a realistic state: one step of the benchmark
    B.cfd_boundary(d, u, v, w, p)
    un, vn, wn = (x.clone() for x in (u, v, w))
    B.cfd_velocity(d, u, v, w, p, un, vn, wn)
    torch.cuda.synchronize()
    U, V, W, P = (x.cpu().numpy() for x in (u, v, w, p))
    Un, Vn, Wn = (x.cpu().numpy() for x in (un, vn, wn))
    rng = np.random.default_rng(3)
    pts = rng.integers(1, N - 2, size=(4096, 3))  # cells away from the walls: every face is advanced
    for (i, j, k) in pts:
        # cells i-1 .. i+1 (padded i .. i+2) and their ghost layer: the
        # centre cell's faces depend on nothing outside this window
        sub = [np.ascontiguousarray(a[k - 1:k + 4, j - 1:j + 4, i - 1:i + 4]) for a in (U, V, W, P)]
        G = cfd.Flow((3, 3, 3), (h, h, h), (False, False, False), nu=1e-3, dt=0.25 * h, alpha=0.3, dtype=np.float32)
        G.u[...], G.v[...], G.w[...], G.p[...] = sub
        G.velocity()
        for got, want in ((Un, G.u), (Vn, G.v), (Wn, G.w)):
            assert abs(got[k + 1, j + 1, i + 1] - want[2, 2, 2]) <= 1e-5 * max(1.0, abs(want[2, 2, 2]))
    # mass half-sweep: every red cell's divergence scales by (1 - omega)
    def div(U, V, W):
        return ((U[1:-1, 1:-1, 1:-1] - U[1:-1, 1:-1, :-2]) + (V[1:-1, 1:-1, 1:-1] - V[1:-1, :-2, 1:-1])
                + (W[1:-1, 1:-1, 1:-1] - W[:-2, 1:-1, 1:-1])) / h
    D0 = div(U, V, W)
    B.cfd_mass(d, 0, u, v, w, p)
    torch.cuda.synchronize()
    D1 = div(*(x.cpu().numpy() for x in (u, v, w)))
    kk, jj, ii = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    red = (ii + jj + kk) % 2 == 0
    assert np.max(np.abs(D1[red] - (1 - 1.7) * D0[red])) < 1e-3 * np.max(np.abs(D0))


STEP_CASES = CASES + [
    ((2, 6, 4), (0.1, 0.1, 0.1), (True, False, True), dict(nu=0.02, dt=0.002, alpha=0.5)),   # two cells on a periodic axis
    ((37, 13, 19), (0.05, 0.07, 0.06), (False, False, False), dict(nu=0.01, dt=0.002, lid=1.0)),  # ragged boxes
    ((34, 18, 36), (0.05, 0.05, 0.05), (True, True, True), dict(nu=0.01, dt=0.002)),           # every axis periodic
    # large enough for boxes away from every wall and seam (the kernel's short path)
    ((70, 14, 38), (0.03, 0.04, 0.05), (False, False, False), dict(nu=0.01, dt=0.001, lid=1.0)),
    ((68, 12, 36), (0.03, 0.04, 0.05), (True, False, True), dict(nu=0.01, dt=0.001, alpha=0.2)),
]


@pytest.mark.parametrize("case", range(len(STEP_CASES)))
@pytest.mark.parametrize("iterations", [0, 1, 3, 4])
def test_step_equals_its_kernels(case, iterations):
    """bssn_cfd_step runs each mass iteration as one fused pass (colour-0
    moves applied on the fly, faces into the other set of arrays) and the
    boundary once at the end. It must equal, bit for bit, the kernels it
    stands for: boundary, velocity, boundary, then per iteration the
    colour-0 and colour-1 half-sweeps and the boundary."""
    torch = need_gpu()
    n, h, per, kw = STEP_CASES[case]
    F = _flow(n, h, per, np.float32, **kw)
    d = _desc(F)
    init = _fields(n, 300 + 10 * case, amp=0.3)
    a = _to_dev(torch, init)
    b = _to_dev(torch, init)
    npts = B.cfd_points(d)
    scratch = torch.full((3 * ((npts + 3) // 4 * 4),), float("nan"), dtype=torch.float32, device="cuda")
    B.cfd_step(d, iterations, *a, scratch)
    u, v, w, p = b
    B.cfd_boundary(d, u, v, w, p)
    un, vn, wn = (torch.full_like(x, float("nan")) for x in (u, v, w))
    B.cfd_velocity(d, u, v, w, p, un, vn, wn)
    u.copy_(un)
    v.copy_(vn)
    w.copy_(wn)
    B.cfd_boundary(d, u, v, w, p)
    for _ in range(iterations):
        B.cfd_mass(d, 0, u, v, w, p)
        B.cfd_mass(d, 1, u, v, w, p)
        B.cfd_boundary(d, u, v, w, p)
    torch.cuda.synchronize()
    for name, x, y in zip("uvwp", a, b):
        assert torch.equal(x, y), (name, float(torch.max(torch.abs(x - y))))


@pytest.mark.parametrize("case", range(len(STEP_CASES)))
def test_mass_iteration_equals_two_half_sweeps(case):
    """bssn_cfd_mass_iteration (one pass, faces into a second set of arrays)
    against bssn_cfd_mass with colour 0 then colour 1 in place: the written
    entries (interior and low wall faces) and p, bit for bit."""
    torch = need_gpu()
    n, h, per, kw = STEP_CASES[case]
    d = _desc(_flow(n, h, per, np.float32, **kw))
    a = _to_dev(torch, _fields(n, 400 + 10 * case, amp=0.3))
    B.cfd_boundary(d, *a)
    b = [x.clone() for x in a]
    un, vn, wn = (torch.full_like(x, float("nan")) for x in a[:3])
    B.cfd_mass_iteration(d, a[0], a[1], a[2], un, vn, wn, a[3])
    B.cfd_mass(d, 0, *b)
    B.cfd_mass(d, 1, *b)
    torch.cuda.synchronize()
    assert torch.equal(a[3], b[3])
    for ax, (got, want) in enumerate(zip((un, vn, wn), b[:3])):
        assert torch.equal(got[1:-1, 1:-1, 1:-1], want[1:-1, 1:-1, 1:-1]), "uvw"[ax]
        if not per[ax]:  # the low wall face (-1) sits in the ghost layer of its own axis
            lo = [slice(1, -1)] * 3
            lo[2 - ax] = 0
            assert torch.equal(got[tuple(lo)], want[tuple(lo)]), "uvw"[ax]
