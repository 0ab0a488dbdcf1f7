"""The C ABI (include/bssn.h) without a GPU: the library loads, exports
every declared entry point, sizes its scratch, and rejects invalid arguments
with a status code before launching anything (no call here reaches a kernel:
each one is invalid for at least one reason the host checks).

Every pointer handed to those calls points into a live allocation large
enough for what the call could touch (device memory when a GPU is present,
host memory otherwise), so that a regression in the host-side checks could
not make a kernel touch memory that does not exist."""
import ctypes
import os
import re

import pytest

from paper_1307_6488_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1307_6488_gb300 import build
    build.build()
    return B.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bssn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bssn_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_inputs_module_holds_no_evolution_arithmetic():
    src = open(os.path.join(ROOT, "paper_1307_6488_gb300", "inputs.py")).read()
    for word in ("rhs", "ko_", "rk4", "stencil", "upwind"):
        assert word not in src.lower().replace("right-hand side", ""), word


def test_status_strings(L):
    for s in range(7):
        assert B.status_string(s)
    assert B.status_string(99) == "unknown status"


def test_work_bytes(L):
    g = B.make_grid(32, 24, 16, ghost=5, dx=0.1)
    p8 = B.make_params(fd_order=8)
    p4 = B.make_params(fd_order=4)
    n8 = B.work_bytes(g, p8)
    n4 = B.work_bytes(g, p4)
    assert n8 >= 2 * 11 * 4 * g.var_stride * 8
    assert n4 >= 2 * 11 * 2 * g.var_stride * 8
    assert n8 > n4
    bad = B.make_grid(32, 24, 16, ghost=4, dx=0.1)  # ghost 4 < 5 needed at 8th order
    assert B.work_bytes(bad, p8) == 0
    assert B.work_bytes(g, p8, 7) == 0


SLOT = 2 << 20  # bytes per live buffer: more than any call below could touch


@pytest.fixture(scope="module")
def P():
    """P(k): address of the k-th of eight live 2 MiB buffers (k = 1..8)."""
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    block = torch.zeros(9 * SLOT, dtype=torch.uint8, device=dev)
    base = (block.data_ptr() + 255) // 256 * 256
    yield lambda k: base + k * SLOT
    del block


def test_invalid_arguments_rejected(L, P):
    G = ctypes.byref
    g = B.make_grid(8, ghost=3, dx=0.1)
    p = B.make_params(fd_order=4)
    nb = B.work_bytes(g, p)
    E = B.ERR_INVALID_ARG
    # order not supported
    assert L.bssn_rhs(G(g), G(B.make_params(fd_order=6)), 0, P(1), P(1) + 4096, P(2), nb, None) == E
    # ghost too small for 8th order
    assert L.bssn_rhs(G(g), G(B.make_params(fd_order=8)), 0, P(1), P(1) + 4096, P(2), nb, None) == E
    # misaligned state pointer
    assert L.bssn_rhs(G(g), G(p), 0, P(1) + 8, P(4), P(2), nb, None) == E
    # aliasing state and rhs
    assert L.bssn_rhs(G(g), G(p), 0, P(1), P(1), P(2), nb, None) == E
    # scratch too small
    assert L.bssn_rhs(G(g), G(p), 0, P(1), P(4), P(2), nb - 8, None) == E
    # unknown precision
    assert L.bssn_rhs(G(g), G(p), 9, P(1), P(4), P(2), nb, None) == E
    # bad stage / non-finite dt / aliasing
    assert L.bssn_rk4_stage(G(g), G(p), 0, 4, 0.1, P(1), P(1), P(2), P(3), P(4), nb, None) == E
    assert L.bssn_rk4_stage(G(g), G(p), 0, 0, float("nan"), P(1), P(1), P(2), P(3), P(4), nb, None) == E
    assert L.bssn_rk4_stage(G(g), G(p), 0, 1, 0.1, P(1), P(3), P(2), P(3), P(4), nb, None) == E
    # bad grid: zero size, odd var_stride, stride too small, bad spacing
    for bad in (B.Grid(0, 8, 8, 3, 0.1, 0.1, 0.1, 4096), B.Grid(8, 8, 8, 3, 0.1, 0.1, 0.1, 14 ** 3 + 1),
                B.Grid(8, 8, 8, 3, 0.1, 0.1, 0.1, 100), B.Grid(8, 8, 8, 3, -0.1, 0.1, 0.1, 4096)):
        assert L.bssn_fill_ghosts(G(bad), 0, None, P(1), None) == E
    # ghost modes
    assert L.bssn_fill_ghosts(G(g), 2, None, P(1), None) == E
    assert L.bssn_fill_ghosts(G(g), 1, None, P(1), None) == E
    # bad gauge selections
    assert L.bssn_rhs(G(g), G(B.make_params(lapse=3)), 0, P(1), P(4), P(2), nb, None) == E
    assert L.bssn_rhs(G(g), G(B.make_params(shift=2)), 0, P(1), P(4), P(2), nb, None) == E
    # constraints without host outputs
    assert L.bssn_constraints(G(g), G(p), P(1), None, None, None, None, None, P(2), nb, None) == E
    # algebraic constraints: no host outputs, misaligned state, scratch too small
    h2 = ctypes.cast((ctypes.c_double * 2)(), ctypes.c_void_p)
    assert L.bssn_algebraic_constraints(G(g), G(p), P(1), None, None, P(2), nb, None) == E
    assert L.bssn_algebraic_constraints(G(g), G(p), P(1) + 8, h2, h2, P(2), nb, None) == E
    assert L.bssn_algebraic_constraints(G(g), G(p), P(1), h2, h2, P(2), nb - 8, None) == E
    # step: bad boundary mode
    assert L.bssn_rk4_step(G(g), G(p), 0, 0.1, 3, None, P(1), P(2), P(4), nb, None) == E
    assert B.last_error() == B.OK


def test_plan_invalid_arguments_rejected(L, P):
    p = B.make_params(fd_order=4)
    good = B.make_grid(8, ghost=4, dx=0.1)
    bad = B.make_grid(8, ghost=2, dx=0.1)  # ghost 2 < 3 needed at 4th order
    with pytest.raises(B.BssnError) as e:
        B.plan_create([(bad, P(1), P(2))], p)
    assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BssnError) as e:
        B.plan_create([(good, P(1), P(1))], p)  # state aliases its ghost source
    assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BssnError) as e:
        B.plan_create([(good, P(1) + 8, P(2))], p)  # misaligned
    assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BssnError) as e:
        B.plan_create([(good, P(1), P(2))], p, prec=5)
    assert e.value.status == B.ERR_INVALID_ARG
    assert L.bssn_plan_destroy(None) == B.ERR_INVALID_ARG


def test_transfer_rejects_invalid_arguments(L, P):
    """Host-side checks of the 2:1 transfer (no kernel is reached)."""
    fake = ctypes.c_void_p(P(1))  # live and 16-byte aligned; never dereferenced
    gf = B.make_grid(8, ghost=1, dx=0.1)
    gc = B.make_grid(4, ghost=2, dx=0.2)
    odd = B.make_grid(9, ghost=1, dx=0.1)
    gc1 = B.make_grid(4, ghost=1, dx=0.2)
    gf0 = B.make_grid(8, ghost=0, dx=0.1)
    L.bssn_restrict.argtypes = [ctypes.POINTER(B.Grid), ctypes.c_void_p, ctypes.POINTER(B.Grid), ctypes.c_void_p,
                                ctypes.c_int, ctypes.c_void_p]
    L.bssn_prolong.argtypes = [ctypes.POINTER(B.Grid), ctypes.c_void_p, ctypes.POINTER(B.Grid), ctypes.c_void_p,
                               ctypes.c_void_p]
    r = lambda f, c, order, pf=fake, pc=ctypes.c_void_p(P(2)): L.bssn_restrict(ctypes.byref(f), pf, ctypes.byref(c),
                                                                              pc, order, None)
    assert r(odd, gc, 4) == B.ERR_INVALID_ARG  # not a 2:1 pair
    assert r(gf, gc, 3) == B.ERR_INVALID_ARG  # unknown order
    assert r(gf0, gc, 4) == B.ERR_INVALID_ARG  # order 4 needs a fine ghost
    assert r(gf, gc, 2, pf=ctypes.c_void_p(P(1) + 4)) == B.ERR_INVALID_ARG  # misaligned
    assert r(gf, gc, 2, pc=fake) == B.ERR_INVALID_ARG  # same buffer
    p = lambda c, f: L.bssn_prolong(ctypes.byref(c), fake, ctypes.byref(f), ctypes.c_void_p(P(2)), None)
    assert p(gc1, gf) == B.ERR_INVALID_ARG  # coarse ghost < 2
    assert p(gc, odd) == B.ERR_INVALID_ARG


def test_mma_rate_probe_rejects_bad_width(L):
    L.bssn_probe_mma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double()
    for n in (0, 16, 48, 512):
        assert L.bssn_probe_mma_rate(n, ctypes.byref(out)) == B.ERR_INVALID_ARG
    assert L.bssn_probe_mma_rate(32, None) == B.ERR_INVALID_ARG


def test_rk3_rejects_invalid_arguments(L, P):
    """Host-side checks of the RK3 entry points (no kernel is reached)."""
    g = B.make_grid(8, ghost=3, dx=0.1)
    p = B.make_params(fd_order=4)
    fake = ctypes.c_void_p(P(1))
    other = ctypes.c_void_p(P(2))
    big = ctypes.c_ulonglong(1 << 40)
    L.bssn_rk3_stage.argtypes = [ctypes.POINTER(B.Grid), ctypes.POINTER(B.Params), ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_void_p]
    st = lambda stage, ys, yn, prec=B.FP64: L.bssn_rk3_stage(ctypes.byref(g), ctypes.byref(p), prec, stage, 0.01,
                                                             fake, ys, yn, fake, big, None)
    assert st(3, other, ctypes.c_void_p(P(3))) == B.ERR_INVALID_ARG  # stages are 0..2
    assert st(-1, other, ctypes.c_void_p(P(3))) == B.ERR_INVALID_ARG
    assert st(1, other, other) == B.ERR_INVALID_ARG  # ynext must not be ys
    assert st(1, other, ctypes.c_void_p(P(3) + 2)) == B.ERR_INVALID_ARG  # misaligned
    assert st(1, other, ctypes.c_void_p(P(3)), prec=7) == B.ERR_INVALID_ARG
    L.bssn_rk3_step.argtypes = [ctypes.POINTER(B.Grid), ctypes.POINTER(B.Params), ctypes.c_int, ctypes.c_double,
                                ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_ulonglong, ctypes.c_void_p]
    assert L.bssn_rk3_step(ctypes.byref(g), ctypes.byref(p), B.FP64, 0.01, 2, None, fake, other, fake, big,
                           None) == B.ERR_INVALID_ARG  # unknown boundary mode
    assert L.bssn_rk3_step(ctypes.byref(g), ctypes.byref(p), B.FP64, 0.01, 1, None, fake, other, fake, big,
                           None) == B.ERR_INVALID_ARG  # static boundary needs ghost_src
    assert L.bssn_rk3_step(ctypes.byref(g), ctypes.byref(p), B.FP64, float("nan"), 0, None, fake, other, fake, big,
                           None) == B.ERR_INVALID_ARG


def test_psi4_rejects_invalid_arguments(L, P):
    g = B.make_grid(8, ghost=3, dx=0.1)
    p = B.make_params(fd_order=4)
    fake = ctypes.c_void_p(P(1))
    big = ctypes.c_ulonglong(1 << 40)
    L.bssn_psi4.argtypes = [ctypes.POINTER(B.Grid), ctypes.POINTER(B.Params), ctypes.c_void_p,
                            ctypes.POINTER(ctypes.c_double)] + [ctypes.c_void_p] * 7 + [ctypes.c_ulonglong,
                                                                                        ctypes.c_void_p]
    ok = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    nan = (ctypes.c_double * 3)(0.0, float("nan"), 0.0)
    call = lambda origin, out, work=fake: L.bssn_psi4(ctypes.byref(g), ctypes.byref(p), fake, origin, out, None,
                                                      None, None, None, None, work, big, None)
    assert call(None, ctypes.c_void_p(P(2))) == B.ERR_INVALID_ARG  # origin required
    assert call(nan, ctypes.c_void_p(P(2))) == B.ERR_INVALID_ARG
    assert call(ok, fake) == B.ERR_INVALID_ARG  # output may not be the state
    assert call(ok, ctypes.c_void_p(P(2) + 8)) == B.ERR_INVALID_ARG  # misaligned output
    bad8 = B.make_grid(8, ghost=4, dx=0.1)
    p8 = B.make_params(fd_order=8)
    assert L.bssn_psi4(ctypes.byref(bad8), ctypes.byref(p8), fake, ok, None, None, None, None, None, None, fake,
                       big, None) == B.ERR_INVALID_ARG  # ghost 4 < 5 at 8th order


def test_amr_rejects_invalid_arguments(L, P):
    """Host-side checks of the refined-hierarchy entry points: each call is
    invalid for a reason checked before any allocation or launch."""
    p4 = B.make_params(fd_order=4)
    g = 4
    vs = (8 + 2 * g) ** 3

    def create(patches, ncells=(8, 8, 8), ghost=g, boundary=2, dt0=0.1, params=p4, prec=B.FP64, h0=1.0):
        with pytest.raises(B.BssnError) as e:
            B.amr_create(patches, ncells, (-4.0, -4.0, -4.0), h0, ghost, boundary, dt0, params, prec)
        return e.value.status

    good = (0, (0, 0, 0), (8, 8, 8), vs, P(1), None)
    E = B.ERR_INVALID_ARG
    assert create([good], ghost=2) == E                              # ghost < 3 at 4th order
    assert create([good], ghost=4, params=B.make_params(fd_order=8)) == E  # ghost < 5 at 8th order
    assert create([good], boundary=3) == E
    assert create([good], dt0=float("nan")) == E
    assert create([good], h0=0.0) == E
    assert create([good], prec=4) == E
    assert create([good], params=B.make_params(fd_order=6)) == E
    assert create([(0, (1, 0, 0), (8, 8, 8), vs, P(1), None)]) == E   # outside the level-0 domain
    assert create([good, (1, (12, 4, 4), (8, 8, 8), vs, P(1), None)]) == E  # outside the level-1 domain
    assert create([good, (2, (8, 8, 8), (8, 8, 8), vs, P(1), None)]) == E   # level 1 missing
    assert create([(0, (0, 0, 0), (8, 8, 8), vs - 2, P(1), None)]) == E     # var_stride too small
    assert create([(0, (0, 0, 0), (8, 8, 8), vs, P(1) + 8, None)]) == E     # misaligned state
    assert create([good], boundary=1) == E                           # static boundary needs ghost_src
    assert create([(0, (0, 0, 0), (8, 8, 8), vs, P(1), P(1))], boundary=1) == E  # ghost_src is the state
    assert create([]) == E
    assert L.bssn_amr_destroy(None) == E
    assert L.bssn_amr_step(None, None) == E
    grid = B.make_grid(8, ghost=3, dx=0.1)
    with pytest.raises(B.BssnError) as e:
        B.sommerfeld_rhs(grid, p4, (1.0, 2.0, 3.0), P(1), P(1), stream=0)  # output is the state
    assert e.value.status == E
    with pytest.raises(B.BssnError) as e:
        B.sommerfeld_rhs(B.make_grid(8, ghost=0, dx=0.1), p4, (1.0, 2.0, 3.0), P(1), P(2), stream=0)
    assert e.value.status == E
    assert B.last_error() == B.OK


def test_cfd_rejects_invalid_arguments(L, P):
    """Host-side checks of the CFD entry points (no kernel is reached)."""
    ok = B.make_cfd((8, 8, 8), 0.1, (1, 0, 0), nu=0.01, dt=0.001)
    assert B.cfd_points(ok) == 10 ** 3
    bad = [B.make_cfd((7, 8, 8), 0.1, (1, 0, 0), nu=0.01, dt=0.001),      # odd periodic axis
           B.make_cfd((1, 8, 8), 0.1, (0, 0, 0), nu=0.01, dt=0.001),      # too few cells
           B.make_cfd((8, 8, 8), 0.1, (0, 0, 0), nu=0.01, dt=0.0),        # dt
           B.make_cfd((8, 8, 8), 0.1, (0, 0, 0), nu=0.01, dt=0.1, omega=2.0),
           B.make_cfd((8, 8, 8), 0.1, (0, 0, 0), nu=0.01, dt=0.1, alpha=1.5),
           B.make_cfd((8, 8, 8), 0.1, (2, 0, 0), nu=0.01, dt=0.1)]
    for d in bad:
        assert B.cfd_points(d) == 0
        with pytest.raises(B.BssnError) as e:
            B.cfd_boundary(d, P(1), P(2), P(3), P(4), stream=0)
        assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BssnError) as e:
        B.cfd_mass(ok, 2, P(1), P(2), P(3), P(4), stream=0)  # colour
    assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BssnError) as e:
        B.cfd_velocity(ok, P(1), P(2), P(3), P(4), P(1), P(5), P(6), stream=0)  # un is u
    assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BssnError) as e:
        B.cfd_step(ok, 4, P(1), P(2), P(3), P(4), P(1) + 4, stream=0)  # misaligned scratch
    assert e.value.status == B.ERR_INVALID_ARG
    for args in ((P(1), P(2), P(3), P(1), P(5), P(6), P(7)),   # un is u
                 (P(1), P(2), P(3), P(4), P(5), P(6), P(6)),  # p is wn
                 (P(1), P(2), P(3), P(4), P(5), P(6), P(1) + 8)):  # misaligned p
        with pytest.raises(B.BssnError) as e:
            B.cfd_mass_iteration(ok, *args, stream=0)
        assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BssnError) as e:
        B.cfd_mass_iteration(bad[0], P(1), P(2), P(3), P(4), P(5), P(6), P(7), stream=0)
    assert e.value.status == B.ERR_INVALID_ARG
    assert B.last_error() == B.OK


def test_amr_regrid_rejects_null(L):
    L.bssn_amr_regrid.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert L.bssn_amr_regrid(None, None, 1, ctypes.byref(out), None) == B.ERR_INVALID_ARG
