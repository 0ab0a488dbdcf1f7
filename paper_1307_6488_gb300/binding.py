"""ctypes binding of libbssn (include/bssn.h): argument marshalling only.

Every function here has the name of the C entry point without the ``bssn_``
prefix and forwards to it; arrays are torch CUDA tensors (float64) or raw
device addresses. The compute path is the CUDA library: if libbssn.so is
missing this module raises instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# BSSN_BOUNDS_CHECK=1 selects the bounds-check build of the same library
LIB_PATH = os.path.join(HERE, "libbssn_check.so" if os.environ.get("BSSN_BOUNDS_CHECK") == "1" else "libbssn.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_NOMEM, ERR_BOUNDS = range(8)
FP64, FP32_RHS = 0, 1
NVAR = 24


class BssnError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("ghost", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("var_stride", ctypes.c_longlong)]

    @property
    def padded(self):
        g = self.ghost
        return (self.nz + 2 * g, self.ny + 2 * g, self.nx + 2 * g)

    @property
    def npad(self):
        z, y, x = self.padded
        return z * y * x


class Params(ctypes.Structure):
    _fields_ = [("fd_order", ctypes.c_int), ("ko_eps", ctypes.c_double), ("lapse", ctypes.c_int),
                ("shift", ctypes.c_int), ("shift_coeff", ctypes.c_double), ("eta", ctypes.c_double),
                ("advect_gauge", ctypes.c_int)]


def make_grid(nx, ny=None, nz=None, ghost=3, dx=1.0, dy=None, dz=None, align=16):
    """Grid with var_stride = padded points rounded up to `align` doubles."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    dy = dx if dy is None else dy
    dz = dx if dz is None else dz
    npad = (nx + 2 * ghost) * (ny + 2 * ghost) * (nz + 2 * ghost)
    vs = (npad + align - 1) // align * align
    return Grid(nx, ny, nz, ghost, dx, dy, dz, vs)


def make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, shift_coeff=0.75, eta=2.0, advect_gauge=1):
    return Params(fd_order, ko_eps, lapse, shift, shift_coeff, eta, advect_gauge)


_L = None
_p = ctypes.c_void_p


def lib():
    global _L
    if _L is not None:
        return _L
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    G, P = ctypes.POINTER(Grid), ctypes.POINTER(Params)
    ull = ctypes.c_ulonglong
    L.bssn_status_string.argtypes = [ctypes.c_int]
    L.bssn_status_string.restype = ctypes.c_char_p
    L.bssn_last_error.restype = ctypes.c_int
    L.bssn_clear_error.restype = None
    L.bssn_work_bytes.argtypes = [G, P, ctypes.c_int]
    L.bssn_work_bytes.restype = ull
    L.bssn_fill_ghosts.argtypes = [G, ctypes.c_int, _p, _p, _p]
    L.bssn_rhs.argtypes = [G, P, ctypes.c_int, _p, _p, _p, ull, _p]
    L.bssn_ko_dissipation.argtypes = [G, P, ctypes.c_int, _p, _p, _p]
    L.bssn_rk4_stage.argtypes = [G, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _p, _p, _p, _p, _p, ull, _p]
    L.bssn_diff_tables.argtypes = [G, P, ctypes.c_int, _p, _p, ull, _p]
    L.bssn_rk4_stage_fused.argtypes = [G, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _p, _p, _p, _p, _p, ull,
                                       _p]
    L.bssn_rk4_step.argtypes = [G, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, _p, _p, _p, _p, ull, _p]
    L.bssn_constraints.argtypes = [G, P, _p, _p, _p, _p, _p, _p, _p, ull, _p]
    L.bssn_algebraic_constraints.argtypes = [G, P, _p, _p, _p, _p, ull, _p]
    L.bssn_hamiltonian.argtypes = [G, P, _p, _p, _p, _p, _p, ull, _p]
    L.bssn_probe_fp_rates.argtypes = [_p]
    for name in ("bssn_fill_ghosts", "bssn_rhs", "bssn_ko_dissipation", "bssn_rk4_stage", "bssn_rk4_step",
                 "bssn_diff_tables", "bssn_rk4_stage_fused",
                 "bssn_constraints", "bssn_hamiltonian", "bssn_algebraic_constraints", "bssn_probe_fp_rates"):
        getattr(L, name).restype = ctypes.c_int
    _L = L
    return L


def status_string(s):
    return lib().bssn_status_string(int(s)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status, where):
    if status != OK:
        raise BssnError(status, where)


def last_error():
    return lib().bssn_last_error()


def clear_error():
    lib().bssn_clear_error()


def bounds_check_enabled():
    L = lib()
    L.bssn_bounds_check_enabled.restype = ctypes.c_int
    return bool(L.bssn_bounds_check_enabled())


def bounds_violations(stream=None):
    """bssn_bounds_violations: (status, count) since the last call, cleared."""
    L = lib()
    L.bssn_bounds_violations.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), _p]
    L.bssn_bounds_violations.restype = ctypes.c_int
    c = ctypes.c_ulonglong(0)
    st = L.bssn_bounds_violations(ctypes.byref(c), _stream(stream))
    return st, c.value


def rms_diff(grid, a, b, work, stream=None):
    """bssn_rms_diff: per-variable RMS of a - b over interior points (numpy, 24)."""
    L = lib()
    L.bssn_rms_diff.argtypes = [ctypes.POINTER(Grid), _p, _p, _p, _p, ctypes.c_ulonglong, _p]
    L.bssn_rms_diff.restype = ctypes.c_int
    out = np.zeros(NVAR)
    _check(L.bssn_rms_diff(ctypes.byref(grid), _ptr(a), _ptr(b), out.ctypes.data_as(_p), _ptr(work), _nbytes(work),
                           _stream(stream)), "rms_diff")
    return out


def check_device(stream=None):
    """bssn_check_device: synchronizes the stream; raises BssnError with
    ERR_TIMEOUT if a bounded wait of a tiled FP32-RHS stage kernel gave up
    since the last check."""
    L = lib()
    L.bssn_check_device.argtypes = [_p]
    L.bssn_check_device.restype = ctypes.c_int
    _check(L.bssn_check_device(_stream(stream)), "bssn_check_device")


def test_conversions(din, fin, f_bits, f_hw, d_bits, d_hw, stream=None):
    """bssn_test_conversions: single/double conversions by the library's
    integer-pipe code and by the hardware instruction, side by side."""
    L = lib()
    L.bssn_test_conversions.argtypes = [ctypes.c_longlong, _p, _p, _p, _p, _p, _p, _p]
    L.bssn_test_conversions.restype = ctypes.c_int
    n = din.numel()
    _check(L.bssn_test_conversions(n, _ptr(din), _ptr(fin), _ptr(f_bits), _ptr(f_hw), _ptr(d_bits), _ptr(d_hw),
                                   _stream(stream)), "bssn_test_conversions")


def work_bytes(grid, params, prec=FP64):
    return int(lib().bssn_work_bytes(ctypes.byref(grid), ctypes.byref(params), prec))


def fill_ghosts(grid, mode, src, state, stream=None):
    _check(lib().bssn_fill_ghosts(ctypes.byref(grid), mode, _ptr(src), _ptr(state), _stream(stream)), "fill_ghosts")


def rhs(grid, params, prec, state, out, work, stream=None):
    _check(lib().bssn_rhs(ctypes.byref(grid), ctypes.byref(params), prec, _ptr(state), _ptr(out), _ptr(work),
                          _nbytes(work), _stream(stream)), "rhs")


def ko_dissipation(grid, params, prec, state, out, stream=None):
    _check(lib().bssn_ko_dissipation(ctypes.byref(grid), ctypes.byref(params), prec, _ptr(state), _ptr(out),
                                     _stream(stream)), "ko_dissipation")


def rk4_stage(grid, params, prec, stage, dt, y0, ys, acc, ynext, work, stream=None):
    _check(lib().bssn_rk4_stage(ctypes.byref(grid), ctypes.byref(params), prec, stage, dt, _ptr(y0), _ptr(ys),
                                _ptr(acc), _ptr(ynext), _ptr(work), _nbytes(work), _stream(stream)), "rk4_stage")


def diff_tables(grid, params, prec, state, work, stream=None):
    _check(lib().bssn_diff_tables(ctypes.byref(grid), ctypes.byref(params), prec, _ptr(state), _ptr(work),
                                  _nbytes(work), _stream(stream)), "diff_tables")


def rk4_stage_fused(grid, params, prec, stage, dt, y0, ys, acc, ynext, work, stream=None):
    _check(lib().bssn_rk4_stage_fused(ctypes.byref(grid), ctypes.byref(params), prec, stage, dt, _ptr(y0), _ptr(ys),
                                      _ptr(acc), _ptr(ynext), _ptr(work), _nbytes(work), _stream(stream)),
           "rk4_stage_fused")


def rk4_stage_noalloc(grid, params, prec, stage, dt, y0, ys, acc, ynext, stream=None):
    """bssn_rk4_stage_noalloc: the stage without a scratch buffer or any
    allocation (the library's static scratch; see include/bssn.h)."""
    L = lib()
    if not getattr(L, "_noalloc_typed", False):
        L.bssn_rk4_stage_noalloc.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, _p, _p, _p, _p, _p]
        L.bssn_rk4_stage_noalloc.restype = ctypes.c_int
        L._noalloc_typed = True
    _check(L.bssn_rk4_stage_noalloc(ctypes.byref(grid), ctypes.byref(params), prec, stage, dt, _ptr(y0), _ptr(ys),
                                    _ptr(acc), _ptr(ynext), _stream(stream)), "rk4_stage_noalloc")


class Block(ctypes.Structure):
    _fields_ = [("grid", Grid), ("state", ctypes.c_void_p), ("ghost_src", ctypes.c_void_p)]


def _plan_lib():
    L = lib()
    if not getattr(L, "_plan_typed", False):
        L.bssn_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Block), ctypes.c_int,
                                       ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int]
        L.bssn_batch_step.argtypes = [_p, ctypes.c_double, _p]
        L.bssn_plan_info.argtypes = [_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _p]
        L.bssn_plan_destroy.argtypes = [_p]
        for n in ("bssn_plan_create", "bssn_batch_step", "bssn_plan_info", "bssn_plan_destroy"):
            getattr(L, n).restype = ctypes.c_int
        L._plan_typed = True
    return L


def plan_create(blocks, params, prec=FP64, autotune=1):
    """blocks: list of (Grid, state, ghost_src) with device tensors/addresses.
    Returns an opaque plan handle (int)."""
    arr = (Block * len(blocks))(*[Block(g, _ptr(s), _ptr(src)) for (g, s, src) in blocks])
    h = ctypes.c_void_p()
    _check(_plan_lib().bssn_plan_create(ctypes.byref(h), arr, len(blocks), ctypes.byref(params), prec, autotune),
           "plan_create")
    return h.value


def batch_step(plan, dt, stream=None):
    _check(_plan_lib().bssn_batch_step(plan, dt, _stream(stream)), "batch_step")


def plan_info(plan, nblocks):
    pts, tiles = ctypes.c_longlong(), ctypes.c_longlong()
    shapes = np.zeros(nblocks, dtype=np.int32)
    _check(_plan_lib().bssn_plan_info(plan, ctypes.byref(pts), ctypes.byref(tiles), shapes.ctypes.data_as(_p)),
           "plan_info")
    return pts.value, tiles.value, shapes


def plan_destroy(plan):
    _check(_plan_lib().bssn_plan_destroy(plan), "plan_destroy")


def _corr_lib():
    L = lib()
    if not getattr(L, "_corr_typed", False):
        vp = ctypes.c_void_p
        L.bssn_corrector_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong]
        L.bssn_corrector_destroy.argtypes = [vp]
        L.bssn_corrector_param_count.restype = ctypes.c_longlong
        L.bssn_corrector_params.argtypes = [vp, vp, ctypes.c_int]
        L.bssn_corrector_grads.argtypes = [vp, vp]
        L.bssn_corrector_set_scales.argtypes = [vp, vp, vp, vp]
        L.bssn_corrector_forward_raw.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        L.bssn_corrector_infer_async.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        L.bssn_corrector_sync.argtypes = [vp, vp]
        L.bssn_corrector_loss_grad_raw.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
        L.bssn_corrector_train_step.argtypes = [vp, ctypes.POINTER(Grid), ctypes.c_int, vp, vp, ctypes.c_float,
                                                ctypes.POINTER(ctypes.c_double), vp]
        L.bssn_corrector_apply.argtypes = [vp, ctypes.POINTER(Grid), vp, vp]
        L.bssn_corrector_layer_output.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
        for n in ("bssn_corrector_create", "bssn_corrector_destroy", "bssn_corrector_params", "bssn_corrector_grads",
                  "bssn_corrector_set_scales", "bssn_corrector_forward_raw", "bssn_corrector_infer_async",
                  "bssn_corrector_sync", "bssn_corrector_loss_grad_raw",
                  "bssn_corrector_train_step", "bssn_corrector_apply", "bssn_corrector_layer_output"):
            getattr(L, n).restype = ctypes.c_int
        L._corr_typed = True
    return L


def corrector_create(n, max_batch, seed=0):
    h = ctypes.c_void_p()
    _check(_corr_lib().bssn_corrector_create(ctypes.byref(h), n, max_batch, seed), "corrector_create")
    return h.value


def corrector_destroy(c):
    _check(_corr_lib().bssn_corrector_destroy(c), "corrector_destroy")


def corrector_param_count():
    return int(_corr_lib().bssn_corrector_param_count())


def corrector_params(c, values=None):
    """Read (values None) or write the packed FP32 parameters."""
    n = corrector_param_count()
    if values is None:
        out = np.zeros(n, dtype=np.float32)
        _check(_corr_lib().bssn_corrector_params(c, out.ctypes.data_as(_p), 0), "corrector_params")
        return out
    v = np.ascontiguousarray(values, dtype=np.float32)
    assert v.size == n
    _check(_corr_lib().bssn_corrector_params(c, v.ctypes.data_as(_p), 1), "corrector_params")


def corrector_grads(c):
    out = np.zeros(corrector_param_count(), dtype=np.float32)
    _check(_corr_lib().bssn_corrector_grads(c, out.ctypes.data_as(_p)), "corrector_grads")
    return out


def corrector_set_scales(c, in_offset, in_scale, out_scale):
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (in_offset, in_scale, out_scale)]
    _check(_corr_lib().bssn_corrector_set_scales(c, *[x.ctypes.data_as(_p) for x in a]), "corrector_set_scales")


def corrector_set_step_scale(c, step_scale):
    a = np.ascontiguousarray(step_scale, dtype=np.float64)
    L = _corr_lib()
    L.bssn_corrector_set_step_scale.argtypes = [_p, _p]
    L.bssn_corrector_set_step_scale.restype = ctypes.c_int
    _check(L.bssn_corrector_set_step_scale(c, a.ctypes.data_as(_p)), "corrector_set_step_scale")


def corrector_forward_raw(c, S, x_bf16, out, stream=None):
    _check(_corr_lib().bssn_corrector_forward_raw(c, S, _ptr(x_bf16), _ptr(out), _stream(stream)),
           "corrector_forward_raw")


def corrector_infer_async(c, S, x_bf16, out, stream=None):
    """Enqueue an inference pass; returns without waiting (see corrector_sync)."""
    _check(_corr_lib().bssn_corrector_infer_async(c, S, _ptr(x_bf16), _ptr(out), _stream(stream)),
           "corrector_infer_async")


def corrector_sync(c, stream=None):
    _check(_corr_lib().bssn_corrector_sync(c, _stream(stream)), "corrector_sync")


def corrector_loss_grad_raw(c, S, x_bf16, target, stream=None):
    loss = ctypes.c_double()
    _check(_corr_lib().bssn_corrector_loss_grad_raw(c, S, _ptr(x_bf16), _ptr(target), ctypes.byref(loss),
                                                    _stream(stream)), "corrector_loss_grad_raw")
    return loss.value


def corrector_train_step(c, grid, coarse, target, lr, stream=None):
    """coarse, target: lists of device state tensors (same length S)."""
    S = len(coarse)
    ca = (ctypes.c_void_p * S)(*[_ptr(x) for x in coarse])
    ta = (ctypes.c_void_p * S)(*[_ptr(x) for x in target])
    loss = ctypes.c_double()
    _check(_corr_lib().bssn_corrector_train_step(c, ctypes.byref(grid), S, ca, ta, lr, ctypes.byref(loss),
                                                 _stream(stream)), "corrector_train_step")
    return loss.value


def _pack_lib():
    L = _corr_lib()
    if not getattr(L, "_pack_typed", False):
        L.bssn_corrector_pack.argtypes = [_p, ctypes.POINTER(Grid), _p, _p, _p, _p, _p]
        L.bssn_corrector_pack.restype = ctypes.c_int
        L.bssn_corrector_train_step_raw.argtypes = [_p, ctypes.c_int, _p, _p, ctypes.c_float,
                                                    ctypes.POINTER(ctypes.c_double), _p]
        L.bssn_corrector_train_step_raw.restype = ctypes.c_int
        L._pack_typed = True
    return L


def corrector_pack(c, grid, coarse, target, x_bf16, t_bf16, stream=None):
    _check(_pack_lib().bssn_corrector_pack(c, ctypes.byref(grid), _ptr(coarse), _ptr(target), _ptr(x_bf16),
                                           _ptr(t_bf16), _stream(stream)), "corrector_pack")


def corrector_train_step_raw(c, xs, ts, lr, stream=None):
    """xs, ts: lists of packed BF16 device tensors (same length S)."""
    L = _pack_lib()
    S = len(xs)
    xa = (ctypes.c_void_p * S)(*[_ptr(x) for x in xs])
    ta = (ctypes.c_void_p * S)(*[_ptr(t) for t in ts])
    loss = ctypes.c_double()
    _check(L.bssn_corrector_train_step_raw(c, S, xa, ta, lr, ctypes.byref(loss), _stream(stream)),
           "corrector_train_step_raw")
    return loss.value


def _transfer_lib():
    L = lib()
    if not getattr(L, "_transfer_typed", False):
        L.bssn_restrict.argtypes = [ctypes.POINTER(Grid), _p, ctypes.POINTER(Grid), _p, ctypes.c_int, _p]
        L.bssn_prolong.argtypes = [ctypes.POINTER(Grid), _p, ctypes.POINTER(Grid), _p, _p]
        L.bssn_add_difference.argtypes = [ctypes.POINTER(Grid), _p, _p, _p, _p, _p]
        for n in ("bssn_restrict", "bssn_prolong", "bssn_add_difference"):
            getattr(L, n).restype = ctypes.c_int
        L._transfer_typed = True
    return L


def restrict(fine_grid, fine_state, coarse_grid, coarse_state, order=4, stream=None):
    """2:1 restriction of the fine state into the coarse interior: order 2 is
    the mean of the 8 children, order 4 tricubic interpolation at the coarse
    centre (fine ghosts >= 1, filled)."""
    _check(_transfer_lib().bssn_restrict(ctypes.byref(fine_grid), _ptr(fine_state), ctypes.byref(coarse_grid),
                                         _ptr(coarse_state), order, _stream(stream)), "restrict")


def add_difference(grid, y, a, b, out, stream=None):
    """bssn_add_difference: out = y + (a - b) at interior points."""
    L = _transfer_lib()
    _check(L.bssn_add_difference(ctypes.byref(grid), _ptr(y), _ptr(a), _ptr(b), _ptr(out), _stream(stream)),
           "add_difference")


def prolong(coarse_grid, coarse_state, fine_grid, fine_state, stream=None):
    """Tricubic 1:2 prolongation of the coarse state (ghosts filled, ghost >= 2)
    onto the fine interior."""
    _check(_transfer_lib().bssn_prolong(ctypes.byref(coarse_grid), _ptr(coarse_state), ctypes.byref(fine_grid),
                                        _ptr(fine_state), _stream(stream)), "prolong")


def psi4(grid, params, state, origin, work, psi_re=None, psi_im=None, inv_re=None, inv_im=None, E=None, B=None,
         stream=None):
    """Weyl diagnostics (E, B, Psi_4, invariant I) at interior points;
    outputs are device tensors in the state layout (E, B: 6 arrays each)."""
    L = lib()
    if not getattr(L, "_psi4_typed", False):
        L.bssn_psi4.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params), _p, ctypes.POINTER(ctypes.c_double),
                                _p, _p, _p, _p, _p, _p, _p, ctypes.c_ulonglong, _p]
        L.bssn_psi4.restype = ctypes.c_int
        L._psi4_typed = True
    o = (ctypes.c_double * 3)(*[float(v) for v in origin])
    _check(L.bssn_psi4(ctypes.byref(grid), ctypes.byref(params), _ptr(state), o, _ptr(psi_re), _ptr(psi_im),
                       _ptr(inv_re), _ptr(inv_im), _ptr(E), _ptr(B), _ptr(work), _nbytes(work), _stream(stream)),
           "psi4")


def probe_mma_rate(n=32):
    """Measured TFLOP/s of back-to-back M=128 K=16 BF16 MMAs with N = n."""
    L = _corr_lib()
    L.bssn_probe_mma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.bssn_probe_mma_rate.restype = ctypes.c_int
    out = ctypes.c_double()
    _check(L.bssn_probe_mma_rate(n, ctypes.byref(out)), "probe_mma_rate")
    return out.value


def corrector_apply(c, grid, state, stream=None):
    _check(_corr_lib().bssn_corrector_apply(c, ctypes.byref(grid), _ptr(state), _stream(stream)), "corrector_apply")


def corrector_layer_output(c, layer, S, out):
    _check(_corr_lib().bssn_corrector_layer_output(c, layer, S, _ptr(out)), "corrector_layer_output")


def _rk3_lib():
    L = lib()
    if not getattr(L, "_rk3_typed", False):
        L.bssn_rk3_stage.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, _p, _p, _p, _p, ctypes.c_ulonglong, _p]
        L.bssn_rk3_step.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params), ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, _p, _p, _p, _p, ctypes.c_ulonglong, _p]
        L.bssn_rk3_stage.restype = ctypes.c_int
        L.bssn_rk3_step.restype = ctypes.c_int
        L._rk3_typed = True
    return L


def rk3_stage(grid, params, prec, stage, dt, y0, ys, ynext, work, stream=None):
    _check(_rk3_lib().bssn_rk3_stage(ctypes.byref(grid), ctypes.byref(params), prec, stage, dt, _ptr(y0), _ptr(ys),
                                     _ptr(ynext), _ptr(work), _nbytes(work), _stream(stream)), "rk3_stage")


def rk3_step(grid, params, prec, dt, bc, ghost_src, state, bufs, work, stream=None):
    """One SSP-RK3 step in place; bufs holds two state-sized buffers."""
    _check(_rk3_lib().bssn_rk3_step(ctypes.byref(grid), ctypes.byref(params), prec, dt, bc, _ptr(ghost_src),
                                    _ptr(state), _ptr(bufs), _ptr(work), _nbytes(work), _stream(stream)), "rk3_step")


def rk4_step(grid, params, prec, dt, bc, ghost_src, state, bufs, work, stream=None):
    _check(lib().bssn_rk4_step(ctypes.byref(grid), ctypes.byref(params), prec, dt, bc, _ptr(ghost_src), _ptr(state),
                               _ptr(bufs), _ptr(work), _nbytes(work), _stream(stream)), "rk4_step")


def constraints(grid, params, state, work, ham=None, mom=None, gcon=None, stream=None):
    """Returns (l2[7], max[7], status); status is OK or ERR_NONFINITE."""
    l2 = np.zeros(7)
    mx = np.zeros(7)
    s = lib().bssn_constraints(ctypes.byref(grid), ctypes.byref(params), _ptr(state), _ptr(ham), _ptr(mom),
                               _ptr(gcon), l2.ctypes.data_as(_p), mx.ctypes.data_as(_p), _ptr(work), _nbytes(work),
                               _stream(stream))
    if s not in (OK, ERR_NONFINITE):
        raise BssnError(s, "constraints")
    return l2, mx, s


def hamiltonian(grid, params, state, work, ham=None, stream=None):
    """Hamiltonian constraint alone: returns (l2, max, status); status is OK
    or ERR_NONFINITE."""
    l2 = np.zeros(1)
    mx = np.zeros(1)
    s = lib().bssn_hamiltonian(ctypes.byref(grid), ctypes.byref(params), _ptr(state), _ptr(ham),
                               l2.ctypes.data_as(_p), mx.ctypes.data_as(_p), _ptr(work), _nbytes(work),
                               _stream(stream))
    if s not in (OK, ERR_NONFINITE):
        raise BssnError(s, "hamiltonian")
    return float(l2[0]), float(mx[0]), s


def algebraic_constraints(grid, params, state, work, stream=None):
    """det(gt) - 1 and gt^ij At_ij over interior points: returns (l2[2],
    max[2], status); status is OK or ERR_NONFINITE."""
    l2 = np.zeros(2)
    mx = np.zeros(2)
    s = lib().bssn_algebraic_constraints(ctypes.byref(grid), ctypes.byref(params), _ptr(state),
                                         l2.ctypes.data_as(_p), mx.ctypes.data_as(_p), _ptr(work), _nbytes(work),
                                         _stream(stream))
    if s not in (OK, ERR_NONFINITE):
        raise BssnError(s, "algebraic_constraints")
    return l2, mx, s


def checkpoint_write(path, grid, params, t, step, state):
    """Write a checkpoint: state is the HOST copy of the full padded state
    (24 * var_stride doubles, e.g. state_tensor.cpu().numpy())."""
    a = np.ascontiguousarray(np.asarray(state, dtype=np.float64).reshape(-1))
    if a.size < NVAR * grid.var_stride:
        raise BssnError(ERR_INVALID_ARG, "checkpoint_write: state smaller than 24 * var_stride")
    _check(_ckp_lib().bssn_checkpoint_write(os.fsencode(path), ctypes.byref(grid), ctypes.byref(params), float(t),
                                           int(step), a.ctypes.data_as(_p)), "checkpoint_write")


def checkpoint_read(path, with_state=True):
    """Read a checkpoint: returns (grid, params, t, step, state) with state a
    HOST numpy array of 24 * var_stride doubles (None without with_state)."""
    L = _ckp_lib()
    grid, params = Grid(), Params()
    t, step = ctypes.c_double(), ctypes.c_longlong()
    _check(L.bssn_checkpoint_read(os.fsencode(path), ctypes.byref(grid), ctypes.byref(params), ctypes.byref(t),
                                  ctypes.byref(step), None, 0), "checkpoint_read")
    state = None
    if with_state:
        state = np.empty(NVAR * grid.var_stride)
        _check(L.bssn_checkpoint_read(os.fsencode(path), ctypes.byref(grid), ctypes.byref(params), ctypes.byref(t),
                                      ctypes.byref(step), state.ctypes.data_as(_p), state.size), "checkpoint_read")
    return grid, params, t.value, step.value, state


def _ckp_lib():
    L = lib()
    if not getattr(L, "_ckp_typed", False):
        Gp, Pp = ctypes.POINTER(Grid), ctypes.POINTER(Params)
        L.bssn_checkpoint_write.argtypes = [ctypes.c_char_p, Gp, Pp, ctypes.c_double, ctypes.c_longlong, _p]
        L.bssn_checkpoint_read.argtypes = [ctypes.c_char_p, Gp, Pp, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong), _p, ctypes.c_ulonglong]
        L.bssn_checkpoint_write.restype = ctypes.c_int
        L.bssn_checkpoint_read.restype = ctypes.c_int
        L._ckp_typed = True
    return L


def probe_wait_timeout(limit_ns):
    """bssn_probe_wait_timeout: returns (status, flags) without raising."""
    L = lib()
    L.bssn_probe_wait_timeout.argtypes = [ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_uint)]
    L.bssn_probe_wait_timeout.restype = ctypes.c_int
    flags = ctypes.c_uint(0)
    st = L.bssn_probe_wait_timeout(limit_ns, ctypes.byref(flags))
    return st, flags.value


def probe_fp_rates():
    out = np.zeros(9)
    _check(lib().bssn_probe_fp_rates(out.ctypes.data_as(_p)), "probe_fp_rates")
    return dict(fp64_fma_per_s=out[0], fp32_fma_per_s=out[1], fp64_add_per_s=out[2],
                fp64_fma_per_clk_sm=out[3], fp32_fma_per_clk_sm=out[4], fp64_add_per_clk_sm=out[5],
                sm_mhz_fp64_fma=out[6], sm_mhz_fp32_fma=out[7], sm_mhz_fp64_add=out[8])


def _nbytes(x):
    if x is None:
        return 0
    if isinstance(x, int):
        raise TypeError("pass work as a tensor so its size is known")
    return x.numel() * x.element_size()


# ------------------------------------------------------------------ host <-> device layout helpers
def alloc_state(grid, device="cuda", n=1):
    """Zeroed device buffer of n states (24 variables, var_stride apart)."""
    import torch
    return torch.zeros(n * NVAR * grid.var_stride, dtype=torch.float64, device=device)


def alloc_work(grid, params, prec=FP64, device="cuda"):
    import torch
    nb = work_bytes(grid, params, prec)
    if nb == 0:
        raise BssnError(ERR_INVALID_ARG, "work_bytes")
    return torch.empty((nb + 7) // 8, dtype=torch.float64, device=device)


def view4(flat, grid, nvar=NVAR):
    """(nvar, nz+2g, ny+2g, nx+2g) view of a flat state buffer."""
    return flat[: nvar * grid.var_stride].view(nvar, grid.var_stride)[:, : grid.npad].view(nvar, *grid.padded)


def upload(state_np, grid, out=None, device="cuda"):
    """Copy a numpy (24, nz+2g, ny+2g, nx+2g) array into a flat device state."""
    import torch
    if out is None:
        out = alloc_state(grid, device)
    view4(out, grid, state_np.shape[0]).copy_(torch.from_numpy(np.ascontiguousarray(state_np)))
    return out


def download(flat, grid, nvar=NVAR):
    return view4(flat, grid, nvar).cpu().numpy()


# ------------------------------------------------------------------ refined hierarchy (Berger-Oliger)
class AmrPatch(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("ox", ctypes.c_int), ("oy", ctypes.c_int), ("oz", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("var_stride", ctypes.c_longlong),
                ("state", ctypes.c_void_p), ("ghost_src", ctypes.c_void_p)]


class AmrDesc(ctypes.Structure):
    _fields_ = [("ncells", ctypes.c_int * 3), ("xlo", ctypes.c_double * 3), ("h0", ctypes.c_double * 3),
                ("ghost", ctypes.c_int), ("boundary", ctypes.c_int), ("dt0", ctypes.c_double)]


def _amr_lib():
    L = lib()
    if not getattr(L, "_amr_typed", False):
        L.bssn_amr_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(AmrPatch), ctypes.c_int,
                                      ctypes.POINTER(AmrDesc), ctypes.POINTER(Params), ctypes.c_int]
        L.bssn_amr_step.argtypes = [_p, _p]
        L.bssn_amr_info.argtypes = [_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int), _p,
                                    ctypes.POINTER(ctypes.c_longlong)]
        L.bssn_amr_destroy.argtypes = [_p]
        L.bssn_sommerfeld_rhs.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params), _p, _p, _p, _p]
        L.bssn_amr_regrid.argtypes = [_p, ctypes.POINTER(AmrPatch), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), _p]
        for n in ("bssn_amr_create", "bssn_amr_step", "bssn_amr_info", "bssn_amr_destroy", "bssn_sommerfeld_rhs",
                  "bssn_amr_regrid"):
            getattr(L, n).restype = ctypes.c_int
        L._amr_typed = True
    return L


def amr_create(patches, ncells, xlo, h0, ghost, boundary, dt0, params, prec=FP64):
    """patches: list of (level, origin (3), n (3), var_stride, state, ghost_src
    or None) with device tensors/addresses. Returns an opaque handle (int)."""
    arr = (AmrPatch * len(patches))(*[AmrPatch(lv, o[0], o[1], o[2], n[0], n[1], n[2], vs, _ptr(s), _ptr(src))
                                      for (lv, o, n, vs, s, src) in patches])
    h0 = (h0,) * 3 if np.isscalar(h0) else tuple(h0)
    d = AmrDesc((ctypes.c_int * 3)(*ncells), (ctypes.c_double * 3)(*xlo), (ctypes.c_double * 3)(*h0), ghost,
                boundary, dt0)
    h = ctypes.c_void_p()
    _check(_amr_lib().bssn_amr_create(ctypes.byref(h), arr, len(patches), ctypes.byref(d), ctypes.byref(params),
                                      prec), "amr_create")
    return h.value


def amr_regrid(amr, patches, stream=None):
    """New hierarchy on `patches` (same tuples as amr_create) filled from
    the hierarchy `amr` at the current time; returns its handle."""
    arr = (AmrPatch * len(patches))(*[AmrPatch(lv, o[0], o[1], o[2], n[0], n[1], n[2], vs, _ptr(s), _ptr(src))
                                      for (lv, o, n, vs, s, src) in patches])
    h = ctypes.c_void_p()
    _check(_amr_lib().bssn_amr_regrid(amr, arr, len(patches), ctypes.byref(h), _stream(stream)), "amr_regrid")
    return h.value


def amr_step(amr, stream=None):
    _check(_amr_lib().bssn_amr_step(amr, _stream(stream)), "amr_step")


def amr_info(amr):
    upd, nodes = ctypes.c_longlong(), ctypes.c_longlong()
    nlev = ctypes.c_int()
    ent = np.zeros(5, dtype=np.int64)
    _check(_amr_lib().bssn_amr_info(amr, ctypes.byref(upd), ctypes.byref(nlev), ent.ctypes.data_as(_p),
                                    ctypes.byref(nodes)), "amr_info")
    return dict(updates_per_step=upd.value, levels=nlev.value, graph_nodes=nodes.value,
                entries=dict(zip(["copy", "prolong", "static", "radiative", "restrict"], (int(x) for x in ent))))


def amr_destroy(amr):
    _check(_amr_lib().bssn_amr_destroy(amr), "amr_destroy")


def sommerfeld_rhs(grid, params, xyz0, state, out, stream=None):
    xyz = np.ascontiguousarray(xyz0, dtype=np.float64)
    _check(_amr_lib().bssn_sommerfeld_rhs(ctypes.byref(grid), ctypes.byref(params), xyz.ctypes.data_as(_p),
                                          _ptr(state), _ptr(out), _stream(stream)), "sommerfeld_rhs")


# ------------------------------------------------------------------ CFD benchmark (SOLA Navier-Stokes)
class CfdDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3), ("periodic", ctypes.c_int * 3),
                ("nu", ctypes.c_double), ("dt", ctypes.c_double), ("omega", ctypes.c_double),
                ("alpha", ctypes.c_double), ("lid", ctypes.c_double), ("g", ctypes.c_double * 3)]


def make_cfd(n, h, periodic, nu, dt, omega=1.7, alpha=0.3, lid=0.0, g=(0.0, 0.0, 0.0)):
    h = (h,) * 3 if np.isscalar(h) else tuple(h)
    return CfdDesc((ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*h), (ctypes.c_int * 3)(*[int(x) for x in periodic]),
                   nu, dt, omega, alpha, lid, (ctypes.c_double * 3)(*g))


def _cfd_lib():
    L = lib()
    if not getattr(L, "_cfd_typed", False):
        D = ctypes.POINTER(CfdDesc)
        L.bssn_cfd_points.argtypes = [D]
        L.bssn_cfd_points.restype = ctypes.c_ulonglong
        L.bssn_cfd_boundary.argtypes = [D, _p, _p, _p, _p, _p]
        L.bssn_cfd_velocity.argtypes = [D, _p, _p, _p, _p, _p, _p, _p, _p]
        L.bssn_cfd_mass.argtypes = [D, ctypes.c_int, _p, _p, _p, _p, _p]
        L.bssn_cfd_step.argtypes = [D, ctypes.c_int, _p, _p, _p, _p, _p, _p]
        L.bssn_cfd_mass_iteration.argtypes = [D, _p, _p, _p, _p, _p, _p, _p, _p]
        for n in ("bssn_cfd_boundary", "bssn_cfd_velocity", "bssn_cfd_mass", "bssn_cfd_mass_iteration",
                  "bssn_cfd_step"):
            getattr(L, n).restype = ctypes.c_int
        L._cfd_typed = True
    return L


def cfd_points(desc):
    return _cfd_lib().bssn_cfd_points(ctypes.byref(desc))


def cfd_boundary(desc, u, v, w, p, stream=None):
    _check(_cfd_lib().bssn_cfd_boundary(ctypes.byref(desc), _ptr(u), _ptr(v), _ptr(w), _ptr(p), _stream(stream)),
           "cfd_boundary")


def cfd_velocity(desc, u, v, w, p, un, vn, wn, stream=None):
    _check(_cfd_lib().bssn_cfd_velocity(ctypes.byref(desc), _ptr(u), _ptr(v), _ptr(w), _ptr(p), _ptr(un), _ptr(vn),
                                        _ptr(wn), _stream(stream)), "cfd_velocity")


def cfd_mass(desc, colour, u, v, w, p, stream=None):
    _check(_cfd_lib().bssn_cfd_mass(ctypes.byref(desc), colour, _ptr(u), _ptr(v), _ptr(w), _ptr(p),
                                    _stream(stream)), "cfd_mass")


def cfd_mass_iteration(desc, u, v, w, un, vn, wn, p, stream=None):
    _check(_cfd_lib().bssn_cfd_mass_iteration(ctypes.byref(desc), _ptr(u), _ptr(v), _ptr(w), _ptr(un), _ptr(vn),
                                              _ptr(wn), _ptr(p), _stream(stream)), "cfd_mass_iteration")


def cfd_step(desc, iterations, u, v, w, p, scratch, stream=None):
    _check(_cfd_lib().bssn_cfd_step(ctypes.byref(desc), iterations, _ptr(u), _ptr(v), _ptr(w), _ptr(p), _ptr(scratch),
                                    _stream(stream)), "cfd_step")
