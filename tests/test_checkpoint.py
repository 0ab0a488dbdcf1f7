"""Checkpoint and resume (bssn_checkpoint_write / bssn_checkpoint_read,
host only): the full padded state with its grid, parameters, time and step
count, and a 64-bit hash of the data. A resumed evolution must continue
from exactly the same bits: checked on the oracle here and on the GPU path
(`-m gpu`)."""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs


@pytest.fixture(scope="module")
def L():
    from paper_1307_6488_gb300 import build
    build.build()
    return B.lib()


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def test_roundtrip_bit_exact(L, tmp_path):
    grid = B.make_grid(5, 4, 3, ghost=2, dx=0.1, dy=0.2, dz=0.3)
    params = B.make_params(fd_order=4, ko_eps=0.07, lapse=1, shift=1, shift_coeff=0.6, eta=1.3, advect_gauge=0)
    rng = np.random.default_rng(1)
    state = rng.normal(size=24 * grid.var_stride)
    state[3] = np.nan
    state[4] = -np.inf
    state[5] = -0.0
    path = tmp_path / "a.ckp"
    B.checkpoint_write(path, grid, params, 1.25, 17, state)
    g2, p2, t, step, s2 = B.checkpoint_read(path)
    assert np.array_equal(_bits(s2), _bits(state))
    assert (t, step) == (1.25, 17)
    for f, _ in B.Grid._fields_:
        assert getattr(g2, f) == getattr(grid, f), f
    for f, _ in B.Params._fields_:
        assert getattr(p2, f) == getattr(params, f), f
    # header only
    g3, _, _, _, none = B.checkpoint_read(path, with_state=False)
    assert none is None and g3.var_stride == grid.var_stride


def test_damaged_files_are_rejected(L, tmp_path):
    grid = B.make_grid(4, ghost=2, dx=0.1)
    params = B.make_params()
    state = np.arange(24 * grid.var_stride, dtype=np.float64)
    good = tmp_path / "good.ckp"
    B.checkpoint_write(good, grid, params, 0.0, 0, state)
    raw = good.read_bytes()
    cases = {
        "flipped data byte": raw[:-100] + bytes([raw[-100] ^ 1]) + raw[-99:],
        "truncated data": raw[:-8],
        "truncated header": raw[:40],
        "foreign magic": b"XSSNCKP1" + raw[8:],
        "other version": raw[:12] + (2).to_bytes(4, "little") + raw[16:],
        "empty": b"",
    }
    for name, blob in cases.items():
        p = tmp_path / (name.replace(" ", "_") + ".ckp")
        p.write_bytes(blob)
        with pytest.raises(B.BssnError) as e:
            B.checkpoint_read(p)
        assert e.value.status == B.ERR_INVALID_ARG, name
    with pytest.raises(B.BssnError):
        B.checkpoint_read(tmp_path / "missing.ckp")


def test_invalid_arguments(L, tmp_path):
    grid = B.make_grid(4, ghost=2, dx=0.1)
    params = B.make_params()
    state = np.zeros(24 * grid.var_stride)
    G, P = ctypes.byref, ctypes.byref
    B.checkpoint_write(tmp_path / "x.ckp", grid, params, 0.0, 0, state)
    E = B.ERR_INVALID_ARG
    ptr = state.ctypes.data_as(ctypes.c_void_p)
    assert L.bssn_checkpoint_write(None, G(grid), P(params), 0.0, 0, ptr) == E
    assert L.bssn_checkpoint_write(os.fsencode(tmp_path / "y.ckp"), G(grid), P(params), float("nan"), 0, ptr) == E
    bad = B.Grid(4, 4, 4, 2, 0.1, 0.1, 0.1, 10)  # var_stride below the padded size
    assert L.bssn_checkpoint_write(os.fsencode(tmp_path / "y.ckp"), G(bad), P(params), 0.0, 0, ptr) == E
    g2, p2 = B.Grid(), B.Params()
    t, step = ctypes.c_double(), ctypes.c_longlong()
    small = np.zeros(10)
    assert L.bssn_checkpoint_read(os.fsencode(tmp_path / "x.ckp"), G(g2), P(p2), ctypes.byref(t), ctypes.byref(step),
                                  small.ctypes.data_as(ctypes.c_void_p), small.size) == E
    assert L.bssn_checkpoint_read(os.fsencode(tmp_path / "x.ckp"), None, P(p2), ctypes.byref(t), ctypes.byref(step),
                                  None, 0) == E
    with pytest.raises(B.BssnError):
        B.checkpoint_write(tmp_path / "z.ckp", grid, params, 0.0, 0, state[:10])


def _flat(u, grid):
    f = np.zeros(24 * grid.var_stride)
    f.reshape(24, grid.var_stride)[:, :grid.npad] = u.reshape(24, -1)
    return f


def _unflat(f, grid):
    return np.ascontiguousarray(f.reshape(24, grid.var_stride)[:, :grid.npad].reshape(24, *grid.padded))


def test_resume_on_the_oracle_is_bit_identical(L, tmp_path):
    """Three oracle RK4 steps straight, and two, a checkpoint, a read and one
    more: the same bits."""
    u, h = inputs.gauge_wave(12, 3, amplitude=0.05, noise=1e-10)
    grid = B.make_grid(12, ghost=3, dx=h)
    p = oracle.Params(fd_order=4, ko_eps=0.1)
    dt = 0.25 * h
    straight = u
    for _ in range(3):
        straight = oracle.rk4_step(straight, 3, h, dt, p, bc=0)
    y = u
    for _ in range(2):
        y = oracle.rk4_step(y, 3, h, dt, p, bc=0)
    path = tmp_path / "gw.ckp"
    B.checkpoint_write(path, grid, B.make_params(fd_order=4, ko_eps=0.1), 2 * dt, 2, _flat(y, grid))
    g2, p2, t, step, f = B.checkpoint_read(path)
    assert step == 2 and t == 2 * dt and p2.fd_order == 4
    resumed = oracle.rk4_step(_unflat(f, g2), 3, g2.dx, dt, p, bc=0)
    assert np.array_equal(_bits(resumed), _bits(straight))


@pytest.mark.gpu
def test_resume_on_the_gpu_is_bit_identical(L, tmp_path):
    """The GPU path: two RK4 steps, the state copied to the host and written,
    read back and uploaded, one more step - the same bits as three steps
    straight (24^3 gauge wave, periodic)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    u, h = inputs.gauge_wave(24, 3, amplitude=0.01, noise=1e-10, seed=1307)
    grid = B.make_grid(24, ghost=3, dx=h)
    p = B.make_params(fd_order=4)
    dt = 0.25 * h
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p)
    a = B.upload(u, grid)
    b = B.upload(u, grid)
    for _ in range(3):
        B.rk4_step(grid, p, B.FP64, dt, 0, None, a, bufs, work)
    for _ in range(2):
        B.rk4_step(grid, p, B.FP64, dt, 0, None, b, bufs, work)
    torch.cuda.synchronize()
    path = tmp_path / "gpu.ckp"
    B.checkpoint_write(path, grid, p, 2 * dt, 2, b.cpu().numpy())
    g2, p2, t, step, f = B.checkpoint_read(path)
    c = torch.from_numpy(f).to("cuda")
    B.rk4_step(g2, p2, B.FP64, dt, 0, None, c, bufs, work)
    torch.cuda.synchronize()
    assert torch.equal(a, c)
