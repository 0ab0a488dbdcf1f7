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
    grid = B.make_grid(5, 4, 3, ghost=3, dx=0.1, dy=0.2, dz=0.3)
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
    grid = B.make_grid(4, ghost=3, dx=0.1)
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
    grid = B.make_grid(4, ghost=3, dx=0.1)
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
    # parameters the stepping entry points would reject
    for bad_p in (B.make_params(fd_order=6), B.make_params(fd_order=8), B.make_params(lapse=3),
                  B.make_params(ko_eps=float("nan"))):
        with pytest.raises(B.BssnError) as e:
            B.checkpoint_write(tmp_path / "w.ckp", grid, bad_p, 0.0, 0, state)
        assert e.value.status == E
    assert not (tmp_path / "w.ckp").exists()


# byte offsets of header fields (the layout bssn_checkpoint.cu writes)
OFF = dict(ghost=28, order=64, eps=68, lapse=76, shift=80, coeff=84, eta=92, adv=100, t=104)


def test_damaged_parameters_are_rejected(L, tmp_path):
    """A file whose parameters no stepping entry point would accept is
    rejected on reading, one damaged field at a time (the data hash does not
    cover the header, so only this check can catch it)."""
    import struct
    grid = B.make_grid(6, ghost=5, dx=0.1)
    params = B.make_params(fd_order=8)
    state = np.zeros(24 * grid.var_stride)
    good = tmp_path / "good.ckp"
    B.checkpoint_write(good, grid, params, 0.5, 3, state)
    raw = bytearray(good.read_bytes())
    B.checkpoint_read(good)  # the untouched file reads

    def patched(off, fmt, value):
        b = bytearray(raw)
        struct.pack_into(fmt, b, off, value)
        return bytes(b)

    cases = {
        "order 6": patched(OFF["order"], "<i", 6),
        "order 4 is fine but ghost 2 is too small": patched(OFF["ghost"], "<i", 2),
        "lapse 3": patched(OFF["lapse"], "<i", 3),
        "shift -1": patched(OFF["shift"], "<i", -1),
        "advect_gauge 2": patched(OFF["adv"], "<i", 2),
        "ko_eps nan": patched(OFF["eps"], "<d", float("nan")),
        "ko_eps negative": patched(OFF["eps"], "<d", -0.1),
        "eta inf": patched(OFF["eta"], "<d", float("inf")),
        "shift_coeff nan": patched(OFF["coeff"], "<d", float("nan")),
        "t nan": patched(OFF["t"], "<d", float("nan")),
    }
    for name, blob in cases.items():
        p = tmp_path / "bad.ckp"
        p.write_bytes(blob)
        with pytest.raises(B.BssnError) as e:
            B.checkpoint_read(p, with_state=False)
        assert e.value.status == B.ERR_INVALID_ARG, name


def test_failed_write_keeps_the_previous_checkpoint(L, tmp_path):
    """The file is written under a temporary name and renamed only when every
    write succeeded: with the temporary name taken by a directory, the write
    fails and the checkpoint already at the path still reads back intact."""
    grid = B.make_grid(4, ghost=3, dx=0.1)
    params = B.make_params()
    old = np.arange(24 * grid.var_stride, dtype=np.float64)
    path = tmp_path / "run.ckp"
    B.checkpoint_write(path, grid, params, 1.0, 10, old)
    (tmp_path / ("run.ckp.tmp%d" % os.getpid())).mkdir()
    with pytest.raises(B.BssnError):
        B.checkpoint_write(path, grid, params, 2.0, 20, old + 1)
    _, _, t, step, s2 = B.checkpoint_read(path)
    assert (t, step) == (1.0, 10)
    assert np.array_equal(s2, old)
    # no stray files besides the blocked temporary name
    assert sorted(f.name for f in tmp_path.iterdir()) == ["run.ckp", "run.ckp.tmp%d" % os.getpid()]


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


@pytest.mark.gpu
def test_resume_with_a_static_boundary_on_the_gpu(L, tmp_path):
    """A static-boundary run (fill mode 1) resumed from its checkpoint: the
    ghost cells keep their t = 0 values and are part of the saved state, so a
    copy of the loaded state serves as ghost_src. Two FP64 RK4 steps of
    Brill-Lindquist data at 8th order, a checkpoint, one more step: the same
    bits as three steps straight."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    u, h = inputs.brill_lindquist(20, 5, lo=-2.5, hi=2.5, masses=(0.5, 0.5), centers=((-0.7, 0.1, 0.05),
                                                                                    (0.7, -0.1, 0.05)))
    grid = B.make_grid(20, ghost=5, dx=h)
    p = B.make_params(fd_order=8)
    dt = 0.25 * h
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p)
    src = B.upload(u, grid)
    a = B.upload(u, grid)
    b = B.upload(u, grid)
    for _ in range(3):
        B.rk4_step(grid, p, B.FP64, dt, 1, src, a, bufs, work)
    for _ in range(2):
        B.rk4_step(grid, p, B.FP64, dt, 1, src, b, bufs, work)
    torch.cuda.synchronize()
    path = tmp_path / "bl.ckp"
    B.checkpoint_write(path, grid, p, 2 * dt, 2, b.cpu().numpy())
    del b
    g2, p2, t, step, f = B.checkpoint_read(path)
    c = torch.from_numpy(f).to("cuda")
    ghost_src = c.clone()
    B.rk4_step(g2, p2, B.FP64, dt, 1, ghost_src, c, bufs, work)
    torch.cuda.synchronize()
    assert torch.equal(a, c)
