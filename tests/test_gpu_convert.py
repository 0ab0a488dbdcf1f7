"""The FP32-RHS kernels convert between single and double precision on the
integer pipes (bssn_cvt.cuh). Those conversions must equal the hardware
instructions bit for bit on every kind of input: normal numbers across the
whole exponent range, exact ties of round-to-nearest-even, results that are
subnormal, overflow to infinity, zeros of both signs, infinities and NaNs."""
import numpy as np
import pytest

from paper_1307_6488_gb300 import binding as B

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _doubles(rng, n):
    bits = rng.integers(0, 2 ** 64, size=n, dtype=np.uint64)
    d = bits.view(np.float64).copy()
    # exponents near the single-precision range, where the field move applies
    e = rng.integers(1023 - 160, 1023 + 140, size=n).astype(np.uint64)
    near = (bits & np.uint64(0x800FFFFFFFFFFFFF)) | (e << np.uint64(52))
    # exact ties and near-ties of the 29 dropped bits
    tie = (near & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000000)
    tie_m = tie - np.uint64(1)
    tie_p = tie + np.uint64(1)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0 ** -126, 2.0 ** -127, 2.0 ** -149,
                         2.0 ** -150, 2.0 ** -151, 3.0 * 2.0 ** -151, 2.0 ** 127, 2.0 ** 128,
                         np.float64(np.finfo(np.float32).max), np.float64(np.finfo(np.float32).max) * (1 + 2 ** -25),
                         np.float64(np.finfo(np.float32).max) * (1 + 2 ** -24), 1e-300, -1e300, 5e-324])
    return np.concatenate([d, near.view(np.float64), tie.view(np.float64), tie_m.view(np.float64),
                           tie_p.view(np.float64), specials])


def _floats(rng, n):
    bits = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, 1e-45, -1e-45, 1.1754942e-38, 1.17549435e-38,
                         3.4028235e38], dtype=np.float32)
    return np.concatenate([bits.view(np.float32), specials])


def test_conversions_equal_the_hardware_bit_for_bit():
    torch = need_gpu()
    rng = np.random.default_rng(2024)
    d = _doubles(rng, 1 << 18)
    f = _floats(rng, d.size)
    f = np.resize(f, d.size)
    f[-11:] = _floats(rng, 0)
    din = torch.from_numpy(d).cuda()
    fin = torch.from_numpy(f).cuda()
    fb, fh = torch.empty_like(fin), torch.empty_like(fin)
    db, dh = torch.empty_like(din), torch.empty_like(din)
    B.test_conversions(din, fin, fb, fh, db, dh)
    torch.cuda.synchronize()
    fb, fh = fb.cpu().numpy().view(np.uint32), fh.cpu().numpy().view(np.uint32)
    db, dh = db.cpu().numpy().view(np.uint64), dh.cpu().numpy().view(np.uint64)
    bad = np.nonzero(fb != fh)[0]
    assert bad.size == 0, [(d[i], hex(fb[i]), hex(fh[i])) for i in bad[:5]]
    bad = np.nonzero(db != dh)[0]
    assert bad.size == 0, [(f[i], hex(db[i]), hex(dh[i])) for i in bad[:5]]
    # and the hardware agrees with numpy's IEEE rounding on the finite inputs
    fin_ok = np.isfinite(d) & (np.abs(d) < 3.5e38)
    assert np.array_equal(fh[fin_ok], d[fin_ok].astype(np.float32).view(np.uint32))
