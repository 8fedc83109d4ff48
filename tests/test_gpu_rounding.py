"""The split path's FP64 -> FP32 rounding (integer-pipe round to nearest, ties to even) against IEEE 754
conversion: numpy's on the host and CUDA's own (torch) on the device, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _cases():
    rng = np.random.default_rng(7)
    f32 = np.finfo(np.float32)
    parts = [
        # normal range, random exponents and signs
        rng.standard_normal(20000) * np.exp2(rng.integers(-120, 120, 20000)),
        # subnormal FP32 results and the boundaries around them
        rng.uniform(-1, 1, 20000) * np.exp2(rng.integers(-152, -124, 20000)),
        np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324, 2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -151,
                  2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -25), float(f32.max), -float(f32.max), 2.0 ** 128,
                  float(f32.max) * (1 + 2.0 ** -25), float(f32.max) * (1 + 2.0 ** -26), 1e300, -1e300]),
    ]
    # exact ties between neighbouring floats (normal and subnormal), both parities
    f = (rng.standard_normal(20000) * np.exp2(rng.integers(-140, 120, 20000))).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    ok = np.isfinite(g)
    parts.append((f[ok].astype(np.float64) + g[ok].astype(np.float64)) / 2)
    # one unit in the last double place on either side of a tie
    mid = parts[-1][:5000]
    parts.append(np.nextafter(mid, np.inf))
    parts.append(np.nextafter(mid, -np.inf))
    return np.concatenate(parts)


@pytest.mark.gpu
def test_round_f32_matches_ieee_and_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08830_gb300 import _lib, build
    build.build()
    L = _lib.lib()
    x = _cases()
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    assert L.tufrg_round_f32(xd.data_ptr(), out.data_ptr(), x.size, None) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.array_equal(got.view(np.uint32), xd.float().cpu().numpy().view(np.uint32))
    # NaN stays NaN (payload not compared)
    nan = torch.tensor([np.nan, -np.nan], dtype=torch.float64, device="cuda")
    o2 = torch.empty(2, dtype=torch.float32, device="cuda")
    assert L.tufrg_round_f32(nan.data_ptr(), o2.data_ptr(), 2, None) == 0
    assert torch.isnan(o2).all()
    assert L.tufrg_round_f32(None, None, 0, None) == 0


@pytest.mark.gpu
def test_widen_f64_is_exact():
    """FP32 -> FP64 on the integer pipe: bit for bit numpy's (IEEE) widening over normal values, every subnormal
    exponent, signed zeros and infinities, and NaNs with their payloads kept."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08830_gb300 import _lib, build
    build.build()
    L = _lib.lib()
    rng = np.random.default_rng(11)
    bits = np.concatenate([
        rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32),            # every class, random
        (rng.integers(1, 2 ** 23, 20000, dtype=np.uint64) | (rng.integers(0, 2, 20000, dtype=np.uint64) << 31)
         ).astype(np.uint32),                                                          # subnormals of both signs
        np.array([0, 1 << 31, 1, (1 << 31) | 1, 0x7fffff, 0x800000, 0x7f800000, 0xff800000, 0x7fc00000,
                  0x7f800001, 0xffbfffff, 0x7f7fffff], dtype=np.uint32)])
    x = bits.view(np.float32)
    xd = torch.from_numpy(x.copy()).cuda()
    out = torch.empty(x.size, dtype=torch.float64, device="cuda")
    assert L.tufrg_widen_f64(xd.data_ptr(), out.data_ptr(), x.size, None) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    fin = ~np.isnan(x)
    want = x[fin].astype(np.float64)
    assert np.array_equal(got[fin].view(np.uint64), want.view(np.uint64))
    # NaN: sign and the 22 payload bits below the quiet bit kept in the top of the FP64 significand
    nb = got[~fin].view(np.uint64)
    src = bits[~fin].astype(np.uint64)
    assert np.all(np.isnan(got[~fin]))
    assert np.array_equal(nb >> np.uint64(63), src >> np.uint64(31))
    assert np.array_equal((nb >> np.uint64(29)) & np.uint64(0x7fffff), src & np.uint64(0x7fffff))
    assert L.tufrg_widen_f64(None, None, 0, None) == 0
