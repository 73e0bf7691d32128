"""The binary64 <-> binary32 conversions that the FP32 form performs with
integer operations (the conversion instructions issue on GB300's FP64 pipe).

The reference is numpy's own conversion (IEEE 754 round to nearest, ties to
even; widening is exact), so the check is independent of the CUDA path.
The values cover random magnitudes across and beyond the binary32 range,
exact ties and the values next to them, the binade edges where rounding
carries into the exponent, the overflow threshold, subnormal results,
zeros of both signs, infinities and NaNs.  Bit patterns must agree.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2510_25702_gb300 import build
    from paper_2510_25702_gb300 import sph as S

    build.build()
    return S


def _doubles(rng):
    out = []
    # random bit patterns over the whole exponent range of binary32 and a
    # margin on both sides
    e = rng.integers(1023 - 160, 1023 + 140, 200_000, dtype=np.uint64)
    f = rng.integers(0, 1 << 52, 200_000, dtype=np.uint64)
    s = rng.integers(0, 2, 200_000, dtype=np.uint64)
    out.append(((s << np.uint64(63)) | (e << np.uint64(52)) | f).view(np.float64))
    # ties: fraction bit 28 set, bits 0..27 clear, even and odd kept parts
    # (and one unit below / above the tie)
    e = rng.integers(1023 - 126, 1023 + 128, 50_000, dtype=np.uint64)
    keep = rng.integers(0, 1 << 23, 50_000, dtype=np.uint64)
    tie = (e << np.uint64(52)) | (keep << np.uint64(29)) | np.uint64(1 << 28)
    one = np.uint64(1)
    out += [tie.view(np.float64), (tie + one).view(np.float64), (tie - one).view(np.float64)]
    # all-ones kept fractions: rounding carries into the exponent
    e = np.arange(1023 - 127, 1023 + 129, dtype=np.uint64)
    ones = (e << np.uint64(52)) | np.uint64(((1 << 23) - 1) << 29)
    for extra in (np.uint64(1 << 28), np.uint64((1 << 28) + 1), np.uint64((1 << 28) - 1)):
        out.append((ones | extra).view(np.float64))
    # special values
    f32max = float(np.finfo(np.float32).max)
    out.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, f32max, -f32max,
                         np.nextafter(f32max, np.inf), 3.4028235677973366e38, 3.4028235677973362e38,
                         2.0 ** 128, 1e300, -1e300, 2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 2.0 ** -150,
                         1.5 * 2.0 ** -149, 1e-300, 5e-324, 0.005, 1000.0, 6.0, 1.3e-3], np.float64))
    return np.concatenate(out)


def _floats(rng):
    u = rng.integers(0, 1 << 32, 300_000, dtype=np.uint64).astype(np.uint32)
    extra = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38, 3.4028235e38,
                      1.0, 0.005], np.float32)
    return np.concatenate([u.view(np.float32), extra])


def test_conversions_match_ieee_round_to_nearest(sph):
    rng = np.random.default_rng(20251029)
    x64 = _doubles(rng)
    x32 = _floats(rng)
    n = max(x64.size, x32.size)
    x64 = np.resize(x64, n)
    x32 = np.resize(x32, n)
    with np.errstate(over="ignore", invalid="ignore"):
        want32 = x64.astype(np.float32)
        want64 = x32.astype(np.float64)
    got32, got64 = sph.debug_convert(x64, x32)
    nan32 = np.isnan(want32)
    assert np.array_equal(np.isnan(got32), nan32)
    bad = np.flatnonzero(got32.view(np.uint32)[~nan32] != want32.view(np.uint32)[~nan32])
    assert bad.size == 0, f"{bad.size} binary64->binary32 mismatches, first input {x64[~nan32][bad[0]]!r}"
    nan64 = np.isnan(want64)
    assert np.array_equal(np.isnan(got64), nan64)
    bad = np.flatnonzero(got64.view(np.uint64)[~nan64] != want64.view(np.uint64)[~nan64])
    assert bad.size == 0, f"{bad.size} binary32->binary64 mismatches, first input {x32[~nan64][bad[0]]!r}"
