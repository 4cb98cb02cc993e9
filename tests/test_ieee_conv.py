"""The integer IEEE-754 conversions of the mixed-precision kernels (csrc/ieee_conv.cuh),
compiled for the host with g++ and checked bit for bit against numpy's conversions, which
round to nearest, ties to even, with subnormals and overflow to infinity. The device
compiles the same source.

Cases: every positive FP32 subnormal and a random sample of all FP32 bit patterns (FP32 ->
FP64); for float(v * 2^k): random values whose scaled exponent spans zero, subnormal,
normal and overflowing results, exact ties in the normal and the subnormal range, FP64
subnormal inputs, signed zeros, infinities and NaNs."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2512_09642_gb300", "csrc", "ieee_conv.cuh")

DRIVER = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include "ieee_conv.cuh"
int main(int argc, char** argv) {
    FILE* f = std::fopen(argv[1], "rb");
    FILE* o = std::fopen(argv[2], "wb");
    long long n32 = 0, n64 = 0;
    if (std::fread(&n32, 8, 1, f) != 1 || std::fread(&n64, 8, 1, f) != 1) return 1;
    std::vector<uint32_t> a(n32), k(n64);
    std::vector<uint64_t> b(n64), ra(n32);
    std::vector<uint32_t> rb(n64);
    if (std::fread(a.data(), 4, n32, f) != (size_t)n32 || std::fread(b.data(), 8, n64, f) != (size_t)n64 ||
        std::fread(k.data(), 4, n64, f) != (size_t)n64) return 2;
    for (long long i = 0; i < n32; ++i) ra[i] = sstep::f32_to_f64_bits(a[i]);
    for (long long i = 0; i < n64; ++i) rb[i] = sstep::f64_to_f32_scaled_bits(b[i], (int)(int32_t)k[i]);
    std::fwrite(ra.data(), 8, n32, o);
    std::fwrite(rb.data(), 4, n64, o);
    std::fclose(o);
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("ieee")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return d, exe


def _run(driver, a32, b64, k):
    d, exe = driver
    inp, out = d / "in.bin", d / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.array([a32.size, b64.size], dtype=np.int64).tobytes())
        f.write(a32.astype(np.uint32).tobytes())
        f.write(b64.astype(np.uint64).tobytes())
        f.write(k.astype(np.int32).tobytes())
    subprocess.run([str(exe), str(inp), str(out)], check=True)
    raw = np.fromfile(out, dtype=np.uint8)
    ra = raw[:8 * a32.size].view(np.uint64)
    rb = raw[8 * a32.size:].view(np.uint32)
    return ra, rb


def _f32_cases(rng):
    sub = np.arange(1, 1 << 23, dtype=np.uint32)                  # every positive subnormal
    special = np.array([0, 0x80000000, 0x00800000, 0x3F800000, 0x7F7FFFFF, 0xFF7FFFFF, 0x7F800000,
                        0xFF800000, 0x7FC00000, 0x7FC12345, 0x7F800001, 0xFFFFFFFF, 0x807FFFFF], dtype=np.uint32)
    rand = rng.integers(0, 1 << 32, size=2_000_000, dtype=np.uint64).astype(np.uint32)
    return np.concatenate([sub, sub | np.uint32(0x80000000), special, rand])


def _f64_cases(rng):
    n = 1_000_000
    sign = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    mant = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    ex = rng.integers(1, 2047, n, dtype=np.uint64)                 # normal FP64 inputs
    bits = sign | (ex << np.uint64(52)) | mant
    E = ex.astype(np.int64) - 1023
    k = rng.integers(-200, 161, n) - E                             # scaled exponent in [-200, 160]
    # exact ties: rest = 2^28 (normal range) with even and odd kept mantissas
    nt = 200_000
    mt = (rng.integers(0, 1 << 23, nt, dtype=np.uint64) << np.uint64(29)) | np.uint64(1 << 28)
    et = rng.integers(1, 2047, nt, dtype=np.uint64)
    bt = (rng.integers(0, 2, nt, dtype=np.uint64) << np.uint64(63)) | (et << np.uint64(52)) | mt
    kt = rng.integers(-126, 128, nt) - (et.astype(np.int64) - 1023)
    # subnormal results with exact ties: keep the top q bits of M and set the next bit only
    ns = 200_000
    s = rng.integers(30, 54, ns)
    msub = rng.integers(0, 1 << 52, ns, dtype=np.uint64)
    lowmask = (np.uint64(1) << s.astype(np.uint64)) - np.uint64(1)
    half = np.uint64(1) << (s - 1).astype(np.uint64)
    tie = rng.integers(0, 2, ns).astype(bool)
    msub = np.where(tie, (msub & ~lowmask) | half, msub) & np.uint64((1 << 52) - 1)
    es = -(s + 97)                                                 # the scaled exponent that gives shift s
    eb = rng.integers(1, 2047, ns, dtype=np.uint64)
    bs = (rng.integers(0, 2, ns, dtype=np.uint64) << np.uint64(63)) | (eb << np.uint64(52)) | msub
    ks = es - (eb.astype(np.int64) - 1023)
    # FP64 subnormal inputs scaled into the FP32 range
    nd = 100_000
    bd = rng.integers(1, 1 << 52, nd, dtype=np.uint64) | (rng.integers(0, 2, nd, dtype=np.uint64) << np.uint64(63))
    kd = rng.integers(900, 1250, nd)
    special = np.array([0, 1 << 63, 0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000000,
                        0x7FF0000000000001, 0x7FEFFFFFFFFFFFFF, 0x0000000000000001, 0x3FF0000000000000,
                        0x47EFFFFFE0000000, 0x47EFFFFFF0000000, 0x47EFFFFFEFFFFFFF, 0x380FFFFFF0000000],
                       dtype=np.uint64)
    kspec = np.zeros(special.size, dtype=np.int64)
    return (np.concatenate([bits, bt, bs, bd, special]),
            np.concatenate([k, kt, ks, kd, kspec]))


def test_integer_conversions_match_ieee(driver):
    rng = np.random.default_rng(20251209)
    a32 = _f32_cases(rng)
    b64, k = _f64_cases(rng)
    ra, rb = _run(driver, a32, b64, k)

    # FP32 -> FP64: exact
    fa = a32.view(np.float32)
    nan_a = np.isnan(fa)
    with np.errstate(invalid="ignore"):
        want_a = fa.astype(np.float64).view(np.uint64)
    assert np.array_equal(ra[~nan_a], want_a[~nan_a])
    assert np.all(np.isnan(ra[nan_a].view(np.float64)))

    # float(v * 2^k): the scaled value is exact in FP64 for these exponents, so numpy's
    # FP64 -> FP32 cast gives the correctly rounded reference
    v = b64.view(np.float64)
    with np.errstate(over="ignore", invalid="ignore"):
        want_b = np.ldexp(v, k).astype(np.float32)
    nan_b = np.isnan(v)
    assert np.array_equal(rb[~nan_b], want_b.view(np.uint32)[~nan_b])
    assert np.all(np.isnan(rb[nan_b].view(np.float32)))
    # the cases reach every result class
    got = rb[~nan_b].view(np.float32)
    assert np.any(got == 0) and np.any(np.isinf(got))
    tiny = np.abs(got)[(got != 0) & np.isfinite(got)]
    assert np.any(tiny < np.finfo(np.float32).tiny) and np.any(tiny >= np.finfo(np.float32).tiny)
