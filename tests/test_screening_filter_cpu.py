"""CPU checks of two pieces of arithmetic the FP32 tier relies on, restated
in numpy with explicit FP32 rounding (the device code is in
csrc/jk_kernels.cuh: jk_screen_bound / jk_near and jk_to_f64).

1. The screening rule of Sec. 2 (keep a quartet iff Q_ab Q_cd Dmax exceeds a
   threshold) is decided from FP32 images of Q and Dmax; only bounds within
   2e-6 (relative) of the threshold are compared again in FP64. Five FP32
   roundings separate the FP32 product from the FP64 one (at most 3.0e-7),
   so every decision equals the FP64 rule's.
2. The bit-level float-to-double widening (option widen_int) is exact.
"""
import struct

import numpy as np

F = np.float32


def _rule64(qa, qb, dm, t):
    return (qa * qb) * dm > t


def _filtered(qa, qb, dm, t):
    b32 = F(F(F(qa) * F(qb)) * F(dm))
    t32 = F(t)
    if abs(float(b32) - float(t32)) < 2e-6 * float(t32):
        return _rule64(qa, qb, dm, t)
    return bool(b32 > t32)


def test_filtered_fp32_screening_equals_the_fp64_rule():
    rng = np.random.default_rng(12)
    mismatches = 0
    rechecked = 0
    plain32_wrong = 0
    n = 0
    for t in (1e-13, 1e-4, 1e-2, 3.7e-9):
        # random bounds over many decades, and bounds placed within a few
        # FP32 ulps of the threshold (the adversarial cases)
        qa = np.exp(rng.uniform(np.log(1e-9), np.log(10.0), 4000))
        qb = np.exp(rng.uniform(np.log(1e-9), np.log(10.0), 4000))
        dm = np.exp(rng.uniform(np.log(1e-6), np.log(1.0), 4000))
        near_dm = t / (qa * qb) * (1.0 + rng.uniform(-1e-6, 1e-6, 4000))
        for a, b, d in list(zip(qa, qb, dm)) + list(zip(qa, qb, near_dm)):
            if not (1e-30 < d < 1e30):
                continue
            n += 1
            b32 = F(F(F(a) * F(b)) * F(d))
            rechecked += abs(float(b32) - float(F(t))) < 2e-6 * float(F(t))
            mismatches += _filtered(a, b, d, t) != _rule64(a, b, d, t)
            plain32_wrong += bool(b32 > F(t)) != _rule64(a, b, d, t)
    assert n > 20000 and mismatches == 0
    # without the recheck, plain FP32 compares do flip some decisions
    assert plain32_wrong > 0
    # the FP64 recheck is taken only for the near-threshold half
    assert 0 < rechecked < 0.6 * n


def test_fp32_product_error_is_below_the_filter_margin():
    rng = np.random.default_rng(13)
    qa = np.exp(rng.uniform(np.log(1e-9), np.log(10.0), 100000))
    qb = np.exp(rng.uniform(np.log(1e-9), np.log(10.0), 100000))
    dm = np.exp(rng.uniform(np.log(1e-6), np.log(1.0), 100000))
    b64 = (qa * qb) * dm
    b32 = (qa.astype(F) * qb.astype(F)).astype(F) * dm.astype(F)
    rel = np.abs(b32.astype(np.float64) / b64 - 1.0)
    assert rel.max() <= 5 * 2.0 ** -24   # five roundings, below the 2e-6 margin


def _widen(x32):
    """float -> double bit pattern, as jk_to_f64 builds it."""
    u = struct.unpack("<I", struct.pack("<f", x32))[0]
    sgn = (u & 0x80000000) << 32
    e, m = (u >> 23) & 0xFF, u & 0x7FFFFF
    if e == 0xFF:
        bits = sgn | (0x7FF << 52) | (m << 29)
    elif e:
        bits = sgn | ((e + 896) << 52) | (m << 29)
    elif m == 0:
        bits = sgn
    else:
        top = m.bit_length() - 1
        bits = sgn | ((top + 874) << 52) | ((m << (52 - top)) & 0xFFFFFFFFFFFFF)
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def test_bit_level_widening_is_exact():
    rng = np.random.default_rng(14)
    xs = np.concatenate([rng.standard_normal(20000),
                         rng.standard_normal(20000) * 1e-40,          # subnormal floats
                         np.exp(rng.uniform(-100, 88, 20000))]).astype(F)
    xs = np.concatenate([xs, np.array([0.0, -0.0, 1e-45, -1e-45, 1.1754942e-38, 3.4e38, np.inf, -np.inf], F)])
    for x in xs:
        got = _widen(float(x))
        ref = float(np.float64(x))
        assert got == ref and np.signbit(got) == np.signbit(ref)
