"""Checks of the Rys roots/weights tables the kernels interpolate from.

The defining property (eq:rys1 of the paper; the Rys rule in u = t^2 is the
Gauss rule of the measure exp(-T u) / (2 sqrt u) on [0, 1]) is moment
exactness: sum_r W_r u_r^n = F_n(T) for n < 2N. The limits are textbook
rules: at T = 0 the positive nodes of Gauss-Legendre(2N) (squared), at large
T the positive nodes of Gauss-Hermite(2N) scaled by 1/T.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_2507_09772_gb300 import rys_gen


@pytest.fixture(scope="module")
def tables():
    return rys_gen.fit_tables(rys_gen.FP64_FIT, nmax=rys_gen.NMAX)


def boys_quad(n, T):
    v, _ = integrate.quad(lambda t: t ** (2 * n) * math.exp(-T * t * t), 0, 1, epsabs=0, epsrel=1e-13,
                          limit=200)
    return v


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 8, 9])
@pytest.mark.parametrize("T", [0.0, 0.37, 2.9, 11.2, 27.5, 39.9, 50.2, 80.0, 91.5, 300.0])
def test_moment_exactness_of_interpolated_rule(tables, N, T):
    tab, params = tables
    u, W = rys_gen.evaluate(tab, params[N - 1], T)
    for n in range(2 * N):
        ref = boys_quad(n, T) if T > 0 else 1.0 / (2 * n + 1)
        got = float(np.sum(W * u ** n))
        assert got == pytest.approx(ref, rel=5e-13), (N, T, n)


@pytest.mark.parametrize("N", range(1, rys_gen.NMAX + 1))
def test_zero_T_limit_is_gauss_legendre(tables, N):
    tab, params = tables
    u, W = rys_gen.evaluate(tab, params[N - 1], 0.0)
    x, w = special.roots_legendre(2 * N)
    pos = x > 0
    assert np.allclose(np.sort(u), np.sort(x[pos] ** 2), rtol=1e-13, atol=0)
    assert np.allclose(W[np.argsort(u)], w[pos][np.argsort(x[pos] ** 2)], rtol=1e-13, atol=0)


@pytest.mark.parametrize("N", range(1, rys_gen.NMAX + 1))
def test_large_T_limit_is_gauss_hermite(tables, N):
    tab, params = tables
    T = 500.0
    u, W = rys_gen.evaluate(tab, params[N - 1], T)
    x, w = special.roots_hermite(2 * N)
    pos = x > 0
    assert np.allclose(np.sort(u), np.sort(x[pos] ** 2 / T), rtol=1e-13, atol=0)
    assert np.allclose(np.sort(W), np.sort(w[pos] / math.sqrt(T)), rtol=1e-13, atol=0)


@pytest.mark.parametrize("N", [2, 4, 7, 8, 9])
def test_interpolation_matches_exact_rule_across_intervals(tables, N):
    tab, params = tables
    rng = np.random.default_rng(N)
    for T in rng.uniform(0, params[N - 1]["tmax"], 60):
        ue, We = rys_gen.rys_exact(N, T)
        u, W = rys_gen.evaluate(tab, params[N - 1], T)
        assert np.max(np.abs(u / ue - 1)) < 5e-14
        assert np.max(np.abs(W / We - 1)) < 5e-14


def test_fp32_tables_are_accurate_to_single_precision():
    tab, params = rys_gen.fit_tables(rys_gen.FP32_FIT, nmax=rys_gen.NMAX)
    rng = np.random.default_rng(0)
    for N in range(1, rys_gen.NMAX + 1):
        for T in rng.uniform(0, params[N - 1]["tmax"], 30):
            ue, We = rys_gen.rys_exact(N, T)
            u, W = rys_gen.evaluate(tab, params[N - 1], T)
            assert np.max(np.abs(u / ue - 1)) < 2e-6
            assert np.max(np.abs(W / We - 1)) < 2e-6


@pytest.mark.parametrize("N", [1, 2, 4, 7, 9])
def test_split_precision_evaluation_matches_exact_rule(tables, N):
    """The FP64 tier's layout: FP64 head c0..c5, FP32 tail c6..c9."""
    tab, params = tables
    packed = rys_gen.pack_split(tab, params)
    rng = np.random.default_rng(10 + N)
    for T in np.concatenate([rng.uniform(0, params[N - 1]["tmax"], 60), [0.0, 1e-7]]):
        ue, We = rys_gen.rys_exact(N, T)
        u, W = rys_gen.evaluate_split(packed, params, N, T)
        assert np.max(np.abs(u / ue - 1)) < 6e-14
        assert np.max(np.abs(W / We - 1)) < 6e-14


@pytest.mark.parametrize("N", range(1, 10))
def test_fp32_large_T_limit_has_no_cancellation(N):
    """The FP32 tier evaluates the Gauss-Hermite limit u = x^2 / T,
    w = w_h / sqrt(T) in single precision from s = rsqrtf(T) (at most 2 ulp,
    CUDA's documented bound). Emulated here with s off by 2 ulp either way
    and every product rounded to FP32: u and w stay within 6 ulp of the FP64
    value (products only, no cancellation), just above the table's end and
    far beyond it."""
    xh, wh = rys_gen.hermite_half(N)
    x2 = (xh * xh).astype(np.float32)
    whf = wh.astype(np.float32)
    tmax = rys_gen.fit_tables(rys_gen.FP32_FIT, nmax=N)[1][N - 1]["tmax"]
    ulp = 2.0 ** -23
    for T in (tmax * (1 + 1e-6), tmax * 1.5, 1e3, 1e6):
        s64 = 1.0 / math.sqrt(T)
        for k in (-2, 0, 2):
            s32 = np.float32(np.float32(s64) * np.float32(1 + k * ulp))
            u32 = np.float32(x2 * np.float32(s32 * s32))
            w32 = np.float32(whf * s32)
            u64 = xh * xh / T
            w64 = wh * s64
            assert np.all(np.abs(u32 / u64 - 1) <= 6 * ulp), (N, T, k)
            assert np.all(np.abs(w32 / w64 - 1) <= 6 * ulp), (N, T, k)
