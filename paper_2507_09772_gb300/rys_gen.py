"""Generator of the Rys roots/weights interpolation tables used by the kernels.

Rys quadrature (Sec. 2, eq:rys1) replaces the Boys-function integral
F_n(T) = int_0^1 t^(2n) exp(-T t^2) dt by an N-point Gauss rule in u = t^2:
sum_r W_r u_r^n = F_n(T) for n = 0 .. 2N-1. The paper interpolates roots and
weights from tabulated data it does not print; this module builds its own
tables from first principles and needs only numpy:

1. Exact roots and weights at a given T: discretise the measure
   exp(-T t^2) dt on [0, 1] with a 200-point Gauss-Legendre rule (nodes from
   Newton's method on the Legendre recurrence), run the discretised
   Stieltjes procedure (Gautschi, "Orthogonal Polynomials: Computation and
   Approximation", 2004, Sec. 2.2.3) in the scaled variable v = max(1,T) u to
   get the three-term recurrence of the orthogonal polynomials, and take
   nodes and weights from the eigen-decomposition of the Jacobi matrix
   (Golub and Welsch, Math. Comp. 23 (1969)).
2. For 0 <= T < T_asym(N): piecewise polynomials in T on intervals of width
   h, fitted at Chebyshev points and stored as monomial coefficients in the
   local variable x = 2 (T - T_k)/h - 1 for Horner evaluation.
3. For T >= T_asym(N): the half-range Gauss-Hermite limit u_r = x_r^2 / T,
   W_r = w_r / sqrt(T), with x_r, w_r the positive nodes and weights of the
   2N-point Gauss-Hermite rule (the measure on [0, inf) differs from the one
   on [0, 1] by less than exp(-T)/(2T)).

Table layout (one flat float64 array, also cast to float32 for the FP32 tier
with its own, shorter fit): for each N, ``nint`` intervals, each holding 2N
functions (u_0..u_{N-1}, W_0..W_{N-1}) of ``deg+1`` coefficients, lowest
power first.
"""
from __future__ import annotations

import math
import os

import numpy as np

NMAX = 9
# Asymptotic switch points: above these T the Gauss-Hermite limit agrees
# with the exact roots and weights to about 1e-15 relative (measured with
# this module's own exact routine).
T_ASYM = {1: 40.0, 2: 48.0, 3: 52.0, 4: 60.0, 5: 64.0, 6: 72.0, 7: 76.0, 8: 84.0, 9: 92.0}
FP64_FIT = (0.5, 9)     # interval width, polynomial degree
FP32_FIT = (1.0, 7)


def gauss_legendre01(m: int):
    """m-point Gauss-Legendre nodes and weights on [0, 1] (Newton on P_m)."""
    k = np.arange(1, m + 1)
    x = np.cos(np.pi * (k - 0.25) / (m + 0.5))
    for _ in range(100):
        p0, p1 = np.ones_like(x), x.copy()
        for n in range(2, m + 1):
            p0, p1 = p1, ((2 * n - 1) * x * p1 - (n - 1) * p0) / n
        dp = m * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-17:
            break
    p0, p1 = np.ones_like(x), x.copy()
    for n in range(2, m + 1):
        p0, p1 = p1, ((2 * n - 1) * x * p1 - (n - 1) * p0) / n
    dp = m * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return (x + 1.0) / 2.0, w / 2.0


_TG, _WG = gauss_legendre01(200)


def rys_exact(N: int, T: float):
    """Roots u_r (= t_r^2, ascending) and weights W_r of the N-point Rys rule."""
    s = max(1.0, T)
    u = _TG * _TG
    w = _WG * np.exp(-T * u)
    v = s * u
    a = np.zeros(N)
    b = np.zeros(N)
    p_prev = np.zeros_like(v)
    p_cur = np.ones_like(v)
    nrm_prev = 1.0
    for j in range(N):
        nrm = np.sum(w * p_cur * p_cur)
        a[j] = np.sum(w * v * p_cur * p_cur) / nrm
        b[j] = nrm if j == 0 else nrm / nrm_prev
        p_prev, p_cur = p_cur, (v - a[j]) * p_cur - (b[j] if j > 0 else 0.0) * p_prev
        nrm_prev = nrm
    jac = np.diag(a) + np.diag(np.sqrt(b[1:]), 1) + np.diag(np.sqrt(b[1:]), -1)
    ev, evec = np.linalg.eigh(jac)
    return ev / s, b[0] * evec[0] ** 2


def hermite_half(N: int):
    """Positive nodes x_r and weights w_r of the 2N-point Gauss-Hermite rule."""
    n = 2 * N
    off = np.sqrt(np.arange(1, n) / 2.0)
    ev, evec = np.linalg.eigh(np.diag(off, 1) + np.diag(off, -1))
    w = math.sqrt(math.pi) * evec[0] ** 2
    keep = ev > 0
    return ev[keep], w[keep]


def rys_asymptotic(N: int, T: float):
    x, w = hermite_half(N)
    return x * x / T, w / math.sqrt(T)


def _cheb_to_mono(c: np.ndarray) -> np.ndarray:
    return np.polynomial.chebyshev.cheb2poly(c)


def fit_tables(fit=FP64_FIT, nmax: int = NMAX):
    """Return (table float64 array, params list of dicts per N)."""
    h, deg = fit
    xs = np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))
    chunks, params = [], []
    off = 0
    for N in range(1, nmax + 1):
        tmax = T_ASYM[N]
        nint = int(math.ceil(tmax / h))
        tab = np.empty((nint, 2 * N, deg + 1))
        for k in range(nint):
            vals = np.array([np.concatenate(rys_exact(N, k * h + h * (x + 1.0) / 2.0)) for x in xs])
            coef = np.polynomial.chebyshev.chebfit(xs, vals, deg)   # (deg+1, 2N)
            for j in range(2 * N):
                tab[k, j] = _cheb_to_mono(coef[:, j])
        chunks.append(tab.ravel())
        xh, wh = hermite_half(N)
        params.append(dict(N=N, offset=off, nint=nint, h=h, deg=deg, tmax=nint * h,
                           x2=(xh * xh).tolist(), wh=wh.tolist()))
        off += tab.size
    return np.concatenate(chunks), params


def evaluate(table: np.ndarray, params: dict, T: float):
    """Host model of the kernels' evaluation (used by the tests)."""
    N = params["N"]
    if T >= params["tmax"]:
        x2 = np.asarray(params["x2"])
        wh = np.asarray(params["wh"])
        return x2 / T, wh / math.sqrt(T)
    h, deg = params["h"], params["deg"]
    k = int(T / h)
    x = 2.0 * (T - k * h) / h - 1.0
    base = params["offset"] + k * 2 * N * (deg + 1)
    c = table[base:base + 2 * N * (deg + 1)].reshape(2 * N, deg + 1)
    acc = c[:, deg].copy()
    for i in range(deg - 1, -1, -1):
        acc = acc * x + c[:, i]
    return acc[:N], acc[N:]


SPLIT = 6   # FP64 tier: coefficients 0..SPLIT-1 in FP64, the rest as an FP32 tail


def pack_split(table: np.ndarray, params: list):
    """FP64-tier layout used by the kernels: per function 8 doubles (64 B):
    c0..c5 as doubles, then c6..c9 as four floats in the last 16 bytes. The
    tail terms are below 2e-7 of c0 on every interval, so summing them in
    FP32 costs about 1e-14 relative while saving FP64 multiply-adds."""
    deg = params[0]["deg"]
    assert deg + 1 == SPLIT + 4
    chunks = []
    for p in params:
        N = p["N"]
        c = table[p["offset"]:p["offset"] + p["nint"] * 2 * N * (deg + 1)].reshape(-1, deg + 1)
        out = np.zeros((c.shape[0], 8), dtype=np.float64)
        out[:, :SPLIT] = c[:, :SPLIT]
        tail = c[:, SPLIT:].astype(np.float32)
        out[:, SPLIT:] = tail.view(np.float64).reshape(-1, 2)
        chunks.append(out.ravel())
    return np.concatenate(chunks)


def evaluate_split(packed: np.ndarray, params: list, N: int, T: float):
    """Host model of the kernel's split evaluation (FP32 tail, FP64 head)."""
    p = params[N - 1]
    if T >= p["tmax"]:
        return evaluate(None, p, T)
    offs = [0]
    for q in params:
        offs.append(offs[-1] + q["nint"] * 2 * q["N"] * 8)
    h = p["h"]
    k = int(T / h)
    x = 2.0 * (T - k * h) / h - 1.0
    base = offs[N - 1] + k * 2 * N * 8
    blk = packed[base:base + 2 * N * 8].reshape(2 * N, 8)
    xf = np.float32(x)
    res = np.empty(2 * N)
    for j in range(2 * N):
        t = blk[j, SPLIT:].view(np.float32)
        a = np.float32(t[3])
        for i in (2, 1, 0):
            a = np.float32(np.float32(a * xf) + t[i])
        acc = float(a)
        for i in range(SPLIT - 1, -1, -1):
            acc = acc * x + blk[j, i]
        res[j] = acc
    return res[:N], res[N:]


def _fmt(v: float) -> str:
    return float(v).hex()


def write_sources(outdir: str) -> dict:
    """Write rys_tables.inc (host data) and rys_params.cuh (device constants)."""
    os.makedirs(outdir, exist_ok=True)
    t64, p64 = fit_tables(FP64_FIT)
    t32, p32 = fit_tables(FP32_FIT)
    with open(os.path.join(outdir, "rys_tables.inc.tmp"), "w") as f:
        f.write("// generated by rys_gen.py: Rys root/weight interpolation tables\n")
        t64p = pack_split(t64, p64)
        f.write(f"static const size_t rys_table64_size = {t64p.size};\n")
        f.write("static const double rys_table64[] = {\n")
        for i in range(0, t64p.size, 4):
            f.write(",".join(_fmt(v) for v in t64p[i:i + 4]) + ",\n")
        f.write("};\n")
        f.write(f"static const int rys32_nint_host[{NMAX + 1}] = {{0,"
                + ",".join(str(p['nint']) for p in p32) + "};\n")
        f.write(f"static const int rys32_deg_host = {p32[0]['deg']};\n")
        f.write(f"static const size_t rys_table32_size = {t32.size};\n")
        f.write("static const double rys_table32_src[] = {\n")
        for i in range(0, t32.size, 4):
            f.write(",".join(_fmt(v) for v in t32[i:i + 4]) + ",\n")
        f.write("};\n")
    os.replace(os.path.join(outdir, "rys_tables.inc.tmp"), os.path.join(outdir, "rys_tables.inc"))
    with open(os.path.join(outdir, "rys_params.cuh.tmp"), "w") as f:
        f.write("// generated by rys_gen.py: Rys table geometry and Gauss-Hermite limits\n")
        f.write("#pragma once\n")
        f.write(f"#define RYS_NMAX {NMAX}\n")
        offs64, o = [], 0
        for p in p64:
            offs64.append(o)
            o += p["nint"] * 2 * p["N"] * 8
        for tag, ps in (("64", p64), ("32", p32)):
            offs = offs64 if tag == "64" else [p['offset'] for p in ps]
            f.write(f"__device__ __constant__ int rys{tag}_offset[{NMAX + 1}] = {{0,"
                    + ",".join(str(x) for x in offs) + "};\n")
            f.write(f"#define RYS{tag}_DEG {ps[0]['deg']}\n")
            f.write(f"#define RYS{tag}_H {ps[0]['h']!r}\n")
            f.write(f"#define RYS{tag}_INVH {1.0 / ps[0]['h']!r}\n")
            f.write(f"__device__ __constant__ double rys{tag}_tmax[{NMAX + 1}] = {{0,"
                    + ",".join(_fmt(p['tmax']) for p in ps) + "};\n")
            f.write(f"__device__ __constant__ int rys{tag}_nint[{NMAX + 1}] = {{0,"
                    + ",".join(str(p['nint']) for p in ps) + "};\n")
        # compile-time interval counts of the FP32 tables (shared-memory sizing)
        f.write(f"constexpr int rys32_nint_c[{NMAX + 1}] = {{0,"
                + ",".join(str(p['nint']) for p in p32) + "};\n")
        # Gauss-Hermite limits, packed per N: x_r^2 then w_r
        offs, flat = [0], []
        for p in p64:
            flat += p["x2"] + p["wh"]
            offs.append(len(flat))
        f.write(f"__device__ __constant__ int rys_gh_offset[{NMAX + 1}] = {{"
                + ",".join(str(o) for o in offs[:-1]) + "};\n")
        f.write(f"__device__ __constant__ double rys_gh[{len(flat)}] = {{"
                + ",".join(_fmt(v) for v in flat) + "};\n")
        # the same limits and the FP32 table ends rounded to FP32, so that the
        # FP32 tier reads floats (no FP64 conversion on its path)
        f.write(f"__device__ __constant__ float rys_gh32[{len(flat)}] = {{"
                + ",".join(_fmt(float(np.float32(v))) + "f" for v in flat) + "};\n")
        f.write(f"__device__ __constant__ float rys32_tmaxf[{NMAX + 1}] = {{0.0f,"
                + ",".join(_fmt(float(np.float32(p['tmax']))) + "f" for p in p32) + "};\n")
    os.replace(os.path.join(outdir, "rys_params.cuh.tmp"), os.path.join(outdir, "rys_params.cuh"))
    return {"fp64_size": int(t64.size), "fp32_size": int(t32.size)}


if __name__ == "__main__":
    import sys
    print(write_sources(sys.argv[1] if len(sys.argv) > 1 else "_build"))
