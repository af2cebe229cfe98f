// Small device kernels of the JK build compiled ahead of time by nvcc:
// primitive-pair tables, density block maxima, zeroing and symmetrisation.
#pragma once
#include "jk_types.h"

// Primitive-pair records of one shell pair per thread (Sec. 3, pair data
// precomputed once per geometry; Table 2 lists the raw inputs).
__global__ void jk_pairdata_kernel(int npair, const int *__restrict__ pa, const int *__restrict__ pb,
                                   const int *__restrict__ pp_off, const int *__restrict__ sh_atom,
                                   const int *__restrict__ sh_nprim, const int *__restrict__ sh_prim,
                                   const double *__restrict__ coords, const double *__restrict__ exps,
                                   const double *__restrict__ coeffs, JkPrimPair64 *__restrict__ out64,
                                   JkPrimPair32 *__restrict__ out32)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npair) return;
    const int a = pa[t], b = pb[t];
    const double *A = coords + 3 * sh_atom[a], *B = coords + 3 * sh_atom[b];
    const double ABx = A[0] - B[0], ABy = A[1] - B[1], ABz = A[2] - B[2];
    const double r2 = ABx * ABx + ABy * ABy + ABz * ABz;
    const int na = sh_nprim[a], nb = sh_nprim[b];
    int o = pp_off[t];
    for (int i = 0; i < na; ++i) {
        const double al = exps[sh_prim[a] + i], ca = coeffs[sh_prim[a] + i];
        for (int j = 0; j < nb; ++j, ++o) {
            const double be = exps[sh_prim[b] + j], cb = coeffs[sh_prim[b] + j];
            const double p = al + be, ip = 1.0 / p;
            JkPrimPair64 r;
            r.Px = (al * A[0] + be * B[0]) * ip;
            r.Py = (al * A[1] + be * B[1]) * ip;
            r.Pz = (al * A[2] + be * B[2]) * ip;
            r.p = p;
            r.PAx = r.Px - A[0];
            r.PAy = r.Py - A[1];
            r.PAz = r.Pz - A[2];
            r.K = ca * cb * exp(-al * be * ip * r2) * ip;
            r.inv2p = 0.5 * ip;
            r.q = 0.0;
            r.qf = r.padf = 0.f;
            r.pad2 = 0.0;
            out64[o] = r;
            JkPrimPair32 s;
            s.Px = (float)r.Px; s.Py = (float)r.Py; s.Pz = (float)r.Pz; s.p = (float)p;
            s.PAx = (float)r.PAx; s.PAy = (float)r.PAy; s.PAz = (float)r.PAz; s.K = (float)r.K;
            s.inv2p = (float)r.inv2p; s.q = 0.f; s.pad1 = s.pad2 = 0.f;
            out32[o] = s;
        }
    }
}

// Block-max |D| over every density: one CTA per (molecule, shell a), the
// threads over shell b. Also the per-molecule maximum (non-negative doubles
// order like their bit patterns, so an integer atomicMax works).
__global__ void jk_dmax_kernel(const JkMol *__restrict__ mols, const int *__restrict__ sh_mol,
                               const int *__restrict__ mol_sh0, const int *__restrict__ sh_ao,
                               const int *__restrict__ sh_nc, int ndm, double *__restrict__ dmax,
                               float *__restrict__ dmax32, unsigned long long *__restrict__ dmax_mol,
                               int *__restrict__ err)
{
    const int s = blockIdx.x;
    const int m = sh_mol[s];
    const JkMol mol = mols[m];
    const int a = s - mol_sh0[m];
    const int na = sh_nc[s], aoa = sh_ao[s];
    const long long nn = (long long)mol.nao * mol.nao;
    double rowmax = 0.0;
    for (int b = threadIdx.x; b < mol.nsh; b += blockDim.x) {
        const int sb = mol_sh0[m] + b;
        const int nb = sh_nc[sb], aob = sh_ao[sb];
        double mx = 0.0;
        bool bad = false;
        for (int k = 0; k < ndm; ++k)
            for (int i = 0; i < na; ++i)
                for (int j = 0; j < nb; ++j) {
                    const double v = fabs(mol.D[k * nn + (long long)(aoa + i) * mol.nao + aob + j]);
                    bad = bad || !(v <= 1.7976931348623157e308);   // NaN or infinity
                    mx = fmax(mx, v);
                }
        if (bad) atomicOr(err, JK_ERR_DEV_NAN);
        dmax[mol.dmax_off + (long long)a * mol.nsh + b] = mx;
        dmax32[mol.dmax_off + (long long)a * mol.nsh + b] = (float)mx;
        rowmax = fmax(rowmax, mx);
    }
    for (int o = 16; o > 0; o >>= 1) rowmax = fmax(rowmax, __shfl_xor_sync(0xffffffffu, rowmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dmax_mol + m, (unsigned long long)__double_as_longlong(rowmax));
}

// In-place J <- X + X^T (and the same for K) per molecule and density, on
// 32 x 32 tiles of the upper triangle. tile_off[m] is the first tile of
// molecule m (prefix over nt(nt+1)/2, nt = ceil(nao/32)).
__global__ void jk_symmetrize_kernel(const JkMol *__restrict__ mols, const long long *__restrict__ tile_off,
                                     int nmol, int ndm, int do_j, int do_k)
{
    __shared__ double t1[32][33], t2[32][33];
    const long long tile = blockIdx.x;
    int lo = 0, hi = nmol - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (tile_off[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    const int m = lo;
    const JkMol mol = mols[m];
    const int n = mol.nao;
    const int nt = (n + 31) / 32;
    long long r = tile - tile_off[m];
    int ti = 0;
    while (r >= nt - ti) { r -= nt - ti; ++ti; }
    const int tj = ti + (int)r;
    const int dm = blockIdx.y;
    double *X = (blockIdx.z == 0) ? mol.J : mol.K;
    if ((blockIdx.z == 0 && !do_j) || (blockIdx.z == 1 && !do_k) || X == nullptr) return;
    X += (long long)dm * n * n;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        int i = ti * 32 + k, j = tj * 32 + tx;
        t1[k][tx] = (i < n && j < n) ? X[(long long)i * n + j] : 0.0;
        i = tj * 32 + k; j = ti * 32 + tx;
        t2[k][tx] = (i < n && j < n) ? X[(long long)i * n + j] : 0.0;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        int i = ti * 32 + k, j = tj * 32 + tx;
        if (i < n && j < n) X[(long long)i * n + j] = t1[k][tx] + t2[tx][k];
        i = tj * 32 + k; j = ti * 32 + tx;
        if (i < n && j < n && ti != tj) X[(long long)i * n + j] = t2[k][tx] + t1[tx][k];
    }
}

// FMA-chain throughput probes: 8 independent chains per thread so that the
// FMA pipe, not latency, bounds the loop. The result is stored only if it
// equals a value it never takes, which keeps the loop alive.
template <typename T>
__global__ void jk_fma_probe_kernel(int iters, T seed, T *sink)
{
    T a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    const T m = (T)0.9999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            a0 = a0 * m + c; a1 = a1 * m + c; a2 = a2 * m + c; a3 = a3 * m + c;
            a4 = a4 * m + c; a5 = a5 * m + c; a6 = a6 * m + c; a7 = a7 * m + c;
        }
    }
    T r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (r == (T)-12345.678) sink[0] = r;
}

// Zero the J/K accumulators of every molecule (pointers read from the
// device descriptors, so a captured graph stays valid when they change).
__global__ void jk_zero_kernel(const JkMol *__restrict__ mols, int ndm)
{
    const JkMol mol = mols[blockIdx.y];
    const long long n = (long long)ndm * mol.nao * mol.nao;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (mol.J) mol.J[i] = 0.0;
        if (mol.K) mol.K[i] = 0.0;
    }
}

// FP32 copy of every molecule's densities for the FP32 tier (one rounding
// per element, as the tier would apply on every load).
__global__ void jk_d32_kernel(const JkMol *__restrict__ mols, int ndm)
{
    const JkMol mol = mols[blockIdx.y];
    float *dst = const_cast<float *>(mol.D32);
    const long long n = (long long)ndm * mol.nao * mol.nao;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)mol.D[i];
}

// Spherical <-> Cartesian transforms, one thread per (shell a, shell b)
// block of one molecule and density. c2s holds, per l, the ncart(l) x (2l+1)
// coefficients (row-major) at c2s_off[l]; a Cartesian shell uses the
// identity. Directions:
//   to_cart = 1: Xc[a][b] = C_a Xs[a][b] C_b^T   (density, spherical -> Cartesian)
//   to_cart = 0: Xs[a][b] = C_a^T Xc[a][b] C_b   (J and K, Cartesian -> spherical)
struct JkSphMol {
    const double *src[2];   // up to two matrices per call (J and K, or D)
    double *dst[2];
    int nsrc;
    int nao_c, nao_s;
    int sh0, nsh;           // global index of the first shell, shell count
};

__global__ void jk_sph_kernel(const JkSphMol *__restrict__ mols, const int *__restrict__ sh_l,
                              const int *__restrict__ sh_sph, const int *__restrict__ sh_aoc,
                              const int *__restrict__ sh_aos, const double *__restrict__ c2s,
                              const int *__restrict__ c2s_off, int ndm, int to_cart)
{
    const JkSphMol M = mols[blockIdx.z];
    const long long nblk = (long long)M.nsh * M.nsh;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nblk) return;
    const int a = M.sh0 + (int)(t / M.nsh), b = M.sh0 + (int)(t % M.nsh);
    const int la = sh_l[a], lb = sh_l[b];
    const int nca = (la + 1) * (la + 2) / 2, ncb = (lb + 1) * (lb + 2) / 2;
    const int nsa = sh_sph[a] ? 2 * la + 1 : nca, nsb = sh_sph[b] ? 2 * lb + 1 : ncb;
    const double *Ca = c2s + c2s_off[la], *Cb = c2s + c2s_off[lb];
    const int dm = blockIdx.y;
    for (int w = 0; w < M.nsrc; ++w) {
        const double *S = M.src[w];
        double *Dst = M.dst[w];
        if (!S || !Dst) continue;
        if (to_cart) {
            S += (long long)dm * M.nao_s * M.nao_s;
            Dst += (long long)dm * M.nao_c * M.nao_c;
            for (int i = 0; i < nca; ++i)
                for (int j = 0; j < ncb; ++j) {
                    double s = 0.0;
                    for (int m = 0; m < nsa; ++m) {
                        const double ca = sh_sph[a] ? Ca[i * nsa + m] : (double)(i == m);
                        if (ca == 0.0) continue;
                        double r = 0.0;
                        for (int n = 0; n < nsb; ++n) {
                            const double cb = sh_sph[b] ? Cb[j * nsb + n] : (double)(j == n);
                            r += cb * S[(long long)(sh_aos[a] + m) * M.nao_s + sh_aos[b] + n];
                        }
                        s += ca * r;
                    }
                    Dst[(long long)(sh_aoc[a] + i) * M.nao_c + sh_aoc[b] + j] = s;
                }
        } else {
            S += (long long)dm * M.nao_c * M.nao_c;
            Dst += (long long)dm * M.nao_s * M.nao_s;
            for (int m = 0; m < nsa; ++m)
                for (int n = 0; n < nsb; ++n) {
                    double s = 0.0;
                    for (int i = 0; i < nca; ++i) {
                        const double ca = sh_sph[a] ? Ca[i * nsa + m] : (double)(i == m);
                        if (ca == 0.0) continue;
                        double r = 0.0;
                        for (int j = 0; j < ncb; ++j) {
                            const double cb = sh_sph[b] ? Cb[j * nsb + n] : (double)(j == n);
                            r += cb * S[(long long)(sh_aoc[a] + i) * M.nao_c + sh_aoc[b] + j];
                        }
                        s += ca * r;
                    }
                    Dst[(long long)(sh_aos[a] + m) * M.nao_s + sh_aos[b] + n] = s;
                }
        }
    }
}

// Primitive Schwarz factors into the pair records, then each shell pair's
// primitive pairs reordered by q (largest first), one thread per shell pair.
__global__ void jk_primsort_kernel(int npair, const int *__restrict__ pp_off, const int *__restrict__ pp_cnt,
                                   const double *__restrict__ qprim, const JkPrimPair64 *__restrict__ in64,
                                   const JkPrimPair32 *__restrict__ in32, JkPrimPair64 *__restrict__ out64,
                                   JkPrimPair32 *__restrict__ out32)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npair) return;
    const int o = pp_off[t], n = pp_cnt[t];
    for (int k = 0; k < n; ++k) {
        // rank of record k: how many records precede it (q descending, ties by index)
        const double qk = qprim[o + k];
        int rank = 0;
        for (int m = 0; m < n; ++m) {
            const double qm = qprim[o + m];
            if (qm > qk || (qm == qk && m < k)) ++rank;
        }
        JkPrimPair64 r = in64[o + k];
        JkPrimPair32 s = in32[o + k];
        r.q = qk;
        r.qf = (float)qk;
        s.q = (float)qk;
        out64[o + rank] = r;
        out32[o + rank] = s;
    }
}
