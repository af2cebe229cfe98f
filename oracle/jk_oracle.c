/*
 * Plain, slow FP64 CPU oracle for the Coulomb/exchange (JK) build.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file. The product path never calls it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (Sec. 2 of the paper):
 *   eq:rys0  contracted ERI = sum over primitive quartets of c c c c (pq|rs)
 *   eq:jk    J_ij = sum_kl (ij|kl) D_kl,   K_ik = sum_jl (ij|kl) D_jl
 *   eq:schwartz  |(ij|kl)| <= sqrt((ij|ij)) sqrt((kl|kl)) at shell level
 *
 * The paper evaluates primitive ERIs by Rys quadrature. The oracle reaches
 * the same integrals by a different route, McMurchie-Davidson (the paper
 * names it in Sec. 2 as the other standard scheme):
 *   1. Hermite expansion coefficients E^{ij}_t per Cartesian direction,
 *      from the two-term Gaussian product and the E recurrences.
 *   2. Hermite Coulomb integrals R^n_{tuv}, from (-2 rho)^n F_n(T) by the
 *      R recurrences.
 *   3. (ab|cd) = 2 pi^{5/2} / (p q sqrt(p+q)) *
 *                sum_{tuv} E^{ab}_{tuv} sum_{t'u'v'} (-1)^{t'+u'+v'}
 *                E^{cd}_{t'u'v'} R_{t+t',u+u',v+v'}.
 * The Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt comes from its
 * power series below T = 30 (then downward recursion) and from the error
 * function with upward recursion above.
 *
 * Readings of the paper used here:
 *   - Cartesian components are ordered x-exponent descending, then y
 *     descending (Sec. 2, the reversed lexicographic order).
 *   - Schwarz factors are taken at shell level: Q_ab = sqrt(max over the
 *     functions mu in a, nu in b of |(mu nu|mu nu)|).
 *   - A shell quartet is kept iff Q_ab Q_cd Dmax > cutoff (strict), with
 *     Dmax the largest |D| over every density and over the shell blocks the
 *     requested outputs read: ab and cd for J; ac, ad, bc, bd for K.
 *     With use_dmax == 0, Dmax := 1 (the paper's profiling setting, Sec. 3.1).
 *   - The unique-quartet rule of Sec. 2 is read at shell level as a >= b,
 *     c >= d, pair(ab) >= pair(cd), with degeneracy factor
 *     f = (a==b ? 1/2 : 1)(c==d ? 1/2 : 1)(ab==cd ? 1/2 : 1); D is symmetric.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LMAX 4              /* up to g shells */
#define LTOT (4 * LMAX)     /* largest total angular momentum of a quartet */
#define NCMAX ((LMAX + 1) * (LMAX + 2) / 2)

typedef struct {
    int32_t atom, l, nprim, prim_off, ao_off, spherical;
} oshell;

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian exponents of component idx of a shell with angular momentum l. */
static void cart_exponents(int l, int idx, int *lx, int *ly, int *lz)
{
    int k = 0;
    for (int x = l; x >= 0; --x)
        for (int y = l - x; y >= 0; --y) {
            if (k == idx) { *lx = x; *ly = y; *lz = l - x - y; return; }
            ++k;
        }
}

/* ------------------------------------------------------------------ Boys */
void oracle_boys(int mmax, double T, double *F)
{
    const double Ts = 30.0;
    if (T < Ts) {
        /* F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) */
        double term = 1.0 / (2 * mmax + 1);
        double sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= 2.0 * T / (2 * mmax + 2 * k + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        double e = exp(-T);
        F[mmax] = e * sum;
        for (int m = mmax; m > 0; --m)
            F[m - 1] = (2.0 * T * F[m] + e) / (2 * m - 1);
    } else {
        double st = sqrt(T);
        double e = exp(-T);
        F[0] = 0.5 * sqrt(M_PI) * erf(st) / st;
        for (int m = 0; m < mmax; ++m)
            F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
    }
}

/* ------------------------------------------------------- Hermite E coefs */
/* E[i][j][t], i <= la, j <= lb, t <= i + j, for one Cartesian direction.
 * E^{00}_0 = exp(-mu X_AB^2) with mu = a b / p. */
#define EDIM (2 * LMAX + 1)
typedef double Etab[LMAX + 1][LMAX + 1][EDIM + 1];

static void hermite_E(int la, int lb, double a, double b, double XA, double XB, Etab E)
{
    double p = a + b;
    double mu = a * b / p;
    double XAB = XA - XB;
    double XP = (a * XA + b * XB) / p;
    double XPA = XP - XA, XPB = XP - XB;
    double h = 0.5 / p;
    memset(E, 0, sizeof(Etab));
    E[0][0][0] = exp(-mu * XAB * XAB);
    for (int i = 0; i <= la; ++i) {
        for (int j = 0; j <= lb; ++j) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; ++t) {
                double v;
                if (j == 0) {
                    /* E^{i,0}_t from E^{i-1,0} */
                    double em1 = (t >= 1) ? E[i - 1][0][t - 1] : 0.0;
                    double e0 = (t <= i - 1) ? E[i - 1][0][t] : 0.0;
                    double ep1 = (t + 1 <= i - 1) ? E[i - 1][0][t + 1] : 0.0;
                    v = h * em1 + XPA * e0 + (t + 1) * ep1;
                } else {
                    double em1 = (t >= 1) ? E[i][j - 1][t - 1] : 0.0;
                    double e0 = (t <= i + j - 1) ? E[i][j - 1][t] : 0.0;
                    double ep1 = (t + 1 <= i + j - 1) ? E[i][j - 1][t + 1] : 0.0;
                    v = h * em1 + XPB * e0 + (t + 1) * ep1;
                }
                E[i][j][t] = v;
            }
        }
    }
}

/* --------------------------------------------------- Hermite R integrals */
/* R[n][t][u][v] with t+u+v <= L - n. */
#define RD (LTOT + 1)
static void hermite_R(int L, double rho, double X, double Y, double Z, double *R /*RD^4*/)
{
    double F[LTOT + 2];
    double T = rho * (X * X + Y * Y + Z * Z);
    oracle_boys(L, T, F);
#define RR(n, t, u, v) R[(((n) * RD + (t)) * RD + (u)) * RD + (v)]
    for (int n = L; n >= 0; --n) {
        int top = L - n;
        for (int t = 0; t <= top; ++t)
            for (int u = 0; u <= top - t; ++u)
                for (int v = 0; v <= top - t - u; ++v) {
                    double val;
                    if (t > 0) {
                        val = X * RR(n + 1, t - 1, u, v);
                        if (t > 1) val += (t - 1) * RR(n + 1, t - 2, u, v);
                    } else if (u > 0) {
                        val = Y * RR(n + 1, t, u - 1, v);
                        if (u > 1) val += (u - 1) * RR(n + 1, t, u - 2, v);
                    } else if (v > 0) {
                        val = Z * RR(n + 1, t, u, v - 1);
                        if (v > 1) val += (v - 1) * RR(n + 1, t, u, v - 2);
                    } else {
                        val = pow(-2.0 * rho, n) * F[n];
                    }
                    RR(n, t, u, v) = val;
                }
    }
#undef RR
}

/* ------------------------------------------- primitive Cartesian ERI block */
/* Unnormalised primitives with coefficient 1:
 *   out[((ia*nb + ib)*nc + ic)*nd + id] = (a_ia b_ib | c_ic d_id)
 * where a_ia = (x-Ax)^lx (y-Ay)^ly (z-Az)^lz exp(-alpha |r-A|^2). */
/* Range separation of the Coulomb operator (Table 1 of the paper, rys_type):
 * g_omega == 0: 1/r; g_omega > 0: erf(omega r)/r (long range);
 * g_omega < 0: erfc(|omega| r)/r = 1/r - erf(|omega| r)/r (short range).
 * For erf(omega r)/r the McMurchie-Davidson formula keeps its form with rho
 * replaced by rho theta, theta = omega^2/(omega^2 + rho), and the prefactor
 * multiplied by sqrt(theta). Set through oracle_set_omega. */
static double g_omega = 0.0;
void oracle_set_omega(double omega) { g_omega = omega; }

static void eri_prim_block_op(int la, int lb, int lc, int ld,
                              double aa, double ab, double ac, double ad,
                              const double *A, const double *B, const double *C, const double *D,
                              double scale, double omega, double *out, double *Rbuf);

static void eri_prim_block(int la, int lb, int lc, int ld,
                           double aa, double ab, double ac, double ad,
                           const double *A, const double *B, const double *C, const double *D,
                           double scale, double *out, double *Rbuf)
{
    if (g_omega == 0.0) {
        eri_prim_block_op(la, lb, lc, ld, aa, ab, ac, ad, A, B, C, D, scale, 0.0, out, Rbuf);
    } else if (g_omega > 0.0) {
        eri_prim_block_op(la, lb, lc, ld, aa, ab, ac, ad, A, B, C, D, scale, g_omega, out, Rbuf);
    } else {
        eri_prim_block_op(la, lb, lc, ld, aa, ab, ac, ad, A, B, C, D, scale, 0.0, out, Rbuf);
        eri_prim_block_op(la, lb, lc, ld, aa, ab, ac, ad, A, B, C, D, -scale, -g_omega, out, Rbuf);
    }
}

static void eri_prim_block_op(int la, int lb, int lc, int ld,
                              double aa, double ab, double ac, double ad,
                              const double *A, const double *B, const double *C, const double *D,
                              double scale, double omega, double *out, double *Rbuf)
{
    Etab Eab[3], Ecd[3];
    double p = aa + ab, q = ac + ad;
    double P[3], Q[3];
    for (int k = 0; k < 3; ++k) {
        hermite_E(la, lb, aa, ab, A[k], B[k], Eab[k]);
        hermite_E(lc, ld, ac, ad, C[k], D[k], Ecd[k]);
        P[k] = (aa * A[k] + ab * B[k]) / p;
        Q[k] = (ac * C[k] + ad * D[k]) / q;
    }
    double rho = p * q / (p + q);
    double theta = omega > 0.0 ? omega * omega / (omega * omega + rho) : 1.0;
    int L = la + lb + lc + ld;
    hermite_R(L, rho * theta, P[0] - Q[0], P[1] - Q[1], P[2] - Q[2], Rbuf);
    double pref = scale * sqrt(theta) * 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));
    int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
#define R0(t, u, v) Rbuf[(((0) * RD + (t)) * RD + (u)) * RD + (v)]
    for (int ia = 0; ia < na; ++ia) {
        int ax, ay, az; cart_exponents(la, ia, &ax, &ay, &az);
        for (int ib = 0; ib < nb; ++ib) {
            int bx, by, bz; cart_exponents(lb, ib, &bx, &by, &bz);
            for (int ic = 0; ic < nc; ++ic) {
                int cx, cy, cz; cart_exponents(lc, ic, &cx, &cy, &cz);
                for (int id = 0; id < nd; ++id) {
                    int dx, dy, dz; cart_exponents(ld, id, &dx, &dy, &dz);
                    double s = 0.0;
                    for (int t = 0; t <= ax + bx; ++t)
                        for (int u = 0; u <= ay + by; ++u)
                            for (int v = 0; v <= az + bz; ++v) {
                                double ebra = Eab[0][ax][bx][t] * Eab[1][ay][by][u] * Eab[2][az][bz][v];
                                if (ebra == 0.0) continue;
                                double inner = 0.0;
                                for (int t2 = 0; t2 <= cx + dx; ++t2)
                                    for (int u2 = 0; u2 <= cy + dy; ++u2)
                                        for (int v2 = 0; v2 <= cz + dz; ++v2) {
                                            double eket = Ecd[0][cx][dx][t2] * Ecd[1][cy][dy][u2] * Ecd[2][cz][dz][v2];
                                            double sg = ((t2 + u2 + v2) & 1) ? -1.0 : 1.0;
                                            inner += sg * eket * R0(t + t2, u + u2, v + v2);
                                        }
                                s += ebra * inner;
                            }
                    out[((ia * nb + ib) * nc + ic) * nd + id] += pref * s;
                }
            }
        }
    }
#undef R0
}

/* Public primitive entry (for the derivative and quadrature pins). */
void oracle_eri_prim(int la, int lb, int lc, int ld,
                     double aa, double ab, double ac, double ad,
                     const double *A, const double *B, const double *C, const double *D,
                     double *out)
{
    double *Rbuf = (double *)malloc(sizeof(double) * RD * RD * RD * RD);
    int n = ncart(la) * ncart(lb) * ncart(lc) * ncart(ld);
    memset(out, 0, sizeof(double) * n);
    eri_prim_block(la, lb, lc, ld, aa, ab, ac, ad, A, B, C, D, 1.0, out, Rbuf);
    free(Rbuf);
}

/* -------------------------------------------- contracted shell quartet */
typedef struct {
    const oshell *sh;
    const double *coords, *exps, *coeffs;
} basis_t;

static void eri_shell(const basis_t *bs, int a, int b, int c, int d, double *out, double *Rbuf)
{
    const oshell *sa = &bs->sh[a], *sb = &bs->sh[b], *sc = &bs->sh[c], *sd = &bs->sh[d];
    int n = ncart(sa->l) * ncart(sb->l) * ncart(sc->l) * ncart(sd->l);
    memset(out, 0, sizeof(double) * n);
    const double *A = bs->coords + 3 * sa->atom, *B = bs->coords + 3 * sb->atom;
    const double *C = bs->coords + 3 * sc->atom, *D = bs->coords + 3 * sd->atom;
    for (int i = 0; i < sa->nprim; ++i)
        for (int j = 0; j < sb->nprim; ++j)
            for (int k = 0; k < sc->nprim; ++k)
                for (int l = 0; l < sd->nprim; ++l) {
                    double cc = bs->coeffs[sa->prim_off + i] * bs->coeffs[sb->prim_off + j] *
                                bs->coeffs[sc->prim_off + k] * bs->coeffs[sd->prim_off + l];
                    eri_prim_block(sa->l, sb->l, sc->l, sd->l,
                                   bs->exps[sa->prim_off + i], bs->exps[sb->prim_off + j],
                                   bs->exps[sc->prim_off + k], bs->exps[sd->prim_off + l],
                                   A, B, C, D, cc, out, Rbuf);
                }
}

void oracle_eri_shell(const oshell *sh, const double *coords, const double *exps,
                      const double *coeffs, int a, int b, int c, int d, double *out)
{
    basis_t bs = {sh, coords, exps, coeffs};
    double *Rbuf = (double *)malloc(sizeof(double) * RD * RD * RD * RD);
    eri_shell(&bs, a, b, c, d, out, Rbuf);
    free(Rbuf);
}

/* Cartesian AO offsets: the oracle works in the Cartesian basis; shells'
 * ao_off fields are ignored and recomputed from the shell order. */
static int cart_offsets(const oshell *sh, int nsh, int *off)
{
    int o = 0;
    for (int s = 0; s < nsh; ++s) { off[s] = o; o += ncart(sh[s].l); }
    return o;
}

/* ------------------------------------------------------- Schwarz factors */
void oracle_schwarz(const oshell *sh, int nsh, const double *coords, const double *exps,
                    const double *coeffs, double *Q /* nsh*nsh */)
{
    basis_t bs = {sh, coords, exps, coeffs};
#pragma omp parallel
    {
        double *Rbuf = (double *)malloc(sizeof(double) * RD * RD * RD * RD);
        double *blk = (double *)malloc(sizeof(double) * NCMAX * NCMAX * NCMAX * NCMAX);
#pragma omp for schedule(dynamic, 1)
        for (int a = 0; a < nsh; ++a)
            for (int b = 0; b <= a; ++b) {
                eri_shell(&bs, a, b, a, b, blk, Rbuf);
                int na = ncart(sh[a].l), nb = ncart(sh[b].l);
                double m = 0.0;
                for (int i = 0; i < na; ++i)
                    for (int j = 0; j < nb; ++j) {
                        double v = fabs(blk[((i * nb + j) * na + i) * nb + j]);
                        if (v > m) m = v;
                    }
                Q[a * nsh + b] = Q[b * nsh + a] = sqrt(m);
            }
        free(Rbuf); free(blk);
    }
}

/* Shell-block max |D| over all densities (Cartesian D, nao x nao each). */
void oracle_dmax(const oshell *sh, int nsh, const double *D, int ndm, int nao, double *Dm)
{
    int *off = (int *)malloc(sizeof(int) * nsh);
    cart_offsets(sh, nsh, off);
    for (int a = 0; a < nsh; ++a)
        for (int b = 0; b < nsh; ++b) {
            double m = 0.0;
            for (int k = 0; k < ndm; ++k)
                for (int i = 0; i < ncart(sh[a].l); ++i)
                    for (int j = 0; j < ncart(sh[b].l); ++j) {
                        double v = fabs(D[((size_t)k * nao + off[a] + i) * nao + off[b] + j]);
                        if (v > m) m = v;
                    }
            Dm[a * nsh + b] = m;
        }
    free(off);
}

static double quartet_bound(const double *Q, const double *Dm, int nsh, int a, int b, int c, int d,
                            int with_j, int with_k, int use_dmax)
{
    double dm = 1.0;
    if (use_dmax) {
        dm = 0.0;
        if (with_j) {
            dm = fmax(dm, Dm[a * nsh + b]);
            dm = fmax(dm, Dm[c * nsh + d]);
        }
        if (with_k) {
            dm = fmax(dm, Dm[a * nsh + c]);
            dm = fmax(dm, Dm[a * nsh + d]);
            dm = fmax(dm, Dm[b * nsh + c]);
            dm = fmax(dm, Dm[b * nsh + d]);
        }
    }
    return Q[a * nsh + b] * Q[c * nsh + d] * dm;
}

/* ------------------------------------------------------ full ERI tensor */
/* eri[((i*nao + j)*nao + k)*nao + l] = (ij|kl) in the Cartesian basis, no
 * screening, every shell quartet evaluated (no symmetry used). */
void oracle_eri_full(const oshell *sh, int nsh, const double *coords, const double *exps,
                     const double *coeffs, double *eri)
{
    basis_t bs = {sh, coords, exps, coeffs};
    int *off = (int *)malloc(sizeof(int) * nsh);
    size_t nao = (size_t)cart_offsets(sh, nsh, off);
#pragma omp parallel
    {
        double *Rbuf = (double *)malloc(sizeof(double) * RD * RD * RD * RD);
        double *blk = (double *)malloc(sizeof(double) * NCMAX * NCMAX * NCMAX * NCMAX);
#pragma omp for collapse(2) schedule(dynamic, 1)
        for (int a = 0; a < nsh; ++a)
            for (int b = 0; b < nsh; ++b)
                for (int c = 0; c < nsh; ++c)
                    for (int d = 0; d < nsh; ++d) {
                        eri_shell(&bs, a, b, c, d, blk, Rbuf);
                        int na = ncart(sh[a].l), nb = ncart(sh[b].l);
                        int nc = ncart(sh[c].l), nd = ncart(sh[d].l);
                        for (int i = 0; i < na; ++i)
                            for (int j = 0; j < nb; ++j)
                                for (int k = 0; k < nc; ++k)
                                    for (int l = 0; l < nd; ++l)
                                        eri[(((off[a] + i) * nao + off[b] + j) * nao + off[c] + k) * nao + off[d] + l] =
                                            blk[((i * nb + j) * nc + k) * nd + l];
                    }
        free(Rbuf); free(blk);
    }
    free(off);
}

/* ------------------------------------------------- brute-force JK build */
/* Definition of eq:jk summed over every shell quartet (no permutational
 * symmetry), each quartet kept by the screening rule above. */
long long oracle_jk_brute(const oshell *sh, int nsh, const double *coords, const double *exps,
                          const double *coeffs, const double *Q, const double *Dm,
                          const double *D, int ndm, int with_j, int with_k,
                          double cutoff, int use_dmax, double *J, double *K)
{
    basis_t bs = {sh, coords, exps, coeffs};
    int *off = (int *)malloc(sizeof(int) * nsh);
    int nao = cart_offsets(sh, nsh, off);
    size_t nn = (size_t)ndm * nao * nao;
    if (J) memset(J, 0, sizeof(double) * nn);
    if (K) memset(K, 0, sizeof(double) * nn);
    long long kept = 0;
#pragma omp parallel reduction(+ : kept)
    {
        double *Rbuf = (double *)malloc(sizeof(double) * RD * RD * RD * RD);
        double *blk = (double *)malloc(sizeof(double) * NCMAX * NCMAX * NCMAX * NCMAX);
        double *Jl = (double *)calloc(nn, sizeof(double));
        double *Kl = (double *)calloc(nn, sizeof(double));
#pragma omp for collapse(2) schedule(dynamic, 1)
        for (int a = 0; a < nsh; ++a)
            for (int b = 0; b < nsh; ++b)
                for (int c = 0; c < nsh; ++c)
                    for (int d = 0; d < nsh; ++d) {
                        if (!(quartet_bound(Q, Dm, nsh, a, b, c, d, with_j, with_k, use_dmax) > cutoff))
                            continue;
                        ++kept;
                        eri_shell(&bs, a, b, c, d, blk, Rbuf);
                        int na = ncart(sh[a].l), nb = ncart(sh[b].l);
                        int nc = ncart(sh[c].l), nd = ncart(sh[d].l);
                        for (int m = 0; m < ndm; ++m) {
                            const double *Dk = D + (size_t)m * nao * nao;
                            double *Jk = Jl + (size_t)m * nao * nao, *Kk = Kl + (size_t)m * nao * nao;
                            for (int i = 0; i < na; ++i)
                                for (int j = 0; j < nb; ++j)
                                    for (int k = 0; k < nc; ++k)
                                        for (int l = 0; l < nd; ++l) {
                                            double v = blk[((i * nb + j) * nc + k) * nd + l];
                                            int I = off[a] + i, Jx = off[b] + j, Kx = off[c] + k, L = off[d] + l;
                                            if (with_j) Jk[I * nao + Jx] += v * Dk[Kx * nao + L];
                                            if (with_k) Kk[I * nao + Kx] += v * Dk[Jx * nao + L];
                                        }
                        }
                    }
#pragma omp critical
        {
            for (size_t i = 0; i < nn; ++i) {
                if (J) J[i] += Jl[i];
                if (K) K[i] += Kl[i];
            }
        }
        free(Rbuf); free(blk); free(Jl); free(Kl);
    }
    free(off);
    return kept;
}

/* -------------------------------------------- screened, 8-fold symmetric */
/* Unique quartets a >= b, c >= d, pair(ab) >= pair(cd) with pair(ab) =
 * a(a+1)/2 + b. Each adds f*T to the half matrices
 *   X_ab += 2 f T D_cd,  X_cd += 2 f T D_ab,
 *   Y_ac += f T D_bd,  Y_ad += f T D_bc,  Y_bc += f T D_ad,  Y_bd += f T D_ac,
 * and J = X + X^T, K = Y + Y^T. Returns the number of quartets kept. */
long long oracle_jk_screened(const oshell *sh, int nsh, const double *coords, const double *exps,
                             const double *coeffs, const double *Q, const double *Dm,
                             const double *D, int ndm, int with_j, int with_k,
                             double cutoff, int use_dmax, double *J, double *K)
{
    basis_t bs = {sh, coords, exps, coeffs};
    int *off = (int *)malloc(sizeof(int) * nsh);
    int nao = cart_offsets(sh, nsh, off);
    size_t nn = (size_t)ndm * nao * nao;
    long long npair = (long long)nsh * (nsh + 1) / 2;
    int *pa = (int *)malloc(sizeof(int) * npair), *pb = (int *)malloc(sizeof(int) * npair);
    for (int a = 0, p = 0; a < nsh; ++a)
        for (int b = 0; b <= a; ++b, ++p) { pa[p] = a; pb[p] = b; }
    double *X = (double *)calloc(nn, sizeof(double));
    double *Y = (double *)calloc(nn, sizeof(double));
    long long kept = 0;
#pragma omp parallel reduction(+ : kept)
    {
        double *Rbuf = (double *)malloc(sizeof(double) * RD * RD * RD * RD);
        double *blk = (double *)malloc(sizeof(double) * NCMAX * NCMAX * NCMAX * NCMAX);
        double *Xl = (double *)calloc(nn, sizeof(double));
        double *Yl = (double *)calloc(nn, sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (long long p1 = 0; p1 < npair; ++p1)
            for (long long p2 = 0; p2 <= p1; ++p2) {
                int a = pa[p1], b = pb[p1], c = pa[p2], d = pb[p2];
                if (!(quartet_bound(Q, Dm, nsh, a, b, c, d, with_j, with_k, use_dmax) > cutoff))
                    continue;
                ++kept;
                double f = 1.0;
                if (a == b) f *= 0.5;
                if (c == d) f *= 0.5;
                if (p1 == p2) f *= 0.5;
                eri_shell(&bs, a, b, c, d, blk, Rbuf);
                int na = ncart(sh[a].l), nb = ncart(sh[b].l);
                int nc = ncart(sh[c].l), nd = ncart(sh[d].l);
                for (int m = 0; m < ndm; ++m) {
                    const double *Dk = D + (size_t)m * nao * nao;
                    double *Xk = Xl + (size_t)m * nao * nao, *Yk = Yl + (size_t)m * nao * nao;
                    for (int i = 0; i < na; ++i)
                        for (int j = 0; j < nb; ++j)
                            for (int k = 0; k < nc; ++k)
                                for (int l = 0; l < nd; ++l) {
                                    double v = f * blk[((i * nb + j) * nc + k) * nd + l];
                                    int I = off[a] + i, Jx = off[b] + j, Kx = off[c] + k, L = off[d] + l;
                                    if (with_j) {
                                        Xk[I * nao + Jx] += 2.0 * v * Dk[Kx * nao + L];
                                        Xk[Kx * nao + L] += 2.0 * v * Dk[I * nao + Jx];
                                    }
                                    if (with_k) {
                                        Yk[I * nao + Kx] += v * Dk[Jx * nao + L];
                                        Yk[I * nao + L] += v * Dk[Jx * nao + Kx];
                                        Yk[Jx * nao + Kx] += v * Dk[I * nao + L];
                                        Yk[Jx * nao + L] += v * Dk[I * nao + Kx];
                                    }
                                }
                }
            }
#pragma omp critical
        {
            for (size_t i = 0; i < nn; ++i) { X[i] += Xl[i]; Y[i] += Yl[i]; }
        }
        free(Rbuf); free(blk); free(Xl); free(Yl);
    }
    for (int m = 0; m < ndm; ++m)
        for (int i = 0; i < nao; ++i)
            for (int j = 0; j < nao; ++j) {
                size_t ij = ((size_t)m * nao + i) * nao + j, ji = ((size_t)m * nao + j) * nao + i;
                if (J) J[ij] = with_j ? X[ij] + X[ji] : 0.0;
                if (K) K[ij] = with_k ? Y[ij] + Y[ji] : 0.0;
            }
    free(X); free(Y); free(pa); free(pb); free(off);
    return kept;
}

/* --------------------------------------------------- row-restricted J/K */
/* Exact J for the shell blocks (jblk[2i], jblk[2i+1]) and K for the shell
 * blocks (kblk[2i], kblk[2i+1]), straight from eq:jk with every shell
 * quartet that the screening rule keeps:
 *   J_{mu nu} = sum over all shells c, d of (a b|c d) D_cd   (mu in a, nu in b)
 *   K_{mu ka} = sum over all shells b, d of (a b|c d) D_bd   (mu in a, ka in c)
 * Output: each block written densely (ndm x na x nb) into jout / kout in
 * the order given. Returns the number of shell quartets evaluated. */
long long oracle_jk_rows(const oshell *sh, int nsh, const double *coords, const double *exps,
                         const double *coeffs, const double *Q, const double *Dm,
                         const double *D, int ndm, int nao, int with_j, int with_k,
                         double cutoff, int use_dmax,
                         const int *jblk, int njblk, double *jout,
                         const int *kblk, int nkblk, double *kout)
{
    basis_t bs = {sh, coords, exps, coeffs};
    int *off = (int *)malloc(sizeof(int) * nsh);
    cart_offsets(sh, nsh, off);
    long long *jpos = (long long *)malloc(sizeof(long long) * (njblk + 1));
    long long *kpos = (long long *)malloc(sizeof(long long) * (nkblk + 1));
    jpos[0] = 0;
    for (int i = 0; i < njblk; ++i)
        jpos[i + 1] = jpos[i] + (long long)ndm * ncart(sh[jblk[2 * i]].l) * ncart(sh[jblk[2 * i + 1]].l);
    kpos[0] = 0;
    for (int i = 0; i < nkblk; ++i)
        kpos[i + 1] = kpos[i] + (long long)ndm * ncart(sh[kblk[2 * i]].l) * ncart(sh[kblk[2 * i + 1]].l);
    if (jout) memset(jout, 0, sizeof(double) * jpos[njblk]);
    if (kout) memset(kout, 0, sizeof(double) * kpos[nkblk]);
    long long count = 0;
    int ntask = njblk + nkblk;
    /* parallel over (block, x): each thread sums into its own copy of the
     * outputs, added up at the end (only the summation order differs from a
     * serial loop) */
#pragma omp parallel reduction(+ : count)
    {
        double *Rbuf = (double *)malloc(sizeof(double) * RD * RD * RD * RD);
        double *blk = (double *)malloc(sizeof(double) * NCMAX * NCMAX * NCMAX * NCMAX);
        double *jl = (double *)calloc((size_t)jpos[njblk] + 1, sizeof(double));
        double *kl = (double *)calloc((size_t)kpos[nkblk] + 1, sizeof(double));
#pragma omp for collapse(2) schedule(dynamic, 1)
        for (int task = 0; task < ntask; ++task)
            for (int x = 0; x < nsh; ++x) {
                int isj = task < njblk;
                int ti = isj ? task : task - njblk;
                const int *bl = isj ? jblk : kblk;
                int s1 = bl[2 * ti], s2 = bl[2 * ti + 1];
                int n1 = ncart(sh[s1].l), n2 = ncart(sh[s2].l);
                double *dst = isj ? jl + jpos[ti] : kl + kpos[ti];
                for (int y = 0; y < nsh; ++y) {
                    int a, b, c, d;
                    if (isj) { a = s1; b = s2; c = x; d = y; }
                    else { a = s1; c = s2; b = x; d = y; }
                    if (!(quartet_bound(Q, Dm, nsh, a, b, c, d, with_j, with_k, use_dmax) > cutoff))
                        continue;
                    ++count;
                    eri_shell(&bs, a, b, c, d, blk, Rbuf);
                    int na = ncart(sh[a].l), nb = ncart(sh[b].l);
                    int nc = ncart(sh[c].l), nd = ncart(sh[d].l);
                    for (int m = 0; m < ndm; ++m) {
                        const double *Dk = D + (size_t)m * nao * nao;
                        for (int i = 0; i < na; ++i)
                            for (int j = 0; j < nb; ++j)
                                for (int k = 0; k < nc; ++k)
                                    for (int l = 0; l < nd; ++l) {
                                        double v = blk[((i * nb + j) * nc + k) * nd + l];
                                        if (isj)
                                            dst[(m * n1 + i) * n2 + j] += v * Dk[(off[c] + k) * nao + off[d] + l];
                                        else
                                            dst[(m * n1 + i) * n2 + k] += v * Dk[(off[b] + j) * nao + off[d] + l];
                                    }
                    }
                }
            }
#pragma omp critical
        {
            if (jout) for (long long i = 0; i < jpos[njblk]; ++i) jout[i] += jl[i];
            if (kout) for (long long i = 0; i < kpos[nkblk]; ++i) kout[i] += kl[i];
        }
        free(Rbuf); free(blk); free(jl); free(kl);
    }
    free(off); free(jpos); free(kpos);
    return count;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
