// Integral kernels of the JK build, compiled at run time by NVRTC for
// sm_103a, one instantiation per (l_a, l_b, l_c, l_d, n_a, n_b, n_c, n_d)
// class and per fragmentation, density count, J/K flags and precision
// (the static parameters of Table 1 of the paper). The library prepends
// jk_types.h and the generated rys_params.cuh.
//
// Method (Sec. 2 of the paper):
//   eq:rys0  (ab|cd) = sum over primitive quartets of c_a c_b c_c c_d (pq|rs)
//   eq:rys1  (pq|rs) = sum_r w_r (pq|rs)(t_r), N_r = floor(L/2) + 1 roots
//   eq:rys2  (pq|rs)(t_r) = I_x I_y I_z, each a 2D table over the Cartesian
//            exponents of the four centres, built per root by the vertical
//            recurrence on (A, C) and the horizontal transfers A->B, C->D
//   eq:jk    J_ab += T D_cd, J_cd += T D_ab, K_ac += T D_bd, K_ad += T D_bc,
//            K_bc += T D_ad, K_bd += T D_ac for each unique quartet (8-fold
//            symmetry, Sec. 2), scaled by the degeneracy factor f: 2f for J
//            and f for K into half matrices that are symmetrised afterwards.
//
// Thread mapping: a group of G = GA*GB*GC*GD threads evaluates one shell
// quartet. Each thread owns a fragment of FA x FB x FC x FD Cartesian
// components (the 1qnt fragmentation of Sec. 3.2; G = 1 is the 1q1t case of
// Sec. 3.1). With G == 1 the 2D tables live in registers; with G > 1 they
// live in shared memory, one set per group, built cooperatively per root and
// direction. A warp owns one bra pair at a time and scans its ket pairs in
// chunks of 32 candidates, screening each (Schwarz times density-block max),
// so the quartet list is never materialised; the J_ab partial stays in
// registers across the whole ket scan and is flushed once per bra pair.

#define JK_TWO_PI_2_5 34.986836655249725  // 2 pi^(5/2)

__device__ constexpr int jk_ncart(int l) { return (l + 1) * (l + 2) / 2; }

// Cartesian exponent along `axis` of component idx of a shell with angular
// momentum l: components ordered x descending, then y descending.
__device__ constexpr int jk_cart_exp(int l, int idx, int axis)
{
    int k = 0;
    for (int x = l; x >= 0; --x)
        for (int y = l - x; y >= 0; --y) {
            if (k == idx) return axis == 0 ? x : (axis == 1 ? y : l - x - y);
            ++k;
        }
    return 0;
}

template <typename R> struct JkPP;
template <> struct JkPP<double> { typedef JkPrimPair64 T; };
template <> struct JkPP<float> { typedef JkPrimPair32 T; };
__device__ __forceinline__ float jk_pp_q(const JkPrimPair64 &r) { return r.qf; }
__device__ __forceinline__ float jk_pp_q(const JkPrimPair32 &r) { return r.q; }

__device__ __forceinline__ double jk_rsqrt(double x) { return rsqrt(x); }

// A - B of a pair in the tier's precision (the FP32 copy is stored, so the
// FP32 tier converts nothing on the FP64 pipe).
__device__ __forceinline__ void jk_pair_ab(const JkPair &p, double &x, double &y, double &z)
{
    x = p.ABx; y = p.ABy; z = p.ABz;
}
__device__ __forceinline__ void jk_pair_ab(const JkPair &p, float &x, float &y, float &z)
{
    x = p.ABxf; y = p.AByf; z = p.ABzf;
}

// An FP32 tier contribution widened to FP64 for the FP64 atomics into J and
// K. A float-to-double conversion is an FP64-pipe instruction (1/64 of the
// FP32 rate on GB300); the alternative builds the IEEE-754 binary64 bit
// pattern with integer operations: sign, exponent rebiased from 127 to
// 1023, fraction shifted left by 29; subnormal floats are normalised first.
// Exact for every float. (Measured: the integer form is the slower of the
// two on the batched workload, so the conversion is the default.)
__device__ __forceinline__ double jk_wide(double x, int) { return x; }
__device__ __forceinline__ double jk_to_f64(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long bits;
    if (e == 0xffu) {
        bits = sgn | (0x7ffull << 52) | ((unsigned long long)m << 29);
    } else if (e != 0) {
        bits = sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (m == 0) {
        bits = sgn;
    } else {
        const int top = 31 - __clz(m);   // leading bit of the subnormal fraction, 0..22
        bits = sgn | ((unsigned long long)(top + 874) << 52) |
               (((unsigned long long)m << (52 - top)) & 0xfffffffffffffull);
    }
    return __longlong_as_double((long long)bits);
}
// wi = 0: the conversion instruction instead (for comparison)
__device__ __forceinline__ double jk_wide(float x, int wi) { return wi ? jk_to_f64(x) : (double)x; }
__device__ __forceinline__ float jk_rsqrt(float x) { return rsqrtf(x); }

// ----------------------------------------------------- Rys roots, weights
// Root r and weight r of the N-point rule at T. The piecewise polynomials
// cover 0 <= T < tmax; above it the half-range Gauss-Hermite limit
// u = x^2 / T, w = w_h / sqrt(T) holds (evaluated in the tier's precision).
template <int N>
__device__ __forceinline__ void jk_rys_one(double T, int r, const double *__restrict__ tab,
                                           double &u, double &w, int /*a64*/)
{
    if (T >= rys64_tmax[N]) {
        double s = rsqrt(T);
        u = rys_gh[rys_gh_offset[N - 1] + r] * (s * s);
        w = rys_gh[rys_gh_offset[N - 1] + N + r] * s;
        return;
    }
    int k = min((int)(T * RYS64_INVH), rys64_nint[N] - 1);
    double x = (T - k * RYS64_H) * (2.0 * RYS64_INVH) - 1.0;
    // per function 8 doubles: c0..c5, then c6..c9 as floats (terms below
    // 2e-7 of c0, summed in FP32 and added to the FP64 Horner head)
    const double *cu = tab + rys64_offset[N] + (long long)k * (2 * N * 8) + r * 8;
    const double *cw = cu + N * 8;
    const float xf = (float)x;
    const float4 tu = __ldg(reinterpret_cast<const float4 *>(cu + 6));
    const float4 tw = __ldg(reinterpret_cast<const float4 *>(cw + 6));
    double au = (double)fmaf(fmaf(fmaf(tu.w, xf, tu.z), xf, tu.y), xf, tu.x);
    double aw = (double)fmaf(fmaf(fmaf(tw.w, xf, tw.z), xf, tw.y), xf, tw.x);
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        au = fma(au, x, __ldg(cu + i));
        aw = fma(aw, x, __ldg(cw + i));
    }
    u = au;
    w = aw;
}

// FP32: `tab` is this N's table alone, as the class kernel stages it in
// shared memory: per interval the 16 N coefficients (per root the eight of u,
// then per root the eight of w) and four floats of padding, so that the
// 16-byte vectors of different intervals fall in different bank groups.
template <int N>
__device__ __forceinline__ void jk_rys_one(float T, int r, const float *__restrict__ tab,
                                           float &u, float &w, int a64)
{
    static_assert(RYS32_DEG == 7, "two float4 per function");
    if (T >= rys32_tmaxf[N]) {
        if (a64) {
            // the same limit evaluated in FP64, rounded once to FP32
            const double s = rsqrt((double)T);
            u = (float)(rys_gh[rys_gh_offset[N - 1] + r] * (s * s));
            w = (float)(rys_gh[rys_gh_offset[N - 1] + N + r] * s);
            return;
        }
        // u = x^2 / T, w = w_h / sqrt(T): no cancellation, so FP32 keeps
        // ~2 ulp; the Gauss-Hermite constants are FP64-derived, stored
        // rounded to FP32
        const float s = rsqrtf(T);
        u = rys_gh32[rys_gh_offset[N - 1] + r] * (s * s);
        w = rys_gh32[rys_gh_offset[N - 1] + N + r] * s;
        return;
    }
    int k = min((int)(T * (float)RYS32_INVH), rys32_nint_c[N] - 1);
    float x = (T - k * (float)RYS32_H) * (float)(2.0 * RYS32_INVH) - 1.0f;
    const float4 *cu = reinterpret_cast<const float4 *>(tab + k * (16 * N + 4) + r * 8);
    const float4 *cw = cu + N * 2;
    const float4 u0 = cu[0], u1 = cu[1], w0 = cw[0], w1 = cw[1];
    float au = fmaf(fmaf(fmaf(u1.w, x, u1.z), x, u1.y), x, u1.x);
    float aw = fmaf(fmaf(fmaf(w1.w, x, w1.z), x, w1.y), x, w1.x);
    au = fmaf(fmaf(fmaf(fmaf(au, x, u0.w), x, u0.z), x, u0.y), x, u0.x);
    aw = fmaf(fmaf(fmaf(fmaf(aw, x, w0.w), x, w0.z), x, w0.y), x, w0.x);
    u = au;
    w = aw;
}

template <typename R> struct JkIsFloat { static constexpr bool v = false; };
template <> struct JkIsFloat<float> { static constexpr bool v = true; };

// Floats of the FP32 Rys table of the N-root rule in its shared-memory
// layout (intervals padded from 16 N to 16 N + 4 floats).
template <int N> struct JkRysTab32 { static constexpr int n = rys32_nint_c[N] * (16 * N + 4); };

// --------------------------------------------------------- 2D integrals
// One direction, one root: vertical recurrence on (n on A, m on C) up to
// (LA+LB, LC+LD), then horizontal transfers to (a, b, c, d). Output layout
// out[((a*(LB+1) + b)*(LC+1) + c)*(LD+1) + d].
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void jk_build_2d(R c00, R c00p, R b10, R b01, R b00, R i00,
                                            R ab, R cd, R *__restrict__ out)
{
    constexpr int NA = LA + LB, NC = LC + LD;
    R V[NA + 1][NC + 1];
    V[0][0] = i00;
    if (NA > 0) V[1][0] = c00 * i00;
#pragma unroll
    for (int n = 1; n < NA; ++n) V[n + 1][0] = c00 * V[n][0] + R(n) * b10 * V[n - 1][0];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
#pragma unroll
        for (int n = 0; n <= NA; ++n) {
            R v = c00p * V[n][m];
            if (m > 0) v += R(m) * b01 * V[n][m - 1];
            if (n > 0) v += R(n) * b00 * V[n - 1][m];
            V[n][m + 1] = v;
        }
    }
    // bra transfer A -> B: H[a][b] = H[a+1][b-1] + AB H[a][b-1]
    R HB[LA + 1][LB + 1][NC + 1];
#pragma unroll
    for (int m = 0; m <= NC; ++m) {
        R t[NA + 1][LB + 1];
#pragma unroll
        for (int n = 0; n <= NA; ++n) t[n][0] = V[n][m];
#pragma unroll
        for (int b = 1; b <= LB; ++b)
#pragma unroll
            for (int a = 0; a <= NA - b; ++a) t[a][b] = t[a + 1][b - 1] + ab * t[a][b - 1];
#pragma unroll
        for (int a = 0; a <= LA; ++a)
#pragma unroll
            for (int b = 0; b <= LB; ++b) HB[a][b][m] = t[a][b];
    }
    // ket transfer C -> D
#pragma unroll
    for (int a = 0; a <= LA; ++a)
#pragma unroll
        for (int b = 0; b <= LB; ++b) {
            R s[NC + 1][LD + 1];
#pragma unroll
            for (int m = 0; m <= NC; ++m) s[m][0] = HB[a][b][m];
#pragma unroll
            for (int d = 1; d <= LD; ++d)
#pragma unroll
                for (int c = 0; c <= NC - d; ++c) s[c][d] = s[c + 1][d - 1] + cd * s[c][d - 1];
#pragma unroll
            for (int c = 0; c <= LC; ++c)
#pragma unroll
                for (int d = 0; d <= LD; ++d) out[((a * (LB + 1) + b) * (LC + 1) + c) * (LD + 1) + d] = s[c][d];
        }
}

// ----------------------------------------------------------- class shape
// OP: 0 the Coulomb operator 1/r; 1 erf(w r)/r (long range); 2 erfc(w r)/r
// (short range) = 1/r minus the long-range part, i.e. a second root set with
// negative weights (the range separation of Table 1, rys_type).
template <int LA, int LB, int LC, int LD, int GA, int GB, int GC, int GD, int OP = 0>
struct JkShape {
    static constexpr int NFA = jk_ncart(LA), NFB = jk_ncart(LB), NFC = jk_ncart(LC), NFD = jk_ncart(LD);
    static constexpr int FA = NFA / GA, FB = NFB / GB, FC = NFC / GC, FD = NFD / GD;
    static constexpr int G = GA * GB * GC * GD;
    static constexpr int EPT = FA * FB * FC * FD;
    static constexpr int L = LA + LB + LC + LD;
    static constexpr int NR = L / 2 + 1;
    static constexpr int NRE = (OP == 2 ? 2 : 1) * NR;   // roots of all sets
    static constexpr int SD = 1, SC = LD + 1, SB = (LC + 1) * (LD + 1), SA = (LB + 1) * SB;
    static constexpr int NI = (LA + 1) * SA;
    // reals of shared memory per group (G > 1): 2D tables and the roots
    static constexpr int SMEM_GROUP = (G == 1) ? 0 : (NRE * 3 * NI + 2 * NRE);
    static_assert(NFA % GA == 0 && NFB % GB == 0 && NFC % GC == 0 && NFD % GD == 0, "fragment");
    static_assert(G <= 16 * 1024, "a group fits 16 CTAs");
};

// Offsets into a 2D table for the components a thread owns (G > 1).
template <class S>
struct JkOffsets {
    int a[3][S::FA], b[3][S::FB], c[3][S::FC], d[3][S::FD];
};

template <int LA, int LB, int LC, int LD, int GA, int GB, int GC, int GD, class S>
__device__ __forceinline__ void jk_make_offsets(int ga, int gb, int gc, int gd, JkOffsets<S> &o)
{
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
        for (int i = 0; i < S::FA; ++i) {
            int idx = ga * S::FA + i, e = 0, k = 0;
            for (int x = LA; x >= 0; --x)
                for (int y = LA - x; y >= 0; --y, ++k)
                    if (k == idx) e = ax == 0 ? x : (ax == 1 ? y : LA - x - y);
            o.a[ax][i] = e * S::SA;
        }
#pragma unroll
        for (int i = 0; i < S::FB; ++i) {
            int idx = gb * S::FB + i, e = 0, k = 0;
            for (int x = LB; x >= 0; --x)
                for (int y = LB - x; y >= 0; --y, ++k)
                    if (k == idx) e = ax == 0 ? x : (ax == 1 ? y : LB - x - y);
            o.b[ax][i] = e * S::SB;
        }
#pragma unroll
        for (int i = 0; i < S::FC; ++i) {
            int idx = gc * S::FC + i, e = 0, k = 0;
            for (int x = LC; x >= 0; --x)
                for (int y = LC - x; y >= 0; --y, ++k)
                    if (k == idx) e = ax == 0 ? x : (ax == 1 ? y : LC - x - y);
            o.c[ax][i] = e * S::SC;
        }
#pragma unroll
        for (int i = 0; i < S::FD; ++i) {
            int idx = gd * S::FD + i, e = 0, k = 0;
            for (int x = LD; x >= 0; --x)
                for (int y = LD - x; y >= 0; --y, ++k)
                    if (k == idx) e = ax == 0 ? x : (ax == 1 ? y : LD - x - y);
            o.d[ax][i] = e * S::SD;
        }
    }
}

// Barrier of one group: a warp-local group syncs its lanes, a group of more
// than 32 threads is the whole CTA.
template <int G>
__device__ __forceinline__ void jk_group_sync(unsigned gmask)
{
    if constexpr (G <= 32) __syncwarp(gmask);
    else __syncthreads();
}

// ------------------------------------------------ one contracted quartet
// Accumulates the thread's fragment T[EPT] of the contracted block (ab|cd)
// over every primitive quartet (eq:rys0). `grp` is the group's shared
// memory (G > 1), gmask the group's lane mask. The roots and 2D tables are
// built by the NT threads that share `grp` (tg < NT: the thread's index
// among them), the whole group, or, for a group split over several CTAs,
// the group's threads in this CTA.
// Root r (< NRE) of the operator: set 0 at T (1/r) or at theta T (erf);
// for OP 2 set 1 is the erf part with negated weight. Returns u and w * pref.
template <int NR, int OP, typename R>
__device__ __forceinline__ void jk_op_root(R Tt, R rho, R pref, double omega, int a64, int r,
                                           const R *__restrict__ rys, R &u, R &wp)
{
    R uu, ww;
    if (OP == 0 || (OP == 2 && r < NR)) {
        jk_rys_one<NR>(Tt, r, rys, uu, ww, a64);
        u = uu;
        wp = ww * pref;
    } else {
        // theta = w^2 / (w^2 + rho), sqrt(theta) = w / sqrt(w^2 + rho)
        const R om = (R)omega;
        const R rd = jk_rsqrt(om * om + rho);
        const R st = om * rd, th = st * st;
        jk_rys_one<NR>(th * Tt, OP == 2 ? r - NR : r, rys, uu, ww, a64);
        u = th * uu;
        wp = (OP == 2 ? -st : st) * ww * pref;
    }
}

template <int LA, int LB, int LC, int LD, int NPA, int NPB, int NPC, int NPD,
          int GA, int GB, int GC, int GD, typename R, int OP = 0,
          int NT = JkShape<LA, LB, LC, LD, GA, GB, GC, GD, OP>::G>
__device__ __forceinline__ int jk_quartet(const JkPair &bra, const JkPair &ket, float qthr, double omega, int a64,
                                           const typename JkPP<R>::T *__restrict__ pp,
                                           const R *__restrict__ rys, R *grp, unsigned gmask, int tg, bool act,
                                           const JkOffsets<JkShape<LA, LB, LC, LD, GA, GB, GC, GD, OP>> &off,
                                           R (&T)[JkShape<LA, LB, LC, LD, GA, GB, GC, GD, OP>::EPT])
{
    typedef JkShape<LA, LB, LC, LD, GA, GB, GC, GD, OP> S;
    typedef typename JkPP<R>::T PPT;
    constexpr int NR = S::NR;
    constexpr int NRE = S::NRE;
    R ABx, ABy, ABz, CDx, CDy, CDz;
    jk_pair_ab(bra, ABx, ABy, ABz);
    jk_pair_ab(ket, CDx, CDy, CDz);
    const PPT *bpp = pp + bra.pp_off;
    const PPT *kpp = pp + ket.pp_off;
    // primitive pairs are sorted by their Schwarz factor q (largest first):
    // stop a loop at the first q_ij q_kl <= qthr (= prim_eps / Dmax), compared
    // in FP32 (a product below the FP32 range is below any threshold that
    // matters; qthr < 0 screens nothing). The ket's primitive pairs (one
    // record per lane and kl) are the outer loop, so each is loaded once; the
    // bra's (the same for the whole group or warp) the inner one.
    const float qthf = qthr;
    const float qb0 = jk_pp_q(bpp[0]);
    int nprim = 0;
#pragma unroll 1
    for (int kl = 0; kl < NPC * NPD; ++kl) {
        const PPT kp = kpp[kl];
        const float qk = jk_pp_q(kp);
        if (qb0 * qk <= qthf) break;
        for (int ij = 0; ij < NPA * NPB; ++ij) {
            const PPT bp = bpp[ij];
            if (jk_pp_q(bp) * qk <= qthf) break;
            ++nprim;
            const R p = bp.p, q = kp.p;
            const R rpq = jk_rsqrt(p + q);
            const R inv_pq = rpq * rpq;
            const R PQx = bp.Px - kp.Px, PQy = bp.Py - kp.Py, PQz = bp.Pz - kp.Pz;
            const R rho = p * q * inv_pq;
            const R Tt = rho * (PQx * PQx + PQy * PQy + PQz * PQz);
            const R pref = (R)JK_TWO_PI_2_5 * bp.K * kp.K * rpq;
            const R qf = q * inv_pq, pf = p * inv_pq;
            if (S::G == 1) {
#pragma unroll
                for (int r = 0; r < NRE; ++r) {
                    R u, wp;
                    jk_op_root<NR, OP, R>(Tt, rho, pref, omega, a64, r, rys, u, wp);
                    const R b00 = (R)0.5 * u * inv_pq;
                    const R b10 = bp.inv2p * ((R)1 - u * qf);
                    const R b01 = kp.inv2p * ((R)1 - u * pf);
                    const R uq = u * qf, up = u * pf;
                    R tx[S::NI], ty[S::NI], tz[S::NI];
                    jk_build_2d<LA, LB, LC, LD, R>(bp.PAx - uq * PQx, kp.PAx + up * PQx, b10, b01, b00, (R)1, ABx, CDx, tx);
                    jk_build_2d<LA, LB, LC, LD, R>(bp.PAy - uq * PQy, kp.PAy + up * PQy, b10, b01, b00, (R)1, ABy, CDy, ty);
                    jk_build_2d<LA, LB, LC, LD, R>(bp.PAz - uq * PQz, kp.PAz + up * PQz, b10, b01, b00, wp, ABz, CDz, tz);
#pragma unroll
                    for (int ia = 0; ia < S::FA; ++ia)
#pragma unroll
                        for (int ib = 0; ib < S::FB; ++ib)
#pragma unroll
                            for (int ic = 0; ic < S::FC; ++ic)
#pragma unroll
                                for (int id = 0; id < S::FD; ++id) {
                                    const int ox = jk_cart_exp(LA, ia, 0) * S::SA + jk_cart_exp(LB, ib, 0) * S::SB +
                                                   jk_cart_exp(LC, ic, 0) * S::SC + jk_cart_exp(LD, id, 0);
                                    const int oy = jk_cart_exp(LA, ia, 1) * S::SA + jk_cart_exp(LB, ib, 1) * S::SB +
                                                   jk_cart_exp(LC, ic, 1) * S::SC + jk_cart_exp(LD, id, 1);
                                    const int oz = jk_cart_exp(LA, ia, 2) * S::SA + jk_cart_exp(LB, ib, 2) * S::SB +
                                                   jk_cart_exp(LC, ic, 2) * S::SC + jk_cart_exp(LD, id, 2);
                                    const int k = ((ia * S::FB + ib) * S::FC + ic) * S::FD + id;
                                    T[k] += tx[ox] * ty[oy] * tz[oz];
                                }
                }
            } else {
                R *roots = grp + NRE * 3 * S::NI;   // [0, NRE): u ; [NRE, 2 NRE): w * pref
                for (int r = tg; r < NRE && tg < NT; r += NT) {
                    R u, wp;
                    jk_op_root<NR, OP, R>(Tt, rho, pref, omega, a64, r, rys, u, wp);
                    roots[r] = u;
                    roots[NRE + r] = wp;
                }
                jk_group_sync<S::G>(gmask);
                for (int task = tg; task < 3 * NRE && tg < NT; task += NT) {
                    const int r = task / 3, dir = task - 3 * r;
                    const R u = roots[r];
                    const R b00 = (R)0.5 * u * inv_pq;
                    const R b10 = bp.inv2p * ((R)1 - u * qf);
                    const R b01 = kp.inv2p * ((R)1 - u * pf);
                    const R uq = u * qf, up = u * pf;
                    R pa, qc, pqd, abd, cdd, i00 = (R)1;
                    if (dir == 0) { pa = bp.PAx; qc = kp.PAx; pqd = PQx; abd = ABx; cdd = CDx; }
                    else if (dir == 1) { pa = bp.PAy; qc = kp.PAy; pqd = PQy; abd = ABy; cdd = CDy; }
                    else { pa = bp.PAz; qc = kp.PAz; pqd = PQz; abd = ABz; cdd = CDz; i00 = roots[NRE + r]; }
                    jk_build_2d<LA, LB, LC, LD, R>(pa - uq * pqd, qc + up * pqd, b10, b01, b00, i00, abd, cdd,
                                                   grp + (r * 3 + dir) * S::NI);
                }
                jk_group_sync<S::G>(gmask);
                if (act) {
#pragma unroll
                for (int ia = 0; ia < S::FA; ++ia)
#pragma unroll
                    for (int ib = 0; ib < S::FB; ++ib)
#pragma unroll
                        for (int ic = 0; ic < S::FC; ++ic)
#pragma unroll
                            for (int id = 0; id < S::FD; ++id) {
                                const int ox = off.a[0][ia] + off.b[0][ib] + off.c[0][ic] + off.d[0][id];
                                const int oy = off.a[1][ia] + off.b[1][ib] + off.c[1][ic] + off.d[1][id];
                                const int oz = off.a[2][ia] + off.b[2][ib] + off.c[2][ic] + off.d[2][id];
                                const int k = ((ia * S::FB + ib) * S::FC + ic) * S::FD + id;
                                R acc = (R)0;
#pragma unroll
                                for (int r = 0; r < NRE; ++r)
                                    acc += grp[(r * 3 + 0) * S::NI + ox] * grp[(r * 3 + 1) * S::NI + oy] *
                                           grp[(r * 3 + 2) * S::NI + oz];
                                T[k] += acc;
                            }
                }
                jk_group_sync<S::G>(gmask);
            }
        }
    }
    return nprim;
}

template <typename R> __device__ __forceinline__ const typename JkPP<R>::T *jk_pp(const JkClassArgs &a);
template <> __device__ __forceinline__ const JkPrimPair64 *jk_pp<double>(const JkClassArgs &a) { return a.pp64; }
template <> __device__ __forceinline__ const JkPrimPair32 *jk_pp<float>(const JkClassArgs &a) { return a.pp32; }
template <typename R> __device__ __forceinline__ const R *jk_rys(const JkClassArgs &a);
template <> __device__ __forceinline__ const double *jk_rys<double>(const JkClassArgs &a) { return a.rys64; }
template <> __device__ __forceinline__ const float *jk_rys<float>(const JkClassArgs &a) { return a.rys32; }

// ---------------------------------------------- routed builds: the FP64 tier
// The FP64 tier of a routed build is the only tier that runs the router: the
// lanes in `rel` (band quartets the router releases) append (bra item, ket j,
// density factor) to the launch's list while it has room, for the FP32 list
// kernel (MODE 3) of the class pair. Returns whether this lane's quartet was
// listed; a quartet that finds the list full stays in FP64. All 32 lanes of
// the warp call it.
__device__ __forceinline__ bool jk_route_out(const JkClassArgs &args, bool rel, int item, int j, float dq)
{
    const unsigned m = __ballot_sync(0xffffffffu, rel);
    if (!m) return false;
    const int lane = threadIdx.x & 31, first = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == first) base = atomicAdd(args.rcount, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, first);
    const long long pos = (long long)base + __popc(m & ((1u << lane) - 1u));
    const bool listed = rel && pos < args.rcap;
    if (listed) {
        JkRouted e;
        e.item = item; e.ket = j; e.dmq = dq; e.pad = 0;
        args.rlist[pos] = e;
    }
    return listed;
}

// ------------------------------------------------- screening of a candidate
template <int MODE>
__device__ __forceinline__ void jk_screen_bound(const JkClassArgs &args, const JkPair &bra, const JkMol &mol,
                                                const double *dmx, double dmol, float dmol32, int j, int ke,
                                                bool &sig, bool &stop, bool &band, float &dmq, float &Bout);
// Keep (bra, ket j) iff lo < Q_ab Q_cd Dmax <= hi; `stop` when even the
// molecule's largest density element cannot lift this ket (and every later
// one, kets being sorted by Q) above lo.
template <int MODE>
__device__ __forceinline__ void jk_screen(const JkClassArgs &args, const JkPair &bra, const JkPairFeat &braf,
                                          const JkMol &mol, const double *dmx, double dmol, float dmol32, int item,
                                          int j, int ke, bool &sig, bool &stop, bool &band, float &dmq,
                                          unsigned short *rsm)
{
    sig = false;
    stop = false;
    band = false;
    dmq = 1.0f;
    float B = 0.0f;
    jk_screen_bound<MODE>(args, bra, mol, dmx, dmol, dmol32, j, ke, sig, stop, band, dmq, B);
    if (MODE == 1) {
        // learned router for the band candidates, all lanes together on the
        // tensor cores; `band` then marks the quartets released to FP32
        bool listed = false;
        if (__ballot_sync(0xffffffffu, band)) {
            const JkPairFeat kf = band ? args.ket_feat[j] : braf;
            const bool to32 = jk_router_to_fp32_warp(args.router, braf, kf, band ? B : 2.0f * args.tau32,
                                                     band ? dmq : 1.0f, args.tau32, rsm);
            listed = jk_route_out(args, band && to32, item, j, dmq);
            if (band) sig = !listed;
        }
        band = listed;
    }
}

// Whether x and y (FP32 images of FP64 quantities, relative error at most
// 5 FP32 roundings, 3.0e-7) are too close for their order to be decided in
// FP32: then the caller redoes the comparison in FP64.
__device__ __forceinline__ bool jk_near(float x, float y)
{
    return fabsf(x - y) < 2e-6f * y;   // false for y = infinity
}

template <int MODE>
__device__ __forceinline__ void jk_screen_bound(const JkClassArgs &args, const JkPair &bra, const JkMol &mol,
                                                const double *dmx, double dmol, float dmol32, int j, int ke,
                                                bool &sig, bool &stop, bool &band, float &dmq, float &Bout)
{
    if (j >= ke) return;
    const JkPair &kt = args.ket[j];
    if (args.scr32) {
        // FP32 bounds: a handful of FP32 operations per candidate instead of
        // FP64-pipe work (an FP64 instruction costs the FP32 tier 64 FP32
        // ones on GB300). scr32 == 2 keeps the FP64 rule exact: the FP32
        // products carry at most 5 roundings, so only a bound within 2e-6 of
        // a threshold can compare differently from its FP64 value, and those
        // few are redone in FP64 (every tier decides alike, as in FP64).
        const float bq = bra.Qf * __ldg(&kt.Qf);
        const float s = bq * dmol32;
        bool st = s <= args.lo32;
        if (args.scr32 == 2 && jk_near(s, args.lo32)) st = (bra.Q * kt.Q) * dmol <= args.lo;
        if (st) { stop = true; return; }
        float dm = 1.0f;
        const int c = __ldg(&kt.a_loc), d = __ldg(&kt.b_loc);
        const int a = bra.a_loc, b = bra.b_loc, ns = mol.nsh;
        if (args.use_dmax) {
            const float *d32 = args.dmax32 + mol.dmax_off;
            dm = 0.0f;
            if (args.with_j) dm = fmaxf(__ldg(d32 + a * ns + b), __ldg(d32 + c * ns + d));
            if (args.with_k) {
                dm = fmaxf(dm, fmaxf(__ldg(d32 + a * ns + c), __ldg(d32 + a * ns + d)));
                dm = fmaxf(dm, fmaxf(__ldg(d32 + b * ns + c), __ldg(d32 + b * ns + d)));
            }
        }
        // the FP32 image of the FP64 maximum is the maximum of the images
        dmq = dm;
        const float B = bq * dm;
        Bout = B;
        sig = (B > args.lo32) && (B <= args.hi32);
        band = MODE == 1 && sig && B > args.tau32 && B <= args.band_hi32;
        if (args.scr32 == 2 &&
            (jk_near(B, args.lo32) || jk_near(B, args.hi32) ||
             (MODE == 1 && (jk_near(B, args.tau32) || jk_near(B, args.band_hi32))))) {
            double dm64 = 1.0;
            if (args.use_dmax) {
                dm64 = 0.0;
                if (args.with_j) dm64 = fmax(__ldg(dmx + a * ns + b), __ldg(dmx + c * ns + d));
                if (args.with_k) {
                    dm64 = fmax(dm64, fmax(__ldg(dmx + a * ns + c), __ldg(dmx + a * ns + d)));
                    dm64 = fmax(dm64, fmax(__ldg(dmx + b * ns + c), __ldg(dmx + b * ns + d)));
                }
            }
            const double B64 = (bra.Q * kt.Q) * dm64;
            sig = (B64 > args.lo) && (B64 <= args.hi);
            band = MODE == 1 && sig && B64 > args.tau && B64 <= args.band_hi;
        }
        return;
    }
    const double bq = bra.Q * kt.Q;
    if (bq * dmol <= args.lo) { stop = true; return; }
    double dm = 1.0;
    if (args.use_dmax) {
        const int c = kt.a_loc, d = kt.b_loc;
        const int a = bra.a_loc, b = bra.b_loc, ns = mol.nsh;
        dm = 0.0;
        if (args.with_j) dm = fmax(__ldg(dmx + a * ns + b), __ldg(dmx + c * ns + d));
        if (args.with_k) {
            dm = fmax(dm, fmax(__ldg(dmx + a * ns + c), __ldg(dmx + a * ns + d)));
            dm = fmax(dm, fmax(__ldg(dmx + b * ns + c), __ldg(dmx + b * ns + d)));
        }
    }
    // dm below the FP32 range only reaches here with lo < 1e-30, where the
    // primitive threshold is 0 and dmq only divides it
    dmq = (float)dm;
    const double B = bq * dm;
    Bout = (float)B;
    sig = (B > args.lo) && (B <= args.hi);
    band = MODE == 1 && sig && B > args.tau && B <= args.band_hi;
}

// Density factor of a quartet (the same lookups as jk_screen).
__device__ __forceinline__ double jk_quartet_dmax(const JkClassArgs &args, const JkPair &bra, const JkPair &ket,
                                                  const JkMol &mol, const double *dmx)
{
    if (!args.use_dmax) return 1.0;
    const int a = bra.a_loc, b = bra.b_loc, c = ket.a_loc, d = ket.b_loc, ns = mol.nsh;
    double dm = 0.0;
    if (args.with_j) dm = fmax(__ldg(dmx + a * ns + b), __ldg(dmx + c * ns + d));
    if (args.with_k) {
        dm = fmax(dm, fmax(__ldg(dmx + a * ns + c), __ldg(dmx + a * ns + d)));
        dm = fmax(dm, fmax(__ldg(dmx + b * ns + c), __ldg(dmx + b * ns + d)));
    }
    return dm;
}

// MODE 2: one training sample (features, label) for a band quartet, written
// by the group's first thread. tmax is the group's max |T|.
__device__ __forceinline__ void jk_log_sample(const JkClassArgs &args, const JkPair &bra, const JkPair &ket,
                                              const JkPairFeat &braf, const JkPairFeat &ketf, double dm, double tmax)
{
    const double B = bra.Q * ket.Q * dm;
    if (!(B > args.tau && B <= args.band_hi)) return;
    const unsigned long long idx = atomicAdd(args.log_n, 1ull);
    if ((long long)idx >= args.log_cap) return;
    float x[JK_RT_NIN];
    // the bound as the FP32 screening path forms it
    jk_router_features(braf, ketf, (bra.Qf * ket.Qf) * (float)dm, (float)dm, args.tau32, x);
    for (int i = 0; i < JK_RT_NIN; ++i) args.log_x[idx * JK_RT_NIN + i] = x[i];
    args.log_y[idx] = (float)log10(fmax(tmax, 1e-300) / (bra.Q * ket.Q));
}

// ------------------------------------------ contraction with the density
// The thread's fragment T of (ab|cd), degeneracy f: J_ab partial kept in
// jab (flushed once per bra pair), the other five blocks by FP64 atomics.
template <typename R> __device__ __forceinline__ const R *jk_dens(const JkMol &mol);
template <> __device__ __forceinline__ const double *jk_dens<double>(const JkMol &mol) { return mol.D; }
template <> __device__ __forceinline__ const float *jk_dens<float>(const JkMol &mol) { return mol.D32; }

// J and K accumulate by FP64 reductions that return nothing (RED): atomicAdd
// on doubles issues ATOM, whose value the L2 sends back although nobody
// reads it (ncu: 9.7e9 ATOM sectors for one all-FP32 build of 8 molecules,
// 34 per quartet). Relaxed, device scope: the ordering atomicAdd gives.
__device__ __forceinline__ void jk_red_add(double *p, double v)
{
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v) : "memory");
}

template <int FA, int FB, int FC, int FD, int NDM, int DOJ, int DOK, typename R>
__device__ __forceinline__ void jk_contract(const R (&T)[FA * FB * FC * FD], R f, const JkMol &mol,
                                            int a0, int b0, int c0, int d0, R (&jab)[NDM][FA][FB], int wi)
{
    const long long nn = (long long)mol.nao * mol.nao;
    const int nao = mol.nao;
#pragma unroll
    for (int m = 0; m < NDM; ++m) {
        // the tier's own copy of D (the FP32 tier reads a pre-rounded one)
        const R *D = jk_dens<R>(mol) + m * nn;
        if (DOJ) {
            R Dcd[FC][FD], Dab[FA][FB];
#pragma unroll
            for (int ic = 0; ic < FC; ++ic)
#pragma unroll
                for (int id = 0; id < FD; ++id) Dcd[ic][id] = (R)__ldg(D + (long long)(c0 + ic) * nao + d0 + id);
#pragma unroll
            for (int ia = 0; ia < FA; ++ia)
#pragma unroll
                for (int ib = 0; ib < FB; ++ib) Dab[ia][ib] = (R)__ldg(D + (long long)(a0 + ia) * nao + b0 + ib);
            R jcd[FC][FD];
#pragma unroll
            for (int ic = 0; ic < FC; ++ic)
#pragma unroll
                for (int id = 0; id < FD; ++id) jcd[ic][id] = (R)0;
#pragma unroll
            for (int ia = 0; ia < FA; ++ia)
#pragma unroll
                for (int ib = 0; ib < FB; ++ib) {
                    R sum = (R)0;
#pragma unroll
                    for (int ic = 0; ic < FC; ++ic)
#pragma unroll
                        for (int id = 0; id < FD; ++id) {
                            const R t = T[((ia * FB + ib) * FC + ic) * FD + id];
                            sum += t * Dcd[ic][id];
                            jcd[ic][id] += t * Dab[ia][ib];
                        }
                    jab[m][ia][ib] += (R)2 * f * sum;
                }
#pragma unroll
            for (int ic = 0; ic < FC; ++ic)
#pragma unroll
                for (int id = 0; id < FD; ++id)
                    jk_red_add(mol.J + m * nn + (long long)(c0 + ic) * nao + d0 + id, jk_wide((R)2 * f * jcd[ic][id], wi));
        }
        if (DOK) {
            R Dbd[FB][FD], Dbc[FB][FC], Dad[FA][FD], Dac[FA][FC];
#pragma unroll
            for (int ib = 0; ib < FB; ++ib) {
#pragma unroll
                for (int id = 0; id < FD; ++id) Dbd[ib][id] = (R)__ldg(D + (long long)(b0 + ib) * nao + d0 + id);
#pragma unroll
                for (int ic = 0; ic < FC; ++ic) Dbc[ib][ic] = (R)__ldg(D + (long long)(b0 + ib) * nao + c0 + ic);
            }
#pragma unroll
            for (int ia = 0; ia < FA; ++ia) {
#pragma unroll
                for (int id = 0; id < FD; ++id) Dad[ia][id] = (R)__ldg(D + (long long)(a0 + ia) * nao + d0 + id);
#pragma unroll
                for (int ic = 0; ic < FC; ++ic) Dac[ia][ic] = (R)__ldg(D + (long long)(a0 + ia) * nao + c0 + ic);
            }
            R kac[FA][FC], kad[FA][FD], kbc[FB][FC], kbd[FB][FD];
#pragma unroll
            for (int ia = 0; ia < FA; ++ia) {
#pragma unroll
                for (int ic = 0; ic < FC; ++ic) kac[ia][ic] = (R)0;
#pragma unroll
                for (int id = 0; id < FD; ++id) kad[ia][id] = (R)0;
            }
#pragma unroll
            for (int ib = 0; ib < FB; ++ib) {
#pragma unroll
                for (int ic = 0; ic < FC; ++ic) kbc[ib][ic] = (R)0;
#pragma unroll
                for (int id = 0; id < FD; ++id) kbd[ib][id] = (R)0;
            }
#pragma unroll
            for (int ia = 0; ia < FA; ++ia)
#pragma unroll
                for (int ib = 0; ib < FB; ++ib)
#pragma unroll
                    for (int ic = 0; ic < FC; ++ic)
#pragma unroll
                        for (int id = 0; id < FD; ++id) {
                            const R t = T[((ia * FB + ib) * FC + ic) * FD + id];
                            kac[ia][ic] += t * Dbd[ib][id];
                            kad[ia][id] += t * Dbc[ib][ic];
                            kbc[ib][ic] += t * Dad[ia][id];
                            kbd[ib][id] += t * Dac[ia][ic];
                        }
            double *K = mol.K + m * nn;
#pragma unroll
            for (int ia = 0; ia < FA; ++ia) {
#pragma unroll
                for (int ic = 0; ic < FC; ++ic)
                    jk_red_add(K + (long long)(a0 + ia) * nao + c0 + ic, jk_wide(f * kac[ia][ic], wi));
#pragma unroll
                for (int id = 0; id < FD; ++id)
                    jk_red_add(K + (long long)(a0 + ia) * nao + d0 + id, jk_wide(f * kad[ia][id], wi));
            }
#pragma unroll
            for (int ib = 0; ib < FB; ++ib) {
#pragma unroll
                for (int ic = 0; ic < FC; ++ic)
                    jk_red_add(K + (long long)(b0 + ib) * nao + c0 + ic, jk_wide(f * kbc[ib][ic], wi));
#pragma unroll
                for (int id = 0; id < FD; ++id)
                    jk_red_add(K + (long long)(b0 + ib) * nao + d0 + id, jk_wide(f * kbd[ib][id], wi));
            }
        }
    }
}

template <int FA, int FB, int NDM, typename R>
__device__ __forceinline__ void jk_flush_jab(R (&jab)[NDM][FA][FB], const JkMol &mol, int a0, int b0, int wi)
{
    const long long nn = (long long)mol.nao * mol.nao;
#pragma unroll
    for (int m = 0; m < NDM; ++m)
#pragma unroll
        for (int ia = 0; ia < FA; ++ia)
#pragma unroll
            for (int ib = 0; ib < FB; ++ib)
                if (jab[m][ia][ib] != (R)0)
                    jk_red_add(mol.J + m * nn + (long long)(a0 + ia) * mol.nao + b0 + ib, jk_wide(jab[m][ia][ib], wi));
}

// Work item t -> bra pair i (binary search in the item prefix) and the ket
// range of its chunk. The last chunk of a bra runs to the molecule's last
// ket, so the partition covers every candidate whatever the estimate was.
__device__ __forceinline__ int jk_item_bra(const JkClassArgs &args, long long t)
{
    int lo = 0, hi = args.nbra - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(args.item_prefix + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------- the class kernel
// Persistent: warps (or, for groups of more than 32 threads, whole CTAs)
// take work items from a global counter until none are left. A group of
// more than 256 threads (the largest classes, e.g. (gg|gg)) is split over
// X CTAs: work item t is slab t % X of quartet item t / X, each CTA builds
// the roots and 2D tables itself and evaluates the elements of its G / X
// threads.
template <int LA, int LB, int LC, int LD, int NPA, int NPB, int NPC, int NPD,
          int GA, int GB, int GC, int GD, int X, int NDM, int DOJ, int DOK, typename R, int MODE, int OP>
__global__ void __launch_bounds__(JkShape<LA, LB, LC, LD, GA, GB, GC, GD>::G <= 32 ? 128
                                  : ((JkShape<LA, LB, LC, LD, GA, GB, GC, GD>::G / X + 31) / 32) * 32)
jk_class_kernel(const JkClassArgs args)
{
    typedef JkShape<LA, LB, LC, LD, GA, GB, GC, GD, OP> S;
    constexpr int G = S::G;
    constexpr int FA = S::FA, FB = S::FB, FC = S::FC, FD = S::FD;
    extern __shared__ __align__(16) double jk_smem_raw[];
    const int lane = threadIdx.x & 31;
    const typename JkPP<R>::T *pp = jk_pp<R>(args);
    const R *rys = jk_rys<R>(args);
    // The FP32 tier reads its Rys table from shared memory: lanes gather
    // coefficients of unrelated intervals, which from global memory costs one
    // L1 wavefront per lane and load. Only this class's N-root table, copied
    // once per (persistent) CTA, ahead of the groups' 2D tables.
    R *smem_groups = reinterpret_cast<R *>(jk_smem_raw);
    if constexpr (JkIsFloat<R>::v) {
        constexpr int NT = JkRysTab32<S::NR>::n, V = 4 * S::NR;   // float4 per interval (unpadded)
        static_assert(NT % 4 == 0, "whole float4 vectors");
        float4 *dst = reinterpret_cast<float4 *>(jk_smem_raw);
        const float4 *src = reinterpret_cast<const float4 *>(args.rys32 + rys32_offset[S::NR]);
        for (int i = threadIdx.x; i < rys32_nint_c[S::NR] * V; i += blockDim.x)
            dst[(i / V) * (V + 1) + i % V] = __ldg(src + i);
        __syncthreads();
        rys = reinterpret_cast<const R *>(jk_smem_raw);
        smem_groups = reinterpret_cast<R *>(jk_smem_raw) + NT;
    }

    static_assert(X == 1 || (G > 32 && G % X == 0), "a split group spans whole CTAs");
    if constexpr (G <= 32) {
        constexpr int NGW = 32 / G;
        const int wib = threadIdx.x >> 5;
        const int gw = lane / G, tg = lane - gw * G;
        const bool active = gw < NGW;
        const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((active ? gw : 0) * G));
        R *grp = smem_groups + (size_t)(wib * NGW + (active ? gw : 0)) * S::SMEM_GROUP;
        // router scratch, 1 KB per warp (MODE 1)
        __shared__ __align__(16) unsigned short s_rsm[MODE == 1 ? 4 * 32 * JK_RT_NINP : 2];
        // ket queue per warp: at most NGW - 1 + 32 entries; band queue (MODE 1):
        // at most 31 + 32
        __shared__ int s_qk[4][64];
        __shared__ float s_qd[4][64];
        __shared__ int s_bk[4][MODE == 1 ? 64 : 1];
        __shared__ float s_bd[4][MODE == 1 ? 64 : 1], s_bb[4][MODE == 1 ? 64 : 1];
        unsigned short *rsm = s_rsm + (MODE == 1 ? wib * 32 * JK_RT_NINP : 0);
        const int gd = tg % GD, gc = (tg / GD) % GC, gb = (tg / (GD * GC)) % GB, ga = tg / (GD * GC * GB);
        JkOffsets<S> off;
        jk_make_offsets<LA, LB, LC, LD, GA, GB, GC, GD, S>(ga, gb, gc, gd, off);
        if constexpr (MODE == 3) {
            // FP32 list kernel of a routed build: the band quartets the FP64
            // tier released, one per group; each bra's J block is flushed on
            // its own (the quartets of a warp belong to unrelated bras)
            const long long n = min((long long)*args.rcount, args.rcap);
            unsigned long long nq = 0, nprim = 0;
            for (;;) {
                long long t = 0;
                if (lane == 0) t = (long long)atomicAdd(args.work, (unsigned long long)NGW);
                t = __shfl_sync(0xffffffffu, t, 0);
                if (t >= n) break;
                const long long e = t + gw;
                if (active && e < n) {
                    const JkRouted rq = args.rlist[e];
                    const JkPair bra = args.bra[rq.item];
                    const JkPair ket = args.ket[rq.ket];
                    const JkMol mol = args.mols[bra.mol];
                    R T[S::EPT];
#pragma unroll
                    for (int k = 0; k < S::EPT; ++k) T[k] = (R)0;
                    const int np = jk_quartet<LA, LB, LC, LD, NPA, NPB, NPC, NPD, GA, GB, GC, GD, R, OP>(
                        bra, ket, __fdiv_rn(args.prim_eps32, rq.dmq), args.omega, args.asym64, pp, rys, grp, gmask,
                        tg, true, off, T);
                    R f = (R)1;
                    if (bra.a == bra.b) f *= (R)0.5;
                    if (ket.a == ket.b) f *= (R)0.5;
                    if (args.same_class && rq.ket == rq.item) f *= (R)0.5;
                    R jab[NDM][FA][FB];
#pragma unroll
                    for (int m = 0; m < NDM; ++m)
#pragma unroll
                        for (int i = 0; i < FA; ++i)
#pragma unroll
                            for (int jj = 0; jj < FB; ++jj) jab[m][i][jj] = (R)0;
                    const int a0 = bra.a_ao + ga * FA, b0 = bra.b_ao + gb * FB;
                    jk_contract<FA, FB, FC, FD, NDM, DOJ, DOK, R>(T, f, mol, a0, b0, ket.a_ao + gc * FC,
                                                                 ket.b_ao + gd * FD, jab, args.widen_int);
                    if (DOJ) jk_flush_jab<FA, FB, NDM, R>(jab, mol, a0, b0, args.widen_int);
                    if (tg == 0) { ++nq; nprim += np; }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                nq += __shfl_xor_sync(0xffffffffu, nq, o);
                nprim += __shfl_xor_sync(0xffffffffu, nprim, o);
            }
            if (lane == 0 && nq) {
                atomicAdd(args.stats, nq);
                atomicAdd(args.stats + 1, nprim);
            }
            return;
        }
        for (;;) {
            long long t = 0;
            if (lane == 0) t = args.item_lo + (long long)atomicAdd(args.work, 1ull);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= args.item_hi) break;
            const int item = jk_item_bra(args, t);
            const int ch = (int)(t - __ldg(args.item_prefix + item));
            const int nch = (int)(__ldg(args.item_prefix + item + 1) - __ldg(args.item_prefix + item));
            const JkPair bra = args.bra[item];
            const JkMol mol = args.mols[bra.mol];
            const int kb0 = args.same_class ? item : args.ket_beg[bra.mol];
            const int kend = args.ket_end[bra.mol];
            const int kb = min(kend, kb0 + ch * args.chunk);
            const int ke = (ch == nch - 1) ? kend : min(kend, kb + args.chunk);
            const double *dmx = args.dmax + mol.dmax_off;
            const double dmol = args.use_dmax ? args.dmax_mol[bra.mol] : 1.0;
            const float dmol32 = (float)dmol;
            const int a0 = bra.a_ao + ga * FA, b0 = bra.b_ao + gb * FB;
            JkPairFeat braf;
            if (MODE != 0) braf = args.bra_feat[item];
            R jab[NDM][FA][FB];
#pragma unroll
            for (int m = 0; m < NDM; ++m)
#pragma unroll
                for (int i = 0; i < FA; ++i)
#pragma unroll
                    for (int j = 0; j < FB; ++j) jab[m][i][j] = (R)0;
            unsigned long long nq = 0, nband = 0, nprim = 0;
            // significant kets wait in a per-warp queue (in scan order) until
            // a round can give every group of the warp one; partial rounds
            // only at the end of the item
            // MODE 1: band candidates wait in a second queue and go through
            // the router 32 at a time (one full MMA tile per evaluation);
            // those this tier keeps join the ket queue
            int qn = 0, nb = 0;
            for (int base = kb; base < ke; base += 32) {
                bool sig = false, stop = false, band = false;
                float dmq = 1.0f, B = 0.0f;
                jk_screen_bound<MODE>(args, bra, mol, dmx, dmol, dmol32, base + lane, ke, sig, stop, band, dmq, B);
                const unsigned lt = (1u << lane) - 1u;
                const bool def = sig && !band;   // decided by the bounds alone
                const unsigned mdef = __ballot_sync(0xffffffffu, def);
                nq += __popc(mdef);
                if (def) {
                    const int pos = qn + __popc(mdef & lt);
                    s_qk[wib][pos] = base + lane;
                    s_qd[wib][pos] = dmq;
                }
                qn += __popc(mdef);
                if (MODE == 1) {
                    const unsigned mb = __ballot_sync(0xffffffffu, band);
                    if (band) {
                        const int pos = nb + __popc(mb & lt);
                        s_bk[wib][pos] = base + lane;
                        s_bd[wib][pos] = dmq;
                        s_bb[wib][pos] = B;
                    }
                    nb += __popc(mb);
                }
                __syncwarp();
                const bool last = __any_sync(0xffffffffu, stop) || base + 32 >= ke;
                for (;;) {
                    const bool full_round = qn >= NGW;
                    const bool band_batch = MODE == 1 && !full_round && (nb >= 32 || (last && nb > 0));
                    const bool tail_round = !full_round && !band_batch && last && qn > 0;
                    if (band_batch) {
                        const int take = nb < 32 ? nb : 32;
                        const bool mine = lane < take;
                        const int j = mine ? s_bk[wib][lane] : 0;
                        const float dj = mine ? s_bd[wib][lane] : 1.0f;
                        const float bj = mine ? s_bb[wib][lane] : 2.0f * args.tau32;
                        const JkPairFeat kf = mine ? args.ket_feat[j] : braf;
                        const bool to32 = jk_router_to_fp32_warp(args.router, braf, kf, bj, dj, args.tau32, rsm);
                        // released quartets go to the FP32 list kernel; the
                        // rest of the band stays here, in FP64
                        const bool listed = jk_route_out(args, mine && to32, item, j, dj);
                        const bool keep = mine && !listed;
                        const unsigned mk = __ballot_sync(0xffffffffu, keep);
                        nq += __popc(mk);
                        nband += __popc(__ballot_sync(0xffffffffu, listed));
                        if (keep) {
                            const int pos = qn + __popc(mk & lt);
                            s_qk[wib][pos] = j;
                            s_qd[wib][pos] = dj;
                        }
                        qn += __popc(mk);
                        // drop the evaluated band entries (at most 31 remain)
                        __syncwarp();
                        const int rest = nb - take;
                        int k2 = 0;
                        float d2 = 0.0f, b2 = 0.0f;
                        if (lane < rest) { k2 = s_bk[wib][take + lane]; d2 = s_bd[wib][take + lane]; b2 = s_bb[wib][take + lane]; }
                        __syncwarp();
                        if (lane < rest) { s_bk[wib][lane] = k2; s_bd[wib][lane] = d2; s_bb[wib][lane] = b2; }
                        __syncwarp();
                        nb = rest;
                        continue;
                    }
                    if (!full_round && !tail_round) break;
                    const int take = qn < NGW ? qn : NGW;
                    int myket = -1;
                    float dmk = 1.0f;
                    if (active && gw < take) {
                        myket = s_qk[wib][gw];
                        dmk = s_qd[wib][gw];
                    }
                    if (myket >= 0) {
                        const JkPair ket = args.ket[myket];
                        R T[S::EPT];
#pragma unroll
                        for (int k = 0; k < S::EPT; ++k) T[k] = (R)0;
                        const int np = jk_quartet<LA, LB, LC, LD, NPA, NPB, NPC, NPD, GA, GB, GC, GD, R, OP>(
                            bra, ket, __fdiv_rn(args.prim_eps32, dmk), args.omega, args.asym64, pp, rys, grp, gmask,
                            tg, true,
                            off, T);
                        if (tg == 0) nprim += np;
                        R f = (R)1;
                        if (bra.a == bra.b) f *= (R)0.5;
                        if (ket.a == ket.b) f *= (R)0.5;
                        if (args.same_class && myket == item) f *= (R)0.5;
                        jk_contract<FA, FB, FC, FD, NDM, DOJ, DOK, R>(T, f, mol, a0, b0, ket.a_ao + gc * FC,
                                                                     ket.b_ao + gd * FD, jab, args.widen_int);
                        if (MODE == 2) {
                            double tm = 0.0;
#pragma unroll
                            for (int k = 0; k < S::EPT; ++k) tm = fmax(tm, fabs((double)T[k]));
                            for (int q = 0; q < G; ++q) tm = fmax(tm, __shfl_sync(gmask, tm, (gw * G + q) & 31));
                            if (tg == 0)
                                jk_log_sample(args, bra, ket, braf, args.ket_feat[myket],
                                              jk_quartet_dmax(args, bra, ket, mol, dmx), tm);
                        }
                    }
                    // drop the round's entries (at most 31 remain)
                    __syncwarp();
                    const int rest = qn - take;
                    int k2 = 0;
                    float d2 = 0.0f;
                    if (lane < rest) { k2 = s_qk[wib][take + lane]; d2 = s_qd[wib][take + lane]; }
                    __syncwarp();
                    if (lane < rest) { s_qk[wib][lane] = k2; s_qd[wib][lane] = d2; }
                    __syncwarp();
                    qn = rest;
                }
                if (last) break;
            }
            if (DOJ && active) jk_flush_jab<FA, FB, NDM, R>(jab, mol, a0, b0, args.widen_int);
            for (int o = 16; o > 0; o >>= 1) nprim += __shfl_xor_sync(0xffffffffu, nprim, o);
            if (lane == 0 && nq) {
                atomicAdd(args.stats, nq);
                atomicAdd(args.stats + 1, nprim);
                if (nband) atomicAdd(args.stats + 2, nband);
            }
        }
    } else {
        // one group (or one of its X slabs) per CTA of round_up(G / X, 32) threads
        constexpr int NTC = G / X;
        __shared__ long long s_item;
        __shared__ float s_dm[32];
        __shared__ unsigned s_mask;
        __shared__ int s_stop;
        __shared__ __align__(16) unsigned short s_rsm[MODE == 1 ? 32 * JK_RT_NINP : 2];
        const int tg = threadIdx.x;
        const bool act = tg < NTC;
        const int tgc = act ? tg : 0;
        int gd = tgc % GD, gc = (tgc / GD) % GC, gb = (tgc / (GD * GC)) % GB, ga = tgc / (GD * GC * GB);
        R *grp = smem_groups;
        JkOffsets<S> off;
        jk_make_offsets<LA, LB, LC, LD, GA, GB, GC, GD, S>(ga, gb, gc, gd, off);
        if constexpr (MODE == 3) {
            // FP32 list kernel of a routed build: one released quartet (or one
            // of its X slabs) per CTA at a time
            const long long n = min((long long)*args.rcount, args.rcap);
            unsigned long long nq = 0, nprim = 0;
            for (;;) {
                if (threadIdx.x == 0) s_item = (long long)atomicAdd(args.work, 1ull);
                __syncthreads();
                const long long tt = s_item;
                __syncthreads();
                if (tt >= n * X) break;
                const long long e = X == 1 ? tt : tt / X;
                const int slab = (int)(tt - e * X);
                if constexpr (X > 1) {
                    const int tgl = slab * NTC + tgc;
                    gd = tgl % GD; gc = (tgl / GD) % GC; gb = (tgl / (GD * GC)) % GB; ga = tgl / (GD * GC * GB);
                    jk_make_offsets<LA, LB, LC, LD, GA, GB, GC, GD, S>(ga, gb, gc, gd, off);
                }
                const JkRouted rq = args.rlist[e];
                const JkPair bra = args.bra[rq.item];
                const JkPair ket = args.ket[rq.ket];
                const JkMol mol = args.mols[bra.mol];
                R T[S::EPT];
#pragma unroll
                for (int k = 0; k < S::EPT; ++k) T[k] = (R)0;
                const int np = jk_quartet<LA, LB, LC, LD, NPA, NPB, NPC, NPD, GA, GB, GC, GD, R, OP, NTC>(
                    bra, ket, __fdiv_rn(args.prim_eps32, rq.dmq), args.omega, args.asym64, pp, rys, grp, 0u, tg, act,
                    off, T);
                if (act) {
                    R f = (R)1;
                    if (bra.a == bra.b) f *= (R)0.5;
                    if (ket.a == ket.b) f *= (R)0.5;
                    if (args.same_class && rq.ket == rq.item) f *= (R)0.5;
                    R jab[NDM][FA][FB];
#pragma unroll
                    for (int m = 0; m < NDM; ++m)
#pragma unroll
                        for (int i = 0; i < FA; ++i)
#pragma unroll
                            for (int jj = 0; jj < FB; ++jj) jab[m][i][jj] = (R)0;
                    const int a0 = bra.a_ao + ga * FA, b0 = bra.b_ao + gb * FB;
                    jk_contract<FA, FB, FC, FD, NDM, DOJ, DOK, R>(T, f, mol, a0, b0, ket.a_ao + gc * FC,
                                                                 ket.b_ao + gd * FD, jab, args.widen_int);
                    if (DOJ) jk_flush_jab<FA, FB, NDM, R>(jab, mol, a0, b0, args.widen_int);
                }
                if (slab == 0) { ++nq; nprim += np; }
                // every thread is done with this entry's shared tables
                __syncthreads();
            }
            if (threadIdx.x == 0 && nq) {
                atomicAdd(args.stats, nq);
                atomicAdd(args.stats + 1, nprim);
            }
            return;
        }
        for (;;) {
            if (threadIdx.x == 0) s_item = args.item_lo + (long long)atomicAdd(args.work, 1ull);
            __syncthreads();
            const long long tt = s_item;
            __syncthreads();
            if (tt >= args.item_hi) break;
            const long long t = X == 1 ? tt : tt / X;
            const int slab = (int)(tt - t * X);
            if constexpr (X > 1) {
                // this CTA's share of the group: logical threads slab * NTC + tg
                const int tgl = slab * NTC + tgc;
                gd = tgl % GD; gc = (tgl / GD) % GC; gb = (tgl / (GD * GC)) % GB; ga = tgl / (GD * GC * GB);
                jk_make_offsets<LA, LB, LC, LD, GA, GB, GC, GD, S>(ga, gb, gc, gd, off);
            }
            const int item = jk_item_bra(args, t);
            const int ch = (int)(t - __ldg(args.item_prefix + item));
            const int nch = (int)(__ldg(args.item_prefix + item + 1) - __ldg(args.item_prefix + item));
            const JkPair bra = args.bra[item];
            const JkMol mol = args.mols[bra.mol];
            const int kb0 = args.same_class ? item : args.ket_beg[bra.mol];
            const int kend = args.ket_end[bra.mol];
            const int kb = min(kend, kb0 + ch * args.chunk);
            const int ke = (ch == nch - 1) ? kend : min(kend, kb + args.chunk);
            const double *dmx = args.dmax + mol.dmax_off;
            const double dmol = args.use_dmax ? args.dmax_mol[bra.mol] : 1.0;
            const float dmol32 = (float)dmol;
            const int a0 = bra.a_ao + ga * FA, b0 = bra.b_ao + gb * FB;
            JkPairFeat braf;
            if (MODE != 0) braf = args.bra_feat[item];
            R jab[NDM][FA][FB];
#pragma unroll
            for (int m = 0; m < NDM; ++m)
#pragma unroll
                for (int i = 0; i < FA; ++i)
#pragma unroll
                    for (int j = 0; j < FB; ++j) jab[m][i][j] = (R)0;
            unsigned long long nq = 0, nband = 0, nprim = 0;
            for (int base = kb; base < ke; base += 32) {
                if (threadIdx.x < 32) {
                    bool sig, stop, band;
                    float dmq;
                    jk_screen<MODE>(args, bra, braf, mol, dmx, dmol, dmol32, item, base + lane, ke, sig, stop, band, dmq,
                                    s_rsm);
                    s_dm[lane] = dmq;
                    const unsigned msk = __ballot_sync(0xffffffffu, sig);
                    const int anystop = __any_sync(0xffffffffu, stop);
                    const unsigned bmsk = __ballot_sync(0xffffffffu, band);
                    if (lane == 0) { s_mask = msk; s_stop = anystop; nband += __popc(bmsk); }
                }
                __syncthreads();
                unsigned mask = s_mask;
                const int stop = s_stop;
                __syncthreads();
                nq += __popc(mask);
                while (mask) {
                    const int myket = base + __ffs(mask) - 1;
                    mask &= mask - 1;
                    const JkPair ket = args.ket[myket];
                    R T[S::EPT];
#pragma unroll
                    for (int k = 0; k < S::EPT; ++k) T[k] = (R)0;
                    const int np = jk_quartet<LA, LB, LC, LD, NPA, NPB, NPC, NPD, GA, GB, GC, GD, R, OP, NTC>(
                        bra, ket, __fdiv_rn(args.prim_eps32, s_dm[myket - base]), args.omega, args.asym64, pp, rys,
                        grp, 0u, tg,
                        act, off, T);
                    nprim += np;
                    if (act) {
                        R f = (R)1;
                        if (bra.a == bra.b) f *= (R)0.5;
                        if (ket.a == ket.b) f *= (R)0.5;
                        if (args.same_class && myket == item) f *= (R)0.5;
                        jk_contract<FA, FB, FC, FD, NDM, DOJ, DOK, R>(T, f, mol, a0, b0, ket.a_ao + gc * FC,
                                                                     ket.b_ao + gd * FD, jab, args.widen_int);
                    }
                    if (MODE == 2 && X == 1) {   // labels need the whole block's max |T|
                        __shared__ double s_tm[32];
                        double tm = 0.0;
                        if (act) {
#pragma unroll
                            for (int k = 0; k < S::EPT; ++k) tm = fmax(tm, fabs((double)T[k]));
                        }
                        for (int o = 16; o > 0; o >>= 1) tm = fmax(tm, __shfl_xor_sync(0xffffffffu, tm, o));
                        if (lane == 0) s_tm[threadIdx.x >> 5] = tm;
                        __syncthreads();
                        if (threadIdx.x == 0) {
                            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) tm = fmax(tm, s_tm[w]);
                            jk_log_sample(args, bra, ket, braf, args.ket_feat[myket],
                                          jk_quartet_dmax(args, bra, ket, mol, dmx), tm);
                        }
                        __syncthreads();
                    }
                    // every thread has read s_dm for this quartet before warp 0
                    // may screen the next chunk (a quartet can skip all its
                    // primitives and so pass no barrier inside jk_quartet)
                    __syncthreads();
                }
                if (stop) break;
            }
            if (DOJ && act) jk_flush_jab<FA, FB, NDM, R>(jab, mol, a0, b0, args.widen_int);
            if (threadIdx.x == 0 && nq && slab == 0) {
                atomicAdd(args.stats, nq);
                atomicAdd(args.stats + 1, nprim);
                if (nband) atomicAdd(args.stats + 2, nband);
            }
        }
    }
}

// ------------------------------------------------- Schwarz factors Q_ab
// Diagonal quartets (ab|ab) of one pair class in FP64; Q_ab is the square
// root of the largest |(mu nu|mu nu)| (eq:schwartz at shell level).
// A group of more than 1024 threads is split over X CTAs (slab t % X of
// pair t / X); the CTAs combine their maxima by an atomic max on Qout, which
// the caller zeroes.
template <int LA, int LB, int NPA, int NPB, int GA, int GB, int GC, int GD, int X>
__global__ void __launch_bounds__(JkShape<LA, LB, LA, LB, GA, GB, GC, GD>::G <= 32 ? 128
                                  : ((JkShape<LA, LB, LA, LB, GA, GB, GC, GD>::G / X + 31) / 32) * 32)
jk_schwarz_kernel(const JkSchwarzArgs args)
{
    typedef JkShape<LA, LB, LA, LB, GA, GB, GC, GD> S;
    static_assert(GA == GC && GB == GD, "diagonal elements must stay inside one thread");
    static_assert(X == 1 || (S::G > 32 && S::G % X == 0), "a split group spans whole CTAs");
    constexpr int G = S::G;
    constexpr int FA = S::FA, FB = S::FB, FC = S::FC, FD = S::FD;
    extern __shared__ __align__(16) double jk_smem_raw[];
    const int lane = threadIdx.x & 31;
    if constexpr (G <= 32) {
        constexpr int NGW = 32 / G;
        const int wib = threadIdx.x >> 5;
        const int gw = lane / G, tg = lane - gw * G;
        const bool active = gw < NGW;
        const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((active ? gw : 0) * G));
        double *grp = jk_smem_raw + (size_t)(wib * NGW + (active ? gw : 0)) * S::SMEM_GROUP;
        const int gd = tg % GD, gc = (tg / GD) % GC, gb = (tg / (GD * GC)) % GB, ga = tg / (GD * GC * GB);
        JkOffsets<S> off;
        jk_make_offsets<LA, LB, LA, LB, GA, GB, GC, GD, S>(ga, gb, gc, gd, off);
        const int warps_total = (gridDim.x * blockDim.x) >> 5;
        const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        for (int base = gwarp * NGW; base < args.npair; base += warps_total * NGW) {
            const int pi = base + gw;
            const bool mine = active && pi < args.npair;
            double mx = 0.0;
            if (mine) {
                const JkPair pr = args.pairs[pi];
                double T[S::EPT];
#pragma unroll
                for (int k = 0; k < S::EPT; ++k) T[k] = 0.0;
                jk_quartet<LA, LB, LA, LB, NPA, NPB, NPA, NPB, GA, GB, GC, GD, double>(pr, pr, -1.0f, 0.0, 0, args.pp64, args.rys64, grp, gmask, tg, true, off, T);
                if (ga == gc && gb == gd) {
#pragma unroll
                    for (int ia = 0; ia < FA; ++ia)
#pragma unroll
                        for (int ib = 0; ib < FB; ++ib)
                            mx = fmax(mx, fabs(T[((ia * FB + ib) * FC + ia) * FD + ib]));
                }
            }
            double gmx = mx;
            for (int q = 0; q < G; ++q) gmx = fmax(gmx, __shfl_sync(0xffffffffu, mx, (gw * G + q) & 31));
            if (mine && tg == 0) args.Qout[pi] = sqrt(gmx);
            __syncwarp();
        }
    } else {
        constexpr int NTC = G / X;
        __shared__ double s_max[32];
        const int tg = threadIdx.x;
        const bool act = tg < NTC;
        const int tgc = act ? tg : 0;
        int gd = tgc % GD, gc = (tgc / GD) % GC, gb = (tgc / (GD * GC)) % GB, ga = tgc / (GD * GC * GB);
        double *grp = jk_smem_raw;
        JkOffsets<S> off;
        jk_make_offsets<LA, LB, LA, LB, GA, GB, GC, GD, S>(ga, gb, gc, gd, off);
        for (long long t = blockIdx.x; t < (long long)args.npair * X; t += gridDim.x) {
            const int pi = (int)(t / X), slab = (int)(t - (long long)pi * X);
            if constexpr (X > 1) {
                const int tgl = slab * NTC + tgc;
                gd = tgl % GD; gc = (tgl / GD) % GC; gb = (tgl / (GD * GC)) % GB; ga = tgl / (GD * GC * GB);
                jk_make_offsets<LA, LB, LA, LB, GA, GB, GC, GD, S>(ga, gb, gc, gd, off);
            }
            const JkPair pr = args.pairs[pi];
            double T[S::EPT];
#pragma unroll
            for (int k = 0; k < S::EPT; ++k) T[k] = 0.0;
            jk_quartet<LA, LB, LA, LB, NPA, NPB, NPA, NPB, GA, GB, GC, GD, double, 0, NTC>(
                pr, pr, -1.0f, 0.0, 0, args.pp64, args.rys64, grp, 0u, tg, act, off, T);
            double mx = 0.0;
            if (act && ga == gc && gb == gd) {
#pragma unroll
                for (int ia = 0; ia < FA; ++ia)
#pragma unroll
                    for (int ib = 0; ib < FB; ++ib)
                        mx = fmax(mx, fabs(T[((ia * FB + ib) * FC + ia) * FD + ib]));
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) s_max[threadIdx.x >> 5] = mx;
            __syncthreads();
            if (threadIdx.x == 0) {
                double m2 = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, s_max[w]);
                // non-negative doubles order like their bit patterns
                if (X == 1) args.Qout[pi] = sqrt(m2);
                else atomicMax(reinterpret_cast<unsigned long long *>(args.Qout + pi),
                               (unsigned long long)__double_as_longlong(sqrt(m2)));
            }
            __syncthreads();
        }
    }
}
