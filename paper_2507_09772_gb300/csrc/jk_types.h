// Plain-data records shared by the host planner (nvcc/g++) and the
// runtime-compiled integral kernels (NVRTC). No includes: NVRTC compiles this
// file without the CUDA toolkit headers.
#pragma once

// One significant shell pair (a, b), oriented so that the shell type of a
// (l, then nprim) is >= that of b. Pairs of one pair class are stored
// contiguously, grouped by molecule and sorted by descending Q inside a
// molecule, so that a ket scan can stop at the first Q that fails the bound.
// 16-byte alignment: records that lanes gather load as 16-byte vectors
struct alignas(16) JkPair {
    int a, b;          // global shell indices
    int mol;           // molecule index
    int pp_off;        // first primitive pair (na*nb of them, a-major)
    int a_ao, b_ao;    // molecule-local Cartesian AO offsets
    int a_loc, b_loc;  // molecule-local shell indices (density-max table)
    double Q;          // Schwarz factor sqrt(max |(mu nu|mu nu)|)
    float ABxf, AByf, ABzf;  // A - B rounded to FP32 (the FP32 tier reads these, no conversion)
    int pad0;
    double pad1;
    double ABx, ABy, ABz;  // A - B (horizontal recurrence)
    float Qf;              // Q rounded to FP32 (the FP32 screening path)
    float padf;
};

// Per primitive pair (alpha_i on a, beta_j on b), p = alpha + beta:
//   P    = (alpha A + beta B) / p
//   PA   = P - A
//   K    = c_i c_j exp(-alpha beta |A-B|^2 / p) / p
//   inv2p = 1 / (2 p)
//   q    = primitive Schwarz factor sqrt(max |(ij|ij)|) (coefficients
//          included); a shell pair's primitive pairs are sorted by q,
//          largest first, so primitive loops can stop at the first
//          q_ij q_kl Dmax at or below the primitive threshold
struct alignas(16) JkPrimPair64 {
    double Px, Py, Pz, p;
    double PAx, PAy, PAz, K;
    double inv2p, q;
    float qf, padf;   // qf: q rounded to FP32 (the primitive screen compares in FP32)
    double pad2;
};
struct alignas(16) JkPrimPair32 {
    float Px, Py, Pz, p;
    float PAx, PAy, PAz, K;
    float inv2p, q, pad1, pad2;
};

// Per molecule of a handle.
struct JkMol {
    const double *D;   // n_dm x nao x nao (Cartesian)
    const float *D32;  // the same rounded to FP32, read by the FP32 tier (nullptr when it does not run)
    double *J;         // half-matrix accumulator X, symmetrised after the build
    double *K;         // half-matrix accumulator Y
    int nao;           // Cartesian functions
    int nsh;           // shells
    long long dmax_off;  // offset of this molecule's nsh x nsh block-max table
};

struct JkRouterDev;
struct JkPairFeat;

// A band quartet the learned router released from the FP64 tier: bra pair
// `item` of the launch's bra class, ket pair `ket` of its ket class, and the
// density factor its screening used. The FP32 list kernel (MODE 3) of the
// same class pair evaluates it.
struct alignas(16) JkRouted {
    int item, ket;
    float dmq;
    int pad;
};

// Arguments of one class-pair launch (passed by value).
struct JkClassArgs {
    const JkPair *bra;           // pairs of the bra class
    const JkPair *ket;           // pairs of the ket class
    const int *ket_beg;          // per molecule: first ket index in the ket class
    const int *ket_end;          // per molecule: one past the last
    const JkPrimPair64 *pp64;
    const JkPrimPair32 *pp32;
    const JkMol *mols;
    const double *dmax;          // block max |D| tables, all molecules
    const float *dmax32;         // the same rounded to FP32
    const double *dmax_mol;      // per molecule: max over its table
    const double *rys64;         // FP64 Rys tables
    const float *rys32;          // FP32 Rys tables
    unsigned long long *work;    // work counter (zeroed before the launch)
    const long long *item_prefix;  // nbra + 1: first work item of each bra pair
    long long item_lo, item_hi;  // this build's share of the items [lo, hi) (partitioned builds)
    int chunk;                   // kets per work item (the last item of a bra runs to ket_end)
    double prim_eps;             // skip primitive quartets with q_ij q_kl Dmax <= prim_eps
    double omega;                // |w| of the range-separated operator (OP 1, 2)
    unsigned long long *stats;   // [0] quartets, [1] primitive quartets, [2] routed band quartets
    int *err;                    // device error word
    double lo, hi;               // keep a quartet iff lo < Q_ab Q_cd Dmax <= hi
    // FP32 screening (scr32 = 1, used when the build's cutoff is >= 1e-30 so
    // that no product of interest leaves the FP32 range): the same bounds and
    // the band in FP32; every tier of a build evaluates them identically
    int scr32;
    float lo32, hi32, tau32, band_hi32, prim_eps32;
    int nbra;
    int same_class;              // ket class == bra class: ket index >= bra index
    int with_j, with_k;          // which outputs (and density blocks) to use
    int use_dmax;                // 0: screen with Dmax := 1
    int ndm;
    // learned router (MODE 1) and label logging (MODE 2)
    const JkPairFeat *bra_feat;  // aligned with bra / ket
    const JkPairFeat *ket_feat;
    const JkRouterDev *router;
    double tau;                  // band (tau, band_hi]
    double band_hi;
    int tier;                    // 0: this launch is the FP64 tier, 1: FP32
    float *log_x;                // MODE 2: features (12 per sample)
    float *log_y;                // MODE 2: labels
    unsigned long long *log_n;   // MODE 2: samples written (may exceed log_cap)
    long long log_cap;
    // routed builds: the FP64 tier (MODE 1) appends the band quartets the
    // router releases to this launch's list (while it has room; a quartet
    // that finds it full stays in FP64); the FP32 list kernel (MODE 3) of the
    // class pair evaluates min(*rcount, rcap) entries
    JkRouted *rlist;
    unsigned long long *rcount;
    long long rcap;
    // 1: the FP32 tier evaluates the large-T (Gauss-Hermite) roots and
    // weights in FP64 and rounds them to FP32
    int asym64;
    // 1: the FP32 tier widens its contributions to FP64 with integer bit
    // operations; 0: with the conversion instruction
    int widen_int;
};

// Arguments of the Schwarz (diagonal-quartet) launch of one pair class.
struct JkSchwarzArgs {
    const JkPair *pairs;
    const JkPrimPair64 *pp64;
    const double *rys64;
    double *Qout;                // one per pair
    int npair;
};

// Bits of the device error word. Only the density check sets one today; no
// kernel of the library waits on another kernel or on the host.
#define JK_ERR_DEV_NAN 4
