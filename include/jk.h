/*
 * jk.h -- C ABI of the GB300 direct-SCF Coulomb/exchange (JK) build.
 *
 * Computes, for one or more densities D (Sec. 2, eq:jk of the paper),
 *     J_ij = sum_kl (ij|kl) D_kl          K_ik = sum_jl (ij|kl) D_jl
 * over contracted Gaussian-type-orbital shells (eq:rys0), with the electron
 * repulsion integrals evaluated by Rys quadrature (eq:rys1, eq:rys2) on the
 * GPU, shell quartets screened by the Schwarz inequality (eq:schwartz) times
 * the largest density element they touch, and the 8-fold permutational
 * symmetry of Sec. 2 (each unique quartet updates two J and four K blocks).
 *
 * Conventions
 *   - Coordinates in bohr; a shell is (atom, l, nprim, prim_off, ao_off,
 *     spherical). Cartesian components are ordered x exponent descending,
 *     then y descending (xx, xy, xz, yy, yz, zz), the order of Sec. 2.
 *   - coeffs[prim_off+i] multiplies the unnormalised primitive
 *     x^lx y^ly z^lz exp(-exps[prim_off+i] r^2): normalisation is folded in
 *     by the caller.
 *   - spherical == 1 shells use real solid harmonics (m = -l..l; p stays
 *     x, y, z). D is then given and J, K returned in that basis; the
 *     Cartesian transform runs on the device (the paper does it outside the
 *     integral kernel, Sec. 2).
 *   - D, J, K: device pointers, n_dm x nao x nao, FP64, row major. D must
 *     be symmetric (the symmetry of Sec. 2 assumes it). J and K are
 *     overwritten. A NULL J (K) is allowed when with_j (with_k) is 0.
 *
 * Ownership and streams
 *   - jk_init copies the basis to the device and owns every device buffer it
 *     makes (pair tables, screening tables, scratch) until jk_destroy.
 *   - The caller owns D, J, K and the CUDA stream. jk_build enqueues its
 *     work on `stream` (NULL = legacy default stream) and returns without
 *     synchronising, unless `stats` is non-NULL: then it synchronises the
 *     stream to fill the counters and to check the device error word.
 *   - A handle is not thread-safe: one build at a time per handle.
 *
 * Errors
 *   Every call returns JK_OK or an error code; jk_last_error() gives a
 *   message for the calling thread. No call aborts the process, traps on the
 *   GPU or throws across the ABI. The kernels report a non-finite density
 *   element through a device error word: a build with stats checks it
 *   before returning; a build without stats queues a copy of it on the
 *   stream, and the next call on the handle (jk_build*, jk_check,
 *   jk_destroy) that finds the copy landed returns JK_ERR_NAN. No kernel of
 *   the library waits on another kernel or on the host, so JK_ERR_TIMEOUT is
 *   reserved and returned by no call.
 */
#ifndef JK_H
#define JK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    JK_OK = 0,
    JK_ERR_ARG = 1,          /* bad argument (NULL pointer, size, flag) */
    JK_ERR_UNSUPPORTED = 2,  /* l > JK_LMAX, nprim > JK_NPRIM_MAX, n_dm > JK_NDM_MAX */
    JK_ERR_CUDA = 3,         /* a CUDA runtime or driver call failed */
    JK_ERR_OOM = 4,          /* device allocation failed or above the memory cap */
    JK_ERR_TIMEOUT = 5,      /* reserved: no call returns it (no device-side waits) */
    JK_ERR_NAN = 6,          /* non-finite density or result detected */
    JK_ERR_COMPILE = 7       /* runtime kernel compilation failed */
};

enum {
    JK_PREC_FP64 = 0,          /* every quartet in FP64 */
    JK_PREC_MIXED = 1,         /* Schwarz x density-max tiering: FP64 above tau32, FP32 below */
    JK_PREC_MIXED_ROUTED = 2,  /* MIXED plus the learned router inside (tau32, K*tau32] */
    JK_PREC_FP32 = 3           /* every quartet in FP32 (FP64 accumulation of J/K) */
};

#define JK_LMAX 4
#define JK_NPRIM_MAX 16
#define JK_NDM_MAX 4

typedef struct {
    int32_t atom, l, nprim, prim_off, ao_off, spherical;
} jk_shell;

typedef struct {
    int64_t quartets_fp64;    /* significant unique shell quartets evaluated in FP64 */
    int64_t quartets_fp32;    /* ... in FP32 */
    int64_t quartets_routed;  /* band quartets the router moved to FP32 (part of quartets_fp32) */
    int64_t prim_quartets;    /* primitive quartets evaluated (both tiers) */
    double flops_model;       /* modelled FLOPs of the integral kernels (per-class count model) */
    double ms;                /* device time of the build, CUDA events on `stream` */
    int64_t kernel_launches;  /* kernels this build launched (integral + helper kernels) */
} jk_stats;

/* Per-launch record of the last build made with option "profile" = 1. */
typedef struct {
    int32_t la, lb, lc, ld, na, nb, nc, nd;  /* class: angular momenta, primitive counts */
    int32_t tier;                            /* 0 FP64, 1 FP32 */
    int32_t threads_per_quartet;             /* fragmentation (1 = one quartet per thread) */
    int32_t regs, local_bytes;               /* registers per thread, local (spill) bytes */
    int64_t quartets, prim_quartets;         /* significant quartets it evaluated */
    double ms;                               /* CUDA-event time of the launch on the build stream */
    double flops_model;                      /* modelled FLOPs of those quartets */
} jk_launch_prof;

/* Learned precision router (the MIXED_ROUTED mode): a 12 -> 64 -> 64 -> 1
 * MLP, BF16 weights in use, FP32 accumulation. It predicts, for a quartet in
 * the band tau32 < B <= K tau32 (B = Q_ab Q_cd Dmax), y = log10(max|T| / (Q_ab
 * Q_cd)), and the quartet runs in FP32 iff log10(B / tau32) + y + margin <= 0.
 * In a routed build the FP64 tier screens the band and runs the router; the
 * quartets it releases are evaluated by an FP32 list kernel per class pair,
 * and the FP32 tier itself keeps the plain Schwarz split (B <= tau32).
 * theta is the FP32 master copy, flat: W1[16][64] b1[64] W2[64][64] b2[64]
 * W3[64] b3 (inputs padded to 16, rows 12..15 unused). The features are
 * normalised as (x - mu) * isd. */
#define JK_ROUTER_NIN 12
#define JK_ROUTER_NPARAM 5313
#define JK_ROUTER_MAGIC 0x4a4b5254u
typedef struct {
    uint32_t magic;     /* JK_ROUTER_MAGIC */
    uint32_t version;   /* 1 */
    float mu[16], isd[16];
    float theta[JK_ROUTER_NPARAM];
    float margin;       /* added to the prediction before the routing test */
    float quantile;     /* the pinball-loss quantile it was trained with */
} jk_router_blob;

typedef struct {
    int32_t steps;      /* optimiser steps */
    int32_t batch;      /* samples per step */
    float lr;           /* Adam learning rate */
    float quantile;     /* pinball-loss quantile in (0, 1) */
    uint64_t seed;      /* initialisation and sampling */
} jk_train_opts;

typedef struct {
    double loss_first, loss_last;  /* mean pinball loss of the first / last 50 steps */
    double ms;                     /* wall time of the training */
} jk_train_stats;

typedef struct jk_handle jk_handle;

/* One molecule: the dynamic inputs of Table 2 of the paper (coordinates,
 * exponents, contraction coefficients) grouped into shells whose (l, nprim)
 * are the static parameters of Table 1. Builds the shell-pair data that
 * Sec. 3 says may be precomputed, and the shell-level Schwarz factors of
 * eq:schwartz. shells: nshell records (host); coords: natm x 3 (host,
 * bohr); exps, coeffs: nprim_total (host). On success *out owns a new
 * handle. Errors: JK_ERR_ARG (NULL, negative sizes, shell fields out of
 * range), JK_ERR_UNSUPPORTED (l or nprim above the limits), JK_ERR_CUDA,
 * JK_ERR_OOM, JK_ERR_COMPILE. */
int jk_init(const jk_shell *shells, int32_t nshell, const double *coords, int32_t natm,
            const double *exps, const double *coeffs, int32_t nprim_total, jk_handle **out);

/* Several independent molecules in one handle (batched builds). Molecule m
 * owns shells [mol_shell_off[m], mol_shell_off[m+1]); shell atom indices are
 * global into coords, prim_off global into exps/coeffs, ao_off local to the
 * molecule. */
int jk_init_batch(int32_t nmol, const int32_t *mol_shell_off, const jk_shell *shells,
                  int32_t nshell, const double *coords, int32_t natm, const double *exps,
                  const double *coeffs, int32_t nprim_total, jk_handle **out);

/* J and K for a single-molecule handle (see the conventions above).
 * cutoff: quartets with Q_ab Q_cd Dmax <= cutoff are skipped (the paper uses
 * 1e-13); the bound and the tier thresholds are compared in FP64 (option
 * "screen64" = 0: in FP32 for cutoff >= 1e-30, every tier alike, so each
 * quartet still runs exactly once). precision_mode: JK_PREC_*. stats may be NULL. */
int jk_build(jk_handle *h, const double *D, int32_t n_dm, int with_j, int with_k, double cutoff,
             int precision_mode, double *J, double *K, void *stream, jk_stats *stats);

/* Batched build: D[m], J[m], K[m] are host arrays of nmol device pointers,
 * one per molecule of the handle; every molecule is processed by the same
 * per-class persistent kernels, captured once into a CUDA graph and
 * replayed on later calls with the same flags. */
int jk_build_batch(jk_handle *h, const double *const *D, int32_t n_dm, int with_j, int with_k,
                   double cutoff, int precision_mode, double *const *J, double *const *K,
                   void *stream, jk_stats *stats);

/* Options (double-valued): "tau32" (FP32 tier threshold on Q_ab Q_cd Dmax,
 * default 1e-4), "router_band" (K, default 100), "pair_cutoff" (shell pairs
 * with Q_ab at or below it are dropped at init, default 1e-18),
 * "use_graph" (0/1), "use_dmax" (0/1: 0 screens with Dmax := 1),
 * "profile" (0/1: CUDA events around every integral launch, see jk_profile;
 * they become event nodes when the build is captured into a graph),
 * "omega" (range separation, Table 1 rys_type of the paper: 0 the Coulomb
 * operator 1/r; w > 0 the long-range erf(w r)/r; w < 0 the short-range
 * erfc(|w| r)/r; the Schwarz factors of 1/r bound both),
 * "prim_eps" (primitive quartets with q_ij q_kl Dmax <= min(prim_eps,
 * cutoff) are skipped; q is the primitive-pair Schwarz factor; default 1e-16),
 * "part_count", "part_index" (a build computes only part part_index of
 * part_count of every class kernel's work; J and K are then partial sums
 * whose sum over the parts is the full result, i.e. one sum all-reduce
 * combines GPUs that split one batch),
 * "branches" (1..8: class kernels forked over this many streams / graph
 * branches),
 * "chunk" (32..65536, default 64: candidate kets per work item of the
 * persistent class kernels; changing it re-plans the work items),
 * "asym64" (0/1, default 0: the FP32 tier evaluates the large-T
 * Gauss-Hermite limit of the Rys roots and weights in FP64 and rounds the
 * result to FP32, instead of evaluating it in FP32),
 * "chunk_fp64tier" (default 512: the same for the FP64 tier of mixed and
 * routed builds, whose kernels keep only the candidates above tau32),
 * "widen_int" (0/1, default 0: the FP32 tier widens its contributions to
 * FP64 for the J/K reductions with the conversion instruction, which runs on the
 * FP64 pipe; 1 builds the FP64 bit pattern with integer operations),
 * "screen64" (0/1, default 1: the screening bounds, tier thresholds and
 * the primitive threshold decide as FP64 compares would: the compare runs
 * in FP32 and is redone in FP64 when the two sides are within a relative
 * 2e-6 of each other; 0 keeps the plain FP32 compare when the cutoff is
 * >= 1e-30),
 * "route_cap" (default 16777216: initial entries of the per-class-pair lists
 * of quartets the router releases from the FP64 tier, shared out by
 * candidate count; a list that overflowed in a build with stats is grown
 * for the next build; a released quartet that finds its list full stays in
 * FP64). With "use_graph" = 1 the first build of a flag combination is
 * captured into a CUDA graph on an internal stream and replayed on `stream`
 * by later builds; the per-call D/J/K pointers are read from a device
 * descriptor copied before each launch, so changing buffers is allowed.
 * JK_ERR_ARG for an unknown key. */
int jk_set_option(jk_handle *h, const char *key, double value);
/* Reads any option above, and the read-only figures "graphs" (captured
 * graphs held), "init_ms" (jk_init wall time), "compile_ms" (NVRTC time spent
 * by this handle), "npairs", "nclasses", "nlaunches" (significant shell
 * pairs, pair classes, class-pair launches per tier). JK_ERR_ARG for an
 * unknown key. */
int jk_get_option(jk_handle *h, const char *key, double *value);

/* Number of molecules, basis functions of molecule m (in the basis D is
 * given in), shells. */
int jk_info(jk_handle *h, int32_t mol, int32_t *nao, int32_t *nshell, int32_t *nmol);

/* Schwarz factors Q_ab of molecule 0 into a host nshell x nshell array
 * (zero for pairs dropped at init). */
int jk_schwarz(jk_handle *h, double *Q_host);

/* Synchronises `stream` and reports the device error word of the builds
 * enqueued on this handle so far (JK_ERR_NAN for a non-finite density
 * element), clearing it. The asynchronous counterpart of passing stats. */
int jk_check(jk_handle *h, void *stream);

/* Releases a handle (resource management; no passage of the paper).
 * Synchronises the device, then frees everything the handle owns (device
 * tables and scratch, captured graphs, streams, events); the caller's D, J
 * and K are untouched. JK_ERR_ARG for NULL; JK_ERR_NAN (after freeing) when
 * a build whose error word nobody looked at saw a non-finite density. */
int jk_destroy(jk_handle *h);

/* Router training data from a full FP64 build (which it also returns in J,
 * K): for every quartet the build evaluates inside the band (tau32, K tau32]
 * it writes the 12 features to X[i*12..] and the label y = log10(max|T| /
 * (Q_ab Q_cd)) to y[i] (X, y: device, capacity cap); *n receives the number
 * of band quartets seen (only the first cap are written). Synchronises. */
int jk_router_collect(jk_handle *h, const double *const *D, int32_t n_dm, double cutoff, double *const *J,
                      double *const *K, float *X, float *y, int64_t cap, int64_t *n, void *stream);

/* Train the router on the device with the library's own forward/backward
 * kernels (Adam, pinball loss). X: n x 12, y: n (device). Writes the result
 * to *out (host). Feature normalisation is computed from X. */
int jk_router_train(const float *X, const float *y, int64_t n, const jk_train_opts *opts, jk_router_blob *out,
                    jk_train_stats *stats);

/* Predictions (margin included) for n feature rows (device in and out). */
int jk_router_forward(const jk_router_blob *w, const float *X, int64_t n, float *y_out);

/* Mean pinball loss over the n rows and its gradient with respect to theta
 * (host array of JK_ROUTER_NPARAM), from the training kernel's backward
 * pass. X, y: device. */
int jk_router_gradient(const jk_router_blob *w, const float *X, const float *y, int64_t n, float quantile,
                       float *grad_host, double *loss);

/* The same result as jk_router_gradient (mean pinball loss and gradient over
 * n rows; X, y on the device; grad_host and loss on the host), from a variant
 * that makes no device allocation. The paper has no counterpart. It is for
 * callers that must not call cudaMalloc: applications whose own allocator
 * (a framework's caching pool, a server that reserves the GPU's memory at
 * start-up) owns every byte of device memory and forbids libraries to take
 * more, and training loops that cannot afford cudaMalloc / cudaFree in the
 * step (cudaFree synchronises the whole device).
 *   - Scratch: one fixed __device__ array in the library (about 560 KB,
 *     present on every GPU that loads the library until the process exits),
 *     holding the weight copies, the row list and the accumulators. At most
 *     JK_NOALLOC_MAX_ROWS rows per call; larger n returns JK_ERR_UNSUPPORTED
 *     and touches nothing.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     process; make that first call before any stream capture. The kept
 *     address does not survive cudaDeviceReset: do not call this after one.
 *   - Every call shares the array and clears the accumulators itself; calls
 *     whose work overlaps on the GPU (other streams, other host threads)
 *     race on it. Work is queued on `stream`; the call synchronises `stream`
 *     and returns with grad_host and loss filled. */
#define JK_NOALLOC_MAX_ROWS 65536
int jk_router_gradient_noalloc(const jk_router_blob *w, const float *X, const float *y, int64_t n, float quantile,
                               float *grad_host, double *loss, void *stream);

/* Install router weights on a handle (enables JK_PREC_MIXED_ROUTED). The
 * router extends the Schwarz-based FP32/FP64 split that Sec. 6 of the paper
 * leaves as future work; the paper itself has no learned router. The blob is
 * copied (BF16-rounded, in MMA fragment order) to the device; the caller
 * keeps it. JK_ERR_ARG for a NULL handle or a blob with a wrong magic or
 * version, JK_ERR_NAN for non-finite weights. */
int jk_router_load(jk_handle *h, const jk_router_blob *w);

/* After a build with option "profile" = 1 and non-NULL stats: copies up to
 * `max` launch records into out and their count into *n. */
int jk_profile(jk_handle *h, jk_launch_prof *out, int32_t max, int32_t *n);

/* FMA-chain throughput of the current device, FLOP/s (FMA = 2):
 * which = 0 FP64, 1 FP32. Runs for about `ms` milliseconds. */
int jk_measure_peak(int32_t which, double ms, double *flops_per_s);

/* Ahead-of-time compilation of one class kernel (angular momenta la..ld,
 * primitive counts na..nd, n_dm, flags, fp32 = 1 for the FP32 tier, mode 0
 * plain / 1 routed FP64 tier (runs the router on its band) / 2 router-label
 * logging (FP64) / 3 routed FP32 list kernel (the quartets mode 1 released),
 * op 0 1/r / 1 erf / 2 erfc) into
 * the on-disk kernel cache (JK_KERNEL_CACHE, else next to the library).
 * Needs no GPU. *threads_per_quartet receives the fragmentation chosen.
 * JK_ERR_COMPILE with the NVRTC log in jk_last_error() on failure. */
int jk_compile_class(int32_t la, int32_t lb, int32_t lc, int32_t ld, int32_t na, int32_t nb, int32_t nc,
                     int32_t nd, int32_t n_dm, int32_t with_j, int32_t with_k, int32_t fp32, int32_t mode,
                     int32_t op, int32_t *threads_per_quartet, double *compile_ms);

/* Ahead-of-time compilation (no GPU needed) of every kernel a basis with
 * these shell types needs: the Schwarz kernels (contracted and primitive)
 * and the class kernels for n_dm, the flags, fp32 and mode (as in
 * jk_compile_class, operator 1/r), in parallel, into the disk cache.
 * *nkernels receives the number of kernels considered. */
int jk_compile_basis(const jk_shell *shells, int32_t nshell, int32_t n_dm, int32_t with_j, int32_t with_k,
                     int32_t fp32, int32_t mode, double *compile_ms, int32_t *nkernels);

/* Result of jk_autotune. */
typedef struct {
    int32_t launches_tuned;    /* class-pair launches (per tier) that had more than one candidate */
    int32_t candidates_timed;  /* candidate kernels timed in all */
    int32_t changed;           /* launches whose fragment shape changed */
    int32_t pad;
    double ms_before;          /* summed launch times of those launches with their previous shapes */
    double ms_after;           /* ... with the chosen shapes */
    double tune_s;             /* wall time of the tuning, compilation included */
} jk_tune_report;

/* Autotuner: the per-device grid search over fragmentations (threads per
 * quartet and how they split the four shells' Cartesian components) of
 * Sec. 3.2 of arXiv 2507.09772, run on the caller's data. Every class-pair
 * launch of the tiers `precision_mode` uses whose estimated share of the
 * work is at least min_share gets up to max_candidates (1..16) shapes
 * (jk_fragment_candidates); each is timed by CUDA events around its launch in
 * two serialised builds of D (arguments as jk_build_batch: n_dm densities per
 * molecule, J and K device buffers of the same shape, overwritten), and the
 * fastest is kept. The choices stay in the handle (captured graphs are
 * dropped) and are written to the tuning table (a text file named for the
 * device model in $JK_TUNING_DIR, else in the kernel cache directory), which
 * later jk_init calls on the same device model read. The
 * call synchronises `stream`. report may be NULL. */
int jk_autotune(jk_handle *h, const double *const *D, int32_t n_dm, int with_j, int with_k, double cutoff,
                int precision_mode, double *const *J, double *const *K, void *stream, int32_t max_candidates,
                double min_share, jk_tune_report *report);

/* The autotuner's candidate shapes for class (la lb|lc ld) (fp32 = 1 for the
 * FP32 tier): the built-in heuristic's shape first, then G = 1 where the class
 * is small, then one shape per group size G = ga*gb*gc*gd (2..256, each g
 * dividing its shell's Cartesian size, at most 64 elements per thread),
 * nearest in log2 G first. frag: max_candidates x 4 (ga gb gc gd), host;
 * *n receives the count. Needs no GPU. */
int jk_fragment_candidates(int32_t la, int32_t lb, int32_t lc, int32_t ld, int32_t fp32, int32_t max_candidates,
                           int32_t *frag, int32_t *n);

/* Message of the last error on the calling thread ("" if none). */
const char *jk_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* JK_H */
