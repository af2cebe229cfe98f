// Host side of the JK build: input checks, shell/pair planning, runtime
// kernel compilation (NVRTC, sm_103a) with an on-disk binary cache, the
// per-build launch sequence, and the C ABI declared in include/jk.h.
//
// Planning follows Sec. 3 of the paper: the static parameters of a kernel
// (Table 1: angular momenta, primitive counts, fragment sizes, n_dm, do_j,
// do_k, precision) are template arguments of one instantiation compiled at
// run time; the dynamic inputs (Table 2: coordinates, exponents,
// coefficients, D) are device arrays. Screening (eq:schwartz, and the
// density-matrix bound of Sec. 2) happens inside the kernels.
#include "jk.h"
#include "jk_types.h"
#include "jk_util.cuh"
#include "jk_train.cuh"

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <dlfcn.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cctype>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "kernel_src.inc"   // jk_kernel_source[]: jk_types.h + rys_params.cuh + jk_kernels.cuh
#include "rys_tables.inc"   // rys_table64[], rys_table32_src[]

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[2048];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// On failure the runtime's (non-sticky) last-error state is cleared, so that
// it is not reported again by a later, unrelated check.
#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            (void)cudaGetLastError();                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? JK_ERR_OOM : JK_ERR_CUDA, "%s: %s",  \
                        #call, cudaGetErrorString(e_));                                        \
        }                                                                                      \
    } while (0)

// ------------------------------------------------------------ driver API
// Resolved through the runtime so that the library does not link libcuda.
struct Driver {
    CUresult (*moduleLoadData)(CUmodule *, const void *) = nullptr;
    CUresult (*moduleGetFunction)(CUfunction *, CUmodule, const char *) = nullptr;
    CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                             unsigned, CUstream, void **, void **) = nullptr;
    CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*funcGetAttribute)(int *, CUfunction_attribute, CUfunction) = nullptr;
    CUresult (*occupancy)(int *, CUfunction, int, size_t) = nullptr;
    bool ok = false;
};

Driver &drv()
{
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        auto get = [](const char *name, void **fp) {
            cudaDriverEntryPointQueryResult q;
            return cudaGetDriverEntryPointByVersion(name, fp, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess && *fp;
        };
        d.ok = get("cuModuleLoadData", (void **)&d.moduleLoadData) &&
               get("cuModuleGetFunction", (void **)&d.moduleGetFunction) &&
               get("cuLaunchKernel", (void **)&d.launchKernel) &&
               get("cuFuncSetAttribute", (void **)&d.funcSetAttribute) &&
               get("cuFuncGetAttribute", (void **)&d.funcGetAttribute) &&
               get("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void **)&d.occupancy);
    });
    return d;
}

static_assert(sizeof(JkPair) == 96 && sizeof(JkPrimPair64) == 96 && sizeof(JkPrimPair32) == 48 &&
                  sizeof(JkPairFeat) == 32,
              "record sizes are part of the device layout");

// ------------------------------------------------------------ kernel spec
int ncart(int l) { return (l + 1) * (l + 2) / 2; }

struct KSpec {
    int kind = 0;  // 0 class kernel, 1 Schwarz kernel
    int la = 0, lb = 0, lc = 0, ld = 0, na = 1, nb = 1, nc = 1, nd = 1;
    int ga = 1, gb = 1, gc = 1, gd = 1;
    int gx = 1;    // CTAs one group is split over (groups of more than 256 threads)
    int ndm = 1, doj = 1, dok = 1, fp32 = 0;
    int mode = 0;  // 0 plain, 1 routed (learned router in the band), 2 label logging
    int op = 0;    // 0 1/r, 1 erf(w r)/r, 2 erfc(w r)/r

    std::string name() const
    {
        char b[256];
        if (kind == 1)
            snprintf(b, sizeof b, "jk_schwarz_kernel<%d,%d,%d,%d,%d,%d,%d,%d,%d>", la, lb, na, nb, ga, gb, gc, gd, gx);
        else
            snprintf(b, sizeof b, "jk_class_kernel<%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%s,%d,%d>", la,
                     lb, lc, ld, na, nb, nc, nd, ga, gb, gc, gd, gx, ndm, doj, dok, fp32 ? "float" : "double", mode,
                     op);
        return b;
    }
    int G() const { return ga * gb * gc * gd; }
    int nr() const { return ((la + lb + lc + ld) / 2 + 1) * (op == 2 ? 2 : 1); }
    int ni() const { return (la + 1) * (lb + 1) * (lc + 1) * (ld + 1); }
    int smem_group_reals() const { return G() == 1 ? 0 : nr() * 3 * ni() + 2 * nr(); }
    // G <= 32: four warps, each holding 32/G groups; G > 32: one group (or
    // one of its gx slabs) per CTA
    int block() const { return G() <= 32 ? 128 : ((G() / gx + 31) / 32) * 32; }
    // FP32 class kernels keep their N-root Rys table in shared memory
    size_t rys_table_bytes() const
    {
        if (kind != 0 || !fp32) return 0;
        const int n = (la + lb + lc + ld) / 2 + 1;
        // per interval 2 n functions x 8 coefficients, padded by 4 floats
        return (size_t)rys32_nint_host[n] * (2 * n * (rys32_deg_host + 1) + 4) * sizeof(float);
    }
    size_t smem_bytes() const
    {
        const size_t groups = G() <= 32 ? (size_t)4 * (32 / G()) : 1;
        return rys_table_bytes() + groups * smem_group_reals() * (fp32 ? 4 : 8);
    }
    int groups_per_cta() const { return G() <= 32 ? 4 * (32 / G()) : 1; }
};

struct KInfo {
    CUfunction fn = nullptr;
    int regs = 0, local_bytes = 0, blocks_per_sm = 0;
    size_t smem = 0;
    double compile_ms = 0;
    bool from_cache = false;
};

// FNV-1a 64
uint64_t fnv(const void *p, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    return h;
}

std::string lib_dir()
{
    Dl_info info;
    if (dladdr((void *)&lib_dir, &info) && info.dli_fname) {
        std::string s = info.dli_fname;
        auto k = s.rfind('/');
        if (k != std::string::npos) return s.substr(0, k);
    }
    return ".";
}

std::string cache_dir()
{
    const char *e = getenv("JK_KERNEL_CACHE");
    std::string d = e && *e ? std::string(e) : lib_dir() + "/kcache";
    mkdir(d.c_str(), 0755);
    return d;
}

std::vector<std::string> nvrtc_options(const KSpec &s)
{
    // No --use_fast_math for the FP32 tier: the pair data already hold every
    // exponential, and the router's arithmetic stays exactly rounded.
    (void)s;
    return {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo"};
}

uint64_t spec_key(const KSpec &s)
{
    int major = 0, minor = 0;
    nvrtcVersion(&major, &minor);
    uint64_t h = fnv(jk_kernel_source, sizeof(jk_kernel_source));
    std::string n = s.name();
    h = fnv(n.data(), n.size(), h);
    for (auto &o : nvrtc_options(s)) h = fnv(o.data(), o.size(), h);
    h = fnv(&major, sizeof major, h);
    h = fnv(&minor, sizeof minor, h);
    return h;
}

// Compile one instantiation to a cubin; returns the lowered (mangled) name.
int nvrtc_compile(const KSpec &s, std::vector<char> &cubin, std::string &lowered, std::string &log)
{
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, jk_kernel_source, "jk_kernels.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        log = "nvrtcCreateProgram failed";
        return JK_ERR_COMPILE;
    }
    std::string name = s.name();
    nvrtcAddNameExpression(prog, name.c_str());
    auto opts = nvrtc_options(s);
    std::vector<const char *> copts;
    for (auto &o : opts) copts.push_back(o.c_str());
    nvrtcResult r = nvrtcCompileProgram(prog, (int)copts.size(), copts.data());
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    log.assign(ls, '\0');
    if (ls) nvrtcGetProgramLog(prog, &log[0]);
    if (r != NVRTC_SUCCESS) {
        nvrtcDestroyProgram(&prog);
        return JK_ERR_COMPILE;
    }
    const char *ln = nullptr;
    nvrtcGetLoweredName(prog, name.c_str(), &ln);
    lowered = ln ? ln : "";
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin.resize(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    return JK_OK;
}

struct KernelCache {
    std::mutex mu;
    std::map<std::pair<int, uint64_t>, KInfo> loaded;  // (device, key)
    std::vector<CUmodule> modules;
};
KernelCache &kcache()
{
    static KernelCache *c = new KernelCache();
    return *c;
}

bool read_cache_file(const std::string &path, std::string &lowered, std::vector<char> &cubin)
{
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    std::getline(f, lowered);
    std::vector<char> buf((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
    if (lowered.empty() || buf.empty()) return false;
    cubin.swap(buf);
    return true;
}

void write_cache_file(const std::string &path, const std::string &lowered, const std::vector<char> &cubin)
{
    std::string tmp = path + ".tmp" + std::to_string(getpid()) + "_" +
                      std::to_string(std::hash<std::thread::id>()(std::this_thread::get_id()));
    {
        std::ofstream f(tmp, std::ios::binary);
        if (!f) return;
        f << lowered << "\n";
        f.write(cubin.data(), (std::streamsize)cubin.size());
    }
    rename(tmp.c_str(), path.c_str());
}

// Make every spec available on the current device: memory, then disk, then
// NVRTC (in parallel threads). Fills out[i].
// Compile the specs that are not yet in the on-disk cache (no device needed).
int compile_to_disk(const std::vector<KSpec> &specs, double *ms_total)
{
    std::string dir = cache_dir();
    std::vector<int> todo;
    std::map<uint64_t, int> seen;
    for (size_t i = 0; i < specs.size(); ++i) {
        uint64_t k = spec_key(specs[i]);
        if (seen.count(k)) continue;
        seen[k] = 1;
        char fn[64];
        snprintf(fn, sizeof fn, "/%016llx.bin", (unsigned long long)k);
        struct stat st;
        if (stat((dir + fn).c_str(), &st) != 0) todo.push_back((int)i);
    }
    std::vector<int> rc(todo.size(), JK_OK);
    std::vector<std::string> logs(todo.size());
    std::atomic<int> next(0);
    auto t0 = std::chrono::steady_clock::now();
    auto worker = [&]() {
        for (;;) {
            int k = next.fetch_add(1);
            if (k >= (int)todo.size()) break;
            const KSpec &s = specs[todo[k]];
            std::vector<char> bin;
            std::string low;
            rc[k] = nvrtc_compile(s, bin, low, logs[k]);
            if (rc[k] == JK_OK) {
                char fn[64];
                snprintf(fn, sizeof fn, "/%016llx.bin", (unsigned long long)spec_key(s));
                write_cache_file(dir + fn, low, bin);
            }
        }
    };
    int nth = (int)std::min<size_t>(todo.size(), std::max(1u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(worker);
    for (auto &t : th) t.join();
    if (ms_total) *ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (size_t k = 0; k < todo.size(); ++k)
        if (rc[k] != JK_OK)
            return fail(JK_ERR_COMPILE, "NVRTC failed for %s:\n%.3000s", specs[todo[k]].name().c_str(), logs[k].c_str());
    return JK_OK;
}

int ensure_kernels(const std::vector<KSpec> &specs, std::vector<KInfo> &out)
{
    Driver &d = drv();
    if (!d.ok) return fail(JK_ERR_CUDA, "CUDA driver entry points unavailable");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    KernelCache &kc = kcache();
    out.assign(specs.size(), KInfo());
    // dynamic shared memory of a CTA: 227 KB on sm_103a, less a margin for
    // the kernels' static shared variables
    for (auto &sp : specs)
        if (sp.smem_bytes() > 220 * 1024)
            return fail(JK_ERR_UNSUPPORTED, "%s needs %zu bytes of shared memory per CTA (at most %d)",
                        sp.name().c_str(), sp.smem_bytes(), 220 * 1024);
    std::vector<int> todo;
    std::vector<uint64_t> keys(specs.size());
    {
        std::lock_guard<std::mutex> g(kc.mu);
        for (size_t i = 0; i < specs.size(); ++i) {
            keys[i] = spec_key(specs[i]);
            auto it = kc.loaded.find({dev, keys[i]});
            if (it != kc.loaded.end()) out[i] = it->second;
            else todo.push_back((int)i);
        }
    }
    if (todo.empty()) return JK_OK;
    // de-duplicate
    std::vector<int> uniq;
    {
        std::map<uint64_t, int> seen;
        for (int i : todo)
            if (!seen.count(keys[i])) { seen[keys[i]] = i; uniq.push_back(i); }
    }
    std::string dir = cache_dir();
    std::vector<std::vector<char>> bins(uniq.size());
    std::vector<std::string> lowered(uniq.size()), logs(uniq.size());
    std::vector<int> rc(uniq.size(), JK_OK);
    std::vector<double> ms(uniq.size(), 0.0);
    std::vector<char> cached(uniq.size(), 0);
    std::atomic<int> next(0);
    auto worker = [&]() {
        for (;;) {
            int k = next.fetch_add(1);
            if (k >= (int)uniq.size()) break;
            const KSpec &s = specs[uniq[k]];
            char fn[64];
            snprintf(fn, sizeof fn, "/%016llx.bin", (unsigned long long)keys[uniq[k]]);
            std::string path = dir + fn;
            if (read_cache_file(path, lowered[k], bins[k])) { cached[k] = 1; continue; }
            auto t0 = std::chrono::steady_clock::now();
            rc[k] = nvrtc_compile(s, bins[k], lowered[k], logs[k]);
            ms[k] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (rc[k] == JK_OK) write_cache_file(path, lowered[k], bins[k]);
        }
    };
    int nth = (int)std::min<size_t>(uniq.size(), std::max(1u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(worker);
    for (auto &t : th) t.join();
    for (size_t k = 0; k < uniq.size(); ++k)
        if (rc[k] != JK_OK)
            return fail(JK_ERR_COMPILE, "NVRTC failed for %s:\n%.1500s", specs[uniq[k]].name().c_str(), logs[k].c_str());
    std::lock_guard<std::mutex> g(kc.mu);
    for (size_t k = 0; k < uniq.size(); ++k) {
        const KSpec &s = specs[uniq[k]];
        CUmodule mod;
        CUresult r = d.moduleLoadData(&mod, bins[k].data());
        if (r != CUDA_SUCCESS) return fail(JK_ERR_CUDA, "cuModuleLoadData(%s) failed: %d", s.name().c_str(), (int)r);
        kc.modules.push_back(mod);
        KInfo ki;
        r = d.moduleGetFunction(&ki.fn, mod, lowered[k].c_str());
        if (r != CUDA_SUCCESS) return fail(JK_ERR_CUDA, "cuModuleGetFunction(%s) failed: %d", s.name().c_str(), (int)r);
        ki.smem = s.smem_bytes();
        // dynamic plus static shared memory above 48 KB needs the opt-in
        // (the routed kernels add 1-4 KB of static router scratch)
        if (ki.smem > 0) {
            r = d.funcSetAttribute(ki.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)ki.smem);
            if (r != CUDA_SUCCESS)
                return fail(JK_ERR_UNSUPPORTED, "%s: %zu bytes of dynamic shared memory refused (%d)", s.name().c_str(),
                            ki.smem, (int)r);
        }
        d.funcGetAttribute(&ki.regs, CU_FUNC_ATTRIBUTE_NUM_REGS, ki.fn);
        d.funcGetAttribute(&ki.local_bytes, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, ki.fn);
        d.occupancy(&ki.blocks_per_sm, ki.fn, s.block(), ki.smem);
        ki.compile_ms = ms[k];
        ki.from_cache = cached[k];
        kc.loaded[{dev, keys[uniq[k]]}] = ki;
    }
    for (size_t i = 0; i < specs.size(); ++i) out[i] = kc.loaded[{dev, keys[i]}];
    return JK_OK;
}

// ------------------------------------------------ real solid harmonics
// Cartesian expansion of the unit-norm real solid harmonics S_lm, m = -l..l
// (Helgaker, Jorgensen and Olsen, "Molecular Electronic-Structure Theory",
// Eqs. 6.4.47-6.4.50; Schlegel and Frisch 1995). Row = Cartesian component
// (x descending, then y), column = m + l. p shells keep (x, y, z). With the
// normalisation N_lm each S_lm has the norm of z^l, i.e. of the (l,0,0)
// component, so unit-norm inputs give unit-norm spherical functions.
std::vector<double> solid_harmonics(int l)
{
    const int nc = ncart(l), ns = 2 * l + 1;
    std::vector<double> C((size_t)nc * ns, 0.0);
    if (l == 0) { C[0] = 1.0; return C; }
    if (l == 1) { for (int i = 0; i < 3; ++i) C[i * 3 + i] = 1.0; return C; }
    auto fact = [](int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; };
    auto binom = [&](int n, int k) { return (k < 0 || k > n) ? 0.0 : fact(n) / (fact(k) * fact(n - k)); };
    auto comp = [&](int lx, int ly) {
        int idx = 0;
        for (int x = l; x >= 0; --x)
            for (int y = l - x; y >= 0; --y, ++idx)
                if (x == lx && y == ly) return idx;
        return -1;
    };
    for (int m = -l; m <= l; ++m) {
        const int am = m < 0 ? -m : m;
        const double N = std::sqrt(2.0 * fact(l + am) * fact(l - am) / (m == 0 ? 2.0 : 1.0)) / (std::ldexp(1.0, am) * fact(l));
        const int vm2 = m < 0 ? 1 : 0;
        for (int t = 0; t <= (l - am) / 2; ++t)
            for (int u = 0; u <= t; ++u)
                for (int k = vm2; k <= am; k += 2) {
                    const int sgn = ((t + (k - vm2) / 2) & 1) ? -1 : 1;
                    const double c = sgn * std::ldexp(1.0, -2 * t) * binom(l, t) * binom(l - t, am + t) * binom(t, u) * binom(am, k);
                    const int lx = 2 * t + am - 2 * u - k, ly = 2 * u + k;
                    C[(size_t)comp(lx, ly) * ns + (m + l)] += N * c;
                }
    }
    return C;
}

// -------------------------------------------------------- fragment choice
// Threads per quartet: G = ga*gb*gc*gd with each g dividing the Cartesian
// size of its shell. G == 1 keeps the 2D tables in registers and is taken
// when elements plus tables stay small; otherwise the smallest G whose
// per-thread fragment fits the register budget within one CTA (G <= 32: a
// warp holds 32 / G groups; up to 256, or 1024 for the Schwarz kernels: one
// group per CTA), else the smallest G that fits when the group is split
// over gx CTAs of at most 256 threads. The autotuner (the 1qnt grid search
// of Sec. 3.2, run on the caller's data) refines the choice per device
// through the tuning table.
void choose_fragments(KSpec &s, bool symmetric)
{
    const int nf[4] = {ncart(s.la), ncart(s.lb), ncart(s.lc), ncart(s.ld)};
    const int ne = nf[0] * nf[1] * nf[2] * nf[3];
    const int ni = s.ni();
    const int reg_cap = 48;                   // per-thread fragment budget (reals)
    const int gmax = symmetric ? 1024 : 256;  // threads per quartet in one CTA
    const int gsplit = 256;                   // threads per CTA of a group split over CTAs
    const int g1_cap = s.fp32 ? 128 : 64;     // register-mode budget: fragment + 3 tables
    s.gx = 1;
    if (ne + 3 * ni <= g1_cap) { s.ga = s.gb = s.gc = s.gd = 1; return; }
    // CTAs for a group of g threads: 1 if it fits one CTA, else the fewest
    // x (<= 16) dividing g with g / x <= gsplit, 0 if there is none
    auto split = [&](int g) {
        if (g <= gmax) return 1;
        for (int x = 2; x <= 16; ++x)
            if (g % x == 0 && g / x <= gsplit) return x;
        return 0;
    };
    int best[5] = {1, 1, 1, 1, 1};
    long best_score = -1;
    auto divisors = [](int n) { std::vector<int> v; for (int i = 1; i <= n; ++i) if (n % i == 0) v.push_back(i); return v; };
    for (int a : divisors(nf[0]))
        for (int b : divisors(nf[1]))
            for (int c : divisors(nf[2]))
                for (int d : divisors(nf[3])) {
                    if (symmetric && (a != c || b != d)) continue;
                    const int g = a * b * c * d;
                    if (g < 2) continue;
                    const int x = split(g);
                    if (x == 0) continue;
                    const int ept = ne / g;
                    const int gc = g / x;   // threads per CTA
                    // prefer: fits the budget in one CTA (fewest threads), then
                    // fits over several CTAs (fewest threads), then the
                    // smallest fragment in one CTA; fewest idle lanes last
                    const long idle = gc <= 32 ? 32 % gc : (32 - gc % 32) % 32;
                    long score;
                    if (ept <= reg_cap && x == 1) score = 300000000L + (4096L - g) * 1000L;
                    else if (ept <= reg_cap) score = 200000000L + (65536L - g) * 1000L / 16;
                    else if (x == 1) score = 100000000L - (long)ept * 10L;
                    else continue;
                    score -= idle;
                    if (score > best_score) {
                        best_score = score;
                        best[0] = a; best[1] = b; best[2] = c; best[3] = d; best[4] = x;
                    }
                }
    s.ga = best[0]; s.gb = best[1]; s.gc = best[2]; s.gd = best[3]; s.gx = best[4];
}

// Candidate fragmentations for the autotuner: the current shape first, then
// G = 1 (register mode) where the class is within twice the register-mode
// budget, then one shape per group size G (2 <= G <= 256, at most 64
// elements per thread, the fewest idle lanes), nearest to the current G
// (in log2 G) first. Shapes whose shared memory exceeds 200 KB are skipped.
std::vector<KSpec> fragment_candidates(const KSpec &s0, int maxc)
{
    std::vector<KSpec> out{s0};
    const int nf[4] = {ncart(s0.la), ncart(s0.lb), ncart(s0.lc), ncart(s0.ld)};
    const int ne = nf[0] * nf[1] * nf[2] * nf[3];
    const int g1_cap = s0.fp32 ? 128 : 64;
    auto push = [&](int a, int b, int c, int d) {
        if ((int)out.size() >= maxc) return;
        for (auto &x : out)
            if (x.ga == a && x.gb == b && x.gc == c && x.gd == d) return;
        KSpec s = s0;
        s.ga = a; s.gb = b; s.gc = c; s.gd = d; s.gx = 1;
        if (s.smem_bytes() > 200 * 1024) return;
        out.push_back(s);
    };
    if (ne + 3 * s0.ni() <= 2 * g1_cap) push(1, 1, 1, 1);
    std::map<int, std::array<int, 5>> byg;   // G -> {idle lanes, ga, gb, gc, gd}
    for (int a = 1; a <= nf[0]; ++a) {
        if (nf[0] % a) continue;
        for (int b = 1; b <= nf[1]; ++b) {
            if (nf[1] % b) continue;
            for (int c = 1; c <= nf[2]; ++c) {
                if (nf[2] % c) continue;
                for (int d = 1; d <= nf[3]; ++d) {
                    if (nf[3] % d) continue;
                    const int g = a * b * c * d;
                    if (g < 2 || g > 256 || ne / g > 64) continue;
                    const int idle = g <= 32 ? 32 % g : (32 - g % 32) % 32;
                    auto it = byg.find(g);
                    if (it == byg.end() || idle < it->second[0]) byg[g] = {idle, a, b, c, d};
                }
            }
        }
    }
    std::vector<std::pair<double, int>> ord;
    const double lg0 = std::log2((double)s0.G());
    for (auto &kv : byg) ord.push_back({std::fabs(std::log2((double)kv.first) - lg0), kv.first});
    std::sort(ord.begin(), ord.end());
    for (auto &o : ord) {
        const auto &v = byg[o.second];
        push(v[1], v[2], v[3], v[4]);
    }
    return out;
}

// Tuning table: the fragment shape the autotuner chose per class
// (angular momenta, primitive counts, tier) and device model, kept in memory
// and in a text file in the kernel cache directory ("key ga gb gc gd" lines).
struct TuneTable {
    std::mutex mu;
    std::map<std::string, std::map<std::string, std::array<int, 4>>> by_dev;   // by file path
    std::set<std::string> loaded;
};
TuneTable &ttable()
{
    static TuneTable t;
    return t;
}

std::string tune_key(const KSpec &s)
{
    char b[64];
    snprintf(b, sizeof b, "%d%d%d%d/%d_%d_%d_%d/%d", s.la, s.lb, s.lc, s.ld, s.na, s.nb, s.nc, s.nd, s.fp32);
    return b;
}

std::string tune_device(int dev)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    std::string n;
    for (const char *c = p.name; *c; ++c) n += (isalnum((unsigned char)*c) ? *c : '_');
    return n + "_sm" + std::to_string(p.major) + std::to_string(p.minor) + "_" + std::to_string(p.multiProcessorCount);
}

// JK_TUNING_DIR overrides the directory (default: the kernel cache)
std::string tune_path(const std::string &devname)
{
    const char *e = getenv("JK_TUNING_DIR");
    std::string d = e && *e ? std::string(e) : cache_dir();
    if (e && *e) mkdir(d.c_str(), 0755);
    return d + "/tune_" + devname + ".txt";
}

// caller holds the table's lock
void tune_load_locked(TuneTable &t, const std::string &path)
{
    if (t.loaded.count(path)) return;
    t.loaded.insert(path);
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return;
    char key[64];
    int a, b, c, d;
    while (fscanf(f, "%63s %d %d %d %d", key, &a, &b, &c, &d) == 5) t.by_dev[path][key] = {a, b, c, d};
    fclose(f);
}

// Apply a stored shape to s if there is one and it is valid for the class.
void tune_lookup(int dev, KSpec &s)
{
    const std::string path = tune_path(tune_device(dev));
    TuneTable &t = ttable();
    std::lock_guard<std::mutex> g(t.mu);
    tune_load_locked(t, path);
    auto di = t.by_dev.find(path);
    if (di == t.by_dev.end()) return;
    auto it = di->second.find(tune_key(s));
    if (it == di->second.end()) return;
    const auto &v = it->second;
    const int nf[4] = {ncart(s.la), ncart(s.lb), ncart(s.lc), ncart(s.ld)};
    for (int i = 0; i < 4; ++i)
        if (v[i] < 1 || nf[i] % v[i]) return;
    KSpec x = s;
    x.ga = v[0]; x.gb = v[1]; x.gc = v[2]; x.gd = v[3]; x.gx = 1;
    if (x.G() > 256 || x.smem_bytes() > 200 * 1024) return;
    s = x;
}

void tune_store(int dev, const std::vector<KSpec> &chosen)
{
    const std::string path = tune_path(tune_device(dev));
    TuneTable &t = ttable();
    std::lock_guard<std::mutex> g(t.mu);
    tune_load_locked(t, path);
    auto &m = t.by_dev[path];
    for (auto &s : chosen) m[tune_key(s)] = {s.ga, s.gb, s.gc, s.gd};
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (auto &kv : m) fprintf(f, "%s %d %d %d %d\n", kv.first.c_str(), kv.second[0], kv.second[1], kv.second[2], kv.second[3]);
    fclose(f);
    rename(tmp.c_str(), path.c_str());
}

// Modelled FLOPs of one contracted quartet of a class (FMA = 2).
double class_flops(const KSpec &s, int ndm)
{
    const double nr = s.nr();
    const double ne = (double)ncart(s.la) * ncart(s.lb) * ncart(s.lc) * ncart(s.ld);
    const double na = s.la + s.lb, nc = s.lc + s.ld;
    const double vrr = 3.0 * 3.0 * (na + 1) * (nc + 1);
    const double hrr = 3.0 * 2.0 * ((s.lb ? (na + 1) * s.lb : 0) * (nc + 1) + (s.ld ? (nc + 1) * s.ld : 0) * (s.la + 1) * (s.lb + 1));
    const double roots = 2.0 * nr * 2.0 * 10.0;
    const double setup = 30.0;
    const double prim = setup + roots + nr * (vrr + hrr) + nr * 3.0 * ne;
    const double P = (double)s.na * s.nb * s.nc * s.nd;
    return P * prim + ndm * 2.0 * 6.0 * ne;
}

// Modelled FLOPs of nq contracted quartets of which np primitive quartets
// were evaluated (the rest skipped by the primitive Schwarz screen).
double flops_of(const KSpec &s, int ndm, unsigned long long nq, unsigned long long np)
{
    KSpec one = s;
    one.na = one.nb = one.nc = one.nd = 1;
    const double contract = ndm * 2.0 * 6.0 * ncart(s.la) * ncart(s.lb) * ncart(s.lc) * ncart(s.ld);
    const double prim = class_flops(one, 0);
    return (double)np * prim + (double)nq * contract;
}

// ------------------------------------------------------------ plan data
struct PairClass {
    int la, lb, na, nb;
    int off = 0, n = 0;              // range in the pair array
    std::vector<int> beg, end;       // per molecule, absolute indices into the pair array
    int *d_beg = nullptr, *d_end = nullptr;
};

struct Launch {
    int c1, c2;        // pair classes (bra, ket)
    KSpec spec[2];     // [0] FP64, [1] FP32
    double cost;       // scheduling estimate
    // nbra + 1 work-item offsets (chunks of kets per bra): [0] with the
    // handle's chunk, [1] with the chunk of the FP64 tier of two-tier builds
    long long *d_prefix[2] = {nullptr, nullptr};
    long long nitems[2] = {0, 0};
    double cand = 0;   // candidate kets summed over the bras (Q_ab Q_cd > JK_ITEM_EPS)
};

// Kets per work item. A bra pair's candidate kets (those whose Schwarz
// product can exceed JK_ITEM_EPS with Dmax = 1) are split into chunks of this
// size; the last chunk always runs to the molecule's last ket.
#define JK_CHUNK 64
// The FP64 tier of a mixed build keeps ~7 % of the candidates; with 512 per
// item the batched mixed build ran 5 % faster than with 64 (and than 2,048).
#define JK_CHUNK_HI 512
#define JK_ITEM_EPS 1e-15

}  // namespace

#define JK_MAX_BRANCHES 7

struct jk_handle {
    int device = 0;
    int nmol = 0;
    int nshell = 0;
    std::vector<jk_shell> shells;
    std::vector<int> mol_sh0;              // nmol + 1
    std::vector<int> nao_cart, nao_user;   // per molecule
    std::vector<int> sh_ao_cart;           // molecule-local Cartesian AO offset per shell
    bool spherical = false;
    // device
    int *d_sh_mol = nullptr, *d_mol_sh0 = nullptr, *d_sh_ao = nullptr, *d_sh_nc = nullptr;
    JkPair *d_pairs = nullptr;
    JkPrimPair64 *d_pp64 = nullptr;
    JkPrimPair32 *d_pp32 = nullptr;
    JkMol *d_mols = nullptr;
    double *d_dmax = nullptr;
    float *d_dmax32 = nullptr;
    unsigned long long *d_dmax_mol = nullptr;
    double *d_rys64 = nullptr;
    float *d_rys32 = nullptr;
    unsigned long long *d_work = nullptr;  // one counter per launch
    unsigned long long *d_stats = nullptr; // three per launch and tier
    int *d_err = nullptr;
    int *h_err = nullptr;                  // pinned copy of d_err taken after each build without stats
    cudaEvent_t err_ev = nullptr;          // recorded after that copy
    bool err_pending = false;              // a copy is in flight and not yet looked at
    long long *d_tile_off = nullptr;
    long long ntiles = 0;
    long long dmax_total = 0;
    JkMol *h_mols = nullptr;               // pinned staging
    cudaEvent_t mol_copied = nullptr, ev0 = nullptr, ev1 = nullptr;
    std::vector<PairClass> classes;
    std::vector<Launch> launches;
    std::vector<JkPair> h_pairs;
    int num_sms = 0;
    // options
    // tau32: a 16-molecule sweep of the batched workload gave max |dJ| 3e-12,
    // 3e-10, 3e-9 at 1e-7, 1e-5, 1e-4 (about linear): 1e-4 keeps a 3x margin
    // to the 1e-8 target
    double tau32 = 1e-4, router_band = 100.0, pair_cutoff = 1e-18;
    int use_graph = 0, use_dmax = 1, profile = 0;
    int part_index = 0, part_count = 1;    // partitioned builds (multi-GPU split of one batch)
    double prim_eps = 1e-16;               // primitive threshold (never above the cutoff)
    double omega = 0.0;                    // range separation: 0 1/r, > 0 erf, < 0 erfc
    double init_ms = 0, compile_ms = 0;
    std::vector<cudaEvent_t> prof_ev;      // two per launch slot
    std::vector<jk_launch_prof> prof;
    std::vector<int> prof_slot;            // launch * 3 + tier of each prof record
    // spherical molecules: Cartesian scratch copies of D, J, K
    std::vector<char> mol_sph;             // per molecule
    std::vector<int> sh_ao_user;           // molecule-local AO offset in the caller's basis
    int *d_sh_l = nullptr, *d_sh_sph = nullptr, *d_sh_aou = nullptr, *d_c2s_off = nullptr;
    double *d_c2s = nullptr;
    double *d_cart = nullptr;              // scratch: per spherical molecule 3 x ndm x nao_c^2
    size_t cart_ndm = 0;
    std::vector<size_t> cart_off;          // per molecule offset into d_cart
    JkSphMol *d_sph = nullptr, *h_sph = nullptr;  // [0, nmol): to Cartesian, [nmol, 2 nmol): back
    size_t cart_gen = 0;                   // bumps when the scratch moves (invalidates graphs)
    float *d_d32 = nullptr;                // FP32 copies of D for the FP32 tier: ndm x nao_c^2 per molecule
    size_t d32_ndm = 0;
    std::vector<size_t> d32_off;
    // learned router
    JkPairFeat *d_pfeat = nullptr;         // aligned with d_pairs
    JkRouterDev *d_router = nullptr;
    bool has_router = false;
    unsigned long long *d_logn = nullptr;
    JkRouted *d_rlist = nullptr;           // routed builds: released quartets, per launch segments
    unsigned long long *d_rcount = nullptr;
    std::vector<long long> rl_off, rl_cap;
    std::vector<long long> rl_need;        // entries each list needed in the last build with stats
    double route_cap = 16777216.0;         // list entries over all launches
    int asym64 = 0;                        // FP32 tier: large-T roots and weights in FP64
    int chunk = 64;                        // kets per work item
    // FP32 tier: float-to-double by integer operations (1) or by the
    // conversion instruction (0, measured 11 % faster on the FP32 tier of
    // the batched workload: the integer sequence costs more issue slots than
    // the FP64-pipe instruction it replaces)
    int widen_int = 0;
    int chunk_hi = 64;                     // ... for the FP64 tier of mixed and routed builds
    // bounds compared in FP64 (0: in FP32 when the cutoff is >= 1e-30); FP64
    // costs about 2 % of a mixed build of the batched workload
    int screen64 = 1;
    // graphs and branch streams
    int branches = 1;
    cudaStream_t cap = nullptr;
    cudaStream_t side[JK_MAX_BRANCHES] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[JK_MAX_BRANCHES] = {};
    std::map<std::string, std::pair<cudaGraphExec_t, int>> graphs;
};

namespace {

void free_handle(jk_handle *h)
{
    if (!h) return;
    for (auto &c : h->classes) { cudaFree(c.d_beg); cudaFree(c.d_end); }
    for (auto &L : h->launches) { cudaFree(L.d_prefix[0]); cudaFree(L.d_prefix[1]); }
    cudaFree(h->d_sh_mol); cudaFree(h->d_mol_sh0); cudaFree(h->d_sh_ao); cudaFree(h->d_sh_nc);
    cudaFree(h->d_pairs); cudaFree(h->d_pp64); cudaFree(h->d_pp32); cudaFree(h->d_mols);
    cudaFree(h->d_dmax); cudaFree(h->d_dmax32); cudaFree(h->d_dmax_mol); cudaFree(h->d_rys64); cudaFree(h->d_rys32);
    cudaFree(h->d_work); cudaFree(h->d_stats); cudaFree(h->d_err); cudaFree(h->d_tile_off);
    if (h->h_mols) cudaFreeHost(h->h_mols);
    if (h->h_err) cudaFreeHost(h->h_err);
    if (h->err_ev) cudaEventDestroy(h->err_ev);
    if (h->mol_copied) cudaEventDestroy(h->mol_copied);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (auto e : h->prof_ev) cudaEventDestroy(e);
    cudaFree(h->d_sh_l); cudaFree(h->d_sh_sph); cudaFree(h->d_sh_aou); cudaFree(h->d_c2s_off);
    cudaFree(h->d_c2s); cudaFree(h->d_cart); cudaFree(h->d_sph); cudaFree(h->d_d32);
    cudaFree(h->d_pfeat); cudaFree(h->d_router); cudaFree(h->d_logn);
    cudaFree(h->d_rlist); cudaFree(h->d_rcount);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second.first);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (int b = 0; b < JK_MAX_BRANCHES; ++b) {
        if (h->side[b]) cudaStreamDestroy(h->side[b]);
        if (h->ev_join[b]) cudaEventDestroy(h->ev_join[b]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->h_sph) cudaFreeHost(h->h_sph);
    delete h;
}

template <typename T>
int upload(T **dst, const std::vector<T> &src)
{
    if (src.empty()) { *dst = nullptr; return JK_OK; }
    CK(cudaMalloc((void **)dst, sizeof(T) * src.size()));
    CK(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return JK_OK;
}

// shell type order: l first, then nprim
long type_key(const jk_shell &s) { return (long)s.l * 64 + s.nprim; }

// Work items of every launch: per bra, ceil(candidates / chunk) (at least
// one), where the candidates are the kets (sorted by Q) with Q_ab Q_cd >
// JK_ITEM_EPS; the last chunk of a bra runs to the molecule's last ket. Two
// partitions: `chunk` for every tier but one, `chunk_hi` for the FP64 tier
// of mixed and routed builds, which keeps only the few candidates above
// tau32, so that its items still fill whole rounds of a warp. Also the
// launch's cost estimate (candidates x modelled FLOPs per quartet).
int plan_items(jk_handle *h, int chunk, int chunk_hi)
{
    for (auto &L : h->launches) {
        const PairClass &A = h->classes[L.c1], &B = h->classes[L.c2];
        std::vector<long long> pre(A.n + 1, 0), pre2(A.n + 1, 0);
        double work = 0;
        for (int m = 0; m < h->nmol; ++m) {
            const int b0 = A.beg[m], b1 = A.end[m];
            const int k0 = B.beg[m], k1 = B.end[m];
            for (int bi = b0; bi < b1; ++bi) {
                const double qa = h->h_pairs[A.off + bi].Q;
                const int kfirst = (L.c1 == L.c2) ? bi : k0;
                // kets with qa * Q_cd > eps form a prefix of [k0, k1)
                int lo = k0, hi = k1;
                while (lo < hi) {
                    int mid = (lo + hi) / 2;
                    if (qa * h->h_pairs[B.off + mid].Q > JK_ITEM_EPS) lo = mid + 1; else hi = mid;
                }
                long long ncand = std::max(0, lo - kfirst);
                pre[bi + 1] = std::max(1LL, (ncand + chunk - 1) / chunk);
                pre2[bi + 1] = std::max(1LL, (ncand + chunk_hi - 1) / chunk_hi);
                work += (double)ncand;
            }
        }
        for (int bi = 0; bi < A.n; ++bi) { pre[bi + 1] += pre[bi]; pre2[bi + 1] += pre2[bi]; }
        L.nitems[0] = pre[A.n];
        L.nitems[1] = pre2[A.n];
        for (int t = 0; t < 2; ++t) { cudaFree(L.d_prefix[t]); L.d_prefix[t] = nullptr; }
        if (int rc = upload(&L.d_prefix[0], pre)) return rc;
        if (int rc = upload(&L.d_prefix[1], pre2)) return rc;
        L.cand = work;
        L.cost = work * class_flops(L.spec[0], 1);
    }
    h->chunk = chunk;
    h->chunk_hi = chunk_hi;
    return JK_OK;
}

int init_impl(int32_t nmol, const int32_t *mol_shell_off, const jk_shell *shells, int32_t nshell,
              const double *coords, int32_t natm, const double *exps, const double *coeffs,
              int32_t nprim_total, jk_handle **out)
{
    if (!out) return fail(JK_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nmol < 1 || !mol_shell_off || !shells || nshell < 1 || !coords || natm < 1 || !exps || !coeffs ||
        nprim_total < 1)
        return fail(JK_ERR_ARG, "empty or NULL basis arguments");
    if (mol_shell_off[0] != 0 || mol_shell_off[nmol] != nshell)
        return fail(JK_ERR_ARG, "mol_shell_off must start at 0 and end at nshell");
    for (int m = 0; m < nmol; ++m)
        if (mol_shell_off[m + 1] <= mol_shell_off[m]) return fail(JK_ERR_ARG, "molecule %d has no shells", m);
    for (int s = 0; s < nshell; ++s) {
        const jk_shell &x = shells[s];
        if (x.l < 0 || x.nprim < 1 || x.atom < 0 || x.atom >= natm || x.prim_off < 0 ||
            x.prim_off + x.nprim > nprim_total || x.ao_off < 0 || (x.spherical != 0 && x.spherical != 1))
            return fail(JK_ERR_ARG, "shell %d has fields out of range", s);
        if (x.l > JK_LMAX) return fail(JK_ERR_UNSUPPORTED, "shell %d: l=%d above JK_LMAX=%d", s, x.l, JK_LMAX);
        if (x.nprim > JK_NPRIM_MAX) return fail(JK_ERR_UNSUPPORTED, "shell %d: nprim=%d above %d", s, x.nprim, JK_NPRIM_MAX);
        for (int i = 0; i < x.nprim; ++i)
            if (!(exps[x.prim_off + i] > 0) || !std::isfinite(coeffs[x.prim_off + i]))
                return fail(JK_ERR_ARG, "shell %d: non-positive exponent or non-finite coefficient", s);
    }
    for (int i = 0; i < 3 * natm; ++i)
        if (!std::isfinite(coords[i])) return fail(JK_ERR_ARG, "non-finite coordinate");

    auto t_start = std::chrono::steady_clock::now();
    std::unique_ptr<jk_handle, void (*)(jk_handle *)> h(new jk_handle(), free_handle);
    CK(cudaGetDevice(&h->device));
    CK(cudaFree(0));
    CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    h->nmol = nmol;
    h->nshell = nshell;
    h->shells.assign(shells, shells + nshell);
    h->mol_sh0.assign(mol_shell_off, mol_shell_off + nmol + 1);
    h->sh_ao_cart.resize(nshell);
    std::vector<int> sh_mol(nshell), sh_nc(nshell);
    h->sh_ao_user.resize(nshell);
    for (int m = 0; m < nmol; ++m) {
        int o = 0, ou = 0;
        bool sph = false;
        for (int s = mol_shell_off[m]; s < mol_shell_off[m + 1]; ++s) {
            sh_mol[s] = m;
            h->sh_ao_cart[s] = o;
            sh_nc[s] = ncart(shells[s].l);
            o += ncart(shells[s].l);
            if (shells[s].ao_off != ou)
                return fail(JK_ERR_ARG, "shell %d: ao_off %d, expected %d (functions are laid out shell by shell)",
                            s, shells[s].ao_off, ou);
            h->sh_ao_user[s] = ou;
            ou += shells[s].spherical ? 2 * shells[s].l + 1 : ncart(shells[s].l);
            sph = sph || shells[s].spherical;
        }
        h->nao_cart.push_back(o);
        h->nao_user.push_back(ou);
        h->mol_sph.push_back(sph ? 1 : 0);
        h->spherical = h->spherical || sph;
    }

    // ---- shell types and pair classes
    std::vector<long> tkeys;
    for (int s = 0; s < nshell; ++s) tkeys.push_back(type_key(shells[s]));
    std::sort(tkeys.begin(), tkeys.end());
    tkeys.erase(std::unique(tkeys.begin(), tkeys.end()), tkeys.end());
    std::reverse(tkeys.begin(), tkeys.end());   // type 0 = largest (l, nprim)
    auto type_of = [&](int s) { return (int)(std::find(tkeys.begin(), tkeys.end(), type_key(shells[s])) - tkeys.begin()); };
    std::vector<int> sh_type(nshell);
    for (int s = 0; s < nshell; ++s) sh_type[s] = type_of(s);
    const int ntype = (int)tkeys.size();
    auto pclass = [&](int ta, int tb) { return ta * ntype + tb; };   // ta <= tb in type index (a is "larger")

    // ---- candidate pairs (host pre-screen: largest Gaussian product factor)
    struct Cand { int a, b, cls; };
    std::vector<Cand> cand;
    for (int m = 0; m < nmol; ++m) {
        for (int s1 = mol_shell_off[m]; s1 < mol_shell_off[m + 1]; ++s1)
            for (int s2 = mol_shell_off[m]; s2 <= s1; ++s2) {
                int a = s1, b = s2;
                if (sh_type[a] > sh_type[b] || (sh_type[a] == sh_type[b] && a < b)) std::swap(a, b);
                const double *A = coords + 3 * shells[a].atom, *B = coords + 3 * shells[b].atom;
                double r2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
                double mu_min = 1e300;
                for (int i = 0; i < shells[a].nprim; ++i)
                    for (int j = 0; j < shells[b].nprim; ++j) {
                        double al = exps[shells[a].prim_off + i], be = exps[shells[b].prim_off + j];
                        mu_min = std::min(mu_min, al * be / (al + be));
                    }
                if (mu_min * r2 > 92.0) continue;   // exp(-92) ~ 1e-40
                cand.push_back({a, b, pclass(sh_type[a], sh_type[b])});
            }
    }
    if (cand.empty()) return fail(JK_ERR_ARG, "no shell pairs");
    std::stable_sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.cls < y.cls; });
    const long long ncand = (long long)cand.size();
    if (ncand > 0x7fffffffLL) return fail(JK_ERR_UNSUPPORTED, "too many shell pairs");
    std::vector<int> ca(ncand), cb(ncand), cpp(ncand);
    long long npp = 0;
    for (long long i = 0; i < ncand; ++i) {
        ca[i] = cand[i].a;
        cb[i] = cand[i].b;
        cpp[i] = (int)npp;
        npp += (long long)shells[cand[i].a].nprim * shells[cand[i].b].nprim;
    }
    if (npp > 0x7fffffffLL) return fail(JK_ERR_UNSUPPORTED, "too many primitive pairs");

    // ---- device copies of the basis
    std::vector<int> sh_atom(nshell), sh_np(nshell), sh_prim(nshell);
    for (int s = 0; s < nshell; ++s) { sh_atom[s] = shells[s].atom; sh_np[s] = shells[s].nprim; sh_prim[s] = shells[s].prim_off; }
    int *d_ca = nullptr, *d_cb = nullptr, *d_cpp = nullptr, *d_atom = nullptr, *d_np = nullptr, *d_prim = nullptr;
    double *d_coords = nullptr, *d_exps = nullptr, *d_coeffs = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_ca); cudaFree(d_cb); cudaFree(d_cpp); cudaFree(d_atom); cudaFree(d_np); cudaFree(d_prim);
        cudaFree(d_coords); cudaFree(d_exps); cudaFree(d_coeffs);
    };
    struct Guard { std::function<void()> f; ~Guard() { f(); } } guard{cleanup};
    int rc;
    if ((rc = upload(&d_ca, ca)) || (rc = upload(&d_cb, cb)) || (rc = upload(&d_cpp, cpp)) ||
        (rc = upload(&d_atom, sh_atom)) || (rc = upload(&d_np, sh_np)) || (rc = upload(&d_prim, sh_prim)))
        return rc;
    if ((rc = upload(&d_coords, std::vector<double>(coords, coords + 3 * natm))) ||
        (rc = upload(&d_exps, std::vector<double>(exps, exps + nprim_total))) ||
        (rc = upload(&d_coeffs, std::vector<double>(coeffs, coeffs + nprim_total))))
        return rc;
    CK(cudaMalloc(&h->d_pp64, sizeof(JkPrimPair64) * npp));
    CK(cudaMalloc(&h->d_pp32, sizeof(JkPrimPair32) * npp));
    jk_pairdata_kernel<<<(unsigned)((ncand + 127) / 128), 128>>>((int)ncand, d_ca, d_cb, d_cpp, d_atom, d_np, d_prim,
                                                                  d_coords, d_exps, d_coeffs, h->d_pp64, h->d_pp32);
    CK(cudaGetLastError());

    // ---- Rys tables
    {
        std::vector<double> t64(rys_table64, rys_table64 + rys_table64_size);
        std::vector<float> t32(rys_table32_size);
        for (size_t i = 0; i < rys_table32_size; ++i) t32[i] = (float)rys_table32_src[i];
        if ((rc = upload(&h->d_rys64, t64)) || (rc = upload(&h->d_rys32, t32))) return rc;
    }

    // ---- JkPair records for the candidates (unsorted), Schwarz per class
    std::vector<JkPair> cp(ncand);
    for (long long i = 0; i < ncand; ++i) {
        JkPair &p = cp[i];
        const int a = ca[i], b = cb[i];
        p.a = a; p.b = b; p.mol = sh_mol[a]; p.pp_off = cpp[i];
        p.a_ao = h->sh_ao_cart[a]; p.b_ao = h->sh_ao_cart[b];
        p.a_loc = a - mol_shell_off[p.mol]; p.b_loc = b - mol_shell_off[p.mol];
        const double *A = coords + 3 * shells[a].atom, *B = coords + 3 * shells[b].atom;
        p.ABx = A[0] - B[0]; p.ABy = A[1] - B[1]; p.ABz = A[2] - B[2];
        p.ABxf = (float)p.ABx; p.AByf = (float)p.ABy; p.ABzf = (float)p.ABz;
        p.pad0 = 0; p.pad1 = 0.0;
        p.Q = 0; p.Qf = 0.f; p.padf = 0.f;
    }
    JkPair *d_cp = nullptr;
    double *d_q = nullptr;
    if ((rc = upload(&d_cp, cp))) return rc;
    struct G2 { JkPair *p; double *q; ~G2() { cudaFree(p); cudaFree(q); } } g2{d_cp, nullptr};
    CK(cudaMalloc(&d_q, sizeof(double) * ncand));
    CK(cudaMemset(d_q, 0, sizeof(double) * ncand));   // split groups combine by atomic max
    g2.q = d_q;
    {
        // one Schwarz launch per pair class
        std::vector<KSpec> specs;
        std::vector<std::pair<long long, long long>> ranges;
        long long i0 = 0;
        while (i0 < ncand) {
            long long i1 = i0;
            while (i1 < ncand && cand[i1].cls == cand[i0].cls) ++i1;
            const jk_shell &sa = shells[cand[i0].a], &sb = shells[cand[i0].b];
            KSpec s;
            s.kind = 1;
            s.la = s.lc = sa.l; s.lb = s.ld = sb.l; s.na = s.nc = sa.nprim; s.nb = s.nd = sb.nprim;
            choose_fragments(s, true);
            specs.push_back(s);
            ranges.push_back({i0, i1});
            i0 = i1;
        }
        std::vector<KInfo> ki;
        auto tc = std::chrono::steady_clock::now();
        if ((rc = ensure_kernels(specs, ki))) return rc;
        h->compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc).count();
        for (size_t k = 0; k < specs.size(); ++k) {
            JkSchwarzArgs a;
            a.pairs = d_cp + ranges[k].first;
            a.pp64 = h->d_pp64;
            a.rys64 = h->d_rys64;
            a.Qout = d_q + ranges[k].first;
            a.npair = (int)(ranges[k].second - ranges[k].first);
            const long long groups = specs[k].groups_per_cta();
            const long long units = (long long)a.npair * specs[k].gx;
            unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((units + groups - 1) / groups,
                                                                                (long long)h->num_sms * 8));
            void *params[] = {&a};
            CUresult r = drv().launchKernel(ki[k].fn, grid, 1, 1, specs[k].block(), 1, 1, (unsigned)ki[k].smem, 0,
                                            params, nullptr);
            if (r != CUDA_SUCCESS) return fail(JK_ERR_CUDA, "Schwarz launch failed: %d", (int)r);
        }
        CK(cudaDeviceSynchronize());
    }
    std::vector<double> q(ncand);
    CK(cudaMemcpy(q.data(), d_q, sizeof(double) * ncand, cudaMemcpyDeviceToHost));

    // ---- primitive-pair Schwarz factors: the Schwarz kernel of each pair
    // class on single-primitive pseudo pairs (same centres, pp_off pointing
    // at one primitive pair), then every shell pair's primitive pairs sorted
    // by them, largest first
    {
        std::vector<JkPair> pseudo((size_t)npp);
        std::vector<KSpec> specs;
        std::vector<std::pair<long long, long long>> ranges;
        long long i0 = 0;
        while (i0 < ncand) {
            long long i1 = i0;
            while (i1 < ncand && cand[i1].cls == cand[i0].cls) ++i1;
            for (long long i = i0; i < i1; ++i) {
                const int n = shells[ca[i]].nprim * shells[cb[i]].nprim;
                for (int k = 0; k < n; ++k) {
                    JkPair pr = cp[i];
                    pr.pp_off = cpp[i] + k;
                    pseudo[cpp[i] + k] = pr;
                }
            }
            const jk_shell &sa = shells[cand[i0].a], &sb = shells[cand[i0].b];
            KSpec sp;
            sp.kind = 1;
            sp.la = sp.lc = sa.l; sp.lb = sp.ld = sb.l; sp.na = sp.nb = sp.nc = sp.nd = 1;
            choose_fragments(sp, true);
            specs.push_back(sp);
            ranges.push_back({cpp[i0], i1 < ncand ? cpp[i1] : npp});
            i0 = i1;
        }
        JkPair *d_pseudo = nullptr;
        double *d_qp = nullptr;
        int *d_cnt = nullptr;
        JkPrimPair64 *n64 = nullptr;
        JkPrimPair32 *n32 = nullptr;
        auto cl2 = [&]() { cudaFree(d_pseudo); cudaFree(d_qp); cudaFree(d_cnt); cudaFree(n64); cudaFree(n32); };
        struct G3 { std::function<void()> f; ~G3() { f(); } } g3{cl2};
        if ((rc = upload(&d_pseudo, pseudo))) return rc;
        CK(cudaMalloc(&d_qp, sizeof(double) * npp));
        CK(cudaMemset(d_qp, 0, sizeof(double) * npp));
        std::vector<KInfo> ki;
        auto tc = std::chrono::steady_clock::now();
        if ((rc = ensure_kernels(specs, ki))) return rc;
        h->compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc).count();
        for (size_t k = 0; k < specs.size(); ++k) {
            JkSchwarzArgs a;
            a.pairs = d_pseudo + ranges[k].first;
            a.pp64 = h->d_pp64;
            a.rys64 = h->d_rys64;
            a.Qout = d_qp + ranges[k].first;
            a.npair = (int)(ranges[k].second - ranges[k].first);
            const long long groups = specs[k].groups_per_cta();
            const long long units = (long long)a.npair * specs[k].gx;
            unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((units + groups - 1) / groups,
                                                                                (long long)h->num_sms * 8));
            void *params[] = {&a};
            CUresult r = drv().launchKernel(ki[k].fn, grid, 1, 1, specs[k].block(), 1, 1, (unsigned)ki[k].smem, 0,
                                            params, nullptr);
            if (r != CUDA_SUCCESS) return fail(JK_ERR_CUDA, "primitive Schwarz launch failed: %d", (int)r);
        }
        std::vector<int> cnt(ncand);
        for (long long i = 0; i < ncand; ++i) cnt[i] = shells[ca[i]].nprim * shells[cb[i]].nprim;
        if ((rc = upload(&d_cnt, cnt))) return rc;
        CK(cudaMalloc(&n64, sizeof(JkPrimPair64) * npp));
        CK(cudaMalloc(&n32, sizeof(JkPrimPair32) * npp));
        jk_primsort_kernel<<<(unsigned)((ncand + 127) / 128), 128>>>((int)ncand, d_cpp, d_cnt, d_qp, h->d_pp64,
                                                                      h->d_pp32, n64, n32);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        std::swap(h->d_pp64, n64);
        std::swap(h->d_pp32, n32);
    }

    // ---- prune, group by (class, molecule), sort by Q descending
    std::vector<long long> order;
    for (long long i = 0; i < ncand; ++i)
        if (q[i] > h->pair_cutoff && std::isfinite(q[i])) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](long long x, long long y) {
        if (cand[x].cls != cand[y].cls) return cand[x].cls < cand[y].cls;
        if (cp[x].mol != cp[y].mol) return cp[x].mol < cp[y].mol;
        return q[x] > q[y];
    });
    h->h_pairs.resize(order.size());
    for (size_t k = 0; k < order.size(); ++k) {
        h->h_pairs[k] = cp[order[k]];
        h->h_pairs[k].Q = q[order[k]];
        h->h_pairs[k].Qf = (float)q[order[k]];
    }
    size_t k0 = 0;
    while (k0 < order.size()) {
        size_t k1 = k0;
        int cls = cand[order[k0]].cls;
        while (k1 < order.size() && cand[order[k1]].cls == cls) ++k1;
        PairClass pc;
        const jk_shell &sa = shells[h->h_pairs[k0].a], &sb = shells[h->h_pairs[k0].b];
        pc.la = sa.l; pc.lb = sb.l; pc.na = sa.nprim; pc.nb = sb.nprim;
        pc.off = (int)k0; pc.n = (int)(k1 - k0);
        // per molecule, indices relative to the class base (empty range if none)
        pc.beg.assign(nmol, 0);
        pc.end.assign(nmol, 0);
        for (size_t k = k0; k < k1;) {
            int m = h->h_pairs[k].mol;
            size_t e = k;
            while (e < k1 && h->h_pairs[e].mol == m) ++e;
            pc.beg[m] = (int)(k - k0); pc.end[m] = (int)(e - k0);
            k = e;
        }
        h->classes.push_back(pc);
        k0 = k1;
    }
    if ((rc = upload(&h->d_pairs, h->h_pairs))) return rc;
    {
        // router features per pair: exponent-sum range, |A-B|, log10 Q, centre
        // of the most diffuse primitive pair, l_a + l_b
        std::vector<JkPairFeat> pf(h->h_pairs.size());
        for (size_t k = 0; k < pf.size(); ++k) {
            const JkPair &pr = h->h_pairs[k];
            const jk_shell &sa = shells[pr.a], &sb = shells[pr.b];
            const double *A = coords + 3 * sa.atom, *B = coords + 3 * sb.atom;
            double pmin = 1e300, pmax = 0, pcx = 0, pcy = 0, pcz = 0;
            for (int i = 0; i < sa.nprim; ++i)
                for (int j = 0; j < sb.nprim; ++j) {
                    const double al = exps[sa.prim_off + i], be = exps[sb.prim_off + j], p = al + be;
                    pmax = std::max(pmax, p);
                    if (p < pmin) {
                        pmin = p;
                        pcx = (al * A[0] + be * B[0]) / p;
                        pcy = (al * A[1] + be * B[1]) / p;
                        pcz = (al * A[2] + be * B[2]) / p;
                    }
                }
            JkPairFeat &f = pf[k];
            f.lpmin = (float)std::log(pmin);
            f.lpmax = (float)std::log(pmax);
            f.rab = (float)std::sqrt(pr.ABx * pr.ABx + pr.ABy * pr.ABy + pr.ABz * pr.ABz);
            f.lq = (float)std::log10(pr.Q);
            f.pcx = (float)pcx; f.pcy = (float)pcy; f.pcz = (float)pcz;
            f.lsum = (float)(sa.l + sb.l);
        }
        if ((rc = upload(&h->d_pfeat, pf))) return rc;
        CK(cudaMalloc(&h->d_router, sizeof(JkRouterDev)));
        CK(cudaMalloc(&h->d_logn, sizeof(unsigned long long)));
    }
    for (auto &c : h->classes) {
        if ((rc = upload(&c.d_beg, c.beg)) || (rc = upload(&c.d_end, c.end))) return rc;
    }

    // ---- class-pair launches (bra class index <= ket class index in type order)
    const int nc = (int)h->classes.size();
    for (int i = 0; i < nc; ++i)
        for (int j = i; j < nc; ++j) {
            Launch L;
            L.c1 = i; L.c2 = j;
            const PairClass &A = h->classes[i], &B = h->classes[j];
            for (int t = 0; t < 2; ++t) {
                KSpec &s = L.spec[t];
                s.kind = 0;
                s.la = A.la; s.lb = A.lb; s.lc = B.la; s.ld = B.lb;
                s.na = A.na; s.nb = A.nb; s.nc = B.na; s.nd = B.nb;
                s.fp32 = t;
                choose_fragments(s, false);
                tune_lookup(h->device, s);
            }
            h->launches.push_back(L);
        }
    if ((rc = plan_items(h.get(), JK_CHUNK, JK_CHUNK_HI))) return rc;
    std::stable_sort(h->launches.begin(), h->launches.end(), [](const Launch &x, const Launch &y) { return x.cost > y.cost; });

    // ---- per-build scratch
    std::vector<int> mol_sh0(h->mol_sh0.begin(), h->mol_sh0.end());
    std::vector<int> sh_ao(h->sh_ao_cart.begin(), h->sh_ao_cart.end());
    if ((rc = upload(&h->d_sh_mol, sh_mol)) || (rc = upload(&h->d_mol_sh0, mol_sh0)) ||
        (rc = upload(&h->d_sh_ao, sh_ao)) || (rc = upload(&h->d_sh_nc, sh_nc)))
        return rc;
    long long dtot = 0;
    std::vector<long long> toff(nmol + 1, 0);
    for (int m = 0; m < nmol; ++m) {
        long long ns = mol_shell_off[m + 1] - mol_shell_off[m];
        dtot += ns * ns;
        long long nt = (h->nao_cart[m] + 31) / 32;
        toff[m + 1] = toff[m] + nt * (nt + 1) / 2;
    }
    h->dmax_total = dtot;
    h->ntiles = toff[nmol];
    if ((rc = upload(&h->d_tile_off, toff))) return rc;
    CK(cudaMalloc(&h->d_dmax, sizeof(double) * dtot));
    CK(cudaMalloc(&h->d_dmax32, sizeof(float) * dtot));
    CK(cudaMalloc(&h->d_dmax_mol, sizeof(unsigned long long) * nmol));
    CK(cudaMalloc(&h->d_mols, sizeof(JkMol) * nmol));
    const size_t nl = h->launches.size() * 3;   // FP64, FP32 and the routed list kernel
    CK(cudaMalloc(&h->d_work, sizeof(unsigned long long) * nl));
    CK(cudaMalloc(&h->d_stats, sizeof(unsigned long long) * 3 * nl));
    CK(cudaMalloc(&h->d_err, sizeof(int)));
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    if (h->spherical) {
        std::vector<int> sl(nshell), ss(nshell), off(JK_LMAX + 2, 0);
        for (int s2 = 0; s2 < nshell; ++s2) { sl[s2] = shells[s2].l; ss[s2] = shells[s2].spherical; }
        std::vector<double> c2s;
        for (int l = 0; l <= JK_LMAX; ++l) {
            off[l] = (int)c2s.size();
            auto C = solid_harmonics(l);
            c2s.insert(c2s.end(), C.begin(), C.end());
        }
        if ((rc = upload(&h->d_sh_l, sl)) || (rc = upload(&h->d_sh_sph, ss)) ||
            (rc = upload(&h->d_sh_aou, h->sh_ao_user)) || (rc = upload(&h->d_c2s_off, off)) ||
            (rc = upload(&h->d_c2s, c2s)))
            return rc;
        CK(cudaMalloc(&h->d_sph, sizeof(JkSphMol) * 2 * nmol));
        CK(cudaMallocHost(&h->h_sph, sizeof(JkSphMol) * 2 * nmol));
    }
    CK(cudaMallocHost(&h->h_mols, sizeof(JkMol) * nmol));
    CK(cudaMallocHost(&h->h_err, sizeof(int)));
    *h->h_err = 0;
    CK(cudaEventCreateWithFlags(&h->err_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->mol_copied, cudaEventDisableTiming));
    CK(cudaEventCreate(&h->ev0));
    CK(cudaEventCreate(&h->ev1));
    CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    for (int b = 0; b < JK_MAX_BRANCHES; ++b) {
        CK(cudaStreamCreateWithFlags(&h->side[b], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_join[b], cudaEventDisableTiming));
    }
    CK(cudaDeviceSynchronize());
    h->init_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    *out = h.release();
    return JK_OK;
}

struct LogSpec {
    float *x, *y;
    long long cap;
};

// The device error word (set by the kernels: a non-finite density element)
// as a status: clears the word and returns the matching error code.
int device_error(jk_handle *h, int err, const char *when)
{
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    *h->h_err = 0;
    if (err & JK_ERR_DEV_NAN) return fail(JK_ERR_NAN, "%s: the density holds NaN or infinite values", when);
    return fail(JK_ERR_CUDA, "%s: device error word %d", when, err);
}

// A build without stats leaves an asynchronous copy of the error word; look
// at it if it has landed (the next build, jk_check and jk_destroy do).
int poll_device_error(jk_handle *h, bool wait)
{
    if (!h->err_pending) return JK_OK;
    cudaError_t q = wait ? cudaEventSynchronize(h->err_ev) : cudaEventQuery(h->err_ev);
    if (q == cudaErrorNotReady) { cudaGetLastError(); return JK_OK; }
    CK(q);
    h->err_pending = false;
    if (*h->h_err) return device_error(h, *h->h_err, "an earlier build on this handle");
    return JK_OK;
}

int build_impl(jk_handle *h, const double *const *D, int32_t ndm, int with_j, int with_k, double cutoff,
               int mode, double *const *J, double *const *K, void *stream, jk_stats *stats,
               const LogSpec *logs = nullptr)
{
    if (!h) return fail(JK_ERR_ARG, "handle is NULL");
    if (!D) return fail(JK_ERR_ARG, "D is NULL");
    if (ndm < 1) return fail(JK_ERR_ARG, "n_dm must be >= 1");
    if (ndm > JK_NDM_MAX) return fail(JK_ERR_UNSUPPORTED, "n_dm=%d above %d", ndm, JK_NDM_MAX);
    if (!with_j && !with_k) return fail(JK_ERR_ARG, "with_j and with_k are both 0");
    if (!(cutoff >= 0) || !std::isfinite(cutoff)) return fail(JK_ERR_ARG, "cutoff must be finite and >= 0");
    if (mode < JK_PREC_FP64 || mode > JK_PREC_FP32) return fail(JK_ERR_ARG, "bad precision_mode %d", mode);
    if (mode == JK_PREC_MIXED_ROUTED && !h->has_router)
        return fail(JK_ERR_ARG, "MIXED_ROUTED needs router weights (jk_router_load)");
    if (logs && mode != JK_PREC_FP64) return fail(JK_ERR_ARG, "label logging runs in FP64");
    if (with_j && !J) return fail(JK_ERR_ARG, "J is NULL with with_j");
    if (with_k && !K) return fail(JK_ERR_ARG, "K is NULL with with_k");
    for (int m = 0; m < h->nmol; ++m) {
        if (!D[m]) return fail(JK_ERR_ARG, "D[%d] is NULL", m);
        if (with_j && !J[m]) return fail(JK_ERR_ARG, "J[%d] is NULL", m);
        if (with_k && !K[m]) return fail(JK_ERR_ARG, "K[%d] is NULL", m);
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev != h->device) return fail(JK_ERR_ARG, "current device %d differs from the handle's %d", dev, h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (int prc = poll_device_error(h, false)) return prc;

    // kernels for this combination
    std::vector<KSpec> specs;
    std::vector<int> lidx, tier;
    // tier 0 FP64, 1 FP32; routed builds add tier 2, the FP32 list kernel
    // of the quartets the router released from the FP64 tier (the router
    // itself runs in the FP64 tier only)
    const bool routed = mode == JK_PREC_MIXED_ROUTED;
    for (size_t i = 0; i < h->launches.size(); ++i) {
        for (int t = 0; t < 3; ++t) {
            const bool two = mode == JK_PREC_MIXED || routed;
            bool use = (t == 0) ? (mode == JK_PREC_FP64 || two) : (t == 1 ? (mode == JK_PREC_FP32 || two) : routed);
            if (!use) continue;
            KSpec s = h->launches[i].spec[t == 0 ? 0 : 1];
            s.ndm = ndm; s.doj = with_j ? 1 : 0; s.dok = with_k ? 1 : 0;
            s.mode = logs ? 2 : (routed ? (t == 0 ? 1 : (t == 2 ? 3 : 0)) : 0);
            s.op = h->omega == 0.0 ? 0 : (h->omega > 0.0 ? 1 : 2);
            specs.push_back(s);
            lidx.push_back((int)i);
            tier.push_back(t);
        }
    }
    std::vector<KInfo> ki;
    auto tc = std::chrono::steady_clock::now();
    int rc = ensure_kernels(specs, ki);
    if (rc) return rc;
    h->compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc).count();

    // Cartesian scratch for spherical molecules (3 x ndm x nao_c^2 each)
    if (h->spherical && h->cart_ndm < (size_t)ndm) {
        CK(cudaStreamSynchronize(st));
        cudaFree(h->d_cart);
        h->d_cart = nullptr;
        h->cart_off.assign(h->nmol, 0);
        size_t tot = 0;
        for (int m = 0; m < h->nmol; ++m)
            if (h->mol_sph[m]) { h->cart_off[m] = tot; tot += 3 * (size_t)ndm * h->nao_cart[m] * h->nao_cart[m]; }
        CK(cudaMalloc(&h->d_cart, sizeof(double) * std::max<size_t>(tot, 1)));
        h->cart_ndm = ndm;
        ++h->cart_gen;
    }
    // FP32 copies of the densities when the FP32 tier runs
    const bool use32 = mode != JK_PREC_FP64;
    if (use32 && h->d32_ndm < (size_t)ndm) {
        CK(cudaStreamSynchronize(st));
        cudaFree(h->d_d32);
        h->d_d32 = nullptr;
        h->d32_off.assign(h->nmol, 0);
        size_t tot = 0;
        for (int m = 0; m < h->nmol; ++m) { h->d32_off[m] = tot; tot += (size_t)ndm * h->nao_cart[m] * h->nao_cart[m]; }
        CK(cudaMalloc(&h->d_d32, sizeof(float) * std::max<size_t>(tot, 1)));
        h->d32_ndm = ndm;
        ++h->cart_gen;
    }
    // routed builds: one list per class pair for the quartets the router
    // releases from the FP64 tier, first sized by the pair's share of the
    // candidate quartets (at least 4,096 entries), then grown to what a
    // build with stats saw it need; a quartet that finds its list full stays
    // in FP64
    bool grow = false;
    if (routed && h->d_rlist)
        for (size_t i = 0; i < h->rl_need.size(); ++i) grow = grow || h->rl_need[i] > h->rl_cap[i];
    if (routed && (!h->d_rlist || grow)) {
        CK(cudaStreamSynchronize(st));
        cudaFree(h->d_rlist); cudaFree(h->d_rcount);
        h->d_rlist = nullptr; h->d_rcount = nullptr;
        double tc2 = 0;
        for (auto &L : h->launches) tc2 += L.cand;
        std::vector<long long> cap(h->launches.size());
        for (size_t i = 0; i < h->launches.size(); ++i) {
            const double share = tc2 > 0 ? h->launches[i].cand / tc2 : 1.0 / h->launches.size();
            cap[i] = std::max(4096LL, (long long)(h->route_cap * share));
            if (i < h->rl_cap.size()) cap[i] = std::max(cap[i], h->rl_cap[i]);
            if (i < h->rl_need.size() && h->rl_need[i] > cap[i]) cap[i] = h->rl_need[i] + h->rl_need[i] / 4 + 4096;
        }
        h->rl_off.assign(h->launches.size(), 0);
        h->rl_cap = cap;
        h->rl_need.assign(h->launches.size(), 0);
        long long tot = 0;
        for (size_t i = 0; i < h->launches.size(); ++i) {
            h->rl_off[i] = tot;
            tot += h->rl_cap[i];
        }
        CK(cudaMalloc(&h->d_rlist, sizeof(JkRouted) * (size_t)std::max(tot, 1LL)));
        CK(cudaMalloc(&h->d_rcount, sizeof(unsigned long long) * std::max<size_t>(h->launches.size(), 1)));
        ++h->cart_gen;
    }
    // per-molecule descriptors
    CK(cudaEventSynchronize(h->mol_copied));
    long long off = 0;
    for (int m = 0; m < h->nmol; ++m) {
        JkMol &x = h->h_mols[m];
        x.nao = h->nao_cart[m];
        if (h->mol_sph[m]) {
            const size_t nn = (size_t)ndm * x.nao * x.nao;
            double *base = h->d_cart + h->cart_off[m];
            x.D = base;
            x.J = with_j ? base + nn : nullptr;
            x.K = with_k ? base + 2 * nn : nullptr;
            JkSphMol &a = h->h_sph[m], &b = h->h_sph[h->nmol + m];
            a.src[0] = D[m]; a.dst[0] = base; a.src[1] = nullptr; a.dst[1] = nullptr; a.nsrc = 1;
            b.src[0] = x.J; b.dst[0] = with_j ? J[m] : nullptr;
            b.src[1] = x.K; b.dst[1] = with_k ? K[m] : nullptr; b.nsrc = 2;
            a.nao_c = b.nao_c = x.nao;
            a.nao_s = b.nao_s = h->nao_user[m];
            a.sh0 = b.sh0 = h->mol_sh0[m];
            a.nsh = b.nsh = h->mol_sh0[m + 1] - h->mol_sh0[m];
        } else {
            x.D = D[m];
            x.J = with_j ? J[m] : nullptr;
            x.K = with_k ? K[m] : nullptr;
            if (h->spherical) {
                JkSphMol &a = h->h_sph[m], &b = h->h_sph[h->nmol + m];
                a = JkSphMol{};
                b = JkSphMol{};
            }
        }
        x.D32 = use32 ? h->d_d32 + h->d32_off[m] : nullptr;
        x.nsh = h->mol_sh0[m + 1] - h->mol_sh0[m];
        x.dmax_off = off;
        off += (long long)x.nsh * x.nsh;
    }
    if (stats) CK(cudaEventRecord(h->ev0, st));
    CK(cudaMemcpyAsync(h->d_mols, h->h_mols, sizeof(JkMol) * h->nmol, cudaMemcpyHostToDevice, st));
    if (h->spherical)
        CK(cudaMemcpyAsync(h->d_sph, h->h_sph, sizeof(JkSphMol) * 2 * h->nmol, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(h->mol_copied, st));
    int max_nsh = 0, max_nao = 0;
    for (int m = 0; m < h->nmol; ++m) {
        max_nsh = std::max(max_nsh, h->mol_sh0[m + 1] - h->mol_sh0[m]);
        max_nao = std::max(max_nao, h->nao_cart[m]);
    }
    const size_t nl = h->launches.size() * 3;   // counters per launch and tier (incl. the routed list tier)
    const double inf = INFINITY;
    const bool prof = h->profile && stats;
    if (prof && h->prof_ev.size() < 2 * specs.size()) {
        size_t have = h->prof_ev.size();
        h->prof_ev.resize(2 * specs.size());
        for (size_t e = have; e < h->prof_ev.size(); ++e) CK(cudaEventCreate(&h->prof_ev[e]));
    }
    const int nbranch = std::max(1, std::min(h->branches, JK_MAX_BRANCHES + 1));
    int nlaunch_aux = 0;

    // Everything a build does on the device, in order, on stream s (and, for
    // nbranch > 1, forked onto the handle's side streams and joined back).
    // capturing: external event records become event nodes of the graph;
    // outside a capture they are plain records
    auto enqueue = [&](cudaStream_t s0, bool capturing) -> int {
        const unsigned rec_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        nlaunch_aux = 0;
        if (h->spherical) {
            dim3 g((unsigned)(((long long)max_nsh * max_nsh + 127) / 128), ndm, h->nmol);
            jk_sph_kernel<<<g, 128, 0, s0>>>(h->d_sph, h->d_sh_l, h->d_sh_sph, h->d_sh_ao, h->d_sh_aou, h->d_c2s,
                                             h->d_c2s_off, ndm, 1);
            CK(cudaGetLastError());
            ++nlaunch_aux;
        }
        {
            long long per = (long long)ndm * max_nao * max_nao;
            dim3 g((unsigned)std::min<long long>((per + 255) / 256, 4096), h->nmol);
            jk_zero_kernel<<<g, 256, 0, s0>>>(h->d_mols, ndm);
            CK(cudaGetLastError());
            ++nlaunch_aux;
        }
        CK(cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long) * nl, s0));
        CK(cudaMemsetAsync(h->d_stats, 0, sizeof(unsigned long long) * 3 * nl, s0));
        CK(cudaMemsetAsync(h->d_dmax_mol, 0, sizeof(unsigned long long) * h->nmol, s0));
        if (routed) CK(cudaMemsetAsync(h->d_rcount, 0, sizeof(unsigned long long) * h->launches.size(), s0));
        jk_dmax_kernel<<<h->nshell, 128, 0, s0>>>(h->d_mols, h->d_sh_mol, h->d_mol_sh0, h->d_sh_ao, h->d_sh_nc, ndm,
                                                  h->d_dmax, h->d_dmax32, h->d_dmax_mol, h->d_err);
        CK(cudaGetLastError());
        ++nlaunch_aux;
        if (use32) {
            long long per = (long long)ndm * max_nao * max_nao;
            dim3 g((unsigned)std::min<long long>((per + 255) / 256, 4096), h->nmol);
            jk_d32_kernel<<<g, 256, 0, s0>>>(h->d_mols, ndm);
            CK(cudaGetLastError());
            ++nlaunch_aux;
        }
        if (nbranch > 1) {
            CK(cudaEventRecord(h->ev_fork, s0));
            for (int b = 1; b < nbranch; ++b) CK(cudaStreamWaitEvent(h->side[b - 1], h->ev_fork, 0));
        }
        for (size_t k = 0; k < specs.size(); ++k) {
            // a routed class pair keeps its three launches on one stream (the
            // list kernel reads what the FP64 launch wrote)
            const size_t br = routed ? (size_t)lidx[k] : k;
            cudaStream_t sk = (nbranch > 1 && br % nbranch) ? h->side[br % nbranch - 1] : s0;
            const Launch &L = h->launches[lidx[k]];
            const PairClass &A = h->classes[L.c1], &B = h->classes[L.c2];
            JkClassArgs a;
            // bra and ket indices are relative to the base of their pair class
            a.bra = h->d_pairs + A.off;
            a.ket = h->d_pairs + B.off;
            a.ket_beg = B.d_beg;
            a.ket_end = B.d_end;
            a.pp64 = h->d_pp64;
            a.pp32 = h->d_pp32;
            a.mols = h->d_mols;
            a.dmax = h->d_dmax;
            a.dmax32 = h->d_dmax32;
            a.dmax_mol = reinterpret_cast<const double *>(h->d_dmax_mol);
            a.rys64 = h->d_rys64;
            a.rys32 = h->d_rys32;
            const int slot = lidx[k] * 3 + tier[k];
            a.work = h->d_work + slot;
            a.stats = h->d_stats + 3 * slot;
            a.err = h->d_err;
            const double tau = std::max(cutoff, h->tau32);
            const double band_hi = tau * h->router_band;
            if (mode == JK_PREC_MIXED) {
                if (tier[k] == 0) { a.lo = tau; a.hi = inf; }
                else { a.lo = cutoff; a.hi = tau; }
            } else if (mode == JK_PREC_MIXED_ROUTED) {
                // the FP32 tier keeps the Schwarz split; the band goes to the
                // FP64 tier, which routes it (tier 2 reads its list)
                if (tier[k] == 0) { a.lo = tau; a.hi = inf; }
                else { a.lo = cutoff; a.hi = tau; }
            } else {
                a.lo = cutoff; a.hi = inf;
            }
            a.bra_feat = h->d_pfeat + A.off;
            a.ket_feat = h->d_pfeat + B.off;
            a.router = h->d_router;
            a.tau = tau;
            a.band_hi = band_hi;
            // FP32 screening unless the cutoff is below the FP32 range; one
            // choice for every launch of the build, so that the tiers of a
            // mixed build compare the same bounds in the same precision
            // screening: FP32 bounds with the FP64 rule kept exact (2, the
            // default), plain FP32 (1, option screen64 = 0), or FP64 (0, for
            // cutoffs below the FP32 range)
            a.scr32 = cutoff >= 1e-30 ? (h->screen64 ? 2 : 1) : 0;
            a.lo32 = (float)a.lo;
            a.hi32 = std::isinf(a.hi) ? INFINITY : (float)a.hi;
            a.tau32 = (float)tau;
            a.band_hi32 = (float)band_hi;
            a.tier = tier[k] == 0 ? 0 : 1;
            a.rlist = routed ? h->d_rlist + h->rl_off[lidx[k]] : nullptr;
            a.rcount = routed ? h->d_rcount + lidx[k] : nullptr;
            a.rcap = routed ? h->rl_cap[lidx[k]] : 0;
            a.asym64 = h->asym64;
            a.widen_int = h->widen_int;
            a.log_x = logs ? logs->x : nullptr;
            a.log_y = logs ? logs->y : nullptr;
            a.log_n = h->d_logn;
            a.log_cap = logs ? logs->cap : 0;
            a.nbra = A.n;
            const int pi = (tier[k] == 0 && (mode == JK_PREC_MIXED || routed)) ? 1 : 0;
            a.item_prefix = L.d_prefix[pi];
            const long long nunits = L.nitems[pi] * specs[k].gx;   // work items x slabs
            a.item_lo = nunits * h->part_index / h->part_count;
            a.item_hi = nunits * (h->part_index + 1) / h->part_count;
            a.chunk = pi ? h->chunk_hi : h->chunk;
            a.prim_eps = std::min(cutoff, h->prim_eps);
            a.prim_eps32 = (float)a.prim_eps;
            a.omega = std::fabs(h->omega);
            a.same_class = (L.c1 == L.c2) ? 1 : 0;
            a.with_j = with_j ? 1 : 0;
            a.with_k = with_k ? 1 : 0;
            a.use_dmax = h->use_dmax;
            a.ndm = ndm;
            int grid = std::max(1, ki[k].blocks_per_sm) * h->num_sms;
            const long long units = specs[k].G() <= 32 ? 4 : 1;   // work items in flight per CTA
            long long need = (a.item_hi - a.item_lo + units - 1) / units;
            if (need < grid) grid = (int)std::max(1LL, need);
            void *params[] = {&a};
            // External records become event nodes when captured into a graph
            if (prof) CK(cudaEventRecordWithFlags(h->prof_ev[2 * k], sk, rec_flags));
            CUresult r = drv().launchKernel(ki[k].fn, grid, 1, 1, specs[k].block(), 1, 1, (unsigned)ki[k].smem,
                                            (CUstream)sk, params, nullptr);
            if (r != CUDA_SUCCESS) return fail(JK_ERR_CUDA, "launch of %s failed: %d", specs[k].name().c_str(), (int)r);
            if (prof) CK(cudaEventRecordWithFlags(h->prof_ev[2 * k + 1], sk, rec_flags));
        }
        if (nbranch > 1) {
            for (int b = 1; b < nbranch; ++b) {
                CK(cudaEventRecord(h->ev_join[b - 1], h->side[b - 1]));
                CK(cudaStreamWaitEvent(s0, h->ev_join[b - 1], 0));
            }
        }
        if (h->ntiles > 0) {
            dim3 grid((unsigned)h->ntiles, ndm, 2);
            jk_symmetrize_kernel<<<grid, dim3(32, 8), 0, s0>>>(h->d_mols, h->d_tile_off, h->nmol, ndm, with_j, with_k);
            CK(cudaGetLastError());
            ++nlaunch_aux;
        }
        if (h->spherical) {
            dim3 g((unsigned)(((long long)max_nsh * max_nsh + 127) / 128), ndm, h->nmol);
            jk_sph_kernel<<<g, 128, 0, s0>>>(h->d_sph + h->nmol, h->d_sh_l, h->d_sh_sph, h->d_sh_ao, h->d_sh_aou,
                                             h->d_c2s, h->d_c2s_off, ndm, 0);
            CK(cudaGetLastError());
            ++nlaunch_aux;
        }
        return JK_OK;
    };

    if (logs) CK(cudaMemsetAsync(h->d_logn, 0, sizeof(unsigned long long), st));
    if (h->use_graph && !logs) {
        // one CUDA graph per flag combination, captured on the handle's own
        // stream and replayed on the caller's; per-call pointers live in the
        // device descriptors copied above, so the graph stays valid.
        char keyb[160];
        snprintf(keyb, sizeof keyb, "%d/%d/%d/%d/%a/%a/%a/%d/%d/%zu/%d/%d/%d/%a/%d/%d", ndm, with_j, with_k, mode,
                 cutoff, h->tau32, h->router_band, h->use_dmax, nbranch, h->cart_gen, prof ? 1 : 0, h->part_index,
                 h->part_count, h->prim_eps, h->asym64, h->screen64 + 2 * h->widen_int);
        std::string key = keyb;
        char ob[40];
        snprintf(ob, sizeof ob, "/%a", h->omega);
        key += ob;
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
            int erc = enqueue(h->cap, true);
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(h->cap, &graph);
            if (erc) { if (graph) cudaGraphDestroy(graph); return erc; }
            if (ce != cudaSuccess) return fail(JK_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            cudaGraphExec_t exec = nullptr;
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(JK_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
            it = h->graphs.emplace(key, std::make_pair(exec, nlaunch_aux)).first;
        }
        nlaunch_aux = it->second.second;
        CK(cudaGraphLaunch(it->second.first, st));
    } else {
        int erc = enqueue(st, false);
        if (erc) return erc;
    }
    if (stats) {
        CK(cudaEventRecord(h->ev1, st));
        CK(cudaStreamSynchronize(st));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        std::vector<unsigned long long> cnt(3 * nl);
        CK(cudaMemcpy(cnt.data(), h->d_stats, sizeof(unsigned long long) * 3 * nl, cudaMemcpyDeviceToHost));
        int err = 0;
        CK(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (routed) {
            std::vector<unsigned long long> rc2(h->launches.size());
            CK(cudaMemcpy(rc2.data(), h->d_rcount, sizeof(unsigned long long) * rc2.size(), cudaMemcpyDeviceToHost));
            h->rl_need.assign(rc2.begin(), rc2.end());
        }
        memset(stats, 0, sizeof(*stats));
        int64_t routed_fp32 = 0;
        stats->ms = ms;
        stats->kernel_launches = (int64_t)specs.size() + nlaunch_aux;
        if (prof) { h->prof.clear(); h->prof_slot.clear(); }
        for (size_t k = 0; k < specs.size(); ++k) {
            const int slot = lidx[k] * 3 + tier[k];
            unsigned long long nq = cnt[3 * slot], np = cnt[3 * slot + 1];
            if (tier[k] == 0) stats->quartets_fp64 += (int64_t)nq;
            else stats->quartets_fp32 += (int64_t)nq;
            if (tier[k] == 2) routed_fp32 += (int64_t)nq;
            stats->prim_quartets += (int64_t)np;
            stats->flops_model += flops_of(specs[k], ndm, nq, np);
            if (prof) {
                jk_launch_prof p;
                const KSpec &x = specs[k];
                p.la = x.la; p.lb = x.lb; p.lc = x.lc; p.ld = x.ld;
                p.na = x.na; p.nb = x.nb; p.nc = x.nc; p.nd = x.nd;
                p.tier = tier[k] == 0 ? 0 : 1;
                p.threads_per_quartet = x.G();
                p.regs = ki[k].regs;
                p.local_bytes = ki[k].local_bytes;
                p.quartets = (int64_t)nq;
                p.prim_quartets = (int64_t)np;
                float lm = 0;
                CK(cudaEventElapsedTime(&lm, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]));
                p.ms = lm;
                p.flops_model = flops_of(x, ndm, nq, np);
                h->prof.push_back(p);
                h->prof_slot.push_back(slot);
            }
        }
        stats->quartets_routed = routed_fp32;
        h->err_pending = false;
        if (err) return device_error(h, err, "this build");
    } else {
        // no synchronisation here: the error word travels back with the
        // stream and is looked at by the next call on the handle
        CK(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(h->err_ev, st));
        h->err_pending = true;
    }
    return JK_OK;
}

// Device weights for inference from the FP32 master copy: BF16 rounding, and
// the matrices laid out as mma.m16n8k16 B fragments. For k-step ks, n-tile nt
// and lane (g = lane / 4, t = lane % 4) the two registers hold
// {W[16ks+2t][n], W[16ks+2t+1][n]} and {W[16ks+2t+8][n], W[16ks+2t+9][n]},
// n = 8nt + g, low half first.
static unsigned router_pack(float lo, float hi) { return (unsigned)jk_f2bf(lo) | ((unsigned)jk_f2bf(hi) << 16); }

template <typename W>
static void router_fragments(W w, int nks, int nnt, unsigned *dst)
{
    for (int ks = 0; ks < nks; ++ks)
        for (int nt = 0; nt < nnt; ++nt)
            for (int lane = 0; lane < 32; ++lane) {
                const int g = lane >> 2, t = lane & 3, n = nt * 8 + g, k = ks * 16 + 2 * t;
                unsigned *r = dst + ((size_t)(ks * nnt + nt) * 32 + lane) * 2;
                r[0] = router_pack(w(k, n), w(k + 1, n));
                r[1] = router_pack(w(k + 8, n), w(k + 9, n));
            }
}

void router_dev_from_blob(const jk_router_blob &w, JkRouterDev &d)
{
    memset(&d, 0, sizeof d);
    for (int i = 0; i < 16; ++i) { d.mu[i] = w.mu[i]; d.isd[i] = w.isd[i]; }
    const float *th = w.theta;
    router_fragments([th](int k, int n) { return th[JK_RT_OFF_W1 + k * JK_RT_NH + n]; }, 1, 8, d.W1p);
    router_fragments([th](int k, int n) { return th[JK_RT_OFF_W2 + k * JK_RT_NH + n]; }, 4, 8, d.W2p);
    router_fragments([th](int k, int n) { return n == 0 ? th[JK_RT_OFF_W3 + k] : 0.0f; }, 4, 1, d.W3p);
    for (int i = 0; i < JK_RT_NH; ++i) d.b1[i] = th[JK_RT_OFF_B1 + i];
    for (int i = 0; i < JK_RT_NH; ++i) d.b2[i] = th[JK_RT_OFF_B2 + i];
    d.b3 = th[JK_RT_OFF_B3];
    d.margin = w.margin;
}

int check_blob(const jk_router_blob *w)
{
    if (!w) return fail(JK_ERR_ARG, "router weights are NULL");
    if (w->magic != JK_ROUTER_MAGIC || w->version != 1) return fail(JK_ERR_ARG, "not a router weight blob");
    for (int i = 0; i < JK_ROUTER_NPARAM; ++i)
        if (!std::isfinite(w->theta[i])) return fail(JK_ERR_NAN, "non-finite router weight %d", i);
    return JK_OK;
}

}  // namespace

// ============================================= no-allocation gradient variant
// Fixed device scratch for jk_router_gradient_noalloc: the weight copies, the
// row list and the two accumulators of jk_mlp_grad_kernel live in one
// file-scope __device__ array (about 560 KB, held by every GPU that loads this
// library until the process exits) instead of buffers from cudaMalloc.
struct JkNoAllocScratch {   // JK_NOALLOC_MAX_ROWS comes from jk.h
    float theta[JK_RT_NPARAM];
    float mu[16], isd[16];
    float grad[JK_RT_NPARAM];
    double loss;
    long long idx[JK_NOALLOC_MAX_ROWS];
};
static __device__ __align__(256) unsigned char jk_noalloc_scratch[sizeof(JkNoAllocScratch)];

__global__ void jk_noalloc_iota_kernel(long long *idx, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) idx[t] = t;
}

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {};

// Device address of the scratch array on the current device. Host code may
// not use the array's name as an address, so it is looked up once per device
// (with that device current) and kept for the process (a cudaDeviceReset
// would invalidate it; the header says so).
int noalloc_scratch(JkNoAllocScratch **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(JK_ERR_UNSUPPORTED, "device ordinal %d above 63", dev);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, jk_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(JK_ERR_CUDA, "cudaGetSymbolAddress(jk_noalloc_scratch): %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = (JkNoAllocScratch *)g_noalloc_ptr[dev];
    return JK_OK;
}
}  // namespace

// ===================================================================== ABI
// Autotuner (the per-device grid search over fragmentations of Sec. 3.2, run
// on the caller's own data): every class-pair launch whose estimated share of
// the work is at least min_share gets up to maxc candidate shapes; round r
// gives every launch its r-th candidate and runs two serialised, profiled
// builds (CUDA events around each launch); each launch keeps its fastest
// candidate. The chosen shapes stay in the handle and go to the tuning table.
int tune_impl(jk_handle *h, const double *const *D, int32_t ndm, int with_j, int with_k, double cutoff, int mode,
              double *const *J, double *const *K, void *stream, int maxc, double min_share, jk_tune_report *rep)
{
    if (!h) return fail(JK_ERR_ARG, "handle is NULL");
    if (maxc < 1 || maxc > 16) return fail(JK_ERR_ARG, "max_candidates must be in 1..16");
    if (!(min_share >= 0.0 && min_share <= 1.0)) return fail(JK_ERR_ARG, "min_share must be in [0, 1]");
    if (mode < JK_PREC_FP64 || mode > JK_PREC_FP32) return fail(JK_ERR_ARG, "bad precision_mode %d", mode);
    if (ndm < 1 || ndm > JK_NDM_MAX) return fail(JK_ERR_ARG, "bad n_dm");
    const auto t0 = std::chrono::steady_clock::now();
    const bool two = mode == JK_PREC_MIXED || mode == JK_PREC_MIXED_ROUTED;
    std::vector<int> tiers;
    if (mode == JK_PREC_FP64 || two) tiers.push_back(0);
    if (mode == JK_PREC_FP32 || two) tiers.push_back(1);
    double total = 0;
    for (auto &L : h->launches) total += L.cost;
    struct Item {
        int l, t;
        std::vector<KSpec> c;
        double first = INFINITY, best = INFINITY;
        int bi = 0;
    };
    std::vector<Item> items;
    for (size_t l = 0; l < h->launches.size(); ++l) {
        const Launch &L = h->launches[l];
        if (L.nitems[0] == 0 || L.cost < min_share * total) continue;
        for (int t : tiers) {
            Item it;
            it.l = (int)l;
            it.t = t;
            it.c = fragment_candidates(L.spec[t], maxc);
            if (it.c.size() > 1) items.push_back(it);
        }
    }
    // every candidate compiled (in parallel) and loaded before any timing;
    // shapes that cannot be resident on an SM are dropped
    {
        std::vector<KSpec> all;
        for (auto &it : items)
            for (auto c : it.c) {
                c.ndm = ndm; c.doj = with_j ? 1 : 0; c.dok = with_k ? 1 : 0;
                c.mode = (mode == JK_PREC_MIXED_ROUTED && it.t == 0) ? 1 : 0;
                c.op = h->omega == 0.0 ? 0 : (h->omega > 0.0 ? 1 : 2);
                all.push_back(c);
            }
        std::vector<KInfo> ki;
        int rc = ensure_kernels(all, ki);
        if (rc) return rc;
        size_t k = 0;
        for (auto &it : items) {
            std::vector<KSpec> keep;
            for (size_t j = 0; j < it.c.size(); ++j, ++k)
                if (j == 0 || ki[k].blocks_per_sm >= 1) keep.push_back(it.c[j]);
            it.c = keep;
        }
    }
    size_t nround = 0;
    for (auto &it : items) nround = std::max(nround, it.c.size());
    std::map<int, int> by_slot;
    for (size_t i = 0; i < items.size(); ++i) by_slot[items[i].l * 3 + items[i].t] = (int)i;
    const int o_prof = h->profile, o_branches = h->branches, o_graph = h->use_graph;
    h->profile = 1;
    h->branches = 1;
    h->use_graph = 0;
    int rc = JK_OK;
    for (size_t r = 0; r < nround && rc == JK_OK; ++r) {
        for (auto &it : items) h->launches[it.l].spec[it.t] = it.c[std::min(r, it.c.size() - 1)];
        std::vector<double> tm(items.size(), INFINITY);
        for (int rep2 = 0; rep2 < 2 && rc == JK_OK; ++rep2) {
            jk_stats st;
            rc = build_impl(h, D, ndm, with_j, with_k, cutoff, mode, J, K, stream, &st);
            if (rc) break;
            for (size_t p = 0; p < h->prof.size(); ++p) {
                auto f = by_slot.find(h->prof_slot[p]);
                if (f != by_slot.end()) tm[f->second] = std::min(tm[f->second], (double)h->prof[p].ms);
            }
        }
        for (size_t i = 0; i < items.size(); ++i) {
            Item &it = items[i];
            if (r >= it.c.size()) continue;
            if (r == 0) it.first = tm[i];
            if (tm[i] < it.best) { it.best = tm[i]; it.bi = (int)r; }
        }
    }
    h->profile = o_prof;
    h->branches = o_branches;
    h->use_graph = o_graph;
    std::vector<KSpec> chosen;
    int changed = 0;
    double before = 0, after = 0;
    for (auto &it : items) {
        const int b = rc == JK_OK ? it.bi : 0;
        h->launches[it.l].spec[it.t] = it.c[b];
        chosen.push_back(it.c[b]);
        changed += b != 0;
        before += it.first;
        after += it.best;
    }
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second.first);
    h->graphs.clear();
    if (rc) return rc;
    tune_store(h->device, chosen);
    if (rep) {
        memset(rep, 0, sizeof(*rep));
        rep->launches_tuned = (int32_t)items.size();
        for (auto &it : items) rep->candidates_timed += (int32_t)it.c.size();
        rep->changed = changed;
        rep->ms_before = before;
        rep->ms_after = after;
        rep->tune_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return JK_OK;
}

extern "C" {

int jk_router_gradient_noalloc(const jk_router_blob *w, const float *X, const float *y, int64_t n, float quantile,
                               float *grad_host, double *loss, void *stream)
{
    int rc = check_blob(w);
    if (rc) return rc;
    if (!X || !y || !grad_host || !loss || n < 1 || !(quantile > 0 && quantile < 1))
        return fail(JK_ERR_ARG, "bad arguments");
    if (n > JK_NOALLOC_MAX_ROWS)
        return fail(JK_ERR_UNSUPPORTED, "n = %lld rows exceeds the fixed scratch of jk_router_gradient_noalloc (%d rows)",
                    (long long)n, JK_NOALLOC_MAX_ROWS);
    JkNoAllocScratch *S = nullptr;
    if ((rc = noalloc_scratch(&S))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(S->theta, w->theta, sizeof(float) * JK_RT_NPARAM, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->mu, w->mu, sizeof(float) * 16, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->isd, w->isd, sizeof(float) * 16, cudaMemcpyHostToDevice, st));
    // the accumulators keep the previous call's values: clear them
    CK(cudaMemsetAsync(S->grad, 0, sizeof(float) * JK_RT_NPARAM, st));
    CK(cudaMemsetAsync(&S->loss, 0, sizeof(double), st));
    jk_noalloc_iota_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S->idx, (long long)n);
    const size_t smem = 2 * JK_RT_NPARAM * sizeof(float);
    jk_mlp_grad_kernel<<<(unsigned)((n + 255) / 256), 256, smem, st>>>(S->theta, S->mu, S->isd, X, y, (long long)n,
                                                                       S->idx, (int)n, 0ull, quantile, S->grad,
                                                                       &S->loss);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(grad_host, S->grad, sizeof(float) * JK_RT_NPARAM, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(loss, &S->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return JK_OK;
}


int jk_init(const jk_shell *shells, int32_t nshell, const double *coords, int32_t natm, const double *exps,
            const double *coeffs, int32_t nprim_total, jk_handle **out)
{
    int32_t off[2] = {0, nshell};
    try {
        return init_impl(1, off, shells, nshell, coords, natm, exps, coeffs, nprim_total, out);
    } catch (const std::exception &e) {
        return fail(JK_ERR_OOM, "host exception: %s", e.what());
    }
}

int jk_init_batch(int32_t nmol, const int32_t *mol_shell_off, const jk_shell *shells, int32_t nshell,
                  const double *coords, int32_t natm, const double *exps, const double *coeffs,
                  int32_t nprim_total, jk_handle **out)
{
    try {
        return init_impl(nmol, mol_shell_off, shells, nshell, coords, natm, exps, coeffs, nprim_total, out);
    } catch (const std::exception &e) {
        return fail(JK_ERR_OOM, "host exception: %s", e.what());
    }
}

int jk_build(jk_handle *h, const double *D, int32_t n_dm, int with_j, int with_k, double cutoff,
             int precision_mode, double *J, double *K, void *stream, jk_stats *stats)
{
    if (!h) return fail(JK_ERR_ARG, "handle is NULL");
    if (h->nmol != 1) return fail(JK_ERR_ARG, "jk_build needs a single-molecule handle (use jk_build_batch)");
    try {
        return build_impl(h, &D, n_dm, with_j, with_k, cutoff, precision_mode, &J, &K, stream, stats);
    } catch (const std::exception &e) {
        return fail(JK_ERR_OOM, "host exception: %s", e.what());
    }
}

int jk_build_batch(jk_handle *h, const double *const *D, int32_t n_dm, int with_j, int with_k, double cutoff,
                   int precision_mode, double *const *J, double *const *K, void *stream, jk_stats *stats)
{
    if (!h) return fail(JK_ERR_ARG, "handle is NULL");
    if ((with_j && !J) || (with_k && !K)) return fail(JK_ERR_ARG, "J or K pointer array is NULL");
    std::vector<double *> Jn(h->nmol, nullptr), Kn(h->nmol, nullptr);
    try {
        return build_impl(h, D, n_dm, with_j, with_k, cutoff, precision_mode, J ? J : Jn.data(), K ? K : Kn.data(),
                          stream, stats);
    } catch (const std::exception &e) {
        return fail(JK_ERR_OOM, "host exception: %s", e.what());
    }
}

int jk_set_option(jk_handle *h, const char *key, double value)
{
    if (!h || !key) return fail(JK_ERR_ARG, "NULL handle or key");
    std::string k = key;
    if (k == "tau32") { if (!(value >= 0)) return fail(JK_ERR_ARG, "tau32 must be >= 0"); h->tau32 = value; }
    else if (k == "router_band") { if (!(value >= 1)) return fail(JK_ERR_ARG, "router_band must be >= 1"); h->router_band = value; }
    else if (k == "pair_cutoff") h->pair_cutoff = value;
    else if (k == "use_graph") h->use_graph = value != 0;
    else if (k == "use_dmax") h->use_dmax = value != 0;
    else if (k == "profile") h->profile = value != 0;
    else if (k == "omega") {
        if (!std::isfinite(value)) return fail(JK_ERR_ARG, "omega must be finite");
        h->omega = value;
    }
    else if (k == "prim_eps") {
        if (!(value >= 0) || !std::isfinite(value)) return fail(JK_ERR_ARG, "prim_eps must be finite and >= 0");
        h->prim_eps = value;
    }
    else if (k == "part_count") {
        if (!(value >= 1 && value <= 65536)) return fail(JK_ERR_ARG, "part_count must be in [1, 65536]");
        h->part_count = (int)value;
        if (h->part_index >= h->part_count) h->part_index = 0;
    }
    else if (k == "part_index") {
        if (!(value >= 0 && value < h->part_count)) return fail(JK_ERR_ARG, "part_index must be in [0, part_count)");
        h->part_index = (int)value;
    }
    else if (k == "branches") {
        if (!(value >= 1 && value <= JK_MAX_BRANCHES + 1)) return fail(JK_ERR_ARG, "branches must be in [1, %d]", JK_MAX_BRANCHES + 1);
        h->branches = (int)value;
    }
    else if (k == "asym64") h->asym64 = value != 0;
    else if (k == "widen_int") h->widen_int = value != 0;
    else if (k == "chunk" || k == "chunk_fp64tier") {
        if (!(value >= 32 && value <= 65536)) return fail(JK_ERR_ARG, "%s must be in [32, 65536]", key);
        const int c0 = k == "chunk" ? (int)value : h->chunk, c1 = k == "chunk" ? h->chunk_hi : (int)value;
        if (c0 != h->chunk || c1 != h->chunk_hi) {
            cudaDeviceSynchronize();
            for (auto &g : h->graphs) cudaGraphExecDestroy(g.second.first);
            h->graphs.clear();
            if (int rc = plan_items(h, c0, c1)) return rc;
        }
    }
    else if (k == "screen64") h->screen64 = value != 0;
    else if (k == "route_cap") {
        if (!(value >= 1 && value <= 1e9)) return fail(JK_ERR_ARG, "route_cap must be in [1, 1e9]");
        if (value != h->route_cap) {
            cudaDeviceSynchronize();
            cudaFree(h->d_rlist); cudaFree(h->d_rcount);
            h->d_rlist = nullptr; h->d_rcount = nullptr;
            h->rl_cap.clear(); h->rl_need.clear();
            for (auto &g : h->graphs) cudaGraphExecDestroy(g.second.first);
            h->graphs.clear();
        }
        h->route_cap = value;
    }
    else return fail(JK_ERR_ARG, "unknown option '%s'", key);
    return JK_OK;
}

int jk_get_option(jk_handle *h, const char *key, double *value)
{
    if (!h || !key || !value) return fail(JK_ERR_ARG, "NULL argument");
    std::string k = key;
    if (k == "tau32") *value = h->tau32;
    else if (k == "router_band") *value = h->router_band;
    else if (k == "pair_cutoff") *value = h->pair_cutoff;
    else if (k == "use_graph") *value = h->use_graph;
    else if (k == "use_dmax") *value = h->use_dmax;
    else if (k == "profile") *value = h->profile;
    else if (k == "branches") *value = h->branches;
    else if (k == "part_count") *value = h->part_count;
    else if (k == "prim_eps") *value = h->prim_eps;
    else if (k == "omega") *value = h->omega;
    else if (k == "part_index") *value = h->part_index;
    else if (k == "asym64") *value = h->asym64;
    else if (k == "widen_int") *value = h->widen_int;
    else if (k == "chunk") *value = h->chunk;
    else if (k == "chunk_fp64tier") *value = h->chunk_hi;
    else if (k == "screen64") *value = h->screen64;
    else if (k == "route_cap") *value = h->route_cap;
    else if (k == "graphs") *value = (double)h->graphs.size();
    else if (k == "init_ms") *value = h->init_ms;
    else if (k == "compile_ms") *value = h->compile_ms;
    else if (k == "npairs") *value = (double)h->h_pairs.size();
    else if (k == "nclasses") *value = (double)h->classes.size();
    else if (k == "nlaunches") *value = (double)h->launches.size();
    else return fail(JK_ERR_ARG, "unknown option '%s'", key);
    return JK_OK;
}

int jk_info(jk_handle *h, int32_t mol, int32_t *nao, int32_t *nshell, int32_t *nmol)
{
    if (!h) return fail(JK_ERR_ARG, "handle is NULL");
    if (mol < 0 || mol >= h->nmol) return fail(JK_ERR_ARG, "molecule index out of range");
    if (nao) *nao = h->nao_user[mol];
    if (nshell) *nshell = h->mol_sh0[mol + 1] - h->mol_sh0[mol];
    if (nmol) *nmol = h->nmol;
    return JK_OK;
}

int jk_schwarz(jk_handle *h, double *Q)
{
    if (!h || !Q) return fail(JK_ERR_ARG, "NULL argument");
    int ns = h->mol_sh0[1] - h->mol_sh0[0];
    std::fill(Q, Q + (size_t)ns * ns, 0.0);
    for (auto &p : h->h_pairs)
        if (p.mol == 0) Q[(size_t)p.a_loc * ns + p.b_loc] = Q[(size_t)p.b_loc * ns + p.a_loc] = p.Q;
    return JK_OK;
}

int jk_check(jk_handle *h, void *stream)
{
    if (!h) return fail(JK_ERR_ARG, "handle is NULL");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    h->err_pending = false;
    int err = 0;
    CK(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) return device_error(h, err, "a build on this handle");
    return JK_OK;
}

int jk_destroy(jk_handle *h)
{
    if (!h) return fail(JK_ERR_ARG, "handle is NULL");
    cudaDeviceSynchronize();
    int err = 0;
    if (h->d_err && cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        err = 0;
    }
    free_handle(h);
    if (err & JK_ERR_DEV_NAN)
        return fail(JK_ERR_NAN, "a build on the destroyed handle saw NaN or infinite density values");
    return JK_OK;
}

int jk_router_load(jk_handle *h, const jk_router_blob *w)
{
    if (!h) return fail(JK_ERR_ARG, "handle is NULL");
    int rc = check_blob(w);
    if (rc) return rc;
    JkRouterDev d;
    router_dev_from_blob(*w, d);
    CK(cudaMemcpy(h->d_router, &d, sizeof d, cudaMemcpyHostToDevice));
    h->has_router = true;
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second.first);
    h->graphs.clear();
    return JK_OK;
}

int jk_router_collect(jk_handle *h, const double *const *D, int32_t n_dm, double cutoff, double *const *J,
                      double *const *K, float *X, float *y, int64_t cap, int64_t *n, void *stream)
{
    if (!h || !X || !y || !n || cap < 1 || !J || !K) return fail(JK_ERR_ARG, "NULL argument or cap < 1");
    LogSpec ls{X, y, (long long)cap};
    jk_stats st;
    int rc;
    try {
        rc = build_impl(h, D, n_dm, 1, 1, cutoff, JK_PREC_FP64, J, K, stream, &st, &ls);
    } catch (const std::exception &e) {
        return fail(JK_ERR_OOM, "host exception: %s", e.what());
    }
    if (rc) return rc;
    unsigned long long cnt = 0;
    CK(cudaMemcpy(&cnt, h->d_logn, sizeof cnt, cudaMemcpyDeviceToHost));
    *n = (int64_t)cnt;
    return JK_OK;
}

int jk_router_forward(const jk_router_blob *w, const float *X, int64_t n, float *y_out)
{
    int rc = check_blob(w);
    if (rc) return rc;
    if (!X || !y_out || n < 0) return fail(JK_ERR_ARG, "bad arguments");
    if (n == 0) return JK_OK;
    JkRouterDev d;
    router_dev_from_blob(*w, d);
    JkRouterDev *dd = nullptr;
    CK(cudaMalloc(&dd, sizeof d));
    cudaMemcpy(dd, &d, sizeof d, cudaMemcpyHostToDevice);
    jk_mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128>>>(dd, X, (long long)n, y_out);
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(dd);
    if (e != cudaSuccess) return fail(JK_ERR_CUDA, "router forward: %s", cudaGetErrorString(e));
    return JK_OK;
}

int jk_router_gradient(const jk_router_blob *w, const float *X, const float *y, int64_t n, float quantile,
                       float *grad_host, double *loss)
{
    int rc = check_blob(w);
    if (rc) return rc;
    if (!X || !y || !grad_host || !loss || n < 1 || n > (1 << 30) || !(quantile > 0 && quantile < 1))
        return fail(JK_ERR_ARG, "bad arguments");
    float *th = nullptr, *mu = nullptr, *isd = nullptr, *g = nullptr;
    double *l = nullptr;
    long long *idx = nullptr;
    std::vector<long long> iota((size_t)n);
    for (int64_t i = 0; i < n; ++i) iota[i] = i;
    auto cleanup = [&]() { cudaFree(th); cudaFree(mu); cudaFree(isd); cudaFree(g); cudaFree(l); cudaFree(idx); };
    struct Guard { std::function<void()> f; ~Guard() { f(); } } guard{cleanup};
    CK(cudaMalloc(&th, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMalloc(&mu, sizeof(float) * 16));
    CK(cudaMalloc(&isd, sizeof(float) * 16));
    CK(cudaMalloc(&g, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMalloc(&l, sizeof(double)));
    CK(cudaMalloc(&idx, sizeof(long long) * n));
    CK(cudaMemcpy(th, w->theta, sizeof(float) * JK_RT_NPARAM, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(mu, w->mu, sizeof(float) * 16, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(isd, w->isd, sizeof(float) * 16, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(idx, iota.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
    CK(cudaMemset(g, 0, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMemset(l, 0, sizeof(double)));
    const size_t smem = 2 * JK_RT_NPARAM * sizeof(float);
    jk_mlp_grad_kernel<<<(unsigned)((n + 255) / 256), 256, smem>>>(th, mu, isd, X, y, (long long)n, idx, (int)n, 0ull,
                                                                 quantile, g, l);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(grad_host, g, sizeof(float) * JK_RT_NPARAM, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(loss, l, sizeof(double), cudaMemcpyDeviceToHost));
    return JK_OK;
}

int jk_router_train(const float *X, const float *y, int64_t n, const jk_train_opts *opts, jk_router_blob *out,
                    jk_train_stats *stats)
{
    if (!X || !y || !opts || !out || n < 2) return fail(JK_ERR_ARG, "bad arguments");
    if (opts->steps < 1 || opts->batch < 1 || opts->batch > (1 << 22) || !(opts->lr > 0) ||
        !(opts->quantile > 0 && opts->quantile < 1))
        return fail(JK_ERR_ARG, "bad training options");
    auto t0 = std::chrono::steady_clock::now();
    // feature normalisation from the data
    std::vector<float> hx((size_t)n * JK_RT_NIN);
    CK(cudaMemcpy(hx.data(), X, sizeof(float) * hx.size(), cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->magic = JK_ROUTER_MAGIC;
    out->version = 1;
    out->quantile = opts->quantile;
    for (int k = 0; k < 16; ++k) { out->mu[k] = 0.f; out->isd[k] = 0.f; }
    for (int k = 0; k < JK_RT_NIN; ++k) {
        double m = 0, v = 0;
        for (int64_t i = 0; i < n; ++i) m += hx[i * JK_RT_NIN + k];
        m /= n;
        for (int64_t i = 0; i < n; ++i) { double d = hx[i * JK_RT_NIN + k] - m; v += d * d; }
        v /= n;
        out->mu[k] = (float)m;
        out->isd[k] = (float)(1.0 / std::max(std::sqrt(v), 1e-6));
    }
    // initial weights: uniform(-a, a), a = sqrt(6 / (fan_in + fan_out)); biases 0
    unsigned long long z = opts->seed ^ 0x6a09e667f3bcc909ull;
    auto rnd = [&]() {
        z += 0x9e3779b97f4a7c15ull;
        unsigned long long r = z;
        r = (r ^ (r >> 30)) * 0xbf58476d1ce4e5b9ull;
        r = (r ^ (r >> 27)) * 0x94d049bb133111ebull;
        r ^= r >> 31;
        return (double)(r >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    float *th = out->theta;
    for (int i = 0; i < JK_RT_NPARAM; ++i) th[i] = 0.f;
    const double a1 = std::sqrt(6.0 / (JK_RT_NIN + JK_RT_NH)), a2 = std::sqrt(6.0 / (2 * JK_RT_NH)),
                 a3 = std::sqrt(6.0 / (JK_RT_NH + 1));
    for (int i = 0; i < JK_RT_NIN; ++i)
        for (int o = 0; o < JK_RT_NH; ++o) th[JK_RT_OFF_W1 + i * JK_RT_NH + o] = (float)(a1 * rnd());
    for (int i = 0; i < JK_RT_NH * JK_RT_NH; ++i) th[JK_RT_OFF_W2 + i] = (float)(a2 * rnd());
    for (int i = 0; i < JK_RT_NH; ++i) th[JK_RT_OFF_W3 + i] = (float)(a3 * rnd());
    {
        std::vector<float> hy((size_t)n);
        CK(cudaMemcpy(hy.data(), y, sizeof(float) * n, cudaMemcpyDeviceToHost));
        double m = 0;
        for (auto v : hy) m += v;
        th[JK_RT_OFF_B3] = (float)(m / n);
    }
    float *dth = nullptr, *mu = nullptr, *isd = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    double *lh = nullptr;
    auto cleanup = [&]() { cudaFree(dth); cudaFree(mu); cudaFree(isd); cudaFree(g); cudaFree(m1); cudaFree(m2); cudaFree(lh); };
    struct Guard { std::function<void()> f; ~Guard() { f(); } } guard{cleanup};
    CK(cudaMalloc(&dth, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMalloc(&g, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMalloc(&m1, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMalloc(&m2, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMalloc(&mu, sizeof(float) * 16));
    CK(cudaMalloc(&isd, sizeof(float) * 16));
    CK(cudaMalloc(&lh, sizeof(double) * opts->steps));
    CK(cudaMemcpy(dth, th, sizeof(float) * JK_RT_NPARAM, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(mu, out->mu, sizeof(float) * 16, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(isd, out->isd, sizeof(float) * 16, cudaMemcpyHostToDevice));
    CK(cudaMemset(m1, 0, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMemset(m2, 0, sizeof(float) * JK_RT_NPARAM));
    CK(cudaMemset(lh, 0, sizeof(double) * opts->steps));
    const size_t smem = 2 * JK_RT_NPARAM * sizeof(float);
    const unsigned gb = (unsigned)((opts->batch + 255) / 256);
    for (int step = 1; step <= opts->steps; ++step) {
        CK(cudaMemsetAsync(g, 0, sizeof(float) * JK_RT_NPARAM));
        jk_mlp_grad_kernel<<<gb, 256, smem>>>(dth, mu, isd, X, y, (long long)n, nullptr, opts->batch,
                                               opts->seed * 1000003ull + (unsigned long long)step, opts->quantile, g,
                                               lh + (step - 1));
        jk_adam_kernel<<<(JK_RT_NPARAM + 255) / 256, 256>>>(dth, g, m1, m2, step, opts->lr, 0.9f, 0.999f, 1e-8f);
    }
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(th, dth, sizeof(float) * JK_RT_NPARAM, cudaMemcpyDeviceToHost));
    std::vector<double> hl(opts->steps);
    CK(cudaMemcpy(hl.data(), lh, sizeof(double) * opts->steps, cudaMemcpyDeviceToHost));
    if (stats) {
        const int w = std::min(50, opts->steps);
        double a = 0, b = 0;
        for (int i = 0; i < w; ++i) { a += hl[i]; b += hl[opts->steps - 1 - i]; }
        stats->loss_first = a / w;
        stats->loss_last = b / w;
        stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return JK_OK;
}

int jk_profile(jk_handle *h, jk_launch_prof *out, int32_t max, int32_t *n)
{
    if (!h || !n || (max > 0 && !out)) return fail(JK_ERR_ARG, "NULL argument");
    int32_t c = (int32_t)std::min<size_t>(h->prof.size(), (size_t)std::max(0, max));
    for (int32_t i = 0; i < c; ++i) out[i] = h->prof[i];
    *n = (int32_t)h->prof.size();
    return JK_OK;
}

int jk_measure_peak(int32_t which, double ms, double *flops_per_s)
{
    if (!flops_per_s || (which != 0 && which != 1) || !(ms > 0)) return fail(JK_ERR_ARG, "bad argument");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    void *sink = nullptr;
    CK(cudaMalloc(&sink, 16));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int threads = 256, blocks = sms * 8;
    auto run = [&](int iters) -> float {
        cudaEventRecord(e0);
        if (which == 0) jk_fma_probe_kernel<double><<<blocks, threads>>>(iters, 1.0, (double *)sink);
        else jk_fma_probe_kernel<float><<<blocks, threads>>>(iters, 1.0f, (float *)sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        return t;
    };
    int iters = 64;
    run(iters);
    float t = run(iters);
    while (t < ms && iters < (1 << 26)) { iters *= 2; t = run(iters); }
    t = run(iters);
    double flops = 2.0 * 8 * 16 * (double)iters * threads * blocks;
    *flops_per_s = flops / (t * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    CK(cudaGetLastError());
    return JK_OK;
}

int jk_compile_class(int32_t la, int32_t lb, int32_t lc, int32_t ld, int32_t na, int32_t nb, int32_t nc,
                     int32_t nd, int32_t n_dm, int32_t with_j, int32_t with_k, int32_t fp32, int32_t mode,
                     int32_t op, int32_t *threads_per_quartet, double *compile_ms)
{
    if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > JK_LMAX || lb > JK_LMAX || lc > JK_LMAX || ld > JK_LMAX)
        return fail(JK_ERR_UNSUPPORTED, "angular momentum out of range");
    if (na < 1 || nb < 1 || nc < 1 || nd < 1 || na > JK_NPRIM_MAX || nb > JK_NPRIM_MAX || nc > JK_NPRIM_MAX ||
        nd > JK_NPRIM_MAX)
        return fail(JK_ERR_UNSUPPORTED, "primitive count out of range");
    if (n_dm < 1 || n_dm > JK_NDM_MAX || (!with_j && !with_k)) return fail(JK_ERR_ARG, "bad n_dm or flags");
    if (mode < 0 || mode > 3 || (mode == 2 && fp32) || (mode == 3 && !fp32)) return fail(JK_ERR_ARG, "bad mode");
    if (op < 0 || op > 2) return fail(JK_ERR_ARG, "bad op");
    KSpec s;
    s.kind = 0;
    s.la = la; s.lb = lb; s.lc = lc; s.ld = ld; s.na = na; s.nb = nb; s.nc = nc; s.nd = nd;
    s.ndm = n_dm; s.doj = with_j ? 1 : 0; s.dok = with_k ? 1 : 0; s.fp32 = fp32 ? 1 : 0;
    s.mode = mode;
    s.op = op;
    choose_fragments(s, false);
    if (threads_per_quartet) *threads_per_quartet = s.G();
    try {
        return compile_to_disk({s}, compile_ms);
    } catch (const std::exception &e) {
        return fail(JK_ERR_COMPILE, "host exception: %s", e.what());
    }
}

int jk_compile_basis(const jk_shell *shells, int32_t nshell, int32_t n_dm, int32_t with_j, int32_t with_k,
                     int32_t fp32, int32_t mode, double *compile_ms, int32_t *nkernels)
{
    if (!shells || nshell < 1) return fail(JK_ERR_ARG, "no shells");
    if (n_dm < 1 || n_dm > JK_NDM_MAX || (!with_j && !with_k)) return fail(JK_ERR_ARG, "bad n_dm or flags");
    if (mode < 0 || mode > 3 || (mode == 2 && fp32) || (mode == 3 && !fp32)) return fail(JK_ERR_ARG, "bad mode");
    // shell types (l, nprim) -> pair classes (larger type first) -> class pairs
    std::vector<std::pair<int, int>> types;
    for (int i = 0; i < nshell; ++i) {
        if (shells[i].l < 0 || shells[i].l > JK_LMAX || shells[i].nprim < 1 || shells[i].nprim > JK_NPRIM_MAX)
            return fail(JK_ERR_UNSUPPORTED, "shell %d out of range", i);
        types.push_back({shells[i].l, shells[i].nprim});
    }
    std::sort(types.begin(), types.end());
    types.erase(std::unique(types.begin(), types.end()), types.end());
    std::reverse(types.begin(), types.end());
    std::vector<std::pair<int, int>> pcs;   // indices into types, a <= b (a is the larger type)
    for (size_t a = 0; a < types.size(); ++a)
        for (size_t b = a; b < types.size(); ++b) pcs.push_back({(int)a, (int)b});
    std::vector<KSpec> specs;
    for (auto &pc : pcs) {
        KSpec s;
        s.kind = 1;
        s.la = s.lc = types[pc.first].first; s.lb = s.ld = types[pc.second].first;
        s.na = s.nc = types[pc.first].second; s.nb = s.nd = types[pc.second].second;
        choose_fragments(s, true);
        specs.push_back(s);
        s.na = s.nb = s.nc = s.nd = 1;
        choose_fragments(s, true);
        specs.push_back(s);
    }
    for (size_t i = 0; i < pcs.size(); ++i)
        for (size_t j = i; j < pcs.size(); ++j) {
            KSpec s;
            s.kind = 0;
            s.la = types[pcs[i].first].first; s.lb = types[pcs[i].second].first;
            s.lc = types[pcs[j].first].first; s.ld = types[pcs[j].second].first;
            s.na = types[pcs[i].first].second; s.nb = types[pcs[i].second].second;
            s.nc = types[pcs[j].first].second; s.nd = types[pcs[j].second].second;
            s.ndm = n_dm; s.doj = with_j ? 1 : 0; s.dok = with_k ? 1 : 0; s.fp32 = fp32 ? 1 : 0; s.mode = mode;
            choose_fragments(s, false);
            specs.push_back(s);
        }
    if (nkernels) *nkernels = (int32_t)specs.size();
    try {
        return compile_to_disk(specs, compile_ms);
    } catch (const std::exception &e) {
        return fail(JK_ERR_COMPILE, "host exception: %s", e.what());
    }
}

int jk_autotune(jk_handle *h, const double *const *D, int32_t n_dm, int with_j, int with_k, double cutoff,
                int precision_mode, double *const *J, double *const *K, void *stream, int32_t max_candidates,
                double min_share, jk_tune_report *report)
{
    try {
        return tune_impl(h, D, n_dm, with_j, with_k, cutoff, precision_mode, J, K, stream, max_candidates, min_share,
                         report);
    } catch (const std::exception &e) {
        return fail(JK_ERR_CUDA, "host exception: %s", e.what());
    }
}

int jk_fragment_candidates(int32_t la, int32_t lb, int32_t lc, int32_t ld, int32_t fp32, int32_t max_candidates,
                           int32_t *frag, int32_t *n)
{
    if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > JK_LMAX || lb > JK_LMAX || lc > JK_LMAX || ld > JK_LMAX)
        return fail(JK_ERR_UNSUPPORTED, "angular momentum out of range");
    if (max_candidates < 1 || max_candidates > 16 || !frag || !n) return fail(JK_ERR_ARG, "bad arguments");
    KSpec s;
    s.kind = 0;
    s.la = la; s.lb = lb; s.lc = lc; s.ld = ld;
    s.fp32 = fp32 ? 1 : 0;
    choose_fragments(s, false);
    auto c = fragment_candidates(s, max_candidates);
    for (size_t i = 0; i < c.size(); ++i) {
        frag[4 * i] = c[i].ga; frag[4 * i + 1] = c[i].gb; frag[4 * i + 2] = c[i].gc; frag[4 * i + 3] = c[i].gd;
    }
    *n = (int32_t)c.size();
    return JK_OK;
}

const char *jk_last_error(void) { return g_err.c_str(); }

}  // extern "C"
