// sbp_api.cu — plans, plan-time tables, launch configuration and the C ABI.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <cstdio>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/sbp.h"

#include <type_traits>
#include "sbp_internal.h"

using namespace sbp;


namespace {

constexpr int kMaxLen = 2048;
constexpr size_t kSmemBudget = 224 * 1024;  // under the 227 KB opt-in limit, leaving room for static smem

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
bool supported_len(int n) {
    if (n < 2 || n > kMaxLen) return false;
    if (is_pow2(n)) return true;
    return n % 3 == 0 && is_pow2(n / 3);
}

bool build_fft_plan(int n, int E, FftPlan& P) {
    std::memset(&P, 0, sizeof(P));
    P.n = n;
    P.E = E;
    if (n % P.E != 0) return false;
    P.Tf = n / P.E;
    int rem = n, ns = 1, s = 0;
    while (rem > 1) {
        const int r = pick_radix(P.E, rem);  // the same choice as the compile-time plans
        if (r == 0 || s >= kMaxStages) return false;
        P.radix[s] = r;
        P.ns[s] = ns;
        P.tws[s] = n / (ns * r);
        ns *= r;
        rem /= r;
        ++s;
    }
    P.nstage = s;
    return true;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct PassCfg {
    int E = 0, C = 0, threads = 0;
    size_t smem = 0;
    dim3 grid;
};

}  // namespace

struct sbp_plan_s {
    int nx = 0, ny = 0, nz = 0;
    double Lx = 0, Ly = 0, Lz = 0, q = 0, Omega = 0, G = 0;
    sbp_dtype dtype = SBP_F64;
    int device = 0;
    int pitch = 0, h = 0;
    size_t rsize = 0;  // bytes per real
    FftPlan px{}, py{}, pz{};
    PassCfg xf, xi, yp, zp;
    int z_variant = 0;         // see SBP_OPT_Z_VARIANT
    bool z_padded = false;     // the chosen kernel takes the length-2nz twiddle table
    // vertical truncation L = alpha·Lz (SBP_OPT_TRUNCATION); alpha > 1 pads
    // the vertical transform to pad = 4 times nz (else 2)
    double alpha = 1.0;
    int pad = 2;
    // method (SBP_OPT_METHOD): 0 = VGF-HybridBC, 1 = SASHA with Φ0's vertex at z0
    // (as printed), 2 = SASHA with the vertex at z0/2
    int method = 0;
    int chunk = 0;  // planes per x/y chunk of a single solve (SBP_OPT_XY_CHUNK; 0: whole box)
    // explicitly requested five-pass variants (SBP_OPT_XY_PASSES, SBP_OPT_Z_VARIANT, SBP_OPT_Y_TMA)
    int xy_req = 0, z_req = 0, ytma_req = 0;
    // schedule (SBP_OPT_SCHEDULE): 0 = automatic, 1 = five passes, 2 = three sweeps
    int schedule = 0;
    bool sweep = false;              // solves run the three-sweep kernels
    SweepKernels sk;
    int sweep_green_blocks = 0;
    SweepBox* sweep_box = nullptr;   // this plan's device descriptor (in `tables`)
    CUtensorMap sweep_tmap;          // its tensor map (also copied into batched descriptors)
    // z-pass geometry: stored columns per row, rows per plane, row pitch
    int zh = 0, zrows = 0, zpitch = 0;
    // physical frame (SBP_OPT_FRAME = 1): y-first passes with the mapping of Sect. 2.1
    int frame = 0;
    void* ry_fwd = nullptr;
    void* ry_inv = nullptr;
    void* rows_fwd = nullptr;
    void* rows_inv = nullptr;
    void* shear_cols = nullptr;
    int ry_threads = 0, ry_tiles = 0, ry_green_blocks = 0, rows_threads = 0, rows_grid = 0;
    size_t ry_smem = 0, rows_smem = 0;
    void* z_fn = nullptr;      // the z-pass kernel of the chosen variant
    int green_blocks = 0;      // x-forward blocks that fill the Green's table
    // fused xy plane kernels (square planes with a built kernel), used by solves
    bool xy_fused = false;
    void* xy_fwd = nullptr;
    void* xy_inv = nullptr;
    int xy_cluster = 0, xy_threads = 0, xy_green_ctas = 0;
    size_t xy_smem_fwd = 0, xy_smem_inv = 0;
    // device memory
    void* W = nullptr;        // half spectrum
    void* tables = nullptr;   // twiddles, kz², c00, tile sums, vk0
    size_t W_bytes = 0, tables_bytes = 0;
    void* tw_x = nullptr;
    void* tw_y = nullptr;
    void* tw_z = nullptr;
    void* tw_2z = nullptr;
    void* tw_M = nullptr;      // e^{-2πi k/(2nz)}, k < 2nz
    void* tw_M4 = nullptr;     // e^{-2πi k/(4nz)}, k < 4nz
    void* paper_tab = nullptr; // per |m| ≤ 2nz: k_z sin(k_z L), 1 - cos(k_z L), k_z², Ĝ(0, k_z) (pad = 4)
    void* kz2 = nullptr;
    double* c00 = nullptr;
    double* tile_sums = nullptr;
    double* vk0 = nullptr;    // FP64 mean-mode potential per plane (FP32 path)
    void* side = nullptr;     // [nz][2][ny] shifted boundary columns (physical-frame force)
    void* green = nullptr;    // GreenT<T>[ny][nx/2+1] for the current solve
    int* err = nullptr;       // device status word: 1 after a bounded wait gave up
    // TMA y passes (static ny): tile loads of the half spectrum
    bool y_tma = false;
    CUtensorMap tmap_y;
    size_t y_tma_smem = 0;
    long long spin_budget = 2000000000LL;  // clock cycles per bounded wait (about 1 s)
    int withhold = 0;                      // test switch (SBP_OPT_DEBUG_WITHHOLD_COPY)
};

namespace {

bool f64_of(const sbp_plan_s* p) { return p->dtype == SBP_F64; }

// The CUDA error behind the calling thread's last SBP_ERR_CUDA from a launch.
thread_local cudaError_t g_last_cuda = cudaSuccess;

sbp_status launch_status() {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return SBP_OK;
    g_last_cuda = e;
    return SBP_ERR_CUDA;
}

template <typename T>
size_t zpass_smem(int n, int C) {
    const size_t cs = sizeof(cpx<T>);
    const size_t kz2_bytes = align_up((size_t)(n + 1) * sizeof(T), 16);
    const size_t gm_bytes = align_up((size_t)C * sizeof(GreenT<T>), 16);
    return 2 * n * cs + kz2_bytes + gm_bytes + 2 * (size_t)n * xstride(C) * cs;
}

template <typename T>
size_t zpad_smem(int n, int C) {
    const size_t cs = sizeof(cpx<T>);
    const size_t gm_bytes = align_up((size_t)C * sizeof(GreenT<T>), 16);
    return 2 * (size_t)n * cs + gm_bytes + (size_t)xchg_slots<T>(2 * n, C) * cs;
}

// k_z_paper: twM[4n] | table [2n+1][4] | green[C] | exchange of C columns of 4n
template <typename T>
size_t zpaper_smem(int n, int C) {
    const size_t cs = sizeof(cpx<T>);
    const size_t tab_bytes = align_up(4 * (size_t)(2 * n + 1) * sizeof(T), 16);
    const size_t gm_bytes = align_up((size_t)C * sizeof(GreenT<T>), 16);
    return 4 * (size_t)n * cs + tab_bytes + gm_bytes + (size_t)xchg_slots<T>(4 * n, C) * cs;
}

template <typename T>
size_t ypass_smem(int n, int C) {
    // static column counts use XchgCol, runtime ones the padded stride
    const size_t slots = std::max((size_t)n * xstride(C), (size_t)xchg_slots<T>(n, C));
    return (size_t)n * sizeof(cpx<T>) + slots * sizeof(cpx<T>);
}

template <typename T>
size_t xfwd_smem(int n, int C) {
    return (size_t)n * sizeof(cpx<T>) + (size_t)C * padded_row(n) * sizeof(cpx<T>);
}

template <typename T>
size_t xinv_smem(int n, int C) {
    return (size_t)n * sizeof(cpx<T>) + (size_t)C * padded_row(n) * sizeof(cpx<T>);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        cudaGetLastError();
    });
    return fn;
}

// TMA y passes: a 2D map over a half spectrum viewed as rows of 2·pitch
// reals (one row per (z, y)), boxes of 2·C reals by min(ny, 256) rows.
template <typename T>
bool encode_ymap(const sbp_plan_s* p, void* spectrum, CUtensorMap* map) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)2 * p->pitch, (cuuint64_t)p->nz * p->ny};
    cuuint64_t strides[1] = {(cuuint64_t)2 * p->pitch * sizeof(T)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * p->yp.C), (cuuint32_t)std::min(p->ny, 256)};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, spectrum,
               dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
bool configure_ytma(sbp_plan_s* p, bool enable) {
    p->y_tma = false;
    if (!enable || !is_static_len<T>(p->ny) || p->W == nullptr) return !enable;
    const KernelSet<T> ky = kernels_for<T>(p->ny, p->py.E);
    auto enc = tensor_map_encoder();
    if (!ky.y_fwd_tma || !ky.y_inv_tma || !enc) return false;
    const int C = p->yp.C;
    const size_t smem = align_up((size_t)tile_slots<T>(p->ny, C) * sizeof(cpx<T>), 16) + (size_t)p->ny * sizeof(cpx<T>) + 16;
    if (smem > kSmemBudget || (2 * C * sizeof(T)) % 16 != 0) return false;
    if (!encode_ymap<T>(p, p->W, &p->tmap_y)) return false;
    if (cudaFuncSetAttribute(ky.y_fwd_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) !=
            cudaSuccess ||
        cudaFuncSetAttribute(ky.y_inv_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    p->y_tma_smem = smem;
    p->y_tma = true;
    return true;
}

// z-pass variant (SBP_OPT_Z_VARIANT): 0 = automatic (3 where built, else 4);
// 1 = E = 8 with joint halves; 2 = E = 8 with split halves; 3 = one padded
// length-2nz transform per column; 4 = plan_E with split halves (every
// length).  Returns false, leaving the plan unchanged, when the variant does
// not exist for this length or does not fit.
template <typename T>
bool configure_z(sbp_plan_s* p, int variant) {
    const bool f64 = std::is_same<T, double>::value;
    const int cmax = f64 ? 8 : 16;
    if (p->pad == 4) {
        // fourfold padding has one kernel: k_z_paper (power-of-two nz ≤ 512 FP32, ≤ 256 FP64)
        if (variant != 0) return false;
        int E = 0;
        ZKernel<T> fn = zpaper_for<T>(p->nz, &E);
        if (!fn) return false;
        FftPlan P;
        if (!build_fft_plan(4 * p->nz, E, P)) return false;
        const int C = zpad_cols(2 * p->nz, E, f64);
        const size_t smem = zpaper_smem<T>(p->nz, C);
        if (C * P.Tf > kMaxThreads || smem > kSmemBudget) return false;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        p->pz = P;
        p->zp.E = E;
        p->zp.C = C;
        p->zp.threads = C * P.Tf;
        p->zp.smem = smem;
        p->zp.grid = dim3((unsigned)((p->zh + C - 1) / C), (unsigned)p->zrows, 1);
        p->z_variant = 0;
        p->z_padded = false;
        p->z_fn = reinterpret_cast<void*>(fn);
        return true;
    }
    if (variant == 0) return configure_z<T>(p, 3) || configure_z<T>(p, 4);
    int E = plan_E(p->nz, f64);
    bool joint = false, padded = false;
    ZKernel<T> fn = nullptr;
    if (variant == 4) {
        fn = kernels_for<T>(p->nz, E).z;
    } else if (variant == 1 || variant == 2) {
        E = 8;
        joint = (variant == 1);
        fn = zvariant_for<T>(p->nz, E, joint);
    } else if (variant == 3) {
        padded = true;
        fn = zpad_for<T>(p->nz, &E);
    }
    if (!fn) return false;
    FftPlan P;
    if (!build_fft_plan(padded ? 2 * p->nz : p->nz, E, P)) return false;
    const int per_col = (padded || joint ? 1 : 2) * P.Tf;
    auto smem = [&](int C) { return padded ? zpad_smem<T>(p->nz, C) : zpass_smem<T>(p->nz, C); };
    int C = std::max(1, std::min(cmax, kMaxThreads / per_col));
    if (padded) {
        C = zpad_cols(p->nz, E, f64);  // compiled into the kernel
    } else {
        C = std::min(C, p->zh);
        while (C > 1 && smem(C) > kSmemBudget) --C;
    }
    if (C * per_col > kMaxThreads || smem(C) > kSmemBudget) return false;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    p->pz = P;
    p->zp.E = E;
    p->zp.C = C;
    p->zp.threads = C * per_col;
    p->zp.smem = smem(C);
    p->zp.grid = dim3((unsigned)((p->zh + C - 1) / C), (unsigned)p->zrows, 1);
    p->z_variant = variant;
    p->z_padded = padded;
    p->z_fn = reinterpret_cast<void*>(fn);
    return true;
}

// xy pass variant (SBP_OPT_XY_PASSES): 0 = automatic, 1 = separate x and y
// passes, 2 = fused plane kernels with one CTA per SM, 3 = fused with two
// CTAs per SM.  Returns false, leaving the plan unchanged, when unavailable.
template <typename T>
bool configure_xy(sbp_plan_s* p, int variant) {
    if (variant == 0) {
        // measured on GB300: the fused plane kernels win for the small FP32
        // planes only; larger planes stream better through the separate passes
        const bool small = !f64_of(p) && p->nx == p->ny && p->nx <= 96;
        return (small && configure_xy<T>(p, 2)) || configure_xy<T>(p, 1);
    }
    if (variant == 1) {
        p->xy_fused = false;
        return true;
    }
    if (p->nx != p->ny || (variant != 2 && variant != 3)) return false;
    if (f64_of(p) && p->method != 0) return false;  // the FP64 plane kernels make no plane sums
    const XYKernels<T> k = xy_kernels_for<T>(p->nx, variant - 1);
    if (!k.fwd || !k.inv || k.smem_fwd > kSmemBudget || k.smem_inv > kSmemBudget) return false;
    if (cudaFuncSetAttribute(k.fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) != cudaSuccess ||
        cudaFuncSetAttribute(k.inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // the FP32 mean-mode tile sums hold one value per CTA of a plane
    if ((long long)p->nz * k.cluster > (long long)p->xf.grid.x) return false;
    p->xy_fused = true;
    p->xy_fwd = reinterpret_cast<void*>(k.fwd);
    p->xy_inv = reinterpret_cast<void*>(k.inv);
    p->xy_cluster = k.cluster;
    p->xy_threads = k.threads;
    p->xy_smem_fwd = k.smem_fwd;
    p->xy_smem_inv = k.smem_inv;
    const int per = k.threads * k.cluster;
    p->xy_green_ctas = (p->h * p->ny + per - 1) / per * k.cluster;
    return true;
}

template <typename T>
bool configure(sbp_plan_s* p) {
    const bool f64 = std::is_same<T, double>::value;
    const int cmax = f64 ? 8 : 16;
    // x passes: C row pairs per block, C | ny/2, threads ≤ kMaxThreads
    {
        const int Tf = p->px.Tf;
        int C = std::max(1, std::min(cmax, kMaxThreads / Tf));
        while (C > 1 && ((p->ny / 2) % C != 0 || xinv_smem<T>(p->nx, C) > kSmemBudget)) --C;
        if ((p->ny / 2) % C != 0) return false;
        const long long pairs = (long long)p->nz * p->ny / 2;
        p->xf.E = p->xi.E = p->px.E;
        p->xf.C = p->xi.C = C;
        p->xf.threads = p->xi.threads = C * Tf;
        p->xf.smem = xfwd_smem<T>(p->nx, C);
        p->xi.smem = xinv_smem<T>(p->nx, C);
        p->xf.grid = p->xi.grid = dim3((unsigned)(pairs / C), 1, 1);
        if (p->xf.threads > kMaxThreads || p->xi.smem > kSmemBudget) return false;
    }
    // y passes: C columns per block
    {
        const int Tf = p->py.Tf;
        int C = std::max(1, std::min(cmax, kMaxThreads / Tf));
        if (is_static_len<T>(p->ny)) {
            C = ypass_cols(p->ny, f64);  // compiled into the static kernel
        } else {
            C = std::min(C, p->h);
            while (C > 1 && ypass_smem<T>(p->ny, C) > kSmemBudget) --C;
        }
        p->yp.E = p->py.E;
        p->yp.C = C;
        p->yp.threads = C * Tf;
        p->yp.smem = ypass_smem<T>(p->ny, C);
        p->yp.grid = dim3((unsigned)((p->h + C - 1) / C), (unsigned)p->nz, 1);
        if (p->yp.threads > kMaxThreads || p->yp.smem > kSmemBudget) return false;
    }
    // Opt in to the full dynamic shared-memory budget for the kernels this
    // plan uses.  Always the same value, so plans never lower each other's limit.
    const KernelSet<T> kx = kernels_for<T>(p->nx, p->px.E), ky = kernels_for<T>(p->ny, p->py.E);
    if (!kx.x_fwd || !ky.y_fwd) return false;
    const int lim = (int)kSmemBudget;
    cudaError_t e = cudaFuncSetAttribute(kx.x_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kx.x_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ky.y_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ky.y_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    // Green's-table blocks in front of the x-forward grid: one table entry per
    // thread, so that the FP64 work spreads over as many SMs as possible.
    p->green_blocks = (p->h * p->ny + p->xf.threads - 1) / p->xf.threads;
    configure_xy<T>(p, 0);
    return e == cudaSuccess && configure_z<T>(p, 0);
}

// FP64 twiddles e^{-2πi k/n}, k < count, scaled angle step `num/den` of 2π.
void host_twiddles(std::vector<double>& out, int count, double frac_den) {
    out.resize(2 * (size_t)count);
    for (int k = 0; k < count; ++k) {
        const double ang = kTwoPi * (double)k / frac_den;
        out[2 * k] = std::cos(ang);
        out[2 * k + 1] = -std::sin(ang);
    }
}

// k = 0 vertical kernel (Eq. Green's function regularized in Fourier, first
// two cases): Ĝ(0,0) = L²/2, Ĝ(0, k_z) = [k_z L sin(k_z L) + cos(k_z L) - 1]/k_z²
// at k_z = 2π m/(pad·Lz), m ∈ [-pad·nz/2, pad·nz/2).
double g0_vertical(double kz, double L) {
    if (kz == 0.0) return 0.5 * L * L;
    const double a = kz * L;
    return (a * std::sin(a) + std::cos(a) - 1.0) / (kz * kz);
}

// c00_n = (1/M) Σ_m Ĝ(0, m) cos(2π m n / M) for |n| < nz, M = pad·nz.  With
// L = Lz and pad = 2 (k_z L = π m) the terms are ((-1)^m - 1)/k_z²; the
// integer phase m·n mod M keeps the cosines exact to rounding.
void host_c00(std::vector<double>& c, int nz, double Lz, int pad, double L) {
    const int M = pad * nz;
    c.assign(2 * (size_t)nz - 1, 0.0);
    std::vector<double> g(M);
    const bool exact = (pad == 2 && L == Lz);
    for (int m = -M / 2; m < M / 2; ++m) {
        const double kz = kTwoPi * (double)m / (pad * Lz);
        g[m + M / 2] = !exact ? g0_vertical(kz, L) : (m == 0 ? 0.5 * L * L : ((m & 1) ? -2.0 / (kz * kz) : 0.0));
    }
    for (int n = -(nz - 1); n <= nz - 1; ++n) {
        double acc = 0.0;
        for (int m = -M / 2; m < M / 2; ++m) {
            long long ph = ((long long)m * n) % M;
            if (ph < 0) ph += M;
            acc += g[m + M / 2] * std::cos(kTwoPi * (double)ph / (double)M);
        }
        c[n + nz - 1] = acc / (double)M;
    }
}

// SASHA: the k = 0 column of Eq. (Poisson spectral) on the 2 nz padded grid,
// c_n = (1/M) Σ_{m ≠ 0} (-1/k_z²) cos(2π m n / M), k_z = π m / Lz.
void host_c00_periodic(std::vector<double>& c, int nz, double Lz) {
    const int M = 2 * nz;
    c.assign(2 * (size_t)nz - 1, 0.0);
    for (int n = -(nz - 1); n <= nz - 1; ++n) {
        double acc = 0.0;
        for (int m = -nz; m < nz; ++m) {
            if (m == 0) continue;
            const double kz = M_PI * (double)m / Lz;
            long long ph = ((long long)m * n) % M;
            if (ph < 0) ph += M;
            acc += (-1.0 / (kz * kz)) * std::cos(kTwoPi * (double)ph / (double)M);
        }
        c[n + nz - 1] = acc / (double)M;
    }
}

// Per |m| ≤ 2nz for fourfold padding: k_z sin(k_z L), 1 - cos(k_z L) (as
// 2 sin²(k_z L/2)), k_z² and Ĝ(0, k_z), with k_z = π m/(2 Lz), L = alpha·Lz,
// laid out [m][4] so that one m is one 16-byte (FP32) load.
void host_paper_tab(std::vector<double>& out, int nz, double Lz, double L) {
    const int NT = 2 * nz + 1;
    out.assign(4 * (size_t)NT, 0.0);
    for (int m = 0; m < NT; ++m) {
        const double kz = kTwoPi * (double)m / (4.0 * Lz);
        const double h = std::sin(0.5 * kz * L);
        out[4 * m] = kz * std::sin(kz * L);
        out[4 * m + 1] = 2.0 * h * h;
        out[4 * m + 2] = kz * kz;
        out[4 * m + 3] = g0_vertical(kz, L);
    }
}

template <typename T>
sbp_status upload_tables(sbp_plan_s* p) {
    std::vector<double> twx, twy, twz, tw2;
    host_twiddles(twx, p->nx, p->nx);
    host_twiddles(twy, p->ny, p->ny);
    host_twiddles(twz, p->nz, p->nz);
    host_twiddles(tw2, p->nz, 2.0 * p->nz);  // e^{-πi p/nz}
    std::vector<double> twM;
    host_twiddles(twM, 2 * p->nz, 2.0 * p->nz);  // e^{-2πi k/(2nz)}
    std::vector<double> kz2(p->nz + 1);
    for (int m = 0; m <= p->nz; ++m) {
        const double kz = M_PI * (double)m / p->Lz;
        kz2[m] = kz * kz;
    }
    const bool f32 = !f64_of(p);
    std::vector<double> c00;
    if (f32) host_c00(c00, p->nz, p->Lz, p->pad, p->alpha * p->Lz);
    std::vector<double> twM4, ptab;
    host_twiddles(twM4, 4 * p->nz, 4.0 * p->nz);  // e^{-2πi k/(4nz)}
    host_paper_tab(ptab, p->nz, p->Lz, p->alpha * p->Lz);

    const size_t cs = sizeof(cpx<T>);
    const int tiles = (int)p->xf.grid.x;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_twx = take(p->nx * cs), o_twy = take(p->ny * cs), o_twz = take(p->nz * cs);
    const size_t o_tw2 = take(p->nz * cs), o_kz2 = take((p->nz + 1) * sizeof(T));
    const size_t o_twM = take(2 * (size_t)p->nz * cs);
    const size_t o_twM4 = take(4 * (size_t)p->nz * cs);
    const size_t o_ptab = take(ptab.size() * sizeof(T));
    const size_t o_c00 = take((2 * (size_t)p->nz) * sizeof(double));
    const int ry_tiles = (p->nx / 2 + ypass_cols(p->ny, !f32) - 1) / ypass_cols(p->ny, !f32) * p->nz;
    const int sweep_tiles = p->nz * std::max(1, sweep_ra(p->ny) > 0 ? p->ny / sweep_ra(p->ny) : 1);
    const size_t o_ts = take((size_t)std::max(std::max(tiles, ry_tiles), sweep_tiles) * sizeof(double));
    const size_t o_vk0 = take((size_t)p->nz * sizeof(double));
    const size_t o_err = take(sizeof(int));
    const size_t o_side = take((size_t)p->nz * 2 * p->ny * sizeof(T));
    const size_t o_green = take(std::max((size_t)p->h * p->ny, (size_t)p->nx * (p->ny / 2 + 1)) * sizeof(GreenT<T>));
    const size_t o_sbox = take(sizeof(SweepBox));
    p->tables_bytes = off;
    if (cudaMalloc(&p->tables, off) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_OUT_OF_MEMORY;
    }
    unsigned char* base = static_cast<unsigned char*>(p->tables);
    p->tw_x = base + o_twx;
    p->tw_y = base + o_twy;
    p->tw_z = base + o_twz;
    p->tw_2z = base + o_tw2;
    p->kz2 = base + o_kz2;
    p->c00 = reinterpret_cast<double*>(base + o_c00);
    p->tile_sums = reinterpret_cast<double*>(base + o_ts);
    p->vk0 = reinterpret_cast<double*>(base + o_vk0);
    p->err = reinterpret_cast<int*>(base + o_err);
    p->side = base + o_side;
    p->tw_M = base + o_twM;
    p->tw_M4 = base + o_twM4;
    p->paper_tab = base + o_ptab;
    p->green = base + o_green;
    p->sweep_box = reinterpret_cast<SweepBox*>(base + o_sbox);

    std::vector<unsigned char> host(off, 0);
    {
        // the plan's descriptor for the three-sweep kernels (FP32 plans; rho,
        // phi and the shear parameter come with each launch)
        SweepBox d;
        std::memset(&d, 0, sizeof(d));
        d.err = p->err;
        d.S = reinterpret_cast<cpx<float>*>(p->W);
        d.green = reinterpret_cast<GreenT<float>*>(p->green);
        d.tile_sums = p->tile_sums;
        d.vk0 = p->vk0;
        d.c00 = p->c00;
        d.Lx = p->Lx;
        d.Ly = p->Ly;
        d.L = p->alpha * p->Lz;
        d.scale = 4.0 * M_PI * p->G / ((double)p->nx * p->ny * 2.0 * p->nz);
        d.kzc = (M_PI / p->Lz) * (M_PI / p->Lz);
        d.k0_coef = 4.0 * M_PI * p->G / ((double)p->nx * p->ny);
        std::memcpy(host.data() + o_sbox, &d, sizeof(d));
    }
    auto put_cpx = [&](size_t o, const std::vector<double>& v) {
        T* d = reinterpret_cast<T*>(host.data() + o);
        for (size_t i = 0; i < v.size(); ++i) d[i] = (T)v[i];
    };
    put_cpx(o_twx, twx);
    put_cpx(o_twy, twy);
    put_cpx(o_twz, twz);
    put_cpx(o_tw2, tw2);
    put_cpx(o_twM, twM);
    put_cpx(o_twM4, twM4);
    put_cpx(o_ptab, ptab);  // real table: same element-wise conversion
    {
        T* d = reinterpret_cast<T*>(host.data() + o_kz2);
        for (int m = 0; m <= p->nz; ++m) d[m] = (T)kz2[m];
    }
    if (f32) std::memcpy(host.data() + o_c00, c00.data(), c00.size() * sizeof(double));
    if (cudaMemcpy(p->tables, host.data(), off, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }
    return SBP_OK;
}

// Re-derive the tables that depend on the vertical truncation (FP32 c00 and
// the fourfold-padding table) after alpha or pad changed.
template <typename T>
sbp_status refresh_vertical_tables(sbp_plan_s* p) {
    std::vector<double> ptab;
    host_paper_tab(ptab, p->nz, p->Lz, p->alpha * p->Lz);
    std::vector<T> pt(ptab.begin(), ptab.end());
    if (cudaMemcpy(p->paper_tab, pt.data(), pt.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }
    if (!f64_of(p) || p->method != 0) {
        std::vector<double> c00;
        if (p->method != 0)
            host_c00_periodic(c00, p->nz, p->Lz);
        else
            host_c00(c00, p->nz, p->Lz, p->pad, p->alpha * p->Lz);
        if (cudaMemcpy(p->c00, c00.data(), c00.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return SBP_ERR_CUDA;
        }
    }
    return SBP_OK;
}

void free_plan(sbp_plan_s* p) {
    if (!p) return;
    if (p->W) cudaFree(p->W);
    if (p->tables) cudaFree(p->tables);
    delete p;
}

double shear_s(const sbp_plan_s* p, double t) {
    double dy0 = std::fmod(p->q * p->Omega * p->Lx * t, p->Ly);
    if (dy0 < 0.0) dy0 += p->Ly;
    if (dy0 >= p->Ly) dy0 -= p->Ly;
    return dy0 / p->Lx;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            prev = -1;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// SASHA k = 0 column (see SashaArgs).  smem: S[nz] doubles (dynamic)
__global__ void __launch_bounds__(256) k_sasha_k0(SashaArgs A) {
    extern __shared__ double S[];
    __shared__ double red[2 * (256 / 32)];
    const int tid = threadIdx.x;
    const int nz = A.nz;
    const double dz = A.Lz / nz;
    double s1 = 0.0, s2 = 0.0;
    for (int j = tid; j < nz; j += blockDim.x) {
        double sacc = 0.0;
        for (int q = 0; q < A.tiles_per_plane; ++q) sacc += A.tile_sums[(size_t)j * A.tiles_per_plane + q];
        S[j] = sacc;
        s1 += sacc;
        s2 += (-0.5 * A.Lz + (j + 0.5) * dz) * sacc;
    }
    const double2 tot = block_sum_d2(make_double2(s1, s2), red);  // its barriers also publish S
    const double rbar = tot.x / (A.cells_xy * nz);
    const double zeta = A.centre * (tot.x != 0.0 ? tot.y / tot.x : 0.0);
    const double sub = rbar * A.cells_xy;
    for (int i = tid; i < nz; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < nz; ++j) acc += A.c00[i - j + nz - 1] * (S[j] - sub);
        const double zi = -0.5 * A.Lz + (i + 0.5) * dz;
        A.vk0[i] = A.k0_coef * acc + A.fourpiG * rbar * zi * (0.5 * zi - zeta);
    }
}

GreenFill make_green_fill(const sbp_plan_s* p, double t, int blocks) {
    GreenFill g;
    g.tab = p->green;
    const int total = p->frame ? p->nx * (p->ny / 2 + 1) : p->h * p->ny;
    g.per_block = (total + blocks - 1) / blocks;
    g.nx = p->nx;
    g.ny = p->ny;
    g.yhalf = p->frame;
    g.Lx = p->Lx;
    g.Ly = p->Ly;
    g.L = p->method != 0 ? HUGE_VAL : p->alpha * p->Lz;  // SASHA: e^{-kL} = 0, Ĝ = -1/|k|²
    g.s = shear_s(p, t);
    g.s_dev = nullptr;
    return g;
}

// SASHA: the k = 0 column after the z pass (the x or y inverse pass adds it).
sbp_status launch_sasha_k0(const sbp_plan_s* p, int tiles_per_plane, cudaStream_t st) {
    SashaArgs a;
    a.tile_sums = p->tile_sums;
    a.tiles_per_plane = tiles_per_plane;
    a.nz = p->nz;
    a.c00 = p->c00;
    a.k0_coef = 4.0 * M_PI * p->G / ((double)p->nx * p->ny);
    a.fourpiG = 4.0 * M_PI * p->G;
    a.cells_xy = (double)p->nx * p->ny;
    a.Lz = p->Lz;
    a.centre = p->method == 2 ? 0.5 : 1.0;
    a.vk0 = p->vk0;
    k_sasha_k0<<<1, 256, (size_t)p->nz * sizeof(double), st>>>(a);
    return launch_status();
}

template <typename T>
XArgs make_xargs(const sbp_plan_s* p) {
    XArgs a;
    std::memset(&a, 0, sizeof(a));
    a.P = p->px;
    a.pitch = p->pitch;
    a.C = p->xf.C;
    a.pairs_per_plane = p->ny / 2;
    a.green_blocks = 0;
    a.gf.tab = nullptr;
    a.vk0 = nullptr;
    return a;
}
TmaCtl make_tmactl(const sbp_plan_s* p) {
    TmaCtl c;
    c.err = p->err;
    c.budget = p->spin_budget;
    c.withhold = p->withhold;
    return c;
}

template <typename T>
YArgs make_yargs(const sbp_plan_s* p) {
    YArgs a;
    a.P = p->py;
    a.pitch = p->pitch;
    a.h = p->h;
    a.C = p->yp.C;
    a.z0 = 0;
    return a;
}
template <typename T>
ZArgs make_zargs(const sbp_plan_s* p, bool with_k0) {
    ZArgs a;
    a.P = p->pz;
    a.pitch = p->zpitch;
    a.h = p->zh;
    a.ny = p->zrows;
    a.C = p->zp.C;
    a.L = p->alpha * p->Lz;
    a.kzc = (M_PI / p->Lz) * (M_PI / p->Lz);
    a.scale = 4.0 * M_PI * p->G / ((double)p->nx * p->ny * (double)p->pad * p->nz);
    a.paper_tab = p->paper_tab;
    const bool f32 = !f64_of(p);
    const bool side_k0 = f32 || p->method != 0;  // k = 0 column on the FP64 side path
    a.zero_k0 = side_k0 ? 1 : 0;
    a.green = p->green;
    a.tile_sums = p->tile_sums;
    a.tiles_per_plane = p->frame ? p->ry_tiles : (p->xy_fused ? p->xy_cluster : (p->ny / 2) / p->xf.C);
    a.c00 = p->c00;
    a.k0_coef = 4.0 * M_PI * p->G / ((double)p->nx * p->ny);
    // SASHA's k = 0 column comes from k_sasha_k0 after the z pass
    a.vk0 = (side_k0 && with_k0 && p->method == 0) ? p->vk0 : nullptr;
    return a;
}

// Launch one stage.  `fused` = part of a full solve: the x forward pass also
// fills the Green's table (and FP32 tile sums), the z pass reduces plane sums
// and the x inverse pass adds the FP64 mean mode.  Run alone, a stage does
// only its own transform; the z pass then fills its table first.
template <typename T>
// z0, nzc: the x and y stages may run on planes [z0, z0 + nzc) only (a chunk
// of the box, see solve_t); nzc < 0 means the whole box.
sbp_status launch_stage(sbp_plan_s* p, int stage, const void* in, void* out, double t, cudaStream_t st,
                        bool fused, const double* s_dev = nullptr, int z0 = 0, int nzc = -1) {
    const KernelSet<T> kx = kernels_for<T>(p->nx, p->px.E), ky = kernels_for<T>(p->ny, p->py.E);
    const bool f32 = !f64_of(p);
    cpx<T>* W = static_cast<cpx<T>*>(out);
    if (nzc < 0) {
        z0 = 0;
        nzc = p->nz;
    }
    const size_t plane_re = (size_t)p->nx * p->ny, plane_sp = (size_t)p->ny * p->pitch;
    const int x_blocks = (int)((long long)nzc * (p->ny / 2) / p->xf.C);  // row-pair blocks of the chunk
    YArgs ya = make_yargs<T>(p);
    ya.z0 = z0;
    const dim3 ygrid(p->yp.grid.x, (unsigned)nzc, 1);
    switch (stage) {
        case SBP_STAGE_X_FORWARD: {
            XArgs a = make_xargs<T>(p);
            dim3 grid = p->xf.grid;
            grid.x = (unsigned)x_blocks;
            if (fused && z0 == 0) {  // the whole Green's table, with the first chunk
                a.green_blocks = p->green_blocks;
                a.gf = make_green_fill(p, t, p->green_blocks);
                a.gf.s_dev = s_dev;
                grid.x += p->green_blocks;
            }
            double* sums = ((f32 || p->method != 0) && fused) ? p->tile_sums : nullptr;
            if (sums) sums += (size_t)z0 * (p->ny / 2) / p->xf.C;
            kx.x_fwd<<<grid, p->xf.threads, p->xf.smem, st>>>(static_cast<const T*>(in) + z0 * plane_re,
                                                             W + z0 * plane_sp,
                                                             static_cast<const cpx<T>*>(p->tw_x), sums, a);
            break;
        }
        case SBP_STAGE_Y_FORWARD:
            if (p->y_tma) {
                // the plan's map covers its own workspace; other buffers get their own
                CUtensorMap local;
                const CUtensorMap* map = &p->tmap_y;
                if (out != p->W) {
                    if (!encode_ymap<T>(p, out, &local)) return SBP_ERR_INVALID_ARG;
                    map = &local;
                }
                ky.y_fwd_tma<<<ygrid, p->yp.threads, p->y_tma_smem, st>>>(
                    W, static_cast<const cpx<T>*>(p->tw_y), ya, make_tmactl(p), *map);
            } else {
                ky.y_fwd<<<ygrid, p->yp.threads, p->yp.smem, st>>>(W, static_cast<const cpx<T>*>(p->tw_y), ya);
            }
            break;
        case SBP_STAGE_GREEN_FILL: {
            const int blocks = (p->h * p->ny + 255) / 256;
            k_green_params<T><<<blocks, 256, 0, st>>>(make_green_fill(p, t, blocks));
            break;
        }
        case SBP_STAGE_Z_CONVOLVE:
            reinterpret_cast<ZKernel<T>>(p->z_fn)<<<p->zp.grid, p->zp.threads, p->zp.smem, st>>>(
                W, static_cast<const cpx<T>*>(p->tw_z),
                static_cast<const cpx<T>*>(p->pad == 4 ? p->tw_M4 : (p->z_padded ? p->tw_M : p->tw_2z)),
                static_cast<const T*>(p->kz2), make_zargs<T>(p, fused));
            if (fused && p->method != 0) {
                const sbp_status s = launch_sasha_k0(p, make_zargs<T>(p, true).tiles_per_plane, st);
                if (s != SBP_OK) return s;
            }
            break;
        case SBP_STAGE_Y_INVERSE:
            if (p->y_tma) {
                // the plan's map covers its own workspace; other buffers get their own
                CUtensorMap local;
                const CUtensorMap* map = &p->tmap_y;
                if (out != p->W) {
                    if (!encode_ymap<T>(p, out, &local)) return SBP_ERR_INVALID_ARG;
                    map = &local;
                }
                ky.y_inv_tma<<<ygrid, p->yp.threads, p->y_tma_smem, st>>>(
                    W, static_cast<const cpx<T>*>(p->tw_y), ya, make_tmactl(p), *map);
            } else {
                ky.y_inv<<<ygrid, p->yp.threads, p->yp.smem, st>>>(W, static_cast<const cpx<T>*>(p->tw_y), ya);
            }
            break;
        case SBP_STAGE_X_INVERSE: {
            XArgs a = make_xargs<T>(p);
            if ((f32 || p->method != 0) && fused) a.vk0 = p->vk0 + z0;
            kx.x_inv<<<dim3((unsigned)x_blocks), p->xi.threads, p->xi.smem, st>>>(
                static_cast<const cpx<T>*>(in) + z0 * plane_sp, static_cast<T*>(out) + z0 * plane_re,
                static_cast<const cpx<T>*>(p->tw_x), a);
            break;
        }
        case SBP_STAGE_GREEN_TABLE: {
            // fill the plan's table exactly as a solve does, then report it as stored
            const int total = p->h * p->ny;
            const int blocks = (total + 255) / 256;
            k_green_params<T><<<blocks, 256, 0, st>>>(make_green_fill(p, t, blocks));
            k_green_dump<T><<<blocks, 256, 0, st>>>(static_cast<const GreenT<T>*>(p->green),
                                                   static_cast<double*>(out), total);
            break;
        }
        default:
            return SBP_ERR_INVALID_ARG;
    }
    return launch_status();
}

// Launch a fused xy plane kernel: one cluster of xy_cluster CTAs per z-plane.
template <typename K, typename... Args>
sbp_status launch_xy(const sbp_plan_s* p, K kernel, int ctas, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas, 1, 1);
    cfg.blockDim = dim3((unsigned)p->xy_threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p->xy_cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kernel, args...) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }
    return SBP_OK;
}

template <typename T>
sbp_status solve_fused_t(sbp_plan_s* p, const void* rho, void* phi, double t, cudaStream_t st,
                         const double* s_dev) {
    const bool f32 = !f64_of(p);
    XYArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pitch = p->pitch;
    a.green_ctas = p->xy_green_ctas;
    a.gf = make_green_fill(p, t, p->xy_green_ctas);
    a.gf.s_dev = s_dev;
    a.tile_sums = f32 ? p->tile_sums : nullptr;
    a.vk0 = nullptr;
    using FwdK = void (*)(const T*, cpx<T>*, const cpx<T>*, XYArgs);
    using InvK = void (*)(const cpx<T>*, T*, const cpx<T>*, XYArgs);
    cpx<T>* W = static_cast<cpx<T>*>(p->W);
    const cpx<T>* tw = static_cast<const cpx<T>*>(p->tw_x);
    sbp_status s = launch_xy(p, reinterpret_cast<FwdK>(p->xy_fwd), p->xy_green_ctas + p->nz * p->xy_cluster,
                             p->xy_smem_fwd, st, static_cast<const T*>(rho), W, tw, a);
    if (s != SBP_OK) return s;
    if ((s = launch_stage<T>(p, SBP_STAGE_Z_CONVOLVE, p->W, p->W, t, st, true)) != SBP_OK) return s;
    XYArgs b = a;
    b.green_ctas = 0;
    b.gf.tab = nullptr;
    b.tile_sums = nullptr;
    b.vk0 = f32 ? p->vk0 : nullptr;
    return launch_xy(p, reinterpret_cast<InvK>(p->xy_inv), p->nz * p->xy_cluster, p->xy_smem_inv, st,
                     static_cast<const cpx<T>*>(p->W), static_cast<T*>(phi), tw, b);
}

// Physical-frame solve (SBP_OPT_FRAME = 1): y pass with the forward mapping
// and the Green's table, forward x rows, z pass, inverse x rows, y pass with
// the mapping back.
template <typename T>
sbp_status solve_physical_t(sbp_plan_s* p, const void* rho, void* phi, double t, cudaStream_t st,
                            const double* s_dev) {
    const bool f32 = !f64_of(p);
    RArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = p->nx;
    a.ny = p->ny;
    a.pitch = p->nx;
    a.pairs = p->nx / 2;
    a.tiles = p->ry_tiles;
    a.green_blocks = p->ry_green_blocks;
    a.gf = make_green_fill(p, t, p->ry_green_blocks);
    a.gf.s_dev = s_dev;
    a.s = shear_s(p, t);
    a.s_dev = s_dev;
    a.lx_over_ly = p->Lx / p->Ly;
    a.vk0 = (f32 || p->method != 0) ? p->vk0 : nullptr;
    cpx<T>* W = static_cast<cpx<T>*>(p->W);
    const int rows = p->nz * (p->ny / 2 + 1);
    using RY = RemapKernels<T>;
    reinterpret_cast<decltype(RY::ry_fwd)>(p->ry_fwd)<<<p->ry_green_blocks + p->ry_tiles * p->nz, p->ry_threads,
                                                         p->ry_smem, st>>>(
        static_cast<const T*>(rho), W, static_cast<const cpx<T>*>(p->tw_y),
        (f32 || p->method != 0) ? p->tile_sums : nullptr, a);
    reinterpret_cast<decltype(RY::rows_fwd)>(p->rows_fwd)<<<p->rows_grid, p->rows_threads, p->rows_smem, st>>>(
        W, static_cast<const cpx<T>*>(p->tw_x), rows, p->nx);
    reinterpret_cast<ZKernel<T>>(p->z_fn)<<<p->zp.grid, p->zp.threads, p->zp.smem, st>>>(
        W, static_cast<const cpx<T>*>(p->tw_z),
        static_cast<const cpx<T>*>(p->pad == 4 ? p->tw_M4 : (p->z_padded ? p->tw_M : p->tw_2z)),
        static_cast<const T*>(p->kz2), make_zargs<T>(p, true));
    if (p->method != 0) {
        const sbp_status s = launch_sasha_k0(p, p->ry_tiles, st);
        if (s != SBP_OK) return s;
    }
    reinterpret_cast<decltype(RY::rows_inv)>(p->rows_inv)<<<p->rows_grid, p->rows_threads, p->rows_smem, st>>>(
        W, static_cast<const cpx<T>*>(p->tw_x), rows, p->nx);
    reinterpret_cast<decltype(RY::ry_inv)>(p->ry_inv)<<<p->ry_tiles * p->nz, p->ry_threads, p->ry_smem, st>>>(
        W, static_cast<T*>(phi), static_cast<const cpx<T>*>(p->tw_y), a);
    return launch_status();
}

// Frame of rho and phi (SBP_OPT_FRAME): 0 = periodic frame (the default
// passes), 1 = physical frame.  Returns false, leaving the plan unchanged,
// when the physical-frame kernels are not built for (nx, ny) or do not fit.
template <typename T>
bool configure_frame(sbp_plan_s* p, int frame) {
    const int old_zh = p->zh, old_zrows = p->zrows, old_zpitch = p->zpitch, old_frame = p->frame;
    auto restore = [&]() {
        p->frame = old_frame;
        p->zh = old_zh;
        p->zrows = old_zrows;
        p->zpitch = old_zpitch;
        configure_z<T>(p, p->z_variant);
    };
    if (frame == 0) {
        p->frame = 0;
        p->zh = p->h;
        p->zrows = p->ny;
        p->zpitch = p->pitch;
        if (!configure_z<T>(p, p->z_variant) && !configure_z<T>(p, 0)) {
            restore();
            return false;
        }
        return true;
    }
    const RemapKernels<T> k = remap_kernels_for<T>(p->nx, p->ny);
    if (!k.ry_fwd || !k.ry_inv || !k.rows_fwd || !k.rows_inv || !k.shear_cols) return false;
    const size_t cs = sizeof(cpx<T>);
    const int tfy = p->ny / k.ry_E, tfx = p->nx / k.rows_E;
    const int rows_C = kMaxThreads / tfx;
    const size_t ry_smem = (size_t)p->ny * cs + (size_t)xchg_slots<T>(p->ny, k.ry_C) * cs;
    const size_t rows_smem = (size_t)p->nx * cs + (size_t)rows_C * padded_row(p->nx) * cs;
    if (rows_C < 1 || k.ry_C * tfy > kMaxThreads || ry_smem > kSmemBudget || rows_smem > kSmemBudget) return false;
    const void* fns[5] = {reinterpret_cast<const void*>(k.ry_fwd), reinterpret_cast<const void*>(k.ry_inv),
                          reinterpret_cast<const void*>(k.rows_fwd), reinterpret_cast<const void*>(k.rows_inv),
                          reinterpret_cast<const void*>(k.shear_cols)};
    for (const void* f : fns) {
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    p->frame = 1;
    p->zh = p->nx;
    p->zrows = p->ny / 2 + 1;
    p->zpitch = p->nx;
    if (!configure_z<T>(p, p->z_variant) && !configure_z<T>(p, 0)) {
        restore();
        return false;
    }
    p->ry_fwd = reinterpret_cast<void*>(k.ry_fwd);
    p->ry_inv = reinterpret_cast<void*>(k.ry_inv);
    p->rows_fwd = reinterpret_cast<void*>(k.rows_fwd);
    p->rows_inv = reinterpret_cast<void*>(k.rows_inv);
    p->shear_cols = reinterpret_cast<void*>(k.shear_cols);
    p->ry_threads = k.ry_C * tfy;
    p->ry_tiles = (p->nx / 2 + k.ry_C - 1) / k.ry_C;
    p->ry_green_blocks = (p->nx * (p->ny / 2 + 1) + p->ry_threads - 1) / p->ry_threads;
    p->ry_smem = ry_smem;
    p->rows_threads = rows_C * tfx;
    p->rows_grid = (p->nz * (p->ny / 2 + 1) + rows_C - 1) / rows_C;
    p->rows_smem = rows_smem;
    return true;
}

// Schedule of the solves (SBP_OPT_SCHEDULE).  The three-sweep kernels serve
// FP32 plans in the periodic frame with the VGF method and 2·nz padding, for
// the box shapes they are built for, unless a five-pass variant was requested
// (SBP_OPT_XY_PASSES, SBP_OPT_Z_VARIANT, SBP_OPT_Y_TMA or SBP_OPT_XY_CHUNK set
// to a non-default value).  Returns false when schedule 2 is asked for and
// unavailable (the plan then keeps five passes).
bool configure_sweep(sbp_plan_s* p) {
    p->sweep = false;
    if (p->schedule == 1) return true;
    const bool eligible = !f64_of(p) && p->frame == 0 && p->method == 0 && p->pad == 2 &&
                          (p->schedule == 2 || (p->xy_req == 0 && p->z_req == 0 && p->ytma_req == 0 && p->chunk == 0));
    const SweepKernels k = eligible ? sweep_kernels_for(p->nx, p->ny, p->nz) : SweepKernels{};
    if (!k.fwd) return p->schedule != 2;
    if (k.smem_ac > kSmemBudget || k.smem_b > kSmemBudget) return p->schedule != 2;
    const void* fns[3] = {reinterpret_cast<const void*>(k.fwd), reinterpret_cast<const void*>(k.mid),
                          reinterpret_cast<const void*>(k.inv)};
    for (const void* f : fns) {
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) != cudaSuccess) {
            cudaGetLastError();
            return p->schedule != 2;
        }
    }
    // the half spectrum as a 4D tensor (z, j, a, k) of 8-byte elements for the
    // TMA path of passes A and C: box (za, 1, nx/2+1, ra)
    {
        auto enc = tensor_map_encoder();
        if (!enc) return p->schedule != 2;
        const cuuint64_t nz = (cuuint64_t)p->nz, rb = (cuuint64_t)k.rb, h = (cuuint64_t)p->h, ra = (cuuint64_t)k.ra;
        cuuint64_t dims[4] = {nz, rb, h, ra};
        cuuint64_t strides[3] = {nz * 8, rb * nz * 8, h * rb * nz * 8};
        cuuint32_t box[4] = {(cuuint32_t)k.za, 1, (cuuint32_t)p->h, (cuuint32_t)k.ra};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&p->sweep_tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, p->W, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return p->schedule != 2;
        if (cudaMemcpy(&p->sweep_box->tmap, &p->sweep_tmap, sizeof(CUtensorMap), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            cudaGetLastError();
            return p->schedule != 2;
        }
    }
    p->sk = k;
    p->sweep_green_blocks = k.green_mid ? 0 : (p->h * p->ny + k.nta - 1) / k.nta;
    p->sweep = true;
    return true;
}

SweepArgs sweep_args(const sbp_plan_s* p) {
    SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.boxes = p->sweep_box;
    a.twx = static_cast<const cpx<float>*>(p->tw_x);
    a.twy = static_cast<const cpx<float>*>(p->tw_y);
    a.twM = static_cast<const cpx<float>*>(p->tw_M);
    a.green_blocks = p->sweep_green_blocks;
    a.budget = p->spin_budget;
    a.withhold = p->withhold;
    return a;
}

// The three sweeps of one solve (see sbp_sweep.cuh), `nbox` boxes of the
// plan's shape at once when `a.boxes` holds their descriptors.
sbp_status launch_sweep(const sbp_plan_s* p, const SweepArgs& a, int nbox, cudaStream_t st) {
    const SweepKernels& k = p->sk;
    const int ablocks = (p->nz / k.za) * k.rb;
    k.fwd<<<dim3((unsigned)(a.green_blocks + ablocks), (unsigned)nbox), k.nta, k.smem_ac, st>>>(a);
    k.mid<<<dim3((unsigned)(k.ra * k.nga + 1), (unsigned)nbox), k.ntb, k.smem_b, st>>>(a);
    k.inv<<<dim3((unsigned)ablocks, (unsigned)nbox), k.nta, k.smem_ac, st>>>(a);
    return launch_status();
}

// One box: the middle and inverse sweeps are launched with programmatic
// stream serialisation, so that each launches during the previous sweep's
// last (partly empty) wave and its blocks wait on griddepcontrol for that
// sweep's results instead of for the launch.
sbp_status solve_sweep(const sbp_plan_s* p, const void* rho, void* phi, double t, cudaStream_t st,
                       const double* s_dev) {
    SweepArgs a = sweep_args(p);
    a.rho = static_cast<const float*>(rho);
    a.phi = static_cast<float*>(phi);
    a.s = shear_s(p, t);
    a.s_dev = s_dev;
    const SweepKernels& k = p->sk;
    const int ablocks = (p->nz / k.za) * k.rb;
    k.fwd<<<dim3((unsigned)(a.green_blocks + ablocks)), k.nta, k.smem_ac, st>>>(a);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(k.ra * k.nga + 1));
    cfg.blockDim = dim3((unsigned)k.ntb);
    cfg.dynamicSmemBytes = k.smem_b;
    if (cudaLaunchKernelEx(&cfg, k.mid, a) != cudaSuccess) return launch_status();
    cfg.gridDim = dim3((unsigned)ablocks);
    cfg.blockDim = dim3((unsigned)k.nta);
    cfg.dynamicSmemBytes = k.smem_ac;
    if (cudaLaunchKernelEx(&cfg, k.inv, a) != cudaSuccess) return launch_status();
    return launch_status();
}

// Kernels one solve launches (solve_t's dispatch; chunk < 0: the plan's own;
// five: the five-pass kernels even where the plan runs the sweeps).
int launches_per_solve(const sbp_plan_s* p, int chunk, bool five = false) {
    if (chunk < 0) chunk = p->chunk;
    if (p->sweep && !five && chunk <= 0) return 3;
    const int sasha = p->method != 0 ? 1 : 0;
    if (p->frame) return 5 + sasha;
    if (p->xy_fused) return 3;
    if (chunk > 0 && chunk < p->nz) return 1 + sasha + 4 * ((p->nz + chunk - 1) / chunk);
    return 5 + sasha;
}

// chunk: planes per x/y chunk (-1: the plan's own setting; -2: the five-pass
// kernels without chunks even where the plan runs the sweeps).
template <typename T>
sbp_status solve_t(sbp_plan_s* p, const void* rho, void* phi, double t, cudaStream_t st,
                   const double* s_dev = nullptr, int chunk = -1) {
    const bool five = (chunk == -2);
    if (five) chunk = 0;
    if (p->sweep && !five && chunk <= 0) return solve_sweep(p, rho, phi, t, st, s_dev);
    if (p->frame) return solve_physical_t<T>(p, rho, phi, t, st, s_dev);
    if (p->xy_fused) return solve_fused_t<T>(p, rho, phi, t, st, s_dev);
    if (chunk < 0) chunk = p->chunk;
    sbp_status s;
    if (chunk > 0 && chunk < p->nz) {
        // x and y passes chunk by chunk, so that a chunk's half spectrum is
        // still in L2 when the next pass reads it (SBP_OPT_XY_CHUNK)
        for (int z0 = 0; z0 < p->nz; z0 += chunk) {
            const int n = std::min(chunk, p->nz - z0);
            if ((s = launch_stage<T>(p, SBP_STAGE_X_FORWARD, rho, p->W, t, st, true, s_dev, z0, n)) != SBP_OK)
                return s;
            if ((s = launch_stage<T>(p, SBP_STAGE_Y_FORWARD, p->W, p->W, t, st, true, nullptr, z0, n)) != SBP_OK)
                return s;
        }
        if ((s = launch_stage<T>(p, SBP_STAGE_Z_CONVOLVE, p->W, p->W, t, st, true)) != SBP_OK) return s;
        for (int z0 = 0; z0 < p->nz; z0 += chunk) {
            const int n = std::min(chunk, p->nz - z0);
            if ((s = launch_stage<T>(p, SBP_STAGE_Y_INVERSE, p->W, p->W, t, st, true, nullptr, z0, n)) != SBP_OK)
                return s;
            if ((s = launch_stage<T>(p, SBP_STAGE_X_INVERSE, p->W, phi, t, st, true, nullptr, z0, n)) != SBP_OK)
                return s;
        }
        return SBP_OK;
    }
    if ((s = launch_stage<T>(p, SBP_STAGE_X_FORWARD, rho, p->W, t, st, true, s_dev)) != SBP_OK) return s;
    if ((s = launch_stage<T>(p, SBP_STAGE_Y_FORWARD, p->W, p->W, t, st, true)) != SBP_OK) return s;
    if ((s = launch_stage<T>(p, SBP_STAGE_Z_CONVOLVE, p->W, p->W, t, st, true)) != SBP_OK) return s;
    if ((s = launch_stage<T>(p, SBP_STAGE_Y_INVERSE, p->W, p->W, t, st, true)) != SBP_OK) return s;
    return launch_stage<T>(p, SBP_STAGE_X_INVERSE, p->W, phi, t, st, true);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

bool aligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

sbp_status check_io(const sbp_plan_s* p, const void* rho, const void* phi, double t) {
    if (!p || !rho || !phi || !std::isfinite(t)) return SBP_ERR_INVALID_ARG;
    if (!aligned16(rho) || !aligned16(phi)) return SBP_ERR_INVALID_ARG;
    const size_t bytes = (size_t)p->nx * p->ny * p->nz * p->rsize;
    const uintptr_t r0 = reinterpret_cast<uintptr_t>(rho), f0 = reinterpret_cast<uintptr_t>(phi);
    if (r0 != f0 && r0 < f0 + bytes && f0 < r0 + bytes) return SBP_ERR_INVALID_ARG;
    return SBP_OK;
}

// ---------------------------------------------------------------------------
// Batched executor.  Boxes whose plans run the three-sweep kernels are grouped
// by shape: one launch per sweep covers every box of the group through a
// device table of per-box descriptors (pointers, shear parameter, physical
// constants).  The other boxes keep their own pass kernels, spread over K
// parallel branches (largest first).  Everything is captured once into a
// CUDA graph, cached by the exact (plans, rho, phi) tuple; a call copies the
// boxes' shear parameters to the device and replays the graph.
//
// The first call of a tuple tunes: each group is timed as grouped sweeps and
// as per-box five-pass kernels and keeps the faster; then the branch count K
// (and chunked x/y passes for five-pass boxes) is timed on the whole graph.
// The candidates write into temporary outputs.  The choice is remembered per
// batch shape and GPU (and in the file named by SBP_TUNE_CACHE, if set).
// ---------------------------------------------------------------------------
struct SweepGroup {
    std::vector<int> boxes;  // box indices of the call, in table order
    int first = 0;           // first descriptor of the group in the table
    bool use = true;         // grouped sweeps (else per-box five-pass kernels)
};

struct BatchExec {
    std::vector<sbp_plan_s*> plans;
    std::vector<const void*> rho;
    std::vector<void*> phi;
    int device = 0;
    double* s_dev = nullptr;
    SweepBox* table = nullptr;           // device descriptors of the grouped boxes
    std::vector<SweepGroup> groups;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int branches = 0;
    int chunked = 0;  // the five-pass boxes' x/y passes run in chunks (auto_chunk)
    int launches = 0;  // kernels one replay launches
    float tuned_ms = 0.f;
};

std::mutex g_exec_mu;
std::vector<BatchExec*> g_execs;

void free_exec(BatchExec* e) {
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->s_dev) cudaFree(e->s_dev);
    if (e->table) cudaFree(e->table);
    delete e;
}

// Batched executors that reference plan p (their graphs hold its launch
// configuration): freed when the plan is destroyed or reconfigured.  The
// caller has synchronised the device.
void drop_executors(const sbp_plan_s* p) {
    std::lock_guard<std::mutex> lock(g_exec_mu);
    for (size_t i = 0; i < g_execs.size();) {
        BatchExec* e = g_execs[i];
        if (std::find(e->plans.begin(), e->plans.end(), p) != e->plans.end()) {
            free_exec(e);
            g_execs.erase(g_execs.begin() + i);
        } else {
            ++i;
        }
    }
}

// Planes per x/y chunk that keep a chunk's half spectrum near 8 MiB (0 when
// the whole box is already that small or the plan takes other passes).
int auto_chunk(const sbp_plan_s* p) {
    if (p->frame || p->xy_fused || p->sweep) return 0;
    const size_t plane = (size_t)p->ny * p->pitch * 2 * p->rsize;
    const int c = (int)std::max<size_t>(1, ((size_t)8 << 20) / plane);
    return c >= p->nz ? 0 : c;
}

// Groups of sweep boxes (same shape) and their descriptor table.  `phi` are
// the outputs the descriptors point to.
sbp_status build_groups(BatchExec* e, const std::vector<void*>& phi, cudaStream_t st) {
    const int n = (int)e->plans.size();
    if (e->groups.empty()) {
        for (int i = 0; i < n; ++i) {
            const sbp_plan_s* p = e->plans[i];
            if (!p->sweep) continue;
            SweepGroup* g = nullptr;
            for (SweepGroup& c : e->groups) {
                const sbp_plan_s* q = e->plans[c.boxes[0]];
                if (q->nx == p->nx && q->ny == p->ny && q->nz == p->nz) g = &c;
            }
            if (!g) {
                e->groups.emplace_back();
                g = &e->groups.back();
            }
            g->boxes.push_back(i);
        }
        int first = 0;
        for (SweepGroup& g : e->groups) {
            g.first = first;
            first += (int)g.boxes.size();
        }
        if (first > 0 && cudaMalloc(&e->table, sizeof(SweepBox) * first) != cudaSuccess) {
            cudaGetLastError();
            e->table = nullptr;
            return SBP_ERR_OUT_OF_MEMORY;
        }
    }
    std::vector<SweepBox> host;
    for (const SweepGroup& g : e->groups) {
        for (int i : g.boxes) {
            const sbp_plan_s* p = e->plans[i];
            SweepBox d;
            std::memset(&d, 0, sizeof(d));
            d.tmap = p->sweep_tmap;
            d.err = p->err;
            d.rho = static_cast<const float*>(e->rho[i]);
            d.phi = static_cast<float*>(phi[i]);
            d.S = reinterpret_cast<cpx<float>*>(p->W);
            d.green = reinterpret_cast<GreenT<float>*>(p->green);
            d.tile_sums = p->tile_sums;
            d.vk0 = p->vk0;
            d.c00 = p->c00;
            d.s_dev = e->s_dev + i;
            d.Lx = p->Lx;
            d.Ly = p->Ly;
            d.L = p->alpha * p->Lz;
            d.scale = 4.0 * M_PI * p->G / ((double)p->nx * p->ny * 2.0 * p->nz);
            d.kzc = (M_PI / p->Lz) * (M_PI / p->Lz);
            d.k0_coef = 4.0 * M_PI * p->G / ((double)p->nx * p->ny);
            host.push_back(d);
        }
    }
    if (!host.empty() && cudaMemcpyAsync(e->table, host.data(), sizeof(SweepBox) * host.size(),
                                         cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    return SBP_OK;
}

// Which boxes a capture covers: all (mask empty) or those with mask[i] != 0.
sbp_status capture_batch(BatchExec* e, int K, bool chunked, cudaGraph_t* graph_out, cudaGraphExec_t* exec_out,
                         int* launches_out, const std::vector<char>& mask = {}) {
    const int n = (int)e->plans.size();
    auto in = [&](int i) { return mask.empty() || mask[i] != 0; };
    std::vector<char> grouped(n, 0);
    int ngroups = 0;
    for (const SweepGroup& g : e->groups) {
        if (!g.use) continue;
        bool any = false;
        for (int i : g.boxes) {
            grouped[i] = 1;
            any = any || in(i);
        }
        if (any) ++ngroups;
    }
    const int nb = K + ngroups;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> br(nb, nullptr);
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join(nb, nullptr);
    sbp_status st = SBP_OK;
    int launches = 0;
    bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < nb; ++k)
        ok = cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming) == cudaSuccess;
    cudaGraph_t graph = nullptr;
    if (ok) ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        cudaEventRecord(fork, cap);
        for (int k = 0; k < nb; ++k) cudaStreamWaitEvent(br[k], fork, 0);
        // grouped sweeps: one branch per group, three launches each
        int gb = K;
        for (const SweepGroup& g : e->groups) {
            if (!g.use) continue;
            bool any = false;
            for (int i : g.boxes) any = any || in(i);
            if (!any) continue;
            const sbp_plan_s* p0 = e->plans[g.boxes[0]];
            SweepArgs a = sweep_args(p0);
            a.boxes = e->table + g.first;
            const sbp_status s = launch_sweep(p0, a, (int)g.boxes.size(), br[gb++]);
            launches += 3;
            if (s != SBP_OK && st == SBP_OK) st = s;
        }
        // the other boxes: largest first, each to the least loaded branch
        std::vector<int> order;
        for (int i = 0; i < n; ++i)
            if (!grouped[i] && in(i)) order.push_back(i);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const sbp_plan_s* pa = e->plans[a];
            const sbp_plan_s* pb = e->plans[b];
            return (size_t)pa->nx * pa->ny * pa->nz > (size_t)pb->nx * pb->ny * pb->nz;
        });
        std::vector<double> load(std::max(K, 1), 0.0);
        for (int i : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            sbp_plan_s* p = e->plans[i];
            load[k] += (double)p->nx * p->ny * p->nz;
            const int chunk = chunked ? auto_chunk(p) : 0;
            // five passes for a sweep plan here (its group chose them): chunk -1 keeps solve_t off the sweeps
            const int c = (p->sweep && chunk == 0) ? -2 : chunk;
            const sbp_status s = f64_of(p)
                                     ? solve_t<double>(p, e->rho[i], e->phi[i], 0.0, br[k], e->s_dev + i, c)
                                     : solve_t<float>(p, e->rho[i], e->phi[i], 0.0, br[k], e->s_dev + i, c);
            launches += launches_per_solve(p, c == -2 ? 0 : chunk, c == -2);
            if (s != SBP_OK && st == SBP_OK) st = s;
        }
        for (int k = 0; k < nb; ++k) {
            cudaEventRecord(join[k], br[k]);
            cudaStreamWaitEvent(cap, join[k], 0);
        }
        if (cudaStreamEndCapture(cap, &graph) != cudaSuccess) ok = false;
    }
    cudaGraphExec_t exec = nullptr;
    if (ok && st == SBP_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) ok = false;
    for (int k = 0; k < nb; ++k) {
        if (br[k]) cudaStreamDestroy(br[k]);
        if (join[k]) cudaEventDestroy(join[k]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    if (!ok || st != SBP_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return st != SBP_OK ? st : SBP_ERR_CUDA;
    }
    *graph_out = graph;
    *exec_out = exec;
    if (launches_out) *launches_out = launches;
    return SBP_OK;
}

// ---- remembered tuning choices (per batch shape and GPU)
struct TuneChoice {
    std::vector<char> group_use;
    int branches = 1, chunked = 0;
};
std::vector<std::pair<std::string, TuneChoice>> g_tune_memo;

std::string tune_key(const BatchExec* e) {
    std::string key;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, e->device) == cudaSuccess) {
        key = prop.name;
    } else {
        cudaGetLastError();
        key = "gpu";
    }
    for (char& c : key)
        if (c == ' ' || c == '\t' || c == '|') c = '_';
    for (const sbp_plan_s* p : e->plans) {
        char buf[96];
        std::snprintf(buf, sizeof(buf), "|%dx%dx%d:%d:%d%d%d%d", p->nx, p->ny, p->nz, (int)p->dtype, p->sweep ? 1 : 0,
                      p->frame, p->method, p->pad);
        key += buf;
    }
    return key;
}

bool tune_lookup(const std::string& key, TuneChoice* out) {
    for (const auto& kv : g_tune_memo)
        if (kv.first == key) {
            *out = kv.second;
            return true;
        }
    const char* path = std::getenv("SBP_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    std::vector<char> line(1 << 16);
    bool found = false;
    while (std::fgets(line.data(), (int)line.size(), f)) {
        std::string s(line.data());
        const size_t tab = s.find('\t');
        if (tab == std::string::npos || s.compare(0, tab, key) != 0 || tab != key.size()) continue;
        TuneChoice c;
        const char* v = s.c_str() + tab + 1;
        int used = 0;
        if (std::sscanf(v, "%d %d%n", &c.branches, &c.chunked, &used) < 2) continue;
        v += used;
        while (*v == ' ') ++v;
        for (; *v == '0' || *v == '1'; ++v) c.group_use.push_back(*v == '1');
        *out = c;
        found = true;
    }
    std::fclose(f);
    if (found) g_tune_memo.push_back({key, *out});
    return found;
}

void tune_store(const std::string& key, const TuneChoice& c) {
    g_tune_memo.push_back({key, c});
    const char* path = std::getenv("SBP_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::string use;
    for (char u : c.group_use) use += u ? '1' : '0';
    std::fprintf(f, "%s\t%d %d %s\n", key.c_str(), c.branches, c.chunked, use.c_str());
    std::fclose(f);
}

// Time one graph: mean ms of 3 replays after one warm-up replay.
sbp_status time_graph(cudaGraphExec_t x, cudaStream_t st, cudaEvent_t a, cudaEvent_t b, float* ms) {
    cudaGraphLaunch(x, st);
    cudaEventRecord(a, st);
    for (int r = 0; r < 3; ++r) cudaGraphLaunch(x, st);
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }
    *ms /= 3.f;
    return SBP_OK;
}

// Build the executor's graph, choosing the schedule of each group, K and the
// chunking by timing when neither forced nor remembered.  The caller holds
// g_exec_mu and has copied the shear parameters to e->s_dev.
sbp_status tune_batch(BatchExec* e, cudaStream_t st) {
    const int n = (int)e->plans.size();
    sbp_status s = build_groups(e, e->phi, st);
    if (s != SBP_OK) return s;
    auto finish = [&](const TuneChoice& c) -> sbp_status {
        for (size_t g = 0; g < e->groups.size(); ++g)
            e->groups[g].use = g < c.group_use.size() ? c.group_use[g] != 0 : true;
        e->branches = c.branches;
        e->chunked = c.chunked;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        int launches = 0;
        const sbp_status r = capture_batch(e, e->branches, e->chunked != 0, &g, &x, &launches);
        if (r != SBP_OK) return r;
        e->graph = g;
        e->exec = x;
        e->launches = launches;
        return SBP_OK;
    };
    // the same plans with other buffers (double buffering) take the existing choice
    for (const BatchExec* c : g_execs) {
        if (c == e || !c->exec || c->plans != e->plans) continue;
        TuneChoice ch;
        for (const SweepGroup& g : c->groups) ch.group_use.push_back(g.use);
        ch.branches = c->branches;
        ch.chunked = c->chunked;
        e->tuned_ms = c->tuned_ms;
        return finish(ch);
    }
    const std::string key = tune_key(e);
    TuneChoice memo;
    const char* env_k = std::getenv("SBP_BATCH_BRANCHES");
    const char* env_c = std::getenv("SBP_BATCH_CHUNK");
    const char* env_s = std::getenv("SBP_BATCH_SCHEDULE");  // 1: five passes everywhere, 2: grouped sweeps
    if (!env_k && !env_c && !env_s && tune_lookup(key, &memo) && memo.group_use.size() == e->groups.size())
        return finish(memo);

    std::vector<int> cands;
    if (env_k) {
        const int k = std::atoi(env_k);
        if (k >= 1) cands.push_back(std::min(k, std::max(1, n)));
    }
    if (cands.empty())
        for (int k : {1, 2, 4, 8, 16, 32})
            if (k <= std::max(1, n)) cands.push_back(k);
    std::vector<int> chunk_modes = {0};
    if (env_c) {
        chunk_modes = {std::atoi(env_c) != 0 ? 1 : 0};
    } else {
        for (const sbp_plan_s* p : e->plans)
            if (auto_chunk(p) > 0) {
                chunk_modes.push_back(1);
                break;
            }
    }
    const bool sched_free = !env_s && !e->groups.empty();
    if (env_s)
        for (SweepGroup& g : e->groups) g.use = std::atoi(env_s) != 1;
    const size_t trials = (sched_free ? 2 * e->groups.size() : 0) + cands.size() * chunk_modes.size();
    if (trials <= 1) {
        TuneChoice c;
        for (const SweepGroup& g : e->groups) c.group_use.push_back(g.use);
        c.branches = cands[0];
        c.chunked = chunk_modes[0];
        return finish(c);
    }

    // The candidate graphs are replayed several times to time them.  They
    // write into temporary outputs, never into the caller's phi: an in-place
    // box (phi == rho) would otherwise be solved again on every replay, and
    // the caller's rho stays untouched.  The chosen configuration is captured
    // once more on the caller's buffers and replayed once by the caller.
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaEventDestroy(a);
        return SBP_ERR_CUDA;
    }
    std::vector<void*> caller_phi = e->phi;
    void* scratch = nullptr;
    {
        std::vector<size_t> offs(n);
        size_t total = 0;
        for (int i = 0; i < n; ++i) {
            const sbp_plan_s* p = e->plans[i];
            offs[i] = total;
            total = align_up(total + (size_t)p->nx * p->ny * p->nz * p->rsize, 256);
        }
        if (cudaMalloc(&scratch, std::max<size_t>(total, 256)) != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return SBP_ERR_OUT_OF_MEMORY;
        }
        for (int i = 0; i < n; ++i) e->phi[i] = static_cast<unsigned char*>(scratch) + offs[i];
    }
    s = build_groups(e, e->phi, st);
    auto run_trial = [&](int K, bool chunked, const std::vector<char>& mask, float* ms) -> sbp_status {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        sbp_status r = capture_batch(e, K, chunked, &g, &x, nullptr, mask);
        if (r != SBP_OK) return r;
        r = time_graph(x, st, a, b, ms);
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        return r;
    };
    // 1. each group alone: grouped sweeps against per-box five-pass kernels
    if (s == SBP_OK && sched_free) {
        for (SweepGroup& g : e->groups) {
            std::vector<char> mask(n, 0);
            for (int i : g.boxes) mask[i] = 1;
            float t_sweep = 0.f, t_five = 0.f;
            g.use = true;
            if ((s = run_trial(1, false, mask, &t_sweep)) != SBP_OK) break;
            g.use = false;
            const int K = (int)std::min<size_t>(16, g.boxes.size());
            if ((s = run_trial(K, false, mask, &t_five)) != SBP_OK) break;
            // grouped sweeps take 3 launches for the whole group: keep them unless clearly slower
            g.use = t_sweep <= 1.02f * t_five;
            if (std::getenv("SBP_TUNE_LOG")) {
                const sbp_plan_s* p0 = e->plans[g.boxes[0]];
                std::fprintf(stderr, "[sbp tune] %zu x %dx%dx%d: grouped sweeps %.3f ms, five passes %.3f ms -> %s\n",
                             g.boxes.size(), p0->nx, p0->ny, p0->nz, t_sweep, t_five, g.use ? "sweeps" : "five");
            }
        }
    }
    // 2. the whole graph: branch count and chunking
    float best = 0.f;
    TuneChoice choice;
    bool have = false;
    for (int K : cands) {
        for (int c : chunk_modes) {
            if (s != SBP_OK) break;
            float ms = 0.f;
            if ((s = run_trial(K, c != 0, {}, &ms)) != SBP_OK) break;
            if (std::getenv("SBP_TUNE_LOG"))
                std::fprintf(stderr, "[sbp tune] whole batch, K = %d, chunked = %d: %.3f ms\n", K, c, ms);
            if (!have || ms < best) {
                have = true;
                best = ms;
                choice.branches = K;
                choice.chunked = c;
            }
        }
    }
    // 3. groups interact in the whole graph (their kernels share the SMs): flip
    //    each group's schedule in turn and keep the flip when the batch is faster
    if (s == SBP_OK && sched_free && have) {
        for (SweepGroup& g : e->groups) {
            g.use = !g.use;
            float ms = 0.f;
            if ((s = run_trial(choice.branches, choice.chunked != 0, {}, &ms)) != SBP_OK) break;
            const bool keep = ms < 0.99f * best;
            if (std::getenv("SBP_TUNE_LOG")) {
                const sbp_plan_s* p0 = e->plans[g.boxes[0]];
                std::fprintf(stderr, "[sbp tune] whole batch with %dx%dx%d on %s: %.3f ms%s\n", p0->nx, p0->ny, p0->nz,
                             g.use ? "sweeps" : "five passes", ms, keep ? " (kept)" : "");
            }
            if (keep)
                best = ms;
            else
                g.use = !g.use;
        }
    }
    for (const SweepGroup& g : e->groups) choice.group_use.push_back(g.use);
    if (std::getenv("SBP_TUNE_LOG")) {
        std::fprintf(stderr, "[sbp tune] choice: K = %d, chunked = %d, groups:", choice.branches, choice.chunked);
        for (size_t g = 0; g < e->groups.size(); ++g) {
            const sbp_plan_s* p0 = e->plans[e->groups[g].boxes[0]];
            std::fprintf(stderr, " %dx%dx%d=%s", p0->nx, p0->ny, p0->nz, e->groups[g].use ? "sweeps" : "five");
        }
        std::fprintf(stderr, " (%.3f ms)\n", best);
    }
    e->phi = caller_phi;
    cudaStreamSynchronize(st);
    cudaFree(scratch);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != SBP_OK) return s;
    if ((s = build_groups(e, e->phi, st)) != SBP_OK) return s;
    e->tuned_ms = best;
    if (!env_k && !env_c && !env_s) tune_store(key, choice);
    return finish(choice);
}

template <typename T>
sbp_status set_method(sbp_plan_s* p, int method) {
    const int old = p->method;
    p->method = method;
    sbp_status st = refresh_vertical_tables<T>(p);
    // FP64 SASHA needs plane sums, which only the separate x passes make
    if (st == SBP_OK && f64_of(p) && method != 0 && p->xy_fused && !configure_xy<T>(p, 1))
        st = SBP_ERR_UNSUPPORTED_SIZE;
    if (st != SBP_OK) {
        p->method = old;
        refresh_vertical_tables<T>(p);
    }
    return st;
}

template <typename T>
sbp_status set_truncation(sbp_plan_s* p, double alpha) {
    const double old_alpha = p->alpha;
    const int old_pad = p->pad;
    p->alpha = alpha;
    p->pad = (alpha == 1.0) ? 2 : 4;
    sbp_status st = refresh_vertical_tables<T>(p);
    if (st == SBP_OK && !configure_z<T>(p, 0)) st = SBP_ERR_UNSUPPORTED_SIZE;
    if (st != SBP_OK) {
        p->alpha = old_alpha;
        p->pad = old_pad;
        refresh_vertical_tables<T>(p);
        configure_z<T>(p, p->z_variant);
    }
    return st;
}

template <typename T>
sbp_status force_t(sbp_plan_s* p, const T* phi, T* force, double t, cudaStream_t st) {
    const T* side = nullptr;
    if (p->frame == 1) {
        using RY = RemapKernels<T>;
        const double u = shear_s(p, t) * p->Lx / p->Ly;  // Δy0 / L_y
        const int tf = p->ny / plan_E(p->ny, f64_of(p));
        const int cp = shear_cols_planes(tf);
        const size_t smem = (size_t)p->ny * sizeof(cpx<T>) + (size_t)xchg_slots<T>(p->ny, cp) * sizeof(cpx<T>);
        reinterpret_cast<decltype(RY::shear_cols)>(p->shear_cols)<<<(p->nz + cp - 1) / cp, cp * tf, smem, st>>>(
            phi, static_cast<T*>(p->side), static_cast<const cpx<T>*>(p->tw_y), p->nx, p->nz, u);
        side = static_cast<const T*>(p->side);
    }
    constexpr int ZC = 16;
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((p->nx + 31) / 32), (unsigned)((p->ny + 7) / 8), (unsigned)((p->nz + ZC - 1) / ZC));
    const double dx = p->Lx / p->nx, dy = p->Ly / p->ny, dz = p->Lz / p->nz;
    k_force<T, ZC><<<grid, block, 0, st>>>(phi, force, side, p->nx, p->ny, p->nz, (T)(0.5 / dx), (T)(0.5 / dy),
                                           (T)(1.0 / dz));
    return launch_status();
}

}  // namespace

extern "C" {

sbp_status sbp_plan_create(sbp_plan* out, int nx, int ny, int nz, double Lx, double Ly, double Lz, double q,
                           double Omega, double G, sbp_dtype dtype) {
    if (!out) return SBP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!finite_pos(Lx) || !finite_pos(Ly) || !finite_pos(Lz) || !finite_pos(Omega) || !finite_pos(G) ||
        !std::isfinite(q))
        return SBP_ERR_INVALID_ARG;
    if (dtype != SBP_F64 && dtype != SBP_F32) {
        if (dtype == SBP_F32_SPLIT_F16 || dtype == SBP_F32_SPLIT_BF16) return SBP_ERR_UNSUPPORTED_DTYPE;
        return SBP_ERR_INVALID_ARG;
    }
    if (nx < 4 || ny < 4 || nz < 2 || (nx & 1) || (ny & 1)) return SBP_ERR_UNSUPPORTED_SIZE;
    if (!supported_len(nx) || !supported_len(ny) || !supported_len(nz)) return SBP_ERR_UNSUPPORTED_SIZE;

    sbp_plan_s* p = new (std::nothrow) sbp_plan_s();
    if (!p) return SBP_ERR_OUT_OF_MEMORY;
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->Lx = Lx;
    p->Ly = Ly;
    p->Lz = Lz;
    p->q = q;
    p->Omega = Omega;
    p->G = G;
    p->dtype = dtype;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return SBP_ERR_CUDA;
    }
    const bool f64 = (dtype == SBP_F64);
    p->rsize = f64 ? sizeof(double) : sizeof(float);
    p->h = nx / 2 + 1;
    p->pitch = (p->h + 1) / 2 * 2;
    p->zh = p->h;
    p->zrows = ny;
    p->zpitch = p->pitch;
    if (!build_fft_plan(nx, plan_E(nx, f64), p->px) || !build_fft_plan(ny, plan_E(ny, f64), p->py)) {
        delete p;
        return SBP_ERR_UNSUPPORTED_SIZE;
    }
    const bool ok = f64 ? configure<double>(p) : configure<float>(p);
    if (!ok) {
        cudaGetLastError();
        delete p;
        return SBP_ERR_UNSUPPORTED_SIZE;
    }
    // the physical-frame passes store the y half spectrum, [nz][ny/2+1][nx]
    p->W_bytes = std::max((size_t)nz * ny * p->pitch, (size_t)nz * (ny / 2 + 1) * nx) * 2 * p->rsize;
    if (cudaMalloc(&p->W, p->W_bytes) != cudaSuccess) {
        cudaGetLastError();
        p->W = nullptr;
        free_plan(p);
        return SBP_ERR_OUT_OF_MEMORY;
    }
    const sbp_status s = f64 ? upload_tables<double>(p) : upload_tables<float>(p);
    if (s != SBP_OK) {
        free_plan(p);
        return s;
    }
    if (f64) {
        configure_ytma<double>(p, true);
    } else {
        configure_ytma<float>(p, true);
    }
    configure_sweep(p);
    *out = p;
    return SBP_OK;
}

sbp_status sbp_solve(sbp_plan p, const void* rho, void* phi, double t, void* stream) {
    const sbp_status v = check_io(p, rho, phi, t);
    if (v != SBP_OK) return v;
    DeviceGuard g(p->device);
    if (!g.ok) return SBP_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return f64_of(p) ? solve_t<double>(p, rho, phi, t, st) : solve_t<float>(p, rho, phi, t, st);
}

sbp_status sbp_solve_batched(int nbox, const sbp_plan* plans, const void* const* rho, void* const* phi,
                             const double* t, void* stream) {
    if (nbox < 0 || (nbox > 0 && (!plans || !rho || !phi || !t))) return SBP_ERR_INVALID_ARG;
    for (int i = 0; i < nbox; ++i) {
        if (!plans[i]) return SBP_ERR_INVALID_ARG;
        if (plans[i]->dtype != plans[0]->dtype) return SBP_ERR_NOT_SAME_DTYPE;
        if (plans[i]->device != plans[0]->device) return SBP_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return SBP_ERR_INVALID_ARG;
        const sbp_status v = check_io(plans[i], rho[i], phi[i], t[i]);
        if (v != SBP_OK) return v;
    }
    // Boxes run concurrently: no box may write memory that another box reads
    // or writes (two boxes reading the same rho is fine).
    {
        struct Span {
            uintptr_t lo, hi;
            int box;
            bool write;
        };
        std::vector<Span> spans;
        spans.reserve(2 * (size_t)nbox);
        for (int i = 0; i < nbox; ++i) {
            const size_t bytes = (size_t)plans[i]->nx * plans[i]->ny * plans[i]->nz * plans[i]->rsize;
            const uintptr_t r0 = reinterpret_cast<uintptr_t>(rho[i]), f0 = reinterpret_cast<uintptr_t>(phi[i]);
            spans.push_back({r0, r0 + bytes, i, false});
            spans.push_back({f0, f0 + bytes, i, true});
        }
        std::sort(spans.begin(), spans.end(), [](const Span& x, const Span& y) { return x.lo < y.lo; });
        for (size_t u = 0; u < spans.size(); ++u)
            for (size_t w = u + 1; w < spans.size() && spans[w].lo < spans[u].hi; ++w)
                if (spans[u].box != spans[w].box && (spans[u].write || spans[w].write)) return SBP_ERR_INVALID_ARG;
    }
    if (nbox == 0) return SBP_OK;
    DeviceGuard g(plans[0]->device);
    if (!g.ok) return SBP_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(g_exec_mu);
    BatchExec* e = nullptr;
    for (BatchExec* c : g_execs) {
        if ((int)c->plans.size() != nbox) continue;
        bool same = true;
        for (int i = 0; same && i < nbox; ++i)
            same = c->plans[i] == plans[i] && c->rho[i] == rho[i] && c->phi[i] == phi[i];
        if (same) {
            e = c;
            break;
        }
    }
    std::vector<double> s_host(nbox);
    for (int i = 0; i < nbox; ++i) s_host[i] = shear_s(plans[i], t[i]);
    const bool fresh = (e == nullptr);
    if (fresh) {
        e = new (std::nothrow) BatchExec();
        if (!e) return SBP_ERR_OUT_OF_MEMORY;
        e->plans.assign(plans, plans + nbox);
        e->rho.assign(rho, rho + nbox);
        e->phi.assign(phi, phi + nbox);
        e->device = plans[0]->device;
        if (cudaMalloc(&e->s_dev, sizeof(double) * nbox) != cudaSuccess) {
            cudaGetLastError();
            e->s_dev = nullptr;
            free_exec(e);
            return SBP_ERR_OUT_OF_MEMORY;
        }
    }
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    if (cudaMemcpyAsync(e->s_dev, s_host.data(), sizeof(double) * nbox, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        if (fresh) free_exec(e);
        return SBP_ERR_CUDA;
    }
    if (fresh) {
        const sbp_status s = tune_batch(e, st);
        if (s != SBP_OK) {
            free_exec(e);
            return s;
        }
        g_execs.push_back(e);
    }
    if (cudaGraphLaunch(e->exec, st) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }
    return SBP_OK;
}

void sbp_plan_destroy(sbp_plan p) {
    if (!p) return;
    {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        cudaGetLastError();
        drop_executors(p);
        free_plan(p);
    }
}

sbp_status sbp_fill_ghosts(sbp_plan p, const void* phi, void* out, int ng, void* stream) {
    if (!p || !phi || !out || ng < 1 || ng > 16) return SBP_ERR_INVALID_ARG;
    if (!aligned16(phi) || !aligned16(out)) return SBP_ERR_INVALID_ARG;
    const size_t plane = (size_t)p->nx * p->ny;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(phi), b0 = reinterpret_cast<uintptr_t>(out);
    const size_t abytes = plane * p->nz * p->rsize, bbytes = plane * (p->nz + 2 * ng) * p->rsize;
    if (a0 < b0 + bbytes && b0 < a0 + abytes) return SBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return SBP_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const dim3 grid((unsigned)((plane + 255) / 256), (unsigned)(p->nz + 2 * ng));
    if (f64_of(p))
        k_fill_ghosts<double><<<grid, 256, 0, st>>>(static_cast<const double*>(phi), static_cast<double*>(out),
                                                    (int)plane, p->nz, ng);
    else
        k_fill_ghosts<float><<<grid, 256, 0, st>>>(static_cast<const float*>(phi), static_cast<float*>(out),
                                                   (int)plane, p->nz, ng);
    return launch_status();
}

sbp_status sbp_force(sbp_plan p, const void* phi, void* force, double t, void* stream) {
    if (!p || !phi || !force || !std::isfinite(t)) return SBP_ERR_INVALID_ARG;
    if (!aligned16(phi) || !aligned16(force)) return SBP_ERR_INVALID_ARG;
    const size_t n = (size_t)p->nx * p->ny * p->nz * p->rsize;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(phi), b0 = reinterpret_cast<uintptr_t>(force);
    if (a0 < b0 + 3 * n && b0 < a0 + n) return SBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return SBP_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return f64_of(p) ? force_t<double>(p, static_cast<const double*>(phi), static_cast<double*>(force), t, st)
                     : force_t<float>(p, static_cast<const float*>(phi), static_cast<float*>(force), t, st);
}

const char* sbp_last_cuda_error(void) {
    return g_last_cuda == cudaSuccess ? "no CUDA error recorded" : cudaGetErrorString(g_last_cuda);
}

const char* sbp_status_string(sbp_status s) {
    switch (s) {
        case SBP_OK: return "ok";
        case SBP_ERR_INVALID_ARG: return "invalid argument";
        case SBP_ERR_UNSUPPORTED_SIZE: return "unsupported size";
        case SBP_ERR_OUT_OF_MEMORY: return "out of device memory";
        case SBP_ERR_CUDA: return "CUDA error";
        case SBP_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        case SBP_ERR_NOT_SAME_DTYPE: return "batched plans differ in dtype";
        case SBP_ERR_UNSUPPORTED_DTYPE: return "dtype not built in this library";
        case SBP_ERR_SCRATCH_LIMIT: return "box exceeds the 40 MiB fixed workspace of sbp_solve_noalloc";
    }
    return "unknown status";
}

static sbp_status set_option_impl(sbp_plan p, int option, double value);

sbp_status sbp_plan_set_option(sbp_plan p, int option, double value) {
    if (!p || !std::isfinite(value)) return SBP_ERR_INVALID_ARG;
    if (option == SBP_OPT_SCHEDULE) {
        const int v = (int)value;
        if ((double)v != value || v < 0 || v > 2) return SBP_ERR_INVALID_ARG;
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        cudaDeviceSynchronize();
        cudaGetLastError();
        drop_executors(p);
        const int old = p->schedule;
        p->schedule = v;
        if (!configure_sweep(p)) {
            p->schedule = old;
            configure_sweep(p);
            return SBP_ERR_UNSUPPORTED_SIZE;
        }
        return SBP_OK;
    }
    const sbp_status st = set_option_impl(p, option, value);
    if (st == SBP_OK) {
        // the requested five-pass variants, and the frame, method and
        // truncation, decide whether the solves keep the three-sweep kernels
        if (option == SBP_OPT_XY_PASSES) p->xy_req = (int)value;
        if (option == SBP_OPT_Z_VARIANT) p->z_req = (int)value;
        if (option == SBP_OPT_Y_TMA) p->ytma_req = (int)value;
        if (option == SBP_OPT_XY_PASSES || option == SBP_OPT_Z_VARIANT || option == SBP_OPT_Y_TMA ||
            option == SBP_OPT_XY_CHUNK || option == SBP_OPT_FRAME || option == SBP_OPT_METHOD ||
            option == SBP_OPT_TRUNCATION) {
            DeviceGuard g(p->device);
            if (!g.ok) return SBP_ERR_CUDA;
            if (!configure_sweep(p)) {  // a forced three-sweep schedule no longer applies
                p->schedule = 0;
                configure_sweep(p);
            }
        }
    }
    return st;
}

static sbp_status set_option_impl(sbp_plan p, int option, double value) {
    if (option == SBP_OPT_Y_TMA || option == SBP_OPT_XY_PASSES || option == SBP_OPT_Z_VARIANT ||
        option == SBP_OPT_TRUNCATION || option == SBP_OPT_FRAME || option == SBP_OPT_METHOD ||
        option == SBP_OPT_XY_CHUNK) {
        // captured batch graphs hold the old kernels and arguments
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        cudaDeviceSynchronize();
        cudaGetLastError();
        drop_executors(p);
    }
    if (option == SBP_OPT_FRAME) {
        if (value != 0.0 && value != 1.0) return SBP_ERR_INVALID_ARG;
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        const bool ok = f64_of(p) ? configure_frame<double>(p, (int)value) : configure_frame<float>(p, (int)value);
        return ok ? SBP_OK : SBP_ERR_UNSUPPORTED_SIZE;
    }
    if (option == SBP_OPT_XY_CHUNK) {
        const int v = (int)value;
        if ((double)v != value || v < 0) return SBP_ERR_INVALID_ARG;
        p->chunk = v;
        return SBP_OK;
    }
    if (option == SBP_OPT_METHOD) {
        const int v = (int)value;
        if ((double)v != value || v < 0 || v > 2) return SBP_ERR_INVALID_ARG;
        if (v != 0 && p->pad != 2) return SBP_ERR_UNSUPPORTED_SIZE;  // SASHA pads to 2 nz
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        return f64_of(p) ? set_method<double>(p, v) : set_method<float>(p, v);
    }
    if (option == SBP_OPT_TRUNCATION) {
        if (!(value == 1.0 || (value > 1.0 && value <= 3.0))) return SBP_ERR_INVALID_ARG;
        if (value != 1.0 && p->method != 0) return SBP_ERR_UNSUPPORTED_SIZE;  // SASHA pads to 2 nz
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        return f64_of(p) ? set_truncation<double>(p, value) : set_truncation<float>(p, value);
    }
    if (option == SBP_OPT_Y_TMA) {
        if (value != 0.0 && value != 1.0) return SBP_ERR_INVALID_ARG;
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        const bool want = (value == 0.0);
        const bool ok = f64_of(p) ? configure_ytma<double>(p, want) : configure_ytma<float>(p, want);
        return ok ? SBP_OK : SBP_ERR_UNSUPPORTED_SIZE;
    }
    if (option == SBP_OPT_SPIN_BUDGET) {
        if (!(value >= 1000.0 && value <= 1e12)) return SBP_ERR_INVALID_ARG;
        p->spin_budget = (long long)value;
        return SBP_OK;
    }
    if (option == SBP_OPT_DEBUG_WITHHOLD_COPY) {
        if (value != 0.0 && value != 1.0) return SBP_ERR_INVALID_ARG;
        p->withhold = (int)value;
        return SBP_OK;
    }
    if (option == SBP_OPT_XY_PASSES) {
        const int v = (int)value;
        if ((double)v != value || v < 0 || v > 3) return SBP_ERR_INVALID_ARG;
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        const bool ok = f64_of(p) ? configure_xy<double>(p, v) : configure_xy<float>(p, v);
        return ok ? SBP_OK : SBP_ERR_UNSUPPORTED_SIZE;
    }
    if (option == SBP_OPT_Z_VARIANT) {
        const int v = (int)value;
        if ((double)v != value || v < 0 || v > 4) return SBP_ERR_INVALID_ARG;
        if (p->pad == 4 && v != 0) return SBP_ERR_UNSUPPORTED_SIZE;  // one kernel for fourfold padding
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        const bool ok = f64_of(p) ? configure_z<double>(p, v) : configure_z<float>(p, v);
        return ok ? SBP_OK : SBP_ERR_UNSUPPORTED_SIZE;
    }
    return SBP_ERR_INVALID_ARG;
}

sbp_status sbp_plan_sync_status(sbp_plan p, void* stream) {
    if (!p) return SBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return SBP_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int flag = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpy(&flag, p->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }
    if (flag != 0) {
        const int zero = 0;
        if (cudaMemcpy(p->err, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return SBP_ERR_CUDA;
        }
        return SBP_ERR_DEVICE_TIMEOUT;
    }
    return SBP_OK;
}

sbp_status sbp_plan_info(sbp_plan p, int* nx, int* ny, int* nz, int* dtype, int* spectrum_pitch,
                         size_t* workspace_bytes) {
    if (!p) return SBP_ERR_INVALID_ARG;
    if (nx) *nx = p->nx;
    if (ny) *ny = p->ny;
    if (nz) *nz = p->nz;
    if (dtype) *dtype = (int)p->dtype;
    if (spectrum_pitch) *spectrum_pitch = p->pitch;
    if (workspace_bytes) *workspace_bytes = p->W_bytes + p->tables_bytes;
    return SBP_OK;
}

sbp_status sbp_run_stage(sbp_plan p, int stage, const void* in, void* out, double t, void* stream) {
    if (!p || !std::isfinite(t)) return SBP_ERR_INVALID_ARG;
    if (stage >= SBP_STAGE_SWEEP_FORWARD && stage <= SBP_STAGE_SWEEP_INVERSE) {
        if (!p->sweep) return SBP_ERR_INVALID_ARG;
        if (stage == SBP_STAGE_SWEEP_FORWARD && (!in || !aligned16(in))) return SBP_ERR_INVALID_ARG;
        if (stage == SBP_STAGE_SWEEP_INVERSE && (!out || !aligned16(out))) return SBP_ERR_INVALID_ARG;
        DeviceGuard g(p->device);
        if (!g.ok) return SBP_ERR_CUDA;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        SweepArgs a = sweep_args(p);
        a.rho = static_cast<const float*>(in != nullptr ? in : p->W);  // non-null: the single-box form
        a.phi = static_cast<float*>(out);
        a.s = shear_s(p, t);
        const SweepKernels& k = p->sk;
        const int ablocks = (p->nz / k.za) * k.rb;
        if (stage == SBP_STAGE_SWEEP_FORWARD)
            k.fwd<<<dim3((unsigned)(a.green_blocks + ablocks)), k.nta, k.smem_ac, st>>>(a);
        else if (stage == SBP_STAGE_SWEEP_MIDDLE)
            k.mid<<<dim3((unsigned)(k.ra * k.nga + 1)), k.ntb, k.smem_b, st>>>(a);
        else
            k.inv<<<dim3((unsigned)ablocks), k.nta, k.smem_ac, st>>>(a);
        return launch_status();
    }
    if (!out) return SBP_ERR_INVALID_ARG;
    if (p->frame != 0 || p->method != 0) return SBP_ERR_INVALID_ARG;  // the stages are the VGF periodic-frame passes
    if (stage < SBP_STAGE_X_FORWARD || stage > SBP_STAGE_GREEN_FILL) return SBP_ERR_INVALID_ARG;
    if (stage != SBP_STAGE_GREEN_TABLE && stage != SBP_STAGE_GREEN_FILL && !in) return SBP_ERR_INVALID_ARG;
    if ((stage == SBP_STAGE_Y_FORWARD || stage == SBP_STAGE_Z_CONVOLVE || stage == SBP_STAGE_Y_INVERSE) &&
        in != out)
        return SBP_ERR_INVALID_ARG;
    if ((in && !aligned16(in)) || !aligned16(out)) return SBP_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return SBP_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return f64_of(p) ? launch_stage<double>(p, stage, in, out, t, st, false)
                     : launch_stage<float>(p, stage, in, out, t, st, false);
}

sbp_status sbp_batch_info(int nbox, const sbp_plan* plans, const void* const* rho, void* const* phi,
                          int* launches, int* grouped_boxes) {
    if (nbox <= 0 || !plans || !rho || !phi) return SBP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_exec_mu);
    for (const BatchExec* c : g_execs) {
        if ((int)c->plans.size() != nbox) continue;
        bool same = true;
        for (int i = 0; same && i < nbox; ++i)
            same = c->plans[i] == plans[i] && c->rho[i] == rho[i] && c->phi[i] == phi[i];
        if (!same) continue;
        if (launches) *launches = c->launches;
        if (grouped_boxes) {
            int g = 0;
            for (const SweepGroup& s : c->groups)
                if (s.use) g += (int)s.boxes.size();
            *grouped_boxes = g;
        }
        return SBP_OK;
    }
    return SBP_ERR_INVALID_ARG;
}

sbp_status sbp_batch_run_stage(int nbox, const sbp_plan* plans, const void* const* rho, void* const* phi, int nx,
                               int ny, int nz, int stage, void* stream) {
    if (nbox <= 0 || !plans || !rho || !phi) return SBP_ERR_INVALID_ARG;
    if (stage < SBP_STAGE_SWEEP_FORWARD || stage > SBP_STAGE_SWEEP_INVERSE) return SBP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_exec_mu);
    for (const BatchExec* c : g_execs) {
        if ((int)c->plans.size() != nbox) continue;
        bool same = true;
        for (int i = 0; same && i < nbox; ++i)
            same = c->plans[i] == plans[i] && c->rho[i] == rho[i] && c->phi[i] == phi[i];
        if (!same) continue;
        for (const SweepGroup& g : c->groups) {
            const sbp_plan_s* p0 = c->plans[g.boxes[0]];
            if (!g.use || p0->nx != nx || p0->ny != ny || p0->nz != nz) continue;
            DeviceGuard dg(p0->device);
            if (!dg.ok) return SBP_ERR_CUDA;
            cudaStream_t st = static_cast<cudaStream_t>(stream);
            SweepArgs a = sweep_args(p0);
            a.boxes = c->table + g.first;
            const SweepKernels& k = p0->sk;
            const int ablocks = (p0->nz / k.za) * k.rb;
            const unsigned nb = (unsigned)g.boxes.size();
            if (stage == SBP_STAGE_SWEEP_FORWARD)
                k.fwd<<<dim3((unsigned)(a.green_blocks + ablocks), nb), k.nta, k.smem_ac, st>>>(a);
            else if (stage == SBP_STAGE_SWEEP_MIDDLE)
                k.mid<<<dim3((unsigned)(k.ra * k.nga + 1), nb), k.ntb, k.smem_b, st>>>(a);
            else
                k.inv<<<dim3((unsigned)ablocks, nb), k.nta, k.smem_ac, st>>>(a);
            return launch_status();
        }
        return SBP_ERR_INVALID_ARG;
    }
    return SBP_ERR_INVALID_ARG;
}

sbp_status sbp_plan_query(sbp_plan p, int what, double* value) {
    if (!p || !value) return SBP_ERR_INVALID_ARG;
    if (what == SBP_QUERY_SCHEDULE) {
        *value = p->sweep ? 2.0 : 1.0;
        return SBP_OK;
    }
    if (what == SBP_QUERY_LAUNCHES_PER_SOLVE) {
        *value = (double)launches_per_solve(p, -1);
        return SBP_OK;
    }
    return SBP_ERR_INVALID_ARG;
}

const char* sbp_version(void) { return "sbp 0.2.0 (sm_103a)"; }

}  // extern "C"
