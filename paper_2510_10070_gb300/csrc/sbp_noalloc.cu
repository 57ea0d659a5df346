// sbp_noalloc.cu — an FP32 solve that allocates no device memory.
//
// Some host programs cannot call cudaMalloc while they run: codes that hand
// all device memory to their own pool allocator at start-up and forbid any
// other allocation, real-time loops that cannot afford the implicit device
// synchronisation of an allocation, and plugin hosts that only give a library
// the buffers they pass in.  sbp_plan_create allocates the spectrum workspace
// and tables, so those programs cannot use a plan.  This entry point keeps
// the workspace in one fixed-size array in device global memory instead,
// declared below; every GPU that loads the library holds it until the
// process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Every byte a call reads is written earlier in the same call, so
// nothing has to start at zero.  Two calls whose work overlaps on the GPU
// (for example on two streams) race on the array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/sbp.h"
#include "sbp_internal.h"

using namespace sbp;

namespace {

constexpr size_t kScratchBytes = (size_t)40 << 20;  // 40 MiB

// The workspace.  In host code this name is only a stand-in for the device
// array; kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (with that device current) and cached.
sbp_status scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return SBP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return SBP_OK;
}

constexpr size_t kSmemLimit = 224 * 1024;

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
bool length_ok(int n) { return n >= 2 && n <= 2048 && (pow2(n) || (n % 3 == 0 && pow2(n / 3))); }
size_t up256(size_t v) { return (v + 255) / 256 * 256; }

bool fft_plan(int n, FftPlan& P) {
    std::memset(&P, 0, sizeof(P));
    P.n = n;
    P.E = plan_E(n, false);
    if (n % P.E != 0) return false;
    P.Tf = n / P.E;
    int rem = n, ns = 1, s = 0;
    while (rem > 1) {
        const int r = pick_radix(P.E, rem);
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

// Where the per-call tables sit in the workspace (byte offsets) and what
// they hold, for the table kernel below.
struct TableArgs {
    unsigned char* base;
    size_t o_tx, o_ty, o_tz, o_t2, o_kz, o_c00;
    int nx, ny, nz;
    double Lz;
};

// Builds every table of a call on the device, in FP64, rounded once to the
// float the kernels read: twiddles e^{-2πi k/n} for n = nx, ny, nz and
// e^{-πi k/nz}; k_z,m² = (π m / Lz)² for m ≤ nz; and the FP64 k = 0 vertical
// kernel c00_n = (1/2nz) [Lz²/2 + Σ_{m odd} (-2/k_z,m²) cos(π m n / nz)],
// |n| < nz (Eq. Green's function regularized in Fourier at k = 0 with L = Lz,
// inverse-transformed over the 2nz padded modes).  Blocks 0 .. 2nz-2 each
// reduce one c00 entry over m (integer phase m·n mod 2nz, so the cosine
// argument is exact); the remaining blocks write the twiddles and k_z².
__global__ void __launch_bounds__(256) k_noalloc_tables(TableArgs A) {
    __shared__ double red[256];
    const int tid = threadIdx.x;
    const int nc = 2 * A.nz - 1;
    if ((int)blockIdx.x < nc) {
        const int n = (int)blockIdx.x - (A.nz - 1);
        const int M = 2 * A.nz;
        const double pi_over_lz = 3.141592653589793238462643383279 / A.Lz;
        double acc = 0.0;
        for (int m = -A.nz + 1 + 2 * tid; m < A.nz; m += 2 * blockDim.x) {  // odd m in [-nz, nz)
            long long ph = ((long long)m * n) % M;
            if (ph < 0) ph += M;
            const double kz = pi_over_lz * (double)m;
            acc += (-2.0 / (kz * kz)) * cospi((double)ph / (double)A.nz);
        }
        red[tid] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (tid < w) red[tid] += red[tid + w];
            __syncthreads();
        }
        if (tid == 0)
            reinterpret_cast<double*>(A.base + A.o_c00)[n + A.nz - 1] = (0.5 * A.Lz * A.Lz + red[0]) / (double)M;
        return;
    }
    // twiddles and k_z²: one entry per thread over the remaining blocks
    const int i = ((int)blockIdx.x - nc) * blockDim.x + tid;
    auto tw = [&](size_t off, int k, int count, double den) {
        if (k >= count) return;
        double sn, cs;
        sincospi(2.0 * (double)k / den, &sn, &cs);
        float* out = reinterpret_cast<float*>(A.base + off);
        out[2 * k] = (float)cs;
        out[2 * k + 1] = (float)-sn;
    };
    tw(A.o_tx, i, A.nx, A.nx);
    tw(A.o_ty, i, A.ny, A.ny);
    tw(A.o_tz, i, A.nz, A.nz);
    tw(A.o_t2, i, A.nz, 2.0 * A.nz);
    if (i <= A.nz) {
        const double kz = 3.141592653589793238462643383279 * (double)i / A.Lz;
        reinterpret_cast<float*>(A.base + A.o_kz)[i] = (float)(kz * kz);
    }
}

}  // namespace

extern "C" sbp_status sbp_solve_noalloc(int nx, int ny, int nz, double Lx, double Ly, double Lz, double q,
                                        double Omega, double G, const float* rho, float* phi, double t,
                                        void* stream) {
    // ---- arguments (the same rules as sbp_plan_create and sbp_solve)
    const auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    if (!pos(Lx) || !pos(Ly) || !pos(Lz) || !pos(Omega) || !pos(G) || !std::isfinite(q) || !std::isfinite(t))
        return SBP_ERR_INVALID_ARG;
    if (!rho || !phi || (reinterpret_cast<uintptr_t>(rho) & 15u) || (reinterpret_cast<uintptr_t>(phi) & 15u))
        return SBP_ERR_INVALID_ARG;
    if (nx < 4 || ny < 4 || nz < 2 || (nx & 1) || (ny & 1) || !length_ok(nx) || !length_ok(ny) || !length_ok(nz))
        return SBP_ERR_UNSUPPORTED_SIZE;
    const size_t cells = (size_t)nx * ny * nz;
    {
        const uintptr_t r0 = reinterpret_cast<uintptr_t>(rho), f0 = reinterpret_cast<uintptr_t>(phi);
        const size_t bytes = cells * sizeof(float);
        if (r0 != f0 && r0 < f0 + bytes && f0 < r0 + bytes) return SBP_ERR_INVALID_ARG;
    }

    // ---- launch configuration (as a plan would choose it; z pass: split halves)
    FftPlan px, py, pz;
    if (!fft_plan(nx, px) || !fft_plan(ny, py) || !fft_plan(nz, pz)) return SBP_ERR_UNSUPPORTED_SIZE;
    const int h = nx / 2 + 1, pitch = (h + 1) / 2 * 2;
    const size_t cs = sizeof(cpx<float>);
    int Cx = std::max(1, std::min(16, kMaxThreads / px.Tf));
    const auto xsm = [&](int C) { return (size_t)nx * cs + (size_t)C * padded_row(nx) * cs; };
    while (Cx > 1 && ((ny / 2) % Cx != 0 || xsm(Cx) > kSmemLimit)) --Cx;
    int Cy = std::min(std::max(1, std::min(16, kMaxThreads / py.Tf)), h);
    const auto ysm = [&](int C) {
        return (size_t)ny * cs + std::max((size_t)ny * xstride(C), (size_t)xchg_slots<float>(ny, C)) * cs;
    };
    if (is_static_len<float>(ny)) {
        Cy = ypass_cols(ny, false);  // compiled into the static y kernel
    } else {
        while (Cy > 1 && ysm(Cy) > kSmemLimit) --Cy;
    }
    int Cz = std::min(std::max(1, std::min(16, kMaxThreads / (2 * pz.Tf))), h);
    const auto zsm = [&](int C) {
        return 2 * (size_t)nz * cs + (((size_t)(nz + 1) * sizeof(float) + 15) / 16 * 16) +
               (((size_t)C * sizeof(GreenT<float>) + 15) / 16 * 16) + 2 * (size_t)nz * xstride(C) * cs;
    };
    while (Cz > 1 && zsm(Cz) > kSmemLimit) --Cz;
    if ((ny / 2) % Cx != 0 || Cx * px.Tf > kMaxThreads || Cy * py.Tf > kMaxThreads || 2 * Cz * pz.Tf > kMaxThreads ||
        xsm(Cx) > kSmemLimit || ysm(Cy) > kSmemLimit || zsm(Cz) > kSmemLimit)
        return SBP_ERR_UNSUPPORTED_SIZE;
    const KernelSet<float> kx = kernels_for<float>(nx, px.E), ky = kernels_for<float>(ny, py.E),
                           kz = kernels_for<float>(nz, pz.E);  // z pass with split halves: every length
    if (!kx.x_fwd || !ky.y_fwd || !kz.z) return SBP_ERR_UNSUPPORTED_SIZE;
    const int xblocks = (int)((size_t)nz * (ny / 2) / Cx);
    const int gblocks = (h * ny + Cx * px.Tf - 1) / (Cx * px.Tf);

    // ---- scratch layout and the size limit
    size_t off = 0;
    const auto take = [&](size_t b) {
        const size_t o = off;
        off = up256(off + b);
        return o;
    };
    const size_t oW = take((size_t)nz * ny * pitch * cs);
    const size_t oTx = take(nx * cs), oTy = take(ny * cs), oTz = take(nz * cs), oT2 = take(nz * cs);
    const size_t oKz = take((nz + 1) * sizeof(float));
    const size_t oC00 = take((2 * (size_t)nz) * sizeof(double));
    const size_t oTs = take((size_t)xblocks * sizeof(double));
    const size_t oVk = take((size_t)nz * sizeof(double));
    const size_t oGr = take((size_t)h * ny * sizeof(GreenT<float>));
    if (off > kScratchBytes) return SBP_ERR_SCRATCH_LIMIT;

    void* base_v = nullptr;
    const sbp_status ss = scratch_address(&base_v);
    if (ss != SBP_OK) return ss;
    unsigned char* base = static_cast<unsigned char*>(base_v);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // ---- tables: built on the device by one kernel (no host staging, no copies)
    {
        TableArgs ta;
        ta.base = base;
        ta.o_tx = oTx;
        ta.o_ty = oTy;
        ta.o_tz = oTz;
        ta.o_t2 = oT2;
        ta.o_kz = oKz;
        ta.o_c00 = oC00;
        ta.nx = nx;
        ta.ny = ny;
        ta.nz = nz;
        ta.Lz = Lz;
        const int entries = std::max(std::max(nx, ny), nz + 1);
        const int blocks = (2 * nz - 1) + (entries + 255) / 256;
        k_noalloc_tables<<<blocks, 256, 0, st>>>(ta);
    }

    const int lim = (int)kSmemLimit;
    if (cudaFuncSetAttribute(kx.x_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
        cudaFuncSetAttribute(kx.x_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
        cudaFuncSetAttribute(ky.y_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
        cudaFuncSetAttribute(ky.y_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
        cudaFuncSetAttribute(kz.z, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) {
        cudaGetLastError();
        return SBP_ERR_CUDA;
    }

    // ---- the five passes, as sbp_solve runs them
    cpx<float>* W = reinterpret_cast<cpx<float>*>(base + oW);
    double dy0 = std::fmod(q * Omega * Lx * t, Ly);
    if (dy0 < 0.0) dy0 += Ly;
    if (dy0 >= Ly) dy0 -= Ly;

    XArgs xa;
    std::memset(&xa, 0, sizeof(xa));
    xa.P = px;
    xa.pitch = pitch;
    xa.C = Cx;
    xa.pairs_per_plane = ny / 2;
    xa.green_blocks = gblocks;
    xa.gf.tab = base + oGr;
    xa.gf.per_block = (h * ny + gblocks - 1) / gblocks;
    xa.gf.nx = nx;
    xa.gf.ny = ny;
    xa.gf.yhalf = 0;
    xa.gf.Lx = Lx;
    xa.gf.Ly = Ly;
    xa.gf.L = Lz;
    xa.gf.s = dy0 / Lx;
    kx.x_fwd<<<xblocks + gblocks, Cx * px.Tf, xsm(Cx), st>>>(rho, W,
                                                           reinterpret_cast<const cpx<float>*>(base + oTx),
                                                           reinterpret_cast<double*>(base + oTs), xa);
    YArgs ya;
    ya.P = py;
    ya.pitch = pitch;
    ya.h = h;
    ya.C = Cy;
    ya.z0 = 0;
    const dim3 ygrid((h + Cy - 1) / Cy, nz);
    const cpx<float>* twy = reinterpret_cast<const cpx<float>*>(base + oTy);
    ky.y_fwd<<<ygrid, Cy * py.Tf, ysm(Cy), st>>>(W, twy, ya);
    ZArgs za;
    std::memset(&za, 0, sizeof(za));
    za.P = pz;
    za.pitch = pitch;
    za.h = h;
    za.ny = ny;
    za.C = Cz;
    za.L = Lz;
    za.paper_tab = nullptr;
    za.kzc = (M_PI / Lz) * (M_PI / Lz);
    za.scale = 4.0 * M_PI * G / ((double)nx * ny * 2.0 * nz);
    za.zero_k0 = 1;
    za.green = base + oGr;
    za.tile_sums = reinterpret_cast<const double*>(base + oTs);
    za.tiles_per_plane = (ny / 2) / Cx;
    za.c00 = reinterpret_cast<const double*>(base + oC00);
    za.k0_coef = 4.0 * M_PI * G / ((double)nx * ny);
    za.vk0 = reinterpret_cast<double*>(base + oVk);
    kz.z<<<dim3((h + Cz - 1) / Cz, ny), 2 * Cz * pz.Tf, zsm(Cz), st>>>(
        W, reinterpret_cast<const cpx<float>*>(base + oTz), reinterpret_cast<const cpx<float>*>(base + oT2),
        reinterpret_cast<const float*>(base + oKz), za);
    ky.y_inv<<<ygrid, Cy * py.Tf, ysm(Cy), st>>>(W, twy, ya);
    XArgs xi = xa;
    xi.green_blocks = 0;
    xi.gf.tab = nullptr;
    xi.vk0 = reinterpret_cast<const double*>(base + oVk);
    kx.x_inv<<<xblocks, Cx * px.Tf, xsm(Cx), st>>>(W, phi, reinterpret_cast<const cpx<float>*>(base + oTx), xi);
    return cudaGetLastError() == cudaSuccess ? SBP_OK : SBP_ERR_CUDA;
}
