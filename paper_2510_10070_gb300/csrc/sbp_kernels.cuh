// sbp_kernels.cuh — the five pass kernels of one VGF-HybridBC solve.
//
//   x forward : real rows → half spectrum X[z][y][a], a ≤ nx/2 (r2c by pairing
//               two real rows into one complex row).
//   y forward : in place, DFT over y of each (z, a) column.
//   z pass    : per column (b, a): zero-pad to 2nz, forward DFT, multiply by
//               4πG/(nx·ny·2nz) · Ĝ_eff(k(t), k_z,m), inverse DFT, keep the
//               first nz outputs (Sect. 2.3, Eq. Green's function regularized
//               in Fourier with L = Lz).
//   y inverse : in place.
//   x inverse : half spectrum → real rows (c2r by pairing).
//
// Spectrum layout: complex [nz][ny][pitch] with pitch ≥ nx/2+1 (even).
#pragma once

#include <type_traits>

#include "sbp_fft.cuh"
#include "sbp_tma.cuh"

namespace sbp {

constexpr int kMaxThreads = 256;  // threads per block of every pass kernel
// Resident blocks per SM the register allocation aims for (launch bounds):
// the FP32 streaming x/y passes want 4 (≤ 64 registers) and the FP32 padded
// z pass 3; FP64 and 24-element variants keep 2 so that they do not spill.
template <typename T, int E>
constexpr int min_blocks_xy() { return (sizeof(T) == 8 || E > 16) ? 2 : 4; }
// The static-length FP32 x passes and TMA y passes up to 256 fit in 48
// registers without spills, which makes room for a fifth block (40 warps) per
// SM: their time goes to waiting on memory and barriers, so more resident
// warps overlap more of it.
template <typename T, int E, int NS>
constexpr int min_blocks_xs() { return (sizeof(T) == 4 && E == 16 && NS > 0 && NS <= 256) ? 5 : min_blocks_xy<T, E>(); }
template <typename T, int E>
constexpr int min_blocks_z() { return (sizeof(T) == 8 || E > 16) ? 2 : 3; }
// The padded z kernel fits 64 registers at E = 16 (its radix-16 stages apply
// their twiddles one first-level group at a time), so four blocks per SM.
template <typename T, int E>
constexpr int min_blocks_zpad() { return (sizeof(T) == 8 || E > 16) ? 2 : 4; }

// Row stride (complex elements) of a [n][C] exchange buffer: one pad column
// spreads consecutive rows over the banks; a single column needs none.
__host__ __device__ constexpr int xstride(int C) { return C == 1 ? 1 : C + 1; }

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Green's-function parameters of one stored mode as the z pass reads them.
template <typename T>
struct GreenT {
    T k2a, omEa, k2b, omEb;  // |k|² and 1 - e^{-|k|L}, for the mode and its partner
    int kzero, same;
};

// Work a pass kernel may do on the side: fill the Green's table for modes
// [blockIdx.x·per_block, …) (FP64 arithmetic, rounded to the table type).
struct GreenFill {
    void* tab;  // GreenT<T>[ny][nx/2+1] (yhalf: [ny/2+1][nx]) or null
    int per_block;
    int nx, ny;
    int yhalf;  // stored modes: 0 = half in x (periodic-frame passes), 1 = half in y
    double Lx, Ly, L, s;
    const double* s_dev;  // if set, s is read from device memory (batched executor)
};

struct XArgs {
    FftPlan P;           // length nx
    int pitch;           // spectrum row pitch (complex elements)
    int C;               // row pairs per block (divides ny/2)
    int pairs_per_plane; // ny/2
    // x forward: the first green_blocks blocks fill the Green's table
    // while the others transform rows
    int green_blocks;
    GreenFill gf;
    // x inverse, FP32 path: FP64 mean-mode potential per plane (null: none)
    const double* vk0;
};

struct YArgs {
    FftPlan P;  // length ny
    int pitch;
    int h;      // nx/2 + 1
    int C;      // columns per block
    int z0;     // first plane of this launch (grid.y planes from there)
};

struct ZArgs {
    FftPlan P;  // length nz
    int pitch;
    int h;
    int ny;
    int C;
    double L;           // L = Lz (enclosure of the truncated Green's function)
    double kzc;         // (π / Lz)²: k_z,m² = kzc · m²
    double scale;       // 4πG / (nx·ny·2nz)
    int zero_k0;        // FP32 path: leave the (0,0) column to the FP64 side path
    const void* green;  // GreenT<T>[ny][h] at this solve's time
    // FP64 mean-mode side path (FP32 path only; vk0 null otherwise): block
    // (0,0) reduces the x-forward tile sums to plane sums S and convolves them
    // with the k = 0 kernel: vk0[i] = coef · Σ_j c00[i - j + nz - 1] S[j].
    const double* tile_sums;
    int tiles_per_plane;
    const double* c00;
    double k0_coef;
    double* vk0;
    // α ≠ 1 with 4·nz padding (the paper's Sect. 2.3 parameters): per |m| ≤ 2nz
    // k_z sin(k_z L), 1 - cos(k_z L), k_z² and Ĝ(0, k_z), [m][4] in the plan's type
    const void* paper_tab;
};

// SASHA (Sect. 2.2): the k = 0 column in FP64 from the plane sums, one block.
// vk0[i] = k0_coef Σ_j c_{i-j} (S_j - ρ̄ nx ny) + 4πG ρ̄ z_i (z_i/2 - centre·z0)
// with ρ̄ = Σ S_j / N, z0 = Σ z_j S_j / Σ S_j (0 without mass) and c the k = 0
// column of the periodic kernel -1/k_z² on the 2 nz padded grid.
struct SashaArgs {
    const double* tile_sums;  // [nz][tiles_per_plane]
    int tiles_per_plane;
    int nz;
    const double* c00;        // [2 nz - 1]
    double k0_coef;           // 4πG / (nx ny)
    double fourpiG;           // 4πG
    double cells_xy;          // nx ny
    double Lz;                // cell centres z_i = -Lz/2 + (i + ½) Lz/nz
    double centre;            // vertex of Φ0 in units of z0
    double* vk0;              // [nz] out
};

// Block-wide sum of a pair of doubles (result in every thread); `tmp` holds
// 2·(blockDim/32) doubles of shared memory.  Contains barriers.
__device__ __forceinline__ double2 block_sum_d2(double2 v, double* tmp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = (blockDim.x + 31) / 32;
    const int wl = min(32, (int)blockDim.x - warp * 32);
    const unsigned mask = (wl == 32) ? 0xffffffffu : ((1u << wl) - 1u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double a = __shfl_xor_sync(mask, v.x, o), b = __shfl_xor_sync(mask, v.y, o);
        if ((lane ^ o) < wl) {
            v.x += a;
            v.y += b;
        }
    }
    if (lane == 0) {
        tmp[2 * warp] = v.x;
        tmp[2 * warp + 1] = v.y;
    }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    for (int w = 0; w < nw; ++w) {
        r.x += tmp[2 * w];
        r.y += tmp[2 * w + 1];
    }
    __syncthreads();
    return r;
}

// Block (0,0) of a z pass: the FP64 mean mode (O(nz²) FP64 work on one SM,
// overlapped with the other blocks).  `scratch` holds nz doubles.
__device__ __forceinline__ void mean_mode_fp64(const ZArgs& A, int nz, double* scratch) {
    const int tid = threadIdx.x;
    for (int j = tid; j < nz; j += blockDim.x) {
        double sacc = 0.0;
        for (int q = 0; q < A.tiles_per_plane; ++q) sacc += A.tile_sums[(size_t)j * A.tiles_per_plane + q];
        scratch[j] = sacc;
    }
    __syncthreads();
    for (int i = tid; i < nz; i += blockDim.x) {
        double acc = 0.0;
#pragma unroll 4
        for (int j = 0; j < nz; ++j) acc = fma(A.c00[i - j + nz - 1], scratch[j], acc);
        A.vk0[i] = A.k0_coef * acc;
    }
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T fast_div(T a, T b);
// FP32: a · rcp.approx(b) (relative error about 2^-23; the divisors here are
// positive and far from the denormal and overflow ranges)
template <>
__device__ __forceinline__ float fast_div<float>(float a, float b) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
    return a * r;
}
template <>
__device__ __forceinline__ double fast_div<double>(double a, double b) { return a / b; }

// Error-free float sum (Knuth's TwoSum) and double-float accumulation.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    float h, l;
    two_sum(s, e, h, l);
    return {h, l};
}
// Compensated (Kahan) running sum: hi holds the sum, lo the negated
// running error; four float operations per value.
__device__ __forceinline__ void kahan_add(FF& a, float x) {
    const float y = x + a.lo;
    const float t = a.hi + y;
    a.lo = y - (t - a.hi);
    a.hi = t;
}
__device__ __forceinline__ FF ff_add_f(FF a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    e += a.lo;
    float h, l;
    two_sum(s, e, h, l);
    return {h, l};
}

// Block-wide double-float sum of every thread's partial; the result is valid
// in thread 0.  Contains a barrier.  The last warp may be partial, so only
// lanes that exist are added.
__device__ __forceinline__ FF block_sum_ff(FF acc) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int wl = min(32, (int)blockDim.x - warp * 32);
    const unsigned mask = (wl == 32) ? 0xffffffffu : ((1u << wl) - 1u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF other = {__shfl_xor_sync(mask, acc.hi, o), __shfl_xor_sync(mask, acc.lo, o)};
        if ((lane ^ o) < wl) acc = ff_add(acc, other);
    }
    __shared__ FF wsum[kMaxThreads / 32];
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    FF tot = {0.f, 0.f};
    if (tid == 0)
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot = ff_add(tot, wsum[w]);
    return tot;
}

// Green's-function parameters of stored mode (a, b), unsigned FFT indices a < nx, b < ny:
// |k|² and 1 - e^{-|k| L} for the mode and for its Hermitian partner
// (Sect. 2.1 wave-vector k_x = K_x + s K_y; Eq. Green's function regularized
// in Fourier needs e^{-kL}).  FP64 throughout.
struct GreenMode {
    double k2a, omEa, k2b, omEb;
    int kzero;  // signed (a, b) == (0, 0)
    int same;   // partner has the same |k|
};

__device__ __forceinline__ int wrap_signed(int v, int n) {
    if (v >= n / 2) v -= n;
    if (v < -(n / 2)) v += n;
    return v;
}

__device__ __forceinline__ GreenMode green_mode(int a, int b, int nx, int ny, double Lx, double Ly, double L,
                                                double s) {
    GreenMode g;
    const int as = (a < nx / 2) ? a : a - nx;
    const int bs = (b < ny / 2) ? b : b - ny;
    const int ap = wrap_signed(-as, nx);
    const int bp = wrap_signed(-bs, ny);
    g.kzero = (as == 0 && bs == 0);
    {
        const double Kx = kTwoPi * (double)as / Lx, Ky = kTwoPi * (double)bs / Ly;
        const double kx = fma(s, Ky, Kx);
        g.k2a = fma(kx, kx, Ky * Ky);
        g.omEa = g.kzero ? 0.0 : -expm1(-sqrt(g.k2a) * L);
    }
    g.same = (ap == -as && bp == -bs);
    if (g.same) {
        g.k2b = g.k2a;
        g.omEb = g.omEa;
    } else {
        const double Kx = kTwoPi * (double)ap / Lx, Ky = kTwoPi * (double)bp / Ly;
        const double kx = fma(s, Ky, Kx);
        g.k2b = fma(kx, kx, Ky * Ky);
        g.omEb = -expm1(-sqrt(g.k2b) * L);
    }
    return g;
}

template <typename T>
__device__ __forceinline__ void green_fill(const GreenFill& gf, int block) {
    if (gf.tab == nullptr) return;
    GreenT<T>* tab = static_cast<GreenT<T>*>(gf.tab);
    const int h = gf.yhalf ? gf.nx : gf.nx / 2 + 1;  // stored modes per row
    const int total = h * (gf.yhalf ? gf.ny / 2 + 1 : gf.ny);
    const int q0 = block * gf.per_block;
    const int q1 = min(total, q0 + gf.per_block);
    const double s = gf.s_dev != nullptr ? *gf.s_dev : gf.s;
    // FP64 for every plan type (the FP32 path stores the FP64 values rounded
    // once to float): one table entry per thread, spread over the blocks the
    // caller reserves for it, so the 1/64-rate FP64 pipe of many SMs shares it.
    for (int q = q0 + (int)threadIdx.x; q < q1; q += blockDim.x) {
        const int b = q / h, a = q - b * h;
        const GreenMode g = green_mode(a, b, gf.nx, gf.ny, gf.Lx, gf.Ly, gf.L, s);
        tab[q] = GreenT<T>{(T)g.k2a, (T)g.omEa, (T)g.k2b, (T)g.omEb, g.kzero, g.same};
    }
}

// The plan's Green's table as doubles, [count][4] = (|k|², 1 - e^{-|k|L}, the
// same for the partner), for stage-level tests of exactly what a solve reads.
template <typename T>
__global__ void k_green_dump(const GreenT<T>* __restrict__ tab, double* __restrict__ out, int count) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const GreenT<T> g = tab[q];
    out[4 * q + 0] = (double)g.k2a;
    out[4 * q + 1] = (double)g.omEa;
    out[4 * q + 2] = (double)g.k2b;
    out[4 * q + 3] = (double)g.omEb;
}

// Vectorised contiguous copy global → shared staging (16-byte chunks when the
// span allows it).  Reals only.
template <typename T>
__device__ __forceinline__ void load_rows_to_smem(const T* __restrict__ src, T* __restrict__ tile, int rows, int n,
                                                  int spitch) {
    const int total = rows * n;
    constexpr int V = 16 / sizeof(T);
    if (n % V == 0) {
        using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        const V4* s4 = reinterpret_cast<const V4*>(src);
        for (int q = threadIdx.x; q < total / V; q += blockDim.x) {
            const V4 w = __ldcs(s4 + q);
            const int e0 = q * V;
            const int r = e0 / n, x = e0 - r * n;
            T* d = tile + r * spitch + x;
            const T* wv = reinterpret_cast<const T*>(&w);
#pragma unroll
            for (int k = 0; k < V; ++k) d[k] = wv[k];
        }
    } else {
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            const int r = q / n, x = q - r * n;
            tile[r * spitch + x] = src[q];
        }
    }
}

template <typename T>
__device__ __forceinline__ void store_rows_from_smem(T* __restrict__ dst, const T* __restrict__ tile, int rows, int n,
                                                     int spitch) {
    const int total = rows * n;
    constexpr int V = 16 / sizeof(T);
    if (n % V == 0) {
        using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        V4* d4 = reinterpret_cast<V4*>(dst);
        for (int q = threadIdx.x; q < total / V; q += blockDim.x) {
            const int e0 = q * V;
            const int r = e0 / n, x = e0 - r * n;
            const T* s = tile + r * spitch + x;
            V4 w;
            T* wv = reinterpret_cast<T*>(&w);
#pragma unroll
            for (int k = 0; k < V; ++k) wv[k] = s[k];
            __stcs(d4 + q, w);
        }
    } else {
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            const int r = q / n, x = q - r * n;
            dst[q] = tile[r * spitch + x];
        }
    }
}

// ---------------------------------------------------------------------------
// x forward: C row pairs per block (2C consecutive real rows of one plane).
// Lanes run along x (t fastest), so each thread loads its E elements of both
// rows straight from global memory with coalesced loads.
// smem: tw[n] | C padded rows (the FFT's exchange; for runtime lengths and
// row pairs wider than a warp, also the paired spectrum Z for the split)
// ---------------------------------------------------------------------------
template <typename T, int E, int NS>
__global__ void __launch_bounds__(kMaxThreads, (min_blocks_xs<T, E, NS>())) k_x_forward(const T* __restrict__ rho, cpx<T>* __restrict__ W,
                                                           const cpx<T>* __restrict__ twg,
                                                           double* __restrict__ tile_sums, XArgs A) {
    if ((int)blockIdx.x < A.green_blocks) {  // Green's table, off the transform blocks
        green_fill<T>(A.gf, blockIdx.x);
        return;
    }
    const int bid = blockIdx.x - A.green_blocks;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = NS > 0 ? NS : A.P.n, C = A.C, Tf = NS > 0 ? NS / E : A.P.Tf;
    const int RP = padded_row(n);
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* xb = tw + n;
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) tw[i] = twg[i];

    const int t = tid % Tf, c = tid / Tf;
    const long long pair0 = (long long)bid * C;
    const T* r0p = rho + (pair0 + c) * 2 * n;
    cpx<T> v[1][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int x = t + Tf * e;
        v[0][e] = {__ldcs(r0p + x), __ldcs(r0p + n + x)};
    }
    if constexpr (sizeof(T) == 4) {
        if (tile_sums != nullptr) {
            // FP64-quality plane sums from error-free float additions
            // two compensated accumulators (even and odd row of the pair) as
            // one packed pair: y = x + lo, t = hi + y, lo = y - (t - hi), hi = t
            cpx<float> hi = {0.f, 0.f}, lo = {0.f, 0.f};
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const cpx<float> y = cadd(cpx<float>{(float)v[0][e].x, (float)v[0][e].y}, lo);
                const cpx<float> tt = cadd(hi, y);
                lo = csub(y, csub(tt, hi));
                hi = tt;
            }
            const FF tot = block_sum_ff(ff_add(FF{hi.x, lo.x}, FF{hi.y, lo.y}));
            if (tid == 0) tile_sums[bid] = (double)tot.hi + (double)tot.lo;
        }
    } else {
        if (tile_sums != nullptr) {  // FP64 plane sums (SASHA)
            __shared__ double dsum[2 * (kMaxThreads / 32)];
            double acc = 0.0;
#pragma unroll
            for (int e = 0; e < E; ++e) acc += (double)v[0][e].x + (double)v[0][e].y;
            const double2 tot = block_sum_d2(make_double2(acc, 0.0), dsum);
            if (tid == 0) tile_sums[bid] = tot.x;
        }
    }
    __syncthreads();  // twiddles visible
    const SmemRow<T> buf[1] = {{xb + c * RP, 0}};
    fft_run<NS, E, 1, T>(v, t, A.P, tw, buf);

    // split the paired transform: X0 = (Z[k] + conj Z[n-k]) / 2, X1 = -i (Z[k] - conj Z[n-k]) / 2
    const T half = (T)0.5;
    if constexpr (NS > 0 && NS / E <= 32) {
        // Static plans whose row pair fits in one warp: Z[n-k] is in a lane of
        // the same row pair (k = t + Tf·e: element E-1-e of lane Tf-t for
        // t > 0, element (E-e) mod E of lane t = 0 itself), so the split runs
        // on warp shuffles instead of a shared-memory round trip.  Tf is a
        // power of two and row pairs never straddle a warp.
        constexpr int TF = NS / E;
        static_assert((TF & (TF - 1)) == 0, "row-pair lane groups must tile a warp");
        const int lane = tid & 31;
        const int src = lane - t + ((TF - t) & (TF - 1));
        const int live = min(32, (int)blockDim.x - (tid & ~31));
        const unsigned mask = live == 32 ? 0xffffffffu : ((1u << live) - 1u);
        const long long row = 2 * (pair0 + c);
        cpx<T>* o0 = W + row * A.pitch;
        cpx<T>* o1 = o0 + A.pitch;
#pragma unroll
        for (int e = 0; e <= E / 2; ++e) {
            const cpx<T> send = v[0][E - 1 - e];
            cpx<T> Bz;
            Bz.x = __shfl_sync(mask, send.x, src);
            Bz.y = __shfl_sync(mask, send.y, src);
            if (t == 0) Bz = v[0][(E - e) % E];
            Bz = cconj(Bz);
            const cpx<T> Az = v[0][e];
            const cpx<T> X0 = {(Az.x + Bz.x) * half, (Az.y + Bz.y) * half};
            const cpx<T> X1 = {(Az.y - Bz.y) * half, (Bz.x - Az.x) * half};
            if (e < E / 2 || t == 0) {
                const int k = t + TF * e;
                o0[k] = X0;
                o1[k] = X1;
            }
        }
        return;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) buf[0][t + Tf * e] = v[0][e];
    __syncthreads();
    const int h = n / 2 + 1;
    for (int q = tid; q < C * h; q += blockDim.x) {
        const int cc = q / h, k = q - cc * h;
        const cpx<T>* zr = xb + cc * RP;
        const cpx<T> Az = zr[k + (k >> 4)];
        const int km = (k == 0) ? 0 : n - k;
        const cpx<T> Bz = cconj(zr[km + (km >> 4)]);
        const cpx<T> X0 = {(Az.x + Bz.x) * half, (Az.y + Bz.y) * half};
        const cpx<T> X1 = {(Az.y - Bz.y) * half, (Bz.x - Az.x) * half};
        const long long row = 2 * (pair0 + cc);
        W[row * A.pitch + k] = X0;
        W[(row + 1) * A.pitch + k] = X1;
    }
}

// ---------------------------------------------------------------------------
// y pass (forward or inverse), in place: block = (a-tile of C columns, plane z).
// smem: tw[n] | exchange [n][C+1]
// ---------------------------------------------------------------------------
template <typename T, int E, bool INV, int NS, int CS = 0>
__global__ void __launch_bounds__(kMaxThreads, (min_blocks_xy<T, E>())) k_y_pass(cpx<T>* __restrict__ W, const cpx<T>* __restrict__ twg, YArgs A) {
    // CS > 0: the column count is a compile-time constant (static lengths),
    // so every exchange-buffer address is a base plus an immediate offset.
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = NS > 0 ? NS : A.P.n, Tf = NS > 0 ? NS / E : A.P.Tf;
    const int C = CS > 0 ? CS : A.C;
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* xb = tw + n;
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) tw[i] = twg[i];

    const int c = tid % C, t = tid / C;
    const int a = blockIdx.x * C + c;
    const bool valid = a < A.h;
    const size_t step = (size_t)Tf * A.pitch;
    cpx<T>* col = W + (((size_t)blockIdx.y + A.z0) * n + t) * A.pitch + a;
    cpx<T> v[1][E];
    {
        const cpx<T>* src = col;
#pragma unroll
        for (int e = 0; e < E; ++e, src += step) {
            cpx<T> x = {(T)0, (T)0};
            if (valid) x = *src;
            v[0][e] = INV ? cconj(x) : x;
        }
    }
    __syncthreads();  // twiddles visible
    if constexpr (CS > 0) {
        const XchgCol<T, CS> buf[1] = {{xb + c, 0}};
        fft_run<NS, E, 1, T>(v, t, A.P, tw, buf);
    } else {
        const SmemCol<T> buf[1] = {{xb + c, xstride(C)}};
        fft_run<NS, E, 1, T>(v, t, A.P, tw, buf);
    }
    if (valid) {
        cpx<T>* dst = col;
#pragma unroll
        for (int e = 0; e < E; ++e, dst += step) *dst = INV ? cconj(v[0][e]) : v[0][e];
    }
}

// y pass with a TMA tile load (static lengths): one thread loads the whole
// [NS][CS] column tile of plane z into shared memory with cp.async.bulk.tensor
// on an mbarrier, the tile then serves as the FFT's exchange buffer, and the
// results are stored straight from registers.
// smem: tile [NS][CS] (128-byte aligned; later the exchange, TileCol) | tw[NS] | mbarrier
template <typename T, int E, bool INV, int NS, int CS>
__global__ void __launch_bounds__(kMaxThreads, (min_blocks_xs<T, E, NS>()))
    k_y_tma(cpx<T>* __restrict__ W, const cpx<T>* __restrict__ twg, YArgs A, TmaCtl ctl,
            const __grid_constant__ CUtensorMap tmap) {
    constexpr int Tf = NS / E;
    constexpr int C = CS;
    constexpr int BOXR = NS < 256 ? NS : 256;  // rows per TMA box (box dimensions are at most 256)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<T>* tile = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* tw = tile + tile_slots<T>(NS, C);  // the tile, then the FFT's exchange
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + NS);
    const int tid = threadIdx.x;
    const int a0 = blockIdx.x * C;
    const int row0 = (blockIdx.y + A.z0) * NS;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0 && !ctl.withhold) {
        mbar_arrive_expect_tx(bar, (uint32_t)(NS * C * sizeof(cpx<T>)));
#pragma unroll
        for (int r = 0; r < NS; r += BOXR) tma_load_2d(tile + r * C, &tmap, 2 * a0, row0 + r, bar);
    }
    for (int i = tid; i < NS; i += blockDim.x) tw[i] = twg[i];
    const bool ok = mbar_wait_bounded(bar, 0, ctl.budget);
    if (!__syncthreads_and(ok)) {  // uniform exit: the copy did not arrive in time
        if (tid == 0) atomicExch(ctl.err, 1);
        // A copy that was issued but is only late still targets this block's
        // shared memory: keep the block resident (a second bounded wait) until
        // it lands, so that it cannot write into memory given to another block.
        if (!ctl.withhold) mbar_wait_bounded(bar, 0, ctl.budget);
        return;
    }

    const int c = tid % C, t = tid / C;
    const int a = a0 + c;
    cpx<T> v[1][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const cpx<T> x = tile[(t + Tf * e) * C + c];
        v[0][e] = INV ? cconj(x) : x;
    }
    const TileCol<T, C> buf[1] = {{tile + c, 0}};
    fft_static<NS, E, 0, 1, T>(v, t, tw, buf);  // first exchange write follows a barrier
    if (a < A.h) {
        cpx<T>* dst = W + ((size_t)row0 + t) * A.pitch + a;
        const size_t step = (size_t)Tf * A.pitch;
#pragma unroll
        for (int e = 0; e < E; ++e, dst += step) *dst = INV ? cconj(v[0][e]) : v[0][e];
    }
}

// ---------------------------------------------------------------------------
// z pass: block = (a-tile of C columns, row b).  The length-2nz padded DFT of
// a column x[0..nz) splits into even outputs FFT_nz(x) and odd outputs
// FFT_nz(x[j]·e^{-πi j/nz}); the truncated inverse recombines
// y[n] = IFFT_nz(Y_even)[n] + e^{+πi n/nz} IFFT_nz(Y_odd)[n] for n < nz.
// smem: tw[n] | tw2[n] (e^{-πi p/n}) | kz2[n+1] | green[C] | exchange 2×[n][C+1]
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T green_eff_elem(int m, int nz, T kz2, T k2a, T omEa, T k2b, T omEb, bool kzero,
                                            bool same, T L2half) {
    // m ∈ [0, 2nz) unsigned; parity of m equals parity of the signed index.
    const bool odd = (m & 1) != 0;
    if (kzero) {
        if (m == 0) return L2half;
        return odd ? fast_div((T)-2, kz2) : (T)0;
    }
    const T na = odd ? ((T)2 - omEa) : omEa;  // 1 ∓ e^{-kL}
    T g = -fast_div(na, k2a + kz2);
    if (!same) {
        const T nb = odd ? ((T)2 - omEb) : omEb;
        g = (T)0.5 * (g - fast_div(nb, k2b + kz2));
    }
    return g;
}

// JOINT = true : each thread holds both halves of its E elements (two
//                 columns of the engine), recombined in registers.
// JOINT = false: threads come in two halves per column: half 0 carries the
//                 even padded outputs FFT_n(x), half 1 the odd ones
//                 FFT_n(x·e^{-πi j/n}); the odd half hands its term over
//                 through shared memory.
template <typename T, int E, int NS, bool JOINT>
__global__ void __launch_bounds__(kMaxThreads) k_z_pass(cpx<T>* __restrict__ W, const cpx<T>* __restrict__ twg,
                                                        const cpx<T>* __restrict__ tw2g, const T* __restrict__ kz2g,
                                                        ZArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = NS > 0 ? NS : A.P.n, C = A.C, Tf = NS > 0 ? NS / E : A.P.Tf;
    const int XS = xstride(C);
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* tw2 = tw + n;
    T* kz2 = reinterpret_cast<T*>(tw2 + n);
    const int kz2_slots = ((n + 1) * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
    GreenT<T>* gm = reinterpret_cast<GreenT<T>*>(kz2 + kz2_slots);
    const int gm_bytes = ((C * (int)sizeof(GreenT<T>)) + 15) / 16 * 16;
    cpx<T>* xb0 = reinterpret_cast<cpx<T>*>(reinterpret_cast<unsigned char*>(gm) + gm_bytes);

    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) {
        tw[i] = twg[i];
        tw2[i] = tw2g[i];
    }
    for (int i = tid; i <= n; i += blockDim.x) kz2[i] = kz2g[i];
    const int b = blockIdx.y;
    if (tid < C) {
        const int a = blockIdx.x * C + tid;
        GreenT<T> g = {};
        if (a < A.h) g = static_cast<const GreenT<T>*>(A.green)[(size_t)b * A.h + a];
        gm[tid] = g;
    }
    if (A.vk0 != nullptr && blockIdx.x == 0 && blockIdx.y == 0)
        mean_mode_fp64(A, n, reinterpret_cast<double*>(xb0));
    __syncthreads();

    constexpr int NH = JOINT ? 2 : 1;  // halves held per thread
    const int c = tid % C;
    const int half = JOINT ? 0 : ((tid / C) & 1);
    const int t = JOINT ? tid / C : tid / (2 * C);
    const int a = blockIdx.x * C + c;
    const bool valid = a < A.h;
    cpx<T>* col = W + (size_t)b * A.pitch + a;
    const size_t zstride = (size_t)A.ny * A.pitch;
    cpx<T> v[NH][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int p = t + Tf * e;
        cpx<T> x = {(T)0, (T)0};
        if (valid) x = col[(size_t)p * zstride];
        if constexpr (JOINT) {
            v[0][e] = x;
            v[1][e] = cmul(x, tw2[p]);
        } else {
            v[0][e] = half ? cmul(x, tw2[p]) : x;
        }
    }
    SmemCol<T> buf[NH];
    if constexpr (JOINT) {
        buf[0] = {xb0 + c, XS};
        buf[1] = {xb0 + (size_t)n * XS + c, XS};
    } else {
        buf[0] = {xb0 + (size_t)half * n * XS + c, XS};
    }
    fft_run<NS, E, NH, T>(v, t, A.P, tw, buf);

    // multiply by scale·Ĝ_eff(m), m = 2p + half, and conjugate for the inverse
    {
        const GreenT<T> g = gm[c];
        const T scale = (T)A.scale;
        const T L2half = (T)(0.5 * A.L * A.L);
        const bool kill = A.zero_k0 && g.kzero;
#pragma unroll
        for (int hh = 0; hh < NH; ++hh) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int p = t + Tf * e;
                const int m = 2 * p + (JOINT ? hh : half);
                const int ms = (m <= n) ? m : 2 * n - m;  // |signed m|
                const T ge = green_eff_elem<T>(m, n, kz2[ms], g.k2a, g.omEa, g.k2b, g.omEb, g.kzero != 0,
                                               g.same != 0, L2half);
                const T f = kill ? (T)0 : ge * scale;
                v[hh][e] = {v[hh][e].x * f, -v[hh][e].y * f};
            }
        }
    }
    fft_run<NS, E, NH, T>(v, t, A.P, tw, buf);

    // y[p] = IFFT(Y_even)[p] + e^{+πi p/n} IFFT(Y_odd)[p]
    if constexpr (JOINT) {
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int p = t + Tf * e;
                col[(size_t)p * zstride] = cadd(cconj(v[0][e]), cmul(cconj(v[1][e]), cconj(tw2[p])));
            }
        }
    } else {
        __syncthreads();
        if (half) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int p = t + Tf * e;
                buf[0][p] = cmul(cconj(v[0][e]), cconj(tw2[p]));
            }
        }
        __syncthreads();
        if (!half && valid) {
            const SmemCol<T> odd = {xb0 + (size_t)n * XS + c, XS};
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int p = t + Tf * e;
                col[(size_t)p * zstride] = cadd(cconj(v[0][e]), odd[p]);
            }
        }
    }
}

// Columns per block of the y pass with static length N (compile-time):
// 16 (FP32) or 8 (FP64), fewer when a column needs more than 256/16 threads.
__host__ __device__ constexpr int ypass_cols(int N, bool f64) {
    const int per_col = N / plan_E(N, f64);
    const int cmax = f64 ? 8 : 16;
    const int c = kMaxThreads / per_col;
    return c < 1 ? 1 : (c < cmax ? c : cmax);
}

// Columns per block of the padded z kernel (compile-time): 16 (FP32) or 8
// (FP64), fewer when a column needs more than 256/16 threads.
__host__ __device__ constexpr int zpad_cols(int N, int E, bool f64) {
    const int per_col = 2 * N / E;
    const int cmax = f64 ? 8 : 16;
    const int c = kMaxThreads / per_col;
    return c < 1 ? 1 : (c < cmax ? c : cmax);
}

// Per-column factors of scale·Ĝ_eff(m) = Σ_branches F(parity)/(k² + k_z,m²):
// for k ≠ 0, F = -scale·(1 ∓ e^{-kL}) for the mode and its Hermitian partner,
// weighted ½ + ½ when their |k| differ and 1 + 0 otherwise; the k = 0 column
// is handled separately.
template <typename T>
struct GreenCoef {
    T k2a, ae, ao, k2b, be, bo;
    bool kzero, same, kill;
};

template <typename T>
__device__ __forceinline__ GreenCoef<T> green_coef(const GreenT<T>& g, T scale, bool zero_k0) {
    GreenCoef<T> q;
    q.kzero = g.kzero != 0;
    q.same = g.same != 0;
    q.kill = zero_k0 && q.kzero;
    // the second branch carries weight 0 when the partner has the same |k|
    const T wa = q.same ? (T)1 : (T)0.5;
    const T wb = q.same ? (T)0 : (T)0.5;
    q.k2a = g.k2a;
    q.ae = -scale * wa * g.omEa;
    q.ao = -scale * wa * ((T)2 - g.omEa);
    q.k2b = q.kzero ? (T)1 : g.k2b;  // keep the unused division finite
    q.be = -scale * wb * g.omEb;
    q.bo = -scale * wb * ((T)2 - g.omEb);
    return q;
}

// scale·Ĝ_eff at unsigned padded index m ∈ [0, 2N) with |signed m| = ms.
// Branch-free: lanes of a warp hold different columns, so per-column cases
// are selected, not branched on (both branches are cheap).
template <typename T>
__device__ __forceinline__ T green_factor(const GreenCoef<T>& q, int m, int ms, T kzc, T scale, T L2half) {
    const T kz2 = kzc * (T)(ms * ms);  // k_z,m² = (π m / Lz)²
    const bool odd = (m & 1) != 0;
    // k ≠ 0: one or two screened terms (the second is zero when the partner's |k| is the same)
    const T f = fast_div(odd ? q.ao : q.ae, q.k2a + kz2) + fast_div(odd ? q.bo : q.be, q.k2b + kz2);
    // k = 0: L²/2 at m = 0, -2/k_z² for odd m, 0 for even m ≠ 0
    const T f0 = (m == 0) ? scale * L2half : (odd ? fast_div((T)-2 * scale, kz2) : (T)0);
    return q.kill ? (T)0 : (q.kzero ? f0 : f);
}

// Padded variant: each column is one length-M = 2N transform.  Thread t holds
// elements t + Tf·e of the padded column; the zero half (e ≥ E/2) never enters
// the pruned first stage, and of the inverse only the kept half (outputs < N)
// is stored, so the compiler drops the rest of the last stage.
// smem: twM[M] | green[C] | exchange of C columns of M (XchgCol)
template <typename T, int E, int N>
__global__ void __launch_bounds__(kMaxThreads, (min_blocks_zpad<T, E>())) k_z_padded(cpx<T>* __restrict__ W, const cpx<T>* __restrict__ /*unused*/,
                                                          const cpx<T>* __restrict__ twMg, const T* __restrict__ /*unused*/,
                                                          ZArgs A) {
    constexpr int M = 2 * N;
    constexpr int Tf = M / E;
    constexpr int C = zpad_cols(N, E, sizeof(T) == 8);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* twM = reinterpret_cast<cpx<T>*>(smem_raw);
    GreenT<T>* gm = reinterpret_cast<GreenT<T>*>(twM + M);
    constexpr int gm_bytes = ((C * (int)sizeof(GreenT<T>)) + 15) / 16 * 16;
    cpx<T>* xb = reinterpret_cast<cpx<T>*>(reinterpret_cast<unsigned char*>(gm) + gm_bytes);

    const int tid = threadIdx.x;
    for (int i = tid; i < M; i += blockDim.x) twM[i] = twMg[i];
    const int b = blockIdx.y;
    if (tid < C) {
        const int a = blockIdx.x * C + tid;
        GreenT<T> g = {};
        if (a < A.h) g = static_cast<const GreenT<T>*>(A.green)[(size_t)b * A.h + a];
        gm[tid] = g;
    }
    if (A.vk0 != nullptr && blockIdx.x == 0 && blockIdx.y == 0)
        mean_mode_fp64(A, N, reinterpret_cast<double*>(xb));

    const int c = tid % C, t = tid / C;
    const int a = blockIdx.x * C + c;
    const bool valid = a < A.h;
    const size_t zstride = (size_t)A.ny * A.pitch;
    const size_t step = (size_t)Tf * zstride;
    cpx<T>* col = W + (size_t)b * A.pitch + a + (size_t)t * zstride;
    cpx<T> v[1][E];
    {
        const cpx<T>* src = col;
#pragma unroll
        for (int e = 0; e < E / 2; ++e, src += step) {
            cpx<T> x = {(T)0, (T)0};
            if (valid) x = *src;
            v[0][e] = x;
        }
    }
    const XchgCol<T, C> buf[1] = {{xb + c, 0}};
    fft_static_padded<M, E, 1, T>(v, t, twM, buf);  // starts with a barrier: tables are visible

    {
        const T scale = (T)A.scale;
        const GreenCoef<T> q = green_coef<T>(gm[c], scale, A.zero_k0 != 0);
        const T kzc = (T)A.kzc;
        const T L2half = (T)(0.5 * A.L * A.L);
        // Tf is even, so every element of this thread has the parity of t.
        static_assert(Tf % 2 == 0 && (C * Tf) % 32 == 0, "padded z kernel shape");
        if (__all_sync(0xffffffffu, q.same && !q.kzero)) {
            // the common case, uniform across the warp: one screened term
            const T num = (t & 1) ? q.ao : q.ae;
            const T tf = (T)t;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                // |signed m| of m = t + Tf·e: m itself below the Nyquist index
                // (e < E/2), M - m from there on; exact small integers in T
                const T ms = (e < E / 2) ? tf + (T)(Tf * e) : (T)(M - Tf * e) - tf;
                const T f = fast_div(num, fma(kzc * ms, ms, q.k2a));
                v[0][e] = cconj_scale(v[0][e], f);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int m = t + Tf * e;
                const int ms = (m <= N) ? m : M - m;
                const T f = green_factor<T>(q, m, ms, kzc, scale, L2half);
                v[0][e] = {v[0][e].x * f, -v[0][e].y * f};
            }
        }
    }
    fft_static<M, E, 0, 1, T>(v, t, twM, buf);
    if (valid) {
        cpx<T>* dst = col;
#pragma unroll
        for (int e = 0; e < E / 2; ++e, dst += step) *dst = cconj(v[0][e]);
    }
}

// Paper-parameter variant (α = L/Lz ≠ 1, padding M = 4N): one length-4N
// transform per column, first stage pruned to the nonzero quarter, and the
// general three-case Ĝ of Eq. (Green's function regularized in Fourier):
//   k ≠ 0: -[e^{-kL}((k_z/k) sin(k_z L) - cos(k_z L)) + 1]/(k² + k_z²)
//        = -[e^{-kL}((k_z/k) sin(k_z L) + (1 - cos k_z L)) + (1 - e^{-kL})]/(k² + k_z²)
//   k = 0: table value (L²/2 at k_z = 0)
// The second form adds no cancellation of its own in FP32: 1 - e^{-kL} comes
// from expm1 and 1 - cos(k_z L) from the FP64 host tables.
// smem: twM[M] | table [2N+1][4] | green[C] | exchange of C columns (XchgCol)
template <typename T, int E, int N>
__global__ void __launch_bounds__(kMaxThreads, (min_blocks_z<T, E>())) k_z_paper(
    cpx<T>* __restrict__ W, const cpx<T>* __restrict__ /*unused*/, const cpx<T>* __restrict__ twMg,
    const T* __restrict__ /*unused*/, ZArgs A) {
    constexpr int M = 4 * N;
    constexpr int Tf = M / E;
    constexpr int C = zpad_cols(2 * N, E, sizeof(T) == 8);  // same rule with 2·(2N) per column
    constexpr int NT = 2 * N + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* twM = reinterpret_cast<cpx<T>*>(smem_raw);
    T* tab = reinterpret_cast<T*>(twM + M);  // per |m|: k_z sin(k_z L), 1 - cos(k_z L), k_z², Ĝ(0, k_z)
    constexpr int tab_bytes = (4 * NT * (int)sizeof(T) + 15) / 16 * 16;
    GreenT<T>* gm = reinterpret_cast<GreenT<T>*>(reinterpret_cast<unsigned char*>(tab) + tab_bytes);
    constexpr int gm_bytes = ((C * (int)sizeof(GreenT<T>)) + 15) / 16 * 16;
    cpx<T>* xb = reinterpret_cast<cpx<T>*>(reinterpret_cast<unsigned char*>(gm) + gm_bytes);

    const int tid = threadIdx.x;
    for (int i = tid; i < M; i += blockDim.x) twM[i] = twMg[i];
    const T* ptab = static_cast<const T*>(A.paper_tab);
    for (int i = tid; i < 4 * NT; i += blockDim.x) tab[i] = ptab[i];
    const int b = blockIdx.y;
    if (tid < C) {
        const int a = blockIdx.x * C + tid;
        GreenT<T> g = {};
        g.kzero = 1;  // columns past the half spectrum: finite, never stored
        g.same = 1;
        if (a < A.h) g = static_cast<const GreenT<T>*>(A.green)[(size_t)b * A.h + a];
        gm[tid] = g;
    }
    if (A.vk0 != nullptr && blockIdx.x == 0 && blockIdx.y == 0)
        mean_mode_fp64(A, N, reinterpret_cast<double*>(xb));

    const int c = tid % C, t = tid / C;
    const int a = blockIdx.x * C + c;
    const bool valid = a < A.h;
    const size_t zstride = (size_t)A.ny * A.pitch;
    const size_t step = (size_t)Tf * zstride;
    cpx<T>* col = W + (size_t)b * A.pitch + a + (size_t)t * zstride;
    cpx<T> v[1][E];
    {
        const cpx<T>* src = col;
#pragma unroll
        for (int e = 0; e < E / 4; ++e, src += step) {
            cpx<T> x = {(T)0, (T)0};
            if (valid) x = *src;
            v[0][e] = x;
        }
    }
    const XchgCol<T, C> buf[1] = {{xb + c, 0}};
    fft_static_quarter<M, E, 1, T>(v, t, twM, buf);  // starts with a barrier: tables are visible

    {
        const GreenT<T> g = gm[c];
        const T scale = (T)A.scale;
        // numerator = A1·(k_z sin k_z L) + A2·(1 - cos k_z L) + A3 per branch
        const T Ea = (T)1 - g.omEa, Eb = (T)1 - g.omEb;  // e^{-kL}
        const T ika = g.kzero ? (T)0 : rsqrt(g.k2a);
        const T ikb = g.kzero ? (T)0 : rsqrt(g.k2b);
        const T wb = g.same ? (T)0 : (T)0.5, wa = (T)1 - wb;
        const T a1 = -scale * wa * Ea * ika, a2 = -scale * wa * Ea, a3 = -scale * wa * g.omEa;
        const T b1 = -scale * wb * Eb * ikb, b2 = -scale * wb * Eb, b3 = -scale * wb * g.omEb;
        const bool kill = A.zero_k0 && g.kzero;
        // warp-uniform fast path: every lane's mode is its own partner and k ≠ 0
        if (__all_sync(0xffffffffu, g.same && !g.kzero)) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int m = t + Tf * e;
                const int ms = (m <= 2 * N) ? m : M - m;  // |signed m|
                const T* q = tab + 4 * ms;
                const T f = fast_div(fma(a1, q[0], fma(a2, q[1], a3)), g.k2a + q[2]);
                v[0][e] = {v[0][e].x * f, -v[0][e].y * f};
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int m = t + Tf * e;
                const int ms = (m <= 2 * N) ? m : M - m;
                const T* q = tab + 4 * ms;
                T f;
                if (g.kzero) {
                    f = kill ? (T)0 : scale * q[3];
                } else {
                    f = fast_div(fma(a1, q[0], fma(a2, q[1], a3)), g.k2a + q[2]) +
                        fast_div(fma(b1, q[0], fma(b2, q[1], b3)), g.k2b + q[2]);
                }
                v[0][e] = {v[0][e].x * f, -v[0][e].y * f};
            }
        }
    }
    fft_static<M, E, 0, 1, T>(v, t, twM, buf);
    if (valid) {
        cpx<T>* dst = col;
#pragma unroll
        for (int e = 0; e < E / 4; ++e, dst += step) *dst = cconj(v[0][e]);
    }
}

// ---------------------------------------------------------------------------
// x inverse: C row pairs per block, lanes along x.  Each thread assembles
// Z[k] = X0[k] + i X1[k] (Hermitian extension above nx/2) straight from
// global memory and stores its real outputs straight back.  Optional FP64
// mean-mode add (A.vk0 != null).
// smem: tw[n] | C padded rows (exchange)
// ---------------------------------------------------------------------------
template <typename T, int E, int NS>
__global__ void __launch_bounds__(kMaxThreads, (min_blocks_xs<T, E, NS>())) k_x_inverse(const cpx<T>* __restrict__ W, T* __restrict__ phi,
                                                           const cpx<T>* __restrict__ twg, XArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = NS > 0 ? NS : A.P.n, C = A.C, Tf = NS > 0 ? NS / E : A.P.Tf;
    const int RP = padded_row(n);
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* xb = tw + n;
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) tw[i] = twg[i];

    const int t = tid % Tf, c = tid / Tf;
    const long long pair0 = (long long)blockIdx.x * C;
    const long long row = 2 * (pair0 + c);
    const cpx<T>* w0 = W + row * A.pitch;
    const cpx<T>* w1 = w0 + A.pitch;
    cpx<T> v[1][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + Tf * e;
        cpx<T> z;
        if (2 * k <= n) {
            cpx<T> x0 = w0[k], x1 = w1[k];
            if (k == 0 || 2 * k == n) {
                x0.y = (T)0;
                x1.y = (T)0;
            }
            z = {x0.x - x1.y, x0.y + x1.x};
        } else {
            const cpx<T> x0 = w0[n - k], x1 = w1[n - k];
            z = {x0.x + x1.y, x1.x - x0.y};
        }
        v[0][e] = cconj(z);
    }
    __syncthreads();  // twiddles visible
    const SmemRow<T> buf[1] = {{xb + c * RP, 0}};
    fft_run<NS, E, 1, T>(v, t, A.P, tw, buf);

    // mean mode (FP32 path): the FP64 per-plane value, added as a double-float pair
    T add_hi = (T)0, add_lo = (T)0;
    const bool addk0 = (A.vk0 != nullptr);
    if (addk0) {
        const double vv = A.vk0[pair0 / A.pairs_per_plane];
        add_hi = (T)vv;
        add_lo = (T)(vv - (double)add_hi);
    }
    T* o0 = phi + row * n;
    T* o1 = o0 + n;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int x = t + Tf * e;
        T p0 = v[0][e].x, p1 = -v[0][e].y;  // conj of the forward result
        if (addk0) {
            if constexpr (sizeof(T) == 4) {
                // TwoSum of (p0, p1) + hi, then + lo, on both rows at once as
                // packed pairs: the same operations and roundings as the
                // scalar form, in half the instructions
                const cpx<float> a = {p0, p1}, hh = {add_hi, add_hi}, ll = {add_lo, add_lo};
                const cpx<float> sm = cadd(a, hh);
                const cpx<float> bb = csub(sm, a);
                const cpx<float> er = cadd(csub(a, csub(sm, bb)), csub(hh, bb));
                const cpx<float> r = cadd(sm, cadd(er, ll));
                p0 = r.x;
                p1 = r.y;
            } else {
                p0 = p0 + add_hi;
                p1 = p1 + add_hi;
            }
        }
        __stcs(o0 + x, p0);
        __stcs(o1 + x, p1);
    }
}

// Standalone Green's-table fill (used when the z pass runs on its own).
template <typename T>
__global__ void k_green_params(GreenFill gf) {
    green_fill<T>(gf, blockIdx.x);
}

}  // namespace sbp
