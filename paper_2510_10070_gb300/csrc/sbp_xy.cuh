// sbp_xy.cuh — fused x and y passes: one z-plane per thread-block cluster.
//
// Forward: each CTA of a cluster of CL transforms N/CL rows of the plane
// along x (row pairs, as k_x_forward) and stores every result straight into
// the shared memory of the CTA that owns its column (distributed shared
// memory stores, which do not wait); the cluster synchronises, and each CTA
// then transforms its share of the nx/2+1 half-spectrum columns along y from
// its own shared memory and writes the spectrum.  The inverse runs the same
// two phases in the opposite order, pushing each y-transformed element to the
// CTA that owns its row.  The half spectrum of a plane goes
// through HBM once per direction instead of twice.
#pragma once

#include <cooperative_groups.h>

#include "sbp_kernels.cuh"

namespace sbp {

namespace cg = cooperative_groups;

struct XYArgs {
    int pitch;          // spectrum row pitch (complex elements)
    int green_ctas;     // forward: leading CTAs that fill the Green's table
    GreenFill gf;
    double* tile_sums;  // forward, FP32: per (plane, CTA) Σρ; null: none
    const double* vk0;  // inverse, FP32: mean-mode potential per plane; null: none
};

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
// Largest divisor of n that is at most cap.
__host__ __device__ constexpr int divisor_at_most(int n, int cap) {
    int d = cap < n ? cap : n;
    while (d > 1 && n % d != 0) --d;
    return d < 1 ? 1 : d;
}

// Compile-time shape of a fused plane kernel (square planes nx = ny = N).
template <typename T, int N, int CL>
struct XYShape {
    static constexpr bool F64 = sizeof(T) == 8;
    static constexpr int E = plan_E(N, F64);
    static constexpr int TF = N / E;                           // threads per transform
    static constexpr int H = N / 2 + 1;                        // stored columns
    static constexpr int ROWS = N / CL;                        // rows per CTA
    static constexpr int PAIRS = ROWS / 2;
    static constexpr int CX = divisor_at_most(PAIRS, kMaxThreads / TF);  // row pairs per round
    static constexpr int NT = CX * TF;                         // threads per CTA
    static constexpr int CY = CX;                              // columns per round
    static constexpr int ACOLS = (H + CL - 1) / CL;            // columns per CTA
    static constexpr int RP = padded_row(N);
    static constexpr int S_FWD = N * ACOLS;                    // forward: all rows, own columns
    static constexpr int S_INV = ROWS * H;                     // inverse: own rows, all columns
    static constexpr int XBUF = cmax(CX * RP, N * xstride(CY));
    static constexpr size_t smem_fwd = (size_t)(S_FWD + N + XBUF) * sizeof(cpx<T>);
    static constexpr size_t smem_inv = (size_t)(S_INV + N + XBUF) * sizeof(cpx<T>);
    static_assert(ROWS % 2 == 0 || CL > N / 2, "each CTA holds whole row pairs");
};

// Smallest power-of-two cluster whose CTAs fit their share of the plane in
// `limit` bytes of shared memory (about 200 KB: one CTA per SM; about 110 KB:
// two CTAs per SM, so that one CTA's memory phase overlaps another's compute).
template <typename T, int N, size_t LIMIT>
constexpr int xy_cluster() {
    return XYShape<T, N, 1>::smem_fwd <= LIMIT && XYShape<T, N, 1>::smem_inv <= LIMIT   ? 1
           : XYShape<T, N, 2>::smem_fwd <= LIMIT && XYShape<T, N, 2>::smem_inv <= LIMIT ? 2
           : XYShape<T, N, 4>::smem_fwd <= LIMIT && XYShape<T, N, 4>::smem_inv <= LIMIT ? 4
                                                                                         : 8;
}
constexpr size_t kXYSmemOnePerSM = 200 * 1024;
constexpr size_t kXYSmemTwoPerSM = 110 * 1024;

template <typename T, int N, int CL>
__global__ void __launch_bounds__(kMaxThreads) k_xy_forward(const T* __restrict__ rho, cpx<T>* __restrict__ W,
                                                               const cpx<T>* __restrict__ twg, XYArgs A) {
    using SH = XYShape<T, N, CL>;
    constexpr int E = SH::E, TF = SH::TF, H = SH::H;
    if ((int)blockIdx.x < A.green_ctas) {  // FP64 Green's table, off the transform CTAs
        green_fill<T>(A.gf, blockIdx.x);
        return;
    }
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int plane = ((int)blockIdx.x - A.green_ctas) / CL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);  // [N][ACOLS]: all rows, own columns
    cpx<T>* tw = S + SH::S_FWD;
    cpx<T>* xb = tw + N;
    const int tid = threadIdx.x;
    for (int i = tid; i < N; i += blockDim.x) tw[i] = twg[i];
    cpx<T>* dst[CL];
#pragma unroll
    for (int r = 0; r < CL; ++r) dst[r] = cluster.map_shared_rank(S, r);
    cluster.sync();  // every CTA has started before any writes into it; twiddles visible

    // ---- phase 1: x transforms of this CTA's row pairs, pushed to the column owners
    FF acc = {0.f, 0.f};
    {
        const int t = tid % TF, c = tid / TF;
        const T half = (T)0.5;
        for (int p0 = 0; p0 < SH::PAIRS; p0 += SH::CX) {
            const int p = p0 + c;
            const T* r0p = rho + ((size_t)plane * N + (size_t)rank * SH::ROWS + 2 * p) * N;
            cpx<T> v[1][E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = t + TF * e;
                v[0][e] = {__ldcs(r0p + x), __ldcs(r0p + N + x)};
                if constexpr (sizeof(T) == 4) {
                    kahan_add(acc, (float)v[0][e].x);
                    kahan_add(acc, (float)v[0][e].y);
                }
            }
            const SmemRow<T> buf[1] = {{xb + c * SH::RP, 0}};
            fft_static<N, E, 0, 1, T>(v, t, tw, buf);
            __syncthreads();  // exchange reads done before Z overwrites it
#pragma unroll
            for (int e = 0; e < E; ++e) buf[0][t + TF * e] = v[0][e];
            __syncthreads();
            for (int q = tid; q < SH::CX * H; q += blockDim.x) {
                const int cc = q / H, k = q - cc * H;
                const cpx<T>* zr = xb + cc * SH::RP;
                const cpx<T> Az = zr[k + (k >> 4)];
                const int km = (k == 0) ? 0 : N - k;
                const cpx<T> Bz = cconj(zr[km + (km >> 4)]);
                const int y = rank * SH::ROWS + 2 * (p0 + cc);
                const int owner = k / SH::ACOLS, ka = k - owner * SH::ACOLS;
                cpx<T>* o = dst[owner] + (size_t)y * SH::ACOLS + ka;
                o[0] = {(Az.x + Bz.x) * half, (Az.y + Bz.y) * half};
                o[SH::ACOLS] = {(Az.y - Bz.y) * half, (Bz.x - Az.x) * half};
            }
            // the next round's first exchange write is preceded by a barrier
        }
    }
    if constexpr (sizeof(T) == 4) {
        if (A.tile_sums != nullptr) {
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
            if (tid == 0) {
                FF tot = {0.f, 0.f};
                for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot = ff_add(tot, wsum[w]);
                A.tile_sums[(size_t)plane * CL + rank] = (double)tot.hi + (double)tot.lo;
            }
        }
    }
    cluster.sync();  // every CTA's columns are in its shared memory

    // ---- phase 2: y transforms of this CTA's columns, from its own shared memory
    {
        const int c = tid % SH::CY, t = tid / SH::CY;
        const int a_begin = rank * SH::ACOLS, a_end = cmin(H, a_begin + SH::ACOLS);
        cpx<T>* wplane = W + (size_t)plane * N * A.pitch;
        for (int a0 = a_begin; a0 < a_end; a0 += SH::CY) {
            const int a = a0 + c;
            const bool valid = a < a_end;
            cpx<T> v[1][E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int y = t + TF * e;
                v[0][e] = valid ? S[(size_t)y * SH::ACOLS + (a - a_begin)] : cpx<T>{(T)0, (T)0};
            }
            const SmemCol<T, xstride(SH::CY)> buf[1] = {{xb + c, 0}};
            fft_static<N, E, 0, 1, T>(v, t, tw, buf);
            if (valid) {
#pragma unroll
                for (int e = 0; e < E; ++e) wplane[(size_t)(t + TF * e) * A.pitch + a] = v[0][e];
            }
        }
    }
    cluster.sync();  // no CTA leaves before the others' pushes into it are consumed
}

template <typename T, int N, int CL>
__global__ void __launch_bounds__(kMaxThreads) k_xy_inverse(const cpx<T>* __restrict__ W, T* __restrict__ phi,
                                                               const cpx<T>* __restrict__ twg, XYArgs A) {
    using SH = XYShape<T, N, CL>;
    constexpr int E = SH::E, TF = SH::TF, H = SH::H;
    constexpr int AC = SH::ACOLS;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int plane = (int)blockIdx.x / CL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);  // [ROWS][H]: own rows, all columns
    cpx<T>* tw = S + SH::S_INV;
    cpx<T>* xb = tw + N;
    const int tid = threadIdx.x;
    for (int i = tid; i < N; i += blockDim.x) tw[i] = twg[i];
    cpx<T>* dst[CL];
#pragma unroll
    for (int r = 0; r < CL; ++r) dst[r] = cluster.map_shared_rank(S, r);
    cluster.sync();  // every CTA has started before any writes into it; twiddles visible

    // ---- phase 1: y inverse of this CTA's columns, pushed to the row owners
    const int a_begin = rank * AC, a_end = cmin(H, a_begin + AC);
    {
        const int c = tid % SH::CY, t = tid / SH::CY;
        const cpx<T>* wplane = W + (size_t)plane * N * A.pitch;
        for (int a0 = a_begin; a0 < a_end; a0 += SH::CY) {
            const int a = a0 + c;
            const bool valid = a < a_end;
            cpx<T> v[1][E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                cpx<T> x = {(T)0, (T)0};
                if (valid) x = wplane[(size_t)(t + TF * e) * A.pitch + a];
                v[0][e] = cconj(x);
            }
            const SmemCol<T, xstride(SH::CY)> buf[1] = {{xb + c, 0}};
            fft_static<N, E, 0, 1, T>(v, t, tw, buf);
            if (valid) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int y = t + TF * e;
                    const int owner = y / SH::ROWS;
                    dst[owner][(size_t)(y - owner * SH::ROWS) * H + a] = cconj(v[0][e]);
                }
            }
        }
    }
    cluster.sync();  // every CTA's rows are in its shared memory

    // ---- phase 2: x inverse of this CTA's row pairs, from its own shared memory
    {
        T add_hi = (T)0, add_lo = (T)0;
        const bool addk0 = (A.vk0 != nullptr);
        if (addk0) {
            const double vv = A.vk0[plane];
            add_hi = (T)vv;
            add_lo = (T)(vv - (double)add_hi);
        }
        const int t = tid % TF, c = tid / TF;
        for (int p0 = 0; p0 < SH::PAIRS; p0 += SH::CX) {
            const int y0 = rank * SH::ROWS + 2 * (p0 + c);
            const int yl = 2 * (p0 + c);  // local row
            cpx<T> v[1][E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = t + TF * e;
                const int kk = (2 * k <= N) ? k : N - k;
                cpx<T> x0 = S[(size_t)yl * H + kk], x1 = S[(size_t)(yl + 1) * H + kk];
                cpx<T> z;
                if (2 * k <= N) {
                    if (k == 0 || 2 * k == N) {
                        x0.y = (T)0;
                        x1.y = (T)0;
                    }
                    z = {x0.x - x1.y, x0.y + x1.x};
                } else {
                    z = {x0.x + x1.y, x1.x - x0.y};
                }
                v[0][e] = cconj(z);
            }
            const SmemRow<T> buf[1] = {{xb + c * SH::RP, 0}};
            fft_static<N, E, 0, 1, T>(v, t, tw, buf);
            T* o0 = phi + ((size_t)plane * N + y0) * N;
            T* o1 = o0 + N;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = t + TF * e;
                T p0v = v[0][e].x, p1v = -v[0][e].y;
                if (addk0) {
                    if constexpr (sizeof(T) == 4) {
                        float s, er;
                        two_sum(p0v, add_hi, s, er);
                        p0v = s + (er + add_lo);
                        two_sum(p1v, add_hi, s, er);
                        p1v = s + (er + add_lo);
                    } else {
                        p0v = p0v + add_hi;
                        p1v = p1v + add_hi;
                    }
                }
                __stcs(o0 + x, p0v);
                __stcs(o1 + x, p1v);
            }
        }
    }
    cluster.sync();  // keeps the cluster together to the end, as in the forward kernel
}

}  // namespace sbp
