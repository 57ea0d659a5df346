// sbp_remap.cuh — solves in the physical (shearing) frame.
//
// Sect. 2.1 maps the density to the periodic frame, ρ̃(x, y) = ρ(x, y - s x)
// with s = Δy0/L_x, solves there and maps the potential back,
// Φ(x, y) = Φ̃(x, y + s x).  The spectral form of the mapping is a phase
// exp(∓i K_y s x) on the y-spectrum of each x-column (Fourier interpolation;
// the Nyquist coefficient takes the real part of its phase, so columns stay
// real).  Here the y transforms run first, with the phases fused in, and the
// x transforms second; the solve keeps five passes:
//
//   k_ry_forward   real y-columns (two per complex transform) → y half
//                  spectrum, phase exp(-i K_y s x), FP64 Green's table blocks,
//                  plane sums for the FP64 mean mode (FP32 path, SASHA)
//   k_rows_c2c     complex x-rows, forward
//   z pass         unchanged (it reads the Green's table per stored mode)
//   k_rows_c2c     complex x-rows, inverse
//   k_ry_inverse   phase exp(+i K_y s x), y half spectrum → real y-columns
//
// Spectrum layout in this mode: V[z][b][a] with b ∈ [0, ny/2] the y-frequency
// and a ∈ [0, nx) the x-frequency, row pitch nx complex values.
//
// x is the cell centre -L_x/2 + (i + ½) dx.  The phase of column x at
// y-frequency k is 2π k u_x with u_x = (s/L_y) x = (s L_x/L_y)(x/L_x); it is
// reduced exactly through a fixed-point turn count: U = frac(u_x)·2^B and
// (k U mod 2^B)/2^B = frac(k u_x) (B = 32 in FP32, 64 in FP64), so the angle
// never exceeds π in magnitude before sincos.
#pragma once

#include "sbp_kernels.cuh"

namespace sbp {

struct RArgs {
    int nx, ny;           // box
    int pitch;            // spectrum row pitch (complex values), = nx
    int pairs;            // nx / 2 column pairs
    int tiles;            // pair tiles per plane in the y kernels
    int green_blocks;     // leading blocks of k_ry_forward that fill the Green's table
    GreenFill gf;
    double s;             // s = Δy0 / L_x
    const double* s_dev;  // if set, s is read from device memory (batched executor)
    double lx_over_ly;    // L_x / L_y
    const double* vk0;    // FP64 mean mode per plane, added by k_ry_inverse (or null)
};

// Turn fraction u of column x (cell centre) as a fixed-point count.
template <typename T>
struct TurnFix;
template <>
struct TurnFix<float> {
    using U = uint32_t;
    static __device__ __forceinline__ U from(double u) {
        const double f = u - floor(u);
        return (U)(unsigned long long)llrint(f * 4294967296.0);  // 2^32 wraps to 0
    }
    // e^{i·2π·frac(k u)}
    static __device__ __forceinline__ cpx<float> phase(int k, U u) {
        const uint32_t ph = (uint32_t)k * u;
        const float th = (float)(int32_t)ph * 1.46291807926715968e-9f;  // 2π / 2^32
        float sn, cs;
        __sincosf(th, &sn, &cs);
        return {cs, sn};
    }
};
template <>
struct TurnFix<double> {
    using U = unsigned long long;
    static __device__ __forceinline__ U from(double u) {
        const double f = u - floor(u);
        const double hi = floor(f * 4294967296.0);         // exact: scaling by 2^32
        const double r = f * 4294967296.0 - hi;            // exact
        const U lo = (U)llrint(r * 4294967296.0);          // ≤ 2^32
        return ((U)hi << 32) + lo;
    }
    static __device__ __forceinline__ cpx<double> phase(int k, U u) {
        const U ph = (U)k * u;
        const double f = (double)(long long)ph * 5.42101086242752217e-20;  // 2^-64: f ∈ [-½, ½)
        double sn, cs;
        sincospi(2.0 * f, &sn, &cs);
        return {cs, sn};
    }
};

__device__ __forceinline__ double column_turns(double sig, int x, int nx) {
    return sig * (((double)x + 0.5) / (double)nx - 0.5);
}

// Forward y pass with the mapping to the periodic frame.  Block = CP column
// pairs (x = 2p, 2p+1) of one z-plane; column pair p is one complex
// transform z = ρ(x_a) + i ρ(x_b), split afterwards with
// A_k = (Z_k + conj Z_{N-k})/2, B_k = -i (Z_k - conj Z_{N-k})/2.
// smem: tw[NY] | exchange (XchgCol)
template <typename T, int E, int NY, int CP>
__global__ void __launch_bounds__(kMaxThreads, (NY >= 64 ? min_blocks_xs<T, E, NY>() : min_blocks_xy<T, E>()))
    k_ry_forward(const T* __restrict__ rho, cpx<T>* __restrict__ V, const cpx<T>* __restrict__ twg,
                 double* __restrict__ tile_sums, RArgs A) {
    if ((int)blockIdx.x < A.green_blocks) {  // Green's table, off the transform blocks
        green_fill<T>(A.gf, blockIdx.x);
        return;
    }
    const int bid = blockIdx.x - A.green_blocks;
    const int z = bid / A.tiles, tile = bid - z * A.tiles;
    constexpr int Tf = NY / E;
    constexpr int H = NY / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* xb = tw + NY;
    const int tid = threadIdx.x;
    for (int i = tid; i < NY; i += blockDim.x) tw[i] = twg[i];

    const int c = tid % CP, t = tid / CP;
    const int p = tile * CP + c;
    const bool valid = p < A.pairs;
    const size_t step = (size_t)Tf * A.nx;
    cpx<T> v[1][E];
    {
        const T* src = rho + ((size_t)z * NY + t) * A.nx + 2 * p;
#pragma unroll
        for (int e = 0; e < E; ++e, src += step) {
            cpx<T> x = {(T)0, (T)0};
            if (valid) x = *reinterpret_cast<const cpx<T>*>(src);
            v[0][e] = x;
        }
    }
    if constexpr (sizeof(T) == 4) {
        if (tile_sums != nullptr) {
            FF acc = {0.f, 0.f};
#pragma unroll
            for (int e = 0; e < E; ++e) {
                kahan_add(acc, (float)v[0][e].x);
                kahan_add(acc, (float)v[0][e].y);
            }
            const FF tot = block_sum_ff(acc);
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
    const XchgCol<T, CP> buf[1] = {{xb + c, 0}};
    fft_static<NY, E, 0, 1, T>(v, t, tw, buf);  // Z_k at k = t + Tf·e
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) buf[0][t + Tf * e] = v[0][e];
    __syncthreads();
    if (!valid) return;

    const double s = A.s_dev != nullptr ? *A.s_dev : A.s;
    const double sig = s * A.lx_over_ly;
    const typename TurnFix<T>::U ua = TurnFix<T>::from(column_turns(sig, 2 * p, A.nx));
    const typename TurnFix<T>::U ub = TurnFix<T>::from(column_turns(sig, 2 * p + 1, A.nx));
    const T half = (T)0.5;
#pragma unroll
    for (int e = 0; e <= E / 2; ++e) {
        const int k = t + Tf * e;
        if (k > H) break;
        const cpx<T> Zk = v[0][e];
        const cpx<T> Zm = cconj(buf[0][k == 0 ? 0 : NY - k]);
        cpx<T> a = {(Zk.x + Zm.x) * half, (Zk.y + Zm.y) * half};
        cpx<T> b = {(Zk.y - Zm.y) * half, (Zm.x - Zk.x) * half};
        const cpx<T> wa = TurnFix<T>::phase(k, ua), wb = TurnFix<T>::phase(k, ub);
        if (k == H) {  // Nyquist: real coefficient times the real part of its phase
            a = {a.x * wa.x, (T)0};
            b = {b.x * wb.x, (T)0};
        } else {  // exp(-i K_y s x)
            a = cmul(a, cconj(wa));
            b = cmul(b, cconj(wb));
        }
        cpx<T>* dst = V + ((size_t)z * (H + 1) + k) * A.pitch + 2 * p;
        dst[0] = a;
        dst[1] = b;
    }
}

// In-place c2c transforms of contiguous complex rows (x-frequency), forward
// or unnormalised inverse.  Block = C rows; lanes along the row.
// smem: tw[NX] | C padded rows
template <typename T, int E, int NX, bool INV>
__global__ void __launch_bounds__(kMaxThreads, (min_blocks_xs<T, E, NX>()))
    k_rows_c2c(cpx<T>* __restrict__ V, const cpx<T>* __restrict__ twg, int rows, int pitch) {
    constexpr int Tf = NX / E;
    constexpr int C = kMaxThreads / Tf;
    constexpr int RP = padded_row(NX);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* xb = tw + NX;
    const int tid = threadIdx.x;
    for (int i = tid; i < NX; i += blockDim.x) tw[i] = twg[i];
    const int t = tid % Tf, c = tid / Tf;
    const long long row = (long long)blockIdx.x * C + c;
    const bool valid = row < rows;
    cpx<T>* r = V + row * pitch;
    cpx<T> v[1][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        cpx<T> x = {(T)0, (T)0};
        if (valid) x = r[t + Tf * e];
        v[0][e] = INV ? cconj(x) : x;
    }
    __syncthreads();  // twiddles visible
    const SmemRow<T> buf[1] = {{xb + c * RP, 0}};
    fft_static<NX, E, 0, 1, T>(v, t, tw, buf);
    if (valid) {
#pragma unroll
        for (int e = 0; e < E; ++e) r[t + Tf * e] = INV ? cconj(v[0][e]) : v[0][e];
    }
}

// Inverse y pass with the mapping back to the physical frame: phase
// exp(+i K_y s x) on the y half spectra of columns x_a, x_b (real parts at
// b = 0 and at the Nyquist row), Hermitian extension, one complex inverse
// transform per pair, φ(x_a) = Re, φ(x_b) = Im; the FP32 path adds the FP64
// mean mode of the plane.  smem: tw[NY] | exchange (XchgCol)
template <typename T, int E, int NY, int CP>
__global__ void __launch_bounds__(kMaxThreads, (NY >= 64 ? min_blocks_xs<T, E, NY>() : min_blocks_xy<T, E>()))
    k_ry_inverse(const cpx<T>* __restrict__ V, T* __restrict__ phi, const cpx<T>* __restrict__ twg, RArgs A) {
    const int bid = blockIdx.x;
    const int z = bid / A.tiles, tile = bid - z * A.tiles;
    constexpr int Tf = NY / E;
    constexpr int H = NY / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* xb = tw + NY;
    const int tid = threadIdx.x;
    for (int i = tid; i < NY; i += blockDim.x) tw[i] = twg[i];

    const int c = tid % CP, t = tid / CP;
    const int p = tile * CP + c;
    const bool valid = p < A.pairs;
    const double s = A.s_dev != nullptr ? *A.s_dev : A.s;
    const double sig = s * A.lx_over_ly;
    const typename TurnFix<T>::U ua = TurnFix<T>::from(column_turns(sig, 2 * p, A.nx));
    const typename TurnFix<T>::U ub = TurnFix<T>::from(column_turns(sig, 2 * p + 1, A.nx));
    cpx<T> v[1][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + Tf * e;
        const int kk = (k <= H) ? k : NY - k;
        cpx<T> a = {(T)0, (T)0}, b = {(T)0, (T)0};
        if (valid) {
            const cpx<T>* src = V + ((size_t)z * (H + 1) + kk) * A.pitch + 2 * p;
            a = src[0];
            b = src[1];
        }
        const cpx<T> wa = TurnFix<T>::phase(kk, ua), wb = TurnFix<T>::phase(kk, ub);
        a = cmul(a, wa);
        b = cmul(b, wb);
        if (kk == 0 || kk == H) {
            a.y = (T)0;
            b.y = (T)0;
        }
        if (k > H) {
            a = cconj(a);
            b = cconj(b);
        }
        v[0][e] = cconj(cpx<T>{a.x - b.y, a.y + b.x});  // inverse through the forward transform
    }
    __syncthreads();  // twiddles visible
    const XchgCol<T, CP> buf[1] = {{xb + c, 0}};
    fft_static<NY, E, 0, 1, T>(v, t, tw, buf);
    if (!valid) return;

    T add_hi = (T)0, add_lo = (T)0;
    const bool addk0 = (A.vk0 != nullptr);
    if (addk0) {
        const double vv = A.vk0[z];
        add_hi = (T)vv;
        add_lo = (T)(vv - (double)add_hi);
    }
    T* out = phi + ((size_t)z * NY + t) * A.nx + 2 * p;
    const size_t step = (size_t)Tf * A.nx;
#pragma unroll
    for (int e = 0; e < E; ++e, out += step) {
        T p0 = v[0][e].x, p1 = -v[0][e].y;  // conj of the forward result
        if (addk0) {
            if constexpr (sizeof(T) == 4) {
                float sm, er;
                two_sum(p0, add_hi, sm, er);
                p0 = sm + (er + add_lo);
                two_sum(p1, add_hi, sm, er);
                p1 = sm + (er + add_lo);
            } else {
                p0 = p0 + add_hi;
                p1 = p1 + add_hi;
            }
        }
        *reinterpret_cast<cpx<T>*>(out) = cpx<T>{p0, p1};
    }
}

}  // namespace sbp
