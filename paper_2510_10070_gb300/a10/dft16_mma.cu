// dft16_mma.cu — measurement behind the "tensor-core radix-16 stage" option:
// a batch of 16-point complex DFTs, the radix-16 butterfly of every
// transform pass, computed three ways on one GB300 and timed with CUDA
// events, with the error of each against an FP64 DFT on the host.
//
//   cc_reg   the FFT engine's FP32 butterfly (Dft<16>), data kept in registers
//            across repetitions: the cost inside a pass, where the data already
//            sits in the threads' registers;
//   cc_smem  the same butterfly with a shared-memory round trip per repetition;
//   mma3     the DFT as a dense contraction on the tensor cores: with
//            X = [Re x; Im x], Re y = [Re F | -Im F] X and Im y = [Im F | Re F] X,
//            each a 16×32 by 32×8 product for 8 transforms; operands split as
//            a = hi + lo in FP16, three products hi·hi + hi·lo + lo·hi
//            accumulated in FP32 (mma.sync m16n8k16), 12 MMAs per 8 transforms,
//            the data moved between shared memory and fragments each repetition
//            (as it would have to be inside a pass);
//   mma1     the hi·hi product alone (the error before the split recovery);
//   mma3_bf16, mma1_bf16   the same two with the operands split in BF16
//            (mma.sync m16n8k16 .bf16.bf16: 8 mantissa bits instead of 11,
//            FP32's exponent range).
//
// Build and run through `python -m paper_2510_10070_gb300.a10.run`; prints one
// JSON line.  Not part of the library: it only measures whether the option
// pays.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../csrc/sbp_fft.cuh"

using sbp::cpx;

constexpr int kThreads = 256;     // one transform per thread (cc), 32 per warp (mma)
constexpr int kTile = kThreads;   // transforms per block
constexpr int kStride = kTile + 4;  // padded row of the [16][tile] planes (conflict-free fragments)

// x = hi + lo with hi = h(x), lo = h(x - hi), h = FP16 or BF16 rounding;
// two values packed per 32-bit fragment register (first in the low half)
template <bool BF>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if constexpr (BF) {
        const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
        const float ra = a - __bfloat162float(ha), rb = b - __bfloat162float(hb);
        __nv_bfloat162 h = __halves2bfloat162(ha, hb);
        __nv_bfloat162 l = __floats2bfloat162_rn(ra, rb);
        hi = *reinterpret_cast<uint32_t*>(&h);
        lo = *reinterpret_cast<uint32_t*>(&l);
    } else {
        const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
        const float ra = a - __half2float(ha), rb = b - __half2float(hb);
        __half2 h = __halves2half2(ha, hb);
        __half2 l = __floats2half2_rn(ra, rb);
        hi = *reinterpret_cast<uint32_t*>(&h);
        lo = *reinterpret_cast<uint32_t*>(&l);
    }
}

// D += A·B, A and B of the same 16-bit type (FP16 or BF16), FP32 accumulate
template <bool BF>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (BF) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// In-place DFTs of the block's tile, reps times; data as planes re[16][kStride], im[16][kStride].
template <int MODE>  // 0: cc_reg, 1: cc_smem, 2: mma3, 3: mma1, 4: mma3_bf16, 5: mma1_bf16
__global__ void __launch_bounds__(kThreads) k_dft16(float* __restrict__ data, int reps) {
    constexpr bool BF = (MODE >= 4);
    constexpr bool THREE = (MODE == 2 || MODE == 4);
    __shared__ float re[16 * kStride], im[16 * kStride];
    const int tid = threadIdx.x;
    float* blk = data + (size_t)blockIdx.x * kTile * 32;  // [tile][16] complex, interleaved
    for (int i = tid; i < kTile * 16; i += kThreads) {
        const int col = i / 16, k = i % 16;
        re[k * kStride + col] = blk[2 * i];
        im[k * kStride + col] = blk[2 * i + 1];
    }
    __syncthreads();
    if constexpr (MODE == 0 || MODE == 1) {
        cpx<float> x[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = {re[k * kStride + tid], im[k * kStride + tid]};
        for (int r = 0; r < reps; ++r) {
            sbp::Dft<16, float>::run(x);
            if constexpr (MODE == 1) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    re[k * kStride + tid] = x[k].x;
                    im[k * kStride + tid] = x[k].y;
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 16; ++k) x[k] = {re[k * kStride + tid], im[k * kStride + tid]};
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            re[k * kStride + tid] = x[k].x;
            im[k * kStride + tid] = x[k].y;
        }
    } else {
        const int lane = tid & 31, warp = tid >> 5;
        const int g = lane >> 2, t = lane & 3;
        // A fragments of Re F, Im F, -Im F (hi and lo), F[m][k] = e^{-2πi mk/16}
        uint32_t fr_h[4], fr_l[4], fi_h[4], fi_l[4], fn_h[4], fn_l[4];
        {
            auto fre = [](int m, int k) { return (float)cospi(-2.0 * ((m * k) % 16) / 16.0); };
            auto fim = [](int m, int k) { return (float)sinpi(-2.0 * ((m * k) % 16) / 16.0); };
            const int rows[4] = {g, g + 8, g, g + 8}, cols[4] = {2 * t, 2 * t, 2 * t + 8, 2 * t + 8};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = rows[q], k = cols[q];
                split2<BF>(fre(m, k), fre(m, k + 1), fr_h[q], fr_l[q]);
                split2<BF>(fim(m, k), fim(m, k + 1), fi_h[q], fi_l[q]);
                split2<BF>(-fim(m, k), -fim(m, k + 1), fn_h[q], fn_l[q]);
            }
        }
        for (int r = 0; r < reps; ++r) {
#pragma unroll
            for (int grp = 0; grp < 4; ++grp) {  // 8 transforms per group, 4 groups per warp
                const int col = warp * 32 + grp * 8;
                uint32_t xr_h0, xr_l0, xr_h1, xr_l1, xi_h0, xi_l0, xi_h1, xi_l1;
                split2<BF>(re[(2 * t) * kStride + col + g], re[(2 * t + 1) * kStride + col + g], xr_h0, xr_l0);
                split2<BF>(re[(2 * t + 8) * kStride + col + g], re[(2 * t + 9) * kStride + col + g], xr_h1, xr_l1);
                split2<BF>(im[(2 * t) * kStride + col + g], im[(2 * t + 1) * kStride + col + g], xi_h0, xi_l0);
                split2<BF>(im[(2 * t + 8) * kStride + col + g], im[(2 * t + 9) * kStride + col + g], xi_h1, xi_l1);
                float yr[4] = {0.f, 0.f, 0.f, 0.f}, yi[4] = {0.f, 0.f, 0.f, 0.f};
                // Re y = Re F·Re x - Im F·Im x;  Im y = Im F·Re x + Re F·Im x
                mma16816<BF>(yr, fr_h, xr_h0, xr_h1);
                mma16816<BF>(yr, fn_h, xi_h0, xi_h1);
                mma16816<BF>(yi, fi_h, xr_h0, xr_h1);
                mma16816<BF>(yi, fr_h, xi_h0, xi_h1);
                if constexpr (THREE) {
                    mma16816<BF>(yr, fr_h, xr_l0, xr_l1);
                    mma16816<BF>(yr, fr_l, xr_h0, xr_h1);
                    mma16816<BF>(yr, fn_h, xi_l0, xi_l1);
                    mma16816<BF>(yr, fn_l, xi_h0, xi_h1);
                    mma16816<BF>(yi, fi_h, xr_l0, xr_l1);
                    mma16816<BF>(yi, fi_l, xr_h0, xr_h1);
                    mma16816<BF>(yi, fr_h, xi_l0, xi_l1);
                    mma16816<BF>(yi, fr_l, xi_h0, xi_h1);
                }
                __syncwarp();
                re[g * kStride + col + 2 * t] = yr[0];
                re[g * kStride + col + 2 * t + 1] = yr[1];
                re[(g + 8) * kStride + col + 2 * t] = yr[2];
                re[(g + 8) * kStride + col + 2 * t + 1] = yr[3];
                im[g * kStride + col + 2 * t] = yi[0];
                im[g * kStride + col + 2 * t + 1] = yi[1];
                im[(g + 8) * kStride + col + 2 * t] = yi[2];
                im[(g + 8) * kStride + col + 2 * t + 1] = yi[3];
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < kTile * 16; i += kThreads) {
        const int col = i / 16, k = i % 16;
        blk[2 * i] = re[k * kStride + col];
        blk[2 * i + 1] = im[k * kStride + col];
    }
}

static double max_rel_l2(const std::vector<float>& got, const std::vector<float>& in, int ndft) {
    // FP64 DFT of each input, one repetition
    double num = 0.0, den = 0.0;
    for (int d = 0; d < ndft; ++d) {
        for (int m = 0; m < 16; ++m) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < 16; ++k) {
                const double a = -2.0 * M_PI * ((m * k) % 16) / 16.0;
                const double xr = in[(size_t)d * 32 + 2 * k], xi = in[(size_t)d * 32 + 2 * k + 1];
                sr += xr * std::cos(a) - xi * std::sin(a);
                si += xr * std::sin(a) + xi * std::cos(a);
            }
            const double er = got[(size_t)d * 32 + 2 * m] - sr, ei = got[(size_t)d * 32 + 2 * m + 1] - si;
            num += er * er + ei * ei;
            den += sr * sr + si * si;
        }
    }
    return std::sqrt(num / den);
}

int main(int argc, char** argv) {
    const int blocks = argc > 1 ? std::atoi(argv[1]) : 152 * 8;
    const int reps = argc > 2 ? std::atoi(argv[2]) : 64;
    const int ndft = blocks * kTile;
    std::vector<float> h((size_t)ndft * 32);
    unsigned s = 12345u;
    for (auto& v : h) {  // uniform in [-1, 1)
        s = s * 1664525u + 1013904223u;
        v = (float)((s >> 8) * (2.0 / 16777216.0) - 1.0);
    }
    float* d = nullptr;
    if (cudaMalloc(&d, h.size() * sizeof(float)) != cudaSuccess) return 1;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const char* names[6] = {"cc_reg", "cc_smem", "mma3", "mma1", "mma3_bf16", "mma1_bf16"};
    std::printf("{\"transforms\": %d, \"reps\": %d", ndft, reps);
    for (int mode = 0; mode < 6; ++mode) {
        // accuracy: one repetition
        cudaMemcpy(d, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
        switch (mode) {
            case 0: k_dft16<0><<<blocks, kThreads>>>(d, 1); break;
            case 1: k_dft16<1><<<blocks, kThreads>>>(d, 1); break;
            case 2: k_dft16<2><<<blocks, kThreads>>>(d, 1); break;
            case 3: k_dft16<3><<<blocks, kThreads>>>(d, 1); break;
            case 4: k_dft16<4><<<blocks, kThreads>>>(d, 1); break;
            default: k_dft16<5><<<blocks, kThreads>>>(d, 1); break;
        }
        std::vector<float> out(h.size());
        if (cudaMemcpy(out.data(), d, out.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
        const int check = ndft < 4096 ? ndft : 4096;
        const double err = max_rel_l2(out, h, check);
        // time: reps repetitions, median of 5
        std::vector<float> ms(5);
        for (int it = 0; it < 6; ++it) {
            cudaEventRecord(a);
            switch (mode) {
                case 0: k_dft16<0><<<blocks, kThreads>>>(d, reps); break;
                case 1: k_dft16<1><<<blocks, kThreads>>>(d, reps); break;
                case 2: k_dft16<2><<<blocks, kThreads>>>(d, reps); break;
                case 3: k_dft16<3><<<blocks, kThreads>>>(d, reps); break;
                case 4: k_dft16<4><<<blocks, kThreads>>>(d, reps); break;
                default: k_dft16<5><<<blocks, kThreads>>>(d, reps); break;
            }
            cudaEventRecord(b);
            cudaEventSynchronize(b);
            if (it > 0) cudaEventElapsedTime(&ms[it - 1], a, b);
        }
        std::sort(ms.begin(), ms.end());
        const double ns_per = ms[2] * 1e6 / ((double)ndft * reps);
        std::printf(", \"%s\": {\"rel_l2\": %.3e, \"ms\": %.4f, \"ns_per_dft16\": %.5f}", names[mode], err, ms[2],
                    ns_per);
    }
    std::printf(", \"status\": \"%s\"}\n", cudaGetErrorString(cudaGetLastError()));
    cudaFree(d);
    return 0;
}
