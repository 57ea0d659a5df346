// sbp_sweep.cuh — the FP32 solve in three sweeps over the half spectrum.
//
// The y transform (length NY = RA·RB) is split into its two Stockham stages
// and each stage is fused into a neighbouring pass, so that a solve reads
// and writes the half spectrum once per pass and makes three passes instead
// of five (Sect. 2.4: the transform and the Green's multiply per column;
// here the transposes are the pass boundaries in HBM):
//
//   pass A (k3_forward): per (plane group, j ∈ [0, RB)): the real rows
//       y = j + RB·r (r < RA) of ZA planes are transformed along x (two rows
//       per complex FFT, Hermitian split on shuffles), then for every (z, a)
//       the radix-RA stage over r is applied and its output k ∈ [0, RA),
//       times the next stage's twiddle ω_NY^{k·j}, is stored at S[k][a][j][z].
//       Unless pass B evaluates the Green's parameters itself (GREEN_MID),
//       the first blocks of the grid fill the Green's table.
//   pass B (k3_middle): per (k, group of AG columns a): the radix-RB stage
//       over j gives the full y spectrum at
//       b = k + RA·r'; each (b, a) column then takes the padded length-2NZ z
//       transform, the multiply by 4πG/(NX·NY·2NZ)·Ĝ_eff and the truncated
//       inverse (as k_z_padded); the inverse y transform's first stage
//       (radix RB over r', on the conjugated data, no twiddle) follows and
//       output k' is stored at S[k][a][k'][z], in place.  One extra block per
//       box (the first) convolves the FP64 plane sums with the k = 0 kernel.
//   pass C (k3_inverse): per (plane group, j): twiddle ω_NY^{j·k} and the
//       radix-RA stage over k give rows y = j + RB·r of the (conjugated)
//       inverse y transform; the x inverse (Hermitian merge, c2r) follows and
//       the FP64 mean mode is added as a double-float pair.
//
// The half spectrum S is [RA][NX/2+1][RB][NZ] complex: pass B's tile of one
// (k, a) is RB·NZ contiguous values, and passes A and C touch ZA consecutive
// z of every (k, a, j).
//
// Every kernel serves a group of boxes of the same shape: blockIdx.y picks
// the box's descriptor (pointers, shear parameter, physical constants).
#pragma once

#include "sbp_kernels.cuh"

namespace sbp {

// Radix of the y stage fused into the x passes (RA) for a length NY; the
// other stage (pass B) has radix NY / RA.  0: no split built for NY.  At 192
// the split is 12 × 16 with 12-element x transforms (RA·TFX = NX keeps passes
// A and C at one item round, the TMA path): 384-thread blocks then fit three
// per SM, and pass B's one round of items leaves threads for the Green's
// parameters (24 × 8 with 24-element x transforms, two blocks per SM: the
// 192² group's pass A 148 µs against 130).  (The 192-wide sweeps are built for
// 192×192×96, where NX = NY.)
__host__ __device__ constexpr int sweep_ra(int NY) {
    return NY == 32 ? 4 : NY == 64 ? 8 : NY == 96 ? 12 : NY == 128 ? 16 : NY == 192 ? 12 : NY == 256 ? 16 : 0;
}

__host__ __device__ constexpr int sweep_stage_pitch(int need, int ZA) {
    // plane stride (16-byte units) of the staging buffer: at least `need`,
    // and ≡ 8/ZA (mod 8) (odd for ZA ≥ 8) so that the ZA planes of one warp
    // access fall in different banks
    const int q = ZA >= 8 ? 1 : 8 / ZA;
    int s = need;
    while (s % 8 != q) ++s;
    return s;
}

// Planes per pass-A/C block (per = threads of one plane's RA/2 row pairs):
// the largest divisor of NZ whose row pairs fit 256 threads in whole warps,
// unless that gives fewer than 4 planes: passes A and C move runs of ZA
// consecutive z per (k, a, j), and runs under 32 bytes (ZA < 4) fill only
// part of each sector and multiply the L1 wavefronts, so blocks then take up
// to 512 threads to reach 4 planes.
__host__ __device__ constexpr int sweep_za(int NZ, int per) {
    for (int za = per > 0 ? 256 / per : 0; za >= 4; --za)
        if (NZ % za == 0 && (za * per) % 32 == 0) return za;
    for (int za = 4; per > 0 && za * per <= 512; ++za)
        if (NZ % za == 0 && (za * per) % 32 == 0) return za;
    for (int za = per > 0 ? 256 / per : 0; za >= 1; --za)
        if (NZ % za == 0 && (za * per) % 32 == 0) return za;
    return 0;
}

// Resident blocks per SM the passes A and C aim for: 512-thread blocks two
// (64 registers), 384-thread blocks three (56), smaller ones as many as fit
// 64 registers (or 8).
__host__ __device__ constexpr int sweep_ac_blocks(int nt) { return nt > 384 ? 2 : nt > 256 ? 3 : (nt <= 128 ? 8 : 4); }

template <int NX, int NY, int NZ>
struct SweepShape {
    static constexpr int RA = sweep_ra(NY);
    static constexpr int RB = RA > 0 ? NY / RA : 1;
    static constexpr int H = NX / 2 + 1;
    // pass A and C: row pairs of ZA planes, TFX threads per pair
    static constexpr int EX = NX == 192 ? 12 : plan_E(NX, false);  // see sweep_ra
    static constexpr int TFX = NX / EX;
    static constexpr int ZA = sweep_za(NZ, (RA / 2) * TFX);
    static constexpr int PA = ZA * RA / 2;
    static constexpr int NTA = PA * TFX;
    static constexpr int RP = padded_row(NX);
    // staging: per plane, RA/2 row pairs of H slots of 16 bytes (X0 and X1 of
    // one a side by side); SP is the plane stride in those slots
    static constexpr int SP = sweep_stage_pitch((RA / 2) * H, ZA);
    static constexpr int XS = (PA * RP > 2 * ZA * SP) ? PA * RP : 2 * ZA * SP;  // complex slots
    // y-stage items of passes A and C: (plane, a) for a < NX/2, the a = 0 item
    // also carrying the real a = NX/2 column as its imaginary part
    static constexpr int ITEMS_AC = ZA * (NX / 2);
    // twiddles | exchange / staging / TMA box | pass A: pair sums (PA) and ω_NY^{k·j} (RA);
    // pass C: ω_NY^{j·k} (RA) and an mbarrier
    static constexpr size_t smem_ac = (size_t)(NX + XS + PA + RA) * sizeof(cpx<float>);
    // pass B: AG columns a, RB y columns each, TFZ threads per padded column
    static constexpr int M = 2 * NZ;
    static constexpr int EZ = plan_E(M, false);
    static constexpr int TFZ = M / EZ;
    static constexpr int AG = 256 / (RB * TFZ) > 0 ? 256 / (RB * TFZ) : 1;
    static constexpr int CB = AG * RB;
    static constexpr int NTB = CB * TFZ;
    static constexpr int NGA = (H + AG - 1) / AG;
    // y-stage items of pass B, (a, z) with one thread each, in ROUNDS_B
    // rounds.  (A lane pair per item costs more instructions than it saves in
    // latency, and so does a table of the Green's factors filled by the
    // threads a round leaves without an item: both measured slower.)
    static constexpr int ITEMS_B = AG * NZ;
    static constexpr int ROUNDS_B = (ITEMS_B + NTB - 1) / NTB;
    // When the one round of items leaves at least CB threads idle, CB of them
    // (from G0 on) evaluate the block's Green's parameters in FP64 meanwhile,
    // and pass A fills no table (GREEN_MID: 256² saves pass A's table blocks,
    // 28 µs of 264 for 16 boxes, against 7 µs more in pass B; 192² qualifies
    // with its 12 × 16 split).  Otherwise pass A's leading blocks fill the
    // table and pass B reads it (with a second round of items the FP64 work
    // lands on the critical path: measured slower).
    static constexpr int G0 = ITEMS_B - (ROUNDS_B - 1) * NTB;
    static constexpr bool GREEN_MID = ROUNDS_B == 1 && NTB - G0 >= CB;
    static constexpr int GM_BYTES = (CB * (int)sizeof(GreenT<float>) + 15) / 16 * 16;
    static constexpr size_t smem_b = (size_t)M * sizeof(cpx<float>) + GM_BYTES +
                                     (size_t)xchg_slots<float>(M, CB) * sizeof(cpx<float>);
    // TMA path of passes A and C: the block's box of the half spectrum,
    // [k < RA][a < H][j: 1][z < ZA], moved by one bulk tensor copy through the
    // staging region (items in one round, box no larger than the region, z run
    // a multiple of 16 bytes, every box dimension ≤ 256)
    static constexpr int BOX = RA * H * ZA;  // complex values
    static constexpr bool TMA = ITEMS_AC == NTA && BOX <= XS && (ZA * 8) % 16 == 0 && H <= 256 && ZA <= 256 &&
                                PA >= RA + 1 && (NX * 8) % 128 == 0;
    static constexpr bool ok = RA > 0 && ZA > 0 && (NY % RA) == 0 && (RA % 2) == 0 &&
                               NTA % 32 == 0 && NTA <= 512 && NTB <= 256 && RB * TFZ <= 256 &&
                               TFZ % 2 == 0 && NTB % 32 == 0 && TFX <= 32 && ITEMS_AC % NTA == 0 && PA >= RA;
};

// Per-box descriptor of a sweep launch (device memory).
struct SweepBox {
    // the half spectrum as a 4D tensor (z, j, a, k), 8-byte elements, box
    // (ZA, 1, H, RA): the TMA path of passes A and C (unused elsewhere)
    CUtensorMap tmap;
    int* err;               // status word: set to 1 when a bounded wait gives up
    const float* rho;       // [NZ][NY][NX]
    float* phi;             // [NZ][NY][NX]
    cpx<float>* S;          // half spectrum, [RA][H][RB][NZ]
    GreenT<float>* green;   // [NY][H] Green's parameters at this solve's time
    double* tile_sums;      // [NZ][RB] FP64 partial plane sums
    double* vk0;            // [NZ] FP64 mean-mode potential
    const double* c00;      // [2NZ - 1] FP64 k = 0 vertical kernel
    const double* s_dev;    // shear parameter on the device (batched), or null
    double Lx, Ly, L;       // box lengths and the truncation length L = Lz
    double scale;           // 4πG / (NX·NY·2NZ)
    double kzc;             // (π / Lz)²
    double k0_coef;         // 4πG / (NX·NY)
};

// Per-launch arguments.  With rho non-null the launch serves one box whose
// rho, phi and shear parameter s are given here (single solves); otherwise
// every box takes them from its descriptor.
struct SweepArgs {
    const SweepBox* boxes;
    const float* rho;
    float* phi;
    double s;
    const double* s_dev;    // single box: its shear parameter on the device (a graph replay), or null
    const cpx<float>* twx;  // e^{-2πi k/NX}, k < NX
    const cpx<float>* twy;  // e^{-2πi k/NY}, k < NY
    const cpx<float>* twM;  // e^{-2πi k/2NZ}, k < 2NZ
    int green_blocks;       // pass A: leading blocks per box that fill the Green's table
    long long budget;       // clock cycles a bounded wait may take
    int withhold;           // test switch: the TMA loads arm no copy, so their waits run out
};

// ---------------------------------------------------------------------------
// pass A
// ---------------------------------------------------------------------------
template <int NX, int NY, int NZ>
__global__ void __launch_bounds__(SweepShape<NX, NY, NZ>::NTA, sweep_ac_blocks(SweepShape<NX, NY, NZ>::NTA))
    k3_forward(SweepArgs A) {
    using SH = SweepShape<NX, NY, NZ>;
    constexpr int RA = SH::RA, RB = SH::RB, H = SH::H, EX = SH::EX, TFX = SH::TFX, ZA = SH::ZA;
    constexpr int RP = SH::RP, SP = SH::SP, XS = SH::XS;
    static_assert(SH::ok, "sweep shape");
    const SweepBox& B = A.boxes[blockIdx.y];
    grid_dep_launch();  // a single solve's middle sweep may launch during this grid's last wave
    if ((int)blockIdx.x < A.green_blocks) {  // Green's table, off the transform blocks
        GreenFill gf;
        gf.tab = B.green;
        gf.per_block = (H * NY + A.green_blocks - 1) / A.green_blocks;
        gf.nx = NX;
        gf.ny = NY;
        gf.yhalf = 0;
        gf.Lx = B.Lx;
        gf.Ly = B.Ly;
        gf.L = B.L;
        gf.s = A.s;
        gf.s_dev = A.rho != nullptr ? A.s_dev : B.s_dev;
        green_fill<float>(gf, blockIdx.x);
        return;
    }
    const float* __restrict__ rho = A.rho != nullptr ? A.rho : B.rho;
    const int bid = (int)blockIdx.x - A.green_blocks;
    const int zg = bid % (NZ / ZA), j = bid / (NZ / ZA);
    const int z0 = zg * ZA;
    extern __shared__ __align__(128) unsigned char smem_raw[];  // the TMA box at xb: 128-byte aligned (NX·8 is)
    cpx<float>* tw = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<float>* xb = tw + NX;
    FF* psum = reinterpret_cast<FF*>(xb + XS);
    cpx<float>* wyk = xb + XS + SH::PA;  // ω_NY^{k·j}, k < RA
    const int tid = threadIdx.x;
    build_stage_twiddles<NX, EX, float>(tw, A.twx);  // the x transform's stage table (fits in NX slots)
    if (tid < RA) wyk[tid] = A.twy[(tid * j) % NY];

    const int t = tid % TFX, c = tid / TFX;
    const int zl = c / (RA / 2), p = c % (RA / 2);
    const int z = z0 + zl;
    const float* r0p = rho + ((size_t)z * NY + j + RB * (2 * p)) * NX;
    const float* r1p = r0p + (size_t)RB * NX;
    cpx<float> v[1][EX];
#pragma unroll
    for (int e = 0; e < EX; ++e) v[0][e] = {__ldcs(r0p + t + TFX * e), __ldcs(r1p + t + TFX * e)};
    {
        // FP64-quality plane sums: compensated float sums of both rows (one
        // packed pair), double-float reduction over the pair's lanes
        cpx<float> hi = {0.f, 0.f}, lo = {0.f, 0.f};
#pragma unroll
        for (int e = 0; e < EX; ++e) {
            const cpx<float> y = cadd(v[0][e], lo);
            const cpx<float> tt = cadd(hi, y);
            lo = csub(y, csub(tt, hi));
            hi = tt;
        }
        FF acc = ff_add(FF{hi.x, lo.x}, FF{hi.y, lo.y});
#pragma unroll
        for (int o = TFX / 2; o > 0; o >>= 1) {
            const FF other = {__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)};
            acc = ff_add(acc, other);
        }
        if (t == 0) psum[c] = acc;
    }
    __syncthreads();  // twiddles visible
    const SmemRow<float> buf[1] = {{xb + c * RP, 0}};
    fft_static_st<NX, EX, 0, 1, float>(v, t, tw, buf);

    // Hermitian split of the paired transform (Z[n-k] is element E-1-e of lane
    // TFX-t of the same pair, or of lane 0 itself): X0 = (Z[k] + conj Z[n-k])/2,
    // X1 = -i (Z[k] - conj Z[n-k])/2, staged as [plane][row][a]
    __syncthreads();  // the exchange buffer becomes the staging buffer
    if (tid < ZA) {
        FF tot = {0.f, 0.f};
        for (int q = 0; q < RA / 2; ++q) tot = ff_add(tot, psum[tid * (RA / 2) + q]);
        if (B.tile_sums != nullptr) B.tile_sums[(size_t)(z0 + tid) * RB + j] = (double)tot.hi + (double)tot.lo;
    }
    float4* st4 = reinterpret_cast<float4*>(xb);  // staging: [plane][pair][a], X0 and X1 side by side
    {
        const int lane = tid & 31;
        const int src = lane - t + ((TFX - t) & (TFX - 1));
        float4* o = st4 + zl * SP + p * H;
        const float half = 0.5f;
#pragma unroll
        for (int e = 0; e <= EX / 2; ++e) {
            const cpx<float> send = v[0][EX - 1 - e];
            cpx<float> Bz;
            Bz.x = __shfl_sync(0xffffffffu, send.x, src);
            Bz.y = __shfl_sync(0xffffffffu, send.y, src);
            if (t == 0) Bz = v[0][(EX - e) % EX];
            Bz = cconj(Bz);
            const cpx<float> Az = v[0][e];
            if (e < EX / 2 || t == 0) {
                const int k = t + TFX * e;
                o[k] = make_float4((Az.x + Bz.x) * half, (Az.y + Bz.y) * half, (Az.y - Bz.y) * half,
                                   (Bz.x - Az.x) * half);
            }
        }
    }
    __syncthreads();
    // y stage 1: for every (z, a) the radix-RA DFT over the rows r.  The a = 0
    // and a = NX/2 columns are real, so one item transforms both at once
    // (a = 0 as the real part, a = NX/2 as the imaginary part) and separates
    // them by the Hermitian symmetry of each: A[k] = (C[k] + conj C[-k]) / 2,
    // B[k] = (C[k] - conj C[-k]) / 2i.
    cpx<float>* __restrict__ S = B.S;
    constexpr size_t KS = (size_t)H * RB * NZ;  // stride of k in S
#pragma unroll 1
    for (int i = tid; i < SH::ITEMS_AC; i += SH::NTA) {
        const int zi = i % ZA, a = i / ZA;
        cpx<float> x[RA];
        const float4* row = st4 + zi * SP;
#pragma unroll
        for (int q = 0; q < RA / 2; ++q) {
            const float4 f = row[q * H + a];
            x[2 * q] = {f.x, f.y};
            x[2 * q + 1] = {f.z, f.w};
        }
        if (a == 0) {
#pragma unroll
            for (int q = 0; q < RA / 2; ++q) {
                const float4 g = row[q * H + NX / 2];
                x[2 * q].y = g.x;
                x[2 * q + 1].y = g.z;
            }
        }
        Dft<RA, float>::run(x);
        // output k, times the next y stage's twiddle ω_NY^{k·j}
        auto tw_k = [&](cpx<float> u, int k) { return k == 0 ? u : cmul(u, wyk[k]); };
        if constexpr (SH::TMA) {
            // one round of items: stage the outputs in box order [k][a][zi]
            // (aliasing the staging, hence the barrier) and store the box by TMA
            cpx<float>* bx = xb;
            __syncthreads();
            if (a != 0) {
#pragma unroll
                for (int k = 0; k < RA; ++k) bx[(k * H + a) * ZA + zi] = tw_k(x[k], k);
            } else {
#pragma unroll
                for (int k = 0; k < RA; ++k) {
                    const cpx<float> c = x[k], d = x[(RA - k) % RA];
                    bx[(k * H) * ZA + zi] = tw_k({0.5f * (c.x + d.x), 0.5f * (c.y - d.y)}, k);
                    bx[(k * H + NX / 2) * ZA + zi] = tw_k({0.5f * (c.y + d.y), 0.5f * (d.x - c.x)}, k);
                }
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                tma_store_4d(&B.tmap, z0, j, 0, 0, bx);
                bulk_commit();
                bulk_wait_read();  // the block's shared memory stays until the copy has read it
            }
            continue;
        }
        cpx<float>* dst = S + ((size_t)a * RB + j) * NZ + z0 + zi;
        if (a != 0) {
#pragma unroll
            for (int k = 0; k < RA; ++k) dst[k * KS] = tw_k(x[k], k);
        } else {
            cpx<float>* dstN = S + ((size_t)(NX / 2) * RB + j) * NZ + z0 + zi;
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const cpx<float> c = x[k], d = x[(RA - k) % RA];
                dst[k * KS] = tw_k({0.5f * (c.x + d.x), 0.5f * (c.y - d.y)}, k);
                dstN[k * KS] = tw_k({0.5f * (c.y + d.y), 0.5f * (d.x - c.x)}, k);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// pass B
// ---------------------------------------------------------------------------
template <int NX, int NY, int NZ>
__global__ void __launch_bounds__(SweepShape<NX, NY, NZ>::NTB, (SweepShape<NX, NY, NZ>::EZ > 16 ? 3 : 4))
    k3_middle(SweepArgs A) {
    using SH = SweepShape<NX, NY, NZ>;
    constexpr int RA = SH::RA, RB = SH::RB, H = SH::H, M = SH::M, EZ = SH::EZ, TFZ = SH::TFZ;
    constexpr int AG = SH::AG, CB = SH::CB, NGA = SH::NGA;
    static_assert(SH::ok, "sweep shape");
    const SweepBox& B = A.boxes[blockIdx.y];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* twM = reinterpret_cast<cpx<float>*>(smem_raw);
    GreenT<float>* gm = reinterpret_cast<GreenT<float>*>(twM + M);
    cpx<float>* xb = reinterpret_cast<cpx<float>*>(reinterpret_cast<unsigned char*>(gm) + SH::GM_BYTES);
    const int tid = threadIdx.x;
    grid_dep_launch();  // likewise the inverse sweep
    grid_dep_wait();    // pass A's spectrum, table and plane sums complete (single solves)
    if (blockIdx.x == 0) {
        // the FP64 mean mode: vk0[i] = coef Σ_j c00[i - j + NZ - 1] S[j] from the
        // plane sums (O(NZ²) at GB300's 1/64-rate FP64: the first block of each
        // box's row, so that it overlaps the transform blocks instead of
        // trailing them)
        if (B.vk0 != nullptr) {
            ZArgs za;
            za.tile_sums = B.tile_sums;
            za.tiles_per_plane = RB;
            za.c00 = B.c00;
            za.k0_coef = B.k0_coef;
            za.vk0 = B.vk0;
            mean_mode_fp64(za, NZ, reinterpret_cast<double*>(xb));
        }
        return;
    }
    const int k = ((int)blockIdx.x - 1) / NGA, ag = ((int)blockIdx.x - 1) % NGA;
    const int a0 = ag * AG;
    for (int i = tid; i < M; i += SH::NTB) twM[i] = A.twM[i];
    // the Green's parameters of column c: mode (a, b), a = a0 + c / RB, b = k + RA·(c % RB)
    auto column_mode = [&](int c, GreenT<float>& g) {
        const int a = a0 + c / RB, b = k + RA * (c % RB);
        g = GreenT<float>{};
        g.kzero = 1;  // columns past the half spectrum: finite, never stored
        g.same = 1;
        return a < H ? (size_t)b * H + a : (size_t)-1;
    };
    if constexpr (!SH::GREEN_MID) {
        if (tid < CB) {
            GreenT<float> g;
            const size_t q = column_mode(tid, g);
            if (q != (size_t)-1) g = B.green[q];
            gm[tid] = g;
        }
    }
    cpx<float>* __restrict__ S = B.S;
    const size_t tile = ((size_t)k * H + a0) * RB * NZ;  // this block's [AG][RB][NZ] tile
    const float scale = (float)B.scale;
    const float kzc = (float)B.kzc;
    const float L2half = (float)(0.5 * B.L * B.L);
    // y stage 2 (forward): item (al, z) takes the radix-RB DFT over j (its
    // twiddle ω_NY^{k·j} came with pass A's output); output r' is column
    // al·RB + r' (b = k + RA·r').  It neither reads nor writes what the setup
    // above writes, so the barrier after it serves both.
    constexpr int ROUNDS = SH::ROUNDS_B;
#pragma unroll 1
    for (int rd = 0; rd < ROUNDS; ++rd) {
        const int item = tid + rd * SH::NTB;
        const int zi = item % NZ, al = item / NZ;
        const bool in_range = item < SH::ITEMS_B;  // warp-uniform: items are contiguous in tid
        const bool valid = in_range && a0 + al < H;
        if (in_range) {
            cpx<float> x[RB];
            const cpx<float>* src = S + tile + (size_t)al * RB * NZ + zi;
#pragma unroll
            for (int n1 = 0; n1 < RB; ++n1) {
                cpx<float> v0 = {0.f, 0.f};
                if (valid) v0 = src[(size_t)n1 * NZ];
                x[n1] = v0;
            }
            Dft<RB, float>::run(x);
#pragma unroll
            for (int k1 = 0; k1 < RB; ++k1) {
                const XchgCol<float, CB> col = {xb + al * RB + k1, 0};
                col[zi] = x[k1];
            }
        }
    }
    if constexpr (SH::GREEN_MID) {
        // FP64 evaluation of the block's CB modes (the table's values: |k(t)|²
        // and 1 - e^{-|k|L}, rounded once to float) by threads the last round
        // left without an item, on the otherwise idle FP64 pipe
        const int c = tid - SH::G0;
        if (c >= 0 && c < CB) {
            GreenT<float> g;
            const size_t q = column_mode(c, g);
            if (q != (size_t)-1) {
                const double sh = A.rho != nullptr ? (A.s_dev != nullptr ? *A.s_dev : A.s) : *B.s_dev;
                const GreenMode m = green_mode(a0 + c / RB, k + RA * (c % RB), NX, NY, B.Lx, B.Ly, B.L, sh);
                g = GreenT<float>{(float)m.k2a, (float)m.omEa, (float)m.k2b, (float)m.omEb, m.kzero, m.same};
            }
            gm[c] = g;
        }
    }
    __syncthreads();

    // padded z transform per column (as k_z_padded)
    const int c = tid % CB, t = tid / CB;
    const XchgCol<float, CB> buf[1] = {{xb + c, 0}};
    cpx<float> v[1][EZ];
#pragma unroll
    for (int e = 0; e < EZ / 2; ++e) v[0][e] = buf[0][t + TFZ * e];
    fft_static_padded<M, EZ, 1, float>(v, t, twM, buf);  // starts with a barrier
    {
        const GreenCoef<float> q = green_coef<float>(gm[c], scale, true);
        static_assert(TFZ % 2 == 0 && (CB * TFZ) % 32 == 0, "padded z shape");
        if (__all_sync(0xffffffffu, q.same && !q.kzero)) {
            const float num = (t & 1) ? q.ao : q.ae;
            const float tf = (float)t;
#pragma unroll
            for (int e = 0; e < EZ; ++e) {
                const float ms = (e < EZ / 2) ? tf + (float)(TFZ * e) : (float)(M - TFZ * e) - tf;
                const float f = fast_div(num, fmaf(kzc * ms, ms, q.k2a));
                v[0][e] = cconj_scale(v[0][e], f);
            }
        } else {
#pragma unroll
            for (int e = 0; e < EZ; ++e) {
                const int m = t + TFZ * e;
                const int ms = (m <= NZ) ? m : M - m;
                const float f = green_factor<float>(q, m, ms, kzc, scale, L2half);
                v[0][e] = {v[0][e].x * f, -v[0][e].y * f};
            }
        }
    }
    fft_static<M, EZ, 0, 1, float>(v, t, twM, buf);
    // v[e] (e < EZ/2) is the conjugate of the convolved column at z = t + TFZ·e:
    // exactly the input the inverse y transform's first stage wants.  The
    // transform's last exchange read of this thread was buf[t + TFZ·e] for
    // every e, slots no other thread reads after that exchange's barrier, so
    // writing them back needs no barrier first.
#pragma unroll
    for (int e = 0; e < EZ / 2; ++e) buf[0][t + TFZ * e] = v[0][e];
    __syncthreads();
#pragma unroll 1
    for (int rd = 0; rd < ROUNDS; ++rd) {
        const int item = tid + rd * SH::NTB;
        const int zi = item % NZ, al = item / NZ;
        const bool in_range = item < SH::ITEMS_B;
        const bool valid = in_range && a0 + al < H;
        if (in_range) {
            cpx<float> x[RB];
#pragma unroll
            for (int n1 = 0; n1 < RB; ++n1) {
                const XchgCol<float, CB> col = {xb + al * RB + n1, 0};
                x[n1] = col[zi];
            }
            Dft<RB, float>::run(x);
            if (valid) {
                cpx<float>* dst = S + tile + (size_t)al * RB * NZ + zi;
#pragma unroll
                for (int k1 = 0; k1 < RB; ++k1) dst[(size_t)k1 * NZ] = x[k1];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// pass C
// ---------------------------------------------------------------------------
template <int NX, int NY, int NZ>
__global__ void __launch_bounds__(SweepShape<NX, NY, NZ>::NTA, sweep_ac_blocks(SweepShape<NX, NY, NZ>::NTA))
    k3_inverse(SweepArgs A) {
    using SH = SweepShape<NX, NY, NZ>;
    constexpr int RA = SH::RA, RB = SH::RB, H = SH::H, EX = SH::EX, TFX = SH::TFX, ZA = SH::ZA;
    constexpr int RP = SH::RP, SP = SH::SP;
    static_assert(SH::ok, "sweep shape");
    const SweepBox& B = A.boxes[blockIdx.y];
    float* __restrict__ phi = A.rho != nullptr ? A.phi : B.phi;
    const int bid = blockIdx.x;
    const int zg = bid % (NZ / ZA), j = bid / (NZ / ZA);
    const int z0 = zg * ZA;
    extern __shared__ __align__(128) unsigned char smem_raw[];  // the TMA box at xb: 128-byte aligned (NX·8 is)
    cpx<float>* tw = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<float>* xb = tw + NX;
    const int tid = threadIdx.x;
    cpx<float>* wy = xb + SH::XS;  // ω_NY^{j·k}, k < RA (PA ≥ RA slots after the staging)
    uint64_t* bar = reinterpret_cast<uint64_t*>(wy + RA);
    grid_dep_wait();  // pass B's spectrum and mean mode complete (single solves)
    if constexpr (SH::TMA) {
        // the block's box [k][a][j][z0 .. z0+ZA) of the half spectrum by one TMA load
        if (tid == 0) {
            mbar_init(bar, 1);
            mbar_fence_init();
            if (!A.withhold) {
                mbar_arrive_expect_tx(bar, (uint32_t)(SH::BOX * sizeof(cpx<float>)));
                tma_load_4d(xb, &B.tmap, z0, j, 0, 0, bar);
            }
        }
    }
    build_stage_twiddles<NX, EX, float>(tw, A.twx);
    if (tid < RA) wy[tid] = A.twy[(j * tid) % NY];
    __syncthreads();
    if constexpr (SH::TMA) {
        const bool ok = mbar_wait_bounded(bar, 0, A.budget);
        if (!__syncthreads_and(ok)) {  // uniform exit: the copy did not arrive in time
            if (tid == 0 && B.err != nullptr) atomicExch(B.err, 1);
            // a copy that is only late still targets this block's shared memory:
            // stay resident (a second bounded wait) until it lands
            if (!A.withhold) mbar_wait_bounded(bar, 0, A.budget);
            return;
        }
    }
    // y stage 2 of the inverse: twiddle ω_NY^{j·k} and the radix-RA DFT over k
    // give rows j + RB·r of the conjugated inverse y transform.  The a = 0 and
    // a = NX/2 columns come out real, so one item transforms both (as u + i v)
    // and keeps the real and imaginary parts of the result.
    const cpx<float>* __restrict__ S = B.S;
    float4* st4 = reinterpret_cast<float4*>(xb);  // staging: [plane][pair][a], rows 2q and 2q+1 side by side
    constexpr size_t KS = (size_t)H * RB * NZ;
#pragma unroll 1
    for (int i = tid; i < SH::ITEMS_AC; i += SH::NTA) {
        const int zi = i % ZA, a = i / ZA;
        cpx<float> x[RA];
        if constexpr (SH::TMA) {
            const cpx<float>* bx = xb;  // box [k][a][zi]
#pragma unroll
            for (int k = 0; k < RA; ++k) x[k] = bx[(k * H + a) * ZA + zi];
            if (a == 0) {
#pragma unroll
                for (int k = 0; k < RA; ++k) {
                    const cpx<float> u = x[k], w = bx[(k * H + NX / 2) * ZA + zi];
                    x[k] = {u.x - w.y, u.y + w.x};
                }
            }
            __syncthreads();  // every item has its inputs: the box region becomes the staging
        } else {
            const cpx<float>* src = S + ((size_t)a * RB + j) * NZ + z0 + zi;
#pragma unroll
            for (int k = 0; k < RA; ++k) x[k] = src[k * KS];
            if (a == 0) {
                const cpx<float>* srcN = S + ((size_t)(NX / 2) * RB + j) * NZ + z0 + zi;
#pragma unroll
                for (int k = 0; k < RA; ++k) {
                    const cpx<float> u = x[k], w = srcN[k * KS];
                    x[k] = {u.x - w.y, u.y + w.x};
                }
            }
        }
#pragma unroll
        for (int k = 1; k < RA; ++k) x[k] = cmul(x[k], wy[k]);
        Dft<RA, float>::run(x);
        float4* row = st4 + zi * SP;
        if (a != 0) {
#pragma unroll
            for (int q = 0; q < RA / 2; ++q) row[q * H + a] = make_float4(x[2 * q].x, x[2 * q].y, x[2 * q + 1].x, x[2 * q + 1].y);
        } else {
#pragma unroll
            for (int q = 0; q < RA / 2; ++q) {
                row[q * H] = make_float4(x[2 * q].x, 0.f, x[2 * q + 1].x, 0.f);
                row[q * H + NX / 2] = make_float4(x[2 * q].y, 0.f, x[2 * q + 1].y, 0.f);
            }
        }
    }
    __syncthreads();

    // x inverse of the row pair (2p, 2p+1) of plane zl.  The staging holds
    // c0 = conj X0 and c1 = conj X1; the transform input is conj Z with
    // Z[k] = X0[k] + i X1[k] (k ≤ n/2) or conj X0[n-k] + i conj X1[n-k].
    const int t = tid % TFX, c = tid / TFX;
    const int zl = c / (RA / 2), p = c % (RA / 2);
    const int z = z0 + zl;
    const float4* w = st4 + zl * SP + p * H;
    cpx<float> v[1][EX];
#pragma unroll
    for (int e = 0; e < EX; ++e) {
        const int k = t + TFX * e;
        if (2 * k <= NX) {
            const float4 f = w[k];
            cpx<float> c0 = {f.x, f.y}, c1 = {f.z, f.w};
            if (k == 0 || 2 * k == NX) {
                c0.y = 0.f;
                c1.y = 0.f;
            }
            v[0][e] = {c0.x + c1.y, c0.y - c1.x};
        } else {
            const float4 f = w[NX - k];
            v[0][e] = {f.x - f.w, -f.y - f.z};
        }
    }
    const SmemRow<float> buf[1] = {{xb + c * RP, 0}};
    fft_static_st<NX, EX, 0, 1, float>(v, t, tw, buf);  // its first exchange follows a barrier
    float add_hi = 0.f, add_lo = 0.f;
    if (B.vk0 != nullptr) {
        const double vv = B.vk0[z];
        add_hi = (float)vv;
        add_lo = (float)(vv - (double)add_hi);
    }
    float* o0 = phi + ((size_t)z * NY + j + RB * (2 * p)) * NX;
    float* o1 = o0 + (size_t)RB * NX;
#pragma unroll
    for (int e = 0; e < EX; ++e) {
        const int x = t + TFX * e;
        // conj of the forward result, plus the FP64 mean mode as a TwoSum of
        // (p0, p1) + hi, then + lo, on both rows at once as packed pairs
        const cpx<float> a = {v[0][e].x, -v[0][e].y}, hh = {add_hi, add_hi}, ll = {add_lo, add_lo};
        const cpx<float> sm = cadd(a, hh);
        const cpx<float> bb = csub(sm, a);
        const cpx<float> er = cadd(csub(a, csub(sm, bb)), csub(hh, bb));
        const cpx<float> r = cadd(sm, cadd(er, ll));
        __stcs(o0 + x, r.x);
        __stcs(o1 + x, r.y);
    }
}

}  // namespace sbp
