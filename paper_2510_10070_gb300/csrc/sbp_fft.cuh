// sbp_fft.cuh — register-resident mixed-radix FFT engine for sm_103a.
//
// A length-N transform is spread over Tf = N/E threads that each hold E
// complex values in registers.  Thread t always holds the elements with
// index t + Tf·e (e < E), in every stage: that is the self-sorting Stockham
// arrangement (Govindaraju et al., SC'08), in which stage s with radix R and
// span Ns = R_0·…·R_{s-1} reads x[j + r·N/R] for butterfly j, multiplies by
// ω_{Ns·R}^{(j mod Ns)·r}, runs an R-point DFT and writes it to
// (j div Ns)·Ns·R + (j mod Ns) + r·Ns.  Consecutive stages exchange through
// shared memory; the first stage reads, and the last stage leaves, the data
// in the thread's own index set, so loads and stores go straight between
// registers and global memory.
//
// Radices: 2, 3, 4, 6, 8, 12, 16, 24.  Every radix used with a given E must
// divide E.  All transforms here are forward (e^{-2πi/N}); inverses use
// conj(FFT(conj(x))).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace sbp {

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x)};
}
// FP32 complex add and subtract as one packed f32x2 instruction (sm_100
// family): the same round-to-nearest results as two scalar FADDs in half the
// issue slots.  The butterflies are mostly complex adds, so this is where
// the transforms spend most of their instructions.
__device__ __forceinline__ cpx<float> cadd(cpx<float> a, cpx<float> b) {
    cpx<float> r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pr, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ cpx<float> csub(cpx<float> a, cpx<float> b) {
    cpx<float> r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
template <typename T>
__device__ __forceinline__ cpx<T> cconj(cpx<T> a) { return {a.x, -a.y}; }
// conj(a)·f for real f; FP32 as one packed multiply by (f, -f).
template <typename T>
__device__ __forceinline__ cpx<T> cconj_scale(cpx<T> a, T f) { return {a.x * f, -a.y * f}; }
__device__ __forceinline__ cpx<float> cconj_scale(cpx<float> a, float f) {
    cpx<float> r;
    asm("{\n\t.reg .b64 pa, pf, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pf, {%4, %5};\n\t"
        "mul.rn.f32x2 pr, pa, pf;\n\t"
        "mov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(f), "f"(-f));
    return r;
}
template <typename T>
__device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return {a.x * s, a.y * s}; }
// a·(-i)
template <typename T>
__device__ __forceinline__ cpx<T> cmul_mi(cpx<T> a) { return {a.y, -a.x}; }
// a·(+i)
template <typename T>
__device__ __forceinline__ cpx<T> cmul_pi(cpx<T> a) { return {-a.y, a.x}; }

// cos(2π i/48) for any integer i, from the first-quadrant values.  Not
// recursive, so that it inlines and folds to a literal for constant i.
__host__ __device__ __forceinline__ constexpr double cos48(int i) {
    constexpr double q[13] = {1.0,
                              0.9914448613738104,
                              0.9659258262890683,
                              0.9238795325112867,
                              0.8660254037844387,
                              0.7933533402912352,
                              0.7071067811865476,
                              0.6087614290087207,
                              0.5,
                              0.38268343236508984,
                              0.25881904510252074,
                              0.1305261922200517,
                              0.0};
    const int m = ((i % 48) + 48) % 48;
    const int j = (m > 24) ? 48 - m : m;  // cos is even: j ∈ [0, 24]
    return (j > 12) ? -q[24 - j] : q[j];  // cos(π - x) = -cos x
}
// sin(2π i/48) = cos(2π (12 - i)/48)
__host__ __device__ __forceinline__ constexpr double sin48(int i) { return cos48(12 - i); }

// a · e^{-2πi J/R} with J a template constant (R divides 48).
template <int R, int J, typename T>
__device__ __forceinline__ cpx<T> twiddle_const(cpx<T> a) {
    constexpr int i48 = ((J % R) + R) % R * (48 / R);
    if constexpr (i48 == 0) {
        return a;
    } else if constexpr (i48 == 12) {
        return cmul_mi(a);
    } else if constexpr (i48 == 24) {
        return {-a.x, -a.y};
    } else if constexpr (i48 == 36) {
        return cmul_pi(a);
    } else {
        constexpr T c = (T)cos48(i48);
        constexpr T s = (T)(-sin48(i48));
        return cmul(a, cpx<T>{c, s});
    }
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1.
template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// ---------------------------------------------------------------------------
// In-register DFTs, natural order in and out, forward sign.
// ---------------------------------------------------------------------------
template <int R, typename T>
struct Dft;

template <typename T>
struct Dft<2, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) {
        const cpx<T> a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

template <typename T>
struct Dft<3, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) {
        const T h = (T)0.8660254037844386;  // sin(2π/3)
        const cpx<T> s = cadd(x[1], x[2]);
        const cpx<T> d = csub(x[1], x[2]);
        const cpx<T> m = {fma((T)-0.5, s.x, x[0].x), fma((T)-0.5, s.y, x[0].y)};
        x[0] = cadd(x[0], s);
        // X1 = m - i·h·d, X2 = m + i·h·d
        x[1] = {fma(h, d.y, m.x), fma(-h, d.x, m.y)};
        x[2] = {fma(-h, d.y, m.x), fma(h, d.x, m.y)};
    }
};

template <typename T>
struct Dft<4, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) {
        const cpx<T> s0 = cadd(x[0], x[2]), d0 = csub(x[0], x[2]);
        const cpx<T> s1 = cadd(x[1], x[3]), d1 = csub(x[1], x[3]);
        x[0] = cadd(s0, s1);
        x[2] = csub(s0, s1);
        x[1] = cadd(d0, cmul_mi(d1));
        x[3] = csub(d0, cmul_mi(d1));
    }
};

template <typename T>
struct Dft<8, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) {
        cpx<T> e[4] = {x[0], x[2], x[4], x[6]};
        cpx<T> o[4] = {x[1], x[3], x[5], x[7]};
        Dft<4, T>::run(e);
        Dft<4, T>::run(o);
        const T r = (T)0.7071067811865476;
        // ω8^1 = r(1 - i), ω8^2 = -i, ω8^3 = -r(1 + i)
        const cpx<T> o1 = {r * (o[1].x + o[1].y), r * (o[1].y - o[1].x)};
        const cpx<T> o2 = cmul_mi(o[2]);
        const cpx<T> o3 = {r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y)};
        x[0] = cadd(e[0], o[0]);
        x[4] = csub(e[0], o[0]);
        x[1] = cadd(e[1], o1);
        x[5] = csub(e[1], o1);
        x[2] = cadd(e[2], o2);
        x[6] = csub(e[2], o2);
        x[3] = cadd(e[3], o3);
        x[7] = csub(e[3], o3);
    }
};

// R = R1·R2 by one Cooley–Tukey split: n = R2·n1 + n2, k = k1 + R1·k2.
template <int R1, int R2, typename T>
__device__ __forceinline__ void dft_split(cpx<T>* x) {
    constexpr int R = R1 * R2;
    cpx<T> y[R];
    static_for<0, R2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        cpx<T> a[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) a[n1] = x[R2 * n1 + n2];
        Dft<R1, T>::run(a);
        static_for<0, R1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            y[n2 * R1 + k1] = twiddle_const<R, n2 * k1>(a[k1]);
        });
    });
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        cpx<T> b[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) b[n2] = y[n2 * R1 + k1];
        Dft<R2, T>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = b[k2];
    }
}

// Twiddled DFT: X = DFT_R(x[r]·w(r)) with w(0) = 1.  The split radices apply
// each first-level group's R1 twiddles just before its DFT_R1, so only R1
// twiddles are live at a time instead of R - 1.
template <int R1, int R2, typename T, typename TW>
__device__ __forceinline__ void dft_split_tw(cpx<T>* x, const TW& w) {
    constexpr int R = R1 * R2;
    cpx<T> y[R];
    static_for<0, R2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        cpx<T> a[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            const int r = R2 * n1 + n2;
            a[n1] = (r == 0) ? x[0] : cmul(x[r], w(r));
        }
        Dft<R1, T>::run(a);
        static_for<0, R1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            y[n2 * R1 + k1] = twiddle_const<R, n2 * k1>(a[k1]);
        });
    });
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        cpx<T> b[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) b[n2] = y[n2 * R1 + k1];
        Dft<R2, T>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = b[k2];
    }
}

template <int R, typename T>
struct DftTw {
    template <typename TW>
    static __device__ __forceinline__ void run(cpx<T>* x, const TW& w) {
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmul(x[r], w(r));
        Dft<R, T>::run(x);
    }
};
template <typename T>
struct DftTw<16, T> {
    template <typename TW>
    static __device__ __forceinline__ void run(cpx<T>* x, const TW& w) { dft_split_tw<4, 4, T>(x, w); }
};
template <typename T>
struct DftTw<24, T> {
    template <typename TW>
    static __device__ __forceinline__ void run(cpx<T>* x, const TW& w) { dft_split_tw<8, 3, T>(x, w); }
};

// DFTs whose upper half of inputs is zero (x[R/2 .. R-1] == 0), used by the
// first stage of a zero-padded transform.
template <int R, typename T>
struct DftHalf;

template <typename T>
struct DftHalf<2, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) { x[1] = x[0]; }
};

template <typename T>
struct DftHalf<4, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) {
        const cpx<T> a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[2] = csub(a, b);
        x[1] = cadd(a, cmul_mi(b));
        x[3] = csub(a, cmul_mi(b));
    }
};

template <typename T>
struct DftHalf<8, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) {
        cpx<T> e[4] = {x[0], x[2], {}, {}};
        cpx<T> o[4] = {x[1], x[3], {}, {}};
        DftHalf<4, T>::run(e);
        DftHalf<4, T>::run(o);
        const T r = (T)0.7071067811865476;
        const cpx<T> o1 = {r * (o[1].x + o[1].y), r * (o[1].y - o[1].x)};
        const cpx<T> o2 = cmul_mi(o[2]);
        const cpx<T> o3 = {r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y)};
        x[0] = cadd(e[0], o[0]);
        x[4] = csub(e[0], o[0]);
        x[1] = cadd(e[1], o1);
        x[5] = csub(e[1], o1);
        x[2] = cadd(e[2], o2);
        x[6] = csub(e[2], o2);
        x[3] = cadd(e[3], o3);
        x[7] = csub(e[3], o3);
    }
};

// R = R1·R2 split with x[n] = 0 for n ≥ R/2: n = R2·n1 + n2 is below R/2
// exactly when n1 < R1/2, so the first-level DFTs are half-zero as well.
template <int R1, int R2, typename T>
__device__ __forceinline__ void dft_split_half(cpx<T>* x) {
    constexpr int R = R1 * R2;
    cpx<T> y[R];
    static_for<0, R2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        cpx<T> a[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1 / 2; ++n1) a[n1] = x[R2 * n1 + n2];
        DftHalf<R1, T>::run(a);
        static_for<0, R1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            y[n2 * R1 + k1] = twiddle_const<R, n2 * k1>(a[k1]);
        });
    });
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        cpx<T> b[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) b[n2] = y[n2 * R1 + k1];
        Dft<R2, T>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = b[k2];
    }
}

template <typename T>
struct DftHalf<16, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) { dft_split_half<4, 4, T>(x); }
};
template <typename T>
struct DftHalf<24, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) { dft_split_half<8, 3, T>(x); }
};
template <typename T>
struct DftHalf<12, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) { dft_split_half<4, 3, T>(x); }
};

// DFTs whose inputs beyond the first quarter are zero (x[R/4 ..] == 0), for
// the first stage of a transform zero-padded to four times its data.
template <int R, typename T>
struct DftQuarter;

template <typename T>
struct DftQuarter<8, T> {  // X_k = x0 + x1·ω8^k
    static __device__ __forceinline__ void run(cpx<T>* x) {
        const cpx<T> a = x[0], b = x[1];
        static_for<0, 8>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            x[k] = cadd(a, twiddle_const<8, k>(b));
        });
    }
};

template <typename T>
struct DftQuarter<16, T> {  // n = 4·n1 + n2 with n1 = 0: X[k1 + 4k2] = Σ_{n2<4} ω16^{n2·k1} ω4^{n2·k2} x[n2]
    static __device__ __forceinline__ void run(cpx<T>* x) {
        cpx<T> in[4] = {x[0], x[1], x[2], x[3]};
        static_for<0, 4>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            cpx<T> b[4];
            static_for<0, 4>([&](auto n2c) {
                constexpr int n2 = decltype(n2c)::value;
                b[n2] = twiddle_const<16, n2 * k1>(in[n2]);
            });
            Dft<4, T>::run(b);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = b[k2];
        });
    }
};

template <typename T>
struct Dft<6, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) { dft_split<3, 2, T>(x); }
};
template <typename T>
struct Dft<12, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) { dft_split<4, 3, T>(x); }
};
template <typename T>
struct Dft<16, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) { dft_split<4, 4, T>(x); }
};
template <typename T>
struct Dft<24, T> {
    static __device__ __forceinline__ void run(cpx<T>* x) { dft_split<8, 3, T>(x); }
};

// ---------------------------------------------------------------------------
// Runtime plan of one 1D length (host builds it, passed by value to kernels).
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 12;

struct FftPlan {
    int n;        // transform length
    int E;        // elements per thread
    int Tf;       // threads per transform = n / E
    int nstage;
    int radix[kMaxStages];
    int ns[kMaxStages];   // span before the stage (product of earlier radices)
    int tws[kMaxStages];  // n / (ns·radix): table stride of the stage twiddle
};

// Shared-memory views of one transform's exchange buffer.
//   S > 0  : column layout with compile-time stride S (element i at base[i·S]);
//   S == 0 : row layout, one pad slot per 16 elements (base[i + i/16]);
//   S < 0  : column layout with the runtime stride `stride`.
// Column layouts serve tiles whose lanes run across columns, the row layout
// tiles whose lanes run along the row.
template <typename T, int S = -1>
struct SmemCol {
    cpx<T>* base;
    int stride;
    __device__ __forceinline__ cpx<T>& operator[](int i) const {
        if constexpr (S > 0) {
            return base[i * S];
        } else if constexpr (S == 0) {
            return base[i + (i >> 4)];
        } else {
            return base[i * stride];
        }
    }
};
template <typename T>
using SmemRow = SmemCol<T, 0>;

// C interleaved columns with a skewed element index: element i of column c
// sits at base_c[C·(i + i/16)].  Lanes of a warp run over (c, t) with c
// fastest; with 4 t per warp (8-byte elements, C = 8) the skew splits every
// exchange access (stride-1 or stride-16 in t) evenly over the banks, so it
// takes the minimum two wavefronts.
template <typename T, int C>
struct SmemColSkew {
    cpx<T>* base;
    int unused;  // same initialiser shape as SmemCol
    __device__ __forceinline__ cpx<T>& operator[](int i) const { return base[C * (i + (i >> 4))]; }
};
// Complex slots of a skewed exchange buffer of C columns of n elements.
__host__ __device__ constexpr int skew_slots(int n, int C) { return C * (n + (n >> 4)); }

// Exchange view for C interleaved columns of a static kernel: once the C
// columns of one element index fill a 128-byte wavefront (C·sizeof(cpx<T>) ≥
// 128), a stride of C + 1 already spreads a warp's accesses evenly and needs
// no index arithmetic; narrower groups take the skewed layout.
template <typename T>
__host__ __device__ constexpr bool xchg_skewed(int C) { return C * (int)sizeof(cpx<T>) < 128; }
template <typename T, int C>
using XchgCol = typename std::conditional<xchg_skewed<T>(C), SmemColSkew<T, C>, SmemCol<T, C + 1>>::type;
template <typename T>
__host__ __device__ constexpr int xchg_slots(int n, int C) { return xchg_skewed<T>(C) ? skew_slots(n, C) : n * (C + 1); }
// A TMA-loaded [n][C] tile that later serves as the exchange: plain stride C
// for full wavefronts, else skewed (the tile then occupies the first n·C slots).
template <typename T, int C>
using TileCol = typename std::conditional<xchg_skewed<T>(C), SmemColSkew<T, C>, SmemCol<T, C>>::type;
template <typename T>
__host__ __device__ constexpr int tile_slots(int n, int C) { return xchg_skewed<T>(C) ? skew_slots(n, C) : n * C; }
// Complex slots of one row-layout buffer of n elements.
__host__ __device__ constexpr int padded_row(int n) { return n + (n >> 4) + 1; }

// One radix-R stage on the E register values of thread t.  If `last`, the
// outputs stay in registers (they land in the thread's own index set);
// otherwise they are written to the exchange buffer.
template <int R, int E, int NCOL, typename T, typename BUF>
__device__ __forceinline__ void stage_radix(cpx<T> (&v)[NCOL][E], int t, int Tf, int Ns, int tws,
                                            const cpx<T>* __restrict__ tw, const BUF (&buf)[NCOL], bool last) {
    constexpr int B = E / R;  // butterflies per thread
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int j = t + Tf * u;
        const int jm = j % Ns;
        const int base = (j - jm) * R + jm;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            cpx<T> x[R];
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = v[c][u + r * B];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) x[r] = cmul(x[r], tw[jm * r * tws]);
            }
            Dft<R, T>::run(x);
            if (last) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[c][u + r * B] = x[r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) buf[c][base + r * Ns] = x[r];
            }
        }
    }
}

// Full forward transform of NCOL independent columns held by this thread.
// Caller contract: every thread of the block calls this the same number of
// times (it contains __syncthreads), `tw` is the length-n table
// tw[k] = e^{-2πi k/n}, and the exchange buffers are not in use by anyone.
template <int E, int NCOL, typename T, typename BUF>
__device__ __forceinline__ void fft_forward(cpx<T> (&v)[NCOL][E], int t, const FftPlan& P,
                                            const cpx<T>* __restrict__ tw, const BUF (&buf)[NCOL]) {
    const int Tf = P.Tf;
    for (int s = 0; s < P.nstage; ++s) {
        const bool last = (s + 1 == P.nstage);
        const int R = P.radix[s], Ns = P.ns[s], tws = P.tws[s];
        if (!last) __syncthreads();  // previous readers of the buffer are done
        switch (R) {
            case 2:
                if constexpr (E % 2 == 0) stage_radix<2, E, NCOL, T, BUF>(v, t, Tf, Ns, tws, tw, buf, last);
                break;
            case 3:
                if constexpr (E % 3 == 0) stage_radix<3, E, NCOL, T, BUF>(v, t, Tf, Ns, tws, tw, buf, last);
                break;
            case 4:
                if constexpr (E % 4 == 0) stage_radix<4, E, NCOL, T, BUF>(v, t, Tf, Ns, tws, tw, buf, last);
                break;
            case 6:
                if constexpr (E % 6 == 0) stage_radix<6, E, NCOL, T, BUF>(v, t, Tf, Ns, tws, tw, buf, last);
                break;
            case 8:
                if constexpr (E % 8 == 0) stage_radix<8, E, NCOL, T, BUF>(v, t, Tf, Ns, tws, tw, buf, last);
                break;
            case 12:
                if constexpr (E % 12 == 0) stage_radix<12, E, NCOL, T, BUF>(v, t, Tf, Ns, tws, tw, buf, last);
                break;
            case 16:
                if constexpr (E % 16 == 0) stage_radix<16, E, NCOL, T, BUF>(v, t, Tf, Ns, tws, tw, buf, last);
                break;
            case 24:
                if constexpr (E % 24 == 0) stage_radix<24, E, NCOL, T, BUF>(v, t, Tf, Ns, tws, tw, buf, last);
                break;
            default:
                break;
        }
        if (!last) {
            __syncthreads();
#pragma unroll
            for (int c = 0; c < NCOL; ++c) {
#pragma unroll
                for (int e = 0; e < E; ++e) v[c][e] = buf[c][t + Tf * e];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Compile-time plans.  The same greedy radix choice as the host planner:
// repeatedly take the largest radix in {24,16,12,8,6,4,3,2} that divides both
// E and the remaining length.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr bool is_pow2_c(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Elements per thread for a length-n transform: 16 (FP32) or 8 (FP64) for
// powers of two, 24 or 12 for 3·2^a; FP64 at n = 2048 takes 16 so that the
// z pass (2·n/E threads per column) stays within 256 threads.
__host__ __device__ constexpr int plan_E(int n, bool f64) {
    if (is_pow2_c(n)) {
        const int e = f64 ? (n >= 2048 ? 16 : 8) : 16;
        return n < e ? n : e;
    }
    const int e = f64 ? 12 : 24;
    return n < e ? n : e;
}

__host__ __device__ constexpr int pick_radix(int E, int rem) {
    const int cand[8] = {24, 16, 12, 8, 6, 4, 3, 2};
    for (int i = 0; i < 8; ++i)
        if (E % cand[i] == 0 && rem % cand[i] == 0) return cand[i];
    return 0;
}
__host__ __device__ constexpr int static_nstage(int n, int E) {
    int rem = n, s = 0;
    while (rem > 1) {
        const int r = pick_radix(E, rem);
        if (r == 0) return -1;
        rem /= r;
        ++s;
    }
    return s;
}
__host__ __device__ constexpr int static_radix(int n, int E, int stage) {
    int rem = n, r = 0;
    for (int i = 0; i <= stage; ++i) {
        r = pick_radix(E, rem);
        rem /= r;
    }
    return r;
}
__host__ __device__ constexpr int static_ns(int n, int E, int stage) {
    int rem = n, ns = 1;
    for (int i = 0; i < stage; ++i) {
        const int r = pick_radix(E, rem);
        rem /= r;
        ns *= r;
    }
    return ns;
}

// One radix-R stage with every size known at compile time.
template <int R, int E, int NCOL, int Ns, int TWS, int TF, bool LAST, typename T, typename BUF>
__device__ __forceinline__ void stage_static(cpx<T> (&v)[NCOL][E], int t, const cpx<T>* __restrict__ tw,
                                             const BUF (&buf)[NCOL]) {
    constexpr int B = E / R;
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int j = t + TF * u;
        const int jm = j % Ns;
        const int base = (j - jm) * R + jm;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            cpx<T> x[R];
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = v[c][u + r * B];
            if constexpr (Ns > 1) {
                DftTw<R, T>::run(x, [&](int r) { return tw[jm * r * TWS]; });
            } else {
                Dft<R, T>::run(x);
            }
            if constexpr (LAST) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[c][u + r * B] = x[r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) buf[c][base + r * Ns] = x[r];
            }
        }
    }
}

template <int N, int E, int S, int NCOL, typename T, typename BUF>
__device__ __forceinline__ void fft_static(cpx<T> (&v)[NCOL][E], int t, const cpx<T>* __restrict__ tw,
                                           const BUF (&buf)[NCOL]) {
    constexpr int NST = static_nstage(N, E);
    static_assert(NST > 0 && NST <= kMaxStages, "length not supported by the radix set");
    if constexpr (S < NST) {
        constexpr int R = static_radix(N, E, S);
        constexpr int Ns = static_ns(N, E, S);
        constexpr int TWS = N / (Ns * R);
        constexpr int TF = N / E;
        constexpr bool LAST = (S + 1 == NST);
        if constexpr (!LAST) __syncthreads();
        stage_static<R, E, NCOL, Ns, TWS, TF, LAST, T, BUF>(v, t, tw, buf);
        if constexpr (!LAST) {
            __syncthreads();
#pragma unroll
            for (int c = 0; c < NCOL; ++c) {
#pragma unroll
                for (int e = 0; e < E; ++e) v[c][e] = buf[c][t + TF * e];
            }
        }
        fft_static<N, E, S + 1, NCOL, T, BUF>(v, t, tw, buf);
    }
}

// ---------------------------------------------------------------------------
// Stage-ordered twiddles.  A twiddled stage s (span Ns > 1, radix R) reads
// ω_N^{jm·r·TWS} for r < R and jm = j mod Ns; with lanes running along the
// transform (consecutive jm) the natural table index jm·r·TWS strides the
// banks by r.  The stage table holds the same values at [r - 1][jm], so that
// consecutive lanes read consecutive slots.  Stages are laid out one after
// the other; stage_tw_offset gives where stage s starts.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int stage_tw_offset(int N, int E, int S) {
    int off = 0;
    for (int s = 1; s < S; ++s) off += (static_radix(N, E, s) - 1) * static_ns(N, E, s);
    return off;
}
__host__ __device__ constexpr int stage_tw_size(int N, int E) { return stage_tw_offset(N, E, static_nstage(N, E)); }

// Fill the stage table from the natural table twg[k] = ω_N^k (global memory).
template <int N, int E, typename T>
__device__ __forceinline__ void build_stage_twiddles(cpx<T>* __restrict__ dst, const cpx<T>* __restrict__ twg) {
    constexpr int NST = static_nstage(N, E);
    static_for<1, NST>([&](auto sc) {
        constexpr int S = decltype(sc)::value;
        constexpr int R = static_radix(N, E, S), Ns = static_ns(N, E, S), TWS = N / (Ns * R);
        constexpr int off = stage_tw_offset(N, E, S);
        for (int i = threadIdx.x; i < (R - 1) * Ns; i += blockDim.x) {
            const int r = i / Ns + 1, jm = i - (r - 1) * Ns;
            dst[off + i] = twg[(jm * r * TWS) % N];
        }
    });
}

// One radix-R stage as stage_static, reading the stage table.
template <int R, int E, int NCOL, int Ns, int TF, int OFF, bool LAST, typename T, typename BUF>
__device__ __forceinline__ void stage_static_st(cpx<T> (&v)[NCOL][E], int t, const cpx<T>* __restrict__ twS,
                                                const BUF (&buf)[NCOL]) {
    constexpr int B = E / R;
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int j = t + TF * u;
        const int jm = j % Ns;
        const int base = (j - jm) * R + jm;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            cpx<T> x[R];
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = v[c][u + r * B];
            if constexpr (Ns > 1) {
                DftTw<R, T>::run(x, [&](int r) { return twS[OFF + (r - 1) * Ns + jm]; });
            } else {
                Dft<R, T>::run(x);
            }
            if constexpr (LAST) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[c][u + r * B] = x[r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) buf[c][base + r * Ns] = x[r];
            }
        }
    }
}

// fft_static with the stage table (build_stage_twiddles) instead of the natural one.
template <int N, int E, int S, int NCOL, typename T, typename BUF>
__device__ __forceinline__ void fft_static_st(cpx<T> (&v)[NCOL][E], int t, const cpx<T>* __restrict__ twS,
                                              const BUF (&buf)[NCOL]) {
    constexpr int NST = static_nstage(N, E);
    static_assert(NST > 0 && NST <= kMaxStages, "length not supported by the radix set");
    if constexpr (S < NST) {
        constexpr int R = static_radix(N, E, S);
        constexpr int Ns = static_ns(N, E, S);
        constexpr int TF = N / E;
        constexpr bool LAST = (S + 1 == NST);
        constexpr int OFF = stage_tw_offset(N, E, S);
        if constexpr (!LAST) __syncthreads();
        stage_static_st<R, E, NCOL, Ns, TF, OFF, LAST, T, BUF>(v, t, twS, buf);
        if constexpr (!LAST) {
            __syncthreads();
#pragma unroll
            for (int c = 0; c < NCOL; ++c) {
#pragma unroll
                for (int e = 0; e < E; ++e) v[c][e] = buf[c][t + TF * e];
            }
        }
        fft_static_st<N, E, S + 1, NCOL, T, BUF>(v, t, twS, buf);
    }
}

// Forward length-M transform of data whose upper half is zero: thread t holds
// v[e] = x[t + Tf·e] with v[e] = 0 for e ≥ E/2 (never read).  The first
// stage must have radix E (one butterfly per thread) so that exactly its
// upper inputs vanish.
template <int M, int E, int NCOL, typename T, typename BUF>
__device__ __forceinline__ void fft_static_padded(cpx<T> (&v)[NCOL][E], int t, const cpx<T>* __restrict__ tw,
                                                  const BUF (&buf)[NCOL]) {
    constexpr int NST = static_nstage(M, E);
    static_assert(static_radix(M, E, 0) == E, "padded first stage needs one butterfly per thread");
    static_assert(NST >= 2, "padded transform needs at least two stages");
    constexpr int TF = M / E;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
        cpx<T> x[E];
#pragma unroll
        for (int r = 0; r < E / 2; ++r) x[r] = v[c][r];
        DftHalf<E, T>::run(x);
#pragma unroll
        for (int r = 0; r < E; ++r) buf[c][t * E + r] = x[r];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[c][e] = buf[c][t + TF * e];
    }
    fft_static<M, E, 1, NCOL, T, BUF>(v, t, tw, buf);
}

// Forward length-M transform of data whose last three quarters are zero:
// v[e] = x[t + Tf·e] with v[e] = 0 for e ≥ E/4 (never read).
template <int M, int E, int NCOL, typename T, typename BUF>
__device__ __forceinline__ void fft_static_quarter(cpx<T> (&v)[NCOL][E], int t, const cpx<T>* __restrict__ tw,
                                                   const BUF (&buf)[NCOL]) {
    constexpr int NST = static_nstage(M, E);
    static_assert(static_radix(M, E, 0) == E, "pruned first stage needs one butterfly per thread");
    static_assert(NST >= 2, "padded transform needs at least two stages");
    constexpr int TF = M / E;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
        cpx<T> x[E];
#pragma unroll
        for (int r = 0; r < E / 4; ++r) x[r] = v[c][r];
        DftQuarter<E, T>::run(x);
#pragma unroll
        for (int r = 0; r < E; ++r) buf[c][t * E + r] = x[r];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[c][e] = buf[c][t + TF * e];
    }
    fft_static<M, E, 1, NCOL, T, BUF>(v, t, tw, buf);
}

// Forward transform: compile-time plan when NS > 0, else the runtime plan P.
template <int NS, int E, int NCOL, typename T, typename BUF>
__device__ __forceinline__ void fft_run(cpx<T> (&v)[NCOL][E], int t, const FftPlan& P, const cpx<T>* __restrict__ tw,
                                        const BUF (&buf)[NCOL]) {
    if constexpr (NS > 0) {
        fft_static<NS, E, 0, NCOL, T, BUF>(v, t, tw, buf);
    } else {
        fft_forward<E, NCOL, T, BUF>(v, t, P, tw, buf);
    }
}

}  // namespace sbp
