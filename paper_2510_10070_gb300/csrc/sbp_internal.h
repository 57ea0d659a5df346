// sbp_internal.h — host-side view of the pass kernels (shared by the
// instantiation units and the API unit).
#pragma once

#include <cuda_runtime.h>

#include "sbp_kernels.cuh"
#include "sbp_force.cuh"
#include "sbp_remap.cuh"
#include "sbp_sweep.cuh"
#include "sbp_xy.cuh"

namespace sbp {

template <typename T>
struct KernelSet {
    void (*x_fwd)(const T*, cpx<T>*, const cpx<T>*, double*, XArgs) = nullptr;
    void (*x_inv)(const cpx<T>*, T*, const cpx<T>*, XArgs) = nullptr;
    void (*y_fwd)(cpx<T>*, const cpx<T>*, YArgs) = nullptr;  // static lengths: C = ypass_cols(n)
    // TMA y passes (static lengths only; C = ypass_cols(n))
    void (*y_fwd_tma)(cpx<T>*, const cpx<T>*, YArgs, TmaCtl, const CUtensorMap) = nullptr;
    void (*y_inv_tma)(cpx<T>*, const cpx<T>*, YArgs, TmaCtl, const CUtensorMap) = nullptr;
    void (*y_inv)(cpx<T>*, const cpx<T>*, YArgs) = nullptr;
    void (*z)(cpx<T>*, const cpx<T>*, const cpx<T>*, const T*, ZArgs) = nullptr;  // default z variant
};

// z-pass variants: elements per thread and joint / split halves.
template <typename T>
using ZKernel = void (*)(cpx<T>*, const cpx<T>*, const cpx<T>*, const T*, ZArgs);
struct ZVariant {
    int E;
    bool joint;
};

// Kernel sets.  Generic sets (runtime length, compile-time elements per
// thread E) cover every supported length; static sets (compile-time length N)
// cover the common lengths with a fully unrolled plan.  Each set is defined in
// one of the sbp_k_*.cu units so that they compile in parallel.
#define SBP_E_LIST_F32(X) X(float, f32, 2) X(float, f32, 3) X(float, f32, 4) X(float, f32, 6) \
    X(float, f32, 8) X(float, f32, 12) X(float, f32, 16) X(float, f32, 24)
#define SBP_E_LIST_F64(X) X(double, f64, 2) X(double, f64, 3) X(double, f64, 4) X(double, f64, 6) \
    X(double, f64, 8) X(double, f64, 12) X(double, f64, 16)
#define SBP_N_LIST_F32(X) X(float, f32, 32) X(float, f32, 64) X(float, f32, 96) X(float, f32, 128) \
    X(float, f32, 192) X(float, f32, 256) X(float, f32, 512) X(float, f32, 1024)
#define SBP_N_LIST_F64(X) X(double, f64, 32) X(double, f64, 64) X(double, f64, 96) X(double, f64, 128) \
    X(double, f64, 192) X(double, f64, 256) X(double, f64, 512) X(double, f64, 1024)

#define SBP_DECLARE_SET(T, TAG, E) KernelSet<T> kernels_##TAG##_e##E();
#define SBP_DECLARE_SET_N(T, TAG, N) KernelSet<T> kernels_##TAG##_n##N();
SBP_E_LIST_F32(SBP_DECLARE_SET)
SBP_E_LIST_F64(SBP_DECLARE_SET)
SBP_N_LIST_F32(SBP_DECLARE_SET_N)
SBP_N_LIST_F64(SBP_DECLARE_SET_N)

#define SBP_CASE_SET(T, TAG, E) \
    case E:                     \
        return kernels_##TAG##_e##E();
#define SBP_CASE_SET_N(T, TAG, N) \
    case N:                       \
        return kernels_##TAG##_n##N();

// Extra static z-pass variants (length N, E, joint), defined next to the
// static sets; zvariant_for returns null when a variant is not built.
#define SBP_ZVAR_LIST(X) X(float, f32, 128, 8, 1) X(float, f32, 128, 8, 0) X(float, f32, 256, 8, 1) \
    X(float, f32, 256, 8, 0) X(float, f32, 64, 8, 1) X(float, f32, 512, 8, 1)
// Padded z variant (one length-2N transform per column): (type, N, E).
#define SBP_ZPAD_LIST(X) X(float, f32, 32, 16) X(float, f32, 64, 16) X(float, f32, 96, 24) X(float, f32, 128, 16) \
    X(float, f32, 192, 24) X(float, f32, 256, 16) X(float, f32, 512, 16) X(double, f64, 32, 8) X(double, f64, 64, 8) \
    X(double, f64, 128, 8) X(double, f64, 256, 8)
#define SBP_DECLARE_ZPAD(T, TAG, N, E) ZKernel<T> zpad_##TAG##_n##N();
SBP_ZPAD_LIST(SBP_DECLARE_ZPAD)
#define SBP_DEFINE_ZPAD(T, TAG, N, E) \
    ZKernel<T> zpad_##TAG##_n##N() { return k_z_padded<T, E, N>; }

// Paper-parameter z variant (α ≠ 1, 4× padding): (type, N, E).
#define SBP_ZPAPER_LIST(X) X(float, f32, 32, 16) X(float, f32, 64, 16) X(float, f32, 128, 16) \
    X(float, f32, 256, 16) X(float, f32, 512, 16) X(double, f64, 32, 8) X(double, f64, 64, 8) X(double, f64, 128, 8) \
    X(double, f64, 256, 8)
#define SBP_DECLARE_ZPAPER(T, TAG, N, E) ZKernel<T> zpaper_##TAG##_n##N();
SBP_ZPAPER_LIST(SBP_DECLARE_ZPAPER)
#define SBP_DEFINE_ZPAPER(T, TAG, N, E) \
    ZKernel<T> zpaper_##TAG##_n##N() { return k_z_paper<T, E, N>; }

template <typename T>
inline ZKernel<T> zpaper_for(int n, int* E_out) {
#define SBP_MATCH_ZPAPER(TT, TAG, N, EE)                                 \
    if (std::is_same<T, TT>::value && n == N) {                          \
        *E_out = EE;                                                     \
        return reinterpret_cast<ZKernel<T>>(zpaper_##TAG##_n##N());      \
    }
    SBP_ZPAPER_LIST(SBP_MATCH_ZPAPER)
#undef SBP_MATCH_ZPAPER
    return nullptr;
}

// Padded z kernel for length n and its elements per thread (null if not built).
template <typename T>
inline ZKernel<T> zpad_for(int n, int* E_out) {
#define SBP_MATCH_ZPAD(TT, TAG, N, EE)                                   \
    if (std::is_same<T, TT>::value && n == N) {                          \
        *E_out = EE;                                                     \
        return reinterpret_cast<ZKernel<T>>(zpad_##TAG##_n##N());        \
    }
    SBP_ZPAD_LIST(SBP_MATCH_ZPAD)
#undef SBP_MATCH_ZPAD
    return nullptr;
}
#define SBP_DECLARE_ZVAR(T, TAG, N, E, J) ZKernel<T> zkernel_##TAG##_n##N##_e##E##_j##J();
SBP_ZVAR_LIST(SBP_DECLARE_ZVAR)
#define SBP_DEFINE_ZVAR(T, TAG, N, E, J) \
    ZKernel<T> zkernel_##TAG##_n##N##_e##E##_j##J() { return k_z_pass<T, E, N, (J != 0)>; }

template <typename T>
inline ZKernel<T> zvariant_for(int n, int E, bool joint) {
#define SBP_MATCH_ZVAR(TT, TAG, N, EE, J)                                                   \
    if (std::is_same<T, TT>::value && n == N && E == EE && joint == (J != 0))               \
        return reinterpret_cast<ZKernel<T>>(zkernel_##TAG##_n##N##_e##EE##_j##J());
    SBP_ZVAR_LIST(SBP_MATCH_ZVAR)
#undef SBP_MATCH_ZVAR
    return nullptr;
}

// Fused xy kernels for square planes nx = ny = N (one z-plane per cluster).
template <typename T>
struct XYKernels {
    void (*fwd)(const T*, cpx<T>*, const cpx<T>*, XYArgs) = nullptr;
    void (*inv)(const cpx<T>*, T*, const cpx<T>*, XYArgs) = nullptr;
    int cluster = 0, threads = 0;
    size_t smem_fwd = 0, smem_inv = 0;
};
// (type, N, variant): variant 1 = one CTA per SM, 2 = two CTAs per SM.
#define SBP_XY_LIST(X) X(float, f32, 64, 1) X(float, f32, 96, 1) X(float, f32, 128, 1) X(float, f32, 192, 1) \
    X(float, f32, 256, 1) X(float, f32, 512, 1) X(double, f64, 64, 1) X(double, f64, 128, 1) X(double, f64, 256, 1) \
    X(float, f32, 128, 2) X(float, f32, 192, 2) X(float, f32, 256, 2) X(float, f32, 512, 2)
#define SBP_DECLARE_XY(T, TAG, N, V) XYKernels<T> xy_##TAG##_n##N##_v##V();
SBP_XY_LIST(SBP_DECLARE_XY)
#define SBP_DEFINE_XY(T, TAG, N, V)                                \
    XYKernels<T> xy_##TAG##_n##N##_v##V() {                        \
        constexpr int CL = xy_cluster<T, N, (V == 1 ? kXYSmemOnePerSM : kXYSmemTwoPerSM)>(); \
        using SH = XYShape<T, N, CL>;                              \
        XYKernels<T> k;                                            \
        k.fwd = k_xy_forward<T, N, CL>;                            \
        k.inv = k_xy_inverse<T, N, CL>;                            \
        k.cluster = CL;                                            \
        k.threads = SH::NT;                                        \
        k.smem_fwd = SH::smem_fwd;                                 \
        k.smem_inv = SH::smem_inv;                                 \
        return k;                                                  \
    }

template <typename T>
inline XYKernels<T> xy_kernels_for(int n, int variant) {
#define SBP_MATCH_XY(TT, TAG, N, V)                                               \
    if (std::is_same<T, TT>::value && n == N && variant == V) {                   \
        auto k = xy_##TAG##_n##N##_v##V();                                        \
        XYKernels<T> r;                                                           \
        r.fwd = reinterpret_cast<decltype(r.fwd)>(k.fwd);                         \
        r.inv = reinterpret_cast<decltype(r.inv)>(k.inv);                         \
        r.cluster = k.cluster;                                                    \
        r.threads = k.threads;                                                    \
        r.smem_fwd = k.smem_fwd;                                                  \
        r.smem_inv = k.smem_inv;                                                  \
        return r;                                                                 \
    }
    SBP_XY_LIST(SBP_MATCH_XY)
#undef SBP_MATCH_XY
    return XYKernels<T>{};
}

// Physical-frame passes (static lengths): y kernels with the mapping of
// Sect. 2.1 fused in (length ny) and complex row transforms (length nx).
template <typename T>
struct RemapKernels {
    void (*ry_fwd)(const T*, cpx<T>*, const cpx<T>*, double*, RArgs) = nullptr;
    void (*ry_inv)(const cpx<T>*, T*, const cpx<T>*, RArgs) = nullptr;
    int ry_E = 0, ry_C = 0;
    void (*rows_fwd)(cpx<T>*, const cpx<T>*, int, int) = nullptr;
    void (*rows_inv)(cpx<T>*, const cpx<T>*, int, int) = nullptr;
    int rows_E = 0;
    // shifted boundary columns for the physical-frame force (length ny)
    void (*shear_cols)(const T*, T*, const cpx<T>*, int, int, double) = nullptr;
};
#define SBP_DECLARE_REMAP(T, TAG, N) \
    RemapKernels<T> remap_y_##TAG##_n##N(); \
    RemapKernels<T> remap_x_##TAG##_n##N();
SBP_N_LIST_F32(SBP_DECLARE_REMAP)
SBP_N_LIST_F64(SBP_DECLARE_REMAP)
#define SBP_DEFINE_REMAP_Y(T, TAG, N)                                  \
    RemapKernels<T> remap_y_##TAG##_n##N() {                           \
        constexpr int E = plan_E(N, sizeof(T) == 8);                   \
        constexpr int CP = ypass_cols(N, sizeof(T) == 8);              \
        RemapKernels<T> k;                                             \
        k.ry_fwd = k_ry_forward<T, E, N, CP>;                          \
        k.ry_inv = k_ry_inverse<T, E, N, CP>;                          \
        k.shear_cols = k_shear_cols<T, E, N, shear_cols_planes(N / E)>; \
        k.ry_E = E;                                                    \
        k.ry_C = CP;                                                   \
        return k;                                                      \
    }
#define SBP_DEFINE_REMAP_X(T, TAG, N)                                  \
    RemapKernels<T> remap_x_##TAG##_n##N() {                           \
        constexpr int E = plan_E(N, sizeof(T) == 8);                   \
        RemapKernels<T> k;                                             \
        k.rows_fwd = k_rows_c2c<T, E, N, false>;                       \
        k.rows_inv = k_rows_c2c<T, E, N, true>;                        \
        k.rows_E = E;                                                  \
        return k;                                                      \
    }

// The y kernels for ny merged with the row kernels for nx (null if not built).
template <typename T>
inline RemapKernels<T> remap_kernels_for(int nx, int ny) {
    RemapKernels<T> r, x;
#define SBP_MATCH_REMAP(TT, TAG, N)                                                     \
    if (std::is_same<T, TT>::value && ny == N) {                                        \
        auto k = remap_y_##TAG##_n##N();                                                \
        r.ry_fwd = reinterpret_cast<decltype(r.ry_fwd)>(k.ry_fwd);                      \
        r.ry_inv = reinterpret_cast<decltype(r.ry_inv)>(k.ry_inv);                      \
        r.shear_cols = reinterpret_cast<decltype(r.shear_cols)>(k.shear_cols);          \
        r.ry_E = k.ry_E;                                                                \
        r.ry_C = k.ry_C;                                                                \
    }                                                                                   \
    if (std::is_same<T, TT>::value && nx == N) {                                        \
        auto k = remap_x_##TAG##_n##N();                                                \
        x.rows_fwd = reinterpret_cast<decltype(x.rows_fwd)>(k.rows_fwd);                \
        x.rows_inv = reinterpret_cast<decltype(x.rows_inv)>(k.rows_inv);                \
        x.rows_E = k.rows_E;                                                            \
    }
    SBP_N_LIST_F32(SBP_MATCH_REMAP)
    SBP_N_LIST_F64(SBP_MATCH_REMAP)
#undef SBP_MATCH_REMAP
    r.rows_fwd = x.rows_fwd;
    r.rows_inv = x.rows_inv;
    r.rows_E = x.rows_E;
    return r;
}

// Three-sweep kernels (FP32) for the box shapes (NX, NY, NZ) built below.
struct SweepKernels {
    void (*fwd)(SweepArgs) = nullptr;
    void (*mid)(SweepArgs) = nullptr;
    void (*inv)(SweepArgs) = nullptr;
    int nta = 0, ntb = 0, za = 0, ra = 0, rb = 0, nga = 0;
    size_t smem_ac = 0, smem_b = 0;
    bool green_mid = false;  // pass B evaluates the Green's parameters itself (no table fill in pass A)
};
#define SBP_SWEEP_LIST(X) X(32, 32, 32) X(64, 64, 32) X(64, 64, 64) X(128, 128, 64) X(128, 128, 128) \
    X(192, 192, 96) X(256, 256, 64) X(256, 256, 128)
#define SBP_DECLARE_SWEEP(NX, NY, NZ) SweepKernels sweep_##NX##_##NY##_##NZ();
SBP_SWEEP_LIST(SBP_DECLARE_SWEEP)
#define SBP_DEFINE_SWEEP(NX, NY, NZ)                   \
    SweepKernels sweep_##NX##_##NY##_##NZ() {          \
        using SH = SweepShape<NX, NY, NZ>;             \
        SweepKernels k;                                \
        k.fwd = k3_forward<NX, NY, NZ>;                \
        k.mid = k3_middle<NX, NY, NZ>;                 \
        k.inv = k3_inverse<NX, NY, NZ>;                \
        k.nta = SH::NTA;                               \
        k.ntb = SH::NTB;                               \
        k.za = SH::ZA;                                 \
        k.ra = SH::RA;                                 \
        k.rb = SH::RB;                                 \
        k.nga = SH::NGA;                               \
        k.smem_ac = SH::smem_ac;                       \
        k.smem_b = SH::smem_b;                         \
        k.green_mid = SH::GREEN_MID;                   \
        return k;                                      \
    }

inline SweepKernels sweep_kernels_for(int nx, int ny, int nz) {
#define SBP_MATCH_SWEEP(NX, NY, NZ) \
    if (nx == NX && ny == NY && nz == NZ) return sweep_##NX##_##NY##_##NZ();
    SBP_SWEEP_LIST(SBP_MATCH_SWEEP)
#undef SBP_MATCH_SWEEP
    return SweepKernels{};
}

// True when length n has static kernels for type T.
template <typename T>
inline bool is_static_len(int n) {
#define SBP_IS_STATIC(TT, TAG, N) \
    if (std::is_same<T, TT>::value && n == N) return true;
    SBP_N_LIST_F32(SBP_IS_STATIC)
    SBP_N_LIST_F64(SBP_IS_STATIC)
#undef SBP_IS_STATIC
    return false;
}

// Kernels for a length-n transform with E elements per thread.
template <typename T>
inline KernelSet<T> kernels_for(int n, int E);
template <>
inline KernelSet<float> kernels_for<float>(int n, int E) {
    switch (n) { SBP_N_LIST_F32(SBP_CASE_SET_N) default: break; }
    switch (E) { SBP_E_LIST_F32(SBP_CASE_SET) default: return KernelSet<float>{}; }
}
template <>
inline KernelSet<double> kernels_for<double>(int n, int E) {
    switch (n) { SBP_N_LIST_F64(SBP_CASE_SET_N) default: break; }
    switch (E) { SBP_E_LIST_F64(SBP_CASE_SET) default: return KernelSet<double>{}; }
}

}  // namespace sbp

#define SBP_SET_BODY(T, E, NS)                                                  \
    KernelSet<T> s;                                                             \
    s.x_fwd = k_x_forward<T, E, NS>;                                            \
    s.x_inv = k_x_inverse<T, E, NS>;                                            \
    s.y_fwd = k_y_pass<T, E, false, NS, (NS > 0 ? ypass_cols(NS, sizeof(T) == 8) : 0)>; \
    s.y_inv = k_y_pass<T, E, true, NS, (NS > 0 ? ypass_cols(NS, sizeof(T) == 8) : 0)>;  \
    s.z = k_z_pass<T, E, NS, false>;                                            \
    return s;

// Defines kernels_<TAG>_e<E>() (generic) in the including unit.
#define SBP_DEFINE_SET(T, TAG, E) \
    KernelSet<T> kernels_##TAG##_e##E() { SBP_SET_BODY(T, E, 0) }
// Defines kernels_<TAG>_n<N>() (static length N) in the including unit.
#define SBP_DEFINE_SET_N(T, TAG, N)                                                             \
    KernelSet<T> kernels_##TAG##_n##N() {                                                       \
        KernelSet<T> s = []() { SBP_SET_BODY(T, plan_E(N, sizeof(T) == 8), N) }();              \
        s.y_fwd_tma = k_y_tma<T, plan_E(N, sizeof(T) == 8), false, N, ypass_cols(N, sizeof(T) == 8)>; \
        s.y_inv_tma = k_y_tma<T, plan_E(N, sizeof(T) == 8), true, N, ypass_cols(N, sizeof(T) == 8)>;  \
        return s;                                                                               \
    }
