// sbp_force.cuh — ghost layers and forces from a solution (Sect. 2.4, last
// paragraph: beyond the last active cell in z the potential keeps that cell's
// gradient, so the ghost layers continue Φ linearly).
//
//   k_fill_ghosts   out[nz + 2 ng][ny][nx]: Φ in the middle, ng continued
//                   layers below and above (one thread per output element)
//   k_force         g = -∇Φ by second-order central differences, [3][nz][ny][nx];
//                   y periodic, x periodic or (physical frame) shear-periodic,
//                   z one-sided in the boundary cells (the ghost rule)
//   k_shear_cols    physical frame: the x-neighbours across the shearing
//                   boundary, Φ(x_0, y + Δy0) and Φ(x_{nx-1}, y - Δy0), by
//                   Fourier interpolation of the two boundary columns
#pragma once

#include "sbp_remap.cuh"

namespace sbp {

// Output plane zo of the ghost-filled array, one element per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_fill_ghosts(const T* __restrict__ phi, T* __restrict__ out, int plane,
                                                     int nz, int ng) {
    const int zo = blockIdx.y;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // element of the plane
    if (i >= plane) return;
    T v;
    if (zo >= ng && zo < ng + nz) {
        v = __ldcs(phi + (size_t)(zo - ng) * plane + i);
    } else if (zo >= ng + nz) {  // above: Φ(nz-1) + g (Φ(nz-1) - Φ(nz-2))
        const T a = phi[(size_t)(nz - 1) * plane + i], b = phi[(size_t)(nz - 2) * plane + i];
        v = fma((T)(zo - (ng + nz - 1)), a - b, a);
    } else {  // below: Φ(0) - g (Φ(1) - Φ(0))
        const T a = phi[i], b = phi[(size_t)plane + i];
        v = fma((T)(ng - zo), a - b, a);
    }
    __stcs(out + (size_t)zo * plane + i, v);
}

// Planes per block of k_shear_cols: one warp at least, so that the few
// blocks (nz / CP) still spread over the SMs.
__host__ __device__ constexpr int shear_cols_planes(int Tf) { return Tf >= 32 ? 1 : 32 / Tf; }

// Physical frame: side[z][0][y] = Φ(x_0, y + Δy0) (right neighbour of column
// nx-1) and side[z][1][y] = Φ(x_{nx-1}, y - Δy0) (left neighbour of column 0).
// Block = CP planes; plane z's two boundary columns form one complex
// transform Z = Φ(x_0) + i Φ(x_{nx-1}), split into A, B, phased by
// exp(±2πi k_s u), u = Δy0/L_y (the Nyquist term by the real part), and
// transformed back.  smem: tw[NY] | exchange (XchgCol)
template <typename T, int E, int NY, int CP>
__global__ void __launch_bounds__(kMaxThreads) k_shear_cols(const T* __restrict__ phi, T* __restrict__ side,
                                                            const cpx<T>* __restrict__ twg, int nx, int nz,
                                                            double u) {
    constexpr int Tf = NY / E;
    constexpr int H = NY / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* xb = tw + NY;
    const int tid = threadIdx.x;
    for (int i = tid; i < NY; i += blockDim.x) tw[i] = twg[i];
    const int c = tid % CP, t = tid / CP;
    const int z = blockIdx.x * CP + c;
    const bool valid = z < nz;
    cpx<T> v[1][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int y = t + Tf * e;
        cpx<T> x = {(T)0, (T)0};
        if (valid) {
            const T* row = phi + ((size_t)z * NY + y) * nx;
            x = {row[0], row[nx - 1]};
        }
        v[0][e] = x;
    }
    __syncthreads();  // twiddles visible
    const XchgCol<T, CP> buf[1] = {{xb + c, 0}};
    fft_static<NY, E, 0, 1, T>(v, t, tw, buf);  // Z_k at k = t + Tf·e
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) buf[0][t + Tf * e] = v[0][e];
    __syncthreads();
    const typename TurnFix<T>::U uf = TurnFix<T>::from(u);
    const T half = (T)0.5;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + Tf * e;
        const cpx<T> Zk = v[0][e];
        const cpx<T> Zm = cconj(buf[0][k == 0 ? 0 : NY - k]);
        cpx<T> a = {(Zk.x + Zm.x) * half, (Zk.y + Zm.y) * half};
        cpx<T> b = {(Zk.y - Zm.y) * half, (Zm.x - Zk.x) * half};
        const int ks = (k < H) ? k : k - NY;  // signed y-frequency
        const cpx<T> w = TurnFix<T>::phase(ks, uf);  // e^{+2πi k_s u}
        if (k == H) {
            a = {a.x * w.x, (T)0};
            b = {b.x * w.x, (T)0};
        } else {
            a = cmul(a, w);         // column 0 read at y + Δy0
            b = cmul(b, cconj(w));  // column nx-1 read at y - Δy0
        }
        v[0][e] = cconj(cpx<T>{a.x - b.y, a.y + b.x});
    }
    fft_static<NY, E, 0, 1, T>(v, t, tw, buf);  // its first exchange write follows a barrier
    if (!valid) return;
    const T inv = (T)1 / (T)NY;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int y = t + Tf * e;
        side[((size_t)z * 2 + 0) * NY + y] = v[0][e].x * inv;
        side[((size_t)z * 2 + 1) * NY + y] = -v[0][e].y * inv;
    }
}

// g = -∇Φ.  Thread = one (x, y) column over ZC consecutive planes, keeping a
// three-plane window in registers; x and y neighbours come through L1.
// side (physical frame) holds the shifted boundary columns, else null.
template <typename T, int ZC>
__global__ void __launch_bounds__(256) k_force(const T* __restrict__ phi, T* __restrict__ g,
                                               const T* __restrict__ side, int nx, int ny, int nz, T rdx2, T rdy2,
                                               T rdz) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int z0 = blockIdx.z * ZC;
    const int z1 = min(nz, z0 + ZC);
    const size_t plane = (size_t)nx * ny;
    const size_t N = plane * nz;
    const int xl = (x == 0) ? nx - 1 : x - 1, xr = (x == nx - 1) ? 0 : x + 1;
    const int yl = (y == 0) ? ny - 1 : y - 1, yr = (y == ny - 1) ? 0 : y + 1;
    const T* col = phi + (size_t)y * nx + x;
    T below = (z0 > 0) ? col[(size_t)(z0 - 1) * plane] : (T)0;
    T cur = col[(size_t)z0 * plane];
    for (int z = z0; z < z1; ++z) {
        const T above = (z + 1 < nz) ? col[(size_t)(z + 1) * plane] : (T)0;
        const T* pl = phi + (size_t)z * plane;
        T r = pl[(size_t)y * nx + xr], l = pl[(size_t)y * nx + xl];
        if (side != nullptr) {
            if (x == nx - 1) r = side[((size_t)z * 2 + 0) * ny + y];
            if (x == 0) l = side[((size_t)z * 2 + 1) * ny + y];
        }
        const T u = pl[(size_t)yr * nx + x], d = pl[(size_t)yl * nx + x];
        T gz;
        if (nz == 1) {
            gz = (T)0;
        } else if (z == 0) {
            gz = -(above - cur) * rdz;
        } else if (z == nz - 1) {
            gz = -(cur - below) * rdz;
        } else {
            gz = -(above - below) * (T)0.5 * rdz;
        }
        const size_t o = (size_t)z * plane + (size_t)y * nx + x;
        __stcs(g + o, -(r - l) * rdx2);
        __stcs(g + N + o, -(u - d) * rdy2);
        __stcs(g + 2 * N + o, gz);
        below = cur;
        cur = above;
    }
}

}  // namespace sbp
