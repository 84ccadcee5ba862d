// 1-D DGFS right-hand side (arXiv:1809.10186, Sec. 3.1 eq. eq_weakForm with the upwind flux of
// eq. eq_numericalFlux_upwind, and the fully diffuse wall condition of Sec. 3.6).
//
// Layout: F [I][K][N^3], element-major, the K Gauss-Lobatto nodes of an element next to each other.
// For element i of width h_i and velocity c (c_1 its x component):
//   dF/dt = (2/h_i) M^{-1} (c_1 S F - Fl) + (1/Kn) M^{-1} C,
//   Fl_m = [m = K-1] F*_R - [m = 0] F*_L,  F*_R = c_1 (c_1 >= 0 ? F_{K-1} : right exterior),
//   F*_L = c_1 (c_1 <= 0 ? F_0 : left exterior),
// with C the element collision term sum H Q (k_dg.cu and the collision path). At a wall the
// exterior value is n_w f_w(c), n_w = (sum over outgoing c of |c_1| f) / (sum over incoming c of
// |c_1| f_w); k_slab_wall reduces the numerators in FP64, the denominators are host constants.
// Both kernels are memory-bound streams over the I K N^3 values.
#include <cstdint>

#include "launchers.h"

namespace dgfs {

namespace {

// one CTA per wall: side 0 reads the first node of element 0 (outgoing c_1 < 0), side 1 the last
// node of element I - 1 (outgoing c_1 > 0)
template <typename T>
__global__ void __launch_bounds__(256) k_slab_wall(const T* __restrict__ F, int N, int I, int K, double L,
                                                   double* __restrict__ num) {
    __shared__ double part[8];
    const int side = blockIdx.x;
    const int64_t n3 = (int64_t)N * N * N, n2 = (int64_t)N * N;
    const T* f = F + (side == 0 ? 0 : ((int64_t)(I - 1) * K + (K - 1)) * n3);
    const double dc = 2.0 * L / N;
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n3; j += blockDim.x) {
        const double c1 = -L + ((double)(j / n2) + 0.5) * dc;
        if (side == 0 ? c1 < 0.0 : c1 > 0.0) acc += fabs(c1) * (double)f[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += part[w];
        num[side] = s;
    }
}

// thread per (velocity j, element i = blockIdx.y)
template <typename T, int K>
__global__ void __launch_bounds__(256) k_slab_rhs(const T* __restrict__ F, const T* __restrict__ C,
                                                  const T* __restrict__ fw, const double* __restrict__ num,
                                                  SlabMatrices mats, const double* __restrict__ hinv2, double invKn,
                                                  int N, int I, double L, T* __restrict__ out) {
    const int64_t n3 = (int64_t)N * N * N, n2 = (int64_t)N * N;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= n3) return;
    const T c1 = (T)(-L + ((double)(j / n2) + 0.5) * (2.0 * L / N));
    const T* Fi = F + (int64_t)i * K * n3 + j;
    T v[K];
#pragma unroll
    for (int l = 0; l < K; ++l) v[l] = Fi[l * n3];
    T fL, fR;
    if (c1 > T(0)) {   // the left face takes the exterior (upstream) value, the right face the interior
        fL = i > 0 ? Fi[-n3] : (T)(num[0] / mats.den[0]) * fw[j];
        fR = v[K - 1];
    } else {
        fL = v[0];
        fR = i < I - 1 ? Fi[K * n3] : (T)(num[1] / mats.den[1]) * fw[n3 + j];
    }
    T t[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
        T s = 0;
#pragma unroll
        for (int l = 0; l < K; ++l) s = fma((T)mats.S[m * K + l], v[l], s);
        t[m] = c1 * s;
    }
    t[K - 1] -= c1 * fR;
    t[0] += c1 * fL;
    const T h2 = (T)hinv2[i], ik = (T)invKn;
    T* oi = out + (int64_t)i * K * n3 + j;
#pragma unroll
    for (int m = 0; m < K; ++m) {
        T s = 0;
#pragma unroll
        for (int l = 0; l < K; ++l) {
            T w = h2 * t[l];
            if (C) w = fma(ik, C[((int64_t)i * K + l) * n3 + j], w);
            s = fma((T)mats.Minv[m * K + l], w, s);
        }
        oi[m * n3] = s;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_slab_wall(const T* F, int N, int I, int K, double L, double* num, cudaStream_t s) {
    k_slab_wall<T><<<2, 256, 0, s>>>(F, N, I, K, L, num);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_slab_rhs(const T* F, const T* C, const T* fw, const double* num, const SlabMatrices& mats,
                            const double* hinv2, double invKn, int N, int I, double L, T* out, cudaStream_t s) {
    if (I <= 0) return cudaSuccess;
    if (I > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    const dim3 grid((unsigned)((n3 + 255) / 256), (unsigned)I);
    switch (mats.K) {
#define DGFS_SLAB_K(KK) \
    case KK: k_slab_rhs<T, KK><<<grid, 256, 0, s>>>(F, C, fw, num, mats, hinv2, invKn, N, I, L, out); break;
        DGFS_SLAB_K(2) DGFS_SLAB_K(3) DGFS_SLAB_K(4) DGFS_SLAB_K(5) DGFS_SLAB_K(6) DGFS_SLAB_K(7) DGFS_SLAB_K(8)
#undef DGFS_SLAB_K
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_slab_wall<float>(const float*, int, int, int, double, double*, cudaStream_t);
template cudaError_t launch_slab_wall<double>(const double*, int, int, int, double, double*, cudaStream_t);
template cudaError_t launch_slab_rhs<float>(const float*, const float*, const float*, const double*,
                                            const SlabMatrices&, const double*, double, int, int, double, float*,
                                            cudaStream_t);
template cudaError_t launch_slab_rhs<double>(const double*, const double*, const double*, const double*,
                                             const SlabMatrices&, const double*, double, int, int, double, double*,
                                             cudaStream_t);

}  // namespace dgfs
