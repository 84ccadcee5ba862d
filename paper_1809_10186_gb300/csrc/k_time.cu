// Space-homogeneous time stepping and velocity moments (arXiv:1809.10186, Sec. 3.3 eq. moments1
// and Sec. 3.5 eqs. SSPRK2, SSPRK3).
//
// k_rk_combine forms one SSP-RK stage, out = a u + b v + c q, elementwise over a batch of fields;
// k_moments reduces every node's field to its mid-point-rule moments n, u, T, P, q and Boltzmann's
// H = int f ln f (over f > 0) in FP64, one CTA per node.
#include <cstdint>

#include "launchers.h"

namespace dgfs {

namespace {

template <typename T>
__global__ void k_rk_combine(int64_t n, double a, const T* __restrict__ u, double b, const T* __restrict__ v,
                             double c, const T* __restrict__ q, T* __restrict__ out, int* __restrict__ flags) {
    const T ta = (T)a, tb = (T)b, tc = (T)c;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T r = ta * u[i] + tc * q[i];
        if (v) r += tb * v[i];
        if (!isfinite(r)) atomicOr(flags, 2);
        out[i] = r;
    }
}

// sum over the block of NV doubles per thread (blockDim.x = 256); the result is in s[0..NV) for thread 0
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* s) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();   // s may hold the previous reduction
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) s[warp * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < 8; ++w)
#pragma unroll
            for (int k = 0; k < NV; ++k) s[k] += s[w * NV + k];
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_moments(const T* __restrict__ f, int N, double L, double* __restrict__ out) {
    __shared__ double s[8 * 11];
    const int64_t node = blockIdx.x, n3 = (int64_t)N * N * N;
    const T* fn = f + node * n3;
    const double dc = 2.0 * L / N, dv = dc * dc * dc;
    double a[4] = {0, 0, 0, 0};   // sum f, f c_x, f c_y, f c_z
    for (int64_t j = threadIdx.x; j < n3; j += blockDim.x) {
        const double fv = (double)fn[j];
        const int x = (int)(j / ((int64_t)N * N)), y = (int)((j / N) % N), z = (int)(j % N);
        a[0] += fv;
        a[1] += fv * (-L + (x + 0.5) * dc);
        a[2] += fv * (-L + (y + 0.5) * dc);
        a[3] += fv * (-L + (z + 0.5) * dc);
    }
    block_sum<4>(a, s);
    const double n = s[0] * dv, ux = s[1] * dv / n, uy = s[2] * dv / n, uz = s[3] * dv / n;
    // sum f d^2, f dx dx, f dy dy, f dz dz, f dx dy, f dx dz, f dy dz, f dx d^2, f dy d^2, f dz d^2, f ln f
    double b[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t j = threadIdx.x; j < n3; j += blockDim.x) {
        const double fv = (double)fn[j];
        const int x = (int)(j / ((int64_t)N * N)), y = (int)((j / N) % N), z = (int)(j % N);
        const double dx = -L + (x + 0.5) * dc - ux, dy = -L + (y + 0.5) * dc - uy, dz = -L + (z + 0.5) * dc - uz;
        const double d2 = dx * dx + dy * dy + dz * dz;
        b[0] += fv * d2;
        b[1] += fv * dx * dx;
        b[2] += fv * dy * dy;
        b[3] += fv * dz * dz;
        b[4] += fv * dx * dy;
        b[5] += fv * dx * dz;
        b[6] += fv * dy * dz;
        b[7] += fv * dx * d2;
        b[8] += fv * dy * d2;
        b[9] += fv * dz * d2;
        if (fv > 0.0) b[10] += fv * log(fv);
    }
    block_sum<11>(b, s);
    if (threadIdx.x == 0) {
        double* o = out + node * 15;
        o[0] = n;
        o[1] = ux;
        o[2] = uy;
        o[3] = uz;
        o[4] = 2.0 / (3.0 * n) * s[0] * dv;
        for (int k = 0; k < 6; ++k) o[5 + k] = 2.0 * s[1 + k] * dv;
        for (int k = 0; k < 3; ++k) o[11 + k] = s[7 + k] * dv;
        o[14] = s[10] * dv;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_rk_combine(int64_t n, double a, const T* u, double b, const T* v, double c, const T* q, T* out,
                              int* flags, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    k_rk_combine<T><<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(n, a, u, b, v, c, q, out, flags);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments(const T* f, int N, double L, int64_t B, double* out, cudaStream_t s) {
    for (int64_t b0 = 0; b0 < B; b0 += 1 << 30) {
        const int64_t nb = B - b0 < (1 << 30) ? B - b0 : (1 << 30);
        k_moments<T><<<(unsigned)nb, 256, 0, s>>>(f + b0 * (int64_t)N * N * N, N, L, out + b0 * 15);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_rk_combine<float>(int64_t, double, const float*, double, const float*, double,
                                              const float*, float*, int*, cudaStream_t);
template cudaError_t launch_rk_combine<double>(int64_t, double, const double*, double, const double*, double,
                                               const double*, double*, int*, cudaStream_t);
template cudaError_t launch_moments<float>(const float*, int, double, int64_t, double*, cudaStream_t);
template cudaError_t launch_moments<double>(const double*, int, double, int64_t, double*, cudaStream_t);

}  // namespace dgfs
