// Kernels of the DG element collision term in its SVD variant (arXiv:1809.10186, Sec. 3.4,
// eqs. HH, eq_coln_derivation_SVD_3 and _4). For every element e, the combined fields of every
// retained singular triple (m, r) are f_r = sum_l U^m[l][r] F_l and g_r = sum_l V^m[r][l] F_l
// (k_dg_combine); after the bilinear collision operator has turned them into Q(f_r, g_r), the
// element's term of test function m is the sum of its R_m results (k_dg_accumulate). Both are
// memory-bound streams over N^3 points. When every slice H[m] is symmetric (always for the nodal
// basis), the factors are taken from its eigen-decomposition, H[m] = sum_r s_r a_r a_r^T with
// a_r = sqrt|lambda_r| u_r and s_r = sign lambda_r: an SVD of H[m] with V[r] = s_r a_r, so that
// Q(f_r, g_r) = s_r Q(f_r, f_r). Then only f_r is formed (B == nullptr) and the accumulation
// carries the signs.
#include <cstdint>

#include "launchers.h"

namespace dgfs {

namespace {

constexpr int kMaxK = 16;

// F [E][K][n3] -> f, g [E][R][n3]; A, B [R][K] (row r: the coefficients of f_r and g_r)
template <typename T>
__global__ void __launch_bounds__(256) k_dg_combine(const T* __restrict__ F, const T* __restrict__ A,
                                                    const T* __restrict__ B, int K, int R, int64_t n3,
                                                    T* __restrict__ f, T* __restrict__ g) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* sa = reinterpret_cast<T*>(sm_raw);   // [R][K]
    T* sb = sa + R * K;                      // [R][K] (unused without B)
    for (int i = threadIdx.x; i < R * K; i += blockDim.x) {
        sa[i] = A[i];
        if (B) sb[i] = B[i];
    }
    __syncthreads();
    const int64_t e = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n3) return;
    T v[kMaxK];
#pragma unroll
    for (int l = 0; l < kMaxK; ++l) v[l] = l < K ? F[(e * K + l) * n3 + j] : T(0);
    for (int r = 0; r < R; ++r) {
        T fr = 0, gr = 0;
#pragma unroll
        for (int l = 0; l < kMaxK; ++l)
            if (l < K) {
                fr = fma(sa[r * K + l], v[l], fr);
                if (B) gr = fma(sb[r * K + l], v[l], gr);
            }
        f[(e * R + r) * n3 + j] = fr;
        if (B) g[(e * R + r) * n3 + j] = gr;
    }
}

// Q [E][R][n3] -> C [E][K][n3]: C[e][m] = sum of rows rs[m] .. rs[m + 1] - 1, each times sgn[r]
// (sgn == nullptr: all +1)
template <typename T>
__global__ void __launch_bounds__(256) k_dg_accumulate(const T* __restrict__ Q, const int* __restrict__ rs,
                                                       const T* __restrict__ sgn, int K, int R, int64_t n3,
                                                       T* __restrict__ C) {
    const int64_t e = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n3) return;
    for (int m = 0; m < K; ++m) {
        T acc = 0;
        for (int r = __ldg(rs + m); r < __ldg(rs + m + 1); ++r) {
            const T q = Q[(e * R + r) * n3 + j];
            acc += sgn ? sgn[r] * q : q;
        }
        C[(e * K + m) * n3 + j] = acc;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_dg_combine(const T* F, const T* A, const T* B, int K, int R, int64_t n3, int64_t E, T* f, T* g,
                              cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    if (K < 1 || K > kMaxK || R < 1 || E > 65535) return cudaErrorInvalidValue;
    const size_t sm = 2 * sizeof(T) * (size_t)R * K;   // B == nullptr: only f is formed
    k_dg_combine<T><<<dim3((unsigned)((n3 + 255) / 256), (unsigned)E), 256, sm, s>>>(F, A, B, K, R, n3, f, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dg_accumulate(const T* Q, const int* rs, const T* sgn, int K, int R, int64_t n3, int64_t E, T* C,
                                 cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    if (E > 65535) return cudaErrorInvalidValue;
    k_dg_accumulate<T><<<dim3((unsigned)((n3 + 255) / 256), (unsigned)E), 256, 0, s>>>(Q, rs, sgn, K, R, n3, C);
    return cudaGetLastError();
}

template cudaError_t launch_dg_combine<float>(const float*, const float*, const float*, int, int, int64_t, int64_t,
                                              float*, float*, cudaStream_t);
template cudaError_t launch_dg_combine<double>(const double*, const double*, const double*, int, int, int64_t,
                                               int64_t, double*, double*, cudaStream_t);
template cudaError_t launch_dg_accumulate<float>(const float*, const int*, const float*, int, int, int64_t, int64_t,
                                                 float*, cudaStream_t);
template cudaError_t launch_dg_accumulate<double>(const double*, const int*, const double*, int, int, int64_t,
                                                  int64_t, double*, cudaStream_t);

}  // namespace dgfs
