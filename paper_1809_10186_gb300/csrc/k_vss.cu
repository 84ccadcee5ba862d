// Gain of the collision operator for the VSS kernel (arXiv:1809.10186, eq. B_gen with alpha != 1;
// Appendix eqs. realGG, lowrank1, apndx_fs_Glm_Qk).
//
// With an angular factor the kernel mode F(k, c_r, sigma) keeps the sphere point, so the gain is
//   gain^_k = sum_r sum_p A_rp(k) DFT[(T_s f)(T_-s g) + (T_-s f)(T_s g)]_k,   s = c_r sigma_p / 2,
// A_rp = w_r w_p F(k, c_r, sigma_p): one forward transform per radial AND sphere point. The
// translates are taken in Fourier space: T_s f = IDFT(mu_s f^) with the separable multiplier
// mu_s(k) = mu_x(k_x) mu_y(k_y) mu_z(k_z), mu_-s = conj(mu_s). Because every translate of a real
// field is real (symmetric Nyquist convention), one complex inverse transform carries two of them:
//   IDFT(mu_s f^ + i mu_-s g^) = T_s f + i T_-s g,   IDFT(mu_-s f^ + i mu_s g^) = T_-s f + i T_s g,
// and the real products of two sphere points share one forward transform (real and imaginary
// parts), separated in Fourier space by Hermitian symmetry. Per radial point r, over a chunk of
// nodes and all sphere points:
//   k_vss_spectra     Z[n][set][p] = the two multiplied spectra above (set 1 only for f != g)
//   inverse DFT       (k_fourier.cu)
//   k_vss_product     W[n][j] = P_2j + i P_2j+1,  P_p = Re Z0 Im Z0 + Re Z1 Im Z1  (2 Re Z0 Im Z0 for f = g)
//   forward DFT
//   k_vss_accumulate  Y[n][0](k) += scale sum_p A_rp(k) P^_p(k)
// All four are elementwise streams over N^3 points; the transforms dominate.
#include <cstdint>

#include "launchers.h"

namespace dgfs {

namespace {

template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
    return Cplx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// grid (ceil(n3 / 256), npairs, nodes); mu_r: [npairs][3][N] complex multipliers of +s_rp
template <typename T>
__global__ void __launch_bounds__(256) k_vss_spectra(const Cplx<T>* __restrict__ Fh, const Cplx<T>* __restrict__ Gh,
                                                     const Cplx<T>* __restrict__ mu_r, int N, int npairs, int sets,
                                                     int64_t n3, Cplx<T>* __restrict__ Z) {
    __shared__ Cplx<T> m[3 * 64];
    const int p = blockIdx.y;
    const int64_t n = blockIdx.z;
    for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) m[i] = mu_r[(int64_t)p * 3 * N + i];
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n3) return;
    const int kx = (int)(j / ((int64_t)N * N)), ky = (int)((j / N) % N), kz = (int)(j % N);
    const Cplx<T> mu = cmul(cmul(m[kx], m[N + ky]), m[2 * N + kz]);   // mu_s(k); mu_-s = conj
    const Cplx<T> f = Fh[n * n3 + j];
    const Cplx<T> g = Gh ? Gh[n * n3 + j] : f;
    const T a = mu.x, b = mu.y;
    // set 0: mu f + i conj(mu) g
    Z[((n * sets) * npairs + p) * n3 + j] =
        Cplx<T>{a * f.x - b * f.y - a * g.y + b * g.x, a * f.y + b * f.x + a * g.x + b * g.y};
    if (sets == 2)   // set 1: conj(mu) f + i mu g
        Z[((n * sets + 1) * npairs + p) * n3 + j] =
            Cplx<T>{a * f.x + b * f.y - a * g.y - b * g.x, a * f.y - b * f.x + a * g.x - b * g.y};
}

// grid (ceil(n3 / 256), (npairs + 1) / 2, nodes)
template <typename T>
__global__ void __launch_bounds__(256) k_vss_product(const Cplx<T>* __restrict__ Z, int npairs, int sets, int64_t n3,
                                                     Cplx<T>* __restrict__ W) {
    const int jw = blockIdx.y, nw = gridDim.y;
    const int64_t n = blockIdx.z;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n3) return;
    T P[2] = {T(0), T(0)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = 2 * jw + h;
        if (p >= npairs) break;
        const Cplx<T> z0 = Z[((n * sets) * npairs + p) * n3 + j];
        if (sets == 2) {
            const Cplx<T> z1 = Z[((n * sets + 1) * npairs + p) * n3 + j];
            P[h] = z0.x * z0.y + z1.x * z1.y;
        } else {
            P[h] = T(2) * z0.x * z0.y;
        }
    }
    W[(n * nw + jw) * n3 + j] = Cplx<T>{P[0], P[1]};
}

// grid (ceil(n3 / 256), nodes); A_r: [npairs][n3] real, W: [nodes][(npairs + 1) / 2][n3]
template <typename T>
__global__ void __launch_bounds__(256) k_vss_accumulate(const Cplx<T>* __restrict__ W, const T* __restrict__ A_r,
                                                        int N, int npairs, int64_t n3, T scale,
                                                        Cplx<T>* __restrict__ Y, int yfields) {
    const int64_t n = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n3) return;
    const int nw = (npairs + 1) / 2;
    const int kx = (int)(j / ((int64_t)N * N)), ky = (int)((j / N) % N), kz = (int)(j % N);
    const int64_t jm = ((int64_t)((N - kx) % N) * N + (N - ky) % N) * N + (N - kz) % N;   // -k
    T re = 0, im = 0;
    for (int jw = 0; jw < nw; ++jw) {
        const Cplx<T> w = W[(n * nw + jw) * n3 + j], wm = W[(n * nw + jw) * n3 + jm];
        // P^_2j = (W(k) + conj W(-k)) / 2,  P^_2j+1 = (W(k) - conj W(-k)) / 2i
        const T a0 = A_r[(int64_t)(2 * jw) * n3 + j];
        re = fma(a0, T(0.5) * (w.x + wm.x), re);
        im = fma(a0, T(0.5) * (w.y - wm.y), im);
        if (2 * jw + 1 < npairs) {
            const T a1 = A_r[(int64_t)(2 * jw + 1) * n3 + j];
            re = fma(a1, T(0.5) * (w.y + wm.y), re);
            im = fma(a1, T(-0.5) * (w.x - wm.x), im);
        }
    }
    Cplx<T>& y = Y[n * yfields * n3 + j];
    y.x += scale * re;
    y.y += scale * im;
}

// Y[n][0] = 0, Y[n][1] = GL Bh, Y[n][2] = GL Ah (yfields == 3)
template <typename T>
__global__ void __launch_bounds__(256) k_vss_loss_init(const Cplx<T>* __restrict__ Ah, const Cplx<T>* __restrict__ Bh,
                                                       const T* __restrict__ GL, int64_t n3, Cplx<T>* __restrict__ Y,
                                                       int yfields) {
    const int64_t n = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n3) return;
    const T gl = GL[j];
    Cplx<T>* Yn = Y + n * yfields * n3;
    Yn[j] = Cplx<T>{T(0), T(0)};
    const Cplx<T> b = Bh[n * n3 + j];
    Yn[n3 + j] = Cplx<T>{gl * b.x, gl * b.y};
    if (yfields == 3) {
        const Cplx<T> a = Ah[n * n3 + j];
        Yn[2 * n3 + j] = Cplx<T>{gl * a.x, gl * a.y};
    }
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

template <typename T>
cudaError_t launch_vss_spectra(const Cplx<T>* Fh, const Cplx<T>* Gh, const Cplx<T>* mu_r, int N, int npairs,
                               int sets, int64_t nodes, Cplx<T>* Z, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (N > 64 || nodes > 65535 || npairs > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    k_vss_spectra<T><<<dim3(nblk(n3), (unsigned)npairs, (unsigned)nodes), 256, 0, s>>>(Fh, Gh, mu_r, N, npairs, sets,
                                                                                       n3, Z);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vss_product(const Cplx<T>* Z, int N, int npairs, int sets, int64_t nodes, Cplx<T>* W,
                               cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    k_vss_product<T><<<dim3(nblk(n3), (unsigned)((npairs + 1) / 2), (unsigned)nodes), 256, 0, s>>>(Z, npairs, sets,
                                                                                                   n3, W);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vss_accumulate(const Cplx<T>* W, const T* A_r, int N, int npairs, int64_t nodes, T scale,
                                  Cplx<T>* Y, int yfields, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    k_vss_accumulate<T><<<dim3(nblk(n3), (unsigned)nodes), 256, 0, s>>>(W, A_r, N, npairs, n3, scale, Y, yfields);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vss_loss_init(const Cplx<T>* Ah, const Cplx<T>* Bh, const T* GL, int N, int64_t nodes,
                                 Cplx<T>* Y, int yfields, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    k_vss_loss_init<T><<<dim3(nblk(n3), (unsigned)nodes), 256, 0, s>>>(Ah, Bh, GL, n3, Y, yfields);
    return cudaGetLastError();
}

#define DGFS_VSS_INST(T)                                                                                          \
    template cudaError_t launch_vss_spectra<T>(const Cplx<T>*, const Cplx<T>*, const Cplx<T>*, int, int, int,    \
                                               int64_t, Cplx<T>*, cudaStream_t);                                  \
    template cudaError_t launch_vss_product<T>(const Cplx<T>*, int, int, int, int64_t, Cplx<T>*, cudaStream_t);  \
    template cudaError_t launch_vss_accumulate<T>(const Cplx<T>*, const T*, int, int, int64_t, T, Cplx<T>*, int, \
                                                  cudaStream_t);                                                  \
    template cudaError_t launch_vss_loss_init<T>(const Cplx<T>*, const Cplx<T>*, const T*, int, int64_t,         \
                                                 Cplx<T>*, int, cudaStream_t);
DGFS_VSS_INST(float)
DGFS_VSS_INST(double)
#undef DGFS_VSS_INST

}  // namespace dgfs
