// Fourier-side kernels of the collision operator (arXiv:1809.10186, Appendix).
//
// After the translate-product step has produced P_r for every radial point, the gain is
//   gain^_k = sum_r w_r F(k, c_r) DFT(P_r)_k,   F(k, c_r) = rho_r sinc(pi c_r |k| / 2L)
// (eqs. realGG, apndx_fs_Glm_Qk), and the loss is f times the convolution of g with the
// kernel mode G(m,m). With the radial kernel compressed as sinc(pi c_r |k| / 2L) ~=
// sum_s Uk[s](k) Vr[s][r], the gain needs only `rank` forward transforms:
//   gain^_k = sum_s Uk[s](k) DFT( sum_r Vr[s][r] w_r rho_r P_r )_k.
// Transforms are separable DFTs of the standard grid ordering, one register-resident FFT line per
// thread and axis (radix 2, plus one radix-3 stage for N = 12, 24); every multiplier is diagonal,
// so the half-cell phase of the cell-centred grid cancels between the forward and inverse
// transforms and the signed lattice index k = q (q < N/2) or q - N is used.
#include <cmath>
#include <cstdint>

#include "fourier_dev.cuh"
#include "launchers.h"

namespace dgfs {

namespace {

using namespace fdev;

// ---- radix-2 / radix-3 FFT passes -------------------------------------------------------

// Strided axes: line l of the field group starts at base(l) and has stride S; consecutive
// threads take consecutive lines whose elements are adjacent in memory (coalesced).
template <typename T, int N>
__global__ void __launch_bounds__(128)
k_fft_strided(Cplx<T>* __restrict__ X, const Cplx<T>* __restrict__ W, int64_t lines, int64_t inner,
              int64_t stride, int forward, T scale) {
    __shared__ Cplx<T> tw[N];
    if (threadIdx.x < N) tw[threadIdx.x] = W[N + threadIdx.x];      // row q = 1 of the DFT table
    __syncthreads();
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= lines) return;
    // line l = (outer o, inner i): base = o * N * stride + i   (inner < stride)
    const int64_t o = l / inner, i = l % inner;
    Cplx<T>* base = X + o * (int64_t)N * stride + i;
    Cplx<T> a[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a[line_slot<N>(k)] = base[(int64_t)k * stride];
    line_fft<T, N>(a, tw, forward != 0);
#pragma unroll
    for (int k = 0; k < N; ++k) base[(int64_t)k * stride] = Cplx<T>{a[k].x * scale, a[k].y * scale};
}

// Contiguous axis: 128 lines staged through shared memory so global accesses stay coalesced.
template <typename T, int N>
__global__ void __launch_bounds__(128)
k_fft_contig(Cplx<T>* __restrict__ X, const Cplx<T>* __restrict__ W, int64_t lines, int forward, T scale) {
    __shared__ Cplx<T> tw[N];
    __shared__ Cplx<T> tile[128 * (N + 1)];
    if (threadIdx.x < N) tw[threadIdx.x] = W[N + threadIdx.x];
    const int64_t l0 = (int64_t)blockIdx.x * 128;
    const int nl = (int)((lines - l0) < 128 ? (lines - l0) : 128);
    Cplx<T>* base = X + l0 * N;
    for (int e = threadIdx.x; e < nl * N; e += 128) tile[(e / N) * (N + 1) + e % N] = base[e];
    __syncthreads();
    if (threadIdx.x < nl) {
        Cplx<T> a[N];
#pragma unroll
        for (int k = 0; k < N; ++k) a[line_slot<N>(k)] = tile[threadIdx.x * (N + 1) + k];
        line_fft<T, N>(a, tw, forward != 0);
#pragma unroll
        for (int k = 0; k < N; ++k) tile[threadIdx.x * (N + 1) + k] = Cplx<T>{a[k].x * scale, a[k].y * scale};
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nl * N; e += 128) base[e] = tile[(e / N) * (N + 1) + e % N];
}

template <typename T, int N>
cudaError_t fft3(Cplx<T>* X, const Cplx<T>* W, int64_t count, bool forward, T scale, cudaStream_t s) {
    const int64_t n2 = (int64_t)N * N;
    const int64_t lines = count * n2;
    const unsigned blocks = (unsigned)((lines + 127) / 128);
    k_fft_strided<T, N><<<blocks, 128, 0, s>>>(X, W, lines, n2, n2, forward, scale);   // axis x
    k_fft_strided<T, N><<<blocks, 128, 0, s>>>(X, W, lines, N, N, forward, scale);     // axis y
    k_fft_contig<T, N><<<blocks, 128, 0, s>>>(X, W, lines, forward, scale);            // axis z
    return cudaGetLastError();
}

// ---- projections and multipliers ----------------------------------------------------------

// two consecutive values from an even index (8- or 16-byte aligned), and two complex values with
// zero imaginary parts stored as one 16-byte (float) or two 16-byte (double) stores
__device__ __forceinline__ void load_pair(const float* p, float& a, float& b) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void load_pair(const double* p, double& a, double& b) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    a = v.x;
    b = v.y;
}
// x[0] = {a0, b0}, x[1] = {a1, b1}: one 16-byte (float) or two 16-byte (double) stores
__device__ __forceinline__ void store_cplx_pair(Cplx<float>* x, float a0, float b0, float a1, float b1) {
    *reinterpret_cast<float4*>(x) = make_float4(a0, b0, a1, b1);
}
__device__ __forceinline__ void store_cplx_pair(Cplx<double>* x, double a0, double b0, double a1, double b1) {
    reinterpret_cast<double2*>(x)[0] = make_double2(a0, b0);
    reinterpret_cast<double2*>(x)[1] = make_double2(a1, b1);
}

// field s = sum_r C[s][r] P[node][r][j],  C[s][r] = Vr[s][r] w_r rho_r(node), stored packed: fields
// 2m and 2m + 1 are the real and imaginary parts of slot m. Memory-bound: P is read once. Each thread owns 2 consecutive j and accumulates SG outputs s in
// registers (one pass when rank <= SG), with the coefficients broadcast from shared memory
// (stored [r][s], rows padded to a multiple of SG).
template <typename T, int SG>
__global__ void __launch_bounds__(256) k_project(const T* __restrict__ P, const T* __restrict__ Vr,
                                                 const double* __restrict__ cr, const double* __restrict__ wr,
                                                 NodeParams np, int Nrho, int rank, int64_t n3,
                                                 Cplx<T>* __restrict__ X, int xslots) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* CT = reinterpret_cast<T*>(sm_raw);                 // [Nrho][rpad]
    T* wrho = CT + Nrho * ((rank + SG - 1) / SG * SG);    // [Nrho]: w_r rho_r of this node
    const int rpad = (rank + SG - 1) / SG * SG;
    const int64_t node = blockIdx.y;
    const double gam = np.gamma ? np.gamma[node] : np.gamma0;
    const double bb = np.b ? np.b[node] : np.b0;
    // one FP64 power per radial point (FP64 is slow on this part), then the coefficient table
    for (int r = threadIdx.x; r < Nrho; r += blockDim.x) wrho[r] = (T)wr[r] * radial_rho<T>(bb, gam, cr[r], np.dlog);
    __syncthreads();
    for (int e = threadIdx.x; e < Nrho * rpad; e += blockDim.x) {
        const int r = e / rpad, sidx = e % rpad;
        CT[e] = sidx < rank ? Vr[sidx * Nrho + r] * wrho[r] : T(0);
    }
    __syncthreads();
    const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (j0 >= n3) return;
    const T* Pn = P + node * Nrho * n3 + j0;
    Cplx<T>* Xn = X + node * (int64_t)xslots * n3 + j0;
    for (int s0 = 0; s0 < rank; s0 += SG) {
        T acc[SG][2];
#pragma unroll
        for (int i = 0; i < SG; ++i) acc[i][0] = acc[i][1] = T(0);
#pragma unroll 4
        for (int r = 0; r < Nrho; ++r) {
            T p0, p1;
            load_pair(Pn + (int64_t)r * n3, p0, p1);
            const T* c = CT + r * rpad + s0;
#pragma unroll
            for (int i = 0; i < SG; ++i) {
                acc[i][0] = fma(c[i], p0, acc[i][0]);
                acc[i][1] = fma(c[i], p1, acc[i][1]);
            }
        }
#pragma unroll
        for (int i = 0; i < SG; i += 2)   // s0 is even: fields s0 + i, s0 + i + 1 share slot (s0 + i) / 2
            if (s0 + i < rank) {
                const bool two = s0 + i + 1 < rank;
                store_cplx_pair(Xn + (int64_t)((s0 + i) / 2) * n3, acc[i][0], two ? acc[i + 1][0] : T(0), acc[i][1],
                                two ? acc[i + 1][1] : T(0));
            }
    }
}

template <typename T>
__global__ void k_load_field(int64_t n3, const T* __restrict__ a, const T* __restrict__ b,
                             const int64_t* __restrict__ offs, Cplx<T>* __restrict__ X, int xfields,
                             int slot, int part) {
    const int64_t node = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n3) return;
    const int64_t base = offs ? offs[node] : node * n3;
    T v = a[base + j];
    if (b) v *= b[base + j];
    Cplx<T>& x = X[(node * xfields + slot) * n3 + j];
    if (part == 0) x = Cplx<T>{v, T(0)};
    else x.y = v;
}

template <typename T>
__global__ void k_combine(const Cplx<T>* __restrict__ X, int xslots, const T* __restrict__ Uk,
                          const T* __restrict__ Lr, const T* __restrict__ GL0, const T* __restrict__ GLd,
                          const double* __restrict__ cr, NodeParams np, int N, int Nrho, int rank, int64_t n3,
                          T scale, int lf0, int lf1, Cplx<T>* __restrict__ Y, int yfields) {
    __shared__ double rho[64];
    const int64_t node = blockIdx.y;
    const bool per_node = np.gamma || np.b;
    const double gam = np.gamma ? np.gamma[node] : np.gamma0;
    const double bb = np.b ? np.b[node] : np.b0;
    if (per_node)
        for (int r = threadIdx.x; r < Nrho; r += blockDim.x) rho[r] = radial_rho<double>(bb, gam, cr[r], np.dlog);
    __syncthreads();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n3) return;
    // index of -k (each axis index q -> (N - q) mod N in the standard DFT ordering)
    const int kz = (int)(k % N), ky = (int)((k / N) % N), kx = (int)(k / ((int64_t)N * N));
    const int64_t km = ((int64_t)((N - kx) % N) * N + (N - ky) % N) * N + (N - kz) % N;
    const Cplx<T>* Xn = X + node * (int64_t)xslots * n3;
    const int nfields = (lf1 >= 0 ? lf1 : lf0) + 1;
    T gr = 0, gi = 0;
    Cplx<T> l0{T(0), T(0)}, l1{T(0), T(0)};
    for (int m = 0; 2 * m < nfields; ++m) {
        const Cplx<T> z = Xn[m * n3 + k], w = Xn[m * n3 + km];
        // spectra of the real fields 2m and 2m + 1 packed in slot m
        const Cplx<T> fa{(z.x + w.x) * T(0.5), (z.y - w.y) * T(0.5)};
        const Cplx<T> fb{(z.y + w.y) * T(0.5), (w.x - z.x) * T(0.5)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int fi = 2 * m + h;
            const Cplx<T> v = h ? fb : fa;
            if (fi < rank) {
                const T u = Uk[fi * n3 + k];
                gr = fma(u, v.x, gr);
                gi = fma(u, v.y, gi);
            } else if (fi == lf0) {
                l0 = v;
            } else if (fi == lf1) {
                l1 = v;
            }
        }
    }
    const T GL = loss_multiplier<T>(GL0, GLd, Lr, rho, per_node, np.dlog, Nrho, n3, k);
    // the gain and each loss convolution get their own inverse transform: packing two real
    // results of very different size into one complex transform would leak the rounding of the
    // larger one (K_L g ~ n everywhere) into the smaller one (the gain, tiny in the tails)
    Cplx<T>* Yn = Y + node * (int64_t)yfields * n3;
    Yn[k] = Cplx<T>{scale * gr, scale * gi};
    Yn[n3 + k] = Cplx<T>{GL * l0.x, GL * l0.y};
    if (lf1 >= 0) Yn[2 * n3 + k] = Cplx<T>{GL * l1.x, GL * l1.y};
}

template <typename T>
__global__ void k_loss_pair(const Cplx<T>* __restrict__ X, int xfields, const T* __restrict__ Lr,
                            const T* __restrict__ GL0, const T* __restrict__ GLd,
                            const double* __restrict__ cr, NodeParams np, int Nrho, int64_t n3,
                            int s0, int s1, Cplx<T>* __restrict__ Y, int yfields) {
    __shared__ double rho[64];
    const int64_t node = blockIdx.y;
    const bool per_node = np.gamma || np.b;
    const double gam = np.gamma ? np.gamma[node] : np.gamma0;
    const double bb = np.b ? np.b[node] : np.b0;
    if (per_node)
        for (int r = threadIdx.x; r < Nrho; r += blockDim.x) rho[r] = radial_rho<double>(bb, gam, cr[r], np.dlog);
    __syncthreads();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n3) return;
    const T GL = loss_multiplier<T>(GL0, GLd, Lr, rho, per_node, np.dlog, Nrho, n3, k);
    const Cplx<T>* Xn = X + node * (int64_t)xfields * n3;
    const Cplx<T> a = Xn[s0 * n3 + k], b = Xn[s1 * n3 + k];
    Cplx<T>* Yn = Y + node * (int64_t)yfields * n3;
    Yn[k] = Cplx<T>{GL * a.x, GL * a.y};
    Yn[n3 + k] = Cplx<T>{GL * b.x, GL * b.y};
}

template <typename T>
__global__ void k_multiply_uk(Cplx<T>* __restrict__ X, int xfields, const T* __restrict__ Uk,
                              int rank, int64_t n3, int src) {
    const int64_t node = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n3) return;
    Cplx<T>* Xn = X + node * (int64_t)xfields * n3;
    const Cplx<T> v = Xn[src * n3 + k];
    for (int s = 0; s < rank; ++s) {
        const T u = Uk[s * n3 + k];
        Xn[s * n3 + k] = Cplx<T>{u * v.x, u * v.y};
    }
}

// U[node][r][j] = w_r rho_r sum_s Vr[s][r] Re X[node][s][j]
template <typename T>
__global__ void k_expand_radial(const Cplx<T>* __restrict__ X, int xfields, const T* __restrict__ Vr,
                                const double* __restrict__ cr, const double* __restrict__ wr,
                                NodeParams np, int Nrho, int rank, int64_t n3, T* __restrict__ U) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* C = reinterpret_cast<T*>(sm_raw);        // [rank][Nrho]
    T* Xt = C + rank * Nrho;                     // [rank][blockDim]
    T* wrho = Xt + rank * blockDim.x;            // [Nrho]: w_r rho_r of this node
    const int64_t node = blockIdx.y;
    const double gam = np.gamma ? np.gamma[node] : np.gamma0;
    const double bb = np.b ? np.b[node] : np.b0;
    for (int r = threadIdx.x; r < Nrho; r += blockDim.x) wrho[r] = (T)wr[r] * radial_rho<T>(bb, gam, cr[r], np.dlog);
    __syncthreads();
    for (int e = threadIdx.x; e < rank * Nrho; e += blockDim.x) C[e] = Vr[e] * wrho[e % Nrho];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const Cplx<T>* Xn = X + node * (int64_t)xfields * n3;
    for (int s = 0; s < rank; ++s) Xt[s * blockDim.x + threadIdx.x] = j < n3 ? Xn[s * n3 + j].x : T(0);
    __syncthreads();
    if (j >= n3) return;
    T* Un = U + node * (int64_t)Nrho * n3;
    for (int r = 0; r < Nrho; ++r) {
        T acc = 0;
        for (int s = 0; s < rank; ++s) acc = fma(C[s * Nrho + r], Xt[s * blockDim.x + threadIdx.x], acc);
        Un[r * n3 + j] = acc;
    }
}

template <typename T>
__global__ void k_finalize(int Nrho, int64_t n3, const Cplx<T>* __restrict__ Y, int yfields,
                           const T* __restrict__ a, const T* __restrict__ c, const T* __restrict__ G,
                           const int64_t* __restrict__ offs, int mode, T* __restrict__ out,
                           int* __restrict__ flags) {
    const int64_t node = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n3) return;
    const int64_t base = offs ? offs[node] : node * n3;
    const Cplx<T>* Yn = Y + node * (int64_t)yfields * n3;
    const Cplx<T> y0 = Yn[j], y1 = Yn[n3 + j];
    T v;
    if (mode == 0) {
        v = y0.x - a[base + j] * y1.x;
        if (c) v -= c[base + j] * Yn[2 * n3 + j].x;
    } else {
        v = T(0);
        const T* Gn = G + node * (int64_t)Nrho * n3;
        for (int r = 0; r < Nrho; ++r) v += Gn[r * n3 + j];
        v -= a[base + j] * y0.x + y1.x;
    }
    if (!isfinite(v)) atomicOr(flags, 2);
    out[base + j] = v;
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

template <typename T>
cudaError_t launch_dft3(const DevTables<T>& t, Cplx<T>* X, int64_t count, bool forward, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int N = t.N;
    const int64_t n2 = (int64_t)N * N;
    const T scale = forward ? T(1) / T(N) : T(1);
    const Cplx<T>* W = reinterpret_cast<const Cplx<T>*>(t.dftw);
    if (N == 8) return fft3<T, 8>(X, W, count, forward, scale, s);
    if (N == 12) return fft3<T, 12>(X, W, count, forward, scale, s);
    if (N == 16) return fft3<T, 16>(X, W, count, forward, scale, s);
    if (N == 24) return fft3<T, 24>(X, W, count, forward, scale, s);
    if (N == 32) return fft3<T, 32>(X, W, count, forward, scale, s);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_project(const DevTables<T>& t, const T* P, NodeParams np, int64_t nodes,
                           Cplx<T>* X, int xfields, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    const int64_t n3 = (int64_t)t.N * t.N * t.N;      // even for every supported N
    const int bs = 256;
    const dim3 grid(blocks_for(n3 / 2, bs), (unsigned)nodes);
    auto go = [&](auto kern, int sg) {
        const size_t sm = sizeof(T) * (size_t)t.Nrho * (size_t)((t.rank + sg - 1) / sg * sg + 1);
        if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<grid, bs, sm, s>>>(P, t.Vr, t.cr, t.wr, np, t.Nrho, t.rank, n3, X, xfields);
    };
    if (t.rank <= 8) go(k_project<T, 8>, 8);
    else if (t.rank <= 16) go(k_project<T, 16>, 16);
    else if (t.rank <= 24) go(k_project<T, 24>, 24);
    else go(k_project<T, 32>, 32);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_load_field(int N, const T* a, const T* b, const int64_t* offs, int64_t nodes,
                              Cplx<T>* X, int xfields, int slot, int part, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    const int64_t n3 = (int64_t)N * N * N;
    k_load_field<T><<<dim3(blocks_for(n3, 256), (unsigned)nodes), 256, 0, s>>>(n3, a, b, offs, X, xfields, slot, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_combine(const DevTables<T>& t, const Cplx<T>* X, int xslots, NodeParams np,
                           int64_t nodes, T scale, int lf0, int lf1, Cplx<T>* Y, int yfields,
                           cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    const int64_t n3 = (int64_t)t.N * t.N * t.N;
    k_combine<T><<<dim3(blocks_for(n3, 256), (unsigned)nodes), 256, 0, s>>>(X, xslots, t.Uk, t.Lr, t.GL0, t.GLd, t.cr, np, t.N, t.Nrho, t.rank, n3, scale, lf0, lf1, Y, yfields);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_loss_pair(const DevTables<T>& t, const Cplx<T>* X, int xfields, NodeParams np,
                             int64_t nodes, int s0, int s1, Cplx<T>* Y, int yfields, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    const int64_t n3 = (int64_t)t.N * t.N * t.N;
    k_loss_pair<T><<<dim3(blocks_for(n3, 256), (unsigned)nodes), 256, 0, s>>>(X, xfields, t.Lr, t.GL0, t.GLd, t.cr, np, t.Nrho, n3, s0, s1, Y, yfields);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_multiply_uk(const DevTables<T>& t, Cplx<T>* X, int xfields, int src, int64_t nodes,
                               cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    const int64_t n3 = (int64_t)t.N * t.N * t.N;
    k_multiply_uk<T><<<dim3(blocks_for(n3, 256), (unsigned)nodes), 256, 0, s>>>(X, xfields, t.Uk, t.rank, n3, src);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_expand_radial(const DevTables<T>& t, const Cplx<T>* X, int xfields, NodeParams np,
                                 int64_t nodes, T* U, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    const int64_t n3 = (int64_t)t.N * t.N * t.N;
    const int bs = 128;
    const size_t sm = sizeof(T) * (size_t)(t.rank * t.Nrho + t.rank * bs + t.Nrho);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_expand_radial<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_expand_radial<T><<<dim3(blocks_for(n3, bs), (unsigned)nodes), bs, sm, s>>>(X, xfields, t.Vr, t.cr, t.wr, np, t.Nrho, t.rank, n3, U);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize(int N, int Nrho, const Cplx<T>* Y, int yfields, const T* a, const T* c,
                            const T* G, const int64_t* offs, int64_t nodes, int mode, T* out,
                            int* flags, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    const int64_t n3 = (int64_t)N * N * N;
    k_finalize<T><<<dim3(blocks_for(n3, 256), (unsigned)nodes), 256, 0, s>>>(Nrho, n3, Y, yfields, a, c, G, offs, mode, out, flags);
    return cudaGetLastError();
}

#define DGFS_INST(T)                                                                                   \
    template cudaError_t launch_dft3<T>(const DevTables<T>&, Cplx<T>*, int64_t, bool, cudaStream_t);  \
    template cudaError_t launch_project<T>(const DevTables<T>&, const T*, NodeParams, int64_t,        \
                                           Cplx<T>*, int, cudaStream_t);                              \
    template cudaError_t launch_load_field<T>(int, const T*, const T*, const int64_t*, int64_t,       \
                                              Cplx<T>*, int, int, int, cudaStream_t);                 \
    template cudaError_t launch_combine<T>(const DevTables<T>&, const Cplx<T>*, int, NodeParams,      \
                                           int64_t, T, int, int, Cplx<T>*, int, cudaStream_t);        \
    template cudaError_t launch_loss_pair<T>(const DevTables<T>&, const Cplx<T>*, int, NodeParams,    \
                                             int64_t, int, int, Cplx<T>*, int, cudaStream_t);         \
    template cudaError_t launch_multiply_uk<T>(const DevTables<T>&, Cplx<T>*, int, int, int64_t,      \
                                               cudaStream_t);                                         \
    template cudaError_t launch_expand_radial<T>(const DevTables<T>&, const Cplx<T>*, int, NodeParams,\
                                                 int64_t, T*, cudaStream_t);                          \
    template cudaError_t launch_finalize<T>(int, int, const Cplx<T>*, int, const T*, const T*,        \
                                            const T*, const int64_t*, int64_t, int, T*, int*,         \
                                            cudaStream_t);
DGFS_INST(float)
DGFS_INST(double)
#undef DGFS_INST

}  // namespace dgfs
