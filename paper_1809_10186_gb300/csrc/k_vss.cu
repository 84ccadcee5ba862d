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
// parts), separated in Fourier space by Hermitian symmetry. Per radial point r, over a batch of
// nodes and all sphere points, with every field stored plane-major ([kz][kx][ky], the z axis
// outermost, so that a plane of fixed kz is contiguous):
//   k_vss_planes<INV>   per (node, field, KZ planes): translate spectra formed while the x lines
//                       load, inverse transforms along x and y                         -> Z
//   k_vss_lines         per (node, sphere-point pair, (x, y) line): inverse transform along z,
//                       the products P_p = Re Z0 Im Z0 + Re Z1 Im Z1 (2 Re Z0 Im Z0 for f = g),
//                       packing P_2j + i P_2j+1, forward transform along z             -> W
//   k_vss_planes<FWD>   forward transforms along x and y of the packed spectra, in place
//   k_vss_accumulate    Y[n][0](k) += scale sum_p A_rp(k) P^_p(k) (the mirror -k is taken per
//                       axis, so any axis order works)
// The VHS path uses the same plane kernel and k_vss_lines_sum, which sums the products over the
// sphere in registers. Lines are transformed in registers: radix 2 for N = 8, 16, 32, one radix-3
// stage over three radix-2 transforms for N = 12, 24 (fourier_dev.cuh).
#include <cstdint>

#include "fourier_dev.cuh"
#include "launchers.h"

namespace dgfs {

namespace {

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

// ---- fused plane / line kernels (power-of-two N) ---------------------------------------------

using fdev::line_fft;
using fdev::line_slot;

// the largest divisor of N with KZ N <= 128 threads
constexpr int planes_per_cta(int N) {
    int kz = 1;
    for (int d = 1; d <= N; ++d)
        if (N % d == 0 && d * N <= 128) kz = d;
    return kz;
}

template <typename T, int N>
struct PlaneGeo {
    static constexpr int KZ = planes_per_cta(N);               // planes per CTA (4 at N = 32 and 24, 8 at 16)
    static constexpr int NT = KZ * N;                          // one line per thread per pass
    static constexpr int P = N + 1;                            // padded row (complex elements)
    static constexpr size_t smem = (size_t)KZ * N * P * sizeof(Cplx<T>);
};

// INV: field f = set * npairs + p of node n; planes kz0 .. kz0 + KZ - 1 of the translate spectra
// (set 0: mu f^ + i conj(mu) g^, set 1: the same with conj(mu) for mu), then inverse transforms
// along x and y; output Z[n][f] plane-major. !INV: forward transforms (scale 1/N each) along x and y
// of X[n][f] in place. grid (N / KZ, fields, nodes). The x lines are read straight from global
// memory (consecutive threads take consecutive ky: coalesced), the y lines go through shared memory.
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(PlaneGeo<T, N>::NT)
    k_vss_planes(const Cplx<T>* __restrict__ Fh, const Cplx<T>* __restrict__ Gh, const Cplx<T>* __restrict__ mu_r,
                 const Cplx<T>* __restrict__ dftw, int npairs, Cplx<T>* __restrict__ X) {
    using G = PlaneGeo<T, N>;
    constexpr int KZ = G::KZ, NT = G::NT, P = G::P;
    constexpr int64_t n2 = (int64_t)N * N, n3 = n2 * N;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Cplx<T>* S = reinterpret_cast<Cplx<T>*>(sm_raw);   // [KZ][N][P]
    __shared__ Cplx<T> tw[N];
    __shared__ Cplx<T> m[3 * N];
    const int tid = threadIdx.x, kz0 = blockIdx.x * KZ, f = blockIdx.y, nf = gridDim.y;
    const int64_t n = blockIdx.z;
    const int pl = tid / N, ln = tid % N;
    if (tid < N) tw[tid] = dftw[N + tid];
    Cplx<T>* Xf = X + (n * nf + f) * n3 + (int64_t)kz0 * n2;
    Cplx<T> v[N];
    if constexpr (INV) {
        const int p = f % npairs;
        const T sgn = f < npairs ? T(1) : T(-1);   // set 1 takes conj(mu) where set 0 takes mu
        for (int i = tid; i < 3 * N; i += NT) m[i] = mu_r[(int64_t)p * 3 * N + i];
        __syncthreads();
        const Cplx<T>* Fp = Fh + n * n3 + (int64_t)(kz0 + pl) * n2 + ln;
        const Cplx<T>* Gp = (Gh ? Gh : Fh) + n * n3 + (int64_t)(kz0 + pl) * n2 + ln;
        const Cplx<T> my = m[N + ln], mz = m[2 * N + kz0 + pl];
        const Cplx<T> myz{my.x * mz.x - my.y * mz.y, my.x * mz.y + my.y * mz.x};
#pragma unroll
        for (int kx = 0; kx < N; ++kx) {
            const Cplx<T> mx = m[kx];
            const T a = mx.x * myz.x - mx.y * myz.y, b = sgn * (mx.x * myz.y + mx.y * myz.x);
            const Cplx<T> fv = Fp[kx * N];
            const Cplx<T> gv = Gh ? Gp[kx * N] : fv;   // g = f: one load
            v[line_slot<N>(kx)] = Cplx<T>{a * fv.x - b * fv.y - a * gv.y + b * gv.x, a * fv.y + b * fv.x + a * gv.x + b * gv.y};
        }
    } else {
        __syncthreads();
#pragma unroll
        for (int x = 0; x < N; ++x) v[line_slot<N>(x)] = Xf[(int64_t)pl * n2 + x * N + ln];
    }
    const T sc = INV ? T(1) : T(1) / T(N);
    // x lines (fixed ky = ln)
    line_fft<T, N>(v, tw, !INV);
#pragma unroll
    for (int k = 0; k < N; ++k) S[(pl * N + k) * P + ln] = Cplx<T>{v[k].x * sc, v[k].y * sc};
    __syncthreads();
    // y lines (fixed x = ln)
#pragma unroll
    for (int k = 0; k < N; ++k) v[line_slot<N>(k)] = S[(pl * N + ln) * P + k];
    line_fft<T, N>(v, tw, !INV);
#pragma unroll
    for (int k = 0; k < N; ++k) S[(pl * N + ln) * P + k] = Cplx<T>{v[k].x * sc, v[k].y * sc};
    __syncthreads();
    for (int e = tid; e < KZ * N * N; e += NT) {
        const int q = e / (N * N), x = (e / N) % N, y = e % N;
        Xf[e] = S[(q * N + x) * P + y];
    }
}

// z-line (x, y) of node n and sphere-point pair j: inverse transform of the translate lines of
// points 2j and 2j + 1 (both sets), products, packing P_2j + i P_2j+1, forward transform (1/N).
// grid (ceil(N^2 / 128), (npairs + 1) / 2, nodes); Z, W plane-major.
template <typename T, int N>
__device__ __forceinline__ void vss_line_products(const Cplx<T>* __restrict__ Z, int64_t stride, int sets,
                                                  int64_t set_stride, const Cplx<T>* tw, T (&P)[N]) {
    Cplx<T> v[N];
    for (int s = 0; s < sets; ++s) {
#pragma unroll
        for (int k = 0; k < N; ++k) v[line_slot<N>(k)] = Z[s * set_stride + k * stride];
        line_fft<T, N>(v, tw, false);
#pragma unroll
        for (int k = 0; k < N; ++k) P[k] = fma(v[k].x, v[k].y, P[k]);
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(128) k_vss_lines(const Cplx<T>* __restrict__ Z, const Cplx<T>* __restrict__ dftw,
                                                   int npairs, int sets, Cplx<T>* __restrict__ W) {
    constexpr int64_t n2 = (int64_t)N * N, n3 = n2 * N;
    __shared__ Cplx<T> tw[N];
    if (threadIdx.x < N) tw[threadIdx.x] = dftw[N + threadIdx.x];
    __syncthreads();
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n2) return;
    const int j = blockIdx.y, nw = gridDim.y;
    const int64_t n = blockIdx.z;
    const int64_t set_stride = (int64_t)npairs * n3;
    T P0[N], P1[N];
#pragma unroll
    for (int k = 0; k < N; ++k) P0[k] = P1[k] = T(0);
    vss_line_products<T, N>(Z + ((n * sets) * npairs + 2 * j) * n3 + l, n2, sets, set_stride, tw, P0);
    if (2 * j + 1 < npairs)
        vss_line_products<T, N>(Z + ((n * sets) * npairs + 2 * j + 1) * n3 + l, n2, sets, set_stride, tw, P1);
    const T two = sets == 1 ? T(2) : T(1), sc = two / T(N);
    Cplx<T> v[N];
#pragma unroll
    for (int k = 0; k < N; ++k) v[line_slot<N>(k)] = Cplx<T>{P0[k], P1[k]};
    line_fft<T, N>(v, tw, true);
    Cplx<T>* w = W + (n * nw + j) * n3 + l;
#pragma unroll
    for (int k = 0; k < N; ++k) w[k * n2] = Cplx<T>{v[k].x * sc, v[k].y * sc};
}

// VHS radial products in Fourier space (the isotropic kernel needs no per-point transform): for
// z-line (x, y) of node n, the inverse z transforms of every sphere point's translate lines give
//   P_r(x, y, z) = sum_p w_p [(T_s f)(T_-s g) + (T_-s f)(T_s g)]     (2 w_p (T_s f)(T_-s f) for g = f)
// summed in registers; P_r is written in the standard layout [x][y][z] through shared memory.
// grid (N^2 / 128, nodes); Z plane-major [n][set][p][kz][x][y]; P_r = P + n stride + r N^3.
template <typename T, int N>
__global__ void __launch_bounds__(128) k_vss_lines_sum(const Cplx<T>* __restrict__ Z, const Cplx<T>* __restrict__ dftw,
                                                       const T* __restrict__ wsig, int npairs, int sets,
                                                       int64_t node_stride, T* __restrict__ P) {
    constexpr int64_t n2 = (int64_t)N * N, n3 = n2 * N;
    constexpr int LINES = 128;
    __shared__ Cplx<T> tw[N];
    __shared__ T tile[LINES * (N + 1)];
    if (threadIdx.x < N) tw[threadIdx.x] = dftw[N + threadIdx.x];
    __syncthreads();
    const int64_t l0 = (int64_t)blockIdx.x * LINES, l = l0 + threadIdx.x;
    const int64_t n = blockIdx.y;
    T acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = T(0);
    Cplx<T> v[N];
    if (l < n2) {
        for (int p = 0; p < npairs; ++p) {
            const T w = wsig[p] * (sets == 1 ? T(2) : T(1));
            for (int s = 0; s < sets; ++s) {
                const Cplx<T>* z = Z + ((n * sets + s) * npairs + p) * n3 + l;
#pragma unroll
                for (int k = 0; k < N; ++k) v[line_slot<N>(k)] = z[k * n2];
                line_fft<T, N>(v, tw, false);
#pragma unroll
                for (int k = 0; k < N; ++k) acc[k] = fma(w * v[k].x, v[k].y, acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < N; ++k) tile[threadIdx.x * (N + 1) + k] = acc[k];
    }
    __syncthreads();
    const int nl = (int)((n2 - l0) < LINES ? (n2 - l0) : LINES);
    T* out = P + n * node_stride + l0 * N;
    for (int e = threadIdx.x; e < nl * N; e += LINES) out[e] = tile[(e / N) * (N + 1) + e % N];
}

// Adjoint (VJP) gain in Fourier space, per radial point r:
//   G_r = sum_p 2 w_p [T_-s(U_r T_-s f) + T_s(U_r T_s f)],   U_r = K_r u,
// with a + i b = IDFT(mu_s f^ + i mu_-s f^) = T_s f + i T_-s f (k_vss_planes<INV>, one set). The two
// products share one forward transform, W = DFT(U_r b + i U_r a), and the back-translates are
// phase multiplies: G^ += 2 w_p [conj(mu_s) (W(k) + conj W(-k)) / 2 + mu_s (W(k) - conj W(-k)) / 2i].
// k_vjp_lines: per (x, y) line, the U_r line (standard layout, staged through shared memory) times
// the inverse z transform of every sphere point's line, packed and transformed forward along z.
// grid (ceil(N^2 / 128), nodes); Z [n][p] and W [n][p] plane-major; U_r = U + n node_stride.
template <typename T, int N>
__global__ void __launch_bounds__(128) k_vjp_lines(const Cplx<T>* __restrict__ Z, const T* __restrict__ U,
                                                   int64_t node_stride, const Cplx<T>* __restrict__ dftw, int npairs,
                                                   Cplx<T>* __restrict__ W) {
    constexpr int64_t n2 = (int64_t)N * N, n3 = n2 * N;
    constexpr int LINES = 128;
    __shared__ Cplx<T> tw[N];
    __shared__ T tile[LINES * (N + 1)];
    const int64_t n = blockIdx.y, l0 = (int64_t)blockIdx.x * LINES, l = l0 + threadIdx.x;
    const int nl = (int)((n2 - l0) < LINES ? (n2 - l0) : LINES);
    if (threadIdx.x < N) tw[threadIdx.x] = dftw[N + threadIdx.x];
    const T* Un = U + n * node_stride + l0 * N;
    for (int e = threadIdx.x; e < nl * N; e += LINES) tile[(e / N) * (N + 1) + e % N] = Un[e];
    __syncthreads();
    if (l >= n2) return;
    T u[N];
#pragma unroll
    for (int k = 0; k < N; ++k) u[k] = tile[threadIdx.x * (N + 1) + k];
    const T sc = T(1) / T(N);
    Cplx<T> v[N];
    for (int p = 0; p < npairs; ++p) {
        const Cplx<T>* z = Z + (n * npairs + p) * n3 + l;
#pragma unroll
        for (int k = 0; k < N; ++k) v[line_slot<N>(k)] = z[k * n2];
        line_fft<T, N>(v, tw, false);
        Cplx<T> w[N];
#pragma unroll
        for (int k = 0; k < N; ++k) w[line_slot<N>(k)] = Cplx<T>{u[k] * v[k].y, u[k] * v[k].x};   // U b + i U a
        line_fft<T, N>(w, tw, true);
        Cplx<T>* o = W + (n * npairs + p) * n3 + l;
#pragma unroll
        for (int k = 0; k < N; ++k) o[k * n2] = Cplx<T>{w[k].x * sc, w[k].y * sc};
    }
}

// G^[n](k) += sum_p 2 w_p [conj(mu_s) P1^ + mu_s P2^],  P1^ = (W + conj W(-k)) / 2,
// P2^ = (W - conj W(-k)) / 2i; mu_r: [npairs][3][N] per-axis multipliers; plane-major index.
// grid (ceil(n3 / 256), nodes); dynamic shared memory: npairs 3 N complex
template <typename T>
__global__ void __launch_bounds__(256) k_vjp_accumulate(const Cplx<T>* __restrict__ W, const Cplx<T>* __restrict__ mu_r,
                                                        const T* __restrict__ wsig, int N, int npairs, int64_t n3,
                                                        Cplx<T>* __restrict__ Gh) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Cplx<T>* m = reinterpret_cast<Cplx<T>*>(sm_raw);
    for (int i = threadIdx.x; i < npairs * 3 * N; i += blockDim.x) m[i] = mu_r[i];
    __syncthreads();
    const int64_t n = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n3) return;
    const int kz = (int)(e / ((int64_t)N * N)), kx = (int)((e / N) % N), ky = (int)(e % N);
    const int64_t em = ((int64_t)((N - kz) % N) * N + (N - kx) % N) * N + (N - ky) % N;
    T re = 0, im = 0;
    for (int p = 0; p < npairs; ++p) {
        const Cplx<T>* mp = m + p * 3 * N;
        const Cplx<T> a = mp[kx], b = mp[N + ky], c = mp[2 * N + kz];
        const Cplx<T> ab{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
        const Cplx<T> mu{ab.x * c.x - ab.y * c.y, ab.x * c.y + ab.y * c.x};
        const Cplx<T> w = W[(n * npairs + p) * n3 + e], wm = W[(n * npairs + p) * n3 + em];
        const Cplx<T> p1{T(0.5) * (w.x + wm.x), T(0.5) * (w.y - wm.y)};
        const Cplx<T> p2{T(0.5) * (w.y + wm.y), T(-0.5) * (w.x - wm.x)};
        const T two_w = T(2) * wsig[p];
        // conj(mu) p1 + mu p2
        re = fma(two_w, (mu.x * p1.x + mu.y * p1.y) + (mu.x * p2.x - mu.y * p2.y), re);
        im = fma(two_w, (mu.x * p1.y - mu.y * p1.x) + (mu.x * p2.y + mu.y * p2.x), im);
    }
    Cplx<T>& g = Gh[n * n3 + e];
    g.x += re;
    g.y += im;
}

// out[n][x][y][z] = Re Gt[n][z][x][y]
template <typename T>
__global__ void __launch_bounds__(256) k_vjp_real_t(const Cplx<T>* __restrict__ Gt, int N, int64_t n3,
                                                    T* __restrict__ out) {
    const int64_t n = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const int64_t n2 = (int64_t)N * N;
    const int x = (int)(i / n2), y = (int)((i / N) % N), z = (int)(i % N);
    out[n * n3 + i] = Gt[n * n3 + ((int64_t)z * N + x) * N + y].x;
}

// X[n][z][x][y] = {f[n][x][y][z], 0}: a real field into a plane-major complex field; node n of f
// starts at offs[n] (offs == nullptr: n N^3)
template <typename T>
__global__ void __launch_bounds__(256) k_vss_load_t(const T* __restrict__ f, const int64_t* __restrict__ offs, int N,
                                                    int64_t n3, Cplx<T>* __restrict__ X) {
    const int64_t n = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // plane-major index
    if (e >= n3) return;
    const int64_t n2 = (int64_t)N * N;
    const int z = (int)(e / n2), x = (int)((e / N) % N), y = (int)(e % N);
    const int64_t base = offs ? offs[n] : n * n3;
    X[n * n3 + e] = Cplx<T>{f[base + ((int64_t)x * N + y) * N + z], T(0)};
}

// out[n][x][y][z] = Re Y0 - a Re Y1 - (c ? c Re Y2 : 0), Y plane-major [n][yfields][z][x][y]
template <typename T>
__global__ void __launch_bounds__(256) k_vss_finalize_t(const Cplx<T>* __restrict__ Y, int yfields, const T* __restrict__ a,
                                                        const T* __restrict__ c, int N, int64_t n3, T* __restrict__ out,
                                                        int* __restrict__ flags) {
    const int64_t n = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // standard index
    if (i >= n3) return;
    const int64_t n2 = (int64_t)N * N;
    const int x = (int)(i / n2), y = (int)((i / N) % N), z = (int)(i % N);
    const int64_t e = ((int64_t)z * N + x) * N + y;
    const Cplx<T>* Yn = Y + n * yfields * n3;
    T v = Yn[e].x - a[n * n3 + i] * Yn[n3 + e].x;
    if (c) v -= c[n * n3 + i] * Yn[2 * n3 + e].x;
    if (!isfinite(v)) atomicOr(flags, 2);
    out[n * n3 + i] = v;
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

template <typename T, int N, bool INV>
cudaError_t planes_launch(const Cplx<T>* Fh, const Cplx<T>* Gh, const Cplx<T>* mu_r, const Cplx<T>* dftw, int npairs,
                          int fields, int64_t nodes, Cplx<T>* X, cudaStream_t s) {
    using G = PlaneGeo<T, N>;
    auto kern = k_vss_planes<T, N, INV>;
    if (G::smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<dim3(N / G::KZ, (unsigned)fields, (unsigned)nodes), G::NT, G::smem, s>>>(Fh, Gh, mu_r, dftw, npairs, X);
    return cudaGetLastError();
}

}  // namespace

bool vss_fused_supported(int N, bool fp64) { return N == 8 || N == 12 || N == 16 || N == 24 || (N == 32 && !fp64); }

bool fft_translate_supported(int N) { return N == 8 || N == 12 || N == 16 || N == 24 || N == 32; }

template <typename T>
cudaError_t launch_vss_load_t(const T* f, const int64_t* offs, int N, int64_t nodes, Cplx<T>* X, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    k_vss_load_t<T><<<dim3(nblk(n3), (unsigned)nodes), 256, 0, s>>>(f, offs, N, n3, X);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vss_inverse_planes(const Cplx<T>* Fh, const Cplx<T>* Gh, const Cplx<T>* mu_r, const Cplx<T>* dftw,
                                      int N, int npairs, int sets, int64_t nodes, Cplx<T>* Z, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const int fields = sets * npairs;
    if (N == 8) return planes_launch<T, 8, true>(Fh, Gh, mu_r, dftw, npairs, fields, nodes, Z, s);
    if (N == 12) return planes_launch<T, 12, true>(Fh, Gh, mu_r, dftw, npairs, fields, nodes, Z, s);
    if (N == 16) return planes_launch<T, 16, true>(Fh, Gh, mu_r, dftw, npairs, fields, nodes, Z, s);
    if (N == 24) return planes_launch<T, 24, true>(Fh, Gh, mu_r, dftw, npairs, fields, nodes, Z, s);
    if (N == 32) return planes_launch<T, 32, true>(Fh, Gh, mu_r, dftw, npairs, fields, nodes, Z, s);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_vss_lines(const Cplx<T>* Z, const Cplx<T>* dftw, int N, int npairs, int sets, int64_t nodes,
                             Cplx<T>* W, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((N * N + 127) / 128), (unsigned)((npairs + 1) / 2), (unsigned)nodes);
    if (N == 8) k_vss_lines<T, 8><<<grid, 128, 0, s>>>(Z, dftw, npairs, sets, W);
    else if (N == 12) k_vss_lines<T, 12><<<grid, 128, 0, s>>>(Z, dftw, npairs, sets, W);
    else if (N == 16) k_vss_lines<T, 16><<<grid, 128, 0, s>>>(Z, dftw, npairs, sets, W);
    else if (N == 24) k_vss_lines<T, 24><<<grid, 128, 0, s>>>(Z, dftw, npairs, sets, W);
    else if (sizeof(T) == 4 && N == 32) k_vss_lines<T, sizeof(T) == 4 ? 32 : 16><<<grid, 128, 0, s>>>(Z, dftw, npairs, sets, W);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vss_forward_planes(const Cplx<T>* dftw, int N, int fields, int64_t nodes, Cplx<T>* W,
                                      cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    if (N == 8) return planes_launch<T, 8, false>(nullptr, nullptr, nullptr, dftw, 0, fields, nodes, W, s);
    if (N == 12) return planes_launch<T, 12, false>(nullptr, nullptr, nullptr, dftw, 0, fields, nodes, W, s);
    if (N == 16) return planes_launch<T, 16, false>(nullptr, nullptr, nullptr, dftw, 0, fields, nodes, W, s);
    if (N == 24) return planes_launch<T, 24, false>(nullptr, nullptr, nullptr, dftw, 0, fields, nodes, W, s);
    if (N == 32) return planes_launch<T, 32, false>(nullptr, nullptr, nullptr, dftw, 0, fields, nodes, W, s);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_vss_lines_sum(const Cplx<T>* Z, const Cplx<T>* dftw, const T* wsig, int N, int npairs, int sets,
                                 int64_t nodes, int64_t node_stride, T* P, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((N * N + 127) / 128), (unsigned)nodes);
    if (N == 8) k_vss_lines_sum<T, 8><<<grid, 128, 0, s>>>(Z, dftw, wsig, npairs, sets, node_stride, P);
    else if (N == 12) k_vss_lines_sum<T, 12><<<grid, 128, 0, s>>>(Z, dftw, wsig, npairs, sets, node_stride, P);
    else if (N == 16) k_vss_lines_sum<T, 16><<<grid, 128, 0, s>>>(Z, dftw, wsig, npairs, sets, node_stride, P);
    else if (N == 24) k_vss_lines_sum<T, 24><<<grid, 128, 0, s>>>(Z, dftw, wsig, npairs, sets, node_stride, P);
    else if (N == 32) k_vss_lines_sum<T, 32><<<grid, 128, 0, s>>>(Z, dftw, wsig, npairs, sets, node_stride, P);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vjp_lines(const Cplx<T>* Z, const T* U, int64_t node_stride, const Cplx<T>* dftw, int N,
                             int npairs, int64_t nodes, Cplx<T>* W, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((N * N + 127) / 128), (unsigned)nodes);
    if (N == 8) k_vjp_lines<T, 8><<<grid, 128, 0, s>>>(Z, U, node_stride, dftw, npairs, W);
    else if (N == 12) k_vjp_lines<T, 12><<<grid, 128, 0, s>>>(Z, U, node_stride, dftw, npairs, W);
    else if (N == 16) k_vjp_lines<T, 16><<<grid, 128, 0, s>>>(Z, U, node_stride, dftw, npairs, W);
    else if (N == 24) k_vjp_lines<T, 24><<<grid, 128, 0, s>>>(Z, U, node_stride, dftw, npairs, W);
    else if (N == 32) k_vjp_lines<T, 32><<<grid, 128, 0, s>>>(Z, U, node_stride, dftw, npairs, W);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vjp_accumulate(const Cplx<T>* W, const Cplx<T>* mu_r, const T* wsig, int N, int npairs,
                                  int64_t nodes, Cplx<T>* Gh, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    const size_t sm = (size_t)npairs * 3 * N * sizeof(Cplx<T>);
    if (sm > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_vjp_accumulate<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_vjp_accumulate<T><<<dim3(nblk(n3), (unsigned)nodes), 256, sm, s>>>(W, mu_r, wsig, N, npairs, n3, Gh);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vjp_real_t(const Cplx<T>* Gt, int N, int64_t nodes, T* out, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    k_vjp_real_t<T><<<dim3(nblk(n3), (unsigned)nodes), 256, 0, s>>>(Gt, N, n3, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vss_finalize_t(const Cplx<T>* Y, int yfields, const T* a, const T* c, int N, int64_t nodes, T* out,
                                  int* flags, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (nodes > 65535) return cudaErrorInvalidValue;
    const int64_t n3 = (int64_t)N * N * N;
    k_vss_finalize_t<T><<<dim3(nblk(n3), (unsigned)nodes), 256, 0, s>>>(Y, yfields, a, c, N, n3, out, flags);
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
    template cudaError_t launch_vss_accumulate<T>(const Cplx<T>*, const T*, int, int, int64_t, T, Cplx<T>*, int, \
                                                  cudaStream_t);                                                  \
    template cudaError_t launch_vss_loss_init<T>(const Cplx<T>*, const Cplx<T>*, const T*, int, int64_t,         \
                                                 Cplx<T>*, int, cudaStream_t);                                    \
    template cudaError_t launch_vss_load_t<T>(const T*, const int64_t*, int, int64_t, Cplx<T>*, cudaStream_t);                    \
    template cudaError_t launch_vss_inverse_planes<T>(const Cplx<T>*, const Cplx<T>*, const Cplx<T>*,            \
                                                      const Cplx<T>*, int, int, int, int64_t, Cplx<T>*,           \
                                                      cudaStream_t);                                              \
    template cudaError_t launch_vss_lines<T>(const Cplx<T>*, const Cplx<T>*, int, int, int, int64_t, Cplx<T>*,   \
                                             cudaStream_t);                                                       \
    template cudaError_t launch_vss_forward_planes<T>(const Cplx<T>*, int, int, int64_t, Cplx<T>*, cudaStream_t); \
    template cudaError_t launch_vss_finalize_t<T>(const Cplx<T>*, int, const T*, const T*, int, int64_t, T*,     \
                                                  int*, cudaStream_t);                                            \
    template cudaError_t launch_vjp_lines<T>(const Cplx<T>*, const T*, int64_t, const Cplx<T>*, int, int, int64_t, \
                                             Cplx<T>*, cudaStream_t);                                             \
    template cudaError_t launch_vjp_accumulate<T>(const Cplx<T>*, const Cplx<T>*, const T*, int, int, int64_t,     \
                                                  Cplx<T>*, cudaStream_t);                                        \
    template cudaError_t launch_vjp_real_t<T>(const Cplx<T>*, int, int64_t, T*, cudaStream_t);                    \
    template cudaError_t launch_vss_lines_sum<T>(const Cplx<T>*, const Cplx<T>*, const T*, int, int, int, int64_t, \
                                                 int64_t, T*, cudaStream_t);
DGFS_VSS_INST(float)
DGFS_VSS_INST(double)
#undef DGFS_VSS_INST

}  // namespace dgfs
