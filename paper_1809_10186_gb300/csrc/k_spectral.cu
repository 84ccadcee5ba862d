// Fused Fourier stage for power-of-two grids (N = 8, 16, 32): the same arithmetic as the
// projection, forward DFT, Fourier combine, inverse DFT and finalisation kernels of
// k_fourier.cu (arXiv:1809.10186, Appendix, eqs. realGG, lowrank1, apndx_fs_Glm_Qk), in three
// launches whose intermediates stay in shared memory between the axis passes:
//
//   k_spec_xz   one (x, z) plane y = const of a node: X_s = sum_r C[s][r] P_r for every s, the loss
//               operand(s), packed two real fields per complex slot; forward FFT along x and z
//   k_spec_y    the planes kx and -kx of every slot: forward FFT along y, the spectra of the
//               packed fields separated with the mirror point -k (in the other plane),
//               gain^ = sum_s Uk[s] X^_s and loss^ = GL(k) g^; inverse FFT along y and z
//   k_spec_xout one plane y = const: inverse FFT along x, Q = gain - f (K_L g)
//
// Per node this moves P (Nrho N^3), the packed slots twice and the two or three result fields
// twice through HBM instead of the slots seven times and the results four times.
#include <cstdint>

#include "fourier_dev.cuh"
#include "launchers.h"

namespace dgfs {

namespace {

using namespace fdev;

template <int N>
struct SpecGeo {
    static constexpr int N2 = N * N;
    static constexpr int ROW = N + 1;                          // padded plane row (complex values)
    static constexpr int PLANE = N * ROW;
    static constexpr int T1 = N == 8 ? 64 : 256;                // k_spec_xz: V points per thread
    static constexpr int V = N2 / T1;
    static constexpr int SL = N == 32 ? 5 : 8;                  // slots (2 SL fields) per k_spec_xz CTA
    static constexpr int RB = 16;                               // radial points of P in flight per thread
    static constexpr int T2 = 256;                             // k_spec_y
    static constexpr int GS = T2 / (2 * N);                    // slots per group: one y line per thread
    static constexpr int PT = (2 * N2 + T2 - 1) / T2;          // points per thread in k_spec_y
    static constexpr int T3 = 256;                             // k_spec_xout
    static_assert(V == 1 || V == 4, "points per thread");
};

template <typename T, int V>
__device__ __forceinline__ void load_v(const T* p, T (&v)[V]) {
    if constexpr (V == 4) {
        static_assert(sizeof(T) == 4, "four points per thread only in float");
        const float4 u = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = u.x;
        v[1] = u.y;
        v[2] = u.z;
        v[3] = u.w;
    } else {
        v[0] = __ldg(p);
    }
}

// signed lattice index of DFT position q
template <int N>
__device__ __forceinline__ int signed_q(int q) { return q < N / 2 ? q : q - N; }

// Asynchronous global -> shared copy of one complex value (8 or 16 bytes, both addresses aligned
// to the size); cp_async_wait_all() before the barrier that publishes the data.
template <typename T>
__device__ __forceinline__ void cp_async_cplx(Cplx<T>* dst, const Cplx<T>* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(Cplx<T>) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }
// V consecutive values (V * sizeof(T) = 4, 8 or 16 bytes, both addresses aligned to it)
template <typename T, int V>
__device__ __forceinline__ void cp_async_v(T* dst, const T* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    constexpr int B = V * (int)sizeof(T);
    if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(B) : "memory");
}

// One line of N complex values in shared memory (element k at base[k * stride]) transformed in
// place in registers, times `scale`.
template <typename T, int N>
__device__ __forceinline__ void fft_smem_line(Cplx<T>* base, int stride, const Cplx<T>* tw, bool forward, T scale) {
    Cplx<T> a[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a[bitrev<N>(k)] = base[k * stride];
    fft_line<T, N>(a, tw, forward);
#pragma unroll
    for (int k = 0; k < N; ++k) base[k * stride] = Cplx<T>{a[k].x * scale, a[k].y * scale};
}

// ---- kernel 1: projection + loss operands + forward FFT along x and z of one plane y -------
// CTA (slot group g, plane y) of a node: slots [g SL, g SL + SL) of the packed fields, i.e.
// fields 2 g SL .. 2 g SL + 2 SL - 1. The slot groups of one plane run next to each other, so
// the plane of P (Nrho N^2 values) comes from HBM once and from L2 for the other groups.
template <typename T, int N>
__global__ void __launch_bounds__(SpecGeo<N>::T1)
k_spec_xz(const T* __restrict__ P, const T* __restrict__ Vr, const double* __restrict__ cr,
          const double* __restrict__ wr, NodeParams np, int Nrho, int rank, const T* __restrict__ la,
          const T* __restrict__ lb, const int64_t* __restrict__ offs, int nloss,
          const Cplx<T>* __restrict__ W, Cplx<T>* __restrict__ X, int xs, int groups) {
    using G = SpecGeo<N>;
    constexpr int FG = 2 * G::SL;                               // fields of one slot group
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Cplx<T>* F = reinterpret_cast<Cplx<T>*>(sm_raw);           // [SL][PLANE]
    Cplx<T>* tw = F + G::SL * G::PLANE;                         // [N]
    T* CT = reinterpret_cast<T*>(tw + N);                       // [Nrho][FG]
    T* wrho = CT + Nrho * FG;                                   // [Nrho]
    T* ring = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(wrho + Nrho) + 15) & ~uintptr_t(15));
                                                                // [RB][T1 V]: asynchronous copies of P
    const int g = blockIdx.x % groups, y = blockIdx.x / groups, t = threadIdx.x;
    const int s0 = g * G::SL, ns = xs - s0 < G::SL ? xs - s0 : G::SL, f0 = 2 * s0;
    const int64_t node = blockIdx.y, n3 = (int64_t)N * G::N2;
    const double gam = np.gamma ? np.gamma[node] : np.gamma0;
    const double bb = np.b ? np.b[node] : np.b0;
    if (t < N) tw[t] = W[N + t];                                // row q = 1 of the DFT table
    for (int r = t; r < Nrho; r += G::T1) wrho[r] = (T)wr[r] * radial_rho<T>(bb, gam, cr[r], np.dlog);
    __syncthreads();
    for (int e = t; e < Nrho * FG; e += G::T1) {
        const int r = e / FG, fi = f0 + e % FG;
        CT[e] = fi < rank ? Vr[fi * Nrho + r] * wrho[r] : T(0);
    }
    __syncthreads();
    // this thread's points: (x, z0 .. z0 + V - 1) of plane y
    const int x = t / (N / G::V), z0 = (t % (N / G::V)) * G::V;
    const int64_t j0 = ((int64_t)x * N + y) * N + z0;
    if (f0 < rank) {
        T acc[G::V][FG];
#pragma unroll
        for (int v = 0; v < G::V; ++v)
#pragma unroll
            for (int i = 0; i < FG; ++i) acc[v][i] = T(0);
        // each thread streams its own V values of P_r through a ring of RB asynchronous copies
        // (one commit group per r), so RB radial points are in flight without holding registers
        const T* Pn = P + node * Nrho * n3 + j0;
        T* mine = ring + t * G::V;
        auto issue = [&](int r) {
            if (r < Nrho) cp_async_v<T, G::V>(mine + (r % G::RB) * (G::T1 * G::V), Pn + (int64_t)r * n3);
            cp_async_commit();
        };
#pragma unroll
        for (int r = 0; r < G::RB; ++r) issue(r);
#pragma unroll 4
        for (int r = 0; r < Nrho; ++r) {
            cp_async_wait_group<G::RB - 1>();   // the copy of P_r has landed
            T p[G::V];
#pragma unroll
            for (int v = 0; v < G::V; ++v) p[v] = mine[(r % G::RB) * (G::T1 * G::V) + v];
            const T* c = CT + r * FG;
#pragma unroll
            for (int i = 0; i < FG; ++i)
#pragma unroll
                for (int v = 0; v < G::V; ++v) acc[v][i] = fma(c[i], p[v], acc[v][i]);
            issue(r + G::RB);   // after the FMAs that consumed the slot's values
        }
        cp_async_wait_all();
#pragma unroll
        for (int i = 0; i < FG; i += 2)
            if (i / 2 < ns)
#pragma unroll
                for (int v = 0; v < G::V; ++v)
                    F[(i / 2) * G::PLANE + x * G::ROW + z0 + v] =
                        Cplx<T>{f0 + i < rank ? acc[v][i] : T(0), f0 + i + 1 < rank ? acc[v][i + 1] : T(0)};
    }
    // loss operand(s): fields rank, rank + 1 (the imaginary part of a slot past the last field is 0)
    const int64_t base = offs ? offs[node] : node * n3;
    for (int jl = 0; jl < nloss; ++jl) {
        const int fi = rank + jl - f0;
        if (fi < 0 || fi >= 2 * ns) continue;
        const T* src = (jl ? lb : la) + base + j0;
#pragma unroll
        for (int v = 0; v < G::V; ++v) {
            Cplx<T>& d = F[(fi / 2) * G::PLANE + x * G::ROW + z0 + v];
            const T val = src[v];
            if (fi % 2 == 0) d = Cplx<T>{val, T(0)};
            else d.y = val;
        }
    }
    __syncthreads();
    const T inv = T(1) / T(N);
    for (int id = t; id < ns * N; id += G::T1) {   // along x: line (slot, z)
        const int m = id / N, z = id % N;
        fft_smem_line<T, N>(F + m * G::PLANE + z, G::ROW, tw, true, inv);
    }
    __syncthreads();
    for (int id = t; id < ns * N; id += G::T1) {   // along z: line (slot, kx)
        const int m = id / N, kx = id % N;
        fft_smem_line<T, N>(F + m * G::PLANE + kx * G::ROW, 1, tw, true, inv);
    }
    __syncthreads();
    Cplx<T>* Xn = X + (node * (int64_t)xs + s0) * n3;
    for (int e = t; e < ns * G::N2; e += G::T1) {   // X[slot][kx][y][kz]
        const int m = e / G::N2, kx = (e / N) % N, kz = e % N;
        Xn[m * n3 + ((int64_t)kx * N + y) * N + kz] = F[m * G::PLANE + kx * G::ROW + kz];
    }
}

// ---- kernel 2: FFT along y, combine, inverse FFT along y and z of the planes kx, -kx ----------
template <typename T, int N, int NL>
__global__ void __launch_bounds__(SpecGeo<N>::T2, NL == 1 ? 2 : 1)
k_spec_y(const Cplx<T>* __restrict__ X, int xs, const T* __restrict__ Uq, int nq2, const T* __restrict__ Lr,
         const T* __restrict__ GL0, const T* __restrict__ GLd, const double* __restrict__ cr, NodeParams np,
         int Nrho, int rank, int lf0, int lf1, T scale, const Cplx<T>* __restrict__ W,
         Cplx<T>* __restrict__ Y, int yf) {
    using G = SpecGeo<N>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Cplx<T>* buf = reinterpret_cast<Cplx<T>*>(sm_raw);         // [GS][2][PLANE]; later [yf][2][PLANE]
    Cplx<T>* tw = buf + G::GS * 2 * G::PLANE;                   // [N]
    double* rho = reinterpret_cast<double*>(tw + N);            // [Nrho]
    const int kx = blockIdx.x, kxm = (N - kx) % N, npl = kx == kxm ? 1 : 2, t = threadIdx.x;
    const int64_t node = blockIdx.y, n3 = (int64_t)N * G::N2;
    const bool per_node = np.gamma || np.b;
    if (t < N) tw[t] = W[N + t];
    if (per_node) {
        const double gam = np.gamma ? np.gamma[node] : np.gamma0;
        const double bb = np.b ? np.b[node] : np.b0;
        for (int r = t; r < Nrho; r += G::T2) rho[r] = radial_rho<double>(bb, gam, cr[r], np.dlog);
    }
    const Cplx<T>* Xn = X + node * (int64_t)xs * n3;
    const T inv = T(1) / T(N);
    T gr[G::PT], gi[G::PT];
    Cplx<T> l0[G::PT], l1[NL == 2 ? G::PT : 1];
#pragma unroll
    for (int i = 0; i < G::PT; ++i) {
        gr[i] = gi[i] = T(0);
        l0[i] = Cplx<T>{T(0), T(0)};
        if constexpr (NL == 2) l1[i] = Cplx<T>{T(0), T(0)};
    }
    for (int g0 = 0; g0 < xs; g0 += G::GS) {
        const int ng = xs - g0 < G::GS ? xs - g0 : G::GS;
        __syncthreads();   // the previous group's combine has read buf
        for (int e = t; e < ng * npl * G::N2; e += G::T2) {
            const int jm = e / (npl * G::N2), rem = e % (npl * G::N2);
            const int pl = rem / G::N2, yy = (rem / N) % N, kz = rem % N;
            const int kxp = pl ? kxm : kx;
            cp_async_cplx(buf + (jm * 2 + pl) * G::PLANE + yy * G::ROW + kz,
                          Xn + (g0 + jm) * n3 + ((int64_t)kxp * N + yy) * N + kz);
        }
        cp_async_wait_all();
        __syncthreads();
        for (int id = t; id < ng * npl * N; id += G::T2) {   // along y: line (slot, plane, kz)
            const int jm = id / (npl * N), rem = id % (npl * N), pl = rem / N, kz = rem % N;
            fft_smem_line<T, N>(buf + (jm * 2 + pl) * G::PLANE + kz, G::ROW, tw, true, inv);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < G::PT; ++i) {
            const int e = t + i * G::T2;
            if (e >= npl * G::N2) continue;
            const int pl = e / G::N2, ky = (e / N) % N, kz = e % N;
            const int pm = npl == 2 ? 1 - pl : 0, kym = (N - ky) % N, kzm = (N - kz) % N;
            const int kxp = pl ? kxm : kx;
            const int q2 = signed_q<N>(kxp) * signed_q<N>(kxp) + signed_q<N>(ky) * signed_q<N>(ky) +
                           signed_q<N>(kz) * signed_q<N>(kz);   // Uk[s](k) = Uq[s][|k|^2]
            for (int jm = 0; jm < ng; ++jm) {
                const Cplx<T> z = buf[(jm * 2 + pl) * G::PLANE + ky * G::ROW + kz];
                const Cplx<T> w = buf[(jm * 2 + pm) * G::PLANE + kym * G::ROW + kzm];
                // spectra of the real fields 2m and 2m + 1 packed in slot m
                const Cplx<T> fa{(z.x + w.x) * T(0.5), (z.y - w.y) * T(0.5)};
                const Cplx<T> fb{(z.y + w.y) * T(0.5), (w.x - z.x) * T(0.5)};
                const int m = g0 + jm;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int fi = 2 * m + h;
                    const Cplx<T> v = h ? fb : fa;
                    if (fi < rank) {
                        const T u = __ldg(Uq + fi * nq2 + q2);
                        gr[i] = fma(u, v.x, gr[i]);
                        gi[i] = fma(u, v.y, gi[i]);
                    } else if (fi == lf0) {
                        l0[i] = v;
                    } else if (NL == 2 && fi == lf1) {
                        l1[NL == 2 ? i : 0] = v;
                    }
                }
            }
        }
    }
    __syncthreads();   // every combine has read buf: it now holds the result fields
#pragma unroll
    for (int i = 0; i < G::PT; ++i) {
        const int e = t + i * G::T2;
        if (e >= npl * G::N2) continue;
        const int pl = e / G::N2, ky = (e / N) % N, kz = e % N;
        const int64_t k = ((int64_t)(pl ? kxm : kx) * N + ky) * N + kz;
        const T GL = loss_multiplier<T>(GL0, GLd, Lr, rho, per_node, np.dlog, Nrho, n3, k);
        const int o = pl * G::PLANE + ky * G::ROW + kz;
        buf[o] = Cplx<T>{scale * gr[i], scale * gi[i]};
        buf[2 * G::PLANE + o] = Cplx<T>{GL * l0[i].x, GL * l0[i].y};
        if constexpr (NL == 2) buf[4 * G::PLANE + o] = Cplx<T>{GL * l1[i].x, GL * l1[i].y};
    }
    __syncthreads();
    for (int id = t; id < yf * npl * N; id += G::T2) {   // inverse along y: line (field, plane, kz)
        const int fo = id / (npl * N), rem = id % (npl * N), pl = rem / N, kz = rem % N;
        fft_smem_line<T, N>(buf + (fo * 2 + pl) * G::PLANE + kz, G::ROW, tw, false, T(1));
    }
    __syncthreads();
    for (int id = t; id < yf * npl * N; id += G::T2) {   // inverse along z: line (field, plane, y)
        const int fo = id / (npl * N), rem = id % (npl * N), pl = rem / N, yy = rem % N;
        fft_smem_line<T, N>(buf + (fo * 2 + pl) * G::PLANE + yy * G::ROW, 1, tw, false, T(1));
    }
    __syncthreads();
    Cplx<T>* Yn = Y + node * (int64_t)yf * n3;
    for (int e = t; e < yf * npl * G::N2; e += G::T2) {   // Y[field][kx][y][z]
        const int fo = e / (npl * G::N2), rem = e % (npl * G::N2);
        const int pl = rem / G::N2, yy = (rem / N) % N, z = rem % N;
        Yn[fo * n3 + ((int64_t)(pl ? kxm : kx) * N + yy) * N + z] = buf[(fo * 2 + pl) * G::PLANE + yy * G::ROW + z];
    }
}

// ---- kernel 3: inverse FFT along x of one plane y, Q = gain - a (K_L g) [- c (K_L f)] --------
template <typename T, int N>
__global__ void __launch_bounds__(SpecGeo<N>::T3)
k_spec_xout(const Cplx<T>* __restrict__ Y, int yf, const T* __restrict__ a, const T* __restrict__ c,
            const int64_t* __restrict__ offs, const Cplx<T>* __restrict__ W, T* __restrict__ out,
            int* __restrict__ flags) {
    using G = SpecGeo<N>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Cplx<T>* yb = reinterpret_cast<Cplx<T>*>(sm_raw);          // [yf][PLANE]
    Cplx<T>* tw = yb + yf * G::PLANE;                           // [N]
    const int y = blockIdx.x, t = threadIdx.x;
    const int64_t node = blockIdx.y, n3 = (int64_t)N * G::N2;
    if (t < N) tw[t] = W[N + t];
    const Cplx<T>* Yn = Y + node * (int64_t)yf * n3;
    for (int e = t; e < yf * G::N2; e += G::T3) {
        const int fo = e / G::N2, kx = (e / N) % N, z = e % N;
        cp_async_cplx(yb + fo * G::PLANE + kx * G::ROW + z, Yn + fo * n3 + ((int64_t)kx * N + y) * N + z);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int id = t; id < yf * N; id += G::T3) {   // inverse along x: line (field, z)
        const int fo = id / N, z = id % N;
        fft_smem_line<T, N>(yb + fo * G::PLANE + z, G::ROW, tw, false, T(1));
    }
    __syncthreads();
    const int64_t base = offs ? offs[node] : node * n3;
    for (int e = t; e < G::N2; e += G::T3) {
        const int xx = e / N, z = e % N;
        const int64_t j = ((int64_t)xx * N + y) * N + z;
        const int o = xx * G::ROW + z;
        T v = yb[o].x - a[base + j] * yb[G::PLANE + o].x;
        if (c) v -= c[base + j] * yb[2 * G::PLANE + o].x;
        if (!isfinite(v)) atomicOr(flags, 2);
        out[base + j] = v;
    }
}

template <typename T, int N>
cudaError_t spectral_n(const DevTables<T>& t, const T* P, NodeParams np, int64_t nodes, const T* la,
                       const T* lb, const int64_t* offs, T gain_scale, Cplx<T>* X, Cplx<T>* Y, const T* fa,
                       const T* fc, T* out, int* flags, cudaStream_t s) {
    using G = SpecGeo<N>;
    const int nloss = lb ? 2 : 1, nfields = t.rank + nloss, xs = (nfields + 1) / 2, yf = lb ? 3 : 2;
    const Cplx<T>* W = reinterpret_cast<const Cplx<T>*>(t.dftw);
    const unsigned nn = (unsigned)nodes;
    cudaError_t e;
    {
        const int groups = (xs + G::SL - 1) / G::SL;
        const size_t sm = sizeof(Cplx<T>) * ((size_t)G::SL * G::PLANE + N) +
                          sizeof(T) * ((size_t)t.Nrho * (2 * G::SL + 1) + (size_t)G::RB * G::T1 * G::V) + 16;
        e = cudaFuncSetAttribute(k_spec_xz<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_spec_xz<T, N><<<dim3(groups * N, nn), G::T1, sm, s>>>(P, t.Vr, t.cr, t.wr, np, t.Nrho, t.rank, la, lb, offs,
                                                                 nloss, W, X, xs, groups);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    {
        const size_t sm = sizeof(Cplx<T>) * ((size_t)G::GS * 2 * G::PLANE + N) + sizeof(double) * (size_t)t.Nrho;
        auto kern = lb ? k_spec_y<T, N, 2> : k_spec_y<T, N, 1>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        kern<<<dim3(N / 2 + 1, nn), G::T2, sm, s>>>(X, xs, t.Uq, 3 * (N / 2) * (N / 2) + 1, t.Lr, t.GL0, t.GLd, t.cr, np, t.Nrho,
                                                               t.rank, t.rank, lb ? t.rank + 1 : -1, gain_scale, W,
                                                               Y, yf);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    {
        const size_t sm = sizeof(Cplx<T>) * ((size_t)yf * G::PLANE + N);
        k_spec_xout<T, N><<<dim3(N, nn), G::T3, sm, s>>>(Y, yf, fa, fc, offs, W, out, flags);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

template <typename T>
bool spectral_supported(const DevTables<T>& t) {
    if (t.rank < 1 || t.rank > 32 || t.Nrho > 64) return false;
    if (t.N == 8 || t.N == 16) return true;
    return t.N == 32 && sizeof(T) == 4;
}

template <typename T>
cudaError_t launch_spectral(const DevTables<T>& t, const T* P, NodeParams np, int64_t nodes, const T* la,
                            const T* lb, const int64_t* offs, T gain_scale, Cplx<T>* X, Cplx<T>* Y,
                            const T* fa, const T* fc, T* out, int* flags, cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    if (!spectral_supported(t)) return cudaErrorNotSupported;
    const int64_t n3 = (int64_t)t.N * t.N * t.N;
    const int nloss = lb ? 2 : 1, xs = (t.rank + nloss + 1) / 2, yf = lb ? 3 : 2;
    for (int64_t n0 = 0; n0 < nodes; n0 += 65535) {   // grid.y limit
        const int64_t nn = nodes - n0 < 65535 ? nodes - n0 : 65535;
        // node-indexed pointers of this sub-range (with offs, field pointers stay chunk bases)
        const int64_t fo = offs ? 0 : n0 * n3;
        const int64_t* o = offs ? offs + n0 : nullptr;
        const T* P0 = P + n0 * t.Nrho * n3;
        Cplx<T>* X0 = X + n0 * xs * n3;
        Cplx<T>* Y0 = Y + n0 * yf * n3;
        const T* la0 = la + fo;
        const T* lb0 = lb ? lb + fo : nullptr;
        const T* fa0 = fa + fo;
        const T* fc0 = fc ? fc + fo : nullptr;
        T* out0 = out + fo;
        NodeParams np0 = np;
        if (np.gamma) np0.gamma = np.gamma + n0;
        if (np.b) np0.b = np.b + n0;
        cudaError_t e = cudaErrorNotSupported;
        if (t.N == 8) e = spectral_n<T, 8>(t, P0, np0, nn, la0, lb0, o, gain_scale, X0, Y0, fa0, fc0, out0, flags, s);
        else if (t.N == 16)
            e = spectral_n<T, 16>(t, P0, np0, nn, la0, lb0, o, gain_scale, X0, Y0, fa0, fc0, out0, flags, s);
        else if constexpr (sizeof(T) == 4)
            e = spectral_n<T, 32>(t, P0, np0, nn, la0, lb0, o, gain_scale, X0, Y0, fa0, fc0, out0, flags, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template bool spectral_supported<float>(const DevTables<float>&);
template bool spectral_supported<double>(const DevTables<double>&);
template cudaError_t launch_spectral<float>(const DevTables<float>&, const float*, NodeParams, int64_t, const float*,
                                            const float*, const int64_t*, float, Cplx<float>*, Cplx<float>*,
                                            const float*, const float*, float*, int*, cudaStream_t);
template cudaError_t launch_spectral<double>(const DevTables<double>&, const double*, NodeParams, int64_t,
                                             const double*, const double*, const int64_t*, double, Cplx<double>*,
                                             Cplx<double>*, const double*, const double*, double*, int*,
                                             cudaStream_t);

}  // namespace dgfs
