// Fused Fourier stage for power-of-two grids (N = 8, 16, 32): the same arithmetic as the
// projection, forward DFT, Fourier combine, inverse DFT and finalisation kernels of
// k_fourier.cu (arXiv:1809.10186, Appendix, eqs. realGG, lowrank1, apndx_fs_Glm_Qk), in four
// launches whose intermediates stay in shared memory or registers between the axis passes:
//
//   k_spec_coef  the projection coefficients C[s][r] = V[s][r] w_r rho_r (once per launch, or per
//                node when gamma or b vary by node)
//   k_spec_xz    one (x, z) plane y = const of a node: X_s = sum_r C[s][r] P_r for every s, the loss
//                operand(s), packed two real fields per complex slot; forward FFT along x and z
//   k_spec_y     the planes kx and -kx of every slot: forward FFT along y (each thread one line,
//                loaded straight into registers), the spectra of the packed fields separated with
//                the mirror point -k (in the other plane), gain^ = sum_s Uk[s] X^_s (the factors
//                staged in shared memory by |k|^2) and loss^ = GL(k) g^; inverse FFT along y and z
//   k_spec_xout  inverse FFT along x (each thread one line per field, in registers) and
//                Q = gain - f (K_L g)
//
// Per node this moves P (Nrho N^3), the packed slots twice and the two or three result fields
// twice through HBM. The forward transforms are unnormalised and the unpacking of the two real
// fields of a slot skips its factor 1/2: both powers of two are applied once, in the combine.
// Twiddles are compile-time constants (cos 2 pi m / 32), so the FFT lines load nothing but data.
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
    static constexpr int RB = N == 32 ? 5 : 8;                  // radial points of P in flight per thread
    static constexpr int T2 = 256;                             // k_spec_y
    static constexpr int YP = N * N <= 256 ? N : 256 / N;      // k_spec_xout: planes y per CTA
    static_assert(V == 1 || V == 4, "points per thread");
};

// ---- constant twiddles ------------------------------------------------------------------
// cos(2 pi m / 32) for m = 0 .. 8; the other angles follow from the symmetries of cos.
__host__ __device__ constexpr double cos_q32(int m) {
    return m == 0 ? 1.0
         : m == 1 ? 0.980785280403230449126182236134239037
         : m == 2 ? 0.923879532511286756128183189396788287
         : m == 3 ? 0.831469612302545237078788377617905757
         : m == 4 ? 0.707106781186547524400844362104849039
         : m == 5 ? 0.555570233019602224742830813948532874
         : m == 6 ? 0.382683432365089771728459984030398867
         : m == 7 ? 0.195090322016128267848284868477022241
         : 0.0;
}
__host__ __device__ constexpr double cos32(int m) {   // cos(2 pi m / 32), any integer m
    m = ((m % 32) + 32) % 32;
    return m <= 8 ? cos_q32(m) : m <= 16 ? -cos_q32(16 - m) : m <= 24 ? -cos_q32(m - 16) : cos_q32(32 - m);
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }   // sin x = cos(x - pi / 2)

// One radix-2 stage of span LEN (then the next): decimation in time on bit-reversed input, the
// twiddle of butterfly j is e^{-+2 pi i j / LEN} = e^{-+2 pi i m / 32}, m = 32 j / LEN, known at
// compile time once the loops are unrolled; 1 and -+i take no multiplication.
template <typename T, int N, int LEN, bool FWD>
__device__ __forceinline__ void fftc_stage(Cplx<T> (&a)[N]) {
    constexpr int half = LEN / 2;
#pragma unroll
    for (int i = 0; i < N; i += LEN)
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const Cplx<T> u = a[i + j], v0 = a[i + j + half];
            const int m = j * (32 / LEN);
            Cplx<T> v;
            if (j == 0) {
                v = v0;
            } else if (4 * j == LEN) {
                v = FWD ? Cplx<T>{v0.y, -v0.x} : Cplx<T>{-v0.y, v0.x};
            } else {
                const T wr = (T)cos32(m), wi = FWD ? (T)(-sin32(m)) : (T)sin32(m);
                v = Cplx<T>{v0.x * wr - v0.y * wi, v0.x * wi + v0.y * wr};
            }
            a[i + j] = Cplx<T>{u.x + v.x, u.y + v.y};
            a[i + j + half] = Cplx<T>{u.x - v.x, u.y - v.y};
        }
    if constexpr (LEN < N) fftc_stage<T, N, 2 * LEN, FWD>(a);
}

// Unnormalised DFT of one line in registers (element k loaded into a[bitrev(k)]), natural order out.
template <typename T, int N, bool FWD>
__device__ __forceinline__ void fftc(Cplx<T> (&a)[N]) {
    static_assert(N <= 32 && (N & (N - 1)) == 0, "power-of-two lines up to 32");
    fftc_stage<T, N, 2, FWD>(a);
}

// 8- or 16-byte accesses of one complex value (Cplx<T> itself is only T-aligned)
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T>
__device__ __forceinline__ Cplx<T> ldc(const Cplx<T>* p) {
    const typename Vec2<T>::type v = *reinterpret_cast<const typename Vec2<T>::type*>(p);
    return Cplx<T>{v.x, v.y};
}
template <typename T>
__device__ __forceinline__ Cplx<T> ldgc(const Cplx<T>* p) {
    const typename Vec2<T>::type v = __ldg(reinterpret_cast<const typename Vec2<T>::type*>(p));
    return Cplx<T>{v.x, v.y};
}
template <typename T>
__device__ __forceinline__ void stc(Cplx<T>* p, Cplx<T> c) {
    typename Vec2<T>::type v;
    v.x = c.x;
    v.y = c.y;
    *reinterpret_cast<typename Vec2<T>::type*>(p) = v;
}

// One line of N complex values in shared memory (element k at base[k * stride]) transformed in place.
template <typename T, int N, bool FWD>
__device__ __forceinline__ void fftc_smem_line(Cplx<T>* base, int stride) {
    Cplx<T> a[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a[bitrev<N>(k)] = ldc(base + k * stride);
    fftc<T, N, FWD>(a);
#pragma unroll
    for (int k = 0; k < N; ++k) stc(base + k * stride, a[k]);
}

// signed lattice index of DFT position q
template <int N>
__device__ __forceinline__ int signed_q(int q) { return q < N / 2 ? q : q - N; }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
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

// two FP32 FMAs in one instruction (each rounded as fmaf): d = a * b + c, elementwise
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
          "l"(*reinterpret_cast<unsigned long long*>(&c)));
    return *reinterpret_cast<float2*>(&d);
}

// ---- kernel 0: projection coefficients ---------------------------------------------------
// C[node][r][s] = Vr[s][r] (w_r rho_r(node)): one block per node (or one for the whole launch).
template <typename T>
__global__ void k_spec_coef(const T* __restrict__ Vr, const double* __restrict__ cr, const double* __restrict__ wr,
                            NodeParams np, int Nrho, int rank, T* __restrict__ C) {
    __shared__ T wrho[64];
    const int64_t node = blockIdx.x;
    const double gam = np.gamma ? np.gamma[node] : np.gamma0;
    const double bb = np.b ? np.b[node] : np.b0;
    for (int r = threadIdx.x; r < Nrho; r += blockDim.x) wrho[r] = (T)wr[r] * radial_rho<T>(bb, gam, cr[r], np.dlog);
    __syncthreads();
    T* Cn = C + node * Nrho * rank;
    for (int e = threadIdx.x; e < Nrho * rank; e += blockDim.x) {
        const int r = e / rank, s = e % rank;
        Cn[e] = Vr[s * Nrho + r] * wrho[r];
    }
}

// ---- kernel 1: projection + loss operands + forward FFT along x and z of one plane y -------
// CTA (slot group g, plane y) of a node: slots [g slg, g slg + ns) of the packed fields (every slot
// in one group when they fit, so that the plane of P, Nrho N^2 values, is read once).
template <typename T, int N, int SL>
__global__ void __launch_bounds__(SpecGeo<N>::T1, N == 32 ? 2 : 1)
k_spec_xz(const T* __restrict__ P, const T* __restrict__ Cg, int64_t c_stride, int Nrho, int rank,
          const T* __restrict__ la, const T* __restrict__ lb, const int64_t* __restrict__ offs, int nloss,
          Cplx<T>* __restrict__ X, int xs, int groups, int slg) {
    using G = SpecGeo<N>;
    constexpr int FG = 2 * SL;                                  // fields of one slot group (at most)
    constexpr bool PAIRS = sizeof(T) == 4 && G::V == 4;         // two points per FP32 FMA instruction
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Cplx<T>* F = reinterpret_cast<Cplx<T>*>(sm_raw);           // [SL][PLANE]
    T* C = reinterpret_cast<T*>(F + SL * G::PLANE);             // [Nrho][FG] (pairs {c, c}: [Nrho][FG][2])
    T* ring = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(C + Nrho * FG * (PAIRS ? 2 : 1)) + 15) &
                                   ~uintptr_t(15));             // [RB][T1 V]: asynchronous copies of P
    const int g = blockIdx.x % groups, y = blockIdx.x / groups, t = threadIdx.x;
    const int s0 = g * slg, ns = xs - s0 < slg ? xs - s0 : slg, f0 = 2 * s0;
    const int64_t node = blockIdx.y, n3 = (int64_t)N * G::N2;
    const T* Cn = Cg + node * c_stride;
    for (int e = t; e < Nrho * FG; e += G::T1) {
        const int r = e / FG, fi = f0 + e % FG;
        const T c = fi < rank && e % FG < 2 * ns ? Cn[r * rank + fi] : T(0);
        if constexpr (PAIRS) {
            C[2 * e] = c;
            C[2 * e + 1] = c;
        } else {
            C[e] = c;
        }
    }
    __syncthreads();
    // this thread's points: (x, z0 .. z0 + V - 1) of plane y
    const int x = t / (N / G::V), z0 = (t % (N / G::V)) * G::V;
    const int64_t j0 = ((int64_t)x * N + y) * N + z0;
    if (f0 < rank) {
        // each thread streams its own V values of P_r through a ring of RB asynchronous copies
        // (one commit group per r), so RB radial points are in flight without holding registers
        const T* Pn = P + node * Nrho * n3 + j0;
        T* mine = ring + t * G::V;
        auto issue = [&](int r, int slot) {
            if (r < Nrho) cp_async_v<T, G::V>(mine + slot * (G::T1 * G::V), Pn + (int64_t)r * n3);
            cp_async_commit();
        };
#pragma unroll
        for (int r = 0; r < G::RB; ++r) issue(r, r);
        if constexpr (PAIRS) {
            float2 acc[2][FG];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < FG; ++i) acc[h][i] = make_float2(0.f, 0.f);
            int slot = 0;
#pragma unroll 1
            for (int r = 0; r < Nrho; ++r) {
                cp_async_wait_group<G::RB - 1>();   // the copy of P_r has landed
                const float4 p = *reinterpret_cast<const float4*>(mine + slot * (G::T1 * G::V));
                const float2 p01 = make_float2(p.x, p.y), p23 = make_float2(p.z, p.w);
                const float4* c4 = reinterpret_cast<const float4*>(C + 2 * r * FG);
#pragma unroll
                for (int i = 0; i < FG; i += 2) {
                    const float4 cc = c4[i / 2];    // {c_i, c_i, c_i+1, c_i+1}
                    const float2 ci = make_float2(cc.x, cc.y), cj = make_float2(cc.z, cc.w);
                    acc[0][i] = fma2(ci, p01, acc[0][i]);
                    acc[1][i] = fma2(ci, p23, acc[1][i]);
                    acc[0][i + 1] = fma2(cj, p01, acc[0][i + 1]);
                    acc[1][i + 1] = fma2(cj, p23, acc[1][i + 1]);
                }
                issue(r + G::RB, slot);   // after the FMAs that consumed the slot's values
                slot = slot + 1 == G::RB ? 0 : slot + 1;
            }
            cp_async_wait_all();
#pragma unroll
            for (int i = 0; i < FG; i += 2)
                if (i / 2 < ns) {
                    Cplx<T>* d = F + (i / 2) * G::PLANE + x * G::ROW + z0;
                    stc(d + 0, Cplx<T>{acc[0][i].x, acc[0][i + 1].x});
                    stc(d + 1, Cplx<T>{acc[0][i].y, acc[0][i + 1].y});
                    stc(d + 2, Cplx<T>{acc[1][i].x, acc[1][i + 1].x});
                    stc(d + 3, Cplx<T>{acc[1][i].y, acc[1][i + 1].y});
                }
        } else {
            T acc[G::V][FG];
#pragma unroll
            for (int v = 0; v < G::V; ++v)
#pragma unroll
                for (int i = 0; i < FG; ++i) acc[v][i] = T(0);
            int slot = 0;
#pragma unroll 1
            for (int r = 0; r < Nrho; ++r) {
                cp_async_wait_group<G::RB - 1>();
                T p[G::V];
#pragma unroll
                for (int v = 0; v < G::V; ++v) p[v] = mine[slot * (G::T1 * G::V) + v];
                const T* c = C + r * FG;
#pragma unroll
                for (int i = 0; i < FG; ++i)
#pragma unroll
                    for (int v = 0; v < G::V; ++v) acc[v][i] = fma(c[i], p[v], acc[v][i]);
                issue(r + G::RB, slot);
                slot = slot + 1 == G::RB ? 0 : slot + 1;
            }
            cp_async_wait_all();
#pragma unroll
            for (int i = 0; i < FG; i += 2)
                if (i / 2 < ns)
#pragma unroll
                    for (int v = 0; v < G::V; ++v)
                        stc(F + (i / 2) * G::PLANE + x * G::ROW + z0 + v, Cplx<T>{acc[v][i], acc[v][i + 1]});
        }
    }
    // loss operand(s): fields rank, rank + 1 (the imaginary part of a slot past the last field is 0)
    const int64_t base = offs ? offs[node] : node * n3;
    for (int jl = 0; jl < nloss; ++jl) {
        const int fi = rank + jl - f0;
        if (fi < 0 || fi >= 2 * ns) continue;
        const T* src = (jl ? lb : la) + base + j0;
#pragma unroll
        for (int v = 0; v < G::V; ++v) {
            T* d = reinterpret_cast<T*>(F + (fi / 2) * G::PLANE + x * G::ROW + z0 + v);
            const T val = src[v];
            if (fi % 2 == 0) {
                d[0] = val;
                d[1] = T(0);
            } else {
                d[1] = val;
            }
        }
    }
    __syncthreads();
    for (int id = t; id < ns * N; id += G::T1) {   // along x: line (slot, z)
        const int m = id / N, z = id % N;
        fftc_smem_line<T, N, true>(F + m * G::PLANE + z, G::ROW);
    }
    __syncthreads();
    for (int id = t; id < ns * N; id += G::T1) {   // along z: line (slot, kx)
        const int m = id / N, kx = id % N;
        fftc_smem_line<T, N, true>(F + m * G::PLANE + kx * G::ROW, 1);
    }
    __syncthreads();
    Cplx<T>* Xn = X + (node * (int64_t)xs + s0) * n3;
    for (int e = t; e < ns * G::N2; e += G::T1) {   // X[slot][kx][y][kz]
        const int m = e / G::N2, kx = (e / N) % N, kz = e % N;
        stc(Xn + m * n3 + ((int64_t)kx * N + y) * N + kz, ldc(F + m * G::PLANE + kx * G::ROW + kz));
    }
}

// ---- kernel 2: FFT along y, combine, inverse FFT along y and z of the planes kx, -kx ----------
// CTA c of a node, c = 0 .. N/2: planes {c, N - c} for 0 < c < N/2 (mirrors of each other), the
// single planes {0} and {N/2} (each its own mirror) for c = 0 and N/2; both planes of a CTA share
// |kx|^2. A group holds GS = T2 / (npl N) slots; thread t transforms the y line (slot t / (npl N),
// plane (t / N) % npl, column t % N), loaded from X into registers, and the next group's line is in
// flight during the current group's combine. The radial factors of the group's fields are staged
// in shared memory by |ky|^2 + |kz|^2 (U_s depends on |k|^2 only), zero for the fields past the
// rank, so the gain sum runs without branches. The loss field(s) are picked up in a separate pass
// of the group that holds them and parked, times their multiplier, in this CTA's planes of Y until
// the inverse transforms.
template <int N>
constexpr int ilog2() { return N == 8 ? 3 : N == 16 ? 4 : 5; }

// Row stride of k_spec_y's factor table: every field of a slot group, plus one pair of padding (an
// even stride, so that a pair of factors loads as 8 bytes; 18 at N = 32 spreads a warp's rows over
// the banks).
template <int N>
constexpr int spec_y_table_stride() { return 2 * (256 / N) + 2; }

template <typename T, int N, int NL>
__global__ void __launch_bounds__(SpecGeo<N>::T2, 2)
k_spec_y(const Cplx<T>* __restrict__ X, int xs, const T* __restrict__ Uq, int nq2, const T* __restrict__ Lr,
         const T* __restrict__ GL0, const T* __restrict__ GLd, const double* __restrict__ cr, NodeParams np,
         int Nrho, int rank, int lf0, int lf1, T gscale, T lscale, Cplx<T>* __restrict__ Y, int yf) {
    using G = SpecGeo<N>;
    constexpr int LN = ilog2<N>();
    constexpr int GSX = G::T2 / N;                      // slots (planes) of the buffer: a group of one-plane CTAs
    constexpr int PT = (2 * G::N2 + G::T2 - 1) / G::T2; // combine points per thread (two planes)
    constexpr int MR = 2 * (N / 2) * (N / 2) + 1;       // |ky|^2 + |kz|^2 = 0 .. 2 (N/2)^2
    constexpr int US = spec_y_table_stride<N>();        // row of the factor table (even: pairs load as 8 bytes)
    constexpr int MRW = (MR + 31) / 32;                 // table rows per lane
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Cplx<T>* buf = reinterpret_cast<Cplx<T>*>(sm_raw);  // [GSX][PLANE]: slot jm, plane pl at jm npl + pl
    T* Us = reinterpret_cast<T*>(buf + GSX * G::PLANE); // [MR][US]
    double* rho = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(Us + MR * US) + 15) & ~uintptr_t(15));
    const int c = blockIdx.x, t = threadIdx.x;
    const int npl = (c == 0 || c == N / 2) ? 1 : 2, sh = npl - 1;
    const int kx0 = c, kx1 = N - c, GS = G::T2 >> (LN + sh);
    const int kq = signed_q<N>(kx0), kx2 = kq * kq;
    const int64_t node = blockIdx.y, n3 = (int64_t)N * G::N2;
    const bool per_node = np.gamma || np.b;
    if (per_node) {
        const double gam = np.gamma ? np.gamma[node] : np.gamma0;
        const double bb = np.b ? np.b[node] : np.b0;
        for (int r = t; r < Nrho; r += G::T2) rho[r] = radial_rho<double>(bb, gam, cr[r], np.dlog);
    }
    const Cplx<T>* Xn = X + node * (int64_t)xs * n3;
    // this thread's y line
    const int ljm = t >> (LN + sh), lpl = (t >> LN) & sh, lkz = t & (N - 1);
    const int64_t loff = (int64_t)(lpl ? kx1 : kx0) * G::N2 + lkz;   // X[m][kx][y][kz] at y = 0
    const int npts = npl * G::N2;
    // this thread's combine points e = t + i T2: plane e / N^2, (ky, kz); row |ky|^2 + |kz|^2 of the table
    int mrow[PT];
    T gr[PT], gi[PT];
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int e = t + i * G::T2, ky = (e >> LN) & (N - 1), kz = e & (N - 1);
        mrow[i] = signed_q<N>(ky) * signed_q<N>(ky) + signed_q<N>(kz) * signed_q<N>(kz);
        gr[i] = gi[i] = T(0);
    }
    Cplx<T>* Yn = Y + node * (int64_t)yf * n3;
    auto kidx = [&](int e) {   // spectrum index of point e
        const int pl = e >> (2 * LN), ky = (e >> LN) & (N - 1), kz = e & (N - 1);
        return ((int64_t)(pl ? kx1 : kx0) * N + ky) * N + kz;
    };
    // the two spectra a slot packs at point e (times 2): field 2m in fa, field 2m + 1 in fb
    auto unpack = [&](int e, int jm, Cplx<T>& fa, Cplx<T>& fb) {
        const int pl = e >> (2 * LN), ky = (e >> LN) & (N - 1), kz = e & (N - 1);
        const int pm = npl == 2 ? 1 - pl : pl, kym = (N - ky) & (N - 1), kzm = (N - kz) & (N - 1);
        const Cplx<T> z = ldc(buf + (jm * npl + pl) * G::PLANE + ky * G::ROW + kz);
        const Cplx<T> w = ldc(buf + (jm * npl + pm) * G::PLANE + kym * G::ROW + kzm);
        fa = Cplx<T>{z.x + w.x, z.y - w.y};
        fb = Cplx<T>{z.y + w.y, w.x - z.x};
    };
    Cplx<T> a[N];
    auto load_line = [&](int g0) {
        if (g0 + ljm < xs) {
            const Cplx<T>* src = Xn + (int64_t)(g0 + ljm) * n3 + loff;
#pragma unroll
            for (int k = 0; k < N; ++k) a[bitrev<N>(k)] = ldgc(src + k * N);
        }
    };
    // factors of the group's fields [f0, f0 + nf) at |k|^2 = |kx|^2 + row, into table columns
    // [c0, c0 + nf) (zero past the rank): one field per warp, rows along the lanes (coalesced reads of
    // the compact table), every load of a lane in flight before its stores
    auto fill = [&](int f0, int nf, int c0) {
        for (int j = t >> 5; j < nf; j += G::T2 / 32) {
            const int fi = f0 + j, lane = t & 31;
            const T* src = Uq + (int64_t)fi * nq2 + kx2;
            T v[MRW];
#pragma unroll
            for (int r = 0; r < MRW; ++r) v[r] = fi < rank && lane + 32 * r < MR ? __ldg(src + lane + 32 * r) : T(0);
#pragma unroll
            for (int r = 0; r < MRW; ++r)
                if (lane + 32 * r < MR) Us[(lane + 32 * r) * US + c0 + j] = v[r];
        }
    };
    load_line(0);
    for (int g0 = 0; g0 < xs; g0 += GS) {
        const int ng = xs - g0 < GS ? xs - g0 : GS, f0 = 2 * g0, nf = 2 * ng;
        const bool mine = ljm < ng;
        if (mine) fftc<T, N, true>(a);
        __syncthreads();   // the previous group's combine has read buf and the factor table
        if (mine) {
            Cplx<T>* d = buf + (ljm * npl + lpl) * G::PLANE + lkz;
#pragma unroll
            for (int k = 0; k < N; ++k) stc(d + k * G::ROW, a[k]);
        }
        fill(f0, nf, 0);
        __syncthreads();
        if (g0 + GS < xs) load_line(g0 + GS);   // in flight during the combine below
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            const int e = t + i * G::T2;
            if (e >= npts) continue;
            const T* urow = Us + mrow[i] * US;
#pragma unroll
            for (int jm = 0; jm < GSX; ++jm) {
                if (jm >= ng) break;
                Cplx<T> fa, fb;
                unpack(e, jm, fa, fb);
                const typename Vec2<T>::type uu = *reinterpret_cast<const typename Vec2<T>::type*>(urow + 2 * jm);
                const T ua = uu.x, ub = uu.y;
                gr[i] = fma(ua, fa.x, gr[i]);
                gi[i] = fma(ua, fa.y, gi[i]);
                gr[i] = fma(ub, fb.x, gr[i]);
                gi[i] = fma(ub, fb.y, gi[i]);
            }
        }
        // the loss operand(s) of this group, times the loss multiplier, parked in Y (field 1 + jl)
#pragma unroll
        for (int jl = 0; jl < NL; ++jl) {
            const int lf = jl ? lf1 : lf0;
            if (lf < f0 || lf >= f0 + nf) continue;
            const int jm = (lf - f0) >> 1, h = (lf - f0) & 1;
#pragma unroll
            for (int i = 0; i < PT; ++i) {
                const int e = t + i * G::T2;
                if (e >= npts) continue;
                Cplx<T> fa, fb;
                unpack(e, jm, fa, fb);
                const Cplx<T> v = h ? fb : fa;
                const int64_t k = kidx(e);
                const T GL = lscale * loss_multiplier<T>(GL0, GLd, Lr, rho, per_node, np.dlog, Nrho, n3, k);
                stc(Yn + (1 + jl) * n3 + k, Cplx<T>{GL * v.x, GL * v.y});
            }
        }
    }
    __syncthreads();   // every combine has read buf, every parked loss value is written (block scope)
    // the result fields [field][plane] into buf: gain from registers, loss back from Y
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int e = t + i * G::T2;
        if (e >= npts) continue;
        const int pl = e >> (2 * LN), ky = (e >> LN) & (N - 1), kz = e & (N - 1);
        const int64_t k = kidx(e);
        const int o = pl * G::PLANE + ky * G::ROW + kz;
        stc(buf + o, Cplx<T>{gscale * gr[i], gscale * gi[i]});
#pragma unroll
        for (int jl = 0; jl < NL; ++jl) stc(buf + (1 + jl) * npl * G::PLANE + o, ldc(Yn + (1 + jl) * n3 + k));
    }
    __syncthreads();
    for (int id = t; id < yf * npl * N; id += G::T2) {   // inverse along y: line (field, plane, kz)
        const int fp = id >> LN, kz = id & (N - 1);     // fp = field npl + plane
        fftc_smem_line<T, N, false>(buf + fp * G::PLANE + kz, G::ROW);
    }
    __syncthreads();
    for (int id = t; id < yf * npl * N; id += G::T2) {   // inverse along z: line (field, plane, y)
        const int fp = id >> LN, yy = id & (N - 1);
        fftc_smem_line<T, N, false>(buf + fp * G::PLANE + yy * G::ROW, 1);
    }
    __syncthreads();
    for (int e = t; e < yf * npl * G::N2; e += G::T2) {   // Y[field][kx][y][z]
        const int fp = e >> (2 * LN), fo = fp >> sh, pl = fp & sh, yy = (e >> LN) & (N - 1), z = e & (N - 1);
        stc(Yn + fo * n3 + ((int64_t)(pl ? kx1 : kx0) * N + yy) * N + z, ldc(buf + fp * G::PLANE + yy * G::ROW + z));
    }
}

// ---- kernel 3: inverse FFT along x, Q = gain - a (K_L g) [- c (K_L f)] --------------------------
// Thread (y, z) of a CTA of YP planes: each field's x line is loaded straight into registers.
template <typename T, int N>
__global__ void __launch_bounds__(SpecGeo<N>::YP * N)
k_spec_xout(const Cplx<T>* __restrict__ Y, int yf, const T* __restrict__ a, const T* __restrict__ c,
            const int64_t* __restrict__ offs, T* __restrict__ out, int* __restrict__ flags) {
    using G = SpecGeo<N>;
    const int y = blockIdx.x * G::YP + threadIdx.x / N, z = threadIdx.x % N;
    const int64_t node = blockIdx.y, n3 = (int64_t)N * G::N2;
    const Cplx<T>* Yn = Y + node * (int64_t)yf * n3 + (int64_t)y * N + z;   // + field n3 + kx N^2
    Cplx<T> line[N];
    T q[N];
#pragma unroll
    for (int k = 0; k < N; ++k) line[bitrev<N>(k)] = ldgc(Yn + k * G::N2);
    fftc<T, N, false>(line);
#pragma unroll
    for (int k = 0; k < N; ++k) q[k] = line[k].x;
    const int64_t base = (offs ? offs[node] : node * n3) + (int64_t)y * N + z;   // + x N^2
    for (int fo = 1; fo < yf; ++fo) {
        const T* mul = fo == 1 ? a : c;
#pragma unroll
        for (int k = 0; k < N; ++k) line[bitrev<N>(k)] = ldgc(Yn + fo * n3 + k * G::N2);
        fftc<T, N, false>(line);
#pragma unroll
        for (int k = 0; k < N; ++k) q[k] -= mul[base + k * G::N2] * line[k].x;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        bad |= !isfinite(q[k]);
        out[base + k * G::N2] = q[k];
    }
    if (bad) atomicOr(flags, 2);
}

template <typename T, int N, int SL>
cudaError_t launch_xz(const T* P, const T* C, int64_t c_stride, int Nrho, int rank, const T* la, const T* lb,
                      const int64_t* offs, int nloss, Cplx<T>* X, int xs, int groups, int slg, unsigned nn,
                      cudaStream_t s) {
    using G = SpecGeo<N>;
    constexpr bool PAIRS = sizeof(T) == 4 && G::V == 4;
    const size_t sm = sizeof(Cplx<T>) * (size_t)SL * G::PLANE + sizeof(T) * (size_t)Nrho * 2 * SL * (PAIRS ? 2 : 1) +
                      16 + sizeof(T) * (size_t)G::RB * G::T1 * G::V;
    cudaError_t e = cudaFuncSetAttribute(k_spec_xz<T, N, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_spec_xz<T, N, SL><<<dim3(groups * N, nn), G::T1, sm, s>>>(P, C, c_stride, Nrho, rank, la, lb, offs, nloss, X,
                                                                 xs, groups, slg);
    return cudaGetLastError();
}

// Largest slot group of one k_spec_xz CTA: the plane buffer stays within ~85 KB so that two CTAs
// share an SM (N = 32) and the accumulators within the register budget.
template <typename T, int N>
constexpr int max_group_slots() {
    return N == 32 ? 10 : 17;
}

template <typename T, int N>
cudaError_t spectral_n(const DevTables<T>& t, const T* P, NodeParams np, int64_t nodes, const T* la,
                       const T* lb, const int64_t* offs, T gain_scale, const T* C, int64_t c_stride,
                       Cplx<T>* X, Cplx<T>* Y, const T* fa, const T* fc, T* out, int* flags, cudaStream_t s) {
    using G = SpecGeo<N>;
    const int nloss = lb ? 2 : 1, nfields = t.rank + nloss, xs = (nfields + 1) / 2, yf = lb ? 3 : 2;
    const unsigned nn = (unsigned)nodes;
    cudaError_t e;
    {
        constexpr int SLMAX = max_group_slots<T, N>();
        const int groups = (xs + SLMAX - 1) / SLMAX;
        const int slg = (xs + groups - 1) / groups;   // balanced groups
        if (slg <= 4)
            e = launch_xz<T, N, 4>(P, C, c_stride, t.Nrho, t.rank, la, lb, offs, nloss, X, xs, groups, slg, nn, s);
        else if (slg <= 10)
            e = launch_xz<T, N, 10>(P, C, c_stride, t.Nrho, t.rank, la, lb, offs, nloss, X, xs, groups, slg, nn, s);
        else if constexpr (SLMAX > 10)
            e = launch_xz<T, N, SLMAX>(P, C, c_stride, t.Nrho, t.rank, la, lb, offs, nloss, X, xs, groups, slg, nn, s);
        else
            e = cudaErrorNotSupported;
        if (e != cudaSuccess) return e;
    }
    {
        // the forward transforms are unnormalised (1 / N^3) and the unpacked spectra carry a factor 2
        const T post = T(0.5) / (T(N) * T(N) * T(N));
        constexpr int GSX = G::T2 / N, MR = 2 * (N / 2) * (N / 2) + 1, US = spec_y_table_stride<N>();
        const size_t sm = sizeof(Cplx<T>) * (size_t)GSX * G::PLANE + (sizeof(T) * (size_t)MR * US + 15) / 16 * 16 +
                          sizeof(double) * (size_t)t.Nrho;
        auto kern = lb ? k_spec_y<T, N, 2> : k_spec_y<T, N, 1>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        kern<<<dim3(N / 2 + 1, nn), G::T2, sm, s>>>(X, xs, t.Uq, 3 * (N / 2) * (N / 2) + 1, t.Lr, t.GL0, t.GLd, t.cr, np,
                                                t.Nrho, t.rank, t.rank, lb ? t.rank + 1 : -1, gain_scale * post, post,
                                                Y, yf);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_spec_xout<T, N><<<dim3(N / G::YP, nn), G::YP * N, 0, s>>>(Y, yf, fa, fc, offs, out, flags);
    return cudaGetLastError();
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
    // the projection coefficients follow the packed slots in X (whose allocation holds rank + 2
    // fields per node, xs <= rank / 2 + 2 slots of which carry data)
    const bool per_node = np.gamma || np.b;
    T* C = reinterpret_cast<T*>(X + nodes * xs * n3);
    const int64_t c_stride = per_node ? (int64_t)t.Nrho * t.rank : 0;
    for (int64_t n0 = 0; n0 < (per_node ? nodes : 1); n0 += 65535) {
        const int64_t nn = (per_node ? nodes : 1) - n0 < 65535 ? (per_node ? nodes : 1) - n0 : 65535;
        NodeParams np0 = np;
        if (np.gamma) np0.gamma = np.gamma + n0;
        if (np.b) np0.b = np.b + n0;
        k_spec_coef<T><<<(unsigned)nn, 128, 0, s>>>(t.Vr, t.cr, t.wr, np0, t.Nrho, t.rank, C + n0 * c_stride);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
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
        const T* C0 = C + n0 * c_stride;
        NodeParams np0 = np;
        if (np.gamma) np0.gamma = np.gamma + n0;
        if (np.b) np0.b = np.b + n0;
        cudaError_t e = cudaErrorNotSupported;
        if (t.N == 8)
            e = spectral_n<T, 8>(t, P0, np0, nn, la0, lb0, o, gain_scale, C0, c_stride, X0, Y0, fa0, fc0, out0, flags, s);
        else if (t.N == 16)
            e = spectral_n<T, 16>(t, P0, np0, nn, la0, lb0, o, gain_scale, C0, c_stride, X0, Y0, fa0, fc0, out0, flags,
                                  s);
        else if constexpr (sizeof(T) == 4)
            e = spectral_n<T, 32>(t, P0, np0, nn, la0, lb0, o, gain_scale, C0, c_stride, X0, Y0, fa0, fc0, out0, flags,
                                  s);
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
