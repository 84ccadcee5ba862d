// CUDA-core (FP32 / FP64) kernels of the gain's translate-product-accumulate step as dense
// circulant passes. The library's CUDA-core calls take their translates in Fourier space
// (k_vss.cu, a fifth of the arithmetic); these kernels serve the allocation-free call of FP32/FP64
// plans.
//
// For every node and radial Gauss-Legendre point c_r this computes
//   P_r = sum_{pairs p} w_p [ (T_s f)(T_{-s} g) + (T_{-s} f)(T_s g) ],   s = c_r sigma_p / 2,
// the grid form of the inner sums of eq. apndx_fs_Glm_Qk (arXiv:1809.10186, Appendix): by
// eq. lowrank1 the kernel mode splits into cos/sin factors of l and m, and the sum over
// l + m = k of those factors times f^_l g^_m is the Fourier coefficient of a product of two
// translated grid functions. T_s is separable, (T_s f)_j = sum_j' a_s[(j - j') mod N] f_j'
// per axis (a circulant matrix), and T_{-s} = T_s^T.
//
// Work decomposition: one CTA per (chunk of XC output x-planes, radial point r, node).
// Per sphere pair the CTA
//   1. x-pass: Z_+- [x'][y][z] = sum_x A_+-[x'][x] f[x][y][z] for its XC planes (f from L2),
//   2. y-pass + z-pass per row (x', y'): each thread owns one row, keeps it in registers,
//   3. multiplies the two translated rows and accumulates 2 w_p f_+ f_- in registers.
// Only the final P_r rows are written, once.
#pragma once
#include <cstdint>

#include "launchers.h"

namespace dgfs {

namespace simt {

template <int N, typename T> struct Cfg;
// XC output planes per CTA; threads = XC * N (one per row of the y/z passes)
template <> struct Cfg<8, float>   { static constexpr int XC = 8; };
template <> struct Cfg<16, float>  { static constexpr int XC = 16; };
template <> struct Cfg<24, float>  { static constexpr int XC = 8; };
template <> struct Cfg<32, float>  { static constexpr int XC = 8; };
template <> struct Cfg<8, double>  { static constexpr int XC = 8; };
template <> struct Cfg<16, double> { static constexpr int XC = 16; };
template <> struct Cfg<24, double> { static constexpr int XC = 4; };

template <int N, typename T, int NF>
constexpr size_t smem_bytes() {
    constexpr int XC = Cfg<N, T>::XC;
    return sizeof(T) * (size_t)(2 * N * XC + 4 * N * N + NF * 2 * XC * N * N);
}

// y-pass of one row: Y[z] = sum_y Am[y][yp] * Zs[y][z]   (Am[y][y'] = A[y'][y])
template <int N, typename T>
__device__ __forceinline__ void ypass(const T* __restrict__ Zs, const T* __restrict__ Am, int yp,
                                      T (&Y)[N]) {
#pragma unroll
    for (int z = 0; z < N; ++z) Y[z] = T(0);
#pragma unroll 4
    for (int y = 0; y < N; ++y) {
        const T a = Am[y * N + yp];
        const T* zr = Zs + y * N;
#pragma unroll
        for (int z = 0; z < N; ++z) Y[z] = fma(a, zr[z], Y[z]);
    }
}

// z-pass of one row, value for output z': sum_z Zm[z'][z] * Y[z]
template <int N, typename T>
__device__ __forceinline__ T zdot(const T* __restrict__ Zrow, const T (&Y)[N]) {
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int z = 0; z < N; z += 2) {
        s0 = fma(Zrow[z], Y[z], s0);
        s1 = fma(Zrow[z + 1], Y[z + 1], s1);
    }
    return s0 + s1;
}

template <int N, typename T, int NF>
__global__ void __launch_bounds__(Cfg<N, T>::XC * N)
k_gain_products(const T* __restrict__ f, const T* __restrict__ g, const int64_t* __restrict__ offs,
                const T* __restrict__ filt, const T* __restrict__ wsig, int npairs, int Nrho,
                T* __restrict__ P) {
    constexpr int XC = Cfg<N, T>::XC;
    constexpr int NT = XC * N;
    constexpr int N2 = N * N;
    constexpr int ZV = N / XC;          // z values per thread in the x-pass (N^2 / NT)
    constexpr int ZG = N / ZV;          // z groups per y row in the x-pass

    const int x0 = blockIdx.x * XC;
    const int r = blockIdx.y;
    const int64_t node = blockIdx.z;
    const int64_t base = offs ? offs[node] : node * (int64_t)N * N2;
    const T* fb = f + base;
    const T* gb = (NF == 2) ? g + base : fb;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* XM = reinterpret_cast<T*>(smem_raw);   // [2][N][XC]: XM[sg][x][xl] = A_sg[x0+xl][x]
    T* YM = XM + 2 * N * XC;                   // [2][N][N]:  YM[sg][y][y'] = A_sg[y'][y]
    T* ZM = YM + 2 * N2;                       // [2][N][N]:  ZM[sg][z'][z] = A_sg[z'][z]
    T* Zb = ZM + 2 * N2;                       // [NF][2][XC][N][N] x-pass output

    const int tid = threadIdx.x;
    const int xl = tid / N, yp = tid % N;      // row of the y/z passes
    const int py = tid / ZG, pz0 = (tid % ZG) * ZV;   // position group of the x-pass

    T acc[N];
#pragma unroll
    for (int z = 0; z < N; ++z) acc[z] = T(0);

    for (int p = 0; p < npairs; ++p) {
        const T* fl = filt + ((size_t)r * npairs + p) * 3 * N;   // [3][N]: x, y, z filters
        __syncthreads();                       // previous pair done with matrices and Zb
        for (int e = tid; e < N2; e += NT) {
            const int i = e / N, j = e % N;
            const int dij = (i - j + N) % N, dji = (j - i + N) % N;
            // A_+[i][j] = a[(i - j) mod N], A_-[i][j] = a[(j - i) mod N]
            YM[j * N + i] = fl[N + dij];
            YM[N2 + j * N + i] = fl[N + dji];
            ZM[i * N + j] = fl[2 * N + dij];
            ZM[N2 + i * N + j] = fl[2 * N + dji];
        }
        for (int e = tid; e < N * XC; e += NT) {
            const int x = e / XC, l = e % XC, xp = x0 + l;
            XM[x * XC + l] = fl[(xp - x + N) % N];
            XM[N * XC + x * XC + l] = fl[(x - xp + N) % N];
        }
        __syncthreads();

        // 1. x-pass for each input field, both signs
#pragma unroll 1
        for (int fi = 0; fi < NF; ++fi) {
            const T* src = (fi == 0 ? fb : gb) + py * N + pz0;
            T za[2][XC][ZV];
#pragma unroll
            for (int sg = 0; sg < 2; ++sg)
#pragma unroll
                for (int l = 0; l < XC; ++l)
#pragma unroll
                    for (int v = 0; v < ZV; ++v) za[sg][l][v] = T(0);
#pragma unroll 2
            for (int x = 0; x < N; ++x) {
                T val[ZV];
#pragma unroll
                for (int v = 0; v < ZV; ++v) val[v] = __ldg(src + (size_t)x * N2 + v);
#pragma unroll
                for (int sg = 0; sg < 2; ++sg)
#pragma unroll
                    for (int l = 0; l < XC; ++l) {
                        const T a = XM[sg * N * XC + x * XC + l];
#pragma unroll
                        for (int v = 0; v < ZV; ++v) za[sg][l][v] = fma(a, val[v], za[sg][l][v]);
                    }
            }
#pragma unroll
            for (int sg = 0; sg < 2; ++sg)
#pragma unroll
                for (int l = 0; l < XC; ++l)
#pragma unroll
                    for (int v = 0; v < ZV; ++v)
                        Zb[(((fi * 2 + sg) * XC + l) * N + py) * N + pz0 + v] = za[sg][l][v];
        }
        __syncthreads();

        // 2.-3. y- and z-passes of this thread's row, product, accumulation
        const T w = wsig[p];
        const T* Zrow = Zb + (size_t)xl * N2;             // [fi][sg] planes are XC*N2 apart
        constexpr int PL = XC * N2;
        if (NF == 1) {
            T Wp[N], Y[N];
            ypass<N, T>(Zrow, YM, yp, Y);                  // + direction
#pragma unroll
            for (int z = 0; z < N; ++z) Wp[z] = zdot<N, T>(ZM + z * N, Y);
            ypass<N, T>(Zrow + PL, YM + N2, yp, Y);        // - direction
            const T w2 = T(2) * w;
#pragma unroll
            for (int z = 0; z < N; ++z) acc[z] = fma(w2 * Wp[z], zdot<N, T>(ZM + N2 + z * N, Y), acc[z]);
        } else {
            T Wa[N], Y[N];
            // term 0: f_+ * g_- ; term 1: f_- * g_+
#pragma unroll 1
            for (int term = 0; term < 2; ++term) {
                const int sa = term, sb = 1 - term;
                ypass<N, T>(Zrow + sa * PL, YM + sa * N2, yp, Y);
#pragma unroll
                for (int z = 0; z < N; ++z) Wa[z] = zdot<N, T>(ZM + sa * N2 + z * N, Y);
                ypass<N, T>(Zrow + (2 + sb) * PL, YM + sb * N2, yp, Y);
#pragma unroll
                for (int z = 0; z < N; ++z) acc[z] = fma(w * Wa[z], zdot<N, T>(ZM + sb * N2 + z * N, Y), acc[z]);
            }
        }
    }

    T* dst = P + ((size_t)node * Nrho + r) * (size_t)N * N2 + (size_t)(x0 + xl) * N2 + (size_t)yp * N;
#pragma unroll
    for (int z = 0; z < N; ++z) dst[z] = acc[z];
}

template <int N, typename T, int NF>
cudaError_t launch_gp(const DevTables<T>& t, const T* f, const T* g, const int64_t* offs,
                      int64_t nodes, T* P, cudaStream_t s) {
    constexpr int XC = Cfg<N, T>::XC;
    constexpr size_t sm = smem_bytes<N, T, NF>();
    auto kern = k_gain_products<N, T, NF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    for (int64_t n0 = 0; n0 < nodes; n0 += 65535) {
        const int64_t nn = nodes - n0 < 65535 ? nodes - n0 : 65535;
        dim3 grid(N / XC, t.Nrho, (unsigned)nn);
        kern<<<grid, XC * N, sm, s>>>(f + (offs ? 0 : n0 * (int64_t)N * N * N),
                                     g ? g + (offs ? 0 : n0 * (int64_t)N * N * N) : nullptr,
                                     offs ? offs + n0 : nullptr, t.filt, t.wsig, t.npairs, t.Nrho,
                                     P + n0 * (int64_t)t.Nrho * N * N * N);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace simt
}  // namespace dgfs
