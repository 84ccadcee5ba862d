// Device helpers shared by the Fourier-side kernels (arXiv:1809.10186, Appendix): the VHS
// radial factor, the loss multiplier and the radix-2 FFT of one line held in registers.
#pragma once

#include <cmath>
#include <cstdint>

#include "launchers.h"

namespace dgfs {
namespace fdev {

constexpr double kPi = 3.14159265358979323846;

template <typename T>
__device__ __forceinline__ T radial_rho(double b, double gamma, double cr, int dlog) {
    // rho_r = 4 pi b c_r^{gamma+2}: the closed form of F(k, c_r) / sinc for VHS (eq. realGG)
    double v = 4.0 * kPi * b * pow(cr, gamma + 2.0);
    if (dlog) v *= log(cr);
    return (T)v;
}

// Loss multiplier at index k of one node. The radial sum of oscillating sinc terms cancels
// strongly at large |k|, so it is taken from the FP64-built table or accumulated in FP64.
template <typename T>
__device__ __forceinline__ T loss_multiplier(const T* __restrict__ GL0, const T* __restrict__ GLd,
                                             const T* __restrict__ Lr, const double* __restrict__ rho,
                                             bool per_node, int dlog, int Nrho, int64_t n3, int64_t k) {
    if (!per_node) return dlog ? GLd[k] : GL0[k];
    double g = 0.0;
    for (int r = 0; r < Nrho; ++r) g = fma(rho[r], (double)Lr[r * n3 + k], g);
    return (T)g;
}

// ---- radix-2 FFT passes (power-of-two N) -------------------------------------------------
//
// One thread transforms one line of N complex values held in registers: decimation in time
// on bit-reversed input, N/2 log2 N butterflies, twiddles e^{-+2 pi i j / N} taken from the
// plan's DFT table (row 1) through shared memory. Same result as the dense passes, in
// 5 N log2 N instead of 8 N^2 flops per line.

template <int N>
__device__ __forceinline__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1, k = N >> 1; b < N; b <<= 1, k >>= 1)
        if (i & b) r |= k;
    return r;
}

// One radix-2 stage of butterfly span LEN, then the next stage. LEN is a template parameter so
// that every loop has a compile-time trip count and the line stays in registers; the twiddles
// 1 and -+i (known once the loops are unrolled) take no multiplication.
template <typename T, int N, int LEN>
__device__ __forceinline__ void fft_stage(Cplx<T> (&a)[N], const Cplx<T>* __restrict__ tw, bool forward) {
    constexpr int half = LEN / 2, step = N / LEN;
#pragma unroll
    for (int i = 0; i < N; i += LEN)
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const Cplx<T> u = a[i + j], v0 = a[i + j + half];
            Cplx<T> v;
            if (j == 0) {                      // twiddle 1
                v = v0;
            } else if (4 * j * step == N) {    // twiddle -i (forward) or +i (inverse)
                v = forward ? Cplx<T>{v0.y, -v0.x} : Cplx<T>{-v0.y, v0.x};
            } else {
                const Cplx<T> w = tw[j * step];
                const T wi = forward ? w.y : -w.y;
                v = Cplx<T>{v0.x * w.x - v0.y * wi, v0.x * wi + v0.y * w.x};
            }
            a[i + j] = Cplx<T>{u.x + v.x, u.y + v.y};
            a[i + j + half] = Cplx<T>{u.x - v.x, u.y - v.y};
        }
    if constexpr (LEN < N) fft_stage<T, N, 2 * LEN>(a, tw, forward);
}

// In-place butterflies; the caller loads element k of the line into a[bitrev(k)].
template <typename T, int N>
__device__ __forceinline__ void fft_line(Cplx<T> (&a)[N], const Cplx<T>* __restrict__ tw, bool forward) {
    fft_stage<T, N, 2>(a, tw, forward);
}

// ---- N = 3 * 2^m (12, 24): one radix-3 stage over three radix-2 transforms of length N/3 ------
//
// Decimation in time by 3: x[3m + j] (j = 0, 1, 2) are transformed with length S = N/3 and
// X[k] = Y_0[k mod S] + w^k Y_1[k mod S] + w^2k Y_2[k mod S], w = e^{-+2 pi i / N}. Element k of a
// line is loaded into slot line_slot<N>(k): bit-reversed for a power of two, block j = k mod 3 and
// the bit-reversed position of k / 3 inside it otherwise. line_fft leaves the result in natural
// order in both cases; tw is row 1 of the N-point DFT table.

template <int N>
__device__ __forceinline__ constexpr int line_slot(int k) {
    if constexpr ((N & (N - 1)) == 0) return bitrev<N>(k);
    else return (k % 3) * (N / 3) + bitrev<N / 3>(k / 3);
}

// radix-2 stages of a length-S transform held in a[OFF .. OFF + S); its twiddle w_S^q is
// tw[q N / S] of the N-row
template <typename T, int NA, int OFF, int S, int LEN>
__device__ __forceinline__ void fft_stage_sub(Cplx<T> (&a)[NA], const Cplx<T>* __restrict__ tw, bool forward) {
    constexpr int half = LEN / 2, step = S / LEN, tstride = NA / S;
#pragma unroll
    for (int i = 0; i < S; i += LEN)
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const Cplx<T> u = a[OFF + i + j], v0 = a[OFF + i + j + half];
            Cplx<T> v;
            if (j == 0) {
                v = v0;
            } else if (4 * j * step == S) {
                v = forward ? Cplx<T>{v0.y, -v0.x} : Cplx<T>{-v0.y, v0.x};
            } else {
                const Cplx<T> w = tw[j * step * tstride];
                const T wi = forward ? w.y : -w.y;
                v = Cplx<T>{v0.x * w.x - v0.y * wi, v0.x * wi + v0.y * w.x};
            }
            a[OFF + i + j] = Cplx<T>{u.x + v.x, u.y + v.y};
            a[OFF + i + j + half] = Cplx<T>{u.x - v.x, u.y - v.y};
        }
    if constexpr (LEN < S) fft_stage_sub<T, NA, OFF, S, 2 * LEN>(a, tw, forward);
}

template <typename T, int N>
__device__ __forceinline__ void line_fft(Cplx<T> (&a)[N], const Cplx<T>* __restrict__ tw, bool forward) {
    if constexpr ((N & (N - 1)) == 0) {
        fft_stage<T, N, 2>(a, tw, forward);
    } else {
        static_assert(N % 3 == 0 && ((N / 3) & (N / 3 - 1)) == 0, "N must be a power of two or 3 times one");
        constexpr int S = N / 3;
        fft_stage_sub<T, N, 0, S, 2>(a, tw, forward);
        fft_stage_sub<T, N, S, S, 2>(a, tw, forward);
        fft_stage_sub<T, N, 2 * S, S, 2>(a, tw, forward);
        Cplx<T> b[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int q = k % S;
            const Cplx<T> y0 = a[q], y1 = a[S + q], y2 = a[2 * S + q];
            const Cplx<T> w1 = tw[k], w2 = tw[(2 * k) % N];
            const T s1 = forward ? w1.y : -w1.y, s2 = forward ? w2.y : -w2.y;
            b[k] = Cplx<T>{y0.x + (y1.x * w1.x - y1.y * s1) + (y2.x * w2.x - y2.y * s2),
                           y0.y + (y1.x * s1 + y1.y * w1.x) + (y2.x * s2 + y2.y * w2.x)};
        }
#pragma unroll
        for (int k = 0; k < N; ++k) a[k] = b[k];
    }
}

}  // namespace fdev
}  // namespace dgfs
