// Internal launcher interface between the C ABI (capi.cu) and the kernel files.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace dgfs {

// Device tables of one plan, in the compute type T (float or double).
template <typename T>
struct DevTables {
    int N, Nrho, npairs, rank;
    const T* filt;      // [Nrho][npairs][3][N] circulant filters of +s_rp
    const T* wsig;      // [npairs]
    const double* cr;   // [Nrho]
    const double* wr;   // [Nrho]
    const T* Uk;        // [rank][N^3]  DFT index order
    const T* Uq;        // [rank][3 (N/2)^2 + 1]: Uk[s](k) = Uq[s][|k|^2] (signed lattice index)
    const T* Vr;        // [rank][Nrho]
    const T* Lr;        // [Nrho][N^3]  DFT index order
    const T* GL0;       // [N^3] sum_r rho_r(gamma, b) Lr[r]: loss multiplier of the plan's kernel
    const T* GLd;       // [N^3] sum_r ln(c_r) rho_r Lr[r]: its derivative with respect to gamma
    const T* dftw;      // [N][N] complex (re, im interleaved): e^{-2 pi i q j / N}
};

// Per-call node parameters: rho_r = 4 pi b_i c_r^{gamma_i + 2} (times ln c_r if dlog).
struct NodeParams {
    const double* gamma;   // [nodes] device, or nullptr -> gamma0
    const double* b;       // [nodes] device, or nullptr -> b0
    double gamma0, b0;
    int dlog;              // 1: derivative with respect to gamma
};

// ---- translate/product kernels (CUDA cores) ------------------------------------------
// P[node][r][N^3] = sum_pairs w_p [(T_s f)(T_-s g) + (T_-s f)(T_s g)] for every radial node.
// g == nullptr means g = f. offs: element offset of every node (nullptr: node * N^3).
cudaError_t launch_gain_products(const DevTables<float>& t, const float* f, const float* g,
                                 const int64_t* offs, int64_t nodes, float* P, cudaStream_t s);
cudaError_t launch_gain_products(const DevTables<double>& t, const double* f, const double* g,
                                 const int64_t* offs, int64_t nodes, double* P, cudaStream_t s);

// ---- Fourier-side kernels -------------------------------------------------------------
template <typename T>
struct Cplx { T x, y; };

// Packed real fields: field i of a node lives in the real (i even) or imaginary (i odd) part of
// complex slot i / 2, so one complex transform carries two real fields.
// Projected field s (s < rank) = sum_r Vr[s][r] w_r rho_r(node) P[node][r], packed into
// X[node][xslots]; with odd rank the imaginary part of the last slot is left zero.
template <typename T>
cudaError_t launch_project(const DevTables<T>& t, const T* P, NodeParams np, int64_t nodes,
                           Cplx<T>* X, int xslots, cudaStream_t s);

// Field a (offs as above) or the product a*b into X[node][slot]: part 0 writes {v, 0}, part 1
// writes only the imaginary part (the real part keeps the field written there before).
template <typename T>
cudaError_t launch_load_field(int N, const T* a, const T* b, const int64_t* offs, int64_t nodes,
                              Cplx<T>* X, int xfields, int slot, int part, cudaStream_t s);

// In-place 3-D DFT of `count` complex fields of N^3 (forward: scale 1/N^3, sign -1).
template <typename T>
cudaError_t launch_dft3(const DevTables<T>& t, Cplx<T>* X, int64_t count, bool forward,
                        cudaStream_t s);

// X holds the forward DFTs of packed real fields (see launch_project); field i's spectrum is
// recovered from slot m = i / 2 as (Z_k + conj Z_-k) / 2 (i even) or (Z_k - conj Z_-k) / 2i.
// Y[node][0] = scale * sum_s Uk[s] Xhat_s;  Y[node][1] = GL Xhat_{loss_field0};
// if loss_field1 >= 0: Y[node][2] = GL Xhat_{loss_field1}. GL = sum_r rho_r(node) Lr[r]: the
// plan's FP64-built table when no per-node parameters are given, else summed in FP64 (the
// radial sum cancels strongly at large |k|, so it is never accumulated in FP32).
template <typename T>
cudaError_t launch_combine(const DevTables<T>& t, const Cplx<T>* X, int xslots, NodeParams np,
                           int64_t nodes, T scale, int loss_field0, int loss_field1, Cplx<T>* Y,
                           int yfields, cudaStream_t s);

// U[node][r] = w_r rho_r(node) sum_s Vr[s][r] Re X[node][s]   (after an inverse DFT)
template <typename T>
cudaError_t launch_expand_radial(const DevTables<T>& t, const Cplx<T>* X, int xfields,
                                 NodeParams np, int64_t nodes, T* U, cudaStream_t s);

// X[node][s] = Uk[s] * X[node][src_slot] for s < rank (Fourier multiply, complex)
template <typename T>
cudaError_t launch_multiply_uk(const DevTables<T>& t, Cplx<T>* X, int xfields, int src_slot,
                               int64_t nodes, cudaStream_t s);

// Y[node][0] = GL X[node][slot0];  Y[node][1] = GL X[node][slot1]
template <typename T>
cudaError_t launch_loss_pair(const DevTables<T>& t, const Cplx<T>* X, int xfields, NodeParams np,
                             int64_t nodes, int slot0, int slot1, Cplx<T>* Y, int yfields,
                             cudaStream_t s);

// out = Re Y0 - a * Re Y1 - (c ? c * Re Y2 : 0)       (mode 0)
// out = sum_r G[node][r] - a * Re Y0 - Re Y1            (mode 1, VJP; a = u)
template <typename T>
cudaError_t launch_finalize(int N, int Nrho, const Cplx<T>* Y, int yfields, const T* a,
                            const T* c, const T* G, const int64_t* offs, int64_t nodes, int mode,
                            T* out, int* flags, cudaStream_t s);

// ---- VSS kernel gain and Fourier-space translates (k_vss.cu) ------------------------------
// Every field plane-major [kz][kx][ky]. Translate spectra of sphere point p (mu_r: [npairs][3][N]
// complex per-axis multipliers of +s_rp): set 0 = mu_s Fh + i conj(mu_s) Gh, set 1 (f != g) =
// conj(mu_s) Fh + i mu_s Gh; Gh == nullptr means Gh = Fh.
// Y[n][0] += scale sum_p A_r[p] P^_p, P^_p separated from the packed spectra W by Hermitian symmetry
template <typename T>
cudaError_t launch_vss_accumulate(const Cplx<T>* W, const T* A_r, int N, int npairs, int64_t nodes, T scale,
                                  Cplx<T>* Y, int yfields, cudaStream_t s);
// Y[n][0] = 0, Y[n][1] = GL Bh[n], Y[n][2] = GL Ah[n] (yfields == 3)
template <typename T>
cudaError_t launch_vss_loss_init(const Cplx<T>* Ah, const Cplx<T>* Bh, const T* GL, int N, int64_t nodes,
                                 Cplx<T>* Y, int yfields, cudaStream_t s);

// the VSS kernels: N = 8, 12, 16, 24 and, in FP32, 32; the VHS translates, the adjoint: every N
bool vss_fused_supported(int N, bool fp64);
bool fft_translate_supported(int N);
// X[n] = {f[n], 0} transposed to plane-major (then transformed with launch_dft3); node n of f at
// offs[n] (device, or nullptr: n N^3)
template <typename T>
cudaError_t launch_vss_load_t(const T* f, const int64_t* offs, int N, int64_t nodes, Cplx<T>* X, cudaStream_t s);
// Z[n][set][p] = inverse x, y transforms of the translate spectra
template <typename T>
cudaError_t launch_vss_inverse_planes(const Cplx<T>* Fh, const Cplx<T>* Gh, const Cplx<T>* mu_r, const Cplx<T>* dftw,
                                      int N, int npairs, int sets, int64_t nodes, Cplx<T>* Z, cudaStream_t s);
// W[n][j] = forward z transform of P_2j + i P_2j+1 after the inverse z transform of the Z lines
template <typename T>
cudaError_t launch_vss_lines(const Cplx<T>* Z, const Cplx<T>* dftw, int N, int npairs, int sets, int64_t nodes,
                             Cplx<T>* W, cudaStream_t s);
// forward y, x transforms of W[n][0 .. fields) in place
template <typename T>
cudaError_t launch_vss_forward_planes(const Cplx<T>* dftw, int N, int fields, int64_t nodes, Cplx<T>* W,
                                      cudaStream_t s);
// VHS: P[n][r] (standard layout, node stride node_stride) = sum_p w_p (products of the translate lines of Z)
template <typename T>
cudaError_t launch_vss_lines_sum(const Cplx<T>* Z, const Cplx<T>* dftw, const T* wsig, int N, int npairs, int sets,
                                 int64_t nodes, int64_t node_stride, T* P, cudaStream_t s);
// adjoint gain in Fourier space (see k_vss.cu): W[n][p] = DFT_z(U_r b + i U_r a) of the translate lines,
// G^[n] += sum_p 2 w_p [conj(mu_s) P1^ + mu_s P2^], and the real part of the transformed-back G^ in the
// standard layout
template <typename T>
cudaError_t launch_vjp_lines(const Cplx<T>* Z, const T* U, int64_t node_stride, const Cplx<T>* dftw, int N,
                             int npairs, int64_t nodes, Cplx<T>* W, cudaStream_t s);
template <typename T>
cudaError_t launch_vjp_accumulate(const Cplx<T>* W, const Cplx<T>* mu_r, const T* wsig, int N, int npairs,
                                  int64_t nodes, Cplx<T>* Gh, cudaStream_t s);
template <typename T>
cudaError_t launch_vjp_real_t(const Cplx<T>* Gt, int N, int64_t nodes, T* out, cudaStream_t s);
// out (standard layout) = Re Y0 - a Re Y1 - (c ? c Re Y2 : 0), Y plane-major
template <typename T>
cudaError_t launch_vss_finalize_t(const Cplx<T>* Y, int yfields, const T* a, const T* c, int N, int64_t nodes, T* out,
                                  int* flags, cudaStream_t s);

// ---- DG element collision, SVD variant (k_dg.cu) ---------------------------------------
// f[e][r] = sum_l A[r][l] F[e][l], g[e][r] = sum_l B[r][l] F[e][l]   (F [E][K][n3], K <= 16; B == nullptr:
// f only)
template <typename T>
cudaError_t launch_dg_combine(const T* F, const T* A, const T* B, int K, int R, int64_t n3, int64_t E, T* f, T* g,
                              cudaStream_t s);
// C[e][m] = sum_{r = rs[m]}^{rs[m+1]-1} sgn[r] Q[e][r]   (rs: device [K + 1]; sgn: device [R] or nullptr)
template <typename T>
cudaError_t launch_dg_accumulate(const T* Q, const int* rs, const T* sgn, int K, int R, int64_t n3, int64_t E, T* C,
                                 cudaStream_t s);

// ---- 1-D DGFS transport (k_slab.cu) ------------------------------------------------------
struct SlabMatrices {
    int K;                 // nodes per element, 2..8
    double S[64];          // [K][K] stiffness S[m][l] = int phi_l phi_m' (reference element)
    double Minv[64];       // [K][K] inverse reference mass matrix
    double den[2];         // wall denominators: sum over incoming c of |c_1| f_w (left, right)
};
// num[0], num[1] = sum over outgoing c of |c_1| f at the left / right wall node (FP64)
template <typename T>
cudaError_t launch_slab_wall(const T* F, int N, int I, int K, double L, double* num, cudaStream_t s);
// out = (2/h_i) M^{-1} (c_1 S F - Fl) + invKn M^{-1} C (C may be nullptr); fw [2][N^3] wall Maxwellians
template <typename T>
cudaError_t launch_slab_rhs(const T* F, const T* C, const T* fw, const double* num, const SlabMatrices& mats,
                            const double* hinv2, double invKn, int N, int I, double L, T* out, cudaStream_t s);

// ---- time stepping and moments (k_time.cu) --------------------------------------------
// out = a u + b v + c q over n values (v may be nullptr); non-finite results raise flag bit 1
template <typename T>
cudaError_t launch_rk_combine(int64_t n, double a, const T* u, double b, const T* v, double c, const T* q, T* out,
                              int* flags, cudaStream_t s);
// out [B][15] (FP64): n, u[3], T, P[xx, yy, zz, xy, xz, yz], q[3], H = int f ln f (f > 0)
template <typename T>
cudaError_t launch_moments(const T* f, int N, double L, int64_t B, double* out, cudaStream_t s);

// ---- fused Fourier stage (k_spectral.cu) ----------------------------------------------
// The whole Fourier side of a non-adjoint call in three launches for N = 8, 16 (float, double)
// and N = 32 (float), rank <= 32, Nrho <= 64: projection of P, loss operands la (field rank)
// and lb (field rank + 1, or nullptr), forward DFT, combine with gain scale `gain_scale`,
// inverse DFT and out = Re gain - fa Re(K_L la) - (fc ? fc Re(K_L lb) : 0). Same workspace
// X [nodes][(rank + nloss + 1) / 2][N^3] and Y [nodes][2 or 3][N^3] as the separate kernels.
template <typename T>
bool spectral_supported(const DevTables<T>& t);
template <typename T>
cudaError_t launch_spectral(const DevTables<T>& t, const T* P, NodeParams np, int64_t nodes, const T* la,
                            const T* lb, const int64_t* offs, T gain_scale, Cplx<T>* X, Cplx<T>* Y,
                            const T* fa, const T* fc, T* out, int* flags, cudaStream_t s);

// ---- device-rate probe (k_peaks.cu) ---------------------------------------------------------
// FP32 and FP64 FMA throughput of the current device in TFLOP/s (2 flops per FMA), best of three
// timed launches of independent FMA chains on every SM. Synchronous.
cudaError_t measure_fma_peaks(double& fp32_tflops, double& fp64_tflops);
// Cycles per back-to-back tcgen05.mma.kind::f16 (M = 128, K = 16, N = n) on the slowest SM; A from
// shared memory (a_tmem = 0) or TMEM (1).
cudaError_t measure_mma_cycles(int n, int a_tmem, double& cycles_per_mma);

}  // namespace dgfs
