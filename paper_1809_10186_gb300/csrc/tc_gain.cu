// Tensor-core (tcgen05) translate-product kernel for the 16-bit precisions.
//
// Computes, like the CUDA-core kernel, P_r = sum_pairs 2 w_p (T_s f)(T_-s f) for Q(f, f)
// (arXiv:1809.10186, Appendix, eqs. lowrank1 and apndx_fs_Glm_Qk). The translates are separable
// circulant operators; their three dense passes run as tcgen05.mma with FP32 accumulators in
// tensor memory, in the order x, z, y:
//
//   pass 1 (x): D1[(y,z)][x'] = sum_x f[x][y][z] Fx[x'][x]       A = f, held in TMEM
//   pass 2 (z): D2[(y,x')][z'] = sum_z D1[(y,z)][x'] Fz[z'][z]   A = MN-major tile in SMEM
//   pass 3 (y): D3[(x',z')][y'] = sum_y D2[(y,x')][z'] Fy[y'][y] A = MN-major full field in SMEM
//
// Data operands are 16-bit (fp16 with a per-node power-of-two scale, or bf16). Every filter F is
// split into a hi and a lo 16-bit part, and the parts are stacked along the MMA's N dimension, so
// one MMA yields both products: pass 1 stacks {+hi, +lo, -hi, -lo} (N = 4 n), passes 2 and 3 stack
// {hi, lo} of one sign (N = 2 n). The epilogue combines hi + 2^-e lo in FP32. The + sign's x filter
// carries the factor 2 w_p, so the products need no further weighting.
//
// One CTA per (radial point, node): 4 n/8 epilogue warpgroups (each owns 8 of the n output
// columns of every tile) and one MMA warp. Three 4n-column TMEM slots hold the accumulators; the
// slots alternate between the passes so that an MMA never waits for the epilogue of the
// accumulator it is about to overwrite when another slot is free. Both signs' pass-3 operands
// (full fields) stay in shared memory until the products of the pair are formed. All hand-offs
// are mbarriers; every wait is bounded: on timeout the CTA raises flag bit 0, every role stops,
// the MMAs and copies in flight are drained (bounded), TMEM is freed and P is not written.
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_gain.h"
#include "tc_ptx.cuh"

namespace dgfs {

namespace {

// lo filter parts are stored times 2^e (keeps them normal in fp16; bf16 has the exponent range)
constexpr int kLoShiftF16 = 11;
constexpr int kLoShiftBF16 = 8;

template <int N>
struct Geo {
    static_assert(N == 16 || N == 32, "tensor-core translates support N = 16 and 32");
    static constexpr int N2 = N * N;
    static constexpr int T = N2 / 128;           // 128-row tiles of one field
    static constexpr int ZT = 128 / N;            // y values per pass-1/2 tile
    static constexpr int KSTEPS = N / 16;         // K = 16 steps of one contraction
    static constexpr int KG = N / 8;              // core-matrix groups along K
    static constexpr int NWG = N / 8;             // epilogue warpgroups (8 output columns each)
    static constexpr int EPI_WARPS = 4 * NWG;
    static constexpr int THREADS = 32 * EPI_WARPS + 32;
    static constexpr int ISSUER = EPI_WARPS;      // warp index of the MMA warp
    // filter block of one (r, pair), K-major B operands: row n, column k at
    // (n/8) FB_SBO + (k/8) FB_LBO + (n%8) 16 + (k%8) 2
    static constexpr uint32_t FB_LBO = 128, FB_SBO = 16 * N;
    static constexpr uint32_t B1_BYTES = 4 * N2 * 2, B23_BYTES = 2 * N2 * 2;
    static constexpr uint32_t OFF_B1 = 0, OFF_B2 = B1_BYTES, OFF_B3 = B1_BYTES + 2 * B23_BYTES;
    static constexpr uint32_t F_BLOCK = B1_BYTES + 4 * B23_BYTES;
    // A2: pass-2 operand of one tile and sign, MN-major: rows m2 = yl N + x', k = z
    static constexpr uint32_t A2_SBO = 128, A2_LBO = 16 * 128, A2_BYTES = KG * A2_LBO;
    // A3: pass-3 operand of one sign (whole field), MN-major: rows m3 = x' N + z', k = y. The
    // padded m-group and tile strides spread one warp's 16-byte stores over all bank groups.
    static constexpr uint32_t A3_SBO = 144, A3_TS = 16 * 144 + 16, A3_LBO = T * A3_TS;
    static constexpr uint32_t A3_BYTES = KG * A3_LBO;
    // TMEM columns: three accumulator slots of 4 N columns, then f (N/2 columns per tile)
    static constexpr uint32_t SLOT = 4 * N;
    static constexpr uint32_t C_F = 3 * SLOT, F_COLS = T * (N / 2);
    static constexpr uint32_t C_USED = C_F + F_COLS;
    static constexpr uint32_t TMEM_COLS = C_USED <= 32 ? 32 : C_USED <= 64 ? 64 : C_USED <= 128 ? 128
                                          : C_USED <= 256 ? 256 : 512;
    static_assert(C_USED <= 512, "TMEM budget");
    // shared memory: A2 [slot 2][sign 2], A3 [sign 2], filters [buffer 2]
    static constexpr uint32_t S_A2 = 0, S_A3 = S_A2 + 4 * A2_BYTES;
    static constexpr uint32_t S_F = (S_A3 + 2 * A3_BYTES + 127) / 128 * 128;
    static constexpr uint32_t S_TOTAL = S_F + 2 * F_BLOCK;
    static_assert(S_TOTAL + 512 <= 232448, "shared-memory budget");
};

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {   // a -> low half, b -> high half
    if (BF) {
        __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    } else {
        __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    }
}

struct Bars {
    uint64_t full[3], freeb[3];        // TMEM slots: MMA completion -> epilogue, epilogue drained -> MMA
    uint64_t a2_full[2], a2_free[2];   // pass-2 operand tiles: epilogue -> MMA, MMA completion -> epilogue
    uint64_t a3_full, a3_free;         // pass-3 operands (both signs)
    uint64_t filt[2], fdone[2];        // filter buffers: copy landed; all MMAs of the pair using it done
    uint64_t drain;
};

// 8 columns of this thread's lane of the hi and lo parts (at c and c + N), combined as
// hi + eps lo in FP32; one sign at a time keeps 16 loaded values live next to the accumulators.
template <int N>
__device__ __forceinline__ void load_combined(uint32_t taddr, float eps, float (&v)[8]) {
    float hi[8], lo[8];
    tc::tmem_ld8(taddr, hi);
    tc::tmem_ld8(taddr + N, lo);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = fmaf(lo[j], eps, hi[j]);
}

template <bool BF>
__device__ __forceinline__ void pack8(const float (&v)[8], uint32_t (&u)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = pack2<BF>(v[2 * j], v[2 * j + 1]);
}

template <int N, bool BF>
__global__ void __launch_bounds__(Geo<N>::THREADS, 1)
k_tc_gain(const float* __restrict__ f, const int64_t* __restrict__ offs, const unsigned char* __restrict__ filt,
          int npairs, int Nrho, float* __restrict__ P, int* __restrict__ flags) {
    using G = Geo<N>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) Bars bars;
    __shared__ uint32_t s_tmem;
    __shared__ float s_red[G::EPI_WARPS];
    __shared__ int s_abort;
    volatile int* abort = &s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == G::ISSUER;
    const int r = blockIdx.x;
    const int64_t node = blockIdx.y;
    constexpr int64_t n3 = (int64_t)N * N * N;
    const float* fb = f + (offs ? offs[node] : node * n3);
    const uint32_t sb = tc::smem_u32(smem);
    const unsigned char* fglob = filt + (size_t)r * npairs * G::F_BLOCK;

    // filter copies issued and waited per buffer 0 / 1 (used by the MMA warp and the drain)
    int copies0 = npairs > 0 ? 1 : 0, copies1 = npairs > 1 ? 1 : 0, waited0 = 0, waited1 = 0;

    // ---- set-up: barriers, first filter copies, TMEM (MMA warp); max |f| (epilogue warps) -----
    if (issuer) {
        if (lane == 0) {
            for (int i = 0; i < 3; ++i) {
                tc::mbar_init(&bars.full[i], 1);
                tc::mbar_init(&bars.freeb[i], G::EPI_WARPS);
            }
            for (int i = 0; i < 2; ++i) {
                tc::mbar_init(&bars.a2_full[i], G::EPI_WARPS);
                tc::mbar_init(&bars.a2_free[i], 1);
                tc::mbar_init(&bars.filt[i], 1);
                tc::mbar_init(&bars.fdone[i], 1);
            }
            tc::mbar_init(&bars.a3_full, G::EPI_WARPS);
            tc::mbar_init(&bars.a3_free, 1);
            tc::mbar_init(&bars.drain, 1);
            tc::fence_mbar_init();
            s_abort = 0;
            for (int p = 0; p < 2 && p < npairs; ++p) {
                tc::mbar_expect_tx(&bars.filt[p], G::F_BLOCK);
                tc::bulk_g2s(smem + G::S_F + p * G::F_BLOCK, fglob + (size_t)p * G::F_BLOCK, G::F_BLOCK, &bars.filt[p]);
            }
        }
        __syncwarp();
        tc::tmem_alloc(&s_tmem, G::TMEM_COLS);
    } else if (!BF) {
        float mx = 0.f;
        for (int e = tid; e < n3; e += 32 * G::EPI_WARPS) mx = fmaxf(mx, fabsf(__ldg(fb + e)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_red[warp] = mx;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;

    float sf = 1.f;
    if (!BF) {
        float mx = s_red[0];
#pragma unroll
        for (int i = 1; i < G::EPI_WARPS; ++i) mx = fmaxf(mx, s_red[i]);
        if (mx > 0.f && isfinite(mx)) sf = exp2f(fminf(60.f, fmaxf(-60.f, floorf(log2f(512.f / mx)))));
    }
    const float eps = exp2f(-(float)(BF ? kLoShiftBF16 : kLoShiftF16));
    const float out_scale = BF ? 1.f : 1.f / (sf * sf);

    // ---- f -> TMEM as the pass-1 A operand: tile t, lane l = yl N + z holds f[0..N)[t ZT + yl][z] --
    if (!issuer) {
        const int q = warp & 3, w = warp >> 2, l = 32 * q + lane, yl = l / N, z = l % N;
        for (int t = w; t < G::T; t += G::NWG) {
            const float* src = fb + (size_t)(t * G::ZT + yl) * N + z;
            uint32_t v[N / 2];
#pragma unroll
            for (int c = 0; c < N / 2; ++c)
                v[c] = pack2<BF>(__ldg(src + (size_t)(2 * c) * G::N2) * sf, __ldg(src + (size_t)(2 * c + 1) * G::N2) * sf);
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + G::C_F + t * (N / 2);
            if constexpr (N == 32) tc::tmem_st16(ta, v);
            else tc::tmem_st8(ta, v);
        }
        tc::tmem_wait_st();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();

    if (issuer) {
        // ================================ MMA warp (converged) ================================
        // per-slot / per-buffer state as bit masks (bit i = slot or buffer i), kept in registers
        uint32_t used = 0, ph_free = 0, ph_a2full = 0, ph_a3full = 0, ph_fdone = 0;
        constexpr uint32_t id1 = tc::idesc_f16(BF, false, false, 4 * N, 128);
        constexpr uint32_t id23 = tc::idesc_f16(BF, true, false, 2 * N, 128);
#define DGFS_WAITW(bar, ph)                                             \
    do {                                                                \
        if (!tc::warp_wait((bar), (ph), abort)) goto mma_done;          \
    } while (0)
#define DGFS_ACQUIRE(s)                                                 \
    do {                                                                \
        if (used & (1u << (s))) {                                       \
            DGFS_WAITW(&bars.freeb[s], (ph_free >> (s)) & 1u);          \
            ph_free ^= 1u << (s);                                       \
        }                                                               \
        used |= 1u << (s);                                              \
        tc::tc_fence_after();                                           \
    } while (0)
        for (int p = 0; p < npairs; ++p) {
            const int fbuf = p & 1;
            DGFS_WAITW(&bars.filt[fbuf], (uint32_t)((fbuf ? waited1 : waited0) & 1));
            if (fbuf) ++waited1;
            else ++waited0;
            tc::tc_fence_after();
            const uint32_t fsm = sb + G::S_F + fbuf * G::F_BLOCK;
            // front: pass 1 of tile t (slot 0) and pass 2 of tile t - 1 (slot 1 + (t - 1) % 2)
            for (int t = 0; t <= G::T; ++t) {
                if (t < G::T) {
                    DGFS_ACQUIRE(0);
#pragma unroll
                    for (int ks = 0; ks < G::KSTEPS; ++ks)
                        tc::mma_ts_warp(tmem, tmem + G::C_F + t * (N / 2) + 8 * ks,
                                        tc::sdesc(fsm + G::OFF_B1 + ks * 2 * G::FB_LBO, G::FB_LBO, G::FB_SBO), id1, ks);
                    tc::mma_commit_warp(&bars.full[0]);
                    // the other filter buffer (pair p - 1, whose MMAs are complete by now) takes pair p + 1
                    if (t == 0 && p >= 1 && p + 1 < npairs) {
                        const int nb = (p + 1) & 1;
                        DGFS_WAITW(&bars.fdone[nb], (ph_fdone >> nb) & 1u);
                        ph_fdone ^= 1u << nb;
                        if (tc::elect_one()) {
                            tc::mbar_expect_tx(&bars.filt[nb], G::F_BLOCK);
                            tc::bulk_g2s(smem + G::S_F + nb * G::F_BLOCK, fglob + (size_t)(p + 1) * G::F_BLOCK,
                                         G::F_BLOCK, &bars.filt[nb]);
                        }
                        __syncwarp();
                        if (nb) ++copies1;
                        else ++copies0;
                    }
                }
                if (t >= 1) {
                    const int a = (t - 1) & 1, s = 1 + a;
                    DGFS_WAITW(&bars.a2_full[a], (ph_a2full >> a) & 1u);
                    ph_a2full ^= 1u << a;
                    DGFS_ACQUIRE(s);
#pragma unroll
                    for (int g = 0; g < 2; ++g)
#pragma unroll
                        for (int ks = 0; ks < G::KSTEPS; ++ks)
                            tc::mma_ss_warp(tmem + s * G::SLOT + g * 2 * N,
                                            tc::sdesc(sb + G::S_A2 + (a * 2 + g) * G::A2_BYTES + ks * 2 * G::A2_LBO,
                                                      G::A2_LBO, G::A2_SBO),
                                            tc::sdesc(fsm + G::OFF_B2 + g * G::B23_BYTES + ks * 2 * G::FB_LBO, G::FB_LBO,
                                                      G::FB_SBO),
                                            id23, ks);
                    tc::mma_commit_warp(&bars.full[s]);
                    tc::mma_commit_warp(&bars.a2_free[a]);
                }
            }
            // back: pass 3 of tile u into slot 2 (u even) or 0 (u odd)
            DGFS_WAITW(&bars.a3_full, ph_a3full);
            ph_a3full ^= 1;
            tc::tc_fence_after();
            for (int u = 0; u < G::T; ++u) {
                const int s = (u & 1) ? 0 : 2;
                DGFS_ACQUIRE(s);
#pragma unroll
                for (int g = 0; g < 2; ++g)
#pragma unroll
                    for (int ks = 0; ks < G::KSTEPS; ++ks)
                        tc::mma_ss_warp(tmem + s * G::SLOT + g * 2 * N,
                                        tc::sdesc(sb + G::S_A3 + g * G::A3_BYTES + u * G::A3_TS + ks * 2 * G::A3_LBO,
                                                  G::A3_LBO, G::A3_SBO),
                                        tc::sdesc(fsm + G::OFF_B3 + g * G::B23_BYTES + ks * 2 * G::FB_LBO, G::FB_LBO,
                                                  G::FB_SBO),
                                        id23, ks);
                tc::mma_commit_warp(&bars.full[s]);
            }
            tc::mma_commit_warp(&bars.a3_free);
            tc::mma_commit_warp(&bars.fdone[fbuf]);
        }
#undef DGFS_ACQUIRE
#undef DGFS_WAITW
    mma_done:;
    } else {
        // ============================== epilogue warpgroups ===================================
        const int q = warp & 3, w = warp >> 2, c0 = 8 * w;
        const int l = 32 * q + lane, yl = l / N, lz = l % N;   // tile row: (yl, z) in pass 1, (yl, x') in pass 2
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        // store offsets: A2 unit (rows yl N + c0 .. +8, k = z = lz); A3 unit (rows lz N + c0 .. +8)
        const uint32_t a2_off = ((uint32_t)(yl * N + c0) >> 3) * G::A2_SBO + (lz >> 3) * G::A2_LBO + (lz & 7) * 16;
        const int mg3 = (lz * N + c0) >> 3;
        const uint32_t a3_off = (mg3 >> 4) * G::A3_TS + (mg3 & 15) * G::A3_SBO;
        uint32_t ph_full = 0, ph_a2free = 0, a2_used = 0, ph_a3free = 0;   // bit masks, as in the MMA warp
        float acc[G::T][8];
#pragma unroll
        for (int u = 0; u < G::T; ++u)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[u][j] = 0.f;
#define DGFS_WAITE(bar, ph)                                             \
    do {                                                                \
        if (!tc::warp_wait((bar), (ph), abort)) goto epi_done;          \
    } while (0)
        for (int p = 0; p < npairs; ++p) {
            for (int t = 0; t <= G::T; ++t) {
                if (t < G::T) {
                    // pass-1 tile t -> pass-2 operands of both signs
                    DGFS_WAITE(&bars.full[0], ph_full & 1u);
                    ph_full ^= 1u;
                    tc::tc_fence_after();
                    uint32_t up[4], um[4];
                    {
                        float v[8];
                        load_combined<N>(trow + c0, eps, v);
                        pack8<BF>(v, up);
                        load_combined<N>(trow + 2 * N + c0, eps, v);
                        pack8<BF>(v, um);
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bars.freeb[0]);
                    const int a = t & 1;
                    if (a2_used & (1u << a)) {
                        DGFS_WAITE(&bars.a2_free[a], (ph_a2free >> a) & 1u);
                        ph_a2free ^= 1u << a;
                    }
                    a2_used |= 1u << a;
                    const uint32_t dst = sb + G::S_A2 + a * 2 * G::A2_BYTES + a2_off;
                    tc::st_shared_v4(dst, up[0], up[1], up[2], up[3]);
                    tc::st_shared_v4(dst + G::A2_BYTES, um[0], um[1], um[2], um[3]);
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bars.a2_full[a]);
                }
                if (t >= 1) {
                    // pass-2 tile t - 1 -> rows of the pass-3 operands of both signs
                    const int tt = t - 1, s = 1 + (tt & 1);
                    DGFS_WAITE(&bars.full[s], (ph_full >> s) & 1u);
                    ph_full ^= 1u << s;
                    tc::tc_fence_after();
                    uint32_t up[4], um[4];
                    {
                        float v[8];
                        load_combined<N>(trow + s * G::SLOT + c0, eps, v);
                        pack8<BF>(v, up);
                        load_combined<N>(trow + s * G::SLOT + 2 * N + c0, eps, v);
                        pack8<BF>(v, um);
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bars.freeb[s]);
                    if (tt == 0 && p > 0) {   // the previous pair's pass 3 has read the operands
                        DGFS_WAITE(&bars.a3_free, ph_a3free);
                        ph_a3free ^= 1;
                    }
                    const int y = tt * G::ZT + yl;
                    const uint32_t dst = sb + G::S_A3 + a3_off + (y >> 3) * G::A3_LBO + (y & 7) * 16;
                    tc::st_shared_v4(dst, up[0], up[1], up[2], up[3]);
                    tc::st_shared_v4(dst + G::A3_BYTES, um[0], um[1], um[2], um[3]);
                    if (tt == G::T - 1) {
                        tc::fence_proxy_async();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&bars.a3_full);
                    }
                }
            }
            // pass-3 tiles: products of the two translates
#pragma unroll
            for (int u = 0; u < G::T; ++u) {
                const int s = (u & 1) ? 0 : 2;
                DGFS_WAITE(&bars.full[s], (ph_full >> s) & 1u);
                ph_full ^= 1u << s;
                tc::tc_fence_after();
                float vp[8], vm[8];
                load_combined<N>(trow + s * G::SLOT + c0, eps, vp);
                load_combined<N>(trow + s * G::SLOT + 2 * N + c0, eps, vm);
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bars.freeb[s]);
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[u][j] = fmaf(vp[j], vm[j], acc[u][j]);
            }
        }
#undef DGFS_WAITE
        if (!*abort) {   // P[node][r][x'][y'][z'], row m3 = x' N + z' of tile u, column y' = c0 + j
            float* dst = P + ((size_t)node * Nrho + r) * n3;
#pragma unroll
            for (int u = 0; u < G::T; ++u) {
                const int m3 = u * 128 + l, xp = m3 / N, zp = m3 % N;
                float* o = dst + (size_t)xp * G::N2 + (size_t)c0 * N + zp;
#pragma unroll
                for (int j = 0; j < 8; ++j) o[(size_t)j * N] = acc[u][j] * out_scale;
            }
        }
    epi_done:;
    }

    // ---- drain: no MMA or copy of this CTA may be in flight when TMEM is freed -----------
    tc::tc_fence_before();
    __syncthreads();
    if (issuer) {
        if (tc::elect_one()) {   // the lane that issued every MMA and copy
            if (*abort) atomicOr(flags, 1);
            tc::mma_commit(&bars.drain);
            if (!tc::mbar_wait(&bars.drain, 0)) atomicOr(flags, 1);
            for (int i = 0; i < 2; ++i)
                for (int k = i ? waited1 : waited0; k < (i ? copies1 : copies0); ++k)
                    if (!tc::mbar_wait(&bars.filt[i], (uint32_t)(k & 1))) {
                        atomicOr(flags, 1);
                        break;
                    }
        }
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, G::TMEM_COLS);
    }
}

template <int N, bool BF>
cudaError_t launch_n(const TcTables& t, const float* f, const int64_t* offs, int64_t nodes, float* P,
                     int* flags, cudaStream_t s) {
    using G = Geo<N>;
    auto kern = k_tc_gain<N, BF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::S_TOTAL);
    if (e != cudaSuccess) return e;
    const int64_t n3 = (int64_t)N * N * N;
    for (int64_t n0 = 0; n0 < nodes; n0 += 65535) {
        const int64_t nn = nodes - n0 < 65535 ? nodes - n0 : 65535;
        kern<<<dim3(t.Nrho, (unsigned)nn), G::THREADS, G::S_TOTAL, s>>>(
            f + (offs ? 0 : n0 * n3), offs ? offs + n0 : nullptr, static_cast<const unsigned char*>(t.mats),
            t.npairs, t.Nrho, P + n0 * t.Nrho * n3, flags);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// host-side rounding of a double to the 16-bit operand types
uint16_t to_half_bits(double x) {
    __half h = __double2half(x);
    uint16_t b;
    std::memcpy(&b, &h, 2);
    return b;
}
double half_bits_value(uint16_t b) {
    __half h;
    std::memcpy(&h, &b, 2);
    return (double)__half2float(h);
}
uint16_t to_bf16_bits(double x) {
    __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    uint16_t b;
    std::memcpy(&b, &h, 2);
    return b;
}
double bf16_bits_value(uint16_t b) {
    __nv_bfloat16 h;
    std::memcpy(&h, &b, 2);
    return (double)__bfloat162float(h);
}

}  // namespace

bool tc_supported(int N) { return N == 16 || N == 32; }

int tc_extra_launches(int) { return 0; }

size_t build_tc_tables(const HostPlan& hp, int prec, std::vector<unsigned char>& blob, TcTables& t) {
    const int N = hp.N, np = hp.npairs, Nr = hp.Nrho;
    const bool bf = prec == DGFS_PREC_BF16S;
    const double lo_scale = std::ldexp(1.0, bf ? kLoShiftBF16 : kLoShiftF16);
    const size_t n2b = (size_t)N * N * 2;            // bytes of one N x N 16-bit matrix
    const size_t b1 = 4 * n2b, b23 = 2 * n2b, block = b1 + 4 * b23;
    blob.assign((size_t)Nr * np * block, 0);
    const size_t sbo = 16 * (size_t)N, lbo = 128;
    // K-major core-matrix layout of a B operand: row n (output index), column k (input index)
    auto put = [&](unsigned char* base, int n, int k, uint16_t bits) {
        std::memcpy(base + (n / 8) * sbo + (k / 8) * lbo + (n % 8) * 16 + (k % 8) * 2, &bits, 2);
    };
    // hi + 2^-e lo split of v, both rounded to the operand type
    auto split = [&](double v, uint16_t& hi, uint16_t& lo) {
        hi = bf ? to_bf16_bits(v) : to_half_bits(v);
        const double hv = bf ? bf16_bits_value(hi) : half_bits_value(hi);
        lo = bf ? to_bf16_bits((v - hv) * lo_scale) : to_half_bits((v - hv) * lo_scale);
    };
    for (int r = 0; r < Nr; ++r)
        for (int p = 0; p < np; ++p) {
            unsigned char* blk = blob.data() + ((size_t)r * np + p) * block;
            // F_+[i][j] = a[(i - j) mod N] (translate by +s along the axis); F_- = F_+^T (T_-s = T_s^T)
            auto F = [&](int axis, int sign, int i, int j) {
                const double* fl = &hp.filt[(((size_t)r * np + p) * 3 + axis) * N];
                const int d = sign == 0 ? i - j : j - i;
                return fl[((d % N) + N) % N];
            };
            const double w2 = 2.0 * hp.wsig[p];
            for (int g = 0; g < 2; ++g)
                for (int i = 0; i < N; ++i)
                    for (int j = 0; j < N; ++j) {
                        uint16_t hi, lo;
                        // pass 1 (x, axis 0): parts (+hi, +lo, -hi, -lo); the + filter carries 2 w_p
                        split(F(0, g, i, j) * (g == 0 ? w2 : 1.0), hi, lo);
                        put(blk, (2 * g) * N + i, j, hi);
                        put(blk, (2 * g + 1) * N + i, j, lo);
                        // pass 2 (z, axis 2) and pass 3 (y, axis 1): parts (hi, lo) per sign
                        split(F(2, g, i, j), hi, lo);
                        put(blk + b1 + g * b23, i, j, hi);
                        put(blk + b1 + g * b23, N + i, j, lo);
                        split(F(1, g, i, j), hi, lo);
                        put(blk + b1 + 2 * b23 + g * b23, i, j, hi);
                        put(blk + b1 + 2 * b23 + g * b23, N + i, j, lo);
                    }
        }
    t.N = N;
    t.Nrho = Nr;
    t.npairs = np;
    t.mats = reinterpret_cast<const void*>((uintptr_t)0);
    return blob.size();
}

void rebase_tc_tables(TcTables& t, void* base) {
    t.mats = static_cast<unsigned char*>(base) + reinterpret_cast<uintptr_t>(t.mats);
}

cudaError_t launch_tc_gain_products(const TcTables& t, int prec, const float* f, const float* g,
                                    const int64_t* offs, int64_t nodes, float* P, int* flags,
                                    cudaStream_t s) {
    if (g) return cudaErrorNotSupported;
    if (nodes <= 0) return cudaSuccess;
    const bool bf = prec == DGFS_PREC_BF16S;
    switch (t.N) {
        case 16: return bf ? launch_n<16, true>(t, f, offs, nodes, P, flags, s) : launch_n<16, false>(t, f, offs, nodes, P, flags, s);
        case 32: return bf ? launch_n<32, true>(t, f, offs, nodes, P, flags, s) : launch_n<32, false>(t, f, offs, nodes, P, flags, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dgfs
