// Split-data tensor-core (tcgen05) translate-product kernel: the precisions F16X3 and BF16X3.
//
// Computes P_r = sum_pairs 2 w_p (T_s f)(T_-s f) for Q(f, f) like the other translate kernels
// (arXiv:1809.10186, Appendix, eqs. lowrank1 and apndx_fs_Glm_Qk): the translates are separable
// circulant operators, three dense passes in the order x, z, y as in tc_gain.cu. Here every data
// operand (f and the two stored intermediates) AND every filter is split into a 16-bit hi part
// and a lo part carrying 2^e (e = 11 for fp16, 8 for bf16):
//
//   x = hi(x) + 2^-e lo(x),       A F = A_hi F_hi + 2^-e (A_hi F_lo + A_lo F_hi) + O(2^-2e)
//
// A K = 16 step of a pass is two MMAs: A_hi x [F_hi | F_lo] into the accumulator pair [hi | lo] of a
// TMEM slot, then A_lo x F_hi into its lo half; the epilogue combines hi + 2^-e lo in FP32 and splits
// the result again for the next pass. FP32 accumulation keeps the translates at about FP32 accuracy
// (fp16: 11 + 11 significand bits; bf16: 8 + 8).
//
// Both signs' pass-3 operands with their lo parts (4 N^3 x 2 bytes) do not fit one SM's shared
// memory at N = 32, so two CTAs of a thread-block cluster share the field of one (node, radial
// points) item. CTA c runs passes 1 and 2 of the y-tiles [c T/2, (c + 1) T/2) (pass-1/2 tiles are
// blocks of y) and pass 3 of the x'-tiles [c T/2, (c + 1) T/2) (pass-3 tiles are blocks of x'),
// both signs. The pass-2 epilogue writes every result row straight into the pass-3 operand of the
// CTA that owns its x' (its own shared memory, or the peer's through non-blocking st.async stores);
// each CTA then forms the products of its x'-tiles with both signs in its own TMEM. Two cluster
// hand-offs per sphere pair: "pass-3 operands complete" (the threads of a CTA whose rows are local
// arrive on its barrier, one of them registering the bytes the peer sends, and the peer's st.async
// stores complete those bytes) and "pass-3 operands released" (both CTAs' pass-3 MMA warps commit
// to both CTAs' barriers by a multicast commit). The pass-2
// operands are handed over one sign at a time, so warpgroup 0 writes one sign while the pass-2 MMAs
// read the other.
//
// Per CTA, as in tc_gain.cu: two epilogue warpgroups and a third warpgroup of four MMA warps
// (pass 1, pass 2, pass 3 into slot 2, pass 3 into slot 3). Epilogue warpgroup w works on sign w:
// it turns the sign-w columns of each pass-1 result into the sign-w pass-2 operands and of each
// pass-2 result into sign-w pass-3 operand rows, software-pipelined (the pass-1 epilogue of front
// tile i, then the pass-2 epilogue of tile i - 1, whose MMAs ran meanwhile); in the back it forms
// the products of the pass-3 tiles in slot 2 + w, accumulating P_r in registers (the slot's two sign
// halves are completed and released separately, so the next tile's + MMAs overlap the read of the
// - half). Every wait is bounded; on
// timeout the CTA raises flag bit 0, every role stops at its next wait, the MMAs and copies in
// flight are drained, TMEM is freed and no P_r is written; both CTAs meet at a final cluster barrier.
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/dgfs.h"
#include "tc_gain.h"
#include "tc_ptx.cuh"

namespace dgfs {

namespace {

constexpr int kLoShiftF16 = 11;
constexpr int kLoShiftBF16 = 8;

template <int N>
struct Geo3 {
    static_assert(N == 16 || N == 32, "split-data tensor-core tiles of N = 16 and 32 (N = 24 runs on 32)");
    static constexpr int N2 = N * N;
    static constexpr int T = N2 / 128;            // 128-row tiles of one field
    static constexpr int TH = T / 2;              // front (y) tiles and back (x') tiles of one CTA
    static constexpr int ZT = 128 / N;            // y values of a pass-1/2 tile, x' values of a pass-3 tile
    static constexpr int KSTEPS = N / 16;
    static constexpr int KG = N / 8;
    static constexpr int EPI_WARPS = 8;
    static constexpr int THREADS = 32 * EPI_WARPS + 128;
    static constexpr int ISSUER = EPI_WARPS;
    static constexpr uint32_t REG_LAUNCH = 168, REG_EPI = 216, REG_MMA = 72;
    static_assert(256 * REG_EPI + 128 * REG_MMA <= 384 * REG_LAUNCH, "register reallocation exceeds the pool");
    // filter block of one (r, pair), K-major B operands, row n, column k at (n/8) FB_SBO + (k/8) FB_LBO +
    // (n%8) 16 + (k%8) 2: B1 (x, pass 1) rows [F+hi; F-hi; F+lo; F-lo]; B2 (z) and B3 (y) per sign [hi; lo]
    static constexpr uint32_t FB_LBO = 128, FB_SBO = 16 * N;
    static constexpr uint32_t SB_BYTES = 2 * N2 * 2;                 // [hi; lo] of one sign
    static constexpr uint32_t OFF_B1 = 0, OFF_B2 = 2 * SB_BYTES, OFF_B3 = 4 * SB_BYTES;
    static constexpr uint32_t F_BLOCK = 6 * SB_BYTES;
    // pass-2 operand of one tile, sign and part, MN-major: rows m2 = yl N + x', k = z
    static constexpr uint32_t A2_SBO = 128, A2_LBO = 16 * 128, A2_BYTES = KG * A2_LBO;
    // pass-3 operand of one sign and part: this CTA's TH x'-tiles, MN-major, rows m3 = x' N + z' (local
    // tile ul = m3 / 128 - c TH), k = y; padded so that a warp's 16-byte stores spread over bank groups
    static constexpr uint32_t A3_SBO = 144, A3_TS = 16 * 144 + 16, A3_LBO = TH * A3_TS;
    static constexpr uint32_t A3_BYTES = KG * A3_LBO;
    // bytes of pass-3 operand rows one CTA's epilogue sends to its peer per sphere pair: the 128 threads
    // whose rows the peer owns, per front tile 2 row groups per 16 columns z', hi and lo, 16 bytes each
    static constexpr uint32_t A3_REMOTE_BYTES = 128u * TH * (N / 16) * 2 * 2 * 16;
    // TMEM columns: pass-1 slot [+main | -main | +lo | -lo], pass-2/3 slots 2, 3 [+hi | +lo | -hi | -lo],
    // then f_hi and f_lo of the TH front tiles
    static constexpr uint32_t C_P1 = 0, C_S2 = 4 * N, C_S3 = 8 * N;
    static constexpr uint32_t C_FH = 12 * N, C_FL = 12 * N + TH * (N / 2), C_USED = 12 * N + TH * N;
    static constexpr uint32_t TMEM_COLS = C_USED <= 32 ? 32 : C_USED <= 64 ? 64 : C_USED <= 128 ? 128
                                          : C_USED <= 256 ? 256 : 512;
    static_assert(C_USED <= 512, "TMEM budget");
    // shared memory: A2 [sign][part], A3 [sign][part], filters [buffer 2]
    static constexpr uint32_t S_A2 = 0, S_A3 = 4 * A2_BYTES;
    static constexpr uint32_t S_F = (S_A3 + 4 * A3_BYTES + 127) / 128 * 128;
    static constexpr uint32_t S_TOTAL = S_F + 2 * F_BLOCK;
    static_assert(S_TOTAL + 1024 <= 232448, "shared-memory budget");
    static_assert(A3_TS % 16 == 0 && A2_BYTES % 16 == 0 && A3_BYTES % 16 == 0 && F_BLOCK % 16 == 0 &&
                  S_A3 % 16 == 0 && S_F % 16 == 0, "descriptor offsets are multiples of 16 bytes");
};

// hi and lo parts (lo times 2^e) of two values, packed: a -> low half, b -> high half
template <bool BF>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if (BF) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        constexpr float s = (float)(1 << kLoShiftBF16);
        const __nv_bfloat162 l = __floats2bfloat162_rn((a - hf.x) * s, (b - hf.y) * s);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        constexpr float s = (float)(1 << kLoShiftF16);
        const __half2 l = __floats2half2_rn((a - hf.x) * s, (b - hf.y) * s);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

struct Bars3 {
    uint64_t full1, free1;             // pass-1 slot: MMA -> both warpgroups, both warpgroups -> MMA
    uint64_t a2_full[2], a2_free[2];   // pass-2 operands of sign s: warpgroup s -> MMA, MMA completion -> warpgroup s
    uint64_t full2[2], free2[2];       // slots 2, 3 used by pass 2 (both warpgroups drain, one sign each)
    uint64_t full3p[2], free3p[2];     // slots 2, 3 used by pass 3 (warpgroup b drains slot 2 + b): + sign
    uint64_t full3m[2], free3m[2];     // and - sign columns, each half released as soon as it is read
    uint64_t free3x[2];                // last pass-3 drain of a slot in a pair
    uint64_t a3_full;                  // the 128 pass-2 epilogue threads (of both CTAs) that own rows here wrote them
    uint64_t a3_free;                  // both CTAs' pass-3 MMAs read this pair's operands
    uint64_t filt[2], fdone[2];        // filter buffers: copy landed; all MMAs of the pair using it done
    uint64_t drain;
};

#define DGFS_WAITW(bar, ph)                                             \
    do {                                                                \
        if (!tc::warp_wait((bar), (ph), abort)) return;                 \
    } while (0)
#define DGFS_WAITWC(bar, ph)                                            \
    do {                                                                \
        if (!tc::warp_wait_cluster((bar), (ph), abort)) return;         \
    } while (0)

// Pass 1 of the CTA's front tiles i (both signs) into the pass-1 slot; refills the filter buffers.
template <int N, bool BF>
__device__ __forceinline__ void mma3_p1_loop(Bars3& bars, unsigned char* smem, uint32_t sb, uint32_t tmem,
                                             const unsigned char* fglob, int nseq, volatile int* abort,
                                             int& copies0, int& copies1, int& waited0, int& waited1) {
    using G = Geo3<N>;
    uint32_t ph_free = 0;
    int uses = 0;
    uint32_t ph_fdone = 0;
    constexpr uint32_t idw = tc::idesc_f16(BF, false, false, 4 * N, 128);   // [+hi; -hi; +lo; -lo]
    constexpr uint32_t idn = tc::idesc_f16(BF, false, false, 2 * N, 128);   // [+hi; -hi]
    constexpr uint64_t dF = tc::sdesc_base(G::FB_LBO, G::FB_SBO);
    const uint32_t sb16 = sb >> 4;
    for (int p = 0; p < nseq; ++p) {
        const int fbuf = p & 1;
        DGFS_WAITW(&bars.filt[fbuf], (uint32_t)((p >> 1) & 1));
        if (fbuf) ++waited1;
        else ++waited0;
        tc::tc_fence_after();
        const uint32_t f16 = sb16 + (G::S_F + fbuf * G::F_BLOCK) / 16;
        for (int i = 0; i < G::TH; ++i) {
            if (uses > 0) {
                DGFS_WAITW(&bars.free1, ph_free);
                ph_free ^= 1u;
            }
            ++uses;
            tc::tc_fence_after();
            const uint32_t d = tmem + G::C_P1;
            const uint32_t fh = tmem + G::C_FH + i * (N / 2), fl = tmem + G::C_FL + i * (N / 2);
#pragma unroll
            for (int ks = 0; ks < G::KSTEPS; ++ks) {
                const uint64_t bd = tc::sdesc_at(dF, f16 + (G::OFF_B1 + ks * 2 * G::FB_LBO) / 16);
                tc::mma_ts_warp(d, fh + 8 * ks, bd, idw, ks);             // f_hi [F+hi | F-hi | F+lo | F-lo]
                tc::mma_ts_warp(d + 2 * N, fl + 8 * ks, bd, idn, 1);      // + f_lo [F+hi | F-hi] into the lo halves
            }
            tc::mma_commit_warp(&bars.full1);
            if (i == 0 && p >= 1 && p + 1 < nseq) {
                const int nb = (p + 1) & 1;
                DGFS_WAITW(&bars.fdone[nb], (ph_fdone >> nb) & 1u);
                ph_fdone ^= 1u << nb;
                if (tc::elect_one()) {
                    tc::mbar_expect_tx(&bars.filt[nb], G::F_BLOCK);
                    tc::bulk_g2s(smem + G::S_F + nb * G::F_BLOCK, fglob + (size_t)(p + 1) * G::F_BLOCK, G::F_BLOCK,
                                 &bars.filt[nb]);
                }
                __syncwarp();
                if (nb) ++copies1;
                else ++copies0;
            }
        }
        tc::mma_commit_warp(&bars.fdone[fbuf]);
    }
}

// Pass 2 of front tile i (both signs) into slot 2 + i % 2. A slot's first pass-2 use in a pair waits
// for the previous pair's last pass-3 drain of it (free3x); later uses for the pass-2 drain (free2).
template <int N, bool BF>
__device__ __forceinline__ void mma3_p2_loop(Bars3& bars, uint32_t sb, uint32_t tmem, int nseq, volatile int* abort) {
    using G = Geo3<N>;
    uint32_t ph_a2 = 0, ph_x = 0, ph_f2 = 0;   // ph_a2: bit s = sign s
    constexpr uint32_t idw = tc::idesc_f16(BF, true, false, 2 * N, 128);
    constexpr uint32_t idn = tc::idesc_f16(BF, true, false, N, 128);
    constexpr uint64_t dF = tc::sdesc_base(G::FB_LBO, G::FB_SBO);
    constexpr uint64_t dA2 = tc::sdesc_base(G::A2_LBO, G::A2_SBO);
    const uint32_t sb16 = sb >> 4;
    for (int p = 0; p < nseq; ++p) {
        const int fbuf = p & 1;
        DGFS_WAITW(&bars.filt[fbuf], (uint32_t)((p >> 1) & 1));
        tc::tc_fence_after();
        const uint32_t f16 = sb16 + (G::S_F + fbuf * G::F_BLOCK) / 16;
        for (int i = 0; i < G::TH; ++i) {
            const int b = i & 1, j = i >> 1;
            if (j == 0) {
                if (p > 0) {
                    DGFS_WAITW(&bars.free3x[b], (ph_x >> b) & 1u);
                    ph_x ^= 1u << b;
                }
            } else {
                DGFS_WAITW(&bars.free2[b], (ph_f2 >> b) & 1u);
                ph_f2 ^= 1u << b;
            }
            tc::tc_fence_after();
            const uint32_t d = tmem + (b ? G::C_S3 : G::C_S2);
#pragma unroll
            for (int sg = 0; sg < 2; ++sg) {
                // the operands of sign sg are in shared memory (warpgroup 0 writes the other sign meanwhile)
                DGFS_WAITW(&bars.a2_full[sg], (ph_a2 >> sg) & 1u);
                ph_a2 ^= 1u << sg;
                tc::tc_fence_after();
                const uint32_t a16 = sb16 + (G::S_A2 + sg * 2 * G::A2_BYTES) / 16;   // [sign][hi, lo]
#pragma unroll
                for (int ks = 0; ks < G::KSTEPS; ++ks) {
                    const uint64_t bd = tc::sdesc_at(dF, f16 + (G::OFF_B2 + sg * G::SB_BYTES + ks * 2 * G::FB_LBO) / 16);
                    tc::mma_ss_warp(d + sg * 2 * N, tc::sdesc_at(dA2, a16 + (ks * 2 * G::A2_LBO) / 16), bd, idw, ks);
                    tc::mma_ss_warp(d + sg * 2 * N + N, tc::sdesc_at(dA2, a16 + (G::A2_BYTES + ks * 2 * G::A2_LBO) / 16),
                                    bd, idn, 1);
                }
                tc::mma_commit_warp(&bars.a2_free[sg]);
            }
            tc::mma_commit_warp(&bars.full2[b]);
        }
        // the pass-2 drains this warp did not wait for (the last use of each slot in the pair)
        // complete free2 phases too: account for them so the parities stay aligned
        for (int b = 0; b < 2; ++b) {
            const int uses_b = (G::TH + 1 - b) / 2;   // pass-2 uses of slot 2 + b per pair
            if (uses_b > 0) ph_f2 ^= 1u << b;         // the pair's last drain of the slot was not waited
        }
        tc::mma_commit_warp(&bars.fdone[fbuf]);
    }
}

// Pass 3 of back tiles k = b, b + 2, ... (both signs) into slot 2 + b once the pass-3 operands of
// both CTAs' epilogues are complete (warpgroup b drains the slot); the release of the operands is
// signalled to both CTAs (multicast commit).
template <int N, bool BF, int b>
__device__ __forceinline__ void mma3_p3_loop(Bars3& bars, uint32_t sb, uint32_t tmem, int nseq, volatile int* abort) {
    using G = Geo3<N>;
    uint32_t ph_a3full = 0, ph_f3p = 0, ph_f3m = 0;
    constexpr uint32_t idw = tc::idesc_f16(BF, true, false, 2 * N, 128);
    constexpr uint32_t idn = tc::idesc_f16(BF, true, false, N, 128);
    constexpr uint64_t dF = tc::sdesc_base(G::FB_LBO, G::FB_SBO);
    constexpr uint64_t dA3 = tc::sdesc_base(G::A3_LBO, G::A3_SBO);
    const uint32_t sb16 = sb >> 4;
    for (int p = 0; p < nseq; ++p) {
        const int fbuf = p & 1;
        DGFS_WAITW(&bars.filt[fbuf], (uint32_t)((p >> 1) & 1));
        const uint32_t f16 = sb16 + (G::S_F + fbuf * G::F_BLOCK) / 16;
        DGFS_WAITWC(&bars.a3_full, ph_a3full);
        ph_a3full ^= 1u;
        tc::fence_proxy_async();   // the peer's st.async rows, acquired with the barrier, to the tensor core
        tc::tc_fence_after();
        int n = 0;
        for (int k = b; k < G::TH; k += 2, ++n) {
            const uint32_t d = tmem + (b ? G::C_S3 : G::C_S2);
#pragma unroll
            for (int sg = 0; sg < 2; ++sg) {   // sign +, then sign -; each half reused once it is read
                if (n > 0) {
                    if (sg) {
                        DGFS_WAITW(&bars.free3m[b], ph_f3m);
                        ph_f3m ^= 1u;
                    } else {
                        DGFS_WAITW(&bars.free3p[b], ph_f3p);
                        ph_f3p ^= 1u;
                    }
                    tc::tc_fence_after();
                }
                const uint32_t a16 = sb16 + (G::S_A3 + sg * 2 * G::A3_BYTES + k * G::A3_TS) / 16;
#pragma unroll
                for (int ks = 0; ks < G::KSTEPS; ++ks) {
                    const uint64_t bd = tc::sdesc_at(dF, f16 + (G::OFF_B3 + sg * G::SB_BYTES + ks * 2 * G::FB_LBO) / 16);
                    tc::mma_ss_warp(d + sg * 2 * N, tc::sdesc_at(dA3, a16 + (ks * 2 * G::A3_LBO) / 16), bd, idw, ks);
                    tc::mma_ss_warp(d + sg * 2 * N + N, tc::sdesc_at(dA3, a16 + (G::A3_BYTES + ks * 2 * G::A3_LBO) / 16),
                                    bd, idn, 1);
                }
                tc::mma_commit_warp(sg ? &bars.full3m[b] : &bars.full3p[b]);
            }
        }
        if (n > 0) {   // the pair's last drains of the slot (not waited here)
            ph_f3p ^= 1u;
            ph_f3m ^= 1u;
        }
        tc::mma_commit_multicast_warp(&bars.a3_free, 0x3);
        tc::mma_commit_warp(&bars.fdone[fbuf]);
    }
}
#undef DGFS_WAITW
#undef DGFS_WAITWC

// PAD: f and P_r on an nsrc^3 grid, nsrc < N (N = 24 on the 32-point tiles: the filters are zero
// outside the nsrc x nsrc block, f is read with zeros outside it and only the nsrc^3 block of P_r is
// written).
template <int N, bool BF, bool PAD>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Geo3<N>::THREADS, 1)
k_tc3_gain(const float* __restrict__ f, const int64_t* __restrict__ offs, const unsigned char* __restrict__ filt,
           int npairs, int Nrho, int rpc, int nsrc, float* __restrict__ P, int* __restrict__ flags, int fault,
           const float* __restrict__ coef, int accum) {
    using G = Geo3<N>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) Bars3 bars;
    __shared__ uint32_t s_tmem;
    __shared__ float s_red[G::EPI_WARPS];
    __shared__ int s_abort;
    volatile int* abort = &s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == G::ISSUER;
    const uint32_t crank = tc::cluster_rank();   // front y-tiles and back x'-tiles [crank TH, crank TH + TH)
    const int r0 = (blockIdx.x >> 1) * rpc, nseq = npairs * rpc;
    const int64_t node = blockIdx.y;
    constexpr int64_t n3 = (int64_t)N * N * N;
    const int64_t n3s = PAD ? (int64_t)nsrc * nsrc * nsrc : n3;
    const float* fb = f + (offs ? offs[node] : node * n3s);
    const uint32_t sb = tc::smem_u32(smem);
    const unsigned char* fglob = filt + (size_t)r0 * npairs * G::F_BLOCK;

    int copies0 = nseq > 0 ? 1 : 0, copies1 = nseq > 1 ? 1 : 0, waited0 = 0, waited1 = 0;

    if (issuer) {
        if (lane == 0) {
            tc::mbar_init(&bars.full1, 1);
            tc::mbar_init(&bars.free1, 256);      // both epilogue warpgroups (one sign each)
            for (int i = 0; i < 2; ++i) {
                tc::mbar_init(&bars.a2_full[i], 128);
                tc::mbar_init(&bars.a2_free[i], 1);
            }
            for (int i = 0; i < 2; ++i) {
                tc::mbar_init(&bars.full2[i], 1);
                tc::mbar_init(&bars.free2[i], 256);
                tc::mbar_init(&bars.full3p[i], 1);
                tc::mbar_init(&bars.free3p[i], 128);
                tc::mbar_init(&bars.full3m[i], 1);
                tc::mbar_init(&bars.free3m[i], 128);
                tc::mbar_init(&bars.free3x[i], 128);
                tc::mbar_init(&bars.filt[i], 1);
                tc::mbar_init(&bars.fdone[i], 4);
            }
            // the epilogue threads of this CTA whose pass-3 rows are here; the peer's rows arrive as
            // st.async bytes (expect_tx registered by one of these arrivals)
            tc::mbar_init(&bars.a3_full, 128);
            tc::mbar_init(&bars.a3_free, 4);     // the pass-3 MMA warps of both CTAs
            tc::mbar_init(&bars.drain, 4);
            tc::fence_mbar_init();
            s_abort = 0;
            for (int p = 0; p < 2 && p < nseq; ++p) {
                tc::mbar_expect_tx(&bars.filt[p], G::F_BLOCK);
                tc::bulk_g2s(smem + G::S_F + p * G::F_BLOCK, fglob + (size_t)p * G::F_BLOCK, G::F_BLOCK, &bars.filt[p]);
            }
        }
        __syncwarp();
        tc::tmem_alloc(&s_tmem, G::TMEM_COLS);
    } else if (!BF && warp < G::EPI_WARPS) {
        constexpr int STRIDE = 32 * G::EPI_WARPS, PER = (int)(n3 / STRIDE);
        static_assert(n3 % STRIDE == 0 && PER % 8 == 0, "scan split");
        float m8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) m8[j] = 0.f;
        if constexpr (!PAD) {
#pragma unroll
            for (int i = 0; i < PER; ++i) m8[i & 7] = fmaxf(m8[i & 7], fabsf(__ldg(fb + tid + i * STRIDE)));
        } else {
            for (int64_t i0 = tid; i0 < n3s; i0 += 8 * STRIDE)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (i0 + j * STRIDE < n3s) m8[j] = fmaxf(m8[j], fabsf(__ldg(fb + i0 + j * STRIDE)));
        }
        float mx = fmaxf(fmaxf(fmaxf(m8[0], m8[1]), fmaxf(m8[2], m8[3])), fmaxf(fmaxf(m8[4], m8[5]), fmaxf(m8[6], m8[7])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_red[warp] = mx;
    }
    tc::tc_fence_before();
    // both CTAs' barriers are initialised before any arrive from the peer (and the set-up is done)
    tc::cluster_sync();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;

    float sf = 1.f;
    if (!BF) {
        float mx = s_red[0];
#pragma unroll
        for (int i = 1; i < G::EPI_WARPS; ++i) mx = fmaxf(mx, s_red[i]);
        if (mx > 0.f && isfinite(mx)) sf = exp2f(fminf(60.f, fmaxf(-60.f, floorf(log2f(2.f / mx)))));
    }
    // 2^-e, the weight of the lo parts, as a pair for the packed FMAs
    const float2 eps2 = make_float2(exp2f(-(float)(BF ? kLoShiftBF16 : kLoShiftF16)),
                                    exp2f(-(float)(BF ? kLoShiftBF16 : kLoShiftF16)));
    const float out_scale = 1.f / (sf * sf);

    // ---- f -> TMEM (f_hi, f_lo) for the front tiles i: y-tile t = crank TH + i, lane l = yl N + z --
    if (warp < G::EPI_WARPS) {
        const int q = warp & 3, w = warp >> 2, l = 32 * q + lane, yl = l / N, z = l % N;
#pragma unroll 1
        for (int i = w; i < G::TH; i += 2) {
            const int t = (int)crank * G::TH + i;
            uint32_t hi[N / 2], lo[N / 2];
            if constexpr (!PAD) {
                const float* src = fb + (size_t)(t * G::ZT + yl) * N + z;
#pragma unroll
                for (int c = 0; c < N / 2; ++c)
                    split2<BF>(__ldg(src + (size_t)(2 * c) * G::N2) * sf, __ldg(src + (size_t)(2 * c + 1) * G::N2) * sf,
                               hi[c], lo[c]);
            } else {   // zeros outside the nsrc^3 block
                const int y = t * G::ZT + yl;
                const bool in = y < nsrc && z < nsrc;
                const float* src = fb + ((size_t)y * nsrc + z);
                const size_t sx = (size_t)nsrc * nsrc;
#pragma unroll
                for (int c = 0; c < N / 2; ++c) {
                    const float a = in && 2 * c < nsrc ? __ldg(src + (size_t)(2 * c) * sx) * sf : 0.f;
                    const float b = in && 2 * c + 1 < nsrc ? __ldg(src + (size_t)(2 * c + 1) * sx) * sf : 0.f;
                    split2<BF>(a, b, hi[c], lo[c]);
                }
            }
            const uint32_t lanebase = tmem + ((uint32_t)(32 * q) << 16);
            if constexpr (N == 32) {
                tc::tmem_st16(lanebase + G::C_FH + i * (N / 2), hi);
                tc::tmem_st16(lanebase + G::C_FL + i * (N / 2), lo);
            } else {
                tc::tmem_st8(lanebase + G::C_FH + i * (N / 2), hi);
                tc::tmem_st8(lanebase + G::C_FL + i * (N / 2), lo);
            }
        }
        tc::tmem_wait_st();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp >= G::EPI_WARPS) {
        tc::setmaxnreg_dec<G::REG_MMA>();
        if (warp == G::ISSUER)
            mma3_p1_loop<N, BF>(bars, smem, sb, tmem, fglob, nseq, abort, copies0, copies1, waited0, waited1);
        else if (warp == G::ISSUER + 1)
            mma3_p2_loop<N, BF>(bars, sb, tmem, nseq, abort);
        else if (warp == G::ISSUER + 2)
            mma3_p3_loop<N, BF, 0>(bars, sb, tmem, nseq, abort);
        else
            mma3_p3_loop<N, BF, 1>(bars, sb, tmem, nseq, abort);
    } else {
        tc::setmaxnreg_inc<G::REG_EPI>();
        // warpgroup w: the epilogues of sign w (w = 0: +s, 1: -s) and the back tiles k = w, w + 2, ...
        const int q = warp & 3, w = warp >> 2;
        const int l = 32 * q + lane, yl = l / N, lz = l % N;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        // pass-2 operand row of this thread (pass-1 lane (yl, z = lz)) in the sign-w region: rows yl N + x', k = z
        const uint32_t a2_row = sb + G::S_A2 + w * 2 * G::A2_BYTES + ((uint32_t)(yl * N) >> 3) * G::A2_SBO +
                                (lz >> 3) * G::A2_LBO + (lz & 7) * 16;
        // pass-3 operand rows of this thread (pass-2 lane (yl, x' = lz)): rows x' N + z' in the CTA that owns
        // x' (its x'-tile (x' N) / 128), sign-w region, as shared::cluster addresses
        const int owner = (lz * N) / (128 * G::TH), ul = (lz * N) / 128 - owner * G::TH;
        const uint32_t a3_dst = tc::map_peer(sb + G::S_A3 + w * 2 * G::A3_BYTES + ul * G::A3_TS, (uint32_t)owner);
        const int rg0 = ((lz * N) & 127) >> 3;   // row group of z' = 0 within the tile
        const bool remote = owner != (int)crank;   // this thread's pass-3 rows live in the peer
        const uint32_t a3full_owner = tc::map_peer(tc::smem_u32(&bars.a3_full), (uint32_t)owner);
        // the first local thread registers the bytes the peer sends with its arrival
        const bool a3_expect = warp == 0 && lane == (crank ? N / 2 : 0);
        uint32_t ph_f1 = 0, ph_a2free = 0, ph_a3free = 0, ph_f2 = 0, ph_f3p = 0, ph_f3m = 0;   // ph_f2: bit per slot
        int p1uses = 0;
        constexpr int NB = (G::TH + 1) / 2;   // back tiles of one warpgroup
        float2 acc[NB][N / 2];   // P_r of the warpgroup's back tiles: (y' = 2j, 2j + 1) per entry
#pragma unroll
        for (int k = 0; k < NB; ++k)
#pragma unroll
            for (int j = 0; j < N / 2; ++j) acc[k][j] = make_float2(0.f, 0.f);
#define DGFS_WAITE(bar, ph)                                             \
    do {                                                                \
        if (!tc::warp_wait((bar), (ph), abort)) goto epi_done;          \
    } while (0)
#define DGFS_WAITEC(bar, ph)                                            \
    do {                                                                \
        if (!tc::warp_wait_cluster((bar), (ph), abort)) goto epi_done;  \
    } while (0)
        for (int rr = 0; rr < rpc; ++rr) {
          for (int pp = 0; pp < npairs; ++pp) {
            const int p = rr * npairs + pp;
            // front, software-pipelined over the front tiles: pass-1 epilogue of tile s, then the pass-2
            // epilogue of tile s - 1 (whose pass-2 MMAs ran meanwhile)
            for (int st = 0; st <= G::TH; ++st) {
                if (st < G::TH) {   // pass-1 result (sign w) of front tile st -> pass-2 operands
                    DGFS_WAITE(&bars.full1, ph_f1);
                    ph_f1 ^= 1u;
                    tc::tc_fence_after();
                    float hv[N], lv[N];
#pragma unroll
                    for (int c = 0; c < N / 16; ++c) {
                        tc::tmem_ld16(trow + G::C_P1 + w * N + 16 * c, *reinterpret_cast<float(*)[16]>(&hv[16 * c]));
                        tc::tmem_ld16(trow + G::C_P1 + 2 * N + w * N + 16 * c, *reinterpret_cast<float(*)[16]>(&lv[16 * c]));
                    }
                    tc::tmem_wait_ld();
                    tc::tc_fence_before();
                    tc::mbar_arrive(&bars.free1);
                    if (p1uses > 0) {   // pass 2 of the previous tile has read this sign's operands
                        DGFS_WAITE(&bars.a2_free[w], ph_a2free);
                        ph_a2free ^= 1u;
                    }
#pragma unroll
                    for (int c = 0; c < N / 8; ++c) {   // 8 columns x' = 8c .. 8c + 7
                        uint32_t uh[4], ulo[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                        {
                            const float2 v = tc::ffma2(make_float2(lv[8 * c + 2 * j], lv[8 * c + 2 * j + 1]), eps2,
                                                       make_float2(hv[8 * c + 2 * j], hv[8 * c + 2 * j + 1]));
                            split2<BF>(v.x, v.y, uh[j], ulo[j]);
                        }
                        tc::st_shared_v4(a2_row + c * G::A2_SBO, uh[0], uh[1], uh[2], uh[3]);
                        tc::st_shared_v4(a2_row + G::A2_BYTES + c * G::A2_SBO, ulo[0], ulo[1], ulo[2], ulo[3]);
                    }
                    tc::fence_proxy_async();
                    tc::mbar_arrive(&bars.a2_full[w]);
                    ++p1uses;
                }
                if (st >= 1) {   // pass-2 result (sign w) of front tile i = st - 1 -> pass-3 operand rows
                    const int i = st - 1, b = i & 1, y = ((int)crank * G::TH + i) * G::ZT + yl;
                    if (i == 0 && p > 0) {   // both CTAs' pass 3 of the previous pair has read the operands
                        DGFS_WAITEC(&bars.a3_free, ph_a3free);
                        ph_a3free ^= 1u;
                    }
                    DGFS_WAITE(&bars.full2[b], (ph_f2 >> b) & 1u);
                    ph_f2 ^= 1u << b;
                    tc::tc_fence_after();
                    const uint32_t ts = trow + (b ? G::C_S3 : G::C_S2) + w * 2 * N;
                    const uint32_t ky = (y >> 3) * G::A3_LBO + (y & 7) * 16;
#pragma unroll
                    for (int cc = 0; cc < N / 16; ++cc) {   // 16 columns z' behind one wait
                        float hv[16], lv[16];
                        tc::tmem_ld16(ts + 16 * cc, hv);
                        tc::tmem_ld16(ts + N + 16 * cc, lv);
                        tc::tmem_wait_ld();
                        if (cc == N / 16 - 1) {
                            tc::tc_fence_before();
                            tc::mbar_arrive(&bars.free2[b]);
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {   // 8 columns z' = 16 cc + 8 h ..: one row group
                            uint32_t uh[4], ulo[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                            {
                                const float2 v = tc::ffma2(make_float2(lv[8 * h + 2 * j], lv[8 * h + 2 * j + 1]), eps2,
                                                           make_float2(hv[8 * h + 2 * j], hv[8 * h + 2 * j + 1]));
                                split2<BF>(v.x, v.y, uh[j], ulo[j]);
                            }
                            const uint32_t o = a3_dst + (rg0 + 2 * cc + h) * G::A3_SBO + ky;
                            if (remote) {   // non-blocking, counted on the owner's a3_full
                                tc::st_async_v4(o, uh[0], uh[1], uh[2], uh[3], a3full_owner);
                                tc::st_async_v4(o + G::A3_BYTES, ulo[0], ulo[1], ulo[2], ulo[3], a3full_owner);
                            } else {
                                tc::st_cluster_v4(o, uh[0], uh[1], uh[2], uh[3]);
                                tc::st_cluster_v4(o + G::A3_BYTES, ulo[0], ulo[1], ulo[2], ulo[3]);
                            }
                        }
                    }
                }
            }
            // this warpgroup's rows of the pair are written: a thread whose rows are local makes them
            // visible to its tensor core and arrives (the first one with the bytes the peer sends);
            // rows sent to the peer are counted there as st.async bytes
            if (!remote) {
                tc::fence_proxy_async();
                if (!(fault == 1 && p == 0 && blockIdx.x == 0 && blockIdx.y == 0)) {
                    if (a3_expect) tc::mbar_expect_tx(&bars.a3_full, G::A3_REMOTE_BYTES);
                    else tc::mbar_arrive(&bars.a3_full);
                }
            }
            // back: pass-3 tiles k = w, w + 2, ... in slot 2 + w, products of the two translates
            const uint32_t tB = trow + (w ? G::C_S3 : G::C_S2);
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                const int k = w + 2 * n;   // warp-uniform
                if (k >= G::TH) break;
                // + half (every column behind one wait), released before the - half is awaited
                DGFS_WAITE(&bars.full3p[w], ph_f3p);
                ph_f3p ^= 1u;
                tc::tc_fence_after();
                float2 xp[N / 2];   // + translate at y' = 2j, 2j + 1
                {
                    float hp[N / 16][16], lp[N / 16][16];
#pragma unroll
                    for (int c = 0; c < N / 16; ++c) {
                        tc::tmem_ld16(tB + 16 * c, hp[c]);
                        tc::tmem_ld16(tB + N + 16 * c, lp[c]);
                    }
                    tc::tmem_wait_ld();
                    tc::tc_fence_before();
                    tc::mbar_arrive(&bars.free3p[w]);
#pragma unroll
                    for (int c = 0; c < N / 16; ++c)
#pragma unroll
                        for (int j = 0; j < 8; ++j)   // two y' per packed FMA, the same roundings as fmaf
                            xp[8 * c + j] = tc::ffma2(make_float2(lp[c][2 * j], lp[c][2 * j + 1]), eps2,
                                                      make_float2(hp[c][2 * j], hp[c][2 * j + 1]));
                }
                DGFS_WAITE(&bars.full3m[w], ph_f3m);
                ph_f3m ^= 1u;
                tc::tc_fence_after();
#pragma unroll
                for (int c = 0; c < N / 16; ++c) {   // - half: 16 columns y' behind one wait
                    float hm[16], lm[16];
                    tc::tmem_ld16(tB + 2 * N + 16 * c, hm);
                    tc::tmem_ld16(tB + 3 * N + 16 * c, lm);
                    tc::tmem_wait_ld();
                    if (c == N / 16 - 1) {
                        tc::tc_fence_before();
                        tc::mbar_arrive(&bars.free3m[w]);
                        if (k + 2 >= G::TH) tc::mbar_arrive(&bars.free3x[w]);
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float2 xm = tc::ffma2(make_float2(lm[2 * j], lm[2 * j + 1]), eps2,
                                                    make_float2(hm[2 * j], hm[2 * j + 1]));
                        acc[n][8 * c + j] = tc::ffma2(xp[8 * c + j], xm, acc[n][8 * c + j]);
                    }
                }
            }
          }
          // radial point r0 + rr done: P_r of this warpgroup's back tiles out, sums cleared
          if (!*abort) {
              float* dst = P + ((size_t)node * Nrho + r0 + rr) * n3s;
              const float sc = out_scale * (coef ? coef[node] : 1.f);   // per-node factor (polarisation)
#pragma unroll
              for (int n = 0; n < NB; ++n) {
                  const int k = w + 2 * n;
                  if (k >= G::TH) break;
                  const int m3 = ((int)crank * G::TH + k) * 128 + l, xp = m3 / N, zp = m3 % N;
                  if constexpr (!PAD) {
                      float* o = dst + (size_t)xp * G::N2 + zp;
#pragma unroll
                      for (int j = 0; j < N; ++j) {
                          const float a = (j & 1) ? acc[n][j / 2].y : acc[n][j / 2].x;
                          if (accum) o[(size_t)j * N] += a * sc;
                          else o[(size_t)j * N] = a * sc;
                      }
                  } else if (xp < nsrc && zp < nsrc) {   // the nsrc^3 block only
                      float* o = dst + (size_t)xp * nsrc * nsrc + zp;
#pragma unroll
                      for (int j = 0; j < N; ++j) {
                          if (j >= nsrc) continue;
                          const float a = (j & 1) ? acc[n][j / 2].y : acc[n][j / 2].x;
                          if (accum) o[(size_t)j * nsrc] += a * sc;
                          else o[(size_t)j * nsrc] = a * sc;
                      }
                  }
              }
          }
#pragma unroll
          for (int k = 0; k < NB; ++k)
#pragma unroll
              for (int j = 0; j < N / 2; ++j) acc[k][j] = make_float2(0.f, 0.f);
        }
#undef DGFS_WAITE
#undef DGFS_WAITEC
    epi_done:;
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp >= G::ISSUER) {
        if (tc::elect_one()) tc::mma_commit(&bars.drain);
        __syncwarp();
    }
    if (issuer) {
        if (tc::elect_one()) {
            if (*abort) atomicOr(flags, 1);
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
    // no CTA leaves while its peer may still write its shared memory, arrive on its barriers or
    // have its multicast commits land there
    tc::cluster_sync();
}

template <int N, bool BF>
cudaError_t launch3_n(const TcTables& t, const float* f, const int64_t* offs, int64_t nodes, float* P, int* flags,
                      cudaStream_t s, int fault, const float* coef, int accum) {
    using G = Geo3<N>;
    const int nsrc = t.nsrc > 0 ? t.nsrc : N;
    auto kern = nsrc == N ? k_tc3_gain<N, BF, false> : k_tc3_gain<N, BF, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::S_TOTAL);
    if (e != cudaSuccess) return e;
    const int64_t n3 = (int64_t)nsrc * nsrc * nsrc;   // f and P_r grid
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // radial points per CTA pair (tc_resolve_rpc: two CTAs per radial block)
    const int rpc = tc_resolve_rpc(t, BF ? DGFS_PREC_BF16X3 : DGFS_PREC_F16X3, nodes, sms);
    for (int64_t n0 = 0; n0 < nodes; n0 += 65535) {
        const int64_t nn = nodes - n0 < 65535 ? nodes - n0 : 65535;
        kern<<<dim3(2 * (t.Nrho / rpc), (unsigned)nn), G::THREADS, G::S_TOTAL, s>>>(
            f + (offs ? 0 : n0 * n3), offs ? offs + n0 : nullptr, static_cast<const unsigned char*>(t.mats),
            t.npairs, t.Nrho, rpc, nsrc, P + n0 * t.Nrho * n3, flags, n0 == 0 ? fault : 0, coef ? coef + n0 : nullptr,
            accum);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

uint16_t f16_bits(double x) {
    const __half h = __double2half(x);
    uint16_t b;
    std::memcpy(&b, &h, 2);
    return b;
}
double f16_value(uint16_t b) {
    __half h;
    std::memcpy(&h, &b, 2);
    return (double)__half2float(h);
}
uint16_t bf16_bits(double x) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    uint16_t b;
    std::memcpy(&b, &h, 2);
    return b;
}
double bf16_value(uint16_t b) {
    __nv_bfloat16 h;
    std::memcpy(&h, &b, 2);
    return (double)__bfloat162float(h);
}

}  // namespace

bool tc3_precision(int prec) { return prec == DGFS_PREC_F16X3 || prec == DGFS_PREC_BF16X3; }

size_t build_tc3_tables(const HostPlan& hp, int prec, std::vector<unsigned char>& blob, TcTables& t) {
    // N = 24 runs on the 32-point tiles: each 24-point circulant sits in the top-left block of a
    // zero 32 x 32 matrix, so the padded passes give the 24-point translates of the zero-padded field
    const int Nd = hp.N, N = Nd == 24 ? 32 : Nd, np = hp.npairs, Nr = hp.Nrho;
    const bool bf = prec == DGFS_PREC_BF16X3;
    const double ls = std::ldexp(1.0, bf ? kLoShiftBF16 : kLoShiftF16);
    const size_t sbytes = (size_t)2 * N * N * 2, block = 6 * sbytes;
    blob.assign((size_t)Nr * np * block, 0);
    const size_t sbo = 16 * (size_t)N, lbo = 128;
    auto put = [&](unsigned char* base, int n, int k, uint16_t bits) {
        std::memcpy(base + (n / 8) * sbo + (k / 8) * lbo + (n % 8) * 16 + (k % 8) * 2, &bits, 2);
    };
    for (int r = 0; r < Nr; ++r)
        for (int p = 0; p < np; ++p) {
            unsigned char* blk = blob.data() + ((size_t)r * np + p) * block;
            // F_+[i][j] = a[(i - j) mod N] (translate by +s along the axis); F_- = F_+^T (T_-s = T_s^T)
            auto F = [&](int axis, int sign, int i, int j) {
                if (i >= Nd || j >= Nd) return 0.0;
                const double* fl = &hp.filt[(((size_t)r * np + p) * 3 + axis) * Nd];
                const int d = sign == 0 ? i - j : j - i;
                return fl[((d % Nd) + Nd) % Nd];
            };
            const double w2 = 2.0 * hp.wsig[p];
            for (int sign = 0; sign < 2; ++sign)
                for (int i = 0; i < N; ++i)
                    for (int j = 0; j < N; ++j) {
                        uint16_t hi, lo;
                        auto split = [&](double v) {
                            hi = bf ? bf16_bits(v) : f16_bits(v);
                            const double hv = bf ? bf16_value(hi) : f16_value(hi);
                            lo = bf ? bf16_bits((v - hv) * ls) : f16_bits((v - hv) * ls);
                        };
                        // B1 (x, axis 0): rows [F+hi; F-hi; F+lo; F-lo]; the + filter carries 2 w_p
                        split(F(0, sign, i, j) * (sign == 0 ? w2 : 1.0));
                        put(blk, sign * N + i, j, hi);
                        put(blk, (2 + sign) * N + i, j, lo);
                        // B2 (z, axis 2) and B3 (y, axis 1): per sign [hi; lo]
                        split(F(2, sign, i, j));
                        put(blk + (2 + sign) * sbytes, i, j, hi);
                        put(blk + (2 + sign) * sbytes, N + i, j, lo);
                        split(F(1, sign, i, j));
                        put(blk + (4 + sign) * sbytes, i, j, hi);
                        put(blk + (4 + sign) * sbytes, N + i, j, lo);
                    }
        }
    t.N = N;
    t.nsrc = Nd;
    t.Nrho = Nr;
    t.npairs = np;
    t.mats = reinterpret_cast<const void*>((uintptr_t)0);
    return blob.size();
}

cudaError_t launch_tc3_gain_products(const TcTables& t, int prec, const float* f, const int64_t* offs, int64_t nodes,
                                     float* P, int* flags, cudaStream_t s, int fault, const float* coef, int accumulate) {
    if (nodes <= 0) return cudaSuccess;
    const bool bf = prec == DGFS_PREC_BF16X3;
    switch (t.N) {
        case 16: return bf ? launch3_n<16, true>(t, f, offs, nodes, P, flags, s, fault, coef, accumulate)
                           : launch3_n<16, false>(t, f, offs, nodes, P, flags, s, fault, coef, accumulate);
        case 32: return bf ? launch3_n<32, true>(t, f, offs, nodes, P, flags, s, fault, coef, accumulate)
                           : launch3_n<32, false>(t, f, offs, nodes, P, flags, s, fault, coef, accumulate);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dgfs
