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
// split into a hi and a lo 16-bit part. Pass 1 stacks the two signs along the MMA's N dimension
// (N = 2 n) and accumulates hi and lo in the same accumulator (two MMAs; both parts carry 2^8 in
// fp16, undone in the epilogue); its A operand comes from TMEM, so these MMAs are compute-bound.
// Passes 2 and 3 stack {hi, lo} of one sign along N (N = 2 n): one MMA per K step reads the
// shared-memory A operand once, and the epilogue combines hi + 2^-e lo in FP32. The + sign's x
// filter carries the factor 2 w_p, so the products need no further weighting.
//
// Persistent: one CTA per SM pulls work items (a node and rpc consecutive radial points) from a
// queue counter in global memory until none are left; the pass-1 MMA warp claims them and hands
// each one to the other warps through a ring in shared memory. Per item the epilogue warps scale f
// and load it into TMEM (once the previous item's pass-1 MMAs are complete); the (radial point,
// pair) steps of consecutive items form one pipelined sequence. Each CTA holds two epilogue
// warpgroups and a third warpgroup of four MMA warps (after set-up the third warpgroup gives
// registers back and the epilogue warpgroups take them, 216 per thread, so that an epilogue step
// loads a whole tile row from TMEM behind one wait). The front of a sphere pair (passes 1 and 2 of every tile) is a producer/consumer chain:
// the pass-1 MMA warp fills two pass-1 TMEM slots, epilogue warpgroup 0 turns each pass-1 result
// into pass-2 operands in two shared-memory buffers, the pass-2 MMA warp fills two pass-2/3 TMEM
// slots, and epilogue warpgroup 1 writes each pass-2 result into the pass-3 operands (both signs'
// full fields, in shared memory); every ring is two deep, so consecutive tiles overlap. The back
// (pass 3) starts once every pass-2 tile is stored: pass-3 MMA warp b fills slot b with the tiles
// u = b (mod 2), and epilogue warpgroup b forms their products (one TMEM lane per thread); the two
// signs' halves of the slot are handed over separately, so the + MMAs of the next tile overlap
// the read of the - half and the products. While
// it waits for the pass-3 operands, warpgroup 0 already turns the first two pass-1 tiles of the
// next step of the item into pass-2 operands (N = 32), so the next front starts two tiles in.
// Barriers shared by several MMA warps (filter buffer done, final drain, pass-3 operands released)
// take one commit from each warp that uses the resource. All hand-offs
// are mbarriers; every lane of the epilogue warps arrives and every wait loop branches on warp
// votes only, so no branch diverges around the .sync.aligned tcgen05 instructions. Every wait is
// bounded: on timeout the CTA raises flag bit 0, every role stops, the MMAs and copies in flight
// are drained (bounded), TMEM is freed and no further P_r is written (the flag marks P invalid).
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_gain.h"
#include "tc_ptx.cuh"

namespace dgfs {

namespace {

// fp16 filters: pass 1 stores hi and lo times 2^8, passes 2 and 3 store lo times 2^11 (both keep
// the lo parts normal); bf16 has the exponent range and stores pass-2/3 lo parts times 2^8
constexpr int kP1ShiftF16 = 8;
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
    static constexpr int TW = T / 2;              // tiles per epilogue warpgroup
    static constexpr int EPI_WARPS = 8;           // epilogue warpgroups 0 and 1 (warp / 4)
    static constexpr int THREADS = 32 * EPI_WARPS + 128;   // + a warpgroup holding the MMA warp
    static constexpr int ISSUER = EPI_WARPS;      // first MMA warp (pass 1); then pass 2, pass 3 of slots 0, 1
    // pass-1 tiles of the next step that warpgroup 0 turns into pass-2 operands while it waits for
    // the pass-3 operands of the current one (at most the two operand buffers; none when a step
    // has only two tiles)
    static constexpr int LOOKAHEAD = T >= 4 ? 2 : 0;
    // registers per thread: 168 at launch (65536 / 384, rounded down to a multiple of 8), then
    // 216 for the epilogue warpgroups and 72 for the third: 256 * 216 + 128 * 72 = 384 * 168
    static constexpr uint32_t REG_LAUNCH = 168, REG_EPI = 216, REG_MMA = 72;
    static_assert(256 * REG_EPI + 128 * REG_MMA <= 384 * REG_LAUNCH, "register reallocation exceeds the pool");
    // filter block of one (r, pair), K-major B operands: row n, column k at
    // (n/8) FB_SBO + (k/8) FB_LBO + (n%8) 16 + (k%8) 2. B1 rows: +hi, -hi, +lo, -lo (n each);
    // B2 and B3, per sign: hi, lo (n each)
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
    // TMEM columns: pass-1 slots 0, 1 (2 N columns: + then -), pass-2/3 slots 2, 3 (4 N columns:
    // +hi, +lo, -hi, -lo), then f (N/2 columns per tile); slots 0 and 2 belong to warpgroup 0
    static constexpr uint32_t C_S0 = 0, C_S1 = 2 * N, C_S2 = 4 * N, C_S3 = 8 * N;
    static constexpr uint32_t C_F = 12 * N, F_COLS = T * (N / 2);
    static constexpr uint32_t C_USED = C_F + F_COLS;
    static constexpr uint32_t TMEM_COLS = C_USED <= 32 ? 32 : C_USED <= 64 ? 64 : C_USED <= 128 ? 128
                                          : C_USED <= 256 ? 256 : 512;
    static_assert(C_USED <= 512, "TMEM budget");
    // shared memory: A2 [slot 2][sign 2], A3 [sign 2], filters [buffer 2]
    static constexpr uint32_t S_A2 = 0, S_A3 = S_A2 + 4 * A2_BYTES;
    static constexpr uint32_t S_F = (S_A3 + 2 * A3_BYTES + 127) / 128 * 128;
    static constexpr uint32_t S_TOTAL = S_F + 2 * F_BLOCK;
    static_assert(S_TOTAL + 512 <= 232448, "shared-memory budget");
    static_assert(A3_TS % 16 == 0 && A2_BYTES % 16 == 0 && A3_BYTES % 16 == 0 && F_BLOCK % 16 == 0 &&
                  S_A3 % 16 == 0 && S_F % 16 == 0, "descriptor offsets are multiples of 16 bytes");
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

// Work items of the persistent kernel: item i = (node i / rblocks, radial points
// r0 .. r0 + rpc - 1 with r0 = (i % rblocks) rpc), pulled from a queue counter in global memory.
// The pass-1 MMA warp claims them and publishes each one in a ring in shared memory, which every
// other warp reads in the same order.
constexpr int kRing = 4;
constexpr uint32_t kRingConsumers = 8 + 3;   // the eight epilogue warps, the pass-2 and pass-3 MMA warps

struct Items {
    int64_t n_items;   // nodes * rblocks
    int rblocks;       // radial blocks per node (N_rho / rpc)
    int rpc;           // radial points per item
    int nseq;          // (radial point, pair) steps per item: rpc * npairs
};

struct Bars {
    // TMEM slot rings (index = tile % 2): MMA completion -> epilogue, epilogue drained -> MMA
    uint64_t full1[2], free1[2];       // pass-1 slots (pass-1 epilogue, warpgroup 0)
    uint64_t full2[2], free2[2];       // pass-2/3 slots used by pass 2 (pass-2 epilogue, warpgroup 1)
    uint64_t full3p[2], free3p[2];     // pass-2/3 slots used by pass 3 (warpgroup = slot): + sign columns
    uint64_t full3m[2], free3m[2];     // and - sign columns, each half released as soon as it is read
    uint64_t free3x[2];                // last pass-3 drain of a slot in a pair (next pair's pass 2 may start)
    uint64_t a2_full[2], a2_free[2];   // pass-2 operand ring: epilogue -> MMA, MMA completion -> epilogue
    uint64_t a3_full, a3_free;         // pass-3 operands (both signs)
    uint64_t filt[2], fdone[2];        // filter buffers: copy landed; all MMAs of the step using it done
    uint64_t item_full[kRing], item_free[kRing];   // work-item ring: published; read by every consumer warp
    uint64_t f_ready, f_free;          // f of the current item in TMEM; pass-1 MMAs of an item complete
    uint64_t scan[2];                  // max |f| partial maxima of an item written (item % 2)
    uint64_t drain;
};

template <bool BF>
__device__ __forceinline__ void pack8(const float (&v)[8], uint32_t (&u)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = pack2<BF>(v[2 * j], v[2 * j + 1]);
}

// The MMA warps (four, converged). Pass 1 of every tile (mma_p1_loop; it also claims the work items
// and refills the filter buffers), pass 2 of every tile (mma_p2_loop) and pass 3 of the tiles of
// warpgroup b (mma_p3_loop<b>) are issued by separate warps, so a group is issued as soon as its own
// inputs and slot are ready. Each commit tracks only the issuing warp's MMAs. The (radial point,
// pair) steps of consecutive items form one sequence; g counts them, and every phase below follows
// g, not the item. Each loop returns early when a wait gave up (abort).
#define DGFS_WAITW(bar, ph)                                             \
    do {                                                                \
        if (!tc::warp_wait((bar), (ph), abort)) return;                 \
    } while (0)

// Item k of this CTA from the ring (every consumer warp, in order); -1 ends the sequence.
__device__ __forceinline__ bool ring_take(Bars& bars, const volatile long long* s_item, int k, long long& item,
                                          volatile int* abort) {
    if (!tc::warp_wait(&bars.item_full[k % kRing], (uint32_t)((k / kRing) & 1), abort)) return false;
    item = s_item[k % kRing];
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&bars.item_free[k % kRing]);
    return true;
}

// The pass-1 warp claims this CTA's item k and publishes it (slot k % kRing, once its previous
// item has been read by every consumer).
__device__ __forceinline__ bool ring_claim(Bars& bars, volatile long long* s_item, int* queue, const Items& it, int k,
                                           long long& item, volatile int* abort) {
    if (k >= kRing && !tc::warp_wait(&bars.item_free[k % kRing], (uint32_t)((k / kRing - 1) & 1), abort)) return false;
    long long v = -1;
    if ((threadIdx.x & 31) == 0) {
        const long long c = atomicAdd(queue, 1);
        v = c < it.n_items ? c : -1;
        s_item[k % kRing] = v;
        tc::mbar_arrive(&bars.item_full[k % kRing]);
    }
    item = __shfl_sync(0xffffffffu, v, 0);
    return true;
}

template <int N>
__device__ __forceinline__ const unsigned char* item_filters(const unsigned char* filt, long long item, const Items& it,
                                                             int npairs) {
    return filt + (size_t)((item % it.rblocks) * it.rpc) * npairs * Geo<N>::F_BLOCK;
}

template <int N, bool BF>
__device__ __forceinline__ void mma_p1_loop(Bars& bars, unsigned char* smem, uint32_t sb, uint32_t tmem,
                                            const unsigned char* filt, int npairs, const Items& it, long long first,
                                            volatile long long* s_item, int* queue, volatile int* abort,
                                            int& copies0, int& copies1, int& waited0, int& waited1) {
    using G = Geo<N>;
    uint32_t used = 0, ph_free = 0, ph_fdone = 0;   // bit masks (bit i = slot or buffer i)
    constexpr uint32_t id1 = tc::idesc_f16(BF, false, false, 2 * N, 128);
    constexpr uint64_t dF = tc::sdesc_base(G::FB_LBO, G::FB_SBO);
    const uint32_t sb16 = sb >> 4;
    long long cur = first;
    int64_t g = 0;
    for (int k = 0; cur >= 0; ++k) {
        // the next item is claimed now: its first filter block is copied during this item's last step
        long long nxt = -1;
        if (!ring_claim(bars, s_item, queue, it, k + 1, nxt, abort)) return;
        const unsigned char* fcur = item_filters<N>(filt, cur, it, npairs);
        const unsigned char* fnxt = nxt >= 0 ? item_filters<N>(filt, nxt, it, npairs) : nullptr;
        DGFS_WAITW(&bars.f_ready, (uint32_t)(k & 1));   // f of this item is in TMEM
        for (int s = 0; s < it.nseq; ++s, ++g) {
            const int fbuf = (int)(g & 1);
            DGFS_WAITW(&bars.filt[fbuf], (uint32_t)((g >> 1) & 1));
            if (fbuf) ++waited1;
            else ++waited0;
            tc::tc_fence_after();
            const uint32_t f16 = sb16 + (G::S_F + fbuf * G::F_BLOCK) / 16;   // filter block of this step
            for (int t = 0; t < G::T; ++t) {   // pass 1 of tile t into pass-1 slot t % 2
                const int b = t & 1;
                if (used & (1u << b)) {
                    DGFS_WAITW(&bars.free1[b], (ph_free >> b) & 1u);
                    ph_free ^= 1u << b;
                }
                used |= 1u << b;
                tc::tc_fence_after();
                const uint32_t d = tmem + b * G::C_S1;
                const uint32_t fa = tmem + G::C_F + t * (N / 2);
#pragma unroll
                for (int ks = 0; ks < G::KSTEPS; ++ks) {   // hi rows [0, 2n), lo rows [2n, 4n) of B1
                    tc::mma_ts_warp(d, fa + 8 * ks, tc::sdesc_at(dF, f16 + (G::OFF_B1 + ks * 2 * G::FB_LBO) / 16), id1, ks);
                    tc::mma_ts_warp(d, fa + 8 * ks,
                                    tc::sdesc_at(dF, f16 + (G::OFF_B1 + (2 * N / 8) * G::FB_SBO + ks * 2 * G::FB_LBO) / 16),
                                    id1, 1);
                }
                tc::mma_commit_warp(&bars.full1[b]);
                // the other filter buffer (step g - 1, whose MMAs are complete by now) takes step g + 1;
                // the set-up copied steps 0 and 1, unless step 1 belongs to the next item (one-step items).
                // With the epilogue's look-ahead the wait comes after tile 1: step g - 1 completes only
                // after warpgroup 0 has turned tiles 0 and 1 of step g into pass-2 operands.
                const unsigned char* src = s + 1 < it.nseq ? fcur + (size_t)(s + 1) * G::F_BLOCK : fnxt;
                if (t == (G::LOOKAHEAD ? 1 : 0) && (g >= 1 || it.nseq == 1) && src) {
                    const int nb = (int)((g + 1) & 1);
                    if (g >= 1) {   // buffer nb held step g - 1
                        DGFS_WAITW(&bars.fdone[nb], (ph_fdone >> nb) & 1u);
                        ph_fdone ^= 1u << nb;
                    }
                    if (tc::elect_one()) {
                        tc::mbar_expect_tx(&bars.filt[nb], G::F_BLOCK);
                        tc::bulk_g2s(smem + G::S_F + nb * G::F_BLOCK, src, G::F_BLOCK, &bars.filt[nb]);
                    }
                    __syncwarp();
                    if (nb) ++copies1;
                    else ++copies0;
                }
            }
            tc::mma_commit_warp(&bars.fdone[fbuf]);
        }
        tc::mma_commit_warp(&bars.f_free);   // f of this item may be replaced once these MMAs complete
        cur = nxt;
    }
}

// Pass 2 of tile t reads pass-2 operand buffer t % 2 and writes pass-2/3 slot t % 2. Slot b is
// reused within a step after the pass-2 epilogue drained it (free2, completions 0..2 of the step's
// four); the step's first use waits for the previous step's last pass-3 drain (free3x).
template <int N, bool BF>
__device__ __forceinline__ void mma_p2_loop(Bars& bars, uint32_t sb, uint32_t tmem, const Items& it,
                                            const volatile long long* s_item, volatile int* abort) {
    using G = Geo<N>;
    uint32_t ph_a2 = 0, ph_x = 0;
    constexpr uint32_t id23 = tc::idesc_f16(BF, true, false, 2 * N, 128);
    constexpr uint64_t dF = tc::sdesc_base(G::FB_LBO, G::FB_SBO);
    constexpr uint64_t dA2 = tc::sdesc_base(G::A2_LBO, G::A2_SBO);
    const uint32_t sb16 = sb >> 4;
    int64_t g = 0;
    for (int k = 0;; ++k) {
        long long item;
        if (!ring_take(bars, s_item, k, item, abort) || item < 0) return;
        for (int s = 0; s < it.nseq; ++s, ++g) {
            const int fbuf = (int)(g & 1);
            DGFS_WAITW(&bars.filt[fbuf], (uint32_t)((g >> 1) & 1));
            tc::tc_fence_after();
            const uint32_t f16 = sb16 + (G::S_F + fbuf * G::F_BLOCK) / 16;
            for (int t = 0; t < G::T; ++t) {
                const int b = t & 1, j = t >> 1;   // j-th use of slot b in this step
                DGFS_WAITW(&bars.a2_full[b], (ph_a2 >> b) & 1u);
                ph_a2 ^= 1u << b;
                if (j == 0) {
                    if (g > 0) {
                        DGFS_WAITW(&bars.free3x[b], (ph_x >> b) & 1u);
                        ph_x ^= 1u << b;
                    }
                } else {
                    DGFS_WAITW(&bars.free2[b], (uint32_t)((j - 1) & 1));   // four completions per step
                }
                tc::tc_fence_after();
                const uint32_t d = tmem + (b ? G::C_S3 : G::C_S2);
                const uint32_t a16 = sb16 + G::S_A2 / 16 + b * (2 * G::A2_BYTES / 16);
#pragma unroll
                for (int gs = 0; gs < 2; ++gs)
#pragma unroll
                    for (int ks = 0; ks < G::KSTEPS; ++ks)
                        tc::mma_ss_warp(d + gs * 2 * N,
                                        tc::sdesc_at(dA2, a16 + (gs * G::A2_BYTES + ks * 2 * G::A2_LBO) / 16),
                                        tc::sdesc_at(dF, f16 + (G::OFF_B2 + gs * G::B23_BYTES + ks * 2 * G::FB_LBO) / 16),
                                        id23, ks);
                tc::mma_commit_warp(&bars.full2[b]);
                tc::mma_commit_warp(&bars.a2_free[b]);
            }
            tc::mma_commit_warp(&bars.fdone[fbuf]);
        }
    }
}

// Pass 3 of the tiles u = 2k + b into slot b once every pass-2 tile is in shared memory (a3_full
// also orders every pass-2 drain of the slot before these MMAs). Each sign's half of the slot has
// its own completion (full3p / full3m) and release (free3p / free3m): the + MMAs of tile k + 1 wait
// only for the + half of tile k to be read, so they run while the epilogue reads the - half and
// forms the products (completions 0..2 of the step's four).
template <int N, bool BF, int b>
__device__ __forceinline__ void mma_p3_loop(Bars& bars, uint32_t sb, uint32_t tmem, const Items& it,
                                            const volatile long long* s_item, volatile int* abort) {
    using G = Geo<N>;
    uint32_t ph_a3full = 0;
    constexpr uint32_t id23 = tc::idesc_f16(BF, true, false, 2 * N, 128);
    constexpr uint64_t dF = tc::sdesc_base(G::FB_LBO, G::FB_SBO);
    constexpr uint64_t dA3 = tc::sdesc_base(G::A3_LBO, G::A3_SBO);
    const uint32_t sb16 = sb >> 4;
    int64_t g = 0;
    for (int ki = 0;; ++ki) {
        long long item;
        if (!ring_take(bars, s_item, ki, item, abort) || item < 0) return;
        for (int s = 0; s < it.nseq; ++s, ++g) {
            const int fbuf = (int)(g & 1);
            DGFS_WAITW(&bars.filt[fbuf], (uint32_t)((g >> 1) & 1));
            const uint32_t f16 = sb16 + (G::S_F + fbuf * G::F_BLOCK) / 16;
            DGFS_WAITW(&bars.a3_full, ph_a3full);
            ph_a3full ^= 1;
            tc::tc_fence_after();
            for (int k = 0; k < G::TW; ++k) {
                const int u = 2 * k + b;
                const uint32_t d = tmem + (b ? G::C_S3 : G::C_S2);
                const uint32_t a16 = sb16 + G::S_A3 / 16 + u * (G::A3_TS / 16);
#pragma unroll
                for (int gs = 0; gs < 2; ++gs) {   // sign +, then sign -
                    if (k > 0) {
                        DGFS_WAITW(gs ? &bars.free3m[b] : &bars.free3p[b], (uint32_t)((k - 1) & 1));   // four per step
                        tc::tc_fence_after();
                    }
#pragma unroll
                    for (int ks = 0; ks < G::KSTEPS; ++ks)
                        tc::mma_ss_warp(d + gs * 2 * N,
                                        tc::sdesc_at(dA3, a16 + (gs * G::A3_BYTES + ks * 2 * G::A3_LBO) / 16),
                                        tc::sdesc_at(dF, f16 + (G::OFF_B3 + gs * G::B23_BYTES + ks * 2 * G::FB_LBO) / 16),
                                        id23, ks);
                    tc::mma_commit_warp(gs ? &bars.full3m[b] : &bars.full3p[b]);
                }
            }
            tc::mma_commit_warp(&bars.a3_free);
            tc::mma_commit_warp(&bars.fdone[fbuf]);
        }
    }
}
#undef DGFS_WAITW

// Persistent: one CTA per SM pulls work items (node, block of rpc radial points) from the queue
// counter queue[0] (zero at launch) until the items run out. PAD: f and P_r on an nsrc^3 grid,
// nsrc < N (N = 24 on the 32-point tiles).
template <int N, bool BF, bool PAD>
__global__ void __launch_bounds__(Geo<N>::THREADS, 1)
k_tc_gain(const float* __restrict__ f, const int64_t* __restrict__ offs, const unsigned char* __restrict__ filt,
          int npairs, int Nrho, Items it, int nsrc, int* __restrict__ queue, float* __restrict__ P,
          int* __restrict__ flags, int fault, const float* __restrict__ coef, int accum) {
    using G = Geo<N>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) Bars bars;
    __shared__ uint32_t s_tmem;
    __shared__ float s_red[2][G::EPI_WARPS];
    __shared__ int s_abort;
    __shared__ long long s_item[kRing];
    volatile int* abort = &s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == G::ISSUER;
    constexpr int64_t n3 = (int64_t)N * N * N;
    // f and P_r live on an nsrc^3 grid: nsrc = N, or nsrc < N (N = 24 run on the 32-point tiles:
    // the filters are zero outside the nsrc x nsrc block, f is read with zeros outside it and only
    // the nsrc^3 block of P_r is written)
    const int64_t n3s = PAD ? (int64_t)nsrc * nsrc * nsrc : n3;
    constexpr bool padded = PAD;
    const uint32_t sb = tc::smem_u32(smem);

    // filter copies issued and waited per buffer 0 / 1 (used by the MMA warp and the drain)
    int copies0 = 0, copies1 = 0, waited0 = 0, waited1 = 0;
    long long first = -1;

    // ---- set-up: barriers, the first item and its first filter copies, TMEM (MMA warp) -----------
    if (issuer) {
        if (lane == 0) {
            for (int i = 0; i < 2; ++i) {
                tc::mbar_init(&bars.full1[i], 1);
                tc::mbar_init(&bars.free1[i], 128);
                tc::mbar_init(&bars.full2[i], 1);
                tc::mbar_init(&bars.free2[i], 128);
                tc::mbar_init(&bars.full3p[i], 1);
                tc::mbar_init(&bars.free3p[i], 128);
                tc::mbar_init(&bars.full3m[i], 1);
                tc::mbar_init(&bars.free3m[i], 128);
                tc::mbar_init(&bars.free3x[i], 128);
                tc::mbar_init(&bars.a2_full[i], 128);
                tc::mbar_init(&bars.a2_free[i], 1);
                tc::mbar_init(&bars.filt[i], 1);
                tc::mbar_init(&bars.fdone[i], 4);   // one commit from each MMA warp
            }
            for (int i = 0; i < kRing; ++i) {
                tc::mbar_init(&bars.item_full[i], 1);
                tc::mbar_init(&bars.item_free[i], kRingConsumers);
            }
            tc::mbar_init(&bars.f_ready, 256);      // the epilogue warpgroups
            tc::mbar_init(&bars.f_free, 1);
            tc::mbar_init(&bars.scan[0], G::EPI_WARPS);
            tc::mbar_init(&bars.scan[1], G::EPI_WARPS);
            tc::mbar_init(&bars.a3_full, 128);     // the pass-2 epilogue warpgroup
            tc::mbar_init(&bars.a3_free, 2);       // the two pass-3 MMA warps
            tc::mbar_init(&bars.drain, 4);
            tc::fence_mbar_init();
            s_abort = 0;
        }
        __syncwarp();
        ring_claim(bars, s_item, queue, it, 0, first, abort);   // slot 0: no wait
        if (lane == 0 && first >= 0) {
            const unsigned char* f0 = item_filters<N>(filt, first, it, npairs);
            for (int p = 0; p < 2 && p < it.nseq; ++p) {
                tc::mbar_expect_tx(&bars.filt[p], G::F_BLOCK);
                tc::bulk_g2s(smem + G::S_F + p * G::F_BLOCK, f0 + (size_t)p * G::F_BLOCK, G::F_BLOCK, &bars.filt[p]);
            }
        }
        __syncwarp();
        if (first >= 0) {
            copies0 = 1;
            copies1 = it.nseq > 1 ? 1 : 0;
        }
        tc::tmem_alloc(&s_tmem, G::TMEM_COLS);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp >= G::EPI_WARPS) {
      tc::setmaxnreg_dec<G::REG_MMA>();   // every warp of the third warpgroup
      // ============================ MMA warps (converged) =====================================
      if (warp == G::ISSUER)
        mma_p1_loop<N, BF>(bars, smem, sb, tmem, filt, npairs, it, first, s_item, queue, abort, copies0, copies1,
                           waited0, waited1);
      else if (warp == G::ISSUER + 1)
        mma_p2_loop<N, BF>(bars, sb, tmem, it, s_item, abort);
      else if (warp == G::ISSUER + 2)
        mma_p3_loop<N, BF, 0>(bars, sb, tmem, it, s_item, abort);
      else
        mma_p3_loop<N, BF, 1>(bars, sb, tmem, it, s_item, abort);
    } else {
        tc::setmaxnreg_inc<G::REG_EPI>();
        // ============================== epilogue warpgroups ===================================
        // per item: max |f| of its node (fp16 scale) and f into TMEM as the pass-1 A operand; then,
        // per step, the front (passes 1 and 2, every tile): warpgroup 0 turns each pass-1 result into
        // the pass-2 operands, warpgroup 1 each pass-2 result into rows of the pass-3 operands, so the
        // two steps of consecutive tiles overlap; back (pass 3): warpgroup w forms the products of the
        // tiles u = 2k + w. Thread = TMEM lane l.
        const int q = warp & 3, w = warp >> 2;
        const int l = 32 * q + lane, yl = l / N, lz = l % N;   // tile row: (yl, z) in pass 1, (yl, x') in pass 2
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        // shared-memory stores (one 16-byte unit = 8 consecutive rows of one k): A2 rows yl N + x',
        // k = z = lz; A3 rows x' N + z' with x' = lz, k = y
        const uint32_t a2_row = sb + G::S_A2 + ((uint32_t)(yl * N) >> 3) * G::A2_SBO + (lz >> 3) * G::A2_LBO + (lz & 7) * 16;
        const int mg3 = (lz * N) >> 3;
        uint32_t ph_f = 0, ph_a2free = 0, ph_a3free = 0, ph_f3p = 0, ph_f3m = 0;   // phase bits (bit b = ring slot b)
        float2 acc[G::TW][N / 2];   // P_r of the warpgroup's pass-3 tiles: (y' = 2j, 2j + 1) per entry
#pragma unroll
        for (int k = 0; k < G::TW; ++k)
#pragma unroll
            for (int j = 0; j < N / 2; ++j) acc[k][j] = make_float2(0.f, 0.f);
        // 2^-e, the weight of the lo parts of passes 2 and 3, as a pair for the packed FMAs
        const float2 eps2 = make_float2(exp2f(-(float)(BF ? kLoShiftBF16 : kLoShiftF16)),
                                        exp2f(-(float)(BF ? kLoShiftBF16 : kLoShiftF16)));
#define DGFS_WAITE(bar, ph)                                             \
    do {                                                                \
        if (!tc::warp_wait((bar), (ph), abort)) goto epi_done;          \
    } while (0)
        int64_t g = 0;   // step of the CTA's (radial point, pair) sequence
        for (int ki = 0;; ++ki) {
          long long item;
          if (!ring_take(bars, s_item, ki, item, abort) || item < 0) break;
          const int64_t node = item / it.rblocks;
          const int r0 = (int)(item % it.rblocks) * it.rpc;
          const float* fb = f + (offs ? offs[node] : node * n3s);
          float sf = 1.f;
          if (!BF) {
              // max |f| of the node; the unrolled loads and eight independent maxima keep the thread's
              // loads in flight together (a loop carried through one maximum costs a memory round trip
              // per element: about a tenth of the kernel at N = 32)
              constexpr int STRIDE = 32 * G::EPI_WARPS, PER = (int)(n3 / STRIDE);
              static_assert(n3 % STRIDE == 0 && PER % 8 == 0, "scan split");
              float m8[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) m8[j] = 0.f;
              if constexpr (!padded) {
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
              if (lane == 0) {
                  s_red[ki & 1][warp] = mx;
                  tc::mbar_arrive(&bars.scan[ki & 1]);
              }
              DGFS_WAITE(&bars.scan[ki & 1], (uint32_t)((ki >> 1) & 1));   // every epilogue warp's maximum
              mx = s_red[ki & 1][0];
#pragma unroll
              for (int i = 1; i < G::EPI_WARPS; ++i) mx = fmaxf(mx, s_red[ki & 1][i]);
              if (mx > 0.f && isfinite(mx)) sf = exp2f(fminf(60.f, fmaxf(-60.f, floorf(log2f(2.f / mx)))));
          }
          // fp16: max |f sf| in (1, 2]; pass 1 multiplies by 2^8 (its filters), which stays in the
          // stored intermediates and is removed, squared, from the products
          const float out_scale = BF ? 1.f : exp2f(-2.f * kP1ShiftF16) / (sf * sf);
          // ---- f -> TMEM as the pass-1 A operand once the previous item's pass-1 MMAs are complete:
          // tile t, lane l = yl N + z holds f[0..N)[t ZT + yl][z]
          if (ki > 0) DGFS_WAITE(&bars.f_free, (uint32_t)((ki - 1) & 1));
          tc::tc_fence_after();
          {
              // tiles t = 2k + w, two at a time: both tiles' loads precede the TMEM stores (whose memory
              // clobber would otherwise keep the next tile's loads behind them)
              constexpr int TB = G::TW >= 2 ? 2 : 1;
              static_assert(G::TW % TB == 0, "tile batches");
#pragma unroll 1
              for (int k0 = 0; k0 < G::TW; k0 += TB) {
                  uint32_t v[TB][N / 2];
#pragma unroll
                  for (int bb = 0; bb < TB; ++bb) {
                      const int y = (2 * (k0 + bb) + w) * G::ZT + yl;
                      if constexpr (!padded) {
                          const float* src = fb + (size_t)y * N + lz;
#pragma unroll
                          for (int c = 0; c < N / 2; ++c)
                              v[bb][c] = pack2<BF>(__ldg(src + (size_t)(2 * c) * G::N2) * sf,
                                                   __ldg(src + (size_t)(2 * c + 1) * G::N2) * sf);
                      } else {   // zeros outside the nsrc^3 block
                          const bool in = y < nsrc && lz < nsrc;
                          const float* src = fb + ((size_t)y * nsrc + lz);
                          const size_t sx = (size_t)nsrc * nsrc;
#pragma unroll
                          for (int c = 0; c < N / 2; ++c) {
                              const float a = in && 2 * c < nsrc ? __ldg(src + (size_t)(2 * c) * sx) * sf : 0.f;
                              const float b = in && 2 * c + 1 < nsrc ? __ldg(src + (size_t)(2 * c + 1) * sx) * sf : 0.f;
                              v[bb][c] = pack2<BF>(a, b);
                          }
                      }
                  }
#pragma unroll
                  for (int bb = 0; bb < TB; ++bb) {
                      const uint32_t ta = trow + G::C_F + (2 * (k0 + bb) + w) * (N / 2);
                      if constexpr (N == 32) tc::tmem_st16(ta, v[bb]);
                      else tc::tmem_st8(ta, v[bb]);
                  }
              }
              tc::tmem_wait_st();
          }
          tc::tc_fence_before();
          tc::mbar_arrive(&bars.f_ready);
          int ahead = 0;   // pass-1 tiles of the current step that warpgroup 0 handled during the last back
          for (int rr = 0; rr < it.rpc; ++rr) {
          for (int pp = 0; pp < npairs; ++pp, ++g) {
            if (w == 0) {
                // the step's remaining tiles, then, when the next step belongs to this item, its first
                // LOOKAHEAD tiles (virtual tiles T, T + 1): their pass-1 MMAs and operand buffers do not
                // depend on this step's pass 3, so warpgroup 0 fills the wait for the pass-3 operands
                // with them (a third would wait for the next step's pass 2, i.e. for this step's back)
                const int tend = G::T + ((pp + 1 < npairs || rr + 1 < it.rpc) ? G::LOOKAHEAD : 0);
                for (int t = ahead; t < tend; ++t) {   // pass-1 tile t (slot t % 2) -> pass-2 operands (buffer t % 2)
                    const int b = t & 1;
                    if (g > 0 || t >= 2) {   // pass 2 of tile t - 2 (of this or the previous step) has read buffer b
                        DGFS_WAITE(&bars.a2_free[b], (ph_a2free >> b) & 1u);
                        ph_a2free ^= 1u << b;
                    }
                    DGFS_WAITE(&bars.full1[b], (ph_f >> b) & 1u);
                    ph_f ^= 1u << b;
                    tc::tc_fence_after();
                    float v[2][N];   // the thread's row of the tile, both signs, behind one wait
                    const uint32_t tP1 = trow + G::C_S0 + b * G::C_S1;   // + at 0, - at N
#pragma unroll
                    for (int gs = 0; gs < 2; ++gs)
#pragma unroll
                        for (int c = 0; c < N / 16; ++c)
                            tc::tmem_ld16(tP1 + gs * N + 16 * c, *reinterpret_cast<float(*)[16]>(&v[gs][16 * c]));
                    tc::tmem_wait_ld();
                    tc::tc_fence_before();
                    tc::mbar_arrive(&bars.free1[b]);
                    const uint32_t a2b = a2_row + b * 2 * G::A2_BYTES;
#pragma unroll
                    for (int gs = 0; gs < 2; ++gs)
#pragma unroll
                        for (int c = 0; c < N / 8; ++c) {   // 8 columns x' = 8c .. 8c + 7
                            uint32_t u[4];
                            pack8<BF>(*reinterpret_cast<const float(*)[8]>(&v[gs][8 * c]), u);
                            tc::st_shared_v4(a2b + gs * G::A2_BYTES + c * G::A2_SBO, u[0], u[1], u[2], u[3]);
                        }
                    tc::fence_proxy_async();
                    tc::mbar_arrive(&bars.a2_full[b]);
                }
                ahead = tend - G::T;
            } else {
                for (int t = 0; t < G::T; ++t) {   // pass-2 tile t (slot t % 2) -> rows of the pass-3 operands
                    const int b = t & 1, y = t * G::ZT + yl;
                    if (t == 0 && g > 0) {   // the previous step's pass 3 has read the operands
                        DGFS_WAITE(&bars.a3_free, ph_a3free);
                        ph_a3free ^= 1;
                    }
                    DGFS_WAITE(&bars.full2[b], (ph_f >> b) & 1u);
                    ph_f ^= 1u << b;
                    tc::tc_fence_after();
                    const uint32_t tB = trow + (b ? G::C_S3 : G::C_S2);   // +hi, +lo, -hi, -lo
                    const uint32_t ky = (y >> 3) * G::A3_LBO + (y & 7) * 16;
#pragma unroll
                    for (int gs = 0; gs < 2; ++gs) {   // one sign: hi and lo of the row behind one wait
                        float hi[N], lo[N];
#pragma unroll
                        for (int c = 0; c < N / 16; ++c) {
                            tc::tmem_ld16(tB + gs * 2 * N + 16 * c, *reinterpret_cast<float(*)[16]>(&hi[16 * c]));
                            tc::tmem_ld16(tB + gs * 2 * N + N + 16 * c, *reinterpret_cast<float(*)[16]>(&lo[16 * c]));
                        }
                        tc::tmem_wait_ld();
                        if (gs == 1) {
                            tc::tc_fence_before();
                            tc::mbar_arrive(&bars.free2[b]);
                        }
#pragma unroll
                        for (int c = 0; c < N / 8; ++c) {   // 8 columns z' = 8c .. 8c + 7
                            uint32_t u[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {   // hi + 2^-e lo, two columns per packed FMA
                                const float2 v = tc::ffma2(make_float2(lo[8 * c + 2 * j], lo[8 * c + 2 * j + 1]), eps2,
                                                       make_float2(hi[8 * c + 2 * j], hi[8 * c + 2 * j + 1]));
                                u[j] = pack2<BF>(v.x, v.y);
                            }
                            const int mg = mg3 + c;
                            tc::st_shared_v4(sb + G::S_A3 + gs * G::A3_BYTES + (mg >> 4) * G::A3_TS + (mg & 15) * G::A3_SBO + ky,
                                             u[0], u[1], u[2], u[3]);
                        }
                    }
                }
                tc::fence_proxy_async();
                // failure test: the first CTA withholds the signal for its first step
                if (!(fault == 1 && g == 0 && blockIdx.x == 0)) tc::mbar_arrive(&bars.a3_full);
            }
            // pass-3 tiles u = 2k + w (slot w): products of the two translates
            const uint32_t tB = trow + (w ? G::C_S3 : G::C_S2);
#pragma unroll
            for (int k = 0; k < G::TW; ++k) {
                // + half, released before the - half is awaited
                DGFS_WAITE(&bars.full3p[w], ph_f3p);
                ph_f3p ^= 1u;
                tc::tc_fence_after();
                float2 xp[N / 2];   // + translate at y' = 2j, 2j + 1
#pragma unroll
                for (int c = 0; c < N / 16; ++c) {   // 16 columns y' = 16c .. 16c + 15 behind one wait
                    float hp[16], lp[16];
                    tc::tmem_ld16(tB + 16 * c, hp);
                    tc::tmem_ld16(tB + N + 16 * c, lp);
                    tc::tmem_wait_ld();
                    if (c == N / 16 - 1) {
                        tc::tc_fence_before();
                        tc::mbar_arrive(&bars.free3p[w]);
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j)   // two y' per packed FMA, the same roundings as fmaf
                        xp[8 * c + j] = tc::ffma2(make_float2(lp[2 * j], lp[2 * j + 1]), eps2,
                                                  make_float2(hp[2 * j], hp[2 * j + 1]));
                }
                DGFS_WAITE(&bars.full3m[w], ph_f3m);
                ph_f3m ^= 1u;
                tc::tc_fence_after();
#pragma unroll
                for (int c = 0; c < N / 16; ++c) {   // - half: 16 columns y' = 16c .. 16c + 15 behind one wait
                    float hm[16], lm[16];
                    tc::tmem_ld16(tB + 2 * N + 16 * c, hm);
                    tc::tmem_ld16(tB + 3 * N + 16 * c, lm);
                    tc::tmem_wait_ld();
                    if (c == N / 16 - 1) {
                        tc::tc_fence_before();
                        tc::mbar_arrive(&bars.free3m[w]);
                        if (k == G::TW - 1) tc::mbar_arrive(&bars.free3x[w]);
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float2 xm = tc::ffma2(make_float2(lm[2 * j], lm[2 * j + 1]), eps2,
                                                make_float2(hm[2 * j], hm[2 * j + 1]));
                        acc[k][8 * c + j] = tc::ffma2(xp[8 * c + j], xm, acc[k][8 * c + j]);
                    }
                }
            }
          }
          // radial point r0 + rr done: P_r out, sums cleared
          if (!*abort) {   // P[node][r][x'][y'][z'], row m3 = x' N + z' of tile u = 2k + w, column y'
              float* dst = P + ((size_t)node * Nrho + r0 + rr) * n3s;
              const float sc = out_scale * (coef ? coef[node] : 1.f);   // per-node factor (polarisation)
#pragma unroll
              for (int k = 0; k < G::TW; ++k) {
                  const int m3 = (2 * k + w) * 128 + l, xp = m3 / N, zp = m3 % N;
                  if constexpr (!padded) {
                      float* o = dst + (size_t)xp * G::N2 + zp;
#pragma unroll
                      for (int j = 0; j < N; ++j) {
                          const float a = (j & 1) ? acc[k][j / 2].y : acc[k][j / 2].x;
                          if (accum) o[(size_t)j * N] += a * sc;
                          else o[(size_t)j * N] = a * sc;
                      }
                  } else if (xp < nsrc && zp < nsrc) {   // the nsrc^3 block only
                      float* o = dst + (size_t)xp * nsrc * nsrc + zp;
#pragma unroll
                      for (int j = 0; j < N; ++j) {
                          if (j >= nsrc) continue;
                          const float a = (j & 1) ? acc[k][j / 2].y : acc[k][j / 2].x;
                          if (accum) o[(size_t)j * nsrc] += a * sc;
                          else o[(size_t)j * nsrc] = a * sc;
                      }
                  }
              }
          }
#pragma unroll
          for (int k = 0; k < G::TW; ++k)
#pragma unroll
              for (int j = 0; j < N / 2; ++j) acc[k][j] = make_float2(0.f, 0.f);
          }
        }
#undef DGFS_WAITE
    epi_done:;
    }

    // ---- drain: no MMA or copy of this CTA may be in flight when TMEM is freed -----------
    tc::tc_fence_before();
    __syncthreads();
    if (warp >= G::ISSUER) {
        if (tc::elect_one()) tc::mma_commit(&bars.drain);   // the lane that issued the warp's MMAs
        __syncwarp();
    }
    if (issuer) {
        if (tc::elect_one()) {   // the lane that issued every copy
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
}

template <int N, bool BF>
cudaError_t launch_n(const TcTables& t, const float* f, const int64_t* offs, int64_t nodes, float* P,
                     int* flags, cudaStream_t s, int fault, const float* coef, int accum) {
    using G = Geo<N>;
    const int nsrc = t.nsrc > 0 ? t.nsrc : N;
    auto kern = nsrc == N ? k_tc_gain<N, BF, false> : k_tc_gain<N, BF, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::S_TOTAL);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // radial points per item (tc_resolve_rpc); one CTA per SM pulls the items
    Items it;
    it.rpc = tc_resolve_rpc(t, BF ? DGFS_PREC_BF16S : DGFS_PREC_F16S, nodes, sms);
    it.rblocks = t.Nrho / it.rpc;
    it.nseq = it.rpc * t.npairs;
    it.n_items = nodes * it.rblocks;
    if (it.n_items > (int64_t)0x7FFFFFFF - 4096 || it.nseq < 1) return cudaErrorInvalidValue;
    int* queue = flags + kQueueWord;
    if ((e = cudaMemsetAsync(queue, 0, sizeof(int), s)) != cudaSuccess) return e;
    const int64_t grid = it.n_items < sms ? it.n_items : sms;
    kern<<<(unsigned)grid, G::THREADS, G::S_TOTAL, s>>>(f, offs, static_cast<const unsigned char*>(t.mats), t.npairs, t.Nrho,
                                                        it, nsrc, queue, P, flags, fault, coef, accum);
    return cudaGetLastError();
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

bool tc_supported(int N, int prec) {
    (void)prec;
    return N == 16 || N == 32 || N == 24;
}

int tc_resolve_rpc(const TcTables& t, int prec, int64_t nodes, int sms) {
    if (t.rpc > 0 && t.Nrho % t.rpc == 0) return t.rpc;
    // CTAs per radial block: two (a cluster) for the split-data kernels
    const int64_t per = tc3_precision(prec) ? 2 : 1;
    int rpc = 1;
    for (int c = 4; c > 1 && rpc == 1; c /= 2)
        if (t.Nrho % c == 0 && per * (int64_t)(t.Nrho / c) * nodes >= 16 * (int64_t)sms) rpc = c;
    return rpc;
}

int tc_extra_launches(int) { return 0; }

size_t build_tc_tables(const HostPlan& hp, int prec, std::vector<unsigned char>& blob, TcTables& t) {
    if (tc3_precision(prec)) return build_tc3_tables(hp, prec, blob, t);
    // N = 24 runs on the 32-point tiles: its circulant filters fill the top-left 24 x 24 block of
    // 32 x 32 matrices that are zero elsewhere, so every pass maps the zero-padded 24^3 field onto
    // the zero-padded translate (the kernel reads and writes only the 24^3 block)
    const int Nd = hp.N, N = Nd == 24 ? 32 : Nd, np = hp.npairs, Nr = hp.Nrho;
    const bool bf = prec == DGFS_PREC_BF16S;
    const double lo_scale = std::ldexp(1.0, bf ? kLoShiftBF16 : kLoShiftF16);
    const double p1_scale = bf ? 1.0 : std::ldexp(1.0, kP1ShiftF16);
    const size_t n2b = (size_t)N * N * 2;            // bytes of one N x N 16-bit matrix
    const size_t b1 = 4 * n2b, b23 = 2 * n2b, block = b1 + 4 * b23;
    blob.assign((size_t)Nr * np * block, 0);
    const size_t sbo = 16 * (size_t)N, lbo = 128;
    // K-major core-matrix layout of a B operand: row n (output index), column k (input index)
    auto put = [&](unsigned char* base, int n, int k, uint16_t bits) {
        std::memcpy(base + (n / 8) * sbo + (k / 8) * lbo + (n % 8) * 16 + (k % 8) * 2, &bits, 2);
    };
    // v = hi + lo / ls, both parts rounded to the operand type
    auto split = [&](double v, double ls, uint16_t& hi, uint16_t& lo) {
        hi = bf ? to_bf16_bits(v) : to_half_bits(v);
        const double hv = bf ? bf16_bits_value(hi) : half_bits_value(hi);
        lo = bf ? to_bf16_bits((v - hv) * ls) : to_half_bits((v - hv) * ls);
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
            for (int g = 0; g < 2; ++g)
                for (int i = 0; i < N; ++i)
                    for (int j = 0; j < N; ++j) {
                        uint16_t hi, lo;
                        // pass 1 (x, axis 0): rows +hi, -hi, +lo, -lo, both parts times p1_scale
                        // (accumulated in one accumulator); the + filter carries 2 w_p
                        split(F(0, g, i, j) * (g == 0 ? w2 : 1.0) * p1_scale, 1.0, hi, lo);
                        put(blk, g * N + i, j, hi);
                        put(blk, (2 + g) * N + i, j, lo);
                        // pass 2 (z, axis 2) and pass 3 (y, axis 1): rows hi, lo per sign
                        split(F(2, g, i, j), lo_scale, hi, lo);
                        put(blk + b1 + g * b23, i, j, hi);
                        put(blk + b1 + g * b23, N + i, j, lo);
                        split(F(1, g, i, j), lo_scale, hi, lo);
                        put(blk + b1 + 2 * b23 + g * b23, i, j, hi);
                        put(blk + b1 + 2 * b23 + g * b23, N + i, j, lo);
                    }
        }
    t.N = N;
    t.nsrc = Nd;
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
                                    cudaStream_t s, int fault, const float* coef, int accumulate) {
    if (g) return cudaErrorNotSupported;
    if (nodes <= 0) return cudaSuccess;
    if (tc3_precision(prec))
        return launch_tc3_gain_products(t, prec, f, offs, nodes, P, flags, s, fault, coef, accumulate);
    const bool bf = prec == DGFS_PREC_BF16S;
    switch (t.N) {
        case 16: return bf ? launch_n<16, true>(t, f, offs, nodes, P, flags, s, fault, coef, accumulate)
                           : launch_n<16, false>(t, f, offs, nodes, P, flags, s, fault, coef, accumulate);
        case 32: return bf ? launch_n<32, true>(t, f, offs, nodes, P, flags, s, fault, coef, accumulate)
                           : launch_n<32, false>(t, f, offs, nodes, P, flags, s, fault, coef, accumulate);
        default: return cudaErrorInvalidValue;
    }
}

namespace {

// Operands of the polarisation of the symmetric translate-product sum, one CTA per node:
// u[n] = f[n] + a_n g[n], u[nodes + n] = f[n] - a_n g[n] with a_n = |f_n| / |g_n| (1 when g_n = 0),
// coef[n] = 1 / (4 a_n) and coef[nodes + n] = -1 / (4 a_n), so that
// P(f, g) = coef[n] P(u[n]) + coef[nodes + n] P(u[nodes + n]).
__global__ void __launch_bounds__(256) k_polar_prep(const float* __restrict__ f, const float* __restrict__ g, int64_t n3,
                                                    int64_t nodes, float* __restrict__ u, float* __restrict__ coef) {
    __shared__ double red[2][8];
    __shared__ float s_a;
    const int64_t n = blockIdx.x;
    const float* fn = f + n * n3;
    const float* gn = g + n * n3;
    double sf = 0.0, sg = 0.0;
    for (int64_t i = threadIdx.x; i < n3; i += blockDim.x) {
        const double a = fn[i], b = gn[i];
        sf += a * a;
        sg += b * b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sf += __shfl_xor_sync(0xffffffffu, sf, o);
        sg += __shfl_xor_sync(0xffffffffu, sg, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sf;
        red[1][threadIdx.x >> 5] = sg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tf = 0.0, tg = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            tf += red[0][i];
            tg += red[1][i];
        }
        double a = (tg > 0.0 && tf > 0.0) ? sqrt(tf / tg) : 1.0;
        s_a = (float)a;
        coef[n] = (float)(0.25 / a);
        coef[nodes + n] = (float)(-0.25 / a);
    }
    __syncthreads();
    const float a = s_a;
    float* up = u + n * n3;
    float* um = u + (nodes + n) * n3;
    for (int64_t i = threadIdx.x; i < n3; i += blockDim.x) {
        const float x = fn[i], y = a * gn[i];
        up[i] = x + y;
        um[i] = x - y;
    }
}

}  // namespace

cudaError_t launch_polar_prep(const float* f, const float* g, int64_t n3, int64_t nodes, float* u, float* coef,
                              cudaStream_t s) {
    if (nodes <= 0) return cudaSuccess;
    k_polar_prep<<<(unsigned)nodes, 256, 0, s>>>(f, g, n3, nodes, u, coef);
    return cudaGetLastError();
}

}  // namespace dgfs
