// Tensor-core (tcgen05) translate-product kernel for the 16-bit precisions.
//
// Computes, like the CUDA-core kernel, P_r = sum_pairs 2 w_p (T_s f)(T_-s f) for Q(f, f)
// (arXiv:1809.10186, Appendix, eqs. lowrank1 and apndx_fs_Glm_Qk), with every dense circulant
// pass of the translates T_{+-s} run as tcgen05.mma (M = 128, N = grid size, K = grid size)
// with FP32 accumulators in tensor memory:
//
//   pass 1 (x): D1[(z,y)][x'] = sum_x f[x][y][z] A_x[x'][x]      A = f (K-major, resident)
//   pass 2 (y): D2[(z,x')][y'] = sum_y D1[(z,y)][x'] A_y[y'][y]  A = MN-major tile of D1
//   pass 3 (z): D3[(x',y')][z'] = sum_z D2[(z,x')][y'] A_z[z'][z] A = MN-major full field
//
// Data operands are 16-bit (fp16 with a per-node power-of-two scale, or bf16); every filter
// matrix is split into hi + lo 16-bit parts (two products per contraction). Each pass's
// epilogue reads its TMEM tile (one row per thread), rescales, rounds to 16 bits and writes
// the next pass's operand with 16-byte shared-memory stores. The + translate of all tiles
// stays in TMEM while the - translate is computed; their products accumulate in registers.
// The - filter is the transpose of the + filter (T_-s = T_s^T): the same shared-memory matrix
// is read as an MN-major operand.
//
// One CTA of 288 threads per (radial point, node), warp-specialised: one warp issues the MMAs
// and copies, two warpgroups convert accumulator tiles into the next pass's operands and form
// the products; all hand-offs are mbarriers. Every wait is bounded: on timeout the CTA raises
// flag bit 0, every role stops, the MMAs and copies in flight are drained (bounded), TMEM is
// freed and P is not written.
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_gain.h"
#include "tc_ptx.cuh"

namespace dgfs {

namespace {

constexpr int kFilterShift = 8;   // fp16 filters are stored times 2^8 (keeps the lo parts normal)

template <int N>
struct Geo {
    static_assert(N == 16 || N == 32, "tensor-core translates support N = 16 and 32");
    static constexpr int N2 = N * N;
    static constexpr int TILES = N2 / 128;    // 128-row M tiles of one field
    static constexpr int ZT = 128 / N;         // z values per pass-1/2 tile
    static constexpr int KSTEPS = N / 16;      // K = 16 steps of one contraction
    static constexpr int KG = N / 8;           // core-matrix groups along K
    static constexpr int HALF = N / 2;         // columns of the product per warpgroup
    static constexpr int ND1 = 3, ND2 = 2, ND3 = 2;   // TMEM buffers of passes 1, 2, 3 (- sign)
    // A1 = f, K-major: rows m1 = z*N + y, k = x
    static constexpr uint32_t A1_LBO = 128, A1_SBO = 16 * N;
    static constexpr uint32_t A1_TILE = 16 * A1_SBO, A1_BYTES = N2 * N * 2;
    // A2, MN-major, one tile: rows m2 = zl*N + x', k = y
    static constexpr uint32_t A2_SBO = 128, A2_LBO = 16 * 128, A2_BYTES = KG * A2_LBO;
    // A3, MN-major, whole field: rows m3 = x'*N + y', k = z; padded m-group and tile strides
    // spread the 16-byte stores of one 8-lane phase over more bank groups
    static constexpr uint32_t A3_SBO = 144, A3_TS = 16 * 144 + 16, A3_LBO = TILES * A3_TS;
    static constexpr uint32_t A3_BYTES = KG * A3_LBO;
    // filters: K-major N x N (row = output index, k = input index), [axis][hi|lo]
    static constexpr uint32_t F_LBO = 128, F_SBO = 16 * N, F_MAT = N2 * 2, F_BLOCK = 6 * F_MAT;
    // TMEM columns
    static constexpr uint32_t C_D1 = 0, C_D2 = ND1 * N, C_D3P = C_D2 + ND2 * N, C_D3M = C_D3P + TILES * N;
    static constexpr uint32_t C_USED = C_D3M + ND3 * N;
    static constexpr uint32_t TMEM_COLS = C_USED <= 32 ? 32 : C_USED <= 64 ? 64 : C_USED <= 128 ? 128
                                          : C_USED <= 256 ? 256 : 512;
    static_assert(C_USED <= 512, "TMEM budget");
    // shared memory
    static constexpr uint32_t S_A1 = 0, S_A2 = S_A1 + A1_BYTES, S_A3 = S_A2 + 2 * A2_BYTES;
    static constexpr uint32_t S_F = (S_A3 + A3_BYTES + 127) / 128 * 128;
    static constexpr uint32_t S_TOTAL = S_F + 2 * F_BLOCK;
};

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if (BF) {
        __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    } else {
        __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    }
}

// Barriers of the pipeline (mbarriers in shared memory).
struct Bars {
    uint64_t d1_full[3], d1_free[3];   // pass-1 accumulator: MMA -> WG0, WG0 -> MMA
    uint64_t a2_full[2];               // pass-2 operand written: WG0 -> MMA
    uint64_t d2_full[2], d2_free[2];   // pass-2 accumulator (its completion also frees A2)
    uint64_t a3_full, a3_free;         // pass-3 operand: WG1 -> MMA, MMA completion -> WG1
    uint64_t d3p_full, d3p_free;       // + translate in TMEM: MMA -> WGs, WGs -> MMA
    uint64_t d3m_full[2], d3m_free[2]; // - translate tiles
    uint64_t pair_done;                // all MMAs of a pair complete: its filter buffer is free
    uint64_t filt[2], drain;
};

// Warp roles: warps 0-3 (WG0) turn pass-1 tiles into pass-2 operands, warps 4-7 (WG1) turn
// pass-2 tiles into the pass-3 operand, both warpgroups form the products (half the columns
// each), warp 8 allocates TMEM and issues the MMAs and copies.
template <int N, bool BF>
__global__ void __launch_bounds__(288, 1)
k_tc_gain(const float* __restrict__ f, const int64_t* __restrict__ offs,
          const unsigned char* __restrict__ filt, const float* __restrict__ wsig, int npairs, int Nrho,
          float* __restrict__ P, int* __restrict__ flags) {
    using G = Geo<N>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) Bars bars;
    __shared__ uint32_t s_tmem;
    __shared__ float s_red[8];
    __shared__ int s_abort;
    volatile int* abort = &s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wg = warp >> 2, q = warp & 3;     // warpgroup (0, 1; 2 = MMA warp), lane quarter
    const int lrow = 32 * q + lane;              // TMEM lane (row) of this thread
    const int r = blockIdx.x;
    const int64_t node = blockIdx.y;
    const int64_t n3 = (int64_t)N * N * N;
    const float* fb = f + (offs ? offs[node] : node * n3);
    const uint32_t sb = tc::smem_u32(smem);

    // ---- set-up: scale, f -> A1 (warps 0-7); barriers, TMEM, first filter copies (warp 8) --
    float sf = 1.f;
    if (!BF) {
        float mx = 0.f;
        if (warp < 8)
            for (int e = tid; e < n3; e += 256) mx = fmaxf(mx, fabsf(__ldg(fb + e)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && warp < 8) s_red[warp] = mx;
        __syncthreads();
        mx = s_red[0];
#pragma unroll
        for (int i = 1; i < 8; ++i) mx = fmaxf(mx, s_red[i]);
        if (mx > 0.f && isfinite(mx)) sf = exp2f(fminf(60.f, fmaxf(-60.f, floorf(log2f(512.f / mx)))));
    }
    const float pass_scale = BF ? 1.f : exp2f(-(float)kFilterShift);   // undo the filter scaling
    const float out_scale = BF ? 1.f : exp2f(-2.f * kFilterShift) / (sf * sf);

    if (warp < 8) {
        for (int it = tid; it < G::N2 * G::KG; it += 256) {
            const int z = it % N, y = (it / N) % N, kg = it / G::N2;
            const int m1 = z * N + y;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __ldg(fb + (size_t)(kg * 8 + i) * G::N2 + y * N + z) * sf;
            tc::st_shared_v4(sb + G::S_A1 + (m1 >> 3) * G::A1_SBO + kg * G::A1_LBO + (m1 & 7) * 16,
                             pack2<BF>(v[0], v[1]), pack2<BF>(v[2], v[3]), pack2<BF>(v[4], v[5]), pack2<BF>(v[6], v[7]));
        }
    } else {
        if (lane == 0) {
            for (int i = 0; i < 3; ++i) {
                tc::mbar_init(&bars.d1_full[i], 1);
                tc::mbar_init(&bars.d1_free[i], 4);
            }
            for (int i = 0; i < 2; ++i) {
                tc::mbar_init(&bars.a2_full[i], 4);
                tc::mbar_init(&bars.d2_full[i], 1);
                tc::mbar_init(&bars.d2_free[i], 4);
                tc::mbar_init(&bars.d3m_full[i], 1);
                tc::mbar_init(&bars.d3m_free[i], 8);
                tc::mbar_init(&bars.filt[i], 1);
            }
            tc::mbar_init(&bars.a3_full, 4);
            tc::mbar_init(&bars.a3_free, 1);
            tc::mbar_init(&bars.d3p_full, 1);
            tc::mbar_init(&bars.d3p_free, 8);
            tc::mbar_init(&bars.pair_done, 1);
            tc::mbar_init(&bars.drain, 1);
            tc::fence_mbar_init();
            s_abort = 0;
            for (int p = 0; p < 2 && p < npairs; ++p) {
                tc::mbar_expect_tx(&bars.filt[p], G::F_BLOCK);
                tc::bulk_g2s(smem + G::S_F + p * G::F_BLOCK, filt + ((size_t)r * npairs + p) * G::F_BLOCK,
                             G::F_BLOCK, &bars.filt[p]);
            }
        }
        __syncwarp();
        tc::tmem_alloc(&s_tmem, G::TMEM_COLS);
    }
    tc::fence_proxy_async();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;

    float acc[G::TILES][G::HALF];
#pragma unroll
    for (int u = 0; u < G::TILES; ++u)
#pragma unroll
        for (int j = 0; j < G::HALF; ++j) acc[u][j] = 0.f;

    // filter copies issued and waited per buffer (only warp 8, lane 0 uses these)
    int filt_copies[2] = {npairs > 0 ? 1 : 0, npairs > 1 ? 1 : 0}, filt_waited[2] = {0, 0};

    if (warp == 8) {
        // ================================ MMA warp ======================================
        if (lane == 0) {
            int d1_use[3] = {0, 0, 0}, d2_use[2] = {0, 0}, d3m_use[2] = {0, 0};
            uint32_t ph_d1free[3] = {0, 0, 0}, ph_a2full[2] = {0, 0}, ph_d2free[2] = {0, 0};
            uint32_t ph_a3full = 0, ph_d3pfree = 0, ph_d3mfree[2] = {0, 0}, ph_pair = 0;
            auto issue = [&](uint32_t dcol, uint32_t a_start, uint32_t a_lbo, uint32_t a_sbo, bool a_mn, int axis,
                             int fbuf, int sg) {
                const uint32_t idesc = tc::idesc_f16(BF, a_mn, sg == 1, N, 128);
#pragma unroll
                for (int ks = 0; ks < G::KSTEPS; ++ks)
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const uint64_t da = tc::sdesc(a_start + ks * 2 * a_lbo, a_lbo, a_sbo);
                        const uint32_t fbase = sb + G::S_F + fbuf * G::F_BLOCK + (axis * 2 + pp) * G::F_MAT;
                        const uint64_t db = sg == 0 ? tc::sdesc(fbase + ks * 2 * G::F_LBO, G::F_LBO, G::F_SBO)
                                                    : tc::sdesc(fbase + ks * 2 * G::F_SBO, G::F_SBO, G::F_LBO);
                        tc::mma_f16(tmem + dcol, da, db, idesc, (ks | pp) != 0);
                    }
            };
            for (int p = 0; p < npairs; ++p) {
                const int fbuf = p & 1;
                if (!tc::mbar_wait_or_abort(&bars.filt[fbuf], (uint32_t)(filt_waited[fbuf] & 1), abort)) goto mma_done;
                filt_waited[fbuf]++;
                for (int sg = 0; sg < 2; ++sg) {
                    for (int step = 0; step <= G::TILES; ++step) {
                        if (step < G::TILES) {                       // pass 1, tile t
                            const int t = step, b = t % 3;
                            if (d1_use[b]++ > 0) {
                                if (!tc::mbar_wait_or_abort(&bars.d1_free[b], ph_d1free[b], abort)) goto mma_done;
                                ph_d1free[b] ^= 1;
                            }
                            tc::tc_fence_after();
                            issue(G::C_D1 + b * N, sb + G::S_A1 + t * G::A1_TILE, G::A1_LBO, G::A1_SBO, false, 0, fbuf, sg);
                            tc::mma_commit(&bars.d1_full[b]);
                            // once pair p - 1 is complete its filter buffer takes pair p + 1
                            // (waited here, after the first tiles of pair p are queued, so the
                            // tensor pipe never drains; every pair_done phase is waited in order)
                            if (sg == 0 && t == 0 && p >= 1) {
                                if (!tc::mbar_wait_or_abort(&bars.pair_done, ph_pair, abort)) goto mma_done;
                                ph_pair ^= 1;
                                if (p + 1 < npairs) {
                                    const int nb = (p + 1) & 1;
                                    tc::mbar_expect_tx(&bars.filt[nb], G::F_BLOCK);
                                    tc::bulk_g2s(smem + G::S_F + nb * G::F_BLOCK,
                                                 filt + ((size_t)r * npairs + p + 1) * G::F_BLOCK, G::F_BLOCK,
                                                 &bars.filt[nb]);
                                    filt_copies[nb]++;
                                }
                            }
                        }
                        if (step >= 1) {                             // pass 2, tile t - 1
                            const int t = step - 1, b = t & 1;
                            if (!tc::mbar_wait_or_abort(&bars.a2_full[b], ph_a2full[b], abort)) goto mma_done;
                            ph_a2full[b] ^= 1;
                            if (d2_use[b]++ > 0) {
                                if (!tc::mbar_wait_or_abort(&bars.d2_free[b], ph_d2free[b], abort)) goto mma_done;
                                ph_d2free[b] ^= 1;
                            }
                            tc::tc_fence_after();
                            issue(G::C_D2 + b * N, sb + G::S_A2 + b * G::A2_BYTES, G::A2_LBO, G::A2_SBO, true, 1, fbuf, sg);
                            tc::mma_commit(&bars.d2_full[b]);
                        }
                    }
                    if (!tc::mbar_wait_or_abort(&bars.a3_full, ph_a3full, abort)) goto mma_done;
                    ph_a3full ^= 1;
                    tc::tc_fence_after();
                    if (sg == 0) {
                        if (p > 0) {                                 // the previous pair's products are done
                            if (!tc::mbar_wait_or_abort(&bars.d3p_free, ph_d3pfree, abort)) goto mma_done;
                            ph_d3pfree ^= 1;
                        }
                        for (int u = 0; u < G::TILES; ++u)
                            issue(G::C_D3P + u * N, sb + G::S_A3 + u * G::A3_TS, G::A3_LBO, G::A3_SBO, true, 2, fbuf, 0);
                        tc::mma_commit(&bars.d3p_full);
                        tc::mma_commit(&bars.a3_free);
                    } else {
                        for (int u = 0; u < G::TILES; ++u) {
                            const int b = u & 1;
                            if (d3m_use[b]++ > 0) {
                                if (!tc::mbar_wait_or_abort(&bars.d3m_free[b], ph_d3mfree[b], abort)) goto mma_done;
                                ph_d3mfree[b] ^= 1;
                            }
                            tc::tc_fence_after();
                            issue(G::C_D3M + b * N, sb + G::S_A3 + u * G::A3_TS, G::A3_LBO, G::A3_SBO, true, 2, fbuf, 1);
                            tc::mma_commit(&bars.d3m_full[b]);
                        }
                        tc::mma_commit(&bars.a3_free);
                        tc::mma_commit(&bars.pair_done);
                    }
                }
            }
        mma_done:;
        }
        __syncwarp();
    } else {
        // ============================ epilogue warpgroups ==================================
        uint32_t ph_d1full[3] = {0, 0, 0}, ph_d2full[2] = {0, 0}, ph_a3free = 0, ph_d3pfull = 0;
        uint32_t ph_d3mfull[2] = {0, 0};
        int a2_use[2] = {0, 0};
        int signs_done = 0;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        for (int p = 0; p < npairs; ++p) {
            const float w2 = 2.f * wsig[p];
            for (int sg = 0; sg < 2; ++sg) {
                if (wg == 0) {
                    // pass-1 tiles -> pass-2 operands
                    for (int t = 0; t < G::TILES; ++t) {
                        const int b = t % 3, b2 = t & 1;
                        if (!tc::mbar_wait_or_abort(&bars.d1_full[b], ph_d1full[b], abort)) goto epi_done;
                        ph_d1full[b] ^= 1;
                        tc::tc_fence_after();
                        float v[N];
                        if constexpr (N == 32) tc::tmem_ld32(trow + G::C_D1 + b * N, v);
                        else tc::tmem_ld16(trow + G::C_D1 + b * N, *reinterpret_cast<float(*)[16]>(v));
                        tc::tmem_wait_ld();
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&bars.d1_free[b]);
                        // A2[b2] is free once the pass-2 MMA of its previous tile has completed
                        if (a2_use[b2]++ > 0) {
                            if (!tc::mbar_wait_or_abort(&bars.d2_full[b2], ph_d2full[b2], abort)) goto epi_done;
                            ph_d2full[b2] ^= 1;
                        }
                        const int m1 = t * 128 + lrow, y = m1 % N, zl = lrow / N;
#pragma unroll
                        for (int c = 0; c < N / 8; ++c) {
                            const int mg = (zl * N + 8 * c) >> 3;
                            const float* w = v + 8 * c;
                            tc::st_shared_v4(sb + G::S_A2 + b2 * G::A2_BYTES + mg * G::A2_SBO + (y >> 3) * G::A2_LBO + (y & 7) * 16,
                                             pack2<BF>(w[0] * pass_scale, w[1] * pass_scale), pack2<BF>(w[2] * pass_scale, w[3] * pass_scale),
                                             pack2<BF>(w[4] * pass_scale, w[5] * pass_scale), pack2<BF>(w[6] * pass_scale, w[7] * pass_scale));
                        }
                        tc::fence_proxy_async();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&bars.a2_full[b2]);
                    }
                } else {
                    // pass-2 tiles -> the pass-3 operand (A3 must be free of the last pass 3)
                    if (signs_done > 0) {
                        if (!tc::mbar_wait_or_abort(&bars.a3_free, ph_a3free, abort)) goto epi_done;
                        ph_a3free ^= 1;
                    }
                    for (int t = 0; t < G::TILES; ++t) {
                        const int b = t & 1;
                        if (!tc::mbar_wait_or_abort(&bars.d2_full[b], ph_d2full[b], abort)) goto epi_done;
                        ph_d2full[b] ^= 1;
                        tc::tc_fence_after();
                        float v[N];
                        if constexpr (N == 32) tc::tmem_ld32(trow + G::C_D2 + b * N, v);
                        else tc::tmem_ld16(trow + G::C_D2 + b * N, *reinterpret_cast<float(*)[16]>(v));
                        tc::tmem_wait_ld();
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&bars.d2_free[b]);
                        const int zl = lrow / N, xp = lrow % N, z = t * G::ZT + zl;
#pragma unroll
                        for (int c = 0; c < N / 8; ++c) {
                            const int mg = (xp * N + 8 * c) >> 3;
                            const int u = mg >> 4, mgl = mg & 15;
                            const float* w = v + 8 * c;
                            tc::st_shared_v4(sb + G::S_A3 + u * G::A3_TS + mgl * G::A3_SBO + (z >> 3) * G::A3_LBO + (z & 7) * 16,
                                             pack2<BF>(w[0] * pass_scale, w[1] * pass_scale), pack2<BF>(w[2] * pass_scale, w[3] * pass_scale),
                                             pack2<BF>(w[4] * pass_scale, w[5] * pass_scale), pack2<BF>(w[6] * pass_scale, w[7] * pass_scale));
                        }
                    }
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bars.a3_full);
                }
                signs_done++;
                if (sg == 1) {
                    // products of the two translates, half of the columns per warpgroup
                    if (!tc::mbar_wait_or_abort(&bars.d3p_full, ph_d3pfull, abort)) goto epi_done;
                    ph_d3pfull ^= 1;
#pragma unroll
                    for (int u = 0; u < G::TILES; ++u) {
                        const int b = u & 1;
                        if (!tc::mbar_wait_or_abort(&bars.d3m_full[b], ph_d3mfull[b], abort)) goto epi_done;
                        ph_d3mfull[b] ^= 1;
                        tc::tc_fence_after();
                        float fm[G::HALF], fp[G::HALF];
                        if constexpr (G::HALF == 16) {
                            tc::tmem_ld16(trow + G::C_D3M + b * N + wg * G::HALF, *reinterpret_cast<float(*)[16]>(fm));
                            tc::tmem_ld16(trow + G::C_D3P + u * N + wg * G::HALF, *reinterpret_cast<float(*)[16]>(fp));
                        } else {
                            tc::tmem_ld8(trow + G::C_D3M + b * N + wg * G::HALF, *reinterpret_cast<float(*)[8]>(fm));
                            tc::tmem_ld8(trow + G::C_D3P + u * N + wg * G::HALF, *reinterpret_cast<float(*)[8]>(fp));
                        }
                        tc::tmem_wait_ld();
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&bars.d3m_free[b]);
#pragma unroll
                        for (int j = 0; j < G::HALF; ++j) acc[u][j] = fmaf(w2 * fp[j], fm[j], acc[u][j]);
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bars.d3p_free);
                }
            }
        }
        if (!*abort) {   // results: P[node][r][x'][y'][z'] = acc * out_scale (this warpgroup's half)
            float* dst = P + ((size_t)node * Nrho + r) * n3;
#pragma unroll
            for (int u = 0; u < G::TILES; ++u) {
                const int m3 = u * 128 + lrow;
                float4* o = reinterpret_cast<float4*>(dst + (size_t)m3 * N + wg * G::HALF);
#pragma unroll
                for (int j = 0; j < G::HALF; j += 4)
                    o[j / 4] = make_float4(acc[u][j] * out_scale, acc[u][j + 1] * out_scale,
                                           acc[u][j + 2] * out_scale, acc[u][j + 3] * out_scale);
            }
        }
    epi_done:;
    }

    // ---- drain: no MMA or copy of this CTA may be in flight when TMEM is freed -----------
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        if (lane == 0) {
            if (*abort) atomicOr(flags, 1);
            tc::mma_commit(&bars.drain);
            if (!tc::mbar_wait(&bars.drain, 0)) atomicOr(flags, 1);
            // wait for every issued filter copy that the pipeline did not wait for
            for (int i = 0; i < 2; ++i)
                for (int k = filt_waited[i]; k < filt_copies[i]; ++k)
                    if (!tc::mbar_wait(&bars.filt[i], (uint32_t)(k & 1))) { atomicOr(flags, 1); break; }
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
        kern<<<dim3(t.Nrho, (unsigned)nn), 288, G::S_TOTAL, s>>>(
            f + (offs ? 0 : n0 * n3), offs ? offs + n0 : nullptr, static_cast<const unsigned char*>(t.mats),
            t.wsig, t.npairs, t.Nrho, P + n0 * t.Nrho * n3, flags);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// host-side rounding of a double to the 16-bit operand types
uint16_t to_half_bits(double x) {
    __half h = __double2half((double)x);
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
    const double fscale = bf ? 1.0 : std::ldexp(1.0, kFilterShift);
    const size_t mat = (size_t)N * N * 2, block = 6 * mat;
    const size_t mats_bytes = (size_t)Nr * np * block;
    const size_t wsig_off = (mats_bytes + 255) / 256 * 256;
    const size_t total = wsig_off + (size_t)np * sizeof(float);
    blob.assign(total, 0);
    const uint32_t lbo = 128, sbo = 16 * N;
    for (int r = 0; r < Nr; ++r)
        for (int p = 0; p < np; ++p)
            for (int a = 0; a < 3; ++a) {
                const double* fl = &hp.filt[(((size_t)r * np + p) * 3 + a) * N];
                for (int i = 0; i < N; ++i)
                    for (int j = 0; j < N; ++j) {
                        const double v = fl[((i - j) % N + N) % N] * fscale;   // A_+[i][j] = a[(i - j) mod N]
                        const uint16_t hi = bf ? to_bf16_bits(v) : to_half_bits(v);
                        const double hv = bf ? bf16_bits_value(hi) : half_bits_value(hi);
                        const uint16_t lo = bf ? to_bf16_bits(v - hv) : to_half_bits(v - hv);
                        const size_t off = (i / 8) * sbo + (j / 8) * lbo + (i % 8) * 16 + (j % 8) * 2;
                        unsigned char* bp = blob.data() + ((size_t)r * np + p) * block + (size_t)(a * 2) * mat;
                        std::memcpy(bp + off, &hi, 2);
                        std::memcpy(bp + mat + off, &lo, 2);
                    }
            }
    float* w = reinterpret_cast<float*>(blob.data() + wsig_off);
    for (int p = 0; p < np; ++p) w[p] = (float)hp.wsig[p];
    t.N = N;
    t.Nrho = Nr;
    t.npairs = np;
    t.mats = reinterpret_cast<const void*>((uintptr_t)0);
    t.wsig = reinterpret_cast<const float*>((uintptr_t)wsig_off);
    return total;
}

void rebase_tc_tables(TcTables& t, void* base) {
    t.mats = static_cast<unsigned char*>(base) + reinterpret_cast<uintptr_t>(t.mats);
    t.wsig = reinterpret_cast<const float*>(static_cast<unsigned char*>(base) + reinterpret_cast<uintptr_t>(t.wsig));
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
