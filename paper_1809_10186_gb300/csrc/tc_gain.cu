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
// One CTA of 256 threads per (radial point, node); thread 0 issues the MMAs; every wait on an
// mbarrier is bounded: on timeout the kernel raises flag bit 0, drains its own MMAs and copies
// (bounded), frees TMEM and returns without writing P.
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
    static constexpr int HALF = N / 2;         // TMEM columns read per thread
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
    // TMEM columns: D1[2], D2[2], + translate (all tiles), - translate tile [2]
    static constexpr uint32_t C_D1 = 0, C_D2 = 2 * N, C_D3P = 4 * N, C_D3M = 4 * N + TILES * N;
    static constexpr uint32_t C_USED = C_D3M + 2 * N;
    static constexpr uint32_t TMEM_COLS = C_USED <= 32 ? 32 : C_USED <= 64 ? 64 : C_USED <= 128 ? 128
                                          : C_USED <= 256 ? 256 : 512;
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

template <int N, bool BF>
__global__ void __launch_bounds__(256, 1)
k_tc_gain(const float* __restrict__ f, const int64_t* __restrict__ offs,
          const unsigned char* __restrict__ filt, const float* __restrict__ wsig, int npairs, int Nrho,
          float* __restrict__ P, int* __restrict__ flags) {
    using G = Geo<N>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mb_p1[2], mb_p2[2], mb_p3[2], mb_p3all, mb_filt[2], mb_drain;
    __shared__ uint32_t s_tmem;
    __shared__ float s_red[8];
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, h = warp >> 2;
    const int lrow = 32 * q + lane;            // TMEM lane of this thread
    const int r = blockIdx.x;
    const int64_t node = blockIdx.y;
    const int64_t n3 = (int64_t)N * N * N;
    const float* fb = f + (offs ? offs[node] : node * n3);
    const uint32_t sb = tc::smem_u32(smem);

    // ---- per-node scale (fp16: max |f| * sf in (256, 512]) ----------------------------------
    float sf = 1.f;
    if (!BF) {
        float mx = 0.f;
        for (int e = tid; e < n3; e += 256) mx = fmaxf(mx, fabsf(__ldg(fb + e)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_red[warp] = mx;
        __syncthreads();
        mx = s_red[0];
#pragma unroll
        for (int i = 1; i < 8; ++i) mx = fmaxf(mx, s_red[i]);
        if (mx > 0.f && isfinite(mx)) sf = exp2f(fminf(60.f, fmaxf(-60.f, floorf(log2f(512.f / mx)))));
    }
    const float pass_scale = BF ? 1.f : exp2f(-(float)kFilterShift);   // undo the filter scaling
    const float out_scale = BF ? 1.f : exp2f(-2.f * kFilterShift) / (sf * sf);

    // ---- f -> A1 (K-major 16-bit, rows (z, y), k = x) ---------------------------------------
    for (int it = tid; it < G::N2 * G::KG; it += 256) {
        const int z = it % N, y = (it / N) % N, kg = it / G::N2;
        const int m1 = z * N + y;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __ldg(fb + (size_t)(kg * 8 + i) * G::N2 + y * N + z) * sf;
        tc::st_shared_v4(sb + G::S_A1 + (m1 >> 3) * G::A1_SBO + kg * G::A1_LBO + (m1 & 7) * 16,
                         pack2<BF>(v[0], v[1]), pack2<BF>(v[2], v[3]), pack2<BF>(v[4], v[5]), pack2<BF>(v[6], v[7]));
    }

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&mb_p1[i], 1);
            tc::mbar_init(&mb_p2[i], 1);
            tc::mbar_init(&mb_p3[i], 1);
            tc::mbar_init(&mb_filt[i], 1);
        }
        tc::mbar_init(&mb_p3all, 1);
        tc::mbar_init(&mb_drain, 1);
        tc::fence_mbar_init();
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(&s_tmem, G::TMEM_COLS);
    tc::fence_proxy_async();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;

    int filt_issued[2] = {0, 0}, filt_waited[2] = {0, 0};
    if (tid == 0) {
        for (int p = 0; p < 2 && p < npairs; ++p) {
            tc::mbar_expect_tx(&mb_filt[p], G::F_BLOCK);
            tc::bulk_g2s(smem + G::S_F + p * G::F_BLOCK, filt + ((size_t)r * npairs + p) * G::F_BLOCK,
                         G::F_BLOCK, &mb_filt[p]);
        }
    }
    for (int p = 0; p < 2 && p < npairs; ++p) filt_issued[p] = 1;

    // MMA issue (thread 0): one contraction = KSTEPS x {hi, lo} instructions
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
    auto issue_p1 = [&](int t, int b, int fbuf, int sg) {
        issue(G::C_D1 + b * N, sb + G::S_A1 + t * G::A1_TILE, G::A1_LBO, G::A1_SBO, false, 0, fbuf, sg);
    };
    auto issue_p2 = [&](int b, int fbuf, int sg) {
        issue(G::C_D2 + b * N, sb + G::S_A2 + b * G::A2_BYTES, G::A2_LBO, G::A2_SBO, true, 1, fbuf, sg);
    };
    auto issue_p3 = [&](int u, uint32_t dcol, int fbuf, int sg) {
        issue(dcol, sb + G::S_A3 + u * G::A3_TS, G::A3_LBO, G::A3_SBO, true, 2, fbuf, sg);
    };
    const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + h * G::HALF;   // this thread's TMEM slice
    auto tload = [&](uint32_t col, float* v) {
        if constexpr (G::HALF == 16) {
            tc::tmem_ld16(trow + col, *reinterpret_cast<float(*)[16]>(v));
        } else {
            tc::tmem_ld8(trow + col, *reinterpret_cast<float(*)[8]>(v));
        }
    };
    // pass-1 epilogue: D1 row (z, y), columns x' -> A2 rows (zl, x'), K-row y
    auto epi1 = [&](int t, int b) {
        float v[G::HALF];
        tload(G::C_D1 + b * N, v);
        tc::tmem_wait_ld();
        const int m1 = t * 128 + lrow, y = m1 % N, zl = lrow / N;
#pragma unroll
        for (int c = 0; c < G::HALF / 8; ++c) {
            const int mg = (zl * N + h * G::HALF + 8 * c) >> 3;
            const float* w = v + 8 * c;
            tc::st_shared_v4(sb + G::S_A2 + b * G::A2_BYTES + mg * G::A2_SBO + (y >> 3) * G::A2_LBO + (y & 7) * 16,
                             pack2<BF>(w[0] * pass_scale, w[1] * pass_scale), pack2<BF>(w[2] * pass_scale, w[3] * pass_scale),
                             pack2<BF>(w[4] * pass_scale, w[5] * pass_scale), pack2<BF>(w[6] * pass_scale, w[7] * pass_scale));
        }
    };
    // pass-2 epilogue: D2 row (zl, x'), columns y' -> A3 rows (x', y'), K-row z
    auto epi2 = [&](int t, int b) {
        float v[G::HALF];
        tload(G::C_D2 + b * N, v);
        tc::tmem_wait_ld();
        const int zl = lrow / N, xp = lrow % N, z = t * G::ZT + zl;
#pragma unroll
        for (int c = 0; c < G::HALF / 8; ++c) {
            const int mg = (xp * N + h * G::HALF + 8 * c) >> 3;
            const int u = mg >> 4, mgl = mg & 15;
            const float* w = v + 8 * c;
            tc::st_shared_v4(sb + G::S_A3 + u * G::A3_TS + mgl * G::A3_SBO + (z >> 3) * G::A3_LBO + (z & 7) * 16,
                             pack2<BF>(w[0] * pass_scale, w[1] * pass_scale), pack2<BF>(w[2] * pass_scale, w[3] * pass_scale),
                             pack2<BF>(w[4] * pass_scale, w[5] * pass_scale), pack2<BF>(w[6] * pass_scale, w[7] * pass_scale));
        }
    };
    auto fail = [&]() { s_abort = 1; if (lane == 0) atomicOr(flags, 1); };
    auto sync = [&]() {
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
    };

    float acc[G::TILES][G::HALF];
#pragma unroll
    for (int u = 0; u < G::TILES; ++u)
#pragma unroll
        for (int j = 0; j < G::HALF; ++j) acc[u][j] = 0.f;
    uint32_t ph1[2] = {0, 0}, ph2[2] = {0, 0}, ph3[2] = {0, 0}, ph3all = 0;

    for (int p = 0; p < npairs; ++p) {
        const int fbuf = p & 1;
        if (!tc::mbar_wait(&mb_filt[fbuf], (uint32_t)(filt_waited[fbuf] & 1))) fail();
        filt_waited[fbuf]++;
        const float w2 = 2.f * wsig[p];
        for (int sg = 0; sg < 2; ++sg) {
            if (tid == 0) {
                issue_p1(0, 0, fbuf, sg);
                tc::mma_commit(&mb_p1[0]);
                if (G::TILES > 1) {
                    issue_p1(1, 1, fbuf, sg);
                    tc::mma_commit(&mb_p1[1]);
                }
            }
            for (int t = 0; t < G::TILES; ++t) {
                const int b = t & 1;
                if (!tc::mbar_wait(&mb_p1[b], ph1[b])) fail();
                ph1[b] ^= 1;
                tc::tc_fence_after();
                epi1(t, b);
                tc::fence_proxy_async();
                sync();
                if (s_abort) goto drain;
                if (tid == 0) {
                    issue_p2(b, fbuf, sg);
                    tc::mma_commit(&mb_p2[b]);
                    if (t + 2 < G::TILES) {
                        issue_p1(t + 2, b, fbuf, sg);
                        tc::mma_commit(&mb_p1[b]);
                    }
                }
                if (t >= 1) {
                    const int b2 = (t - 1) & 1;
                    if (sg == 1 && t == 1) {        // the + pass 3 must be done with A3
                        if (!tc::mbar_wait(&mb_p3all, ph3all)) fail();
                        ph3all ^= 1;
                    }
                    if (!tc::mbar_wait(&mb_p2[b2], ph2[b2])) fail();
                    ph2[b2] ^= 1;
                    tc::tc_fence_after();
                    epi2(t - 1, b2);
                }
            }
            {
                const int b2 = (G::TILES - 1) & 1;
                if (!tc::mbar_wait(&mb_p2[b2], ph2[b2])) fail();
                ph2[b2] ^= 1;
                tc::tc_fence_after();
                epi2(G::TILES - 1, b2);
            }
            tc::fence_proxy_async();
            sync();
            if (s_abort) goto drain;
            if (sg == 0) {
                if (tid == 0) {
#pragma unroll
                    for (int u = 0; u < G::TILES; ++u) issue_p3(u, G::C_D3P + u * N, fbuf, 0);
                    tc::mma_commit(&mb_p3all);
                }
            } else {
                if (tid == 0) {
                    issue_p3(0, G::C_D3M, fbuf, 1);
                    tc::mma_commit(&mb_p3[0]);
                    if (G::TILES > 1) {
                        issue_p3(1, G::C_D3M + N, fbuf, 1);
                        tc::mma_commit(&mb_p3[1]);
                    }
                }
#pragma unroll
                for (int u = 0; u < G::TILES; ++u) {
                    const int b = u & 1;
                    if (!tc::mbar_wait(&mb_p3[b], ph3[b])) fail();
                    ph3[b] ^= 1;
                    tc::tc_fence_after();
                    float fm[G::HALF], fp[G::HALF];
                    tload(G::C_D3M + b * N, fm);
                    tload(G::C_D3P + u * N, fp);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < G::HALF; ++j) acc[u][j] = fmaf(w2 * fp[j], fm[j], acc[u][j]);
                    sync();
                    if (s_abort) goto drain;
                    if (tid == 0 && u + 2 < G::TILES) {
                        issue_p3(u + 2, G::C_D3M + b * N, fbuf, 1);
                        tc::mma_commit(&mb_p3[b]);
                    }
                }
            }
        }
        // every MMA of pair p has completed: its filter buffer can take pair p + 2
        if (p + 2 < npairs) {
            if (tid == 0) {
                tc::mbar_expect_tx(&mb_filt[fbuf], G::F_BLOCK);
                tc::bulk_g2s(smem + G::S_F + fbuf * G::F_BLOCK, filt + ((size_t)r * npairs + p + 2) * G::F_BLOCK,
                             G::F_BLOCK, &mb_filt[fbuf]);
            }
            filt_issued[fbuf]++;
        }
    }

    {   // results: P[node][r][x'][y'][z'] = acc * out_scale
        float* dst = P + ((size_t)node * Nrho + r) * n3;
#pragma unroll
        for (int u = 0; u < G::TILES; ++u) {
            const int m3 = u * 128 + lrow;
            float4* o = reinterpret_cast<float4*>(dst + (size_t)m3 * N + h * G::HALF);
#pragma unroll
            for (int j = 0; j < G::HALF; j += 4)
                o[j / 4] = make_float4(acc[u][j] * out_scale, acc[u][j + 1] * out_scale, acc[u][j + 2] * out_scale,
                                       acc[u][j + 3] * out_scale);
        }
    }

drain:
    // make sure no MMA or copy of this CTA is still in flight before TMEM is freed
    sync();
    if (tid == 0) {
        tc::mma_commit(&mb_drain);
        if (!tc::mbar_wait(&mb_drain, 0)) atomicOr(flags, 1);
        for (int i = 0; i < 2; ++i)
            while (filt_waited[i] < filt_issued[i]) {
                if (!tc::mbar_wait(&mb_filt[i], (uint32_t)(filt_waited[i] & 1))) { atomicOr(flags, 1); break; }
                filt_waited[i]++;
            }
    }
    sync();
    if (warp == 0) tc::tmem_dealloc(tmem, G::TMEM_COLS);
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
        kern<<<dim3(t.Nrho, (unsigned)nn), 256, G::S_TOTAL, s>>>(
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
