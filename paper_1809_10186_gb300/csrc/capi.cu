// C ABI of the fast spectral collision operator (declared in include/dgfs.h).
//
// A plan owns: the FP64 host plan (plan_host.cpp), the device tables rounded to the compute
// type, one device workspace sized for a chunk of nodes, and a device flag word. Every
// compute call loops over node chunks and enqueues, per chunk,
//   1. the translate products                  P_r = sum_p w_p [(T_s f)(T_-s g) + (T_-s f)(T_s g)]
//      (tensor cores for Q(f, f) of F16S/BF16S plans, tc_gain.cu; Fourier-space translates for every
//      other call, k_vss.cu; the dense circulant kernel, k_gain_simt.cuh, for the allocation-free
//      call of FP32/FP64 plans)
//   2. the radial projection                   X_s = sum_r Vr[s][r] w_r rho_r P_r
//   3. forward DFTs of X_s and the loss operand
//   4. the Fourier combine                     sum_s Uk[s] X^_s + i G_loss g^
//   5. one inverse DFT and the finalisation    Q = Re - f Im
// on the caller's stream; nothing is allocated after dgfs_plan_create. Plans of the VSS kernel
// (alpha != 1) take the per-sphere-point path of k_vss.cu instead (vss_chunk below).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/dgfs.h"
#include "launchers.h"
#include "plan_host.h"
#include "tc_gain.h"

using namespace dgfs;

namespace {

thread_local std::string g_last_error;

dgfs_status fail(dgfs_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

dgfs_status cuda_fail(cudaError_t e, const char* where) {
    return fail(DGFS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define DGFS_CUDA(call, where)                              \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

constexpr uint64_t kMagic = 0x44474653504c414eull;   // "DGFSPLAN"

// Makes `dev` the calling thread's current device while the object lives and then restores the
// caller's device: no entry point leaves its caller on another device.
class DeviceScope {
  public:
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        if (prev_ != dev) {
            err_ = cudaSetDevice(dev);
            changed_ = err_ == cudaSuccess && prev_ >= 0;
        }
    }
    ~DeviceScope() {
        if (changed_) cudaSetDevice(prev_);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
    cudaError_t error() const { return err_; }

  private:
    int prev_ = -1;
    bool changed_ = false;
    cudaError_t err_ = cudaSuccess;
};

#define DGFS_ON_DEVICE(dev)                                                           \
    DeviceScope dgfs_scope_(dev);                                                     \
    if (dgfs_scope_.error() != cudaSuccess) return cuda_fail(dgfs_scope_.error(), "cudaSetDevice")

}  // namespace

struct dgfs_plan_s {
    uint64_t magic = kMagic;
    HostPlan hp;
    int prec = DGFS_PREC_FP32;
    int device = 0;
    int64_t chunk = 1;
    int64_t run_chunk = 0;   // nodes per chunk of the compute calls (autotuned); 0: chunk
    size_t ws_bytes = 0, table_bytes = 0;
    void* d_tables = nullptr;
    void* d_ws = nullptr;
    int* d_flags = nullptr;
    DevTables<float> tf{};
    DevTables<double> td{};
    TcTables tc{};           // tensor-core translate tables (16-bit precisions only)
    // workspace carve (byte offsets into d_ws)
    size_t off_P = 0, off_G = 0, off_X = 0, off_Y = 0, off_io = 0, off_node = 0;
    // VSS kernel: nodes per transform batch, its workspace region and the device tables
    int64_t vchunk = 0;
    bool vss_planes = false;   // fused plane/line kernels, plane-major fields and tables
    // VHS translate products in Fourier space (FP32/FP64, N = 8, 16, 32): nodes per transform batch
    bool fftx = false;
    int64_t xchunk = 0;
    size_t off_Xt = 0;
    const void* d_mu = nullptr;   // [Nrho][npairs][3][N] complex multipliers (inside d_vss)
    size_t off_V = 0, vss_bytes = 0;
    void* d_vss = nullptr;   // A [Nrho][npairs][N^3] (T) | GL [N^3] (T) | mu [Nrho][npairs][3][N] (complex T)
    int xfields = 0;
    std::mutex host_mu;      // serialises host-side staging of per-node arrays
    int fault = 0;           // failure-test injection for the next tensor-core launch (dgfs_debug_inject)
    // host-buffer entry point: copy streams and the events that pipeline copies with compute
    cudaStream_t cs_h2d = nullptr, cs_d2h = nullptr;
    cudaEvent_t ev_start = nullptr, ev_h2d[2] = {}, ev_comp[2] = {}, ev_d2h[2] = {};
    // profiling session
    bool prof = false;
    std::vector<cudaEvent_t> ev;   // pairs
    int64_t prof_launches = 0, prof_gain = 0, prof_timed = 0, prof_nodes = 0;
};

namespace {

// NVTX range around a phase of a call (visible in a profiler's timeline; no cost without one).
// end() closes it early; the destructor closes it otherwise.
struct NvtxRange {
    bool open = true;
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    void end() {
        if (open) nvtxRangePop();
        open = false;
    }
    ~NvtxRange() { end(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

bool is_tc(int prec) {
    return prec == DGFS_PREC_F16S || prec == DGFS_PREC_BF16S || prec == DGFS_PREC_F16X3 || prec == DGFS_PREC_BF16X3;
}

size_t elem_size(int prec) { return prec == DGFS_PREC_FP64 ? 8 : 4; }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool check_plan(dgfs_plan_t p) { return p && p->magic == kMagic; }

void destroy_io(dgfs_plan_s* p) {
    for (cudaEvent_t* ev : {&p->ev_start, &p->ev_h2d[0], &p->ev_h2d[1], &p->ev_comp[0], &p->ev_comp[1], &p->ev_d2h[0],
                            &p->ev_d2h[1]})
        if (*ev) {
            cudaEventDestroy(*ev);
            *ev = nullptr;
        }
    if (p->cs_h2d) cudaStreamDestroy(p->cs_h2d);
    if (p->cs_d2h) cudaStreamDestroy(p->cs_d2h);
    p->cs_h2d = p->cs_d2h = nullptr;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Bytes of the VSS path per node of a transform batch: the operand spectra (2), the translate
// spectra (2 sets x npairs), the packed products ((npairs + 1) / 2) and the output spectra (3).
size_t vss_node_bytes(const HostPlan& h, int prec) {
    const size_t n3 = (size_t)h.N * h.N * h.N;
    return 2 * elem_size(prec) * n3 * (2 + 2 * (size_t)h.npairs + (size_t)(h.npairs + 1) / 2 + 3);
}

// Per-node workspace bytes (all operations share one layout). VSS plans use only the staging
// area and their own region (off_V, vchunk nodes).
void workspace_layout(dgfs_plan_s* p, int64_t C) {
    const size_t es = elem_size(p->prec);
    const size_t n3 = (size_t)p->hp.N * p->hp.N * p->hp.N;
    const size_t Nr = p->hp.aniso ? 0 : p->hp.Nrho;
    p->xfields = p->hp.rank + 2;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes, 256); return o; };
    if (p->hp.aniso) {
        p->off_V = take((size_t)p->vchunk * vss_node_bytes(p->hp, p->prec));
        p->off_P = p->off_G = p->off_X = p->off_Y = p->off_V;
        p->off_io = take(C * 2 * n3 * es);
        p->off_node = take(C * (sizeof(int64_t) + 2 * sizeof(double)));
        p->ws_bytes = off;
        return;
    }
    p->off_P = take(C * Nr * n3 * es);                 // P_r (also K_r u for the VJP)
    p->off_G = take(C * n3 * es);                      // VJP: the gain's radial sum
    // X also holds, during the translate stage of a bilinear call of a tensor-core plan, the
    // polarisation operands (2 fields per node) and their per-node factors
    p->off_X = take(C * std::max<size_t>((size_t)p->xfields * n3 * 2 * es, 2 * n3 * es + 2 * sizeof(float)));
    p->off_Y = take(C * 3 * n3 * 2 * es);
    p->off_io = take(C * 2 * n3 * es);                 // host-buffer staging (f in, Q out)
    p->off_node = take(C * (sizeof(int64_t) + 2 * sizeof(double)));
    // operand spectra and translate spectra of a batch of the Fourier-space translate products
    p->off_Xt = take((size_t)p->xchunk * (2 + 2 * (size_t)p->hp.npairs) * n3 * 2 * es);
    p->ws_bytes = off;
}

template <typename T>
void fill_tables(dgfs_plan_s* p, std::vector<unsigned char>& blob, DevTables<T>& t, size_t& bytes) {
    const HostPlan& h = p->hp;
    const int N = h.N;
    const size_t n3 = (size_t)N * N * N;
    size_t off = 0;
    std::vector<std::pair<size_t, size_t>> spans;
    auto take = [&](size_t b) { const size_t o = off; off = align_up(off + b, 256); return o; };
    const size_t o_filt = take(h.filt.size() * sizeof(T));
    const size_t o_wsig = take(h.wsig.size() * sizeof(T));
    const size_t o_cr = take(h.cr.size() * sizeof(double));
    const size_t o_wr = take(h.wr.size() * sizeof(double));
    const size_t o_Uk = take(h.Uk.size() * sizeof(T));
    const int nq2 = 3 * (N / 2) * (N / 2) + 1;
    const size_t o_Uq = take((size_t)h.rank * nq2 * sizeof(T));
    const size_t o_Vr = take(h.Vr.size() * sizeof(T));
    const size_t o_Lr = take(h.Lr.size() * sizeof(T));
    const size_t o_GL0 = take(n3 * sizeof(T));
    const size_t o_GLd = take(n3 * sizeof(T));
    const size_t o_W = take((size_t)N * N * 2 * sizeof(T));
    bytes = off;
    blob.assign(off, 0);
    auto put = [&](size_t o, const std::vector<double>& v) {
        T* d = reinterpret_cast<T*>(blob.data() + o);
        for (size_t i = 0; i < v.size(); ++i) d[i] = (T)v[i];
    };
    auto putd = [&](size_t o, const std::vector<double>& v) {
        std::memcpy(blob.data() + o, v.data(), v.size() * sizeof(double));
    };
    put(o_filt, h.filt);
    put(o_wsig, h.wsig);
    putd(o_cr, h.cr);
    putd(o_wr, h.wr);
    put(o_Uk, h.Uk);
    {
        // the radial kernel factors depend on |k|^2 only: a compact copy indexed by it
        T* d = reinterpret_cast<T*>(blob.data() + o_Uq);
        auto sk = [N](int q) { return q < N / 2 ? q : q - N; };
        for (size_t i = 0; i < n3; ++i) {
            const int kx = sk((int)(i / ((size_t)N * N))), ky = sk((int)((i / N) % N)), kz = sk((int)(i % N));
            const int q2 = kx * kx + ky * ky + kz * kz;
            for (int s = 0; s < h.rank; ++s) d[(size_t)s * nq2 + q2] = (T)h.Uk[(size_t)s * n3 + i];
        }
    }
    put(o_Vr, h.Vr);
    put(o_Lr, h.Lr);
    {
        // loss multiplier of the plan's kernel and its gamma-derivative, summed over r in FP64
        std::vector<double> g0(n3, 0.0), gd(n3, 0.0);
        for (int r = 0; r < h.Nrho; ++r) {
            const double rho = 4.0 * 3.14159265358979323846 * h.b * std::pow(h.cr[r], h.gamma + 2.0);
            const double lrho = std::log(h.cr[r]) * rho;
            for (size_t i = 0; i < n3; ++i) {
                g0[i] += rho * h.Lr[(size_t)r * n3 + i];
                gd[i] += lrho * h.Lr[(size_t)r * n3 + i];
            }
        }
        put(o_GL0, g0);
        put(o_GLd, gd);
    }
    {
        T* W = reinterpret_cast<T*>(blob.data() + o_W);
        const double tp = 2.0 * 3.14159265358979323846 / N;
        for (int q = 0; q < N; ++q)
            for (int j = 0; j < N; ++j) {
                const long m = ((long)q * j) % N;
                W[2 * (q * N + j)] = (T)std::cos(tp * m);
                W[2 * (q * N + j) + 1] = (T)(-std::sin(tp * m));
            }
    }
    t.N = N;
    t.Nrho = h.Nrho;
    t.npairs = h.npairs;
    t.rank = h.rank;
    // device pointers are set after the upload: store offsets for now
    t.filt = reinterpret_cast<const T*>(o_filt);
    t.wsig = reinterpret_cast<const T*>(o_wsig);
    t.cr = reinterpret_cast<const double*>(o_cr);
    t.wr = reinterpret_cast<const double*>(o_wr);
    t.Uk = reinterpret_cast<const T*>(o_Uk);
    t.Uq = reinterpret_cast<const T*>(o_Uq);
    t.Vr = reinterpret_cast<const T*>(o_Vr);
    t.Lr = reinterpret_cast<const T*>(o_Lr);
    t.GL0 = reinterpret_cast<const T*>(o_GL0);
    t.GLd = reinterpret_cast<const T*>(o_GLd);
    t.dftw = reinterpret_cast<const T*>(o_W);
}

// VSS tables in the compute type: A = w_r w_p F(k, c_r, sigma_p), the loss weight, the multipliers;
// A and the loss weight plane-major ([kz][kx][ky]) for the fused kernels.
template <typename T>
void fill_vss_tables(const HostPlan& h, bool planes, std::vector<unsigned char>& blob) {
    const int N = h.N;
    const size_t n3 = (size_t)N * N * N;
    blob.assign((h.Fa.size() + h.GLa.size() + h.mu.size()) * sizeof(T), 0);
    T* d = reinterpret_cast<T*>(blob.data());
    auto dst = [&](size_t i) {   // standard index (kx N + ky) N + kz -> stored index
        if (!planes) return i;
        const size_t kx = i / ((size_t)N * N), ky = (i / N) % N, kz = i % N;
        return (kz * N + kx) * N + ky;
    };
    for (size_t f = 0; f < h.Fa.size() / n3; ++f)
        for (size_t i = 0; i < n3; ++i) d[f * n3 + dst(i)] = (T)h.Fa[f * n3 + i];
    d += h.Fa.size();
    for (size_t i = 0; i < n3; ++i) d[dst(i)] = (T)h.GLa[i];
    d += n3;
    for (size_t i = 0; i < h.mu.size(); ++i) d[i] = (T)h.mu[i];
}

template <typename T>
void rebase(DevTables<T>& t, void* base) {
    auto fix = [&](auto& ptr) {
        using P = std::remove_reference_t<decltype(ptr)>;
        ptr = reinterpret_cast<P>(static_cast<unsigned char*>(base) + reinterpret_cast<uintptr_t>(ptr));
    };
    fix(t.filt); fix(t.wsig); fix(t.cr); fix(t.wr); fix(t.Uk); fix(t.Uq); fix(t.Vr); fix(t.Lr); fix(t.GL0); fix(t.GLd);
    fix(t.dftw);
}

template <typename T> DevTables<T>& tables(dgfs_plan_s* p);
template <> DevTables<float>& tables<float>(dgfs_plan_s* p) { return p->tf; }
template <> DevTables<double>& tables<double>(dgfs_plan_s* p) { return p->td; }

unsigned char* ws(dgfs_plan_s* p, size_t off) { return static_cast<unsigned char*>(p->d_ws) + off; }

enum class Op { Collide, Collide2, Jvp, Dgamma, Vjp };

// The VSS kernel (alpha != 1): gain^ = scale sum_r sum_p A_rp DFT(products of the translates by
// +-s_rp), one transform per radial and sphere point (k_vss.cu), in batches of vchunk nodes;
// loss and finalisation as for VHS: out = Re gain - a Re(GL * b) [- b Re(GL * a) for the JVP].
template <typename T>
dgfs_status vss_chunk(dgfs_plan_s* p, Op op, const T* f, const T* g, T* out, const int64_t* offs, int64_t nodes,
                      cudaStream_t s) {
    if (op == Op::Vjp || op == Op::Dgamma)
        return fail(DGFS_ERR_UNSUPPORTED, "the VSS kernel (alpha != 1) supports Q(f,f), Q(f,g) and the JVP");
    NvtxRange range("dgfs VSS chunk");
    if (offs) return fail(DGFS_ERR_UNSUPPORTED, "the VSS kernel (alpha != 1) takes no node offsets");
    const DevTables<T>& t = tables<T>(p);
    const int N = t.N, np = t.npairs, Nr = t.Nrho, nw = (np + 1) / 2;
    const int64_t n3 = (int64_t)N * N * N;
    // equal transform batches of at most vchunk nodes (no small ragged tail batch)
    const int64_t nbatch = (nodes + p->vchunk - 1) / std::max<int64_t>(1, p->vchunk);
    const int64_t C = nbatch > 0 ? (nodes + nbatch - 1) / nbatch : p->vchunk;
    const bool two = op != Op::Collide;
    const int sets = two ? 2 : 1, yf = op == Op::Jvp ? 3 : 2;
    const T scale = op == Op::Jvp ? T(2) : T(1);
    const T* a = f;
    const T* b = two ? g : f;
    Cplx<T>* Fh = reinterpret_cast<Cplx<T>*>(ws(p, p->off_V));
    Cplx<T>* Gh = Fh + C * n3;
    Cplx<T>* Z = Gh + C * n3;
    Cplx<T>* W = Z + C * 2 * np * n3;
    Cplx<T>* Y = W + C * nw * n3;
    const T* A = static_cast<const T*>(p->d_vss);
    const T* GL = A + (size_t)Nr * np * n3;
    const Cplx<T>* mu = reinterpret_cast<const Cplx<T>*>(GL + n3);
    const Cplx<T>* dftw = reinterpret_cast<const Cplx<T>*>(t.dftw);
    for (int64_t n0 = 0; n0 < nodes; n0 += C) {
        const int64_t nn = std::min<int64_t>(C, nodes - n0);
        cudaError_t e = launch_vss_load_t<T>(a + n0 * n3, nullptr, N, nn, Fh, s);
        if (!e) e = launch_dft3<T>(t, Fh, nn, true, s);
        if (!e && two) e = launch_vss_load_t<T>(b + n0 * n3, nullptr, N, nn, Gh, s);
        if (!e && two) e = launch_dft3<T>(t, Gh, nn, true, s);
        if (!e) e = launch_vss_loss_init<T>(Fh, two ? Gh : Fh, GL, N, nn, Y, yf, s);
        if (e) return cuda_fail(e, "VSS operand transforms");
        for (int r = 0; r < Nr && !e; ++r) {
            e = launch_vss_inverse_planes<T>(Fh, two ? Gh : nullptr, mu + (size_t)r * np * 3 * N, dftw, N, np, sets, nn,
                                             Z, s);
            if (!e) e = launch_vss_lines<T>(Z, dftw, N, np, sets, nn, W, s);
            if (!e) e = launch_vss_forward_planes<T>(dftw, N, nw, nn, W, s);
            if (!e) e = launch_vss_accumulate<T>(W, A + (size_t)r * np * n3, N, np, nn, scale, Y, yf, s);
        }
        if (e) return cuda_fail(e, "VSS gain");
        e = launch_dft3<T>(t, Y, nn * yf, false, s);
        if (!e) e = launch_vss_finalize_t<T>(Y, yf, a + n0 * n3, op == Op::Jvp ? b + n0 * n3 : nullptr, N, nn,
                                             out + n0 * n3, p->d_flags, s);
        if (e) return cuda_fail(e, "VSS loss and finalisation");
        if (p->prof) {
            p->prof_launches += (two ? 8 : 4) + 1 + (int64_t)Nr * 4 + 4;
            p->prof_nodes += nn;
        }
    }
    return DGFS_OK;
}

// P[node][r] = sum_p w_p [(T_s f)(T_-s g) + (T_-s f)(T_s g)] with the translates taken in Fourier
// space (k_vss.cu: one complex inverse transform gives T_s f + i T_-s g), in batches of xchunk nodes;
// the same P as the dense circulant passes of launch_gain_products at a fifth of the arithmetic.
template <typename T>
cudaError_t fft_gain_products(dgfs_plan_s* p, const T* f, const T* g, const int64_t* offs, int64_t nodes, T* P,
                              cudaStream_t s) {
    const DevTables<T>& t = tables<T>(p);
    const int N = t.N, np = t.npairs, Nr = t.Nrho, sets = g ? 2 : 1;
    const int64_t n3 = (int64_t)N * N * N, C = p->xchunk;
    Cplx<T>* Fh = reinterpret_cast<Cplx<T>*>(ws(p, p->off_Xt));
    Cplx<T>* Gh = Fh + C * n3;
    Cplx<T>* Z = Gh + C * n3;
    const Cplx<T>* mu = static_cast<const Cplx<T>*>(p->d_mu);
    const Cplx<T>* dftw = reinterpret_cast<const Cplx<T>*>(t.dftw);
    for (int64_t n0 = 0; n0 < nodes; n0 += C) {
        const int64_t nn = std::min<int64_t>(C, nodes - n0);
        cudaError_t e = offs ? launch_vss_load_t<T>(f, offs + n0, N, nn, Fh, s)
                             : launch_vss_load_t<T>(f + n0 * n3, nullptr, N, nn, Fh, s);
        if (!e) e = launch_dft3<T>(t, Fh, nn, true, s);
        if (!e && g) e = offs ? launch_vss_load_t<T>(g, offs + n0, N, nn, Gh, s)
                              : launch_vss_load_t<T>(g + n0 * n3, nullptr, N, nn, Gh, s);
        if (!e && g) e = launch_dft3<T>(t, Gh, nn, true, s);
        for (int r = 0; r < Nr && !e; ++r) {
            e = launch_vss_inverse_planes<T>(Fh, g ? Gh : nullptr, mu + (size_t)r * np * 3 * N, dftw, N, np, sets, nn,
                                             Z, s);
            if (!e) e = launch_vss_lines_sum<T>(Z, dftw, t.wsig, N, np, sets, nn, (int64_t)Nr * n3,
                                                P + n0 * Nr * n3 + (int64_t)r * n3, s);
        }
        if (e) return e;
        if (p->prof) p->prof_launches += (g ? 8 : 4) + 2 * (int64_t)Nr;
    }
    return cudaSuccess;
}

// Adjoint gain sum_r G_r (G_r = sum_p 2 w_p [T_-s(U_r T_-s f) + T_s(U_r T_s f)], U[node][r] = K_r u)
// with the translates and back-translates in Fourier space (k_vss.cu), in batches of xchunk nodes:
// Gsum [nodes][N^3], standard layout.
template <typename T>
cudaError_t fft_vjp_products(dgfs_plan_s* p, const T* f, const T* U, int64_t nodes, T* Gsum, cudaStream_t s) {
    const DevTables<T>& t = tables<T>(p);
    const int N = t.N, np = t.npairs, Nr = t.Nrho;
    const int64_t n3 = (int64_t)N * N * N, C = p->xchunk;
    Cplx<T>* Fh = reinterpret_cast<Cplx<T>*>(ws(p, p->off_Xt));
    Cplx<T>* Gh = Fh + C * n3;
    Cplx<T>* Z = Gh + C * n3;
    Cplx<T>* W = Z + C * np * n3;
    const Cplx<T>* mu = static_cast<const Cplx<T>*>(p->d_mu);
    const Cplx<T>* dftw = reinterpret_cast<const Cplx<T>*>(t.dftw);
    for (int64_t n0 = 0; n0 < nodes; n0 += C) {
        const int64_t nn = std::min<int64_t>(C, nodes - n0);
        cudaError_t e = launch_vss_load_t<T>(f + n0 * n3, nullptr, N, nn, Fh, s);
        if (!e) e = launch_dft3<T>(t, Fh, nn, true, s);
        if (!e) e = cudaMemsetAsync(Gh, 0, (size_t)nn * n3 * sizeof(Cplx<T>), s);
        for (int r = 0; r < Nr && !e; ++r) {
            const Cplx<T>* mu_r = mu + (size_t)r * np * 3 * N;
            e = launch_vss_inverse_planes<T>(Fh, nullptr, mu_r, dftw, N, np, 1, nn, Z, s);
            if (!e) e = launch_vjp_lines<T>(Z, U + n0 * Nr * n3 + (int64_t)r * n3, (int64_t)Nr * n3, dftw, N, np, nn, W, s);
            if (!e) e = launch_vss_forward_planes<T>(dftw, N, np, nn, W, s);
            if (!e) e = launch_vjp_accumulate<T>(W, mu_r, t.wsig, N, np, nn, Gh, s);
        }
        if (!e) e = launch_dft3<T>(t, Gh, nn, false, s);
        if (!e) e = launch_vjp_real_t<T>(Gh, N, nn, Gsum + n0 * n3, s);
        if (e) return e;
        if (p->prof) p->prof_launches += 4 + 4 * (int64_t)Nr + 4;
    }
    return cudaSuccess;
}

// One chunk of nodes through the whole pipeline. a/b/f_loss are chunk-base pointers.
template <typename T>
dgfs_status run_chunk(dgfs_plan_s* p, Op op, const T* f, const T* g, T* out, const int64_t* offs,
                      NodeParams np, int64_t nodes, cudaStream_t s) {
    if (p->hp.aniso) return vss_chunk<T>(p, op, f, g, out, offs, nodes, s);
    NvtxRange chunk_range("dgfs chunk");
    const DevTables<T>& t = tables<T>(p);
    const int xf = p->xfields;
    T* P = reinterpret_cast<T*>(ws(p, p->off_P));
    Cplx<T>* X = reinterpret_cast<Cplx<T>*>(ws(p, p->off_X));
    Cplx<T>* Y = reinterpret_cast<Cplx<T>*>(ws(p, p->off_Y));
    const int rank = t.rank;
    cudaError_t e;
    if (op == Op::Vjp) {
        // g holds u. 1) K_r u for every r:  DFT(u) -> Uk[s] u^ -> IDFT -> sum_s Vr w_r rho_r
        e = launch_load_field<T>(t.N, g, nullptr, offs, nodes, X, xf, rank, 0, s);
        if (!e) e = launch_dft3<T>(t, X + (size_t)0, nodes * xf, true, s);
        if (!e) e = launch_multiply_uk<T>(t, X, xf, rank, nodes, s);
        if (!e) e = launch_dft3<T>(t, X, nodes * xf, false, s);
        if (!e) e = launch_expand_radial<T>(t, X, xf, np, nodes, P, s);
        if (e) return cuda_fail(e, "vjp: radial multipliers");
        // 2) adjoint translate-products, summed over r, with the translates in Fourier space
        T* G = reinterpret_cast<T*>(ws(p, p->off_G));
        if (offs) return fail(DGFS_ERR_UNSUPPORTED, "vjp with node offsets");
        if (!p->fftx) return fail(DGFS_ERR_UNSUPPORTED, "vjp: no Fourier-space translates for this plan");
        if (p->prof) p->prof_nodes += nodes;
        e = fft_vjp_products<T>(p, f, P, nodes, G, s);
        if (e) return cuda_fail(e, "vjp: translate-product kernels");
        // 3) loss: K_L f + i K_L (u f)
        e = launch_load_field<T>(t.N, f, nullptr, offs, nodes, X, xf, 0, 0, s);
        if (!e) e = launch_load_field<T>(t.N, f, g, offs, nodes, X, xf, 1, 0, s);
        if (!e) e = launch_dft3<T>(t, X, nodes * xf, true, s);
        if (!e) e = launch_loss_pair<T>(t, X, xf, np, nodes, 0, 1, Y, 2, s);
        if (!e) e = launch_dft3<T>(t, Y, nodes * 2, false, s);
        // the Fourier-space adjoint leaves the radial sum in G (one field per node)
        if (!e) e = launch_finalize<T>(t.N, 1, Y, 2, g, nullptr, G, offs, nodes, 1, out, p->d_flags, s);
        if (e) return cuda_fail(e, "vjp: loss and finalisation");
        return DGFS_OK;
    }
    // gain products: Q(f,f) and dQ/dgamma use (f, f); Q(f,g) uses (f, g); JVP uses (f, v)
    const T* gg = (op == Op::Collide || op == Op::Dgamma) ? nullptr : g;
    NvtxRange translate_range("dgfs translate products");
    if (p->prof) {
        p->prof_launches += (spectral_supported(tables<T>(p)) ? 5 : 11 + (op == Op::Jvp ? 1 : 0)) +
                            tc_extra_launches(p->prec);
        p->prof_gain += 1;
        p->prof_nodes += nodes;
        if (p->prof_timed < (int64_t)p->ev.size() / 2) cudaEventRecord(p->ev[2 * p->prof_timed], s);
    }
    if (is_tc(p->prec) && std::is_same<T, float>::value && gg == nullptr) {
        e = launch_tc_gain_products(p->tc, p->prec, reinterpret_cast<const float*>(f),
                                    reinterpret_cast<const float*>(gg), offs, nodes,
                                    reinterpret_cast<float*>(P), p->d_flags, s, p->fault);
        p->fault = 0;
    } else if (is_tc(p->prec) && std::is_same<T, float>::value && offs == nullptr) {
        // bilinear calls (Q(f, g), the JVP) on the tensor cores: the translate-product sum is symmetric in
        // (f, g), so P(f, g) = [P(f + a g) - P(f - a g)] / (4 a), two quadratic launches; the operands u and
        // the per-node factors live in the Fourier slots' workspace, which the Fourier stage fills only later
        const int64_t n3 = (int64_t)t.N * t.N * t.N;
        float* U = reinterpret_cast<float*>(X);
        float* coef = U + 2 * nodes * n3;
        e = launch_polar_prep(reinterpret_cast<const float*>(f), reinterpret_cast<const float*>(gg), n3, nodes, U, coef, s);
        if (!e) e = launch_tc_gain_products(p->tc, p->prec, U, nullptr, nullptr, nodes, reinterpret_cast<float*>(P),
                                            p->d_flags, s, 0, coef, 0);
        if (!e) e = launch_tc_gain_products(p->tc, p->prec, U + nodes * n3, nullptr, nullptr, nodes,
                                            reinterpret_cast<float*>(P), p->d_flags, s, 0, coef + nodes, 1);
        if (p->prof) p->prof_launches += 2;
    } else if (p->fftx) {
        e = fft_gain_products<T>(p, f, gg, offs, nodes, P, s);
    } else {
        e = launch_gain_products(t, f, gg, offs, nodes, P, s);
    }
    if (e) return cuda_fail(e, "translate-product kernel");
    translate_range.end();
    NvtxRange fourier_range("dgfs Fourier stage");
    if (p->prof && p->prof_timed < (int64_t)p->ev.size() / 2) {
        cudaEventRecord(p->ev[2 * p->prof_timed + 1], s);
        p->prof_timed += 1;
    }
    // real fields packed two per complex slot: the rank projected fields, then the loss
    // operand(s): Q(f,g) -> field rank = g;  JVP -> field rank = v, field rank + 1 = f
    if (spectral_supported(t)) {   // the fused three-launch Fourier stage
        const T* la = (op == Op::Collide || op == Op::Dgamma) ? f : g;
        e = launch_spectral<T>(t, P, np, nodes, la, op == Op::Jvp ? f : nullptr, offs,
                               op == Op::Jvp ? T(2) : T(1), X, Y, f, op == Op::Jvp ? g : nullptr, out,
                               p->d_flags, s);
        if (e) return cuda_fail(e, "Fourier stage");
        return DGFS_OK;
    }
    const int nfields = rank + (op == Op::Jvp ? 2 : 1), xs = (nfields + 1) / 2;
    e = launch_project<T>(t, P, np, nodes, X, xs, s);
    if (e) return cuda_fail(e, "radial projection");
    const T* loss0 = (op == Op::Collide || op == Op::Dgamma) ? f : g;
    e = launch_load_field<T>(t.N, loss0, nullptr, offs, nodes, X, xs, rank / 2, rank % 2, s);
    if (!e && op == Op::Jvp) e = launch_load_field<T>(t.N, f, nullptr, offs, nodes, X, xs, (rank + 1) / 2, (rank + 1) % 2, s);
    if (e) return cuda_fail(e, "loss operand");
    // forward DFT of the packed slots
    e = launch_dft3<T>(t, X, nodes * xs, true, s);
    if (e) return cuda_fail(e, "forward DFT");
    const T scale = op == Op::Jvp ? T(2) : T(1);
    const int yf = op == Op::Jvp ? 3 : 2;
    e = launch_combine<T>(t, X, xs, np, nodes, scale, rank, op == Op::Jvp ? rank + 1 : -1, Y, yf, s);
    if (!e) e = launch_dft3<T>(t, Y, nodes * yf, false, s);
    if (e) return cuda_fail(e, "Fourier combine / inverse DFT");
    // Q = gain - f (K_L g)   (JVP: 2 gain(f,v) - f K_L v - v K_L f)
    e = launch_finalize<T>(t.N, t.Nrho, Y, yf, f, op == Op::Jvp ? g : nullptr, nullptr, offs, nodes, 0,
                           out, p->d_flags, s);
    if (e) return cuda_fail(e, "finalisation");
    return DGFS_OK;
}

template <typename T>
dgfs_status run(dgfs_plan_s* p, Op op, const void* f, const void* g, void* out, int64_t B,
                cudaStream_t s) {
    const int64_t n3 = (int64_t)p->hp.N * p->hp.N * p->hp.N;
    DGFS_ON_DEVICE(p->device);
    NodeParams np{nullptr, nullptr, p->hp.gamma, p->hp.b, op == Op::Dgamma ? 1 : 0};
    const int64_t C = p->run_chunk > 0 ? std::min<int64_t>(p->run_chunk, p->chunk) : p->chunk;
    for (int64_t n0 = 0; n0 < B; n0 += C) {
        const int64_t nn = std::min<int64_t>(C, B - n0);
        const T* fc = static_cast<const T*>(f) + n0 * n3;
        const T* gc = g ? static_cast<const T*>(g) + n0 * n3 : nullptr;
        T* oc = static_cast<T*>(out) + n0 * n3;
        const dgfs_status st = run_chunk<T>(p, op, fc, gc, oc, nullptr, np, nn, s);
        if (st != DGFS_OK) return st;
    }
    return DGFS_OK;
}

dgfs_status compute(dgfs_plan_t plan, Op op, const void* f, const void* g, void* out, int64_t B,
                    void* stream, bool need_g) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (B < 0) return fail(DGFS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return DGFS_OK;
    if (!f || !out || (need_g && !g)) return fail(DGFS_ERR_INVALID_ARG, "NULL field pointer");
    if (!aligned16(f) || !aligned16(out) || (g && !aligned16(g)))
        return fail(DGFS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (out == f || (g && out == g)) return fail(DGFS_ERR_INVALID_ARG, "output aliases an input");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return plan->prec == DGFS_PREC_FP64 ? run<double>(plan, op, f, g, out, B, s)
                                        : run<float>(plan, op, f, g, out, B, s);
}

}  // namespace

// ---- exported API ------------------------------------------------------------------------

extern "C" {

const char* dgfs_last_error_message(void) { return g_last_error.c_str(); }

dgfs_status dgfs_plan_desc_init(dgfs_plan_desc* d) {
    if (!d) return fail(DGFS_ERR_INVALID_ARG, "NULL descriptor");
    std::memset(d, 0, sizeof(*d));
    d->N = 32;
    d->L = 7.0;
    d->R = 0.0;
    d->gamma = 0.0;
    d->b = 0.0;
    d->M = 38;
    d->sphere_xyzw = nullptr;
    d->N_rho = 0;
    d->svd_tol = 0.0;
    d->svd_rank = 0;
    d->precision = DGFS_PREC_FP32;
    d->loss_mode = DGFS_LOSS_PAPER;
    d->max_batch = 0;
    d->alpha = 0.0;
    return DGFS_OK;
}

dgfs_status dgfs_plan_create(const dgfs_plan_desc* desc, dgfs_plan_t* plan_out) {
    if (!desc || !plan_out) return fail(DGFS_ERR_INVALID_ARG, "NULL argument");
    *plan_out = nullptr;
    if (desc->precision < DGFS_PREC_FP64 || desc->precision > DGFS_PREC_BF16X3)
        return fail(DGFS_ERR_INVALID_ARG, "unknown precision");
    std::unique_ptr<dgfs_plan_s> p(new (std::nothrow) dgfs_plan_s);
    if (!p) return fail(DGFS_ERR_OOM, "host allocation failed");
    std::string err;
    dgfs_status st = build_host_plan(*desc, p->hp, err);
    if (st != DGFS_OK) return fail(st, err);
    p->prec = desc->precision;
    if (p->hp.aniso && !vss_fused_supported(p->hp.N, p->prec == DGFS_PREC_FP64))
        return fail(DGFS_ERR_UNSUPPORTED, "the VSS kernel supports N <= 24 in FP64");
    if (is_tc(p->prec) && !tc_supported(p->hp.N, p->prec))
        return fail(DGFS_ERR_UNSUPPORTED, "tensor-core precisions support N = 16 and 32 (F16S and BF16S also N = 24)");
    if (p->hp.aniso && is_tc(p->prec))
        return fail(DGFS_ERR_UNSUPPORTED, "the VSS kernel (alpha != 1) runs in FP64 or FP32");
    DGFS_CUDA(cudaGetDevice(&p->device), "cudaGetDevice");
    // chunk: about 1.5 GB of workspace
    {
        dgfs_plan_s probe;
        probe.hp.N = p->hp.N;
        probe.hp.Nrho = p->hp.Nrho;
        probe.hp.rank = p->hp.rank;
        probe.hp.npairs = p->hp.npairs;
        probe.hp.aniso = p->hp.aniso;
        probe.prec = p->prec;
        probe.vchunk = 0;
        workspace_layout(&probe, 1);
        const size_t per_node = probe.ws_bytes;
        int64_t C = (int64_t)((size_t)4096 << 20) / (int64_t)per_node;   // about 4 GB of workspace
        C = std::max<int64_t>(1, std::min<int64_t>(C, 4096));
        if (desc->max_batch > 0) C = std::min<int64_t>(desc->max_batch, (int64_t)1 << 20);   // the caller's choice
        p->chunk = C;
        if (p->hp.aniso) {
            // transform batches of about 1.5 GB of translate spectra and products: enough CTAs per launch
            // (64 MB, which stays in L2, measured 3.2k node-evals/s at N = 32; 512 MB 6.0k; 1.5 GB 6.7k)
            const size_t n3 = (size_t)p->hp.N * p->hp.N * p->hp.N;
            const size_t zw = 2 * elem_size(p->prec) * n3 * (2 * (size_t)p->hp.npairs + (p->hp.npairs + 1) / 2);
            p->vchunk = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(C, (int64_t)(((size_t)1536 << 20) / zw)), 65535));
        }
    }
    // tensor-core plans keep their kernel for Q(f, f) and dQ/dgamma; their bilinear calls (Q(f, g),
    // the JVP) and the VJP take the Fourier-space translates in FP32 like the FP32 plans
    p->fftx = !p->hp.aniso && fft_translate_supported(p->hp.N);
    if (p->fftx) {
        // transform batches of about 1.5 GB of operand and translate spectra
        const size_t n3 = (size_t)p->hp.N * p->hp.N * p->hp.N;
        const size_t per = (2 + 2 * (size_t)p->hp.npairs) * n3 * 2 * elem_size(p->prec);
        p->xchunk = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(p->chunk, (int64_t)(((size_t)1536 << 20) / per)),
                                                           65535));
    }
    workspace_layout(p.get(), p->chunk);
    std::vector<unsigned char> blob;
    if (p->prec == DGFS_PREC_FP64) fill_tables<double>(p.get(), blob, p->td, p->table_bytes);
    else fill_tables<float>(p.get(), blob, p->tf, p->table_bytes);
    std::vector<unsigned char> tcblob;
    size_t tc_bytes = 0;
    if (is_tc(p->prec)) tc_bytes = build_tc_tables(p->hp, p->prec, tcblob, p->tc);
    if (p->hp.aniso) {
        std::vector<unsigned char> vblob;
        p->vss_planes = vss_fused_supported(p->hp.N, p->prec == DGFS_PREC_FP64);
        if (p->prec == DGFS_PREC_FP64) fill_vss_tables<double>(p->hp, p->vss_planes, vblob);
        else fill_vss_tables<float>(p->hp, p->vss_planes, vblob);
        cudaError_t ev = cudaMalloc(&p->d_vss, vblob.size());
        if (ev != cudaSuccess) return fail(DGFS_ERR_OOM, std::string("VSS tables: ") + cudaGetErrorString(ev));
        ev = cudaMemcpy(p->d_vss, vblob.data(), vblob.size(), cudaMemcpyHostToDevice);
        if (ev != cudaSuccess) {
            cudaFree(p->d_vss);
            return cuda_fail(ev, "VSS table upload");
        }
        p->vss_bytes = vblob.size();
        p->d_mu = static_cast<unsigned char*>(p->d_vss) + (p->hp.Fa.size() + p->hp.GLa.size()) * elem_size(p->prec);
        // the FP64 host copies are no longer needed
        std::vector<double>().swap(p->hp.Fa);
        std::vector<double>().swap(p->hp.mu);
    } else if (p->fftx) {
        const size_t es = elem_size(p->prec);
        std::vector<unsigned char> mblob(p->hp.mu.size() * es);
        for (size_t i = 0; i < p->hp.mu.size(); ++i) {
            if (es == 8) reinterpret_cast<double*>(mblob.data())[i] = p->hp.mu[i];
            else reinterpret_cast<float*>(mblob.data())[i] = (float)p->hp.mu[i];
        }
        cudaError_t ev = cudaMalloc(&p->d_vss, mblob.size());
        if (ev != cudaSuccess) return fail(DGFS_ERR_OOM, std::string("translate multipliers: ") + cudaGetErrorString(ev));
        ev = cudaMemcpy(p->d_vss, mblob.data(), mblob.size(), cudaMemcpyHostToDevice);
        if (ev != cudaSuccess) {
            cudaFree(p->d_vss);
            return cuda_fail(ev, "translate multiplier upload");
        }
        p->vss_bytes = mblob.size();
        p->d_mu = p->d_vss;
    }
    cudaError_t e = cudaMalloc(&p->d_tables, p->table_bytes + tc_bytes);
    if (e != cudaSuccess) {
        if (p->d_vss) cudaFree(p->d_vss);
        return fail(DGFS_ERR_OOM, std::string("device tables: ") + cudaGetErrorString(e));
    }
    e = cudaMalloc(&p->d_ws, p->ws_bytes);
    if (e != cudaSuccess) {
        cudaFree(p->d_tables);
        if (p->d_vss) cudaFree(p->d_vss);
        return fail(DGFS_ERR_OOM, std::string("device workspace: ") + cudaGetErrorString(e));
    }
    e = cudaMalloc(&p->d_flags, 64);
    if (e == cudaSuccess) e = cudaMemset(p->d_flags, 0, 64);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tables, blob.data(), p->table_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && tc_bytes)
        e = cudaMemcpy(static_cast<unsigned char*>(p->d_tables) + p->table_bytes, tcblob.data(), tc_bytes,
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->d_tables);
        cudaFree(p->d_ws);
        if (p->d_flags) cudaFree(p->d_flags);
        if (p->d_vss) cudaFree(p->d_vss);
        return cuda_fail(e, "plan upload");
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cs_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cs_d2h, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&p->ev_start, &p->ev_h2d[0], &p->ev_h2d[1], &p->ev_comp[0], &p->ev_comp[1], &p->ev_d2h[0],
                            &p->ev_d2h[1]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        destroy_io(p.get());
        cudaFree(p->d_tables);
        cudaFree(p->d_ws);
        cudaFree(p->d_flags);
        if (p->d_vss) cudaFree(p->d_vss);
        return cuda_fail(e, "plan streams and events");
    }
    if (p->prec == DGFS_PREC_FP64) rebase(p->td, p->d_tables);
    else rebase(p->tf, p->d_tables);
    if (tc_bytes) rebase_tc_tables(p->tc, static_cast<unsigned char*>(p->d_tables) + p->table_bytes);
    p->table_bytes += tc_bytes + p->vss_bytes;
    *plan_out = p.release();
    return DGFS_OK;
}

dgfs_status dgfs_plan_destroy(dgfs_plan_t plan) {
    if (!plan) return DGFS_OK;
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    {
        DeviceScope scope(plan->device);
        cudaDeviceSynchronize();
        cudaFree(plan->d_tables);
        cudaFree(plan->d_ws);
        cudaFree(plan->d_flags);
        if (plan->d_vss) cudaFree(plan->d_vss);
        for (auto& e : plan->ev) cudaEventDestroy(e);
        destroy_io(plan);
    }
    plan->magic = 0;
    delete plan;
    return DGFS_OK;
}

dgfs_status dgfs_plan_info(dgfs_plan_t plan, dgfs_plan_info_t* info) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (!info) return fail(DGFS_ERR_INVALID_ARG, "NULL info");
    const HostPlan& h = plan->hp;
    info->N = h.N;
    info->N_rho = h.Nrho;
    info->n_pairs = h.npairs;
    info->svd_rank_used = h.rank;
    info->precision = plan->prec;
    info->loss_mode = h.loss_mode;
    info->L = h.L;
    info->R = h.R;
    info->gamma = h.gamma;
    info->b = h.b;
    info->chunk_nodes = plan->chunk;
    info->workspace_bytes = plan->ws_bytes;
    info->table_bytes = plan->table_bytes;
    info->alpha = h.alpha;
    return DGFS_OK;
}

dgfs_status dgfs_collide(dgfs_plan_t plan, const void* f, void* Q, int64_t B, void* stream) {
    return compute(plan, Op::Collide, f, nullptr, Q, B, stream, false);
}

dgfs_status dgfs_collide2(dgfs_plan_t plan, const void* f, const void* g, void* Q, int64_t B,
                          void* stream) {
    return compute(plan, Op::Collide2, f, g, Q, B, stream, true);
}

dgfs_status dgfs_collide_jvp(dgfs_plan_t plan, const void* f, const void* v, void* dQ, int64_t B,
                             void* stream) {
    return compute(plan, Op::Jvp, f, v, dQ, B, stream, true);
}

dgfs_status dgfs_collide_vjp(dgfs_plan_t plan, const void* f, const void* u, void* gf, int64_t B,
                             void* stream) {
    return compute(plan, Op::Vjp, f, u, gf, B, stream, true);
}

dgfs_status dgfs_collide_dgamma(dgfs_plan_t plan, const void* f, void* dQdg, int64_t B, void* stream) {
    return compute(plan, Op::Dgamma, f, nullptr, dQdg, B, stream, false);
}

// Validation shared by the ragged entry points (host arrays).
static dgfs_status check_ragged(const dgfs_plan_t* plans, int nplans, const int32_t* node_plan,
                                const int64_t* node_offset, int64_t B) {
    if (!plans || nplans <= 0) return fail(DGFS_ERR_INVALID_ARG, "no plans");
    for (int i = 0; i < nplans; ++i) {
        if (!check_plan(plans[i])) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
        if (plans[i]->hp.aniso) return fail(DGFS_ERR_UNSUPPORTED, "ragged batches of VSS plans (alpha != 1)");
    }
    for (int i = 1; i < nplans; ++i) {
        if ((plans[i]->prec == DGFS_PREC_FP64) != (plans[0]->prec == DGFS_PREC_FP64))
            return fail(DGFS_ERR_INVALID_ARG, "ragged plans must share the element type");
        if (plans[i]->device != plans[0]->device) return fail(DGFS_ERR_INVALID_ARG, "ragged plans must share the device");
    }
    if (B < 0) return fail(DGFS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return DGFS_OK;
    if (!node_plan || !node_offset) return fail(DGFS_ERR_INVALID_ARG, "NULL argument");
    for (int64_t i = 0; i < B; ++i) {
        if (node_plan[i] < 0 || node_plan[i] >= nplans) return fail(DGFS_ERR_INVALID_ARG, "node_plan out of range");
        if (node_offset[i] < 0) return fail(DGFS_ERR_INVALID_ARG, "negative node_offset");
        if ((node_offset[i] * (int64_t)elem_size(plans[node_plan[i]]->prec)) % 16)
            return fail(DGFS_ERR_INVALID_ARG, "node offsets must keep 16-byte alignment");
    }
    return DGFS_OK;
}

dgfs_status dgfs_collide_ragged(const dgfs_plan_t* plans, int nplans, const int32_t* node_plan,
                                const int64_t* node_offset, const double* node_gamma,
                                const double* node_b, int64_t B, const void* f, void* Q,
                                void* stream) {
    const dgfs_status chk = check_ragged(plans, nplans, node_plan, node_offset, B);
    if (chk != DGFS_OK || B == 0) return chk;
    if (!f || !Q) return fail(DGFS_ERR_INVALID_ARG, "NULL argument");
    if (!aligned16(f) || !aligned16(Q)) return fail(DGFS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (f == Q) return fail(DGFS_ERR_INVALID_ARG, "output aliases the input");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NvtxRange range("dgfs ragged batch");
    for (int pi = 0; pi < nplans; ++pi) {
        dgfs_plan_s* p = plans[pi];
        std::lock_guard<std::mutex> lock(p->host_mu);
        DGFS_ON_DEVICE(p->device);
        std::vector<int64_t> offs;
        std::vector<double> gam, bb;
        for (int64_t i = 0; i < B; ++i)
            if (node_plan[i] == pi) {
                offs.push_back(node_offset[i]);
                gam.push_back(node_gamma ? node_gamma[i] : p->hp.gamma);
                bb.push_back(node_b ? node_b[i] : p->hp.b);
            }
        const int64_t cnt = (int64_t)offs.size();
        for (int64_t n0 = 0; n0 < cnt; n0 += p->chunk) {
            const int64_t nn = std::min<int64_t>(p->chunk, cnt - n0);
            unsigned char* nb = ws(p, p->off_node);
            int64_t* d_offs = reinterpret_cast<int64_t*>(nb);
            double* d_gam = reinterpret_cast<double*>(nb + p->chunk * sizeof(int64_t));
            double* d_b = d_gam + p->chunk;
            DGFS_CUDA(cudaMemcpyAsync(d_offs, offs.data() + n0, nn * sizeof(int64_t), cudaMemcpyHostToDevice, s), "ragged offsets");
            DGFS_CUDA(cudaMemcpyAsync(d_gam, gam.data() + n0, nn * sizeof(double), cudaMemcpyHostToDevice, s), "ragged gamma");
            DGFS_CUDA(cudaMemcpyAsync(d_b, bb.data() + n0, nn * sizeof(double), cudaMemcpyHostToDevice, s), "ragged b");
            NodeParams np{d_gam, d_b, p->hp.gamma, p->hp.b, 0};
            dgfs_status st;
            if (p->prec == DGFS_PREC_FP64)
                st = run_chunk<double>(p, Op::Collide, static_cast<const double*>(f), nullptr,
                                       static_cast<double*>(Q), d_offs, np, nn, s);
            else
                st = run_chunk<float>(p, Op::Collide, static_cast<const float*>(f), nullptr,
                                      static_cast<float*>(Q), d_offs, np, nn, s);
            if (st != DGFS_OK) return st;
        }
        // the host vectors are staged by the copies above before they return (pageable source)
    }
    return DGFS_OK;
}

// ---- ragged schedule: per-class node arrays resident on the device ----------------------------

constexpr uint64_t kRaggedMagic = 0x4447465352414747ull;   // "DGFSRAGG"

struct dgfs_ragged_s {
    uint64_t magic = kRaggedMagic;
    std::vector<dgfs_plan_t> plans;
    std::vector<int64_t> count;        // nodes per plan class
    std::vector<size_t> base;          // first index of the class in the device arrays
    int device = 0;
    void* d_mem = nullptr;             // [B] offsets (int64), [B] gamma, [B] b (double), by class
    // classes with nodes run concurrently, one schedule-owned stream each (forked from and joined
    // back to the caller's stream), when their plans are distinct; else one after the other
    bool concurrent = false;
    std::vector<cudaStream_t> streams; // per class (nullptr for an empty class)
    std::vector<cudaEvent_t> done;     // per class: its work on its stream is enqueued
    cudaEvent_t fork = nullptr;
};

static void ragged_release_streams(dgfs_ragged_s* r) {
    for (cudaStream_t st : r->streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : r->done)
        if (ev) cudaEventDestroy(ev);
    if (r->fork) cudaEventDestroy(r->fork);
    r->streams.clear();
    r->done.clear();
    r->fork = nullptr;
    r->concurrent = false;
}

static bool check_ragged_handle(dgfs_ragged_t r) { return r && r->magic == kRaggedMagic; }

dgfs_status dgfs_ragged_create(const dgfs_plan_t* plans, int nplans, const int32_t* node_plan,
                               const int64_t* node_offset, const double* node_gamma,
                               const double* node_b, int64_t B, dgfs_ragged_t* out) {
    if (!out) return fail(DGFS_ERR_INVALID_ARG, "NULL output handle");
    *out = nullptr;
    const dgfs_status chk = check_ragged(plans, nplans, node_plan, node_offset, B);
    if (chk != DGFS_OK) return chk;
    auto r = std::make_unique<dgfs_ragged_s>();
    r->plans.assign(plans, plans + nplans);
    r->device = plans[0]->device;
    r->count.assign(nplans, 0);
    r->base.assign(nplans, 0);
    for (int64_t i = 0; i < B; ++i) r->count[node_plan[i]]++;
    for (int c = 1; c < nplans; ++c) r->base[c] = r->base[c - 1] + (size_t)r->count[c - 1];
    std::vector<int64_t> offs((size_t)B);
    std::vector<double> gam((size_t)B), bb((size_t)B);
    std::vector<size_t> fill(r->base);
    for (int64_t i = 0; i < B; ++i) {
        const int c = node_plan[i];
        const size_t k = fill[c]++;
        offs[k] = node_offset[i];
        gam[k] = node_gamma ? node_gamma[i] : plans[c]->hp.gamma;
        bb[k] = node_b ? node_b[i] : plans[c]->hp.b;
    }
    if (B > 0) {
        DGFS_ON_DEVICE(r->device);
        const size_t bytes = (size_t)B * (sizeof(int64_t) + 2 * sizeof(double));
        cudaError_t e = cudaMalloc(&r->d_mem, bytes);
        if (e != cudaSuccess) return fail(DGFS_ERR_OOM, "ragged schedule: cudaMalloc failed");
        unsigned char* m = static_cast<unsigned char*>(r->d_mem);
        e = cudaMemcpy(m, offs.data(), (size_t)B * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m + (size_t)B * sizeof(int64_t), gam.data(), (size_t)B * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m + (size_t)B * (sizeof(int64_t) + sizeof(double)), bb.data(), (size_t)B * sizeof(double),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(r->d_mem);
            return cuda_fail(e, "ragged schedule: upload");
        }
        // concurrency: at least two classes with nodes, on distinct plans (each plan owns its
        // workspace, flag word and work-item queue)
        int active = 0;
        bool distinct = true;
        for (int c = 0; c < nplans; ++c) {
            if (r->count[c] == 0) continue;
            ++active;
            for (int d = 0; d < c; ++d)
                if (r->count[d] > 0 && plans[d] == plans[c]) distinct = false;
        }
        if (active >= 2 && distinct) {
            r->streams.assign(nplans, nullptr);
            r->done.assign(nplans, nullptr);
            e = cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming);
            for (int c = 0; c < nplans && e == cudaSuccess; ++c) {
                if (r->count[c] == 0) continue;
                e = cudaStreamCreateWithFlags(&r->streams[c], cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done[c], cudaEventDisableTiming);
            }
            if (e != cudaSuccess) {
                ragged_release_streams(r.get());
                cudaFree(r->d_mem);
                return cuda_fail(e, "ragged schedule: streams");
            }
            r->concurrent = true;
        }
    }
    *out = r.release();
    return DGFS_OK;
}

dgfs_status dgfs_ragged_collide(dgfs_ragged_t r, const void* f, void* Q, void* stream) {
    if (!check_ragged_handle(r)) return fail(DGFS_ERR_STATE, "invalid or destroyed ragged schedule");
    NvtxRange range("dgfs ragged schedule");
    int64_t B = 0;
    for (int64_t c : r->count) B += c;
    if (B == 0) return DGFS_OK;
    if (!f || !Q) return fail(DGFS_ERR_INVALID_ARG, "NULL argument");
    if (!aligned16(f) || !aligned16(Q)) return fail(DGFS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (f == Q) return fail(DGFS_ERR_INVALID_ARG, "output aliases the input");
    for (dgfs_plan_t p : r->plans)
        if (!check_plan(p)) return fail(DGFS_ERR_STATE, "a plan of the ragged schedule was destroyed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* m = static_cast<unsigned char*>(r->d_mem);
    const int64_t* d_offs = reinterpret_cast<const int64_t*>(m);
    const double* d_gam = reinterpret_cast<const double*>(m + (size_t)B * sizeof(int64_t));
    const double* d_b = d_gam + B;
    DGFS_ON_DEVICE(r->device);
    if (r->concurrent) DGFS_CUDA(cudaEventRecord(r->fork, s), "event record");   // work before the call
    dgfs_status result = DGFS_OK;
    for (size_t c = 0; c < r->plans.size(); ++c) {
        dgfs_plan_s* p = r->plans[c];
        if (r->count[c] == 0) continue;
        cudaStream_t sc = s;
        if (r->concurrent) {
            sc = r->streams[c];
            DGFS_CUDA(cudaStreamWaitEvent(sc, r->fork, 0), "stream wait");
        }
        {
            std::lock_guard<std::mutex> lock(p->host_mu);
            for (int64_t n0 = 0; n0 < r->count[c] && result == DGFS_OK; n0 += p->chunk) {
                const int64_t nn = std::min<int64_t>(p->chunk, r->count[c] - n0);
                const size_t k = r->base[c] + (size_t)n0;
                NodeParams np{d_gam + k, d_b + k, p->hp.gamma, p->hp.b, 0};
                result = p->prec == DGFS_PREC_FP64
                    ? run_chunk<double>(p, Op::Collide, static_cast<const double*>(f), nullptr, static_cast<double*>(Q),
                                        d_offs + k, np, nn, sc)
                    : run_chunk<float>(p, Op::Collide, static_cast<const float*>(f), nullptr, static_cast<float*>(Q),
                                       d_offs + k, np, nn, sc);
            }
        }
        if (r->concurrent) {   // joined back to the caller's stream even after a failed launch
            DGFS_CUDA(cudaEventRecord(r->done[c], sc), "event record");
            DGFS_CUDA(cudaStreamWaitEvent(s, r->done[c], 0), "stream wait");
        }
        if (result != DGFS_OK) return result;
    }
    return DGFS_OK;
}

dgfs_status dgfs_ragged_destroy(dgfs_ragged_t r) {
    if (!r) return DGFS_OK;
    if (!check_ragged_handle(r)) return fail(DGFS_ERR_STATE, "invalid or destroyed ragged schedule");
    {
        DeviceScope scope(r->device);
        cudaDeviceSynchronize();
        ragged_release_streams(r);
        cudaFree(r->d_mem);
    }
    r->magic = 0;
    delete r;
    return DGFS_OK;
}

// ---- space-homogeneous SSP-RK time stepping and moments (Secs. 3.3, 3.5) ----------------------

}  // extern "C"

namespace {

// Stages (eqs. SSPRK2, SSPRK3) with L(u) = scale Q(u, u) evaluated by run_chunk into q:
//   v1 = u + dt L(u)
//   RK2: u <- 1/2 u + 1/2 v1 + 1/2 dt L(v1)
//   RK3: v2 = 3/4 u + 1/4 v1 + 1/4 dt L(v1);  u <- 1/3 u + 2/3 v2 + 2/3 dt L(v2)
template <typename T>
dgfs_status ssprk_run(dgfs_plan_s* p, int order, T* f, int64_t B, double dt, double scale, int nsteps,
                      cudaStream_t s) {
    const int64_t n3 = (int64_t)p->hp.N * p->hp.N * p->hp.N;
    T* stage = reinterpret_cast<T*>(ws(p, p->off_io));   // the staging area holds 2 chunks of fields
    T* q = stage + p->chunk * n3;
    const NodeParams np{nullptr, nullptr, p->hp.gamma, p->hp.b, 0};
    const double h = dt * scale;
    for (int64_t n0 = 0; n0 < B; n0 += p->chunk) {
        const int64_t nn = std::min<int64_t>(p->chunk, B - n0), n = nn * n3;
        T* u = f + n0 * n3;
        for (int it = 0; it < nsteps; ++it) {
            dgfs_status st = run_chunk<T>(p, Op::Collide, u, nullptr, q, nullptr, np, nn, s);
            if (st != DGFS_OK) return st;
            cudaError_t e = launch_rk_combine<T>(n, 1.0, u, 0.0, nullptr, h, q, stage, p->d_flags, s);
            if (e) return cuda_fail(e, "SSP-RK stage");
            st = run_chunk<T>(p, Op::Collide, stage, nullptr, q, nullptr, np, nn, s);
            if (st != DGFS_OK) return st;
            if (order == 2) {
                e = launch_rk_combine<T>(n, 0.5, u, 0.5, stage, 0.5 * h, q, u, p->d_flags, s);
            } else {
                e = launch_rk_combine<T>(n, 0.75, u, 0.25, stage, 0.25 * h, q, stage, p->d_flags, s);
                if (!e) {
                    st = run_chunk<T>(p, Op::Collide, stage, nullptr, q, nullptr, np, nn, s);
                    if (st != DGFS_OK) return st;
                    e = launch_rk_combine<T>(n, 1.0 / 3.0, u, 2.0 / 3.0, stage, 2.0 / 3.0 * h, q, u, p->d_flags, s);
                }
            }
            if (e) return cuda_fail(e, "SSP-RK stage");
            if (p->prof) p->prof_launches += order;
        }
    }
    return DGFS_OK;
}

}  // namespace

extern "C" {

dgfs_status dgfs_ssprk(dgfs_plan_t plan, int order, void* f, int64_t B, double dt, double scale, int nsteps,
                       void* stream) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (order != 2 && order != 3) return fail(DGFS_ERR_INVALID_ARG, "order must be 2 or 3");
    NvtxRange range("dgfs SSP-RK steps");
    if (B < 0 || nsteps < 0) return fail(DGFS_ERR_INVALID_ARG, "B and nsteps must be >= 0");
    if (!std::isfinite(dt) || !std::isfinite(scale)) return fail(DGFS_ERR_INVALID_ARG, "dt and scale must be finite");
    if (B == 0 || nsteps == 0) return DGFS_OK;
    if (!f) return fail(DGFS_ERR_INVALID_ARG, "NULL field pointer");
    if (!aligned16(f)) return fail(DGFS_ERR_INVALID_ARG, "field pointer must be 16-byte aligned");
    DGFS_ON_DEVICE(plan->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return plan->prec == DGFS_PREC_FP64
               ? ssprk_run<double>(plan, order, static_cast<double*>(f), B, dt, scale, nsteps, s)
               : ssprk_run<float>(plan, order, static_cast<float*>(f), B, dt, scale, nsteps, s);
}

dgfs_status dgfs_moments(dgfs_plan_t plan, const void* f, double* out, int64_t B, void* stream) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (B < 0) return fail(DGFS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return DGFS_OK;
    if (!f || !out) return fail(DGFS_ERR_INVALID_ARG, "NULL pointer");
    DGFS_ON_DEVICE(plan->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaError_t e = plan->prec == DGFS_PREC_FP64
                              ? launch_moments<double>(static_cast<const double*>(f), plan->hp.N, plan->hp.L, B, out, s)
                              : launch_moments<float>(static_cast<const float*>(f), plan->hp.N, plan->hp.L, B, out, s);
    if (e) return cuda_fail(e, "moments");
    if (plan->prof) plan->prof_launches += 1;
    return DGFS_OK;
}

// ---- DG element collision (Sec. 3.4, SVD variant) -------------------------------------------

constexpr uint64_t kDgMagic = 0x444746534447454cull;   // "DGFSDGEL"

}  // extern "C"

struct dgfs_dg_s {
    uint64_t magic = kDgMagic;
    dgfs_plan_s* plan = nullptr;
    int K = 0, R = 0, device = 0;
    int64_t emax = 0;
    bool sym = false;        // every H[m] symmetric: terms s_r Q(f_r, f_r) (see k_dg.cu)
    std::vector<int> ranks;
    void* d_mem = nullptr;   // A [R][K] | B [R][K] | sgn [R] | rs [K + 1] | f | g | Q ([emax][R][N^3] each)
    size_t off_A = 0, off_B = 0, off_sgn = 0, off_rs = 0, off_f = 0, off_g = 0, off_Q = 0;
};

namespace {

bool check_dg(dgfs_dg_t d) { return d && d->magic == kDgMagic; }

template <typename T>
dgfs_status dg_run(dgfs_dg_s* d, const T* F, T* C, int64_t E, cudaStream_t s) {
    dgfs_plan_s* p = d->plan;
    const int64_t n3 = (int64_t)p->hp.N * p->hp.N * p->hp.N;
    unsigned char* base = static_cast<unsigned char*>(d->d_mem);
    const T* A = reinterpret_cast<const T*>(base + d->off_A);
    const T* B = d->sym ? nullptr : reinterpret_cast<const T*>(base + d->off_B);
    const T* sgn = d->sym ? reinterpret_cast<const T*>(base + d->off_sgn) : nullptr;
    const int* rs = reinterpret_cast<const int*>(base + d->off_rs);
    T* f = reinterpret_cast<T*>(base + d->off_f);
    T* g = reinterpret_cast<T*>(base + d->off_g);
    T* Q = reinterpret_cast<T*>(base + d->off_Q);
    for (int64_t e0 = 0; e0 < E; e0 += d->emax) {
        const int64_t ne = std::min<int64_t>(d->emax, E - e0);
        const T* Fe = F + e0 * d->K * n3;
        T* Ce = C + e0 * d->K * n3;
        if (d->R > 0) {
            cudaError_t e = launch_dg_combine<T>(Fe, A, B, d->K, d->R, n3, ne, f, g, s);
            if (e) return cuda_fail(e, "DG combination");
            const dgfs_status st = d->sym ? run<T>(p, Op::Collide, f, nullptr, Q, ne * d->R, s)
                                          : run<T>(p, Op::Collide2, f, g, Q, ne * d->R, s);
            if (st != DGFS_OK) return st;
        }
        cudaError_t e = launch_dg_accumulate<T>(Q, rs, sgn, d->K, d->R, n3, ne, Ce, s);
        if (e) return cuda_fail(e, "DG accumulation");
        if (p->prof) p->prof_launches += d->R > 0 ? 2 : 1;
    }
    return DGFS_OK;
}

template <typename T>
void put_coeffs(std::vector<unsigned char>& blob, size_t off, const std::vector<double>& v) {
    T* d = reinterpret_cast<T*>(blob.data() + off);
    for (size_t i = 0; i < v.size(); ++i) d[i] = (T)v[i];
}

}  // namespace

extern "C" {

dgfs_status dgfs_dg_create(dgfs_plan_t plan, int K, const double* H, double svd_tol, int64_t max_elements,
                           dgfs_dg_t* out) {
    if (!out) return fail(DGFS_ERR_INVALID_ARG, "NULL output");
    *out = nullptr;
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (K < 2 || K > 16) return fail(DGFS_ERR_INVALID_ARG, "K must be in [2, 16]");
    if (!H) return fail(DGFS_ERR_INVALID_ARG, "NULL H");
    if (!(svd_tol >= 0.0) || svd_tol >= 1.0) return fail(DGFS_ERR_INVALID_ARG, "svd_tol must be in [0, 1)");
    if (max_elements < 1 || max_elements > 65535) return fail(DGFS_ERR_INVALID_ARG, "max_elements must be in [1, 65535]");
    std::unique_ptr<dgfs_dg_s> d(new (std::nothrow) dgfs_dg_s);
    if (!d) return fail(DGFS_ERR_OOM, "host allocation failed");
    d->plan = plan;
    d->K = K;
    d->emax = max_elements;
    d->device = plan->device;
    // SVD of every slice H[m] (column-major K x K): H[m] = U diag(sv) V^T; row r of the
    // f coefficients is column r of U, row r of the g coefficients is sv[r] times column r of V.
    // Symmetric slices (the nodal basis always gives them): the eigen-decomposition
    // H[m] = sum_r lambda_r u_r u_r^T is such an SVD with f_r = sqrt|lambda_r| u_r . F and
    // g_r = sign(lambda_r) f_r, so every term is sign(lambda_r) Q(f_r, f_r)
    std::vector<double> A, B, sg;
    std::vector<int> rs(1, 0);
    bool sym = true;
    for (size_t m = 0; m < (size_t)K && sym; ++m)
        for (int a = 0; a < K && sym; ++a)
            for (int b = 0; b < a; ++b) {
                const double x = H[(m * K + a) * K + b], y = H[(m * K + b) * K + a];
                if (std::fabs(x - y) > 1e-13 * (std::fabs(x) + std::fabs(y)) + 1e-300) {
                    sym = false;
                    break;
                }
            }
    d->sym = sym;
    for (int m = 0; m < K && sym; ++m) {
        std::vector<double> Hm(H + (size_t)m * K * K, H + (size_t)(m + 1) * K * K), w, V;
        sym_eig_small(K, Hm, w, V);
        std::vector<int> order(K);
        for (int r = 0; r < K; ++r) order[r] = r;
        std::sort(order.begin(), order.end(), [&](int x, int y) { return std::fabs(w[x]) > std::fabs(w[y]); });
        const double thr = (svd_tol > 0 ? svd_tol : 1e-14) * std::fabs(w[order[0]]);
        int Rm = 0;
        for (int r : order) {
            if (!(std::fabs(w[r]) > thr)) continue;
            const double sc = std::sqrt(std::fabs(w[r]));
            for (int l = 0; l < K; ++l) A.push_back(sc * V[(size_t)l * K + r]);
            sg.push_back(w[r] > 0 ? 1.0 : -1.0);
            ++Rm;
        }
        d->ranks.push_back(Rm);
        rs.push_back(rs.back() + Rm);
    }
    for (int m = 0; m < K && !sym; ++m) {
        std::vector<double> Hm((size_t)K * K), sv, U, V;
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) Hm[(size_t)b * K + a] = H[((size_t)m * K + a) * K + b];
        svd_small(K, K, Hm, sv, U, V);
        const double thr = (svd_tol > 0 ? svd_tol : 1e-14) * sv[0];
        int Rm = 0;
        for (int r = 0; r < K; ++r) {
            if (!(sv[r] > thr)) continue;
            for (int l = 0; l < K; ++l) {
                A.push_back(U[(size_t)r * K + l]);
                B.push_back(sv[r] * V[(size_t)r * K + l]);
            }
            ++Rm;
        }
        d->ranks.push_back(Rm);
        rs.push_back(rs.back() + Rm);
    }
    d->R = rs.back();
    const size_t es = elem_size(plan->prec);
    const size_t n3 = (size_t)plan->hp.N * plan->hp.N * plan->hp.N;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off = align_up(off + b, 256); return o; };
    d->off_A = take(A.size() * es + es);
    d->off_B = take(B.size() * es + es);
    d->off_sgn = take(sg.size() * es + es);
    d->off_rs = take(rs.size() * sizeof(int));
    d->off_f = take((size_t)max_elements * d->R * n3 * es);
    d->off_g = take(sym ? 0 : (size_t)max_elements * d->R * n3 * es);
    d->off_Q = take((size_t)max_elements * d->R * n3 * es);
    std::vector<unsigned char> blob(d->off_f, 0);
    if (plan->prec == DGFS_PREC_FP64) {
        put_coeffs<double>(blob, d->off_A, A);
        put_coeffs<double>(blob, d->off_B, B);
        put_coeffs<double>(blob, d->off_sgn, sg);
    } else {
        put_coeffs<float>(blob, d->off_A, A);
        put_coeffs<float>(blob, d->off_B, B);
        put_coeffs<float>(blob, d->off_sgn, sg);
    }
    std::memcpy(blob.data() + d->off_rs, rs.data(), rs.size() * sizeof(int));
    DGFS_ON_DEVICE(plan->device);
    cudaError_t e = cudaMalloc(&d->d_mem, off);
    if (e != cudaSuccess) return fail(DGFS_ERR_OOM, std::string("DG workspace: ") + cudaGetErrorString(e));
    e = cudaMemcpy(d->d_mem, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d->d_mem);
        return cuda_fail(e, "DG coefficients upload");
    }
    *out = d.release();
    return DGFS_OK;
}

dgfs_status dgfs_dg_info(dgfs_dg_t dg, int* ranks, int* total) {
    if (!check_dg(dg)) return fail(DGFS_ERR_STATE, "invalid or destroyed DG operator");
    if (ranks)
        for (int m = 0; m < dg->K; ++m) ranks[m] = dg->ranks[m];
    if (total) *total = dg->R;
    return DGFS_OK;
}

dgfs_status dgfs_dg_collide(dgfs_dg_t dg, const void* F, void* C, int64_t E, void* stream) {
    if (!check_dg(dg)) return fail(DGFS_ERR_STATE, "invalid or destroyed DG operator");
    if (!check_plan(dg->plan)) return fail(DGFS_ERR_STATE, "the DG operator's plan was destroyed");
    if (E < 0) return fail(DGFS_ERR_INVALID_ARG, "E must be >= 0");
    NvtxRange range("dgfs DG element collision");
    if (E == 0) return DGFS_OK;
    if (!F || !C) return fail(DGFS_ERR_INVALID_ARG, "NULL field pointer");
    if (!aligned16(F) || !aligned16(C)) return fail(DGFS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (F == C) return fail(DGFS_ERR_INVALID_ARG, "output aliases the input");
    DGFS_ON_DEVICE(dg->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return dg->plan->prec == DGFS_PREC_FP64
               ? dg_run<double>(dg, static_cast<const double*>(F), static_cast<double*>(C), E, s)
               : dg_run<float>(dg, static_cast<const float*>(F), static_cast<float*>(C), E, s);
}

dgfs_status dgfs_dg_destroy(dgfs_dg_t dg) {
    if (!dg) return DGFS_OK;
    if (!check_dg(dg)) return fail(DGFS_ERR_STATE, "invalid or destroyed DG operator");
    {
        DeviceScope scope(dg->device);
        cudaDeviceSynchronize();
        cudaFree(dg->d_mem);
    }
    dg->magic = 0;
    delete dg;
    return DGFS_OK;
}

dgfs_status dgfs_host_dg_tensor(int K, double* nodes, double* M, double* H) {
    if (!nodes || !M || !H) return fail(DGFS_ERR_INVALID_ARG, "NULL output");
    std::vector<double> x, m, h;
    if (!dg_tensor_1d(K, x, m, h)) return fail(DGFS_ERR_INVALID_ARG, "K must be in [2, 16]");
    std::memcpy(nodes, x.data(), x.size() * sizeof(double));
    std::memcpy(M, m.data(), m.size() * sizeof(double));
    std::memcpy(H, h.data(), h.size() * sizeof(double));
    return DGFS_OK;
}

}  // extern "C"

// ---- 1-D DGFS solver: DG transport, diffuse walls, element collision, SSP-RK (Sec. 3) ----------

constexpr uint64_t kSlabMagic = 0x4447465353424c53ull;   // "DGFSSLBS"

struct dgfs_slab_s {
    uint64_t magic = kSlabMagic;
    dgfs_plan_s* plan = nullptr;
    dgfs_dg_s* dg = nullptr;   // the element collision term (nullptr: collisionless, Kn = inf)
    int K = 0, I = 0, device = 0;
    double invKn = 0.0;
    SlabMatrices mats{};
    void* d_mem = nullptr;     // fw [2][N^3] | num [2] | 2/h [I] | C | stage | q ([I][K][N^3] each)
    size_t off_fw = 0, off_num = 0, off_h = 0, off_C = 0, off_stage = 0, off_q = 0;
    // one SSP-RK step captured as a CUDA graph and replayed: the step's ~100 small launches cost one
    // graph launch. Valid for the field, step size, order and plan tuning it was captured with; the
    // wall update drops it (the wall denominators are kernel arguments).
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* gF = nullptr;
    double gdt = 0.0;
    int gorder = 0, grpc = 0;
    int64_t gchunk = 0;
};

namespace {

bool check_slab(dgfs_slab_t s) { return s && s->magic == kSlabMagic; }

void slab_release_graph(dgfs_slab_s* sl) {
    if (sl->gexec) cudaGraphExecDestroy(sl->gexec);
    sl->gexec = nullptr;
    sl->gF = nullptr;
}

// Wall Maxwellians f_w = exp(-|c - u_w|^2 / T_w) in the compute type and the FP64 denominators
// sum over the incoming velocities of |c_1| f_w (left wall: c_1 > 0, right wall: c_1 < 0).
dgfs_status slab_walls(dgfs_slab_s* sl, const double* wl, const double* wr) {
    if (!wl || !wr) return fail(DGFS_ERR_INVALID_ARG, "NULL wall state");
    const double* w[2] = {wl, wr};
    for (int k = 0; k < 2; ++k) {
        for (int a = 0; a < 4; ++a)
            if (!std::isfinite(w[k][a])) return fail(DGFS_ERR_INVALID_ARG, "non-finite wall state");
        if (w[k][0] != 0.0) return fail(DGFS_ERR_INVALID_ARG, "walls move parallel to themselves: u_x must be 0");
        if (!(w[k][3] > 0.0)) return fail(DGFS_ERR_INVALID_ARG, "wall temperature must be positive");
    }
    const HostPlan& h = sl->plan->hp;
    const int N = h.N;
    const size_t n3 = (size_t)N * N * N, es = elem_size(sl->plan->prec);
    const double dc = 2.0 * h.L / N;
    std::vector<unsigned char> blob(2 * n3 * es);
    for (int k = 0; k < 2; ++k) {
        double den = 0.0;
        for (size_t j = 0; j < n3; ++j) {
            const double c[3] = {-h.L + ((double)(j / ((size_t)N * N)) + 0.5) * dc,
                                 -h.L + ((double)((j / N) % N) + 0.5) * dc, -h.L + ((double)(j % N) + 0.5) * dc};
            const double d2 = (c[0] - w[k][0]) * (c[0] - w[k][0]) + (c[1] - w[k][1]) * (c[1] - w[k][1]) +
                              (c[2] - w[k][2]) * (c[2] - w[k][2]);
            const double fw = std::exp(-d2 / w[k][3]);
            if (k == 0 ? c[0] > 0.0 : c[0] < 0.0) den += std::fabs(c[0]) * fw;
            if (es == 8) reinterpret_cast<double*>(blob.data())[k * n3 + j] = fw;
            else reinterpret_cast<float*>(blob.data())[k * n3 + j] = (float)fw;
        }
        if (!(den > 0.0)) return fail(DGFS_ERR_INVALID_ARG, "wall Maxwellian vanishes on the velocity grid");
        sl->mats.den[k] = den;
    }
    DGFS_ON_DEVICE(sl->device);
    DGFS_CUDA(cudaDeviceSynchronize(), "synchronise before the wall update");
    DGFS_CUDA(cudaMemcpy(static_cast<unsigned char*>(sl->d_mem) + sl->off_fw, blob.data(), blob.size(),
                         cudaMemcpyHostToDevice), "wall tables upload");
    slab_release_graph(sl);
    return DGFS_OK;
}

template <typename T>
dgfs_status slab_rhs(dgfs_slab_s* sl, const T* F, T* out, cudaStream_t s) {
    dgfs_plan_s* p = sl->plan;
    unsigned char* base = static_cast<unsigned char*>(sl->d_mem);
    T* C = reinterpret_cast<T*>(base + sl->off_C);
    if (sl->dg) {
        const dgfs_status st = dg_run<T>(sl->dg, F, C, sl->I, s);
        if (st != DGFS_OK) return st;
    }
    double* num = reinterpret_cast<double*>(base + sl->off_num);
    cudaError_t e = launch_slab_wall<T>(F, p->hp.N, sl->I, sl->K, p->hp.L, num, s);
    if (!e) e = launch_slab_rhs<T>(F, sl->dg ? C : nullptr, reinterpret_cast<const T*>(base + sl->off_fw), num,
                                   sl->mats, reinterpret_cast<const double*>(base + sl->off_h), sl->invKn, p->hp.N,
                                   sl->I, p->hp.L, out, s);
    if (e) return cuda_fail(e, "slab transport");
    if (p->prof) p->prof_launches += 2;
    return DGFS_OK;
}

// One SSP-RK2 / RK3 step (eqs. SSPRK2, SSPRK3) of dF/dt = rhs(F), in place, stages in the slab's buffers
template <typename T>
dgfs_status slab_step(dgfs_slab_s* sl, int order, T* F, double dt, cudaStream_t s) {
    unsigned char* base = static_cast<unsigned char*>(sl->d_mem);
    T* stage = reinterpret_cast<T*>(base + sl->off_stage);
    T* q = reinterpret_cast<T*>(base + sl->off_q);
    const int64_t n = (int64_t)sl->I * sl->K * sl->plan->hp.N * sl->plan->hp.N * sl->plan->hp.N;
    int* flags = sl->plan->d_flags;
    dgfs_status st = slab_rhs<T>(sl, F, q, s);
    if (st != DGFS_OK) return st;
    cudaError_t e = launch_rk_combine<T>(n, 1.0, F, 0.0, nullptr, dt, q, stage, flags, s);
    if (e) return cuda_fail(e, "slab SSP-RK stage");
    st = slab_rhs<T>(sl, stage, q, s);
    if (st != DGFS_OK) return st;
    if (order == 2) {
        e = launch_rk_combine<T>(n, 0.5, F, 0.5, stage, 0.5 * dt, q, F, flags, s);
    } else {
        e = launch_rk_combine<T>(n, 0.75, F, 0.25, stage, 0.25 * dt, q, stage, flags, s);
        if (!e) {
            st = slab_rhs<T>(sl, stage, q, s);
            if (st != DGFS_OK) return st;
            e = launch_rk_combine<T>(n, 1.0 / 3.0, F, 2.0 / 3.0, stage, 2.0 / 3.0 * dt, q, F, flags, s);
        }
    }
    if (e) return cuda_fail(e, "slab SSP-RK stage");
    if (sl->plan->prof) sl->plan->prof_launches += order;
    return DGFS_OK;
}

// nsteps steps. Two or more steps on a stream that is not being captured, with the plan not
// profiling (its counters and events follow eager launches), replay one captured step. A new graph
// is captured after one eager step, so that every kernel's one-time setup has run outside capture.
template <typename T>
dgfs_status slab_ssprk(dgfs_slab_s* sl, int order, T* F, double dt, int nsteps, cudaStream_t s) {
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    DGFS_CUDA(cudaStreamIsCapturing(s, &capturing), "stream capture status");
    dgfs_plan_s* p = sl->plan;
    if (nsteps < 2 || p->prof || capturing != cudaStreamCaptureStatusNone) {
        for (int it = 0; it < nsteps; ++it) {
            const dgfs_status st = slab_step<T>(sl, order, F, dt, s);
            if (st != DGFS_OK) return st;
        }
        return DGFS_OK;
    }
    int done = 0;
    if (!sl->gexec || sl->gF != F || sl->gdt != dt || sl->gorder != order || sl->grpc != p->tc.rpc ||
        sl->gchunk != p->run_chunk) {
        slab_release_graph(sl);
        dgfs_status st = slab_step<T>(sl, order, F, dt, s);
        if (st != DGFS_OK) return st;
        done = 1;
        // the graph only saves launches: if creating the stream, capturing or instantiating fails,
        // that error is cleared and the remaining steps run eagerly
        bool ok = sl->cap || cudaStreamCreateWithFlags(&sl->cap, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) ok = cudaStreamBeginCapture(sl->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cudaGraph_t g = nullptr;
            const dgfs_status sc = slab_step<T>(sl, order, F, dt, sl->cap);
            const cudaError_t ec = cudaStreamEndCapture(sl->cap, &g);
            ok = sc == DGFS_OK && ec == cudaSuccess && g && cudaGraphInstantiate(&sl->gexec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        if (!ok) {
            sl->gexec = nullptr;
            (void)cudaGetLastError();
            for (int it = done; it < nsteps; ++it) {
                st = slab_step<T>(sl, order, F, dt, s);
                if (st != DGFS_OK) return st;
            }
            return DGFS_OK;
        }
        sl->gF = F;
        sl->gdt = dt;
        sl->gorder = order;
        sl->grpc = p->tc.rpc;
        sl->gchunk = p->run_chunk;
    }
    for (int it = done; it < nsteps; ++it) DGFS_CUDA(cudaGraphLaunch(sl->gexec, s), "graph launch");
    return DGFS_OK;
}

}  // namespace

extern "C" {

dgfs_status dgfs_slab_create(dgfs_plan_t plan, int K, int I, const double* edges, double Kn, const double* wall_left,
                             const double* wall_right, double svd_tol, dgfs_slab_t* out) {
    if (!out) return fail(DGFS_ERR_INVALID_ARG, "NULL output");
    *out = nullptr;
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (K < 2 || K > 8) return fail(DGFS_ERR_INVALID_ARG, "K must be in [2, 8]");
    if (I < 1 || I > 65535) return fail(DGFS_ERR_INVALID_ARG, "I must be in [1, 65535]");
    if (!edges) return fail(DGFS_ERR_INVALID_ARG, "NULL edges");
    for (int i = 0; i < I; ++i)
        if (!std::isfinite(edges[i]) || !std::isfinite(edges[i + 1]) || !(edges[i + 1] > edges[i]))
            return fail(DGFS_ERR_INVALID_ARG, "edges must be finite and strictly increasing");
    if (!(Kn > 0.0)) return fail(DGFS_ERR_INVALID_ARG, "Kn must be positive (infinity: collisionless)");
    std::unique_ptr<dgfs_slab_s> sl(new (std::nothrow) dgfs_slab_s);
    if (!sl) return fail(DGFS_ERR_OOM, "host allocation failed");
    sl->plan = plan;
    sl->K = K;
    sl->I = I;
    sl->device = plan->device;
    sl->invKn = std::isfinite(Kn) ? 1.0 / Kn : 0.0;
    sl->mats.K = K;
    std::vector<double> S, Minv, nodes, M, H;
    if (!dg_stiffness_1d(K, S, Minv) || !dg_tensor_1d(K, nodes, M, H)) return fail(DGFS_ERR_INVALID_ARG, "bad K");
    std::copy(S.begin(), S.end(), sl->mats.S);
    std::copy(Minv.begin(), Minv.end(), sl->mats.Minv);
    const size_t es = elem_size(plan->prec);
    const size_t n3 = (size_t)plan->hp.N * plan->hp.N * plan->hp.N;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off = align_up(off + b, 256); return o; };
    sl->off_fw = take(2 * n3 * es);
    sl->off_num = take(2 * sizeof(double));
    sl->off_h = take((size_t)I * sizeof(double));
    sl->off_C = take((size_t)I * K * n3 * es);
    sl->off_stage = take((size_t)I * K * n3 * es);
    sl->off_q = take((size_t)I * K * n3 * es);
    DGFS_ON_DEVICE(plan->device);
    cudaError_t e = cudaMalloc(&sl->d_mem, off);
    if (e != cudaSuccess) return fail(DGFS_ERR_OOM, std::string("slab workspace: ") + cudaGetErrorString(e));
    std::vector<double> h2(I);
    for (int i = 0; i < I; ++i) h2[i] = 2.0 / (edges[i + 1] - edges[i]);
    e = cudaMemcpy(static_cast<unsigned char*>(sl->d_mem) + sl->off_h, h2.data(), I * sizeof(double),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(sl->d_mem);
        return cuda_fail(e, "slab upload");
    }
    dgfs_status st = slab_walls(sl.get(), wall_left, wall_right);
    if (st == DGFS_OK && std::isfinite(Kn)) st = dgfs_dg_create(plan, K, H.data(), svd_tol, I, &sl->dg);
    if (st != DGFS_OK) {
        cudaFree(sl->d_mem);
        return st;
    }
    *out = sl.release();
    return DGFS_OK;
}

dgfs_status dgfs_slab_set_walls(dgfs_slab_t slab, const double* wall_left, const double* wall_right) {
    if (!check_slab(slab)) return fail(DGFS_ERR_STATE, "invalid or destroyed slab");
    return slab_walls(slab, wall_left, wall_right);
}

dgfs_status dgfs_slab_rhs(dgfs_slab_t slab, const void* F, void* dFdt, void* stream) {
    if (!check_slab(slab)) return fail(DGFS_ERR_STATE, "invalid or destroyed slab");
    if (!F || !dFdt) return fail(DGFS_ERR_INVALID_ARG, "NULL field pointer");
    if (!aligned16(F) || !aligned16(dFdt)) return fail(DGFS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (F == dFdt) return fail(DGFS_ERR_INVALID_ARG, "output aliases the input");
    DGFS_ON_DEVICE(slab->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NvtxRange range("dgfs slab right-hand side");
    return slab->plan->prec == DGFS_PREC_FP64
               ? slab_rhs<double>(slab, static_cast<const double*>(F), static_cast<double*>(dFdt), s)
               : slab_rhs<float>(slab, static_cast<const float*>(F), static_cast<float*>(dFdt), s);
}

dgfs_status dgfs_slab_ssprk(dgfs_slab_t slab, int order, void* F, double dt, int nsteps, void* stream) {
    if (!check_slab(slab)) return fail(DGFS_ERR_STATE, "invalid or destroyed slab");
    if (order != 2 && order != 3) return fail(DGFS_ERR_INVALID_ARG, "order must be 2 or 3");
    if (nsteps < 0 || !std::isfinite(dt)) return fail(DGFS_ERR_INVALID_ARG, "nsteps >= 0 and finite dt required");
    if (nsteps == 0) return DGFS_OK;
    if (!F) return fail(DGFS_ERR_INVALID_ARG, "NULL field pointer");
    NvtxRange range("dgfs slab SSP-RK steps");
    if (!aligned16(F)) return fail(DGFS_ERR_INVALID_ARG, "field pointer must be 16-byte aligned");
    DGFS_ON_DEVICE(slab->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return slab->plan->prec == DGFS_PREC_FP64 ? slab_ssprk<double>(slab, order, static_cast<double*>(F), dt, nsteps, s)
                                              : slab_ssprk<float>(slab, order, static_cast<float*>(F), dt, nsteps, s);
}

dgfs_status dgfs_slab_destroy(dgfs_slab_t slab) {
    if (!slab) return DGFS_OK;
    if (!check_slab(slab)) return fail(DGFS_ERR_STATE, "invalid or destroyed slab");
    {
        DeviceScope scope(slab->device);
        cudaDeviceSynchronize();
        slab_release_graph(slab);
        if (slab->cap) cudaStreamDestroy(slab->cap);
        if (slab->dg) dgfs_dg_destroy(slab->dg);
        cudaFree(slab->d_mem);
    }
    slab->magic = 0;
    delete slab;
    return DGFS_OK;
}

dgfs_status dgfs_host_dg_stiffness(int K, double* S, double* Minv) {
    std::vector<double> s, mi;
    if (!dg_stiffness_1d(K, s, mi)) return fail(DGFS_ERR_INVALID_ARG, "K must be in [2, 16]");
    if (S) std::memcpy(S, s.data(), s.size() * sizeof(double));
    if (Minv) std::memcpy(Minv, mi.data(), mi.size() * sizeof(double));
    return DGFS_OK;
}

// Sub-batch sizes of the host-buffer pipeline (B >= 1, chunk >= 1): at most H = chunk / 2 nodes each
// (one staging buffer of one node when chunk == 1), ramping up from B / 32 by a factor of 4 while the
// ramp fits twice into B, the rest split evenly into as few sub-batches of at most H as possible,
// then the ramp down.
static std::vector<int64_t> host_pipeline_sizes(int64_t B, int64_t chunk) {
    const int64_t H = chunk >= 2 ? chunk / 2 : 1;
    std::vector<int64_t> front;
    int64_t ramp_sum = 0;
    for (int64_t r = std::max<int64_t>(1, (B + 31) / 32); r < H && 2 * (ramp_sum + r) <= B; r *= 4) {
        front.push_back(r);
        ramp_sum += r;
    }
    const int64_t mid = B - 2 * ramp_sum;
    const int64_t nmid = (mid + H - 1) / H;
    std::vector<int64_t> sizes(front);
    for (int64_t k = 0; k < nmid; ++k) sizes.push_back(mid / nmid + (k < mid % nmid ? 1 : 0));
    sizes.insert(sizes.end(), front.rbegin(), front.rend());
    return sizes;
}

dgfs_status dgfs_host_pipeline_schedule(int64_t B, int64_t chunk, int64_t* sizes, int64_t cap, int64_t* count) {
    if (!count || B < 0 || chunk < 1 || cap < 0) return fail(DGFS_ERR_INVALID_ARG, "B >= 0, chunk >= 1, cap >= 0, count non-NULL");
    const std::vector<int64_t> v = B > 0 ? host_pipeline_sizes(B, chunk) : std::vector<int64_t>();
    *count = (int64_t)v.size();
    if (sizes)
        for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)v.size()); ++i) sizes[i] = v[(size_t)i];
    return DGFS_OK;
}

dgfs_status dgfs_collide_host(dgfs_plan_t plan, const void* f_host, void* Q_host, int64_t B,
                              void* stream) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    NvtxRange range("dgfs host-buffer pipeline");
    if (B < 0) return fail(DGFS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return DGFS_OK;
    if (!f_host || !Q_host) return fail(DGFS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DGFS_ON_DEVICE(plan->device);
    const size_t es = elem_size(plan->prec);
    const int64_t n3 = (int64_t)plan->hp.N * plan->hp.N * plan->hp.N;
    // The staging area (2 chunk fields) holds nbuf buffers of up to H nodes in and H nodes out.
    // Sub-batch i uses buffer i % nbuf: its host-to-device copy (copy stream 1) overlaps the compute of
    // sub-batch i - 1 (stream s), and the device-to-host copy of sub-batch i - 1 (copy stream 2)
    // overlaps the compute of sub-batch i. A buffer is refilled once the compute that read it has
    // finished, and its output half is rewritten once the copy that read it has finished. Only the
    // first sub-batch's input copy and the last one's output copy are exposed, so the sizes ramp up
    // from B / 32 nodes by a factor of 4 and down again at the end: each copy then hides behind a
    // compute about ten times longer even when host copies run an order of magnitude below their
    // usual 200 GB/s (the compute takes ~25 us per node at N = 32, a copy ~0.65 us); the middle is
    // split into as few sub-batches of at most H nodes as fit (each boundary costs about half a work
    // item of the persistent translate kernel's tail).
    const int nbuf = plan->chunk >= 2 ? 2 : 1;
    const int64_t H = plan->chunk / nbuf;
    const std::vector<int64_t> sizes = host_pipeline_sizes(B, plan->chunk);
    DGFS_CUDA(cudaEventRecord(plan->ev_start, s), "event record");   // earlier work on s that used the plan
    DGFS_CUDA(cudaStreamWaitEvent(plan->cs_h2d, plan->ev_start, 0), "stream wait");
    DGFS_CUDA(cudaStreamWaitEvent(plan->cs_d2h, plan->ev_start, 0), "stream wait");
    int64_t n0 = 0;
    for (size_t i = 0; i < sizes.size(); n0 += sizes[i], ++i) {
        const int b = (int)(i % nbuf);
        unsigned char* fin = ws(plan, plan->off_io) + (size_t)b * 2 * H * n3 * es;
        unsigned char* qout = fin + (size_t)H * n3 * es;
        const int64_t nn = sizes[i];
        const size_t bytes = (size_t)nn * n3 * es;
        if ((int)i >= nbuf) DGFS_CUDA(cudaStreamWaitEvent(plan->cs_h2d, plan->ev_comp[b], 0), "stream wait");
        DGFS_CUDA(cudaMemcpyAsync(fin, static_cast<const unsigned char*>(f_host) + (size_t)n0 * n3 * es, bytes,
                                  cudaMemcpyHostToDevice, plan->cs_h2d), "host to device");
        DGFS_CUDA(cudaEventRecord(plan->ev_h2d[b], plan->cs_h2d), "event record");
        DGFS_CUDA(cudaStreamWaitEvent(s, plan->ev_h2d[b], 0), "stream wait");
        if ((int)i >= nbuf) DGFS_CUDA(cudaStreamWaitEvent(s, plan->ev_d2h[b], 0), "stream wait");
        dgfs_status st = plan->prec == DGFS_PREC_FP64
            ? run_chunk<double>(plan, Op::Collide, reinterpret_cast<const double*>(fin), nullptr,
                                reinterpret_cast<double*>(qout), nullptr,
                                NodeParams{nullptr, nullptr, plan->hp.gamma, plan->hp.b, 0}, nn, s)
            : run_chunk<float>(plan, Op::Collide, reinterpret_cast<const float*>(fin), nullptr,
                               reinterpret_cast<float*>(qout), nullptr,
                               NodeParams{nullptr, nullptr, plan->hp.gamma, plan->hp.b, 0}, nn, s);
        if (st != DGFS_OK) return st;
        DGFS_CUDA(cudaEventRecord(plan->ev_comp[b], s), "event record");
        DGFS_CUDA(cudaStreamWaitEvent(plan->cs_d2h, plan->ev_comp[b], 0), "stream wait");
        DGFS_CUDA(cudaMemcpyAsync(static_cast<unsigned char*>(Q_host) + (size_t)n0 * n3 * es, qout, bytes,
                                  cudaMemcpyDeviceToHost, plan->cs_d2h), "device to host");
        DGFS_CUDA(cudaEventRecord(plan->ev_d2h[b], plan->cs_d2h), "event record");
    }
    DGFS_CUDA(cudaStreamSynchronize(plan->cs_d2h), "stream synchronise");
    DGFS_CUDA(cudaStreamSynchronize(s), "stream synchronise");
    return DGFS_OK;
}

dgfs_status dgfs_profile_begin(dgfs_plan_t plan) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    DGFS_ON_DEVICE(plan->device);
    if (plan->ev.empty()) {
        plan->ev.resize(2 * 65536);
        for (auto& e : plan->ev) DGFS_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    }
    plan->prof = true;
    plan->prof_launches = plan->prof_gain = plan->prof_timed = plan->prof_nodes = 0;
    return DGFS_OK;
}

dgfs_status dgfs_profile_end(dgfs_plan_t plan, dgfs_profile_t* out) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (!out) return fail(DGFS_ERR_INVALID_ARG, "NULL output");
    DGFS_ON_DEVICE(plan->device);
    double ms = 0;
    for (int64_t i = 0; i < plan->prof_timed; ++i) {
        DGFS_CUDA(cudaEventSynchronize(plan->ev[2 * i + 1]), "cudaEventSynchronize");
        float t = 0;
        DGFS_CUDA(cudaEventElapsedTime(&t, plan->ev[2 * i], plan->ev[2 * i + 1]), "cudaEventElapsedTime");
        ms += t;
    }
    out->launches = plan->prof_launches;
    out->gain_launches = plan->prof_gain;
    out->gain_timed = plan->prof_timed;
    out->gain_ms = ms;
    out->nodes = plan->prof_nodes;
    plan->prof = false;
    return DGFS_OK;
}

// ---- autotuner: radial points per CTA of the tensor-core kernels and nodes per chunk ----------

namespace {

struct TuneKey {
    int N, npairs, Nrho, rank, prec, bucket;
    bool operator<(const TuneKey& o) const {
        return std::tie(N, npairs, Nrho, rank, prec, bucket) < std::tie(o.N, o.npairs, o.Nrho, o.rank, o.prec, o.bucket);
    }
};
struct TuneVal {
    int rpc;
    int64_t chunk;
    double ms_default, ms_tuned;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

int floor_log2(int64_t v) {
    int b = 0;
    while (v > 1) {
        v >>= 1;
        ++b;
    }
    return b;
}

}  // namespace

dgfs_status dgfs_plan_autotune(dgfs_plan_t plan, const void* f, int64_t B, void* stream, dgfs_tune_report* report) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (B < 1 || !f || !report) return fail(DGFS_ERR_INVALID_ARG, "autotune needs B >= 1, f and a report");
    if (!aligned16(f)) return fail(DGFS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (plan->hp.aniso) return fail(DGFS_ERR_UNSUPPORTED, "autotune of a VSS plan (alpha != 1)");
    NvtxRange range("dgfs autotune");
    dgfs_plan_s* p = plan;
    const int64_t nodes = std::min<int64_t>(B, p->chunk);
    const TuneKey key{p->hp.N, p->hp.npairs, p->hp.Nrho, p->hp.rank, p->prec, floor_log2(nodes)};
    std::memset(report, 0, sizeof *report);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {   // the same shape was tuned before in this process
            p->tc.rpc = it->second.rpc;
            p->run_chunk = it->second.chunk;
            report->rpc = it->second.rpc;
            report->chunk_nodes = it->second.chunk;
            report->ms_per_node_default = it->second.ms_default;
            report->ms_per_node_tuned = it->second.ms_tuned;
            report->cached = 1;
            return DGFS_OK;
        }
    }
    DGFS_ON_DEVICE(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    DGFS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device), "cudaDeviceGetAttribute");
    const size_t n3 = (size_t)p->hp.N * p->hp.N * p->hp.N, es = elem_size(p->prec);
    void* Q = ws(p, p->off_io) + (size_t)p->chunk * n3 * es;   // the output half of the host staging area
    // candidates: radial points per work item (tensor-core plans; 0 = the batch-size rule) x nodes per chunk
    std::vector<int> rpcs{0};
    if (is_tc(p->prec))
        for (int c : {1, 2, 4, 8})
            if (p->hp.Nrho % c == 0) rpcs.push_back(c);
    std::vector<int64_t> chunks{nodes};
    for (int64_t c = nodes / 2; c >= 1 && chunks.size() < 3; c /= 2) chunks.push_back(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DGFS_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    cudaError_t e = cudaEventCreate(&e1);
    const int saved_rpc = p->tc.rpc;
    const int64_t saved_chunk = p->run_chunk;
    double best = -1.0, ms_default = -1.0;
    int best_rpc = 0, count = 0;
    int64_t best_chunk = nodes;
    for (int64_t ch : chunks)
        for (int rp : rpcs) {
            if (e != cudaSuccess) break;
            p->tc.rpc = rp;
            p->run_chunk = ch;
            dgfs_status st = DGFS_OK;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && st == DGFS_OK; ++rep) {   // rep 0 warms up
                if (rep == 1) e = cudaEventRecord(e0, s);
                for (int k = 0; k < (rep ? 3 : 1) && st == DGFS_OK; ++k)
                    st = p->prec == DGFS_PREC_FP64 ? run<double>(p, Op::Collide, f, nullptr, Q, nodes, s)
                                                   : run<float>(p, Op::Collide, f, nullptr, Q, nodes, s);
            }
            if (st != DGFS_OK) {
                p->tc.rpc = saved_rpc;
                p->run_chunk = saved_chunk;
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st;
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            const double per = ms / 3.0 / (double)nodes;
            ++count;
            if (ch == nodes && rp == 0) ms_default = per;
            if (best < 0 || per < best) {
                best = per;
                best_rpc = rp;
                best_chunk = ch;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        p->tc.rpc = saved_rpc;
        p->run_chunk = saved_chunk;
        return cuda_fail(e, "autotune timing");
    }
    // record the resolved value of the batch-size rule, so that a cached choice means the same (the
    // rule reads the plan's rpc, which still holds the last candidate: clear it first)
    if (best_rpc == 0 && is_tc(p->prec)) {
        p->tc.rpc = 0;
        best_rpc = tc_resolve_rpc(p->tc, p->prec, best_chunk, sms);
    }
    p->tc.rpc = best_rpc;
    p->run_chunk = best_chunk;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = TuneVal{best_rpc, best_chunk, ms_default, best};
    }
    report->rpc = best_rpc;
    report->chunk_nodes = best_chunk;
    report->ms_per_node_default = ms_default;
    report->ms_per_node_tuned = best;
    report->candidates = count;
    report->cached = 0;
    return DGFS_OK;
}

dgfs_status dgfs_plan_set_tuning(dgfs_plan_t plan, int rpc, int64_t chunk_nodes) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (rpc < 0 || (rpc > 0 && plan->hp.Nrho % rpc) || chunk_nodes < 0)
        return fail(DGFS_ERR_INVALID_ARG, "rpc must divide N_rho (0: the batch-size rule); chunk_nodes >= 0");
    plan->tc.rpc = rpc;
    plan->run_chunk = chunk_nodes;
    return DGFS_OK;
}

dgfs_status dgfs_device_fma_peaks(double* fp32_tflops, double* fp64_tflops) {
    double a = 0.0, b = 0.0;
    const cudaError_t e = measure_fma_peaks(a, b);
    if (e != cudaSuccess) return cuda_fail(e, "FMA rate probe");
    if (fp32_tflops) *fp32_tflops = a;
    if (fp64_tflops) *fp64_tflops = b;
    return DGFS_OK;
}

dgfs_status dgfs_device_mma_cycles(int n, int a_from_tmem, double* cycles_per_mma) {
    if (!cycles_per_mma || n < 16 || n > 256 || n % 16 || (a_from_tmem != 0 && a_from_tmem != 1))
        return fail(DGFS_ERR_INVALID_ARG, "n must be a multiple of 16 in [16, 256], a_from_tmem 0 or 1, output non-NULL");
    double c = 0.0;
    const cudaError_t e = measure_mma_cycles(n, a_from_tmem, c);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core rate probe");
    *cycles_per_mma = c;
    return DGFS_OK;
}

dgfs_status dgfs_debug_inject(dgfs_plan_t plan, int mode) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (mode != 0 && mode != 1) return fail(DGFS_ERR_INVALID_ARG, "unknown injection mode");
    plan->fault = mode;
    return DGFS_OK;
}

dgfs_status dgfs_stream_status(dgfs_plan_t plan, void* stream) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DGFS_ON_DEVICE(plan->device);
    DGFS_CUDA(cudaStreamSynchronize(s), "stream synchronise");
    int flags = 0;
    DGFS_CUDA(cudaMemcpy(&flags, plan->d_flags, sizeof(int), cudaMemcpyDeviceToHost), "read flags");
    DGFS_CUDA(cudaMemset(plan->d_flags, 0, sizeof(int)), "clear flags");
    if (flags & 1) return fail(DGFS_ERR_TIMEOUT, "a device-side wait gave up");
    if (flags & 2) return fail(DGFS_ERR_NUMERIC, "non-finite value in an output");
    return DGFS_OK;
}

dgfs_status dgfs_host_quadrature(const dgfs_plan_desc* desc, double* c_r, double* w_r,
                                 double* sigma_xyzw, int* n_pairs, double* R_used, double* b_used) {
    if (!desc) return fail(DGFS_ERR_INVALID_ARG, "NULL descriptor");
    HostPlan hp;
    std::string err;
    const dgfs_status st = build_quadrature(*desc, hp, err);
    if (st != DGFS_OK) return fail(st, err);
    if (n_pairs) *n_pairs = hp.npairs;
    if (R_used) *R_used = hp.R;
    if (b_used) *b_used = hp.b;
    if (c_r) std::memcpy(c_r, hp.cr.data(), hp.cr.size() * sizeof(double));
    if (w_r) std::memcpy(w_r, hp.wr.data(), hp.wr.size() * sizeof(double));
    if (sigma_xyzw)
        for (int i = 0; i < hp.npairs; ++i) {
            sigma_xyzw[4 * i + 0] = hp.sig[3 * i + 0];
            sigma_xyzw[4 * i + 1] = hp.sig[3 * i + 1];
            sigma_xyzw[4 * i + 2] = hp.sig[3 * i + 2];
            sigma_xyzw[4 * i + 3] = hp.wsig[i];
        }
    return DGFS_OK;
}

dgfs_status dgfs_host_plan_fingerprint(const dgfs_plan_desc* desc, uint64_t* fingerprint) {
    if (!desc || !fingerprint) return fail(DGFS_ERR_INVALID_ARG, "NULL argument");
    HostPlan hp;
    std::string err;
    const dgfs_status st = build_host_plan(*desc, hp, err);
    if (st != DGFS_OK) return fail(st, err);
    *fingerprint = plan_fingerprint(hp, desc->precision);
    return DGFS_OK;
}

dgfs_status dgfs_plan_fingerprint(dgfs_plan_t plan, uint64_t* fingerprint) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (!fingerprint) return fail(DGFS_ERR_INVALID_ARG, "NULL argument");
    *fingerprint = plan_fingerprint(plan->hp, plan->prec);
    return DGFS_OK;
}

dgfs_status dgfs_host_translate_filter(int N, double L, double t, double* a) {
    if (N < 2 || N % 2 || N > 4096 || !(L > 0) || !a || !std::isfinite(t))
        return fail(DGFS_ERR_INVALID_ARG, "bad translate-filter arguments");
    translate_filter(N, L, t, a);
    return DGFS_OK;
}

dgfs_status dgfs_host_vss_tables(const dgfs_plan_desc* desc, double* A, double* GL) {
    if (!desc) return fail(DGFS_ERR_INVALID_ARG, "NULL descriptor");
    HostPlan hp;
    std::string err;
    const dgfs_status st = build_host_plan(*desc, hp, err);
    if (st != DGFS_OK) return fail(st, err);
    if (!hp.aniso) return fail(DGFS_ERR_INVALID_ARG, "not a VSS descriptor (alpha must differ from 0 and 1)");
    if (A) std::memcpy(A, hp.Fa.data(), hp.Fa.size() * sizeof(double));
    if (GL) std::memcpy(GL, hp.GLa.data(), hp.GLa.size() * sizeof(double));
    return DGFS_OK;
}

dgfs_status dgfs_host_vss_factor(double L, double gamma, double b, double alpha, int n, const double* k_abs,
                                 const double* mu, const double* c_r, double* F) {
    if (!(L > 0) || !std::isfinite(gamma) || !(alpha >= 1.0 && alpha <= 2.0) || n < 0 || !std::isfinite(b))
        return fail(DGFS_ERR_INVALID_ARG, "bad VSS factor arguments");
    if (n > 0 && (!k_abs || !mu || !c_r || !F)) return fail(DGFS_ERR_INVALID_ARG, "NULL argument");
    const double bb = b > 0 ? b : default_b_vss(gamma, alpha);
    for (int i = 0; i < n; ++i) {
        if (!(k_abs[i] >= 0) || !(c_r[i] >= 0) || !(std::fabs(mu[i]) <= 1.0))
            return fail(DGFS_ERR_INVALID_ARG, "k_abs, c_r >= 0 and |mu| <= 1 required");
        F[i] = vss_F(bb, gamma, alpha, L, k_abs[i], mu[i], c_r[i]);
    }
    return DGFS_OK;
}

}  // extern "C"

// ---- Q(f,f) with its scratch in a fixed device array (no device allocation) --------------
//
// dgfs_collide keeps its intermediate fields (the radial products P_r, the spectra X and
// Y) in the plan's workspace, which dgfs_plan_create allocates. dgfs_collide_noalloc runs
// the same kernels on the same data but takes that scratch from one file-scope device array
// of kNoAllocScratchBytes instead: it calls no allocating routine of CUDA or of any library.
// The array exists once per GPU that loads this library and lives until the process exits;
// its address on a device is looked up (cudaGetSymbolAddress) by the first call made on
// that device, which is why the first call should not be made while a stream is being
// captured. All calls share the array: two calls whose work overlaps on the GPU (different
// streams, or plans on the same device used concurrently) race on it. Every scratch element
// a call reads is written earlier by the same call, so nothing needs clearing between calls.

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mu;
std::vector<void*> g_noalloc_ptr;   // device address of the array, per device (nullptr: not looked up)

// bytes of scratch one node needs: P_r for every radial point, rank + 2 spectra, 2 result spectra
size_t noalloc_node_bytes(const dgfs_plan_s* p) {
    const size_t es = elem_size(p->prec);
    const size_t n3 = (size_t)p->hp.N * p->hp.N * p->hp.N;
    return align_up((size_t)p->hp.Nrho * n3 * es, 256) + align_up((size_t)(p->hp.rank + 2) * n3 * 2 * es, 256) +
           align_up(2 * n3 * 2 * es, 256);
}

template <typename T>
dgfs_status noalloc_run(dgfs_plan_s* p, const T* f, T* Q, int64_t B, unsigned char* scratch, cudaStream_t s) {
    const DevTables<T>& t = tables<T>(p);
    const size_t n3 = (size_t)t.N * t.N * t.N;
    const int xf = t.rank + 2;
    T* P = reinterpret_cast<T*>(scratch);
    Cplx<T>* X = reinterpret_cast<Cplx<T>*>(scratch + align_up((size_t)B * t.Nrho * n3 * sizeof(T), 256));
    Cplx<T>* Y = X + align_up((size_t)B * xf * n3 * sizeof(Cplx<T>), 256) / sizeof(Cplx<T>);
    NodeParams np{nullptr, nullptr, p->hp.gamma, p->hp.b, 0};
    cudaError_t e;
    if (is_tc(p->prec) && std::is_same<T, float>::value)
        e = launch_tc_gain_products(p->tc, p->prec, reinterpret_cast<const float*>(f), nullptr, nullptr, B,
                                    reinterpret_cast<float*>(P), p->d_flags, s);
    else
        e = launch_gain_products(t, f, nullptr, nullptr, B, P, s);
    if (!e && spectral_supported(t)) {   // the fused Fourier stage, as in dgfs_collide
        e = launch_spectral<T>(t, P, np, B, f, nullptr, nullptr, T(1), X, Y, f, nullptr, Q, p->d_flags, s);
        if (e) return cuda_fail(e, "dgfs_collide_noalloc");
        return DGFS_OK;
    }
    const int xs = (t.rank + 2) / 2;   // rank projected fields and f, packed two per slot
    if (!e) e = launch_project<T>(t, P, np, B, X, xs, s);
    if (!e) e = launch_load_field<T>(t.N, f, nullptr, nullptr, B, X, xs, t.rank / 2, t.rank % 2, s);
    if (!e) e = launch_dft3<T>(t, X, B * xs, true, s);
    if (!e) e = launch_combine<T>(t, X, xs, np, B, T(1), t.rank, -1, Y, 2, s);
    if (!e) e = launch_dft3<T>(t, Y, B * 2, false, s);
    if (!e) e = launch_finalize<T>(t.N, t.Nrho, Y, 2, f, nullptr, nullptr, nullptr, B, 0, Q, p->d_flags, s);
    if (e) return cuda_fail(e, "dgfs_collide_noalloc");
    return DGFS_OK;
}

}  // namespace

extern "C" dgfs_status dgfs_collide_noalloc(dgfs_plan_t plan, const void* f, void* Q, int64_t B, void* stream) {
    if (!check_plan(plan)) return fail(DGFS_ERR_STATE, "invalid or destroyed plan");
    if (B < 0) return fail(DGFS_ERR_INVALID_ARG, "B must be >= 0");
    if (B == 0) return DGFS_OK;
    if (!f || !Q) return fail(DGFS_ERR_INVALID_ARG, "NULL field pointer");
    if (!aligned16(f) || !aligned16(Q)) return fail(DGFS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
    if (f == Q) return fail(DGFS_ERR_INVALID_ARG, "output aliases the input");
    if (plan->hp.aniso) return fail(DGFS_ERR_UNSUPPORTED, "dgfs_collide_noalloc of a VSS plan (alpha != 1)");
    if (plan->prec == DGFS_PREC_FP64 && plan->hp.N > 24)
        return fail(DGFS_ERR_UNSUPPORTED, "dgfs_collide_noalloc of an FP64 plan supports N <= 24");
    const size_t per_node = noalloc_node_bytes(plan);
    const int64_t capacity = (int64_t)(kNoAllocScratchBytes / per_node);
    if (B > capacity) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "dgfs_collide_noalloc: B = %lld exceeds the %lld nodes whose scratch (%zu bytes each) fits "
                      "the fixed %zu-byte device array; call it again on the remaining nodes",
                      (long long)B, (long long)capacity, per_node, kNoAllocScratchBytes);
        return fail(DGFS_ERR_INVALID_ARG, msg);
    }
    DGFS_ON_DEVICE(plan->device);
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if ((int)g_noalloc_ptr.size() <= plan->device) g_noalloc_ptr.resize(plan->device + 1, nullptr);
        if (!g_noalloc_ptr[plan->device]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                                          "cudaGetSymbolAddress of the fixed scratch array");
            g_noalloc_ptr[plan->device] = ptr;
        }
        base = g_noalloc_ptr[plan->device];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* scratch = static_cast<unsigned char*>(base);
    return plan->prec == DGFS_PREC_FP64
               ? noalloc_run<double>(plan, static_cast<const double*>(f), static_cast<double*>(Q), B, scratch, s)
               : noalloc_run<float>(plan, static_cast<const float*>(f), static_cast<float*>(Q), B, scratch, s);
}
