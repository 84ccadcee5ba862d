// Tensor-core (tcgen05) translate-product path for the 16-bit precisions.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "plan_host.h"

namespace dgfs {

struct TcTables {
    int N = 0, Nrho = 0, npairs = 0;   // N: points per axis of the tiles
    int nsrc = 0;                   // points per axis of f and P_r (N, or 24 on 32-point tiles)
    const void* mats = nullptr;     // per (r, pair, axis, sign) N x N operand tiles
    const float* wsig = nullptr;
    int rpc = 0;                    // radial points per work item: 0 = chosen from the batch (tc_resolve_rpc)
};

// Radial points per work item of the persistent kernel (per CTA pair for the split-data kernels)
// of a launch over `nodes` nodes:
// t.rpc when it divides N_rho, else the most of 4, 2, 1 that divides N_rho while the grid still fills
// the GPU's `sms` SMs at least 16 times over.
int tc_resolve_rpc(const TcTables& t, int prec, int64_t nodes, int sms);

// N = 16, 32; N = 24 on the 32-point tiles (zero-padded filters and data), every tensor-core precision.
bool tc_supported(int N, int prec);
int tc_extra_launches(int prec);   // launches the tensor-core path adds per chunk (beyond one)
size_t build_tc_tables(const HostPlan& hp, int prec, std::vector<unsigned char>& blob, TcTables& t);
void rebase_tc_tables(TcTables& t, void* base);
// Word of the plan's device flag array that counts the work items claimed by the persistent
// translate kernel (set to zero on the stream before each launch).
constexpr int kQueueWord = 4;

// fault: 0, or 1 = the first CTA withholds its pass-3-operands-complete signal (failure test).
// coef (device [nodes] or nullptr): P_r of node n is written times coef[n]; accumulate: added to P
// instead of overwriting it (the two halves of a polarisation).
cudaError_t launch_tc_gain_products(const TcTables& t, int prec, const float* f, const float* g,
                                    const int64_t* offs, int64_t nodes, float* P, int* flags,
                                    cudaStream_t s, int fault = 0, const float* coef = nullptr, int accumulate = 0);

// The operands of the bilinear translate-product sum by polarisation (it is symmetric in f, g):
// u [2 nodes][n3] = f + a g, f - a g (a = |f| / |g| per node), coef [2 nodes] = +-1 / (4 a), so
// P(f, g) = coef[n] P(u[n]) + coef[nodes + n] P(u[nodes + n]).
cudaError_t launch_polar_prep(const float* f, const float* g, int64_t n3, int64_t nodes, float* u, float* coef,
                              cudaStream_t s);

// The split-data precisions F16X3 and BF16X3 (tc_gain3.cu); build_tc_tables and
// launch_tc_gain_products dispatch to these for them.
bool tc3_precision(int prec);
size_t build_tc3_tables(const HostPlan& hp, int prec, std::vector<unsigned char>& blob, TcTables& t);
cudaError_t launch_tc3_gain_products(const TcTables& t, int prec, const float* f, const int64_t* offs, int64_t nodes,
                                     float* P, int* flags, cudaStream_t s, int fault, const float* coef, int accumulate);

}  // namespace dgfs
