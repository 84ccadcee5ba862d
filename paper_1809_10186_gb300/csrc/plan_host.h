// Host-side FP64 plan builder of the fast spectral collision operator.
//
// Everything the device kernels need that depends only on the discretisation
// (arXiv:1809.10186, Appendix): the radial Gauss-Legendre rule, the antipodal sphere
// rule, the per-axis translate filters of the shifts s_rp = c_r sigma_p / 2, the radial
// kernel S(|k|, r) = sinc(pi c_r |k| / 2L) with its optional SVD compression, and the
// loss weights. Computed once in double precision; the CUDA side rounds them.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dgfs.h"

namespace dgfs {

struct HostPlan {
    int N = 0, Nrho = 0, npairs = 0, rank = 0, loss_mode = 0;
    double L = 0, R = 0, gamma = 0, b = 0;
    std::vector<double> cr, wr;          // Gauss-Legendre on [0, R]
    std::vector<double> sig;             // [npairs][3] pair representatives sigma_p
    std::vector<double> wsig;            // [npairs]   weight of each point of a pair
    std::vector<double> filt;            // [Nrho][npairs][3][N] circulant filters of +s_rp
    // radial kernel, compressed: gain^(k) = sum_s Uk[s][k] * DFT( sum_r Vr[s][r] w_r rho_r P_r )
    std::vector<double> Uk;              // [rank][N^3] in DFT index order
    std::vector<double> Vr;              // [rank][Nrho]
    // loss: G_loss(k) = sum_r rho_r(gamma, b) * Lr[r][k]
    std::vector<double> Lr;              // [Nrho][N^3] in DFT index order
    // VSS kernel (alpha != 1, eq. B_gen): the kernel factor depends on the sphere point
    double alpha = 1.0;
    bool aniso = false;
    std::vector<double> Fa;              // [Nrho][npairs][N^3] w_r w_p F(k, c_r, sigma_p), DFT index order
    std::vector<double> GLa;             // [N^3] loss weight G(m, m) of the VSS kernel
    std::vector<double> mu;              // [Nrho][npairs][3][N][2] per-axis multipliers of +s_rp (every plan)
};

// F(k, c_r, sigma) of eq. realGG for the VSS kernel b c_r^gamma (1 + cos chi)^(alpha - 1), as the
// Funk-Hecke series of its Legendre expansion; k_abs = |k|, mu = sigma.k / |k|.
double vss_F(double b, double gamma, double alpha, double L, double k_abs, double mu, double c_r);

// 64-bit FNV-1a hash of everything a plan of precision prec is built from: the sizes, the scalars
// and every table of the host plan (doubles by their bit patterns, in a fixed order). Two plans
// with the same fingerprint compute the same arithmetic.
uint64_t plan_fingerprint(const HostPlan& hp, int prec);

// Gauss-Legendre rule on [a, b] by Newton iteration on the Legendre recurrence.
void gauss_legendre(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);

// Built-in antipodal sphere rules (M = 6, 12, 26, 38): one point per pair and the weight
// of each point. Returns false for an unsupported M.
bool sphere_pairs(int M, std::vector<double>& sig, std::vector<double>& w);

// Circulant filter a[N] of the translate by t (multiplier e^{i pi k t / L}, Nyquist cos).
void translate_filter(int N, double L, double t, double* a);

// Dense SVD A = U diag(sv) V^T of a column-major m x n matrix (m >= n), one-sided Jacobi; sv
// descending, U m x n and V n x n column-major.
void svd_small(int m, int n, const std::vector<double>& A, std::vector<double>& sv, std::vector<double>& U,
               std::vector<double>& V);

// 1-D nodal DG basis (Sec. 3.4): K Gauss-Lobatto points of [-1, 1], mass matrix M[m][l] and
// H[m][l1][l2] = int phi_m phi_l1 phi_l2 (eqs. eq_massMatrix, eq_stiffMatrix3). False for K
// outside [2, 16].
bool dg_tensor_1d(int K, std::vector<double>& nodes, std::vector<double>& M, std::vector<double>& H);

// Eigen-decomposition of a symmetric n x n matrix (row-major) by cyclic Jacobi rotations:
// A = V diag(w) V^T, V row-major with column k the k-th eigenvector (unsorted).
void sym_eig_small(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V);

// Stiffness matrix S[m][l] = int phi_l dphi_m/dxi (eq. eq_stiffMatrix1 on [-1, 1]) and the inverse
// mass matrix of the same basis. False for K outside [2, 16].
bool dg_stiffness_1d(int K, std::vector<double>& S, std::vector<double>& Minv);

double default_b(double gamma);
double default_b_vss(double gamma, double alpha);
double default_R(double L);

// Validates the descriptor and fills the plan. On failure returns a status and a message.
dgfs_status build_host_plan(const dgfs_plan_desc& d, HostPlan& p, std::string& err);

// Quadrature only (no tables), for introspection.
dgfs_status build_quadrature(const dgfs_plan_desc& d, HostPlan& p, std::string& err);

}  // namespace dgfs
