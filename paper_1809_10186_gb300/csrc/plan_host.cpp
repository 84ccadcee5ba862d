// Host-side FP64 plan builder (see plan_host.h).
#include "plan_host.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <thread>

namespace dgfs {

static const double kPi = 3.14159265358979323846;

double default_b(double gamma) {
    // nondimensional VHS constant, alpha = 1 (Sec. 2.1): 1 / (2^{3-omega} Gamma(5/2-omega) pi)
    const double omega = 1.0 - 0.5 * gamma;
    return 1.0 / (std::pow(2.0, 3.0 - omega) * std::tgamma(2.5 - omega) * kPi);
}

double default_R(double L) { return 4.0 * L / (3.0 + std::sqrt(2.0)); }  // Appendix

double default_b_vss(double gamma, double alpha) {
    // nondimensional VSS constant alpha / (2^{2-omega+alpha} Gamma(5/2-omega) pi) (Sec. 2.2)
    const double omega = 1.0 - 0.5 * gamma;
    return alpha / (std::pow(2.0, 2.0 - omega + alpha) * std::tgamma(2.5 - omega) * kPi);
}

void gauss_legendre(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double p1 = 0, p2 = 0, dp = 0;
        for (int it = 0; it < 100; ++it) {
            p1 = 1.0;
            p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            dp = n * (z * p1 - p2) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        // derivative at the converged node for the weight
        p1 = 1.0;
        p2 = 0.0;
        for (int j = 1; j <= n; ++j) {
            const double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        dp = n * (z * p1 - p2) / (z * z - 1.0);
        const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = wi;
    }
    const double h = 0.5 * (b - a), m = 0.5 * (b + a);
    for (int i = 0; i < n; ++i) {
        x[i] = h * x[i] + m;
        w[i] *= h;
    }
}

// ---- sphere rules ------------------------------------------------------------------------

namespace {

struct Pt { double x, y, z; };

void add_unique(std::vector<Pt>& v, Pt p) {
    for (const Pt& q : v)
        if (std::fabs(q.x - p.x) + std::fabs(q.y - p.y) + std::fabs(q.z - p.z) < 1e-12) return;
    v.push_back(p);
}

// all coordinate permutations and sign changes of (a, b, c)
std::vector<Pt> orbit(double a, double b, double c) {
    const double v[3] = {a, b, c};
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    std::vector<Pt> out;
    for (auto& pm : perm)
        for (int s = 0; s < 8; ++s) {
            Pt p{v[pm[0]] * ((s & 1) ? -1 : 1), v[pm[1]] * ((s & 2) ? -1 : 1),
                 v[pm[2]] * ((s & 4) ? -1 : 1)};
            p.x += 0.0; p.y += 0.0; p.z += 0.0;   // no negative zeros
            add_unique(out, p);
        }
    return out;
}

// one representative per antipodal pair: the point whose first nonzero coordinate is > 0
void push_pairs(const std::vector<Pt>& pts, double w, std::vector<double>& sig,
                std::vector<double>& ws) {
    for (const Pt& p : pts) {
        const double lead = (std::fabs(p.x) > 1e-14) ? p.x : (std::fabs(p.y) > 1e-14) ? p.y : p.z;
        if (lead > 0) {
            sig.push_back(p.x);
            sig.push_back(p.y);
            sig.push_back(p.z);
            ws.push_back(w);
        }
    }
}

}  // namespace

bool sphere_pairs(int M, std::vector<double>& sig, std::vector<double>& w) {
    sig.clear();
    w.clear();
    const double fourpi = 4.0 * kPi;
    if (M == 6) {                         // octahedron, degree 3
        push_pairs(orbit(1, 0, 0), fourpi / 6, sig, w);
        return true;
    }
    if (M == 12) {                        // icosahedron, degree 5
        const double phi = 0.5 * (1.0 + std::sqrt(5.0));
        const double n = std::sqrt(1.0 + phi * phi);
        std::vector<Pt> pts;
        for (int s1 = -1; s1 <= 1; s1 += 2)
            for (int s2 = -1; s2 <= 1; s2 += 2) {
                const double a = 0.0, b = s1 / n, c = s2 * phi / n;
                add_unique(pts, {a, b, c});
                add_unique(pts, {b, c, a});
                add_unique(pts, {c, a, b});
            }
        push_pairs(pts, fourpi / 12, sig, w);
        return true;
    }
    // Octahedral orbits: vertices (6), edge midpoints (12), corners (8), (p, q, 0) (24).
    // Exact monomial integrals over S^2: int 1 = 4pi, int x^4 = 4pi/5,
    // int x^2 y^2 z^2 = 4pi/105, int x^8 = 4pi/9.
    const double w3 = (fourpi / 105.0) / (8.0 / 27.0);   // corners: only orbit with x^2y^2z^2
    if (M == 26) {                        // degree 7
        // 6 w1 + 12 w2 + 8 w3 = 4pi ;  2 w1 + 2 w2 + (8/9) w3 = 4pi/5
        const double r1 = fourpi - 8.0 * w3, r2 = fourpi / 5.0 - 8.0 / 9.0 * w3;
        // solve [[6,12],[2,2]] [w1,w2] = [r1, r2]
        const double det = 6.0 * 2.0 - 12.0 * 2.0;
        const double w1 = (r1 * 2.0 - 12.0 * r2) / det;
        const double w2 = (6.0 * r2 - 2.0 * r1) / det;
        const double s2 = 1.0 / std::sqrt(2.0), s3 = 1.0 / std::sqrt(3.0);
        push_pairs(orbit(1, 0, 0), w1, sig, w);
        push_pairs(orbit(s2, s2, 0), w2, sig, w);
        push_pairs(orbit(s3, s3, s3), w3, sig, w);
        return true;
    }
    if (M == 38) {                        // degree 9
        auto solve = [&](double p, double& w1, double& wc) {
            const double q = std::sqrt(1.0 - p * p);
            // 6 w1 + 8 w3 + 24 wc = 4pi ;  2 w1 + (8/9) w3 + 8 (p^4 + q^4) wc = 4pi/5
            const double a11 = 6, a12 = 24, a21 = 2, a22 = 8.0 * (std::pow(p, 4) + std::pow(q, 4));
            const double r1 = fourpi - 8.0 * w3, r2 = fourpi / 5.0 - 8.0 / 9.0 * w3;
            const double det = a11 * a22 - a12 * a21;
            w1 = (r1 * a22 - a12 * r2) / det;
            wc = (a11 * r2 - a21 * r1) / det;
            // residual of the degree-8 moment: 2 w1 + (8/81) w3 + 8 (p^8 + q^8) wc - 4pi/9
            return 2.0 * w1 + 8.0 / 81.0 * w3 + 8.0 * (std::pow(p, 8) + std::pow(q, 8)) * wc
                   - fourpi / 9.0;
        };
        double lo = 0.3, hi = 0.7, w1 = 0, wc = 0;
        double flo = solve(lo, w1, wc);
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            const double fm = solve(mid, w1, wc);
            if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
            if (hi - lo < 1e-17) break;
        }
        const double p = 0.5 * (lo + hi);
        solve(p, w1, wc);
        const double s3 = 1.0 / std::sqrt(3.0);
        push_pairs(orbit(1, 0, 0), w1, sig, w);
        push_pairs(orbit(s3, s3, s3), w3, sig, w);
        push_pairs(orbit(p, std::sqrt(1.0 - p * p), 0), wc, sig, w);
        return true;
    }
    return false;
}

void translate_filter(int N, double L, double t, double* a) {
    // a[d] = (1/N) sum_k m(k) e^{2 pi i k d / N}, m(k) = e^{i pi k t / L} for |k| < N/2 and
    // cos(pi N t / 2L) at k = -N/2; pairing k with -k gives cosines.
    const double nyq = std::cos(kPi * N * t / (2.0 * L));
    for (int d = 0; d < N; ++d) {
        double s = 1.0;
        for (int k = 1; k < N / 2; ++k) s += 2.0 * std::cos(2.0 * kPi * k * d / N + kPi * k * t / L);
        s += ((d & 1) ? -1.0 : 1.0) * nyq;
        a[d] = s / N;
    }
}

// ---- SVD (one-sided Jacobi) -----------------------------------------------------------

namespace {

// A: m x n column-major (m >= n). On return: sv[n] descending, U (m x n) column-major,
// V (n x n) column-major with A = U diag(sv) V^T.
void jacobi_svd(int m, int n, std::vector<double> A, std::vector<double>& sv,
                std::vector<double>& U, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 80; ++sweep) {
        bool rotated = false;
        for (int i = 0; i < n - 1; ++i)
            for (int j = i + 1; j < n; ++j) {
                double al = 0, be = 0, ga = 0;
                const double* ci = &A[(size_t)i * m];
                const double* cj = &A[(size_t)j * m];
                for (int r = 0; r < m; ++r) {
                    al += ci[r] * ci[r];
                    be += cj[r] * cj[r];
                    ga += ci[r] * cj[r];
                }
                if (std::fabs(ga) <= 1e-15 * std::sqrt(al * be) || ga == 0.0) continue;
                rotated = true;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                double* ai = &A[(size_t)i * m];
                double* aj = &A[(size_t)j * m];
                for (int r = 0; r < m; ++r) {
                    const double x = ai[r], y = aj[r];
                    ai[r] = c * x - s * y;
                    aj[r] = s * x + c * y;
                }
                double* vi = &V[(size_t)i * n];
                double* vj = &V[(size_t)j * n];
                for (int r = 0; r < n; ++r) {
                    const double x = vi[r], y = vj[r];
                    vi[r] = c * x - s * y;
                    vj[r] = s * x + c * y;
                }
            }
        if (!rotated) break;
    }
    std::vector<double> norms(n);
    for (int i = 0; i < n; ++i) {
        double s = 0;
        for (int r = 0; r < m; ++r) s += A[(size_t)i * m + r] * A[(size_t)i * m + r];
        norms[i] = std::sqrt(s);
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return norms[a] > norms[b]; });
    sv.resize(n);
    U.assign((size_t)m * n, 0.0);
    std::vector<double> V2((size_t)n * n);
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        sv[k] = norms[i];
        for (int r = 0; r < m; ++r) U[(size_t)k * m + r] = norms[i] > 0 ? A[(size_t)i * m + r] / norms[i] : 0.0;
        for (int r = 0; r < n; ++r) V2[(size_t)k * n + r] = V[(size_t)i * n + r];
    }
    V.swap(V2);
}

inline int signed_k(int q, int N) { return q < N / 2 ? q : q - N; }

// P_n(x) and P'_n(x) by the three-term recurrence (|x| < 1 for the derivative formula)
void legendre_pd(int n, double x, double& p, double& dp) {
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        p = 1.0;
        dp = 0.0;
        return;
    }
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    p = p1;
    dp = n * (x * p1 - p0) / (x * x - 1.0);
}

}  // namespace

void svd_small(int m, int n, const std::vector<double>& A, std::vector<double>& sv, std::vector<double>& U,
               std::vector<double>& V) {
    jacobi_svd(m, n, A, sv, U, V);
}

bool dg_tensor_1d(int K, std::vector<double>& nodes, std::vector<double>& M, std::vector<double>& H) {
    if (K < 2 || K > 16) return false;
    // Gauss-Lobatto points: -1, the roots of P'_{K-1} (Newton from the Chebyshev-Lobatto points,
    // with P''_n = (2 x P'_n - n (n + 1) P_n) / (1 - x^2) from Legendre's equation), 1
    const int n = K - 1;
    nodes.assign(K, 0.0);
    nodes[0] = -1.0;
    nodes[K - 1] = 1.0;
    for (int j = 1; j < K - 1; ++j) {
        double x = -std::cos(kPi * j / n);
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre_pd(n, x, p, dp);
            const double d2p = (2.0 * x * dp - n * (n + 1.0) * p) / (1.0 - x * x);
            const double dx = dp / d2p;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        nodes[j] = x;
    }
    // Lagrange basis at Gauss-Legendre points exact for the degree 3 (K - 1) integrands
    std::vector<double> xq, wq;
    gauss_legendre(3 * K / 2 + 1, -1.0, 1.0, xq, wq);
    const int nq = (int)xq.size();
    std::vector<double> phi((size_t)K * nq);
    for (int l = 0; l < K; ++l)
        for (int q = 0; q < nq; ++q) {
            double v = 1.0;
            for (int j = 0; j < K; ++j)
                if (j != l) v *= (xq[q] - nodes[j]) / (nodes[l] - nodes[j]);
            phi[(size_t)l * nq + q] = v;
        }
    M.assign((size_t)K * K, 0.0);
    H.assign((size_t)K * K * K, 0.0);
    for (int m = 0; m < K; ++m)
        for (int a = 0; a < K; ++a)
            for (int q = 0; q < nq; ++q) {
                const double pm = phi[(size_t)m * nq + q] * phi[(size_t)a * nq + q] * wq[q];
                M[(size_t)m * K + a] += pm;
                for (int b = 0; b < K; ++b) H[((size_t)m * K + a) * K + b] += pm * phi[(size_t)b * nq + q];
            }
    return true;
}

void sym_eig_small(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
    // cyclic Jacobi: rotations in the (p, q) planes zero A[p][q] in turn until the off-diagonal
    // part vanishes; V accumulates the rotations (row-major, column k = eigenvector k)
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    double norm2 = 0.0;
    for (double x : A) norm2 += x * x;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a(p, q) * a(p, q);
        if (!(off > 1e-32 * norm2)) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (a(p, q) == 0.0) continue;
                const double theta = (a(q, q) - a(p, p)) / (2.0 * a(p, q));
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
                    const double kp = a(k, p), kq = a(k, q);
                    a(k, p) = c * kp - sn * kq;
                    a(k, q) = sn * kp + c * kq;
                }
                for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
                    const double pk = a(p, k), qk = a(q, k);
                    a(p, k) = c * pk - sn * qk;
                    a(q, k) = sn * pk + c * qk;
                }
                for (int k = 0; k < n; ++k) {
                    const double kp = V[(size_t)k * n + p], kq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * kp - sn * kq;
                    V[(size_t)k * n + q] = sn * kp + c * kq;
                }
            }
    }
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) w[i] = a(i, i);
}

bool dg_stiffness_1d(int K, std::vector<double>& S, std::vector<double>& Minv) {
    std::vector<double> nodes, M, H;
    if (!dg_tensor_1d(K, nodes, M, H)) return false;
    // S[m][l] = int phi_l phi_m' on the reference element, phi_m' by the product rule of the
    // Lagrange formula; Gauss-Legendre with K points is exact for the degree 2K - 3 integrand
    std::vector<double> xq, wq;
    gauss_legendre(K, -1.0, 1.0, xq, wq);
    S.assign((size_t)K * K, 0.0);
    for (int q = 0; q < K; ++q) {
        std::vector<double> phi(K, 1.0), dphi(K, 0.0);
        for (int l = 0; l < K; ++l)
            for (int j = 0; j < K; ++j)
                if (j != l) phi[l] *= (xq[q] - nodes[j]) / (nodes[l] - nodes[j]);
        for (int m = 0; m < K; ++m)
            for (int j = 0; j < K; ++j) {
                if (j == m) continue;
                double t = 1.0 / (nodes[m] - nodes[j]);
                for (int k = 0; k < K; ++k)
                    if (k != m && k != j) t *= (xq[q] - nodes[k]) / (nodes[m] - nodes[k]);
                dphi[m] += t;
            }
        for (int m = 0; m < K; ++m)
            for (int l = 0; l < K; ++l) S[(size_t)m * K + l] += wq[q] * phi[l] * dphi[m];
    }
    // M^{-1} by Gauss-Jordan elimination with partial pivoting (M is symmetric positive definite)
    std::vector<double> A = M;
    Minv.assign((size_t)K * K, 0.0);
    for (int i = 0; i < K; ++i) Minv[(size_t)i * K + i] = 1.0;
    for (int c = 0; c < K; ++c) {
        int piv = c;
        for (int r = c + 1; r < K; ++r)
            if (std::fabs(A[(size_t)r * K + c]) > std::fabs(A[(size_t)piv * K + c])) piv = r;
        for (int k = 0; k < K; ++k) {
            std::swap(A[(size_t)c * K + k], A[(size_t)piv * K + k]);
            std::swap(Minv[(size_t)c * K + k], Minv[(size_t)piv * K + k]);
        }
        const double d = A[(size_t)c * K + c];
        for (int k = 0; k < K; ++k) {
            A[(size_t)c * K + k] /= d;
            Minv[(size_t)c * K + k] /= d;
        }
        for (int r = 0; r < K; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * K + c];
            for (int k = 0; k < K; ++k) {
                A[(size_t)r * K + k] -= f * A[(size_t)c * K + k];
                Minv[(size_t)r * K + k] -= f * Minv[(size_t)c * K + k];
            }
        }
    }
    return true;
}

// ---- VSS kernel factor (alpha != 1) ---------------------------------------------------------
//
// With B = b c_r^gamma (1 + cos chi)^beta, beta = alpha - 1 (eq. B_gen), the factor of eq. realGG,
// F(k, c_r, sigma) = 2 c_r^2 int_{S2+} B_sym(c_r, sigma.e) cos(pi c_r k.e / 2L) de, is evaluated
// through the Legendre expansion of the angular factor and the Funk-Hecke formula
// int_S2 P_l(sigma.e) e^{i a khat.e} de = 4 pi i^l j_l(a) P_l(sigma.khat): only even l survive
// the symmetrisation and the cosine, and
//   F = 2 pi b c_r^{gamma+2} sum_{l even} (2l+1) c_l (-1)^{l/2} j_l(a) P_l(mu),
//   a = pi c_r |k| / 2L, mu = sigma.khat, c_l = int_{-1}^{1} (1 + t)^beta P_l(t) dt.
// The Legendre moments follow c_0 = 2^{beta+1}/(beta+1), c_{l+1} = c_l (beta - l)/(beta + l + 2)
// (the ratio of the Beta-function closed form); j_l(a) decays faster than geometrically once l > a,
// so the series stops at l = a + 40.

namespace {

// j_0..j_lmax(a), a >= 0: backward recurrence j_{l-1} = (2l+1)/a j_l - j_{l+1} from far above
// max(lmax, a), normalised with sum_l (2l+1) j_l(a)^2 = 1 and signed by the closed form of j_0 or j_1.
void sph_bessel(int lmax, double a, std::vector<double>& j) {
    j.assign((size_t)lmax + 1, 0.0);
    if (a < 1e-8) {          // j_l(a) = O(a^l): only j_0 = 1 matters to double precision for even l
        j[0] = 1.0;
        return;
    }
    const double hi = std::max((double)lmax, a);
    const int top = (int)hi + 40 + (int)std::sqrt(40.0 * hi);
    std::vector<double> v((size_t)top + 2, 0.0);
    v[top] = 1e-300;
    for (int l = top; l >= 1; --l) {
        v[l - 1] = (2.0 * l + 1.0) / a * v[l] - v[l + 1];
        if (std::fabs(v[l - 1]) > 1e200)
            for (int m = l - 1; m <= top; ++m) v[m] *= 1e-200;
    }
    double vmax = 0.0;
    for (int l = 0; l <= top; ++l) vmax = std::max(vmax, std::fabs(v[l]));
    double sum = 0.0;
    for (int l = 0; l <= top; ++l) sum += (2.0 * l + 1.0) * (v[l] / vmax) * (v[l] / vmax);
    double scale = 1.0 / (vmax * std::sqrt(sum));
    const double j0 = std::sin(a) / a, j1 = std::sin(a) / (a * a) - std::cos(a) / a;
    if (std::fabs(j0) >= std::fabs(j1) ? ((j0 < 0) != (v[0] < 0)) : ((j1 < 0) != (v[1] < 0))) scale = -scale;
    for (int l = 0; l <= lmax; ++l) j[l] = v[l] * scale;
}

// Series coefficients g_l = (2l+1) c_l (-1)^{l/2} j_l(a) for even l (0 for odd l), l <= lmax.
void vss_series(double beta, double a, std::vector<double>& g) {
    const int lmax = 2 * (((int)a + 41) / 2);
    std::vector<double> j;
    sph_bessel(lmax, a, j);
    g.assign((size_t)lmax + 1, 0.0);
    double c = std::pow(2.0, beta + 1.0) / (beta + 1.0);
    for (int l = 0; l <= lmax; ++l) {
        if (l % 2 == 0) g[l] = (2.0 * l + 1.0) * c * ((l / 2) % 2 ? -1.0 : 1.0) * j[l];
        c *= (beta - l) / (beta + l + 2.0);
    }
}

// sum_l g_l P_l(mu) by the three-term recurrence (l + 1) P_{l+1} = (2l + 1) mu P_l - l P_{l-1}
double legendre_sum(const std::vector<double>& g, double mu) {
    double pm = 1.0, pc = mu, s = g[0];
    for (size_t l = 1; l < g.size(); ++l) {
        if (g[l] != 0.0) s += g[l] * pc;
        const double pn = ((2.0 * l + 1.0) * mu * pc - (double)l * pm) / (double)(l + 1);
        pm = pc;
        pc = pn;
    }
    return s;
}

}  // namespace

double vss_F(double b, double gamma, double alpha, double L, double k_abs, double mu, double c_r) {
    std::vector<double> g;
    vss_series(alpha - 1.0, kPi * c_r * k_abs / (2.0 * L), g);
    return 2.0 * kPi * b * std::pow(c_r, gamma + 2.0) * legendre_sum(g, std::max(-1.0, std::min(1.0, mu)));
}

namespace {

// Gain factors Fa[r][q][i] = w_r w_q F(k_i, c_r, sigma_q), the VSS loss weight and the per-axis
// translate multipliers; one worker thread per group of radial points.
void build_vss_tables(HostPlan& p) {
    const int N = p.N, Nr = p.Nrho, np = p.npairs;
    const size_t n3 = (size_t)N * N * N;
    const double beta = p.alpha - 1.0;
    std::vector<int> kv(3 * n3);
    std::vector<int> q2(n3);
    for (size_t i = 0; i < n3; ++i) {
        kv[3 * i] = signed_k((int)(i / ((size_t)N * N)), N);
        kv[3 * i + 1] = signed_k((int)((i / N) % N), N);
        kv[3 * i + 2] = signed_k((int)(i % N), N);
        q2[i] = kv[3 * i] * kv[3 * i] + kv[3 * i + 1] * kv[3 * i + 1] + kv[3 * i + 2] * kv[3 * i + 2];
    }
    const int qmax = 3 * (N / 2) * (N / 2);
    p.Fa.assign((size_t)Nr * np * n3, 0.0);
    std::vector<double> lossr((size_t)Nr * n3, 0.0);
    auto work = [&](int r) {
        const double pref = 2.0 * kPi * p.b * std::pow(p.cr[r], p.gamma + 2.0);
        std::vector<std::vector<double>> gq(qmax + 1), gq2(qmax + 1);
        for (size_t i = 0; i < n3; ++i)
            if (gq[q2[i]].empty()) {
                const double kk = std::sqrt((double)q2[i]);
                vss_series(beta, kPi * p.cr[r] * kk / (2.0 * p.L), gq[q2[i]]);
                if (p.loss_mode == DGFS_LOSS_PAPER) vss_series(beta, kPi * p.cr[r] * kk / p.L, gq2[q2[i]]);
            }
        for (int q = 0; q < np; ++q) {
            const double* sg = &p.sig[3 * q];
            double* out = &p.Fa[((size_t)r * np + q) * n3];
            for (size_t i = 0; i < n3; ++i) {
                // F is even in k (even Legendre degrees only): one evaluation serves k and -k when -k
                // is on the lattice (no Nyquist component); the DFT mirror index of a Nyquist mode is
                // a different lattice vector and gets its own evaluation
                const size_t im = ((size_t)((N - (int)(i / ((size_t)N * N))) % N) * N + (N - (int)((i / N) % N)) % N) * N +
                                  (N - (int)(i % N)) % N;
                const bool pair = kv[3 * im] == -kv[3 * i] && kv[3 * im + 1] == -kv[3 * i + 1] &&
                                  kv[3 * im + 2] == -kv[3 * i + 2];
                if (pair && im < i) continue;
                const double kk = std::sqrt((double)q2[i]);
                const double mu = kk > 0 ? (kv[3 * i] * sg[0] + kv[3 * i + 1] * sg[1] + kv[3 * i + 2] * sg[2]) / kk : 0.0;
                out[i] = p.wr[r] * p.wsig[q] * pref * legendre_sum(gq[q2[i]], mu);
                if (pair) out[im] = out[i];
                if (p.loss_mode == DGFS_LOSS_PAPER) {   // eq. lowrank1 at l = m: F(2m, c_r, sigma_q)
                    const double l0 = 2.0 * p.wr[r] * p.wsig[q] * pref * legendre_sum(gq2[q2[i]], mu);
                    lossr[(size_t)r * n3 + i] += l0;
                    if (pair && im != i) lossr[(size_t)r * n3 + im] += l0;
                }
            }
        }
    };
    const int nt = std::max(1, std::min<int>(Nr, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&, t] {
            for (int r = t; r < Nr; r += nt) work(r);
        });
    for (auto& th : pool) th.join();
    p.GLa.assign(n3, 0.0);
    if (p.loss_mode == DGFS_LOSS_PAPER) {
        for (int r = 0; r < Nr; ++r)
            for (size_t i = 0; i < n3; ++i) p.GLa[i] += lossr[(size_t)r * n3 + i];
    } else {
        // G(-m, m) = 2 sum_r w_r F(0, c_r) sum_q w_q cos(...): Lr carries w_r sum_q w_q [mu_s^2 + mu_-s^2],
        // and F(0, c_r) = 2 pi b c_r^{gamma+2} c_0 is isotropic
        const double c0 = std::pow(2.0, beta + 1.0) / (beta + 1.0);
        for (int r = 0; r < Nr; ++r) {
            const double F0 = 2.0 * kPi * p.b * std::pow(p.cr[r], p.gamma + 2.0) * c0;
            for (size_t i = 0; i < n3; ++i) p.GLa[i] += F0 * p.Lr[(size_t)r * n3 + i];
        }
    }
}

// per-axis multipliers of the translate by +s_rp: e^{i pi k t / L}, Nyquist cos(pi N t / 2L)
void build_translate_multipliers(HostPlan& p) {
    const int N = p.N, Nr = p.Nrho, np = p.npairs;
    p.mu.assign((size_t)Nr * np * 3 * N * 2, 0.0);
    for (int r = 0; r < Nr; ++r)
        for (int q = 0; q < np; ++q)
            for (int a = 0; a < 3; ++a) {
                const double t = 0.5 * p.cr[r] * p.sig[3 * q + a];
                double* m = &p.mu[(((size_t)r * np + q) * 3 + a) * N * 2];
                for (int kq = 0; kq < N; ++kq) {
                    const int k = signed_k(kq, N);
                    if (k == -N / 2) {
                        m[2 * kq] = std::cos(kPi * N * t / (2.0 * p.L));
                    } else {
                        m[2 * kq] = std::cos(kPi * k * t / p.L);
                        m[2 * kq + 1] = std::sin(kPi * k * t / p.L);
                    }
                }
            }
}

}  // namespace

// ---- plan --------------------------------------------------------------------------------

static bool supported_N(int N) { return N == 8 || N == 12 || N == 16 || N == 24 || N == 32; }

dgfs_status build_quadrature(const dgfs_plan_desc& d, HostPlan& p, std::string& err) {
    if (!supported_N(d.N)) {
        err = "N must be one of 8, 12, 16, 24, 32";
        return DGFS_ERR_INVALID_ARG;
    }
    if (!(d.L > 0) || !std::isfinite(d.L)) { err = "L must be positive"; return DGFS_ERR_INVALID_ARG; }
    if (!std::isfinite(d.gamma) || d.gamma < -2.5 || d.gamma > 2.0) {
        err = "gamma must lie in [-2.5, 2]";
        return DGFS_ERR_INVALID_ARG;
    }
    p.N = d.N;
    p.L = d.L;
    p.gamma = d.gamma;
    p.R = d.R > 0 ? d.R : default_R(d.L);
    p.alpha = (d.alpha == 0.0) ? 1.0 : d.alpha;
    if (!(p.alpha >= 1.0 && p.alpha <= 2.0)) { err = "alpha must lie in [1, 2] (0: VHS)"; return DGFS_ERR_INVALID_ARG; }
    p.aniso = p.alpha != 1.0;
    p.b = d.b > 0 ? d.b : (p.aniso ? default_b_vss(d.gamma, p.alpha) : default_b(d.gamma));
    p.Nrho = d.N_rho > 0 ? d.N_rho : d.N;
    p.loss_mode = d.loss_mode;
    if (p.Nrho > 64) { err = "N_rho must be <= 64"; return DGFS_ERR_INVALID_ARG; }
    if (!std::isfinite(p.R) || !std::isfinite(p.b)) { err = "non-finite R or b"; return DGFS_ERR_INVALID_ARG; }
    gauss_legendre(p.Nrho, 0.0, p.R, p.cr, p.wr);
    if (d.sphere_xyzw) {
        if (d.M < 2 || d.M % 2 || d.M > 512) { err = "M must be even, 2..512"; return DGFS_ERR_INVALID_ARG; }
        p.sig.clear();
        p.wsig.clear();
        double wsum = 0;
        for (int i = 0; i < d.M / 2; ++i) {
            const double* q = d.sphere_xyzw + 4 * i;
            const double nrm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
            if (!(std::fabs(nrm - 1.0) < 1e-12) || !(q[3] > 0)) {
                err = "sphere_xyzw: points must be unit vectors with positive weights";
                return DGFS_ERR_INVALID_ARG;
            }
            p.sig.insert(p.sig.end(), {q[0], q[1], q[2]});
            p.wsig.push_back(q[3]);
            wsum += 2.0 * q[3];
        }
        if (std::fabs(wsum - 4.0 * kPi) > 1e-10 * 4.0 * kPi) {
            err = "sphere_xyzw: weights of the full antipodal rule must sum to 4 pi";
            return DGFS_ERR_INVALID_ARG;
        }
    } else if (!sphere_pairs(d.M, p.sig, p.wsig)) {
        err = "no built-in sphere rule for this M (have 6, 12, 26, 38); pass sphere_xyzw";
        return DGFS_ERR_INVALID_ARG;
    }
    p.npairs = (int)p.wsig.size();
    return DGFS_OK;
}

dgfs_status build_host_plan(const dgfs_plan_desc& d, HostPlan& p, std::string& err) {
    dgfs_status st = build_quadrature(d, p, err);
    if (st != DGFS_OK) return st;
    if (d.loss_mode != DGFS_LOSS_PAPER && d.loss_mode != DGFS_LOSS_CONSERVATIVE) {
        err = "unknown loss_mode";
        return DGFS_ERR_INVALID_ARG;
    }
    if (!(d.svd_tol >= 0) || d.svd_rank < 0) { err = "svd_tol and svd_rank must be >= 0"; return DGFS_ERR_INVALID_ARG; }
    const int N = p.N, Nr = p.Nrho, np = p.npairs;
    const size_t n3 = (size_t)N * N * N;

    // translate filters of s_rp = c_r sigma_p / 2 (eq. apndx_Q: c' = c - c_r/2 + c_r sigma/2)
    p.filt.assign((size_t)Nr * np * 3 * N, 0.0);
    for (int r = 0; r < Nr; ++r)
        for (int q = 0; q < np; ++q)
            for (int a = 0; a < 3; ++a)
                translate_filter(N, p.L, 0.5 * p.cr[r] * p.sig[3 * q + a],
                                 &p.filt[(((size_t)r * np + q) * 3 + a) * N]);

    // distinct |k|^2 on the lattice, multiplicities, and the map k -> class
    const int qmax = 3 * (N / 2) * (N / 2);
    std::vector<int> cls_of_q(qmax + 1, -1), mult;
    std::vector<int> qvals;
    std::vector<int> cls_of_k(n3);
    for (size_t i = 0; i < n3; ++i) {
        const int kx = signed_k((int)(i / (N * N)), N), ky = signed_k((int)((i / N) % N), N),
                  kz = signed_k((int)(i % N), N);
        const int q2 = kx * kx + ky * ky + kz * kz;
        if (cls_of_q[q2] < 0) {
            cls_of_q[q2] = (int)qvals.size();
            qvals.push_back(q2);
            mult.push_back(0);
        }
        cls_of_k[i] = cls_of_q[q2];
        mult[cls_of_q[q2]]++;
    }
    const int nq = (int)qvals.size();
    // S(|k|, r) = sinc(pi c_r |k| / 2L): the isotropic closed form of F / rho_r (eq. realGG)
    auto sinc = [](double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; };
    std::vector<double> S((size_t)nq * Nr);     // row-major [q][r]
    for (int c = 0; c < nq; ++c)
        for (int r = 0; r < Nr; ++r)
            S[(size_t)c * Nr + r] = sinc(kPi * p.cr[r] * std::sqrt((double)qvals[c]) / (2.0 * p.L));

    std::vector<double> Seff_cls((size_t)nq * Nr);   // effective (possibly truncated) S
    if (d.svd_tol > 0 || d.svd_rank > 0) {
        if (nq < Nr) { err = "radial kernel has fewer |k| classes than radial points"; return DGFS_ERR_UNSUPPORTED; }
        std::vector<double> A((size_t)nq * Nr);       // column-major, rows weighted by sqrt(mult)
        for (int r = 0; r < Nr; ++r)
            for (int c = 0; c < nq; ++c) A[(size_t)r * nq + c] = std::sqrt((double)mult[c]) * S[(size_t)c * Nr + r];
        std::vector<double> sv, U, V;
        jacobi_svd(nq, Nr, A, sv, U, V);
        int rank = d.svd_rank > 0 ? d.svd_rank : 0;
        if (rank == 0)
            for (int s = 0; s < Nr; ++s)
                if (sv[s] > d.svd_tol * sv[0]) rank = s + 1;
        rank = std::max(1, std::min(rank, Nr));
        p.rank = rank;
        p.Uk.assign((size_t)rank * n3, 0.0);
        p.Vr.assign((size_t)rank * Nr, 0.0);
        std::vector<double> Ucls((size_t)rank * nq);
        for (int s = 0; s < rank; ++s) {
            for (int c = 0; c < nq; ++c) Ucls[(size_t)s * nq + c] = U[(size_t)s * nq + c] * sv[s] / std::sqrt((double)mult[c]);
            for (int r = 0; r < Nr; ++r) p.Vr[(size_t)s * Nr + r] = V[(size_t)s * Nr + r];
        }
        for (size_t i = 0; i < n3; ++i)
            for (int s = 0; s < rank; ++s) p.Uk[(size_t)s * n3 + i] = Ucls[(size_t)s * nq + cls_of_k[i]];
        for (int c = 0; c < nq; ++c)
            for (int r = 0; r < Nr; ++r) {
                double v = 0;
                for (int s = 0; s < rank; ++s) v += Ucls[(size_t)s * nq + c] * p.Vr[(size_t)s * Nr + r];
                Seff_cls[(size_t)c * Nr + r] = v;
            }
    } else {
        p.rank = Nr;
        p.Uk.assign((size_t)Nr * n3, 0.0);
        p.Vr.assign((size_t)Nr * Nr, 0.0);
        for (int r = 0; r < Nr; ++r) p.Vr[(size_t)r * Nr + r] = 1.0;
        for (size_t i = 0; i < n3; ++i)
            for (int r = 0; r < Nr; ++r) p.Uk[(size_t)r * n3 + i] = S[(size_t)cls_of_k[i] * Nr + r];
        Seff_cls = S;
    }

    // loss weights per radial node: G_loss(k) = sum_r rho_r Lr[r][k]
    p.Lr.assign((size_t)Nr * n3, 0.0);
    if (p.loss_mode == DGFS_LOSS_PAPER) {
        // G(m,m) = 4 pi sum_r w_r F(2m, c_r), F(2m, c_r) = rho_r sinc(pi c_r |m| / L)
        for (int r = 0; r < Nr; ++r)
            for (size_t i = 0; i < n3; ++i)
                p.Lr[(size_t)r * n3 + i] = 4.0 * kPi * p.wr[r] *
                    sinc(kPi * p.cr[r] * std::sqrt((double)qvals[cls_of_k[i]]) / p.L);
    } else {
        // G(-m,m) = sum_r w_r rho_r S(0,r) sum_pairs w_p Re[mu_s(m)^2 + mu_-s(m)^2]
        const int c0 = cls_of_q[0];
        for (int r = 0; r < Nr; ++r) {
            const double s0 = Seff_cls[(size_t)c0 * Nr + r];
            for (int q = 0; q < np; ++q) {
                double sh[3];
                for (int a = 0; a < 3; ++a) sh[a] = 0.5 * p.cr[r] * p.sig[3 * q + a];
                for (size_t i = 0; i < n3; ++i) {
                    const int kk[3] = {signed_k((int)(i / (N * N)), N), signed_k((int)((i / N) % N), N),
                                       signed_k((int)(i % N), N)};
                    // product over axes of mu(k_a)^2 for +s and for -s
                    double re_p = 1, im_p = 0, re_m = 1, im_m = 0;
                    for (int a = 0; a < 3; ++a) {
                        double mr, mi;           // mu_{s_a}(k_a)^2
                        if (kk[a] == -N / 2) {
                            const double c = std::cos(kPi * N * sh[a] / (2.0 * p.L));
                            mr = c * c;
                            mi = 0;
                        } else {
                            const double ang = 2.0 * kPi * kk[a] * sh[a] / p.L;
                            mr = std::cos(ang);
                            mi = std::sin(ang);
                        }
                        const double tr = re_p * mr - im_p * mi, ti = re_p * mi + im_p * mr;
                        re_p = tr; im_p = ti;
                        const double ur = re_m * mr + im_m * mi, ui = -re_m * mi + im_m * mr;  // conj
                        re_m = ur; im_m = ui;
                    }
                    p.Lr[(size_t)r * n3 + i] += p.wr[r] * s0 * p.wsig[q] * (re_p + re_m);
                }
            }
        }
    }
    build_translate_multipliers(p);
    if (p.aniso) {
        if (d.svd_tol > 0 || d.svd_rank > 0) {
            err = "the VSS kernel factor is not compressed: svd_tol and svd_rank must be 0";
            return DGFS_ERR_UNSUPPORTED;
        }
        build_vss_tables(p);
    }
    return DGFS_OK;
}

uint64_t plan_fingerprint(const HostPlan& hp, int prec) {
    uint64_t h = 1469598103934665603ull;   // FNV-1a offset basis
    auto bytes = [&](const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;   // FNV prime
        }
    };
    auto i64 = [&](int64_t v) { bytes(&v, sizeof v); };
    auto f64 = [&](double v) { bytes(&v, sizeof v); };
    auto vec = [&](const std::vector<double>& v) {
        i64((int64_t)v.size());
        if (!v.empty()) bytes(v.data(), v.size() * sizeof(double));
    };
    i64(prec);
    i64(hp.N);
    i64(hp.Nrho);
    i64(hp.npairs);
    i64(hp.rank);
    i64(hp.loss_mode);
    i64(hp.aniso ? 1 : 0);
    f64(hp.L);
    f64(hp.R);
    f64(hp.gamma);
    f64(hp.b);
    f64(hp.alpha);
    for (const std::vector<double>* v : {&hp.cr, &hp.wr, &hp.sig, &hp.wsig, &hp.filt, &hp.Uk, &hp.Vr, &hp.Lr, &hp.Fa,
                                         &hp.GLa, &hp.mu})
        vec(*v);
    return h;
}

}  // namespace dgfs
