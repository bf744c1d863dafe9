// Host-side setup of the immersed discretisation and the multigrid hierarchy.
//
// Follows Sec. 2 (cut-cell quadrature, weak form, activity), Sec. 3.3 (two-scale
// restriction, Galerkin coarse operators, Remark 3.1) and Sec. 3.4 (Schwarz blocks by
// encapsulating supports, relaxation, Remark 3.3) of de Prenter et al., arXiv 1903.10977.
// The readings of the points the paper leaves open are the ones stated in imgm.h and in
// the comments below; the kernels only ever see the arrays produced here.
#include "setup.hpp"

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace imgm {
namespace {

constexpr int FULL = 0, EMPTY = 1, CUT = 2;
constexpr double PRUNE_RATIO = 1e-16;   // Remark 3.3
constexpr int MAX_COARSE_ROWS = 8192;   // dense coarsest-level inverse: at most 512 MiB

// ----------------------------------------------------------------------------------
// Small dense linear algebra (row-major n x n)
// ----------------------------------------------------------------------------------

// Gauss-Legendre rule on [0, 1] by Newton's method on the Legendre polynomial.
void gauss01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        {   // final derivative at the converged root
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        // roots come out in decreasing z; store increasing in [0, 1]
        x[n - 1 - i] = 0.5 * (z + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);   // 2/((1-z^2) P'^2) on [-1,1], halved
    }
}

// Cyclic Jacobi eigenvalue method for a symmetric matrix (A is overwritten).
// Rotations are applied while |a_pq| > eps sqrt(|a_pp a_qq|) (the Demmel-Veselic
// stopping rule, which keeps small eigenvalues of graded matrices accurate).  V (row-major) holds eigenvectors in columns.
void jacobi_eigen(std::vector<double>& A, int n, std::vector<double>& lam, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                if (apq == 0.0) continue;
                if (std::fabs(apq) <= 2.220446049250313e-16 * std::sqrt(std::fabs(app * aqq))) {
                    continue;
                }
                rotated = true;
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
        if (!rotated) break;
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

// Inverse of an SPD matrix through the Cholesky factor of its Jacobi-scaled form
// (A = D S D, A^{-1} = D^{-1} S^{-1} D^{-1}); false if S has a non-positive pivot.
bool scaled_cholesky_inverse(const std::vector<double>& A, int n, std::vector<double>& Ainv) {
    std::vector<double> d(n), L((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double a = A[(size_t)i * n + i];
        if (!(a > 0.0)) return false;
        d[i] = std::sqrt(a);
    }
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j] / (d[j] * d[j]);
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        double ljj = std::sqrt(s);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j] / (d[i] * d[j]);
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    // S^{-1} = L^{-T} L^{-1}: invert L column by column
    std::vector<double> Li((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c) {
        for (int i = c; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= L[(size_t)i * n + k] * Li[(size_t)k * n + c];
            Li[(size_t)i * n + c] = s / L[(size_t)i * n + i];
        }
    }
    Ainv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = 0.0;
            for (int k = i; k < n; ++k) s += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
            s /= d[i] * d[j];
            Ainv[(size_t)i * n + j] = Ainv[(size_t)j * n + i] = s;
        }
    return true;
}

// Remark 3.3: while lambda_min(A_j) < 1e-16 max_i (A_j)_ii, remove the function that
// dominates the eigenvector of lambda_min (lowest index on ties).  lambda_min is taken
// as 1/lambda_max(A_j^{-1}) with the inverse formed through the scaled Cholesky factor
// (lambda_max(A^{-1}) <= trace(A^{-1}) settles most blocks without an eigensolve).
// `keep` lists the kept positions; returns the number removed; Ainv receives the
// inverse of the kept block (empty when the kept block could not be factored).
int prune_and_invert(const std::vector<double>& Afull, int n, std::vector<int>& keep,
                     std::vector<double>& Ainv) {
    keep.resize(n);
    std::iota(keep.begin(), keep.end(), 0);
    int removed = 0;
    std::vector<double> A, lam, V;
    while (true) {
        int k = (int)keep.size();
        A.assign((size_t)k * k, 0.0);
        double maxdiag = 0.0;
        for (int i = 0; i < k; ++i) {
            for (int j = 0; j < k; ++j) A[(size_t)i * k + j] = Afull[(size_t)keep[i] * n + keep[j]];
            maxdiag = std::max(maxdiag, A[(size_t)i * k + i]);
        }
        double thr = PRUNE_RATIO * maxdiag;
        if (k == 1) {
            if (!(A[0] > 0.0)) return -1;
            Ainv.assign(1, 1.0 / A[0]);
            return removed;
        }
        int drop = -1;
        if (scaled_cholesky_inverse(A, k, Ainv)) {
            double tr = 0.0;
            for (int i = 0; i < k; ++i) tr += Ainv[(size_t)i * k + i];
            if (1.0 / tr >= thr) return removed;
            std::vector<double> B = Ainv;
            jacobi_eigen(B, k, lam, V);
            int top = (int)(std::max_element(lam.begin(), lam.end()) - lam.begin());
            if (1.0 / lam[top] >= thr) return removed;
            double best = -1.0;
            for (int i = 0; i < k; ++i) {
                double v = std::fabs(V[(size_t)i * k + top]);
                if (v > best) { best = v; drop = i; }
            }
        } else {
            std::vector<double> B = A;
            jacobi_eigen(B, k, lam, V);
            int bot = (int)(std::min_element(lam.begin(), lam.end()) - lam.begin());
            if (lam[bot] >= thr) return -1;      // positive definite yet not factorable
            double best = -1.0;
            for (int i = 0; i < k; ++i) {
                double v = std::fabs(V[(size_t)i * k + bot]);
                if (v > best) { best = v; drop = i; }
            }
        }
        keep.erase(keep.begin() + drop);
        ++removed;
    }
}

// ----------------------------------------------------------------------------------
// One-dimensional open uniform B-spline basis (triangular de Boor evaluation)
// ----------------------------------------------------------------------------------
struct Basis1D {
    int n = 0, p = 0, m = 0;
    double lo = 0.0, hi = 1.0, h = 1.0;
    std::vector<double> t;

    Basis1D() = default;
    Basis1D(int n_, int p_, double lo_, double hi_) : n(n_), p(p_), m(n_ + p_), lo(lo_), hi(hi_) {
        h = (hi - lo) / n;
        for (int k = 0; k <= p; ++k) t.push_back(lo);
        for (int k = 1; k < n; ++k) t.push_back(lo + k * h);
        for (int k = 0; k <= p; ++k) t.push_back(hi);
    }
    int sup_lo(int i) const { return std::max(0, i - p); }
    int sup_hi(int i) const { return std::min(n - 1, i); }

    // values N[0..p] and derivatives dN[0..p] of functions e..e+p at x in element e
    void eval(int e, double x, double* N, double* dN) const {
        const int s = e + p;
        double ndu[4][4], left[4], right[4];
        ndu[0][0] = 1.0;
        for (int j = 1; j <= p; ++j) {
            left[j] = x - t[s + 1 - j];
            right[j] = t[s + j] - x;
            double saved = 0.0;
            for (int r = 0; r < j; ++r) {
                ndu[j][r] = right[r + 1] + left[j - r];
                double tmp = ndu[r][j - 1] / ndu[j][r];
                ndu[r][j] = saved + right[r + 1] * tmp;
                saved = left[j - r] * tmp;
            }
            ndu[j][j] = saved;
        }
        for (int r = 0; r <= p; ++r) N[r] = ndu[r][p];
        for (int r = 0; r <= p; ++r) {
            double d = 0.0;
            if (p > 0) {
                if (r >= 1) d += ndu[r - 1][p - 1] / ndu[p][r - 1];
                if (r <= p - 1) d -= ndu[r][p - 1] / ndu[p][r];
            }
            dN[r] = p * d;
        }
    }
};

// Two-scale matrix R1 (m_c x m_f, row-major): phi^c_i = sum_a R1[i][a] phi^f_a, by
// Boehm's algorithm inserting the midpoint of every coarse element.
std::vector<double> two_scale(const Basis1D& c, const Basis1D& f) {
    const int p = c.p;
    std::vector<double> T = c.t;
    int mc = c.m, cur = c.m;
    std::vector<double> P((size_t)mc * cur, 0.0);
    for (int i = 0; i < mc; ++i) P[(size_t)i * cur + i] = 1.0;
    for (int e = 0; e < c.n; ++e) {
        double u = c.lo + (e + 0.5) * c.h;
        int k = (int)(std::upper_bound(T.begin(), T.end(), u) - T.begin()) - 1;   // T[k] <= u < T[k+1]
        std::vector<double> Q((size_t)mc * (cur + 1), 0.0);
        for (int i = 0; i < mc; ++i) {
            const double* Pi = &P[(size_t)i * cur];
            double* Qi = &Q[(size_t)i * (cur + 1)];
            for (int j = 0; j <= cur; ++j) {
                if (j <= k - p) {
                    Qi[j] = Pi[j];
                } else if (j >= k + 1) {
                    Qi[j] = Pi[j - 1];
                } else {
                    double a = (u - T[j]) / (T[j + p] - T[j]);
                    Qi[j] = a * Pi[j] + (1.0 - a) * Pi[j - 1];
                }
            }
        }
        T.insert(T.begin() + k + 1, u);
        P.swap(Q);
        ++cur;
    }
    if (cur != f.m) throw std::runtime_error("two-scale: knot insertion did not reach the fine basis");
    for (double& v : P)
        if (std::fabs(v) < 1e-14) v = 0.0;
    return P;
}

// ----------------------------------------------------------------------------------
// Geometry and cut-cell quadrature (Sec. 2, Fig. 1)
// ----------------------------------------------------------------------------------
struct Geometry {
    int dim;
    std::vector<Ball> balls;

    double psi(const double* x) const {
        double best = INFINITY;
        for (const Ball& b : balls) {
            double s = 0.0;
            for (int k = 0; k < dim; ++k) s += (x[k] - b.c[k]) * (x[k] - b.c[k]);
            best = std::min(best, std::sqrt(s) - b.r);
        }
        return best;
    }
    // exact classification of the closed box [lo, hi] against the balls
    int classify(const double* lo, const double* hi) const {
        bool cut = false;
        for (const Ball& b : balls) {
            double dmin = 0.0, dmax = 0.0;
            for (int k = 0; k < dim; ++k) {
                double nearest = std::min(std::max(b.c[k], lo[k]), hi[k]);
                dmin += (nearest - b.c[k]) * (nearest - b.c[k]);
                double far = std::fabs(b.c[k] - lo[k]) > std::fabs(b.c[k] - hi[k]) ? lo[k] : hi[k];
                dmax += (far - b.c[k]) * (far - b.c[k]);
            }
            dmin = std::sqrt(dmin);
            dmax = std::sqrt(dmax);
            if (dmax <= b.r) return EMPTY;
            if (dmin < b.r) cut = true;
        }
        return cut ? CUT : FULL;
    }
};

struct Rule {
    std::vector<double> vp, vw;          // volume points (npts x dim) and weights
    std::vector<double> bp, bw, bn;      // boundary points, weights, normals
};

struct Pt { double x[3]; };

static void simplex_rule(const Pt* V, int dim, int n, const std::vector<double>& g, const std::vector<double>& w,
                         Rule& R) {
    if (dim == 2) {
        double e1[2] = {V[1].x[0] - V[0].x[0], V[1].x[1] - V[0].x[1]};
        double e2[2] = {V[2].x[0] - V[1].x[0], V[2].x[1] - V[1].x[1]};
        double det = std::fabs(e1[0] * e2[1] - e1[1] * e2[0]);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double u = g[i], v = g[j];
                for (int k = 0; k < 2; ++k) R.vp.push_back(V[0].x[k] + u * e1[k] + u * v * e2[k]);
                R.vw.push_back(w[i] * w[j] * u * det);
            }
    } else {
        double e1[3], e2[3], e3[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = V[1].x[k] - V[0].x[k];
            e2[k] = V[2].x[k] - V[1].x[k];
            e3[k] = V[3].x[k] - V[2].x[k];
        }
        double det = std::fabs(e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                               e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]));
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int l = 0; l < n; ++l) {
                    double u = g[i], v = g[j], s = g[l];
                    for (int k = 0; k < 3; ++k)
                        R.vp.push_back(V[0].x[k] + u * e1[k] + u * v * e2[k] + u * v * s * e3[k]);
                    R.vw.push_back(w[i] * w[j] * w[l] * u * u * v * det);
                }
    }
}

static void facet_rule(const Pt* F, int dim, int n, const std::vector<double>& g, const std::vector<double>& w,
                       const double* normal, Rule& R) {
    if (dim == 2) {
        double e[2] = {F[1].x[0] - F[0].x[0], F[1].x[1] - F[0].x[1]};
        double L = std::sqrt(e[0] * e[0] + e[1] * e[1]);
        for (int i = 0; i < n; ++i) {
            for (int k = 0; k < 2; ++k) R.bp.push_back(F[0].x[k] + g[i] * e[k]);
            R.bw.push_back(w[i] * L);
            for (int k = 0; k < 2; ++k) R.bn.push_back(normal[k]);
        }
    } else {
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = F[1].x[k] - F[0].x[k];
            e2[k] = F[2].x[k] - F[1].x[k];
        }
        double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
        double area2 = std::sqrt(cx * cx + cy * cy + cz * cz);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double u = g[i], v = g[j];
                for (int k = 0; k < 3; ++k) R.bp.push_back(F[0].x[k] + u * e1[k] + u * v * e2[k]);
                R.bw.push_back(w[i] * w[j] * u * area2);
                for (int k = 0; k < 3; ++k) R.bn.push_back(normal[k]);
            }
    }
}

static Pt crossing(const Pt& a, const Pt& b, double pa, double pb, int dim) {
    Pt r{};
    double s = pa / (pa - pb);
    for (int k = 0; k < dim; ++k) r.x[k] = a.x[k] + s * (b.x[k] - a.x[k]);
    return r;
}

// Clips the simplex V (dim+1 vertices) at psi_lin = 0 and appends the rules of the kept
// sub-simplices and boundary facets (canonical decomposition of the quadrature reading).
static void clip_simplex(const Pt* V, const double* ps, int dim, int np, const std::vector<double>& g,
                         const std::vector<double>& w, Rule& R) {
    int in[4], out[4], ni = 0, no = 0;
    for (int i = 0; i <= dim; ++i) {
        if (ps[i] > 0) in[ni++] = i;
        else out[no++] = i;
    }
    if (ni == 0) return;
    if (ni == dim + 1) {
        simplex_rule(V, dim, np, g, w, R);
        return;
    }
    // gradient of the linear interpolant: (V_i - V_0) . grad = psi_i - psi_0
    double M[3][3], rhs[3], grad[3];
    for (int i = 0; i < dim; ++i) {
        for (int k = 0; k < dim; ++k) M[i][k] = V[i + 1].x[k] - V[0].x[k];
        rhs[i] = ps[i + 1] - ps[0];
    }
    if (dim == 2) {
        double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
        grad[0] = (rhs[0] * M[1][1] - M[0][1] * rhs[1]) / det;
        grad[1] = (M[0][0] * rhs[1] - rhs[0] * M[1][0]) / det;
    } else {
        double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                     M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        for (int c = 0; c < 3; ++c) {
            double Mc[3][3];
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) Mc[i][k] = (k == c) ? rhs[i] : M[i][k];
            double dc = Mc[0][0] * (Mc[1][1] * Mc[2][2] - Mc[1][2] * Mc[2][1]) -
                        Mc[0][1] * (Mc[1][0] * Mc[2][2] - Mc[1][2] * Mc[2][0]) +
                        Mc[0][2] * (Mc[1][0] * Mc[2][1] - Mc[1][1] * Mc[2][0]);
            grad[c] = dc / det;
        }
    }
    double gn = 0.0;
    for (int k = 0; k < dim; ++k) gn += grad[k] * grad[k];
    gn = std::sqrt(gn);
    double normal[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) normal[k] = -grad[k] / gn;
    auto X = [&](int i, int j) { return crossing(V[i], V[j], ps[i], ps[j], dim); };
    if (dim == 2) {
        if (ni == 1) {
            int a = in[0], b = out[0], c = out[1];
            Pt T[3] = {V[a], X(a, b), X(a, c)};
            simplex_rule(T, 2, np, g, w, R);
            Pt F[2] = {X(a, b), X(a, c)};
            facet_rule(F, 2, np, g, w, normal, R);
        } else {
            int a = in[0], b = in[1], c = out[0];
            Pt T1[3] = {V[a], V[b], X(b, c)};
            Pt T2[3] = {V[a], X(b, c), X(a, c)};
            simplex_rule(T1, 2, np, g, w, R);
            simplex_rule(T2, 2, np, g, w, R);
            Pt F[2] = {X(a, c), X(b, c)};
            facet_rule(F, 2, np, g, w, normal, R);
        }
        return;
    }
    auto prism = [&](const Pt* P, const Pt* Q) {
        Pt T1[4] = {P[0], P[1], P[2], Q[2]};
        Pt T2[4] = {P[0], P[1], Q[1], Q[2]};
        Pt T3[4] = {P[0], Q[0], Q[1], Q[2]};
        simplex_rule(T1, 3, np, g, w, R);
        simplex_rule(T2, 3, np, g, w, R);
        simplex_rule(T3, 3, np, g, w, R);
    };
    if (ni == 1) {
        int a = in[0], b = out[0], c = out[1], d = out[2];
        Pt T[4] = {V[a], X(a, b), X(a, c), X(a, d)};
        simplex_rule(T, 3, np, g, w, R);
        Pt F[3] = {X(a, b), X(a, c), X(a, d)};
        facet_rule(F, 3, np, g, w, normal, R);
    } else if (ni == 2) {
        int a = in[0], b = in[1], c = out[0], d = out[1];
        Pt P[3] = {V[a], X(a, c), X(a, d)};
        Pt Q[3] = {V[b], X(b, c), X(b, d)};
        prism(P, Q);
        Pt F1[3] = {X(a, c), X(a, d), X(b, d)};
        Pt F2[3] = {X(a, c), X(b, d), X(b, c)};
        facet_rule(F1, 3, np, g, w, normal, R);
        facet_rule(F2, 3, np, g, w, normal, R);
    } else {
        int a = in[0], b = in[1], c = in[2], d = out[0];
        Pt P[3] = {V[a], V[b], V[c]};
        Pt Q[3] = {X(a, d), X(b, d), X(c, d)};
        prism(P, Q);
        Pt F[3] = {X(a, d), X(b, d), X(c, d)};
        facet_rule(F, 3, np, g, w, normal, R);
    }
}

static void box_rule(const double* lo, const double* hi, int dim, int n, const std::vector<double>& g,
                     const std::vector<double>& w, Rule& R) {
    int tot = 1;
    for (int k = 0; k < dim; ++k) tot *= n;
    for (int q = 0; q < tot; ++q) {
        int idx[3] = {q % n, (q / n) % n, q / (n * n)};
        double wt = 1.0;
        for (int k = 0; k < dim; ++k) {
            R.vp.push_back(lo[k] + (hi[k] - lo[k]) * g[idx[k]]);
            wt *= (hi[k] - lo[k]) * w[idx[k]];
        }
        R.vw.push_back(wt);
    }
}

// The cut-element rule: bisect `depth` times, classify leaves, Gauss on full leaves,
// Kuhn simplices clipped at psi_lin = 0 on cut leaves.
Rule cut_element_rule(const Geometry& G, const double* lo, const double* hi, int p, int depth) {
    const int dim = G.dim;
    Rule R;
    std::vector<double> g1, w1, g2, w2;
    gauss01(p + 1, g1, w1);
    gauss01(p + 2, g2, w2);
    const int k = 1 << depth;
    double step[3];
    for (int d = 0; d < dim; ++d) step[d] = (hi[d] - lo[d]) / k;
    int nleaf = 1;
    for (int d = 0; d < dim; ++d) nleaf *= k;
    for (int l = 0; l < nleaf; ++l) {
        int idx[3] = {l % k, (l / k) % k, l / (k * k)};
        double a[3], b[3];
        for (int d = 0; d < dim; ++d) {
            a[d] = lo[d] + idx[d] * step[d];
            b[d] = a[d] + step[d];
        }
        int cls = G.classify(a, b);
        if (cls == EMPTY) continue;
        if (cls == FULL) {
            box_rule(a, b, dim, p + 1, g1, w1, R);
            continue;
        }
        auto corner = [&](int bx, int by, int bz) {
            Pt c{};
            c.x[0] = bx ? b[0] : a[0];
            c.x[1] = by ? b[1] : a[1];
            if (dim == 3) c.x[2] = bz ? b[2] : a[2];
            return c;
        };
        if (dim == 2) {
            Pt S1[3] = {corner(0, 0, 0), corner(1, 0, 0), corner(1, 1, 0)};
            Pt S2[3] = {corner(0, 0, 0), corner(1, 1, 0), corner(0, 1, 0)};
            for (const Pt* S : {S1, S2}) {
                double ps[3];
                for (int i = 0; i < 3; ++i) ps[i] = G.psi(S[i].x);
                clip_simplex(S, ps, 2, p + 2, g2, w2, R);
            }
        } else {
            static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
            for (const auto& pm : perms) {
                int bits[3] = {0, 0, 0};
                Pt S[4];
                S[0] = corner(0, 0, 0);
                for (int s = 0; s < 3; ++s) {
                    bits[pm[s]] = 1;
                    S[s + 1] = corner(bits[0], bits[1], bits[2]);
                }
                double ps[4];
                for (int i = 0; i < 4; ++i) ps[i] = G.psi(S[i].x);
                clip_simplex(S, ps, 3, p + 2, g2, w2, R);
            }
        }
    }
    return R;
}

// ----------------------------------------------------------------------------------
// Element systems
// ----------------------------------------------------------------------------------
inline double f_rhs(const double* x, int dim) {      // f = d pi^2 prod sin(pi x_k)
    double s = 1.0;
    for (int k = 0; k < dim; ++k) s *= std::sin(M_PI * x[k]);
    return dim * M_PI * M_PI * s;
}
inline double g_bc(const double* x, int dim) {       // g = u = prod sin(pi x_k)
    double s = 1.0;
    for (int k = 0; k < dim; ++k) s *= std::sin(M_PI * x[k]);
    return s;
}

struct TensorEval {
    int dim, p, nloc;
    const Basis1D* b;
    // values and gradients of the local functions of element e (multi-index) at x
    void operator()(const int* e, const double* x, double* val, double* grad /* dim x nloc */) const {
        double N[3][4], dN[3][4];
        for (int k = 0; k < dim; ++k) b->eval(e[k], x[k], N[k], dN[k]);
        const int q = p + 1;
        for (int a = 0; a < nloc; ++a) {
            int ai[3] = {a % q, (a / q) % q, a / (q * q)};
            double v = 1.0;
            for (int k = 0; k < dim; ++k) v *= N[k][ai[k]];
            val[a] = v;
            for (int j = 0; j < dim; ++j) {
                double gj = 1.0;
                for (int k = 0; k < dim; ++k) gj *= (k == j) ? dN[k][ai[k]] : N[k][ai[k]];
                grad[j * nloc + a] = gj;
            }
        }
    }
};

// beta_K = 2^ceil(log2(2 max(lambda, 1/h))), lambda the largest eigenvalue of
// (Bn, S) on the functions orthogonal to the constants (reading of Nitsche's parameter).
double nitsche_beta(const std::vector<double>& S, const std::vector<double>& Bn, int n, double h) {
    // Householder reflector H = I - 2 v v^T / v^T v maps 1/sqrt(n) to -e_0; columns 1..n-1
    // of H are an orthonormal basis of the complement of the constants
    std::vector<double> v(n, 1.0);
    v[0] += std::sqrt((double)n);
    double vv = 0.0;
    for (double x : v) vv += x * x;
    const int k = n - 1;
    std::vector<double> Q((size_t)n * k);
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < k; ++c) Q[(size_t)i * k + c] = ((i == c + 1) ? 1.0 : 0.0) - 2.0 * v[i] * v[c + 1] / vv;
    auto project = [&](const std::vector<double>& A) {
        std::vector<double> AQ((size_t)n * k, 0.0), out((size_t)k * k, 0.0);
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < k; ++c) {
                double s = 0.0;
                for (int j = 0; j < n; ++j) s += A[(size_t)i * n + j] * Q[(size_t)j * k + c];
                AQ[(size_t)i * k + c] = s;
            }
        for (int r = 0; r < k; ++r)
            for (int c = 0; c < k; ++c) {
                double s = 0.0;
                for (int i = 0; i < n; ++i) s += Q[(size_t)i * k + r] * AQ[(size_t)i * k + c];
                out[(size_t)r * k + c] = s;
            }
        for (int r = 0; r < k; ++r)
            for (int c = 0; c < r; ++c) {
                double m = 0.5 * (out[(size_t)r * k + c] + out[(size_t)c * k + r]);
                out[(size_t)r * k + c] = out[(size_t)c * k + r] = m;
            }
        return out;
    };
    std::vector<double> Sh = project(S), Bh = project(Bn);
    std::vector<double> mu, W;
    jacobi_eigen(Sh, k, mu, W);
    double mumax = *std::max_element(mu.begin(), mu.end());
    std::vector<int> keep;
    for (int i = 0; i < k; ++i)
        if (mu[i] > 1e-14 * mumax) keep.push_back(i);
    const int r = (int)keep.size();
    std::vector<double> T((size_t)k * r);
    for (int i = 0; i < k; ++i)
        for (int c = 0; c < r; ++c) T[(size_t)i * r + c] = W[(size_t)i * k + keep[c]] / std::sqrt(mu[keep[c]]);
    std::vector<double> BT((size_t)k * r, 0.0), C((size_t)r * r, 0.0);
    for (int i = 0; i < k; ++i)
        for (int c = 0; c < r; ++c) {
            double s = 0.0;
            for (int j = 0; j < k; ++j) s += Bh[(size_t)i * k + j] * T[(size_t)j * r + c];
            BT[(size_t)i * r + c] = s;
        }
    for (int a = 0; a < r; ++a)
        for (int c = 0; c < r; ++c) {
            double s = 0.0;
            for (int i = 0; i < k; ++i) s += T[(size_t)i * r + a] * BT[(size_t)i * r + c];
            C[(size_t)a * r + c] = s;
        }
    for (int a = 0; a < r; ++a)
        for (int c = 0; c < a; ++c) {
            double m = 0.5 * (C[(size_t)a * r + c] + C[(size_t)c * r + a]);
            C[(size_t)a * r + c] = C[(size_t)c * r + a] = m;
        }
    std::vector<double> lam, V;
    jacobi_eigen(C, r, lam, V);
    double lmax = *std::max_element(lam.begin(), lam.end());
    lmax = std::max(lmax, 1.0 / h);
    return std::ldexp(1.0, (int)std::ceil(std::log2(2.0 * lmax)));
}

struct CutElem {
    int64_t E;
    double volume;
    std::vector<double> A;   // nloc x nloc
    std::vector<double> b;   // nloc
};

// S (upper triangle) += w sum_j g_j g_j^T for the nloc-vectors g_j = grad + j nloc;
// NL > 0 fixes nloc at compile time so that the inner loop is unrolled and vectorised
template <int NL>
void add_grad_outer(double* S, const double* grad, int dim, int nloc_rt, double w) {
    const int nloc = NL > 0 ? NL : nloc_rt;
    for (int j = 0; j < dim; ++j) {
        const double* gj = grad + (size_t)j * nloc;
        for (int a = 0; a < nloc; ++a) {
            const double t = w * gj[a];
            double* Sa = S + (size_t)a * nloc;
            for (int c = a; c < nloc; ++c) Sa[c] += t * gj[c];
        }
    }
}

void add_grad_outer_any(double* S, const double* grad, int dim, int nloc, double w) {
    switch (nloc) {
        case 4: add_grad_outer<4>(S, grad, dim, nloc, w); break;
        case 8: add_grad_outer<8>(S, grad, dim, nloc, w); break;
        case 9: add_grad_outer<9>(S, grad, dim, nloc, w); break;
        case 16: add_grad_outer<16>(S, grad, dim, nloc, w); break;
        case 27: add_grad_outer<27>(S, grad, dim, nloc, w); break;
        case 64: add_grad_outer<64>(S, grad, dim, nloc, w); break;
        default: add_grad_outer<0>(S, grad, dim, nloc, w); break;
    }
}

void cut_element_system(const Geometry& G, const Basis1D& B, int dim, int p, int depth, int bc, const int* e,
                        const double* lo, const double* hi, CutElem& out) {
    const int nloc = (dim == 2) ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1);
    Rule R = cut_element_rule(G, lo, hi, p, depth);
    TensorEval te{dim, p, nloc, &B};
    std::vector<double> S((size_t)nloc * nloc, 0.0), rhs(nloc, 0.0);
    std::vector<double> val(nloc), grad((size_t)dim * nloc);
    double vol = 0.0;
    const size_t nv = R.vw.size();
    // S = sum_q w_q sum_j grad_j(q) grad_j(q)^T, upper triangle accumulated with the
    // contiguous index innermost, then mirrored
    for (size_t q = 0; q < nv; ++q) {
        const double* x = &R.vp[q * dim];
        double w = R.vw[q];
        vol += w;
        te(e, x, val.data(), grad.data());
        double fw = w * f_rhs(x, dim);
        for (int a = 0; a < nloc; ++a) rhs[a] += val[a] * fw;
        add_grad_outer_any(S.data(), grad.data(), dim, nloc, w);
    }
    for (int a = 0; a < nloc; ++a)
        for (int c = 0; c < a; ++c) S[(size_t)a * nloc + c] = S[(size_t)c * nloc + a];
    std::vector<double> A = S;
    const size_t nb = R.bw.size();
    if (nb > 0) {
        std::vector<double> Bn((size_t)nloc * nloc, 0.0), C((size_t)nloc * nloc, 0.0), Mb((size_t)nloc * nloc, 0.0);
        std::vector<double> bv((size_t)nb * nloc), dn((size_t)nb * nloc), gq(nb);
        for (size_t q = 0; q < nb; ++q) {
            const double* x = &R.bp[q * dim];
            te(e, x, val.data(), grad.data());
            for (int a = 0; a < nloc; ++a) {
                double s = 0.0;
                for (int j = 0; j < dim; ++j) s += grad[j * nloc + a] * R.bn[q * dim + j];
                dn[q * nloc + a] = s;
                bv[q * nloc + a] = val[a];
            }
            gq[q] = g_bc(x, dim);
        }
        for (size_t q = 0; q < nb; ++q) {
            const double w = R.bw[q];
            const double* bq = &bv[q * nloc];
            const double* dq = &dn[q * nloc];
            for (int a = 0; a < nloc; ++a) {
                const double wb = w * bq[a], wd = w * dq[a];
                double* Ma = &Mb[(size_t)a * nloc];
                double* Ba = &Bn[(size_t)a * nloc];
                double* Ca = &C[(size_t)a * nloc];
                for (int c = a; c < nloc; ++c) {
                    Ma[c] += wb * bq[c];
                    Ba[c] += wd * dq[c];
                }
                for (int c = 0; c < nloc; ++c) Ca[c] += wd * bq[c];
            }
        }
        for (int a = 0; a < nloc; ++a)
            for (int c = 0; c < a; ++c) {
                Mb[(size_t)a * nloc + c] = Mb[(size_t)c * nloc + a];
                Bn[(size_t)a * nloc + c] = Bn[(size_t)c * nloc + a];
            }
        double beta;
        if (bc == 0) {
            beta = 2.0 / B.h;                    // the paper's penalty parameter 2/h
            for (size_t i = 0; i < A.size(); ++i) A[i] += beta * Mb[i];
            for (size_t q = 0; q < nb; ++q)
                for (int a = 0; a < nloc; ++a) rhs[a] += beta * R.bw[q] * bv[q * nloc + a] * gq[q];
        } else {
            beta = nitsche_beta(S, Bn, nloc, B.h);
            for (int a = 0; a < nloc; ++a)
                for (int c = 0; c < nloc; ++c)
                    A[(size_t)a * nloc + c] += -(C[(size_t)a * nloc + c] + C[(size_t)c * nloc + a]) + beta * Mb[(size_t)a * nloc + c];
            for (size_t q = 0; q < nb; ++q)
                for (int a = 0; a < nloc; ++a)
                    rhs[a] += R.bw[q] * gq[q] * (-dn[q * nloc + a] + beta * bv[q * nloc + a]);
        }
    }
    out.volume = vol;
    out.A.swap(A);
    out.b.swap(rhs);
}

// 1-D element stiffness / mass (p+1)^2 of every element of a basis, by Gauss with p+1 points
void element_matrices_1d(const Basis1D& B, std::vector<double>& Ke, std::vector<double>& Me) {
    const int q = B.p + 1;
    std::vector<double> g, w;
    gauss01(q, g, w);
    Ke.assign((size_t)B.n * q * q, 0.0);
    Me.assign((size_t)B.n * q * q, 0.0);
    double N[4], dN[4];
    for (int e = 0; e < B.n; ++e) {
        double lo = B.lo + e * B.h, hi = lo + B.h;
        for (int k = 0; k < q; ++k) {
            double x = lo + (hi - lo) * g[k], wt = (hi - lo) * w[k];
            B.eval(e, x, N, dN);
            for (int a = 0; a < q; ++a)
                for (int c = 0; c < q; ++c) {
                    Ke[((size_t)e * q + a) * q + c] += wt * dN[a] * dN[c];
                    Me[((size_t)e * q + a) * q + c] += wt * N[a] * N[c];
                }
        }
    }
}

// ----------------------------------------------------------------------------------
// Hierarchy construction
// ----------------------------------------------------------------------------------
struct Builder {
    const Problem& pb;
    Hierarchy& H;
    int dim, p, L, W, ncoef;     // W = 2p+1
    std::vector<Basis1D> basis;  // per level index (0 = coarsest)
    std::vector<std::vector<double>> Ke, Me;

    Builder(const Problem& pb_, Hierarchy& H_) : pb(pb_), H(H_) {
        dim = pb.dim;
        p = pb.p;
        L = pb.levels;
        W = 2 * p + 1;
        ncoef = (dim == 2) ? W * W : W * W * W;
    }

    int64_t pw(int64_t m, int k) const { return k == 0 ? 1 : m * pw(m, k - 1); }

    void unflat(int64_t i, int64_t m, int* c) const {
        c[0] = (int)(i % m);
        c[1] = (int)((i / m) % m);
        c[2] = (dim == 3) ? (int)(i / (m * m)) : 0;
    }
    int64_t flat(const int* c, int64_t m) const { return c[0] + m * (c[1] + (dim == 3 ? m * c[2] : 0)); }

    // coefficient index of offset o (each in -p..p), x-fastest
    int coef_index(const int* o) const { return (o[0] + p) + W * ((o[1] + p) + (dim == 3 ? W * (o[2] + p) : 0)); }

    // full (2p+1)^d row of level lv: tensor formula, stored row, or zeros
    void row_coeffs(const LevelData& lv, int64_t row, double* out) const {
        std::fill(out, out + ncoef, 0.0);
        int ri = lv.rowinfo[row];
        if (ri == -2) return;
        const int64_t nb = (int64_t)lv.band_rows.size();
        if (ri >= 0) {
            for (int c = 0; c < ncoef; ++c) out[c] = lv.band_coef[(size_t)c * nb + ri];
            return;
        }
        int i[3];
        unflat(row, lv.m, i);
        for (int c = 0; c < ncoef; ++c) {
            int o[3] = {c % W - p, (c / W) % W - p, (dim == 3) ? c / (W * W) - p : 0};
            int j[3] = {i[0] + o[0], i[1] + o[1], i[2] + o[2]};
            bool ok = true;
            for (int k = 0; k < dim; ++k) ok = ok && j[k] >= 0 && j[k] < lv.m;
            if (!ok || !lv.active[flat(j, lv.m)]) continue;
            const double* K = &lv.K1[0];
            const double* M = &lv.M1[0];
            double v;
            if (dim == 2) {
                v = K[i[0] * W + o[0] + p] * M[i[1] * W + o[1] + p] + M[i[0] * W + o[0] + p] * K[i[1] * W + o[1] + p];
            } else {
                double kx = K[i[0] * W + o[0] + p], mx = M[i[0] * W + o[0] + p];
                double ky = K[i[1] * W + o[1] + p], my = M[i[1] * W + o[1] + p];
                double kz = K[i[2] * W + o[2] + p], mz = M[i[2] * W + o[2] + p];
                v = kx * my * mz + mx * ky * mz + mx * my * kz;
            }
            out[c] = v;
        }
    }

    void build_1d_tables(LevelData& lv, int li) {
        const Basis1D& B = basis[li];
        const int q = p + 1;
        lv.K1.assign((size_t)B.m * W, 0.0);
        lv.M1.assign((size_t)B.m * W, 0.0);
        for (int e = 0; e < B.n; ++e)
            for (int a = 0; a < q; ++a)
                for (int c = 0; c < q; ++c) {
                    int i = e + a, j = e + c;
                    lv.K1[(size_t)i * W + (j - i + p)] += Ke[li][((size_t)e * q + a) * q + c];
                    lv.M1[(size_t)i * W + (j - i + p)] += Me[li][((size_t)e * q + a) * q + c];
                }
    }

    // functions active / rows stored, from the element status of the level
    void classify_rows(LevelData& lv) {
        const int64_t m = lv.m, N = lv.N;
        lv.active.assign(N, 0);
        lv.rowinfo.assign(N, -2);
        std::vector<uint8_t> band(N, 0);
        const int n = lv.n;
        for (int64_t r = 0; r < N; ++r) {
            int i[3];
            unflat(r, m, i);
            bool on_box = false;
            for (int k = 0; k < dim; ++k) on_box = on_box || i[k] == 0 || i[k] == m - 1;
            int lo3[3] = {0, 0, 0}, hi3[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k) {
                lo3[k] = std::max(0, i[k] - p);
                hi3[k] = std::min(n - 1, i[k]);
            }
            bool act = false, nonfull = false;
            for (int ez = lo3[2]; ez <= hi3[2]; ++ez)
                for (int ey = lo3[1]; ey <= hi3[1]; ++ey)
                    for (int ex = lo3[0]; ex <= hi3[0]; ++ex) {
                        int64_t E = ex + (int64_t)n * (ey + (dim == 3 ? (int64_t)n * ez : 0));
                        act = act || lv.elem_active[E];
                        nonfull = nonfull || !lv.elem_full[E];
                    }
            if (act && !on_box) {
                lv.active[r] = 1;
                band[r] = nonfull;
            }
        }
        lv.band_rows.clear();
        lv.n_active = 0;
        for (int64_t r = 0; r < N; ++r) {
            if (!lv.active[r]) continue;
            ++lv.n_active;
            if (band[r]) {
                lv.rowinfo[r] = (int32_t)lv.band_rows.size();
                lv.band_rows.push_back((int32_t)r);
            } else {
                lv.rowinfo[r] = -1;
            }
        }
        lv.band_coef.assign((size_t)ncoef * lv.band_rows.size(), 0.0);
    }

    bool build_finest(std::string& err) {
        const int li = L - 1;
        LevelData& lv = H.lv[li];
        const Basis1D& B = basis[li];
        Geometry G{dim, pb.holes};
        const int n = B.n;
        const int64_t NE = pw(n, dim);
        lv.elem_active.assign(NE, 0);
        lv.elem_full.assign(NE, 0);
        std::vector<int64_t> cut;
        for (int64_t E = 0; E < NE; ++E) {
            int e[3];
            unflat(E, n, e);
            double lo[3], hi[3];
            for (int k = 0; k < dim; ++k) {
                lo[k] = pb.lo + e[k] * B.h;
                hi[k] = lo[k] + B.h;
            }
            int c = G.classify(lo, hi);
            if (c == FULL) {
                lv.elem_full[E] = 1;
                lv.elem_active[E] = 1;
            } else if (c == CUT) {
                cut.push_back(E);
            }
        }
        H.n_cut = (int64_t)cut.size();
        const bool verbose = std::getenv("IMGM_VERBOSE") != nullptr;
        auto t = std::chrono::steady_clock::now();
        auto phase = [&](const char* name) {
            const auto now = std::chrono::steady_clock::now();
            if (verbose) std::fprintf(stderr, "imgm: setup   %-20s %8.3f s\n", name, std::chrono::duration<double>(now - t).count());
            t = now;
        };
        std::vector<CutElem> ce(cut.size());
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t c = 0; c < (int64_t)cut.size(); ++c) {
            int e[3];
            unflat(cut[c], n, e);
            double lo[3], hi[3];
            for (int k = 0; k < dim; ++k) {
                lo[k] = pb.lo + e[k] * B.h;
                hi[k] = lo[k] + B.h;
            }
            ce[c].E = cut[c];
            cut_element_system(G, B, dim, p, pb.depth, pb.bc, e, lo, hi, ce[c]);
        }
        phase("cut elements");
        std::vector<int32_t> cut_id(NE, -1);
        for (size_t c = 0; c < ce.size(); ++c) {
            cut_id[ce[c].E] = (int32_t)c;
            if (ce[c].volume > 0) lv.elem_active[ce[c].E] = 1;
        }
        classify_rows(lv);
        build_1d_tables(lv, li);

        const int q = p + 1;
        const int nloc = (dim == 2) ? q * q : q * q * q;
        const std::vector<double>& ke = Ke[li];
        const std::vector<double>& me = Me[li];
        // element matrix entry (a, c) of a full element e (tensor of 1-D element matrices)
        auto full_entry = [&](const int* e, const int* a, const int* c) {
            double kx = ke[((size_t)e[0] * q + a[0]) * q + c[0]], mx = me[((size_t)e[0] * q + a[0]) * q + c[0]];
            double ky = ke[((size_t)e[1] * q + a[1]) * q + c[1]], my = me[((size_t)e[1] * q + a[1]) * q + c[1]];
            if (dim == 2) return kx * my + mx * ky;
            double kz = ke[((size_t)e[2] * q + a[2]) * q + c[2]], mz = me[((size_t)e[2] * q + a[2]) * q + c[2]];
            return kx * my * mz + mx * ky * mz + mx * my * kz;
        };
        // stored rows: sum of the element matrices of the active support elements
        const int64_t nb = (int64_t)lv.band_rows.size();
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t bi = 0; bi < nb; ++bi) {
            const int64_t r = lv.band_rows[bi];
            int i[3];
            unflat(r, lv.m, i);
            int lo3[3] = {0, 0, 0}, hi3[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k) {
                lo3[k] = std::max(0, i[k] - p);
                hi3[k] = std::min(n - 1, i[k]);
            }
            std::vector<double> row(ncoef, 0.0);
            for (int ez = lo3[2]; ez <= hi3[2]; ++ez)
                for (int ey = lo3[1]; ey <= hi3[1]; ++ey)
                    for (int ex = lo3[0]; ex <= hi3[0]; ++ex) {
                        int e[3] = {ex, ey, ez};
                        int64_t E = flat(e, n);
                        if (!lv.elem_active[E]) continue;
                        int a[3] = {i[0] - e[0], i[1] - e[1], dim == 3 ? i[2] - e[2] : 0};
                        int aflat = a[0] + q * (a[1] + q * a[2]);
                        for (int cl = 0; cl < nloc; ++cl) {
                            int c[3] = {cl % q, (cl / q) % q, cl / (q * q)};
                            int j[3] = {e[0] + c[0], e[1] + c[1], dim == 3 ? e[2] + c[2] : 0};
                            if (!lv.active[flat(j, lv.m)]) continue;
                            int o[3] = {j[0] - i[0], j[1] - i[1], j[2] - i[2]};
                            double v = lv.elem_full[E] ? full_entry(e, a, c)
                                                        : ce[cut_id[E]].A[(size_t)aflat * nloc + cl];
                            row[coef_index(o)] += v;
                        }
                    }
            for (int c = 0; c < ncoef; ++c) lv.band_coef[(size_t)c * nb + bi] = row[c];
        }
        phase("stored rows");
        // right-hand side, element by element; elements are taken in (p+1)^d colour
        // classes (e_k mod (p+1) per direction) whose members share no function, so each
        // class scatters into b in parallel without races
        H.b.assign(lv.N, 0.0);
        std::vector<double> g1, w1;
        gauss01(q, g1, w1);
        const int ncol = (dim == 2) ? q * q : q * q * q;
        for (int col = 0; col < ncol; ++col) {
            const int c0 = col % q, c1 = (col / q) % q, c2 = col / (q * q);
            const int64_t n0 = (n - c0 + q - 1) / q, n1 = (n - c1 + q - 1) / q;
            const int64_t n2 = (dim == 3) ? (n - c2 + q - 1) / q : 1;
            const int64_t cnt = n0 * n1 * n2;
#pragma omp parallel
            {
                TensorEval te{dim, p, nloc, &B};
                std::vector<double> val(nloc), grad((size_t)dim * nloc), bl(nloc);
                Rule R;
#pragma omp for schedule(static)
                for (int64_t k = 0; k < cnt; ++k) {
                    int e[3] = {c0 + q * (int)(k % n0), c1 + q * (int)((k / n0) % n1),
                                dim == 3 ? c2 + q * (int)(k / (n0 * n1)) : 0};
                    const int64_t E = flat(e, n);
                    if (!lv.elem_active[E]) continue;
                    const double* src;
                    if (lv.elem_full[E]) {
                        double lo[3], hi[3];
                        for (int kk = 0; kk < dim; ++kk) {
                            lo[kk] = pb.lo + e[kk] * B.h;
                            hi[kk] = lo[kk] + B.h;
                        }
                        R.vp.clear();
                        R.vw.clear();
                        box_rule(lo, hi, dim, q, g1, w1, R);
                        std::fill(bl.begin(), bl.end(), 0.0);
                        for (size_t t = 0; t < R.vw.size(); ++t) {
                            te(e, &R.vp[t * dim], val.data(), grad.data());
                            const double fw = R.vw[t] * f_rhs(&R.vp[t * dim], dim);
                            for (int a = 0; a < nloc; ++a) bl[a] += val[a] * fw;
                        }
                        src = bl.data();
                    } else {
                        src = ce[cut_id[E]].b.data();
                    }
                    for (int a = 0; a < nloc; ++a) {
                        int c[3] = {a % q, (a / q) % q, a / (q * q)};
                        int j[3] = {e[0] + c[0], e[1] + c[1], dim == 3 ? e[2] + c[2] : 0};
                        H.b[flat(j, lv.m)] += src[a];
                    }
                }
            }
        }
        for (int64_t r = 0; r < lv.N; ++r)
            if (!lv.active[r]) H.b[r] = 0.0;
        phase("right-hand side");
        (void)err;
        return true;
    }

    // restriction tables of level index li (fine) to li-1 (coarse)
    void build_transfer(int li) {
        LevelData& f = H.lv[li];
        const Basis1D& bc = basis[li - 1];
        const Basis1D& bf = basis[li];
        std::vector<double> R1 = two_scale(bc, bf);
        const int mc = bc.m, mf = bf.m, P2 = p + 2;
        f.r_first.assign(mc, 0);
        f.r_w.assign((size_t)mc * P2, 0.0);
        for (int i = 0; i < mc; ++i) {
            int first = -1, last = -1;
            for (int a = 0; a < mf; ++a)
                if (R1[(size_t)i * mf + a] != 0.0) {
                    if (first < 0) first = a;
                    last = a;
                }
            if (last - first + 1 > P2) throw std::runtime_error("two-scale row wider than p+2");
            first = std::min(first, mf - P2);
            f.r_first[i] = first;
            for (int k = 0; k < P2; ++k) f.r_w[(size_t)i * P2 + k] = R1[(size_t)i * mf + first + k];
        }
        int TW = 0;
        std::vector<int> tf(mf), tl(mf);
        for (int a = 0; a < mf; ++a) {
            int first = -1, last = -1;
            for (int i = 0; i < mc; ++i)
                if (R1[(size_t)i * mf + a] != 0.0) {
                    if (first < 0) first = i;
                    last = i;
                }
            tf[a] = first;
            tl[a] = last;
            TW = std::max(TW, last - first + 1);
        }
        f.TW = TW;
        f.t_first.assign(mf, 0);
        f.t_w.assign((size_t)mf * TW, 0.0);
        for (int a = 0; a < mf; ++a) {
            int first = std::min(tf[a], mc - TW);
            f.t_first[a] = first;
            for (int k = 0; k < TW; ++k) f.t_w[(size_t)a * TW + k] = R1[(size_t)(first + k) * mf + a];
        }
    }

    // coarse level li from fine level li+1: element status, rows, Galerkin stored rows
    void build_coarse(int li) {
        LevelData& c = H.lv[li];
        const LevelData& f = H.lv[li + 1];
        const int nc = c.n, nf = f.n;
        const int64_t NE = pw(nc, dim);
        c.elem_active.assign(NE, 0);
        c.elem_full.assign(NE, 1);
        for (int64_t E = 0; E < NE; ++E) {
            int e[3];
            unflat(E, nc, e);
            for (int ch = 0; ch < (1 << dim); ++ch) {
                int fe[3] = {2 * e[0] + (ch & 1), 2 * e[1] + ((ch >> 1) & 1), dim == 3 ? 2 * e[2] + ((ch >> 2) & 1) : 0};
                int64_t F = flat(fe, nf);
                c.elem_active[E] |= f.elem_active[F];
                c.elem_full[E] &= f.elem_full[F];
            }
        }
        classify_rows(c);
        build_1d_tables(c, li);
        // Galerkin stored rows: A_c[i][j] = sum_a sum_b R[i][a] A_f[a][b] R[j][b] over active a, b
        const int P2 = p + 2, TW = f.TW;
        const int64_t nb = (int64_t)c.band_rows.size();
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t bi = 0; bi < nb; ++bi) {
            const int64_t r = c.band_rows[bi];
            int i[3];
            unflat(r, c.m, i);
            std::vector<double> row(ncoef, 0.0), frow(ncoef);
            int na[3] = {P2, P2, dim == 3 ? P2 : 1};
            for (int kz = 0; kz < na[2]; ++kz)
                for (int ky = 0; ky < na[1]; ++ky)
                    for (int kx = 0; kx < na[0]; ++kx) {
                        int a[3] = {f.r_first[i[0]] + kx, f.r_first[i[1]] + ky, dim == 3 ? f.r_first[i[2]] + kz : 0};
                        double wa = f.r_w[(size_t)i[0] * P2 + kx] * f.r_w[(size_t)i[1] * P2 + ky] *
                                    (dim == 3 ? f.r_w[(size_t)i[2] * P2 + kz] : 1.0);
                        if (wa == 0.0) continue;
                        int64_t af = flat(a, f.m);
                        if (!f.active[af]) continue;
                        row_coeffs(f, af, frow.data());
                        for (int cf = 0; cf < ncoef; ++cf) {
                            if (frow[cf] == 0.0) continue;
                            int o[3] = {cf % W - p, (cf / W) % W - p, dim == 3 ? cf / (W * W) - p : 0};
                            int b[3] = {a[0] + o[0], a[1] + o[1], a[2] + o[2]};
                            double wab = wa * frow[cf];
                            // coarse parents j of b
                            int nt[3] = {TW, TW, dim == 3 ? TW : 1};
                            for (int tz = 0; tz < nt[2]; ++tz)
                                for (int ty = 0; ty < nt[1]; ++ty)
                                    for (int tx = 0; tx < nt[0]; ++tx) {
                                        int j[3] = {f.t_first[b[0]] + tx, f.t_first[b[1]] + ty,
                                                    dim == 3 ? f.t_first[b[2]] + tz : 0};
                                        double wb = f.t_w[(size_t)b[0] * TW + tx] * f.t_w[(size_t)b[1] * TW + ty] *
                                                    (dim == 3 ? f.t_w[(size_t)b[2] * TW + tz] : 1.0);
                                        if (wb == 0.0) continue;
                                        int oc[3] = {j[0] - i[0], j[1] - i[1], j[2] - i[2]};
                                        bool in = true;
                                        for (int k = 0; k < dim; ++k) in = in && oc[k] >= -p && oc[k] <= p;
                                        if (!in) continue;          // cannot happen for nested B-splines
                                        if (!c.active[flat(j, c.m)]) continue;
                                        row[coef_index(oc)] += wab * wb;
                                    }
                        }
                    }
            for (int cc = 0; cc < ncoef; ++cc) c.band_coef[(size_t)cc * nb + bi] = row[cc];
        }
    }

    // Schwarz blocks of a level (encapsulating supports), pruned and inverted
    bool build_blocks(int li, std::string& err) {
        LevelData& lv = H.lv[li];
        const int64_t N = lv.N, m = lv.m;
        const int n = lv.n;
        lv.dinv.assign(N, 0.0);
        std::vector<int64_t> rows;
        for (int64_t r = 0; r < N; ++r)
            if (lv.active[r]) rows.push_back(r);
        const int64_t nr = (int64_t)rows.size();
        std::vector<std::vector<int32_t>> bidx(nr);
        std::vector<std::vector<double>> binv(nr);
        std::vector<int> nprune(nr, 0);
        int fail = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : fail)
        for (int64_t t = 0; t < nr; ++t) {
            const int64_t r = rows[t];
            int j[3];
            unflat(r, m, j);
            std::vector<int64_t> blk;
            int lo3[3] = {0, 0, 0}, hi3[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k) {
                lo3[k] = std::max(0, j[k] - p);
                hi3[k] = std::min((int)m - 1, j[k] + p);
            }
            for (int kz = lo3[2]; kz <= hi3[2]; ++kz)
                for (int ky = lo3[1]; ky <= hi3[1]; ++ky)
                    for (int kx = lo3[0]; kx <= hi3[0]; ++kx) {
                        int k3[3] = {kx, ky, kz};
                        int64_t kf = flat(k3, m);
                        if (!lv.active[kf]) continue;
                        bool inside = true;
                        int elo[3] = {0, 0, 0}, ehi[3] = {0, 0, 0};
                        for (int d = 0; d < dim; ++d) {
                            elo[d] = std::max(0, k3[d] - p);
                            ehi[d] = std::min(n - 1, k3[d]);
                        }
                        for (int ez = elo[2]; ez <= ehi[2] && inside; ++ez)
                            for (int ey = elo[1]; ey <= ehi[1] && inside; ++ey)
                                for (int ex = elo[0]; ex <= ehi[0] && inside; ++ex) {
                                    int e[3] = {ex, ey, ez};
                                    if (!lv.elem_active[flat(e, n)]) continue;
                                    for (int d = 0; d < dim; ++d)
                                        if (e[d] < j[d] - p || e[d] > j[d]) inside = false;
                                }
                        if (inside) blk.push_back(kf);
                    }
            const int nj = (int)blk.size();
            std::vector<double> A((size_t)nj * nj, 0.0), row(ncoef);
            for (int a = 0; a < nj; ++a) {
                row_coeffs(lv, blk[a], row.data());
                int ia[3];
                unflat(blk[a], m, ia);
                for (int c = 0; c < nj; ++c) {
                    int ic[3];
                    unflat(blk[c], m, ic);
                    int o[3] = {ic[0] - ia[0], ic[1] - ia[1], ic[2] - ia[2]};
                    bool near = true;       // two members of a block can lie up to 2p apart
                    for (int d = 0; d < dim; ++d) near = near && o[d] >= -p && o[d] <= p;
                    A[(size_t)a * nj + c] = near ? row[coef_index(o)] : 0.0;
                }
            }
            std::vector<int> keep;
            std::vector<double> inv;
            int removed = prune_and_invert(A, nj, keep, inv);
            if (removed < 0) {
                ++fail;
                continue;
            }
            nprune[t] = removed;
            for (int k : keep) bidx[t].push_back((int32_t)blk[k]);
            binv[t] = inv;
        }
        if (fail) {
            err = "a Schwarz block is not positive definite after the Remark 3.3 rule";
            return false;
        }
        lv.blk_ptr.assign(1, 0);
        lv.blk_vptr.assign(1, 0);
        lv.blk_idx.clear();
        lv.blk_val.clear();
        lv.pruned = 0;
        lv.max_block = 1;
        // block order: by owner (additive), or by the owner's colour and then by owner
        // (multiplicative): colour = sum_k (j_k mod (p+1)) (p+1)^k, so that functions of
        // equal colour have disjoint supports (Sec. 3.4)
        std::vector<int64_t> order(nr);
        std::iota(order.begin(), order.end(), 0);
        std::vector<int> colour(nr, 0);
        const int ncol = (dim == 2) ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1);
        for (int64_t t = 0; t < nr; ++t) {
            int j[3];
            unflat(rows[t], m, j);
            colour[t] = (j[0] % (p + 1)) + (p + 1) * ((j[1] % (p + 1)) + (dim == 3 ? (p + 1) * (j[2] % (p + 1)) : 0));
        }
        const bool mult = pb.smoother == 1;
        if (mult) std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return colour[a] < colour[b]; });
        lv.ncolour = mult ? ncol : 0;
        lv.blk_cptr.assign(mult ? ncol + 1 : 0, 0);
        lv.sg_cptr.assign(mult ? ncol + 1 : 0, 0);
        lv.sg_row.clear();
        lv.sg_inv.clear();
        for (int64_t ot = 0; ot < nr; ++ot) {
            const int64_t t = order[ot];
            lv.pruned += nprune[t];
            const int nj = (int)bidx[t].size();
            if (nj == 1) {
                lv.dinv[bidx[t][0]] += binv[t][0];
                if (mult) {
                    lv.sg_row.push_back(bidx[t][0]);
                    lv.sg_inv.push_back(binv[t][0]);
                    lv.sg_cptr[colour[t] + 1] = (int64_t)lv.sg_row.size();
                }
                continue;
            }
            lv.max_block = std::max<int64_t>(lv.max_block, nj);
            for (int a = 0; a < nj; ++a) lv.blk_idx.push_back(bidx[t][a]);
            // column-major: value (row a, col c) at c*nj + a (the inverse is symmetric)
            for (int c = 0; c < nj; ++c)
                for (int a = 0; a < nj; ++a) lv.blk_val.push_back(binv[t][(size_t)a * nj + c]);
            lv.blk_ptr.push_back((int64_t)lv.blk_idx.size());
            lv.blk_vptr.push_back((int64_t)lv.blk_val.size());
            if (mult) lv.blk_cptr[colour[t] + 1] = (int64_t)lv.blk_ptr.size() - 1;
        }
        // colours without blocks of one kind: ranges start where the previous one ends
        for (int c = 1; c <= (mult ? ncol : 0); ++c) {
            lv.blk_cptr[c] = std::max(lv.blk_cptr[c], lv.blk_cptr[c - 1]);
            lv.sg_cptr[c] = std::max(lv.sg_cptr[c], lv.sg_cptr[c - 1]);
        }
        return true;
    }

    bool build_coarse_solve(std::string& err) {
        const LevelData& c = H.lv[0];
        std::vector<int64_t> rows;
        for (int64_t r = 0; r < c.N; ++r)
            if (c.active[r]) rows.push_back(r);
        const int nr = (int)rows.size();
        if (nr > MAX_COARSE_ROWS) {
            err = "the coarsest level has " + std::to_string(nr) + " active functions; its dense inverse allows at most " +
                  std::to_string(MAX_COARSE_ROWS) + " (use more levels)";
            return false;
        }
        std::vector<int64_t> pos(c.N, -1);
        for (int a = 0; a < nr; ++a) pos[rows[a]] = a;
        std::vector<double> A((size_t)nr * nr, 0.0), row(ncoef);
        for (int a = 0; a < nr; ++a) {
            row_coeffs(c, rows[a], row.data());
            int i[3];
            unflat(rows[a], c.m, i);
            for (int cc = 0; cc < ncoef; ++cc) {
                if (row[cc] == 0.0) continue;
                int o[3] = {cc % W - p, (cc / W) % W - p, dim == 3 ? cc / (W * W) - p : 0};
                int j[3] = {i[0] + o[0], i[1] + o[1], i[2] + o[2]};
                A[(size_t)a * nr + pos[flat(j, c.m)]] = row[cc];
            }
        }
        std::vector<int> keep;
        std::vector<double> inv;
        int removed = prune_and_invert(A, nr, keep, inv);
        if (removed < 0) {
            err = "the coarsest-level matrix is not positive definite after the Remark 3.3 rule";
            return false;
        }
        H.coarse_pruned = removed;
        H.c_rows.clear();
        for (int k : keep) H.c_rows.push_back((int32_t)rows[k]);
        H.c_inv = inv;
        return true;
    }

    // FP32 copies of every level in Jacobi-scaled variables (mixed-precision V-cycle)
    void build_fp32() {
        for (int li = 0; li < L; ++li) {
            LevelData& lv = H.lv[li];
            const int64_t N = lv.N, m = lv.m, nb = (int64_t)lv.band_rows.size();
            std::vector<double> dg(N, 0.0), row(ncoef);
            for (int64_t r = 0; r < N; ++r) {
                if (!lv.active[r]) continue;
                row_coeffs(lv, r, row.data());
                dg[r] = std::sqrt(row[ncoef / 2]);
            }
            lv.f_d.assign(N, 0.0f);
            lv.f_s.assign(N, 0.0f);
            for (int64_t r = 0; r < N; ++r)
                if (dg[r] > 0.0) {
                    lv.f_d[r] = (float)dg[r];
                    lv.f_s[r] = (float)(1.0 / dg[r]);
                }
            lv.f_band_coef.assign(lv.band_coef.size(), 0.0f);
            for (int64_t bi = 0; bi < nb; ++bi) {
                const int64_t r = lv.band_rows[bi];
                int i[3];
                unflat(r, m, i);
                for (int c = 0; c < ncoef; ++c) {
                    const double v = lv.band_coef[(size_t)c * nb + bi];
                    if (v == 0.0) continue;
                    int o[3] = {c % W - p, (c / W) % W - p, dim == 3 ? c / (W * W) - p : 0};
                    int j[3] = {i[0] + o[0], i[1] + o[1], i[2] + o[2]};
                    const int64_t jf = flat(j, m);
                    if (dg[r] > 0.0 && dg[jf] > 0.0) lv.f_band_coef[(size_t)c * nb + bi] = (float)(v / (dg[r] * dg[jf]));
                }
            }
            lv.f_K1.assign(lv.K1.begin(), lv.K1.end());
            lv.f_M1.assign(lv.M1.begin(), lv.M1.end());
            lv.f_r_w.assign(lv.r_w.begin(), lv.r_w.end());
            lv.f_t_w.assign(lv.t_w.begin(), lv.t_w.end());
            lv.f_dinv.assign(N, 0.0f);
            for (int64_t r = 0; r < (int64_t)lv.dinv.size(); ++r) lv.f_dinv[r] = (float)(lv.dinv[r] * dg[r] * dg[r]);
            lv.f_blk_val.assign(lv.blk_val.size(), 0.0f);
            const int64_t nblk = lv.blk_ptr.empty() ? 0 : (int64_t)lv.blk_ptr.size() - 1;
            for (int64_t b = 0; b < nblk; ++b) {
                const int64_t s0 = lv.blk_ptr[b], nj = lv.blk_ptr[b + 1] - s0, v0 = lv.blk_vptr[b];
                for (int64_t c = 0; c < nj; ++c)
                    for (int64_t a = 0; a < nj; ++a)
                        lv.f_blk_val[v0 + c * nj + a] =
                            (float)(lv.blk_val[v0 + c * nj + a] * dg[lv.blk_idx[s0 + a]] * dg[lv.blk_idx[s0 + c]]);
            }
            lv.f_sg_inv.resize(lv.sg_inv.size());
            for (size_t k = 0; k < lv.sg_inv.size(); ++k)
                lv.f_sg_inv[k] = (float)(lv.sg_inv[k] * dg[lv.sg_row[k]] * dg[lv.sg_row[k]]);
            if (li == 0) {
                const size_t nc = H.c_rows.size();
                H.f_c_inv.assign(nc * nc, 0.0f);
                for (size_t a = 0; a < nc; ++a)
                    for (size_t c = 0; c < nc; ++c)
                        H.f_c_inv[a * nc + c] = (float)(H.c_inv[a * nc + c] * dg[H.c_rows[a]] * dg[H.c_rows[c]]);
            }
        }
    }

    bool run(std::string& err) {
        basis.resize(L);
        Ke.resize(L);
        Me.resize(L);
        H.lv.assign(L, LevelData());
        for (int li = 0; li < L; ++li) {
            int nl = pb.n >> (L - 1 - li);
            basis[li] = Basis1D(nl, p, pb.lo, pb.hi);
            element_matrices_1d(basis[li], Ke[li], Me[li]);
            LevelData& lv = H.lv[li];
            lv.n = nl;
            lv.m = basis[li].m;
            lv.h = basis[li].h;
            lv.N = pw(lv.m, dim);
        }
        const bool verbose = std::getenv("IMGM_VERBOSE") != nullptr;
        auto t = std::chrono::steady_clock::now();
        auto phase = [&](const char* name) {
            const auto now = std::chrono::steady_clock::now();
            if (verbose) std::fprintf(stderr, "imgm: setup %-22s %8.3f s\n", name, std::chrono::duration<double>(now - t).count());
            t = now;
        };
        if (!build_finest(err)) return false;
        phase("finest level");
        for (int li = L - 1; li >= 1; --li) {
            build_transfer(li);
            build_coarse(li - 1);
        }
        phase("Galerkin levels");
        if (!build_coarse_solve(err)) return false;
        phase("coarsest solve");
        for (int li = L - 1; li >= 1; --li)
            if (!build_blocks(li, err)) return false;
        phase("Schwarz blocks");
        if (pb.precision >= 1) build_fp32();
        phase("FP32 copies");
        return true;
    }
};

}  // namespace

bool build_hierarchy(const Problem& pb, Hierarchy& H, std::string& err) {
    auto t0 = std::chrono::steady_clock::now();
    if (pb.dim != 2 && pb.dim != 3) { err = "dim must be 2 or 3"; return false; }
    if (pb.p < 1 || pb.p > 3) { err = "degree must be 1, 2 or 3"; return false; }
    if (pb.basis == 1 && pb.p != 1) { err = "Lagrange bases are implemented for degree 1 only"; return false; }
    if (pb.basis != 0 && pb.basis != 1) { err = "basis must be 0 (B-spline) or 1 (Lagrange)"; return false; }
    if (pb.levels < 2) { err = "levels must be >= 2"; return false; }
    if (pb.n <= 0 || pb.n % (1 << (pb.levels - 1)) != 0) { err = "n must be a positive multiple of 2^(levels-1)"; return false; }
    if ((pb.n >> (pb.levels - 1)) < 1) { err = "too many levels"; return false; }
    if (pb.depth < 0 || pb.depth > 6) { err = "depth must be in 0..6"; return false; }
    if (pb.bc != 0 && pb.bc != 1) { err = "bc must be 0 (penalty) or 1 (Nitsche)"; return false; }
    if (!(pb.hi > pb.lo)) { err = "hi must exceed lo"; return false; }
    if (pb.precision < 0 || pb.precision > 2) {
        err = "precision must be 0 (FP64), 1 (FP32 V-cycle) or 2 (FP64 finest level, FP32 below)";
        return false;
    }
    if (pb.precision == 2 && pb.smoother != 0) { err = "precision 2 is built for the additive smoother only"; return false; }
    if (pb.smoother != 0 && pb.smoother != 1) { err = "smoother must be 0 (additive) or 1 (multiplicative)"; return false; }
    double Nd = std::pow((double)(pb.n + pb.p), pb.dim);
    if (Nd > 2.0e9) { err = "grid too large for 32-bit row indices"; return false; }
    H = Hierarchy();
    H.dim = pb.dim;
    H.p = pb.p;
    H.L = pb.levels;
    H.bc = pb.bc;
    H.smoother = pb.smoother;
    const int W = 2 * pb.p + 1;
    H.ncoef = (pb.dim == 2) ? W * W : W * W * W;
    H.gamma = pb.gamma > 0 ? pb.gamma : 1.0 / std::pow((double)(pb.p + 1), pb.dim);
    try {
        Builder B(pb, H);
        if (!B.run(err)) return false;
    } catch (const std::exception& e) {
        err = e.what();
        return false;
    }
    H.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return true;
}

}  // namespace imgm
