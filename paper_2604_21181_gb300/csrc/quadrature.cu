// Quadrature tables of the library, derived on the host at run time.
//
// * Symmetric triangle rules (Sec. 5.1: the 12-point rule of degree 6 of
//   Witherden & Vincent; the 6-point rule of degree 4 for the small-sphere
//   workload) are obtained by solving their moment equations -- exactness on
//   every monomial xi^a eta^b up to the degree -- with Gauss-Newton from
//   rough starting orbits.
// * Gauss-Legendre nodes and weights for the Sauter-Schwab tensor rules
//   (Sec. 4.2) come from the eigen-decomposition of the Legendre Jacobi
//   matrix (Golub-Welsch), by implicit QL iterations.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace mu {
namespace {

double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// exact integral of xi^a eta^b over the reference simplex
double simplex_moment(int a, int b) { return factorial(a) * factorial(b) / factorial(a + b + 2); }

struct OrbitSpec {
  int n3;   // number of (a, b, b) orbits
  int n6;   // number of (a, b, c) orbits
};

// parameters: per 3-orbit (a, w), per 6-orbit (a, b, w); weights normalised to
// sum 1 and multiplied by 1/2 when the points are produced
void expand(const OrbitSpec& sp, const std::vector<double>& th, std::vector<double>& xi,
            std::vector<double>& eta, std::vector<double>& w) {
  xi.clear();
  eta.clear();
  w.clear();
  int k = 0;
  for (int o = 0; o < sp.n3; ++o) {
    double a = th[k++], wt = th[k++];
    double b = 0.5 * (1.0 - a);
    const double bar[3][3] = {{a, b, b}, {b, a, b}, {b, b, a}};
    for (int i = 0; i < 3; ++i) {
      xi.push_back(bar[i][1]);
      eta.push_back(bar[i][2]);
      w.push_back(0.5 * wt);
    }
  }
  for (int o = 0; o < sp.n6; ++o) {
    double a = th[k++], b = th[k++], wt = th[k++];
    double c = 1.0 - a - b;
    const double bar[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
    for (int i = 0; i < 6; ++i) {
      xi.push_back(bar[i][1]);
      eta.push_back(bar[i][2]);
      w.push_back(0.5 * wt);
    }
  }
}

void residual(const OrbitSpec& sp, int deg, const std::vector<double>& th,
              std::vector<double>& r) {
  std::vector<double> xi, eta, w;
  expand(sp, th, xi, eta, w);
  r.clear();
  for (int a = 0; a <= deg; ++a)
    for (int b = 0; a + b <= deg; ++b) {
      double s = 0.0;
      for (size_t i = 0; i < w.size(); ++i) s += w[i] * pow(xi[i], a) * pow(eta[i], b);
      r.push_back(s - simplex_moment(a, b));
    }
}

// small dense solve (Gaussian elimination with partial pivoting)
bool dense_solve(int n, std::vector<double> A, std::vector<double>& b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
    b[i] = s / A[i * n + i];
  }
  return true;
}

bool solve_moments(const OrbitSpec& sp, int deg, std::vector<double>& th) {
  const int np = (int)th.size();
  std::vector<double> r, rp, rm;
  for (int it = 0; it < 60; ++it) {
    residual(sp, deg, th, r);
    double rn = 0.0;
    for (double v : r) rn = std::max(rn, fabs(v));
    if (rn < 1e-17) return true;
    const int m = (int)r.size();
    std::vector<double> J((size_t)m * np);
    for (int j = 0; j < np; ++j) {
      std::vector<double> tp = th, tm = th;
      double h = 1e-7 * std::max(1.0, fabs(th[j]));
      tp[j] += h;
      tm[j] -= h;
      residual(sp, deg, tp, rp);
      residual(sp, deg, tm, rm);
      for (int i = 0; i < m; ++i) J[(size_t)i * np + j] = (rp[i] - rm[i]) / (2 * h);
    }
    std::vector<double> A((size_t)np * np, 0.0), g(np, 0.0);
    for (int a = 0; a < np; ++a) {
      for (int b = 0; b < np; ++b) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += J[(size_t)i * np + a] * J[(size_t)i * np + b];
        A[a * np + b] = s;
      }
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += J[(size_t)i * np + a] * r[i];
      g[a] = -s;
    }
    if (!dense_solve(np, A, g)) return false;
    double step = 0.0;
    for (int j = 0; j < np; ++j) {
      th[j] += g[j];
      step = std::max(step, fabs(g[j]));
    }
    if (step < 1e-16) {
      residual(sp, deg, th, r);
      double rn2 = 0.0;
      for (double v : r) rn2 = std::max(rn2, fabs(v));
      return rn2 < 1e-14;
    }
  }
  residual(sp, deg, th, r);
  double rn = 0.0;
  for (double v : r) rn = std::max(rn, fabs(v));
  return rn < 1e-14;
}

}  // namespace

bool triangle_rule(int q, TriangleRule& out) {
  OrbitSpec sp;
  std::vector<double> th;
  int deg;
  if (q == 6) {
    sp = {2, 0};
    th = {0.11, 0.22, 0.82, 0.11};
    deg = 4;
  } else if (q == 12) {
    sp = {2, 1};
    th = {0.50, 0.12, 0.87, 0.05, 0.05, 0.31, 0.08};
    deg = 6;
  } else {
    return false;
  }
  if (!solve_moments(sp, deg, th)) return false;
  out.q = q;
  expand(sp, th, out.xi, out.eta, out.w);
  return (int)out.w.size() == q;
}

// Golub-Welsch: eigenvalues of the symmetric tridiagonal Jacobi matrix of
// the Legendre polynomials (zero diagonal, off-diagonal k / sqrt(4k^2 - 1))
// are the nodes on [-1, 1]; the weights are 2 * (first eigenvector
// component)^2.  Implicit QL with Wilkinson-type shifts.
void gauss_legendre_unit(int n, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> d(n, 0.0), e(n, 0.0), Z((size_t)n * n, 0.0);
  for (int k = 1; k < n; ++k) e[k - 1] = k / sqrt(4.0 * k * k - 1.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0; iter < 200; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= 1e-300 + 2.2e-16 * dd) break;
      }
      if (m == l) break;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? fabs(r) : -fabs(r)));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      for (; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        for (int k = 0; k < n; ++k) {
          double zf = Z[(size_t)k * n + i + 1];
          Z[(size_t)k * n + i + 1] = s * Z[(size_t)k * n + i] + c * zf;
          Z[(size_t)k * n + i] = c * Z[(size_t)k * n + i] - s * zf;
        }
      }
      if (r == 0.0 && i >= l) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    int i = idx[k];
    double t = d[i];
    double v0 = Z[i];  // first component of eigenvector i
    x[k] = 0.5 * (t + 1.0);
    w[k] = v0 * v0;  // 2 v0^2 on [-1,1], halved on [0,1]
  }
}

}  // namespace mu
