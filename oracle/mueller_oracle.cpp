// ============================================================================
// ORACLE -- test infrastructure only.
//
// Plain, slow, obviously-correct FP64 implementation of the nodal P2 Mueller
// boundary-integral method (Luo, "A High-Order Nodal Galerkin Formulation for
// the Mueller Equation", arXiv 2604.21181).  It exists to check the CUDA
// library; only the tests, the smoke check and the CPU-baseline leg of the
// benchmark may load it.  It shares no source with the CUDA library: its own
// quadrature tables, geometry, kernels, Sauter-Schwab maps, LU and GMRES.
//
// Every function cites the part of the paper it follows ("Sec.", "Eq.").
// Readings of passages the paper leaves open are marked READING.
// ============================================================================
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cd;
static const double PI = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------- 3-vectors
struct V3 {
  double x, y, z;
};
static inline V3 v3(double a, double b, double c) { return V3{a, b, c}; }
static inline V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
static inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
static inline V3 unit(V3 a) { return (1.0 / norm(a)) * a; }

// complex 3-vectors for currents
struct C3 {
  cd x, y, z;
};
static inline C3 c3zero() { return C3{0.0, 0.0, 0.0}; }
static inline C3 operator+(C3 a, C3 b) { return C3{a.x + b.x, a.y + b.y, a.z + b.z}; }
static inline C3 cscale(cd s, V3 a) { return C3{s * a.x, s * a.y, s * a.z}; }
static inline C3 cscale(cd s, C3 a) { return C3{s * a.x, s * a.y, s * a.z}; }
static inline cd cdotr(V3 a, C3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline C3 ccross(V3 a, C3 b) {
  return C3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ======================================================= quadrature rules
// Triangle rules on the reference simplex {xi, eta >= 0, xi + eta <= 1}; the
// weights sum to 1/2 (the simplex area).
//   q = 6 : symmetric 6-point rule of degree 4 (Dunavant 1985, p = 4)
//   q = 12: symmetric 12-point rule of degree 6, the rule Sec. 5.1 names
//           (Witherden & Vincent 2015; the same points as Dunavant p = 6).
// READING: the 6-point rule stands for the "6-point Gauss" of the small-sphere
// workload.
struct TriRule {
  std::vector<double> xi, eta, w;
};

static void push_s21(TriRule& r, double a, double wt) {
  // barycentric orbit (a, b, b), b = (1 - a)/2
  double b = 0.5 * (1.0 - a);
  double l[3][3] = {{a, b, b}, {b, a, b}, {b, b, a}};
  for (int k = 0; k < 3; ++k) {
    r.xi.push_back(l[k][1]);
    r.eta.push_back(l[k][2]);
    r.w.push_back(0.5 * wt);
  }
}
static void push_s111(TriRule& r, double a, double b, double wt) {
  double c = 1.0 - a - b;
  double l[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
  for (int k = 0; k < 6; ++k) {
    r.xi.push_back(l[k][1]);
    r.eta.push_back(l[k][2]);
    r.w.push_back(0.5 * wt);
  }
}

static bool tri_rule(int q, TriRule& r) {
  r.xi.clear();
  r.eta.clear();
  r.w.clear();
  if (q == 6) {
    push_s21(r, 0.108103018168070, 0.223381589678011);
    push_s21(r, 0.816847572980459, 0.109951743655322);
    return true;
  }
  if (q == 12) {
    push_s21(r, 0.501426509658179, 0.116786275726379);
    push_s21(r, 0.873821971016996, 0.050844906370207);
    push_s111(r, 0.053145049844817, 0.310352451033784, 0.082851075618374);
    return true;
  }
  return false;
}

// Gauss-Legendre on [0, 1] by Newton iteration on P_n (three-term recurrence).
static void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
    }
    // map [-1,1] -> [0,1]
    x[n - 1 - i] = 0.5 * (t + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
}

// ================================================================ Morton
// Sec. 5 (double Morton permutation).  READING: bounding box of the nodes,
// scaled by its largest extent, 21 bits per axis, x in the least significant
// bit; stable sort by (key, original index).  Elements are keyed by the
// centroid of their three corner vertices in the same box.
static uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}
static uint64_t morton_key(const double* p, const double* lo, double ext) {
  uint64_t q[3];
  for (int a = 0; a < 3; ++a) {
    double s = (p[a] - lo[a]) / ext * 2097152.0;  // 2^21
    if (!(s > 0.0)) s = 0.0;
    if (s > 2097151.0) s = 2097151.0;
    q[a] = (uint64_t)std::floor(s);
  }
  return spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
}

static void morton_perms(const double* xyz, int64_t nn, const int32_t* tri6, int64_t nt,
                         std::vector<int32_t>& node_perm, std::vector<int32_t>& elem_perm) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < nn; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], xyz[3 * i + a]);
      hi[a] = std::max(hi[a], xyz[3 * i + a]);
    }
  double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  if (!(ext > 0.0)) ext = 1.0;
  std::vector<uint64_t> key(nn);
  for (int64_t i = 0; i < nn; ++i) key[i] = morton_key(xyz + 3 * i, lo, ext);
  node_perm.resize(nn);
  std::iota(node_perm.begin(), node_perm.end(), 0);
  std::stable_sort(node_perm.begin(), node_perm.end(),
                   [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  std::vector<uint64_t> ek(nt);
  for (int64_t e = 0; e < nt; ++e) {
    double c[3];
    for (int a = 0; a < 3; ++a)
      c[a] = (xyz[3 * tri6[6 * e + 0] + a] + xyz[3 * tri6[6 * e + 1] + a] +
              xyz[3 * tri6[6 * e + 2] + a]) / 3.0;
    ek[e] = morton_key(c, lo, ext);
  }
  elem_perm.resize(nt);
  std::iota(elem_perm.begin(), elem_perm.end(), 0);
  std::stable_sort(elem_perm.begin(), elem_perm.end(),
                   [&](int32_t a, int32_t b) { return ek[a] < ek[b]; });
}

// ================================================================ P2 element
// Sec. 3.3 / 4: six-node isoparametric triangle; nodes v0 (0,0), v1 (1,0),
// v2 (0,1), m01 (1/2,0), m12 (1/2,1/2), m20 (0,1/2); standard quadratic
// Lagrange functions in barycentrics l0 = 1-xi-eta, l1 = xi, l2 = eta.
static void p2_shape(double xi, double eta, double N[6], double dxi[6], double deta[6]) {
  double l0 = 1.0 - xi - eta, l1 = xi, l2 = eta;
  N[0] = l0 * (2.0 * l0 - 1.0);
  N[1] = l1 * (2.0 * l1 - 1.0);
  N[2] = l2 * (2.0 * l2 - 1.0);
  N[3] = 4.0 * l0 * l1;
  N[4] = 4.0 * l1 * l2;
  N[5] = 4.0 * l2 * l0;
  dxi[0] = -(4.0 * l0 - 1.0);
  dxi[1] = 4.0 * l1 - 1.0;
  dxi[2] = 0.0;
  dxi[3] = 4.0 * (l0 - l1);
  dxi[4] = 4.0 * l2;
  dxi[5] = -4.0 * l2;
  deta[0] = -(4.0 * l0 - 1.0);
  deta[1] = 0.0;
  deta[2] = 4.0 * l2 - 1.0;
  deta[3] = -4.0 * l1;
  deta[4] = 4.0 * l1;
  deta[5] = 4.0 * (l0 - l2);
}

// ================================================================ the mesh
struct Mesh {
  int64_t nn = 0, nt = 0;
  std::vector<V3> X;             // nodes (Morton order)
  std::vector<int32_t> T;        // [nt][6] (Morton order of elements)
  std::vector<int32_t> node_perm, elem_perm;
  std::vector<V3> n, t1, t2;     // nodal frame (Sec. 3.1-3.2)
  int status = 0;
  double min_gs = 1e300;         // smallest Gram-Schmidt norm seen (diagnostic)
};

struct Geo {  // geometry and frame at one parametric point of an element
  V3 x, a1, a2, n;
  double J;
  V3 t[2], s[2];
  double N[6];
  double gs_min;
};

// Sec. 3.3: position, covariant vectors, exact normal, interpolated nodal
// frame projected on the tangent plane and Gram-Schmidt orthonormalised; the
// rotated test vectors s_alpha = t_alpha x n (Sec. 4.1).
static Geo geo_at(const Mesh& m, int64_t e, double xi, double eta) {
  Geo g;
  double dxi[6], deta[6];
  p2_shape(xi, eta, g.N, dxi, deta);
  g.x = v3(0, 0, 0);
  g.a1 = v3(0, 0, 0);
  g.a2 = v3(0, 0, 0);
  V3 tt1 = v3(0, 0, 0), tt2 = v3(0, 0, 0);
  for (int k = 0; k < 6; ++k) {
    int32_t nd = m.T[6 * e + k];
    g.x = g.x + g.N[k] * m.X[nd];
    g.a1 = g.a1 + dxi[k] * m.X[nd];
    g.a2 = g.a2 + deta[k] * m.X[nd];
    tt1 = tt1 + g.N[k] * m.t1[nd];
    tt2 = tt2 + g.N[k] * m.t2[nd];
  }
  V3 c = cross(g.a1, g.a2);
  g.J = norm(c);
  g.n = (1.0 / g.J) * c;
  V3 p1 = tt1 - dot(g.n, tt1) * g.n;
  double n1 = norm(p1);
  g.t[0] = (1.0 / n1) * p1;
  V3 p2 = tt2 - dot(g.n, tt2) * g.n;
  p2 = p2 - dot(g.t[0], p2) * g.t[0];
  double n2 = norm(p2);
  g.t[1] = (1.0 / n2) * p2;
  g.s[0] = cross(g.t[0], g.n);
  g.s[1] = cross(g.t[1], g.n);
  g.gs_min = std::min(n1, n2);
  return g;
}

// Sec. 3.1, Eq. (U_contribution): U = (a1 x a2)/(g11 g22) at the node of each
// adjacent element; n_v = sum U / |sum U|.  READING: at a corner node the
// element is relabelled cyclically so that the node is the parametric origin
// (the covariant vectors then run along the two element edges leaving the
// node, as in the appendix); at an edge node the canonical d/dxi, d/deta are
// used.  Sec. 3.2, Eqs. (t1), (t2): v_ref = x if |n.z| > 0.9 else z,
// t1 = v_ref x n / |.|, t2 = n x t1.
// READING (frame_rule = 1, not the paper's): v_ref = z everywhere except
// within 1e-8 of the poles, where x is used.  The paper's switch (rule 0)
// interpolates unrelated nodal frames inside the elements that straddle
// |n.z| = 0.9; rule 1 confines that to the few elements around the poles.
static void nodal_frame(Mesh& m, int frame_rule) {
  std::vector<V3> U(m.nn, v3(0, 0, 0));
  const double pxi[6] = {0, 1, 0, 0.5, 0.5, 0};
  const double peta[6] = {0, 0, 1, 0, 0.5, 0.5};
  for (int64_t e = 0; e < m.nt; ++e) {
    for (int k = 0; k < 6; ++k) {
      double N[6], dxi[6], deta[6];
      p2_shape(pxi[k], peta[k], N, dxi, deta);
      V3 A = v3(0, 0, 0), B = v3(0, 0, 0);  // canonical d/dxi, d/deta
      for (int j = 0; j < 6; ++j) {
        A = A + dxi[j] * m.X[m.T[6 * e + j]];
        B = B + deta[j] * m.X[m.T[6 * e + j]];
      }
      V3 a1, a2;
      if (k == 0) {
        a1 = A;
        a2 = B;
      } else if (k == 1) {  // relabel (v1, v2, v0): xi = 1-xi'-eta', eta = xi'
        a1 = B - A;
        a2 = -1.0 * A;
      } else if (k == 2) {  // relabel (v2, v0, v1): xi = eta', eta = 1-xi'-eta'
        a1 = -1.0 * B;
        a2 = A - B;
      } else {
        a1 = A;
        a2 = B;
      }
      V3 u = (1.0 / (dot(a1, a1) * dot(a2, a2))) * cross(a1, a2);
      U[m.T[6 * e + k]] = U[m.T[6 * e + k]] + u;
    }
  }
  m.n.resize(m.nn);
  m.t1.resize(m.nn);
  m.t2.resize(m.nn);
  for (int64_t i = 0; i < m.nn; ++i) {
    V3 nv = unit(U[i]);
    V3 ref;
    if (frame_rule == 1)
      ref = (std::fabs(nv.z) > 1.0 - 1e-8) ? v3(1, 0, 0) : v3(0, 0, 1);
    else
      ref = (std::fabs(nv.z) > 0.9) ? v3(1, 0, 0) : v3(0, 0, 1);
    V3 t1 = unit(cross(ref, nv));
    m.n[i] = nv;
    m.t1[i] = t1;
    m.t2[i] = cross(nv, t1);
  }
}

// ========================================================= kernel scalars
// Sec. 2.3 and 4: with c = 1/(4 pi), z = i k R,
//   k^2 phi - g   = -(c/R^3) (z^2 - z + 1) e^z                 (S1 per k)
//   f             =  (c/R^3) (z^2 - 3z + 3) e^z                 (Eq. Hdiff_exact)
//   phi'(R)       =  (c/R^2) (z - 1) e^z                         (grad phi = phi' R^)
// so that H_diff = (f_a - f_i) R^R^ - (g_a - g_i) I and
//   kappa_1 = S1 (s.t) + S2 (s.R^)(R^.t),  S1 = (ka^2 phi_a - ki^2 phi_i) - (g_a - g_i),
//   S2 = f_a - f_i;  kappa_2^chi = D_chi [(t.t)(n.R^) - (t.R^)(n.t)],
//   D_chi = chi_a phi_a' - chi_i phi_i'.
// Each function is split into its singular leading term and a remainder
// Q(z) = (Taylor tail of the bracket times e^z).  The leading terms
//   S1^s = S2^s = (ka^2 - ki^2)/(8 pi R),  D^s = -(chi_a - chi_i)/(4 pi R^2)
// are Eq. (kappa_S) and Eq. (kappa2_S); the n = 0 and n = 1 terms of
// Eq. (Hdiff_infinite) cancel exactly and never appear.
//   Q1(z) = sum_{m>=3} (m-1)^2      z^m/m! = (z^2 - z + 1)e^z - 1 - z^2/2
//   Q2(z) = sum_{m>=4} (m-1)(m-3)   z^m/m! = (z^2 - 3z + 3)e^z - 3 + z^2/2
//   Q3(z) = sum_{m>=2} (m-1)        z^m/m! = (z - 1)e^z + 1
// READING (stable small-kR form): the power series is summed when |z| < 1,
// the closed form otherwise.
static void qfuncs(cd z, cd& q1, cd& q2, cd& q3) {
  if (std::abs(z) < 1.0) {
    cd t = z;  // z^m/m! at m = 1
    q1 = q2 = q3 = 0.0;
    for (int mm = 2; mm < 80; ++mm) {
      t *= z / (double)mm;
      double m = mm;
      cd d1 = (mm >= 3) ? (m - 1.0) * (m - 1.0) * t : cd(0.0);
      cd d2 = (mm >= 4) ? (m - 1.0) * (m - 3.0) * t : cd(0.0);
      cd d3 = (m - 1.0) * t;
      q1 += d1;
      q2 += d2;
      q3 += d3;
      if (mm > 6 && std::abs(t) * m * m < 1e-18 * std::abs(q2)) break;
    }
  } else {
    cd ez = std::exp(z);
    q1 = (z * z - z + 1.0) * ez - 1.0 - 0.5 * z * z;
    q2 = (z * z - 3.0 * z + 3.0) * ez - 3.0 + 0.5 * z * z;
    q3 = (z - 1.0) * ez + 1.0;
  }
}

struct Phys {
  double ka;            // exterior wavenumber = omega (eps_a = mu_a = 1)
  cd ki;                // interior wavenumber, principal branch
  cd eps_a, eps_i, mu_a, mu_i;
  cd C1;                // (ka^2 - ki^2)/(8 pi)
  cd Ce, Cm;            // -(chi_a - chi_i)/(4 pi)
  cd ae, am;            // (chi_i + chi_a)/2  (Eq. global_system)
};

static Phys make_phys(double ka, double er_re, double er_im, double mr_re, double mr_im) {
  Phys p;
  p.ka = ka;
  p.eps_a = 1.0;
  p.mu_a = 1.0;
  p.eps_i = cd(er_re, er_im);
  p.mu_i = cd(mr_re, mr_im);
  p.ki = ka * std::sqrt(p.eps_i * p.mu_i);
  if (p.ki.imag() < 0) p.ki = -p.ki;
  p.C1 = (ka * ka - p.ki * p.ki) / (8.0 * PI);
  p.Ce = -(p.eps_a - p.eps_i) / (4.0 * PI);
  p.Cm = -(p.mu_a - p.mu_i) / (4.0 * PI);
  p.ae = 0.5 * (p.eps_i + p.eps_a);
  p.am = 0.5 * (p.mu_i + p.mu_a);
  return p;
}

// Scalars S1, S2, D_eps, D_mu at distance R.  If 'remainder', the singular
// leading terms are left out (touching pairs: kappa - kappa^s, Sec. 4.1).
static void kernel_scalars(const Phys& P, double R, bool remainder, cd& S1, cd& S2, cd& De,
                           cd& Dm) {
  const double c = 1.0 / (4.0 * PI);
  cd za = cd(0.0, P.ka * R), zi = cd(0.0, 1.0) * P.ki * R;
  cd q1a, q2a, q3a, q1i, q2i, q3i;
  qfuncs(za, q1a, q2a, q3a);
  qfuncs(zi, q1i, q2i, q3i);
  double R2 = R * R, R3 = R2 * R;
  S1 = -(c / R3) * (q1a - q1i);
  S2 = (c / R3) * (q2a - q2i);
  De = (c / R2) * (P.eps_a * q3a - P.eps_i * q3i);
  Dm = (c / R2) * (P.mu_a * q3a - P.mu_i * q3i);
  if (!remainder) {
    cd s = c * (P.ka * P.ka - P.ki * P.ki) / (2.0 * R);
    S1 += s;
    S2 += s;
    De += -c * (P.eps_a - P.eps_i) / R2;
    Dm += -c * (P.mu_a - P.mu_i) / R2;
  }
}

// Eq. (kappa1_alphabeta) and Eq. (kappa2_alpha_beta) for one point pair;
// out[4*op + 2*alpha + beta], op = 0: K1, 1: K2^eps, 2: K2^mu.
static void kappa(const Phys& P, const Geo& gx, const Geo& gy, bool remainder, cd out[12]) {
  V3 Rv = gx.x - gy.x;
  double R = norm(Rv);
  if (R == 0.0) {
    // coincident quadrature points of a coincident pair (remainder only):
    // limits kappa1 - kappa1^s -> i(ka^3 - ki^3)/(6 pi) s.t,  kappa2 - kappa2^s -> 0
    cd lim = cd(0.0, 1.0) * (P.ka * P.ka * P.ka - P.ki * P.ki * P.ki) / (6.0 * PI);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        out[2 * a + b] = lim * dot(gx.s[a], gy.t[b]);
        out[4 + 2 * a + b] = 0.0;
        out[8 + 2 * a + b] = 0.0;
      }
    return;
  }
  V3 Rh = (1.0 / R) * Rv;
  cd S1, S2, De, Dm;
  kernel_scalars(P, R, remainder, S1, S2, De, Dm);
  double nR = dot(gx.n, Rh);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double st = dot(gx.s[a], gy.t[b]);
      double sR = dot(gx.s[a], Rh), Rt = dot(Rh, gy.t[b]);
      double tt = dot(gx.t[a], gy.t[b]);
      double tR = dot(gx.t[a], Rh), nt = dot(gx.n, gy.t[b]);
      double G = tt * nR - tR * nt;
      out[2 * a + b] = S1 * st + S2 * (sR * Rt);
      out[4 + 2 * a + b] = De * G;
      out[8 + 2 * a + b] = Dm * G;
    }
}

// =================================================== Sauter-Schwab quadrature
// Sec. 4.2 / 5.1: Duffy-type maps of the coincident (6 regions), common-edge
// (5) and common-vertex (2) triangle pairs to [0,1]^4 with tensor
// Gauss-Legendre (Sauter & Schwab, "Boundary Element Methods", Sec. 5.2).
// Reference triangle of the maps: {(u, v): 0 <= v <= u <= 1}; the shared edge
// is v = 0 in both triangles, the shared vertex is (0, 0).  A point (u, v)
// corresponds to the relabelled parametric point (xi', eta') = (u - v, v).
// READING: "order N" is N Gauss points per dimension in every region.
struct SSPt {
  double xu, xv, yu, yv, w;
};

static void ss_points(int cls, int ns, std::vector<SSPt>& pts) {
  std::vector<double> g, gw;
  gauss_legendre01(ns, g, gw);
  pts.clear();
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b)
      for (int c = 0; c < ns; ++c)
        for (int d = 0; d < ns; ++d) {
          double xi = g[a], e1 = g[b], e2 = g[c], e3 = g[d];
          double W = gw[a] * gw[b] * gw[c] * gw[d];
          if (cls == 3) {  // identical triangles, weight xi^3 e1^2 e2
            double j = W * xi * xi * xi * e1 * e1 * e2;
            pts.push_back({xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1), j});
            pts.push_back({xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2), j});
            pts.push_back({xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2), j});
            pts.push_back({xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3), j});
            pts.push_back({xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2), j});
            pts.push_back({xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), j});
          } else if (cls == 2) {  // common edge
            double j1 = W * xi * xi * xi * e1 * e1;
            double j2 = j1 * e2;
            pts.push_back({xi, xi * e1 * e3, xi * (1 - e1 * e2), xi * e1 * (1 - e2), j1});
            pts.push_back({xi, xi * e1, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), j2});
            pts.push_back({xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * e2 * e3, j2});
            pts.push_back({xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), xi, xi * e1, j2});
            pts.push_back({xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * e2, j2});
          } else if (cls == 1) {  // common vertex, weight xi^3 e2
            double j = W * xi * xi * xi * e2;
            pts.push_back({xi, xi * e1, xi * e2, xi * e2 * e3, j});
            pts.push_back({xi * e2, xi * e2 * e3, xi, xi * e1, j});
          }
        }
}

// relabelled reference point (u, v) -> canonical (xi, eta) of the element.
// perm[k] = canonical corner index of relabelled corner k.
static void relabel_to_canonical(const int perm[3], double u, double v, double& xi, double& eta) {
  double lp[3] = {1.0 - u, u - v, v};  // barycentrics of (xi', eta') = (u - v, v)
  double l[3];
  for (int k = 0; k < 3; ++k) l[perm[k]] = lp[k];
  xi = l[1];
  eta = l[2];
}

// Pair classification by shared corner vertices (3 coincident, 2 common
// edge, 1 common vertex, 0 regular) and the relabellings that put the shared
// edge at (v0', v1') / the shared vertex at v0' in both triangles.
static int classify(const Mesh& m, int64_t ex, int64_t ey, int px[3], int py[3], bool alt) {
  const int32_t* a = &m.T[6 * ex];
  const int32_t* b = &m.T[6 * ey];
  int ia[3], ib[3], ns = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (a[i] == b[j]) {
        ia[ns] = i;
        ib[ns] = j;
        ++ns;
      }
  if (ns == 3) {
    for (int k = 0; k < 3; ++k) px[k] = py[k] = k;
  } else if (ns == 2) {
    // order the shared edge as it runs in ex's cyclic order
    int i0 = ia[0], i1 = ia[1], j0 = ib[0], j1 = ib[1];
    if ((i0 + 1) % 3 != i1) {
      std::swap(i0, i1);
      std::swap(j0, j1);
    }
    if (alt) {
      std::swap(i0, i1);
      std::swap(j0, j1);
    }
    px[0] = i0;
    px[1] = i1;
    px[2] = 3 - i0 - i1;
    py[0] = j0;
    py[1] = j1;
    py[2] = 3 - j0 - j1;
  } else if (ns == 1) {
    int i0 = ia[0], j0 = ib[0];
    px[0] = i0;
    px[1] = (i0 + 1) % 3;
    px[2] = (i0 + 2) % 3;
    py[0] = j0;
    if (alt) {
      py[1] = (j0 + 2) % 3;
      py[2] = (j0 + 1) % 3;
    } else {
      py[1] = (j0 + 1) % 3;
      py[2] = (j0 + 2) % 3;
    }
  }
  return ns;
}

// Singular geometric integrals of a touching pair, Eq. (kappa_S) and
// Eq. (kappa2_S) without their complex constants:
//   G1[i][j][ab] = int int N_i N_j [s_a.t_b + (s_a.R^)(R^.t_b)] / R
//   G2[i][j][ab] = int int N_i N_j [(t_a.t_b)(n.R^) - (t_a.R^)(n.t_b)] / R^2
static void ssq_singular(const Mesh& m, int64_t ex, int64_t ey, int cls, const int px[3],
                         const int py[3], int ns, double G1[6][6][4], double G2[6][6][4]) {
  std::vector<SSPt> pts;
  ss_points(cls, ns, pts);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j)
      for (int c = 0; c < 4; ++c) G1[i][j][c] = G2[i][j][c] = 0.0;
  for (const SSPt& s : pts) {
    double xi, eta, yxi, yeta;
    relabel_to_canonical(px, s.xu, s.xv, xi, eta);
    relabel_to_canonical(py, s.yu, s.yv, yxi, yeta);
    Geo gx = geo_at(m, ex, xi, eta);
    Geo gy = geo_at(m, ey, yxi, yeta);
    V3 Rv = gx.x - gy.x;
    double R = norm(Rv);
    if (R == 0.0) continue;  // measure-zero set (never hit by interior Gauss points)
    V3 Rh = (1.0 / R) * Rv;
    double w = s.w * gx.J * gy.J;
    double g1[4], g2[4];
    double nR = dot(gx.n, Rh);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        g1[2 * a + b] = (dot(gx.s[a], gy.t[b]) + dot(gx.s[a], Rh) * dot(Rh, gy.t[b])) / R;
        g2[2 * a + b] =
            (dot(gx.t[a], gy.t[b]) * nR - dot(gx.t[a], Rh) * dot(gx.n, gy.t[b])) / (R * R);
      }
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        double nn = w * gx.N[i] * gy.N[j];
        for (int c = 0; c < 4; ++c) {
          G1[i][j][c] += nn * g1[c];
          G2[i][j][c] += nn * g2[c];
        }
      }
  }
}

// ================================================================ assembly
struct Params {
  double ka, er_re, er_im, mr_re, mr_im;
  int q_regular, ssq_order;
};

// Z layout (Eq. global_system), row-major N x N, N = 4 nn:
//   row    h*(N/2) + 2*i + alpha  (h = 0: electric equation, 1: magnetic)
//   column g*(N/2) + 2*j + beta   (g = 0: c_j, 1: c_jm)
//   Z00 = (i/omega) K1,  Z01 = a_eps M + K2^eps,  Z10 = a_mu M + K2^mu,
//   Z11 = -(i/omega) K1.
// rows_of: if non-null, maps a test node to its output row block (-1 = skip):
// the output then has 4 rows per selected node, ordered (h, alpha).
struct Assembler {
  const Mesh& m;
  Phys P;
  TriRule rule;
  int ns;
  bool alt;
  Assembler(const Mesh& mesh, const Params& pr, bool alt_relabel)
      : m(mesh), P(make_phys(pr.ka, pr.er_re, pr.er_im, pr.mr_re, pr.mr_im)), ns(pr.ssq_order),
        alt(alt_relabel) {
    tri_rule(pr.q_regular, rule);
  }

  // local 6x6x12 block of one ordered element pair (all contributions of the
  // pair: regular rule, or SSQ singular part + regular-rule remainder)
  void pair_block(int64_t ex, int64_t ey, const std::vector<Geo>& gX, const std::vector<Geo>& gY,
                  cd L[6][6][12]) const {
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j)
        for (int c = 0; c < 12; ++c) L[i][j][c] = 0.0;
    int px[3], py[3];
    int cls = classify(m, ex, ey, px, py, alt);
    bool touching = cls > 0;
    size_t Q = rule.w.size();
    for (size_t p = 0; p < Q; ++p)
      for (size_t q = 0; q < Q; ++q) {
        cd kv[12];
        kappa(P, gX[p], gY[q], touching, kv);
        double w = rule.w[p] * gX[p].J * rule.w[q] * gY[q].J;
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j) {
            double nn = w * gX[p].N[i] * gY[q].N[j];
            for (int c = 0; c < 12; ++c) L[i][j][c] += nn * kv[c];
          }
      }
    if (touching) {
      double G1[6][6][4], G2[6][6][4];
      ssq_singular(m, ex, ey, cls, px, py, ns, G1, G2);
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
          for (int c = 0; c < 4; ++c) {
            L[i][j][c] += P.C1 * G1[i][j][c];
            L[i][j][4 + c] += P.Ce * G2[i][j][c];
            L[i][j][8 + c] += P.Cm * G2[i][j][c];
          }
    }
  }
};

// elements coloured so that two elements of one colour share no node
static std::vector<std::vector<int64_t>> color_elements(const Mesh& m) {
  std::vector<std::vector<int64_t>> node_elems(m.nn);
  for (int64_t e = 0; e < m.nt; ++e)
    for (int k = 0; k < 6; ++k) node_elems[m.T[6 * e + k]].push_back(e);
  std::vector<int> col(m.nt, -1);
  int ncol = 0;
  for (int64_t e = 0; e < m.nt; ++e) {
    std::vector<char> used(64, 0);
    for (int k = 0; k < 6; ++k)
      for (int64_t f : node_elems[m.T[6 * e + k]])
        if (col[f] >= 0 && col[f] < 64) used[col[f]] = 1;
    int c = 0;
    while (used[c]) ++c;
    col[e] = c;
    ncol = std::max(ncol, c + 1);
  }
  std::vector<std::vector<int64_t>> out(ncol);
  for (int64_t e = 0; e < m.nt; ++e) out[col[e]].push_back(e);
  return out;
}

static void assemble(const Mesh& m, const Params& pr, bool alt, cd* Z, const int32_t* rows_of,
                     int64_t nrows_out) {
  Assembler A(m, pr, alt);
  const int64_t N = 4 * m.nn, H = 2 * m.nn;
  const cd iw = cd(0.0, 1.0) / A.P.ka;
  size_t Q = A.rule.w.size();
  // precomputed point geometry of every element at the regular rule
  std::vector<std::vector<Geo>> G(m.nt);
  for (int64_t e = 0; e < m.nt; ++e)
    for (size_t p = 0; p < Q; ++p) G[e].push_back(geo_at(m, e, A.rule.xi[p], A.rule.eta[p]));
  auto rowidx = [&](int32_t node, int h, int a) -> int64_t {
    if (!rows_of) return h * H + 2 * (int64_t)node + a;
    int32_t r = rows_of[node];
    if (r < 0) return -1;
    return 4 * (int64_t)r + 2 * h + a;
  };
  (void)nrows_out;
  auto colors = color_elements(m);
  for (auto& cl : colors) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ci = 0; ci < (int64_t)cl.size(); ++ci) {
      int64_t ex = cl[ci];
      bool any = false;
      for (int k = 0; k < 6; ++k)
        if (rowidx(m.T[6 * ex + k], 0, 0) >= 0) any = true;
      if (!any) continue;
      cd L[6][6][12];
      for (int64_t ey = 0; ey < m.nt; ++ey) {
        A.pair_block(ex, ey, G[ex], G[ey], L);
        for (int i = 0; i < 6; ++i) {
          int32_t ni = m.T[6 * ex + i];
          if (rowidx(ni, 0, 0) < 0) continue;
          for (int j = 0; j < 6; ++j) {
            int32_t nj = m.T[6 * ey + j];
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b) {
                int ab = 2 * a + b;
                int64_t c0 = 2 * (int64_t)nj + b, c1 = H + c0;
                Z[rowidx(ni, 0, a) * N + c0] += iw * L[i][j][ab];
                Z[rowidx(ni, 0, a) * N + c1] += L[i][j][4 + ab];
                Z[rowidx(ni, 1, a) * N + c0] += L[i][j][8 + ab];
                Z[rowidx(ni, 1, a) * N + c1] += -iw * L[i][j][ab];
              }
          }
        }
      }
      // Eq. (mass_matrix): delta_ab int N_i N_j, added with a_eps / a_mu
      for (int i = 0; i < 6; ++i) {
        int32_t ni = m.T[6 * ex + i];
        if (rowidx(ni, 0, 0) < 0) continue;
        for (int j = 0; j < 6; ++j) {
          int32_t nj = m.T[6 * ex + j];
          double mij = 0.0;
          for (size_t p = 0; p < Q; ++p) mij += A.rule.w[p] * G[ex][p].J * G[ex][p].N[i] * G[ex][p].N[j];
          for (int a = 0; a < 2; ++a) {
            int64_t c = 2 * (int64_t)nj + a;
            Z[rowidx(ni, 0, a) * N + H + c] += A.P.ae * mij;
            Z[rowidx(ni, 1, a) * N + c] += A.P.am * mij;
          }
        }
      }
    }
  }
}

// Eqs. (rhs_E), (rhs_H): b_E = -eps_a int N_i s_a . E_inc, b_H = mu_a int N_i s_a . H_inc
// READING: E_inc = p exp(i k_a k.x), H_inc = k x E_inc (eta_a = 1).
static void rhs(const Mesh& m, const Params& pr, const double* inc, int r, cd* B) {
  TriRule rule;
  tri_rule(pr.q_regular, rule);
  Phys P = make_phys(pr.ka, pr.er_re, pr.er_im, pr.mr_re, pr.mr_im);
  const int64_t N = 4 * m.nn, H = 2 * m.nn;
  for (int s = 0; s < r; ++s) {
    V3 k = v3(inc[6 * s], inc[6 * s + 1], inc[6 * s + 2]);
    V3 p = v3(inc[6 * s + 3], inc[6 * s + 4], inc[6 * s + 5]);
    V3 h = cross(k, p);
    cd* b = B + (int64_t)s * N;
    for (int64_t i = 0; i < N; ++i) b[i] = 0.0;
    for (int64_t e = 0; e < m.nt; ++e)
      for (size_t q = 0; q < rule.w.size(); ++q) {
        Geo g = geo_at(m, e, rule.xi[q], rule.eta[q]);
        cd ph = std::exp(cd(0.0, P.ka * dot(k, g.x)));
        double w = rule.w[q] * g.J;
        for (int i = 0; i < 6; ++i) {
          int32_t ni = m.T[6 * e + i];
          for (int a = 0; a < 2; ++a) {
            b[2 * (int64_t)ni + a] += -P.eps_a * w * g.N[i] * dot(g.s[a], p) * ph;
            b[H + 2 * (int64_t)ni + a] += P.mu_a * w * g.N[i] * dot(g.s[a], h) * ph;
          }
        }
      }
  }
}

// ================================================================ dense LU
// Partial pivoting; READING: pivot = first row maximising |Re| + |Im|.
static int lu_factor(int64_t n, cd* A, int64_t lda, int32_t* piv) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    double best = -1.0;
    for (int64_t i = k; i < n; ++i) {
      double v = std::fabs(A[i * lda + k].real()) + std::fabs(A[i * lda + k].imag());
      if (v > best) {
        best = v;
        p = i;
      }
    }
    piv[k] = (int32_t)p;
    if (best == 0.0) return (int)(k + 1);
    if (p != k)
      for (int64_t j = 0; j < n; ++j) std::swap(A[k * lda + j], A[p * lda + j]);
    cd inv = 1.0 / A[k * lda + k];
    for (int64_t i = k + 1; i < n; ++i) {
      cd l = A[i * lda + k] * inv;
      A[i * lda + k] = l;
      for (int64_t j = k + 1; j < n; ++j) A[i * lda + j] -= l * A[k * lda + j];
    }
  }
  return 0;
}

static void lu_solve(int64_t n, const cd* A, int64_t lda, const int32_t* piv, cd* b) {
  for (int64_t k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < i; ++j) b[i] -= A[i * lda + j] * b[j];
  for (int64_t i = n - 1; i >= 0; --i) {
    for (int64_t j = i + 1; j < n; ++j) b[i] -= A[i * lda + j] * b[j];
    b[i] /= A[i * lda + i];
  }
}

// ================================================================ MBJ
// Sec. 5, Eq. (precond_block): contiguous clusters I_m of B per-current
// indices (2*node + alpha, Morton order) -> 2|I_m| x 2|I_m| coupled blocks
// taken from all four quadrants.  READING: ceil((N/2)/B) clusters, the last
// one smaller.
struct MBJ {
  int64_t N, H, B, nb;
  std::vector<std::vector<cd>> blk;
  std::vector<std::vector<int32_t>> piv;
  std::vector<int64_t> off, sz;
  int status = 0;
  void build(const cd* Z, int64_t n, int64_t bsz) {
    N = n;
    H = n / 2;
    B = bsz;
    nb = (H + B - 1) / B;
    blk.resize(nb);
    piv.resize(nb);
    off.resize(nb);
    sz.resize(nb);
    for (int64_t b = 0; b < nb; ++b) {
      int64_t o = b * B, s = std::min(B, H - o), d = 2 * s;
      off[b] = o;
      sz[b] = s;
      blk[b].assign(d * d, 0.0);
      for (int64_t i = 0; i < d; ++i) {
        int64_t gi = (i < s) ? o + i : H + o + (i - s);
        for (int64_t j = 0; j < d; ++j) {
          int64_t gj = (j < s) ? o + j : H + o + (j - s);
          blk[b][i * d + j] = Z[gi * N + gj];
        }
      }
      piv[b].resize(d);
      int st = lu_factor(d, blk[b].data(), d, piv[b].data());
      if (st && !status) status = 1;
    }
  }
  void apply(const cd* v, cd* out) const {
    std::vector<cd> t;
    for (int64_t b = 0; b < nb; ++b) {
      int64_t o = off[b], s = sz[b], d = 2 * s;
      t.resize(d);
      for (int64_t i = 0; i < s; ++i) {
        t[i] = v[o + i];
        t[s + i] = v[H + o + i];
      }
      lu_solve(d, blk[b].data(), d, piv[b].data(), t.data());
      for (int64_t i = 0; i < s; ++i) {
        out[o + i] = t[i];
        out[H + o + i] = t[s + i];
      }
    }
  }
};

static void matvec(int64_t n, const cd* Z, const cd* x, cd* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    cd s = 0.0;
    const cd* row = Z + i * n;
    for (int64_t j = 0; j < n; ++j) s += row[j] * x[j];
    y[i] = s;
  }
}

static double vnorm(int64_t n, const cd* v) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += std::norm(v[i]);
  return std::sqrt(s);
}

// Sec. 5 (GMRES with right MBJ preconditioning).  READING: restarted
// GMRES(m), x0 = 0 unless given, classical Gram-Schmidt applied twice, complex
// Givens rotations; stop when the Arnoldi estimate or the true residual at a
// restart reaches ||b - Zx|| <= tol ||b||.
struct GmresInfo {
  int iters, restarts, converged;
  double relres;
};

static GmresInfo gmres(int64_t n, const cd* Z, const MBJ* M, const cd* b, cd* x, int m,
                       double tol, int maxit) {
  GmresInfo info{0, 0, 0, 0.0};
  double bn = vnorm(n, b);
  if (bn == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    info.converged = 1;
    return info;
  }
  std::vector<cd> r(n), w(n), z(n), V((size_t)(m + 1) * n), Hm((size_t)(m + 1) * m), g(m + 1),
      cs(m), sn(m);
  auto residual = [&]() {
    matvec(n, Z, x, w.data());
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
    return vnorm(n, r.data());
  };
  double beta = residual();
  info.relres = beta / bn;
  if (info.relres <= tol) {
    info.converged = 1;
    return info;
  }
  while (info.iters < maxit) {
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    std::fill(g.begin(), g.end(), cd(0.0));
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && info.iters < maxit; ++j) {
      const cd* vj = &V[(size_t)j * n];
      if (M)
        M->apply(vj, z.data());
      else
        std::copy(vj, vj + n, z.begin());
      matvec(n, Z, z.data(), w.data());
      std::vector<cd> h(j + 2, 0.0);
      // classical Gram-Schmidt, twice
      for (int pass = 0; pass < 2; ++pass) {
        std::vector<cd> d(j + 1, 0.0);
        for (int l = 0; l <= j; ++l) {
          const cd* vl = &V[(size_t)l * n];
          cd s = 0.0;
          for (int64_t i = 0; i < n; ++i) s += std::conj(vl[i]) * w[i];
          d[l] = s;
        }
        for (int l = 0; l <= j; ++l) {
          const cd* vl = &V[(size_t)l * n];
          for (int64_t i = 0; i < n; ++i) w[i] -= d[l] * vl[i];
          h[l] += d[l];
        }
      }
      double hn = vnorm(n, w.data());
      h[j + 1] = hn;
      if (hn > 0.0)
        for (int64_t i = 0; i < n; ++i) V[(size_t)(j + 1) * n + i] = w[i] / hn;
      for (int l = 0; l < j; ++l) {
        cd a = h[l], bb = h[l + 1];
        h[l] = cs[l] * a + sn[l] * bb;
        h[l + 1] = -std::conj(sn[l]) * a + cs[l] * bb;
      }
      cd a = h[j], bb = h[j + 1];
      double rho = std::sqrt(std::norm(a) + std::norm(bb));
      if (std::abs(a) == 0.0) {
        cs[j] = 0.0;
        sn[j] = 1.0;
      } else {
        cs[j] = std::abs(a) / rho;
        sn[j] = (a / std::abs(a)) * std::conj(bb) / rho;
      }
      h[j] = cs[j] * a + sn[j] * bb;
      h[j + 1] = 0.0;
      cd gj = g[j];
      g[j] = cs[j] * gj;
      g[j + 1] = -std::conj(sn[j]) * gj;
      for (int l = 0; l <= j; ++l) Hm[(size_t)l * m + j] = h[l];
      ++info.iters;
      k = j + 1;
      if (std::abs(g[j + 1]) / bn <= tol || hn == 0.0) break;
    }
    // y = H^{-1} g, x += M^{-1} V y
    std::vector<cd> y(k);
    for (int i = k - 1; i >= 0; --i) {
      cd s = g[i];
      for (int l = i + 1; l < k; ++l) s -= Hm[(size_t)i * m + l] * y[l];
      y[i] = s / Hm[(size_t)i * m + i];
    }
    std::fill(w.begin(), w.end(), cd(0.0));
    for (int l = 0; l < k; ++l)
      for (int64_t i = 0; i < n; ++i) w[i] += y[l] * V[(size_t)l * n + i];
    if (M)
      M->apply(w.data(), z.data());
    else
      z = w;
    for (int64_t i = 0; i < n; ++i) x[i] += z[i];
    beta = residual();
    info.relres = beta / bn;
    if (info.relres <= tol) {
      info.converged = 1;
      break;
    }
    ++info.restarts;
  }
  return info;
}

// ============================================================ far field
// Scattered far field of the total-field equivalent currents (reading of the
// cross-section formulas, which the paper does not print):
//   E_s ~ e^{ikr}/r F(r^),  F = (i k_a / 4 pi) [ (N~ - r^(r^.N~)) - r^ x L~ ],
//   N~ = int j e^{-i k_a r^.y},  L~ = int j_m e^{-i k_a r^.y}.
//   C_ext = (4 pi / k_a) Im(p . F(k)),  C_sca = int |F|^2 dOmega,
//   C_abs = Re int j_m . (conj(j) x n) dGamma.
static void currents_at(const Mesh& m, const Geo& g, int64_t e, const cd* x, C3& J, C3& Jm) {
  const int64_t H = 2 * m.nn;
  J = c3zero();
  Jm = c3zero();
  for (int k = 0; k < 6; ++k) {
    int32_t nd = m.T[6 * e + k];
    for (int b = 0; b < 2; ++b) {
      J = J + cscale(g.N[k] * x[2 * (int64_t)nd + b], g.t[b]);
      Jm = Jm + cscale(g.N[k] * x[H + 2 * (int64_t)nd + b], g.t[b]);
    }
  }
}

static C3 far_amp(const Mesh& m, const std::vector<std::vector<Geo>>& G, const TriRule& rule,
                  double ka, const cd* x, V3 rh) {
  C3 Nt = c3zero(), Lt = c3zero();
  for (int64_t e = 0; e < m.nt; ++e)
    for (size_t q = 0; q < rule.w.size(); ++q) {
      const Geo& g = G[e][q];
      C3 J, Jm;
      currents_at(m, g, e, x, J, Jm);
      cd ph = std::exp(cd(0.0, -ka * dot(rh, g.x))) * (rule.w[q] * g.J);
      Nt = Nt + cscale(ph, J);
      Lt = Lt + cscale(ph, Jm);
    }
  cd rN = cdotr(rh, Nt);
  C3 tN = Nt + cscale(-rN, rh);
  C3 rL = ccross(rh, Lt);
  cd pre = cd(0.0, ka) / (4.0 * PI);
  return C3{pre * (tN.x - rL.x), pre * (tN.y - rL.y), pre * (tN.z - rL.z)};
}

// ============================================ brute-force singular integrals
// A second, independent route to the singular integrals G1, G2 of a touching
// pair (Eqs. kappa_S, kappa2_S, the integrals that ssq_singular takes by
// Sauter-Schwab), used only to pin ssq_singular: no Sauter-Schwab map, no
// relabelling table.  The test element's parametric triangle T and the trial
// element's triangle T' placed in the same plane by an affine map A --
// coincident: A = identity; common edge: T' folded across the shared edge so
// that the two parametrisations of that edge coincide; common vertex: T'
// reflected through the shared corner -- turn the pair integral into one over
// p in T and q in A(T'), singular only at q = p.  In relative polar
// coordinates q = p + rho e(theta),
//   int_T int_A(T') F dq dp = int dtheta int rho drho
//                              int_{T cap (A(T') - rho e)} F(p, p + rho e) dp,
// and the factor rho cancels the 1/R of the kernels (R >= c rho on these
// placements), so every integrand below is bounded and analytic on its
// piece.  The polygon T cap (A(T') - rho e) is cut from the six edge
// half-planes; theta is split at the directions where the polygon's shape
// changes (edge directions and corner-to-corner vectors), rho at the values
// where three edge lines meet.  Tensor Gauss-Legendre on every piece then
// converges exponentially in the order n (checked in the tests by raising n).
struct P2d {
  double x, y;
};

static double cross2(P2d a, P2d b) { return a.x * b.y - a.y * b.x; }

// half-plane a.p <= b
struct HalfPlane {
  double ax, ay, b;
};

// the three half-planes of a triangle (either orientation)
static void tri_halfplanes(const P2d v[3], HalfPlane h[3]) {
  const double s = cross2(P2d{v[1].x - v[0].x, v[1].y - v[0].y},
                          P2d{v[2].x - v[0].x, v[2].y - v[0].y}) > 0 ? 1.0 : -1.0;
  for (int k = 0; k < 3; ++k) {
    const P2d a = v[k], b = v[(k + 1) % 3];
    // outward normal of edge a -> b for a counter-clockwise triangle
    const double nx = s * (b.y - a.y), ny = -s * (b.x - a.x);
    h[k] = HalfPlane{nx, ny, nx * a.x + ny * a.y};
  }
}

// Sutherland-Hodgman: clip polygon P by a.p <= b
static std::vector<P2d> clip(const std::vector<P2d>& P, double ax, double ay, double b) {
  std::vector<P2d> out;
  const size_t n = P.size();
  for (size_t i = 0; i < n; ++i) {
    const P2d c = P[i], d = P[(i + 1) % n];
    const double fc = ax * c.x + ay * c.y - b, fd = ax * d.x + ay * d.y - b;
    if (fc <= 0) out.push_back(c);
    if ((fc < 0 && fd > 0) || (fc > 0 && fd < 0)) {
      const double t = fc / (fc - fd);
      out.push_back(P2d{c.x + t * (d.x - c.x), c.y + t * (d.y - c.y)});
    }
  }
  return out;
}

static double poly_area(const std::vector<P2d>& P) {
  double a = 0;
  for (size_t i = 0; i < P.size(); ++i) a += cross2(P[i], P[(i + 1) % P.size()]);
  return 0.5 * a;
}

// G[i][j][0..3] = G1, G[i][j][4..7] = G2 (node i of ex, node j of ey, the
// elements' own node order; component 2a + b for s_a or t_a at x, t_b at y)
static int brute_singular(const Mesh& m, int64_t ex, int64_t ey, int n, double G[6][6][8]) {
  const int32_t* tx = &m.T[6 * ex];
  const int32_t* ty = &m.T[6 * ey];
  int sx[3], sy[3], nsh = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (tx[i] == ty[j]) {
        sx[nsh] = i;
        sy[nsh] = j;
        ++nsh;
      }
  if (nsh == 0) return 0;
  const P2d C[3] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};  // canonical corners
  // images of the trial element's corners in the test element's plane
  P2d img[3];
  if (nsh == 3) {
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        if (sy[k] == j) img[j] = C[sx[k]];
  } else if (nsh == 2) {
    const P2d a = C[sx[0]], b = C[sx[1]], c = C[3 - sx[0] - sx[1]];
    // reflection of the test element's third corner across the shared edge
    const double dx = b.x - a.x, dy = b.y - a.y, t = ((c.x - a.x) * dx + (c.y - a.y) * dy) /
                                                     (dx * dx + dy * dy);
    const P2d foot{a.x + t * dx, a.y + t * dy};
    img[sy[0]] = a;
    img[sy[1]] = b;
    img[3 - sy[0] - sy[1]] = P2d{2 * foot.x - c.x, 2 * foot.y - c.y};
  } else {
    const P2d a = C[sx[0]];
    const int i1 = (sx[0] + 1) % 3, i2 = (sx[0] + 2) % 3;
    img[sy[0]] = a;
    img[(sy[0] + 1) % 3] = P2d{2 * a.x - C[i1].x, 2 * a.y - C[i1].y};
    img[(sy[0] + 2) % 3] = P2d{2 * a.x - C[i2].x, 2 * a.y - C[i2].y};
  }
  // A maps the trial element's parametric point (xi, eta) to
  // img0 + xi (img1 - img0) + eta (img2 - img0); its inverse takes q back
  const P2d e1{img[1].x - img[0].x, img[1].y - img[0].y};
  const P2d e2{img[2].x - img[0].x, img[2].y - img[0].y};
  const double detA = cross2(e1, e2);
  auto to_trial = [&](P2d q, double& xi, double& eta) {
    const P2d d{q.x - img[0].x, q.y - img[0].y};
    xi = cross2(d, e2) / detA;
    eta = cross2(e1, d) / detA;
  };
  HalfPlane hx[3], hy[3];
  tri_halfplanes(C, hx);
  tri_halfplanes(img, hy);
  // critical directions: edges of both triangles and corner-to-corner vectors
  std::vector<double> crit;
  auto add_dir = [&](double x, double y) {
    if (std::hypot(x, y) < 1e-14) return;
    double a = std::atan2(y, x);
    if (a < 0) a += 2 * PI;
    crit.push_back(a);
    double b = a + PI;
    if (b >= 2 * PI) b -= 2 * PI;
    crit.push_back(b);
  };
  for (int k = 0; k < 3; ++k) {
    add_dir(C[(k + 1) % 3].x - C[k].x, C[(k + 1) % 3].y - C[k].y);
    add_dir(img[(k + 1) % 3].x - img[k].x, img[(k + 1) % 3].y - img[k].y);
    for (int j = 0; j < 3; ++j) add_dir(img[j].x - C[k].x, img[j].y - C[k].y);
  }
  crit.push_back(0.0);
  crit.push_back(2 * PI);
  std::sort(crit.begin(), crit.end());
  std::vector<double> th;
  for (double a : crit)
    if (th.empty() || a - th.back() > 1e-12) th.push_back(a);
  std::vector<double> g, gw;
  gauss_legendre01(n, g, gw);
  // one work item per (theta piece, theta node)
  const int npiece = (int)th.size() - 1;
  std::vector<double> acc((size_t)npiece * n * 288, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int item = 0; item < npiece * n; ++item) {
    const int ip = item / n, it = item % n;
    const double t0 = th[ip], t1 = th[ip + 1];
    const double theta = t0 + (t1 - t0) * g[it];
    const double wth = (t1 - t0) * gw[it];
    const P2d e{std::cos(theta), std::sin(theta)};
    // lines a.p = b + rho c: test triangle (c = 0), shifted trial triangle
    double la[6][2], lb[6], lc[6];
    for (int k = 0; k < 3; ++k) {
      la[k][0] = hx[k].ax;
      la[k][1] = hx[k].ay;
      lb[k] = hx[k].b;
      lc[k] = 0.0;
      la[3 + k][0] = hy[k].ax;
      la[3 + k][1] = hy[k].ay;
      lb[3 + k] = hy[k].b;
      lc[3 + k] = -(hy[k].ax * e.x + hy[k].ay * e.y);
    }
    std::vector<double> br{0.0};
    for (int a = 0; a < 6; ++a)
      for (int b = a + 1; b < 6; ++b)
        for (int c = b + 1; c < 6; ++c) {
          auto det3 = [&](const double* col) {
            return la[a][0] * (la[b][1] * col[c] - la[c][1] * col[b]) -
                   la[a][1] * (la[b][0] * col[c] - la[c][0] * col[b]) +
                   col[a] * (la[b][0] * la[c][1] - la[c][0] * la[b][1]);
          };
          const double D0 = det3(lb), D1 = det3(lc);
          if (std::fabs(D1) < 1e-14) continue;
          const double r = -D0 / D1;
          if (r > 1e-13 && r < 10.0) br.push_back(r);
        }
    std::sort(br.begin(), br.end());
    double* out = &acc[(size_t)item * 288];
    for (size_t k = 0; k + 1 < br.size(); ++k) {
      const double r0 = br[k], r1 = br[k + 1];
      if (r1 - r0 < 1e-13) continue;
      for (int ir = 0; ir < n; ++ir) {
        const double rho = r0 + (r1 - r0) * g[ir];
        const double wr = (r1 - r0) * gw[ir] * rho * wth;
        std::vector<P2d> P(C, C + 3);
        for (int j = 0; j < 3 && !P.empty(); ++j)
          P = clip(P, hy[j].ax, hy[j].ay, hy[j].b - rho * (hy[j].ax * e.x + hy[j].ay * e.y));
        if (P.size() < 3 || std::fabs(poly_area(P)) < 1e-300) continue;
        for (size_t f = 1; f + 1 < P.size(); ++f) {
          const P2d A0 = P[0], B0 = P[f], C0 = P[f + 1];
          const double jac = std::fabs(cross2(P2d{B0.x - A0.x, B0.y - A0.y},
                                              P2d{C0.x - A0.x, C0.y - A0.y}));
          for (int is = 0; is < n; ++is)
            for (int jt = 0; jt < n; ++jt) {
              const double s = g[is], t = g[jt];
              const P2d p{A0.x + s * ((1 - t) * (B0.x - A0.x) + t * (C0.x - A0.x)),
                          A0.y + s * ((1 - t) * (B0.y - A0.y) + t * (C0.y - A0.y))};
              const double wp = gw[is] * gw[jt] * s * jac;
              double yxi, yeta;
              to_trial(P2d{p.x + rho * e.x, p.y + rho * e.y}, yxi, yeta);
              const Geo gx = geo_at(m, ex, p.x, p.y);
              const Geo gy = geo_at(m, ey, yxi, yeta);
              const V3 d = gx.x - gy.x;
              const double R = norm(d);
              const V3 u = (1.0 / R) * d;
              const double w = wr * wp * gx.J * gy.J / std::fabs(detA);
              const double nu = dot(gx.n, u);
              double k1[4], k2[4];
              for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                  const double ty_b_u = dot(gy.t[b], u);
                  k1[2 * a + b] = (dot(gx.s[a], gy.t[b]) + dot(gx.s[a], u) * ty_b_u) / R;
                  k2[2 * a + b] =
                      (dot(gx.t[a], gy.t[b]) * nu - dot(gx.t[a], u) * dot(gx.n, gy.t[b])) / (R * R);
                }
              for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                  const double nn = w * gx.N[i] * gy.N[j];
                  for (int c = 0; c < 4; ++c) {
                    out[(i * 6 + j) * 8 + c] += nn * k1[c];
                    out[(i * 6 + j) * 8 + 4 + c] += nn * k2[c];
                  }
                }
            }
        }
      }
    }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j)
      for (int c = 0; c < 8; ++c) {
        double s = 0;
        for (int item = 0; item < npiece * n; ++item) s += acc[(size_t)item * 288 + (i * 6 + j) * 8 + c];
        G[i][j][c] = s;
      }
  return nsh;
}

// ================================================================ C API
struct OracleMesh {
  Mesh m;
};

extern "C" {

int oracle_version(void) { return 1; }

int oracle_tri_rule(int q, double* xi, double* eta, double* w) {
  TriRule r;
  if (!tri_rule(q, r)) return -1;
  for (size_t i = 0; i < r.w.size(); ++i) {
    xi[i] = r.xi[i];
    eta[i] = r.eta[i];
    w[i] = r.w[i];
  }
  return (int)r.w.size();
}

void oracle_gauss_legendre01(int n, double* x, double* w) {
  std::vector<double> a, b;
  gauss_legendre01(n, a, b);
  for (int i = 0; i < n; ++i) {
    x[i] = a[i];
    w[i] = b[i];
  }
}

void oracle_morton(const double* xyz, int64_t nn, const int32_t* tri6, int64_t nt,
                   int32_t* node_perm, int32_t* elem_perm) {
  std::vector<int32_t> np, ep;
  morton_perms(xyz, nn, tri6, nt, np, ep);
  std::copy(np.begin(), np.end(), node_perm);
  std::copy(ep.begin(), ep.end(), elem_perm);
}

// Build the oracle mesh: Morton permutation (unless flags & 1), nodal frame
// with rule (flags >> 1) & 1.
void* oracle_mesh_new(const double* xyz, int64_t nn, const int32_t* tri6, int64_t nt,
                      int32_t flags) {
  OracleMesh* h = new OracleMesh();
  Mesh& m = h->m;
  m.nn = nn;
  m.nt = nt;
  if (flags & 1) {
    m.node_perm.resize(nn);
    m.elem_perm.resize(nt);
    std::iota(m.node_perm.begin(), m.node_perm.end(), 0);
    std::iota(m.elem_perm.begin(), m.elem_perm.end(), 0);
  } else {
    morton_perms(xyz, nn, tri6, nt, m.node_perm, m.elem_perm);
  }
  std::vector<int32_t> inv(nn);
  for (int64_t i = 0; i < nn; ++i) inv[m.node_perm[i]] = (int32_t)i;
  m.X.resize(nn);
  for (int64_t i = 0; i < nn; ++i) {
    int64_t o = m.node_perm[i];
    m.X[i] = v3(xyz[3 * o], xyz[3 * o + 1], xyz[3 * o + 2]);
  }
  m.T.resize(6 * nt);
  for (int64_t e = 0; e < nt; ++e)
    for (int k = 0; k < 6; ++k) m.T[6 * e + k] = inv[tri6[6 * m.elem_perm[e] + k]];
  nodal_frame(m, (flags >> 1) & 1);
  return h;
}

void oracle_mesh_free(void* h) { delete (OracleMesh*)h; }

void oracle_mesh_perm(void* h, int32_t* node_perm, int32_t* elem_perm) {
  Mesh& m = ((OracleMesh*)h)->m;
  std::copy(m.node_perm.begin(), m.node_perm.end(), node_perm);
  std::copy(m.elem_perm.begin(), m.elem_perm.end(), elem_perm);
}

// nodal frame [nn][9] = (n, t1, t2), Morton order
void oracle_frame(void* h, double* out) {
  Mesh& m = ((OracleMesh*)h)->m;
  for (int64_t i = 0; i < m.nn; ++i) {
    V3 v[3] = {m.n[i], m.t1[i], m.t2[i]};
    for (int a = 0; a < 3; ++a) {
      out[9 * i + 3 * a] = v[a].x;
      out[9 * i + 3 * a + 1] = v[a].y;
      out[9 * i + 3 * a + 2] = v[a].z;
    }
  }
}

// geometry at a parametric point: out[22] = x(3), n(3), t1(3), t2(3), s1(3),
// s2(3), J, gs_min, N0..N5 dropped; returns J
double oracle_point_geo(void* h, int64_t e, double xi, double eta, double* out) {
  Mesh& m = ((OracleMesh*)h)->m;
  Geo g = geo_at(m, e, xi, eta);
  V3 v[6] = {g.x, g.n, g.t[0], g.t[1], g.s[0], g.s[1]};
  for (int a = 0; a < 6; ++a) {
    out[3 * a] = v[a].x;
    out[3 * a + 1] = v[a].y;
    out[3 * a + 2] = v[a].z;
  }
  out[18] = g.J;
  out[19] = g.gs_min;
  return g.J;
}

// kernel scalars at distance R: out = [S1, S2, De, Dm] as (re, im) pairs
void oracle_kernel_scalars(double ka, double er_re, double er_im, double mr_re, double mr_im,
                           double R, int remainder, double* out) {
  Phys P = make_phys(ka, er_re, er_im, mr_re, mr_im);
  cd v[4];
  kernel_scalars(P, R, remainder != 0, v[0], v[1], v[2], v[3]);
  for (int i = 0; i < 4; ++i) {
    out[2 * i] = v[i].real();
    out[2 * i + 1] = v[i].imag();
  }
}

// Hessian difference H_diff = A R^R^ + B I (Eq. Hdiff_exact): out = [A, B]
// as (re, im) pairs, A = f_a - f_i = S2, B = -(g_a - g_i).
void oracle_hdiff(double ka, double er_re, double er_im, double mr_re, double mr_im, double R,
                  double* out) {
  Phys P = make_phys(ka, er_re, er_im, mr_re, mr_im);
  Phys Q = P;
  Q.eps_a = 1.0;
  Q.eps_i = 1.0;
  cd S1, S2, De, Dm;
  kernel_scalars(Q, R, false, S1, S2, De, Dm);
  // with chi_a = chi_i = 1, D = phi_a' - phi_i' and g = -phi'/R
  cd B = De / R;
  out[0] = S2.real();
  out[1] = S2.imag();
  out[2] = B.real();
  out[3] = B.imag();
}

// Q-functions at complex z (pins of the series/closed-form switch)
void oracle_qfuncs(double zr, double zi, double* out) {
  cd q1, q2, q3;
  qfuncs(cd(zr, zi), q1, q2, q3);
  out[0] = q1.real();
  out[1] = q1.imag();
  out[2] = q2.real();
  out[3] = q2.imag();
  out[4] = q3.real();
  out[5] = q3.imag();
}

// Sauter-Schwab points of a class on the reference triangle {0<=v<=u<=1}:
// returns the count; if out != NULL writes rows (xu, xv, yu, yv, w).
int64_t oracle_ss_points(int cls, int ns, double* out) {
  std::vector<SSPt> p;
  ss_points(cls, ns, p);
  if (out)
    for (size_t i = 0; i < p.size(); ++i) {
      out[5 * i] = p[i].xu;
      out[5 * i + 1] = p[i].xv;
      out[5 * i + 2] = p[i].yu;
      out[5 * i + 3] = p[i].yv;
      out[5 * i + 4] = p[i].w;
    }
  return (int64_t)p.size();
}

// pair classification: returns class, writes both relabellings
int oracle_classify(void* h, int64_t ex, int64_t ey, int alt, int32_t* px, int32_t* py) {
  Mesh& m = ((OracleMesh*)h)->m;
  int a[3] = {0, 1, 2}, b[3] = {0, 1, 2};
  int c = classify(m, ex, ey, a, b, alt != 0);
  for (int k = 0; k < 3; ++k) {
    px[k] = a[k];
    py[k] = b[k];
  }
  return c;
}

// singular integrals of a touching pair: out[6][6][8] = (G1[4], G2[4])
int oracle_ssq_singular(void* h, int64_t ex, int64_t ey, int ns, int alt, double* out) {
  Mesh& m = ((OracleMesh*)h)->m;
  int px[3], py[3];
  int cls = classify(m, ex, ey, px, py, alt != 0);
  if (cls == 0) return 0;
  double G1[6][6][4], G2[6][6][4];
  ssq_singular(m, ex, ey, cls, px, py, ns, G1, G2);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j)
      for (int c = 0; c < 4; ++c) {
        out[((i * 6 + j) * 8) + c] = G1[i][j][c];
        out[((i * 6 + j) * 8) + 4 + c] = G2[i][j][c];
      }
  return cls;
}

// SSQ of an arbitrary test integrand over a touching pair of the mesh, to pin
// the maps: which = 0: 1, 1: 1/R, 2: |x - y|^2 (x, y physical points).
double oracle_ssq_test(void* h, int64_t ex, int64_t ey, int ns, int alt, int which) {
  Mesh& m = ((OracleMesh*)h)->m;
  int px[3], py[3];
  int cls = classify(m, ex, ey, px, py, alt != 0);
  if (cls == 0) return NAN;
  std::vector<SSPt> pts;
  ss_points(cls, ns, pts);
  double s = 0.0;
  for (const SSPt& p : pts) {
    double xi, eta, yxi, yeta;
    relabel_to_canonical(px, p.xu, p.xv, xi, eta);
    relabel_to_canonical(py, p.yu, p.yv, yxi, yeta);
    Geo gx = geo_at(m, ex, xi, eta), gy = geo_at(m, ey, yxi, yeta);
    double R = norm(gx.x - gy.x);
    double f = (which == 0) ? 1.0 : (which == 1 ? 1.0 / R : R * R);
    s += p.w * gx.J * gy.J * f;
  }
  return s;
}

// The whole kernel kappa (not only its singular part) integrated by
// Sauter-Schwab over a touching pair: the reference that the split
// "singular part by SSQ + remainder by the regular rule" must approach.
// out: 6x6x12 complex (re, im) interleaved.
int oracle_ssq_full(void* h, double ka, double er_re, double er_im, double mr_re, double mr_im,
                    int64_t ex, int64_t ey, int ns, double* out) {
  Mesh& m = ((OracleMesh*)h)->m;
  Phys P = make_phys(ka, er_re, er_im, mr_re, mr_im);
  int px[3], py[3];
  int cls = classify(m, ex, ey, px, py, false);
  if (cls == 0) return 0;
  std::vector<SSPt> pts;
  ss_points(cls, ns, pts);
  std::vector<cd> L(6 * 6 * 12, 0.0);
  for (const SSPt& s : pts) {
    double xi, eta, yxi, yeta;
    relabel_to_canonical(px, s.xu, s.xv, xi, eta);
    relabel_to_canonical(py, s.yu, s.yv, yxi, yeta);
    Geo gx = geo_at(m, ex, xi, eta), gy = geo_at(m, ey, yxi, yeta);
    cd kv[12];
    kappa(P, gx, gy, false, kv);
    double w = s.w * gx.J * gy.J;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j)
        for (int c = 0; c < 12; ++c) L[(i * 6 + j) * 12 + c] += w * gx.N[i] * gy.N[j] * kv[c];
  }
  for (int k = 0; k < 6 * 6 * 12; ++k) {
    out[2 * k] = L[k].real();
    out[2 * k + 1] = L[k].imag();
  }
  return cls;
}

// local 6x6x12 block of one element pair, complex (re, im) interleaved
int oracle_pair_block(void* h, double ka, double er_re, double er_im, double mr_re, double mr_im,
                      int q_regular, int ssq_order, int64_t ex, int64_t ey, double* out) {
  Mesh& m = ((OracleMesh*)h)->m;
  Params pr{ka, er_re, er_im, mr_re, mr_im, q_regular, ssq_order};
  Assembler A(m, pr, false);
  std::vector<Geo> gx, gy;
  for (size_t p = 0; p < A.rule.w.size(); ++p) {
    gx.push_back(geo_at(m, ex, A.rule.xi[p], A.rule.eta[p]));
    gy.push_back(geo_at(m, ey, A.rule.xi[p], A.rule.eta[p]));
  }
  cd L[6][6][12];
  A.pair_block(ex, ey, gx, gy, L);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j)
      for (int c = 0; c < 12; ++c) {
        out[2 * ((i * 6 + j) * 12 + c)] = L[i][j][c].real();
        out[2 * ((i * 6 + j) * 12 + c) + 1] = L[i][j][c].imag();
      }
  int px[3], py[3];
  return classify(m, ex, ey, px, py, false);
}

// Dense assembly of Z (N x N complex128, row-major, zero-initialised by the
// caller).  If rows_of != NULL only the rows of the selected test nodes are
// produced (4 rows per node, see 'assemble').
void oracle_assemble(void* h, double ka, double er_re, double er_im, double mr_re, double mr_im,
                     int q_regular, int ssq_order, int alt, double* Z, const int32_t* rows_of,
                     int64_t nrows) {
  Mesh& m = ((OracleMesh*)h)->m;
  Params pr{ka, er_re, er_im, mr_re, mr_im, q_regular, ssq_order};
  assemble(m, pr, alt != 0, (cd*)Z, rows_of, nrows);
}

void oracle_rhs(void* h, double ka, double er_re, double er_im, double mr_re, double mr_im,
                int q_regular, const double* inc, int r, double* B) {
  Mesh& m = ((OracleMesh*)h)->m;
  Params pr{ka, er_re, er_im, mr_re, mr_im, q_regular, 5};
  rhs(m, pr, inc, r, (cd*)B);
}

// singular integrals of a touching pair by the brute-force route (pin of
// ssq_singular): out[6][6][8] = (G1[4], G2[4]), the elements' own node
// order; n = Gauss order of every direction of every piece.  Returns the
// number of shared corners (0: not a touching pair, nothing written).
int oracle_brute_singular(void* h, int64_t ex, int64_t ey, int n, double* out) {
  Mesh& m = ((OracleMesh*)h)->m;
  double G[6][6][8];
  int c = brute_singular(m, ex, ey, n, G);
  if (c == 0) return 0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j)
      for (int k = 0; k < 8; ++k) out[(i * 6 + j) * 8 + k] = G[i][j][k];
  return c;
}

// Mass matrix of the scalar P2 Gram (Eq. mass_matrix), dense nn x nn, real.
void oracle_mass(void* h, int q_regular, double* M) {
  Mesh& m = ((OracleMesh*)h)->m;
  TriRule rule;
  tri_rule(q_regular, rule);
  for (int64_t e = 0; e < m.nt; ++e)
    for (size_t q = 0; q < rule.w.size(); ++q) {
      Geo g = geo_at(m, e, rule.xi[q], rule.eta[q]);
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
          M[(int64_t)m.T[6 * e + i] * m.nn + m.T[6 * e + j]] += rule.w[q] * g.J * g.N[i] * g.N[j];
    }
}

// Dense LU solve of Z X = B (X, B: r rows of N), Z overwritten by its factors.
int oracle_lu_solve(int64_t n, double* Z, const double* B, int r, double* X) {
  std::vector<int32_t> piv(n);
  int st = lu_factor(n, (cd*)Z, n, piv.data());
  if (st) return st;
  for (int s = 0; s < r; ++s) {
    cd* x = (cd*)X + (int64_t)s * n;
    const cd* b = (const cd*)B + (int64_t)s * n;
    std::copy(b, b + n, x);
    lu_solve(n, (cd*)Z, n, piv.data(), x);
  }
  return 0;
}

// GMRES(m) with MBJ (block > 0) or without (block == 0).  x: in/out (x0).
// info[4] = iterations, restarts, converged, relres.
int oracle_gmres(int64_t n, const double* Z, const double* b, double* x, int64_t block, int m,
                 double tol, int maxit, double* info) {
  MBJ M;
  if (block > 0) {
    M.build((const cd*)Z, n, block);
    if (M.status) return 1;
  }
  GmresInfo gi = gmres(n, (const cd*)Z, block > 0 ? &M : nullptr, (const cd*)b, (cd*)x, m, tol,
                       maxit);
  info[0] = gi.iters;
  info[1] = gi.restarts;
  info[2] = gi.converged;
  info[3] = gi.relres;
  return 0;
}

// MBJ apply of one vector (for tests of the preconditioner alone)
int oracle_mbj_apply(int64_t n, const double* Z, int64_t block, const double* v, double* out) {
  MBJ M;
  M.build((const cd*)Z, n, block);
  if (M.status) return 1;
  M.apply((const cd*)v, (cd*)out);
  return 0;
}

// Far field amplitudes F (r x ndir x 3 complex) and cross sections
// xs (r x 3: C_ext, C_sca, C_abs).  X: r rows of N.  C_sca uses a
// Gauss-Legendre(n_theta) x trapezoid(n_phi) rule on the unit sphere.
void oracle_far_field(void* h, double ka, int q_regular, const double* X, int r,
                      const double* inc, const double* dirs, int64_t ndir, double* F, double* xs,
                      int n_theta, int n_phi) {
  Mesh& m = ((OracleMesh*)h)->m;
  TriRule rule;
  tri_rule(q_regular, rule);
  std::vector<std::vector<Geo>> G(m.nt);
  for (int64_t e = 0; e < m.nt; ++e)
    for (size_t q = 0; q < rule.w.size(); ++q) G[e].push_back(geo_at(m, e, rule.xi[q], rule.eta[q]));
  const int64_t N = 4 * m.nn;
  std::vector<double> gt, gw;
  gauss_legendre01(n_theta, gt, gw);
  for (int s = 0; s < r; ++s) {
    const cd* x = (const cd*)X + (int64_t)s * N;
    for (int64_t d = 0; d < ndir; ++d) {
      C3 f = far_amp(m, G, rule, ka, x, v3(dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]));
      cd* o = (cd*)F + ((int64_t)s * ndir + d) * 3;
      o[0] = f.x;
      o[1] = f.y;
      o[2] = f.z;
    }
    V3 k = v3(inc[6 * s], inc[6 * s + 1], inc[6 * s + 2]);
    V3 p = v3(inc[6 * s + 3], inc[6 * s + 4], inc[6 * s + 5]);
    C3 fk = far_amp(m, G, rule, ka, x, k);
    double cext = 4.0 * PI / ka * cdotr(p, fk).imag();
    double csca = 0.0;
#pragma omp parallel for reduction(+ : csca) collapse(2)
    for (int it = 0; it < n_theta; ++it)
      for (int ip = 0; ip < n_phi; ++ip) {
        double ct = 2.0 * gt[it] - 1.0, st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
        double ph = 2.0 * PI * ip / n_phi;
        C3 f = far_amp(m, G, rule, ka, x, v3(st * std::cos(ph), st * std::sin(ph), ct));
        double a = std::norm(f.x) + std::norm(f.y) + std::norm(f.z);
        csca += a * 2.0 * gw[it] * (2.0 * PI / n_phi);
      }
    double cabs = 0.0;
    for (int64_t e = 0; e < m.nt; ++e)
      for (size_t q = 0; q < rule.w.size(); ++q) {
        const Geo& g = G[e][q];
        C3 J, Jm;
        currents_at(m, g, e, x, J, Jm);
        C3 Jc{std::conj(J.x), std::conj(J.y), std::conj(J.z)};
        // conj(J) x n
        C3 jxn{Jc.y * g.n.z - Jc.z * g.n.y, Jc.z * g.n.x - Jc.x * g.n.z,
               Jc.x * g.n.y - Jc.y * g.n.x};
        cd v = Jm.x * jxn.x + Jm.y * jxn.y + Jm.z * jxn.z;
        cabs += rule.w[q] * g.J * v.real();
      }
    xs[3 * s] = cext;
    xs[3 * s + 1] = csca;
    xs[3 * s + 2] = cabs;
  }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
