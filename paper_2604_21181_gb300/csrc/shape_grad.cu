// Gradients with respect to the P2 node coordinates (adjoint method).
//
// The cross sections C depend on the node coordinates X through the
// operator, the right-hand side and the far-field functionals:
//   Z(X) x = b(X),  dC/dX = dC/dX|_x + 2 Re lam^H (db/dX - (dZ/dX) x),
//   Z^H lam = g^*,  dC = 2 Re(g^T dx) at fixed X.
// This file computes the three X-gradients at given x and lam as vector-
// Jacobian products, in reverse mode, without forming any derivative of Z:
//   * every element pair's kernel values (Sec. 4.1: regular pairs on the
//     product rule, the remainder kappa - kappa^s of touching pairs, the
//     Sauter-Schwab integrals of the singular parts of Eqs. kappa_S and
//     kappa2_S, the mass term of Eq. mass_matrix) are recomputed together
//     with their derivatives with respect to the point geometry and
//     contracted with lam at the test points and x at the trial points;
//   * the adjoints of the point geometry (position, normal, frame, weight)
//     are carried back through the continuous frame of Sec. 3.3 (Gram-
//     Schmidt of the interpolated nodal frame) and the P2 map to the node
//     positions and nodal frames, and through Sec. 3.2 (t1 = v_ref x n/|.|,
//     t2 = n x t1) and Sec. 3.1 (n_v = sum U/|sum U|, U = a1 x a2/(g11 g22))
//     to the node positions;
//   * the right-hand side (Eqs. rhs_E, rhs_H) and the far-field cross
//     sections the same way.
// The reference-axis switch of the frame rule and the sign of the
// Gram-Schmidt side are piecewise constant and contribute nothing.
#include <math.h>

#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "p2.cuh"
#include "ssq.cuh"

namespace mu {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kC4pi = 0.0795774715459476678844418816862571885;  // 1/(4 pi)

struct RuleC {
  int Q;
  double xi[MAX_Q], eta[MAX_Q], w[MAX_Q];
};

struct GLC {
  int ns;
  double x[MAX_NS], w[MAX_NS];
};

__device__ __forceinline__ void p2N(double xi, double eta, double N[6]) {
  const double l0 = 1.0 - xi - eta;
  N[0] = l0 * (2.0 * l0 - 1.0);
  N[1] = xi * (2.0 * xi - 1.0);
  N[2] = eta * (2.0 * eta - 1.0);
  N[3] = 4.0 * l0 * xi;
  N[4] = 4.0 * xi * eta;
  N[5] = 4.0 * eta * l0;
}

__device__ __forceinline__ d3 ld3(const double* p) { return mk(p[0], p[1], p[2]); }
__device__ __forceinline__ void acc3(double* g, d3 v) {
  g[0] += v.x;
  g[1] += v.y;
  g[2] += v.z;
}
__device__ __forceinline__ void acc3s(double* g, double s, d3 v) {
  g[0] += s * v.x;
  g[1] += s * v.y;
  g[2] += s * v.z;
}

// ------------------------------------------------------------------ radial
// The radial functions of the kernel (S1, S2, De, Dm; see kernels.cuh) and
// their derivatives in r.  With z = i k r, d/dr Q(z) = Q'(z) i k.
__device__ void radial_d(const KConst<double>& K, double r, bool remainder, cx<double> f[4],
                         cx<double> df[4]) {
  const double c = kC4pi;
  const cx<double> za = cmk(0.0, K.ka * r);
  const cx<double> zi = cmk(-K.ki_im * r, K.ki_re * r);
  cx<double> q1a, q2a, q3a, q1i, q2i, q3i, p1a, p2a, p3a, p1i, p2i, p3i, t;
  qfuncs(za, q1a, q2a, q3a);
  qfuncs(zi, q1i, q2i, q3i);
  qfuncs_d(za, p1a, p2a, p3a, t);
  qfuncs_d(zi, p1i, p2i, p3i, t);
  const cx<double> ika = cmk(0.0, K.ka), iki = cmk(-K.ki_im, K.ki_re);
  const double ir = 1.0 / r, ir2 = ir * ir, ir3 = ir2 * ir, ir4 = ir2 * ir2;
  const cx<double> eps = cmk(K.eps_re, K.eps_im), mu = cmk(K.mu_re, K.mu_im);
  const cx<double> d1 = csub(q1a, q1i), d2 = csub(q2a, q2i);
  const cx<double> dd1 = csub(cmul(p1a, ika), cmul(p1i, iki));
  const cx<double> dd2 = csub(cmul(p2a, ika), cmul(p2i, iki));
  f[0] = crs(-c * ir3, d1);
  df[0] = cadd(crs(3.0 * c * ir4, d1), crs(-c * ir3, dd1));
  f[1] = crs(c * ir3, d2);
  df[1] = cadd(crs(-3.0 * c * ir4, d2), crs(c * ir3, dd2));
  const cx<double> q3d = cmul(p3a, ika), q3di = cmul(p3i, iki);
  const cx<double> de = csub(q3a, cmul(eps, q3i)), dm = csub(q3a, cmul(mu, q3i));
  const cx<double> dde = csub(q3d, cmul(eps, q3di)), ddm = csub(q3d, cmul(mu, q3di));
  f[2] = crs(c * ir2, de);
  df[2] = cadd(crs(-2.0 * c * ir3, de), crs(c * ir2, dde));
  f[3] = crs(c * ir2, dm);
  df[3] = cadd(crs(-2.0 * c * ir3, dm), crs(c * ir2, ddm));
  if (!remainder) {
    const cx<double> ki2 = cmk(K.ki_re * K.ki_re - K.ki_im * K.ki_im, 2.0 * K.ki_re * K.ki_im);
    const cx<double> s0 = crs(0.5 * c, cmk(K.ka * K.ka - ki2.re, -ki2.im));
    f[0] = cadd(f[0], crs(ir, s0));
    f[1] = cadd(f[1], crs(ir, s0));
    df[0] = cadd(df[0], crs(-ir2, s0));
    df[1] = cadd(df[1], crs(-ir2, s0));
    const cx<double> ce = cmk(1.0 - K.eps_re, -K.eps_im), cm = cmk(1.0 - K.mu_re, -K.mu_im);
    f[2] = cadd(f[2], crs(-c * ir2, ce));
    f[3] = cadd(f[3], crs(-c * ir2, cm));
    df[2] = cadd(df[2], crs(2.0 * c * ir3, ce));
    df[3] = cadd(df[3], crs(2.0 * c * ir3, cm));
  }
}

// Value and gradient of  V = sum_ab [ c1_ab (s_a.t_b) + c2_ab (s_a.h)(h.t_b)
//                                    + cG_ab ((t_a.t_b)(n.h) - (t_a.h)(n.t_b)) ]
// with real coefficients, s_a, t_a, n of the test point x, t_b of the trial
// point y, h = (x - y)/r; and dV/dr at fixed h for the radial parts (given
// as dc1, dc2, dcG).  Outputs: gR = dV/dR (R = x - y), gs[a], gtx[a], gn,
// gty[b] (3-vectors).
struct PairGeo {
  d3 s[2], t[2], n, u[2];  // s, t, n at x; u = t at y
};

__device__ __forceinline__ double kernel_vjp(const PairGeo& G, d3 h, double r, const double c1[4],
                                             const double c2[4], const double cG[4],
                                             const double dc1[4], const double dc2[4],
                                             const double dcG[4], d3& gR, d3* gs, d3* gtx,
                                             d3& gn, d3* gty) {
  double V = 0.0, dVdr = 0.0;
  d3 gh = mk(0, 0, 0);
  gn = mk(0, 0, 0);
  for (int k = 0; k < 2; ++k) gs[k] = gtx[k] = gty[k] = mk(0, 0, 0);
  const double nh = dot(G.n, h);
  double sh[2], th[2], ht[2], nt[2];
  for (int a = 0; a < 2; ++a) {
    sh[a] = dot(G.s[a], h);
    th[a] = dot(G.t[a], h);
    ht[a] = dot(h, G.u[a]);
    nt[a] = dot(G.n, G.u[a]);
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int ab = 2 * a + b;
      const double st = dot(G.s[a], G.u[b]);
      const double tt = dot(G.t[a], G.u[b]);
      const double Gv = tt * nh - th[a] * nt[b];
      V += c1[ab] * st + c2[ab] * sh[a] * ht[b] + cG[ab] * Gv;
      dVdr += dc1[ab] * st + dc2[ab] * sh[a] * ht[b] + dcG[ab] * Gv;
      // d/dh
      gh = fma3(c2[ab] * ht[b], G.s[a], gh);
      gh = fma3(c2[ab] * sh[a], G.u[b], gh);
      gh = fma3(cG[ab] * tt, G.n, gh);
      gh = fma3(-cG[ab] * nt[b], G.t[a], gh);
      // d/ds_a(x)
      gs[a] = fma3(c1[ab], G.u[b], gs[a]);
      gs[a] = fma3(c2[ab] * ht[b], h, gs[a]);
      // d/dt_a(x)
      gtx[a] = fma3(cG[ab] * nh, G.u[b], gtx[a]);
      gtx[a] = fma3(-cG[ab] * nt[b], h, gtx[a]);
      // d/dn(x)
      gn = fma3(cG[ab] * tt, h, gn);
      gn = fma3(-cG[ab] * th[a], G.u[b], gn);
      // d/dt_b(y)
      gty[b] = fma3(c1[ab], G.s[a], gty[b]);
      gty[b] = fma3(c2[ab] * sh[a], h, gty[b]);
      gty[b] = fma3(cG[ab] * nh, G.t[a], gty[b]);
      gty[b] = fma3(-cG[ab] * th[a], G.n, gty[b]);
    }
  // dh/dR = (I - h h^T)/r
  const double hg = dot(h, gh);
  gR = add(scl(dVdr, h), scl(1.0 / r, sub(gh, scl(hg, h))));
  return V;
}

// ------------------------------------------------- lam, x at the rule points
// Lp[e][p][2h + a] = sum_i conj(lam[h H + 2 T[e][i] + a]) N_i(p);
// Xp[e][p][2g + b] = sum_j x[g H + 2 T[e][j] + b] N_j(p).
__global__ void pt_fields_kernel(int64_t nt, RuleC rule, const int32_t* __restrict__ T,
                                 const double2* __restrict__ lam, const double2* __restrict__ x,
                                 int64_t H, double2* __restrict__ Lp, double2* __restrict__ Xp) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt * rule.Q) return;
  const int64_t e = t / rule.Q;
  const int p = (int)(t % rule.Q);
  double N[6];
  p2N(rule.xi[p], rule.eta[p], N);
  double2 L[4] = {}, X[4] = {};
  for (int i = 0; i < 6; ++i) {
    const int64_t node = T[6 * e + i];
    for (int h = 0; h < 2; ++h)
      for (int a = 0; a < 2; ++a) {
        const int64_t u = h * H + 2 * node + a;
        const double2 l = lam[u], v = x[u];
        L[2 * h + a].x += N[i] * l.x;
        L[2 * h + a].y -= N[i] * l.y;  // conjugate
        X[2 * h + a].x += N[i] * v.x;
        X[2 * h + a].y += N[i] * v.y;
      }
  }
  for (int k = 0; k < 4; ++k) {
    Lp[t * 4 + k] = L[k];
    Xp[t * 4 + k] = X[k];
  }
}

__device__ __forceinline__ bool share_corner_d(const int32_t* a, const int32_t* b) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (a[i] == b[j]) return true;
  return false;
}

// coefficients of the 12 kernel components of a point pair:
// A1[ab] multiplies K1_ab W (rows Z00 with i/omega and Z11 = -Z00),
// Ae[ab] K2eps_ab W (Z01), Am[ab] K2mu_ab W (Z10)
__device__ __forceinline__ void pair_coef(const double2* L, const double2* X, double iw,
                                          cx<double> A1[4], cx<double> Ae[4], cx<double> Am[4]) {
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const cx<double> l0 = cmk(L[a].x, L[a].y), l1 = cmk(L[2 + a].x, L[2 + a].y);
      const cx<double> x0 = cmk(X[b].x, X[b].y), x1 = cmk(X[2 + b].x, X[2 + b].y);
      const cx<double> d = csub(cmul(l0, x0), cmul(l1, x1));
      A1[2 * a + b] = cmk(-iw * d.im, iw * d.re);  // (i/omega) d
      Ae[2 * a + b] = cmul(l0, x1);
      Am[2 * a + b] = cmul(l1, x0);
    }
}

// One point pair (p of the test element, q of the trial element) of
// Re lam^H Z x: value and gradient with respect to the test-point record
// (SIDE 0) or the trial-point record (SIDE 1), added into g[19]
// (x 0-2, n 3-5, t1 6-8, t2 9-11, s1 12-14, s2 15-17, W 18).
template <int SIDE>
__device__ void pair_point_vjp(const KConst<double>& K, const double* px, const double* qy,
                               bool remainder, const cx<double> A1[4], const cx<double> Ae[4],
                               const cx<double> Am[4], double* g) {
  const d3 R = sub(ld3(px), ld3(qy));
  const double r2 = dot(R, R);
  const double Wp = px[18], Wq = qy[18], W = Wp * Wq;
  PairGeo G;
  G.n = ld3(px + 3);
  for (int a = 0; a < 2; ++a) {
    G.t[a] = ld3(px + 6 + 3 * a);
    G.s[a] = ld3(px + 12 + 3 * a);
    G.u[a] = ld3(qy + 6 + 3 * a);
  }
  if (r2 == 0.0) {
    // coincident rule points (remainder): kappa1 - kappa1^s -> lim s.t
    const double ka3 = K.ka * K.ka * K.ka;
    const cx<double> ki2 = cmk(K.ki_re * K.ki_re - K.ki_im * K.ki_im, 2.0 * K.ki_re * K.ki_im);
    const cx<double> ki3 = cmul(ki2, cmk(K.ki_re, K.ki_im));
    const double inv6pi = 1.0 / (6.0 * kPi);
    const cx<double> lim = cmk(ki3.im * inv6pi, (ka3 - ki3.re) * inv6pi);
    double V = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const double c = cmul(A1[2 * a + b], lim).re;
        const double st = dot(G.s[a], G.u[b]);
        V += c * st;
        if (SIDE == 0)
          acc3s(g + 12 + 3 * a, c * W, G.u[b]);
        else
          acc3s(g + 6 + 3 * b, c * W, G.s[a]);
      }
    g[18] += V * (SIDE == 0 ? Wq : Wp);
    return;
  }
  const double r = sqrt(r2);
  const d3 h = scl(1.0 / r, R);
  cx<double> f[4], df[4];
  radial_d(K, r, remainder, f, df);
  double c1[4], c2[4], cG[4], dc1[4], dc2[4], dcG[4];
  for (int k = 0; k < 4; ++k) {
    c1[k] = cmul(A1[k], f[0]).re;
    c2[k] = cmul(A1[k], f[1]).re;
    cG[k] = cmul(Ae[k], f[2]).re + cmul(Am[k], f[3]).re;
    dc1[k] = cmul(A1[k], df[0]).re;
    dc2[k] = cmul(A1[k], df[1]).re;
    dcG[k] = cmul(Ae[k], df[2]).re + cmul(Am[k], df[3]).re;
  }
  d3 gR, gs[2], gtx[2], gn, gty[2];
  const double V = kernel_vjp(G, h, r, c1, c2, cG, dc1, dc2, dcG, gR, gs, gtx, gn, gty);
  if (SIDE == 0) {
    acc3s(g, W, gR);
    acc3s(g + 3, W, gn);
    for (int a = 0; a < 2; ++a) {
      acc3s(g + 6 + 3 * a, W, gtx[a]);
      acc3s(g + 12 + 3 * a, W, gs[a]);
    }
    g[18] += V * Wq;
  } else {
    acc3s(g, -W, gR);
    for (int b = 0; b < 2; ++b) acc3s(g + 6 + 3 * b, W, gty[b]);
    g[18] += V * Wp;
  }
}

// Regular pairs and the remainder of touching pairs, SIDE 0: CTA per test
// element e, warp w <-> test point w, lanes over the trial elements; SIDE 1:
// CTA per trial element, warp <-> trial point, lanes over test elements.
// The point-record adjoints of the CTA's element are added into radj.
template <int SIDE>
__global__ void __launch_bounds__(32 * MAX_Q) pair_vjp_kernel(
    int64_t nt, int Q, const double* __restrict__ qd, const int32_t* __restrict__ T,
    const double2* __restrict__ Lp, const double2* __restrict__ Xp, KConst<double> K,
    double* __restrict__ radj) {
  const int64_t e = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= Q) return;
  const double* own = qd + (e * Q + w) * QD_STRIDE;
  double rec[19];
  for (int c = 0; c < 19; ++c) rec[c] = own[c];
  int32_t te[3];
  for (int k = 0; k < 3; ++k) te[k] = T[6 * e + k];
  const double2* Lown = Lp + (e * Q + w) * 4;
  const double2* Xown = Xp + (e * Q + w) * 4;
  double2 Lo[4], Xo[4];
  for (int k = 0; k < 4; ++k) {
    Lo[k] = Lown[k];
    Xo[k] = Xown[k];
  }
  const double iw = 1.0 / K.ka;
  double g[19];
  for (int c = 0; c < 19; ++c) g[c] = 0.0;
  for (int64_t f = lane; f < nt; f += 32) {
    int32_t tf[3];
    for (int k = 0; k < 3; ++k) tf[k] = T[6 * f + k];
    const bool touch = share_corner_d(te, tf);
    for (int q = 0; q < Q; ++q) {
      const double* other = qd + (f * Q + q) * QD_STRIDE;
      cx<double> A1[4], Ae[4], Am[4];
      if (SIDE == 0) {
        pair_coef(Lo, Xp + (f * Q + q) * 4, iw, A1, Ae, Am);
        pair_point_vjp<0>(K, rec, other, touch, A1, Ae, Am, g);
      } else {
        pair_coef(Lp + (f * Q + q) * 4, Xo, iw, A1, Ae, Am);
        pair_point_vjp<1>(K, other, rec, touch, A1, Ae, Am, g);
      }
    }
  }
  for (int c = 0; c < 19; ++c) {
    double v = g[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) radj[(e * Q + w) * 19 + c] += v;
  }
}

// Mass term (Eq. mass_matrix; coincident pairs): Z01 += a_eps M, Z10 +=
// a_mu M with M_ij = sum_p W_p N_i N_j: the adjoint of W_p.
__global__ void mass_vjp_kernel(int64_t n, const double2* __restrict__ Lp,
                                const double2* __restrict__ Xp, double ae_re, double ae_im,
                                double am_re, double am_im, double* __restrict__ radj) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double2* L = Lp + t * 4;
  const double2* X = Xp + t * 4;
  const cx<double> ae = cmk(ae_re, ae_im), am = cmk(am_re, am_im);
  double v = 0.0;
  for (int a = 0; a < 2; ++a) {
    const cx<double> l0 = cmk(L[a].x, L[a].y), l1 = cmk(L[2 + a].x, L[2 + a].y);
    const cx<double> x0 = cmk(X[a].x, X[a].y), x1 = cmk(X[2 + a].x, X[2 + a].y);
    v += cmul(ae, cmul(l0, x1)).re + cmul(am, cmul(l1, x0)).re;
  }
  radj[t * 19 + 18] += v;
}

// ---------------------------------------------------- geometry reverse
// Adjoints of (x, n, t1, t2, J) of a point whose geometry is
//   x = P2(X), a1, a2 its derivatives, c = a1 x a2, J = |c|, n = c/J,
//   t1 = p1/|p1| with p1 = u1 - n (n.u1), u1 = P2(T1),
//   t2 = sig n x t1 (the Gram-Schmidt vector of u2; no dependence on T2)
// carried to the adjoints of x, a1, a2 and u1.
struct GeoRev {
  d3 gx, ga1, ga2, gu1;
};

__device__ GeoRev geo_reverse(d3 a1, d3 a2, d3 u1, d3 n, d3 t1, double J, double sig, d3 gx,
                              d3 gn, d3 gt1, d3 gt2, double gJ) {
  // t2 = sig (n x t1)
  const d3 gm = scl(sig, gt2);
  gn = add(gn, cross(t1, gm));
  gt1 = add(gt1, cross(gm, n));
  // t1 = p1/|p1|, p1 = u1 - n (n.u1)
  const double nu = dot(n, u1);
  const d3 p1 = sub(u1, scl(nu, n));
  const double ip = 1.0 / sqrt(dot(p1, p1));
  const d3 gp = scl(ip, sub(gt1, scl(dot(t1, gt1), t1)));
  const double ngp = dot(n, gp);
  GeoRev o;
  o.gu1 = sub(gp, scl(ngp, n));
  gn = sub(gn, add(scl(nu, gp), scl(ngp, u1)));
  // n = c/J, J = |c|
  const d3 gc = add(scl(1.0 / J, sub(gn, scl(dot(n, gn), n))), scl(gJ, n));
  o.ga1 = cross(a2, gc);
  o.ga2 = cross(gc, a1);
  o.gx = gx;
  return o;
}

// Regular-rule point records -> element inputs: eadj[e][0..17] node
// positions, [18..35] nodal t1, [36..53] nodal t2 (zero: see geo_reverse).
// The records' s_a = t_a x n and W = w J fold into the adjoints of t, n, J.
__global__ void rec_backprop_kernel(int64_t nt, RuleC rule, const double* __restrict__ X,
                                    const int32_t* __restrict__ T,
                                    const double* __restrict__ frame,
                                    const double* __restrict__ qd,
                                    const double* __restrict__ radj, double* __restrict__ eadj) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt * rule.Q) return;
  const int64_t e = t / rule.Q;
  const int p = (int)(t % rule.Q);
  double N[6], dxi[6], deta[6];
  p2_eval(rule.xi[p], rule.eta[p], N, dxi, deta);
  d3 a1 = mk(0, 0, 0), a2 = mk(0, 0, 0), u1 = mk(0, 0, 0), u2 = mk(0, 0, 0);
  for (int k = 0; k < 6; ++k) {
    const int64_t v = T[6 * e + k];
    const d3 xv = mk(X[3 * v], X[3 * v + 1], X[3 * v + 2]);
    a1 = fma3(dxi[k], xv, a1);
    a2 = fma3(deta[k], xv, a2);
    u1 = fma3(N[k], ld3(frame + 9 * v + 3), u1);
    u2 = fma3(N[k], ld3(frame + 9 * v + 6), u2);
  }
  const double* rc = qd + t * QD_STRIDE;
  const double* ga = radj + t * 19;
  const d3 n = ld3(rc + 3), t1 = ld3(rc + 6), t2 = ld3(rc + 9);
  const double J = rc[18] / rule.w[p];
  const double sig = dot(cross(n, t1), u2) < 0.0 ? -1.0 : 1.0;
  d3 gn = ld3(ga + 3), gt1 = ld3(ga + 6), gt2 = ld3(ga + 9);
  // s_a = t_a x n
  const d3 gs1 = ld3(ga + 12), gs2 = ld3(ga + 15);
  gt1 = add(gt1, cross(n, gs1));
  gn = add(gn, cross(gs1, t1));
  gt2 = add(gt2, cross(n, gs2));
  gn = add(gn, cross(gs2, t2));
  const double gJ = ga[18] * rule.w[p];
  const GeoRev o = geo_reverse(a1, a2, u1, n, t1, J, sig, ld3(ga), gn, gt1, gt2, gJ);
  double* out = eadj + e * 54;
  for (int k = 0; k < 6; ++k) {
    const d3 gX = add(scl(N[k], o.gx), add(scl(dxi[k], o.ga1), scl(deta[k], o.ga2)));
    const d3 gT = scl(N[k], o.gu1);
    atomicAdd(out + 3 * k, gX.x);
    atomicAdd(out + 3 * k + 1, gX.y);
    atomicAdd(out + 3 * k + 2, gX.z);
    atomicAdd(out + 18 + 3 * k, gT.x);
    atomicAdd(out + 18 + 3 * k + 1, gT.y);
    atomicAdd(out + 18 + 3 * k + 2, gT.z);
  }
}

// ----------------------------------------------------- Sauter-Schwab part
// Singular parts of the touching pairs (Eqs. kappa_S, kappa2_S): with the
// interpolated lam (test point) and x (trial point) at every Sauter-Schwab
// point pair, V = w J_x J_y sum_c Re(gamma_c) g_c, g the 8 geometric kernels.
// One CTA per touching pair; SIDE 0 carries the adjoints to the test
// element's monomial coefficients, SIDE 1 to the trial element's; at the end
// they go to the nodal values (transpose of p2_coef) and into eadj.
constexpr int SST = 128;

__device__ __forceinline__ void mono6(double xi, double eta, double m[6]) {
  m[0] = 1.0;
  m[1] = xi;
  m[2] = eta;
  m[3] = xi * xi;
  m[4] = xi * eta;
  m[5] = eta * eta;
}

struct SSPoint {
  d3 x, a1, a2, u1, n, t1, t2;
  double J, sig;
  double N[6];
};

__device__ __forceinline__ void ss_point_geo(const d3* CX, const d3* CU1, const d3* CU2,
                                             double xi, double eta, SSPoint& g) {
  p2N(xi, eta, g.N);
  g.x = p2_val(CX, xi, eta);
  g.a1 = fma3(2.0 * xi, CX[3], fma3(eta, CX[4], CX[1]));
  g.a2 = fma3(xi, CX[4], fma3(2.0 * eta, CX[5], CX[2]));
  const d3 c = cross(g.a1, g.a2);
  g.J = sqrt(dot(c, c));
  g.n = scl(1.0 / g.J, c);
  g.u1 = p2_val(CU1, xi, eta);
  const d3 p1 = sub(g.u1, scl(dot(g.n, g.u1), g.n));
  g.t1 = scl(1.0 / sqrt(dot(p1, p1)), p1);
  const d3 m = cross(g.n, g.t1);
  g.sig = dot(m, p2_val(CU2, xi, eta)) < 0.0 ? -1.0 : 1.0;
  g.t2 = scl(g.sig, m);
}

template <int SIDE>
__global__ void __launch_bounds__(SST) ss_vjp_kernel(
    const TouchPair* __restrict__ tp, const double* __restrict__ X, const int32_t* __restrict__ T,
    const double* __restrict__ frame, const double2* __restrict__ lam,
    const double2* __restrict__ xv, int64_t H, GLC gl, cx<double> c1, cx<double> ce,
    cx<double> cm, double iw, double* __restrict__ eadj) {
  __shared__ d3 sC[2][3][6];  // [side][X, T1, T2][monomial]
  __shared__ double2 sL[6][4], sXv[6][4];  // conj lam at the test nodes, x at the trial nodes
  const TouchPair P = tp[blockIdx.x];
  const int tid = threadIdx.x;
  if (tid < 18) {
    const int side = tid / 9, fld = (tid / 3) % 3, k0 = (tid % 3) * 2;
    const int64_t e = side ? P.ey : P.ex;
    for (int k = k0; k < k0 + 2; ++k) {
      const int64_t v = T[6 * e + k];
      sC[side][fld][k] = fld == 0 ? mk(X[3 * v], X[3 * v + 1], X[3 * v + 2])
                                  : ld3(frame + 9 * v + 3 * fld);
    }
  }
  if (tid >= 32 && tid < 32 + 24) {
    const int i = (tid - 32) / 4, k = (tid - 32) % 4;  // k = 2h + a
    const int h = k >> 1, a = k & 1;
    const double2 l = lam[h * H + 2 * (int64_t)T[6 * P.ex + i] + a];
    sL[i][k] = make_double2(l.x, -l.y);
    sXv[i][k] = xv[h * H + 2 * (int64_t)T[6 * P.ey + i] + a];
  }
  __syncthreads();
  if (tid < 6) {
    const int side = tid / 3, fld = tid % 3;
    d3 v[6], c[6];
    for (int k = 0; k < 6; ++k) v[k] = sC[side][fld][k];
    p2_coef(v, c);
    for (int k = 0; k < 6; ++k) sC[side][fld][k] = c[k];
  }
  __syncthreads();
  const int px = P.perm & 0x3f, py = (P.perm >> 8) & 0x3f;
  const int nreg = P.cls == 3 ? 6 : (P.cls == 2 ? 5 : 2);
  const int ns = gl.ns;
  const int64_t npts = (int64_t)nreg * ns * ns * ns * ns;
  double acc[36];
  for (int k = 0; k < 36; ++k) acc[k] = 0.0;
  for (int64_t pt = tid; pt < npts; pt += SST) {
    double xu, xvv, yu, yv, w;
    ss_point(P.cls, ns, pt, gl.x, gl.w, xu, xvv, yu, yv, w);
    double xi, eta, yxi, yeta;
    to_canonical(px, xu, xvv, xi, eta);
    to_canonical(py, yu, yv, yxi, yeta);
    SSPoint gx, gy;
    ss_point_geo(sC[0][0], sC[0][1], sC[0][2], xi, eta, gx);
    ss_point_geo(sC[1][0], sC[1][1], sC[1][2], yxi, yeta, gy);
    // gamma_c from lam (test side) and x (trial side) at the points
    cx<double> Lx[4], Xy[4];
    for (int k = 0; k < 4; ++k) {
      Lx[k] = cmk(0.0, 0.0);
      Xy[k] = cmk(0.0, 0.0);
      for (int i = 0; i < 6; ++i) {
        Lx[k].re += gx.N[i] * sL[i][k].x;
        Lx[k].im += gx.N[i] * sL[i][k].y;
        Xy[k].re += gy.N[i] * sXv[i][k].x;
        Xy[k].im += gy.N[i] * sXv[i][k].y;
      }
    }
    double c1v[4], c2v[4], cGv[4], d1v[4], d2v[4], dGv[4];
    const d3 R = sub(gx.x, gy.x);
    const double r = sqrt(dot(R, R));
    const d3 h = scl(1.0 / r, R);
    const double ir = 1.0 / r, ir2 = ir * ir;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const int ab = 2 * a + b;
        const cx<double> d = csub(cmul(Lx[a], Xy[b]), cmul(Lx[2 + a], Xy[2 + b]));
        const cx<double> g1 = cmul(c1, cmk(-iw * d.im, iw * d.re));
        const double G2 = cmul(ce, cmul(Lx[a], Xy[2 + b])).re + cmul(cm, cmul(Lx[2 + a], Xy[b])).re;
        c1v[ab] = g1.re * ir;
        c2v[ab] = g1.re * ir;
        cGv[ab] = G2 * ir2;
        d1v[ab] = -g1.re * ir2;
        d2v[ab] = -g1.re * ir2;
        dGv[ab] = -2.0 * G2 * ir2 * ir;
      }
    PairGeo G;
    G.n = gx.n;
    G.t[0] = gx.t1;
    G.t[1] = gx.t2;
    G.s[0] = scl(-gx.sig, gx.t2);  // s1 = t1 x n = -sig t2
    G.s[1] = scl(gx.sig, gx.t1);   // s2 = t2 x n = sig t1
    G.u[0] = gy.t1;
    G.u[1] = gy.t2;
    d3 gR, gs[2], gtx[2], gn, gty[2];
    const double V = kernel_vjp(G, h, r, c1v, c2v, cGv, d1v, d2v, dGv, gR, gs, gtx, gn, gty);
    const double Wt = w * gx.J * gy.J;
    GeoRev o;
    double m[6];
    if (SIDE == 0) {
      // s1 = -sig t2, s2 = sig t1
      d3 gt1 = add(scl(Wt, gtx[0]), scl(Wt * gx.sig, gs[1]));
      d3 gt2 = add(scl(Wt, gtx[1]), scl(-Wt * gx.sig, gs[0]));
      o = geo_reverse(gx.a1, gx.a2, gx.u1, gx.n, gx.t1, gx.J, gx.sig, scl(Wt, gR), scl(Wt, gn),
                      gt1, gt2, V * w * gy.J);
      mono6(xi, eta, m);
    } else {
      o = geo_reverse(gy.a1, gy.a2, gy.u1, gy.n, gy.t1, gy.J, gy.sig, scl(-Wt, gR), mk(0, 0, 0),
                      scl(Wt, gty[0]), scl(Wt, gty[1]), V * w * gx.J);
      mono6(yxi, yeta, m);
    }
    // x = sum m_k CX_k, a1 = CX1 + 2 xi CX3 + eta CX4, a2 = CX2 + xi CX4 + 2 eta CX5
    const double s = SIDE == 0 ? xi : yxi, t = SIDE == 0 ? eta : yeta;
    d3 gC[6];
    for (int k = 0; k < 6; ++k) gC[k] = scl(m[k], o.gx);
    gC[1] = add(gC[1], o.ga1);
    gC[3] = add(gC[3], scl(2.0 * s, o.ga1));
    gC[4] = add(gC[4], add(scl(t, o.ga1), scl(s, o.ga2)));
    gC[2] = add(gC[2], o.ga2);
    gC[5] = add(gC[5], scl(2.0 * t, o.ga2));
    for (int k = 0; k < 6; ++k) {
      acc[3 * k] += gC[k].x;
      acc[3 * k + 1] += gC[k].y;
      acc[3 * k + 2] += gC[k].z;
      acc[18 + 3 * k] += m[k] * o.gu1.x;
      acc[18 + 3 * k + 1] += m[k] * o.gu1.y;
      acc[18 + 3 * k + 2] += m[k] * o.gu1.z;
    }
  }
  // CTA sums of the 36 monomial-coefficient adjoints: warp sums, then the
  // SST / 32 warps' partials
  __shared__ double wsum[SST / 32][36];
  __shared__ double sum[36];
  const int lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < 36; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[warp][k] = v;
  }
  __syncthreads();
  if (tid < 36) {
    double v = 0.0;
    for (int q = 0; q < SST / 32; ++q) v += wsum[q][tid];
    sum[tid] = v;
  }
  __syncthreads();
  // monomial coefficients c = P v (p2_coef) -> nodal values: adj v = P^T adj c
  if (tid < 6) {
    const int fld = tid / 3, d = tid % 3;  // fld 0: positions, 1: nodal t1
    double gc[6], gv[6];
    for (int k = 0; k < 6; ++k) gc[k] = sum[18 * fld + 3 * k + d];
    gv[0] = gc[0] - 3.0 * gc[1] - 3.0 * gc[2] + 2.0 * gc[3] + 4.0 * gc[4] + 2.0 * gc[5];
    gv[1] = -gc[1] + 2.0 * gc[3];
    gv[2] = -gc[2] + 2.0 * gc[5];
    gv[3] = 4.0 * gc[1] - 4.0 * gc[3] - 4.0 * gc[4];
    gv[4] = 4.0 * gc[4];
    gv[5] = 4.0 * gc[2] - 4.0 * gc[4] - 4.0 * gc[5];
    const int64_t e = SIDE == 0 ? P.ex : P.ey;
    for (int k = 0; k < 6; ++k) atomicAdd(eadj + e * 54 + 18 * fld + 3 * k + d, gv[k]);
  }
}

// ------------------------------------------------------ frame reverse
// Per node: the nodal-frame adjoints gathered from the node's elements, the
// reverse of t1 = v_ref x n/|.|, t2 = n x t1 (Sec. 3.2) to the nodal normal,
// of n = U/|U| to U, and of each element's U = a1 x a2/(g11 g22) (Sec. 3.1)
// to the element's node positions (atomic adds into gpos); the position
// adjoints gathered from the elements are added too.
__global__ void frame_backprop_kernel(int64_t nn, const double* __restrict__ X,
                                      const int32_t* __restrict__ T,
                                      const int32_t* __restrict__ ptr,
                                      const int32_t* __restrict__ n2e, int frame_rule,
                                      const double* __restrict__ frame,
                                      const double* __restrict__ eadj, double* __restrict__ gpos) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double px[6] = {0.0, 1.0, 0.0, 0.5, 0.5, 0.0};
  const double py[6] = {0.0, 0.0, 1.0, 0.0, 0.5, 0.5};
  d3 gt1 = mk(0, 0, 0), gt2 = mk(0, 0, 0), gp = mk(0, 0, 0);
  for (int32_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int32_t e = n2e[q] >> 3, k = n2e[q] & 7;
    gp = add(gp, ld3(eadj + (int64_t)e * 54 + 3 * k));
    gt1 = add(gt1, ld3(eadj + (int64_t)e * 54 + 18 + 3 * k));
    gt2 = add(gt2, ld3(eadj + (int64_t)e * 54 + 36 + 3 * k));
  }
  atomicAdd(gpos + 3 * i, gp.x);
  atomicAdd(gpos + 3 * i + 1, gp.y);
  atomicAdd(gpos + 3 * i + 2, gp.z);
  const d3 n = ld3(frame + 9 * i), t1 = ld3(frame + 9 * i + 3);
  // t2 = n x t1
  d3 gn = cross(t1, gt2);
  gt1 = add(gt1, cross(gt2, n));
  // t1 = c/|c|, c = v_ref x n
  d3 ref;
  if (frame_rule == 1)
    ref = (fabs(n.z) > 1.0 - 1e-8) ? mk(1, 0, 0) : mk(0, 0, 1);
  else
    ref = (fabs(n.z) > 0.9) ? mk(1, 0, 0) : mk(0, 0, 1);
  const d3 c = cross(ref, n);
  const double ic = 1.0 / sqrt(dot(c, c));
  const d3 gc = scl(ic, sub(gt1, scl(dot(t1, gt1), t1)));
  gn = add(gn, cross(gc, ref));
  // n = U/|U|: recompute U
  d3 U = mk(0, 0, 0);
  for (int32_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int32_t e = n2e[q] >> 3, k = n2e[q] & 7;
    double N[6], dxi[6], deta[6];
    p2_eval(px[k], py[k], N, dxi, deta);
    d3 A = mk(0, 0, 0), B = mk(0, 0, 0);
    for (int j = 0; j < 6; ++j) {
      const d3 xj = ld3(X + 3 * (int64_t)T[6 * (int64_t)e + j]);
      A = fma3(dxi[j], xj, A);
      B = fma3(deta[j], xj, B);
    }
    d3 a1, a2;
    if (k == 1) {
      a1 = sub(B, A);
      a2 = scl(-1.0, A);
    } else if (k == 2) {
      a1 = scl(-1.0, B);
      a2 = sub(A, B);
    } else {
      a1 = A;
      a2 = B;
    }
    U = add(U, scl(1.0 / (dot(a1, a1) * dot(a2, a2)), cross(a1, a2)));
  }
  const double iu = 1.0 / sqrt(dot(U, U));
  const d3 gU = scl(iu, sub(gn, scl(dot(n, gn), n)));
  // each element's U_e = w (a1 x a2), w = 1/(g11 g22)
  for (int32_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int32_t e = n2e[q] >> 3, k = n2e[q] & 7;
    double N[6], dxi[6], deta[6];
    p2_eval(px[k], py[k], N, dxi, deta);
    d3 A = mk(0, 0, 0), B = mk(0, 0, 0);
    for (int j = 0; j < 6; ++j) {
      const d3 xj = ld3(X + 3 * (int64_t)T[6 * (int64_t)e + j]);
      A = fma3(dxi[j], xj, A);
      B = fma3(deta[j], xj, B);
    }
    d3 a1, a2;
    if (k == 1) {
      a1 = sub(B, A);
      a2 = scl(-1.0, A);
    } else if (k == 2) {
      a1 = scl(-1.0, B);
      a2 = sub(A, B);
    } else {
      a1 = A;
      a2 = B;
    }
    const double g11 = dot(a1, a1), g22 = dot(a2, a2), w = 1.0 / (g11 * g22);
    const d3 cr = cross(a1, a2);
    const double uc = dot(gU, cr);
    // d(w cr) = w (da1 x a2 + a1 x da2) - w cr (2 a1.da1/g11 + 2 a2.da2/g22)
    const d3 ga1 = sub(scl(w, cross(a2, gU)), scl(2.0 * w * uc / g11, a1));
    const d3 ga2 = sub(scl(w, cross(gU, a1)), scl(2.0 * w * uc / g22, a2));
    d3 gA, gB;
    if (k == 1) {  // a1 = B - A, a2 = -A
      gA = scl(-1.0, add(ga1, ga2));
      gB = ga1;
    } else if (k == 2) {  // a1 = -B, a2 = A - B
      gA = ga2;
      gB = scl(-1.0, add(ga1, ga2));
    } else {
      gA = ga1;
      gB = ga2;
    }
    for (int j = 0; j < 6; ++j) {
      const d3 gj = add(scl(dxi[j], gA), scl(deta[j], gB));
      const int64_t v = T[6 * (int64_t)e + j];
      atomicAdd(gpos + 3 * v, gj.x);
      atomicAdd(gpos + 3 * v + 1, gj.y);
      atomicAdd(gpos + 3 * v + 2, gj.z);
    }
  }
}

inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// ----------------------------------------------------------- drivers
// Shared workspace: point fields, record adjoints, element adjoints.
struct ShapeWork {
  double2 *Lp = nullptr, *Xp = nullptr;
  double *radj = nullptr, *eadj = nullptr, *gpos = nullptr;
};

static mueller_status shape_alloc(mueller_mesh* m, int Q, ShapeWork& W, cudaStream_t s) {
  const int64_t np = m->nt * Q;
  MU_CUDA(cudaMallocAsync((void**)&W.Lp, (size_t)np * 4 * sizeof(double2), s));
  MU_CUDA(cudaMallocAsync((void**)&W.Xp, (size_t)np * 4 * sizeof(double2), s));
  MU_CUDA(cudaMallocAsync((void**)&W.radj, (size_t)np * 19 * sizeof(double), s));
  MU_CUDA(cudaMallocAsync((void**)&W.eadj, (size_t)m->nt * 54 * sizeof(double), s));
  MU_CUDA(cudaMallocAsync((void**)&W.gpos, (size_t)m->nn * 3 * sizeof(double), s));
  MU_CUDA(cudaMemsetAsync(W.radj, 0, (size_t)np * 19 * sizeof(double), s));
  MU_CUDA(cudaMemsetAsync(W.eadj, 0, (size_t)m->nt * 54 * sizeof(double), s));
  MU_CUDA(cudaMemsetAsync(W.gpos, 0, (size_t)m->nn * 3 * sizeof(double), s));
  return MUELLER_OK;
}

static void shape_free(ShapeWork& W, cudaStream_t s) {
  for (void* p : {(void*)W.Lp, (void*)W.Xp, (void*)W.radj, (void*)W.eadj, (void*)W.gpos})
    if (p) cudaFreeAsync(p, s);
}

static RuleC rule_c(const TriangleRule& rule) {
  RuleC rc;
  rc.Q = rule.q;
  for (int p = 0; p < rule.q; ++p) {
    rc.xi[p] = rule.xi[p];
    rc.eta[p] = rule.eta[p];
    rc.w[p] = rule.w[p];
  }
  return rc;
}

// records -> element inputs -> node positions; the result (node order of the
// mesh's input) into grad (host, nn x 3), added to what is there
static mueller_status shape_finish(mueller_mesh* m, const RuleC& rc, ShapeWork& W, double* grad,
                                   cudaStream_t s) {
  { Prof prof_("rec_backprop_kernel", s); rec_backprop_kernel<<<nblk(m->nt * rc.Q, 128), 128, 0, s>>>(m->nt, rc, m->X, m->T, m->frame, m->qd64, W.radj, W.eadj); }
  MU_CHECK_LAUNCH("rec_backprop_kernel");
  { Prof prof_("frame_backprop_kernel", s); frame_backprop_kernel<<<nblk(m->nn, 128), 128, 0, s>>>(m->nn, m->X, m->T, m->n2e_ptr, m->n2e, m->frame_rule, m->frame, W.eadj, W.gpos); }
  MU_CHECK_LAUNCH("frame_backprop_kernel");
  std::vector<double> g((size_t)m->nn * 3);
  MU_CUDA(cudaMemcpyAsync(g.data(), W.gpos, g.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  MU_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < m->nn; ++i)
    for (int d = 0; d < 3; ++d) grad[3 * (int64_t)m->node_perm[i] + d] += g[3 * i + d];
  return MUELLER_OK;
}

mueller_status zshape_vjp(mueller_mesh* m, const PhysConsts& P, int Q, int ns, const void* lam,
                          const void* x, double* grad, cudaStream_t s) {
  TriangleRule rule;
  if (!triangle_rule(Q, rule)) {
    set_error("q_regular must be 6 or 12");
    return MUELLER_ERR_INVALID_ARG;
  }
  const RuleC rc = rule_c(rule);
  ShapeWork W;
  mueller_status st = shape_alloc(m, Q, W, s);
  const int64_t N = 4 * m->nn, H = N / 2;
  KConst<double> K;
  K.ka = P.ka;
  K.ki_re = P.ki_re;
  K.ki_im = P.ki_im;
  K.eps_re = P.eps_re;
  K.eps_im = P.eps_im;
  K.mu_re = P.mu_re;
  K.mu_im = P.mu_im;
  K.sing = 0.0;
  if (!st) {
    { Prof prof_("pt_fields_kernel", s); pt_fields_kernel<<<nblk(m->nt * Q, 128), 128, 0, s>>>(m->nt, rc, m->T, (const double2*)lam, (const double2*)x, H, W.Lp, W.Xp); }
    { Prof prof_("pair_vjp_kernel<0>", s); pair_vjp_kernel<0><<<(unsigned)m->nt, 32 * Q, 0, s>>>(m->nt, Q, m->qd64, m->T, W.Lp, W.Xp, K, W.radj); }
    { Prof prof_("pair_vjp_kernel<1>", s); pair_vjp_kernel<1><<<(unsigned)m->nt, 32 * Q, 0, s>>>(m->nt, Q, m->qd64, m->T, W.Lp, W.Xp, K, W.radj); }
    { Prof prof_("mass_vjp_kernel", s); mass_vjp_kernel<<<nblk(m->nt * Q, 128), 128, 0, s>>>(m->nt * Q, W.Lp, W.Xp, 0.5 * (1.0 + P.eps_re), 0.5 * P.eps_im, 0.5 * (1.0 + P.mu_re), 0.5 * P.mu_im, W.radj); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "pair adjoint kernels");
  }
  if (!st && m->n_touch > 0) {
    GLC gl;
    std::vector<double> gx, gw;
    gauss_legendre_unit(ns, gx, gw);
    gl.ns = ns;
    for (int k = 0; k < ns; ++k) {
      gl.x[k] = gx[k];
      gl.w[k] = gw[k];
    }
    const cx<double> ki2 = cmk(P.ki_re * P.ki_re - P.ki_im * P.ki_im, 2.0 * P.ki_re * P.ki_im);
    const cx<double> c1 = crs(1.0 / (8.0 * kPi), cmk(P.ka * P.ka - ki2.re, -ki2.im));
    const cx<double> ce = crs(-kC4pi, cmk(1.0 - P.eps_re, -P.eps_im));
    const cx<double> cm = crs(-kC4pi, cmk(1.0 - P.mu_re, -P.mu_im));
    { Prof prof_("ss_vjp_kernel<0>", s); ss_vjp_kernel<0><<<(unsigned)m->n_touch, SST, 0, s>>>(m->tp, m->X, m->T, m->frame, (const double2*)lam, (const double2*)x, H, gl, c1, ce, cm, 1.0 / P.ka, W.eadj); }
    { Prof prof_("ss_vjp_kernel<1>", s); ss_vjp_kernel<1><<<(unsigned)m->n_touch, SST, 0, s>>>(m->tp, m->X, m->T, m->frame, (const double2*)lam, (const double2*)x, H, gl, c1, ce, cm, 1.0 / P.ka, W.eadj); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "Sauter-Schwab adjoint kernels");
  }
  if (!st) st = shape_finish(m, rc, W, grad, s);
  shape_free(W, s);
  return st;
}

}  // namespace mu
