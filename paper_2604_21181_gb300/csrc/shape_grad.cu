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

#include <algorithm>
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
// Re lam_o^H Z x for R adjoint vectors lam_o: value and gradient with respect
// to the test-point record (SIDE 0) or the trial-point record (SIDE 1), added
// into g[o][19] (x 0-2, n 3-5, t1 6-8, t2 9-11, s1 12-14, s2 15-17, W 18).
// Lt[o]: the 4 fields of conj(lam_o) at the test point, Xq: those of x at
// the trial point.  The radial functions and their derivatives, which do not
// depend on lam, are evaluated once for the R vectors.
template <int SIDE, int R>
__device__ void pair_point_vjp(const KConst<double>& K, const double* px, const double* qy,
                               bool remainder, const double2* const* Lt, const double2* Xq,
                               double iw, double (*g)[19]) {
  const d3 Rv = sub(ld3(px), ld3(qy));
  const double r2 = dot(Rv, Rv);
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
    for (int o = 0; o < R; ++o) {
      cx<double> A1[4], Ae[4], Am[4];
      pair_coef(Lt[o], Xq, iw, A1, Ae, Am);
      double V = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const double c = cmul(A1[2 * a + b], lim).re;
          const double st = dot(G.s[a], G.u[b]);
          V += c * st;
          if (SIDE == 0)
            acc3s(g[o] + 12 + 3 * a, c * W, G.u[b]);
          else
            acc3s(g[o] + 6 + 3 * b, c * W, G.s[a]);
        }
      g[o][18] += V * (SIDE == 0 ? Wq : Wp);
    }
    return;
  }
  const double r = sqrt(r2);
  const d3 h = scl(1.0 / r, Rv);
  cx<double> f[4], df[4];
  radial_d(K, r, remainder, f, df);
#pragma unroll 1
  for (int o = 0; o < R; ++o) {
    cx<double> A1[4], Ae[4], Am[4];
    pair_coef(Lt[o], Xq, iw, A1, Ae, Am);
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
    double* go = g[o];
    if (SIDE == 0) {
      acc3s(go, W, gR);
      acc3s(go + 3, W, gn);
      for (int a = 0; a < 2; ++a) {
        acc3s(go + 6 + 3 * a, W, gtx[a]);
        acc3s(go + 12 + 3 * a, W, gs[a]);
      }
      go[18] += V * Wq;
    } else {
      acc3s(go, -W, gR);
      for (int b = 0; b < 2; ++b) acc3s(go + 6 + 3 * b, W, gty[b]);
      go[18] += V * Wp;
    }
  }
}

// The point-field and record-adjoint arrays of up to kVjpR adjoint vectors
// (one pt_fields / radj set per vector; x is the same for all of them).
constexpr int kVjpR = 3;
struct VjpSet {
  const double2* Lp[kVjpR];
  double* radj[kVjpR];
};

// Regular pairs and the remainder of touching pairs, SIDE 0: CTA per test
// element e, warp w <-> test point w, lanes over the trial elements; SIDE 1:
// CTA per trial element, warp <-> trial point, lanes over test elements.
// The point-record adjoints of the CTA's element are added into radj of
// each of the R adjoint vectors.
template <int SIDE, int R>
__global__ void __launch_bounds__(32 * MAX_Q) pair_vjp_kernel(
    int64_t nt, int Q, const double* __restrict__ qd, const int32_t* __restrict__ T,
    VjpSet V, const double2* __restrict__ Xp, KConst<double> K) {
  const int64_t e = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= Q) return;
  const double* own = qd + (e * Q + w) * QD_STRIDE;
  double rec[19];
  for (int c = 0; c < 19; ++c) rec[c] = own[c];
  int32_t te[3];
  for (int k = 0; k < 3; ++k) te[k] = T[6 * e + k];
  double2 Lo[R][4], Xo[4];
  for (int k = 0; k < 4; ++k) {
    Xo[k] = Xp[(e * Q + w) * 4 + k];
    for (int o = 0; o < R; ++o) Lo[o][k] = V.Lp[o][(e * Q + w) * 4 + k];
  }
  const double iw = 1.0 / K.ka;
  double g[R][19];
  for (int o = 0; o < R; ++o)
    for (int c = 0; c < 19; ++c) g[o][c] = 0.0;
  for (int64_t f = lane; f < nt; f += 32) {
    int32_t tf[3];
    for (int k = 0; k < 3; ++k) tf[k] = T[6 * f + k];
    const bool touch = share_corner_d(te, tf);
    for (int q = 0; q < Q; ++q) {
      const double* other = qd + (f * Q + q) * QD_STRIDE;
      const double2* Lt[R];
      for (int o = 0; o < R; ++o) Lt[o] = SIDE == 0 ? Lo[o] : V.Lp[o] + (f * Q + q) * 4;
      if (SIDE == 0)
        pair_point_vjp<0, R>(K, rec, other, touch, Lt, Xp + (f * Q + q) * 4, iw, g);
      else
        pair_point_vjp<1, R>(K, other, rec, touch, Lt, Xo, iw, g);
    }
  }
  for (int o = 0; o < R; ++o)
    for (int c = 0; c < 19; ++c) {
      double v = g[o][c];
      for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
      if (lane == 0) V.radj[o][(e * Q + w) * 19 + c] += v;
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

// R adjoint vectors per CTA (lam[o], eadj[o]): the two points' geometry and
// the trial-side field of x are evaluated once per point for all of them.
struct SsVjpSet {
  const double2* lam[kVjpR];
  double* eadj[kVjpR];
};

template <int SIDE, int R>
__global__ void __launch_bounds__(SST) ss_vjp_kernel(
    const TouchPair* __restrict__ tp, const double* __restrict__ X, const int32_t* __restrict__ T,
    const double* __restrict__ frame, SsVjpSet V, const double2* __restrict__ xv, int64_t H,
    GLC gl, cx<double> c1, cx<double> ce, cx<double> cm, double iw) {
  __shared__ d3 sC[2][3][6];  // [side][X, T1, T2][monomial]
  __shared__ double2 sL[R][6][4], sXv[6][4];  // conj lam at the test nodes, x at the trial nodes
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
    for (int o = 0; o < R; ++o) {
      const double2 l = V.lam[o][h * H + 2 * (int64_t)T[6 * P.ex + i] + a];
      sL[o][i][k] = make_double2(l.x, -l.y);
    }
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
  double acc[R][36];
  for (int o = 0; o < R; ++o)
    for (int k = 0; k < 36; ++k) acc[o][k] = 0.0;
  for (int64_t pt = tid; pt < npts; pt += SST) {
    double xu, xvv, yu, yv, w;
    ss_point(P.cls, ns, pt, gl.x, gl.w, xu, xvv, yu, yv, w);
    double xi, eta, yxi, yeta;
    to_canonical(px, xu, xvv, xi, eta);
    to_canonical(py, yu, yv, yxi, yeta);
    SSPoint gx, gy;
    ss_point_geo(sC[0][0], sC[0][1], sC[0][2], xi, eta, gx);
    ss_point_geo(sC[1][0], sC[1][1], sC[1][2], yxi, yeta, gy);
    // x (trial side) at the point; lam (test side) per vector below
    cx<double> Xy[4];
    for (int k = 0; k < 4; ++k) {
      Xy[k] = cmk(0.0, 0.0);
      for (int i = 0; i < 6; ++i) {
        Xy[k].re += gy.N[i] * sXv[i][k].x;
        Xy[k].im += gy.N[i] * sXv[i][k].y;
      }
    }
    const d3 Rv = sub(gx.x, gy.x);
    const double r = sqrt(dot(Rv, Rv));
    const d3 h = scl(1.0 / r, Rv);
    const double ir = 1.0 / r, ir2 = ir * ir;
    PairGeo G;
    G.n = gx.n;
    G.t[0] = gx.t1;
    G.t[1] = gx.t2;
    G.s[0] = scl(-gx.sig, gx.t2);  // s1 = t1 x n = -sig t2
    G.s[1] = scl(gx.sig, gx.t1);   // s2 = t2 x n = sig t1
    G.u[0] = gy.t1;
    G.u[1] = gy.t2;
    const double Wt = w * gx.J * gy.J;
    double m[6];
    if (SIDE == 0)
      mono6(xi, eta, m);
    else
      mono6(yxi, yeta, m);
    const double sa = SIDE == 0 ? xi : yxi, ta = SIDE == 0 ? eta : yeta;
#pragma unroll 1
    for (int o = 0; o < R; ++o) {
      cx<double> Lx[4];
      for (int k = 0; k < 4; ++k) {
        Lx[k] = cmk(0.0, 0.0);
        for (int i = 0; i < 6; ++i) {
          Lx[k].re += gx.N[i] * sL[o][i][k].x;
          Lx[k].im += gx.N[i] * sL[o][i][k].y;
        }
      }
      // gamma_c from lam (test side) and x (trial side) at the points
      double c1v[4], c2v[4], cGv[4], d1v[4], d2v[4], dGv[4];
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
      d3 gR, gs[2], gtx[2], gn, gty[2];
      const double Vv = kernel_vjp(G, h, r, c1v, c2v, cGv, d1v, d2v, dGv, gR, gs, gtx, gn, gty);
      GeoRev rv;
      if (SIDE == 0) {
        // s1 = -sig t2, s2 = sig t1
        d3 gt1 = add(scl(Wt, gtx[0]), scl(Wt * gx.sig, gs[1]));
        d3 gt2 = add(scl(Wt, gtx[1]), scl(-Wt * gx.sig, gs[0]));
        rv = geo_reverse(gx.a1, gx.a2, gx.u1, gx.n, gx.t1, gx.J, gx.sig, scl(Wt, gR), scl(Wt, gn),
                         gt1, gt2, Vv * w * gy.J);
      } else {
        rv = geo_reverse(gy.a1, gy.a2, gy.u1, gy.n, gy.t1, gy.J, gy.sig, scl(-Wt, gR), mk(0, 0, 0),
                         scl(Wt, gty[0]), scl(Wt, gty[1]), Vv * w * gx.J);
      }
      // x = sum m_k CX_k, a1 = CX1 + 2 xi CX3 + eta CX4, a2 = CX2 + xi CX4 + 2 eta CX5
      d3 gC[6];
      for (int k = 0; k < 6; ++k) gC[k] = scl(m[k], rv.gx);
      gC[1] = add(gC[1], rv.ga1);
      gC[3] = add(gC[3], scl(2.0 * sa, rv.ga1));
      gC[4] = add(gC[4], add(scl(ta, rv.ga1), scl(sa, rv.ga2)));
      gC[2] = add(gC[2], rv.ga2);
      gC[5] = add(gC[5], scl(2.0 * ta, rv.ga2));
      double* ac = acc[o];
      for (int k = 0; k < 6; ++k) {
        ac[3 * k] += gC[k].x;
        ac[3 * k + 1] += gC[k].y;
        ac[3 * k + 2] += gC[k].z;
        ac[18 + 3 * k] += m[k] * rv.gu1.x;
        ac[18 + 3 * k + 1] += m[k] * rv.gu1.y;
        ac[18 + 3 * k + 2] += m[k] * rv.gu1.z;
      }
    }
  }
  // CTA sums of the 36 monomial-coefficient adjoints per vector: warp sums,
  // then the SST / 32 warps' partials
  __shared__ double wsum[SST / 32][36];
  __shared__ double sum[36];
  const int lane = tid & 31, warp = tid >> 5;
  for (int o = 0; o < R; ++o) {
    for (int k = 0; k < 36; ++k) {
      double v = acc[o][k];
      for (int q = 16; q > 0; q >>= 1) v += __shfl_xor_sync(0xffffffffu, v, q);
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
      for (int k = 0; k < 6; ++k) atomicAdd(V.eadj[o] + e * 54 + 18 * fld + 3 * k + d, gv[k]);
    }
    __syncthreads();  // before the next vector's partials overwrite wsum and sum
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

// ------------------------------------------------------- right-hand side
// Re lam^H b (Eqs. rhs_E, rhs_H): b rows (h = 0, node, a) = sum_p W_p N(p)
// (-s_a . p) e^{i phi_p}, (h = 1) = sum_p W_p N(p) (s_a . (k x p)) e^{i phi_p},
// phi_p = k_a k . y_p; the adjoints of s_a, y and W at each rule point.
__global__ void rhs_vjp_kernel(int64_t n, const double* __restrict__ qd,
                               const double2* __restrict__ Lp, d3 kh, d3 ph, double ka,
                               double* __restrict__ radj) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double* rc = qd + t * QD_STRIDE;
  const double2* L = Lp + t * 4;
  const d3 hk = cross(kh, ph);
  double sn, cs;
  sincos(ka * dot(kh, ld3(rc)), &sn, &cs);
  const double W = rc[18];
  double vr = 0.0, vi = 0.0;
  for (int a = 0; a < 2; ++a) {
    // E_a = e^{i phi} (-L0a p + L1a hk): real and imaginary 3-vectors
    const cx<double> l0 = cmk(L[a].x, L[a].y), l1 = cmk(L[2 + a].x, L[2 + a].y);
    const cx<double> e = cmk(cs, sn);
    const cx<double> c0 = cmul(e, l0), c1 = cmul(e, l1);
    const d3 Er = sub(scl(c1.re, hk), scl(c0.re, ph));
    const d3 Ei = sub(scl(c1.im, hk), scl(c0.im, ph));
    const d3 sa = ld3(rc + 12 + 3 * a);
    vr += dot(sa, Er);
    vi += dot(sa, Ei);
    double* g = radj + t * 19 + 12 + 3 * a;
    g[0] += W * Er.x;
    g[1] += W * Er.y;
    g[2] += W * Er.z;
  }
  // d/dy of e^{i phi}: i k_a k -> Re(i k_a k W v) = -k_a W Im(v) k
  double* g = radj + t * 19;
  g[0] += -ka * W * vi * kh.x;
  g[1] += -ka * W * vi * kh.y;
  g[2] += -ka * W * vi * kh.z;
  g[18] += vr;
}

// ------------------------------------------------------------ far field
// Currents at the rule points: cur[p] = (W j, W j_m) (complex 3-vectors),
// j = sum_b Xi_0b t_b, j_m = sum_b Xi_1b t_b (Sec. 4.1 basis).
__global__ void far_currents_kernel(int64_t n, const double* __restrict__ qd,
                                    const double2* __restrict__ Xp, double2* __restrict__ cur) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double* rc = qd + t * QD_STRIDE;
  const double2* X = Xp + t * 4;
  const double W = rc[18];
  for (int c = 0; c < 3; ++c) {
    double2 j = make_double2(0, 0), m = make_double2(0, 0);
    for (int b = 0; b < 2; ++b) {
      const double tb = rc[6 + 3 * b + c];
      j.x += X[b].x * tb;
      j.y += X[b].y * tb;
      m.x += X[2 + b].x * tb;
      m.y += X[2 + b].y * tb;
    }
    cur[t * 6 + c] = make_double2(W * j.x, W * j.y);
    cur[t * 6 + 3 + c] = make_double2(W * m.x, W * m.y);
  }
}

// F(d) = (i k/4 pi) sum_p e^{-i k d.y_p} [P_d W j - d x W j_m], one CTA per
// direction (the directions in dirs[nd][3])
__global__ void __launch_bounds__(256) far_sum_kernel(int64_t np, const double* __restrict__ qd,
                                                      const double2* __restrict__ cur,
                                                      const double* __restrict__ dirs, double ka,
                                                      double2* __restrict__ F) {
  const int64_t di = blockIdx.x;
  const d3 d = ld3(dirs + 3 * di);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t p = threadIdx.x; p < np; p += blockDim.x) {
    double sn, cs;
    sincos(-ka * dot(d, ld3(qd + p * QD_STRIDE)), &sn, &cs);
    const double2* c = cur + p * 6;
    d3 jr = mk(c[0].x, c[1].x, c[2].x), ji = mk(c[0].y, c[1].y, c[2].y);
    const d3 mr = mk(c[3].x, c[4].x, c[5].x), mi = mk(c[3].y, c[4].y, c[5].y);
    jr = sub(sub(jr, scl(dot(d, jr), d)), cross(d, mr));
    ji = sub(sub(ji, scl(dot(d, ji), d)), cross(d, mi));
    // (cs + i sn)(jr + i ji)
    acc[0] += cs * jr.x - sn * ji.x;
    acc[1] += cs * ji.x + sn * jr.x;
    acc[2] += cs * jr.y - sn * ji.y;
    acc[3] += cs * ji.y + sn * jr.y;
    acc[4] += cs * jr.z - sn * ji.z;
    acc[5] += cs * ji.z + sn * jr.z;
  }
  __shared__ double red[6][256];
  for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) {
    // times i k/(4 pi)
    const double f = ka * kC4pi, re = red[2 * threadIdx.x][0], im = red[2 * threadIdx.x + 1][0];
    F[di * 3 + threadIdx.x] = make_double2(-f * im, f * re);
  }
}

// Per rule point and output o (0 C_ext, 1 C_sca, 2 C_abs): JA, MA with
// dC = 2 Re(JA . dj + MA . dj_m) at fixed geometry, and the explicit
// adjoints of y, W, n.  C_sca sums over the sphere rule (directions 1..nsph
// of dirs with weights wd); one CTA per point.
struct FarArgs {
  int64_t np, nsph;
  const double* qd;
  const double2* cur;   // W j, W j_m
  const double* dirs;   // [0] forward, then the sphere rule
  const double* wd;     // weights of the sphere directions
  const double2* F;     // far fields of dirs
  double ka;
  d3 kh, ph;
  double2* JA;          // [3][np][3]
  double2* MA;          // [3][np][3]
  double* radj;         // [3][np][19]
  double* cab;          // [np]: W Re j_m . (conj(j) x n)
};

__global__ void __launch_bounds__(128) far_adjoint_kernel(FarArgs a) {
  const int64_t p = blockIdx.x;
  const double* rc = a.qd + p * QD_STRIDE;
  const d3 y = ld3(rc);
  const double W = rc[18];
  const double2* c = a.cur + p * 6;
  // j and j_m themselves (cur holds W j)
  const double iW = 1.0 / W;
  cx<double> j[3], m[3];
  for (int k = 0; k < 3; ++k) {
    j[k] = cmk(c[k].x * iW, c[k].y * iW);
    m[k] = cmk(c[3 + k].x * iW, c[3 + k].y * iW);
  }
  // ---- C_sca: sums over the sphere directions
  double acc[16];
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  const cx<double> ikf = cmk(0.0, a.ka * kC4pi);  // i k/(4 pi)
  for (int64_t dd = threadIdx.x; dd < a.nsph; dd += blockDim.x) {
    const d3 d = ld3(a.dirs + 3 * (1 + dd));
    double sn, cs;
    sincos(-a.ka * dot(d, y), &sn, &cs);
    const cx<double> ph = cmul(cmk(a.wd[dd] * cs, a.wd[dd] * sn), ikf);  // wd (ik/4pi) e^{-ik d.y}
    const double2* Fd = a.F + (1 + dd) * 3;
    const cx<double> Fc[3] = {cmk(Fd[0].x, -Fd[0].y), cmk(Fd[1].x, -Fd[1].y), cmk(Fd[2].x, -Fd[2].y)};
    // P_d conj(F) and conj(F) x d
    const cx<double> dF = cadd(cadd(crs(d.x, Fc[0]), crs(d.y, Fc[1])), crs(d.z, Fc[2]));
    const double dv[3] = {d.x, d.y, d.z};
    cx<double> PF[3], Fxd[3];
    for (int k = 0; k < 3; ++k) PF[k] = csub(Fc[k], crs(dv[k], dF));
    Fxd[0] = csub(crs(d.z, Fc[1]), crs(d.y, Fc[2]));
    Fxd[1] = csub(crs(d.x, Fc[2]), crs(d.z, Fc[0]));
    Fxd[2] = csub(crs(d.y, Fc[0]), crs(d.x, Fc[1]));
    // JA += ph W P conj(F);  MA += -ph W (conj(F) x d)
    for (int k = 0; k < 3; ++k) {
      const cx<double> u = cmul(ph, PF[k]);
      const cx<double> v = cmul(ph, Fxd[k]);
      acc[2 * k] += W * u.re;
      acc[2 * k + 1] += W * u.im;
      acc[6 + 2 * k] -= W * v.re;
      acc[6 + 2 * k + 1] -= W * v.im;
    }
    // conj(F) . [P j - d x j_m]  =  PF . j - Fxd . j_m
    cx<double> q = cmk(0.0, 0.0);
    for (int k = 0; k < 3; ++k) q = csub(cadd(q, cmul(PF[k], j[k])), cmul(Fxd[k], m[k]));
    const cx<double> qq = cmul(ph, q);
    // W: 2 Re(qq);  y: 2 Re(qq (-i k) W) d = 2 k W Im(qq) d
    acc[12] += 2.0 * qq.re;
    const double gy = 2.0 * a.ka * W * qq.im;
    acc[13] += gy * d.x;
    acc[14] += gy * d.y;
    acc[15] += gy * d.z;
  }
  __shared__ double red[16][128];
  for (int k = 0; k < 16; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 16; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const int64_t np = a.np;
  // C_sca (o = 1)
  for (int k = 0; k < 3; ++k) {
    a.JA[(1 * np + p) * 3 + k] = make_double2(red[2 * k][0], red[2 * k + 1][0]);
    a.MA[(1 * np + p) * 3 + k] = make_double2(red[6 + 2 * k][0], red[6 + 2 * k + 1][0]);
  }
  double* g1 = a.radj + (1 * np + p) * 19;
  g1[0] += red[13][0];
  g1[1] += red[14][0];
  g1[2] += red[15][0];
  g1[18] += red[12][0];
  // C_ext (o = 0): Re sum W e^{-i psi} [p.j - (p x k).j_m], psi = k kh.y
  {
    double sn, cs;
    sincos(-a.ka * dot(a.kh, y), &sn, &cs);
    const cx<double> e = cmk(cs, sn);
    const d3 pk = cross(a.ph, a.kh);
    const double pv[3] = {a.ph.x, a.ph.y, a.ph.z}, kv[3] = {pk.x, pk.y, pk.z};
    cx<double> v = cmk(0.0, 0.0);
    for (int k = 0; k < 3; ++k) {
      v = csub(cadd(v, crs(pv[k], j[k])), crs(kv[k], m[k]));
      a.JA[p * 3 + k] = make_double2(0.5 * W * e.re * pv[k], 0.5 * W * e.im * pv[k]);
      a.MA[p * 3 + k] = make_double2(-0.5 * W * e.re * kv[k], -0.5 * W * e.im * kv[k]);
    }
    const cx<double> ev = cmul(e, v);
    double* g0 = a.radj + p * 19;
    g0[18] += ev.re;
    // d/dy e^{-i k kh.y} = -i k kh e: Re(-i k W ev) kh = k W Im(ev) kh
    g0[0] += a.ka * W * ev.im * a.kh.x;
    g0[1] += a.ka * W * ev.im * a.kh.y;
    g0[2] += a.ka * W * ev.im * a.kh.z;
  }
  // C_abs (o = 2): Re sum W j_m . (conj(j) x n)
  {
    const d3 n = ld3(rc + 3);
    const double nv[3] = {n.x, n.y, n.z};
    cx<double> cj[3] = {cmk(j[0].re, -j[0].im), cmk(j[1].re, -j[1].im), cmk(j[2].re, -j[2].im)};
    cx<double> cjn[3], nm[3], mcj[3];
    for (int k = 0; k < 3; ++k) {
      const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      cjn[k] = csub(crs(nv[k2], cj[k1]), crs(nv[k1], cj[k2]));      // conj(j) x n
      nm[k] = csub(crs(nv[k1], m[k2]), crs(nv[k2], m[k1]));          // n x j_m
      mcj[k] = csub(cmul(m[k1], cj[k2]), cmul(m[k2], cj[k1]));       // j_m x conj(j)
    }
    double val = 0.0;
    for (int k = 0; k < 3; ++k) {
      val += cmul(m[k], cjn[k]).re;
      a.JA[(2 * np + p) * 3 + k] = make_double2(0.5 * W * nm[k].re, -0.5 * W * nm[k].im);
      a.MA[(2 * np + p) * 3 + k] = make_double2(0.5 * W * cjn[k].re, 0.5 * W * cjn[k].im);
    }
    double* g2 = a.radj + (2 * np + p) * 19;
    g2[18] += val;
    a.cab[p] = W * val;
    g2[3] += W * mcj[0].re;
    g2[4] += W * mcj[1].re;
    g2[5] += W * mcj[2].re;
  }
}

// From JA, MA of each output: the frame adjoints 2 Re(Xi_0b JA + Xi_1b MA)
// at the points, and G[o][u] = sum over the points of N_k (JA . t_b) (g = 0)
// or N_k (MA . t_b) (g = 1) for u = g H + 2 node_k + b, conjugated on output
// (the right-hand sides of Z^H lam = G).
__global__ void far_finish_kernel(int64_t nt, RuleC rule, const int32_t* __restrict__ T,
                                  const double* __restrict__ qd, const double2* __restrict__ Xp,
                                  const double2* __restrict__ JA, const double2* __restrict__ MA,
                                  int64_t H, double* __restrict__ radj, double2* __restrict__ G) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t np = nt * rule.Q;
  if (t >= 3 * np) return;
  const int o = (int)(t / np);
  const int64_t pt = t % np;
  const int64_t e = pt / rule.Q;
  const int p = (int)(pt % rule.Q);
  const double* rc = qd + pt * QD_STRIDE;
  const double2* X = Xp + pt * 4;
  const double2* ja = JA + (o * np + pt) * 3;
  const double2* ma = MA + (o * np + pt) * 3;
  double* g = radj + (o * np + pt) * 19;
  double N[6];
  p2N(rule.xi[p], rule.eta[p], N);
  for (int b = 0; b < 2; ++b) {
    const cx<double> x0 = cmk(X[b].x, X[b].y), x1 = cmk(X[2 + b].x, X[2 + b].y);
    cx<double> jt = cmk(0.0, 0.0), mt = cmk(0.0, 0.0);
    for (int k = 0; k < 3; ++k) {
      const cx<double> jk = cmk(ja[k].x, ja[k].y), mk_ = cmk(ma[k].x, ma[k].y);
      g[6 + 3 * b + k] += 2.0 * (cmul(x0, jk).re + cmul(x1, mk_).re);
      jt = cadd(jt, crs(rc[6 + 3 * b + k], jk));
      mt = cadd(mt, crs(rc[6 + 3 * b + k], mk_));
    }
    for (int i = 0; i < 6; ++i) {
      const int64_t node = T[6 * e + i];
      double2* g0 = G + (int64_t)o * 2 * H + 2 * node + b;
      double2* g1 = G + (int64_t)o * 2 * H + H + 2 * node + b;
      atomicAdd(&g0->x, N[i] * jt.re);
      atomicAdd(&g0->y, -N[i] * jt.im);
      atomicAdd(&g1->x, N[i] * mt.re);
      atomicAdd(&g1->y, -N[i] * mt.im);
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

// The gradients of Re lam_o^H Z(X) x for r adjoint vectors lam_o (lam: r x N,
// contiguous), into grad + o * nn * 3.  The regular-pair and remainder kernels
// take up to kVjpR vectors per launch, so that each point pair's radial
// functions serve all of them; the other passes run per vector.
mueller_status zshape_vjp(mueller_mesh* m, const PhysConsts& P, int Q, int ns, const void* lam,
                          const void* x, int r, double* grad, cudaStream_t s) {
  MU_CUDA(cis64_table_ready());  // the radial functions' exp(i theta) table
  TriangleRule rule;
  if (!triangle_rule(Q, rule)) {
    set_error("q_regular must be 6 or 12");
    return MUELLER_ERR_INVALID_ARG;
  }
  const RuleC rc = rule_c(rule);
  const int64_t N = 4 * m->nn, H = N / 2;
  const double2* L = (const double2*)lam;
  std::vector<ShapeWork> W(r);
  mueller_status st = MUELLER_OK;
  for (int o = 0; o < r && !st; ++o) st = shape_alloc(m, Q, W[o], s);
  KConst<double> K;
  K.ka = P.ka;
  K.ki_re = P.ki_re;
  K.ki_im = P.ki_im;
  K.eps_re = P.eps_re;
  K.eps_im = P.eps_im;
  K.mu_re = P.mu_re;
  K.mu_im = P.mu_im;
  K.sing = 0.0;
  for (int o = 0; o < r && !st; ++o) {
    { Prof prof_("pt_fields_kernel", s); pt_fields_kernel<<<nblk(m->nt * Q, 128), 128, 0, s>>>(m->nt, rc, m->T, L + o * N, (const double2*)x, H, W[o].Lp, W[o].Xp); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "pt_fields_kernel");
  }
  for (int o0 = 0; o0 < r && !st; o0 += kVjpR) {
    const int R = std::min(kVjpR, r - o0);
    VjpSet V = {};
    for (int o = 0; o < R; ++o) {
      V.Lp[o] = W[o0 + o].Lp;
      V.radj[o] = W[o0 + o].radj;
    }
    const double2* Xp = W[o0].Xp;
    {
      Prof prof_("pair_vjp_kernel<0>", s);
      if (R == 1) pair_vjp_kernel<0, 1><<<(unsigned)m->nt, 32 * Q, 0, s>>>(m->nt, Q, m->qd64, m->T, V, Xp, K);
      else if (R == 2) pair_vjp_kernel<0, 2><<<(unsigned)m->nt, 32 * Q, 0, s>>>(m->nt, Q, m->qd64, m->T, V, Xp, K);
      else pair_vjp_kernel<0, 3><<<(unsigned)m->nt, 32 * Q, 0, s>>>(m->nt, Q, m->qd64, m->T, V, Xp, K);
    }
    {
      Prof prof_("pair_vjp_kernel<1>", s);
      if (R == 1) pair_vjp_kernel<1, 1><<<(unsigned)m->nt, 32 * Q, 0, s>>>(m->nt, Q, m->qd64, m->T, V, Xp, K);
      else if (R == 2) pair_vjp_kernel<1, 2><<<(unsigned)m->nt, 32 * Q, 0, s>>>(m->nt, Q, m->qd64, m->T, V, Xp, K);
      else pair_vjp_kernel<1, 3><<<(unsigned)m->nt, 32 * Q, 0, s>>>(m->nt, Q, m->qd64, m->T, V, Xp, K);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "pair adjoint kernels");
  }
  for (int o = 0; o < r && !st; ++o) {
    { Prof prof_("mass_vjp_kernel", s); mass_vjp_kernel<<<nblk(m->nt * Q, 128), 128, 0, s>>>(m->nt * Q, W[o].Lp, W[o].Xp, 0.5 * (1.0 + P.eps_re), 0.5 * P.eps_im, 0.5 * (1.0 + P.mu_re), 0.5 * P.mu_im, W[o].radj); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "mass_vjp_kernel");
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
    for (int o0 = 0; o0 < r && !st; o0 += kVjpR) {
      const int R = std::min(kVjpR, r - o0);
      SsVjpSet V = {};
      for (int o = 0; o < R; ++o) {
        V.lam[o] = L + (o0 + o) * N;
        V.eadj[o] = W[o0 + o].eadj;
      }
      const unsigned g = (unsigned)m->n_touch;
      const double2* xv = (const double2*)x;
      {
        Prof prof_("ss_vjp_kernel<0>", s);
        if (R == 1) ss_vjp_kernel<0, 1><<<g, SST, 0, s>>>(m->tp, m->X, m->T, m->frame, V, xv, H, gl, c1, ce, cm, 1.0 / P.ka);
        else if (R == 2) ss_vjp_kernel<0, 2><<<g, SST, 0, s>>>(m->tp, m->X, m->T, m->frame, V, xv, H, gl, c1, ce, cm, 1.0 / P.ka);
        else ss_vjp_kernel<0, 3><<<g, SST, 0, s>>>(m->tp, m->X, m->T, m->frame, V, xv, H, gl, c1, ce, cm, 1.0 / P.ka);
      }
      {
        Prof prof_("ss_vjp_kernel<1>", s);
        if (R == 1) ss_vjp_kernel<1, 1><<<g, SST, 0, s>>>(m->tp, m->X, m->T, m->frame, V, xv, H, gl, c1, ce, cm, 1.0 / P.ka);
        else if (R == 2) ss_vjp_kernel<1, 2><<<g, SST, 0, s>>>(m->tp, m->X, m->T, m->frame, V, xv, H, gl, c1, ce, cm, 1.0 / P.ka);
        else ss_vjp_kernel<1, 3><<<g, SST, 0, s>>>(m->tp, m->X, m->T, m->frame, V, xv, H, gl, c1, ce, cm, 1.0 / P.ka);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_fail(e, "Sauter-Schwab adjoint kernels");
    }
  }
  for (int o = 0; o < r && !st; ++o) st = shape_finish(m, rc, W[o], grad + (size_t)o * m->nn * 3, s);
  for (ShapeWork& w : W) shape_free(w, s);
  return st;
}

mueller_status rhs_shape_vjp(mueller_mesh* m, const PhysConsts& P, int Q, const void* lam,
                             const double* inc, double* grad, cudaStream_t s) {
  TriangleRule rule;
  if (!triangle_rule(Q, rule)) {
    set_error("q_regular must be 6 or 12");
    return MUELLER_ERR_INVALID_ARG;
  }
  const RuleC rc = rule_c(rule);
  ShapeWork W;
  mueller_status st = shape_alloc(m, Q, W, s);
  const int64_t N = 4 * m->nn, H = N / 2;
  if (!st) {
    const d3 kh = mk(inc[0], inc[1], inc[2]), ph = mk(inc[3], inc[4], inc[5]);
    { Prof prof_("pt_fields_kernel", s); pt_fields_kernel<<<nblk(m->nt * Q, 128), 128, 0, s>>>(m->nt, rc, m->T, (const double2*)lam, (const double2*)lam, H, W.Lp, W.Xp); }
    { Prof prof_("rhs_vjp_kernel", s); rhs_vjp_kernel<<<nblk(m->nt * Q, 128), 128, 0, s>>>(m->nt * Q, m->qd64, W.Lp, kh, ph, P.ka, W.radj); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "right-hand-side adjoint kernels");
  }
  if (!st) st = shape_finish(m, rc, W, grad, s);
  shape_free(W, s);
  return st;
}

// dC/dx (as the right-hand sides G of Z^H lam = G, device 3 x N complex128)
// and dC/dX at fixed x (host, 3 x n_nodes x 3, added) for C_ext, C_sca,
// C_abs of one incident wave; xs (host, 3): the cross sections of x.
mueller_status cross_section_partials(mueller_mesh* m, const PhysConsts& P, int Q, const void* x,
                                      const double* inc, int n_theta, int n_phi, void* G,
                                      double* grad, double* xs, cudaStream_t s) {
  TriangleRule rule;
  if (!triangle_rule(Q, rule)) {
    set_error("q_regular must be 6 or 12");
    return MUELLER_ERR_INVALID_ARG;
  }
  const RuleC rc = rule_c(rule);
  const int64_t np = m->nt * Q, N = 4 * m->nn, H = N / 2;
  const int64_t nsph = (int64_t)n_theta * n_phi, nd = 1 + nsph;
  // directions: forward, then cos(theta) on Gauss-Legendre nodes x phi on
  // n_phi equal steps, weights 2 w_theta 2 pi / n_phi (the sphere rule of
  // the cross sections)
  std::vector<double> gth, wth;
  gauss_legendre_unit(n_theta, gth, wth);
  std::vector<double> hd(nd * 3), hw(nsph);
  hd[0] = inc[0];
  hd[1] = inc[1];
  hd[2] = inc[2];
  for (int it = 0; it < n_theta; ++it) {
    const double ct = 2.0 * gth[it] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
    for (int ip = 0; ip < n_phi; ++ip) {
      const double ph = 2.0 * kPi * ip / n_phi;
      const int64_t k = (int64_t)it * n_phi + ip;
      hd[3 * (1 + k)] = st * cos(ph);
      hd[3 * (1 + k) + 1] = st * sin(ph);
      hd[3 * (1 + k) + 2] = ct;
      hw[k] = 2.0 * wth[it] * (2.0 * kPi / n_phi);
    }
  }
  // three outputs share the point fields; radj holds 3 x np x 19
  double2 *Lp = nullptr, *Xp = nullptr, *cur = nullptr, *F = nullptr, *JA = nullptr, *MA = nullptr;
  double *dirs = nullptr, *wd = nullptr, *radj = nullptr, *eadj = nullptr, *gpos = nullptr;
  double* cab = nullptr;
  mueller_status st = MUELLER_OK;
  auto take = [&](void** ptr, size_t bytes) {
    if (st) return;
    cudaError_t e = cudaMallocAsync(ptr, bytes, s);
    if (e != cudaSuccess) st = cuda_fail(e, "cross-section partials workspace");
  };
  take((void**)&Lp, np * 4 * sizeof(double2));
  take((void**)&Xp, np * 4 * sizeof(double2));
  take((void**)&cur, np * 6 * sizeof(double2));
  take((void**)&F, nd * 3 * sizeof(double2));
  take((void**)&JA, 3 * np * 3 * sizeof(double2));
  take((void**)&MA, 3 * np * 3 * sizeof(double2));
  take((void**)&dirs, nd * 3 * sizeof(double));
  take((void**)&wd, nsph * sizeof(double));
  take((void**)&radj, 3 * np * 19 * sizeof(double));
  take((void**)&eadj, m->nt * 54 * sizeof(double));
  take((void**)&gpos, m->nn * 3 * sizeof(double));
  take((void**)&cab, np * sizeof(double));
  std::vector<double> Fh(nd * 6), cabh(np);
  if (!st) {
    cudaError_t e = cudaMemcpyAsync(dirs, hd.data(), hd.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(wd, hw.data(), hw.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(radj, 0, 3 * np * 19 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, 3 * N * sizeof(double2), s);
    if (e != cudaSuccess) st = cuda_fail(e, "cross-section partials setup");
  }
  if (!st) {
    const d3 kh = mk(inc[0], inc[1], inc[2]), ph = mk(inc[3], inc[4], inc[5]);
    { Prof prof_("pt_fields_kernel", s); pt_fields_kernel<<<nblk(np, 128), 128, 0, s>>>(m->nt, rc, m->T, (const double2*)x, (const double2*)x, H, Lp, Xp); }
    { Prof prof_("far_currents_kernel", s); far_currents_kernel<<<nblk(np, 128), 128, 0, s>>>(np, m->qd64, Xp, cur); }
    { Prof prof_("far_sum_kernel", s); far_sum_kernel<<<(unsigned)nd, 256, 0, s>>>(np, m->qd64, cur, dirs, P.ka, F); }
    FarArgs fa;
    fa.np = np;
    fa.nsph = nsph;
    fa.qd = m->qd64;
    fa.cur = cur;
    fa.dirs = dirs;
    fa.wd = wd;
    fa.F = F;
    fa.ka = P.ka;
    fa.kh = kh;
    fa.ph = ph;
    fa.JA = JA;
    fa.MA = MA;
    fa.radj = radj;
    fa.cab = cab;
    { Prof prof_("far_adjoint_kernel", s); far_adjoint_kernel<<<(unsigned)np, 128, 0, s>>>(fa); }
    { Prof prof_("far_finish_kernel", s); far_finish_kernel<<<nblk(3 * np, 128), 128, 0, s>>>(m->nt, rc, m->T, m->qd64, Xp, JA, MA, H, radj, (double2*)G); }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(Fh.data(), F, nd * 3 * sizeof(double2), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cabh.data(), cab, np * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_fail(e, "cross-section partial kernels");
  }
  // geometry adjoints of each output through the records
  for (int o = 0; o < 3 && !st; ++o) {
    cudaError_t e = cudaMemsetAsync(eadj, 0, m->nt * 54 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gpos, 0, m->nn * 3 * sizeof(double), s);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cross-section partials");
      break;
    }
    ShapeWork W;
    W.radj = radj + (size_t)o * np * 19;
    W.eadj = eadj;
    W.gpos = gpos;
    st = shape_finish(m, rc, W, grad + (size_t)o * m->nn * 3, s);
  }
  if (!st && xs) {
    // C_ext = (4 pi/k) Im(p . F(k)), C_sca = sum wd |F|^2, C_abs = sum of cab
    const double pv[3] = {inc[3], inc[4], inc[5]};
    double im = 0.0;
    for (int k = 0; k < 3; ++k) im += pv[k] * Fh[2 * k + 1];
    xs[0] = 4.0 * kPi / P.ka * im;
    double cs = 0.0;
    for (int64_t k = 0; k < nsph; ++k)
      for (int c = 0; c < 6; ++c) cs += hw[k] * Fh[6 * (1 + k) + c] * Fh[6 * (1 + k) + c];
    xs[1] = cs;
    double ca = 0.0;
    for (int64_t k = 0; k < np; ++k) ca += cabh[k];
    xs[2] = ca;
  }
  for (void* q : {(void*)Lp, (void*)Xp, (void*)cur, (void*)F, (void*)JA, (void*)MA, (void*)dirs,
                  (void*)wd, (void*)radj, (void*)eadj, (void*)gpos, (void*)cab})
    if (q) cudaFreeAsync(q, s);
  return st;
}

}  // namespace mu
