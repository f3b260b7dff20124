// Device evaluation of the Mueller kernel scalars (Sec. 2.3, Sec. 4).
//
// With c = 1/(4 pi) and z = i k R the three radial functions that build the
// kernels are
//   k^2 phi - g = -(c/R^3) (z^2 - z + 1) e^z,   f = (c/R^3)(z^2 - 3z + 3) e^z,
//   phi'        =  (c/R^2) (z - 1) e^z
// (Eq. Hdiff_exact; grad phi = phi' R^).  Writing each bracket times e^z as
// its Taylor series, the terms of order z^0 and z^1 are exactly the
// O(R^-3) / O(R^-2) parts that cancel between the exterior and the interior
// kernel (Eq. Hdiff_infinite: the n = 0 and n = 1 terms vanish), and the
// z^2 terms are the singular parts of Eqs. kappa_S and kappa2_S.  What is
// left are the tails
//   Q1(z) = sum_{m>=3} (m-1)^2    z^m/m!,  Q2(z) = sum_{m>=4} (m-1)(m-3) z^m/m!,
//   Q3(z) = sum_{m>=2} (m-1)      z^m/m!,
// evaluated by their power series when |z| < 1 (no cancellation at small
// kR) and in closed form otherwise.  Then
//   S1 = (ka^2-ki^2)/(8 pi R) - (c/R^3)(Q1(za) - Q1(zi))   coefficient of s.t
//   S2 = (ka^2-ki^2)/(8 pi R) + (c/R^3)(Q2(za) - Q2(zi))   coefficient of (s.R^)(R^.t)
//   D_chi = -(chi_a - chi_i) c/R^2 + (c/R^2)(chi_a Q3(za) - chi_i Q3(zi))
// and kappa_1 = S1 (s.t) + S2 (s.R^)(R^.t), kappa_2^chi = D_chi [(t.t)(n.R^) - (t.R^)(n.t)].
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

namespace mu {

// exp(i th) in FP64 by a table-driven reduction (P. T. P. Tang, ACM TOMS 15
// (1989)): th = n pi/128 + d, n the nearest integer to th 128/pi, |d| <=
// pi/256; exp(i th) = T[n mod 256] exp(i d) with T[j] = exp(i pi j/128) and
// exp(i d) from the Taylor series of cos to degree 6 and of sin to degree 7
// (truncation below 2e-20).  The reduction is Cody-Waite with pi/128 = kC1 +
// kC2 (kC1: 32 significant bits, so n kC1 is exact for |n| < 2^21).  Beyond
// |th| = 2^20 pi/128 it falls back to sincos.  About 16 FP64 operations
// against about three times as many for sincos.  The table lives in global
// memory (4 KB, served by L1); every translation unit that uses it has its
// own copy, filled once per device by cis64_table_ready().
namespace cis64 {
constexpr int kN = 256;
constexpr double kInv = 0x1.45f306dc9c883p+5;   // 128 / pi
constexpr double kC1 = 0x1.921fb544p-6;         // pi/128, leading 32 bits
constexpr double kC2 = 0x1.0b4611a626331p-40;   // pi/128 - kC1
constexpr double kMax = 1048576.0 * 0x1.921fb544p-6;  // 2^20 pi/128
constexpr double kRound = 6755399441055744.0;   // 1.5 * 2^52
}  // namespace cis64

static __device__ double2 g_cis64_tab[cis64::kN];

__device__ __forceinline__ double2 cis64_eval(double th) {
  if (fabs(th) > cis64::kMax) {
    double sn, cs;
    sincos(th, &sn, &cs);
    return make_double2(cs, sn);
  }
  const double t = fma(th, cis64::kInv, cis64::kRound);  // n in the low mantissa bits
  const int n = __double2loint(t);
  const double nf = t - cis64::kRound;
  double d = fma(-nf, cis64::kC1, th);
  d = fma(-nf, cis64::kC2, d);
  const double z = d * d;
  const double c = fma(z, fma(z, fma(z, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
  const double p = fma(z, fma(z, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0);
  const double sn = fma(d * z, p, d);
  const double2 T = __ldg(&g_cis64_tab[n & (cis64::kN - 1)]);
  return make_double2(fma(T.x, c, -T.y * sn), fma(T.y, c, T.x * sn));
}

// fill this translation unit's table on the current device (once per device)
static inline cudaError_t cis64_table_ready() {
  static std::mutex mu_;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu_);
  if (done[dev]) return cudaSuccess;
  double2 h[cis64::kN];
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < cis64::kN; ++j) h[j] = make_double2(cos(pi * j / 128.0), sin(pi * j / 128.0));
  e = cudaMemcpyToSymbol(g_cis64_tab, h, sizeof(h));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// exp(i y) for the radial functions: the table form in FP64 device code
template <class R>
__host__ __device__ __forceinline__ void cis_r(R y, R& s, R& c) {
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(R) == 8) {
    const double2 e = cis64_eval(y);
    c = e.x;
    s = e.y;
  } else {
    sincosf(y, &s, &c);
  }
#else
  if constexpr (sizeof(R) == 8) {
    sincos(y, &s, &c);
  } else {
    sincosf(y, &s, &c);
  }
#endif
}

template <class R>
struct cx {
  R re, im;
};
template <class R>
__host__ __device__ __forceinline__ cx<R> cmk(R a, R b) {
  return cx<R>{a, b};
}
template <class R>
__host__ __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
  return cx<R>{a.re + b.re, a.im + b.im};
}
template <class R>
__host__ __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) {
  return cx<R>{a.re - b.re, a.im - b.im};
}
template <class R>
__host__ __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return cx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R>
__host__ __device__ __forceinline__ cx<R> crs(R s, cx<R> a) {
  return cx<R>{s * a.re, s * a.im};
}

template <class R>
struct SeriesLen;
template <>
struct SeriesLen<double> {
  static constexpr int n = 24;  // |z| < 1: tail below 1e-20 of the sums
};
template <>
struct SeriesLen<float> {
  static constexpr int n = 13;
};

// Q1, Q2, Q3 at z (see above).  'z' is i k R.
template <class R>
__host__ __device__ __forceinline__ void qfuncs(cx<R> z, cx<R>& q1, cx<R>& q2, cx<R>& q3) {
  const R az2 = z.re * z.re + z.im * z.im;
  if (az2 < R(1)) {
    cx<R> t = z;  // z^m/m! at m = 1
    q1 = q2 = q3 = cmk<R>(0, 0);
#pragma unroll
    for (int m = 2; m <= SeriesLen<R>::n; ++m) {
      t = crs(R(1) / R(m), cmul(t, z));
      const R c1 = R((m - 1) * (m - 1)) * R(m >= 3);
      const R c2 = R((m - 1) * (m - 3)) * R(m >= 4);
      const R c3 = R(m - 1);
      q1.re = fma(c1, t.re, q1.re);
      q1.im = fma(c1, t.im, q1.im);
      q2.re = fma(c2, t.re, q2.re);
      q2.im = fma(c2, t.im, q2.im);
      q3.re = fma(c3, t.re, q3.re);
      q3.im = fma(c3, t.im, q3.im);
    }
  } else {
    R s, c;
    cis_r(z.im, s, c);
    // exterior arguments and lossless interiors have Re z = 0 exactly
    const R ex = z.re == R(0) ? R(1)
                              : ((sizeof(R) == 8) ? R(exp((double)z.re)) : R(expf((float)z.re)));
    const cx<R> ez = cmk<R>(ex * c, ex * s);
    const cx<R> z2 = cmul(z, z);
    // (z^2 - z + 1) e^z - 1 - z^2/2
    q1 = cmul(cmk<R>(z2.re - z.re + R(1), z2.im - z.im), ez);
    q1.re -= R(1) + R(0.5) * z2.re;
    q1.im -= R(0.5) * z2.im;
    q2 = cmul(cmk<R>(z2.re - R(3) * z.re + R(3), z2.im - R(3) * z.im), ez);
    q2.re += R(0.5) * z2.re - R(3);
    q2.im += R(0.5) * z2.im;
    q3 = cmul(cmk<R>(z.re - R(1), z.im), ez);
    q3.re += R(1);
  }
}

// The derivatives Q1'(z), Q2'(z), Q3'(z) and Q3(z) itself, split the same
// way: power series (term by term: sum c_m z^(m-1)/(m-1)!) for |z| < 1, else
// the closed forms Q1' = (z^2 + z) e^z - z, Q2' = (z^2 - z) e^z + z,
// Q3' = z e^z (derivatives of the closed forms above).
template <class R>
__host__ __device__ __forceinline__ void qfuncs_d(cx<R> z, cx<R>& p1, cx<R>& p2, cx<R>& p3,
                                                  cx<R>& q3) {
  const R az2 = z.re * z.re + z.im * z.im;
  if (az2 < R(1)) {
    cx<R> t = cmk<R>(1, 0);  // z^(m-1)/(m-1)! at m = 1
    cx<R> u = z;             // z^m/m! at m = 1
    p1 = p2 = p3 = q3 = cmk<R>(0, 0);
#pragma unroll
    for (int m = 2; m <= SeriesLen<R>::n; ++m) {
      t = crs(R(1) / R(m - 1), cmul(t, z));
      u = crs(R(1) / R(m), cmul(u, z));
      const R c1 = R((m - 1) * (m - 1)) * R(m >= 3);
      const R c2 = R((m - 1) * (m - 3)) * R(m >= 4);
      const R c3 = R(m - 1);
      p1.re = fma(c1, t.re, p1.re);
      p1.im = fma(c1, t.im, p1.im);
      p2.re = fma(c2, t.re, p2.re);
      p2.im = fma(c2, t.im, p2.im);
      p3.re = fma(c3, t.re, p3.re);
      p3.im = fma(c3, t.im, p3.im);
      q3.re = fma(c3, u.re, q3.re);
      q3.im = fma(c3, u.im, q3.im);
    }
  } else {
    R s, c;
    cis_r(z.im, s, c);
    // exterior arguments and lossless interiors have Re z = 0 exactly
    const R ex = z.re == R(0) ? R(1)
                              : ((sizeof(R) == 8) ? R(exp((double)z.re)) : R(expf((float)z.re)));
    const cx<R> ez = cmk<R>(ex * c, ex * s);
    const cx<R> z2 = cmul(z, z);
    p1 = csub(cmul(cadd(z2, z), ez), z);
    p2 = cadd(cmul(csub(z2, z), ez), z);
    p3 = cmul(z, ez);
    q3 = cmul(cmk<R>(z.re - R(1), z.im), ez);
    q3.re += R(1);
  }
}

template <class R>
struct KConst {
  R ka, ki_re, ki_im;
  R eps_re, eps_im, mu_re, mu_im;  // interior; exterior = 1
  R sing;                           // placeholder (unused)
};

// S1, S2, De, Dm at distance R (> 0); remainder = drop the singular parts.
template <class R>
__host__ __device__ __forceinline__ void kernel_scalars(const KConst<R>& K, R r, bool remainder,
                                               cx<R>& S1, cx<R>& S2, cx<R>& De, cx<R>& Dm) {
  const R c = R(0.0795774715459476678844418816862571885);  // 1/(4 pi)
  const cx<R> za = cmk<R>(R(0), K.ka * r);
  const cx<R> zi = cmk<R>(-K.ki_im * r, K.ki_re * r);
  cx<R> q1a, q2a, q3a, q1i, q2i, q3i;
  qfuncs(za, q1a, q2a, q3a);
  qfuncs(zi, q1i, q2i, q3i);
  const R ir = R(1) / r;
  const R ir2 = ir * ir, ir3 = ir2 * ir;
  S1 = crs(-c * ir3, csub(q1a, q1i));
  S2 = crs(c * ir3, csub(q2a, q2i));
  const cx<R> ei = cmk(K.eps_re, K.eps_im), mi = cmk(K.mu_re, K.mu_im);
  De = crs(c * ir2, csub(q3a, cmul(ei, q3i)));
  Dm = crs(c * ir2, csub(q3a, cmul(mi, q3i)));
  if (!remainder) {
    // (ka^2 - ki^2)/(8 pi R);  -(1 - chi_i)/(4 pi R^2)
    const cx<R> ki2 = cmk(K.ki_re * K.ki_re - K.ki_im * K.ki_im, R(2) * K.ki_re * K.ki_im);
    const cx<R> s = crs(R(0.5) * c * ir, cmk(K.ka * K.ka - ki2.re, -ki2.im));
    S1 = cadd(S1, s);
    S2 = cadd(S2, s);
    De = cadd(De, crs(-c * ir2, cmk(R(1) - K.eps_re, -K.eps_im)));
    Dm = cadd(Dm, crs(-c * ir2, cmk(R(1) - K.mu_re, -K.mu_im)));
  }
}

template <class R>
__host__ __device__ __forceinline__ cx<R> cdivc(cx<R> a, cx<R> b) {
  const R den = b.re * b.re + b.im * b.im;
  return cmk<R>((a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den);
}

// d/dtheta of S1, S2, De, Dm for theta = eps_r (which = 1) or mu_r (which = 2),
// complex derivatives (the scalars are holomorphic in eps_r, mu_r):
// k_i = k_a sqrt(eps_r mu_r) gives dk_i/dtheta = k_i / (2 theta) and
// dz_i = i R dk_i; the exterior terms do not depend on theta.
template <class R>
__host__ __device__ __forceinline__ void kernel_scalars_d(const KConst<R>& K, R r, bool remainder,
                                                          int which, cx<R>& S1, cx<R>& S2,
                                                          cx<R>& De, cx<R>& Dm) {
  const R c = R(0.0795774715459476678844418816862571885);  // 1/(4 pi)
  const cx<R> ki = cmk(K.ki_re, K.ki_im);
  const cx<R> ei = cmk(K.eps_re, K.eps_im), mi = cmk(K.mu_re, K.mu_im);
  const cx<R> dki = crs(R(0.5), cdivc(ki, which == 1 ? ei : mi));
  const cx<R> zi = cmk<R>(-K.ki_im * r, K.ki_re * r);
  const cx<R> dzi = cmk<R>(-r * dki.im, r * dki.re);
  cx<R> p1, p2, p3, q3i;
  qfuncs_d(zi, p1, p2, p3, q3i);
  const cx<R> dq1 = cmul(p1, dzi), dq2 = cmul(p2, dzi), dq3 = cmul(p3, dzi);
  const R ir = R(1) / r;
  const R ir2 = ir * ir, ir3 = ir2 * ir;
  S1 = crs(c * ir3, dq1);
  S2 = crs(-c * ir3, dq2);
  // De = (c/R^2)(Q3(za) - eps Q3(zi)), Dm likewise with mu
  De = crs(-c * ir2, cmul(ei, dq3));
  Dm = crs(-c * ir2, cmul(mi, dq3));
  if (which == 1) De = csub(De, crs(c * ir2, q3i));
  else Dm = csub(Dm, crs(c * ir2, q3i));
  if (!remainder) {
    // d[(ka^2 - ki^2)/(8 pi R)] = -(c/R) ki dki;  d[-(1 - chi)/(4 pi R^2)] = c/R^2
    const cx<R> s = crs(-c * ir, cmul(ki, dki));
    S1 = cadd(S1, s);
    S2 = cadd(S2, s);
    if (which == 1) De.re += c * ir2;
    else Dm.re += c * ir2;
  }
}

// 12 kernel components of one point pair, times the weights:// 12 kernel components of one point pair, times the weights:
// out[4*op + 2*alpha + beta], op = 0 K1, 1 K2^eps, 2 K2^mu.
// WHICH = 0: the components; 1, 2: their derivatives with respect to eps_r,
// mu_r (kernel_scalars_d; the geometry factors do not depend on them).
template <class R, int WHICH = 0>
__host__ __device__ __forceinline__ void point_pair(const KConst<R>& K, const R* __restrict__ px,
                                           const R* __restrict__ qy, bool remainder,
                                           cx<R> out[12]) {
  const R rx = px[0] - qy[0], ry = px[1] - qy[1], rz = px[2] - qy[2];
  const R r2 = rx * rx + ry * ry + rz * rz;
  const R W = px[18] * qy[18];
  // x record: x 0-2, n 3-5, t1 6-8, t2 9-11, s1 12-14, s2 15-17, W 18
  if (r2 == R(0)) {
    // coincident rule points of a coincident pair (remainder only):
    // kappa1 - kappa1^s -> i (ka^3 - ki^3)/(6 pi) s.t,  kappa2 - kappa2^s -> 0
    const R ka3 = K.ka * K.ka * K.ka;
    const cx<R> ki2 = cmk(K.ki_re * K.ki_re - K.ki_im * K.ki_im, R(2) * K.ki_re * K.ki_im);
    const cx<R> ki3 = cmul(ki2, cmk(K.ki_re, K.ki_im));
    const R inv6pi = R(0.0530516476972984452562945877908381257);
    cx<R> lim = cmk(ki3.im * inv6pi, (ka3 - ki3.re) * inv6pi);  // i (ka^3 - ki^3)/(6 pi)
    if constexpr (WHICH != 0) {
      // d lim = -i ki^2 dki / (2 pi),  dki = ki / (2 chi)
      const cx<R> dki = crs(R(0.5), cdivc(cmk(K.ki_re, K.ki_im),
                                          WHICH == 1 ? cmk(K.eps_re, K.eps_im) : cmk(K.mu_re, K.mu_im)));
      const cx<R> t = cmul(ki2, dki);
      const R inv2pi = R(0.159154943091895335768883763372514362);
      lim = cmk(t.im * inv2pi, -t.re * inv2pi);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const R* s = px + 12 + 3 * a;
        const R* t = qy + 6 + 3 * b;
        const R st = (s[0] * t[0] + s[1] * t[1] + s[2] * t[2]) * W;
        out[2 * a + b] = crs(st, lim);
        out[4 + 2 * a + b] = cmk<R>(0, 0);
        out[8 + 2 * a + b] = cmk<R>(0, 0);
      }
    return;
  }
  const R r = sqrt(r2);
  const R ir = R(1) / r;
  const R hx = rx * ir, hy = ry * ir, hz = rz * ir;
  cx<R> S1, S2, De, Dm;
  if constexpr (WHICH == 0)
    kernel_scalars<R>(K, r, remainder, S1, S2, De, Dm);
  else
    kernel_scalars_d<R>(K, r, remainder, WHICH, S1, S2, De, Dm);
  const R nR = px[3] * hx + px[4] * hy + px[5] * hz;
  R tR[2], sR[2], Rt[2], nt[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const R* t = px + 6 + 3 * a;
    const R* s = px + 12 + 3 * a;
    const R* u = qy + 6 + 3 * a;  // t_beta(y) with beta = a
    tR[a] = t[0] * hx + t[1] * hy + t[2] * hz;
    sR[a] = s[0] * hx + s[1] * hy + s[2] * hz;
    Rt[a] = hx * u[0] + hy * u[1] + hz * u[2];
    nt[a] = px[3] * u[0] + px[4] * u[1] + px[5] * u[2];
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const R* t = px + 6 + 3 * a;
      const R* s = px + 12 + 3 * a;
      const R* u = qy + 6 + 3 * b;
      const R st = s[0] * u[0] + s[1] * u[1] + s[2] * u[2];
      const R tt = t[0] * u[0] + t[1] * u[1] + t[2] * u[2];
      const R G = (tt * nR - tR[a] * nt[b]) * W;
      const R sRt = sR[a] * Rt[b] * W;
      const R stw = st * W;
      out[2 * a + b] = cmk(S1.re * stw + S2.re * sRt, S1.im * stw + S2.im * sRt);
      out[4 + 2 * a + b] = crs(G, De);
      out[8 + 2 * a + b] = crs(G, Dm);
    }
}

}  // namespace mu
