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

namespace mu {

template <class R>
struct cx {
  R re, im;
};
template <class R>
__device__ __forceinline__ cx<R> cmk(R a, R b) {
  return cx<R>{a, b};
}
template <class R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
  return cx<R>{a.re + b.re, a.im + b.im};
}
template <class R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) {
  return cx<R>{a.re - b.re, a.im - b.im};
}
template <class R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return cx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R>
__device__ __forceinline__ cx<R> crs(R s, cx<R> a) {
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
__device__ __forceinline__ void qfuncs(cx<R> z, cx<R>& q1, cx<R>& q2, cx<R>& q3) {
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
    if constexpr (sizeof(R) == 8) {
      sincos(z.im, &s, &c);
    } else {
      sincosf(z.im, &s, &c);
    }
    const R ex = (sizeof(R) == 8) ? R(exp((double)z.re)) : R(expf((float)z.re));
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

template <class R>
struct KConst {
  R ka, ki_re, ki_im;
  R eps_re, eps_im, mu_re, mu_im;  // interior; exterior = 1
  R sing;                           // placeholder (unused)
};

// S1, S2, De, Dm at distance R (> 0); remainder = drop the singular parts.
template <class R>
__device__ __forceinline__ void kernel_scalars(const KConst<R>& K, R r, bool remainder,
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

}  // namespace mu
