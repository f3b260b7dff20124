// Device helpers: P2 isoparametric triangle (Sec. 3.3) and small vector math.
#pragma once
#include <cuda_runtime.h>

namespace mu {

struct d3 {
  double x, y, z;
};
__host__ __device__ __forceinline__ d3 mk(double a, double b, double c) { return d3{a, b, c}; }
__host__ __device__ __forceinline__ d3 add(d3 a, d3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ __forceinline__ d3 sub(d3 a, d3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ __forceinline__ d3 scl(double s, d3 a) { return mk(s * a.x, s * a.y, s * a.z); }
__host__ __device__ __forceinline__ d3 fma3(double s, d3 a, d3 b) {
  return mk(fma(s, a.x, b.x), fma(s, a.y, b.y), fma(s, a.z, b.z));
}
__host__ __device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ d3 cross(d3 a, d3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// 1 / sqrt(x): the device's reciprocal square root (one rounding step
// instead of a square root and a division)
__host__ __device__ __forceinline__ double inv_sqrt(double x) {
#ifdef __CUDA_ARCH__
  return rsqrt(x);
#else
  return 1.0 / sqrt(x);
#endif
}

// Quadratic Lagrange functions on the reference simplex with barycentrics
// l0 = 1 - xi - eta, l1 = xi, l2 = eta; node order v0 v1 v2 m01 m12 m20.
__host__ __device__ __forceinline__ void p2_eval(double xi, double eta, double N[6], double dxi[6],
                                        double deta[6]) {
  const double l0 = 1.0 - xi - eta, l1 = xi, l2 = eta;
  N[0] = l0 * (2.0 * l0 - 1.0);
  N[1] = l1 * (2.0 * l1 - 1.0);
  N[2] = l2 * (2.0 * l2 - 1.0);
  N[3] = 4.0 * l0 * l1;
  N[4] = 4.0 * l1 * l2;
  N[5] = 4.0 * l2 * l0;
  const double g0 = 4.0 * l0 - 1.0;
  dxi[0] = -g0;
  dxi[1] = 4.0 * l1 - 1.0;
  dxi[2] = 0.0;
  dxi[3] = 4.0 * (l0 - l1);
  dxi[4] = 4.0 * l2;
  dxi[5] = -4.0 * l2;
  deta[0] = -g0;
  deta[1] = 0.0;
  deta[2] = 4.0 * l2 - 1.0;
  deta[3] = -4.0 * l1;
  deta[4] = 4.0 * l1;
  deta[5] = 4.0 * (l0 - l2);
}

// Geometry and continuous frame at a parametric point (Sec. 3.3):
// X: 6 node positions, T1/T2: nodal t1/t2 of the 6 nodes.
struct PointGeo {
  d3 x, n, t1, t2, s1, s2;
  double J, gs;
  double N[6];
};

// normal, continuous frame and Jacobian from x, the covariant vectors a1, a2
// and the interpolated nodal frame vectors u1, u2 (Sec. 3.3)
__host__ __device__ __forceinline__ void frame_from(d3 x, d3 a1, d3 a2, d3 u1, d3 u2, PointGeo& g) {
  d3 c = cross(a1, a2);
  const double cc = dot(c, c);
  const double iJ = inv_sqrt(cc);
  const double J = cc * iJ;
  d3 n = scl(iJ, c);
  d3 p1 = sub(u1, scl(dot(n, u1), n));
  const double q1 = dot(p1, p1), i1 = inv_sqrt(q1);
  const double n1 = q1 * i1;
  d3 t1 = scl(i1, p1);
  d3 p2 = sub(u2, scl(dot(n, u2), n));
  p2 = sub(p2, scl(dot(t1, p2), t1));
  const double q2 = dot(p2, p2), i2 = inv_sqrt(q2);
  const double n2 = q2 * i2;
  d3 t2 = scl(i2, p2);
  g.x = x;
  g.n = n;
  g.t1 = t1;
  g.t2 = t2;
  g.s1 = cross(t1, n);
  g.s2 = cross(t2, n);
  g.J = J;
  g.gs = fmin(n1, n2);
}

__host__ __device__ __forceinline__ void point_geo(const d3* X, const d3* T1, const d3* T2, double xi,
                                          double eta, PointGeo& g) {
  double dxi[6], deta[6];
  p2_eval(xi, eta, g.N, dxi, deta);
  d3 x = mk(0, 0, 0), a1 = mk(0, 0, 0), a2 = mk(0, 0, 0), u1 = mk(0, 0, 0), u2 = mk(0, 0, 0);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    x = fma3(g.N[k], X[k], x);
    a1 = fma3(dxi[k], X[k], a1);
    a2 = fma3(deta[k], X[k], a2);
    u1 = fma3(g.N[k], T1[k], u1);
    u2 = fma3(g.N[k], T2[k], u2);
  }
  frame_from(x, a1, a2, u1, u2, g);
}

// Monomial coefficients of a P2 field with nodal values v (node order v0 v1
// v2 m01 m12 m20): f = c0 + c1 xi + c2 eta + c3 xi^2 + c4 xi eta + c5 eta^2.
__host__ __device__ __forceinline__ void p2_coef(const d3* v, d3* c) {
  c[0] = v[0];
  c[1] = add(add(scl(-3.0, v[0]), scl(-1.0, v[1])), scl(4.0, v[3]));
  c[2] = add(add(scl(-3.0, v[0]), scl(-1.0, v[2])), scl(4.0, v[5]));
  c[3] = add(add(scl(2.0, v[0]), scl(2.0, v[1])), scl(-4.0, v[3]));
  c[4] = scl(4.0, add(sub(v[0], v[3]), sub(v[4], v[5])));
  c[5] = add(add(scl(2.0, v[0]), scl(2.0, v[2])), scl(-4.0, v[5]));
}

__host__ __device__ __forceinline__ d3 p2_val(const d3* c, double xi, double eta) {
  const d3 a = fma3(xi, c[3], fma3(eta, c[4], c[1]));
  const d3 b = fma3(eta, c[5], c[2]);
  return fma3(xi, a, fma3(eta, b, c[0]));
}

// point_geo from monomial coefficients of the position (CX) and of the
// nodal frame fields (CU1, CU2): the same quantities, fewer operations
__host__ __device__ __forceinline__ void point_geo_c(const d3* CX, const d3* CU1, const d3* CU2,
                                            double xi, double eta, PointGeo& g) {
  const double l0 = 1.0 - xi - eta;
  g.N[0] = l0 * (2.0 * l0 - 1.0);
  g.N[1] = xi * (2.0 * xi - 1.0);
  g.N[2] = eta * (2.0 * eta - 1.0);
  g.N[3] = 4.0 * l0 * xi;
  g.N[4] = 4.0 * xi * eta;
  g.N[5] = 4.0 * eta * l0;
  const d3 x = p2_val(CX, xi, eta);
  const d3 a1 = fma3(2.0 * xi, CX[3], fma3(eta, CX[4], CX[1]));
  const d3 a2 = fma3(xi, CX[4], fma3(2.0 * eta, CX[5], CX[2]));
  frame_from(x, a1, a2, p2_val(CU1, xi, eta), p2_val(CU2, xi, eta), g);
}

// Point geometry for the Sauter-Schwab points (touching pairs), from
// monomial coefficients: x, n, t1 as in point_geo_c; t2 = sig (n x t1) with
// sig = sign((n x t1) . u2).  For orthonormal n, t1 the Gram-Schmidt vector
// of u2 against n and t1 is the unit vector orthogonal to both on the side
// of u2, i.e. exactly this one, so the frame is the one of Sec. 3.3 at about
// two thirds of the operations.  The co-normals need no storage either:
// s1 = t1 x n = -sig t2 and s2 = t2 x n = sig t1.
struct SSGeo {
  d3 x, n, t1, t2;
  double J, sig;
  double N[6];
};

__host__ __device__ __forceinline__ void ss_geo(const d3* CX, const d3* CU1, const d3* CU2,
                                                double xi, double eta, SSGeo& g) {
  const double l0 = 1.0 - xi - eta;
  g.N[0] = l0 * (2.0 * l0 - 1.0);
  g.N[1] = xi * (2.0 * xi - 1.0);
  g.N[2] = eta * (2.0 * eta - 1.0);
  g.N[3] = 4.0 * l0 * xi;
  g.N[4] = 4.0 * xi * eta;
  g.N[5] = 4.0 * eta * l0;
  g.x = p2_val(CX, xi, eta);
  const d3 a1 = fma3(2.0 * xi, CX[3], fma3(eta, CX[4], CX[1]));
  const d3 a2 = fma3(xi, CX[4], fma3(2.0 * eta, CX[5], CX[2]));
  const d3 c = cross(a1, a2);
  const double cc = dot(c, c);
  const double iJ = inv_sqrt(cc);
  g.J = cc * iJ;
  const d3 n = scl(iJ, c);
  const d3 u1 = p2_val(CU1, xi, eta);
  const d3 p1 = sub(u1, scl(dot(n, u1), n));
  const d3 t1 = scl(inv_sqrt(dot(p1, p1)), p1);
  const d3 m = cross(n, t1);
  g.sig = dot(m, p2_val(CU2, xi, eta)) < 0.0 ? -1.0 : 1.0;
  g.n = n;
  g.t1 = t1;
  g.t2 = scl(g.sig, m);
}

}  // namespace mu
