// Sauter-Schwab quadrature points (Sec. 4.2, Sec. 5.1): Duffy-type maps of
// the coincident (6 regions), common-edge (5) and common-vertex (2) triangle
// pairs onto [0,1]^4 with a tensor Gauss-Legendre rule of ns points per
// dimension (Sauter & Schwab, "Boundary Element Methods", Sec. 5.2).  The
// reference triangle is {0 <= v <= u <= 1}; the shared edge is v = 0 and
// the shared vertex (0,0) in both triangles; a point (u, v) is the
// relabelled parametric point (xi', eta') = (u - v, v).
#pragma once
#include <stdint.h>

namespace mu {

// Point (xu, xv) on the test triangle, (yu, yv) on the trial triangle and
// weight of region 'reg' of class cls (3 coincident, 2 common edge, 1 common
// vertex) at (xi, eta1, eta2, eta3), W the product of the four Gauss weights.
__host__ __device__ __forceinline__ void ss_point_val(int cls, int reg, double xi, double e1,
                                                      double e2, double e3, double W,
                                                      double& xu, double& xv, double& yu,
                                                      double& yv, double& w) {
  const double x3 = xi * xi * xi;
  if (cls == 3) {  // identical triangles: weight xi^3 e1^2 e2
    w = W * x3 * e1 * e1 * e2;
    switch (reg) {
      case 0: xu = xi; xv = xi * (1 - e1 + e1 * e2); yu = xi * (1 - e1 * e2 * e3); yv = xi * (1 - e1); break;
      case 1: xu = xi * (1 - e1 * e2 * e3); xv = xi * (1 - e1); yu = xi; yv = xi * (1 - e1 + e1 * e2); break;
      case 2: xu = xi; xv = xi * e1 * (1 - e2 + e2 * e3); yu = xi * (1 - e1 * e2); yv = xi * e1 * (1 - e2); break;
      case 3: xu = xi * (1 - e1 * e2); xv = xi * e1 * (1 - e2); yu = xi; yv = xi * e1 * (1 - e2 + e2 * e3); break;
      case 4: xu = xi * (1 - e1 * e2 * e3); xv = xi * e1 * (1 - e2 * e3); yu = xi; yv = xi * e1 * (1 - e2); break;
      default: xu = xi; xv = xi * e1 * (1 - e2); yu = xi * (1 - e1 * e2 * e3); yv = xi * e1 * (1 - e2 * e3); break;
    }
  } else if (cls == 2) {  // common edge v = 0
    const double j1 = W * x3 * e1 * e1;
    w = reg == 0 ? j1 : j1 * e2;
    switch (reg) {
      case 0: xu = xi; xv = xi * e1 * e3; yu = xi * (1 - e1 * e2); yv = xi * e1 * (1 - e2); break;
      case 1: xu = xi; xv = xi * e1; yu = xi * (1 - e1 * e2 * e3); yv = xi * e1 * e2 * (1 - e3); break;
      case 2: xu = xi * (1 - e1 * e2); xv = xi * e1 * (1 - e2); yu = xi; yv = xi * e1 * e2 * e3; break;
      case 3: xu = xi * (1 - e1 * e2 * e3); xv = xi * e1 * e2 * (1 - e3); yu = xi; yv = xi * e1; break;
      default: xu = xi * (1 - e1 * e2 * e3); xv = xi * e1 * (1 - e2 * e3); yu = xi; yv = xi * e1 * e2; break;
    }
  } else {  // common vertex (0, 0): weight xi^3 e2
    w = W * x3 * e2;
    if (reg == 0) {
      xu = xi; xv = xi * e1; yu = xi * e2; yv = xi * e2 * e3;
    } else {
      xu = xi * e2; xv = xi * e2 * e3; yu = xi; yv = xi * e1;
    }
  }
}


// the same at the Gauss-Legendre indices (a, b, c, d)
__host__ __device__ __forceinline__ void ss_point_idx(int cls, int reg, int a, int b, int c, int d,
                                                      const double* gl, const double* glw,
                                                      double& xu, double& xv, double& yu,
                                                      double& yv, double& w) {
  ss_point_val(cls, reg, gl[a], gl[b], gl[c], gl[d], glw[a] * glw[b] * glw[c] * glw[d], xu, xv,
               yu, yv, w);
}

// In every region the four point coordinates are affine in eta3 and the
// weight does not depend on it: for the ns points of a group (a, b, c, .)
// coords(eta3) = A + B eta3 and w = wb * glw[d].  A and B come from the map
// at eta3 = 0 and 1, wb with the weight product of the indices a, b, c.
__host__ __device__ __forceinline__ void ss_group_affine(int cls, int reg, int a, int b, int c,
                                                         const double* gl, const double* glw,
                                                         double A[4], double B[4], double& wb) {
  const double W3 = glw[a] * glw[b] * glw[c];
  double w1;
  ss_point_val(cls, reg, gl[a], gl[b], gl[c], 0.0, W3, A[0], A[1], A[2], A[3], wb);
  ss_point_val(cls, reg, gl[a], gl[b], gl[c], 1.0, W3, B[0], B[1], B[2], B[3], w1);
#pragma unroll
  for (int k = 0; k < 4; ++k) B[k] -= A[k];
}

// the same, for the flat index pt = ((((a*ns + b)*ns + c)*ns + d)*nreg + reg)
__host__ __device__ __forceinline__ void ss_point(int cls, int ns, int64_t pt, const double* gl,
                                                  const double* glw, double& xu, double& xv,
                                                  double& yu, double& yv, double& w) {
  const int nreg = cls == 3 ? 6 : (cls == 2 ? 5 : 2);
  const int reg = (int)(pt % nreg);
  int64_t rest = pt / nreg;
  const int d = (int)(rest % ns);
  rest /= ns;
  const int c = (int)(rest % ns);
  rest /= ns;
  const int b = (int)(rest % ns);
  const int a = (int)(rest / ns);
  ss_point_idx(cls, reg, a, b, c, d, gl, glw, xu, xv, yu, yv, w);
}

// In every region one of the two points does not depend on eta3 (index d):
// 1 = the test point x, 0 = the trial point y.  Points that differ only in
// d therefore share the geometry of that side.
__host__ __device__ __forceinline__ int ss_shared_x(int cls, int reg) {
  if (cls == 3) return (0x29 >> reg) & 1;  // regions 0, 3, 5
  if (cls == 2) return (0x06 >> reg) & 1;  // regions 1, 2
  return reg == 0;
}

// Regions whose shared side depends on (xi, eta1) only (Gauss indices a, b):
// common vertex, both regions; common edge, regions 1 and 3.  The ns groups
// (a, b, 0..ns-1) of such a region share the shared side's shape values, so
// their trial-side sums can be added before the contraction.
__host__ __device__ __forceinline__ bool ss_shared_ab(int cls, int reg) {
  if (cls == 1) return true;
  if (cls == 2) return reg == 1 || reg == 3;
  return false;
}

// relabelled reference point (u, v) -> canonical (xi, eta); perm holds the
// canonical corner of each relabelled corner in 2-bit fields
__host__ __device__ __forceinline__ void to_canonical(int perm, double u, double v, double& xi, double& eta) {
  const double lp[3] = {1.0 - u, u - v, v};
  double l[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) l[(perm >> (2 * k)) & 3] = lp[k];
  xi = l[1];
  eta = l[2];
}


}  // namespace mu
