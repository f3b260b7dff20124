// Nodal frame (Sec. 3.1-3.2) and regular-rule point geometry (Sec. 3.3).
#include <math.h>

#include "common.cuh"
#include "p2.cuh"

namespace mu {
namespace {

// Sec. 3.1 Eq. (U_contribution): one thread per node gathers
// U = (a1 x a2)/(g11 g22) from its elements in ascending element order.
// Corner nodes use the element relabelled so that the node is the
// parametric origin (derivatives along the two edges leaving it); edge
// nodes use the canonical d/dxi, d/deta.  Sec. 3.2: reference-axis rule and
// t1 = v_ref x n/|.|, t2 = n x t1.
__global__ void __launch_bounds__(128) frame_kernel(int64_t nn, const double* __restrict__ X,
                                                    const int32_t* __restrict__ T,
                                                    const int32_t* __restrict__ ptr,
                                                    const int32_t* __restrict__ n2e,
                                                    int frame_rule, double* __restrict__ frame) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double px[6] = {0.0, 1.0, 0.0, 0.5, 0.5, 0.0};
  const double py[6] = {0.0, 0.0, 1.0, 0.0, 0.5, 0.5};
  d3 U = mk(0, 0, 0);
  for (int32_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int32_t e = n2e[q] >> 3, k = n2e[q] & 7;
    double N[6], dxi[6], deta[6];
    p2_eval(px[k], py[k], N, dxi, deta);
    d3 A = mk(0, 0, 0), B = mk(0, 0, 0);
    for (int j = 0; j < 6; ++j) {
      const double* xj = X + 3 * (int64_t)T[6 * (int64_t)e + j];
      d3 p = mk(xj[0], xj[1], xj[2]);
      A = add(A, scl(dxi[j], p));
      B = add(B, scl(deta[j], p));
    }
    d3 a1, a2;
    if (k == 1) {  // origin at v1: edges v1->v2, v1->v0
      a1 = sub(B, A);
      a2 = scl(-1.0, A);
    } else if (k == 2) {  // origin at v2: edges v2->v0, v2->v1
      a1 = scl(-1.0, B);
      a2 = sub(A, B);
    } else {
      a1 = A;
      a2 = B;
    }
    const double w = 1.0 / (dot(a1, a1) * dot(a2, a2));
    U = add(U, scl(w, cross(a1, a2)));
  }
  const double un = sqrt(dot(U, U));
  d3 n = scl(1.0 / un, U);
  d3 ref;
  if (frame_rule == 1)
    ref = (fabs(n.z) > 1.0 - 1e-8) ? mk(1, 0, 0) : mk(0, 0, 1);
  else
    ref = (fabs(n.z) > 0.9) ? mk(1, 0, 0) : mk(0, 0, 1);
  d3 c = cross(ref, n);
  d3 t1 = scl(1.0 / sqrt(dot(c, c)), c);
  d3 t2 = cross(n, t1);
  double* f = frame + 9 * i;
  f[0] = n.x;
  f[1] = n.y;
  f[2] = n.z;
  f[3] = t1.x;
  f[4] = t1.y;
  f[5] = t1.z;
  f[6] = t2.x;
  f[7] = t2.y;
  f[8] = t2.z;
}

struct RuleArgs {
  double xi[MAX_Q], eta[MAX_Q], w[MAX_Q];
};

// Sec. 3.3: geometry and Gram-Schmidt frame at every regular-rule point,
// stored as x n t1 t2 s1 s2 W (W = w J).  Also the smallest Gram-Schmidt
// norm over all points (positive doubles order like their bit patterns).
__global__ void __launch_bounds__(128) quad_geometry_kernel(int64_t nt, int Q, RuleArgs rule,
                                                            const double* __restrict__ X,
                                                            const int32_t* __restrict__ T,
                                                            const double* __restrict__ frame,
                                                            double* __restrict__ qd64,
                                                            float* __restrict__ qd32,
                                                            unsigned long long* gs_min) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double gs = 1e300;
  if (t < nt * Q) {
    const int64_t e = t / Q;
    const int p = (int)(t % Q);
    d3 Xn[6], T1[6], T2[6];
    for (int k = 0; k < 6; ++k) {
      const int64_t v = T[6 * e + k];
      Xn[k] = mk(X[3 * v], X[3 * v + 1], X[3 * v + 2]);
      const double* f = frame + 9 * v;
      T1[k] = mk(f[3], f[4], f[5]);
      T2[k] = mk(f[6], f[7], f[8]);
    }
    PointGeo g;
    point_geo(Xn, T1, T2, rule.xi[p], rule.eta[p], g);
    double rec[QD_STRIDE] = {g.x.x,  g.x.y,  g.x.z,  g.n.x,  g.n.y,  g.n.z,  g.t1.x,
                             g.t1.y, g.t1.z, g.t2.x, g.t2.y, g.t2.z, g.s1.x, g.s1.y,
                             g.s1.z, g.s2.x, g.s2.y, g.s2.z, rule.w[p] * g.J, 0.0};
    for (int c = 0; c < QD_STRIDE; ++c) {
      qd64[t * QD_STRIDE + c] = rec[c];
      qd32[t * QD_STRIDE + c] = (float)rec[c];
    }
    gs = g.gs;
  }
  // block minimum
  __shared__ double red[128];
  red[threadIdx.x] = gs;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMin(gs_min, (unsigned long long)__double_as_longlong(red[0]));
}

}  // namespace

mueller_status launch_frame(mueller_mesh* m, int frame_rule, cudaStream_t s) {
  const int bs = 128;
  { Prof prof_("frame_kernel", s); frame_kernel<<<(unsigned)((m->nn + bs - 1) / bs), bs, 0, s>>>(m->nn, m->X, m->T, m->n2e_ptr,
                                                               m->n2e, frame_rule, m->frame); }
  MU_CHECK_LAUNCH("frame_kernel");
  return MUELLER_OK;
}

mueller_status launch_quad_geometry(mueller_mesh* m, const TriangleRule& rule, cudaStream_t s) {
  RuleArgs ra;
  for (int p = 0; p < rule.q; ++p) {
    ra.xi[p] = rule.xi[p];
    ra.eta[p] = rule.eta[p];
    ra.w[p] = rule.w[p];
  }
  const double big = 1e300;
  MU_CUDA(cudaMemcpyAsync(m->d_scal, &big, sizeof(double), cudaMemcpyHostToDevice, s));
  const int bs = 128;
  const int64_t n = m->nt * rule.q;
  { Prof prof_("quad_geometry_kernel", s); quad_geometry_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(
      m->nt, rule.q, ra, m->X, m->T, m->frame, m->qd64, m->qd32, (unsigned long long*)m->d_scal); }
  MU_CHECK_LAUNCH("quad_geometry_kernel");
  // 'big' lives on the host stack: make sure the copy above has consumed it
  MU_CUDA(cudaStreamSynchronize(s));
  return MUELLER_OK;
}

}  // namespace mu
