// Galerkin assembly of the Mueller system (Sec. 4, Sec. 5.1):
//   * regular_kernel  : every ordered pair of non-touching elements, product
//                       rule Q x Q, fused evaluation of the 12 kernel
//                       components (K1, K2^eps, K2^mu for the four alpha,
//                       beta) per point pair, FP64 or FP32;
//   * touching_kernel : coincident / common-edge / common-vertex pairs in
//                       FP64: singular parts (Eqs. kappa_S, kappa2_S) by
//                       Sauter-Schwab, remainder kappa - kappa^s by the
//                       product rule, plus the mass term on coincident pairs;
//   * rhs_kernel      : Eqs. rhs_E, rhs_H;
//   * mirror_kernel   : Z11 = -Z00 (both are +-(i/omega) K1).
// Contributions of element pairs meet in Z (or in the near blocks) through
// atomic additions.
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "p2.cuh"
#include "ssq.cuh"

namespace mu {

// ------------------------------------------------------------ rule tables
__constant__ double c_phi64[MAX_Q * 6];   // N_k at the regular-rule points
__constant__ float c_phi32[MAX_Q * 6];
__constant__ double c_rxi[MAX_Q], c_reta[MAX_Q], c_rw[MAX_Q];
__constant__ double c_gl[MAX_NS], c_glw[MAX_NS];  // Gauss-Legendre on [0,1]

static int g_uploaded_q = -1, g_uploaded_ns = -1;
static int g_uploaded_dev = -1;

mueller_status upload_rules(const TriangleRule& rule, int ns) {
  int dev = 0;
  MU_CUDA(cudaGetDevice(&dev));
  MU_CUDA(cis64_table_ready());  // the radial functions' exp(i theta) table
  if (rule.q == g_uploaded_q && ns == g_uploaded_ns && dev == g_uploaded_dev) return MUELLER_OK;
  double phi[MAX_Q * 6];
  float phif[MAX_Q * 6];
  for (int p = 0; p < rule.q; ++p) {
    const double l0 = 1.0 - rule.xi[p] - rule.eta[p], l1 = rule.xi[p], l2 = rule.eta[p];
    const double N[6] = {l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                         4 * l0 * l1,       4 * l1 * l2,       4 * l2 * l0};
    for (int k = 0; k < 6; ++k) {
      phi[p * 6 + k] = N[k];
      phif[p * 6 + k] = (float)N[k];
    }
  }
  std::vector<double> g, gw;
  gauss_legendre_unit(ns, g, gw);
  MU_CUDA(cudaMemcpyToSymbol(c_phi64, phi, sizeof(double) * rule.q * 6));
  MU_CUDA(cudaMemcpyToSymbol(c_phi32, phif, sizeof(float) * rule.q * 6));
  MU_CUDA(cudaMemcpyToSymbol(c_rxi, rule.xi.data(), sizeof(double) * rule.q));
  MU_CUDA(cudaMemcpyToSymbol(c_reta, rule.eta.data(), sizeof(double) * rule.q));
  MU_CUDA(cudaMemcpyToSymbol(c_rw, rule.w.data(), sizeof(double) * rule.q));
  MU_CUDA(cudaMemcpyToSymbol(c_gl, g.data(), sizeof(double) * ns));
  MU_CUDA(cudaMemcpyToSymbol(c_glw, gw.data(), sizeof(double) * ns));
  g_uploaded_q = rule.q;
  g_uploaded_ns = ns;
  g_uploaded_dev = dev;
  return MUELLER_OK;
}

namespace {

template <class R>
__device__ __forceinline__ R phi_at(int p, int k);
template <>
__device__ __forceinline__ double phi_at<double>(int p, int k) {
  return c_phi64[p * 6 + k];
}
template <>
__device__ __forceinline__ float phi_at<float>(int p, int k) {
  return c_phi32[p * 6 + k];
}

// complex accumulation into Z
__device__ __forceinline__ void zadd(double* Z, int64_t idx, double re, double im) {
  atomicAdd(Z + 2 * idx, re);
  atomicAdd(Z + 2 * idx + 1, im);
}
__device__ __forceinline__ void zadd(float* Z, int64_t idx, float re, float im) {
  atomicAdd(reinterpret_cast<float2*>(Z) + idx, make_float2(re, im));
}

template <class R>
__device__ __forceinline__ bool share_corner(const int32_t* a, const int32_t* b) {
  bool s = false;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s |= (a[i] == b[j]);
  return s;
}

// ------------------------------------------------------- regular pairs
// CTA: 4 warps, each owns one test element ex; the CTA shares a tile of TY
// trial elements staged in shared memory.  Per element pair a warp
//   1. evaluates the Q*Q point pairs (lanes over point pairs) into Kt[p][q][c],
//   2. contracts q -> j with the shape values (in place, lanes over (p, c)),
//   3. contracts p -> i and adds the 6 x 6 x 12 block into Z (lanes over (j, c)).
// Pair-tile shapes (test elements per CTA = warps, trial elements staged):
// the autotuner picks one per (precision, rule, mesh size).
constexpr int NSHAPE = 4;
constexpr int SHAPE_W[NSHAPE] = {4, 8, 2, 4};
constexpr int SHAPE_TY[NSHAPE] = {32, 16, 64, 16};
constexpr size_t kMaxRegSmem = 200 * 1024;

template <class R, int Q, int W_, int TY_>
struct RegCfg {
  static constexpr int TY = TY_;
  static constexpr int WARPS = W_;
  // element pairs a warp processes together (Q = 6: 4 x 36 point pairs fill
  // the lanes; Q = 12: 144 point pairs already do)
  static constexpr int NB = Q == 6 ? 4 : 1;
  static constexpr size_t smem =
      sizeof(R) * ((size_t)TY * Q * QD_STRIDE + (size_t)WARPS * Q * QD_STRIDE +
                   (size_t)WARPS * NB * Q * Q * 24) +
      sizeof(int) * (size_t)WARPS * TY;
};

// One CTA tile (test elements bx*WARPS.., trial elements by*TY..) of one body.
// WHICH = 0 adds the blocks into Z; WHICH = 1, 2 forms the blocks of dZ/deps_r,
// dZ/dmu_r and adds their product with x into y (complex128, length 2H)
// without forming the blocks: x is interpolated at the trial points, each
// lane sums one (test point, a, half) output in registers over the tile, and
// the 24 rows of the test element are added to y once per tile.
template <class R, int Q, int W, int TYT, int WHICH = 0>
__device__ __forceinline__ void regular_tile(int64_t bx, int64_t by, int64_t nt,
                                             const R* __restrict__ qd,
                                             const int32_t* __restrict__ T, const KConst<R>& K,
                                             R* __restrict__ Z, int64_t ldz, int64_t H,
                                             const double2* __restrict__ xd = nullptr,
                                             double2* __restrict__ yd = nullptr) {
  using C = RegCfg<R, Q, W, TYT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sY = reinterpret_cast<R*>(smem_raw);               // TY*Q*QD_STRIDE
  R* sX = sY + (size_t)C::TY * Q * QD_STRIDE;           // WARPS*Q*QD_STRIDE
  R* sK = sX + (size_t)C::WARPS * Q * QD_STRIDE;        // WARPS*Q*Q*24
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ex = bx * C::WARPS + warp;
  const int64_t ey0 = by * C::TY;
  const int ny = (int)((nt - ey0) < (int64_t)C::TY ? (nt - ey0) : (int64_t)C::TY);
  // stage the trial tile and the test elements
  for (int i = threadIdx.x; i < ny * Q * QD_STRIDE; i += blockDim.x)
    sY[i] = qd[ey0 * Q * QD_STRIDE + i];
  R* myX = sX + (size_t)warp * Q * QD_STRIDE;
  if (ex < nt)
    for (int i = lane; i < Q * QD_STRIDE; i += 32) myX[i] = qd[ex * Q * QD_STRIDE + i];
  __syncthreads();
  if (ex >= nt) return;
  int32_t tx[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) tx[k] = T[6 * ex + k];
  constexpr int NB = C::NB;
  R* Kt = sK + (size_t)warp * NB * Q * Q * 24;  // [b][p][q][c] complex (re, im)
  // Derivative mode contracts with x at the quadrature points instead of
  // forming the 6 x 6 x 12 blocks: per trial element u[q][bb][hx] =
  // sum_j N_j(q) x[2 ty_j + bb + hx H], and lane o = (p, a, h) of the test
  // element keeps A0 = sum K0[p][q][a bb] u[q][bb][h] and
  // A1 = sum K_{1+h}[p][q][a bb] u[q][bb][1-h] over the tile's trial elements.
  constexpr int NO = Q * 4;            // outputs (p, a, h)
  constexpr int NOL = (NO + 31) / 32;  // outputs per lane
  double dacc[NOL][4] = {};            // A0 re, im, A1 re, im
  double* su = nullptr;                // [b][q][bb][hx] complex
  if constexpr (WHICH != 0) {
    __shared__ double s_u[W][C::NB * Q * 8];
    su = s_u[warp];
  }
  int* myList = reinterpret_cast<int*>(sK + (size_t)C::WARPS * NB * Q * Q * 24) + warp * C::TY;
  const R wre = R(0), wim = R(1) / K.ka;   // i / omega
  // the trial elements of the tile that do not touch ex, compacted
  int cnt = 0;
  for (int base = 0; base < ny; base += 32) {
    const int yy = base + lane;
    bool ok = false;
    if (yy < ny) {
      int32_t ty[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) ty[k] = T[6 * (ey0 + yy) + k];
      ok = !share_corner<R>(tx, ty);  // touching pairs: touching_kernel
    }
    const unsigned msk = __ballot_sync(0xffffffffu, ok);
    if (ok) myList[cnt + __popc(msk & ((1u << lane) - 1u))] = yy;
    cnt += __popc(msk);
  }
  __syncwarp();
  for (int b0 = 0; b0 < cnt; b0 += NB) {
    const int nbb = cnt - b0 < NB ? cnt - b0 : NB;
    // 1. point pairs of nbb element pairs
    for (int it = lane; it < nbb * Q * Q; it += 32) {
      const int b = it / (Q * Q), pq = it % (Q * Q);
      const int p = pq / Q, q = pq % Q;
      const R* Y = sY + (size_t)myList[b0 + b] * Q * QD_STRIDE;
      cx<R> kv[12];
      point_pair<R, WHICH>(K, myX + p * QD_STRIDE, Y + q * QD_STRIDE, false, kv);
      R* o = Kt + (size_t)it * 24;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        o[2 * c] = kv[c].re;
        o[2 * c + 1] = kv[c].im;
      }
    }
    __syncwarp();
    if constexpr (WHICH != 0) {
      for (int it = lane; it < nbb * Q * 4; it += 32) {
        const int b = it / (Q * 4), r = it % (Q * 4);
        const int q = r >> 2, bb = (r >> 1) & 1, hx = r & 1;
        const int32_t* ty = T + 6 * (ey0 + myList[b0 + b]);
        double ur = 0, ui = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const double ph = phi_at<double>(q, j);
          const double2 xv = xd[2 * (int64_t)ty[j] + bb + (hx ? H : 0)];
          ur = fma(ph, xv.x, ur);
          ui = fma(ph, xv.y, ui);
        }
        su[2 * it] = ur;
        su[2 * it + 1] = ui;
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < NOL; ++k) {
        const int o = lane + 32 * k;
        if (o < NO) {
          const int p = o >> 2, a = (o >> 1) & 1, h = o & 1;
          for (int b = 0; b < nbb; ++b) {
            const R* Kb = Kt + ((size_t)b * Q * Q + (size_t)p * Q) * 24;
            const double* ub = su + (size_t)b * Q * 8;
            for (int q = 0; q < Q; ++q) {
#pragma unroll
              for (int bb = 0; bb < 2; ++bb) {
                const int c0 = 2 * a + bb, c1 = 4 * (1 + h) + 2 * a + bb;
                const double k0r = Kb[q * 24 + 2 * c0], k0i = Kb[q * 24 + 2 * c0 + 1];
                const double k1r = Kb[q * 24 + 2 * c1], k1i = Kb[q * 24 + 2 * c1 + 1];
                const double* u = ub + 2 * (q * 4 + 2 * bb);
                const double uhr = u[2 * h], uhi = u[2 * h + 1];
                const double uor = u[2 - 2 * h], uoi = u[3 - 2 * h];
                dacc[k][0] += k0r * uhr - k0i * uhi;
                dacc[k][1] += k0r * uhi + k0i * uhr;
                dacc[k][2] += k1r * uor - k1i * uoi;
                dacc[k][3] += k1r * uoi + k1i * uor;
              }
            }
          }
        }
      }
      __syncwarp();
      continue;
    }
    // 2. T[p][j][c] = sum_q Kt[p][q][c] N_j(q), written over Kt[p][j][c]
    for (int it = lane; it < nbb * Q * 12; it += 32) {
      const int b = it / (Q * 12), pc = it % (Q * 12);
      const int p = pc / 12, c = pc % 12;
      R* Kb = Kt + (size_t)b * Q * Q * 24;
      R vre[Q], vim[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        vre[q] = Kb[((size_t)p * Q + q) * 24 + 2 * c];
        vim[q] = Kb[((size_t)p * Q + q) * 24 + 2 * c + 1];
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        R are = 0, aim = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const R ph = phi_at<R>(q, j);
          are = fma(ph, vre[q], are);
          aim = fma(ph, vim[q], aim);
        }
        Kb[((size_t)p * Q + j) * 24 + 2 * c] = are;
        Kb[((size_t)p * Q + j) * 24 + 2 * c + 1] = aim;
      }
    }
    __syncwarp();
    // 3. L[i][j][c] = sum_p N_i(p) T[p][j][c]; scatter into Z
    for (int it = lane; it < nbb * 6 * 12; it += 32) {
      const int b = it / 72, jc = it % 72;
      const int j = jc / 12, c = jc % 12;
      const R* Kb = Kt + (size_t)b * Q * Q * 24;
      R vre[Q], vim[Q];
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        vre[p] = Kb[((size_t)p * Q + j) * 24 + 2 * c];
        vim[p] = Kb[((size_t)p * Q + j) * 24 + 2 * c + 1];
      }
      const int op = c >> 2, a = (c >> 1) & 1, bb = c & 1;
      const int64_t tyj = T[6 * (ey0 + myList[b0 + b]) + j];
      const int64_t col = 2 * tyj + bb + (op == 1 ? H : 0);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        R are = 0, aim = 0;
#pragma unroll
        for (int p = 0; p < Q; ++p) {
          const R ph = phi_at<R>(p, i);
          are = fma(ph, vre[p], are);
          aim = fma(ph, vim[p], aim);
        }
        const int64_t row = 2 * (int64_t)tx[i] + a + (op == 2 ? H : 0);
        if (op == 0) {  // (i/omega) K1
          const R zr = wre * are - wim * aim, zi = wre * aim + wim * are;
          zadd(Z, row * ldz + col, zr, zi);
        } else {
          zadd(Z, row * ldz + col, are, aim);
        }
      }
    }
    __syncwarp();
  }
  if constexpr (WHICH != 0) {
    // top rows: (i/omega) A0 + A1; bottom rows (Z11 = -Z00): -(i/omega) A0 + A1;
    // then y[row(i, a, h)] += sum_p N_i(p) acc[p][a][h]
    __shared__ double s_acc[W][NO * 2];
    double* acc = s_acc[warp];
#pragma unroll
    for (int k = 0; k < NOL; ++k) {
      const int o = lane + 32 * k;
      if (o < NO) {
        const double sg = (o & 1) ? -1.0 : 1.0, w = (double)wim;
        acc[2 * o] = dacc[k][2] - sg * w * dacc[k][1];
        acc[2 * o + 1] = dacc[k][3] + sg * w * dacc[k][0];
      }
    }
    __syncwarp();
    if (lane < 24) {
      const int i = lane >> 2, a = (lane >> 1) & 1, h = lane & 1;
      double vr = 0, vi = 0;
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        const double ph = phi_at<double>(p, i);
        vr = fma(ph, acc[2 * (p * 4 + 2 * a + h)], vr);
        vi = fma(ph, acc[2 * (p * 4 + 2 * a + h) + 1], vi);
      }
      const int64_t row = (h ? H : 0) + 2 * (int64_t)tx[i] + a;
      atomicAdd(&yd[row].x, vr);
      atomicAdd(&yd[row].y, vi);
    }
  }
}

template <class R, int Q, int W, int TYT>
__global__ void __launch_bounds__(32 * W) regular_kernel(int64_t nt, const R* __restrict__ qd,
                                                         const int32_t* __restrict__ T, KConst<R> K,
                                                         R* __restrict__ Z, int64_t ldz, int64_t H) {
  regular_tile<R, Q, W, TYT>(blockIdx.x, blockIdx.y, nt, qd, T, K, Z, ldz, H);
}

// y += (dZ/dtheta)_regular x (theta = eps_r for WHICH 1, mu_r for 2), FP64
template <int Q, int W, int TYT, int WHICH>
__global__ void __launch_bounds__(32 * W) regular_deriv_kernel(int64_t nt, const double* __restrict__ qd,
                                                               const int32_t* __restrict__ T,
                                                               KConst<double> K,
                                                               const double2* __restrict__ x,
                                                               double2* __restrict__ y, int64_t H) {
  regular_tile<double, Q, W, TYT, WHICH>(blockIdx.x, blockIdx.y, nt, qd, T, K, nullptr, 0, H, x, y);
}

// Many bodies in one launch: CTA t takes tile t - tile0 of the body whose
// range [tile0, tile0 + tiles) holds t (bodies listed with increasing tile0).
struct RegBody {
  int64_t nt, H, ldz, tile0, tiles_x;
  const void* qd;
  const int32_t* T;
  KConst<float> K32;
  KConst<double> K64;
  void* Z;
};

__device__ __forceinline__ int find_body(const int64_t* first, int nb, int64_t t) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <class R, int Q, int W, int TYT>
__global__ void __launch_bounds__(32 * W) regular_batch_kernel(const RegBody* __restrict__ bodies,
                                                               const int64_t* __restrict__ first,
                                                               int nb) {
  const int64_t t = blockIdx.x;
  const RegBody& B = bodies[find_body(first, nb, t)];
  const int64_t local = t - B.tile0;
  KConst<R> K;
  if constexpr (sizeof(R) == 4)
    K = B.K32;
  else
    K = B.K64;
  regular_tile<R, Q, W, TYT>(local % B.tiles_x, local / B.tiles_x, B.nt, (const R*)B.qd, B.T, K,
                             (R*)B.Z, B.ldz, B.H);
}

// ------------------------------------------------------- touching pairs
constexpr int TT = 96;  // threads per touching pair (= SSQ points per batch)
constexpr int kTouchMinBlocksCE = 3;  // CTAs per SM of the table-free launch

// Geometry record of one Sauter-Schwab point side in shared memory:
// x, n, t1, t2 (3 each), J, sig, N[6].
constexpr int GT = 20;
constexpr int MAX_TAB_NS = 5;  // vertex-pair tables: 2 (ns^2 + ns^3) records <= 48 KB

__device__ __forceinline__ void geo_store(double* t, const SSGeo& g) {
  const d3 v[4] = {g.x, g.n, g.t1, g.t2};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    t[3 * k] = v[k].x;
    t[3 * k + 1] = v[k].y;
    t[3 * k + 2] = v[k].z;
  }
  t[12] = g.J;
  t[13] = g.sig;
#pragma unroll
  for (int k = 0; k < 6; ++k) t[14 + k] = g.N[k];
}

__device__ __forceinline__ void geo_load(const double* t, SSGeo& g) {
  g.x = mk(t[0], t[1], t[2]);
  g.n = mk(t[3], t[4], t[5]);
  g.t1 = mk(t[6], t[7], t[8]);
  g.t2 = mk(t[9], t[10], t[11]);
  g.J = t[12];
  g.sig = t[13];
#pragma unroll
  for (int k = 0; k < 6; ++k) g.N[k] = t[14 + k];
}

// One Sauter-Schwab group: the ns points of region 'reg' at Gauss indices
// (a, b, c, 0..ns-1).  The side that does not depend on eta3 (x if SHX) is
// evaluated once; U receives its 6 shape values and V the 6 x 8 sums over the
// group of  W N_k(other) g_c  (g: the 8 singular geometric kernels).  Xn,
// T1, T2 hold the monomial coefficients of position and nodal frame.  With
// TAB the geometry of both sides is read from shared-memory records (tab_s:
// the shared side, tab_o: the other side, one record per eta3 index) instead
// of being evaluated.  The map is affine in eta3 (ss_group_affine).
template <bool SHX, bool TAB>
__device__ __forceinline__ void ssq_group(int cls, int reg, int a, int b, int c, int ns, int px,
                                          int py, const d3 (*Xn)[6], const d3 (*T1)[6],
                                          const d3 (*T2)[6], const double* tab_s,
                                          const double* tab_o, double* U, double* V) {
  double A[4], B[4], wb, xi, eta;
  ss_group_affine(cls, reg, a, b, c, c_gl, c_glw, A, B, wb);
  SSGeo gs;
  if (TAB) {
    geo_load(tab_s, gs);
  } else {
    if (SHX)
      to_canonical(px, A[0], A[1], xi, eta);
    else
      to_canonical(py, A[2], A[3], xi, eta);
    ss_geo(Xn[SHX ? 0 : 1], T1[SHX ? 0 : 1], T2[SHX ? 0 : 1], xi, eta, gs);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) U[i] = gs.N[i];
#pragma unroll
  for (int k = 0; k < 48; ++k) V[k] = 0.0;
  for (int d = 0; d < ns; ++d) {
    const double e3 = c_gl[d];
    const double w = wb * c_glw[d];
    SSGeo go;
    if (TAB) {
      geo_load(tab_o + d * GT, go);
    } else {
      if (SHX)
        to_canonical(py, fma(B[2], e3, A[2]), fma(B[3], e3, A[3]), xi, eta);
      else
        to_canonical(px, fma(B[0], e3, A[0]), fma(B[1], e3, A[1]), xi, eta);
      ss_geo(Xn[SHX ? 1 : 0], T1[SHX ? 1 : 0], T2[SHX ? 1 : 0], xi, eta, go);
    }
    const SSGeo& gx = SHX ? gs : go;
    const SSGeo& gy = SHX ? go : gs;
    const d3 Rv = sub(gx.x, gy.x);
    const double ir = inv_sqrt(dot(Rv, Rv));
    const d3 h = scl(ir, Rv);
    const double W = w * gx.J * gy.J;
    // kernels of Eqs. kappa_S, kappa2_S from the frame dot products; the
    // co-normals of x enter as s1 = -sig t2, s2 = sig t1
    const double nR = dot(gx.n, h);
    const double H0 = dot(h, gy.t1), H1 = dot(h, gy.t2);
    const double N0 = dot(gx.n, gy.t1), N1 = dot(gx.n, gy.t2);
    const double Q0 = dot(gx.t1, h), Q1 = dot(gx.t2, h);
    const double P00 = dot(gx.t1, gy.t1), P01 = dot(gx.t1, gy.t2);
    const double P10 = dot(gx.t2, gy.t1), P11 = dot(gx.t2, gy.t2);
    const double sir = gx.sig * ir, ir2 = ir * ir;
    double g[8];
    g[0] = -sir * fma(Q1, H0, P10);
    g[1] = -sir * fma(Q1, H1, P11);
    g[2] = sir * fma(Q0, H0, P00);
    g[3] = sir * fma(Q0, H1, P01);
    g[4] = fma(P00, nR, -Q0 * N0) * ir2;
    g[5] = fma(P01, nR, -Q0 * N1) * ir2;
    g[6] = fma(P10, nR, -Q1 * N0) * ir2;
    g[7] = fma(P11, nR, -Q1 * N1) * ir2;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double wn = W * go.N[k];
#pragma unroll
      for (int q = 0; q < 8; ++q) V[k * 8 + q] = fma(wn, g[q], V[k * 8 + q]);
    }
  }
}

// One touching element pair (index pid of the body's pair list) per CTA.
// WHICH = 1, 2: the pair's block of dZ/deps_r, dZ/dmu_r times x added into y
// (the Sauter-Schwab integrals do not depend on the material; only their
// constants, the remainder and the mass coefficient do).
template <int Q, int WHICH = 0>
__device__ __forceinline__ void touching_pair(
    int64_t pid, const TouchPair* __restrict__ tp, const double* __restrict__ X,
    const int32_t* __restrict__ T, const double* __restrict__ frame,
    const double* __restrict__ qd, int ns, const KConst<double>& K, double ae_re, double ae_im,
    double am_re, double am_im, int dtype, void* __restrict__ Zv, int64_t ldz, int64_t H,
    double* __restrict__ near, const int32_t* __restrict__ tp_slot, int use_tables,
    const double2* __restrict__ xd = nullptr, double2* __restrict__ yd = nullptr) {
  __shared__ d3 sXn[2][6], sT1[2][6], sT2[2][6];
  // common-vertex pairs: geometry records of the two sides (dynamic)
  extern __shared__ double sTab[];
  __shared__ double sG[6 * 48];
  __shared__ int sFlag[TT];
  // staging of the SSQ points (sU, sV), reused afterwards for the remainder
  // point pairs (sK, Q*Q*24 <= TT*54 doubles)
  __shared__ double sbuf[TT * 54];
  static_assert(MAX_Q * MAX_Q * 24 <= TT * 54, "remainder buffer must fit in the staging buffer");
  double(*sU)[6] = reinterpret_cast<double(*)[6]>(sbuf);
  double(*sV)[48] = reinterpret_cast<double(*)[48]>(sbuf + TT * 6);
  double* sK = sbuf;
  const TouchPair P = tp[pid];
  const int tid = threadIdx.x;
  if (tid < 12) {
    const int side = tid / 6, k = tid % 6;
    const int64_t e = side ? P.ey : P.ex;
    const int64_t v = T[6 * e + k];
    sXn[side][k] = mk(X[3 * v], X[3 * v + 1], X[3 * v + 2]);
    const double* f = frame + 9 * v;
    sT1[side][k] = mk(f[3], f[4], f[5]);
    sT2[side][k] = mk(f[6], f[7], f[8]);
  }
  __syncthreads();
  // nodal values -> monomial coefficients (in place; ss_geo reads them)
  if (tid < 6) {
    const int side = tid / 3, fld = tid % 3;
    d3* a = fld == 0 ? sXn[side] : (fld == 1 ? sT1[side] : sT2[side]);
    d3 v[6], c[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = a[k];
    p2_coef(v, c);
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = c[k];
  }
  __syncthreads();
  const int px = P.perm & 0x3f, py = (P.perm >> 8) & 0x3f;
  const int nreg = P.cls == 3 ? 6 : (P.cls == 2 ? 5 : 2);
  // In both common-vertex regions one side depends on (xi, eta1) only and the
  // other on (xi, eta2, eta3) only: ns^2 + ns^3 distinct points per region
  // instead of ns^3 + ns^4 evaluations.  Record index per region:
  // (a, b) -> a ns + b, (a, c, d) -> ns^2 + (a ns + c) ns + d.
  const bool tab = use_tables && P.cls == 1;
  const int tper = ns * ns + ns * ns * ns;
  if (tab) {
    for (int e = tid; e < 2 * tper; e += TT) {
      const int reg = e / tper, k = e % tper;
      const bool small = k < ns * ns;
      int a, b = 0, c = 0, d = 0;
      if (small) {
        a = k / ns;
        b = k % ns;
      } else {
        const int kk = k - ns * ns;
        a = kk / (ns * ns);
        c = (kk / ns) % ns;
        d = kk % ns;
      }
      double xu, xv, yu, yv, w, xi, eta;
      ss_point_idx(1, reg, a, b, c, d, c_gl, c_glw, xu, xv, yu, yv, w);
      const int side = ((reg == 0) == small) ? 0 : 1;  // 0: x, 1: y
      if (side == 0)
        to_canonical(px, xu, xv, xi, eta);
      else
        to_canonical(py, yu, yv, xi, eta);
      SSGeo g;
      ss_geo(sXn[side], sT1[side], sT2[side], xi, eta, g);
      geo_store(sTab + (size_t)e * GT, g);
    }
    __syncthreads();
  }
  // ---- singular parts by Sauter-Schwab (8 real geometric integrals).
  // Work unit: a group of ns points that differ only in eta3, so that one
  // side (x or y, ss_shared_x) is common to the group: its geometry is
  // evaluated once and the 48 trial-side values are summed over the group
  // before the 6 x 48 contraction (5x fewer multiply-adds).
  const int ngroups = nreg * ns * ns * ns;
  const int ns3 = ns * ns * ns;
  // batches of whole (region, a, b) sets of ns groups (ns divides ns^3)
  const int step = (TT / ns) * ns;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int base = 0; base < ngroups; base += step) {
    // region-major numbering keeps whole warps in one region (one branch)
    const int grp = base + tid;
    double* myV = sV[tid];
    int shx = 1;
    if (tid < step && grp < ngroups) {
      const int reg = grp / ns3;
      int rest = grp % ns3;
      const int ci = rest % ns;
      rest /= ns;
      const int bi = rest % ns;
      const int ai = rest / ns;
      shx = ss_shared_x(P.cls, reg);
      if (tab) {
        const double* ts = sTab + (size_t)(reg * tper + ai * ns + bi) * GT;
        const double* to = sTab + (size_t)(reg * tper + ns * ns + (ai * ns + ci) * ns) * GT;
        if (shx)
          ssq_group<true, true>(P.cls, reg, ai, bi, ci, ns, px, py, sXn, sT1, sT2, ts, to, sU[tid], myV);
        else
          ssq_group<false, true>(P.cls, reg, ai, bi, ci, ns, px, py, sXn, sT1, sT2, ts, to, sU[tid], myV);
      } else if (shx) {
        ssq_group<true, false>(P.cls, reg, ai, bi, ci, ns, px, py, sXn, sT1, sT2, nullptr, nullptr, sU[tid], myV);
      } else {
        ssq_group<false, false>(P.cls, reg, ai, bi, ci, ns, px, py, sXn, sT1, sT2, nullptr, nullptr, sU[tid], myV);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i) sU[tid][i] = 0.0;
#pragma unroll
      for (int c = 0; c < 48; ++c) myV[c] = 0.0;
    }
    sFlag[tid] = shx;
    __syncthreads();
    // where the shared side depends on (a, b) only, the ns groups of a set
    // have the same shape values U: their sums V are added into the first
    // record (all threads over (set, component)) and the others are skipped
    // by the contraction
    for (int e = tid; e < (step / ns) * 48; e += TT) {
      const int set = e / 48, c = e % 48;
      const int g0 = base + set * ns;
      if (g0 < ngroups && ss_shared_ab(P.cls, g0 / ns3)) {
        double v = sV[set * ns][c];
        for (int k = 1; k < ns; ++k) v += sV[set * ns + k][c];
        sV[set * ns][c] = v;
      }
    }
    if (tid < step && grp < ngroups && (grp % ns) != 0 && ss_shared_ab(P.cls, grp / ns3))
      sFlag[tid] = -1;
    __syncthreads();
    // G[i][j][c] += N_i(x) V[j][c]  (x shared)  or  V[i][c] N_j(y)  (y shared)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int o = tid + k * TT;  // output (i, j, c), 288 of them
      const int i = o / 48, jc = o % 48, j = jc >> 3, c = jc & 7;
      double s2 = acc[k];
      for (int q = 0; q < TT; ++q) {
        if (sFlag[q] < 0) continue;
        const bool fx = sFlag[q] != 0;
        const double u = sU[q][fx ? i : j];
        const double v = sV[q][fx ? jc : i * 8 + c];
        s2 = fma(u, v, s2);
      }
      acc[k] = s2;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) sG[tid + k * TT] = acc[k];
  // ---- remainder kappa - kappa^s by the product rule (Q x Q point pairs)
  const double* QX = qd + (int64_t)P.ex * Q * QD_STRIDE;
  const double* QY = qd + (int64_t)P.ey * Q * QD_STRIDE;
  for (int pq = tid; pq < Q * Q; pq += TT) {
    const int p = pq / Q, q = pq % Q;
    double px_[QD_STRIDE], qy_[QD_STRIDE];
#pragma unroll
    for (int c = 0; c < 19; ++c) {
      px_[c] = QX[p * QD_STRIDE + c];
      qy_[c] = QY[q * QD_STRIDE + c];
    }
    cx<double> kv[12];
    point_pair<double, WHICH>(K, px_, qy_, true, kv);
    for (int c = 0; c < 12; ++c) {
      sK[(size_t)pq * 24 + 2 * c] = kv[c].re;
      sK[(size_t)pq * 24 + 2 * c + 1] = kv[c].im;
    }
  }
  __syncthreads();
  for (int pc = tid; pc < Q * 12; pc += TT) {
    const int p = pc / 12, c = pc % 12;
    double vre[Q], vim[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      vre[q] = sK[((size_t)p * Q + q) * 24 + 2 * c];
      vim[q] = sK[((size_t)p * Q + q) * 24 + 2 * c + 1];
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double are = 0, aim = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        are = fma(c_phi64[q * 6 + j], vre[q], are);
        aim = fma(c_phi64[q * 6 + j], vim[q], aim);
      }
      sK[((size_t)p * Q + j) * 24 + 2 * c] = are;
      sK[((size_t)p * Q + j) * 24 + 2 * c + 1] = aim;
    }
  }
  __syncthreads();
  // ---- L = remainder + singular (+ mass on coincident pairs), scatter
  double C1re = (K.ka * K.ka - (K.ki_re * K.ki_re - K.ki_im * K.ki_im)) * 0.0397887357729738339422209408431285943;
  double C1im = -(2.0 * K.ki_re * K.ki_im) * 0.0397887357729738339422209408431285943;  // /(8 pi)
  double Cere = -(1.0 - K.eps_re) * 0.0795774715459476678844418816862571885;
  double Ceim = K.eps_im * 0.0795774715459476678844418816862571885;
  double Cmre = -(1.0 - K.mu_re) * 0.0795774715459476678844418816862571885;
  double Cmim = K.mu_im * 0.0795774715459476678844418816862571885;
  if constexpr (WHICH != 0) {
    // d/dtheta: C1 -> -ki dki / (4 pi), dki = ki / (2 theta); C_chi -> 1/(4 pi)
    // for chi = theta, else 0; the mass coefficient a_chi -> 1/2, else 0
    const cx<double> ki = cmk(K.ki_re, K.ki_im);
    const cx<double> th = WHICH == 1 ? cmk(K.eps_re, K.eps_im) : cmk(K.mu_re, K.mu_im);
    const cx<double> kdk = cmul(ki, crs(0.5, cdivc(ki, th)));
    C1re = -kdk.re * 0.0795774715459476678844418816862571885;
    C1im = -kdk.im * 0.0795774715459476678844418816862571885;
    Cere = WHICH == 1 ? 0.0795774715459476678844418816862571885 : 0.0;
    Cmre = WHICH == 2 ? 0.0795774715459476678844418816862571885 : 0.0;
    Ceim = Cmim = 0.0;
    ae_re = WHICH == 1 ? 0.5 : 0.0;
    am_re = WHICH == 2 ? 0.5 : 0.0;
    ae_im = am_im = 0.0;
  }
  const double wim = 1.0 / K.ka;  // i / omega
  for (int jc = tid; jc < 6 * 12; jc += TT) {
    const int j = jc / 12, c = jc % 12;
    const int op = c >> 2, a = (c >> 1) & 1, b = c & 1, ab = c & 3;
    double vre[Q], vim[Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      vre[p] = sK[((size_t)p * Q + j) * 24 + 2 * c];
      vim[p] = sK[((size_t)p * Q + j) * 24 + 2 * c + 1];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double are = 0, aim = 0;
#pragma unroll
      for (int p = 0; p < Q; ++p) {
        are = fma(c_phi64[p * 6 + i], vre[p], are);
        aim = fma(c_phi64[p * 6 + i], vim[p], aim);
      }
      // singular part
      if (op == 0) {
        const double g = sG[i * 48 + j * 8 + ab];
        are += C1re * g;
        aim += C1im * g;
      } else {
        const double g = sG[i * 48 + j * 8 + 4 + ab];
        are += (op == 1 ? Cere : Cmre) * g;
        aim += (op == 1 ? Ceim : Cmim) * g;
      }
      // mass (Eq. mass_matrix) on coincident pairs: a_chi delta_ab int N_i N_j
      if (P.cls == 3 && op > 0 && a == b) {
        double mij = 0.0;
        for (int p = 0; p < Q; ++p) mij += QX[p * QD_STRIDE + 18] * c_phi64[p * 6 + i] * c_phi64[p * 6 + j];
        are += (op == 1 ? ae_re : am_re) * mij;
        aim += (op == 1 ? ae_im : am_im) * mij;
      }
      if (op == 0) {  // times i / omega
        const double t = are;
        are = -wim * aim;
        aim = wim * t;
      }
      if constexpr (WHICH != 0) {
        const int64_t row = 2 * (int64_t)T[6 * P.ex + i] + a + (op == 2 ? H : 0);
        const int64_t col = 2 * (int64_t)T[6 * P.ey + j] + b + (op == 1 ? H : 0);
        const double2 xv = xd[col];
        atomicAdd(&yd[row].x, are * xv.x - aim * xv.y);
        atomicAdd(&yd[row].y, are * xv.y + aim * xv.x);
        if (op == 0) {  // Z11 = -Z00
          const double2 xb = xd[col + H];
          atomicAdd(&yd[row + H].x, -(are * xb.x - aim * xb.y));
          atomicAdd(&yd[row + H].y, -(are * xb.y + aim * xb.x));
        }
      } else if (dtype == MUELLER_C128) {
        double* Z = (double*)Zv;
        const int64_t row = 2 * (int64_t)T[6 * P.ex + i] + a + (op == 2 ? H : 0);
        const int64_t col = 2 * (int64_t)T[6 * P.ey + j] + b + (op == 1 ? H : 0);
        zadd(Z, row * ldz + col, are, aim);
      } else {
        // near block [h][alpha][g][beta]; K1 goes to (0,0) and, negated, (1,1)
        const int64_t slot = tp_slot[pid * 36 + i * 6 + j];
        double* blk = near + slot * 32;
        if (op == 0) {
          zadd(blk, ((0 * 2 + a) * 2 + 0) * 2 + b, are, aim);
          zadd(blk, ((1 * 2 + a) * 2 + 1) * 2 + b, -are, -aim);
        } else if (op == 1) {
          zadd(blk, ((0 * 2 + a) * 2 + 1) * 2 + b, are, aim);
        } else {
          zadd(blk, ((1 * 2 + a) * 2 + 0) * 2 + b, are, aim);
        }
      }
    }
  }
}

// CTA b takes pair order[off + b] (n pairs in this launch).  MINB CTAs per
// SM: 3 for the coincident and common-edge pairs (no tables: the static
// shared memory allows it, the register cap costs some spills), 2 with the
// common-vertex tables.
template <int Q, int MINB>
__global__ void __launch_bounds__(TT, MINB) touching_kernel(
    int64_t n, const int32_t* __restrict__ order, int64_t off, const TouchPair* __restrict__ tp,
    const double* __restrict__ X, const int32_t* __restrict__ T, const double* __restrict__ frame,
    const double* __restrict__ qd, int ns, KConst<double> K, double ae_re, double ae_im,
    double am_re, double am_im, int dtype, void* __restrict__ Zv, int64_t ldz, int64_t H,
    double* __restrict__ near, const int32_t* __restrict__ tp_slot, int use_tables) {
  if ((int64_t)blockIdx.x >= n) return;
  touching_pair<Q>(order[off + blockIdx.x], tp, X, T, frame, qd, ns, K, ae_re, ae_im, am_re,
                   am_im, dtype, Zv, ldz, H, near, tp_slot, use_tables);
}

struct TouchBody {
  int64_t n_touch, pair0, H, ldz;
  const int32_t* order;  // the body's pairs of this launch: order[0 .. n_touch)
  const TouchPair* tp;
  const double* X;
  const int32_t* T;
  const double* frame;
  const double* qd;
  const int32_t* tp_slot;
  KConst<double> K;
  double ae_re, ae_im, am_re, am_im;
  void* Z;
  double* near;
};

// Many bodies in one launch: CTA t takes pair order[t - pair0] of its body
// (one launch per pair class, as for one body).
template <int Q, int MINB>
__global__ void __launch_bounds__(TT, MINB) touching_batch_kernel(const TouchBody* __restrict__ bodies,
                                                                  const int64_t* __restrict__ first,
                                                                  int nb, int ns, int dtype,
                                                                  int use_tables) {
  const int64_t t = blockIdx.x;
  const TouchBody& B = bodies[find_body(first, nb, t)];
  touching_pair<Q>(B.order[t - B.pair0], B.tp, B.X, B.T, B.frame, B.qd, ns, B.K, B.ae_re,
                   B.ae_im, B.am_re, B.am_im, dtype, B.Z, B.ldz, B.H, B.near, B.tp_slot,
                   use_tables);
}

// y += (dZ/dtheta)_touching x over all touching pairs (CTA per pair)
template <int Q, int WHICH>
__global__ void __launch_bounds__(TT, 2) touching_deriv_kernel(
    int64_t n_touch, const TouchPair* __restrict__ tp, const double* __restrict__ X,
    const int32_t* __restrict__ T, const double* __restrict__ frame,
    const double* __restrict__ qd, int ns, KConst<double> K, int64_t H, int use_tables,
    const double2* __restrict__ x, double2* __restrict__ y) {
  if ((int64_t)blockIdx.x >= n_touch) return;
  touching_pair<Q, WHICH>(blockIdx.x, tp, X, T, frame, qd, ns, K, 0.0, 0.0, 0.0, 0.0,
                          MUELLER_C128, nullptr, 0, H, nullptr, nullptr, use_tables, x, y);
}

// Eqs. (rhs_E), (rhs_H): one thread per (RHS, element, local node).
__global__ void rhs_kernel(int64_t nt, int Q, const double* __restrict__ qd,
                           const int32_t* __restrict__ T, const double* __restrict__ inc, int r,
                           double ka, int64_t N, double* __restrict__ B) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * nt * 6) return;
  const int i = (int)(t % 6);
  const int64_t e = (t / 6) % nt;
  const int s = (int)(t / (6 * nt));
  const double* w = inc + 6 * s;
  const d3 k = mk(w[0], w[1], w[2]), pp = mk(w[3], w[4], w[5]);
  const d3 h = cross(k, pp);
  double bE[2][2] = {{0, 0}, {0, 0}}, bH[2][2] = {{0, 0}, {0, 0}};
  for (int p = 0; p < Q; ++p) {
    const double* rec = qd + (e * Q + p) * QD_STRIDE;
    double sn, cs;
    sincos(ka * (k.x * rec[0] + k.y * rec[1] + k.z * rec[2]), &sn, &cs);
    const double wn = rec[18] * c_phi64[p * 6 + i];
    for (int a = 0; a < 2; ++a) {
      const d3 s_ = mk(rec[12 + 3 * a], rec[13 + 3 * a], rec[14 + 3 * a]);
      const double ce = -wn * dot(s_, pp), ch = wn * dot(s_, h);
      bE[a][0] += ce * cs;
      bE[a][1] += ce * sn;
      bH[a][0] += ch * cs;
      bH[a][1] += ch * sn;
    }
  }
  const int64_t node = T[6 * e + i];
  double* b = B + 2 * (int64_t)s * N;
  for (int a = 0; a < 2; ++a) {
    zadd(b, 2 * node + a, bE[a][0], bE[a][1]);
    zadd(b, N / 2 + 2 * node + a, bH[a][0], bH[a][1]);
  }
}

template <class R>
__global__ void mirror_kernel(int64_t H, R* __restrict__ Z, int64_t ldz) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= H * H) return;
  const int64_t r = t / H, c = t % H;
  const int64_t src = r * ldz + c, dst = (H + r) * ldz + H + c;
  Z[2 * dst] = -Z[2 * src];
  Z[2 * dst + 1] = -Z[2 * src + 1];
}

template <class R>
KConst<R> kconst(const PhysConsts& P) {
  KConst<R> K;
  K.ka = (R)P.ka;
  K.ki_re = (R)P.ki_re;
  K.ki_im = (R)P.ki_im;
  K.eps_re = (R)P.eps_re;
  K.eps_im = (R)P.eps_im;
  K.mu_re = (R)P.mu_re;
  K.mu_im = (R)P.mu_im;
  K.sing = 0;
  return K;
}

// one single-body launch of pair-tile shape S (false if it does not fit)
template <class R, int Q, int S>
bool regular_shape_launch(int64_t nt, const R* qd, const int32_t* T, const KConst<R>& K, R* Z,
                          int64_t ldz, int64_t H, cudaStream_t s) {
  constexpr int W = SHAPE_W[S], TYT = SHAPE_TY[S];
  using C = RegCfg<R, Q, W, TYT>;
  if (C::smem > kMaxRegSmem) return false;
  auto kern = regular_kernel<R, Q, W, TYT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem) != cudaSuccess)
    return false;
  dim3 grid((unsigned)((nt + W - 1) / W), (unsigned)((nt + TYT - 1) / TYT));
  { Prof prof_("regular_kernel<R,Q>", s); kern<<<grid, 32 * W, C::smem, s>>>(nt, qd, T, K, Z, ldz, H); }
  return true;
}

template <class R, int Q>
bool regular_launch(int shape, int64_t nt, const R* qd, const int32_t* T, const KConst<R>& K, R* Z,
                    int64_t ldz, int64_t H, cudaStream_t s) {
  switch (shape) {
    case 0: return regular_shape_launch<R, Q, 0>(nt, qd, T, K, Z, ldz, H, s);
    case 1: return regular_shape_launch<R, Q, 1>(nt, qd, T, K, Z, ldz, H, s);
    case 2: return regular_shape_launch<R, Q, 2>(nt, qd, T, K, Z, ldz, H, s);
    default: return regular_shape_launch<R, Q, 3>(nt, qd, T, K, Z, ldz, H, s);
  }
}

template <class R, int Q>
constexpr int default_shape() {
  return RegCfg<R, Q, SHAPE_W[0], SHAPE_TY[0]>::smem <= kMaxRegSmem ? 0 : 3;
}

// Autotuner of the regular-pair tile shape, per (precision, rule, mesh size
// rounded up to a power of two).  MUELLER_REGULAR_TILE = 0..3 forces a shape,
// MUELLER_AUTOTUNE = 0 keeps the default one.  Tuning times every shape that
// fits once on the caller's mesh (adding into its Z, which is zeroed again
// afterwards) and remembers the fastest for the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int64_t>, int> g_tuned;

int forced_shape() {
  const char* e = getenv("MUELLER_REGULAR_TILE");
  if (!e || !*e) return -1;
  const int v = atoi(e);
  return v >= 0 && v < NSHAPE ? v : -1;
}

template <class R, int Q>
mueller_status regular_shape_for(int64_t nt, const R* qd, const int32_t* T, const KConst<R>& K,
                                 R* Z, int64_t ldz, int64_t H, cudaStream_t s, int* shape) {
  const int f = forced_shape();
  if (f >= 0) {
    *shape = f;
    return MUELLER_OK;
  }
  const char* a = getenv("MUELLER_AUTOTUNE");
  if (a && a[0] == '0') {
    *shape = default_shape<R, Q>();
    return MUELLER_OK;
  }
  int64_t bucket = 1;
  while (bucket < nt) bucket <<= 1;
  const auto key = std::make_tuple((int)sizeof(R), Q, bucket);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(key);
  if (it != g_tuned.end()) {
    *shape = it->second;
    return MUELLER_OK;
  }
  cudaEvent_t e0, e1;
  MU_CUDA(cudaEventCreate(&e0));
  MU_CUDA(cudaEventCreate(&e1));
  int best = default_shape<R, Q>();
  float best_ms = 1e30f;
  for (int sh = 0; sh < NSHAPE; ++sh) {
    if (!regular_launch<R, Q>(sh, nt, qd, T, K, Z, ldz, H, s)) continue;  // warm-up
    MU_CUDA(cudaEventRecord(e0, s));
    regular_launch<R, Q>(sh, nt, qd, T, K, Z, ldz, H, s);
    MU_CUDA(cudaEventRecord(e1, s));
    MU_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    MU_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = sh;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MU_CHECK_LAUNCH("regular_kernel (tuning)");
  MU_CUDA(cudaMemsetAsync(Z, 0, (size_t)(2 * H) * ldz * 2 * sizeof(R), s));
  g_tuned[key] = best;
  *shape = best;
  return MUELLER_OK;
}

template <class R, int Q>
mueller_status launch_regular_t(mueller_mesh* m, const PhysConsts& P, R* Z, int64_t ldz,
                                cudaStream_t s) {
  const R* qd;
  if constexpr (sizeof(R) == 8)
    qd = m->qd64;
  else
    qd = m->qd32;
  const KConst<R> K = kconst<R>(P);
  int shape = 0;
  mueller_status st = regular_shape_for<R, Q>(m->nt, qd, m->T, K, Z, ldz, 2 * m->nn, s, &shape);
  if (st) return st;
  if (!regular_launch<R, Q>(shape, m->nt, qd, m->T, K, Z, ldz, 2 * m->nn, s)) {
    set_error("regular-pair tile shape does not fit in shared memory");
    return MUELLER_ERR_INVALID_ARG;
  }
  MU_CHECK_LAUNCH("regular_kernel");
  return MUELLER_OK;
}

template <class R, int Q>
mueller_status tune_regular_t(mueller_mesh* m, const PhysConsts& P, R* Z, int64_t ldz,
                              cudaStream_t s) {
  const R* qd;
  if constexpr (sizeof(R) == 8)
    qd = m->qd64;
  else
    qd = m->qd32;
  int shape = 0;
  return regular_shape_for<R, Q>(m->nt, qd, m->T, kconst<R>(P), Z, ldz, 2 * m->nn, s, &shape);
}

}  // namespace

mueller_status tune_regular(mueller_mesh* m, const PhysConsts& P, int Q, int dtype, void* Z,
                            int64_t ldz, cudaStream_t s) {
  if (dtype == MUELLER_C128) {
    return Q == 6 ? tune_regular_t<double, 6>(m, P, (double*)Z, ldz, s)
                  : tune_regular_t<double, 12>(m, P, (double*)Z, ldz, s);
  }
  return Q == 6 ? tune_regular_t<float, 6>(m, P, (float*)Z, ldz, s)
                : tune_regular_t<float, 12>(m, P, (float*)Z, ldz, s);
}

// One high-priority side stream per device, for work that runs beside the
// caller's stream: the touching-pair kernel next to the regular-pair kernel,
// the panel chain of the block LU next to its trailing updates.  (Two grids
// share SMs mainly where one grid's last CTAs leave room: CTAs of a grid
// that still has CTAs waiting for dispatch keep the other grid's CTAs out.)
static std::mutex g_side_mu;
static cudaStream_t g_side[64] = {};

mueller_status side_stream(cudaStream_t* out) {
  int dev = 0;
  MU_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device index out of range for the side stream");
    return MUELLER_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_side_mu);
  if (!g_side[dev]) {
    int lo = 0, hi = 0;
    MU_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    MU_CUDA(cudaStreamCreateWithPriority(&g_side[dev], cudaStreamNonBlocking, hi));
  }
  *out = g_side[dev];
  return MUELLER_OK;
}

// s2 waits for the work queued on s so far (fork), or s for s2 (join)
mueller_status stream_order(cudaStream_t before, cudaStream_t after) {
  cudaEvent_t ev;
  MU_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, before);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(after, ev, 0);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
  return MUELLER_OK;
}

mueller_status launch_regular(mueller_mesh* m, const PhysConsts& P, int Q, int dtype, void* Z,
                              int64_t ldz, cudaStream_t s) {
  if (dtype == MUELLER_C128) {
    return Q == 6 ? launch_regular_t<double, 6>(m, P, (double*)Z, ldz, s)
                  : launch_regular_t<double, 12>(m, P, (double*)Z, ldz, s);
  }
  return Q == 6 ? launch_regular_t<float, 6>(m, P, (float*)Z, ldz, s)
                : launch_regular_t<float, 12>(m, P, (float*)Z, ldz, s);
}

mueller_status launch_touching(mueller_mesh* m, const PhysConsts& P, int Q, int ns, int dtype,
                               void* Z, int64_t ldz, void* near, cudaStream_t s) {
  if (m->n_touch == 0) return MUELLER_OK;
  const double ae_re = 0.5 * (P.eps_re + 1.0), ae_im = 0.5 * P.eps_im;
  const double am_re = 0.5 * (P.mu_re + 1.0), am_im = 0.5 * P.mu_im;
  auto kern_ce = Q == 6 ? touching_kernel<6, kTouchMinBlocksCE> : touching_kernel<12, kTouchMinBlocksCE>;
  auto kern_v = Q == 6 ? touching_kernel<6, 2> : touching_kernel<12, 2>;
  const int use_tables = ns <= MAX_TAB_NS ? 1 : 0;
  const size_t tab_bytes = use_tables ? (size_t)2 * (ns * ns + ns * ns * ns) * GT * sizeof(double) : 0;
  MU_CUDA(cudaFuncSetAttribute(kern_v, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab_bytes));
  MU_CUDA(cudaFuncSetAttribute(kern_ce, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  // coincident and common-edge pairs (no tables), then common-vertex pairs
  const int64_t n_ce = m->n_touch_ce, n_v = m->n_touch - m->n_touch_ce;
  if (n_ce > 0)
    { Prof prof_("touching_kernel<Q>", s); kern_ce<<<(unsigned)n_ce, TT, 0, s>>>(n_ce, m->tp_order, 0, m->tp, m->X, m->T, m->frame, m->qd64, ns,
                                            kconst<double>(P), ae_re, ae_im, am_re, am_im, dtype,
                                            Z, ldz, 2 * m->nn, (double*)near, m->tp_slot, 0); }
  if (n_v > 0)
    { Prof prof_("touching_kernel<Q>", s); kern_v<<<(unsigned)n_v, TT, tab_bytes, s>>>(n_v, m->tp_order, n_ce, m->tp, m->X, m->T, m->frame, m->qd64, ns,
                                            kconst<double>(P), ae_re, ae_im, am_re, am_im, dtype,
                                            Z, ldz, 2 * m->nn, (double*)near, m->tp_slot, use_tables); }
  MU_CHECK_LAUNCH("touching_kernel");
  return MUELLER_OK;
}

namespace {

// bodies in decreasing order of work, so that the large ones start first
template <class W>
std::vector<int> by_decreasing(int nb, W work) {
  std::vector<int> order(nb);
  for (int b = 0; b < nb; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
  return order;
}

template <class Body>
mueller_status upload_bodies(const std::vector<Body>& bodies, const std::vector<int64_t>& first,
                             void** buf, Body** d_bodies, int64_t** d_first, cudaStream_t s) {
  const size_t nb = bodies.size();
  const size_t bytes_b = (nb * sizeof(Body) + 255) & ~size_t(255);
  MU_CUDA(cudaMallocAsync(buf, bytes_b + nb * sizeof(int64_t), s));
  *d_bodies = (Body*)*buf;
  *d_first = (int64_t*)((char*)*buf + bytes_b);
  // pageable sources: the copies have consumed them when the calls return
  MU_CUDA(cudaMemcpyAsync(*d_bodies, bodies.data(), nb * sizeof(Body), cudaMemcpyHostToDevice, s));
  MU_CUDA(cudaMemcpyAsync(*d_first, first.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  return MUELLER_OK;
}

template <class R, int Q, int S>
mueller_status regular_batch_shape(int nb, mueller_mesh* const* meshes, const PhysConsts* P,
                                   void* const* Z, const int64_t* ldz, cudaStream_t s) {
  constexpr int W = SHAPE_W[S], TYT = SHAPE_TY[S];
  using C = RegCfg<R, Q, W, TYT>;
  std::vector<int> order = by_decreasing(nb, [&](int b) { return meshes[b]->nt; });
  std::vector<RegBody> bodies;
  std::vector<int64_t> first;
  int64_t tiles = 0;
  for (int b : order) {
    const mueller_mesh* m = meshes[b];
    RegBody B;
    B.nt = m->nt;
    B.H = 2 * m->nn;
    B.ldz = ldz[b];
    B.tiles_x = (m->nt + W - 1) / W;
    B.tile0 = tiles;
    B.qd = sizeof(R) == 8 ? (const void*)m->qd64 : (const void*)m->qd32;
    B.T = m->T;
    B.K32 = kconst<float>(P[b]);
    B.K64 = kconst<double>(P[b]);
    B.Z = Z[b];
    bodies.push_back(B);
    first.push_back(tiles);
    tiles += B.tiles_x * ((m->nt + TYT - 1) / TYT);
  }
  void* buf = nullptr;
  RegBody* d_bodies = nullptr;
  int64_t* d_first = nullptr;
  mueller_status st = upload_bodies(bodies, first, &buf, &d_bodies, &d_first, s);
  if (st) return st;
  auto kern = regular_batch_kernel<R, Q, W, TYT>;
  MU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem));
  { Prof prof_("regular_batch_kernel<R,Q>", s); kern<<<(unsigned)tiles, 32 * W, C::smem, s>>>(d_bodies, d_first, nb); }
  MU_CHECK_LAUNCH("regular_batch_kernel");
  cudaFreeAsync(buf, s);
  return MUELLER_OK;
}

// the shape tuned for the largest body (tuning on it if needed)
template <class R, int Q>
mueller_status regular_batch_t(int nb, mueller_mesh* const* meshes, const PhysConsts* P,
                               void* const* Z, const int64_t* ldz, cudaStream_t s) {
  int big = 0;
  for (int b = 1; b < nb; ++b)
    if (meshes[b]->nt > meshes[big]->nt) big = b;
  const mueller_mesh* m = meshes[big];
  const R* qd = sizeof(R) == 8 ? (const R*)(const void*)m->qd64 : (const R*)(const void*)m->qd32;
  int shape = 0;
  mueller_status st = regular_shape_for<R, Q>(m->nt, qd, m->T, kconst<R>(P[big]), (R*)Z[big],
                                              ldz[big], 2 * m->nn, s, &shape);
  if (st) return st;
  switch (shape) {
    case 0: return regular_batch_shape<R, Q, 0>(nb, meshes, P, Z, ldz, s);
    case 1: return regular_batch_shape<R, Q, 1>(nb, meshes, P, Z, ldz, s);
    case 2: return regular_batch_shape<R, Q, 2>(nb, meshes, P, Z, ldz, s);
    default: return regular_batch_shape<R, Q, 3>(nb, meshes, P, Z, ldz, s);
  }
}

template <int Q, int MINB>
mueller_status touching_batch_class(int nb, mueller_mesh* const* meshes, const PhysConsts* P,
                                    int ns, int dtype, void* const* Z, const int64_t* ldz,
                                    void* const* near, bool vertex, cudaStream_t s) {
  auto count = [&](const mueller_mesh* m) {
    return vertex ? m->n_touch - m->n_touch_ce : m->n_touch_ce;
  };
  std::vector<int> order = by_decreasing(nb, [&](int b) { return count(meshes[b]); });
  std::vector<TouchBody> bodies;
  std::vector<int64_t> first;
  int64_t pairs = 0;
  for (int b : order) {
    const mueller_mesh* m = meshes[b];
    const int64_t n = count(m);
    if (n == 0) continue;
    TouchBody B;
    B.n_touch = n;
    B.pair0 = pairs;
    B.H = 2 * m->nn;
    B.ldz = ldz[b];
    B.order = m->tp_order + (vertex ? m->n_touch_ce : 0);
    B.tp = m->tp;
    B.X = m->X;
    B.T = m->T;
    B.frame = m->frame;
    B.qd = m->qd64;
    B.tp_slot = m->tp_slot;
    B.K = kconst<double>(P[b]);
    B.ae_re = 0.5 * (P[b].eps_re + 1.0);
    B.ae_im = 0.5 * P[b].eps_im;
    B.am_re = 0.5 * (P[b].mu_re + 1.0);
    B.am_im = 0.5 * P[b].mu_im;
    B.Z = Z[b];
    B.near = near ? (double*)near[b] : nullptr;
    bodies.push_back(B);
    first.push_back(pairs);
    pairs += n;
  }
  if (pairs == 0) return MUELLER_OK;
  void* buf = nullptr;
  TouchBody* d_bodies = nullptr;
  int64_t* d_first = nullptr;
  mueller_status st = upload_bodies(bodies, first, &buf, &d_bodies, &d_first, s);
  if (st) return st;
  auto kern = touching_batch_kernel<Q, MINB>;
  const int use_tables = vertex && ns <= MAX_TAB_NS ? 1 : 0;
  const size_t tab_bytes = use_tables ? (size_t)2 * (ns * ns + ns * ns * ns) * GT * sizeof(double) : 0;
  MU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab_bytes));
  { Prof prof_("touching_batch_kernel<Q>", s); kern<<<(unsigned)pairs, TT, tab_bytes, s>>>(d_bodies, d_first, (int)bodies.size(), ns, dtype, use_tables); }
  MU_CHECK_LAUNCH("touching_batch_kernel");
  cudaFreeAsync(buf, s);
  return MUELLER_OK;
}

// the coincident and common-edge pairs of all bodies, then their
// common-vertex pairs
template <int Q>
mueller_status touching_batch_t(int nb, mueller_mesh* const* meshes, const PhysConsts* P, int ns,
                                int dtype, void* const* Z, const int64_t* ldz,
                                void* const* near, cudaStream_t s) {
  mueller_status st = touching_batch_class<Q, kTouchMinBlocksCE>(nb, meshes, P, ns, dtype, Z, ldz,
                                                                 near, false, s);
  if (st) return st;
  return touching_batch_class<Q, 2>(nb, meshes, P, ns, dtype, Z, ldz, near, true, s);
}

}  // namespace

// regular and touching pairs of nb bodies (same rule Q and order ns), one
// launch each
mueller_status launch_assemble_batch(int nb, mueller_mesh* const* meshes, const PhysConsts* P,
                                     int Q, int ns, int dtype, void* const* Z,
                                     const int64_t* ldz, void* const* near, cudaStream_t s) {
  // tile shape first (a tuning run re-zeroes the largest body's Z), then the
  // touching pairs on the side stream concurrently with the regular pairs
  int big = 0;
  for (int b = 1; b < nb; ++b)
    if (meshes[b]->nt > meshes[big]->nt) big = b;
  mueller_status st = tune_regular(meshes[big], P[big], Q, dtype, Z[big], ldz[big], s);
  if (st) return st;
  cudaStream_t s2;
  st = side_stream(&s2);
  if (!st) st = stream_order(s, s2);
  if (st) return st;
  st = Q == 6 ? touching_batch_t<6>(nb, meshes, P, ns, dtype, Z, ldz, near, s2)
              : touching_batch_t<12>(nb, meshes, P, ns, dtype, Z, ldz, near, s2);
  mueller_status st2;
  if (dtype == MUELLER_C128)
    st2 = Q == 6 ? regular_batch_t<double, 6>(nb, meshes, P, Z, ldz, s)
                 : regular_batch_t<double, 12>(nb, meshes, P, Z, ldz, s);
  else
    st2 = Q == 6 ? regular_batch_t<float, 6>(nb, meshes, P, Z, ldz, s)
                 : regular_batch_t<float, 12>(nb, meshes, P, Z, ldz, s);
  const mueller_status sj = stream_order(s2, s);
  return st ? st : (st2 ? st2 : sj);
}

mueller_status launch_mass_rhs(mueller_mesh* m, const PhysConsts& P, int Q, int dtype, void* Z,
                               int64_t ldz, void* near, void* B, const double* inc_dev, int r,
                               cudaStream_t s) {
  (void)dtype;
  (void)Z;
  (void)ldz;
  (void)near;
  if (!B || r == 0) return MUELLER_OK;
  const int64_t n = (int64_t)r * m->nt * 6;
  { Prof prof_("rhs_kernel", s); rhs_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(m->nt, Q, m->qd64, m->T, inc_dev, r,
                                                         P.ka, 4 * m->nn, (double*)B); }
  MU_CHECK_LAUNCH("rhs_kernel");
  return MUELLER_OK;
}

namespace {

template <int Q, int WHICH>
mueller_status dz_matvec_t(mueller_mesh* m, const PhysConsts& P, int ns, const double2* x,
                           double2* y, cudaStream_t s) {
  constexpr int W = 4, TYT = 32;
  using C = RegCfg<double, Q, W, TYT>;
  const KConst<double> K = kconst<double>(P);
  const int64_t H = 2 * m->nn;
  auto kr = regular_deriv_kernel<Q, W, TYT, WHICH>;
  MU_CUDA(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem));
  dim3 grid((unsigned)((m->nt + W - 1) / W), (unsigned)((m->nt + TYT - 1) / TYT));
  { Prof prof_("regular_deriv_kernel", s); kr<<<grid, 32 * W, C::smem, s>>>(m->nt, m->qd64, m->T, K, x, y, H); }
  MU_CHECK_LAUNCH("regular_deriv_kernel");
  if (m->n_touch > 0) {
    auto kt = touching_deriv_kernel<Q, WHICH>;
    const int use_tables = ns <= MAX_TAB_NS ? 1 : 0;
    const size_t tab_bytes = use_tables ? (size_t)2 * (ns * ns + ns * ns * ns) * GT * sizeof(double) : 0;
    MU_CUDA(cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab_bytes));
    { Prof prof_("touching_deriv_kernel", s); kt<<<(unsigned)m->n_touch, TT, tab_bytes, s>>>(m->n_touch, m->tp, m->X, m->T, m->frame, m->qd64,
                                                                   ns, K, H, use_tables, x, y); }
    MU_CHECK_LAUNCH("touching_deriv_kernel");
  }
  return MUELLER_OK;
}

}  // namespace

// y = (dZ/dtheta) x, theta = eps_r (which 1) or mu_r (which 2), complex128
mueller_status launch_dz_matvec(mueller_mesh* m, const PhysConsts& P, int Q, int ns, int which,
                                const void* x, void* y, cudaStream_t s) {
  MU_CUDA(cudaMemsetAsync(y, 0, (size_t)4 * m->nn * sizeof(double2), s));
  const double2* xd = (const double2*)x;
  double2* yd = (double2*)y;
  if (Q == 6)
    return which == 1 ? dz_matvec_t<6, 1>(m, P, ns, xd, yd, s) : dz_matvec_t<6, 2>(m, P, ns, xd, yd, s);
  return which == 1 ? dz_matvec_t<12, 1>(m, P, ns, xd, yd, s) : dz_matvec_t<12, 2>(m, P, ns, xd, yd, s);
}

mueller_status launch_mirror_k1(int64_t N, int dtype, void* Z, int64_t ldz, cudaStream_t s) {
  const int64_t H = N / 2;
  const unsigned grid = (unsigned)((H * H + 255) / 256);
  if (dtype == MUELLER_C128)
    { Prof prof_("mirror_kernel<double>", s); mirror_kernel<double><<<grid, 256, 0, s>>>(H, (double*)Z, ldz); }
  else
    { Prof prof_("mirror_kernel<float>", s); mirror_kernel<float><<<grid, 256, 0, s>>>(H, (float*)Z, ldz); }
  MU_CHECK_LAUNCH("mirror_kernel");
  return MUELLER_OK;
}

}  // namespace mu
