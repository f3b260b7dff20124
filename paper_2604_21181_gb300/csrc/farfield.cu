// Far field and cross sections of the solved surface currents.
//
// The currents j = sum c_j N t^ and j_m = sum c_jm N t^ (Sec. 4.1 basis)
// radiate the scattered field; with exp(-i omega t) and eta_a = 1
//   F(r) = (i k_a / 4 pi) [ (N~ - r (r.N~)) - r x L~ ],
//   N~ = int j e^{-i k_a r.y} dGamma,  L~ = int j_m e^{-i k_a r.y} dGamma,
//   C_ext = (4 pi / k_a) Im(p . F(k)),  C_sca = int |F|^2 dOmega,
//   C_abs = Re int j_m . (conj(j) x n) dGamma
// (j = n x H and j_m = -n x E, Sec. 2.1, give the Poynting flux).
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace mu {
namespace {

// exp(i th) by a table-driven reduction (P. T. P. Tang, ACM TOMS 15 (1989)):
// th = n pi/128 + d with n the nearest integer to th 128/pi and |d| <= pi/256;
// exp(i th) = T[n mod 256] exp(i d), T[j] = exp(i pi j/128), and exp(i d) from
// the Taylor series of cos to degree 6 and of sin to degree 7 (truncation
// below 2e-20 at |d| = pi/256).  The reduction is Cody-Waite with
// pi/128 = kC1 + kC2 (kC1: 32 significant bits, so n kC1 is exact for
// |n| < 2^21; kC1 + kC2 equals pi/128 to 6e-29).  Beyond |n| = 2^20 the call
// falls back to sincos.  Per call 16 FP64 operations against about three
// times as many for sincos.
constexpr int kCisN = 256;
constexpr double kCisInv = 0x1.45f306dc9c883p+5;   // 128 / pi
constexpr double kC1 = 0x1.921fb544p-6;             // pi/128, leading 32 bits
constexpr double kC2 = 0x1.0b4611a626331p-40;       // pi/128 - kC1
constexpr double kCisMax = 1048576.0 * 0x1.921fb544p-6;  // 2^20 pi/128
constexpr double kRound = 6755399441055744.0;       // 1.5 * 2^52

__device__ __forceinline__ void cis_fill(double2* tab) {
  for (int j = threadIdx.x; j < kCisN; j += blockDim.x) {
    double sn, cs;
    sincospi(j * (1.0 / 128.0), &sn, &cs);
    tab[j] = make_double2(cs, sn);
  }
}

__device__ __forceinline__ double2 cis_tab(double th, const double2* __restrict__ tab) {
  if (fabs(th) > kCisMax) {
    double sn, cs;
    sincos(th, &sn, &cs);
    return make_double2(cs, sn);
  }
  const double t = fma(th, kCisInv, kRound);  // n in the low mantissa bits
  const int n = __double2loint(t);
  const double nf = t - kRound;
  double d = fma(-nf, kC1, th);
  d = fma(-nf, kC2, d);
  const double z = d * d;
  const double c = fma(z, fma(z, fma(z, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
  const double p = fma(z, fma(z, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0);
  const double sn = fma(d * z, p, d);
  const double2 T = tab[n & (kCisN - 1)];
  return make_double2(fma(T.x, c, -T.y * sn), fma(T.y, c, T.x * sn));
}

// weighted currents at the regular-rule points: rec[s][pt] =
// (W j (3 complex), W j_m (3 complex)); one thread per (s, point)
__global__ void currents_kernel(int64_t nt, int Q, const double* __restrict__ qd,
                                const int32_t* __restrict__ T, const double2* __restrict__ X,
                                int r, int64_t N, const double* __restrict__ phi,
                                double2* __restrict__ rec, double* __restrict__ cabs_part) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t np = nt * Q;
  double ca = 0.0;
  const int s = blockIdx.y;
  if (t < np && s < r) {
    const int64_t e = t / Q;
    const int p = (int)(t % Q);
    const double* q = qd + t * QD_STRIDE;
    const double2* x = X + (int64_t)s * N;
    const int64_t H = N / 2;
    double jr[3] = {0, 0, 0}, ji[3] = {0, 0, 0}, mr[3] = {0, 0, 0}, mi[3] = {0, 0, 0};
    for (int k = 0; k < 6; ++k) {
      const int64_t node = T[6 * e + k];
      const double Nk = phi[p * 6 + k];
      for (int b = 0; b < 2; ++b) {
        const double* tb = q + 6 + 3 * b;
        const double2 cj = x[2 * node + b], cm = x[H + 2 * node + b];
        for (int a = 0; a < 3; ++a) {
          jr[a] += Nk * cj.x * tb[a];
          ji[a] += Nk * cj.y * tb[a];
          mr[a] += Nk * cm.x * tb[a];
          mi[a] += Nk * cm.y * tb[a];
        }
      }
    }
    const double W = q[18];
    double2* o = rec + ((int64_t)s * np + t) * 6;
    for (int a = 0; a < 3; ++a) {
      o[a] = make_double2(W * jr[a], W * ji[a]);
      o[3 + a] = make_double2(W * mr[a], W * mi[a]);
    }
    // Re j_m . (conj(j) x n)
    const double n[3] = {q[3], q[4], q[5]};
    const double cxr[3] = {jr[1] * n[2] - jr[2] * n[1], jr[2] * n[0] - jr[0] * n[2], jr[0] * n[1] - jr[1] * n[0]};
    const double cxi[3] = {-(ji[1] * n[2] - ji[2] * n[1]), -(ji[2] * n[0] - ji[0] * n[2]),
                           -(ji[0] * n[1] - ji[1] * n[0])};
    for (int a = 0; a < 3; ++a) ca += mr[a] * cxr[a] - mi[a] * cxi[a];
    ca *= W;
  }
  __shared__ double red[256];
  red[threadIdx.x] = ca;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) cabs_part[(int64_t)s * gridDim.x + blockIdx.x] = red[0];
}

// Block reduction of the 12 partial sums (N~ and L~, complex) and
// F = (i k / 4 pi)[(N~ - r (r.N~)) - r x L~] into F_out[0..2] (thread 0).
// Block sums of the 12 partials (256 threads); the sums end in red[c][0].
__device__ __forceinline__ void block_sum12(double (*red)[256], const double* acc) {
  for (int c = 0; c < 12; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int c = 0; c < 12; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
}

// F(r) from the twelve sums (N~ re/im, L~ re/im per component) of one
// direction
__device__ __forceinline__ void far_store(const double* sum, double rx, double ry, double rz,
                                          double ka, double2* __restrict__ F_out) {
  double Nr[3], Ni[3], Lr[3], Li[3];
  for (int a = 0; a < 3; ++a) {
    Nr[a] = sum[2 * a];
    Ni[a] = sum[2 * a + 1];
    Lr[a] = sum[6 + 2 * a];
    Li[a] = sum[7 + 2 * a];
  }
  const double r[3] = {rx, ry, rz};
  const double rNr = r[0] * Nr[0] + r[1] * Nr[1] + r[2] * Nr[2];
  const double rNi = r[0] * Ni[0] + r[1] * Ni[1] + r[2] * Ni[2];
  const double cLr[3] = {r[1] * Lr[2] - r[2] * Lr[1], r[2] * Lr[0] - r[0] * Lr[2], r[0] * Lr[1] - r[1] * Lr[0]};
  const double cLi[3] = {r[1] * Li[2] - r[2] * Li[1], r[2] * Li[0] - r[0] * Li[2], r[0] * Li[1] - r[1] * Li[0]};
  const double pre = ka / (4.0 * 3.14159265358979323846);  // i k / 4 pi -> multiply by i
  for (int a = 0; a < 3; ++a) {
    const double vr = Nr[a] - r[a] * rNr - cLr[a];
    const double vi = Ni[a] - r[a] * rNi - cLi[a];
    F_out[a] = make_double2(-pre * vi, pre * vr);
  }
}

__device__ __forceinline__ void far_finish(double (*red)[256], const double* acc, double rx,
                                           double ry, double rz, double ka,
                                           double2* __restrict__ F_out) {
  block_sum12(red, acc);
  if (threadIdx.x == 0) {
    double sum[12];
    for (int c = 0; c < 12; ++c) sum[c] = red[c][0];
    far_store(sum, rx, ry, rz, ka, F_out);
  }
}

// F at directions 0 .. nd_eval-1 of one right-hand side: DT directions per
// CTA, threads over points; each current record is loaded once for the DT
// directions.
constexpr int kFarDT = 4;
template <int DT>
__global__ void __launch_bounds__(256) far_kernel(int64_t np, const double* __restrict__ qd,
                                                  const double2* __restrict__ rec,
                                                  const double* __restrict__ dirs, int64_t nd_eval,
                                                  double ka, double2* __restrict__ F) {
  __shared__ double2 tab[kCisN];
  __shared__ double red[12][256];
  cis_fill(tab);
  __syncthreads();
  const int64_t d0 = (int64_t)blockIdx.x * DT;
  double rk[DT][3];
#pragma unroll
  for (int k = 0; k < DT; ++k) {
    const int64_t d = d0 + k < nd_eval ? d0 + k : nd_eval - 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) rk[k][a] = -ka * dirs[3 * d + a];
  }
  double acc[DT][12];
#pragma unroll
  for (int k = 0; k < DT; ++k)
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[k][c] = 0.0;
  for (int64_t t = threadIdx.x; t < np; t += blockDim.x) {
    const double* q = qd + t * QD_STRIDE;
    const double y0 = q[0], y1 = q[1], y2 = q[2];
    const double2* o = rec + t * 6;
    double2 v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = o[c];
#pragma unroll
    for (int k = 0; k < DT; ++k) {
      const double2 e = cis_tab(fma(rk[k][0], y0, fma(rk[k][1], y1, rk[k][2] * y2)), tab);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        acc[k][2 * c] = fma(v[c].x, e.x, fma(-v[c].y, e.y, acc[k][2 * c]));
        acc[k][2 * c + 1] = fma(v[c].x, e.y, fma(v[c].y, e.x, acc[k][2 * c + 1]));
      }
    }
  }
#pragma unroll
  for (int k = 0; k < DT; ++k) {
    const int64_t d = d0 + k;
    if (d < nd_eval) far_finish(red, acc[k], dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2], ka, F + d * 3);
    __syncthreads();
  }
}

inline unsigned far_grid(int64_t nd_eval) { return (unsigned)((nd_eval + kFarDT - 1) / kFarDT); }

// The forward direction (k-hat of each RHS, read from its incident wave inc
// [r][6]; index 0 of its far-field list) of every RHS: one direction has too
// little work for one CTA, so CTA (g, s) sums the partials of point chunk g
// of RHS s and far_fwd_finish_kernel adds the chunks up and forms F.
constexpr int kFwdChunks = 64;
__global__ void __launch_bounds__(256) far_fwd_part_kernel(int64_t np, const double* __restrict__ qd,
                                                           const double2* __restrict__ rec,
                                                           const double* __restrict__ inc,
                                                           double ka, double* __restrict__ part) {
  __shared__ double2 tab[kCisN];
  __shared__ double red[12][256];
  cis_fill(tab);
  __syncthreads();
  const int s = blockIdx.y, g = blockIdx.x, G = gridDim.x;
  const double* dd = inc + (int64_t)s * 6;
  const double rk0 = -ka * dd[0], rk1 = -ka * dd[1], rk2 = -ka * dd[2];
  const int64_t chunk = (np + G - 1) / G, t0 = (int64_t)g * chunk;
  const int64_t t1 = t0 + chunk < np ? t0 + chunk : np;
  double acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = 0.0;
  for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const double* q = qd + t * QD_STRIDE;
    const double2 e = cis_tab(fma(rk0, q[0], fma(rk1, q[1], rk2 * q[2])), tab);
    const double2* o = rec + ((int64_t)s * np + t) * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double2 v = o[c];
      acc[2 * c] = fma(v.x, e.x, fma(-v.y, e.y, acc[2 * c]));
      acc[2 * c + 1] = fma(v.x, e.y, fma(v.y, e.x, acc[2 * c + 1]));
    }
  }
  block_sum12(red, acc);
  if (threadIdx.x < 12) part[((int64_t)s * G + g) * 12 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) far_fwd_finish_kernel(const double* __restrict__ part, int G,
                                                             const double* __restrict__ inc,
                                                             int64_t nd, double ka,
                                                             double2* __restrict__ F) {
  __shared__ double red[12][256];
  const int s = blockIdx.x;
  double acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c)
    acc[c] = (int)threadIdx.x < G ? part[((int64_t)s * G + threadIdx.x) * 12 + c] : 0.0;
  const double* dd = inc + (int64_t)s * 6;
  far_finish(red, acc, dd[0], dd[1], dd[2], ka, F + (int64_t)s * nd * 3);
}

// Antipodal pair p of the sphere rule (n_phi even): direction k2 = -k1, the
// ring n_theta-1-it against ring it, or for odd n_theta the middle ring
// against itself turned by pi.
__host__ __device__ __forceinline__ void sphere_pair(int64_t p, int n_theta, int n_phi,
                                                     int64_t& k1, int64_t& k2) {
  const int64_t full = (int64_t)(n_theta / 2) * n_phi;
  if (p < full) {
    const int64_t it = p / n_phi, ip = p % n_phi;
    k1 = it * n_phi + ip;
    k2 = (n_theta - 1 - it) * n_phi + (ip + n_phi / 2) % n_phi;
  } else {
    const int64_t mid = n_theta / 2, ip = p - full;
    k1 = mid * n_phi + ip;
    k2 = mid * n_phi + ip + n_phi / 2;
  }
}

// F at the sphere-rule directions, which come in antipodal pairs
// (d_k2 = -d_k1 exactly): exp(-i k d_k2.y) = conj(exp(-i k d_k1.y)), so one
// phase serves both directions of a pair, and so do the four real products
// of a current component v with it:
//   F(d_k1) += (v.x e.x - v.y e.y, v.x e.y + v.y e.x),
//   F(d_k2) += (v.x e.x + v.y e.y, v.y e.x - v.x e.y),
// summed as the four sums of v.x e.x, v.y e.y, v.x e.y, v.y e.x (4 FMAs per
// component for both directions).  A warp takes DP pairs and RS right-hand
// sides (blockIdx.y: right-hand sides RS*y ..), its lanes stride over the
// points and its sums meet by shuffles, so no CTA-wide reduction stalls the
// CTA's other pairs.  dirs and F point at the sphere block (index k) of
// right-hand side 0; F of right-hand side s is F + s * f_stride, its
// currents rec + s * np * 6.
constexpr int kFarMRS = 4;  // several right-hand sides: per warp (one pair each)
constexpr int kFarWarps = 8;
template <int DP, int RS>
__global__ void __launch_bounds__(32 * kFarWarps, RS > 2 ? 1 : 2) far_pair_kernel(
    int64_t np, const double* __restrict__ qd, const double2* __restrict__ rec, int r,
    const double* __restrict__ dirs, int n_theta, int n_phi, double ka, double2* __restrict__ F,
    int64_t f_stride) {
  __shared__ double2 tab[kCisN];
  cis_fill(tab);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t npairs = (int64_t)n_theta * n_phi / 2;
  const int64_t p0 = ((int64_t)blockIdx.x * kFarWarps + warp) * DP;
  if (p0 >= npairs) return;  // whole warps; no CTA barrier follows
  const int s0 = blockIdx.y * RS;
  double rk[DP][3];
#pragma unroll
  for (int q = 0; q < DP; ++q) {
    int64_t k1, k2;
    sphere_pair(p0 + q < npairs ? p0 + q : npairs - 1, n_theta, n_phi, k1, k2);
#pragma unroll
    for (int a = 0; a < 3; ++a) rk[q][a] = -ka * dirs[3 * k1 + a];
  }
  double acc[DP][RS][4][6];  // sums of v.x e.x, v.y e.y, v.x e.y, v.y e.x
#pragma unroll
  for (int q = 0; q < DP; ++q)
#pragma unroll
    for (int k = 0; k < RS; ++k)
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[q][k][h][c] = 0.0;
  for (int64_t t = lane; t < np; t += 32) {
    const double* qp = qd + t * QD_STRIDE;
    const double y0 = qp[0], y1 = qp[1], y2 = qp[2];
    double2 e[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) e[q] = cis_tab(fma(rk[q][0], y0, fma(rk[q][1], y1, rk[q][2] * y2)), tab);
#pragma unroll
    for (int k = 0; k < RS; ++k) {
      if (s0 + k < r) {
        const double2* o = rec + ((int64_t)(s0 + k) * np + t) * 6;
        double2 v[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = o[c];
#pragma unroll
        for (int q = 0; q < DP; ++q)
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            acc[q][k][0][c] = fma(v[c].x, e[q].x, acc[q][k][0][c]);
            acc[q][k][1][c] = fma(v[c].y, e[q].y, acc[q][k][1][c]);
            acc[q][k][2][c] = fma(v[c].x, e[q].y, acc[q][k][2][c]);
            acc[q][k][3][c] = fma(v[c].y, e[q].x, acc[q][k][3][c]);
          }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < DP; ++q)
#pragma unroll
    for (int k = 0; k < RS; ++k)
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          double v = acc[q][k][h][c];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          acc[q][k][h][c] = v;
        }
  if (lane != 0) return;
#pragma unroll
  for (int q = 0; q < DP; ++q) {
    if (p0 + q >= npairs) continue;
    int64_t kk[2];
    sphere_pair(p0 + q, n_theta, n_phi, kk[0], kk[1]);
#pragma unroll
    for (int k = 0; k < RS; ++k) {
      if (s0 + k >= r) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        double a[12];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const double xx = acc[q][k][0][c], yy = acc[q][k][1][c];
          const double xy = acc[q][k][2][c], yx = acc[q][k][3][c];
          a[2 * c] = h ? xx + yy : xx - yy;
          a[2 * c + 1] = h ? yx - xy : xy + yx;
        }
        const double* dd = dirs + 3 * kk[h];
        far_store(a, dd[0], dd[1], dd[2], ka, F + (s0 + k) * f_stride + kk[h] * 3);
      }
    }
  }
}

// Directions shared by all right-hand sides (indices d0, d0 + 1, .. of the
// list: the user directions, or with an odd n_phi the whole sphere rule too)
// for RS right-hand sides per CTA: each phase exp(-i k r.y) is computed once
// and applied to the RS current records.  Per right-hand side the sums run in
// the same order as in far_kernel.
template <int RS>
__global__ void __launch_bounds__(256) far_multi_kernel(int64_t np, const double* __restrict__ qd,
                                                        const double2* __restrict__ rec, int r,
                                                        const double* __restrict__ dirs,
                                                        int64_t nd, int64_t d0, double ka,
                                                        double2* __restrict__ F) {
  const int64_t d = d0 + blockIdx.x;
  const int s0 = blockIdx.y * RS;
  const double rx = dirs[3 * d], ry = dirs[3 * d + 1], rz = dirs[3 * d + 2];
  __shared__ double2 tab[kCisN];
  __shared__ double red[12][256];
  cis_fill(tab);
  __syncthreads();
  const double kx = -ka * rx, ky = -ka * ry, kz = -ka * rz;
  double acc[RS][12];
#pragma unroll
  for (int k = 0; k < RS; ++k)
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[k][c] = 0.0;
  for (int64_t t = threadIdx.x; t < np; t += blockDim.x) {
    const double* q = qd + t * QD_STRIDE;
    const double2 e = cis_tab(fma(kx, q[0], fma(ky, q[1], kz * q[2])), tab);
#pragma unroll
    for (int k = 0; k < RS; ++k) {
      if (s0 + k < r) {
        const double2* o = rec + ((int64_t)(s0 + k) * np + t) * 6;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const double2 v = o[c];
          acc[k][2 * c] = fma(v.x, e.x, fma(-v.y, e.y, acc[k][2 * c]));
          acc[k][2 * c + 1] = fma(v.x, e.y, fma(v.y, e.x, acc[k][2 * c + 1]));
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < RS; ++k) {
    if (s0 + k < r) far_finish(red, acc[k], rx, ry, rz, ka, F + ((int64_t)(s0 + k) * nd + d) * 3);
    __syncthreads();
  }
}

// cross sections per RHS from the far fields: C_ext from the forward
// direction (index 0), C_sca from the sphere rule (indices 1..), C_abs from
// the block partials
__global__ void xs_kernel(const double2* __restrict__ F, int64_t nd, int nth, int nph,
                          const double* __restrict__ wth, const double* __restrict__ inc,
                          double ka, const double* __restrict__ cabs_part, int nparts,
                          double* __restrict__ xs) {
  const int s = blockIdx.x;
  __shared__ double red[256];
  double acc = 0.0;
  const int64_t nsph = (int64_t)nth * nph;
  for (int64_t k = threadIdx.x; k < nsph; k += blockDim.x) {
    const int it = (int)(k / nph);
    const double2* f = F + ((int64_t)s * nd + 1 + k) * 3;
    const double a = f[0].x * f[0].x + f[0].y * f[0].y + f[1].x * f[1].x + f[1].y * f[1].y +
                     f[2].x * f[2].x + f[2].y * f[2].y;
    acc += a * 2.0 * wth[it] * (2.0 * 3.14159265358979323846 / nph);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double csca = red[0];
  __syncthreads();
  double ca = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) ca += cabs_part[(int64_t)s * nparts + k];
  red[threadIdx.x] = ca;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double2* f = F + ((int64_t)s * nd) * 3;
    const double* p = inc + 6 * s + 3;
    const double im = p[0] * f[0].y + p[1] * f[1].y + p[2] * f[2].y;
    xs[3 * s] = 4.0 * 3.14159265358979323846 / ka * im;
    xs[3 * s + 1] = csca;
    xs[3 * s + 2] = red[0];
  }
}

__global__ void copy_user_dirs_kernel(const double2* __restrict__ Fall, int64_t nd_all, int64_t off,
                                      int64_t ndir, int r, double2* __restrict__ Fout) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)r * ndir * 3) return;
  const int64_t a = t % 3, d = (t / 3) % ndir, s = t / (3 * ndir);
  Fout[t] = Fall[((s * nd_all) + off + d) * 3 + a];
}

// Direction list of every RHS: forward k (index 0), the sphere rule
// (1 + it n_phi + ip: cos(theta) on Gauss-Legendre nodes, phi on n_phi
// equal steps), the user directions.  With n_phi even the sphere rule is
// written in exact antipodal pairs (sphere_pair), the second direction of
// each pair the negated first (Gauss-Legendre nodes are symmetric, up to
// the rounding of their computation).
std::vector<double> far_dirs(const double* inc, int n_theta, int n_phi,
                             const std::vector<double>& gth, const double* dirs, int64_t ndir) {
  const int64_t nsph = (int64_t)n_theta * n_phi, nd = 1 + nsph + ndir;
  std::vector<double> hd((size_t)nd * 3);
  double* o = hd.data();
  o[0] = inc[0];
  o[1] = inc[1];
  o[2] = inc[2];
  for (int it = 0; it < n_theta; ++it) {
    const double ct = 2.0 * gth[it] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
    for (int ip = 0; ip < n_phi; ++ip) {
      const double ph = 2.0 * 3.14159265358979323846 * ip / n_phi;
      double* dd = o + 3 * (1 + (int64_t)it * n_phi + ip);
      dd[0] = st * cos(ph);
      dd[1] = st * sin(ph);
      dd[2] = ct;
    }
  }
  if (n_phi % 2 == 0)
    for (int64_t p = 0; p < nsph / 2; ++p) {
      int64_t k1, k2;
      sphere_pair(p, n_theta, n_phi, k1, k2);
      for (int a = 0; a < 3; ++a) o[3 * (1 + k2) + a] = -o[3 * (1 + k1) + a];
    }
  for (int64_t d = 0; d < ndir; ++d)
    for (int a = 0; a < 3; ++a) o[3 * (1 + nsph + d) + a] = dirs[3 * d + a];
  return hd;
}

// F of one RHS at its sphere-rule and user directions (the forward direction
// is far_fwd's): the sphere rule by antipodal pairs (far_pair_kernel) when
// n_phi is even, else with the user directions by far_kernel.
mueller_status far_one_rhs(int64_t np, const double* qd, const double2* rec, const double* dirs,
                           int64_t nd, int n_theta, int n_phi, int64_t ndir, double ka,
                           double2* F, cudaStream_t s) {
  const int64_t nsph = (int64_t)n_theta * n_phi;
  if (n_phi % 2 != 0) {
    { Prof prof_("far_kernel", s); far_kernel<kFarDT><<<far_grid(nd - 1), 256, 0, s>>>(np, qd, rec, dirs + 3, nd - 1, ka, F + 3); }
    MU_CHECK_LAUNCH("far_kernel");
    return MUELLER_OK;
  }
  const int64_t npairs = nsph / 2;
  { Prof prof_("far_pair_kernel", s); far_pair_kernel<1, 1><<<(unsigned)((npairs + kFarWarps - 1) / kFarWarps), 32 * kFarWarps, 0, s>>>(
      np, qd, rec, 1, dirs + 3, n_theta, n_phi, ka, F + 3, 0); }
  if (ndir > 0)
    { Prof prof_("far_kernel", s); far_kernel<kFarDT><<<far_grid(ndir), 256, 0, s>>>(np, qd, rec, dirs + 3 * (1 + nsph), ndir, ka,
                                                                                     F + 3 * (1 + nsph)); }
  MU_CHECK_LAUNCH("far_kernel");
  return MUELLER_OK;
}

// F of all r right-hand sides at the directions they share (sphere rule and
// user list, indices 1 .. nd-1 of each list; rec, dirs and F hold r blocks).
// One right-hand side: far_one_rhs.  Several: the sphere rule by antipodal
// pairs (even n_phi), kFarMRS right-hand sides per CTA, and the remaining
// directions 4 right-hand sides per CTA.
mueller_status far_shared(int64_t np, const double* qd, const double2* rec, int r,
                          const double* dirs, int64_t nd, int n_theta, int n_phi, int64_t ndir,
                          double ka, double2* F, cudaStream_t s) {
  if (r == 1) return far_one_rhs(np, qd, rec, dirs, nd, n_theta, n_phi, ndir, ka, F, s);
  const int64_t nsph = (int64_t)n_theta * n_phi;
  int64_t d0 = 1;
  if (n_phi % 2 == 0) {
    Prof prof_("far_pair_kernel", s);
    far_pair_kernel<1, kFarMRS><<<dim3((unsigned)((nsph / 2 + kFarWarps - 1) / kFarWarps), (unsigned)((r + kFarMRS - 1) / kFarMRS)), 32 * kFarWarps, 0, s>>>(
        np, qd, rec, r, dirs + 3, n_theta, n_phi, ka, F + 3, nd * 3);
    d0 = 1 + nsph;
  }
  if (nd > d0) {
    Prof prof_("far_multi_kernel", s);
    far_multi_kernel<4><<<dim3((unsigned)(nd - d0), (unsigned)((r + 3) / 4)), 256, 0, s>>>(
        np, qd, rec, r, dirs, nd, d0, ka, F);
  }
  MU_CHECK_LAUNCH("far_shared");
  return MUELLER_OK;
}

// the forward direction of all r right-hand sides (part: r x kFwdChunks x 12)
mueller_status far_fwd(int64_t np, const double* qd, const double2* rec, const double* inc,
                       int64_t nd, int r, double ka, double* part, double2* F, cudaStream_t s) {
  { Prof prof_("far_fwd_part_kernel", s); far_fwd_part_kernel<<<dim3(kFwdChunks, (unsigned)r), 256, 0, s>>>(np, qd, rec, inc, ka, part); }
  { Prof prof_("far_fwd_finish_kernel", s); far_fwd_finish_kernel<<<(unsigned)r, 256, 0, s>>>(part, kFwdChunks, inc, nd, ka, F); }
  MU_CHECK_LAUNCH("far_fwd");
  return MUELLER_OK;
}

}  // namespace

mueller_status far_field(mueller_mesh* m, const PhysConsts& P, int Q, const void* X, int r,
                         const double* inc, const double* dirs, int64_t ndir, void* F, double* xs,
                         int n_theta, int n_phi, cudaStream_t s) {
  TriangleRule rule;
  if (!triangle_rule(Q, rule)) return MUELLER_ERR_INVALID_ARG;
  const int64_t np = m->nt * Q, N = 4 * m->nn;
  // direction list per RHS: forward k, sphere rule (theta-major), user dirs
  std::vector<double> gth, wth;
  gauss_legendre_unit(n_theta, gth, wth);
  const int64_t nsph = (int64_t)n_theta * n_phi;
  const int64_t nd = 1 + nsph + ndir;
  const std::vector<double> hd = far_dirs(inc, n_theta, n_phi, gth, dirs, ndir);
  double phi[MAX_Q * 6];
  for (int p = 0; p < Q; ++p) {
    const double l0 = 1.0 - rule.xi[p] - rule.eta[p], l1 = rule.xi[p], l2 = rule.eta[p];
    const double Nv[6] = {l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                          4 * l0 * l1,       4 * l1 * l2,       4 * l2 * l0};
    for (int k = 0; k < 6; ++k) phi[p * 6 + k] = Nv[k];
  }
  const unsigned nblk_pts = (unsigned)((np + 255) / 256);
  // scratch
  size_t off = 0;
  auto al = [&](size_t b) {
    size_t o = off;
    off += (b + 255) & ~size_t(255);
    return o;
  };
  const size_t o_rec = al((size_t)r * np * 6 * 16);
  const size_t o_dirs = al(hd.size() * 8);
  const size_t o_F = al((size_t)r * nd * 3 * 16);
  const size_t o_wth = al(wth.size() * 8);
  const size_t o_inc = al((size_t)r * 6 * 8);
  const size_t o_phi = al(sizeof(phi));
  const size_t o_cab = al((size_t)r * nblk_pts * 8);
  const size_t o_xs = al((size_t)r * 3 * 8);
  const size_t o_part = al((size_t)r * kFwdChunks * 12 * 8);
  char* buf = nullptr;
  MU_CUDA(cudaMallocAsync((void**)&buf, off, s));
  double2* rec = (double2*)(buf + o_rec);
  double* ddirs = (double*)(buf + o_dirs);
  double2* Fall = (double2*)(buf + o_F);
  double* dwth = (double*)(buf + o_wth);
  double* dinc = (double*)(buf + o_inc);
  double* dphi = (double*)(buf + o_phi);
  double* cab = (double*)(buf + o_cab);
  double* dxs = (double*)(buf + o_xs);
  mueller_status st = MUELLER_OK;
  cudaError_t e = cudaMemcpyAsync(ddirs, hd.data(), hd.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dwth, wth.data(), wth.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dinc, inc, (size_t)r * 6 * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dphi, phi, sizeof(phi), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) st = cuda_fail(e, "far-field setup");
  if (!st) {
    { Prof prof_("currents_kernel", s); currents_kernel<<<dim3(nblk_pts, r), 256, 0, s>>>(m->nt, Q, m->qd64, m->T, (const double2*)X, r,
                                                       N, dphi, rec, cab); }
    st = far_fwd(np, m->qd64, rec, dinc, nd, r, P.ka, (double*)(buf + o_part), Fall, s);
    if (!st) st = far_shared(np, m->qd64, rec, r, ddirs, nd, n_theta, n_phi, ndir, P.ka, Fall, s);
    if (!st) {
      { Prof prof_("xs_kernel", s); xs_kernel<<<r, 256, 0, s>>>(Fall, nd, n_theta, n_phi, dwth, dinc, P.ka, cab, (int)nblk_pts, dxs); }
      if (ndir > 0)
        { Prof prof_("copy_user_dirs_kernel", s); copy_user_dirs_kernel<<<(unsigned)(((int64_t)r * ndir * 3 + 255) / 256), 256, 0, s>>>(
            Fall, nd, 1 + nsph, ndir, r, (double2*)F); }
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(xs, dxs, (size_t)r * 3 * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_fail(e, "far field");
    }
  }
  cudaFreeAsync(buf, s);
  return st;
}

}  // namespace mu

// ---------------------------------------------------------------------------
// Allocation-free far field.  Some callers must not allocate device memory
// at this point of their program: a framework that owns all device memory
// through its own pool (a raw allocation outside the pool can fail or
// fragment it), or a service that reserves its memory at start-up and
// forbids allocation afterwards to keep latency and footprint predictable.
// mueller_far_field_noalloc serves them: its scratch is a fixed array in
// device memory that exists for as long as the library is loaded, on every
// GPU that loads it.  The caller still provides the inputs and outputs.
// ---------------------------------------------------------------------------
namespace mu {
namespace {

constexpr size_t kFarFieldScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_far_scratch[kFarFieldScratchBytes];

// Device address of g_far_scratch on each device.  In host code the symbol
// name is only a stand-in, so the address is looked up once per device, with
// that device current, and then handed to the kernels.
constexpr int kMaxDevices = 64;
static std::mutex g_far_scratch_mu;
static void* g_far_scratch_ptr[kMaxDevices] = {};

mueller_status far_scratch_address(void** out) {
  int dev = 0;
  MU_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal beyond the supported range of the allocation-free far field");
    return MUELLER_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_far_scratch_mu);
  if (!g_far_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_far_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(far-field scratch)");
    g_far_scratch_ptr[dev] = p;
  }
  *out = g_far_scratch_ptr[dev];
  return MUELLER_OK;
}

}  // namespace

mueller_status far_field_noalloc(mueller_mesh* m, const PhysConsts& P, int Q, const void* X, int r,
                                 const double* inc, const double* dirs, int64_t ndir, void* F,
                                 double* xs, int n_theta, int n_phi, cudaStream_t s) {
  TriangleRule rule;
  if (!triangle_rule(Q, rule)) return MUELLER_ERR_INVALID_ARG;
  const int64_t np = m->nt * Q, N = 4 * m->nn;
  std::vector<double> gth, wth;
  gauss_legendre_unit(n_theta, gth, wth);
  const int64_t nsph = (int64_t)n_theta * n_phi;
  const int64_t nd = 1 + nsph + ndir;
  const unsigned nblk_pts = (unsigned)((np + 255) / 256);
  size_t off = 0;
  auto al = [&](size_t b) {
    size_t o = off;
    off += (b + 255) & ~size_t(255);
    return o;
  };
  const size_t o_rec = al((size_t)r * np * 6 * 16);
  const size_t o_dirs = al((size_t)nd * 3 * 8);
  const size_t o_F = al((size_t)r * nd * 3 * 16);
  const size_t o_wth = al(wth.size() * 8);
  const size_t o_inc = al((size_t)r * 6 * 8);
  const size_t o_phi = al(sizeof(double) * MAX_Q * 6);
  const size_t o_cab = al((size_t)r * nblk_pts * 8);
  const size_t o_xs = al((size_t)r * 3 * 8);
  const size_t o_part = al((size_t)r * kFwdChunks * 12 * 8);
  if (off > kFarFieldScratchBytes) {
    set_error("far field needs " + std::to_string(off) + " bytes of scratch, more than the " +
              std::to_string(kFarFieldScratchBytes) +
              " bytes of the allocation-free variant: use fewer right-hand sides, directions or "
              "sphere points, or mueller_far_field");
    return MUELLER_ERR_INVALID_ARG;
  }
  char* buf = nullptr;
  mueller_status st = far_scratch_address((void**)&buf);
  if (st) return st;
  const std::vector<double> hd = far_dirs(inc, n_theta, n_phi, gth, dirs, ndir);
  double phi[MAX_Q * 6];
  for (int p = 0; p < Q; ++p) {
    const double l0 = 1.0 - rule.xi[p] - rule.eta[p], l1 = rule.xi[p], l2 = rule.eta[p];
    const double Nv[6] = {l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                          4 * l0 * l1,       4 * l1 * l2,       4 * l2 * l0};
    for (int k = 0; k < 6; ++k) phi[p * 6 + k] = Nv[k];
  }
  double2* rec = (double2*)(buf + o_rec);
  double* ddirs = (double*)(buf + o_dirs);
  double2* Fall = (double2*)(buf + o_F);
  double* dwth = (double*)(buf + o_wth);
  double* dinc = (double*)(buf + o_inc);
  double* dphi = (double*)(buf + o_phi);
  double* cab = (double*)(buf + o_cab);
  double* dxs = (double*)(buf + o_xs);
  // every scratch region is overwritten before it is read (currents, far
  // fields, per-block partials, cross sections): nothing needs clearing
  cudaError_t e = cudaMemcpyAsync(ddirs, hd.data(), hd.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dwth, wth.data(), wth.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dinc, inc, (size_t)r * 6 * 8, cudaMemcpyHostToDevice, s);
  // From the first copy on, work sits on the stream that uses the shared
  // scratch: every return below waits for the stream first (keeping the
  // first error), so that a later call on another stream cannot overlap it.
  auto drain = [&](mueller_status status) {
    cudaStreamSynchronize(s);
    return status;
  };
  if (e == cudaSuccess) e = cudaMemcpyAsync(dphi, phi, sizeof(double) * Q * 6, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return drain(cuda_fail(e, "far-field (allocation-free) setup"));
  { Prof prof_("currents_kernel", s); currents_kernel<<<dim3(nblk_pts, r), 256, 0, s>>>(m->nt, Q, m->qd64, m->T, (const double2*)X, r, N, dphi, rec, cab); }
  st = far_fwd(np, m->qd64, rec, dinc, nd, r, P.ka, (double*)(buf + o_part), Fall, s);
  if (st) return drain(st);
  st = far_shared(np, m->qd64, rec, r, ddirs, nd, n_theta, n_phi, ndir, P.ka, Fall, s);
  if (st) return drain(st);
  { Prof prof_("xs_kernel", s); xs_kernel<<<r, 256, 0, s>>>(Fall, nd, n_theta, n_phi, dwth, dinc, P.ka, cab, (int)nblk_pts, dxs); }
  if (ndir > 0) {
    Prof prof_("copy_user_dirs_kernel", s);
    copy_user_dirs_kernel<<<(unsigned)(((int64_t)r * ndir * 3 + 255) / 256), 256, 0, s>>>(
        Fall, nd, 1 + nsph, ndir, r, (double2*)F);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(xs, dxs, (size_t)r * 3 * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return drain(cuda_fail(e, "far field (allocation-free)"));
  return MUELLER_OK;
}

}  // namespace mu
