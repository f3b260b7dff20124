// Dense complex linear algebra of the solver (Sec. 5):
//   * matrix-vector products with Z (complex128 FP64, complex64 FP32, and
//     complex64 storage with FP64 arithmetic for the refinement residual),
//     plus the near blocks of the mixed operator;
//   * batched blocked LU with partial pivoting (FP64) of the Morton
//     block-Jacobi blocks (Eq. precond_block) and their explicit inverses;
//   * restarted GMRES with right preconditioning (classical Gram-Schmidt
//     applied twice, complex Givens rotations) and the mixed-precision
//     iterative refinement around it.
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>
#include <type_traits>

#include "common.cuh"

namespace mu {
namespace {

__host__ __device__ __forceinline__ int64_t mn64(int64_t a, int64_t b) { return a < b ? a : b; }

// ===================================================================== GEMV
// y = Z x, Z row-major complex128 (N x ldz).  One warp per 4 rows, lanes
// stride over columns; FP64 FMA bound on GB300.
__global__ void __launch_bounds__(256) gemv_c128_kernel(int64_t N, const double2* __restrict__ Z,
                                                        int64_t ldz, const double2* __restrict__ x,
                                                        double2* __restrict__ y, int64_t xs,
                                                        int64_t ys, int r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = ((int64_t)blockIdx.x * 8 + warp) * 4;
  const int s = blockIdx.y;
  if (row0 >= N || s >= r) return;
  const double2* xv = x + s * xs;
  double ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
  const int nr = (int)mn64(4, N - row0);
  for (int64_t c = lane; c < N; c += 32) {
    const double2 xc = __ldg(xv + c);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k < nr) {
        const double2 z = __ldg(Z + (row0 + k) * ldz + c);
        ar[k] = fma(z.x, xc.x, fma(-z.y, xc.y, ar[k]));
        ai[k] = fma(z.x, xc.y, fma(z.y, xc.x, ai[k]));
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], o);
      ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], o);
    }
  }
  if (lane < nr) {
    double vr = ar[0], vi = ai[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
      if (lane == k) {
        vr = ar[k];
        vi = ai[k];
      }
    y[s * ys + row0 + lane] = make_double2(vr, vi);
  }
}

// y = Z^H x (complex128), the adjoint operator (MUELLER_OP_ADJOINT).  A CTA
// owns a block of rows [i0, i1) and a tile of 512 columns: its 256 threads
// stream the block's row segments (8 KB each, contiguous) two columns per
// thread, four rows per step, and add their partial sums into y by atomic
// additions (y zeroed by the caller).
constexpr int kGemvhCols = 512;
__global__ void __launch_bounds__(256) gemvh_c128_kernel(int64_t N, const double2* __restrict__ Z,
                                                         int64_t ldz, const double2* __restrict__ x,
                                                         double2* __restrict__ y, int64_t xs,
                                                         int64_t ys, int64_t rows) {
  constexpr int U = 4;
  const int s = blockIdx.z;
  const int64_t j0 = (int64_t)blockIdx.x * kGemvhCols + threadIdx.x, j1 = j0 + 256;
  const int64_t i0 = (int64_t)blockIdx.y * rows, i1 = i0 + rows < N ? i0 + rows : N;
  const bool v0 = j0 < N, v1 = j1 < N;
  const double2* xv = x + s * xs;
  double ar0 = 0.0, ai0 = 0.0, ar1 = 0.0, ai1 = 0.0;
  const double2 zero = make_double2(0.0, 0.0);
  int64_t i = i0;
  for (; i + U <= i1; i += U) {
    double2 z0[U], z1[U], xi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const double2* row = Z + (i + u) * ldz;
      z0[u] = v0 ? __ldg(row + j0) : zero;
      z1[u] = v1 ? __ldg(row + j1) : zero;
      xi[u] = __ldg(xv + i + u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      // conj(z) x
      ar0 = fma(z0[u].x, xi[u].x, fma(z0[u].y, xi[u].y, ar0));
      ai0 = fma(z0[u].x, xi[u].y, fma(-z0[u].y, xi[u].x, ai0));
      ar1 = fma(z1[u].x, xi[u].x, fma(z1[u].y, xi[u].y, ar1));
      ai1 = fma(z1[u].x, xi[u].y, fma(-z1[u].y, xi[u].x, ai1));
    }
  }
  for (; i < i1; ++i) {
    const double2* row = Z + i * ldz;
    const double2 xi = __ldg(xv + i);
    const double2 z0 = v0 ? __ldg(row + j0) : zero, z1 = v1 ? __ldg(row + j1) : zero;
    ar0 = fma(z0.x, xi.x, fma(z0.y, xi.y, ar0));
    ai0 = fma(z0.x, xi.y, fma(-z0.y, xi.x, ai0));
    ar1 = fma(z1.x, xi.x, fma(z1.y, xi.y, ar1));
    ai1 = fma(z1.x, xi.y, fma(-z1.y, xi.x, ai1));
  }
  if (v0) {
    atomicAdd(&y[s * ys + j0].x, ar0);
    atomicAdd(&y[s * ys + j0].y, ai0);
  }
  if (v1) {
    atomicAdd(&y[s * ys + j1].x, ar1);
    atomicAdd(&y[s * ys + j1].y, ai1);
  }
}

// float -> double with integer instructions only (exact for every input:
// the exponent is rebiased and the mantissa shifted; subnormal floats are
// normalised through a leading-zero count).  The conversion instruction
// would take FP64-pipe slots that the FP64 residual needs for its FMAs.
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  uint64_t bits;
  if (e == 0xFFu) {
    bits = sign | (0x7FFull << 52) | ((uint64_t)m << 29);
  } else if (e != 0u) {
    bits = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  } else if (m == 0u) {
    bits = sign;
  } else {
    const int lz = __clz(m) - 8;
    bits = sign | ((uint64_t)(1023 - 126 - lz) << 52) | ((uint64_t)((m << lz) & 0x7FFFFFu) << 29);
  }
  return __longlong_as_double((long long)bits);
}
template <class ACC>
__device__ __forceinline__ ACC widen(float f) {
  if constexpr (sizeof(ACC) == 8)
    return f2d_int(f);
  else
    return f;
}

// y = Z x with Z complex64; ACC = float (inner solves) or double (the FP64
// refinement residual, x and y complex128).  Each warp owns 2 rows and reads
// two complex64 entries per lane per step (16-byte loads).
template <class ACC>
__global__ void __launch_bounds__(256) gemv_c64_kernel(int64_t N, const float4* __restrict__ Z4,
                                                       int64_t ldz, const void* __restrict__ xv_,
                                                       void* __restrict__ yv_, int64_t xs,
                                                       int64_t ys, int r,
                                                       const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 2;
  const int s = blockIdx.y;
  if (row0 >= N || s >= r) return;
  const int nr = (int)mn64(2, N - row0);
  ACC ar[2] = {0, 0}, ai[2] = {0, 0};
  const int64_t npair = N / 2;  // full float4 pairs (N even)
  const int64_t ld4 = ldz / 2;
  for (int64_t c2 = lane; c2 < npair; c2 += 32) {
    ACC x0r, x0i, x1r, x1i;
    if constexpr (sizeof(ACC) == 4) {
      const float4 xx = __ldg(reinterpret_cast<const float4*>(xv_) + s * (xs / 2) + c2);
      x0r = xx.x; x0i = xx.y; x1r = xx.z; x1i = xx.w;
    } else {
      const double2* xd = reinterpret_cast<const double2*>(xv_) + s * xs + 2 * c2;
      const double2 a = __ldg(xd), b = __ldg(xd + 1);
      x0r = a.x; x0i = a.y; x1r = b.x; x1i = b.y;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (k < nr) {
        const float4 z4 = __ldg(Z4 + (row0 + k) * ld4 + c2);
        const ACC zx = widen<ACC>(z4.x), zy = widen<ACC>(z4.y), zz = widen<ACC>(z4.z),
                  zw = widen<ACC>(z4.w);
        ar[k] = fma(zx, x0r, fma(-zy, x0i, ar[k]));
        ai[k] = fma(zx, x0i, fma(zy, x0r, ai[k]));
        ar[k] = fma(zz, x1r, fma(-zw, x1i, ar[k]));
        ai[k] = fma(zz, x1i, fma(zw, x1r, ai[k]));
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], o);
      ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], o);
    }
  }
  if (lane < nr) {
    const ACC vr = lane == 0 ? ar[0] : ar[1];
    const ACC vi = lane == 0 ? ai[0] : ai[1];
    if constexpr (sizeof(ACC) == 4)
      reinterpret_cast<float2*>(yv_)[s * ys + row0 + lane] = make_float2(vr, vi);
    else
      reinterpret_cast<double2*>(yv_)[s * ys + row0 + lane] = make_double2(vr, vi);
  }
}

// Y = Z X for r complex128 vectors with the stored complex64 Z widened to
// FP64 (the refinement residual of several right-hand sides).  Each warp
// owns 2 rows and RS vectors (blockIdx.y: vectors RS*y ..), so every Z
// entry is read and widened once for RS vectors, and the complex products
// take the 3M form: with s_z = z.x + z.y and s_x = x.x + x.y (XS, formed
// once per vector entry by xsum_kernel)
//   Re(z x) = z.x x.x - z.y x.y,   Im(z x) = s_z s_x - z.x x.x - z.y x.y,
// three FP64 multiply-adds per entry and vector instead of four (the FP64
// pipe bounds this product).  Its rounding error is bounded like that of
// the usual form up to a small constant (normwise; Higham, Accuracy and
// Stability of Numerical Algorithms, Sec. 23.2.4).
template <int RS>
__global__ void __launch_bounds__(64) gemv_c64_f64_3m_kernel(int64_t N,
                                                             const float4* __restrict__ Z4,
                                                             int64_t ldz,
                                                             const double2* __restrict__ X,
                                                             const double* __restrict__ XS,
                                                             double2* __restrict__ Y, int r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 2;
  const int s0 = blockIdx.y * RS;
  if (row0 >= N || s0 >= r) return;
  const int nr = (int)mn64(2, N - row0);
  double pxx[2][RS], pyy[2][RS], pss[2][RS];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int q = 0; q < RS; ++q) pxx[k][q] = pyy[k][q] = pss[k][q] = 0.0;
  const int64_t npair = N / 2;  // full float4 pairs (N even)
  const int64_t ld4 = ldz / 2;
  for (int64_t c2 = lane; c2 < npair; c2 += 32) {
    double zx[2][2], zy[2][2], zs[2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < nr) z4 = __ldg(Z4 + (row0 + k) * ld4 + c2);
      zx[k][0] = f2d_int(z4.x);
      zy[k][0] = f2d_int(z4.y);
      zx[k][1] = f2d_int(z4.z);
      zy[k][1] = f2d_int(z4.w);
      zs[k][0] = zx[k][0] + zy[k][0];
      zs[k][1] = zx[k][1] + zy[k][1];
    }
#pragma unroll
    for (int q = 0; q < RS; ++q) {
      if (s0 + q < r) {
        const double2* xd = X + (int64_t)(s0 + q) * N + 2 * c2;
        const double2 a = __ldg(xd), b = __ldg(xd + 1);
        const double2 sv = __ldg(reinterpret_cast<const double2*>(XS + (int64_t)(s0 + q) * N) + c2);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          pxx[k][q] = fma(zx[k][0], a.x, fma(zx[k][1], b.x, pxx[k][q]));
          pyy[k][q] = fma(zy[k][0], a.y, fma(zy[k][1], b.y, pyy[k][q]));
          pss[k][q] = fma(zs[k][0], sv.x, fma(zs[k][1], sv.y, pss[k][q]));
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int q = 0; q < RS; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        pxx[k][q] += __shfl_xor_sync(0xffffffffu, pxx[k][q], o);
        pyy[k][q] += __shfl_xor_sync(0xffffffffu, pyy[k][q], o);
        pss[k][q] += __shfl_xor_sync(0xffffffffu, pss[k][q], o);
      }
  if (lane != 0) return;
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int q = 0; q < RS; ++q)
      if (k < nr && s0 + q < r)
        Y[(int64_t)(s0 + q) * N + row0 + k] =
            make_double2(pxx[k][q] - pyy[k][q], pss[k][q] - pxx[k][q] - pyy[k][q]);
}

// XS[i] = X[i].x + X[i].y (the vectors' sums of the 3M products)
__global__ void xsum_kernel(const double2* __restrict__ X, double* __restrict__ XS, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 v = X[i];
    XS[i] = v.x + v.y;
  }
}
constexpr int kResidRS = 4;  // vectors per warp of the several-vector FP64 product

// y = Z x (complex64, FP32 accumulation) for a Z whose lower-right quadrant
// is minus the upper-left one (Z11 = -Z00 = -(i/omega) K1, Eq.
// global_system): with x = [x0; x1] the rows i and H + i come from row i of
// Z00, Z01 and Z10,
//   y_i = Z00_i x0 + Z01_i x1,   y_{H+i} = Z10_i x0 - Z00_i x1,
// so three quarters of Z are read.  One warp per top row i (and its bottom
// partner), two complex64 entries per lane per quadrant row and step
// (16-byte loads), two steps in flight.  (The FP64-accumulating products are
// bound by the FP64 pipe, whose work this does not reduce, and read all of
// Z.)  With nblk (complex64 near blocks, [h][alpha][g][beta] per block) the
// near part of rows i and H + i -- node i/2, alpha = i mod 2 -- is added in
// the same pass, lanes over the node's blocks.
__global__ void __launch_bounds__(256) gemv3_c64_kernel(int64_t H, const float4* __restrict__ Z4,
                                                        int64_t ldz, const float4* __restrict__ x4,
                                                        float2* __restrict__ y,
                                                        const int* __restrict__ stop,
                                                        const int32_t* __restrict__ nrowptr,
                                                        const int32_t* __restrict__ ncol,
                                                        const float2* __restrict__ nblk) {
  if (stop && *stop) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= H) return;
  float tr = 0.f, ti = 0.f, br = 0.f, bi = 0.f;
  const int64_t hp = H / 2;  // float4 pairs per quadrant row (H even)
  const float4* z00 = Z4 + i * (ldz / 2);
  const float4* z01 = z00 + hp;
  const float4* z10 = Z4 + (H + i) * (ldz / 2);
#pragma unroll 2
  for (int64_t c2 = lane; c2 < hp; c2 += 32) {
    const float4 xa = __ldg(x4 + c2), xb = __ldg(x4 + hp + c2);
    const float4 d = __ldg(z00 + c2), e = __ldg(z01 + c2), f = __ldg(z10 + c2);
    // top: Z00 x0 + Z01 x1
    tr = fmaf(d.x, xa.x, fmaf(-d.y, xa.y, tr));
    ti = fmaf(d.x, xa.y, fmaf(d.y, xa.x, ti));
    tr = fmaf(d.z, xa.z, fmaf(-d.w, xa.w, tr));
    ti = fmaf(d.z, xa.w, fmaf(d.w, xa.z, ti));
    tr = fmaf(e.x, xb.x, fmaf(-e.y, xb.y, tr));
    ti = fmaf(e.x, xb.y, fmaf(e.y, xb.x, ti));
    tr = fmaf(e.z, xb.z, fmaf(-e.w, xb.w, tr));
    ti = fmaf(e.z, xb.w, fmaf(e.w, xb.z, ti));
    // bottom: Z10 x0 - Z00 x1
    br = fmaf(f.x, xa.x, fmaf(-f.y, xa.y, br));
    bi = fmaf(f.x, xa.y, fmaf(f.y, xa.x, bi));
    br = fmaf(f.z, xa.z, fmaf(-f.w, xa.w, br));
    bi = fmaf(f.z, xa.w, fmaf(f.w, xa.z, bi));
    br = fmaf(-d.x, xb.x, fmaf(d.y, xb.y, br));
    bi = fmaf(-d.x, xb.y, fmaf(-d.y, xb.x, bi));
    br = fmaf(-d.z, xb.z, fmaf(d.w, xb.w, br));
    bi = fmaf(-d.z, xb.w, fmaf(-d.w, xb.z, bi));
  }
  if (nblk) {
    const int64_t n = i >> 1;
    const int al = (int)(i & 1);
    const float2* xf = reinterpret_cast<const float2*>(x4);
    for (int32_t q = nrowptr[n] + lane; q < nrowptr[n + 1]; q += 32) {
      const int64_t jn = ncol[q];
      const float2* b = nblk + (int64_t)q * 16;
#pragma unroll
      for (int gb = 0; gb < 4; ++gb) {
        const float2 xv = xf[(gb >> 1) * H + 2 * jn + (gb & 1)];
        const float2 mt = b[al * 4 + gb], mb = b[(2 + al) * 4 + gb];
        tr = fmaf(mt.x, xv.x, fmaf(-mt.y, xv.y, tr));
        ti = fmaf(mt.x, xv.y, fmaf(mt.y, xv.x, ti));
        br = fmaf(mb.x, xv.x, fmaf(-mb.y, xv.y, br));
        bi = fmaf(mb.x, xv.y, fmaf(mb.y, xv.x, bi));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    ti += __shfl_xor_sync(0xffffffffu, ti, o);
    br += __shfl_xor_sync(0xffffffffu, br, o);
    bi += __shfl_xor_sync(0xffffffffu, bi, o);
  }
  if (lane == 0) y[i] = make_float2(tr, ti);
  if (lane == 1) y[H + i] = make_float2(br, bi);
}

// y += near * x for the near blocks (test node rows, 4 x 4 complex blocks
// [h][alpha][g][beta]).  One warp per test node: lanes take the row's
// blocks, each block contributes to the node's 4 outputs, then a warp
// reduction.  BT = block element type, VT = vector element type.
template <class BT, class VT>
__global__ void __launch_bounds__(256) near_spmv_kernel(int64_t nn, const int32_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col,
                                                        const BT* __restrict__ blk,
                                                        const VT* __restrict__ x, VT* __restrict__ y,
                                                        int64_t xs, int64_t ys, int r,
                                                        const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  const int s = blockIdx.y;
  if (i >= nn || s >= r) return;
  const int64_t H = 2 * nn;
  using R = decltype(x[0].x);
  R ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
  const VT* xv = x + s * xs;
  for (int32_t q = rowptr[i] + lane; q < rowptr[i + 1]; q += 32) {
    const int64_t j = col[q];
    VT xj[4];
#pragma unroll
    for (int gb = 0; gb < 4; ++gb) xj[gb] = xv[(gb >> 1) * H + 2 * j + (gb & 1)];
    const BT* b = blk + (int64_t)q * 16;
#pragma unroll
    for (int ha = 0; ha < 4; ++ha)
#pragma unroll
      for (int gb = 0; gb < 4; ++gb) {
        const BT m = b[ha * 4 + gb];
        ar[ha] = fma((R)m.x, xj[gb].x, fma(-(R)m.y, xj[gb].y, ar[ha]));
        ai[ha] = fma((R)m.x, xj[gb].y, fma((R)m.y, xj[gb].x, ai[ha]));
      }
  }
#pragma unroll
  for (int ha = 0; ha < 4; ++ha)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar[ha] += __shfl_xor_sync(0xffffffffu, ar[ha], o);
      ai[ha] += __shfl_xor_sync(0xffffffffu, ai[ha], o);
    }
  if (lane < 4) {
    R vr = ar[0], vi = ai[0];
#pragma unroll
    for (int ha = 1; ha < 4; ++ha)
      if (lane == ha) {
        vr = ar[ha];
        vi = ai[ha];
      }
    VT* yo = y + s * ys + (lane >> 1) * H + 2 * i + (lane & 1);
    yo->x += vr;
    yo->y += vi;
  }
}

// ============================================================ batched LU
// Blocks are d x d complex128 row-major, block b at offset b*d*d, its
// active size sz[b] <= d.  Right-looking blocked LU with panels of LUW
// columns (narrow: the panels run one block per CTA, on few SMs, and their
// FP64 work per row grows with the width); the explicit inverses and the
// dense solves use tiles of NBK columns.
constexpr int NBK = 32;
constexpr int LUW = 16;

template <class CT>
__device__ __forceinline__ auto cabs1T(CT a) -> decltype(a.x) {
  return fabs(a.x) + fabs(a.y);
}
template <class CT>
__device__ __forceinline__ CT cdivT(CT a, CT b) {
  const auto den = b.x * b.x + b.y * b.y;
  return CT{(a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den};
}
// a -= b c and a += b c (complex) as four multiply-adds: written out, the
// compiler would form each part as a product, a multiply-add and an addition
template <class CT>
__device__ __forceinline__ void cfms(CT& a, CT b, CT c) {
  a.x = fma(-b.x, c.x, a.x);
  a.x = fma(b.y, c.y, a.x);
  a.y = fma(-b.x, c.y, a.y);
  a.y = fma(-b.y, c.x, a.y);
}
template <class CT>
__device__ __forceinline__ void cfma(CT& a, CT b, CT c) {
  a.x = fma(b.x, c.x, a.x);
  a.x = fma(-b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y);
  a.y = fma(b.y, c.x, a.y);
}
__device__ __forceinline__ double2 cdiv2(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// factor panel columns [k0, k0+W) of every block; row swaps are applied
// to whole rows, or with 'defer' to the panel's columns only (the others
// then take them from lu_swap_trsm_kernel).  READING: pivot = first row
// maximising |Re| + |Im|.
template <class CT, int W>
__global__ void __launch_bounds__(256) lu_panel_kernel(CT* __restrict__ A, int64_t d,
                                                       const int32_t* __restrict__ sz, int k0,
                                                       int32_t* __restrict__ piv,
                                                       int32_t* __restrict__ status, int defer) {
  const int b = blockIdx.x;
  const int n = sz[b];
  if (k0 >= n) return;
  using RT = decltype(CT{}.x);
  CT* M = A + (int64_t)b * d * d;
  __shared__ RT sv[256];
  __shared__ int si[256];
  __shared__ CT spiv;
  const int kend = min(k0 + W, n);
  for (int k = k0; k < kend; ++k) {
    // pivot search in column k, rows k..n-1
    RT best = -1;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const RT v = cabs1T(M[(int64_t)i * d + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const RT v2 = sv[threadIdx.x + o];
        const int i2 = si[threadIdx.x + o];
        if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
          sv[threadIdx.x] = v2;
          si[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    const int p = si[0];
    const bool singular = !(sv[0] > 0.0);
    if (threadIdx.x == 0) {
      piv[(int64_t)b * d + k] = p;
      if (singular) atomicCAS(status, 0, b + 1);
    }
    if (p != k)
      for (int j = (defer ? k0 : 0) + threadIdx.x; j < (defer ? kend : n); j += blockDim.x) {
        const CT t = M[(int64_t)k * d + j];
        M[(int64_t)k * d + j] = M[(int64_t)p * d + j];
        M[(int64_t)p * d + j] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) spiv = singular ? CT{1, 0} : M[(int64_t)k * d + k];
    __syncthreads();
    const CT pv = spiv;
    const auto pden = pv.x * pv.x + pv.y * pv.y;
    const CT rpv = CT{pv.x / pden, -pv.y / pden};
    // multipliers (by the pivot's reciprocal) and rank-1 update of the panel
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const CT a = M[(int64_t)i * d + k];
      const CT l = CT{a.x * rpv.x - a.y * rpv.y, a.x * rpv.y + a.y * rpv.x};
      M[(int64_t)i * d + k] = l;
      for (int j = k + 1; j < kend; ++j) {
        const CT u = M[(int64_t)k * d + j];
        CT a = M[(int64_t)i * d + j];
        cfms(a, l, u);
        M[(int64_t)i * d + j] = a;
      }
    }
    __syncthreads();
  }
}

// Same factorisation of panel columns [k0, k0+W), with rows k0..n-1 of the
// panel held in shared memory (one thread per row, blockDim >= n - k0): the
// pivot search is a warp-shuffle arg-max, the rank-1 updates run on shared
// memory, and the panel's row swaps are applied to the columns outside it
// afterwards, in the order they were chosen (the same matrix as swapping
// whole rows at each step), unless 'defer' leaves them to lu_swap_trsm_kernel.
// Pivot: first row maximising |Re| + |Im|.
// barrier of the panel's nthr threads (a multiple of 32; id 9: the
// tile groups of lu_step_kernel use 1 .. 8)
__device__ __forceinline__ void panel_bar(int nthr) {
  asm volatile("bar.sync 9, %0;" ::"r"(nthr) : "memory");
}

template <class CT, int W>
__device__ __forceinline__ void lu_panel_smem_body(CT* __restrict__ A, int64_t d,
                                                   const int32_t* __restrict__ sz, int k0,
                                                   int32_t* __restrict__ piv,
                                                   int32_t* __restrict__ status, int defer,
                                                   int b, unsigned char* lu_smem, int nthr) {
  using RT = decltype(CT{}.x);
  constexpr int LD = W + 1;
  __shared__ RT wv[32];
  __shared__ int wi[32];
  __shared__ int sp[W];
  __shared__ CT srpv;
  const int n = sz[b];
  if (k0 >= n || (int)threadIdx.x >= nthr) return;
  const int w = min(W, n - k0);
  const int rows = n - k0;
  const int t = threadIdx.x;
  CT* P = (CT*)lu_smem;  // [rows][LD]
  CT* M = A + (int64_t)b * d * d;
  for (int e = t; e < rows * w; e += nthr) {
    const int i = e / w, j = e - i * w;
    P[i * LD + j] = M[(int64_t)(k0 + i) * d + k0 + j];
  }
  panel_bar(nthr);
  for (int k = 0; k < w; ++k) {
    RT v = -1;
    int vi = rows;
    if (t >= k && t < rows) {
      v = cabs1T(P[t * LD + k]);
      vi = t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const RT v2 = __shfl_down_sync(0xffffffffu, v, o);
      const int i2 = __shfl_down_sync(0xffffffffu, vi, o);
      if (v2 > v || (v2 == v && i2 < vi)) {
        v = v2;
        vi = i2;
      }
    }
    if ((t & 31) == 0) {
      wv[t >> 5] = v;
      wi[t >> 5] = vi;
    }
    panel_bar(nthr);
    if (t < 32) {
      const int nw = (nthr >> 5);
      v = t < nw ? wv[t] : (RT)-1;
      vi = t < nw ? wi[t] : rows;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const RT v2 = __shfl_down_sync(0xffffffffu, v, o);
        const int i2 = __shfl_down_sync(0xffffffffu, vi, o);
        if (v2 > v || (v2 == v && i2 < vi)) {
          v = v2;
          vi = i2;
        }
      }
      if (t == 0) {
        const bool singular = !(v > 0);
        if (singular) {
          vi = k;
          atomicCAS(status, 0, b + 1);
        }
        sp[k] = vi;
        // reciprocal of the pivot (row vi before the swap), once per column
        const CT pv = singular ? CT{1, 0} : P[vi * LD + k];
        const auto pden = pv.x * pv.x + pv.y * pv.y;
        srpv = CT{pv.x / pden, -pv.y / pden};
        piv[(int64_t)b * d + k0 + k] = k0 + vi;
      }
    }
    panel_bar(nthr);
    const int p = sp[k];
    if (p != k && t < w) {
      const CT x = P[k * LD + t];
      P[k * LD + t] = P[p * LD + t];
      P[p * LD + t] = x;
    }
    panel_bar(nthr);
    const CT rpv = srpv;  // multipliers by the pivot's reciprocal
    if (t > k && t < rows) {
      CT* row = P + t * LD;
      const CT* prow = P + k * LD;
      const CT a = row[k];
      const CT l = CT{a.x * rpv.x - a.y * rpv.y, a.x * rpv.y + a.y * rpv.x};
      row[k] = l;
      for (int j = k + 1; j < w; ++j) {
        const CT u = prow[j];
        cfms(row[j], l, u);
      }
    }
    panel_bar(nthr);
  }
  for (int e = t; e < rows * w; e += nthr) {
    const int i = e / w, j = e - i * w;
    M[(int64_t)(k0 + i) * d + k0 + j] = P[i * LD + j];
  }
  if (defer) return;
  for (int c = t; c < n; c += nthr) {
    if (c >= k0 && c < k0 + w) continue;
    for (int k = 0; k < w; ++k) {
      const int p = sp[k];
      if (p != k) {
        const CT x = M[(int64_t)(k0 + k) * d + c];
        M[(int64_t)(k0 + k) * d + c] = M[(int64_t)(k0 + p) * d + c];
        M[(int64_t)(k0 + p) * d + c] = x;
      }
    }
  }
}

template <class CT, int W>
__global__ void __launch_bounds__(1024) lu_panel_smem_kernel(CT* __restrict__ A, int64_t d,
                                                             const int32_t* __restrict__ sz,
                                                             int k0, int32_t* __restrict__ piv,
                                                             int32_t* __restrict__ status,
                                                             int defer) {
  extern __shared__ __align__(16) unsigned char lu_smem[];
  lu_panel_smem_body<CT, W>(A, d, sz, k0, piv, status, defer, blockIdx.x, lu_smem, blockDim.x);
}

// One 32 x TN tile of the trailing update, C -= A B with A the tile's rows
// of the panel columns [k0, k0 + W) and B the panel's rows of the tile's
// columns, staged in shared memory together with the sums s = x + y of
// every entry.  The complex products take the 3M form (three real products
// instead of four): Re(ab) = a.x b.x - a.y b.y and
// Im(ab) = s_a s_b - a.x b.x - a.y b.y, so the contraction costs three FP64
// multiply-adds per complex multiply-add; the sums cost one addition per
// staged entry.  Its rounding error is bounded like that of the usual form
// up to a small constant (normwise; Higham, Accuracy and Stability of
// Numerical Algorithms, Sec. 23.2.4).
template <int W, int TN, int TR = 32>
struct Tile3M {
  double2 a[TR][W + 1];
  double as[TR][W + 1];
  double2 b[W][TN + 1];
  double bs[W][TN + 1];
};

// stage the tile with rows [tr, tr + TR), columns [tc, tc + TN) of block M
// (active size n, columns below c1, panel width w); GT threads, lt = rank
template <int W, int TN, int GT, int TR = 32>
__device__ __forceinline__ void tile3m_load(Tile3M<W, TN, TR>& T, const double2* __restrict__ M,
                                            int64_t d, int64_t tr, int64_t tc, int k0, int n,
                                            int64_t c1, int w, int lt) {
  for (int t = lt; t < TR * W; t += GT) {
    const int i = t / W, k = t % W;
    const int64_t gr = tr + i;
    const double2 v = (gr < n && k < w) ? M[gr * d + k0 + k] : make_double2(0.0, 0.0);
    T.a[i][k] = v;
    T.as[i][k] = v.x + v.y;
  }
  for (int t = lt; t < W * TN; t += GT) {
    const int k = t / TN, j = t % TN;
    const int64_t gc = tc + j;
    const double2 v = (gc < c1 && k < w) ? M[(int64_t)(k0 + k) * d + gc] : make_double2(0.0, 0.0);
    T.b[k][j] = v;
    T.bs[k][j] = v.x + v.y;
  }
}

// C -= A B for the staged tile: thread lt owns rows ty + 8 i (i < TR / 8)
// and columns tx + (TN / JN) j (j < JN) of the tile, 8 * TN / JN threads
template <int W, int TN, int JN, int TR = 32>
__device__ __forceinline__ void tile3m_update(const Tile3M<W, TN, TR>& T, double2* __restrict__ M,
                                              int64_t d, int64_t tr, int64_t tc, int n,
                                              int64_t c1, int lt) {
  constexpr int CX = TN / JN, RI = TR / 8;
  const int ty = lt / CX, tx = lt % CX;
  double pxx[RI][JN], pyy[RI][JN], pss[RI][JN];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < JN; ++j) pxx[i][j] = pyy[i][j] = pss[i][j] = 0.0;
#pragma unroll 4
  for (int k = 0; k < W; ++k) {
    double2 av[RI], bv[JN];
    double as[RI], bs[JN];
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      av[i] = T.a[ty + 8 * i][k];
      as[i] = T.as[ty + 8 * i][k];
    }
#pragma unroll
    for (int j = 0; j < JN; ++j) {
      bv[j] = T.b[k][tx + CX * j];
      bs[j] = T.bs[k][tx + CX * j];
    }
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < JN; ++j) {
        pxx[i][j] = fma(av[i].x, bv[j].x, pxx[i][j]);
        pyy[i][j] = fma(av[i].y, bv[j].y, pyy[i][j]);
        pss[i][j] = fma(as[i], bs[j], pss[i][j]);
      }
  }
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < JN; ++j) {
      const int64_t gr = tr + ty + 8 * i, gc = tc + tx + CX * j;
      if (gr < n && gc < c1) {
        double2 v = M[gr * d + gc];
        v.x -= pxx[i][j] - pyy[i][j];
        v.y -= pss[i][j] - pxx[i][j] - pyy[i][j];
        M[gr * d + gc] = v;
      }
    }
}

// One step of the blocked LU in one launch.  The dynamic shared memory
// (kLuStepSmem) admits one CTA per SM, so no two CTAs share an SM's FP64
// pipe.  CTAs 0 .. nb-1 first factor panel k1 of their block (rows in shared
// memory, swaps held back); then each group of 128 threads of every CTA takes
// 32 x 32 tiles of the trailing update of panel k0 over columns [c0, d) one
// at a time (the first one assigned so that the tiles spread over the SMs,
// the others from a queue, an atomic counter) and synchronises with a
// barrier of its own.  The panel's columns [k1, k1 + W) were updated before
// this launch and lie outside [c0, d), so the two roles touch disjoint
// entries and never wait on each other.  Without a panel (k1 < 0) every CTA
// only takes tiles.
constexpr int kLuStepThreads = 512;
constexpr int kLuGroup = 128;  // threads per tile group (4 x 2 outputs each)
constexpr size_t kLuStepSmem = 140 * 1024;
static_assert(sizeof(Tile3M<LUW, 32>) * (kLuStepThreads / kLuGroup) <= kLuStepSmem,
              "the tile groups' staging must fit in the step kernel's shared memory");
__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kLuGroup) : "memory");
}
template <int W>
__global__ void __launch_bounds__(kLuStepThreads) lu_step_kernel(
    double2* __restrict__ A, int64_t d, const int32_t* __restrict__ sz, int k0, int k1,
    int64_t c0, int nb, int32_t* __restrict__ piv, int32_t* __restrict__ status,
    unsigned* __restrict__ queue) {
  extern __shared__ __align__(16) unsigned char lu_smem[];
  if (k1 >= 0 && (int)blockIdx.x < nb) {
    // one thread per panel row (whole warps): fewer threads in the column
    // reductions of the short late panels
    const int rows = (int)(d - k1);
    const int nthr = max(32, min((int)blockDim.x, (rows + 31) / 32 * 32));
    lu_panel_smem_body<double2, W>(A, d, sz, k1, piv, status, 1, blockIdx.x, lu_smem, nthr);
    __syncthreads();  // the shared memory is the tiles' from here on
  }
  constexpr int TN = 32, GT = kLuGroup;
  const int64_t r0 = k0 + W;
  const int64_t rt_n = (d - r0 + 31) / 32, ct_n = (d - c0 + TN - 1) / TN;
  const int64_t per_b = rt_n * ct_n;
  const unsigned tiles = (unsigned)((int64_t)nb * per_b);
  if (rt_n <= 0 || ct_n <= 0) return;
  const int grp = threadIdx.x / GT, lt = threadIdx.x % GT;
  Tile3M<W, TN>& T = reinterpret_cast<Tile3M<W, TN>*>(lu_smem)[grp];
  __shared__ unsigned tb[kLuStepThreads / GT];
  const int bar = 1 + grp;  // barrier 0 is __syncthreads'
  // The first tile of each group of the CTAs without a panel is assigned
  // statically, tile g * (G - np) + (c - np) to group g of CTA c, so that few
  // tiles spread over the SMs instead of filling the first SMs to ask; the
  // rest come from the queue (tickets after the static ones).
  const unsigned npan = k1 >= 0 ? (unsigned)min(nb, (int)gridDim.x) : 0u;
  const unsigned nfree = gridDim.x - npan;
  const unsigned nstatic = nfree * (kLuStepThreads / GT);
  bool stat = blockIdx.x >= npan;
  for (;;) {
    if (lt == 0) tb[grp] = stat ? (unsigned)grp * nfree + (blockIdx.x - npan)
                                : nstatic + atomicAdd(queue, 1u);
    stat = false;
    group_bar(bar);
    const unsigned tile = tb[grp];
    if (tile >= tiles) break;  // uniform over the group
    const int b = (int)(tile / per_b);
    const int64_t rem = (int64_t)tile - (int64_t)b * per_b;
    const int n = sz[b];
    const int64_t c1 = mn64(d, n);
    const int64_t tr = r0 + (rem / ct_n) * 32, tc = c0 + (rem % ct_n) * TN;
    const bool act = !(k0 >= n || tr >= n || tc >= c1);
    const int w = act ? min(W, n - k0) : 0;
    double2* M = A + (int64_t)b * d * d;
    if (act) tile3m_load<W, TN, GT>(T, M, d, tr, tc, k0, n, c1, w, lt);
    group_bar(bar);
    if (act) tile3m_update<W, TN, 2>(T, M, d, tr, tc, n, c1, lt);
    group_bar(bar);  // before the group's next tile loads and queue read
  }
}

// B[k0:k0+w, c0:c1] <- L_kk^{-1} B[...] (unit lower, L from A) or
// U_kk^{-1} B[...] (upper, non-unit); one thread per column, the W x W
// diagonal tile staged in shared memory (its entries are read by every
// thread in the same order: broadcasts).
template <class CT, int W>
__global__ void trsm_tile_kernel(const CT* __restrict__ A, CT* __restrict__ B, int64_t d,
                                 int64_t ldb, int64_t bstride, const int32_t* __restrict__ sz,
                                 int k0, int w_max, int64_t c0, int64_t c1_cap, int upper) {
  __shared__ CT T[W][W];
  const int b = blockIdx.y;
  const int n = sz[b];
  if (k0 >= n) return;
  const int w = min(w_max, n - k0);
  const int64_t c1 = c1_cap < 0 ? n : mn64(c1_cap, n);
  if (c0 + (int64_t)blockIdx.x * blockDim.x >= c1) return;  // uniform over the CTA
  const CT* M = A + (int64_t)b * d * d;
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    const int i = e / W, j = e % W;
    T[i][j] = (i < w && j < w) ? M[(int64_t)(k0 + i) * d + k0 + j] : CT{0, 0};
  }
  __syncthreads();
  const int64_t c = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= c1) return;
  CT* X = B + (int64_t)b * bstride;
  // fixed-size, fully unrolled loops keep v[] in registers; rows >= w are
  // inert (zero right-hand side, never written back)
  CT v[W];
#pragma unroll
  for (int i = 0; i < W; ++i)
    v[i] = i < w ? X[(int64_t)(k0 + i) * ldb + c] : CT{0, 0};
  if (!upper) {
#pragma unroll
    for (int i = 1; i < W; ++i)
#pragma unroll
      for (int j = 0; j < i; ++j) {
        const CT l = T[i][j];
        cfms(v[i], l, v[j]);
      }
  } else {
#pragma unroll
    for (int i = W - 1; i >= 0; --i) {
      if (i < w) {
#pragma unroll
        for (int j = i + 1; j < W; ++j) {
          const CT u = T[i][j];
          cfms(v[i], u, v[j]);
        }
        v[i] = cdivT(v[i], T[i][i]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < W; ++i)
    if (i < w) X[(int64_t)(k0 + i) * ldb + c] = v[i];
}

// Inverses of the 32 x 32 diagonal tiles of every block's complex64 LU
// factors (the unit lower L and the upper U), rows and columns beyond the
// block's active size taken from the identity: CTA (tile, block, lu) with
// thread j computing column j by substitution.  Tinv holds [nb][ntile][2]
// tiles of 32 x 32 (row-major).
__global__ void __launch_bounds__(32) tile_inverse_kernel(const float2* __restrict__ A, int64_t d,
                                                          const int32_t* __restrict__ sz,
                                                          int ntile, float2* __restrict__ Tinv) {
  __shared__ float2 sD[32][33];
  const int tile = blockIdx.x, b = blockIdx.y, lu = blockIdx.z;
  const int n = sz[b], r = tile * 32;
  if (r >= n) return;
  const int kn = min(32, n - r);
  const int j = threadIdx.x;
  const float2* F = A + (int64_t)b * d * d;
  for (int i = 0; i < 32; ++i)
    sD[i][j] = (i < kn && j < kn) ? F[(int64_t)(r + i) * d + r + j] : make_float2(i == j ? 1.f : 0.f, 0.f);
  __syncwarp();
  float2 x[32];
  if (lu == 0) {  // L (unit lower)
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float2 a = make_float2(i == j ? 1.f : 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < i; ++k) {
        const float2 l = sD[i][k];
        cfms(a, l, x[k]);
      }
      x[i] = a;
    }
  } else {  // U (upper)
#pragma unroll
    for (int i = 31; i >= 0; --i) {
      float2 a = make_float2(i == j ? 1.f : 0.f, 0.f);
#pragma unroll
      for (int k = i + 1; k < 32; ++k) {
        const float2 u = sD[i][k];
        cfms(a, u, x[k]);
      }
      x[i] = cdivT(a, sD[i][i]);
    }
  }
  float2* O = Tinv + (((int64_t)b * ntile + tile) * 2 + lu) * 1024;
#pragma unroll
  for (int i = 0; i < 32; ++i) O[i * 32 + j] = x[i];
}

// Explicit inverses of the blocks from their complex64 LU factors (unit
// lower L and upper U in A, the row swaps in piv, the diagonal tiles'
// inverses in Tinv) in one launch.  CTA (x, b) computes the CW columns
// j0 = x CW .. j0 + CW - 1 of M = U^{-1} L^{-1} of block b, i.e. solves
// L U m_j = e_j, by forward and back substitution in tiles of 32 rows.
// Thread t holds rows t, t + 512, .. (RPT of them) of those columns in
// registers.  Per tile: the tile's rows go to shared memory and are
// multiplied by the inverse of the diagonal tile (thread (lane, warp) gives
// row lane of column warp); then every row outside the tile subtracts the
// tile's contribution, its factor entries read as 16-byte loads.  Column j of
// L^{-1} is zero above row j, so the forward pass starts at the tile of the
// CTA's first column.  With P e_c = e_pi(c) for the recorded swaps
// (P A = L U), the inverse U^{-1} L^{-1} P has column c equal to column
// pi(c) of M.
constexpr int kInvCW = 16;        // columns of M per CTA (= warps per CTA)
constexpr int kInvThreads = 512;  // 32 * kInvCW

// the tile after (pass, tile): forward tiles up to the last, then backward
__device__ __forceinline__ bool tile_after(int& pass, int& tile, int ntile) {
  if (pass == 0) {
    if (tile + 1 < ntile) {
      ++tile;
    } else {
      pass = 1;
      tile = ntile - 1;
    }
    return true;
  }
  if (tile == 0) return false;
  --tile;
  return true;
}

template <int RPT>
__global__ void __launch_bounds__(kInvThreads, RPT == 1 ? 2 : 1) block_inverse_cols_kernel(
    const float2* __restrict__ A, int64_t d, const int32_t* __restrict__ sz,
    const int32_t* __restrict__ piv, const float2* __restrict__ Tinv, int ntile_max,
    float2* __restrict__ inv) {
  constexpr int CW = kInvCW;
  __shared__ __align__(16) float2 sT[32][CW];   // the tile's rows
  __shared__ __align__(16) float2 sT2[32][CW];  // the same, finished
  __shared__ float2 sD[32][33];                 // inverse of the diagonal tile
  __shared__ int sPiv[kInvThreads * RPT];
  __shared__ int sTarget[CW];
  const int b = blockIdx.y;
  const int n = sz[b];
  const int j0 = blockIdx.x * CW;
  if (j0 >= n) return;  // uniform over the CTA
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const float2* F = A + (int64_t)b * d * d;
  const float2* TI = Tinv + (int64_t)b * ntile_max * 2 * 1024;
  for (int k = t; k < n; k += kInvThreads) sPiv[k] = piv[(int64_t)b * d + k];
  if (t < CW) sTarget[t] = -1;
  const int ntile = (n + 31) / 32;
  float2 dg[2];
  // two entries of the diagonal inverse of tile (pass, tile), loaded one
  // tile ahead
  auto fetch = [&](int pass, int tile) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      dg[h] = __ldg(TI + ((int64_t)tile * 2 + pass) * 1024 + t + h * kInvThreads);
  };
  int pass = 0, tile = j0 / 32;
  fetch(pass, tile);
  __syncthreads();
  // targets: the inverse's column c with pi(c) = j0 + jj
  for (int c = t; c < n; c += kInvThreads) {
    int pos = c;
    for (int k = 0; k < n; ++k) {
      const int p = sPiv[k];
      pos = pos == k ? p : (pos == p ? k : pos);
    }
    if (pos >= j0 && pos < j0 + CW) sTarget[pos - j0] = c;
  }
  float2 x[RPT][CW];
#pragma unroll
  for (int q = 0; q < RPT; ++q)
#pragma unroll
    for (int jj = 0; jj < CW; ++jj)
      x[q][jj] = make_float2(t + q * kInvThreads == j0 + jj ? 1.f : 0.f, 0.f);
  for (;;) {
    const bool lower = pass == 0;
    const int r = tile * 32, kn = min(32, n - r);
    const int ow = (r % kInvThreads) / 32, oq = r / kInvThreads;  // owner warp, slot
    // 1. the tile's rows and the diagonal tile's inverse to shared memory
    if (warp == ow) {
#pragma unroll
      for (int q = 0; q < RPT; ++q)
        if (q == oq) {
#pragma unroll
          for (int jj = 0; jj < CW; ++jj) sT[lane][jj] = x[q][jj];
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = t + h * kInvThreads;
      sD[e / 32][e % 32] = dg[h];
    }
    __syncthreads();
    // 2. finished rows: row lane of column warp of (diagonal tile)^-1 sT
    {
      float2 v = make_float2(0.f, 0.f);
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        const float2 a = sD[lane][k], xk = sT[k][warp];
        cfma(v, a, xk);
      }
      sT2[lane][warp] = v;
    }
    __syncthreads();
    // 3. the tile's rows back to their owners; the rows below (L) or above
    //    (U) subtract F[row, r:r+kn) times the tile
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int row = t + q * kInvThreads;
      if (row >= n) continue;
      if (row >= r && row < r + 32) {
#pragma unroll
        for (int jj = 0; jj < CW; ++jj) x[q][jj] = sT2[row - r][jj];
        continue;
      }
      if (lower ? row < r + 32 : row >= r) continue;
      const float4* f4 = reinterpret_cast<const float4*>(F + (int64_t)row * d + r);
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        if (2 * k2 >= kn) break;
        const float4 ff = __ldg(f4 + k2);  // entries k = 2 k2, 2 k2 + 1
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = 2 * k2 + h;
          if (k >= kn) break;
          const float fx = h ? ff.z : ff.x, fy = h ? ff.w : ff.y;
          const float4* tk = reinterpret_cast<const float4*>(&sT2[k][0]);
#pragma unroll
          for (int j2 = 0; j2 < CW / 2; ++j2) {
            const float4 tv = tk[j2];
            const float2 f2 = make_float2(fx, fy);
            cfms(x[q][2 * j2], f2, make_float2(tv.x, tv.y));
            cfms(x[q][2 * j2 + 1], f2, make_float2(tv.z, tv.w));
          }
        }
      }
    }
    // the next tile's diagonal inverse, in flight across the barrier
    const bool more = tile_after(pass, tile, ntile);
    if (more) fetch(pass, tile);
    __syncthreads();  // before the next tile overwrites sT, sT2 and sD
    if (!more) break;
  }
  float2* O = inv + (int64_t)b * d * d;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int row = t + q * kInvThreads;
    if (row >= n) continue;
#pragma unroll
    for (int jj = 0; jj < CW; ++jj) {
      const int c = sTarget[jj];
      if (j0 + jj < n && c >= 0) O[(int64_t)row * d + c] = x[q][jj];
    }
  }
}

// C[r0:r1, c0:c1] -= A[r0:r1, k0:k0+w] * Bm[k0:k0+w, c0:c1] per block:
// 64 x 64 output tiles, 256 threads with 4 x 4 complex accumulators each.
// Row range is [r0, r1) with r1 = n (the block's size) if r1_cap < 0.
template <class CT, int W>
__global__ void __launch_bounds__(256) gemm_update_kernel(const CT* __restrict__ A,
                                                          const CT* __restrict__ Bm,
                                                          CT* __restrict__ Cm, int64_t d,
                                                          int64_t ldb, int64_t bstride,
                                                          const int32_t* __restrict__ sz, int k0,
                                                          int64_t r0, int64_t r1_cap, int64_t c0,
                                                          int64_t c1_cap) {
  const int b = blockIdx.z;
  const int n = sz[b];
  if (k0 >= n) return;
  const int w = min(W, n - k0);
  const int64_t r1 = r1_cap < 0 ? n : mn64(r1_cap, n);
  const int64_t c1 = c1_cap < 0 ? n : mn64(c1_cap, n);
  const int64_t tr = r0 + (int64_t)blockIdx.y * 64, tc = c0 + (int64_t)blockIdx.x * 64;
  if (tr >= r1 || tc >= c1) return;
  const CT* M = A + (int64_t)b * d * d;
  const CT* Bb = Bm + (int64_t)b * bstride;
  CT* Cb = Cm + (int64_t)b * bstride;
  __shared__ CT sA[64][W + 1];
  __shared__ CT sB[W][64 + 1];
  for (int t = threadIdx.x; t < 64 * W; t += 256) {
    const int i = t / W, k = t % W;
    const int64_t gr = tr + i;
    sA[i][k] = (gr < r1 && k < w) ? M[gr * d + k0 + k] : CT{0, 0};
  }
  for (int t = threadIdx.x; t < W * 64; t += 256) {
    const int k = t / 64, j = t % 64;
    const int64_t gc = tc + j;
    sB[k][j] = (gc < c1 && k < w) ? Bb[(int64_t)(k0 + k) * ldb + gc] : CT{0, 0};
  }
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  CT acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = CT{0, 0};
  for (int k = 0; k < W; ++k) {
    CT a[4], bb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = sA[ty + 16 * i][k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bb[j] = sB[k][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j].x = fma(a[i].x, bb[j].x, fma(-a[i].y, bb[j].y, acc[i][j].x));
        acc[i][j].y = fma(a[i].x, bb[j].y, fma(a[i].y, bb[j].x, acc[i][j].y));
      }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gr = tr + ty + 16 * i, gc = tc + tx + 16 * j;
      if (gr < r1 && gc < c1) {
        CT v = Cb[gr * ldb + gc];
        v.x -= acc[i][j].x;
        v.y -= acc[i][j].y;
        Cb[gr * ldb + gc] = v;
      }
    }
}

// After panel [k0, k0+W) is factored: its row swaps (recorded in piv, in
// order) applied to every column outside the panel, and for the columns
// right of it the row panel of U, U12 = L11^{-1} A12 (L11 unit lower from
// the panel).  One thread per column, one warp per CTA (the FP64 work of
// the solves spreads over all SMs).  (Composing the swaps into one gather of
// the at most 2W rows they reach, per warp, made the kernel slower: 34 vs
// 27 us per launch at level 3.)
template <int W>
__global__ void __launch_bounds__(32) lu_swap_trsm_kernel(double2* __restrict__ A, int64_t d,
                                                          const int32_t* __restrict__ sz, int k0,
                                                          const int32_t* __restrict__ piv) {
  __shared__ double2 T[W][W];
  __shared__ double Ts[W][W];
  const int b = blockIdx.y;
  const int n = sz[b];
  if (k0 >= n) return;
  const int w = min(W, n - k0);
  if ((int64_t)blockIdx.x * blockDim.x >= n) return;  // uniform over the CTA
  double2* M = A + (int64_t)b * d * d;
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    const int i = e / W, j = e % W;
    const double2 l = (i < w && j < w) ? M[(int64_t)(k0 + i) * d + k0 + j] : make_double2(0.0, 0.0);
    T[i][j] = l;
    Ts[i][j] = l.x + l.y;
  }
  __syncthreads();
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n || (c >= k0 && c < k0 + w)) return;
  const int32_t* pv = piv + (int64_t)b * d + k0;
  for (int k = 0; k < w; ++k) {
    const int p = pv[k];
    if (p != k0 + k) {
      const double2 x = M[(int64_t)(k0 + k) * d + c];
      M[(int64_t)(k0 + k) * d + c] = M[(int64_t)p * d + c];
      M[(int64_t)p * d + c] = x;
    }
  }
  if (c < k0 + w) return;
  // forward substitution with the 3M products (tile3m_update): the sums of
  // v[j] are formed once it is final, those of L in shared memory
  double2 v[W];
  double vs[W];
#pragma unroll
  for (int i = 0; i < W; ++i) v[i] = i < w ? M[(int64_t)(k0 + i) * d + c] : make_double2(0.0, 0.0);
  vs[0] = v[0].x + v[0].y;
#pragma unroll
  for (int i = 1; i < W; ++i) {
    double pxx = 0.0, pyy = 0.0, pss = 0.0;
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const double2 l = T[i][j];
      pxx = fma(l.x, v[j].x, pxx);
      pyy = fma(l.y, v[j].y, pyy);
      pss = fma(Ts[i][j], vs[j], pss);
    }
    v[i].x -= pxx - pyy;
    v[i].y -= pss - pxx - pyy;
    vs[i] = v[i].x + v[i].y;
  }
#pragma unroll
  for (int i = 0; i < W; ++i)
    if (i < w) M[(int64_t)(k0 + i) * d + c] = v[i];
}

// FP64 trailing update of the block LU: A[r0:n, c0:c1) -= A[r0:n, k0:k0+w)
// A[k0:k0+w, c0:c1), r0 = k0 + W, over all blocks.  TR x TN output tiles,
// 64 threads with TR/8 x TN/8 outputs each (3M products, tile3m_update); CTAs
// stride over the tiles when the grid is smaller than the tile count.  The
// FP64 pipe (two DFMA per clock per SM) bounds every tile shape, so small
// tiles cost nothing and mask less of the late, narrow updates.
template <int W, int TN, int TR>
__global__ void __launch_bounds__(64) lu_update_kernel(double2* __restrict__ A, int64_t d,
                                                       const int32_t* __restrict__ sz, int k0,
                                                       int64_t c0, int64_t c1_cap, int nb) {
  const int64_t r0 = k0 + W;
  const int64_t cend = c1_cap < 0 ? d : c1_cap;
  const int64_t rt_n = (d - r0 + TR - 1) / TR, ct_n = (cend - c0 + TN - 1) / TN;
  const int64_t per_b = rt_n * ct_n, tiles = (int64_t)nb * per_b;
  __shared__ Tile3M<W, TN, TR> T;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int b = (int)(tile / per_b);
    const int64_t rem = tile - (int64_t)b * per_b;
    const int n = sz[b];
    const int64_t c1 = mn64(cend, n);
    const int64_t tr = r0 + (rem / ct_n) * TR, tc = c0 + (rem % ct_n) * TN;
    if (k0 >= n || tr >= n || tc >= c1) continue;  // uniform over the CTA
    const int w = min(W, n - k0);
    double2* M = A + (int64_t)b * d * d;
    tile3m_load<W, TN, 64, TR>(T, M, d, tr, tc, k0, n, c1, w, threadIdx.x);
    __syncthreads();
    tile3m_update<W, TN, TN / 8, TR>(T, M, d, tr, tc, n, c1, threadIdx.x);
    __syncthreads();  // before the next tile's loads overwrite the staging
  }
}

// X <- P I: row k of the identity permuted by the recorded swaps
template <class CT>
__global__ void perm_identity_kernel(CT* __restrict__ X, int64_t d,
                                     const int32_t* __restrict__ sz,
                                     const int32_t* __restrict__ piv) {
  const int b = blockIdx.y;
  const int n = sz[b];
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  CT* M = X + (int64_t)b * d * d;
  // column c of P: start from e_c and apply the swaps in order
  int64_t pos = c;
  for (int k = 0; k < n; ++k) {
    const int p = piv[(int64_t)b * d + k];
    if (pos == k)
      pos = p;
    else if (pos == p)
      pos = k;
  }
  for (int64_t i = 0; i < n; ++i) M[i * d + c] = CT{i == pos ? 1.0f : 0.0f, 0.0f};
}

// gather the MBJ blocks of the operator: block b rows/cols I_b in both halves
template <int DT>
__global__ void gather_blocks_kernel(const void* __restrict__ Zv, int64_t ldz, int64_t H,
                                     int64_t B, int64_t d, const int32_t* __restrict__ sz,
                                     double2* __restrict__ out) {
  const int b = blockIdx.z;
  const int s = sz[b] / 2;
  const int64_t i = blockIdx.y, j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 2 * s || j >= 2 * s) return;
  const int64_t o = (int64_t)b * B;
  const int64_t gi = i < s ? o + i : H + o + (i - s);
  const int64_t gj = j < s ? o + j : H + o + (j - s);
  double2 v;
  if (DT == MUELLER_C128) {
    v = reinterpret_cast<const double2*>(Zv)[gi * ldz + gj];
  } else {
    const float2 f = reinterpret_cast<const float2*>(Zv)[gi * ldz + gj];
    v = make_double2(f.x, f.y);
  }
  out[(int64_t)b * d * d + i * d + j] = v;
}

// add the near blocks that fall inside MBJ block b (C64_NEAR64 operator)
__global__ void __launch_bounds__(256) gather_near_kernel(int64_t nn, const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const double2* __restrict__ nearb, int64_t B,
                                                          int64_t d, const int32_t* __restrict__ sz,
                                                          double2* __restrict__ out) {
  // one warp per test node; lanes over its near blocks' 16 entries.  Every
  // (node pair, h, alpha, g, beta) is one entry of one block, so no two lanes
  // write the same place.
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;  // test node
  const int lane = threadIdx.x & 31;
  if (i >= nn) return;
  const int32_t q0 = rowptr[i], q1 = rowptr[i + 1];
  for (int64_t e = (int64_t)q0 * 16 + lane; e < (int64_t)q1 * 16; e += 32) {
    const int64_t q = e >> 4;
    const int ha = (int)(e >> 2) & 3, gb = (int)e & 3;
    const int64_t j = col[q];
    const int h = ha >> 1, a = ha & 1, g = gb >> 1, be = gb & 1;
    const int64_t ri = 2 * i + a, cj = 2 * j + be;  // per-current indices
    const int64_t bi = ri / B, bj = cj / B;
    if (bi != bj) continue;
    const int s = sz[bi] / 2;
    const int64_t li = (ri - bi * B) + (h ? s : 0), lj = (cj - bj * B) + (g ? s : 0);
    const double2 v = nearb[e];
    double2* t = out + bi * d * d + li * d + lj;
    t->x += v.x;
    t->y += v.y;
  }
}

// ============================================================ MBJ apply
// z = P^{-1} v: block b multiplies its explicit inverse with the gathered
// piece of v; one warp per row, lanes over columns.  Blocks of d x d.
template <class BT, class VT>
__global__ void __launch_bounds__(256) mbj_apply_kernel(const BT* __restrict__ inv, int64_t d,
                                                        const int32_t* __restrict__ sz, int64_t B,
                                                        int64_t H, const VT* __restrict__ v,
                                                        VT* __restrict__ z) {
  const int b = blockIdx.y;
  const int n = sz[b], s = n / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  if (i >= n) return;
  using R = decltype(v[0].x);
  const int64_t o = (int64_t)b * B;
  const BT* row = inv + (int64_t)b * d * d + i * d;
  R ar = 0, ai = 0;
  for (int j = lane; j < n; j += 32) {
    const int64_t gj = j < s ? o + j : H + o + (j - s);
    const VT x = v[gj];
    const BT m = row[j];
    ar = fma((R)m.x, x.x, fma(-(R)m.y, x.y, ar));
    ai = fma((R)m.x, x.y, fma((R)m.y, x.x, ai));
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o2);
    ai += __shfl_xor_sync(0xffffffffu, ai, o2);
  }
  if (lane == 0) {
    const int64_t gi = i < s ? o + i : H + o + (i - s);
    z[gi].x = ar;
    z[gi].y = ai;
  }
}

// z = (P^{-1})^H v (complex128): block b's explicit inverse conjugate-
// transposed, one thread per output entry (column i of the inverse; the
// threads of a warp read consecutive entries of each row).
__global__ void __launch_bounds__(128) mbj_apply_h_kernel(const double2* __restrict__ inv,
                                                          int64_t d, const int32_t* __restrict__ sz,
                                                          int64_t B, int64_t H,
                                                          const double2* __restrict__ v,
                                                          double2* __restrict__ z) {
  const int b = blockIdx.y;
  const int n = sz[b], half = n / 2;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t o = (int64_t)b * B;
  const double2* M = inv + (int64_t)b * d * d;
  double ar = 0.0, ai = 0.0;
  for (int j = 0; j < n; ++j) {
    const double2 m = M[(int64_t)j * d + i];
    const int64_t gj = j < half ? o + j : H + o + (j - half);
    const double2 x = v[gj];
    ar = fma(m.x, x.x, fma(m.y, x.y, ar));
    ai = fma(m.x, x.y, fma(-m.y, x.x, ai));
  }
  const int64_t gi = i < half ? o + i : H + o + (i - half);
  z[gi] = make_double2(ar, ai);
}

__global__ void c128_to_c64_kernel(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) b[t] = make_float2((float)a[t].x, (float)a[t].y);
}

// ============================================================ GMRES pieces
// partial sums of conj(V_l) . w over G chunks: part[l*G + g]
template <class VT>
__global__ void __launch_bounds__(256) dots_kernel(const VT* __restrict__ V, int64_t N, int nl,
                                                   const VT* __restrict__ w,
                                                   double2* __restrict__ part, int G) {
  const int l = blockIdx.y, g = blockIdx.x;
  if (l >= nl) return;
  const VT* v = V + (int64_t)l * N;
  double sr = 0, si = 0;
  for (int64_t i = (int64_t)g * blockDim.x + threadIdx.x; i < N; i += (int64_t)G * blockDim.x) {
    const VT a = v[i], b = w[i];
    sr += (double)a.x * b.x + (double)a.y * b.y;
    si += (double)a.x * b.y - (double)a.y * b.x;
  }
  __shared__ double rr[256], ri[256];
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rr[threadIdx.x] += rr[threadIdx.x + o];
      ri[threadIdx.x] += ri[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)l * G + g] = make_double2(rr[0], ri[0]);
}

// h[l] = sum_g part[l*G+g]; hacc[l] += h[l]; w -= sum_l h[l] V_l
template <class VT>
__global__ void __launch_bounds__(256) orth_update_kernel(const VT* __restrict__ V, int64_t N,
                                                          int nl, const double2* __restrict__ part,
                                                          int G, VT* __restrict__ w,
                                                          double2* __restrict__ hacc) {
  __shared__ double2 h[128];
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    double2 s = make_double2(0, 0);
    for (int g = 0; g < G; ++g) {
      s.x += part[(int64_t)l * G + g].x;
      s.y += part[(int64_t)l * G + g].y;
    }
    h[l] = s;
    if (blockIdx.x == 0) {
      hacc[l].x += s.x;
      hacc[l].y += s.y;
    }
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  using R = decltype(w[0].x);
  double ar = w[i].x, ai = w[i].y;
  for (int l = 0; l < nl; ++l) {
    const VT v = V[(int64_t)l * N + i];
    ar -= h[l].x * v.x - h[l].y * v.y;
    ai -= h[l].x * v.y + h[l].y * v.x;
  }
  w[i].x = (R)ar;
  w[i].y = (R)ai;
}

// sum of squares partials
template <class VT>
__global__ void __launch_bounds__(256) nrm2_kernel(const VT* __restrict__ w, int64_t N,
                                                   double* __restrict__ part, int G) {
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)G * blockDim.x)
    s += (double)w[i].x * w[i].x + (double)w[i].y * w[i].y;
  __shared__ double r[256];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) r[threadIdx.x] += r[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = r[0];
}

// v_out = w / ||w|| (norm from the partials); stores ||w|| to *nrm
template <class VT>
__global__ void normalize_kernel(const VT* __restrict__ w, int64_t N, const double* __restrict__ part,
                                 int G, VT* __restrict__ out, double* __restrict__ nrm) {
  double s = 0;
  for (int g = 0; g < G; ++g) s += part[g];
  const double n = sqrt(s);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) *nrm = n;
  if (i >= N) return;
  using R = decltype(w[0].x);
  const double inv = n > 0 ? 1.0 / n : 0.0;
  out[i].x = (R)(w[i].x * inv);
  out[i].y = (R)(w[i].y * inv);
}

// Givens step of Arnoldi column j (single thread).  Hcol = accumulated
// Gram-Schmidt coefficients (j+1 of them), hn = ||w||.  H is (m+1) x m
// column-major complex; cs real, sn complex; g complex; res = |g[j+1]|.
__global__ void givens_kernel(int j, int m, double2* __restrict__ hacc, const double* __restrict__ hn,
                              double2* __restrict__ Hm, double* __restrict__ cs,
                              double2* __restrict__ sn, double2* __restrict__ g,
                              double* __restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double2* col = Hm + (int64_t)j * (m + 1);
  // earlier rotations [c s; -conj(s) c] down the new column, the entry
  // rotated into position l + 1 carried in a register
  double2 a = hacc[0];
  for (int l = 0; l < j; ++l) {
    const double2 b = hacc[l + 1];
    const double c = cs[l];
    const double2 s = sn[l];
    col[l] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
    a = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
  }
  const double2 b = make_double2(*hn, 0.0);
  const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
  const double rho = hypot(aa, bb);
  double c;
  double2 s;
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
  } else {
    c = aa / rho;
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    // s = (a/|a|) conj(b) / rho
    s = make_double2((ph.x * b.x + ph.y * b.y) / rho, (ph.y * b.x - ph.x * b.y) / rho);
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
  col[j + 1] = make_double2(0, 0);
  const double2 gj = g[j];
  g[j] = make_double2(c * gj.x, c * gj.y);
  g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
  *res = hypot(g[j + 1].x, g[j + 1].y);
  for (int l = 0; l <= j + 1; ++l) hacc[l] = make_double2(0, 0);
}

// y = H(0:k,0:k)^{-1} g (back substitution, single thread)
__global__ void backsub_kernel(int k, int m, const double2* __restrict__ Hm,
                               const double2* __restrict__ g, double2* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double2 s = g[i];
    for (int l = i + 1; l < k; ++l) {
      const double2 h = Hm[(int64_t)l * (m + 1) + i];
      s.x -= h.x * y[l].x - h.y * y[l].y;
      s.y -= h.x * y[l].y + h.y * y[l].x;
    }
    y[i] = cdiv2(s, Hm[(int64_t)i * (m + 1) + i]);
  }
}

// u = sum_l y_l V_l
template <class VT>
__global__ void combine_kernel(const VT* __restrict__ V, int64_t N, int k,
                               const double2* __restrict__ y, VT* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double ar = 0, ai = 0;
  for (int l = 0; l < k; ++l) {
    const VT v = V[(int64_t)l * N + i];
    ar += y[l].x * v.x - y[l].y * v.y;
    ai += y[l].x * v.y + y[l].y * v.x;
  }
  using R = decltype(u[0].x);
  u[i].x = (R)ar;
  u[i].y = (R)ai;
}

// x += alpha * u  (x in XT, u in UT)
template <class XT, class UT>
__global__ void axpy_kernel(XT* __restrict__ x, const UT* __restrict__ u, int64_t N, double alpha) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  using R = decltype(x[0].x);
  x[i].x = (R)(x[i].x + alpha * u[i].x);
  x[i].y = (R)(x[i].y + alpha * u[i].y);
}

// r = b - y (complex128); also r_lo = r * scale in complex64 if r_lo
__global__ void residual_kernel(const double2* __restrict__ b, const double2* __restrict__ y,
                                double2* __restrict__ r, int64_t N) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  r[i] = make_double2(b[i].x - y[i].x, b[i].y - y[i].y);
}

template <class VT>
__global__ void set_first_kernel(double2* __restrict__ g, int m, const double* __restrict__ beta) {
  if (threadIdx.x != 0) return;
  for (int l = 0; l <= m; ++l) g[l] = make_double2(0, 0);
  g[0] = make_double2(*beta, 0.0);
}

template <class AT, class BT2>
__global__ void scale_copy_kernel(const AT* __restrict__ a, BT2* __restrict__ b, int64_t N,
                                  const double* __restrict__ nrm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double inv = (*nrm > 0) ? 1.0 / *nrm : 0.0;
  using R = decltype(b[0].x);
  b[i].x = (R)(a[i].x * inv);
  b[i].y = (R)(a[i].y * inv);
}

// ===================================================== lockstep multi-RHS GMRES
// r right-hand sides advance together; vectors are stored RHS-major
// ([s][N]) and the Krylov basis as V[j][s][N].  blockIdx.y (or .z) is s.

// partial dots conj(V_l[s]) . w[s] over G chunks: part[(s*(m1) + l)*G + g]
__global__ void __launch_bounds__(256) dots_b_kernel(const float2* __restrict__ V, int64_t N, int r,
                                                     int nl, int m1, const float2* __restrict__ w,
                                                     double2* __restrict__ part, int G) {
  const int g = blockIdx.x, l = blockIdx.y, s = blockIdx.z;
  const float2* v = V + ((int64_t)l * r + s) * N;
  const float2* ww = w + (int64_t)s * N;
  double sr = 0, si = 0;
  for (int64_t i = (int64_t)g * blockDim.x + threadIdx.x; i < N; i += (int64_t)G * blockDim.x) {
    const float2 a = v[i], b = ww[i];
    sr += (double)a.x * b.x + (double)a.y * b.y;
    si += (double)a.x * b.y - (double)a.y * b.x;
  }
  __shared__ double rr[256], ri[256];
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rr[threadIdx.x] += rr[threadIdx.x + o];
      ri[threadIdx.x] += ri[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[((int64_t)s * m1 + l) * G + g] = make_double2(rr[0], ri[0]);
}

// w[s] -= sum_l h[s][l] V_l[s], h from the partials; hacc[s][l] += h
__global__ void __launch_bounds__(256) orth_b_kernel(const float2* __restrict__ V, int64_t N, int r,
                                                     int nl, int m1, const double2* __restrict__ part,
                                                     int G, float2* __restrict__ w,
                                                     double2* __restrict__ hacc) {
  const int s = blockIdx.y;
  __shared__ double2 h[128];
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    double2 a = make_double2(0, 0);
    for (int g = 0; g < G; ++g) {
      const double2 q = part[((int64_t)s * m1 + l) * G + g];
      a.x += q.x;
      a.y += q.y;
    }
    h[l] = a;
    if (blockIdx.x == 0) {
      hacc[(int64_t)s * (m1 + 1) + l].x += a.x;
      hacc[(int64_t)s * (m1 + 1) + l].y += a.y;
    }
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float2* wp = w + (int64_t)s * N + i;
  double ar = wp->x, ai = wp->y;
  for (int l = 0; l < nl; ++l) {
    const float2 v = V[((int64_t)l * r + s) * N + i];
    ar -= h[l].x * v.x - h[l].y * v.y;
    ai -= h[l].x * v.y + h[l].y * v.x;
  }
  *wp = make_float2((float)ar, (float)ai);
}

template <class VT>
__global__ void __launch_bounds__(256) nrm2_b_kernel(const VT* __restrict__ w, int64_t N,
                                                     double* __restrict__ part, int G) {
  const int s = blockIdx.y;
  const VT* ws = w + (int64_t)s * N;
  double a = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)G * blockDim.x)
    a += (double)ws[i].x * ws[i].x + (double)ws[i].y * ws[i].y;
  __shared__ double red[256];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)s * G + blockIdx.x] = red[0];
}

// nrm[s] = sqrt(sum of partials) * mask[s]  (mask 0 freezes a right-hand side)
__global__ void norm_finish_b_kernel(const double* __restrict__ part, int G, int r,
                                     const int* __restrict__ mask, double* __restrict__ nrm) {
  const int s = threadIdx.x + blockIdx.x * blockDim.x;
  if (s >= r) return;
  double a = 0;
  for (int g = 0; g < G; ++g) a += part[(int64_t)s * G + g];
  nrm[s] = (mask && !mask[s]) ? 0.0 : sqrt(a);
}

// out[s] = w[s] / nrm[s]  (0 if nrm[s] == 0)
template <class IT, class OT>
__global__ void scale_b_kernel(const IT* __restrict__ w, int64_t N, const double* __restrict__ nrm,
                               OT* __restrict__ out) {
  const int s = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double n = nrm[s];
  const double inv = n > 0 ? 1.0 / n : 0.0;
  const IT a = w[(int64_t)s * N + i];
  out[(int64_t)s * N + i].x = (decltype(out[0].x))(a.x * inv);
  out[(int64_t)s * N + i].y = (decltype(out[0].x))(a.y * inv);
}

// Givens step of Arnoldi column j of right-hand side s: the earlier
// rotations applied to the accumulated Gram-Schmidt coefficients hacc[s],
// a new rotation against ||w|| = hn, the rotated column stored in Hm and
// the residual estimate |g[j+1]| in res[s]; hacc[s] is cleared.
__device__ void givens_column(int j, int m, int s, double2* __restrict__ hacc, double hn_s,
                              double2* __restrict__ Hm, double* __restrict__ cs,
                              double2* __restrict__ sn, double2* __restrict__ g,
                              double* __restrict__ res) {
  double2* ha = hacc + (int64_t)s * (m + 2);
  double2* col = Hm + ((int64_t)s * m + j) * (m + 1);
  double* c_ = cs + (int64_t)s * (m + 1);
  double2* s_ = sn + (int64_t)s * (m + 1);
  double2* gg = g + (int64_t)s * (m + 1);
  // the earlier rotations, applied down the new column; the entry being
  // rotated into position l + 1 is carried in a register (a), so only the
  // loads of ha, c_ and s_ (independent of the chain) touch memory
  double2 a = ha[0];
  for (int l = 0; l < j; ++l) {
    const double2 b = ha[l + 1];
    const double c = c_[l];
    const double2 sv = s_[l];
    col[l] = make_double2(c * a.x + sv.x * b.x - sv.y * b.y, c * a.y + sv.x * b.y + sv.y * b.x);
    a = make_double2(-(sv.x * a.x + sv.y * a.y) + c * b.x, -(sv.x * a.y - sv.y * a.x) + c * b.y);
  }
  const double2 b = make_double2(hn_s, 0.0);
  const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
  const double rho = hypot(aa, bb);
  double c;
  double2 sv;
  if (aa == 0.0) {
    c = 0.0;
    sv = make_double2(1.0, 0.0);
  } else {
    c = aa / rho;
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    sv = make_double2((ph.x * b.x + ph.y * b.y) / rho, (ph.y * b.x - ph.x * b.y) / rho);
  }
  c_[j] = c;
  s_[j] = sv;
  col[j] = make_double2(c * a.x + sv.x * b.x - sv.y * b.y, c * a.y + sv.x * b.y + sv.y * b.x);
  col[j + 1] = make_double2(0, 0);
  const double2 gj = gg[j];
  gg[j] = make_double2(c * gj.x, c * gj.y);
  gg[j + 1] = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));
  res[s] = hypot(gg[j + 1].x, gg[j + 1].y);
  for (int l = 0; l <= j + 1; ++l) ha[l] = make_double2(0, 0);
}

// Givens step of column j for every right-hand side (thread s)
__global__ void givens_b_kernel(int j, int m, int r, double2* __restrict__ hacc,
                                const double* __restrict__ hn, double2* __restrict__ Hm,
                                double* __restrict__ cs, double2* __restrict__ sn,
                                double2* __restrict__ g, double* __restrict__ res) {
  const int s = threadIdx.x + blockIdx.x * blockDim.x;
  if (s >= r) return;
  givens_column(j, m, s, hacc, hn[s], Hm, cs, sn, g, res);
}

// ------------------------------------------------ fused Arnoldi step tail
// One Arnoldi step after the product w = A P^-1 v_j, for all r right-hand
// sides in one launch: a cluster of CS CTAs per right-hand side, each CTA
// owning a contiguous chunk of the vector.  Classical Gram-Schmidt twice
// against v_0..v_j (per pass: the chunk's partial dot products in shared
// memory, a cluster barrier, every CTA of the cluster sums the CS partials of
// every coefficient in the same order through distributed shared memory, then
// updates its chunk), the norm the same way, v_{j+1} = w / ||w||, the Givens
// step and the convergence test of the right-hand side by the cluster's
// first CTA.  The clusters never wait on one another: the last one to finish
// (a ticket counter) decides whether every active right-hand side has
// converged and sets the stop flag, after which every queued step returns at
// once, so the host reads the flag only now and then.
constexpr int kTailMaxM = 128;  // restart length limit of the lockstep solver

struct TailArgs {
  const float2* V;  // Krylov basis V[(l r + s) N + i], l <= j read, l = j + 1 written
  float2* w;        // A z_j for the r right-hand sides (orthogonalised in place)
  int64_t N;
  int r, j, m, cs;  // cs: CTAs per right-hand side (the cluster size)
  double2* hacc;    // [r][m + 2] coefficients summed over both passes
  double2* Hm;
  double* cs_;
  double2* sn;
  double2* g;
  double* res;      // [r] Arnoldi residual estimates
  int* kk;          // [r] converged step count (0: not yet)
  const int* active;
  int* bad;         // [r] set when a residual estimate is not a number
  double tol;
  int* stop;        // set when every active right-hand side has converged
  int* jstop;       // steps taken when stop was set
  unsigned* ticket; // clusters finished in this step (reset by the last one)
};

__global__ void __launch_bounds__(256) arnoldi_tail_kernel(TailArgs a) {
  if (*a.stop) return;  // written only between launches: uniform over the grid
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double2 part[2][kTailMaxM + 1];  // this CTA's partial dots, per pass
  __shared__ double2 hsh[kTailMaxM + 1];      // the summed coefficients of the pass
  __shared__ double npart, hn;
  const int q = (int)cl.block_rank(), CS = a.cs;
  const int s = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = a.j + 1;
  // chunks of whole float4 pairs (N is a multiple of 4, so every chunk
  // boundary and every pair is 16-byte aligned)
  const int64_t np2 = a.N / 2, ch = (np2 + CS - 1) / CS;
  const int64_t p0 = (int64_t)q * ch, p1 = min(np2, p0 + ch);
  float4* ww = reinterpret_cast<float4*>(a.w + (int64_t)s * a.N);
  const int64_t vstride = (int64_t)a.r * a.N / 2;  // in float4
  const float4* V0 = reinterpret_cast<const float4*>(a.V + (int64_t)s * a.N);
  for (int pass = 0; pass < 2; ++pass) {
    // partial dots conj(v_l) . w over the chunk: a warp per basis vector,
    // two entries per load, four independent accumulators per lane
    for (int l = warp; l < nl; l += 8) {
      const float4* v = V0 + l * vstride;
      float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
      int64_t i = p0 + lane;
      for (; i + 96 < p1; i += 128) {
        float4 x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          x[u] = v[i + 32 * u];
          y[u] = ww[i + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ar[u] = fmaf(x[u].x, y[u].x, fmaf(x[u].y, y[u].y, ar[u]));
          ai[u] = fmaf(x[u].x, y[u].y, fmaf(-x[u].y, y[u].x, ai[u]));
          ar[u] = fmaf(x[u].z, y[u].z, fmaf(x[u].w, y[u].w, ar[u]));
          ai[u] = fmaf(x[u].z, y[u].w, fmaf(-x[u].w, y[u].z, ai[u]));
        }
      }
      for (; i < p1; i += 32) {
        const float4 x = v[i], y = ww[i];
        ar[0] = fmaf(x.x, y.x, fmaf(x.y, y.y, ar[0]));
        ai[0] = fmaf(x.x, y.y, fmaf(-x.y, y.x, ai[0]));
        ar[1] = fmaf(x.z, y.z, fmaf(x.w, y.w, ar[1]));
        ai[1] = fmaf(x.z, y.w, fmaf(-x.w, y.z, ai[1]));
      }
      double dr = (double)(ar[0] + ar[1]) + (double)(ar[2] + ar[3]);
      double di = (double)(ai[0] + ai[1]) + (double)(ai[2] + ai[3]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dr += __shfl_xor_sync(0xffffffffu, dr, o);
        di += __shfl_xor_sync(0xffffffffu, di, o);
      }
      if (lane == 0) part[pass][l] = make_double2(dr, di);
    }
    cl.sync();
    // every CTA sums the partials of the cluster in rank order
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      double dr = 0.0, di = 0.0;
      for (int k = 0; k < CS; ++k) {
        const double2 t = cl.map_shared_rank(&part[pass][0], k)[l];
        dr += t.x;
        di += t.y;
      }
      hsh[l] = make_double2(dr, di);
      if (q == 0) {
        double2* acc = a.hacc + (int64_t)s * (a.m + 2) + l;
        acc->x += dr;
        acc->y += di;
      }
    }
    __syncthreads();
    // w -= sum_l h_l v_l on the chunk, eight basis vectors' loads in flight
    for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
      float4 acc = ww[i];
      int l = 0;
      for (; l + 8 <= nl; l += 8) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = V0[(l + u) * vstride + i];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const double2 hd = hsh[l + u];
          const float hr = (float)hd.x, hi = (float)hd.y;
          acc.x = fmaf(-hr, v[u].x, fmaf(hi, v[u].y, acc.x));
          acc.y = fmaf(-hr, v[u].y, fmaf(-hi, v[u].x, acc.y));
          acc.z = fmaf(-hr, v[u].z, fmaf(hi, v[u].w, acc.z));
          acc.w = fmaf(-hr, v[u].w, fmaf(-hi, v[u].z, acc.w));
        }
      }
      for (; l < nl; ++l) {
        const float4 v = V0[l * vstride + i];
        const double2 hd = hsh[l];
        const float hr = (float)hd.x, hi = (float)hd.y;
        acc.x = fmaf(-hr, v.x, fmaf(hi, v.y, acc.x));
        acc.y = fmaf(-hr, v.y, fmaf(-hi, v.x, acc.y));
        acc.z = fmaf(-hr, v.z, fmaf(hi, v.w, acc.z));
        acc.w = fmaf(-hr, v.w, fmaf(-hi, v.z, acc.w));
      }
      ww[i] = acc;
    }
    __syncthreads();  // hsh is rewritten by the next pass; the chunk is this CTA's own
  }
  // squared norm of the chunk
  {
    double qn = 0.0;
    for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
      const float4 x = ww[i];
      qn += (double)x.x * x.x + (double)x.y * x.y + (double)x.z * x.z + (double)x.w * x.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qn += __shfl_xor_sync(0xffffffffu, qn, o);
    double* wsum = reinterpret_cast<double*>(&hsh[0]);
    if (lane == 0) wsum[warp] = qn;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < 8; ++k) t += wsum[k];
      npart = t;
    }
  }
  cl.sync();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < CS; ++k) t += *cl.map_shared_rank(&npart, k);
    hn = sqrt(t);
  }
  // no CTA may leave while another still reads its shared memory
  cl.sync();
  {
    const double inv = hn > 0 ? 1.0 / hn : 0.0;
    float4* vn = const_cast<float4*>(V0) + (int64_t)(a.j + 1) * vstride;
    for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
      const float4 x = ww[i];
      vn[i] = make_float4((float)(x.x * inv), (float)(x.y * inv), (float)(x.z * inv),
                          (float)(x.w * inv));
    }
  }
  if (q != 0 || threadIdx.x != 0) return;
  givens_column(a.j, a.m, s, a.hacc, hn, a.Hm, a.cs_, a.sn, a.g, a.res);
  if (a.active[s] && a.kk[s] == 0) {
    const double v = a.res[s];
    if (!(v == v)) {
      a.bad[s] = 1;
      a.kk[s] = a.j + 1;
    } else if (v <= a.tol) {
      a.kk[s] = a.j + 1;
    }
  }
  __threadfence();
  if (atomicAdd(a.ticket, 1u) != (unsigned)a.r - 1) return;
  // the last cluster of the step: every right-hand side's kk is visible
  __threadfence();
  bool all = true;
  for (int k = 0; k < a.r; ++k) {
    if (!a.active[k]) continue;
    if (((volatile int*)a.kk)[k] == 0) all = false;
  }
  if (all) {
    *a.jstop = a.j + 1;
    *a.stop = 1;
  }
  *a.ticket = 0u;
}

// g[s] = beta[s] e1
__global__ void set_first_b_kernel(double2* __restrict__ g, int m, int r,
                                   const double* __restrict__ beta) {
  const int s = threadIdx.x + blockIdx.x * blockDim.x;
  if (s >= r) return;
  for (int l = 0; l <= m; ++l) g[(int64_t)s * (m + 1) + l] = make_double2(0, 0);
  g[(int64_t)s * (m + 1)] = make_double2(beta[s], 0.0);
}

// y[s] = H_s(0:k,0:k)^{-1} g[s] with k = kk[s] (0: no update)
__global__ void backsub_b_kernel(int m, int r, const int* __restrict__ kk,
                                 const double2* __restrict__ Hm, const double2* __restrict__ g,
                                 double2* __restrict__ y) {
  const int s = threadIdx.x + blockIdx.x * blockDim.x;
  if (s >= r) return;
  const int k = kk[s];
  double2* ys = y + (int64_t)s * (m + 1);
  for (int l = 0; l <= m; ++l) ys[l] = make_double2(0, 0);
  const double2* H = Hm + (int64_t)s * m * (m + 1);
  for (int i = k - 1; i >= 0; --i) {
    double2 a = g[(int64_t)s * (m + 1) + i];
    for (int l = i + 1; l < k; ++l) {
      const double2 h = H[(int64_t)l * (m + 1) + i];
      a.x -= h.x * ys[l].x - h.y * ys[l].y;
      a.y -= h.x * ys[l].y + h.y * ys[l].x;
    }
    ys[i] = cdiv2(a, H[(int64_t)i * (m + 1) + i]);
  }
}

// u[s] = sum_{l < kmax} y[s][l] V_l[s]
__global__ void combine_b_kernel(const float2* __restrict__ V, int64_t N, int r, int kmax, int m,
                                 const double2* __restrict__ y, float2* __restrict__ u) {
  const int s = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double ar = 0, ai = 0;
  for (int l = 0; l < kmax; ++l) {
    const double2 c = y[(int64_t)s * (m + 1) + l];
    const float2 v = V[((int64_t)l * r + s) * N + i];
    ar += c.x * v.x - c.y * v.y;
    ai += c.x * v.y + c.y * v.x;
  }
  u[(int64_t)s * N + i] = make_float2((float)ar, (float)ai);
}

// w[s] = b[s] - w[s]  (complex64)
__global__ void resid_b_kernel(const float2* __restrict__ b, float2* __restrict__ w, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  w[i] = make_float2(b[i].x - w[i].x, b[i].y - w[i].y);
}

// x[s] += alpha[s] u[s]  (x complex128 or complex64, u complex64)
template <class XT>
__global__ void axpy_b_kernel(XT* __restrict__ x, const float2* __restrict__ u, int64_t N,
                              const double* __restrict__ alpha) {
  const int s = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double a = alpha ? alpha[s] : 1.0;
  XT* xp = x + (int64_t)s * N + i;
  const float2 v = u[(int64_t)s * N + i];
  xp->x = (decltype(x[0].x))(xp->x + a * v.x);
  xp->y = (decltype(x[0].x))(xp->y + a * v.y);
}

// z = P^{-1} v for r vectors (complex64 inverses)
__global__ void __launch_bounds__(256) mbj_apply_b_kernel(const float2* __restrict__ inv, int64_t d,
                                                          const int32_t* __restrict__ sz, int64_t B,
                                                          int64_t H, int64_t N,
                                                          const float2* __restrict__ v,
                                                          float2* __restrict__ z,
                                                          const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int b = blockIdx.y, s = blockIdx.z;
  const int n = sz[b], half = n / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  if (i >= n) return;
  const int64_t o = (int64_t)b * B;
  const float2* row = inv + (int64_t)b * d * d + i * d;
  const float2* vs = v + (int64_t)s * N;
  float ar = 0, ai = 0;
  for (int j0 = lane; j0 < n; j0 += 128) {
    float2 mm[4], xx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // four independent loads in flight per lane
      const int j = j0 + 32 * u;
      if (j < n) {
        const int64_t gj = j < half ? o + j : H + o + (j - half);
        mm[u] = row[j];
        xx[u] = vs[gj];
      } else {
        mm[u] = make_float2(0.f, 0.f);
        xx[u] = make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ar = fmaf(mm[u].x, xx[u].x, fmaf(-mm[u].y, xx[u].y, ar));
      ai = fmaf(mm[u].x, xx[u].y, fmaf(mm[u].y, xx[u].x, ai));
    }
  }
#pragma unroll
  for (int q = 16; q > 0; q >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, q);
    ai += __shfl_xor_sync(0xffffffffu, ai, q);
  }
  if (lane == 0) {
    const int64_t gi = i < half ? o + i : H + o + (i - half);
    z[(int64_t)s * N + gi] = make_float2(ar, ai);
  }
}

// The same for RS right-hand sides at once (s0 = blockIdx.z * RS): the CTA
// stages the block's piece of the RS vectors in shared memory (RS x n
// complex64, dynamic), then each warp multiplies rows of the inverse with
// all RS of them, so every inverse entry is read once for RS vectors.  Rows
// kMbjRows per CTA (blockIdx.x).
constexpr int kMbjRows = 64;
template <int RS>
__global__ void __launch_bounds__(256) mbj_apply_rs_kernel(const float2* __restrict__ inv, int64_t d,
                                                           const int32_t* __restrict__ sz, int64_t B,
                                                           int64_t H, int64_t N, int r,
                                                           const float2* __restrict__ v,
                                                           float2* __restrict__ z,
                                                           const int* __restrict__ stop) {
  if (stop && *stop) return;
  extern __shared__ float2 sv[];  // [RS][n]
  const int b = blockIdx.y, s0 = blockIdx.z * RS;
  const int n = sz[b], half = n / 2;
  const int i0 = blockIdx.x * kMbjRows;
  if (i0 >= n) return;  // uniform for the CTA
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t o = (int64_t)b * B;
  for (int t = threadIdx.x; t < RS * n; t += blockDim.x) {
    const int k = t / n, j = t % n;
    const int64_t gj = j < half ? o + j : H + o + (j - half);
    sv[t] = s0 + k < r ? v[(int64_t)(s0 + k) * N + gj] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int i1 = min(n, i0 + kMbjRows);
  for (int i = i0 + warp; i < i1; i += 8) {
    const float2* row = inv + (int64_t)b * d * d + (int64_t)i * d;
    float ar[RS], ai[RS];
#pragma unroll
    for (int k = 0; k < RS; ++k) ar[k] = ai[k] = 0.f;
    for (int j = lane; j < n; j += 32) {
      const float2 m = row[j];
#pragma unroll
      for (int k = 0; k < RS; ++k) {
        const float2 x = sv[k * n + j];
        ar[k] = fmaf(m.x, x.x, fmaf(-m.y, x.y, ar[k]));
        ai[k] = fmaf(m.x, x.y, fmaf(m.y, x.x, ai[k]));
      }
    }
#pragma unroll
    for (int k = 0; k < RS; ++k)
#pragma unroll
      for (int q = 16; q > 0; q >>= 1) {
        ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], q);
        ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], q);
      }
    const int64_t gi = i < half ? o + i : H + o + (i - half);
#pragma unroll
    for (int k = 0; k < RS; ++k)
      if (lane == k && s0 + k < r) z[(int64_t)(s0 + k) * N + gi] = make_float2(ar[k], ai[k]);
  }
}

// RHS block transposes: dir 0: T[i][k] = B[k][i]; dir 1: X[k][i] = T[i][k]
__global__ void transpose_rhs_kernel(const double2* __restrict__ a, double2* __restrict__ b,
                                     int64_t N, int r, int dir) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * r) return;
  if (dir == 0) {
    const int64_t k = t / N, i = t % N;
    b[i * r + k] = a[k * N + i];
  } else {
    const int64_t i = t / r, k = t % r;
    b[k * N + i] = a[i * r + k];
  }
}

// apply the LU row swaps to the columns of T (one thread per column)
__global__ void permute_rows_kernel(double2* __restrict__ T, int64_t N, int r,
                                    const int32_t* __restrict__ piv) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= r) return;
  for (int64_t i = 0; i < N; ++i) {
    const int64_t p = piv[i];
    if (p != i) {
      const double2 t = T[i * r + k];
      T[i * r + k] = T[p * r + k];
      T[p * r + k] = t;
    }
  }
}

inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// ======================================================= operator products
// y = Z x of the complex64 dense part for one complex64 vector (FP32
// accumulation), reading three quarters of Z when Z11 = -Z00
// With near32 (complex64 near blocks) and the three-quadrant product, the
// near part is added in the same kernel (*fused set to 1); otherwise the
// caller adds it.
static mueller_status gemv_c64_f32(const mueller_operator* op, const void* x, void* y,
                                   cudaStream_t s, const int* stop = nullptr,
                                   const float2* near32 = nullptr, int* fused = nullptr) {
  if (fused) *fused = 0;
  const int64_t N = 4 * op->mesh->nn, H = N / 2;
  if (op->flags & MUELLER_OP_K1_MIRRORED) {
    { Prof prof_("gemv3_c64_kernel", s); gemv3_c64_kernel<<<(unsigned)nblk(H, 8), 256, 0, s>>>(H, (const float4*)op->Z_dev, op->ldz, (const float4*)x, (float2*)y, stop,
        near32 ? op->mesh->near_rowptr : nullptr, near32 ? op->mesh->near_col : nullptr, near32); }
    if (fused && near32) *fused = 1;
    MU_CHECK_LAUNCH("gemv3_c64_kernel");
  } else {
    { Prof prof_("gemv_c64_kernel<float>", s); gemv_c64_kernel<float><<<dim3(nblk(N, 16), 1), 256, 0, s>>>(N, (const float4*)op->Z_dev, op->ldz, x, y, N, N, 1, stop); }
    MU_CHECK_LAUNCH("gemv_c64_kernel<float>");
  }
  return MUELLER_OK;
}

size_t op_matvec_work(const mueller_operator* op, int r) {
  (void)op;
  (void)r;
  return 0;
}

// Y = Z X in the operator's storage: C128 -> FP64; C64_NEAR64 -> complex64
// storage with FP64 arithmetic (X, Y complex128) plus the FP64 near blocks.
mueller_status op_matvec(const mueller_operator* op, const void* X, void* Y, int r, void* work,
                         size_t work_bytes, cudaStream_t s) {
  (void)work;
  (void)work_bytes;
  const mueller_mesh* m = op->mesh;
  const int64_t N = 4 * m->nn;
  if (op->dtype == MUELLER_C128 && (op->flags & MUELLER_OP_ADJOINT)) {
    MU_CUDA(cudaMemsetAsync(Y, 0, (size_t)N * r * sizeof(double2), s));
    // row blocks: about four CTAs per SM over the column tiles
    const int64_t ct = nblk(N, kGemvhCols);
    const int64_t nrb = std::max<int64_t>(1, std::min<int64_t>(N, (4 * 152 + ct - 1) / ct));
    const int64_t rows = (N + nrb - 1) / nrb;
    dim3 grid((unsigned)ct, (unsigned)nblk(N, (int)rows), r);
    { Prof prof_("gemvh_c128_kernel", s); gemvh_c128_kernel<<<grid, 256, 0, s>>>(N, (const double2*)op->Z_dev, op->ldz, (const double2*)X,
                                           (double2*)Y, N, N, rows); }
    MU_CHECK_LAUNCH("gemvh_c128_kernel");
  } else if (op->dtype == MUELLER_C128) {
    dim3 grid(nblk(N, 32), r);
    { Prof prof_("gemv_c128_kernel", s); gemv_c128_kernel<<<grid, 256, 0, s>>>(N, (const double2*)op->Z_dev, op->ldz, (const double2*)X,
                                          (double2*)Y, N, N, r); }
    MU_CHECK_LAUNCH("gemv_c128_kernel");
  } else {
    // FP64-bound: small blocks (2 warps, 4 rows) spread the rows evenly over the SMs
    if (r >= 2) {
      // several vectors: each Z entry read once for kResidRS of them, 3M products
      double* xs = nullptr;
      MU_CUDA(cudaMallocAsync((void**)&xs, (size_t)r * N * sizeof(double), s));
      { Prof prof_("xsum_kernel", s); xsum_kernel<<<nblk((int64_t)r * N, 256), 256, 0, s>>>((const double2*)X, xs, (int64_t)r * N); }
      dim3 grid(nblk(N, 4), (unsigned)((r + kResidRS - 1) / kResidRS));
      { Prof prof_("gemv_c64_f64_3m_kernel", s); gemv_c64_f64_3m_kernel<kResidRS><<<grid, 64, 0, s>>>(N, (const float4*)op->Z_dev, op->ldz, (const double2*)X, xs, (double2*)Y, r); }
      const cudaError_t le = cudaGetLastError();
      cudaFreeAsync(xs, s);
      if (le != cudaSuccess) return cuda_fail(le, "gemv_c64_f64_3m_kernel");
    } else {
      { Prof prof_("gemv_c64_kernel<double>", s); gemv_c64_kernel<double><<<dim3(nblk(N, 4), 1), 64, 0, s>>>(N, (const float4*)op->Z_dev, op->ldz, X, Y, N, N, r, nullptr); }
      MU_CHECK_LAUNCH("gemv_c64_kernel<double>");
    }
    dim3 g2(nblk(m->nn, 8), r);
    { Prof prof_("near_spmv_kernel<double2, double2>", s); near_spmv_kernel<double2, double2><<<g2, 256, 0, s>>>(m->nn, m->near_rowptr, m->near_col,
                                                          (const double2*)op->near_dev,
                                                          (const double2*)X, (double2*)Y, N, N, r, nullptr); }
    MU_CHECK_LAUNCH("near_spmv_kernel");
  }
  return MUELLER_OK;
}

// The same for several complex64 right-hand sides at once: each near block
// (complex128, read once and rounded to complex64) is applied to RS vectors,
// so the blocks are read ceil(r / RS) times instead of r times.
template <int RS, class BT>
__global__ void __launch_bounds__(256, 2) near_spmv_c64_mrhs_kernel(
    int64_t nn, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const BT* __restrict__ blk, const float2* __restrict__ x, float2* __restrict__ y,
    int64_t xs, int64_t ys, int r, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  const int s0 = blockIdx.y * RS;
  if (i >= nn) return;
  const int64_t H = 2 * nn;
  float ar[RS][4], ai[RS][4];
#pragma unroll
  for (int k = 0; k < RS; ++k)
#pragma unroll
    for (int h = 0; h < 4; ++h) ar[k][h] = ai[k][h] = 0.f;
  for (int32_t q = rowptr[i] + lane; q < rowptr[i + 1]; q += 32) {
    const int64_t j = col[q];
    const BT* b = blk + (int64_t)q * 16;
    float2 m[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const BT v = b[e];
      m[e] = make_float2((float)v.x, (float)v.y);
    }
#pragma unroll
    for (int k = 0; k < RS; ++k) {
      if (s0 + k < r) {
        const float2* xv = x + (int64_t)(s0 + k) * xs;
        float2 xj[4];
#pragma unroll
        for (int gb = 0; gb < 4; ++gb) xj[gb] = xv[(gb >> 1) * H + 2 * j + (gb & 1)];
#pragma unroll
        for (int ha = 0; ha < 4; ++ha)
#pragma unroll
          for (int gb = 0; gb < 4; ++gb) {
            const float2 mm = m[ha * 4 + gb];
            ar[k][ha] = fmaf(mm.x, xj[gb].x, fmaf(-mm.y, xj[gb].y, ar[k][ha]));
            ai[k][ha] = fmaf(mm.x, xj[gb].y, fmaf(mm.y, xj[gb].x, ai[k][ha]));
          }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < RS; ++k)
#pragma unroll
    for (int ha = 0; ha < 4; ++ha)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ar[k][ha] += __shfl_xor_sync(0xffffffffu, ar[k][ha], o);
        ai[k][ha] += __shfl_xor_sync(0xffffffffu, ai[k][ha], o);
      }
  // lane 4k + ha writes output ha of right-hand side s0 + k
  float vr = 0.f, vi = 0.f;
#pragma unroll
  for (int k = 0; k < RS; ++k)
#pragma unroll
    for (int ha = 0; ha < 4; ++ha)
      if (lane == 4 * k + ha) {
        vr = ar[k][ha];
        vi = ai[k][ha];
      }
  const int k = lane >> 2, ha = lane & 3;
  if (k < RS && s0 + k < r) {
    float2* yo = y + (int64_t)(s0 + k) * ys + (ha >> 1) * H + 2 * i + (ha & 1);
    yo->x += vr;
    yo->y += vi;
  }
}

// y += near x for r complex64 vectors, near blocks complex128 (FP32 arithmetic)
mueller_status near_apply_c64(const mueller_mesh* m, const void* near_c128, const void* X, void* Y,
                              int r, cudaStream_t s) {
  const int64_t N = 4 * m->nn;
  if (r >= 2) {
    constexpr int RS = 8;
    dim3 g(nblk(m->nn, 8), (r + RS - 1) / RS);
    { Prof prof_("near_spmv_c64_mrhs_kernel", s); near_spmv_c64_mrhs_kernel<RS, double2><<<g, 256, 0, s>>>(m->nn, m->near_rowptr, m->near_col, (const double2*)near_c128, (const float2*)X, (float2*)Y, N, N, r, nullptr); }
    MU_CHECK_LAUNCH("near_spmv_c64_mrhs_kernel");
    return MUELLER_OK;
  }
  dim3 g(nblk(m->nn, 8), r);
  { Prof prof_("near_spmv_kernel<double2, float2>", s); near_spmv_kernel<double2, float2><<<g, 256, 0, s>>>(m->nn, m->near_rowptr, m->near_col, (const double2*)near_c128, (const float2*)X, (float2*)Y, N, N, r, nullptr); }
  MU_CHECK_LAUNCH("near_spmv_kernel<double2, float2>");
  return MUELLER_OK;
}

// y += near x for r complex64 vectors with complex64 near blocks (the inner
// solver's copy of the FP64 blocks, rounded once per solve)
static mueller_status near_apply_c64_b32(const mueller_mesh* m, const float2* near32,
                                         const float2* X, float2* Y, int r, cudaStream_t s,
                                         const int* stop = nullptr) {
  const int64_t N = 4 * m->nn;
  if (r >= 2) {
    constexpr int RS = 8;
    dim3 g(nblk(m->nn, 8), (r + RS - 1) / RS);
    { Prof prof_("near_spmv_c64_mrhs_kernel", s); near_spmv_c64_mrhs_kernel<RS, float2><<<g, 256, 0, s>>>(m->nn, m->near_rowptr, m->near_col, near32, X, Y, N, N, r, stop); }
    MU_CHECK_LAUNCH("near_spmv_c64_mrhs_kernel");
    return MUELLER_OK;
  }
  dim3 g(nblk(m->nn, 8), 1);
  { Prof prof_("near_spmv_kernel<float2, float2>", s); near_spmv_kernel<float2, float2><<<g, 256, 0, s>>>(m->nn, m->near_rowptr, m->near_col, near32, X, Y, N, N, 1, stop); }
  MU_CHECK_LAUNCH("near_spmv_kernel<float2, float2>");
  return MUELLER_OK;
}

// ================================================================= MBJ build
struct BlockLayout {
  int64_t H, B, nb, d;
  std::vector<int32_t> sz;  // 2 * |I_m|
};

static BlockLayout layout(int64_t N, int64_t B) {
  BlockLayout L;
  L.H = N / 2;
  L.B = B;
  L.nb = (L.H + B - 1) / B;
  L.d = 2 * std::min(B, L.H);
  for (int64_t b = 0; b < L.nb; ++b) L.sz.push_back((int32_t)(2 * std::min(B, L.H - b * B)));
  return L;
}

template <class CT>
static mueller_status block_inverse(const CT* A, int64_t d, int nb, const int32_t* sz_dev,
                                    const int32_t* piv, CT* inv, cudaStream_t s);

// Panel [k0, k0+LUW) of every block: in shared memory when its rows fit.
static mueller_status lu_panel(double2* A, int64_t d, int nb, const int32_t* sz_dev, int k0,
                               int32_t* piv, int32_t* status, int defer, cudaStream_t s) {
  constexpr size_t kPanelSmem = 200 * 1024;
  const size_t panel_bytes = (size_t)(d - k0) * (LUW + 1) * sizeof(double2);
  if (d - k0 <= 1024 && panel_bytes <= kPanelSmem) {
    MU_CUDA(cudaFuncSetAttribute(lu_panel_smem_kernel<double2, LUW>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmem));
    // one thread per remaining row: no idle warps in the per-column reductions
    const unsigned threads = (unsigned)std::max<int64_t>(32, ((d - k0) + 31) / 32 * 32);
    { Prof prof_("lu_panel_smem_kernel", s); lu_panel_smem_kernel<double2, LUW><<<nb, threads, panel_bytes, s>>>(A, d, sz_dev, k0, piv, status, defer); }
    MU_CHECK_LAUNCH("lu_panel_smem_kernel");
  } else {
    { Prof prof_("lu_panel_kernel", s); lu_panel_kernel<double2, LUW><<<nb, 256, 0, s>>>(A, d, sz_dev, k0, piv, status, defer); }
    MU_CHECK_LAUNCH("lu_panel_kernel");
  }
  return MUELLER_OK;
}

// trailing update A[k0+LUW:n, c0:c1) of panel k0: the next panel's columns
// (TN = LUW) or the rest (TN = 32), one CTA per tile.  (A grid of a few
// persistent CTAs per SM, which leaves room for the panel beside it, was
// slower: the panel then shares its SM's FP64 pipe and the chain of panels
// becomes the critical path.)
template <int TN, int TR = 32>
static mueller_status lu_update(double2* A, int64_t d, int nb, const int32_t* sz_dev, int k0,
                                int64_t c0, int64_t c1, cudaStream_t s) {
  const int64_t rows = d - (k0 + LUW), cols = (c1 < 0 ? d : c1) - c0;
  if (rows <= 0 || cols <= 0) return MUELLER_OK;
  const int64_t grid = nb * nblk(rows, TR) * nblk(cols, TN);
  { Prof prof_("lu_update_kernel", s); lu_update_kernel<LUW, TN, TR><<<(unsigned)grid, 64, 0, s>>>(A, d, sz_dev, k0, c0, c1, nb); }
  MU_CHECK_LAUNCH("lu_update_kernel");
  return MUELLER_OK;
}

// In-place FP64 LU with partial pivoting of nb blocks of size d (active
// sizes sz_dev), right-looking in panels of LUW columns with a look-ahead of
// one panel.  Per panel k0: its row swaps reach the other columns and the
// row panel of U is solved (one kernel); the columns of panel k0+LUW are
// updated; then that panel is factored (its swaps held back) while the
// remaining columns take the trailing update: in one lu_step_kernel launch
// on separate SMs when the panel's rows fit one CTA (d - k1 <= 512), else on
// the side stream next to the caller's stream.
// Then, if inv, the inverses in 'inv' (d x d per block).
template <class CT>
static mueller_status batched_lu_inverse(CT* A, int64_t d, int nb, const int32_t* sz_dev,
                                         int32_t* piv, int32_t* status, CT* inv,
                                         cudaStream_t s) {
  static_assert(sizeof(CT) == 16, "the block LU is FP64");
  cudaStream_t s2 = nullptr;
  mueller_status st = side_stream(&s2);
  // one tile-queue counter per panel step
  const int nsteps = (int)((d + LUW - 1) / LUW);
  unsigned* queue = nullptr;
  if (!st) {
    cudaError_t e = cudaMallocAsync((void**)&queue, (size_t)nsteps * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, (size_t)nsteps * sizeof(unsigned), s);
    if (e != cudaSuccess) st = cuda_fail(e, "LU tile queues");
  }
  int nsm = 0, dev = 0;
  if (!st && (cudaGetDevice(&dev) != cudaSuccess ||
              cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
    nsm = 148;
  if (!st) {
    cudaError_t e = cudaFuncSetAttribute(lu_step_kernel<LUW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kLuStepSmem);
    if (e != cudaSuccess) st = cuda_fail(e, "LU step kernel attributes");
  }
  if (!st) st = lu_panel(A, d, nb, sz_dev, 0, piv, status, 1, s);
  for (int k0 = 0, step = 0; !st && k0 < d; k0 += LUW, ++step) {
    // one warp per 32 columns: the FP64 work of the triangular solves spreads
    // over all SMs
    { Prof prof_("lu_swap_trsm_kernel", s); lu_swap_trsm_kernel<LUW><<<dim3(nblk(d, 32), nb), 32, 0, s>>>(A, d, sz_dev, k0, piv); }
    MU_CHECK_LAUNCH("lu_swap_trsm_kernel");
    const int k1 = k0 + LUW;
    if (k1 >= d) break;
    // the next panel's columns first, alone on the GPU: FP64-bound CTAs that
    // share an SM slow down together, so next to the bulk update this small
    // update would last as long as the bulk update and hold the panel back
    st = lu_update<LUW, 16>(A, d, nb, sz_dev, k0, k1, k1 + LUW, s);
    if (st) break;
    if (d - k1 <= kLuStepThreads) {
      // panel k1 and the rest of update k0 in one launch, on separate SMs
      const int64_t c0 = k1 + LUW;
      const unsigned grid = (unsigned)std::max(nsm, nb);
      {
        Prof prof_("lu_step_kernel", s);
        lu_step_kernel<LUW><<<grid, kLuStepThreads, kLuStepSmem, s>>>(A, d, sz_dev, k0, k1, c0, nb,
                                                                      piv, status, queue + step);
      }
      MU_CHECK_LAUNCH("lu_step_kernel");
      continue;
    }
    // panels too tall for one CTA's threads: the panel on the side stream
    // while the caller's stream updates the remaining columns
    st = stream_order(s, s2);
    if (!st) st = lu_panel(A, d, nb, sz_dev, k1, piv, status, 1, s2);
    const mueller_status su = st ? st : lu_update<32>(A, d, nb, sz_dev, k0, k1 + LUW, -1, s);
    const mueller_status sj = stream_order(s2, s);
    if (!st) st = su ? su : sj;
  }
  if (queue) cudaFreeAsync(queue, s);
  if (st || !inv) return st;
  return block_inverse<CT>(A, d, nb, sz_dev, piv, inv, s);
}

// inv = U^{-1} L^{-1} P from the LU factors in A (complex type CT)
template <class CT>
static mueller_status block_inverse(const CT* A, int64_t d, int nb, const int32_t* sz_dev,
                                    const int32_t* piv, CT* inv, cudaStream_t s) {
  // entries outside a block's active size are zero (the kernels below write
  // the active part only)
  MU_CUDA(cudaMemsetAsync(inv, 0, (size_t)nb * d * d * sizeof(CT), s));
  if constexpr (std::is_same<CT, float2>::value) {
    if (d <= 2 * kInvThreads) {  // diagonal tiles' inverses, then one launch for the rest
      const int ntile = (int)nblk(d, 32);
      float2* Tinv = nullptr;
      MU_CUDA(cudaMallocAsync((void**)&Tinv, (size_t)nb * ntile * 2 * 1024 * sizeof(float2), s));
      { Prof prof_("tile_inverse_kernel", s); tile_inverse_kernel<<<dim3(ntile, nb, 2), 32, 0, s>>>(A, d, sz_dev, ntile, Tinv); }
      cudaError_t le = cudaGetLastError();
      if (le == cudaSuccess) {
        const dim3 grid((unsigned)nblk(d, kInvCW), (unsigned)nb);
        Prof prof_("block_inverse_cols_kernel", s);
        if (d <= kInvThreads)
          block_inverse_cols_kernel<1><<<grid, kInvThreads, 0, s>>>(A, d, sz_dev, piv, Tinv, ntile, inv);
        else
          block_inverse_cols_kernel<2><<<grid, kInvThreads, 0, s>>>(A, d, sz_dev, piv, Tinv, ntile, inv);
        le = cudaGetLastError();
      }
      cudaFreeAsync(Tinv, s);
      if (le != cudaSuccess) return cuda_fail(le, "block inverse kernels");
      return MUELLER_OK;
    }
  }
  { Prof prof_("perm_identity_kernel", s); perm_identity_kernel<CT><<<dim3(nblk(d, 128), nb), 128, 0, s>>>(inv, d, sz_dev, piv); }
  MU_CHECK_LAUNCH("perm_identity_kernel");
  for (int k0 = 0; k0 < d; k0 += NBK) {  // forward: L (unit lower)
    { Prof prof_("trsm_tile_kernel", s); trsm_tile_kernel<CT, NBK><<<dim3(nblk(d, 128), nb), 128, 0, s>>>(A, inv, d, d, d * d, sz_dev, k0, NBK, 0, -1, 0); }
    MU_CHECK_LAUNCH("trsm_tile_kernel(L)");
    const int64_t below = d - (k0 + NBK);
    if (below > 0) {
      dim3 gg(nblk(d, 64), nblk(below, 64), nb);
      { Prof prof_("gemm_update_kernel", s); gemm_update_kernel<CT, NBK><<<gg, 256, 0, s>>>(A, inv, inv, d, d, d * d, sz_dev, k0, k0 + NBK, -1, 0, -1); }
      MU_CHECK_LAUNCH("gemm_update_kernel(L)");
    }
  }
  const int64_t ntile = (d + NBK - 1) / NBK;
  for (int64_t t = ntile - 1; t >= 0; --t) {  // backward: U
    const int k0 = (int)(t * NBK);
    { Prof prof_("trsm_tile_kernel", s); trsm_tile_kernel<CT, NBK><<<dim3(nblk(d, 128), nb), 128, 0, s>>>(A, inv, d, d, d * d, sz_dev, k0, NBK, 0, -1, 1); }
    MU_CHECK_LAUNCH("trsm_tile_kernel(U)");
    if (k0 > 0) {
      dim3 gg(nblk(d, 64), nblk(k0, 64), nb);
      { Prof prof_("gemm_update_kernel", s); gemm_update_kernel<CT, NBK><<<gg, 256, 0, s>>>(A, inv, inv, d, d, d * d, sz_dev, k0, 0, k0, 0, -1); }
      MU_CHECK_LAUNCH("gemm_update_kernel(U)");
    }
  }
  return MUELLER_OK;
}

// precond_dev layout: [nb][d][d] inverses, then int32 sz[nb].  The inverses
// are complex128 for a C128 operator (FP64 GMRES applies them in FP64) and
// complex64 for a C64_NEAR64 operator, whose inner GMRES applies them in
// FP32: the LU factorisation is FP64 in both cases; for the mixed operator
// the explicit inverse is then formed from the FP64 factors in FP32.
static const int32_t* precond_sizes(const mueller_operator* op, const BlockLayout& L) {
  const size_t elem = op->dtype == MUELLER_C128 ? 16 : 8;
  return (const int32_t*)((const char*)op->precond_dev + (size_t)L.nb * L.d * L.d * elem);
}

mueller_status precond_build(const mueller_operator* op, int64_t block, void* P, cudaStream_t s) {
  const mueller_mesh* m = op->mesh;
  const int64_t N = 4 * m->nn;
  BlockLayout L = layout(N, block);
  const size_t elem = op->dtype == MUELLER_C128 ? 16 : 8;
  int32_t* sz_dev = (int32_t*)((char*)P + (size_t)L.nb * L.d * L.d * elem);
  MU_CUDA(cudaMemcpyAsync(sz_dev, L.sz.data(), L.nb * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  double2* A = nullptr;
  int32_t* piv = nullptr;
  MU_CUDA(cudaMallocAsync((void**)&A, (size_t)L.nb * L.d * L.d * sizeof(double2), s));
  MU_CUDA(cudaMallocAsync((void**)&piv, (size_t)L.nb * L.d * sizeof(int32_t) + 64, s));
  int32_t* status = piv + L.nb * L.d;
  MU_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
  dim3 g(nblk(L.d, 128), L.d, L.nb);
  if (op->dtype == MUELLER_C128) {
    { Prof prof_("gather_blocks_kernel", s); gather_blocks_kernel<MUELLER_C128><<<g, 128, 0, s>>>(op->Z_dev, op->ldz, L.H, L.B, L.d, sz_dev, A); }
  } else {
    { Prof prof_("gather_blocks_kernel", s); gather_blocks_kernel<MUELLER_C64_NEAR64><<<g, 128, 0, s>>>(op->Z_dev, op->ldz, L.H, L.B, L.d, sz_dev, A); }
    MU_CHECK_LAUNCH("gather_blocks_kernel");
    { Prof prof_("gather_near_kernel", s); gather_near_kernel<<<nblk(m->nn, 8), 256, 0, s>>>(m->nn, m->near_rowptr, m->near_col,
                                                        (const double2*)op->near_dev, L.B, L.d,
                                                        sz_dev, A); }
  }
  MU_CHECK_LAUNCH("gather kernels");
  mueller_status st = MUELLER_OK;
  float2* A32 = nullptr;
  if (op->dtype == MUELLER_C128) {
    st = batched_lu_inverse<double2>(A, L.d, (int)L.nb, sz_dev, piv, status, (double2*)P, s);
  } else {
    // the preconditioner of the complex64 inner solver: FP64 factorisation,
    // explicit inverse formed from the FP64 factors in FP32
    st = batched_lu_inverse<double2>(A, L.d, (int)L.nb, sz_dev, piv, status, nullptr, s);
    const int64_t cnt = (int64_t)L.nb * L.d * L.d;
    if (!st) {
      cudaError_t e = cudaMallocAsync((void**)&A32, cnt * sizeof(float2), s);
      if (e != cudaSuccess) st = cuda_fail(e, "precond FP32 factors");
    }
    if (!st) {
      { Prof prof_("c128_to_c64_kernel", s); c128_to_c64_kernel<<<nblk(cnt, 256), 256, 0, s>>>(A, A32, cnt); }
      MU_CHECK_LAUNCH("c128_to_c64_kernel");
      st = block_inverse<float2>(A32, L.d, (int)L.nb, sz_dev, piv, (float2*)P, s);
    }
  }
  int32_t hst = 0;
  if (!st) {
    cudaError_t e = cudaMemcpyAsync(&hst, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "precond status");
  }
  cudaFreeAsync(A, s);
  cudaFreeAsync(piv, s);
  if (A32) cudaFreeAsync(A32, s);
  if (st) return st;
  if (hst) {
    set_error("zero pivot in block-Jacobi block " + std::to_string(hst - 1));
    return MUELLER_ERR_SINGULAR_BLOCK;
  }
  return MUELLER_OK;
}

// Block-Jacobi preconditioners of n operators (bodies) at once: the blocks
// of every body (same block dimension d = 2 min(B, H)) are gathered into one
// array and factorised by one batched LU, so that many small bodies fill the
// GPU together; each body's inverses then go to its own buffer.  Bodies with
// another d are built in their own batch.
mueller_status precond_build_batch(int n, const mueller_operator* ops, const int64_t* blocks,
                                   void* const* P, cudaStream_t s) {
  std::vector<BlockLayout> Ls(n);
  for (int b = 0; b < n; ++b) Ls[b] = layout(4 * ops[b].mesh->nn, blocks[b]);
  std::vector<int> done(n, 0);
  for (int lead = 0; lead < n; ++lead) {
    if (done[lead]) continue;
    const int64_t d = Ls[lead].d;
    const int dtype = ops[lead].dtype;
    std::vector<int> grp;
    for (int b = lead; b < n; ++b)
      if (!done[b] && Ls[b].d == d && ops[b].dtype == dtype) {
        grp.push_back(b);
        done[b] = 1;
      }
    // block offsets of the group's bodies in the batch
    std::vector<int64_t> off(grp.size() + 1, 0);
    std::vector<int32_t> sz_all;
    for (size_t g = 0; g < grp.size(); ++g) {
      off[g + 1] = off[g] + Ls[grp[g]].nb;
      sz_all.insert(sz_all.end(), Ls[grp[g]].sz.begin(), Ls[grp[g]].sz.end());
    }
    const int64_t nbt = off.back();
    const size_t elem = dtype == MUELLER_C128 ? 16 : 8;
    double2* A = nullptr;
    int32_t* piv = nullptr;
    int32_t* sz_dev = nullptr;
    void* inv = nullptr;
    float2* A32 = nullptr;
    mueller_status st = MUELLER_OK;
    auto take = [&](void** ptr, size_t bytes) {
      if (st) return;
      cudaError_t e = cudaMallocAsync(ptr, bytes, s);
      if (e != cudaSuccess) st = cuda_fail(e, "batched precond workspace");
    };
    take((void**)&A, (size_t)nbt * d * d * sizeof(double2));
    take((void**)&piv, (size_t)nbt * d * sizeof(int32_t) + 64);
    take((void**)&sz_dev, (size_t)nbt * sizeof(int32_t));
    take(&inv, (size_t)nbt * d * d * elem);
    int32_t* status = piv ? piv + nbt * d : nullptr;
    if (!st) {
      cudaError_t e = cudaMemcpyAsync(sz_dev, sz_all.data(), nbt * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
      if (e != cudaSuccess) st = cuda_fail(e, "batched precond setup");
    }
    for (size_t g = 0; g < grp.size() && !st; ++g) {
      const mueller_operator* op = &ops[grp[g]];
      const BlockLayout& L = Ls[grp[g]];
      const mueller_mesh* m = op->mesh;
      double2* Ab = A + off[g] * d * d;
      const int32_t* szb = sz_dev + off[g];
      dim3 gg(nblk(d, 128), d, L.nb);
      if (dtype == MUELLER_C128) {
        { Prof prof_("gather_blocks_kernel", s); gather_blocks_kernel<MUELLER_C128><<<gg, 128, 0, s>>>(op->Z_dev, op->ldz, L.H, L.B, d, szb, Ab); }
      } else {
        { Prof prof_("gather_blocks_kernel", s); gather_blocks_kernel<MUELLER_C64_NEAR64><<<gg, 128, 0, s>>>(op->Z_dev, op->ldz, L.H, L.B, d, szb, Ab); }
        { Prof prof_("gather_near_kernel", s); gather_near_kernel<<<nblk(m->nn, 8), 256, 0, s>>>(m->nn, m->near_rowptr, m->near_col,
                                                            (const double2*)op->near_dev, L.B, d, szb, Ab); }
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_fail(e, "batched precond gather");
    }
    if (!st) {
      if (dtype == MUELLER_C128) {
        st = batched_lu_inverse<double2>(A, d, (int)nbt, sz_dev, piv, status, (double2*)inv, s);
      } else {
        st = batched_lu_inverse<double2>(A, d, (int)nbt, sz_dev, piv, status, nullptr, s);
        const int64_t cnt = nbt * d * d;
        take((void**)&A32, cnt * sizeof(float2));
        if (!st) {
          { Prof prof_("c128_to_c64_kernel", s); c128_to_c64_kernel<<<nblk(cnt, 256), 256, 0, s>>>(A, A32, cnt); }
          MU_CHECK_LAUNCH("c128_to_c64_kernel");
          st = block_inverse<float2>(A32, d, (int)nbt, sz_dev, piv, (float2*)inv, s);
        }
      }
    }
    // each body's inverses and block sizes into its buffer (layout of precond_build)
    for (size_t g = 0; g < grp.size() && !st; ++g) {
      const BlockLayout& L = Ls[grp[g]];
      char* Pb = (char*)P[grp[g]];
      const size_t bytes = (size_t)L.nb * d * d * elem;
      cudaError_t e = cudaMemcpyAsync(Pb, (const char*)inv + (size_t)off[g] * d * d * elem, bytes,
                                      cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(Pb + bytes, L.sz.data(), L.nb * sizeof(int32_t), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) st = cuda_fail(e, "batched precond copy-out");
    }
    int32_t hst = 0;
    if (!st) {
      cudaError_t e = cudaMemcpyAsync(&hst, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_fail(e, "batched precond status");
    }
    if (A) cudaFreeAsync(A, s);
    if (piv) cudaFreeAsync(piv, s);
    if (sz_dev) cudaFreeAsync(sz_dev, s);
    if (inv) cudaFreeAsync(inv, s);
    if (A32) cudaFreeAsync(A32, s);
    if (st) return st;
    if (hst) {
      const int64_t k = hst - 1;
      size_t g = 0;
      while (g + 1 < off.size() && off[g + 1] <= k) ++g;
      set_error("zero pivot in block-Jacobi block " + std::to_string(k - off[g]) + " of body " +
                std::to_string(grp[g]));
      return MUELLER_ERR_SINGULAR_BLOCK;
    }
  }
  return MUELLER_OK;
}

// ================================================================= solvers
namespace {

struct GmresWork {
  int64_t N;
  int m, G;
  void* V;      // (m+1) x N complex (T)
  void* w;      // N
  void* z;      // N
  void* u;      // N
  double2* Hm;  // (m+1) x m
  double2* hacc;
  double2* part;
  double* npart;
  double* cs;
  double2* sn;
  double2* g;
  double2* y;
  double* scal;  // [0] res estimate, [1] hn, [2] beta, [3] norm scratch
  double* hs;    // pinned host scalar
};

size_t gmres_bytes(int64_t N, int m, size_t elem) {
  const int G = 16;
  size_t b = 0;
  b += (size_t)(m + 1) * N * elem + 3 * (size_t)N * elem;
  b += (size_t)(m + 1) * m * 16 + (size_t)(m + 2) * 16 + (size_t)(m + 1) * G * 16 + G * 8;
  b += (size_t)(m + 1) * (8 + 16 + 16 + 16) + 16 * 8;
  return b + 16 * 256;
}

template <class VT>
GmresWork carve_gmres(char*& p, int64_t N, int m) {
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~size_t(255);
    return (void*)r;
  };
  GmresWork W;
  W.N = N;
  W.m = m;
  W.G = 16;
  W.V = take((size_t)(m + 1) * N * sizeof(VT));
  W.w = take(N * sizeof(VT));
  W.z = take(N * sizeof(VT));
  W.u = take(N * sizeof(VT));
  W.Hm = (double2*)take((size_t)(m + 1) * m * 16);
  W.hacc = (double2*)take((size_t)(m + 2) * 16);
  W.part = (double2*)take((size_t)(m + 1) * W.G * 16);
  W.npart = (double*)take(W.G * 8);
  W.cs = (double*)take((m + 1) * 8);
  W.sn = (double2*)take((m + 1) * 16);
  W.g = (double2*)take((m + 1) * 16);
  W.y = (double2*)take((m + 1) * 16);
  W.scal = (double*)take(16 * 8);
  return W;
}

// The operator as seen by one GMRES: matvec and preconditioner in VT.
struct InnerOp {
  const mueller_operator* op;
  int precision;             // 0: complex128, 1: complex64
  const float2* near32;      // complex64 near blocks (precision 1)
  const float2* inv32;       // complex64 inverses (precision 1)
  BlockLayout L;
  const int32_t* sz_dev;
};

template <class VT>
mueller_status inner_matvec(const InnerOp& I, const VT* x, VT* y, cudaStream_t s) {
  const mueller_mesh* m = I.op->mesh;
  const int64_t N = 4 * m->nn;
  if constexpr (sizeof(VT) == 16) {
    return op_matvec(I.op, x, y, 1, nullptr, 0, s);
  } else {
    mueller_status st = gemv_c64_f32(I.op, x, y, s);
    if (st) return st;
    { Prof prof_("near_spmv_kernel<float2, float2>", s); near_spmv_kernel<float2, float2><<<dim3(nblk(m->nn, 8), 1), 256, 0, s>>>(
        m->nn, m->near_rowptr, m->near_col, I.near32, x, y, N, N, 1, nullptr); }
    MU_CHECK_LAUNCH("near_spmv_kernel<float>");
    return MUELLER_OK;
  }
}

template <class VT>
mueller_status inner_precond(const InnerOp& I, const VT* v, VT* z, cudaStream_t s) {
  const int64_t N = 4 * I.op->mesh->nn;
  if (!I.op->precond_dev) {
    MU_CUDA(cudaMemcpyAsync(z, v, N * sizeof(VT), cudaMemcpyDeviceToDevice, s));
    return MUELLER_OK;
  }
  dim3 g(nblk(I.L.d, 8), I.L.nb);
  if constexpr (sizeof(VT) == 16) {
    if (I.op->flags & MUELLER_OP_ADJOINT) {
      { Prof prof_("mbj_apply_h_kernel", s); mbj_apply_h_kernel<<<dim3(nblk(I.L.d, 128), I.L.nb), 128, 0, s>>>((const double2*)I.op->precond_dev, I.L.d, I.sz_dev, I.L.B, I.L.H, (const double2*)v, (double2*)z); }
      MU_CHECK_LAUNCH("mbj_apply_h_kernel");
      return MUELLER_OK;
    }
    { Prof prof_("mbj_apply_kernel<double2, double2>", s); mbj_apply_kernel<double2, double2><<<g, 256, 0, s>>>((const double2*)I.op->precond_dev, I.L.d,
                                                        I.sz_dev, I.L.B, I.L.H, v, z); }
  } else {
    { Prof prof_("mbj_apply_kernel<float2, float2>", s); mbj_apply_kernel<float2, float2><<<g, 256, 0, s>>>(I.inv32, I.L.d, I.sz_dev, I.L.B, I.L.H, v, z); }
  }
  MU_CHECK_LAUNCH("mbj_apply_kernel");
  return MUELLER_OK;
}

// One GMRES(m) solve of A x = b in precision VT, right-preconditioned.
// x holds x0 on entry.  Convergence on the Arnoldi estimate and on the true
// residual (in VT) at each restart; rel tolerance 'tol'.  Host reads one
// scalar per Arnoldi step.
template <class VT>
mueller_status gmres(const InnerOp& I, GmresWork& W, const VT* b, VT* x, double tol, int maxit,
                     int& iters, int& restarts, double& relres, cudaStream_t s) {
  const int64_t N = W.N;
  const int m = W.m, G = W.G;
  VT* V = (VT*)W.V;
  VT* w = (VT*)W.w;
  VT* z = (VT*)W.z;
  VT* u = (VT*)W.u;
  double* hs = W.hs;
  auto read = [&](const double* dptr, double& out) -> mueller_status {
    MU_CUDA(cudaMemcpyAsync(hs, dptr, sizeof(double), cudaMemcpyDeviceToHost, s));
    MU_CUDA(cudaStreamSynchronize(s));
    out = hs[0];
    return MUELLER_OK;
  };
  mueller_status st = MUELLER_OK;
  auto norm_into = [&](const VT* v, double* dst) -> mueller_status {
    { Prof prof_("nrm2_kernel<VT>", s); nrm2_kernel<VT><<<G, 256, 0, s>>>(v, N, W.npart, G); }
    MU_CHECK_LAUNCH("nrm2_kernel");
    { Prof prof_("normalize_kernel<VT>", s); normalize_kernel<VT><<<1, 1, 0, s>>>(v, 0, W.npart, G, nullptr, dst); }
    MU_CHECK_LAUNCH("normalize_kernel");
    return MUELLER_OK;
  };
  // ||b||
  double bn = 0;
  if ((st = norm_into(b, W.scal + 3))) goto done;
  if ((st = read(W.scal + 3, bn))) goto done;
  iters = 0;
  restarts = 0;
  if (bn == 0.0) {
    MU_CUDA(cudaMemsetAsync(x, 0, N * sizeof(VT), s));
    relres = 0.0;
    goto done;
  }
  // r = b - A x  (in w), beta
  for (;;) {
    if ((st = inner_matvec<VT>(I, x, w, s))) goto done;
    {
      // w = b - w
      { Prof prof_("axpy_kernel<VT, VT>", s); axpy_kernel<VT, VT><<<nblk(N, 256), 256, 0, s>>>(w, w, N, -2.0); }  // w := -w
      MU_CHECK_LAUNCH("axpy");
      { Prof prof_("axpy_kernel<VT, VT>", s); axpy_kernel<VT, VT><<<nblk(N, 256), 256, 0, s>>>(w, b, N, 1.0); }
      MU_CHECK_LAUNCH("axpy");
    }
    if ((st = norm_into(w, W.scal + 2))) goto done;
    double beta;
    if ((st = read(W.scal + 2, beta))) goto done;
    relres = beta / bn;
    if (relres <= tol || iters >= maxit) goto done;
    // V0 = w / beta, g = beta e1
    { Prof prof_("normalize_kernel<VT>", s); normalize_kernel<VT><<<nblk(N, 256), 256, 0, s>>>(w, N, W.npart, G, V, W.scal + 2); }
    MU_CHECK_LAUNCH("normalize");
    { Prof prof_("set_first_kernel<VT>", s); set_first_kernel<VT><<<1, 1, 0, s>>>(W.g, m, W.scal + 2); }
    MU_CUDA(cudaMemsetAsync(W.hacc, 0, (m + 2) * sizeof(double2), s));
    int k = 0;
    for (int j = 0; j < m && iters < maxit; ++j) {
      const VT* vj = V + (int64_t)j * N;
      if ((st = inner_precond<VT>(I, vj, z, s))) goto done;
      if ((st = inner_matvec<VT>(I, z, w, s))) goto done;
      for (int pass = 0; pass < 2; ++pass) {
        { Prof prof_("dots_kernel<VT>", s); dots_kernel<VT><<<dim3(G, j + 1), 256, 0, s>>>(V, N, j + 1, w, W.part, G); }
        MU_CHECK_LAUNCH("dots_kernel");
        { Prof prof_("orth_update_kernel<VT>", s); orth_update_kernel<VT><<<nblk(N, 256), 256, 0, s>>>(V, N, j + 1, W.part, G, w, W.hacc); }
        MU_CHECK_LAUNCH("orth_update_kernel");
      }
      { Prof prof_("nrm2_kernel<VT>", s); nrm2_kernel<VT><<<G, 256, 0, s>>>(w, N, W.npart, G); }
      MU_CHECK_LAUNCH("nrm2");
      { Prof prof_("normalize_kernel<VT>", s); normalize_kernel<VT><<<nblk(N, 256), 256, 0, s>>>(w, N, W.npart, G, V + (int64_t)(j + 1) * N,
                                                        W.scal + 1); }
      MU_CHECK_LAUNCH("normalize");
      { Prof prof_("givens_kernel", s); givens_kernel<<<1, 1, 0, s>>>(j, m, W.hacc, W.scal + 1, W.Hm, W.cs, W.sn, W.g, W.scal); }
      MU_CHECK_LAUNCH("givens_kernel");
      ++iters;
      k = j + 1;
      double est;
      if ((st = read(W.scal, est))) goto done;
      if (est / bn <= tol || !(est == est)) break;
    }
    { Prof prof_("backsub_kernel", s); backsub_kernel<<<1, 1, 0, s>>>(k, m, W.Hm, W.g, W.y); }
    MU_CHECK_LAUNCH("backsub_kernel");
    { Prof prof_("combine_kernel<VT>", s); combine_kernel<VT><<<nblk(N, 256), 256, 0, s>>>(V, N, k, W.y, u); }
    MU_CHECK_LAUNCH("combine_kernel");
    if ((st = inner_precond<VT>(I, u, z, s))) goto done;
    { Prof prof_("axpy_kernel<VT, VT>", s); axpy_kernel<VT, VT><<<nblk(N, 256), 256, 0, s>>>(x, z, N, 1.0); }
    MU_CHECK_LAUNCH("axpy");
    ++restarts;
  }
done:
  return st;
}

}  // namespace

// ----------------------------------------------------------------------
// Mixed-precision solve of r right-hand sides: complex64 GMRES(m) with all
// r systems advancing in lockstep (one product with Z per Arnoldi step for
// all of them: tensor cores for r >= 2), right preconditioned by the
// complex64 block-Jacobi inverses, inside FP64 iterative refinement on the
// stored operator.
struct LockWork {
  int64_t N;
  int r, m, G;
  float2 *V, *W, *Zt, *U, *rhs32, *d32;
  double2 *r64, *y64;
  double2 *Hm, *hacc, *part, *sn, *g, *y;
  double *npart, *cs, *bn, *beta, *hn, *res, *rn, *alpha;
  int *mask, *kk;
  void* mwork;
  float2* near32;  // complex64 copy of the near blocks (nnzb x 16), or null
  // fused Arnoldi step (arnoldi_tail_kernel): tcs CTAs per right-hand side
  int tcs;
  int* flags;      // [0] stop, [1] steps at stop, [8] finished-cluster ticket
  int* bad;        // [r] residual estimate not a number
};

// CTAs per right-hand side in the fused Arnoldi step (its cluster size): a
// power of two with at least about 640 vector entries per CTA, at most 16
// (more than 8 is a non-portable cluster size, taken only where the device
// can run such a cluster of this kernel)
static int tail_cluster(int64_t N) {
  static int cmax = 0;
  if (cmax == 0) {
    cmax = 8;
    if (cudaFuncSetAttribute(arnoldi_tail_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3(16, 1);
      lc.blockDim = dim3(256);
      cudaLaunchAttribute la[1];
      la[0].id = cudaLaunchAttributeClusterDimension;
      la[0].val.clusterDim.x = 16;
      la[0].val.clusterDim.y = 1;
      la[0].val.clusterDim.z = 1;
      lc.attrs = la;
      lc.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, arnoldi_tail_kernel, &lc) == cudaSuccess && ncl > 0)
        cmax = 16;
    }
    cudaGetLastError();
  }
  int c = 1;
  while (c < cmax && N > (int64_t)640 * c) c *= 2;
  return c;
}

static size_t lock_bytes(int64_t N, int r, int m, int64_t nnzb) {
  const int G = 16;
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~size_t(255); };
  add((size_t)(m + 1) * r * N * 8);
  for (int k = 0; k < 6; ++k) add((size_t)r * N * 8);
  add((size_t)r * N * 16);
  add((size_t)r * N * 16);
  add((size_t)r * m * (m + 1) * 16);
  add((size_t)r * (m + 2) * 16);
  add((size_t)r * (m + 1) * G * 16);
  for (int k = 0; k < 3; ++k) add((size_t)r * (m + 1) * 16);
  add((size_t)r * G * 8);
  add((size_t)r * (m + 1) * 8);
  for (int k = 0; k < 6; ++k) add((size_t)r * 8);
  add((size_t)r * 4);
  add((size_t)r * 4);
  if (r >= 2) add(mrhs_work_bytes(N, r));
  if (nnzb > 0) add((size_t)nnzb * 16 * 8);
  add(64 * 4);
  add((size_t)r * 4);
  return b + 1024;
}

static LockWork carve_lock(char* p, int64_t N, int r, int m, int64_t nnzb) {
  LockWork W;
  W.N = N;
  W.r = r;
  W.m = m;
  W.G = 16;
  auto take = [&](size_t x) {
    char* q = p;
    p += (x + 255) & ~size_t(255);
    return (void*)q;
  };
  W.V = (float2*)take((size_t)(m + 1) * r * N * 8);
  W.W = (float2*)take((size_t)r * N * 8);
  W.Zt = (float2*)take((size_t)r * N * 8);
  W.U = (float2*)take((size_t)r * N * 8);
  W.rhs32 = (float2*)take((size_t)r * N * 8);
  W.d32 = (float2*)take((size_t)r * N * 8);
  take((size_t)r * N * 8);
  W.r64 = (double2*)take((size_t)r * N * 16);
  W.y64 = (double2*)take((size_t)r * N * 16);
  W.Hm = (double2*)take((size_t)r * m * (m + 1) * 16);
  W.hacc = (double2*)take((size_t)r * (m + 2) * 16);
  W.part = (double2*)take((size_t)r * (m + 1) * W.G * 16);
  W.sn = (double2*)take((size_t)r * (m + 1) * 16);
  W.g = (double2*)take((size_t)r * (m + 1) * 16);
  W.y = (double2*)take((size_t)r * (m + 1) * 16);
  W.npart = (double*)take((size_t)r * W.G * 8);
  W.cs = (double*)take((size_t)r * (m + 1) * 8);
  W.bn = (double*)take((size_t)r * 8);
  W.beta = (double*)take((size_t)r * 8);
  W.hn = (double*)take((size_t)r * 8);
  W.res = (double*)take((size_t)r * 8);
  W.rn = (double*)take((size_t)r * 8);
  W.alpha = (double*)take((size_t)r * 8);
  W.mask = (int*)take((size_t)r * 4);
  W.kk = (int*)take((size_t)r * 4);
  W.mwork = r >= 2 ? take(mrhs_work_bytes(N, r)) : nullptr;
  W.near32 = nnzb > 0 ? (float2*)take((size_t)nnzb * 16 * 8) : nullptr;
  W.tcs = tail_cluster(N);
  W.flags = (int*)take(64 * 4);
  W.bad = (int*)take((size_t)r * 4);
  return W;
}

// complex64 product of the stored operator for the r vectors of X
// (stop: device flag; nonzero skips the kernels, see arnoldi_tail_kernel)
static mueller_status lock_matvec(const InnerOp& I, const LockWork& W, const float2* X, float2* Y,
                                  cudaStream_t s, const int* stop = nullptr) {
  const mueller_mesh* m = I.op->mesh;
  const int64_t N = W.N;
  if (W.r >= 2) {
    mueller_status st = mrhs_matvec_c64(I.op->Z_dev, N, I.op->ldz, X, Y, W.r, W.mwork, s, stop,
                                         (I.op->flags & MUELLER_OP_K1_MIRRORED) ? 1 : 0);
    if (st) return st;
  } else {
    int fused = 0;
    mueller_status st = gemv_c64_f32(I.op, X, Y, s, stop, I.near32, &fused);
    if (st) return st;
    if (fused) return MUELLER_OK;
  }
  if (I.near32) return near_apply_c64_b32(m, I.near32, X, Y, W.r, s, stop);
  return near_apply_c64(m, I.op->near_dev, X, Y, W.r, s);
}

static mueller_status lock_precond(const InnerOp& I, const LockWork& W, const float2* v, float2* z,
                                   cudaStream_t s, const int* stop = nullptr) {
  if (!I.op->precond_dev) {
    MU_CUDA(cudaMemcpyAsync(z, v, (size_t)W.r * W.N * 8, cudaMemcpyDeviceToDevice, s));
    return MUELLER_OK;
  }
  constexpr int RS = 8;
  const size_t smem = (size_t)RS * I.L.d * sizeof(float2);
  if (W.r >= 2 && smem <= 200 * 1024) {
    dim3 g(nblk(I.L.d, kMbjRows), I.L.nb, (W.r + RS - 1) / RS);
    MU_CUDA(cudaFuncSetAttribute(mbj_apply_rs_kernel<RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    { Prof prof_("mbj_apply_rs_kernel", s); mbj_apply_rs_kernel<RS><<<g, 256, smem, s>>>(I.inv32, I.L.d, I.sz_dev, I.L.B, I.L.H, W.N, W.r, v, z, stop); }
    MU_CHECK_LAUNCH("mbj_apply_rs_kernel");
    return MUELLER_OK;
  }
  dim3 g(nblk(I.L.d, 8), I.L.nb, W.r);
  { Prof prof_("mbj_apply_b_kernel", s); mbj_apply_b_kernel<<<g, 256, 0, s>>>(I.inv32, I.L.d, I.sz_dev, I.L.B, I.L.H, W.N, v, z, stop); }
  MU_CHECK_LAUNCH("mbj_apply_b_kernel");
  return MUELLER_OK;
}

// norms of the r vectors of w (type VT) into dst (device, r doubles); mask optional
template <class VT>
static mueller_status lock_norms(const LockWork& W, const VT* w, double* dst, const int* mask,
                                 cudaStream_t s) {
  { Prof prof_("nrm2_b_kernel", s); nrm2_b_kernel<VT><<<dim3(W.G, W.r), 256, 0, s>>>(w, W.N, W.npart, W.G); }
  { Prof prof_("norm_finish_b_kernel", s); norm_finish_b_kernel<<<nblk(W.r, 64), 64, 0, s>>>(W.npart, W.G, W.r, mask, dst); }
  MU_CHECK_LAUNCH("lock_norms");
  return MUELLER_OK;
}

// inner GMRES on rhs32 (r unit-norm vectors) -> d32; tol relative to 1
static mueller_status lock_gmres(const InnerOp& I, LockWork& W, double tol, int maxit, int& iters,
                                 int& restarts, double* hbuf, std::vector<int>& active,
                                 cudaStream_t s) {
  const int64_t N = W.N;
  const int r = W.r, m = W.m, G = W.G;
  std::vector<int> kk(r), mask(r);
  std::vector<double> beta(r), bn(r, 1.0);
  mueller_status st = MUELLER_OK;
  MU_CUDA(cudaMemsetAsync(W.d32, 0, (size_t)r * N * 8, s));
  bool converged = false;
  for (int cycle = 0; iters < maxit && !converged; ++cycle) {
    // residual of the inner system: w = rhs - A d (d = 0 in the first cycle)
    if (cycle == 0) {
      MU_CUDA(cudaMemcpyAsync(W.W, W.rhs32, (size_t)r * N * 8, cudaMemcpyDeviceToDevice, s));
    } else {
      if ((st = lock_matvec(I, W, W.d32, W.W, s))) return st;
      { Prof prof_("resid_b_kernel", s); resid_b_kernel<<<nblk((int64_t)r * N, 256), 256, 0, s>>>(W.rhs32, W.W, (int64_t)r * N); }
    }
    for (int k = 0; k < r; ++k) mask[k] = active[k];
    MU_CUDA(cudaMemcpyAsync(W.mask, mask.data(), r * 4, cudaMemcpyHostToDevice, s));
    if ((st = lock_norms<float2>(W, W.W, W.beta, W.mask, s))) return st;
    MU_CUDA(cudaMemcpyAsync(hbuf, W.beta, r * 8, cudaMemcpyDeviceToHost, s));
    MU_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    for (int k = 0; k < r; ++k) {
      beta[k] = hbuf[k];
      if (active[k] && beta[k] <= tol) active[k] = 0;
      if (active[k]) any = true;
    }
    if (!any) break;
    for (int k = 0; k < r; ++k) mask[k] = active[k];
    MU_CUDA(cudaMemcpyAsync(W.mask, mask.data(), r * 4, cudaMemcpyHostToDevice, s));
    if ((st = lock_norms<float2>(W, W.W, W.beta, W.mask, s))) return st;
    { Prof prof_("scale_b_kernel", s); scale_b_kernel<float2, float2><<<dim3(nblk(N, 256), r), 256, 0, s>>>(W.W, N, W.beta, W.V); }
    { Prof prof_("set_first_b_kernel", s); set_first_b_kernel<<<nblk(r, 64), 64, 0, s>>>(W.g, m, r, W.beta); }
    MU_CUDA(cudaMemsetAsync(W.hacc, 0, (size_t)r * (m + 2) * 16, s));
    std::fill(kk.begin(), kk.end(), 0);
    int jlast = 0;
    if (r <= 128) {
      // Arnoldi steps queued ahead: the convergence test runs on the device
      // (arnoldi_tail_kernel sets the stop flag, after which every queued
      // kernel returns at once); the host reads the flags every kSync steps
      constexpr int kSync = 8;
      MU_CUDA(cudaMemsetAsync(W.kk, 0, (size_t)r * 4, s));
      MU_CUDA(cudaMemsetAsync(W.flags, 0, 3 * sizeof(int), s));
      const int* stop = W.flags;
      TailArgs ta;
      ta.V = W.V;
      ta.w = W.W;
      ta.N = N;
      ta.r = r;
      ta.m = m;
      ta.cs = W.tcs;
      ta.hacc = W.hacc;
      ta.Hm = W.Hm;
      ta.cs_ = W.cs;
      ta.sn = W.sn;
      ta.g = W.g;
      ta.res = W.res;
      ta.kk = W.kk;
      ta.active = W.mask;
      ta.bad = W.bad;
      ta.tol = tol;
      ta.stop = W.flags;
      ta.jstop = W.flags + 1;
      ta.ticket = (unsigned*)(W.flags + 8);
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3(W.tcs, r);
      lc.blockDim = dim3(256);
      lc.stream = s;
      cudaLaunchAttribute la[1];
      la[0].id = cudaLaunchAttributeClusterDimension;
      la[0].val.clusterDim.x = W.tcs;
      la[0].val.clusterDim.y = 1;
      la[0].val.clusterDim.z = 1;
      lc.attrs = la;
      lc.numAttrs = 1;
      int queued = 0, hf[3] = {0, 0, 0};
      for (int j = 0; j < m && iters + queued < maxit; ++j) {
        const float2* Vj = W.V + (int64_t)j * r * N;
        if ((st = lock_precond(I, W, Vj, W.Zt, s, stop))) return st;
        if ((st = lock_matvec(I, W, W.Zt, W.W, s, stop))) return st;
        ta.j = j;
        {
          Prof prof_("arnoldi_tail_kernel", s);
          MU_CUDA(cudaLaunchKernelEx(&lc, arnoldi_tail_kernel, ta));
        }
        ++queued;
        if ((j + 1) % kSync == 0 || j == m - 1 || iters + queued >= maxit) {
          MU_CUDA(cudaMemcpyAsync(hf, W.flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
          MU_CUDA(cudaStreamSynchronize(s));
          if (hf[0]) break;
        }
      }
      const int done = hf[0] ? hf[1] : queued;
      // every active right-hand side met the tolerance on its Arnoldi
      // estimate: the cycle's update ends the inner solve (the outer FP64
      // residual checks the result; a shortfall costs one more refinement)
      converged = hf[0] != 0;
      iters += done;
      jlast = done - 1;
      MU_CUDA(cudaMemcpyAsync(kk.data(), W.kk, (size_t)r * 4, cudaMemcpyDeviceToHost, s));
      MU_CUDA(cudaStreamSynchronize(s));
    } else {
      for (int j = 0; j < m && iters < maxit; ++j) {
        const float2* Vj = W.V + (int64_t)j * r * N;
        if ((st = lock_precond(I, W, Vj, W.Zt, s))) return st;
        if ((st = lock_matvec(I, W, W.Zt, W.W, s))) return st;
        for (int pass = 0; pass < 2; ++pass) {
          { Prof prof_("dots_b_kernel", s); dots_b_kernel<<<dim3(G, j + 1, r), 256, 0, s>>>(W.V, N, r, j + 1, m + 1, W.W, W.part, G); }
          { Prof prof_("orth_b_kernel", s); orth_b_kernel<<<dim3(nblk(N, 256), r), 256, 0, s>>>(W.V, N, r, j + 1, m + 1, W.part, G, W.W, W.hacc); }
        }
        if ((st = lock_norms<float2>(W, W.W, W.hn, nullptr, s))) return st;
        { Prof prof_("scale_b_kernel", s); scale_b_kernel<float2, float2><<<dim3(nblk(N, 256), r), 256, 0, s>>>(W.W, N, W.hn, W.V + (int64_t)(j + 1) * r * N); }
        { Prof prof_("givens_b_kernel", s); givens_b_kernel<<<nblk(r, 64), 64, 0, s>>>(j, m, r, W.hacc, W.hn, W.Hm, W.cs, W.sn, W.g, W.res); }
        MU_CHECK_LAUNCH("lockstep Arnoldi step");
        ++iters;
        jlast = j;
        MU_CUDA(cudaMemcpyAsync(hbuf, W.res, r * 8, cudaMemcpyDeviceToHost, s));
        MU_CUDA(cudaStreamSynchronize(s));
        bool all = true;
        for (int k = 0; k < r; ++k) {
          if (!active[k]) continue;
          if (kk[k] == 0 && (hbuf[k] <= tol || !(hbuf[k] == hbuf[k]))) kk[k] = j + 1;
          if (kk[k] == 0) all = false;
        }
        if (all) {
          converged = true;
          break;
        }
      }
    }
    int kmax = 0;
    for (int k = 0; k < r; ++k) {
      if (!active[k]) kk[k] = 0;
      else if (kk[k] == 0) kk[k] = jlast + 1;
      kmax = std::max(kmax, kk[k]);
    }
    MU_CUDA(cudaMemcpyAsync(W.kk, kk.data(), r * 4, cudaMemcpyHostToDevice, s));
    { Prof prof_("backsub_b_kernel", s); backsub_b_kernel<<<nblk(r, 64), 64, 0, s>>>(m, r, W.kk, W.Hm, W.g, W.y); }
    { Prof prof_("combine_b_kernel", s); combine_b_kernel<<<dim3(nblk(N, 256), r), 256, 0, s>>>(W.V, N, r, kmax, m, W.y, W.U); }
    if ((st = lock_precond(I, W, W.U, W.Zt, s))) return st;
    { Prof prof_("axpy_b_kernel<float2>", s); axpy_b_kernel<float2><<<dim3(nblk(N, 256), r), 256, 0, s>>>(W.d32, W.Zt, N, nullptr); }
    MU_CHECK_LAUNCH("lockstep update");
    ++restarts;
  }
  return st;
}

static mueller_status solve_lockstep(const mueller_operator* op, const double2* B, double2* X,
                                     int r, const mueller_solver_opts* o, mueller_solve_info* info,
                                     char* p, cudaStream_t s) {
  const mueller_mesh* m = op->mesh;
  const int64_t N = 4 * m->nn;
  const int mres = std::max(1, std::min(120, (int)o->restart));
  InnerOp I;
  I.op = op;
  I.near32 = nullptr;
  I.inv32 = op->precond_dev ? (const float2*)op->precond_dev : nullptr;
  I.sz_dev = nullptr;
  if (op->precond_dev) {
    I.L = layout(N, op->block);
    I.sz_dev = precond_sizes(op, I.L);
  }
  LockWork W = carve_lock(p, N, r, mres, op->near_dev ? m->nnzb : 0);
  if (op->near_dev && m->nnzb > 0) {
    // the inner products read the near blocks rounded to complex64 once
    const int64_t cnt = m->nnzb * 16;
    { Prof prof_("c128_to_c64_kernel", s); c128_to_c64_kernel<<<nblk(cnt, 256), 256, 0, s>>>((const double2*)op->near_dev, W.near32, cnt); }
    MU_CHECK_LAUNCH("near blocks to complex64");
    I.near32 = W.near32;
  }
  double* hbuf = nullptr;
  MU_CUDA(cudaMallocHost((void**)&hbuf, (size_t)std::max(8, 2 * r) * sizeof(double)));
  MU_CUDA(cudaMemsetAsync(W.flags, 0, 64 * sizeof(int), s));
  MU_CUDA(cudaMemsetAsync(W.bad, 0, (size_t)r * sizeof(int), s));
  mueller_status st = MUELLER_OK;
  const int maxref = o->max_refine > 0 ? o->max_refine : 20;
  const double itol = o->inner_tol > 0 ? o->inner_tol : 1e-5;
  std::vector<double> bn(r), rn(r);
  std::vector<int> active(r, 1), bad(r, 0);
  int it_left = o->maxit;
  if (!o->warm_start) MU_CUDA(cudaMemsetAsync(X, 0, (size_t)r * N * 16, s));
  if ((st = lock_norms<double2>(W, B, W.bn, nullptr, s))) goto out;
  MU_CUDA(cudaMemcpyAsync(hbuf, W.bn, r * 8, cudaMemcpyDeviceToHost, s));
  MU_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < r; ++k) bn[k] = hbuf[k];
  for (int ref = 0; ref <= maxref; ++ref) {
    // FP64 residual on the stored operator (r = b while x is still zero)
    if (ref == 0 && !o->warm_start) {
      MU_CUDA(cudaMemcpyAsync(W.r64, B, (size_t)r * N * 16, cudaMemcpyDeviceToDevice, s));
    } else {
      if ((st = op_matvec(op, X, W.y64, r, nullptr, 0, s))) goto out;
      { Prof prof_("residual_kernel", s); residual_kernel<<<nblk((int64_t)r * N, 256), 256, 0, s>>>(B, W.y64, W.r64, (int64_t)r * N); }
    }
    if ((st = lock_norms<double2>(W, W.r64, W.rn, nullptr, s))) goto out;
    MU_CUDA(cudaMemcpyAsync(hbuf, W.rn, r * 8, cudaMemcpyDeviceToHost, s));
    MU_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    double worst = 0;
    for (int k = 0; k < r; ++k) {
      rn[k] = hbuf[k];
      const double rel = bn[k] > 0 ? rn[k] / bn[k] : 0.0;
      if (!(rel == rel) || rel == HUGE_VAL) {  // NaN or Inf: that right-hand side stops
        bad[k] = 1;
        active[k] = 0;
        continue;
      }
      worst = std::max(worst, rel);
      active[k] = rel > o->tol;
      any |= active[k] != 0;
    }
    info->relres = worst;
    if (!any || it_left <= 0 || ref == maxref) break;
    // inner system A d = r / ||r|| in complex64 for the active right-hand sides
    { Prof prof_("scale_b_kernel", s); scale_b_kernel<double2, float2><<<dim3(nblk(N, 256), r), 256, 0, s>>>(W.r64, N, W.rn, W.rhs32); }
    int it = 0, rs = 0;
    // each refinement only has to bring the worst residual down to tol
    st = lock_gmres(I, W, std::max(itol, 0.5 * o->tol / std::max(worst, 1e-300)), it_left, it, rs,
                    hbuf, active, s);
    if (st) goto out;
    it_left -= it;
    info->iters += it * r;
    info->restarts += rs;
    info->refinements += 1;
    // x += ||r|| d
    MU_CUDA(cudaMemcpyAsync(W.alpha, W.rn, r * 8, cudaMemcpyDeviceToDevice, s));
    { Prof prof_("axpy_b_kernel<double2>", s); axpy_b_kernel<double2><<<dim3(nblk(N, 256), r), 256, 0, s>>>(X, W.d32, N, W.alpha); }
    MU_CHECK_LAUNCH("refinement update");
  }
  for (int k = 0; k < r; ++k)
    if (!bad[k] && (bn[k] == 0 || rn[k] / bn[k] <= o->tol)) info->converged++;
  if (r >= 2 && !st) st = mrhs_check_error(W.mwork, N, r, s);
  if (!st) {
    // right-hand sides whose Arnoldi estimate or FP64 residual was not a number
    std::vector<int> dbad(r, 0);
    MU_CUDA(cudaMemcpyAsync(dbad.data(), W.bad, (size_t)r * sizeof(int), cudaMemcpyDeviceToHost, s));
    MU_CUDA(cudaStreamSynchronize(s));
    int nbad = 0, first = -1;
    for (int k = 0; k < r; ++k)
      if (bad[k] || dbad[k]) {
        ++nbad;
        if (first < 0) first = k;
      }
    if (nbad) {
      set_error(std::to_string(nbad) + " right-hand side(s) produced a NaN or infinite residual "
                "(first: right-hand side " + std::to_string(first) + "); the others are solved");
      st = MUELLER_ERR_NAN;
    }
  }
out:
  cudaFreeHost(hbuf);
  return st;
}

size_t solve_work(const mueller_operator* op, int r, const mueller_solver_opts* o) {
  (void)r;
  const int64_t N = 4 * op->mesh->nn;
  if (o->mode == MUELLER_SOLVE_DENSE_LU) {
    return (size_t)N * N * 16 + (size_t)N * 4 + 512 + (size_t)N * r * 16 + 256;
  }
  const int m = std::max(1, (int)o->restart);
  size_t b = 0;
  if (o->mode == MUELLER_SOLVE_GMRES && op->dtype == MUELLER_C128) {
    b = gmres_bytes(N, m, 16);
  } else {
    b = lock_bytes(N, r, std::min(120, m), op->near_dev ? op->mesh->nnzb : 0);
  }
  return b + 4096;
}

mueller_status solve(const mueller_operator* op, const void* Bv, void* Xv, int r,
                     const mueller_solver_opts* o, mueller_solve_info* info, void* work,
                     size_t work_bytes, cudaStream_t s) {
  const mueller_mesh* m = op->mesh;
  const int64_t N = 4 * m->nn;
  *info = mueller_solve_info{0, 0, 0, 0, 0.0, 0.0};
  const size_t need = solve_work(op, r, o);
  void* own = nullptr;
  if (!work) {
    MU_CUDA(cudaMallocAsync(&own, need, s));
    work = own;
  }
  (void)work_bytes;
  char* p = (char*)work;
  mueller_status st = MUELLER_OK;
  const double2* B = (const double2*)Bv;
  double2* X = (double2*)Xv;
  if (o->mode == MUELLER_SOLVE_DENSE_LU) {
    // LU of a copy of Z, then the row swaps and the two triangular solves on
    // the r right-hand sides stored as an N x r column block T.
    double2* A = (double2*)p;
    int32_t* piv = (int32_t*)(A + (size_t)N * N);
    int32_t* sz_dev = piv + N;
    int32_t* status = sz_dev + 4;
    double2* T = (double2*)(((uintptr_t)(status + 4) + 255) & ~(uintptr_t)255);
    int32_t nsz = (int32_t)N;
    cudaError_t e = cudaMemcpy2DAsync(A, N * 16, op->Z_dev, op->ldz * 16, N * 16, N,
                                      cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sz_dev, &nsz, 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 4, s);
    if (e != cudaSuccess) st = cuda_fail(e, "dense LU setup");
    if (!st) st = batched_lu_inverse<double2>(A, N, 1, sz_dev, piv, status, nullptr, s);
    if (!st) {
      { Prof prof_("transpose_rhs_kernel", s); transpose_rhs_kernel<<<nblk((int64_t)N * r, 256), 256, 0, s>>>(B, T, N, r, 0); }
      { Prof prof_("permute_rows_kernel", s); permute_rows_kernel<<<nblk(r, 64), 64, 0, s>>>(T, N, r, piv); }
      for (int k0 = 0; k0 < N; k0 += NBK) {
        { Prof prof_("trsm_tile_kernel", s); trsm_tile_kernel<double2, NBK><<<dim3(nblk(r, 128), 1), 128, 0, s>>>(A, T, N, r, 0, sz_dev, k0, NBK, 0, r, 0); }
        const int64_t below = N - (k0 + NBK);
        if (below > 0)
          { Prof prof_("gemm_update_kernel", s); gemm_update_kernel<double2, NBK><<<dim3(nblk(r, 64), nblk(below, 64), 1), 256, 0, s>>>(
              A, T, T, N, r, 0, sz_dev, k0, k0 + NBK, -1, 0, r); }
      }
      const int64_t ntile = (N + NBK - 1) / NBK;
      for (int64_t t = ntile - 1; t >= 0; --t) {
        const int k0 = (int)(t * NBK);
        { Prof prof_("trsm_tile_kernel", s); trsm_tile_kernel<double2, NBK><<<dim3(nblk(r, 128), 1), 128, 0, s>>>(A, T, N, r, 0, sz_dev, k0, NBK, 0, r, 1); }
        if (k0 > 0)
          { Prof prof_("gemm_update_kernel", s); gemm_update_kernel<double2, NBK><<<dim3(nblk(r, 64), nblk(k0, 64), 1), 256, 0, s>>>(
              A, T, T, N, r, 0, sz_dev, k0, 0, k0, 0, r); }
      }
      { Prof prof_("transpose_rhs_kernel", s); transpose_rhs_kernel<<<nblk((int64_t)N * r, 256), 256, 0, s>>>(T, X, N, r, 1); }
      e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_fail(e, "dense LU solve");
    }
    int32_t hst = 0;
    if (!st) {
      e = cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_fail(e, "dense LU status");
      if (!st && hst) {
        set_error("matrix is singular to working precision");
        st = MUELLER_ERR_SINGULAR_BLOCK;
      }
    }
    if (!st) {
      info->converged = r;
      info->relres = 0.0;
    }
    if (own) cudaFreeAsync(own, s);
    if (!st) MU_CUDA(cudaStreamSynchronize(s));
    return st;
  }
  InnerOp I;
  I.op = op;
  I.near32 = nullptr;
  I.inv32 = nullptr;
  I.sz_dev = nullptr;
  if (op->precond_dev) {
    I.L = layout(N, op->block);
    I.sz_dev = precond_sizes(op, I.L);
  }
  const int mres = std::max(1, (int)o->restart);
  if (o->mode == MUELLER_SOLVE_GMRES && op->dtype == MUELLER_C128) {
    I.precision = 0;
    GmresWork W = carve_gmres<double2>(p, N, mres);
    MU_CUDA(cudaMallocHost((void**)&W.hs, 8 * sizeof(double)));
    int it_left = o->maxit;
    for (int k = 0; k < r && !st; ++k) {
      const double2* b = B + (int64_t)k * N;
      double2* x = X + (int64_t)k * N;
      if (!o->warm_start) MU_CUDA(cudaMemsetAsync(x, 0, N * 16, s));
      int it = 0, rs = 0;
      double rel = 0;
      st = gmres<double2>(I, W, b, x, o->tol, it_left, it, rs, rel, s);
      info->iters += it;
      info->restarts += rs;
      info->relres = std::max(info->relres, rel);
      if (rel <= o->tol) info->converged++;
    }
    cudaFreeHost(W.hs);
  } else {
    st = solve_lockstep(op, B, X, r, o, info, p, s);
  }
  if (own) cudaFreeAsync(own, s);
  if (!st) MU_CUDA(cudaStreamSynchronize(s));
  if (!st && info->converged < r) {
    set_error("GMRES did not reach the tolerance within maxit");
    return MUELLER_ERR_NOT_CONVERGED;
  }
  return st;
}

}  // namespace mu
