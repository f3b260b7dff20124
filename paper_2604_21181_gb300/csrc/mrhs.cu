// Multi-right-hand-side product Y = Z X on the tcgen05 tensor cores.  Two
// kernels: mrhs_zn_kernel (r <= 64, Z on the MMA's N side, described before
// it) and mrhs_tf32_kernel (any r up to 128, Z on the M side), described here.
//
// Z is the complex64 N x N matrix of the mixed operator (row-major, ldz), X
// and Y hold r complex64 vectors.  The complex product is a real GEMM:
//   Y_real[i][2s + 0] = sum_j  zr xr - zi xi,  Y_real[i][2s + 1] = sum_j zr xi + zi xr
// i.e. the rows of Z read as real vectors of length 2N (re, im interleaved)
// against B' (2r x 2N, K-major) with rows  2s: ( xr_j, -xi_j )  and
// 2s+1: ( xi_j, xr_j ).  The MMA kind is tf32 with FP32 accumulation in
// TMEM; each operand is split into a TF32 head (its top 19 bits, which is
// what the tensor core reads from an FP32 word) and the exact remainder
// (x = hi + lo), and hi*hi + hi*lo + lo*hi are accumulated, which brings the
// product to FP32 accuracy.
//
// CTA (192 threads): warp 0 issues the TMA loads of the Z tile (128 rows x
// 32 floats) and of the B' head / remainder tiles; warps 2-5 split the Z
// tile into head and remainder in shared memory and, at the end, read the
// accumulator from TMEM; warp 1 allocates TMEM and one of its threads issues
// the MMAs.  Each tcgen05.mma of kind tf32 with M = 128 costs about the same
// whatever its N (up to 256), so the number of MMAs per Z byte bounds the
// kernel: where 2 nprime <= 256 the head meets [B'hi; B'lo] in one MMA of
// N = 2 nprime (the two halves are adjacent in shared memory), which makes
// two MMAs per K step instead of three.  Stages are handed over with
// mbarriers; every wait is bounded (in time) and reports a timeout through an
// error word instead of hanging.  K is split
// across CTAs (split-K) so that the grid fills the 152 SMs; the partial sums
// meet in Y by atomic additions.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace mu {
namespace {

constexpr int BM = 128;   // rows of Z per CTA (MMA M)
constexpr int BK = 32;    // floats per K tile = one 128-byte swizzle row
constexpr int MMA_K = 8;  // tf32 elements per tcgen05.mma
constexpr int THREADS = 192;
constexpr uint32_t WAIT_LIMIT = 1u << 30;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s
constexpr int SMEM_BUDGET = 224 * 1024;      // stages + barriers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: false after about WAIT_NS nanoseconds (or WAIT_LIMIT polls)
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > WAIT_NS) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// UMMA shared-memory descriptor of a K-major tile in the 128-byte swizzle
// layout written by TMA: 8-row groups of 1024 bytes (stride byte offset),
// descriptor version 1, layout type SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 16 consecutive TMEM columns of this thread's lane -> v[0..15]
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

struct MrhsArgs {
  int64_t N;        // rows of Z (= columns / 2 of the real view)
  int nprime;       // padded 2r (MMA N), multiple of 16
  int r;            // right-hand sides
  int ktiles;       // K tiles of the real view (2N / 32 rounded up)
  int kchunk;       // K tiles per CTA (split-K)
  int stages;
  int stacked;      // 1: the head meets [B'hi; B'lo] in one MMA of N = 2 nprime
  uint32_t tmem_cols;
  float* Y;         // complex64 r x N, accumulated (atomic adds)
  int* err;         // error word
  const int* stop;  // nonzero: skip the product (solver converged); may be null
};

// dynamic shared memory: [stages][A 16 KB | Alo 16 KB | Bhi | Blo] + barriers
__global__ void __launch_bounds__(THREADS, 1)
    mrhs_tf32_kernel(const __grid_constant__ CUtensorMap mapZ,
                     const __grid_constant__ CUtensorMap mapBhi,
                     const __grid_constant__ CUtensorMap mapBlo, MrhsArgs a) {
  if (a.stop && *a.stop) return;  // uniform: before any barrier or TMEM allocation
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t bbytes = (uint32_t)a.nprime * BK * 4;
  const uint32_t stage_bytes = 2u * BM * BK * 4 + 2u * bbytes;
  uint64_t* full = (uint64_t*)(base + a.stages * stage_bytes);
  uint64_t* split = full + a.stages;
  uint64_t* empty = split + a.stages;
  uint64_t* accf = empty + a.stages;
  uint32_t* tmem_slot = (uint32_t*)(accf + 1);
  volatile int* bail = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int kt0 = blockIdx.y * a.kchunk;
  const int kt1 = min(a.ktiles, kt0 + a.kchunk);
  const int nk = kt1 - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&split[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *bail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  auto A_of = [&](int s) { return base + (size_t)s * stage_bytes; };
  auto Alo_of = [&](int s) { return base + (size_t)s * stage_bytes + BM * BK * 4; };
  auto Bhi_of = [&](int s) { return base + (size_t)s * stage_bytes + 2 * BM * BK * 4; };
  auto Blo_of = [&](int s) { return base + (size_t)s * stage_bytes + 2 * BM * BK * 4 + bbytes; };

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nk; ++it) {
        const int s = it % a.stages;
        const uint32_t ph = (it / a.stages) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1) || *bail) {
          atomicExch(a.err, 1);
          *bail = 1;
          break;
        }
        mbar_expect_tx(&full[s], stage_bytes - BM * BK * 4);
        const int kc = (kt0 + it) * BK;
        tma_load_2d(A_of(s), &mapZ, &full[s], kc, (int)m0);
        tma_load_2d(Bhi_of(s), &mapBhi, &full[s], kc, 0);
        tma_load_2d(Blo_of(s), &mapBlo, &full[s], kc, 0);
        ++issued;
      }
      // wait for the copies still in flight before the CTA may exit
      for (int it = max(0, issued - a.stages); it < issued; ++it)
        mbar_wait(&full[it % a.stages], (it / a.stages) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t id0 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BM >> 4) << 24);
      const uint32_t idn = id0 | ((uint32_t)(a.nprime >> 3) << 17);
      const uint32_t id2n = id0 | ((uint32_t)(a.nprime >> 2) << 17);
      for (int it = 0; it < nk; ++it) {
        const int s = it % a.stages;
        const uint32_t ph = (it / a.stages) & 1;
        if (!mbar_wait(&split[s], ph) || *bail) {
          atomicExch(a.err, 2);
          *bail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint64_t dA = sw128_desc(smem_u32(A_of(s)));
        const uint64_t dAl = sw128_desc(smem_u32(Alo_of(s)));
        const uint64_t dB = sw128_desc(smem_u32(Bhi_of(s)));
        const uint64_t dBl = sw128_desc(smem_u32(Blo_of(s)));
#pragma unroll
        for (int k = 0; k < BK / MMA_K; ++k) {
          const uint64_t off = (uint64_t)((k * MMA_K * 4) >> 4);  // 32 bytes per K step
          const uint32_t acc = (it > 0 || k > 0) ? 1u : 0u;
          if (a.stacked) {
            // B'hi and B'lo are adjacent in shared memory: one descriptor
            // covers both, the MMA writes hi*B'hi | hi*B'lo side by side
            mma_tf32(tmem, dA + off, dB + off, id2n, acc);
            mma_tf32(tmem, dAl + off, dB + off, idn, 1u);
          } else {
            mma_tf32(tmem, dA + off, dB + off, idn, acc);
            mma_tf32(tmem, dA + off, dBl + off, idn, 1u);
            mma_tf32(tmem, dAl + off, dB + off, idn, 1u);
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(accf);
    }
  } else {
    // ---------------- split Z tiles into TF32 head and remainder
    const int t = threadIdx.x - 64;  // 0..127
    for (int it = 0; it < nk; ++it) {
      const int s = it % a.stages;
      const uint32_t ph = (it / a.stages) & 1;
      if (!mbar_wait(&full[s], ph) || *bail) {
        atomicExch(a.err, 3);
        *bail = 1;
        break;
      }
      // the tensor core reads the raw FP32 tile as its TF32 head (the low 13
      // mantissa bits are ignored); only the exact remainder is written
      const uint4* __restrict__ A4 = (const uint4*)A_of(s);
      uint4* __restrict__ Al4 = (uint4*)Alo_of(s);
      uint4 v[BM * BK / 4 / 128];
#pragma unroll
      for (int e = 0; e < BM * BK / 4 / 128; ++e) v[e] = A4[t + 128 * e];
#pragma unroll
      for (int e = 0; e < BM * BK / 4 / 128; ++e) {
        uint4 o;
        o.x = __float_as_uint(__uint_as_float(v[e].x) - __uint_as_float(v[e].x & 0xFFFFE000u));
        o.y = __float_as_uint(__uint_as_float(v[e].y) - __uint_as_float(v[e].y & 0xFFFFE000u));
        o.z = __float_as_uint(__uint_as_float(v[e].z) - __uint_as_float(v[e].z & 0xFFFFE000u));
        o.w = __float_as_uint(__uint_as_float(v[e].w) - __uint_as_float(v[e].w & 0xFFFFE000u));
        Al4[t + 128 * e] = o;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&split[s]);
    }
    // ---------------- epilogue: TMEM -> Y (atomic adds of the partial sums)
    const bool ok = mbar_wait(accf, 0);
    if (!ok) atomicExch(a.err, 4);
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int64_t row = m0 + quarter * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int c0 = 0; c0 < a.nprime; c0 += 16) {
      uint32_t v[16], w[16];
      tmem_ld16(lane_addr + (uint32_t)c0, v);
      if (a.stacked) tmem_ld16(lane_addr + (uint32_t)(a.nprime + c0), w);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (ok && row < a.N) {
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          const int sidx = (c0 + q) >> 1;
          float re = __uint_as_float(v[q]), im = __uint_as_float(v[q + 1]);
          if (a.stacked) {  // hi*B'hi + lo*B'hi  +  hi*B'lo
            re += __uint_as_float(w[q]);
            im += __uint_as_float(w[q + 1]);
          }
          if (sidx < a.r)
            atomicAdd(reinterpret_cast<float2*>(a.Y) + (int64_t)sidx * a.N + row,
                      make_float2(re, im));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}

// ---------------------------------------------------------------------------
// The same product with Z on the N side of the MMA: D (M = 128 lanes: rows of
// X' = [B'hi; B'lo] stacked, or one of them) x (N = 256 columns: Z rows).  A
// tcgen05 MMA costs about the same for any N up to 256, so one MMA now covers
// 256 Z rows instead of 128.  K tiles are 16 floats (64-byte rows, 64-byte
// swizzle) so that five stages of {Z 16 KB, Z remainder 16 KB, X' 8 KB} fit.
// Stacked (2 nprime <= 128): per K step D += X'[hi;lo] Zhi + X'[hi;lo] Zlo,
// lanes c and nprime + c both add into output component c.  Unstacked
// (nprime <= 128): D += X'hi Zhi + X'lo Zhi + X'hi Zlo.
constexpr int ZN = 256;   // Z rows per CTA (MMA N)
constexpr int ZBK = 16;   // floats per K tile (64 bytes)

// UMMA descriptor of a K-major tile in the 64-byte swizzle layout: 8-row
// groups of 512 bytes, layout type SWIZZLE_64B.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

struct ZnArgs {
  int64_t N;
  int nprime, r, ktiles, kchunk, stages, stacked;
  float* Y;  // complex64 r x N, accumulated (atomic adds of the real parts)
  int* err;
  const int* stop;  // nonzero: skip the product (solver converged); may be null
  // Z11 = -Z00 (three quarters of Z read), stacked with 4 nprime <= 128:
  // mirror 1: the Z rows of the upper half (Z00 | Z01, K over 2N) against
  //   A = [X'(k); X'(k + N)] for k < N and [X'(k); 0] beyond, lanes
  //   [0, 2 nprime) -> rows i, lanes [2 nprime, 4 nprime) -> -(rows H + i);
  // mirror 2: the Z rows of the lower half (Z10 only, K over N) against
  //   A = [X'(k); -], lanes [0, 2 nprime) -> rows H + i.
  // A is then loaded as two boxes of 2 nprime rows (box rows abox).
  int mirror;
  int64_t H;
  int xoob;  // an aligned K coordinate beyond the operand: the box reads zeros
};

// dynamic shared memory: [stages][Z 16 KB | Zlo 16 KB | A0 8 KB | A1 8 KB (unstacked)]
__global__ void __launch_bounds__(THREADS, 1)
    mrhs_zn_kernel(const __grid_constant__ CUtensorMap mapZ,
                   const __grid_constant__ CUtensorMap mapA0,
                   const __grid_constant__ CUtensorMap mapA1, ZnArgs a) {
  if (a.stop && *a.stop) return;  // uniform: before any barrier or TMEM allocation
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr uint32_t ZB = ZN * ZBK * 4;   // 16 KB
  constexpr uint32_t AB = BM * ZBK * 4;   // 8 KB
  const uint32_t stage_bytes = 2 * ZB + (a.stacked ? 1 : 2) * AB;
  uint64_t* full = (uint64_t*)(base + (size_t)a.stages * stage_bytes);
  uint64_t* split = full + a.stages;
  uint64_t* empty = split + a.stages;
  uint64_t* accf = empty + a.stages;
  uint32_t* tmem_slot = (uint32_t*)(accf + 1);
  volatile int* bail = (volatile int*)(tmem_slot + 1);
  const uint32_t half_box = (uint32_t)(2 * a.nprime) * ZBK * 4;  // bytes of one A half (mirror)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.x * ZN;
  const int kt0 = blockIdx.y * a.kchunk;
  const int nk = min(a.ktiles, kt0 + a.kchunk) - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&split[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *bail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  auto Z_of = [&](int s) { return base + (size_t)s * stage_bytes; };
  auto Zlo_of = [&](int s) { return base + (size_t)s * stage_bytes + ZB; };
  auto A0_of = [&](int s) { return base + (size_t)s * stage_bytes + 2 * ZB; };
  auto A1_of = [&](int s) { return base + (size_t)s * stage_bytes + 2 * ZB + AB; };

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nk; ++it) {
        const int s = it % a.stages;
        if (!mbar_wait(&empty[s], ((it / a.stages) & 1) ^ 1) || *bail) {
          atomicExch(a.err, 1);
          *bail = 1;
          break;
        }
        const int kc = (kt0 + it) * ZBK;
        if (a.mirror) {
          // two A boxes of 2 nprime rows: X'(kc) and, upper half only,
          // X'(kc + N) below it (zeros for the Z01 columns, kc >= N)
          mbar_expect_tx(&full[s], ZB + (a.mirror == 1 ? 2 : 1) * half_box);
          tma_load_2d(Z_of(s), &mapZ, &full[s], kc, (int)n0);
          tma_load_2d(A0_of(s), &mapA1, &full[s], kc, 0);
          if (a.mirror == 1)
            tma_load_2d(A0_of(s) + half_box, &mapA1, &full[s],
                        kc < (int)a.N ? kc + (int)a.N : a.xoob, 0);
        } else {
          mbar_expect_tx(&full[s], ZB + (a.stacked ? 1 : 2) * AB);
          tma_load_2d(Z_of(s), &mapZ, &full[s], kc, (int)n0);
          tma_load_2d(A0_of(s), &mapA0, &full[s], kc, 0);
          if (!a.stacked) tma_load_2d(A1_of(s), &mapA1, &full[s], kc, 0);
        }
        ++issued;
      }
      for (int it = max(0, issued - a.stages); it < issued; ++it)
        mbar_wait(&full[it % a.stages], (it / a.stages) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(ZN >> 3) << 17) |
                             ((uint32_t)(BM >> 4) << 24);
      for (int it = 0; it < nk; ++it) {
        const int s = it % a.stages;
        if (!mbar_wait(&split[s], (it / a.stages) & 1) || *bail) {
          atomicExch(a.err, 2);
          *bail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint64_t dZ = sw64_desc(smem_u32(Z_of(s)));
        const uint64_t dZl = sw64_desc(smem_u32(Zlo_of(s)));
        const uint64_t dA0 = sw64_desc(smem_u32(A0_of(s)));
        const uint64_t dA1 = sw64_desc(smem_u32(A1_of(s)));
#pragma unroll
        for (int k = 0; k < ZBK / MMA_K; ++k) {
          const uint64_t off = (uint64_t)((k * MMA_K * 4) >> 4);  // 32 bytes per K step
          mma_tf32(tmem, dA0 + off, dZ + off, idesc, (it > 0 || k > 0) ? 1u : 0u);
          if (!a.stacked) mma_tf32(tmem, dA1 + off, dZ + off, idesc, 1u);
          mma_tf32(tmem, dA0 + off, dZl + off, idesc, 1u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(accf);
    }
  } else if (warp < 6) {
    // ---------------- Z remainder (element-wise: same swizzled offsets)
    const int t = threadIdx.x - 64;  // 0..127
    for (int it = 0; it < nk; ++it) {
      const int s = it % a.stages;
      if (!mbar_wait(&full[s], (it / a.stages) & 1) || *bail) {
        atomicExch(a.err, 3);
        *bail = 1;
        break;
      }
      const uint4* __restrict__ Z4 = (const uint4*)Z_of(s);
      uint4* __restrict__ L4 = (uint4*)Zlo_of(s);
      constexpr int PER = ZB / 16 / 128;  // 8
      uint4 v[PER];
#pragma unroll
      for (int e = 0; e < PER; ++e) v[e] = Z4[t + 128 * e];
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        uint4 o;
        o.x = __float_as_uint(__uint_as_float(v[e].x) - __uint_as_float(v[e].x & 0xFFFFE000u));
        o.y = __float_as_uint(__uint_as_float(v[e].y) - __uint_as_float(v[e].y & 0xFFFFE000u));
        o.z = __float_as_uint(__uint_as_float(v[e].z) - __uint_as_float(v[e].z & 0xFFFFE000u));
        o.w = __float_as_uint(__uint_as_float(v[e].w) - __uint_as_float(v[e].w & 0xFFFFE000u));
        L4[t + 128 * e] = o;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&split[s]);
    }
    // ---------------- epilogue: lane l of D = component l (mod nprime if stacked)
    const bool ok = mbar_wait(accf, 0);
    if (!ok) atomicExch(a.err, 4);
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int quarter = warp & 3;
    const int l = quarter * 32 + lane;
    int comp, nlanes;
    float sgn = 1.f;
    int64_t rows = a.N, roff = 0;  // output rows roff + (n0 + ...), below rows
    if (a.mirror) {
      const int np2 = 2 * a.nprime;
      const int ll = l % np2;
      comp = ll >= a.nprime ? ll - a.nprime : ll;
      nlanes = a.mirror == 1 ? 2 * np2 : np2;
      rows = a.H;
      if (a.mirror == 2 || l >= np2) roff = a.H;
      if (a.mirror == 1 && l >= np2) sgn = -1.f;  // Z11 = -Z00
    } else {
      comp = a.stacked && l >= a.nprime ? l - a.nprime : l;
      nlanes = a.stacked ? 2 * a.nprime : a.nprime;
    }
    const bool valid = ok && l < nlanes && (comp >> 1) < a.r;
    float* yb = a.Y + 2 * ((int64_t)(comp >> 1) * a.N + roff) + (comp & 1);
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int c0 = 0; c0 < ZN; c0 += 16) {
      uint32_t v[16];
      tmem_ld16(lane_addr + (uint32_t)c0, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (valid) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int64_t row = n0 + c0 + e;
          if (row < rows) atomicAdd(yb + 2 * row, sgn * __uint_as_float(v[e]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
  }
}

// B' head / remainder (nprime x 2N, K-major) from X (complex64 r x N)
__global__ void build_bprime_kernel(const float2* __restrict__ X, int64_t N, int r, int nprime,
                                    float* __restrict__ Bhi, float* __restrict__ Blo,
                                    const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nprime * N) return;
  const int row = (int)(t / N);
  const int64_t j = t % N;
  float v0 = 0.f, v1 = 0.f;
  const int s = row >> 1;
  if (s < r) {
    const float2 x = X[(int64_t)s * N + j];
    if ((row & 1) == 0) {
      v0 = x.x;
      v1 = -x.y;
    } else {
      v0 = x.y;
      v1 = x.x;
    }
  }
  const float h0 = __uint_as_float(__float_as_uint(v0) & 0xFFFFE000u);
  const float h1 = __uint_as_float(__float_as_uint(v1) & 0xFFFFE000u);
  const int64_t o = (int64_t)row * 2 * N + 2 * j;
  Bhi[o] = h0;
  Bhi[o + 1] = h1;
  Blo[o] = v0 - h0;
  Blo[o + 1] = v1 - h1;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::mutex mu_;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lk(mu_);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool make_map(CUtensorMap* map, const void* ptr, uint64_t inner, uint64_t outer,
              uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
              CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

size_t mrhs_work_bytes(int64_t N, int r) {
  const int64_t np = cdiv(2 * r, 16) * 16;
  return (size_t)2 * np * 2 * N * sizeof(float) + 512 + 256;
}

// Y (complex64 r x N) = Z (complex64, N x ldz) X (complex64 r x N); work:
// mrhs_work_bytes(N, r) bytes of device scratch.
mueller_status mrhs_matvec_c64(const void* Z, int64_t N, int64_t ldz, const void* X, void* Y,
                               int r, void* work, cudaStream_t s, const int* stop, int mirrored) {
  if (r < 1 || r > 128) {
    set_error("tensor-core product supports 1..128 right-hand sides");
    return MUELLER_ERR_INVALID_ARG;
  }
  if ((ldz & 1) || ((uintptr_t)Z & 15)) {
    set_error("tensor-core product needs an even ldz and a 16-byte aligned Z");
    return MUELLER_ERR_INVALID_ARG;
  }
  const int nprime = (int)cdiv(2 * r, 16) * 16;
  const int stacked = 2 * nprime <= 256 ? 1 : 0;
  const int acc_cols = stacked ? 2 * nprime : nprime;
  uint32_t tmem_cols = 32;
  while ((int)tmem_cols < acc_cols) tmem_cols <<= 1;
  float* Bhi = (float*)work;
  float* Blo = Bhi + (size_t)nprime * 2 * N;
  int* err = (int*)(Blo + (size_t)nprime * 2 * N);
  MU_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  MU_CUDA(cudaMemsetAsync(Y, 0, (size_t)r * N * 8, s));
  {
    Prof prof_("build_bprime_kernel", s);
    build_bprime_kernel<<<(unsigned)cdiv((int64_t)nprime * N, 256), 256, 0, s>>>(
        (const float2*)X, N, r, nprime, Bhi, Blo, stop);
  }
  MU_CHECK_LAUNCH("build_bprime_kernel");
  if (mirrored && 4 * nprime <= BM && (N & 1) == 0) {
    // Z11 = -Z00: the upper rows read Z00 once for both diagonal blocks
    const int64_t H = N / 2;
    CUtensorMap mZt, mZb, mA;
    if (!make_map(&mZt, Z, (uint64_t)2 * N, (uint64_t)H, (uint64_t)ldz * 8, ZBK, ZN,
                  CU_TENSOR_MAP_SWIZZLE_64B) ||
        // lower rows: Z10 only (N real columns; a K tile across column N
        // reads zeros there instead of Z11)
        !make_map(&mZb, (const float*)Z + (size_t)H * ldz * 2, (uint64_t)N, (uint64_t)H,
                  (uint64_t)ldz * 8, ZBK, ZN, CU_TENSOR_MAP_SWIZZLE_64B) ||
        !make_map(&mA, Bhi, (uint64_t)2 * N, 2 * (uint64_t)nprime, (uint64_t)2 * N * 4, ZBK,
                  2 * nprime, CU_TENSOR_MAP_SWIZZLE_64B)) {
      set_error("cuTensorMapEncodeTiled failed (driver entry point or layout)");
      return MUELLER_ERR_CUDA;
    }
    const size_t stage_bytes = 2 * (size_t)ZN * ZBK * 4 + (size_t)BM * ZBK * 4;
    const int stages = (int)std::min<size_t>(8, (SMEM_BUDGET - 2048) / stage_bytes);
    const size_t smem = 1024 + stages * stage_bytes + (3 * stages + 1) * 8 + 16;
    MU_CUDA(cudaFuncSetAttribute(mrhs_zn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t ntiles = cdiv(H, ZN);
    for (int half = 1; half <= 2; ++half) {
      ZnArgs z;
      z.N = N;
      z.nprime = nprime;
      z.r = r;
      z.ktiles = (int)cdiv(half == 1 ? 2 * N : N, ZBK);
      z.stacked = 1;
      z.Y = (float*)Y;
      z.err = err;
      z.stop = stop;
      z.mirror = half;
      z.H = H;
      z.xoob = (int)(cdiv(2 * N, ZBK) * ZBK + ZBK);
      z.stages = stages;
      int ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(z.ktiles / 16, cdiv(4 * 152, ntiles)));
      z.kchunk = (int)cdiv(z.ktiles, ksplit);
      ksplit = (int)cdiv(z.ktiles, z.kchunk);
      Prof prof_("mrhs_zn_kernel", s);
      mrhs_zn_kernel<<<dim3((unsigned)ntiles, (unsigned)ksplit), THREADS, smem, s>>>(
          half == 1 ? mZt : mZb, mA, mA, z);
    }
    MU_CHECK_LAUNCH("mrhs_zn_kernel (mirrored)");
    return MUELLER_OK;
  }
  if (nprime <= BM) {
    // Z on the N side: 256 Z rows per MMA
    const int zstacked = 2 * nprime <= BM ? 1 : 0;
    CUtensorMap mZ, mA0, mA1;
    const uint64_t arows = zstacked ? 2 * (uint64_t)nprime : (uint64_t)nprime;
    if (!make_map(&mZ, Z, (uint64_t)2 * N, (uint64_t)N, (uint64_t)ldz * 8, ZBK, ZN,
                  CU_TENSOR_MAP_SWIZZLE_64B) ||
        !make_map(&mA0, Bhi, (uint64_t)2 * N, arows, (uint64_t)2 * N * 4, ZBK, BM,
                  CU_TENSOR_MAP_SWIZZLE_64B) ||
        !make_map(&mA1, Blo, (uint64_t)2 * N, (uint64_t)nprime, (uint64_t)2 * N * 4, ZBK, BM,
                  CU_TENSOR_MAP_SWIZZLE_64B)) {
      set_error("cuTensorMapEncodeTiled failed (driver entry point or layout)");
      return MUELLER_ERR_CUDA;
    }
    ZnArgs z;
    z.N = N;
    z.nprime = nprime;
    z.r = r;
    z.ktiles = (int)cdiv(2 * N, ZBK);
    z.stacked = zstacked;
    z.Y = (float*)Y;
    z.err = err;
    z.stop = stop;
    z.mirror = 0;
    z.H = N / 2;
    z.xoob = 0;
    const int64_t ntiles = cdiv(N, ZN);
    int ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(z.ktiles / 16, cdiv(4 * 152, ntiles)));
    z.kchunk = (int)cdiv(z.ktiles, ksplit);
    ksplit = (int)cdiv(z.ktiles, z.kchunk);
    const size_t stage_bytes = 2 * (size_t)ZN * ZBK * 4 + (zstacked ? 1 : 2) * (size_t)BM * ZBK * 4;
    z.stages = (int)std::min<size_t>(8, (SMEM_BUDGET - 2048) / stage_bytes);
    const size_t smem = 1024 + z.stages * stage_bytes + (3 * z.stages + 1) * 8 + 16;
    MU_CUDA(cudaFuncSetAttribute(mrhs_zn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
      Prof prof_("mrhs_zn_kernel", s);
      mrhs_zn_kernel<<<dim3((unsigned)ntiles, (unsigned)ksplit), THREADS, smem, s>>>(mZ, mA0, mA1, z);
    }
    MU_CHECK_LAUNCH("mrhs_zn_kernel");
    return MUELLER_OK;
  }
  CUtensorMap mZ, mBh, mBl;
  if (!make_map(&mZ, Z, (uint64_t)2 * N, (uint64_t)N, (uint64_t)ldz * 8, BK, BM) ||
      !make_map(&mBh, Bhi, (uint64_t)2 * N, (uint64_t)nprime, (uint64_t)2 * N * 4, BK, nprime) ||
      !make_map(&mBl, Blo, (uint64_t)2 * N, (uint64_t)nprime, (uint64_t)2 * N * 4, BK, nprime)) {
    set_error("cuTensorMapEncodeTiled failed (driver entry point or layout)");
    return MUELLER_ERR_CUDA;
  }
  MrhsArgs a;
  a.N = N;
  a.nprime = nprime;
  a.r = r;
  a.ktiles = (int)cdiv(2 * N, BK);
  a.stacked = stacked;
  a.tmem_cols = tmem_cols;
  a.Y = (float*)Y;
  a.err = err;
  a.stop = stop;
  const int64_t mtiles = cdiv(N, BM);
  // split K so that the grid covers the SMs about 4 times
  int ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(a.ktiles / 8, cdiv(4 * 152, mtiles)));
  a.kchunk = (int)cdiv(a.ktiles, ksplit);
  ksplit = (int)cdiv(a.ktiles, a.kchunk);
  const size_t bbytes = (size_t)nprime * BK * 4;
  const size_t stage_bytes = 2 * (size_t)BM * BK * 4 + 2 * bbytes;
  a.stages = (int)std::min<size_t>(6, (SMEM_BUDGET - 2048) / stage_bytes);
  const size_t smem = 1024 + a.stages * stage_bytes + (3 * a.stages + 1) * 8 + 16;
  MU_CUDA(cudaFuncSetAttribute(mrhs_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    Prof prof_("mrhs_tf32_kernel", s);
    mrhs_tf32_kernel<<<dim3((unsigned)mtiles, (unsigned)ksplit), THREADS, smem, s>>>(mZ, mBh, mBl, a);
  }
  MU_CHECK_LAUNCH("mrhs_tf32_kernel");
  return MUELLER_OK;
}

mueller_status mrhs_check_error(void* work, int64_t N, int r, cudaStream_t s) {
  const int nprime = (int)cdiv(2 * r, 16) * 16;
  int* err = (int*)((float*)work + (size_t)2 * nprime * 2 * N);
  int h = 0;
  MU_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MU_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error("tensor-core product: a pipeline wait timed out (stage " + std::to_string(h) + ")");
    return MUELLER_ERR_TIMEOUT;
  }
  return MUELLER_OK;
}

}  // namespace mu
