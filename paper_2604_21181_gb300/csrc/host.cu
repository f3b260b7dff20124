// C ABI entry points of libmueller.so and the host side of the mesh:
// validation, the double Morton permutation (Sec. 5), node-element
// adjacency, touching-pair classification (Sec. 4.2) and the near-part
// block layout.  All compute of the method runs in the CUDA kernels of the
// other translation units; this file only prepares integer tables and
// orchestrates launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "common.cuh"

namespace mu {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

mueller_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MUELLER_ERR_OOM : MUELLER_ERR_CUDA;
}

// ----------------------------------------------------- launch profiling
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static int64_t g_launches = 0;
static std::map<std::string, std::pair<double, int64_t>> g_prof;

Prof::Prof(const char* name, cudaStream_t s) : name_(name), s_(s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ++g_launches;
  if (g_prof_on) {
    cudaEventCreate(&a_);
    cudaEventCreate(&b_);
    cudaEventRecord(a_, s_);
  }
}

Prof::~Prof() {
  if (!a_) return;
  cudaEventRecord(b_, s_);
  cudaEventSynchronize(b_);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a_, b_);
  cudaEventDestroy(a_);
  cudaEventDestroy(b_);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  auto& e = g_prof[name_];
  e.first += ms;
  e.second += 1;
}

static const char* const kHostOnlyMsg =
    "the mesh was loaded with MUELLER_MESH_HOST_ONLY and has no device data";

static mueller_status fail(mueller_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

PhysConsts make_phys(const mueller_params* p) {
  PhysConsts P;
  P.ka = p->ka;
  std::complex<double> er(p->eps_r[0], p->eps_r[1]), mr(p->mu_r[0], p->mu_r[1]);
  std::complex<double> ki = p->ka * std::sqrt(er * mr);
  if (ki.imag() < 0) ki = -ki;
  P.ki_re = ki.real();
  P.ki_im = ki.imag();
  P.eps_re = er.real();
  P.eps_im = er.imag();
  P.mu_re = mr.real();
  P.mu_im = mr.imag();
  return P;
}

// ------------------------------------------------------------- Morton
// 21 bits per axis interleaved, x in the least significant bit.
static uint64_t interleave3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

static uint64_t zkey(const double p[3], const double lo[3], double ext) {
  uint64_t c[3];
  for (int a = 0; a < 3; ++a) {
    double s = (p[a] - lo[a]) / ext * 2097152.0;
    s = (s > 0.0) ? s : 0.0;  // also maps NaN-free negatives and -0 to 0
    s = (s < 2097151.0) ? s : 2097151.0;
    c[a] = (uint64_t)floor(s);
  }
  return interleave3(c[0]) | (interleave3(c[1]) << 1) | (interleave3(c[2]) << 2);
}

static void z_order(const std::vector<uint64_t>& key, std::vector<int32_t>& perm) {
  perm.resize(key.size());
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(),
                   [&](int32_t a, int32_t b) { return key[a] < key[b]; });
}

// --------------------------------------------------------- validation
static mueller_status validate(const double* xyz, int64_t nn, const int32_t* T, int64_t nt) {
  for (int64_t i = 0; i < 3 * nn; ++i)
    if (!std::isfinite(xyz[i])) return fail(MUELLER_ERR_MESH, "non-finite node coordinate");
  for (int64_t e = 0; e < nt; ++e) {
    for (int k = 0; k < 6; ++k) {
      int32_t v = T[6 * e + k];
      if (v < 0 || v >= nn)
        return fail(MUELLER_ERR_MESH, "triangle " + std::to_string(e) + " has a node id out of range");
      for (int l = 0; l < k; ++l)
        if (T[6 * e + l] == v)
          return fail(MUELLER_ERR_MESH, "triangle " + std::to_string(e) + " repeats a node");
    }
    const double* a = xyz + 3 * T[6 * e];
    const double* b = xyz + 3 * T[6 * e + 1];
    const double* c = xyz + 3 * T[6 * e + 2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    if (!(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2] > 0.0))
      return fail(MUELLER_ERR_MESH, "triangle " + std::to_string(e) + " is degenerate");
  }
  // every corner edge in exactly two triangles, opposite directions, same edge node
  struct Use {
    int32_t lo, hi;
    int64_t tri;
    int32_t from, mid;
  };
  // ordered by (lo, hi, tri): a counting sort on lo (the uses of one lo come
  // in increasing tri), then an insertion sort on hi inside each short bucket
  const int emid[3] = {3, 4, 5};
  std::vector<int64_t> first(nn + 1, 0);
  for (int64_t e = 0; e < nt; ++e)
    for (int k = 0; k < 3; ++k) first[std::min(T[6 * e + k], T[6 * e + (k + 1) % 3]) + 1]++;
  for (int64_t i = 0; i < nn; ++i) first[i + 1] += first[i];
  std::vector<Use> uses((size_t)3 * nt);
  {
    std::vector<int64_t> fill(first.begin(), first.end() - 1);
    for (int64_t e = 0; e < nt; ++e)
      for (int k = 0; k < 3; ++k) {
        const int32_t a = T[6 * e + k], b = T[6 * e + (k + 1) % 3];
        uses[fill[std::min(a, b)]++] = {std::min(a, b), std::max(a, b), e, a, T[6 * e + emid[k]]};
      }
  }
  for (int64_t i = 0; i < nn; ++i)
    for (int64_t k = first[i] + 1; k < first[i + 1]; ++k) {
      const Use x = uses[k];
      int64_t j = k;
      while (j > first[i] && (uses[j - 1].hi > x.hi || (uses[j - 1].hi == x.hi && uses[j - 1].tri > x.tri))) {
        uses[j] = uses[j - 1];
        --j;
      }
      uses[j] = x;
    }
  for (size_t k = 0; k < uses.size();) {
    size_t l = k;
    while (l < uses.size() && uses[l].lo == uses[k].lo && uses[l].hi == uses[k].hi) ++l;
    if (l - k != 2)
      return fail(MUELLER_ERR_MESH, "edge (" + std::to_string(uses[k].lo) + "," +
                                        std::to_string(uses[k].hi) + ") is used by " +
                                        std::to_string(l - k) + " triangles (not a closed manifold)");
    const Use &u0 = uses[k], &u1 = uses[k + 1];
    if (u0.from == u1.from)
      return fail(MUELLER_ERR_MESH, "triangles " + std::to_string(u0.tri) + " and " +
                                        std::to_string(u1.tri) + " are inconsistently oriented");
    if (u0.mid != u1.mid)
      return fail(MUELLER_ERR_MESH, "edge node mismatch between triangles " +
                                        std::to_string(u0.tri) + " and " + std::to_string(u1.tri));
    k = l;
  }
  return MUELLER_OK;
}

// touching classification by shared corner vertices, and the relabellings
// putting the shared edge at (v0', v1') (ordered as it runs in ex) or the
// shared vertex at v0' in both triangles.  Conventions of Sec. 4.2 maps:
// reference triangle {0 <= v <= u <= 1}, shared edge v = 0, vertex (0,0).
static int classify_pair(const int32_t* a, const int32_t* b, int32_t& packed) {
  int ia[3], ib[3], ns = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (a[i] == b[j]) {
        ia[ns] = i;
        ib[ns] = j;
        ++ns;
      }
  int px[3] = {0, 1, 2}, py[3] = {0, 1, 2};
  if (ns == 2) {
    int i0 = ia[0], i1 = ia[1], j0 = ib[0], j1 = ib[1];
    if ((i0 + 1) % 3 != i1) {
      std::swap(i0, i1);
      std::swap(j0, j1);
    }
    px[0] = i0;
    px[1] = i1;
    px[2] = 3 - i0 - i1;
    py[0] = j0;
    py[1] = j1;
    py[2] = 3 - j0 - j1;
  } else if (ns == 1) {
    for (int k = 0; k < 3; ++k) {
      px[k] = (ia[0] + k) % 3;
      py[k] = (ib[0] + k) % 3;
    }
  }
  packed = 0;
  for (int k = 0; k < 3; ++k) packed |= (px[k] << (2 * k)) | (py[k] << (8 + 2 * k));
  return ns;
}

// Sorts v[0 .. len) of distinct ids ascending.  Ids of neighbouring nodes or
// elements in Morton order fall in a narrow range, so they are marked in the
// bitmap (all zero on entry and on return) and read back in order when the
// range spans at most 4 words per id; otherwise std::sort.
static void sort_ids(int32_t* v, size_t len, uint64_t* bits) {
  if (len < 2) return;
  int32_t lo = v[0], hi = v[0];
  for (size_t k = 1; k < len; ++k) {
    lo = std::min(lo, v[k]);
    hi = std::max(hi, v[k]);
  }
  const int64_t w0 = lo >> 6, w1 = hi >> 6;
  if (w1 - w0 + 1 > (int64_t)(4 * len)) {
    std::sort(v, v + len);
    return;
  }
  for (size_t k = 0; k < len; ++k) bits[v[k] >> 6] |= 1ull << (v[k] & 63);
  size_t o = 0;
  for (int64_t w = w0; w <= w1; ++w) {
    uint64_t b = bits[w];
    bits[w] = 0;
    while (b) {
      v[o++] = (int32_t)((w << 6) + __builtin_ctzll(b));
      b &= b - 1;
    }
  }
}

template <class Tp>
static mueller_status upload(Tp** dst, const Tp* src, size_t n, cudaStream_t s) {
  MU_CUDA(cudaMalloc((void**)dst, std::max<size_t>(1, n) * sizeof(Tp)));
  if (n) MU_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(Tp), cudaMemcpyHostToDevice, s));
  return MUELLER_OK;
}

// Touching-pair classification, the touching kernel's launch order and the
// near-part block layout of a loaded mesh (its host tables).
static void build_tables(mueller_mesh* m, const std::vector<int32_t>& ptr,
                         const std::vector<int32_t>& n2e, std::vector<TouchPair>& tp,
                         std::vector<int32_t>& order, std::vector<int32_t>& slot) {
  const int64_t nn = m->nn, nt = m->nt;
  const int32_t* T = m->T_h.data();
  // host threads for the table passes below: each takes a contiguous range
  // of elements or rows, and the tables do not depend on the thread count
  const int64_t nthreads = std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)std::thread::hardware_concurrency(), 16, nn / 256}));
  auto run = [&](auto&& fn) {
    if (nthreads == 1) {
      fn((int64_t)0);
      return;
    }
    std::vector<std::thread> pool;
    pool.reserve(nthreads);
    for (int64_t t = 0; t < nthreads; ++t) pool.emplace_back(fn, t);
    for (std::thread& th : pool) th.join();
  };
  // ---- touching pairs (sorted by ex, then ey)
  tp.clear();
  {
    std::vector<std::vector<TouchPair>> part(nthreads);
    run([&](int64_t t) {
      const int64_t e0 = nt * t / nthreads, e1 = nt * (t + 1) / nthreads;
      std::vector<int32_t> cand;
      std::vector<int32_t> seen(nt, -1);
      std::vector<uint64_t> bits((nt + 63) / 64 + 1, 0);
      for (int64_t ex = e0; ex < e1; ++ex) {
        cand.clear();
        for (int k = 0; k < 3; ++k) {
          int32_t v = T[6 * ex + k];
          for (int32_t q = ptr[v]; q < ptr[v + 1]; ++q) {
            const int32_t ey = n2e[q] >> 3;
            if (seen[ey] != (int32_t)ex) {
              seen[ey] = (int32_t)ex;
              cand.push_back(ey);
            }
          }
        }
        sort_ids(cand.data(), cand.size(), bits.data());
        for (int32_t ey : cand) {
          int32_t packed;
          int cls = classify_pair(T + 6 * ex, T + 6 * ey, packed);
          if (cls > 0) part[t].push_back({(int32_t)ex, ey, cls, packed});
        }
      }
    });
    size_t total = 0;
    for (const auto& v : part) total += v.size();
    tp.reserve(total);
    for (const auto& v : part) tp.insert(tp.end(), v.begin(), v.end());
  }
  m->n_touch = (int64_t)tp.size();
  // launch order of the touching kernel: coincident and common-edge pairs,
  // then the common-vertex pairs (which use shared-memory tables)
  order.clear();
  order.reserve(tp.size());
  for (int pass = 0; pass < 2; ++pass)
    for (size_t q = 0; q < tp.size(); ++q)
      if ((tp[q].cls == 1) == (pass == 1)) order.push_back((int32_t)q);
  m->n_touch_ce = 0;
  for (const TouchPair& q : tp) m->n_touch_ce += q.cls != 1;
  // ---- near-part block layout: node pairs of the touching element pairs.
  // Row by row: the columns of test node ni are the nodes of every trial
  // element touching an element that holds ni (deduplicated with a stamp
  // array, then sorted), and the slot of (pair, i, j) is found through a
  // column -> position array valid for the current row.
  std::vector<int64_t> pfirst(nt + 1, 0);  // tp is sorted by ex
  for (const TouchPair& q : tp) pfirst[q.ex + 1]++;
  for (int64_t e = 0; e < nt; ++e) pfirst[e + 1] += pfirst[e];
  slot.assign((size_t)m->n_touch * 36, 0);
  {
    // Rows are independent: phase 1 finds each row's sorted columns, phase 2
    // (after the prefix sum of the row lengths) places them and fills the
    // slots of the row's (pair, i) entries, which no other row writes.
    std::vector<std::vector<int32_t>> cols(nthreads);
    std::vector<int32_t> len_of(nn, 0);
    auto range = [&](int64_t t, int64_t& r0, int64_t& r1) {
      r0 = nn * t / nthreads;
      r1 = nn * (t + 1) / nthreads;
    };
    auto phase1 = [&](int64_t t) {
      int64_t r0, r1;
      range(t, r0, r1);
      std::vector<int32_t> stamp(nn, -1), row;
      std::vector<uint64_t> bits((nn + 63) / 64 + 1, 0);
      std::vector<int32_t>& out = cols[t];
      for (int64_t ni = r0; ni < r1; ++ni) {
        row.clear();
        for (int32_t q = ptr[ni]; q < ptr[ni + 1]; ++q) {
          const int64_t ex = n2e[q] >> 3;
          for (int64_t p = pfirst[ex]; p < pfirst[ex + 1]; ++p)
            for (int j = 0; j < 6; ++j) {
              const int32_t nj = T[6 * tp[p].ey + j];
              if (stamp[nj] != (int32_t)ni) {
                stamp[nj] = (int32_t)ni;
                row.push_back(nj);
              }
            }
        }
        sort_ids(row.data(), row.size(), bits.data());
        out.insert(out.end(), row.begin(), row.end());
        len_of[ni] = (int32_t)row.size();
      }
    };
    run(phase1);
    m->near_rowptr_h.assign(nn + 1, 0);
    for (int64_t ni = 0; ni < nn; ++ni) m->near_rowptr_h[ni + 1] = m->near_rowptr_h[ni] + len_of[ni];
    m->near_col_h.assign((size_t)m->near_rowptr_h[nn], 0);
    auto phase2 = [&](int64_t t) {
      int64_t r0, r1;
      range(t, r0, r1);
      std::vector<int32_t> pos(nn, 0);
      const int32_t* src = cols[t].data();
      for (int64_t ni = r0; ni < r1; ++ni) {
        const int32_t start = m->near_rowptr_h[ni], len = len_of[ni];
        for (int32_t k = 0; k < len; ++k) {
          m->near_col_h[(size_t)start + k] = src[k];
          pos[src[k]] = start + k;
        }
        src += len;
        for (int32_t q = ptr[ni]; q < ptr[ni + 1]; ++q) {
          const int64_t ex = n2e[q] >> 3;
          const int i = n2e[q] & 7;
          for (int64_t p = pfirst[ex]; p < pfirst[ex + 1]; ++p)
            for (int j = 0; j < 6; ++j) slot[(size_t)p * 36 + i * 6 + j] = pos[T[6 * tp[p].ey + j]];
        }
      }
    };
    run(phase2);
    m->nnzb = m->near_rowptr_h[nn];
  }
}

// The host tables of a mesh are ready (their thread joined); their status.
mueller_status mesh_tables(const mueller_mesh* m) {
  std::lock_guard<std::mutex> g(m->tables_mu);
  if (m->tables_thread.joinable()) m->tables_thread.join();
  if (m->tables_st) return fail(m->tables_st, m->tables_msg);
  return MUELLER_OK;
}

}  // namespace mu

using namespace mu;

extern "C" {

int32_t mueller_version(void) { return 1; }

const char* mueller_last_error(void) { return g_last_error.c_str(); }

const char* mueller_status_string(mueller_status s) {
  switch (s) {
    case MUELLER_OK: return "ok";
    case MUELLER_ERR_INVALID_ARG: return "invalid argument";
    case MUELLER_ERR_MESH: return "invalid mesh";
    case MUELLER_ERR_DEGENERATE_FRAME: return "degenerate tangent frame";
    case MUELLER_ERR_SINGULAR_BLOCK: return "singular preconditioner block";
    case MUELLER_ERR_NOT_CONVERGED: return "not converged";
    case MUELLER_ERR_TIMEOUT: return "device wait timed out";
    case MUELLER_ERR_CUDA: return "CUDA error";
    case MUELLER_ERR_OOM: return "out of device memory";
    case MUELLER_ERR_STATE: return "call order violated";
    case MUELLER_ERR_NAN: return "NaN or infinite residual";
  }
  return "unknown status";
}

void mueller_mesh_free(mueller_mesh* m) {
  if (!m) return;
  mesh_tables(m);  // the table thread writes into m
  void* ptrs[] = {m->X, m->T, m->n2e_ptr, m->n2e, m->frame, m->qd64, m->qd32, m->tp,
                  m->near_rowptr, m->near_col, m->tp_slot, m->tp_order, m->d_flags, m->d_scal};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

mueller_status mueller_mesh_load(const double* xyz, int64_t nn, const int32_t* tri6, int64_t nt,
                                 int32_t flags, void* stream, mueller_mesh** out) {
  if (!out) return fail(MUELLER_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!xyz || !tri6) return fail(MUELLER_ERR_INVALID_ARG, "xyz or tri6 is NULL");
  if (nn < 6 || nt < 4) return fail(MUELLER_ERR_INVALID_ARG, "mesh too small (closed surface needs >= 4 triangles)");
  if (nn > (1ll << 28) || nt > (1ll << 27)) return fail(MUELLER_ERR_INVALID_ARG, "mesh too large");
  mueller_status st = validate(xyz, nn, tri6, nt);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  mueller_mesh* m = new mueller_mesh();
  m->nn = nn;
  m->nt = nt;
  // ---- double Morton permutation (Sec. 5)
  if (flags & MUELLER_MESH_KEEP_ORDER) {
    m->node_perm.resize(nn);
    m->elem_perm.resize(nt);
    std::iota(m->node_perm.begin(), m->node_perm.end(), 0);
    std::iota(m->elem_perm.begin(), m->elem_perm.end(), 0);
  } else {
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = xyz[a];
    for (int64_t i = 0; i < nn; ++i)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], xyz[3 * i + a]);
        hi[a] = std::max(hi[a], xyz[3 * i + a]);
      }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    if (!(ext > 0.0)) ext = 1.0;
    std::vector<uint64_t> key(nn);
    for (int64_t i = 0; i < nn; ++i) key[i] = zkey(xyz + 3 * i, lo, ext);
    z_order(key, m->node_perm);
    std::vector<uint64_t> ek(nt);
    for (int64_t e = 0; e < nt; ++e) {
      double c[3];
      for (int a = 0; a < 3; ++a)
        c[a] = (xyz[3 * tri6[6 * e] + a] + xyz[3 * tri6[6 * e + 1] + a] + xyz[3 * tri6[6 * e + 2] + a]) / 3.0;
      ek[e] = zkey(c, lo, ext);
    }
    z_order(ek, m->elem_perm);
  }
  std::vector<int32_t> inv(nn);
  for (int64_t i = 0; i < nn; ++i) inv[m->node_perm[i]] = (int32_t)i;
  m->X_h.resize(3 * nn);
  for (int64_t i = 0; i < nn; ++i)
    for (int a = 0; a < 3; ++a) m->X_h[3 * i + a] = xyz[3 * m->node_perm[i] + a];
  m->T_h.resize(6 * nt);
  for (int64_t e = 0; e < nt; ++e)
    for (int k = 0; k < 6; ++k) m->T_h[6 * e + k] = inv[tri6[6 * m->elem_perm[e] + k]];
  const int32_t* T = m->T_h.data();
  // ---- node -> (element, local index), ascending element order
  std::vector<int32_t> ptr(nn + 1, 0), n2e(6 * nt);
  for (int64_t e = 0; e < nt; ++e)
    for (int k = 0; k < 6; ++k) ptr[T[6 * e + k] + 1]++;
  for (int64_t i = 0; i < nn; ++i) ptr[i + 1] += ptr[i];
  {
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < nt; ++e)
      for (int k = 0; k < 6; ++k) n2e[fill[T[6 * e + k]]++] = (int32_t)((e << 3) | k);
  }
  if (flags & MUELLER_MESH_HOST_ONLY) {
    m->host_only = true;
    std::vector<TouchPair> tp;
    std::vector<int32_t> order, slot;
    build_tables(m, ptr, n2e, tp, order, slot);
    m->tp_h = std::move(tp);
    m->tp_slot_h = std::move(slot);
    *out = m;
    return MUELLER_OK;
  }
  // ---- upload of what the frame, the point geometry and the regular pairs read
  st = upload(&m->X, m->X_h.data(), m->X_h.size(), s);
  if (!st) st = upload(&m->T, m->T_h.data(), m->T_h.size(), s);
  if (!st) st = upload(&m->n2e_ptr, ptr.data(), ptr.size(), s);
  if (!st) st = upload(&m->n2e, n2e.data(), n2e.size(), s);
  int dev = 0;
  if (!st) {
    cudaError_t e = cudaMalloc((void**)&m->d_flags, 64 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->d_scal, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_flags, 0, 64 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // ptr and n2e move on below
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e != cudaSuccess) st = cuda_fail(e, "mesh upload");
  }
  if (st) {
    mueller_mesh_free(m);
    return st;
  }
  // ---- the host tables and their upload on a host thread of their own, so
  // that the caller's frame, point-geometry and regular-pair launches need
  // not wait for them; every call that reads them joins it first
  // (mesh_tables), and its status and message surface there.
  struct Inputs {
    std::vector<int32_t> ptr, n2e;
  };
  auto in = std::make_shared<Inputs>();
  in->ptr = std::move(ptr);
  in->n2e = std::move(n2e);
  auto work = [m, dev, in]() {
    std::vector<TouchPair> tp;
    std::vector<int32_t> order, slot;
    mueller_status st = MUELLER_OK;
    try {
      build_tables(m, in->ptr, in->n2e, tp, order, slot);
    } catch (const std::bad_alloc&) {
      st = fail(MUELLER_ERR_OOM, "host memory for the touching pairs and the near layout");
    } catch (const std::exception& x) {  // e.g. no host thread for the table passes
      st = fail(MUELLER_ERR_OOM, std::string("host resources for the mesh tables: ") + x.what());
    }
    cudaStream_t ts = nullptr;
    if (!st) {
      cudaError_t e = cudaSetDevice(dev);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
      if (e != cudaSuccess) st = cuda_fail(e, "mesh table stream");
    }
    if (!st) st = upload(&m->tp, tp.data(), tp.size(), ts);
    if (!st) st = upload(&m->near_rowptr, m->near_rowptr_h.data(), m->near_rowptr_h.size(), ts);
    if (!st) st = upload(&m->near_col, m->near_col_h.data(), m->near_col_h.size(), ts);
    if (!st) st = upload(&m->tp_slot, slot.data(), slot.size(), ts);
    if (!st) st = upload(&m->tp_order, order.data(), order.size(), ts);
    if (ts) {
      const cudaError_t e = cudaStreamSynchronize(ts);
      if (!st && e != cudaSuccess) st = cuda_fail(e, "mesh table upload");
      cudaStreamDestroy(ts);
    }
    m->tp_h = std::move(tp);
    m->tp_slot_h = std::move(slot);
    m->tables_st = st;
    if (st) m->tables_msg = mueller_last_error();
  };
  try {
    m->tables_thread = std::thread(work);
  } catch (const std::system_error&) {
    work();  // no thread to be had: build the tables here
  }
  *out = m;
  return MUELLER_OK;
}

mueller_status mueller_mesh_get_info(const mueller_mesh* m, mueller_mesh_info* info) {
  if (!m || !info) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  info->n_nodes = m->nn;
  info->n_tri = m->nt;
  info->n_dof = 4 * m->nn;
  info->n_touching = m->n_touch;
  info->n_near_blocks = m->nnzb;
  info->min_gs_norm = m->min_gs;
  return MUELLER_OK;
}

mueller_status mueller_mesh_perm(const mueller_mesh* m, int32_t* node_perm, int32_t* elem_perm) {
  if (!m) return fail(MUELLER_ERR_INVALID_ARG, "mesh is NULL");
  if (node_perm) std::copy(m->node_perm.begin(), m->node_perm.end(), node_perm);
  if (elem_perm) std::copy(m->elem_perm.begin(), m->elem_perm.end(), elem_perm);
  return MUELLER_OK;
}

mueller_status mueller_quadrature_rule(int32_t kind, int32_t n, double* a, double* b, double* w) {
  if (!a || !w) return fail(MUELLER_ERR_INVALID_ARG, "a or w is NULL");
  if (kind == MUELLER_RULE_TRIANGLE) {
    TriangleRule r;
    if (!b) return fail(MUELLER_ERR_INVALID_ARG, "b is NULL");
    if ((n != 6 && n != 12) || !triangle_rule(n, r))
      return fail(MUELLER_ERR_INVALID_ARG, "triangle rules have 6 or 12 points");
    std::copy(r.xi.begin(), r.xi.end(), a);
    std::copy(r.eta.begin(), r.eta.end(), b);
    std::copy(r.w.begin(), r.w.end(), w);
  } else if (kind == MUELLER_RULE_GAUSS_LEGENDRE) {
    if (n < 1 || n > 512) return fail(MUELLER_ERR_INVALID_ARG, "Gauss-Legendre n in 1..512");
    std::vector<double> x, ww;
    gauss_legendre_unit(n, x, ww);
    std::copy(x.begin(), x.end(), a);
    std::copy(ww.begin(), ww.end(), w);
  } else {
    return fail(MUELLER_ERR_INVALID_ARG, "unknown rule kind");
  }
  return MUELLER_OK;
}

mueller_status mueller_mesh_touching(const mueller_mesh* m, int32_t* ex, int32_t* ey, int32_t* cls,
                                     int32_t* relabel) {
  if (!m) return fail(MUELLER_ERR_INVALID_ARG, "mesh is NULL");
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  for (size_t q = 0; q < m->tp_h.size(); ++q) {
    const TouchPair& t = m->tp_h[q];
    if (ex) ex[q] = t.ex;
    if (ey) ey[q] = t.ey;
    if (cls) cls[q] = t.cls;
    if (relabel) relabel[q] = t.perm;
  }
  return MUELLER_OK;
}

mueller_status mueller_mesh_near_layout(const mueller_mesh* m, int32_t* rowptr, int32_t* col,
                                        int32_t* slot) {
  if (!m) return fail(MUELLER_ERR_INVALID_ARG, "mesh is NULL");
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  if (rowptr) std::copy(m->near_rowptr_h.begin(), m->near_rowptr_h.end(), rowptr);
  if (col) std::copy(m->near_col_h.begin(), m->near_col_h.end(), col);
  if (slot) std::copy(m->tp_slot_h.begin(), m->tp_slot_h.end(), slot);
  return MUELLER_OK;
}

mueller_status mueller_point_records(const mueller_mesh* m, int32_t q_regular, double* out) {
  if (!m || !out) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  if (m->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  if (!m->has_frame || m->qd_q != q_regular || !m->qd64)
    return fail(MUELLER_ERR_STATE, "no point geometry for this rule: call mueller_assemble or "
                                   "mueller_far_field with it first");
  const int64_t n = m->nt * q_regular;
  std::vector<double> rec((size_t)n * QD_STRIDE);
  MU_CUDA(cudaMemcpy(rec.data(), m->qd64, rec.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int64_t t = 0; t < n; ++t)
    std::copy(rec.begin() + t * QD_STRIDE, rec.begin() + t * QD_STRIDE + 19, out + t * 19);
  return MUELLER_OK;
}

mueller_status mueller_tangent_frame(mueller_mesh* m, int32_t frame_rule, double* frame_dev,
                                     void* stream) {
  if (!m) return fail(MUELLER_ERR_INVALID_ARG, "mesh is NULL");
  if (frame_rule != MUELLER_FRAME_PAPER && frame_rule != MUELLER_FRAME_POLAR)
    return fail(MUELLER_ERR_INVALID_ARG, "unknown frame_rule");
  if (m->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  cudaStream_t s = (cudaStream_t)stream;
  if (!m->frame) MU_CUDA(cudaMalloc((void**)&m->frame, 9 * m->nn * sizeof(double)));
  mueller_status st = launch_frame(m, frame_rule, s);
  if (st) return st;
  m->has_frame = true;
  m->frame_rule = frame_rule;
  m->qd_q = 0;  // point geometry depends on the frame
  if (frame_dev)
    MU_CUDA(cudaMemcpyAsync(frame_dev, m->frame, 9 * m->nn * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
  return MUELLER_OK;
}

size_t mueller_near_bytes(const mueller_mesh* m) {
  if (!m || mesh_tables(m)) return 0;
  return (size_t)m->nnzb * 16 * 2 * sizeof(double);
}

// Incident waves: rows (k-hat, p-hat) of orthonormal real vectors; far-field
// directions: unit vectors (both to 1e-10 in the squared norms and k.p).
static mueller_status check_inc(const double* inc, int64_t r) {
  for (int64_t q = 0; q < r; ++q) {
    const double* k = inc + 6 * q;
    const double* e = k + 3;
    for (int a = 0; a < 6; ++a)
      if (!std::isfinite(k[a]))
        return fail(MUELLER_ERR_INVALID_ARG, "incident wave " + std::to_string(q) + " is not finite");
    const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    const double ke = k[0] * e[0] + k[1] * e[1] + k[2] * e[2];
    if (!(std::fabs(kk - 1.0) <= 1e-10 && std::fabs(ee - 1.0) <= 1e-10 && std::fabs(ke) <= 1e-10))
      return fail(MUELLER_ERR_INVALID_ARG, "incident wave " + std::to_string(q) +
                                               ": k-hat and p-hat must be orthonormal");
  }
  return MUELLER_OK;
}

static mueller_status check_dirs(const double* d, int64_t n) {
  for (int64_t q = 0; q < n; ++q) {
    const double dd = d[3 * q] * d[3 * q] + d[3 * q + 1] * d[3 * q + 1] + d[3 * q + 2] * d[3 * q + 2];
    if (!(std::fabs(dd - 1.0) <= 1e-10))
      return fail(MUELLER_ERR_INVALID_ARG, "direction " + std::to_string(q) + " is not a unit vector");
  }
  return MUELLER_OK;
}

static mueller_status check_params(const mueller_params* p) {
  if (!p) return fail(MUELLER_ERR_INVALID_ARG, "params is NULL");
  if (!(p->ka > 0.0) || !std::isfinite(p->ka)) return fail(MUELLER_ERR_INVALID_ARG, "ka must be positive");
  if (p->q_regular != 6 && p->q_regular != 12) return fail(MUELLER_ERR_INVALID_ARG, "q_regular must be 6 or 12");
  if (p->ssq_order < 1 || p->ssq_order > MAX_NS) return fail(MUELLER_ERR_INVALID_ARG, "ssq_order must be in 1..16");
  for (double v : {p->eps_r[0], p->eps_r[1], p->mu_r[0], p->mu_r[1]})
    if (!std::isfinite(v)) return fail(MUELLER_ERR_INVALID_ARG, "non-finite material");
  if (p->eps_r[0] == 0.0 && p->eps_r[1] == 0.0) return fail(MUELLER_ERR_INVALID_ARG, "eps_r = 0");
  if (p->mu_r[0] == 0.0 && p->mu_r[1] == 0.0) return fail(MUELLER_ERR_INVALID_ARG, "mu_r = 0");
  return MUELLER_OK;
}

// point geometry for rule q (cached in the handle); reads back the smallest
// Gram-Schmidt norm (synchronises the stream once per rule change)
static mueller_status ensure_geometry(mueller_mesh* m, int q, cudaStream_t s) {
  if (!m->has_frame) return fail(MUELLER_ERR_STATE, "mueller_tangent_frame must be called first");
  if (m->qd_q == q) return MUELLER_OK;
  TriangleRule rule;
  if (!triangle_rule(q, rule)) return fail(MUELLER_ERR_INVALID_ARG, "triangle rule derivation failed");
  if (m->qd64) cudaFree(m->qd64);
  if (m->qd32) cudaFree(m->qd32);
  m->qd64 = nullptr;
  m->qd32 = nullptr;
  size_t n = (size_t)m->nt * q * QD_STRIDE;
  MU_CUDA(cudaMalloc((void**)&m->qd64, n * sizeof(double)));
  MU_CUDA(cudaMalloc((void**)&m->qd32, n * sizeof(float)));
  mueller_status st = launch_quad_geometry(m, rule, s);
  if (st) return st;
  double gs = 0.0;
  MU_CUDA(cudaMemcpyAsync(&gs, m->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MU_CUDA(cudaStreamSynchronize(s));
  m->min_gs = gs;
  m->qd_q = q;
  if (!(gs > 1e-6))
    return fail(MUELLER_ERR_DEGENERATE_FRAME,
                "interpolated tangent frame degenerates (Gram-Schmidt norm " + std::to_string(gs) + ")");
  return MUELLER_OK;
}

mueller_status mueller_assemble(mueller_mesh* m, const mueller_params* p, int32_t dtype,
                                void* Z, int64_t ldz, void* near, void* B, const double* inc,
                                int32_t r, void* stream) {
  if (!m) return fail(MUELLER_ERR_INVALID_ARG, "mesh is NULL");
  mueller_status st = check_params(p);
  if (st) return st;
  const int64_t N = 4 * m->nn;
  if (dtype != MUELLER_C128 && dtype != MUELLER_C64_NEAR64)
    return fail(MUELLER_ERR_INVALID_ARG, "unknown dtype");
  if (!Z || ldz < N) return fail(MUELLER_ERR_INVALID_ARG, "Z is NULL or ldz < N");
  if (dtype == MUELLER_C64_NEAR64 && !near) return fail(MUELLER_ERR_INVALID_ARG, "near buffer required");
  if (B && (r < 1 || !inc)) return fail(MUELLER_ERR_INVALID_ARG, "B given without r >= 1 and inc");
  if (B && (st = check_inc(inc, r))) return st;
  if (p->frame_rule != m->frame_rule || !m->has_frame)
    return fail(MUELLER_ERR_STATE, "call mueller_tangent_frame with params->frame_rule first");
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_geometry(m, p->q_regular, s);
  if (st) return st;
  TriangleRule rule;
  triangle_rule(p->q_regular, rule);
  st = upload_rules(rule, p->ssq_order);
  if (st) return st;
  PhysConsts P = make_phys(p);
  size_t esz = dtype == MUELLER_C128 ? 16 : 8;
  MU_CUDA(cudaMemsetAsync(Z, 0, (size_t)N * ldz * esz, s));
  double* inc_dev = nullptr;
  if (B) {
    MU_CUDA(cudaMemsetAsync(B, 0, (size_t)r * N * 16, s));
    MU_CUDA(cudaMallocAsync((void**)&inc_dev, (size_t)r * 6 * sizeof(double), s));
    MU_CUDA(cudaMemcpyAsync(inc_dev, inc, (size_t)r * 6 * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  // regular pairs on s and touching pairs on the side stream s2, concurrently
  // (the tile-shape choice comes first: a tuning run re-zeroes Z)
  st = tune_regular(m, P, p->q_regular, dtype, Z, ldz, s);
  cudaStream_t s2 = nullptr;
  if (!st) st = side_stream(&s2);
  if (!st) st = stream_order(s, s2);
  if (!st) {
    // the regular pairs need no host tables: they are launched before the
    // wait for the mesh's table thread, the touching pairs (and the zeroing
    // of the near blocks they add into) after it
    st = launch_regular(m, P, p->q_regular, dtype, Z, ldz, s);
    if (!st) st = mesh_tables(m);
    if (!st && dtype == MUELLER_C64_NEAR64) {
      cudaError_t e = cudaMemsetAsync(near, 0, mueller_near_bytes(m), s2);
      if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync(near)");
    }
    if (!st) st = launch_touching(m, P, p->q_regular, p->ssq_order, dtype, Z, ldz, near, s2);
    const mueller_status sj = stream_order(s2, s);
    if (!st) st = sj;
  }
  if (!st) st = launch_mass_rhs(m, P, p->q_regular, dtype, Z, ldz, near, B, inc_dev, B ? r : 0, s);
  if (!st) st = launch_mirror_k1(N, dtype, Z, ldz, s);
  if (inc_dev) cudaFreeAsync(inc_dev, s);
  return st;
}

mueller_status mueller_dz_matvec(mueller_mesh* m, const mueller_params* p, int32_t which,
                                 const void* X, void* Y, void* stream) {
  if (!m || !X || !Y) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  mueller_status st = check_params(p);
  if (st) return st;
  if (which != 1 && which != 2) return fail(MUELLER_ERR_INVALID_ARG, "which must be 1 (eps_r) or 2 (mu_r)");
  if (p->frame_rule != m->frame_rule || !m->has_frame)
    return fail(MUELLER_ERR_STATE, "call mueller_tangent_frame with params->frame_rule first");
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_geometry(m, p->q_regular, s);
  if (st) return st;
  TriangleRule rule;
  triangle_rule(p->q_regular, rule);
  st = upload_rules(rule, p->ssq_order);
  if (st) return st;
  return launch_dz_matvec(m, make_phys(p), p->q_regular, p->ssq_order, which, X, Y, s);
}

mueller_status mueller_zshape_vjp_multi(mueller_mesh* m, const mueller_params* p, const void* lam,
                                        int32_t r, const void* X, double* grad, void* stream) {
  if (!m || !lam || !X || !grad) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  if (r < 1) return fail(MUELLER_ERR_INVALID_ARG, "r must be >= 1");
  mueller_status st = check_params(p);
  if (st) return st;
  if (m->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  if (p->frame_rule != m->frame_rule || !m->has_frame)
    return fail(MUELLER_ERR_STATE, "call mueller_tangent_frame with params->frame_rule first");
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_geometry(m, p->q_regular, s);
  if (st) return st;
  std::fill(grad, grad + (size_t)r * 3 * m->nn, 0.0);
  return zshape_vjp(m, make_phys(p), p->q_regular, p->ssq_order, lam, X, r, grad, s);
}

mueller_status mueller_zshape_vjp(mueller_mesh* m, const mueller_params* p, const void* lam,
                                  const void* X, double* grad, void* stream) {
  return mueller_zshape_vjp_multi(m, p, lam, 1, X, grad, stream);
}

mueller_status mueller_rhs_shape_vjp(mueller_mesh* m, const mueller_params* p, const void* lam,
                                     const double* inc, double* grad, void* stream) {
  if (!m || !lam || !inc || !grad) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  mueller_status st = check_params(p);
  if (st) return st;
  if ((st = check_inc(inc, 1))) return st;
  if (m->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  if (p->frame_rule != m->frame_rule || !m->has_frame)
    return fail(MUELLER_ERR_STATE, "call mueller_tangent_frame with params->frame_rule first");
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_geometry(m, p->q_regular, s);
  if (st) return st;
  std::fill(grad, grad + 3 * m->nn, 0.0);
  return rhs_shape_vjp(m, make_phys(p), p->q_regular, lam, inc, grad, s);
}

mueller_status mueller_cross_section_partials(mueller_mesh* m, const mueller_params* p,
                                              const void* X, const double* inc, int32_t n_theta,
                                              int32_t n_phi, void* G, double* grad, double* xs,
                                              void* stream) {
  if (!m || !X || !inc || !G || !grad) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  mueller_status st = check_params(p);
  if (st) return st;
  if ((st = check_inc(inc, 1))) return st;
  if (n_theta < 2 || n_phi < 3 || n_theta > 512 || n_phi > 1024)
    return fail(MUELLER_ERR_INVALID_ARG, "n_theta must be in [2, 512] and n_phi in [3, 1024]");
  if (m->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  if (p->frame_rule != m->frame_rule || !m->has_frame)
    return fail(MUELLER_ERR_STATE, "call mueller_tangent_frame with params->frame_rule first");
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_geometry(m, p->q_regular, s);
  if (st) return st;
  std::fill(grad, grad + 9 * m->nn, 0.0);
  return cross_section_partials(m, make_phys(p), p->q_regular, X, inc, n_theta, n_phi, G, grad,
                                xs, s);
}

mueller_status mueller_assemble_batch(int32_t n_bodies, mueller_mesh* const* meshes,
                                      const mueller_params* params, int32_t dtype,
                                      void* const* Z, const int64_t* ldz, void* const* near,
                                      void* const* B, const double* const* inc, const int32_t* r,
                                      void* stream) {
  if (n_bodies < 1 || !meshes || !params || !Z || !ldz)
    return fail(MUELLER_ERR_INVALID_ARG, "n_bodies < 1 or a NULL array");
  if (dtype != MUELLER_C128 && dtype != MUELLER_C64_NEAR64)
    return fail(MUELLER_ERR_INVALID_ARG, "unknown dtype");
  if (dtype == MUELLER_C64_NEAR64 && !near) return fail(MUELLER_ERR_INVALID_ARG, "near buffers required");
  if (B && (!inc || !r)) return fail(MUELLER_ERR_INVALID_ARG, "B given without inc and r");
  const int q = params[0].q_regular, ns = params[0].ssq_order;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<PhysConsts> P(n_bodies);
  for (int b = 0; b < n_bodies; ++b) {
    mueller_mesh* m = meshes[b];
    const mueller_params* p = params + b;
    const std::string who = "body " + std::to_string(b) + ": ";
    if (!m) return fail(MUELLER_ERR_INVALID_ARG, who + "mesh is NULL");
    if (mueller_status ts_ = mesh_tables(m)) return ts_;
    mueller_status st = check_params(p);
    if (st) return st;
    if (p->q_regular != q || p->ssq_order != ns)
      return fail(MUELLER_ERR_INVALID_ARG, who + "all bodies must share q_regular and ssq_order");
    const int64_t N = 4 * m->nn;
    if (!Z[b] || ldz[b] < N) return fail(MUELLER_ERR_INVALID_ARG, who + "Z is NULL or ldz < N");
    if (dtype == MUELLER_C64_NEAR64 && !near[b]) return fail(MUELLER_ERR_INVALID_ARG, who + "near is NULL");
    if (B && B[b] && (r[b] < 1 || !inc[b])) return fail(MUELLER_ERR_INVALID_ARG, who + "B without r >= 1 and inc");
    if (B && B[b] && (st = check_inc(inc[b], r[b]))) return st;
    if (p->frame_rule != m->frame_rule || !m->has_frame)
      return fail(MUELLER_ERR_STATE, who + "call mueller_tangent_frame with params->frame_rule first");
    st = ensure_geometry(m, q, s);
    if (st) return st;
    P[b] = make_phys(p);
  }
  TriangleRule rule;
  triangle_rule(q, rule);
  mueller_status st = upload_rules(rule, ns);
  if (st) return st;
  const size_t esz = dtype == MUELLER_C128 ? 16 : 8;
  for (int b = 0; b < n_bodies; ++b) {
    const int64_t N = 4 * meshes[b]->nn;
    MU_CUDA(cudaMemsetAsync(Z[b], 0, (size_t)N * ldz[b] * esz, s));
    if (dtype == MUELLER_C64_NEAR64) MU_CUDA(cudaMemsetAsync(near[b], 0, mueller_near_bytes(meshes[b]), s));
  }
  st = launch_assemble_batch(n_bodies, meshes, P.data(), q, ns, dtype, Z, ldz, near, s);
  for (int b = 0; b < n_bodies && !st; ++b) {
    mueller_mesh* m = meshes[b];
    const int64_t N = 4 * m->nn;
    double* inc_dev = nullptr;
    if (B && B[b]) {
      MU_CUDA(cudaMemsetAsync(B[b], 0, (size_t)r[b] * N * 16, s));
      MU_CUDA(cudaMallocAsync((void**)&inc_dev, (size_t)r[b] * 6 * sizeof(double), s));
      MU_CUDA(cudaMemcpyAsync(inc_dev, inc[b], (size_t)r[b] * 6 * sizeof(double), cudaMemcpyHostToDevice, s));
      st = launch_mass_rhs(m, P[b], q, dtype, Z[b], ldz[b], near ? near[b] : nullptr, B[b], inc_dev, r[b], s);
    }
    if (!st) st = launch_mirror_k1(N, dtype, Z[b], ldz[b], s);
    if (inc_dev) cudaFreeAsync(inc_dev, s);
  }
  return st;
}

size_t mueller_precond_bytes(int64_t n_dof, int64_t block) {
  if (n_dof <= 0 || block <= 0) return 0;
  int64_t H = n_dof / 2, nb = (H + block - 1) / block;
  int64_t d = 2 * block;
  return (size_t)nb * d * d * 16 + (size_t)nb * d * sizeof(int32_t) + 256;
}

mueller_status mueller_precond_build(const mueller_operator* op, int64_t block, void* P,
                                     void* stream) {
  if (!op || !op->mesh || !op->Z_dev || !P) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  if (block < 1) return fail(MUELLER_ERR_INVALID_ARG, "block must be >= 1");
  if (op->dtype == MUELLER_C64_NEAR64 && !op->near_dev)
    return fail(MUELLER_ERR_INVALID_ARG, "operator lacks its near part");
  if (op->mesh->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  if (mueller_status ts_ = mesh_tables(op->mesh)) return ts_;
  return precond_build(op, block, P, (cudaStream_t)stream);
}

mueller_status mueller_precond_build_batch(int32_t n, const mueller_operator* ops,
                                           const int64_t* blocks, void* const* precond_dev,
                                           void* stream) {
  if (n < 1 || !ops || !blocks || !precond_dev) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument or n < 1");
  for (int32_t b = 0; b < n; ++b) {
    const std::string who = "body " + std::to_string(b) + ": ";
    const mueller_operator* op = &ops[b];
    if (!op->mesh || !op->Z_dev || !precond_dev[b]) return fail(MUELLER_ERR_INVALID_ARG, who + "NULL argument");
    if (mueller_status ts_ = mesh_tables(op->mesh)) return ts_;
    if (blocks[b] < 1) return fail(MUELLER_ERR_INVALID_ARG, who + "block must be >= 1");
    if (op->dtype != MUELLER_C128 && op->dtype != MUELLER_C64_NEAR64)
      return fail(MUELLER_ERR_INVALID_ARG, who + "unknown operator dtype");
    if (op->dtype == MUELLER_C64_NEAR64 && !op->near_dev)
      return fail(MUELLER_ERR_INVALID_ARG, who + "operator lacks its near part");
    if (op->mesh->host_only) return fail(MUELLER_ERR_STATE, who + kHostOnlyMsg);
  }
  return precond_build_batch(n, ops, blocks, precond_dev, (cudaStream_t)stream);
}

size_t mueller_solve_workspace_bytes(const mueller_operator* op, int32_t r,
                                     const mueller_solver_opts* o) {
  if (!op || !o || r < 1 || (op->mesh && mesh_tables(op->mesh))) return 0;
  return solve_work(op, r, o);
}

mueller_status mueller_solve(const mueller_operator* op, const void* B, void* X, int32_t r,
                             const mueller_solver_opts* o, mueller_solve_info* info, void* work,
                             size_t work_bytes, void* stream) {
  if (!op || !op->mesh || !op->Z_dev || !B || !X || !o || !info)
    return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  if (r < 1) return fail(MUELLER_ERR_INVALID_ARG, "r must be >= 1");
  if (o->mode < 0 || o->mode > 2) return fail(MUELLER_ERR_INVALID_ARG, "unknown solve mode");
  if (o->mode != MUELLER_SOLVE_DENSE_LU && (o->restart < 1 || o->maxit < 1 || !(o->tol > 0)))
    return fail(MUELLER_ERR_INVALID_ARG, "restart, maxit and tol must be positive");
  if (o->mode == MUELLER_SOLVE_DENSE_LU && op->dtype != MUELLER_C128)
    return fail(MUELLER_ERR_INVALID_ARG, "dense LU needs a complex128 operator");
  if (o->mode == MUELLER_SOLVE_GMRES_IR && op->dtype != MUELLER_C64_NEAR64)
    return fail(MUELLER_ERR_INVALID_ARG, "GMRES_IR needs a C64_NEAR64 operator");
  if (o->use_precond && !op->precond_dev)
    return fail(MUELLER_ERR_INVALID_ARG, "use_precond set but operator has no precond_dev");
  if ((op->flags & MUELLER_OP_ADJOINT) &&
      (op->dtype != MUELLER_C128 || o->mode != MUELLER_SOLVE_GMRES))
    return fail(MUELLER_ERR_INVALID_ARG,
                "the adjoint operator needs a complex128 operator and MUELLER_SOLVE_GMRES");
  if (op->mesh->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  if (mueller_status ts_ = mesh_tables(op->mesh)) return ts_;
  size_t need = solve_work(op, r, o);
  if (work && work_bytes < need) return fail(MUELLER_ERR_INVALID_ARG, "workspace too small");
  auto t0 = std::chrono::steady_clock::now();
  mueller_status st = solve(op, B, X, r, o, info, work, work_bytes, (cudaStream_t)stream);
  info->t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

size_t mueller_matvec_workspace_bytes(const mueller_operator* op, int32_t r) {
  if (!op || r < 1) return 0;
  return op_matvec_work(op, r);
}

mueller_status mueller_matvec(const mueller_operator* op, const void* X, void* Y, int32_t r,
                              void* work, size_t work_bytes, void* stream) {
  if (!op || !op->mesh || !op->Z_dev || !X || !Y) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  if (r < 1) return fail(MUELLER_ERR_INVALID_ARG, "r must be >= 1");
  if (op->dtype == MUELLER_C64_NEAR64 && !op->near_dev)
    return fail(MUELLER_ERR_INVALID_ARG, "operator lacks its near part");
  if ((op->flags & MUELLER_OP_ADJOINT) && op->dtype != MUELLER_C128)
    return fail(MUELLER_ERR_INVALID_ARG, "the adjoint operator needs a complex128 operator");
  if (op->mesh->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  if (mueller_status ts_ = mesh_tables(op->mesh)) return ts_;
  if (work && work_bytes < op_matvec_work(op, r)) return fail(MUELLER_ERR_INVALID_ARG, "workspace too small");
  return op_matvec(op, X, Y, r, work, work_bytes, (cudaStream_t)stream);
}

size_t mueller_matvec_mrhs_workspace_bytes(const mueller_operator* op, int32_t r) {
  if (!op || !op->mesh || r < 1) return 0;
  return mrhs_work_bytes(4 * op->mesh->nn, r);
}

mueller_status mueller_matvec_mrhs(const mueller_operator* op, const void* X, void* Y, int32_t r,
                                   void* work, size_t work_bytes, void* stream) {
  if (!op || !op->mesh || !op->Z_dev || !X || !Y) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  if (op->dtype != MUELLER_C64_NEAR64 || !op->near_dev)
    return fail(MUELLER_ERR_INVALID_ARG, "the tensor-core product needs a C64_NEAR64 operator");
  if (op->mesh->host_only) return fail(MUELLER_ERR_STATE, kHostOnlyMsg);
  if (mueller_status ts_ = mesh_tables(op->mesh)) return ts_;
  const int64_t N = 4 * op->mesh->nn;
  if (r < 1 || r > 128) return fail(MUELLER_ERR_INVALID_ARG, "r must be in 1..128");
  if (!work || work_bytes < mrhs_work_bytes(N, r))
    return fail(MUELLER_ERR_INVALID_ARG, "workspace missing or too small");
  cudaStream_t s = (cudaStream_t)stream;
  mueller_status st = mrhs_matvec_c64(op->Z_dev, N, op->ldz, X, Y, r, work, s, nullptr,
                                      (op->flags & MUELLER_OP_K1_MIRRORED) ? 1 : 0);
  if (!st) st = near_apply_c64(op->mesh, op->near_dev, X, Y, r, s);
  if (!st) st = mrhs_check_error(work, N, r, s);
  return st;
}

mueller_status mueller_far_field(mueller_mesh* m, const mueller_params* p, const void* X,
                                 int32_t r, const double* inc, const double* dirs, int64_t ndir,
                                 void* F, double* xs, int32_t n_theta, int32_t n_phi,
                                 void* stream) {
  if (!m || !X || !inc || !xs) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  mueller_status st = check_params(p);
  if (st) return st;
  if (r < 1 || ndir < 0 || (ndir > 0 && (!dirs || !F))) return fail(MUELLER_ERR_INVALID_ARG, "bad r/n_dir");
  if (n_theta < 2 || n_phi < 3 || n_theta > 512 || n_phi > 1024)
    return fail(MUELLER_ERR_INVALID_ARG, "n_theta in 2..512, n_phi in 3..1024");
  if ((st = check_inc(inc, r)) || (st = check_dirs(dirs, ndir))) return st;
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_geometry(m, p->q_regular, s);
  if (st) return st;
  return far_field(m, make_phys(p), p->q_regular, X, r, inc, dirs, ndir, F, xs, n_theta, n_phi, s);
}

void mueller_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
}

void mueller_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.clear();
  g_launches = 0;
}

int64_t mueller_launch_count(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_launches;
}

int32_t mueller_profile_get(const char* name, double* total_ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!name) return 0;
  auto it = g_prof.find(name);
  if (it == g_prof.end()) {
    if (total_ms) *total_ms = 0.0;
    if (launches) *launches = 0;
    return 0;
  }
  if (total_ms) *total_ms = it->second.first;
  if (launches) *launches = it->second.second;
  return 1;
}

int32_t mueller_profile_names(char* buf, size_t buflen) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::string all;
  for (auto& kv : g_prof) all += kv.first + "\n";
  if (buf && buflen) {
    size_t n = std::min(buflen - 1, all.size());
    memcpy(buf, all.data(), n);
    buf[n] = 0;
  }
  return (int32_t)g_prof.size();
}

mueller_status mueller_far_field_noalloc(mueller_mesh* m, const mueller_params* p,
                                         const void* X, int32_t r, const double* inc,
                                         const double* dirs, int64_t ndir, void* F, double* xs,
                                         int32_t n_theta, int32_t n_phi, void* stream) {
  if (!m || !X || !inc || !xs) return fail(MUELLER_ERR_INVALID_ARG, "NULL argument");
  mueller_status st = check_params(p);
  if (st) return st;
  if (r < 1 || ndir < 0 || (ndir > 0 && (!dirs || !F))) return fail(MUELLER_ERR_INVALID_ARG, "bad r/n_dir");
  if (n_theta < 2 || n_phi < 3 || n_theta > 512 || n_phi > 1024)
    return fail(MUELLER_ERR_INVALID_ARG, "n_theta in 2..512, n_phi in 3..1024");
  if ((st = check_inc(inc, r)) || (st = check_dirs(dirs, ndir))) return st;
  // the point geometry is allocated by mueller_assemble / mueller_far_field;
  // this variant never allocates, so it must already exist for the rule
  if (!m->has_frame || p->frame_rule != m->frame_rule || m->qd_q != p->q_regular)
    return fail(MUELLER_ERR_STATE, "call mueller_assemble (or mueller_far_field) with these "
                                   "params on this mesh first");
  if (mueller_status ts_ = mesh_tables(m)) return ts_;
  return far_field_noalloc(m, make_phys(p), p->q_regular, X, r, inc, dirs, ndir, F, xs, n_theta,
                           n_phi, (cudaStream_t)stream);
}

mueller_status mueller_sync(void* stream) {
  MU_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return MUELLER_OK;
}

}  // extern "C"
