// Internal declarations shared by the translation units of libmueller.so.
// Not part of the public ABI (include/mueller.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mueller.h"

namespace mu {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
mueller_status cuda_fail(cudaError_t e, const char* what);

#define MU_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return mu::cuda_fail(e_, #call); \
  } while (0)

#define MU_CHECK_LAUNCH(what)                                \
  do {                                                       \
    cudaError_t e_ = cudaGetLastError();                     \
    if (e_ != cudaSuccess) return mu::cuda_fail(e_, what);   \
  } while (0)

// ----------------------------------------------------- launch profiling
// Every kernel launch is wrapped in a Prof scope: it counts the launch and,
// when profiling is enabled (mueller_profile_enable), records CUDA events
// around the launch on its stream, waits for the end event and accumulates
// the elapsed time under the kernel's name.
class Prof {
 public:
  Prof(const char* name, cudaStream_t s);
  ~Prof();

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// --------------------------------------------------- quadrature tables
// Triangle rule on the reference simplex (weights sum to 1/2) and Gauss-
// Legendre on [0,1]; derived on the host (see quadrature.cu).
struct TriangleRule {
  int q = 0;
  std::vector<double> xi, eta, w;
};
bool triangle_rule(int q, TriangleRule& out);
void gauss_legendre_unit(int n, std::vector<double>& x, std::vector<double>& w);

// Per-point record of the regular-rule geometry (Sec. 3.3):
// x(3) n(3) t1(3) t2(3) s1(3) s2(3) W = w*J (1), padded to 20 values.
constexpr int QD_STRIDE = 20;
constexpr int MAX_Q = 12;
constexpr int MAX_NS = 16;

// touching pair record: ex, ey, class, packed relabellings (px | py << 8,
// each 3 x 2 bits)
struct TouchPair {
  int32_t ex, ey, cls, perm;
};

}  // namespace mu

// ---------------------------------------------------------------- handle
struct mueller_mesh {
  int64_t nn = 0, nt = 0;
  std::vector<int32_t> node_perm, elem_perm;
  std::vector<double> X_h;   // Morton order
  std::vector<int32_t> T_h;  // Morton order
  // device copies
  double* X = nullptr;        // nn x 3
  int32_t* T = nullptr;       // nt x 6
  int32_t* n2e_ptr = nullptr; // nn + 1
  int32_t* n2e = nullptr;     // (element << 3) | local node index
  double* frame = nullptr;    // nn x 9
  bool has_frame = false;
  int frame_rule = 0;
  // regular-rule point geometry, cached per rule
  int qd_q = 0;
  double* qd64 = nullptr;     // nt x Q x QD_STRIDE
  float* qd32 = nullptr;
  double min_gs = 0.0;
  // touching pairs and the near-part block layout
  int64_t n_touch = 0;
  mu::TouchPair* tp = nullptr;
  int64_t nnzb = 0;
  int32_t* near_rowptr = nullptr;  // nn + 1
  int32_t* near_col = nullptr;     // nnzb
  int32_t* tp_slot = nullptr;      // n_touch x 36 near slots of the pair's node pairs
  int32_t* tp_order = nullptr;     // pair indices: coincident and common-edge first
  int64_t n_touch_ce = 0;          // how many of them come before the common-vertex pairs
  std::vector<int32_t> near_rowptr_h, near_col_h;
  std::vector<mu::TouchPair> tp_h;  // host copies of tp and tp_slot
  std::vector<int32_t> tp_slot_h;
  bool host_only = false;           // loaded with MUELLER_MESH_HOST_ONLY: no device data
  // small device scratch
  int32_t* d_flags = nullptr;      // status words
  double* d_scal = nullptr;        // 64 doubles
  // the host thread that builds the touching pairs and the near layout
  // (and uploads them) after mueller_mesh_load returns; mu::mesh_tables
  // joins it
  mutable std::thread tables_thread;
  mutable std::mutex tables_mu;
  mueller_status tables_st = MUELLER_OK;
  std::string tables_msg;
};

namespace mu {
// The host tables of m (touching pairs, near layout) are ready; their status.
mueller_status mesh_tables(const mueller_mesh* m);
// ----------------------------------------------------------- launchers
// geometry.cu
mueller_status launch_frame(mueller_mesh* m, int frame_rule, cudaStream_t s);
mueller_status launch_quad_geometry(mueller_mesh* m, const TriangleRule& rule, cudaStream_t s);

// assemble.cu
struct PhysConsts {
  double ka;
  double ki_re, ki_im;
  double eps_re, eps_im, mu_re, mu_im;  // interior (exterior = 1)
};
mueller_status upload_rules(const TriangleRule& rule, int ns);
mueller_status launch_regular(mueller_mesh* m, const PhysConsts& P, int Q, int dtype, void* Z,
                              int64_t ldz, cudaStream_t s);
mueller_status launch_touching(mueller_mesh* m, const PhysConsts& P, int Q, int ns, int dtype,
                               void* Z, int64_t ldz, void* near, cudaStream_t s);
// tile-shape choice (autotuned once per precision, rule and mesh size; a
// tuning run adds into Z and zeroes it again) ahead of launch_regular
mueller_status tune_regular(mueller_mesh* m, const PhysConsts& P, int Q, int dtype, void* Z,
                            int64_t ldz, cudaStream_t s);
// the device's high-priority side stream (touching pairs beside the regular
// pairs, panel chain of the block LU beside its trailing updates)
mueller_status side_stream(cudaStream_t* out);
// 'after' waits for the work queued on 'before' so far
mueller_status stream_order(cudaStream_t before, cudaStream_t after);
mueller_status launch_mass_rhs(mueller_mesh* m, const PhysConsts& P, int Q, int dtype, void* Z,
                               int64_t ldz, void* near, void* B, const double* inc_dev, int r,
                               cudaStream_t s);
mueller_status launch_mirror_k1(int64_t N, int dtype, void* Z, int64_t ldz, cudaStream_t s);
mueller_status launch_dz_matvec(mueller_mesh* m, const PhysConsts& P, int Q, int ns, int which,
                                const void* x, void* y, cudaStream_t s);
mueller_status launch_assemble_batch(int nb, mueller_mesh* const* meshes, const PhysConsts* P,
                                     int Q, int ns, int dtype, void* const* Z,
                                     const int64_t* ldz, void* const* near, cudaStream_t s);

// linalg.cu
mueller_status op_matvec(const mueller_operator* op, const void* X, void* Y, int r, void* work,
                         size_t work_bytes, cudaStream_t s);
size_t op_matvec_work(const mueller_operator* op, int r);
mueller_status precond_build(const mueller_operator* op, int64_t block, void* P, cudaStream_t s);
mueller_status precond_build_batch(int n, const mueller_operator* ops, const int64_t* blocks,
                                   void* const* P, cudaStream_t s);
mueller_status solve(const mueller_operator* op, const void* B, void* X, int r,
                     const mueller_solver_opts* o, mueller_solve_info* info, void* work,
                     size_t work_bytes, cudaStream_t s);
size_t solve_work(const mueller_operator* op, int r, const mueller_solver_opts* o);

// mrhs.cu
size_t mrhs_work_bytes(int64_t N, int r);
// stop (device, may be null): nonzero skips the product (a converged solver
// that queued its steps ahead)
// mirrored: Z11 = -Z00 bit for bit (MUELLER_OP_K1_MIRRORED): Z00 is then read
// once for both diagonal blocks where r <= 16
mueller_status mrhs_matvec_c64(const void* Z, int64_t N, int64_t ldz, const void* X, void* Y,
                               int r, void* work, cudaStream_t s, const int* stop = nullptr,
                               int mirrored = 0);
mueller_status mrhs_check_error(void* work, int64_t N, int r, cudaStream_t s);
mueller_status near_apply_c64(const mueller_mesh* m, const void* near_c128, const void* X, void* Y,
                              int r, cudaStream_t s);

// farfield.cu
mueller_status far_field(mueller_mesh* m, const PhysConsts& P, int Q, const void* X, int r,
                         const double* inc, const double* dirs, int64_t ndir, void* F,
                         double* xs, int n_theta, int n_phi, cudaStream_t s);
mueller_status far_field_noalloc(mueller_mesh* m, const PhysConsts& P, int Q, const void* X, int r,
                                 const double* inc, const double* dirs, int64_t ndir, void* F,
                                 double* xs, int n_theta, int n_phi, cudaStream_t s);

PhysConsts make_phys(const mueller_params* p);

// shape_grad.cu: grad (host, n_nodes x 3, input node order) += the gradient
// of Re lam^H Z(X) x with respect to the node coordinates
mueller_status zshape_vjp(mueller_mesh* m, const PhysConsts& P, int Q, int ns, const void* lam,
                          const void* x, int r, double* grad, cudaStream_t s);
// grad (host, n_nodes x 3) += the gradient of Re lam^H b(X)
mueller_status rhs_shape_vjp(mueller_mesh* m, const PhysConsts& P, int Q, const void* lam,
                             const double* inc, double* grad, cudaStream_t s);
// dC/dx (device G, 3 x N, the right-hand sides of Z^H lam = G) and dC/dX at
// fixed x (host grad, 3 x n_nodes x 3, added) for C_ext, C_sca, C_abs
mueller_status cross_section_partials(mueller_mesh* m, const PhysConsts& P, int Q, const void* x,
                                      const double* inc, int n_theta, int n_phi, void* G,
                                      double* grad, double* xs, cudaStream_t s);
}  // namespace mu
