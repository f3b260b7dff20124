/*
 * mueller.h -- C ABI of the GB300 (sm_103a) implementation of the nodal,
 * high-order Galerkin Mueller boundary-integral solver of
 *   Y. Luo, "A High-Order Nodal Galerkin Formulation for the Mueller
 *   Equation: Bypassing Divergence Conformity via Kernel Cancellation",
 *   arXiv 2604.21181.
 *
 * Conventions used by every call
 * ------------------------------
 * Units: exterior eps_a = mu_a = 1, so omega = k_a; interior
 *   eps_i = eps_r, mu_i = mu_r, k_i = k_a sqrt(eps_r mu_r) (principal root).
 *   Time dependence exp(-i omega t) (Sec. 2.1).
 * Mesh: curved six-node (P2) triangles, nodes (v0, v1, v2, m01, m12, m20),
 *   corners counter-clockwise seen from outside (Sec. 3.3).  Inside the
 *   library everything is stored in Morton order (Sec. 5, double Morton
 *   permutation); node_perm[new] = old and elem_perm[new] = old map back.
 * Unknowns: N = 4 * n_nodes.  x = [c_j ; c_jm] (Eq. global_system), each
 *   half indexed 2 * node + alpha (alpha = 0, 1 = tangent t1, t2), nodes in
 *   Morton order.
 * Matrix Z (Eq. global_system): dense, row-major, leading dimension ldz
 *   (elements), row    h*(N/2) + 2*i + alpha  (h = 0 electric equation,
 *   1 magnetic equation), column g*(N/2) + 2*j + beta (g = 0: c_j,
 *   1: c_jm):  Z00 = (i/omega) K1, Z01 = a_eps M + K2^eps,
 *   Z10 = a_mu M + K2^mu, Z11 = -(i/omega) K1, a_chi = (chi_i + chi_a)/2.
 * Complex numbers: interleaved (re, im); complex128 = 2 doubles,
 *   complex64 = 2 floats.
 * Right-hand sides / solutions: r vectors of length N stored one after the
 *   other (vector s at offset s*N).
 * Memory: pointers named *_dev are device pointers owned by the caller
 *   (e.g. torch tensors); pointers without the suffix are host pointers.
 *   The library owns only the mesh handle and what it allocates inside it.
 * Streams: every call takes a cudaStream_t passed as void* (NULL = legacy
 *   default stream) and only enqueues work on it, except where a call is
 *   documented as synchronising.
 * Errors: every call returns a mueller_status; nothing aborts.  The text of
 *   the last error of the calling thread is returned by mueller_last_error().
 *   Asynchronous device faults surface at the next synchronising call.
 */
#ifndef MUELLER_H_
#define MUELLER_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MUELLER_OK = 0,
  MUELLER_ERR_INVALID_ARG = 1,      /* null pointer, bad size or option       */
  MUELLER_ERR_MESH = 2,             /* non-manifold, unoriented, degenerate   */
  MUELLER_ERR_DEGENERATE_FRAME = 3, /* Gram-Schmidt norm below threshold      */
  MUELLER_ERR_SINGULAR_BLOCK = 4,   /* zero pivot in a block-Jacobi block     */
  MUELLER_ERR_NOT_CONVERGED = 5,    /* GMRES hit maxit (info still filled)    */
  MUELLER_ERR_TIMEOUT = 6,          /* a bounded device wait gave up          */
  MUELLER_ERR_CUDA = 7,             /* CUDA runtime error                     */
  MUELLER_ERR_OOM = 8,              /* device allocation failed               */
  MUELLER_ERR_STATE = 9,            /* call order violated (e.g. no frame)    */
  MUELLER_ERR_NAN = 10              /* a right-hand side's residual became NaN
                                       or infinite (named in the message)     */
} mueller_status;

/* Matrix storage types */
enum {
  MUELLER_C128 = 0,       /* dense complex128 Z holding the whole operator */
  MUELLER_C64_NEAR64 = 1  /* dense complex64 Z of the regular (non-touching)
                             element pairs + FP64 near part (touching pairs
                             and mass) in the mesh's block-sparse layout   */
};

/* Solver modes */
enum {
  MUELLER_SOLVE_DENSE_LU = 0,   /* dense LU with partial pivoting (C128 only) */
  MUELLER_SOLVE_GMRES = 1,      /* GMRES(m) in the operator's own precision   */
  MUELLER_SOLVE_GMRES_IR = 2    /* complex64 inner GMRES + FP64 refinement    */
};

/* Reference-axis rule of the nodal tangent frame (Sec. 3.2). */
enum {
  MUELLER_FRAME_PAPER = 0, /* v_ref = x if |n.z| > 0.9 else z (Eqs. t1, t2)  */
  MUELLER_FRAME_POLAR = 1  /* v_ref = z except within 1e-8 of the poles      */
};

/* mueller_mesh_load flags (bits) */
enum {
  MUELLER_MESH_KEEP_ORDER = 1, /* keep the input node and element order      */
  MUELLER_MESH_HOST_ONLY = 2   /* build the host tables only: no device data */
};

/* Quadrature tables (mueller_quadrature_rule) */
enum {
  MUELLER_RULE_TRIANGLE = 0,       /* symmetric rule on the reference triangle */
  MUELLER_RULE_GAUSS_LEGENDRE = 1  /* Gauss-Legendre on [0, 1]                 */
};

typedef struct mueller_mesh mueller_mesh;

typedef struct {
  double ka;          /* exterior wavenumber k_a = omega                     */
  double eps_r[2];    /* interior relative permittivity (re, im)            */
  double mu_r[2];     /* interior relative permeability (re, im)            */
  int32_t q_regular;  /* triangle rule: 6 (degree 4) or 12 (degree 6)        */
  int32_t ssq_order;  /* Sauter-Schwab Gauss points per dimension, 1..16    */
  int32_t frame_rule; /* MUELLER_FRAME_*                                     */
  int32_t reserved;   /* must be 0                                           */
} mueller_params;

typedef struct {
  int64_t n_nodes, n_tri, n_dof;
  int64_t n_touching;   /* ordered touching element pairs (incl. coincident) */
  int64_t n_near_blocks;/* node-pair blocks of the near part                 */
  double min_gs_norm;   /* smallest Gram-Schmidt norm (after tangent_frame)  */
} mueller_mesh_info;

typedef struct {
  int32_t mode;        /* MUELLER_SOLVE_*                                    */
  int32_t restart;     /* GMRES restart length m (>= 1)                      */
  int32_t maxit;       /* total Arnoldi steps allowed (per RHS)              */
  int32_t warm_start;  /* nonzero: X_dev holds x0 on entry                   */
  double tol;          /* ||b - Zx|| <= tol ||b|| (FP64, on the stored operator) */
  double inner_tol;    /* GMRES_IR: relative tolerance of each inner solve   */
  int32_t max_refine;  /* GMRES_IR: outer refinement steps allowed           */
  int32_t use_precond; /* nonzero: right Morton block-Jacobi preconditioner  */
} mueller_solver_opts;

typedef struct {
  int32_t iters;       /* Arnoldi steps, summed over RHS                     */
  int32_t restarts;    /* restart cycles, summed over RHS                    */
  int32_t refinements; /* GMRES_IR outer steps, summed over RHS              */
  int32_t converged;   /* number of RHS that reached tol                     */
  double relres;       /* worst final FP64 relative residual over the RHS    */
  double t_ms;         /* wall time of the call                              */
} mueller_solve_info;

/* Operator flag: Z11 equals -Z00 bit for bit, as mueller_assemble and
 * mueller_assemble_batch write it (both are +-(i/omega) K1, Eq.
 * global_system).  The complex64 single-vector products of the inner GMRES
 * then read Z00 in place of Z11: three quarters of Z per product instead of
 * all of it.  Leave it clear for a Z that was changed or written by other
 * means. */
#define MUELLER_OP_K1_MIRRORED 1

/* Operator flag: the call works with the adjoint Z^H instead of Z (and a
 * preconditioner built from Z applied as (P^{-1})^H, the block-Jacobi
 * preconditioner of Z^H).  For the adjoint solves of the gradients (Z^H lam
 * = g^*).  Complex128 operators only, with mueller_matvec and mueller_solve
 * in MUELLER_SOLVE_GMRES mode (else INVALID_ARG). */
#define MUELLER_OP_ADJOINT 2

/* The operator handed to the preconditioner and the solver. */
typedef struct {
  const mueller_mesh* mesh; /* for the near-part layout (C64_NEAR64)         */
  const void* Z_dev;        /* dense Z, dtype below, row-major, ldz          */
  int64_t ldz;
  int32_t dtype;            /* MUELLER_C128 or MUELLER_C64_NEAR64            */
  int32_t flags;            /* MUELLER_OP_* bits (0 = none)                  */
  const void* near_dev;     /* complex128 near blocks (C64_NEAR64) or NULL   */
  const void* precond_dev;  /* factors from mueller_precond_build or NULL    */
  int64_t block;            /* cluster size B used to build precond_dev      */
} mueller_operator;

/*
 * mueller_quadrature_rule -- the quadrature tables the library derives on the
 * host and uses: the regular-pair triangle rules (Sec. 5.1; 6 points of
 * degree 4, 12 points of degree 6, from their moment equations) and
 * Gauss-Legendre (the Sauter-Schwab tensor rules of Sec. 4.2, the far-field
 * sphere rule in cos(theta)).  Host outputs of n entries:
 *   MUELLER_RULE_TRIANGLE        n = 6 or 12; a = xi, b = eta on the
 *                                reference triangle {xi, eta >= 0,
 *                                xi + eta <= 1}; w sums to its area 1/2.
 *   MUELLER_RULE_GAUSS_LEGENDRE  n in 1..512; a = nodes on [0, 1] ascending,
 *                                w sums to 1; b unused (may be NULL).
 * Errors: INVALID_ARG (kind, n, NULL outputs).
 */
mueller_status mueller_quadrature_rule(int32_t kind, int32_t n, double* a, double* b, double* w);

/* Library version; text of the calling thread's last error. */
int32_t mueller_version(void);
const char* mueller_last_error(void);
const char* mueller_status_string(mueller_status s);

/*
 * mueller_mesh_load -- Sec. 3.3 (P2 isoparametric mesh) and Sec. 5 (double
 * Morton permutation).  Validates the mesh (every corner edge shared by two
 * triangles with opposite orientation and the same edge node, finite
 * coordinates, non-degenerate elements), computes the Morton node and element
 * orders (21-bit keys in the node bounding box scaled by its largest extent,
 * x in the least significant bit, ties by original index; elements keyed by
 * the centroid of their corners), classifies the touching element pairs
 * (shared corners: 3 coincident, 2 common edge, 1 common vertex), lays out
 * the near-part blocks and uploads everything to the device.  The node and
 * element arrays are uploaded on 'stream' before the call returns; the
 * touching pairs and the near layout are built and uploaded by a host thread
 * of the library after it returns, so that the frame, point-geometry and
 * regular-pair launches of the caller need not wait for them.  Every call
 * that reads them (mueller_mesh_get_info, mueller_mesh_touching,
 * mueller_mesh_near_layout, mueller_near_bytes, the touching-pair part of
 * mueller_assemble, and the calls after it) waits for that thread first and
 * returns its error, if it had one; mueller_mesh_free waits for it too.
 *   xyz   host, n_nodes x 3 float64, read only, copied.
 *   tri6  host, n_tri x 6 int32 node ids, read only, copied.
 *   flags MUELLER_MESH_KEEP_ORDER: keep the input order (no Morton
 *         permutation).  MUELLER_MESH_HOST_ONLY: validate and build the
 *         host tables (orders, touching pairs, near-block layout) but touch
 *         no device: the handle serves mueller_mesh_get_info,
 *         mueller_mesh_perm, mueller_mesh_touching, mueller_mesh_near_layout
 *         and mueller_near_bytes; calls that need device data return STATE.
 *   out   receives the handle (owned by the library; free with
 *         mueller_mesh_free).
 * Errors: INVALID_ARG (null/sizes), MESH (validation), OOM, CUDA.
 */
mueller_status mueller_mesh_load(const double* xyz, int64_t n_nodes, const int32_t* tri6,
                                 int64_t n_tri, int32_t flags, void* stream,
                                 mueller_mesh** out);
void mueller_mesh_free(mueller_mesh* mesh);
mueller_status mueller_mesh_get_info(const mueller_mesh* mesh, mueller_mesh_info* info);
/*
 * mueller_point_records -- the point geometry of the regular rule (Sec. 3.3)
 * that the assembly and the far field use: per element (the mesh's element
 * order) and rule point, 19 doubles: x (3), the unit normal n (3), the
 * continuous frame t1, t2 (3 each), the co-normals s1 = t1 x n, s2 = t2 x n
 * (3 each), and the rule weight times the surface Jacobian.  For tests and
 * inspection.
 *   q_regular  6 or 12: the rule of the last mueller_assemble / mueller_far_field
 *              on this mesh (else STATE).
 *   out        host, n_tri x q_regular x 19 doubles.  Synchronous.
 * Errors: INVALID_ARG, STATE, CUDA.
 */
mueller_status mueller_point_records(const mueller_mesh* mesh, int32_t q_regular, double* out);
/* host outputs: node_perm[n_nodes], elem_perm[n_tri] (new -> old); either may be NULL */
mueller_status mueller_mesh_perm(const mueller_mesh* mesh, int32_t* node_perm,
                                 int32_t* elem_perm);

/*
 * mueller_mesh_touching -- Sec. 4.2: the touching element pairs the
 * Sauter-Schwab quadrature takes, in the order the library keeps them
 * (test element ascending, then trial element), n_touching entries per
 * output (host arrays, any may be NULL; element ids in the mesh's order):
 *   ex, ey   test and trial element;
 *   cls      shared corners: 3 coincident, 2 common edge, 1 common vertex;
 *   relabel  the corner relabellings of the two elements, packed: bits
 *            2k..2k+1 hold the test element's local corner that becomes
 *            corner k of the relabelled triangle, bits 8+2k..9+2k the trial
 *            element's (k = 0, 1, 2).  Common edge: the shared edge is
 *            corners 0 -> 1 as it runs in the test element; common vertex:
 *            the shared corner is corner 0 of both, the others follow
 *            cyclically; coincident: identity.
 * Errors: INVALID_ARG (mesh NULL).
 */
mueller_status mueller_mesh_touching(const mueller_mesh* mesh, int32_t* ex, int32_t* ey,
                                     int32_t* cls, int32_t* relabel);

/*
 * mueller_mesh_near_layout -- the block layout of the near part (the node
 * pairs of the touching element pairs, Eq. global_system split into the
 * far part in Z and the near blocks): host outputs, any may be NULL,
 *   rowptr  n_nodes + 1: blocks of test node i are rowptr[i] .. rowptr[i+1]-1;
 *   col     n_near_blocks: their trial nodes, ascending within a row;
 *   slot    36 n_touching: slot[(p*6 + i)*6 + j] is the block of the node
 *           pair (node i of ex_p, node j of ey_p) of touching pair p.
 * Errors: INVALID_ARG (mesh NULL).
 */
mueller_status mueller_mesh_near_layout(const mueller_mesh* mesh, int32_t* rowptr, int32_t* col,
                                        int32_t* slot);

/*
 * mueller_tangent_frame -- Sec. 3.1 Eq. (U_contribution) and Sec. 3.2
 * Eqs. (t1), (t2): metric-weighted nodal normal n_v = sum U / |sum U| with
 * U = (a1 x a2)/(g11 g22) (corner nodes: the element relabelled so that the
 * node is the parametric origin; edge nodes: canonical derivatives), then
 * t1 = v_ref x n/|.|, t2 = n x t1 with the given frame_rule.  Stores the
 * frame in the handle.
 *   frame_dev  optional device output, n_nodes x 9 float64 (n, t1, t2).
 * Errors: INVALID_ARG, CUDA.
 */
mueller_status mueller_tangent_frame(mueller_mesh* mesh, int32_t frame_rule, double* frame_dev,
                                     void* stream);

/*
 * mueller_assemble -- Sec. 4 (Eqs. kappa1_alphabeta, K1_matrix_entry,
 * Hdiff_exact, kappa_S, kappa2_alpha_beta, K2_matrix_entry, kappa2_S,
 * global_system, mass_matrix, rhs_E, rhs_H) and Sec. 5.1 (fused pass).
 * Regular element pairs: product rule q_regular x q_regular with the exact
 * kernels evaluated through a stable series at |k R| < 1.  Touching pairs:
 * the singular parts (Eqs. kappa_S, kappa2_S) by Sauter-Schwab quadrature of
 * order ssq_order, the remainder kappa - kappa^s by the product rule.
 *   dtype    MUELLER_C128: Z_dev = complex128 N x ldz, whole operator.
 *            MUELLER_C64_NEAR64: Z_dev = complex64 N x ldz with the regular
 *            pairs (computed in FP32), near_dev = complex128 near blocks
 *            (mueller_near_bytes) with touching pairs and mass (FP64).
 *   Z_dev, near_dev are overwritten (zeroed first).
 *   B_dev    optional complex128 r x N right-hand sides (Eqs. rhs_E, rhs_H)
 *            for the plane waves inc (host, r x 6: k-hat, real p-hat with
 *            p.k = 0; E_inc = p exp(i k_a k.x), H_inc = k x E_inc; rows not
 *            orthonormal to 1e-10 are refused with INVALID_ARG).
 * Requires mueller_tangent_frame first (else STATE).
 * Errors: INVALID_ARG, STATE, DEGENERATE_FRAME, CUDA.
 */
mueller_status mueller_assemble(mueller_mesh* mesh, const mueller_params* params, int32_t dtype,
                                void* Z_dev, int64_t ldz, void* near_dev, void* B_dev,
                                const double* inc, int32_t r, void* stream);
/*
 * mueller_assemble_batch -- what mueller_assemble computes, for n_bodies
 * bodies at once: the regular pairs of every body run in one kernel launch
 * and the touching pairs of every body in another (a work list of (body,
 * tile) and (body, pair) entries, largest bodies first), so that many small
 * bodies fill the GPU together.  The paper treats one body; batching many
 * scatterers is an extension of this library.
 *   meshes[b], params[b]   one loaded mesh (mueller_tangent_frame done) and
 *            its parameters per body; every body must use the same q_regular
 *            and ssq_order (else INVALID_ARG); k_a, eps_r, mu_r may differ.
 *   dtype    as in mueller_assemble, for every body.
 *   Z[b], ldz[b], near[b]   per-body outputs as in mueller_assemble (near may
 *            be NULL for MUELLER_C128).
 *   B, inc, r   optional (all NULL, or all given): B[b] may be NULL for a
 *            body without right-hand sides; else inc[b] (host, r[b] x 6,
 *            orthonormal rows as for mueller_assemble).
 * Errors: INVALID_ARG (naming the body), STATE, DEGENERATE_FRAME, CUDA.
 */
mueller_status mueller_assemble_batch(int32_t n_bodies, mueller_mesh* const* meshes,
                                      const mueller_params* params, int32_t dtype,
                                      void* const* Z_dev, const int64_t* ldz,
                                      void* const* near_dev, void* const* B_dev,
                                      const double* const* inc, const int32_t* r, void* stream);

/*
 * mueller_dz_matvec -- Y = (dZ/dtheta) X for theta = eps_r (which = 1) or
 * mu_r (which = 2): the complex derivative of the operator of Eq.
 * global_system (Z is holomorphic in eps_r and mu_r through
 * k_i = k_a sqrt(eps_r mu_r) and the explicit eps_r, mu_r factors of the
 * kernels of Eqs. kappa_S, kappa2_S and of the mass terms), applied to one
 * vector without forming dZ: every element pair's block of dZ is recomputed
 * from the derivatives of the radial functions (FP64) and multiplied into Y.
 * Used for the gradients of the cross sections with respect to the material.
 *   X_dev    complex128, length N = 4 * n_nodes, read only.
 *   Y_dev    complex128, length N, overwritten.
 * Needs mueller_tangent_frame with params->frame_rule (else STATE).
 * Errors: INVALID_ARG (NULL, which not 1 or 2, bad params), STATE, CUDA.
 */
mueller_status mueller_dz_matvec(mueller_mesh* mesh, const mueller_params* params, int32_t which,
                                 const void* X_dev, void* Y_dev, void* stream);

/*
 * mueller_zshape_vjp -- the gradient of Re lam^H Z(X) x with respect to the
 * node coordinates X (the operator of Eq. global_system as a function of
 * the P2 geometry, Sec. 3), for given lam and x: the term of the adjoint
 * relation dC/dX = dC/dX|_x + 2 Re lam^H (db/dX - (dZ/dX) x) that involves
 * the operator.  Every element pair's kernel values are recomputed with
 * their derivatives with respect to the point geometry (regular pairs,
 * touching-pair remainders, the Sauter-Schwab integrals of the singular
 * parts, the mass term) and contracted with lam and x; the adjoints are
 * carried back through the continuous frame (Sec. 3.3), the nodal frame
 * (Sec. 3.2) and the metric-weighted nodal normal (Sec. 3.1) to the node
 * positions.  No derivative of Z is stored.  FP64.
 *   lam_dev, X_dev  complex128, length N = 4 n_nodes, the mesh's unknown
 *                   order; read only.
 *   grad            host, n_nodes x 3, the node order of the mesh's input
 *                   (node_perm applied); overwritten.  Synchronising.
 * Needs mueller_tangent_frame with params->frame_rule (else STATE).
 * Errors: INVALID_ARG, STATE, OOM, CUDA.
 */
mueller_status mueller_zshape_vjp(mueller_mesh* mesh, const mueller_params* params,
                                  const void* lam_dev, const void* X_dev, double* grad,
                                  void* stream);

/*
 * mueller_zshape_vjp_multi -- mueller_zshape_vjp for r adjoint vectors at
 * once (the gradients of several outputs at one solution x): the regular-pair
 * and remainder passes evaluate each point pair's radial functions, and the
 * Sauter-Schwab passes each point's geometry, once for up to three of them.
 *   lam_dev  complex128, r x N (vector o at lam_dev + o N); read only.
 *   r        >= 1.
 *   grad     host, r x n_nodes x 3 (vector o's gradient at grad + 3 o n_nodes),
 *            the node order of the mesh's input; overwritten.  Synchronising.
 * Errors: as mueller_zshape_vjp, and INVALID_ARG for r < 1.
 */
mueller_status mueller_zshape_vjp_multi(mueller_mesh* mesh, const mueller_params* params,
                                        const void* lam_dev, int32_t r, const void* X_dev,
                                        double* grad, void* stream);

/*
 * mueller_rhs_shape_vjp -- the gradient of Re lam^H b(X) with respect to
 * the node coordinates X, b the plane-wave right-hand side of Eqs. (rhs_E),
 * (rhs_H) for the incident wave inc (host, 6: k-hat, p-hat, orthonormal):
 * the db/dX term of the adjoint relation of mueller_zshape_vjp.  The
 * derivatives of the rule points, weights and test frames are carried back
 * to the node positions as there.  FP64.
 *   lam_dev  complex128, length N = 4 n_nodes, the mesh's unknown order.
 *   grad     host, n_nodes x 3, input node order; overwritten.  Synchronising.
 * Needs mueller_tangent_frame with params->frame_rule (else STATE).
 * Errors: INVALID_ARG, STATE, OOM, CUDA.
 */
mueller_status mueller_rhs_shape_vjp(mueller_mesh* mesh, const mueller_params* params,
                                     const void* lam_dev, const double* inc, double* grad,
                                     void* stream);

/*
 * mueller_cross_section_partials -- the partial derivatives of the three
 * cross sections of mueller_far_field (C_ext, C_sca, C_abs, in that order)
 * for one solution x and incident wave inc:
 *   G_dev  device complex128 3 x N output: row o is conj(dC_o/dx), with
 *          dC_o = 2 Re sum_u (dC_o/dx_u) dx_u for a change dx of x at fixed
 *          geometry -- the right-hand side of the adjoint system
 *          Z^H lam_o = G_o (mueller_solve with MUELLER_OP_ADJOINT).
 *   grad   host 3 x n_nodes x 3 output: dC_o/dX at fixed x (through the
 *          rule points, weights, normals and current frames), input node
 *          order; overwritten.
 *   xs     host 3 output (may be NULL): C_ext, C_sca, C_abs of x, computed
 *          on the same rules.
 * C_sca uses the sphere rule of mueller_far_field (n_theta Gauss-Legendre
 * nodes in cos(theta) x n_phi trapezoid steps in phi).  With
 * mueller_zshape_vjp and mueller_rhs_shape_vjp this gives the shape
 * gradient dC_o/dX = grad_o + 2 Re(rhs_vjp(lam_o) - zshape_vjp(lam_o, x)).
 * Synchronising.  Needs mueller_tangent_frame with params->frame_rule.
 * Errors: INVALID_ARG, STATE, OOM, CUDA.
 */
mueller_status mueller_cross_section_partials(mueller_mesh* mesh, const mueller_params* params,
                                              const void* X_dev, const double* inc,
                                              int32_t n_theta, int32_t n_phi, void* G_dev,
                                              double* grad, double* xs, void* stream);

/* bytes of the complex128 near-part buffer of a loaded mesh */
size_t mueller_near_bytes(const mueller_mesh* mesh);

/*
 * mueller_precond_build -- Sec. 5, Eq. (precond_block): the Morton block
 * Jacobi preconditioner.  Per-current indices (2*node + alpha) are split into
 * ceil((N/2)/block) contiguous clusters I_m (the last one smaller); block m
 * is the 2|I_m| x 2|I_m| restriction of the operator to I_m in both halves
 * (all four quadrants).  Each block is factorised by LU with partial
 * pivoting in FP64 and stored as its explicit inverse: complex128 for a
 * C128 operator, complex64 (formed from the FP64 factors) for a
 * C64_NEAR64 operator.  Layout: the inverses [nb][d][d] row-major,
 * d = 2 min(block, N/2), entries beyond a block's own size zero; then the
 * nb block sizes (int32).
 *   precond_dev  caller-owned, mueller_precond_bytes(N, block) bytes.
 *   status_dev   optional device int32: set to the first singular block + 1.
 * The operator's precond_dev/block fields are ignored.
 * Errors: INVALID_ARG, SINGULAR_BLOCK (checked when the call synchronises:
 * it reads the pivot status before returning), CUDA.
 */
mueller_status mueller_precond_build(const mueller_operator* op, int64_t block,
                                     void* precond_dev, void* stream);
size_t mueller_precond_bytes(int64_t n_dof, int64_t block);

/*
 * mueller_precond_build_batch -- what mueller_precond_build computes, for n
 * operators (bodies) at once: the blocks of every body (Sec. 5, Eq.
 * precond_block; block dimension 2 min(block[b], N_b / 2)) are gathered
 * into one batch and factorised by one batched FP64 LU, so that many small
 * bodies fill the GPU together.  Bodies whose block dimension or dtype
 * differ from the others' go into batches of their own.  The paper treats
 * one body; batching many scatterers is an extension of this library.
 *   ops[b], block[b]  as in mueller_precond_build, one per body.
 *   precond_dev[b]    caller-owned, mueller_precond_bytes(N_b, block[b])
 *                     bytes, the same layout as mueller_precond_build.
 * Synchronising.  Errors: INVALID_ARG (naming the body), STATE,
 * SINGULAR_BLOCK (naming the body and block), OOM, CUDA.
 */
mueller_status mueller_precond_build_batch(int32_t n, const mueller_operator* ops,
                                           const int64_t* block, void* const* precond_dev,
                                           void* stream);

/*
 * mueller_solve -- Sec. 5 (GMRES with right block-Jacobi preconditioning)
 * and the mixed-precision refinement.  Solves Z X = B for r right-hand
 * sides.  Synchronising: returns when X is final.
 *   B_dev, X_dev  complex128 r x N (X_dev holds x0 if opts->warm_start).
 *   work_dev      caller scratch of mueller_solve_workspace_bytes() bytes, or
 *                 NULL to let the call allocate (and free) it on the stream.
 *   info          host, filled on OK, NOT_CONVERGED and NAN.
 * GMRES_IR (the complex64 inner solver, all right-hand sides in lockstep)
 * tests convergence on the device and reads it back every few Arnoldi
 * steps; steps queued past convergence do no work.
 * Errors: INVALID_ARG, NOT_CONVERGED, NAN (a right-hand side's Arnoldi
 * estimate or FP64 residual was NaN or infinite: it is frozen, the others
 * are solved, the message names the first such right-hand side),
 * SINGULAR_BLOCK, TIMEOUT (a bounded device wait gave up), OOM, CUDA.
 */
mueller_status mueller_solve(const mueller_operator* op, const void* B_dev, void* X_dev,
                             int32_t r, const mueller_solver_opts* opts, mueller_solve_info* info,
                             void* work_dev, size_t work_bytes, void* stream);
size_t mueller_solve_workspace_bytes(const mueller_operator* op, int32_t r,
                                     const mueller_solver_opts* opts);

/*
 * mueller_matvec -- Y = Z X for r vectors (complex128 in and out), in FP64
 * arithmetic on the operator's storage (C128: complex128 Z; C64_NEAR64:
 * complex64 Z read as exact values plus the FP64 near blocks).  This is the
 * refinement residual product; exposed for tests and benchmarks.
 *   work_dev  NULL or scratch of mueller_matvec_workspace_bytes() bytes.
 */
mueller_status mueller_matvec(const mueller_operator* op, const void* X_dev, void* Y_dev,
                              int32_t r, void* work_dev, size_t work_bytes, void* stream);
size_t mueller_matvec_workspace_bytes(const mueller_operator* op, int32_t r);

/*
 * mueller_matvec_mrhs -- Y = Z X for r = 1..128 complex64 vectors (r x N in
 * and out) of a C64_NEAR64 operator on the tensor cores: the complex64 far
 * part as a real GEMM on tcgen05 (kind::tf32, each operand split into a TF32
 * head and remainder, three products, FP32 accumulation in tensor memory),
 * plus the near blocks in FP32.  Accuracy is that of an FP32 product
 * (relative error ~1e-6).  This is the product of the multi-RHS inner GMRES
 * (the paper's GMRES matvec, Sec. 5, for many incidences at once).
 *   work_dev  mueller_matvec_mrhs_workspace_bytes(op, r) bytes of scratch.
 * Synchronising (reads the kernel's error word).  Errors: INVALID_ARG,
 * TIMEOUT (a pipeline wait in the kernel gave up), CUDA.
 */
mueller_status mueller_matvec_mrhs(const mueller_operator* op, const void* X_dev, void* Y_dev,
                                   int32_t r, void* work_dev, size_t work_bytes, void* stream);
size_t mueller_matvec_mrhs_workspace_bytes(const mueller_operator* op, int32_t r);

/*
 * mueller_far_field -- scattered far field of the solved currents and the
 * cross sections (the paper reports C_ext, C_sca, C_abs and their balance;
 * the formulas follow from the current definitions of Sec. 2.1):
 *   F(r) = (i k_a/4 pi)[(N~ - r (r.N~)) - r x L~],
 *   N~ = int j e^{-i k_a r.y}, L~ = int j_m e^{-i k_a r.y};
 *   C_ext = (4 pi/k_a) Im(p . F(k)), C_sca = int |F|^2 dOmega
 *   (Gauss-Legendre n_theta in cos(theta) x n_phi trapezoid in phi),
 *   C_abs = Re int j_m . (conj(j) x n).
 *   X_dev    complex128 r x N solutions.
 *   inc      host r x 6 incident waves (for C_ext), orthonormal rows
 *            (k-hat, p-hat) as for mueller_assemble.
 *   dirs     host n_dir x 3 unit directions (may be NULL if n_dir == 0;
 *            squared norms off 1 by more than 1e-10 give INVALID_ARG).
 *   F_dev    optional complex128 r x n_dir x 3 output.
 *   xs       host r x 3 output (C_ext, C_sca, C_abs).  Synchronising.
 * Errors: INVALID_ARG, STATE, CUDA.
 */
mueller_status mueller_far_field(mueller_mesh* mesh, const mueller_params* params,
                                 const void* X_dev, int32_t r, const double* inc,
                                 const double* dirs, int64_t n_dir, void* F_dev, double* xs,
                                 int32_t n_theta, int32_t n_phi, void* stream);

/*
 * mueller_far_field_noalloc -- the far field and cross sections of
 * mueller_far_field, computed without allocating any device memory.  (The
 * paper has no counterpart: this is an interface for callers that cannot
 * allocate, such as a framework that routes all device memory through its
 * own pool, or a service that reserves its memory at start-up and forbids
 * allocation later.)
 * Same arguments, outputs and errors as mueller_far_field, and:
 *   - scratch is a fixed MUELLER_FAR_FIELD_NOALLOC_SCRATCH_BYTES (16 MiB)
 *     array in device memory, held by every GPU that loads the library until
 *     the process exits.  A request that needs more (it grows with
 *     r * (n_tri * q_regular + n_theta * n_phi + n_dir)) is rejected with
 *     INVALID_ARG and a message naming the size.  The level-3 sphere (1280
 *     triangles, q_regular = 6) with the default 48 x 96 sphere rule needs
 *     about 0.97 MB per right-hand side: up to 17 right-hand sides fit, 18
 *     are refused.
 *   - the mesh must already hold the point geometry for params (call
 *     mueller_assemble or mueller_far_field with the same params first), else
 *     STATE: this call never creates it.
 *   - the first call on a device looks up the device address of the scratch
 *     array (cudaGetSymbolAddress); make that first call before any stream
 *     capture.
 *   - every call uses the same scratch: calls whose GPU work overlaps (on
 *     different streams or host threads) race and give wrong results; the
 *     call synchronises its stream before returning, on success and on
 *     every error after its first copy, so calls issued one after another
 *     on one thread are safe.  Nothing in the scratch needs to
 *     start at zero: each region is fully written before it is read.
 */
#define MUELLER_FAR_FIELD_NOALLOC_SCRATCH_BYTES (16u << 20)
mueller_status mueller_far_field_noalloc(mueller_mesh* mesh, const mueller_params* params,
                                         const void* X_dev, int32_t r, const double* inc,
                                         const double* dirs, int64_t n_dir, void* F_dev,
                                         double* xs, int32_t n_theta, int32_t n_phi,
                                         void* stream);

/*
 * Launch accounting and per-kernel timing (no counterpart in the paper: a
 * measurement aid).  Every kernel launch of the library is counted.  With
 * profiling enabled, each launch is bracketed by CUDA events on its own
 * stream and the call waits for the closing event, so enabled profiling
 * serialises the host with the device; it is off by default.
 *   mueller_profile_get: total milliseconds and launches of a kernel name
 *   (returns 0 if the name was never timed).  mueller_profile_names writes
 *   the timed names, newline separated, into buf (truncated to buflen) and
 *   returns their count.
 */
void mueller_profile_enable(int32_t on);
void mueller_profile_reset(void);
int64_t mueller_launch_count(void);
int32_t mueller_profile_get(const char* name, double* total_ms, int64_t* launches);
int32_t mueller_profile_names(char* buf, size_t buflen);

/* Block until all work queued on the stream is done; surfaces device faults. */
mueller_status mueller_sync(void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MUELLER_H_ */
