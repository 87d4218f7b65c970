/*
 * mfpoisson.h - C ABI of the GB300 matrix-free high-order Poisson library.
 *
 * The library evaluates the operator of -div(kappa grad u) = f (Sec. 2,
 * Eq. 1) on a structured hexahedral brick of the unit cube (or of a cube
 * [box_lo, box_hi]^3, optionally curved by an analytic map) without
 * assembling a matrix: cell integrals by sum factorization (Sec. 3, Eq. 12)
 * for continuous Q_k elements (Sec. 2.1, Eq. 4) and for the symmetric
 * interior penalty DG method (Sec. 2.2, Eq. 6, boundary extension Eq. 7),
 * and solves with CG preconditioned by a geometric multigrid V-cycle with
 * Chebyshev-Jacobi smoothing (Sec. 4.1).
 *
 * General conventions
 *  - Every pointer argument named *_dev is DEVICE memory on the context's
 *    device, owned by the caller, contiguous, aligned to at least 16 bytes,
 *    and must stay valid until the work queued on `stream` has finished.
 *    Pointers named *_host are host memory read or written before return.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is queued asynchronously unless stated otherwise.
 *  - Every call returns an mfp_status.  On failure nothing is written to
 *    the outputs that the status does not describe, and the message is
 *    available from mfp_last_error() (per thread).
 *  - The library owns all level data (geometry, diagonals, scratch) and
 *    frees it in mfp_destroy().
 *
 * Vector layouts (level l of a context; level n_levels-1 is the finest)
 *  - cells c = cx + nx*(cy + ny*cz), cell size L/nx x L/ny x L/nz before
 *    the mapping, L = box_hi - box_lo (1 by default);
 *  - local node / quadrature point a = ax + p*ay + p*p*az, p = k+1, x fastest;
 *  - CG (disc = MFP_CG): one value per node of the (nx k+1)(ny k+1)(nz k+1)
 *    grid, x fastest; boundary nodes are present, and those on Dirichlet
 *    sides carry the identity rows / columns of the eliminated Dirichlet
 *    conditions (Sec. 2.1);
 *  - SIPG (disc = MFP_SIPG): cell-major blocks of p^3 nodal values;
 *  - batched vectors (n_rhs = R > 1): entry (i, r) at [i*R + r];
 *  - cell coefficient / gradient: [ncells][p^3] in local quadrature order;
 *  - face coefficient / gradient: all x-normal faces, then y-, then
 *    z-normal ones; inside one direction lexicographic (x fastest) over the
 *    (n_x+dx) x (n_y+dy) x (n_z+dz) face grid, d* = 1 on the normal axis;
 *    p^2 points per face, q = qa + p*qb with a < b the tangential axes.
 *  - the nodal basis is Lagrange in the Gauss-Lobatto points, quadrature is
 *    the (k+1)-point Gauss rule per direction (Sec. 2.1, Sec. 3).
 */
#ifndef MFPOISSON_H
#define MFPOISSON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mfp_ctx mfp_ctx;

typedef enum {
  MFP_OK = 0,
  MFP_ERR_ARG = -1,           /* invalid argument; nothing was queued      */
  MFP_ERR_CUDA = -2,          /* a CUDA call failed; context still usable
                                 unless the CUDA error is sticky           */
  MFP_ERR_OOM = -3,           /* device allocation failed                  */
  MFP_ERR_NOT_CONVERGED = -4, /* solve hit max_it; outputs hold the last
                                 iterate, iteration count and residual     */
  MFP_ERR_STATE = -6          /* call not valid for this context           */
} mfp_status;

enum { MFP_CG = 0, MFP_SIPG = 1 };
enum { MFP_FP64 = 0, MFP_FP32 = 1, MFP_MIXED = 2 };
enum { MFP_MAP_IDENTITY = 0, MFP_MAP_SINE = 1, MFP_MAP_NODES = 2 };
enum { MFP_ARITH_DF = 0, MFP_ARITH_NATIVE = 1 };

typedef struct {
  int nx, ny, nz;        /* fine-level cells per axis (>= 1)                */
  int degree;            /* k in 1..8                                      */
  int disc;              /* MFP_CG or MFP_SIPG                              */
  int n_levels;          /* multigrid levels; 0 = halve while every count
                            is even and >= 4 (coarsest has >= 2 cells/axis);
                            each coarsening needs all counts even          */
  int mapping;           /* MFP_MAP_IDENTITY: affine brick (one Jacobian per
                            level); MFP_MAP_SINE: x -> x + map_param
                            sin(pi x) sin(pi y) sin(pi z) (1,1,1), degree-k
                            isoparametric interpolation through the
                            Gauss-Lobatto support points (Sec. 2);
                            MFP_MAP_NODES: the support points are given in
                            map_nodes (Sec. 2: a degree-k polynomial map
                            through Gauss-Lobatto support points)          */
  double map_param;      /* amplitude for MFP_MAP_SINE (|amp| < 1/(pi sqrt 3)) */
  double kappa;          /* constant coefficient (> 0) until
                            mfp_set_coefficient is called                   */
  double penalty_factor; /* SIPG: sigma_F = penalty_factor (k+1)^2 / h_F with
                            1/h_F = (|F|/|K-| + |F|/|K+|)/2 (|F|/|K| on the
                            boundary); Sec. 2.2 (paper value: 3)            */
  int mg_precision;      /* V-cycle arithmetic: MFP_FP64 or MFP_FP32; the
                            outer CG, its residuals and dot products are
                            always float64 (MFP_MIXED is a synonym of FP32) */
  int cheb_degree;       /* Chebyshev smoother degree (Sec. 4.1: 5)         */
  int eig_cg_iters;      /* CG iterations of the eigenvalue estimate (15)   */
  int fp64_arith;        /* float64 operator applies: MFP_ARITH_DF (default)
                            carries every intermediate as a pair of floats
                            (about 48 bits, error-free TwoSum / FMA TwoProd)
                            on the FP32 pipes, about 58x wider than the FP64
                            pipe on GB300; vector entries must lie in
                            [2^-80, 2^127] in magnitude (smaller ones lose
                            their low part).  MFP_ARITH_NATIVE uses DFMA.
                            Float64 vectors in HBM either way.             */
  int neumann_sides;     /* sides with Neumann data: bit 2e for x_e = lo,
                            bit 2e+1 for x_e = hi (e = 0, 1, 2 for x, y, z).
                            CG: those nodes stay free (natural condition);
                            SIPG: no operator terms on those boundary faces
                            (Eq. 7 leaves only data there).  The other sides
                            are Dirichlet (identity rows for CG, the mirror
                            state of Eq. 7 for SIPG).  0 (default): all six
                            Dirichlet; at least one side must stay Dirichlet
                            (values 0..62).                                 */
  double box_lo, box_hi; /* domain [box_lo, box_hi]^3: the unit cube mapped
                            by `mapping`, then by x -> box_lo + (box_hi -
                            box_lo) x (default 0, 1; Sec. 4.3 uses -1, 1);
                            MFP_MAP_NODES needs the default (the nodes are
                            physical points)                                */
  const double* map_nodes; /* MFP_MAP_NODES: HOST array [ncells][(k+1)^3][3]
                            of the physical support points of every finest
                            cell (cell and local node order of the vector
                            layouts above), the images of the cell's
                            Gauss-Lobatto grid.  Neighbouring cells must
                            give identical points on their common face (a
                            conforming mesh).  Copied during mfp_create; the
                            caller keeps ownership.  Coarse levels take the
                            finer level's isoparametric map evaluated at
                            their own Gauss-Lobatto points (a point on the
                            interface of two children from the upper one).
                            A map with det J <= 0 at a quadrature point
                            returns MFP_ERR_ARG.  NULL otherwise.          */
} mfp_desc;

/* Fill `desc` with the defaults (1 cell, k=1, CG, identity map, kappa 1,
 * penalty_factor 1, FP64 V-cycle, Chebyshev degree 5, 15 CG iterations,
 * double-float arithmetic for float64 applies, Dirichlet on all sides,
 * domain [0, 1]^3). */
void mfp_desc_default(mfp_desc* desc);

/* Create a context on the current CUDA device: builds every multigrid level
 * (geometry at quadrature points, inverse Jacobi diagonal, eigenvalue
 * estimates and Chebyshev parameters; Sec. 4.1 "setup").  With more than
 * one level and at most 2048 dofs on the coarsest level, that level's
 * operator is also assembled once as a dense matrix (from matrix-free
 * applies to identity columns) for the coarse Chebyshev solve.  Synchronises
 * `stream`.  *out receives an opaque handle owned by the library.  Start
 * `desc` from mfp_desc_default: a zero-filled one is rejected (box_hi must
 * exceed box_lo).  Invalid fields return MFP_ERR_ARG before any CUDA call. */
mfp_status mfp_create(const mfp_desc* desc, void* stream, mfp_ctx** out);

/* Free all device and host memory of the context (synchronises the device
 * work of the context first).  NULL is accepted. */
mfp_status mfp_destroy(mfp_ctx* ctx);

/* Number of levels of the context. */
int mfp_n_levels(const mfp_ctx* ctx);

/* Sizes on `level` (0 = coarsest): dofs, cell quadrature points
 * (ncells p^3) and face quadrature points (nfaces p^2).  NULL outputs are
 * skipped. */
mfp_status mfp_sizes(const mfp_ctx* ctx, int level, int64_t* n_dofs,
                     int64_t* n_cell_qp, int64_t* n_face_qp);

/* Replace the coefficient by per-quadrature-point values on the finest
 * level: a_cell_dev [ncells][p^3], a_face_dev [nfaces][p^2] (the face
 * values are used by the SIPG face terms and may be NULL for CG).  All
 * values must be > 0.  Coarser levels receive the quadrature-weighted mean
 * over the children of each coarse cell / coarse face; every level's
 * geometry, diagonal and eigenvalue estimate are rebuilt.  Synchronises. */
mfp_status mfp_set_coefficient(mfp_ctx* ctx, const double* a_cell_dev,
                               const double* a_face_dev, void* stream);

/* Load vector b_i = sum_q w_q det J f(x_q) phi_i(x_q) on the finest level
 * (Eq. 4 / Eq. 6 right-hand side), written to b_dev[i * stride] (stride >=
 * 1, e.g. R for column r of a batch when the pointer is offset by r).
 *  - f_kind 0: f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) (params unused),
 *    homogeneous boundary data: zero on constrained (CG Dirichlet) dofs.
 *  - f_kind 1: f = sum_j A_j exp(-|x - c_j|^2 / w_j^2) with params_host =
 *    n_terms blocks (c_x, c_y, c_z, w, A), homogeneous boundary data.
 *  - f_kind 2: the problem whose exact solution is u = sum_j A_j exp(-|x -
 *    c_j|^2 / w_j^2) (same params; Sec. 4.3 uses three such terms on
 *    (-1, 1)^3): f = -kappa Laplace u, Dirichlet data u on the Dirichlet
 *    sides and Neumann data kappa grad u . n on the Neumann sides.  CG: a
 *    constrained dof holds u at its node and the free rows have the lifted
 *    data subtracted (so the solve returns the complete solution); SIPG:
 *    the data terms of Eq. 7 on Dirichlet faces.  Needs the constant
 *    coefficient (MFP_ERR_ARG after mfp_set_coefficient). */
mfp_status mfp_rhs(mfp_ctx* ctx, int f_kind, const double* params_host,
                   int n_terms, double* b_dev, int64_t stride, void* stream);

/* Same load vector as mfp_rhs, for callers that must not allocate device
 * memory once their set-up is done: for example applications that hand all
 * device memory to their own pool up front (a library cudaMalloc would fail
 * or fragment it), or latency-bound loops that cannot afford the implicit
 * device synchronisation of cudaMalloc / cudaFree.  mfp_rhs stages the
 * Gaussian parameters in a device buffer it allocates when n_terms grows;
 * this entry point copies them into a fixed array compiled into the library
 * instead (160 KiB, held on every device that loads the library until the
 * process exits) and calls no allocating routine.
 *  - n_terms <= 4096 for f_kind 1 and 2 (the limit of mfp_rhs too); larger
 *    counts return MFP_ERR_ARG.
 *  - mfp_create sets this entry point up on its device: it resolves the
 *    array's device address and loads the array and the load-vector kernels
 *    there, so that this call makes CUDA load nothing.  Call it with the
 *    context's device current (MFP_ERR_STATE otherwise).
 *  - All calls share the array, which keeps the last call's parameters.
 *    Calls whose work overlaps on the GPU (different streams without
 *    ordering) race on it; calls on one stream are safe.
 *  - params_host may be pageable (copied before return) or page-locked (it
 *    must then stay valid until the call's work on `stream` has run).
 * The paper has no counterpart; arguments and output as in mfp_rhs. */
mfp_status mfp_rhs_noalloc(mfp_ctx* ctx, int f_kind, const double* params_host,
                           int n_terms, double* b_dev, int64_t stride,
                           void* stream);

/* HDG mixed matrix-free operator (Sec. 3, "HDG mixed matrix-free", on the
 * hybridizable DG form of Sec. 2.3):
 *   y = ([A B^T; B D] + [C^T; G^T] H^{-1} [C G]) x
 * on the finest cells of an SIPG context (same mesh, box and Neumann sides),
 * with A = (w, kappa^-1 q), B^T = -(div w, u), D = -<v, tau u>,
 * C^T = <w . n, lambda>, G^T = <v, tau lambda>, H = sum <mu, tau lambda> and
 * tau = tau_factor times the largest coefficient value on the face (Sec. 4.2:
 * tau_factor 5).  Dirichlet faces hold data traces and add no H^{-1}
 * coupling.  x_dev and y_dev hold the cell unknowns (q_x, q_y, q_z, u) in
 * cell-major blocks of 4 (k+1)^3 nodal values (the SIPG cell layout per
 * field), 4 ncells (k+1)^3 doubles each, distinct.  Any mapping; the
 * coefficient is the constant one or the per-point values of
 * mfp_set_coefficient (cell and face values both needed).  The arithmetic
 * follows fp64_arith (double-float on the FP32 pipes by default, DFMA for
 * MFP_ARITH_NATIVE); x and y are float64 either way.  The first call
 * allocates the context's trace buffer (nfaces (k+1)^2 doubles) and, on
 * curved cells, per-point geometry (10 doubles per cell point, 4 per face
 * point): make it outside a stream capture.  Calls on one context share
 * those buffers: issue them in stream order.
 * Launches four kernels (traces per face direction, then the cells). */
mfp_status mfp_hdg_apply(mfp_ctx* ctx, double tau_factor, const double* x_dev,
                         double* y_dev, void* stream);

/* dst = A src on `level` (Eq. 12, plus the SIPG face terms of Eq. 6/7 and
 * identity rows / columns for CG Dirichlet nodes).  prec MFP_FP64 takes
 * double vectors, MFP_FP32 float vectors (FP32 level data must exist, i.e.
 * mg_precision FP32).  n_rhs = R >= 1 applies to R right-hand sides in the
 * batched layout; CG is one launch, SIPG one cell-kernel launch plus one
 * launch that adds the face terms each cell left for its upper neighbours
 * in a per-level face buffer (grown on first use with more columns, so the
 * first apply with a new maximum R allocates and must not be inside a stream
 * capture).  The result does not depend on launch shapes (no atomics for
 * SIPG).  Applies of one level share that buffer and scratch: issue them in
 * stream order.  src and dst must not alias. */
mfp_status mfp_apply(mfp_ctx* ctx, int level, int prec, const void* src_dev,
                     void* dst_dev, int n_rhs, void* stream);

/* Inverse of diag(A) on `level` in precision `prec` (copied to diag_dev,
 * n_dofs values): the Jacobi diagonal of Sec. 4.1, 1 on constrained dofs. */
mfp_status mfp_inverse_diagonal(mfp_ctx* ctx, int level, int prec,
                                void* diag_dev, void* stream);

/* Eigenvalue estimates of D^{-1}A on `level` from the Lanczos tridiagonal of
 * `eig_cg_iters` Jacobi-PCG steps (Sec. 4.1), and the Chebyshev interval
 * [lo, hi] and degree used there (coarsest level: coarse solve). */
mfp_status mfp_level_info(const mfp_ctx* ctx, int level, double* lam_max,
                          double* lam_min, double* cheb_lo, double* cheb_hi,
                          int* cheb_degree);

/* Transfer between level `level` (fine) and level-1 (coarse): prolongation
 * (geometric embedding of the coarse Q_k space, Sec. 4.1) or restriction
 * (its transpose).  Vectors in precision `prec`; single right-hand side. */
mfp_status mfp_prolongate(mfp_ctx* ctx, int level, int prec,
                          const void* coarse_dev, void* fine_dev,
                          void* stream);
mfp_status mfp_restrict(mfp_ctx* ctx, int level, int prec,
                        const void* fine_dev, void* coarse_dev, void* stream);

/* Chebyshev-Jacobi smoother of `level` (Sec. 4.1): x <- smoothed iterate for
 * A x = b.  zero_start != 0 ignores the input x (x0 = 0, first update
 * without an operator application).  On the coarsest level this is the
 * coarse solve. */
mfp_status mfp_smooth(mfp_ctx* ctx, int level, int prec, const void* b_dev,
                      void* x_dev, int zero_start, void* stream);

/* One V-cycle z = B r on the finest level (Sec. 4.1), float64 in and out;
 * the internal arithmetic is the context's mg_precision. */
mfp_status mfp_vcycle(mfp_ctx* ctx, const double* r_dev, double* z_dev,
                      int n_rhs, void* stream);

/* CG preconditioned by one V-cycle from x = 0 (Sec. 4.1) for A x = b on the
 * finest level, float64 residuals, dot products and stopping test
 * ||b - A x||_2 <= rtol ||b||_2 (recursively updated residual), for n_rhs
 * independent right-hand sides in the batched layout (each column stops on
 * its own).  Synchronises `stream` once per iteration.  iters_host[n_rhs] and
 * relres_host[n_rhs] receive the iteration counts and final relative
 * residuals (may be NULL).  Returns MFP_ERR_NOT_CONVERGED if any column hit
 * max_it.  The V-cycle runs as a CUDA graph, captured once per column count
 * on a stream of the context and replayed on `stream`; the environment
 * variable MFP_CUDA_GRAPHS=0 launches its kernels one by one instead. */
mfp_status mfp_solve(mfp_ctx* ctx, const double* b_dev, double* x_dev,
                     int n_rhs, double rtol, int max_it, int* iters_host,
                     double* relres_host, void* stream);

/* Gradient of L = 0.5 |u - u_t|^2 subject to A(a) u = f with respect to
 * the per-quadrature-point coefficient a, given the forward solution u and
 * the adjoint solution lambda of A lambda = u - u_t (A is symmetric):
 *   dL/da_q = -lambda^T (dA/da_q) u,
 * i.e. -w_q det J (J^{-T} grad lambda).(J^{-T} grad u) at cell points and
 * minus the SIPG face form (Eq. 6/7) with kappa replaced by the point's
 * indicator at face points.  g_cell_dev [ncells][p^3]; g_face_dev
 * [nfaces][p^2] (SIPG only; may be NULL for CG).  Not in the paper. */
mfp_status mfp_gradient(mfp_ctx* ctx, const double* u_dev,
                        const double* lambda_dev, double* g_cell_dev,
                        double* g_face_dev, void* stream);

/* Autotuner (not in the paper): times the operator apply of `level` in
 * precision `prec` for n_rhs columns with every admissible number of cells
 * per thread block (1..32, at most 1024 threads per block), on scratch
 * vectors it allocates and frees itself, and keeps the fastest choice in the
 * context for later applies with the same (level, prec, n_rhs); for float
 * CG applies with k <= 4 and one column it also times the kernel that gives
 * each cell one warp (reported as cells_out = 0).  Captured V-cycles are
 * re-captured.  Synchronises `stream`.  cells_out / ms_out receive the choice
 * and its time per apply (may be NULL).  The environment variable
 * MFP_CELLS_PER_BLOCK overrides every choice (1000 selects the warp-per-cell
 * kernel where it applies). */
mfp_status mfp_autotune(mfp_ctx* ctx, int level, int prec, int n_rhs,
                        int* cells_out, double* ms_out, void* stream);

/* Counters: operator applications per level since creation (array of
 * mfp_n_levels entries), V-cycles since creation, and the number of CUDA
 * kernels this library has launched in the process.  NULL outputs are
 * skipped. */
mfp_status mfp_counters(const mfp_ctx* ctx, int64_t* applies_per_level,
                        int64_t* vcycles, int64_t* kernel_launches);

/* Last error message of the calling thread ("" if none). */
const char* mfp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MFPOISSON_H */
