// Internal declarations of the mfpoisson library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mfpoisson.h"

namespace mfp {

constexpr int kMaxP = 9;  // k <= 8

// ---------------------------------------------------------------------------
// 1D reference-element tables on [0, 1] (Sec. 2.1: Lagrange basis in the
// k+1 Gauss-Lobatto points; Sec. 3: (k+1)-point Gauss quadrature).
// Row-major p x p matrices, entry [q * p + j].
// ---------------------------------------------------------------------------
template <typename T>
struct DevTab {
  T S[kMaxP * kMaxP];     // S[q][j]    = phi_j(g_q)       GLL basis at Gauss
  T D[kMaxP * kMaxP];     // D[q][j]    = l_j'(g_q)        Gauss collocation
  T Dphi[kMaxP * kMaxP];  // Dphi[q][j] = phi_j'(g_q)      GLL basis slope
  T E0[kMaxP * kMaxP];    // E0[i][j]   = phi_j(x_i / 2)   left-child embed
  T E1[kMaxP * kMaxP];    // E1[i][j]   = phi_j((1+x_i)/2) right-child embed
  T dphi0[kMaxP];         // phi_j'(0)
  T dphi1[kMaxP];         // phi_j'(1)
  T w[kMaxP];             // Gauss weights on [0, 1]
  T g[kMaxP];             // Gauss points on [0, 1]
  T x[kMaxP];             // GLL points on [0, 1]
  T gv0[kMaxP], gv1[kMaxP];  // Lagrange basis of the Gauss points at 0, 1
  T gd0[kMaxP], gd1[kMaxP];  // and its slopes there
};

// The same tables as double-float pairs (value = hi + lo, |lo| <= ulp(hi)/2)
// for the FP64-accurate kernels that run on the FP32 pipes.
struct DevTabDF {
  float Sh[kMaxP * kMaxP], Sl[kMaxP * kMaxP];
  float Dh[kMaxP * kMaxP], Dl[kMaxP * kMaxP];
  float d0h[kMaxP], d0l[kMaxP], d1h[kMaxP], d1l[kMaxP];
  float wh[kMaxP], wl[kMaxP];
  // Lagrange basis on the Gauss points: values l_q(0), l_q(1) and slopes
  // l_q'(0), l_q'(1) at the ends of [0, 1] (traces from quadrature data)
  float gv0h[kMaxP], gv0l[kMaxP], gv1h[kMaxP], gv1l[kMaxP];
  float gd0h[kMaxP], gd0l[kMaxP], gd1h[kMaxP], gd1l[kMaxP];
};

// Even-odd split of the double-float 1D sweeps (DF kernels only).  The
// matrices M = S, D and their transposes satisfy M[p-1-q][p-1-j] = s M[q][j]
// (s = +1 for S, -1 for D: GLL nodes and Gauss points are symmetric), so
// with h = p/2, e_j = x_j + x_{p-1-j}, o_j = x_j - x_{p-1-j} (j < h) and,
// for odd p, e_h = x_h:
//   A_q = sum_j a[q][j] e_j,  B_q = sum_{j<h} b[q][j] o_j,
//   (M x)_q = A_q + B_q,  (M x)_{p-1-q} = s (A_q - B_q)   (q < h),
// with a[q][j] = (M[q][j] + M[q][p-1-j]) / 2, b = the difference / 2,
// a[q][h] = M[q][h]; the middle row of an odd p needs A (S) or B (D) only.
// Index w = 2 W + TR (W: 0 = S, 1 = D; TR: transposed), rows and columns
// up to kMaxH.
constexpr int kMaxH = 5;
struct DevTabEO {
  float ah[4][kMaxH * kMaxH], al[4][kMaxH * kMaxH];
  float bh[4][kMaxH * kMaxH], bl[4][kMaxH * kMaxH];
};

struct HostTables {
  DevTab<double> d[8];  // index k-1
  DevTab<float> f[8];
  DevTabDF df[8];
  DevTabEO eo[8];
};
const HostTables& host_tables();

// ---------------------------------------------------------------------------
// Error state
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
void clear_error();
// Count of kernels this library has launched (process-wide).
void note_launch();
int64_t launches_total();
void add_launches(int64_t n);

struct Fail {
  mfp_status st;
};
#define MFP_CHECK_CUDA(call)                                                  \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ::mfp::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
      throw ::mfp::Fail{e_ == cudaErrorMemoryAllocation ? MFP_ERR_OOM         \
                                                        : MFP_ERR_CUDA};      \
    }                                                                         \
  } while (0)
#define MFP_REQUIRE(cond, msg)                  \
  do {                                          \
    if (!(cond)) {                              \
      ::mfp::set_error(msg);                    \
      throw ::mfp::Fail{MFP_ERR_ARG};           \
    }                                           \
  } while (0)

// ---------------------------------------------------------------------------
// Device scalars of the CG iterations, slot-major: scal[slot * R + column]
// ---------------------------------------------------------------------------
enum ScalarSlot {
  S_RZ = 0,      // (r, z)
  S_RZ0,         // initial (r, z)
  S_ALPHA,
  S_BETA,
  S_RN2,         // |r|^2 after the update
  S_BN2,         // |b|^2
  S_ACTIVE,      // 1 while the column iterates
  S_STOP,        // set on breakdown / convergence of the eigenvalue CG
  S_COUNT_IT,    // completed eigenvalue-CG iterations
  S_COUNT
};
constexpr int kMaxRedBlocks = 1024;
constexpr int kMaxRhs = 256;
constexpr int kMaxGaussTerms = 4096;  // forcing terms of mfp_rhs (f_kind 1, 2)
constexpr int kWarpCells = 1000;  // cells-per-block value of the warp-per-cell CG kernel
constexpr int kDenseMax = 2048;   // dofs of a coarsest level stored dense
constexpr int kDenseRows = 128;   // rows per block of k_dense_apply
constexpr int kDenseSplit = 32;   // column ranges per row block
struct RedScratch {
  double* part = nullptr;  // [kMaxRedBlocks][R]
  unsigned* cnt = nullptr; // zero between launches
};

// ---------------------------------------------------------------------------
// Boundary conditions of the six sides x_d = lo / hi (side 2d / 2d + 1).
// CG: node (X, Y, Z) of the node grid is Dirichlet-constrained when one of
// its coordinates equals the lo / hi entry of its axis; a Neumann side holds
// -1 there, which no coordinate matches (natural boundary condition, Eq. 4).
// SIPG: bit 2d + s of `neumann` drops the operator terms of the faces on
// side (d, s) (the extension of Eq. 7 leaves only data there).
// ---------------------------------------------------------------------------
// Vector update fused into the last kernel of an SIPG apply (the face-add
// kernel, which completes y = (A src)_i of every dof), so that y itself is
// never written and read back (Sec. 4.1 smoother and V-cycle residual):
//   EPI_STORE       dst = y
//   EPI_RESIDUAL    dst = b - y
//   EPI_CHEB_FIRST  e = c1 dinv (b - y);        d = e; x += e  (dst unused)
//   EPI_CHEB_STEP   e = c1 d + c2 dinv (b - y); d = e; x += e  (dst unused)
// Vectors in the batched layout; dinv has one entry per dof.
enum { EPI_STORE = 0, EPI_RESIDUAL = 1, EPI_CHEB_FIRST = 2, EPI_CHEB_STEP = 3 };
template <typename T>
struct Epi {
  int mode;
  const T* b;
  const T* dinv;
  T* d;
  T* x;
  double c1, c2;
};

// Applies the update of `e` to the finished value y of entry gi, given the
// inputs b, dinv, d, x of that entry (loaded by the caller as the mode needs
// them, ahead of its arithmetic).
template <typename T, typename Y>
__device__ __forceinline__ void epi_finish(const Epi<T>& e, T* dst, size_t gi,
                                           Y y, T b, T dinv, T d, T x) {
  if (e.mode == EPI_STORE) {
    dst[gi] = (T)y;
    return;
  }
  const Y r = (Y)b - y;
  if (e.mode == EPI_RESIDUAL) {
    dst[gi] = (T)r;
    return;
  }
  const Y dr = (Y)e.c2 * ((Y)dinv * r);
  const Y v = e.mode == EPI_CHEB_FIRST ? (Y)e.c1 * ((Y)dinv * r)
                                       : (Y)e.c1 * (Y)d + dr;
  e.d[gi] = (T)v;
  e.x[gi] = (T)((Y)x + v);
}

struct Bc {
  int lo[3] = {0, 0, 0};
  int hi[3] = {0, 0, 0};
  int neumann = 0;
};
__host__ __device__ __forceinline__ bool bc_con(const Bc& b, int64_t X,
                                                int64_t Y, int64_t Z) {
  return X == b.lo[0] || X == b.hi[0] || Y == b.lo[1] || Y == b.hi[1] ||
         Z == b.lo[2] || Z == b.hi[2];
}

// ---------------------------------------------------------------------------
// Level data
// ---------------------------------------------------------------------------
template <typename T>
struct LevelData {
  T* G = nullptr;      // curved: [ncells][6][p^3] w det J J^{-1} J^{-T}
  T* kcell = nullptr;  // per-point coefficient [ncells][p^3] (or null)
  T* kface = nullptr;  // per-point face coefficient [nfaces][p^2] (or null)
  T* fdata = nullptr;  // curved SIPG: [nfaces][7][p^2] dA, nJ_L(3), nJ_R(3)
  T* sigma = nullptr;  // curved SIPG: [nfaces] penalty
  T* dinv = nullptr;   // [ndofs] inverse Jacobi diagonal
  bool valid = false;
};

// Double-float copies of the float64 level data (hi / lo float arrays)
struct LevelDF {
  float *Gh = nullptr, *Gl = nullptr;    // [ncells][6][p^3]
  float *kch = nullptr, *kcl = nullptr;  // [ncells][p^3]
  float *kfh = nullptr, *kfl = nullptr;  // [nfaces][p^2]
  float *fdh = nullptr, *fdl = nullptr;  // [nfaces][7][p^2]
  float *sgh = nullptr, *sgl = nullptr;  // [nfaces]
  bool valid = false;
};

struct Level {
  int n[3] = {0, 0, 0};
  int k = 1, p = 2;
  int disc = MFP_CG;
  bool curved = false;
  int64_t ncells = 0, ndofs = 0, nfaces = 0;
  int gdim[3] = {0, 0, 0};    // CG node grid
  int face_off[3] = {0, 0, 0};
  double h[3] = {0, 0, 0};     // physical cell size (box length / n)
  double box_lo = 0.0, box_len = 1.0;  // domain [box_lo, box_lo + box_len]^3
  Bc bc;
  double kappa = 1.0;
  double penalty = 1.0;
  double map_amp = 0.0;
  double* nodes = nullptr;    // given support points [ncells][p^3][3]
  int* err = nullptr;         // the context's kernel error word (device)
  bool df_arith = false;      // float64 applies in double-float arithmetic
  double* vol = nullptr;      // curved: cell volumes [ncells]
  LevelData<double> d64;
  LevelData<float> d32;
  LevelDF ddf;
  // eigenvalue estimate and Chebyshev parameters (Sec. 4.1)
  double lam_max = 0, lam_min = 0, cheb_lo = 0, cheb_hi = 0;
  int cheb_degree = 0;
  int64_t applies = 0;
  // V-cycle scratch in the V-cycle precision, scratch_rhs columns
  void* t_res = nullptr;  // operator output / residual / correction
  void* t_d = nullptr;    // Chebyshev update
  void* t_x = nullptr;    // iterate (levels below the finest)
  void* t_b = nullptr;    // right-hand side (levels below the finest)
  int scratch_rhs = 0;
  // SIPG applies: the face terms each cell leaves for its upper neighbours,
  // [ncells][6][p^2] x fbuf_rhs entries of 8 bytes (float, float64 or a
  // double-float pair; the applies of one level are stream-ordered)
  void* fbuf = nullptr;
  int fbuf_rhs = 0;
  // Coarsest level with at most kDenseMax dofs: the operator assembled once
  // as a dense column-major matrix (float64, and float for a float V-cycle).
  // The coarse Chebyshev solve applies it with k_dense_apply: on a handful of
  // cells the cell kernels are latency-bound (about 30 us per apply).
  double* dense64 = nullptr;
  float* dense32 = nullptr;
  // the coarse solve (zero-start Chebyshev of the bound-derived degree) as
  // its dense matrix p(D^{-1} A) D^{-1}, column-major [ndofs][ndofs]
  double* csolve64 = nullptr;
  float* csolve32 = nullptr;
  double* dpart = nullptr;   // partial sums [kDenseSplit][kMaxRhs][ndofs]
  unsigned* dcnt = nullptr;  // arrival counters [row blocks][kMaxRhs]
};

template <typename T>
inline LevelData<T>& level_data(Level& L);
template <>
inline LevelData<double>& level_data<double>(Level& L) { return L.d64; }
template <>
inline LevelData<float>& level_data<float>(Level& L) { return L.d32; }

}  // namespace mfp

struct mfp_ctx {
  mfp_desc desc;
  int device = 0;
  bool has_coef = false;
  std::vector<mfp::Level> levels;
  int vprec = MFP_FP64;     // V-cycle arithmetic
  // outer CG (float64), sized for cg_rhs columns
  double* cg_r = nullptr;
  double* cg_p = nullptr;
  double* cg_ap = nullptr;
  double* cg_z = nullptr;
  double* scal = nullptr;   // [S_COUNT][cg_rhs]
  double* hist = nullptr;   // eigenvalue CG coefficients [128]
  double* eig_out = nullptr;
  double* params = nullptr; // device copy of forcing parameters
  int params_cap = 0;
  double* hdg_lam = nullptr;    // HDG traces at the face points [nfaces][p^2]
  double* hdg_cell = nullptr;   // curved HDG: [cell][10][p^3] (w det J, J^-1)
  double* hdg_face = nullptr;   // curved HDG: [face][4][p^2] (dA, normal)
  mfp::RedScratch red;
  double* host_scal = nullptr;  // pinned [S_COUNT][kMaxRhs]
  float* mix_r = nullptr;       // float V-cycle input / output on the finest
  float* mix_z = nullptr;
  int cg_rhs = 0;
  int64_t vcycles = 0;
  int* dev_err = nullptr;       // kernel error word: 1 = a copy wait timed out
  // V-cycles of mfp_solve captured as CUDA graphs, one per column count;
  // replays add the captured counter increments
  struct VGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> applies;
    int64_t launches = 0;
    int64_t vcycles = 0;
  };
  std::vector<VGraph> graphs;  // index: column count
  cudaStream_t cap_stream = nullptr;  // capture stream (legacy stream can't)
  // tuned cells per block: key (level, precision, columns) -> cells
  std::vector<std::pair<int64_t, int>> tuned;
};

namespace mfp {

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------
// dst = A src for nrhs interleaved columns ([N][nrhs]); cells = cells per
// block for this column count (0: default choice).
void launch_apply_cg(const Level& L, const LevelData<double>& D,
                     const double* src, double* dst, int nrhs, int cells,
                     cudaStream_t s);
void launch_apply_cg(const Level& L, const LevelData<float>& D,
                     const float* src, float* dst, int nrhs, int cells,
                     cudaStream_t s);
// SIPG: `epi` (may be null = EPI_STORE) is applied by the face-add kernel
void launch_apply_dg(const Level& L, const LevelData<double>& D,
                     const double* src, double* dst, int nrhs, int cells,
                     cudaStream_t s, const Epi<double>* epi);
void launch_apply_dg(const Level& L, const LevelData<float>& D,
                     const float* src, float* dst, int nrhs, int cells,
                     cudaStream_t s, const Epi<float>* epi);

// dst = A src in float64 I/O with double-float arithmetic on the FP32 pipes
// (one translation unit per degree range; false if p is not in its range)
bool apply_cg_df_lo(const Level& L, const double* src, double* dst, int nrhs,
                    int cells, cudaStream_t s);
bool apply_cg_df_hi(const Level& L, const double* src, double* dst, int nrhs,
                    int cells, cudaStream_t s);
bool apply_dg_df_lo(const Level& L, const double* src, double* dst, int nrhs,
                    int cells, cudaStream_t s, const Epi<double>* epi);
bool apply_dg_df_hi(const Level& L, const double* src, double* dst, int nrhs,
                    int cells, cudaStream_t s, const Epi<double>* epi);
// hi / lo split of a float64 array
void launch_split(const double* a, float* hi, float* lo, int64_t n,
                  cudaStream_t s);

// curved geometry; hdg_cell / hdg_face (may be null) also receive the HDG
// mixed operator's data: [cell][10][p^3] (w det J, J^{-1}[e][d]) and
// [face][4][p^2] (dA, unit normal along +e_D)
void launch_curved_cell_geometry(Level& L, cudaStream_t s,
                                 double* hdg_cell = nullptr);
// support points of `coarse` from the isoparametric map of `fine`
void launch_coarsen_nodes(const Level& fine, Level& coarse, cudaStream_t s);
void launch_curved_face_geometry(Level& L, cudaStream_t s,
                                 double* hdg_face = nullptr);
void launch_diagonal(const Level& L, double* diag, cudaStream_t s);
void launch_rhs(const Level& L, int kind, const double* params_dev,
                int nterms, double* b, int64_t stride, cudaStream_t s);
void launch_coarsen_coefficient(const Level& fine, const Level& coarse,
                                cudaStream_t s);
void preload_rhs_kernels(int p);
// Set-up of mfp_rhs_noalloc on the current device: resolves the device
// address of its fixed parameter array and loads the load-vector kernels,
// so that the entry point itself never makes CUDA load code or data.
void noalloc_prepare(int device, int p);
void launch_start_vector(const Level& L, double* v, cudaStream_t s);
void launch_gradient(const Level& L, const double* u, const double* lam,
                     double* gc, double* gf, cudaStream_t s);
// HDG mixed operator on Cartesian cells (k_hdg.cu); lam: [nfaces][p^2]
void launch_hdg_apply(const Level& L, double tau, double* lam,
                      const double* hdg_cell, const double* hdg_face,
                      const double* x, double* y, cudaStream_t s);

template <typename T>
void launch_prolongate(const Level& fine, const Level& coarse, const T* xc,
                       T* xf, int stride, int col, cudaStream_t s);
template <typename T>
void launch_restrict(const Level& fine, const Level& coarse, const T* xf,
                     T* xc, int stride, int col, cudaStream_t s);

template <typename T>
void launch_fill(T* x, T v, int64_t n, cudaStream_t s);
void launch_invert_diag(const Level& L, double* diag, cudaStream_t s);
void launch_to_float(const double* a, float* b, int64_t n, cudaStream_t s);
// dense coarse operator: assembly helpers and y = A x for R columns
void launch_identity_block(double* e, int64_t n, int64_t c0, int R,
                           cudaStream_t s);
void launch_store_columns(const double* y, double* a, int64_t n, int64_t c0,
                          int R, cudaStream_t s);
template <typename T>
void launch_dense_apply(const T* A, const T* x, T* y, int n, int R,
                        double* part, unsigned* cnt, cudaStream_t s);
void launch_to_double(const float* a, double* b, int64_t n, cudaStream_t s);
template <typename T>
void launch_cheb_first(const T* b, const T* dinv, T* d, T* x, const T* ax,
                       double c, int64_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_cheb_step(const T* b, const T* dinv, T* d, T* x, const T* ax,
                      double cd, double cr, int64_t n, int nrhs,
                      cudaStream_t s);
template <typename T>
void launch_residual(const T* b, const T* ax, T* r, int64_t n,
                     cudaStream_t s);
template <typename T>
void launch_axpy(T* y, const T* x, double a, int64_t n, cudaStream_t s);

void launch_dot(const double* a, const double* b, int64_t n, int R,
                RedScratch& rs, double* scal, int op, double* hist, int hidx,
                cudaStream_t s);
void launch_cg_update(double* x, double* r, const double* p, const double* ap,
                      int64_t n, int R, RedScratch& rs, double* scal,
                      cudaStream_t s);
void launch_cg_p(double* p, const double* z, int64_t n, int R,
                 const double* scal, cudaStream_t s);
void launch_jacobi(const double* r, const double* dinv, double* z, int64_t n,
                   int R, cudaStream_t s);
void launch_lanczos(const double* hist, const double* scal, double* out,
                    cudaStream_t s);

}  // namespace mfp
