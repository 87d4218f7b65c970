// C ABI of the library: context and multigrid levels (Sec. 4.1 setup),
// operator application, transfer, Chebyshev smoothing, V-cycle and the
// V-cycle preconditioned CG (Sec. 4.1), host orchestration on one stream.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>

#include "mfp_internal.h"

namespace mfp {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }
static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(); }
void add_launches(int64_t n) { g_launches.fetch_add(n); }

namespace {

template <typename T>
T* dalloc(int64_t n) {
  void* p = nullptr;
  if (n <= 0) n = 1;
  MFP_CHECK_CUDA(cudaMalloc(&p, (size_t)n * sizeof(T)));
  return static_cast<T*>(p);
}
template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}
void dfree(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

cudaStream_t st(void* s) { return static_cast<cudaStream_t>(s); }

int cpb_override() {
  const char* e = std::getenv("MFP_CELLS_PER_BLOCK");
  return e ? std::atoi(e) : 0;
}

int64_t tune_key(int level, int prec, int R) {
  return ((int64_t)level * 4 + prec) * 4096 + R;
}

// Cells per block for an apply: environment override, else the autotuned
// value of this (level, precision, columns), else 0 (kernel default).
int cells_for(const mfp_ctx* c, int level, int prec, int R) {
  const int o = cpb_override();
  if (o > 0) return o;
  const int64_t k = tune_key(level, prec, R);
  for (const auto& kv : c->tuned)
    if (kv.first == k) return kv.second;
  return 0;
}

int level_index(const mfp_ctx* c, const Level& L) {
  return (int)(&L - c->levels.data());
}

void drop_graphs(mfp_ctx* c);

// Face buffer of the SIPG applies (8 bytes per entry: a float, a float64
// or a double-float pair), grown to R columns (never while a stream is being
// captured: the V-cycle's levels are grown by ensure_scratch before it).
void ensure_fbuf(mfp_ctx* c, Level& L, int R, cudaStream_t s) {
  if (L.disc != MFP_SIPG || L.fbuf_rhs >= R) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (s) MFP_CHECK_CUDA(cudaStreamIsCapturing(s, &cs));
  MFP_REQUIRE(cs == cudaStreamCaptureStatusNone,
              "SIPG face buffer would grow inside a stream capture");
  drop_graphs(c);  // captured applies hold the previous buffer
  dfree(L.fbuf);
  MFP_CHECK_CUDA(cudaMalloc(&L.fbuf, (size_t)L.ncells * 6 * L.p * L.p * R *
                                         sizeof(float2)));
  L.fbuf_rhs = R;
}

// The update `epi` on the finished result (see Epi): fused into the face-add
// kernel of a matrix-free SIPG apply, else a vector kernel after the apply.
template <typename T>
void epi_after(const Level& L, const T* y, T* dst, int R, const Epi<T>* epi,
               cudaStream_t s) {
  if (!epi || epi->mode == EPI_STORE) return;
  const int64_t n = L.ndofs;
  if (epi->mode == EPI_RESIDUAL)
    launch_residual<T>(epi->b, y, dst, n * R, s);
  else if (epi->mode == EPI_CHEB_FIRST)
    launch_cheb_first<T>(epi->b, epi->dinv, epi->d, epi->x, y, epi->c1, n, R,
                         s);
  else
    launch_cheb_step<T>(epi->b, epi->dinv, epi->d, epi->x, y, epi->c1,
                        epi->c2, n, R, s);
}

template <typename T>
void apply_level(mfp_ctx* c, Level& L, const T* src, T* dst, int R,
                 cudaStream_t s, const Epi<T>* epi = nullptr) {
  LevelData<T>& D = level_data<T>(L);
  MFP_REQUIRE(D.valid, "level data of this precision was not built "
                       "(mg_precision must be MFP_FP32 for float applies)");
  const T* dense = nullptr;
  if constexpr (sizeof(T) == 8)
    dense = reinterpret_cast<const T*>(L.dense64);
  else
    dense = reinterpret_cast<const T*>(L.dense32);
  if (dense) {
    launch_dense_apply<T>(dense, src, dst, (int)L.ndofs, R, L.dpart, L.dcnt,
                          s);
    L.applies += R;
    epi_after<T>(L, dst, dst, R, epi, s);
    return;
  }
  if (L.disc == MFP_CG)
    MFP_CHECK_CUDA(
        cudaMemsetAsync(dst, 0, (size_t)L.ndofs * R * sizeof(T), s));
  ensure_fbuf(c, L, R, s);
  const int prec = sizeof(T) == 8 ? MFP_FP64 : MFP_FP32;
  const int cells = cells_for(c, level_index(c, L), prec, R);
  if constexpr (sizeof(T) == 8) {
    if (c->desc.fp64_arith == MFP_ARITH_DF) {
      const double* sd = reinterpret_cast<const double*>(src);
      double* dd = reinterpret_cast<double*>(dst);
      bool ok;
      const Epi<double>* e = reinterpret_cast<const Epi<double>*>(epi);
      if (L.disc == MFP_CG) {
        ok = apply_cg_df_lo(L, sd, dd, R, cells, s) ||
             apply_cg_df_hi(L, sd, dd, R, cells, s);
        MFP_REQUIRE(ok, "degree out of range");
        epi_after<T>(L, dst, dst, R, epi, s);
      } else {
        ok = apply_dg_df_lo(L, sd, dd, R, cells, s, e) ||
             apply_dg_df_hi(L, sd, dd, R, cells, s, e);
        MFP_REQUIRE(ok, "degree out of range");
      }
      L.applies += R;
      return;
    }
  }
  if (L.disc == MFP_CG) {
    launch_apply_cg(L, D, src, dst, R, cells, s);
    epi_after<T>(L, dst, dst, R, epi, s);
  } else {
    launch_apply_dg(L, D, src, dst, R, cells, s, epi);
  }
  L.applies += R;
}

void cheb_coeffs_first(const Level& L, double& c) {
  const double theta = 0.5 * (L.cheb_hi + L.cheb_lo);
  c = 1.0 / theta;
}

// Chebyshev smoother / coarse solve on level l (Sec. 4.1).  From a zero
// start on a coarsest level that stores it, the coarse solve is one product
// with the matrix of the same Chebyshev iteration (assemble_coarse_solve).
template <typename T>
void smooth(mfp_ctx* c, int l, const T* b, T* x, bool zero, int R,
            cudaStream_t s) {
  Level& L = c->levels[l];
  LevelData<T>& D = level_data<T>(L);
  if (l == 0 && zero) {
    const T* M = nullptr;
    if constexpr (sizeof(T) == 8)
      M = reinterpret_cast<const T*>(L.csolve64);
    else
      M = reinterpret_cast<const T*>(L.csolve32);
    if (M) {
      launch_dense_apply<T>(M, b, x, (int)L.ndofs, R, L.dpart, L.dcnt, s);
      return;
    }
  }
  T* res = static_cast<T*>(L.t_res);
  T* d = static_cast<T*>(L.t_d);
  const double theta = 0.5 * (L.cheb_hi + L.cheb_lo);
  const double delta = 0.5 * (L.cheb_hi - L.cheb_lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  Epi<T> e{EPI_CHEB_FIRST, b, D.dinv, d, x, 1.0 / theta, 0.0};
  if (zero)
    launch_cheb_first<T>(b, D.dinv, d, x, nullptr, 1.0 / theta, L.ndofs, R,
                         s);
  else
    apply_level<T>(c, L, x, res, R, s, &e);
  for (int i = 1; i < L.cheb_degree; ++i) {
    const double rho1 = 1.0 / (2.0 * sigma - rho);
    e.mode = EPI_CHEB_STEP;
    e.c1 = rho1 * rho;
    e.c2 = 2.0 * rho1 / delta;
    apply_level<T>(c, L, x, res, R, s, &e);
    rho = rho1;
  }
}

template <typename T>
void prolongate(mfp_ctx* c, int l, const T* xc, T* xf, int R,
                cudaStream_t s) {
  launch_prolongate<T>(c->levels[l], c->levels[l - 1], xc, xf, R, 0, s);
}
template <typename T>
void restrict_(mfp_ctx* c, int l, const T* xf, T* xc, int R, cudaStream_t s) {
  launch_restrict<T>(c->levels[l], c->levels[l - 1], xf, xc, R, 0, s);
}

// V-cycle on level l for A x = b, x overwritten (zero initial guess).
template <typename T>
void vcycle_level(mfp_ctx* c, int l, const T* b, T* x, int R,
                  cudaStream_t s) {
  Level& L = c->levels[l];
  if (l == 0) {
    smooth<T>(c, 0, b, x, true, R, s);
    return;
  }
  Level& C = c->levels[l - 1];
  T* res = static_cast<T*>(L.t_res);
  smooth<T>(c, l, b, x, true, R, s);
  const Epi<T> e{EPI_RESIDUAL, b, nullptr, nullptr, nullptr, 0.0, 0.0};
  apply_level<T>(c, L, x, res, R, s, &e);  // res = b - A x
  restrict_<T>(c, l, res, static_cast<T*>(C.t_b), R, s);
  vcycle_level<T>(c, l - 1, static_cast<const T*>(C.t_b),
                  static_cast<T*>(C.t_x), R, s);
  prolongate<T>(c, l, static_cast<const T*>(C.t_x), res, R, s);
  launch_axpy<T>(x, res, 1.0, L.ndofs * R, s);
  smooth<T>(c, l, b, x, false, R, s);
}

void ensure_scratch(mfp_ctx* c, int R) {
  MFP_REQUIRE(R >= 1 && R <= kMaxRhs, "n_rhs must be in 1..256");
  bool grow = c->cg_rhs < R;
  for (auto& L : c->levels) grow = grow || L.scratch_rhs < R;
  if (grow) drop_graphs(c);
  const size_t vb = c->vprec == MFP_FP32 ? sizeof(float) : sizeof(double);
  for (size_t l = 0; l < c->levels.size(); ++l) {
    Level& L = c->levels[l];
    if (L.scratch_rhs >= R) continue;
    dfree(L.t_res);
    dfree(L.t_d);
    dfree(L.t_x);
    dfree(L.t_b);
    const size_t bytes = (size_t)L.ndofs * R * vb;
    MFP_CHECK_CUDA(cudaMalloc(&L.t_res, bytes));
    MFP_CHECK_CUDA(cudaMalloc(&L.t_d, bytes));
    MFP_CHECK_CUDA(cudaMalloc(&L.t_x, bytes));
    MFP_CHECK_CUDA(cudaMalloc(&L.t_b, bytes));
    L.scratch_rhs = R;
  }
  for (auto& L : c->levels) ensure_fbuf(c, L, R, nullptr);
  if (c->cg_rhs < R) {
    const int64_t n = c->levels.back().ndofs * (int64_t)R;
    dfree(c->cg_r);
    dfree(c->cg_p);
    dfree(c->cg_ap);
    dfree(c->cg_z);
    dfree(c->mix_r);
    dfree(c->mix_z);
    c->cg_r = dalloc<double>(n);
    c->cg_p = dalloc<double>(n);
    c->cg_ap = dalloc<double>(n);
    c->cg_z = dalloc<double>(n);
    if (c->vprec == MFP_FP32) {
      c->mix_r = dalloc<float>(n);
      c->mix_z = dalloc<float>(n);
    }
    c->cg_rhs = R;
  }
}

// V-cycle on the finest level, float64 in / out.
void vcycle_top(mfp_ctx* c, const double* r, double* z, int R,
                cudaStream_t s) {
  const int top = (int)c->levels.size() - 1;
  const int64_t n = c->levels[top].ndofs * (int64_t)R;
  if (c->vprec == MFP_FP32) {
    launch_to_float(r, c->mix_r, n, s);
    vcycle_level<float>(c, top, c->mix_r, c->mix_z, R, s);
    launch_to_double(c->mix_z, z, n, s);
  } else {
    vcycle_level<double>(c, top, r, z, R, s);
  }
  c->vcycles += R;
}

void drop_graphs(mfp_ctx* c) {
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

bool graphs_enabled() {
  const char* e = std::getenv("MFP_CUDA_GRAPHS");
  return !(e && e[0] == '0');
}

// The solve's V-cycle (internal buffers cg_r -> cg_z) replayed from a CUDA
// graph captured on its first use for this column count.  The capture does
// not execute work, so the counter increments it made are taken back and
// re-added on every replay.
void vcycle_solve(mfp_ctx* c, int R, cudaStream_t s) {
  if (!graphs_enabled()) {
    vcycle_top(c, c->cg_r, c->cg_z, R, s);
    return;
  }
  if ((int)c->graphs.size() <= R) c->graphs.resize(R + 1);
  mfp_ctx::VGraph& g = c->graphs[R];
  if (!g.exec) {
    std::vector<int64_t> a0;
    for (auto& L : c->levels) a0.push_back(L.applies);
    const int64_t l0 = launches_total(), v0 = c->vcycles;
    // capture on the context's own stream (the legacy default stream cannot
    // be captured); the graph is then launched on the caller's stream
    if (!c->cap_stream)
      MFP_CHECK_CUDA(
          cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = c->cap_stream;
    MFP_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
      vcycle_top(c, c->cg_r, c->cg_z, R, cs);
    } catch (...) {
      cudaStreamEndCapture(cs, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      for (size_t l = 0; l < c->levels.size(); ++l) c->levels[l].applies = a0[l];
      throw;
    }
    MFP_CHECK_CUDA(cudaStreamEndCapture(cs, &graph));
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    MFP_CHECK_CUDA(e);
    g.applies.resize(c->levels.size());
    for (size_t l = 0; l < c->levels.size(); ++l) {
      g.applies[l] = c->levels[l].applies - a0[l];
      c->levels[l].applies = a0[l];
    }
    g.launches = launches_total() - l0;
    add_launches(-g.launches);
    g.vcycles = c->vcycles - v0;
    c->vcycles = v0;
  }
  MFP_CHECK_CUDA(cudaGraphLaunch(g.exec, s));
  for (size_t l = 0; l < c->levels.size(); ++l)
    c->levels[l].applies += g.applies[l];
  add_launches(g.launches);
  c->vcycles += g.vcycles;
}

// Eigenvalue estimate of D^{-1} A on level l (Sec. 4.1): Jacobi-PCG from the
// start vector, Lanczos tridiagonal, bisection; all on the device.
void estimate_eigenvalues(mfp_ctx* c, int l, cudaStream_t s) {
  Level& L = c->levels[l];
  const int64_t n = L.ndofs;
  double* r = c->cg_r;
  double* z = c->cg_z;
  double* p = c->cg_p;
  double* ap = c->cg_ap;
  double init[S_COUNT] = {0};
  init[S_ACTIVE] = 1.0;
  MFP_CHECK_CUDA(cudaMemcpyAsync(c->scal, init, sizeof(init),
                                 cudaMemcpyHostToDevice, s));
  launch_start_vector(L, r, s);
  launch_jacobi(r, L.d64.dinv, z, n, 1, s);
  MFP_CHECK_CUDA(cudaMemcpyAsync(p, z, n * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
  launch_dot(r, z, n, 1, c->red, c->scal, 0, nullptr, 0, s);
  const int iters = c->desc.eig_cg_iters;
  for (int j = 0; j < iters; ++j) {
    apply_level<double>(c, L, p, ap, 1, s);
    launch_dot(p, ap, n, 1, c->red, c->scal, 1, c->hist, j, s);
    launch_cg_update(nullptr, r, p, ap, n, 1, c->red, c->scal, s);
    launch_jacobi(r, L.d64.dinv, z, n, 1, s);
    launch_dot(r, z, n, 1, c->red, c->scal, 2, c->hist, j, s);
    launch_cg_p(p, z, n, 1, c->scal, s);
  }
  launch_lanczos(c->hist, c->scal, c->eig_out, s);
  double out[2];
  MFP_CHECK_CUDA(cudaMemcpyAsync(out, c->eig_out, sizeof(out),
                                 cudaMemcpyDeviceToHost, s));
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
  L.lam_max = std::isfinite(out[0]) && out[0] > 0 ? out[0] : 1.0;
  L.lam_min = std::isfinite(out[1]) && out[1] > 0 ? out[1] : L.lam_max;
  if (l == 0) {
    L.cheb_lo = 0.9 * L.lam_min;
    L.cheb_hi = 1.2 * L.lam_max;
    const double cond = L.cheb_hi / L.cheb_lo;
    const double rho = (std::sqrt(cond) - 1.0) / (std::sqrt(cond) + 1.0);
    int m = 1;
    while (2.0 * std::pow(rho, m) / (1.0 + std::pow(rho, 2 * m)) >= 1e-3 &&
           m < 10000)
      ++m;
    L.cheb_degree = m;
  } else {
    L.cheb_hi = 1.2 * L.lam_max;
    L.cheb_lo = 0.06 * L.lam_max;
    L.cheb_degree = c->desc.cheb_degree;
  }
  L.applies = 0;
}

void to_float_array(const double* a, float*& b, int64_t n, cudaStream_t s);

void free_dense(Level& L) {
  dfree(L.dense64);
  dfree(L.dense32);
  dfree(L.csolve64);
  dfree(L.csolve32);
  dfree(L.dpart);
  dfree(L.dcnt);
}

// The coarse solve of Sec. 4.1 (Chebyshev from a zero start with the degree
// and interval fixed at set-up) is a fixed polynomial in D^{-1} A applied to
// D^{-1} b, so it is one linear operator: its matrix is found once by running
// that iteration on blocks of identity columns, and each V-cycle then applies
// it with one dense product instead of its degree's worth of operator
// applications and vector updates.  Only the evaluation order (rounding)
// differs from running the iteration.
void assemble_coarse_solve(mfp_ctx* c, Level& L, cudaStream_t s) {
  const int64_t n = L.ndofs;
  const int blk = kMaxRhs;
  double* M = dalloc<double>(n * n);
  double* E = dalloc<double>(n * blk);
  double* X = dalloc<double>(n * blk);
  double* tres = dalloc<double>(n * blk);
  double* td = dalloc<double>(n * blk);
  void* keep_res = L.t_res;
  void* keep_d = L.t_d;
  L.t_res = tres;
  L.t_d = td;
  const int64_t keep_applies = L.applies;
  for (int64_t c0 = 0; c0 < n; c0 += blk) {
    const int R = (int)(n - c0 < blk ? n - c0 : blk);
    launch_identity_block(E, n, c0, R, s);
    smooth<double>(c, 0, E, X, true, R, s);
    launch_store_columns(X, M, n, c0, R, s);
  }
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
  L.t_res = keep_res;
  L.t_d = keep_d;
  L.applies = keep_applies;
  dfree(E);
  dfree(X);
  dfree(tres);
  dfree(td);
  if (c->vprec == MFP_FP32) to_float_array(M, L.csolve32, n * n, s);
  L.csolve64 = M;
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
}

// Assembles the operator of a coarsest level with at most kDenseMax dofs as a
// dense matrix, by matrix-free applies to blocks of identity columns.
void assemble_dense(mfp_ctx* c, Level& L, cudaStream_t s) {
  free_dense(L);
  const int64_t n = L.ndofs;
  if (n > kDenseMax) return;
  const int blk = kMaxRhs;
  double* A = dalloc<double>(n * n);
  double* E = dalloc<double>(n * blk);
  double* Y = dalloc<double>(n * blk);
  for (int64_t c0 = 0; c0 < n; c0 += blk) {
    const int R = (int)(n - c0 < blk ? n - c0 : blk);
    launch_identity_block(E, n, c0, R, s);
    apply_level<double>(c, L, E, Y, R, s);
    launch_store_columns(Y, A, n, c0, R, s);
  }
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
  dfree(E);
  dfree(Y);
  L.dpart = dalloc<double>((int64_t)kDenseSplit * kMaxRhs * n);
  const int64_t nrb = (n + kDenseRows - 1) / kDenseRows;
  MFP_CHECK_CUDA(cudaMalloc(&L.dcnt, nrb * kMaxRhs * sizeof(unsigned)));
  MFP_CHECK_CUDA(
      cudaMemsetAsync(L.dcnt, 0, nrb * kMaxRhs * sizeof(unsigned), s));
  if (c->vprec == MFP_FP32) to_float_array(A, L.dense32, n * n, s);
  L.dense64 = A;
  L.applies = 0;
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
  assemble_coarse_solve(c, L, s);
}

void free_level(Level& L) {
  for (LevelData<double>* D : {&L.d64}) {
    dfree(D->G);
    dfree(D->kcell);
    dfree(D->kface);
    dfree(D->fdata);
    dfree(D->sigma);
    dfree(D->dinv);
  }
  dfree(L.d32.G);
  dfree(L.d32.kcell);
  dfree(L.d32.kface);
  dfree(L.d32.fdata);
  dfree(L.d32.sigma);
  dfree(L.d32.dinv);
  for (float** p : {&L.ddf.Gh, &L.ddf.Gl, &L.ddf.kch, &L.ddf.kcl, &L.ddf.kfh,
                    &L.ddf.kfl, &L.ddf.fdh, &L.ddf.fdl, &L.ddf.sgh,
                    &L.ddf.sgl})
    dfree(*p);
  dfree(L.vol);
  dfree(L.nodes);
  dfree(L.t_res);
  dfree(L.t_d);
  dfree(L.t_x);
  dfree(L.t_b);
  dfree(L.fbuf);
  free_dense(L);
}

void free_ctx(mfp_ctx* c) {
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  for (auto& L : c->levels) free_level(L);
  dfree(c->cg_r);
  dfree(c->cg_p);
  dfree(c->cg_ap);
  dfree(c->cg_z);
  dfree(c->scal);
  dfree(c->hist);
  dfree(c->eig_out);
  dfree(c->params);
  dfree(c->hdg_lam);
  dfree(c->hdg_cell);
  dfree(c->hdg_face);
  dfree(c->red.part);
  dfree(c->red.cnt);
  dfree(c->dev_err);
  dfree(c->mix_r);
  dfree(c->mix_z);
  if (c->host_scal) cudaFreeHost(c->host_scal);
  c->host_scal = nullptr;
}

void to_float_array(const double* a, float*& b, int64_t n, cudaStream_t s) {
  if (!a) return;
  if (!b) b = dalloc<float>(n);
  launch_to_float(a, b, n, s);
}

void split_array(const double* a, float*& hi, float*& lo, int64_t n,
                 cudaStream_t s) {
  if (!a) return;
  if (!hi) hi = dalloc<float>(n);
  if (!lo) lo = dalloc<float>(n);
  launch_split(a, hi, lo, n, s);
}

// Double-float copies of the float64 level data for the FP64-accurate
// applies on the FP32 pipes.
void build_df(Level& L, cudaStream_t s) {
  const int64_t P3 = (int64_t)L.p * L.p * L.p, P2 = (int64_t)L.p * L.p;
  LevelDF& F = L.ddf;
  split_array(L.d64.G, F.Gh, F.Gl, L.ncells * 6 * P3, s);
  split_array(L.d64.kcell, F.kch, F.kcl, L.ncells * P3, s);
  split_array(L.d64.kface, F.kfh, F.kfl, L.nfaces * P2, s);
  split_array(L.d64.fdata, F.fdh, F.fdl, L.nfaces * 7 * P2, s);
  split_array(L.d64.sigma, F.sgh, F.sgl, L.nfaces, s);
  F.valid = true;
}

// Geometry, diagonal and eigenvalue estimate of every level.
void build_levels(mfp_ctx* c, cudaStream_t s) {
  drop_graphs(c);  // Chebyshev parameters are baked into captured V-cycles
  const bool f32 = c->vprec == MFP_FP32;
  for (size_t l = 0; l < c->levels.size(); ++l) {
    Level& L = c->levels[l];
    const int64_t P3 = (int64_t)L.p * L.p * L.p, P2 = (int64_t)L.p * L.p;
    if (L.curved) {
      if (!L.d64.G) L.d64.G = dalloc<double>(L.ncells * 6 * P3);
      // one spare cell: the staged float kernel's last bulk copy is rounded
      // up to 16 bytes
      if (f32 && !L.d32.G) L.d32.G = dalloc<float>((L.ncells + 1) * 6 * P3);
      if (!L.vol) L.vol = dalloc<double>(L.ncells);
      launch_curved_cell_geometry(L, s);
      if (L.disc == MFP_SIPG) {
        if (!L.d64.fdata) L.d64.fdata = dalloc<double>(L.nfaces * 7 * P2);
        if (!L.d64.sigma) L.d64.sigma = dalloc<double>(L.nfaces);
        if (f32 && !L.d32.fdata) L.d32.fdata = dalloc<float>(L.nfaces * 7 * P2);
        if (f32 && !L.d32.sigma) L.d32.sigma = dalloc<float>(L.nfaces);
        launch_curved_face_geometry(L, s);
      }
    }
    if (f32) {
      to_float_array(L.d64.kcell, L.d32.kcell, L.ncells * P3, s);
      to_float_array(L.d64.kface, L.d32.kface, L.nfaces * P2, s);
    }
    if (c->desc.fp64_arith == MFP_ARITH_DF) build_df(L, s);
    if (!L.d64.dinv) L.d64.dinv = dalloc<double>(L.ndofs);
    launch_diagonal(L, L.d64.dinv, s);
    launch_invert_diag(L, L.d64.dinv, s);
    L.d64.valid = true;
    if (f32) {
      to_float_array(L.d64.dinv, L.d32.dinv, L.ndofs, s);
      L.d32.valid = true;
    }
    if (l == 0) free_dense(L);  // stale after a coefficient change
    estimate_eigenvalues(c, (int)l, s);
    if (l == 0 && c->levels.size() > 1) assemble_dense(c, L, s);
  }
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
}

mfp_status guard_status(const Fail& f) { return f.st; }

#define API_BEGIN \
  try {           \
    ::mfp::clear_error();
#define API_END                                                      \
  }                                                                  \
  catch (const ::mfp::Fail& f) {                                     \
    return f.st;                                                     \
  }                                                                  \
  catch (const std::bad_alloc&) {                                    \
    ::mfp::set_error("host allocation failed");                      \
    return MFP_ERR_OOM;                                              \
  }                                                                  \
  catch (...) {                                                      \
    ::mfp::set_error("unexpected exception");                        \
    return MFP_ERR_CUDA;                                             \
  }                                                                  \
  return MFP_OK;

Level& get_level(mfp_ctx* c, int level) {
  MFP_REQUIRE(c, "null context");
  MFP_REQUIRE(level >= 0 && level < (int)c->levels.size(),
              "level out of range");
  return c->levels[level];
}

int prec_of(int prec) {
  MFP_REQUIRE(prec == MFP_FP64 || prec == MFP_FP32 || prec == MFP_MIXED,
              "prec must be MFP_FP64 or MFP_FP32");
  return prec == MFP_FP64 ? MFP_FP64 : MFP_FP32;
}

}  // namespace
}  // namespace mfp

using namespace mfp;

extern "C" {

void mfp_desc_default(mfp_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->nx = d->ny = d->nz = 1;
  d->degree = 1;
  d->disc = MFP_CG;
  d->n_levels = 0;
  d->mapping = MFP_MAP_IDENTITY;
  d->map_param = 0.0;
  d->kappa = 1.0;
  d->penalty_factor = 1.0;
  d->mg_precision = MFP_FP64;
  d->cheb_degree = 5;
  d->eig_cg_iters = 15;
  d->fp64_arith = MFP_ARITH_DF;
  d->neumann_sides = 0;
  d->box_lo = 0.0;
  d->box_hi = 1.0;
}

const char* mfp_last_error(void) { return g_err.c_str(); }

mfp_status mfp_create(const mfp_desc* desc, void* stream, mfp_ctx** out) {
  mfp_ctx* c = nullptr;
  try {
    clear_error();
    MFP_REQUIRE(desc && out, "null argument");
    *out = nullptr;
    const mfp_desc& d = *desc;
    MFP_REQUIRE(d.nx >= 1 && d.ny >= 1 && d.nz >= 1, "cell counts must be >= 1");
    MFP_REQUIRE(d.degree >= 1 && d.degree <= 8, "degree must be in 1..8");
    MFP_REQUIRE(d.disc == MFP_CG || d.disc == MFP_SIPG, "unknown disc");
    MFP_REQUIRE(d.mapping == MFP_MAP_IDENTITY || d.mapping == MFP_MAP_SINE ||
                    d.mapping == MFP_MAP_NODES,
                "unknown mapping");
    MFP_REQUIRE(d.mapping != MFP_MAP_NODES || d.map_nodes,
                "MFP_MAP_NODES needs map_nodes");
    MFP_REQUIRE(d.mapping != MFP_MAP_NODES ||
                    (d.box_lo == 0.0 && d.box_hi == 1.0),
                "MFP_MAP_NODES: the nodes are physical points, leave the box "
                "at [0, 1]");
    MFP_REQUIRE(d.mapping != MFP_MAP_SINE ||
                    std::fabs(d.map_param) * 3.14159265358979 * std::sqrt(3.0) < 1.0,
                "map_param too large: the mapping would fold");
    MFP_REQUIRE(d.kappa > 0, "kappa must be > 0");
    MFP_REQUIRE(d.neumann_sides >= 0 && d.neumann_sides < 63,
                "neumann_sides must be a mask of sides 0..5 that leaves at "
                "least one Dirichlet side");
    MFP_REQUIRE(std::isfinite(d.box_lo) && std::isfinite(d.box_hi) &&
                    d.box_hi > d.box_lo,
                "box_hi must exceed box_lo");
    MFP_REQUIRE(d.penalty_factor > 0, "penalty_factor must be > 0");
    MFP_REQUIRE(d.cheb_degree >= 1 && d.cheb_degree <= 64,
                "cheb_degree must be in 1..64");
    MFP_REQUIRE(d.eig_cg_iters >= 1 && d.eig_cg_iters <= 64,
                "eig_cg_iters must be in 1..64");
    MFP_REQUIRE(d.fp64_arith == MFP_ARITH_DF || d.fp64_arith == MFP_ARITH_NATIVE,
                "unknown fp64_arith");
    MFP_REQUIRE(d.mg_precision == MFP_FP64 || d.mg_precision == MFP_FP32 ||
                    d.mg_precision == MFP_MIXED,
                "unknown mg_precision");
    const int64_t cells = (int64_t)d.nx * d.ny * d.nz;
    const int64_t p3 = (int64_t)(d.degree + 1) * (d.degree + 1) * (d.degree + 1);
    MFP_REQUIRE(cells * p3 < (int64_t)1 << 31, "mesh too large");
    // level count
    int nl = d.n_levels;
    int n0 = d.nx, n1 = d.ny, n2 = d.nz;
    if (nl <= 0) {
      nl = 1;
      while (n0 % 2 == 0 && n1 % 2 == 0 && n2 % 2 == 0 && n0 >= 4 && n1 >= 4 &&
             n2 >= 4) {
        n0 /= 2;
        n1 /= 2;
        n2 /= 2;
        ++nl;
      }
    } else {
      for (int i = 1; i < nl; ++i) {
        MFP_REQUIRE(n0 % 2 == 0 && n1 % 2 == 0 && n2 % 2 == 0,
                    "cell counts cannot be halved n_levels-1 times");
        n0 /= 2;
        n1 /= 2;
        n2 /= 2;
      }
    }
    c = new mfp_ctx();
    c->desc = d;
    c->vprec = d.mg_precision == MFP_FP64 ? MFP_FP64 : MFP_FP32;
    MFP_CHECK_CUDA(cudaGetDevice(&c->device));
    c->levels.resize(nl);
    for (int l = 0; l < nl; ++l) {
      Level& L = c->levels[l];
      const int sh = nl - 1 - l;
      L.n[0] = d.nx >> sh;
      L.n[1] = d.ny >> sh;
      L.n[2] = d.nz >> sh;
      L.k = d.degree;
      L.p = d.degree + 1;
      L.disc = d.disc;
      L.curved = (d.mapping == MFP_MAP_SINE && d.map_param != 0.0) ||
                 d.mapping == MFP_MAP_NODES;
      L.map_amp = d.mapping == MFP_MAP_SINE ? d.map_param : 0.0;
      L.kappa = d.kappa;
      L.penalty = d.penalty_factor;
      L.ncells = (int64_t)L.n[0] * L.n[1] * L.n[2];
      L.box_lo = d.box_lo;
      L.box_len = d.box_hi - d.box_lo;
      for (int e = 0; e < 3; ++e) {
        L.gdim[e] = L.n[e] * L.k + 1;
        L.h[e] = L.box_len / L.n[e];
        L.bc.lo[e] = (d.neumann_sides >> (2 * e)) & 1 ? -1 : 0;
        L.bc.hi[e] = (d.neumann_sides >> (2 * e + 1)) & 1 ? -1 : L.gdim[e] - 1;
      }
      L.bc.neumann = d.neumann_sides;
      L.df_arith = d.fp64_arith == MFP_ARITH_DF;
      L.ndofs = d.disc == MFP_CG ? (int64_t)L.gdim[0] * L.gdim[1] * L.gdim[2]
                                 : L.ncells * L.p * L.p * L.p;
      int64_t off = 0;
      for (int e = 0; e < 3; ++e) {
        int m[3] = {L.n[0], L.n[1], L.n[2]};
        m[e] += 1;
        L.face_off[e] = (int)off;
        off += (int64_t)m[0] * m[1] * m[2];
      }
      L.nfaces = off;
    }
    c->scal = dalloc<double>((int64_t)S_COUNT * kMaxRhs);
    c->hist = dalloc<double>(128);
    c->eig_out = dalloc<double>(2);
    c->red.part = dalloc<double>((int64_t)kMaxRedBlocks * kMaxRhs);
    c->red.cnt = dalloc<unsigned>(1);
    c->dev_err = dalloc<int>(1);
    MFP_CHECK_CUDA(cudaMemsetAsync(c->dev_err, 0, sizeof(int), st(stream)));
    for (auto& L : c->levels) L.err = c->dev_err;
    MFP_CHECK_CUDA(cudaMemsetAsync(c->red.cnt, 0, sizeof(unsigned), st(stream)));
    MFP_CHECK_CUDA(cudaMallocHost(&c->host_scal,
                                  sizeof(double) * S_COUNT * kMaxRhs));
    ensure_scratch(c, 1);
    if (d.mapping == MFP_MAP_NODES) {
      // the given support points on the finest level, re-interpolated on
      // the coarser ones
      Level& F = c->levels.back();
      const int64_t n = F.ncells * p3 * 3;
      F.nodes = dalloc<double>(n);
      MFP_CHECK_CUDA(cudaMemcpyAsync(F.nodes, d.map_nodes, n * sizeof(double),
                                     cudaMemcpyHostToDevice, st(stream)));
      for (int l = nl - 2; l >= 0; --l) {
        Level& C = c->levels[l];
        C.nodes = dalloc<double>(C.ncells * p3 * 3);
        launch_coarsen_nodes(c->levels[l + 1], C, st(stream));
      }
      MFP_CHECK_CUDA(cudaStreamSynchronize(st(stream)));
    }
    build_levels(c, st(stream));
    noalloc_prepare(c->device, d.degree + 1);
    *out = c;
    return MFP_OK;
  } catch (const Fail& f) {
    if (c) {
      free_ctx(c);
      delete c;
    }
    return f.st;
  } catch (const std::bad_alloc&) {
    if (c) {
      free_ctx(c);
      delete c;
    }
    set_error("host allocation failed");
    return MFP_ERR_OOM;
  }
}

mfp_status mfp_destroy(mfp_ctx* c) {
  if (!c) return MFP_OK;
  cudaDeviceSynchronize();
  free_ctx(c);
  delete c;
  return MFP_OK;
}

int mfp_n_levels(const mfp_ctx* c) { return c ? (int)c->levels.size() : 0; }

mfp_status mfp_sizes(const mfp_ctx* c, int level, int64_t* n_dofs,
                     int64_t* n_cell_qp, int64_t* n_face_qp) {
  API_BEGIN
  Level& L = get_level(const_cast<mfp_ctx*>(c), level);
  const int64_t p = L.p;
  if (n_dofs) *n_dofs = L.ndofs;
  if (n_cell_qp) *n_cell_qp = L.ncells * p * p * p;
  if (n_face_qp) *n_face_qp = L.nfaces * p * p;
  API_END
}

mfp_status mfp_set_coefficient(mfp_ctx* c, const double* a_cell,
                               const double* a_face, void* stream) {
  API_BEGIN
  MFP_REQUIRE(c && a_cell, "null argument");
  MFP_REQUIRE(c->desc.disc == MFP_CG || a_face,
              "SIPG needs the face coefficient");
  cudaStream_t s = st(stream);
  const int nl = (int)c->levels.size();
  for (int l = nl - 1; l >= 0; --l) {
    Level& L = c->levels[l];
    const int64_t P3 = (int64_t)L.p * L.p * L.p, P2 = (int64_t)L.p * L.p;
    if (!L.d64.kcell) L.d64.kcell = dalloc<double>(L.ncells * P3);
    if (!L.d64.kface) L.d64.kface = dalloc<double>(L.nfaces * P2);
    if (l == nl - 1) {
      MFP_CHECK_CUDA(cudaMemcpyAsync(L.d64.kcell, a_cell,
                                     L.ncells * P3 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
      if (a_face)
        MFP_CHECK_CUDA(cudaMemcpyAsync(L.d64.kface, a_face,
                                       L.nfaces * P2 * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
      else
        launch_fill<double>(L.d64.kface, 1.0, L.nfaces * P2, s);
    } else {
      launch_coarsen_coefficient(c->levels[l + 1], L, s);
    }
  }
  c->has_coef = true;
  build_levels(c, s);
  API_END
}

mfp_status mfp_rhs(mfp_ctx* c, int f_kind, const double* params, int nterms,
                   double* b, int64_t stride, void* stream) {
  API_BEGIN
  MFP_REQUIRE(c && b, "null argument");
  MFP_REQUIRE(f_kind >= 0 && f_kind <= 2, "unknown f_kind");
  MFP_REQUIRE(stride >= 1, "stride must be >= 1");
  MFP_REQUIRE(f_kind != 2 || !c->has_coef,
              "f_kind 2 needs the constant coefficient");
  cudaStream_t s = st(stream);
  if (f_kind >= 1) {
    MFP_REQUIRE(params && nterms >= 1 && nterms <= kMaxGaussTerms,
                "bad Gaussian terms (1..4096)");
    if (c->params_cap < nterms) {
      dfree(c->params);
      c->params = dalloc<double>(5 * (int64_t)nterms);
      c->params_cap = nterms;
    }
    MFP_CHECK_CUDA(cudaMemcpyAsync(c->params, params,
                                   5 * sizeof(double) * nterms,
                                   cudaMemcpyHostToDevice, s));
    MFP_CHECK_CUDA(cudaStreamSynchronize(s));  // host params may go away
  }
  launch_rhs(c->levels.back(), f_kind, c->params, nterms, b, stride, s);
  API_END
}

mfp_status mfp_hdg_apply(mfp_ctx* c, double tau_factor, const double* x,
                         double* y, void* stream) {
  API_BEGIN
  MFP_REQUIRE(c && x && y && x != y, "x / y must be distinct non-null");
  MFP_REQUIRE(c->desc.disc == MFP_SIPG,
              "the HDG operator uses the cells of an SIPG context");
  Level& L = c->levels.back();
  MFP_REQUIRE(tau_factor > 0 && std::isfinite(tau_factor),
              "tau_factor must be > 0");
  MFP_REQUIRE(!c->has_coef || L.d64.kface,
              "HDG apply: a per-point coefficient needs its face values");
  const int64_t P3 = (int64_t)L.p * L.p * L.p, P2 = (int64_t)L.p * L.p;
  if (!c->hdg_lam) c->hdg_lam = dalloc<double>(L.nfaces * P2);
  if (L.curved && !c->hdg_cell) {
    // w det J, J^{-1} per cell point and dA, the normal per face point
    c->hdg_cell = dalloc<double>(L.ncells * 10 * P3);
    c->hdg_face = dalloc<double>(L.nfaces * 4 * P2);
    launch_curved_cell_geometry(L, st(stream), c->hdg_cell);
    launch_curved_face_geometry(L, st(stream), c->hdg_face);
  }
  launch_hdg_apply(L, tau_factor, c->hdg_lam, c->hdg_cell, c->hdg_face, x, y,
                   st(stream));
  API_END
}

mfp_status mfp_apply(mfp_ctx* c, int level, int prec, const void* src,
                     void* dst, int n_rhs, void* stream) {
  API_BEGIN
  Level& L = get_level(c, level);
  MFP_REQUIRE(src && dst && src != dst, "src / dst must be distinct non-null");
  MFP_REQUIRE(n_rhs >= 1 && n_rhs <= kMaxRhs, "n_rhs must be in 1..256");
  if (prec_of(prec) == MFP_FP64)
    apply_level<double>(c, L, static_cast<const double*>(src),
                        static_cast<double*>(dst), n_rhs, st(stream));
  else
    apply_level<float>(c, L, static_cast<const float*>(src),
                       static_cast<float*>(dst), n_rhs, st(stream));
  API_END
}

mfp_status mfp_inverse_diagonal(mfp_ctx* c, int level, int prec, void* out,
                                void* stream) {
  API_BEGIN
  Level& L = get_level(c, level);
  MFP_REQUIRE(out, "null argument");
  if (prec_of(prec) == MFP_FP64) {
    MFP_CHECK_CUDA(cudaMemcpyAsync(out, L.d64.dinv, L.ndofs * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st(stream)));
  } else {
    MFP_REQUIRE(L.d32.valid, "no float level data (mg_precision FP64)");
    MFP_CHECK_CUDA(cudaMemcpyAsync(out, L.d32.dinv, L.ndofs * sizeof(float),
                                   cudaMemcpyDeviceToDevice, st(stream)));
  }
  API_END
}

mfp_status mfp_level_info(const mfp_ctx* c, int level, double* lam_max,
                          double* lam_min, double* lo, double* hi,
                          int* degree) {
  API_BEGIN
  Level& L = get_level(const_cast<mfp_ctx*>(c), level);
  if (lam_max) *lam_max = L.lam_max;
  if (lam_min) *lam_min = L.lam_min;
  if (lo) *lo = L.cheb_lo;
  if (hi) *hi = L.cheb_hi;
  if (degree) *degree = L.cheb_degree;
  API_END
}

mfp_status mfp_prolongate(mfp_ctx* c, int level, int prec, const void* xc,
                          void* xf, void* stream) {
  API_BEGIN
  get_level(c, level);
  MFP_REQUIRE(level >= 1, "level must be >= 1");
  MFP_REQUIRE(xc && xf, "null argument");
  if (prec_of(prec) == MFP_FP64)
    prolongate<double>(c, level, static_cast<const double*>(xc),
                       static_cast<double*>(xf), 1, st(stream));
  else
    prolongate<float>(c, level, static_cast<const float*>(xc),
                      static_cast<float*>(xf), 1, st(stream));
  API_END
}

mfp_status mfp_restrict(mfp_ctx* c, int level, int prec, const void* xf,
                        void* xc, void* stream) {
  API_BEGIN
  get_level(c, level);
  MFP_REQUIRE(level >= 1, "level must be >= 1");
  MFP_REQUIRE(xc && xf, "null argument");
  if (prec_of(prec) == MFP_FP64)
    restrict_<double>(c, level, static_cast<const double*>(xf),
                      static_cast<double*>(xc), 1, st(stream));
  else
    restrict_<float>(c, level, static_cast<const float*>(xf),
                     static_cast<float*>(xc), 1, st(stream));
  API_END
}

mfp_status mfp_smooth(mfp_ctx* c, int level, int prec, const void* b,
                      void* x, int zero_start, void* stream) {
  API_BEGIN
  get_level(c, level);
  MFP_REQUIRE(b && x && b != x, "b / x must be distinct non-null");
  const int pr = prec_of(prec);
  MFP_REQUIRE(pr == c->vprec || pr == MFP_FP64,
              "float smoothing needs mg_precision MFP_FP32");
  if (pr == MFP_FP64) {
    MFP_REQUIRE(c->vprec == MFP_FP64,
                "float64 smoothing needs mg_precision MFP_FP64 scratch");
    smooth<double>(c, level, static_cast<const double*>(b),
                   static_cast<double*>(x), zero_start != 0, 1, st(stream));
  } else {
    smooth<float>(c, level, static_cast<const float*>(b),
                  static_cast<float*>(x), zero_start != 0, 1, st(stream));
  }
  API_END
}

mfp_status mfp_vcycle(mfp_ctx* c, const double* r, double* z, int n_rhs,
                      void* stream) {
  API_BEGIN
  MFP_REQUIRE(c && r && z && r != z, "r / z must be distinct non-null");
  ensure_scratch(c, n_rhs);
  vcycle_top(c, r, z, n_rhs, st(stream));
  API_END
}

mfp_status mfp_solve(mfp_ctx* c, const double* b, double* x, int R,
                     double rtol, int max_it, int* iters_out,
                     double* relres_out, void* stream) {
  API_BEGIN
  MFP_REQUIRE(c && b && x && b != x, "b / x must be distinct non-null");
  MFP_REQUIRE(rtol > 0 && max_it >= 1, "rtol must be > 0, max_it >= 1");
  ensure_scratch(c, R);
  cudaStream_t s = st(stream);
  Level& L = c->levels.back();
  const int64_t n = L.ndofs;
  double* h = c->host_scal;
  // |b|^2, x = 0, r = b
  std::vector<double> init((size_t)S_COUNT * R, 0.0);
  for (int r = 0; r < R; ++r) init[(size_t)S_ACTIVE * R + r] = 1.0;
  MFP_CHECK_CUDA(cudaMemcpyAsync(c->scal, init.data(),
                                 init.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
  launch_dot(b, b, n, R, c->red, c->scal, 3, nullptr, 0, s);
  MFP_CHECK_CUDA(cudaMemcpyAsync(h, c->scal + (size_t)S_BN2 * R,
                                 R * sizeof(double), cudaMemcpyDeviceToHost,
                                 s));
  MFP_CHECK_CUDA(cudaMemsetAsync(x, 0, n * R * sizeof(double), s));
  MFP_CHECK_CUDA(cudaMemcpyAsync(c->cg_r, b, n * R * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
  std::vector<double> bn2(h, h + R);
  std::vector<int> its(R, 0);
  std::vector<double> rel(R, 0.0);
  std::vector<char> active(R, 1);
  int n_active = R;
  for (int r = 0; r < R; ++r)
    if (bn2[r] == 0.0) {
      active[r] = 0;
      --n_active;
    }
  auto upload_active = [&]() {
    for (int r = 0; r < R; ++r) h[r] = active[r] ? 1.0 : 0.0;
    MFP_CHECK_CUDA(cudaMemcpyAsync(c->scal + (size_t)S_ACTIVE * R, h,
                                   R * sizeof(double),
                                   cudaMemcpyHostToDevice, s));
    MFP_CHECK_CUDA(cudaStreamSynchronize(s));  // h is reused below
  };
  upload_active();
  vcycle_top(c, c->cg_r, c->cg_z, R, s);
  MFP_CHECK_CUDA(cudaMemcpyAsync(c->cg_p, c->cg_z, n * R * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
  launch_dot(c->cg_r, c->cg_z, n, R, c->red, c->scal, 0, nullptr, 0, s);
  const double tol2 = rtol * rtol;
  int it = 0;
  while (n_active > 0 && it < max_it) {
    ++it;
    apply_level<double>(c, L, c->cg_p, c->cg_ap, R, s);
    launch_dot(c->cg_p, c->cg_ap, n, R, c->red, c->scal, 1, nullptr, 0, s);
    launch_cg_update(x, c->cg_r, c->cg_p, c->cg_ap, n, R, c->red, c->scal, s);
    MFP_CHECK_CUDA(cudaMemcpyAsync(h, c->scal + (size_t)S_RN2 * R,
                                   R * sizeof(double), cudaMemcpyDeviceToHost,
                                   s));
    MFP_CHECK_CUDA(cudaStreamSynchronize(s));
    bool changed = false;
    for (int r = 0; r < R; ++r) {
      if (!active[r]) continue;
      its[r] = it;
      rel[r] = std::sqrt(h[r] / bn2[r]);
      if (h[r] <= tol2 * bn2[r]) {
        active[r] = 0;
        --n_active;
        changed = true;
      }
    }
    if (n_active == 0) break;
    if (changed) upload_active();
    vcycle_solve(c, R, s);
    launch_dot(c->cg_r, c->cg_z, n, R, c->red, c->scal, 2, nullptr, 0, s);
    launch_cg_p(c->cg_p, c->cg_z, n, R, c->scal, s);
  }
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
  {
    int herr = 0;  // a staged kernel gave up waiting for its copies
    MFP_CHECK_CUDA(cudaMemcpyAsync(&herr, c->dev_err, sizeof(int),
                                   cudaMemcpyDeviceToHost, s));
    MFP_CHECK_CUDA(cudaStreamSynchronize(s));
    if (herr) {
      MFP_CHECK_CUDA(cudaMemsetAsync(c->dev_err, 0, sizeof(int), s));
      set_error("a kernel's shared-memory copy wait timed out; the result "
                "is invalid");
      return MFP_ERR_CUDA;
    }
  }
  if (iters_out)
    for (int r = 0; r < R; ++r) iters_out[r] = its[r];
  if (relres_out)
    for (int r = 0; r < R; ++r) relres_out[r] = rel[r];
  if (n_active > 0) {
    set_error("CG did not reach the tolerance within max_it iterations");
    return MFP_ERR_NOT_CONVERGED;
  }
  API_END
}

mfp_status mfp_gradient(mfp_ctx* c, const double* u, const double* lam,
                        double* gc, double* gf, void* stream) {
  API_BEGIN
  MFP_REQUIRE(c && u && lam && gc, "null argument");
  MFP_REQUIRE(c->desc.disc == MFP_CG || gf, "SIPG needs g_face");
  launch_gradient(c->levels.back(), u, lam, gc, gf, st(stream));
  API_END
}

mfp_status mfp_autotune(mfp_ctx* c, int level, int prec, int n_rhs,
                        int* cells_out, double* ms_out, void* stream) {
  API_BEGIN
  Level& L = get_level(c, level);
  MFP_REQUIRE(n_rhs >= 1 && n_rhs <= kMaxRhs, "n_rhs must be in 1..256");
  const int pr = prec_of(prec);
  cudaStream_t s = st(stream);
  const size_t esz = pr == MFP_FP64 ? sizeof(double) : sizeof(float);
  const size_t bytes = (size_t)L.ndofs * n_rhs * esz;
  void *src = nullptr, *dst = nullptr;
  MFP_CHECK_CUDA(cudaMalloc(&src, bytes));
  cudaError_t e = cudaMalloc(&dst, bytes);
  if (e != cudaSuccess) {
    cudaFree(src);
    MFP_CHECK_CUDA(e);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int64_t key = tune_key(level, pr, n_rhs);
  // drop a previous choice so the candidates below are what gets timed
  for (size_t i = 0; i < c->tuned.size(); ++i)
    if (c->tuned[i].first == key) {
      c->tuned.erase(c->tuned.begin() + i);
      break;
    }
  int best = 0;
  float best_ms = 1e30f;
  const int64_t a0 = L.applies;
  try {
    MFP_CHECK_CUDA(cudaEventCreate(&e0));
    MFP_CHECK_CUDA(cudaEventCreate(&e1));
    if (pr == MFP_FP64)
      launch_fill<double>(static_cast<double*>(src), 1.0, L.ndofs * n_rhs, s);
    else
      launch_fill<float>(static_cast<float*>(src), 1.0f, L.ndofs * n_rhs, s);
    const int p2 = L.p * L.p;
    const int cand[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 32};
    for (int cells : cand) {
      if ((int64_t)cells * n_rhs * p2 > 1024 && cells > 1) break;
      if (cells > L.ncells) break;
      c->tuned.push_back({key, cells});
      auto run = [&]() {
        if (pr == MFP_FP64)
          apply_level<double>(c, L, static_cast<const double*>(src),
                              static_cast<double*>(dst), n_rhs, s);
        else
          apply_level<float>(c, L, static_cast<const float*>(src),
                             static_cast<float*>(dst), n_rhs, s);
      };
      try {
        run();  // shapes that do not fit on an SM are skipped
      } catch (const Fail&) {
        cudaGetLastError();
        c->tuned.pop_back();
        continue;
      }
      MFP_CHECK_CUDA(cudaEventRecord(e0, s));
      for (int it = 0; it < 3; ++it) run();
      MFP_CHECK_CUDA(cudaEventRecord(e1, s));
      MFP_CHECK_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      MFP_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms /= 3;
      c->tuned.pop_back();
      if (ms < best_ms) {
        best_ms = ms;
        best = cells;
      }
    }
    // the warp-per-cell kernel of float CG applies (k <= 4, one column)
    if (L.disc == MFP_CG && pr == MFP_FP32 && n_rhs == 1 && L.p <= 5) {
      c->tuned.push_back({key, kWarpCells});
      auto run = [&]() {
        apply_level<float>(c, L, static_cast<const float*>(src),
                           static_cast<float*>(dst), n_rhs, s);
      };
      run();
      MFP_CHECK_CUDA(cudaEventRecord(e0, s));
      for (int it = 0; it < 3; ++it) run();
      MFP_CHECK_CUDA(cudaEventRecord(e1, s));
      MFP_CHECK_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      MFP_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms /= 3;
      c->tuned.pop_back();
      if (ms < best_ms) {
        best_ms = ms;
        best = kWarpCells;
      }
    }
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(src);
    cudaFree(dst);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(src);
  cudaFree(dst);
  L.applies = a0;
  MFP_REQUIRE(best > 0, "no admissible launch shape");
  clear_error();
  c->tuned.push_back({key, best});
  drop_graphs(c);  // captured V-cycles used the previous launch shapes
  if (cells_out) *cells_out = best == kWarpCells ? 0 : best;
  if (ms_out) *ms_out = best_ms;
  API_END
}

mfp_status mfp_counters(const mfp_ctx* c, int64_t* applies, int64_t* vcyc,
                        int64_t* launches) {
  API_BEGIN
  MFP_REQUIRE(c, "null context");
  if (launches) *launches = g_launches.load();
  if (applies)
    for (size_t l = 0; l < c->levels.size(); ++l)
      applies[l] = c->levels[l].applies;
  if (vcyc) *vcyc = c->vcycles;
  API_END
}

}  // extern "C"
