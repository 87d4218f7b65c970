// Vector kernels of the solver (Sec. 4.1): Chebyshev-Jacobi updates, level
// transfer by the tensorial geometric embedding, fused CG updates with
// deterministic two-stage reductions finished on the device, and the
// bisection for the extreme eigenvalues of the Lanczos tridiagonal.
#include "df.cuh"
#include "dev_tables.cuh"

namespace mfp {
namespace {

constexpr int kVecThreads = 256;

inline int vec_grid(int64_t n) {
  int64_t b = (n + kVecThreads - 1) / kVecThreads;
  int64_t cap = (int64_t)sm_count() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

#define GRID_STRIDE(i, n)                                                 \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

template <typename T>
__global__ void k_fill(T* x, T v, int64_t n) {
  GRID_STRIDE(i, n) x[i] = v;
}

__global__ void k_invert_diag(double* d, int64_t n, int g0, int g1, Bc bc,
                              int cg) {
  GRID_STRIDE(i, n) {
    bool con = false;
    if (cg) {
      const int64_t ix = i % g0, iy = (i / g0) % g1,
                    iz = i / ((int64_t)g0 * g1);
      con = bc_con(bc, ix, iy, iz);
    }
    d[i] = con ? 1.0 : 1.0 / d[i];
  }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b,
                           int64_t n) {
  GRID_STRIDE(i, n) b[i] = (float)a[i];
}
__global__ void k_split(const double* __restrict__ a, float* __restrict__ hi,
                        float* __restrict__ lo, int64_t n) {
  GRID_STRIDE(i, n) {
    const float h = __double2float_rn(a[i]);
    hi[i] = h;
    lo[i] = __double2float_rn(a[i] - (double)h);
  }
}

__global__ void k_to_double(const float* __restrict__ a,
                            double* __restrict__ b, int64_t n) {
  GRID_STRIDE(i, n) b[i] = (double)a[i];
}

// Chebyshev (Sec. 4.1; three-term recurrence on D^{-1} A):
//   first update: d = c D^{-1} (b - A x)   (ax == null: x = 0, residual b)
//   later:        d = cd d + cr D^{-1} (b - A x);   x += d.
// Vectors hold nrhs interleaved columns; dinv has one entry per row.
template <typename T>
__global__ void k_cheb_first(const T* __restrict__ b,
                             const T* __restrict__ dinv, T* __restrict__ d,
                             T* __restrict__ x, const T* __restrict__ ax, T c,
                             int64_t n, int nrhs) {
  GRID_STRIDE(i, n * nrhs) {
    const T r = ax ? b[i] - ax[i] : b[i];
    const T di = c * dinv[nrhs == 1 ? i : i / nrhs] * r;
    d[i] = di;
    x[i] = ax ? x[i] + di : di;
  }
}

template <typename T>
__global__ void k_cheb_step(const T* __restrict__ b,
                            const T* __restrict__ dinv, T* __restrict__ d,
                            T* __restrict__ x, const T* __restrict__ ax, T cd,
                            T cr, int64_t n, int nrhs) {
  GRID_STRIDE(i, n * nrhs) {
    const T di = cd * d[i] + cr * dinv[nrhs == 1 ? i : i / nrhs] * (b[i] - ax[i]);
    d[i] = di;
    x[i] += di;
  }
}

template <typename T>
__global__ void k_residual(const T* b, const T* ax, T* r, int64_t n) {
  GRID_STRIDE(i, n) r[i] = b[i] - ax[i];
}

template <typename T>
__global__ void k_axpy(T* __restrict__ y, const T* __restrict__ x, T a,
                       int64_t n) {
  GRID_STRIDE(i, n) y[i] += a * x[i];
}

// ---------------------------------------------------------------------------
// Transfer (Sec. 4.1: geometric embedding, done tensorially).  One block per
// coarse cell.  1D embedding E [M][p]: CG M = 2k+1 fine nodes inside the
// coarse cell (rows 0..k from the left child, k..2k from the right one, the
// middle row shared); SIPG M = 2p (left child's p rows, then right child's).
// ---------------------------------------------------------------------------
struct XferArgs {
  int nc[3];  // coarse cells per axis
  int gc[3];  // coarse CG grid
  int gf[3];  // fine CG grid
  int nf[3];  // fine cells per axis
  Bc bcc, bcf;  // CG constrained nodes of the coarse / fine grid
  int dg;
  int stride;  // columns (batched layout)
  int col;
};

template <typename T, int P>
__device__ __forceinline__ T emb(int o, int r, int j) {
  if constexpr (std::is_same<T, double>::value)
    return o ? c_tab64[P - 2].E1[r * P + j] : c_tab64[P - 2].E0[r * P + j];
  else
    return o ? c_tab32[P - 2].E1[r * P + j] : c_tab32[P - 2].E0[r * P + j];
}

// Arithmetic of the transfer sweeps: plain T, or (DF, float64 vectors of a
// double-float context) pairs of floats in shared memory accumulated with
// TwoSum / FMA TwoProd on the FP32 pipes; on GB300 the FP64 pipe would bound
// these sweeps (p multiply-adds per output) well below the memory rate.
template <typename T, bool DF>
struct XArith {
  using S = T;  // shared-memory element
  struct Acc {
    T v;
  };
  static __device__ __forceinline__ S load(T x) { return x; }
  static __device__ __forceinline__ Acc zero() { return Acc{T(0)}; }
  static __device__ __forceinline__ void mac(Acc& a, S e, S u) { a.v += e * u; }
  static __device__ __forceinline__ S get(const Acc& a) { return a.v; }
  static __device__ __forceinline__ T out(const Acc& a) { return a.v; }
};
template <>
struct XArith<double, true> {
  using S = float2;
  struct Acc {
    dacc d;
  };
  static __device__ __forceinline__ S load(double x) {
    const df v = df_from_double(x);
    return make_float2(v.h, v.l);
  }
  static __device__ __forceinline__ Acc zero() {
    Acc a;
    a.d.h = 0.f;
    a.d.l = 0.f;
    return a;
  }
  static __device__ __forceinline__ void mac(Acc& a, S e, S u) {
    acc_mac(a.d, e.x, e.y, u.x, u.y);
  }
  static __device__ __forceinline__ S get(const Acc& a) {
    const df v = acc_get(a.d);
    return make_float2(v.h, v.l);
  }
  static __device__ __forceinline__ double out(const Acc& a) {
    return df_to_double(acc_get(a.d));
  }
};

template <typename T, int P, bool DF>
__device__ void load_embedding(typename XArith<T, DF>::S* E, int dg) {
  using A = XArith<T, DF>;
  constexpr int K = P - 1;
  const int M = dg ? 2 * P : 2 * K + 1;
  for (int i = threadIdx.x; i < M * P; i += blockDim.x) {
    const int r = i / P, j = i % P;
    if (dg)
      E[i] = A::load(r < P ? emb<T, P>(0, r, j) : emb<T, P>(1, r - P, j));
    else
      E[i] = A::load(r <= K ? emb<T, P>(0, r, j) : emb<T, P>(1, r - K, j));
  }
}

template <typename T, int P, bool DF>
__global__ void k_prolongate(XferArgs a, const T* __restrict__ xc,
                             T* __restrict__ xf) {
  using A = XArith<T, DF>;
  using S = typename A::S;
  constexpr int K = P - 1;
  const int M = a.dg ? 2 * P : 2 * K + 1;
  extern __shared__ __align__(16) unsigned char xsm[];
  S* E = reinterpret_cast<S*>(xsm);
  S* u = E + M * P;
  S* t1 = u + P * P * P;
  S* t2 = t1 + P * P * M;
  const int C = blockIdx.x;
  a.col = blockIdx.y;  // one column of the batch per grid row
  const int cx = C % a.nc[0], cy = (C / a.nc[0]) % a.nc[1],
            cz = C / (a.nc[0] * a.nc[1]);
  load_embedding<T, P, DF>(E, a.dg);
  for (int i = threadIdx.x; i < P * P * P; i += blockDim.x) {
    const int ix = i % P, iy = (i / P) % P, iz = i / (P * P);
    T v;
    if (a.dg) {
      v = xc[((size_t)C * P * P * P + i) * a.stride + a.col];
    } else {
      const int X = cx * K + ix, Y = cy * K + iy, Z = cz * K + iz;
      v = bc_con(a.bcc, X, Y, Z)
              ? T(0)
              : xc[((size_t)X + (size_t)a.gc[0] * (Y + (size_t)a.gc[1] * Z)) *
                       a.stride +
                   a.col];
    }
    u[i] = A::load(v);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P * P * M; i += blockDim.x) {  // x
    const int fx = i % M, r = i / M;                            // r = iy + P iz
    auto s = A::zero();
    for (int j = 0; j < P; ++j) A::mac(s, E[fx * P + j], u[r * P + j]);
    t1[r * M + fx] = A::get(s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P * M * M; i += blockDim.x) {  // y
    const int fx = i % M, fy = (i / M) % M, iz = i / (M * M);
    auto s = A::zero();
    for (int j = 0; j < P; ++j)
      A::mac(s, E[fy * P + j], t1[(iz * P + j) * M + fx]);
    t2[i] = A::get(s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < M * M * M; i += blockDim.x) {  // z
    const int fx = i % M, fy = (i / M) % M, fz = i / (M * M);
    auto acc = A::zero();
    for (int j = 0; j < P; ++j)
      A::mac(acc, E[fz * P + j], t2[(j * M + fy) * M + fx]);
    const T s = A::out(acc);
    if (a.dg) {
      const int ox = fx / P, oy = fy / P, oz = fz / P;
      const int F = (2 * cx + ox) + a.nf[0] * ((2 * cy + oy) + a.nf[1] * (2 * cz + oz));
      const int loc = (fx % P) + P * ((fy % P) + P * (fz % P));
      xf[((size_t)F * P * P * P + loc) * a.stride + a.col] = s;
    } else {
      // each fine node is written by the coarse cell owning it
      const bool own = (fx < 2 * K || cx == a.nc[0] - 1) &&
                       (fy < 2 * K || cy == a.nc[1] - 1) &&
                       (fz < 2 * K || cz == a.nc[2] - 1);
      if (!own) continue;
      const int X = 2 * K * cx + fx, Y = 2 * K * cy + fy, Z = 2 * K * cz + fz;
      const size_t gi = (size_t)X + (size_t)a.gf[0] * (Y + (size_t)a.gf[1] * Z);
      xf[gi * a.stride + a.col] = bc_con(a.bcf, X, Y, Z) ? T(0) : s;
    }
  }
}

template <typename T, int P, bool DF>
__global__ void k_restrict(XferArgs a, const T* __restrict__ xf,
                           T* __restrict__ xc) {
  using A = XArith<T, DF>;
  using S = typename A::S;
  constexpr int K = P - 1;
  const int M = a.dg ? 2 * P : 2 * K + 1;
  extern __shared__ __align__(16) unsigned char xsm[];
  S* E = reinterpret_cast<S*>(xsm);
  S* u = E + M * P;
  S* t1 = u + M * M * M;
  S* t2 = t1 + M * M * P;
  const int C = blockIdx.x;
  a.col = blockIdx.y;  // one column of the batch per grid row
  const int cx = C % a.nc[0], cy = (C / a.nc[0]) % a.nc[1],
            cz = C / (a.nc[0] * a.nc[1]);
  load_embedding<T, P, DF>(E, a.dg);
  for (int i = threadIdx.x; i < M * M * M; i += blockDim.x) {
    const int fx = i % M, fy = (i / M) % M, fz = i / (M * M);
    T v;
    if (a.dg) {
      const int ox = fx / P, oy = fy / P, oz = fz / P;
      const int F = (2 * cx + ox) + a.nf[0] * ((2 * cy + oy) + a.nf[1] * (2 * cz + oz));
      const int loc = (fx % P) + P * ((fy % P) + P * (fz % P));
      v = xf[((size_t)F * P * P * P + loc) * a.stride + a.col];
    } else {
      // a fine node on a coarse-cell face is counted by its owner only
      const bool own = (fx < 2 * K || cx == a.nc[0] - 1) &&
                       (fy < 2 * K || cy == a.nc[1] - 1) &&
                       (fz < 2 * K || cz == a.nc[2] - 1);
      const int X = 2 * K * cx + fx, Y = 2 * K * cy + fy, Z = 2 * K * cz + fz;
      v = (!own || bc_con(a.bcf, X, Y, Z))
              ? T(0)
              : xf[((size_t)X + (size_t)a.gf[0] * (Y + (size_t)a.gf[1] * Z)) *
                       a.stride +
                   a.col];
    }
    u[i] = A::load(v);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < M * M * P; i += blockDim.x) {  // x
    const int ix = i % P, r = i / P;                            // r = fy + M fz
    auto s = A::zero();
    for (int f = 0; f < M; ++f) A::mac(s, E[f * P + ix], u[r * M + f]);
    t1[i] = A::get(s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < M * P * P; i += blockDim.x) {  // y
    const int ix = i % P, iy = (i / P) % P, fz = i / (P * P);
    auto s = A::zero();
    for (int f = 0; f < M; ++f)
      A::mac(s, E[f * P + iy], t1[(f + M * fz) * P + ix]);
    t2[i] = A::get(s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P * P * P; i += blockDim.x) {  // z
    const int ix = i % P, iy = (i / P) % P, iz = i / (P * P);
    auto acc = A::zero();
    for (int f = 0; f < M; ++f)
      A::mac(acc, E[f * P + iz], t2[(f * P + iy) * P + ix]);
    const T s = A::out(acc);
    if (a.dg) {
      xc[((size_t)C * P * P * P + i) * a.stride + a.col] = s;
    } else {
      const int X = cx * K + ix, Y = cy * K + iy, Z = cz * K + iz;
      if (!bc_con(a.bcc, X, Y, Z))
        atomicAdd(xc + ((size_t)X + (size_t)a.gc[0] * (Y + (size_t)a.gc[1] * Z)) *
                           a.stride +
                      a.col,
                  s);
    }
  }
}

// ---------------------------------------------------------------------------
// Reductions: per-column sums over interleaved [n][R] vectors.  Thread t of a
// block handles column t % R; the block's per-column sums go to part[], and
// the last block to finish adds them in block order (deterministic) and
// applies the finishing operation on device scalars.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool last_block(unsigned* cnt) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

__device__ void column_sums(double v, int R, double* part, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  const int groups = blockDim.x / R;
  if (threadIdx.x < R) {
    double s = 0;
    for (int g = 0; g < groups; ++g) s += sh[threadIdx.x + g * R];
    part[blockIdx.x * R + threadIdx.x] = s;
  }
}

// Sum over the grid's blocks of the partials of each column, by the whole
// last block: thread (c, g) adds the partials g, g + groups, ... in order,
// then a fixed pairwise tree over g; the result is valid for threadIdx.x < R.
__device__ double finish_sum(int R, const double* part, double* sh) {
  const int groups = blockDim.x / R;
  const int c = threadIdx.x % R, g = threadIdx.x / R;
  double s = 0;
  if (g < groups)
    for (int b = g; b < (int)gridDim.x; b += groups) s += part[b * R + c];
  __syncthreads();
  sh[threadIdx.x] = g < groups ? s : 0.0;
  __syncthreads();
  for (int w = 1; w < groups; w *= 2) {
    if (g < groups && g % (2 * w) == 0 && g + w < groups)
      sh[threadIdx.x] += sh[threadIdx.x + w * R];
    __syncthreads();
  }
  return sh[c];
}

// dot(a, b) per column and finishing operation on the slot-major scalars
// st(slot) = scal[slot * R + column]:
//   op 0: rz = rz0 = dot
//   op 1: alpha = rz / dot while the column is active (else 0; dot <= 0 or
//         a stopped column gives 0 and stops it); history records alpha
//   op 2: beta = dot / rz, rz = dot; with history: record beta, count the
//         iteration and stop on (r, z) <= 1e-30 (r0, z0)
//   op 3: bn2 = dot
__global__ void k_dot(const double* __restrict__ a,
                      const double* __restrict__ b, int64_t n, int R,
                      double* part, unsigned* cnt, double* scal, int op,
                      double* hist, int hidx) {
  __shared__ double sh[kVecThreads];
  const int groups = blockDim.x / R;
  const int c = threadIdx.x % R, g = threadIdx.x / R;
  double v = 0;
  if (g < groups)
    for (int64_t row = (int64_t)blockIdx.x * groups + g; row < n;
         row += (int64_t)gridDim.x * groups)
      v += a[row * R + c] * b[row * R + c];
  column_sums(g < groups ? v : 0.0, R, part, sh);
  if (!last_block(cnt)) return;
  const double s = finish_sum(R, part, sh);
  if (threadIdx.x < R) {
    const int cc = threadIdx.x;
#define ST(slot) scal[(slot) * R + cc]
    switch (op) {
      case 0:
        ST(S_RZ) = s;
        ST(S_RZ0) = s;
        break;
      case 1: {
        const bool go = ST(S_ACTIVE) != 0.0 && s > 0.0 && ST(S_STOP) == 0.0;
        ST(S_ALPHA) = go ? ST(S_RZ) / s : 0.0;
        if (!go && hist) ST(S_STOP) = 1.0;
        if (hist && go) hist[2 * hidx] = ST(S_ALPHA);
        break;
      }
      case 2: {
        if (ST(S_STOP) != 0.0) break;
        const double beta = ST(S_RZ) != 0.0 ? s / ST(S_RZ) : 0.0;
        ST(S_BETA) = beta;
        ST(S_RZ) = s;
        if (hist) {
          hist[2 * hidx + 1] = beta;
          ST(S_COUNT_IT) = hidx + 1;
          if (s <= 1e-30 * ST(S_RZ0)) ST(S_STOP) = 1.0;
        }
        break;
      }
      default:
        ST(S_BN2) = s;
    }
#undef ST
  }
  if (threadIdx.x == 0) *cnt = 0u;
}

// x += alpha p; r -= alpha Ap; rn2 = |r|^2 per column.
__global__ void k_cg_update(double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p,
                            const double* __restrict__ ap, int64_t n, int R,
                            double* part, unsigned* cnt, double* scal) {
  __shared__ double sh[kVecThreads];
  const int groups = blockDim.x / R;
  const int c = threadIdx.x % R, g = threadIdx.x / R;
  double v = 0;
  if (g < groups) {
    const double al = scal[S_ALPHA * R + c];
    for (int64_t row = (int64_t)blockIdx.x * groups + g; row < n;
         row += (int64_t)gridDim.x * groups) {
      const int64_t i = row * R + c;
      if (x) x[i] += al * p[i];
      const double ri = r[i] - al * ap[i];
      r[i] = ri;
      v += ri * ri;
    }
  }
  column_sums(g < groups ? v : 0.0, R, part, sh);
  if (!last_block(cnt)) return;
  const double s = finish_sum(R, part, sh);
  if (threadIdx.x < R) scal[S_RN2 * R + threadIdx.x] = s;
  if (threadIdx.x == 0) *cnt = 0u;
}

// p = z + beta p per column (beta = 0 for inactive columns keeps p = z).
__global__ void k_cg_p(double* __restrict__ p, const double* __restrict__ z,
                       int64_t n, int R, const double* scal) {
  GRID_STRIDE(i, n * R) {
    const int c = (int)(i % R);
    p[i] = z[i] + scal[S_BETA * R + c] * p[i];
  }
}

// Start vector of the eigenvalue estimate: 1 + 0.1 sin(i), 0 on constrained
// dofs.
__global__ void k_start_vector(double* v, int64_t n, int g0, int g1, Bc bc,
                               int cg) {
  GRID_STRIDE(i, n) {
    bool con = false;
    if (cg) {
      const int64_t ix = i % g0, iy = (i / g0) % g1,
                    iz = i / ((int64_t)g0 * g1);
      con = bc_con(bc, ix, iy, iz);
    }
    v[i] = con ? 0.0 : 1.0 + 0.1 * sin((double)i);
  }
}

__global__ void k_jacobi(const double* __restrict__ r,
                         const double* __restrict__ dinv,
                         double* __restrict__ z, int64_t n, int R) {
  GRID_STRIDE(i, n * R) z[i] = dinv[i / R] * r[i];
}

// Extreme eigenvalues of the Lanczos tridiagonal built from CG coefficients
// (diag_j = 1/alpha_j + beta_{j-1}/alpha_{j-1}, off_j = sqrt(beta_j)/alpha_j)
// by Sturm-sequence bisection; single thread.
__device__ int sturm_count(const double* dg, const double* of, int m,
                           double x) {
  int cnt = 0;
  double q = 1.0;
  for (int j = 0; j < m; ++j) {
    q = dg[j] - x - (j ? of[j - 1] * of[j - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0) ++cnt;
  }
  return cnt;
}

__global__ void k_lanczos(const double* hist, const double* scal,
                          double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int m = (int)scal[S_COUNT_IT];
  if (m > 64) m = 64;
  if (m < 1) {  // no free dofs: any positive interval is harmless
    out[0] = out[1] = 1.0;
    return;
  }
  double dg[64], of[64];
  for (int j = 0; j < m; ++j) {
    const double al = hist[2 * j], be = hist[2 * j + 1];
    dg[j] = 1.0 / al + (j ? hist[2 * j - 1] / hist[2 * j - 2] : 0.0);
    of[j] = sqrt(be) / al;
  }
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < m; ++j) {
    double r = (j ? fabs(of[j - 1]) : 0.0) + (j < m - 1 ? fabs(of[j]) : 0.0);
    lo = fmin(lo, dg[j] - r);
    hi = fmax(hi, dg[j] + r);
  }
  for (int which = 0; which < 2; ++which) {
    double a = lo, b = hi;
    const int target = which == 0 ? m - 1 : 0;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a + b);
      if (sturm_count(dg, of, m, mid) > target)
        b = mid;
      else
        a = mid;
      if (b - a <= 1e-12 * fmax(fabs(a), fabs(b))) break;
    }
    out[which] = 0.5 * (a + b);  // 0: max, 1: min
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
void launch_fill(T* x, T v, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<T><<<vec_grid(n), kVecThreads, 0, s>>>(x, v, n);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
template void launch_fill<double>(double*, double, int64_t, cudaStream_t);
template void launch_fill<float>(float*, float, int64_t, cudaStream_t);

void launch_invert_diag(const Level& L, double* diag, cudaStream_t s) {
  k_invert_diag<<<vec_grid(L.ndofs), kVecThreads, 0, s>>>(
      diag, L.ndofs, L.gdim[0], L.gdim[1], L.bc, L.disc == MFP_CG);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}

void launch_to_float(const double* a, float* b, int64_t n, cudaStream_t s) {
  k_to_float<<<vec_grid(n), kVecThreads, 0, s>>>(a, b, n);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
void launch_split(const double* a, float* hi, float* lo, int64_t n,
                  cudaStream_t s) {
  if (n <= 0) return;
  k_split<<<vec_grid(n), kVecThreads, 0, s>>>(a, hi, lo, n);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
void launch_to_double(const float* a, double* b, int64_t n, cudaStream_t s) {
  k_to_double<<<vec_grid(n), kVecThreads, 0, s>>>(a, b, n);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}

template <typename T>
void launch_cheb_first(const T* b, const T* dinv, T* d, T* x, const T* ax,
                       double c, int64_t n, int nrhs, cudaStream_t s) {
  k_cheb_first<T><<<vec_grid(n * nrhs), kVecThreads, 0, s>>>(b, dinv, d, x,
                                                              ax, (T)c, n,
                                                              nrhs);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
template <typename T>
void launch_cheb_step(const T* b, const T* dinv, T* d, T* x, const T* ax,
                      double cd, double cr, int64_t n, int nrhs,
                      cudaStream_t s) {
  k_cheb_step<T><<<vec_grid(n * nrhs), kVecThreads, 0, s>>>(
      b, dinv, d, x, ax, (T)cd, (T)cr, n, nrhs);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
template <typename T>
void launch_residual(const T* b, const T* ax, T* r, int64_t n,
                     cudaStream_t s) {
  k_residual<T><<<vec_grid(n), kVecThreads, 0, s>>>(b, ax, r, n);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
template <typename T>
void launch_axpy(T* y, const T* x, double a, int64_t n, cudaStream_t s) {
  k_axpy<T><<<vec_grid(n), kVecThreads, 0, s>>>(y, x, (T)a, n);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
#define INST_VEC(T)                                                           \
  template void launch_cheb_first<T>(const T*, const T*, T*, T*, const T*,   \
                                     double, int64_t, int, cudaStream_t);     \
  template void launch_cheb_step<T>(const T*, const T*, T*, T*, const T*,    \
                                    double, double, int64_t, int,            \
                                    cudaStream_t);                            \
  template void launch_residual<T>(const T*, const T*, T*, int64_t,          \
                                   cudaStream_t);                             \
  template void launch_axpy<T>(T*, const T*, double, int64_t, cudaStream_t);
INST_VEC(double)
INST_VEC(float)

static XferArgs xfer_args(const Level& fine, const Level& coarse, int stride,
                          int col) {
  XferArgs a;
  for (int d = 0; d < 3; ++d) {
    a.nc[d] = coarse.n[d];
    a.gc[d] = coarse.gdim[d];
    a.gf[d] = fine.gdim[d];
    a.nf[d] = fine.n[d];
  }
  a.bcc = coarse.bc;
  a.bcf = fine.bc;
  a.dg = fine.disc == MFP_SIPG;
  a.stride = stride;
  a.col = col;
  return a;
}

template <typename T>
void launch_prolongate(const Level& fine, const Level& coarse, const T* xc,
                       T* xf, int stride, int col, cudaStream_t s) {
  ensure_tables();
  XferArgs a = xfer_args(fine, coarse, stride, col);
  dispatch_p(fine.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    const int M = a.dg ? 2 * P : 2 * P - 1;
    const size_t smem = (size_t)(M * P + P * P * P + P * P * M + P * M * M) *
                        sizeof(T);
    auto kern = std::is_same<T, double>::value && fine.df_arith
                    ? k_prolongate<T, P, std::is_same<T, double>::value>
                    : k_prolongate<T, P, false>;
    if (smem > 48 * 1024)
      MFP_CHECK_CUDA(cudaFuncSetAttribute(
          kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<dim3((unsigned)coarse.ncells, (unsigned)stride), 256, smem, s>>>(a, xc, xf);
  });
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
template <typename T>
void launch_restrict(const Level& fine, const Level& coarse, const T* xf,
                     T* xc, int stride, int col, cudaStream_t s) {
  ensure_tables();
  XferArgs a = xfer_args(fine, coarse, stride, col);
  if (fine.disc == MFP_CG)
    MFP_CHECK_CUDA(cudaMemsetAsync(
        xc, 0, (size_t)coarse.ndofs * stride * sizeof(T), s));
  dispatch_p(fine.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    const int M = a.dg ? 2 * P : 2 * P - 1;
    const size_t smem = (size_t)(M * P + M * M * M + M * M * P + M * P * P) *
                        sizeof(T);
    auto kern = std::is_same<T, double>::value && fine.df_arith
                    ? k_restrict<T, P, std::is_same<T, double>::value>
                    : k_restrict<T, P, false>;
    if (smem > 48 * 1024)
      MFP_CHECK_CUDA(cudaFuncSetAttribute(
          kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<dim3((unsigned)coarse.ncells, (unsigned)stride), 256, smem, s>>>(a, xf, xc);
  });
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
template void launch_prolongate<double>(const Level&, const Level&,
                                        const double*, double*, int, int,
                                        cudaStream_t);
template void launch_prolongate<float>(const Level&, const Level&,
                                       const float*, float*, int, int,
                                       cudaStream_t);
template void launch_restrict<double>(const Level&, const Level&,
                                      const double*, double*, int, int,
                                      cudaStream_t);
template void launch_restrict<float>(const Level&, const Level&, const float*,
                                     float*, int, int, cudaStream_t);

// reductions
static int red_grid(int64_t rows, int R) {
  const int groups = kVecThreads / R;
  int64_t b = (rows + groups - 1) / groups;
  const int64_t cap = kMaxRedBlocks;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------------------
// Dense coarse operator (coarsest level, at most kDenseMax dofs).
// ---------------------------------------------------------------------------
// e = the columns c0 .. c0+R-1 of the identity, [n][R]
__global__ void k_identity_block(double* e, int64_t n, int64_t c0, int R) {
  GRID_STRIDE(i, n * R) {
    const int64_t row = i / R;
    e[i] = row == c0 + (i - row * R) ? 1.0 : 0.0;
  }
}

// a[(c0 + r) * n + row] = y[row * R + r]  (column-major store)
__global__ void k_store_columns(const double* y, double* a, int64_t n,
                                int64_t c0, int R) {
  GRID_STRIDE(i, n * R) {
    const int64_t row = i % n, r = i / n;
    a[(c0 + r) * n + row] = y[row * R + r];
  }
}

// y = A x for column blockIdx.z of [n][R] vectors, A column-major n x n.
// Block (row block, column range ks) forms partial sums over its range; the
// last block of a row block to arrive adds the kDenseSplit partials in order
// (deterministic).
template <typename T>
__global__ void __launch_bounds__(kDenseRows)
    k_dense_apply(const T* __restrict__ A, const T* __restrict__ x,
                  T* __restrict__ y, int n, int R, double* part,
                  unsigned* cnt) {
  const int i = blockIdx.x * kDenseRows + threadIdx.x;
  const int ks = blockIdx.y, r = blockIdx.z;
  const int j0 = (int)((int64_t)n * ks / kDenseSplit);
  const int j1 = (int)((int64_t)n * (ks + 1) / kDenseSplit);
  // four independent partial sums keep several loads in flight
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  if (i < n) {
    int j = j0;
    for (; j + 3 < j1; j += 4) {
      s0 = fma(A[(size_t)j * n + i], x[(size_t)j * R + r], s0);
      s1 = fma(A[(size_t)(j + 1) * n + i], x[(size_t)(j + 1) * R + r], s1);
      s2 = fma(A[(size_t)(j + 2) * n + i], x[(size_t)(j + 2) * R + r], s2);
      s3 = fma(A[(size_t)(j + 3) * n + i], x[(size_t)(j + 3) * R + r], s3);
    }
    for (; j < j1; ++j)
      s0 = fma(A[(size_t)j * n + i], x[(size_t)j * R + r], s0);
    part[((size_t)ks * R + r) * n + i] = (double)((s0 + s1) + (s2 + s3));
  }
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    last = atomicAdd(&cnt[blockIdx.x * R + r], 1u) == kDenseSplit - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (i < n) {
    double t = 0.0;
    for (int k = 0; k < kDenseSplit; ++k)
      t += part[((size_t)k * R + r) * n + i];
    y[(size_t)i * R + r] = (T)t;
  }
  if (threadIdx.x == 0) cnt[blockIdx.x * R + r] = 0u;
}

void launch_identity_block(double* e, int64_t n, int64_t c0, int R,
                           cudaStream_t s) {
  k_identity_block<<<vec_grid(n * R), kVecThreads, 0, s>>>(e, n, c0, R);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
void launch_store_columns(const double* y, double* a, int64_t n, int64_t c0,
                          int R, cudaStream_t s) {
  k_store_columns<<<vec_grid(n * R), kVecThreads, 0, s>>>(y, a, n, c0, R);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
template <typename T>
void launch_dense_apply(const T* A, const T* x, T* y, int n, int R,
                        double* part, unsigned* cnt, cudaStream_t s) {
  MFP_REQUIRE(n <= kDenseMax && R >= 1 && R <= kMaxRhs,
              "dense coarse apply: size out of range");
  const dim3 grid((n + kDenseRows - 1) / kDenseRows, kDenseSplit, R);
  k_dense_apply<T><<<grid, kDenseRows, 0, s>>>(A, x, y, n, R, part, cnt);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
template void launch_dense_apply<double>(const double*, const double*,
                                         double*, int, int, double*,
                                         unsigned*, cudaStream_t);
template void launch_dense_apply<float>(const float*, const float*, float*,
                                        int, int, double*, unsigned*,
                                        cudaStream_t);

void launch_dot(const double* a, const double* b, int64_t n, int R,
                RedScratch& rs, double* scal, int op, double* hist, int hidx,
                cudaStream_t s) {
  k_dot<<<red_grid(n, R), kVecThreads, 0, s>>>(a, b, n, R, rs.part, rs.cnt,
                                               scal, op, hist, hidx);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
void launch_cg_update(double* x, double* r, const double* p, const double* ap,
                      int64_t n, int R, RedScratch& rs, double* scal,
                      cudaStream_t s) {
  k_cg_update<<<red_grid(n, R), kVecThreads, 0, s>>>(x, r, p, ap, n, R,
                                                     rs.part, rs.cnt, scal);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
void launch_cg_p(double* p, const double* z, int64_t n, int R,
                 const double* scal, cudaStream_t s) {
  k_cg_p<<<vec_grid(n * R), kVecThreads, 0, s>>>(p, z, n, R, scal);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
void launch_start_vector(const Level& L, double* v, cudaStream_t s) {
  k_start_vector<<<vec_grid(L.ndofs), kVecThreads, 0, s>>>(
      v, L.ndofs, L.gdim[0], L.gdim[1], L.bc, L.disc == MFP_CG);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
void launch_jacobi(const double* r, const double* dinv, double* z, int64_t n,
                   int R, cudaStream_t s) {
  k_jacobi<<<vec_grid(n * R), kVecThreads, 0, s>>>(r, dinv, z, n, R);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}
void launch_lanczos(const double* hist, const double* scal, double* out,
                    cudaStream_t s) {
  k_lanczos<<<1, 32, 0, s>>>(hist, scal, out);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}

}  // namespace mfp
