// Matrix-free operator evaluation by sum factorization (Sec. 3, Eq. 12) for
// continuous Q_k (Eq. 4) and SIPG (Eq. 6, boundary extension Eq. 7).
//
// Mapping: a thread block owns `cpb` cells; each cell is worked on by p*p
// threads.  In every 1D sweep a thread owns one line of p values along the
// sweep direction and keeps it in registers, so each sweep is p^2 FMAs per
// thread with the 1D matrix as constant-bank operands; lines change
// direction through shared memory.  Per cell:
//   gather -> S (z, y, x) -> collocation derivative D (x, y, z) at the Gauss
//   points -> t_q = G_q grad u_q (kappa, w, det J, J^{-1} J^{-T}) ->
//   D^T (z, y, x) -> S^T (x, y, z) -> scatter.
// CG scatters with atomics into the node grid (boundary rows are identity);
// SIPG adds the face integrals at the Gauss points before the S^T sweeps:
// the cell below each interior face evaluates it for both sides and leaves
// the upper neighbour's share in a face buffer that k_dg_face_add_t adds.
#pragma once

#include <map>

#include "bulk_copy.cuh"
#include "dev_tables.cuh"

namespace mfp {
namespace {

template <typename T>
struct ApplyArgs {
  const T* __restrict__ src;
  T* __restrict__ dst;
  int n[3];
  int ncells;
  int g[3];          // CG node grid
  int blo[3], bhi[3];  // CG: constrained node coordinates per axis (-1: none)
  int neumann;         // SIPG: bit 2d + s = Neumann side (no face terms)
  int face_off[3];
  const T* __restrict__ G;      // curved: [cell][6][p^3]
  const T* __restrict__ kcell;  // [cell][p^3] or null
  const T* __restrict__ kface;  // [face][p^2] or null
  const T* __restrict__ fdata;  // curved SIPG: [face][7][p^2]
  const T* __restrict__ sigma;  // curved SIPG: [face]
  T* fb;                        // SIPG face buffer [cell][6][p^2] x columns
  T kappa;
  T gs[3];  // Cartesian: |K| / h_d^2
  T ns[3];  // Cartesian: 1 / h_d
  T fa[3];  // Cartesian: face area of a d-face
  T sg[3];  // Cartesian: penalty of a d-face
  int stride;  // batched layout: value i of column r at [i*stride + r]
  int col;     // first column of this launch
  int cpb;     // cells per block
  int ncols;   // columns per block
  int cs;      // shared-memory stride of a virtual cell (pick_cell_stride)
  Epi<T> epi;  // SIPG: update fused into k_dg_face_add_t
  int* err;    // set to 1 by a staged kernel whose copy wait timed out
};

template <int P>
__device__ __forceinline__ int idx3(int x, int y, int z) {
  return x + P * (y + P * z);
}

// Shared-memory layout of a virtual cell.  Its arrays of p^3 values are
// indexed x + p y + zs z, with the z stride padded (lay_zs) so that the
// lines of all three sweep directions spread over the 32 banks; a cell holds
// Aq, GX, GY (SIPG also U) at multiples of the array size lay_arr, and the
// virtual cells of a block follow each other at a cell stride chosen per
// launch shape (pick_cell_stride).  The SIPG face scratch (pairs of face
// arrays, face_gp) lies in a region of its own after the cells and tables.
template <int P>
__host__ __device__ constexpr int lay_zs() {
  return P == 2 ? 5 : P == 3 ? 11 : P == 4 ? 19 : P == 5 ? 29
       : P == 6 ? 37 : P == 7 ? 53 : P == 8 ? 65 : 85;
}
template <int P>
__host__ __device__ constexpr int lay_arr() {
  return (P - 1) * (1 + P + lay_zs<P>()) + 1;
}
template <int P>
__host__ __device__ constexpr int sidx(int x, int y, int z) {
  return x + P * y + lay_zs<P>() * z;
}
template <int P, bool DG>
__host__ __device__ constexpr int cell_min_elems() {
  return (DG ? 4 : 3) * lay_arr<P>();
}
template <int P>
__host__ __device__ constexpr int table_smem_elems() {
  return 3 * P * P + 3 * P;
}

// Shared-memory wavefronts above one per warp access that a launch shape
// (cpb cells x nc columns per block, p^2 threads per virtual cell, columns
// adjacent) would cost at cell stride cs: the z-lines, one per thread in
// thread order, plus the y- and x-lines that the greedy assignment of
// assign_line cannot give a bank of their own.
template <int P>
int layout_conflicts(int cpb, int nc, int cs) {
  constexpr int P2 = P * P, ZS = lay_zs<P>();
  const int items = cpb * nc * P2, nthr = (items + 31) / 32 * 32,
            nw = nthr / 32;
  int cost = 0;
  for (int w = 0; w < nw; ++w) {  // z-lines: distinct starts per bank
    int addr[32], n = 0;
    for (int l = 0; l < 32; ++l) {
      const int t = w * 32 + l;
      if (t >= items) break;
      const int rest = t / nc, rr = t % nc, m = rest % P2;
      addr[n++] = ((rest / P2) * nc + rr) * cs + m % P + P * (m / P);
    }
    int worst = 0;
    for (int b = 0; b < 32; ++b) {
      int cnt = 0;
      for (int i = 0; i < n; ++i) {
        if ((addr[i] & 31) != b) continue;
        bool dup = false;
        for (int j = 0; j < i; ++j) dup |= addr[j] == addr[i];
        cnt += !dup;
      }
      worst = cnt > worst ? cnt : worst;
    }
    cost += worst > 1 ? (worst - 1) * 32 : 0;
  }
  for (int mode = 0; mode < 2; ++mode) {  // y-, x-lines: per bank <= nw
    int cnt[32] = {0};
    for (int v = 0; v < cpb * nc; ++v)
      for (int m = 0; m < P2; ++m) {
        const int a = m % P, b = m / P;
        ++cnt[(v * cs + (mode == 0 ? a + ZS * b : P * a + ZS * b)) & 31];
      }
    for (int b = 0; b < 32; ++b) cost += cnt[b] > nw ? cnt[b] - nw : 0;
  }
  return cost;
}

// Cell stride of a launch shape: of the 32 strides from the cell's size up,
// the one with the fewest bank conflicts (cached per shape).
template <int P, bool DG>
int pick_cell_stride(int cpb, int nc) {
  static std::mutex mu;
  static std::map<long long, int> cache;
  const long long key = (long long)cpb * 4096 + nc;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const int base = cell_min_elems<P, DG>();
  int best = base, best_cost = -1;
  for (int cs = base; cs < base + 32; ++cs) {
    const int c = layout_conflicts<P>(cpb, nc, cs);
    if (best_cost < 0 || c < best_cost) {
      best = cs;
      best_cost = c;
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = best;
  return best;
}

// Greedy assignment of the block's lines of one sweep direction (mode 0:
// y-lines, start x + zs z; mode 1: x-lines, start p y + zs z, for every
// virtual cell) to its threads, so that the lanes of a warp read and write
// distinct banks: the k-th line whose start falls into bank r goes to lane r
// of warp k, the lines left over (more than one per warp in a bank) to the
// threads still without one.  Returns the shared-memory offset of the
// thread's line start, or -1 for none.  scr: 34 + 2 blockDim.x ints of
// scratch; every thread of the block calls it.
template <int P>
__device__ int assign_line(int* scr, int nv, int cs, int mode) {
  constexpr int P2 = P * P, ZS = lay_zs<P>();
  const int nthr = blockDim.x, tid = threadIdx.x, nw = nthr >> 5;
  int* cnt = scr;
  int* tab = scr + 34;
  int* ovf = tab + nthr;
  for (int i = tid; i < 34; i += nthr) scr[i] = 0;
  tab[tid] = -1;
  __syncthreads();
  for (int i = tid; i < nv * P2; i += nthr) {
    const int v = i / P2, m = i - v * P2;
    const int a = m % P, b = m / P;
    const int st = v * cs + (mode == 0 ? a + ZS * b : P * a + ZS * b);
    const int r = st & 31;
    const int k = atomicAdd(&cnt[r], 1);
    if (k < nw)
      tab[(k << 5) + r] = st;
    else
      ovf[atomicAdd(&scr[32], 1)] = st;
  }
  __syncthreads();
  int my = tab[tid];
  if (my < 0) {
    const int j = atomicAdd(&scr[33], 1);
    if (j < scr[32]) my = ovf[j];
  }
  __syncthreads();
  return my;
}

// One face of the own cell (axis D a runtime value), SIPG (Eq. 6, mirror
// states Eq. 7).  The own side works on the cell's values at its Gauss
// points U: its trace and reference normal slope at face point (ta, tb)
// come from the line of U along D through it (Lagrange basis of the Gauss
// points at the cell end, exact for the degree-k polynomial), and its test
// terms go back onto the same line of the Gauss-point accumulator Aq ahead
// of the cell's S^T sweeps.  Each interior face is evaluated once, by the
// cell below it (S = 1): the upper neighbour's trace comes from its nodal
// values (face layer and normal slope, then S x S to the face points, one
// point per thread with the table rows in registers), and its test terms
// go through S^T x S^T to its face nodes and into the face buffer fb (slot
// 2D: value part, 2D + 1: normal-slope part) for k_dg_face_add_t.  A
// boundary face is one-sided; an interior lower face (S = 0) adds nothing.
// The face scratch FS holds pairs of face arrays (two fields that the same
// sweep takes, read by one 64-bit access): Q0 nodal (vn, dnn), then (vn,
// c0n) of the neighbour's test terms; Q1 the sweeps' temporary; Q2 (uo,
// un) for the tangential slopes; Q3, Q4 the tangential test-slope factors
// (own, neighbour) along a and b.
template <typename T>
struct PairOf {
  using type = float2;
};
template <>
struct PairOf<double> {
  using type = double2;
};
template <typename T>
using pair_t = typename PairOf<T>::type;
template <typename T>
__device__ __forceinline__ pair_t<T> mkpair(T x, T y) {
  pair_t<T> r;
  r.x = x;
  r.y = y;
  return r;
}
constexpr int kFacePairs = 5;

template <int P, typename T, bool CURVED, int S>
__device__ __forceinline__ void face_gp(const ApplyArgs<T>& a, int col, int D,
                                        bool active, int cx, int cy, int cz,
                                        const T* U, T* Aq, pair_t<T>* FS,
                                        const T* sS, const T* sD, const T* sw,
                                        int ta, int tb) {
  constexpr int P2 = P * P, P3 = P2 * P;
  pair_t<T>* Q0 = FS;
  pair_t<T>* Q1 = FS + P2;
  pair_t<T>* Q2 = FS + 2 * P2;
  pair_t<T>* Q3 = FS + 3 * P2;
  pair_t<T>* Q4 = FS + 4 * P2;
  constexpr int GV = S ? T_GV1 : T_GV0;
  constexpr int GD = S ? T_GD1 : T_GD0;
  const int t = ta + P * tb;
  // point (l, ta, tb) of the own line normal to D: n0 + l * ls in the nodal
  // vectors, s0 + l * ss in the shared arrays
  constexpr int ZS = lay_zs<P>();
  const int ls = D == 0 ? 1 : (D == 1 ? P : P2);
  const int n0 = D == 0 ? P * t : (D == 1 ? ta + P2 * tb : t);
  const int ss = D == 0 ? 1 : (D == 1 ? P : ZS);
  const int s0 = D == 0 ? P * ta + ZS * tb : (D == 1 ? ta + ZS * tb : t);
  const int cD = D == 0 ? cx : (D == 1 ? cy : cz);
  const int f = a.face_off[D] + cx + (D == 0 ? S : 0) +
                (a.n[0] + (D == 0)) *
                    (cy + (D == 1 ? S : 0) +
                     (a.n[1] + (D == 1)) * (cz + (D == 2 ? S : 0)));
  const bool bnd = S ? cD + 1 >= a.n[D] : cD == 0;
  // a boundary face on a Neumann side has no operator terms
  const bool own =
      (S == 1 || bnd) && !(bnd && ((a.neumann >> (2 * D + S)) & 1));
  const bool pair = S == 1 && !bnd && active;
  const int nb = pair ? cx + a.n[0] * (cy + a.n[1] * cz) +
                            (D == 0 ? 1 : (D == 1 ? a.n[0] : a.n[0] * a.n[1]))
                      : 0;
  // own trace and reference normal slope at the face point (ta, tb)
  T uo = T(0), so = T(0);
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const T u = U[s0 + l * ss];
    uo = fma(tv<T, P, GV>(l), u, uo);
    so = fma(tv<T, P, GD>(l), u, so);
  }
  if constexpr (CURVED) Q2[t].x = uo;
  T un = T(0), q3 = T(0);
  if constexpr (S == 1) {
    // the upper neighbour's face layer and normal slope (nodal), then
    // interpolated to the face points
    T vn = T(0), dnn = T(0);
    if (pair) {
      const T* u0 = a.src + ((size_t)nb * P3 + n0) * a.stride + col;
      const size_t lstr = (size_t)ls * a.stride;
#pragma unroll
      for (int l = 0; l < P; ++l) {
        const T u = u0[l * lstr];
        dnn = fma(tv<T, P, T_DPHI0>(l), u, dnn);
        if (l == 0) vn = u;
      }
    }
    Q0[t] = mkpair(vn, dnn);
    __syncthreads();
    T ra[P];
#pragma unroll
    for (int j = 0; j < P; ++j) ra[j] = sS[ta * P + j];
    T s2 = T(0), s3 = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const pair_t<T> q = Q0[j + P * tb];
      s2 = fma(ra[j], q.x, s2);
      s3 = fma(ra[j], q.y, s3);
    }
    Q1[t] = mkpair(s2, s3);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) ra[j] = sS[tb * P + j];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const pair_t<T> q = Q1[ta + P * j];
      un = fma(ra[j], q.x, un);
      q3 = fma(ra[j], q.y, q3);
    }
    if constexpr (CURVED) Q2[t].y = un;
  }
  if constexpr (CURVED) __syncthreads();
  // flux at the face quadrature point (ta, tb)
  T cv, c0o, c0n;
  {
    const T kap = a.kface ? a.kface[(size_t)f * P2 + t] : a.kappa;
    T dno, dnn, dA, sig, go1 = T(0), go2 = T(0), gn1 = T(0), gn2 = T(0), gvD,
                              gnD;
    if constexpr (!CURVED) {
      const T nsc = (S ? T(1) : T(-1)) * a.ns[D];
      dA = sw[ta] * sw[tb] * a.fa[D];
      sig = a.sg[D];
      dno = nsc * so;
      dnn = bnd ? dno : nsc * q3;
      gvD = nsc;
      gnD = nsc;
    } else {
      const int T1 = D == 0 ? 1 : 0;
      const int T2 = D == 2 ? 1 : 2;
      const T* fd = a.fdata + (size_t)f * 7 * P2 + t;
      dA = fd[0];
      sig = a.sigma[f];
      T t1o = T(0), t2o = T(0), t1n = T(0), t2n = T(0);
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const pair_t<T> qa = Q2[j + P * tb], qb = Q2[ta + P * j];
        t1o = fma(sD[ta * P + j], qa.x, t1o);
        t2o = fma(sD[tb * P + j], qb.x, t2o);
        if constexpr (S == 1) {
          t1n = fma(sD[ta * P + j], qa.y, t1n);
          t2n = fma(sD[tb * P + j], qb.y, t2n);
        }
      }
      // J^-1 n of the lower (L) and upper (R) cell, face-local components
      const T RD = fd[(4 + D) * P2], R1 = fd[(4 + T1) * P2],
              R2 = fd[(4 + T2) * P2];
      if constexpr (S == 1) {  // own cell is the lower one: outward = +n
        const T LD = fd[(1 + D) * P2], L1 = fd[(1 + T1) * P2],
                L2 = fd[(1 + T2) * P2];
        dno = LD * so + L1 * t1o + L2 * t2o;
        dnn = bnd ? dno : RD * q3 + R1 * t1n + R2 * t2n;
        gvD = LD;
        go1 = L1;
        go2 = L2;
        gnD = RD;
        gn1 = R1;
        gn2 = R2;
      } else {  // own cell is the upper one (boundary only): outward = -n
        dno = -(RD * so + R1 * t1o + R2 * t2o);
        dnn = dno;
        gvD = -RD;
        go1 = -R1;
        go2 = -R2;
        gnD = gvD;
      }
    }
    if (bnd) un = -uo;  // mirror state u+ = -u-, grad u+ = grad u- (Eq. 7)
    const T kdA = kap * dA;
    const T jump = uo - un;
    cv = kdA * (sig * jump - T(0.5) * (dno + dnn));
    const T cg = T(-0.5) * kdA * jump;
    c0o = cg * gvD;
    c0n = cg * gnD;
    if constexpr (CURVED) {
      Q3[t] = mkpair(cg * go1, S == 1 ? cg * gn1 : T(0));
      Q4[t] = mkpair(cg * go2, S == 1 ? cg * gn2 : T(0));
    }
  }
  // fold the tangential test slopes into the value parts (D^T at the face
  // points)
  T vo = cv, vn = -cv;
  if constexpr (CURVED) {
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const pair_t<T> qa = Q3[j + P * tb], qb = Q4[ta + P * j];
      vo = fma(sD[j * P + ta], qa.x, vo);
      vo = fma(sD[j * P + tb], qb.x, vo);
      if constexpr (S == 1) {
        vn = fma(sD[j * P + ta], qa.y, vn);
        vn = fma(sD[j * P + tb], qb.y, vn);
      }
    }
  }
  // own test terms onto the line of Gauss points along D
  if (own) {
#pragma unroll
    for (int l = 0; l < P; ++l) {
      T& y = Aq[s0 + l * ss];
      y = fma(tv<T, P, GV>(l), vo, fma(tv<T, P, GD>(l), c0o, y));
    }
  }
  // the neighbour's test terms to its face nodes: S^T along a, then b
  if constexpr (S == 1) {
    Q0[t] = mkpair(vn, c0n);
    __syncthreads();
    T ra[P];
#pragma unroll
    for (int j = 0; j < P; ++j) ra[j] = sS[j * P + ta];
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const pair_t<T> q = Q0[j + P * tb];
      s0 = fma(ra[j], q.x, s0);
      s1 = fma(ra[j], q.y, s1);
    }
    Q1[t] = mkpair(s0, s1);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) ra[j] = sS[j * P + tb];
    T r0 = T(0), r1 = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const pair_t<T> q = Q1[ta + P * j];
      r0 = fma(ra[j], q.x, r0);
      r1 = fma(ra[j], q.y, r1);
    }
    if (pair) {
      T* fbn = a.fb + ((size_t)nb * 6 + 2 * D) * P2 * a.stride + col;
      fbn[(size_t)t * a.stride] = r0;
      fbn[(size_t)(P2 + t) * a.stride] = r1;
    }
  }
}

template <int P, typename T, bool CURVED>
__device__ __noinline__ void face_lower_gp(const ApplyArgs<T>& a, int col,
                                           int D, bool active, int cx, int cy,
                                           int cz, const T* U, T* Aq,
                                           pair_t<T>* FS,
                                           const T* sS, const T* sD,
                                           const T* sw, int ta, int tb) {
  face_gp<P, T, CURVED, 0>(a, col, D, active, cx, cy, cz, U, Aq, FS, sS, sD,
                           sw, ta, tb);
  __syncthreads();
}

// Adds the terms that the cell below each interior face left for the cell
// above it (face buffer slots 2D: value part on the face layer, 2D + 1:
// normal-slope part on every layer with the weight dphi_l(0)) and applies the
// fused update; one thread per node line along z of a row of cells
// (blockIdx.y: cy, cz; blockIdx.z: column).  Float values are cheap to keep
// in registers, so a thread takes the whole line and every load of it is in
// flight at once (the double-float kernel works per node instead).
// Resident blocks of 256 threads the registers must allow: float lines take
// about 124 registers uncapped (two blocks per SM), three blocks measured 4 %
// faster at Q4 and p >= 8 would spill at three; float64 lines need twice the
// registers and stay uncapped.
template <int P, typename T>
constexpr int face_add_min_blocks() {
  return sizeof(T) == 4 ? (P <= 7 ? 3 : 2) : 1;
}
template <int P, typename T>
__global__ void __launch_bounds__(256, (face_add_min_blocks<P, T>()))
    k_dg_face_add_t(const ApplyArgs<T> a) {
  constexpr int P2 = P * P, P3 = P2 * P;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n[0] * P2) return;
  const int R = a.stride, col = blockIdx.z;
  const int cx = i / P2, xy = i - cx * P2;
  const int x = xy % P, y = xy / P;
  const int rows = a.n[1] * a.n[2];
  for (int row = blockIdx.y; row < rows; row += gridDim.y) {
    const int cy = row % a.n[1], cz = row / a.n[1];
    const size_t cell = (size_t)row * a.n[0] + cx;
    const T* fb = a.fb + cell * 6 * P2 * R + col;
    T* out = a.dst + (cell * P3 + xy) * R + col;
    T u[P], gx[P], vx[P], gy[P], vy[P];
#pragma unroll
    for (int z = 0; z < P; ++z) {
      u[z] = out[(size_t)z * P2 * R];
      gx[z] = fb[(size_t)(1 * P2 + y + P * z) * R];
      vx[z] = x == 0 ? fb[(size_t)(0 * P2 + y + P * z) * R] : T(0);
      gy[z] = fb[(size_t)(3 * P2 + x + P * z) * R];
      vy[z] = y == 0 ? fb[(size_t)(2 * P2 + x + P * z) * R] : T(0);
    }
    const T gz = fb[(size_t)(5 * P2 + xy) * R];
    const T vz = fb[(size_t)(4 * P2 + xy) * R];
    const T wx = tv<T, P, T_DPHI0>(x), wy = tv<T, P, T_DPHI0>(y);
    // the fused update's inputs, loaded with the rest
    const size_t dof = cell * P3 + xy;
    const int mode = a.epi.mode;
    T eb[P], edi[P], ed[P], ex[P];
#pragma unroll
    for (int z = 0; z < P; ++z) {
      const size_t gi = (dof + (size_t)z * P2) * R + col;
      eb[z] = mode != EPI_STORE ? a.epi.b[gi] : T(0);
      edi[z] = mode >= EPI_CHEB_FIRST ? a.epi.dinv[dof + (size_t)z * P2] : T(0);
      ex[z] = mode >= EPI_CHEB_FIRST ? a.epi.x[gi] : T(0);
      ed[z] = mode == EPI_CHEB_STEP ? a.epi.d[gi] : T(0);
    }
#pragma unroll
    for (int z = 0; z < P; ++z) {
      T s = u[z];
      if (cx > 0) s += fma(wx, gx[z], vx[z]);
      if (cy > 0) s += fma(wy, gy[z], vy[z]);
      if (cz > 0) s += fma(tv<T, P, T_DPHI0>(z), gz, z == 0 ? vz : T(0));
      epi_finish(a.epi, a.dst, (dof + (size_t)z * P2) * R + col, s, eb[z],
                 edi[z], ed[z], ex[z]);
    }
  }
}

// Stored geometry staging of the float curved kernel (STAGE): the G block of
// a group of cells ([cell][6][p^3], contiguous) arrives in shared memory by
// one bulk copy, double-buffered, so that the copy of the next group runs
// while the current one is computed.  Bytes of one buffer:
template <int P, typename T>
__host__ __device__ constexpr size_t stage_g_bytes(int cpb) {
  return (size_t)cpb * 6 * P * P * P * sizeof(T);
}
// SIPG face scratch of a virtual cell, in pairs: kFacePairs face arrays,
// the stride congruent to p^2 modulo the pairs per 128 bytes so that the
// virtual cells' scratch follows on in bank order
template <int P, typename T>
__host__ __device__ constexpr int fs_stride() {
  constexpr int m = 128 / (int)sizeof(pair_t<T>);
  int st = kFacePairs * P * P;
  while (st % m != (P * P) % m) ++st;
  return st;
}
// offset of the face scratch (16-aligned), after the cells and the tables
template <int P, typename T>
__host__ __device__ constexpr size_t fs_offset(int cpb, int ncols, int cs) {
  return (((size_t)(cpb * ncols + 1) * cs + table_smem_elems<P>()) *
              sizeof(T) + 15) / 16 * 16;
}
// bytes of the cells, tables and (SIPG) face scratch
template <int P, typename T, bool DG>
__host__ __device__ constexpr size_t cells_bytes(int cpb, int ncols, int cs) {
  return DG ? fs_offset<P, T>(cpb, ncols, cs) +
                  (size_t)(cpb * ncols + 1) * fs_stride<P, T>() *
                      sizeof(pair_t<T>)
            : ((size_t)(cpb * ncols + 1) * cs + table_smem_elems<P>()) *
                  sizeof(T);
}
// offset of the staging buffers in the dynamic shared memory (16-aligned)
template <int P, typename T, bool DG>
__host__ __device__ constexpr size_t stage_offset(int cpb, int ncols, int cs) {
  return (cells_bytes<P, T, DG>(cpb, ncols, cs) + 15) / 16 * 16;
}

// Work decomposition: a block owns `cpb` cells and `ncols` right-hand-side
// columns; each (cell, column) pair is a virtual cell worked on by p*p
// threads.  A thread owns one z-line of its virtual cell (gather, the
// quadrature-point operation, scatter); the y- and x-lines of the block's
// cells are dealt to its threads by assign_line so that the lanes of a warp
// use distinct shared-memory banks.  The block is padded to whole warps;
// padding threads work on a dummy virtual cell and write nothing to global
// memory.  Columns of one cell are adjacent threads, so batched vectors
// [N][R] are read coalesced and the geometry of a cell is loaded once per
// point for all its columns (same address across the warp).
// STAGE (float, curved, one column): the cells' stored geometry is staged
// through shared memory by bulk copies (see stage_g_bytes) instead of
// per-thread loads; a block's successive cell groups alternate between two
// buffers, each completed on its own mbarrier.
template <int P, typename T, bool DG, bool CURVED, bool STAGE = false>
__global__ void k_apply(const ApplyArgs<T> a) {
  constexpr int P2 = P * P, P3 = P2 * P, ZS = lay_zs<P>(), AR = lay_arr<P>();
  // float geometry is prefetched into registers during the gather (the float
  // apply is latency-bound) unless it is staged; float64 is bound by the
  // FP64 pipe instead
  constexpr bool PREFETCH = !STAGE && CURVED && sizeof(T) == 4 && P <= 7;
  // 32-bit values: y- and x-lines dealt by bank (64-bit accesses keep the
  // thread's own lines)
  constexpr bool DEAL = sizeof(T) == 4;
  static_assert(!STAGE || CURVED, "staging is for stored geometry");
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int cpb = a.cpb, nc = a.ncols, cs = a.cs;
  const int items = cpb * nc * P2;
  const int tid = threadIdx.x;
  const bool item_ok = tid < items;
  const int rr = tid % nc;
  const int rest = tid / nc;
  const int ta = rest % P, tb = (rest / P) % P;
  const int lc = item_ok ? rest / P2 : 0;
  const int v = item_ok ? lc * nc + rr : cpb * nc;  // dummy slot for padding
  T* base = sm + (size_t)v * cs;
  T* Aq = base;
  T* U = base + 3 * AR;   // DG: values at the Gauss points
  // DG: face scratch (face_gp)
  pair_t<T>* FS = reinterpret_cast<pair_t<T>*>(
                      smraw + fs_offset<P, T>(cpb, nc, cs)) +
                  (size_t)v * fs_stride<P, T>();
  const int own = v * cs + ta + P * tb;  // own z-line: own + ZS * z
  T* tabs = sm + (size_t)(cpb * nc + 1) * cs;
  T* sS = tabs;
  T* sD = tabs + P2;
  T* sDphi = tabs + 2 * P2;
  T* s0 = tabs + 3 * P2;
  T* s1 = s0 + P;
  T* sw = s1 + P;
  T* gbuf = nullptr;
  uint64_t* bars = nullptr;
  const int gstep = gridDim.x * cpb;
  // thread 0 copies the stored geometry of the group at cell c0 into buffer
  // slot; the last group's copy is rounded up to 16 bytes (the geometry
  // array is allocated with one spare cell)
  auto issue = [&](int c0, int slot) {
    const int cnt = a.ncells - c0 < cpb ? a.ncells - c0 : cpb;
    const uint32_t bytes =
        (uint32_t)((stage_g_bytes<P, T>(cnt) + 15) / 16 * 16);
    fence_proxy_async_smem();
    bulk_load(gbuf + (size_t)slot * cpb * 6 * P3,
              a.G + (size_t)c0 * 6 * P3, bytes, &bars[slot]);
  };
  // the thread's y-line (offset yl, step p) and x-line (xl, step 1), -1:
  // none; the assignment's scratch (apply_smem_bytes covers it) is free
  // again when it returns
  int yl, xl;
  if constexpr (DEAL) {
    int* scr = reinterpret_cast<int*>(sm);
    yl = assign_line<P>(scr, cpb * nc, cs, 0);
    xl = assign_line<P>(scr, cpb * nc, cs, 1);
  } else {
    yl = v * cs + ta + ZS * tb;
    xl = v * cs + P * ta + ZS * tb;
  }
  const bool hy = yl >= 0, hx = xl >= 0;
  if constexpr (STAGE) {
    const size_t off = stage_offset<P, T, DG>(cpb, nc, cs);
    gbuf = reinterpret_cast<T*>(smraw + off);
    bars = reinterpret_cast<uint64_t*>(smraw + off +
                                       2 * stage_g_bytes<P, T>(cpb));
    if (tid == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      mbar_init_fence();
    }
  }
  load_tables_shared<T, P>(sS, sD, sDphi, s0, s1, sw);
  __syncthreads();
  if constexpr (STAGE) {
    if (tid == 0 && blockIdx.x * cpb < a.ncells) issue(blockIdx.x * cpb, 0);
  }
  const int gx0 = a.g[0], gy0 = a.g[1];
  const int col = a.col + rr;

  int it = 0;
  for (int cbase = blockIdx.x * cpb; cbase < a.ncells;
       cbase += gstep, ++it) {
    if constexpr (STAGE) {
      // the other buffer was last read by the previous group, which ended
      // with a barrier
      if (tid == 0 && cbase + gstep < a.ncells)
        issue(cbase + gstep, (it + 1) & 1);
    }
    const int cell = cbase + lc;
    const bool active = item_ok && cell < a.ncells;
    const int cc = active ? cell : 0;
    const int cx = cc % a.n[0];
    const int cy = (cc / a.n[0]) % a.n[1];
    const int cz = cc / (a.n[0] * a.n[1]);
    T r[P], o[P];
    T gp[PREFETCH ? 6 : 1][PREFETCH ? P : 1];
    if constexpr (PREFETCH) {
#pragma unroll
      for (int qz = 0; qz < P; ++qz) {
        const T* Gp = a.G + (size_t)cc * 6 * P3 + idx3<P>(ta, tb, qz);
#pragma unroll
        for (int c = 0; c < 6; ++c) gp[c][qz] = Gp[c * P3];
      }
    }
    // ---- gather the z-line (x = ta, y = tb)
    if constexpr (DG) {
#pragma unroll
      for (int z = 0; z < P; ++z) {
        const size_t gi = (size_t)cc * P3 + idx3<P>(ta, tb, z);
        r[z] = active ? a.src[gi * a.stride + col] : T(0);
      }
    } else {
      const int X = cx * (P - 1) + ta, Y = cy * (P - 1) + tb;
      const bool bxy = X == a.blo[0] || X == a.bhi[0] || Y == a.blo[1] ||
                       Y == a.bhi[1];
#pragma unroll
      for (int z = 0; z < P; ++z) {
        const int Z = cz * (P - 1) + z;
        const bool con = bxy || Z == a.blo[2] || Z == a.bhi[2];
        const size_t gi = (size_t)X + (size_t)gx0 * (Y + (size_t)gy0 * Z);
        r[z] = (active && !con) ? a.src[gi * a.stride + col] : T(0);
      }
    }
    // ---- values at Gauss points: z (registers), y, x
    mv<T, P, T_S>(r, o);
#pragma unroll
    for (int z = 0; z < P; ++z) sm[own + ZS * z] = o[z];
    __syncthreads();
    if (hy) {
#pragma unroll
      for (int j = 0; j < P; ++j) r[j] = sm[yl + P * j];
      mv<T, P, T_S>(r, o);
#pragma unroll
      for (int j = 0; j < P; ++j) sm[yl + P * j] = o[j];
    }
    __syncthreads();
    if (hx) {
#pragma unroll
      for (int j = 0; j < P; ++j) r[j] = sm[xl + j];
      mv<T, P, T_S>(r, o);
#pragma unroll
      for (int j = 0; j < P; ++j) sm[xl + j] = o[j];
      if constexpr (DG) {  // values at the Gauss points for the face terms
#pragma unroll
        for (int j = 0; j < P; ++j) sm[xl + 3 * AR + j] = o[j];
      }
      mv<T, P, T_D>(o, r);
#pragma unroll
      for (int j = 0; j < P; ++j) sm[xl + AR + j] = r[j];  // GX
    }
    __syncthreads();
    // ---- reference gradient: y into GY, z kept in registers
    if (hy) {
#pragma unroll
      for (int j = 0; j < P; ++j) r[j] = sm[yl + P * j];
      mv<T, P, T_D>(r, o);
#pragma unroll
      for (int j = 0; j < P; ++j) sm[yl + 2 * AR + P * j] = o[j];  // GY
    }
    T gz[P];
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = sm[own + ZS * j];
    mv<T, P, T_D>(r, gz);
    __syncthreads();
    // ---- quadrature-point operation t = G_q grad u (Eq. 12)
    {
      const T* Gs = nullptr;
      if constexpr (STAGE) {
        mbar_wait(&bars[it & 1], (uint32_t)((it >> 1) & 1), a.err);
        Gs = gbuf + ((size_t)(it & 1) * cpb + lc) * 6 * P3;
      }
      const T wab = sw[ta] * sw[tb];
#pragma unroll
      for (int qz = 0; qz < P; ++qz) {
        const int q = idx3<P>(ta, tb, qz);  // in the cell's global blocks
        const int qs = own + ZS * qz;       // in shared memory
        const T ux = sm[qs + AR], uy = sm[qs + 2 * AR], uz = gz[qz];
        const T kap = a.kcell ? a.kcell[(size_t)cc * P3 + q] : a.kappa;
        T tx, ty, tz;
        if constexpr (CURVED) {
          T g0, g1, g2, g3, g4, g5;
          if constexpr (STAGE) {
            g0 = Gs[q]; g1 = Gs[P3 + q]; g2 = Gs[2 * P3 + q];
            g3 = Gs[3 * P3 + q]; g4 = Gs[4 * P3 + q]; g5 = Gs[5 * P3 + q];
          } else if constexpr (PREFETCH) {
            g0 = gp[0][qz]; g1 = gp[1][qz]; g2 = gp[2][qz];
            g3 = gp[3][qz]; g4 = gp[4][qz]; g5 = gp[5][qz];
          } else {
            const T* Gp = a.G + (size_t)cc * 6 * P3 + q;
            g0 = Gp[0]; g1 = Gp[P3]; g2 = Gp[2 * P3];
            g3 = Gp[3 * P3]; g4 = Gp[4 * P3]; g5 = Gp[5 * P3];
          }
          tx = kap * (g0 * ux + g1 * uy + g2 * uz);
          ty = kap * (g1 * ux + g3 * uy + g4 * uz);
          tz = kap * (g2 * ux + g4 * uy + g5 * uz);
        } else {
          const T wk = kap * wab * sw[qz];
          tx = wk * a.gs[0] * ux;
          ty = wk * a.gs[1] * uy;
          tz = wk * a.gs[2] * uz;
        }
        sm[qs + AR] = tx;
        sm[qs + 2 * AR] = ty;
        r[qz] = tz;
      }
      mtv<T, P, T_D>(r, o);
#pragma unroll
      for (int j = 0; j < P; ++j) sm[own + ZS * j] = o[j];
    }
    __syncthreads();
    // ---- transposed derivative y (added), x (added) then S^T x, y, z
    if (hy) {
#pragma unroll
      for (int j = 0; j < P; ++j) r[j] = sm[yl + 2 * AR + P * j];
      mtv<T, P, T_D>(r, o);
#pragma unroll
      for (int j = 0; j < P; ++j) sm[yl + P * j] += o[j];
    }
    __syncthreads();
    if (hx) {
#pragma unroll
      for (int j = 0; j < P; ++j) r[j] = sm[xl + AR + j];
      mtv<T, P, T_D>(r, o);
#pragma unroll
      for (int j = 0; j < P; ++j) o[j] += sm[xl + j];
    }
    if constexpr (DG) {
      // ---- SIPG face terms (Eq. 6, Eq. 7), added at the Gauss points
      if (hx) {
#pragma unroll
        for (int j = 0; j < P; ++j) sm[xl + j] = o[j];
      }
      __syncthreads();
#pragma unroll 1
      for (int D = 0; D < 3; ++D) {
        // lower faces only where a cell of the block lies on the boundary
        const int cD = D == 0 ? cx : (D == 1 ? cy : cz);
        if (!((a.neumann >> (2 * D)) & 1) &&
            __syncthreads_or(active && cD == 0))
          face_lower_gp<P, T, CURVED>(a, col, D, active, cx, cy, cz, U, Aq,
                                      FS, sS, sD, sw, ta, tb);
        face_gp<P, T, CURVED, 1>(a, col, D, active, cx, cy, cz, U, Aq, FS, sS,
                                 sD, sw, ta, tb);
      }
      __syncthreads();
      if (hx) {
#pragma unroll
        for (int j = 0; j < P; ++j) o[j] = sm[xl + j];
      }
    }
    if (hx) {
      mtv<T, P, T_S>(o, r);
#pragma unroll
      for (int j = 0; j < P; ++j) sm[xl + j] = r[j];
    }
    __syncthreads();
    if (hy) {
#pragma unroll
      for (int j = 0; j < P; ++j) r[j] = sm[yl + P * j];
      mtv<T, P, T_S>(r, o);
#pragma unroll
      for (int j = 0; j < P; ++j) sm[yl + P * j] = o[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = sm[own + ZS * j];
    mtv<T, P, T_S>(r, o);
    // ---- scatter
    if constexpr (!DG) {
      const int X = cx * (P - 1) + ta, Y = cy * (P - 1) + tb;
      const bool bxy = X == a.blo[0] || X == a.bhi[0] || Y == a.blo[1] ||
                       Y == a.bhi[1];
      if (active) {
#pragma unroll
        for (int z = 0; z < P; ++z) {
          const int Z = cz * (P - 1) + z;
          const bool con = bxy || Z == a.blo[2] || Z == a.bhi[2];
          const size_t gi =
              ((size_t)X + (size_t)gx0 * (Y + (size_t)gy0 * Z)) * a.stride +
              col;
          if (con)
            a.dst[gi] = a.src[gi];  // identity row (same value from all cells)
          else
            atomicAdd(a.dst + gi, o[z]);
        }
      }
      __syncthreads();
    } else {
      if (active) {
#pragma unroll
        for (int z = 0; z < P; ++z) {
          const size_t gi = (size_t)cc * P3 + idx3<P>(ta, tb, z);
          a.dst[gi * a.stride + col] = o[z];
        }
      }
      __syncthreads();
    }
  }
}

// Cells per block for one column: the block (padded to whole warps) keeps
// at least 97 % of its lanes busy: p^2 * cpb close to 128 or 256.
inline int default_cpb(int p) {
  switch (p) {
    case 2: return 32;
    case 3: return 14;
    case 4: return 8;
    case 5: return 5;
    case 6: return 7;
    case 7: return 5;
    case 8: return 4;
    default: return 3;
  }
}

template <int P, typename T, bool DG, bool STAGE = false>
size_t apply_smem_bytes(int cpb, int ncols) {
  const int cs = pick_cell_stride<P, DG>(cpb, ncols);
  size_t bytes;
  if constexpr (STAGE)
    bytes = stage_offset<P, T, DG>(cpb, ncols, cs) +
            2 * stage_g_bytes<P, T>(cpb) + 2 * sizeof(uint64_t);
  else
    bytes = cells_bytes<P, T, DG>(cpb, ncols, cs);
  // the line assignment's scratch (assign_line) at the start
  const size_t nthr = ((size_t)cpb * ncols * P * P + 31) / 32 * 32;
  const size_t scratch = (34 + 2 * nthr) * sizeof(int);
  return bytes > scratch ? bytes : scratch;
}

// Resident blocks per SM of a launch shape (cached per shape).
template <int P, typename T, bool DG, bool CURVED, bool STAGE = false>
int apply_blocks_per_sm(int cpb, int ncols) {
  static std::mutex mu;
  static int cache[64][4] = {};
  constexpr int P2 = P * P;
  const int threads = ((cpb * ncols * P2 + 31) / 32) * 32;
  const size_t smem = apply_smem_bytes<P, T, DG, STAGE>(cpb, ncols);
  const bool cacheable = ncols == 1 && cpb < 64;
  int dev = 0;
  MFP_CHECK_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(mu);
    if (cacheable && dev < 4 && cache[cpb][dev]) return cache[cpb][dev];
  }
  auto kern = k_apply<P, T, DG, CURVED, STAGE>;
  if (smem > 48 * 1024)
    MFP_CHECK_CUDA(cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MFP_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, kern, threads, smem));
  if (cacheable && dev < 4) {
    std::lock_guard<std::mutex> lk(mu);
    cache[cpb][dev] = per_sm;
  }
  return per_sm;
}

template <int P, typename T, bool DG, bool CURVED, bool STAGE = false>
void run_apply(ApplyArgs<T> a, int cpb, int ncols, cudaStream_t s) {
  constexpr int P2 = P * P;
  a.cpb = cpb;
  a.ncols = ncols;
  a.cs = pick_cell_stride<P, DG>(cpb, ncols);
  const int threads = ((cpb * ncols * P2 + 31) / 32) * 32;
  const size_t smem = apply_smem_bytes<P, T, DG, STAGE>(cpb, ncols);
  auto kern = k_apply<P, T, DG, CURVED, STAGE>;
  const int per_sm = apply_blocks_per_sm<P, T, DG, CURVED, STAGE>(cpb, ncols);
  if (smem > 48 * 1024)
    MFP_CHECK_CUDA(cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MFP_REQUIRE(per_sm >= 1,
              "apply launch shape does not fit on an SM (cells per block too "
              "large for the registers or shared memory)");
  const int64_t need = (a.ncells + cpb - 1) / cpb;
  const int64_t cap = (int64_t)per_sm * sm_count();
  const int grid = (int)(need < cap ? need : cap);
  if (grid <= 0) return;
  kern<<<grid, threads, smem, s>>>(a);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}

// Launch plan for R columns: columns per launch limited by 1024 threads per
// block; cells per block `cells_req` (0: the one-column default divided
// among the columns).
template <int P, typename T, bool DG, bool CURVED>
void run_apply_cols(const ApplyArgs<T>& a0, int R, int cells_req,
                    cudaStream_t s) {
  constexpr int P2 = P * P;
  // block size limit of this kernel given its registers
  cudaFuncAttributes fa;
  MFP_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_apply<P, T, DG, CURVED>));
  const int maxthr = fa.maxThreadsPerBlock > 0 ? fa.maxThreadsPerBlock : 1024;
  const int maxcols = maxthr / P2 > 0 ? maxthr / P2 : 1;
  for (int c0 = 0; c0 < R; c0 += maxcols) {
    const int nc = R - c0 < maxcols ? R - c0 : maxcols;
    // float curved geometry staged by bulk copies (one column, an even
    // number of cells per block, so that every group's block of it starts on
    // a 16-byte boundary); the autotuner's choice of cells per block decides
    // between the variants (at 32^3 Q4 the default, odd shape with the
    // register prefetch measured 7 % faster)
    constexpr bool can_stage = CURVED && sizeof(T) == 4;
    int cells = cells_req > 0 ? cells_req : default_cpb(P) / nc;
    if (cells < 1) cells = 1;
    while (cells > 1 && cells * nc * P2 > maxthr) --cells;
    ApplyArgs<T> a = a0;
    a.col = c0;
    if (can_stage && nc == 1 && cells % 2 == 0)
      run_apply<P, T, DG, CURVED, can_stage>(a, cells, nc, s);
    else
      run_apply<P, T, DG, CURVED>(a, cells, nc, s);
  }
  if constexpr (DG) {
    MFP_REQUIRE(a0.fb, "SIPG face buffer missing");
    const int threads = 256;
    const int bx = (a0.n[0] * P2 + threads - 1) / threads;
    const int rows = a0.n[1] * a0.n[2];
    const int by = rows < 65535 ? rows : 65535;
    if (a0.ncells > 0) {
      k_dg_face_add_t<P, T><<<dim3(bx, by, R), threads, 0, s>>>(a0);
      MFP_CHECK_CUDA(cudaGetLastError());
      note_launch();
    }
  }
}

template <typename T>
ApplyArgs<T> make_apply_args(const Level& L, const LevelData<T>& D,
                             const T* src, T* dst) {
  ApplyArgs<T> a{};
  a.src = src;
  a.dst = dst;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = L.n[d];
    a.g[d] = L.gdim[d];
    a.blo[d] = L.bc.lo[d];
    a.bhi[d] = L.bc.hi[d];
    a.face_off[d] = L.face_off[d];
  }
  a.neumann = L.bc.neumann;
  a.ncells = (int)L.ncells;
  a.G = D.G;
  a.kcell = D.kcell;
  a.kface = D.kface;
  a.fdata = D.fdata;
  a.sigma = D.sigma;
  a.fb = static_cast<T*>(L.fbuf);
  a.kappa = (T)L.kappa;
  const double vol = L.h[0] * L.h[1] * L.h[2];
  const double pen = L.penalty * (double)L.p * L.p;
  for (int d = 0; d < 3; ++d) {
    a.gs[d] = (T)(vol / (L.h[d] * L.h[d]));
    a.ns[d] = (T)(1.0 / L.h[d]);
    a.fa[d] = (T)(vol / L.h[d]);
    a.sg[d] = (T)(pen / L.h[d]);
  }
  a.stride = 1;
  a.col = 0;
  a.cpb = 1;
  a.ncols = 1;
  a.err = L.err;
  return a;
}

}  // namespace
}  // namespace mfp
