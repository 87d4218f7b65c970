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
// SIPG adds the six face integrals of its own test functions (each interior
// face is evaluated once from either side, with that side's outward normal;
// Eq. 6 visits each face twice in the same way) and stores its block.
#pragma once

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
  int face_off[3];
  const T* __restrict__ G;      // curved: [cell][6][p^3]
  const T* __restrict__ kcell;  // [cell][p^3] or null
  const T* __restrict__ kface;  // [face][p^2] or null
  const T* __restrict__ fdata;  // curved SIPG: [face][7][p^2]
  const T* __restrict__ sigma;  // curved SIPG: [face]
  T kappa;
  T gs[3];  // Cartesian: |K| / h_d^2
  T ns[3];  // Cartesian: 1 / h_d
  T fa[3];  // Cartesian: face area of a d-face
  T sg[3];  // Cartesian: penalty of a d-face
  int stride;  // batched layout: value i of column r at [i*stride + r]
  int col;     // first column of this launch
  int cpb;     // cells per block
  int ncols;   // columns per block
};

template <int P>
__device__ __forceinline__ int idx3(int x, int y, int z) {
  return x + P * (y + P * z);
}

// node (layer l along axis D, tangential coordinates a < b)
template <int P, int D>
__device__ __forceinline__ int fnode(int l, int a, int b) {
  if constexpr (D == 0) return l + P * (a + P * b);
  if constexpr (D == 1) return a + P * (l + P * b);
  return a + P * (b + P * l);
}

// Shared-memory stride of one virtual cell, odd so that the columns of a
// batch (adjacent threads, one virtual cell each) fall into distinct banks.
template <typename T, int P, bool DG>
__host__ __device__ constexpr int cell_smem_elems() {
  return ((DG ? 4 : 3) * P * P * P + (DG ? 8 * P * P : 0)) | 1;
}
template <int P>
__host__ __device__ constexpr int table_smem_elems() {
  return 3 * P * P + 3 * P;
}

// One line of a p x p face array: Y[line] = M X[line] (or M^T) along the
// first (DIR 0, index q + p c) or second (DIR 1, index c + p q) tangential
// axis; the 1D matrix is a constant-bank operand.
template <int P, typename T, int W, bool TRANS, int DIR>
__device__ __forceinline__ void face_line(const T* X, T* Y, int c) {
  T in[P], out[P];
#pragma unroll
  for (int j = 0; j < P; ++j) in[j] = X[DIR == 0 ? j + P * c : c + P * j];
  if constexpr (TRANS)
    mtv<T, P, W>(in, out);
  else
    mv<T, P, W>(in, out);
#pragma unroll
  for (int q = 0; q < P; ++q) Y[DIR == 0 ? q + P * c : c + P * q] = out[q];
}

// Face terms of SIPG (Eq. 6, mirror states Eq. 7) for one face of the own
// cell, in three parts: the trace gather and the final scatter depend on the
// face (axis D, side S: 0 lower, 1 upper) and are instantiated for each; the
// interpolation to the face Gauss points, the flux and the transposed
// interpolation are face-independent and exist once (the six faces run in a
// loop, which keeps the kernel's code within the instruction cache).
// Per-point parts use thread (ta, tb) for face point / node line (ta, tb);
// interpolations are line sweeps, one line per thread.  FS: 8 p^2 arrays.
template <int P, typename T, int D, int S>
__device__ __forceinline__ void face_gather(const ApplyArgs<T>& a, bool active,
                                            int nb, bool bnd, const T* U,
                                            T* FS, int ta, int tb) {
  constexpr int P2 = P * P, P3 = P2 * P;
  constexpr int SLO = S ? T_DPHI1 : T_DPHI0;  // own slope table
  constexpr int SLN = S ? T_DPHI0 : T_DPHI1;  // neighbour slope table
  constexpr int lo = S ? P - 1 : 0;
  constexpr int ln = S ? 0 : P - 1;
  const int t = ta + P * tb;
  T vo = U[fnode<P, D>(lo, ta, tb)];
  T dno = T(0);
#pragma unroll
  for (int l = 0; l < P; ++l)
    dno = fma(tv<T, P, SLO>(l), U[fnode<P, D>(l, ta, tb)], dno);
  T vn = T(0), dnn = T(0);
  if (!bnd && active) {
    const size_t cb = (size_t)nb * P3;
#pragma unroll
    for (int l = 0; l < P; ++l) {
      const T u = a.src[(cb + fnode<P, D>(l, ta, tb)) * a.stride + a.col];
      dnn = fma(tv<T, P, SLN>(l), u, dnn);
      if (l == ln) vn = u;
    }
  }
  FS[0 * P2 + t] = vo;
  FS[1 * P2 + t] = dno;
  FS[2 * P2 + t] = vn;
  FS[3 * P2 + t] = dnn;
}

template <int P, typename T, int D, int S>
__device__ __forceinline__ void face_scatter(T* Aq, const T* FS, int ta,
                                             int tb) {
  constexpr int P2 = P * P;
  constexpr int SLO = S ? T_DPHI1 : T_DPHI0;
  constexpr int lo = S ? P - 1 : 0;
  const int t = ta + P * tb;
  const T vf = FS[0 * P2 + t], nf = FS[1 * P2 + t];
  Aq[fnode<P, D>(lo, ta, tb)] += vf;
#pragma unroll
  for (int l = 0; l < P; ++l)
    Aq[fnode<P, D>(l, ta, tb)] += tv<T, P, SLO>(l) * nf;
}

// FS[0..3] = own value, own reference normal slope, neighbour value,
// neighbour slope at the face nodes  ->  FS[0] = value part, FS[1] =
// normal-slope part of the own test functions at the face nodes.
template <int P, typename T, bool CURVED>
__device__ __forceinline__ void face_core(const ApplyArgs<T>& a, int D, int S,
                                          int f, bool bnd, T* FS, const T* sw,
                                          int ta, int tb) {
  constexpr int P2 = P * P;
  const int t = ta + P * tb;
  for (int it = t; it < 4 * P; it += P2)
    face_line<P, T, T_S, false, 0>(FS + (it / P) * P2, FS + (4 + it / P) * P2,
                                   it % P);
  __syncthreads();
  for (int it = t; it < 4 * P; it += P2)
    face_line<P, T, T_S, false, 1>(FS + (4 + it / P) * P2, FS + (it / P) * P2,
                                   it % P);
  __syncthreads();
  if constexpr (CURVED) {  // tangential slopes of both traces
    for (int it = t; it < 4 * P; it += P2) {
      const int k = it / P;  // 0: d_a u-, 1: d_b u-, 2: d_a u+, 3: d_b u+
      const T* src = FS + (k < 2 ? 0 : 2) * P2;
      if (k & 1)
        face_line<P, T, T_D, false, 1>(src, FS + (4 + k) * P2, it % P);
      else
        face_line<P, T, T_D, false, 0>(src, FS + (4 + k) * P2, it % P);
    }
    __syncthreads();
  }
  // flux at face quadrature point (ta, tb)
  T cv, c0, c1 = T(0), c2 = T(0);
  {
    const T kap = a.kface ? a.kface[(size_t)f * P2 + t] : a.kappa;
    T uo = FS[0 * P2 + t], un = FS[2 * P2 + t], dno, dnn, dA, sig;
    if constexpr (!CURVED) {
      const T nsc = (S ? T(1) : T(-1)) * a.ns[D];
      dA = sw[ta] * sw[tb] * a.fa[D];
      sig = a.sg[D];
      dno = nsc * FS[1 * P2 + t];
      dnn = bnd ? dno : nsc * FS[3 * P2 + t];
      if (bnd) un = -uo;  // mirror state u+ = -u-, grad u+ = grad u- (Eq. 7)
      const T kdA = kap * dA;
      const T jump = uo - un;
      cv = kdA * (sig * jump - T(0.5) * (dno + dnn));
      c0 = T(-0.5) * kdA * jump * nsc;
    } else {
      const T* fd = a.fdata + (size_t)f * 7 * P2;
      dA = fd[t];
      sig = a.sigma[f];
      // reference gradients in (x, y, z) from (normal, first, second
      // tangential) components
      const T on = FS[1 * P2 + t], o1 = FS[4 * P2 + t], o2 = FS[5 * P2 + t];
      const T nn = FS[3 * P2 + t], n1 = FS[6 * P2 + t], n2 = FS[7 * P2 + t];
      const T gox = D == 0 ? on : o1, goy = D == 1 ? on : (D == 0 ? o1 : o2),
              goz = D == 2 ? on : o2;
      const T gnx = D == 0 ? nn : n1, gny = D == 1 ? nn : (D == 0 ? n1 : n2),
              gnz = D == 2 ? nn : n2;
      const int oo = S ? 1 : 4, on_ = S ? 4 : 1;  // own / neighbour J^{-1} n
      const T sgn = S ? T(1) : T(-1);  // own outward normal is sgn * n
      const T ox = fd[oo * P2 + t], oy = fd[(oo + 1) * P2 + t],
              oz = fd[(oo + 2) * P2 + t];
      const T mx = fd[on_ * P2 + t], my = fd[(on_ + 1) * P2 + t],
              mz = fd[(on_ + 2) * P2 + t];
      dno = sgn * (ox * gox + oy * goy + oz * goz);
      dnn = bnd ? dno : sgn * (mx * gnx + my * gny + mz * gnz);
      if (bnd) un = -uo;
      const T kdA = kap * dA;
      const T jump = uo - un;
      cv = kdA * (sig * jump - T(0.5) * (dno + dnn));
      const T cg = T(-0.5) * kdA * jump * sgn;
      const T gD = D == 0 ? ox : (D == 1 ? oy : oz);
      const T g1 = D == 0 ? oy : ox;
      const T g2 = D == 2 ? oy : oz;
      c0 = cg * gD;
      c1 = cg * g1;
      c2 = cg * g2;
    }
  }
  __syncthreads();
  FS[0 * P2 + t] = cv;
  FS[1 * P2 + t] = c0;
  if constexpr (CURVED) {
    FS[2 * P2 + t] = c1;
    FS[3 * P2 + t] = c2;
    __syncthreads();
    // tangential test slopes fold into the face-layer values
    for (int it = t; it < 2 * P; it += P2) {
      if (it < P)
        face_line<P, T, T_D, true, 0>(FS + 2 * P2, FS + 4 * P2, it);
      else
        face_line<P, T, T_D, true, 1>(FS + 3 * P2, FS + 5 * P2, it - P);
    }
    __syncthreads();
    FS[0 * P2 + t] += FS[4 * P2 + t] + FS[5 * P2 + t];
  }
  __syncthreads();
  // S^T along a, then along b, for the value and normal-slope parts
  for (int it = t; it < 2 * P; it += P2)
    face_line<P, T, T_S, true, 0>(FS + (it / P) * P2, FS + (2 + it / P) * P2,
                                  it % P);
  __syncthreads();
  for (int it = t; it < 2 * P; it += P2)
    face_line<P, T, T_S, true, 1>(FS + (2 + it / P) * P2, FS + (it / P) * P2,
                                  it % P);
  __syncthreads();
}

// One face of the own cell with line sweeps (the float variant: per-point
// table reads would saturate the load/store unit).
template <int P, typename T, bool CURVED, int D, int S>
__device__ __forceinline__ void face_contrib_ln(
    const ApplyArgs<T>& a, bool active, int cx, int cy, int cz, const T* U,
    T* Aq, T* FS, const T* sw, int ta, int tb) {
  int m[3] = {a.n[0], a.n[1], a.n[2]};
  m[D] += 1;
  int fc[3] = {cx, cy, cz};
  fc[D] += S;
  const int f = a.face_off[D] + fc[0] + m[0] * (fc[1] + m[1] * fc[2]);
  int nbc[3] = {cx, cy, cz};
  nbc[D] += S ? 1 : -1;
  const bool bnd = nbc[D] < 0 || nbc[D] >= a.n[D];
  const int nb = bnd ? 0 : nbc[0] + a.n[0] * (nbc[1] + a.n[1] * nbc[2]);
  face_gather<P, T, D, S>(a, active, nb, bnd, U, FS, ta, tb);
  __syncthreads();
  face_core<P, T, CURVED>(a, D, S, f, bnd, FS, sw, ta, tb);
  face_scatter<P, T, D, S>(Aq, FS, ta, tb);
  __syncthreads();
}

// One face of the own cell (axis D, side S: 0 lower, 1 upper), per face
// point: thread (ta, tb) interpolates all four traces to its own Gauss point
// with table rows from shared memory (the float64 variant: its FP64 pipe,
// not the load/store unit, is the limit).  Adds the face integrals tested
// with the own cell's basis into Aq (nodal values).
template <int P, typename T, bool CURVED, int D, int S>
__device__ __forceinline__ void face_contrib_pt(
    const ApplyArgs<T>& a, bool active, int cx, int cy, int cz, const T* U,
    T* Aq, T* FS, const T* sS, const T* sD, const T* s0, const T* s1,
    const T* sw, int ta, int tb) {
  constexpr int P2 = P * P, P3 = P2 * P;
  constexpr int T1 = D == 0 ? 1 : 0;
  constexpr int T2 = D == 2 ? 1 : 2;
  const int t = ta + P * tb;
  int m[3] = {a.n[0], a.n[1], a.n[2]};
  m[D] += 1;
  int fc[3] = {cx, cy, cz};
  fc[D] += S;
  const int f = a.face_off[D] + fc[0] + m[0] * (fc[1] + m[1] * fc[2]);
  int nbc[3] = {cx, cy, cz};
  nbc[D] += S ? 1 : -1;
  const bool bnd = nbc[D] < 0 || nbc[D] >= a.n[D];
  const int nb = bnd ? 0 : nbc[0] + a.n[0] * (nbc[1] + a.n[1] * nbc[2]);
  const T* dS = S ? s1 : s0;  // own slope at its face
  const T* dN = S ? s0 : s1;  // neighbour slope at its face
  constexpr int lo = S ? P - 1 : 0;
  constexpr int ln = S ? 0 : P - 1;
  // F1: nodal face values and reference normal slopes of both sides
  {
    T vo = U[fnode<P, D>(lo, ta, tb)];
    T dno = T(0);
#pragma unroll
    for (int l = 0; l < P; ++l) dno = fma(dS[l], U[fnode<P, D>(l, ta, tb)], dno);
    T vn = T(0), dnn = T(0);
    if (!bnd && active) {
      const T* sp = a.src;
      const size_t cb = (size_t)nb * P3;
#pragma unroll
      for (int l = 0; l < P; ++l) {
        T u = sp[(cb + fnode<P, D>(l, ta, tb)) * a.stride + a.col];
        dnn = fma(dN[l], u, dnn);
        if (l == ln) vn = u;
      }
    }
    FS[0 * P2 + t] = vo;
    FS[1 * P2 + t] = dno;
    FS[2 * P2 + t] = vn;
    FS[3 * P2 + t] = dnn;
  }
  __syncthreads();
  // F2: interpolate along the first tangential axis (a)
#pragma unroll
  for (int arr = 0; arr < 4; ++arr) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j)
      s = fma(sS[ta * P + j], FS[arr * P2 + j + P * tb], s);
    FS[(4 + arr) * P2 + t] = s;
  }
  __syncthreads();
  // F3: along the second tangential axis (b)
  T q[4];
#pragma unroll
  for (int arr = 0; arr < 4; ++arr) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j)
      s = fma(sS[tb * P + j], FS[(4 + arr) * P2 + ta + P * j], s);
    q[arr] = s;
  }
  __syncthreads();
  if constexpr (CURVED) {
    FS[0 * P2 + t] = q[0];
    FS[2 * P2 + t] = q[2];
    __syncthreads();
  }
  // flux at face quadrature point (ta, tb)
  {
    const T kap = a.kface ? a.kface[(size_t)f * P2 + t] : a.kappa;
    T uo = q[0], un = q[2], dno, dnn, dA, sig;
    T gvec[3] = {T(0), T(0), T(0)};  // own outward n J^{-T}... in xi coords
    if constexpr (!CURVED) {
      const T sgn = S ? T(1) : T(-1);
      dA = sw[ta] * sw[tb] * a.fa[D];
      sig = a.sg[D];
      dno = sgn * a.ns[D] * q[1];
      dnn = bnd ? dno : sgn * a.ns[D] * q[3];
      gvec[D] = sgn * a.ns[D];
    } else {
      const T* fd = a.fdata + (size_t)f * 7 * P2;
      dA = fd[t];
      sig = a.sigma[f];
      T go[3], gn[3];
      go[D] = q[1];
      gn[D] = q[3];
      T s1o = T(0), s2o = T(0), s1n = T(0), s2n = T(0);
#pragma unroll
      for (int j = 0; j < P; ++j) {
        s1o = fma(sD[ta * P + j], FS[0 * P2 + j + P * tb], s1o);
        s2o = fma(sD[tb * P + j], FS[0 * P2 + ta + P * j], s2o);
        s1n = fma(sD[ta * P + j], FS[2 * P2 + j + P * tb], s1n);
        s2n = fma(sD[tb * P + j], FS[2 * P2 + ta + P * j], s2n);
      }
      go[T1] = s1o;
      go[T2] = s2o;
      gn[T1] = s1n;
      gn[T2] = s2n;
      T nL[3], nR[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        nL[e] = fd[(1 + e) * P2 + t];
        nR[e] = fd[(4 + e) * P2 + t];
      }
      if constexpr (S == 1) {  // own cell is the left one: outward = +n
        dno = nL[0] * go[0] + nL[1] * go[1] + nL[2] * go[2];
        dnn = nR[0] * gn[0] + nR[1] * gn[1] + nR[2] * gn[2];
#pragma unroll
        for (int e = 0; e < 3; ++e) gvec[e] = nL[e];
      } else {  // own cell is the right one: outward = -n
        dno = -(nR[0] * go[0] + nR[1] * go[1] + nR[2] * go[2]);
        dnn = -(nL[0] * gn[0] + nL[1] * gn[1] + nL[2] * gn[2]);
#pragma unroll
        for (int e = 0; e < 3; ++e) gvec[e] = -nR[e];
      }
      if (bnd) dnn = dno;
    }
    if (bnd) un = -uo;  // mirror state u+ = -u-, grad u+ = grad u- (Eq. 7)
    const T kdA = kap * dA;
    const T jump = uo - un;
    const T avg = T(0.5) * (dno + dnn);
    const T cv = kdA * (sig * jump - avg);
    const T cg = T(-0.5) * kdA * jump;
    FS[4 * P2 + t] = cv;
    FS[5 * P2 + t] = cg * gvec[D];
    FS[6 * P2 + t] = cg * gvec[T1];
    FS[7 * P2 + t] = cg * gvec[T2];
  }
  __syncthreads();
  // tangential test slopes fold into the face-layer values
  T vq = FS[4 * P2 + t];
  if constexpr (CURVED) {
#pragma unroll
    for (int j = 0; j < P; ++j) {
      vq = fma(sD[j * P + ta], FS[6 * P2 + j + P * tb], vq);
      vq = fma(sD[j * P + tb], FS[7 * P2 + ta + P * j], vq);
    }
  }
  FS[0 * P2 + t] = vq;
  FS[1 * P2 + t] = FS[5 * P2 + t];
  __syncthreads();
  // S^T along a
#pragma unroll
  for (int arr = 0; arr < 2; ++arr) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j)
      s = fma(sS[j * P + ta], FS[arr * P2 + j + P * tb], s);
    FS[(2 + arr) * P2 + t] = s;
  }
  __syncthreads();
  // S^T along b and distribution onto the own nodes of line (ta, tb)
  {
    T vf = T(0), nf = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      vf = fma(sS[j * P + tb], FS[2 * P2 + ta + P * j], vf);
      nf = fma(sS[j * P + tb], FS[3 * P2 + ta + P * j], nf);
    }
    Aq[fnode<P, D>(lo, ta, tb)] += vf;
#pragma unroll
    for (int l = 0; l < P; ++l) Aq[fnode<P, D>(l, ta, tb)] += dS[l] * nf;
  }
  __syncthreads();
}

// Work decomposition: a block owns `cpb` cells and `ncols` right-hand-side
// columns; each (cell, column) pair is a virtual cell worked on by p*p
// threads (thread = one line of each sweep).  The block is padded to whole
// warps; padding threads work on a dummy virtual cell and write nothing to
// global memory.  Columns of one cell are adjacent threads, so batched
// vectors [N][R] are read coalesced and the geometry of a cell is loaded
// once per point for all its columns (same address across the warp).
template <int P, typename T, bool DG, bool CURVED>
__global__ void k_apply(const ApplyArgs<T> a) {
  constexpr int P2 = P * P, P3 = P2 * P;
  // float geometry is prefetched into registers during the gather (the float
  // apply is latency-bound); float64 is bound by the FP64 pipe instead
  constexpr bool PREFETCH = CURVED && sizeof(T) == 4 && P <= 7;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int cpb = a.cpb, nc = a.ncols;
  const int items = cpb * nc * P2;
  const int tid = threadIdx.x;
  const bool item_ok = tid < items;
  const int rr = tid % nc;
  const int rest = tid / nc;
  const int ta = rest % P, tb = (rest / P) % P;
  const int lc = item_ok ? rest / P2 : 0;
  const int v = item_ok ? lc * nc + rr : cpb * nc;  // dummy slot for padding
  T* base = sm + (size_t)v * cell_smem_elems<T, P, DG>();
  T* Aq = base;
  T* GX = base + P3;
  T* GY = base + 2 * P3;
  T* U = base + 3 * P3;   // DG: nodal input
  T* FS = base + 4 * P3;  // DG: face scratch [8][p^2]
  T* tabs = sm + (size_t)(cpb * nc + 1) * cell_smem_elems<T, P, DG>();
  T* sS = tabs;
  T* sD = tabs + P2;
  T* sDphi = tabs + 2 * P2;
  T* s0 = tabs + 3 * P2;
  T* s1 = s0 + P;
  T* sw = s1 + P;
  load_tables_shared<T, P>(sS, sD, sDphi, s0, s1, sw);
  __syncthreads();
  const int gx0 = a.g[0], gy0 = a.g[1], gz0 = a.g[2];
  ApplyArgs<T> ac = a;
  ac.col = a.col + rr;

  for (int cbase = blockIdx.x * cpb; cbase < a.ncells;
       cbase += gridDim.x * cpb) {
    const int cell = cbase + lc;
    const bool active = item_ok && cell < a.ncells;
    const int cc = active ? cell : 0;
    const int cx = cc % a.n[0];
    const int cy = (cc / a.n[0]) % a.n[1];
    const int cz = cc / (a.n[0] * a.n[1]);
    const int col = ac.col;
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
        U[idx3<P>(ta, tb, z)] = r[z];
      }
    } else {
      const int X = cx * (P - 1) + ta, Y = cy * (P - 1) + tb;
      const bool bxy = X == 0 || X == gx0 - 1 || Y == 0 || Y == gy0 - 1;
#pragma unroll
      for (int z = 0; z < P; ++z) {
        const int Z = cz * (P - 1) + z;
        const bool con = bxy || Z == 0 || Z == gz0 - 1;
        const size_t gi = (size_t)X + (size_t)gx0 * (Y + (size_t)gy0 * Z);
        r[z] = (active && !con) ? a.src[gi * a.stride + col] : T(0);
      }
    }
    // ---- values at Gauss points: z (registers), y, x
    mv<T, P, T_S>(r, o);
#pragma unroll
    for (int z = 0; z < P; ++z) Aq[idx3<P>(ta, tb, z)] = o[z];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(ta, j, tb)];
    mv<T, P, T_S>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(ta, j, tb)] = o[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(j, ta, tb)];
    mv<T, P, T_S>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(j, ta, tb)] = o[j];
    mv<T, P, T_D>(o, r);
#pragma unroll
    for (int j = 0; j < P; ++j) GX[idx3<P>(j, ta, tb)] = r[j];
    __syncthreads();
    // ---- reference gradient: y into GY, z kept in registers
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(ta, j, tb)];
    mv<T, P, T_D>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) GY[idx3<P>(ta, j, tb)] = o[j];
    T gz[P];
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(ta, tb, j)];
    mv<T, P, T_D>(r, gz);
    __syncthreads();
    // ---- quadrature-point operation t = G_q grad u (Eq. 12)
    {
      const T wab = sw[ta] * sw[tb];
#pragma unroll
      for (int qz = 0; qz < P; ++qz) {
        const int q = idx3<P>(ta, tb, qz);
        const T ux = GX[q], uy = GY[q], uz = gz[qz];
        const T kap = a.kcell ? a.kcell[(size_t)cc * P3 + q] : a.kappa;
        T tx, ty, tz;
        if constexpr (CURVED) {
          T g0, g1, g2, g3, g4, g5;
          if constexpr (PREFETCH) {
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
        GX[q] = tx;
        GY[q] = ty;
        r[qz] = tz;
      }
      mtv<T, P, T_D>(r, o);
#pragma unroll
      for (int j = 0; j < P; ++j) Aq[idx3<P>(ta, tb, j)] = o[j];
    }
    __syncthreads();
    // ---- transposed derivative y (added), x (added) then S^T x, y, z
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = GY[idx3<P>(ta, j, tb)];
    mtv<T, P, T_D>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(ta, j, tb)] += o[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = GX[idx3<P>(j, ta, tb)];
    mtv<T, P, T_D>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) o[j] += Aq[idx3<P>(j, ta, tb)];
    mtv<T, P, T_S>(o, r);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(j, ta, tb)] = r[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(ta, j, tb)];
    mtv<T, P, T_S>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(ta, j, tb)] = o[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(ta, tb, j)];
    mtv<T, P, T_S>(r, o);
    // ---- scatter
    if constexpr (!DG) {
      const int X = cx * (P - 1) + ta, Y = cy * (P - 1) + tb;
      const bool bxy = X == 0 || X == gx0 - 1 || Y == 0 || Y == gy0 - 1;
      if (active) {
#pragma unroll
        for (int z = 0; z < P; ++z) {
          const int Z = cz * (P - 1) + z;
          const bool con = bxy || Z == 0 || Z == gz0 - 1;
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
#pragma unroll
      for (int z = 0; z < P; ++z) Aq[idx3<P>(ta, tb, z)] = o[z];
      __syncthreads();
      if constexpr (sizeof(T) == 4) {
#define FACE(DD, SS)                                                          \
  face_contrib_ln<P, T, CURVED, DD, SS>(ac, active, cx, cy, cz, U, Aq, FS, sw, \
                                        ta, tb)
        FACE(0, 0); FACE(0, 1); FACE(1, 0); FACE(1, 1); FACE(2, 0); FACE(2, 1);
#undef FACE
      } else {
#define FACE(DD, SS)                                                          \
  face_contrib_pt<P, T, CURVED, DD, SS>(ac, active, cx, cy, cz, U, Aq, FS, sS, \
                                        sD, s0, s1, sw, ta, tb)
        FACE(0, 0); FACE(0, 1); FACE(1, 0); FACE(1, 1); FACE(2, 0); FACE(2, 1);
#undef FACE
      }
      if (active) {
#pragma unroll
        for (int z = 0; z < P; ++z) {
          const size_t gi = (size_t)cc * P3 + idx3<P>(ta, tb, z);
          a.dst[gi * a.stride + col] = Aq[idx3<P>(ta, tb, z)];
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

template <int P, typename T, bool DG, bool CURVED>
void run_apply(ApplyArgs<T> a, int cpb, int ncols, cudaStream_t s) {
  constexpr int P2 = P * P;
  a.cpb = cpb;
  a.ncols = ncols;
  const int threads = ((cpb * ncols * P2 + 31) / 32) * 32;
  const size_t smem = ((size_t)(cpb * ncols + 1) * cell_smem_elems<T, P, DG>() +
                       table_smem_elems<P>()) *
                      sizeof(T);
  auto kern = k_apply<P, T, DG, CURVED>;
  if (smem > 48 * 1024)
    MFP_CHECK_CUDA(cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MFP_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, kern, threads, smem));
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
    int cells = cells_req > 0 ? cells_req : default_cpb(P) / nc;
    if (cells < 1) cells = 1;
    while (cells > 1 && cells * nc * P2 > maxthr) --cells;
    ApplyArgs<T> a = a0;
    a.col = c0;
    run_apply<P, T, DG, CURVED>(a, cells, nc, s);
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
    a.face_off[d] = L.face_off[d];
  }
  a.ncells = (int)L.ncells;
  a.G = D.G;
  a.kcell = D.kcell;
  a.kface = D.kface;
  a.fdata = D.fdata;
  a.sigma = D.sigma;
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
  return a;
}

}  // namespace
}  // namespace mfp
