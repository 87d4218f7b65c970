// FP64-accurate operator evaluation on the FP32 pipes (double-float).
//
// The same sum-factorized cell integral (Sec. 3, Eq. 12) and SIPG face terms
// (Eq. 6, Eq. 7) as k_apply.cuh, with float64 vectors in HBM and every
// intermediate carried as a double-float pair (df.cuh).  On GB300 the FP64
// pipe issues 2 DFMA per clock per SM while the FP32 pipe issues 128 FFMA;
// a double-float multiply-accumulate costs 12 FP32 instructions, so the FP32
// pipe delivers about 5x the FP64 rate at about 48 significant bits.  Only
// the conversions of the float64 inputs and outputs use the FP64 pipe.
//
// Per cell: gather, interpolation to the Gauss points (S along z, y, x,
// even-odd split for p >= 4), collocation derivatives, the quadrature-point
// operation, the transposed derivatives, then (SIPG) the face terms added at
// the Gauss points (df_face_gp: each interior face once, by the cell below
// it; the upper neighbour's share through the face buffer and
// k_dg_face_add), then S^T along x, y, z and the store (CG: atomic scatter).
#pragma once

#define MFP_DF_TABLES
#include "dev_tables.cuh"
#include "df.cuh"

// Resident blocks per SM the register allocation must allow (blocks of at
// most 128 threads for p <= 5, 256 above), measured on 24^3..64^3 meshes
// for k = 2..8: more resident warps hide the latency of the shared-memory
// sweeps and the gathers, down to about 73 registers per thread; CG p >= 7
// keeps its larger line arrays in registers.  At p = 5, with one block per
// cell group, the concurrent CG and SIPG solves of 32^3 curved cells
// measured best at 6 (CG, 80 registers) and 8 (SIPG, 64) blocks: 60.7 ->
// 58.9 ms per pair of solves (SIPG apply alone 0.399 -> 0.412 ms, its
// solve's coarser levels faster; CG apply 0.181 -> 0.158 ms).

namespace mfp {
namespace {

struct ApplyArgsDF {
  const double* __restrict__ src;
  double* __restrict__ dst;
  int n[3];
  int ncells;
  int g[3];
  int blo[3], bhi[3];        // CG: constrained node coordinates (-1: none)
  int neumann;               // SIPG: bit 2d + s = Neumann side
  int face_off[3];
  const float *Gh, *Gl;      // curved: [cell][6][p^3]
  const float *kch, *kcl;    // [cell][p^3] or null
  const float *kfh, *kfl;    // [face][p^2] or null
  const float *fdh, *fdl;    // curved SIPG: [face][7][p^2]
  const float *sgh, *sgl;    // curved SIPG: [face]
  float2* fb;                // SIPG: [cell][6][p^2] x columns, see below
  df kappa;
  bool kappa_one;            // constant coefficient exactly 1
  df gs[3], ns[3], fa[3], sg[3];
  int stride, col, cpb, ncols;
  Epi<double> epi;           // SIPG: update fused into k_dg_face_add
  df epi_c1, epi_c2;         // its coefficients as double-float pairs
};

// The fused update of Epi in double-float arithmetic on the FP32 pipes: the
// float64 inputs (loaded by the caller ahead of its arithmetic: b, dinv, d,
// x as the mode needs them) are split with integer operations and only the
// float64 results take one FP64 addition each.
__device__ __forceinline__ void epi_finish_df(const ApplyArgsDF& a, size_t gi,
                                              df y, double b, double dinv,
                                              double d, double x) {
  const Epi<double>& e = a.epi;
  if (e.mode == EPI_STORE) {
    a.dst[gi] = df_to_double(y);
    return;
  }
  const df r = df_from_double(b) - y;
  if (e.mode == EPI_RESIDUAL) {
    a.dst[gi] = df_to_double(r);
    return;
  }
  const df dr = df_from_double(dinv) * r;
  const df v = e.mode == EPI_CHEB_FIRST
                   ? a.epi_c1 * dr
                   : a.epi_c1 * df_from_double(d) + a.epi_c2 * dr;
  e.d[gi] = df_to_double(v);
  e.x[gi] = df_to_double(df_from_double(x) + v);
}

__device__ __forceinline__ df f2df(float2 v) { return df_make(v.x, v.y); }
__device__ __forceinline__ float2 df2f(df v) { return make_float2(v.h, v.l); }
__device__ __forceinline__ void st2(float2* a, int i, df v) { a[i] = df2f(v); }
__device__ __forceinline__ dacc acc_first(float2 a, float2 b) {
  return acc_first(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void acc_mac(dacc& s, float2 a, float2 b) {
  acc_mac(s, a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ dacc acc_first(float ah, float al, float2 b) {
  return acc_first(ah, al, b.x, b.y);
}
__device__ __forceinline__ void acc_mac(dacc& s, float ah, float al,
                                        float2 b) {
  acc_mac(s, ah, al, b.x, b.y);
}

__device__ __forceinline__ df ld(const float* h, const float* l, int i) {
  return df_make(h[i], l[i]);
}

enum DfTab { DF_S, DF_D };

template <int P, int W>
__device__ __forceinline__ float tdh(int i) {
  if constexpr (W == DF_S) return c_tabdf[P - 2].Sh[i];
  return c_tabdf[P - 2].Dh[i];
}
template <int P, int W>
__device__ __forceinline__ float tdl(int i) {
  if constexpr (W == DF_S) return c_tabdf[P - 2].Sl[i];
  return c_tabdf[P - 2].Dl[i];
}

// out[j] = sum_q M[q][j] in[q]
template <int P, int W>
__device__ __forceinline__ void dmtv(const float (&ih)[P],
                                     const float (&il)[P], float (&oh)[P],
                                     float (&ol)[P]) {
#pragma unroll
  for (int j = 0; j < P; ++j) {
    dacc s = acc_first(tdh<P, W>(j), tdl<P, W>(j), ih[0], il[0]);
#pragma unroll
    for (int q = 1; q < P; ++q)
      acc_mac(s, tdh<P, W>(q * P + j), tdl<P, W>(q * P + j), ih[q], il[q]);
    const df r = acc_get(s);
    oh[j] = r.h;
    ol[j] = r.l;
  }
}

// Rolled sum-factorization sweeps (p >= 4): a loop over the
// output index with the table entries read by index keeps the double-float
// code P times shorter than the unrolled matrix-vector product; unrolled,
// the sweeps and faces of a cell overflow the instruction caches and
// instruction fetch limits the issue rate (p <= 3 stays unrolled, its code
// is short and the indexed table reads would cost more than they save).
#define MFP_DF_STR2(x) #x
#define MFP_DF_STR(x) MFP_DF_STR2(x)
#define MFP_DF_LOOP _Pragma(MFP_DF_STR(unroll(P >= 4 ? 1 : P)))

// Even-odd split of the sweeps (p >= 4, MFP_DF_EO): the mirror symmetry of
// S and D (tables c_tabeo) halves the multiply-adds of each sweep for the
// price of 2 p double-float additions.
#ifndef MFP_DF_EO
#define MFP_DF_EO 1
#endif

// o[base + q * st] (+)= sum_j M[q][j] in[j]  (TR: M[j][q]), q = 0..P-1
template <int P, int W, bool TR, bool ADD>
__device__ __forceinline__ void dsweep(const float (&ih)[P],
                                       const float (&il)[P], float2* out,
                                       int base, int st) {
  if constexpr (P >= 4 && MFP_DF_EO) {
    constexpr int H = P / 2, MC = H + P % 2;
    constexpr int w = 2 * (W == DF_D ? 1 : 0) + (TR ? 1 : 0);
    const DevTabEO& E = c_tabeo[P - 2];
    float eh[MC], el[MC], odh[H], odl[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const df xa = df_make(ih[j], il[j]);
      const df xb = df_make(ih[P - 1 - j], il[P - 1 - j]);
      const df e = xa + xb, o = xa - xb;
      eh[j] = e.h;
      el[j] = e.l;
      odh[j] = o.h;
      odl[j] = o.l;
    }
    if constexpr (P % 2 == 1) {
      eh[H] = ih[H];
      el[H] = il[H];
    }
    MFP_DF_LOOP
    for (int q = 0; q < H; ++q) {
      const int r = q * kMaxH;
      dacc sa = acc_first(E.ah[w][r], E.al[w][r], eh[0], el[0]);
#pragma unroll
      for (int j = 1; j < MC; ++j)
        acc_mac(sa, E.ah[w][r + j], E.al[w][r + j], eh[j], el[j]);
      dacc sb = acc_first(E.bh[w][r], E.bl[w][r], odh[0], odl[0]);
#pragma unroll
      for (int j = 1; j < H; ++j)
        acc_mac(sb, E.bh[w][r + j], E.bl[w][r + j], odh[j], odl[j]);
      const df A = acc_get(sa), B = acc_get(sb);
      df r1 = A + B, r2 = A - B;
      if constexpr (W == DF_D) r2 = -r2;
      const int o1 = base + q * st, o2 = base + (P - 1 - q) * st;
      if constexpr (ADD) {
        r1 = f2df(out[o1]) + r1;
        r2 = f2df(out[o2]) + r2;
      }
      out[o1] = df2f(r1);
      out[o2] = df2f(r2);
    }
    if constexpr (P % 2 == 1) {  // middle row: A (S) or B (D) only
      constexpr int r = H * kMaxH;
      dacc sm;
      if constexpr (W == DF_S) {
        sm = acc_first(E.ah[w][r], E.al[w][r], eh[0], el[0]);
#pragma unroll
        for (int j = 1; j < MC; ++j)
          acc_mac(sm, E.ah[w][r + j], E.al[w][r + j], eh[j], el[j]);
      } else {
        sm = acc_first(E.bh[w][r], E.bl[w][r], odh[0], odl[0]);
#pragma unroll
        for (int j = 1; j < H; ++j)
          acc_mac(sm, E.bh[w][r + j], E.bl[w][r + j], odh[j], odl[j]);
      }
      df rm = acc_get(sm);
      const int o = base + H * st;
      if constexpr (ADD) rm = f2df(out[o]) + rm;
      out[o] = df2f(rm);
    }
  } else {
    MFP_DF_LOOP
    for (int q = 0; q < P; ++q) {
      const int i0 = TR ? q : q * P;
      constexpr int js = TR ? P : 1;
      dacc s = acc_first(tdh<P, W>(i0), tdl<P, W>(i0), ih[0], il[0]);
#pragma unroll
      for (int j = 1; j < P; ++j)
        acc_mac(s, tdh<P, W>(i0 + j * js), tdl<P, W>(i0 + j * js), ih[j],
                il[j]);
      df r = acc_get(s);
      const int o = base + q * st;
      if constexpr (ADD) r = f2df(out[o]) + r;
      out[o] = df2f(r);
    }
  }
}

// load the line base + j * st of a shared array into registers
template <int P>
__device__ __forceinline__ void dline(const float2* x, int base, int st,
                                      float (&oh)[P], float (&ol)[P]) {
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const float2 v = x[base + j * st];
    oh[j] = v.x;
    ol[j] = v.y;
  }
}

template <int P>
__device__ __forceinline__ int dx3(int x, int y, int z) {
  return x + P * (y + P * z);
}

// Shared memory holds double-float values as float2 (hi, lo): one 64-bit
// access per value.  Per virtual cell, in float2 units: A, X, Y (and U for
// SIPG) of p^3 values and the SIPG face scratch of 8 p^2, which for p >= 4
// reuses X and Y (dead while the faces run); the odd stride puts the
// columns of a batch into distinct banks.
#ifndef MFP_DF_FS_ALIAS
#define MFP_DF_FS_ALIAS 1
#endif
template <int P>
__host__ __device__ constexpr bool df_fs_alias() {
  return MFP_DF_FS_ALIAS && 2 * P >= 8;
}
template <int P, bool DG>
__host__ __device__ constexpr int df_cell_pairs() {
  return ((DG ? 4 : 3) * P * P * P +
          (DG && !df_fs_alias<P>() ? 8 * P * P : 0)) |
         1;
}
template <int P>
__host__ __device__ constexpr int df_table_pairs() {
  return 2 * P * P + 3 * P;
}

// shared DF table views (row-major p x p)
struct ShDF {
  const float2 *S, *D, *d0, *d1, *w;
};

template <int P>
__device__ __forceinline__ ShDF make_shdf(const float2* tabs) {
  constexpr int P2 = P * P;
  ShDF t;
  t.S = tabs;
  t.D = tabs + P2;
  t.d0 = tabs + 2 * P2;
  t.d1 = t.d0 + P;
  t.w = t.d1 + P;
  return t;
}

// One face of the own cell (axis D a runtime value, one copy of the face
// code in the kernel).  The own side works on the cell's values at its
// Gauss points: its trace and reference normal slope at face point
// (ta, tb) come from the line of Gauss-point values along D through it
// (Lagrange basis of the Gauss points at the cell end, exact for the
// degree-k polynomial), and its value and normal-slope test terms go back
// onto the same line of the Gauss-point accumulator A, which the cell's
// S^T sweeps then take to the nodes.  Each interior face is evaluated
// once, by the cell below it (S = 1): the upper neighbour's trace comes
// from its float64 nodal values (face layer and normal slope, then S x S
// to the face points), and its test terms go through S^T x S^T to its
// face nodes and into the face buffer fb (slot 2D: value part, 2D + 1:
// normal-slope part) for k_dg_face_add.  A boundary face is one-sided
// with the mirror state of Eq. 7; an interior lower face (S = 0) adds
// nothing here.  FS holds 8 hi arrays then 8 lo arrays.
template <int P, bool CURVED, int S>
__device__ __forceinline__ void df_face_gp(const ApplyArgsDF& a, int col,
                                           int D, bool active, int cx, int cy,
                                           int cz, const float2* U,
                                           float2* A, float2* FS,
                                           const ShDF& t, int ta, int tb) {
  constexpr int P2 = P * P, P3 = P2 * P;
  const int ti = ta + P * tb;
  // point (l, ta, tb) of the own line normal to D is n0 + l * ls (the same
  // for Gauss points and nodes)
  const int ls = D == 0 ? 1 : (D == 1 ? P : P2);
  const int n0 = D == 0 ? P * ti : (D == 1 ? ta + P2 * tb : ti);
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
  const DevTabDF& T = c_tabdf[P - 2];
  const float* gvh = S ? T.gv1h : T.gv0h;
  const float* gvl = S ? T.gv1l : T.gv0l;
  const float* gdh = S ? T.gd1h : T.gd0h;
  const float* gdl = S ? T.gd1l : T.gd0l;
  // own trace and reference normal slope at the face point (ta, tb)
  df uo, so;
  {
    dacc sv = acc_first(gvh[0], gvl[0], U[n0]);
    dacc sd = acc_first(gdh[0], gdl[0], U[n0]);
#pragma unroll
    for (int l = 1; l < P; ++l) {
      acc_mac(sv, gvh[l], gvl[l], U[n0 + l * ls]);
      acc_mac(sd, gdh[l], gdl[l], U[n0 + l * ls]);
    }
    uo = acc_get(sv);
    so = acc_get(sd);
  }
  if constexpr (CURVED) st2(FS, 0 * P2 + ti, uo);
  // the upper neighbour's face layer and reference normal slope (nodal),
  // interpolated to the face points: FS[2, 3] -> FS[6, 7] -> FS[2, 3]
  if constexpr (S == 1) {
    df vn = df_make(0.f), dnn = df_make(0.f);
    if (pair) {
      const double* u0 = a.src + ((size_t)nb * P3 + n0) * a.stride + col;
      const size_t lstr = (size_t)ls * a.stride;
      dacc sn;
      sn.h = 0.f;
      sn.l = 0.f;
#pragma unroll
      for (int l = 0; l < P; ++l) {
        const df u = df_from_double(u0[l * lstr]);
        if (l == 0) {
          sn = acc_first(t.d0[0], make_float2(u.h, u.l));
          vn = u;
        } else {
          acc_mac(sn, t.d0[l], make_float2(u.h, u.l));
        }
      }
      dnn = acc_get(sn);
    }
    st2(FS, 2 * P2 + ti, vn);
    st2(FS, 3 * P2 + ti, dnn);
    __syncthreads();
#pragma unroll 1
    for (int arr = 2; arr < 4; ++arr) {
      const float2* iv = FS + arr * P2 + P * tb;
      dacc s = acc_first(t.S[ta * P], iv[0]);
#pragma unroll
      for (int j = 1; j < P; ++j)
        acc_mac(s, t.S[ta * P + j], iv[j]);
      st2(FS, (4 + arr) * P2 + ti, acc_get(s));
    }
    __syncthreads();
#pragma unroll 1
    for (int arr = 2; arr < 4; ++arr) {
      const float2* iv = FS + (4 + arr) * P2 + ta;
      dacc s = acc_first(t.S[tb * P], iv[0]);
#pragma unroll
      for (int j = 1; j < P; ++j)
        acc_mac(s, t.S[tb * P + j], iv[P * j]);
      st2(FS, arr * P2 + ti, acc_get(s));
    }
  }
  if constexpr (CURVED) __syncthreads();
  // flux at the face quadrature points: value coefficient cv of the own
  // side (-cv on the neighbour) and test-slope coefficients cg J^-1 n of
  // each side, in face-local components (normal, tangential 1, 2)
  df cv, c0o, c0n;
  {
    const df kap = a.kfh ? df_make(a.kfh[(size_t)f * P2 + ti],
                                   a.kfl[(size_t)f * P2 + ti])
                         : a.kappa;
    df un = S ? f2df(FS[2 * P2 + ti]) : df_make(0.f);
    const df q3 = S ? f2df(FS[3 * P2 + ti]) : df_make(0.f);
    df dno, dnn, dA, sig;
    df go1, go2, gn1, gn2;  // tangential test-slope factors, both sides
    df gvD, gnD;            // normal ones
    if constexpr (!CURVED) {
      const float sgn = S ? 1.f : -1.f;
      const df w2 = f2df(t.w[ta]) * f2df(t.w[tb]);
      dA = w2 * a.fa[D];
      sig = a.sg[D];
      const df nsc = df_make(sgn * a.ns[D].h, sgn * a.ns[D].l);
      dno = nsc * so;
      dnn = bnd ? dno : nsc * q3;
      gvD = nsc;
      gnD = nsc;
    } else {
      const int T1 = D == 0 ? 1 : 0;
      const int T2 = D == 2 ? 1 : 2;
      const size_t fb = (size_t)f * 7 * P2 + ti;
      dA = ld(a.fdh, a.fdl, fb);
      sig = df_make(a.sgh[f], a.sgl[f]);
      // reference tangential slopes of the own trace
      dacc s1o = acc_first(t.D[ta * P], FS[P * tb]);
      dacc s2o = acc_first(t.D[tb * P], FS[ta]);
      MFP_DF_LOOP
      for (int j = 1; j < P; ++j) {
        acc_mac(s1o, t.D[ta * P + j], FS[j + P * tb]);
        acc_mac(s2o, t.D[tb * P + j], FS[ta + P * j]);
      }
      const df t1o = acc_get(s1o), t2o = acc_get(s2o);
      // J^-1 n of the lower (L) and upper (R) cell, face-local components
      const df RD = ld(a.fdh, a.fdl, fb + (4 + D) * P2),
               R1 = ld(a.fdh, a.fdl, fb + (4 + T1) * P2),
               R2 = ld(a.fdh, a.fdl, fb + (4 + T2) * P2);
      if constexpr (S == 1) {  // own cell is the lower one: outward = +n
        const df LD = ld(a.fdh, a.fdl, fb + (1 + D) * P2),
                 L1 = ld(a.fdh, a.fdl, fb + (1 + T1) * P2),
                 L2 = ld(a.fdh, a.fdl, fb + (1 + T2) * P2);
        // and of the neighbour's trace
        dacc s1n = acc_first(t.D[ta * P], FS[2 * P2 + P * tb]);
        dacc s2n = acc_first(t.D[tb * P], FS[2 * P2 + ta]);
        MFP_DF_LOOP
        for (int j = 1; j < P; ++j) {
          acc_mac(s1n, t.D[ta * P + j], FS[2 * P2 + j + P * tb]);
          acc_mac(s2n, t.D[tb * P + j], FS[2 * P2 + ta + P * j]);
        }
        dacc sa = acc_first(LD.h, LD.l, so.h, so.l);
        acc_mac(sa, L1.h, L1.l, t1o.h, t1o.l);
        acc_mac(sa, L2.h, L2.l, t2o.h, t2o.l);
        const df t1n = acc_get(s1n), t2n = acc_get(s2n);
        dacc sb = acc_first(RD.h, RD.l, q3.h, q3.l);
        acc_mac(sb, R1.h, R1.l, t1n.h, t1n.l);
        acc_mac(sb, R2.h, R2.l, t2n.h, t2n.l);
        dno = acc_get(sa);
        dnn = bnd ? dno : acc_get(sb);
        gvD = LD;
        go1 = L1;
        go2 = L2;
        gnD = RD;
        gn1 = R1;
        gn2 = R2;
      } else {  // own cell is the upper one (boundary only): outward = -n
        dacc sa = acc_first(RD.h, RD.l, so.h, so.l);
        acc_mac(sa, R1.h, R1.l, t1o.h, t1o.l);
        acc_mac(sa, R2.h, R2.l, t2o.h, t2o.l);
        dno = -acc_get(sa);
        dnn = dno;
        gvD = -RD;
        go1 = -R1;
        go2 = -R2;
        gnD = gvD;
      }
    }
    if (bnd) un = -uo;  // mirror state (Eq. 7)
    const df kdA = kap * dA;
    const df jump = uo - un;
    const df avg = df_scale2(dno + dnn, 0.5f);
    cv = kdA * (sig * jump - avg);
    const df cg = df_scale2(kdA * jump, -0.5f);
    c0o = cg * gvD;
    c0n = cg * gnD;
    if constexpr (CURVED) {
      st2(FS, 4 * P2 + ti, cg * go1);
      st2(FS, 5 * P2 + ti, cg * go2);
      if constexpr (S == 1) {
        st2(FS, 6 * P2 + ti, cg * gn1);
        st2(FS, 7 * P2 + ti, cg * gn2);
      }
    }
  }
  // fold the tangential test slopes into the value parts (D^T at the face
  // points)
  df vo = cv, vn = -cv;
  if constexpr (CURVED) {
    __syncthreads();
    dacc sa, sb;
    sa.h = cv.h;
    sa.l = cv.l;
    sb.h = vn.h;
    sb.l = vn.l;
    MFP_DF_LOOP
    for (int j = 0; j < P; ++j) {
      acc_mac(sa, t.D[j * P + ta], FS[4 * P2 + j + P * tb]);
      acc_mac(sa, t.D[j * P + tb], FS[5 * P2 + ta + P * j]);
      if constexpr (S == 1) {
        acc_mac(sb, t.D[j * P + ta], FS[6 * P2 + j + P * tb]);
        acc_mac(sb, t.D[j * P + tb], FS[7 * P2 + ta + P * j]);
      }
    }
    vo = acc_get(sa);
    vn = acc_get(sb);
  }
  // own test terms onto the line of Gauss points along D
  if (own) {
    MFP_DF_LOOP
    for (int l = 0; l < P; ++l) {
      const int j = n0 + l * ls;
      dacc s;
      s.h = A[j].x;
      s.l = A[j].y;
      acc_mac(s, gvh[l], gvl[l], vo.h, vo.l);
      acc_mac(s, gdh[l], gdl[l], c0o.h, c0o.l);
      st2(A, j, acc_get(s));
    }
  }
  // the neighbour's test terms to its face nodes: S^T along a, then b
  if constexpr (S == 1) {
    st2(FS, 0 * P2 + ti, vn);
    st2(FS, 1 * P2 + ti, c0n);
    __syncthreads();
#pragma unroll 1
    for (int arr = 0; arr < 2; ++arr) {
      const float2* iv = FS + arr * P2 + P * tb;
      dacc s = acc_first(t.S[ta], iv[0]);
#pragma unroll
      for (int j = 1; j < P; ++j)
        acc_mac(s, t.S[j * P + ta], iv[j]);
      st2(FS, (4 + arr) * P2 + ti, acc_get(s));
    }
    __syncthreads();
    df res[2];
#pragma unroll
    for (int arr = 0; arr < 2; ++arr) {
      const float2* iv = FS + (4 + arr) * P2 + ta;
      dacc s = acc_first(t.S[tb], iv[0]);
#pragma unroll
      for (int j = 1; j < P; ++j)
        acc_mac(s, t.S[j * P + tb], iv[P * j]);
      res[arr] = acc_get(s);
    }
    if (pair) {
      float2* fbn = a.fb + ((size_t)nb * 6 + 2 * D) * P2 * a.stride + col;
      fbn[(size_t)ti * a.stride] = make_float2(res[0].h, res[0].l);
      fbn[(size_t)(P2 + ti) * a.stride] = make_float2(res[1].h, res[1].l);
    }
  }
}

template <int P, bool CURVED>
__device__ __noinline__ void df_face_lower_gp(const ApplyArgsDF& a, int col,
                                              int D, bool active, int cx,
                                              int cy, int cz, const float2* U,
                                              float2* A, float2* FS,
                                              const float2* tabs,
                                              int ta, int tb) {
  df_face_gp<P, CURVED, 0>(a, col, D, active, cx, cy, cz, U, A, FS,
                           make_shdf<P>(tabs), ta, tb);
  __syncthreads();
}

template <int P>
constexpr int df_max_threads() { return P <= 5 ? 128 : 256; }
template <int P, bool DG>
constexpr int df_min_blocks() {
  if (DG) return P <= 3 ? 5 : (P == 4 ? 7 : (P == 5 ? 8 : 2));
  return P <= 4 ? 8 : (P == 5 ? 6 : (P == 6 ? 3 : 1));
}

template <int P, bool DG>
constexpr int df_max_regs() {
  return 65536 / (df_min_blocks<P, DG>() * df_max_threads<P>());
}

// __maxnreg__ caps the registers without capping the block size (batched
// launches use up to 1024 threads; shapes that do not fit are rejected).
template <int P, bool DG, bool CURVED>
__global__ void __maxnreg__((df_max_regs<P, DG>() > 255 ? 255
                                                       : df_max_regs<P, DG>()))
    k_apply_df(const __grid_constant__ ApplyArgsDF a) {
  constexpr int P2 = P * P, P3 = P2 * P;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int cpb = a.cpb, nc = a.ncols;
  const int items = cpb * nc * P2;
  const int tid = threadIdx.x;
  const bool item_ok = tid < items;
  const int rr = tid % nc;
  const int rest = tid / nc;
  const int ta = rest % P, tb = (rest / P) % P;
  const int lc = item_ok ? rest / P2 : 0;
  const int v = item_ok ? lc * nc + rr : cpb * nc;
  float2* base = sm + (size_t)v * df_cell_pairs<P, DG>();
  float2* A = base;
  float2* X = base + P3;      // GX
  float2* Y = base + 2 * P3;  // GY
  float2* U = base + 3 * P3;  // DG: values at the Gauss points
  float2* FS = df_fs_alias<P>() ? X : base + 4 * P3;
  float2* tabs = sm + (size_t)(cpb * nc + 1) * df_cell_pairs<P, DG>();
  const ShDF t = make_shdf<P>(tabs);
  {
    const DevTabDF& T = c_tabdf[P - 2];
    for (int i = tid; i < P2; i += blockDim.x) {
      tabs[i] = make_float2(T.Sh[i], T.Sl[i]);
      tabs[P2 + i] = make_float2(T.Dh[i], T.Dl[i]);
    }
    float2* p = tabs + 2 * P2;
    for (int i = tid; i < P; i += blockDim.x) {
      p[i] = make_float2(T.d0h[i], T.d0l[i]);
      p[P + i] = make_float2(T.d1h[i], T.d1l[i]);
      p[2 * P + i] = make_float2(T.wh[i], T.wl[i]);
    }
  }
  __syncthreads();
  const int gx0 = a.g[0], gy0 = a.g[1];
  const int col = a.col + rr;
  // Cartesian quadrature weights times |K|/h_d^2 for this thread's (x, y)
  df wg[3];
  if constexpr (!CURVED) {
    const df wab = f2df(t.w[ta]) * f2df(t.w[tb]);
#pragma unroll
    for (int d = 0; d < 3; ++d) wg[d] = wab * a.gs[d];
  }

  for (int cbase = blockIdx.x * cpb; cbase < a.ncells;
       cbase += gridDim.x * cpb) {
    const int cell = cbase + lc;
    const bool active = item_ok && cell < a.ncells;
    const int cc = active ? cell : 0;
    const int cx = cc % a.n[0];
    const int cy = (cc / a.n[0]) % a.n[1];
    const int cz = cc / (a.n[0] * a.n[1]);
    float rh[P], rl[P], oh[P], ol[P];
    // ---- gather the z-line (x = ta, y = tb), float64 -> double-float
    if constexpr (DG) {
#pragma unroll
      for (int z = 0; z < P; ++z) {
        const size_t gi = (size_t)cc * P3 + dx3<P>(ta, tb, z);
        const df u = df_from_double(active ? a.src[gi * a.stride + col] : 0.0);
        rh[z] = u.h;
        rl[z] = u.l;
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
        const df u = df_from_double((active && !con)
                                        ? a.src[gi * a.stride + col]
                                        : 0.0);
        rh[z] = u.h;
        rl[z] = u.l;
      }
    }
    // ---- values at Gauss points: S along z, y, x (one copy of the sweep
    // code for p >= 4: line (base, stride) of the thread per direction)
    if constexpr (P >= 4) {
#pragma unroll
      for (int j = 0; j < P; ++j)
        A[dx3<P>(ta, tb, j)] = make_float2(rh[j], rl[j]);
#pragma unroll 1
      for (int d = 2; d >= 0; --d) {
        const int b0 = d == 2   ? dx3<P>(ta, tb, 0)
                       : d == 1 ? dx3<P>(ta, 0, tb)
                                : dx3<P>(0, ta, tb);
        const int st = d == 2 ? P2 : (d == 1 ? P : 1);
        if (d < 2) __syncthreads();
        dline<P>(A, b0, st, rh, rl);
        dsweep<P, DF_S, false, false>(rh, rl, A, b0, st);
      }
    } else {
      dsweep<P, DF_S, false, false>(rh, rl, A, dx3<P>(ta, tb, 0), P2);
      __syncthreads();
      dline<P>(A, dx3<P>(ta, 0, tb), P, rh, rl);
      dsweep<P, DF_S, false, false>(rh, rl, A, dx3<P>(ta, 0, tb), P);
      __syncthreads();
      dline<P>(A, dx3<P>(0, ta, tb), 1, rh, rl);
      dsweep<P, DF_S, false, false>(rh, rl, A, dx3<P>(0, ta, tb), 1);
    }
    dline<P>(A, dx3<P>(0, ta, tb), 1, rh, rl);  // own line
    if constexpr (DG) {  // values at the Gauss points for the face terms
#pragma unroll
      for (int j = 0; j < P; ++j) {
        U[dx3<P>(j, ta, tb)] = make_float2(rh[j], rl[j]);
      }
    }
    dsweep<P, DF_D, false, false>(rh, rl, X, dx3<P>(0, ta, tb), 1);
    __syncthreads();
    // ---- reference gradient: y into GY, z kept in registers
    dline<P>(A, dx3<P>(ta, 0, tb), P, rh, rl);
    dsweep<P, DF_D, false, false>(rh, rl, Y, dx3<P>(ta, 0, tb), P);
    dline<P>(A, dx3<P>(ta, tb, 0), P2, rh, rl);  // z-line of values
    __syncthreads();
    // ---- quadrature-point operation t = kappa G_q grad u (Eq. 12), the z
    // derivative taken at each point from the z-line in registers
    {
      MFP_DF_LOOP
      for (int qz = 0; qz < P; ++qz) {
        const int q = dx3<P>(ta, tb, qz);
        dacc dz = acc_first(tdh<P, DF_D>(qz * P), tdl<P, DF_D>(qz * P), rh[0],
                            rl[0]);
#pragma unroll
        for (int j = 1; j < P; ++j)
          acc_mac(dz, tdh<P, DF_D>(qz * P + j), tdl<P, DF_D>(qz * P + j),
                  rh[j], rl[j]);
        const df ux = f2df(X[q]), uy = f2df(Y[q]), uz = acc_get(dz);
        df tx, ty, tz;
        if constexpr (CURVED) {
          const size_t gb = (size_t)cc * 6 * P3 + q;
          const df g0 = ld(a.Gh, a.Gl, gb), g1 = ld(a.Gh, a.Gl, gb + P3),
                   g2 = ld(a.Gh, a.Gl, gb + 2 * P3),
                   g3 = ld(a.Gh, a.Gl, gb + 3 * P3),
                   g4 = ld(a.Gh, a.Gl, gb + 4 * P3),
                   g5 = ld(a.Gh, a.Gl, gb + 5 * P3);
          dacc sx = acc_first(g0.h, g0.l, ux.h, ux.l);
          acc_mac(sx, g1.h, g1.l, uy.h, uy.l);
          acc_mac(sx, g2.h, g2.l, uz.h, uz.l);
          dacc sy = acc_first(g1.h, g1.l, ux.h, ux.l);
          acc_mac(sy, g3.h, g3.l, uy.h, uy.l);
          acc_mac(sy, g4.h, g4.l, uz.h, uz.l);
          dacc sz = acc_first(g2.h, g2.l, ux.h, ux.l);
          acc_mac(sz, g4.h, g4.l, uy.h, uy.l);
          acc_mac(sz, g5.h, g5.l, uz.h, uz.l);
          tx = acc_get(sx);
          ty = acc_get(sy);
          tz = acc_get(sz);
        } else {
          const df wz = f2df(t.w[qz]);
          tx = (wg[0] * wz) * ux;
          ty = (wg[1] * wz) * uy;
          tz = (wg[2] * wz) * uz;
        }
        if (a.kch) {
          const df kap = ld(a.kch, a.kcl, (size_t)cc * P3 + q);
          tx = kap * tx;
          ty = kap * ty;
          tz = kap * tz;
        } else if (!a.kappa_one) {
          tx = a.kappa * tx;
          ty = a.kappa * ty;
          tz = a.kappa * tz;
        }
        st2(X, q, tx);
        st2(Y, q, ty);
        st2(A, q, tz);
      }
      dline<P>(A, dx3<P>(ta, tb, 0), P2, rh, rl);  // own z-line
      dsweep<P, DF_D, true, false>(rh, rl, A, dx3<P>(ta, tb, 0), P2);
    }
    __syncthreads();
    // ---- transposed derivative y (added), x (added) then S^T x, y, z
    dline<P>(Y, dx3<P>(ta, 0, tb), P, rh, rl);
    dsweep<P, DF_D, true, true>(rh, rl, A, dx3<P>(ta, 0, tb), P);
    __syncthreads();
    dline<P>(X, dx3<P>(0, ta, tb), 1, rh, rl);
    dsweep<P, DF_D, true, true>(rh, rl, A, dx3<P>(0, ta, tb), 1);
    if constexpr (DG) {
      // ---- SIPG face terms (Eq. 6, Eq. 7), added at the Gauss points
      __syncthreads();
#pragma unroll 1
      for (int D = 0; D < 3; ++D) {
        // lower faces only where a cell of the block lies on the boundary
        const int cD = D == 0 ? cx : (D == 1 ? cy : cz);
        if (!((a.neumann >> (2 * D)) & 1) &&
            __syncthreads_or(active && cD == 0))
          df_face_lower_gp<P, CURVED>(a, col, D, active, cx, cy, cz, U, A, FS,
                                      tabs, ta, tb);
        df_face_gp<P, CURVED, 1>(a, col, D, active, cx, cy, cz, U, A, FS, t,
                                 ta, tb);
      }
      __syncthreads();
    }
    // ---- S^T along x, y (and z for SIPG), one copy of the sweep for p >= 4
    if constexpr (P >= 4) {
#pragma unroll 1
      for (int d = 0; d < (DG ? 3 : 2); ++d) {
        const int b0 = d == 0   ? dx3<P>(0, ta, tb)
                       : d == 1 ? dx3<P>(ta, 0, tb)
                                : dx3<P>(ta, tb, 0);
        const int st = d == 0 ? 1 : (d == 1 ? P : P2);
        if (d > 0) __syncthreads();
        dline<P>(A, b0, st, rh, rl);
        dsweep<P, DF_S, true, false>(rh, rl, A, b0, st);
      }
      if constexpr (!DG) {
        __syncthreads();
        dline<P>(A, dx3<P>(ta, tb, 0), P2, rh, rl);
      }
    } else {
      dline<P>(A, dx3<P>(0, ta, tb), 1, rh, rl);  // own line
      dsweep<P, DF_S, true, false>(rh, rl, A, dx3<P>(0, ta, tb), 1);
      __syncthreads();
      dline<P>(A, dx3<P>(ta, 0, tb), P, rh, rl);
      dsweep<P, DF_S, true, false>(rh, rl, A, dx3<P>(ta, 0, tb), P);
      __syncthreads();
      dline<P>(A, dx3<P>(ta, tb, 0), P2, rh, rl);
      if constexpr (DG)
        dsweep<P, DF_S, true, false>(rh, rl, A, dx3<P>(ta, tb, 0), P2);
    }
    // ---- S^T along z and scatter (float64)
    if constexpr (!DG) {
      dmtv<P, DF_S>(rh, rl, oh, ol);
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
            a.dst[gi] = a.src[gi];
          else
            atomicAdd(a.dst + gi, df_to_double(df_make(oh[z], ol[z])));
        }
      }
      __syncthreads();
    } else {
      if (active) {
#pragma unroll
        for (int z = 0; z < P; ++z) {
          const size_t gi = (size_t)cc * P3 + dx3<P>(ta, tb, z);
          a.dst[gi * a.stride + col] =
              df_to_double(f2df(A[dx3<P>(ta, tb, z)]));
        }
      }
      __syncthreads();
    }
  }
}

// SIPG with each interior face evaluated once: adds the terms that the
// cell below each interior face left for the cell above it (face buffer
// slots 2D: value part at the face nodes, 2D+1: normal-slope part).  The
// value part enters the face layer l = 0 along D, the slope part every
// layer with the weight dphi_l(0) of the reference normal derivative.
template <int P>
__global__ void __launch_bounds__(256) k_dg_face_add(const ApplyArgsDF a) {
  constexpr int P2 = P * P, P3 = P2 * P;
  // one thread per node (cell, x, y, z) of a row of cells (cy, cz) =
  // blockIdx.y, column blockIdx.z; the face buffer slots of a cell are read
  // by its p^3 threads (cached)
  const int R = a.stride, col = blockIdx.z;
  const float* d0h = c_tabdf[P - 2].d0h;
  const float* d0l = c_tabdf[P - 2].d0l;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n[0] * P3) return;
  const int cx = t / P3, loc = t - cx * P3;
  const int x = loc % P, y = (loc / P) % P, z = loc / P2;
  const int mode = a.epi.mode;
  const float2 f0 = make_float2(0.f, 0.f);
  const int rows = a.n[1] * a.n[2];
  // the inputs of one node: the cell-kernel result, the face-buffer terms of
  // the lower faces inside the mesh, the fused update's inputs
  struct In {
    size_t gi;
    int cx, cy, cz;
    double u, eb, edi, ex, ed;
    float2 gx, vx, gy, vy, gz, vz;
  };
  auto load = [&](int row) {
    In v;
    v.cx = cx;
    v.cy = row % a.n[1];
    v.cz = row / a.n[1];
    const size_t cell = (size_t)row * a.n[0] + cx;
    const size_t i = cell * P3 + loc;
    const float2* fb = a.fb + cell * 6 * P2 * R + col;
    v.gi = i * R + col;
    v.u = a.dst[v.gi];
    v.gx = v.cx > 0 ? fb[(size_t)(1 * P2 + y + P * z) * R] : f0;
    v.vx = v.cx > 0 && x == 0 ? fb[(size_t)(0 * P2 + y + P * z) * R] : f0;
    v.gy = v.cy > 0 ? fb[(size_t)(3 * P2 + x + P * z) * R] : f0;
    v.vy = v.cy > 0 && y == 0 ? fb[(size_t)(2 * P2 + x + P * z) * R] : f0;
    v.gz = v.cz > 0 ? fb[(size_t)(5 * P2 + x + P * y) * R] : f0;
    v.vz = v.cz > 0 && z == 0 ? fb[(size_t)(4 * P2 + x + P * y) * R] : f0;
    v.eb = mode != EPI_STORE ? a.epi.b[v.gi] : 0.0;
    v.edi = mode >= EPI_CHEB_FIRST ? a.epi.dinv[i] : 0.0;
    v.ex = mode >= EPI_CHEB_FIRST ? a.epi.x[v.gi] : 0.0;
    v.ed = mode == EPI_CHEB_STEP ? a.epi.d[v.gi] : 0.0;
    return v;
  };
  // the slope part on every layer along the face normal (weight dphi_l(0)),
  // the value part on layer 0; then the update
  auto finish = [&](const In& v) {
    const df uz = df_from_double(v.u);
    dacc s;
    s.h = uz.h;
    s.l = uz.l;
    if (v.cx > 0) {
      acc_mac(s, d0h[x], d0l[x], v.gx.x, v.gx.y);
      if (x == 0) acc_add(s, df_make(v.vx.x, v.vx.y));
    }
    if (v.cy > 0) {
      acc_mac(s, d0h[y], d0l[y], v.gy.x, v.gy.y);
      if (y == 0) acc_add(s, df_make(v.vy.x, v.vy.y));
    }
    if (v.cz > 0) {
      acc_mac(s, d0h[z], d0l[z], v.gz.x, v.gz.y);
      if (z == 0) acc_add(s, df_make(v.vz.x, v.vz.y));
    }
    epi_finish_df(a, v.gi, acc_get(s), v.eb, v.edi, v.ed, v.ex);
  };
  // two rows per iteration, every load of both first
  for (int row = blockIdx.y; row < rows; row += 2 * gridDim.y) {
    const int row2 = row + gridDim.y;
    const In v0 = load(row);
    In v1;
    if (row2 < rows) v1 = load(row2);
    finish(v0);
    if (row2 < rows) finish(v1);
  }
}

template <int P, bool DG>
size_t df_smem_bytes(int cpb, int ncols) {
  return ((size_t)(cpb * ncols + 1) * df_cell_pairs<P, DG>() +
          df_table_pairs<P>()) *
         sizeof(float2);
}

// Resident blocks per SM of a launch shape (cached per shape).
template <int P, bool DG, bool CURVED>
int df_blocks_per_sm(int cpb, int ncols) {
  static std::mutex mu;
  static int cache[64][4] = {};
  constexpr int P2 = P * P;
  const int threads = ((cpb * ncols * P2 + 31) / 32) * 32;
  const size_t smem = df_smem_bytes<P, DG>(cpb, ncols);
  const bool cacheable = ncols == 1 && cpb < 64;
  int dev = 0;
  MFP_CHECK_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(mu);
    if (cacheable && dev < 4 && cache[cpb][dev]) return cache[cpb][dev];
  }
  auto kern = k_apply_df<P, DG, CURVED>;
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

template <int P, bool DG, bool CURVED>
void run_apply_df(ApplyArgsDF a, int cpb, int ncols, cudaStream_t s) {
  constexpr int P2 = P * P;
  a.cpb = cpb;
  a.ncols = ncols;
  const int threads = ((cpb * ncols * P2 + 31) / 32) * 32;
  const size_t smem = df_smem_bytes<P, DG>(cpb, ncols);
  auto kern = k_apply_df<P, DG, CURVED>;
  const int per_sm = df_blocks_per_sm<P, DG, CURVED>(cpb, ncols);
  if (smem > 48 * 1024)
    MFP_CHECK_CUDA(cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MFP_REQUIRE(per_sm >= 1,
              "apply launch shape does not fit on an SM (cells per block too "
              "large for the registers or shared memory)");
  // one block per group of cells (the kernel's loop over groups then runs
  // once): short-lived blocks let the block scheduler interleave the kernels
  // of concurrent solves (the FP64 bench step measured 62.8 -> 60.6 ms
  // against a grid of resident blocks looping over the groups)
  const int64_t need = (a.ncells + cpb - 1) / cpb;
  const int grid = (int)need;
  if (grid <= 0) return;
  kern<<<grid, threads, smem, s>>>(a);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}

inline int default_cpb_df(int p) {
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

template <int P, bool DG, bool CURVED>
void run_apply_df_cols(const ApplyArgsDF& a0, int R, int cells_req,
                       cudaStream_t s) {
  constexpr int P2 = P * P;
  // block size limit of this kernel given its registers
  cudaFuncAttributes fa;
  MFP_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_apply_df<P, DG, CURVED>));
  const int maxthr = fa.maxThreadsPerBlock > 0 ? fa.maxThreadsPerBlock : 1024;
  const int maxcols = maxthr / P2 > 0 ? maxthr / P2 : 1;
  for (int c0 = 0; c0 < R; c0 += maxcols) {
    const int nc = R - c0 < maxcols ? R - c0 : maxcols;
    int cells = cells_req > 0 ? cells_req : default_cpb_df(P) / nc;
    if (cells < 1) cells = 1;
    while (cells > 1 && cells * nc * P2 > maxthr) --cells;
    ApplyArgsDF a = a0;
    a.col = c0;
    run_apply_df<P, DG, CURVED>(a, cells, nc, s);
  }
  if constexpr (DG) {
    MFP_REQUIRE(a0.fb, "SIPG face buffer missing");
    const int threads = 256;
    const int bx = (a0.n[0] * P2 * P + threads - 1) / threads;
    const int rows = (a0.n[1] * a0.n[2] + 1) / 2;  // two rows per block
    const int by = rows < 65535 ? rows : 65535;
    if (a0.ncells > 0) {
      k_dg_face_add<P><<<dim3(bx, by, R), threads, 0, s>>>(a0);
      MFP_CHECK_CUDA(cudaGetLastError());
      note_launch();
    }
  }
}

inline df host_df(double v) {
  df r;
  r.h = (float)v;
  r.l = (float)(v - (double)r.h);
  return r;
}

inline ApplyArgsDF make_apply_args_df(const Level& L, const double* src,
                                      double* dst) {
  ApplyArgsDF a{};
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
  const LevelDF& D = L.ddf;
  a.Gh = D.Gh;
  a.Gl = D.Gl;
  a.kch = D.kch;
  a.kcl = D.kcl;
  a.kfh = D.kfh;
  a.kfl = D.kfl;
  a.fdh = D.fdh;
  a.fdl = D.fdl;
  a.sgh = D.sgh;
  a.sgl = D.sgl;
  a.fb = static_cast<float2*>(L.fbuf);
  a.kappa = host_df(L.kappa);
  a.kappa_one = L.kappa == 1.0;
  const double vol = L.h[0] * L.h[1] * L.h[2];
  const double pen = L.penalty * (double)L.p * L.p;
  for (int d = 0; d < 3; ++d) {
    a.gs[d] = host_df(vol / (L.h[d] * L.h[d]));
    a.ns[d] = host_df(1.0 / L.h[d]);
    a.fa[d] = host_df(vol / L.h[d]);
    a.sg[d] = host_df(pen / L.h[d]);
  }
  a.stride = 1;
  a.col = 0;
  a.cpb = 1;
  a.ncols = 1;
  return a;
}

}  // namespace
}  // namespace mfp
