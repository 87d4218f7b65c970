// FP64-accurate operator evaluation on the FP32 pipes (double-float).
//
// The same sum-factorized cell integral (Sec. 3, Eq. 12) and SIPG face terms
// (Eq. 6, Eq. 7) as k_apply.cuh, with float64 vectors in HBM and every
// intermediate carried as a double-float pair (df.cuh).  On GB300 the FP64
// pipe issues 2 DFMA per clock per SM while the FP32 pipe issues 128 FFMA;
// a double-float multiply-add costs 11 FP32 instructions, so the FP32 pipe
// delivers about 5x the FP64 rate at about 48 significant bits.  Only the
// conversions of the float64 inputs and outputs use the FP64 pipe.
#pragma once

#include "dev_tables.cuh"
#include "df.cuh"

// Resident 128-thread blocks per SM the register allocation must allow:
// CG gains from more warps (latency of the gather and geometry loads), SIPG
// from more registers (its face code spills below 128 per thread); measured
// on 32^3 Q3/Q4 Cartesian and curved meshes.
#ifndef MFP_DF_MIN_BLOCKS_CG
#define MFP_DF_MIN_BLOCKS_CG 8
#endif
#ifndef MFP_DF_MIN_BLOCKS_DG
#define MFP_DF_MIN_BLOCKS_DG 4
#endif

namespace mfp {
namespace {

struct ApplyArgsDF {
  const double* __restrict__ src;
  double* __restrict__ dst;
  int n[3];
  int ncells;
  int g[3];
  int face_off[3];
  const float *Gh, *Gl;      // curved: [cell][6][p^3]
  const float *kch, *kcl;    // [cell][p^3] or null
  const float *kfh, *kfl;    // [face][p^2] or null
  const float *fdh, *fdl;    // curved SIPG: [face][7][p^2]
  const float *sgh, *sgl;    // curved SIPG: [face]
  df kappa;
  bool kappa_one;            // constant coefficient exactly 1
  df gs[3], ns[3], fa[3], sg[3];
  int stride, col, cpb, ncols;
};

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

// out[q] = sum_j M[q][j] in[j]
template <int P, int W>
__device__ __forceinline__ void dmv(const float (&ih)[P], const float (&il)[P],
                                    float (&oh)[P], float (&ol)[P]) {
#pragma unroll
  for (int q = 0; q < P; ++q) {
    dacc s = acc_first(tdh<P, W>(q * P), tdl<P, W>(q * P), ih[0], il[0]);
#pragma unroll
    for (int j = 1; j < P; ++j)
      acc_mac(s, tdh<P, W>(q * P + j), tdl<P, W>(q * P + j), ih[j], il[j]);
    const df r = acc_get(s);
    oh[q] = r.h;
    ol[q] = r.l;
  }
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

template <int P>
__device__ __forceinline__ int dx3(int x, int y, int z) {
  return x + P * (y + P * z);
}
template <int P, int D>
__device__ __forceinline__ int dfnode(int l, int a, int b) {
  if constexpr (D == 0) return l + P * (a + P * b);
  if constexpr (D == 1) return a + P * (l + P * b);
  return a + P * (b + P * l);
}

// odd stride: the columns of a batch fall into distinct shared-memory banks
template <int P, bool DG>
__host__ __device__ constexpr int df_cell_floats() {
  return ((DG ? 8 : 6) * P * P * P + (DG ? 16 * P * P : 0)) | 1;
}
template <int P>
__host__ __device__ constexpr int df_table_floats() {
  return 4 * P * P + 6 * P;
}

// shared DF table views (row-major p x p)
struct ShDF {
  const float *Sh, *Sl, *Dh, *Dl, *d0h, *d0l, *d1h, *d1l, *wh, *wl;
};

__device__ __forceinline__ df ld(const float* h, const float* l, int i) {
  return df_make(h[i], l[i]);
}
__device__ __forceinline__ void stv(float* h, float* l, int i, df v) {
  h[i] = v.h;
  l[i] = v.l;
}

// One face of the own cell (axis D, side S), double-float version of
// face_contrib in k_apply.cuh.  FS holds 8 hi arrays then 8 lo arrays.
template <int P, bool CURVED, int D, int S>
__device__ __forceinline__ void df_face(const ApplyArgsDF& a, bool active,
                                        int cx, int cy, int cz,
                                        const float* Uh, const float* Ul,
                                        float* Ah, float* Al, float* FSh,
                                        float* FSl, const ShDF& t, int ta,
                                        int tb) {
  constexpr int P2 = P * P, P3 = P2 * P;
  constexpr int T1 = D == 0 ? 1 : 0;
  constexpr int T2 = D == 2 ? 1 : 2;
  const int ti = ta + P * tb;
  int m[3] = {a.n[0], a.n[1], a.n[2]};
  m[D] += 1;
  int fc[3] = {cx, cy, cz};
  fc[D] += S;
  const int f = a.face_off[D] + fc[0] + m[0] * (fc[1] + m[1] * fc[2]);
  int nbc[3] = {cx, cy, cz};
  nbc[D] += S ? 1 : -1;
  const bool bnd = nbc[D] < 0 || nbc[D] >= a.n[D];
  const int nb = bnd ? 0 : nbc[0] + a.n[0] * (nbc[1] + a.n[1] * nbc[2]);
  const float* dSh = S ? t.d1h : t.d0h;
  const float* dSl = S ? t.d1l : t.d0l;
  const float* dNh = S ? t.d0h : t.d1h;
  const float* dNl = S ? t.d0l : t.d1l;
  constexpr int lo = S ? P - 1 : 0;
  constexpr int ln = S ? 0 : P - 1;
  // F1: nodal face values and reference normal slopes of both sides
  {
    const df vo = ld(Uh, Ul, dfnode<P, D>(lo, ta, tb));
    dacc so = acc_first(dSh[0], dSl[0], Uh[dfnode<P, D>(0, ta, tb)],
                        Ul[dfnode<P, D>(0, ta, tb)]);
#pragma unroll
    for (int l = 1; l < P; ++l)
      acc_mac(so, dSh[l], dSl[l], Uh[dfnode<P, D>(l, ta, tb)],
              Ul[dfnode<P, D>(l, ta, tb)]);
    df vn = df_make(0.f), dnn = df_make(0.f);
    if (!bnd && active) {
      const size_t cb = (size_t)nb * P3;
      dacc sn;
      sn.h = 0.f;
      sn.l = 0.f;
#pragma unroll
      for (int l = 0; l < P; ++l) {
        const df u = df_from_double(
            a.src[(cb + dfnode<P, D>(l, ta, tb)) * a.stride + a.col]);
        if (l == 0)
          sn = acc_first(dNh[0], dNl[0], u.h, u.l);
        else
          acc_mac(sn, dNh[l], dNl[l], u.h, u.l);
        if (l == ln) vn = u;
      }
      dnn = acc_get(sn);
    }
    stv(FSh, FSl, 0 * P2 + ti, vo);
    stv(FSh, FSl, 1 * P2 + ti, acc_get(so));
    stv(FSh, FSl, 2 * P2 + ti, vn);
    stv(FSh, FSl, 3 * P2 + ti, dnn);
  }
  __syncthreads();
  // F2: interpolate along the first tangential axis
#pragma unroll
  for (int arr = 0; arr < 4; ++arr) {
    dacc s = acc_first(t.Sh[ta * P], t.Sl[ta * P], FSh[arr * P2 + P * tb],
                       FSl[arr * P2 + P * tb]);
#pragma unroll
    for (int j = 1; j < P; ++j)
      acc_mac(s, t.Sh[ta * P + j], t.Sl[ta * P + j],
              FSh[arr * P2 + j + P * tb], FSl[arr * P2 + j + P * tb]);
    stv(FSh, FSl, (4 + arr) * P2 + ti, acc_get(s));
  }
  __syncthreads();
  // F3: along the second tangential axis
  df q[4];
#pragma unroll
  for (int arr = 0; arr < 4; ++arr) {
    dacc s = acc_first(t.Sh[tb * P], t.Sl[tb * P], FSh[(4 + arr) * P2 + ta],
                       FSl[(4 + arr) * P2 + ta]);
#pragma unroll
    for (int j = 1; j < P; ++j)
      acc_mac(s, t.Sh[tb * P + j], t.Sl[tb * P + j],
              FSh[(4 + arr) * P2 + ta + P * j],
              FSl[(4 + arr) * P2 + ta + P * j]);
    q[arr] = acc_get(s);
  }
  __syncthreads();
  if constexpr (CURVED) {
    stv(FSh, FSl, 0 * P2 + ti, q[0]);
    stv(FSh, FSl, 2 * P2 + ti, q[2]);
    __syncthreads();
  }
  {
    const df kap = a.kfh ? df_make(a.kfh[(size_t)f * P2 + ti],
                                   a.kfl[(size_t)f * P2 + ti])
                         : a.kappa;
    df uo = q[0], un = q[2], dno, dnn, dA, sig;
    df gvec[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
    if constexpr (!CURVED) {
      const float sgn = S ? 1.f : -1.f;
      const df w2 = df_make(t.wh[ta], t.wl[ta]) * df_make(t.wh[tb], t.wl[tb]);
      dA = w2 * a.fa[D];
      sig = a.sg[D];
      const df nsc = df_make(sgn * a.ns[D].h, sgn * a.ns[D].l);
      dno = nsc * q[1];
      dnn = bnd ? dno : nsc * q[3];
      gvec[D] = nsc;
    } else {
      const size_t fb = (size_t)f * 7 * P2;
      dA = ld(a.fdh, a.fdl, fb + ti);
      sig = df_make(a.sgh[f], a.sgl[f]);
      df go[3], gn[3];
      go[D] = q[1];
      gn[D] = q[3];
      dacc s1o = acc_first(t.Dh[ta * P], t.Dl[ta * P], FSh[P * tb],
                           FSl[P * tb]);
      dacc s2o = acc_first(t.Dh[tb * P], t.Dl[tb * P], FSh[ta], FSl[ta]);
      dacc s1n = acc_first(t.Dh[ta * P], t.Dl[ta * P], FSh[2 * P2 + P * tb],
                           FSl[2 * P2 + P * tb]);
      dacc s2n = acc_first(t.Dh[tb * P], t.Dl[tb * P], FSh[2 * P2 + ta],
                           FSl[2 * P2 + ta]);
#pragma unroll
      for (int j = 1; j < P; ++j) {
        acc_mac(s1o, t.Dh[ta * P + j], t.Dl[ta * P + j], FSh[j + P * tb],
                FSl[j + P * tb]);
        acc_mac(s2o, t.Dh[tb * P + j], t.Dl[tb * P + j], FSh[ta + P * j],
                FSl[ta + P * j]);
        acc_mac(s1n, t.Dh[ta * P + j], t.Dl[ta * P + j],
                FSh[2 * P2 + j + P * tb], FSl[2 * P2 + j + P * tb]);
        acc_mac(s2n, t.Dh[tb * P + j], t.Dl[tb * P + j],
                FSh[2 * P2 + ta + P * j], FSl[2 * P2 + ta + P * j]);
      }
      go[T1] = acc_get(s1o);
      go[T2] = acc_get(s2o);
      gn[T1] = acc_get(s1n);
      gn[T2] = acc_get(s2n);
      df nL[3], nR[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        nL[e] = ld(a.fdh, a.fdl, fb + (1 + e) * P2 + ti);
        nR[e] = ld(a.fdh, a.fdl, fb + (4 + e) * P2 + ti);
      }
      if constexpr (S == 1) {  // own cell is the left one: outward = +n
        dacc so = acc_first(nL[0].h, nL[0].l, go[0].h, go[0].l);
        acc_mac(so, nL[1].h, nL[1].l, go[1].h, go[1].l);
        acc_mac(so, nL[2].h, nL[2].l, go[2].h, go[2].l);
        dacc sn = acc_first(nR[0].h, nR[0].l, gn[0].h, gn[0].l);
        acc_mac(sn, nR[1].h, nR[1].l, gn[1].h, gn[1].l);
        acc_mac(sn, nR[2].h, nR[2].l, gn[2].h, gn[2].l);
        dno = acc_get(so);
        dnn = acc_get(sn);
#pragma unroll
        for (int e = 0; e < 3; ++e) gvec[e] = nL[e];
      } else {  // own cell is the right one: outward = -n
        dacc so = acc_first(nR[0].h, nR[0].l, go[0].h, go[0].l);
        acc_mac(so, nR[1].h, nR[1].l, go[1].h, go[1].l);
        acc_mac(so, nR[2].h, nR[2].l, go[2].h, go[2].l);
        dacc sn = acc_first(nL[0].h, nL[0].l, gn[0].h, gn[0].l);
        acc_mac(sn, nL[1].h, nL[1].l, gn[1].h, gn[1].l);
        acc_mac(sn, nL[2].h, nL[2].l, gn[2].h, gn[2].l);
        dno = -acc_get(so);
        dnn = -acc_get(sn);
#pragma unroll
        for (int e = 0; e < 3; ++e) gvec[e] = -nR[e];
      }
      if (bnd) dnn = dno;
    }
    if (bnd) un = -uo;  // mirror state (Eq. 7)
    const df kdA = kap * dA;
    const df jump = uo - un;
    const df avg = df_scale2(dno + dnn, 0.5f);
    const df cv = kdA * (sig * jump - avg);
    const df cg = df_scale2(kdA * jump, -0.5f);
    stv(FSh, FSl, 4 * P2 + ti, cv);
    stv(FSh, FSl, 5 * P2 + ti, cg * gvec[D]);
    if constexpr (CURVED) {
      stv(FSh, FSl, 6 * P2 + ti, cg * gvec[T1]);
      stv(FSh, FSl, 7 * P2 + ti, cg * gvec[T2]);
    }
  }
  __syncthreads();
  {
    dacc vq;
    vq.h = FSh[4 * P2 + ti];
    vq.l = FSl[4 * P2 + ti];
    if constexpr (CURVED) {
#pragma unroll
      for (int j = 0; j < P; ++j) {
        acc_mac(vq, t.Dh[j * P + ta], t.Dl[j * P + ta], FSh[6 * P2 + j + P * tb],
                FSl[6 * P2 + j + P * tb]);
        acc_mac(vq, t.Dh[j * P + tb], t.Dl[j * P + tb],
                FSh[7 * P2 + ta + P * j], FSl[7 * P2 + ta + P * j]);
      }
    }
    const df v = acc_get(vq);
    const df g5 = ld(FSh, FSl, 5 * P2 + ti);
    __syncthreads();
    stv(FSh, FSl, 0 * P2 + ti, v);
    stv(FSh, FSl, 1 * P2 + ti, g5);
  }
  __syncthreads();
  // S^T along a
#pragma unroll
  for (int arr = 0; arr < 2; ++arr) {
    dacc s = acc_first(t.Sh[ta], t.Sl[ta], FSh[arr * P2 + P * tb],
                       FSl[arr * P2 + P * tb]);
#pragma unroll
    for (int j = 1; j < P; ++j)
      acc_mac(s, t.Sh[j * P + ta], t.Sl[j * P + ta], FSh[arr * P2 + j + P * tb],
              FSl[arr * P2 + j + P * tb]);
    stv(FSh, FSl, (2 + arr) * P2 + ti, acc_get(s));
  }
  __syncthreads();
  // S^T along b and distribution onto the own nodes of line (ta, tb)
  {
    dacc sv = acc_first(t.Sh[tb], t.Sl[tb], FSh[2 * P2 + ta], FSl[2 * P2 + ta]);
    dacc sn = acc_first(t.Sh[tb], t.Sl[tb], FSh[3 * P2 + ta], FSl[3 * P2 + ta]);
#pragma unroll
    for (int j = 1; j < P; ++j) {
      acc_mac(sv, t.Sh[j * P + tb], t.Sl[j * P + tb], FSh[2 * P2 + ta + P * j],
              FSl[2 * P2 + ta + P * j]);
      acc_mac(sn, t.Sh[j * P + tb], t.Sl[j * P + tb], FSh[3 * P2 + ta + P * j],
              FSl[3 * P2 + ta + P * j]);
    }
    const df vf = acc_get(sv), nf = acc_get(sn);
    {
      const int i = dfnode<P, D>(lo, ta, tb);
      stv(Ah, Al, i, ld(Ah, Al, i) + vf);
    }
#pragma unroll
    for (int l = 0; l < P; ++l) {
      const int i = dfnode<P, D>(l, ta, tb);
      stv(Ah, Al, i, ld(Ah, Al, i) + df_make(dSh[l], dSl[l]) * nf);
    }
  }
  __syncthreads();
}

// Register budget: enough resident warps to hide the load latency
// (blocks of at most 128 threads for p <= 5, 256 above).
template <int P>
constexpr int df_max_threads() { return P <= 5 ? 128 : 256; }
template <int P, bool DG>
constexpr int df_min_blocks() {
  // p >= 6: no cap (the larger line arrays would spill kilobytes)
  return P <= 5 ? (DG ? MFP_DF_MIN_BLOCKS_DG : MFP_DF_MIN_BLOCKS_CG) : 1;
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
    k_apply_df(const ApplyArgsDF a) {
  constexpr int P2 = P * P, P3 = P2 * P;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* sm = reinterpret_cast<float*>(smraw);
  const int cpb = a.cpb, nc = a.ncols;
  const int items = cpb * nc * P2;
  const int tid = threadIdx.x;
  const bool item_ok = tid < items;
  const int rr = tid % nc;
  const int rest = tid / nc;
  const int ta = rest % P, tb = (rest / P) % P;
  const int lc = item_ok ? rest / P2 : 0;
  const int v = item_ok ? lc * nc + rr : cpb * nc;
  float* base = sm + (size_t)v * df_cell_floats<P, DG>();
  float* Ah = base;
  float* Al = base + P3;
  float* Xh = base + 2 * P3;  // GX
  float* Xl = base + 3 * P3;
  float* Yh = base + 4 * P3;  // GY
  float* Yl = base + 5 * P3;
  float* Uh = base + 6 * P3;  // DG nodal input
  float* Ul = base + 7 * P3;
  float* FSh = base + 8 * P3;
  float* FSl = FSh + 8 * P2;
  float* tabs = sm + (size_t)(cpb * nc + 1) * df_cell_floats<P, DG>();
  ShDF t;
  {
    float* p = tabs;
    t.Sh = p; t.Sl = p + P2; t.Dh = p + 2 * P2; t.Dl = p + 3 * P2;
    p += 4 * P2;
    t.d0h = p; t.d0l = p + P; t.d1h = p + 2 * P; t.d1l = p + 3 * P;
    t.wh = p + 4 * P; t.wl = p + 5 * P;
    for (int i = tid; i < P2; i += blockDim.x) {
      tabs[i] = c_tabdf[P - 2].Sh[i];
      tabs[P2 + i] = c_tabdf[P - 2].Sl[i];
      tabs[2 * P2 + i] = c_tabdf[P - 2].Dh[i];
      tabs[3 * P2 + i] = c_tabdf[P - 2].Dl[i];
    }
    for (int i = tid; i < P; i += blockDim.x) {
      p[i] = c_tabdf[P - 2].d0h[i];
      p[P + i] = c_tabdf[P - 2].d0l[i];
      p[2 * P + i] = c_tabdf[P - 2].d1h[i];
      p[3 * P + i] = c_tabdf[P - 2].d1l[i];
      p[4 * P + i] = c_tabdf[P - 2].wh[i];
      p[5 * P + i] = c_tabdf[P - 2].wl[i];
    }
  }
  __syncthreads();
  const int gx0 = a.g[0], gy0 = a.g[1], gz0 = a.g[2];
  ApplyArgsDF ac = a;
  ac.col = a.col + rr;
  // Cartesian quadrature weights times |K|/h_d^2 for this thread's (x, y)
  df wg[3];
  if constexpr (!CURVED) {
    const df wab = ld(t.wh, t.wl, ta) * ld(t.wh, t.wl, tb);
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
    const int col = ac.col;
    float rh[P], rl[P], oh[P], ol[P];
    // ---- gather the z-line (x = ta, y = tb), float64 -> double-float
    if constexpr (DG) {
#pragma unroll
      for (int z = 0; z < P; ++z) {
        const size_t gi = (size_t)cc * P3 + dx3<P>(ta, tb, z);
        const df u = df_from_double(active ? a.src[gi * a.stride + col] : 0.0);
        rh[z] = u.h;
        rl[z] = u.l;
        Uh[dx3<P>(ta, tb, z)] = u.h;
        Ul[dx3<P>(ta, tb, z)] = u.l;
      }
    } else {
      const int X = cx * (P - 1) + ta, Y = cy * (P - 1) + tb;
      const bool bxy = X == 0 || X == gx0 - 1 || Y == 0 || Y == gy0 - 1;
#pragma unroll
      for (int z = 0; z < P; ++z) {
        const int Z = cz * (P - 1) + z;
        const bool con = bxy || Z == 0 || Z == gz0 - 1;
        const size_t gi = (size_t)X + (size_t)gx0 * (Y + (size_t)gy0 * Z);
        const df u = df_from_double((active && !con)
                                        ? a.src[gi * a.stride + col]
                                        : 0.0);
        rh[z] = u.h;
        rl[z] = u.l;
      }
    }
    // ---- values at Gauss points: z (registers), y, x
    dmv<P, DF_S>(rh, rl, oh, ol);
#pragma unroll
    for (int z = 0; z < P; ++z) {
      Ah[dx3<P>(ta, tb, z)] = oh[z];
      Al[dx3<P>(ta, tb, z)] = ol[z];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) {
      rh[j] = Ah[dx3<P>(ta, j, tb)];
      rl[j] = Al[dx3<P>(ta, j, tb)];
    }
    dmv<P, DF_S>(rh, rl, oh, ol);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      Ah[dx3<P>(ta, j, tb)] = oh[j];
      Al[dx3<P>(ta, j, tb)] = ol[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) {
      rh[j] = Ah[dx3<P>(j, ta, tb)];
      rl[j] = Al[dx3<P>(j, ta, tb)];
    }
    dmv<P, DF_S>(rh, rl, oh, ol);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      Ah[dx3<P>(j, ta, tb)] = oh[j];
      Al[dx3<P>(j, ta, tb)] = ol[j];
    }
    dmv<P, DF_D>(oh, ol, rh, rl);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      Xh[dx3<P>(j, ta, tb)] = rh[j];
      Xl[dx3<P>(j, ta, tb)] = rl[j];
    }
    __syncthreads();
    // ---- reference gradient: y into GY, z kept in registers
#pragma unroll
    for (int j = 0; j < P; ++j) {
      rh[j] = Ah[dx3<P>(ta, j, tb)];
      rl[j] = Al[dx3<P>(ta, j, tb)];
    }
    dmv<P, DF_D>(rh, rl, oh, ol);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      Yh[dx3<P>(ta, j, tb)] = oh[j];
      Yl[dx3<P>(ta, j, tb)] = ol[j];
    }
    float gzh[P], gzl[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      rh[j] = Ah[dx3<P>(ta, tb, j)];
      rl[j] = Al[dx3<P>(ta, tb, j)];
    }
    dmv<P, DF_D>(rh, rl, gzh, gzl);
    __syncthreads();
    // ---- quadrature-point operation t = kappa G_q grad u (Eq. 12)
    {
#pragma unroll
      for (int qz = 0; qz < P; ++qz) {
        const int q = dx3<P>(ta, tb, qz);
        const df ux = ld(Xh, Xl, q), uy = ld(Yh, Yl, q),
                 uz = df_make(gzh[qz], gzl[qz]);
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
          const df wz = ld(t.wh, t.wl, qz);
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
        stv(Xh, Xl, q, tx);
        stv(Yh, Yl, q, ty);
        rh[qz] = tz.h;
        rl[qz] = tz.l;
      }
      dmtv<P, DF_D>(rh, rl, oh, ol);
#pragma unroll
      for (int j = 0; j < P; ++j) {
        Ah[dx3<P>(ta, tb, j)] = oh[j];
        Al[dx3<P>(ta, tb, j)] = ol[j];
      }
    }
    __syncthreads();
    // ---- transposed derivative y (added), x (added) then S^T x, y, z
#pragma unroll
    for (int j = 0; j < P; ++j) {
      rh[j] = Yh[dx3<P>(ta, j, tb)];
      rl[j] = Yl[dx3<P>(ta, j, tb)];
    }
    dmtv<P, DF_D>(rh, rl, oh, ol);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int i = dx3<P>(ta, j, tb);
      stv(Ah, Al, i, ld(Ah, Al, i) + df_make(oh[j], ol[j]));
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) {
      rh[j] = Xh[dx3<P>(j, ta, tb)];
      rl[j] = Xl[dx3<P>(j, ta, tb)];
    }
    dmtv<P, DF_D>(rh, rl, oh, ol);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const df s = df_make(oh[j], ol[j]) + ld(Ah, Al, dx3<P>(j, ta, tb));
      oh[j] = s.h;
      ol[j] = s.l;
    }
    dmtv<P, DF_S>(oh, ol, rh, rl);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      Ah[dx3<P>(j, ta, tb)] = rh[j];
      Al[dx3<P>(j, ta, tb)] = rl[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) {
      rh[j] = Ah[dx3<P>(ta, j, tb)];
      rl[j] = Al[dx3<P>(ta, j, tb)];
    }
    dmtv<P, DF_S>(rh, rl, oh, ol);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      Ah[dx3<P>(ta, j, tb)] = oh[j];
      Al[dx3<P>(ta, j, tb)] = ol[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P; ++j) {
      rh[j] = Ah[dx3<P>(ta, tb, j)];
      rl[j] = Al[dx3<P>(ta, tb, j)];
    }
    dmtv<P, DF_S>(rh, rl, oh, ol);
    // ---- scatter (float64)
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
            a.dst[gi] = a.src[gi];
          else
            atomicAdd(a.dst + gi, df_to_double(df_make(oh[z], ol[z])));
        }
      }
      __syncthreads();
    } else {
#pragma unroll
      for (int z = 0; z < P; ++z) {
        Ah[dx3<P>(ta, tb, z)] = oh[z];
        Al[dx3<P>(ta, tb, z)] = ol[z];
      }
      __syncthreads();
      df_face<P, CURVED, 0, 0>(ac, active, cx, cy, cz, Uh, Ul, Ah, Al, FSh,
                               FSl, t, ta, tb);
      df_face<P, CURVED, 0, 1>(ac, active, cx, cy, cz, Uh, Ul, Ah, Al, FSh,
                               FSl, t, ta, tb);
      df_face<P, CURVED, 1, 0>(ac, active, cx, cy, cz, Uh, Ul, Ah, Al, FSh,
                               FSl, t, ta, tb);
      df_face<P, CURVED, 1, 1>(ac, active, cx, cy, cz, Uh, Ul, Ah, Al, FSh,
                               FSl, t, ta, tb);
      df_face<P, CURVED, 2, 0>(ac, active, cx, cy, cz, Uh, Ul, Ah, Al, FSh,
                               FSl, t, ta, tb);
      df_face<P, CURVED, 2, 1>(ac, active, cx, cy, cz, Uh, Ul, Ah, Al, FSh,
                               FSl, t, ta, tb);
      if (active) {
#pragma unroll
        for (int z = 0; z < P; ++z) {
          const size_t gi = (size_t)cc * P3 + dx3<P>(ta, tb, z);
          a.dst[gi * a.stride + col] =
              df_to_double(ld(Ah, Al, dx3<P>(ta, tb, z)));
        }
      }
      __syncthreads();
    }
  }
}

template <int P, bool DG, bool CURVED>
void run_apply_df(ApplyArgsDF a, int cpb, int ncols, cudaStream_t s) {
  constexpr int P2 = P * P;
  a.cpb = cpb;
  a.ncols = ncols;
  const int threads = ((cpb * ncols * P2 + 31) / 32) * 32;
  const size_t smem =
      ((size_t)(cpb * ncols + 1) * df_cell_floats<P, DG>() +
       df_table_floats<P>()) *
      sizeof(float);
  auto kern = k_apply_df<P, DG, CURVED>;
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
    a.face_off[d] = L.face_off[d];
  }
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
