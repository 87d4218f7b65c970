// HDG mixed matrix-free operator (Sec. 3, "HDG mixed matrix-free", on the
// hybridizable DG form of Sec. 2.3):
//   y = ([A B^T; B D] + [C^T; G^T] H^{-1} [C G]) x
// with the cell unknowns (q_x, q_y, q_z, u) in cell-major blocks of 4 p^3
// nodal values (Lagrange in the Gauss-Lobatto points), where
//   A = (w, kappa^-1 q), B^T = -(div w, u), D = -<v, tau u>,
//   C^T = <w . n, lambda>, G^T = <v, tau lambda>, H = sum_sides <mu, tau lambda>.
// The trace is never an unknown: H^{-1} [C G] x is the face trace
//   lambda = sum_sides (q . n + tau u) / sum_sides tau
// at the face Gauss points (H is tau times the face mass in a basis as large
// as the Gauss rule, so its inverse acts point by point; on a curved face
// both sides see the same area element); it is zero on Dirichlet faces,
// whose traces are data.  k_hdg_trace (a few faces per block) forms lambda,
// k_hdg_cell (a few cells per block) adds the cell integrals by sum
// factorization (values at the Gauss points by S, reference derivatives by
// the Gauss collocation matrix D, mapped by J^{-1}) and the six faces' terms
// -<v, tau u> + <w . n, lambda> + <v, tau lambda> on the face-layer nodes.
// tau = tau_factor times the largest coefficient on the face (Sec. 4.2).
// Cartesian cells use their constant Jacobian; curved ones read w det J and
// J^{-1} per cell point and dA and the unit normal per face point.  The
// kernels are generic over the arithmetic: float64 (DFMA) for native-FP64
// contexts, double-float pairs on the FP32 pipes for double-float ones (the
// default), with the vectors float64 either way.
#include "df.cuh"
#include "dev_tables.cuh"

namespace mfp {
namespace {

struct HdgArgs {
  const double* __restrict__ x;
  double* __restrict__ y;
  double* __restrict__ lam;  // [nfaces][p^2] at the face Gauss points
  int n[3];
  int face_off[3];
  int neumann;  // bit 2d + s: side (d, s) has Neumann data
  double h[3];  // physical cell size (Cartesian cells)
  double ih[3];  // 1 / h (host-computed: no float64 divisions per point)
  double vol;    // h_x h_y h_z
  double fa[3];  // area of a face normal to d: h_a h_b
  double kappa;  // constant coefficient (when kcell / kface are null)
  double kinv;   // 1 / kappa
  double tau_factor;
  const double* __restrict__ kcell;  // [cell][p^3] or null
  const double* __restrict__ kface;  // [face][p^2] or null
  const double* __restrict__ gc;     // curved: [cell][10][p^3] or null
  const double* __restrict__ gf;     // curved: [face][4][p^2] or null
};

// tau of face f: tau_factor times the largest coefficient on the face
template <int P>
__device__ __forceinline__ double face_tau(const HdgArgs& a, size_t f) {
  if (!a.kface) return a.tau_factor * a.kappa;
  double m = a.kface[f * P * P];
  for (int q = 1; q < P * P; ++q) m = fmax(m, a.kface[f * P * P + q]);
  return a.tau_factor * m;
}

// Arithmetic of the HDG kernels: V the value type, S its shared-memory
// element, Acc a dot-product accumulator.
template <typename V>
struct HT;
template <>
struct HT<double> {
  using S = double;
  using Acc = double;
  static __device__ __forceinline__ double v(S x) { return x; }
  static __device__ __forceinline__ S s(double x) { return x; }
  static __device__ __forceinline__ double d2v(double x) { return x; }
  static __device__ __forceinline__ double v2d(double x) { return x; }
  static __device__ __forceinline__ Acc zero() { return 0.0; }
  static __device__ __forceinline__ void mac(Acc& a, S m, S x) { a += m * x; }
  static __device__ __forceinline__ double get(const Acc& a) { return a; }
  static __device__ __forceinline__ double recip(double x) { return 1.0 / x; }
};
template <>
struct HT<df> {
  using S = float2;
  using Acc = dacc;
  static __device__ __forceinline__ df v(S x) { return df_make(x.x, x.y); }
  static __device__ __forceinline__ S s(df x) { return make_float2(x.h, x.l); }
  static __device__ __forceinline__ df d2v(double x) {
    return df_from_double(x);
  }
  static __device__ __forceinline__ double v2d(df x) { return df_to_double(x); }
  static __device__ __forceinline__ Acc zero() {
    Acc a;
    a.h = 0.f;
    a.l = 0.f;
    return a;
  }
  static __device__ __forceinline__ void mac(Acc& a, S m, S x) {
    acc_mac(a, m.x, m.y, x.x, x.y);
  }
  static __device__ __forceinline__ df get(const Acc& a) { return acc_get(a); }
  // 1/x: the float reciprocal refined by one Newton step in double-float
  static __device__ __forceinline__ df recip(df x) {
    const df y = df_make(__frcp_rn(x.h));
    return y + y * (df_make(1.f) - x * y);
  }
};

#define HDG_STR2(x) #x
#define HDG_STR(x) HDG_STR2(x)
#define HDG_OUT_LOOP _Pragma(HDG_STR(unroll(P <= 4 ? P : 1)))

// Even-odd split of S or S^T (TR), which are mirror-symmetric
// (M[p-1-q][p-1-j] = M[q][j]): with h = p/2, e_j = x_j + x_{p-1-j} and
// o_j = x_j - x_{p-1-j} (j < h),
//   out_q = A_q + B_q, out_{p-1-q} = A_q - B_q (q < h), out_h = A_h (odd p),
//   A_q = sum_j ae[q][j] e_j + am[q] x_h,  B_q = sum_j bo[q][j] o_j,
// ae = (M[q][j] + M[q][p-1-j]) / 2, bo = (M[q][j] - M[q][p-1-j]) / 2 and
// am = M[q][h] (odd p): the sweep takes (h + p%2)(h + 1) + h^2 multiply-adds
// per line instead of p^2.  Table layout: ae [h + p%2][h], am [h + p%2],
// bo [h][h].
template <int P>
constexpr int eo_elems() {
  return (P / 2 + P % 2) * (P / 2) + (P / 2 + P % 2) + (P / 2) * (P / 2);
}
template <int P, typename V, bool TR>
__device__ __forceinline__ void load_eo(typename HT<V>::S* E) {
  using H = HT<V>;
  constexpr int Hh = P / 2, MC = Hh + P % 2;
  const double* S = c_tab64[P - 2].S;
  auto M = [&](int q, int j) { return TR ? S[j * P + q] : S[q * P + j]; };
  for (int i = threadIdx.x; i < eo_elems<P>(); i += blockDim.x) {
    double v;
    if (i < MC * Hh) {
      const int q = i / Hh, j = i % Hh;
      v = 0.5 * (M(q, j) + M(q, P - 1 - j));
    } else if (i < MC * Hh + MC) {
      v = P % 2 ? M(i - MC * Hh, Hh) : 0.0;
    } else {
      const int r = i - MC * Hh - MC, q = r / Hh, j = r % Hh;
      v = 0.5 * (M(q, j) - M(q, P - 1 - j));
    }
    E[i] = H::s(H::d2v(v));
  }
}

// out = M applied along AXIS of nf fields of p^3 values (M = S or S^T as
// the even-odd table E holds it), one line of p values per thread: its
// inputs are read once into registers and the table entries at fixed
// offsets (broadcast to the warp).
template <int P, typename V, int AXIS>
__device__ void sweep3(const typename HT<V>::S* E,
                       const typename HT<V>::S* in, typename HT<V>::S* out,
                       int nf) {
  using H = HT<V>;
  constexpr int N = P * P * P, P2 = P * P;
  constexpr int Hh = P / 2, MC = Hh + P % 2;
  constexpr int st = AXIS == 0 ? 1 : (AXIS == 1 ? P : P2);
  const typename H::S* am = E + MC * Hh;
  const typename H::S* bo = am + MC;
  for (int l = threadIdx.x; l < nf * P2; l += blockDim.x) {
    const int f = l / P2, r = l - f * P2;
    const int base = f * N + (AXIS == 0 ? P * r
                              : AXIS == 1 ? r % P + P2 * (r / P) : r);
    typename H::S x[P], e[Hh], o[Hh];
#pragma unroll
    for (int j = 0; j < P; ++j) x[j] = in[base + j * st];
#pragma unroll
    for (int j = 0; j < Hh; ++j) {
      const V xa = H::v(x[j]), xb = H::v(x[P - 1 - j]);
      e[j] = H::s(xa + xb);
      o[j] = H::s(xa - xb);
    }
    // unrolled over the outputs up to p = 4 (measured faster than 5)
    HDG_OUT_LOOP
    for (int q = 0; q < MC; ++q) {
      typename H::Acc sa = H::zero();
#pragma unroll
      for (int j = 0; j < Hh; ++j) H::mac(sa, E[q * Hh + j], e[j]);
      if constexpr (P % 2 == 1) H::mac(sa, am[q], x[Hh]);
      const V A = H::get(sa);
      if (q < Hh) {
        typename H::Acc sb = H::zero();
#pragma unroll
        for (int j = 0; j < Hh; ++j) H::mac(sb, bo[q * Hh + j], o[j]);
        const V B = H::get(sb);
        out[base + q * st] = H::s(A + B);
        out[base + (P - 1 - q) * st] = H::s(A - B);
      } else {
        out[base + q * st] = H::s(A);
      }
    }
  }
}

// the same on nf fields of p^2 face values (AXIS 0: a, 1: b), one output
// point per thread (the face fields are too few for a line per thread)
template <int P, typename V, int AXIS, bool TR>
__device__ void sweep2(const typename HT<V>::S* M,
                       const typename HT<V>::S* in, typename HT<V>::S* out,
                       int nf) {
  using H = HT<V>;
  constexpr int F = P * P;
  constexpr int st = AXIS == 0 ? 1 : P;
  for (int t = threadIdx.x; t < nf * F; t += blockDim.x) {
    const int i = t % F;
    const int ii = AXIS == 0 ? i % P : i / P;
    const typename H::S* src = in + (t - ii * st);
    typename H::Acc acc = H::zero();
#pragma unroll
    for (int j = 0; j < P; ++j)
      H::mac(acc, TR ? M[j * P + ii] : M[ii * P + j], src[j * st]);
    out[t] = H::s(H::get(acc));
  }
}

// local index of node (ja, jb) of the layer of face (D, s) of a cell
template <int P>
__device__ __forceinline__ int layer_node(int D, int s, int ja, int jb) {
  int ii[3];
  ii[D] = s ? P - 1 : 0;
  ii[D == 0 ? 1 : 0] = ja;
  ii[D == 2 ? 1 : 2] = jb;
  return ii[0] + P * (ii[1] + P * ii[2]);
}

// Faces of direction D per block of the trace kernel (two layers of 8 face
// arrays each in static shared memory, under 48 KB).
template <int P>
constexpr int hdg_faces_per_block() {
  return P <= 3 ? 16 : (P <= 5 ? 8 : 4);
}

// Where face fl of direction D sits: its lower (L) and upper (R) cells, and
// whether its trace is data (a Dirichlet boundary face).
struct HdgFace {
  bool hasL, hasR, dir;
  int cellL, cellR;
};
__device__ __forceinline__ HdgFace hdg_face(const HdgArgs& a, int D, int fl) {
  int m[3] = {a.n[0], a.n[1], a.n[2]};
  m[D] += 1;
  const int fc[3] = {fl % m[0], (fl / m[0]) % m[1], fl / (m[0] * m[1])};
  HdgFace h;
  h.hasL = fc[D] >= 1;
  h.hasR = fc[D] < a.n[D];
  const int side = h.hasL ? (h.hasR ? -1 : 2 * D + 1) : 2 * D;
  h.dir = side >= 0 && !((a.neumann >> side) & 1);
  int cL[3] = {fc[0], fc[1], fc[2]};
  cL[D] -= 1;
  h.cellL = h.hasL ? cL[0] + a.n[0] * (cL[1] + a.n[1] * cL[2]) : 0;
  h.cellR = h.hasR ? fc[0] + a.n[0] * (fc[1] + a.n[1] * fc[2]) : 0;
  return h;
}

// Trace lambda at the Gauss points of the faces of direction D, a few faces
// per block:
//   lambda = sum_sides (q . n_out + tau u) / (tau * number of sides),
// n_out the side's outward unit normal (+n for the cell below the face, -n
// for the one above; n = e_D on Cartesian cells); zero on Dirichlet faces.
template <int P, typename V>
__global__ void __launch_bounds__(256) k_hdg_trace(HdgArgs a, int D) {
  using H = HT<V>;
  using S = typename H::S;
  constexpr int F = P * P, N = P * P * P, C = hdg_faces_per_block<P>();
  __shared__ S sS[P * P];
  // [face][side][q_x, q_y, q_z, u][F]
  __shared__ S lay[C * 8 * F], tmp[C * 8 * F];
  int m[3] = {a.n[0], a.n[1], a.n[2]};
  m[D] += 1;
  const int nface = m[0] * m[1] * m[2];
  const int fl0 = blockIdx.x * C;
  // per face: the first x index of each side's four fields, -1 where that
  // side is missing or the trace is data
  __shared__ long long xoff[C][2];
  __shared__ unsigned char fkind[C];  // bit 0: lower cell, 1: upper, 2: data
  for (int i = threadIdx.x; i < P * P; i += blockDim.x)
    sS[i] = H::s(H::d2v(c_tab64[P - 2].S[i]));
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    unsigned char k = 4;
    xoff[c][0] = xoff[c][1] = -1;
    if (fl0 + c < nface) {
      const HdgFace h = hdg_face(a, D, fl0 + c);
      k = (h.hasL ? 1 : 0) | (h.hasR ? 2 : 0) | (h.dir ? 4 : 0);
      if (!h.dir && h.hasL) xoff[c][0] = (long long)h.cellL * 4 * N;
      if (!h.dir && h.hasR) xoff[c][1] = (long long)h.cellR * 4 * N;
    }
    fkind[c] = k;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < C * 8 * F; t += blockDim.x) {
    const int c = t / (8 * F), r = t - c * 8 * F;
    const int sf = r / F, j = r - sf * F;  // side 0: lower cell, 1: upper
    const int sd = sf / 4, fld = sf % 4;
    const long long o = xoff[c][sd];
    const int loc = layer_node<P>(D, sd == 0 ? 1 : 0, j % P, j / P);
    lay[t] = H::s(H::d2v(o >= 0 ? a.x[o + fld * N + loc] : 0.0));
  }
  __syncthreads();
  sweep2<P, V, 0, false>(sS, lay, tmp, 8 * C);
  __syncthreads();
  sweep2<P, V, 1, false>(sS, tmp, lay, 8 * C);
  __syncthreads();
  for (int t = threadIdx.x; t < C * F; t += blockDim.x) {
    const int c = t / F, q = t - c * F;
    if (fl0 + c >= nface) continue;
    const int k = fkind[c];
    const bool hasL = k & 1, hasR = k & 2;
    const size_t f = (size_t)a.face_off[D] + fl0 + c;
    if (k & 4) {  // Dirichlet: data, not x
      a.lam[f * F + q] = 0.0;
      continue;
    }
    const double tf = face_tau<P>(a, f);
    const V tau = H::d2v(tf);
    const V inv = H::recip(H::d2v((hasL && hasR ? 2.0 : 1.0) * tf));
    V nv[3] = {H::d2v(0.0), H::d2v(0.0), H::d2v(0.0)};
    if (a.gf) {
      for (int e = 0; e < 3; ++e) nv[e] = H::d2v(a.gf[(f * 4 + 1 + e) * F + q]);
    } else {
      nv[D] = H::d2v(1.0);
    }
    V num = H::d2v(0.0);
    for (int sd = 0; sd < 2; ++sd) {
      if (!(sd == 0 ? hasL : hasR)) continue;
      const S* L = lay + (c * 8 + 4 * sd) * F;
      const V qn = nv[0] * H::v(L[q]) + nv[1] * H::v(L[F + q]) +
                   nv[2] * H::v(L[2 * F + q]);
      num = num + (sd == 0 ? qn : V(-qn)) + tau * H::v(L[3 * F + q]);
    }
    a.lam[f * F + q] = H::v2d(num * inv);
  }
}

// Shared memory of one cell of the cell kernel: A and B (4 fields of p^3
// values each) and the face scratch (10 p^2 values).
template <int P>
constexpr size_t hdg_cell_bytes() {
  return (size_t)(8 * P * P * P + 10 * P * P) * sizeof(double);
}
// Cells per block: several cells share each barrier interval, up to 40 KB.
template <int P>
constexpr int hdg_cells_per_block() {
  const int c = (int)((40 * 1024) / hdg_cell_bytes<P>());
  return c < 1 ? 1 : (c > 16 ? 16 : c);
}

// Geometry of cell point t: w det J and J^{-1}[e][d] (row e, column d); on
// Cartesian cells from the block's table of w_q det J (sW3) and 1/h.
template <int P, typename V>
__device__ __forceinline__ void point_geo(const HdgArgs& a, int cell, int t,
                                          const typename HT<V>::S* sW3,
                                          const V (&ih)[3], V& wdet,
                                          V (&Ji)[3][3]) {
  using H = HT<V>;
  constexpr int N = P * P * P;
  if (a.gc) {
    const double* g = a.gc + (size_t)cell * 10 * N + t;
    wdet = H::d2v(g[0]);
    for (int e = 0; e < 3; ++e)
      for (int d = 0; d < 3; ++d) Ji[e][d] = H::d2v(g[(1 + 3 * e + d) * N]);
  } else {
    wdet = H::v(sW3[t]);
    for (int e = 0; e < 3; ++e)
      for (int d = 0; d < 3; ++d) Ji[e][d] = e == d ? ih[d] : H::d2v(0.0);
  }
}

// Cell kernel: a block takes C = hdg_cells_per_block<P>() consecutive cells,
// their cell integrals and the terms of their six faces.  The C cells' four
// fields lie one after the other in shared memory, so every sweep runs over
// 4 C fields at once and each barrier interval holds C cells' work.  At the
// Gauss points (w det = w_q det J, J^{-1} = dxi/dx):
//   q_d rows: w det kappa^-1 q_d - sum_e D_e^T (w det J^{-1}[e][d] u)
//   u rows:   -w det sum_{d,e} J^{-1}[e][d] D_e q_d
template <int P, typename V>
__global__ void k_hdg_cell(HdgArgs a) {
  using H = HT<V>;
  using S = typename H::S;
  constexpr int F = P * P, N = P * P * P, C = hdg_cells_per_block<P>();
  __shared__ S sS[P * P], sD[P * P];
  __shared__ S sE[eo_elems<P>()], sET[eo_elems<P>()];  // S, S^T even-odd
  __shared__ S sW3[P * P * P], sW2[P * P];  // w_q det J (Cartesian), w_a w_b
  __shared__ double sw[P];
  extern __shared__ __align__(16) unsigned char hraw[];
  S* A = reinterpret_cast<S*>(hraw);  // [C][4][N]
  S* B = A + 4 * C * N;                 // [C][4][N]
  S* ul = B + 4 * C * N;                // [C][F]: u layer, then u at the points
  S* ut = ul + C * F;                   // [C][F]: sweep temporary
  S* gcf = ut + C * F;                  // [C][4][F]: w_x, w_y, w_z, v terms
  S* gt = gcf + 4 * C * F;              // [C][4][F]: sweep temporary
  const int cell0 = blockIdx.x * C;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    sS[i] = H::s(H::d2v(c_tab64[P - 2].S[i]));
    sD[i] = H::s(H::d2v(c_tab64[P - 2].D[i]));
  }
  load_eo<P, V, false>(sE);
  load_eo<P, V, true>(sET);
  for (int i = threadIdx.x; i < P; i += blockDim.x) sw[i] = c_tab64[P - 2].w[i];
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const double* w = c_tab64[P - 2].w;
    sW3[t] = H::s(H::d2v(w[t % P] * w[(t / P) % P] * w[t / (P * P)] * a.vol));
  }
  for (int q = threadIdx.x; q < F; q += blockDim.x) {
    const double* w = c_tab64[P - 2].w;
    sW2[q] = H::s(H::d2v(w[q % P] * w[q / P]));
  }
  const V ih[3] = {H::d2v(a.ih[0]), H::d2v(a.ih[1]), H::d2v(a.ih[2])};
  const V kconst = H::d2v(a.kinv);
  const int ncells = a.n[0] * a.n[1] * a.n[2];
  // cells past the last one compute on zeros and store nothing
  for (int t = threadIdx.x; t < 4 * C * N; t += blockDim.x) {
    const int cell = cell0 + t / (4 * N);
    A[t] = H::s(H::d2v(cell < ncells ? a.x[(size_t)cell0 * 4 * N + t] : 0.0));
  }
  __syncthreads();
  // values of the four fields at the Gauss points
  sweep3<P, V, 0>(sE, A, B, 4 * C);
  __syncthreads();
  sweep3<P, V, 1>(sE, B, A, 4 * C);
  __syncthreads();
  sweep3<P, V, 2>(sE, A, B, 4 * C);
  __syncthreads();
  const int st[3] = {1, P, P * P};
  // u rows and the mass part of the q rows
  for (int tt = threadIdx.x; tt < C * N; tt += blockDim.x) {
    const int c = tt / N, t = tt - c * N;
    const int cell = cell0 + c < ncells ? cell0 + c : ncells - 1;
    S* Ac = A + c * 4 * N;
    const S* Bc = B + c * 4 * N;
    const int ii[3] = {t % P, (t / P) % P, t / (P * P)};
    V wdet, Ji[3][3];
    point_geo<P, V>(a, cell, t, sW3, ih, wdet, Ji);
    const V kinv =
        a.kcell ? H::recip(H::d2v(a.kcell[(size_t)cell * N + t])) : kconst;
    V dv = H::d2v(0.0);
    for (int d = 0; d < 3; ++d) {
      for (int e = 0; e < 3; ++e) {
        if (!a.gc && e != d) continue;
        const int base = t - ii[e] * st[e];
        typename H::Acc s1 = H::zero();
        for (int j = 0; j < P; ++j)
          H::mac(s1, sD[ii[e] * P + j], Bc[d * N + base + j * st[e]]);
        dv = dv + Ji[e][d] * H::get(s1);
      }
      Ac[d * N + t] = H::s(wdet * kinv * H::v(Bc[d * N + t]));
    }
    Ac[3 * N + t] = H::s(V(-(wdet * dv)));
  }
  __syncthreads();
  // -sum_e D_e^T (w det J^{-1}[e][d] u) into the q_d rows, one d at a time
  // (the q values at the points in B are no longer needed)
  for (int d = 0; d < 3; ++d) {
    for (int tt = threadIdx.x; tt < C * N; tt += blockDim.x) {
      const int c = tt / N, t = tt - c * N;
      const int cell = cell0 + c < ncells ? cell0 + c : ncells - 1;
      S* Bc = B + c * 4 * N;
      V wdet, Ji[3][3];
      point_geo<P, V>(a, cell, t, sW3, ih, wdet, Ji);
      for (int e = 0; e < 3; ++e)
        Bc[e * N + t] = H::s(wdet * Ji[e][d] * H::v(Bc[3 * N + t]));
    }
    __syncthreads();
    for (int tt = threadIdx.x; tt < C * N; tt += blockDim.x) {
      const int c = tt / N, t = tt - c * N;
      S* Ac = A + c * 4 * N;
      const S* Bc = B + c * 4 * N;
      const int ii[3] = {t % P, (t / P) % P, t / (P * P)};
      typename H::Acc s2 = H::zero();
      for (int e = 0; e < 3; ++e) {
        if (!a.gc && e != d) continue;
        const int base = t - ii[e] * st[e];
        for (int j = 0; j < P; ++j)
          H::mac(s2, sD[j * P + ii[e]], Bc[e * N + base + j * st[e]]);
      }
      Ac[d * N + t] = H::s(H::v(Ac[d * N + t]) - H::get(s2));
    }
    __syncthreads();
  }
  sweep3<P, V, 2>(sET, A, B, 4 * C);
  __syncthreads();
  sweep3<P, V, 1>(sET, B, A, 4 * C);
  __syncthreads();
  sweep3<P, V, 0>(sET, A, B, 4 * C);
  __syncthreads();
  // faces, one (direction, side) at a time for all C cells of the block
  for (int D = 0; D < 3; ++D) {
    int m[3] = {a.n[0], a.n[1], a.n[2]};
    m[D] += 1;
    for (int s = 0; s < 2; ++s) {
      for (int tt = threadIdx.x; tt < C * F; tt += blockDim.x) {
        const int c = tt / F, j = tt - c * F;
        const int cell = cell0 + c;
        ul[tt] = H::s(H::d2v(
            cell < ncells ? a.x[(size_t)cell * 4 * N + 3 * N +
                                layer_node<P>(D, s, j % P, j / P)]
                          : 0.0));
      }
      __syncthreads();
      sweep2<P, V, 0, false>(sS, ul, ut, C);
      __syncthreads();
      sweep2<P, V, 1, false>(sS, ut, ul, C);
      __syncthreads();
      for (int tt = threadIdx.x; tt < C * F; tt += blockDim.x) {
        const int c = tt / F, q = tt - c * F;
        const int cell = cell0 + c < ncells ? cell0 + c : ncells - 1;
        int fc[3] = {cell % a.n[0], (cell / a.n[0]) % a.n[1],
                     cell / (a.n[0] * a.n[1])};
        fc[D] += s;
        const size_t f = (size_t)a.face_off[D] + fc[0] +
                         (size_t)m[0] * (fc[1] + (size_t)m[1] * fc[2]);
        const V tau = H::d2v(face_tau<P>(a, f));
        V dA, nv[3] = {H::d2v(0.0), H::d2v(0.0), H::d2v(0.0)};
        if (a.gf) {
          dA = H::d2v(a.gf[(f * 4) * F + q]);
          for (int e = 0; e < 3; ++e)
            nv[e] = H::d2v(a.gf[(f * 4 + 1 + e) * F + q]);
        } else {
          dA = H::v(sW2[q]) * H::d2v(a.fa[D]);
          nv[D] = H::d2v(1.0);
        }
        // outward normal: +n on the upper face (s = 1), -n on the lower one
        const V lq = H::d2v(a.lam[f * F + q]);
        const V dl = s ? V(dA * lq) : V(-(dA * lq));
        S* g = gcf + c * 4 * F;
        for (int e = 0; e < 3; ++e)
          g[e * F + q] = H::s(dl * nv[e]);                       // <w . n, lambda>
        g[3 * F + q] = H::s(dA * tau * (lq - H::v(ul[tt])));     // <v, tau(lambda-u)>
      }
      __syncthreads();
      sweep2<P, V, 1, true>(sS, gcf, gt, 4 * C);
      __syncthreads();
      sweep2<P, V, 0, true>(sS, gt, gcf, 4 * C);
      __syncthreads();
      for (int tt = threadIdx.x; tt < C * F; tt += blockDim.x) {
        const int c = tt / F, j = tt - c * F;
        const int loc = layer_node<P>(D, s, j % P, j / P);
        S* Bc = B + c * 4 * N;
        const S* g = gcf + c * 4 * F;
        for (int e = 0; e < 4; ++e)
          Bc[e * N + loc] = H::s(H::v(Bc[e * N + loc]) + H::v(g[e * F + j]));
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < 4 * C * N; t += blockDim.x)
    if (cell0 + t / (4 * N) < ncells)
      a.y[(size_t)cell0 * 4 * N + t] = H::v2d(H::v(B[t]));
}

template <typename V>
void run_hdg(const Level& L, const HdgArgs& a, cudaStream_t s) {
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    for (int D = 0; D < 3; ++D) {
      int m[3] = {L.n[0], L.n[1], L.n[2]};
      m[D] += 1;
      constexpr int CF = hdg_faces_per_block<P>();
      k_hdg_trace<P, V><<<(m[0] * m[1] * m[2] + CF - 1) / CF, 256, 0, s>>>(
          a, D);
      MFP_CHECK_CUDA(cudaGetLastError());
      note_launch();
    }
    constexpr int C = hdg_cells_per_block<P>();
    constexpr size_t smem = C * hdg_cell_bytes<P>();
    if (smem > 48 * 1024)
      MFP_CHECK_CUDA(cudaFuncSetAttribute(
          k_hdg_cell<P, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
          (int)smem));
    const int blocks = (int)((L.ncells + C - 1) / C);
    k_hdg_cell<P, V><<<blocks, C > 1 ? 256 : 128, smem, s>>>(a);
    MFP_CHECK_CUDA(cudaGetLastError());
    note_launch();
  });
}

}  // namespace

void launch_hdg_apply(const Level& L, double tau_factor, double* lam,
                      const double* hdg_cell, const double* hdg_face,
                      const double* x, double* y, cudaStream_t s) {
  ensure_tables();
  HdgArgs a{};
  a.x = x;
  a.y = y;
  a.lam = lam;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = L.n[d];
    a.face_off[d] = L.face_off[d];
    a.h[d] = L.h[d];
  }
  a.neumann = L.bc.neumann;
  a.kappa = L.kappa;
  a.kinv = 1.0 / L.kappa;
  for (int d = 0; d < 3; ++d) a.ih[d] = 1.0 / L.h[d];
  a.vol = L.h[0] * L.h[1] * L.h[2];
  a.fa[0] = L.h[1] * L.h[2];
  a.fa[1] = L.h[0] * L.h[2];
  a.fa[2] = L.h[0] * L.h[1];
  a.tau_factor = tau_factor;
  a.kcell = L.d64.kcell;
  a.kface = L.d64.kface;
  a.gc = hdg_cell;
  a.gf = hdg_face;
  if (L.df_arith)
    run_hdg<df>(L, a, s);
  else
    run_hdg<double>(L, a, s);
}

}  // namespace mfp
