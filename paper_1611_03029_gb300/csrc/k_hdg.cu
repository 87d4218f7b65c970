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
// whose traces are data.  k_hdg_trace (one block per face) forms lambda,
// k_hdg_cell (one block per cell) adds the cell integrals by sum
// factorization (values at the Gauss points by S, reference derivatives by
// the Gauss collocation matrix D, mapped by J^{-1}) and the six faces' terms
// -<v, tau u> + <w . n, lambda> + <v, tau lambda> on the face-layer nodes.
// tau = tau_factor times the largest coefficient on the face (Sec. 4.2).
// Cartesian cells use their constant Jacobian; curved ones read w det J and
// J^{-1} per cell point and dA and the unit normal per face point.  Plain
// float64 arithmetic.
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
  double kappa;  // constant coefficient (when kcell / kface are null)
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

// out = M (or M^T) applied along `axis` of nf fields of p^3 values
template <int P>
__device__ void sweep3(const double* M, bool tr, int axis, const double* in,
                       double* out, int nf) {
  constexpr int N = P * P * P;
  const int st = axis == 0 ? 1 : (axis == 1 ? P : P * P);
  for (int t = threadIdx.x; t < nf * N; t += blockDim.x) {
    const int i = t % N;
    const int ii = axis == 0 ? i % P : (axis == 1 ? (i / P) % P : i / (P * P));
    const double* src = in + (t - i) + (i - ii * st);
    double acc = 0;
    for (int j = 0; j < P; ++j)
      acc += (tr ? M[j * P + ii] : M[ii * P + j]) * src[j * st];
    out[t] = acc;
  }
}

// the same on nf fields of p^2 face values (axis 0: a, 1: b)
template <int P>
__device__ void sweep2(const double* M, bool tr, int axis, const double* in,
                       double* out, int nf) {
  constexpr int F = P * P;
  const int st = axis == 0 ? 1 : P;
  for (int t = threadIdx.x; t < nf * F; t += blockDim.x) {
    const int i = t % F;
    const int ii = axis == 0 ? i % P : i / P;
    const double* src = in + (t - i) + (i - ii * st);
    double acc = 0;
    for (int j = 0; j < P; ++j)
      acc += (tr ? M[j * P + ii] : M[ii * P + j]) * src[j * st];
    out[t] = acc;
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


// One block per face of direction D: lambda at the face Gauss points,
//   lambda = sum_sides (q . n_out + tau u) / (tau * number of sides),
// n_out the side's outward unit normal (+n for the cell below the face, -n
// for the one above; n = e_D on Cartesian cells).
template <int P>
__global__ void k_hdg_trace(HdgArgs a, int D) {
  constexpr int F = P * P, N = P * P * P;
  __shared__ double sS[P * P];
  __shared__ double lay[8 * F], tmp[8 * F];  // [side][q_x, q_y, q_z, u][F]
  int m[3] = {a.n[0], a.n[1], a.n[2]};
  m[D] += 1;
  const int fl = blockIdx.x;
  const int fc[3] = {fl % m[0], (fl / m[0]) % m[1], fl / (m[0] * m[1])};
  const bool hasL = fc[D] >= 1, hasR = fc[D] < a.n[D];
  const int side = hasL ? (hasR ? -1 : 2 * D + 1) : 2 * D;
  const size_t f = (size_t)a.face_off[D] + fl;
  if (side >= 0 && !((a.neumann >> side) & 1)) {  // Dirichlet: data, not x
    for (int q = threadIdx.x; q < F; q += blockDim.x) a.lam[f * F + q] = 0.0;
    return;
  }
  int cL[3] = {fc[0], fc[1], fc[2]};
  cL[D] -= 1;
  const int cellL = hasL ? cL[0] + a.n[0] * (cL[1] + a.n[1] * cL[2]) : 0;
  const int cellR = hasR ? fc[0] + a.n[0] * (fc[1] + a.n[1] * fc[2]) : 0;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x)
    sS[i] = c_tab64[P - 2].S[i];
  for (int t = threadIdx.x; t < 8 * F; t += blockDim.x) {
    const int sf = t / F, j = t % F;  // side 0: lower cell, 1: upper cell
    const int s = sf / 4, fld = sf % 4;
    const bool has = s == 0 ? hasL : hasR;
    const int loc = layer_node<P>(D, s == 0 ? 1 : 0, j % P, j / P);
    const double* xc = a.x + (size_t)(s == 0 ? cellL : cellR) * 4 * N;
    lay[t] = has ? xc[fld * N + loc] : 0.0;
  }
  __syncthreads();
  sweep2<P>(sS, false, 0, lay, tmp, 8);
  __syncthreads();
  sweep2<P>(sS, false, 1, tmp, lay, 8);
  __syncthreads();
  const double tau = face_tau<P>(a, f);
  for (int q = threadIdx.x; q < F; q += blockDim.x) {
    double nv[3] = {0.0, 0.0, 0.0};
    if (a.gf) {
      for (int e = 0; e < 3; ++e) nv[e] = a.gf[(f * 4 + 1 + e) * F + q];
    } else {
      nv[D] = 1.0;
    }
    double num = 0, den = 0;
    for (int s = 0; s < 2; ++s) {
      if (!(s == 0 ? hasL : hasR)) continue;
      const double* L = lay + 4 * s * F;
      const double qn = nv[0] * L[q] + nv[1] * L[F + q] + nv[2] * L[2 * F + q];
      num += (s == 0 ? qn : -qn) + tau * L[3 * F + q];
      den += tau;
    }
    a.lam[f * F + q] = num / den;
  }
}

template <int P>
constexpr size_t hdg_cell_smem() {
  return (size_t)(8 * P * P * P + 10 * P * P) * sizeof(double);
}

// Geometry of cell point t: w det J and J^{-1}[e][d] (row e, column d).
template <int P>
__device__ __forceinline__ void point_geo(const HdgArgs& a, int cell, int t,
                                          const double* sw, double& wdet,
                                          double (&Ji)[3][3]) {
  constexpr int N = P * P * P;
  if (a.gc) {
    const double* g = a.gc + (size_t)cell * 10 * N + t;
    wdet = g[0];
    for (int e = 0; e < 3; ++e)
      for (int d = 0; d < 3; ++d) Ji[e][d] = g[(1 + 3 * e + d) * N];
  } else {
    wdet = sw[t % P] * sw[(t / P) % P] * sw[t / (P * P)] * a.h[0] * a.h[1] *
           a.h[2];
    for (int e = 0; e < 3; ++e)
      for (int d = 0; d < 3; ++d) Ji[e][d] = e == d ? 1.0 / a.h[d] : 0.0;
  }
}

// One block per cell: cell integrals and the terms of its six faces.  At the
// Gauss points (w det = w_q det J, J^{-1} = dxi/dx):
//   q_d rows: w det kappa^-1 q_d - sum_e D_e^T (w det J^{-1}[e][d] u)
//   u rows:   -w det sum_{d,e} J^{-1}[e][d] D_e q_d
template <int P>
__global__ void k_hdg_cell(HdgArgs a) {
  constexpr int F = P * P, N = P * P * P;
  __shared__ double sS[P * P], sD[P * P], sw[P];
  extern __shared__ __align__(16) double hsm[];
  double* A = hsm;
  double* B = hsm + 4 * N;
  double* FS = hsm + 8 * N;
  const int cell = blockIdx.x;
  const int c3[3] = {cell % a.n[0], (cell / a.n[0]) % a.n[1],
                     cell / (a.n[0] * a.n[1])};
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    sS[i] = c_tab64[P - 2].S[i];
    sD[i] = c_tab64[P - 2].D[i];
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) sw[i] = c_tab64[P - 2].w[i];
  const double* xc = a.x + (size_t)cell * 4 * N;
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) A[t] = xc[t];
  __syncthreads();
  // values of the four fields at the Gauss points
  sweep3<P>(sS, false, 0, A, B, 4);
  __syncthreads();
  sweep3<P>(sS, false, 1, B, A, 4);
  __syncthreads();
  sweep3<P>(sS, false, 2, A, B, 4);
  __syncthreads();
  const int st[3] = {1, P, P * P};
  // u rows and the mass part of the q rows
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int ii[3] = {t % P, (t / P) % P, t / (P * P)};
    double wdet, Ji[3][3];
    point_geo<P>(a, cell, t, sw, wdet, Ji);
    const double kinv =
        1.0 / (a.kcell ? a.kcell[(size_t)cell * N + t] : a.kappa);
    double dv = 0;
    for (int d = 0; d < 3; ++d) {
      for (int e = 0; e < 3; ++e) {
        if (!a.gc && e != d) continue;
        const int base = t - ii[e] * st[e];
        double s1 = 0;
        for (int j = 0; j < P; ++j)
          s1 += sD[ii[e] * P + j] * B[d * N + base + j * st[e]];
        dv += Ji[e][d] * s1;
      }
      A[d * N + t] = wdet * kinv * B[d * N + t];
    }
    A[3 * N + t] = -wdet * dv;
  }
  __syncthreads();
  // -sum_e D_e^T (w det J^{-1}[e][d] u) into the q_d rows, one d at a time
  // (the q values at the points in B are no longer needed)
  for (int d = 0; d < 3; ++d) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
      double wdet, Ji[3][3];
      point_geo<P>(a, cell, t, sw, wdet, Ji);
      for (int e = 0; e < 3; ++e) B[e * N + t] = wdet * Ji[e][d] * B[3 * N + t];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
      const int ii[3] = {t % P, (t / P) % P, t / (P * P)};
      double s2 = 0;
      for (int e = 0; e < 3; ++e) {
        if (!a.gc && e != d) continue;
        const int base = t - ii[e] * st[e];
        for (int j = 0; j < P; ++j)
          s2 += sD[j * P + ii[e]] * B[e * N + base + j * st[e]];
      }
      A[d * N + t] -= s2;
    }
    __syncthreads();
  }
  sweep3<P>(sS, true, 2, A, B, 4);
  __syncthreads();
  sweep3<P>(sS, true, 1, B, A, 4);
  __syncthreads();
  sweep3<P>(sS, true, 0, A, B, 4);
  __syncthreads();
  // faces: scratch FS (10 p^2 values)
  double* ul = FS;           // u layer, then u at the face points
  double* ut = FS + F;       // sweep temporary
  double* gcf = FS + 2 * F;  // [w_x, w_y, w_z, v] terms at the face points
  double* gt = FS + 6 * F;   // sweep temporary for the four fields
  for (int D = 0; D < 3; ++D) {
    const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
    int m[3] = {a.n[0], a.n[1], a.n[2]};
    m[D] += 1;
    for (int s = 0; s < 2; ++s) {
      int fc[3] = {c3[0], c3[1], c3[2]};
      fc[D] += s;
      const size_t f = (size_t)a.face_off[D] + fc[0] +
                       (size_t)m[0] * (fc[1] + (size_t)m[1] * fc[2]);
      for (int j = threadIdx.x; j < F; j += blockDim.x)
        ul[j] = xc[3 * N + layer_node<P>(D, s, j % P, j / P)];
      __syncthreads();
      sweep2<P>(sS, false, 0, ul, ut, 1);
      __syncthreads();
      sweep2<P>(sS, false, 1, ut, ul, 1);
      __syncthreads();
      const double tau = face_tau<P>(a, f);
      const double so = s ? 1.0 : -1.0;  // outward: +n on the upper face
      for (int q = threadIdx.x; q < F; q += blockDim.x) {
        double dA, nv[3] = {0.0, 0.0, 0.0};
        if (a.gf) {
          dA = a.gf[(f * 4) * F + q];
          for (int e = 0; e < 3; ++e) nv[e] = a.gf[(f * 4 + 1 + e) * F + q];
        } else {
          dA = sw[q % P] * sw[q / P] * a.h[T1] * a.h[T2];
          nv[D] = 1.0;
        }
        const double lq = a.lam[f * F + q];
        for (int e = 0; e < 3; ++e)
          gcf[e * F + q] = dA * so * nv[e] * lq;       // <w . n, lambda>
        gcf[3 * F + q] = dA * tau * (lq - ul[q]);      // <v, tau (lambda - u)>
      }
      __syncthreads();
      sweep2<P>(sS, true, 1, gcf, gt, 4);
      __syncthreads();
      sweep2<P>(sS, true, 0, gt, gcf, 4);
      __syncthreads();
      for (int j = threadIdx.x; j < F; j += blockDim.x) {
        const int loc = layer_node<P>(D, s, j % P, j / P);
        for (int e = 0; e < 4; ++e) B[e * N + loc] += gcf[e * F + j];
      }
      __syncthreads();
    }
  }
  double* yc = a.y + (size_t)cell * 4 * N;
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) yc[t] = B[t];
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
  a.tau_factor = tau_factor;
  a.kcell = L.d64.kcell;
  a.kface = L.d64.kface;
  a.gc = hdg_cell;
  a.gf = hdg_face;
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    for (int D = 0; D < 3; ++D) {
      int m[3] = {L.n[0], L.n[1], L.n[2]};
      m[D] += 1;
      k_hdg_trace<P><<<m[0] * m[1] * m[2], 64, 0, s>>>(a, D);
      MFP_CHECK_CUDA(cudaGetLastError());
      note_launch();
    }
    constexpr size_t smem = hdg_cell_smem<P>();
    if (smem > 48 * 1024)
      MFP_CHECK_CUDA(cudaFuncSetAttribute(
          k_hdg_cell<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
          (int)smem));
    k_hdg_cell<P><<<(int)L.ncells, 128, smem, s>>>(a);
    MFP_CHECK_CUDA(cudaGetLastError());
    note_launch();
  });
}

}  // namespace mfp
