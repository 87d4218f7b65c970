// HDG mixed matrix-free operator (Sec. 3, "HDG mixed matrix-free", on the
// hybridizable DG form of Sec. 2.3) on Cartesian cells:
//   y = ([A B^T; B D] + [C^T; G^T] H^{-1} [C G]) x
// with the cell unknowns (q_x, q_y, q_z, u) in cell-major blocks of 4 p^3
// nodal values (Lagrange in the Gauss-Lobatto points), where
//   A = (w, kappa^-1 q), B^T = -(div w, u), D = -<v, tau u>,
//   C^T = <w . n, lambda>, G^T = <v, tau lambda>, H = sum_sides <mu, tau lambda>.
// The trace is never an unknown: H^{-1} [C G] x is the face trace
//   lambda = sum_sides (q . n + tau u) / sum_sides tau
// at the face Gauss points (H is tau times the face mass in a basis as large
// as the Gauss rule, so its inverse acts point by point); it is zero on
// Dirichlet faces, whose traces are data.  k_hdg_trace (one block per face)
// forms lambda, k_hdg_cell (one block per cell) adds the cell integrals by
// sum factorization (values at the Gauss points by S, derivatives by the
// Gauss collocation matrix D) and the six faces' terms
// -<v, tau u> + <w . n, lambda> + <v, tau lambda> on the face-layer nodes.
// Plain float64 arithmetic.
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
  double h[3];  // physical cell size
  double kinv;  // 1 / kappa
  double tau;
};

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

// One block per face of direction D: lambda at the face Gauss points.
template <int P>
__global__ void k_hdg_trace(HdgArgs a, int D) {
  constexpr int F = P * P, N = P * P * P;
  __shared__ double sS[P * P];
  __shared__ double lay[4 * F], tmp[4 * F];  // [side][field q_D, u][F]
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
  for (int t = threadIdx.x; t < 2 * F; t += blockDim.x) {
    const int s = t / F, j = t % F;  // s = 0: lower cell, 1: upper cell
    const bool has = s == 0 ? hasL : hasR;
    const int loc = layer_node<P>(D, s == 0 ? 1 : 0, j % P, j / P);
    const double* xc = a.x + (size_t)(s == 0 ? cellL : cellR) * 4 * N;
    lay[(2 * s) * F + j] = has ? xc[D * N + loc] : 0.0;      // q_D
    lay[(2 * s + 1) * F + j] = has ? xc[3 * N + loc] : 0.0;  // u
  }
  __syncthreads();
  sweep2<P>(sS, false, 0, lay, tmp, 4);
  __syncthreads();
  sweep2<P>(sS, false, 1, tmp, lay, 4);
  __syncthreads();
  for (int q = threadIdx.x; q < F; q += blockDim.x) {
    double num = 0, den = 0;
    if (hasL) {  // outward normal +e_D
      num += lay[q] + a.tau * lay[F + q];
      den += a.tau;
    }
    if (hasR) {  // outward normal -e_D
      num += -lay[2 * F + q] + a.tau * lay[3 * F + q];
      den += a.tau;
    }
    a.lam[f * F + q] = num / den;
  }
}

// One block per cell: cell integrals and the terms of its six faces.
template <int P>
__global__ void k_hdg_cell(HdgArgs a) {
  constexpr int F = P * P, N = P * P * P;
  __shared__ double sS[P * P], sD[P * P], sw[P];
  __shared__ double A[4 * N], B[4 * N];
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
  // integrands at the Gauss points (w det = w_x w_y w_z h_x h_y h_z):
  //   q_d rows: w det kappa^-1 q_d - (1/h_d) D^T_d (w det u)
  //   u rows:   -w det sum_d (1/h_d) D_d q_d
  const double vol = a.h[0] * a.h[1] * a.h[2];
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int ii[3] = {t % P, (t / P) % P, t / (P * P)};
    const int st[3] = {1, P, P * P};
    const double wq = sw[ii[0]] * sw[ii[1]] * sw[ii[2]] * vol;
    double dv = 0;
    for (int d = 0; d < 3; ++d) {
      const int base = t - ii[d] * st[d];
      double s1 = 0, s2 = 0;
      for (int j = 0; j < P; ++j) {
        const int tj = base + j * st[d];
        const int jj[3] = {tj % P, (tj / P) % P, tj / (P * P)};
        const double wj = sw[jj[0]] * sw[jj[1]] * sw[jj[2]] * vol;
        s1 += sD[ii[d] * P + j] * B[d * N + tj];
        s2 += sD[j * P + ii[d]] * wj * B[3 * N + tj];
      }
      dv += s1 / a.h[d];
      A[d * N + t] = wq * a.kinv * B[d * N + t] - s2 / a.h[d];
    }
    A[3 * N + t] = -wq * dv;
  }
  __syncthreads();
  sweep3<P>(sS, true, 2, A, B, 4);
  __syncthreads();
  sweep3<P>(sS, true, 1, B, A, 4);
  __syncthreads();
  sweep3<P>(sS, true, 0, A, B, 4);
  __syncthreads();
  // faces: scratch in A (5 p^2 values)
  double* ul = A;          // u layer, then u at the face points
  double* ut = A + F;      // sweep temporary
  double* gc = A + F;      // [cq, cu] at the face points (after ut is free)
  double* gt = A + 3 * F;  // sweep temporary for the two fields
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
      const double nD = s ? 1.0 : -1.0;
      for (int q = threadIdx.x; q < F; q += blockDim.x) {
        const double dA = sw[q % P] * sw[q / P] * a.h[T1] * a.h[T2];
        const double lq = a.lam[f * F + q];
        gc[q] = dA * nD * lq;                       // <w . n, lambda>
        gc[F + q] = dA * a.tau * (lq - ul[q]);      // <v, tau (lambda - u)>
      }
      __syncthreads();
      sweep2<P>(sS, true, 1, gc, gt, 2);
      __syncthreads();
      sweep2<P>(sS, true, 0, gt, gc, 2);
      __syncthreads();
      for (int j = threadIdx.x; j < F; j += blockDim.x) {
        const int loc = layer_node<P>(D, s, j % P, j / P);
        B[D * N + loc] += gc[j];
        B[3 * N + loc] += gc[F + j];
      }
      __syncthreads();
    }
  }
  double* yc = a.y + (size_t)cell * 4 * N;
  for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) yc[t] = B[t];
}

}  // namespace

void launch_hdg_apply(const Level& L, double tau, double* lam,
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
  a.kinv = 1.0 / L.kappa;
  a.tau = tau;
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    for (int D = 0; D < 3; ++D) {
      int m[3] = {L.n[0], L.n[1], L.n[2]};
      m[D] += 1;
      k_hdg_trace<P><<<m[0] * m[1] * m[2], 64, 0, s>>>(a, D);
      MFP_CHECK_CUDA(cudaGetLastError());
      note_launch();
    }
    k_hdg_cell<P><<<(int)L.ncells, 128, 0, s>>>(a);
    MFP_CHECK_CUDA(cudaGetLastError());
    note_launch();
  });
}

}  // namespace mfp
