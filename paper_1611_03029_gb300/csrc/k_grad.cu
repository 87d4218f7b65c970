// Gradient of a solve-based loss with respect to the per-quadrature-point
// coefficient (not in the paper): with A(a) u = f and A lambda = u - u_t,
//   dL/da_q = -lambda^T (dA/da_q) u.
// Cell points: -(grad_xi lambda)^T G0_q (grad_xi u) with G0 = w det J
// J^{-1} J^{-T}, both reference gradients obtained by sum factorization
// (interpolate to the Gauss points, then collocation derivatives).
// Face points (SIPG, Eq. 6/7): minus the face form at that point with the
// coefficient replaced by one.
#include "dev_tables.cuh"

namespace mfp {
namespace {

struct GradArgs {
  int n[3];
  int g[3];
  int face_off[3];
  Bc bc;  // constrained CG nodes; SIPG faces on Neumann sides
  int disc;
  bool curved;
  double gs[3], ns[3], fa[3], sg[3];
  const double* G;
  const double* fdata;
  const double* sigma;
};

// One block per cell; every stage gives each thread whole output points.
template <int P>
__global__ void k_grad_cells(GradArgs a, const double* __restrict__ u,
                             const double* __restrict__ lam,
                             double* __restrict__ gc) {
  constexpr int P3 = P * P * P;
  __shared__ double sS[P * P], sD[P * P], sw[P];
  __shared__ double f0[2][P3], f1[2][P3], gy[2][P3], gz[2][P3];
  double(*gx)[P3] = f0;  // f0 is free once the values are in f1
  const int cell = blockIdx.x;
  const int cx = cell % a.n[0], cy = (cell / a.n[0]) % a.n[1],
            cz = cell / (a.n[0] * a.n[1]);
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    sS[i] = c_tab64[P - 2].S[i];
    sD[i] = c_tab64[P - 2].D[i];
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) sw[i] = c_tab64[P - 2].w[i];
  for (int i = threadIdx.x; i < P3; i += blockDim.x) {
    const int ix = i % P, iy = (i / P) % P, iz = i / (P * P);
    double vu, vl;
    if (a.disc == MFP_SIPG) {
      vu = u[(size_t)cell * P3 + i];
      vl = lam[(size_t)cell * P3 + i];
    } else {
      const int X = cx * (P - 1) + ix, Y = cy * (P - 1) + iy,
                Z = cz * (P - 1) + iz;
      const bool con = bc_con(a.bc, X, Y, Z);
      const size_t gi = (size_t)X + (size_t)a.g[0] * (Y + (size_t)a.g[1] * Z);
      vu = con ? 0.0 : u[gi];
      vl = con ? 0.0 : lam[gi];
    }
    f0[0][i] = vu;
    f0[1][i] = vl;
  }
  __syncthreads();
  // values at Gauss points: x, y, z sweeps (f0 -> f1 -> f0 -> f1)
  for (int i = threadIdx.x; i < 2 * P3; i += blockDim.x) {
    const int fld = i / P3, q = i % P3, qx = q % P, r = q / P;
    double s = 0;
    for (int j = 0; j < P; ++j) s += sS[qx * P + j] * f0[fld][j + P * r];
    f1[fld][q] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * P3; i += blockDim.x) {
    const int fld = i / P3, q = i % P3, qx = q % P, qy = (q / P) % P,
              qz = q / (P * P);
    double s = 0;
    for (int j = 0; j < P; ++j)
      s += sS[qy * P + j] * f1[fld][qx + P * (j + P * qz)];
    f0[fld][q] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * P3; i += blockDim.x) {
    const int fld = i / P3, q = i % P3, qx = q % P, qy = (q / P) % P,
              qz = q / (P * P);
    double s = 0;
    for (int j = 0; j < P; ++j)
      s += sS[qz * P + j] * f0[fld][qx + P * (qy + P * j)];
    f1[fld][q] = s;
  }
  __syncthreads();
  // collocation derivatives at the Gauss points
  for (int i = threadIdx.x; i < 2 * P3; i += blockDim.x) {
    const int fld = i / P3, q = i % P3, qx = q % P, qy = (q / P) % P,
              qz = q / (P * P);
    double sx = 0, sy = 0, sz = 0;
    for (int j = 0; j < P; ++j) {
      sx += sD[qx * P + j] * f1[fld][j + P * (qy + P * qz)];
      sy += sD[qy * P + j] * f1[fld][qx + P * (j + P * qz)];
      sz += sD[qz * P + j] * f1[fld][qx + P * (qy + P * j)];
    }
    gx[fld][q] = sx;
    gy[fld][q] = sy;
    gz[fld][q] = sz;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < P3; q += blockDim.x) {
    const double ux = gx[0][q], uy = gy[0][q], uz = gz[0][q];
    const double lx = gx[1][q], ly = gy[1][q], lz = gz[1][q];
    double v;
    if (a.curved) {
      const double* Gp = a.G + (size_t)cell * 6 * P3 + q;
      const double g0 = Gp[0], g1 = Gp[P3], g2 = Gp[2 * P3], g3 = Gp[3 * P3],
                   g4 = Gp[4 * P3], g5 = Gp[5 * P3];
      v = lx * (g0 * ux + g1 * uy + g2 * uz) + ly * (g1 * ux + g3 * uy + g4 * uz) +
          lz * (g2 * ux + g4 * uy + g5 * uz);
    } else {
      const double w = sw[q % P] * sw[(q / P) % P] * sw[q / (P * P)];
      v = w * (a.gs[0] * lx * ux + a.gs[1] * ly * uy + a.gs[2] * lz * uz);
    }
    gc[(size_t)cell * P3 + q] = -v;
  }
}

// One block per face of axis D; one thread per face point.  Values and
// reference gradients of u and lambda on each side by direct sums of the
// 1D tables over the cell's nodes.
template <int P>
__global__ void k_grad_faces(GradArgs a, int D, const double* __restrict__ u,
                             const double* __restrict__ lam,
                             double* __restrict__ gf) {
  constexpr int P2 = P * P, P3 = P2 * P;
  __shared__ double sS[P * P], sDphi[P * P], s0[P], s1[P], sw[P];
  __shared__ double nodes[2][2][P3];  // side, field
  int m[3] = {a.n[0], a.n[1], a.n[2]};
  m[D] += 1;
  const int fl = blockIdx.x;
  const int fc[3] = {fl % m[0], (fl / m[0]) % m[1], fl / (m[0] * m[1])};
  const bool hasL = fc[D] >= 1, hasR = fc[D] < a.n[D];
  int cL[3] = {fc[0], fc[1], fc[2]};
  cL[D] -= 1;
  const int cellL = hasL ? cL[0] + a.n[0] * (cL[1] + a.n[1] * cL[2]) : 0;
  const int cellR = hasR ? fc[0] + a.n[0] * (fc[1] + a.n[1] * fc[2]) : 0;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    sS[i] = c_tab64[P - 2].S[i];
    sDphi[i] = c_tab64[P - 2].Dphi[i];
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    s0[i] = c_tab64[P - 2].dphi0[i];
    s1[i] = c_tab64[P - 2].dphi1[i];
    sw[i] = c_tab64[P - 2].w[i];
  }
  for (int i = threadIdx.x; i < P3; i += blockDim.x) {
    nodes[0][0][i] = hasL ? u[(size_t)cellL * P3 + i] : 0.0;
    nodes[0][1][i] = hasL ? lam[(size_t)cellL * P3 + i] : 0.0;
    nodes[1][0][i] = hasR ? u[(size_t)cellR * P3 + i] : 0.0;
    nodes[1][1][i] = hasR ? lam[(size_t)cellR * P3 + i] : 0.0;
  }
  __syncthreads();
  const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
  const size_t f = (size_t)a.face_off[D] + fl;
  for (int q = threadIdx.x; q < P2; q += blockDim.x) {
    const int qa = q % P, qb = q / P;
    double val[2][2], dn[2][2];  // [side][field], dn along +D normal
    for (int side = 0; side < 2; ++side) {
      const bool has = side == 0 ? hasL : hasR;
      const double* sl = side == 0 ? s1 : s0;  // slope at the face
      const int lay = side == 0 ? P - 1 : 0;
      for (int fld = 0; fld < 2; ++fld) {
        double v = 0, gD = 0, g1 = 0, g2 = 0;
        if (has) {
          const double* nd = nodes[side][fld];
          for (int l = 0; l < P; ++l)
            for (int j = 0; j < P; ++j)
              for (int mm = 0; mm < P; ++mm) {
                int idx[3];
                idx[D] = l;
                idx[T1] = j;
                idx[T2] = mm;
                const double x = nd[idx[0] + P * (idx[1] + P * idx[2])];
                const double ss = sS[qa * P + j] * sS[qb * P + mm];
                gD += sl[l] * ss * x;
                if (l == lay) {
                  v += ss * x;
                  g1 += sDphi[qa * P + j] * sS[qb * P + mm] * x;
                  g2 += sS[qa * P + j] * sDphi[qb * P + mm] * x;
                }
              }
        }
        double dnv;
        if (!a.curved) {
          dnv = a.ns[D] * gD;
        } else {
          const double* fd = a.fdata + f * 7 * P2;
          const int off = side == 0 ? 1 : 4;
          double gr[3];
          gr[D] = gD;
          gr[T1] = g1;
          gr[T2] = g2;
          dnv = fd[(off + 0) * P2 + q] * gr[0] + fd[(off + 1) * P2 + q] * gr[1] +
                fd[(off + 2) * P2 + q] * gr[2];
        }
        val[side][fld] = v;
        dn[side][fld] = dnv;
      }
    }
    double dA, sig;
    if (!a.curved) {
      dA = sw[qa] * sw[qb] * a.fa[D];
      sig = a.sg[D];
    } else {
      dA = a.fdata[f * 7 * P2 + q];
      sig = a.sigma[f];
    }
    double form;
    if (hasL && hasR) {
      const double ju = val[0][0] - val[1][0], jl = val[0][1] - val[1][1];
      const double au = 0.5 * (dn[0][0] + dn[1][0]);
      const double al = 0.5 * (dn[0][1] + dn[1][1]);
      form = -jl * au - al * ju + sig * jl * ju;
    } else {
      const int sd = hasL ? 0 : 1;
      const double sgn = hasL ? 1.0 : -1.0;  // own outward normal
      const double uu = val[sd][0], ll = val[sd][1];
      const double du = sgn * dn[sd][0], dl = sgn * dn[sd][1];
      form = -ll * du - uu * dl + 2.0 * sig * ll * uu;
      // a face on a Neumann side has no term of the form (Eq. 7)
      if ((a.bc.neumann >> (2 * D + (hasL ? 1 : 0))) & 1) form = 0.0;
    }
    gf[f * P2 + q] = -dA * form;
  }
}

}  // namespace

void launch_gradient(const Level& L, const double* u, const double* lam,
                     double* gc, double* gf, cudaStream_t s) {
  ensure_tables();
  GradArgs a{};
  for (int d = 0; d < 3; ++d) {
    a.n[d] = L.n[d];
    a.g[d] = L.gdim[d];
    a.face_off[d] = L.face_off[d];
  }
  a.bc = L.bc;
  a.disc = L.disc;
  a.curved = L.curved;
  const double vol = L.h[0] * L.h[1] * L.h[2];
  const double pen = L.penalty * (double)L.p * L.p;
  for (int d = 0; d < 3; ++d) {
    a.gs[d] = vol / (L.h[d] * L.h[d]);
    a.ns[d] = 1.0 / L.h[d];
    a.fa[d] = vol / L.h[d];
    a.sg[d] = pen / L.h[d];
  }
  a.G = L.d64.G;
  a.fdata = L.d64.fdata;
  a.sigma = L.d64.sigma;
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    k_grad_cells<P><<<(int)L.ncells, 256, 0, s>>>(a, u, lam, gc);
    MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
    if (L.disc == MFP_SIPG && gf) {
      for (int D = 0; D < 3; ++D) {
        int m[3] = {L.n[0], L.n[1], L.n[2]};
        m[D] += 1;
        k_grad_faces<P><<<m[0] * m[1] * m[2], ((P * P + 31) / 32) * 32, 0, s>>>(
            a, D, u, lam, gf);
        MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
      }
    }
  });
}

}  // namespace mfp
