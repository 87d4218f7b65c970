// Setup kernels: isoparametric geometry at quadrature points (Sec. 2,
// Sec. 3 "pre-compute the Jacobian on all quadrature points"), the Jacobi
// diagonal (Sec. 4.1), the load vector (Eq. 4 / Eq. 6 right-hand side) and
// the coarse-level coefficient.  These run once per context (or per
// coefficient change), so they favour plain per-point sums over speed.
#include "dev_tables.cuh"

namespace mfp {
namespace {

struct GeoArgs {
  int n[3];
  int p;
  double h[3];  // cell size on the unit cube (1 / n)
  double amp;
  double lo, len;  // then x -> lo + len x onto the box [lo, lo + len]^3
  const double* nodes;  // given support points [ncells][p^3][3], or null
};

// All tables of degree P-1 in shared memory.
template <int P>
struct ShTab {
  double S[P * P], D[P * P], Dphi[P * P], d0[P], d1[P], w[P], g[P], x[P];
};

template <int P>
__device__ void load_shtab(ShTab<P>& t) {
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    t.S[i] = c_tab64[P - 2].S[i];
    t.D[i] = c_tab64[P - 2].D[i];
    t.Dphi[i] = c_tab64[P - 2].Dphi[i];
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    t.d0[i] = c_tab64[P - 2].dphi0[i];
    t.d1[i] = c_tab64[P - 2].dphi1[i];
    t.w[i] = c_tab64[P - 2].w[i];
    t.g[i] = c_tab64[P - 2].g[i];
    t.x[i] = c_tab64[P - 2].x[i];
  }
}

// The analytic map of the unit cube (identity or sine bump).
__device__ __forceinline__ void phi_map(double amp, double& x, double& y,
                                        double& z) {
  if (amp != 0.0) {
    const double s = sinpi(x) * sinpi(y) * sinpi(z);
    x += amp * s;
    y += amp * s;
    z += amp * s;
  }
}

// Support points (images of the GLL nodes) of cell (cx,cy,cz) into X[p^3][3]:
// the given nodes, or the analytic map at the cell's GLL grid.
template <int P>
__device__ void support_points(const GeoArgs& g, const ShTab<P>& t, int cx,
                               int cy, int cz, double* X) {
  if (g.nodes) {
    const size_t cell = cx + (size_t)g.n[0] * (cy + (size_t)g.n[1] * cz);
    const double* src = g.nodes + cell * 3 * P * P * P;
    for (int i = threadIdx.x; i < 3 * P * P * P; i += blockDim.x)
      X[i] = src[i];
    return;
  }
  for (int a = threadIdx.x; a < P * P * P; a += blockDim.x) {
    const int ax = a % P, ay = (a / P) % P, az = a / (P * P);
    double x = (cx + t.x[ax]) * g.h[0];
    double y = (cy + t.x[ay]) * g.h[1];
    double z = (cz + t.x[az]) * g.h[2];
    phi_map(g.amp, x, y, z);
    X[3 * a] = g.lo + g.len * x;
    X[3 * a + 1] = g.lo + g.len * y;
    X[3 * a + 2] = g.lo + g.len * z;
  }
}

// Jacobian J[d][e] = dx_d / dxi_e of the interpolated map at a reference
// point given by 1D basis values / slopes per axis (v[e][j], s[e][j]).
template <int P>
__device__ void jacobian(const double* X, const double (&v)[3][P],
                         const double (&s)[3][P], double (&J)[3][3],
                         double (&x)[3]) {
  for (int d = 0; d < 3; ++d) {
    x[d] = 0;
    for (int e = 0; e < 3; ++e) J[d][e] = 0;
  }
  for (int az = 0; az < P; ++az)
    for (int ay = 0; ay < P; ++ay)
      for (int ax = 0; ax < P; ++ax) {
        const int a = ax + P * (ay + P * az);
        const double bx = v[0][ax] * v[1][ay] * v[2][az];
        const double dx = s[0][ax] * v[1][ay] * v[2][az];
        const double dy = v[0][ax] * s[1][ay] * v[2][az];
        const double dz = v[0][ax] * v[1][ay] * s[2][az];
        for (int d = 0; d < 3; ++d) {
          const double X_ = X[3 * a + d];
          x[d] += X_ * bx;
          J[d][0] += X_ * dx;
          J[d][1] += X_ * dy;
          J[d][2] += X_ * dz;
        }
      }
}

__device__ __forceinline__ double inv3(const double (&J)[3][3],
                                       double (&I)[3][3]) {
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const double id = 1.0 / det;
  I[0][0] = c00 * id;
  I[1][0] = c01 * id;
  I[2][0] = c02 * id;
  I[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  I[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  I[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  I[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  I[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  I[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  return det;
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (blockDim.x + 31) / 32; ++i) s += red[i];
  return s;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// Curved cells: G_q = w_q det J J^{-1} J^{-T} (6 entries, no coefficient)
// and the cell volume.  One block per cell, one thread per point.
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_cell_geometry(GeoArgs g, double* G, float* G32,
                                double* vol, int* bad, double* hdg) {
  constexpr int P3 = P * P * P;
  __shared__ ShTab<P> t;
  __shared__ double X[3 * P3];
  __shared__ double red[32];
  const int cell = blockIdx.x;
  const int cx = cell % g.n[0], cy = (cell / g.n[0]) % g.n[1],
            cz = cell / (g.n[0] * g.n[1]);
  load_shtab<P>(t);
  __syncthreads();
  support_points<P>(g, t, cx, cy, cz, X);
  __syncthreads();
  double wdet = 0;
  for (int q = threadIdx.x; q < P3; q += blockDim.x) {
    const int qx = q % P, qy = (q / P) % P, qz = q / (P * P);
    double v[3][P], s[3][P];
    const int qq[3] = {qx, qy, qz};
    for (int e = 0; e < 3; ++e)
      for (int j = 0; j < P; ++j) {
        v[e][j] = t.S[qq[e] * P + j];
        s[e][j] = t.Dphi[qq[e] * P + j];
      }
    double J[3][3], x[3], I[3][3];
    jacobian<P>(X, v, s, J, x);
    const double det = inv3(J, I);
    if (!(det > 0)) atomicExch(bad, 1);
    const double w = t.w[qx] * t.w[qy] * t.w[qz] * det;
    wdet += w;
    // G = w det J^{-1} J^{-T}: G_ef = sum_d I[e][d] I[f][d]
    double Gm[6];
    int c = 0;
    for (int e = 0; e < 3; ++e)
      for (int f = e; f < 3; ++f)
        Gm[c++] = w * (I[e][0] * I[f][0] + I[e][1] * I[f][1] +
                       I[e][2] * I[f][2]);
    for (int c2 = 0; c2 < 6; ++c2) {
      G[((size_t)cell * 6 + c2) * P3 + q] = Gm[c2];
      if (G32) G32[((size_t)cell * 6 + c2) * P3 + q] = (float)Gm[c2];
    }
    if (hdg) {  // HDG mixed operator: w det J and J^{-1} [e][d] per point
      double* o = hdg + (size_t)cell * 10 * P3 + q;
      o[0] = w;
      for (int e = 0; e < 3; ++e)
        for (int d = 0; d < 3; ++d) o[(1 + 3 * e + d) * P3] = I[e][d];
    }
  }
  const double sum = block_sum(wdet, red);
  if (threadIdx.x == 0) vol[cell] = sum;
}

// ---------------------------------------------------------------------------
// Curved SIPG faces: per face point dA = det J |J^{-T} e_D| w_a w_b,
// n = J^{-T} e_D / |.| (pointing along +D), nJ_L = J_L^{-1} n,
// nJ_R = J_R^{-1} n; sigma_F from |F| and the cell volumes.
// One block per face, one thread per face point.
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_face_geometry(GeoArgs g, int D, int face_off,
                                double penalty, const double* vol,
                                double* fdata, float* fdata32, double* sigma,
                                float* sigma32, double* hdg) {
  constexpr int P2 = P * P, P3 = P2 * P;
  __shared__ ShTab<P> t;
  __shared__ double XL[3 * P3], XR[3 * P3];
  __shared__ double red[32];
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[D] += 1;
  const int fl = blockIdx.x;
  int fc[3] = {fl % m[0], (fl / m[0]) % m[1], fl / (m[0] * m[1])};
  const bool hasL = fc[D] >= 1, hasR = fc[D] < g.n[D];
  int cL[3] = {fc[0], fc[1], fc[2]};
  cL[D] -= 1;
  load_shtab<P>(t);
  __syncthreads();
  if (hasL) support_points<P>(g, t, cL[0], cL[1], cL[2], XL);
  if (hasR) support_points<P>(g, t, fc[0], fc[1], fc[2], XR);
  __syncthreads();
  const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
  double area = 0;
  const size_t f = (size_t)face_off + fl;
  for (int q = threadIdx.x; q < P2; q += blockDim.x) {
    const int qa = q % P, qb = q / P;
    double nJ[2][3] = {{0, 0, 0}, {0, 0, 0}};
    double n[3] = {0, 0, 0}, dA = 0;
    for (int side = 0; side < 2; ++side) {
      const bool has = side == 0 ? hasL : hasR;
      if (!has) continue;
      double v[3][P], s[3][P];
      for (int j = 0; j < P; ++j) {
        v[D][j] = (side == 0) ? (j == P - 1 ? 1.0 : 0.0) : (j == 0 ? 1.0 : 0.0);
        s[D][j] = (side == 0) ? t.d1[j] : t.d0[j];
        v[T1][j] = t.S[qa * P + j];
        s[T1][j] = t.Dphi[qa * P + j];
        v[T2][j] = t.S[qb * P + j];
        s[T2][j] = t.Dphi[qb * P + j];
      }
      double J[3][3], x[3], I[3][3];
      jacobian<P>(side == 0 ? XL : XR, v, s, J, x);
      const double det = inv3(J, I);
      // J^{-T} e_D = row D of J^{-1}
      const double c0 = I[D][0], c1 = I[D][1], c2 = I[D][2];
      const double len = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
      if (side == 0 || !hasL) {
        n[0] = c0 / len;
        n[1] = c1 / len;
        n[2] = c2 / len;
        dA = det * len * t.w[qa] * t.w[qb];
      }
      for (int e = 0; e < 3; ++e)
        nJ[side][e] = I[e][0] * n[0] + I[e][1] * n[1] + I[e][2] * n[2];
    }
    area += dA;
    double out[7] = {dA, nJ[0][0], nJ[0][1], nJ[0][2],
                     nJ[1][0], nJ[1][1], nJ[1][2]};
    for (int c = 0; c < 7; ++c) {
      fdata[(f * 7 + c) * P2 + q] = out[c];
      if (fdata32) fdata32[(f * 7 + c) * P2 + q] = (float)out[c];
    }
    if (hdg) {  // HDG: area element and the unit normal along +e_D
      hdg[(f * 4 + 0) * P2 + q] = dA;
      for (int e = 0; e < 3; ++e) hdg[(f * 4 + 1 + e) * P2 + q] = n[e];
    }
  }
  const double A = block_sum(area, red);
  if (threadIdx.x == 0) {
    const int cl = cL[0] + g.n[0] * (cL[1] + g.n[1] * cL[2]);
    const int cr = fc[0] + g.n[0] * (fc[1] + g.n[1] * fc[2]);
    double inv_h;
    if (hasL && hasR)
      inv_h = 0.5 * (A / vol[cl] + A / vol[cr]);
    else
      inv_h = A / vol[hasL ? cl : cr];
    const double sg = penalty * P * P * inv_h;
    sigma[f] = sg;
    if (sigma32) sigma32[f] = (float)sg;
  }
}

// ---------------------------------------------------------------------------
// Jacobi diagonal in float64: cell part sum_q grad phi_i . G_q grad phi_i
// and, for SIPG, the own-side face terms.  One block per cell, one thread
// per node; CG accumulates with atomics.
// ---------------------------------------------------------------------------
struct DiagArgs {
  int n[3];
  int g[3];
  int face_off[3];
  Bc bc;
  int disc;
  bool curved;
  double kappa;
  double gs[3], ns[3], fa[3], sg[3];
  const double* G;
  const double* kcell;
  const double* kface;
  const double* fdata;
  const double* sigma;
};

template <int P>
__global__ void k_diagonal(DiagArgs a, double* diag) {
  constexpr int P2 = P * P, P3 = P2 * P;
  __shared__ ShTab<P> t;
  const int cell = blockIdx.x;
  const int cx = cell % a.n[0], cy = (cell / a.n[0]) % a.n[1],
            cz = cell / (a.n[0] * a.n[1]);
  load_shtab<P>(t);
  __syncthreads();
  for (int i = threadIdx.x; i < P3; i += blockDim.x) {
    const int ix = i % P, iy = (i / P) % P, iz = i / (P * P);
    double acc = 0;
    for (int q = 0; q < P3; ++q) {
      const int qx = q % P, qy = (q / P) % P, qz = q / (P * P);
      const double vx = t.S[qx * P + ix], vy = t.S[qy * P + iy],
                   vz = t.S[qz * P + iz];
      const double gx = t.Dphi[qx * P + ix] * vy * vz;
      const double gy = vx * t.Dphi[qy * P + iy] * vz;
      const double gz = vx * vy * t.Dphi[qz * P + iz];
      const double kap = a.kcell ? a.kcell[(size_t)cell * P3 + q] : a.kappa;
      if (a.curved) {
        const double* Gp = a.G + (size_t)cell * 6 * P3 + q;
        const double g0 = Gp[0], g1 = Gp[P3], g2 = Gp[2 * P3],
                     g3 = Gp[3 * P3], g4 = Gp[4 * P3], g5 = Gp[5 * P3];
        acc += kap * (gx * (g0 * gx + g1 * gy + g2 * gz) +
                      gy * (g1 * gx + g3 * gy + g4 * gz) +
                      gz * (g2 * gx + g4 * gy + g5 * gz));
      } else {
        const double w = t.w[qx] * t.w[qy] * t.w[qz] * kap;
        acc += w * (a.gs[0] * gx * gx + a.gs[1] * gy * gy + a.gs[2] * gz * gz);
      }
    }
    if (a.disc == MFP_SIPG) {
      const int ii[3] = {ix, iy, iz};
      const int cc[3] = {cx, cy, cz};
      for (int D = 0; D < 3; ++D) {
        const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
        int m[3] = {a.n[0], a.n[1], a.n[2]};
        m[D] += 1;
        for (int S = 0; S < 2; ++S) {
          int fc[3] = {cc[0], cc[1], cc[2]};
          fc[D] += S;
          const size_t f = a.face_off[D] + fc[0] + m[0] * (fc[1] + m[1] * fc[2]);
          const bool bnd = (S == 0 && cc[D] == 0) || (S == 1 && cc[D] == a.n[D] - 1);
          if (bnd && ((a.bc.neumann >> (2 * D + S)) & 1)) continue;  // Neumann
          const int lo = S ? P - 1 : 0;
          const double* dS = S ? t.d1 : t.d0;
          const bool onface = ii[D] == lo;
          for (int q = 0; q < P2; ++q) {
            const int qa = q % P, qb = q / P;
            const double va = t.S[qa * P + ii[T1]], vb = t.S[qb * P + ii[T2]];
            const double phi = onface ? va * vb : 0.0;
            double gref[3];
            gref[D] = dS[ii[D]] * va * vb;
            gref[T1] = onface ? t.Dphi[qa * P + ii[T1]] * vb : 0.0;
            gref[T2] = onface ? va * t.Dphi[qb * P + ii[T2]] : 0.0;
            double dn, dA, sig;
            if (!a.curved) {
              dn = (S ? 1.0 : -1.0) * a.ns[D] * gref[D];
              dA = t.w[qa] * t.w[qb] * a.fa[D];
              sig = a.sg[D];
            } else {
              const double* fd = a.fdata + f * 7 * P2;
              dA = fd[q];
              sig = a.sigma[f];
              const int off = S ? 1 : 4;
              const double sgn = S ? 1.0 : -1.0;
              dn = sgn * (fd[(off + 0) * P2 + q] * gref[0] +
                          fd[(off + 1) * P2 + q] * gref[1] +
                          fd[(off + 2) * P2 + q] * gref[2]);
            }
            const double kap = a.kface ? a.kface[f * P2 + q] : a.kappa;
            const double c = kap * dA * (sig * phi * phi - phi * dn);
            acc += bnd ? 2.0 * c : c;
          }
        }
      }
      diag[(size_t)cell * P3 + i] = acc;
    } else {
      const int X = cx * (P - 1) + ix, Y = cy * (P - 1) + iy,
                Z = cz * (P - 1) + iz;
      const bool con = bc_con(a.bc, X, Y, Z);
      if (!con)
        atomicAdd(diag + (size_t)X + (size_t)a.g[0] * (Y + (size_t)a.g[1] * Z),
                  acc);
    }
  }
}

// ---------------------------------------------------------------------------
// Load vector b_i = sum_q w_q det J f(x_q) phi_i(x_q).
// ---------------------------------------------------------------------------
struct RhsArgs {
  GeoArgs geo;
  int g[3];
  int disc;
  int kind;
  int nterms;
  const double* params;  // device copy, nterms * 5
  int64_t stride;
  Bc bc;
  double kappa;           // constant coefficient (kind 2)
  int face_off[3];
  const double* sigma;    // curved SIPG: penalty per face
  double sg[3];           // Cartesian SIPG: penalty of a d-face
};

// kind 2: u = sum_j A_j exp(-|x - c_j|^2 / w_j^2); returns u(x) and grad u.
__device__ double gauss_sum(const RhsArgs& a, const double (&x)[3],
                            double (&gr)[3]) {
  double u = 0;
  gr[0] = gr[1] = gr[2] = 0;
  for (int j = 0; j < a.nterms; ++j) {
    const double* c = a.params + 5 * j;
    const double dx = x[0] - c[0], dy = x[1] - c[1], dz = x[2] - c[2];
    const double iw2 = 1.0 / (c[3] * c[3]);
    const double e = c[4] * exp(-(dx * dx + dy * dy + dz * dz) * iw2);
    u += e;
    gr[0] -= 2.0 * iw2 * dx * e;
    gr[1] -= 2.0 * iw2 * dy * e;
    gr[2] -= 2.0 * iw2 * dz * e;
  }
  return u;
}

__device__ double forcing(const RhsArgs& a, double x, double y, double z) {
  if (a.kind == 0) {
    const double pi2 = 9.869604401089358;
    return 3.0 * pi2 * sinpi(x) * sinpi(y) * sinpi(z);
  }
  double f = 0;
  for (int j = 0; j < a.nterms; ++j) {
    const double* c = a.params + 5 * j;
    const double dx = x - c[0], dy = y - c[1], dz = z - c[2];
    if (a.kind == 1) {
      f += c[4] * exp(-(dx * dx + dy * dy + dz * dz) / (c[3] * c[3]));
    } else {
      // kind 2: f = -kappa Laplace u, Laplace of exp(-r^2/w^2) in 3D being
      // (4 r^2 / w^2 - 6) / w^2 times the exponential
      const double iw2 = 1.0 / (c[3] * c[3]);
      const double r2 = (dx * dx + dy * dy + dz * dz) * iw2;
      f += a.kappa * iw2 * (6.0 - 4.0 * r2) * c[4] * exp(-r2);
    }
  }
  return f;
}

template <int P>
__global__ void k_rhs(RhsArgs a, double* b) {
  constexpr int P3 = P * P * P;
  __shared__ ShTab<P> t;
  __shared__ double X[3 * P3];
  __shared__ double F[P3];
  const GeoArgs& g = a.geo;
  const int cell = blockIdx.x;
  const int cx = cell % g.n[0], cy = (cell / g.n[0]) % g.n[1],
            cz = cell / (g.n[0] * g.n[1]);
  load_shtab<P>(t);
  __syncthreads();
  const bool curved = g.amp != 0.0 || g.nodes != nullptr;
  if (curved) support_points<P>(g, t, cx, cy, cz, X);
  __syncthreads();
  for (int q = threadIdx.x; q < P3; q += blockDim.x) {
    const int qx = q % P, qy = (q / P) % P, qz = q / (P * P);
    double x[3], wdet;
    if (curved) {
      double v[3][P], s[3][P];
      const int qq[3] = {qx, qy, qz};
      for (int e = 0; e < 3; ++e)
        for (int j = 0; j < P; ++j) {
          v[e][j] = t.S[qq[e] * P + j];
          s[e][j] = t.Dphi[qq[e] * P + j];
        }
      double J[3][3], I[3][3];
      jacobian<P>(X, v, s, J, x);
      wdet = inv3(J, I);
    } else {
      x[0] = g.lo + g.len * (cx + t.g[qx]) * g.h[0];
      x[1] = g.lo + g.len * (cy + t.g[qy]) * g.h[1];
      x[2] = g.lo + g.len * (cz + t.g[qz]) * g.h[2];
      wdet = g.len * g.len * g.len * g.h[0] * g.h[1] * g.h[2];
    }
    wdet *= t.w[qx] * t.w[qy] * t.w[qz];
    F[q] = wdet * forcing(a, x[0], x[1], x[2]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P3; i += blockDim.x) {
    const int ix = i % P, iy = (i / P) % P, iz = i / (P * P);
    double acc = 0;
    for (int q = 0; q < P3; ++q) {
      const int qx = q % P, qy = (q / P) % P, qz = q / (P * P);
      acc += t.S[qx * P + ix] * t.S[qy * P + iy] * t.S[qz * P + iz] * F[q];
    }
    if (a.disc == MFP_SIPG) {
      b[((size_t)cell * P3 + i) * a.stride] = acc;
    } else {
      const int X_ = cx * (P - 1) + ix, Y = cy * (P - 1) + iy,
                Z = cz * (P - 1) + iz;
      const bool con = bc_con(a.bc, X_, Y, Z);
      if (!con)
        atomicAdd(b + ((size_t)X_ + (size_t)a.g[0] * (Y + (size_t)a.g[1] * Z)) *
                          a.stride,
                  acc);
    }
  }
}

// kind 2, CG: Dirichlet data on the constrained nodes, lifted out of the
// free rows (Sec. 2.1): a constrained row takes the data value at its node,
// a free row i loses a(g_h, phi_i) with g_h the cell's interpolant of the
// data on its constrained nodes, i.e. sum_q grad_xi phi_i . M_q grad_xi g_h
// with M_q = w_q det J kappa J^{-1} J^{-T}.  Runs after k_rhs.
template <int P>
__global__ void k_rhs_lift(RhsArgs a, double* b) {
  constexpr int P3 = P * P * P;
  __shared__ ShTab<P> t;
  __shared__ double X[3 * P3];
  __shared__ double gN[P3];
  __shared__ double Fl[3 * P3];
  const GeoArgs& g = a.geo;
  const int cell = blockIdx.x;
  const int c3[3] = {cell % g.n[0], (cell / g.n[0]) % g.n[1],
                     cell / (g.n[0] * g.n[1])};
  // only cells with a node on a Dirichlet side (uniform over the block)
  bool touch = false;
  for (int d = 0; d < 3; ++d)
    touch = touch || (c3[d] == 0 && a.bc.lo[d] == 0) ||
            (c3[d] == g.n[d] - 1 && a.bc.hi[d] >= 0);
  if (!touch) return;
  load_shtab<P>(t);
  __syncthreads();
  const bool curved = g.amp != 0.0 || g.nodes != nullptr;
  if (curved) support_points<P>(g, t, c3[0], c3[1], c3[2], X);
  __syncthreads();
  for (int i = threadIdx.x; i < P3; i += blockDim.x) {
    const int ii[3] = {i % P, (i / P) % P, i / (P * P)};
    const int64_t N[3] = {(int64_t)c3[0] * (P - 1) + ii[0],
                          (int64_t)c3[1] * (P - 1) + ii[1],
                          (int64_t)c3[2] * (P - 1) + ii[2]};
    double v = 0;
    if (bc_con(a.bc, N[0], N[1], N[2])) {
      double x[3], gr[3];
      for (int d = 0; d < 3; ++d)
        x[d] = curved ? X[3 * i + d]
                      : g.lo + g.len * (c3[d] + t.x[ii[d]]) * g.h[d];
      v = gauss_sum(a, x, gr);
      b[(N[0] + (int64_t)a.g[0] * (N[1] + (int64_t)a.g[1] * N[2])) *
        a.stride] = v;  // the same value from every cell of the node
    }
    gN[i] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < P3; q += blockDim.x) {
    const int qq[3] = {q % P, (q / P) % P, q / (P * P)};
    double r[3] = {0, 0, 0};  // grad_xi g_h at the point
    for (int j = 0; j < P3; ++j) {
      const double gj = gN[j];
      if (gj == 0.0) continue;
      const int jx = j % P, jy = (j / P) % P, jz = j / (P * P);
      const double sx = t.S[qq[0] * P + jx], sy = t.S[qq[1] * P + jy],
                   sz = t.S[qq[2] * P + jz];
      r[0] += t.Dphi[qq[0] * P + jx] * sy * sz * gj;
      r[1] += sx * t.Dphi[qq[1] * P + jy] * sz * gj;
      r[2] += sx * sy * t.Dphi[qq[2] * P + jz] * gj;
    }
    const double w =
        t.w[qq[0]] * t.w[qq[1]] * t.w[qq[2]] * a.kappa;
    if (curved) {
      double v[3][P], s[3][P];
      for (int e = 0; e < 3; ++e)
        for (int j = 0; j < P; ++j) {
          v[e][j] = t.S[qq[e] * P + j];
          s[e][j] = t.Dphi[qq[e] * P + j];
        }
      double J[3][3], I[3][3], x[3];
      jacobian<P>(X, v, s, J, x);
      const double det = inv3(J, I);
      double pr[3];  // J^{-T} grad_xi g_h
      for (int d = 0; d < 3; ++d)
        pr[d] = I[0][d] * r[0] + I[1][d] * r[1] + I[2][d] * r[2];
      for (int e = 0; e < 3; ++e)
        Fl[3 * q + e] =
            w * det * (I[e][0] * pr[0] + I[e][1] * pr[1] + I[e][2] * pr[2]);
    } else {
      double H[3], det = 1;
      for (int d = 0; d < 3; ++d) {
        H[d] = g.len * g.h[d];
        det *= H[d];
      }
      for (int e = 0; e < 3; ++e) Fl[3 * q + e] = w * det * r[e] / (H[e] * H[e]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P3; i += blockDim.x) {
    const int ii[3] = {i % P, (i / P) % P, i / (P * P)};
    const int64_t N[3] = {(int64_t)c3[0] * (P - 1) + ii[0],
                          (int64_t)c3[1] * (P - 1) + ii[1],
                          (int64_t)c3[2] * (P - 1) + ii[2]};
    if (bc_con(a.bc, N[0], N[1], N[2])) continue;
    double acc = 0;
    for (int q = 0; q < P3; ++q) {
      const int qx = q % P, qy = (q / P) % P, qz = q / (P * P);
      const double sx = t.S[qx * P + ii[0]], sy = t.S[qy * P + ii[1]],
                   sz = t.S[qz * P + ii[2]];
      acc += t.Dphi[qx * P + ii[0]] * sy * sz * Fl[3 * q] +
             sx * t.Dphi[qy * P + ii[1]] * sz * Fl[3 * q + 1] +
             sx * sy * t.Dphi[qz * P + ii[2]] * Fl[3 * q + 2];
    }
    atomicAdd(b + (N[0] + (int64_t)a.g[0] * (N[1] + (int64_t)a.g[1] * N[2])) *
                      a.stride,
              -acc);
  }
}

// kind 2: boundary data on the faces of side `side` (x_D = lo for side 2D,
// hi for 2D + 1), one block per face, one cell per face (so SIPG adds
// without atomics; the sides go in separate launches).
//  - Neumann side: the natural term int phi_i kappa grad u . n ds (Eq. 1
//    with Neumann data; SIPG: the only term Eq. 7 leaves on such a face).
//  - SIPG Dirichlet side: the data part of the extension u+ = 2 g - u- of
//    Eq. 7, kappa dA (2 sigma g phi_i - g d_n phi_i).
template <int P>
__global__ void k_rhs_face(RhsArgs a, int side, double* b) {
  constexpr int P2 = P * P, P3 = P2 * P;
  __shared__ ShTab<P> t;
  __shared__ double X[3 * P3];
  __shared__ double cv[P2], cm[3 * P2];
  const GeoArgs& g = a.geo;
  const int D = side / 2, s = side % 2;
  const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
  const bool neu = (a.bc.neumann >> side) & 1;
  int c3[3];
  c3[D] = s ? g.n[D] - 1 : 0;
  c3[T1] = blockIdx.x % g.n[T1];
  c3[T2] = blockIdx.x / g.n[T1];
  const int cell = c3[0] + g.n[0] * (c3[1] + g.n[1] * c3[2]);
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[D] += 1;
  int fc[3] = {c3[0], c3[1], c3[2]};
  fc[D] += s;
  const int64_t f =
      a.face_off[D] + fc[0] + (int64_t)m[0] * (fc[1] + (int64_t)m[1] * fc[2]);
  load_shtab<P>(t);
  __syncthreads();
  const bool curved = g.amp != 0.0 || g.nodes != nullptr;
  if (curved) support_points<P>(g, t, c3[0], c3[1], c3[2], X);
  __syncthreads();
  const double* dS = s ? t.d1 : t.d0;  // GLL basis slopes at the cell end
  const int end = s ? P - 1 : 0;
  for (int q = threadIdx.x; q < P2; q += blockDim.x) {
    const int qa = q % P, qb = q / P;
    double x[3], I[3][3], det;
    if (curved) {
      double v[3][P], sl[3][P];
      for (int j = 0; j < P; ++j) {
        v[D][j] = j == end ? 1.0 : 0.0;
        sl[D][j] = dS[j];
        v[T1][j] = t.S[qa * P + j];
        sl[T1][j] = t.Dphi[qa * P + j];
        v[T2][j] = t.S[qb * P + j];
        sl[T2][j] = t.Dphi[qb * P + j];
      }
      double J[3][3];
      jacobian<P>(X, v, sl, J, x);
      det = inv3(J, I);
    } else {
      double r[3];
      r[D] = s;
      r[T1] = t.g[qa];
      r[T2] = t.g[qb];
      det = 1;
      for (int d = 0; d < 3; ++d) {
        const double H = g.len * g.h[d];
        x[d] = g.lo + H * (c3[d] + r[d]);
        for (int e = 0; e < 3; ++e) I[d][e] = d == e ? 1.0 / H : 0.0;
        det *= H;
      }
    }
    // outward unit normal: +-(row D of J^{-1}) normalised; area element
    const double nl = sqrt(I[D][0] * I[D][0] + I[D][1] * I[D][1] +
                           I[D][2] * I[D][2]);
    const double sg = s ? 1.0 : -1.0;
    double n[3];
    for (int d = 0; d < 3; ++d) n[d] = sg * I[D][d] / nl;
    const double kdA = a.kappa * t.w[qa] * t.w[qb] * det * nl;
    double gr[3];
    const double u = gauss_sum(a, x, gr);
    if (neu) {
      cv[q] = kdA * (gr[0] * n[0] + gr[1] * n[1] + gr[2] * n[2]);
      for (int e = 0; e < 3; ++e) cm[3 * q + e] = 0.0;
    } else {
      const double sig = a.sigma ? a.sigma[f] : a.sg[D];
      cv[q] = 2.0 * sig * kdA * u;
      // d_n phi = (J^{-1} n) . grad_xi phi
      for (int e = 0; e < 3; ++e)
        cm[3 * q + e] =
            -kdA * u * (I[e][0] * n[0] + I[e][1] * n[1] + I[e][2] * n[2]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P3; i += blockDim.x) {
    const int ii[3] = {i % P, (i / P) % P, i / P2};
    const bool on = ii[D] == end;
    if (a.disc != MFP_SIPG && !on) continue;  // CG: Neumann data only
    double acc = 0;
    for (int q = 0; q < P2; ++q) {
      const int qa = q % P, qb = q / P;
      const double va = t.S[qa * P + ii[T1]], vb = t.S[qb * P + ii[T2]];
      double gref[3];
      gref[D] = dS[ii[D]] * va * vb;
      gref[T1] = on ? t.Dphi[qa * P + ii[T1]] * vb : 0.0;
      gref[T2] = on ? va * t.Dphi[qb * P + ii[T2]] : 0.0;
      const double phi = on ? va * vb : 0.0;
      acc += cv[q] * phi + cm[3 * q] * gref[0] + cm[3 * q + 1] * gref[1] +
             cm[3 * q + 2] * gref[2];
    }
    if (a.disc == MFP_SIPG) {
      b[((size_t)cell * P3 + i) * a.stride] += acc;
    } else {
      const int64_t N[3] = {(int64_t)c3[0] * (P - 1) + ii[0],
                            (int64_t)c3[1] * (P - 1) + ii[1],
                            (int64_t)c3[2] * (P - 1) + ii[2]};
      if (!bc_con(a.bc, N[0], N[1], N[2]))
        atomicAdd(b + (N[0] + (int64_t)a.g[0] * (N[1] + (int64_t)a.g[1] * N[2])) *
                          a.stride,
                  acc);
    }
  }
}

__global__ void k_zero_strided(double* b, int64_t n, int64_t stride) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i * stride] = 0.0;
}

// ---------------------------------------------------------------------------
// Coarse coefficient: quadrature-weighted mean over the 8 children of each
// coarse cell, and over the 4 child faces of each coarse face.
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_coarsen_cells(const double* fine, double* coarse, int nf0,
                                int nf1, int nc0, int nc1, int nc2) {
  constexpr int P3 = P * P * P;
  const int C = blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= nc0 * nc1 * nc2) return;
  const int cx = C % nc0, cy = (C / nc0) % nc1, cz = C / (nc0 * nc1);
  double wsum = 0;
  for (int q = 0; q < P3; ++q)
    wsum += c_tab64[P - 2].w[q % P] * c_tab64[P - 2].w[(q / P) % P] *
            c_tab64[P - 2].w[q / (P * P)];
  double acc = 0;
  for (int o = 0; o < 8; ++o) {
    const int fx = 2 * cx + (o & 1), fy = 2 * cy + ((o >> 1) & 1),
              fz = 2 * cz + (o >> 2);
    const double* a = fine + ((size_t)fx + (size_t)nf0 * (fy + (size_t)nf1 * fz)) * P3;
    double s = 0;
    for (int q = 0; q < P3; ++q)
      s += c_tab64[P - 2].w[q % P] * c_tab64[P - 2].w[(q / P) % P] *
           c_tab64[P - 2].w[q / (P * P)] * a[q];
    acc += s / wsum;
  }
  acc *= 0.125;
  for (int q = 0; q < P3; ++q) coarse[(size_t)C * P3 + q] = acc;
}

template <int P>
__global__ void k_coarsen_faces(const double* fine, double* coarse, int D,
                                int fine_off, int coarse_off, int nc0,
                                int nc1, int nc2) {
  constexpr int P2 = P * P;
  int mc[3] = {nc0, nc1, nc2};
  mc[D] += 1;
  int mf[3] = {2 * nc0, 2 * nc1, 2 * nc2};
  mf[D] = 2 * mc[D] - 1;
  const int F = blockIdx.x * blockDim.x + threadIdx.x;
  if (F >= mc[0] * mc[1] * mc[2]) return;
  const int fc[3] = {F % mc[0], (F / mc[0]) % mc[1], F / (mc[0] * mc[1])};
  double wsum = 0;
  for (int q = 0; q < P2; ++q)
    wsum += c_tab64[P - 2].w[q % P] * c_tab64[P - 2].w[q / P];
  double acc = 0;
  const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
  for (int o = 0; o < 4; ++o) {
    int ff[3];
    ff[D] = 2 * fc[D];
    ff[T1] = 2 * fc[T1] + (o & 1);
    ff[T2] = 2 * fc[T2] + (o >> 1);
    const double* a =
        fine + ((size_t)fine_off + ff[0] + (size_t)mf[0] * (ff[1] + (size_t)mf[1] * ff[2])) * P2;
    double s = 0;
    for (int q = 0; q < P2; ++q)
      s += c_tab64[P - 2].w[q % P] * c_tab64[P - 2].w[q / P] * a[q];
    acc += s / wsum;
  }
  acc *= 0.25;
  for (int q = 0; q < P2; ++q)
    coarse[((size_t)coarse_off + F) * P2 + q] = acc;
}

// Support points of the coarse cells of a mesh given by its nodes: the fine
// isoparametric map evaluated at each coarse cell's Gauss-Lobatto points.
// Coarse point a lies, per axis, in child offset o = min(floor(2 x_a), 1) at
// the child's unit coordinate 2 x_a - o (x_a the GLL node on [0, 1]); a point
// on the interface of two children is taken from the upper one.  One block
// per coarse cell, one thread per point.
template <int P>
__global__ void k_coarsen_nodes(const double* fine, double* coarse, int nf0,
                                int nf1, int nc0, int nc1) {
  constexpr int P3 = P * P * P;
  __shared__ double gx[P];
  if (threadIdx.x < P) gx[threadIdx.x] = c_tab64[P - 2].x[threadIdx.x];
  __syncthreads();
  const int C = blockIdx.x;
  const int c3[3] = {C % nc0, (C / nc0) % nc1, C / (nc0 * nc1)};
  for (int a = threadIdx.x; a < P3; a += blockDim.x) {
    const int ai[3] = {a % P, (a / P) % P, a / (P * P)};
    double L[3][P];
    int f3[3];
    for (int e = 0; e < 3; ++e) {
      const double u = 2.0 * gx[ai[e]];
      const int o = u >= 1.0 ? 1 : 0;
      f3[e] = 2 * c3[e] + o;
      const double xi = u - o;
      for (int b = 0; b < P; ++b) {  // Lagrange basis of the GLL nodes at xi
        double v = 1.0;
        for (int m = 0; m < P; ++m)
          if (m != b) v *= (xi - gx[m]) / (gx[b] - gx[m]);
        L[e][b] = v;
      }
    }
    const size_t fc = f3[0] + (size_t)nf0 * (f3[1] + (size_t)nf1 * f3[2]);
    const double* X = fine + fc * 3 * P3;
    double y[3] = {0, 0, 0};
    for (int bz = 0; bz < P; ++bz)
      for (int by = 0; by < P; ++by)
        for (int bx = 0; bx < P; ++bx) {
          const double w = L[0][bx] * L[1][by] * L[2][bz];
          const int b = bx + P * (by + P * bz);
          for (int d = 0; d < 3; ++d) y[d] += w * X[3 * b + d];
        }
    for (int d = 0; d < 3; ++d) coarse[((size_t)C * P3 + a) * 3 + d] = y[d];
  }
}

GeoArgs geo_args(const Level& L) {
  GeoArgs g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = L.n[d];
    g.h[d] = 1.0 / L.n[d];
  }
  g.p = L.p;
  g.amp = L.map_amp;
  g.lo = L.box_lo;
  g.len = L.box_len;
  g.nodes = L.nodes;
  return g;
}

}  // namespace

void launch_curved_cell_geometry(Level& L, cudaStream_t s,
                                 double* hdg_cell) {
  ensure_tables();
  int* bad = nullptr;
  MFP_CHECK_CUDA(cudaMallocAsync(&bad, sizeof(int), s));
  MFP_CHECK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  GeoArgs g = geo_args(L);
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    const int thr = P * P * P < 256 ? ((P * P * P + 31) / 32) * 32 : 256;
    k_cell_geometry<P><<<(int)L.ncells, thr, 0, s>>>(g, L.d64.G, L.d32.G,
                                                      L.vol, bad, hdg_cell);
  });
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
  int hbad = 0;
  MFP_CHECK_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int),
                                 cudaMemcpyDeviceToHost, s));
  MFP_CHECK_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(bad, s);
  MFP_REQUIRE(!hbad, "mapping is not invertible (det J <= 0)");
}

void launch_coarsen_nodes(const Level& fine, Level& coarse, cudaStream_t s) {
  ensure_tables();
  dispatch_p(fine.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    const int thr = P * P * P < 256 ? ((P * P * P + 31) / 32) * 32 : 256;
    k_coarsen_nodes<P><<<(int)coarse.ncells, thr, 0, s>>>(
        fine.nodes, coarse.nodes, fine.n[0], fine.n[1], coarse.n[0],
        coarse.n[1]);
  });
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}

void launch_curved_face_geometry(Level& L, cudaStream_t s,
                                 double* hdg_face) {
  ensure_tables();
  GeoArgs g = geo_args(L);
  for (int D = 0; D < 3; ++D) {
    int m[3] = {L.n[0], L.n[1], L.n[2]};
    m[D] += 1;
    const int nf = m[0] * m[1] * m[2];
    dispatch_p(L.p, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      const int thr = ((P * P + 31) / 32) * 32;
      k_face_geometry<P><<<nf, thr, 0, s>>>(
          g, D, L.face_off[D], L.penalty, L.vol, L.d64.fdata, L.d32.fdata,
          L.d64.sigma, L.d32.sigma, hdg_face);
    });
    MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
  }
}

void launch_diagonal(const Level& L, double* diag, cudaStream_t s) {
  ensure_tables();
  DiagArgs a{};
  for (int d = 0; d < 3; ++d) {
    a.n[d] = L.n[d];
    a.g[d] = L.gdim[d];
    a.face_off[d] = L.face_off[d];
  }
  a.bc = L.bc;
  a.disc = L.disc;
  a.curved = L.curved;
  a.kappa = L.kappa;
  const double vol = L.h[0] * L.h[1] * L.h[2];
  const double pen = L.penalty * (double)L.p * L.p;
  for (int d = 0; d < 3; ++d) {
    a.gs[d] = vol / (L.h[d] * L.h[d]);
    a.ns[d] = 1.0 / L.h[d];
    a.fa[d] = vol / L.h[d];
    a.sg[d] = pen / L.h[d];
  }
  a.G = L.d64.G;
  a.kcell = L.d64.kcell;
  a.kface = L.d64.kface;
  a.fdata = L.d64.fdata;
  a.sigma = L.d64.sigma;
  MFP_CHECK_CUDA(cudaMemsetAsync(diag, 0, L.ndofs * sizeof(double), s));
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    const int thr = P * P * P < 256 ? ((P * P * P + 31) / 32) * 32 : 256;
    k_diagonal<P><<<(int)L.ncells, thr, 0, s>>>(a, diag);
  });
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}

void launch_rhs(const Level& L, int kind, const double* params_dev,
                int nterms, double* b, int64_t stride, cudaStream_t s) {
  ensure_tables();
  RhsArgs a{};
  a.geo = geo_args(L);
  for (int d = 0; d < 3; ++d) a.g[d] = L.gdim[d];
  a.disc = L.disc;
  a.kind = kind;
  a.nterms = nterms;
  a.params = params_dev;
  a.stride = stride;
  a.bc = L.bc;
  a.kappa = L.kappa;
  for (int d = 0; d < 3; ++d) {
    a.face_off[d] = L.face_off[d];
    a.sg[d] = L.penalty * (double)L.p * L.p / L.h[d];
  }
  a.sigma = L.curved ? L.d64.sigma : nullptr;
  k_zero_strided<<<256, 256, 0, s>>>(b, L.ndofs, stride);
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    const int thr = P * P * P < 256 ? ((P * P * P + 31) / 32) * 32 : 256;
    k_rhs<P><<<(int)L.ncells, thr, 0, s>>>(a, b);
    MFP_CHECK_CUDA(cudaGetLastError());
    note_launch();
    if (kind != 2) return;
    // boundary data (kind 2): CG lifting, then one launch per side
    if (L.disc == MFP_CG) {
      k_rhs_lift<P><<<(int)L.ncells, thr, 0, s>>>(a, b);
      MFP_CHECK_CUDA(cudaGetLastError());
      note_launch();
    }
    for (int side = 0; side < 6; ++side) {
      const bool neu = (L.bc.neumann >> side) & 1;
      if (!neu && L.disc == MFP_CG) continue;  // lifted above
      const int D = side / 2;
      const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
      k_rhs_face<P><<<L.n[T1] * L.n[T2], thr, 0, s>>>(a, side, b);
      MFP_CHECK_CUDA(cudaGetLastError());
      note_launch();
    }
  });
}

// Loads the load-vector kernels of degree p - 1 on the current device (a
// kernel's code is otherwise loaded, and its device memory taken, at its
// first launch when CUDA loads modules lazily).
void preload_rhs_kernels(int p) {
  cudaFuncAttributes fa;
  MFP_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_zero_strided));
  dispatch_p(p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    MFP_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_rhs<P>));
    MFP_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_rhs_lift<P>));
    MFP_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_rhs_face<P>));
  });
}

void launch_coarsen_coefficient(const Level& fine, const Level& coarse,
                                cudaStream_t s) {
  ensure_tables();
  dispatch_p(fine.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    const int nc = (int)coarse.ncells;
    k_coarsen_cells<P><<<(nc + 127) / 128, 128, 0, s>>>(
        fine.d64.kcell, coarse.d64.kcell, fine.n[0], fine.n[1], coarse.n[0],
        coarse.n[1], coarse.n[2]);
    if (fine.d64.kface && coarse.d64.kface) {
      for (int D = 0; D < 3; ++D) {
        int mc[3] = {coarse.n[0], coarse.n[1], coarse.n[2]};
        mc[D] += 1;
        const int nf = mc[0] * mc[1] * mc[2];
        k_coarsen_faces<P><<<(nf + 127) / 128, 128, 0, s>>>(
            fine.d64.kface, coarse.d64.kface, D, fine.face_off[D],
            coarse.face_off[D], coarse.n[0], coarse.n[1], coarse.n[2]);
      }
    }
  });
  MFP_CHECK_CUDA(cudaGetLastError());
  note_launch();
}

}  // namespace mfp
