// Continuous Q_k operator apply (Sec. 3, Eq. 12; Eq. 4) with each cell owned
// by one warp, for p^2 <= 32 (k <= 4) and one right-hand side: the same
// sum-factorization steps as k_apply (gather, S along z, y, x, the Gauss
// collocation derivative, t = G grad u, D^T, S^T, atomic scatter with
// identity rows), but a warp holds floor(32 / p^2) whole cells, so the line
// transposes between sweep directions need only __syncwarp and the warps of
// a block never wait for each other.
#pragma once

#include "k_apply.cuh"

namespace mfp {
namespace {

template <int P>
constexpr int wcells() {
  return 32 / (P * P);
}
constexpr int kWarpBlock = 128;  // 4 independent warps per block

template <int P, typename T>
__host__ __device__ constexpr int wcell_smem_elems() {
  return (3 * P * P * P) | 1;  // Aq, GX, GY; odd stride (banks)
}

// at least 4 resident blocks (16 warps) per SM: at most 128 registers (at
// 5 blocks the curved p = 5 kernel spills)
template <int P, typename T, bool CURVED>
__global__ void __launch_bounds__(kWarpBlock, 4)
    k_apply_cg_warp(const ApplyArgs<T> a) {
  constexpr int P2 = P * P, P3 = P2 * P, C = wcells<P>();
  constexpr int WPB = kWarpBlock / 32;
  extern __shared__ __align__(16) unsigned char wsm[];
  T* sm = reinterpret_cast<T*>(wsm);
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  const bool lane_ok = lane < C * P2;
  const int lc = lane_ok ? lane / P2 : 0;
  const int rest = lane_ok ? lane % P2 : 0;
  const int ta = rest % P, tb = rest / P;
  // per warp C cells plus one dummy slot for the idle lanes
  T* base = sm + ((size_t)wid * (C + 1) + (lane_ok ? lc : C)) *
                     wcell_smem_elems<P, T>();
  T* Aq = base;
  T* GX = base + P3;
  T* GY = base + 2 * P3;
  T* sw = sm + (size_t)WPB * (C + 1) * wcell_smem_elems<P, T>();
  for (int i = threadIdx.x; i < P; i += blockDim.x) sw[i] = tv<T, P, T_W>(i);
  __syncthreads();  // the only block-wide barrier
  const int gx0 = a.g[0], gy0 = a.g[1];
  const int nwarps = gridDim.x * WPB;
  for (int c0 = (blockIdx.x * WPB + wid) * C; c0 < a.ncells; c0 += nwarps * C) {
    const int cell = c0 + lc;
    const bool active = lane_ok && cell < a.ncells;
    const int cc = active ? cell : 0;
    const int cx = cc % a.n[0];
    const int cy = (cc / a.n[0]) % a.n[1];
    const int cz = cc / (a.n[0] * a.n[1]);
    T r[P], o[P];
    T gp[CURVED ? 6 : 1][CURVED ? P : 1];
    if constexpr (CURVED) {  // stored geometry into registers first
#pragma unroll
      for (int qz = 0; qz < P; ++qz) {
        const T* Gp = a.G + (size_t)cc * 6 * P3 + idx3<P>(ta, tb, qz);
#pragma unroll
        for (int c = 0; c < 6; ++c) gp[c][qz] = Gp[c * P3];
      }
    }
    // ---- gather the z-line (x = ta, y = tb); constrained nodes read 0
    const int X = cx * (P - 1) + ta, Y = cy * (P - 1) + tb;
    const bool bxy =
        X == a.blo[0] || X == a.bhi[0] || Y == a.blo[1] || Y == a.bhi[1];
#pragma unroll
    for (int z = 0; z < P; ++z) {
      const int Z = cz * (P - 1) + z;
      const bool con = bxy || Z == a.blo[2] || Z == a.bhi[2];
      const size_t gi = (size_t)X + (size_t)gx0 * (Y + (size_t)gy0 * Z);
      r[z] = (active && !con) ? a.src[gi] : T(0);
    }
    // ---- values at the Gauss points: z (registers), y, x
    mv<T, P, T_S>(r, o);
#pragma unroll
    for (int z = 0; z < P; ++z) Aq[idx3<P>(ta, tb, z)] = o[z];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(ta, j, tb)];
    mv<T, P, T_S>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(ta, j, tb)] = o[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(j, ta, tb)];
    mv<T, P, T_S>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(j, ta, tb)] = o[j];
    mv<T, P, T_D>(o, r);
#pragma unroll
    for (int j = 0; j < P; ++j) GX[idx3<P>(j, ta, tb)] = r[j];
    __syncwarp();
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
    __syncwarp();
    // ---- quadrature-point operation t = G_q grad u
    {
      const T wab = sw[ta] * sw[tb];
#pragma unroll
      for (int qz = 0; qz < P; ++qz) {
        const int q = idx3<P>(ta, tb, qz);
        const T ux = GX[q], uy = GY[q], uz = gz[qz];
        const T kap = a.kcell ? a.kcell[(size_t)cc * P3 + q] : a.kappa;
        T tx, ty, tz;
        if constexpr (CURVED) {
          tx = kap * (gp[0][qz] * ux + gp[1][qz] * uy + gp[2][qz] * uz);
          ty = kap * (gp[1][qz] * ux + gp[3][qz] * uy + gp[4][qz] * uz);
          tz = kap * (gp[2][qz] * ux + gp[4][qz] * uy + gp[5][qz] * uz);
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
    __syncwarp();
    // ---- transposed derivative y (added), x (added), then S^T x, y, z
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = GY[idx3<P>(ta, j, tb)];
    mtv<T, P, T_D>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(ta, j, tb)] += o[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = GX[idx3<P>(j, ta, tb)];
    mtv<T, P, T_D>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) o[j] += Aq[idx3<P>(j, ta, tb)];
    mtv<T, P, T_S>(o, r);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(j, ta, tb)] = r[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(ta, j, tb)];
    mtv<T, P, T_S>(r, o);
#pragma unroll
    for (int j = 0; j < P; ++j) Aq[idx3<P>(ta, j, tb)] = o[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = Aq[idx3<P>(ta, tb, j)];
    mtv<T, P, T_S>(r, o);
    // ---- scatter (identity rows on constrained nodes)
    if (active) {
#pragma unroll
      for (int z = 0; z < P; ++z) {
        const int Z = cz * (P - 1) + z;
        const bool con = bxy || Z == a.blo[2] || Z == a.bhi[2];
        const size_t gi = (size_t)X + (size_t)gx0 * (Y + (size_t)gy0 * Z);
        if (con)
          a.dst[gi] = a.src[gi];
        else
          atomicAdd(a.dst + gi, o[z]);
      }
    }
    __syncwarp();  // the next cell overwrites this warp's scratch
  }
}

template <int P, typename T>
size_t warp_smem_bytes() {
  return ((size_t)(kWarpBlock / 32) * (wcells<P>() + 1) *
              wcell_smem_elems<P, T>() +
          P) *
         sizeof(T);
}

// Launches the warp-per-cell CG kernel (p <= 5, one column), at most as many
// blocks as fit on the GPU at once; returns false where it does not apply.
template <int P, typename T, bool CURVED>
bool run_apply_cg_warp(const ApplyArgs<T>& a, cudaStream_t s) {
  if constexpr (P * P > 32) {
    return false;
  } else {
    auto kern = k_apply_cg_warp<P, T, CURVED>;
    const size_t smem = warp_smem_bytes<P, T>();
    static int per_sm_cache[4] = {0, 0, 0, 0};
    int dev = 0;
    MFP_CHECK_CUDA(cudaGetDevice(&dev));
    int per_sm = dev < 4 ? per_sm_cache[dev] : 0;
    if (!per_sm) {
      MFP_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, kern, kWarpBlock, smem));
      if (dev < 4) per_sm_cache[dev] = per_sm;
    }
    if (per_sm < 1) return false;
    constexpr int cpb = (kWarpBlock / 32) * wcells<P>();
    const int64_t need = (a.ncells + cpb - 1) / cpb;
    const int64_t cap = (int64_t)per_sm * sm_count();
    const int grid = (int)(need < cap ? need : cap);
    if (grid <= 0) return true;
    kern<<<grid, kWarpBlock, smem, s>>>(a);
    MFP_CHECK_CUDA(cudaGetLastError());
    note_launch();
    return true;
  }
}

}  // namespace
}  // namespace mfp
