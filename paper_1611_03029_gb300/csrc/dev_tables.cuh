// Per-translation-unit constant-memory copy of the 1D tables.  Every kernel
// TU includes this header once; its launchers call ensure_tables() first.
#pragma once

#include <mutex>
#include <type_traits>

#include "mfp_internal.h"

namespace mfp {
namespace {

// The double-float kernels' TUs (MFP_DF_TABLES) hold the double-float and
// even-odd tables, the others the float64 and float ones: every TU has 64 KB
// of constant memory.
#ifndef MFP_DF_TABLES
__constant__ DevTab<double> c_tab64[8];
__constant__ DevTab<float> c_tab32[8];
#else
__constant__ DevTabEO c_tabeo[8];
__constant__ DevTabDF c_tabdf[8];
#endif

// Uploads the tables to the current device once per device per TU.
inline void ensure_tables() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  MFP_CHECK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && done[dev]) return;
  const HostTables& h = host_tables();
#ifndef MFP_DF_TABLES
  MFP_CHECK_CUDA(cudaMemcpyToSymbol(c_tab64, h.d, sizeof(h.d)));
  MFP_CHECK_CUDA(cudaMemcpyToSymbol(c_tab32, h.f, sizeof(h.f)));
#else
  MFP_CHECK_CUDA(cudaMemcpyToSymbol(c_tabeo, h.eo, sizeof(h.eo)));
  MFP_CHECK_CUDA(cudaMemcpyToSymbol(c_tabdf, h.df, sizeof(h.df)));
#endif
  if (dev < 64) done[dev] = true;
}

#ifndef MFP_DF_TABLES
// Table selectors (P = k+1; W picks the table).  With compile-time indices
// these become constant-bank operands.
enum TabId {
  T_S, T_D, T_DPHI, T_E0, T_E1, T_DPHI0, T_DPHI1, T_W, T_G, T_X,
  T_GV0, T_GV1, T_GD0, T_GD1
};

template <typename T, int P, int W>
__device__ __forceinline__ T tv(int i) {
  const DevTab<T>* t;
  if constexpr (std::is_same<T, double>::value)
    t = &c_tab64[P - 2];
  else
    t = &c_tab32[P - 2];
  if constexpr (W == T_S) return t->S[i];
  if constexpr (W == T_D) return t->D[i];
  if constexpr (W == T_DPHI) return t->Dphi[i];
  if constexpr (W == T_E0) return t->E0[i];
  if constexpr (W == T_E1) return t->E1[i];
  if constexpr (W == T_DPHI0) return t->dphi0[i];
  if constexpr (W == T_DPHI1) return t->dphi1[i];
  if constexpr (W == T_W) return t->w[i];
  if constexpr (W == T_G) return t->g[i];
  if constexpr (W == T_X) return t->x[i];
  if constexpr (W == T_GV0) return t->gv0[i];
  if constexpr (W == T_GV1) return t->gv1[i];
  if constexpr (W == T_GD0) return t->gd0[i];
  if constexpr (W == T_GD1) return t->gd1[i];
  return T(0);
}

// out[q] = sum_j M[q][j] in[j]
template <typename T, int P, int W>
__device__ __forceinline__ void mv(const T (&in)[P], T (&out)[P]) {
#pragma unroll
  for (int q = 0; q < P; ++q) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < P; ++j) s = fma(tv<T, P, W>(q * P + j), in[j], s);
    out[q] = s;
  }
}

// out[j] = sum_q M[q][j] in[q]
template <typename T, int P, int W>
__device__ __forceinline__ void mtv(const T (&in)[P], T (&out)[P]) {
#pragma unroll
  for (int j = 0; j < P; ++j) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < P; ++q) s = fma(tv<T, P, W>(q * P + j), in[q], s);
    out[j] = s;
  }
}

// Copy the tables of degree P-1 into shared memory (for thread-dependent
// indexing): S, D, Dphi (P*P each), dphi0, dphi1, w (P each).
template <typename T, int P>
__device__ __forceinline__ void load_tables_shared(T* sS, T* sD, T* sDphi,
                                                   T* s0, T* s1, T* sw) {
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    if constexpr (std::is_same<T, double>::value) {
      sS[i] = c_tab64[P - 2].S[i];
      sD[i] = c_tab64[P - 2].D[i];
      sDphi[i] = c_tab64[P - 2].Dphi[i];
    } else {
      sS[i] = c_tab32[P - 2].S[i];
      sD[i] = c_tab32[P - 2].D[i];
      sDphi[i] = c_tab32[P - 2].Dphi[i];
    }
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if constexpr (std::is_same<T, double>::value) {
      s0[i] = c_tab64[P - 2].dphi0[i];
      s1[i] = c_tab64[P - 2].dphi1[i];
      sw[i] = c_tab64[P - 2].w[i];
    } else {
      s0[i] = c_tab32[P - 2].dphi0[i];
      s1[i] = c_tab32[P - 2].dphi1[i];
      sw[i] = c_tab32[P - 2].w[i];
    }
  }
}

#endif  // MFP_DF_TABLES

// Dispatch a functor templated on P = k+1 (k in 1..8).
template <typename F>
inline void dispatch_p(int p, F&& f) {
  switch (p) {
    case 2: f(std::integral_constant<int, 2>()); break;
    case 3: f(std::integral_constant<int, 3>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    case 5: f(std::integral_constant<int, 5>()); break;
    case 6: f(std::integral_constant<int, 6>()); break;
    case 7: f(std::integral_constant<int, 7>()); break;
    case 8: f(std::integral_constant<int, 8>()); break;
    case 9: f(std::integral_constant<int, 9>()); break;
    default: break;
  }
}

inline int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace
}  // namespace mfp
