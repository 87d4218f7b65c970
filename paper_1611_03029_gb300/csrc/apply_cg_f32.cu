// Operator-apply kernels: cg discretization, float arithmetic.
#include "k_apply_warp.cuh"

namespace mfp {

void launch_apply_cg(const Level& L, const LevelData<float>& D,
                       const float* src, float* dst, int nrhs, int cells,
                       cudaStream_t s) {
  ensure_tables();
  ApplyArgs<float> a = make_apply_args<float>(L, D, src, dst);
  a.stride = nrhs;
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    // cells == kWarpCells: one warp per cell (k <= 4, one column)
    if (cells == kWarpCells && nrhs == 1) {
      const bool done = L.curved ? run_apply_cg_warp<P, float, true>(a, s)
                                 : run_apply_cg_warp<P, float, false>(a, s);
      if (done) return;
      cells = 0;
    }
    if (cells == kWarpCells) cells = 0;
    if (L.curved)
      run_apply_cols<P, float, false, true>(a, nrhs, cells, s);
    else
      run_apply_cols<P, float, false, false>(a, nrhs, cells, s);
  });
}

}  // namespace mfp
