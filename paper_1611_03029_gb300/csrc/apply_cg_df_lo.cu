// Operator-apply kernels: cg discretization, float64 vectors with
// double-float arithmetic on the FP32 pipes; degrees p = 2 3 4 5.
#include "k_apply_df.cuh"

namespace mfp {

bool apply_cg_df_lo(const Level& L, const double* src, double* dst,
                     int nrhs, int cells, cudaStream_t s) {
  if (L.p > 5) return false;
  ensure_tables();
  ApplyArgsDF a = make_apply_args_df(L, src, dst);
  a.stride = nrhs;
  switch (L.p) {
    case 2:
      if (L.curved)
        run_apply_df_cols<2, false, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<2, false, false>(a, nrhs, cells, s);
      break;
    case 3:
      if (L.curved)
        run_apply_df_cols<3, false, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<3, false, false>(a, nrhs, cells, s);
      break;
    case 4:
      if (L.curved)
        run_apply_df_cols<4, false, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<4, false, false>(a, nrhs, cells, s);
      break;
    case 5:
      if (L.curved)
        run_apply_df_cols<5, false, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<5, false, false>(a, nrhs, cells, s);
      break;
    default:
      return false;
  }
  return true;
}

}  // namespace mfp
