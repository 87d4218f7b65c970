// Operator-apply kernels: dg discretization, float64 vectors with
// double-float arithmetic on the FP32 pipes; degrees p = 2 3 4 5.
#include "k_apply_df.cuh"

namespace mfp {

bool apply_dg_df_lo(const Level& L, const double* src, double* dst,
                     int nrhs, int cells, cudaStream_t s,
                     const Epi<double>* epi) {
  if (L.p > 5) return false;
  ensure_tables();
  ApplyArgsDF a = make_apply_args_df(L, src, dst);
  a.stride = nrhs;
  if (epi) {
    a.epi = *epi;
    a.epi_c1 = host_df(epi->c1);
    a.epi_c2 = host_df(epi->c2);
  }
  switch (L.p) {
    case 2:
      if (L.curved)
        run_apply_df_cols<2, true, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<2, true, false>(a, nrhs, cells, s);
      break;
    case 3:
      if (L.curved)
        run_apply_df_cols<3, true, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<3, true, false>(a, nrhs, cells, s);
      break;
    case 4:
      if (L.curved)
        run_apply_df_cols<4, true, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<4, true, false>(a, nrhs, cells, s);
      break;
    case 5:
      if (L.curved)
        run_apply_df_cols<5, true, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<5, true, false>(a, nrhs, cells, s);
      break;
    default:
      return false;
  }
  return true;
}

}  // namespace mfp
