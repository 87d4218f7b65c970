// Operator-apply kernels: dg discretization, float64 vectors with
// double-float arithmetic on the FP32 pipes; degrees p = 6 7 8 9.
#include "k_apply_df.cuh"

namespace mfp {

bool apply_dg_df_hi(const Level& L, const double* src, double* dst,
                     int nrhs, int cells, cudaStream_t s,
                     const Epi<double>* epi) {
  if (L.p < 6) return false;
  ensure_tables();
  ApplyArgsDF a = make_apply_args_df(L, src, dst);
  a.stride = nrhs;
  if (epi) {
    a.epi = *epi;
    a.epi_c1 = host_df(epi->c1);
    a.epi_c2 = host_df(epi->c2);
  }
  switch (L.p) {
    case 6:
      if (L.curved)
        run_apply_df_cols<6, true, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<6, true, false>(a, nrhs, cells, s);
      break;
    case 7:
      if (L.curved)
        run_apply_df_cols<7, true, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<7, true, false>(a, nrhs, cells, s);
      break;
    case 8:
      if (L.curved)
        run_apply_df_cols<8, true, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<8, true, false>(a, nrhs, cells, s);
      break;
    case 9:
      if (L.curved)
        run_apply_df_cols<9, true, true>(a, nrhs, cells, s);
      else
        run_apply_df_cols<9, true, false>(a, nrhs, cells, s);
      break;
    default:
      return false;
  }
  return true;
}

}  // namespace mfp
