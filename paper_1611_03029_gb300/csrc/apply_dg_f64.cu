// Operator-apply kernels: dg discretization, double arithmetic.
#include "k_apply.cuh"

namespace mfp {

void launch_apply_dg(const Level& L, const LevelData<double>& D,
                       const double* src, double* dst, int nrhs, int cells,
                       cudaStream_t s, const Epi<double>* epi) {
  ensure_tables();
  ApplyArgs<double> a = make_apply_args<double>(L, D, src, dst);
  a.stride = nrhs;
  if (epi) a.epi = *epi;
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    if (L.curved)
      run_apply_cols<P, double, true, true>(a, nrhs, cells, s);
    else
      run_apply_cols<P, double, true, false>(a, nrhs, cells, s);
  });
}

}  // namespace mfp
