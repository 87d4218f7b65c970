// Operator-apply kernels: dg discretization, float arithmetic.
#include "k_apply.cuh"

namespace mfp {

void launch_apply_dg(const Level& L, const LevelData<float>& D,
                       const float* src, float* dst, int nrhs, int cells,
                       cudaStream_t s, const Epi<float>* epi) {
  ensure_tables();
  ApplyArgs<float> a = make_apply_args<float>(L, D, src, dst);
  a.stride = nrhs;
  if (epi) a.epi = *epi;
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    if (L.curved)
      run_apply_cols<P, float, true, true>(a, nrhs, cells, s);
    else
      run_apply_cols<P, float, true, false>(a, nrhs, cells, s);
  });
}

}  // namespace mfp
