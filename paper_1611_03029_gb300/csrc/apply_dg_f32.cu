// Operator-apply kernels: dg discretization, float arithmetic.
#include "k_apply.cuh"

namespace mfp {

void launch_apply_dg(const Level& L, const LevelData<float>& D,
                       const float* src, float* dst, int stride, int col,
                       int cpb, cudaStream_t s) {
  ensure_tables();
  ApplyArgs<float> a = make_apply_args<float>(L, D, src, dst);
  a.stride = stride;
  a.col = col;
  if (cpb <= 0) cpb = default_cpb(L.p);
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    if (L.curved)
      run_apply<P, float, true, true>(a, cpb, s);
    else
      run_apply<P, float, true, false>(a, cpb, s);
  });
}

}  // namespace mfp
