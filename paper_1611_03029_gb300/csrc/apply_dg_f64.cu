// Operator-apply kernels: dg discretization, double arithmetic.
#include "k_apply.cuh"

namespace mfp {

void launch_apply_dg(const Level& L, const LevelData<double>& D,
                       const double* src, double* dst, int stride, int col,
                       int cpb, cudaStream_t s) {
  ensure_tables();
  ApplyArgs<double> a = make_apply_args<double>(L, D, src, dst);
  a.stride = stride;
  a.col = col;
  if (cpb <= 0) cpb = default_cpb(L.p);
  dispatch_p(L.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    if (L.curved)
      run_apply<P, double, true, true>(a, cpb, s);
    else
      run_apply<P, double, true, false>(a, cpb, s);
  });
}

}  // namespace mfp
