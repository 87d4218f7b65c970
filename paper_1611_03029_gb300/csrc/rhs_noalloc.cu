// Allocation-free load vector: the same computation as mfp_rhs, with the
// forcing parameters staged in a fixed device array instead of a buffer the
// library allocates on demand.
#include <mutex>

#include "mfp_internal.h"

namespace mfp {
namespace {

constexpr int kNoAllocMaxTerms = 4096;  // 4096 * 5 doubles = 160 KiB

// Forcing parameters of the latest mfp_rhs_noalloc call on this device.  The
// array lives as long as the library is loaded and is shared by all calls.
static __device__ __align__(256) double g_rhs_params[5 * kNoAllocMaxTerms];

std::mutex g_mu;
double* g_params_addr[64] = {nullptr};  // device address per device ordinal

// Device address of g_rhs_params on the current device; looked up on the
// first call per device (the host-side symbol is not a device address).
double* params_address() {
  int dev = 0;
  MFP_CHECK_CUDA(cudaGetDevice(&dev));
  MFP_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_params_addr[dev]) {
    void* p = nullptr;
    MFP_CHECK_CUDA(cudaGetSymbolAddress(&p, g_rhs_params));
    g_params_addr[dev] = static_cast<double*>(p);
  }
  return g_params_addr[dev];
}

}  // namespace
}  // namespace mfp

using namespace mfp;

extern "C" mfp_status mfp_rhs_noalloc(mfp_ctx* ctx, int f_kind,
                                      const double* params_host, int n_terms,
                                      double* b_dev, int64_t stride,
                                      void* stream) {
  try {
    clear_error();
    MFP_REQUIRE(ctx && b_dev, "null argument");
    MFP_REQUIRE(f_kind >= 0 && f_kind <= 2, "unknown f_kind");
    MFP_REQUIRE(stride >= 1, "stride must be >= 1");
    MFP_REQUIRE(f_kind != 2 || !ctx->has_coef,
                "f_kind 2 needs the constant coefficient");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* params = nullptr;
    if (f_kind >= 1) {
      MFP_REQUIRE(params_host && n_terms >= 1, "bad Gaussian terms");
      MFP_REQUIRE(n_terms <= kNoAllocMaxTerms,
                  "n_terms exceeds the allocation-free maximum of 4096 "
                  "terms; use mfp_rhs");
      params = params_address();
      MFP_CHECK_CUDA(cudaMemcpyAsync(params, params_host,
                                     sizeof(double) * 5 * n_terms,
                                     cudaMemcpyHostToDevice, s));
    }
    launch_rhs(ctx->levels.back(), f_kind, params, n_terms, b_dev, stride, s);
    return MFP_OK;
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("unexpected exception");
    return MFP_ERR_CUDA;
  }
}
