// Allocation-free load vector: the same computation as mfp_rhs, with the
// forcing parameters staged in a fixed device array instead of a buffer the
// library allocates on demand.
#include <mutex>

#include "mfp_internal.h"

namespace mfp {
namespace {

constexpr int kMaxDevices = 64;

// Forcing parameters of the latest mfp_rhs_noalloc call on this device
// (kMaxGaussTerms blocks of 5 doubles, 160 KiB).  The array lives as long as
// the library is loaded and is shared by all calls.
static __device__ __align__(256) double g_rhs_params[5 * kMaxGaussTerms];

std::mutex g_mu;
double* g_params_addr[kMaxDevices] = {nullptr};  // per device ordinal

double* params_address(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_params_addr[dev];
}

}  // namespace

// Called by mfp_create with `device` current.  The host-side name of the
// array is not a device address: cudaGetSymbolAddress gives the address on
// the current device, and with lazily loaded modules it is also the call that
// makes CUDA load this file's module and place the array in device memory.
// Doing it here keeps that allocation inside the set-up call.
void noalloc_prepare(int device, int p) {
  MFP_REQUIRE(device >= 0 && device < kMaxDevices,
              "device ordinal out of range");
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_params_addr[device]) {
      void* a = nullptr;
      MFP_CHECK_CUDA(cudaGetSymbolAddress(&a, g_rhs_params));
      g_params_addr[device] = static_cast<double*>(a);
    }
  }
  preload_rhs_kernels(p);
}

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
    int dev = -1;
    MFP_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev != ctx->device) {
      set_error("mfp_rhs_noalloc: the current device is not the context's");
      return MFP_ERR_STATE;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* params = nullptr;
    if (f_kind >= 1) {
      MFP_REQUIRE(params_host && n_terms >= 1, "bad Gaussian terms");
      MFP_REQUIRE(n_terms <= kMaxGaussTerms,
                  "n_terms exceeds the maximum of 4096 Gaussian terms");
      params = params_address(dev);
      if (!params) {
        set_error("mfp_rhs_noalloc: parameter array not set up on this device");
        return MFP_ERR_STATE;
      }
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
