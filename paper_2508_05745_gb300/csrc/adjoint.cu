// C ABI of the differentiation entry points (unravel_grad, unravel_descend).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lemps.h"
#include "adjoint.cuh"

using namespace lemps;

extern "C" lemps_status lemps_set_error_(int st, const char* msg);

extern "C" {

lemps_status unravel_grad(const void* theta, int32_t theta_fp64, int64_t batch, int32_t chi, const double* p,
                          const double* h, double* cost, double* grad, double* rho_out, void* stream) {
  if (!theta || !p || !h || !cost || batch < 0 || chi < 1)
    return lemps_set_error_(LEMPS_EINVAL, "unravel_grad: bad argument");
  if (batch == 0) return LEMPS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  zd* rho = reinterpret_cast<zd*>(rho_out);
  bool own = false;
  if (!rho) {
    if (cudaMallocAsync((void**)&rho, sizeof(zd) * 4 * batch, st) != cudaSuccess)
      return lemps_set_error_(LEMPS_ENOMEM, "unravel_grad: scratch allocation failed");
    own = true;
  }
  if (theta_fp64)
    adj::k_rho_target<double><<<(unsigned)batch, 256, 0, st>>>((const zd*)theta, batch, chi, rho);
  else
    adj::k_rho_target<float><<<(unsigned)batch, 256, 0, st>>>((const zf*)theta, batch, chi, rho);
  adj::k_cost_grad<<<(unsigned)((batch + 63) / 64), 64, 0, st>>>(rho, p, (const zd*)h, batch, cost, (zd*)grad);
  if (own) cudaFreeAsync(rho, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lemps_set_error_(LEMPS_ECUDA, cudaGetErrorString(e));
  return LEMPS_OK;
}

lemps_status unravel_descend(const double* rho_a, const double* p, int64_t batch, int32_t steps, double lr, double* h,
                             double* cost_trace, void* stream) {
  if (!rho_a || !p || !h || batch < 0 || steps < 0) return lemps_set_error_(LEMPS_EINVAL, "unravel_descend: bad argument");
  if (batch == 0 || steps == 0) return LEMPS_OK;
  adj::k_descend<<<(unsigned)((batch + 63) / 64), 64, 0, (cudaStream_t)stream>>>((const zd*)rho_a, p, batch, steps, lr,
                                                                                 (zd*)h, cost_trace);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lemps_set_error_(LEMPS_ECUDA, cudaGetErrorString(e));
  return LEMPS_OK;
}

}  // extern "C"

// ---- allocation-free variant of unravel_grad ------------------------------------
// unravel_grad needs one scratch buffer (the reduced target states) when the
// caller does not ask for them.  Callers that cannot allocate device memory
// during a call use unravel_grad_noalloc instead; its scratch is the
// module-scope array below.
namespace {

constexpr int64_t kNoAllocMaxBatch = 16384;   // problems per call
constexpr int kMaxDevices = 64;

// kNoAllocMaxBatch 2x2 complex doubles = 1 MiB.  Every GPU that loads the
// library holds this array until the process exits; every call shares it.
static __device__ __align__(256) double g_noalloc_rho[kNoAllocMaxBatch * 8];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};   // device address per device id

}  // namespace

extern "C" lemps_status unravel_grad_noalloc(const void* theta, int32_t theta_fp64, int64_t batch, int32_t chi,
                                             const double* p, const double* h, double* cost, double* grad,
                                             void* stream) {
  if (!theta || !p || !h || !cost || batch < 0 || chi < 1)
    return lemps_set_error_(LEMPS_EINVAL, "unravel_grad_noalloc: bad argument");
  if (batch > kNoAllocMaxBatch)
    return lemps_set_error_(LEMPS_EINVAL,
                            "unravel_grad_noalloc: batch exceeds the allocation-free maximum of 16384 problems");
  if (batch == 0) return LEMPS_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lemps_set_error_(LEMPS_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return lemps_set_error_(LEMPS_EINVAL, "unravel_grad_noalloc: device id >= 64");
  void* scratch = nullptr;
  {
    // First call on a device: look up the array's device address with that
    // device current.  In host code the symbol itself is only a stand-in.  The
    // address is cached for the process: a cudaDeviceReset would leave it
    // stale (the header tells callers not to use this entry point after one).
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      e = cudaGetSymbolAddress(&scratch, g_noalloc_rho);
      if (e != cudaSuccess)
        return lemps_set_error_(LEMPS_ECUDA, (std::string("unravel_grad_noalloc: cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e)).c_str());
      g_noalloc_ptr[dev] = scratch;
    }
    scratch = g_noalloc_ptr[dev];
  }
  // k_rho_target writes every scratch entry that k_cost_grad reads, so the
  // array needs no clearing between calls.
  zd* rho = reinterpret_cast<zd*>(scratch);
  cudaStream_t st = (cudaStream_t)stream;
  if (theta_fp64)
    adj::k_rho_target<double><<<(unsigned)batch, 256, 0, st>>>((const zd*)theta, batch, chi, rho);
  else
    adj::k_rho_target<float><<<(unsigned)batch, 256, 0, st>>>((const zf*)theta, batch, chi, rho);
  adj::k_cost_grad<<<(unsigned)((batch + 63) / 64), 64, 0, st>>>(rho, p, (const zd*)h, batch, cost, (zd*)grad);
  e = cudaGetLastError();
  if (e != cudaSuccess) return lemps_set_error_(LEMPS_ECUDA, cudaGetErrorString(e));
  return LEMPS_OK;
}
