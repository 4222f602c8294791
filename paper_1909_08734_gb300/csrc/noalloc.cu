// Operator apply without any device allocation (cpm_op_apply_noalloc).
//
// The regular cpm_op_apply keeps its extension-value scratch (one FP64 value per band node)
// in memory the preconditioner handle allocated.  This variant is for callers that cannot
// allocate device memory themselves: the scratch lives in the file-scope array below,
// which every GPU that loads the library reserves until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "cuda/kernels.h"
#include "host/cpm_internal.h"

// Scratch for the extension values v_k of one operator apply.  In host code this name is
// only a stand-in for the device symbol: its device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) double g_noalloc_ext[CPM_NOALLOC_MAX_NODES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ext_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on first use).
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ext_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ext);
    if (e != cudaSuccess) return e;
    g_ext_ptr[dev] = (double*)p;
  }
  *out = g_ext_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" cpm_status cpm_op_apply_noalloc(const int32_t* pencil_dev, const double* weights_dev,
                                           const int32_t* nbr_dev, int64_t n_active,
                                           int64_t n_nodes, int p, double c, double h,
                                           const double* x_dev, double* y_dev, void* stream) {
  if (!pencil_dev || !weights_dev || !nbr_dev || !x_dev || !y_dev || (p != 2 && p != 3) ||
      n_active < 1 || n_nodes < n_active || !(h > 0.0)) {
    cpm::set_error("cpm_op_apply_noalloc: NULL pointer or invalid size / degree / spacing");
    return CPM_ERR_INVALID_ARG;
  }
  if (n_nodes > (int64_t)CPM_NOALLOC_MAX_NODES) {
    cpm::set_error("cpm_op_apply_noalloc: the band has " + std::to_string(n_nodes) +
                   " nodes, more than the static scratch holds (CPM_NOALLOC_MAX_NODES = " +
                   std::to_string((long long)CPM_NOALLOC_MAX_NODES) + ")");
    return CPM_ERR_BUDGET;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cpm::set_error(std::string("cpm_op_apply_noalloc: no usable current device: ") +
                   cudaGetErrorString(e));
    return CPM_ERR_CUDA;
  }
  double* ext = nullptr;
  e = scratch_address(dev, &ext);
  if (e != cudaSuccess) {
    cpm::set_error(std::string("cpm_op_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return CPM_ERR_CUDA;
  }
  // Every scratch entry the second kernel reads is written by the first in the same call,
  // so nothing has to be cleared between calls.
  cpmdev::OperatorDev op{pencil_dev, weights_dev, nbr_dev, n_active, n_nodes, p + 1,
                         c + 6.0 / (h * h), 1.0 / (h * h)};
  e = cpmdev::launch_apply(op, cpmdev::direct(const_cast<double*>(x_dev), n_active), ext, nullptr,
                           cpmdev::direct(y_dev, n_active), 1, 0, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cpm::set_error(std::string("cpm_op_apply_noalloc: launch: ") + cudaGetErrorString(e));
    return CPM_ERR_CUDA;
  }
  return CPM_OK;
}
