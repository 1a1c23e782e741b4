// Error reporting: per-thread last error of stage-level calls and the per-device status word
// that kernels raise instead of trapping when a bounded wait runs out.
#include <mutex>
#include <string>

#include "common.cuh"

namespace ipc {

namespace {
thread_local std::string g_last_error;
std::mutex g_status_mu;
uint32_t* g_status[64] = {nullptr};
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

const char* thread_last_error() { return g_last_error.c_str(); }

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return IPC_ECUDA;
}

uint32_t* status_ptr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_status_mu);
  if (!g_status[dev]) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(uint32_t)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(uint32_t)) != cudaSuccess) return nullptr;
    g_status[dev] = static_cast<uint32_t*>(p);
  }
  return g_status[dev];
}

}  // namespace ipc

extern "C" int ipc_status(void) {
  IPC_CUDA_TRY(cudaDeviceSynchronize());
  uint32_t* p = ipc::status_ptr();
  if (!p) return ipc::cuda_fail(cudaErrorMemoryAllocation, "status word");
  uint32_t v = 0;
  IPC_CUDA_TRY(cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost));
  IPC_CUDA_TRY(cudaMemset(p, 0, sizeof v));
  if (v) {
    ipc::set_error("device status " + std::to_string(v) + ": a kernel gave up a bounded wait or saw a bad argument");
    return IPC_EDEVICE;
  }
  return IPC_OK;
}
