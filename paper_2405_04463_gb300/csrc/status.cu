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

namespace {

// Waits for *flag to become non-zero, giving up after limit_ns of global time; on giving up it
// raises the status word exactly as a pipeline kernel's bounded wait does.
__global__ void bounded_wait_kernel(const volatile uint32_t* flag, uint64_t limit_ns, uint32_t* status) {
  if (threadIdx.x != 0) return;
  const uint64_t t0 = global_ns();
  while (*flag == 0u) {
    if (global_ns() - t0 > limit_ns) {
      raise_status(status, ST_WAIT_TIMEOUT);
      return;
    }
  }
}

}  // namespace
}  // namespace ipc

namespace ipc {
// Enqueues, without synchronising, a wait on `flag` (which nothing sets) that gives up after
// limit_us and raises the status word: a stalled party, injected on the host.
int stall_launch(const uint32_t* flag, uint32_t limit_us, cudaStream_t st) {
  uint32_t* status = status_ptr();
  if (!status) return cuda_fail(cudaErrorMemoryAllocation, "status word");
  bounded_wait_kernel<<<1, 32, 0, st>>>(flag, 1000ull * limit_us, status);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}
}  // namespace ipc

extern "C" int ipc_selftest_bounded_wait(uint32_t limit_us, void* stream) {
  if (limit_us == 0 || limit_us > 1000000) {
    ipc::set_error("ipc_selftest_bounded_wait: limit_us must be in 1..1000000");
    return IPC_EINVAL;
  }
  uint32_t* status = ipc::status_ptr();
  if (!status) return ipc::cuda_fail(cudaErrorMemoryAllocation, "status word");
  cudaStream_t st = ipc::as_stream(stream);
  uint32_t* flag = nullptr;
  IPC_CUDA_TRY(cudaMalloc(&flag, sizeof(uint32_t)));
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(uint32_t), st);  // nothing ever sets it
  if (e == cudaSuccess) {
    ipc::bounded_wait_kernel<<<1, 32, 0, st>>>(flag, 1000ull * limit_us, status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(flag);
  if (e != cudaSuccess) return ipc::cuda_fail(e, "ipc_selftest_bounded_wait");
  return IPC_OK;
}

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
