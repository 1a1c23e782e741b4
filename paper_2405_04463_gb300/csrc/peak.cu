// Roofline denominators measured on the running GPU: the issue-limited rate of
// mma.sync.m16n8k32 s8 (no memory traffic, 8 independent accumulators per warp) and of
// 32-bit IMAD. Used by the benchmark to state the fraction of peak of the ring GEMMs.
#include <cuda_runtime.h>

#include "common.cuh"

namespace {

__global__ void mma_s8_loop(int* out, int iters) {
  const uint32_t a0 = threadIdx.x * 0x01010101u, a1 = a0 ^ 0x5a5a5a5au, a2 = a0 + 7u, a3 = a0 * 3u;
  const uint32_t b0 = threadIdx.x ^ 0x33333333u, b1 = b0 + 11u;
  int c[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[i][j] = i + j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
          : "+r"(c[i][0]), "+r"(c[i][1]), "+r"(c[i][2]), "+r"(c[i][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  int s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s ^= c[i][j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void imad_loop(uint32_t* out, int iters, uint32_t p, uint32_t q) {
  uint32_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * (i + 1) + p;
  const uint32_t y = q ^ threadIdx.x, z = q + blockIdx.x;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = x[i] * y + z;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s ^= x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dp4a_loop(uint32_t* out, int iters, uint32_t p, uint32_t q) {
  int x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * (i + 1) + p;
  const int y = static_cast<int>(q ^ threadIdx.x), z = static_cast<int>(q + blockIdx.x);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = __dp4a(x[i], y, z);
  int s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s ^= x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = static_cast<uint32_t>(s);
}

}  // namespace

// what = 0: mma.sync s8 (returns TOP/s, 2 ops per MAC); what = 1: IMAD (returns T IMAD/s);
// what = 2: dp4a (returns TOP/s, 4 MACs = 8 ops per instruction).
extern "C" int ipc_measure_peak(int what, void* stream, double* out) {
  if (!out || what < 0 || what > 2) {
    ipc::set_error("ipc_measure_peak: what must be 0, 1 or 2 and out non-null");
    return IPC_EINVAL;
  }
  int dev = 0, sms = 0;
  IPC_CUDA_TRY(cudaGetDevice(&dev));
  IPC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 2, threads = 256;
  const int iters = what == 0 ? 4096 : 2048;  // each variant runs a few milliseconds
  int* buf = nullptr;
  IPC_CUDA_TRY(cudaMalloc(&buf, sizeof(int) * 4 * blocks * threads));  // imad_loop runs 4x the CTAs
  cudaStream_t st = ipc::as_stream(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0, st);
    if (what == 0)
      mma_s8_loop<<<blocks, threads, 0, st>>>(buf, iters);
    else if (what == 1)
      imad_loop<<<blocks * 4, threads, 0, st>>>(reinterpret_cast<uint32_t*>(buf), iters, 3u, 5u);
    else
      dp4a_loop<<<blocks * 4, threads, 0, st>>>(reinterpret_cast<uint32_t*>(buf), iters, 3u, 5u);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return ipc::cuda_fail(e, "ipc_measure_peak");
  const double warps = blocks * threads / 32.0;
  if (what == 0)
    *out = warps * iters * 8 * (16.0 * 8 * 32 * 2) / (best * 1e-3) / 1e12;
  else if (what == 1)
    *out = 4.0 * blocks * threads * iters * 4 * 8 / (best * 1e-3) / 1e12;
  else
    *out = 8.0 * 4.0 * blocks * threads * iters * 4 * 8 / (best * 1e-3) / 1e12;
  return IPC_OK;
}
