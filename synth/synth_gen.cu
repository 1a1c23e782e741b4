// Device implementation of the database-bit generator of synth/__init__.py (same definition:
// SplitMix64 output function used counter-style). Holds none of the method's arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kMaskP16 = 58982u;
constexpr uint64_t kStreamCode = 1, kStreamMask = 2;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ inline uint64_t h(uint64_t base, uint64_t idx) { return mix64(base + (idx + 1) * kGamma); }

// one thread per (row, output word) of both the code and the mask bit rows
__global__ void db_bits_kernel(uint64_t base_code, uint64_t base_mask, uint64_t row0, uint32_t n, uint32_t l,
                               uint64_t* code, uint64_t* mask) {
  const uint32_t nw = (l + 63) / 64, nd = (l + 3) / 4;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (tid >= static_cast<uint64_t>(n) * nw) return;
  const uint64_t r = tid / nw;
  const uint32_t w = static_cast<uint32_t>(tid % nw);
  const uint64_t grow = row0 + r;
  uint64_t c = h(base_code, grow * nw + w);
  uint64_t m = 0;
  for (uint32_t t = 0; t < 16; ++t) {
    const uint32_t d = w * 16 + t;  // draw index: bits 4d .. 4d+3
    if (d >= nd) break;
    const uint64_t draw = h(base_mask, grow * nd + d);
    for (uint32_t j = 0; j < 4; ++j) {
      const uint32_t bit = 4 * d + j;
      if (bit >= l) break;
      if (((draw >> (16 * j)) & 0xFFFFu) < kMaskP16) m |= 1ull << (bit & 63);
    }
  }
  if (w == nw - 1 && (l % 64)) c &= (1ull << (l % 64)) - 1;
  code[tid] = c;
  mask[tid] = m;
}

}  // namespace

// code, mask: device [n][ceil(l/64)] uint64 outputs for global rows row0 .. row0+n-1.
extern "C" int synth_db_bits(uint64_t seed, uint64_t row0, uint32_t n, uint32_t l, uint64_t* code, uint64_t* mask,
                             void* stream) {
  if (n == 0) return 0;
  const uint64_t base_code = mix64(seed ^ (kStreamCode << 56));
  const uint64_t base_mask = mix64(seed ^ (kStreamMask << 56));
  const uint64_t threads = static_cast<uint64_t>(n) * ((l + 63) / 64);
  db_bits_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      base_code, base_mask, row0, n, l, code, mask);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
