// Device helpers shared by the tcgen05 kernels: mbarriers with bounded waits, TMA tile loads,
// shared-memory matrix descriptors (K-major, 64-byte swizzle), tcgen05.mma / commit / fences,
// tensor-memory loads and stores, the widening of int8 limb tiles to fp16 in shared memory, and
// the host-side tensor-map encoders.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "common.cuh"

namespace ipc {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of the given parity. Gives up after 2 s (raising the status word and the
// CTA's abort flag) or, when `abort` is given, as soon as another role has raised that flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* status, volatile uint32_t* abort) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (abort && *abort) return false;
    if (global_ns() - t0 > 2000000000ull) {
      raise_status(status, ST_WAIT_TIMEOUT);
      if (abort) *abort = 1u;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row core-matrix groups 512 bytes
// apart (SBO), LBO unused for this layout (1), descriptor version 1 (bits 46-47), layout type
// SWIZZLE_64B (4 at bits 61-63). Stage tiles are 1024-byte aligned, so the base offset is 0.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (static_cast<uint64_t>(512 >> 4) << 32) |
         (1ull << 46) | (4ull << 61);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(1u)
      : "memory");
}

// Arrives on the mbarrier once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// Stores v into 32 consecutive TMEM columns of this thread's lane.
// 16 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_fill16(uint32_t taddr, uint32_t v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1};" ::"r"(taddr),
      "r"(v)
      : "memory");
}

__device__ __forceinline__ void tmem_fill32(uint32_t taddr, uint32_t v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(v)
      : "memory");
}

// Two 16-bit lanes added independently (mod 2^16 each).
__device__ __forceinline__ uint32_t add16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("add.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Low 16 bits of x (lane 0) and of y (lane 1): the L contributions of two columns.
__device__ __forceinline__ uint32_t pack_lo16(uint32_t x, uint32_t y) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, 0x5410;" : "=r"(d) : "r"(x), "r"(y));
  return d;
}

// (x << 8) mod 2^16 and (y << 8) mod 2^16 in lanes 0 and 1: the 256 C contributions of two
// columns. Byte 0 of each goes to bit 8 of its lane; the zero bytes are the replicated sign of
// byte 3 of x, which is 0x4B for every accumulator value in [2^23, 2^24).
__device__ __forceinline__ uint32_t pack_c16(uint32_t x, uint32_t y) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, 0x4B0B;" : "=r"(d) : "r"(x), "r"(y));
  return d;
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Orders this thread's generic-proxy shared-memory writes before later async-proxy reads
// (tcgen05.mma operands), once the writer's mbarrier arrive has been observed.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}

__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

// Two int8 limbs (bytes 2i, 2i+1 of the word, selected by SEL) as two fp16 values, exactly:
// with the sign bit flipped a byte is u = v + 128 in [0, 255], the fp16 pattern 0x6400 | u is
// 1024 + u (exponent 10, u in the low mantissa bits), and subtracting 1152 leaves v, an integer
// far inside fp16's 11-bit significand, so the subtraction is exact.
template <uint32_t SEL>
__device__ __forceinline__ uint32_t widen2(uint32_t flipped) {
  uint32_t h, d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(h) : "r"(flipped), "r"(0x64646464u), "n"(SEL));
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(h), "r"(0x64806480u));  // (1024 + u) - 1152
  return d;
}

// Sixteen int8 limbs (one 16-byte raw chunk, K order) -> the two 16-byte fp16 chunks of the
// same sixteen elements.
__device__ __forceinline__ void widen16(uint4 raw, uint4& c0, uint4& c1) {
  const uint32_t a = raw.x ^ 0x80808080u, b = raw.y ^ 0x80808080u, c = raw.z ^ 0x80808080u,
                 d = raw.w ^ 0x80808080u;
  c0 = make_uint4(widen2<0x4140>(a), widen2<0x4342>(a), widen2<0x4140>(b), widen2<0x4342>(b));
  c1 = make_uint4(widen2<0x4140>(c), widen2<0x4342>(c), widen2<0x4140>(d), widen2<0x4342>(d));
}

// Widens `planes` raw database tiles of a stage to the MMA's operand layout. A raw tile is
// [128 rows][32] int8, rows 32 bytes apart (TMA, no swizzle); its widened tile is [128][32]
// fp16 in the 64-byte swizzled K-major layout that TMA would have written for an fp16 box:
// row r at r * 64, its 16-byte chunk c (elements 8c..8c+7) at chunk position c ^ ((r >> 1) & 3).
// `ct` in [0, NTHREADS) numbers the widening threads; each takes rows (ct >> 1) + (NTHREADS / 2) j,
// half ct & 1 (16 elements), so its swizzle term (ct >> 2) & 3 is fixed.
template <int PLANES, int NTHREADS>
__device__ __forceinline__ void widen_tiles(uint32_t raw, uint32_t raw_stride, uint32_t dst, uint32_t dst_stride,
                                            uint32_t ct) {
  static_assert(NTHREADS == 32 || NTHREADS == 64 || NTHREADS == 128, "one, two or four widening warps");
  constexpr int JOBS = PLANES * 256 / NTHREADS;   // 16-element jobs per thread
  constexpr int ROWS_STEP = NTHREADS / 2;           // rows between a thread's jobs in one plane
  constexpr int PER_PLANE = 128 / ROWS_STEP;        // jobs per plane
  const uint32_t h = ct & 1u, r0 = ct >> 1, sw = (ct >> 2) & 3u;
  const uint32_t o0 = ((2u * h) ^ sw) * 16u, o1 = ((2u * h + 1u) ^ sw) * 16u;
  uint4 v[JOBS];
#pragma unroll
  for (int j = 0; j < JOBS; ++j)
    v[j] = lds128(raw + (j / PER_PLANE) * raw_stride + (r0 + ROWS_STEP * (j % PER_PLANE)) * 32u + 16u * h);
#pragma unroll
  for (int j = 0; j < JOBS; ++j) {
    uint4 c0, c1;
    widen16(v[j], c0, c1);
    const uint32_t row = dst + (j / PER_PLANE) * dst_stride + (r0 + ROWS_STEP * (j % PER_PLANE)) * 64u;
    sts128(row + o0, c0.x, c0.y, c0.z, c0.w);
    sts128(row + o1, c1.x, c1.y, c1.z, c1.w);
  }
}

__device__ __forceinline__ void named_sync(uint32_t id, uint32_t n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// The driver entry point that encodes tensor maps, looked up once.
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// fp16 tensor [rows][cols] (row stride cols * 2 bytes) as a TMA tensor map: box 32 elements
// (one 64-byte swizzled row) x box_rows, 64-byte swizzle, zero fill outside the tensor (query
// rows past n_pad).
inline int make_map_f16(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return IPC_ECUDA;
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {32, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (fp16) failed with CUresult " + std::to_string(static_cast<int>(r)));
    return IPC_ECUDA;
  }
  return IPC_OK;
}

// int8 limb plane [rows][cols] (row stride cols bytes, a multiple of 16) as a TMA tensor map:
// box 32 bytes x box_rows, no swizzle (rows 32 bytes apart in shared memory), zero fill past the
// last row (ragged row tails).
inline int make_map_i8(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return IPC_ECUDA;
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols};
  cuuint32_t box[2] = {32, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (int8) failed with CUresult " + std::to_string(static_cast<int>(r)));
    return IPC_ECUDA;
  }
  return IPC_OK;
}

// Runs a set-up step (a kernel attribute) once per device: attributes belong to the device's
// context, so a process that drives several devices needs it on each.
class PerDevice {
 public:
  template <class F>
  cudaError_t run(F&& f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu_);
    if (dev >= 0 && dev < 64 && ((done_ >> dev) & 1u)) return cudaSuccess;
    e = f();
    if (e == cudaSuccess && dev >= 0 && dev < 64) done_ |= 1ull << dev;
    return e;
  }

 private:
  std::mutex mu_;
  uint64_t done_ = 0;
};

// Number of SMs of the current device.
inline int sm_count_current() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n <= 0)
    return 1;
  return n;
}

}  // namespace tc
}  // namespace ipc
