// A3 -- the plain int32 CUDA-core ring GEMM over Z_{2^16}: one 32-bit IMAD per ring
// multiply-accumulate, accumulating mod 2^32 (a multiple of 2^16, so reduction at the end
// is exact). It reads the same resident limb planes as the tensor-core path and rebuilds
// each u16 element as 256*hi + lo when staging a tile into shared memory.
#include "common.cuh"

namespace ipc {
namespace {

constexpr int TQ = 128, TD = 128, KT = 16;  // tile: query columns x database rows x K elements
constexpr int THREADS = 256;                // 16 x 16 threads, 8 x 8 outputs each
constexpr int LDS = TQ + 4;                 // padded row of the k-major shared tiles (words)

struct Params {
  uint32_t n_cols, x_rows, l;
  const int8_t* b_lo;
  const int8_t* b_hi;
  uint64_t ldb;  // 2l
  const int8_t* x_lo0;
  const int8_t* x_hi0;
  const int8_t* x_lo1;
  const int8_t* x_hi1;
  const uint32_t* col_tags;
  uint64_t seed_own, seed_prev;
  uint32_t vec;
  uint16_t* z;
  uint64_t ldz;
  uint64_t row0;
};

__device__ __forceinline__ uint32_t rebuild(uint32_t lo4, uint32_t hi4, int e) {
  const int lo = static_cast<int8_t>((lo4 >> (8 * e)) & 0xFFu);
  const int hi = static_cast<int8_t>((hi4 >> (8 * e)) & 0xFFu);
  return static_cast<uint32_t>(hi * 256 + lo) & 0xFFFFu;
}

// Loads 8 consecutive K elements of one row from a limb-plane pair.
__device__ __forceinline__ void load8(const int8_t* lo, const int8_t* hi, bool valid, uint32_t (&v)[8]) {
  uint2 a = make_uint2(0, 0), b = make_uint2(0, 0);
  if (valid) {
    a = *reinterpret_cast<const uint2*>(lo);
    b = *reinterpret_cast<const uint2*>(hi);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    v[e] = rebuild(a.x, b.x, e);
    v[4 + e] = rebuild(a.y, b.y, e);
  }
}

__global__ void __launch_bounds__(THREADS) gemm_i32_kernel(const Params p) {
  __shared__ __align__(16) uint32_t As[2][KT][LDS];  // query tile, k-major
  __shared__ __align__(16) uint32_t Bs[2][KT][LDS];  // database tile, k-major
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const uint32_t q0 = blockIdx.x * TQ, d0 = blockIdx.y * TD;
  const uint32_t K = 2 * p.l;
  // staging: thread -> (row, 8-element half of the KT = 16 slice)
  const int srow = tid >> 1, shalf = tid & 1;
  const bool qvalid = q0 + srow < p.n_cols;
  const bool dvalid = d0 + srow < p.x_rows;
  const int8_t* qlo = p.b_lo + static_cast<uint64_t>(q0 + srow) * p.ldb + 8 * shalf;
  const int8_t* qhi = p.b_hi + static_cast<uint64_t>(q0 + srow) * p.ldb + 8 * shalf;
  const uint64_t drow = static_cast<uint64_t>(d0 + srow) * p.l + 8 * shalf;

  uint32_t acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0;

  uint32_t va[8], vb[8];
  auto fetch = [&](uint32_t k0) {
    load8(qlo + k0, qhi + k0, qvalid, va);
    const bool first = k0 < p.l;
    const uint64_t off = drow + (first ? k0 : k0 - p.l);
    load8((first ? p.x_lo0 : p.x_lo1) + off, (first ? p.x_hi0 : p.x_hi1) + off, dvalid, vb);
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      As[buf][8 * shalf + e][srow] = va[e];
      Bs[buf][8 * shalf + e][srow] = vb[e];
    }
  };

  fetch(0);
  stage(0);
  __syncthreads();
  int buf = 0;
  for (uint32_t k0 = 0; k0 < K; k0 += KT) {
    const bool more = k0 + KT < K;
    if (more) fetch(k0 + KT);
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const uint4 a0 = *reinterpret_cast<const uint4*>(&As[buf][k][ty * 8]);
      const uint4 a1 = *reinterpret_cast<const uint4*>(&As[buf][k][ty * 8 + 4]);
      const uint4 b0 = *reinterpret_cast<const uint4*>(&Bs[buf][k][tx * 8]);
      const uint4 b1 = *reinterpret_cast<const uint4*>(&Bs[buf][k][tx * 8 + 4]);
      const uint32_t a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const uint32_t b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
    }
    if (more) {
      stage(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

  // epilogue: + r_i (App. C zero share), store 8 consecutive rows of each of 8 columns
  const uint32_t r = d0 + tx * 8;
  if (r >= p.x_rows) return;
  const uint64_t gr = p.row0 + r;  // multiple of 8
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t col = q0 + ty * 8 + i;
    if (col >= p.n_cols) continue;
    const uint32_t req = p.col_tags[2 * col], tag = p.col_tags[2 * col + 1];
    const uint4 fo = philox(static_cast<uint32_t>(gr >> 3), tag, req, (IPC_D_ZA << 24) | p.vec, p.seed_own);
    const uint4 fp = philox(static_cast<uint32_t>(gr >> 3), tag, req, (IPC_D_ZA << 24) | p.vec, p.seed_prev);
    const uint32_t wo[4] = {fo.x, fo.y, fo.z, fo.w}, wp[4] = {fp.x, fp.y, fp.z, fp.w};
    uint32_t out[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t z0 = acc[i][2 * e] + (wo[e] & 0xFFFFu) - (wp[e] & 0xFFFFu);
      const uint32_t z1 = acc[i][2 * e + 1] + (wo[e] >> 16) - (wp[e] >> 16);
      out[e] = (z0 & 0xFFFFu) | (z1 << 16);
    }
    uint16_t* zc = p.z + static_cast<uint64_t>(col) * p.ldz + r;
    if (r + 8 <= p.x_rows && (p.ldz % 8) == 0) {
      *reinterpret_cast<uint4*>(zc) = make_uint4(out[0], out[1], out[2], out[3]);
    } else {
      for (int e = 0; e < 8 && r + e < p.x_rows; ++e) zc[e] = static_cast<uint16_t>(out[e >> 1] >> (16 * (e & 1)));
    }
  }
}

}  // namespace

int ring_gemm_i32(const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows, const int8_t* b_lo,
                  const int8_t* b_hi, uint32_t n_cols, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                  uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0, cudaStream_t stream) {
  Params p;
  p.n_cols = n_cols;
  p.x_rows = static_cast<uint32_t>(x_rows);
  p.l = l;
  p.b_lo = b_lo;
  p.b_hi = b_hi;
  p.ldb = 2ull * l;
  p.x_lo0 = x_lo[0];
  p.x_hi0 = x_hi[0];
  p.x_lo1 = x_lo[1];
  p.x_hi1 = x_hi[1];
  p.col_tags = col_tags;
  p.seed_own = seed_own;
  p.seed_prev = seed_prev;
  p.vec = vec;
  p.z = z;
  p.ldz = ldz;
  p.row0 = row0;
  dim3 grid((n_cols + TQ - 1) / TQ, static_cast<unsigned>((x_rows + TD - 1) / TD));
  gemm_i32_kernel<<<grid, THREADS, 0, stream>>>(p);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

}  // namespace ipc
