// A4-A8 -- the comparison phase of Alg. 3 on reshared dot products, bit-sliced.
//
// A small group of threads simulates the three parties for one query column and one
// block of 32-row words (each thread a part of the block, joined by the block's upper OR
// gates): 32 comparisons share one 32-bit word per bit position and share component. The arithmetic-to-boolean steps (ShareSplit, full-adder layer,
// ripple-carry BinAdd; App. D) then run 32 comparisons per logic instruction.
// Party p only ever combines its own pair of components (c_p, c_{p-1}) and the
// PRF outputs of its two seeds, as in the App. C product.
#include <mutex>

#include "compare.cuh"
#include "tcgen05.cuh"  // PerDevice

namespace ipc {
namespace {

using namespace cmp;

constexpr int CT = 64;  // threads per CTA
// One thread per part of each (column, OR block) unit, the parts of a unit in consecutive lanes,
// joined by warp shuffles; the modes are those of part_root.
template <int MODE>
__global__ void __launch_bounds__(CT) compare_kernel(const CmpParams P) {
  extern __shared__ uint32_t sm[];  // [S_WORDS][CT]
  const uint32_t tid = threadIdx.x;
  const uint64_t gtid = blockIdx.x * static_cast<uint64_t>(CT) + tid;
  // all threads of a unit leave together, so the group stays complete for the final shuffles
  const uint32_t ks = P.p < LOG2_SPLIT ? P.p : LOG2_SPLIT;
  const uint64_t unit = gtid >> ks;
  const uint32_t part = static_cast<uint32_t>(gtid & ((1u << ks) - 1u));
  if (unit >= static_cast<uint64_t>(P.n_cols) * P.n_blocks) return;
  uint32_t n = static_cast<uint32_t>(unit % P.n_cols);
  const uint32_t blk = static_cast<uint32_t>(unit / P.n_cols);
  if (P.col_tiles) {
    // the first (listed tiles x tile_cols) units of each block row take the listed columns
    const uint32_t active = *P.n_col_list * P.tile_cols;
    if (n >= active) return;
    n = P.col_tiles[n / P.tile_cols] * P.tile_cols + n % P.tile_cols;
    if (n >= P.n_cols) return;
  }
  B3 root;
  uint32_t nwords;
  part_root<MODE, CT>(P, n, blk, part, ks, sm, tid, root, nwords);
  const uint32_t req = P.col_tags[2 * n], tag = P.col_tags[2 * n + 1];
  const uint32_t sub_p = P.p - ks;
  const uint64_t bword0 = (P.row0 + (static_cast<uint64_t>(blk) << (5 + P.p))) >> 5;  // the block's first word
  // ---- join the parts: at step s, part t (t a multiple of 2^s) is the left child and part
  // t + 2^(s-1) the right child of the level sub_p + s node; a part without words is carried
  // (words fill the parts from the first, so a right child with words has a left one). ----
  const uint32_t group_mask = ((1u << (1u << ks)) - 1u) << (tid & (32u - (1u << ks)));
  uint32_t has = nwords > 0 ? 1u : 0u;
  for (uint32_t s = 1; s <= ks; ++s) {
    const uint32_t d = 1u << (s - 1);
    B3 right;
    right.c0 = __shfl_xor_sync(group_mask, root.c0, d);
    right.c1 = __shfl_xor_sync(group_mask, root.c1, d);
    right.c2 = __shfl_xor_sync(group_mask, root.c2, d);
    const uint32_t right_has = __shfl_xor_sync(group_mask, has, d);
    if ((part & ((2u << (s - 1)) - 1u)) == 0 && right_has) {
      const uint32_t lvl = sub_p + s;
      root = bor(P.seeds, root, right, static_cast<uint32_t>((bword0 >> lvl) + (part >> s)), tag, req,
                 (IPC_D_OR << 24) | (1u << 16) | lvl);
    }
    has |= right_has;
  }
  if (part != 0) return;
  const uint64_t bglob = (P.row0 >> (5 + P.p)) + blk;
  const uint64_t plane = static_cast<uint64_t>(P.n_cols) * P.ld_roots;
  const uint64_t at = static_cast<uint64_t>(n) * P.ld_roots + bglob;
  P.roots[at] = root.c0;
  P.roots[plane + at] = root.c1;
  P.roots[2 * plane + at] = root.c2;
}

// Rows stage of the OR tree above the block roots: per column, pairwise levels p+1, p+2, ...
__global__ void or_rows_kernel(uint32_t* roots, uint64_t ld_roots, uint64_t plane, uint32_t n_cols, uint32_t n_blocks,
                               uint32_t p, const uint32_t* col_tags, Seeds sd) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_cols) return;
  const uint32_t req = col_tags[2 * n], tag = col_tags[2 * n + 1];
  uint32_t* r0 = roots + static_cast<uint64_t>(n) * ld_roots;
  uint32_t cnt = n_blocks, level = p + 1;
  while (cnt > 1) {
    const uint32_t half = cnt / 2;
    for (uint32_t j = 0; j < half; ++j) {
      const B3 a = {r0[2 * j], r0[plane + 2 * j], r0[2 * plane + 2 * j]};
      const B3 b = {r0[2 * j + 1], r0[plane + 2 * j + 1], r0[2 * plane + 2 * j + 1]};
      const B3 c = bor(sd, a, b, j, tag, req, (IPC_D_OR << 24) | (1u << 16) | level);
      r0[j] = c.c0;
      r0[plane + j] = c.c1;
      r0[2 * plane + j] = c.c2;
    }
    if (cnt & 1u) {
      r0[half] = r0[cnt - 1];
      r0[plane + half] = r0[plane + cnt - 1];
      r0[2 * plane + half] = r0[2 * plane + cnt - 1];
    }
    cnt = half + (cnt & 1u);
    ++level;
  }
}

// Block roots from the part roots of the fused GEMM + comparison kernel: per (column, 1,024-row
// block), the block's eight 128-row parts joined with the block's upper three OR levels, gate
// for gate as the shuffle join of compare_kernel (part t is the left child at step s when t is a
// multiple of 2^s; a part past the last row is carried).
__global__ void or_join_parts_kernel(const uint32_t* parts, uint64_t ld_parts, uint64_t n_rt, uint32_t n_cols,
                                     uint32_t n_blocks, uint64_t row0, const uint32_t* col_tags, Seeds sd,
                                     uint32_t* roots, uint64_t ld_roots, uint64_t roots_plane) {
  constexpr uint32_t P5 = 5, KS = LOG2_SPLIT, SUB_P = P5 - KS, NPART = 1u << KS;
  const uint64_t u = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (u >= static_cast<uint64_t>(n_cols) * n_blocks) return;
  const uint32_t n = static_cast<uint32_t>(u % n_cols), blk = static_cast<uint32_t>(u / n_cols);
  const uint32_t req = col_tags[2 * n], tag = col_tags[2 * n + 1];
  const uint64_t plane = static_cast<uint64_t>(n_cols) * ld_parts;
  const uint64_t bword0 = (row0 >> 5) + (static_cast<uint64_t>(blk) << P5);
  B3 r[NPART];
  uint32_t has[NPART];
#pragma unroll
  for (uint32_t t = 0; t < NPART; ++t) {
    const uint64_t rt = static_cast<uint64_t>(blk) * NPART + t;
    has[t] = rt < n_rt ? 1u : 0u;
    const uint64_t at = static_cast<uint64_t>(n) * ld_parts + rt;
    r[t] = has[t] ? B3{parts[at], parts[plane + at], parts[2 * plane + at]} : B3{0u, 0u, 0u};
  }
#pragma unroll
  for (uint32_t s = 1; s <= KS; ++s) {
    const uint32_t d = 1u << (s - 1), lvl = SUB_P + s;
#pragma unroll
    for (uint32_t t = 0; t < NPART; t += 2 * d) {
      if (has[t + d])
        r[t] = bor(sd, r[t], r[t + d], static_cast<uint32_t>((bword0 >> lvl) + (t >> s)), tag, req,
                   (IPC_D_OR << 24) | (1u << 16) | lvl);
      has[t] |= has[t + d];
    }
  }
  const uint64_t at = static_cast<uint64_t>(n) * ld_roots + (row0 >> (5 + P5)) + blk;
  roots[at] = r[0].c0;
  roots[roots_plane + at] = r[0].c1;
  roots[2 * roots_plane + at] = r[0].c2;
}

// Rotation stage and lane fold, per query.
__global__ void or_queries_kernel(const uint32_t* roots, uint64_t ld_roots, uint64_t plane, uint32_t Q, uint32_t R,
                                  const uint32_t* col_tags, Seeds sd, uint8_t* bit_shares) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const uint32_t req = col_tags[2 * (q * R)], tag = col_tags[2 * (q * R) + 1] & ~31u;
  B3 w[32];
  for (uint32_t rho = 0; rho < R; ++rho) {
    const uint64_t at = static_cast<uint64_t>(q * R + rho) * ld_roots;
    w[rho] = {roots[at], roots[plane + at], roots[2 * plane + at]};
  }
  uint32_t cnt = R, level = 1;
  while (cnt > 1) {
    const uint32_t half = cnt / 2;
    for (uint32_t j = 0; j < half; ++j) w[j] = bor(sd, w[2 * j], w[2 * j + 1], j, tag, req, (IPC_D_OR << 24) | (2u << 16) | level);
    if (cnt & 1u) w[half] = w[cnt - 1];
    cnt = half + (cnt & 1u);
    ++level;
  }
  B3 x = w[0];
  for (uint32_t L = 1; L <= 5; ++L) {
    const uint32_t h = 32u >> L;
    const uint32_t m = (1u << h) - 1u;
    const B3 lo = {x.c0 & m, x.c1 & m, x.c2 & m};
    const B3 hi = {(x.c0 >> h) & m, (x.c1 >> h) & m, (x.c2 >> h) & m};
    const B3 y = bor(sd, lo, hi, 0u, tag, req, (IPC_D_OR << 24) | (3u << 16) | L);
    x = {y.c0 & m, y.c1 & m, y.c2 & m};
  }
  bit_shares[q] = x.c0 & 1u;
  bit_shares[Q + q] = x.c1 & 1u;
  bit_shares[2 * Q + q] = x.c2 & 1u;
}

int launch_compare(CmpParams& P, int mode, cudaStream_t st) {
  if (P.p > 5) {  // a part's OR stack holds levels 0..5 - LOG2_SPLIT
    set_error("compare: log2_block_words must be <= 5");
    return IPC_EINVAL;
  }
  P.n_blocks = static_cast<uint32_t>((P.n_rows + (32ull << P.p) - 1) >> (5 + P.p));
  const uint64_t threads = (static_cast<uint64_t>(P.n_cols) * P.n_blocks) << (P.p < LOG2_SPLIT ? P.p : LOG2_SPLIT);
  const size_t smem = sizeof(uint32_t) * S_WORDS * CT;
  static tc::PerDevice attr;  // a kernel attribute belongs to one device's context
  IPC_CUDA_TRY(attr.run([smem] {
    cudaError_t e = cudaFuncSetAttribute(compare_kernel<MODE_LIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(compare_kernel<MODE_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(compare_kernel<MODE_LIFTFREE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
    return e;
  }));
  const unsigned grid = static_cast<unsigned>((threads + CT - 1) / CT);
  if (mode == MODE_PLAIN)
    compare_kernel<MODE_PLAIN><<<grid, CT, smem, st>>>(P);
  else if (mode == MODE_LIFTFREE)
    compare_kernel<MODE_LIFTFREE><<<grid, CT, smem, st>>>(P);
  else
    compare_kernel<MODE_LIFT><<<grid, CT, smem, st>>>(P);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

CmpParams base_params(size_t ldz, uint32_t n_cols, size_t n_rows, uint64_t row0, const uint32_t* col_tags,
                      const uint64_t seeds[3], uint32_t thr_a, uint32_t p, uint32_t* roots, size_t ld_roots,
                      uint8_t* msb_out, size_t ld_msb) {
  CmpParams P{};
  for (int j = 0; j < 3; ++j) P.seeds.s[j] = seeds[j];
  P.ldz = ldz;
  P.n_cols = n_cols;
  P.n_rows = n_rows;
  P.row0 = row0;
  P.col_tags = col_tags;
  P.thr_a = thr_a;
  P.p = p;
  P.roots = roots;
  P.ld_roots = ld_roots;
  P.msb_out = msb_out;
  P.ld_msb = ld_msb;
  return P;
}

}  // namespace

int compare_launch_tiles(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz,
                         uint32_t n_cols, size_t n_rows, uint64_t row0, const uint32_t* col_tags,
                         const uint64_t seeds[3], uint32_t thr_a, uint32_t p, uint32_t* roots, size_t ld_roots,
                         uint8_t* msb_out, size_t ld_msb, const uint32_t* col_tiles, const uint32_t* n_col_list,
                         uint32_t tile_cols, cudaStream_t st, const uint32_t* col_rows, bool plain) {
  CmpParams P = base_params(ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, p, roots, ld_roots, msb_out, ld_msb);
  for (int j = 0; j < 3; ++j) {
    P.zc[j] = z_code[j];
    P.zm[j] = z_mask[j];
  }
  P.col_tiles = col_tiles;
  P.n_col_list = n_col_list;
  P.tile_cols = tile_cols;
  P.col_rows = col_rows;
  return launch_compare(P, plain ? MODE_PLAIN : MODE_LIFT, st);
}

// ConstLift (zc16 set, zc32 null) or NoLift (zc32 set): ml32 the Z_2^32 components of ml.
int compare_launch_liftfree(const uint16_t* const zc16[3], const uint32_t* const zc32[3],
                            const uint32_t* const ml32[3], size_t ldz, uint32_t n_cols, size_t n_rows, uint64_t row0,
                            const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a, uint32_t thr_b,
                            uint32_t p, uint32_t* roots, size_t ld_roots, uint8_t* msb_out, size_t ld_msb,
                            cudaStream_t st) {
  CmpParams P = base_params(ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, p, roots, ld_roots, msb_out, ld_msb);
  for (int j = 0; j < 3; ++j) {
    P.zc[j] = zc16 ? zc16[j] : nullptr;
    P.zc32[j] = zc32 ? zc32[j] : nullptr;
    P.zm32[j] = ml32[j];
  }
  P.thr_b = zc32 ? (thr_b == 0 ? 65536u : thr_b) : 65536u;
  return launch_compare(P, MODE_LIFTFREE, st);
}

int compare_launch(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz, uint32_t n_cols,
                   size_t n_rows, uint64_t row0, const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a,
                   uint32_t p, uint32_t* roots, size_t ld_roots, uint8_t* msb_out, size_t ld_msb, cudaStream_t st) {
  return compare_launch_tiles(z_code, z_mask, ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, p, roots, ld_roots,
                              msb_out, ld_msb, nullptr, nullptr, 0, st, nullptr, false);
}

// Block roots of one chunk (rows [row0, row0 + n_rows), row0 a multiple of 1,024) from the part
// roots of ring_gemm_compare_tc: parts [3][n_cols][ld_parts], roots [3][n_cols][ld_roots].
int or_join_parts_launch(const uint32_t* parts, size_t ld_parts, uint32_t n_cols, size_t n_rows, uint64_t row0,
                         const uint32_t* col_tags, const uint64_t seeds[3], uint32_t* roots, size_t ld_roots,
                         cudaStream_t st) {
  Seeds sd;
  for (int j = 0; j < 3; ++j) sd.s[j] = seeds[j];
  const uint64_t n_rt = (n_rows + 127) / 128;
  const uint32_t n_blocks = static_cast<uint32_t>((n_rows + 1023) / 1024);
  const uint64_t units = static_cast<uint64_t>(n_cols) * n_blocks;
  if (units == 0) return IPC_OK;
  or_join_parts_kernel<<<static_cast<unsigned>((units + 127) / 128), 128, 0, st>>>(
      parts, ld_parts, n_rt, n_cols, n_blocks, row0, col_tags, sd, roots, ld_roots,
      static_cast<uint64_t>(n_cols) * ld_roots);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

// plane: words between the three components' root planes (n_cols * ld_roots for a stand-alone
// request; the pool's column count * ld_roots for a request occupying a range of a column pool).
int or_finalize_strided(uint32_t* roots, size_t ld_roots, size_t plane, uint32_t n_blocks, uint32_t p, uint32_t Q,
                        uint32_t R, const uint32_t* col_tags, const uint64_t seeds[3], uint8_t* bit_shares,
                        cudaStream_t st) {
  Seeds sd;
  for (int j = 0; j < 3; ++j) sd.s[j] = seeds[j];
  const uint32_t n_cols = Q * R;
  or_rows_kernel<<<(n_cols + 127) / 128, 128, 0, st>>>(roots, ld_roots, plane, n_cols, n_blocks, p, col_tags, sd);
  IPC_CUDA_TRY(cudaGetLastError());
  or_queries_kernel<<<(Q + 63) / 64, 64, 0, st>>>(roots, ld_roots, plane, Q, R, col_tags, sd, bit_shares);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

// Per person: (b0 OR b1) OR (b2 OR b3) on boolean sharings; gate t (0: b0|b1, 1: b2|b3, 2: the
// root) of person p takes its zero-share bits from bit 0 of word 0 of
// Philox(seed_j, (p, 0, req, D_COMB << 24 | t)).
__global__ void or_combine_kernel(const uint8_t* b0, const uint8_t* b1, const uint8_t* b2, const uint8_t* b3,
                                  uint32_t P, uint32_t req, Seeds sd, uint8_t* out) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  auto load = [&](const uint8_t* b) { return B3{b[p] & 1u, b[P + p] & 1u, b[2 * P + p] & 1u}; };
  auto gate = [&](const B3& x, const B3& y, uint32_t t) {
    const uint32_t F0 = philox(p, 0u, req, (IPC_D_COMB << 24) | t, sd.s[0]).x & 1u;
    const uint32_t F1 = philox(p, 0u, req, (IPC_D_COMB << 24) | t, sd.s[1]).x & 1u;
    const uint32_t F2 = philox(p, 0u, req, (IPC_D_COMB << 24) | t, sd.s[2]).x & 1u;
    return bx(bx(x, y), band(x, y, F0, F1, F2));
  };
  const B3 left = gate(load(b0), load(b1), 0), right = gate(load(b2), load(b3), 1);
  const B3 root = gate(left, right, 2);
  out[p] = root.c0 & 1u;
  out[P + p] = root.c1 & 1u;
  out[2 * P + p] = root.c2 & 1u;
}

int or_combine_launch(const uint8_t* const bits[4], uint32_t P, uint32_t req, const uint64_t seeds[3], uint8_t* out,
                      cudaStream_t st) {
  Seeds sd;
  for (int j = 0; j < 3; ++j) sd.s[j] = seeds[j];
  or_combine_kernel<<<(P + 127) / 128, 128, 0, st>>>(bits[0], bits[1], bits[2], bits[3], P, req, sd, out);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

int or_finalize_launch(uint32_t* roots, size_t ld_roots, uint32_t n_blocks, uint32_t p, uint32_t Q, uint32_t R,
                       const uint32_t* col_tags, const uint64_t seeds[3], uint8_t* bit_shares, cudaStream_t st) {
  return or_finalize_strided(roots, ld_roots, static_cast<size_t>(Q) * R * ld_roots, n_blocks, p, Q, R, col_tags, seeds,
                             bit_shares, st);
}

}  // namespace ipc

// ---------------------------------------------------------------------------------------------
// Allocation-free comparison + OR reduction.
//
// Some callers may not allocate device memory once they are running: a host framework that
// owns the whole device memory pool and forbids extensions from calling cudaMalloc, or a
// service that reserves all of its memory at start-up so that no allocation can fail or
// synchronise the device mid-flight. For them the block-root scratch that ipc_compare
// writes and ipc_or_finalize reads lives in a fixed array compiled into this library
// (g_noalloc_roots, 4 MiB, present on every GPU that loads the library until exit).
// ---------------------------------------------------------------------------------------------
#include <mutex>

namespace ipc {
namespace {

constexpr size_t kNoAllocRootWords = size_t(1) << 20;  // 4 MiB of 32-bit block-root words
constexpr uint32_t kNoAllocLog2Block = 5;              // 1024-row blocks

__device__ __align__(256) uint32_t g_noalloc_roots[kNoAllocRootWords];

std::mutex g_noalloc_mu;
uint32_t* g_noalloc_addr[128] = {};

// Device address of g_noalloc_roots on the current device (looked up once per device; the
// host-side symbol is only a stand-in for it and must never be handed to a kernel).
int noalloc_scratch(uint32_t** out) {
  int dev = 0;
  IPC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    set_error("ipc_compare_or_noalloc: device ordinal out of range");
    return IPC_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    IPC_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_roots));
    g_noalloc_addr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_noalloc_addr[dev];
  return IPC_OK;
}

}  // namespace
}  // namespace ipc

extern "C" int ipc_compare_or_noalloc(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz,
                                      uint32_t Q, uint32_t R, size_t n_rows, const uint32_t* col_tags,
                                      const uint64_t seeds[3], uint32_t thr_a, uint8_t* bit_shares, void* stream) {
  using namespace ipc;
  if (!z_code || !z_mask || !col_tags || !seeds || !bit_shares) {
    set_error("ipc_compare_or_noalloc: null pointer");
    return IPC_EINVAL;
  }
  for (int j = 0; j < 3; ++j)
    if (!z_code[j] || !z_mask[j] || (reinterpret_cast<uintptr_t>(z_code[j]) & 15) ||
        (reinterpret_cast<uintptr_t>(z_mask[j]) & 15)) {
      set_error("ipc_compare_or_noalloc: dot planes must be non-null and 16-byte aligned");
      return IPC_EINVAL;
    }
  if (Q == 0 || R == 0 || R > 31 || n_rows == 0 || ldz % 8 != 0 || ldz < n_rows) {
    set_error("ipc_compare_or_noalloc: need Q >= 1, 1 <= R <= 31, n_rows >= 1, ldz >= n_rows, ldz % 8 == 0");
    return IPC_EINVAL;
  }
  const uint64_t n_cols = static_cast<uint64_t>(Q) * R;
  const uint64_t n_blocks = (n_rows + (32ull << kNoAllocLog2Block) - 1) >> (5 + kNoAllocLog2Block);
  if (3 * n_cols * n_blocks > kNoAllocRootWords) {
    set_error("ipc_compare_or_noalloc: 3 * Q * R * ceil(n_rows / 1024) = " + std::to_string(3 * n_cols * n_blocks) +
              " block-root words exceed the fixed scratch of " + std::to_string(kNoAllocRootWords) +
              " words; use ipc_compare + ipc_or_finalize with caller-allocated roots");
    return IPC_EINVAL;
  }
  uint32_t* roots = nullptr;
  int rc = noalloc_scratch(&roots);
  if (rc) return rc;
  // Every root word that ipc_or_finalize reads is written first by this same call, so the
  // previous call's contents never leak into the result and nothing needs clearing.
  rc = compare_launch(z_code, z_mask, ldz, static_cast<uint32_t>(n_cols), n_rows, 0, col_tags, seeds, thr_a,
                      kNoAllocLog2Block, roots, n_blocks, nullptr, 0, as_stream(stream));
  if (rc) return rc;
  return or_finalize_launch(roots, n_blocks, static_cast<uint32_t>(n_blocks), kNoAllocLog2Block, Q, R, col_tags,
                            seeds, bit_shares, as_stream(stream));
}
