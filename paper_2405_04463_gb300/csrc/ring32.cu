// A0-A3 over Z_{2^32} for the lifting variants (Sec. 5.1, Sec. 6.2): ConstLift computes ml,
// NoLift also the code dot product, over Z_{2^32}.
//
// A0: client sharing of the masked bits and mask bits read in Z_{2^32}.
// A1/A2: four balanced int8 limbs per element, x = x0 + 2^8 x1 + 2^16 x2 + 2^24 x3 (mod 2^32),
//        each written as the bf16 bit pattern of the limb (exact).
// A3 (gemm_tc32_kernel): the ring dot product on tcgen05 with fp32 TMEM accumulators, exact:
//     z = sum_s 2^(8s) S_s (mod 2^32),  S_s = sum over a + b = s of sum_k x_a[k] y_b[k],
//   ten limb products per k (1 + 2 + 3 + 4 for s = 0..3); products with a + b > 3 vanish mod
//   2^32. S_s has its own accumulator, started at M = 1.5 * 2^23 and drained while every partial
//   sum stays within M +- 2^22 (so every fp32 addition is exact, as in the 16-bit kernel): S_s
//   gains at most (s + 1) 2^14 per k, so S_3 and S_2 are drained every 64 k, S_1 every 128 k,
//   S_0 every 256 k. A drain adds (bits - bits(M)) << 8s to a 32-bit running sum per column;
//   bits(M) << 8s vanishes mod 2^32 for s >= 2, and the S_1 and S_0 terms are subtracted once,
//   up front.
//
// One CTA per tile of 128 database rows x 128 query columns (MMA 128 x 128 x 16), 10 warps:
//   warp 0 lane 0  TMA producer: per k-block of 32 elements, eight tiles (database limbs 0-3,
//                  query limbs 0-3; 128 x 32 bf16 each, 64-byte swizzle) into a 3-stage ring.
//   warp 1 lane 0  MMA issuer: per k-block the S_3, S_2, S_1, S_0 products in that order,
//                  committing S_s-full after the last k-block of its drain period and the stage
//                  after the k-block's S_0 products. S_3's drain overlaps the k-block's other six
//                  products; S_2's the S_1, S_0 products and the next k-block's S_3 products.
//   warps 2-9      drain: each thread owns one TMEM lane (database row) and 64 columns.
// TMEM: S_s in columns [128 s, 128 s + 128), all 512 columns.
// Every wait is bounded (2 s, or sooner once another role has failed); a failed CTA raises the
// status word, lets its copies and MMAs finish, frees its tensor memory and stores nothing.
#include <mutex>
#include <string>

#include "tcgen05_pair.cuh"

namespace ipc {
namespace {

using namespace tc;

// Balanced signed limbs of x mod 2^32, least significant first, each in [-128, 127].
__device__ __forceinline__ void limbs32(uint32_t x, int8_t (&o)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int v = static_cast<int8_t>(x & 0xFFu);
    o[i] = static_cast<int8_t>(v);
    x = (x - static_cast<uint32_t>(v)) >> 8;  // exact: x - v is 0 mod 256
  }
}

__device__ __forceinline__ uint16_t bf16_of8(int8_t v) {
  return static_cast<uint16_t>(__float_as_uint(static_cast<float>(v)) >> 16);
}

// A0 over Z_{2^32}: one thread per (row, 2 consecutive elements); one Philox call per vector
// gives both elements' x_0, x_1 (words 2e, 2e + 1).
__global__ void encode_share32_kernel(const uint64_t* __restrict__ code_bits, const uint64_t* __restrict__ mask_bits,
                                      uint32_t n, uint32_t l, uint64_t seed, uint32_t side, uint32_t idx0,
                                      uint32_t* __restrict__ code_sh, uint32_t* __restrict__ mask_sh) {
  const uint32_t pairs = l >> 1;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (tid >= static_cast<uint64_t>(n) * pairs) return;
  const uint32_t r = static_cast<uint32_t>(tid / pairs), t = static_cast<uint32_t>(tid % pairs);
  const uint32_t nw = (l + 63) >> 6;
  const uint32_t b0 = t << 1;
  const uint32_t cw = static_cast<uint32_t>(code_bits[static_cast<uint64_t>(r) * nw + (b0 >> 6)] >> (b0 & 63)) & 3u;
  const uint32_t mw = static_cast<uint32_t>(mask_bits[static_cast<uint64_t>(r) * nw + (b0 >> 6)] >> (b0 & 63)) & 3u;
  const uint64_t plane = static_cast<uint64_t>(n) * l;
  const uint64_t at = static_cast<uint64_t>(r) * l + b0;
#pragma unroll
  for (uint32_t vec = 0; vec < 2; ++vec) {
    const uint4 w = philox(t, idx0 + r, (side << 8) | vec, IPC_D_SHARE32 << 24, seed);
    uint32_t x0[2] = {w.x, w.z}, x1[2] = {w.y, w.w}, x2[2];
#pragma unroll
    for (uint32_t e = 0; e < 2; ++e) {
      const uint32_t cb = (cw >> e) & 1u, mb = (mw >> e) & 1u;
      const uint32_t val = vec == 0 ? (mb - 2u * (cb & mb)) : mb;  // T = -1, U = 0, F = +1 / mask bit
      x2[e] = val - x0[e] - x1[e];
    }
    uint32_t* dst = vec == 0 ? code_sh : mask_sh;
    *reinterpret_cast<uint2*>(dst + at) = make_uint2(x0[0], x0[1]);
    *reinterpret_cast<uint2*>(dst + plane + at) = make_uint2(x1[0], x1[1]);
    *reinterpret_cast<uint2*>(dst + 2 * plane + at) = make_uint2(x2[0], x2[1]);
  }
}

// A1 over Z_{2^32}: 4 elements per thread, one bf16 limb plane per limb.
__global__ void split_limbs32_kernel(const uint32_t* __restrict__ x, size_t count, uint16_t* __restrict__ o0,
                                     uint16_t* __restrict__ o1, uint16_t* __restrict__ o2,
                                     uint16_t* __restrict__ o3) {
  const size_t i4 = (blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x) * 4;
  if (i4 >= count) return;
  uint16_t* out[4] = {o0, o1, o2, o3};
  if (i4 + 4 <= count) {
    const uint4 v = *reinterpret_cast<const uint4*>(x + i4);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t packed[4][2] = {};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int8_t lb[4];
      limbs32(w[e], lb);
#pragma unroll
      for (int i = 0; i < 4; ++i) packed[i][e >> 1] |= static_cast<uint32_t>(bf16_of8(lb[i])) << (16 * (e & 1));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) *reinterpret_cast<uint2*>(out[i] + i4) = make_uint2(packed[i][0], packed[i][1]);
  } else {
    for (size_t e = i4; e < count; ++e) {
      int8_t lb[4];
      limbs32(x[e], lb);
      for (int i = 0; i < 4; ++i) out[i][e] = bf16_of8(lb[i]);
    }
  }
}

// A2 over Z_{2^32}: party i's operand [rot(Y_i + Y_{i-1}) | rot(Y_i)] (K = 2l), or, for one
// segment, rot(Y_i) alone (K = l); one thread per output element, four bf16 limb planes.
__global__ void prep_query32_kernel(const uint32_t* __restrict__ y, uint64_t plane, uint32_t Q, ipc_geom g,
                                    uint32_t party, uint32_t segments, uint16_t* __restrict__ o0,
                                    uint16_t* __restrict__ o1, uint16_t* __restrict__ o2, uint16_t* __restrict__ o3,
                                    uint32_t n_pad) {
  const uint32_t l = g.rows * g.cols * g.cell, K = segments * l;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const uint64_t total = static_cast<uint64_t>(n_pad) * K;
  if (tid >= total) return;
  const uint32_t n = static_cast<uint32_t>(tid / K);
  const uint32_t k = static_cast<uint32_t>(tid % K);
  uint32_t val = 0;
  if (n < Q * g.R) {
    const uint32_t q = n / g.R, rho = n % g.R;
    const int32_t shift = g.rot_lo + static_cast<int32_t>(rho);
    const uint32_t kk = k < l ? k : k - l;
    const uint32_t c = kk % g.cell, j = (kk / g.cell) % g.cols, r = kk / (g.cell * g.cols);
    int32_t js = (static_cast<int32_t>(j) - shift) % static_cast<int32_t>(g.cols);
    if (js < 0) js += g.cols;
    const uint32_t src = (r * g.cols + static_cast<uint32_t>(js)) * g.cell + c;
    const uint32_t prev = (party + 2) % 3;
    val = y[party * plane + static_cast<uint64_t>(q) * l + src];
    if (segments == 2 && k < l) val += y[prev * plane + static_cast<uint64_t>(q) * l + src];  // y_i + y_{i-1}
  }
  int8_t lb[4];
  limbs32(val, lb);
  o0[tid] = bf16_of8(lb[0]);
  o1[tid] = bf16_of8(lb[1]);
  o2[tid] = bf16_of8(lb[2]);
  o3[tid] = bf16_of8(lb[3]);
}

// ----------------------------------- A3 -----------------------------------
// PAIR = false: one CTA per 128-row x 128-column tile (MMA 128 x 128 x 16).
// PAIR = true:  a cluster of two CTAs per 256-row x 128-column tile (cta_group::2, M = 256): CTA
//   rank r owns rows 128 r .. 128 r + 127 and holds query columns 64 r .. 64 r + 63 of the tile in
//   its shared memory, so each SM reads half the query tile per MMA. With N = 128 a single CTA's
//   MMAs read 8 KiB of shared memory per 64 tensor cycles, the whole read rate; the pair reads
//   6 KiB. The leader (rank 0) issues the MMAs and commits to both CTAs' barriers; both CTAs'
//   producers count their copies on the leader's full barrier; the drain-empty barriers live in
//   the leader and count both CTAs' drain warps.
constexpr int TM = 128, TN = 128, KB = 32, LIMBS = 4;
constexpr int TILE_BYTES = TM * KB * 2;  // 8 KiB database tile
constexpr int THREADS = 10 * 32, DRAIN_THREADS = 8 * 32;
constexpr uint32_t KB_PER_CHUNK = 2;  // 64 k: the shortest drain period
constexpr uint32_t TMEM_COLS = 4 * TN;
constexpr uint32_t MAGIC = 0x4B400000u;  // fp32 bits of 1.5 * 2^23

template <bool PAIR>
struct Cfg32 {
  static constexpr int HN = PAIR ? TN / 2 : TN;                  // query columns held by this CTA
  static constexpr int B_TILE = HN * KB * 2;                     // 4 or 8 KiB
  static constexpr int STAGE_BYTES = LIMBS * TILE_BYTES + LIMBS * B_TILE;  // 48 or 64 KiB
  static constexpr int STAGES = PAIR ? 4 : 3;
  // full[S], empty[S], g_full[4], g_empty[4], done
  static constexpr int NUM_BARS = 2 * STAGES + 9;
  // pair: 16 KiB after the ring, so that every MMA operand read stays inside the allocation
  static constexpr int SLACK = PAIR ? 16384 : 0;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + SLACK + 1024 + 8 * NUM_BARS;
  // kind::f16: D f32, A and B bf16, both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(TN >> 3) << 17) |
                                    (static_cast<uint32_t>((PAIR ? 2 * TM : TM) >> 4) << 24);
  static_assert(TN * TM * 4 <= STAGES * STAGE_BYTES, "the z tile is staged in the stage ring");
};

// Drain period of S_s in 64-k chunks.
__host__ __device__ constexpr uint32_t period(int s) { return s == 0 ? 4u : (s == 1 ? 2u : 1u); }

struct Maps32 {
  CUtensorMap b[LIMBS];   // query limbs [n_pad][K]
  CUtensorMap a0[LIMBS];  // database limbs of the first K segment [x_rows][l]
  CUtensorMap a1[LIMBS];  // and of the second
};

struct Tc32Params {
  uint32_t n_cols;
  uint32_t x_rows;
  uint32_t kb_total;  // K / KB
  uint32_t kb_half;   // l / KB: k-blocks below it read the first segment's planes
  const uint32_t* col_tags;
  uint64_t seed_own, seed_prev;
  uint32_t vec;
  uint32_t* z;
  uint64_t ldz;
  uint64_t row0;
  uint32_t* status;
};

template <bool PAIR>
__global__ void __launch_bounds__(THREADS, 1) gemm_tc32_kernel(const __grid_constant__ Maps32 m, const Tc32Params p) {
  using C = Cfg32<PAIR>;
  constexpr int STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ uint32_t s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t tiles = smem_addr(smem);
  const uint32_t bars = tiles + STAGES * STAGE_BYTES + C::SLACK;
  const uint32_t full0 = bars, empty0 = bars + 8 * STAGES;
  const uint32_t g_full = bars + 16 * STAGES, g_empty = g_full + 32, done_bar = g_full + 64;
  volatile uint32_t* abort = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  const uint32_t q0 = (PAIR ? (blockIdx.x >> 1) : blockIdx.x) * TN;  // the tile's first query column
  const uint32_t qh = q0 + rank * C::HN;                              // this CTA's query columns
  const uint32_t d0 = PAIR ? blockIdx.y * (2 * TM) + rank * TM : blockIdx.y * TM;
  const uint32_t n_chunks = p.kb_total / KB_PER_CHUNK;  // a multiple of 4: K is a multiple of 256

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int g = 0; g < 4; ++g) {
      mbar_init(g_full + 8 * g, 1);
      mbar_init(g_empty + 8 * g, (PAIR ? 2 : 1) * DRAIN_THREADS / 32);
    }
    mbar_init(done_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    if constexpr (PAIR) {
      // one warp of each CTA of the pair allocates, collectively, the same columns in both
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // both CTAs' barriers exist before any remote arrive or TMA
  fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    // ------------------------------- TMA producer -------------------------------
    if (lane == 0) {
      uint32_t issued = 0;
      for (uint32_t kb = 0; kb < p.kb_total; ++kb) {
        const uint32_t s = kb % STAGES;
        if (!mbar_wait(empty0 + 8 * s, ((kb / STAGES) & 1u) ^ 1u, p.status, abort)) break;
        const uint32_t full_own = full0 + 8 * s, base = tiles + s * STAGE_BYTES;
        const bool first = kb < p.kb_half;
        const int32_t kx = static_cast<int32_t>((first ? kb : kb - p.kb_half) * KB);
        if constexpr (PAIR) {
          if (leader) mbar_expect_tx(full_own, 2 * STAGE_BYTES);  // both CTAs' halves
          const uint32_t full = peer_addr(full_own, 0);
#pragma unroll
          for (int a = 0; a < LIMBS; ++a)
            tma_load_pair(base + a * TILE_BYTES, first ? &m.a0[a] : &m.a1[a], kx, static_cast<int32_t>(d0), full);
#pragma unroll
          for (int b = 0; b < LIMBS; ++b)
            tma_load_pair(base + LIMBS * TILE_BYTES + b * C::B_TILE, &m.b[b], static_cast<int32_t>(kb * KB),
                          static_cast<int32_t>(qh), full);
        } else {
          mbar_expect_tx(full_own, STAGE_BYTES);
#pragma unroll
          for (int a = 0; a < LIMBS; ++a)
            tma_load(base + a * TILE_BYTES, first ? &m.a0[a] : &m.a1[a], kx, static_cast<int32_t>(d0), full_own);
#pragma unroll
          for (int b = 0; b < LIMBS; ++b)
            tma_load(base + LIMBS * TILE_BYTES + b * C::B_TILE, &m.b[b], static_cast<int32_t>(kb * KB),
                     static_cast<int32_t>(qh), full_own);
        }
        issued = kb + 1;
      }
      if (*abort) {
        // copies that may still be in flight land before the CTA goes on (bounded, no abort);
        // a pair's copies are counted on the leader's barriers, so its own stage-empty phases
        // stand in for them
        for (uint32_t kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
          mbar_wait((PAIR ? empty0 : full0) + 8 * (kb % STAGES), (kb / STAGES) & 1u, p.status, nullptr);
      }
    }
  } else if (warp == 1) {
    // ------------------------- MMA issuer (the leader of a pair) -------------------------
    if (leader && lane == 0) {
      bool ok = true;
      for (uint32_t kb = 0; kb < p.kb_total && ok; ++kb) {
        const uint32_t s = kb % STAGES, c = kb / KB_PER_CHUNK, j = kb % KB_PER_CHUNK;
        if (!mbar_wait(full0 + 8 * s, (kb / STAGES) & 1u, p.status, abort)) break;
        fence_after();
        const uint32_t base = tiles + s * STAGE_BYTES;
#pragma unroll
        for (int g = 3; g >= 0; --g) {
          const uint32_t per = period(g);
          if (j == 0 && c % per == 0) {
            // first k-block of a drain period of S_g: its previous period has been drained
            if (!mbar_wait(g_empty + 8 * g, (c / per) & 1u, p.status, abort)) {
              ok = false;
              break;
            }
            fence_after();
          }
          const uint32_t t = tmem + TN * static_cast<uint32_t>(g);
#pragma unroll
          for (uint32_t ks = 0; ks < KB / 16; ++ks) {
            const uint32_t o = 32u * ks;  // 16 bf16 = 32 bytes along K inside the swizzled row
#pragma unroll
            for (int a = 0; a <= g; ++a) {
              const uint64_t da = sdesc(base + a * TILE_BYTES + o);
              const uint64_t db = sdesc(base + LIMBS * TILE_BYTES + (g - a) * C::B_TILE + o);
              if constexpr (PAIR)
                umma_pair_desc(t, da, db, C::IDESC);
              else
                umma(t, da, db, C::IDESC);
            }
          }
          if (j == KB_PER_CHUNK - 1 && c % per == per - 1) {
            if constexpr (PAIR)
              umma_commit_pair(g_full + 8 * g);
            else
              umma_commit(g_full + 8 * g);
          }
        }
        if (ok) {  // stage free once these (and all earlier) MMAs are done
          if constexpr (PAIR)
            umma_commit_pair(empty0 + 8 * s);
          else
            umma_commit(empty0 + 8 * s);
        }
      }
      // every MMA issued above completes before the tensor memory is freed
      if constexpr (PAIR)
        umma_commit_pair(done_bar);
      else
        umma_commit(done_bar);
      mbar_wait(done_bar, 0, p.status, nullptr);
    }
  } else {
    // ----------------------------------- drain ----------------------------------
    const uint32_t q = static_cast<uint32_t>(warp) & 3u, h = static_cast<uint32_t>(warp - 2) >> 2;
    const uint32_t tl = tmem + ((32u * q) << 16) + 64u * h;
    auto release = [&](int g) {
      if constexpr (PAIR)
        arrive_leader(g_empty + 8 * g, leader);
      else
        mbar_arrive(g_empty + 8 * g);
    };
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      tmem_fill32(tl + TN * g, MAGIC);
      tmem_fill32(tl + TN * g + 32, MAGIC);
    }
    tmem_wait_st();
    fence_before();
    __syncwarp();
    if (lane == 0)
      for (int g = 0; g < 4; ++g) release(g);
    // each S_1 drain adds bits(M) << 8 and each S_0 drain bits(M) once too often
    const uint32_t corr = 0u - (n_chunks / period(1)) * (MAGIC << 8) - (n_chunks / period(0)) * MAGIC;
    uint32_t acc[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) acc[k] = corr;
    bool ok = true;
    for (uint32_t c = 0; c < n_chunks && ok; ++c) {
#pragma unroll
      for (int g = 3; g >= 0; --g) {
        const uint32_t per = period(g);
        if (c % per != per - 1) continue;
        if (!__all_sync(0xFFFFFFFFu, mbar_wait(g_full + 8 * g, (c / per) & 1u, p.status, abort))) {
          ok = false;
          break;
        }
        fence_after();
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t r[32];
          tmem_ld32(tl + TN * g + 32 * hh, r);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 32; ++k) acc[32 * hh + k] += r[k] << (8 * g);
          tmem_fill32(tl + TN * g + 32 * hh, MAGIC);
        }
        tmem_wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) release(g);
      }
    }
    // ---- epilogue: z + r_i, r_i = F(seed_own) - F(seed_prev) over Z_{2^32} (App. C) ----
    // The sums go to shared memory (the stage ring is idle: the last S_0-full followed every
    // MMA), then each (column, 4-row group) item adds the zero shares of its four rows, one
    // Philox block per seed, and writes 16 bytes of z.
    named_sync(1, DRAIN_THREADS);
    if (!*abort) {  // uniform: read after the barrier that every drainer reaches
      uint32_t* zs = reinterpret_cast<uint32_t*>(smem);  // [TN][TM]
      const uint32_t row = 32 * q + lane;
#pragma unroll
      for (int k = 0; k < 64; ++k) zs[(64 * h + k) * TM + row] = acc[k];
      named_sync(1, DRAIN_THREADS);
      const uint32_t dt = threadIdx.x - 64;
      const uint32_t grp0 = static_cast<uint32_t>((p.row0 + d0) >> 2);
      const uint32_t ctr3 = (IPC_D_ZA32 << 24) | p.vec;
      for (uint32_t it = dt; it < TN * (TM / 4); it += DRAIN_THREADS) {
        const uint32_t cc = it / (TM / 4), g4 = it % (TM / 4), col = q0 + cc, r0 = d0 + 4 * g4;
        if (col >= p.n_cols || r0 >= p.x_rows) continue;
        const uint32_t req = p.col_tags[2 * col], tag = p.col_tags[2 * col + 1];
        const uint4 fo = philox(grp0 + g4, tag, req, ctr3, p.seed_own);
        const uint4 fp = philox(grp0 + g4, tag, req, ctr3, p.seed_prev);
        const uint4 a = *reinterpret_cast<const uint4*>(zs + cc * TM + 4 * g4);
        const uint4 v = make_uint4(a.x + fo.x - fp.x, a.y + fo.y - fp.y, a.z + fo.z - fp.z, a.w + fo.w - fp.w);
        uint32_t* dst = p.z + static_cast<uint64_t>(col) * p.ldz + r0;
        if (r0 + 4 <= p.x_rows) {
          *reinterpret_cast<uint4*>(dst) = v;
        } else {
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
          for (uint32_t e = 0; e < p.x_rows - r0; ++e) dst[e] = w[e];
        }
      }
    }
  }
  // a pair's MMAs are complete (the leader's issuer waited for them) before either CTA frees
  // tensor memory or leaves
  fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();
  if (warp == 0) {
    fence_after();
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <bool PAIR>
int launch_tc32(const Maps32& m, const Tc32Params& p, uint32_t n_cols, size_t x_rows, cudaStream_t stream) {
  using C = Cfg32<PAIR>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(gemm_tc32_kernel<PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
  });
  IPC_CUDA_TRY(attr);
  const uint32_t rows_per = PAIR ? 2 * TM : TM;
  const dim3 grid((PAIR ? 2 : 1) * ((n_cols + TN - 1) / TN), static_cast<unsigned>((x_rows + rows_per - 1) / rows_per));
  if constexpr (PAIR) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = C::SMEM_BYTES;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    IPC_CUDA_TRY(cudaLaunchKernelEx(&cfg, gemm_tc32_kernel<true>, m, p));
  } else {
    gemm_tc32_kernel<false><<<grid, THREADS, C::SMEM_BYTES, stream>>>(m, p);
  }
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

}  // namespace

// segments: 2 for K = 2l over [x[0..3] | x[4..7]] (ABY3 replicated sharing, x[4..7] the
// previous party's component), 1 for K = l over x[0..3] alone. K must be a multiple of 256.
// pair: CTA pairs (256-row tiles) instead of one CTA per 128-row tile; the same z bit for bit.
int ring_gemm_tc32(uint32_t segments, const uint16_t* const x[8], size_t x_rows, const uint16_t* const b[4],
                   uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                   uint64_t seed_prev, uint32_t vec, uint32_t* z, size_t ldz, uint64_t row0, cudaStream_t stream,
                   bool pair) {
  if (segments != 1 && segments != 2) {
    set_error("Z_2^32 ring GEMM: one or two K segments");
    return IPC_EINVAL;
  }
  if ((segments * l) % (4 * KB_PER_CHUNK * KB) != 0) {
    set_error("Z_2^32 ring GEMM: K must be a multiple of 256");
    return IPC_EINVAL;
  }
  if (n_pad % TN != 0 || n_cols > n_pad || ldz % 4 != 0 || ldz < x_rows || !aligned16(z)) {
    set_error("Z_2^32 ring GEMM: n_pad % 128, n_cols <= n_pad, ldz % 4, ldz >= x_rows and a 16-byte aligned z");
    return IPC_EINVAL;
  }
  if (x_rows == 0 || n_cols == 0) return IPC_OK;
  if (x_rows > 65535ull * TM) {
    set_error("Z_2^32 ring GEMM: too many rows for one launch");
    return IPC_EINVAL;
  }
  const uint32_t hn = pair ? TN / 2 : TN;
  Maps32 m;
  int rc;
  for (int i = 0; i < LIMBS; ++i) {
    if ((rc = make_map_bf16(&m.b[i], b[i], static_cast<uint64_t>(segments) * l, n_pad, hn)) ||
        (rc = make_map_bf16(&m.a0[i], x[i], l, x_rows, TM)) ||
        (rc = make_map_bf16(&m.a1[i], x[segments == 2 ? LIMBS + i : i], l, x_rows, TM)))
      return rc;
  }
  Tc32Params p;
  p.n_cols = n_cols;
  p.x_rows = static_cast<uint32_t>(x_rows);
  p.kb_total = segments * l / KB;
  p.kb_half = l / KB;
  p.col_tags = col_tags;
  p.seed_own = seed_own;
  p.seed_prev = seed_prev;
  p.vec = vec;
  p.z = z;
  p.ldz = ldz;
  p.row0 = row0;
  p.status = status_ptr();
  return pair ? launch_tc32<true>(m, p, n_cols, x_rows, stream) : launch_tc32<false>(m, p, n_cols, x_rows, stream);
}

int prep_query32(const uint32_t* y, uint64_t y_plane, uint32_t Q, const ipc_geom* g, uint32_t party,
                 uint32_t segments, uint16_t* const b[4], uint32_t n_pad, cudaStream_t stream) {
  const uint64_t l = g ? static_cast<uint64_t>(g->rows) * g->cols * g->cell : 0;
  if (!g || l == 0 || g->R == 0 || g->R > 31 || party > 2 || (segments != 1 && segments != 2) || !y || !b || !b[0] ||
      !b[1] || !b[2] || !b[3] || Q == 0 || static_cast<uint64_t>(Q) * g->R > n_pad) {
    set_error("Z_2^32 query operand: bad geometry, party, segments, pointers or n_pad < Q*R");
    return IPC_EINVAL;
  }
  const uint64_t total = static_cast<uint64_t>(n_pad) * segments * l;
  const uint32_t bs = 256;
  prep_query32_kernel<<<static_cast<unsigned>((total + bs - 1) / bs), bs, 0, stream>>>(
      y, y_plane, Q, *g, party, segments, b[0], b[1], b[2], b[3], n_pad);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

}  // namespace ipc

using namespace ipc;

extern "C" int ipc_encode_share32(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                                  uint64_t client_seed, uint32_t side, uint32_t idx0, uint32_t* code_sh,
                                  uint32_t* mask_sh, void* stream) {
  if (l == 0 || l % 2 != 0 || !code_bits || !mask_bits || !code_sh || !mask_sh) {
    set_error("ipc_encode_share32: l must be a positive even number and pointers non-null");
    return IPC_EINVAL;
  }
  if (n == 0) return IPC_OK;
  const uint64_t total = static_cast<uint64_t>(n) * (l / 2);
  const uint32_t bs = 256;
  encode_share32_kernel<<<static_cast<unsigned>((total + bs - 1) / bs), bs, 0, static_cast<cudaStream_t>(stream)>>>(
      code_bits, mask_bits, n, l, client_seed, side, idx0, code_sh, mask_sh);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

extern "C" int ipc_split_limbs32_bf16(const uint32_t* x, size_t count, uint16_t* const limbs[4], void* stream) {
  if (!x || !limbs || !limbs[0] || !limbs[1] || !limbs[2] || !limbs[3]) {
    set_error("ipc_split_limbs32_bf16: null pointer");
    return IPC_EINVAL;
  }
  if (!aligned16(x)) {
    set_error("ipc_split_limbs32_bf16: x must be 16-byte aligned");
    return IPC_EINVAL;
  }
  for (int i = 0; i < 4; ++i)
    if (reinterpret_cast<uintptr_t>(limbs[i]) & 7u) {
      set_error("ipc_split_limbs32_bf16: limb planes must be 8-byte aligned");
      return IPC_EINVAL;
    }
  if (count == 0) return IPC_OK;
  const size_t threads = (count + 3) / 4;
  const uint32_t bs = 256;
  split_limbs32_kernel<<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, static_cast<cudaStream_t>(stream)>>>(
      x, count, limbs[0], limbs[1], limbs[2], limbs[3]);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

extern "C" int ipc_prep_query32_bf16(const uint32_t* y, uint32_t Q, const ipc_geom* g, uint32_t party,
                                     uint32_t segments, uint16_t* const b[4], uint32_t n_pad, void* stream) {
  const uint64_t l = g ? static_cast<uint64_t>(g->rows) * g->cols * g->cell : 0;
  return prep_query32(y, Q * l, Q, g, party, segments, b, n_pad, static_cast<cudaStream_t>(stream));
}

extern "C" int ipc_ring_gemm_tc32(uint32_t segments, const uint16_t* const x[8], size_t x_rows,
                                  const uint16_t* const b[4], uint32_t n_cols, uint32_t n_pad, uint32_t l,
                                  const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec,
                                  uint32_t* z, size_t ldz, uint64_t row0, uint32_t pair, void* stream) {
  if (!x || !b || !col_tags || !z) {
    set_error("ipc_ring_gemm_tc32: null pointer");
    return IPC_EINVAL;
  }
  for (int i = 0; i < 4; ++i)
    if (!x[i] || !b[i] || (segments == 2 && !x[4 + i]) || !aligned16(x[i]) || !aligned16(b[i]) ||
        (segments == 2 && !aligned16(x[4 + i]))) {
      set_error("ipc_ring_gemm_tc32: limb planes must be non-null and 16-byte aligned");
      return IPC_EINVAL;
    }
  if (x_rows > IPC_MAX_GEMM_ROWS) {
    set_error("ipc_ring_gemm_tc32: x_rows above IPC_MAX_GEMM_ROWS");
    return IPC_EINVAL;
  }
  return ring_gemm_tc32(segments, x, x_rows, b, n_cols, n_pad, l, col_tags, seed_own, seed_prev, vec, z, ldz, row0,
                        static_cast<cudaStream_t>(stream), pair != 0);
}
