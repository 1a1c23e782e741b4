// A0-A3 over Z_{2^32} for the lifting variants (Sec. 5.1, Sec. 6.2): ConstLift computes ml,
// NoLift also the code dot product, over Z_{2^32}.
//
// A0: client sharing of the masked bits and mask bits read in Z_{2^32}.
// A1: four balanced int8 limbs per element, x = x0 + 2^8 x1 + 2^16 x2 + 2^24 x3 (mod 2^32), in
//     four resident int8 planes (the size of the u32 shares).
// A2: the query operand's four limbs as fp16 bit patterns (exact).
// A3 (gemm_tc32_kernel): the ring dot product on tcgen05 with fp32 TMEM accumulators, exact:
//     z = sum_s 2^(8s) S_s (mod 2^32),  S_s = sum over a + b = s of sum_k x_a[k] y_b[k],
//   ten limb products per k (1 + 2 + 3 + 4 for s = 0..3); products with a + b > 3 vanish mod
//   2^32. Each S_s is accumulated in a TMEM accumulator started at M = 1.5 * 2^23 and drained
//   while every partial sum stays within M +- 2^22 (so every fp32 addition is exact, as in the
//   16-bit kernel): S_s gains at most (s + 1) 2^14 per k, so S_3 and S_2 are drained every 64 k,
//   S_1 every 128 k, S_0 every 256 k. Two passes per tile (S_3 and S_2, then S_1 and S_0) share
//   the 512 TMEM columns; a drain adds the raw bits, shifted by 8s, to running sums: mod 2^16
//   for (S_2 + 2^8 S_3), whose bits(M) terms vanish, and mod 2^32 for S_0 + 2^8 S_1, whose
//   bits(M) terms are subtracted once, up front. The database limbs are widened from int8 to
//   fp16 in shared memory, as in the 16-bit kernel. Every wait is bounded (2 s, or sooner once
//   another role has failed); a failed CTA raises the status word, lets its copies and MMAs
//   finish and frees its tensor memory.
#include <cuda_fp16.h>

#include <mutex>
#include <string>
#include <type_traits>

#include "tcgen05.cuh"

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

__device__ __forceinline__ uint16_t f16_of8(int8_t v) { return __half_as_ushort(__short2half_rn(v)); }

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

// A1 over Z_{2^32}: 4 elements per thread, one int8 limb plane per limb.
__global__ void split_limbs32_kernel(const uint32_t* __restrict__ x, size_t count, int8_t* __restrict__ o0,
                                     int8_t* __restrict__ o1, int8_t* __restrict__ o2, int8_t* __restrict__ o3) {
  const size_t i4 = (blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x) * 4;
  if (i4 >= count) return;
  int8_t* out[4] = {o0, o1, o2, o3};
  if (i4 + 4 <= count) {
    const uint4 v = *reinterpret_cast<const uint4*>(x + i4);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t packed[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int8_t lb[4];
      limbs32(w[e], lb);
#pragma unroll
      for (int i = 0; i < 4; ++i) packed[i] |= static_cast<uint32_t>(static_cast<uint8_t>(lb[i])) << (8 * e);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) *reinterpret_cast<uint32_t*>(out[i] + i4) = packed[i];
  } else {
    for (size_t e = i4; e < count; ++e) {
      int8_t lb[4];
      limbs32(x[e], lb);
      for (int i = 0; i < 4; ++i) out[i][e] = lb[i];
    }
  }
}

// A2 over Z_{2^32}: party i's operand [rot(Y_i + Y_{i-1}) | rot(Y_i)] (K = 2l), or, for one
// segment, rot(Y_i) alone (K = l); four fp16 limb planes. Eight consecutive k of one row n per
// thread (l a multiple of 8, so a group stays in one half), one 16-byte store per plane.
__global__ void prep_query32_kernel(const uint32_t* __restrict__ y, uint64_t plane, uint32_t Q, ipc_geom g,
                                    uint32_t party, uint32_t segments, uint16_t* __restrict__ o0,
                                    uint16_t* __restrict__ o1, uint16_t* __restrict__ o2, uint16_t* __restrict__ o3,
                                    uint32_t n_pad) {
  const uint32_t l = g.rows * g.cols * g.cell, K = segments * l, groups = K / 8;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (tid >= static_cast<uint64_t>(n_pad) * groups) return;
  const uint32_t n = static_cast<uint32_t>(tid / groups);
  const uint32_t k0 = static_cast<uint32_t>(tid % groups) * 8;
  uint32_t val[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  if (n < Q * g.R) {
    const uint32_t q = n / g.R, rho = n % g.R;
    const int32_t shift = g.rot_lo + static_cast<int32_t>(rho);
    const bool sum = segments == 2 && k0 < l;  // first half of K = 2l: y_i + y_{i-1}
    const uint32_t kk = k0 < l ? k0 : k0 - l;
    uint32_t c = kk % g.cell;
    const uint32_t cidx = kk / g.cell;
    uint32_t j = cidx % g.cols, r = cidx / g.cols;
    int32_t jsi = (static_cast<int32_t>(j) - shift) % static_cast<int32_t>(g.cols);
    uint32_t js = static_cast<uint32_t>(jsi < 0 ? jsi + static_cast<int32_t>(g.cols) : jsi);
    const uint32_t prev = (party + 2) % 3;
    const uint32_t* yi = y + party * plane + static_cast<uint64_t>(q) * l;
    const uint32_t* yp = y + prev * plane + static_cast<uint64_t>(q) * l;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint32_t src = (r * g.cols + js) * g.cell + c;
      val[e] = sum ? yi[src] + yp[src] : yi[src];
      if (++c == g.cell) {
        c = 0;
        if (++js == g.cols) js = 0;
        if (++j == g.cols) {
          j = 0;
          ++r;
        }
      }
    }
  }
  uint32_t w[4][4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    int8_t a[4], b[4];
    limbs32(val[2 * v], a);
    limbs32(val[2 * v + 1], b);
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i][v] = f16_of8(a[i]) | (static_cast<uint32_t>(f16_of8(b[i])) << 16);
  }
  uint16_t* out[4] = {o0, o1, o2, o3};
#pragma unroll
  for (int i = 0; i < 4; ++i) *reinterpret_cast<uint4*>(out[i] + tid * 8) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}

// ----------------------------------- A3 -----------------------------------
// One CTA per tile of 128 database rows x 256 query columns (MMA 128 x 256 x 16). Four 256-column
// accumulators would need 1,024 TMEM columns (an SM has 512), so the tile runs in two passes of
// two accumulators each, over the same rings:
//   pass A (stages 0 .. KBT-1, one k-block each): S_3 and S_2, seven limb products over limbs
//     0-3. Only U = (S_2 + 2^8 S_3) mod 2^16 matters (it enters z shifted by 16), so its running
//     sums are kept mod 2^16, two columns to a register; at the end of the pass they go to z as
//     U << 16 (global memory, read back by the epilogue).
//   pass B (stages KBT .. KBT + KBT/2 - 1, two k-blocks each): S_1 and S_0, three limb products
//     over limbs 0-1, whose sums are kept mod 2^32.
// A stage holds four tiles of each operand: limbs 0-3 of one k-block (pass A) or limbs 0-1 of
// two k-blocks (pass B), so the rings run on from one pass into the other.
constexpr int TM = 128, TN = 256, KB = 32, SLOTS = 4;
constexpr int W_TILE = TM * KB * 2;  // 8 KiB widened (fp16) database tile
constexpr int RAW_TILE = TM * KB;    // 4 KiB raw (int8) database tile
constexpr int B_TILE = TN * KB * 2;  // 16 KiB query tile
constexpr int QS = 2, WS = 2, RS = 2;  // stages of the query, widened and raw rings
constexpr int Q_STAGE = SLOTS * B_TILE;    // 64 KiB
constexpr int W_STAGE = SLOTS * W_TILE;    // 32 KiB
constexpr int R_STAGE = SLOTS * RAW_TILE;  // 16 KiB
constexpr int W_OFF = QS * Q_STAGE, R_OFF = W_OFF + WS * W_STAGE, BAR_OFF = R_OFF + RS * R_STAGE;
constexpr int THREADS = 12 * 32, DRAIN_THREADS = 8 * 32;
constexpr int WIDEN_WARP0 = 2, WIDEN_THREADS = 2 * 32, DRAIN_WARP0 = 4;
constexpr uint32_t TMEM_COLS = 2 * TN;  // region 0 (S_2, then S_0) and region 1 (S_3, then S_1)
constexpr uint32_t MAGIC = 0x4B400000u;  // fp32 bits of 1.5 * 2^23
// q_full[QS], q_empty[QS], w_full[WS], w_empty[WS], r_full[RS], r_empty[RS], a_full[2],
// a_empty[2], done
constexpr int NUM_BARS = 2 * QS + 2 * WS + 2 * RS + 5;
constexpr int SMEM_BYTES = BAR_OFF + 1024 + 8 * NUM_BARS;
static_assert(SMEM_BYTES <= 232448, "dynamic shared memory per block");
static_assert(TN * TM * 4 <= QS * Q_STAGE, "the z tile is staged in the Q ring");
// kind::f16: D f32, A and B f16, both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (static_cast<uint32_t>(TN >> 3) << 17) | (static_cast<uint32_t>(TM >> 4) << 24);

// Drain periods, in stages: pass A drains both regions every 2 stages (64 k: S_3 gains at most
// 4 * 2^14 per k); pass B drains S_1 every 2 stages (128 k) and S_0 every 4 (256 k).
// Operand tile t of stage G: its limb and k-block.
__device__ __forceinline__ void stage_slot(uint32_t G, uint32_t kbt, uint32_t t, uint32_t& limb, uint32_t& kb) {
  if (G < kbt) {
    limb = t;
    kb = G;
  } else {
    limb = t & 1u;
    kb = 2u * (G - kbt) + (t >> 1);
  }
}

struct Maps32 {
  CUtensorMap b[4];   // query limbs [n_pad][K], fp16
  CUtensorMap a0[4];  // database limbs of the first K segment [x_rows][l], int8
  CUtensorMap a1[4];  // and of the second
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

// Roles (12 warps), with three rings as in the 16-bit kernel (query, raw database, widened
// database), so that the widening runs ahead of the MMAs:
//   warp 0 lane 0  query producer: per stage, four fp16 query tiles (256 x 32, 64-byte swizzle).
//   warps 2-3      raw copies and widening: a stage's four raw int8 database tiles (copied RS
//                  stages ahead) become fp16 operand tiles in the W ring.
//   warp 1 lane 0  MMA issuer: per stage, region 1's products (S_3, or S_1), then region 0's
//                  (S_2, or S_0), committing a region's full barrier after the last stage of its
//                  drain period, then the stage's Q and W slots. Region 1 drains while region
//                  0's products of the same stage run.
//   warps 4-11     drain: each thread owns one TMEM lane (database row) and 128 columns.
// Every wait is bounded (2 s, or sooner once another role has failed); a failed CTA raises the
// status word, lets its copies and MMAs finish and frees its tensor memory (its z tile is then
// undefined).
__global__ void __launch_bounds__(THREADS, 1) gemm_tc32_kernel(const __grid_constant__ Maps32 m, const Tc32Params p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ uint32_t s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t qring = smem_addr(smem), wring = qring + W_OFF, rring = qring + R_OFF, bars = qring + BAR_OFF;
  const uint32_t q_full = bars, q_empty = q_full + 8 * QS, w_full = q_empty + 8 * QS, w_empty = w_full + 8 * WS,
                 r_full = w_empty + 8 * WS, r_empty = r_full + 8 * RS;
  const uint32_t a_full = r_empty + 8 * RS, a_empty = a_full + 16, done_bar = a_full + 32;
  volatile uint32_t* abort = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t q0 = blockIdx.x * TN, d0 = blockIdx.y * TM;
  const uint32_t kbt = p.kb_total;           // a multiple of 8: K is a multiple of 256
  const uint32_t n_stages = kbt + kbt / 2;   // pass A, then pass B

  if (threadIdx.x == 0) {
    for (int s = 0; s < QS; ++s) {
      mbar_init(q_full + 8 * s, 1);
      mbar_init(q_empty + 8 * s, 1);
    }
    for (int s = 0; s < WS; ++s) {
      mbar_init(w_full + 8 * s, WIDEN_THREADS / 32);
      mbar_init(w_empty + 8 * s, 1);
    }
    for (int s = 0; s < RS; ++s) {
      mbar_init(r_full + 8 * s, 1);
      mbar_init(r_empty + 8 * s, WIDEN_THREADS / 32);
    }
    for (int g = 0; g < 2; ++g) {
      mbar_init(a_full + 8 * g, 1);
      mbar_init(a_empty + 8 * g, DRAIN_THREADS / 32);
    }
    mbar_init(done_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    // ---------------------------- query TMA producer -----------------------------
    if (lane == 0) {
      uint32_t issued = 0;
      for (uint32_t G = 0; G < n_stages; ++G) {
        const uint32_t s = G % QS;
        if (!mbar_wait(q_empty + 8 * s, ((G / QS) & 1u) ^ 1u, p.status, abort)) break;
        const uint32_t full = q_full + 8 * s, base = qring + s * Q_STAGE;
        mbar_expect_tx(full, Q_STAGE);
#pragma unroll
        for (uint32_t t = 0; t < SLOTS; ++t) {
          uint32_t limb, kb;
          stage_slot(G, kbt, t, limb, kb);
          tma_load(base + t * B_TILE, &m.b[limb], static_cast<int32_t>(kb * KB), static_cast<int32_t>(q0), full);
        }
        issued = G + 1;
      }
      if (*abort) {
        // copies that may still be in flight land before the CTA goes on (bounded, no abort)
        for (uint32_t G = issued > QS ? issued - QS : 0; G < issued; ++G)
          mbar_wait(q_full + 8 * (G % QS), (G / QS) & 1u, p.status, nullptr);
      }
    }
  } else if (warp == 1) {
    // -------------------------------- MMA issuer --------------------------------
    if (lane == 0) {
      const uint32_t t0 = tmem, t1 = tmem + TN;
      uint32_t started0 = 0, started1 = 0;  // drain periods started per region
      bool ok = true;
      for (uint32_t G = 0; G < n_stages && ok; ++G) {
        const uint32_t s = G % QS;  // QS == WS
        if (!mbar_wait(q_full + 8 * s, (G / QS) & 1u, p.status, abort) ||
            !mbar_wait(w_full + 8 * s, (G / WS) & 1u, p.status, abort))
          break;
        fence_after();
        const bool pass_a = G < kbt;
        const uint32_t j = pass_a ? G : G - kbt;
        const bool open1 = (j & 1u) == 0, close1 = (j & 1u) == 1;
        const bool open0 = pass_a ? (j & 1u) == 0 : (j & 3u) == 0;
        const bool close0 = pass_a ? (j & 1u) == 1 : (j & 3u) == 3;
        const uint32_t qb = qring + s * Q_STAGE, wb = wring + s * W_STAGE;
        if (open1) {
          if (!mbar_wait(a_empty + 8, started1 & 1u, p.status, abort)) break;
          ++started1;
          fence_after();
        }
        if (pass_a) {
#pragma unroll
          for (uint32_t ks = 0; ks < KB / 16; ++ks) {
            const uint32_t o = 32u * ks;  // 16 fp16 = 32 bytes along K inside the swizzled row
#pragma unroll
            for (uint32_t a = 0; a < 4; ++a)  // S_3: x_a y_(3-a)
              umma(t1, sdesc(wb + a * W_TILE + o), sdesc(qb + (3 - a) * B_TILE + o), IDESC);
          }
        } else {
#pragma unroll
          for (uint32_t sub = 0; sub < 2; ++sub)
#pragma unroll
            for (uint32_t ks = 0; ks < KB / 16; ++ks) {
              const uint32_t o = 32u * ks, w = wb + 2 * sub * W_TILE + o, q = qb + 2 * sub * B_TILE + o;
              umma(t1, sdesc(w), sdesc(q + B_TILE), IDESC);  // S_1: x_0 y_1
              umma(t1, sdesc(w + W_TILE), sdesc(q), IDESC);  //      x_1 y_0
            }
        }
        if (close1) umma_commit(a_full + 8);
        if (open0) {
          if (!mbar_wait(a_empty, started0 & 1u, p.status, abort)) {
            ok = false;
            break;
          }
          ++started0;
          fence_after();
        }
        if (pass_a) {
#pragma unroll
          for (uint32_t ks = 0; ks < KB / 16; ++ks) {
            const uint32_t o = 32u * ks;
#pragma unroll
            for (uint32_t a = 0; a < 3; ++a)  // S_2: x_a y_(2-a)
              umma(t0, sdesc(wb + a * W_TILE + o), sdesc(qb + (2 - a) * B_TILE + o), IDESC);
          }
        } else {
#pragma unroll
          for (uint32_t sub = 0; sub < 2; ++sub)
#pragma unroll
            for (uint32_t ks = 0; ks < KB / 16; ++ks) {
              const uint32_t o = 32u * ks;  // S_0: x_0 y_0
              umma(t0, sdesc(wb + 2 * sub * W_TILE + o), sdesc(qb + 2 * sub * B_TILE + o), IDESC);
            }
        }
        if (close0) umma_commit(a_full);
        // both slots free once these (and all earlier) MMAs are done
        umma_commit(q_empty + 8 * s);
        umma_commit(w_empty + 8 * s);
      }
      // every MMA issued above completes before the tensor memory is freed
      umma_commit(done_bar);
      mbar_wait(done_bar, 0, p.status, nullptr);
    }
  } else if (warp < DRAIN_WARP0) {
    // ------------------------- raw copies and widening ---------------------------
    const uint32_t ct = threadIdx.x - WIDEN_WARP0 * 32;
    uint32_t issued = 0;
    auto load_raw = [&](uint32_t G) {
      const uint32_t s = G % RS, full = r_full + 8 * s, base = rring + s * R_STAGE;
      mbar_expect_tx(full, R_STAGE);
#pragma unroll
      for (uint32_t t = 0; t < SLOTS; ++t) {
        uint32_t limb, kb;
        stage_slot(G, kbt, t, limb, kb);
        const bool first = kb < p.kb_half;
        const int32_t kx = static_cast<int32_t>((first ? kb : kb - p.kb_half) * KB);
        tma_load(base + t * RAW_TILE, first ? &m.a0[limb] : &m.a1[limb], kx, static_cast<int32_t>(d0), full);
      }
      issued = G + 1;
    };
    if (ct == 0)
      for (uint32_t G = 0; G < n_stages && G < RS; ++G) load_raw(G);
    uint32_t G = 0;
    for (; G < n_stages; ++G) {
      const uint32_t rs = G % RS, ws = G % WS;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(r_full + 8 * rs, (G / RS) & 1u, p.status, abort) &&
                                       mbar_wait(w_empty + 8 * ws, ((G / WS) & 1u) ^ 1u, p.status, abort)))
        break;
      widen_tiles<SLOTS, WIDEN_THREADS>(rring + rs * R_STAGE, RAW_TILE, wring + ws * W_STAGE, W_TILE, ct);
      fence_proxy_async();  // the MMAs read these tiles through the async proxy
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(w_full + 8 * ws);
        mbar_arrive(r_empty + 8 * rs);  // this warp has read raw stage rs
      }
      if (warp == WIDEN_WARP0 && G + RS < n_stages) {
        // refill once both warps have read the stage (a bounded wait, warp-uniform like the others)
        if (!__all_sync(0xFFFFFFFFu, mbar_wait(r_empty + 8 * rs, (G / RS) & 1u, p.status, abort))) break;
        if (lane == 0) load_raw(G + RS);
      }
    }
    if (ct == 0 && *abort) {
      // raw copies that may still be in flight land before the CTA leaves (bounded, no abort)
      for (uint32_t h = G; h < issued; ++h) mbar_wait(r_full + 8 * (h % RS), (h / RS) & 1u, p.status, nullptr);
    }
  } else {
    // ----------------------------------- drain ----------------------------------
    const uint32_t q = static_cast<uint32_t>(warp) & 3u, h = static_cast<uint32_t>(warp - DRAIN_WARP0) >> 2;
    const uint32_t tl = tmem + ((32u * q) << 16) + 128u * h;  // region 0; region 1 at + TN
    const uint32_t row = d0 + 32 * q + lane;
#pragma unroll
    for (uint32_t g = 0; g < 4; ++g) {
      tmem_fill32(tl + 32 * g, MAGIC);
      tmem_fill32(tl + TN + 32 * g, MAGIC);
    }
    tmem_wait_st();
    fence_before();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(a_empty);
      mbar_arrive(a_empty + 8);
    }
    uint32_t done0 = 0, done1 = 0;  // drains per region
    // one drain of a region: wait for its full barrier, hand each 32-column group's fp32 bit
    // patterns to f, re-base the accumulator, release the region
    // (W columns a load: 32 in pass A, two loads before each wait; 16 in pass B, one load a wait,
    // whose 32-bit sums take 128 registers)
    auto drain = [&](uint32_t region, uint32_t& done, auto&& f, auto width) -> bool {
      constexpr uint32_t W = decltype(width)::value;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(a_full + 8 * region, done & 1u, p.status, abort))) return false;
      ++done;
      fence_after();
      auto ld_ = [&](uint32_t g, uint32_t (&r)[W]) {
        if constexpr (W == 32) {
          tmem_ld32(tl + TN * region + W * g, r);
        } else {
          tmem_ld16(tl + TN * region + W * g, r);
        }
      };
      auto fill_ = [&](uint32_t g) {
        if constexpr (W == 32) {
          tmem_fill32(tl + TN * region + W * g, MAGIC);
        } else {
          tmem_fill16(tl + TN * region + W * g, MAGIC);
        }
      };
      if constexpr (W == 32) {
        // two loads in flight before each wait (pass A: 64 packed sums leave room for them)
#pragma unroll
        for (uint32_t g = 0; g < 128 / W; g += 2) {
          uint32_t r[W], r2[W];
          ld_(g, r);
          ld_(g + 1, r2);
          tmem_wait_ld();
          f(g, r);
          f(g + 1, r2);
          fill_(g);
          fill_(g + 1);
        }
      } else {
#pragma unroll
        for (uint32_t g = 0; g < 128 / W; ++g) {
          uint32_t r[W];
          ld_(g, r);
          tmem_wait_ld();
          f(g, r);
          fill_(g);
        }
      }
      tmem_wait_st();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(a_empty + 8 * region);
      return true;
    };
    bool ok = true;
    {
      // pass A: u[k] holds U mod 2^16 of columns 2k (low half) and 2k + 1 (high half); bits(M)
      // is 0 mod 2^16, so the raw bits of a drained S_2 add as they are, S_3's shifted by 8
      uint32_t u[64];
#pragma unroll
      for (int k = 0; k < 64; ++k) u[k] = 0;
      for (uint32_t d = 0; d < kbt / 2 && ok; ++d) {
        ok = drain(
            1, done1,
            [&](uint32_t g, const uint32_t (&r)[32]) {
#pragma unroll
              for (int k = 0; k < 16; ++k) u[16 * g + k] = add16x2(u[16 * g + k], pack_c16(r[2 * k], r[2 * k + 1]));
            },
            std::integral_constant<uint32_t, 32>{});
        if (ok)
          ok = drain(
              0, done0,
              [&](uint32_t g, const uint32_t (&r)[32]) {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                  u[16 * g + k] = add16x2(u[16 * g + k], pack_lo16(r[2 * k], r[2 * k + 1]));
              },
              std::integral_constant<uint32_t, 32>{});
      }
      // U << 16 goes to z, where the epilogue adds pass B's sums and the zero shares to it
      if (ok && row < p.x_rows) {
#pragma unroll
        for (int k = 0; k < 64; ++k) {
          const uint32_t c = q0 + 128 * h + 2 * k;
          if (c < p.n_cols) p.z[static_cast<uint64_t>(c) * p.ldz + row] = u[k] << 16;
          if (c + 1 < p.n_cols) p.z[static_cast<uint64_t>(c + 1) * p.ldz + row] = u[k] & 0xFFFF0000u;
        }
      }
    }
    // pass B: 32-bit sums; each S_1 drain adds bits(M) << 8 and each S_0 drain bits(M) once too
    // often, subtracted up front
    const uint32_t corr = 0u - (kbt / 4) * (MAGIC << 8) - (kbt / 8) * MAGIC;
    uint32_t acc[128];
#pragma unroll
    for (int k = 0; k < 128; ++k) acc[k] = corr;
    for (uint32_t j = 0; j < kbt / 2 && ok; ++j) {
      if ((j & 1u) == 1)
        ok = drain(
            1, done1,
            [&](uint32_t g, const uint32_t (&r)[16]) {
#pragma unroll
              for (int k = 0; k < 16; ++k) acc[16 * g + k] += r[k] << 8;
            },
            std::integral_constant<uint32_t, 16>{});
      if (ok && (j & 3u) == 3)
        ok = drain(
            0, done0,
            [&](uint32_t g, const uint32_t (&r)[16]) {
#pragma unroll
              for (int k = 0; k < 16; ++k) acc[16 * g + k] += r[k];
            },
            std::integral_constant<uint32_t, 16>{});
    }
    // ---- epilogue: z = U << 16 + pass B + r_i, r_i = F(seed_own) - F(seed_prev) (App. C) ----
    // The sums go to shared memory (the Q ring is idle: the last S_0-full followed every MMA,
    // and every copy was consumed), then each (column, 4-row group) item adds U << 16 (from z)
    // and the zero shares of its four rows, one Philox block per seed, and writes 16 bytes of z.
    named_sync(1, DRAIN_THREADS);
    if (!*abort) {  // uniform: read after the barrier that every drainer reaches
      uint32_t* zs = reinterpret_cast<uint32_t*>(smem);  // [TN][TM]
      const uint32_t trow = 32 * q + lane;
#pragma unroll
      for (int k = 0; k < 128; ++k) zs[(128 * h + k) * TM + trow] = acc[k];
      named_sync(1, DRAIN_THREADS);
      const uint32_t dt = threadIdx.x - DRAIN_WARP0 * 32;
      const uint32_t grp0 = static_cast<uint32_t>((p.row0 + d0) >> 2);
      const uint32_t ctr3 = (IPC_D_ZA32 << 24) | p.vec;
      for (uint32_t it = dt; it < TN * (TM / 4); it += DRAIN_THREADS) {
        const uint32_t cc = it / (TM / 4), g4 = it % (TM / 4), col = q0 + cc, r0 = d0 + 4 * g4;
        if (col >= p.n_cols || r0 >= p.x_rows) continue;
        const uint32_t req = p.col_tags[2 * col], tag = p.col_tags[2 * col + 1];
        const uint4 fo = philox(grp0 + g4, tag, req, ctr3, p.seed_own);
        const uint4 fp = philox(grp0 + g4, tag, req, ctr3, p.seed_prev);
        const uint4 a = *reinterpret_cast<const uint4*>(zs + cc * TM + 4 * g4);
        uint32_t* dst = p.z + static_cast<uint64_t>(col) * p.ldz + r0;
        if (r0 + 4 <= p.x_rows) {
          const uint4 u = *reinterpret_cast<const uint4*>(dst);
          const uint4 v = make_uint4(a.x + u.x + fo.x - fp.x, a.y + u.y + fo.y - fp.y, a.z + u.z + fo.z - fp.z,
                                     a.w + u.w + fo.w - fp.w);
          __stcs(reinterpret_cast<uint4*>(dst), v);  // streamed: z is read by a later kernel, not from L2
        } else {
          const uint32_t av[4] = {a.x, a.y, a.z, a.w}, f[4] = {fo.x - fp.x, fo.y - fp.y, fo.z - fp.z, fo.w - fp.w};
          for (uint32_t e = 0; e < p.x_rows - r0; ++e) dst[e] = av[e] + dst[e] + f[e];
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int launch_tc32(const Maps32& m, const Tc32Params& p, uint32_t n_cols, size_t x_rows, cudaStream_t stream) {
  static PerDevice attr;
  IPC_CUDA_TRY(attr.run(
      [] { return cudaFuncSetAttribute(gemm_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES); }));
  const dim3 grid((n_cols + TN - 1) / TN, static_cast<unsigned>((x_rows + TM - 1) / TM));
  gemm_tc32_kernel<<<grid, THREADS, SMEM_BYTES, stream>>>(m, p);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

}  // namespace

// segments: 2 for K = 2l over [x[0..3] | x[4..7]] (ABY3 replicated sharing, x[4..7] the
// previous party's component), 1 for K = l over x[0..3] alone. K must be a multiple of 256.
int ring_gemm_tc32(uint32_t segments, const int8_t* const x[8], size_t x_rows, const uint16_t* const b[4],
                   uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                   uint64_t seed_prev, uint32_t vec, uint32_t* z, size_t ldz, uint64_t row0, cudaStream_t stream) {
  if (segments != 1 && segments != 2) {
    set_error("Z_2^32 ring GEMM: one or two K segments");
    return IPC_EINVAL;
  }
  if ((segments * l) % (8 * KB) != 0) {
    set_error("Z_2^32 ring GEMM: K must be a multiple of 256");
    return IPC_EINVAL;
  }
  if (n_pad % 128 != 0 || n_cols > n_pad || ldz % 4 != 0 || ldz < x_rows || !aligned16(z)) {
    set_error("Z_2^32 ring GEMM: n_pad % 128, n_cols <= n_pad, ldz % 4, ldz >= x_rows and a 16-byte aligned z");
    return IPC_EINVAL;
  }
  if (x_rows == 0 || n_cols == 0) return IPC_OK;
  if (x_rows > 65535ull * TM) {
    set_error("Z_2^32 ring GEMM: too many rows for one launch");
    return IPC_EINVAL;
  }
  Maps32 m;
  int rc;
  for (int i = 0; i < 4; ++i) {
    if ((rc = make_map_f16(&m.b[i], b[i], static_cast<uint64_t>(segments) * l, n_pad, TN)) ||
        (rc = make_map_i8(&m.a0[i], x[i], l, x_rows, TM)) ||
        (rc = make_map_i8(&m.a1[i], x[segments == 2 ? 4 + i : i], l, x_rows, TM)))
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
  return launch_tc32(m, p, n_cols, x_rows, stream);
}

int prep_query32(const uint32_t* y, uint64_t y_plane, uint32_t Q, const ipc_geom* g, uint32_t party,
                 uint32_t segments, uint16_t* const b[4], uint32_t n_pad, cudaStream_t stream) {
  const uint64_t l = g ? static_cast<uint64_t>(g->rows) * g->cols * g->cell : 0;
  if (!g || l == 0 || g->R == 0 || g->R > 31 || party > 2 || (segments != 1 && segments != 2) || !y || !b || !b[0] ||
      !b[1] || !b[2] || !b[3] || Q == 0 || static_cast<uint64_t>(Q) * g->R > n_pad) {
    set_error("Z_2^32 query operand: bad geometry, party, segments, pointers or n_pad < Q*R");
    return IPC_EINVAL;
  }
  for (int i = 0; i < 4; ++i)
    if (reinterpret_cast<uintptr_t>(b[i]) & 15u) {
      set_error("Z_2^32 query operand: limb planes must be 16-byte aligned");
      return IPC_EINVAL;
    }
  const uint64_t threads = static_cast<uint64_t>(n_pad) * segments * l / 8;
  const uint32_t bs = 256;
  prep_query32_kernel<<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, stream>>>(
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

extern "C" int ipc_split_limbs32(const uint32_t* x, size_t count, int8_t* const limbs[4], void* stream) {
  if (!x || !limbs || !limbs[0] || !limbs[1] || !limbs[2] || !limbs[3]) {
    set_error("ipc_split_limbs32: null pointer");
    return IPC_EINVAL;
  }
  if (!aligned16(x)) {
    set_error("ipc_split_limbs32: x must be 16-byte aligned");
    return IPC_EINVAL;
  }
  for (int i = 0; i < 4; ++i)
    if (reinterpret_cast<uintptr_t>(limbs[i]) & 3u) {
      set_error("ipc_split_limbs32: limb planes must be 4-byte aligned");
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

extern "C" int ipc_prep_query32_f16(const uint32_t* y, uint32_t Q, const ipc_geom* g, uint32_t party,
                                    uint32_t segments, uint16_t* const b[4], uint32_t n_pad, void* stream) {
  const uint64_t l = g ? static_cast<uint64_t>(g->rows) * g->cols * g->cell : 0;
  return prep_query32(y, Q * l, Q, g, party, segments, b, n_pad, static_cast<cudaStream_t>(stream));
}

extern "C" int ipc_ring_gemm_tc32(uint32_t segments, const int8_t* const x[8], size_t x_rows,
                                  const uint16_t* const b[4], uint32_t n_cols, uint32_t n_pad, uint32_t l,
                                  const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec,
                                  uint32_t* z, size_t ldz, uint64_t row0, void* stream) {
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
  if (l % 16 != 0) {
    set_error("ipc_ring_gemm_tc32: l must be a multiple of 16");
    return IPC_EINVAL;
  }
  return ring_gemm_tc32(segments, x, x_rows, b, n_cols, n_pad, l, col_tags, seed_own, seed_prev, vec, z, ldz, row0,
                        static_cast<cudaStream_t>(stream));
}
