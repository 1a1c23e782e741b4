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
//   2^32. S_s has its own accumulator, started at M = 1.5 * 2^23 and drained while every partial
//   sum stays within M +- 2^22 (so every fp32 addition is exact, as in the 16-bit kernel): S_s
//   gains at most (s + 1) 2^14 per k, so S_3 and S_2 are drained every 64 k, S_1 every 128 k,
//   S_0 every 256 k. A drain adds (bits - bits(M)) << 8s to a 32-bit running sum per column;
//   bits(M) << 8s vanishes mod 2^32 for s >= 2, and the S_1 and S_0 terms are subtracted once,
//   up front. The database limbs are widened from int8 to fp16 in shared memory, as in the
//   16-bit kernel. Every wait is bounded (2 s, or sooner once another role has failed); a failed
//   CTA raises the status word, lets its copies and MMAs finish, frees its tensor memory and
//   stores nothing.
#include <cuda_fp16.h>

#include <mutex>
#include <string>

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
// One CTA per tile of 128 database rows x 128 query columns (MMA 128 x 128 x 16).
constexpr int TM = 128, TN = 128, KB = 32, LIMBS = 4;
constexpr int W_TILE = TM * KB * 2;  // 8 KiB widened (fp16) database tile
constexpr int RAW_TILE = TM * KB;    // 4 KiB raw (int8) database tile
constexpr int B_TILE = TN * KB * 2;  // 8 KiB query tile
constexpr int QS = 3, WS = 2, RS = 4;  // stages of the query, widened and raw rings
constexpr int Q_STAGE = LIMBS * B_TILE;    // 32 KiB: query limbs 0-3
constexpr int W_STAGE = LIMBS * W_TILE;    // 32 KiB: widened database limbs 0-3
constexpr int R_STAGE = LIMBS * RAW_TILE;  // 16 KiB: raw database limbs 0-3
constexpr int W_OFF = QS * Q_STAGE, R_OFF = W_OFF + WS * W_STAGE, BAR_OFF = R_OFF + RS * R_STAGE;
constexpr int THREADS = 12 * 32, DRAIN_THREADS = 8 * 32;
constexpr int WIDEN_WARP0 = 10, WIDEN_THREADS = 2 * 32;
constexpr uint32_t KB_PER_CHUNK = 2;  // 64 k: the shortest drain period
constexpr uint32_t TMEM_COLS = 4 * TN;
constexpr uint32_t MAGIC = 0x4B400000u;  // fp32 bits of 1.5 * 2^23
// q_full[QS], q_empty[QS], w_full[WS], w_empty[WS], r_full[RS], r_empty[RS], g_full[4],
// g_empty[4], done
constexpr int NUM_BARS = 2 * QS + 2 * WS + 2 * RS + 9;
constexpr int SMEM_BYTES = BAR_OFF + 1024 + 8 * NUM_BARS;
static_assert(SMEM_BYTES <= 232448, "dynamic shared memory per block");
static_assert(TN * TM * 4 <= QS * Q_STAGE, "the z tile is staged in the Q ring");
// kind::f16: D f32, A and B f16, both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (static_cast<uint32_t>(TN >> 3) << 17) | (static_cast<uint32_t>(TM >> 4) << 24);

// Drain period of S_s in 64-k chunks.
__host__ __device__ constexpr uint32_t period(int s) { return s == 0 ? 4u : (s == 1 ? 2u : 1u); }

struct Maps32 {
  CUtensorMap b[LIMBS];   // query limbs [n_pad][K], fp16
  CUtensorMap a0[LIMBS];  // database limbs of the first K segment [x_rows][l], int8
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

// Roles (12 warps), with three rings as in the 16-bit kernel (query, raw database, widened
// database), so that the widening runs ahead of the MMAs:
//   warp 0 lane 0  query producer: per k-block of 32 elements, the four fp16 query limb tiles
//                  (128 x 32, 64-byte swizzle).
//   warps 10-11    raw copies and widening: the four raw int8 database limb tiles of a k-block
//                  (copied RS k-blocks ahead) become fp16 operand tiles in the W ring.
//   warp 1 lane 0  MMA issuer: per k-block the S_3, S_2, S_1, S_0 products in that order,
//                  committing S_s-full after the last k-block of its drain period and the Q and
//                  W stages after the k-block's S_0 products. S_3's drain overlaps the k-block's
//                  other six products; S_2's the S_1, S_0 products and the next k-block's S_3.
//   warps 2-9      drain: each thread owns one TMEM lane (database row) and 64 columns.
// TMEM: S_s in columns [128 s, 128 s + 128), all 512 columns.
__global__ void __launch_bounds__(THREADS, 1) gemm_tc32_kernel(const __grid_constant__ Maps32 m, const Tc32Params p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ uint32_t s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t qring = smem_addr(smem), wring = qring + W_OFF, rring = qring + R_OFF, bars = qring + BAR_OFF;
  const uint32_t q_full = bars, q_empty = q_full + 8 * QS, w_full = q_empty + 8 * QS, w_empty = w_full + 8 * WS,
                 r_full = w_empty + 8 * WS, r_empty = r_full + 8 * RS;
  const uint32_t g_full = r_empty + 8 * RS, g_empty = g_full + 32, done_bar = g_full + 64;
  volatile uint32_t* abort = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t q0 = blockIdx.x * TN, d0 = blockIdx.y * TM;
  const uint32_t n_chunks = p.kb_total / KB_PER_CHUNK;  // a multiple of 4: K is a multiple of 256

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
    for (int g = 0; g < 4; ++g) {
      mbar_init(g_full + 8 * g, 1);
      mbar_init(g_empty + 8 * g, DRAIN_THREADS / 32);
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
      for (uint32_t kb = 0; kb < p.kb_total; ++kb) {
        const uint32_t s = kb % QS;
        if (!mbar_wait(q_empty + 8 * s, ((kb / QS) & 1u) ^ 1u, p.status, abort)) break;
        const uint32_t full = q_full + 8 * s, base = qring + s * Q_STAGE;
        mbar_expect_tx(full, Q_STAGE);
#pragma unroll
        for (int b = 0; b < LIMBS; ++b)
          tma_load(base + b * B_TILE, &m.b[b], static_cast<int32_t>(kb * KB), static_cast<int32_t>(q0), full);
        issued = kb + 1;
      }
      if (*abort) {
        // copies that may still be in flight land before the CTA goes on (bounded, no abort)
        for (uint32_t kb = issued > QS ? issued - QS : 0; kb < issued; ++kb)
          mbar_wait(q_full + 8 * (kb % QS), (kb / QS) & 1u, p.status, nullptr);
      }
    }
  } else if (warp == 1) {
    // -------------------------------- MMA issuer --------------------------------
    if (lane == 0) {
      bool ok = true;
      for (uint32_t kb = 0; kb < p.kb_total && ok; ++kb) {
        const uint32_t qs = kb % QS, ws = kb % WS, c = kb / KB_PER_CHUNK, j = kb % KB_PER_CHUNK;
        if (!mbar_wait(q_full + 8 * qs, (kb / QS) & 1u, p.status, abort) ||
            !mbar_wait(w_full + 8 * ws, (kb / WS) & 1u, p.status, abort))
          break;
        fence_after();
        const uint32_t qbase = qring + qs * Q_STAGE, dbase = wring + ws * W_STAGE;
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
            const uint32_t o = 32u * ks;  // 16 fp16 = 32 bytes along K inside the swizzled row
#pragma unroll
            for (int a = 0; a <= g; ++a)
              umma(t, sdesc(dbase + a * W_TILE + o), sdesc(qbase + (g - a) * B_TILE + o), IDESC);
          }
          if (j == KB_PER_CHUNK - 1 && c % per == per - 1) umma_commit(g_full + 8 * g);
        }
        if (ok) {  // both stages free once these (and all earlier) MMAs are done
          umma_commit(q_empty + 8 * qs);
          umma_commit(w_empty + 8 * ws);
        }
      }
      // every MMA issued above completes before the tensor memory is freed
      umma_commit(done_bar);
      mbar_wait(done_bar, 0, p.status, nullptr);
    }
  } else if (warp >= WIDEN_WARP0) {
    // ------------------------- raw copies and widening ---------------------------
    const uint32_t ct = threadIdx.x - WIDEN_WARP0 * 32;
    uint32_t issued = 0;
    auto load_raw = [&](uint32_t kb) {
      const uint32_t s = kb % RS, full = r_full + 8 * s, base = rring + s * R_STAGE;
      const bool first = kb < p.kb_half;
      const int32_t kx = static_cast<int32_t>((first ? kb : kb - p.kb_half) * KB);
      mbar_expect_tx(full, R_STAGE);
#pragma unroll
      for (int a = 0; a < LIMBS; ++a)
        tma_load(base + a * RAW_TILE, first ? &m.a0[a] : &m.a1[a], kx, static_cast<int32_t>(d0), full);
      issued = kb + 1;
    };
    if (ct == 0)
      for (uint32_t kb = 0; kb < p.kb_total && kb < RS; ++kb) load_raw(kb);
    uint32_t kb = 0;
    for (; kb < p.kb_total; ++kb) {
      const uint32_t rs = kb % RS, ws = kb % WS;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(r_full + 8 * rs, (kb / RS) & 1u, p.status, abort) &&
                                       mbar_wait(w_empty + 8 * ws, ((kb / WS) & 1u) ^ 1u, p.status, abort)))
        break;
      widen_tiles<LIMBS, WIDEN_THREADS>(rring + rs * R_STAGE, RAW_TILE, wring + ws * W_STAGE, W_TILE, ct);
      fence_proxy_async();  // the MMAs read these tiles through the async proxy
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(w_full + 8 * ws);
        mbar_arrive(r_empty + 8 * rs);  // this warp has read raw stage rs
      }
      if (warp == WIDEN_WARP0 && kb + RS < p.kb_total) {
        // refill once both warps have read the stage (a bounded wait, warp-uniform like the others)
        if (!__all_sync(0xFFFFFFFFu, mbar_wait(r_empty + 8 * rs, (kb / RS) & 1u, p.status, abort))) break;
        if (lane == 0) load_raw(kb + RS);
      }
    }
    if (ct == 0 && *abort) {
      // raw copies that may still be in flight land before the CTA leaves (bounded, no abort)
      for (uint32_t h = kb; h < issued; ++h) mbar_wait(r_full + 8 * (h % RS), (h / RS) & 1u, p.status, nullptr);
    }
  } else {
    // ----------------------------------- drain ----------------------------------
    const uint32_t q = static_cast<uint32_t>(warp) & 3u, h = static_cast<uint32_t>(warp - 2) >> 2;
    const uint32_t tl = tmem + ((32u * q) << 16) + 64u * h;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      tmem_fill32(tl + TN * g, MAGIC);
      tmem_fill32(tl + TN * g + 32, MAGIC);
    }
    tmem_wait_st();
    fence_before();
    __syncwarp();
    if (lane == 0)
      for (int g = 0; g < 4; ++g) mbar_arrive(g_empty + 8 * g);
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
        if (lane == 0) mbar_arrive(g_empty + 8 * g);
      }
    }
    // ---- epilogue: z + r_i, r_i = F(seed_own) - F(seed_prev) over Z_{2^32} (App. C) ----
    // The sums go to shared memory (the Q ring is idle: the last S_0-full followed every MMA,
    // and every copy was consumed), then each (column, 4-row group) item adds the zero shares of
    // its four rows, one Philox block per seed, and writes 16 bytes of z.
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
  Maps32 m;
  int rc;
  for (int i = 0; i < LIMBS; ++i) {
    if ((rc = make_map_f16(&m.b[i], b[i], static_cast<uint64_t>(segments) * l, n_pad, TN)) ||
        (rc = make_map_i8(&m.a0[i], x[i], l, x_rows, TM)) ||
        (rc = make_map_i8(&m.a1[i], x[segments == 2 ? LIMBS + i : i], l, x_rows, TM)))
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
