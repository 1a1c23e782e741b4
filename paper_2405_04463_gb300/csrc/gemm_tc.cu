// A3 on the 5th-generation tensor cores: tcgen05.mma (kind::f16) with fp16 operands carrying the
// balanced int8 limbs, fp32 accumulators in tensor memory.
//
// The ring product is the same three limb products as the int8 paths (Sec. 6.1):
//     z = L + 256 C + r  (mod 2^16),  L = sum lo*lo',  C = sum (lo*hi' + hi*lo').
// sm_103a has no integer tcgen05 kind, but the arithmetic stays exact on the f16 kind:
//   * every limb is an integer in [-128, 127], exactly an fp16 value;
//   * every product is an integer with |p| <= 2^14, exact in fp32;
//   * an accumulator starts at M = 1.5 * 2^23 and is drained and reset to M after at most 256
//     products (C every 128 k: two per k; L every 256 k), so every partial sum, in any order or
//     grouping, is an integer within M +- 2^22, i.e. in [2^23, 2^24], where consecutive fp32
//     values are 1 apart (2^24 included): each addition is exact whatever its rounding;
//   * on [2^23, 2^24] the fp32 bit pattern of M + v is bits(M) + v, and bits(M) = 0x4B400000 is
//     0 mod 2^16, so the raw bits of the two accumulators, added as integers (L + (C << 8)) over
//     all chunks, give z - r mod 2^16 with no conversion instruction.
//
// The database stays resident as int8 limb planes (the size of its u16 shares): TMA brings each
// k-block's raw int8 tiles into shared memory and two widening warps rewrite them as fp16 tiles
// in the MMA's swizzled layout, next to the query tiles (already fp16, prepared per request).
// Three rings decouple the steps, so that the widening never sits on the MMA's critical path:
//   Q ring (QS stages)  query lo/hi tiles, TN x 32 fp16 each, 64-byte swizzle (TMA);
//   R ring (RS stages)  raw database lo/hi tiles, 128 x 32 int8 each (TMA);
//   W ring (WS stages)  widened database lo/hi tiles, 128 x 32 fp16 each (widening warps).
// Each widening warp owns one limb plane: it issues that plane's raw copies itself, RS k-blocks
// ahead, and widens them into the W ring up to WS - 1 k-blocks ahead of the MMAs; the two warps
// never wait for each other.
//
// Roles (one CTA per tile of 128 database rows x TN query columns, 12 warps):
//   warp 0 lane 0  query producer: per k-block of 32 elements, the two query tiles.
//   warps 10-11    raw copies and widening of the lo (warp 10) and hi (warp 11) limb plane.
//   warp 1 lane 0  MMA issuer: per chunk of four k-blocks, the C products (2 MMAs of 128xTNx16
//                  per 16 k) with the L products (1 MMA per 16 k) one k-block behind, committing
//                  C-full after the last C k-block, the k-block's Q and W stages after its L
//                  products, and L-full after every second chunk.
//   warps 2-9      drain: each thread owns one TMEM lane (database row) and TN/2 columns, their
//                  running sums kept mod 2^16 two to a register; after C-full it reads C, adds
//                  C << 8 to the sums and stores M back, and likewise for L after L-full. C is
//                  drained while the chunk's last L products run, L while the next chunk's first
//                  C products run, so the tensor pipe does not wait for the drain.
// TMEM: L in columns [0, TN), C in [TN, 2 TN).
// Tile widths TN = 256 (the fixed-shape launch) and 128; see gemm_tc_kernel for the list mode.
// Every wait is bounded (2 s, or sooner once another role has failed); a failed CTA raises the
// status word, lets its copies and MMAs finish, frees its tensor memory and stores nothing.
#include "compare.cuh"
#include "tcgen05.cuh"

namespace ipc {
namespace {

using namespace tc;

constexpr int TM = 128;          // database rows per tile (MMA M = TMEM lanes)
constexpr int KB = 32;           // elements of K per stage: one 64-byte swizzled fp16 row
constexpr int QS = 4, WS = QS, RS = 4;  // stages of the query, widened and raw rings
static_assert(WS == QS, "a k-block's Q and W stages are released by one commit");
constexpr int KB_PER_CHUNK = 4;  // k-blocks per accumulator chunk (128 k)
static_assert(KB_PER_CHUNK >= 2, "the L products lag the C products by one k-block");
constexpr int A_BYTES = TM * KB * 2;  // 8 KiB widened (fp16) database tile
constexpr int A_RAW = TM * KB;        // 4 KiB raw (int8) database tile
constexpr int THREADS = 12 * 32;
constexpr int DRAIN_THREADS = 8 * 32;
constexpr int WIDEN_WARP0 = 10, WIDEN_THREADS = 2 * 32;
// q_full[QS], q_empty[QS] (also the W stages' release), w_full[WS], r_full[2][RS] (per plane),
// c_full, c_empty, l_full, l_empty, done, epi_done
constexpr int NUM_BARS = 2 * QS + WS + 2 * RS + 6;
constexpr uint32_t MAGIC = 0x4B400000u;  // fp32 bits of 1.5 * 2^23

// Tile shape: TN query columns per tile (MMA N = 256 or 128). Shared memory, 1024-byte aligned:
// the Q ring (first: the epilogue stages z there), the W ring, the R ring, the barriers.
template <int TN>
struct Shape {
  static_assert(TN == 256 || TN == 128, "tile width");
  static constexpr int B_BYTES = TN * KB * 2;
  static constexpr int Q_STAGE = 2 * B_BYTES, W_STAGE = 2 * A_BYTES, R_STAGE = 2 * A_RAW;
  static constexpr int W_OFF = QS * Q_STAGE, R_OFF = W_OFF + WS * W_STAGE, BAR_OFF = R_OFF + RS * R_STAGE;
  static_assert(Q_STAGE % 1024 == 0 && W_STAGE % 1024 == 0 && R_STAGE % 1024 == 0, "aligned stages");
  static constexpr int SMEM_BYTES = BAR_OFF + 1024 + 8 * NUM_BARS;
  static_assert(SMEM_BYTES <= 232448, "dynamic shared memory per block");
  static constexpr uint32_t TMEM_COLS = 2 * TN;  // L in [0, TN), C in [TN, 2 TN)
  static constexpr uint32_t TMEM_C = TN;
  static constexpr int DCOLS = TN / 2;       // columns per drain thread (two drain warps per lane quarter)
  static constexpr int GROUPS = DCOLS / 32;  // 32-column TMEM loads per accumulator and drain
  // Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B f16 (bits 7-9, 10-12 = 0),
  // both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
  static constexpr uint32_t IDESC =
      (1u << 4) | (static_cast<uint32_t>(TN >> 3) << 17) | (static_cast<uint32_t>(TM >> 4) << 24);
  // z of one tile, [TN][TM] uint16, staged in the (then idle) Q ring
  static_assert(TN * TM * 2 <= QS * Q_STAGE, "z tile must fit the Q ring");
};

struct TcParams {
  uint32_t n_cols;
  uint32_t x_rows;
  uint32_t kb_total;  // K / KB (K = 2l, or l for Galois-ring shares)
  uint32_t kb_half;   // l / KB: k-blocks below it read the first database plane pair
  uint32_t n_row_tiles;
  const uint32_t* col_tiles;   // list mode: the column tiles to compute (device)
  const uint32_t* n_col_list;  // list mode: their count (device), read when the kernel starts
  const uint32_t* col_tags;
  uint64_t seed_own, seed_prev;
  uint32_t vec;
  uint16_t* z;
  uint64_t ldz;
  uint64_t row0;
  uint32_t* status;
};

// Fused form (gemm_cmp_kernel, Sec. 6.4's dots followed by the comparisons of the same rows): the
// six ring GEMMs of one chunk -- pass ps = 0..5 is party ps / 2, vector ps % 2 -- run tile after
// tile in one persistent launch, each a complete item of the pipeline above with its own query
// and database tensor maps, zero shares and z output. z stays in L2 (plain stores), and after a
// tile's sixth pass the drain warps run the comparison phase (A4-A8) on the tile: one (column,
// 128-row part) unit per drain thread, through the same part routine and gate numbering as the
// stand-alone comparison kernel, its scratch in the Q ring (idle until the drain releases it).
// The part roots are joined into 1,024-row block roots by or_join_parts afterwards.
constexpr uint32_t NPASS = 6;
struct FuseMaps {
  CUtensorMap q[NPASS][2];  // query operand of pass ps (party ps / 2, vector ps % 2): lo, hi limbs
  CUtensorMap x[NPASS][2];  // database planes of component c, vector v at 2 c + v: lo, hi limbs
};
struct FuseParams {
  uint32_t n_ct;           // column tiles of the launch
  uint16_t* z[NPASS];      // z of pass ps, [n_cols][ldz]
  uint64_t seeds[3];       // seeds[j] shared by parties j and j + 1
  uint32_t thr_a;
  uint32_t* part_roots;    // [3][n_cols][ld_parts]: OR root of (column, row tile) of the chunk
  uint64_t ld_parts;
};
// The six tensor maps of a one-pass launch (kernel parameters).
struct MapRefs {
  const CUtensorMap *b_lo, *b_hi, *a0_lo, *a0_hi, *a1_lo, *a1_hi;
};
constexpr uint32_t FUSE_LOG2_BLOCK = 5;  // 1,024-row OR blocks: 8 row tiles of 128 rows

// Without a list (LIST false) the grid is (column tiles, row tiles), one tile per CTA. With a list,
// gridDim.x persistent CTAs walk items w = blockIdx.x + i * gridDim.x: column tile
// list[w % n_ct], row tile w / n_ct; k-block and chunk counters run on across items, and the
// query producer starts an item's copies once the previous item's epilogue has left the Q ring
// (the raw and widened rings run on into the next item meanwhile).
// bar.sync over n threads that also returns, to every one of them, whether any had pred set.
__device__ __forceinline__ bool named_sync_or(uint32_t id, uint32_t n, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred ? 1u : 0u), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// The comparison phase of one (column n, row tile rt) part in the fused form: z of the chunk's six
// passes from global memory, the part's OR root to fp.part_roots. Not inlined, so that its
// registers do not weigh on the drain loop around it.
__device__ __noinline__ void fused_part_compare(const TcParams& p, const FuseParams& fp, uint32_t n, uint32_t rt,
                                                uint32_t* scratch, uint32_t tid) {
  cmp::CmpParams P{};
  for (int j = 0; j < 3; ++j) {
    P.zc[j] = fp.z[2 * j];
    P.zm[j] = fp.z[2 * j + 1];
    P.seeds.s[j] = fp.seeds[j];
  }
  P.ldz = p.ldz;
  P.n_cols = p.n_cols;
  P.n_rows = p.x_rows;
  P.row0 = p.row0;
  P.col_tags = p.col_tags;
  P.thr_a = fp.thr_a;
  P.p = FUSE_LOG2_BLOCK;
  cmp::B3 root;
  uint32_t nw;
  cmp::part_root<cmp::MODE_LIFT, DRAIN_THREADS>(P, n, rt >> 3, rt & 7u, 3u, scratch, tid, root, nw);
  const uint64_t plane = static_cast<uint64_t>(p.n_cols) * fp.ld_parts;
  const uint64_t at = static_cast<uint64_t>(n) * fp.ld_parts + rt;
  fp.part_roots[at] = root.c0;
  fp.part_roots[plane + at] = root.c1;
  fp.part_roots[2 * plane + at] = root.c2;
}

template <int TN, bool LIST, bool FUSE>
__device__ __forceinline__ void gemm_tc_body(const MapRefs& mr, const FuseMaps* fm, const TcParams& p,
                                             const FuseParams& fp) {
  static_assert(!(LIST && FUSE), "the fused form walks the fixed shape");
  constexpr bool PERSIST = LIST || FUSE;
  using S = Shape<TN>;
  constexpr int B_BYTES = S::B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ uint32_t s_abort;
  uint32_t n_ct = 0, my_items = 1;
  if (LIST) {
    n_ct = *p.n_col_list;
    const uint32_t n_items = n_ct * p.n_row_tiles;
    my_items = n_items > blockIdx.x ? (n_items - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (my_items == 0) return;  // uniform for the CTA, before any barrier or allocation
  }
  if (FUSE) {
    // items: the six passes of each of this CTA's tiles, tile after tile
    n_ct = fp.n_ct;
    const uint32_t n_tiles = n_ct * p.n_row_tiles;
    const uint32_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (my_tiles == 0) return;
    my_items = my_tiles * NPASS;
  }
  // Tiles are taken in linear order (blocks are dispatched in blockIdx order; a persistent CTA
  // takes items blockIdx.x + i gridDim.x). The order walks bands of up to kBand column tiles,
  // all row tiles of a band before the next, so that the tiles in flight at once (one CTA per
  // SM) cover about 19 row tiles x 8 column tiles: each database tile is read by the band's
  // CTAs together and the band's query tiles stay in L2 while the rows stream past (with many
  // query columns the whole query operand is several times the L2).
  constexpr uint32_t kBand = 8;
  auto coords = [&](uint32_t i, uint32_t& q0, uint32_t& d0) {
    const uint32_t n_cols_t = PERSIST ? n_ct : gridDim.x;
    const uint32_t n_rt = PERSIST ? p.n_row_tiles : gridDim.y;
    const uint32_t lin = FUSE   ? blockIdx.x + (i / NPASS) * gridDim.x
                         : LIST ? blockIdx.x + i * gridDim.x
                                : blockIdx.x + gridDim.x * blockIdx.y;
    const uint32_t band = lin / (kBand * n_rt), c0 = band * kBand;
    const uint32_t width = n_cols_t - c0 < kBand ? n_cols_t - c0 : kBand;
    const uint32_t in_band = lin - band * kBand * n_rt;
    const uint32_t ct = c0 + in_band % width;
    q0 = (LIST ? p.col_tiles[ct] : ct) * TN;
    d0 = (in_band / width) * TM;
  };
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t qring = smem_addr(smem), wring = qring + S::W_OFF, rring = qring + S::R_OFF;
  const uint32_t bars = qring + S::BAR_OFF;
  const uint32_t q_full = bars, q_empty = q_full + 8 * QS, w_full = q_empty + 8 * QS, r_full = w_full + 8 * WS;
  const uint32_t c_full = r_full + 16 * RS, c_empty = c_full + 8, l_full = c_full + 16, l_empty = c_full + 24,
                 done_bar = c_full + 32, epi_done = c_full + 40;
  volatile uint32_t* abort = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n_chunks = p.kb_total / KB_PER_CHUNK;  // even: l is a multiple of 128
  const uint32_t total_kb = my_items * p.kb_total;

  if (threadIdx.x == 0) {
    for (int s = 0; s < QS; ++s) {
      mbar_init(q_full + 8 * s, 1);
      mbar_init(q_empty + 8 * s, 1);
    }
    for (int s = 0; s < WS; ++s) mbar_init(w_full + 8 * s, WIDEN_THREADS / 32);
    for (int s = 0; s < 2 * RS; ++s) mbar_init(r_full + 8 * s, 1);
    mbar_init(c_full, 1);
    mbar_init(c_empty, DRAIN_THREADS / 32);
    mbar_init(l_full, 1);
    mbar_init(l_empty, DRAIN_THREADS / 32);
    mbar_init(done_bar, 1);
    mbar_init(epi_done, DRAIN_THREADS / 32);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(S::TMEM_COLS)
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
      bool ok = true;
      for (uint32_t i = 0; i < my_items && ok; ++i) {
        uint32_t q0, d0;
        coords(i, q0, d0);
        if (i > 0 && !mbar_wait(epi_done, (i - 1) & 1u, p.status, abort)) break;
        for (uint32_t kb = 0; kb < p.kb_total; ++kb) {
          const uint32_t G = i * p.kb_total + kb, s = G % QS;
          if (!mbar_wait(q_empty + 8 * s, ((G / QS) & 1u) ^ 1u, p.status, abort)) {
            ok = false;
            break;
          }
          const uint32_t full = q_full + 8 * s, base = qring + s * S::Q_STAGE;
          const CUtensorMap* mlo = FUSE ? &fm->q[i % NPASS][0] : mr.b_lo;
          const CUtensorMap* mhi = FUSE ? &fm->q[i % NPASS][1] : mr.b_hi;
          mbar_expect_tx(full, 2 * B_BYTES);
          tma_load(base, mlo, static_cast<int32_t>(kb * KB), static_cast<int32_t>(q0), full);
          tma_load(base + B_BYTES, mhi, static_cast<int32_t>(kb * KB), static_cast<int32_t>(q0), full);
          issued = G + 1;
        }
      }
      if (*abort) {
        // copies that may still be in flight land before the CTA leaves (bounded, no abort)
        for (uint32_t G = issued > QS ? issued - QS : 0; G < issued; ++G)
          mbar_wait(q_full + 8 * (G % QS), (G / QS) & 1u, p.status, nullptr);
      }
    }
  } else if (warp == 1) {
    // -------------------------------- MMA issuer --------------------------------
    if (lane == 0) {
      const uint32_t tL = tmem, tC = tmem + S::TMEM_C;
      // C products of k-block j, L products of k-block j - 1, so that the C drain of a chunk
      // overlaps its last two L k-blocks and the L drain the next chunk's first two C k-blocks:
      //   C0 C1 L0 C2 L1 C3 [C-full] L2 L3 [L-full]
      auto issue_c = [&](uint32_t qb, uint32_t wb) {
#pragma unroll
        for (uint32_t ks = 0; ks < KB / 16; ++ks) {
          const uint32_t o = 32u * ks;  // 16 fp16 = 32 bytes along K inside the swizzled row
          umma(tC, sdesc(wb + o), sdesc(qb + B_BYTES + o), S::IDESC);  // lo * hi'
          umma(tC, sdesc(wb + A_BYTES + o), sdesc(qb + o), S::IDESC);  // hi * lo'
        }
      };
      auto issue_l = [&](uint32_t G) {
        const uint32_t qs = G % QS, ws = G % WS, qb = qring + qs * S::Q_STAGE, wb = wring + ws * S::W_STAGE;
#pragma unroll
        for (uint32_t ks = 0; ks < KB / 16; ++ks) {
          const uint32_t o = 32u * ks;
          umma(tL, sdesc(wb + o), sdesc(qb + o), S::IDESC);  // lo * lo'
        }
        // the k-block's Q and W stages are free once these (and all earlier) MMAs are done: one
        // commit (an mbarrier that the query producer and the widening warps both wait on)
        umma_commit(q_empty + 8 * qs);
      };
      // C restarts every chunk (128 k), L every other chunk (256 k): L gains at most 2^14 per
      // k, C twice that, so both stay within 2^22 of the base between drains.
      const uint32_t total_chunks = my_items * n_chunks;
      for (uint32_t c = 0; c < total_chunks; ++c) {
        const uint32_t par = c & 1u, G0 = c * KB_PER_CHUNK;
        const bool l_opens = (c & 1u) == 0, l_closes = (c & 1u) == 1;
        if (!mbar_wait(c_empty, par, p.status, abort)) break;
        fence_after();
        bool ok = true;
        for (uint32_t kb = 0; kb < KB_PER_CHUNK; ++kb) {
          const uint32_t G = G0 + kb, qs = G % QS, ws = G % WS;
          // the query tiles landed (TMA) and the database tiles were widened
          if (!mbar_wait(q_full + 8 * qs, (G / QS) & 1u, p.status, abort) ||
              !mbar_wait(w_full + 8 * ws, (G / WS) & 1u, p.status, abort)) {
            ok = false;
            break;
          }
          fence_after();
          issue_c(qring + qs * S::Q_STAGE, wring + ws * S::W_STAGE);
          if (kb == KB_PER_CHUNK - 1) umma_commit(c_full);
          if (kb == 1 && l_opens) {
            if (!mbar_wait(l_empty, (c >> 1) & 1u, p.status, abort)) {
              ok = false;
              break;
            }
            fence_after();
          }
          if (kb >= 1) issue_l(G - 1);
        }
        if (!ok) break;
        issue_l(G0 + KB_PER_CHUNK - 1);
        if (l_closes) umma_commit(l_full);
      }
      // every MMA issued above completes before the tensor memory is freed
      umma_commit(done_bar);
      mbar_wait(done_bar, 0, p.status, nullptr);
    }
  } else if (warp >= WIDEN_WARP0) {
    // ------------------------- raw copies and widening ---------------------------
    // Lane 0 issues this warp's plane's raw copies: the first RS k-blocks up front, then
    // k-block G + RS into raw stage G % RS once the warp has read k-block G from it.
    const uint32_t pl = static_cast<uint32_t>(warp - WIDEN_WARP0);  // 0: lo limbs, 1: hi limbs
    const uint32_t rf = r_full + 8 * RS * pl;
    // the database planes of item i's two K segments: components ps / 2 and ps / 2 - 1 of the
    // pass's vector in the fused form
    auto seg_maps = [&](uint32_t i, const CUtensorMap*& m0, const CUtensorMap*& m1) {
      if (FUSE) {
        const uint32_t ps = i % NPASS, party = ps >> 1, vec = ps & 1u;
        m0 = &fm->x[2 * party + vec][pl];
        m1 = &fm->x[2 * ((party + 2) % 3) + vec][pl];
      } else {
        m0 = pl ? mr.a0_hi : mr.a0_lo;
        m1 = pl ? mr.a1_hi : mr.a1_lo;
      }
    };
    const CUtensorMap *map0, *map1;
    // the next raw copy (lane 0): k-block li_kb of item li, whose row offset li_d0 and tensor
    // maps are looked up once per item, so that a copy costs no division
    uint32_t issued = 0, li = 0, li_kb = 0, li_q0 = 0, li_d0 = 0;
    coords(0, li_q0, li_d0);
    seg_maps(0, map0, map1);
    auto load_raw = [&](uint32_t G) {
      const uint32_t s = G % RS;
      const bool first = li_kb < p.kb_half;
      const int32_t kx = static_cast<int32_t>((first ? li_kb : li_kb - p.kb_half) * KB);
      mbar_expect_tx(rf + 8 * s, A_RAW);
      tma_load(rring + s * S::R_STAGE + pl * A_RAW, first ? map0 : map1, kx, static_cast<int32_t>(li_d0), rf + 8 * s);
      issued = G + 1;
      if (++li_kb == p.kb_total) {
        li_kb = 0;
        if (++li < my_items) {
          coords(li, li_q0, li_d0);
          seg_maps(li, map0, map1);
        }
      }
    };
    if (lane == 0)
      for (uint32_t G = 0; G < total_kb && G < RS; ++G) load_raw(G);
    uint32_t G = 0;
    for (; G < total_kb; ++G) {
      const uint32_t rs = G % RS, ws = G % WS;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(rf + 8 * rs, (G / RS) & 1u, p.status, abort) &&
                                       mbar_wait(q_empty + 8 * ws, ((G / WS) & 1u) ^ 1u, p.status, abort)))
        break;
      widen_tiles<1, 32>(rring + rs * S::R_STAGE + pl * A_RAW, 0, wring + ws * S::W_STAGE + pl * A_BYTES, 0, lane);
      fence_proxy_async();  // the MMAs read these tiles through the async proxy
      __syncwarp();         // every lane has read raw stage rs
      if (lane == 0) {
        mbar_arrive(w_full + 8 * ws);
        if (G + RS < total_kb) load_raw(G + RS);
      }
    }
    if (lane == 0 && *abort) {
      // raw copies that may still be in flight land before the CTA leaves (bounded, no abort)
      for (uint32_t H = G; H < issued; ++H) mbar_wait(rf + 8 * (H % RS), (H / RS) & 1u, p.status, nullptr);
    }
  } else {
    // ----------------------------------- drain ----------------------------------
    // z2[k] holds the running sums (mod 2^16) of columns 2k (low half) and 2k + 1 (high half)
    // of this thread's DCOLS columns.
    constexpr int DCOLS = S::DCOLS, GROUPS = S::GROUPS;
    const uint32_t q = static_cast<uint32_t>(warp) & 3u, h = static_cast<uint32_t>(warp - 2) >> 2;
    const uint32_t tL = tmem + ((32u * q) << 16) + DCOLS * h, tC = tL + S::TMEM_C;
#pragma unroll
    for (uint32_t g = 0; g < GROUPS; ++g) {
      tmem_fill32(tL + 32 * g, MAGIC);
      tmem_fill32(tC + 32 * g, MAGIC);
    }
    tmem_wait_st();
    fence_before();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(c_empty);
      mbar_arrive(l_empty);
    }
    bool ok = true;
    for (uint32_t i = 0; i < my_items && ok; ++i) {
      uint32_t z2[DCOLS / 2];
#pragma unroll
      for (int k = 0; k < DCOLS / 2; ++k) z2[k] = 0;
      for (uint32_t cc = 0; cc < n_chunks; ++cc) {
        const uint32_t gc = i * n_chunks + cc, par = gc & 1u;
        if (!__all_sync(0xFFFFFFFFu, mbar_wait(c_full, par, p.status, abort))) {
          ok = false;
          break;
        }
        fence_after();
#pragma unroll
        for (uint32_t g = 0; g < GROUPS; ++g) {
          uint32_t r[32];
          tmem_ld32(tC + 32 * g, r);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; ++k) z2[16 * g + k] = add16x2(z2[16 * g + k], pack_c16(r[2 * k], r[2 * k + 1]));
          tmem_fill32(tC + 32 * g, MAGIC);
        }
        tmem_wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(c_empty);
        if ((gc & 1u) == 0) continue;  // L closes every other chunk
        if (!__all_sync(0xFFFFFFFFu, mbar_wait(l_full, (gc >> 1) & 1u, p.status, abort))) {
          ok = false;
          break;
        }
        fence_after();
#pragma unroll
        for (uint32_t g = 0; g < GROUPS; ++g) {
          uint32_t r[32];
          tmem_ld32(tL + 32 * g, r);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; ++k) z2[16 * g + k] = add16x2(z2[16 * g + k], pack_lo16(r[2 * k], r[2 * k + 1]));
          tmem_fill32(tL + 32 * g, MAGIC);
        }
        tmem_wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(l_empty);
      }
      // ---- epilogue: z + r_i, r_i = F(seed_own) - F(seed_prev) (App. C) ----
      // The running sums go to shared memory (the Q ring is idle once every drainer has seen the
      // item's last L-full and before the query producer sees epi-done), then each (column, 8-row
      // group) item adds its zero shares, which one Philox block per seed gives for all 8 rows,
      // and writes 16 bytes of z.
      // every drainer takes the same decision: the barrier returns whether any of them saw the
      // abort flag
      if (named_sync_or(1, DRAIN_THREADS, *abort != 0)) break;
      uint32_t q0, d0;
      coords(i, q0, d0);
      const uint32_t ps = FUSE ? i % NPASS : 0u, party = ps >> 1;
      const uint64_t seed_own = FUSE ? fp.seeds[party] : p.seed_own;
      const uint64_t seed_prev = FUSE ? fp.seeds[(party + 2) % 3] : p.seed_prev;
      const uint32_t vec = FUSE ? (ps & 1u) : p.vec;
      uint16_t* const zout = FUSE ? fp.z[ps] : p.z;
      uint16_t* zs = reinterpret_cast<uint16_t*>(smem);  // [TN][TM]
      const uint32_t row = 32 * q + lane;
#pragma unroll
      for (int k = 0; k < DCOLS / 2; ++k) {
        zs[(DCOLS * h + 2 * k) * TM + row] = static_cast<uint16_t>(z2[k]);
        zs[(DCOLS * h + 2 * k + 1) * TM + row] = static_cast<uint16_t>(z2[k] >> 16);
      }
      named_sync(1, DRAIN_THREADS);
      const uint32_t dt = threadIdx.x - 64;
      const uint32_t grp0 = static_cast<uint32_t>((p.row0 + d0) >> 3);
      const uint32_t ctr3 = (IPC_D_ZA << 24) | vec;
      for (uint32_t it = dt; it < TN * (TM / 8); it += DRAIN_THREADS) {
        const uint32_t cc = it / (TM / 8), g = it % (TM / 8), col = q0 + cc, r0 = d0 + 8 * g;
        if (col >= p.n_cols || r0 >= p.x_rows) continue;
        const uint32_t req = p.col_tags[2 * col], tag = p.col_tags[2 * col + 1];
        const uint4 fo = philox(grp0 + g, tag, req, ctr3, seed_own);
        const uint4 fq = philox(grp0 + g, tag, req, ctr3, seed_prev);
        const uint4 acc = *reinterpret_cast<const uint4*>(zs + cc * TM + 8 * g);
        // per 16-bit half: z = acc + (F_own - F_prev)  (mod 2^16)
        auto add2 = [](uint32_t a, uint32_t o, uint32_t f) {
          const uint32_t lo = (a + o - f) & 0xFFFFu;
          const uint32_t hi = ((a >> 16) + (o >> 16) - (f >> 16)) << 16;
          return lo | hi;
        };
        const uint4 v = make_uint4(add2(acc.x, fo.x, fq.x), add2(acc.y, fo.y, fq.y), add2(acc.z, fo.z, fq.z),
                                   add2(acc.w, fo.w, fq.w));
        uint16_t* dst = zout + static_cast<uint64_t>(col) * p.ldz + r0;
        if (r0 + 8 <= p.x_rows) {
          if (FUSE)
            *reinterpret_cast<uint4*>(dst) = v;  // kept in L2: this CTA reads it back after the tile's last pass
          else
            __stcs(reinterpret_cast<uint4*>(dst), v);  // streamed: z is read by a later kernel, not from L2
        } else {
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
          for (uint32_t e = 0; e < p.x_rows - r0; ++e) dst[e] = static_cast<uint16_t>(w[e >> 1] >> (16 * (e & 1)));
        }
      }
      if (FUSE && ps == NPASS - 1) {
        // ---- A4-A8 on the tile: its six z tiles are in global memory (L2), written by this
        // CTA's drainers; the barrier orders those stores before the reads below ----
        named_sync(1, DRAIN_THREADS);
        const uint32_t n = q0 + dt;
        if (n < p.n_cols) fused_part_compare(p, fp, n, d0 / TM, reinterpret_cast<uint32_t*>(smem), dt);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(epi_done);  // this warp is done with the Q ring
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS) : "memory");
  }
}

template <int TN, bool LIST>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tb_lo, const __grid_constant__ CUtensorMap tb_hi,
                   const __grid_constant__ CUtensorMap ta0_lo, const __grid_constant__ CUtensorMap ta0_hi,
                   const __grid_constant__ CUtensorMap ta1_lo, const __grid_constant__ CUtensorMap ta1_hi,
                   const TcParams p) {
  gemm_tc_body<TN, LIST, false>(MapRefs{&tb_lo, &tb_hi, &ta0_lo, &ta0_hi, &ta1_lo, &ta1_hi}, nullptr, p,
                                FuseParams{});
}

__global__ void __launch_bounds__(THREADS, 1)
    gemm_cmp_kernel(const __grid_constant__ FuseMaps fm, const __grid_constant__ TcParams p,
                    const __grid_constant__ FuseParams fp) {
  gemm_tc_body<256, false, true>(MapRefs{}, &fm, p, fp);
}

template <int TN, bool LIST>
int launch_tc(const CUtensorMap* m, const TcParams& p, dim3 grid, cudaStream_t stream) {
  static PerDevice attr;
  IPC_CUDA_TRY(attr.run([] {
    return cudaFuncSetAttribute(gemm_tc_kernel<TN, LIST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Shape<TN>::SMEM_BYTES);
  }));
  gemm_tc_kernel<TN, LIST><<<grid, THREADS, Shape<TN>::SMEM_BYTES, stream>>>(m[0], m[1], m[2], m[3], m[4], m[5], p);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

}  // namespace

// tile_cols: 256 or 128 query columns per tile. With col_tiles set, only the listed tiles of
// that width are computed (n_col_list, on the device, holds their count) by one persistent CTA
// per SM; otherwise every tile of [0, n_cols), one CTA each. segments: 2 for K = 2l over the
// planes [x_lo[0] | x_lo[1]] (replicated sharing), 1 for K = l over x_lo[0] alone (Galois-ring
// Shamir shares; l a multiple of 256 so that L's 256-k drains tile K).
int ring_gemm_tc_variant(uint32_t tile_cols, uint32_t segments, const int8_t* const x_lo[2],
                         const int8_t* const x_hi[2], size_t x_rows, const uint16_t* b_lo, const uint16_t* b_hi,
                         uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                         uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                         const uint32_t* col_tiles, const uint32_t* n_col_list, cudaStream_t stream) {
  if (tile_cols != 256 && tile_cols != 128) {
    set_error("tcgen05 ring GEMM: tile width must be 128 or 256");
    return IPC_EINVAL;
  }
  if (segments != 1 && segments != 2) {
    set_error("tcgen05 ring GEMM: one or two K segments");
    return IPC_EINVAL;
  }
  if ((segments * l) % (2 * KB_PER_CHUNK * KB) != 0) {
    set_error("tcgen05 ring GEMM: K must be a multiple of 256");
    return IPC_EINVAL;
  }
  CUtensorMap m[6];
  int rc;
  if ((rc = make_map_f16(&m[0], b_lo, static_cast<uint64_t>(segments) * l, n_pad, tile_cols)) ||
      (rc = make_map_f16(&m[1], b_hi, static_cast<uint64_t>(segments) * l, n_pad, tile_cols)) ||
      (rc = make_map_i8(&m[2], x_lo[0], l, x_rows, TM)) || (rc = make_map_i8(&m[3], x_hi[0], l, x_rows, TM)) ||
      (rc = make_map_i8(&m[4], x_lo[1], l, x_rows, TM)) || (rc = make_map_i8(&m[5], x_hi[1], l, x_rows, TM)))
    return rc;
  TcParams p;
  p.n_cols = n_cols;
  p.x_rows = static_cast<uint32_t>(x_rows);
  p.kb_total = segments * l / KB;
  p.kb_half = l / KB;  // with one segment every k-block reads x_lo[0] / x_hi[0]
  p.n_row_tiles = static_cast<uint32_t>((x_rows + TM - 1) / TM);
  p.col_tiles = col_tiles;
  p.n_col_list = n_col_list;
  p.col_tags = col_tags;
  p.seed_own = seed_own;
  p.seed_prev = seed_prev;
  p.vec = vec;
  p.z = z;
  p.ldz = ldz;
  p.row0 = row0;
  p.status = status_ptr();
  if (col_tiles) {
    const dim3 grid(static_cast<unsigned>(sm_count_current()));
    return tile_cols == 256 ? launch_tc<256, true>(m, p, grid, stream) : launch_tc<128, true>(m, p, grid, stream);
  }
  const dim3 grid((n_cols + tile_cols - 1) / tile_cols, p.n_row_tiles);
  return tile_cols == 256 ? launch_tc<256, false>(m, p, grid, stream) : launch_tc<128, false>(m, p, grid, stream);
}

// The fused chunk step: the six ring GEMMs of a chunk (replicated sharing, segments = 2: party i
// reads components i and i - 1 of each vector; Galois-ring Shamir shares, segments = 1: party i
// reads its own share) and the comparison phase of every tile, in one persistent launch of one CTA
// per SM. x_lo / x_hi[2 c + v]: database limb planes of component c, vector v (0 code, 1 mask),
// [x_rows][l] int8; b_lo / b_hi[2 i + v]: party i's query operand of vector v, [n_pad][segments l]
// fp16 patterns; z[2 i + v]: party i's z of vector v, [n_cols][ldz]. part_roots: [3][n_cols][ld_parts]
// words, ld_parts >= ceil(x_rows / 128); the chunk must start on a 1,024-row block (row0 % 1024 == 0).
int ring_gemm_compare_tc(uint32_t segments, const int8_t* const x_lo[6], const int8_t* const x_hi[6], size_t x_rows,
                         const uint16_t* const b_lo[6], const uint16_t* const b_hi[6], uint32_t n_cols, uint32_t n_pad,
                         uint32_t l, const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a,
                         uint16_t* const z[6], size_t ldz, uint64_t row0, uint32_t* part_roots, size_t ld_parts,
                         cudaStream_t stream) {
  if (segments != 1 && segments != 2) {
    set_error("fused GEMM + comparison: one or two K segments");
    return IPC_EINVAL;
  }
  if ((segments * l) % (2 * KB_PER_CHUNK * KB) != 0) {
    set_error("fused GEMM + comparison: K must be a multiple of 256");
    return IPC_EINVAL;
  }
  const uint32_t n_rt = static_cast<uint32_t>((x_rows + TM - 1) / TM);
  if (row0 % (32u << FUSE_LOG2_BLOCK) != 0 || ld_parts < n_rt || ldz % 8 != 0 || ldz < x_rows || n_cols == 0 ||
      x_rows == 0 || n_pad < n_cols) {
    set_error("fused GEMM + comparison: need row0 % 1024 == 0, ld_parts >= ceil(rows / 128), ldz % 8 == 0, "
              "ldz >= rows, 1 <= n_cols <= n_pad, rows >= 1");
    return IPC_EINVAL;
  }
  FuseMaps fm;  // passed by value as kernel parameters (3 KiB)
  int rc;
  for (uint32_t s = 0; s < NPASS; ++s) {
    if ((rc = make_map_f16(&fm.q[s][0], b_lo[s], static_cast<uint64_t>(segments) * l, n_pad, 256)) ||
        (rc = make_map_f16(&fm.q[s][1], b_hi[s], static_cast<uint64_t>(segments) * l, n_pad, 256)) ||
        (rc = make_map_i8(&fm.x[s][0], x_lo[s], l, x_rows, TM)) || (rc = make_map_i8(&fm.x[s][1], x_hi[s], l, x_rows, TM)))
      return rc;
  }
  TcParams p{};
  p.n_cols = n_cols;
  p.x_rows = static_cast<uint32_t>(x_rows);
  p.kb_total = segments * l / KB;
  p.kb_half = l / KB;
  p.n_row_tiles = n_rt;
  p.col_tags = col_tags;
  p.ldz = ldz;
  p.row0 = row0;
  p.status = status_ptr();
  FuseParams fp{};
  fp.n_ct = (n_cols + 255) / 256;
  for (uint32_t s = 0; s < NPASS; ++s) fp.z[s] = z[s];
  for (int j = 0; j < 3; ++j) fp.seeds[j] = seeds[j];
  fp.thr_a = thr_a;
  fp.part_roots = part_roots;
  fp.ld_parts = ld_parts;
  static PerDevice attr;
  IPC_CUDA_TRY(attr.run([] {
    return cudaFuncSetAttribute(gemm_cmp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape<256>::SMEM_BYTES);
  }));
  const uint32_t n_tiles = fp.n_ct * n_rt;
  const uint32_t sms = static_cast<uint32_t>(sm_count_current());
  const dim3 grid(n_tiles < sms ? n_tiles : sms);
  gemm_cmp_kernel<<<grid, THREADS, Shape<256>::SMEM_BYTES, stream>>>(fm, p, fp);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

int ring_gemm_tc(const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows, const uint16_t* b_lo,
                 const uint16_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags,
                 uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                 cudaStream_t stream) {
  return ring_gemm_tc_variant(256, 2, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own,
                              seed_prev, vec, z, ldz, row0, nullptr, nullptr, stream);
}

}  // namespace ipc
