// A3 -- share-domain dot products as an int8-limb ring GEMM on the tensor cores.
//
// Each Z_{2^16} operand is stored as balanced signed limbs x = 256*hi + lo, so
//     x*y = lo*lo' + 256*(lo*hi' + hi*lo') + 2^16*hi*hi'  ==  L + 256*C  (mod 2^16)
// and only three int8 products are needed (Sec. 6.1: 3 int8 GEMMs for Z_{2^16}; the
// higher cross term vanishes mod 2^16). |L|, |C| < 2^30 for K <= 2^15, so the int32
// accumulators never wrap and the result is exact.
//
// sm_103a has no tcgen05 integer MMA kind, so the tensor-core path is the warp-level
// mma.sync.m16n8k32.s32.s8.s8.s32. Operand tiles are moved by TMA (cp.async.bulk.tensor,
// 128-byte swizzle) into a 3-stage shared-memory ring guarded by mbarriers; one producer
// lane issues the copies, the consumer warps read them.
//
// Two consumer layouts (template MODE):
//   MODE 0 (IPC_PATH_I8MMA): eight mma.sync warps, 2 (query) x 4 (database) of 64 x 32.
//   MODE 1 (IPC_PATH_I8MIX): eight mma.sync warps (32 x 32) cover database rows 0..63 of the
//     tile and eight dp4a warps cover rows 64..127. On sm_103 the int8 mma.sync rate (256 MAC/clk/SM)
//     equals the dp4a rate of the integer pipe, and the two do not share an issue pipe, so
//     splitting each tile between them runs both units at once on the same staged operands.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "tcgen05.cuh"  // PerDevice, sm_count_current

namespace ipc {
namespace {

constexpr int BND = 128;  // database rows per tile (mma N)
constexpr int BK = 128;   // bytes of K per stage and limb plane (= swizzle span)
constexpr int STAGES = 3;
constexpr int XT = BND * BK;  // bytes of one database limb tile
// MODE 0: 8 mma warps (two per SM sub-partition).
// MODE 1: 8 mma warps (32 x 32 each) + 8 dp4a warps (8 x 4 per thread): two of each per SM
// sub-partition, every consumer thread with 64 accumulators, which keeps both the tensor pipe and
// the integer pipe near their full rates when they run together.
// In both, one consumer lane also issues the TMA copies (no producer warp, so that a block has
// at most 4 warps per sub-partition and 255 registers per thread in MODE 0).
template <int MODE>
constexpr int kConsumerWarps = MODE == 0 ? 8 : 16;
template <int MODE>
constexpr int kThreads = kConsumerWarps<MODE> * 32;
// Stage layout for query tiles of BQ columns: [query lo | query hi | database lo | database hi].
template <int BQ>
constexpr int kQT = BQ * BK;
template <int BQ>
constexpr int kStageBytes = 2 * kQT<BQ> + 2 * XT;
template <int BQ>
constexpr int kSmemBytes = STAGES * kStageBytes<BQ> + 1024 + 2 * STAGES * 8;

struct Params {
  uint32_t n_cols;
  uint32_t x_rows;
  uint32_t ktiles;       // 2l / BK
  uint32_t ktiles_half;  // l / BK
  uint32_t n_row_tiles;  // ceil(x_rows / BND)
  uint32_t n_col_tiles;  // column tiles when col_tiles is null
  const uint32_t* col_tiles;    // optional list of the column tiles to compute (device)
  const uint32_t* n_col_list;   // its length (device), read when col_tiles is set
  const uint32_t* col_tags;
  uint64_t seed_own, seed_prev;
  uint32_t vec;
  uint16_t* z;
  uint64_t ldz;
  uint64_t row0;
  uint32_t* status;
};

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

// Waits for the phase of the given parity; gives up after 2 s of wall time, raising the status word.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* status) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > 2000000000ull) {
      raise_status(status, ST_WAIT_TIMEOUT);
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

__device__ __forceinline__ void ldsm4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_s8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 32-bit shared-memory load (volatile: it must stay after the stage's barrier wait).
__device__ __forceinline__ int lds32(uint32_t addr) {
  int v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// Byte offset of the 16-byte chunk `chunk` of row `row` in a 128-byte-row tile written by TMA
// with CU_TENSOR_MAP_SWIZZLE_128B (chunk index XOR row mod 8, tile base 1024-byte aligned).
__device__ __forceinline__ uint32_t swz(uint32_t row, uint32_t chunk) {
  return row * 128u + ((chunk ^ (row & 7u)) << 4);
}

// Party i's zero share for query column `col` and global row gr: F(seed_own) - F(seed_prev)
// with F = half (gr & 1) of word ((gr >> 1) & 3) of Philox(seed, (gr >> 3, tag, req, D_ZA | vec)).
__device__ __forceinline__ uint32_t zero_share_word(const Params& p, uint32_t col, uint64_t gr) {
  const uint32_t req = p.col_tags[2 * col], tag = p.col_tags[2 * col + 1];
  const uint32_t grp = static_cast<uint32_t>(gr >> 3), wi = static_cast<uint32_t>((gr >> 1) & 3u);
  const uint32_t fo = word_of(philox(grp, tag, req, (IPC_D_ZA << 24) | p.vec, p.seed_own), wi);
  const uint32_t fp = word_of(philox(grp, tag, req, (IPC_D_ZA << 24) | p.vec, p.seed_prev), wi);
  // both halves at once: low half for the even row, high half for the odd row
  return (((fo & 0xFFFFu) - (fp & 0xFFFFu)) & 0xFFFFu) | (((fo >> 16) - (fp >> 16)) << 16);
}

// z = L + 256 C + r (mod 2^16) for rows r (even) and r+1 of query column col.
__device__ __forceinline__ void store_pair(const Params& p, uint32_t col, uint32_t r, uint32_t L0, uint32_t C0,
                                           uint32_t L1, uint32_t C1) {
  if (r >= p.x_rows) return;
  const uint32_t zs = zero_share_word(p, col, p.row0 + r);
  const uint32_t z0 = L0 + (C0 << 8) + (zs & 0xFFFFu);
  const uint32_t z1 = L1 + (C1 << 8) + (zs >> 16);
  uint16_t* zc = p.z + static_cast<uint64_t>(col) * p.ldz;
  if (r + 1 < p.x_rows)
    *reinterpret_cast<uint32_t*>(zc + r) = (z0 & 0xFFFFu) | (z1 << 16);
  else
    zc[r] = static_cast<uint16_t>(z0);
}

// Work of one CTA. Without a tile list (LIST false) the grid is (column tiles, row tiles) and a CTA
// computes the one tile of its block index. With a list (LIST true) gridDim.x CTAs walk items
// w = blockIdx.x + i * gridDim.x, i = 0, 1, ...; item w is column tile list[w % n_ct] and database
// row tile w / n_ct, so the CTAs running at the same time share database tiles through L2. Every
// k-tile a CTA streams has a global index G = i * ktiles + kt, which drives the stage ring (stage
// G % STAGES, phase (G / STAGES) & 1).
template <bool LIST>
struct Work {
  uint32_t n_ct, my_items;
  __device__ Work(const Params& p) {
    if (LIST) {
      n_ct = *p.n_col_list;
      const uint32_t n_items = n_ct * p.n_row_tiles;
      my_items = n_items > blockIdx.x ? (n_items - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    } else {
      n_ct = gridDim.x;
      my_items = 1;
    }
  }
  __device__ __forceinline__ uint32_t items() const { return LIST ? my_items : 1u; }
  template <int BQ>
  __device__ __forceinline__ void coords(const Params& p, uint32_t i, uint32_t& q0, uint32_t& d0) const {
    if (LIST) {
      const uint32_t w = blockIdx.x + i * gridDim.x;
      q0 = p.col_tiles[w % n_ct] * BQ;
      d0 = (w / n_ct) * BND;
    } else {
      q0 = blockIdx.x * BQ;
      d0 = blockIdx.y * BND;
    }
  }
};

// dp4a consumer warps of MODE 1: 256 threads cover query rows 0..127 x database rows 64..127
// of each tile, 8 x 4 per thread: thread (tq, td), tq < 16, td < 16, owns query rows tq + 16 i and
// database rows 64 + td + 16 j. All rows of a thread share one swizzle phase (row & 7), so one XOR
// offset serves all its loads of a k-quad. A warp holds 8 tq (lane & 7) x 4 td (lane >> 3): each
// of its loads touches 8 (A) or 4 (B) rows of distinct phases, i.e. distinct banks, so every
// shared load is a single wavefront. Per k-quad and thread: 24 loads, 96 dp4a.
template <bool LIST, typename Refill, typename Drain>
__device__ __forceinline__ void dp4a_consumer(const Params& p, const Work<LIST>& wk, const uint8_t* smem, uint32_t bars,
                                              int dw, int lane, Refill refill, Drain drain) {
  constexpr int QT = kQT<128>, SB = kStageBytes<128>;
  const uint32_t tq = (lane & 7u) + 8u * (dw & 1), td = (lane >> 3) + 4u * (dw >> 1);
  const uint32_t ra7 = tq & 7u, rb7 = td & 7u;  // swizzle phase of this thread's rows
  for (uint32_t i = 0; i < wk.items(); ++i) {
    uint32_t q0, d0;
    wk.template coords<128>(p, i, q0, d0);
    int accL[8][4], accC[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        accL[a][b] = 0;
        accC[a][b] = 0;
      }
    for (uint32_t kt = 0; kt < p.ktiles; ++kt) {
      const uint32_t G = i * p.ktiles + kt;
      const uint32_t s = G % STAGES, ph = (G / STAGES) & 1u;
      if (!mbar_wait(bars + 8 * s, ph, p.status)) {
        drain(G);
        return;
      }
      const uint32_t base = smem_addr(smem) + s * SB;
      const uint32_t qlo = base + tq * 128u, qhi = qlo + QT;
      const uint32_t xlo = base + 2 * QT + (64u + td) * 128u, xhi = xlo + XT;
#pragma unroll 1
      for (uint32_t c = 0; c < BK / 16; ++c) {
        const uint32_t oa = (c ^ ra7) << 4, ob = (c ^ rb7) << 4;
#pragma unroll 1  // the sibling dp4a warp hides this warp's load latency; unrolling would spill
        for (uint32_t wv = 0; wv < 4; ++wv) {
          int alo[8], ahi[8], blo[4], bhi[4];
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            alo[a] = lds32(qlo + 2048u * a + oa + 4u * wv);
            ahi[a] = lds32(qhi + 2048u * a + oa + 4u * wv);
          }
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            blo[b] = lds32(xlo + 2048u * b + ob + 4u * wv);
            bhi[b] = lds32(xhi + 2048u * b + ob + 4u * wv);
          }
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              accL[a][b] = __dp4a(alo[a], blo[b], accL[a][b]);
              accC[a][b] = __dp4a(alo[a], bhi[b], accC[a][b]);
              accC[a][b] = __dp4a(ahi[a], blo[b], accC[a][b]);
            }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + 8 * (STAGES + s));
      if (!refill(G)) {
        drain(G);
        return;
      }
    }
    // epilogue: lanes l and l + 8 (l & 8 == 0) hold database rows td and td + 1; the lower lane
    // takes its partner's pair through a shuffle and stores both rows
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const uint32_t col = q0 + tq + 16 * a;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t L_nb = __shfl_down_sync(0xFFFFFFFFu, static_cast<uint32_t>(accL[a][b]), 8);
        const uint32_t C_nb = __shfl_down_sync(0xFFFFFFFFu, static_cast<uint32_t>(accC[a][b]), 8);
        if ((td & 1u) == 0 && col < p.n_cols) {
          const uint32_t r = d0 + 64 + td + 16 * b;
          store_pair(p, col, r, static_cast<uint32_t>(accL[a][b]), static_cast<uint32_t>(accC[a][b]), L_nb, C_nb);
        }
      }
    }
  }
}

// MODE 0: BQ in {32, 64, 128}; MODE 1: BQ = 128. LIST: persistent CTAs walking a column-tile list.
template <int MODE, int BQ, bool LIST>
__global__ void __launch_bounds__(kThreads<MODE>, 1)
    gemm_i8_kernel(const __grid_constant__ CUtensorMap tq_lo, const __grid_constant__ CUtensorMap tq_hi,
                   const __grid_constant__ CUtensorMap tx0_lo, const __grid_constant__ CUtensorMap tx0_hi,
                   const __grid_constant__ CUtensorMap tx1_lo, const __grid_constant__ CUtensorMap tx1_hi,
                   const Params p) {
  constexpr int QT = kQT<BQ>, SB = kStageBytes<BQ>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t tiles = smem_addr(smem);
  const uint32_t bars = tiles + STAGES * SB;  // full[s] at bars + 8s, empty[s] at bars + 8(STAGES + s)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Work<LIST> wk(p);
  if (wk.items() == 0) return;
  const uint32_t total = wk.items() * p.ktiles;  // k-tiles this CTA streams

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bars + 8 * s, 1);
      mbar_init(bars + 8 * (STAGES + s), kConsumerWarps<MODE>);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Issues the four TMA copies of global k-tile G into stage G % STAGES.
  auto issue = [&](uint32_t G) {
    const uint32_t i = G / p.ktiles, kt = G % p.ktiles;
    uint32_t q0, d0;
    wk.template coords<BQ>(p, i, q0, d0);
    const uint32_t s = G % STAGES;
    const uint32_t full = bars + 8 * s;
    const uint32_t base = tiles + s * SB;
    mbar_expect_tx(full, SB);
    tma_load(base, &tq_lo, static_cast<int32_t>(kt * BK), static_cast<int32_t>(q0), full);
    tma_load(base + QT, &tq_hi, static_cast<int32_t>(kt * BK), static_cast<int32_t>(q0), full);
    const bool first = kt < p.ktiles_half;
    const int32_t kx = static_cast<int32_t>((first ? kt : kt - p.ktiles_half) * BK);
    tma_load(base + 2 * QT, first ? &tx0_lo : &tx1_lo, kx, static_cast<int32_t>(d0), full);
    tma_load(base + 2 * QT + XT, first ? &tx0_hi : &tx1_hi, kx, static_cast<int32_t>(d0), full);
  };

  // The issuing lane (warp 0 in MODE 0, the first dp4a warp in MODE 1) primes the ring, and after
  // finishing k-tile G refills the stage of k-tile G-1 (all consumers are done with it by then in
  // the common case) with k-tile G-1+STAGES; its sibling warp on the same sub-partition keeps that
  // unit busy while it waits.
  constexpr uint32_t kIssuer = MODE == 0 ? 0 : 8 * 32;
  if (threadIdx.x == kIssuer) {
    const uint32_t pro = total < STAGES ? total : STAGES;
    for (uint32_t G = 0; G < pro; ++G) issue(G);
  }
  auto refill = [&](uint32_t G) -> bool {
    if (threadIdx.x != kIssuer || G == 0) return true;
    const uint32_t Gr = G - 1 + STAGES;
    if (Gr >= total) return true;
    const uint32_t sp = (G - 1) % STAGES, php = ((G - 1) / STAGES) & 1u;
    if (!mbar_wait(bars + 8 * (STAGES + sp), php, p.status)) return false;
    issue(Gr);
    return true;
  };
  // Before leaving early, the issuing thread waits (bounded) for its copies still in flight.
  auto drain = [&](uint32_t G_failed) {
    if (threadIdx.x != kIssuer) return;
    // copies issued so far: k-tiles below G_failed + STAGES - 1 (refills run one tile behind)
    const uint32_t issued = (G_failed + STAGES - 1 < total) ? G_failed + STAGES - 1 : total;
    for (uint32_t G = G_failed; G < issued; ++G) mbar_wait(bars + 8 * (G % STAGES), (G / STAGES) & 1u, p.status);
  };

  if (MODE == 1 && warp >= 8) {
    dp4a_consumer(p, wk, smem, bars, warp - 8, lane, refill, drain);
    return;
  }
  // ------------- mma.sync consumers: WQ (query) x WD (database) warps of (16 MF) x 32 -------------
  constexpr int WD = MODE == 0 ? 4 : 2;          // warps along the database rows
  constexpr int MF = MODE == 0 ? BQ / 32 : 2;    // 16-row query fragments per warp
  const int wq = warp / WD, wd = warp % WD;
  // ldmatrix row/chunk of this lane: A (query) x4 = rows 0-7/8-15 x k-chunks 0/1;
  // B (database) x4 = (n 0-7, k0), (n 0-7, k1), (n 8-15, k0), (n 8-15, k1).
  const uint32_t a_row = wq * (16 * MF) + (lane & 7) + ((lane >> 3) & 1) * 8;
  const uint32_t a_chk = lane >> 4;
  const uint32_t b_row = wd * 32 + (lane & 7) + (lane >> 4) * 8;
  const uint32_t b_chk = (lane >> 3) & 1;

  for (uint32_t i = 0; i < wk.items(); ++i) {
    uint32_t q0, d0;
    wk.template coords<BQ>(p, i, q0, d0);
    int accL[MF][4][4], accC[MF][4][4];
#pragma unroll
    for (int m = 0; m < MF; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          accL[m][n][e] = 0;
          accC[m][n][e] = 0;
        }
    for (uint32_t kt = 0; kt < p.ktiles; ++kt) {
      const uint32_t G = i * p.ktiles + kt;
      const uint32_t s = G % STAGES, ph = (G / STAGES) & 1u;
      if (!mbar_wait(bars + 8 * s, ph, p.status)) {
        drain(G);
        return;
      }
      const uint32_t base = tiles + s * SB;
      const uint32_t qlo = base, qhi = base + QT, xlo = base + 2 * QT, xhi = base + 2 * QT + XT;
#pragma unroll
      for (uint32_t ks = 0; ks < BK / 32; ++ks) {
        uint32_t alo[MF][4], ahi[MF][4], blo[4][2], bhi[4][2];
#pragma unroll
        for (int m = 0; m < MF; ++m) {
          const uint32_t off = swz(a_row + 16 * m, 2 * ks + a_chk);
          ldsm4(qlo + off, alo[m][0], alo[m][1], alo[m][2], alo[m][3]);
          ldsm4(qhi + off, ahi[m][0], ahi[m][1], ahi[m][2], ahi[m][3]);
        }
#pragma unroll
        for (int np = 0; np < 2; ++np) {
          const uint32_t off = swz(b_row + 16 * np, 2 * ks + b_chk);
          ldsm4(xlo + off, blo[2 * np][0], blo[2 * np][1], blo[2 * np + 1][0], blo[2 * np + 1][1]);
          ldsm4(xhi + off, bhi[2 * np][0], bhi[2 * np][1], bhi[2 * np + 1][0], bhi[2 * np + 1][1]);
        }
#pragma unroll
        for (int m = 0; m < MF; ++m)
#pragma unroll
          for (int n = 0; n < 4; ++n) {
            mma_s8(accL[m][n], alo[m], blo[n][0], blo[n][1]);
            mma_s8(accC[m][n], alo[m], bhi[n][0], bhi[n][1]);
            mma_s8(accC[m][n], ahi[m], blo[n][0], blo[n][1]);
          }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + 8 * (STAGES + s));
      if (!refill(G)) {
        drain(G);
        return;
      }
    }
    // ---------------- epilogue: z = L + 256 C + r_i  (mod 2^16) ----------------
    const uint32_t g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int m = 0; m < MF; ++m)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t col = q0 + wq * (16 * MF) + m * 16 + g + 8 * h;
        if (col >= p.n_cols) continue;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          const uint32_t r = d0 + wd * 32 + n * 8 + 2 * t;  // even; rows r, r+1
          store_pair(p, col, r, static_cast<uint32_t>(accL[m][n][2 * h]), static_cast<uint32_t>(accC[m][n][2 * h]),
                     static_cast<uint32_t>(accL[m][n][2 * h + 1]), static_cast<uint32_t>(accC[m][n][2 * h + 1]));
        }
      }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 2-D int8 tensor [rows][cols] (row stride `cols` bytes), box 128 bytes x box_rows, 128-byte swizzle,
// zero fill outside the tensor (ragged row tails).
int make_map(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return IPC_ECUDA;
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols};
  cuuint32_t box[2] = {BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string(static_cast<int>(r)));
    return IPC_ECUDA;
  }
  return IPC_OK;
}

}  // namespace

namespace {

template <int MODE, int BQ, bool LIST>
int launch_variant(const CUtensorMap* m, const Params& p, dim3 grid, cudaStream_t stream) {
  static tc::PerDevice attr;  // a kernel attribute belongs to one device's context
  IPC_CUDA_TRY(attr.run([] {
    return cudaFuncSetAttribute(gemm_i8_kernel<MODE, BQ, LIST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmemBytes<BQ>);
  }));
  gemm_i8_kernel<MODE, BQ, LIST><<<grid, kThreads<MODE>, kSmemBytes<BQ>, stream>>>(m[0], m[1], m[2], m[3], m[4], m[5], p);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

}  // namespace

// variant: 0 = mma.sync + dp4a (BQ 128), 1 = mma.sync (BQ 128), 2 = mma.sync (BQ 64),
// 3 = mma.sync (BQ 32). With col_tiles set, the GEMM covers only the listed BQ-column tiles,
// n_col_list (device) holding their count, and the grid is one persistent CTA per SM.
int ring_gemm_i8_variant(int variant, const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows,
                         const int8_t* b_lo, const int8_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                         const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z,
                         size_t ldz, uint64_t row0, const uint32_t* col_tiles, const uint32_t* n_col_list,
                         cudaStream_t stream) {
  static const uint32_t kBQ[4] = {128, 128, 64, 32};
  if (variant < 0 || variant > 3) {
    set_error("ring GEMM: unknown variant");
    return IPC_EINVAL;
  }
  const uint32_t bq = kBQ[variant];
  CUtensorMap m[6];
  int rc;
  if ((rc = make_map(&m[0], b_lo, 2ull * l, n_pad, bq)) || (rc = make_map(&m[1], b_hi, 2ull * l, n_pad, bq)) ||
      (rc = make_map(&m[2], x_lo[0], l, x_rows, BND)) || (rc = make_map(&m[3], x_hi[0], l, x_rows, BND)) ||
      (rc = make_map(&m[4], x_lo[1], l, x_rows, BND)) || (rc = make_map(&m[5], x_hi[1], l, x_rows, BND)))
    return rc;
  Params p;
  p.n_cols = n_cols;
  p.x_rows = static_cast<uint32_t>(x_rows);
  p.ktiles = 2 * l / BK;
  p.ktiles_half = l / BK;
  p.n_row_tiles = static_cast<uint32_t>((x_rows + BND - 1) / BND);
  p.n_col_tiles = (n_cols + bq - 1) / bq;
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
  // Without a tile list every tile gets its own CTA (a 2-D grid, measured faster for a fixed
  // shape); with a list whose length is known only on the device, one persistent CTA per SM walks it.
  if (col_tiles) {
    const dim3 grid(static_cast<unsigned>(tc::sm_count_current()));
    switch (variant) {
      case 0: return launch_variant<1, 128, true>(m, p, grid, stream);
      case 1: return launch_variant<0, 128, true>(m, p, grid, stream);
      case 2: return launch_variant<0, 64, true>(m, p, grid, stream);
      default: return launch_variant<0, 32, true>(m, p, grid, stream);
    }
  }
  if (p.n_row_tiles > 65535u) {
    set_error("ring GEMM: too many database rows in one call for a 2-D grid");
    return IPC_EINVAL;
  }
  const dim3 grid(p.n_col_tiles, p.n_row_tiles);
  switch (variant) {
    case 0: return launch_variant<1, 128, false>(m, p, grid, stream);
    case 1: return launch_variant<0, 128, false>(m, p, grid, stream);
    case 2: return launch_variant<0, 64, false>(m, p, grid, stream);
    default: return launch_variant<0, 32, false>(m, p, grid, stream);
  }
}

int ring_gemm_i8(int mode, const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows, const int8_t* b_lo,
                 const int8_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags,
                 uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                 cudaStream_t stream) {
  return ring_gemm_i8_variant(mode == 1 ? 0 : 1, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own,
                              seed_prev, vec, z, ldz, row0, nullptr, nullptr, stream);
}

}  // namespace ipc
