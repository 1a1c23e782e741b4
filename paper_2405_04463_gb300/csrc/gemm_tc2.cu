// A3 on tcgen05 with CTA pairs (cta_group::2): the ring product of gemm_tc.cu (same exact
// bf16-carried int8 limbs, the same three limb products and the same accumulator schedule),
// computed by two CTAs on the two SMs of a cluster as one 256 x 256 MMA tile.
//
// Why: an MMA of 128 x 256 x 16 on one SM reads its 4 KiB database tile and 8 KiB query tile from
// that SM's shared memory per 128 tensor cycles, and the TMA fills of the stage ring share the
// same bandwidth; together they cap the single-CTA kernel near 80 % of tensor cycles. In a pair
// MMA (M = 256) each SM holds its own 128 database rows and half of the 256 query columns, so
// per tensor cycle each SM reads and fills a third less.
//
// Pair tile: 256 database rows (CTA rank r of the cluster owns rows 128 r .. 128 r + 127) x 256
// query columns (rank r's shared memory holds columns 128 r .. 128 r + 127 of the query tile).
// Each CTA's tensor memory holds its 128 rows x 256 columns of the L and C accumulators.
//   warp 0 lane 0, both CTAs   TMA producer for its own half of every stage, signalling the
//                              leader's (rank 0's) full barrier (.cta_group::2 TMA).
//   warp 1 lane 0, rank 0      MMA issuer: tcgen05.mma.cta_group::2, commits multicast to both
//                              CTAs' barriers (stage empty, C-full, L-full, done).
//   warps 2-9, both CTAs       drain of its own TMEM lanes, as in gemm_tc.cu; the C-empty and
//                              L-empty barriers live in the leader and count both CTAs' warps.
// Every mbarrier wait is bounded (2 s); a failed CTA raises the status word and stores nothing.
// The pair meets at cluster barriers after set-up and before the tensor memory is freed, so
// neither CTA leaves while MMAs of the pair may still read its shared memory or write its TMEM.
#include <mutex>
#include <string>

#include "tcgen05_pair.cuh"

namespace ipc {
namespace {

using namespace tc;

constexpr int TM = 128;           // database rows per CTA (TMEM lanes)
constexpr int TN = 256;           // query columns per pair tile (MMA N)
constexpr int HN = TN / 2;        // query columns held by each CTA
constexpr int KB = 32;            // bf16 elements of K per stage: one 64-byte swizzled row
constexpr int STAGES = 6;
constexpr int KB_PER_CHUNK = 4;   // k-blocks per C drain (128 k)
constexpr int TILE_BYTES = TM * KB * 2;            // 8 KiB (HN == TM)
constexpr int STAGE_BYTES = 4 * TILE_BYTES;        // database lo/hi, query lo/hi halves: 32 KiB
constexpr int THREADS = 10 * 32;
constexpr int DRAIN_THREADS = 8 * 32;
// full[S], empty[S], c_full, c_empty, l_full, l_empty, done
constexpr int NUM_BARS = 2 * STAGES + 5;
// SLACK: 16 KiB after the ring so that every MMA operand read stays inside the allocation even
// if a query tile were read at its full 256 rows from one CTA.
constexpr int SLACK = 16384;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + SLACK + 1024 + 8 * NUM_BARS;
constexpr uint32_t TMEM_COLS = 2 * TN;  // L in [0, TN), C in [TN, 2 TN)
constexpr uint32_t MAGIC = 0x4B400000u;  // fp32 bits of 1.5 * 2^23
constexpr int DCOLS = TN / 2;           // columns per drain thread
constexpr int GROUPS = DCOLS / 32;
// kind::f16: D f32, A and B bf16, both K-major, N >> 3 at bits 17-22, M >> 4 (M = 256 for the
// pair) at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(TN >> 3) << 17) |
                           (static_cast<uint32_t>((2 * TM) >> 4) << 24);
static_assert(TN * TM * 2 <= STAGES * STAGE_BYTES, "the z tile is staged in the stage ring");

struct Tc2Params {
  uint32_t n_cols;
  uint32_t x_rows;
  uint32_t kb_total;
  uint32_t kb_half;
  const uint32_t* col_tags;
  uint64_t seed_own, seed_prev;
  uint32_t vec;
  uint16_t* z;
  uint64_t ldz;
  uint64_t row0;
  uint32_t* status;
};

__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t a, uint64_t b) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(1u)
      : "memory");
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
    gemm_tc2_kernel(const __grid_constant__ CUtensorMap tb_lo, const __grid_constant__ CUtensorMap tb_hi,
                    const __grid_constant__ CUtensorMap ta0_lo, const __grid_constant__ CUtensorMap ta0_hi,
                    const __grid_constant__ CUtensorMap ta1_lo, const __grid_constant__ CUtensorMap ta1_hi,
                    const Tc2Params p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ uint32_t s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t tiles = smem_addr(smem);
  const uint32_t bars = tiles + STAGES * STAGE_BYTES + SLACK;
  const uint32_t full0 = bars, empty0 = bars + 8 * STAGES;
  const uint32_t c_full = bars + 16 * STAGES, c_empty = c_full + 8, l_full = c_full + 16, l_empty = c_full + 24,
                 done_bar = c_full + 32;
  volatile uint32_t* abort = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t q0 = (blockIdx.x >> 1) * TN;             // the pair's first query column
  const uint32_t qh = q0 + rank * HN;                      // this CTA's half of the query tile
  const uint32_t d0 = blockIdx.y * (2 * TM) + rank * TM;   // this CTA's database rows
  const uint32_t n_chunks = p.kb_total / KB_PER_CHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(c_full, 1);
    mbar_init(c_empty, 2 * DRAIN_THREADS / 32);
    mbar_init(l_full, 1);
    mbar_init(l_empty, 2 * DRAIN_THREADS / 32);
    mbar_init(done_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    // one warp of each CTA of the pair allocates, collectively, the same columns in both
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers are initialised before any remote arrive or TMA
  fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    // ------------------------------- TMA producers ------------------------------
    if (lane == 0) {
      uint32_t issued = 0;
      for (uint32_t kb = 0; kb < p.kb_total; ++kb) {
        const uint32_t s = kb % STAGES;
        if (!mbar_wait(empty0 + 8 * s, ((kb / STAGES) & 1u) ^ 1u, p.status, abort)) break;
        const uint32_t full_own = full0 + 8 * s, base = tiles + s * STAGE_BYTES;
        if (leader) mbar_expect_tx(full_own, 2 * STAGE_BYTES);  // both CTAs' halves
        const uint32_t full = peer_addr(full_own, 0);
        const bool first = kb < p.kb_half;
        const int32_t kx = static_cast<int32_t>((first ? kb : kb - p.kb_half) * KB);
        tma_load_pair(base, first ? &ta0_lo : &ta1_lo, kx, static_cast<int32_t>(d0), full);
        tma_load_pair(base + TILE_BYTES, first ? &ta0_hi : &ta1_hi, kx, static_cast<int32_t>(d0), full);
        tma_load_pair(base + 2 * TILE_BYTES, &tb_lo, static_cast<int32_t>(kb * KB), static_cast<int32_t>(qh), full);
        tma_load_pair(base + 3 * TILE_BYTES, &tb_hi, static_cast<int32_t>(kb * KB), static_cast<int32_t>(qh), full);
        issued = kb + 1;
      }
      if (*abort) {
        // this CTA's copies still in flight complete before it goes on (bounded): they are
        // counted on the leader's barriers, so wait for this CTA's stage-empty phases instead
        for (uint32_t kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
          mbar_wait(empty0 + 8 * (kb % STAGES), (kb / STAGES) & 1u, p.status, nullptr);
      }
    }
  } else if (warp == 1) {
    // --------------------------- MMA issuer (leader only) ---------------------------
    if (leader && lane == 0) {
      const uint32_t tL = tmem, tC = tmem + TN;
      // C of k-block j with L of k-block j - 1: C0 C1 L0 C2 L1 C3 [C-full] L2 L3 (as gemm_tc.cu)
      auto issue_c = [&](uint32_t base) {
#pragma unroll
        for (uint32_t ks = 0; ks < KB / 16; ++ks) {
          const uint32_t o = 32u * ks;
          umma_pair(tC, sdesc(base + o), sdesc(base + 3 * TILE_BYTES + o));               // lo * hi'
          umma_pair(tC, sdesc(base + TILE_BYTES + o), sdesc(base + 2 * TILE_BYTES + o));  // hi * lo'
        }
      };
      auto issue_l = [&](uint32_t kb) {
        const uint32_t s = kb % STAGES, base = tiles + s * STAGE_BYTES;
#pragma unroll
        for (uint32_t ks = 0; ks < KB / 16; ++ks) {
          const uint32_t o = 32u * ks;
          umma_pair(tL, sdesc(base + o), sdesc(base + 2 * TILE_BYTES + o));  // lo * lo'
        }
        umma_commit_pair(empty0 + 8 * s);  // both CTAs' stage s free once these MMAs are done
      };
      for (uint32_t c = 0; c < n_chunks; ++c) {
        const uint32_t par = c & 1u, G0 = c * KB_PER_CHUNK;
        const bool l_opens = (c & 1u) == 0, l_closes = (c & 1u) == 1;
        if (!mbar_wait(c_empty, par, p.status, abort)) break;
        fence_after();
        bool ok = true;
        for (uint32_t kb = 0; kb < KB_PER_CHUNK; ++kb) {
          const uint32_t G = G0 + kb, s = G % STAGES;
          if (!mbar_wait(full0 + 8 * s, (G / STAGES) & 1u, p.status, abort)) {
            ok = false;
            break;
          }
          fence_after();
          issue_c(tiles + s * STAGE_BYTES);
          if (kb == KB_PER_CHUNK - 1) umma_commit_pair(c_full);
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
        if (l_closes) umma_commit_pair(l_full);
      }
      umma_commit_pair(done_bar);
      mbar_wait(done_bar, 0, p.status, nullptr);
    }
  } else {
    // ----------------------------------- drain ----------------------------------
    const uint32_t q = static_cast<uint32_t>(warp) & 3u, h = static_cast<uint32_t>(warp - 2) >> 2;
    const uint32_t tL = tmem + ((32u * q) << 16) + DCOLS * h, tC = tL + TN;
    // the empty barriers the MMA issuer waits on are the leader's
#pragma unroll
    for (uint32_t g = 0; g < GROUPS; ++g) {
      tmem_fill32(tL + 32 * g, MAGIC);
      tmem_fill32(tC + 32 * g, MAGIC);
    }
    tmem_wait_st();
    fence_before();
    __syncwarp();
    if (lane == 0) {
      arrive_leader(c_empty, leader);
      arrive_leader(l_empty, leader);
    }
    uint32_t z2[DCOLS / 2];
#pragma unroll
    for (int k = 0; k < DCOLS / 2; ++k) z2[k] = 0;
    for (uint32_t cc = 0; cc < n_chunks; ++cc) {
      const uint32_t par = cc & 1u;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(c_full, par, p.status, abort))) break;
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
      if (lane == 0) arrive_leader(c_empty, leader);
      if ((cc & 1u) == 0) continue;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(l_full, (cc >> 1) & 1u, p.status, abort))) break;
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
      if (lane == 0) arrive_leader(l_empty, leader);
    }
    // ---- epilogue: z + r_i (App. C), through the idle stage ring as in gemm_tc.cu ----
    named_sync(1, DRAIN_THREADS);
    if (!*abort) {
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
      const uint32_t ctr3 = (IPC_D_ZA << 24) | p.vec;
      for (uint32_t it = dt; it < TN * (TM / 8); it += DRAIN_THREADS) {
        const uint32_t cc = it / (TM / 8), g = it % (TM / 8), col = q0 + cc, r0 = d0 + 8 * g;
        if (col >= p.n_cols || r0 >= p.x_rows) continue;
        const uint32_t req = p.col_tags[2 * col], tag = p.col_tags[2 * col + 1];
        const uint4 fo = philox(grp0 + g, tag, req, ctr3, p.seed_own);
        const uint4 fp = philox(grp0 + g, tag, req, ctr3, p.seed_prev);
        const uint4 acc = *reinterpret_cast<const uint4*>(zs + cc * TM + 8 * g);
        auto add2 = [](uint32_t a, uint32_t o, uint32_t f) {
          const uint32_t lo = (a + o - f) & 0xFFFFu;
          const uint32_t hi = ((a >> 16) + (o >> 16) - (f >> 16)) << 16;
          return lo | hi;
        };
        const uint4 v = make_uint4(add2(acc.x, fo.x, fp.x), add2(acc.y, fo.y, fp.y), add2(acc.z, fo.z, fp.z),
                                   add2(acc.w, fo.w, fp.w));
        uint16_t* dst = p.z + static_cast<uint64_t>(col) * p.ldz + r0;
        if (r0 + 8 <= p.x_rows) {
          *reinterpret_cast<uint4*>(dst) = v;
        } else {
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
          for (uint32_t e = 0; e < p.x_rows - r0; ++e) dst[e] = static_cast<uint16_t>(w[e >> 1] >> (16 * (e & 1)));
        }
      }
    }
  }
  // the pair's MMAs are complete (the leader's issuer waited for them) before either frees
  // tensor memory or leaves
  fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

// The fixed-shape ring GEMM of ring_gemm_tc_variant (256-column tiles) on CTA pairs: one
// cluster of two CTAs per 256-row x 256-column tile. segments as there.
int ring_gemm_tc_pair(uint32_t segments, const uint16_t* const x_lo[2], const uint16_t* const x_hi[2], size_t x_rows,
                      const uint16_t* b_lo, const uint16_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                      const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z,
                      size_t ldz, uint64_t row0, cudaStream_t stream) {
  if (segments != 1 && segments != 2) {
    set_error("tcgen05 pair GEMM: one or two K segments");
    return IPC_EINVAL;
  }
  if ((segments * l) % (2 * KB_PER_CHUNK * KB) != 0) {
    set_error("tcgen05 pair GEMM: K must be a multiple of 256");
    return IPC_EINVAL;
  }
  if (n_pad % 128 != 0 || n_cols > n_pad) {
    set_error("tcgen05 pair GEMM: n_pad must be a multiple of 128 and at least n_cols");
    return IPC_EINVAL;
  }
  if (x_rows == 0 || n_cols == 0) return IPC_OK;
  if ((x_rows + 2 * TM - 1) / (2 * TM) > 65535) {
    set_error("tcgen05 pair GEMM: too many rows for one launch");
    return IPC_EINVAL;
  }
  CUtensorMap m[6];
  int rc;
  if ((rc = make_map_bf16(&m[0], b_lo, static_cast<uint64_t>(segments) * l, n_pad, HN)) ||
      (rc = make_map_bf16(&m[1], b_hi, static_cast<uint64_t>(segments) * l, n_pad, HN)) ||
      (rc = make_map_bf16(&m[2], x_lo[0], l, x_rows, TM)) || (rc = make_map_bf16(&m[3], x_hi[0], l, x_rows, TM)) ||
      (rc = make_map_bf16(&m[4], x_lo[1], l, x_rows, TM)) || (rc = make_map_bf16(&m[5], x_hi[1], l, x_rows, TM)))
    return rc;
  Tc2Params p;
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
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(gemm_tc2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  IPC_CUDA_TRY(attr);
  // x: two CTAs (one cluster) per 256-column tile; y: 256-row pair tiles
  const dim3 grid(2 * ((n_cols + TN - 1) / TN), static_cast<unsigned>((x_rows + 2 * TM - 1) / (2 * TM)));
  gemm_tc2_kernel<<<grid, THREADS, SMEM_BYTES, stream>>>(m[0], m[1], m[2], m[3], m[4], m[5], p);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

}  // namespace ipc
