// Device code of the comparison phase (A4-A8, Alg. 3 and App. D), shared by the stand-alone
// comparison kernel and the fused GEMM + comparison kernel: the boolean sharing of 32 lanes, the
// App. C AND gate, the PRF words of the gates, BitExtract, the bit transpose, and the root of one
// part of a (column, OR block) unit -- the comparisons of up to four 32-row words and the OR
// tree over them. Both kernels call the same part routine with the same gate numbering, so
// their shares are equal by construction.
#pragma once

#include "common.cuh"

namespace ipc {
namespace cmp {

constexpr int LIFT_GATE0 = 0;  // 33 gates (17 full-adder layer, 16 ripple)
constexpr int MSB_GATE0 = 36;  // 61 gates (31 full-adder layer, 30 ripple)

struct B3 {
  uint32_t c0, c1, c2;  // components of a boolean sharing of 32 lanes
};

__device__ __forceinline__ B3 bx(const B3& a, const B3& b) { return {a.c0 ^ b.c0, a.c1 ^ b.c1, a.c2 ^ b.c2}; }

// App. C product over F_2, each party from its own view plus alpha_p = F_p ^ F_{p-1}.
__device__ __forceinline__ B3 band(const B3& x, const B3& y, uint32_t F0, uint32_t F1, uint32_t F2) {
  B3 z;
  z.c0 = (x.c0 & y.c0) ^ (x.c0 & y.c2) ^ (x.c2 & y.c0) ^ F0 ^ F2;
  z.c1 = (x.c1 & y.c1) ^ (x.c1 & y.c0) ^ (x.c0 & y.c1) ^ F1 ^ F0;
  z.c2 = (x.c2 & y.c2) ^ (x.c2 & y.c1) ^ (x.c1 & y.c2) ^ F2 ^ F1;
  return z;
}

struct Seeds {
  uint64_t s[3];
};

// Zero-share words of the AND gates of one 32-row word: gate G uses word (G & 3) of
// Philox(seed_j, (g >> 5, tag, req, D_AND << 24 | G >> 2)).
struct GateRng {
  uint32_t c0, tag, req;
  uint4 w[3];
  __device__ __forceinline__ void refresh(const Seeds& sd, uint32_t quad) {
#pragma unroll
    for (int j = 0; j < 3; ++j) w[j] = philox(c0, tag, req, (IPC_D_AND << 24) | quad, sd.s[j]);
  }
  __device__ __forceinline__ void get(const Seeds& sd, uint32_t gate, bool first, uint32_t& F0, uint32_t& F1,
                                      uint32_t& F2) {
    if (first || (gate & 3u) == 0) refresh(sd, gate >> 2);
    F0 = word_of(w[0], gate & 3u);
    F1 = word_of(w[1], gate & 3u);
    F2 = word_of(w[2], gate & 3u);
  }
};

// BitExtract(x, {M, M-1}) over bit-sliced inputs: X(j, b) is word b of component j
// (b > top_in gives 0). Full-adder layer on positions 0..M-1 (gates G0 + b), the sum
// only at position M; ripple BinAdd of (carries << 1) and sums, positions 1..M-1 with
// gates G0 + M + b - 1; r[M] = a ^ s ^ carry. Both layers are streamed by position, in a
// loop unrolled 4 times (one PRF refresh per layer per pass): against full unrolling, the
// kernel's instructions stay in the SM's instruction cache and its registers drop from about
// 250 to 128-160, at 6-13 % less time per comparison in every mode.
template <int M, int G0, typename Xf>
__device__ __forceinline__ void bit_extract(const Seeds& sd, GateRng& fa, GateRng& rc, Xf X, B3& top, B3& below) {
  // full adder of position b: sum s (local) and carry c (one AND)
  auto full_adder = [&](uint32_t b, bool first, B3& s, B3& c) {
    const B3 x0 = {X(0, b), 0u, 0u}, x1 = {0u, X(1, b), 0u}, x2 = {0u, 0u, X(2, b)};
    const B3 t1 = bx(x0, x2), t2 = bx(x1, x2);
    s = bx(t1, x1);
    uint32_t F0, F1, F2;
    fa.get(sd, G0 + b, first, F0, F1, F2);
    c = bx(band(t1, t2, F0, F1, F2), x2);
  };
  B3 carry = {0u, 0u, 0u}, cprev, s;
  full_adder(0u, true, s, cprev);
  below = M == 1 ? s : B3{0u, 0u, 0u};
#pragma unroll 4
  for (uint32_t b = 1; b < static_cast<uint32_t>(M); ++b) {
    B3 c;
    full_adder(b, false, s, c);
    const B3 t1 = bx(cprev, carry), t2 = bx(s, carry);
    const B3 sum = bx(t1, s);
    uint32_t F0, F1, F2;
    rc.get(sd, G0 + M + b - 1, b == 1, F0, F1, F2);
    carry = bx(band(t1, t2, F0, F1, F2), carry);
    if (b == static_cast<uint32_t>(M) - 1) below = sum;
    cprev = c;
  }
  const B3 sM = {X(0, M), X(1, M), X(2, M)};
  top = bx(bx(cprev, sM), carry);
}

// In-register 32x32 bit transpose: afterwards bit i of a[j] is the former bit j of a[i].
__device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int j = 16 >> st;
    const uint32_t m = masks[st];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & j) continue;
      const uint32_t t = ((a[k] >> j) ^ a[k + j]) & m;
      a[k] ^= t << j;
      a[k + j] ^= t;
    }
  }
}

struct CmpParams {
  const uint16_t* zc[3];
  const uint16_t* zm[3];
  uint64_t ldz;
  uint32_t n_cols;
  uint64_t n_rows;
  uint64_t row0;
  const uint32_t* col_tags;
  Seeds seeds;
  uint32_t thr_a;
  uint32_t p;  // log2 words per block
  uint32_t n_blocks;
  uint32_t* roots;
  uint64_t ld_roots;
  uint8_t* msb_out;
  uint64_t ld_msb;
  const uint32_t* col_tiles;   // optional device list of tile_cols-wide column tiles
  const uint32_t* n_col_list;  // its length (device)
  uint32_t tile_cols;
  const uint32_t* col_rows;    // optional per column: global rows >= col_rows[n] are the public 0
  // lift-free comparison (ConstLift / NoLift): ml components over Z_2^32, and the dot's either
  // over Z_2^32 (zc32, NoLift, times thr_b) or over Z_2^16 (zc, ConstLift, times 2^16)
  const uint32_t* zm32[3];
  const uint32_t* zc32[3];
  uint32_t thr_b;
};

constexpr int MODE_LIFT = 0, MODE_PLAIN = 1, MODE_LIFTFREE = 2;

// 2^ks threads share one (column, OR block), ks = min(LOG2_SPLIT, p): thread t takes the t-th
// part of the block's words (a level sub_p = p - ks subtree) and the group joins the parts
// pairwise with the block's upper ks levels of OR gates. Gate indices are global node indices
// at each level, so the tree and every share are the same as one thread walking the whole
// block. With 1,024-row blocks each thread takes 4 words.
constexpr uint32_t LOG2_SPLIT = 3;

// Shared memory per thread (index [slot][threadIdx.x], conflict-free): X, 3 x 32 words (per
// component: the lift input bit-slices in words 0..15 and the raw ml pairs in words 16..31,
// then the 32 rows of v and their bit-slices); the OR stack, 3 x (levels 0..5 - LOG2_SPLIT).
constexpr int S_X = 0, S_STK = 96, S_WORDS = S_STK + 3 * (6 - static_cast<int>(LOG2_SPLIT));

__device__ __forceinline__ B3 bor(const Seeds& sd, const B3& a, const B3& b, uint32_t j, uint32_t tag, uint32_t req,
                                  uint32_t c3) {
  const uint32_t F0 = philox(j, tag, req, c3, sd.s[0]).x;
  const uint32_t F1 = philox(j, tag, req, c3, sd.s[1]).x;
  const uint32_t F2 = philox(j, tag, req, c3, sd.s[2]).x;
  return bx(bx(a, b), band(a, b, F0, F1, F2));
}

// The 32 u16 values of rows 0..31 of a column as 16 words of two (rows past nvalid read 0).
__device__ __forceinline__ void load_pairs(const uint16_t* p, uint32_t nvalid, uint32_t (&w)[16]) {
  if (nvalid == 32) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const uint4 q = reinterpret_cast<const uint4*>(p)[v];
      w[4 * v + 0] = q.x;
      w[4 * v + 1] = q.y;
      w[4 * v + 2] = q.z;
      w[4 * v + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int v = 0; v < 16; ++v) {
      const uint32_t r0 = 2 * v, r1 = 2 * v + 1;
      w[v] = (r0 < nvalid ? static_cast<uint32_t>(p[r0]) : 0u) | ((r1 < nvalid ? static_cast<uint32_t>(p[r1]) : 0u) << 16);
    }
  }
}

// Rows l and l+1 of a column as one word (rows past nvalid read 0).
__device__ __forceinline__ uint32_t load_pair(const uint16_t* p, uint32_t l, uint32_t nvalid) {
  if (nvalid == 32) return *reinterpret_cast<const uint32_t*>(p + l);
  return (l < nvalid ? static_cast<uint32_t>(p[l]) : 0u) | ((l + 1 < nvalid ? static_cast<uint32_t>(p[l + 1]) : 0u) << 16);
}

// MODE_LIFT (Alg. 3): Lift of ml, ConstLift of dot, v = a ml' - 2^16 dot', BitExtract(v, {31}).
// MODE_PLAIN (protocol 1, Sec. 4, Alg. 2): zm[0] holds the public ml of each comparison (all three
// pointers may point to it); v = floor(a ml / 2^16) - dot over Z_{2^16}, the public term entering
// component 0, and the match bit is BitExtract(v, {15}) (29 ANDs, gates from 0).
// MODE_LIFTFREE (ConstLift / NoLift, Sec. 5.1, Sec. 6.2): ml already shared over Z_{2^32}, so
// v = a ml - b dot over Z_{2^32} directly and BitExtract(v, {31}) (61 ANDs, the MSB gates).
// The root of part `part` of the unit (column n, OR block blk): the comparisons of the part's
// words and the OR tree over them (a level sub_p = P.p - ks subtree of the block's tree; a
// ragged part is flushed upwards with the node indices of the full tree). The scratch of this
// thread is sm[slot * STRIDE + tid] for slots [0, S_WORDS). nwords_out: the part's word count
// (0: the part lies past the last row and root is the public 0).
template <int MODE, int STRIDE>
__device__ __forceinline__ void part_root(const CmpParams& P, uint32_t n, uint32_t blk, uint32_t part, uint32_t ks,
                                          uint32_t* sm, uint32_t tid, B3& root, uint32_t& nwords_out) {
  auto S = [&](int slot) -> uint32_t& { return sm[slot * STRIDE + tid]; };
  const uint32_t req = P.col_tags[2 * n], tag = P.col_tags[2 * n + 1];
  const uint32_t words_per_block = 1u << P.p;
  const uint64_t blk_row = static_cast<uint64_t>(blk) << (5 + P.p);  // local first row of this block
  const uint64_t rem_words = (P.n_rows - blk_row + 31) >> 5;
  const uint32_t blk_words = static_cast<uint32_t>(rem_words < words_per_block ? rem_words : words_per_block);
  const uint64_t bword0 = (P.row0 + blk_row) >> 5;  // global index of the block's first word
  // this thread's part: words [w_begin, w_end) of the block, a level sub_p subtree
  const uint32_t sub_p = P.p - ks;
  const uint32_t w_begin = part << sub_p;
  const uint32_t w_lim = (part + 1) << sub_p;
  const uint32_t w_end = blk_words < w_lim ? blk_words : w_lim;
  const uint32_t nwords = w_end > w_begin ? w_end - w_begin : 0u;
  const uint64_t gword0 = bword0 + w_begin;

  uint32_t valid_levels = 0;
  for (uint32_t w = 0; w < nwords; ++w) {
    const uint64_t lrow = blk_row + 32ull * (w_begin + w);
    const uint64_t grow = P.row0 + lrow;
    const uint32_t nvalid = static_cast<uint32_t>(P.n_rows - lrow < 32 ? P.n_rows - lrow : 32);
    const uint32_t lane_mask = nvalid == 32 ? 0xFFFFFFFFu : ((1u << nvalid) - 1u);
    const uint64_t coff = static_cast<uint64_t>(n) * P.ldz + lrow;
    B3 msb, b30;
    if constexpr (MODE == MODE_LIFTFREE) {
      // ---- v = a ml - b dot over Z_{2^32}, straight from the loads; bit-slice; MSB ----
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const uint32_t* pm = P.zm32[j] + coff;
        if (nvalid == 32) {
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const uint4 a = reinterpret_cast<const uint4*>(pm)[v];
            S(S_X + 32 * j + 4 * v + 0) = P.thr_a * a.x;
            S(S_X + 32 * j + 4 * v + 1) = P.thr_a * a.y;
            S(S_X + 32 * j + 4 * v + 2) = P.thr_a * a.z;
            S(S_X + 32 * j + 4 * v + 3) = P.thr_a * a.w;
          }
        } else {
          for (uint32_t l = 0; l < 32; ++l) S(S_X + 32 * j + l) = l < nvalid ? P.thr_a * pm[l] : 0u;
        }
        if (P.zc32[0]) {  // NoLift: dot components over Z_{2^32}, times b
          const uint32_t* pd = P.zc32[j] + coff;
          if (nvalid == 32) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
              const uint4 d = reinterpret_cast<const uint4*>(pd)[v];
              S(S_X + 32 * j + 4 * v + 0) -= P.thr_b * d.x;
              S(S_X + 32 * j + 4 * v + 1) -= P.thr_b * d.y;
              S(S_X + 32 * j + 4 * v + 2) -= P.thr_b * d.z;
              S(S_X + 32 * j + 4 * v + 3) -= P.thr_b * d.w;
            }
          } else {
            for (uint32_t l = 0; l < nvalid; ++l) S(S_X + 32 * j + l) -= P.thr_b * pd[l];
          }
        } else {  // ConstLift: each Z_{2^16} component read as an integer, times 2^16
          uint32_t d[16];
          load_pairs(P.zc[j] + coff, nvalid, d);
#pragma unroll
          for (int v = 0; v < 16; ++v) {
            S(S_X + 32 * j + 2 * v) -= d[v] << 16;
            S(S_X + 32 * j + 2 * v + 1) -= d[v] & 0xFFFF0000u;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        uint32_t a[32];
#pragma unroll
        for (int v = 0; v < 32; ++v) a[v] = S(S_X + 32 * j + v);
        transpose32(a);
#pragma unroll
        for (int v = 0; v < 32; ++v) S(S_X + 32 * j + v) = a[v];
      }
      GateRng fa{static_cast<uint32_t>(grow >> 5), tag, req, {}}, rc{static_cast<uint32_t>(grow >> 5), tag, req, {}};
      bit_extract<31, MSB_GATE0>(P.seeds, fa, rc, [&](int j, int b) -> uint32_t { return S(S_X + 32 * j + b); }, msb,
                                 b30);
    } else if constexpr (MODE == MODE_PLAIN) {
      // ---- v = t - dot, t = floor(a ml / 2^16) public (component 0); bit-slice; MSB of 16 bits ----
      uint32_t mlw[16];
      load_pairs(P.zm[0] + coff, nvalid, mlw);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        uint32_t dw[16];
        load_pairs(P.zc[j] + coff, nvalid, dw);
        uint32_t a[32];
#pragma unroll
        for (int l = 0; l < 32; ++l) {
          const uint32_t ml = (mlw[l >> 1] >> (16 * (l & 1))) & 0xFFFFu;
          const uint32_t dt = (dw[l >> 1] >> (16 * (l & 1))) & 0xFFFFu;
          a[l] = ((j == 0 ? (P.thr_a * ml) >> 16 : 0u) - dt) & 0xFFFFu;
        }
        transpose32(a);
#pragma unroll
        for (int v = 0; v < 16; ++v) S(S_X + 32 * j + v) = a[v];
      }
      GateRng fa{static_cast<uint32_t>(grow >> 5), tag, req, {}}, rc{static_cast<uint32_t>(grow >> 5), tag, req, {}};
      bit_extract<15, 0>(P.seeds, fa, rc, [&](int j, int b) -> uint32_t { return S(S_X + 32 * j + b); }, msb, b30);
    } else {
      // ---- ShareSplit of ml: bit-slice each component (bits 0..15); keep its raw pairs ----
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        uint32_t raw[16];
        load_pairs(P.zm[j] + coff, nvalid, raw);
        uint32_t a[32];
#pragma unroll
        for (int v = 0; v < 16; ++v) {
          S(S_X + 32 * j + 16 + v) = raw[v];
          a[2 * v] = raw[v] & 0xFFFFu;
          a[2 * v + 1] = raw[v] >> 16;
        }
        transpose32(a);
#pragma unroll
        for (int b = 0; b < 16; ++b) S(S_X + 32 * j + b) = a[b];
      }
      // the dot is read from global one row pair ahead of its use
      const uint16_t* pd[3] = {P.zc[0] + coff, P.zc[1] + coff, P.zc[2] + coff};
      uint32_t dnext[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) dnext[j] = load_pair(pd[j], 0u, nvalid);
      GateRng fa{static_cast<uint32_t>(grow >> 5), tag, req, {}}, rc{static_cast<uint32_t>(grow >> 5), tag, req, {}};
      B3 r17, r16;
      bit_extract<17, LIFT_GATE0>(
          P.seeds, fa, rc, [&](int j, int b) -> uint32_t { return b < 16 ? S(S_X + 32 * j + b) : 0u; }, r17, r16);
      // ---- per comparison: BitInject (3-party OT), ConstLift, v = a*ml' - 2^16*dot ----
      // Row pair (l, l+1) reads raw ml word 16 + l/2 of each component before writing v to
      // words l and l+1; those overwrite raw words l-16 and l-15 <= l/2 only once they are read.
      uint4 q0w = make_uint4(0u, 0u, 0u, 0u);  // D_INJ0 words: one Philox call per 4 rows
#pragma unroll 1
      for (uint32_t l = 0; l < 32; l += 2) {
        uint32_t dcur[3], mlw[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          dcur[j] = dnext[j];
          mlw[j] = S(S_X + 32 * j + 16 + (l >> 1));
        }
        if (l + 2 < 32) {
#pragma unroll
          for (int j = 0; j < 3; ++j) dnext[j] = load_pair(pd[j], l + 2, nvalid);
        }
#pragma unroll
        for (uint32_t e = 0; e < 2; ++e) {
          const uint32_t r = l + e;
          const uint64_t g = grow + r;
          if ((r & 3u) == 0) q0w = philox(static_cast<uint32_t>(g >> 2), tag, req, IPC_D_INJ0 << 24, P.seeds.s[0]);
          const uint32_t inj0 = word_of(q0w, r & 3u);
          const uint4 w2 = philox(static_cast<uint32_t>(g), tag, req, IPC_D_INJ2 << 24, P.seeds.s[2]);
          uint32_t A[3], Bv[3];
#pragma unroll
          for (int which = 0; which < 2; ++which) {
            const uint32_t k = which == 0 ? 15u : 16u;
            const uint32_t mask = (1u << k) - 1u;
            const uint32_t sh = which == 0 ? 0u : 16u;
            const B3& bit = which == 0 ? r17 : r16;
            const uint32_t x0 = (bit.c0 >> r) & 1u, x1 = (bit.c1 >> r) & 1u, x2 = (bit.c2 >> r) & 1u;
            const uint32_t c0 = (inj0 >> sh) & mask, c2 = (w2.x >> sh) & mask;
            const uint32_t w0 = (w2.y >> sh) & mask, w1 = (w2.z >> sh) & mask;
            // party 0 (OT sender): m_beta = (beta ^ x_0 ^ x_2) - c_0 - c_2, masked k_beta = w_beta ^ m_beta
            const uint32_t m0 = ((0u ^ x0 ^ x2) - c0 - c2) & mask;
            const uint32_t m1 = ((1u ^ x0 ^ x2) - c0 - c2) & mask;
            const uint32_t k0 = w0 ^ m0, k1 = w1 ^ m1;
            // party 2 (helper) sends w_{x_1}; party 1 (receiver) unmasks k_{x_1}
            const uint32_t wsel = x1 ? w1 : w0;
            const uint32_t c1 = (wsel ^ (x1 ? k1 : k0)) & mask;
            uint32_t* out = which == 0 ? A : Bv;
            out[0] = c0;
            out[1] = c1;
            out[2] = c2;
          }
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const uint32_t ml = (mlw[j] >> (16 * e)) & 0xFFFFu, dt = (dcur[j] >> (16 * e)) & 0xFFFFu;
            const uint32_t mll = ml - (A[j] << 17) - (Bv[j] << 16);
            S(S_X + 32 * j + r) = P.thr_a * mll - (dt << 16);
          }
        }
      }
      // ---- MSB: bit-slice v and BitExtract(v, {31}) ----
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        uint32_t a[32];
#pragma unroll
        for (int v = 0; v < 32; ++v) a[v] = S(S_X + 32 * j + v);
        transpose32(a);
#pragma unroll
        for (int v = 0; v < 32; ++v) S(S_X + 32 * j + v) = a[v];
      }
      GateRng fa2{static_cast<uint32_t>(grow >> 5), tag, req, {}}, rc2{static_cast<uint32_t>(grow >> 5), tag, req, {}};
      bit_extract<31, MSB_GATE0>(P.seeds, fa2, rc2, [&](int j, int b) -> uint32_t { return S(S_X + 32 * j + b); },
                                 msb, b30);
    }
    // rows past the end (and, with col_rows, rows past the column's limit) are the public 0
    // of the OR tree
    uint32_t keep = lane_mask;
    if (P.col_rows) {
      const uint64_t lim = P.col_rows[n];
      keep &= lim <= grow ? 0u : (lim - grow >= 32 ? 0xFFFFFFFFu : ((1u << (lim - grow)) - 1u));
    }
    msb.c0 &= keep;
    msb.c1 &= keep;
    msb.c2 &= keep;
    if (P.msb_out) {
      for (uint32_t l = 0; l < nvalid; ++l) {
        const uint64_t at = static_cast<uint64_t>(n) * P.ld_msb + lrow + l;
        const uint64_t plane = static_cast<uint64_t>(P.n_cols) * P.ld_msb;
        P.msb_out[at] = (msb.c0 >> l) & 1u;
        P.msb_out[plane + at] = (msb.c1 >> l) & 1u;
        P.msb_out[2 * plane + at] = (msb.c2 >> l) & 1u;
      }
    }
    // ---- OR tree inside this part (binary counter over word indices) ----
    B3 cur = msb;
    uint64_t idx = gword0 + w;
    uint32_t lvl = 0;
    while (lvl < sub_p && (idx & 1u) && (valid_levels >> lvl & 1u)) {
      const B3 left = {S(S_STK + 3 * lvl), S(S_STK + 3 * lvl + 1), S(S_STK + 3 * lvl + 2)};
      cur = bor(P.seeds, left, cur, static_cast<uint32_t>(idx >> 1), tag, req,
                (IPC_D_OR << 24) | (1u << 16) | (lvl + 1));
      valid_levels &= ~(1u << lvl);
      ++lvl;
      idx >>= 1;
    }
    S(S_STK + 3 * lvl) = cur.c0;
    S(S_STK + 3 * lvl + 1) = cur.c1;
    S(S_STK + 3 * lvl + 2) = cur.c2;
    valid_levels |= 1u << lvl;
  }
  // ---- root of this part: a full part ends at level sub_p; a ragged one is flushed upwards ----
  root = {0u, 0u, 0u};
  if (valid_levels >> sub_p & 1u) {
    root = {S(S_STK + 3 * sub_p), S(S_STK + 3 * sub_p + 1), S(S_STK + 3 * sub_p + 2)};
  } else {
    bool have = false;
    uint64_t idx = 0;
    for (uint32_t lvl = 0; lvl < sub_p; ++lvl) {
      if (have) {
        if (valid_levels >> lvl & 1u) {
          const B3 left = {S(S_STK + 3 * lvl), S(S_STK + 3 * lvl + 1), S(S_STK + 3 * lvl + 2)};
          root = bor(P.seeds, left, root, static_cast<uint32_t>(idx >> 1), tag, req,
                     (IPC_D_OR << 24) | (1u << 16) | (lvl + 1));
        }
        idx >>= 1;
      } else if (valid_levels >> lvl & 1u) {
        root = {S(S_STK + 3 * lvl), S(S_STK + 3 * lvl + 1), S(S_STK + 3 * lvl + 2)};
        // index of this entry at level lvl: its words start after the higher entries of the part
        const uint64_t cnt = nwords;
        const uint64_t start = gword0 + (cnt & ~((2ull << lvl) - 1ull));
        idx = start >> lvl;
        have = true;
        idx >>= 1;
      }
    }
  }
  nwords_out = nwords;
}

}  // namespace cmp
}  // namespace ipc
