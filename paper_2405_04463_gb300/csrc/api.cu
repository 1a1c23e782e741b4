// Stage-level C entry points: argument checks, then the kernels of gemm_i8.cu, gemm_i32.cu
// and compare.cu.
#include <string>

#include "common.cuh"

namespace ipc {
int ring_gemm_i8(int mode, const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows, const int8_t* b_lo,
                 const int8_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags,
                 uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                 cudaStream_t stream);
int ring_gemm_i8_variant(int variant, const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows,
                         const int8_t* b_lo, const int8_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                         const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z,
                         size_t ldz, uint64_t row0, const uint32_t* col_tiles, const uint32_t* n_col_list,
                         cudaStream_t stream);
int ring_gemm_i32(const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows, const int8_t* b_lo,
                  const int8_t* b_hi, uint32_t n_cols, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                  uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0, cudaStream_t stream);
int compare_launch(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz, uint32_t n_cols,
                   size_t n_rows, uint64_t row0, const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a,
                   uint32_t p, uint32_t* roots, size_t ld_roots, uint8_t* msb_out, size_t ld_msb, cudaStream_t st);
int compare_launch_tiles(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz,
                         uint32_t n_cols, size_t n_rows, uint64_t row0, const uint32_t* col_tags,
                         const uint64_t seeds[3], uint32_t thr_a, uint32_t p, uint32_t* roots, size_t ld_roots,
                         uint8_t* msb_out, size_t ld_msb, const uint32_t* col_tiles, const uint32_t* n_col_list,
                         uint32_t tile_cols, cudaStream_t st, const uint32_t* col_rows, bool plain);
int compare_launch_liftfree(const uint16_t* const zc16[3], const uint32_t* const zc32[3],
                            const uint32_t* const ml32[3], size_t ldz, uint32_t n_cols, size_t n_rows, uint64_t row0,
                            const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a, uint32_t thr_b,
                            uint32_t p, uint32_t* roots, size_t ld_roots, uint8_t* msb_out, size_t ld_msb,
                            cudaStream_t st);
int or_finalize_launch(uint32_t* roots, size_t ld_roots, uint32_t n_blocks, uint32_t p, uint32_t Q, uint32_t R,
                       const uint32_t* col_tags, const uint64_t seeds[3], uint8_t* bit_shares, cudaStream_t st);
int ring_gemm_tc(const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows, const uint16_t* b_lo,
                 const uint16_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags,
                 uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                 cudaStream_t stream);
int ring_gemm_tc_variant(uint32_t tile_cols, uint32_t segments, const int8_t* const x_lo[2],
                         const int8_t* const x_hi[2], size_t x_rows, const uint16_t* b_lo, const uint16_t* b_hi,
                         uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                         uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                         const uint32_t* col_tiles, const uint32_t* n_col_list, cudaStream_t stream);
const char* thread_last_error();

namespace {
bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }
int bad(const char* msg) {
  set_error(msg);
  return IPC_EINVAL;
}
}  // namespace
}  // namespace ipc

using namespace ipc;

extern "C" int ipc_ring_gemm(int path, const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows,
                             const int8_t* b_lo, const int8_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                             const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec,
                             uint16_t* z, size_t ldz, uint64_t row0, void* stream) {
  if (!x_lo || !x_hi || !b_lo || !b_hi || !col_tags || !z) return bad("ipc_ring_gemm: null pointer");
  for (int i = 0; i < 2; ++i)
    if (!x_lo[i] || !x_hi[i] || !aligned(x_lo[i], 16) || !aligned(x_hi[i], 16))
      return bad("ipc_ring_gemm: database planes must be non-null and 16-byte aligned");
  if (!aligned(b_lo, 16) || !aligned(b_hi, 16) || !aligned(z, 16)) return bad("ipc_ring_gemm: unaligned operand");
  if (l == 0 || l % 128 != 0 || l > 16384) return bad("ipc_ring_gemm: l must be a multiple of 128, at most 16384");
  if (ldz % 8 != 0 || ldz < x_rows) return bad("ipc_ring_gemm: ldz must be a multiple of 8 and >= x_rows");
  if (n_pad < n_cols || n_pad % 128 != 0) return bad("ipc_ring_gemm: n_pad must be >= n_cols and a multiple of 128");
  if (row0 % 8 != 0) return bad("ipc_ring_gemm: row0 must be a multiple of 8");
  if (vec > 1) return bad("ipc_ring_gemm: vec is 0 (code) or 1 (mask)");
  if (x_rows > IPC_MAX_GEMM_ROWS) return bad("ipc_ring_gemm: too many rows in one call");
  if (x_rows == 0 || n_cols == 0) return IPC_OK;
  if (path == IPC_PATH_I8MMA || path == IPC_PATH_I8MIX)
    return ring_gemm_i8(path == IPC_PATH_I8MMA ? 0 : 1, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own, seed_prev, vec, z, ldz,
                        row0, as_stream(stream));
  if (path == IPC_PATH_I32)
    return ring_gemm_i32(x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, l, col_tags, seed_own, seed_prev, vec, z, ldz, row0,
                         as_stream(stream));
  return bad("ipc_ring_gemm: unknown path");
}

namespace {
// b_lo, b_hi: int8 limb planes (mma.sync and int32 paths) or their fp16 patterns (tcgen05).
int check_gemm_args(const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows, const void* b_lo,
                    const void* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags,
                    uint32_t vec, const uint16_t* z, size_t ldz, uint64_t row0, const char* who) {
  auto fail = [&](const char* what) { return bad((std::string(who) + ": " + what).c_str()); };
  if (!x_lo || !x_hi || !b_lo || !b_hi || !col_tags || !z) return fail("null pointer");
  for (int i = 0; i < 2; ++i)
    if (!x_lo[i] || !x_hi[i] || !aligned(x_lo[i], 16) || !aligned(x_hi[i], 16))
      return fail("database planes must be non-null and 16-byte aligned");
  if (!aligned(b_lo, 16) || !aligned(b_hi, 16) || !aligned(z, 16)) return fail("unaligned operand");
  if (l == 0 || l % 128 != 0 || l > 16384) return fail("l must be a multiple of 128, at most 16384");
  if (ldz % 8 != 0 || ldz < x_rows) return fail("ldz must be a multiple of 8 and >= x_rows");
  if (n_pad < n_cols || n_pad % 128 != 0) return fail("n_pad must be >= n_cols and a multiple of 128");
  if (row0 % 8 != 0) return fail("row0 must be a multiple of 8");
  if (vec > 1) return fail("vec is 0 (code) or 1 (mask)");
  if (x_rows > IPC_MAX_GEMM_ROWS) return fail("too many rows in one call");
  return IPC_OK;
}
}  // namespace

extern "C" int ipc_ring_gemm_tiles(int variant, const int8_t* const x_lo[2], const int8_t* const x_hi[2],
                                   size_t x_rows, const int8_t* b_lo, const int8_t* b_hi, uint32_t n_cols,
                                   uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                                   uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                                   const uint32_t* col_tiles, const uint32_t* n_col_list, void* stream) {
  int rc = check_gemm_args(x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, vec, z, ldz, row0,
                           "ipc_ring_gemm_tiles");
  if (rc) return rc;
  if (variant < IPC_GEMM_MIX128 || variant > IPC_GEMM_MMA32) return bad("ipc_ring_gemm_tiles: unknown variant");
  if ((col_tiles == nullptr) != (n_col_list == nullptr))
    return bad("ipc_ring_gemm_tiles: col_tiles and n_col_list go together");
  if (x_rows == 0 || n_cols == 0) return IPC_OK;
  return ring_gemm_i8_variant(variant, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own,
                              seed_prev, vec, z, ldz, row0, col_tiles, n_col_list, as_stream(stream));
}

extern "C" int ipc_ring_gemm_tc(const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows,
                                const uint16_t* b_lo, const uint16_t* b_hi, uint32_t n_cols, uint32_t n_pad,
                                uint32_t l, const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev,
                                uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0, void* stream) {
  int rc = check_gemm_args(x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, vec, z, ldz, row0,
                           "ipc_ring_gemm_tc");
  if (rc) return rc;
  if (x_rows == 0 || n_cols == 0) return IPC_OK;
  return ring_gemm_tc(x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own, seed_prev, vec, z, ldz,
                      row0, as_stream(stream));
}

extern "C" int ipc_ring_gemm_tc_tiles(uint32_t tile_cols, const int8_t* const x_lo[2], const int8_t* const x_hi[2],
                                      size_t x_rows, const uint16_t* b_lo, const uint16_t* b_hi, uint32_t n_cols,
                                      uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                                      uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                                      const uint32_t* col_tiles, const uint32_t* n_col_list, void* stream) {
  int rc = check_gemm_args(x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, vec, z, ldz, row0,
                           "ipc_ring_gemm_tc_tiles");
  if (rc) return rc;
  if (tile_cols != 128 && tile_cols != 256) return bad("ipc_ring_gemm_tc_tiles: tile_cols must be 128 or 256");
  if ((col_tiles == nullptr) != (n_col_list == nullptr))
    return bad("ipc_ring_gemm_tc_tiles: col_tiles and n_col_list go together");
  if (x_rows == 0 || n_cols == 0) return IPC_OK;
  return ring_gemm_tc_variant(tile_cols, 2, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own,
                              seed_prev, vec, z, ldz, row0, col_tiles, n_col_list, as_stream(stream));
}

extern "C" int ipc_ring_gemm_tc_galois(uint32_t tile_cols, const int8_t* x_lo, const int8_t* x_hi, size_t x_rows,
                                       const uint16_t* b_lo, const uint16_t* b_hi, uint32_t n_cols, uint32_t n_pad,
                                       uint32_t l, const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev,
                                       uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                                       const uint32_t* col_tiles, const uint32_t* n_col_list, void* stream) {
  const int8_t* xl[2] = {x_lo, x_lo};
  const int8_t* xh[2] = {x_hi, x_hi};
  int rc = check_gemm_args(xl, xh, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, vec, z, ldz, row0,
                           "ipc_ring_gemm_tc_galois");
  if (rc) return rc;
  if (l % 256 != 0) return bad("ipc_ring_gemm_tc_galois: l must be a multiple of 256");
  if (tile_cols != 128 && tile_cols != 256) return bad("ipc_ring_gemm_tc_galois: tile_cols must be 128 or 256");
  if ((col_tiles == nullptr) != (n_col_list == nullptr))
    return bad("ipc_ring_gemm_tc_galois: col_tiles and n_col_list go together");
  if (x_rows == 0 || n_cols == 0) return IPC_OK;
  return ring_gemm_tc_variant(tile_cols, 1, xl, xh, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own,
                              seed_prev, vec, z, ldz, row0, col_tiles, n_col_list, as_stream(stream));
}

extern "C" int ipc_compare(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz,
                           uint32_t n_cols, size_t n_rows, uint64_t row0, const uint32_t* col_tags,
                           const uint64_t seeds[3], uint32_t thr_a, uint32_t log2_block_words, uint32_t* roots,
                           size_t ld_roots, uint8_t* msb_out, size_t ld_msb, void* stream) {
  if (!z_code || !z_mask || !col_tags || !seeds || !roots) return bad("ipc_compare: null pointer");
  for (int j = 0; j < 3; ++j)
    if (!z_code[j] || !z_mask[j] || !aligned(z_code[j], 16) || !aligned(z_mask[j], 16))
      return bad("ipc_compare: dot planes must be non-null and 16-byte aligned");
  if (log2_block_words > 5) return bad("ipc_compare: log2_block_words must be <= 5");
  if (ldz % 8 != 0 || ldz < n_rows) return bad("ipc_compare: ldz must be a multiple of 8 and >= n_rows");
  if (row0 % (32ull << log2_block_words) != 0) return bad("ipc_compare: row0 must be block aligned");
  const uint64_t blocks = (n_rows + (32ull << log2_block_words) - 1) >> (5 + log2_block_words);
  if (ld_roots < (row0 >> (5 + log2_block_words)) + blocks) return bad("ipc_compare: ld_roots too small");
  if (msb_out && ld_msb < n_rows) return bad("ipc_compare: ld_msb too small");
  if (n_rows == 0 || n_cols == 0) return IPC_OK;
  return compare_launch(z_code, z_mask, ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, log2_block_words, roots,
                        ld_roots, msb_out, ld_msb, as_stream(stream));
}

extern "C" int ipc_compare_plain(const uint16_t* const z_code[3], const uint16_t* ml, size_t ldz, uint32_t n_cols,
                                 size_t n_rows, uint64_t row0, const uint32_t* col_tags, const uint64_t seeds[3],
                                 uint32_t thr_a, uint32_t log2_block_words, uint32_t* roots, size_t ld_roots,
                                 uint8_t* msb_out, size_t ld_msb, void* stream) {
  if (!z_code || !ml || !col_tags || !seeds || !roots) return bad("ipc_compare_plain: null pointer");
  if (!aligned(ml, 16)) return bad("ipc_compare_plain: ml must be 16-byte aligned");
  for (int j = 0; j < 3; ++j)
    if (!z_code[j] || !aligned(z_code[j], 16))
      return bad("ipc_compare_plain: dot planes must be non-null and 16-byte aligned");
  if (log2_block_words > 5) return bad("ipc_compare_plain: log2_block_words must be <= 5");
  if (ldz % 8 != 0 || ldz < n_rows) return bad("ipc_compare_plain: ldz must be a multiple of 8 and >= n_rows");
  if (row0 % (32ull << log2_block_words) != 0) return bad("ipc_compare_plain: row0 must be block aligned");
  const uint64_t blocks = (n_rows + (32ull << log2_block_words) - 1) >> (5 + log2_block_words);
  if (ld_roots < (row0 >> (5 + log2_block_words)) + blocks) return bad("ipc_compare_plain: ld_roots too small");
  if (msb_out && ld_msb < n_rows) return bad("ipc_compare_plain: ld_msb too small");
  if (n_rows == 0 || n_cols == 0) return IPC_OK;
  const uint16_t* zm[3] = {ml, ml, ml};
  return compare_launch_tiles(z_code, zm, ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, log2_block_words, roots,
                              ld_roots, msb_out, ld_msb, nullptr, nullptr, 0, as_stream(stream), nullptr, true);
}

extern "C" int ipc_compare_liftfree(const uint16_t* const z16[3], const uint32_t* const z32[3],
                                    const uint32_t* const ml32[3], size_t ldz, uint32_t n_cols, size_t n_rows,
                                    uint64_t row0, const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a,
                                    uint32_t thr_b, uint32_t log2_block_words, uint32_t* roots, size_t ld_roots,
                                    uint8_t* msb_out, size_t ld_msb, void* stream) {
  if (!ml32 || !col_tags || !seeds || !roots || (!z16) == (!z32))
    return bad("ipc_compare_liftfree: null pointer, or not exactly one of z16 and z32");
  for (int j = 0; j < 3; ++j) {
    const void* d = z16 ? static_cast<const void*>(z16[j]) : static_cast<const void*>(z32[j]);
    if (!ml32[j] || !d || !aligned(ml32[j], 16) || !aligned(d, 16))
      return bad("ipc_compare_liftfree: planes must be non-null and 16-byte aligned");
  }
  if (log2_block_words > 5) return bad("ipc_compare_liftfree: log2_block_words must be <= 5");
  if (ldz % 8 != 0 || ldz < n_rows) return bad("ipc_compare_liftfree: ldz must be a multiple of 8 and >= n_rows");
  if (thr_b > 65536 || (z16 && thr_b != 0 && thr_b != 65536))
    return bad("ipc_compare_liftfree: thr_b must be 2^16 with Z_2^16 dots, and at most 2^16");
  if (row0 % (32ull << log2_block_words) != 0) return bad("ipc_compare_liftfree: row0 must be block aligned");
  const uint64_t blocks = (n_rows + (32ull << log2_block_words) - 1) >> (5 + log2_block_words);
  if (ld_roots < (row0 >> (5 + log2_block_words)) + blocks) return bad("ipc_compare_liftfree: ld_roots too small");
  if (msb_out && ld_msb < n_rows) return bad("ipc_compare_liftfree: ld_msb too small");
  if (n_rows == 0 || n_cols == 0) return IPC_OK;
  return compare_launch_liftfree(z16, z32, ml32, ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, thr_b,
                                 log2_block_words, roots, ld_roots, msb_out, ld_msb, as_stream(stream));
}

extern "C" int ipc_or_finalize(uint32_t* roots, size_t ld_roots, uint32_t n_blocks, uint32_t log2_block_words,
                               uint32_t Q, uint32_t R, const uint32_t* col_tags, const uint64_t seeds[3],
                               uint8_t* bit_shares, void* stream) {
  if (!roots || !col_tags || !seeds || !bit_shares) return bad("ipc_or_finalize: null pointer");
  if (log2_block_words > 5 || R == 0 || R > 31 || Q == 0 || n_blocks == 0 || ld_roots < n_blocks)
    return bad("ipc_or_finalize: bad sizes");
  return or_finalize_launch(roots, ld_roots, n_blocks, log2_block_words, Q, R, col_tags, seeds, bit_shares,
                            as_stream(stream));
}
