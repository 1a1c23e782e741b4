/*
 * ipcheck.h -- C ABI of the GB300 share-domain iris uniqueness check.
 *
 * The library evaluates, for the 3-party replicated secret sharing of
 * arXiv 2405.04463 ("Large-Scale MPC: Scaling Private Iris Code Uniqueness
 * Checks to Millions of Users"), the data-parallel hot path of Alg. 3:
 * share-domain masked dot products over Z_{2^16} (query code/mask shares
 * against every database share, for every rotation), the lift of the mask
 * length to Z_{2^32}, the threshold test as an MSB extraction, and the OR
 * tree to one shared match bit per query. All three parties are simulated on
 * one GPU; their messages are device buffers.
 *
 * Conventions used throughout:
 *  - Parties are numbered 0, 1, 2 (the paper counts from 1). A value x in
 *    Z_{2^k} has additive components x_0, x_1, x_2 (x = sum mod 2^k); party i
 *    holds the replicated pair (x_i, x_{i-1}) (App. C). Boolean sharings use XOR.
 *  - seeds[j] is the PRF key shared by parties j and j+1 (App. D, 3OT and
 *    BitInject). Every random value the protocol draws is one output word of
 *    Philox4x32-10 (Salmon et al., SC'11) keyed by a seed, with the counter
 *    layout documented at each entry point, so results are reproducible and
 *    independent of launch shapes.
 *  - A code has l = rows*cols*cell bits, bit (r*cols + j)*cell + k; the deployed
 *    geometry is 16 x 200 x 4 = 12800 (Sec. 3). Rotation index rho in [0, R)
 *    shifts the 200-column axis by s = rot_lo + rho: out[r][j][k] =
 *    in[r][(j - s) mod cols][k].
 *  - Column n of a query batch is (query q, rotation rho) with n = q*R + rho.
 *    Its PRF tag is col_tags[2n] = request id, col_tags[2n+1] = (q << 5) | rho.
 *  - Unless stated otherwise pointers are DEVICE pointers owned by the caller,
 *    calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and return IPC_OK or a negative IPC_E* code without launching
 *    anything. Errors of an earlier asynchronous call surface at the next call
 *    that synchronises (ipc_status, fetch_*).
 *
 * Thread safety: the stage-level calls are reentrant. A context must not be
 * used from two host threads at once.
 */
#ifndef IPCHECK_H
#define IPCHECK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IPC_OK 0
#define IPC_EINVAL -1     /* bad argument (size, alignment, geometry) */
#define IPC_ENOMEM -2     /* device or host allocation failed, or admission refused */
#define IPC_ECUDA -3      /* a CUDA runtime call failed (see ipc_last_error) */
#define IPC_ETIMEOUT -4   /* fetch_* gave up waiting */
#define IPC_EAGAIN -5     /* request not admitted now; retry later */
#define IPC_ENOTFOUND -6  /* unknown request id */
#define IPC_EDEVICE -7    /* a kernel hit a bounded wait limit and returned early */
#define IPC_ENOSYS -8     /* feature not built for this device */

#define IPC_PATH_I8MMA 0  /* int8 limb GEMM on the tensor cores (mma.sync s8, TMA-fed) */
#define IPC_PATH_I32 1    /* plain int32 CUDA-core ring GEMM (IMAD) */
#define IPC_PATH_I8MIX 2  /* int8 limb GEMM split between mma.sync s8 and dp4a in every tile */
#define IPC_PATH_TC 3     /* the same limbs on tcgen05 as fp16 operands (TMEM accumulators, exact) */
#define IPC_PATH_TCG 4    /* tcgen05, dot products on Galois-ring Shamir shares (Sec. 4.3.2) */

/* PRF domains: high byte of Philox counter word 3. */
#define IPC_D_SHARE 1u
#define IPC_D_ZA 2u
#define IPC_D_AND 3u
#define IPC_D_INJ0 4u
#define IPC_D_INJ2 5u
#define IPC_D_OR 6u
#define IPC_D_GSHARE 7u /* client randomness of the Galois-ring Shamir sharing */
#define IPC_D_COMB 8u   /* AND gates of the per-person OR of eyes and batch parts */
#define IPC_D_SHARE32 9u /* client randomness of the Z_2^32 sharing (lifting variants) */
#define IPC_D_ZA32 10u   /* zero shares of the Z_2^32 dot products (lifting variants) */

/* Lifting variants (Sec. 5.1, Sec. 6.2 Table 2), ipc_config.lift. 0 (MPCLift, the default):
 * code and mask dot products over Z_2^16, ml lifted to Z_2^32 in MPC. */
#define IPC_LIFT_CONST 1 /* ConstLift: ml over Z_2^32 (32-bit mask shares), dot over Z_2^16 */
#define IPC_LIFT_NONE 2  /* NoLift: code and mask dot products both over Z_2^32 */

typedef struct {
  uint32_t rows, cols, cell; /* code geometry; l = rows*cols*cell, a multiple of 128 */
  int32_t rot_lo;            /* shift of rotation 0 (-15 for the deployed +-15 range) */
  uint32_t R;                /* number of rotations, 1..31 */
} ipc_geom;

/* ======================================================================== */
/* Stage-level entry points (one per step of the hot path).                  */
/* ======================================================================== */

/*
 * A0 -- input encoding and sharing (client side; Sec. 4.1.1, App. C).
 * code_bits/mask_bits: [n][ceil(l/64)] uint64, bit b of row r in word b/64 at
 * position b%64. Each code bit becomes the masked bit m - 2(c AND m) in
 * Z_{2^16} (T=-1, U=0, F=+1), each mask bit 0/1; each value x is split as
 * x = x_0 + x_1 + x_2 with x_0 = low and x_1 = high 16 bits of word (b%4) of
 * Philox(client_seed, (b/4, idx0 + r, side<<8 | vec, IPC_D_SHARE<<24)),
 * vec = 0 for code, 1 for mask; side = 0 for database rows, 1 for queries.
 * Output code_sh, mask_sh: [3][n][l] uint16 (component-major).
 * Errors: IPC_EINVAL if l is 0 or n*l overflows.
 */
int ipc_encode_share(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                     uint64_t client_seed, uint32_t side, uint32_t idx0, uint16_t* code_sh,
                     uint16_t* mask_sh, void* stream);

/*
 * A0 of protocol 1 (Sec. 4.3, Alg. 2: the client secret-shares the code but sends the mask in
 * the clear): the public mask operand. mask_bits: [n][ceil(l/64)] uint64 packed as in
 * ipc_encode_share; mask_out: [n][l] uint16 with mask_out[r][b] = bit b of row r (0 or 1),
 * 16-byte aligned. This is the mask[0] input of load_db_shares and submit_queries for a
 * context with plain_mask set. Errors: IPC_EINVAL if l is 0 or not a multiple of 8, a pointer
 * is null or mask_out is unaligned.
 */
int ipc_encode_plain_mask(const uint64_t* mask_bits, uint32_t n, uint32_t l, uint16_t* mask_out, void* stream);

/*
 * A1 -- resident limb planes. Splits each Z_{2^16} element x into balanced
 * signed bytes lo = (int8)(x & 0xFF), hi = (int8)((x - lo) >> 8) so that
 * x = 256*hi + lo (mod 2^16) (the operand decomposition of Sec. 6.1, here
 * with signed limbs so that no fix-up kernels are needed). x: count uint16;
 * lo, hi: count int8 each. Errors: IPC_EINVAL if count is 0.
 */
int ipc_split_limbs(const uint16_t* x, size_t count, int8_t* lo, int8_t* hi, void* stream);

/*
 * A2 -- query preparation for one party. y: [3][Q][l] uint16, the additive
 * components of one query vector (code or mask), unrotated. For party i and
 * column n = q*R + rho it writes the row
 *     B_i[n] = [ rot_rho(y_i + y_{i-1}) | rot_rho(y_i) ]   (length 2l)
 * so that [x_i | x_{i-1}] . B_i[n] = x_i y_i + x_i y_{i-1} + x_{i-1} y_i, the
 * App. C product, with the database kept as raw components. Rotation is
 * linear, so rotating shares rotates the secret. Rows n >= Q*R up to n_pad
 * are zero. b_lo, b_hi: [n_pad][2l] int8 limb planes as in A1.
 * Errors: IPC_EINVAL if party > 2, n_pad < Q*R or the geometry is invalid.
 */
int ipc_prep_query(const uint16_t* y, uint32_t Q, const ipc_geom* g, uint32_t party, int8_t* b_lo,
                   int8_t* b_hi, uint32_t n_pad, void* stream);

/* A2 for IPC_PATH_TC: as ipc_prep_query, each limb written as the fp16 bit pattern of its
 * integer value (exact: |limb| <= 128), the operand type of the tcgen05 GEMM. */
int ipc_prep_query_f16(const uint16_t* y, uint32_t Q, const ipc_geom* g, uint32_t party, uint16_t* b_lo,
                       uint16_t* b_hi, uint32_t n_pad, void* stream);

/*
 * A0 and A2 for Galois-ring Shamir dot products (Sec. 4.3.2; IPC_PATH_TCG).
 * GR = Z_{2^16}[X]/(X^2 - X - 1). Bits 2e, 2e+1 of a code (or mask) form the element
 * g_e = v_{2e} + v_{2e+1} X (v the masked bit or mask bit as in ipc_encode_share), shared
 * with the degree-1 polynomial g_e + r_e Y: party p receives g_e + r_e alpha_p with
 * alpha = (1, X, 1 + X); r_e = (low, high half of word e & 3 of Philox(client_seed,
 * (e >> 2, idx0 + row, side<<8 | vec, IPC_D_GSHARE<<24))). Shares are stored with element e's
 * coefficients at indices 2e, 2e+1, so a share vector has the bit layout; code_sh, mask_sh:
 * [3][n][l] uint16, party-major. l must be a multiple of 8.
 */
int ipc_encode_share_galois(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                            uint64_t client_seed, uint32_t side, uint32_t idx0, uint16_t* code_sh,
                            uint16_t* mask_sh, void* stream);

/*
 * Party p's query operand for Galois-ring shares: B[n][k] (K = l, fp16 limbs as in
 * ipc_prep_query_f16; b_lo, b_hi 16-byte aligned) holds coefficient k & 1 of lambda_p * y_p[e] for the element e that
 * rotation rho = n % R brings to position k / 2, lambda_p the Lagrange coefficient at 0 of
 * party p's point for polynomials of degree <= 2. Then the constant term of the product with
 * party p's database share, summed over elements, is sum_k B[n][k] * x_p[k]: a plain dot
 * product of length l, whose three party components add up to the masked dot product.
 * y: [3][Q][l] the parties' query shares. Errors as ipc_prep_query; the cell size must be even.
 */
int ipc_prep_query_galois(const uint16_t* y, uint32_t Q, const ipc_geom* g, uint32_t party, uint16_t* b_lo,
                          uint16_t* b_hi, uint32_t n_pad, void* stream);

/*
 * A3 -- share-domain dot products of one party for one vector (App. C), as a
 * ring GEMM over Z_{2^16}:
 *     z[n][r] = sum_k [x_i | x_{i-1}][r][k] * B_i[n][k] + r_i(n, r)  (mod 2^16)
 * x_lo[0], x_hi[0]: limb planes of the party's own database component x_i;
 * x_lo[1], x_hi[1]: those of x_{i-1}; each [x_rows][l] int8, row-contiguous.
 * b_lo, b_hi: A2 output [n_pad][2l] int8 (n_pad >= n_cols, multiple of 128).
 * r_i = F(seed_own) - F(seed_prev) mod 2^16 is party i's arithmetic zero share
 * (App. C); F(seed) for global row g = row0 + r is half (g & 1) of word
 * ((g >> 1) & 3) of Philox(seed, (g >> 3, col_tags[2n+1], col_tags[2n],
 * IPC_D_ZA<<24 | vec)). z: [n_cols][ldz] uint16, column-major in the sense
 * that the rows of one query column are contiguous; z_i is the message party
 * i sends to party i+1 (resharing). path selects the int8 tensor-core GEMM
 * (exact: |int32 partial sums| < 2^30), the int8 GEMM split between the tensor
 * cores and the integer pipe's dp4a, or the int32 CUDA-core GEMM; all give
 * identical results. Errors: IPC_EINVAL for l not a multiple of 128, odd
 * ldz, ldz < x_rows, x_rows > IPC_MAX_GEMM_ROWS, or unaligned pointers (16 B);
 * IPC_ECUDA if the tensor map cannot be encoded.
 */
#define IPC_MAX_GEMM_ROWS (65535u * 128u)
int ipc_ring_gemm(int path, const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows,
                  const int8_t* b_lo, const int8_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                  const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec,
                  uint16_t* z, size_t ldz, uint64_t row0, void* stream);

/*
 * A3 with an explicit kernel variant and an optional list of column tiles (the form the
 * serving loop replays inside a CUDA graph). variant: IPC_GEMM_MIX128 (mma.sync + dp4a,
 * 128-column tiles), IPC_GEMM_MMA128, IPC_GEMM_MMA64, IPC_GEMM_MMA32 (mma.sync only, 128/64/32
 * query columns per tile). col_tiles (device, may be NULL): indices of the tiles of that width
 * to compute, n_col_list (device) their count, read when the kernel starts; with NULL every tile
 * of [0, n_cols) is computed, one CTA per tile. With a list the launch is persistent (one CTA
 * per SM walking the list), so its grid does not depend on the list's length and the launch can
 * be replayed from a CUDA graph while the list changes. n_pad must be a multiple of 128 and
 * cover every listed tile. Other arguments and errors as ipc_ring_gemm.
 */
#define IPC_GEMM_MIX128 0
#define IPC_GEMM_MMA128 1
#define IPC_GEMM_MMA64 2
#define IPC_GEMM_MMA32 3
int ipc_ring_gemm_tiles(int variant, const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows,
                        const int8_t* b_lo, const int8_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                        const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z,
                        size_t ldz, uint64_t row0, const uint32_t* col_tiles, const uint32_t* n_col_list,
                        void* stream);

/*
 * A3 on the tcgen05 tensor cores (IPC_PATH_TC): the same ring GEMM and the same
 * z as ipc_ring_gemm. The database operand is the same int8 limb planes as the
 * integer paths (ipc_split_limbs; x planes [x_rows][l], the size of the u16
 * shares); the query operand comes from ipc_prep_query_f16 (fp16 bit patterns
 * of the int8 limbs, b planes [n_pad][2l]). Each k-block of the database tile is
 * widened from int8 to fp16 in shared memory inside the kernel. The products run
 * as fp16 MMAs with fp32 accumulators in tensor memory; each accumulator is
 * drained and restarts at 1.5 * 2^23 after at most 256 products, so all partial
 * sums stay integers inside [2^23, 2^24], where fp32 addition is exact, and the
 * result is bit-identical to the integer paths.
 * Arguments, alignment rules and errors as ipc_ring_gemm.
 */
int ipc_ring_gemm_tc(const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows,
                     const uint16_t* b_lo, const uint16_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                     const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z,
                     size_t ldz, uint64_t row0, void* stream);

/*
 * IPC_PATH_TC with a tile width and an optional list of column tiles (the form the serving
 * loop replays inside a CUDA graph). tile_cols: 256 or 128 query columns per tile.
 * col_tiles (device, may be NULL): indices of the tiles of that width to compute, n_col_list
 * (device) their count, read when the kernel starts; with NULL every tile of [0, n_cols) is
 * computed, one CTA per tile. With a list the launch is persistent (one CTA per SM walking the
 * list), so its grid does not depend on the list. Other arguments and errors as ipc_ring_gemm_tc.
 */
int ipc_ring_gemm_tc_tiles(uint32_t tile_cols, const int8_t* const x_lo[2], const int8_t* const x_hi[2],
                           size_t x_rows, const uint16_t* b_lo, const uint16_t* b_hi, uint32_t n_cols,
                           uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                           uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                           const uint32_t* col_tiles, const uint32_t* n_col_list, void* stream);

/*
 * A3 for Galois-ring Shamir shares (IPC_PATH_TCG): party p's GEMM over its own database
 * share only, K = l: z[n][r] = sum_k B[n][k] x_p[r][k] + r_p(n, r) (mod 2^16), with B from
 * ipc_prep_query_galois and r_p the zero share of ipc_ring_gemm. x_lo, x_hi: int8 limb planes
 * [x_rows][l] of party p's share (ipc_split_limbs). l must be a multiple of 256. tile_cols, col_tiles and
 * n_col_list as in ipc_ring_gemm_tc_tiles. Other arguments and errors as ipc_ring_gemm_tc.
 */
int ipc_ring_gemm_tc_galois(uint32_t tile_cols, const int8_t* x_lo, const int8_t* x_hi, size_t x_rows,
                            const uint16_t* b_lo, const uint16_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                            const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec,
                            uint16_t* z, size_t ldz, uint64_t row0, const uint32_t* col_tiles,
                            const uint32_t* n_col_list, void* stream);

/*
 * A4-A8 (per comparison, and the OR tree inside aligned row blocks).
 * z_code[j], z_mask[j]: the j-th additive components over Z_{2^16} of the
 * code dot and of ml, [n_cols][ldz] uint16 (A3 outputs of parties 0..2).
 * For every column n and row r < n_rows (global row g = row0 + r):
 *   Lift (Sec. 5.1, App. D): BitExtract of bits 17, 16 of ml_0+ml_1+ml_2 over
 *     Z_{2^32} (33 ANDs), BitInject of bit 17 into Z_{2^15} and bit 16 into
 *     Z_{2^16} with the 3-party OT, ConstLift by 2^17 and 2^16, subtract;
 *   ConstLift of the dot by b = 2^16; v = thr_a*ml' - 2^16*dot over Z_{2^32};
 *   MSB by BitExtract(v, {31}) (61 ANDs; App. D). MSB = 1 means a match.
 * Boolean AND gates are the App. C product over F_2 with zero share
 * F_j(gate) = bit (g & 31) of word (G & 3) of Philox(seed_j, (g >> 5,
 * col_tags[2n+1], col_tags[2n], IPC_D_AND<<24 | G>>2)); Lift gates are
 * G = 0..32 (full-adder layer positions 0..16, then ripple positions 1..16),
 * MSB gates G = 36..96 (positions 0..30, then 1..30). BitInject draws c_0 as
 * half (k-bit) of word (g & 3) of Philox(seed_0, (g >> 2, tag, req,
 * IPC_D_INJ0<<24)) -- low half for bit 17, high half for bit 16 -- and c_2,
 * w_0, w_1 from words 0, 1, 2 of Philox(seed_2, (g, tag, req, IPC_D_INJ2<<24)).
 * The MSB bits of the rows of 32*2^log2_block_words consecutive rows (rows
 * past n_rows are the public 0) are OR-reduced by the fixed pairwise tree of
 * ipc_or_finalize; each block's root words (three components, 32 lanes) go to
 * roots[j][n][b], b = (row0 >> (5 + log2_block_words)) + local block.
 * msb_out (optional, may be NULL): [3][n_cols][ld_msb] uint8 components of
 * every comparison's MSB. row0 must be a multiple of 32 << log2_block_words.
 * Errors: IPC_EINVAL for bad sizes or log2_block_words > 5.
 */
int ipc_compare(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz, uint32_t n_cols,
                size_t n_rows, uint64_t row0, const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a,
                uint32_t log2_block_words, uint32_t* roots, size_t ld_roots, uint8_t* msb_out, size_t ld_msb,
                void* stream);

/* ---- Lifting variants (Sec. 5.1, Sec. 6.2): A0-A3 over Z_2^32 ---- */

/*
 * A0 over Z_2^32: the masked bits (T = -1, U = 0, F = +1) and mask bits read in Z_2^32, shared
 * as x_0 + x_1 + x_2 with x_0, x_1 words 2(b & 1), 2(b & 1) + 1 of Philox(client_seed,
 * (b >> 1, idx0 + r, side<<8 | vec, IPC_D_SHARE32<<24)). code_sh, mask_sh: [3][n][l] uint32,
 * 8-byte aligned. Errors: IPC_EINVAL for odd l or null pointers.
 */
int ipc_encode_share32(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                       uint64_t client_seed, uint32_t side, uint32_t idx0, uint32_t* code_sh, uint32_t* mask_sh,
                       void* stream);

/*
 * A1 over Z_2^32: x = l0 + 2^8 l1 + 2^16 l2 + 2^24 l3 (mod 2^32) with balanced limbs in
 * [-128, 127], written as int8 planes limbs[0..3] ([count] each, 4-byte aligned; x 16-byte
 * aligned): the resident database keeps the size of its u32 shares.
 */
int ipc_split_limbs32(const uint32_t* x, size_t count, int8_t* const limbs[4], void* stream);

/*
 * A2 over Z_2^32: party's query operand, four fp16 limb planes b[0..3] of [n_pad][K] (16-byte
 * aligned), each limb the fp16 pattern of its integer value: with
 * segments = 2, K = 2l and row n = q R + rho holds [rot(Y_p + Y_{p-1}) | rot(Y_p)] (the ABY3
 * product, as ipc_prep_query); with segments = 1, K = l and rot(Y_p) alone. y: [3][Q][l] uint32
 * components. Rows Q R .. n_pad - 1 are zero.
 */
int ipc_prep_query32_f16(const uint32_t* y, uint32_t Q, const ipc_geom* g, uint32_t party, uint32_t segments,
                         uint16_t* const b[4], uint32_t n_pad, void* stream);

/*
 * A3 over Z_2^32 on tcgen05 (the ring product of ipc_ring_gemm_tc with four limbs: ten limb
 * products, exact): z[n][r] = sum_k X[r][k] B[n][k] + F(seed_own) - F(seed_prev) (mod 2^32),
 * X = [x[0..3] | x[4..7]] (segments = 2; int8 limb planes [x_rows][l] of this party's and the
 * previous party's components, from ipc_split_limbs32) or x[0..3] (segments = 1), B from
 * ipc_prep_query32_f16. The zero share of row g (global, row0 + r) and column n is word g & 3
 * of Philox(seed, (g >> 2, col_tags[2n+1], col_tags[2n], IPC_D_ZA32<<24 | vec)). z:
 * [n_cols][ldz] uint32, 16-byte aligned, ldz % 4 == 0. Requires segments * l % 256 == 0,
 * n_pad % 128 == 0, n_cols <= n_pad. Errors: IPC_EINVAL for bad sizes or unaligned pointers.
 */
int ipc_ring_gemm_tc32(uint32_t segments, const int8_t* const x[8], size_t x_rows, const uint16_t* const b[4],
                       uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                       uint64_t seed_prev, uint32_t vec, uint32_t* z, size_t ldz, uint64_t row0, void* stream);

/*
 * A5-A7 without Lift (ConstLift and NoLift): ml32: [3] components over Z_2^32 of ml,
 * [n_cols][ldz] uint32 each. The dot product's components are either over Z_2^16 (z16, then
 * z32 = NULL; ConstLift: each component read as an integer and multiplied by 2^16) or over
 * Z_2^32 (z32, then z16 = NULL; NoLift: multiplied by b = thr_b, 1 <= thr_b <= 2^16, 0 meaning
 * 2^16). v = thr_a ml - b dot over Z_2^32 and MSB(v) = BitExtract(v, {31}) (61 ANDs; gates
 * G = 36..96 as in ipc_compare). Block roots, msb_out, alignment and errors as in ipc_compare.
 */
int ipc_compare_liftfree(const uint16_t* const z16[3], const uint32_t* const z32[3], const uint32_t* const ml32[3],
                         size_t ldz, uint32_t n_cols, size_t n_rows, uint64_t row0, const uint32_t* col_tags,
                         const uint64_t seeds[3], uint32_t thr_a, uint32_t thr_b, uint32_t log2_block_words,
                         uint32_t* roots, size_t ld_roots, uint8_t* msb_out, size_t ld_msb, void* stream);

/*
 * A4-A7 of protocol 1 (Sec. 4, Alg. 2: the masks are public) -- the comparison
 * with a public mask length. ml: [n_cols][ldz] uint16, the plaintext ml of each
 * comparison (the same value at every party); z_code as in ipc_compare. For
 * every column n and row r < n_rows: t = floor(thr_a * ml / 2^16) (public;
 * since dot is an integer, dot < thr_a * ml / 2^16 iff dot < t, which is why
 * the floor and not the lemma's ceiling), v = t - dot over Z_{2^16} with t entering
 * component 0, and MSB(v) by BitExtract(v, {15}) (29 ANDs; App. D) with gates
 * G = 0..28 (positions 0..14, then ripple positions 1..14) drawn as in
 * ipc_compare. MSB = 1 means a match. Block roots, msb_out, row0 alignment and
 * errors as in ipc_compare; ml must be 16-byte aligned.
 */
int ipc_compare_plain(const uint16_t* const z_code[3], const uint16_t* ml, size_t ldz, uint32_t n_cols,
                      size_t n_rows, uint64_t row0, const uint32_t* col_tags, const uint64_t seeds[3],
                      uint32_t thr_a, uint32_t log2_block_words, uint32_t* roots, size_t ld_roots,
                      uint8_t* msb_out, size_t ld_msb, void* stream);

/*
 * A8 -- rest of the OR tree (Sec. 4.2: x OR y = x + y + xy, evaluated as a
 * binary tree). The tree has a fixed shape so that shares do not depend on
 * launch shapes: per column, the 32-row words g = 0, 1, ... are combined
 * pairwise level by level (pair j of level L ORs nodes 2j, 2j+1; an odd last
 * node moves up unchanged), then per query the R column words are combined the
 * same way, then the 32 lanes are folded in halves (16, 8, 4, 2, 1). The AND
 * of pair j at level L uses word 0 of Philox(seed_j', (j, tag, req,
 * IPC_D_OR<<24 | stage<<16 | L)), lane bit = lane, with stage 1 and tag
 * (q<<5)|rho for rows, stage 2 and tag q<<5 for rotations, stage 3 (j = 0)
 * for the fold. roots: [3][Q*R][ld_roots] uint32 from ipc_compare, n_blocks
 * per column; it is overwritten (scratch). bit_shares: [3][Q] uint8 output
 * components of the OR bit of each query (1 = some row matched).
 */
int ipc_or_finalize(uint32_t* roots, size_t ld_roots, uint32_t n_blocks, uint32_t log2_block_words, uint32_t Q,
                    uint32_t R, const uint32_t* col_tags, const uint64_t seeds[3], uint8_t* bit_shares,
                    void* stream);

/*
 * A4-A8 without any device allocation (no counterpart in the paper: a convenience for
 * callers that may not allocate). Same result as ipc_compare(..., row0 = 0,
 * log2_block_words = 5, ...) followed by ipc_or_finalize over n_cols = Q*R columns: the
 * bit components [3][Q] of each query's OR over all rows and rotations. Meant for callers
 * that cannot call cudaMalloc once running -- e.g. a host framework that owns the device
 * memory pool, or a service that reserves all memory at start-up. The block-root scratch
 * is a fixed 4 MiB array inside the library (held on every GPU that loads it until exit),
 * so 3 * Q * R * ceil(n_rows / 1024) must not exceed 2^20 words; larger calls fail with
 * IPC_EINVAL before launching anything. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array: calls that may overlap on the GPU (different streams,
 * or different host threads) race with each other and must be serialised by the caller.
 * Arguments as in ipc_compare / ipc_or_finalize; bit_shares: [3][Q] uint8 device output.
 */
int ipc_compare_or_noalloc(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz, uint32_t Q,
                           uint32_t R, size_t n_rows, const uint32_t* col_tags, const uint64_t seeds[3],
                           uint32_t thr_a, uint8_t* bit_shares, void* stream);

/* Reads and clears the device status word of the calling device after
 * synchronising it: IPC_OK, or IPC_EDEVICE if a kernel gave up a bounded wait. */
int ipc_status(void);

/*
 * A test aid for the error path (no counterpart in the paper): runs, on the calling device and
 * stream, a one-thread kernel that waits for a device flag that nothing sets, gives up after
 * limit_us microseconds of global time (1..1,000,000) and raises the status word as a pipeline
 * kernel's bounded wait does. Returns when the kernel has finished; the next ipc_status (or
 * the next fetch of a context on this device) then reports IPC_EDEVICE.
 */
int ipc_selftest_bounded_wait(uint32_t limit_us, void* stream);

/* ======================================================================== */
/* Context-level API: resident database, request submission and fetch.      */
/* ======================================================================== */

typedef struct ipc_ctx ipc_ctx;

typedef struct {
  ipc_geom geom;            /* {16, 200, 4, -15, 31} for the deployed system */
  uint32_t thr_a;           /* a of the threshold a/b with b = 2^16; 16384 for MATCH_RATIO 0.375 */
  int32_t path;             /* IPC_PATH_I8MMA, IPC_PATH_I8MIX, IPC_PATH_I32, IPC_PATH_TC or IPC_PATH_TCG
                               (TCG: load_db_shares and submit_queries take the three parties'
                               Galois-ring Shamir shares from ipc_encode_share_galois) */
  uint32_t db_chunk_rows;   /* rows per resident chunk and pipeline step; multiple of 1024; 0 = 65536 */
  uint32_t max_queries;     /* largest request accepted by submit_queries; 0 = 256 */
  uint64_t seeds[3];        /* pairwise PRF seeds; seeds[j] shared by parties j and j+1 */
  uint32_t keep_distances;  /* nonzero: keep each request's dot products for fetch_distances */
  int32_t device;           /* CUDA device ordinal */
  uint32_t plain_mask;      /* nonzero: protocol 1 (Sec. 4, Alg. 2), masks public (IPC_PATH_TC or
                               IPC_PATH_TCG): load_db_shares and submit_queries take the plain
                               mask bits as 0/1 uint16 in mask[0] (mask[1], mask[2] unused); ml is
                               a plaintext GEMM and a match is MSB(floor(thr_a ml / 2^16) - dot),
                               a 16-bit BitExtract. Not for serving or ipc_check_persons. */
  uint32_t lift;            /* 0, IPC_LIFT_CONST or IPC_LIFT_NONE (IPC_PATH_TC with shared masks
                               only; not for serving or ipc_check_persons). With a lifting
                               variant the vectors shared over Z_2^32 (the mask; with NoLift the
                               code too) are passed to load_db_shares and submit_queries as
                               uint32 components (from ipc_encode_share32) through the same
                               pointer arrays, cast; the others stay uint16. */
  uint32_t thr_b;           /* b of the threshold a/b: 0 or 2^16, or with IPC_LIFT_NONE any value
                               in 1..2^16 (0 meaning 2^16) */
  uint32_t max_requests;    /* request slots: requests submitted and not yet fetched or released,
                               at most 64; 0 = 4. Each slot holds every per-request buffer for
                               max_queries queries, allocated by the first submit_queries. */
  uint32_t fused;           /* nonzero: each resident chunk of a request runs as one fused launch,
                               the six ring GEMMs (A3) tile by tile with each tile's comparison
                               phase (A4-A8) after its sixth GEMM, in place of six GEMM launches on
                               the party streams and one comparison launch (Sec. 6.4 runs the dots
                               and then the comparisons of the same rows). IPC_PATH_TC or
                               IPC_PATH_TCG with shared masks and MPCLift; submit_queries only (not
                               serving or ipc_check_persons). Same shares, bits and messages. */
} ipc_config;

/* Creates a context on cfg->device: the three MPC parties of Alg. 3 (Sec. 2, App. C: 3-party
 * replicated sharing, pairwise PRF seeds cfg->seeds), each with its own stream, plus a control
 * stream on which the comparison phase runs. The geometry is the iris code layout of Sec. 3
 * (l = 12800 bits, 31 rotations) and thr_a the numerator a of the threshold a/b ~ 1 - 2
 * MATCH_RATIO (Sec. 5, Lemma 2). Ownership of *out passes to the caller (release with
 * ipc_destroy). Errors: IPC_EINVAL for an invalid geometry or path, IPC_ECUDA if the device
 * cannot be used. */
int ipc_create(const ipc_config* cfg, ipc_ctx** out);

/* Stream ordering only (no counterpart in the paper). Device inputs of load_db_shares and
 * submit_queries (src_is_device != 0) are read on the library's own non-blocking streams,
 * ordered after all work enqueued so far on `stream` (a cudaStream_t; NULL, the default,
 * means the legacy default stream). Set it to the stream on which the caller produces those
 * inputs. */
int ipc_set_input_stream(ipc_ctx* ctx, void* stream);

/* Appends n_rows rows to the shared database [[C_DB]], [[M_DB]] of Alg. 3 (Sec. 4.3: the MPC
 * nodes hold every enrolled code as shares of its masked bitvector, Sec. 4.1.1; Sec. 5 shares
 * the masks too). code[j], mask[j]: [n_rows][l] uint16, the j-th additive components (A0
 * output layout per component); host memory if src_is_device == 0, else device memory. The
 * library copies them into its resident limb planes (A1; the limb decomposition of the dot
 * products, Sec. 6.1); the caller keeps ownership. Returns IPC_OK, IPC_ENOMEM when the device
 * cannot hold the rows (nothing is appended). */
int load_db_shares(ipc_ctx* ctx, const uint16_t* const code[3], const uint16_t* const mask[3], size_t n_rows,
                   int src_is_device);
/* (load_db_shares returns after the rows are copied: the inputs may be freed on return.) */

/* Submits a batch of n_queries new codes, each secret-shared by the capturing client (Sec.
 * 4.3: the orb shares the code, and under Sec. 5 the mask, to the MPC nodes), for one run of
 * Alg. 3 per query against every resident row, at each of the R rotations of Sec. 3; several
 * persons per batch as in the deployed system (Sec. 6.4). code[j]/mask[j]: [n_queries][l]
 * uint16 unrotated components (host if src_is_device == 0, else device). Non-blocking: the
 * inputs may be reused on return. *req_id receives the request id (also the PRF request tag).
 * Errors: IPC_EINVAL (0 or > max_queries), IPC_ENOMEM, IPC_EAGAIN (every request slot of the
 * context is in use; fetch or release one first). */
int submit_queries(ipc_ctx* ctx, const uint16_t* const code[3], const uint16_t* const mask[3], size_t n_queries,
                   int src_is_device, uint64_t* req_id);

/* Waits up to timeout_ms (< 0: forever) for request req_id and opens each query's shared
 * result bit, as the output node of Sec. 4.3 does: the XOR of its three boolean components.
 * Writes host bits_out[n_queries], 1 = a database row matched at some rotation (Alg. 1 returns
 * true), i.e. the query is not unique. The request is released afterwards. Errors:
 * IPC_ETIMEOUT (request kept), IPC_ENOTFOUND, IPC_EINVAL (n_queries mismatch), IPC_EDEVICE. */
int fetch_match_bits(ipc_ctx* ctx, uint64_t req_id, uint8_t* bits_out, size_t n_queries, int timeout_ms);

/* As fetch_match_bits but writes the three boolean components [3][n_queries] (host) of the
 * OrTree output of Alg. 3 without opening them (Sec. 4.2, Sec. 4.3), and keeps the request. */
int fetch_bit_shares(ipc_ctx* ctx, uint64_t req_id, uint8_t* shares_out, size_t n_queries, int timeout_ms);

/*
 * A test entry point with no counterpart in the paper: a 64-bit fingerprint of a request's
 * messages, for comparing runs and implementations without moving the messages. It covers every
 * message of A4 (App. C: each party's reshared code and mask dot products, for every column and
 * database row; protocol 1's public ml is not a message) and the three output bit components.
 * H = XOR over messages of f(key, v), f(k, v) = mix(mix(k) + v) with mix the SplitMix64 output
 * function, key = kind << 60 | party << 58 | column << 32 | row (kind 0 code, 1 mask, 2 output
 * bit with column = query and row = 0), v the message as an unsigned integer (Z_2^16 or Z_2^32).
 * Waits like fetch_bit_shares. Needs keep_distances: IPC_ENOSYS otherwise.
 */
int fetch_transcript_hash(ipc_ctx* ctx, uint64_t req_id, uint64_t* hash_out, int timeout_ms);

/* Debug: reconstructed masked dot product <c', C'> = ml - 2 hd (App. B; int16) and mask
 * length ml (Alg. 1) of query q at rotation rho for database rows [row_begin, row_end), from
 * the kept A4 messages; host outputs. Needs keep_distances. Waits for the request. Errors:
 * IPC_EINVAL, IPC_ENOTFOUND, IPC_ENOSYS (distances not kept). */
int fetch_distances(ipc_ctx* ctx, uint64_t req_id, uint32_t q, uint32_t rho, size_t row_begin, size_t row_end,
                    int16_t* dot, uint16_t* ml);

/* Fault injection for tests (no counterpart in the paper): the next request submitted on this
 * context simulates party `party` (0..2) dropping out. Before that party computes its messages,
 * its stream waits for a device flag that nothing ever sets; the wait gives up after limit_us
 * (1..1,000,000) of global time and raises the device status word, as every bounded wait in the
 * pipeline does, instead of hanging. A fetch with a shorter timeout returns IPC_ETIMEOUT and
 * keeps the request; the next fetch after the limit returns IPC_EDEVICE once (the word is then
 * cleared), and later fetches return the request's results, which are unaffected. */
int ipc_debug_stall_party(ipc_ctx* ctx, uint32_t party, uint32_t limit_us);

/* Resource management (no counterpart in the paper): releases a request that will not be
 * fetched, returning its slot to the context; waits for its device work first. */
int ipc_release(ipc_ctx* ctx, uint64_t req_id);

/* Number of resident database rows: s of Alg. 3. */
size_t ipc_db_rows(const ipc_ctx* ctx);

/* Measurement aid (no counterpart in the paper). The context's control stream (cudaStream_t):
 * every request's work is joined into it before its completion event, so events recorded on
 * it before submit_queries and after it bracket the request's device time. Owned by the
 * context. */
void* ipc_ctx_stream(const ipc_ctx* ctx);

/* Resource management (no counterpart in the paper): frees every device and host resource
 * of the context, after its device work has finished. */
void ipc_destroy(ipc_ctx* ctx);

/* Error reporting (no counterpart in the paper): text of the last error on this context (or
 * of the last stage-level error of the calling thread when ctx is NULL). Valid until the next
 * call. */
const char* ipc_last_error(const ipc_ctx* ctx);

/* ======================================================================== */
/* Measurement utility (no counterpart in the paper).                        */
/* ======================================================================== */

/* Measures a roofline denominator on the current device with a register-only loop:
 * what = 0 -> mma.sync.m16n8k32 s8 rate in TOP/s (2 ops per multiply-add);
 * what = 1 -> 32-bit IMAD rate in T IMAD/s; what = 2 -> dp4a rate in TOP/s (8 ops per
 * instruction). Synchronous; allocates a small buffer. */
int ipc_measure_peak(int what, void* stream, double* out);

/*
 * Both eyes and inner-batch matching (Sec. 5.4: a query is a person's two iris codes, each
 * rotated R times; the persons of a batch are also matched with each other). ctx[e] holds the
 * database of eye e (both contexts with the same path, geometry, seeds and threshold).
 * code[3e + j], mask[3e + j]: component (or Galois-ring share) j of the P persons' eye-e codes,
 * [P][l] uint16 (host, or device if src_is_device). Per person p the result is
 *   (db_0 OR db_1) OR (batch_0 OR batch_1)
 * with db_e the eye-e code against the eye-e database, and batch_e the eye-e code against the
 * unrotated eye-e codes of the persons p' < p of the batch (later persons enter p's OR tree as
 * the public 0, so of two duplicates the earlier one passes). The OR gates of the combination
 * use Philox(seed_j, (p, 0, req, IPC_D_COMB<<24 | t)), bit 0 of word 0, t = 0 (db_0|db_1),
 * 1 (batch_0|batch_1), 2 (root). Synchronous: writes the bit components [3][P] to host
 * shares_out and the request ids of the five parts (db_0, db_1, batch_0, batch_1, combination)
 * to req_ids. Errors as submit_queries / fetch_bit_shares; IPC_EINVAL for mismatched contexts.
 */
int ipc_check_persons(ipc_ctx* const ctx[2], const uint16_t* const code[6], const uint16_t* const mask[6], uint32_t P,
                      int src_is_device, uint8_t* shares_out, uint64_t req_ids[5], int timeout_ms);

/* ======================================================================== */
/* Serving (A9): continuous batching over the resident database.           */
/* ======================================================================== */
/*
 * ipc_serve_start turns a context (database loaded, path IPC_PATH_TC, I8MMA or I8MIX) into a
 * request loop on its own host thread. Requests (ipc_serve_submit) wait in FIFO order until
 * Q consecutive query slots of a column pool are free (admission by device memory: the pool
 * is allocated once, sized by pool_queries or from free device memory). One loop step runs
 * one resident chunk for every admitted column: the six GEMMs (A3) as one persistent launch
 * per party and vector over a device-side list of the column tiles in use, and the comparison
 * phase (A4-A8) over the same list, replayed from a CUDA graph per (chunk, GEMM variant). A
 * request visits every chunk once, starting wherever the loop is when it is admitted, then
 * its OR tree is finished (A8) and its slots freed. Its result does not depend on the other
 * requests: each PRF counter depends on its request id, query, rotation and row only.
 * fetch_bit_shares / fetch_match_bits / ipc_release take serving request ids. While serving,
 * ipc_serve_* and fetch_* may be called from any host thread; submit_queries and
 * load_db_shares are refused. ipc_serve_stop (or ipc_destroy) finishes every submitted
 * request and stops the loop.
 */
#define IPC_SERVE_AUTOTUNE -1
typedef struct {
  uint32_t pool_queries;   /* query slots (R columns each); 0 = 2 x max_queries, or less if memory is short */
  uint32_t max_pending;    /* submitted, not yet admitted requests before IPC_EAGAIN; 0 = 1024 */
  int32_t variant;         /* GEMM variant for every step, or IPC_SERVE_AUTOTUNE. IPC_PATH_TC:
                              0 = 256-column tcgen05 tiles, 1 = 128-column; int8 paths: the
                              IPC_GEMM_* variants */
  const char* tune_cache;  /* autotuner table (JSON) read if it matches this device and shape,
                              else measured and written; NULL = measure, keep in memory */
} ipc_serve_config;

typedef struct {
  uint64_t steps, admitted, completed, pending;
  double comparisons;       /* database rows x active columns over all steps so far */
  double elapsed_s;         /* since ipc_serve_start */
  uint32_t pool_queries, pool_cols, n_chunks;
  uint64_t variant_steps[4];  /* steps run with each GEMM variant */
} ipc_serve_counters;

/* Errors: IPC_EINVAL (already serving, no rows, int32 path, bad variant), IPC_ENOMEM (pool). */
int ipc_serve_start(ipc_ctx* ctx, const ipc_serve_config* cfg);
/* code[j], mask[j]: HOST [n_queries][l] uint16, copied before return. Returns IPC_EAGAIN when
 * max_pending requests are waiting; IPC_EINVAL if n_queries exceeds max_queries or the pool. */
int ipc_serve_submit(ipc_ctx* ctx, const uint16_t* const code[3], const uint16_t* const mask[3], size_t n_queries,
                     uint64_t* req_id);
int ipc_serve_stop(ipc_ctx* ctx);
int ipc_serve_stats(ipc_ctx* ctx, ipc_serve_counters* out);
/* out: submit, admit and completion times of a request in seconds since ipc_serve_start
 * (-1 while not reached). The completion time is taken on the host when the request's bit
 * components have arrived in host memory. */
int ipc_serve_times(ipc_ctx* ctx, uint64_t req_id, double out[3]);
/* The autotuner's table as JSON (empty if a fixed variant was given). */
int ipc_serve_tuning(ipc_ctx* ctx, char* buf, size_t len);
/* Host-only helpers of the loop, exported for tests: the sorted distinct tiles of width
 * tile_cols covering column ranges [col0[i], col0[i] + ncols[i]) (returns the count; at most
 * max_tiles written), and the first run of `want` free slots (-1 if none). */
int ipc_serve_tile_list(const uint32_t* col0, const uint32_t* ncols, uint32_t n_ranges, uint32_t tile_cols,
                        uint32_t* tiles_out, uint32_t max_tiles);
int64_t ipc_serve_first_fit(const uint8_t* used, uint32_t n_slots, uint32_t want);

#ifdef __cplusplus
}
#endif
#endif
