/*
 * oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU restatement of the share-domain masked iris-code
 * uniqueness check of "Large-Scale MPC: Scaling Private Iris Code Uniqueness
 * Checks to Millions of Users" (arXiv 2405.04463). Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may call it; the CUDA library
 * never links it and shares no code with it.
 *
 * Conventions (0-based parties P0,P1,P2; the paper counts from 1):
 *   - additive components x_0,x_1,x_2 with x = x_0+x_1+x_2 (mod 2^k);
 *   - party i holds the replicated pair (x_i, x_{i-1}) (App. C);
 *   - seed_j is shared by parties j and j+1, so party i holds seed_i and
 *     seed_{i-1} (App. D, 3OT and BitInject);
 *   - boolean sharings are the same with XOR in place of +.
 *
 * Randomness: every random value the protocol draws comes from
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by a 64-bit seed,
 * with the counter layout of the PRF table below. The CUDA library implements
 * the same generator from the same published definition on its own side.
 */
#ifndef IPC_ORACLE_H
#define IPC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* PRF domains (high byte of counter word 3). */
#define ORC_D_SHARE 1u /* client sharing randomness (App. C input sharing)            */
#define ORC_D_ZA    2u /* arithmetic zero shares re-randomising the dot products       */
#define ORC_D_AND   3u /* boolean zero shares of the AND gates of Lift and MSB         */
#define ORC_D_INJ0  4u /* BitInject c_0 (seed_0)                                       */
#define ORC_D_INJ2  5u /* BitInject c_2, w_0, w_1 (seed_2)                             */
#define ORC_D_OR    6u /* boolean zero shares of the OR-tree AND gates                 */
#define ORC_D_GSHARE 7u /* client randomness of the Galois-ring Shamir sharing        */
#define ORC_D_COMB  8u /* boolean zero shares of the per-person OR combination      */
#define ORC_D_SHARE32 9u /* client sharing randomness over Z_{2^32} (lifting variants) */
#define ORC_D_ZA32 10u /* 32-bit arithmetic zero shares of Z_{2^32} dot products    */

/* Gate numbering of the comparison circuit (D_AND counter). */
#define ORC_LIFT_GATE0 0u  /* 33 gates of BitExtract(.,{17,16}) inside Lift      */
#define ORC_MSB_GATE0 36u  /* 61 gates of BitExtract(.,{31}) for the MSB        */

/* Philox4x32-10: out = Philox(key, ctr). */
void orc_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]);

/* Code geometry and rotation. l = rows*cols*cell bits; bit index (r*cols+j)*cell+k.
 * Rotation by shift s: out[r][j][k] = in[r][(j-s) mod cols][k]. */
typedef struct {
  uint32_t rows, cols, cell; /* 16, 200, 4 in the deployed system */
  int32_t rot_lo;            /* first shift (-15) */
  uint32_t R;                /* number of rotations (31); shift of index rho is rot_lo+rho */
} orc_geom;

void orc_rotate_u16(const orc_geom* g, const uint16_t* in, uint16_t* out, int32_t shift);
void orc_rotate_bits(const orc_geom* g, const uint64_t* in, uint64_t* out, int32_t shift);

/* Masked-bit encoding (Sec. 4.1.1) and client-side sharing (App. C). Bits are packed
 * 64 per word, bit b of a row in word b/64 at position b%64. Output shares are
 * [3][n][l] u16 for code and for mask. side = 0 for database rows, 1 for queries;
 * idx0 is the global index of the first row (enters the PRF counter). */
void orc_encode_share(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                      uint64_t client_seed, uint32_t side, uint32_t idx0,
                      uint16_t* code_sh, uint16_t* mask_sh);

/* Alg. 1 for one pair of packed rows: ml = |m & M|, hd = |(c ^ C) & m & M|. */
void orc_plain_pair(const uint64_t* c, const uint64_t* m, const uint64_t* C, const uint64_t* M,
                    uint32_t nwords, int32_t* ml, int32_t* hd);

/* Alg. 1 with rotations over a database: for every query q, rotation rho, row i
 * computes (ml, hd); ml_out/hd_out are [Q][R][s] (may be NULL). match_out[q] is the
 * OR over rho, i of the rule: rule 0 = hd/ml < tau_num/tau_den with ml > 0 (Alg. 1);
 * rule 1 = b*dot > a*ml with dot = ml - 2 hd, b = 2^16, a = thr_a (Alg. 3).
 * threads > 1 uses OpenMP where the library was built with it. */
void orc_plain_match(const orc_geom* g, const uint64_t* qc, const uint64_t* qm, uint32_t Q,
                     const uint64_t* dc, const uint64_t* dm, uint32_t s,
                     int rule, uint32_t tau_num, uint32_t tau_den, uint32_t thr_a,
                     int32_t* ml_out, int32_t* hd_out, uint8_t* match_out, int threads);

/* ---- 3-party replicated-sharing simulation (App. C, App. D, Alg. 3) ---- */

typedef struct {
  uint64_t seeds[3]; /* seed_j shared by parties j and j+1 */
  uint32_t req;      /* request id entering every counter */
  uint32_t thr_a;    /* a of the threshold a/b, b = 2^16 */
} orc_mpc_cfg;

typedef struct {
  uint64_t and_gates;      /* boolean AND gates evaluated */
  uint64_t bits_sent[3];   /* bits sent by each party */
  uint32_t depth_lift;     /* rounds of the Lift of one comparison */
  uint32_t depth_msb;      /* rounds of the MSB extraction of one comparison */
  uint32_t depth_total;    /* rounds of one comparison from the dot products to its MSB */
  uint32_t depth_or;       /* rounds of the OR tree of one query */
  uint32_t and_lift, and_msb; /* gates per comparison */
  uint32_t replication_errors; /* views that broke (x_i, x_{i-1}) consistency */
} orc_stats;

/* App. C dot product of DB row x (components [3][l]) with query y ([3][l], already
 * rotated), re-randomised with the D_ZA zero share of (q, rho, i, vec). Writes the
 * three additive components z_0,z_1,z_2 (z_i is what party i sends to i+1). */
void orc_mpc_dot(const orc_mpc_cfg* cfg, const uint16_t* x, uint64_t x_stride,
                 const uint16_t* y, uint64_t y_stride, uint32_t l,
                 uint32_t q, uint32_t rho, uint32_t i, uint32_t vec, uint16_t z[3], orc_stats* st);

/* One comparison: from the additive components of dot and ml over Z_{2^16}
 * (after resharing) run Lift, ConstLift, a*ml' - b*dot' and BitExtract(.,{31}).
 * Writes the three boolean components of the MSB (1 = match). Optionally returns the
 * lifted ml' components (Z_{2^32}) and v components. */
void orc_mpc_compare(const orc_mpc_cfg* cfg, const uint16_t dot[3], const uint16_t ml[3],
                     uint32_t q, uint32_t rho, uint32_t i, uint8_t msb[3],
                     uint32_t ml_lift[3], uint32_t v_out[3], orc_stats* st);

/* BitExtract([x]_{2^32}, {m, m-1}) on explicit additive components, with the D_AND
 * counter of (q, rho, i) and first gate number gate0. Returns bits m and m-1. */
void orc_bit_extract(const orc_mpc_cfg* cfg, const uint32_t x[3], uint32_t m,
                     uint32_t q, uint32_t rho, uint32_t i, uint32_t gate0,
                     uint8_t top[3], uint8_t below[3], orc_stats* st);

/* orc_bit_extract over n independent sharings x[n][3] (row i uses counter row i), writing
 * top[n][3] and below[n][3]: a loop, for pins over many values. */
void orc_bit_extract_batch(const orc_mpc_cfg* cfg, const uint32_t* x, uint32_t n, uint32_t m, uint32_t gate0,
                           uint8_t* top, uint8_t* below);

/* OR tree of one query over its MSB bit components msb[3][R][s] -> bit[3]. */
void orc_or_tree(const orc_mpc_cfg* cfg, const uint8_t* msb, uint32_t R, uint32_t s,
                 uint32_t q, uint8_t bit[3], orc_stats* st);

/* Whole Alg. 3 for Q queries against s DB rows. Shares are [3][n][l] u16. Outputs
 * (each may be NULL): z_code/z_mask [3][Q*R][s], msb [3][Q*R][s], bits [3][Q]. */
void orc_mpc_match(const orc_mpc_cfg* cfg, const orc_geom* g,
                   const uint16_t* db_code, const uint16_t* db_mask, uint32_t s,
                   const uint16_t* q_code, const uint16_t* q_mask, uint32_t Q,
                   uint16_t* z_code, uint16_t* z_mask, uint8_t* msb, uint8_t* bits,
                   orc_stats* st);

/* ---- Galois-ring Shamir dot products (Sec. 4.3.2, Shamir sharing over Galois rings) ----
 * GR = Z_{2^16}[X]/(X^2 - X - 1); an element c0 + c1 X is stored as uint16_t[2] = {c0, c1}.
 * Two consecutive code (or mask) bits 2e, 2e+1 form one element, so a share vector of l
 * coefficients keeps the bit layout: coefficient t of element e sits at index 2e + t. */
void orc_gr_mul(const uint16_t a[2], const uint16_t b[2], uint16_t out[2]);
/* Returns 1 and writes a^-1 if a is a unit of GR, else returns 0. */
int orc_gr_inv(const uint16_t a[2], uint16_t out[2]);
/* Evaluation points of parties 0, 1, 2 (reading: the non-zero elements of the exceptional
 * set {0, 1, X, 1+X}; the secret sits at 0): alpha = [3][2]. */
void orc_gr_points(uint16_t alpha[6]);
/* Lagrange coefficients at 0 for the three points, degree <= 2: lambda = [3][2]. */
void orc_gr_lagrange(uint16_t lambda[6]);
/* Client sharing: each element g is shared with the degree-1 polynomial g + r Y, party p
 * holding g + r alpha_p; r from Philox(client_seed, (e >> 2, idx0 + row, side<<8 | vec,
 * D_GSHARE << 24)), word e & 3 (c0 = low half, c1 = high half). Output [3][n][l] u16, the
 * three parties' shares, for the masked code bits and for the mask bits. */
void orc_encode_share_galois(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                             uint64_t client_seed, uint32_t side, uint32_t idx0,
                             uint16_t* code_sh, uint16_t* mask_sh);
/* Party p's share of the dot product of DB row x (party shares [3][l]) with the rotated
 * query y (party shares [3][l]): the constant term of sum_e (lambda_p y_p[e]) x_p[e], then the
 * D_ZA zero share of (q, rho, i, vec) as in orc_mpc_dot. z: the three additive components. */
void orc_mpc_dot_galois(const orc_mpc_cfg* cfg, const uint16_t* x, uint64_t x_stride,
                        const uint16_t* y, uint64_t y_stride, uint32_t l,
                        uint32_t q, uint32_t rho, uint32_t i, uint32_t vec, uint16_t z[3], orc_stats* st);
/* orc_mpc_match with the dot products on Galois-ring Shamir shares (inputs from
 * orc_encode_share_galois); the comparison phase and OR tree are unchanged. */
void orc_mpc_match_galois(const orc_mpc_cfg* cfg, const orc_geom* g,
                          const uint16_t* db_code, const uint16_t* db_mask, uint32_t s,
                          const uint16_t* q_code, const uint16_t* q_mask, uint32_t Q,
                          uint16_t* z_code, uint16_t* z_mask, uint8_t* msb, uint8_t* bits,
                          orc_stats* st);

/* ---- Both eyes and inner-batch matching (Sec. 5.4: a query is a person's two irises, and
 * the persons of a batch are also matched with each other). ----
 * Inner-batch part of one eye: the batch's own shares serve as database rows; query q (all R
 * rotations) is compared with the unrotated codes of the persons p' < q only (rows p' >= q are
 * the public 0 in q's OR tree), so of two duplicates in one batch the earlier one passes.
 * galois selects the Galois-ring Shamir dot products. bits: [3][P]. */
void orc_mpc_match_batch(const orc_mpc_cfg* cfg, const orc_geom* g, int galois,
                         const uint16_t* q_code, const uint16_t* q_mask, uint32_t P, uint8_t* bits,
                         orc_stats* st);
/* Person bit = (b0 OR b1) OR (b2 OR b3) on boolean sharings (b0, b1: the two eyes against the
 * database; b2, b3: the two eyes inside the batch). Gate t in {0: b0|b1, 1: b2|b3, 2: root}
 * of person p uses bit 0 of word 0 of Philox(seed_j, (p, 0, req, D_COMB << 24 | t)).
 * bits4: [4][3][P]; out: [3][P]. */
void orc_or_combine(const orc_mpc_cfg* cfg, const uint8_t* bits4, uint32_t P, uint8_t* out, orc_stats* st);

/* ---- Protocol 1 (Sec. 4, Alg. 2): shared codes, public masks ----
 * ml = CountOnes(rot(m_q) AND M_i) is public; only the code dot product is shared. A match is
 * MSB(t - <c', C'>) over Z_{2^16} with the public t = floor(a * ml / 2^16) (reading: the floor
 * makes the test exactly <c', C'> > (a / 2^16) ml, Alg. 1's strict rule), added by component 0;
 * BitExtract of bit 15 (29 ANDs, 15 rounds; gates from 0 in the D_AND counters). */
void orc_mpc_compare_plain(const orc_mpc_cfg* cfg, const uint16_t dot[3], uint32_t ml, uint32_t q, uint32_t rho,
                           uint32_t i, uint8_t msb[3], orc_stats* st);
/* Alg. 2 for all queries: code shares [3][n][l] (additive components, or Galois-ring Shamir
 * shares when galois != 0), masks as packed bits [n][ceil(l/64)]. Outputs (may be NULL):
 * z_code [3][Q*R][s] (the dot-product components), ml [Q*R][s], bits [3][Q]. */
void orc_mpc_match_plain(const orc_mpc_cfg* cfg, const orc_geom* g, int galois,
                         const uint16_t* db_code, const uint64_t* db_mask_bits, uint32_t s,
                         const uint16_t* q_code, const uint64_t* q_mask_bits, uint32_t Q,
                         uint16_t* z_code, uint16_t* ml_out, uint8_t* bits, orc_stats* st);

/* ---- Lifting variants (Sec. 5.1 and Sec. 6.2, Table 2) ----
 * MPCLift (the default of Alg. 3 above): dot and ml over Z_{2^16}, ml lifted to Z_{2^32} in
 * MPC. ConstLift: ml computed over Z_{2^32} from 32-bit mask shares, dot over Z_{2^16} and
 * lifted for free by ConstLift with b = 2^16. NoLift: dot and ml both computed over Z_{2^32}
 * (b any 16-bit constant). Either way v = a ml - b dot over Z_{2^32} and the match bit is
 * MSB(v) = BitExtract(v, {31}) (61 ANDs, gates from ORC_MSB_GATE0) -- no Lift. */
#define ORC_LIFT_CONST 1
#define ORC_LIFT_NONE 2
/* Client sharing over Z_{2^32} of the masked code bits and of the mask bits (values -1, 0, 1
 * and 0, 1 read in Z_{2^32}): x_0, x_1 are words 2(b & 1), 2(b & 1) + 1 of
 * Philox(client_seed, (b >> 1, idx0 + row, side<<8 | vec, D_SHARE32 << 24)), x_2 = v - x_0 - x_1.
 * Output [3][n][l] u32. */
void orc_encode_share32(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                        uint64_t client_seed, uint32_t side, uint32_t idx0, uint32_t* code_sh, uint32_t* mask_sh);
/* orc_mpc_dot over Z_{2^32}; the zero share of (q, rho, i, vec) under one seed is word i & 3
 * of Philox(seed, (i >> 2, (q<<5)|rho, req, D_ZA32 << 24 | vec)). */
void orc_mpc_dot32(const orc_mpc_cfg* cfg, const uint32_t* x, uint64_t x_stride, const uint32_t* y,
                   uint64_t y_stride, uint32_t l, uint32_t q, uint32_t rho, uint32_t i, uint32_t vec, uint32_t z[3],
                   orc_stats* st);
/* One comparison without Lift. ml: components over Z_{2^32}. dot: components over Z_{2^16}
 * (mode ORC_LIFT_CONST; b must be 2^16) or over Z_{2^32} (ORC_LIFT_NONE, b = thr_b < 2^16, or
 * 2^16 when thr_b is 0 or 2^16). Writes the MSB's boolean components, optionally v's. */
void orc_mpc_compare_liftfree(const orc_mpc_cfg* cfg, int mode, const uint32_t dot[3], const uint32_t ml[3],
                              uint32_t thr_b, uint32_t q, uint32_t rho, uint32_t i, uint8_t msb[3],
                              uint32_t v_out[3], orc_stats* st);
/* Alg. 3 with a lifting variant. db_code / q_code: [3][n][l] u16 shares (ORC_LIFT_CONST) or
 * u32 shares (ORC_LIFT_NONE); db_mask / q_mask: [3][n][l] u32 shares. Outputs (may be NULL):
 * z_code [3][Q*R][s] (u16 or u32 as the code shares), z_mask [3][Q*R][s] u32, bits [3][Q]. */
void orc_mpc_match_lift(const orc_mpc_cfg* cfg, const orc_geom* g, int mode, uint32_t thr_b,
                        const void* db_code, const uint32_t* db_mask, uint32_t s, const void* q_code,
                        const uint32_t* q_mask, uint32_t Q, void* z_code, uint32_t* z_mask, uint8_t* bits,
                        orc_stats* st);

/* ---- Transcript hash (a test aid; no counterpart in the paper) ----
 * A 64-bit fingerprint of a request's messages: every A4 message (each party's reshared code and
 * mask dot products, App. C) and the three output bit components. H = XOR over messages of
 * f(key, v) = mix(mix(key) + v), mix = the SplitMix64 output function (Steele, Lea, Flood 2014),
 * key = kind << 60 | party << 58 | column << 32 | row (kind 0 code, 1 mask, 2 output bit with
 * column = query and row = 0), v the message as an unsigned integer. z_code, z_mask: [3][n][s]
 * of elem_code / elem_mask bytes (2 or 4); z_mask may be NULL (protocol 1: ml is public); bits
 * [3][Q]. orc_mix64 is exposed for its pin. */
uint64_t orc_mix64(uint64_t z);
uint64_t orc_transcript_hash(const void* z_code, uint32_t elem_code, const void* z_mask, uint32_t elem_mask,
                             uint32_t n_cols, uint32_t s, const uint8_t* bits, uint32_t Q);

#ifdef __cplusplus
}
#endif
#endif
