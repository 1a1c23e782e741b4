/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain CPU restatement of arXiv 2405.04463, written for reading against the
 * paper rather than for speed. Every function names the passage it follows;
 * the functions are pinned by tests/test_oracle_pins.py.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplies; the key  */
/* is bumped by the Weyl constants between rounds.                            */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]) {
  uint32_t k0 = key[0], k1 = key[1];
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* PRF(seed, counter): Philox keyed by the two halves of a 64-bit seed. */
static void prf(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {c0, c1, c2, c3};
  orc_philox4x32_10(key, ctr, out);
}

static uint32_t col_tag(uint32_t q, uint32_t rho) { return (q << 5) | rho; }

/* ------------------------------------------------------------------------ */
/* Rotation (Sec. 3: each query code is checked at r = 31 small offsets).    */
/* Shift s moves column j-s of the 200-column axis to column j, cyclically.  */
/* ------------------------------------------------------------------------ */
static uint32_t src_col(const orc_geom* g, uint32_t j, int32_t shift) {
  int64_t c = ((int64_t)j - shift) % (int64_t)g->cols;
  if (c < 0) c += g->cols;
  return (uint32_t)c;
}

void orc_rotate_u16(const orc_geom* g, const uint16_t* in, uint16_t* out, int32_t shift) {
  for (uint32_t r = 0; r < g->rows; r++)
    for (uint32_t j = 0; j < g->cols; j++)
      for (uint32_t k = 0; k < g->cell; k++)
        out[(r * g->cols + j) * g->cell + k] = in[(r * g->cols + src_col(g, j, shift)) * g->cell + k];
}

static int get_bit(const uint64_t* v, uint32_t b) { return (int)((v[b >> 6] >> (b & 63)) & 1u); }

void orc_rotate_bits(const orc_geom* g, const uint64_t* in, uint64_t* out, int32_t shift) {
  uint32_t l = g->rows * g->cols * g->cell;
  uint32_t nw = (l + 63) / 64;
  memset(out, 0, nw * sizeof(uint64_t));
  for (uint32_t r = 0; r < g->rows; r++)
    for (uint32_t j = 0; j < g->cols; j++)
      for (uint32_t k = 0; k < g->cell; k++) {
        uint32_t dst = (r * g->cols + j) * g->cell + k;
        uint32_t src = (r * g->cols + src_col(g, j, shift)) * g->cell + k;
        if (get_bit(in, src)) out[dst >> 6] |= (uint64_t)1 << (dst & 63);
      }
}

/* ------------------------------------------------------------------------ */
/* Input encoding and sharing.                                               */
/* Masked bit (Sec. 4.1.1): a' = m_a - 2 (a AND m_a), i.e. T=-1, U=0, F=+1;   */
/* the mask itself is shared as 0/1. Shares (App. C): x = x0 + x1 + x2 over  */
/* Z_{2^16}; x0, x1 are the client's random draws (D_SHARE, one Philox call  */
/* per 4 elements: word k%4, low half x0, high half x1), x2 = x - x0 - x1.   */
/* ------------------------------------------------------------------------ */
void orc_encode_share(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                      uint64_t client_seed, uint32_t side, uint32_t idx0,
                      uint16_t* code_sh, uint16_t* mask_sh) {
  uint32_t nw = (l + 63) / 64;
  size_t plane = (size_t)n * l;
  for (uint32_t r = 0; r < n; r++) {
    const uint64_t* c = code_bits + (size_t)r * nw;
    const uint64_t* m = mask_bits + (size_t)r * nw;
    uint32_t w[2][4];
    for (uint32_t b = 0; b < l; b++) {
      int cb = get_bit(c, b), mb = get_bit(m, b);
      uint16_t val[2];
      val[0] = (uint16_t)(mb - 2 * (cb & mb));
      val[1] = (uint16_t)mb;
      if ((b & 3u) == 0)
        for (uint32_t vec = 0; vec < 2; vec++)
          prf(client_seed, b >> 2, idx0 + r, (side << 8) | vec, ORC_D_SHARE << 24, w[vec]);
      for (uint32_t vec = 0; vec < 2; vec++) {
        uint32_t word = w[vec][b & 3];
        uint16_t x0 = (uint16_t)(word & 0xFFFFu);
        uint16_t x1 = (uint16_t)(word >> 16);
        uint16_t x2 = (uint16_t)(val[vec] - x0 - x1);
        uint16_t* dst = vec == 0 ? code_sh : mask_sh;
        size_t at = (size_t)r * l + b;
        dst[at] = x0;
        dst[plane + at] = x1;
        dst[2 * plane + at] = x2;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (plaintext membership), one pair: m' = m AND M, ml = CountOnes(m'), */
/* hd = CountOnes((c XOR C) AND m').                                         */
/* ------------------------------------------------------------------------ */
static int popcount64(uint64_t x) { return __builtin_popcountll(x); }

void orc_plain_pair(const uint64_t* c, const uint64_t* m, const uint64_t* C, const uint64_t* M,
                    uint32_t nwords, int32_t* ml, int32_t* hd) {
  int32_t a = 0, h = 0;
  for (uint32_t w = 0; w < nwords; w++) {
    uint64_t mm = m[w] & M[w];
    a += popcount64(mm);
    h += popcount64((c[w] ^ C[w]) & mm);
  }
  *ml = a;
  *hd = h;
}

/* Match rule. Rule 0 is Alg. 1's hd/ml < MATCH_RATIO with MATCH_RATIO =
 * tau_num/tau_den (false when ml = 0, where the ratio is undefined). Rule 1 is
 * Alg. 3's MSB(a*ml - b*dot) with dot = <c',C'> = ml - 2 hd (App. B), b = 2^16:
 * true iff b*dot > a*ml. */
static int match_rule(int rule, int32_t ml, int32_t hd, uint32_t tau_num, uint32_t tau_den, uint32_t thr_a) {
  if (rule == 0) {
    if (ml <= 0) return 0;
    return (int64_t)hd * tau_den < (int64_t)tau_num * ml;
  }
  int64_t dot = (int64_t)ml - 2 * (int64_t)hd;
  return 65536 * dot > (int64_t)thr_a * ml;
}

void orc_plain_match(const orc_geom* g, const uint64_t* qc, const uint64_t* qm, uint32_t Q,
                     const uint64_t* dc, const uint64_t* dm, uint32_t s,
                     int rule, uint32_t tau_num, uint32_t tau_den, uint32_t thr_a,
                     int32_t* ml_out, int32_t* hd_out, uint8_t* match_out, int threads) {
  uint32_t l = g->rows * g->cols * g->cell;
  uint32_t nw = (l + 63) / 64;
  uint32_t R = g->R;
  uint32_t ncol = Q * R;
  uint8_t* colmatch = (uint8_t*)calloc(ncol ? ncol : 1, 1);
#ifdef _OPENMP
  if (threads < 1) threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
  for (int64_t n = 0; n < (int64_t)ncol; n++) {
    uint32_t q = (uint32_t)n / R, rho = (uint32_t)n % R;
    int32_t shift = g->rot_lo + (int32_t)rho;
    uint64_t* rc = (uint64_t*)malloc(nw * sizeof(uint64_t));
    uint64_t* rm = (uint64_t*)malloc(nw * sizeof(uint64_t));
    orc_rotate_bits(g, qc + (size_t)q * nw, rc, shift);
    orc_rotate_bits(g, qm + (size_t)q * nw, rm, shift);
    uint8_t any = 0;
    for (uint32_t i = 0; i < s; i++) {
      int32_t ml, hd;
      orc_plain_pair(rc, rm, dc + (size_t)i * nw, dm + (size_t)i * nw, nw, &ml, &hd);
      if (ml_out) ml_out[(size_t)n * s + i] = ml;
      if (hd_out) hd_out[(size_t)n * s + i] = hd;
      if (match_rule(rule, ml, hd, tau_num, tau_den, thr_a)) any = 1;
    }
    colmatch[n] = any;
    free(rc);
    free(rm);
  }
  for (uint32_t q = 0; q < Q; q++) {
    uint8_t any = 0;
    for (uint32_t rho = 0; rho < R; rho++) any |= colmatch[q * R + rho];
    match_out[q] = any;
  }
  free(colmatch);
  (void)threads;
}

/* ------------------------------------------------------------------------ */
/* Replicated sharing with explicit per-party views (App. C).                */
/* view[p] = (own, prev) = (x_p, x_{p-1}); a message from party p reaches    */
/* party p+1, which stores it as its prev component.                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t own, prev;
} view_t;

typedef struct {
  view_t v[3];
  uint32_t depth; /* communication rounds behind this value */
} rss_t;

static int P(int p) { return ((p % 3) + 3) % 3; }

static rss_t rss_zero(void) {
  rss_t z;
  memset(&z, 0, sizeof z);
  return z;
}

/* Additive components already held in replicated form (after resharing). */
static rss_t rss_from_components(const uint32_t x[3], uint32_t depth) {
  rss_t r;
  for (int p = 0; p < 3; p++) {
    r.v[p].own = x[p];
    r.v[p].prev = x[P(p - 1)];
  }
  r.depth = depth;
  return r;
}

static void rss_check(const rss_t* r, orc_stats* st) {
  for (int p = 0; p < 3; p++)
    if (r->v[p].prev != r->v[P(p - 1)].own) st->replication_errors++;
}

/* Reconstruct: x_0 + x_1 + x_2 read from the parties' own components. */
static uint32_t rss_component(const rss_t* r, int j) { return r->v[j].own; }

/* XOR of boolean sharings: local. */
static rss_t bxor(rss_t a, rss_t b) {
  rss_t r;
  for (int p = 0; p < 3; p++) {
    r.v[p].own = a.v[p].own ^ b.v[p].own;
    r.v[p].prev = a.v[p].prev ^ b.v[p].prev;
  }
  r.depth = a.depth > b.depth ? a.depth : b.depth;
  return r;
}

/* AND of boolean sharings: the App. C multiplication over F_2,
 * z_i = x_i y_i + x_i y_{i-1} + x_{i-1} y_i + alpha_i with the zero share
 * alpha_i = F(seed_i) + F(seed_{i-1}); party i then sends z_i to party i+1. */
static rss_t band(rss_t a, rss_t b, const uint32_t F[3], orc_stats* st) {
  uint32_t z[3];
  for (int p = 0; p < 3; p++) {
    uint32_t alpha = (F[p] ^ F[P(p - 1)]) & 1u;
    z[p] = ((a.v[p].own & b.v[p].own) ^ (a.v[p].own & b.v[p].prev) ^ (a.v[p].prev & b.v[p].own) ^ alpha) & 1u;
  }
  rss_t r;
  for (int p = 0; p < 3; p++) {
    r.v[p].own = z[p];
    r.v[P(p + 1)].prev = z[p]; /* message p -> p+1 */
    st->bits_sent[p] += 1;
  }
  r.depth = (a.depth > b.depth ? a.depth : b.depth) + 1;
  st->and_gates++;
  rss_check(&r, st);
  return r;
}

/* InpLocal(x, j, 2) (App. D) for bit b of additive component j of X: the value
 * is known to parties j (as own) and j+1 (as prev); component j of the boolean
 * sharing is that bit and the other two are zero. Each party reads the bit from
 * its own view. */
static rss_t inp_local_bit(const rss_t* X, int j, uint32_t b) {
  rss_t r = rss_zero();
  r.v[j].own = (X->v[j].own >> b) & 1u;        /* party j: (x_j, 0)       */
  r.v[P(j + 1)].prev = (X->v[P(j + 1)].prev >> b) & 1u; /* party j+1: (0, x_j) */
  r.depth = X->depth;
  return r;
}

/* Source of the three PRF bits of one AND gate. */
typedef struct {
  const orc_mpc_cfg* cfg;
  uint32_t c0, c1;  /* counter words 0,1 */
  uint32_t domain;  /* counter word 3 high byte */
  uint32_t lane;    /* bit inside the returned word */
} gate_rng;

/* D_AND: gate G of comparison (q, rho, i) takes bit i%32 of word G%4 of
 * Philox(seed_j, (i/32, col, req, D_AND<<24 | G/4)). */
static void and_bits(const gate_rng* g, uint32_t gate, uint32_t F[3]) {
  for (int j = 0; j < 3; j++) {
    uint32_t w[4];
    prf(g->cfg->seeds[j], g->c0, g->c1, g->cfg->req, (g->domain << 24) | (gate >> 2), w);
    F[j] = (w[gate & 3] >> g->lane) & 1u;
  }
}

/* FA (App. D): t1 = a+c, t2 = b+c, s = t1+b, o = t1*t2 + c over F_2. */
static void full_adder(rss_t a, rss_t b, rss_t c, const gate_rng* g, uint32_t* gate, rss_t* s, rss_t* o,
                       orc_stats* st) {
  rss_t t1 = bxor(a, c);
  rss_t t2 = bxor(b, c);
  *s = bxor(t1, b);
  uint32_t F[3];
  and_bits(g, (*gate)++, F);
  *o = bxor(band(t1, t2, F, st), c);
}

/*
 * BitExtract([x]_{2^32}, I) with max I = m (App. D): ShareSplit into the
 * trivial boolean sharings of each component's bits, one layer of full adders
 * (3 -> 2), then a ripple-carry BinAdd of (carries << 1) and the sums. Gates
 * whose output is never used (the carry out of the top position) or that
 * multiply by the public constant 0 (the shifted-in carry at position 0) are not
 * evaluated; this gives the counts the paper states for k-bit extraction,
 * 2k-3 ANDs in k-1 rounds (Sec. 4.3.1, Sec. 5.2). Returns bits m and m-1.
 */
static void bit_extract_rss(const rss_t* X, uint32_t m, const gate_rng* g, uint32_t gate0,
                            rss_t* top, rss_t* below, orc_stats* st) {
  rss_t s[33], c[33];
  uint32_t gate = gate0;
  for (uint32_t b = 0; b <= m; b++) {
    rss_t x0 = inp_local_bit(X, 0, b);
    rss_t x1 = inp_local_bit(X, 1, b);
    rss_t x2 = inp_local_bit(X, 2, b);
    if (b < m)
      full_adder(x0, x1, x2, g, &gate, &s[b], &c[b], st);
    else
      s[b] = bxor(bxor(x0, x1), x2);
  }
  /* BinAdd((c[m-1..0], 0), s[m..0]); r[0] = s[0] because the shifted operand is 0 there. */
  rss_t r_prev = s[0], r_top;
  rss_t carry = rss_zero();
  carry.depth = 0;
  for (uint32_t b = 1; b <= m; b++) {
    rss_t a = c[b - 1];
    if (b < m) {
      rss_t sum, cout;
      full_adder(a, s[b], carry, g, &gate, &sum, &cout, st);
      carry = cout;
      if (b == m - 1) r_prev = sum;
    } else {
      r_top = bxor(bxor(a, s[b]), carry);
    }
  }
  if (m == 0) r_top = s[0];
  *top = r_top;
  *below = r_prev;
}

void orc_bit_extract(const orc_mpc_cfg* cfg, const uint32_t x[3], uint32_t m,
                     uint32_t q, uint32_t rho, uint32_t i, uint32_t gate0,
                     uint8_t top[3], uint8_t below[3], orc_stats* st) {
  rss_t X = rss_from_components(x, 0);
  gate_rng g = {cfg, i >> 5, col_tag(q, rho), ORC_D_AND, i & 31u};
  rss_t t, b;
  bit_extract_rss(&X, m, &g, gate0, &t, &b, st);
  for (int j = 0; j < 3; j++) {
    top[j] = (uint8_t)rss_component(&t, j);
    below[j] = (uint8_t)rss_component(&b, j);
  }
}

/*
 * BitInject([x]_2, 2^k) (App. D) with the 3-party OT (App. D, after ABY3).
 * 0-based roles: P0 = OT sender (paper's party 1), P1 = receiver (party 2),
 * P2 = helper (party 3). c_0 comes from seed_0 (P0, P1); c_2, w_0, w_1 from
 * seed_2 (P2, P0). P0 forms m_beta = (beta ^ x_0 ^ x_2) - c_0 - c_2, masks them
 * as k_beta = w_beta ^ m_beta and sends both to P1; P2 sends w_{x_1} to P1; P1
 * recovers c_1 = m_{x_1} and forwards it to P2. Result components (c_0,c_1,c_2).
 */
static rss_t bit_inject(rss_t X, uint32_t k, uint32_t c0, uint32_t c2, uint32_t w0, uint32_t w1,
                        orc_stats* st) {
  uint32_t mask = (k >= 32) ? 0xFFFFFFFFu : ((1u << k) - 1u);
  c0 &= mask;
  c2 &= mask;
  w0 &= mask;
  w1 &= mask;
  /* P0: knows x_0 (own) and x_2 (prev) */
  uint32_t x0 = X.v[0].own & 1u, x2 = X.v[0].prev & 1u;
  uint32_t m0 = ((0u ^ x0 ^ x2) - c0 - c2) & mask;
  uint32_t m1 = ((1u ^ x0 ^ x2) - c0 - c2) & mask;
  uint32_t k0 = w0 ^ m0, k1 = w1 ^ m1; /* P0 -> P1 */
  st->bits_sent[0] += 2 * k;
  /* P2: knows x_1 as its prev component */
  uint32_t wsel = (X.v[2].prev & 1u) ? w1 : w0; /* P2 -> P1 */
  st->bits_sent[2] += k;
  /* P1: choice bit x_1 is its own component */
  uint32_t c1 = (wsel ^ ((X.v[1].own & 1u) ? k1 : k0)) & mask; /* P1 -> P2 */
  st->bits_sent[1] += k;
  rss_t r;
  r.v[0].own = c0;
  r.v[0].prev = c2;
  r.v[1].own = c1;
  r.v[1].prev = c0;
  r.v[2].own = c2;
  r.v[2].prev = c1;
  r.depth = X.depth + 2;
  rss_check(&r, st);
  return r;
}

/* ConstLift([a]_c, d) (App. D): each component a_i read as an integer in [0,c)
 * and multiplied by d, giving a sharing over Z_{c*d} (here c*d = 2^32). */
static rss_t const_lift(rss_t a, uint32_t d) {
  for (int p = 0; p < 3; p++) {
    a.v[p].own = a.v[p].own * d;
    a.v[p].prev = a.v[p].prev * d;
  }
  return a;
}

/* Lift([x]_{2^16}, 2^32) (Sec. 5.1, App. D). */
static rss_t lift16(const orc_mpc_cfg* cfg, const uint16_t ml[3], uint32_t depth, uint32_t q, uint32_t rho,
                    uint32_t i, orc_stats* st) {
  /* Components re-read over Z_{2^32}; InpLocal of each plus the local sum gives
   * the sharing whose component j is ml_j, i.e. [ml_0 + ml_1 + ml_2]. */
  uint32_t comp[3] = {ml[0], ml[1], ml[2]};
  rss_t S = rss_from_components(comp, depth);
  gate_rng g = {cfg, i >> 5, col_tag(q, rho), ORC_D_AND, i & 31u};
  rss_t a, b; /* a = bit 17, b = bit 16 of ml_0 + ml_1 + ml_2 */
  bit_extract_rss(&S, 17, &g, ORC_LIFT_GATE0, &a, &b, st);
  /* BitInject randomness (D_INJ0 from seed_0, D_INJ2 from seed_2). */
  uint32_t w0[4], w2[4];
  prf(cfg->seeds[0], i >> 2, col_tag(q, rho), cfg->req, ORC_D_INJ0 << 24, w0);
  prf(cfg->seeds[2], i, col_tag(q, rho), cfg->req, ORC_D_INJ2 << 24, w2);
  uint32_t c0w = w0[i & 3];
  rss_t A = bit_inject(a, 15, c0w & 0xFFFFu, w2[0] & 0xFFFFu, w2[1] & 0xFFFFu, w2[2] & 0xFFFFu, st);
  rss_t B = bit_inject(b, 16, c0w >> 16, w2[0] >> 16, w2[1] >> 16, w2[2] >> 16, st);
  A = const_lift(A, 1u << 17);
  B = const_lift(B, 1u << 16);
  rss_t out;
  for (int p = 0; p < 3; p++) {
    out.v[p].own = S.v[p].own - A.v[p].own - B.v[p].own;
    out.v[p].prev = S.v[p].prev - A.v[p].prev - B.v[p].prev;
  }
  out.depth = A.depth > B.depth ? A.depth : B.depth;
  rss_check(&out, st);
  return out;
}

/* D_ZA zero-share half-word of (q, rho, i, vec) under one seed. */
static uint32_t za_value(uint64_t seed, uint32_t req, uint32_t q, uint32_t rho, uint32_t i, uint32_t vec) {
  uint32_t w[4];
  prf(seed, i >> 3, col_tag(q, rho), req, (ORC_D_ZA << 24) | vec, w);
  return (w[(i >> 1) & 3] >> (16 * (i & 1))) & 0xFFFFu;
}

/* App. C: z_i = x_i y_i + x_{i-1} y_i + x_i y_{i-1} + r_i summed over the
 * vector (a dot product needs one resharing only), r_i = F_i - F_{i-1}. */
void orc_mpc_dot(const orc_mpc_cfg* cfg, const uint16_t* x, uint64_t x_stride,
                 const uint16_t* y, uint64_t y_stride, uint32_t l,
                 uint32_t q, uint32_t rho, uint32_t i, uint32_t vec, uint16_t z[3], orc_stats* st) {
  for (int p = 0; p < 3; p++) {
    const uint16_t* xp = x + (size_t)p * x_stride;
    const uint16_t* xm = x + (size_t)P(p - 1) * x_stride;
    const uint16_t* yp = y + (size_t)p * y_stride;
    const uint16_t* ym = y + (size_t)P(p - 1) * y_stride;
    uint32_t acc = 0;
    for (uint32_t k = 0; k < l; k++)
      acc += (uint32_t)xp[k] * yp[k] + (uint32_t)xm[k] * yp[k] + (uint32_t)xp[k] * ym[k];
    uint32_t r = za_value(cfg->seeds[p], cfg->req, q, rho, i, vec) - za_value(cfg->seeds[P(p - 1)], cfg->req, q, rho, i, vec);
    z[p] = (uint16_t)(acc + r);
    if (st) st->bits_sent[p] += 16; /* resharing: z_p to party p+1 */
  }
}

/* One comparison of Alg. 3 after the dot products: Lift ml, ConstLift dot by
 * b = 2^16, v = a*ml' - b*dot', MSB(v) by BitExtract(v, {31}). */
void orc_mpc_compare(const orc_mpc_cfg* cfg, const uint16_t dot[3], const uint16_t ml[3],
                     uint32_t q, uint32_t rho, uint32_t i, uint8_t msb[3],
                     uint32_t ml_lift[3], uint32_t v_out[3], orc_stats* st) {
  uint64_t and0 = st->and_gates;
  /* after resharing the dot products are one round deep */
  rss_t L = lift16(cfg, ml, 1, q, rho, i, st);
  uint64_t and1 = st->and_gates;
  uint32_t dcomp[3] = {dot[0], dot[1], dot[2]};
  rss_t D = rss_from_components(dcomp, 1);
  D = const_lift(D, 1u << 16); /* lift_hd: [2^16 dot]_{2^32}, free */
  rss_t V;
  for (int p = 0; p < 3; p++) {
    V.v[p].own = cfg->thr_a * L.v[p].own - D.v[p].own;
    V.v[p].prev = cfg->thr_a * L.v[p].prev - D.v[p].prev;
  }
  V.depth = L.depth > D.depth ? L.depth : D.depth;
  gate_rng g = {cfg, i >> 5, col_tag(q, rho), ORC_D_AND, i & 31u};
  rss_t top, below;
  bit_extract_rss(&V, 31, &g, ORC_MSB_GATE0, &top, &below, st);
  for (int j = 0; j < 3; j++) {
    msb[j] = (uint8_t)rss_component(&top, j);
    if (ml_lift) ml_lift[j] = rss_component(&L, j);
    if (v_out) v_out[j] = rss_component(&V, j);
  }
  st->and_lift = (uint32_t)(and1 - and0);
  st->and_msb = (uint32_t)(st->and_gates - and1);
  st->depth_lift = L.depth - 1;
  st->depth_msb = top.depth - V.depth;
  st->depth_total = top.depth;
}

void orc_bit_extract_batch(const orc_mpc_cfg* cfg, const uint32_t* x, uint32_t n, uint32_t m, uint32_t gate0,
                           uint8_t* top, uint8_t* below) {
  orc_stats st;
  memset(&st, 0, sizeof st);
  for (uint32_t i = 0; i < n; i++)
    orc_bit_extract(cfg, x + 3 * (size_t)i, m, 0, 0, i, gate0, top + 3 * (size_t)i, below + 3 * (size_t)i, &st);
}

/* OR of two boolean sharings (Sec. 4.2): x OR y = x + y + x*y. */
static rss_t bor(rss_t a, rss_t b, uint32_t F[3], orc_stats* st) {
  return bxor(bxor(a, b), band(a, b, F, st));
}

/* One word-level OR step of the tree: lanes [0, nbits) of a with those of b,
 * AND randomness bit `lane` of word 0 of Philox(seed_j, (c0, c1, req, c3)). */
static void or_words(const orc_mpc_cfg* cfg, rss_t* a, const rss_t* b, uint32_t nbits, uint32_t c0, uint32_t c1,
                     uint32_t c3, orc_stats* st) {
  uint32_t w[3][4];
  for (int j = 0; j < 3; j++) prf(cfg->seeds[j], c0, c1, cfg->req, c3, w[j]);
  for (uint32_t lane = 0; lane < nbits; lane++) {
    uint32_t F[3] = {(w[0][0] >> lane) & 1u, (w[1][0] >> lane) & 1u, (w[2][0] >> lane) & 1u};
    a[lane] = bor(a[lane], b[lane], F, st);
  }
}

/* Pairwise tree over n words: at each level pair (2j, 2j+1) is ORed into j and
 * an odd last word moves up unchanged. */
static void or_pairwise(const orc_mpc_cfg* cfg, rss_t* words, uint32_t n, uint32_t c1, uint32_t stage,
                        orc_stats* st) {
  uint32_t level = 1;
  while (n > 1) {
    uint32_t half = n / 2;
    for (uint32_t j = 0; j < half; j++) {
      or_words(cfg, &words[(size_t)(2 * j) * 32], &words[(size_t)(2 * j + 1) * 32], 32, j, c1,
               (ORC_D_OR << 24) | (stage << 16) | level, st);
      if (j != 2 * j) memcpy(&words[(size_t)j * 32], &words[(size_t)(2 * j) * 32], 32 * sizeof(rss_t));
    }
    if (n & 1u) memmove(&words[(size_t)half * 32], &words[(size_t)(n - 1) * 32], 32 * sizeof(rss_t));
    n = half + (n & 1u);
    level++;
  }
}

/*
 * OrTree (Sec. 4.2, Alg. 3) for one query, with a fixed shape so that any
 * evaluation order gives the same shares: (1) for each rotation, the MSB bits of
 * rows 32g..32g+31 form word g (rows past s are the public 0), and the words are
 * combined by the pairwise tree; (2) the rotation words are combined by the
 * pairwise tree; (3) the 32 lanes of the last word are folded in halves.
 */
void orc_or_tree(const orc_mpc_cfg* cfg, const uint8_t* msb, uint32_t R, uint32_t s,
                 uint32_t q, uint8_t bit[3], orc_stats* st) {
  uint32_t G = (s + 31) / 32;
  if (G == 0) G = 1;
  rss_t* words = (rss_t*)calloc((size_t)G * 32, sizeof(rss_t));
  rss_t* rot = (rss_t*)calloc((size_t)R * 32, sizeof(rss_t));
  size_t plane = (size_t)R * s;
  uint32_t d0 = 0;
  for (uint32_t rho = 0; rho < R; rho++) {
    memset(words, 0, (size_t)G * 32 * sizeof(rss_t));
    for (uint32_t i = 0; i < s; i++) {
      uint32_t comp[3];
      for (int j = 0; j < 3; j++) comp[j] = msb[j * plane + (size_t)rho * s + i];
      words[i] = rss_from_components(comp, d0);
    }
    or_pairwise(cfg, words, G, col_tag(q, rho), 1, st);
    memcpy(&rot[(size_t)rho * 32], words, 32 * sizeof(rss_t));
  }
  or_pairwise(cfg, rot, R, col_tag(q, 0), 2, st);
  for (uint32_t level = 1; level <= 5; level++) {
    uint32_t h = 32u >> level;
    or_words(cfg, rot, rot + h, h, 0, col_tag(q, 0), (ORC_D_OR << 24) | (3u << 16) | level, st);
  }
  for (int j = 0; j < 3; j++) bit[j] = (uint8_t)rss_component(&rot[0], j);
  st->depth_or = rot[0].depth;
  free(words);
  free(rot);
}

typedef void (*dot_fn)(const orc_mpc_cfg*, const uint16_t*, uint64_t, const uint16_t*, uint64_t, uint32_t,
                       uint32_t, uint32_t, uint32_t, uint32_t, uint16_t[3], orc_stats*);

/* valid_rows (may be NULL): for query q, rows i >= valid_rows[q] enter q's OR tree as the
 * public 0 (all three components 0) instead of their comparison bit. */
static void mpc_match_with(dot_fn dot, const orc_mpc_cfg* cfg, const orc_geom* g,
                           const uint16_t* db_code, const uint16_t* db_mask, uint32_t s,
                           const uint16_t* q_code, const uint16_t* q_mask, uint32_t Q,
                           const uint32_t* valid_rows,
                           uint16_t* z_code, uint16_t* z_mask, uint8_t* msb_out, uint8_t* bits,
                           orc_stats* st) {
  uint32_t l = g->rows * g->cols * g->cell;
  uint32_t R = g->R;
  uint64_t db_plane = (uint64_t)s * l, q_plane = (uint64_t)Q * l;
  size_t zplane = (size_t)Q * R * s;
  /* rotated query: code components 0..2 then mask components 0..2 */
  uint16_t* ry = (uint16_t*)malloc(sizeof(uint16_t) * 6 * l);
  uint8_t* msb = (uint8_t*)malloc(3 * (size_t)R * s + 1);
  for (uint32_t q = 0; q < Q; q++) {
    for (uint32_t rho = 0; rho < R; rho++) {
      int32_t shift = g->rot_lo + (int32_t)rho;
      /* rotation is linear, so rotating each share component rotates the secret */
      for (int j = 0; j < 3; j++) {
        orc_rotate_u16(g, q_code + j * q_plane + (size_t)q * l, ry + (size_t)j * l, shift);
        orc_rotate_u16(g, q_mask + j * q_plane + (size_t)q * l, ry + (size_t)(3 + j) * l, shift);
      }
      size_t n = (size_t)q * R + rho;
      for (uint32_t i = 0; i < s; i++) {
        uint16_t zc[3], zm[3];
        dot(cfg, db_code + (size_t)i * l, db_plane, ry, l, l, q, rho, i, 0, zc, st);
        dot(cfg, db_mask + (size_t)i * l, db_plane, ry + (size_t)3 * l, l, l, q, rho, i, 1, zm, st);
        if (z_code)
          for (int p = 0; p < 3; p++) z_code[p * zplane + n * s + i] = zc[p];
        if (z_mask)
          for (int p = 0; p < 3; p++) z_mask[p * zplane + n * s + i] = zm[p];
        uint8_t b[3];
        orc_mpc_compare(cfg, zc, zm, q, rho, i, b, NULL, NULL, st);
        if (valid_rows && i >= valid_rows[q]) b[0] = b[1] = b[2] = 0;
        for (int p = 0; p < 3; p++) {
          msb[(size_t)p * R * s + (size_t)rho * s + i] = b[p];
          if (msb_out) msb_out[p * zplane + n * s + i] = b[p];
        }
      }
    }
    uint8_t bit[3];
    orc_or_tree(cfg, msb, R, s, q, bit, st);
    if (bits)
      for (int p = 0; p < 3; p++) bits[(size_t)p * Q + q] = bit[p];
  }
  free(ry);
  free(msb);
}

void orc_mpc_match(const orc_mpc_cfg* cfg, const orc_geom* g,
                   const uint16_t* db_code, const uint16_t* db_mask, uint32_t s,
                   const uint16_t* q_code, const uint16_t* q_mask, uint32_t Q,
                   uint16_t* z_code, uint16_t* z_mask, uint8_t* msb_out, uint8_t* bits,
                   orc_stats* st) {
  mpc_match_with(orc_mpc_dot, cfg, g, db_code, db_mask, s, q_code, q_mask, Q, NULL, z_code, z_mask, msb_out, bits,
                 st);
}

/* ------------------------------------------------------------------------ */
/* Galois-ring Shamir dot products (Sec. 4.3.2). GR = Z_{2^16}[X]/(X^2-X-1):  */
/* X^2 = X + 1, so                                                            */
/*   (a0 + a1 X)(b0 + b1 X) = (a0 b0 + a1 b1) + (a0 b1 + a1 b0 + a1 b1) X.   */
/* ------------------------------------------------------------------------ */
void orc_gr_mul(const uint16_t a[2], const uint16_t b[2], uint16_t out[2]) {
  uint32_t a0 = a[0], a1 = a[1], b0 = b[0], b1 = b[1];
  uint32_t x2 = a1 * b1; /* the X^2 term, folded into both coefficients */
  out[0] = (uint16_t)(a0 * b0 + x2);
  out[1] = (uint16_t)(a0 * b1 + a1 * b0 + x2);
}

/* Inverse of an odd n modulo 2^16 by Newton's iteration x <- x (2 - n x), which doubles the
 * number of correct low bits; x = n is right to 3 bits since n^2 = 1 (mod 8) for odd n. */
static uint16_t inv_odd16(uint16_t n) {
  uint32_t x = n;
  for (int it = 0; it < 4; it++) x = x * (2u - n * x);
  return (uint16_t)x;
}

/* The conjugate maps X to the other root 1 - X of X^2 - X - 1; a * conj(a) is the norm
 * N = a0^2 + a0 a1 - a1^2 in Z_{2^16}, and a is a unit iff N is (i.e. N odd). */
int orc_gr_inv(const uint16_t a[2], uint16_t out[2]) {
  uint16_t conj[2] = {(uint16_t)(a[0] + a[1]), (uint16_t)(0u - a[1])};
  uint16_t nrm[2];
  orc_gr_mul(a, conj, nrm);
  if (nrm[1] != 0 || (nrm[0] & 1u) == 0) return 0;
  uint16_t ninv[2] = {inv_odd16(nrm[0]), 0};
  orc_gr_mul(conj, ninv, out);
  return 1;
}

static void gr_sub(const uint16_t a[2], const uint16_t b[2], uint16_t out[2]) {
  out[0] = (uint16_t)(a[0] - b[0]);
  out[1] = (uint16_t)(a[1] - b[1]);
}

void orc_gr_points(uint16_t alpha[6]) {
  alpha[0] = 1; alpha[1] = 0; /* 1     */
  alpha[2] = 0; alpha[3] = 1; /* X     */
  alpha[4] = 1; alpha[5] = 1; /* 1 + X */
}

/* lambda_p = prod_{j != p} alpha_j / (alpha_j - alpha_p) */
void orc_gr_lagrange(uint16_t lambda[6]) {
  uint16_t alpha[6];
  orc_gr_points(alpha);
  for (int p = 0; p < 3; p++) {
    uint16_t acc[2] = {1, 0};
    for (int j = 0; j < 3; j++) {
      if (j == p) continue;
      uint16_t diff[2], inv[2], t[2];
      gr_sub(alpha + 2 * j, alpha + 2 * p, diff);
      if (!orc_gr_inv(diff, inv)) abort(); /* the points are exceptional: differences are units */
      orc_gr_mul(alpha + 2 * j, inv, t);
      orc_gr_mul(acc, t, acc);
    }
    lambda[2 * p] = acc[0];
    lambda[2 * p + 1] = acc[1];
  }
}

void orc_encode_share_galois(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                             uint64_t client_seed, uint32_t side, uint32_t idx0,
                             uint16_t* code_sh, uint16_t* mask_sh) {
  uint32_t nw = (l + 63) / 64;
  size_t plane = (size_t)n * l;
  uint16_t alpha[6];
  orc_gr_points(alpha);
  for (uint32_t r = 0; r < n; r++) {
    const uint64_t* c = code_bits + (size_t)r * nw;
    const uint64_t* m = mask_bits + (size_t)r * nw;
    uint32_t w[2][4];
    for (uint32_t e = 0; 2 * e < l; e++) {
      uint16_t val[2][2]; /* [vec][coefficient]: bits 2e and 2e+1 */
      for (uint32_t t = 0; t < 2; t++) {
        int cb = get_bit(c, 2 * e + t), mb = get_bit(m, 2 * e + t);
        val[0][t] = (uint16_t)(mb - 2 * (cb & mb)); /* masked bit (Sec. 4.1.1) */
        val[1][t] = (uint16_t)mb;
      }
      if ((e & 3u) == 0)
        for (uint32_t vec = 0; vec < 2; vec++)
          prf(client_seed, e >> 2, idx0 + r, (side << 8) | vec, ORC_D_GSHARE << 24, w[vec]);
      for (uint32_t vec = 0; vec < 2; vec++) {
        uint16_t rnd[2] = {(uint16_t)(w[vec][e & 3] & 0xFFFFu), (uint16_t)(w[vec][e & 3] >> 16)};
        uint16_t* dst = vec == 0 ? code_sh : mask_sh;
        for (int p = 0; p < 3; p++) {
          uint16_t ra[2]; /* share_p = g + r alpha_p */
          orc_gr_mul(rnd, alpha + 2 * p, ra);
          size_t at = (size_t)p * plane + (size_t)r * l + 2 * e;
          dst[at] = (uint16_t)(val[vec][0] + ra[0]);
          dst[at + 1] = (uint16_t)(val[vec][1] + ra[1]);
        }
      }
    }
  }
}

void orc_mpc_dot_galois(const orc_mpc_cfg* cfg, const uint16_t* x, uint64_t x_stride,
                        const uint16_t* y, uint64_t y_stride, uint32_t l,
                        uint32_t q, uint32_t rho, uint32_t i, uint32_t vec, uint16_t z[3], orc_stats* st) {
  uint16_t lambda[6];
  orc_gr_lagrange(lambda);
  for (int p = 0; p < 3; p++) {
    const uint16_t* xp = x + (size_t)p * x_stride;
    const uint16_t* yp = y + (size_t)p * y_stride;
    uint32_t acc = 0;
    for (uint32_t e = 0; 2 * e < l; e++) {
      uint16_t a[2], prod[2];
      orc_gr_mul(lambda + 2 * p, yp + 2 * e, a); /* the query share times lambda_p */
      orc_gr_mul(a, xp + 2 * e, prod);           /* its product with the DB share: keep the constant term */
      acc += prod[0];
    }
    uint32_t r = za_value(cfg->seeds[p], cfg->req, q, rho, i, vec) - za_value(cfg->seeds[P(p - 1)], cfg->req, q, rho, i, vec);
    z[p] = (uint16_t)(acc + r);
    if (st) st->bits_sent[p] += 16; /* resharing: z_p to party p+1 */
  }
}

void orc_mpc_match_galois(const orc_mpc_cfg* cfg, const orc_geom* g,
                          const uint16_t* db_code, const uint16_t* db_mask, uint32_t s,
                          const uint16_t* q_code, const uint16_t* q_mask, uint32_t Q,
                          uint16_t* z_code, uint16_t* z_mask, uint8_t* msb_out, uint8_t* bits,
                          orc_stats* st) {
  if (g->cell % 2 != 0) abort(); /* element pairs must not straddle rotated cells */
  mpc_match_with(orc_mpc_dot_galois, cfg, g, db_code, db_mask, s, q_code, q_mask, Q, NULL, z_code, z_mask, msb_out,
                 bits, st);
}

/* ------------------------------------------------------------------------ */
/* Both eyes and inner-batch matching (Sec. 5.4).                            */
/* ------------------------------------------------------------------------ */
void orc_mpc_match_batch(const orc_mpc_cfg* cfg, const orc_geom* g, int galois,
                         const uint16_t* q_code, const uint16_t* q_mask, uint32_t P, uint8_t* bits,
                         orc_stats* st) {
  uint32_t* valid = (uint32_t*)malloc(sizeof(uint32_t) * (P ? P : 1));
  for (uint32_t q = 0; q < P; q++) valid[q] = q; /* persons before q in the batch */
  mpc_match_with(galois ? orc_mpc_dot_galois : orc_mpc_dot, cfg, g, q_code, q_mask, P, q_code, q_mask, P, valid,
                 NULL, NULL, NULL, bits, st);
  free(valid);
}

void orc_or_combine(const orc_mpc_cfg* cfg, const uint8_t* bits4, uint32_t P, uint8_t* out, orc_stats* st) {
  size_t part = 3 * (size_t)P;
  for (uint32_t p = 0; p < P; p++) {
    rss_t b[4];
    for (int k = 0; k < 4; k++) {
      uint32_t comp[3];
      for (int j = 0; j < 3; j++) comp[j] = bits4[k * part + (size_t)j * P + p];
      b[k] = rss_from_components(comp, 0);
    }
    rss_t r[3];
    for (uint32_t t = 0; t < 3; t++) {
      uint32_t w[3][4], F[3];
      for (int j = 0; j < 3; j++) {
        prf(cfg->seeds[j], p, 0, cfg->req, (ORC_D_COMB << 24) | t, w[j]);
        F[j] = w[j][0] & 1u;
      }
      rss_t x = t == 0 ? b[0] : (t == 1 ? b[2] : r[0]);
      rss_t y = t == 0 ? b[1] : (t == 1 ? b[3] : r[1]);
      r[t] = bor(x, y, F, st);
    }
    for (int j = 0; j < 3; j++) out[(size_t)j * P + p] = (uint8_t)(rss_component(&r[2], j) & 1u);
  }
}

/* ------------------------------------------------------------------------ */
/* Protocol 1 (Sec. 4, Alg. 2): shared codes, public masks.                  */
/* ------------------------------------------------------------------------ */
void orc_mpc_compare_plain(const orc_mpc_cfg* cfg, const uint16_t dot[3], uint32_t ml, uint32_t q, uint32_t rho,
                           uint32_t i, uint8_t msb[3], orc_stats* st) {
  uint32_t t = (uint32_t)(((uint64_t)cfg->thr_a * ml) >> 16); /* floor(f ml), f = a / 2^16 */
  /* public t enters through component 0; the dot product is reshared (one round deep) */
  uint32_t v[3] = {(t - dot[0]) & 0xFFFFu, (0u - dot[1]) & 0xFFFFu, (0u - dot[2]) & 0xFFFFu};
  rss_t V = rss_from_components(v, 1);
  gate_rng g = {cfg, i >> 5, col_tag(q, rho), ORC_D_AND, i & 31u};
  rss_t top, below;
  uint64_t and0 = st->and_gates;
  bit_extract_rss(&V, 15, &g, 0, &top, &below, st);
  for (int j = 0; j < 3; j++) msb[j] = (uint8_t)rss_component(&top, j);
  st->and_msb = (uint32_t)(st->and_gates - and0);
  st->depth_msb = top.depth - V.depth;
  st->depth_total = top.depth;
}

void orc_mpc_match_plain(const orc_mpc_cfg* cfg, const orc_geom* g, int galois,
                         const uint16_t* db_code, const uint64_t* db_mask_bits, uint32_t s,
                         const uint16_t* q_code, const uint64_t* q_mask_bits, uint32_t Q,
                         uint16_t* z_code, uint16_t* ml_out, uint8_t* bits, orc_stats* st) {
  uint32_t l = g->rows * g->cols * g->cell, nw = (l + 63) / 64, R = g->R;
  uint64_t db_plane = (uint64_t)s * l, q_plane = (uint64_t)Q * l;
  size_t zplane = (size_t)Q * R * s;
  dot_fn dot = galois ? orc_mpc_dot_galois : orc_mpc_dot;
  uint16_t* ry = (uint16_t*)malloc(sizeof(uint16_t) * 3 * l);
  uint64_t* rm = (uint64_t*)malloc(sizeof(uint64_t) * nw);
  uint8_t* msb = (uint8_t*)malloc(3 * (size_t)R * s + 1);
  for (uint32_t q = 0; q < Q; q++) {
    for (uint32_t rho = 0; rho < R; rho++) {
      int32_t shift = g->rot_lo + (int32_t)rho;
      for (int j = 0; j < 3; j++)
        orc_rotate_u16(g, q_code + j * q_plane + (size_t)q * l, ry + (size_t)j * l, shift);
      orc_rotate_bits(g, q_mask_bits + (size_t)q * nw, rm, shift);
      size_t n = (size_t)q * R + rho;
      for (uint32_t i = 0; i < s; i++) {
        uint16_t zc[3];
        dot(cfg, db_code + (size_t)i * l, db_plane, ry, l, l, q, rho, i, 0, zc, st);
        uint32_t ml = 0; /* public: CountOnes(rot(m) AND M_i) */
        for (uint32_t w = 0; w < nw; w++) ml += (uint32_t)popcount64(rm[w] & db_mask_bits[(size_t)i * nw + w]);
        if (z_code)
          for (int p = 0; p < 3; p++) z_code[p * zplane + n * s + i] = zc[p];
        if (ml_out) ml_out[n * s + i] = (uint16_t)ml;
        uint8_t b[3];
        orc_mpc_compare_plain(cfg, zc, ml, q, rho, i, b, st);
        for (int p = 0; p < 3; p++) msb[(size_t)p * R * s + (size_t)rho * s + i] = b[p];
      }
    }
    uint8_t bit[3];
    orc_or_tree(cfg, msb, R, s, q, bit, st);
    if (bits)
      for (int p = 0; p < 3; p++) bits[(size_t)p * Q + q] = bit[p];
  }
  free(ry);
  free(rm);
  free(msb);
}

/* ------------------------------------------------------------------------ */
/* Lifting variants (Sec. 5.1, Sec. 6.2 Table 2): ConstLift and NoLift.      */
/* ------------------------------------------------------------------------ */
void orc_encode_share32(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                        uint64_t client_seed, uint32_t side, uint32_t idx0, uint32_t* code_sh, uint32_t* mask_sh) {
  uint32_t nw = (l + 63) / 64;
  size_t plane = (size_t)n * l;
  for (uint32_t r = 0; r < n; r++) {
    const uint64_t* c = code_bits + (size_t)r * nw;
    const uint64_t* m = mask_bits + (size_t)r * nw;
    for (uint32_t b = 0; b < l; b++) {
      int cb = get_bit(c, b), mb = get_bit(m, b);
      uint32_t val[2] = {(uint32_t)(mb - 2 * (cb & mb)), (uint32_t)mb}; /* masked bit (Sec. 4.1.1) and mask */
      for (uint32_t vec = 0; vec < 2; vec++) {
        uint32_t w[4];
        prf(client_seed, b >> 1, idx0 + r, (side << 8) | vec, ORC_D_SHARE32 << 24, w);
        uint32_t x0 = w[2 * (b & 1u)], x1 = w[2 * (b & 1u) + 1];
        uint32_t* dst = vec == 0 ? code_sh : mask_sh;
        size_t at = (size_t)r * l + b;
        dst[at] = x0;
        dst[plane + at] = x1;
        dst[2 * plane + at] = val[vec] - x0 - x1;
      }
    }
  }
}

static uint32_t za32_value(uint64_t seed, uint32_t req, uint32_t q, uint32_t rho, uint32_t i, uint32_t vec) {
  uint32_t w[4];
  prf(seed, i >> 2, col_tag(q, rho), req, (ORC_D_ZA32 << 24) | vec, w);
  return w[i & 3u];
}

/* App. C over Z_{2^32}: z_i = x_i y_i + x_{i-1} y_i + x_i y_{i-1} + r_i. */
void orc_mpc_dot32(const orc_mpc_cfg* cfg, const uint32_t* x, uint64_t x_stride, const uint32_t* y,
                   uint64_t y_stride, uint32_t l, uint32_t q, uint32_t rho, uint32_t i, uint32_t vec, uint32_t z[3],
                   orc_stats* st) {
  for (int p = 0; p < 3; p++) {
    const uint32_t* xp = x + (size_t)p * x_stride;
    const uint32_t* xm = x + (size_t)P(p - 1) * x_stride;
    const uint32_t* yp = y + (size_t)p * y_stride;
    const uint32_t* ym = y + (size_t)P(p - 1) * y_stride;
    uint32_t acc = 0;
    for (uint32_t k = 0; k < l; k++) acc += xp[k] * yp[k] + xm[k] * yp[k] + xp[k] * ym[k];
    z[p] = acc + za32_value(cfg->seeds[p], cfg->req, q, rho, i, vec) -
           za32_value(cfg->seeds[P(p - 1)], cfg->req, q, rho, i, vec);
    if (st) st->bits_sent[p] += 32; /* resharing: z_p to party p+1 */
  }
}

void orc_mpc_compare_liftfree(const orc_mpc_cfg* cfg, int mode, const uint32_t dot[3], const uint32_t ml[3],
                              uint32_t thr_b, uint32_t q, uint32_t rho, uint32_t i, uint8_t msb[3],
                              uint32_t v_out[3], orc_stats* st) {
  /* ml is already a sharing over Z_{2^32}: no Lift */
  rss_t L = rss_from_components(ml, 1);
  rss_t D;
  if (mode == ORC_LIFT_CONST) {
    uint32_t d16[3] = {dot[0] & 0xFFFFu, dot[1] & 0xFFFFu, dot[2] & 0xFFFFu};
    D = const_lift(rss_from_components(d16, 1), 1u << 16); /* [2^16 dot]_{2^32}, free */
  } else {
    uint32_t b = (thr_b == 0) ? (1u << 16) : thr_b;
    D = rss_from_components(dot, 1);
    for (int p = 0; p < 3; p++) { /* multiplication by a public constant is local */
      D.v[p].own *= b;
      D.v[p].prev *= b;
    }
  }
  rss_t V;
  for (int p = 0; p < 3; p++) {
    V.v[p].own = cfg->thr_a * L.v[p].own - D.v[p].own;
    V.v[p].prev = cfg->thr_a * L.v[p].prev - D.v[p].prev;
  }
  V.depth = 1;
  gate_rng g = {cfg, i >> 5, col_tag(q, rho), ORC_D_AND, i & 31u};
  rss_t top, below;
  uint64_t and0 = st->and_gates;
  bit_extract_rss(&V, 31, &g, ORC_MSB_GATE0, &top, &below, st);
  for (int j = 0; j < 3; j++) {
    msb[j] = (uint8_t)rss_component(&top, j);
    if (v_out) v_out[j] = rss_component(&V, j);
  }
  st->and_lift = 0;
  st->and_msb = (uint32_t)(st->and_gates - and0);
  st->depth_lift = 0;
  st->depth_msb = top.depth - V.depth;
  st->depth_total = top.depth;
}

static void rotate_u32(const orc_geom* g, const uint32_t* in, uint32_t* out, int32_t shift) {
  for (uint32_t r = 0; r < g->rows; r++)
    for (uint32_t j = 0; j < g->cols; j++)
      for (uint32_t k = 0; k < g->cell; k++)
        out[(r * g->cols + j) * g->cell + k] = in[(r * g->cols + src_col(g, j, shift)) * g->cell + k];
}

void orc_mpc_match_lift(const orc_mpc_cfg* cfg, const orc_geom* g, int mode, uint32_t thr_b,
                        const void* db_code, const uint32_t* db_mask, uint32_t s, const void* q_code,
                        const uint32_t* q_mask, uint32_t Q, void* z_code, uint32_t* z_mask, uint8_t* bits,
                        orc_stats* st) {
  uint32_t l = g->rows * g->cols * g->cell, R = g->R;
  uint64_t db_plane = (uint64_t)s * l, q_plane = (uint64_t)Q * l;
  size_t zplane = (size_t)Q * R * s;
  int wide = mode == ORC_LIFT_NONE; /* code shares over Z_{2^32} */
  uint32_t* ry = (uint32_t*)malloc(sizeof(uint32_t) * 6 * l); /* rotated query: code 0..2, mask 0..2 */
  uint16_t* ry16 = (uint16_t*)malloc(sizeof(uint16_t) * 3 * l);
  uint8_t* msb = (uint8_t*)malloc(3 * (size_t)R * s + 1);
  for (uint32_t q = 0; q < Q; q++) {
    for (uint32_t rho = 0; rho < R; rho++) {
      int32_t shift = g->rot_lo + (int32_t)rho;
      for (int j = 0; j < 3; j++) {
        if (wide)
          rotate_u32(g, (const uint32_t*)q_code + j * q_plane + (size_t)q * l, ry + (size_t)j * l, shift);
        else
          orc_rotate_u16(g, (const uint16_t*)q_code + j * q_plane + (size_t)q * l, ry16 + (size_t)j * l, shift);
        rotate_u32(g, q_mask + j * q_plane + (size_t)q * l, ry + (size_t)(3 + j) * l, shift);
      }
      size_t n = (size_t)q * R + rho;
      for (uint32_t i = 0; i < s; i++) {
        uint32_t zc[3], zm[3];
        if (wide) {
          orc_mpc_dot32(cfg, (const uint32_t*)db_code + (size_t)i * l, db_plane, ry, l, l, q, rho, i, 0, zc, st);
        } else {
          uint16_t z16[3];
          orc_mpc_dot(cfg, (const uint16_t*)db_code + (size_t)i * l, db_plane, ry16, l, l, q, rho, i, 0, z16, st);
          for (int p = 0; p < 3; p++) zc[p] = z16[p];
        }
        orc_mpc_dot32(cfg, db_mask + (size_t)i * l, db_plane, ry + (size_t)3 * l, l, l, q, rho, i, 1, zm, st);
        for (int p = 0; p < 3; p++) {
          size_t at = p * zplane + n * s + i;
          if (z_code) {
            if (wide)
              ((uint32_t*)z_code)[at] = zc[p];
            else
              ((uint16_t*)z_code)[at] = (uint16_t)zc[p];
          }
          if (z_mask) z_mask[at] = zm[p];
        }
        uint8_t b[3];
        orc_mpc_compare_liftfree(cfg, mode, zc, zm, thr_b, q, rho, i, b, NULL, st);
        for (int p = 0; p < 3; p++) msb[(size_t)p * R * s + (size_t)rho * s + i] = b[p];
      }
    }
    uint8_t bit[3];
    orc_or_tree(cfg, msb, R, s, q, bit, st);
    if (bits)
      for (int p = 0; p < 3; p++) bits[(size_t)p * Q + q] = bit[p];
  }
  free(ry);
  free(ry16);
  free(msb);
}

/* ------------------------------------------------------------------------ */
/* Transcript hash.                                                          */
/* ------------------------------------------------------------------------ */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t msg_hash(uint64_t kind, uint64_t party, uint64_t col, uint64_t row, uint64_t v) {
  uint64_t key = (kind << 60) | (party << 58) | (col << 32) | row;
  return orc_mix64(orc_mix64(key) + v);
}

static uint64_t elem(const void* base, uint32_t bytes, size_t at) {
  return bytes == 4 ? ((const uint32_t*)base)[at] : ((const uint16_t*)base)[at];
}

uint64_t orc_transcript_hash(const void* z_code, uint32_t elem_code, const void* z_mask, uint32_t elem_mask,
                             uint32_t n_cols, uint32_t s, const uint8_t* bits, uint32_t Q) {
  uint64_t h = 0;
  for (uint32_t p = 0; p < 3; p++)
    for (uint32_t n = 0; n < n_cols; n++)
      for (uint32_t i = 0; i < s; i++) {
        size_t at = ((size_t)p * n_cols + n) * s + i;
        h ^= msg_hash(0, p, n, i, elem(z_code, elem_code, at));
        if (z_mask) h ^= msg_hash(1, p, n, i, elem(z_mask, elem_mask, at));
      }
  for (uint32_t p = 0; p < 3; p++)
    for (uint32_t q = 0; q < Q; q++) h ^= msg_hash(2, p, q, 0, bits[(size_t)p * Q + q]);
  return h;
}
