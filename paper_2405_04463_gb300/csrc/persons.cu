// Both eyes and inner-batch matching (Sec. 5.4): a query is a person's two iris codes, each
// checked (31 rotations) against the database of the same eye, and the persons of a batch are
// also matched with each other so that the batch itself holds no duplicates.
//
// Per person p the result is (db_0 OR db_1) OR (batch_0 OR batch_1):
//   db_e     the person's eye-e code against the eye-e database (the context's request path);
//   batch_e  the eye-e code (all rotations) against the unrotated eye-e codes of the persons
//            p' < p of the batch: the batch's own shares act as database rows, and rows
//            p' >= p enter p's OR tree as the public 0, so of two duplicates the earlier passes.
// Every part has its own request id, so no two parts share a PRF counter.
#include "context.cuh"

namespace ipc {
int or_combine_launch(const uint8_t* const bits[4], uint32_t P, uint32_t req, const uint64_t seeds[3], uint8_t* out,
                      cudaStream_t st);
}  // namespace ipc

using namespace ipc;

namespace {

// The two contexts share seeds, so every part must draw a distinct request id: both counters
// are moved to a common value n; the parts then take n .. n+4 (the database parts through
// submit_queries on each context in turn) and both counters continue after them.
uint64_t align_ids(ipc_ctx* a, ipc_ctx* b) {
  std::lock_guard<std::mutex> la(a->id_mu);
  std::lock_guard<std::mutex> lb(b->id_mu);
  const uint64_t n = std::max(a->next_id, b->next_id);
  a->next_id = b->next_id = n;
  return n;
}

void set_next(ipc_ctx* c, uint64_t v) {
  std::lock_guard<std::mutex> lock(c->id_mu);
  c->next_id = std::max(c->next_id, v);
}

// Device buffers of one eye's inner-batch part, freed on scope exit.
struct BatchBuffers {
  uint16_t* y = nullptr;      // [vec][3][P][l] query shares
  uint8_t* planes = nullptr;  // [comp][vec][limb][P][l] limbs (the batch as database rows)
  uint8_t* bq = nullptr;      // [party][vec][limb][n_pad][kq] limbs
  uint32_t* tags = nullptr;   // [N][2]
  uint32_t* col_rows = nullptr;
  uint16_t* z = nullptr;      // [vec][party][N][ldz]
  uint32_t* roots = nullptr;  // [3][N][nb]
  uint8_t* bits = nullptr;    // [3][P]
  ~BatchBuffers() {
    cudaFree(y);
    cudaFree(planes);
    cudaFree(bq);
    cudaFree(tags);
    cudaFree(col_rows);
    cudaFree(z);
    cudaFree(roots);
    cudaFree(bits);
  }
};

#define P_TRY(expr)                                     \
  do {                                                  \
    cudaError_t e__ = (expr);                           \
    if (e__ != cudaSuccess) return ctx_cfail(c, e__, #expr); \
  } while (0)
#define P_RC(expr)                     \
  do {                                 \
    int rc__ = (expr);                 \
    if (rc__ != IPC_OK) {              \
      c->err = thread_last_error();    \
      return rc__;                     \
    }                                  \
  } while (0)

// The inner-batch part of one eye on context c (its path, geometry and seeds), synchronous on
// c's control stream. Output: bit components [3][P] in bb.bits.
int batch_part(ipc_ctx* c, const uint16_t* const code[3], const uint16_t* const mask[3], uint32_t P, int src_is_device,
               uint64_t req, BatchBuffers& bb) {
  const ipc_geom& g = c->cfg.geom;
  const uint32_t l = c->l, R = g.R, N = P * R;
  const uint32_t n_pad = (N + 127) / 128 * 128;
  const size_t ldz = (P + 7) / 8 * 8;
  const uint32_t nb = (P + 1023) / 1024;  // 1024-row OR blocks
  const size_t qsz = c->qsz, kq = c->kq;
  const size_t plane_bytes = (static_cast<size_t>(P) * l + 15) / 16 * 16;  // int8 limb planes
  const size_t qplane = static_cast<size_t>(n_pad) * kq * qsz;
  const bool ok = cudaMalloc(&bb.y, 6ull * P * l * sizeof(uint16_t)) == cudaSuccess &&
                  cudaMalloc(&bb.planes, 12 * plane_bytes) == cudaSuccess &&
                  cudaMalloc(&bb.bq, 12 * qplane) == cudaSuccess &&
                  cudaMalloc(&bb.tags, 2ull * N * sizeof(uint32_t)) == cudaSuccess &&
                  cudaMalloc(&bb.col_rows, static_cast<size_t>(N) * sizeof(uint32_t)) == cudaSuccess &&
                  cudaMalloc(&bb.z, 6ull * N * ldz * sizeof(uint16_t)) == cudaSuccess &&
                  cudaMalloc(&bb.roots, 3ull * N * nb * sizeof(uint32_t)) == cudaSuccess &&
                  cudaMalloc(&bb.bits, 3ull * P) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return ctx_fail(c, IPC_ENOMEM, "ipc_check_persons: device memory for the inner-batch part");
  }
  cudaStream_t st = c->sc;
  if (src_is_device) {
    P_TRY(cudaEventRecord(c->ev_input, c->input_stream));
    P_TRY(cudaStreamWaitEvent(st, c->ev_input, 0));
  }
  const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int vec = 0; vec < 2; ++vec)
    for (int j = 0; j < 3; ++j)
      P_TRY(cudaMemcpyAsync(bb.y + (static_cast<size_t>(vec) * 3 + j) * P * l, vec == 0 ? code[j] : mask[j],
                            static_cast<size_t>(P) * l * sizeof(uint16_t), kind, st));
  std::vector<uint32_t> tags(2ull * N), rows(N);
  for (uint32_t n = 0; n < N; ++n) {
    tags[2 * n] = static_cast<uint32_t>(req);
    tags[2 * n + 1] = ((n / R) << 5) | (n % R);
    rows[n] = n / R;  // query q meets the persons before it
  }
  P_TRY(cudaMemcpyAsync(bb.tags, tags.data(), tags.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  P_TRY(cudaMemcpyAsync(bb.col_rows, rows.data(), rows.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  auto pl = [&](int comp, int vec, int limb) { return bb.planes + ((comp * 2 + vec) * 2 + limb) * plane_bytes; };
  auto bq = [&](int party, int vec, int limb) { return bb.bq + ((party * 2 + vec) * 2 + limb) * qplane; };
  // A1: the batch's shares as database limb planes
  for (int vec = 0; vec < 2; ++vec)
    for (int j = 0; j < 3; ++j) {
      const uint16_t* x = bb.y + (static_cast<size_t>(vec) * 3 + j) * P * l;
      P_RC(ipc_split_limbs(x, static_cast<size_t>(P) * l, reinterpret_cast<int8_t*>(pl(j, vec, 0)),
                           reinterpret_cast<int8_t*>(pl(j, vec, 1)), st));
    }
  // A2 and A3 per party and vector
  uint16_t* zc[3];
  uint16_t* zm[3];
  for (int i = 0; i < 3; ++i) {
    zc[i] = bb.z + (static_cast<size_t>(0) * 3 + i) * N * ldz;
    zm[i] = bb.z + (static_cast<size_t>(1) * 3 + i) * N * ldz;
  }
  for (int i = 0; i < 3; ++i) {
    const int prev = (i + 2) % 3;
    for (int vec = 0; vec < 2; ++vec) {
      const uint16_t* y = bb.y + static_cast<size_t>(vec) * 3 * P * l;
      uint16_t* zo = vec == 0 ? zc[i] : zm[i];
      auto p16 = [](const uint8_t* p) { return reinterpret_cast<const uint16_t*>(p); };
      auto p8 = [](const uint8_t* p) { return reinterpret_cast<const int8_t*>(p); };
      if (c->cfg.path == IPC_PATH_TCG) {
        P_RC(ipc_prep_query_galois(y, P, &g, i, reinterpret_cast<uint16_t*>(bq(i, vec, 0)),
                                   reinterpret_cast<uint16_t*>(bq(i, vec, 1)), n_pad, st));
        const int8_t* xl[2] = {p8(pl(i, vec, 0)), p8(pl(i, vec, 0))};
        const int8_t* xh[2] = {p8(pl(i, vec, 1)), p8(pl(i, vec, 1))};
        P_RC(ring_gemm_tc_variant(256, 1, xl, xh, P, p16(bq(i, vec, 0)), p16(bq(i, vec, 1)), N, n_pad, l, bb.tags,
                                  c->cfg.seeds[i], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo, ldz, 0,
                                  nullptr, nullptr, st));
      } else if (c->cfg.path == IPC_PATH_TC) {
        P_RC(ipc_prep_query_f16(y, P, &g, i, reinterpret_cast<uint16_t*>(bq(i, vec, 0)),
                                reinterpret_cast<uint16_t*>(bq(i, vec, 1)), n_pad, st));
        const int8_t* xl[2] = {p8(pl(i, vec, 0)), p8(pl(prev, vec, 0))};
        const int8_t* xh[2] = {p8(pl(i, vec, 1)), p8(pl(prev, vec, 1))};
        P_RC(ipc_ring_gemm_tc(xl, xh, P, p16(bq(i, vec, 0)), p16(bq(i, vec, 1)), N, n_pad, l, bb.tags, c->cfg.seeds[i],
                              c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo, ldz, 0, st));
      } else {
        P_RC(ipc_prep_query(y, P, &g, i, reinterpret_cast<int8_t*>(bq(i, vec, 0)),
                            reinterpret_cast<int8_t*>(bq(i, vec, 1)), n_pad, st));
        const int8_t* xl[2] = {p8(pl(i, vec, 0)), p8(pl(prev, vec, 0))};
        const int8_t* xh[2] = {p8(pl(i, vec, 1)), p8(pl(prev, vec, 1))};
        P_RC(ipc_ring_gemm(c->cfg.path, xl, xh, P, p8(bq(i, vec, 0)), p8(bq(i, vec, 1)), N, n_pad, l, bb.tags,
                           c->cfg.seeds[i], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo, ldz, 0, st));
      }
    }
  }
  // A4-A8 with the rows of later persons as public zeros, then the rest of the OR tree
  const uint16_t* zcc[3] = {zc[0], zc[1], zc[2]};
  const uint16_t* zmc[3] = {zm[0], zm[1], zm[2]};
  P_RC(compare_launch_tiles(zcc, zmc, ldz, N, P, 0, bb.tags, c->cfg.seeds, c->cfg.thr_a, kLog2BlockWords, bb.roots, nb,
                            nullptr, 0, nullptr, nullptr, 0, st, bb.col_rows, c->cfg.plain_mask != 0));
  P_RC(ipc_or_finalize(bb.roots, nb, nb, kLog2BlockWords, P, R, bb.tags, c->cfg.seeds, bb.bits, st));
  return IPC_OK;
}

}  // namespace

extern "C" int ipc_check_persons(ipc_ctx* const ctx[2], const uint16_t* const code[6], const uint16_t* const mask[6],
                                 uint32_t P, int src_is_device, uint8_t* shares_out, uint64_t req_ids[5],
                                 int timeout_ms) {
  if (!ctx || !ctx[0] || !ctx[1] || !code || !mask || !shares_out || !req_ids)
    return ctx_fail(ctx ? ctx[0] : nullptr, IPC_EINVAL, "ipc_check_persons: null argument");
  ipc_ctx* c = ctx[0];
  const ipc_config &a = ctx[0]->cfg, &b = ctx[1]->cfg;
  if (a.path != b.path || a.device != b.device || std::memcmp(&a.geom, &b.geom, sizeof a.geom) != 0 ||
      std::memcmp(a.seeds, b.seeds, sizeof a.seeds) != 0 || a.thr_a != b.thr_a)
    return ctx_fail(c, IPC_EINVAL, "ipc_check_persons: the two eyes' contexts must share path, geometry and seeds");
  if (ctx[0]->srv || ctx[1]->srv) return ctx_fail(c, IPC_EINVAL, "ipc_check_persons: a context is serving");
  if (ctx[0] == ctx[1]) return ctx_fail(c, IPC_EINVAL, "ipc_check_persons: one context per eye");
  if (a.plain_mask || b.plain_mask) return ctx_fail(c, IPC_EINVAL, "ipc_check_persons: protocol 1 is not supported");
  if (a.lift || b.lift) return ctx_fail(c, IPC_EINVAL, "ipc_check_persons: the lifting variants are not supported");
  if (P == 0 || P > a.max_queries || P > b.max_queries)
    return ctx_fail(c, IPC_EINVAL, "ipc_check_persons: P must be in 1..max_queries");
  for (int k = 0; k < 6; ++k)
    if (!code[k] || !mask[k]) return ctx_fail(c, IPC_EINVAL, "ipc_check_persons: null component");
  // database parts, one request per eye (asynchronous); ids n (eye 0) and n + 1 (eye 1)
  const uint64_t n0 = align_ids(ctx[0], ctx[1]);
  uint64_t rid[2];
  for (int e = 0; e < 2; ++e) {
    set_next(ctx[e], n0 + e);
    int rc = submit_queries(ctx[e], code + 3 * e, mask + 3 * e, P, src_is_device, &rid[e]);
    if (rc) {
      if (e == 1) ipc_release(ctx[0], rid[0]);
      return rc;
    }
  }
  // inner-batch parts: ids n + 2, n + 3; the combination: n + 4
  BatchBuffers bb[2];
  uint64_t req_b[2];
  for (int e = 0; e < 2; ++e) {
    ipc_ctx* ce = ctx[e];
    req_b[e] = n0 + 2 + e;
    int rc = batch_part(ce, code + 3 * e, mask + 3 * e, P, src_is_device, req_b[e], bb[e]);
    if (rc) {
      ipc_release(ctx[0], rid[0]);
      ipc_release(ctx[1], rid[1]);
      return rc;
    }
  }
  // database bits (waits for the requests), then the per-person OR on the device
  std::vector<uint8_t> host(6ull * P);
  int fetch_rc = IPC_OK;
  for (int e = 0; e < 2; ++e) {  // both requests are released whatever happens
    const int rc = fetch_rc ? fetch_rc : fetch_bit_shares(ctx[e], rid[e], host.data() + 3ull * P * e, P, timeout_ms);
    ipc_release(ctx[e], rid[e]);
    fetch_rc = rc;
  }
  if (fetch_rc) return fetch_rc;
  uint8_t* dev = nullptr;
  if (cudaMalloc(&dev, 12ull * P) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, IPC_ENOMEM, "ipc_check_persons: device memory for the combination");
  }
  struct Free {
    uint8_t* p;
    ~Free() { cudaFree(p); }
  } guard{dev};
  const uint64_t req_c = n0 + 4;
  set_next(ctx[0], n0 + 5);
  set_next(ctx[1], n0 + 5);
  cudaStream_t st = c->sc;
  P_TRY(cudaMemcpyAsync(dev, host.data(), 6ull * P, cudaMemcpyHostToDevice, st));
  // the second eye's batch part ran on its own context's control stream
  cudaEvent_t done_b1 = nullptr;
  P_TRY(cudaEventCreateWithFlags(&done_b1, cudaEventDisableTiming));
  struct FreeEv {
    cudaEvent_t e;
    ~FreeEv() { cudaEventDestroy(e); }
  } guard_ev{done_b1};
  P_TRY(cudaEventRecord(done_b1, ctx[1]->sc));
  P_TRY(cudaStreamWaitEvent(st, done_b1, 0));
  const uint8_t* parts[4] = {dev, dev + 3ull * P, bb[0].bits, bb[1].bits};
  P_RC(or_combine_launch(parts, P, static_cast<uint32_t>(req_c), a.seeds, dev + 6ull * P, st));
  P_TRY(cudaMemcpyAsync(shares_out, dev + 6ull * P, 3ull * P, cudaMemcpyDeviceToHost, st));
  P_TRY(cudaStreamSynchronize(st));
  int rc = ctx_check_device_status(c);
  if (rc) return rc;
  req_ids[0] = rid[0];
  req_ids[1] = rid[1];
  req_ids[2] = req_b[0];
  req_ids[3] = req_b[1];
  req_ids[4] = req_c;
  return IPC_OK;
}
