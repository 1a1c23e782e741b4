// Context-level API: resident database chunks, per-party streams and request lifecycle.
//
// Pipeline of one request, per resident database chunk c (buffer set b = c % 2):
//   party streams 0..2 : wait(compare of the chunk that last used set b)
//                        A3 GEMM code, A3 GEMM mask  -> z[b][vec][party]   (party i's message to i+1)
//   compare stream     : wait(all three parties), A4-A8 per comparison + in-block OR -> roots
// then A8 (rest of the OR tree) and the copy of the three bit components to pinned host memory.
// Queries are prepared once per request on the party streams (A2).
#include "context.cuh"

using namespace ipc;

namespace {

int fail(ipc_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  set_error(msg);
  return code;
}

int cfail(ipc_ctx* c, cudaError_t e, const char* what) {
  return fail(c, IPC_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define CTX_TRY(ctx, expr)                               \
  do {                                                   \
    cudaError_t e__ = (expr);                            \
    if (e__ != cudaSuccess) return cfail(ctx, e__, #expr); \
  } while (0)

#define CTX_RC(ctx, expr)                          \
  do {                                             \
    int rc__ = (expr);                             \
    if (rc__ != IPC_OK) {                          \
      (ctx)->err = ipc::thread_last_error();       \
      return rc__;                                 \
    }                                              \
  } while (0)

uint8_t* plane(const ipc_ctx* c, const Chunk& ch, int comp, int vec, int limb) {
  return ch.planes + static_cast<size_t>((comp * 2 + vec) * c->nlimb + limb) * ch.cap * c->l * c->esz;
}

// The Z_2^32 ring GEMM on one CTA per tile: its CTA-pair form gives the same z in the same time.
constexpr bool kTc32Pair = false;

// Whether a vector (0 code, 1 mask) is shared over Z_2^32 (lifting variants) rather than Z_2^16.
bool wide(const ipc_ctx* c, int vec) {
  return vec == 1 ? c->cfg.lift != 0 : c->cfg.lift == IPC_LIFT_NONE;
}

uint32_t round_up(uint32_t x, uint32_t m) { return (x + m - 1) / m * m; }

// Frees a request's buffers on every early return of submit_queries, after the device has
// finished whatever was already enqueued on them; keep() hands them to the context instead.
class RequestGuard {
 public:
  RequestGuard(ipc_ctx* c, Request* r) : c_(c), r_(r) {}
  ~RequestGuard();
  void keep() { r_ = nullptr; }

 private:
  ipc_ctx* c_;
  Request* r_;
};

void free_request(ipc_ctx* c, Request& r);

RequestGuard::~RequestGuard() {
  if (!r_) return;
  cudaDeviceSynchronize();
  cudaGetLastError();
  free_request(c_, *r_);
}

void free_request(ipc_ctx* c, Request& r) {
  cudaFree(r.bq);
  cudaFree(r.qstage);
  cudaFree(r.tags);
  cudaFree(r.roots);
  cudaFree(r.shares_dev);
  cudaFree(r.zkeep);
  if (r.shares_host) cudaFreeHost(r.shares_host);
  if (r.done) cudaEventDestroy(r.done);
  (void)c;
}

int ensure_zbuf(ipc_ctx* c, uint32_t n_pad) {
  if (c->cfg.keep_distances) return IPC_OK;
  if (c->zbuf_cols >= n_pad) return IPC_OK;
  CTX_TRY(c, cudaDeviceSynchronize());
  cudaFree(c->zbuf);
  c->zbuf = nullptr;
  const size_t bytes = 2ull * 2 * 3 * n_pad * static_cast<size_t>(c->cfg.db_chunk_rows) * c->zsz;
  if (cudaMalloc(&c->zbuf, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->zbuf_cols = 0;
    return fail(c, IPC_ENOMEM, "cannot allocate the dot-product scratch for " + std::to_string(n_pad) + " columns");
  }
  c->zbuf_cols = n_pad;
  return IPC_OK;
}

uint8_t* zslot(ipc_ctx* c, int set, int vec, int party) {
  return c->zbuf + ((static_cast<size_t>(set) * 2 + vec) * 3 + party) * c->zbuf_cols * c->cfg.db_chunk_rows * c->zsz;
}

int wait_event(ipc_ctx* c, cudaEvent_t ev, int timeout_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return IPC_OK;
    if (e != cudaErrorNotReady) return cfail(c, e, "request completion");
    if (timeout_ms >= 0) {
      const auto ms =
          std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
      if (ms >= timeout_ms) return fail(c, IPC_ETIMEOUT, "request not finished within the timeout");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// Device inputs are produced by the caller's work on c->input_stream; the library's streams
// are non-blocking, so they must wait for that work explicitly before reading the inputs.
int order_after_input(ipc_ctx* c) {
  CTX_TRY(c, cudaEventRecord(c->ev_input, c->input_stream));
  CTX_TRY(c, cudaStreamWaitEvent(c->sc, c->ev_input, 0));
  return IPC_OK;
}

int check_device_status(ipc_ctx* c) {
  uint32_t* st = status_ptr();
  if (!st) return IPC_OK;
  uint32_t v = 0;
  CTX_TRY(c, cudaMemcpy(&v, st, sizeof v, cudaMemcpyDeviceToHost));
  if (v) {
    CTX_TRY(c, cudaMemset(st, 0, sizeof v));
    return fail(c, IPC_EDEVICE, "a kernel gave up a bounded wait (device status " + std::to_string(v) + ")");
  }
  return IPC_OK;
}

}  // namespace

namespace ipc {
int ctx_fail(ipc_ctx* c, int code, const std::string& msg) { return fail(c, code, msg); }
int ctx_cfail(ipc_ctx* c, cudaError_t e, const char* what) { return cfail(c, e, what); }
uint8_t* ctx_plane(const ipc_ctx* c, const Chunk& ch, int comp, int vec, int limb) {
  return plane(c, ch, comp, vec, limb);
}
int ctx_check_device_status(ipc_ctx* c) { return check_device_status(c); }
}  // namespace ipc

extern "C" int ipc_create(const ipc_config* cfg, ipc_ctx** out) {
  if (!cfg || !out) return fail(nullptr, IPC_EINVAL, "ipc_create: null argument");
  const ipc_geom& g = cfg->geom;
  const uint64_t l = static_cast<uint64_t>(g.rows) * g.cols * g.cell;
  if (l == 0 || l % 128 != 0 || l > 16384 || g.R == 0 || g.R > 31)
    return fail(nullptr, IPC_EINVAL, "ipc_create: l must be a multiple of 128 up to 16384 and 1 <= R <= 31");
  if (cfg->path != IPC_PATH_I8MMA && cfg->path != IPC_PATH_I32 && cfg->path != IPC_PATH_I8MIX &&
      cfg->path != IPC_PATH_TC && cfg->path != IPC_PATH_TCG)
    return fail(nullptr, IPC_EINVAL, "ipc_create: path");
  if (cfg->path == IPC_PATH_TCG && (l % 256 != 0 || g.cell % 2 != 0))
    return fail(nullptr, IPC_EINVAL, "ipc_create: Galois-ring shares need l % 256 == 0 and an even cell size");
  if (cfg->plain_mask && ((cfg->path != IPC_PATH_TC && cfg->path != IPC_PATH_TCG) || l % 256 != 0 || g.cell % 2 != 0))
    return fail(nullptr, IPC_EINVAL,
                "ipc_create: plain masks (protocol 1) need the tc or tcg path, l % 256 == 0 and an even cell size");
  if (cfg->lift > IPC_LIFT_NONE || (cfg->lift != 0 && (cfg->path != IPC_PATH_TC || cfg->plain_mask)))
    return fail(nullptr, IPC_EINVAL, "ipc_create: the lifting variants need the tc path and shared masks");
  if (cfg->thr_b > 65536 || (cfg->lift != IPC_LIFT_NONE && cfg->thr_b != 0 && cfg->thr_b != 65536))
    return fail(nullptr, IPC_EINVAL, "ipc_create: thr_b is 2^16 unless lift is IPC_LIFT_NONE (then 1..2^16)");
  if (cfg->db_chunk_rows % 1024 != 0) return fail(nullptr, IPC_EINVAL, "ipc_create: db_chunk_rows % 1024 != 0");
  ipc_ctx* c = new ipc_ctx();
  c->cfg = *cfg;
  if (c->cfg.db_chunk_rows == 0) c->cfg.db_chunk_rows = 65536;
  if (c->cfg.max_queries == 0) c->cfg.max_queries = 256;
  c->l = static_cast<uint32_t>(l);
  c->esz = (cfg->path == IPC_PATH_TC || cfg->path == IPC_PATH_TCG) ? 2 : 1;
  c->kq = cfg->path == IPC_PATH_TCG ? c->l : 2 * c->l;
  c->nlimb = cfg->lift ? 4 : 2;
  c->zsz = cfg->lift ? 4 : 2;
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    delete c;
    return cfail(nullptr, e, "cudaSetDevice");
  }
  for (int i = 0; i < 3; ++i) cudaStreamCreateWithFlags(&c->sp[i], cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&c->sc, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&c->ev_setup, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&c->ev_input, cudaEventDisableTiming);
  for (int s = 0; s < 2; ++s) {
    cudaEventCreateWithFlags(&c->ev_cmp[s], cudaEventDisableTiming);
    for (int i = 0; i < 3; ++i) cudaEventCreateWithFlags(&c->ev_gemm[i][s], cudaEventDisableTiming);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    ipc_destroy(c);
    return cfail(nullptr, e, "stream/event creation");
  }
  *out = c;
  return IPC_OK;
}

extern "C" void ipc_destroy(ipc_ctx* c) {
  if (!c) return;
  serve_shutdown(c);
  cudaSetDevice(c->cfg.device);
  cudaDeviceSynchronize();
  for (auto& kv : c->reqs) free_request(c, kv.second);
  for (auto& ch : c->chunks) cudaFree(ch.planes);
  cudaFree(c->zbuf);
  cudaFree(c->stage);
  for (int i = 0; i < 3; ++i)
    if (c->sp[i]) cudaStreamDestroy(c->sp[i]);
  if (c->sc) cudaStreamDestroy(c->sc);
  if (c->ev_setup) cudaEventDestroy(c->ev_setup);
  if (c->ev_input) cudaEventDestroy(c->ev_input);
  for (int s = 0; s < 2; ++s) {
    if (c->ev_cmp[s]) cudaEventDestroy(c->ev_cmp[s]);
    for (int i = 0; i < 3; ++i)
      if (c->ev_gemm[i][s]) cudaEventDestroy(c->ev_gemm[i][s]);
  }
  delete c;
}

extern "C" const char* ipc_last_error(const ipc_ctx* c) { return c ? c->err.c_str() : ipc::thread_last_error(); }

extern "C" size_t ipc_db_rows(const ipc_ctx* c) { return c ? c->rows : 0; }

extern "C" void* ipc_ctx_stream(const ipc_ctx* c) { return c ? static_cast<void*>(c->sc) : nullptr; }

extern "C" int ipc_set_input_stream(ipc_ctx* c, void* stream) {
  if (!c) return fail(c, IPC_EINVAL, "ipc_set_input_stream: null context");
  c->input_stream = static_cast<cudaStream_t>(stream);
  return IPC_OK;
}

extern "C" int load_db_shares(ipc_ctx* c, const uint16_t* const code[3], const uint16_t* const mask[3],
                              size_t n_rows, int src_is_device) {
  if (!c || !code || !mask) return fail(c, IPC_EINVAL, "load_db_shares: null argument");
  if (c->srv) return fail(c, IPC_EINVAL, "load_db_shares: the context is serving");
  const int mask_parts = c->cfg.plain_mask ? 1 : 3;
  for (int j = 0; j < 3; ++j)
    if (!code[j] || (j < mask_parts && !mask[j])) return fail(c, IPC_EINVAL, "load_db_shares: null component");
  if (n_rows == 0) return IPC_OK;
  CTX_TRY(c, cudaSetDevice(c->cfg.device));
  const size_t cap = c->cfg.db_chunk_rows, l = c->l;
  if (!c->stage) {
    if (cudaMalloc(&c->stage, cap * l * (c->cfg.lift ? 4 : 2)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, IPC_ENOMEM, "load_db_shares: staging buffer");
    }
  }
  // allocate every chunk needed first, so that a failure appends nothing
  const size_t free_in_last = c->chunks.empty() ? 0 : c->chunks.back().cap - c->chunks.back().rows;
  std::vector<Chunk> fresh;
  size_t need = n_rows > free_in_last ? n_rows - free_in_last : 0;
  uint64_t next_row0 = c->chunks.empty() ? 0 : c->chunks.back().row0 + c->chunks.back().cap;
  while (need > 0) {
    Chunk ch;
    ch.cap = cap;
    ch.row0 = next_row0;
    if (cudaMalloc(&ch.planes, 6 * c->nlimb * cap * l * c->esz) != cudaSuccess) {
      cudaGetLastError();
      for (auto& f : fresh) cudaFree(f.planes);
      return fail(c, IPC_ENOMEM, "load_db_shares: device memory exhausted");
    }
    fresh.push_back(ch);
    next_row0 += cap;
    need = need > cap ? need - cap : 0;
  }
  for (auto& f : fresh) c->chunks.push_back(f);
  if (src_is_device) {
    int rc = order_after_input(c);
    if (rc) return rc;
  }
  const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  size_t done = 0;
  while (done < n_rows) {
    Chunk* ch = nullptr;
    for (auto& x : c->chunks)
      if (x.rows < x.cap) {
        ch = &x;
        break;
      }
    const size_t take = std::min(n_rows - done, ch->cap - ch->rows);
    for (int vec = 0; vec < 2; ++vec)
      for (int j = 0; j < (vec == 0 ? 3 : mask_parts); ++j) {
        const size_t es = wide(c, vec) ? 4 : 2;  // bytes per input element
        const uint8_t* src = reinterpret_cast<const uint8_t*>(vec == 0 ? code[j] : mask[j]) + done * l * es;
        CTX_TRY(c, cudaMemcpyAsync(c->stage, src, take * l * es, kind, c->sc));
        uint8_t* lo = plane(c, *ch, j, vec, 0) + ch->rows * l * c->esz;
        uint8_t* hi = plane(c, *ch, j, vec, 1) + ch->rows * l * c->esz;
        if (es == 4) {
          uint16_t* out[4];
          for (int t = 0; t < 4; ++t)
            out[t] = reinterpret_cast<uint16_t*>(plane(c, *ch, j, vec, t) + ch->rows * l * c->esz);
          CTX_RC(c, ipc_split_limbs32_bf16(reinterpret_cast<const uint32_t*>(c->stage), take * l, out, c->sc));
        } else if (c->esz == 2)
          CTX_RC(c, ipc_split_limbs_bf16(reinterpret_cast<const uint16_t*>(c->stage), take * l, reinterpret_cast<uint16_t*>(lo),
                                         reinterpret_cast<uint16_t*>(hi), c->sc));
        else
          CTX_RC(c, ipc_split_limbs(reinterpret_cast<const uint16_t*>(c->stage), take * l, reinterpret_cast<int8_t*>(lo), reinterpret_cast<int8_t*>(hi),
                                    c->sc));
      }
    ch->rows += take;
    done += take;
  }
  c->rows += n_rows;
  CTX_TRY(c, cudaStreamSynchronize(c->sc));
  return IPC_OK;
}

extern "C" int submit_queries(ipc_ctx* c, const uint16_t* const code[3], const uint16_t* const mask[3],
                              size_t n_queries, int src_is_device, uint64_t* req_id) {
  if (!c || !code || !mask || !req_id) return fail(c, IPC_EINVAL, "submit_queries: null argument");
  if (n_queries == 0 || n_queries > c->cfg.max_queries)
    return fail(c, IPC_EINVAL, "submit_queries: n_queries must be in 1..max_queries");
  if (c->srv) return fail(c, IPC_EINVAL, "submit_queries: the context is serving; use ipc_serve_submit");
  if (c->rows == 0) return fail(c, IPC_EINVAL, "submit_queries: no database rows loaded");
  const bool plain = c->cfg.plain_mask != 0;
  const int mask_parts = plain ? 1 : 3;
  for (int j = 0; j < 3; ++j)
    if (!code[j] || (j < mask_parts && !mask[j])) return fail(c, IPC_EINVAL, "submit_queries: null component");
  CTX_TRY(c, cudaSetDevice(c->cfg.device));
  const ipc_geom& g = c->cfg.geom;
  const uint32_t l = c->l, Q = static_cast<uint32_t>(n_queries), R = g.R, N = Q * R;
  const uint32_t n_pad = round_up(N, 128);
  int rc = ensure_zbuf(c, n_pad);
  if (rc) return rc;

  // declared before the request guard, so that an early return synchronises before the host
  // source of the tag copy goes away
  std::vector<uint32_t> tags(2ull * N);
  Request r;
  {
    std::lock_guard<std::mutex> lock(c->id_mu);
    r.id = c->next_id++;
  }
  r.Q = Q;
  r.N = N;
  r.n_pad = n_pad;
  const size_t total_blocks = (c->chunks.size() * c->cfg.db_chunk_rows) >> (5 + kLog2BlockWords);
  r.ld_roots = total_blocks;
  const size_t qes = c->cfg.lift ? 4 : 2;  // bytes per staged query element
  bool ok = cudaMalloc(&r.bq, 6ull * c->nlimb * n_pad * c->kq * c->esz) == cudaSuccess &&
            cudaMalloc(&r.qstage, 2ull * 3 * Q * l * qes) == cudaSuccess &&
            cudaMalloc(&r.tags, 2ull * N * sizeof(uint32_t)) == cudaSuccess &&
            cudaMalloc(&r.roots, 3ull * N * r.ld_roots * sizeof(uint32_t)) == cudaSuccess &&
            cudaMalloc(&r.shares_dev, 3ull * Q) == cudaSuccess &&
            cudaMallocHost(&r.shares_host, 3ull * Q) == cudaSuccess &&
            cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) == cudaSuccess;
  if (ok && c->cfg.keep_distances) {
    r.zkeep_rows = round_up(static_cast<uint32_t>(c->chunks.size() * c->cfg.db_chunk_rows), 8);
    ok = cudaMalloc(&r.zkeep, 2ull * 3 * N * r.zkeep_rows * c->zsz) == cudaSuccess;
  }
  RequestGuard guard(c, &r);  // from here on every early return frees the request
  if (!ok) {
    cudaGetLastError();
    return fail(c, IPC_ENOMEM, "submit_queries: not enough device memory for the request");
  }
  // column tags: (request id, q << 5 | rho)
  for (uint32_t q = 0; q < Q; ++q)
    for (uint32_t rho = 0; rho < R; ++rho) {
      tags[2 * (q * R + rho)] = static_cast<uint32_t>(r.id);
      tags[2 * (q * R + rho) + 1] = (q << 5) | rho;
    }
  if (src_is_device) {
    rc = order_after_input(c);
    if (rc) return rc;
  }
  const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CTX_TRY(c, cudaMemcpyAsync(r.tags, tags.data(), tags.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, c->sc));
  auto qvec = [&](int vec) { return r.qstage + static_cast<size_t>(vec) * 3 * Q * l * qes; };
  for (int vec = 0; vec < 2; ++vec)
    for (int j = 0; j < (vec == 0 ? 3 : mask_parts); ++j) {
      const size_t es = wide(c, vec) ? 4 : 2;
      CTX_TRY(c, cudaMemcpyAsync(qvec(vec) + static_cast<size_t>(j) * Q * l * es, vec == 0 ? code[j] : mask[j],
                                 static_cast<size_t>(Q) * l * es, kind, c->sc));
    }
  CTX_TRY(c, cudaEventRecord(c->ev_setup, c->sc));
  // the host tags vector dies at return: make the copy complete before that
  const size_t qplane = static_cast<size_t>(n_pad) * c->kq * c->esz;
  auto bq = [&](int party, int vec, int limb) { return r.bq + ((party * 2 + vec) * c->nlimb + limb) * qplane; };
  for (int i = 0; i < 3; ++i) {
    CTX_TRY(c, cudaStreamWaitEvent(c->sp[i], c->ev_setup, 0));
    for (int vec = 0; vec < 2; ++vec) {
      const uint16_t* y = reinterpret_cast<const uint16_t*>(qvec(vec));
      if (wide(c, vec)) {
        uint16_t* b4[4];
        for (int t = 0; t < 4; ++t) b4[t] = reinterpret_cast<uint16_t*>(bq(i, vec, t));
        CTX_RC(c, prep_query32(reinterpret_cast<const uint32_t*>(qvec(vec)), static_cast<uint64_t>(Q) * l, Q, &g, i, 2,
                               b4, n_pad, c->sp[i]));
      } else if (plain && vec == 1) {
        // protocol 1: the rotated public query mask, prepared once (party 0's stream runs the ml GEMM)
        if (i == 0)
          CTX_RC(c, prep_query_rotate_plain(y, Q, &g, reinterpret_cast<uint16_t*>(bq(0, 1, 0)),
                                            reinterpret_cast<uint16_t*>(bq(0, 1, 1)), n_pad, c->sp[0]));
      } else if (c->cfg.path == IPC_PATH_TCG)
        CTX_RC(c, prep_query_galois_strided(y, static_cast<uint64_t>(Q) * l, Q, &g, i,
                                            reinterpret_cast<uint16_t*>(bq(i, vec, 0)),
                                            reinterpret_cast<uint16_t*>(bq(i, vec, 1)), n_pad, c->sp[i]));
      else if (c->esz == 2)
        CTX_RC(c, ipc_prep_query_bf16(y, Q, &g, i, reinterpret_cast<uint16_t*>(bq(i, vec, 0)),
                                      reinterpret_cast<uint16_t*>(bq(i, vec, 1)), n_pad, c->sp[i]));
      else
        CTX_RC(c, ipc_prep_query(y, Q, &g, i, reinterpret_cast<int8_t*>(bq(i, vec, 0)),
                                 reinterpret_cast<int8_t*>(bq(i, vec, 1)), n_pad, c->sp[i]));
    }
  }
  for (size_t ci = 0; ci < c->chunks.size(); ++ci) {
    const Chunk& ch = c->chunks[ci];
    if (ch.rows == 0) continue;
    const int set = static_cast<int>(ci & 1);
    uint8_t* zc[3];  // 2-byte (Z_2^16) or 4-byte (Z_2^32) elements, ldz per column
    uint8_t* zm[3];
    size_t ldz;
    for (int i = 0; i < 3; ++i) {
      if (c->cfg.keep_distances) {
        // slot (vec, party) holds N columns of zkeep_rows elements; this chunk starts at row0
        const size_t slot = static_cast<size_t>(N) * r.zkeep_rows * c->zsz;
        zc[i] = r.zkeep + (0 * 3 + i) * slot + ch.row0 * (wide(c, 0) ? 4 : 2);
        zm[i] = r.zkeep + (1 * 3 + i) * slot + ch.row0 * (wide(c, 1) ? 4 : 2);
        ldz = r.zkeep_rows;
      } else {
        zc[i] = zslot(c, set, 0, i);
        zm[i] = zslot(c, set, 1, i);
        ldz = c->cfg.db_chunk_rows;
      }
    }
    for (int i = 0; i < 3; ++i) {
      const int prev = (i + 2) % 3;
      CTX_TRY(c, cudaStreamWaitEvent(c->sp[i], c->ev_cmp[set], 0));
      for (int vec = 0; vec < 2; ++vec) {
        uint16_t* zo = reinterpret_cast<uint16_t*>(vec == 0 ? zc[i] : zm[i]);
        if (wide(c, vec)) {
          // lifting variants: the ring product over Z_2^32, four limbs, K = 2l
          const uint16_t* x8[8];
          const uint16_t* b4[4];
          for (int t = 0; t < 4; ++t) {
            x8[t] = reinterpret_cast<const uint16_t*>(plane(c, ch, i, vec, t));
            x8[4 + t] = reinterpret_cast<const uint16_t*>(plane(c, ch, prev, vec, t));
            b4[t] = reinterpret_cast<const uint16_t*>(bq(i, vec, t));
          }
          CTX_RC(c, ring_gemm_tc32(2, x8, ch.rows, b4, N, n_pad, l, r.tags, c->cfg.seeds[i], c->cfg.seeds[prev],
                                   static_cast<uint32_t>(vec), reinterpret_cast<uint32_t*>(zo), ldz, ch.row0,
                                   c->sp[i], kTc32Pair));
        } else if (plain && vec == 1) {
          // protocol 1: ml = <rotated query mask, database mask> in the clear, K = l; equal seeds
          // make the zero share vanish
          if (i != 0) continue;
          auto p16 = [](const uint8_t* p) { return reinterpret_cast<const uint16_t*>(p); };
          const uint16_t* xl[2] = {p16(plane(c, ch, 0, 1, 0)), p16(plane(c, ch, 0, 1, 0))};
          const uint16_t* xh[2] = {p16(plane(c, ch, 0, 1, 1)), p16(plane(c, ch, 0, 1, 1))};
          CTX_RC(c, ring_gemm_tc_variant(256, 1, xl, xh, ch.rows, p16(bq(0, 1, 0)), p16(bq(0, 1, 1)), N, n_pad, l,
                                         r.tags, c->cfg.seeds[0], c->cfg.seeds[0], 1u, zo, ldz, ch.row0, nullptr,
                                         nullptr, c->sp[0]));
        } else if (c->cfg.path == IPC_PATH_TCG) {
          // Galois-ring Shamir: party i's own share only, K = l
          auto p16 = [](const uint8_t* p) { return reinterpret_cast<const uint16_t*>(p); };
          const uint16_t* xl[2] = {p16(plane(c, ch, i, vec, 0)), p16(plane(c, ch, i, vec, 0))};
          const uint16_t* xh[2] = {p16(plane(c, ch, i, vec, 1)), p16(plane(c, ch, i, vec, 1))};
          CTX_RC(c, ring_gemm_tc_variant(256, 1, xl, xh, ch.rows, p16(bq(i, vec, 0)), p16(bq(i, vec, 1)), N, n_pad, l,
                                         r.tags, c->cfg.seeds[i], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo,
                                         ldz, ch.row0, nullptr, nullptr, c->sp[i]));
        } else if (c->cfg.path == IPC_PATH_TC) {
          auto p16 = [](const uint8_t* p) { return reinterpret_cast<const uint16_t*>(p); };
          const uint16_t* xl[2] = {p16(plane(c, ch, i, vec, 0)), p16(plane(c, ch, prev, vec, 0))};
          const uint16_t* xh[2] = {p16(plane(c, ch, i, vec, 1)), p16(plane(c, ch, prev, vec, 1))};
          CTX_RC(c, ipc_ring_gemm_tc(xl, xh, ch.rows, p16(bq(i, vec, 0)), p16(bq(i, vec, 1)), N, n_pad, l, r.tags,
                                     c->cfg.seeds[i], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo, ldz,
                                     ch.row0, c->sp[i]));
        } else {
          auto p8 = [](const uint8_t* p) { return reinterpret_cast<const int8_t*>(p); };
          const int8_t* xl[2] = {p8(plane(c, ch, i, vec, 0)), p8(plane(c, ch, prev, vec, 0))};
          const int8_t* xh[2] = {p8(plane(c, ch, i, vec, 1)), p8(plane(c, ch, prev, vec, 1))};
          CTX_RC(c, ipc_ring_gemm(c->cfg.path, xl, xh, ch.rows, p8(bq(i, vec, 0)), p8(bq(i, vec, 1)), N, n_pad, l,
                                  r.tags, c->cfg.seeds[i], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo, ldz,
                                  ch.row0, c->sp[i]));
        }
      }
      CTX_TRY(c, cudaEventRecord(c->ev_gemm[i][set], c->sp[i]));
      CTX_TRY(c, cudaStreamWaitEvent(c->sc, c->ev_gemm[i][set], 0));
    }
    auto u16p = [](const uint8_t* p) { return reinterpret_cast<const uint16_t*>(p); };
    auto u32p = [](const uint8_t* p) { return reinterpret_cast<const uint32_t*>(p); };
    if (c->cfg.lift) {
      const uint32_t* ml32[3] = {u32p(zm[0]), u32p(zm[1]), u32p(zm[2])};
      const uint32_t* zc32[3] = {u32p(zc[0]), u32p(zc[1]), u32p(zc[2])};
      const uint16_t* zc16[3] = {u16p(zc[0]), u16p(zc[1]), u16p(zc[2])};
      const bool nolift = c->cfg.lift == IPC_LIFT_NONE;
      CTX_RC(c, compare_launch_liftfree(nolift ? nullptr : zc16, nolift ? zc32 : nullptr, ml32, ldz, N, ch.rows,
                                        ch.row0, r.tags, c->cfg.seeds, c->cfg.thr_a, c->cfg.thr_b, kLog2BlockWords,
                                        r.roots, r.ld_roots, nullptr, 0, c->sc));
    } else {
      const uint16_t* zcc[3] = {u16p(zc[0]), u16p(zc[1]), u16p(zc[2])};
      const uint16_t* zmc[3] = {u16p(zm[0]), u16p(plain ? zm[0] : zm[1]), u16p(plain ? zm[0] : zm[2])};
      CTX_RC(c, compare_launch_tiles(zcc, zmc, ldz, N, ch.rows, ch.row0, r.tags, c->cfg.seeds, c->cfg.thr_a,
                                     kLog2BlockWords, r.roots, r.ld_roots, nullptr, 0, nullptr, nullptr, 0, c->sc,
                                     nullptr, plain));
    }
    CTX_TRY(c, cudaEventRecord(c->ev_cmp[set], c->sc));
  }
  const uint32_t n_blocks =
      static_cast<uint32_t>((c->rows + (32ull << kLog2BlockWords) - 1) >> (5 + kLog2BlockWords));
  CTX_RC(c, ipc_or_finalize(r.roots, r.ld_roots, n_blocks, kLog2BlockWords, Q, R, r.tags, c->cfg.seeds, r.shares_dev,
                            c->sc));
  CTX_TRY(c, cudaMemcpyAsync(r.shares_host, r.shares_dev, 3ull * Q, cudaMemcpyDeviceToHost, c->sc));
  CTX_TRY(c, cudaEventRecord(r.done, c->sc));
  CTX_TRY(c, cudaEventSynchronize(c->ev_setup));  // the tag vector above is a host temporary
  guard.keep();
  c->reqs[r.id] = r;
  *req_id = r.id;
  return IPC_OK;
}

extern "C" int fetch_bit_shares(ipc_ctx* c, uint64_t req_id, uint8_t* shares_out, size_t n_queries, int timeout_ms) {
  if (!c || !shares_out) return fail(c, IPC_EINVAL, "fetch_bit_shares: null argument");
  auto it = c->reqs.find(req_id);
  if (it == c->reqs.end()) {
    const int rc = serve_fetch_shares(c, req_id, shares_out, n_queries, timeout_ms);
    return rc == IPC_ENOTFOUND ? fail(c, IPC_ENOTFOUND, "unknown request id") : rc;
  }
  Request& r = it->second;
  if (n_queries != r.Q) return fail(c, IPC_EINVAL, "n_queries does not match the request");
  int rc = wait_event(c, r.done, timeout_ms);
  if (rc) return rc;
  rc = check_device_status(c);
  if (rc) return rc;
  std::memcpy(shares_out, r.shares_host, 3ull * r.Q);
  return IPC_OK;
}

extern "C" int fetch_match_bits(ipc_ctx* c, uint64_t req_id, uint8_t* bits_out, size_t n_queries, int timeout_ms) {
  if (!c || !bits_out) return fail(c, IPC_EINVAL, "fetch_match_bits: null argument");
  std::vector<uint8_t> sh(3 * n_queries);
  int rc = fetch_bit_shares(c, req_id, sh.data(), n_queries, timeout_ms);
  if (rc) return rc;
  // Open the bit at the output node: XOR of the three boolean components.
  for (size_t q = 0; q < n_queries; ++q) bits_out[q] = (sh[q] ^ sh[n_queries + q] ^ sh[2 * n_queries + q]) & 1u;
  return ipc_release(c, req_id);
}

extern "C" int fetch_distances(ipc_ctx* c, uint64_t req_id, uint32_t q, uint32_t rho, size_t row_begin,
                               size_t row_end, int16_t* dot, uint16_t* ml) {
  if (!c || !dot || !ml) return fail(c, IPC_EINVAL, "fetch_distances: null argument");
  auto it = c->reqs.find(req_id);
  if (it == c->reqs.end()) return fail(c, IPC_ENOTFOUND, "unknown request id");
  Request& r = it->second;
  if (!r.zkeep) return fail(c, IPC_ENOSYS, "fetch_distances needs keep_distances");
  if (q >= r.Q || rho >= c->cfg.geom.R || row_begin > row_end || row_end > c->rows)
    return fail(c, IPC_EINVAL, "fetch_distances: range");
  int rc = wait_event(c, r.done, -1);
  if (rc) return rc;
  const size_t n = static_cast<size_t>(q) * c->cfg.geom.R + rho, cnt = row_end - row_begin;
  std::vector<uint8_t> tmp(cnt * 4);
  std::vector<uint32_t> acc[2] = {std::vector<uint32_t>(cnt, 0), std::vector<uint32_t>(cnt, 0)};
  const bool plain = c->cfg.plain_mask != 0;
  const size_t slot = static_cast<size_t>(r.N) * r.zkeep_rows * c->zsz;
  for (int vec = 0; vec < 2; ++vec) {
    const size_t es = wide(c, vec) ? 4 : 2;
    for (int i = 0; i < (plain && vec == 1 ? 1 : 3); ++i) {  // protocol 1 keeps ml itself in component 0
      const uint8_t* src = r.zkeep + (static_cast<size_t>(vec) * 3 + i) * slot + (n * r.zkeep_rows + row_begin) * es;
      CTX_TRY(c, cudaMemcpy(tmp.data(), src, cnt * es, cudaMemcpyDeviceToHost));
      // the components sum to the value mod 2^16 or mod 2^32; its low 16 bits are returned
      for (size_t k = 0; k < cnt; ++k) {
        uint32_t v = 0;
        if (es == 4) {
          std::memcpy(&v, tmp.data() + 4 * k, 4);
        } else {
          uint16_t h;
          std::memcpy(&h, tmp.data() + 2 * k, 2);
          v = h;
        }
        acc[vec][k] += v;
      }
    }
  }
  for (size_t k = 0; k < cnt; ++k) {
    dot[k] = static_cast<int16_t>(static_cast<uint16_t>(acc[0][k] & 0xFFFFu));
    ml[k] = static_cast<uint16_t>(acc[1][k] & 0xFFFFu);
  }
  return IPC_OK;
}

namespace {

// The SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t msg_hash(uint64_t kind, uint64_t party, uint64_t col, uint64_t row,
                                                      uint64_t v) {
  return mix64(mix64((kind << 60) | (party << 58) | (col << 32) | row) + v);
}

// XOR of msg_hash over one (kind, party) plane of kept dot products [n_cols][ld] (es-byte
// elements, rows < n_rows), reduced per warp and folded into *out.
__global__ void transcript_kernel(const uint8_t* __restrict__ z, uint32_t es, uint64_t ld, uint32_t n_cols,
                                  uint64_t n_rows, uint32_t kind, uint32_t party, unsigned long long* out) {
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  uint64_t h = 0;
  if (tid < static_cast<uint64_t>(n_cols) * n_rows) {
    const uint64_t n = tid / n_rows, i = tid % n_rows;
    const uint64_t at = n * ld + i;
    const uint64_t v = es == 4 ? reinterpret_cast<const uint32_t*>(z)[at] : reinterpret_cast<const uint16_t*>(z)[at];
    h = msg_hash(kind, party, n, i, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xFFFFFFFFu, h, o);
  if ((threadIdx.x & 31) == 0 && h) atomicXor(out, static_cast<unsigned long long>(h));
}

}  // namespace

extern "C" int fetch_transcript_hash(ipc_ctx* c, uint64_t req_id, uint64_t* hash_out, int timeout_ms) {
  if (!c || !hash_out) return fail(c, IPC_EINVAL, "fetch_transcript_hash: null argument");
  auto it = c->reqs.find(req_id);
  if (it == c->reqs.end()) return fail(c, IPC_ENOTFOUND, "unknown request id");
  Request& r = it->second;
  if (!r.zkeep) return fail(c, IPC_ENOSYS, "fetch_transcript_hash needs keep_distances");
  int rc = wait_event(c, r.done, timeout_ms);
  if (rc) return rc;
  rc = check_device_status(c);
  if (rc) return rc;
  CTX_TRY(c, cudaSetDevice(c->cfg.device));
  unsigned long long* acc = nullptr;
  CTX_TRY(c, cudaMalloc(&acc, sizeof *acc));
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof *acc, c->sc);
  const size_t slot = static_cast<size_t>(r.N) * r.zkeep_rows * c->zsz;
  const uint32_t bs = 256;
  const uint64_t total = static_cast<uint64_t>(r.N) * c->rows;
  for (int vec = 0; vec < 2 && e == cudaSuccess; ++vec) {
    if (vec == 1 && c->cfg.plain_mask) break;  // protocol 1: ml is public, not a message
    for (int p = 0; p < 3 && e == cudaSuccess; ++p) {
      transcript_kernel<<<static_cast<unsigned>((total + bs - 1) / bs), bs, 0, c->sc>>>(
          r.zkeep + (static_cast<size_t>(vec) * 3 + p) * slot, wide(c, vec) ? 4u : 2u, r.zkeep_rows, r.N, c->rows,
          static_cast<uint32_t>(vec), static_cast<uint32_t>(p), acc);
      e = cudaGetLastError();
    }
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, acc, sizeof h, cudaMemcpyDeviceToHost, c->sc);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->sc);
  cudaFree(acc);
  if (e != cudaSuccess) return cfail(c, e, "fetch_transcript_hash");
  for (uint32_t p = 0; p < 3; ++p)
    for (uint32_t q = 0; q < r.Q; ++q) h ^= msg_hash(2, p, q, 0, r.shares_host[static_cast<size_t>(p) * r.Q + q]);
  *hash_out = h;
  return IPC_OK;
}

extern "C" int ipc_release(ipc_ctx* c, uint64_t req_id) {
  if (!c) return fail(c, IPC_EINVAL, "ipc_release: null context");
  auto it = c->reqs.find(req_id);
  if (it == c->reqs.end()) {
    const int rc = serve_release(c, req_id);
    return rc == IPC_ENOTFOUND ? fail(c, IPC_ENOTFOUND, "unknown request id") : rc;
  }
  cudaEventSynchronize(it->second.done);
  free_request(c, it->second);
  c->reqs.erase(it);
  return IPC_OK;
}
