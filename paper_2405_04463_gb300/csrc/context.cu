// Context-level API: resident database chunks, per-party streams and request lifecycle.
//
// Pipeline of one request, per resident database chunk c (buffer set b = c % 2):
//   party streams 0..2 : wait(compare of the chunk that last used set b)
//                        A3 GEMM code, A3 GEMM mask  -> z[b][vec][party]   (party i's message to i+1)
//   compare stream     : wait(all three parties), A4-A8 per comparison + in-block OR -> roots
// then A8 (rest of the OR tree) and the copy of the three bit components to pinned host memory.
// Queries are prepared once per request on the party streams (A2).
//
// Memory: the database chunks are allocated by load_db_shares; every per-request buffer lives in
// one of max_requests request slots, allocated for max_queries queries by the first
// submit_queries, so that submitting, fetching and releasing allocate and free nothing (only a
// database grown since a slot was last used makes that slot's OR-tree roots grow once, and
// keep_distances requests allocate their kept messages, a test aid).
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
  return ch.planes + static_cast<size_t>((comp * 2 + vec) * c->nlimb + limb) * ch.cap * c->l;
}

// Whether a vector (0 code, 1 mask) is shared over Z_2^32 (lifting variants) rather than Z_2^16.
bool wide(const ipc_ctx* c, int vec) {
  return vec == 1 ? c->cfg.lift != 0 : c->cfg.lift == IPC_LIFT_NONE;
}

uint32_t round_up(uint32_t x, uint32_t m) { return (x + m - 1) / m * m; }

size_t total_blocks(const ipc_ctx* c) {
  return (c->chunks.size() * c->cfg.db_chunk_rows) >> (5 + kLog2BlockWords);
}

void free_slot(Slot& s) {
  cudaFree(s.bq);
  cudaFree(s.qstage);
  cudaFree(s.tags);
  cudaFree(s.roots);
  cudaFree(s.shares_dev);
  if (s.tags_host) cudaFreeHost(s.tags_host);
  if (s.shares_host) cudaFreeHost(s.shares_host);
  if (s.done) cudaEventDestroy(s.done);
  s = Slot();
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

// The fused step's part roots of one chunk: 3 components x n_pad columns x chunk_rows / 128 parts.
int ensure_parts(ipc_ctx* c, uint32_t n_pad) {
  if (!c->cfg.fused || c->parts_cols >= n_pad) return IPC_OK;
  const size_t bytes = 3ull * n_pad * (c->cfg.db_chunk_rows / 128) * sizeof(uint32_t);
  if (cudaMalloc(&c->parts, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, IPC_ENOMEM, "cannot allocate the fused step's part roots for " + std::to_string(n_pad) + " columns");
  }
  c->parts_cols = n_pad;
  return IPC_OK;
}

// Creates the request slots and the dot-product scratch for max_queries queries (once).
int ensure_slots(ipc_ctx* c) {
  if (!c->slots.empty()) return IPC_OK;
  const uint32_t Qm = c->cfg.max_queries, n_pad = round_up(Qm * c->cfg.geom.R, 128);
  int rc = ensure_zbuf(c, n_pad);
  if (rc) return rc;
  rc = ensure_parts(c, n_pad);
  if (rc) return rc;
  const size_t qes = c->cfg.lift ? 4 : 2;  // bytes per staged query element
  std::vector<Slot> slots(c->cfg.max_requests);
  bool ok = true;
  for (auto& s : slots) {
    ok = ok && cudaMalloc(&s.bq, 6ull * c->nlimb * n_pad * c->kq * c->qsz) == cudaSuccess &&
         cudaMalloc(&s.qstage, 2ull * 3 * Qm * c->l * qes) == cudaSuccess &&
         cudaMalloc(&s.tags, 2ull * n_pad * sizeof(uint32_t)) == cudaSuccess &&
         cudaMallocHost(&s.tags_host, 2ull * n_pad * sizeof(uint32_t)) == cudaSuccess &&
         cudaMalloc(&s.shares_dev, 3ull * Qm) == cudaSuccess && cudaMallocHost(&s.shares_host, 3ull * Qm) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    for (auto& s : slots) free_slot(s);
    return fail(c, IPC_ENOMEM, "cannot allocate " + std::to_string(c->cfg.max_requests) + " request slots for " +
                                   std::to_string(Qm) + " queries each");
  }
  c->slots = std::move(slots);
  c->n_pad_max = n_pad;
  return IPC_OK;
}

// Frees a request's own buffers (kept messages) and returns its slot; its device work is done.
void release_request(ipc_ctx* c, Request& r) {
  cudaFree(r.zkeep);
  r.zkeep = nullptr;
  if (r.slot >= 0) c->slots[r.slot].busy = false;
  r.slot = -1;
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
  if (cfg->max_requests > 64) return fail(nullptr, IPC_EINVAL, "ipc_create: max_requests is at most 64");
  if (cfg->fused && ((cfg->path != IPC_PATH_TC && cfg->path != IPC_PATH_TCG) || cfg->plain_mask || cfg->lift))
    return fail(nullptr, IPC_EINVAL, "ipc_create: the fused step needs the tc or tcg path with shared masks and MPCLift");
  ipc_ctx* c = new ipc_ctx();
  c->cfg = *cfg;
  if (c->cfg.db_chunk_rows == 0) c->cfg.db_chunk_rows = 65536;
  if (c->cfg.max_queries == 0) c->cfg.max_queries = 256;
  if (c->cfg.max_requests == 0) c->cfg.max_requests = 4;
  c->l = static_cast<uint32_t>(l);
  c->qsz = (cfg->path == IPC_PATH_TC || cfg->path == IPC_PATH_TCG) ? 2 : 1;
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
  for (auto& kv : c->reqs) release_request(c, kv.second);
  for (auto& s : c->slots) free_slot(s);
  for (auto& ch : c->chunks) cudaFree(ch.planes);
  cudaFree(c->zbuf);
  cudaFree(c->parts);
  cudaFree(c->stage);
  cudaFree(c->stall_flag);
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
    if (cudaMalloc(&ch.planes, 6 * c->nlimb * cap * l) != cudaSuccess) {
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
        if (es == 4) {
          int8_t* out[4];
          for (int t = 0; t < 4; ++t) out[t] = reinterpret_cast<int8_t*>(plane(c, *ch, j, vec, t) + ch->rows * l);
          CTX_RC(c, ipc_split_limbs32(reinterpret_cast<const uint32_t*>(c->stage), take * l, out, c->sc));
        } else {
          CTX_RC(c, ipc_split_limbs(reinterpret_cast<const uint16_t*>(c->stage), take * l,
                                    reinterpret_cast<int8_t*>(plane(c, *ch, j, vec, 0) + ch->rows * l),
                                    reinterpret_cast<int8_t*>(plane(c, *ch, j, vec, 1) + ch->rows * l), c->sc));
        }
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
  int rc = ensure_slots(c);
  if (rc) return rc;
  int si = -1;
  for (size_t k = 0; k < c->slots.size(); ++k)
    if (!c->slots[k].busy) {
      si = static_cast<int>(k);
      break;
    }
  if (si < 0)
    return fail(c, IPC_EAGAIN, "submit_queries: all " + std::to_string(c->slots.size()) +
                                   " request slots are in use; fetch or release a request first");
  Slot& sl = c->slots[si];
  const ipc_geom& g = c->cfg.geom;
  const uint32_t l = c->l, Q = static_cast<uint32_t>(n_queries), R = g.R, N = Q * R;
  const uint32_t n_pad = round_up(N, 128);
  // the OR-tree roots cover every resident block; they grow only after the database has grown
  const size_t ld_roots = total_blocks(c), roots_words = 3ull * N * ld_roots;
  const size_t roots_cap = 3ull * c->n_pad_max * ld_roots;
  if (sl.roots_words < roots_words) {
    CTX_TRY(c, cudaEventSynchronize(sl.done));
    cudaFree(sl.roots);
    sl.roots = nullptr;
    sl.roots_words = 0;
    if (cudaMalloc(&sl.roots, roots_cap * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, IPC_ENOMEM, "submit_queries: not enough device memory for the OR-tree roots");
    }
    sl.roots_words = roots_cap;
  }
  Request r;
  r.Q = Q;
  r.N = N;
  r.n_pad = n_pad;
  r.ld_roots = ld_roots;
  if (c->cfg.keep_distances) {
    r.zkeep_rows = round_up(static_cast<uint32_t>(c->chunks.size() * c->cfg.db_chunk_rows), 8);
    if (cudaMalloc(&r.zkeep, 2ull * 3 * N * r.zkeep_rows * c->zsz) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, IPC_ENOMEM, "submit_queries: not enough device memory to keep the messages");
    }
  }
  {
    std::lock_guard<std::mutex> lock(c->id_mu);
    r.id = c->next_id++;
  }
  // From here on the request owns the slot; an error releases it after the device has finished
  // whatever was enqueued on its buffers.
  r.slot = si;
  sl.busy = true;
  auto abandon = [&](int code) {
    cudaDeviceSynchronize();
    cudaGetLastError();
    release_request(c, r);
    return code;
  };
#define SUB_TRY(expr)                                     \
  do {                                                    \
    cudaError_t e__ = (expr);                             \
    if (e__ != cudaSuccess) return abandon(cfail(c, e__, #expr)); \
  } while (0)
#define SUB_RC(expr)                           \
  do {                                         \
    int rc__ = (expr);                         \
    if (rc__ != IPC_OK) {                      \
      c->err = ipc::thread_last_error();       \
      return abandon(rc__);                    \
    }                                          \
  } while (0)
  // The slot's pinned tag buffer may still feed the copy of the request that used it last:
  // that request's completion event covers the copy.
  SUB_TRY(cudaEventSynchronize(sl.done));
  // column tags: (request id, q << 5 | rho)
  for (uint32_t q = 0; q < Q; ++q)
    for (uint32_t rho = 0; rho < R; ++rho) {
      sl.tags_host[2 * (q * R + rho)] = static_cast<uint32_t>(r.id);
      sl.tags_host[2 * (q * R + rho) + 1] = (q << 5) | rho;
    }
  if (src_is_device) {
    rc = order_after_input(c);
    if (rc) return abandon(rc);
  }
  const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  SUB_TRY(cudaMemcpyAsync(sl.tags, sl.tags_host, 2ull * N * sizeof(uint32_t), cudaMemcpyHostToDevice, c->sc));
  const size_t qes = c->cfg.lift ? 4 : 2;  // bytes per staged query element
  auto qvec = [&](int vec) { return sl.qstage + static_cast<size_t>(vec) * 3 * Q * l * qes; };
  for (int vec = 0; vec < 2; ++vec)
    for (int j = 0; j < (vec == 0 ? 3 : mask_parts); ++j) {
      const size_t es = wide(c, vec) ? 4 : 2;
      SUB_TRY(cudaMemcpyAsync(qvec(vec) + static_cast<size_t>(j) * Q * l * es, vec == 0 ? code[j] : mask[j],
                              static_cast<size_t>(Q) * l * es, kind, c->sc));
    }
  SUB_TRY(cudaEventRecord(c->ev_setup, c->sc));
  const size_t qplane = static_cast<size_t>(n_pad) * c->kq * c->qsz;
  auto bq = [&](int party, int vec, int limb) { return sl.bq + ((party * 2 + vec) * c->nlimb + limb) * qplane; };
  auto f16p = [](uint8_t* p) { return reinterpret_cast<uint16_t*>(p); };
  for (int i = 0; i < 3; ++i) {
    SUB_TRY(cudaStreamWaitEvent(c->sp[i], c->ev_setup, 0));
    if (c->stall_party == i) {
      // injected failure: this party's work waits for a message that never comes (bounded)
      SUB_RC(stall_launch(c->stall_flag, c->stall_us, c->sp[i]));
      c->stall_party = -1;
    }
    for (int vec = 0; vec < 2; ++vec) {
      const uint16_t* y = reinterpret_cast<const uint16_t*>(qvec(vec));
      if (wide(c, vec)) {
        uint16_t* b4[4];
        for (int t = 0; t < 4; ++t) b4[t] = f16p(bq(i, vec, t));
        SUB_RC(prep_query32(reinterpret_cast<const uint32_t*>(qvec(vec)), static_cast<uint64_t>(Q) * l, Q, &g, i, 2,
                            b4, n_pad, c->sp[i]));
      } else if (plain && vec == 1) {
        // protocol 1: the rotated public query mask, prepared once (party 0's stream runs the ml GEMM)
        if (i == 0) SUB_RC(prep_query_rotate_plain(y, Q, &g, f16p(bq(0, 1, 0)), f16p(bq(0, 1, 1)), n_pad, c->sp[0]));
      } else if (c->cfg.path == IPC_PATH_TCG)
        SUB_RC(prep_query_galois_strided(y, static_cast<uint64_t>(Q) * l, Q, &g, i, f16p(bq(i, vec, 0)),
                                         f16p(bq(i, vec, 1)), n_pad, c->sp[i]));
      else if (c->cfg.path == IPC_PATH_TC)
        SUB_RC(ipc_prep_query_f16(y, Q, &g, i, f16p(bq(i, vec, 0)), f16p(bq(i, vec, 1)), n_pad, c->sp[i]));
      else
        SUB_RC(ipc_prep_query(y, Q, &g, i, reinterpret_cast<int8_t*>(bq(i, vec, 0)),
                              reinterpret_cast<int8_t*>(bq(i, vec, 1)), n_pad, c->sp[i]));
    }
  }
  auto i8p = [](const uint8_t* p) { return reinterpret_cast<const int8_t*>(p); };
  auto cf16 = [](const uint8_t* p) { return reinterpret_cast<const uint16_t*>(p); };
  const bool fused = c->cfg.fused != 0;
  if (fused) {
    // one kernel per chunk on the control stream runs every party's GEMMs and the comparison phase
    for (int i = 0; i < 3; ++i) {
      SUB_TRY(cudaEventRecord(c->ev_gemm[i][0], c->sp[i]));
      SUB_TRY(cudaStreamWaitEvent(c->sc, c->ev_gemm[i][0], 0));
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
    if (fused) {
      // Sec. 6.4's two phases of a chunk in one launch: the six ring GEMMs tile by tile, each
      // tile's comparison after its sixth pass; then the block roots from the part roots
      const int8_t* xl[6];
      const int8_t* xh[6];
      const uint16_t* bl[6];
      const uint16_t* bh[6];
      uint16_t* zo[6];
      for (int j = 0; j < 3; ++j)
        for (int vec = 0; vec < 2; ++vec) {
          xl[2 * j + vec] = i8p(plane(c, ch, j, vec, 0));
          xh[2 * j + vec] = i8p(plane(c, ch, j, vec, 1));
          bl[2 * j + vec] = cf16(bq(j, vec, 0));
          bh[2 * j + vec] = cf16(bq(j, vec, 1));
          zo[2 * j + vec] = reinterpret_cast<uint16_t*>(vec == 0 ? zc[j] : zm[j]);
        }
      const size_t ld_parts = c->cfg.db_chunk_rows / 128;
      SUB_RC(ring_gemm_compare_tc(c->cfg.path == IPC_PATH_TCG ? 1u : 2u, xl, xh, ch.rows, bl, bh, N, n_pad, l, sl.tags,
                                  c->cfg.seeds, c->cfg.thr_a, zo, ldz, ch.row0, c->parts, ld_parts, c->sc));
      SUB_RC(or_join_parts_launch(c->parts, ld_parts, N, ch.rows, ch.row0, sl.tags, c->cfg.seeds, sl.roots,
                                  r.ld_roots, c->sc));
      continue;
    }
    for (int i = 0; i < 3; ++i) {
      const int prev = (i + 2) % 3;
      SUB_TRY(cudaStreamWaitEvent(c->sp[i], c->ev_cmp[set], 0));
      for (int vec = 0; vec < 2; ++vec) {
        uint16_t* zo = reinterpret_cast<uint16_t*>(vec == 0 ? zc[i] : zm[i]);
        if (wide(c, vec)) {
          // lifting variants: the ring product over Z_2^32, four limbs, K = 2l
          const int8_t* x8[8];
          const uint16_t* b4[4];
          for (int t = 0; t < 4; ++t) {
            x8[t] = i8p(plane(c, ch, i, vec, t));
            x8[4 + t] = i8p(plane(c, ch, prev, vec, t));
            b4[t] = cf16(bq(i, vec, t));
          }
          SUB_RC(ring_gemm_tc32(2, x8, ch.rows, b4, N, n_pad, l, sl.tags, c->cfg.seeds[i], c->cfg.seeds[prev],
                                static_cast<uint32_t>(vec), reinterpret_cast<uint32_t*>(zo), ldz, ch.row0, c->sp[i]));
        } else if (plain && vec == 1) {
          // protocol 1: ml = <rotated query mask, database mask> in the clear, K = l; equal seeds
          // make the zero share vanish
          if (i != 0) continue;
          const int8_t* xl[2] = {i8p(plane(c, ch, 0, 1, 0)), i8p(plane(c, ch, 0, 1, 0))};
          const int8_t* xh[2] = {i8p(plane(c, ch, 0, 1, 1)), i8p(plane(c, ch, 0, 1, 1))};
          SUB_RC(ring_gemm_tc_variant(256, 1, xl, xh, ch.rows, cf16(bq(0, 1, 0)), cf16(bq(0, 1, 1)), N, n_pad, l,
                                      sl.tags, c->cfg.seeds[0], c->cfg.seeds[0], 1u, zo, ldz, ch.row0, nullptr,
                                      nullptr, c->sp[0]));
        } else if (c->cfg.path == IPC_PATH_TCG) {
          // Galois-ring Shamir: party i's own share only, K = l
          const int8_t* xl[2] = {i8p(plane(c, ch, i, vec, 0)), i8p(plane(c, ch, i, vec, 0))};
          const int8_t* xh[2] = {i8p(plane(c, ch, i, vec, 1)), i8p(plane(c, ch, i, vec, 1))};
          SUB_RC(ring_gemm_tc_variant(256, 1, xl, xh, ch.rows, cf16(bq(i, vec, 0)), cf16(bq(i, vec, 1)), N, n_pad, l,
                                      sl.tags, c->cfg.seeds[i], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo,
                                      ldz, ch.row0, nullptr, nullptr, c->sp[i]));
        } else if (c->cfg.path == IPC_PATH_TC) {
          const int8_t* xl[2] = {i8p(plane(c, ch, i, vec, 0)), i8p(plane(c, ch, prev, vec, 0))};
          const int8_t* xh[2] = {i8p(plane(c, ch, i, vec, 1)), i8p(plane(c, ch, prev, vec, 1))};
          SUB_RC(ipc_ring_gemm_tc(xl, xh, ch.rows, cf16(bq(i, vec, 0)), cf16(bq(i, vec, 1)), N, n_pad, l, sl.tags,
                                  c->cfg.seeds[i], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo, ldz, ch.row0,
                                  c->sp[i]));
        } else {
          const int8_t* xl[2] = {i8p(plane(c, ch, i, vec, 0)), i8p(plane(c, ch, prev, vec, 0))};
          const int8_t* xh[2] = {i8p(plane(c, ch, i, vec, 1)), i8p(plane(c, ch, prev, vec, 1))};
          SUB_RC(ipc_ring_gemm(c->cfg.path, xl, xh, ch.rows, i8p(bq(i, vec, 0)), i8p(bq(i, vec, 1)), N, n_pad, l,
                               sl.tags, c->cfg.seeds[i], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo, ldz,
                               ch.row0, c->sp[i]));
        }
      }
      SUB_TRY(cudaEventRecord(c->ev_gemm[i][set], c->sp[i]));
      SUB_TRY(cudaStreamWaitEvent(c->sc, c->ev_gemm[i][set], 0));
    }
    auto u16p = [](const uint8_t* p) { return reinterpret_cast<const uint16_t*>(p); };
    auto u32p = [](const uint8_t* p) { return reinterpret_cast<const uint32_t*>(p); };
    if (c->cfg.lift) {
      const uint32_t* ml32[3] = {u32p(zm[0]), u32p(zm[1]), u32p(zm[2])};
      const uint32_t* zc32[3] = {u32p(zc[0]), u32p(zc[1]), u32p(zc[2])};
      const uint16_t* zc16[3] = {u16p(zc[0]), u16p(zc[1]), u16p(zc[2])};
      const bool nolift = c->cfg.lift == IPC_LIFT_NONE;
      SUB_RC(compare_launch_liftfree(nolift ? nullptr : zc16, nolift ? zc32 : nullptr, ml32, ldz, N, ch.rows, ch.row0,
                                     sl.tags, c->cfg.seeds, c->cfg.thr_a, c->cfg.thr_b, kLog2BlockWords, sl.roots,
                                     r.ld_roots, nullptr, 0, c->sc));
    } else {
      const uint16_t* zcc[3] = {u16p(zc[0]), u16p(zc[1]), u16p(zc[2])};
      const uint16_t* zmc[3] = {u16p(zm[0]), u16p(plain ? zm[0] : zm[1]), u16p(plain ? zm[0] : zm[2])};
      SUB_RC(compare_launch_tiles(zcc, zmc, ldz, N, ch.rows, ch.row0, sl.tags, c->cfg.seeds, c->cfg.thr_a,
                                  kLog2BlockWords, sl.roots, r.ld_roots, nullptr, 0, nullptr, nullptr, 0, c->sc,
                                  nullptr, plain));
    }
    SUB_TRY(cudaEventRecord(c->ev_cmp[set], c->sc));
  }
  const uint32_t n_blocks =
      static_cast<uint32_t>((c->rows + (32ull << kLog2BlockWords) - 1) >> (5 + kLog2BlockWords));
  SUB_RC(ipc_or_finalize(sl.roots, r.ld_roots, n_blocks, kLog2BlockWords, Q, R, sl.tags, c->cfg.seeds, sl.shares_dev,
                         c->sc));
  SUB_TRY(cudaMemcpyAsync(sl.shares_host, sl.shares_dev, 3ull * Q, cudaMemcpyDeviceToHost, c->sc));
  SUB_TRY(cudaEventRecord(sl.done, c->sc));
#undef SUB_TRY
#undef SUB_RC
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
  const Slot& sl = c->slots[r.slot];
  int rc = wait_event(c, sl.done, timeout_ms);
  if (rc) return rc;
  rc = check_device_status(c);
  if (rc) return rc;
  std::memcpy(shares_out, sl.shares_host, 3ull * r.Q);
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
  int rc = wait_event(c, c->slots[r.slot].done, -1);
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
  const Slot& sl = c->slots[r.slot];
  int rc = wait_event(c, sl.done, timeout_ms);
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
    for (uint32_t q = 0; q < r.Q; ++q) h ^= msg_hash(2, p, q, 0, sl.shares_host[static_cast<size_t>(p) * r.Q + q]);
  *hash_out = h;
  return IPC_OK;
}

extern "C" int ipc_debug_stall_party(ipc_ctx* c, uint32_t party, uint32_t limit_us) {
  if (!c || party > 2 || limit_us == 0 || limit_us > 1000000)
    return fail(c, IPC_EINVAL, "ipc_debug_stall_party: party 0..2 and limit_us in 1..1000000");
  CTX_TRY(c, cudaSetDevice(c->cfg.device));
  if (!c->stall_flag) {
    CTX_TRY(c, cudaMalloc(&c->stall_flag, sizeof(uint32_t)));
    CTX_TRY(c, cudaMemset(c->stall_flag, 0, sizeof(uint32_t)));  // nothing ever sets it
  }
  c->stall_party = static_cast<int>(party);
  c->stall_us = limit_us;
  return IPC_OK;
}

extern "C" int ipc_release(ipc_ctx* c, uint64_t req_id) {
  if (!c) return fail(c, IPC_EINVAL, "ipc_release: null context");
  auto it = c->reqs.find(req_id);
  if (it == c->reqs.end()) {
    const int rc = serve_release(c, req_id);
    return rc == IPC_ENOTFOUND ? fail(c, IPC_ENOTFOUND, "unknown request id") : rc;
  }
  cudaEventSynchronize(c->slots[it->second.slot].done);
  release_request(c, it->second);
  c->reqs.erase(it);
  return IPC_OK;
}
