// A9 -- serving: continuous batching of query requests over the resident database.
//
// A request of Q queries occupies Q consecutive query slots of a column pool (R columns per
// slot, columns q*R + rho as in a stand-alone request). One serving step runs one resident
// database chunk for every active column: the six share-domain GEMMs (A3, three party streams)
// and the comparison phase (A4-A8 with the in-block OR) over the column tiles that hold active
// columns, replayed from a CUDA graph keyed by (chunk, GEMM tile variant); the tile list lives
// in device memory and is rewritten before each replay, so one graph serves every mix of
// requests. A request admitted while the loop is at chunk c visits chunks c, c+1, ... and
// after the last one its OR tree is finished (A8) and its bit components copied out; its slots
// are then free for the next pending request. Every PRF counter depends on the request id,
// query, rotation and database row only, so a request's shares do not depend on which other
// requests shared its steps, nor on its slot or starting chunk.
//
// Admission: requests wait in FIFO order until a contiguous run of free slots can hold them;
// the pool is sized from free device memory at start (or fixed by the caller).
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <fstream>
#include <memory>
#include <sstream>

#include "context.cuh"

namespace ipc {
int ring_gemm_i8_variant(int variant, const int8_t* const x_lo[2], const int8_t* const x_hi[2], size_t x_rows,
                         const int8_t* b_lo, const int8_t* b_hi, uint32_t n_cols, uint32_t n_pad, uint32_t l,
                         const uint32_t* col_tags, uint64_t seed_own, uint64_t seed_prev, uint32_t vec, uint16_t* z,
                         size_t ldz, uint64_t row0, const uint32_t* col_tiles, const uint32_t* n_col_list,
                         cudaStream_t stream);
int or_finalize_strided(uint32_t* roots, size_t ld_roots, size_t plane, uint32_t n_blocks, uint32_t p, uint32_t Q,
                        uint32_t R, const uint32_t* col_tags, const uint64_t seeds[3], uint8_t* bit_shares,
                        cudaStream_t st);
template <typename T>
int prep_query_strided(const uint16_t* y, uint64_t y_plane, uint32_t Q, const ipc_geom* g, uint32_t party, T* b_lo,
                       T* b_hi, uint32_t n_pad, void* stream, const char* who);

namespace {

constexpr uint32_t kPoolAlign = 256;  // pool columns are padded to the widest tile

struct Variant {
  const char* name;
  uint32_t tile_cols;
  int id;  // tcgen05: tile width; int8 paths: ring_gemm_i8_variant index
};
const Variant kTcVariants[] = {{"tc256", 256, 256}, {"tc128", 128, 128}};
const Variant kI8Variants[] = {{"mix128", 128, 0}, {"mma128", 128, 1}, {"mma64", 64, 2}, {"mma32", 32, 3}};

double now_s() {
  using namespace std::chrono;
  return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct SReq {
  uint64_t id = 0;
  uint32_t Q = 0, N = 0;
  std::vector<uint16_t> y;       // [vec][3][Q][l] query shares (host copy)
  std::vector<uint32_t> tags;    // [N][2]
  std::vector<uint8_t> shares;   // [3][Q] bit components, once done
  uint32_t slot0 = 0;
  uint32_t chunks_left = 0;
  int state = 0;  // 0 pending, 1 active, 2 done
  double t_submit = 0, t_admit = -1, t_done = -1;
  struct Server* srv = nullptr;
};

struct Bucket {
  uint32_t cols;  // active columns up to this many
  int variant;
};

struct Server {
  ipc_ctx* c = nullptr;
  ipc_serve_config cfg{};
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::string worker_err;

  const Variant* variants = nullptr;
  int n_variants = 0;
  std::vector<Bucket> buckets;  // ascending cols; empty = always cfg.variant
  std::string tuning_json;

  uint32_t R = 0, slots = 0, pool_pad = 0, n_chunks = 0;
  size_t ld_roots = 0;
  uint8_t* bq = nullptr;         // [party][vec][limb][pool_pad][2l] limbs
  uint16_t* ystage = nullptr;    // [vec][3][slots][l]
  uint32_t* tags = nullptr;      // [pool_pad][2]
  uint32_t* roots = nullptr;     // [3][pool_pad][ld_roots]
  uint16_t* z = nullptr;         // [vec][party][pool_pad][chunk_rows]
  uint8_t* shares_dev = nullptr;   // [3 * slots]
  uint8_t* shares_host = nullptr;  // pinned [3 * slots]
  std::vector<uint32_t*> list_dev;   // per variant: [pool_pad / tile_cols] tile indices
  std::vector<uint32_t*> count_dev;  // per variant: 1 word
  uint32_t* list_host[2] = {nullptr, nullptr};  // pinned staging, one per in-flight step
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {}, ev_step[2] = {};
  std::map<std::pair<uint32_t, int>, cudaGraphExec_t> graphs;

  std::vector<uint8_t> slot_used;
  std::deque<SReq*> pending;
  std::vector<SReq*> active;  // worker thread only
  std::map<uint64_t, std::unique_ptr<SReq>> reqs;
  uint32_t cursor = 0;
  double t0 = 0;
  // statistics (under mu)
  uint64_t steps = 0, admitted = 0, completed = 0;
  double comparisons = 0;
  std::vector<uint32_t> variant_steps;
};

namespace {

// First fit: the lowest start of `want` consecutive free slots, or -1.
int64_t first_fit(const std::vector<uint8_t>& used, uint32_t want) {
  uint32_t run = 0;
  for (uint32_t s = 0; s < used.size(); ++s) {
    run = used[s] ? 0 : run + 1;
    if (run == want) return static_cast<int64_t>(s + 1 - want);
  }
  return -1;
}

// Sorted distinct tiles of width tw covering the column ranges [col0[i], col0[i] + ncols[i]).
uint32_t tile_list(const uint32_t* col0, const uint32_t* ncols, uint32_t n, uint32_t tw, uint32_t* out,
                   uint32_t max_out) {
  std::vector<uint32_t> t;
  for (uint32_t i = 0; i < n; ++i) {
    if (ncols[i] == 0) continue;
    for (uint32_t k = col0[i] / tw; k <= (col0[i] + ncols[i] - 1) / tw; ++k) t.push_back(k);
  }
  std::sort(t.begin(), t.end());
  t.erase(std::unique(t.begin(), t.end()), t.end());
  const uint32_t m = static_cast<uint32_t>(std::min<size_t>(t.size(), max_out));
  std::copy(t.begin(), t.begin() + m, out);
  return static_cast<uint32_t>(t.size());
}

int pick_variant(const Server& S, uint32_t active_cols) {
  for (const Bucket& b : S.buckets)
    if (active_cols <= b.cols) return b.variant;
  return S.buckets.empty() ? S.cfg.variant : S.buckets.back().variant;
}

#define SRV_TRY(expr)                                         \
  do {                                                        \
    cudaError_t e__ = (expr);                                 \
    if (e__ != cudaSuccess) return ctx_cfail(S.c, e__, #expr); \
  } while (0)
#define SRV_RC(expr)                           \
  do {                                         \
    int rc__ = (expr);                         \
    if (rc__ != IPC_OK) {                      \
      S.c->err = thread_last_error();          \
      return rc__;                             \
    }                                          \
  } while (0)

uint8_t* bq_plane(const Server& S, int party, int vec, int limb) {
  return S.bq + static_cast<size_t>((party * 2 + vec) * 2 + limb) * S.pool_pad * S.c->kq * S.c->qsz;
}

uint16_t* z_plane(const Server& S, int vec, int party) {
  return S.z + static_cast<size_t>(vec * 3 + party) * S.pool_pad * S.c->cfg.db_chunk_rows;
}

// A3 of one party and vector over the listed tiles of the pool, for one chunk.
int gemm(Server& S, int v, const Chunk& ch, int party, int vec, cudaStream_t st) {
  ipc_ctx* c = S.c;
  const int prev = (party + 2) % 3;
  const Variant& V = S.variants[v];
  uint16_t* zo = z_plane(S, vec, party);
  const size_t ldz = c->cfg.db_chunk_rows;
  if (c->cfg.path == IPC_PATH_TC || c->cfg.path == IPC_PATH_TCG) {
    // replicated sharing: [own | previous] components, K = 2l; Galois-ring Shamir: own share, K = l
    const bool gal = c->cfg.path == IPC_PATH_TCG;
    const int other = gal ? party : prev;
    auto p16 = [](const uint8_t* p) { return reinterpret_cast<const uint16_t*>(p); };
    auto p8 = [](const uint8_t* p) { return reinterpret_cast<const int8_t*>(p); };
    const int8_t* xl[2] = {p8(ctx_plane(c, ch, party, vec, 0)), p8(ctx_plane(c, ch, other, vec, 0))};
    const int8_t* xh[2] = {p8(ctx_plane(c, ch, party, vec, 1)), p8(ctx_plane(c, ch, other, vec, 1))};
    return ring_gemm_tc_variant(V.tile_cols, gal ? 1 : 2, xl, xh, ch.rows, p16(bq_plane(S, party, vec, 0)),
                                p16(bq_plane(S, party, vec, 1)), S.pool_pad, S.pool_pad, c->l, S.tags,
                                c->cfg.seeds[party], c->cfg.seeds[prev], static_cast<uint32_t>(vec), zo, ldz, ch.row0,
                                S.list_dev[v], S.count_dev[v], st);
  }
  auto p8 = [](const uint8_t* p) { return reinterpret_cast<const int8_t*>(p); };
  const int8_t* xl[2] = {p8(ctx_plane(c, ch, party, vec, 0)), p8(ctx_plane(c, ch, prev, vec, 0))};
  const int8_t* xh[2] = {p8(ctx_plane(c, ch, party, vec, 1)), p8(ctx_plane(c, ch, prev, vec, 1))};
  return ring_gemm_i8_variant(V.id, xl, xh, ch.rows, p8(bq_plane(S, party, vec, 0)), p8(bq_plane(S, party, vec, 1)),
                              S.pool_pad, S.pool_pad, c->l, S.tags, c->cfg.seeds[party], c->cfg.seeds[prev],
                              static_cast<uint32_t>(vec), zo, ldz, ch.row0, S.list_dev[v], S.count_dev[v], st);
}

int compare(Server& S, int v, const Chunk& ch, cudaStream_t st) {
  const uint16_t* zc[3] = {z_plane(S, 0, 0), z_plane(S, 0, 1), z_plane(S, 0, 2)};
  const uint16_t* zm[3] = {z_plane(S, 1, 0), z_plane(S, 1, 1), z_plane(S, 1, 2)};
  return compare_launch_tiles(zc, zm, S.c->cfg.db_chunk_rows, S.pool_pad, ch.rows, ch.row0, S.tags, S.c->cfg.seeds,
                              S.c->cfg.thr_a, kLog2BlockWords, S.roots, S.ld_roots, nullptr, 0, S.list_dev[v],
                              S.count_dev[v], S.variants[v].tile_cols, st, nullptr, S.c->cfg.plain_mask != 0);
}

// The graph of one step: fork the party streams off the control stream, two GEMMs per party,
// join, then the comparison phase on the control stream.
int step_graph(Server& S, uint32_t chunk, int v, cudaGraphExec_t* out) {
  auto it = S.graphs.find({chunk, v});
  if (it != S.graphs.end()) {
    *out = it->second;
    return IPC_OK;
  }
  ipc_ctx* c = S.c;
  const Chunk& ch = c->chunks[chunk];
  cudaGraph_t g = nullptr;
  SRV_TRY(cudaStreamBeginCapture(c->sc, cudaStreamCaptureModeThreadLocal));
  int rc = IPC_OK;
  cudaError_t e = cudaEventRecord(S.ev_fork, c->sc);
  for (int i = 0; i < 3 && e == cudaSuccess && rc == IPC_OK; ++i) {
    e = cudaStreamWaitEvent(c->sp[i], S.ev_fork, 0);
    for (int vec = 0; vec < 2 && e == cudaSuccess && rc == IPC_OK; ++vec) rc = gemm(S, v, ch, i, vec, c->sp[i]);
    if (e == cudaSuccess && rc == IPC_OK) e = cudaEventRecord(S.ev_join[i], c->sp[i]);
    if (e == cudaSuccess && rc == IPC_OK) e = cudaStreamWaitEvent(c->sc, S.ev_join[i], 0);
  }
  if (e == cudaSuccess && rc == IPC_OK) rc = compare(S, v, ch, c->sc);
  const cudaError_t e_end = cudaStreamEndCapture(c->sc, &g);
  if (rc != IPC_OK) {
    if (g) cudaGraphDestroy(g);
    S.c->err = thread_last_error();
    return rc;
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ctx_cfail(c, e, "serving step capture");
  }
  if (e_end != cudaSuccess) return ctx_cfail(c, e_end, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return ctx_cfail(c, ei, "cudaGraphInstantiate");
  S.graphs[{chunk, v}] = exec;
  *out = exec;
  return IPC_OK;
}

// Writes n tiles (and the count) of variant v to its device list, through the pinned staging
// slot of this step.
int upload_list(Server& S, int v, const std::vector<uint32_t>& tiles, uint64_t step) {
  uint32_t* h = S.list_host[step & 1];
  h[0] = static_cast<uint32_t>(tiles.size());
  std::copy(tiles.begin(), tiles.end(), h + 1);
  SRV_TRY(cudaMemcpyAsync(S.count_dev[v], h, sizeof(uint32_t), cudaMemcpyHostToDevice, S.c->sc));
  if (!tiles.empty())
    SRV_TRY(cudaMemcpyAsync(S.list_dev[v], h + 1, tiles.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, S.c->sc));
  return IPC_OK;
}

// A2 for an admitted request into its slots of the pool.
int admit(Server& S, SReq* r) {
  ipc_ctx* c = S.c;
  const size_t l = c->l;
  const uint32_t col0 = r->slot0 * S.R;
  for (int vec = 0; vec < 2; ++vec)
    for (int j = 0; j < 3; ++j)
      SRV_TRY(cudaMemcpyAsync(S.ystage + ((static_cast<size_t>(vec) * 3 + j) * S.slots + r->slot0) * l,
                              r->y.data() + (static_cast<size_t>(vec) * 3 + j) * r->Q * l, r->Q * l * sizeof(uint16_t),
                              cudaMemcpyHostToDevice, c->sc));
  SRV_TRY(cudaMemcpyAsync(S.tags + 2ull * col0, r->tags.data(), r->tags.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, c->sc));
  const size_t row_bytes = static_cast<size_t>(c->kq) * c->qsz;
  for (int i = 0; i < 3; ++i)
    for (int vec = 0; vec < 2; ++vec) {
      const uint16_t* y = S.ystage + (static_cast<size_t>(vec) * 3 * S.slots + r->slot0) * l;
      uint8_t* lo = bq_plane(S, i, vec, 0) + col0 * row_bytes;
      uint8_t* hi = bq_plane(S, i, vec, 1) + col0 * row_bytes;
      if (c->cfg.path == IPC_PATH_TCG)
        SRV_RC(prep_query_galois_strided(y, static_cast<uint64_t>(S.slots) * l, r->Q, &c->cfg.geom, i,
                                         reinterpret_cast<uint16_t*>(lo), reinterpret_cast<uint16_t*>(hi), r->N, c->sc));
      else if (c->qsz == 2)
        SRV_RC(prep_query_strided<uint16_t>(y, static_cast<uint64_t>(S.slots) * l, r->Q, &c->cfg.geom, i,
                                            reinterpret_cast<uint16_t*>(lo), reinterpret_cast<uint16_t*>(hi), r->N,
                                            c->sc, "serving admission"));
      else
        SRV_RC(prep_query_strided<int8_t>(y, static_cast<uint64_t>(S.slots) * l, r->Q, &c->cfg.geom, i,
                                          reinterpret_cast<int8_t*>(lo), reinterpret_cast<int8_t*>(hi), r->N, c->sc,
                                          "serving admission"));
    }
  return IPC_OK;
}

void CUDART_CB on_done(void* arg) {
  SReq* r = static_cast<SReq*>(arg);
  Server* S = r->srv;
  std::lock_guard<std::mutex> lock(S->mu);
  r->shares.resize(3ull * r->Q);
  std::memcpy(r->shares.data(), S->shares_host + 3ull * r->slot0, 3ull * r->Q);
  r->t_done = now_s() - S->t0;
  r->state = 2;
  ++S->completed;
  S->cv_done.notify_all();
}

// A8 for a request that has visited every chunk, and the copy of its bit components.
int finish(Server& S, SReq* r) {
  ipc_ctx* c = S.c;
  const uint32_t col0 = r->slot0 * S.R;
  const uint32_t n_blocks =
      static_cast<uint32_t>((c->rows + (32ull << kLog2BlockWords) - 1) >> (5 + kLog2BlockWords));
  SRV_RC(or_finalize_strided(S.roots + static_cast<size_t>(col0) * S.ld_roots, S.ld_roots,
                             static_cast<size_t>(S.pool_pad) * S.ld_roots, n_blocks, kLog2BlockWords, r->Q, S.R,
                             S.tags + 2ull * col0, c->cfg.seeds, S.shares_dev + 3ull * r->slot0, c->sc));
  SRV_TRY(cudaMemcpyAsync(S.shares_host + 3ull * r->slot0, S.shares_dev + 3ull * r->slot0, 3ull * r->Q,
                          cudaMemcpyDeviceToHost, c->sc));
  SRV_TRY(cudaLaunchHostFunc(c->sc, on_done, r));
  return IPC_OK;
}

int run_step(Server& S, uint64_t step, const std::vector<SReq*>& admitted) {
  ipc_ctx* c = S.c;
  // at most two steps in flight: the staging slot of this step was last used two steps ago
  SRV_TRY(cudaEventSynchronize(S.ev_step[step & 1]));
  for (SReq* r : admitted) SRV_RC(admit(S, r));
  std::vector<uint32_t> c0, nc;
  uint32_t active_cols = 0;
  for (SReq* r : S.active) {
    c0.push_back(r->slot0 * S.R);
    nc.push_back(r->N);
    active_cols += r->N;
  }
  const int v = pick_variant(S, active_cols);
  const uint32_t tw = S.variants[v].tile_cols;
  std::vector<uint32_t> tiles(S.pool_pad / tw);
  tiles.resize(tile_list(c0.data(), nc.data(), static_cast<uint32_t>(c0.size()), tw, tiles.data(),
                         static_cast<uint32_t>(tiles.size())));
  SRV_RC(upload_list(S, v, tiles, step));
  cudaGraphExec_t exec = nullptr;
  SRV_RC(step_graph(S, S.cursor, v, &exec));
  SRV_TRY(cudaGraphLaunch(exec, c->sc));
  SRV_TRY(cudaEventRecord(S.ev_step[step & 1], c->sc));
  const Chunk& ch = c->chunks[S.cursor];
  std::vector<SReq*> still;
  std::vector<SReq*> done;
  for (SReq* r : S.active) {
    if (--r->chunks_left == 0)
      done.push_back(r);
    else
      still.push_back(r);
  }
  for (SReq* r : done) SRV_RC(finish(S, r));
  {
    std::lock_guard<std::mutex> lock(S.mu);
    for (SReq* r : done)
      for (uint32_t k = 0; k < r->Q; ++k) S.slot_used[r->slot0 + k] = 0;
    ++S.steps;
    S.comparisons += static_cast<double>(active_cols) * ch.rows;
    ++S.variant_steps[v];
  }
  S.active.swap(still);
  do {
    S.cursor = (S.cursor + 1) % static_cast<uint32_t>(c->chunks.size());
  } while (c->chunks[S.cursor].rows == 0);
  return IPC_OK;
}

void worker_main(Server* Sp) {
  Server& S = *Sp;
  cudaSetDevice(S.c->cfg.device);
  for (uint64_t step = 0;; ++step) {
    std::vector<SReq*> admitted;
    {
      std::unique_lock<std::mutex> lk(S.mu);
      S.cv_work.wait(lk, [&] { return S.stop || !S.pending.empty() || !S.active.empty(); });
      if (S.pending.empty() && S.active.empty()) break;  // stop requested and nothing left
      const double t = now_s() - S.t0;
      while (!S.pending.empty()) {
        SReq* r = S.pending.front();
        const int64_t s0 = first_fit(S.slot_used, r->Q);
        if (s0 < 0) break;
        for (uint32_t k = 0; k < r->Q; ++k) S.slot_used[s0 + k] = 1;
        r->slot0 = static_cast<uint32_t>(s0);
        r->state = 1;
        r->t_admit = t;
        r->chunks_left = S.n_chunks;
        S.pending.pop_front();
        admitted.push_back(r);
        ++S.admitted;
      }
    }
    for (SReq* r : admitted) S.active.push_back(r);
    if (S.active.empty()) continue;
    const int rc = run_step(S, step, admitted);
    if (rc != IPC_OK) {
      std::lock_guard<std::mutex> lock(S.mu);
      S.worker_err = S.c->err.empty() ? "serving step failed" : S.c->err;
      S.stop = true;
      S.cv_done.notify_all();
      break;
    }
  }
  cudaStreamSynchronize(S.c->sc);
}

// ---------------------------------------------------------------------------------------------
// Autotuner: per bucket of active columns, the GEMM variant with the shortest launch over the
// first resident chunk, one party and vector, the listed tiles covering that many columns.
// The table is cached as JSON keyed by device, geometry, chunk rows, path and pool width.
// ---------------------------------------------------------------------------------------------

std::string tune_key(const Server& S) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, S.c->cfg.device);
  std::ostringstream k;
  k << prop.name << "|sm" << prop.multiProcessorCount << "|l" << S.c->l << "|rows" << S.c->cfg.db_chunk_rows << "|path"
    << S.c->cfg.path << "|pool" << S.pool_pad;
  return k.str();
}

bool load_tuning(Server& S, const std::string& path, const std::string& key) {
  std::ifstream f(path);
  if (!f) return false;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string txt = ss.str();
  if (txt.find("\"key\": \"" + key + "\"") == std::string::npos) return false;
  std::vector<Bucket> b;
  size_t at = 0;
  while ((at = txt.find("\"cols\": ", at)) != std::string::npos) {
    at += 8;
    const uint32_t cols = static_cast<uint32_t>(std::strtoul(txt.c_str() + at, nullptr, 10));
    const size_t vn = txt.find("\"variant\": \"", at);
    if (vn == std::string::npos) return false;
    const size_t v0 = vn + 12, v1 = txt.find('"', v0);
    const std::string name = txt.substr(v0, v1 - v0);
    int v = -1;
    for (int i = 0; i < S.n_variants; ++i)
      if (name == S.variants[i].name) v = i;
    if (v < 0) return false;
    b.push_back({cols, v});
    at = v1;
  }
  if (b.empty()) return false;
  S.buckets = b;
  S.tuning_json = txt;
  return true;
}

int autotune(Server& S) {
  ipc_ctx* c = S.c;
  const std::string key = tune_key(S);
  if (S.cfg.tune_cache && load_tuning(S, S.cfg.tune_cache, key)) return IPC_OK;
  const Chunk& ch = c->chunks[0];
  cudaEvent_t e0, e1;
  SRV_TRY(cudaEventCreate(&e0));
  SRV_TRY(cudaEventCreate(&e1));
  std::ostringstream js;
  js << "{\"key\": \"" << key << "\", \"buckets\": [";
  std::vector<Bucket> b;
  bool first = true;
  for (uint32_t cols = kPoolAlign; ; cols *= 2) {
    const uint32_t w = std::min(cols, S.pool_pad);
    float best = 1e30f;
    int best_v = 0;
    std::ostringstream ms;
    for (int v = 0; v < S.n_variants; ++v) {
      const uint32_t tw = S.variants[v].tile_cols;
      std::vector<uint32_t> tiles((w + tw - 1) / tw);
      for (uint32_t k = 0; k < tiles.size(); ++k) tiles[k] = k;
      SRV_RC(upload_list(S, v, tiles, 0));
      SRV_TRY(cudaStreamSynchronize(c->sc));
      SRV_RC(gemm(S, v, ch, 0, 0, c->sc));  // warm-up (also sets the kernel attributes before any capture)
      SRV_TRY(cudaEventRecord(e0, c->sc));
      for (int rep = 0; rep < 2; ++rep) SRV_RC(gemm(S, v, ch, 0, 0, c->sc));
      SRV_TRY(cudaEventRecord(e1, c->sc));
      SRV_TRY(cudaEventSynchronize(e1));
      float t = 0;
      SRV_TRY(cudaEventElapsedTime(&t, e0, e1));
      t /= 2;
      ms << (v ? ", " : "") << "\"" << S.variants[v].name << "\": " << t;
      if (t < best) {
        best = t;
        best_v = v;
      }
    }
    b.push_back({w, best_v});
    js << (first ? "" : ", ") << "{\"cols\": " << w << ", \"variant\": \"" << S.variants[best_v].name
       << "\", \"ms\": {" << ms.str() << "}}";
    first = false;
    if (w == S.pool_pad) break;
  }
  js << "]}";
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  S.buckets = b;
  S.tuning_json = js.str();
  if (S.cfg.tune_cache) {
    std::ofstream f(S.cfg.tune_cache);
    if (f) f << S.tuning_json << "\n";
  }
  return IPC_OK;
}

void free_server(Server* S) {
  if (!S) return;
  cudaSetDevice(S->c->cfg.device);
  cudaDeviceSynchronize();
  for (auto& kv : S->graphs) cudaGraphExecDestroy(kv.second);
  cudaFree(S->bq);
  cudaFree(S->ystage);
  cudaFree(S->tags);
  cudaFree(S->roots);
  cudaFree(S->z);
  cudaFree(S->shares_dev);
  if (S->shares_host) cudaFreeHost(S->shares_host);
  for (int k = 0; k < 2; ++k)
    if (S->list_host[k]) cudaFreeHost(S->list_host[k]);
  for (auto* p : S->list_dev) cudaFree(p);
  for (auto* p : S->count_dev) cudaFree(p);
  if (S->ev_fork) cudaEventDestroy(S->ev_fork);
  for (auto e : S->ev_join)
    if (e) cudaEventDestroy(e);
  for (auto e : S->ev_step)
    if (e) cudaEventDestroy(e);
  delete S;
}

// Per query slot: R columns of B planes (12 x 2l limbs), of z (6 x chunk rows) and of roots
// (3 x ld_roots), the slot's query shares (6 x l) and bit components.
size_t bytes_per_slot(const ipc_ctx* c, uint32_t R, size_t ld_roots) {
  const size_t per_col = 12ull * c->kq * c->qsz + 6ull * c->cfg.db_chunk_rows * 2 + 3ull * ld_roots * 4 + 8;
  return R * per_col + 6ull * c->l * 2 + 3;
}

}  // namespace

int serve_fetch_shares(ipc_ctx* c, uint64_t id, uint8_t* out, size_t n, int timeout_ms) {
  Server* S = c->srv;
  if (!S) return IPC_ENOTFOUND;
  SReq* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return IPC_ENOTFOUND;
    r = it->second.get();
    if (n != r->Q) return ctx_fail(c, IPC_EINVAL, "n_queries does not match the request");
    auto ready = [&] { return r->state == 2 || !S->worker_err.empty(); };
    if (timeout_ms < 0)
      S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
      return ctx_fail(c, IPC_ETIMEOUT, "request not finished within the timeout");
    if (r->state != 2) return ctx_fail(c, IPC_ECUDA, "serving loop stopped: " + S->worker_err);
    std::memcpy(out, r->shares.data(), 3ull * r->Q);
  }
  return ctx_check_device_status(c);
}

int serve_release(ipc_ctx* c, uint64_t id) {
  Server* S = c->srv;
  if (!S) return IPC_ENOTFOUND;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return IPC_ENOTFOUND;
  if (it->second->state != 2) return ctx_fail(c, IPC_EAGAIN, "ipc_release: the request is still running");
  S->reqs.erase(it);
  return IPC_OK;
}

void serve_shutdown(ipc_ctx* c) {
  Server* S = c ? c->srv : nullptr;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  c->srv = nullptr;
  free_server(S);
}

}  // namespace ipc

using namespace ipc;

extern "C" int ipc_serve_start(ipc_ctx* c, const ipc_serve_config* cfg) {
  if (!c || !cfg) return ctx_fail(c, IPC_EINVAL, "ipc_serve_start: null argument");
  if (c->srv) return ctx_fail(c, IPC_EINVAL, "ipc_serve_start: already serving");
  if (c->rows == 0) return ctx_fail(c, IPC_EINVAL, "ipc_serve_start: no database rows loaded");
  if (c->cfg.path == IPC_PATH_I32) return ctx_fail(c, IPC_EINVAL, "ipc_serve_start: the int32 path has no tile variants");
  if (c->cfg.plain_mask) return ctx_fail(c, IPC_EINVAL, "ipc_serve_start: protocol 1 (plain masks) is not served");
  if (c->cfg.lift) return ctx_fail(c, IPC_EINVAL, "ipc_serve_start: the lifting variants are not served");
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return ctx_cfail(c, e, "cudaSetDevice");
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return ctx_cfail(c, e, "cudaDeviceSynchronize");
  auto* Sp = new Server();
  Server& S = *Sp;
  S.c = c;
  S.cfg = *cfg;
  const bool tc = c->cfg.path == IPC_PATH_TC || c->cfg.path == IPC_PATH_TCG;
  S.variants = tc ? kTcVariants : kI8Variants;
  S.n_variants = tc ? 2 : 4;
  if (cfg->variant != IPC_SERVE_AUTOTUNE && (cfg->variant < 0 || cfg->variant >= S.n_variants)) {
    delete Sp;
    return ctx_fail(c, IPC_EINVAL, "ipc_serve_start: unknown variant");
  }
  S.R = c->cfg.geom.R;
  S.n_chunks = 0;
  for (const Chunk& ch : c->chunks) S.n_chunks += ch.rows > 0;
  S.ld_roots = (c->chunks.size() * c->cfg.db_chunk_rows) >> (5 + kLog2BlockWords);
  // pool size: as asked, else two of the largest requests if free device memory allows
  // (keeping 4 GiB and 10 % of the device in reserve), else what it allows
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t reserve = std::max<size_t>(4ull << 30, total_b / 10);
  const size_t per_slot = bytes_per_slot(c, S.R, S.ld_roots);
  uint32_t slots = cfg->pool_queries;
  if (slots == 0) {
    const size_t avail = free_b > reserve ? free_b - reserve : 0;
    slots = static_cast<uint32_t>(std::min<size_t>(avail / per_slot, 2u * c->cfg.max_queries));
  }
  if (slots == 0) {
    delete Sp;
    return ctx_fail(c, IPC_ENOMEM, "ipc_serve_start: not enough device memory for a column pool");
  }
  S.slots = slots;
  S.pool_pad = (slots * S.R + kPoolAlign - 1) / kPoolAlign * kPoolAlign;
  S.slot_used.assign(slots, 0);
  S.variant_steps.assign(S.n_variants, 0);
  const size_t l = c->l;
  bool ok = cudaMalloc(&S.bq, 12ull * S.pool_pad * c->kq * c->qsz) == cudaSuccess &&
            cudaMalloc(&S.ystage, 6ull * slots * l * sizeof(uint16_t)) == cudaSuccess &&
            cudaMalloc(&S.tags, 2ull * S.pool_pad * sizeof(uint32_t)) == cudaSuccess &&
            cudaMalloc(&S.roots, 3ull * S.pool_pad * S.ld_roots * sizeof(uint32_t)) == cudaSuccess &&
            cudaMalloc(&S.z, 6ull * S.pool_pad * c->cfg.db_chunk_rows * sizeof(uint16_t)) == cudaSuccess &&
            cudaMalloc(&S.shares_dev, 3ull * slots) == cudaSuccess &&
            cudaMallocHost(&S.shares_host, 3ull * slots) == cudaSuccess &&
            cudaMallocHost(&S.list_host[0], (S.pool_pad / 32 + 1) * sizeof(uint32_t)) == cudaSuccess &&
            cudaMallocHost(&S.list_host[1], (S.pool_pad / 32 + 1) * sizeof(uint32_t)) == cudaSuccess;
  for (int v = 0; v < S.n_variants && ok; ++v) {
    uint32_t* ld = nullptr;
    uint32_t* cd = nullptr;
    ok = cudaMalloc(&ld, (S.pool_pad / S.variants[v].tile_cols) * sizeof(uint32_t)) == cudaSuccess &&
         cudaMalloc(&cd, sizeof(uint32_t)) == cudaSuccess;
    S.list_dev.push_back(ld);
    S.count_dev.push_back(cd);
  }
  ok = ok && cudaEventCreateWithFlags(&S.ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&S.ev_step[0], cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&S.ev_step[1], cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 3 && ok; ++i) ok = cudaEventCreateWithFlags(&S.ev_join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_server(Sp);
    return ctx_fail(c, IPC_ENOMEM, "ipc_serve_start: device memory for the column pool");
  }
  // every pool byte defined (tiles of partly used columns compute on them); tags of unused
  // columns are request id 0
  ok = cudaMemsetAsync(S.bq, 0, 12ull * S.pool_pad * c->kq * c->qsz, c->sc) == cudaSuccess &&
       cudaMemsetAsync(S.tags, 0, 2ull * S.pool_pad * sizeof(uint32_t), c->sc) == cudaSuccess &&
       cudaMemsetAsync(S.z, 0, 6ull * S.pool_pad * c->cfg.db_chunk_rows * sizeof(uint16_t), c->sc) == cudaSuccess;
  for (int v = 0; v < S.n_variants && ok; ++v) ok = cudaMemsetAsync(S.count_dev[v], 0, 4, c->sc) == cudaSuccess;
  if (ok) ok = cudaStreamSynchronize(c->sc) == cudaSuccess;
  status_ptr();  // the status word exists before any capture
  int rc = ok ? IPC_OK : ctx_cfail(c, cudaGetLastError(), "ipc_serve_start: pool initialisation");
  if (rc == IPC_OK) {
    if (cfg->variant == IPC_SERVE_AUTOTUNE) {
      rc = autotune(S);
    } else {
      // warm-up launch of the chosen variant (kernel attributes are set outside any capture)
      rc = gemm(S, cfg->variant, c->chunks[0], 0, 0, c->sc);
    }
  }
  if (rc == IPC_OK) {
    // one comparison launch with an empty list: attributes set before capture
    for (int v = 0; v < S.n_variants && rc == IPC_OK; ++v) rc = upload_list(S, v, {}, 0);
    if (rc == IPC_OK) rc = compare(S, 0, c->chunks[0], c->sc);
    if (rc == IPC_OK && cudaStreamSynchronize(c->sc) != cudaSuccess) rc = ctx_cfail(c, cudaGetLastError(), "warm-up");
  }
  if (rc != IPC_OK) {
    free_server(Sp);
    return rc;
  }
  S.cursor = 0;
  while (c->chunks[S.cursor].rows == 0) ++S.cursor;
  S.t0 = now_s();
  c->srv = Sp;
  S.worker = std::thread(worker_main, Sp);
  return IPC_OK;
}

extern "C" int ipc_serve_submit(ipc_ctx* c, const uint16_t* const code[3], const uint16_t* const mask[3],
                                size_t n_queries, uint64_t* req_id) {
  if (!c || !code || !mask || !req_id) return ctx_fail(c, IPC_EINVAL, "ipc_serve_submit: null argument");
  Server* S = c->srv;
  if (!S) return ctx_fail(c, IPC_EINVAL, "ipc_serve_submit: the context is not serving");
  for (int j = 0; j < 3; ++j)
    if (!code[j] || !mask[j]) return ctx_fail(c, IPC_EINVAL, "ipc_serve_submit: null component");
  if (n_queries == 0 || n_queries > c->cfg.max_queries || n_queries > S->slots)
    return ctx_fail(c, IPC_EINVAL, "ipc_serve_submit: n_queries must be in 1..min(max_queries, pool slots)");
  const uint32_t max_pending = S->cfg.max_pending ? S->cfg.max_pending : 1024;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (!S->worker_err.empty()) return ctx_fail(c, IPC_ECUDA, "serving loop stopped: " + S->worker_err);
    if (S->stop) return ctx_fail(c, IPC_EINVAL, "ipc_serve_submit: the loop is stopping");
    if (S->pending.size() >= max_pending) return ctx_fail(c, IPC_EAGAIN, "ipc_serve_submit: pending queue full");
  }
  auto r = std::make_unique<SReq>();
  r->Q = static_cast<uint32_t>(n_queries);
  r->N = r->Q * S->R;
  r->srv = S;
  const size_t l = c->l, n = static_cast<size_t>(r->Q) * l;
  r->y.resize(6 * n);
  for (int vec = 0; vec < 2; ++vec)
    for (int j = 0; j < 3; ++j) std::memcpy(r->y.data() + (vec * 3 + j) * n, vec ? mask[j] : code[j], n * 2);
  {
    std::lock_guard<std::mutex> lock(c->id_mu);
    r->id = c->next_id++;
  }
  r->tags.resize(2ull * r->N);
  for (uint32_t q = 0; q < r->Q; ++q)
    for (uint32_t rho = 0; rho < S->R; ++rho) {
      r->tags[2 * (q * S->R + rho)] = static_cast<uint32_t>(r->id);
      r->tags[2 * (q * S->R + rho) + 1] = (q << 5) | rho;
    }
  *req_id = r->id;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    r->t_submit = now_s() - S->t0;
    S->pending.push_back(r.get());
    S->reqs[r->id] = std::move(r);
  }
  S->cv_work.notify_one();
  return IPC_OK;
}

extern "C" int ipc_serve_stop(ipc_ctx* c) {
  if (!c || !c->srv) return ctx_fail(c, IPC_EINVAL, "ipc_serve_stop: the context is not serving");
  std::string err;
  {
    std::lock_guard<std::mutex> lock(c->srv->mu);
    err = c->srv->worker_err;
  }
  serve_shutdown(c);
  return err.empty() ? IPC_OK : ctx_fail(c, IPC_ECUDA, "serving loop stopped: " + err);
}

extern "C" int ipc_serve_stats(ipc_ctx* c, ipc_serve_counters* out) {
  if (!c || !out) return ctx_fail(c, IPC_EINVAL, "ipc_serve_stats: null argument");
  Server* S = c->srv;
  if (!S) return ctx_fail(c, IPC_EINVAL, "ipc_serve_stats: the context is not serving");
  std::lock_guard<std::mutex> lock(S->mu);
  std::memset(out, 0, sizeof *out);
  out->steps = S->steps;
  out->admitted = S->admitted;
  out->completed = S->completed;
  out->pending = S->pending.size();
  out->comparisons = S->comparisons;
  out->pool_queries = S->slots;
  out->pool_cols = S->pool_pad;
  out->n_chunks = S->n_chunks;
  out->elapsed_s = now_s() - S->t0;
  for (int v = 0; v < S->n_variants && v < 4; ++v) out->variant_steps[v] = S->variant_steps[v];
  return IPC_OK;
}

extern "C" int ipc_serve_times(ipc_ctx* c, uint64_t req_id, double out[3]) {
  if (!c || !out) return ctx_fail(c, IPC_EINVAL, "ipc_serve_times: null argument");
  Server* S = c->srv;
  if (!S) return ctx_fail(c, IPC_EINVAL, "ipc_serve_times: the context is not serving");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(req_id);
  if (it == S->reqs.end()) return ctx_fail(c, IPC_ENOTFOUND, "unknown request id");
  out[0] = it->second->t_submit;
  out[1] = it->second->t_admit;
  out[2] = it->second->t_done;
  return IPC_OK;
}

extern "C" int ipc_serve_tuning(ipc_ctx* c, char* buf, size_t len) {
  if (!c || !buf || len == 0) return ctx_fail(c, IPC_EINVAL, "ipc_serve_tuning: null argument");
  Server* S = c->srv;
  if (!S) return ctx_fail(c, IPC_EINVAL, "ipc_serve_tuning: the context is not serving");
  std::lock_guard<std::mutex> lock(S->mu);
  const std::string& t = S->tuning_json;
  const size_t m = std::min(len - 1, t.size());
  std::memcpy(buf, t.data(), m);
  buf[m] = 0;
  return t.size() < len ? IPC_OK : IPC_EINVAL;
}

extern "C" int ipc_serve_tile_list(const uint32_t* col0, const uint32_t* ncols, uint32_t n_ranges,
                                   uint32_t tile_cols, uint32_t* tiles_out, uint32_t max_tiles) {
  if ((n_ranges && (!col0 || !ncols)) || tile_cols == 0 || (max_tiles && !tiles_out)) {
    set_error("ipc_serve_tile_list: bad argument");
    return IPC_EINVAL;
  }
  return static_cast<int>(tile_list(col0, ncols, n_ranges, tile_cols, tiles_out, max_tiles));
}

extern "C" int64_t ipc_serve_first_fit(const uint8_t* used, uint32_t n_slots, uint32_t want) {
  if (!used || want == 0) return -1;
  return first_fit(std::vector<uint8_t>(used, used + n_slots), want);
}
