// Internal state of a context, shared by context.cu (load, submit, fetch) and serve.cu (the
// continuous-batching request loop).
#pragma once

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace ipc {
const char* thread_last_error();

constexpr uint32_t kLog2BlockWords = 5;  // 1024-row OR blocks inside ipc_compare

struct Chunk {
  uint8_t* planes = nullptr;  // 6 * nlimb int8 planes [cap][l]: ((component * 2 + vec) * nlimb + limb)
  size_t cap = 0;
  size_t rows = 0;
  uint64_t row0 = 0;
};

// A request slot: every per-request buffer, allocated once for max_queries queries when the
// context takes its first request, and reused by later requests.
struct Slot {
  uint8_t* bq = nullptr;          // [party][vec][limb][n_pad_max][kq] query operand limbs
  uint8_t* qstage = nullptr;      // [vec][3][max_queries][l] query shares (u16, or u32 for Z_2^32 vectors)
  uint32_t* tags = nullptr;       // [N][2] column tags
  uint32_t* tags_host = nullptr;  // pinned [n_pad_max][2], the source of the tag copy
  uint32_t* roots = nullptr;      // [3][N][ld_roots] block roots of the OR tree
  size_t roots_words = 0;         // capacity of roots (grown only when the database has grown)
  uint8_t* shares_dev = nullptr;  // [3][Q]
  uint8_t* shares_host = nullptr; // pinned [3][Q]
  cudaEvent_t done = nullptr;     // recorded after the request's last copy
  bool busy = false;
};

struct Request {
  uint64_t id = 0;
  uint32_t Q = 0, N = 0, n_pad = 0;
  int slot = -1;
  size_t ld_roots = 0;
  uint8_t* zkeep = nullptr;       // [vec][party][N][rows] of zsz-byte dots, when distances are kept
  size_t zkeep_rows = 0;
};

struct Server;  // serve.cu

// Context helpers defined in context.cu.
int ctx_fail(ipc_ctx* c, int code, const std::string& msg);
int ctx_cfail(ipc_ctx* c, cudaError_t e, const char* what);
uint8_t* ctx_plane(const ipc_ctx* c, const Chunk& ch, int comp, int vec, int limb);
int ctx_check_device_status(ipc_ctx* c);
int stall_launch(const uint32_t* flag, uint32_t limit_us, cudaStream_t st);
int prep_query_rotate_plain(const uint16_t* y, uint32_t Q, const ipc_geom* g, uint16_t* b_lo, uint16_t* b_hi,
                            uint32_t n_pad, void* stream);
int compare_launch_tiles(const uint16_t* const z_code[3], const uint16_t* const z_mask[3], size_t ldz,
                         uint32_t n_cols, size_t n_rows, uint64_t row0, const uint32_t* col_tags,
                         const uint64_t seeds[3], uint32_t thr_a, uint32_t p, uint32_t* roots, size_t ld_roots,
                         uint8_t* msb_out, size_t ld_msb, const uint32_t* col_tiles, const uint32_t* n_col_list,
                         uint32_t tile_cols, cudaStream_t st, const uint32_t* col_rows, bool plain);
int prep_query_galois_strided(const uint16_t* y, uint64_t y_plane, uint32_t Q, const ipc_geom* g, uint32_t party,
                              uint16_t* b_lo, uint16_t* b_hi, uint32_t n_pad, void* stream);
int ring_gemm_tc32(uint32_t segments, const int8_t* const x[8], size_t x_rows, const uint16_t* const b[4],
                   uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                   uint64_t seed_prev, uint32_t vec, uint32_t* z, size_t ldz, uint64_t row0, cudaStream_t stream);
int prep_query32(const uint32_t* y, uint64_t y_plane, uint32_t Q, const ipc_geom* g, uint32_t party,
                 uint32_t segments, uint16_t* const b[4], uint32_t n_pad, cudaStream_t stream);
int compare_launch_liftfree(const uint16_t* const zc16[3], const uint32_t* const zc32[3],
                            const uint32_t* const ml32[3], size_t ldz, uint32_t n_cols, size_t n_rows, uint64_t row0,
                            const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a, uint32_t thr_b,
                            uint32_t p, uint32_t* roots, size_t ld_roots, uint8_t* msb_out, size_t ld_msb,
                            cudaStream_t st);
int ring_gemm_compare_tc(uint32_t segments, const int8_t* const x_lo[6], const int8_t* const x_hi[6], size_t x_rows,
                         const uint16_t* const b_lo[6], const uint16_t* const b_hi[6], uint32_t n_cols, uint32_t n_pad,
                         uint32_t l, const uint32_t* col_tags, const uint64_t seeds[3], uint32_t thr_a,
                         uint16_t* const z[6], size_t ldz, uint64_t row0, uint32_t* part_roots, size_t ld_parts,
                         cudaStream_t stream);
int or_join_parts_launch(const uint32_t* parts, size_t ld_parts, uint32_t n_cols, size_t n_rows, uint64_t row0,
                         const uint32_t* col_tags, const uint64_t seeds[3], uint32_t* roots, size_t ld_roots,
                         cudaStream_t st);
int ring_gemm_tc_variant(uint32_t tile_cols, uint32_t segments, const int8_t* const x_lo[2],
                         const int8_t* const x_hi[2], size_t x_rows, const uint16_t* b_lo, const uint16_t* b_hi,
                         uint32_t n_cols, uint32_t n_pad, uint32_t l, const uint32_t* col_tags, uint64_t seed_own,
                         uint64_t seed_prev, uint32_t vec, uint16_t* z, size_t ldz, uint64_t row0,
                         const uint32_t* col_tiles, const uint32_t* n_col_list, cudaStream_t stream);

// Serving hooks defined in serve.cu. serve_fetch_shares and serve_release return IPC_ENOTFOUND
// for ids that are not serving requests.
int serve_fetch_shares(ipc_ctx* c, uint64_t id, uint8_t* out, size_t n, int timeout_ms);
int serve_release(ipc_ctx* c, uint64_t id);
void serve_shutdown(ipc_ctx* c);
}  // namespace ipc

struct ipc_ctx {
  ipc_config cfg{};
  uint32_t l = 0;
  uint32_t qsz = 1;  // bytes per query-operand limb: int8, or its fp16 pattern for IPC_PATH_TC / IPC_PATH_TCG
  uint32_t kq = 0;   // K of the query operand: 2l (replicated sharing) or l (Galois-ring Shamir)
  uint32_t nlimb = 2;  // limb planes per component and vector: 4 when a vector lives in Z_2^32
  uint32_t zsz = 2;    // bytes per dot-product element in z buffers (4 with a lifting variant)
  cudaStream_t sp[3] = {nullptr, nullptr, nullptr};
  cudaStream_t sc = nullptr;
  cudaEvent_t ev_setup = nullptr, ev_gemm[3][2] = {}, ev_cmp[2] = {};
  cudaEvent_t ev_input = nullptr;        // recorded on input_stream before reading caller device buffers
  cudaStream_t input_stream = nullptr;   // stream whose earlier work produces device inputs (NULL = legacy)
  std::vector<ipc::Chunk> chunks;
  size_t rows = 0;
  uint8_t* zbuf = nullptr;  // [2 sets][vec][party][zbuf_cols][chunk_rows] of zsz-byte elements
  size_t zbuf_cols = 0;
  uint32_t* parts = nullptr;  // fused step: [3][parts_cols][chunk_rows / 128] part roots of one chunk
  size_t parts_cols = 0;
  uint8_t* stage = nullptr;  // load staging [chunk_rows][l] u16 (u32 with a lifting variant)
  std::map<uint64_t, ipc::Request> reqs;
  std::vector<ipc::Slot> slots;  // request slots, created by the first submit_queries
  uint32_t n_pad_max = 0;        // query columns of a slot: max_queries * R rounded up to 128
  uint64_t next_id = 1;
  std::mutex id_mu;            // next_id, when the serving loop runs
  ipc::Server* srv = nullptr;  // the serving loop, while one runs
  std::string err;
  // test aid: the next request's party stall_party first waits for a flag that nothing sets
  int stall_party = -1;
  uint32_t stall_us = 0;
  uint32_t* stall_flag = nullptr;
};
