// A0 (client encoding and sharing), A1 (limb planes) and A2 (query preparation).
#include <cuda_fp16.h>

#include <string>

#include "common.cuh"

namespace ipc {
namespace {

// Balanced signed limbs: x = 256*hi + lo (mod 2^16), lo, hi in [-128, 127].
__device__ __forceinline__ void limbs(uint32_t x, int8_t& lo, int8_t& hi) {
  const int l = static_cast<int8_t>(x & 0xFFu);
  lo = static_cast<int8_t>(l);
  hi = static_cast<int8_t>(((x - static_cast<uint32_t>(l)) & 0xFFFFu) >> 8);
}

// A0 of protocol 1 (Sec. 4.3, Alg. 2): the client sends the mask in the clear, so the mask
// operand is the 0/1 element of each mask bit. One thread per (row, 8 consecutive bits), one
// 16-byte store.
__global__ void encode_plain_mask_kernel(const uint64_t* __restrict__ mask_bits, uint32_t n, uint32_t l,
                                         uint16_t* __restrict__ out) {
  const uint32_t groups = l >> 3;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (tid >= static_cast<uint64_t>(n) * groups) return;
  const uint32_t r = static_cast<uint32_t>(tid / groups), b0 = static_cast<uint32_t>(tid % groups) << 3;
  const uint32_t nw = (l + 63) >> 6;
  const uint32_t m = static_cast<uint32_t>(mask_bits[static_cast<uint64_t>(r) * nw + (b0 >> 6)] >> (b0 & 63)) & 0xFFu;
  uint32_t w[4];
#pragma unroll
  for (uint32_t e = 0; e < 4; ++e) w[e] = ((m >> (2 * e)) & 1u) | (((m >> (2 * e + 1)) & 1u) << 16);
  *reinterpret_cast<uint4*>(out + static_cast<uint64_t>(r) * l + b0) = make_uint4(w[0], w[1], w[2], w[3]);
}

// A0: one thread per (row, 4 consecutive elements); one Philox call per vector covers them.
__global__ void encode_share_kernel(const uint64_t* __restrict__ code_bits, const uint64_t* __restrict__ mask_bits,
                                    uint32_t n, uint32_t l, uint64_t seed, uint32_t side, uint32_t idx0,
                                    uint16_t* __restrict__ code_sh, uint16_t* __restrict__ mask_sh) {
  const uint32_t groups = l >> 2;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (tid >= static_cast<uint64_t>(n) * groups) return;
  const uint32_t r = static_cast<uint32_t>(tid / groups), t = static_cast<uint32_t>(tid % groups);
  const uint32_t nw = (l + 63) >> 6;
  const uint32_t b0 = t << 2;
  const uint32_t cw = static_cast<uint32_t>(code_bits[static_cast<uint64_t>(r) * nw + (b0 >> 6)] >> (b0 & 63)) & 0xFu;
  const uint32_t mw = static_cast<uint32_t>(mask_bits[static_cast<uint64_t>(r) * nw + (b0 >> 6)] >> (b0 & 63)) & 0xFu;
  const uint64_t plane = static_cast<uint64_t>(n) * l;
  const uint64_t at = static_cast<uint64_t>(r) * l + b0;
#pragma unroll
  for (uint32_t vec = 0; vec < 2; ++vec) {
    const uint4 w = philox(t, idx0 + r, (side << 8) | vec, IPC_D_SHARE << 24, seed);
    uint16_t x0[4], x1[4], x2[4];
#pragma unroll
    for (uint32_t e = 0; e < 4; ++e) {
      const uint32_t cb = (cw >> e) & 1u, mb = (mw >> e) & 1u;
      const uint32_t val = vec == 0 ? (mb - 2u * (cb & mb)) : mb;  // masked bit T=-1, U=0, F=+1 / mask bit
      const uint32_t word = word_of(w, e);
      x0[e] = static_cast<uint16_t>(word & 0xFFFFu);
      x1[e] = static_cast<uint16_t>(word >> 16);
      x2[e] = static_cast<uint16_t>(val - x0[e] - x1[e]);
    }
    uint16_t* dst = vec == 0 ? code_sh : mask_sh;
    *reinterpret_cast<uint2*>(dst + at) = make_uint2(x0[0] | (uint32_t(x0[1]) << 16), x0[2] | (uint32_t(x0[3]) << 16));
    *reinterpret_cast<uint2*>(dst + plane + at) =
        make_uint2(x1[0] | (uint32_t(x1[1]) << 16), x1[2] | (uint32_t(x1[3]) << 16));
    *reinterpret_cast<uint2*>(dst + 2 * plane + at) =
        make_uint2(x2[0] | (uint32_t(x2[1]) << 16), x2[2] | (uint32_t(x2[3]) << 16));
  }
}

// fp16 bit pattern of a limb (an integer in [-128, 127], exactly an fp16 value): the operand
// encoding of the tcgen05 paths' query side.
__device__ __forceinline__ uint16_t f16_of(int8_t v) { return __half_as_ushort(__short2half_rn(v)); }

// A1: 8 elements per thread.
__global__ void split_limbs_kernel(const uint16_t* __restrict__ x, size_t count, int8_t* __restrict__ lo,
                                   int8_t* __restrict__ hi) {
  const size_t i8 = (blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x) * 8;
  if (i8 >= count) return;
  if (i8 + 8 <= count) {
    const uint4 v = *reinterpret_cast<const uint4*>(x + i8);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t l2[2] = {0, 0}, h2[2] = {0, 0};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int8_t a, b;
      limbs((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu, a, b);
      l2[e >> 2] |= (uint32_t(uint8_t(a)) << (8 * (e & 3)));
      h2[e >> 2] |= (uint32_t(uint8_t(b)) << (8 * (e & 3)));
    }
    *reinterpret_cast<uint2*>(lo + i8) = make_uint2(l2[0], l2[1]);
    *reinterpret_cast<uint2*>(hi + i8) = make_uint2(h2[0], h2[1]);
  } else {
    for (size_t i = i8; i < count; ++i) limbs(x[i], lo[i], hi[i]);
  }
}

// A2: one thread per output element of B_i (row n, position k of 2l). Limb type T: int8_t, or
// uint16_t for the fp16 bit patterns of the same limbs.
template <typename T>
__global__ void prep_query_kernel(const uint16_t* __restrict__ y, uint64_t plane, uint32_t Q, ipc_geom g,
                                  uint32_t party, T* __restrict__ b_lo, T* __restrict__ b_hi, uint32_t n_pad) {
  const uint32_t l = g.rows * g.cols * g.cell;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const uint64_t total = static_cast<uint64_t>(n_pad) * 2 * l;
  if (tid >= total) return;
  const uint32_t n = static_cast<uint32_t>(tid / (2 * l));
  const uint32_t k = static_cast<uint32_t>(tid % (2 * l));
  uint32_t val = 0;
  if (n < Q * g.R) {
    const uint32_t q = n / g.R, rho = n % g.R;
    const int32_t shift = g.rot_lo + static_cast<int32_t>(rho);
    const uint32_t kk = k < l ? k : k - l;
    const uint32_t c = kk % g.cell, j = (kk / g.cell) % g.cols, r = kk / (g.cell * g.cols);
    int32_t js = (static_cast<int32_t>(j) - shift) % static_cast<int32_t>(g.cols);
    if (js < 0) js += g.cols;
    const uint32_t src = (r * g.cols + static_cast<uint32_t>(js)) * g.cell + c;
    const uint32_t prev = (party + 2) % 3;
    const uint32_t yi = y[party * plane + static_cast<uint64_t>(q) * l + src];
    if (k < l) {
      val = yi + y[prev * plane + static_cast<uint64_t>(q) * l + src];  // y_i + y_{i-1}
    } else {
      val = yi;  // y_i
    }
  }
  int8_t a, b;
  limbs(val & 0xFFFFu, a, b);
  if constexpr (sizeof(T) == 1) {
    b_lo[tid] = a;
    b_hi[tid] = b;
  } else {
    b_lo[tid] = f16_of(a);
    b_hi[tid] = f16_of(b);
  }
}

// A2 with eight consecutive elements of one row n of B_i per thread (l a multiple of 8, so a
// group never straddles a row or the two halves): one 16-byte store per limb plane for fp16
// limbs, 8 bytes for int8. The first element's (r, j, c) takes the divisions; the next ones
// step c, then the rotated column js (mod cols) and the row.
template <typename T>
__global__ void prep_query_vec_kernel(const uint16_t* __restrict__ y, uint64_t plane, uint32_t Q, ipc_geom g,
                                      uint32_t party, T* __restrict__ b_lo, T* __restrict__ b_hi, uint32_t n_pad) {
  const uint32_t l = g.rows * g.cols * g.cell;
  const uint32_t groups = (2 * l) / 8;  // per output row
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (tid >= static_cast<uint64_t>(n_pad) * groups) return;
  const uint32_t n = static_cast<uint32_t>(tid / groups);
  const uint32_t k0 = static_cast<uint32_t>(tid % groups) * 8;
  uint32_t val[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  if (n < Q * g.R) {
    const uint32_t q = n / g.R, rho = n % g.R;
    const int32_t shift = g.rot_lo + static_cast<int32_t>(rho);
    const bool sum = k0 < l;  // first half: y_i + y_{i-1}; second half: y_i
    const uint32_t kk = sum ? k0 : k0 - l;
    uint32_t c = kk % g.cell;
    const uint32_t cidx = kk / g.cell;
    uint32_t j = cidx % g.cols, r = cidx / g.cols;
    int32_t jsi = (static_cast<int32_t>(j) - shift) % static_cast<int32_t>(g.cols);
    uint32_t js = static_cast<uint32_t>(jsi < 0 ? jsi + static_cast<int32_t>(g.cols) : jsi);
    const uint32_t prev = (party + 2) % 3;
    const uint16_t* yi = y + party * plane + static_cast<uint64_t>(q) * l;
    const uint16_t* yp = y + prev * plane + static_cast<uint64_t>(q) * l;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint32_t src = (r * g.cols + js) * g.cell + c;
      val[e] = sum ? static_cast<uint32_t>(yi[src]) + yp[src] : yi[src];
      if (++c == g.cell) {
        c = 0;
        if (++js == g.cols) js = 0;
        if (++j == g.cols) {
          j = 0;
          ++r;
        }
      }
    }
  }
  int8_t a[8], b[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) limbs(val[e] & 0xFFFFu, a[e], b[e]);
  if constexpr (sizeof(T) == 1) {
    uint32_t l2[2] = {0u, 0u}, h2[2] = {0u, 0u};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      l2[e >> 2] |= static_cast<uint32_t>(static_cast<uint8_t>(a[e])) << (8 * (e & 3));
      h2[e >> 2] |= static_cast<uint32_t>(static_cast<uint8_t>(b[e])) << (8 * (e & 3));
    }
    *reinterpret_cast<uint2*>(b_lo + tid * 8) = make_uint2(l2[0], l2[1]);
    *reinterpret_cast<uint2*>(b_hi + tid * 8) = make_uint2(h2[0], h2[1]);
  } else {
    uint32_t l4[4], h4[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      l4[v] = f16_of(a[2 * v]) | (static_cast<uint32_t>(f16_of(a[2 * v + 1])) << 16);
      h4[v] = f16_of(b[2 * v]) | (static_cast<uint32_t>(f16_of(b[2 * v + 1])) << 16);
    }
    *reinterpret_cast<uint4*>(b_lo + tid * 8) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
    *reinterpret_cast<uint4*>(b_hi + tid * 8) = make_uint4(h4[0], h4[1], h4[2], h4[3]);
  }
}

// ---- Galois-ring Shamir sharing (Sec. 4.3.2): GR = Z_{2^16}[X]/(X^2 - X - 1) ----
// An element c0 + c1 X holds two consecutive code bits 2e, 2e+1; in a share vector its
// coefficients sit at indices 2e, 2e+1, so share vectors keep the bit layout (and a rotation
// of whole 4-bit cells moves whole elements).
struct Gr {
  uint32_t c0, c1;  // taken mod 2^16 where stored
};

// (a0 + a1 X)(b0 + b1 X) with X^2 = X + 1: the a1 b1 X^2 term adds to both coefficients.
__host__ __device__ __forceinline__ Gr gr_mul(Gr a, Gr b) {
  const uint32_t t = a.c1 * b.c1;
  return {(a.c0 * b.c0 + t) & 0xFFFFu, (a.c0 * b.c1 + a.c1 * b.c0 + t) & 0xFFFFu};
}

// Party p's evaluation point: 1, X, 1 + X (the non-zero elements of the exceptional set
// {0, 1, X, 1 + X}; the secret is the value at 0).
__host__ __device__ __forceinline__ Gr gr_point(uint32_t p) {
  return p == 0 ? Gr{1, 0} : (p == 1 ? Gr{0, 1} : Gr{1, 1});
}

// A0, Galois-ring Shamir: one thread per (row, 4 elements = 8 bits); one Philox call per
// vector gives the 4 elements' random slopes r (word e & 3: c0 low half, c1 high half); party
// p's share of element g is g + r * alpha_p.
__global__ void encode_share_galois_kernel(const uint64_t* __restrict__ code_bits,
                                           const uint64_t* __restrict__ mask_bits, uint32_t n, uint32_t l,
                                           uint64_t seed, uint32_t side, uint32_t idx0,
                                           uint16_t* __restrict__ code_sh, uint16_t* __restrict__ mask_sh) {
  const uint32_t groups = l >> 3;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (tid >= static_cast<uint64_t>(n) * groups) return;
  const uint32_t r = static_cast<uint32_t>(tid / groups), t = static_cast<uint32_t>(tid % groups);
  const uint32_t nw = (l + 63) >> 6;
  const uint32_t b0 = t << 3;  // first bit of the 4 elements
  const uint32_t cw = static_cast<uint32_t>(code_bits[static_cast<uint64_t>(r) * nw + (b0 >> 6)] >> (b0 & 63)) & 0xFFu;
  const uint32_t mw = static_cast<uint32_t>(mask_bits[static_cast<uint64_t>(r) * nw + (b0 >> 6)] >> (b0 & 63)) & 0xFFu;
  const uint64_t plane = static_cast<uint64_t>(n) * l;
  const uint64_t at = static_cast<uint64_t>(r) * l + b0;
#pragma unroll
  for (uint32_t vec = 0; vec < 2; ++vec) {
    const uint4 w = philox(t, idx0 + r, (side << 8) | vec, IPC_D_GSHARE << 24, seed);
    uint32_t out[3][4];  // [party][element]: c0 | c1 << 16
#pragma unroll
    for (uint32_t e = 0; e < 4; ++e) {
      uint32_t v[2];
#pragma unroll
      for (uint32_t k = 0; k < 2; ++k) {
        const uint32_t cb = (cw >> (2 * e + k)) & 1u, mb = (mw >> (2 * e + k)) & 1u;
        v[k] = vec == 0 ? (mb - 2u * (cb & mb)) : mb;
      }
      const uint32_t word = word_of(w, e);
      const Gr slope = {word & 0xFFFFu, word >> 16};
#pragma unroll
      for (uint32_t p = 0; p < 3; ++p) {
        const Gr ra = gr_mul(slope, gr_point(p));
        out[p][e] = ((v[0] + ra.c0) & 0xFFFFu) | (((v[1] + ra.c1) & 0xFFFFu) << 16);
      }
    }
    uint16_t* dst = vec == 0 ? code_sh : mask_sh;
#pragma unroll
    for (uint32_t p = 0; p < 3; ++p)
      *reinterpret_cast<uint4*>(dst + p * plane + at) = make_uint4(out[p][0], out[p][1], out[p][2], out[p][3]);
  }
}

// A2 for Galois-ring shares: B_p[n][k] = coefficient k & 1 of lambda_p * y_p[e'] where e' is the
// element of the unrotated query that rotation rho brings to position k / 2. K = l. Eight
// consecutive k (four elements) of one row n per thread, one 16-byte store per limb plane; the
// cell size is even, so an element's two coefficients stay in one cell and move together.
__global__ void prep_query_galois_kernel(const uint16_t* __restrict__ y, uint64_t plane, uint32_t Q, ipc_geom g,
                                         uint32_t party, Gr lambda, uint16_t* __restrict__ b_lo,
                                         uint16_t* __restrict__ b_hi, uint32_t n_pad) {
  const uint32_t l = g.rows * g.cols * g.cell;
  const uint32_t groups = l / 8;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (tid >= static_cast<uint64_t>(n_pad) * groups) return;
  const uint32_t n = static_cast<uint32_t>(tid / groups);
  const uint32_t k0 = static_cast<uint32_t>(tid % groups) * 8;
  uint32_t val[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  if (n < Q * g.R) {
    const uint32_t q = n / g.R, rho = n % g.R;
    const int32_t shift = g.rot_lo + static_cast<int32_t>(rho);
    uint32_t c = k0 % g.cell;
    const uint32_t cidx = k0 / g.cell;
    uint32_t j = cidx % g.cols, r = cidx / g.cols;
    int32_t jsi = (static_cast<int32_t>(j) - shift) % static_cast<int32_t>(g.cols);
    uint32_t js = static_cast<uint32_t>(jsi < 0 ? jsi + static_cast<int32_t>(g.cols) : jsi);
    const uint16_t* yq = y + party * plane + static_cast<uint64_t>(q) * l;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t src = (r * g.cols + js) * g.cell + c;  // even: c is even
      const Gr a = gr_mul(lambda, Gr{yq[src], yq[src + 1]});
      val[2 * e] = a.c0;
      val[2 * e + 1] = a.c1;
      c += 2;
      if (c == g.cell) {
        c = 0;
        if (++js == g.cols) js = 0;
        if (++j == g.cols) {
          j = 0;
          ++r;
        }
      }
    }
  }
  uint32_t l4[4], h4[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    int8_t a0, b0, a1, b1;
    limbs(val[2 * v] & 0xFFFFu, a0, b0);
    limbs(val[2 * v + 1] & 0xFFFFu, a1, b1);
    l4[v] = f16_of(a0) | (static_cast<uint32_t>(f16_of(a1)) << 16);
    h4[v] = f16_of(b0) | (static_cast<uint32_t>(f16_of(b1)) << 16);
  }
  *reinterpret_cast<uint4*>(b_lo + tid * 8) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
  *reinterpret_cast<uint4*>(b_hi + tid * 8) = make_uint4(h4[0], h4[1], h4[2], h4[3]);
}

bool geom_ok(const ipc_geom* g) {
  if (!g || g->rows == 0 || g->cols == 0 || g->cell == 0 || g->R == 0 || g->R > 31) return false;
  const uint64_t l = static_cast<uint64_t>(g->rows) * g->cols * g->cell;
  return l > 0 && l % 128 == 0 && l <= (1u << 14);  // l < 2^14 keeps b*l < 2^32/4 (Lemma 2 with b = 2^16)
}

}  // namespace
}  // namespace ipc

using namespace ipc;

extern "C" int ipc_encode_share(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                                uint64_t client_seed, uint32_t side, uint32_t idx0, uint16_t* code_sh,
                                uint16_t* mask_sh, void* stream) {
  if (l == 0 || l % 4 != 0 || !code_bits || !mask_bits || !code_sh || !mask_sh) {
    set_error("ipc_encode_share: l must be a positive multiple of 4 and pointers non-null");
    return IPC_EINVAL;
  }
  if (n == 0) return IPC_OK;
  const uint64_t threads = static_cast<uint64_t>(n) * (l / 4);
  const uint32_t bs = 256;
  encode_share_kernel<<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
      code_bits, mask_bits, n, l, client_seed, side, idx0, code_sh, mask_sh);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

extern "C" int ipc_encode_plain_mask(const uint64_t* mask_bits, uint32_t n, uint32_t l, uint16_t* mask_out,
                                     void* stream) {
  if (l == 0 || l % 8 != 0 || !mask_bits || !mask_out || (reinterpret_cast<uintptr_t>(mask_out) & 15)) {
    set_error("ipc_encode_plain_mask: l must be a positive multiple of 8, pointers non-null, mask_out 16-byte aligned");
    return IPC_EINVAL;
  }
  if (n == 0) return IPC_OK;
  const uint64_t threads = static_cast<uint64_t>(n) * (l / 8);
  const uint32_t bs = 256;
  encode_plain_mask_kernel<<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
      mask_bits, n, l, mask_out);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

extern "C" int ipc_split_limbs(const uint16_t* x, size_t count, int8_t* lo, int8_t* hi, void* stream) {
  if (count == 0 || !x || !lo || !hi || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(lo) & 7) ||
      (reinterpret_cast<uintptr_t>(hi) & 7)) {
    set_error("ipc_split_limbs: count > 0, x 16-byte and lo/hi 8-byte aligned");
    return IPC_EINVAL;
  }
  const size_t threads = (count + 7) / 8;
  const uint32_t bs = 256;
  split_limbs_kernel<<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(x, count, lo, hi);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

namespace ipc {
// y_plane: elements between the three components of y (Q * l when they are packed).
template <typename T>
int prep_query_strided(const uint16_t* y, uint64_t y_plane, uint32_t Q, const ipc_geom* g, uint32_t party, T* b_lo,
                       T* b_hi, uint32_t n_pad, void* stream, const char* who) {
  if (!geom_ok(g) || party > 2 || !y || !b_lo || !b_hi || Q == 0 || static_cast<uint64_t>(Q) * g->R > n_pad) {
    set_error(std::string(who) + ": invalid geometry, party, or n_pad < Q*R");
    return IPC_EINVAL;
  }
  const uint64_t l = static_cast<uint64_t>(g->rows) * g->cols * g->cell;
  const uint64_t total = static_cast<uint64_t>(n_pad) * 2 * l;
  const uint32_t bs = 256;
  if (y_plane < static_cast<uint64_t>(Q) * l) {
    set_error(std::string(who) + ": component stride shorter than Q * l");
    return IPC_EINVAL;
  }
  const uintptr_t align = 8 * sizeof(T) - 1;  // one group's store: 16 bytes (fp16) or 8 (int8)
  if (l % 8 == 0 && !(reinterpret_cast<uintptr_t>(b_lo) & align) && !(reinterpret_cast<uintptr_t>(b_hi) & align)) {
    const uint64_t threads = total / 8;
    prep_query_vec_kernel<T><<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
        y, y_plane, Q, *g, party, b_lo, b_hi, n_pad);
  } else {
    prep_query_kernel<T><<<static_cast<unsigned>((total + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
        y, y_plane, Q, *g, party, b_lo, b_hi, n_pad);
  }
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}
template int prep_query_strided<int8_t>(const uint16_t*, uint64_t, uint32_t, const ipc_geom*, uint32_t, int8_t*,
                                        int8_t*, uint32_t, void*, const char*);
template int prep_query_strided<uint16_t>(const uint16_t*, uint64_t, uint32_t, const ipc_geom*, uint32_t, uint16_t*,
                                          uint16_t*, uint32_t, void*, const char*);
}  // namespace ipc

extern "C" int ipc_prep_query(const uint16_t* y, uint32_t Q, const ipc_geom* g, uint32_t party, int8_t* b_lo,
                              int8_t* b_hi, uint32_t n_pad, void* stream) {
  const uint64_t l = g ? static_cast<uint64_t>(g->rows) * g->cols * g->cell : 0;
  return prep_query_strided(y, Q * l, Q, g, party, b_lo, b_hi, n_pad, stream, "ipc_prep_query");
}

extern "C" int ipc_prep_query_f16(const uint16_t* y, uint32_t Q, const ipc_geom* g, uint32_t party, uint16_t* b_lo,
                                  uint16_t* b_hi, uint32_t n_pad, void* stream) {
  const uint64_t l = g ? static_cast<uint64_t>(g->rows) * g->cols * g->cell : 0;
  return prep_query_strided(y, Q * l, Q, g, party, b_lo, b_hi, n_pad, stream, "ipc_prep_query_f16");
}

namespace {
// Host-side GR arithmetic for the Lagrange coefficients (the library's own, computed once).
struct HGr {
  uint16_t c0, c1;
};
HGr hmul(HGr a, HGr b) {
  const uint32_t t = static_cast<uint32_t>(a.c1) * b.c1;
  return {static_cast<uint16_t>(static_cast<uint32_t>(a.c0) * b.c0 + t),
          static_cast<uint16_t>(static_cast<uint32_t>(a.c0) * b.c1 + static_cast<uint32_t>(a.c1) * b.c0 + t)};
}
// a^-1 = conj(a) / N(a) with conj(X) = 1 - X and N(a) = a conj(a) in Z_{2^16}, inverted by
// Hensel lifting (each step x <- x (2 - N x) doubles the correct low bits; x = N is right mod 8).
bool hinv(HGr a, HGr* out) {
  const HGr conj = {static_cast<uint16_t>(a.c0 + a.c1), static_cast<uint16_t>(-a.c1)};
  const HGr nrm = hmul(a, conj);
  if (nrm.c1 != 0 || (nrm.c0 & 1u) == 0) return false;
  uint32_t x = nrm.c0;
  for (int i = 0; i < 4; ++i) x = x * (2u - nrm.c0 * x);
  *out = hmul(conj, HGr{static_cast<uint16_t>(x), 0});
  return true;
}
// lambda_p = prod_{j != p} alpha_j (alpha_j - alpha_p)^-1
Gr lagrange_at_zero(uint32_t p) {
  const HGr alpha[3] = {{1, 0}, {0, 1}, {1, 1}};
  HGr acc = {1, 0};
  for (uint32_t j = 0; j < 3; ++j) {
    if (j == p) continue;
    HGr inv;
    const HGr d = {static_cast<uint16_t>(alpha[j].c0 - alpha[p].c0), static_cast<uint16_t>(alpha[j].c1 - alpha[p].c1)};
    if (!hinv(d, &inv)) return {0, 0};  // unreachable: the points' differences are units
    acc = hmul(acc, hmul(alpha[j], inv));
  }
  return {acc.c0, acc.c1};
}
}  // namespace

extern "C" int ipc_encode_share_galois(const uint64_t* code_bits, const uint64_t* mask_bits, uint32_t n, uint32_t l,
                                       uint64_t client_seed, uint32_t side, uint32_t idx0, uint16_t* code_sh,
                                       uint16_t* mask_sh, void* stream) {
  if (l == 0 || l % 8 != 0 || !code_bits || !mask_bits || !code_sh || !mask_sh ||
      (reinterpret_cast<uintptr_t>(code_sh) & 15) || (reinterpret_cast<uintptr_t>(mask_sh) & 15)) {
    set_error("ipc_encode_share_galois: l must be a positive multiple of 8, outputs 16-byte aligned");
    return IPC_EINVAL;
  }
  if (n == 0) return IPC_OK;
  const uint64_t threads = static_cast<uint64_t>(n) * (l / 8);
  const uint32_t bs = 256;
  encode_share_galois_kernel<<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
      code_bits, mask_bits, n, l, client_seed, side, idx0, code_sh, mask_sh);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

namespace ipc {
int prep_query_galois_strided(const uint16_t* y, uint64_t y_plane, uint32_t Q, const ipc_geom* g, uint32_t party,
                              uint16_t* b_lo, uint16_t* b_hi, uint32_t n_pad, void* stream) {
  if (!geom_ok(g) || g->cell % 2 != 0 || party > 2 || !y || !b_lo || !b_hi || Q == 0 ||
      static_cast<uint64_t>(Q) * g->R > n_pad) {
    set_error("ipc_prep_query_galois: invalid geometry (even cell), party, or n_pad < Q*R");
    return IPC_EINVAL;
  }
  const uint64_t l = static_cast<uint64_t>(g->rows) * g->cols * g->cell;
  if (y_plane < static_cast<uint64_t>(Q) * l) {
    set_error("ipc_prep_query_galois: component stride shorter than Q * l");
    return IPC_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(b_lo) & 15) || (reinterpret_cast<uintptr_t>(b_hi) & 15)) {
    set_error("ipc_prep_query_galois: b_lo and b_hi must be 16-byte aligned");
    return IPC_EINVAL;
  }
  const uint64_t threads = static_cast<uint64_t>(n_pad) * (l / 8);
  const uint32_t bs = 256;
  prep_query_galois_kernel<<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
      y, y_plane, Q, *g, party, lagrange_at_zero(party), b_lo, b_hi, n_pad);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}
// Public operand of protocol 1: B[n][k] = fp16 limbs of rot_rho(y[q])[k] for 0/1 values y [Q][l]
// (the plain mask bits; K = l): the Galois preparation with lambda = 1 reads each element
// unchanged.
int prep_query_rotate_plain(const uint16_t* y, uint32_t Q, const ipc_geom* g, uint16_t* b_lo, uint16_t* b_hi,
                            uint32_t n_pad, void* stream) {
  if (!geom_ok(g) || g->cell % 2 != 0 || !y || !b_lo || !b_hi || Q == 0 || static_cast<uint64_t>(Q) * g->R > n_pad ||
      (reinterpret_cast<uintptr_t>(b_lo) & 15) || (reinterpret_cast<uintptr_t>(b_hi) & 15)) {
    set_error("plain-mask operand: invalid geometry (even cell), n_pad < Q*R or unaligned outputs");
    return IPC_EINVAL;
  }
  const uint64_t l = static_cast<uint64_t>(g->rows) * g->cols * g->cell;
  const uint64_t threads = static_cast<uint64_t>(n_pad) * (l / 8);
  const uint32_t bs = 256;
  prep_query_galois_kernel<<<static_cast<unsigned>((threads + bs - 1) / bs), bs, 0, as_stream(stream)>>>(
      y, static_cast<uint64_t>(Q) * l, Q, *g, 0, Gr{1, 0}, b_lo, b_hi, n_pad);
  IPC_CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}
}  // namespace ipc

extern "C" int ipc_prep_query_galois(const uint16_t* y, uint32_t Q, const ipc_geom* g, uint32_t party,
                                     uint16_t* b_lo, uint16_t* b_hi, uint32_t n_pad, void* stream) {
  const uint64_t l = g ? static_cast<uint64_t>(g->rows) * g->cols * g->cell : 0;
  return prep_query_galois_strided(y, Q * l, Q, g, party, b_lo, b_hi, n_pad, stream);
}
