// Combinatorial companions of the solver on the same device graph:
//
//  * the greedy MaxCut comparator (App. C.1): a run fixes a vertex ordering,
//    puts the first vertex in S and every later one on the side that cuts
//    more edges to the vertices already placed (ties: S).  Run b uses the
//    random ordering pi_b of [0, n): a balanced 4-round Feistel network on
//    [0, 4^h) whose round function is word 0 of Philox counter
//    (R, b, round, STREAM_ORDER), with cycle walking onto [0, n).  One warp
//    per run; the runs are independent.
//
//  * 1-flip local search on rounded vectors (bit-packed, n x ceil(B/32)
//    words): every round computes the cut change of flipping each node alone,
//    gain_v = sum_u w_vu s_u s_v (s = +-1 side), and flips every node whose
//    gain is positive and larger than the gain of each neighbour with a
//    positive gain (equal gains: the lower index wins).  Those nodes are
//    pairwise non-adjacent, so the cut grows by the sum of their gains; the
//    search ends at a 1-flip local optimum or after max_rounds rounds.  A
//    device flag per round lets the remaining rounds return at once.
#include <algorithm>

#include "api_util.cuh"
#include "deco_internal.cuh"

namespace deco {
namespace {

struct Feistel {
  int h;            // bits per half
  uint32_t mask;    // 2^h - 1
  uint32_t n;
  uint32_t k0, k1;

  __device__ __forceinline__ uint32_t net(uint32_t x, uint32_t b) const {
    uint32_t L = x >> h, R = x & mask;
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
      const uint4 f = philox4x32_10(make_uint4(R, b, i, STREAM_ORDER), k0, k1);
      const uint32_t t = R;
      R = L ^ (f.x & mask);
      L = t;
    }
    return (L << h) | R;
  }
  // pi_b(k): walk the network until the value falls in [0, n); a cycle of the
  // bijection on [0, 4^h) holds at most 4^h values, so the walk ends
  __device__ __forceinline__ uint32_t at(uint32_t k, uint32_t b) const {
    uint32_t x = net(k, b);
    const uint64_t cap = 1ull << (2 * h);
    for (uint64_t it = 0; x >= n && it < cap; ++it) x = net(x, b);
    return x;
  }
};

__global__ void k_orders(Feistel F, int32_t B, int32_t* order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)F.n * B) return;
  const uint32_t b = (uint32_t)(i / F.n), k = (uint32_t)(i % F.n);
  order[i] = (int32_t)F.at(k, b);
}

// z (n x B bytes) starts at 2 (not placed); warp b places run b's vertices in order
__global__ void k_greedy(int32_t n, int32_t B, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* wint,
                         const int32_t* order, uint8_t* z) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= B) return;
  const int32_t b = (int32_t)wid;
  for (int32_t k = 0; k < n; ++k) {
    const int32_t v = order[(size_t)b * n + k];
    long long g1 = 0, g0 = 0;   // cut gained by placing v in S (side 1) / in S-bar (side 0)
    for (int32_t e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) {
      const uint8_t s = z[(size_t)col_idx[e] * B + b];
      const long long w = wint ? wint[e] : 1;
      if (s == 0) g1 += w;
      else if (s == 1) g0 += w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      g1 += __shfl_xor_sync(0xFFFFFFFFu, g1, o);
      g0 += __shfl_xor_sync(0xFFFFFFFFu, g0, o);
    }
    if (lane == 0) z[(size_t)v * B + b] = g1 >= g0 ? 1 : 0;
    __syncwarp();   // the next vertices read this side
  }
}

// bytes (n x B) <-> bits (n x W words, bit b % 32 of word b / 32)
__global__ void k_bytes_to_bits(int32_t n, int32_t B, int32_t W, const uint8_t* z, uint32_t* bits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * W) return;
  const int32_t v = (int32_t)(i / W), k = (int32_t)(i % W);
  uint32_t w = 0;
  for (int c = 0; c < 32 && 32 * k + c < B; ++c) w |= (z[(size_t)v * B + 32 * k + c] ? 1u : 0u) << c;
  bits[i] = w;
}
__global__ void k_bits_to_bytes(int32_t n, int32_t B, int32_t W, const uint32_t* bits, uint8_t* z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * B) return;
  const int32_t v = (int32_t)(i / B), b = (int32_t)(i % B);
  z[i] = (uint8_t)((bits[(size_t)v * W + b / 32] >> (b % 32)) & 1u);
}

// gains[v][32k + c] = sum_u w_vu (+1 same side, -1 other side) for column 32k + c
__global__ void k_ls_gain(int32_t n, int32_t W, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* wint,
                          const uint32_t* zb, int32_t* gains, const int32_t* run) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * W || !*run) return;
  const int32_t v = (int32_t)(i / W), k = (int32_t)(i % W);
  const uint32_t zv = zb[i];
  int32_t acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0;
  for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
    const int32_t u = col_idx[e];
    const int32_t w = wint ? wint[e] : 1;
    const uint32_t x = zb[(size_t)u * W + k] ^ zv;
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] += ((x >> c) & 1u) ? -w : w;
  }
  int32_t* out = gains + (size_t)v * 32 * W + 32 * k;
#pragma unroll
  for (int c = 0; c < 32; ++c) out[c] = acc[c];
}

__global__ void k_ls_flip(int32_t n, int32_t W, int32_t B, const int32_t* row_ptr, const int32_t* col_idx,
                          const int32_t* gains, uint32_t* zb, const int32_t* run, int32_t* next) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * W || !*run) return;
  const int32_t v = (int32_t)(i / W), k = (int32_t)(i % W);
  const int32_t* gv = gains + (size_t)v * 32 * W + 32 * k;
  int32_t g[32];
  uint32_t pos = 0;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    g[c] = gv[c];
    if (g[c] > 0 && 32 * k + c < B) pos |= 1u << c;
  }
  if (!pos) return;
  uint32_t beaten = 0;
  for (int32_t e = row_ptr[v]; e < row_ptr[v + 1] && (pos & ~beaten); ++e) {
    const int32_t u = col_idx[e];
    const int32_t* gu = gains + (size_t)u * 32 * W + 32 * k;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const int32_t x = gu[c];
      if (((pos >> c) & 1u) && x > 0 && (x > g[c] || (x == g[c] && u < v))) beaten |= 1u << c;
    }
  }
  const uint32_t flip = pos & ~beaten;
  if (flip) {
    zb[i] ^= flip;
    *next = 1;
  }
}

unsigned blocks_for(int64_t threads, int per) { return (unsigned)((threads + per - 1) / per); }

}  // namespace

// The rounds of the local search on bit-packed columns (stream-ordered).
// gains: n x 32W int32 scratch; changed: max_rounds + 1 int32 scratch.
int launch_local_search(const deco_graph* g, int32_t B, uint32_t* zbits, int32_t max_rounds, int32_t* gains,
                        int32_t* changed, cudaStream_t st) {
  const int32_t W = (B + 31) / 32;
  if (max_rounds <= 0 || g->n == 0) return DECO_OK;
  DECO_CUDA_TRY(cudaMemsetAsync(changed, 0, sizeof(int32_t) * (size_t)(max_rounds + 1), st));
  DECO_CUDA_TRY(cudaMemsetAsync(changed, 1, sizeof(int32_t), st));   // round 0 runs (any nonzero word)
  const int64_t threads = (int64_t)g->n * W;
  for (int32_t r = 0; r < max_rounds; ++r) {
    k_ls_gain<<<blocks_for(threads, 128), 128, 0, st>>>(g->n, W, g->row_ptr, g->col_idx, g->wint, zbits, gains,
                                                        changed + r);
    k_ls_flip<<<blocks_for(threads, 128), 128, 0, st>>>(g->n, W, B, g->row_ptr, g->col_idx, gains, zbits,
                                                        changed + r, changed + r + 1);
  }
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

}  // namespace deco

using namespace deco;

extern "C" int deco_greedy(const deco_graph* g, int32_t B, uint64_t seed, uint8_t* z, int64_t* cuts, void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (B < 1 || !z || !cuts) { set_error("need B >= 1 and device z, cuts"); return DECO_ERR_ARG; }
  if (g->n >= (1 << 30)) { set_error("n too large for the greedy orderings"); return DECO_ERR_UNSUPPORTED; }
  cudaStream_t st = as_stream(stream);
  Scratch s(st);
  int32_t* order = nullptr;
  if ((rc = s.alloc(&order, sizeof(int32_t) * (size_t)g->n * B))) return rc;
  Feistel F{};
  F.h = 1;
  while ((1ull << (2 * F.h)) < (uint64_t)g->n) ++F.h;
  F.mask = (uint32_t)((1ull << F.h) - 1);
  F.n = (uint32_t)g->n;
  F.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  F.k1 = (uint32_t)(seed >> 32);
  if (g->n > 0) {
    k_orders<<<blocks_for((int64_t)g->n * B, 256), 256, 0, st>>>(F, B, order);
    DECO_CUDA_TRY(cudaMemsetAsync(z, 2, (size_t)g->n * B, st));
    k_greedy<<<blocks_for((int64_t)B * 32, 128), 128, 0, st>>>(g->n, B, g->row_ptr, g->col_idx, g->wint, order, z);
    DECO_CUDA_TRY(cudaGetLastError());
  }
  return launch_cut_bytes(g, B, z, cuts, st);
}

extern "C" int deco_local_search(const deco_graph* g, int32_t B, uint8_t* z, int32_t max_rounds, int64_t* cuts,
                                 int32_t* rounds, void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (B < 1 || !z || max_rounds < 0) { set_error("need B >= 1, device z and max_rounds >= 0"); return DECO_ERR_ARG; }
  cudaStream_t st = as_stream(stream);
  const int32_t W = (B + 31) / 32;
  Scratch s(st);
  uint32_t* bits = nullptr;
  int32_t* gains = nullptr;
  int32_t* changed = nullptr;
  if ((rc = s.alloc(&bits, sizeof(uint32_t) * (size_t)g->n * W)) ||
      (rc = s.alloc(&gains, sizeof(int32_t) * (size_t)g->n * 32 * W)) ||
      (rc = s.alloc(&changed, sizeof(int32_t) * (size_t)(max_rounds + 1))))
    return rc;
  if (g->n > 0) {
    k_bytes_to_bits<<<blocks_for((int64_t)g->n * W, 256), 256, 0, st>>>(g->n, B, W, z, bits);
    if ((rc = launch_local_search(g, B, bits, max_rounds, gains, changed, st))) return rc;
    k_bits_to_bytes<<<blocks_for((int64_t)g->n * B, 256), 256, 0, st>>>(g->n, B, W, bits, z);
    DECO_CUDA_TRY(cudaGetLastError());
  }
  if (cuts && (rc = launch_cut_bytes(g, B, z, cuts, st))) return rc;
  if (rounds) {
    std::vector<int32_t> h((size_t)max_rounds + 1, 0);
    DECO_CUDA_TRY(cudaMemcpyAsync(h.data(), changed, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaStreamSynchronize(st));
    int32_t c = 0;
    for (int32_t r = 1; r <= max_rounds; ++r) c += h[r] ? 1 : 0;
    *rounds = g->n > 0 ? c : 0;
  }
  return DECO_OK;
}
