// Internal declarations shared by the translation units of libdeco.
// Device helpers (counter-based RNG, bf16 packing), the graph handle and the
// kernel launchers.  Nothing here is part of the public ABI (include/deco.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "deco.h"

#include <nvtx3/nvToolsExt.h>

namespace deco {

// Runs f(t, r0, r1) on nt host threads over consecutive ranges [r0, r1) of
// [0, n) (thread 0 is the caller), nt chosen from `work` (about 2^18 units per
// thread, at most the host's cores).  Returns nt; f's ranges are in order of t.
template <class F>
int host_parallel(int64_t n, int64_t work, F&& f) {
  const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({hw, work / 262144 + 1, std::max<int64_t>(n, 1)}));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back([&f, t, n, nt] { f(t, n * t / nt, n * (t + 1) / nt); });
  f(0, (int64_t)0, n / nt);
  for (auto& th : pool) th.join();
  return nt;
}

// NVTX range on the calling host thread for the lifetime of the object (the
// enqueue of a solve, a phase, its steps and its rounding), so that a
// profiler can attribute the kernels of each part (ncu --nvtx); without a
// tool attached the calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char* what);   // records message, returns DECO_ERR_CUDA / OOM

#define DECO_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::deco::cuda_fail(_e, #expr); \
  } while (0)

// Weight storage of a graph.
enum WeightMode : int {
  W_UNIT = 0,     // all weights 1: no weight array
  W_SIGN = 1,     // weights in {-1,+1}: sign stored in bit 31 of the column index
  W_GENERAL = 2   // integral weights in a float array
};

}  // namespace deco

// Shared-memory CSR image of a row split of a graph for the on-chip kernel
// (built once per cluster size and kept with the graph).
struct SlabImage {
  int k = 0;
  uint32_t* data = nullptr;          // device, all parts back to back
  int32_t off[9] = {0};              // part i at data + 4 * off[i] (16-byte units)
  int32_t split[9] = {0};            // row split
  int32_t max_own = 0;
  int32_t max_words = 0;             // largest part in 32-bit words
};

// Per-warp record streams of the pipelined per-step kernel (step_stream.cu),
// built once per (slice height, entries per item, warp count, weights) and
// kept with the graph: rows sorted by degree in slices of ng rows, slice s
// given to warp s mod nw, each warp's items one contiguous run of rw-word
// records starting at record soff[warp].
struct StreamImage {
  int ng = 0, maxe = 0, nw = 0;
  bool gen = false;             // records carry general weights
  int32_t rw = 0;               // words per record
  int64_t records = 0;
  uint32_t* rec = nullptr;      // device records
  int32_t* soff = nullptr;      // device, nw + 1
};

// Launch shape of the pipelined per-step kernel.
struct StreamShape {
  int G = 16;          // lanes per row segment (32 / slice height)
  int maxe = 16;       // entries per item
  int stages = 3;      // shared-memory gather stages per warp
  int wpb = 8;         // warps per block
  int blocks = 0;      // grid: the blocks resident at once
  int nw = 0;          // blocks * wpb
  bool weighted = false, gen = false;
  int acc = 0;         // BF16 unit-weight sums: 0 widen + add, 1 mixed-precision add
  bool hints = false;  // records and new rows evict-first in L2
  int U = 1;           // 16-byte vectors per lane (2: the wide form)
  int fe = 0;          // entries per item fixed at compile time (8 or 12, two stages), or 0
};

// The opaque handle of the ABI.
struct deco_graph {
  int32_t n = 0;
  int64_t nnz = 0;
  int weighted = 0;             // caller supplied weights
  int wmode = deco::W_UNIT;     // storage used by the kernels
  int32_t max_abs_w = 1;        // largest |w|
  int device = 0;
  // host-side facts (degree statistics for IDI / DUI)
  int64_t deg_s1 = 0, deg_s2 = 0;
  int32_t max_deg = 0;
  std::vector<int32_t> h_row_ptr;   // host copy (row splits of the on-chip kernel)
  std::vector<int32_t> h_col;       // host copy of the device edge order
  std::vector<float> h_w;           // host copy of the device-order weights (or empty)
  std::vector<SlabImage> images;    // on-chip CSR images, one per cluster size used
  std::deque<StreamImage> streams;  // record streams of the pipelined step kernel, one per launch shape
                                    // (a deque: phase plans keep pointers to them while others are added)
  __nv_bfloat16* dense = nullptr;   // dense BF16 copy of A for the tensor-core kernel (built on first use)
  int32_t dense_ld = 0;             // its row stride, round_up(n, 128)
  struct Tuning {
    int32_t C, prec, kernel;
  };
  std::vector<Tuning> tuning;       // autotuned launch shapes (deco_autotune / deco_set_tuning)
  // device arrays
  int32_t* row_ptr = nullptr;   // n+1
  int32_t* col_idx = nullptr;   // nnz, plain indices
  uint32_t* col_sw = nullptr;   // nnz, index | sign bit (W_SIGN only)
  float* w = nullptr;           // nnz (W_GENERAL only)
  int32_t* wint = nullptr;      // nnz integer weights (weighted graphs; cut evaluation)
  float* dnet = nullptr;        // n, net weighted degree d_v = sum_u w_vu
  int32_t* deg = nullptr;       // n, |N(v)|
};

namespace deco {

// ------------------------------------------------------------- device helpers

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, key advanced by
// the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
    uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Uniform in (0,1): (2*(x>>9)+1) * 2^-24, exact in FP32.
__device__ __forceinline__ float u01(uint32_t x) {
  return (float)(2u * (x >> 9) + 1u) * 5.9604644775390625e-8f;
}

// Standard normal by the Box-Muller transform of two uniforms.
__device__ __forceinline__ float box_muller(uint32_t a, uint32_t b) {
  float r = sqrtf(-2.0f * logf(u01(a)));
  return r * cospif(2.0f * u01(b));
}

enum RngStream : uint32_t { STREAM_INIT = 0, STREAM_IDI = 1, STREAM_DUI = 2, STREAM_EVOLVE = 3, STREAM_ORDER = 6 };

// bf16 <-> fp32 packing of a 32-bit word holding two bf16 values (low half first).
__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------- launchers

struct StepLaunch {
  int32_t n, C, ld;
  int precision, objective, wmode;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const uint32_t* col_sw;
  const float* w;
  const float* dnet;
  const void* yin;
  void* yout;
  float* v;
  float alpha;          // step size (before the objective's factor)
  float mu;
  const float* alpha_cols;
  const int32_t* steps_cols;
  int32_t t;
  int32_t* flag;
};
int launch_step_global(const StepLaunch& s, cudaStream_t st);
// The pipelined form of the same step (bit-identical iterates): the shape
// for a block of C columns (stream_shape, which also sizes the grid), the
// graph's record streams for that shape (stream_image), one launch.
int stream_group_lanes(int32_t C, int prec, int U);
int stream_shape(int32_t C, int prec, int maxe, int stages, int wpb, bool weighted, bool gen, bool mixed,
                 bool hints, bool wide, StreamShape* out);
int stream_image(deco_graph* g, const StreamShape& sh, const StreamImage** out);
void free_stream_image(StreamImage& im);
int launch_step_stream(const StepLaunch& s, const StreamImage& im, const StreamShape& sh, cudaStream_t st);
// row-major n x ld (columns < C)  <->  S dense slabs of n x w (column c in slab c / w)
int launch_slab_layout(int32_t n, int32_t ld, int32_t C, int32_t w, int32_t S, size_t esz, const void* src,
                       void* dst, bool to_slabs, cudaStream_t st);

int launch_pack(const deco_graph* g, int32_t B, int32_t lift, int32_t ld, int precision,
                const void* y, uint32_t* zbits, cudaStream_t st);
int launch_cut_bits(const deco_graph* g, int32_t B, const uint32_t* zbits, int64_t* cuts,
                    cudaStream_t st);
int launch_cut_bytes(const deco_graph* g, int32_t B, const uint8_t* z, int64_t* cuts,
                     cudaStream_t st);
int launch_argmax(int32_t B, const int64_t* cuts, int32_t* best, cudaStream_t st);
// 1-flip local search on bit-packed columns (n x ceil(B/32) words), in place;
// gains: n x 32 ceil(B/32) int32 scratch, changed: max_rounds + 1 int32 scratch
int launch_local_search(const deco_graph* g, int32_t B, uint32_t* zbits, int32_t max_rounds, int32_t* gains,
                        int32_t* changed, cudaStream_t st);

// Phase bookkeeping of deco_solve: best of the phase, global best record.
struct BestRecord {
  long long cut;
  int32_t init;
  int32_t phase;
  int32_t improved;   // last phase improved the record
  int32_t pad;
};
// argmax of `cuts` into best_idx; the global record (first evaluation of a
// solve, or a strictly larger cut) and its vector best_z; the evaluation's
// best vector into phase_best_z (if not NULL)
int launch_phase_finish(const deco_graph* g, int32_t B, int32_t phase, bool first, const int64_t* cuts,
                        const uint32_t* zbits, int32_t* best_idx, BestRecord* rec,
                        uint8_t* phase_best_z, uint8_t* best_z, cudaStream_t st);

struct InitLaunch {
  int32_t n, B, lift, ld;
  int precision, objective, init;
  float eta, scale, uniform_half_width;
  uint32_t k0, k1;
  int32_t phase;
  const float* mean;          // n floats (Gaussian modes)
  const uint8_t* mean_bits;   // n bytes z* (mean = 2z-1) instead of `mean`
  const float* x0;            // explicit start (ld stride)
  void* y;
  const int32_t* gid;         // batch: graph of every row (null for one graph)
  const int32_t* goff;        // batch: first row of every graph
};

// Key and row index of the counter-based draws of row v of a batch: graph i
// draws with key (seed + i) and counts its own rows from 0.
__device__ __forceinline__ void batch_key(const int32_t* gid, const int32_t* goff, int32_t v, uint32_t& k0,
                                          uint32_t& k1, uint32_t& vr) {
  const int32_t g = gid[v];
  const uint64_t s = (((uint64_t)k1 << 32) | (uint64_t)k0) + (uint64_t)g;
  k0 = (uint32_t)s;
  k1 = (uint32_t)(s >> 32);
  vr = (uint32_t)(v - goff[g]);
}
int launch_init(const InitLaunch& p, cudaStream_t st);
int launch_idi(const deco_graph* g, double thresh, uint32_t k0, uint32_t k1, int32_t phase,
               float* h, int8_t* side_scratch, cudaStream_t st);
int launch_idi_batch(const deco_graph* g, double thresh, const double* gthresh, const int32_t* gid,
                     const int32_t* goff, uint32_t k0, uint32_t k1, int32_t phase, float* h,
                     int8_t* side_scratch, cudaStream_t st);
int launch_dui(const deco_graph* g, uint32_t k0, uint32_t k1, int32_t phase, float* h,
               cudaStream_t st);

double idi_threshold(const deco_graph* g, float beta);

int create_graph_impl(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                      const float* weights, uint32_t flags, bool device_order, deco_graph** out);

}  // namespace deco
