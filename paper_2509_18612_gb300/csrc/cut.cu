// Rounding, integer cut evaluation and argmax over starting points
// (the rounding and selection steps of Alg. 1 / Alg. 2; Eq. 5, Eq. 11, Eq. 1).
//
//  pack:   one warp per (row, 32 starting points); lane b forms z_{v,b} from
//          the iterate and __ballot_sync packs the 32 bits into one word.
//  cut:    one warp per (row block, word); lane b accumulates
//          w_uv * ((z_v xor z_u) >> b & 1) over the neighbours u > v of its
//          rows (each unordered edge once), in integers; the block reduces and
//          issues one 64-bit atomic per starting point.  Integer atomics are
//          associative, so the result is exact and run-to-run identical.
//  argmax: one block; lowest index among the maximal cuts.
#include "deco_internal.cuh"

namespace deco {
namespace {

template <int PREC>
__device__ __forceinline__ float load_y(const void* y, size_t i) {
  if (PREC == DECO_PREC_FP32) return __ldg(static_cast<const float*>(y) + i);
  return __bfloat162float(static_cast<const __nv_bfloat16*>(y)[i]);
}

template <int PREC>
__global__ void k_pack(int32_t n, int32_t B, int32_t lift, int32_t ld, int32_t W, const void* y,
                       uint32_t* zbits) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= (int64_t)n * W) return;
  const int32_t v = (int32_t)(warp / W);
  const int32_t k = (int32_t)(warp % W);
  const int32_t b = k * 32 + lane;
  bool bit = false;
  if (b < B) {
    const size_t base = (size_t)v * ld + (size_t)b * lift;
    if (lift == 1) {
      bit = load_y<PREC>(y, base) > 0.0f;               // Eq. 5: strict
    } else {
      float s = 0.0f;
      for (int i = 0; i < lift; ++i) s += load_y<PREC>(y, base + i);
      bit = s >= 0.0f;                                   // Eq. 11: non-strict
    }
  }
  const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
  if (lane == 0) zbits[(size_t)v * W + k] = word;
}

constexpr int CUT_BLOCK = 256;

// zb(v, k): word k of row v, either from packed bits or from a byte matrix.
struct BitsSrc {
  const uint32_t* zbits;  // n x W
  int32_t W;
  __device__ __forceinline__ uint32_t word(int32_t v, int32_t k) const {
    return __ldg(zbits + (size_t)v * W + k);
  }
};
struct BytesSrc {
  const uint8_t* z;  // n x B
  int32_t B;
  __device__ __forceinline__ uint32_t word(int32_t v, int32_t k) const {
    // lane-independent word assembled from 32 bytes (used only by deco_eval_cuts)
    uint32_t w = 0;
    const int32_t b0 = k * 32;
    for (int i = 0; i < 32 && b0 + i < B; ++i) w |= (z[(size_t)v * B + b0 + i] ? 1u : 0u) << i;
    return w;
  }
};

template <typename Src>
__global__ void __launch_bounds__(CUT_BLOCK) k_cut(int32_t n, int32_t B, int32_t W,
                                                   const int32_t* row_ptr, const int32_t* col_idx,
                                                   const int32_t* wint, Src src, int64_t* cuts) {
  __shared__ long long part[CUT_BLOCK / 32][32];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int32_t k = blockIdx.y;                      // word (32 starting points)
  const int64_t warps_total = (int64_t)gridDim.x * (CUT_BLOCK / 32);
  long long acc = 0;
  for (int64_t v64 = (int64_t)blockIdx.x * (CUT_BLOCK / 32) + wib; v64 < n; v64 += warps_total) {
    const int32_t v = (int32_t)v64;
    const uint32_t zv = src.word(v, k);
    const int32_t e0 = __ldg(row_ptr + v), e1 = __ldg(row_ptr + v + 1);
    int32_t racc = 0;   // |sum| <= sum |w| over the row <= 2^24 (checked at creation)
    // neighbours are sorted: skip u < v, keep u > v (each unordered edge once)
    for (int32_t e = e0; e < e1; ++e) {
      const int32_t u = __ldg(col_idx + e);
      if (u <= v) continue;
      const uint32_t x = (zv ^ src.word(u, k)) >> lane & 1u;
      racc += wint ? (int32_t)x * __ldg(wint + e) : (int32_t)x;
    }
    acc += racc;
  }
  part[wib][lane] = acc;
  __syncthreads();
  if (wib == 0) {
    long long s = 0;
    for (int i = 0; i < CUT_BLOCK / 32; ++i) s += part[i][lane];
    const int32_t b = k * 32 + lane;
    if (b < B && s != 0) atomicAdd(reinterpret_cast<unsigned long long*>(cuts + b), (unsigned long long)s);
  }
}

__global__ void k_argmax(int32_t B, const int64_t* cuts, int32_t* best) {
  __shared__ long long sv[1024];
  __shared__ int32_t si[1024];
  long long bv = LLONG_MIN;
  int32_t bi = INT32_MAX;
  for (int32_t b = threadIdx.x; b < B; b += blockDim.x) {
    long long c = cuts[b];
    if (c > bv) { bv = c; bi = b; }   // ascending b per thread: first max kept
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      long long ov = sv[threadIdx.x + s];
      int32_t oi = si[threadIdx.x + s];
      if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *best = si[0];
}

// Record update: the evaluation's best becomes the global best if it is the
// first evaluation of the solve or strictly larger.
__global__ void k_record(int32_t phase, int32_t first, const int64_t* cuts, const int32_t* best_idx,
                         BestRecord* rec) {
  const int32_t b = *best_idx;
  const long long c = cuts[b];
  if (first || c > rec->cut) {
    rec->cut = c;
    rec->init = b;
    rec->phase = phase;
    rec->improved = 1;
  } else {
    rec->improved = 0;
  }
}

__global__ void k_extract(int32_t n, int32_t W, const uint32_t* zbits, const int32_t* best_idx,
                          const BestRecord* rec, uint8_t* phase_best_z, uint8_t* best_z) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int32_t b = *best_idx;
  const uint8_t z = (uint8_t)((zbits[(size_t)v * W + (b >> 5)] >> (b & 31)) & 1u);
  if (phase_best_z) phase_best_z[v] = z;
  if (rec->improved && best_z) best_z[v] = z;
}

int cut_grid_x(const deco_graph* g, int32_t W) {
  int dev_sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = ((int64_t)g->n + CUT_BLOCK / 32 - 1) / (CUT_BLOCK / 32);
  int64_t cap = (int64_t)dev_sms * 8 / (W > 0 ? W : 1);
  if (cap < dev_sms) cap = dev_sms;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

int launch_pack(const deco_graph* g, int32_t B, int32_t lift, int32_t ld, int precision,
                const void* y, uint32_t* zbits, cudaStream_t st) {
  const int32_t W = (B + 31) / 32;
  const int64_t threads = (int64_t)g->n * W * 32;
  const int block = 256;
  const unsigned grid = (unsigned)((threads + block - 1) / block);
  if (precision == DECO_PREC_BF16) k_pack<DECO_PREC_BF16><<<grid, block, 0, st>>>(g->n, B, lift, ld, W, y, zbits);
  else k_pack<DECO_PREC_FP32><<<grid, block, 0, st>>>(g->n, B, lift, ld, W, y, zbits);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

int launch_cut_bits(const deco_graph* g, int32_t B, const uint32_t* zbits, int64_t* cuts,
                    cudaStream_t st) {
  const int32_t W = (B + 31) / 32;
  DECO_CUDA_TRY(cudaMemsetAsync(cuts, 0, sizeof(int64_t) * (size_t)B, st));
  dim3 grid(cut_grid_x(g, W), W);
  BitsSrc src{zbits, W};
  k_cut<BitsSrc><<<grid, CUT_BLOCK, 0, st>>>(g->n, B, W, g->row_ptr, g->col_idx, g->wint, src, cuts);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

int launch_cut_bytes(const deco_graph* g, int32_t B, const uint8_t* z, int64_t* cuts,
                     cudaStream_t st) {
  const int32_t W = (B + 31) / 32;
  DECO_CUDA_TRY(cudaMemsetAsync(cuts, 0, sizeof(int64_t) * (size_t)B, st));
  dim3 grid(cut_grid_x(g, W), W);
  BytesSrc src{z, B};
  k_cut<BytesSrc><<<grid, CUT_BLOCK, 0, st>>>(g->n, B, W, g->row_ptr, g->col_idx, g->wint, src, cuts);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

int launch_argmax(int32_t B, const int64_t* cuts, int32_t* best, cudaStream_t st) {
  k_argmax<<<1, 1024, 0, st>>>(B, cuts, best);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

int launch_phase_finish(const deco_graph* g, int32_t B, int32_t phase, bool first, const int64_t* cuts,
                        const uint32_t* zbits, int32_t* best_idx, BestRecord* rec,
                        uint8_t* phase_best_z, uint8_t* best_z, cudaStream_t st) {
  int rc = launch_argmax(B, cuts, best_idx, st);
  if (rc) return rc;
  k_record<<<1, 1, 0, st>>>(phase, first ? 1 : 0, cuts, best_idx, rec);
  DECO_CUDA_TRY(cudaGetLastError());
  const int32_t W = (B + 31) / 32;
  k_extract<<<(g->n + 255) / 256, 256, 0, st>>>(g->n, W, zbits, best_idx, rec, phase_best_z, best_z);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

}  // namespace deco
