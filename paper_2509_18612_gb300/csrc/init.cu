// Starting blocks (Sec. 4.1 DUI / IDI, Sec. 4.2 batch Gaussian starts, Sec. 5
// down-scaling).  Random draws come from Philox4x32-10 keyed by the seed with
// counter (row, column, phase, stream); one counter per element, so every
// element is independent of the launch shape.
//   uniform u  = word 0            (u in (0,1), 23 random bits)
//   normal  N  = Box-Muller(word 0, word 1)
//   coins      = bit 0 of words 2 and 3 (IDI)
#include "deco_internal.cuh"

namespace deco {
namespace {

template <int PREC>
__device__ __forceinline__ void store_y(void* y, size_t i, float v) {
  if (PREC == DECO_PREC_FP32) static_cast<float*>(y)[i] = v;
  else static_cast<__nv_bfloat16*>(y)[i] = __float2bfloat16_rn(v);
}

template <int PREC>
__global__ void k_init(InitLaunch p) {
  const int32_t C = p.B * p.lift;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)p.n * C) return;
  const int32_t v = (int32_t)(idx / C);
  const int32_t c = (int32_t)(idx % C);
  const size_t o = (size_t)v * p.ld + c;
  if (p.init == DECO_INIT_EXPLICIT) {
    const float x = p.x0[o];
    store_y<PREC>(p.y, o, p.objective == DECO_OBJ_MULTILINEAR01 ? 2.0f * x - 1.0f : x);
    return;
  }
  uint32_t k0 = p.k0, k1 = p.k1, vr = (uint32_t)v;
  if (p.gid) batch_key(p.gid, p.goff, v, k0, k1, vr);   // graph i of a batch: key seed + i, own rows
  const uint4 r = philox4x32_10(make_uint4(vr, (uint32_t)c, (uint32_t)p.phase, STREAM_INIT), k0, k1);
  bool gaussian = p.init != DECO_INIT_UNIFORM;
  float half = p.uniform_half_width;
  if (p.init == DECO_INIT_IDI_HALF_UNIFORM && (c / p.lift) >= p.B / 2) {
    gaussian = false;   // second half of the starting points: scaled uniform
    half = p.scale;
  }
  float out;
  if (gaussian) {
    float m;
    if (p.mean_bits) m = p.mean_bits[v] ? 1.0f : -1.0f;
    else m = p.mean[v];
    const float eps = box_muller(r.x, r.y);
    out = p.scale * (m + sqrtf(p.eta) * eps);
    out = fminf(fmaxf(out, -1.0f), 1.0f);
  } else {
    out = half * (2.0f * u01(r.x) - 1.0f);
  }
  store_y<PREC>(p.y, o, out);
}

// IDI stage 1: side of every important node (p_i ~ U{-1,1}), 0 elsewhere.
// A batch passes the row -> graph map and one threshold per graph.
__global__ void k_idi_sides(int32_t n, const int32_t* deg, double thresh, const double* gthresh,
                            const int32_t* gid, const int32_t* goff, uint32_t k0, uint32_t k1,
                            int32_t phase, int8_t* side) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint32_t vr = (uint32_t)v;
  if (gid) {
    thresh = gthresh[gid[v]];
    batch_key(gid, goff, v, k0, k1, vr);
  }
  const bool imp = (double)deg[v] > thresh;
  int8_t s = 0;
  if (imp) {
    const uint4 r = philox4x32_10(make_uint4(vr, 0u, (uint32_t)phase, STREAM_IDI), k0, k1);
    s = (r.z & 1u) ? 1 : -1;
  }
  side[v] = s;
}

// IDI stage 2: unimportant nodes compare (A a)_i with (A b)_i (integers).
__global__ void k_idi_mean(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                           const int32_t* wint, const int8_t* side, const int32_t* gid, const int32_t* goff,
                           uint32_t k0, uint32_t k1, int32_t phase, float* h) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint32_t vr = (uint32_t)v;
  if (gid) batch_key(gid, goff, v, k0, k1, vr);
  const int8_t s = side[v];
  if (s != 0) { h[v] = (float)s; return; }
  long long aa = 0, ab = 0;
  for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
    const int8_t su = side[col_idx[e]];
    const int32_t w = wint ? wint[e] : 1;
    if (su > 0) aa += w;
    else if (su < 0) ab += w;
  }
  float out;
  if (aa < ab) out = 1.0f;
  else if (aa > ab) out = -1.0f;
  else {
    const uint4 r = philox4x32_10(make_uint4(vr, 0u, (uint32_t)phase, STREAM_IDI), k0, k1);
    out = (r.w & 1u) ? 1.0f : -1.0f;
  }
  h[v] = out;
}

__global__ void k_dui(int32_t n, const int32_t* deg, int32_t max_deg, uint32_t k0, uint32_t k1,
                      int32_t phase, float* h) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)v, 0u, (uint32_t)phase, STREAM_DUI), k0, k1);
  const float hw = max_deg > 0 ? 1.0f - (float)deg[v] / (float)max_deg : 0.0f;
  h[v] = (2.0f * u01(r.x) - 1.0f) * hw;
}

}  // namespace

int launch_init(const InitLaunch& p, cudaStream_t st) {
  const int64_t total = (int64_t)p.n * p.B * p.lift;
  if (total == 0) return DECO_OK;
  const int block = 256;
  const unsigned grid = (unsigned)((total + block - 1) / block);
  if (p.precision == DECO_PREC_BF16) k_init<DECO_PREC_BF16><<<grid, block, 0, st>>>(p);
  else k_init<DECO_PREC_FP32><<<grid, block, 0, st>>>(p);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

int launch_idi(const deco_graph* g, double thresh, uint32_t k0, uint32_t k1, int32_t phase,
               float* h, int8_t* side_scratch, cudaStream_t st) {
  return launch_idi_batch(g, thresh, nullptr, nullptr, nullptr, k0, k1, phase, h, side_scratch, st);
}

int launch_idi_batch(const deco_graph* g, double thresh, const double* gthresh, const int32_t* gid,
                     const int32_t* goff, uint32_t k0, uint32_t k1, int32_t phase, float* h,
                     int8_t* side_scratch, cudaStream_t st) {
  const int block = 256;
  const unsigned grid = (unsigned)((g->n + block - 1) / block);
  k_idi_sides<<<grid, block, 0, st>>>(g->n, g->deg, thresh, gthresh, gid, goff, k0, k1, phase, side_scratch);
  k_idi_mean<<<grid, block, 0, st>>>(g->n, g->row_ptr, g->col_idx, g->wint, side_scratch, gid, goff, k0, k1,
                                     phase, h);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

int launch_dui(const deco_graph* g, uint32_t k0, uint32_t k1, int32_t phase, float* h,
               cudaStream_t st) {
  const int block = 256;
  const unsigned grid = (unsigned)((g->n + block - 1) / block);
  k_dui<<<grid, block, 0, st>>>(g->n, g->deg, g->max_deg, k0, k1, phase, h);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

}  // namespace deco
