// Fused PGA step, one launch per step, iterate in global memory.
//
//   G = A Y                                  (CSR gather, FP32 accumulation)
//   grad = d (.) y - G   (Laplacian, Eq. 6 / 9)     or  -G   (multilinear)
//   V <- mu V + grad     (heavy-ball momentum, Sec. 4.2), else V = grad
//   y <- Proj[-1,1](y + alpha_eff V)         (Eq. 7 / 10)
//
// Layout: a group of G lanes owns one (row, column chunk); each lane owns one
// 16-byte vector of the row (4 FP32 or 8 BF16 columns).  Every gathered
// neighbour row segment is therefore read as G x 16 contiguous bytes; the
// gather itself (spmm.cuh) keeps eight independent gathers in flight per
// lane.  Used for graphs whose iterate does not fit on chip and as the
// reference launch shape for the persistent kernels.
#include <algorithm>

#include "deco_internal.cuh"
#include "spmm.cuh"

namespace deco {
namespace {

struct KArgs {
  int32_t n, C, ld, G, nchunks;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const uint32_t* col_sw;
  const float* w;
  const float* dnet;
  const void* yin;
  void* yout;
  float* v;
  float alpha_eff;      // alpha * objective factor
  float afac;           // objective factor applied to alpha_cols (1 or 2)
  float mu;
  const float* alpha_cols;
  const int32_t* steps_cols;
  int32_t t;
  int32_t* flag;
};

template <int PREC, int WMODE, bool MOM, bool LAP>
__global__ void __launch_bounds__(256) k_step_global(KArgs a) {
  using V = VecT<PREC>;
  constexpr int VN = V::N;
  const int lane = threadIdx.x & 31;
  const int gl = lane % a.G;                      // lane within the group
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / a.G;
  const int64_t total = (int64_t)a.n * a.nchunks;
  if (group >= total) return;
  const int32_t r = (int32_t)(group / a.nchunks);
  const int32_t ch = (int32_t)(group % a.nchunks);
  const int32_t vi = ch * a.G + gl;               // vector index within the row
  const int32_t c0 = vi * VN;                     // first column of this lane
  if (c0 >= a.C) return;                          // lane beyond the last column

  float acc[VN];
#pragma unroll
  for (int k = 0; k < VN; ++k) acc[k] = 0.0f;
  const int32_t e0 = __ldg(a.row_ptr + r), e1 = __ldg(a.row_ptr + r + 1);
  const CsrView A{a.col_idx, a.col_sw, a.w};
  csr_gather_row<PREC, WMODE>(A, a.yin, a.ld, c0, e0, e1, acc);

  // ---- epilogue: gradient, momentum, step, projection
  const size_t base = (size_t)r * a.ld + c0;
  float y[VN], out[VN];
  V::load(a.yin, base, y);
  const float dr = LAP ? __ldg(a.dnet + r) : 0.0f;
  float vv[VN];
  if (MOM) {
#pragma unroll
    for (int k = 0; k < VN; k += 4) {
      float4 q = *reinterpret_cast<const float4*>(a.v + base + k);
      vv[k] = q.x; vv[k + 1] = q.y; vv[k + 2] = q.z; vv[k + 3] = q.w;
    }
  }
  bool bad = false;
#pragma unroll
  for (int k = 0; k < VN; ++k) {
    const int32_t c = c0 + k;
    float grad = LAP ? fmaf(dr, y[k], -acc[k]) : -acc[k];
    float step = grad;
    if (MOM) {
      step = fmaf(a.mu, vv[k], grad);
    }
    float alpha = a.alpha_cols ? a.afac * __ldg(a.alpha_cols + (c < a.C ? c : 0)) : a.alpha_eff;
    bool active = (c < a.C) && (!a.steps_cols || a.t < __ldg(a.steps_cols + c));
    float yn = fmaf(alpha, step, y[k]);
    if (active && !isfinite(yn)) bad = true;
    yn = fminf(fmaxf(yn, -1.0f), 1.0f);
    out[k] = active ? yn : y[k];
    if (MOM && active) vv[k] = step;
  }
  if (c0 + VN <= a.C) {
    V::store(a.yout, base, out);
    if (MOM) {
#pragma unroll
      for (int k = 0; k < VN; k += 4)
        *reinterpret_cast<float4*>(a.v + base + k) = make_float4(vv[k], vv[k + 1], vv[k + 2], vv[k + 3]);
    }
  } else {
    // ragged last vector: only columns < C are written
    for (int k = 0; k < VN && c0 + k < a.C; ++k) {
      if (PREC == DECO_PREC_FP32) static_cast<float*>(a.yout)[base + k] = out[k];
      else static_cast<__nv_bfloat16*>(a.yout)[base + k] = __float2bfloat16_rn(out[k]);
      if (MOM) a.v[base + k] = vv[k];
    }
  }
  if (bad && a.flag) atomicExch(a.flag, 1);
}

template <int PREC, int WMODE, bool MOM, bool LAP>
void launch_t(const KArgs& a, int64_t threads, cudaStream_t st) {
  const int block = 256;
  const int64_t grid = (threads + block - 1) / block;
  k_step_global<PREC, WMODE, MOM, LAP><<<(unsigned)grid, block, 0, st>>>(a);
}

template <int PREC, int WMODE>
void launch_w(const KArgs& a, bool mom, bool lap, int64_t threads, cudaStream_t st) {
  if (mom) {
    if (lap) launch_t<PREC, WMODE, true, true>(a, threads, st);
    else launch_t<PREC, WMODE, true, false>(a, threads, st);
  } else {
    if (lap) launch_t<PREC, WMODE, false, true>(a, threads, st);
    else launch_t<PREC, WMODE, false, false>(a, threads, st);
  }
}

template <int PREC>
void launch_p(const KArgs& a, int wmode, bool mom, bool lap, int64_t threads, cudaStream_t st) {
  if (wmode == W_UNIT) launch_w<PREC, W_UNIT>(a, mom, lap, threads, st);
  else if (wmode == W_SIGN) launch_w<PREC, W_SIGN>(a, mom, lap, threads, st);
  else launch_w<PREC, W_GENERAL>(a, mom, lap, threads, st);
}

}  // namespace

int launch_step_global(const StepLaunch& s, cudaStream_t st) {
  KArgs a{};
  const int VN = s.precision == DECO_PREC_BF16 ? 8 : 4;
  const int nvec = (s.C + VN - 1) / VN;
  int G = 1;
  while (G < nvec && G < 32) G <<= 1;
  a.n = s.n;
  a.C = s.C;
  a.ld = s.ld;
  a.G = G;
  a.nchunks = (nvec + G - 1) / G;
  a.row_ptr = s.row_ptr;
  a.col_idx = s.col_idx;
  a.col_sw = s.col_sw;
  a.w = s.w;
  a.dnet = s.dnet;
  a.yin = s.yin;
  a.yout = s.yout;
  a.v = s.v;
  const float fac = s.objective == DECO_OBJ_MULTILINEAR01 ? 2.0f : 1.0f;
  a.alpha_eff = fac * s.alpha;
  a.afac = fac;
  a.mu = s.mu;
  a.alpha_cols = s.alpha_cols;
  a.steps_cols = s.steps_cols;
  a.t = s.t;
  a.flag = s.flag;
  const int64_t threads = (int64_t)s.n * a.nchunks * G;
  if (threads == 0) return DECO_OK;
  const bool mom = s.mu != 0.0f;
  const bool lap = s.objective == DECO_OBJ_LAPLACIAN;
  if (s.precision == DECO_PREC_BF16) launch_p<DECO_PREC_BF16>(a, s.wmode, mom, lap, threads, st);
  else launch_p<DECO_PREC_FP32>(a, s.wmode, mom, lap, threads, st);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

// ---- slab-major layout: row-major n x ld  <->  S slabs of dense n x w
// element (r, c) of the row-major block is element (r, c % w) of slab c / w.
namespace {
template <typename T>
__global__ void k_to_slabs(int32_t n, int32_t ld, int32_t C, int32_t w, int32_t S, const T* __restrict__ src,
                           T* __restrict__ dst, int to_slabs) {
  const int64_t total = (int64_t)n * C;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / C;
    const int32_t c = (int32_t)(i % C);   // column of the row-major block
    const int64_t slab_idx = (int64_t)(c / w) * n * w + r * w + (c % w);
    if (to_slabs) dst[slab_idx] = src[r * ld + c];
    else dst[r * ld + c] = src[slab_idx];
  }
}
}  // namespace

int launch_slab_layout(int32_t n, int32_t ld, int32_t C, int32_t w, int32_t S, size_t esz, const void* src,
                       void* dst, bool to_slabs, cudaStream_t st) {
  const int64_t total = (int64_t)n * C;
  if (total == 0) return DECO_OK;
  (void)S;
  const int block = 256;
  const unsigned grid = (unsigned)std::min<int64_t>((total + block - 1) / block, 152 * 32);
  if (esz == 2)
    k_to_slabs<uint16_t><<<grid, block, 0, st>>>(n, ld, C, w, S, static_cast<const uint16_t*>(src),
                                                  static_cast<uint16_t*>(dst), to_slabs ? 1 : 0);
  else
    k_to_slabs<uint32_t><<<grid, block, 0, st>>>(n, ld, C, w, S, static_cast<const uint32_t*>(src),
                                                  static_cast<uint32_t*>(dst), to_slabs ? 1 : 0);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

}  // namespace deco
