// CSR gather (one row of A Y for one lane's 16-byte vector of columns),
// shared by the projected-gradient step kernel and the message-passing
// aggregation of the learned proposal.
#pragma once

#include "deco_internal.cuh"

namespace deco {

template <int PREC>
struct VecT;
template <>
struct VecT<DECO_PREC_FP32> {
  static constexpr int N = 4;
  __device__ static void load(const void* base, size_t idx, float* out) {
    float4 q = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(base) + idx));
    out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
  }
  __device__ static void store(void* base, size_t idx, const float* in) {
    *reinterpret_cast<float4*>(static_cast<float*>(base) + idx) = make_float4(in[0], in[1], in[2], in[3]);
  }
};
template <>
struct VecT<DECO_PREC_BF16> {
  static constexpr int N = 8;
  __device__ static void load(const void* base, size_t idx, float* out) {
    uint4 q = __ldg(reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(base) + idx));
    out[0] = bf16lo(q.x); out[1] = bf16hi(q.x); out[2] = bf16lo(q.y); out[3] = bf16hi(q.y);
    out[4] = bf16lo(q.z); out[5] = bf16hi(q.z); out[6] = bf16lo(q.w); out[7] = bf16hi(q.w);
  }
  __device__ static void store(void* base, size_t idx, const float* in) {
    uint4 q = make_uint4(pack_bf16x2(in[0], in[1]), pack_bf16x2(in[2], in[3]),
                         pack_bf16x2(in[4], in[5]), pack_bf16x2(in[6], in[7]));
    *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(base) + idx) = q;
  }
};

struct CsrView {
  const int32_t* col_idx;
  const uint32_t* col_sw;   // index | sign bit (W_SIGN)
  const float* w;           // weights (W_GENERAL)
};

template <int WMODE>
__device__ __forceinline__ void csr_edge(const CsrView& A, int32_t e, int32_t& j, float& wt) {
  if (WMODE == W_UNIT) {
    j = __ldg(A.col_idx + e);
    wt = 1.0f;
  } else if (WMODE == W_SIGN) {
    uint32_t s = __ldg(A.col_sw + e);
    j = (int32_t)(s & 0x7FFFFFFFu);
    wt = (s & 0x80000000u) ? -1.0f : 1.0f;
  } else {
    j = __ldg(A.col_idx + e);
    wt = __ldg(A.w + e);
  }
}

// acc[k] += sum over entries e in [e0, e1) of w_e * Y[j_e, c0 + k], in CSR
// order, for this lane's VN = 16 / element-size columns.  Eight gathers are
// kept in flight per lane, then four, then one.
template <int PREC, int WMODE>
__device__ __forceinline__ void csr_gather_row(const CsrView& A, const void* Y, int32_t ld, int32_t c0,
                                               int32_t e0, int32_t e1, float* acc) {
  using V = VecT<PREC>;
  constexpr int VN = V::N;
  int32_t e = e0;
  for (; e + 8 <= e1; e += 8) {
    int32_t j[8];
    float wt[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) csr_edge<WMODE>(A, e + q, j[q], wt[q]);
    uint4 raw[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const size_t off = (size_t)j[q] * ld + c0;
      raw[q] = PREC == DECO_PREC_FP32
                   ? __ldg(reinterpret_cast<const uint4*>(static_cast<const float*>(Y) + off))
                   : __ldg(reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(Y) + off));
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float val[VN];
      if (PREC == DECO_PREC_FP32) {
        val[0] = __uint_as_float(raw[q].x); val[1] = __uint_as_float(raw[q].y);
        val[2] = __uint_as_float(raw[q].z); val[3] = __uint_as_float(raw[q].w);
      } else {
        const uint32_t u[4] = {raw[q].x, raw[q].y, raw[q].z, raw[q].w};
#pragma unroll
        for (int h = 0; h < VN / 2; ++h) { val[2 * h] = bf16lo(u[h]); val[2 * h + 1] = bf16hi(u[h]); }
      }
#pragma unroll
      for (int k = 0; k < VN; ++k) acc[k] = (WMODE == W_UNIT) ? acc[k] + val[k] : fmaf(wt[q], val[k], acc[k]);
    }
  }
  for (; e + 4 <= e1; e += 4) {
    int32_t j[4];
    float wt[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) csr_edge<WMODE>(A, e + q, j[q], wt[q]);
    float val[4][VN];
#pragma unroll
    for (int q = 0; q < 4; ++q) V::load(Y, (size_t)j[q] * ld + c0, val[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < VN; ++k) acc[k] = (WMODE == W_UNIT) ? acc[k] + val[q][k] : fmaf(wt[q], val[q][k], acc[k]);
  }
  for (; e < e1; ++e) {
    int32_t j;
    float wt, val[VN];
    csr_edge<WMODE>(A, e, j, wt);
    V::load(Y, (size_t)j * ld + c0, val);
#pragma unroll
    for (int k = 0; k < VN; ++k) acc[k] = (WMODE == W_UNIT) ? acc[k] + val[k] : fmaf(wt, val[k], acc[k]);
  }
}

}  // namespace deco
