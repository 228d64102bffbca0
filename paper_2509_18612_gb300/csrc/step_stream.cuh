// Per-step PGA kernel for graphs whose iterate does not fit on chip, in its
// pipelined form (the launch shape DECO_KERNEL_GLOBAL | DECO_KERNEL_PIPELINED).
//
// The step is the same as k_step_global's (step_global.cu):
//   G = A Y                  (neighbour rows summed in the device CSR order, FP32)
//   grad = d (.) y - G  (Laplacian, Eq. 6 / 9)   or   -G  (multilinear)
//   V <- mu V + grad    (heavy-ball momentum, Sec. 4.2)
//   y <- Proj[-1,1](y + alpha_eff V)   (Eq. 7 / 10)
// with the same FP32 operations in the same order for every element, so the
// two kernels' iterates are bit-identical.  What differs is how the work
// reaches the SM.
//
// Work items: the rows sorted by degree (largest first, ties by index) are
// cut into slices of NG rows, one group of G = 32 / NG lanes per row, so the
// rows of a warp have (nearly) the same degree.  Each lane carries U 16-byte
// vectors of its row (U = 1, or 2 in the wide form: twice the rows per item
// for the same columns): vector u of lane j holds the columns
// (cc G U + u G + j) VN ... + VN - 1 of column chunk cc, so the G lanes of a
// group read G x 16 contiguous bytes per vector.  A slice whose rows have
// more than `maxe` entries becomes several items (parts of maxe entries, the
// accumulator carried from one to the next).  Slice s belongs to warp
// s mod #warps; each warp's items are one contiguous stream of fixed-size
// records (stream_image), built once per graph and launch shape:
//   [0]                     kmax: the largest entry count of the item's rows
//   [1 .. NG]               the row of group g (-1: none)
//   [1 + NG .. 2 NG]        entries of group g in this item | first part << 16 | last part << 17
//   [E0 + k NG + g]         column index of entry k of group g (sign of a +-1 weight in bit 31)
//   [E0 + maxe NG + k NG + g]  its weight (general integral weights only)
// with E0 = 1 + 2 NG, padded to a multiple of 4 words.
//
// Per iteration a warp copies (cp.async, L2 only) the record of the item
// 2S - 1 ahead into a ring of 2S records, then the neighbour row segments of
// the item S - 1 ahead (and its own row and momentum) into one of S
// shared-memory stages, then sums the oldest stage in CSR order and writes its
// rows.  No load sits in a dependency chain of registers: indices come from
// shared memory, gathered rows arrive S - 1 items after they are requested.
//
// FE > 0 fixes the entries per item (FE) and the stages (2) at compile time:
// the per-entry loops unroll completely and the shapes' runtime arithmetic
// folds away.  Shapes with other entry or stage counts run the FE = 0 form,
// which reads them from the arguments.
#pragma once

#include <cstdint>

#include "deco_internal.cuh"
#include "spmm.cuh"

namespace deco {

// kernel entry points of the pipelined step (the instantiations live in
// step_stream.cu for FE = 0 and in step_stream_e8.cu / step_stream_e12.cu)
void* stream_kernel_runtime(int prec, int G, bool wt, int acc);
void* stream_kernel_e8(int prec, int G, bool wt, int acc, int U);
void* stream_kernel_e12(int prec, int G, bool wt, int acc, int U);

namespace {

constexpr uint32_t REC_PAD = 0xFFFFFFFFu;   // entry past a row's count

struct StreamArgs {
  int32_t n, C, ld;
  int32_t ncc;            // column chunks of G x U x VN columns (the stream is taken once per chunk)
  int32_t maxe;           // entries per item
  int32_t stages;         // S shared-memory stages per warp (2..4); the record ring holds 2S
  int32_t rw;             // words per record
  uint32_t stage_bytes;   // bytes of one gather stage
  uint32_t group_bytes;   // bytes of one row group inside a stage
  const uint32_t* rec;    // records of all warps
  const int32_t* soff;    // first record of every warp (#warps + 1)
  const float* dnet;
  const void* yin;
  void* yout;
  float* v;
  float alpha_eff, afac, mu;
  const float* alpha_cols;
  const int32_t* steps_cols;
  int32_t t;
  int32_t* flag;
  int32_t lap, mom, gen;
  int32_t hints;          // 1: the records and the new rows evict-first in L2 (the gathered block keeps L2)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// the same copy with an L2 eviction priority (createpolicy)
__device__ __forceinline__ void cp16_hint(uint32_t dst, const void* src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_hint_v4(void* p, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// every group but the S - 1 most recent has landed
__device__ __forceinline__ void cp_wait_but(int S) {
  if (S == 2) asm volatile("cp.async.wait_group 1;" ::: "memory");
  else if (S == 3) asm volatile("cp.async.wait_group 2;" ::: "memory");
  else asm volatile("cp.async.wait_group 3;" ::: "memory");
}

// acc[k] += y[k] for the 8 BF16 values of q (low half of each word first),
// with Blackwell's mixed-precision add: the BF16 operand is widened exactly
// and the sum rounded once in FP32, the same operation as acc + float(y).
__device__ __forceinline__ void add_bf16x8(float* acc, const uint4 q) {
  const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    asm("{\n .reg .b16 lo, hi;\n mov.b32 {lo, hi}, %2;\n add.rn.f32.bf16 %0, lo, %0;\n add.rn.f32.bf16 %1, hi, %1;\n}"
        : "+f"(acc[2 * h]), "+f"(acc[2 * h + 1])
        : "r"(u[h]));
  }
}

template <int PREC>
__device__ __forceinline__ void unpack(const uint4 q, float* out) {
  if (PREC == DECO_PREC_FP32) {
    out[0] = __uint_as_float(q.x); out[1] = __uint_as_float(q.y);
    out[2] = __uint_as_float(q.z); out[3] = __uint_as_float(q.w);
  } else {
    const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) { out[2 * h] = bf16lo(u[h]); out[2 * h + 1] = bf16hi(u[h]); }
  }
}

// a position in the warp's item sequence: record r of the stream, column chunk cc
struct Pos {
  int32_t r, cc;
  __device__ void next(int32_t m) {
    if (++r == m) { r = 0; ++cc; }
  }
};

// words of one record for NG rows of maxe entries (general weights: a weight per entry)
__host__ __device__ constexpr int stream_record_words(int ng, int maxe, bool gen) {
  return (1 + 2 * ng + maxe * ng * (gen ? 2 : 1) + 3) / 4 * 4;
}

// ACC: how the BF16 rows of unit-weight graphs are summed (the same value
// either way): 0 widened and added in FP32, 1 with the mixed-precision add.
// U: 16-byte vectors per lane (1 or 2).  FE: entries per item fixed at
// compile time (two stages), or 0 (shape from the arguments).
template <int PREC, int G, bool WT, int ACC, int U, int FE>
__global__ void __launch_bounds__(256) k_step_stream(const __grid_constant__ StreamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using V = VecT<PREC>;
  constexpr int NG = 32 / G;
  constexpr int VN = V::N;                        // values of one 16-byte vector
  constexpr int W = 16 * G * U;                   // bytes of one row segment in a stage
  constexpr int E0 = 1 + 2 * NG;
  constexpr size_t ESZ = PREC == DECO_PREC_BF16 ? 2 : 4;
  constexpr size_t USTEP = (size_t)G * VN * ESZ;  // bytes from one vector of a lane to its next
  constexpr int RWMAX = FE ? stream_record_words(NG, FE, WT) : 0;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int g = lane / G, j = lane % G;
  const int S = FE ? 2 : a.stages, RR = 2 * S, MAXE = FE ? FE : a.maxe, RW = a.rw;
  const bool hints = a.hints != 0;
  const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
  const int32_t i0 = __ldg(a.soff + warp);
  const int32_t m = __ldg(a.soff + warp + 1) - i0;   // records of this warp
  if (m == 0) return;
  const int32_t total = m * a.ncc;                    // the host keeps records x chunks below 2^31
  const uint32_t rec_bytes = (uint32_t)RW * 4u;
  unsigned char* const wsm = smem + (size_t)wib * (RR * rec_bytes + S * a.stage_bytes);
  const uint32_t wsm_s = smem_u32(wsm);
  const uint32_t* const ring = reinterpret_cast<const uint32_t*>(wsm);
  const uint32_t stg_s = wsm_s + (uint32_t)RR * rec_bytes;
  const unsigned char* const stg = wsm + (size_t)RR * rec_bytes;
  const size_t row_bytes = (size_t)a.ld * ESZ;
  const uint32_t* const wrec = a.rec + (size_t)i0 * RW;
  const bool mom = a.mom != 0, lap = a.lap != 0;
  const uint64_t pol_first = hints ? policy_evict_first() : 0;

  // per-lane column parameters of the current column chunk
  int cc_have = -1;
  float alpha[U * VN];
  int32_t budget[U * VN];
  float acc[U * VN];
#pragma unroll
  for (int k = 0; k < U * VN; ++k) acc[k] = 0.0f;
  bool bad = false;

  // the three positions of the pipeline: record fetch (2S - 1 ahead), gather
  // issue (S - 1 ahead) and consumption, with their ring / stage slots
  Pos pf{0, 0}, pi{0, 0}, pc{0, 0};
  int sf = 0, si = 0, sc = 0, gi = 0, gc = 0;
  for (int32_t t = -(2 * S - 1); t < total; ++t) {
    // ---- record of item t + 2S - 1
    if (t + 2 * S - 1 < total) {
      const uint32_t dst = wsm_s + (uint32_t)sf * rec_bytes;
      const uint32_t* src = wrec + (size_t)pf.r * RW;
      if (FE && RWMAX <= 128) {
        if (lane * 4 < RW) {
          if (hints) cp16_hint(dst + (uint32_t)lane * 16u, src + lane * 4, pol_first);
          else cp16(dst + (uint32_t)lane * 16u, src + lane * 4);
        }
      } else {
        for (int l = lane; l * 4 < RW; l += 32) {
          if (hints) cp16_hint(dst + (uint32_t)l * 16u, src + l * 4, pol_first);
          else cp16(dst + (uint32_t)l * 16u, src + l * 4);
        }
      }
      pf.next(m);
      if (++sf == RR) sf = 0;
    }
    // ---- neighbour rows (and own row, momentum) of item t + S - 1
    if (t + S - 1 >= 0 && t + S - 1 < total) {
      const uint32_t* rc = ring + (size_t)si * RW;
      const int v0 = pi.cc * (G * U) + j;              // this lane's first vector of the row
      const bool ok1 = U == 2 && (v0 + G) * VN < a.C;  // its second vector holds columns < C
      const int row = (int)rc[1 + g];
      const uint32_t info = rc[1 + NG + g];
      const int cnt = (int)(info & 0xFFFFu);
      const uint32_t sb = stg_s + (uint32_t)gi * a.stage_bytes + (uint32_t)g * a.group_bytes + (uint32_t)j * 16u;
      const char* yb = static_cast<const char*>(a.yin) + (size_t)v0 * VN * ESZ;
      if (v0 * VN < a.C) {
        if constexpr (FE > 0) {
#pragma unroll
          for (int k = 0; k < FE; ++k) {
            if (k < cnt) {
              const uint32_t e = rc[E0 + k * NG + g];
              const char* src = yb + (size_t)(WT ? (e & 0x7FFFFFFFu) : e) * row_bytes;
              cp16(sb + (uint32_t)(k * W), src);
              if (U == 2 && ok1) cp16(sb + (uint32_t)(k * W + 16 * G), src + USTEP);
            }
          }
        } else {
          const int kmax = (int)rc[0];
          for (int k = 0; k < kmax; ++k) {
            const uint32_t e = rc[E0 + k * NG + g];
            if (k < cnt) {
              const char* src = yb + (size_t)(e & 0x7FFFFFFFu) * row_bytes;
              cp16(sb + (uint32_t)(k * W), src);
              if (U == 2 && ok1) cp16(sb + (uint32_t)(k * W + 16 * G), src + USTEP);
            }
          }
        }
        if (((info >> 17) & 1u) && row >= 0) {
          const char* src = yb + (size_t)row * row_bytes;
          cp16(sb + (uint32_t)(MAXE * W), src);
          if (U == 2 && ok1) cp16(sb + (uint32_t)(MAXE * W + 16 * G), src + USTEP);
          if (mom) {
            // momentum of vector u of lane j at float (u G + j) VN after the row segments
            const uint32_t vd = sb - (uint32_t)j * 16u + (uint32_t)((MAXE + 1) * W);
#pragma unroll
            for (int u = 0; u < U; ++u) {
              if (u == 0 || ok1) {
                const float* vrow = a.v + (size_t)row * a.ld + (size_t)(v0 + u * G) * VN;
#pragma unroll
                for (int h = 0; h < VN / 4; ++h) cp16(vd + (uint32_t)((u * G + j) * VN * 4 + 16 * h), vrow + 4 * h);
              }
            }
          }
        }
      }
      pi.next(m);
      if (++si == RR) si = 0;
      if (++gi == S) gi = 0;
    }
    cp_commit();
    cp_wait_but(S);
    __syncwarp();
    if (t >= 0) {
      // ---- consume item t
      const uint32_t* rc = ring + (size_t)sc * RW;
      const int v0 = pc.cc * (G * U) + j;
      const int row = (int)rc[1 + g];
      const uint32_t info = rc[1 + NG + g];
      const int cnt = (int)(info & 0xFFFFu);
      const unsigned char* gp = stg + (size_t)gc * a.stage_bytes + (size_t)g * a.group_bytes + (size_t)j * 16;
      if (info & 0x10000u) {
#pragma unroll
        for (int k = 0; k < U * VN; ++k) acc[k] = 0.0f;
      }
      // entry k in CSR order: acc = acc + y_j (unit) or fma(w, y_j, acc)
      auto entry = [&](int k) {
        float wt = 1.0f;
        if (WT) {
          const uint32_t e = rc[E0 + k * NG + g];
          wt = a.gen ? __uint_as_float(rc[E0 + MAXE * NG + k * NG + g]) : ((e & 0x80000000u) ? -1.0f : 1.0f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint4 q = *reinterpret_cast<const uint4*>(gp + (size_t)k * W + (size_t)u * 16 * G);
          if (ACC == 1 && PREC == DECO_PREC_BF16 && !WT) {
            add_bf16x8(acc + u * VN, q);
          } else {
            float val[VN];
            unpack<PREC>(q, val);
#pragma unroll
            for (int h = 0; h < VN; ++h) acc[u * VN + h] = WT ? fmaf(wt, val[h], acc[u * VN + h]) : acc[u * VN + h] + val[h];
          }
        }
      };
      if constexpr (FE > 0) {
#pragma unroll
        for (int k = 0; k < FE; ++k)
          if (k < cnt) entry(k);
      } else {
        const int kmax = (int)rc[0];
#pragma unroll 4
        for (int k = 0; k < kmax; ++k)
          if (k < cnt) entry(k);
      }
      if (((info >> 17) & 1u) && row >= 0 && v0 * VN < a.C) {
        if (pc.cc != cc_have) {
          cc_have = pc.cc;
#pragma unroll
          for (int k = 0; k < U * VN; ++k) {
            const int c = (v0 + (k / VN) * G) * VN + k % VN;
            alpha[k] = a.alpha_cols ? a.afac * __ldg(a.alpha_cols + (c < a.C ? c : 0)) : a.alpha_eff;
            budget[k] = c < a.C ? (a.steps_cols ? __ldg(a.steps_cols + c) : INT32_MAX) : -1;
          }
        }
        // ---- epilogue: gradient, momentum, step, projection (as in k_step_global)
        const float dr = lap ? __ldg(a.dnet + row) : 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c0 = (v0 + u * G) * VN;
          if (u > 0 && c0 >= a.C) break;
          float y[VN], vv[VN], out[VN];
          unpack<PREC>(*reinterpret_cast<const uint4*>(gp + (size_t)MAXE * W + (size_t)u * 16 * G), y);
          if (mom) {
            const float* vs = reinterpret_cast<const float*>(gp - (size_t)j * 16 + (size_t)(MAXE + 1) * W +
                                                             (size_t)(u * G + j) * VN * 4);
#pragma unroll
            for (int k = 0; k < VN; ++k) vv[k] = vs[k];
          }
#pragma unroll
          for (int k = 0; k < VN; ++k) {
            const float grad = lap ? fmaf(dr, y[k], -acc[u * VN + k]) : -acc[u * VN + k];
            const float step = mom ? fmaf(a.mu, vv[k], grad) : grad;
            const bool active = a.t < budget[u * VN + k];
            float yn = fmaf(alpha[u * VN + k], step, y[k]);
            if (active && !isfinite(yn)) bad = true;
            yn = fminf(fmaxf(yn, -1.0f), 1.0f);
            out[k] = active ? yn : y[k];
            if (mom && active) vv[k] = step;
          }
          const size_t base = (size_t)row * a.ld + c0;
          if (c0 + VN <= a.C) {
            if (hints) {
              uint4 q;
              if (PREC == DECO_PREC_FP32) {
                q = make_uint4(__float_as_uint(out[0]), __float_as_uint(out[1]), __float_as_uint(out[2]),
                               __float_as_uint(out[3]));
              } else {
                q = make_uint4(pack_bf16x2(out[0], out[1]), pack_bf16x2(out[2], out[3]),
                               pack_bf16x2(out[4], out[5]), pack_bf16x2(out[6], out[7]));
              }
              st_hint_v4(static_cast<char*>(a.yout) + base * ESZ, q, pol_first);
            } else {
              V::store(a.yout, base, out);
            }
            if (mom) {
#pragma unroll
              for (int k = 0; k < VN; k += 4)
                *reinterpret_cast<float4*>(a.v + base + k) = make_float4(vv[k], vv[k + 1], vv[k + 2], vv[k + 3]);
            }
          } else {
            for (int k = 0; k < VN && c0 + k < a.C; ++k) {
              if (PREC == DECO_PREC_FP32) static_cast<float*>(a.yout)[base + k] = out[k];
              else static_cast<__nv_bfloat16*>(a.yout)[base + k] = __float2bfloat16_rn(out[k]);
              if (mom) a.v[base + k] = vv[k];
            }
          }
        }
      }
      pc.next(m);
      if (++sc == RR) sc = 0;
      if (++gc == S) gc = 0;
    }
    __syncwarp();   // every lane is done with the record and the stage before they are refilled
  }
  if (bad && a.flag) atomicExch(a.flag, 1);
}

// the instantiations of one entries-per-item form, by data type, lanes per
// row, weights, summation and vectors per lane
template <int PREC, int G, int U, int FE>
void* stream_kernel_wt(bool wt, int acc) {
  if (wt) return reinterpret_cast<void*>(k_step_stream<PREC, G, true, 0, U, FE>);
  if (PREC == DECO_PREC_BF16 && acc == 1) return reinterpret_cast<void*>(k_step_stream<PREC, G, false, 1, U, FE>);
  return reinterpret_cast<void*>(k_step_stream<PREC, G, false, 0, U, FE>);
}

template <int PREC, int U, int FE>
void* stream_kernel_g(int G, bool wt, int acc) {
  switch (G) {
    case 2:   // two lanes per row: the wide form only
      if constexpr (U == 2) return stream_kernel_wt<PREC, 2, U, FE>(wt, acc);
      return nullptr;
    case 4: return stream_kernel_wt<PREC, 4, U, FE>(wt, acc);
    case 8: return stream_kernel_wt<PREC, 8, U, FE>(wt, acc);
    case 16: return stream_kernel_wt<PREC, 16, U, FE>(wt, acc);
    default: return stream_kernel_wt<PREC, 32, U, FE>(wt, acc);
  }
}

template <int U, int FE>
void* stream_kernel_for(int prec, int G, bool wt, int acc) {
  if (prec == DECO_PREC_BF16) return stream_kernel_g<DECO_PREC_BF16, U, FE>(G, wt, acc);
  return stream_kernel_g<DECO_PREC_FP32, U, FE>(G, wt, 0);
}

}  // namespace
}  // namespace deco
