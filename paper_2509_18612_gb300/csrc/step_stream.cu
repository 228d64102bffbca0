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
// cut into slices of NG rows, one group of G = 32 / NG lanes per row (16
// bytes of the row segment per lane), so the rows of a warp have (nearly) the
// same degree.  A slice whose rows have more than `maxe` entries becomes
// several items (parts of maxe entries, the accumulator carried from one to
// the next).  Slice s belongs to warp s mod #warps; each warp's items are one
// contiguous stream of fixed-size records (stream_image), built once per
// graph and launch shape:
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
#include <algorithm>
#include <numeric>
#include <vector>

#include "deco_internal.cuh"
#include "spmm.cuh"

namespace deco {

int device_sm_count();

namespace {

constexpr uint32_t REC_PAD = 0xFFFFFFFFu;   // entry past a row's count

struct StreamArgs {
  int32_t n, C, ld;
  int32_t ncc;            // column chunks of G x VN columns (the stream is taken once per chunk)
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
__device__ __forceinline__ void add_bf16x8(float (&acc)[8], const uint4 q) {
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

// ACC: how the BF16 rows of unit-weight graphs are summed (the same value
// either way): 0 widened and added in FP32, 1 with the mixed-precision add.
template <int PREC, int G, bool WT, int ACC>
__global__ void __launch_bounds__(256) k_step_stream(const __grid_constant__ StreamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using V = VecT<PREC>;
  constexpr int NG = 32 / G;
  constexpr int VN = V::N;
  constexpr int W = 16 * G;
  constexpr int E0 = 1 + 2 * NG;
  constexpr size_t ESZ = PREC == DECO_PREC_BF16 ? 2 : 4;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int g = lane / G, j = lane % G;
  const int S = a.stages, RR = 2 * a.stages, MAXE = a.maxe, RW = a.rw;
  const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
  const int32_t i0 = __ldg(a.soff + warp);
  const int32_t m = __ldg(a.soff + warp + 1) - i0;   // records of this warp
  if (m == 0) return;
  const int64_t total = (int64_t)m * a.ncc;
  const uint32_t rec_bytes = (uint32_t)RW * 4u;
  unsigned char* const wsm = smem + (size_t)wib * (RR * rec_bytes + S * a.stage_bytes);
  const uint32_t wsm_s = smem_u32(wsm);
  const uint32_t* const ring = reinterpret_cast<const uint32_t*>(wsm);
  const uint32_t stg_s = wsm_s + (uint32_t)RR * rec_bytes;
  const unsigned char* const stg = wsm + (size_t)RR * rec_bytes;
  const size_t row_bytes = (size_t)a.ld * ESZ;
  const uint32_t* const wrec = a.rec + (size_t)i0 * RW;
  const bool mom = a.mom != 0, lap = a.lap != 0;
  const uint64_t pol_first = a.hints ? policy_evict_first() : 0;

  // per-lane column parameters of the current column chunk
  int cc_have = -1;
  float alpha[VN];
  int32_t budget[VN];
  float acc[VN];
#pragma unroll
  for (int k = 0; k < VN; ++k) acc[k] = 0.0f;
  bool bad = false;

  // the three positions of the pipeline: record fetch (2S - 1 ahead), gather
  // issue (S - 1 ahead) and consumption, with their ring / stage slots
  Pos pf{0, 0}, pi{0, 0}, pc{0, 0};
  int sf = 0, si = 0, sc = 0, gi = 0, gc = 0;
  for (int64_t t = -(2 * S - 1); t < total; ++t) {
    // ---- record of item t + 2S - 1
    if (t + 2 * S - 1 < total) {
      for (int l = lane; l * 4 < RW; l += 32) {
        const uint32_t dst = wsm_s + (uint32_t)sf * rec_bytes + (uint32_t)l * 16u;
        const uint32_t* src = wrec + (size_t)pf.r * RW + l * 4;
        if (a.hints) cp16_hint(dst, src, pol_first);
        else cp16(dst, src);
      }
      pf.next(m);
      if (++sf == RR) sf = 0;
    }
    // ---- neighbour rows (and own row, momentum) of item t + S - 1
    if (t + S - 1 >= 0 && t + S - 1 < total) {
      const uint32_t* rc = ring + (size_t)si * RW;
      const int c0 = (pi.cc * G + j) * VN;
      const bool col_ok = c0 < a.C;
      const int kmax = (int)rc[0];
      const int row = (int)rc[1 + g];
      const uint32_t info = rc[1 + NG + g];
      const int cnt = (int)(info & 0xFFFFu);
      const uint32_t sb = stg_s + (uint32_t)gi * a.stage_bytes + (uint32_t)g * a.group_bytes + (uint32_t)j * 16u;
      const char* yb = static_cast<const char*>(a.yin) + (size_t)c0 * ESZ;
      if (col_ok) {
        for (int k = 0; k < kmax; ++k) {
          const uint32_t e = rc[E0 + k * NG + g];
          if (k < cnt) cp16(sb + (uint32_t)(k * W), yb + (size_t)(e & 0x7FFFFFFFu) * row_bytes);
        }
        if (((info >> 17) & 1u) && row >= 0) {
          cp16(sb + (uint32_t)(MAXE * W), yb + (size_t)row * row_bytes);
          if (mom) {
            const float* vrow = a.v + (size_t)row * a.ld + c0;
            const uint32_t vd = sb - (uint32_t)j * 16u + (uint32_t)((MAXE + 1) * W) + (uint32_t)j * (uint32_t)(VN * 4);
#pragma unroll
            for (int h = 0; h < VN / 4; ++h) cp16(vd + 16u * h, vrow + 4 * h);
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
      const int c0 = (pc.cc * G + j) * VN;
      const int kmax = (int)rc[0];
      const int row = (int)rc[1 + g];
      const uint32_t info = rc[1 + NG + g];
      const int cnt = (int)(info & 0xFFFFu);
      const unsigned char* gp = stg + (size_t)gc * a.stage_bytes + (size_t)g * a.group_bytes + (size_t)j * 16;
      if (info & 0x10000u) {
#pragma unroll
        for (int k = 0; k < VN; ++k) acc[k] = 0.0f;
      }
      // entries in CSR order: acc = acc + y_j (unit) or fma(w, y_j, acc)
#pragma unroll 4
      for (int k = 0; k < kmax; ++k) {
        if (k < cnt) {
          const uint4 q = *reinterpret_cast<const uint4*>(gp + (size_t)k * W);
          if (ACC == 1 && PREC == DECO_PREC_BF16 && !WT) {
            add_bf16x8(*reinterpret_cast<float(*)[8]>(acc), q);
          } else {
            float val[VN];
            unpack<PREC>(q, val);
            if (WT) {
              const uint32_t e = rc[E0 + k * NG + g];
              const float wt = a.gen ? __uint_as_float(rc[E0 + MAXE * NG + k * NG + g])
                                     : ((e & 0x80000000u) ? -1.0f : 1.0f);
#pragma unroll
              for (int h = 0; h < VN; ++h) acc[h] = fmaf(wt, val[h], acc[h]);
            } else {
#pragma unroll
              for (int h = 0; h < VN; ++h) acc[h] = acc[h] + val[h];
            }
          }
        }
      }
      if (((info >> 17) & 1u) && row >= 0 && c0 < a.C) {
        if (pc.cc != cc_have) {
          cc_have = pc.cc;
#pragma unroll
          for (int k = 0; k < VN; ++k) {
            const int c = c0 + k;
            alpha[k] = a.alpha_cols ? a.afac * __ldg(a.alpha_cols + (c < a.C ? c : 0)) : a.alpha_eff;
            budget[k] = c < a.C ? (a.steps_cols ? __ldg(a.steps_cols + c) : INT32_MAX) : -1;
          }
        }
        // ---- epilogue: gradient, momentum, step, projection (as in k_step_global)
        float y[VN], vv[VN], out[VN];
        unpack<PREC>(*reinterpret_cast<const uint4*>(gp + (size_t)MAXE * W), y);
        if (mom) {
          const float* vs = reinterpret_cast<const float*>(gp - (size_t)j * 16 + (size_t)(MAXE + 1) * W +
                                                           (size_t)j * VN * 4);
#pragma unroll
          for (int k = 0; k < VN; ++k) vv[k] = vs[k];
        }
        const float dr = lap ? __ldg(a.dnet + row) : 0.0f;
#pragma unroll
        for (int k = 0; k < VN; ++k) {
          const float grad = lap ? fmaf(dr, y[k], -acc[k]) : -acc[k];
          const float step = mom ? fmaf(a.mu, vv[k], grad) : grad;
          const bool active = a.t < budget[k];
          float yn = fmaf(alpha[k], step, y[k]);
          if (active && !isfinite(yn)) bad = true;
          yn = fminf(fmaxf(yn, -1.0f), 1.0f);
          out[k] = active ? yn : y[k];
          if (mom && active) vv[k] = step;
        }
        const size_t base = (size_t)row * a.ld + c0;
        if (c0 + VN <= a.C) {
          if (a.hints) {
            uint4 q;
            if (PREC == DECO_PREC_FP32) {
              q = make_uint4(__float_as_uint(out[0]), __float_as_uint(out[1]), __float_as_uint(out[2]),
                             __float_as_uint(out[3]));
            } else {
              q = make_uint4(pack_bf16x2(out[0], out[1]), pack_bf16x2(out[2], out[3]), pack_bf16x2(out[4], out[5]),
                             pack_bf16x2(out[6], out[7]));
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
      pc.next(m);
      if (++sc == RR) sc = 0;
      if (++gc == S) gc = 0;
    }
    __syncwarp();   // every lane is done with the record and the stage before they are refilled
  }
  if (bad && a.flag) atomicExch(a.flag, 1);
}

template <int PREC, int G>
void* pick_wt(bool wt, int acc) {
  if (wt) return reinterpret_cast<void*>(k_step_stream<PREC, G, true, 0>);
  if (PREC == DECO_PREC_BF16 && acc == 1) return reinterpret_cast<void*>(k_step_stream<PREC, G, false, 1>);
  return reinterpret_cast<void*>(k_step_stream<PREC, G, false, 0>);
}

void* pick_kernel(int prec, int G, bool wt, int acc) {
  if (prec == DECO_PREC_BF16) {
    switch (G) {
      case 4: return pick_wt<DECO_PREC_BF16, 4>(wt, acc);
      case 8: return pick_wt<DECO_PREC_BF16, 8>(wt, acc);
      case 16: return pick_wt<DECO_PREC_BF16, 16>(wt, acc);
      default: return pick_wt<DECO_PREC_BF16, 32>(wt, acc);
    }
  }
  switch (G) {
    case 4: return pick_wt<DECO_PREC_FP32, 4>(wt, 0);
    case 8: return pick_wt<DECO_PREC_FP32, 8>(wt, 0);
    case 16: return pick_wt<DECO_PREC_FP32, 16>(wt, 0);
    default: return pick_wt<DECO_PREC_FP32, 32>(wt, 0);
  }
}

// bytes of the per-warp areas of a shape
void stream_sizes(int G, int prec, int maxe, int stages, bool mom, bool gen, int32_t* rw, uint32_t* group,
                  uint32_t* stage, size_t* per_warp) {
  const int NG = 32 / G, VN = prec == DECO_PREC_BF16 ? 8 : 4, W = 16 * G;
  const int words = 1 + 2 * NG + maxe * NG * (gen ? 2 : 1);
  *rw = (words + 3) / 4 * 4;
  *group = (uint32_t)(maxe + 1) * W + (mom ? (uint32_t)(G * VN * 4) : 0u);
  *stage = (uint32_t)NG * *group;
  *per_warp = (size_t)2 * stages * *rw * 4 + (size_t)stages * *stage;
}

}  // namespace

// lanes per row segment for C columns: enough 16-byte vectors for the row,
// at least 4, at most 32 (wider blocks run as column chunks of 32 vectors)
int stream_group_lanes(int32_t C, int prec) {
  const int VN = prec == DECO_PREC_BF16 ? 8 : 4;
  const int nvec = (C + VN - 1) / VN;
  int G = 4;
  while (G < nvec && G < 32) G <<= 1;
  return G;
}

int stream_shape(int32_t C, int prec, int maxe, int stages, int wpb, bool weighted, bool gen, bool mixed,
                 bool hints, StreamShape* out) {
  if (maxe < 1 || maxe > 0xFFFF || stages < 2 || stages > 4 || wpb < 0 || wpb > 8) {
    set_error("pipelined step: bad shape (entries=%d, stages=%d, warps=%d)", maxe, stages, wpb);
    return DECO_ERR_ARG;
  }
  StreamShape sh;
  sh.G = stream_group_lanes(C, prec);
  sh.maxe = maxe;
  sh.stages = stages;
  sh.gen = gen;
  sh.weighted = weighted;
  sh.acc = (mixed && prec == DECO_PREC_BF16 && !weighted) ? 1 : 0;
  sh.hints = hints;
  int32_t rw;
  uint32_t group, stage;
  size_t per_warp, per_warp_mom;
  stream_sizes(sh.G, prec, maxe, stages, false, gen, &rw, &group, &stage, &per_warp);
  stream_sizes(sh.G, prec, maxe, stages, true, gen, &rw, &group, &stage, &per_warp_mom);
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // Warps per block: every warp keeps its own items in flight, so the shape
  // that keeps the most warps resident per SM wins (shared memory and
  // registers decide); a block must also fit with the momentum slots.  The
  // grid is sized for the layout without them (a phase with momentum then
  // takes a little more than one wave).
  void* fn = pick_kernel(prec, sh.G, weighted, sh.acc);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return cuda_fail(e, "pipelined step shared memory");
  auto resident = [&](int w, int* per_sm) -> cudaError_t {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, 32 * w, per_warp * w);
  };
  int per_sm = 0;
  if (!wpb) {
    int best_warps = 0;
    for (int w = 8; w >= 1; --w) {
      if (per_warp_mom * w > (size_t)max_smem) continue;
      int b = 0;
      if ((e = resident(w, &b)) != cudaSuccess) return cuda_fail(e, "pipelined step occupancy");
      if (b * w > best_warps) { best_warps = b * w; wpb = w; per_sm = b; }
    }
  } else if (per_warp_mom * wpb <= (size_t)max_smem) {
    if ((e = resident(wpb, &per_sm)) != cudaSuccess) return cuda_fail(e, "pipelined step occupancy");
  }
  if (!wpb || per_warp_mom * wpb > (size_t)max_smem) {
    set_error("the pipelined step kernel does not fit %d warps of %d entries x %d stages", wpb, maxe, stages);
    return DECO_ERR_UNSUPPORTED;
  }
  sh.wpb = wpb;
  sh.blocks = std::max(1, per_sm) * device_sm_count();
  sh.nw = sh.blocks * wpb;
  *out = sh;
  return DECO_OK;
}

int stream_image(deco_graph* g, const StreamShape& sh, const StreamImage** out) {
  const int ng = 32 / sh.G;
  for (auto& im : g->streams)
    if (im.ng == ng && im.maxe == sh.maxe && im.nw == sh.nw && im.gen == sh.gen) { *out = &im; return DECO_OK; }
  const int32_t n = g->n;
  const int maxe = sh.maxe;
  const bool gen = sh.gen, sgn = g->wmode == W_SIGN;
  StreamImage im;
  im.ng = ng;
  im.maxe = maxe;
  im.nw = sh.nw;
  im.gen = gen;
  const int words = 1 + 2 * ng + maxe * ng * (gen ? 2 : 1);
  im.rw = (words + 3) / 4 * 4;
  // rows by degree, largest first; ties keep the row order (a counting sort)
  auto deg = [&](int32_t v) { return g->h_row_ptr[v + 1] - g->h_row_ptr[v]; };
  int32_t dmax = 0;
  for (int32_t v = 0; v < n; ++v) dmax = std::max(dmax, deg(v));
  std::vector<int64_t> start((size_t)dmax + 2, 0);
  for (int32_t v = 0; v < n; ++v) ++start[(size_t)(dmax - deg(v)) + 1];
  for (size_t d = 1; d < start.size(); ++d) start[d] += start[d - 1];
  std::vector<int32_t> order((size_t)n);
  for (int32_t v = 0; v < n; ++v) order[(size_t)start[(size_t)(dmax - deg(v))]++] = v;
  const int32_t nslices = (n + ng - 1) / ng;
  // records per warp: slice s belongs to warp s mod nw, its parts consecutive
  std::vector<int64_t> count((size_t)im.nw + 1, 0);
  auto parts_of = [&](int32_t s) {
    const int32_t w = deg(order[(size_t)s * ng]);   // the slice's first row is its longest
    return w > maxe ? (w + maxe - 1) / maxe : 1;
  };
  for (int32_t s = 0; s < nslices; ++s) count[s % im.nw] += parts_of(s);
  std::vector<int32_t> soff((size_t)im.nw + 1, 0);
  int64_t acc = 0;
  for (int w = 0; w < im.nw; ++w) {
    soff[w] = (int32_t)acc;
    acc += count[w];
  }
  soff[im.nw] = (int32_t)acc;
  if (acc * im.rw > ((int64_t)1 << 31)) {
    set_error("the pipelined step kernel's records exceed 2^31 words (n=%d)", n);
    return DECO_ERR_UNSUPPORTED;
  }
  std::vector<uint32_t> rec((size_t)std::max<int64_t>(acc, 1) * im.rw, 0u);
  std::vector<int64_t> fill(soff.begin(), soff.end());
  for (int32_t s = 0; s < nslices; ++s) {
    const int w = s % im.nw;
    const int parts = parts_of(s);
    for (int p = 0; p < parts; ++p) {
      uint32_t* r = rec.data() + (size_t)fill[w]++ * im.rw;
      int kmax = 0;
      for (int i = 0; i < ng; ++i) {
        const int64_t rr = (int64_t)s * ng + i;
        const int32_t v = rr < n ? order[rr] : -1;
        const int32_t d = v >= 0 ? deg(v) : 0;
        const int32_t cnt = std::max(0, std::min(maxe, d - p * maxe));
        kmax = std::max(kmax, cnt);
        r[1 + i] = (uint32_t)v;
        r[1 + ng + i] = (uint32_t)cnt | (p == 0 ? 0x10000u : 0u) | (p == parts - 1 ? 0x20000u : 0u);
        const int32_t e0 = v >= 0 ? g->h_row_ptr[v] + p * maxe : 0;
        for (int k = 0; k < maxe; ++k) {
          uint32_t c = REC_PAD;
          float wt = 0.0f;
          if (k < cnt) {
            c = (uint32_t)g->h_col[e0 + k];
            if (sgn && g->h_w[e0 + k] < 0.0f) c |= 0x80000000u;
            if (gen) wt = g->h_w[e0 + k];
          }
          r[1 + 2 * ng + k * ng + i] = c;
          if (gen) {
            uint32_t u;
            memcpy(&u, &wt, 4);
            r[1 + 2 * ng + maxe * ng + k * ng + i] = u;
          }
        }
      }
      r[0] = (uint32_t)kmax;
    }
  }
  cudaError_t e = cudaMalloc((void**)&im.rec, rec.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(im.rec, rec.data(), rec.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&im.soff, soff.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(im.soff, soff.data(), soff.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_stream_image(im);
    return cuda_fail(e, "sliced record image");
  }
  im.records = acc;
  g->streams.push_back(std::move(im));
  *out = &g->streams.back();
  return DECO_OK;
}

void free_stream_image(StreamImage& im) {
  cudaFree(im.rec);
  cudaFree(im.soff);
  im.rec = nullptr;
  im.soff = nullptr;
}

int launch_step_stream(const StepLaunch& s, const StreamImage& im, const StreamShape& sh, cudaStream_t st) {
  if (s.n == 0 || s.C == 0) return DECO_OK;
  if (s.ld % 8 != 0 || im.ng * sh.G != 32 || im.maxe != sh.maxe || im.nw != sh.nw) {
    set_error("pipelined step: image and shape disagree (ld=%d)", s.ld);
    return DECO_ERR_ARG;
  }
  const int VN = s.precision == DECO_PREC_BF16 ? 8 : 4;
  const bool mom = s.mu != 0.0f;
  StreamArgs a{};
  a.n = s.n;
  a.C = s.C;
  a.ld = s.ld;
  a.ncc = (s.C + sh.G * VN - 1) / (sh.G * VN);
  a.maxe = sh.maxe;
  a.stages = sh.stages;
  size_t per_warp;
  stream_sizes(sh.G, s.precision, sh.maxe, sh.stages, mom, im.gen, &a.rw, &a.group_bytes, &a.stage_bytes, &per_warp);
  a.rec = im.rec;
  a.soff = im.soff;
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
  a.lap = s.objective == DECO_OBJ_LAPLACIAN;
  a.mom = mom;
  a.gen = im.gen;
  a.hints = sh.hints ? 1 : 0;
  const size_t smem = per_warp * sh.wpb;
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)max_smem) {
    set_error("pipelined step: %zu bytes of shared memory exceed the %d available", smem, max_smem);
    return DECO_ERR_UNSUPPORTED;
  }
  void* fn = pick_kernel(s.precision, sh.G, sh.weighted, sh.acc);
  void* args[] = {&a};
  cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)sh.blocks), dim3(32 * sh.wpb), args, smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "k_step_stream launch");
  return DECO_OK;
}

}  // namespace deco
