// Per-step PGA kernel for graphs whose iterate does not fit on chip, in its
// pipelined form (the launch shape DECO_KERNEL_GLOBAL | DECO_KERNEL_PIPELINED).
//
// The step is the same as k_step_global's (step_global.cu):
//   G = A Y                  (neighbour rows summed in the device CSR order, FP32)
//   grad = d (.) y - G  (Laplacian, Eq. 6 / 9)   or   -G  (multilinear)
//   V <- mu V + grad    (heavy-ball momentum, Sec. 4.2)
//   y <- Proj[-1,1](y + alpha_eff V)   (Eq. 7 / 10)
// with the same FP32 operations in the same order for every element, so the
// two kernels' iterates are bit-identical.  What differs is how the gathers
// reach the SM.
//
// Work: a sliced copy of the CSR, built once per graph (sell_image): rows
// sorted by degree (largest first, ties by index) and cut into slices of NG
// rows, entry k of the slice's row i at off[s] + k NG + i.  A warp owns slices
// s = warp, warp + #warps, ... (one group of G lanes per row of the slice, 16
// bytes of the row segment per lane); the rows of a slice have (nearly) the
// same degree, so the groups of a warp stay in step.
//
// Memory-level parallelism: every neighbour row segment is copied into shared
// memory with cp.async (16 bytes per lane, L2 only) several slices ahead of
// its use, so a warp keeps S - 1 slices of gathers in flight without holding
// them in registers.  Per iteration a warp (A) loads the next slice's
// metadata, (B) the column indices of the slice after that one, (C) issues
// the copies of the slice after that into one of S shared-memory stages, and
// then sums the oldest stage in CSR order and writes its rows.  A row of more
// than `maxe` entries is taken in parts of maxe entries, consecutive items of
// the same warp, the accumulator carried from one part to the next; its own
// row (and momentum) are copied with its last part.
#include <algorithm>
#include <numeric>
#include <vector>

#include "deco_internal.cuh"
#include "spmm.cuh"

namespace deco {

int device_sm_count();

namespace {

constexpr uint32_t SELL_PAD = 0xFFFFFFFFu;   // entry of a row shorter than its slice

struct SellArgs {
  int32_t n, C, ld;
  int32_t nslices;        // slices of the image
  int32_t ncc;            // column chunks of G x VN columns
  int32_t maxe;           // entries per part (<= 32)
  int32_t stages;         // S shared-memory stages per warp (2..4)
  uint32_t stage_bytes;   // bytes of one stage
  uint32_t group_bytes;   // bytes of one row group inside a stage
  uint32_t hdr_bytes;     // header (per group: row, degree, chunk, part) + weights
  const int64_t* off;
  const int2* rows;
  const int32_t* width;
  const uint32_t* idx;
  const float* w;
  const float* dnet;
  const void* yin;
  void* yout;
  float* v;
  float alpha_eff, afac, mu;
  const float* alpha_cols;
  const int32_t* steps_cols;
  int32_t t;
  int32_t* flag;
  int32_t lap, mom;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_stages(int S) {
  // the oldest of the S in-flight groups has landed (the S - 1 newest may be pending)
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

// One work item of a warp: part `part` of the slice with ordinal m (global
// slice index z = warp + m * #warps over column chunk x slice).
struct Meta {
  int64_t off;       // first entry of the slice
  int2 rd;           // this lane's row of the slice and its degree
  int32_t width;     // entries per row of the slice (its largest degree)
  int32_t cc;        // column chunk
  int32_t part;      // part index; < 0: no item
  int32_t last;      // 1 if this is the row's last part
};

template <int PREC, int G, bool WT, bool MIX>
__global__ void __launch_bounds__(256) k_step_sell(const __grid_constant__ SellArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using V = VecT<PREC>;
  constexpr int NG = 32 / G;   // rows per slice (groups per warp)
  constexpr int VN = V::N;     // columns per lane
  constexpr int W = 16 * G;    // bytes of a row segment
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int g = lane / G, j = lane % G;
  const int S = a.stages, MAXE = a.maxe;
  const int nwb = blockDim.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * nwb;
  const int64_t wid = (int64_t)blockIdx.x * nwb + wib;
  const int64_t total = (int64_t)a.ncc * a.nslices;
  const uint32_t wsm = smem_u32(smem) + (uint32_t)wib * (uint32_t)S * a.stage_bytes;
  unsigned char* const wsm_p = smem + (size_t)wib * S * a.stage_bytes;
  const size_t vrow_elems = (size_t)a.ld;
  const bool mom = a.mom != 0;

  // ---- the warp's item sequence: slice ordinals m with their part counts,
  // widths read from a window of 32 ordinals (one per lane), the next window
  // requested when the current one is entered
  auto load_width = [&](int64_t m) -> int32_t {
    const int64_t z = wid + m * nw;
    if (z >= total) return -1;
    return __ldg(a.width + (a.ncc == 1 ? (int32_t)z : (int32_t)(z % a.nslices)));
  };
  int64_t wbase = 0;
  int32_t win_cur = load_width(lane), win_next = load_width(32 + lane);
  int64_t cm = 0;        // cursor: slice ordinal
  int32_t cp = 0;        // cursor: part
  auto next_item = [&](Meta& mt) {
    if (cm - wbase >= 32) {
      win_cur = win_next;
      wbase += 32;
      win_next = load_width(wbase + 32 + lane);
    }
    const int32_t wdt = __shfl_sync(0xFFFFFFFFu, win_cur, (int)(cm - wbase));
    if (wdt < 0) { mt.part = -1; return; }
    const int64_t z = wid + cm * nw;
    const int32_t s = a.ncc == 1 ? (int32_t)z : (int32_t)(z % a.nslices);
    const int32_t parts = wdt > MAXE ? (wdt + MAXE - 1) / MAXE : 1;
    mt.off = __ldg(a.off + s);
    mt.rd = __ldg(a.rows + (size_t)s * NG + g);
    mt.width = wdt;
    mt.cc = a.ncc == 1 ? 0 : (int32_t)(z / a.nslices);
    mt.part = cp;
    mt.last = cp + 1 == parts;
    if (++cp == parts) { cp = 0; ++cm; }
  };

  // ---- (B) indices (and weights) of an item: entry k = part * MAXE + j + G q
  auto load_idx = [&](const Meta& mt, uint32_t (&ix)[NG], float (&wq)[NG]) {
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      ix[q] = SELL_PAD;
      wq[q] = 0.0f;
      const int kl = j + G * q;                    // entry within the part
      const int k = mt.part * MAXE + kl;
      if (mt.part >= 0 && kl < MAXE && k < mt.width) {
        const int64_t e = mt.off + (int64_t)k * NG + g;
        ix[q] = __ldg(a.idx + e);
        if (WT && a.w) wq[q] = __ldg(a.w + e);
      }
    }
  };

  // ---- (C) copies of an item into stage `st`
  auto issue = [&](const Meta& mt, const uint32_t (&ix)[NG], const float (&wq)[NG], int st) {
    if (mt.part < 0) return;
    const uint32_t sbase = wsm + (uint32_t)st * a.stage_bytes;
    int* hdr = reinterpret_cast<int*>(wsm_p + (size_t)st * a.stage_bytes);
    const int c0 = (mt.cc * G + j) * VN;
    const int k0 = mt.part * MAXE;
    const int cnt = min(MAXE, mt.width - k0);          // entries of this part (warp-uniform)
    const int my = min(cnt, mt.rd.y - k0);             // of them, this row's
    if (j == 0) {
      hdr[4 * g + 0] = mt.rd.x;
      hdr[4 * g + 1] = my;
      hdr[4 * g + 2] = mt.cc;
      hdr[4 * g + 3] = (mt.part == 0 ? 1 : 0) | (mt.last ? 2 : 0);
    }
    if (WT) {
      float* wsl = reinterpret_cast<float*>(wsm_p + (size_t)st * a.stage_bytes + 16 * NG) + g * MAXE;
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        const int kl = j + G * q;
        if (kl < cnt) {
          float wt = wq[q];
          if (!a.w) wt = (ix[q] & 0x80000000u) ? -1.0f : 1.0f;
          wsl[kl] = wt;
        }
      }
    }
    const uint32_t gbase = sbase + a.hdr_bytes + (uint32_t)g * a.group_bytes + (uint32_t)j * 16u;
    const bool col_ok = c0 < a.C;
    const char* ybase = static_cast<const char*>(a.yin) + (size_t)c0 * (PREC == DECO_PREC_BF16 ? 2 : 4);
    const size_t row_bytes = (size_t)a.ld * (PREC == DECO_PREC_BF16 ? 2 : 4);
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      if (G * q >= cnt) break;
      const int lim = min(G, cnt - G * q);
      for (int jj = 0; jj < lim; ++jj) {
        const uint32_t e = __shfl_sync(0xFFFFFFFFu, ix[q], g * G + jj);
        const int kl = G * q + jj;
        if (kl < my && col_ok)
          cp16(gbase + (uint32_t)kl * W, ybase + (size_t)(e & 0x7FFFFFFFu) * row_bytes);
      }
    }
    if (mt.last && mt.rd.x >= 0 && col_ok) {
      // own row (and momentum, FP32) for the update
      cp16(gbase + (uint32_t)MAXE * W, ybase + (size_t)mt.rd.x * row_bytes);
      if (mom) {
        const float* vrow = a.v + (size_t)mt.rd.x * vrow_elems + c0;
        const uint32_t vdst = sbase + a.hdr_bytes + (uint32_t)g * a.group_bytes + (uint32_t)(MAXE + 1) * W +
                              (uint32_t)j * (uint32_t)(VN * 4);
#pragma unroll
        for (int h = 0; h < VN / 4; ++h) cp16(vdst + 16u * h, vrow + 4 * h);
      }
    }
  };

  // ---- consumer state: the accumulator of the row in progress
  float acc[VN];
#pragma unroll
  for (int k = 0; k < VN; ++k) acc[k] = 0.0f;
  bool bad = false;

  auto consume = [&](int st) {
    const unsigned char* sp = wsm_p + (size_t)st * a.stage_bytes;
    const int* hdr = reinterpret_cast<const int*>(sp);
    const int row = hdr[4 * g + 0], my = hdr[4 * g + 1], cc = hdr[4 * g + 2], fl = hdr[4 * g + 3];
    const int cnt0 = hdr[1];   // group 0 holds the longest row of the slice
    const unsigned char* gp = sp + a.hdr_bytes + (size_t)g * a.group_bytes + (size_t)j * 16;
    const float* wsl = reinterpret_cast<const float*>(sp + 16 * NG) + g * MAXE;
    if (fl & 1) {
#pragma unroll
      for (int k = 0; k < VN; ++k) acc[k] = 0.0f;
    }
    // entries in CSR order: acc = acc + y_j (unit) or fma(w, y_j, acc)
#pragma unroll 4
    for (int kl = 0; kl < cnt0; ++kl) {
      if (kl < my) {
        const uint4 q = *reinterpret_cast<const uint4*>(gp + (size_t)kl * W);
        if (MIX && PREC == DECO_PREC_BF16 && !WT) {
          add_bf16x8(*reinterpret_cast<float(*)[8]>(acc), q);
          continue;
        }
        float val[VN];
        if (PREC == DECO_PREC_FP32) {
          val[0] = __uint_as_float(q.x); val[1] = __uint_as_float(q.y);
          val[2] = __uint_as_float(q.z); val[3] = __uint_as_float(q.w);
        } else {
          const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int h = 0; h < VN / 2; ++h) { val[2 * h] = bf16lo(u[h]); val[2 * h + 1] = bf16hi(u[h]); }
        }
        if (WT) {
          const float wt = wsl[kl];
#pragma unroll
          for (int k = 0; k < VN; ++k) acc[k] = fmaf(wt, val[k], acc[k]);
        } else {
#pragma unroll
          for (int k = 0; k < VN; ++k) acc[k] = acc[k] + val[k];
        }
      }
    }
    if (!(fl & 2) || row < 0) return;
    const int c0 = (cc * G + j) * VN;
    if (c0 >= a.C) return;
    // ---- epilogue: gradient, momentum, step, projection (as in k_step_global)
    float y[VN], vv[VN], out[VN];
    {
      const uint4 q = *reinterpret_cast<const uint4*>(gp + (size_t)MAXE * W);
      if (PREC == DECO_PREC_FP32) {
        y[0] = __uint_as_float(q.x); y[1] = __uint_as_float(q.y);
        y[2] = __uint_as_float(q.z); y[3] = __uint_as_float(q.w);
      } else {
        const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int h = 0; h < VN / 2; ++h) { y[2 * h] = bf16lo(u[h]); y[2 * h + 1] = bf16hi(u[h]); }
      }
    }
    if (mom) {
      const float* vs = reinterpret_cast<const float*>(sp + a.hdr_bytes + (size_t)g * a.group_bytes +
                                                       (size_t)(MAXE + 1) * W + (size_t)j * VN * 4);
#pragma unroll
      for (int k = 0; k < VN; ++k) vv[k] = vs[k];
    }
    const float dr = a.lap ? __ldg(a.dnet + row) : 0.0f;
#pragma unroll
    for (int k = 0; k < VN; ++k) {
      const int32_t c = c0 + k;
      const float grad = a.lap ? fmaf(dr, y[k], -acc[k]) : -acc[k];
      float step = grad;
      if (mom) step = fmaf(a.mu, vv[k], grad);
      const float alpha = a.alpha_cols ? a.afac * __ldg(a.alpha_cols + (c < a.C ? c : 0)) : a.alpha_eff;
      const bool active = (c < a.C) && (!a.steps_cols || a.t < __ldg(a.steps_cols + c));
      float yn = fmaf(alpha, step, y[k]);
      if (active && !isfinite(yn)) bad = true;
      yn = fminf(fmaxf(yn, -1.0f), 1.0f);
      out[k] = active ? yn : y[k];
      if (mom && active) vv[k] = step;
    }
    const size_t base = (size_t)row * a.ld + c0;
    if (c0 + VN <= a.C) {
      V::store(a.yout, base, out);
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
  };

  // ---- the pipeline: each iteration fetches the metadata of one item (A),
  // the indices of the item fetched one iteration earlier (B), issues the
  // copies of the item fetched two iterations earlier (C) and commits one
  // cp.async group.  Once S items are in flight the oldest is consumed: the
  // S - 1 newer ones are the S - 1 most recent groups, so wait_group(S - 1)
  // has landed it.  When nothing is left to issue, the remaining items are
  // consumed after wait_group(0).
  Meta mA, mB, mC;
  mA.part = mB.part = mC.part = -1;
  uint32_t ixB[NG], ixC[NG];
  float wB[NG], wC[NG];
#pragma unroll
  for (int q = 0; q < NG; ++q) { ixB[q] = ixC[q] = SELL_PAD; wB[q] = wC[q] = 0.0f; }
  int inflight = 0, st_issue = 0, st_take = 0;
  for (;;) {
    mC = mB;
#pragma unroll
    for (int q = 0; q < NG; ++q) { ixC[q] = ixB[q]; wC[q] = wB[q]; }
    mB = mA;
    next_item(mA);
    load_idx(mB, ixB, wB);
    if (mC.part >= 0) {
      issue(mC, ixC, wC, st_issue);
      if (++st_issue == S) st_issue = 0;
      ++inflight;
    }
    cp_commit();
    const bool draining = mA.part < 0 && mB.part < 0 && mC.part < 0;
    if (inflight == S) {
      cp_wait_stages(S);
    } else if (draining) {
      if (inflight == 0) break;
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else {
      continue;
    }
    __syncwarp();
    consume(st_take);
    __syncwarp();   // every lane is done with the stage before it is refilled
    if (++st_take == S) st_take = 0;
    --inflight;
  }
  if (bad && a.flag) atomicExch(a.flag, 1);
}

template <int PREC, int G, bool WT, bool MIX>
cudaError_t launch_g(const SellArgs& a, int wpb, cudaStream_t st) {
  const size_t smem = (size_t)wpb * a.stages * a.stage_bytes;
  static int set_bytes = 0;   // per instantiation
  auto kern = k_step_sell<PREC, G, WT, MIX>;
  if ((int)smem > set_bytes) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    set_bytes = (int)smem;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpb, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t warps_needed = (int64_t)a.ncc * a.nslices;
  int64_t blocks = (int64_t)device_sm_count() * per_sm;
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (warps_needed + wpb - 1) / wpb));
  kern<<<(unsigned)blocks, 32 * wpb, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PREC, int G>
cudaError_t launch_wt(const SellArgs& a, bool wt, bool mix, int wpb, cudaStream_t st) {
  if (wt) return launch_g<PREC, G, true, false>(a, wpb, st);
  if (PREC == DECO_PREC_BF16 && mix) return launch_g<PREC, G, false, true>(a, wpb, st);
  return launch_g<PREC, G, false, false>(a, wpb, st);
}

template <int PREC>
cudaError_t launch_p(const SellArgs& a, int G, bool wt, bool mix, int wpb, cudaStream_t st) {
  switch (G) {
    case 4: return launch_wt<PREC, 4>(a, wt, mix, wpb, st);
    case 8: return launch_wt<PREC, 8>(a, wt, mix, wpb, st);
    case 16: return launch_wt<PREC, 16>(a, wt, mix, wpb, st);
    default: return launch_wt<PREC, 32>(a, wt, mix, wpb, st);
  }
}

}  // namespace

// lanes per row segment for C columns: enough 16-byte vectors for the row,
// at least 4, at most 32 (wider blocks run as column chunks of 32 vectors)
int sell_group_lanes(int32_t C, int prec) {
  const int VN = prec == DECO_PREC_BF16 ? 8 : 4;
  const int nvec = (C + VN - 1) / VN;
  int G = 4;
  while (G < nvec && G < 32) G <<= 1;
  return G;
}

int sell_image(deco_graph* g, int ng, const SellImage** out) {
  for (auto& im : g->sells)
    if (im.ng == ng) { *out = &im; return DECO_OK; }
  const int32_t n = g->n;
  SellImage im;
  im.ng = ng;
  im.nslices = (n + ng - 1) / ng;
  // rows by degree, largest first; ties keep the row order
  std::vector<int32_t> order((size_t)n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    return g->h_row_ptr[x + 1] - g->h_row_ptr[x] > g->h_row_ptr[y + 1] - g->h_row_ptr[y];
  });
  std::vector<int64_t> off((size_t)im.nslices + 1);
  std::vector<int2> rows((size_t)im.nslices * ng);
  im.width.assign((size_t)im.nslices, 0);
  int64_t total = 0;
  for (int32_t s = 0; s < im.nslices; ++s) {
    off[s] = total;
    int32_t wdt = 0;
    for (int i = 0; i < ng; ++i) {
      const int64_t r = (int64_t)s * ng + i;
      if (r < n) {
        const int32_t v = order[r];
        const int32_t d = g->h_row_ptr[v + 1] - g->h_row_ptr[v];
        rows[r] = make_int2(v, d);
        wdt = std::max(wdt, d);
      } else {
        rows[r] = make_int2(-1, 0);
      }
    }
    im.width[s] = wdt;
    total += (int64_t)wdt * ng;
  }
  off[im.nslices] = total;
  const bool gen = g->wmode == W_GENERAL, sgn = g->wmode == W_SIGN;
  std::vector<uint32_t> idx((size_t)std::max<int64_t>(total, 1), SELL_PAD);
  std::vector<float> wts(gen ? (size_t)std::max<int64_t>(total, 1) : 0, 0.0f);
  for (int32_t s = 0; s < im.nslices; ++s) {
    for (int i = 0; i < ng; ++i) {
      const int2 rd = rows[(size_t)s * ng + i];
      if (rd.x < 0) continue;
      const int32_t e0 = g->h_row_ptr[rd.x];
      for (int32_t k = 0; k < rd.y; ++k) {
        const int64_t at = off[s] + (int64_t)k * ng + i;
        uint32_t c = (uint32_t)g->h_col[e0 + k];
        if (sgn && g->h_w[e0 + k] < 0.0f) c |= 0x80000000u;
        idx[at] = c;
        if (gen) wts[at] = g->h_w[e0 + k];
      }
    }
  }
  auto upload = [&](void** dst, const void* src, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(sliced image)");
    e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(sliced image)");
    return DECO_OK;
  };
  int rc = upload((void**)&im.off, off.data(), off.size() * sizeof(int64_t));
  if (!rc) rc = upload((void**)&im.rows, rows.data(), rows.size() * sizeof(int2));
  if (!rc) rc = upload((void**)&im.width_d, im.width.data(), im.width.size() * sizeof(int32_t));
  if (!rc) rc = upload((void**)&im.idx, idx.data(), idx.size() * sizeof(uint32_t));
  if (!rc && gen) rc = upload((void**)&im.w, wts.data(), wts.size() * sizeof(float));
  if (rc) {
    free_sell_image(im);
    return rc;
  }
  g->sells.push_back(std::move(im));
  *out = &g->sells.back();
  return DECO_OK;
}

void free_sell_image(SellImage& im) {
  cudaFree(im.off);
  cudaFree(im.rows);
  cudaFree(im.width_d);
  cudaFree(im.idx);
  cudaFree(im.w);
  im.off = nullptr;
  im.rows = nullptr;
  im.width_d = nullptr;
  im.idx = nullptr;
  im.w = nullptr;
}

// shared-memory bytes of one stage for (C, prec, maxe, momentum)
static void sell_sizes(int G, int prec, int maxe, bool mom, bool wt, uint32_t* hdr, uint32_t* group,
                       uint32_t* stage) {
  const int NG = 32 / G, VN = prec == DECO_PREC_BF16 ? 8 : 4, W = 16 * G;
  uint32_t h = 16u * NG + (wt ? 4u * NG * maxe : 0u);
  h = (h + 15u) & ~15u;
  const uint32_t gb = (uint32_t)(maxe + 1) * W + (mom ? (uint32_t)(G * VN * 4) : 0u);
  *hdr = h;
  *group = gb;
  *stage = h + (uint32_t)NG * gb;
}

size_t sell_smem_bytes(int32_t C, int prec, int maxe, int stages, int wpb, bool mom, bool weighted) {
  uint32_t h, gb, sb;
  sell_sizes(sell_group_lanes(C, prec), prec, maxe, mom, weighted, &h, &gb, &sb);
  return (size_t)wpb * stages * sb;
}

int launch_step_sell(const StepLaunch& s, const SellImage& im, int maxe, int stages, int wpb, bool mixed_add,
                     cudaStream_t st) {
  // lanes per row from the image (a narrower block, e.g. the ragged last
  // column slab, leaves the lanes past its columns idle)
  const int G = im.ng > 0 ? 32 / im.ng : 0;
  if ((G != 4 && G != 8 && G != 16 && G != 32) || maxe < 1 || maxe > 32 || stages < 2 || stages > 4 || wpb < 1 ||
      wpb > 8) {
    set_error("pipelined step: bad shape (ng=%d, maxe=%d, stages=%d, warps=%d)", im.ng, maxe, stages, wpb);
    return DECO_ERR_ARG;
  }
  const int VN = s.precision == DECO_PREC_BF16 ? 8 : 4;
  if (s.ld % 8 != 0) {
    set_error("pipelined step: ld %% 8 != 0");
    return DECO_ERR_ARG;
  }
  SellArgs a{};
  a.n = s.n;
  a.C = s.C;
  a.ld = s.ld;
  a.nslices = im.nslices;
  a.ncc = (s.C + G * VN - 1) / (G * VN);
  a.maxe = maxe;
  a.stages = stages;
  const bool mom = s.mu != 0.0f;
  const bool wt = s.wmode != W_UNIT;
  sell_sizes(G, s.precision, maxe, mom, wt, &a.hdr_bytes, &a.group_bytes, &a.stage_bytes);
  a.off = im.off;
  a.rows = im.rows;
  a.width = im.width_d;
  a.idx = im.idx;
  a.w = s.wmode == W_GENERAL ? im.w : nullptr;
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
  if (s.n == 0 || s.C == 0) return DECO_OK;
  const size_t smem = (size_t)wpb * stages * a.stage_bytes;
  int max_smem = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)max_smem) {
    set_error("pipelined step: %zu bytes of shared memory exceed the %d available", smem, max_smem);
    return DECO_ERR_UNSUPPORTED;
  }
  cudaError_t e = s.precision == DECO_PREC_BF16 ? launch_p<DECO_PREC_BF16>(a, G, wt, mixed_add, wpb, st)
                                                : launch_p<DECO_PREC_FP32>(a, G, wt, false, wpb, st);
  if (e != cudaSuccess) return cuda_fail(e, "k_step_sell launch");
  return DECO_OK;
}

}  // namespace deco
