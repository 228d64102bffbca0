// Persistent on-chip PGA kernel for graphs whose iterate slab fits in shared
// memory: all T steps of one phase (the step loop of Alg. 1 / Alg. 2) run inside one
// launch, with no trip through global memory between steps.
//
// Work unit ("item") = (graph, column slab).  A slab is 128 bytes of every row:
// 32 FP32 columns or 64 BF16 columns.  Because the columns of the block evolve
// independently (remark after Eq. 11), a slab needs no data from other slabs.
// An item is processed by a thread-block cluster of k CTAs:
//   * every CTA keeps a full replica of the slab (n rows x 128 B) in shared
//     memory, so every neighbour gather is a conflict-free 128-byte row read
//     (lane l reads word l of row j: one shared-memory wavefront per edge);
//   * the rows are split between the k CTAs by gather cost; each CTA keeps its
//     own rows' CSR image, momentum and a staging area in shared memory (the
//     lean form keeps only the CSR image: momentum in global memory, new rows
//     through L2, so that larger graphs or smaller clusters fit);
//   * per step: gather + fused update of the own rows into the staging area,
//     cluster barrier, broadcast of the staged rows into all k replicas
//     through distributed shared memory, cluster barrier.
// The CSR image (built once per graph and cluster size on the host) stores
// every neighbour as the byte offset of its replica row, in 16-byte aligned
// per-row lists, so one edge costs one 16-byte broadcast index load per four
// edges, one address add, one shared load and one add.
// Row-pair form: the two halves of a warp work on two rows at once, every
// lane on 8 bytes of the replica row, so one shared load instruction covers
// an entry of each row and a warp walks half as many per-row chains (the
// same wavefronts per edge, the same sums per column).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "deco_internal.cuh"
#include "slab.cuh"

namespace cg = cooperative_groups;

namespace deco {
namespace {


struct SmemLayout {
  size_t rep, stage, vsm, dn, img, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// lean: no staging area (the new rows go through L2) and the momentum in
// global memory, so that a whole graph of up to ~1 500 rows fits one CTA
__host__ __device__ inline SmemLayout slab_layout(int max_n, int max_own, int max_img_words, int prec,
                                                  bool lean) {
  SmemLayout L{};
  size_t o = 0;
  L.rep = o;   o = align16(o + (size_t)max_n * 128);
  L.stage = o; o = align16(o + (lean ? 0 : (size_t)max_own * 128));
  L.vsm = o;   o = align16(o + (lean ? 0 : (size_t)max_own * (prec == DECO_PREC_BF16 ? 256 : 128)));
  L.dn = o;    o = align16(o + (size_t)max_own * 4);
  L.img = o;   o = align16(o + (size_t)max_img_words * 4);
  L.total = o;
  return L;
}

// first local row whose cumulative cost reaches `target`; cost of a row =
// its padded list length + 8 (epilogue)
__device__ __forceinline__ int cost_search(const int4* ri, int rows, long long target) {
  int lo = 0, hi = rows;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((long long)ri[mid].x + 8LL * mid < target) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Sum (SIGN = +1) or subtract (SIGN = -1) the replica words of `cnt` edges
// whose byte offsets start at `p` (16-byte aligned); FP32 replica.
template <int SIGN, bool GEN>
__device__ __forceinline__ float gather_f32(const unsigned char* lb, const uint32_t* p, const float* w,
                                            int cnt, float acc) {
#define DECO_ACC(q, wv)                                                            \
  {                                                                                \
    const float y_ = *reinterpret_cast<const float*>(lb + (q));                    \
    acc = GEN ? fmaf((wv), y_, acc) : (SIGN > 0 ? acc + y_ : acc - y_);            \
  }
#pragma unroll 1
  for (; cnt >= 8; cnt -= 8, p += 8, w += 8) {
    const uint4 q0 = *reinterpret_cast<const uint4*>(p);
    const uint4 q1 = *reinterpret_cast<const uint4*>(p + 4);
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0;
    if (GEN) { w0 = *reinterpret_cast<const float4*>(w); w1 = *reinterpret_cast<const float4*>(w + 4); }
    DECO_ACC(q0.x, w0.x) DECO_ACC(q0.y, w0.y) DECO_ACC(q0.z, w0.z) DECO_ACC(q0.w, w0.w)
    DECO_ACC(q1.x, w1.x) DECO_ACC(q1.y, w1.y) DECO_ACC(q1.z, w1.z) DECO_ACC(q1.w, w1.w)
  }
  if (cnt > 0) {
    const uint4 q0 = *reinterpret_cast<const uint4*>(p);
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (GEN) w0 = *reinterpret_cast<const float4*>(w);
    DECO_ACC(q0.x, w0.x)
    if (cnt > 1) DECO_ACC(q0.y, w0.y)
    if (cnt > 2) DECO_ACC(q0.z, w0.z)
    if (cnt > 3) DECO_ACC(q0.w, w0.w)
    if (cnt > 4) {
      const uint4 q1 = *reinterpret_cast<const uint4*>(p + 4);
      float4 w1 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (GEN) w1 = *reinterpret_cast<const float4*>(w + 4);
      DECO_ACC(q1.x, w1.x)
      if (cnt > 5) DECO_ACC(q1.y, w1.y)
      if (cnt > 6) DECO_ACC(q1.z, w1.z)
    }
  }
#undef DECO_ACC
  return acc;
}

// Same for a BF16 replica (each lane owns two columns of the 128-byte row).
template <int SIGN, bool GEN>
__device__ __forceinline__ void gather_bf16(const unsigned char* lb, const uint32_t* p, const float* w,
                                            int cnt, float& a0, float& a1) {
#define DECO_ACC2(q, wv)                                                           \
  {                                                                                \
    const uint32_t u_ = *reinterpret_cast<const uint32_t*>(lb + (q));              \
    const float lo_ = bf16lo(u_), hi_ = bf16hi(u_);                                \
    if (GEN) { a0 = fmaf((wv), lo_, a0); a1 = fmaf((wv), hi_, a1); }               \
    else if (SIGN > 0) { a0 = a0 + lo_; a1 = a1 + hi_; }                           \
    else { a0 = a0 - lo_; a1 = a1 - hi_; }                                         \
  }
#pragma unroll 1
  for (; cnt >= 8; cnt -= 8, p += 8, w += 8) {
    const uint4 q0 = *reinterpret_cast<const uint4*>(p);
    const uint4 q1 = *reinterpret_cast<const uint4*>(p + 4);
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0;
    if (GEN) { w0 = *reinterpret_cast<const float4*>(w); w1 = *reinterpret_cast<const float4*>(w + 4); }
    DECO_ACC2(q0.x, w0.x) DECO_ACC2(q0.y, w0.y) DECO_ACC2(q0.z, w0.z) DECO_ACC2(q0.w, w0.w)
    DECO_ACC2(q1.x, w1.x) DECO_ACC2(q1.y, w1.y) DECO_ACC2(q1.z, w1.z) DECO_ACC2(q1.w, w1.w)
  }
  if (cnt > 0) {
    const uint4 q0 = *reinterpret_cast<const uint4*>(p);
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (GEN) w0 = *reinterpret_cast<const float4*>(w);
    DECO_ACC2(q0.x, w0.x)
    if (cnt > 1) DECO_ACC2(q0.y, w0.y)
    if (cnt > 2) DECO_ACC2(q0.z, w0.z)
    if (cnt > 3) DECO_ACC2(q0.w, w0.w)
    if (cnt > 4) {
      const uint4 q1 = *reinterpret_cast<const uint4*>(p + 4);
      float4 w1 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (GEN) w1 = *reinterpret_cast<const float4*>(w + 4);
      DECO_ACC2(q1.x, w1.x)
      if (cnt > 5) DECO_ACC2(q1.y, w1.y)
      if (cnt > 6) DECO_ACC2(q1.z, w1.z)
    }
  }
#undef DECO_ACC2
}

// Row-pair form: lanes 0-15 and 16-31 of a warp each work on their own row,
// every lane on 8 bytes of the 128-byte replica row (2 FP32 or 4 BF16
// columns), so one shared load serves one entry of each of the two rows.  Per
// column the sums are the same as in gather_f32 / gather_bf16: the same
// operation per entry, in list order.
template <int SIGN, bool GEN, int PREC>
__device__ __forceinline__ void gather_pair(const unsigned char* lb, const uint32_t* p, const float* w, int cnt,
                                            float* acc) {
#define DECO_ACCP(q, wv)                                                            \
  {                                                                                 \
    const uint2 u_ = *reinterpret_cast<const uint2*>(lb + (q));                     \
    float v_[4];                                                                    \
    if (PREC == DECO_PREC_FP32) {                                                   \
      v_[0] = __uint_as_float(u_.x); v_[1] = __uint_as_float(u_.y);                 \
    } else {                                                                        \
      v_[0] = bf16lo(u_.x); v_[1] = bf16hi(u_.x); v_[2] = bf16lo(u_.y); v_[3] = bf16hi(u_.y); \
    }                                                                               \
    _Pragma("unroll") for (int c_ = 0; c_ < (PREC == DECO_PREC_FP32 ? 2 : 4); ++c_) \
      acc[c_] = GEN ? fmaf((wv), v_[c_], acc[c_]) : (SIGN > 0 ? acc[c_] + v_[c_] : acc[c_] - v_[c_]); \
  }
#pragma unroll 1
  for (; cnt >= 8; cnt -= 8, p += 8, w += 8) {
    const uint4 q0 = *reinterpret_cast<const uint4*>(p);
    const uint4 q1 = *reinterpret_cast<const uint4*>(p + 4);
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0;
    if (GEN) { w0 = *reinterpret_cast<const float4*>(w); w1 = *reinterpret_cast<const float4*>(w + 4); }
    DECO_ACCP(q0.x, w0.x) DECO_ACCP(q0.y, w0.y) DECO_ACCP(q0.z, w0.z) DECO_ACCP(q0.w, w0.w)
    DECO_ACCP(q1.x, w1.x) DECO_ACCP(q1.y, w1.y) DECO_ACCP(q1.z, w1.z) DECO_ACCP(q1.w, w1.w)
  }
  if (cnt > 0) {
    const uint4 q0 = *reinterpret_cast<const uint4*>(p);
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (GEN) w0 = *reinterpret_cast<const float4*>(w);
    DECO_ACCP(q0.x, w0.x)
    if (cnt > 1) DECO_ACCP(q0.y, w0.y)
    if (cnt > 2) DECO_ACCP(q0.z, w0.z)
    if (cnt > 3) DECO_ACCP(q0.w, w0.w)
    if (cnt > 4) {
      const uint4 q1 = *reinterpret_cast<const uint4*>(p + 4);
      float4 w1 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (GEN) w1 = *reinterpret_cast<const float4*>(w + 4);
      DECO_ACCP(q1.x, w1.x)
      if (cnt > 5) DECO_ACCP(q1.y, w1.y)
      if (cnt > 6) DECO_ACCP(q1.z, w1.z)
    }
  }
#undef DECO_ACCP
}

// ---- exchange helpers (inline PTX: mbarrier, bulk async copy, proxy fences)
enum { XCHG_LOCAL = 0, XCHG_DSMEM = 1, XCHG_L2 = 2 };
constexpr uint32_t XCHG_CHUNK = 32768;
constexpr uint32_t XCHG_SPIN_LIMIT = 1u << 24;        // bounded wait: far above any real copy time ...
constexpr uint64_t XCHG_WAIT_NS = 2000000000ull;     // ... and 2 s at most

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the phase with the given parity to complete; false after the limit
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 1; i < XCHG_SPIN_LIMIT; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0 && gtimer() - t0 > XCHG_WAIT_NS) return false;
  }
  return false;
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int PREC, int WMODE, int NT, bool LEAN, bool PAIR>
__global__ void __launch_bounds__(NT, 1) k_slab(SlabParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_xbar;
  cg::cluster_group cluster = cg::this_cluster();
  const int k = P.k;
  const int rank = (int)cluster.block_rank();
  const int item = blockIdx.x / k;
  constexpr int COLS = PREC == DECO_PREC_BF16 ? 64 : 32;   // columns per slab
  constexpr size_t ESZ = PREC == DECO_PREC_BF16 ? 2 : 4;
  constexpr bool GEN = WMODE == W_GENERAL;
  int gi = 0, col0 = item * COLS;
  if (P.items) { const int2 it = P.items[item]; gi = it.x; col0 = it.y; }
  const SlabGraph& G = P.graphs ? P.graphs[gi] : P.g0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SmemLayout L = slab_layout(P.max_n, P.max_own, P.max_img_words, PREC, LEAN);
  uint32_t* rep = reinterpret_cast<uint32_t*>(smem + L.rep);
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem + L.stage);
  float* vsm = reinterpret_cast<float*>(smem + L.vsm);
  float* dn = reinterpret_cast<float*>(smem + L.dn);
  uint32_t* img = reinterpret_cast<uint32_t*>(smem + L.img);

  const int n = G.n, ld = G.ld, C = G.C;
  const int r0 = G.split[rank], r1 = G.split[rank + 1];
  const int own = r1 - r0;

  // ---- load the replica (all rows of the slab), the own CSR image and momentum
  const unsigned char* ybase = static_cast<const unsigned char*>(G.y) + (size_t)col0 * ESZ;
  for (int i = tid; i < n * 8; i += NT) {
    const int r = i >> 3, q = i & 7;
    reinterpret_cast<uint4*>(rep)[i] = *reinterpret_cast<const uint4*>(ybase + (size_t)r * ld * ESZ + q * 16);
  }
  {
    const uint4* src = G.image + G.img_off[rank];
    const int n16 = G.img_off[rank + 1] - G.img_off[rank];
    for (int i = tid; i < n16; i += NT) reinterpret_cast<uint4*>(img)[i] = src[i];
  }
  for (int i = tid; i < own; i += NT) dn[i] = __ldg(G.dnet + r0 + i);
  if (!LEAN) {
    for (int i = tid; i < own * COLS; i += NT) {
      const int rl = i / COLS, c = i % COLS;
      vsm[i] = (P.load_v && G.v) ? G.v[(size_t)(r0 + rl) * ld + col0 + c] : 0.0f;
    }
  }

  // ---- per-lane column parameters: CPL columns from slab column cl0 (the
  // row-pair form: half-warp hw, lane hl of it)
  constexpr int CPL = PAIR ? (PREC == DECO_PREC_BF16 ? 4 : 2) : (PREC == DECO_PREC_BF16 ? 2 : 1);
  const int hl = PAIR ? (lane & 15) : lane;
  const int hw = PAIR ? (lane >> 4) : 0;
  const int cl0 = hl * CPL;
  float alpha[4];
  int32_t tmax[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int c = col0 + cl0 + h;
    const bool valid = h < CPL && c < C;
    alpha[h] = valid ? (G.alpha_cols ? P.afac * __ldg(G.alpha_cols + c) : P.alpha) : 0.0f;
    tmax[h] = valid ? (G.steps_cols ? __ldg(G.steps_cols + c) : P.steps) : 0;
  }
  __syncthreads();

  const int4* rinfo = reinterpret_cast<const int4*>(img);
  const int E = rinfo[own].x;
  const uint32_t* offs = img + 4 * (own + 1);
  const float* wts = reinterpret_cast<const float*>(offs + E);

  // ---- rows of this warp (cost-balanced split of the own rows)
  const long long total = (long long)E + 8LL * own;
  const int wr0 = cost_search(rinfo, own, total * warp / (NT / 32));
  const int wr1 = cost_search(rinfo, own, total * (warp + 1) / (NT / 32));

  const unsigned char* lb = smem + L.rep + (PAIR ? hl * 8 : lane * 4);   // this lane's bytes of replica row 0
  const bool lap = P.objective == DECO_OBJ_LAPLACIAN;
  const bool mom = P.mu != 0.0f;
  bool bad = false, timed_out = false;
  // exchange of the new rows between the CTAs of the cluster (LEAN: through L2
  // even for a single CTA, which has no staging area)
  const int xmode = LEAN ? XCHG_L2 : (k == 1 ? XCHG_LOCAL : P.xmode);
  const int slab = col0 / COLS;
  unsigned char* x0buf = G.xbuf + (size_t)slab * n * 128;
  unsigned char* x1buf = G.xbuf + ((size_t)G.nslabs + slab) * n * 128;
  unsigned char* xnext = x0buf;
  uint64_t* xbar = &s_xbar;
  uint32_t xphase = 0;
  if (tid == 0) {
    mbar_init(xbar, 1);
    fence_mbar_init();
  }
  cluster.sync();   // every replica is loaded (and the barrier initialised) before any exchange

  // a device-side bound (the longest budget of a population round) keeps the
  // launch as short as the round, inside a captured graph as well
  const int nsteps = P.steps_dev ? min(P.steps, __ldg(P.steps_dev)) : P.steps;
  for (int t = 0; t < nsteps; ++t) {
    if constexpr (PAIR) {
      // two rows per warp, one per half-warp (the second half idles on the
      // last row of an odd range)
      for (int rb = wr0; rb < wr1; rb += 2) {
        const int rl = rb + hw;
        const bool has = rl < wr1;
        const int4 ri = has ? rinfo[rl] : make_int4(0, 0, 0, 0);
        const int r = r0 + rl;
        float vg[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (LEAN && mom && has) {
          const float* vrow = G.v + (size_t)r * ld + col0 + cl0;
#pragma unroll
          for (int h = 0; h < CPL; ++h) vg[h] = vrow[h];
        }
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        gather_pair<+1, GEN, PREC>(lb, offs + ri.x, wts + ri.x, ri.y, acc);
        if (WMODE == W_SIGN) gather_pair<-1, false, PREC>(lb, offs + ri.z, wts, ri.w, acc);
        if (has) {
          const uint2 wold = *reinterpret_cast<const uint2*>(smem + L.rep + (size_t)r * 128 + hl * 8);
          float y[4];
          if (PREC == DECO_PREC_FP32) {
            y[0] = __uint_as_float(wold.x); y[1] = __uint_as_float(wold.y); y[2] = 0.0f; y[3] = 0.0f;
          } else {
            y[0] = bf16lo(wold.x); y[1] = bf16hi(wold.x); y[2] = bf16lo(wold.y); y[3] = bf16hi(wold.y);
          }
          const float dr = lap ? dn[rl] : 0.0f;
          float out[4];
#pragma unroll
          for (int h = 0; h < CPL; ++h) {
            const float grad = lap ? fmaf(dr, y[h], -acc[h]) : -acc[h];
            float step = grad;
            float* vp = LEAN ? G.v + (size_t)r * ld + col0 + cl0 + h : vsm + (size_t)rl * COLS + cl0 + h;
            if (mom) step = fmaf(P.mu, LEAN ? vg[h] : *vp, grad);
            const bool active = t < tmax[h];
            float yn = fmaf(alpha[h], step, y[h]);
            if (active && !isfinite(yn)) bad = true;
            yn = fminf(fmaxf(yn, -1.0f), 1.0f);
            out[h] = active ? yn : y[h];
            if (mom && active) *vp = step;
          }
          uint2 word;
          if (PREC == DECO_PREC_FP32) word = make_uint2(__float_as_uint(out[0]), __float_as_uint(out[1]));
          else word = make_uint2(pack_bf16x2(out[0], out[1]), pack_bf16x2(out[2], out[3]));
          unsigned char* dst = xmode == XCHG_L2 ? xnext + (size_t)r * 128
                                                : reinterpret_cast<unsigned char*>(stage) + (size_t)rl * 128;
          *reinterpret_cast<uint2*>(dst + hl * 8) = word;
        }
      }
    } else {
    for (int rl = wr0; rl < wr1; ++rl) {
      const int4 ri = rinfo[rl];
      // LEAN: the row's momentum comes from global memory; its load is issued
      // before the gather so that its latency hides behind it
      float vg[2] = {0.0f, 0.0f};
      if (LEAN && mom) {
        const float* vrow = G.v + (size_t)(r0 + rl) * ld + col0 + (PREC == DECO_PREC_BF16 ? 2 * lane : lane);
        vg[0] = vrow[0];
        if (PREC == DECO_PREC_BF16) vg[1] = vrow[1];
      }
      float acc[2] = {0.0f, 0.0f};
      if (PREC == DECO_PREC_FP32) {
        acc[0] = gather_f32<+1, GEN>(lb, offs + ri.x, wts + ri.x, ri.y, 0.0f);
        if (WMODE == W_SIGN) acc[0] = gather_f32<-1, false>(lb, offs + ri.z, wts, ri.w, acc[0]);
      } else {
        gather_bf16<+1, GEN>(lb, offs + ri.x, wts + ri.x, ri.y, acc[0], acc[1]);
        if (WMODE == W_SIGN) gather_bf16<-1, false>(lb, offs + ri.z, wts, ri.w, acc[0], acc[1]);
      }
      // fused epilogue: gradient, momentum, step, projection
      const int r = r0 + rl;
      const uint32_t wold = rep[r * 32 + lane];
      float y[2];
      if (PREC == DECO_PREC_FP32) { y[0] = __uint_as_float(wold); y[1] = 0.0f; }
      else { y[0] = bf16lo(wold); y[1] = bf16hi(wold); }
      const float dr = lap ? dn[rl] : 0.0f;
      float out[2];
#pragma unroll
      for (int h = 0; h < (PREC == DECO_PREC_BF16 ? 2 : 1); ++h) {
        const float grad = lap ? fmaf(dr, y[h], -acc[h]) : -acc[h];
        float step = grad;
        float* vp = LEAN ? G.v + (size_t)r * ld + col0 + (PREC == DECO_PREC_BF16 ? 2 * lane + h : lane)
                         : vsm + (size_t)rl * COLS + (PREC == DECO_PREC_BF16 ? 2 * lane + h : lane);
        if (mom) step = fmaf(P.mu, LEAN ? vg[h] : *vp, grad);
        const bool active = t < tmax[h];
        float yn = fmaf(alpha[h], step, y[h]);
        if (active && !isfinite(yn)) bad = true;
        yn = fminf(fmaxf(yn, -1.0f), 1.0f);
        out[h] = active ? yn : y[h];
        if (mom && active) *vp = step;
      }
      const uint32_t word = PREC == DECO_PREC_FP32 ? __float_as_uint(out[0]) : pack_bf16x2(out[0], out[1]);
      if (xmode == XCHG_L2) reinterpret_cast<uint32_t*>(xnext)[(size_t)r * 32 + lane] = word;
      else stage[rl * 32 + lane] = word;
    }
    }
    if (xmode == XCHG_L2) {
      // publish the own rows through L2, then refresh the whole replica with
      // one bulk copy (async proxy) once every CTA of the cluster has written
      fence_proxy_async_global();
      fence_proxy_async_shared();
      cluster.sync();
      const uint32_t bytes = (uint32_t)n * 128u;
      if (tid == 0) {
        mbar_arrive_expect_tx(xbar, bytes);
        for (uint32_t off = 0; off < bytes; off += XCHG_CHUNK)
          bulk_g2s(smem + L.rep + off, xnext + off, min(XCHG_CHUNK, bytes - off), xbar);
      }
      if (!mbar_wait_bounded(xbar, xphase)) timed_out = true;
      xphase ^= 1u;
      xnext = (xnext == x0buf) ? x1buf : x0buf;
    } else if (xmode == XCHG_DSMEM) {
      cluster.sync();   // every CTA has finished reading its replica for step t
      const uint4* src = reinterpret_cast<const uint4*>(stage);
      for (int q = 0; q < k; ++q) {
        uint4* dst = reinterpret_cast<uint4*>(cluster.map_shared_rank(rep, q) + (size_t)r0 * 32);
        for (int i = tid; i < own * 8; i += NT) dst[i] = src[i];
      }
      cluster.sync();   // all replicas hold step t+1
    } else {
      __syncthreads();  // single CTA: the staged rows replace its own replica rows
      const uint4* src = reinterpret_cast<const uint4*>(stage);
      uint4* dst = reinterpret_cast<uint4*>(rep + (size_t)r0 * 32);
      for (int i = tid; i < own * 8; i += NT) dst[i] = src[i];
      __syncthreads();
    }
  }

  // ---- write the own rows (and momentum) back
  unsigned char* yout = static_cast<unsigned char*>(G.y) + (size_t)col0 * ESZ;
  for (int i = tid; i < own * 8; i += NT) {
    const int rl = i >> 3, q = i & 7;
    *reinterpret_cast<uint4*>(yout + (size_t)(r0 + rl) * ld * ESZ + q * 16) =
        reinterpret_cast<const uint4*>(rep)[(size_t)(r0 + rl) * 8 + q];
  }
  if (!LEAN && P.store_v && G.v) {
    for (int i = tid; i < own * COLS; i += NT) {
      const int rl = i / COLS, c = i % COLS;
      G.v[(size_t)(r0 + rl) * ld + col0 + c] = vsm[i];
    }
  }
  if (bad && P.flag) atomicOr(P.flag, 1);
  if (timed_out && P.flag) atomicOr(P.flag, 2);
}

template <int PREC, int WMODE, int NT, bool LEAN>
cudaError_t launch_t(const SlabParams& p, int n_items, size_t smem, cudaStream_t st) {
  auto fn = p.pairs ? k_slab<PREC, WMODE, NT, LEAN, true> : k_slab<PREC, WMODE, NT, LEAN, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(n_items * p.k), 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = p.k;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, p);
}

template <int PREC, int NT>
cudaError_t launch_n(const SlabParams& p, int wmode, int n_items, size_t smem, cudaStream_t st) {
  if (p.lean) {
    if (wmode == W_UNIT) return launch_t<PREC, W_UNIT, 1024, true>(p, n_items, smem, st);
    if (wmode == W_SIGN) return launch_t<PREC, W_SIGN, 1024, true>(p, n_items, smem, st);
    return launch_t<PREC, W_GENERAL, 1024, true>(p, n_items, smem, st);
  }
  if (wmode == W_UNIT) return launch_t<PREC, W_UNIT, NT, false>(p, n_items, smem, st);
  if (wmode == W_SIGN) return launch_t<PREC, W_SIGN, NT, false>(p, n_items, smem, st);
  return launch_t<PREC, W_GENERAL, NT, false>(p, n_items, smem, st);
}

template <int PREC>
cudaError_t launch_w(const SlabParams& p, int wmode, int n_items, size_t smem, cudaStream_t st) {
  return p.threads == 1024 ? launch_n<PREC, 1024>(p, wmode, n_items, smem, st)
                           : launch_n<PREC, 512>(p, wmode, n_items, smem, st);
}

// Wait-timeout probe: the exchange wait of k_slab on an mbarrier nobody
// arrives at; gives up after its limit and reports it in bit 1 of *flag.
__global__ void k_probe_xchg_wait(int32_t* flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0)) atomicOr(flag, 2);
}

}  // namespace

size_t slab_smem_bytes(int max_n, int max_own, int max_img_words, int prec, bool lean) {
  return slab_layout(max_n, max_own, max_img_words, prec, lean).total;
}

int slab_max_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    v = 227 * 1024;
  }
  return v - 1024;   // room for the kernel's static shared memory (mbarrier)
}

// Row split of one graph into k parts by cost(r) = row_ptr[r] + 2 r.
void slab_split(const int32_t* row_ptr_host, int32_t n, int k, int32_t* split) {
  const long long total = (long long)row_ptr_host[n] + 2LL * n;
  split[0] = 0;
  for (int i = 1; i < k; ++i) {
    const long long target = total * i / k;
    int lo = 0, hi = n;
    while (lo < hi) {
      int mid = (lo + hi) / 2;
      if ((long long)row_ptr_host[mid] + 2LL * mid < target) lo = mid + 1; else hi = mid;
    }
    split[i] = std::max(lo, split[i - 1]);
  }
  split[k] = n;
}

// On-chip CSR image of rows [row0, row0 + n) of a CSR whose columns in that
// range refer to the same rows (one member graph of a disjoint union, or a
// whole graph with row0 = 0), for cluster size k; device memory in im->data.
int slab_image_rows(const int32_t* row_ptr, const int32_t* col, const float* w, int wmode, int32_t row0,
                    int32_t n, int k, SlabImage* out) {
  SlabImage im;
  im.k = k;
  std::vector<int32_t> lrp((size_t)n + 1);
  for (int32_t r = 0; r <= n; ++r) lrp[r] = row_ptr[row0 + r] - row_ptr[row0];
  slab_split(lrp.data(), n, k, im.split);
  for (int i = k + 1; i <= SLAB_MAX_CLUSTER; ++i) im.split[i] = n;
  const bool gen = wmode == W_GENERAL;
  std::vector<uint32_t> words;
  for (int part = 0; part < k; ++part) {
    im.off[part] = (int32_t)(words.size() / 4);
    const int r0 = im.split[part], r1 = im.split[part + 1], own = r1 - r0;
    std::vector<int32_t> info(4 * (size_t)(own + 1), 0);
    std::vector<uint32_t> offs;
    std::vector<float> wts;
    for (int rl = 0; rl < own; ++rl) {
      const int r = row0 + r0 + rl;
      const int e0 = row_ptr[r], e1 = row_ptr[r + 1];
      int np = 0, nn = 0;
      for (int e = e0; e < e1; ++e) {
        if (wmode == W_SIGN && w[e] < 0.0f) ++nn; else ++np;
      }
      // positive (or all) entries, then negative entries; device order keeps
      // the positives of a +-1 row first
      info[4 * rl + 0] = (int32_t)offs.size();
      info[4 * rl + 1] = np;
      for (int e = e0; e < e0 + np; ++e) {
        offs.push_back((uint32_t)(col[e] - row0) * 128u);
        wts.push_back(gen ? w[e] : 1.0f);
      }
      while (offs.size() % 4) { offs.push_back(0); wts.push_back(0.0f); }
      info[4 * rl + 2] = (int32_t)offs.size();
      info[4 * rl + 3] = nn;
      for (int e = e0 + np; e < e1; ++e) {
        offs.push_back((uint32_t)(col[e] - row0) * 128u);
        wts.push_back(-1.0f);
      }
      while (offs.size() % 4) { offs.push_back(0); wts.push_back(0.0f); }
    }
    for (int i = 0; i < 8; ++i) { offs.push_back(0); wts.push_back(0.0f); }   // tail reads
    info[4 * own] = (int32_t)offs.size();
    words.insert(words.end(), info.begin(), info.end());
    words.insert(words.end(), offs.begin(), offs.end());
    if (gen) {
      for (float x : wts) {
        uint32_t u;
        memcpy(&u, &x, 4);
        words.push_back(u);
      }
    }
    while (words.size() % 4) words.push_back(0);
    im.max_own = std::max(im.max_own, own);
    im.max_words = std::max<int32_t>(im.max_words, (int32_t)(words.size() - 4 * (size_t)im.off[part]));
  }
  im.off[k] = (int32_t)(words.size() / 4);
  for (int i = k + 1; i <= SLAB_MAX_CLUSTER; ++i) im.off[i] = im.off[k];
  cudaError_t e = cudaMalloc((void**)&im.data, words.size() * 4);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(slab image)");
  e = cudaMemcpy(im.data, words.data(), words.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(im.data);
    return cuda_fail(e, "cudaMemcpy(slab image)");
  }
  *out = im;
  return DECO_OK;
}

int slab_image(deco_graph* g, int k, const SlabImage** out) {
  for (auto& im : g->images) {
    if (im.k == k) { *out = &im; return DECO_OK; }
  }
  SlabImage im;
  int rc = slab_image_rows(g->h_row_ptr.data(), g->h_col.data(), g->h_w.empty() ? nullptr : g->h_w.data(),
                           g->wmode, 0, g->n, k, &im);
  if (rc) return rc;
  g->images.push_back(im);
  *out = &g->images.back();
  return DECO_OK;
}

int launch_slab(const SlabParams& p, int n_items, int prec, int wmode, cudaStream_t st) {
  if (p.lean && (p.xmode != 2 || (p.mu != 0.0f && !p.load_v))) {
    set_error("lean slab launch: needs the L2 exchange and momentum loaded from global memory");
    return DECO_ERR_ARG;
  }
  const size_t smem = slab_smem_bytes(p.max_n, p.max_own, p.max_img_words, prec, p.lean != 0);
  if (smem > (size_t)slab_max_smem()) {
    set_error("slab kernel needs %zu bytes of shared memory", smem);
    return DECO_ERR_UNSUPPORTED;
  }
  cudaError_t e = prec == DECO_PREC_BF16 ? launch_w<DECO_PREC_BF16>(p, wmode, n_items, smem, st)
                                         : launch_w<DECO_PREC_FP32>(p, wmode, n_items, smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "k_slab launch");
  return DECO_OK;
}

int launch_wait_probe_slab(int32_t* flag, cudaStream_t st) {
  k_probe_xchg_wait<<<1, 32, 0, st>>>(flag);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DECO_OK : cuda_fail(e, "wait probe launch");
}

}  // namespace deco
