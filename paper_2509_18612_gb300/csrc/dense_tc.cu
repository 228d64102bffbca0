// Tensor-core PGA step for dense graphs (DECO_KERNEL_DENSE):
//
//   G = A Y   dense BF16 x BF16 products, FP32 accumulation in tensor memory
//             (A is 0 / integral weights |w| <= 256, exact in BF16; Y is the
//             BF16 iterate, so every product is exact)
//   grad = d (.) y - G (Laplacian, Eq. 6 / 9)  or  -G (multilinear)
//   V <- mu V + grad (Sec. 4.2), y <- Proj[-1,1](y + alpha_eff V) (Eq. 7 / 10)
//
// The iterate is kept transposed, YT = Y^T (cpad x kpad, node index
// contiguous), so both MMA operands are K-major: the A tile is 128 nodes x 64
// neighbour nodes, the B tile is N columns x the same 64 neighbour nodes of
// YT, each a stack of 128-byte rows in the 128-byte swizzled layout written by
// TMA.  One lane issues the TMA loads of a stage ring; the MMAs (M = 128,
// N <= 256, K = 16 each) of the even chunks of the contraction range
// accumulate into D0, those of the odd chunks into D1, and the partial product
// is D0 + D1 (the same order in both kernels, so their results agree bit for
// bit).  The per-step kernel issues both from one lane; the phase kernel from
// one lane of each of two warps: an M = 128, N = 128, K = 16 instruction takes
// the tensor core ~33 ns (deco_probe_mma_rate), well under the loop's time per
// chunk, which the stage handshakes (waits on TMA arrivals, commits) set; two
// issuers overlap the waits of consecutive chunks.  Full / empty mbarriers
// hand the stages between producer and issuers, so no block barrier runs
// inside the contraction.
//
// Grid: (row tiles x KS) CTAs along x, column tiles of <= 256 along y.  The KS
// CTAs of a cluster split the contraction of one 128 x N output tile.  After
// the contraction each CTA pushes the rows of its partial product owned by a
// peer into that peer's shared memory (distributed shared memory stores), and
// CTA r reduces rows [r 128/KS, (r+1) 128/KS) over the KS partials in rank
// order and applies the update, eight rows of one column per 16-byte vector.
// The y and V operands of the update are loaded into registers before the
// contraction starts.  Every mbarrier wait is bounded (globaltimer); the
// accumulator's tensor-memory columns are released on every path.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "dense_tc.cuh"

namespace cg = cooperative_groups;

namespace deco {
namespace {

constexpr int BM = DENSE_BM, BK = DENSE_BK, NTHREADS = 128, MAX_STAGES = 8, PF = 4;
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s per wait at most
constexpr uint32_t RING_BUDGET = 200u * 1024u;

struct DenseArgs {
  CUtensorMap tmA;   // dense A, box 64 x 128
  CUtensorMap tmY;   // YT of this step, box 64 x min(256, cpad)
  DenseStep p;
  int stages;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the completion of phase `parity`; false after WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 1; i < (1u << 30); ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 63u) == 0 && gtimer() - t0 > WAIT_NS) return false;
  }
  return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

// 2-D tiled TMA load into this CTA's shared memory, completion counted on bar
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

// Shared-memory matrix descriptor of the tcgen05 family for a K-major operand
// in the 128-byte swizzled layout: start address, leading byte offset (unused
// for this layout, 16), stride byte offset 1024 (eight 128-byte rows), bit 46
// set, base offset 0 (atoms are 1024-byte aligned), layout type 2.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: D in FP32, A and B in BF16, both
// K-major, dense; N / 8 at bit 17, M / 16 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// the same MMA with the A operand (128 rows x 16 K, two BF16 per 32-bit
// column, K-major) read from tensor memory
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* out) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) out[i] = __uint_as_float(r[i]);
}

// 32 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void unpack8(uint4 q, float* y) {
  y[0] = bf16lo(q.x); y[1] = bf16hi(q.x); y[2] = bf16lo(q.y); y[3] = bf16hi(q.y);
  y[4] = bf16lo(q.z); y[5] = bf16hi(q.z); y[6] = bf16lo(q.w); y[7] = bf16hi(q.w);
}

template <bool MOM, bool LAP, int KS>
__global__ void __launch_bounds__(NTHREADS, 1) k_dense_step(const __grid_constant__ DenseArgs args) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[MAX_STAGES], empty[MAX_STAGES], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int sh_issued, sh_consumed, sh_timeout;
  const DenseStep& p = args.p;
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = (int)cluster.block_rank();
  const int m0 = (int)(blockIdx.x / KS) * BM;
  const int cbase = (int)blockIdx.y * 256;
  const int nt = min(256, p.cpad - cbase);   // MMA N of this column tile, a multiple of 32
  const int ntmax = min(256, p.cpad);        // rows of the YT box (the last tile's excess is zero-filled)
  const int S = args.stages;
  const int nk = p.kpad / BK;
  const int kb = (int)((int64_t)nk * r / KS), ke = (int)((int64_t)nk * (r + 1) / KS);
  const int nloc = ke - kb;   // >= 1 (the launcher keeps KS <= nk)
  const uint32_t a_bytes = BM * BK * 2;
  const uint32_t stage_bytes = a_bytes + (uint32_t)ntmax * BK * 2;
  const uint32_t base = (saddr(smem_raw) + 1023u) & ~1023u;   // swizzle atoms are 1024-byte aligned
  unsigned char* const sbase = smem_raw + (base - saddr(smem_raw));
  // two accumulators: D0 (columns [0, half)) sums the even chunks of the
  // contraction range, D1 ([half, 2 half)) the odd ones; the partial is D0 + D1
  const uint32_t half = nt <= 32 ? 32u : (nt <= 64 ? 64u : (nt <= 128 ? 128u : 256u));
  const uint32_t tmem_cols = 2 * half;
  constexpr int ROWS = BM / KS;   // rows of the tile updated by this CTA
  constexpr int OCT = ROWS / 8;   // 8-row vectors per column
  const int nvec = OCT * nt;
  const int i_base = m0 + r * ROWS;

  // y and V of this thread's first PF update vectors, loaded during the contraction
  uint4 ypf[PF];
  float4 vpf[PF][2];
  auto load_vectors = [&](int g0) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int vi = g0 + tid + NTHREADS * u;
      if (vi < nvec) {
        const size_t off = (size_t)(cbase + vi / OCT) * p.kpad + i_base + 8 * (vi % OCT);
        ypf[u] = __ldg(reinterpret_cast<const uint4*>(p.YT + off));
        if (MOM) {
          vpf[u][0] = *reinterpret_cast<const float4*>(p.VT + off);
          vpf[u][1] = *reinterpret_cast<const float4*>(p.VT + off + 4);
        }
      }
    }
  };
  load_vectors(0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh_issued = 0;
    sh_consumed = 0;
    sh_timeout = 0;
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&args.tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&args.tmY)) : "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool timed_out = false;

  if (tid == 0) {
    // TMA producer: chunk kc into stage kc % S once the MMAs of chunk kc - S have read it
    int kc = 0;
    for (; kc < nloc; ++kc) {
      const int s = kc % S;
      if (kc >= S && !mbar_wait(&empty[s], (uint32_t)(kc / S - 1) & 1u)) { timed_out = true; break; }
      const uint32_t sa = base + (uint32_t)s * stage_bytes;
      mbar_expect_tx(&full[s], stage_bytes);
      tma_load_2d(sa, &args.tmA, (kb + kc) * BK, m0, &full[s]);
      tma_load_2d(sa + a_bytes, &args.tmY, (kb + kc) * BK, cbase, &full[s]);
    }
    sh_issued = kc;
  } else if (tid == 32) {
    // MMA issuer
    const uint32_t idesc = idesc_bf16(BM, nt);
    int kc = 0;
    for (; kc < nloc; ++kc) {
      const int s = kc % S;
      if (!mbar_wait(&full[s], (uint32_t)(kc / S) & 1u)) { timed_out = true; break; }
      tc_fence_after();
      const uint32_t sa = base + (uint32_t)s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
      for (int q = 0; q < BK / 16; ++q)   // K = 16: 32 bytes along the swizzled 128-byte row
        mma_bf16(tmem + (uint32_t)(kc & 1) * half, desc_sw128(sa + 32u * q), desc_sw128(sb + 32u * q), idesc,
                 (kc > 1 || q > 0) ? 1u : 0u);
      mma_commit(&empty[s]);   // stage s is free once these MMAs have read it
    }
    sh_consumed = kc;
    mma_commit(&done);         // arrives once every MMA issued above has completed
  }
  __syncwarp();
  if (!mbar_wait(&done, 0)) timed_out = true;
  tc_fence_after();
  if (timed_out) atomicOr(&sh_timeout, 1);
  cluster.sync();   // #1: every accumulator of the cluster is complete, every ring is free
  if (tid == 0 && sh_timeout) {
    // a wait gave up: let this CTA's issued loads land before its memory is reused
    for (int kc = sh_consumed; kc < sh_issued; ++kc) (void)mbar_wait(&full[kc % S], (uint32_t)(kc / S) & 1u);
  }

  // push: row (TMEM lane) 32 warp + lane belongs to the CTA of rank row / ROWS;
  // it receives the partial in recv[src][c][row % ROWS] (floats)
  float* recv = reinterpret_cast<float*>(sbase);
  {
    const int row = warp * 32 + lane;
    float* dst = cluster.map_shared_rank(recv, row / ROWS) + (size_t)r * nt * ROWS + (row % ROWS);
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < nt; c0 += 32) {
      float g[32], g1[32];
      tmem_ld32(tl + (uint32_t)c0, g);
      if (nloc > 1) {
        tmem_ld32(tl + half + (uint32_t)c0, g1);
#pragma unroll
        for (int k = 0; k < 32; ++k) g[k] += g1[k];
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) dst[(size_t)(c0 + k) * ROWS] = g[k];
    }
  }
  tc_fence_before();
  cluster.sync();   // #2: every partial has arrived
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");

  // update: vector vi = (column c = vi / OCT, rows i_base + 8 (vi % OCT) .. + 7)
  bool bad = false;
  for (int g0 = 0;;) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int vi = g0 + tid + NTHREADS * u;
      if (vi >= nvec) continue;
      const int c = vi / OCT, o = vi % OCT;
      const int col = cbase + c;
      const int i0 = i_base + 8 * o;
      float acc[8];
      {
        const float4* src = reinterpret_cast<const float4*>(recv + (size_t)c * ROWS + 8 * o);
        float4 a0 = src[0], a1 = src[1];
        acc[0] = a0.x; acc[1] = a0.y; acc[2] = a0.z; acc[3] = a0.w;
        acc[4] = a1.x; acc[5] = a1.y; acc[6] = a1.z; acc[7] = a1.w;
#pragma unroll
        for (int q = 1; q < KS; ++q) {   // partial sums added in rank order
          const float4* sq = reinterpret_cast<const float4*>(recv + ((size_t)q * nt + c) * ROWS + 8 * o);
          a0 = sq[0];
          a1 = sq[1];
          acc[0] += a0.x; acc[1] += a0.y; acc[2] += a0.z; acc[3] += a0.w;
          acc[4] += a1.x; acc[5] += a1.y; acc[6] += a1.z; acc[7] += a1.w;
        }
      }
      float y[8], v[8];
      unpack8(ypf[u], y);
      if (MOM) {
        v[0] = vpf[u][0].x; v[1] = vpf[u][0].y; v[2] = vpf[u][0].z; v[3] = vpf[u][0].w;
        v[4] = vpf[u][1].x; v[5] = vpf[u][1].y; v[6] = vpf[u][1].z; v[7] = vpf[u][1].w;
      }
      const bool active = col < p.C && (!p.steps_cols || p.t < p.steps_cols[col]);
      const float alpha = p.alpha_cols ? p.afac * p.alpha_cols[col < p.C ? col : 0] : p.alpha;
      float out[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        // rows >= n: y, V and the row of A are zero, so the new value is zero as well
        const float dr = (LAP && i0 + k < p.n) ? __ldg(p.dnet + i0 + k) : 0.0f;
        const float grad = LAP ? fmaf(dr, y[k], -acc[k]) : -acc[k];
        const float step = MOM ? fmaf(p.mu, v[k], grad) : grad;
        float yn = fmaf(alpha, step, y[k]);
        if (active && !isfinite(yn)) bad = true;
        yn = fminf(fmaxf(yn, -1.0f), 1.0f);
        out[k] = active ? yn : y[k];
        if (MOM) v[k] = step;
      }
      const size_t off = (size_t)col * p.kpad + i0;
      *reinterpret_cast<uint4*>(p.YTout + off) =
          make_uint4(pack_bf16x2(out[0], out[1]), pack_bf16x2(out[2], out[3]), pack_bf16x2(out[4], out[5]),
                     pack_bf16x2(out[6], out[7]));
      if (MOM && active) {
        *reinterpret_cast<float4*>(p.VT + off) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(p.VT + off + 4) = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
    g0 += NTHREADS * PF;
    if (g0 >= nvec) break;
    load_vectors(g0);
  }
  if (p.flag && (bad || timed_out)) atomicOr(p.flag, (bad ? 1 : 0) | (timed_out ? 2 : 0));
}

// ---------------------------------------------------------------- persistent phase kernel
//
// All steps of a phase in one cooperative cluster launch (every CTA resident).
// Warp 0 lane 0 loads (TMA); warp 1 lane 0 issues the MMAs of the even chunks
// of the contraction range into accumulator D0, warp 2 lane 0 those of the odd
// chunks into D1 (so the wait for one chunk's tiles overlaps the other
// issuer's MMAs); warps 3-10 run the update on D0 + D1 (two warps per lane
// quarter of tensor memory, each on half of the columns); the stage ring runs
// on across steps.  Between steps a grid barrier
// (a counter in global memory, bounded spin) orders the new YT of every CTA
// before the next step's B tiles are loaded; the A tiles of the next step are
// requested before that barrier, as A does not change.  The y and V of the
// update vectors stay in registers for the whole phase (V is written back at
// the end); the CTA's partial product is staged in shared memory as one block
// per owning CTA and sent with one bulk shared-memory copy per peer, whose
// bytes complete the owner's receive barrier.

constexpr int P_UPD = 256;       // update threads (warps 3 - 10: two warps per tensor-memory lane quarter)
constexpr int PT = 96 + P_UPD;   // threads of the phase kernel
constexpr int PNV = 4;           // update vectors per thread at most
constexpr int P_MAX_SB = 16;     // B stages (one YT tile each)
constexpr int P_MAX_SA = 5;      // A stages (the streamed A tiles)
constexpr int P_RESIDENT = 8;    // A chunks kept in tensor memory (8 x 32 columns + two 128-column accumulators)

struct PhaseArgs {
  CUtensorMap tmA;
  CUtensorMap tmY[2];
  DenseStep p;                   // YT / YTout unused: the phase ping-pongs yt[0] / yt[1]
  __nv_bfloat16* yt[2];
  const __nv_bfloat16* A;        // the dense A (kpad x kpad), for the chunks kept in tensor memory
  unsigned int* gbar;            // grid barrier counter, zero at launch
  int32_t resident;              // contraction chunks of A kept in tensor memory (the last ones of the range)
  int32_t steps;
  int32_t w;                     // column tile width (multiple of 32, <= 128)
  int32_t sb, sa;                // B and A stage counts
  int32_t ncta;
};

__device__ __forceinline__ bool mbar_try_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  if (mbar_try_cluster(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 1; i < (1u << 30); ++i) {
    if (mbar_try_cluster(bar, parity)) return true;
    if ((i & 63u) == 0 && gtimer() - t0 > WAIT_NS) return false;
  }
  return false;
}
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
// bulk copy of `bytes` from this CTA's shared memory into a peer's; the bytes
// complete the peer's mbarrier (both given as shared::cluster addresses)
__device__ __forceinline__ void bulk_to_peer(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "r"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
// named barrier over `threads` threads that also ORs a predicate across them
// (every update thread leaves a step on the same decision)
__device__ __forceinline__ bool named_sync_or(int id, int threads, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(threads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ uint32_t ld_acquire(const unsigned int* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// wait until the grid barrier counter reaches target; false after WAIT_NS
__device__ __forceinline__ bool grid_wait(const unsigned int* gbar, uint32_t target) {
  bool ok = ld_acquire(gbar) >= target;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 0; !ok && i < (1u << 30); ++i) {
    ok = ld_acquire(gbar) >= target;
    if ((i & 63u) == 0 && gtimer() - t0 > WAIT_NS) break;
  }
  return ok;
}

template <bool MOM, bool LAP, int KS>
__global__ void __launch_bounds__(PT, 1) k_dense_phase(const __grid_constant__ PhaseArgs args) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[P_MAX_SB], empty[P_MAX_SB], emptyA[P_MAX_SA], done, recv_full, out_free,
      drain[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int sh_timeout;
  const DenseStep& p = args.p;
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = (int)cluster.block_rank();
  const int m0 = (int)(blockIdx.x / KS) * BM;
  const int W = args.w;
  const int cbase = (int)blockIdx.y * W;
  const int nt = min(W, p.cpad - cbase);   // MMA N of this column tile, a multiple of 32
  const int SB = args.sb, SA = args.sa;
  const int nk = p.kpad / BK;
  const int kb = (int)((int64_t)nk * r / KS), ke = (int)((int64_t)nk * (r + 1) / KS);
  const int nloc = ke - kb;
  const uint32_t a_bytes = BM * BK * 2;
  const uint32_t b_bytes = (uint32_t)W * BK * 2;
  // shared memory: B ring (SB x b_bytes), A ring (SA x a_bytes), receive area;
  // the partial-product staging `out` reuses the rings between steps
  const uint32_t base = (saddr(smem_raw) + 1023u) & ~1023u;
  unsigned char* const sbase = smem_raw + (base - saddr(smem_raw));
  const uint32_t abase = base + (uint32_t)SB * b_bytes;
  constexpr int ROWS = BM / KS;
  constexpr int OCT = ROWS / 8;
  const uint32_t blk_bytes = (uint32_t)W * ROWS * 4;                       // one owner's share of the partial
  float* const out = reinterpret_cast<float*>(sbase);                                      // [KS][W][ROWS]
  float* const recv = reinterpret_cast<float*>(sbase + (size_t)SB * b_bytes + (size_t)SA * a_bytes);   // [KS-1][W][ROWS]
  // tensor memory: accumulators D0 (columns [0, half)) and D1 ([half, 2 half));
  // chunks [kr, nloc) keep their A tile in it for the whole phase: columns
  // 256 + 32 c (64 BF16 per row, two per column) hold chunk kr + c
  const int R = min(args.resident, nloc);
  const int kr = nloc - R;
  const uint32_t half = R > 0 ? 128u : (nt <= 32 ? 32u : (nt <= 64 ? 64u : 128u));
  const uint32_t tmem_cols = R > 0 ? 512u : 2u * half;
  const int nvec = OCT * nt;
  const int i_base = m0 + r * ROWS;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < SB; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < SA; ++s) mbar_init(&emptyA[s], 1);
    mbar_init(&done, nloc > 1 ? 2 : 1);   // one commit per issuer with chunks
    mbar_init(&recv_full, 1);
    mbar_init(&out_free, 1);   // the update warps are done with `out` (ring memory) for the step
    mbar_init(&drain[0], 1);   // give-up path: an MMA issuer's last commit
    mbar_init(&drain[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh_timeout = 0;
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&args.tmA)) : "memory");
  }
  tc_fence_before();
  cluster.sync();   // barriers initialised and every CTA of the cluster running
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool timed_out = false;
  if (R > 0 && warp >= 3) {
    // the resident A tiles: row (TMEM lane) 32 quarter + lane, straight from
    // global memory; the two warps of a quarter take alternate chunks
    const int quarter = warp & 3, row = quarter * 32 + lane, colhalf = (warp - 3) >> 2;
    const __nv_bfloat16* arow = args.A + (size_t)(m0 + row) * p.kpad;
    for (int c = colhalf; c < R; c += 2) {
      uint32_t v[32];
      const uint4* src = reinterpret_cast<const uint4*>(arow + (size_t)(kb + kr + c) * BK);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint4 q = __ldg(src + k);
        v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
      }
      tmem_st32(tmem + ((uint32_t)(quarter * 32) << 16) + 256u + 32u * (uint32_t)c, v);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();   // the resident tiles are in place before any MMA
  tc_fence_after();

  if (tid == 0) {
    // ---------------- TMA producer.  The chunks of a phase take the B stages
    // in turn (and the streamed ones the A stages in turn); slot and round
    // advance by one per chunk, the stage of round u is free once the MMAs of
    // its round u - 1 have completed (phase (u - 1) & 1 of its empty barrier).
    int bslot = 0, bround = 0, aslot = 0, around = 0;
    int pre_slot[P_MAX_SB];
    // per B stage: round of the last phase of full[s] armed with expect_tx
    // (-1: never), and the x coordinate of a B tile counted in that phase but
    // not requested yet (-1: none) -- what the give-up path must complete
    int last_round[P_MAX_SB], pend_x[P_MAX_SB];
    for (int q = 0; q < P_MAX_SB; ++q) last_round[q] = pend_x[q] = -1;
    int t = 0;
    for (; t < args.steps && !timed_out; ++t) {
      const CUtensorMap* tmY = &args.tmY[t & 1];
      // the rings also hold `out` between steps: wait until the update of step t-1 is done with it
      if (t > 0 && !mbar_wait(&out_free, (uint32_t)(t - 1) & 1u)) { timed_out = true; break; }
      auto acquire = [&](int kc, int& bs) -> bool {   // the chunk's stages are free, its bytes expected
        bs = bslot;
        const int rnd = bround;
        if (bround > 0 && !mbar_wait(&empty[bslot], (uint32_t)(bround - 1) & 1u)) return false;
        if (++bslot == SB) { bslot = 0; ++bround; }
        if (kc < kr) {
          if (around > 0 && !mbar_wait(&emptyA[aslot], (uint32_t)(around - 1) & 1u)) return false;
          mbar_expect_tx(&full[bs], a_bytes + b_bytes);
          tma_load_2d(abase + (uint32_t)aslot * a_bytes, &args.tmA, (kb + kc) * BK, m0, &full[bs]);
          if (++aslot == SA) { aslot = 0; ++around; }
        } else {
          mbar_expect_tx(&full[bs], b_bytes);
        }
        last_round[bs] = rnd;
        pend_x[bs] = (kb + kc) * BK;
        return true;
      };
      // A tiles of the first streamed chunks: no dependence on the new iterate
      const int pre = min(min(SB, nloc), min(SA, kr));
      for (int kc = 0; kc < pre && !timed_out; ++kc)
        if (!acquire(kc, pre_slot[kc])) timed_out = true;
      if (timed_out) break;
      if (t > 0) {
        // grid barrier: every CTA has written its rows of the iterate of step t
        if (!grid_wait(args.gbar, (uint32_t)args.ncta * (uint32_t)t)) { timed_out = true; break; }
        asm volatile("fence.proxy.async.global;" ::: "memory");   // generic writes -> TMA reads
      }
      for (int kc = 0; kc < nloc; ++kc) {
        int bs = 0;
        if (kc < pre) bs = pre_slot[kc];
        else if (!acquire(kc, bs)) { timed_out = true; break; }
        tma_load_2d(base + (uint32_t)bs * b_bytes, tmY, (kb + kc) * BK, cbase, &full[bs]);
        pend_x[bs] = -1;
      }
    }
    if (timed_out) {
      // Give-up path.  A stage armed for a B tile that was never requested
      // (the wait for the grid barrier or a stage gave up in between) would
      // never complete: request the tile now (an in-bounds read whose bytes
      // are discarded).  Then wait for the last armed phase of every stage,
      // so that no TMA write into this CTA's shared memory is in flight when
      // the CTA releases it.
      const int tl = t < args.steps ? t : args.steps - 1;
      for (int q = 0; q < SB; ++q)
        if (pend_x[q] >= 0) tma_load_2d(base + (uint32_t)q * b_bytes, &args.tmY[tl & 1], pend_x[q], cbase, &full[q]);
      for (int q = 0; q < SB; ++q)
        if (last_round[q] >= 0) (void)mbar_wait(&full[q], (uint32_t)last_round[q] & 1u);
    }
  } else if (tid == 32 || (tid == 64 && nloc > 1)) {
    // ---------------- MMA issuers (the same slot / round walk as the producer;
    // issuer `my` takes the chunks kc with kc % 2 == my, into D_my; a range of
    // one chunk has one issuer, an idle one would run ahead of the steps)
    const int my = tid == 64 ? 1 : 0;
    const uint32_t d = tmem + (uint32_t)my * half;
    const uint32_t idesc = idesc_bf16(BM, nt);
    int bslot = 0, bround = 0, aslot = 0;
    for (int t = 0; t < args.steps && !timed_out; ++t) {
      for (int kc = 0; kc < nloc; ++kc) {
        const int s = bslot, rnd = bround, as_ = aslot;
        if (++bslot == SB) { bslot = 0; ++bround; }
        if (kc < kr && ++aslot == SA) aslot = 0;
        if ((kc & 1) != my) continue;
        if (!mbar_wait(&full[s], (uint32_t)rnd & 1u)) { timed_out = true; break; }
        tc_fence_after();
        const uint32_t sb = base + (uint32_t)s * b_bytes;
        if (kc < kr) {
          const uint32_t as = abase + (uint32_t)as_ * a_bytes;
#pragma unroll
          for (int q = 0; q < BK / 16; ++q)
            mma_bf16(d, desc_sw128(as + 32u * q), desc_sw128(sb + 32u * q), idesc, (kc > 1 || q > 0) ? 1u : 0u);
          mma_commit(&emptyA[as_]);
        } else {
          const uint32_t at = tmem + 256u + 32u * (uint32_t)(kc - kr);   // K = 16: 8 columns
#pragma unroll
          for (int q = 0; q < BK / 16; ++q)
            mma_bf16_ta(d, at + 8u * q, desc_sw128(sb + 32u * q), idesc, (kc > 1 || q > 0) ? 1u : 0u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&done);   // phase t of `done` completes with both issuers' accumulators of step t
    }
    if (timed_out) {
      // give-up path: every MMA this thread issued has completed (its writes
      // to tensor memory and its reads of the stages) before the teardown
      mma_commit(&drain[my]);
      (void)mbar_wait(&drain[my], 0u);
    }
  } else if (warp >= 3) {
    // ---------------- update warps: et = row-vector owner index, quarter = TMEM lanes
    const int et = tid - 96;
    const int quarter = warp & 3;
    const int colhalf = (warp - 3) >> 2;   // which 32-column chunks of the accumulator this warp stages
    const int row = quarter * 32 + lane;   // tile row read from tensor memory
    const int qown = row / ROWS;
    uint4 yr[PNV];
    float vr[PNV][8];
    float acol[PNV];
    int32_t scol[PNV];
#pragma unroll
    for (int u = 0; u < PNV; ++u) {
      const int vi = et + P_UPD * u;
      yr[u] = make_uint4(0, 0, 0, 0);
      acol[u] = 0.0f;
      scol[u] = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) vr[u][k] = 0.0f;
      if (vi < nvec) {
        const int col = cbase + vi / OCT;
        const size_t off = (size_t)col * p.kpad + i_base + 8 * (vi % OCT);
        yr[u] = *reinterpret_cast<const uint4*>(args.yt[0] + off);
        if (MOM) {
          const float4 a = *reinterpret_cast<const float4*>(p.VT + off);
          const float4 b = *reinterpret_cast<const float4*>(p.VT + off + 4);
          vr[u][0] = a.x; vr[u][1] = a.y; vr[u][2] = a.z; vr[u][3] = a.w;
          vr[u][4] = b.x; vr[u][5] = b.y; vr[u][6] = b.z; vr[u][7] = b.w;
        }
        acol[u] = p.alpha_cols ? p.afac * p.alpha_cols[col < p.C ? col : 0] : p.alpha;
        scol[u] = col < p.C ? (p.steps_cols ? p.steps_cols[col] : INT32_MAX) : -1;   // -1: padding column
      }
    }
    bool bad = false;
    for (int t = 0; t < args.steps && !timed_out; ++t) {
      if (KS > 1 && et == 0) mbar_expect_tx(&recv_full, (uint32_t)(KS - 1) * blk_bytes);
      if (named_sync_or(1, P_UPD, !mbar_wait(&done, (uint32_t)t & 1u))) { timed_out = true; break; }
      tc_fence_after();
      // accumulator -> out[owner][c][row % ROWS]
      {
        float* dst = out + (size_t)qown * W * ROWS + (row % ROWS);
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        for (int c0 = 32 * colhalf; c0 < nt; c0 += 64) {
          float gv[32], g1[32];
          tmem_ld32(tl + (uint32_t)c0, gv);
          if (nloc > 1) {   // D0 + D1
            tmem_ld32(tl + half + (uint32_t)c0, g1);
#pragma unroll
            for (int k = 0; k < 32; ++k) gv[k] += g1[k];
          }
#pragma unroll
          for (int k = 0; k < 32; ++k) dst[(size_t)(c0 + k) * ROWS] = gv[k];
        }
      }
      tc_fence_before();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staged rows -> bulk copy reads
      named_sync(1, P_UPD);
      if (KS > 1 && et == 0) {
        for (int q = 0; q < KS; ++q) {
          if (q == r) continue;
          const int slot = r < q ? r : r - 1;   // this CTA's slot in q's receive area
          bulk_to_peer(mapa(saddr(recv + (size_t)slot * W * ROWS), (uint32_t)q),
                       saddr(out + (size_t)q * W * ROWS), blk_bytes, mapa(saddr(&recv_full), (uint32_t)q));
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
      if (KS > 1 && named_sync_or(1, P_UPD, !mbar_wait_cluster(&recv_full, (uint32_t)t & 1u))) {
        timed_out = true;
        break;
      }
      __nv_bfloat16* YTo = args.yt[(t + 1) & 1];
#pragma unroll
      for (int u = 0; u < PNV; ++u) {
        const int vi = et + P_UPD * u;
        if (vi >= nvec) continue;
        const int c = vi / OCT, o = vi % OCT;
        float acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
#pragma unroll
        for (int q = 0; q < KS; ++q) {   // partial sums added in rank order
          const float* src = q == r ? out + ((size_t)r * W + c) * ROWS + 8 * o
                                    : recv + ((size_t)(q < r ? q : q - 1) * W + c) * ROWS + 8 * o;
          const float4 a0 = reinterpret_cast<const float4*>(src)[0];
          const float4 a1 = reinterpret_cast<const float4*>(src)[1];
          if (q == 0) {
            acc[0] = a0.x; acc[1] = a0.y; acc[2] = a0.z; acc[3] = a0.w;
            acc[4] = a1.x; acc[5] = a1.y; acc[6] = a1.z; acc[7] = a1.w;
          } else {
            acc[0] += a0.x; acc[1] += a0.y; acc[2] += a0.z; acc[3] += a0.w;
            acc[4] += a1.x; acc[5] += a1.y; acc[6] += a1.z; acc[7] += a1.w;
          }
        }
        const int i0 = i_base + 8 * o;
        float y[8];
        unpack8(yr[u], y);
        const bool active = t < scol[u];
        float outv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          // rows >= n: y, V and the row of A are zero, so the new value is zero as well
          const float dr = (LAP && i0 + k < p.n) ? __ldg(p.dnet + i0 + k) : 0.0f;
          const float grad = LAP ? fmaf(dr, y[k], -acc[k]) : -acc[k];
          const float step = MOM ? fmaf(p.mu, vr[u][k], grad) : grad;
          float yn = fmaf(acol[u], step, y[k]);
          if (active && !isfinite(yn)) bad = true;
          yn = fminf(fmaxf(yn, -1.0f), 1.0f);
          outv[k] = active ? yn : y[k];
          if (MOM && active) vr[u][k] = step;
        }
        yr[u] = make_uint4(pack_bf16x2(outv[0], outv[1]), pack_bf16x2(outv[2], outv[3]),
                           pack_bf16x2(outv[4], outv[5]), pack_bf16x2(outv[6], outv[7]));
        *reinterpret_cast<uint4*>(YTo + (size_t)(cbase + c) * p.kpad + i0) = yr[u];
      }
      if (KS > 1 && et == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // `out` reusable
      asm volatile("fence.proxy.async.global;" ::: "memory");   // new rows -> the next step's TMA reads
      named_sync(1, P_UPD);
      if (et == 0 && t + 1 < args.steps) {
        mbar_arrive_local(&out_free);   // the rings may take the next step's tiles
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(args.gbar) : "memory");
      }
    }
    if (MOM) {
#pragma unroll
      for (int u = 0; u < PNV; ++u) {
        const int vi = et + P_UPD * u;
        if (vi >= nvec || scol[u] < 0) continue;
        const size_t off = (size_t)(cbase + vi / OCT) * p.kpad + i_base + 8 * (vi % OCT);
        *reinterpret_cast<float4*>(p.VT + off) = make_float4(vr[u][0], vr[u][1], vr[u][2], vr[u][3]);
        *reinterpret_cast<float4*>(p.VT + off + 4) = make_float4(vr[u][4], vr[u][5], vr[u][6], vr[u][7]);
      }
    }
    if (p.flag && bad) atomicOr(p.flag, 1);
  }
  // The exchange's issuing thread waits until its bulk copies have been
  // written into the peers (not only read here): once every CTA of the
  // cluster has passed the cluster barrier below, no copy into any of them is
  // in flight.  The producer and the MMA issuers drained their own loads and
  // MMAs above on the give-up path, so tensor memory and shared memory are
  // quiet when they are released.
  if (tid == 96) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  __syncwarp();
  if (timed_out) atomicOr(&sh_timeout, 1);
  __syncthreads();
  if (sh_timeout && tid == 0 && p.flag) atomicOr(p.flag, 2);
  tc_fence_before();
  cluster.sync();   // no peer copies into this CTA any more
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---- dense copy of A: one warp per row
__global__ void k_dense_from_csr(int32_t n, int32_t kpad, int wmode, const int32_t* row_ptr,
                                 const int32_t* col_idx, const uint32_t* col_sw, const float* w,
                                 __nv_bfloat16* A) {
  const int32_t v = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= n) return;
  for (int32_t e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) {
    int32_t j;
    float wt;
    if (wmode == W_SIGN) {
      const uint32_t s = col_sw[e];
      j = (int32_t)(s & 0x7FFFFFFFu);
      wt = (s & 0x80000000u) ? -1.0f : 1.0f;
    } else {
      j = col_idx[e];
      wt = wmode == W_GENERAL ? w[e] : 1.0f;
    }
    A[(size_t)v * kpad + j] = __float2bfloat16_rn(wt);
  }
}

// out (cols x ldout) = in (rows x cols, row stride ldin) transposed
template <typename T>
__global__ void k_transpose(int32_t rows, int32_t cols, const T* in, int32_t ldin, T* out, int32_t ldout) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int rr = by + j, c = bx + threadIdx.x;
    if (rr < rows && c < cols) tile[j][threadIdx.x] = in[(size_t)rr * ldin + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int orow = bx + j, ocol = by + threadIdx.x;   // out row = in column
    if (orow < cols && ocol < rows) out[(size_t)orow * ldout + ocol] = tile[threadIdx.x][j];
  }
}

template <typename T>
int transpose(int32_t rows, int32_t cols, const T* in, int32_t ldin, T* out, int32_t ldout, cudaStream_t st) {
  if (rows == 0 || cols == 0) return DECO_OK;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)), block(32, 8);
  k_transpose<T><<<grid, block, 0, st>>>(rows, cols, in, ldin, out, ldout);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

// largest dynamic shared memory enabled per kernel instance [MOM][LAP][log2 KS]
std::atomic<int> g_smem_set[2][2][4];

using KernelFn = void (*)(DenseArgs);

template <bool MOM, bool LAP>
KernelFn pick_ks(int ks) {
  switch (ks) {
    case 1: return k_dense_step<MOM, LAP, 1>;
    case 2: return k_dense_step<MOM, LAP, 2>;
    case 4: return k_dense_step<MOM, LAP, 4>;
    default: return k_dense_step<MOM, LAP, 8>;
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
  });
  return fn;
}

// BF16 matrix of `rows` x `cols` (row stride cols), boxes of 64 columns x box_rows rows, 128-byte swizzle
int make_map(CUtensorMap* m, const void* base, int32_t cols, int32_t rows, int32_t box_rows) {
  EncodeTiled enc = encode_tiled();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return DECO_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a %d x %d BF16 matrix", (int)r, rows, cols);
    return DECO_ERR_CUDA;
  }
  return DECO_OK;
}

int stages_for(int ntmax) {
  const uint32_t stage = (uint32_t)BM * BK * 2 + (uint32_t)ntmax * BK * 2;
  return std::max(2, std::min(MAX_STAGES, (int)(RING_BUDGET / stage)));
}

// Wait-timeout probe: the kernels' own bounded waits on something that never
// completes -- (0) a CTA mbarrier nobody arrives at, (1) the grid barrier
// counter nobody increments.  The wait gives up after WAIT_NS and the kernel
// reports it in bit 1 of *flag, as the dense kernels do.
__global__ void k_probe_wait(int which, unsigned int* counter, int32_t* flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  bool ok;
  if (which == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ok = mbar_wait(&bar, 0);
  } else {
    ok = grid_wait(counter, 1u);
  }
  if (!ok) atomicOr(flag, 2);
}

}  // namespace

int dense_make_maps(const __nv_bfloat16* A, int32_t kpad, __nv_bfloat16* const yt[2], int32_t cpad, int w,
                    DenseMaps* maps) {
  int rc = make_map(&maps->a, A, kpad, kpad, BM);
  for (int i = 0; i < 2 && rc == DECO_OK; ++i) rc = make_map(&maps->y[i], yt[i], kpad, cpad, std::min(256, cpad));
  for (int i = 0; i < 2 && rc == DECO_OK && w > 0; ++i) rc = make_map(&maps->yw[i], yt[i], kpad, cpad, w);
  return rc;
}

int dense_phase_shape(int32_t kpad, int32_t cpad, int ks, int w, DensePhaseShape* out) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    optin = 227 * 1024;
  }
  const int rows = BM / ks;
  const size_t out_b = (size_t)ks * w * rows * 4, recv_b = (size_t)(ks - 1) * w * rows * 4;
  const size_t a_st = (size_t)BM * BK * 2, b_st = (size_t)w * BK * 2;
  const long long room = (long long)optin - 1024 - 512 - (long long)recv_b;
  const int nk = kpad / BK;
  if (w < 32 || w > 128 || w % 32 || ks > nk || (ks & (ks - 1)) || ks > 8 || (w + 16 * ks - 1) / (16 * ks) > PNV ||
      room <= 0) {
    set_error("dense phase kernel: no shape for w=%d ks=%d", w, ks);
    return DECO_ERR_UNSUPPORTED;
  }
  // the streamed chunks (nk/ks - P_RESIDENT at most) take up to five A stages
  // (measured at n = 4096, C = 128, ks = 4: 2 / 3 / 4 / 5 / 8 stages give
  // 10.5 / 10.0 / 9.6 / 9.5 / 10.2 us per step); the rest goes to B stages
  const int streamed = std::max(0, nk / ks - P_RESIDENT);
  const int SA = std::max(1, std::min(P_MAX_SA, streamed));
  const long long left = room - (long long)SA * (long long)a_st;
  const int SB = left > 0 ? (int)std::min<long long>(P_MAX_SB, left / (long long)b_st) : 0;
  if (SB < 2 || (size_t)SB * b_st + (size_t)SA * a_st < out_b) {
    set_error("dense phase kernel: no shape for w=%d ks=%d", w, ks);
    return DECO_ERR_UNSUPPORTED;
  }
  out->w = w;
  out->ks = ks;
  out->stages = SB;
  out->stages_a = SA;
  out->smem = (size_t)SB * b_st + (size_t)SA * a_st + recv_b + 1024;
  out->ctas = kpad / BM * ks * ((cpad + w - 1) / w);
  return DECO_OK;
}

int dense_build(const deco_graph* g, int32_t kpad, __nv_bfloat16** out, cudaStream_t st) {
  const size_t bytes = (size_t)kpad * kpad * 2;
  __nv_bfloat16* A = nullptr;
  cudaError_t e = cudaMalloc((void**)&A, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(dense adjacency)");
  e = cudaMemsetAsync(A, 0, bytes, st);
  if (e == cudaSuccess && g->n > 0) {
    const int64_t threads = (int64_t)g->n * 32;
    k_dense_from_csr<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g->n, kpad, g->wmode, g->row_ptr,
                                                                        g->col_idx, g->col_sw, g->w, A);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the copy outlives this stream's ordering
  if (e != cudaSuccess) {
    cudaFree(A);
    return cuda_fail(e, "dense adjacency");
  }
  *out = A;
  return DECO_OK;
}

int dense_to_t(const void* y, int32_t n, int32_t ld, int32_t C, void* yt, int32_t kpad, size_t esz,
               cudaStream_t st) {
  if (esz == 2)
    return transpose<uint16_t>(n, C, static_cast<const uint16_t*>(y), ld, static_cast<uint16_t*>(yt), kpad, st);
  return transpose<uint32_t>(n, C, static_cast<const uint32_t*>(y), ld, static_cast<uint32_t*>(yt), kpad, st);
}

int dense_from_t(const void* yt, int32_t kpad, int32_t C, void* y, int32_t n, int32_t ld, size_t esz,
                 cudaStream_t st) {
  if (esz == 2)
    return transpose<uint16_t>(C, n, static_cast<const uint16_t*>(yt), kpad, static_cast<uint16_t*>(y), ld, st);
  return transpose<uint32_t>(C, n, static_cast<const uint32_t*>(yt), kpad, static_cast<uint32_t*>(y), ld, st);
}

namespace {

using PhaseFn = void (*)(PhaseArgs);

template <bool MOM, bool LAP>
PhaseFn pick_phase(int ks) {
  switch (ks) {
    case 1: return k_dense_phase<MOM, LAP, 1>;
    case 2: return k_dense_phase<MOM, LAP, 2>;
    case 4: return k_dense_phase<MOM, LAP, 4>;
    default: return k_dense_phase<MOM, LAP, 8>;
  }
}

std::atomic<int> g_phase_smem[2][2][4];

}  // namespace

int launch_dense_phase(const DenseStep& p, const DenseMaps& maps, __nv_bfloat16* const yt[2],
                       const DensePhaseShape& sh, int32_t steps, unsigned int* gbar, cudaStream_t st) {
  if (steps <= 0) return DECO_OK;
  const bool mom = p.mu != 0.0f, lap = p.objective == DECO_OBJ_LAPLACIAN;
  PhaseFn fn = mom ? (lap ? pick_phase<true, true>(sh.ks) : pick_phase<true, false>(sh.ks))
                   : (lap ? pick_phase<false, true>(sh.ks) : pick_phase<false, false>(sh.ks));
  const int lk = sh.ks == 1 ? 0 : (sh.ks == 2 ? 1 : (sh.ks == 4 ? 2 : 3));
  std::atomic<int>& set = g_phase_smem[mom][lap][lk];
  if (set.load() < (int)sh.smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    if (e != cudaSuccess) return cuda_fail(e, "dense phase shared memory");
    set.store((int)sh.smem);
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(p.kpad / BM * sh.ks), (unsigned)((p.cpad + sh.w - 1) / sh.w), 1);
  cfg.blockDim = dim3(PT, 1, 1);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sh.ks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // every CTA waits on every other between steps: all of them must be resident at once
  int clusters = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg);
  if (e != cudaSuccess || (int64_t)clusters * sh.ks < sh.ctas) {
    cudaGetLastError();
    set_error("dense phase kernel: %d CTAs cannot all be resident (%d clusters of %d)", sh.ctas, clusters, sh.ks);
    return DECO_ERR_UNSUPPORTED;
  }
  PhaseArgs args;
  args.tmA = maps.a;
  args.tmY[0] = maps.yw[0];
  args.tmY[1] = maps.yw[1];
  args.p = p;
  args.yt[0] = yt[0];
  args.yt[1] = yt[1];
  args.A = p.A;
  args.resident = p.A && sh.w <= 128 ? P_RESIDENT : 0;
  args.gbar = gbar;
  args.steps = steps;
  args.w = sh.w;
  args.sb = sh.stages;
  args.sa = sh.stages_a;
  args.ncta = sh.ctas;
  if ((e = cudaMemsetAsync(gbar, 0, sizeof(unsigned int), st)) != cudaSuccess) return cuda_fail(e, "memset");
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelEx(&cfg, fn, args);
  if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported || e == cudaErrorNotPermitted) {
    // The grid barrier needs every CTA resident at once, which only the
    // cooperative launch guarantees (the occupancy figure above is a bound,
    // not a promise on a GPU shared with other work): without it the caller
    // runs the per-step kernel instead.
    cudaGetLastError();
    set_error("dense phase kernel: the cooperative cluster launch was refused (%s)", cudaGetErrorString(e));
    return DECO_ERR_UNSUPPORTED;
  }
  if (e != cudaSuccess) return cuda_fail(e, "dense phase launch");
  return DECO_OK;
}

int launch_dense_step(const DenseStep& p, const DenseMaps& maps, int which, cudaStream_t st) {
  const int nk = p.kpad / BK;
  if (p.kpad % BM || p.cpad % 32 || p.cpad < 32 || p.ks < 1 || p.ks > 8 || (p.ks & (p.ks - 1)) || p.ks > nk ||
      (which & ~1)) {
    set_error("dense step: bad shape (kpad=%d cpad=%d ks=%d)", p.kpad, p.cpad, p.ks);
    return DECO_ERR_ARG;
  }
  const int ntmax = std::min(256, p.cpad);
  const int S = stages_for(ntmax);
  const size_t smem = (size_t)S * ((size_t)BM * BK * 2 + (size_t)ntmax * BK * 2) + 1024;   // + alignment slack
  const bool mom = p.mu != 0.0f, lap = p.objective == DECO_OBJ_LAPLACIAN;
  KernelFn fn = mom ? (lap ? pick_ks<true, true>(p.ks) : pick_ks<true, false>(p.ks))
                    : (lap ? pick_ks<false, true>(p.ks) : pick_ks<false, false>(p.ks));
  const int lk = p.ks == 1 ? 0 : (p.ks == 2 ? 1 : (p.ks == 4 ? 2 : 3));
  std::atomic<int>& set = g_smem_set[mom][lap][lk];
  if (set.load() < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "dense step shared memory");
    set.store((int)smem);
  }
  DenseArgs args;
  args.tmA = maps.a;
  args.tmY = maps.y[which];
  args.p = p;
  args.stages = S;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(p.kpad / BM * p.ks), (unsigned)((p.cpad + 255) / 256), 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)p.ks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, fn, args);
  if (e != cudaSuccess) return cuda_fail(e, "dense step launch");
  return DECO_OK;
}

int launch_wait_probe_dense(int which, unsigned int* counter, int32_t* flag, cudaStream_t st) {
  k_probe_wait<<<1, 32, 0, st>>>(which, counter, flag);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DECO_OK : cuda_fail(e, "wait probe launch");
}

}  // namespace deco
