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
// YT.  Tiles are staged in shared memory in the no-swizzle K-major layout
// (8-row x 16-byte core matrices, core (r/8, k/8) at (r/8) * 1024 + (k/8) *
// 128 bytes) by cp.async through a four-stage ring; one thread issues the
// MMAs (M = 128, N <= 256, K = 16 each) and commits every stage to an
// mbarrier that frees it for the next load.
//
// Grid: (row tiles x ks) CTAs along x, column tiles of <= 256 along y.  The ks
// CTAs of a cluster split the contraction of one 128 x N output tile; each
// moves its partial product from tensor memory to shared memory, the cluster
// synchronises, and CTA r reduces rows [r 128/ks, (r+1) 128/ks) over the ks
// partials (rank order, through distributed shared memory) and applies the
// update.  Every mbarrier wait is bounded (globaltimer); the accumulator's
// tensor-memory columns are released on every path.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "dense_tc.cuh"

namespace cg = cooperative_groups;

namespace deco {
namespace {

constexpr int BM = DENSE_BM, BK = DENSE_BK, STAGES = 4, NTHREADS = 128;
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s per wait at most

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

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory matrix descriptor of the tcgen05 family: start address,
// leading-dimension byte offset (between core matrices along K), stride byte
// offset (between 8-row groups), all in 16-byte units; bit 46 set; base
// offset 0; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
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

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One stage: A rows [m0, m0+128) x k [k0, k0+64) and YT rows [0, nt) x the
// same k, each 16-byte chunk (row r, k-group q) at (r/8) 1024 + q 128 + (r%8) 16.
__device__ __forceinline__ void load_stage(unsigned char* sA, unsigned char* sB, const __nv_bfloat16* A,
                                           int32_t kpad, const __nv_bfloat16* YT, int m0, int k0, int nt,
                                           int tid) {
  for (int i = tid; i < BM * (BK / 8); i += NTHREADS) {
    const int r = i >> 3, q = i & 7;
    cp16(sA + (r >> 3) * 1024 + q * 128 + (r & 7) * 16, A + (size_t)(m0 + r) * kpad + k0 + q * 8);
  }
  for (int i = tid; i < nt * (BK / 8); i += NTHREADS) {
    const int r = i >> 3, q = i & 7;
    cp16(sB + (r >> 3) * 1024 + q * 128 + (r & 7) * 16, YT + (size_t)r * kpad + k0 + q * 8);
  }
}

template <bool MOM, bool LAP>
__global__ void __launch_bounds__(NTHREADS, 1) k_dense_step(DenseStep p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[STAGES + 1];
  __shared__ uint32_t tmem_slot;
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ks = p.ks;
  const int r = (int)cluster.block_rank();
  const int m0 = (int)(blockIdx.x / ks) * BM;
  const int cbase = (int)blockIdx.y * 256;
  const int nt = min(256, p.cpad - cbase);   // MMA N of this column tile, a multiple of 32
  const int ntmax = min(256, p.cpad);        // stage size is that of the widest tile
  const int nk = p.kpad / BK;
  const int kb = (int)((int64_t)nk * r / ks), ke = (int)((int64_t)nk * (r + 1) / ks);
  const int nloc = ke - kb;   // >= 1 (the launcher keeps ks <= nk)
  const size_t a_bytes = (size_t)BM * BK * 2;
  const size_t stage_bytes = a_bytes + (size_t)ntmax * BK * 2;
  const uint32_t tmem_cols = nt <= 32 ? 32u : (nt <= 64 ? 64u : (nt <= 128 ? 128u : 256u));
  const __nv_bfloat16* YT = p.YT + (size_t)cbase * p.kpad;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s <= STAGES; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(BM, nt);
  bool timed_out = false;

  // prologue: chunks 0 .. STAGES-2, one cp.async group each (empty past the end)
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nloc) {
      unsigned char* sA = smem + (size_t)s * stage_bytes;
      load_stage(sA, sA + a_bytes, p.A, p.kpad, YT, m0, (kb + s) * BK, nt, tid);
    }
    cp_commit();
  }
  for (int kc = 0; kc < nloc; ++kc) {
    const int s = kc % STAGES;
    cp_wait<STAGES - 2>();   // this thread's copies of chunk kc have landed
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = saddr(smem + (size_t)s * stage_bytes);
      const uint32_t b0 = a0 + (uint32_t)a_bytes;
#pragma unroll
      for (int q = 0; q < BK / 16; ++q) {   // K = 16: two core matrices along K
        const uint64_t ad = smem_desc(a0 + q * 256, 128, 1024);
        const uint64_t bd = smem_desc(b0 + q * 256, 128, 1024);
        mma_bf16(tmem, ad, bd, idesc, (kc > 0 || q > 0) ? 1u : 0u);
      }
      mma_commit(&bars[s]);   // stage s is free once these MMAs have read it
    }
    // refill: chunk kc + STAGES - 1 into the stage of chunk kc - 1
    const int kn = kc + STAGES - 1;
    if (kn < nloc) {
      const int sn = kn % STAGES;
      if (kn >= STAGES && !mbar_wait(&bars[sn], (uint32_t)((kn - STAGES) / STAGES) & 1u)) timed_out = true;
      unsigned char* sA = smem + (size_t)sn * stage_bytes;
      load_stage(sA, sA + a_bytes, p.A, p.kpad, YT, m0, (kb + kn) * BK, nt, tid);
    }
    cp_commit();
  }
  cp_wait<0>();
  if (tid == 0) mma_commit(&bars[STAGES]);   // tracks every MMA issued above
  if (!mbar_wait(&bars[STAGES], 0)) timed_out = true;
  tc_fence_after();

  // partial product -> shared memory, column-major (part[c * 128 + row]):
  // warp w reads tensor-memory lanes 32w .. 32w+31 (rows of the tile)
  float* part = reinterpret_cast<float*>(smem);
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c0 = 0; c0 < nt; c0 += 32) {
    float g[32];
    tmem_ld32(tl + (uint32_t)c0, g);
#pragma unroll
    for (int k = 0; k < 32; ++k) part[(c0 + k) * BM + warp * 32 + lane] = g[k];
  }
  tc_fence_before();
  cluster.sync();   // every partial of the tile is in place
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");

  // reduction over the ks partials and the fused update
  const int rows_per = BM / ks;
  const int lr = r * rows_per + tid % rows_per;   // row within the tile
  const int i = m0 + lr;
  bool bad = false;
  if (i < p.n && !timed_out) {
    const float dr = LAP ? p.dnet[i] : 0.0f;
    for (int c = tid / rows_per; c < nt; c += ks) {
      float acc = *cluster.map_shared_rank(part + c * BM + lr, 0);
      for (int q = 1; q < ks; ++q) acc += *cluster.map_shared_rank(part + c * BM + lr, q);
      const int col = cbase + c;
      const size_t o = (size_t)col * p.kpad + i;
      const float y = __bfloat162float(p.YT[o]);
      const float grad = LAP ? fmaf(dr, y, -acc) : -acc;
      float step = grad;
      if (MOM) step = fmaf(p.mu, p.VT[o], grad);
      const bool active = col < p.C && (!p.steps_cols || p.t < p.steps_cols[col]);
      const float alpha = p.alpha_cols ? p.afac * p.alpha_cols[col < p.C ? col : 0] : p.alpha;
      float yn = fmaf(alpha, step, y);
      if (active && !isfinite(yn)) bad = true;
      yn = fminf(fmaxf(yn, -1.0f), 1.0f);
      p.YTout[o] = __float2bfloat16_rn(active ? yn : y);
      if (MOM && active) p.VT[o] = step;
    }
  }
  cluster.sync();   // peers have finished reading this CTA's partial
  if (p.flag && (bad || timed_out)) atomicOr(p.flag, (bad ? 1 : 0) | (timed_out ? 2 : 0));
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

std::atomic<int> g_smem_set[2][2];   // largest dynamic shared memory enabled per instance

}  // namespace

size_t dense_smem_bytes(int ntile) { return (size_t)STAGES * ((size_t)BM * BK * 2 + (size_t)ntile * BK * 2); }

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

int launch_dense_step(const DenseStep& p, cudaStream_t st) {
  const int nk = p.kpad / BK;
  if (p.kpad % BM || p.cpad % 32 || p.cpad < 32 || p.ks < 1 || p.ks > 8 || (p.ks & (p.ks - 1)) || p.ks > nk) {
    set_error("dense step: bad shape (kpad=%d cpad=%d ks=%d)", p.kpad, p.cpad, p.ks);
    return DECO_ERR_ARG;
  }
  const size_t smem = dense_smem_bytes(std::min(256, p.cpad));
  const bool mom = p.mu != 0.0f, lap = p.objective == DECO_OBJ_LAPLACIAN;
  void (*fn)(DenseStep) = mom ? (lap ? k_dense_step<true, true> : k_dense_step<true, false>)
                              : (lap ? k_dense_step<false, true> : k_dense_step<false, false>);
  std::atomic<int>& set = g_smem_set[mom][lap];
  if (set.load() < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "dense step shared memory");
    set.store((int)smem);
  }
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
  cudaError_t e = cudaLaunchKernelEx(&cfg, fn, p);
  if (e != cudaSuccess) return cuda_fail(e, "dense step launch");
  return DECO_OK;
}

}  // namespace deco
