// Diagnostic: the rate at which tcgen05.mma instructions (kind::f16, M = 128,
// N = 64 / 128 / 256, K = 16, BF16 operands in shared memory, FP32
// accumulators in tensor memory) complete on this GPU when issued back to
// back by one or two threads per SM: the tensor-core ceiling of the dense
// kernels' contraction, whose instructions have N = the iterate's columns
// (128 for the dense workload).
#include <algorithm>

#include "api_util.cuh"
#include "deco_internal.cuh"
#include "phase.cuh"

using namespace deco;

namespace {

constexpr int PROBE_THREADS = 128;
constexpr uint64_t PROBE_WAIT_NS = 1000000000ull;   // 1 s per wait at most

__device__ __forceinline__ uint32_t p_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t p_gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// K-major operand in the 128-byte swizzled layout (the dense kernels' form)
__device__ __forceinline__ uint64_t p_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024u >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// One CTA per SM.  Issuer i (thread 32 (i + 1)) issues `count` MMAs into its
// own accumulator (tensor-memory columns [256 i, 256 i + n)), commits them to
// its mbarrier and waits; out[2 blockIdx + i] = its issue-to-completion time
// in ns, or 0 if its wait gave up.
__global__ void __launch_bounds__(PROBE_THREADS, 1) k_probe_mma(int n, int issuers, int count,
                                                                 unsigned long long* out) {
  extern __shared__ unsigned char raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t slot;
  const uint32_t base = (p_saddr(raw) + 1023u) & ~1023u;
  unsigned char* const sb = raw + (base - p_saddr(raw));
  const int tid = threadIdx.x;
  for (int i = tid; i < 16384 + 32768; i += PROBE_THREADS) sb[i] = 0;   // A 128 x 64, B 256 x 64 (BF16 zeros)
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(p_saddr(&slot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(p_saddr(&bar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // zeroed operands -> tensor-core reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = slot;
  const int me = tid / 32 - 1;
  if ((tid & 31) == 0 && me >= 0 && me < issuers) {
    const uint32_t a = base, b = base + 16384;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t d = tmem + 256u * (uint32_t)me;
    const uint64_t t0 = p_gtimer();
    for (int i = 0; i < count; ++i) {
      const uint32_t q = (uint32_t)(i & 3);
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
          "l"(p_desc(a + 32u * q)), "l"(p_desc(b + 32u * q)), "r"(idesc), "r"(i > 0 ? 1u : 0u)
          : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     p_saddr(&bar[me]))
                 : "memory");
    bool ok = false;
    for (uint32_t it = 0; it < (1u << 30) && !ok; ++it) {
      uint32_t r;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(r)
          : "r"(p_saddr(&bar[me]))
          : "memory");
      ok = r != 0;
      if (!ok && (it & 63u) == 0 && p_gtimer() - t0 > PROBE_WAIT_NS) break;
    }
    out[2 * blockIdx.x + me] = ok ? p_gtimer() - t0 : 0ull;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

}  // namespace

extern "C" int deco_probe_mma_rate(int32_t n, int32_t issuers, int32_t count, float* ns_per_instruction,
                                   void* stream) {
  clear_error();
  if ((n != 64 && n != 128 && n != 256) || issuers < 1 || issuers > 2 || count < 1 || count > (1 << 24) ||
      !ns_per_instruction) {
    set_error("bad arguments (n=%d issuers=%d count=%d)", n, issuers, count);
    return DECO_ERR_ARG;
  }
  cudaStream_t st = as_stream(stream);
  const int sms = device_sm_count();
  // more than half of an SM's shared memory: one CTA (one 512-column tensor-memory allocation) per SM
  const size_t smem = 1024 + 16384 + 32768 + 96 * 1024;
  DECO_CUDA_TRY(cudaFuncSetAttribute(k_probe_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  Scratch s(st);
  unsigned long long* d = nullptr;
  int rc = s.alloc((void**)&d, sizeof(unsigned long long) * 2 * (size_t)sms);
  if (rc) return rc;
  DECO_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * 2 * (size_t)sms, st));
  k_probe_mma<<<(unsigned)sms, PROBE_THREADS, smem, st>>>(n, issuers, count, d);
  DECO_CUDA_TRY(cudaGetLastError());
  std::vector<unsigned long long> h(2 * (size_t)sms);
  DECO_CUDA_TRY(cudaMemcpyAsync(h.data(), d, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  DECO_CUDA_TRY(cudaStreamSynchronize(st));
  double sum = 0.0;
  for (int b = 0; b < sms; ++b) {
    unsigned long long worst = 0;
    for (int i = 0; i < issuers; ++i) {
      if (h[2 * b + i] == 0) {
        set_error("tensor-core probe: a wait gave up on SM block %d", b);
        return DECO_ERR_TIMEOUT;
      }
      worst = std::max(worst, h[2 * b + i]);
    }
    sum += (double)worst;
  }
  // per SM: instructions of all its issuers over the slowest issuer's time
  *ns_per_instruction = (float)(sum / sms / ((double)count * issuers));
  return DECO_OK;
}

namespace {

constexpr int SMEM_PROBE_THREADS = 1024;
constexpr int SMEM_PROBE_BYTES = 131072;  // the buffer every CTA reads (power of two, >= 8 x 1024 x 16 B)

// Shared-memory load bandwidth: every thread reads W-byte words of a 128 KB
// buffer, the 32 lanes of a warp consecutive words (no bank conflicts), the
// buffer walked in steps of the CTA's width, `iters` times; the 8 loads of
// one round are at distinct addresses (so none can be merged with another)
// and the words are folded into one value per thread, so no load is dropped.
template <int W>
__global__ void __launch_bounds__(SMEM_PROBE_THREADS, 1) k_probe_smem(int iters, uint32_t* out) {
  extern __shared__ __align__(16) unsigned char buf[];
  const int tid = threadIdx.x;
  for (int i = tid; i < SMEM_PROBE_BYTES / 4; i += SMEM_PROBE_THREADS)
    reinterpret_cast<uint32_t*>(buf)[i] = (uint32_t)i * 2654435761u;
  __syncthreads();
  uint32_t acc = 0;
  uint32_t off = (uint32_t)tid * W;
  constexpr uint32_t STEP = (uint32_t)SMEM_PROBE_THREADS * W, MASK = SMEM_PROBE_BYTES - 1;
  for (int it = 0; it < iters; it += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const uint32_t o = (off + (uint32_t)u * STEP) & MASK;
      if (W == 16) {
        const uint4 q = *reinterpret_cast<const uint4*>(buf + o);
        acc ^= q.x ^ q.y ^ q.z ^ q.w;
      } else {
        const uint2 q = *reinterpret_cast<const uint2*>(buf + o);
        acc ^= q.x ^ q.y;
      }
    }
    off = (off + 8u * STEP + (uint32_t)W) & MASK;   // shift by a word each round: no address repeats in order
  }
  out[(size_t)blockIdx.x * SMEM_PROBE_THREADS + tid] = acc;
}

}  // namespace

extern "C" int deco_probe_smem_rate(int32_t width, int32_t iters, float* gbs, void* stream) {
  clear_error();
  if ((width != 8 && width != 16) || iters < 8 || iters > (1 << 24) || iters % 8 != 0 || !gbs) {
    set_error("bad arguments (width=%d iters=%d)", width, iters);
    return DECO_ERR_ARG;
  }
  cudaStream_t st = as_stream(stream);
  const int sms = device_sm_count();
  auto fn = width == 16 ? k_probe_smem<16> : k_probe_smem<8>;
  // the buffer plus enough extra to keep one CTA per SM
  const size_t smem = SMEM_PROBE_BYTES + 32 * 1024;
  DECO_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  Scratch s(st);
  uint32_t* d = nullptr;
  int rc = s.alloc((void**)&d, sizeof(uint32_t) * (size_t)sms * SMEM_PROBE_THREADS);
  if (rc) return rc;
  cudaEvent_t ev[2];
  DECO_CUDA_TRY(cudaEventCreate(&ev[0]));
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return cuda_fail(cudaGetLastError(), "event");
  }
  fn<<<(unsigned)sms, SMEM_PROBE_THREADS, smem, st>>>(8, d);   // warm-up
  cudaEventRecord(ev[0], st);
  fn<<<(unsigned)sms, SMEM_PROBE_THREADS, smem, st>>>(iters, d);
  cudaEventRecord(ev[1], st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return cuda_fail(e, "shared-memory probe");
  const double bytes = (double)sms * SMEM_PROBE_THREADS * (double)iters * width;
  *gbs = (float)(bytes / (ms * 1e-3) / 1e9);
  return DECO_OK;
}

extern "C" int deco_probe_wait_timeout(int32_t which, float* waited_ms, void* stream) {
  clear_error();
  if (which < 0 || which > 2) {
    set_error("bad wait kind %d", which);
    return DECO_ERR_ARG;
  }
  cudaStream_t st = as_stream(stream);
  Scratch s(st);
  int32_t* d = nullptr;   // [0] the flag, [1] the counter nobody increments
  int rc = s.alloc((void**)&d, 2 * sizeof(int32_t));
  if (rc) return rc;
  DECO_CUDA_TRY(cudaMemsetAsync(d, 0, 2 * sizeof(int32_t), st));
  cudaEvent_t ev[2];
  DECO_CUDA_TRY(cudaEventCreate(&ev[0]));
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return cuda_fail(cudaGetLastError(), "event");
  }
  cudaEventRecord(ev[0], st);
  rc = which == 2 ? launch_wait_probe_slab(d, st)
                  : launch_wait_probe_dense(which, reinterpret_cast<unsigned int*>(d + 1), d, st);
  cudaEventRecord(ev[1], st);
  int32_t flag = 0;
  cudaError_t e = rc ? cudaSuccess : cudaMemcpyAsync(&flag, d, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !rc) e = cudaStreamSynchronize(st);
  float ms = 0.0f;
  if (e == cudaSuccess && !rc) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  if (waited_ms) *waited_ms = ms;
  if (flag & 2) {
    set_error("wait probe %d: the bounded wait gave up after %.1f ms", which, ms);
    return DECO_ERR_TIMEOUT;
  }
  return DECO_OK;
}
