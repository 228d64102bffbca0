// Helpers shared by the C-ABI entry points: argument checks, stream-ordered
// scratch allocation, pointer kind detection.
#pragma once

#include <atomic>
#include <vector>

#include "deco_internal.cuh"

namespace deco {

// Host-side fault injection (deco_debug_fail_scratch_alloc): while positive,
// every scratch allocation counts it down, and the one that brings it to zero
// fails with DECO_ERR_OOM instead of allocating.
extern std::atomic<int> g_scratch_fail_countdown;

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

inline int check_graph(const deco_graph* g) {
  if (!g) { set_error("graph is NULL"); return DECO_ERR_ARG; }
  return DECO_OK;
}

inline int check_prec(int p) {
  if (p != DECO_PREC_FP32 && p != DECO_PREC_BF16) { set_error("bad precision %d", p); return DECO_ERR_ARG; }
  return DECO_OK;
}

inline int check_obj(int o) {
  if (o != DECO_OBJ_MULTILINEAR01 && o != DECO_OBJ_LAPLACIAN) { set_error("bad objective %d", o); return DECO_ERR_ARG; }
  return DECO_OK;
}

inline size_t elem_size(int prec) { return prec == DECO_PREC_BF16 ? 2 : 4; }

// Stream-ordered scratch memory of one call, released (stream-ordered) when
// the object goes out of scope.
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
  template <typename T>
  int alloc(T** out, size_t bytes) {
    if (g_scratch_fail_countdown.load(std::memory_order_relaxed) > 0 &&
        g_scratch_fail_countdown.fetch_sub(1, std::memory_order_relaxed) == 1) {
      set_error("injected scratch allocation failure");
      return DECO_ERR_OOM;
    }
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(scratch)");
    ptrs.push_back(p);
    *out = static_cast<T*>(p);
    return DECO_OK;
  }
};

inline void fill_init(InitLaunch& il, const deco_graph* g, int32_t B, int32_t lift, int32_t ld,
                      const deco_params* p, uint64_t seed, int32_t phase) {
  il.n = g->n; il.B = B; il.lift = lift; il.ld = ld;
  il.precision = p->precision; il.objective = p->objective; il.init = p->init;
  il.eta = p->eta; il.scale = p->scale; il.uniform_half_width = p->uniform_half_width;
  il.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  il.k1 = (uint32_t)(seed >> 32);
  il.phase = phase;
}

int convert_bf16_to_f32(int64_t count, const void* in, float* out, cudaStream_t st);

}  // namespace deco
