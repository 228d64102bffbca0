// Autotuner of the phase launch shape: times every feasible candidate on the
// caller's graph and records the fastest with the graph (deco_autotune), or
// records a given shape (deco_set_tuning).
#include <vector>

#include "api_util.cuh"
#include "deco_internal.cuh"
#include "phase.cuh"

using namespace deco;

namespace {

__global__ void k_probe_fill(int64_t count, int prec, uint32_t seed, void* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 7u), seed, 0u);
  const float v = 1e-4f * (2.0f * u01(r.x) - 1.0f);
  if (prec == DECO_PREC_BF16) static_cast<__nv_bfloat16*>(y)[i] = __float2bfloat16_rn(v);
  else static_cast<float*>(y)[i] = v;
}

}  // namespace

extern "C" int deco_set_tuning(const deco_graph* g, int32_t C, int32_t precision, int32_t kernel) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if ((rc = check_prec(precision))) return rc;
  if (C < 1 || !valid_selector(kernel) || kernel == DECO_KERNEL_AUTO) {
    set_error("bad tuning entry (C=%d kernel=0x%x)", C, kernel);
    return DECO_ERR_ARG;
  }
  record_tuning(g, C, precision, kernel);
  return DECO_OK;
}

extern "C" int deco_autotune(const deco_graph* g, int32_t C, int32_t precision, int32_t objective, float momentum,
                             int32_t probe_steps, int32_t* best_kernel, float* best_us_per_step, void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if ((rc = check_prec(precision)) || (rc = check_obj(objective))) return rc;
  if (C < 1 || probe_steps < 1 || !best_kernel) { set_error("bad arguments"); return DECO_ERR_ARG; }
  cudaStream_t st = as_stream(stream);
  const int32_t ld = (C + 63) / 64 * 64;
  const size_t elems = (size_t)g->n * ld;
  const size_t esz = elem_size(precision);

  std::vector<int> cands = {DECO_KERNEL_GLOBAL};
  for (int s = 1; s <= 4; ++s) cands.push_back(DECO_KERNEL_GLOBAL | (s << 16));   // 2..16 column slabs
  // the pipelined per-step form (record streams, cp.async stages), with the
  // mixed-precision BF16 add: 8 / 12 / 16 entries per item and 2 stages, or 8
  // entries and 3 stages, on the whole block and on 2 or 4 column slabs; the
  // wide form (two vectors per lane) of the 8- and 12-entry shapes on the
  // whole block and on 2 slabs (the shapes that measured competitive on a
  // 10^6-node graph)
  for (int s = 0; s <= 2; ++s) {
    for (int e : {1, 3, 0})
      cands.push_back(DECO_KERNEL_GLOBAL | (s << 16) | DECO_KERNEL_PIPELINED | DECO_KERNEL_PIPE_ENTRIES(e) |
                      DECO_KERNEL_PIPE_STAGES(1) | DECO_KERNEL_PIPE_MIXED_ADD);
    cands.push_back(DECO_KERNEL_GLOBAL | (s << 16) | DECO_KERNEL_PIPELINED | DECO_KERNEL_PIPE_ENTRIES(1) |
                    DECO_KERNEL_PIPE_STAGES(0) | DECO_KERNEL_PIPE_MIXED_ADD);
    if (s <= 1)
      for (int e : {1, 3})
        cands.push_back(DECO_KERNEL_GLOBAL | (s << 16) | DECO_KERNEL_PIPELINED | DECO_KERNEL_PIPE_ENTRIES(e) |
                        DECO_KERNEL_PIPE_STAGES(1) | DECO_KERNEL_PIPE_MIXED_ADD | DECO_KERNEL_PIPE_WIDE);
  }
  for (int k = 1; k <= 8; k *= 2)
    for (int t = 1; t <= 2; ++t)
      for (int x = 1; x <= 2; ++x) {
        if (k == 1 && x == 1) continue;   // a single CTA exchanges nothing
        cands.push_back(DECO_KERNEL_ONCHIP | (k << 8) | (t << 12) | (x << 14));
      }
  // the lean on-chip form (momentum in global memory, no staging area): a
  // cluster half as large fits, e.g. one wave instead of two
  for (int k = 1; k <= 8; k *= 2) cands.push_back(DECO_KERNEL_ONCHIP | (k << 8) | (2 << 12) | (2 << 14) | DECO_KERNEL_LEAN);
  // every on-chip shape also in the row-pair form (a half-warp per row)
  for (size_t i = 0, n0 = cands.size(); i < n0; ++i)
    if ((cands[i] & 0x3) == DECO_KERNEL_ONCHIP) cands.push_back(cands[i] | DECO_KERNEL_ROW_PAIRS);
  // dense tensor-core kernel: BF16 blocks of graphs with at least n^2 / 64 entries
  if (precision == DECO_PREC_BF16 && (double)g->nnz * 64.0 >= (double)g->n * (double)g->n)
    for (int k = 1; k <= 8; k *= 2) cands.push_back(DECO_KERNEL_DENSE | (k << 8));

  float best_ms = -1.0f;
  int best = DECO_KERNEL_GLOBAL;
  {
    Scratch s(st);
    void* y[2] = {nullptr, nullptr};
    float* v = nullptr;
    if ((rc = s.alloc(&y[0], elems * esz)) || (rc = s.alloc(&y[1], elems * esz))) return rc;
    if (momentum != 0.0f && (rc = s.alloc(&v, elems * sizeof(float)))) return rc;
    if (v) DECO_CUDA_TRY(cudaMemsetAsync(v, 0, elems * sizeof(float), st));
    cudaEvent_t e0, e1;
    DECO_CUDA_TRY(cudaEventCreate(&e0));
    DECO_CUDA_TRY(cudaEventCreate(&e1));
    struct EvGuard {
      cudaEvent_t a, b;
      ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evg{e0, e1};
    for (int sel : cands) {
      PhaseRunner R;
      PhasePlan plan;
      if (plan_phase(g, C, ld, precision, sel, &plan) != DECO_OK) {   // does not fit
        clear_error();
        continue;
      }
      if ((rc = R.prepare(g, C, ld, precision, sel, st))) { R.release(st); return rc; }
      float ms = 0.0f;
      for (int rep = 0; rep < 2 && rc == DECO_OK; ++rep) {   // first pass warms up
        k_probe_fill<<<(unsigned)((elems + 255) / 256), 256, 0, st>>>((int64_t)elems, precision, 1234u, y[0]);
        int cur = 0;
        cudaEventRecord(e0, st);
        rc = R.run(y, cur, v, probe_steps, objective, 0.01f, momentum, nullptr, nullptr, v != nullptr,
                   v != nullptr, nullptr, st, nullptr);
        cudaEventRecord(e1, st);
        if (rc == DECO_OK) {
          cudaError_t e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) rc = cuda_fail(e, "autotune probe");
          else cudaEventElapsedTime(&ms, e0, e1);
        }
      }
      R.release(st);
      if (rc) return rc;
      if (best_ms < 0.0f || ms < best_ms) {
        best_ms = ms;
        best = sel;
      }
    }
  }
  record_tuning(g, C, precision, best);
  *best_kernel = best;
  if (best_us_per_step) *best_us_per_step = best_ms * 1e3f / (float)probe_steps;
  return DECO_OK;
}
