// deco_run_phase_noalloc: the per-step phase runner with its scratch block in
// a fixed, library-owned device array instead of memory allocated per call.
//
// Who needs it: host programs that cannot let a library allocate device
// memory while they run -- for example a runtime whose own pool has already
// reserved (nearly) all of the device, or a latency-bound loop in which a
// cudaMalloc / cudaFree (which can synchronise the whole device) is not
// acceptable.  Such callers still provide the iterate, the momentum buffer and
// the flag; the only memory this entry point needs beyond them is the second
// block of the step kernel's ping-pong, which lives in `g_phase_scratch` below.
#include <mutex>

#include "api_util.cuh"
#include "deco_internal.cuh"

using namespace deco;

namespace {

// Fixed scratch: the second block of the ping-pong between steps.  It is a
// file-scope device array, so every GPU that loads the library keeps these
// 16 MiB until the process exits.
constexpr size_t kPhaseScratchBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_phase_scratch[kPhaseScratchBytes];

// Device address of g_phase_scratch, looked up once per (device, context).
// Host code may not use the symbol itself as a device pointer: on the host it
// only names a host-side stand-in.  The address belongs to the CUDA context
// that loaded the module, so it is cached together with that context's
// unique id (cuCtxGetId: never reused within a process): after a
// cudaDeviceReset, or any other teardown and re-creation of the context, the
// next call sees a new id and looks the address up again instead of handing
// the kernel a stale pointer.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
  unsigned long long ctx_id = 0;   // id of the context current when the address was taken
  void* addr = nullptr;
};
ScratchSlot g_scratch_slot[kMaxDevices];
std::mutex g_scratch_mutex;

// cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry-point
// query, so that the library needs no link-time dependency on the driver API.
using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);
template <typename F>
int driver_fn(const char* name, F* fn) {
  if (*fn) return DECO_OK;
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q{};
  cudaError_t e = cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDriverEntryPointByVersion");
  if (q != cudaDriverEntryPointSuccess || !f) {
    set_error("%s is not available from the driver", name);
    return DECO_ERR_CUDA;
  }
  *fn = reinterpret_cast<F>(f);
  return DECO_OK;
}

// unique id of the current context (DECO_ERR_CUDA when none is current)
int current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  int rc = driver_fn("cuCtxGetCurrent", &get_current);
  if (rc || (rc = driver_fn("cuCtxGetId", &get_id))) return rc;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) {
    set_error("no current CUDA context");
    return DECO_ERR_CUDA;
  }
  if (get_id(ctx, id) != 0) {
    set_error("cuCtxGetId failed");
    return DECO_ERR_CUDA;
  }
  return DECO_OK;
}

int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d is beyond the %d devices this entry point tracks", dev, kMaxDevices);
    return DECO_ERR_UNSUPPORTED;
  }
  // the context the kernels will run in; with none current yet, cudaSetDevice
  // makes the device's primary context current (creating it on first use)
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  unsigned long long ctx_id = 0;
  int rc = current_context_id(&ctx_id);
  if (rc) {
    clear_error();
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if ((rc = current_context_id(&ctx_id))) return rc;
  }
  ScratchSlot& slot = g_scratch_slot[dev];
  if (!slot.addr || slot.ctx_id != ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_phase_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_phase_scratch)");
    slot.addr = p;
    slot.ctx_id = ctx_id;
  }
  *out = slot.addr;
  return DECO_OK;
}

}  // namespace

extern "C" int deco_run_phase_noalloc(const deco_graph* g, int32_t C, int32_t ld, void* y, float* v,
                                      int32_t steps, const deco_step_args* a, int32_t* nonfinite_flag,
                                      void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (!a) { set_error("NULL step arguments"); return DECO_ERR_ARG; }
  if ((rc = check_prec(a->precision)) || (rc = check_obj(a->objective))) return rc;
  if (C < 1 || ld < C || ld % 8) {
    set_error("need 1 <= C <= ld and ld %% 8 == 0 (C=%d ld=%d)", C, ld);
    return DECO_ERR_ARG;
  }
  if (!y) { set_error("NULL block"); return DECO_ERR_ARG; }
  if (steps < 0) { set_error("steps must be >= 0"); return DECO_ERR_ARG; }
  if (a->momentum != 0.0f && !v) { set_error("momentum needs the v buffer"); return DECO_ERR_ARG; }
  const size_t block_bytes = (size_t)g->n * (size_t)ld * elem_size(a->precision);
  if (block_bytes > kPhaseScratchBytes) {
    set_error("block of %zu bytes (n=%d, ld=%d) exceeds the fixed %zu-byte scratch of "
              "deco_run_phase_noalloc; use deco_run_phase", block_bytes, g->n, ld, kPhaseScratchBytes);
    return DECO_ERR_UNSUPPORTED;
  }
  void* scratch = nullptr;
  if ((rc = scratch_address(&scratch))) return rc;
  if (steps == 0) return DECO_OK;

  cudaStream_t st = as_stream(stream);
  StepLaunch sl{};
  sl.n = g->n; sl.C = C; sl.ld = ld;
  sl.precision = a->precision; sl.objective = a->objective; sl.wmode = g->wmode;
  sl.row_ptr = g->row_ptr; sl.col_idx = g->col_idx; sl.col_sw = g->col_sw; sl.w = g->w; sl.dnet = g->dnet;
  sl.v = v; sl.alpha = a->alpha; sl.mu = a->momentum;
  sl.alpha_cols = a->alpha_cols; sl.steps_cols = a->steps_cols;
  sl.flag = nonfinite_flag;
  // Columns >= C of the scratch keep whatever an earlier call left there; the
  // step kernel never lets them reach a result column, so nothing needs
  // clearing.
  void* blk[2] = {y, scratch};
  int cur = 0;
  for (int32_t t = 0; t < steps; ++t) {
    sl.yin = blk[cur];
    sl.yout = blk[cur ^ 1];
    sl.t = t;
    if ((rc = launch_step_global(sl, st))) return rc;
    cur ^= 1;
  }
  if (cur != 0) {
    const size_t esz = elem_size(a->precision);
    DECO_CUDA_TRY(cudaMemcpy2DAsync(y, (size_t)ld * esz, scratch, (size_t)ld * esz, (size_t)C * esz, g->n,
                                    cudaMemcpyDeviceToDevice, st));
  }
  return DECO_OK;
}
