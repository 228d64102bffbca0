// C-ABI entry points for the individual stages of the hot path: one step, one
// phase, rounding + cut + argmax, cut evaluation, starting blocks.
#include "api_util.cuh"
#include "deco_internal.cuh"
#include "phase.cuh"

using namespace deco;

namespace deco {
namespace {
__global__ void k_bf16_to_f32(int64_t count, const __nv_bfloat16* in, float* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = __bfloat162float(in[i]);
}
}  // namespace

int convert_bf16_to_f32(int64_t count, const void* in, float* out, cudaStream_t st) {
  if (count <= 0) return DECO_OK;
  k_bf16_to_f32<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(
      count, static_cast<const __nv_bfloat16*>(in), out);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}
}  // namespace deco

static int check_step_args(const deco_graph* g, int32_t C, int32_t ld, const deco_step_args* a) {
  int rc = check_graph(g);
  if (rc) return rc;
  if (!a) { set_error("NULL step arguments"); return DECO_ERR_ARG; }
  if ((rc = check_prec(a->precision)) || (rc = check_obj(a->objective))) return rc;
  if (C < 1 || ld < C || ld % 8) {
    set_error("need 1 <= C <= ld and ld %% 8 == 0 (C=%d ld=%d)", C, ld);
    return DECO_ERR_ARG;
  }
  return DECO_OK;
}

namespace deco {
std::atomic<int> g_scratch_fail_countdown{0};
}

extern "C" int deco_debug_fail_scratch_alloc(int32_t k) {
  clear_error();
  if (k < 0) {
    set_error("k must be >= 0");
    return DECO_ERR_ARG;
  }
  g_scratch_fail_countdown.store(k);
  return DECO_OK;
}

extern "C" int deco_debug_pool_usage(int64_t* used_now, int64_t* used_high, int32_t reset) {
  clear_error();
  int dev = 0;
  DECO_CUDA_TRY(cudaGetDevice(&dev));
  cudaMemPool_t pool = nullptr;
  DECO_CUDA_TRY(cudaDeviceGetMemPool(&pool, dev));
  cuuint64_t now = 0, high = 0;
  DECO_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &now));
  DECO_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
  if (used_now) *used_now = (int64_t)now;
  if (used_high) *used_high = (int64_t)high;
  if (reset) {
    cuuint64_t zero = 0;   // the high-water mark restarts from the current use
    DECO_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
  }
  return DECO_OK;
}

extern "C" int deco_step(const deco_graph* g, int32_t C, int32_t ld, const void* y_in, void* y_out,
                         float* v, const deco_step_args* a, int32_t* nonfinite_flag, void* stream) {
  clear_error();
  int rc = check_step_args(g, C, ld, a);
  if (rc) return rc;
  if (!y_in || !y_out) { set_error("NULL block"); return DECO_ERR_ARG; }
  if (y_in == y_out) { set_error("y_out must not alias y_in"); return DECO_ERR_ARG; }
  if (a->momentum != 0.0f && !v) { set_error("momentum needs the v buffer"); return DECO_ERR_ARG; }
  StepLaunch s{};
  s.n = g->n; s.C = C; s.ld = ld;
  s.precision = a->precision; s.objective = a->objective; s.wmode = g->wmode;
  s.row_ptr = g->row_ptr; s.col_idx = g->col_idx; s.col_sw = g->col_sw; s.w = g->w; s.dnet = g->dnet;
  s.yin = y_in; s.yout = y_out; s.v = v;
  s.alpha = a->alpha; s.mu = a->momentum;
  s.alpha_cols = a->alpha_cols; s.steps_cols = a->steps_cols; s.t = a->t;
  s.flag = nonfinite_flag;
  return launch_step_global(s, as_stream(stream));
}

extern "C" int deco_run_phase(const deco_graph* g, int32_t C, int32_t ld, void* y, float* v, int32_t steps,
                              const deco_step_args* a, int32_t kernel, int32_t* nonfinite_flag, void* stream) {
  clear_error();
  int rc = check_step_args(g, C, ld, a);
  if (rc) return rc;
  if (!y) { set_error("NULL block"); return DECO_ERR_ARG; }
  if (steps < 0) { set_error("steps must be >= 0"); return DECO_ERR_ARG; }
  if (!valid_selector(kernel)) {
    set_error("bad kernel selector 0x%x", kernel);
    return DECO_ERR_ARG;
  }
  if (a->momentum != 0.0f && !v) { set_error("momentum needs the v buffer"); return DECO_ERR_ARG; }
  cudaStream_t st = as_stream(stream);
  PhaseRunner R;
  if ((rc = R.prepare(g, C, ld, a->precision, kernel, st))) { R.release(st); return rc; }
  Scratch s(st);
  void* yb[2] = {y, nullptr};
  if (R.plan.kernel == KERNEL_GLOBAL && steps > 0) {
    if ((rc = s.alloc(&yb[1], (size_t)g->n * ld * elem_size(a->precision)))) { R.release(st); return rc; }
  }
  int cur = 0;
  const bool mom = a->momentum != 0.0f;
  rc = R.run(yb, cur, v, steps, a->objective, a->alpha, a->momentum, a->alpha_cols, a->steps_cols,
             mom, mom, nonfinite_flag, st, nullptr);
  if (rc == DECO_OK && cur != 0) {
    const size_t esz = elem_size(a->precision);
    cudaError_t e = cudaMemcpy2DAsync(y, (size_t)ld * esz, yb[1], (size_t)ld * esz, (size_t)C * esz, g->n,
                                      cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpy2DAsync(run_phase)");
  }
  R.release(st);
  return rc;
}

extern "C" int deco_round_cut(const deco_graph* g, int32_t B, int32_t lift, int32_t ld,
                              int32_t precision, const void* y, uint32_t* zbits, int64_t* cuts,
                              int32_t* best, void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if ((rc = check_prec(precision))) return rc;
  if (B < 1 || lift < 1 || ld < B * lift || !y || !zbits || !cuts) {
    set_error("bad arguments (B=%d lift=%d ld=%d)", B, lift, ld);
    return DECO_ERR_ARG;
  }
  cudaStream_t st = as_stream(stream);
  if ((rc = launch_pack(g, B, lift, ld, precision, y, zbits, st))) return rc;
  if ((rc = launch_cut_bits(g, B, zbits, cuts, st))) return rc;
  if (best && (rc = launch_argmax(B, cuts, best, st))) return rc;
  return DECO_OK;
}

extern "C" int deco_eval_cuts(const deco_graph* g, int32_t B, const uint8_t* z, int64_t* cuts, void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (B < 1 || !z || !cuts) { set_error("bad arguments"); return DECO_ERR_ARG; }
  return launch_cut_bytes(g, B, z, cuts, as_stream(stream));
}

extern "C" int deco_eval_cut(const deco_graph* g, const uint8_t* z, int64_t* cut_out) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (!z || !cut_out) { set_error("NULL argument"); return DECO_ERR_ARG; }
  cudaStream_t st = 0;
  int64_t c = 0;
  {
    Scratch s(st);
    uint8_t* dz = nullptr;
    int64_t* dc = nullptr;
    if ((rc = s.alloc(&dz, (size_t)g->n)) || (rc = s.alloc(&dc, sizeof(int64_t)))) return rc;
    DECO_CUDA_TRY(cudaMemcpyAsync(dz, z, (size_t)g->n, cudaMemcpyHostToDevice, st));
    if ((rc = launch_cut_bytes(g, 1, dz, dc, st))) return rc;
    DECO_CUDA_TRY(cudaMemcpyAsync(&c, dc, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  }
  DECO_CUDA_TRY(cudaStreamSynchronize(st));
  *cut_out = c;
  return DECO_OK;
}

extern "C" int deco_idi_mean(const deco_graph* g, float beta, uint64_t seed, int32_t phase, float* h,
                             void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (!h) { set_error("h is NULL"); return DECO_ERR_ARG; }
  cudaStream_t st = as_stream(stream);
  Scratch s(st);
  int8_t* side = nullptr;
  if ((rc = s.alloc(&side, (size_t)g->n))) return rc;
  return launch_idi(g, idi_threshold(g, beta), (uint32_t)seed, (uint32_t)(seed >> 32), phase, h, side, st);
}

extern "C" int deco_dui_mean(const deco_graph* g, uint64_t seed, int32_t phase, float* h, void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (!h) { set_error("h is NULL"); return DECO_ERR_ARG; }
  return launch_dui(g, (uint32_t)seed, (uint32_t)(seed >> 32), phase, h, as_stream(stream));
}

extern "C" int deco_init_block(const deco_graph* g, int32_t B, int32_t lift, int32_t ld,
                               const deco_params* p, uint64_t seed, int32_t phase, const float* mean,
                               const float* x0, void* y, void* stream) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (!p || !y) { set_error("NULL argument"); return DECO_ERR_ARG; }
  if ((rc = check_prec(p->precision)) || (rc = check_obj(p->objective))) return rc;
  if (B < 1 || lift < 1 || ld < B * lift || ld % 8) { set_error("bad sizes"); return DECO_ERR_ARG; }
  cudaStream_t st = as_stream(stream);
  InitLaunch il{};
  fill_init(il, g, B, lift, ld, p, seed, phase);
  il.y = y;
  Scratch s(st);
  switch (p->init) {
    case DECO_INIT_UNIFORM:
      break;
    case DECO_INIT_EXPLICIT:
      if (!x0) { set_error("explicit init needs x0"); return DECO_ERR_ARG; }
      il.x0 = x0;
      break;
    case DECO_INIT_MEAN:
      if (!mean) { set_error("mean init needs mean"); return DECO_ERR_ARG; }
      il.mean = mean;
      break;
    case DECO_INIT_IDI:
    case DECO_INIT_IDI_HALF_UNIFORM:
    case DECO_INIT_DUI: {
      float* h = nullptr;
      int8_t* side = nullptr;
      if ((rc = s.alloc(&h, sizeof(float) * g->n)) || (rc = s.alloc(&side, (size_t)g->n))) return rc;
      if (p->init == DECO_INIT_DUI) rc = launch_dui(g, il.k0, il.k1, phase, h, st);
      else rc = launch_idi(g, idi_threshold(g, p->beta), il.k0, il.k1, phase, h, side, st);
      if (rc) return rc;
      il.mean = h;
      break;
    }
    default:
      set_error("bad init %d", p->init);
      return DECO_ERR_ARG;
  }
  return launch_init(il, st);
}
