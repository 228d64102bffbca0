// One phase of projected gradient ascent (the step loop of Alg. 1 / Alg. 2): T steps
// on a device block, by the persistent on-chip kernel (slab.cu) when one
// column slab of the graph fits in shared memory, otherwise by one launch of
// the global-memory kernel (step_global.cu) per step.
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "deco_internal.cuh"
#include "phase.cuh"
#include "slab.cuh"

namespace deco {

int device_sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
  }
  return sms;
}

// Exact sizes of the on-chip CSR image of a split (see slab.cuh).
static void image_sizes(const deco_graph* g, int k, const int32_t* split, int32_t* max_own,
                        int64_t* max_words, int64_t* max_edges) {
  *max_own = 0;
  *max_words = 0;
  *max_edges = 0;
  const bool gen = g->wmode == W_GENERAL;
  for (int part = 0; part < k; ++part) {
    const int r0 = split[part], r1 = split[part + 1];
    int64_t E = 0;
    for (int r = r0; r < r1; ++r) {
      const int e0 = g->h_row_ptr[r], e1 = g->h_row_ptr[r + 1];
      int nn = 0;
      if (g->wmode == W_SIGN)
        for (int e = e0; e < e1; ++e) nn += g->h_w[e] < 0.0f;
      const int np = (e1 - e0) - nn;
      E += (np + 3) / 4 * 4 + (nn + 3) / 4 * 4;
    }
    E += 8;
    int64_t words = 4 * (int64_t)(r1 - r0 + 1) + E * (gen ? 2 : 1);
    words = (words + 3) / 4 * 4;
    *max_own = std::max(*max_own, r1 - r0);
    *max_words = std::max(*max_words, words);
    *max_edges = std::max<int64_t>(*max_edges, g->h_row_ptr[r1] - g->h_row_ptr[r0]);
  }
}

// Cost model of one step of the on-chip kernel, in units of one 128-byte
// shared-memory row read: own gathers + broadcast of the staged rows (all n
// rows land in every replica when k > 1) + epilogue + barrier latency.
static double onchip_cost(int64_t own_nnz, int32_t own, int32_t n, int k, int waves) {
  const double per_cta = 1.25 * (double)own_nnz + (k > 1 ? (double)n : (double)own) + 4.0 * own + 1500.0;
  return per_cta * waves;
}

bool valid_selector(int kernel) {
  const int kind = kernel & 0x3, k = (kernel >> 8) & 0xF, t = (kernel >> 12) & 0x3, x = (kernel >> 14) & 0x3;
  const int s = (kernel >> 16) & 0x7;
  const int l2hints = (kernel >> 19) & 1;
  const int lean = (kernel >> 20) & 1;
  const int pairs = (kernel >> 21) & 1;
  const int pipe = (kernel >> 22) & 1;
  const int pipe_shape = (kernel >> 23) & 0x7F;   // entries, stages, warps
  const int mixed = (kernel >> 30) & 1;
  const int wide = (kernel >> 2) & 1;
  if (kernel & ~0x7FFFFFFF) return false;
  if (kernel & 0xF8) return false;   // bits 3..7 are not defined
  if (wide && !pipe) return false;
  if (mixed && !pipe) return false;
  if (l2hints && !pipe) return false;
  if (pipe && ((pipe_shape >> 2) & 3) == 3) return false;   // stage code 3 is not defined
  if (pipe && kind != DECO_KERNEL_GLOBAL) return false;
  if (!pipe && pipe_shape) return false;
  if (lean && kind != DECO_KERNEL_ONCHIP) return false;
  if (pairs && kind != DECO_KERNEL_ONCHIP) return false;
  if (lean && x == 1) return false;   // the lean form exchanges through L2
  if (kind < DECO_KERNEL_AUTO || kind > DECO_KERNEL_DENSE || t == 3 || x == 3) return false;
  if (x && kind != DECO_KERNEL_ONCHIP) return false;
  if (t && kind != DECO_KERNEL_ONCHIP && !(kind == DECO_KERNEL_DENSE && t == 1)) return false;
  if (k && kind != DECO_KERNEL_ONCHIP && kind != DECO_KERNEL_DENSE) return false;
  if (s && (kind != DECO_KERNEL_GLOBAL || s > 6)) return false;
  if (k && ((k & (k - 1)) || k > 8)) return false;
  return true;
}

static std::mutex g_image_mutex;

int tuned_selector(const deco_graph* g, int32_t C, int prec) {
  std::lock_guard<std::mutex> lock(g_image_mutex);
  for (const auto& t : g->tuning)
    if (t.C == C && t.prec == prec) return t.kernel;
  return -1;
}

void record_tuning(const deco_graph* g, int32_t C, int prec, int kernel) {
  std::lock_guard<std::mutex> lock(g_image_mutex);
  auto& tv = const_cast<deco_graph*>(g)->tuning;
  for (auto& t : tv)
    if (t.C == C && t.prec == prec) { t.kernel = kernel; return; }
  tv.push_back({C, prec, kernel});
}

// Dense tensor-core kernel: limits, padding and the contraction split (the
// largest power of two <= 8 that keeps row tiles x column tiles x split within
// one wave of the SMs, unless fixed by the caller).
static int plan_dense(const deco_graph* g, int32_t C, int want_k, bool per_step, PhasePlan* plan) {
  if (g->n < 1 || g->n > DENSE_MAX_N || C > DENSE_MAX_C || g->max_abs_w > DENSE_MAX_W) {
    set_error("the dense kernel needs n <= %d, C <= %d and |w| <= %d (n=%d, C=%d, max |w|=%d)", DENSE_MAX_N,
              DENSE_MAX_C, DENSE_MAX_W, g->n, C, g->max_abs_w);
    return DECO_ERR_UNSUPPORTED;
  }
  plan->kernel = KERNEL_DENSE;
  plan->kpad = (g->n + DENSE_BM - 1) / DENSE_BM * DENSE_BM;
  plan->cpad = (C + 31) / 32 * 32;
  const int nk = plan->kpad / DENSE_BK;
  const int64_t tiles = (int64_t)(plan->kpad / DENSE_BM) * ((plan->cpad + 255) / 256);
  int ks = want_k;
  if (!ks) {
    ks = 1;
    while (ks < 8 && 2 * ks <= nk && tiles * 2 * ks <= device_sm_count()) ks *= 2;
  }
  if (ks > nk) {
    set_error("dense kernel: a split of %d exceeds the %d contraction chunks of n=%d", ks, nk, g->n);
    return DECO_ERR_UNSUPPORTED;
  }
  plan->ks = ks;
  if (!per_step) {
    // persistent phase kernel: column tiles of <= 128, the largest split whose
    // CTAs fit in one wave (residency is checked again at launch)
    const int w = std::min(128, plan->cpad);
    const int64_t tiles_p = (int64_t)(plan->kpad / DENSE_BM) * ((plan->cpad + w - 1) / w);
    for (int kp = 8; kp >= 1; kp /= 2) {
      if (want_k && kp != want_k) continue;
      if (!want_k && tiles_p * kp > device_sm_count()) continue;
      DensePhaseShape sh;
      if (dense_phase_shape(plan->kpad, plan->cpad, kp, w, &sh) == DECO_OK) {
        plan->dpersist = true;
        plan->dphase = sh;
        break;
      }
      clear_error();
    }
  }
  return DECO_OK;
}

int plan_phase(const deco_graph* g, int32_t C, int32_t ld, int prec, int force, PhasePlan* plan) {
  if (force == DECO_KERNEL_AUTO) {
    const int tuned = tuned_selector(g, C, prec);
    if (tuned > 0) {
      const int rc = plan_phase(g, C, ld, prec, tuned, plan);
      if (rc == DECO_OK) return rc;
      clear_error();   // a recorded shape that no longer fits: fall back to the cost model
    }
  }
  *plan = PhasePlan{};
  plan->kernel = KERNEL_GLOBAL;
  const int cols = prec == DECO_PREC_BF16 ? 64 : 32;
  const int want_k = (force >> 8) & 0xF;
  const int want_t = (force >> 12) & 0x3;
  const int want_x = (force >> 14) & 0x3;
  const int want_s = (force >> 16) & 0x7;
  const bool want_hints = ((force >> 19) & 1) != 0;
  const bool want_lean = ((force >> 20) & 1) != 0;
  const bool want_pipe = ((force >> 22) & 1) != 0;
  const int pipe_e = (force >> 23) & 3, pipe_s = (force >> 25) & 3, pipe_w = (force >> 27) & 7;
  const bool pipe_mix = ((force >> 30) & 1) != 0;
  const bool pipe_wide = ((force >> 2) & 1) != 0;
  // the row-pair form is also the cost model's choice (measured faster on
  // every on-chip shape of the benchmark); the autotuner times both forms
  const bool want_pairs = ((force >> 21) & 1) != 0 || (force & 0x3) == DECO_KERNEL_AUTO;
  force &= 0x3;
  if (force == DECO_KERNEL_DENSE) {
    // BF16 blocks only; an FP32 block (e.g. the FP32 polish) is planned as AUTO
    if (prec != DECO_PREC_BF16) return plan_phase(g, C, ld, prec, DECO_KERNEL_AUTO, plan);
    return plan_dense(g, C, want_k, want_t == 1, plan);
  }
  plan->threads = want_t == 1 ? 512 : 1024;
  plan->xmode = want_x == 1 ? 1 : 2;   // DSMEM broadcast or L2 exchange (default)
  plan->lean = want_lean;
  plan->pairs = want_pairs;
  if (force == DECO_KERNEL_GLOBAL) {
    if (want_pipe) plan->pipe = true;
    if (want_s) {
      // column slabs of width w, run one after another in a slab-major copy
      const int S = 1 << want_s;
      const int w = ((C + 8 * S - 1) / (8 * S)) * 8;
      if (w * S > ld) {
        set_error("%d column slabs do not fit ld = %d for C = %d", S, ld, C);
        return DECO_ERR_UNSUPPORTED;
      }
      plan->col_slabs = S;
      plan->slab_w = w;
    }
    if (plan->pipe) {
      static const int entries[4] = {16, 8, 24, 12};
      static const int stages[3] = {3, 2, 4};
      const int cols = plan->col_slabs > 1 ? plan->slab_w : C;
      const bool weighted = g->wmode != W_UNIT, gen = g->wmode == W_GENERAL;
      int rc = stream_shape(cols, prec, entries[pipe_e], stages[pipe_s], pipe_w, weighted, gen, pipe_mix, want_hints,
                            pipe_wide, &plan->stream);
      if (rc) return rc;
    }
    return DECO_OK;
  }
  const bool aligned = ld % cols == 0;
  const int max_smem = slab_max_smem();
  const int items = (C + cols - 1) / cols;
  const int sms = device_sm_count();
  double best = 0.0;
  // the replica alone must fit before any split is worth sizing
  const bool replica_fits = (size_t)g->n * 128 + 4096 <= (size_t)max_smem;
  for (int k = 1; k <= SLAB_MAX_CLUSTER && aligned && replica_fits; k *= 2) {
    if (k > g->n) break;
    if (want_k && k != want_k) continue;
    int32_t split[SLAB_MAX_CLUSTER + 1];
    slab_split(g->h_row_ptr.data(), g->n, k, split);
    int32_t max_own = 0;
    int64_t max_words = 0, max_edges = 0;
    image_sizes(g, k, split, &max_own, &max_words, &max_edges);
    if (max_words > (1 << 26)) continue;
    const size_t smem = slab_smem_bytes(g->n, max_own, (int)max_words, prec, want_lean);
    if (smem > (size_t)max_smem) continue;
    const int per_sm = std::max(1, std::min(4, (int)((size_t)(max_smem + 1024) / (smem + 1024))));
    const int waves = (int)((items * (int64_t)k + (int64_t)sms * per_sm - 1) / ((int64_t)sms * per_sm));
    const double cost = onchip_cost(max_edges, max_own, g->n, k, waves);
    if (plan->kernel != KERNEL_ONCHIP || cost < best) {
      best = cost;
      plan->kernel = KERNEL_ONCHIP;
      plan->k = k;
      plan->max_own = max_own;
      plan->max_img_words = (int32_t)max_words;
      plan->items = items;
    }
  }
  if (force == DECO_KERNEL_ONCHIP && plan->kernel != KERNEL_ONCHIP) {
    set_error("the on-chip kernel does not fit this graph (n=%d, nnz=%lld, ld=%d)", g->n,
              (long long)g->nnz, ld);
    return DECO_ERR_UNSUPPORTED;
  }
  return DECO_OK;
}

int PhaseRunner::prepare(const deco_graph* g_, int32_t C_, int32_t ld_, int prec_, int force,
                         cudaStream_t st) {
  (void)st;
  g = g_;
  C = C_;
  ld = ld_;
  prec = prec_;
  int rc = plan_phase(g, C, ld, prec, force, &plan);
  if (rc) return rc;
  if (plan.kernel == KERNEL_DENSE) {
    {
      std::lock_guard<std::mutex> lock(g_image_mutex);
      // the dense copy lives with the graph, like the on-chip CSR images
      if (!g->dense) {
        __nv_bfloat16* A = nullptr;
        if ((rc = dense_build(g, plan.kpad, &A, st))) return rc;
        const_cast<deco_graph*>(g)->dense = A;
        const_cast<deco_graph*>(g)->dense_ld = plan.kpad;
      }
    }
    const size_t elems = (size_t)plan.cpad * plan.kpad;
    for (int i = 0; i < 2; ++i) {
      cudaError_t e = cudaMallocAsync((void**)&yt[i], elems * 2, st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(transposed block)");
      // node padding of YT must stay zero (finite) for the products with A's zero columns
      if ((e = cudaMemsetAsync(yt[i], 0, elems * 2, st)) != cudaSuccess) return cuda_fail(e, "memset");
    }
    cudaError_t e = cudaMallocAsync((void**)&vt, elems * sizeof(float), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(transposed momentum)");
    if ((e = cudaMemsetAsync(vt, 0, elems * sizeof(float), st)) != cudaSuccess) return cuda_fail(e, "memset");
    maps = new (std::nothrow) DenseMaps;
    if (!maps) { set_error("out of host memory"); return DECO_ERR_OOM; }
    if (plan.dpersist) {
      if ((e = cudaMallocAsync((void**)&gbar, sizeof(unsigned int), st)) != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync(grid barrier)");
    }
    return dense_make_maps(g->dense, plan.kpad, yt, plan.cpad, plan.dpersist ? plan.dphase.w : 0, maps);
  }
  if (plan.kernel == KERNEL_GLOBAL && plan.pipe) {
    std::lock_guard<std::mutex> lock(g_image_mutex);
    // the record streams live with the graph, like the on-chip CSR images
    return stream_image(const_cast<deco_graph*>(g), plan.stream, &plan.rec);
  }
  if (plan.kernel != KERNEL_ONCHIP) return DECO_OK;
  {
    std::lock_guard<std::mutex> lock(g_image_mutex);
    // the image cache lives with the graph; building it does not change the
    // graph's meaning, only how the on-chip kernel reads it
    const SlabImage* im = nullptr;
    rc = slab_image(const_cast<deco_graph*>(g), plan.k, &im);
    if (rc) return rc;
    plan.image = *im;
  }
  if ((plan.k > 1 && plan.xmode == 2) || plan.lean) {
    const size_t bytes = 2 * (size_t)plan.items * g->n * 128;
    cudaError_t e = cudaMallocAsync((void**)&xbuf, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(exchange buffer)");
  }
  return DECO_OK;
}

int PhaseRunner::run(void* y[2], int& cur, float* v, int32_t steps, int objective, float alpha, float mu,
                     const float* alpha_cols, const int32_t* steps_cols, bool load_v, bool store_v,
                     int32_t* flag, cudaStream_t st, int64_t* kernels) {
  if (plan.kernel == KERNEL_ONCHIP) {
    SlabParams p{};
    SlabGraph& sg = p.g0;
    sg.n = g->n; sg.ld = ld; sg.C = C;
    sg.dnet = g->dnet;
    sg.image = reinterpret_cast<const uint4*>(plan.image.data);
    std::copy(plan.image.off, plan.image.off + SLAB_MAX_CLUSTER + 1, sg.img_off);
    std::copy(plan.image.split, plan.image.split + SLAB_MAX_CLUSTER + 1, sg.split);
    sg.y = y[cur];
    sg.v = v;
    sg.alpha_cols = alpha_cols;
    sg.steps_cols = steps_cols;
    sg.xbuf = xbuf;
    sg.nslabs = plan.items;
    p.graphs = nullptr;
    p.items = nullptr;
    p.k = plan.k;
    p.threads = plan.threads;
    p.xmode = plan.lean ? 2 : plan.xmode;
    p.lean = plan.lean ? 1 : 0;
    p.pairs = plan.pairs ? 1 : 0;
    p.steps = steps;
    const float fac = objective == DECO_OBJ_MULTILINEAR01 ? 2.0f : 1.0f;
    p.alpha = fac * alpha;
    p.afac = fac;
    p.mu = mu;
    p.objective = objective;
    p.load_v = load_v ? 1 : 0;
    p.store_v = store_v ? 1 : 0;
    p.max_n = g->n;
    p.max_own = plan.image.max_own;
    p.max_img_words = plan.image.max_words;
    p.flag = flag;
    int rc = launch_slab(p, plan.items, prec, g->wmode, st);
    if (rc) return rc;
    if (kernels) *kernels += 1;
    return DECO_OK;
  }
  if (plan.kernel == KERNEL_DENSE) {
    // transposed copy in, `steps` tensor-core steps ping-ponging yt[0] / yt[1], copy back
    const bool momv = mu != 0.0f && v != nullptr;
    const int32_t kpad = plan.kpad;
    int rc = dense_to_t(y[cur], g->n, ld, C, yt[0], kpad, 2, st);
    if (rc) return rc;
    if (momv) {
      if (load_v) rc = dense_to_t(v, g->n, ld, C, vt, kpad, 4, st);
      else if (cudaError_t e = cudaMemsetAsync(vt, 0, sizeof(float) * (size_t)plan.cpad * kpad, st))
        rc = cuda_fail(e, "memset");
      if (rc) return rc;
    }
    DenseStep p{};
    p.n = g->n;
    p.kpad = kpad;
    p.cpad = plan.cpad;
    p.C = C;
    p.ks = plan.ks;
    p.objective = objective;
    p.A = g->dense;
    p.VT = momv ? vt : nullptr;
    p.dnet = g->dnet;
    const float fac = objective == DECO_OBJ_MULTILINEAR01 ? 2.0f : 1.0f;
    p.alpha = fac * alpha;
    p.afac = fac;
    p.mu = momv ? mu : 0.0f;
    p.alpha_cols = alpha_cols;
    p.steps_cols = steps_cols;
    p.flag = flag;
    int c = 0;
    bool done = false;
    if (plan.dpersist) {
      rc = launch_dense_phase(p, *maps, yt, plan.dphase, steps, gbar, st);
      if (rc == DECO_OK) {
        done = true;
        c = steps & 1;
      } else if (rc == DECO_ERR_UNSUPPORTED) {
        clear_error();   // not every CTA can be resident now: one launch per step instead
      } else {
        return rc;
      }
    }
    for (int32_t t = 0; t < steps && !done; ++t) {
      p.YT = yt[c];
      p.YTout = yt[c ^ 1];
      p.t = t;
      if ((rc = launch_dense_step(p, *maps, c, st))) return rc;
      c ^= 1;
    }
    if ((rc = dense_from_t(yt[c], kpad, C, y[cur], g->n, ld, 2, st))) return rc;
    if (momv && store_v && (rc = dense_from_t(vt, kpad, C, v, g->n, ld, 4, st))) return rc;
    if (kernels) *kernels += (done ? 1 : steps) + 2 + (momv ? 1 + (store_v ? 1 : 0) : 0);
    return DECO_OK;
  }
  // one step: the pipelined form where planned, else the lane-group form
  auto step_launch = [&](const StepLaunch& s, cudaStream_t stream) -> int {
    if (plan.pipe) return launch_step_stream(s, *plan.rec, plan.stream, stream);
    return launch_step_global(s, stream);
  };
  StepLaunch sl{};
  sl.n = g->n; sl.C = C; sl.ld = ld;
  sl.precision = prec; sl.objective = objective; sl.wmode = g->wmode;
  sl.row_ptr = g->row_ptr; sl.col_idx = g->col_idx; sl.col_sw = g->col_sw; sl.w = g->w;
  sl.dnet = g->dnet;
  sl.v = v; sl.alpha = alpha; sl.mu = mu;
  sl.alpha_cols = alpha_cols; sl.steps_cols = steps_cols; sl.flag = flag;
  if (plan.col_slabs > 1 && steps > 0) {
    // Column-slab schedule: copy the block into S dense n x w slabs, run all
    // steps of one slab before the next (a narrow dense slab and the CSR stay
    // resident in L2), copy back.  Columns are independent (remark after
    // Eq. 11), so the arithmetic of every column is unchanged.
    const int S = plan.col_slabs, w = plan.slab_w;
    const size_t esz = prec == DECO_PREC_BF16 ? 2 : 4;
    const bool momv = mu != 0.0f && v != nullptr;
    if (!ypart) {
      cudaError_t e = cudaMallocAsync((void**)&ypart, (size_t)g->n * w * S * esz, st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(slab partner)");
    }
    // y[cur] is only read (into slab-major A) and, at the end, its columns
    // < C are rewritten; its padding columns are never touched
    unsigned char* A = static_cast<unsigned char*>(y[cur ^ 1]);   // slab-major data
    unsigned char* Bp = ypart;                                    // ping-pong partner
    int rc = launch_slab_layout(g->n, ld, C, w, S, esz, y[cur], A, true, st);
    if (rc) return rc;
    if (momv) {
      if (!vslab) {
        cudaError_t e = cudaMallocAsync((void**)&vslab, (size_t)g->n * w * S * sizeof(float), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(slab momentum)");
      }
      if ((rc = launch_slab_layout(g->n, ld, C, w, S, 4, v, vslab, true, st))) return rc;
    }
    for (int s = 0; s < S; ++s) {
      const int c0 = s * w;
      const int Cs = std::min(w, C - c0);
      if (Cs <= 0) break;
      sl.C = Cs;
      sl.ld = w;
      sl.alpha_cols = alpha_cols ? alpha_cols + c0 : nullptr;
      sl.steps_cols = steps_cols ? steps_cols + c0 : nullptr;
      sl.v = momv ? vslab + (size_t)c0 * g->n : nullptr;
      unsigned char* blk[2] = {A + (size_t)c0 * g->n * esz, Bp + (size_t)c0 * g->n * esz};
      int c = 0;
      for (int32_t t = 0; t < steps; ++t) {
        sl.yin = blk[c];
        sl.yout = blk[c ^ 1];
        sl.t = t;
        if ((rc = step_launch(sl, st))) return rc;
        c ^= 1;
      }
    }
    unsigned char* res = (steps % 2 == 0) ? A : Bp;
    if ((rc = launch_slab_layout(g->n, ld, C, w, S, esz, res, y[cur], false, st))) return rc;
    if (momv && (rc = launch_slab_layout(g->n, ld, C, w, S, 4, vslab, v, false, st))) return rc;
    if (kernels) *kernels += (int64_t)steps * S + 2 + (momv ? 2 : 0);
    return DECO_OK;
  }
  for (int32_t t = 0; t < steps; ++t) {
    sl.yin = y[cur];
    sl.yout = y[cur ^ 1];
    sl.t = t;
    int rc = step_launch(sl, st);
    if (rc) return rc;
    cur ^= 1;
  }
  if (kernels) *kernels += steps;
  return DECO_OK;
}

void PhaseRunner::release(cudaStream_t st) {
  if (xbuf) cudaFreeAsync(xbuf, st);
  if (vslab) cudaFreeAsync(vslab, st);
  if (ypart) cudaFreeAsync(ypart, st);
  for (auto& p : yt) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
  }
  if (vt) cudaFreeAsync(vt, st);
  vt = nullptr;
  delete maps;
  maps = nullptr;
  if (gbar) cudaFreeAsync(gbar, st);
  gbar = nullptr;
  xbuf = nullptr;
  vslab = nullptr;
  ypart = nullptr;
}

}  // namespace deco
