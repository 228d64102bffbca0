// deco_solve: the whole pDECO schedule (Alg. 3) on the device.
//
// Per phase k: starting block (phase 0: the requested initialisation; later
// phases: Gaussian around 2 z* - 1 of the previous phase's best, Sec. 4.2, or
// a fresh start of the first phase's kind), T_k projected gradient steps
// (phase runner: persistent on-chip, per-step global or dense kernel; run in
// segments of eval_every steps when intermediate roundings are asked for),
// rounding (Eq. 5 / 11), integer cuts (Eq. 1), argmax and the global best
// record -- all stream-ordered, with one host synchronisation at the end.
#include <algorithm>
#include <memory>
#include <vector>

#include "api_util.cuh"
#include "deco_internal.cuh"
#include "phase.cuh"

using namespace deco;

namespace {

struct RunnerCache {
  std::vector<std::unique_ptr<PhaseRunner>> runners;
  cudaStream_t st;
  explicit RunnerCache(cudaStream_t s) : st(s) {}
  ~RunnerCache() {
    for (auto& r : runners) r->release(st);
  }
  int get(const deco_graph* g, int32_t C, int32_t ld, int prec, int force, PhaseRunner** out) {
    for (auto& r : runners) {
      if (r->C == C && r->prec == prec) { *out = r.get(); return DECO_OK; }
    }
    runners.emplace_back(new PhaseRunner());
    int rc = runners.back()->prepare(g, C, ld, prec, force, st);
    *out = runners.back().get();
    return rc;
  }
};

}  // namespace

extern "C" int deco_solve(const deco_graph* g, int32_t B, const deco_phase* phases, int32_t n_phases,
                          const deco_params* p, uint64_t seed, const float* x0, const float* mean,
                          uint8_t* assignment, int64_t* phase_cuts, void* stream, deco_result* out) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (!phases || !p || !out) { set_error("NULL argument"); return DECO_ERR_ARG; }
  if (B < 1 || n_phases < 1 || n_phases > 64) { set_error("need B >= 1 and 1 <= n_phases <= 64"); return DECO_ERR_ARG; }
  if ((rc = check_prec(p->precision)) || (rc = check_obj(p->objective))) return rc;
  if (!valid_selector(p->kernel)) { set_error("bad kernel selector 0x%x", p->kernel); return DECO_ERR_ARG; }
  if (p->local_search < 0) { set_error("local_search must be >= 0"); return DECO_ERR_ARG; }
  if (p->phase_init != DECO_PHASE_INIT_BEST && p->phase_init != DECO_PHASE_INIT_FRESH) {
    set_error("bad phase_init %d", p->phase_init);
    return DECO_ERR_ARG;
  }
  if (p->phase_init == DECO_PHASE_INIT_FRESH && p->init == DECO_INIT_EXPLICIT) {
    set_error("fresh later phases need a drawn initialisation, not an explicit block");
    return DECO_ERR_ARG;
  }
  if (p->eval_every < 0) { set_error("eval_every must be >= 0"); return DECO_ERR_ARG; }
  int32_t max_lift = 1;
  bool any_mom = false;
  for (int k = 0; k < n_phases; ++k) {
    if (phases[k].lift < 1 || phases[k].lift > 64 || phases[k].steps < 0) {
      set_error("phase %d: need 1 <= lift <= 64 and steps >= 0", k);
      return DECO_ERR_ARG;
    }
    max_lift = std::max(max_lift, phases[k].lift);
    any_mom = any_mom || phases[k].momentum != 0.0f;
  }
  if (p->init < DECO_INIT_UNIFORM || p->init > DECO_INIT_MEAN) { set_error("bad init %d", p->init); return DECO_ERR_ARG; }
  if (p->init == DECO_INIT_EXPLICIT && !x0) { set_error("explicit init needs x0"); return DECO_ERR_ARG; }
  if (p->init == DECO_INIT_MEAN && !mean) { set_error("mean init needs mean"); return DECO_ERR_ARG; }
  if ((int64_t)B * max_lift > (1 << 24)) { set_error("B * lift too large"); return DECO_ERR_ARG; }

  cudaStream_t st = as_stream(stream);
  const int32_t n = g->n;
  const int32_t Cmax = B * max_lift;
  const int32_t ld = (Cmax + 63) / 64 * 64;   // 128-byte slabs for the on-chip kernel
  const int32_t W = (B + 31) / 32;
  const size_t block_elems = (size_t)n * ld;
  const bool polish = p->precision == DECO_PREC_BF16 && p->polish_steps > 0;

  int64_t hbuf[4] = {0, 0, 0, 0};
  float ms = 0.0f;
  int64_t edge_updates = 0, kernels = 0;
  {
    Scratch s(st);
    RunnerCache runners(st);
    void* ybuf[2] = {nullptr, nullptr};
    float* vbuf = nullptr;
    uint32_t* zbits = nullptr;
    int64_t* cuts = nullptr;
    int32_t* best_idx = nullptr;
    BestRecord* rec = nullptr;
    uint8_t* pbz = nullptr;
    uint8_t* bz = nullptr;
    float* h = nullptr;
    int8_t* side = nullptr;
    int32_t* flag = nullptr;
    float* dx0 = nullptr;
    float* dmean = nullptr;
    const size_t ybytes = block_elems * (polish ? 4 : elem_size(p->precision));
    if ((rc = s.alloc(&ybuf[0], ybytes)) || (rc = s.alloc(&ybuf[1], ybytes))) return rc;
    DECO_CUDA_TRY(cudaMemsetAsync(ybuf[0], 0, ybytes, st));   // padding columns stay finite
    DECO_CUDA_TRY(cudaMemsetAsync(ybuf[1], 0, ybytes, st));
    if (any_mom && (rc = s.alloc(&vbuf, block_elems * sizeof(float)))) return rc;
    if ((rc = s.alloc(&zbits, sizeof(uint32_t) * (size_t)n * W))) return rc;
    if ((rc = s.alloc(&cuts, sizeof(int64_t) * (size_t)B * (n_phases + 1)))) return rc;   // + intermediate roundings
    if ((rc = s.alloc(&best_idx, sizeof(int32_t) * (size_t)(n_phases + 1)))) return rc;
    if ((rc = s.alloc(&rec, sizeof(BestRecord)))) return rc;
    if ((rc = s.alloc(&pbz, (size_t)n)) || (rc = s.alloc(&bz, (size_t)n))) return rc;
    if ((rc = s.alloc(&h, sizeof(float) * n)) || (rc = s.alloc(&side, (size_t)n))) return rc;
    if ((rc = s.alloc(&flag, sizeof(int32_t)))) return rc;
    int32_t* ls_gains = nullptr;
    int32_t* ls_changed = nullptr;
    if (p->local_search > 0) {
      if ((rc = s.alloc(&ls_gains, sizeof(int32_t) * (size_t)n * 32 * W)) ||
          (rc = s.alloc(&ls_changed, sizeof(int32_t) * ((size_t)p->local_search + 1))))
        return rc;
    }

    cudaEvent_t ev0, ev1;
    DECO_CUDA_TRY(cudaEventCreate(&ev0));
    DECO_CUDA_TRY(cudaEventCreate(&ev1));
    struct EvGuard {
      cudaEvent_t a, b;
      ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evg{ev0, ev1};

    const int32_t C0 = B * phases[0].lift;
    if (p->init == DECO_INIT_EXPLICIT) {
      if ((rc = s.alloc(&dx0, block_elems * sizeof(float)))) return rc;
      DECO_CUDA_TRY(cudaMemcpy2DAsync(dx0, sizeof(float) * ld, x0, sizeof(float) * C0, sizeof(float) * C0, n,
                                      is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    }
    if (p->init == DECO_INIT_MEAN) {
      if (is_device_ptr(mean)) {
        dmean = const_cast<float*>(mean);
      } else {
        if ((rc = s.alloc(&dmean, sizeof(float) * n))) return rc;
        DECO_CUDA_TRY(cudaMemcpyAsync(dmean, mean, sizeof(float) * n, cudaMemcpyHostToDevice, st));
      }
    }
    // plan every distinct block shape before the timed region
    for (int32_t k = 0; k < n_phases; ++k) {
      PhaseRunner* R = nullptr;
      const int prec0 = (polish && phases[k].steps <= p->polish_steps) ? DECO_PREC_FP32 : p->precision;
      if ((rc = runners.get(g, B * phases[k].lift, ld, prec0, p->kernel, &R))) return rc;
      if (polish && (rc = runners.get(g, B * phases[k].lift, ld, DECO_PREC_FP32, p->kernel, &R))) return rc;
    }
    NvtxRange r_solve("deco_solve");
    DECO_CUDA_TRY(cudaEventRecord(ev0, st));
    DECO_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t), st));

    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    bool first_eval = true;   // the first rounding of the solve initialises the record
    int64_t* ecuts = cuts + (size_t)B * n_phases;   // intermediate roundings' cuts
    for (int32_t k = 0; k < n_phases; ++k) {
      const deco_phase& ph = phases[k];
      NvtxRange r_phase(ph.lift > 1 ? "deco phase (lifted)" : "deco phase (unlifted)");
      const int32_t C = B * ph.lift;
      InitLaunch il{};
      fill_init(il, g, B, ph.lift, ld, p, seed, k);
      il.y = ybuf[0];
      if (k == 0 || p->phase_init == DECO_PHASE_INIT_FRESH) {
        // the first phase's initialisation (later phases: draws with phase index k)
        switch (p->init) {
          case DECO_INIT_EXPLICIT: il.x0 = dx0; break;
          case DECO_INIT_MEAN: il.mean = dmean; break;
          case DECO_INIT_DUI:
            if ((rc = launch_dui(g, k0, k1, k, h, st))) return rc;
            kernels += 1;
            il.mean = h;
            break;
          case DECO_INIT_IDI:
          case DECO_INIT_IDI_HALF_UNIFORM:
            if ((rc = launch_idi(g, idi_threshold(g, p->beta), k0, k1, k, h, side, st))) return rc;
            kernels += 2;
            il.mean = h;
            break;
          default: break;
        }
      } else {
        il.init = DECO_INIT_MEAN;   // Gaussian around 2 z* - 1 of the previous phase
        il.mean_bits = pbz;
      }
      int prec = (polish && ph.steps <= p->polish_steps) ? DECO_PREC_FP32 : p->precision;
      il.precision = prec;
      if ((rc = launch_init(il, st))) return rc;
      kernels += 1;
      const bool mom = ph.momentum != 0.0f;
      if (mom) DECO_CUDA_TRY(cudaMemsetAsync(vbuf, 0, block_elems * sizeof(float), st));

      int cur = 0;
      PhaseRunner* R = nullptr;
      if ((rc = runners.get(g, C, ld, prec, p->kernel, &R))) return rc;
      const int32_t T = ph.steps;
      const int32_t main_steps = (prec == DECO_PREC_BF16 && polish) ? T - p->polish_steps : T;
      // rounding, cuts and the record (phase best vector only for the final rounding)
      auto evaluate = [&](int64_t* cut_out, int32_t* idx, uint8_t* phase_best) -> int {
        NvtxRange r_eval("deco round + cut + argmax");
        int e = launch_pack(g, B, ph.lift, ld, prec, ybuf[cur], zbits, st);
        if (e) return e;
        if (p->local_search > 0) {
          // 1-flip polish of the rounded vectors (off by default)
          if ((e = launch_local_search(g, B, zbits, p->local_search, ls_gains, ls_changed, st))) return e;
          kernels += 2 * (int64_t)p->local_search;
        }
        if ((e = launch_cut_bits(g, B, zbits, cut_out, st))) return e;
        if ((e = launch_phase_finish(g, B, k, first_eval, cut_out, zbits, idx, rec, phase_best, bz, st))) return e;
        first_eval = false;
        kernels += 5;   // pack, cut, argmax, record, extract
        return DECO_OK;
      };
      // steps in segments that end at the intermediate roundings (every
      // eval_every steps) and at the switch to the FP32 polish
      const int32_t E = p->eval_every;
      for (int32_t s = 0; s < T;) {
        int32_t next = T;
        if (E > 0) next = std::min(next, (s / E + 1) * E);
        if (s < main_steps) next = std::min(next, main_steps);
        NvtxRange r_steps("deco steps");
        if ((rc = R->run(ybuf, cur, vbuf, next - s, p->objective, ph.alpha, ph.momentum, nullptr, nullptr, mom,
                         mom, flag, st, &kernels)))
          return rc;
        s = next;
        if (E > 0 && s < T && s % E == 0 && (rc = evaluate(ecuts, best_idx + n_phases, nullptr))) return rc;
        if (s == main_steps && s < T) {
          // FP32 polish: widen the BF16 iterate and finish the phase in FP32
          if ((rc = convert_bf16_to_f32((int64_t)block_elems, ybuf[cur], static_cast<float*>(ybuf[cur ^ 1]), st)))
            return rc;
          kernels += 1;
          cur ^= 1;
          prec = DECO_PREC_FP32;
          if ((rc = runners.get(g, C, ld, prec, p->kernel, &R))) return rc;
        }
      }
      edge_updates += g->nnz * (int64_t)C * T;
      if ((rc = evaluate(cuts + (size_t)k * B, best_idx + k, pbz))) return rc;
    }
    DECO_CUDA_TRY(cudaEventRecord(ev1, st));

    BestRecord hrec{};
    int32_t hflag = 0;
    DECO_CUDA_TRY(cudaMemcpyAsync(&hrec, rec, sizeof(BestRecord), cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (assignment) DECO_CUDA_TRY(cudaMemcpyAsync(assignment, bz, (size_t)n, cudaMemcpyDeviceToHost, st));
    if (phase_cuts)
      DECO_CUDA_TRY(cudaMemcpyAsync(phase_cuts, cuts, sizeof(int64_t) * (size_t)B * n_phases,
                                    cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaStreamSynchronize(st));
    DECO_CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
    if (hflag & 2) {
      set_error("a bounded device wait of the on-chip or dense kernel gave up");
      return DECO_ERR_TIMEOUT;
    }
    if (hflag) {
      set_error("a non-finite value appeared in the iterate");
      return DECO_ERR_NONFINITE;
    }
    hbuf[0] = hrec.cut;
    hbuf[1] = hrec.init;
    hbuf[2] = hrec.phase;
  }
  out->best_cut = hbuf[0];
  out->best_init = (int32_t)hbuf[1];
  out->best_phase = (int32_t)hbuf[2];
  out->edge_updates = edge_updates;
  out->device_ms = ms;
  out->kernel_launches = kernels;
  return DECO_OK;
}

extern "C" int deco_solve_budget(const deco_graph* g, int32_t B, const deco_phase* phases, int32_t n_phases,
                                 const deco_params* p, uint64_t seed, double budget_ms, int32_t max_repeats,
                                 const uint8_t* warm, uint8_t* assignment, int32_t* repeats, void* stream,
                                 deco_result* out) {
  clear_error();
  int rc = check_graph(g);
  if (rc) return rc;
  if (!p || !out || !phases) { set_error("NULL argument"); return DECO_ERR_ARG; }
  if (max_repeats < 1 || !(budget_ms >= 0.0)) { set_error("need max_repeats >= 1 and budget_ms >= 0"); return DECO_ERR_ARG; }
  const int32_t n = g->n;
  std::vector<uint8_t> best_z((size_t)n, 0), z((size_t)n, 0);
  std::vector<float> mean((size_t)n, 0.0f);
  deco_result total{};
  total.best_cut = -1;   // below any cut: the first repetition always records its best
  total.best_init = -1;
  total.best_phase = -1;
  bool have_best = false;
  if (warm) {
    for (int32_t v = 0; v < n; ++v) best_z[v] = warm[v] ? 1 : 0;
    if ((rc = deco_eval_cut(g, best_z.data(), &total.best_cut))) return rc;
    have_best = true;
  }
  int32_t r = 0;
  double used = 0.0;
  for (; r < max_repeats; ++r) {
    deco_params pr = *p;
    const float* m = nullptr;
    if (have_best) {
      // Gaussian starts around 2 z* - 1 of the best vector so far (Sec. 4.2)
      for (int32_t v = 0; v < n; ++v) mean[v] = best_z[v] ? 1.0f : -1.0f;
      pr.init = DECO_INIT_MEAN;
      m = mean.data();
    }
    deco_result res{};
    if ((rc = deco_solve(g, B, phases, n_phases, &pr, seed + (uint64_t)r, nullptr, m, z.data(), nullptr, stream,
                         &res)))
      return rc;
    if (res.best_cut > total.best_cut) {   // strictly better: earlier repetitions win ties
      total.best_cut = res.best_cut;
      total.best_init = res.best_init;
      total.best_phase = res.best_phase;
      best_z = z;
    }
    have_best = true;
    total.edge_updates += res.edge_updates;
    total.device_ms += res.device_ms;
    total.kernel_launches += res.kernel_launches;
    used += res.device_ms;
    if (used >= budget_ms) {
      ++r;
      break;
    }
  }
  if (assignment) std::copy(best_z.begin(), best_z.end(), assignment);
  if (repeats) *repeats = r;
  *out = total;
  return DECO_OK;
}
