// Host side of the pipelined per-step kernel (step_stream.cuh): the launch
// shape, the per-warp record streams of a graph, and the launch.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "step_stream.cuh"

namespace deco {

int device_sm_count();

// the form with the shape read from the arguments (one vector per lane)
void* stream_kernel_runtime(int prec, int G, bool wt, int acc) { return stream_kernel_for<1, 0>(prec, G, wt, acc); }

namespace {

void* pick_kernel(int prec, int G, bool wt, int acc, int U, int fe) {
  if (fe == 8) return stream_kernel_e8(prec, G, wt, acc, U);
  if (fe == 12) return stream_kernel_e12(prec, G, wt, acc, U);
  return stream_kernel_runtime(prec, G, wt, acc);
}

// bytes of the per-warp areas of a shape
void stream_sizes(int G, int U, int prec, int maxe, int stages, bool mom, bool gen, int32_t* rw, uint32_t* group,
                  uint32_t* stage, size_t* per_warp) {
  const int NG = 32 / G, VN = prec == DECO_PREC_BF16 ? 8 : 4, W = 16 * G * U;
  *rw = stream_record_words(NG, maxe, gen);
  *group = (uint32_t)(maxe + 1) * W + (mom ? (uint32_t)(G * U * VN * 4) : 0u);
  // with two lanes per row, the four groups that one 128-byte shared-memory
  // wavefront serves must start in distinct 32-byte bank windows
  if (G == 2 && *group % 64 == 0) *group += 32;
  *stage = (uint32_t)NG * *group;
  *per_warp = (size_t)2 * stages * *rw * 4 + (size_t)stages * *stage;
}

}  // namespace

// lanes per row segment for C columns and U vectors per lane: enough lanes
// for the row's 16-byte vectors, at least 4 (2 in the wide form), at most 32
// (wider blocks run as column chunks of 32 U vectors)
int stream_group_lanes(int32_t C, int prec, int U) {
  const int VN = prec == DECO_PREC_BF16 ? 8 : 4;
  const int lanes = ((C + VN - 1) / VN + U - 1) / U;
  int G = U == 2 ? 2 : 4;
  while (G < lanes && G < 32) G <<= 1;
  return G;
}

int stream_shape(int32_t C, int prec, int maxe, int stages, int wpb, bool weighted, bool gen, bool mixed,
                 bool hints, bool wide, StreamShape* out) {
  if (maxe < 1 || maxe > 0xFFFF || stages < 2 || stages > 4 || wpb < 0 || wpb > 8) {
    set_error("pipelined step: bad shape (entries=%d, stages=%d, warps=%d)", maxe, stages, wpb);
    return DECO_ERR_ARG;
  }
  StreamShape sh;
  // the compile-time form where the shape has one: 8 or 12 entries, 2 stages
  sh.fe = (stages == 2 && (maxe == 8 || maxe == 12)) ? maxe : 0;
  sh.U = wide ? 2 : 1;
  if (wide && !sh.fe) {
    set_error("the wide pipelined step runs 8 or 12 entries per item in 2 stages");
    return DECO_ERR_UNSUPPORTED;
  }
  sh.G = stream_group_lanes(C, prec, sh.U);
  sh.maxe = maxe;
  sh.stages = stages;
  sh.gen = gen;
  sh.weighted = weighted;
  sh.acc = (mixed && prec == DECO_PREC_BF16 && !weighted) ? 1 : 0;
  sh.hints = hints;
  int32_t rw;
  uint32_t group, stage;
  size_t per_warp, per_warp_mom;
  stream_sizes(sh.G, sh.U, prec, maxe, stages, false, gen, &rw, &group, &stage, &per_warp);
  stream_sizes(sh.G, sh.U, prec, maxe, stages, true, gen, &rw, &group, &stage, &per_warp_mom);
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // Warps per block: every warp keeps its own items in flight, so the shape
  // that keeps the most warps resident per SM wins (shared memory and
  // registers decide); a block must also fit with the momentum slots.  The
  // grid is sized for the layout without them (a phase with momentum then
  // takes a little more than one wave).
  void* fn = pick_kernel(prec, sh.G, weighted, sh.acc, sh.U, sh.fe);
  if (!fn) {
    set_error("pipelined step: no kernel for %d lanes per row and %d vectors per lane", sh.G, sh.U);
    return DECO_ERR_UNSUPPORTED;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return cuda_fail(e, "pipelined step shared memory");
  auto resident = [&](int w, int* per_sm) -> cudaError_t {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, 32 * w, per_warp * w);
  };
  int per_sm = 0;
  if (!wpb) {
    int best_warps = 0;
    for (int w = 8; w >= 1; --w) {
      if (per_warp_mom * w > (size_t)max_smem) continue;
      int b = 0;
      if ((e = resident(w, &b)) != cudaSuccess) return cuda_fail(e, "pipelined step occupancy");
      if (b * w > best_warps) { best_warps = b * w; wpb = w; per_sm = b; }
    }
  } else if (per_warp_mom * wpb <= (size_t)max_smem) {
    if ((e = resident(wpb, &per_sm)) != cudaSuccess) return cuda_fail(e, "pipelined step occupancy");
  }
  if (!wpb || per_warp_mom * wpb > (size_t)max_smem) {
    set_error("the pipelined step kernel does not fit %d warps of %d entries x %d stages", wpb, maxe, stages);
    return DECO_ERR_UNSUPPORTED;
  }
  sh.wpb = wpb;
  sh.blocks = std::max(1, per_sm) * device_sm_count();
  sh.nw = sh.blocks * wpb;
  *out = sh;
  return DECO_OK;
}

namespace {

// Fills the records of the per-warp streams: one thread per (slice, row of
// the slice), writing that row's fields in every part of the slice; the
// slice's first record is srec[s], its rows order[s ng ...] (-1 past n), its
// first row the longest (it gives every part's kmax and the number of parts).
__global__ void k_stream_fill(int32_t n, int32_t nslices, int ng, int maxe, int rw, int wmode, bool gen,
                              const int32_t* __restrict__ order, const int64_t* __restrict__ srec,
                              const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                              const uint32_t* __restrict__ col_sw, const float* __restrict__ w, uint32_t* rec) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)nslices * ng) return;
  const int32_t s = (int32_t)(tid / ng);
  const int i = (int)(tid % ng);
  const int64_t rr = (int64_t)s * ng + i;
  const int32_t v = rr < n ? order[rr] : -1;
  const int32_t v0 = order[(int64_t)s * ng];
  const int32_t d0 = row_ptr[v0 + 1] - row_ptr[v0];
  const int parts = d0 > maxe ? (d0 + maxe - 1) / maxe : 1;
  const int32_t d = v >= 0 ? row_ptr[v + 1] - row_ptr[v] : 0;
  const int E0 = 1 + 2 * ng, words = E0 + maxe * ng * (gen ? 2 : 1);
  for (int p = 0; p < parts; ++p) {
    uint32_t* r = rec + (size_t)(srec[s] + p) * rw;
    const int32_t cnt = max(0, min(maxe, d - p * maxe));
    r[1 + i] = (uint32_t)v;
    r[1 + ng + i] = (uint32_t)cnt | (p == 0 ? 0x10000u : 0u) | (p == parts - 1 ? 0x20000u : 0u);
    const int32_t e0 = v >= 0 ? row_ptr[v] + p * maxe : 0;
    for (int k = 0; k < maxe; ++k) {
      uint32_t c = REC_PAD;
      float wt = 0.0f;
      if (k < cnt) {
        c = wmode == W_SIGN ? col_sw[e0 + k] : (uint32_t)col_idx[e0 + k];
        if (gen) wt = w[e0 + k];
      }
      r[E0 + k * ng + i] = c;
      if (gen) r[E0 + maxe * ng + k * ng + i] = __float_as_uint(wt);
    }
    if (i == 0) {
      r[0] = (uint32_t)max(0, min(maxe, d0 - p * maxe));   // kmax: the count of the slice's longest row
      for (int k = words; k < rw; ++k) r[k] = 0u;           // padding
    }
  }
}

}  // namespace

int stream_image(deco_graph* g, const StreamShape& sh, const StreamImage** out) {
  const int ng = 32 / sh.G;
  for (auto& im : g->streams)
    if (im.ng == ng && im.maxe == sh.maxe && im.nw == sh.nw && im.gen == sh.gen) { *out = &im; return DECO_OK; }
  const int32_t n = g->n;
  const int maxe = sh.maxe;
  const bool gen = sh.gen;
  StreamImage im;
  im.ng = ng;
  im.maxe = maxe;
  im.nw = sh.nw;
  im.gen = gen;
  im.rw = stream_record_words(ng, maxe, gen);
  // rows by degree, largest first; ties keep the row order (a counting sort)
  auto deg = [&](int32_t v) { return g->h_row_ptr[v + 1] - g->h_row_ptr[v]; };
  int32_t dmax = 0;
  for (int32_t v = 0; v < n; ++v) dmax = std::max(dmax, deg(v));
  std::vector<int64_t> start((size_t)dmax + 2, 0);
  for (int32_t v = 0; v < n; ++v) ++start[(size_t)(dmax - deg(v)) + 1];
  for (size_t d = 1; d < start.size(); ++d) start[d] += start[d - 1];
  std::vector<int32_t> order((size_t)n);
  for (int32_t v = 0; v < n; ++v) order[(size_t)start[(size_t)(dmax - deg(v))]++] = v;
  const int32_t nslices = (n + ng - 1) / ng;
  // records per warp: slice s belongs to warp s mod nw, its parts consecutive
  std::vector<int64_t> count((size_t)im.nw + 1, 0);
  auto parts_of = [&](int32_t s) {
    const int32_t w = deg(order[(size_t)s * ng]);   // the slice's first row is its longest
    return w > maxe ? (w + maxe - 1) / maxe : 1;
  };
  for (int32_t s = 0; s < nslices; ++s) count[s % im.nw] += parts_of(s);
  std::vector<int32_t> soff((size_t)im.nw + 1, 0);
  int64_t acc = 0;
  for (int w = 0; w < im.nw; ++w) {
    soff[w] = (int32_t)acc;
    acc += count[w];
  }
  soff[im.nw] = (int32_t)acc;
  if (acc * im.rw > ((int64_t)1 << 31)) {
    set_error("the pipelined step kernel's records exceed 2^31 words (n=%d)", n);
    return DECO_ERR_UNSUPPORTED;
  }
  // the first record of every slice (a slice's parts are consecutive in its
  // warp's stream); the records themselves are filled on the device
  std::vector<int64_t> srec((size_t)std::max(nslices, 1), 0);
  {
    std::vector<int64_t> fill(soff.begin(), soff.end());
    for (int32_t s = 0; s < nslices; ++s) {
      const int w = s % im.nw;
      srec[(size_t)s] = fill[(size_t)w];
      fill[(size_t)w] += parts_of(s);
    }
  }
  const size_t rec_words = (size_t)std::max<int64_t>(acc, 1) * im.rw;
  int32_t* d_order = nullptr;
  int64_t* d_srec = nullptr;
  cudaError_t e = cudaMalloc((void**)&im.rec, rec_words * 4);
  if (e == cudaSuccess && acc == 0) e = cudaMemset(im.rec, 0, rec_words * 4);
  if (e == cudaSuccess && nslices > 0) {
    e = cudaMalloc((void**)&d_order, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_srec, (size_t)nslices * 8);
    if (e == cudaSuccess) e = cudaMemcpy(d_order, order.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_srec, srec.data(), (size_t)nslices * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      const int64_t threads = (int64_t)nslices * ng;
      k_stream_fill<<<(unsigned)((threads + 255) / 256), 256>>>(n, nslices, ng, maxe, im.rw, g->wmode, gen, d_order,
                                                                 d_srec, g->row_ptr, g->col_idx, g->col_sw, g->w,
                                                                 im.rec);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // the records outlive this call's ordering
  }
  cudaFree(d_order);
  cudaFree(d_srec);
  if (e == cudaSuccess) e = cudaMalloc((void**)&im.soff, soff.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(im.soff, soff.data(), soff.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_stream_image(im);
    return cuda_fail(e, "sliced record image");
  }
  im.records = acc;
  g->streams.push_back(std::move(im));
  *out = &g->streams.back();
  return DECO_OK;
}

void free_stream_image(StreamImage& im) {
  cudaFree(im.rec);
  cudaFree(im.soff);
  im.rec = nullptr;
  im.soff = nullptr;
}

int launch_step_stream(const StepLaunch& s, const StreamImage& im, const StreamShape& sh, cudaStream_t st) {
  if (s.n == 0 || s.C == 0) return DECO_OK;
  if (s.ld % 8 != 0 || im.ng * sh.G != 32 || im.maxe != sh.maxe || im.nw != sh.nw) {
    set_error("pipelined step: image and shape disagree (ld=%d)", s.ld);
    return DECO_ERR_ARG;
  }
  const int VN = s.precision == DECO_PREC_BF16 ? 8 : 4;
  const bool mom = s.mu != 0.0f;
  StreamArgs a{};
  a.n = s.n;
  a.C = s.C;
  a.ld = s.ld;
  a.ncc = (s.C + sh.G * sh.U * VN - 1) / (sh.G * sh.U * VN);
  if ((int64_t)im.records * a.ncc >= ((int64_t)1 << 31)) {
    set_error("pipelined step: %lld records x %d column chunks exceed 2^31 items", (long long)im.records, a.ncc);
    return DECO_ERR_UNSUPPORTED;
  }
  a.maxe = sh.maxe;
  a.stages = sh.stages;
  size_t per_warp;
  stream_sizes(sh.G, sh.U, s.precision, sh.maxe, sh.stages, mom, im.gen, &a.rw, &a.group_bytes, &a.stage_bytes,
               &per_warp);
  a.rec = im.rec;
  a.soff = im.soff;
  a.dnet = s.dnet;
  a.yin = s.yin;
  a.yout = s.yout;
  a.v = s.v;
  const float fac = s.objective == DECO_OBJ_MULTILINEAR01 ? 2.0f : 1.0f;
  a.alpha_eff = fac * s.alpha;
  a.afac = fac;
  a.mu = s.mu;
  a.alpha_cols = s.alpha_cols;
  a.steps_cols = s.steps_cols;
  a.t = s.t;
  a.flag = s.flag;
  a.lap = s.objective == DECO_OBJ_LAPLACIAN;
  a.mom = mom;
  a.gen = im.gen;
  a.hints = sh.hints ? 1 : 0;
  const size_t smem = per_warp * sh.wpb;
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)max_smem) {
    set_error("pipelined step: %zu bytes of shared memory exceed the %d available", smem, max_smem);
    return DECO_ERR_UNSUPPORTED;
  }
  void* fn = pick_kernel(s.precision, sh.G, sh.weighted, sh.acc, sh.U, sh.fe);
  void* args[] = {&a};
  cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)sh.blocks), dim3(32 * sh.wpb), args, smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "k_step_stream launch");
  return DECO_OK;
}

}  // namespace deco
