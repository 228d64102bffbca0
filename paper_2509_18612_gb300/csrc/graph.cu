// Graph handle: host-side validation of the CSR, device upload, error state.
// Def. 1 / Eq. 1 (undirected graph, each crossing edge counted once) and the
// Sec. 2 notation (A symmetric adjacency, D degree matrix, L = D - A).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "deco_internal.cuh"

namespace deco {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  cudaGetLastError();  // clear the sticky-free error state of the runtime
  return e == cudaErrorMemoryAllocation ? DECO_ERR_OOM : DECO_ERR_CUDA;
}

double idi_threshold(const deco_graph* g, float beta) {
  // Sec. 4.1.2: I = {v : d_v > mean + beta * sigma}, population moments.
  // Integer power sums make the FP64 mean and variance independent of the
  // summation order.
  const double n = (double)g->n;
  const double mean = (double)g->deg_s1 / n;
  const long double num = (long double)g->n * (long double)g->deg_s2 -
                          (long double)g->deg_s1 * (long double)g->deg_s1;
  const double var = (double)(int64_t)num / ((double)g->n * (double)g->n);
  return mean + (double)beta * std::sqrt(var);
}

static void free_graph(deco_graph* g) {
  if (!g) return;
  for (auto& im : g->images) cudaFree(im.data);
  for (auto& im : g->streams) free_stream_image(im);
  cudaFree(g->dense);
  cudaFree(g->row_ptr);
  cudaFree(g->col_idx);
  cudaFree(g->col_sw);
  cudaFree(g->w);
  cudaFree(g->wint);
  cudaFree(g->dnet);
  cudaFree(g->deg);
  delete g;
}

}  // namespace deco

using namespace deco;

extern "C" const char* deco_last_error(void) { return g_err; }

extern "C" int deco_abi_version(void) { return DECO_ABI_VERSION; }

extern "C" int deco_create_graph(int32_t n, int64_t nnz, const int32_t* row_ptr,
                                 const int32_t* col_idx, const float* weights, uint32_t flags,
                                 deco_graph** out) {
  return deco::create_graph_impl(n, nnz, row_ptr, col_idx, weights, flags, false, out);
}

namespace {

// The lowest row v that stores an entry (v, u) whose mirror (u, v) is
// missing (binary search of row u), into *bad_row (atomicMin; left alone when
// every entry has its mirror).  One warp per row, its lanes over the row's
// entries; the indices are already known to lie in [0, n).
__global__ void k_symmetry(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           int32_t* bad_row) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    bool miss = false;
    const int32_t e1 = rp[v + 1];
    for (int32_t e = rp[v] + lane; e < e1; e += 32) {
      const int32_t u = ci[e];
      int32_t lo = rp[u], hi = rp[u + 1];
      const int32_t end = hi;
      while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (ci[mid] < (int32_t)v) lo = mid + 1; else hi = mid;
      }
      if (lo >= end || ci[lo] != (int32_t)v) miss = true;
    }
    if (__any_sync(0xFFFFFFFFu, miss) && lane == 0) atomicMin(bad_row, (int32_t)v);
  }
}

}  // namespace

// `device_order`: the rows come from validated graphs in device edge order
// (a +-1 row lists its positive entries first), so sortedness is not checked.
int deco::create_graph_impl(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                            const float* weights, uint32_t flags, bool device_order, deco_graph** out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return DECO_ERR_ARG; }
  if (n < 1) { set_error("n must be >= 1 (got %d)", n); return DECO_ERR_ARG; }
  if (nnz < 0 || nnz >= ((int64_t)1 << 31)) {
    set_error("nnz must be in [0, 2^31) (got %lld)", (long long)nnz);
    return DECO_ERR_ARG;
  }
  if (!row_ptr) { set_error("row_ptr is NULL"); return DECO_ERR_ARG; }
  if (nnz > 0 && !col_idx) { set_error("col_idx is NULL"); return DECO_ERR_ARG; }

  // ---- structure: row_ptr non-decreasing first (so every row's entries lie
  // inside col_idx), then the entries of all rows, split over the host's
  // cores; the error reported is the one of the lowest row, as a single pass
  // would find it.
  if (row_ptr[0] != 0) { set_error("row_ptr[0] = %d, expected 0", row_ptr[0]); return DECO_ERR_GRAPH; }
  if ((int64_t)row_ptr[n] != nnz) {
    set_error("row_ptr[n] = %d, expected nnz = %lld", row_ptr[n], (long long)nnz);
    return DECO_ERR_GRAPH;
  }
  for (int32_t v = 0; v < n; ++v) {
    if (row_ptr[v + 1] < row_ptr[v]) {
      set_error("row_ptr decreases at row %d", v);
      return DECO_ERR_GRAPH;
    }
  }
  {
    struct Bad { int32_t row = -1, e = 0, u = 0, kind = 0; };   // kind 1 range, 2 self loop, 3 order
    std::vector<Bad> bad(std::max<unsigned>(1, std::thread::hardware_concurrency()));
    host_parallel(n, nnz, [&](int t, int64_t r0, int64_t r1) {
      for (int32_t v = (int32_t)r0; v < (int32_t)r1; ++v) {
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
          const int32_t u = col_idx[e];
          const int kind = (u < 0 || u >= n) ? 1 : u == v ? 2
                           : (!device_order && e > row_ptr[v] && col_idx[e - 1] >= u) ? 3 : 0;
          if (kind) { bad[t] = Bad{v, e, u, kind}; return; }
        }
      }
    });
    for (const Bad& b : bad) {
      if (b.row < 0) continue;
      if (b.kind == 1) set_error("col_idx[%d] = %d out of range (row %d)", b.e, b.u, b.row);
      else if (b.kind == 2) set_error("self loop at row %d", b.row);
      else set_error("row %d: column indices not strictly increasing at entry %d", b.row, b.e);
      return DECO_ERR_GRAPH;
    }
  }
  // ---- weights: nonzero integers, |w| <= 2^20 (exact in FP32 sums and in int cut sums)
  bool all_unit = true, all_pm1 = true;
  float max_abs_w = 1.0f;
  if (weights) {
    for (int64_t e = 0; e < nnz; ++e) {
      float x = weights[e];
      if (!std::isfinite(x)) { set_error("weight %lld is not finite", (long long)e); return DECO_ERR_GRAPH; }
      if (x != std::nearbyint(x)) {
        set_error("weight %lld = %g is not integral (exact cut values need integral weights)",
                  (long long)e, (double)x);
        return DECO_ERR_UNSUPPORTED;
      }
      if (x == 0.0f || std::fabs(x) > 1048576.0f) {
        set_error("weight %lld = %g outside the supported set (nonzero, |w| <= 2^20)",
                  (long long)e, (double)x);
        return DECO_ERR_UNSUPPORTED;
      }
      if (x != 1.0f) all_unit = false;
      if (x != 1.0f && x != -1.0f) all_pm1 = false;
      max_abs_w = std::max(max_abs_w, std::fabs(x));
    }
  }
  // ---- symmetry: (u,v) present with the same weight as (v,u); binary search
  // in row u.  Large graphs of unit weights (nnz >= 2^20) are checked on the
  // device after the upload (k_symmetry); the others here, the rows split
  // over the host's cores.  Either way the error reported is the one of the
  // lowest row, as a single pass would find it.
  // first offending row of [r0, r1) (its kind in *kind: 1 structure, 2 weights), or r1
  auto check_rows = [&](int32_t r0, int32_t r1, int* kind, int32_t* bad_u) -> int32_t {
    for (int32_t v = r0; v < r1; ++v) {
      for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        const int32_t u = col_idx[e];
        int32_t lo = row_ptr[u], hi = row_ptr[u + 1];
        while (lo < hi) {
          const int32_t mid = lo + (hi - lo) / 2;
          if (col_idx[mid] < v) lo = mid + 1; else hi = mid;
        }
        if (lo >= row_ptr[u + 1] || col_idx[lo] != v) { *kind = 1; *bad_u = u; return v; }
        if (weights && weights[lo] != weights[e]) { *kind = 2; *bad_u = u; return v; }
      }
    }
    return r1;
  };
  const bool device_check = (!weights || all_unit) && nnz >= ((int64_t)1 << 20);
  if (!(flags & DECO_GRAPH_SKIP_SYMMETRY_CHECK) && !device_check) {
    const int hw = (int)std::max<unsigned>(1, std::thread::hardware_concurrency());
    std::vector<int32_t> first(hw, n);
    std::vector<int> kinds(hw, 0);
    std::vector<int32_t> us(hw, 0);
    const int nt = host_parallel(n, nnz, [&](int t, int64_t r0, int64_t r1) {
      first[t] = check_rows((int32_t)r0, (int32_t)r1, &kinds[t], &us[t]);
      if (first[t] == (int32_t)r1) first[t] = n;
    });
    for (int t = 0; t < nt; ++t) {
      if (first[t] >= n) continue;
      const int32_t v = first[t], u = us[t];
      if (kinds[t] == 1) set_error("asymmetric structure: (%d,%d) stored but (%d,%d) missing", v, u, u, v);
      else set_error("asymmetric weights on edge (%d,%d)", v, u);
      return DECO_ERR_GRAPH;
    }
  }

  // ---- host facts
  deco_graph* g = new (std::nothrow) deco_graph();
  if (!g) { set_error("host allocation failed"); return DECO_ERR_OOM; }
  g->n = n;
  g->nnz = nnz;
  g->weighted = weights ? 1 : 0;
  g->wmode = (!weights || all_unit) ? W_UNIT : (all_pm1 ? W_SIGN : W_GENERAL);
  g->max_abs_w = (int32_t)max_abs_w;
  cudaGetDevice(&g->device);
  g->h_row_ptr.assign(row_ptr, row_ptr + (size_t)n + 1);
  std::vector<int32_t> deg(n);
  std::vector<float> dnet(n);
  {
    // degrees, their sums and maximum, net weighted degrees; per thread, then
    // combined in thread order (integer sums: the same totals in any order)
    struct Part { int64_t s1 = 0, s2 = 0; int32_t maxd = 0, bad = -1; double sabs = 0.0; };
    std::vector<Part> part(std::max<unsigned>(1, std::thread::hardware_concurrency()));
    const int nt = host_parallel(n, nnz, [&](int t, int64_t r0, int64_t r1) {
      Part& P = part[t];
      for (int32_t v = (int32_t)r0; v < (int32_t)r1; ++v) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        P.s1 += deg[v];
        P.s2 += (int64_t)deg[v] * deg[v];
        P.maxd = std::max(P.maxd, deg[v]);
        double s = 0.0, sabs = 0.0;
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
          s += weights ? weights[e] : 1.0;
          sabs += weights ? std::fabs(weights[e]) : 1.0;
        }
        if (sabs > 16777216.0 && P.bad < 0) { P.bad = v; P.sabs = sabs; }
        dnet[v] = (float)s;   // integral and |s| <= 2^24: exact in FP32
      }
    });
    for (int t = 0; t < nt; ++t) {
      if (part[t].bad >= 0) {
        set_error("row %d: sum of |w| = %g exceeds 2^24 (FP32 sums of binary iterates "
                  "would no longer be exact)", part[t].bad, part[t].sabs);
        delete g;
        return DECO_ERR_UNSUPPORTED;
      }
      g->deg_s1 += part[t].s1;
      g->deg_s2 += part[t].s2;
      g->max_deg = std::max(g->max_deg, part[t].maxd);
    }
  }

  // ---- device upload
  auto up = [&](void** dst, const void* src, size_t bytes) -> int {
    if (bytes == 0) { *dst = nullptr; return DECO_OK; }
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(graph)");
    e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(graph)");
    return DECO_OK;
  };
  // Device edge order: the caller's order, except that rows of a +-1 graph keep
  // their positive entries first and their negative entries second (each in
  // ascending column order), so every kernel can sum +y over one sub-list and
  // -y over the other in the same order.
  g->h_col.assign(col_idx, col_idx + nnz);
  if (weights) g->h_w.assign(weights, weights + nnz);
  if (g->wmode == W_SIGN) {
    for (int32_t v = 0; v < n; ++v) {
      std::vector<std::pair<int32_t, float>> row;
      for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) row.push_back({col_idx[e], weights[e]});
      std::stable_partition(row.begin(), row.end(), [](const std::pair<int32_t, float>& x) { return x.second > 0.0f; });
      for (size_t i = 0; i < row.size(); ++i) {
        g->h_col[row_ptr[v] + i] = row[i].first;
        g->h_w[row_ptr[v] + i] = row[i].second;
      }
    }
  }
  int rc = up((void**)&g->row_ptr, row_ptr, sizeof(int32_t) * (size_t)(n + 1));
  // the caller's indices where the device order is theirs (a pinned caller
  // buffer then uploads at full link speed)
  if (rc == DECO_OK)
    rc = up((void**)&g->col_idx, g->wmode == W_SIGN ? g->h_col.data() : col_idx, sizeof(int32_t) * (size_t)nnz);
  if (rc == DECO_OK) rc = up((void**)&g->deg, deg.data(), sizeof(int32_t) * (size_t)n);
  if (rc == DECO_OK) rc = up((void**)&g->dnet, dnet.data(), sizeof(float) * (size_t)n);
  if (rc == DECO_OK && g->wmode == W_SIGN) {
    std::vector<uint32_t> sw((size_t)nnz);
    for (int64_t e = 0; e < nnz; ++e)
      sw[e] = (uint32_t)g->h_col[e] | (g->h_w[e] < 0.0f ? 0x80000000u : 0u);
    rc = up((void**)&g->col_sw, sw.data(), sizeof(uint32_t) * (size_t)nnz);
  }
  if (rc == DECO_OK && g->wmode == W_GENERAL)
    rc = up((void**)&g->w, g->h_w.data(), sizeof(float) * (size_t)nnz);
  if (rc == DECO_OK && g->wmode != W_UNIT) {
    std::vector<int32_t> wi((size_t)nnz);
    for (int64_t e = 0; e < nnz; ++e) wi[e] = (int32_t)g->h_w[e];
    rc = up((void**)&g->wint, wi.data(), sizeof(int32_t) * (size_t)nnz);
  }
  if (rc == DECO_OK && !(flags & DECO_GRAPH_SKIP_SYMMETRY_CHECK) && device_check) {
    int32_t* d_bad = nullptr;
    int32_t bad = n;
    cudaError_t e = cudaMalloc((void**)&d_bad, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemcpy(d_bad, &bad, sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)n + 7) / 8, 4096);
      k_symmetry<<<blocks, 256>>>(n, g->row_ptr, g->col_idx, d_bad);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(d_bad);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "symmetry check");
    } else if (bad < n) {
      int kind = 0;
      int32_t u = 0;
      check_rows(bad, bad + 1, &kind, &u);   // the offending entry of that row, for the message
      set_error("asymmetric structure: (%d,%d) stored but (%d,%d) missing", bad, u, u, bad);
      rc = DECO_ERR_GRAPH;
    }
  }
  if (rc != DECO_OK) {
    free_graph(g);
    return rc;
  }
  *out = g;
  return DECO_OK;
}

extern "C" void deco_destroy_graph(deco_graph* g) { free_graph(g); }

extern "C" int deco_graph_info(const deco_graph* g, int32_t* n, int64_t* nnz, int32_t* weighted) {
  clear_error();
  if (!g) { set_error("graph is NULL"); return DECO_ERR_ARG; }
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (weighted) *weighted = g->weighted;
  return DECO_OK;
}
