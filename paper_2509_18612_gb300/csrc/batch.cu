// Batched pDECO over many graphs with the evolution-based hyper-parameter
// search of Sec. 4.3, one shared population for the batch.
//
// The batch is the disjoint union of its graphs (block-diagonal A), so every
// step kernel runs over all graphs at once without knowing about them; a
// row -> graph map drives the per-graph IDI thresholds, cut sums, argmax and
// best records.  Candidate k of the population owns starts
// [k B/P, (k+1) B/P) and runs T_k steps with alpha_k = 10^{e_k} through the
// per-column step-size and step-budget arrays of the phase kernels (when
// every graph's iterate slab fits in shared memory: one on-chip launch whose
// items are (graph, 128-byte column slab), each graph's replica on chip;
// otherwise the per-step kernels over the union).  Rounds
// alternate the lift as listed (Alg. 3); after every round a device kernel
// ranks the candidates (sum over graphs of the candidate's best cut) and
// replaces the bottom half by perturbed copies of the top half, and the next
// round's set-up kernel turns the population into the per-column step sizes
// and budgets.  No round needs the host, so all rounds of a solve are
// captured in one CUDA graph and launched once.
#include <algorithm>
#include <climits>
#include <cmath>
#include <memory>
#include <vector>

#include "api_util.cuh"
#include "deco_internal.cuh"
#include "phase.cuh"

using namespace deco;

struct deco_batch {
  deco_graph* U = nullptr;            // union graph
  int32_t n_graphs = 0;
  std::vector<int32_t> h_goff;        // first row of every graph (n_graphs + 1)
  std::vector<int64_t> s1, s2;        // degree power sums per graph (IDI thresholds)
  int32_t* gid = nullptr;             // device, row -> graph
  int32_t* goff = nullptr;            // device, n_graphs + 1
  int32_t* gmax = nullptr;            // device, maximum degree per graph
  double* gmean = nullptr;            // device, mean degree per graph
  int32_t* gsize = nullptr;           // device, nodes per graph
};

namespace deco {
int batch_feature_info(const deco_batch* b, const deco_graph** g, const int32_t** gid, const int32_t** goff,
                       const int32_t** gmax, const double** gmean, const int32_t** gsize, int32_t* n_graphs) {
  *g = b->U;
  *gid = b->gid;
  *goff = b->goff;
  *gmax = b->gmax;
  *gmean = b->gmean;
  *gsize = b->gsize;
  *n_graphs = b->n_graphs;
  return DECO_OK;
}
}  // namespace deco

namespace {

// ---- host Philox4x32-10 (same definition as the device version)
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    const uint32_t n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}
double u01_host(uint32_t x) { return (2.0 * (double)(x >> 9) + 1.0) * 5.9604644775390625e-8; }

// ---- per-graph bookkeeping kernels
constexpr int GCUT_ROWS = 32;   // rows per warp

__global__ void k_cut_graphs(int32_t n, int32_t B, int32_t W, const int32_t* row_ptr, const int32_t* col_idx,
                             const int32_t* wint, const uint32_t* zbits, const int32_t* gid, int64_t* cuts) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int32_t k = blockIdx.y;
  const int64_t r0 = warp * GCUT_ROWS;
  if (r0 >= n) return;
  const int32_t r1 = (int32_t)std::min<int64_t>(n, r0 + GCUT_ROWS);
  const int32_t b = k * 32 + lane;
  long long acc = 0;
  int32_t cg = gid[r0];
  for (int32_t v = (int32_t)r0; v < r1; ++v) {
    const int32_t g = gid[v];
    if (g != cg) {
      if (b < B && acc) atomicAdd(reinterpret_cast<unsigned long long*>(cuts + (size_t)cg * B + b), (unsigned long long)acc);
      acc = 0;
      cg = g;
    }
    const uint32_t zv = zbits[(size_t)v * W + k];
    int32_t racc = 0;
    for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      const int32_t u = col_idx[e];
      if (u <= v) continue;
      const uint32_t x = (zv ^ zbits[(size_t)u * W + k]) >> lane & 1u;
      racc += wint ? (int32_t)x * wint[e] : (int32_t)x;
    }
    acc += racc;
  }
  if (b < B && acc) atomicAdd(reinterpret_cast<unsigned long long*>(cuts + (size_t)cg * B + b), (unsigned long long)acc);
}

// one block per graph: lowest index among the maximal cuts
__global__ void k_argmax_graphs(int32_t B, const int64_t* cuts, int32_t* best) {
  __shared__ long long sv[256];
  __shared__ int32_t si[256];
  const int32_t g = blockIdx.x;
  long long bv = LLONG_MIN;
  int32_t bi = INT32_MAX;
  for (int32_t b = threadIdx.x; b < B; b += blockDim.x) {
    const long long c = cuts[(size_t)g * B + b];
    if (c > bv) { bv = c; bi = b; }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const long long ov = sv[threadIdx.x + s];
      const int32_t oi = si[threadIdx.x + s];
      if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) best[g] = si[0];
}

// global best record per graph: strictly larger cuts replace it
__global__ void k_record_graphs(int32_t n_graphs, int32_t B, const int64_t* cuts, const int32_t* best,
                                const int32_t* round, long long* rec_cut, int32_t* rec_round, int32_t* improved) {
  const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_graphs) return;
  const long long c = cuts[(size_t)g * B + best[g]];
  const bool up = c > rec_cut[g];
  if (up) { rec_cut[g] = c; rec_round[g] = *round; }
  improved[g] = up ? 1 : 0;
}

__global__ void k_extract_graphs(int32_t n, int32_t W, const uint32_t* zbits, const int32_t* gid,
                                 const int32_t* best, const int32_t* improved, uint8_t* round_best_z,
                                 uint8_t* best_z) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int32_t g = gid[v];
  const int32_t b = best[g];
  const uint8_t z = (uint8_t)((zbits[(size_t)v * W + (b >> 5)] >> (b & 31)) & 1u);
  round_best_z[v] = z;
  if (improved[g]) best_z[v] = z;
}

// ---- the population on the device (Sec. 4.3), so that the rounds of a
// batched solve run back to back (and are captured in one CUDA graph)
// without a trip to the host.  Population state: e (FP64 exponents,
// alpha = 10^e), T (step budgets).

// Round set-up: column c of the block belongs to candidate k = (c / l) / (B / P);
// its step size (float)10^{e_k} and budget T_k; the round's longest budget;
// the population the round runs with (kept for the caller).
__global__ void k_pop_columns(int32_t C, int32_t lift, int32_t per, int32_t P, const double* e, const int32_t* T,
                              float* alpha_cols, int32_t* steps_cols, int32_t* tmax, double* hist_e,
                              int32_t* hist_T) {
  __shared__ int32_t smax;
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  int32_t m = 0;
  for (int32_t c = threadIdx.x; c < C; c += blockDim.x) {
    const int32_t k = (c / lift) / per;
    alpha_cols[c] = (float)pow(10.0, e[k]);
    steps_cols[c] = T[k];
    m = max(m, T[k]);
  }
  atomicMax(&smax, m);
  for (int32_t k = threadIdx.x; k < P; k += blockDim.x) {
    hist_e[k] = e[k];
    hist_T[k] = T[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) *tmax = smax;
}

// Round close (one block, P <= blockDim.x): the score of candidate k is the
// sum over graphs of the best cut among its starts; the round's scores (and
// cuts, if kept) are stored; unless it is the last round, the population
// evolves: candidates ranked by score (descending, ties keep the lower
// index), the top half kept, the j-th worst replaced from the j-th best kept
// with e' = Proj[e_lo, e_hi](e + 0.2 eps), T' = Proj[t_lo, t_hi](floor(T (1 +
// 0.2 (2 eps' - 1)))), eps ~ N(0,1) by Box-Muller and eps' ~ U(0,1) from
// Philox counter (j, round, 1, STREAM_EVOLVE).
__global__ void k_pop_close(int32_t r, int32_t G, int32_t B, int32_t P, const int64_t* cuts, double* e, int32_t* T,
                            long long* scores_out, int64_t* cuts_out, int32_t evolve, uint32_t k0, uint32_t k1,
                            double e_lo, double e_hi, int32_t t_lo, int32_t t_hi) {
  extern __shared__ __align__(8) unsigned char sm_pop[];
  long long* score = reinterpret_cast<long long*>(sm_pop);
  double* e0 = reinterpret_cast<double*>(score + P);
  int32_t* T0 = reinterpret_cast<int32_t*>(e0 + P);
  int32_t* order = T0 + P;
  const int32_t per = B / P;
  for (int32_t k = threadIdx.x; k < P; k += blockDim.x) {
    long long sc = 0;
    for (int32_t g = 0; g < G; ++g) {
      long long m = LLONG_MIN;
      for (int32_t j = k * per; j < (k + 1) * per; ++j) m = max(m, (long long)cuts[(size_t)g * B + j]);
      sc += m;
    }
    score[k] = sc;
    scores_out[k] = sc;
    e0[k] = e[k];
    T0[k] = T[k];
  }
  if (cuts_out)
    for (int64_t i = threadIdx.x; i < (int64_t)G * B; i += blockDim.x) cuts_out[i] = cuts[i];
  __syncthreads();
  if (!evolve) return;
  for (int32_t k = threadIdx.x; k < P; k += blockDim.x) {
    int32_t rank = 0;
    for (int32_t j = 0; j < P; ++j) rank += (score[j] > score[k]) || (score[j] == score[k] && j < k);
    order[rank] = k;
  }
  __syncthreads();
  const int32_t nkeep = P / 2, nrep = P - nkeep;
  for (int32_t j = threadIdx.x; j < nrep; j += blockDim.x) {
    const int32_t victim = order[P - 1 - j];
    const int32_t src = order[nkeep > 0 ? j % nkeep : 0];
    const uint4 c = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)r, 1u, STREAM_EVOLVE), k0, k1);
    const double u1 = (2.0 * (double)(c.x >> 9) + 1.0) * 5.9604644775390625e-8;
    const double u2 = (2.0 * (double)(c.y >> 9) + 1.0) * 5.9604644775390625e-8;
    const double u3 = (2.0 * (double)(c.z >> 9) + 1.0) * 5.9604644775390625e-8;
    const double kPi = 3.141592653589793;
    const double eps = sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2);
    e[victim] = fmin(fmax(e0[src] + 0.2 * eps, e_lo), e_hi);
    const double t = floor((double)T0[src] * (1.0 + 0.2 * (2.0 * u3 - 1.0)));
    T[victim] = (int32_t)fmin(fmax(t, (double)t_lo), (double)t_hi);
  }
}

__global__ void k_fill_round(int32_t r, int32_t* d_round) { *d_round = r; }

__global__ void k_fill_ll(int32_t n, long long v, long long* p) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// One on-chip launch over a batch: item = (graph, column slab), one CTA per
// item, every member graph's replica and CSR image on chip.  Where the
// largest member's staging area and momentum do not fit as well, the lean
// form keeps the momentum in global memory and refreshes the replica from L2.
struct BatchSlab {
  bool ok = false;
  bool lean = false;
  std::vector<SlabImage> images;
  SlabGraph* d_graphs = nullptr;
  int2* d_items = nullptr;
  unsigned char* xbuf = nullptr;   // lean: 2 x slabs x n x 128 B per graph
  int32_t n_items = 0, max_n = 0, max_own = 0, max_words = 0;
  void release() {
    for (auto& im : images) cudaFree(im.data);
    images.clear();
    if (d_graphs) cudaFree(d_graphs);
    if (d_items) cudaFree(d_items);
    if (xbuf) cudaFree(xbuf);
    d_graphs = nullptr;
    d_items = nullptr;
    xbuf = nullptr;
    ok = false;
  }
};

// ok stays false (nothing allocated) when a member does not fit on chip
int batch_slab_prepare(const deco_batch* b, int32_t C, int32_t ld, int prec, void* y, float* v, bool mom_needed,
                       const float* alpha_cols, const int32_t* steps_cols, BatchSlab* bs) {
  const deco_graph* U = b->U;
  const int cols = prec == DECO_PREC_BF16 ? 64 : 32;
  if (ld % cols) return DECO_OK;
  const int max_smem = slab_max_smem();
  int32_t max_n = 0;
  for (int32_t i = 0; i < b->n_graphs; ++i) max_n = std::max(max_n, b->h_goff[i + 1] - b->h_goff[i]);
  if ((size_t)max_n * 128 + 4096 > (size_t)max_smem) return DECO_OK;
  std::vector<SlabGraph> hg((size_t)b->n_graphs);
  const int32_t slabs = (C + cols - 1) / cols;
  std::vector<int2> items;
  const size_t esz = elem_size(prec);
  for (int32_t i = 0; i < b->n_graphs; ++i) {
    const int32_t row0 = b->h_goff[i], n = b->h_goff[i + 1] - row0;
    SlabImage im;
    int rc = slab_image_rows(U->h_row_ptr.data(), U->h_col.data(), U->h_w.empty() ? nullptr : U->h_w.data(),
                             U->wmode, row0, n, 1, &im);
    if (rc) { bs->release(); return rc; }
    bs->images.push_back(im);
    bs->max_own = std::max(bs->max_own, im.max_own);
    bs->max_words = std::max(bs->max_words, im.max_words);
    SlabGraph& sg = hg[(size_t)i];
    sg.n = n;
    sg.ld = ld;
    sg.C = C;
    sg.dnet = U->dnet + row0;
    sg.image = reinterpret_cast<const uint4*>(im.data);
    std::copy(im.off, im.off + SLAB_MAX_CLUSTER + 1, sg.img_off);
    std::copy(im.split, im.split + SLAB_MAX_CLUSTER + 1, sg.split);
    sg.xbuf = nullptr;
    sg.nslabs = slabs;
    sg.y = static_cast<unsigned char*>(y) + (size_t)row0 * ld * esz;
    sg.v = v ? v + (size_t)row0 * ld : nullptr;
    sg.alpha_cols = alpha_cols;
    sg.steps_cols = steps_cols;
  }
  // items in decreasing order of their graph's work (stored entries plus
  // rows): CTAs start in item order, so the last wave holds the small graphs
  std::vector<int32_t> order((size_t)b->n_graphs);
  for (int32_t i = 0; i < b->n_graphs; ++i) order[(size_t)i] = i;
  auto work = [&](int32_t i) {
    const int32_t r0 = b->h_goff[i], r1 = b->h_goff[i + 1];
    return (int64_t)(U->h_row_ptr[r1] - U->h_row_ptr[r0]) + 8LL * (r1 - r0);
  };
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return work(a) > work(c); });
  for (int32_t i : order)
    for (int32_t sl = 0; sl < slabs; ++sl) items.push_back(make_int2(i, sl * cols));
  bs->max_n = max_n;
  cudaError_t e = cudaSuccess;
  if (slab_smem_bytes(max_n, bs->max_own, bs->max_words, prec) > (size_t)max_smem) {
    if (slab_smem_bytes(max_n, bs->max_own, bs->max_words, prec, true) > (size_t)max_smem || (mom_needed && !v)) {
      bs->release();
      return DECO_OK;
    }
    bs->lean = true;
    e = cudaMalloc((void**)&bs->xbuf, (size_t)2 * slabs * U->n * 128);
    if (e != cudaSuccess) {
      bs->release();
      return cuda_fail(e, "cudaMalloc(batch exchange buffer)");
    }
    for (int32_t i = 0; i < b->n_graphs; ++i) hg[(size_t)i].xbuf = bs->xbuf + (size_t)2 * slabs * b->h_goff[i] * 128;
  }
  e = cudaMalloc((void**)&bs->d_graphs, sizeof(SlabGraph) * hg.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&bs->d_items, sizeof(int2) * items.size());
  if (e == cudaSuccess) e = cudaMemcpy(bs->d_graphs, hg.data(), sizeof(SlabGraph) * hg.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bs->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    bs->release();
    return cuda_fail(e, "batch on-chip parameters");
  }
  bs->n_items = (int32_t)items.size();
  bs->ok = true;
  return DECO_OK;
}

}  // namespace

extern "C" int deco_create_batch(const deco_graph* const* graphs, int32_t n_graphs, deco_batch** out) {
  clear_error();
  if (!graphs || !out || n_graphs < 1) { set_error("need graphs, out and n_graphs >= 1"); return DECO_ERR_ARG; }
  int64_t n = 0, nnz = 0;
  bool weighted = false;
  for (int32_t i = 0; i < n_graphs; ++i) {
    if (!graphs[i]) { set_error("graph %d is NULL", i); return DECO_ERR_ARG; }
    n += graphs[i]->n;
    nnz += graphs[i]->nnz;
    weighted = weighted || graphs[i]->weighted;
  }
  if (n >= INT32_MAX || nnz >= INT32_MAX) { set_error("the union is too large"); return DECO_ERR_ARG; }
  std::vector<int32_t> rp((size_t)n + 1), ci((size_t)nnz);
  std::vector<float> w(weighted ? (size_t)nnz : 0);
  std::unique_ptr<deco_batch> b(new deco_batch());
  b->n_graphs = n_graphs;
  b->h_goff.resize(n_graphs + 1);
  int64_t ro = 0, eo = 0;
  for (int32_t i = 0; i < n_graphs; ++i) {
    const deco_graph* g = graphs[i];
    b->h_goff[i] = (int32_t)ro;
    b->s1.push_back(g->deg_s1);
    b->s2.push_back(g->deg_s2);
    for (int32_t v = 0; v < g->n; ++v) rp[ro + v] = (int32_t)(eo + g->h_row_ptr[v]);
    for (int64_t e = 0; e < g->nnz; ++e) {
      ci[eo + e] = (int32_t)(g->h_col[e] + ro);
      if (weighted) w[eo + e] = g->weighted ? g->h_w[e] : 1.0f;
    }
    ro += g->n;
    eo += g->nnz;
  }
  rp[n] = (int32_t)nnz;
  b->h_goff[n_graphs] = (int32_t)n;
  // every component was validated when it was created; rows of a +-1 graph are
  // already in device order (positives first) and stay so
  int rc = create_graph_impl((int32_t)n, nnz, rp.data(), ci.data(), weighted ? w.data() : nullptr,
                             DECO_GRAPH_SKIP_SYMMETRY_CHECK, true, &b->U);
  if (rc) return rc;
  std::vector<int32_t> gid((size_t)n), gmax(n_graphs), gsize(n_graphs);
  std::vector<double> gmean(n_graphs);
  for (int32_t i = 0; i < n_graphs; ++i) {
    for (int32_t v = b->h_goff[i]; v < b->h_goff[i + 1]; ++v) gid[v] = i;
    gmax[i] = graphs[i]->max_deg;
    gsize[i] = graphs[i]->n;
    gmean[i] = (double)graphs[i]->deg_s1 / (double)graphs[i]->n;
  }
  auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t e2 = cudaMalloc(dst, bytes);
    if (e2 == cudaSuccess) e2 = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    return e2;
  };
  cudaError_t e = up((void**)&b->gid, gid.data(), sizeof(int32_t) * (size_t)n);
  if (e == cudaSuccess) e = up((void**)&b->goff, b->h_goff.data(), sizeof(int32_t) * (size_t)(n_graphs + 1));
  if (e == cudaSuccess) e = up((void**)&b->gmax, gmax.data(), sizeof(int32_t) * (size_t)n_graphs);
  if (e == cudaSuccess) e = up((void**)&b->gsize, gsize.data(), sizeof(int32_t) * (size_t)n_graphs);
  if (e == cudaSuccess) e = up((void**)&b->gmean, gmean.data(), sizeof(double) * (size_t)n_graphs);
  if (e != cudaSuccess) {
    cudaFree(b->gid);
    cudaFree(b->goff);
    cudaFree(b->gmax);
    cudaFree(b->gsize);
    cudaFree(b->gmean);
    deco_destroy_graph(b->U);
    return cuda_fail(e, "batch upload");
  }
  *out = b.release();
  return DECO_OK;
}

extern "C" void deco_destroy_batch(deco_batch* b) {
  if (!b) return;
  cudaFree(b->gid);
  cudaFree(b->goff);
  cudaFree(b->gmax);
  cudaFree(b->gsize);
  cudaFree(b->gmean);
  deco_destroy_graph(b->U);
  delete b;
}

extern "C" int deco_batch_graph(const deco_batch* b, const deco_graph** out) {
  clear_error();
  if (!b || !out) { set_error("NULL argument"); return DECO_ERR_ARG; }
  *out = b->U;
  return DECO_OK;
}

extern "C" int deco_solve_batch(const deco_batch* b, int32_t B, const deco_params* p, const deco_population* pop,
                                uint64_t seed, int64_t* best_cuts, uint8_t* assignment, int64_t* round_cuts,
                                int64_t* round_scores, float* final_e, int32_t* final_T, void* stream,
                                deco_result* out) {
  clear_error();
  if (!b || !p || !pop || !best_cuts || !out) { set_error("NULL argument"); return DECO_ERR_ARG; }
  int rc = check_prec(p->precision);
  if (rc || (rc = check_obj(p->objective))) return rc;
  if (!valid_selector(p->kernel)) { set_error("bad kernel selector 0x%x", p->kernel); return DECO_ERR_ARG; }
  if (p->local_search != 0) { set_error("the local search is not available in batched solves"); return DECO_ERR_UNSUPPORTED; }
  if (p->phase_init != DECO_PHASE_INIT_BEST || p->eval_every != 0) {
    set_error("fresh later phases and intermediate roundings are not available in batched solves");
    return DECO_ERR_UNSUPPORTED;
  }
  const int32_t P = pop->candidates;
  if (B < 1 || P < 1 || B % P || pop->rounds < 1 || pop->t_lo < 0 || pop->t_hi < pop->t_lo ||
      !(pop->e_hi >= pop->e_lo) || pop->n_lifts < 1 || pop->n_lifts > 8) {
    set_error("bad population (B=%d P=%d rounds=%d T=[%d,%d] e=[%g,%g] lifts=%d)", B, P, pop->rounds, pop->t_lo,
              pop->t_hi, (double)pop->e_lo, (double)pop->e_hi, pop->n_lifts);
    return DECO_ERR_ARG;
  }
  int32_t max_lift = 1;
  for (int i = 0; i < pop->n_lifts; ++i) {
    if (pop->lifts[i] < 1 || pop->lifts[i] > 64) { set_error("bad lift %d", pop->lifts[i]); return DECO_ERR_ARG; }
    max_lift = std::max(max_lift, pop->lifts[i]);
  }
  if (p->init == DECO_INIT_EXPLICIT || p->init == DECO_INIT_MEAN) {
    set_error("batched solves draw their own starts (UNIFORM, IDI, DUI or IDI_HALF_UNIFORM)");
    return DECO_ERR_UNSUPPORTED;
  }
  if (p->precision == DECO_PREC_BF16 && p->polish_steps > 0) {
    set_error("FP32 polish is not available in batched solves");
    return DECO_ERR_UNSUPPORTED;
  }
  const deco_graph* U = b->U;
  const int32_t n = U->n, G = b->n_graphs;
  const int32_t Cmax = B * max_lift;
  const int32_t ld = (Cmax + 63) / 64 * 64;
  const int32_t W = (B + 31) / 32;
  const size_t block_elems = (size_t)n * ld;
  // The rounds are captured into CUDA graphs, which the legacy default stream
  // does not allow: the solve runs on a private stream ordered after the
  // caller's stream on entry and before it on exit.
  cudaStream_t caller = as_stream(stream);
  cudaStream_t st = nullptr;
  cudaEvent_t order_ev = nullptr;
  DECO_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s, caller;
    cudaEvent_t* ev;
    ~StreamGuard() {
      if (*ev) {
        cudaEventRecord(*ev, s);
        cudaStreamWaitEvent(caller, *ev, 0);
        cudaEventDestroy(*ev);
      }
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } sguard{st, caller, &order_ev};
  DECO_CUDA_TRY(cudaEventCreateWithFlags(&order_ev, cudaEventDisableTiming));
  DECO_CUDA_TRY(cudaEventRecord(order_ev, caller));
  DECO_CUDA_TRY(cudaStreamWaitEvent(st, order_ev, 0));
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);

  // ---- initial population (Sec. 4.3): counter (k, 0, 0, STREAM_EVOLVE)
  std::vector<double> e(P);
  std::vector<int64_t> T(P);
  for (int32_t k = 0; k < P; ++k) {
    uint32_t c[4] = {(uint32_t)k, 0u, 0u, STREAM_EVOLVE};
    philox_host(c, k0, k1);
    e[k] = (double)pop->e_lo + ((double)pop->e_hi - (double)pop->e_lo) * u01_host(c[0]);
    T[k] = pop->t_lo + (int64_t)(c[1] % (uint32_t)(pop->t_hi - pop->t_lo + 1));
  }
  std::vector<double> gthresh(G);
  for (int32_t i = 0; i < G; ++i) {
    deco_graph tmp;
    tmp.n = b->h_goff[i + 1] - b->h_goff[i];
    tmp.deg_s1 = b->s1[i];
    tmp.deg_s2 = b->s2[i];
    gthresh[i] = idi_threshold(&tmp, p->beta);
  }

  int64_t edge_updates = 0, kernels = 0;
  float ms = 0.0f;
  std::vector<long long> hrec(G);
  {
    Scratch s(st);
    void* ybuf[2] = {nullptr, nullptr};
    float* vbuf = nullptr;
    uint32_t* zbits = nullptr;
    int64_t* cuts = nullptr;
    int32_t *best_idx = nullptr, *improved = nullptr, *rec_round = nullptr, *d_round = nullptr;
    long long* rec_cut = nullptr;
    uint8_t *rbz = nullptr, *bz = nullptr;
    float *h = nullptr, *alpha_cols = nullptr;
    int32_t* steps_cols = nullptr;
    int8_t* side = nullptr;
    double* d_thresh = nullptr;
    int32_t* flag = nullptr;
    const size_t esz = elem_size(p->precision);
    if ((rc = s.alloc(&ybuf[0], block_elems * esz)) || (rc = s.alloc(&ybuf[1], block_elems * esz))) return rc;
    DECO_CUDA_TRY(cudaMemsetAsync(ybuf[0], 0, block_elems * esz, st));
    DECO_CUDA_TRY(cudaMemsetAsync(ybuf[1], 0, block_elems * esz, st));
    if (pop->momentum != 0.0f && (rc = s.alloc(&vbuf, block_elems * sizeof(float)))) return rc;
    if ((rc = s.alloc(&zbits, sizeof(uint32_t) * (size_t)n * W))) return rc;
    if ((rc = s.alloc(&cuts, sizeof(int64_t) * (size_t)G * B))) return rc;
    if ((rc = s.alloc(&best_idx, sizeof(int32_t) * G)) || (rc = s.alloc(&improved, sizeof(int32_t) * G)) ||
        (rc = s.alloc(&rec_round, sizeof(int32_t) * G)) || (rc = s.alloc(&d_round, sizeof(int32_t))) ||
        (rc = s.alloc(&rec_cut, sizeof(long long) * G)))
      return rc;
    if ((rc = s.alloc(&rbz, (size_t)n)) || (rc = s.alloc(&bz, (size_t)n))) return rc;
    if ((rc = s.alloc(&h, sizeof(float) * n)) || (rc = s.alloc(&side, (size_t)n))) return rc;
    if ((rc = s.alloc(&alpha_cols, sizeof(float) * Cmax)) || (rc = s.alloc(&steps_cols, sizeof(int32_t) * Cmax)))
      return rc;
    if ((rc = s.alloc(&d_thresh, sizeof(double) * G)) || (rc = s.alloc(&flag, sizeof(int32_t)))) return rc;
    DECO_CUDA_TRY(cudaMemcpyAsync(d_thresh, gthresh.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st));
    DECO_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t), st));
    k_fill_ll<<<(G + 255) / 256, 256, 0, st>>>(G, LLONG_MIN, rec_cut);
    DECO_CUDA_TRY(cudaGetLastError());

    // one phase runner (and one captured graph) per distinct lift
    struct Lane {
      int lift = 0;
      PhaseRunner R;
      BatchSlab S;     // the batched on-chip launch, when every graph fits
    };
    std::vector<std::unique_ptr<Lane>> lanes;
    struct Cleanup {
      std::vector<std::unique_ptr<Lane>>* l;
      cudaStream_t st;
      ~Cleanup() {
        for (auto& x : *l) {
          x->R.release(st);
          cudaStreamSynchronize(st);   // no launch still reads the on-chip parameters
          x->S.release();
        }
      }
    } cleanup{&lanes, st};
    for (int i = 0; i < pop->n_lifts; ++i) {
      bool have = false;
      for (auto& x : lanes) have = have || x->lift == pop->lifts[i];
      if (have) continue;
      lanes.emplace_back(new Lane());
      lanes.back()->lift = pop->lifts[i];
      if ((rc = lanes.back()->R.prepare(U, B * pop->lifts[i], ld, p->precision, p->kernel, st))) return rc;
      const int kind = p->kernel & 0x3;
      if ((kind == DECO_KERNEL_AUTO || kind == DECO_KERNEL_ONCHIP) &&
          (rc = batch_slab_prepare(b, B * pop->lifts[i], ld, p->precision, ybuf[0],
                                   pop->momentum != 0.0f ? vbuf : nullptr, pop->momentum != 0.0f, alpha_cols,
                                   steps_cols, &lanes.back()->S)))
        return rc;
    }

    cudaEvent_t ev0, ev1;
    DECO_CUDA_TRY(cudaEventCreate(&ev0));
    DECO_CUDA_TRY(cudaEventCreate(&ev1));
    struct EvGuard {
      cudaEvent_t a, b;
      ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evg{ev0, ev1};
    DECO_CUDA_TRY(cudaEventRecord(ev0, st));

    const int32_t per = B / P;
    // population on the device: e, T, the round's longest budget, the
    // population of every round, the round scores (and cuts, if kept)
    double *d_e = nullptr, *d_hist_e = nullptr;
    int32_t *d_T = nullptr, *d_hist_T = nullptr, *d_tmax = nullptr;
    long long* d_scores = nullptr;
    int64_t* d_rcuts = nullptr;
    const int32_t R = pop->rounds;
    if ((rc = s.alloc(&d_e, sizeof(double) * P)) || (rc = s.alloc(&d_T, sizeof(int32_t) * P)) ||
        (rc = s.alloc(&d_hist_e, sizeof(double) * (size_t)R * P)) ||
        (rc = s.alloc(&d_hist_T, sizeof(int32_t) * (size_t)R * P)) || (rc = s.alloc(&d_tmax, sizeof(int32_t) * R)) ||
        (rc = s.alloc(&d_scores, sizeof(long long) * (size_t)R * P)))
      return rc;
    if (round_cuts && (rc = s.alloc(&d_rcuts, sizeof(int64_t) * (size_t)R * G * B))) return rc;
    {
      std::vector<int32_t> T32(P);
      for (int32_t k = 0; k < P; ++k) T32[k] = (int32_t)T[k];
      DECO_CUDA_TRY(cudaMemcpyAsync(d_e, e.data(), sizeof(double) * P, cudaMemcpyHostToDevice, st));
      DECO_CUDA_TRY(cudaMemcpyAsync(d_T, T32.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
    }
    const size_t close_smem = (size_t)P * (sizeof(long long) + sizeof(double) + 2 * sizeof(int32_t));
    if (P > 1024 || close_smem > 48 * 1024) {
      set_error("population of %d candidates: at most 1024 in a batched solve", P);
      return DECO_ERR_UNSUPPORTED;
    }

    // Every round: set-up (step sizes, budgets), starting block, phase,
    // rounding + cuts + per-graph records, scores + evolution -- all on the
    // device, so the rounds are enqueued back to back and, when nothing in
    // them allocates, captured as one CUDA graph and launched once.  The
    // on-chip phase reads the round's longest budget from the device; the
    // per-step kernels run the largest possible budget, t_hi steps, with the
    // columns past their own budgets left unchanged (the same iterates).
    bool can_capture = true;
    for (auto& x : lanes) can_capture = can_capture && (x->S.ok || x->R.plan.col_slabs <= 1);
    auto enqueue_rounds = [&](int64_t* kc) -> int {
      for (int32_t r = 0; r < R; ++r) {
        NvtxRange r_round("deco batch round");
        const int32_t lift = pop->lifts[r % pop->n_lifts];
        const int32_t C = B * lift;
        k_pop_columns<<<1, 256, 0, st>>>(C, lift, per, P, d_e, d_T, alpha_cols, steps_cols, d_tmax + r,
                                         d_hist_e + (size_t)r * P, d_hist_T + (size_t)r * P);
        k_fill_round<<<1, 1, 0, st>>>(r, d_round);
        cudaError_t ce = cudaSuccess;
        // starting block of this round
        InitLaunch il{};
        fill_init(il, U, B, lift, ld, p, seed, r);
        il.y = ybuf[0];
        il.gid = b->gid;
        il.goff = b->goff;
        int e2 = DECO_OK;
        if (r == 0) {
          if (p->init == DECO_INIT_IDI || p->init == DECO_INIT_IDI_HALF_UNIFORM) {
            if ((e2 = launch_idi_batch(U, 0.0, d_thresh, b->gid, b->goff, k0, k1, 0, h, side, st))) return e2;
            *kc += 2;
            il.mean = h;
          }
        } else {
          il.init = DECO_INIT_MEAN;
          il.mean_bits = rbz;
        }
        if ((e2 = launch_init(il, st))) return e2;
        *kc += 3;
        if (vbuf) {
          ce = cudaMemsetAsync(vbuf, 0, block_elems * sizeof(float), st);
          if (ce != cudaSuccess) return cuda_fail(ce, "memset momentum");
        }
        Lane* L = nullptr;
        for (auto& x : lanes) if (x->lift == lift) L = x.get();
        const bool mom = vbuf != nullptr;
        int cur = 0;
        if (L->S.ok) {
          // every graph's slabs in one on-chip launch, in place in ybuf[0]
          SlabParams sp{};
          sp.graphs = L->S.d_graphs;
          sp.items = L->S.d_items;
          sp.k = 1;
          sp.threads = 1024;
          sp.xmode = L->S.lean ? 2 : 0;
          sp.lean = L->S.lean ? 1 : 0;
          sp.pairs = 1;   // row-pair form (256 BA graphs, FP32: 2.17 -> 1.83 s, same iterates)
          sp.steps = pop->t_hi;
          sp.steps_dev = d_tmax + r;
          const float fac = p->objective == DECO_OBJ_MULTILINEAR01 ? 2.0f : 1.0f;
          sp.alpha = 0.0f;
          sp.afac = fac;
          sp.mu = pop->momentum;
          sp.objective = p->objective;
          sp.load_v = mom ? 1 : 0;
          sp.store_v = 0;
          sp.max_n = L->S.max_n;
          sp.max_own = L->S.max_own;
          sp.max_img_words = L->S.max_words;
          sp.flag = flag;
          if ((e2 = launch_slab(sp, L->S.n_items, p->precision, U->wmode, st))) return e2;
          *kc += 1;
        } else {
          if ((e2 = L->R.run(ybuf, cur, vbuf, pop->t_hi, p->objective, 0.0f, pop->momentum, alpha_cols, steps_cols,
                             mom, false, flag, st, kc)))
            return e2;
        }
        if ((e2 = launch_pack(U, B, lift, ld, p->precision, ybuf[cur], zbits, st))) return e2;
        ce = cudaMemsetAsync(cuts, 0, sizeof(int64_t) * (size_t)G * B, st);
        if (ce != cudaSuccess) return cuda_fail(ce, "memset cuts");
        dim3 grid((unsigned)((((int64_t)n + GCUT_ROWS - 1) / GCUT_ROWS + 7) / 8), (unsigned)W);
        k_cut_graphs<<<grid, 256, 0, st>>>(n, B, W, U->row_ptr, U->col_idx, U->wint, zbits, b->gid, cuts);
        k_argmax_graphs<<<G, 256, 0, st>>>(B, cuts, best_idx);
        k_record_graphs<<<(G + 127) / 128, 128, 0, st>>>(G, B, cuts, best_idx, d_round, rec_cut, rec_round, improved);
        k_extract_graphs<<<(n + 255) / 256, 256, 0, st>>>(n, W, zbits, b->gid, best_idx, improved, rbz, bz);
        k_pop_close<<<1, 256, close_smem, st>>>(r, G, B, P, cuts, d_e, d_T, d_scores + (size_t)r * P,
                                                d_rcuts ? d_rcuts + (size_t)r * G * B : nullptr, r + 1 < R ? 1 : 0,
                                                k0, k1, (double)pop->e_lo, (double)pop->e_hi, pop->t_lo, pop->t_hi);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "batch round");
        *kc += 6;
      }
      return DECO_OK;
    };
    if (can_capture) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      DECO_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      int64_t kc = 0;
      const int brc = enqueue_rounds(&kc);
      cudaError_t ce = cudaStreamEndCapture(st, &graph);
      if (brc) { if (graph) cudaGraphDestroy(graph); return brc; }
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
      ce = cudaGraphLaunch(exec, st);
      cudaGraphExecDestroy(exec);   // released once the launch completes
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphLaunch");
      kernels += kc;
    } else if ((rc = enqueue_rounds(&kernels))) {
      return rc;
    }
    DECO_CUDA_TRY(cudaEventRecord(ev1, st));
    int32_t hflag = 0;
    std::vector<int32_t> h_tmax(R), h_T(P);
    std::vector<double> h_e(P);
    DECO_CUDA_TRY(cudaMemcpyAsync(h_tmax.data(), d_tmax, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaMemcpyAsync(h_e.data(), d_e, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaMemcpyAsync(h_T.data(), d_T, sizeof(int32_t) * P, cudaMemcpyDeviceToHost, st));
    std::vector<long long> h_scores((size_t)R * P);
    DECO_CUDA_TRY(cudaMemcpyAsync(h_scores.data(), d_scores, sizeof(long long) * (size_t)R * P,
                                  cudaMemcpyDeviceToHost, st));
    if (round_cuts)
      DECO_CUDA_TRY(cudaMemcpyAsync(round_cuts, d_rcuts, sizeof(int64_t) * (size_t)R * G * B, cudaMemcpyDeviceToHost,
                                    st));
    DECO_CUDA_TRY(cudaMemcpyAsync(hrec.data(), rec_cut, sizeof(long long) * G, cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (assignment) DECO_CUDA_TRY(cudaMemcpyAsync(assignment, bz, (size_t)n, cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaStreamSynchronize(st));
    DECO_CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
    if (round_scores) for (size_t i = 0; i < (size_t)R * P; ++i) round_scores[i] = h_scores[i];
    for (int32_t k = 0; k < P; ++k) {
      e[k] = h_e[k];
      T[k] = h_T[k];
    }
    // every column is swept for the round's longest budget (the on-chip
    // phase), or for t_hi steps (the per-step kernels)
    for (int32_t r = 0; r < R; ++r) {
      const int32_t lift = pop->lifts[r % pop->n_lifts];
      bool onchip = false;
      for (auto& x : lanes) if (x->lift == lift) onchip = x->S.ok;
      edge_updates += U->nnz * (int64_t)B * lift * (onchip ? h_tmax[r] : pop->t_hi);
    }
    if (hflag & 2) { set_error("a bounded device wait of the on-chip or dense kernel gave up"); return DECO_ERR_TIMEOUT; }
    if (hflag) { set_error("a non-finite value appeared in the iterate"); return DECO_ERR_NONFINITE; }
  }
  long long total = 0;
  for (int32_t g = 0; g < G; ++g) {
    best_cuts[g] = hrec[g];
    total += hrec[g];
  }
  if (final_e) for (int32_t k = 0; k < P; ++k) final_e[k] = (float)e[k];
  if (final_T) for (int32_t k = 0; k < P; ++k) final_T[k] = (int32_t)T[k];
  out->best_cut = total;
  out->best_init = -1;
  out->best_phase = -1;
  out->edge_updates = edge_updates;
  out->device_ms = ms;
  out->kernel_launches = kernels;
  return DECO_OK;
}
