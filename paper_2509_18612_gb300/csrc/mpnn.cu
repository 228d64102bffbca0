// Learned initial-mean proposal: a small message-passing network whose
// output h = tanh(o) in (-1,1)^n becomes the mean of the Gaussian starts of
// the solver (Sec. 4.2's "Gaussian around a mean vector", with a learned mean
// instead of IDI).  Inference, loss, backward pass and Adam run in these
// kernels; the neighbour aggregation uses the same CSR gather as the
// projected-gradient step (spmm.cuh).
//
//   X  = node features [d/Delta, d/mean(d), 1/sqrt(d+1), 5 x U(-1,1)]   (n x 8)
//   H0 = relu(X W0 + b0)
//   M  = D^-1 A H_{l-1};   H_l = relu(H_{l-1} Ws_l + M Wn_l + b_l),  l = 1..L
//   o  = H_L wo + bo,      h = tanh(o)
//   loss per graph: min over the two labellings z, 1 - z of the mean
//   logistic loss softplus(-t o), t = 2z - 1 (a cut does not change when
//   both sides swap); batch loss = mean over graphs.
// Weight gradients are reductions over nodes in a fixed order (chunks of
// nodes in node order, then the chunks in order), so they are deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "api_util.cuh"
#include "deco_internal.cuh"
#include "spmm.cuh"

using namespace deco;

namespace {
constexpr int F_IN = 8;
constexpr int N_RANDOM = 5;
constexpr uint32_t STREAM_FEAT = 4, STREAM_PARAM = 5;
}  // namespace

struct deco_mpnn {
  int32_t hidden = 64, layers = 3;
  int64_t n_params = 0;
  float* theta = nullptr;   // device parameters (flat, see mpnn oracle layout)
  float* m = nullptr;       // Adam first moment
  float* v = nullptr;       // Adam second moment
  int64_t t = 0;            // Adam step count
};

namespace {

struct Layout {
  int64_t W0, b0, wo, bo, total;
  std::vector<int64_t> Ws, Wn, b;
};

Layout layout(int32_t H, int32_t L) {
  Layout o;
  int64_t p = 0;
  o.W0 = p; p += (int64_t)F_IN * H;
  o.b0 = p; p += H;
  for (int l = 0; l < L; ++l) {
    o.Ws.push_back(p); p += (int64_t)H * H;
    o.Wn.push_back(p); p += (int64_t)H * H;
    o.b.push_back(p); p += H;
  }
  o.wo = p; p += H;
  o.bo = p; p += 1;
  o.total = p;
  return o;
}

// ---------------------------------------------------------------- kernels

__global__ void k_init_params(int64_t count, const int64_t* starts, const double* bounds, int32_t n_ranges,
                              uint32_t k0, uint32_t k1, float* theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double a = 0.0;
  for (int r = 0; r < n_ranges; ++r)
    if (i >= starts[2 * r] && i < starts[2 * r + 1]) a = bounds[r];
  if (a == 0.0) { theta[i] = 0.0f; return; }
  const uint4 x = philox4x32_10(make_uint4((uint32_t)i, 0u, 0u, STREAM_PARAM), k0, k1);
  // (2u - 1) a with u exact in FP32; the product is formed in FP64 and rounded
  theta[i] = (float)((2.0 * (double)u01(x.x) - 1.0) * a);
}

__global__ void k_features(int32_t n, const int32_t* deg, const int32_t* gid, const int32_t* goff,
                           const int32_t* gmax, const double* gmean, int32_t max_deg, double mean_deg,
                           uint32_t k0, uint32_t k1, float* X) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint32_t kk0 = k0, kk1 = k1, vr = (uint32_t)v;
  double delta = max_deg > 0 ? (double)max_deg : 1.0, mean = mean_deg > 0 ? mean_deg : 1.0;
  if (gid) {
    const int32_t g = gid[v];
    delta = gmax[g] > 0 ? (double)gmax[g] : 1.0;
    mean = gmean[g] > 0 ? gmean[g] : 1.0;
    batch_key(gid, goff, v, kk0, kk1, vr);
  }
  const double d = (double)deg[v];
  float* x = X + (size_t)v * F_IN;
  x[0] = (float)(d / delta);
  x[1] = (float)(d / mean);
  x[2] = (float)(1.0 / sqrt(d + 1.0));
  for (int j = 0; j < N_RANDOM; ++j) {
    const uint4 r = philox4x32_10(make_uint4(vr, (uint32_t)j, 0u, STREAM_FEAT), kk0, kk1);
    x[3 + j] = (float)(2.0 * (double)u01(r.x) - 1.0);
  }
}

// pre = in1 W1 (+ in2 W2) + b;  post = relu(pre) (optionally rounded to BF16).
// One thread per (node, output column); the weights live in shared memory.
__global__ void k_dense(int32_t n, int32_t F1, int32_t Hout, const float* in1, const float* W1, const float* in2,
                        const float* W2, int32_t F2, const float* b, float* pre, float* post, int relu, int bf16) {
  extern __shared__ float sw[];
  float* s1 = sw;
  float* s2 = sw + F1 * Hout;
  for (int i = threadIdx.x; i < F1 * Hout; i += blockDim.x) s1[i] = W1[i];
  if (in2)
    for (int i = threadIdx.x; i < F2 * Hout; i += blockDim.x) s2[i] = W2[i];
  __syncthreads();
  const int32_t j = threadIdx.x % Hout;
  const int32_t rows_per_block = blockDim.x / Hout;
  const int64_t v = (int64_t)blockIdx.x * rows_per_block + threadIdx.x / Hout;
  if (v >= n) return;
  float acc = 0.0f;
  for (int i = 0; i < F1; ++i) acc = fmaf(in1[v * F1 + i], s1[i * Hout + j], acc);
  if (in2)
    for (int i = 0; i < F2; ++i) acc = fmaf(in2[v * F2 + i], s2[i * Hout + j], acc);
  if (b) acc += b[j];
  if (pre) pre[v * Hout + j] = acc;
  float y = relu ? fmaxf(acc, 0.0f) : acc;
  if (bf16) y = __bfloat162float(__float2bfloat16_rn(y));
  post[v * Hout + j] = y;
}

// out = in W^T (+ accumulate): out[v][i] = sum_j in[v][j] W[i][j]; W is F x H.
__global__ void k_dense_t(int32_t n, int32_t F, int32_t H, const float* in, const float* W, float* out, int accumulate) {
  extern __shared__ float sw[];
  for (int i = threadIdx.x; i < F * H; i += blockDim.x) sw[i] = W[i];
  __syncthreads();
  const int32_t i = threadIdx.x % F;
  const int32_t rows_per_block = blockDim.x / F;
  const int64_t v = (int64_t)blockIdx.x * rows_per_block + threadIdx.x / F;
  if (v >= n) return;
  float acc = 0.0f;
  for (int j = 0; j < H; ++j) acc = fmaf(in[v * H + j], sw[i * H + j], acc);
  out[v * F + i] = accumulate ? out[v * F + i] + acc : acc;
}

// M = D^-1 (A H): the projected-gradient step's CSR gather over H columns.
template <int WMODE>
__global__ void k_spmm_mean(int32_t n, int32_t H, const int32_t* row_ptr, CsrView A, const float* Hin,
                            const float* dinv, float* out) {
  const int G = H / 4;                         // lanes per row (4 FP32 columns each)
  const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int gl = threadIdx.x % G;
  if (grp >= n) return;
  const int32_t r = (int32_t)grp;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  csr_gather_row<DECO_PREC_FP32, WMODE>(A, Hin, H, gl * 4, row_ptr[r], row_ptr[r + 1], acc);
  const float s = dinv ? dinv[r] : 1.0f;
  float* o = out + (size_t)r * H + gl * 4;
  o[0] = acc[0] * s; o[1] = acc[1] * s; o[2] = acc[2] * s; o[3] = acc[3] * s;
}

__global__ void k_scale_rows(int32_t n, int32_t H, const float* in, const float* s, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * H) return;
  out[i] = in[i] * s[i / H];
}

__global__ void k_dinv(int32_t n, const int32_t* deg, float* dinv) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) dinv[v] = deg[v] > 0 ? (float)(1.0 / (double)deg[v]) : 0.0f;
}

__global__ void k_head(int32_t n, int32_t H, const float* Hin, const float* wo, const float* bo, float* o, float* h) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  float acc = 0.0f;
  for (int j = 0; j < H; ++j) acc = fmaf(Hin[(size_t)v * H + j], wo[j], acc);
  acc += bo[0];
  if (o) o[v] = acc;
  if (h) h[v] = tanhf(acc);
}

__device__ __forceinline__ double softplus_d(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }
__device__ __forceinline__ double sigmoid_d(double x) {
  return x >= 0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x));
}

// per-graph sums of softplus(-t o) and softplus(t o), in FP64
__global__ void k_loss_terms(int32_t n, const float* o, const uint8_t* z, const int32_t* gid, double* lp, double* lm) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double t = z[v] ? 1.0 : -1.0;
  const double x = (double)o[v];
  const int32_t g = gid ? gid[v] : 0;
  atomicAdd(lp + g, softplus_d(-t * x));
  atomicAdd(lm + g, softplus_d(t * x));
}

// batch loss = mean over graphs of min(lp, lm) / n_g
__global__ void k_loss_reduce(int32_t n, int32_t n_graphs, const int32_t* gsize, const double* lp, const double* lm,
                              double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double tot = 0.0;
  for (int32_t g = 0; g < n_graphs; ++g) {
    const double ng = gsize ? (double)gsize[g] : (double)n;
    tot += fmin(lp[g], lm[g]) / ng;
  }
  *out = tot / (double)n_graphs;
}

__global__ void k_loss_dout(int32_t n, int32_t n_graphs, const float* o, const uint8_t* z, const int32_t* gid,
                            const int32_t* gsize, const double* lp, const double* lm, float* dout) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int32_t g = gid ? gid[v] : 0;
  const double ng = gsize ? (double)gsize[g] : (double)n;
  const double s = (lp[g] / ng <= lm[g] / ng) ? 1.0 : -1.0;
  const double t = z[v] ? 1.0 : -1.0;
  dout[v] = (float)(-s * t * sigmoid_d(-s * t * (double)o[v]) / (ng * (double)n_graphs));
}

// Weight gradients dW[i][j] = sum_v in[v][i] d[v][j] (in == NULL: in = 1, the
// bias gradient) as a two-level reduction with a fixed order: chunks of
// WG_CHUNK nodes summed in node order, then the chunks summed in chunk order.
constexpr int WG_CHUNK = 256, WG_TILE = 32, WG_THREADS = 256, WG_PER = 16;

__global__ void __launch_bounds__(WG_THREADS) k_wgrad_part(int32_t n, int32_t F, int32_t H, const float* in,
                                                            const float* d, float* part) {
  extern __shared__ float tile[];   // WG_TILE x (F + H)
  const int32_t c = blockIdx.x;
  const int32_t v0 = c * WG_CHUNK, v1 = min(n, v0 + WG_CHUNK);
  const int32_t FH = F * H;
  float* tin = tile;
  float* td = tile + WG_TILE * F;
  for (int32_t e0 = 0; e0 < FH; e0 += WG_THREADS * WG_PER) {
    float acc[WG_PER];
#pragma unroll
    for (int k = 0; k < WG_PER; ++k) acc[k] = 0.0f;
    for (int32_t t0 = v0; t0 < v1; t0 += WG_TILE) {
      const int32_t cnt = min(WG_TILE, v1 - t0);
      __syncthreads();
      for (int32_t x = threadIdx.x; x < cnt * F; x += WG_THREADS)
        tin[x] = in ? in[(size_t)t0 * F + x] : 1.0f;
      for (int32_t x = threadIdx.x; x < cnt * H; x += WG_THREADS) td[x] = d[(size_t)t0 * H + x];
      __syncthreads();
      for (int32_t r = 0; r < cnt; ++r) {
#pragma unroll
        for (int k = 0; k < WG_PER; ++k) {
          const int32_t e = e0 + k * WG_THREADS + threadIdx.x;
          if (e < FH) acc[k] = fmaf(tin[r * F + e / H], td[r * H + e % H], acc[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < WG_PER; ++k) {
      const int32_t e = e0 + k * WG_THREADS + threadIdx.x;
      if (e < FH) part[(size_t)c * FH + e] = acc[k];
    }
  }
}

__global__ void k_wgrad_sum(int32_t chunks, int32_t FH, const float* part, float* dW) {
  const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= FH) return;
  float acc = 0.0f;
  for (int32_t c = 0; c < chunks; ++c) acc += part[(size_t)c * FH + e];
  dW[e] = acc;
}

__global__ void k_relu_mask(int64_t count, const float* pre, float* dh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count && !(pre[i] > 0.0f)) dh[i] = 0.0f;
}

__global__ void k_outer(int32_t n, int32_t H, const float* d, const float* w, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (int64_t)n * H) out[i] = d[i / H] * w[i % H];
}

__global__ void k_adam(int64_t count, float* theta, const float* g, float* m, float* v, float lr, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / c1, vh = vi / c2;
  theta[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

unsigned nb(int64_t count, int block = 256) { return (unsigned)((count + block - 1) / block); }

// ---------------------------------------------------------------- forward / backward

struct Acts {
  Scratch* s;
  float *X = nullptr, *dinv = nullptr, *o = nullptr;
  std::vector<float*> pre, Hs, Ms;   // pre[l], H[l] for l = 0..L;  M[l] for l = 1..L (index l-1)
};

int spmm_mean(const deco_graph* g, int32_t H, const float* in, const float* dinv, float* out, cudaStream_t st) {
  const CsrView A{g->col_idx, g->col_sw, g->w};
  const int G = H / 4;
  const int64_t threads = (int64_t)g->n * G;
  if (g->wmode == W_UNIT) k_spmm_mean<W_UNIT><<<nb(threads), 256, 0, st>>>(g->n, H, g->row_ptr, A, in, dinv, out);
  else if (g->wmode == W_SIGN) k_spmm_mean<W_SIGN><<<nb(threads), 256, 0, st>>>(g->n, H, g->row_ptr, A, in, dinv, out);
  else k_spmm_mean<W_GENERAL><<<nb(threads), 256, 0, st>>>(g->n, H, g->row_ptr, A, in, dinv, out);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

int dense(int32_t n, int32_t F1, int32_t H, const float* in1, const float* W1, const float* in2, const float* W2,
          int32_t F2, const float* b, float* pre, float* post, bool relu, bool bf16, cudaStream_t st) {
  const int rows = 256 / H > 0 ? 256 / H : 1;
  const size_t smem = sizeof(float) * ((size_t)F1 * H + (in2 ? (size_t)F2 * H : 0));
  k_dense<<<(unsigned)((n + rows - 1) / rows), rows * H, smem, st>>>(n, F1, H, in1, W1, in2, W2, F2, b, pre, post,
                                                                       relu ? 1 : 0, bf16 ? 1 : 0);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

struct FeatureInfo {
  const int32_t* gid = nullptr;
  const int32_t* goff = nullptr;
  const int32_t* gmax = nullptr;
  const double* gmean = nullptr;
  const int32_t* gsize = nullptr;
  int32_t n_graphs = 1;
};

int forward(const deco_mpnn* m, const deco_graph* g, const FeatureInfo& fi, uint64_t feat_seed, bool bf16,
            Acts& a, cudaStream_t st) {
  const int32_t n = g->n, H = m->hidden, L = m->layers;
  const Layout lo = layout(H, L);
  int rc;
  if ((rc = a.s->alloc(&a.X, sizeof(float) * (size_t)n * F_IN)) || (rc = a.s->alloc(&a.dinv, sizeof(float) * n)) ||
      (rc = a.s->alloc(&a.o, sizeof(float) * n)))
    return rc;
  const double mean = g->n ? (double)g->deg_s1 / (double)g->n : 1.0;
  k_features<<<nb(n), 256, 0, st>>>(n, g->deg, fi.gid, fi.goff, fi.gmax, fi.gmean, g->max_deg, mean,
                                    (uint32_t)feat_seed, (uint32_t)(feat_seed >> 32), a.X);
  k_dinv<<<nb(n), 256, 0, st>>>(n, g->deg, a.dinv);
  DECO_CUDA_TRY(cudaGetLastError());
  a.pre.assign(L + 1, nullptr);
  a.Hs.assign(L + 1, nullptr);
  a.Ms.assign(L, nullptr);
  for (int l = 0; l <= L; ++l) {
    if ((rc = a.s->alloc(&a.pre[l], sizeof(float) * (size_t)n * H)) ||
        (rc = a.s->alloc(&a.Hs[l], sizeof(float) * (size_t)n * H)))
      return rc;
    if (l < L && (rc = a.s->alloc(&a.Ms[l], sizeof(float) * (size_t)n * H))) return rc;
  }
  const float* th = m->theta;
  if ((rc = dense(n, F_IN, H, a.X, th + lo.W0, nullptr, nullptr, 0, th + lo.b0, a.pre[0], a.Hs[0], true, bf16, st)))
    return rc;
  for (int l = 1; l <= L; ++l) {
    if ((rc = spmm_mean(g, H, a.Hs[l - 1], a.dinv, a.Ms[l - 1], st))) return rc;
    if ((rc = dense(n, H, H, a.Hs[l - 1], th + lo.Ws[l - 1], a.Ms[l - 1], th + lo.Wn[l - 1], H, th + lo.b[l - 1],
                    a.pre[l], a.Hs[l], true, bf16, st)))
      return rc;
  }
  k_head<<<nb(n), 256, 0, st>>>(n, H, a.Hs[L], th + lo.wo, th + lo.bo, a.o, nullptr);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

// dW (F x H) = in^T d over all n nodes (in == NULL: the column sums of d); part: chunk scratch
int wgrad(int32_t n, int32_t F, int32_t H, const float* in, const float* d, float* part, float* dW, cudaStream_t st) {
  const int32_t chunks = std::max(1, (n + WG_CHUNK - 1) / WG_CHUNK);
  if (n == 0) {
    DECO_CUDA_TRY(cudaMemsetAsync(dW, 0, sizeof(float) * (size_t)F * H, st));
    return DECO_OK;
  }
  k_wgrad_part<<<chunks, WG_THREADS, sizeof(float) * WG_TILE * (F + H), st>>>(n, F, H, in, d, part);
  k_wgrad_sum<<<(F * H + 255) / 256, 256, 0, st>>>(chunks, F * H, part, dW);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

int loss_backward(const deco_mpnn* m, const deco_graph* g, const FeatureInfo& fi, const uint8_t* z, Acts& a,
                  float* grad, double* loss_out, cudaStream_t st, double* loss_dev = nullptr) {
  const int32_t n = g->n, H = m->hidden, L = m->layers, G = fi.n_graphs;
  const Layout lo = layout(H, L);
  int rc;
  double *lp = nullptr, *lm = nullptr;
  float *dout = nullptr, *dH = nullptr, *dH2 = nullptr, *tmp = nullptr;
  if ((rc = a.s->alloc(&lp, sizeof(double) * G)) || (rc = a.s->alloc(&lm, sizeof(double) * G)) ||
      (rc = a.s->alloc(&dout, sizeof(float) * n)) || (rc = a.s->alloc(&dH, sizeof(float) * (size_t)n * H)) ||
      (rc = a.s->alloc(&dH2, sizeof(float) * (size_t)n * H)) || (rc = a.s->alloc(&tmp, sizeof(float) * (size_t)n * H)))
    return rc;
  float* part = nullptr;   // partial weight-gradient sums, one block of H x H per node chunk
  if ((rc = a.s->alloc(&part, sizeof(float) * (size_t)std::max(1, (n + WG_CHUNK - 1) / WG_CHUNK) *
                                  std::max(H * H, F_IN * H))))
    return rc;
  DECO_CUDA_TRY(cudaMemsetAsync(lp, 0, sizeof(double) * G, st));
  DECO_CUDA_TRY(cudaMemsetAsync(lm, 0, sizeof(double) * G, st));
  k_loss_terms<<<nb(n), 256, 0, st>>>(n, a.o, z, fi.gid, lp, lm);
  k_loss_dout<<<nb(n), 256, 0, st>>>(n, G, a.o, z, fi.gid, fi.gsize, lp, lm, dout);
  if (loss_dev) k_loss_reduce<<<1, 32, 0, st>>>(n, G, fi.gsize, lp, lm, loss_dev);
  DECO_CUDA_TRY(cudaGetLastError());
  if (loss_out) {
    std::vector<double> hp(G), hm(G);
    std::vector<int32_t> gs(G, n);
    DECO_CUDA_TRY(cudaMemcpyAsync(hp.data(), lp, sizeof(double) * G, cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaMemcpyAsync(hm.data(), lm, sizeof(double) * G, cudaMemcpyDeviceToHost, st));
    if (fi.gsize) DECO_CUDA_TRY(cudaMemcpyAsync(gs.data(), fi.gsize, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaStreamSynchronize(st));
    double tot = 0.0;
    for (int i = 0; i < G; ++i) tot += std::min(hp[i], hm[i]) / (double)gs[i];
    *loss_out = tot / (double)G;
  }
  if (!grad) return DECO_OK;
  const float* th = m->theta;
  // head: dwo = H_L^T dout, dbo = sum dout, dH_L = dout wo^T
  if ((rc = wgrad(n, H, 1, a.Hs[L], dout, part, grad + lo.wo, st)) ||   // H x 1
      (rc = wgrad(n, 1, 1, nullptr, dout, part, grad + lo.bo, st)))
    return rc;
  k_outer<<<nb((int64_t)n * H), 256, 0, st>>>(n, H, dout, th + lo.wo, dH);
  DECO_CUDA_TRY(cudaGetLastError());
  for (int l = L; l >= 1; --l) {
    k_relu_mask<<<nb((int64_t)n * H), 256, 0, st>>>((int64_t)n * H, a.pre[l], dH);   // dH -> dpre
    if ((rc = wgrad(n, H, H, a.Hs[l - 1], dH, part, grad + lo.Ws[l - 1], st)) ||
        (rc = wgrad(n, H, H, a.Ms[l - 1], dH, part, grad + lo.Wn[l - 1], st)) ||
        (rc = wgrad(n, 1, H, nullptr, dH, part, grad + lo.b[l - 1], st)))
      return rc;
    // dH_{l-1} = dpre Ws^T + A (D^-1 (dpre Wn^T))
    k_dense_t<<<(unsigned)((n + 256 / H - 1) / (256 / H)), (256 / H) * H, sizeof(float) * H * H, st>>>(
        n, H, H, dH, th + lo.Wn[l - 1], tmp, 0);
    k_scale_rows<<<nb((int64_t)n * H), 256, 0, st>>>(n, H, tmp, a.dinv, tmp);
    if ((rc = spmm_mean(g, H, tmp, nullptr, dH2, st))) return rc;
    k_dense_t<<<(unsigned)((n + 256 / H - 1) / (256 / H)), (256 / H) * H, sizeof(float) * H * H, st>>>(
        n, H, H, dH, th + lo.Ws[l - 1], dH2, 1);
    DECO_CUDA_TRY(cudaGetLastError());
    std::swap(dH, dH2);
  }
  k_relu_mask<<<nb((int64_t)n * H), 256, 0, st>>>((int64_t)n * H, a.pre[0], dH);
  DECO_CUDA_TRY(cudaGetLastError());
  if ((rc = wgrad(n, F_IN, H, a.X, dH, part, grad + lo.W0, st)) ||
      (rc = wgrad(n, 1, H, nullptr, dH, part, grad + lo.b0, st)))
    return rc;
  return DECO_OK;
}

int check_model(const deco_mpnn* m) {
  if (!m) { set_error("model is NULL"); return DECO_ERR_ARG; }
  return DECO_OK;
}

}  // namespace

// Batch side-information for the features and the per-graph loss (batch.cu).
namespace deco {
int batch_feature_info(const deco_batch* b, const deco_graph** g, const int32_t** gid, const int32_t** goff,
                       const int32_t** gmax, const double** gmean, const int32_t** gsize, int32_t* n_graphs);
}

static int resolve(const deco_graph* g, const deco_batch* b, const deco_graph** G, FeatureInfo* fi) {
  if ((g == nullptr) == (b == nullptr)) { set_error("pass exactly one of a graph and a batch"); return DECO_ERR_ARG; }
  *fi = FeatureInfo{};
  if (g) { *G = g; return DECO_OK; }
  return batch_feature_info(b, G, &fi->gid, &fi->goff, &fi->gmax, &fi->gmean, &fi->gsize, &fi->n_graphs);
}

extern "C" int deco_mpnn_create(int32_t hidden, int32_t layers, uint64_t seed, deco_mpnn** out) {
  clear_error();
  if (!out || hidden < 4 || hidden > 128 || hidden % 4 || layers < 1 || layers > 8) {
    set_error("need hidden in [4, 128], a multiple of 4, and 1 <= layers <= 8");
    return DECO_ERR_ARG;
  }
  deco_mpnn* m = new deco_mpnn();
  m->hidden = hidden;
  m->layers = layers;
  const Layout lo = layout(hidden, layers);
  m->n_params = lo.total;
  cudaError_t e = cudaMalloc((void**)&m->theta, sizeof(float) * lo.total);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->m, sizeof(float) * lo.total);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->v, sizeof(float) * lo.total);
  if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * lo.total);
  if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * lo.total);
  if (e != cudaSuccess) {
    cudaFree(m->theta); cudaFree(m->m); cudaFree(m->v);
    delete m;
    return cuda_fail(e, "model allocation");
  }
  // Xavier-uniform weight ranges: [start, end) and bound per weight matrix
  std::vector<int64_t> ranges;
  std::vector<double> bounds;
  auto add = [&](int64_t s, int64_t count, int fi, int fo) {
    ranges.push_back(s);
    ranges.push_back(s + count);
    bounds.push_back(std::sqrt(6.0 / (double)(fi + fo)));
  };
  add(lo.W0, (int64_t)F_IN * hidden, F_IN, hidden);
  for (int l = 0; l < layers; ++l) {
    add(lo.Ws[l], (int64_t)hidden * hidden, hidden, hidden);
    add(lo.Wn[l], (int64_t)hidden * hidden, hidden, hidden);
  }
  add(lo.wo, hidden, hidden, 1);
  int64_t* dr = nullptr;
  double* db = nullptr;
  e = cudaMalloc((void**)&dr, sizeof(int64_t) * ranges.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&db, sizeof(double) * bounds.size());
  if (e == cudaSuccess) e = cudaMemcpy(dr, ranges.data(), sizeof(int64_t) * ranges.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(db, bounds.data(), sizeof(double) * bounds.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_init_params<<<nb(lo.total), 256>>>(lo.total, dr, db, (int32_t)bounds.size(), (uint32_t)seed,
                                         (uint32_t)(seed >> 32), m->theta);
    e = cudaDeviceSynchronize();
  }
  cudaFree(dr);
  cudaFree(db);
  if (e != cudaSuccess) {
    cudaFree(m->theta); cudaFree(m->m); cudaFree(m->v);
    delete m;
    return cuda_fail(e, "model initialisation");
  }
  *out = m;
  return DECO_OK;
}

extern "C" void deco_mpnn_destroy(deco_mpnn* m) {
  if (!m) return;
  cudaFree(m->theta);
  cudaFree(m->m);
  cudaFree(m->v);
  delete m;
}

extern "C" int deco_mpnn_num_params(const deco_mpnn* m, int64_t* count) {
  clear_error();
  int rc = check_model(m);
  if (rc) return rc;
  if (!count) { set_error("count is NULL"); return DECO_ERR_ARG; }
  *count = m->n_params;
  return DECO_OK;
}

extern "C" int deco_mpnn_get_params(const deco_mpnn* m, float* host, int64_t count) {
  clear_error();
  int rc = check_model(m);
  if (rc) return rc;
  if (!host || count != m->n_params) { set_error("need a host buffer of %lld floats", (long long)m->n_params); return DECO_ERR_ARG; }
  DECO_CUDA_TRY(cudaMemcpy(host, m->theta, sizeof(float) * count, cudaMemcpyDeviceToHost));
  return DECO_OK;
}

extern "C" int deco_mpnn_set_params(deco_mpnn* m, const float* host, int64_t count) {
  clear_error();
  int rc = check_model(m);
  if (rc) return rc;
  if (!host || count != m->n_params) { set_error("need a host buffer of %lld floats", (long long)m->n_params); return DECO_ERR_ARG; }
  DECO_CUDA_TRY(cudaMemcpy(m->theta, host, sizeof(float) * count, cudaMemcpyHostToDevice));
  DECO_CUDA_TRY(cudaMemset(m->m, 0, sizeof(float) * count));
  DECO_CUDA_TRY(cudaMemset(m->v, 0, sizeof(float) * count));
  m->t = 0;
  return DECO_OK;
}

extern "C" int deco_mpnn_infer(const deco_mpnn* m, const deco_graph* g, const deco_batch* b, uint64_t feat_seed,
                               int32_t precision, float* h, void* stream) {
  clear_error();
  int rc = check_model(m);
  if (rc) return rc;
  if (!h || (rc = check_prec(precision))) { if (!rc) set_error("h is NULL"); return rc ? rc : DECO_ERR_ARG; }
  const deco_graph* G = nullptr;
  FeatureInfo fi;
  if ((rc = resolve(g, b, &G, &fi))) return rc;
  cudaStream_t st = as_stream(stream);
  Scratch s(st);
  Acts a;
  a.s = &s;
  if ((rc = forward(m, G, fi, feat_seed, precision == DECO_PREC_BF16, a, st))) return rc;
  const Layout lo = layout(m->hidden, m->layers);
  k_head<<<nb(G->n), 256, 0, st>>>(G->n, m->hidden, a.Hs[m->layers], m->theta + lo.wo, m->theta + lo.bo, nullptr, h);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}

extern "C" int deco_mpnn_loss_grad(const deco_mpnn* m, const deco_graph* g, const deco_batch* b, const uint8_t* z,
                                   uint64_t feat_seed, double* loss, float* grad, void* stream) {
  clear_error();
  int rc = check_model(m);
  if (rc) return rc;
  if (!z) { set_error("labels are NULL"); return DECO_ERR_ARG; }
  const deco_graph* G = nullptr;
  FeatureInfo fi;
  if ((rc = resolve(g, b, &G, &fi))) return rc;
  cudaStream_t st = as_stream(stream);
  Scratch s(st);
  Acts a;
  a.s = &s;
  if ((rc = forward(m, G, fi, feat_seed, false, a, st))) return rc;
  return loss_backward(m, G, fi, z, a, grad, loss, st);
}

extern "C" int deco_mpnn_train(deco_mpnn* m, const deco_graph* g, const deco_batch* b, const uint8_t* z,
                               uint64_t feat_seed, float lr, int32_t steps, double* losses, void* stream) {
  clear_error();
  int rc = check_model(m);
  if (rc) return rc;
  if (!z || !(lr > 0.0f) || steps < 0) { set_error("need labels, lr > 0 and steps >= 0"); return DECO_ERR_ARG; }
  const deco_graph* G = nullptr;
  FeatureInfo fi;
  if ((rc = resolve(g, b, &G, &fi))) return rc;
  cudaStream_t st = as_stream(stream);
  Scratch s(st);
  float* grad = nullptr;
  double* ldev = nullptr;
  if ((rc = s.alloc(&grad, sizeof(float) * m->n_params)) ||
      (rc = s.alloc(&ldev, sizeof(double) * (size_t)(steps > 0 ? steps : 1))))
    return rc;
  for (int32_t it = 0; it < steps; ++it) {
    Scratch si(st);   // activations of this step, released in stream order
    Acts a;
    a.s = &si;
    if ((rc = forward(m, G, fi, feat_seed, false, a, st))) return rc;
    if ((rc = loss_backward(m, G, fi, z, a, grad, nullptr, st, ldev + it))) return rc;
    m->t += 1;
    const float c1 = 1.0f - std::pow(0.9f, (float)m->t), c2 = 1.0f - std::pow(0.999f, (float)m->t);
    k_adam<<<nb(m->n_params), 256, 0, st>>>(m->n_params, m->theta, grad, m->m, m->v, lr, c1, c2);
    DECO_CUDA_TRY(cudaGetLastError());
  }
  if (losses && steps > 0) {
    DECO_CUDA_TRY(cudaMemcpyAsync(losses, ldev, sizeof(double) * steps, cudaMemcpyDeviceToHost, st));
    DECO_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return DECO_OK;
}

extern "C" int deco_mpnn_train_step(deco_mpnn* m, const deco_graph* g, const deco_batch* b, const uint8_t* z,
                                    uint64_t feat_seed, float lr, double* loss, void* stream) {
  clear_error();
  int rc = check_model(m);
  if (rc) return rc;
  if (!z || !(lr > 0.0f)) { set_error("need labels and lr > 0"); return DECO_ERR_ARG; }
  const deco_graph* G = nullptr;
  FeatureInfo fi;
  if ((rc = resolve(g, b, &G, &fi))) return rc;
  cudaStream_t st = as_stream(stream);
  Scratch s(st);
  Acts a;
  a.s = &s;
  float* grad = nullptr;
  if ((rc = s.alloc(&grad, sizeof(float) * m->n_params))) return rc;
  if ((rc = forward(m, G, fi, feat_seed, false, a, st))) return rc;
  if ((rc = loss_backward(m, G, fi, z, a, grad, loss, st))) return rc;
  m->t += 1;
  const float c1 = 1.0f - std::pow(0.9f, (float)m->t), c2 = 1.0f - std::pow(0.999f, (float)m->t);
  k_adam<<<nb(m->n_params), 256, 0, st>>>(m->n_params, m->theta, grad, m->m, m->v, lr, c1, c2);
  DECO_CUDA_TRY(cudaGetLastError());
  return DECO_OK;
}
