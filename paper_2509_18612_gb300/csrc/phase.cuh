// Phase runner: choice between the on-chip persistent kernel and the
// per-step global-memory kernel, and the launch of one phase.
#pragma once

#include "deco_internal.cuh"
#include "dense_tc.cuh"
#include "slab.cuh"

namespace deco {

enum KernelKind { KERNEL_GLOBAL = 0, KERNEL_ONCHIP = 1, KERNEL_DENSE = 2 };

struct PhasePlan {
  int kernel = KERNEL_GLOBAL;
  int k = 1;                     // cluster size of the on-chip kernel
  int threads = 1024;            // CTA size of the on-chip kernel
  int xmode = 2;                 // exchange between cluster CTAs: 1 DSMEM, 2 L2
  bool lean = false;             // on-chip kernel: no staging area, momentum in global memory (L2 exchange)
  bool pairs = false;            // on-chip kernel: row-pair form (a half-warp per row)
  int col_slabs = 1;             // global kernel: column slabs run one after another (slab-major)
  int slab_w = 0;                // their width
  bool pipe = false;             // global kernel: the pipelined form (step_stream.cu)
  StreamShape stream;            // its launch shape
  const StreamImage* rec = nullptr;   // its record streams (owned by the graph)
  int items = 0;                 // column slabs
  int32_t max_own = 0, max_img_words = 0;
  SlabImage image;               // on-chip CSR image (owned by the graph)
  int ks = 1;                    // dense kernel: contraction split over a cluster (per-step launches)
  int32_t kpad = 0, cpad = 0;    // dense kernel: padded n and C
  bool dpersist = false;         // dense kernel: one persistent launch per phase
  DensePhaseShape dphase;        // its shape
};

int device_sm_count();
// a well-formed DECO_KERNEL_* selector (kind and the modifiers it accepts)
bool valid_selector(int kernel);
// recorded launch shape for (C, prec) on g, or -1
int tuned_selector(const deco_graph* g, int32_t C, int prec);
void record_tuning(const deco_graph* g, int32_t C, int prec, int kernel);
// force: DECO_KERNEL_* optionally | DECO_KERNEL_CLUSTER(k)
int plan_phase(const deco_graph* g, int32_t C, int32_t ld, int prec, int force, PhasePlan* plan);

struct PhaseRunner {
  const deco_graph* g = nullptr;
  int32_t C = 0, ld = 0;
  int prec = 0;
  PhasePlan plan;
  unsigned char* xbuf = nullptr;  // exchange buffer of the on-chip kernel (k > 1)
  float* vslab = nullptr;         // slab-major momentum of the column-slab schedule
  unsigned char* ypart = nullptr; // slab-major ping-pong partner of the column-slab schedule
  __nv_bfloat16* yt[2] = {nullptr, nullptr};   // dense kernel: transposed iterate pair
  float* vt = nullptr;                         // dense kernel: transposed momentum
  DenseMaps* maps = nullptr;                   // dense kernel: TMA descriptors of A and yt[0], yt[1]
  unsigned int* gbar = nullptr;                // dense phase kernel: grid barrier counter

  // choose the kernel for a C-column block of g (builds the CSR image once)
  int prepare(const deco_graph* g, int32_t C, int32_t ld, int prec, int force, cudaStream_t st);
  // `steps` steps on y[cur] (the global kernel ping-pongs y[0] / y[1] and
  // updates cur; the on-chip and dense kernels work in place)
  int run(void* y[2], int& cur, float* v, int32_t steps, int objective, float alpha, float mu,
          const float* alpha_cols, const int32_t* steps_cols, bool load_v, bool store_v, int32_t* flag,
          cudaStream_t st, int64_t* kernels);
  void release(cudaStream_t st);
};

}  // namespace deco
