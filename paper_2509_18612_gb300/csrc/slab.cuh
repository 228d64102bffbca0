// Persistent on-chip PGA kernel (slab.cu): parameter blocks and host helpers.
#pragma once

#include <stdint.h>

#include "deco_internal.cuh"

namespace deco {

constexpr int SLAB_MAX_CLUSTER = 8;

// One graph of a launch.  The rows are split between the k CTAs of a cluster
// (split[0..k]); part i's shared-memory CSR image starts at image + off[i]
// (16-byte units).  Image of a part with `own` rows (32-bit words):
//   rinfo  (own + 1) x {ps, np, ns, nn}: row rl adds y over the np entries at
//          offs[ps..], subtracts y over the nn entries at offs[ns..] (ps, ns
//          multiples of 4); entry own holds {E, 0, 0, 0}
//   offs   E byte offsets (128 * neighbour row) into the replica, each list
//          padded to a multiple of 4 entries
//   wts    E weights (general integral weights only)
struct SlabGraph {
  int32_t n, ld, C;
  const float* dnet;
  const uint4* image;
  int32_t img_off[SLAB_MAX_CLUSTER + 1];
  int32_t split[SLAB_MAX_CLUSTER + 1];
  unsigned char* xbuf;        // exchange buffer: 2 x nslabs x n x 128 B (cluster size > 1)
  int32_t nslabs;
  void* y;                    // n x ld iterate in global memory (in/out)
  float* v;                   // n x ld momentum in global memory (in/out) or null
  const float* alpha_cols;    // per column or null
  const int32_t* steps_cols;  // per column or null
};

struct SlabParams {
  SlabGraph g0;                // the graph of a single-graph launch (graphs == null)
  const SlabGraph* graphs;     // device array of a batched launch, or null
  const int2* items;           // batched launch: (graph, first column) per item
  int32_t k;                   // cluster size (CTAs per item)
  int32_t threads;             // CTA size: 512 or 1024
  int32_t xmode;               // exchange between the cluster's CTAs: 1 DSMEM, 2 L2 (k > 1)
  int32_t steps;               // steps of this launch
  const int32_t* steps_dev;    // device value bounding the steps (min with `steps`), or null
  float alpha;                 // scalar step size with the objective factor applied
  float afac;                  // objective factor applied to alpha_cols
  float mu;
  int32_t objective;
  int32_t load_v, store_v;
  int32_t max_n, max_own, max_img_words;
  int32_t lean;                // no staging area, momentum in global memory (needs xmode 2 and load_v)
  int32_t pairs;               // row-pair form: a half-warp per row, two rows per warp
  int32_t* flag;
};

size_t slab_smem_bytes(int max_n, int max_own, int max_img_words, int prec, bool lean = false);
int slab_max_smem();
// one thread waits, with k_slab's bounded exchange wait, on an mbarrier that
// never completes; sets bit 1 of *flag when the wait gives up
int launch_wait_probe_slab(int32_t* flag, cudaStream_t st);
void slab_split(const int32_t* row_ptr_host, int32_t n, int k, int32_t* split);
// builds (or finds) the on-chip CSR image of g for cluster size k
int slab_image(deco_graph* g, int k, const SlabImage** out);
// the image of rows [row0, row0 + n) of a host CSR (a member graph of a
// disjoint union: its columns in the same range), owned by the caller
int slab_image_rows(const int32_t* row_ptr, const int32_t* col, const float* w, int wmode, int32_t row0,
                    int32_t n, int k, SlabImage* out);
int launch_slab(const SlabParams& p, int n_items, int prec, int wmode, cudaStream_t st);

}  // namespace deco
