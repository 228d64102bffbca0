// Tensor-core step for dense graphs (DECO_KERNEL_DENSE): launch interface.
#pragma once

#include <cuda.h>

#include "deco_internal.cuh"

namespace deco {

constexpr int DENSE_BM = 128;        // rows of A per CTA (tcgen05 M)
constexpr int DENSE_BK = 64;         // contraction depth of one pipeline stage (one 128-byte swizzle row)
constexpr int DENSE_MAX_N = 32768;   // dense copy of A at most 2 GiB
constexpr int DENSE_MAX_C = 1024;    // columns of the block (tiles of <= 256)
constexpr int DENSE_MAX_W = 256;     // |w| exact in BF16

struct DenseStep {
  int32_t n;            // nodes
  int32_t kpad;         // round_up(n, 128): rows / columns of the dense A, row length of YT / VT
  int32_t cpad;         // rows of YT / VT: round_up(C, 32)
  int32_t C;            // active columns
  int32_t ks;           // contraction split (cluster size along K)
  int objective;
  const __nv_bfloat16* A;   // kpad x kpad dense A (read directly by the phase kernel's resident tiles)
  const __nv_bfloat16* YT;  // cpad x kpad, transposed iterate (zero for nodes >= n)
  __nv_bfloat16* YTout;     // cpad x kpad, next iterate (distinct from YT)
  float* VT;                // cpad x kpad momentum (MOM only)
  const float* dnet;        // n, net weighted degree
  float alpha, afac, mu;    // alpha already multiplied by the objective's factor
  const float* alpha_cols;
  const int32_t* steps_cols;
  int32_t t;
  int32_t* flag;            // bit 0 nonfinite, bit 1 a bounded wait gave up
};

// TMA descriptors of the dense A and of the two transposed iterates, with the
// B boxes of the per-step kernel (min(256, cpad) rows) and of the phase kernel (w rows)
struct DenseMaps {
  CUtensorMap a;
  CUtensorMap y[2];
  CUtensorMap yw[2];
};

// launch shape of the persistent phase kernel
struct DensePhaseShape {
  int w = 0;          // column tile width (multiple of 32, <= 128)
  int ks = 1;         // contraction split (cluster size)
  int stages = 0;     // B stages (YT tiles)
  int stages_a = 0;   // A stages (the streamed A tiles)
  size_t smem = 0;    // dynamic shared memory
  int ctas = 0;       // row tiles x ks x column tiles
};

// dense BF16 copy of A, row stride kpad, zero-filled (device memory owned by the graph)
int dense_build(const deco_graph* g, int32_t kpad, __nv_bfloat16** out, cudaStream_t st);
int dense_make_maps(const __nv_bfloat16* A, int32_t kpad, __nv_bfloat16* const yt[2], int32_t cpad, int w,
                    DenseMaps* maps);
// shape of the phase kernel for split ks and width w; DECO_ERR_UNSUPPORTED if it
// does not fit in shared memory
int dense_phase_shape(int32_t kpad, int32_t cpad, int ks, int w, DensePhaseShape* out);
// all `steps` steps in one launch; the result is in yt[steps & 1].
// DECO_ERR_UNSUPPORTED (nothing launched) if its CTAs cannot all be resident.
int launch_dense_phase(const DenseStep& p, const DenseMaps& maps, __nv_bfloat16* const yt[2],
                       const DensePhaseShape& sh, int32_t steps, unsigned int* gbar, cudaStream_t st);
// y (n x ld, first C columns) -> yt (C x kpad), and back; esz 2 (BF16) or 4 (FP32)
int dense_to_t(const void* y, int32_t n, int32_t ld, int32_t C, void* yt, int32_t kpad, size_t esz,
               cudaStream_t st);
int dense_from_t(const void* yt, int32_t kpad, int32_t C, void* y, int32_t n, int32_t ld, size_t esz,
                 cudaStream_t st);
// one step: YT = yt[which] -> YTout = yt[which ^ 1] (p.YT / p.YTout must match)
int launch_dense_step(const DenseStep& p, const DenseMaps& maps, int which, cudaStream_t st);
// one thread waits, with the dense kernels' bounded waits, on something that
// never completes: which 0 a CTA mbarrier, 1 the grid barrier counter
// (*counter must be 0); sets bit 1 of *flag when the wait gives up
int launch_wait_probe_dense(int which, unsigned int* counter, int32_t* flag, cudaStream_t st);

}  // namespace deco
