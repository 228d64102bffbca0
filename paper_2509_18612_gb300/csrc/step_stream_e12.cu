// The pipelined per-step kernel (step_stream.cuh) with 12 entries per item and
// two stages fixed at compile time, one or two vectors per lane.
#include "step_stream.cuh"

namespace deco {

void* stream_kernel_e12(int prec, int G, bool wt, int acc, int U) {
  return U == 2 ? stream_kernel_for<2, 12>(prec, G, wt, acc) : stream_kernel_for<1, 12>(prec, G, wt, acc);
}

}  // namespace deco
