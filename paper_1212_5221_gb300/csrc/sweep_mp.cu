// sweep_mp.cu -- instantiations of the sweep kernel for float storage with
// Step 1 (the gathered K or MAG vector, the subgroup choices) in FP64 and
// Step 2 (applying the update to the links) in FP32: the mixed-precision
// variant of Sec. 4.5.
#include "sweep_launch_f32.cuh"

namespace gfk {

cudaError_t launch_sweep_mp(const SweepArgs<float>& a, int gauge, int algo, int lpt, cudaStream_t st) {
  return launch_sweep_f32<true>(a, gauge, algo, lpt, st);
}

}  // namespace gfk
