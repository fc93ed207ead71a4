// sweep_f32.cu -- instantiations of the sweep kernel for float storage.
#include "sweep_launch_f32.cuh"

namespace gfk {

template <>
cudaError_t launch_sweep<float>(const SweepArgs<float>& a, int gauge, int algo, int lpt, cudaStream_t st) {
  return launch_sweep_f32<false>(a, gauge, algo, lpt, st);
}

}  // namespace gfk
