// sweep_group.cu -- the overrelaxation sweep of several lattices of different
// extents in one persistent launch (instantiations per storage, gauge and
// links per lane).
#include "gf_sweep.cuh"
#include "gf_launch.h"

namespace gfk {

// the members' arguments are kernel parameters (at most 32764 bytes)
static_assert(sizeof(GroupArgs<double>) <= 32764 && sizeof(GroupArgs<float>) <= 32764, "group too large");

template <typename R, int GAUGE, int LPT>
static cudaError_t launch_g(const GroupArgs<R>& g, cudaStream_t st) {
  auto kernel = sweep_group_kernel<R, GAUGE, ALG_OR, LPT>;
  static const unsigned resident = [&] {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BLOCK,
                                                      sizeof(R) == 4 ? acc_smem_bytes<LPT>() : 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      return 0u;
    }
    return (unsigned)(sms * per_sm);
  }();
  const unsigned blocks = (unsigned)((resident && g.ntiles > resident) ? resident : g.ntiles);
  // FP32 members with GF_MIXED's accumulator stage it in dynamic shared memory
  const size_t smem = sizeof(R) == 4 ? acc_smem_bytes<LPT>() : 0;
  kernel<<<blocks, BLOCK, smem, st>>>(g);
  return cudaGetLastError();
}

template <typename R, int GAUGE>
static cudaError_t launch_gl(const GroupArgs<R>& g, int lpt, cudaStream_t st) {
  switch (lpt) {
    case 1: return launch_g<R, GAUGE, 1>(g, st);
    case 2: return launch_g<R, GAUGE, 2>(g, st);
    case 4: return launch_g<R, GAUGE, 4>(g, st);
    case 8:
      if constexpr (GAUGE == MAG && sizeof(R) == 8) return launch_g<R, GAUGE, 4>(g, st);
      else return launch_g<R, GAUGE, 8>(g, st);
  }
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_group(const GroupArgs<R>& g, int gauge, int lpt, cudaStream_t st) {
  switch (gauge) {
    case LANDAU: return launch_gl<R, LANDAU>(g, lpt, st);
    case COULOMB: return launch_gl<R, COULOMB>(g, lpt, st);
    case MAG: return launch_gl<R, MAG>(g, lpt, st);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_group<float>(const GroupArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_group<double>(const GroupArgs<double>&, int, int, cudaStream_t);

}  // namespace gfk
