// sweep_f64.cu -- instantiations of the sweep kernel for double storage.
#include "gf_sweep.cuh"
#include "gf_launch.h"

namespace gfk {

// Persistent grid: as many blocks as fit on the device at once (queried once
// per kernel instance), each looping over tiles of BLOCK/L sites.
template <typename K>
static unsigned resident_blocks(K kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BLOCK, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return (unsigned)(sms * per_sm);
}

template <typename R, int GAUGE, int ALGO, int LPT, bool OBS>
static cudaError_t launch_kernel(const SweepArgs<R>& a, cudaStream_t st) {
  constexpr uint32_t TILE = BLOCK / (8 / LPT);
  const uint64_t ntiles = (uint64_t)((a.sp_n + TILE - 1) / TILE) * a.ncopies;  // the launch's site range
  auto kernel = sweep_kernel<R, GAUGE, ALGO, LPT, OBS>;
  static const unsigned resident = resident_blocks(kernel);
  const unsigned blocks = (unsigned)((resident && ntiles > resident) ? resident : ntiles);
  if (blocks == 0) return cudaSuccess;  // an empty range
  kernel<<<blocks, BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

// The fused-observables variant exists for overrelaxation only.
template <typename R, int GAUGE, int ALGO, int LPT>
static cudaError_t launch_one(const SweepArgs<R>& a, cudaStream_t st) {
  if (a.obs == 0) return launch_kernel<R, GAUGE, ALGO, LPT, false>(a, st);
  if constexpr (ALGO == ALG_OR) return launch_kernel<R, GAUGE, ALGO, LPT, true>(a, st);
  return cudaErrorInvalidValue;
}

template <typename R, int GAUGE, int ALGO>
static cudaError_t launch_lpt(const SweepArgs<R>& a, int lpt, cudaStream_t st) {
  switch (lpt) {
    case 1: return launch_one<R, GAUGE, ALGO, 1>(a, st);
    case 2: return launch_one<R, GAUGE, ALGO, 2>(a, st);
    case 4: return launch_one<R, GAUGE, ALGO, 4>(a, st);
    case 8:
      // the MAG per-slot form holds every slot as a full 3x3 matrix: eight
      // FP64 matrices per lane would spill, so eight links per lane run as four
      if constexpr (GAUGE == MAG) return launch_one<R, GAUGE, ALGO, 4>(a, st);
      else return launch_one<R, GAUGE, ALGO, 8>(a, st);
  }
  return cudaErrorInvalidValue;
}

template <typename R, int GAUGE>
static cudaError_t launch_gauge(const SweepArgs<R>& a, int algo, int lpt, cudaStream_t st) {
  switch (algo) {
    case ALG_OR: return launch_lpt<R, GAUGE, ALG_OR>(a, lpt, st);
    case ALG_MICRO: return launch_lpt<R, GAUGE, ALG_MICRO>(a, lpt, st);
    case ALG_SR: return launch_lpt<R, GAUGE, ALG_SR>(a, lpt, st);
    case ALG_SA: return launch_lpt<R, GAUGE, ALG_SA>(a, lpt, st);
  }
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_sweep<double>(const SweepArgs<double>& a, int gauge, int algo, int lpt, cudaStream_t st) {
  switch (gauge) {
    case LANDAU: return launch_gauge<double, LANDAU>(a, algo, lpt, st);
    case COULOMB: return launch_gauge<double, COULOMB>(a, algo, lpt, st);
    case MAG: return launch_gauge<double, MAG>(a, algo, lpt, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gfk
