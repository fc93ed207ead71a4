// sweep_launch_f32.cuh -- launch of the FP32-storage sweep kernels, shared by
// the FP32 (sweep_f32.cu) and the FP64-Step-1 MP (sweep_mp.cu) instantiations,
// which compile as separate translation units.
#pragma once
#include "gf_sweep.cuh"
#include "gf_launch.h"

namespace gfk {

// Persistent grid: as many blocks as fit on the device at once with the
// given dynamic shared memory (queried once per kernel instance and mode),
// each looping over tiles of BLOCK/L sites.
template <typename K>
static unsigned resident_blocks(K kernel, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BLOCK, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return (unsigned)(sms * per_sm);
}

// Prefetch mode 2 stages tiles in shared memory: the kernel is given the
// two stage buffers as dynamic shared memory (above the 48 KB default, so
// the limit is raised once per kernel instance).
template <typename R, int GAUGE, int ALGO, int LPT, bool OBS, bool MP>
static cudaError_t launch_kernel(const SweepArgs<R>& a, cudaStream_t st) {
  constexpr uint32_t TILE = BLOCK / (8 / LPT);
  const uint64_t ntiles = (uint64_t)((a.geom.Vh + TILE - 1) / TILE) * a.ncopies;
  auto kernel = sweep_kernel<R, GAUGE, ALGO, LPT, OBS, MP>;
  constexpr size_t smem_staged = stage_smem_bytes<LPT>();
  static const cudaError_t attr = [&] {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_staged);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    return e;
  }();
  const bool staged = a.prefetch == 2;
  if (staged && attr != cudaSuccess) return attr;
  static const unsigned resident_plain = resident_blocks(kernel, 0);
  static const unsigned resident_staged = attr == cudaSuccess ? resident_blocks(kernel, smem_staged) : 0;
  const unsigned resident = staged ? resident_staged : resident_plain;
  const unsigned blocks = (unsigned)((resident && ntiles > resident) ? resident : ntiles);
  const size_t smem = staged ? smem_staged : (a.acc && a.obs == 0 ? acc_smem_bytes<LPT>() : 0);
  kernel<<<blocks, BLOCK, smem, st>>>(a);
  return cudaGetLastError();
}

// The fused-observables variant exists for overrelaxation with FP32 Step 1 only.
template <typename R, int GAUGE, int ALGO, int LPT, bool MP>
static cudaError_t launch_one(const SweepArgs<R>& a, cudaStream_t st) {
  if (a.obs == 0) return launch_kernel<R, GAUGE, ALGO, LPT, false, MP>(a, st);
  if constexpr (ALGO == ALG_OR && !MP) return launch_kernel<R, GAUGE, ALGO, LPT, true, MP>(a, st);
  return cudaErrorInvalidValue;
}

template <typename R, int GAUGE, int ALGO, bool MP>
static cudaError_t launch_lpt(const SweepArgs<R>& a, int lpt, cudaStream_t st) {
  switch (lpt) {
    case 1: return launch_one<R, GAUGE, ALGO, 1, MP>(a, st);
    case 2: return launch_one<R, GAUGE, ALGO, 2, MP>(a, st);
    case 4: return launch_one<R, GAUGE, ALGO, 4, MP>(a, st);
    case 8: return launch_one<R, GAUGE, ALGO, 8, MP>(a, st);
  }
  return cudaErrorInvalidValue;
}

template <typename R, int GAUGE, bool MP>
static cudaError_t launch_gauge(const SweepArgs<R>& a, int algo, int lpt, cudaStream_t st) {
  switch (algo) {
    case ALG_OR: return launch_lpt<R, GAUGE, ALG_OR, MP>(a, lpt, st);
    case ALG_MICRO: return launch_lpt<R, GAUGE, ALG_MICRO, MP>(a, lpt, st);
    case ALG_SR: return launch_lpt<R, GAUGE, ALG_SR, MP>(a, lpt, st);
    case ALG_SA: return launch_lpt<R, GAUGE, ALG_SA, MP>(a, lpt, st);
  }
  return cudaErrorInvalidValue;
}

template <bool MP>
static cudaError_t launch_sweep_f32(const SweepArgs<float>& a, int gauge, int algo, int lpt, cudaStream_t st) {
  switch (gauge) {
    case LANDAU: return launch_gauge<float, LANDAU, MP>(a, algo, lpt, st);
    case COULOMB: return launch_gauge<float, COULOMB, MP>(a, algo, lpt, st);
    case MAG: return launch_gauge<float, MAG, MP>(a, algo, lpt, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gfk
