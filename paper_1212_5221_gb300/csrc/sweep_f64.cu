// sweep_f64.cu -- instantiations of the sweep kernel for double storage.
#include "gf_sweep.cuh"
#include "gf_launch.h"

namespace gfk {

template <typename R, int GAUGE, int ALGO>
static cudaError_t launch_lpt(const SweepArgs<R>& a, int lpt, cudaStream_t st) {
  const uint64_t threads = (uint64_t)a.ncopies * a.geom.Vh * (uint64_t)(8 / lpt);
  const unsigned blocks = (unsigned)((threads + BLOCK - 1) / BLOCK);
  switch (lpt) {
    case 1: sweep_kernel<R, GAUGE, ALGO, 1><<<blocks, BLOCK, 0, st>>>(a); break;
    case 2: sweep_kernel<R, GAUGE, ALGO, 2><<<blocks, BLOCK, 0, st>>>(a); break;
    case 4: sweep_kernel<R, GAUGE, ALGO, 4><<<blocks, BLOCK, 0, st>>>(a); break;
    case 8: sweep_kernel<R, GAUGE, ALGO, 8><<<blocks, BLOCK, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
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
