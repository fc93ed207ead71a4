// gf_aux.cu -- launchers of the auxiliary kernels (observables, re-unitarise,
// precision switch, layout conversion, random gauge transform, Coulomb fold).
#include "gf_kernels.cuh"
#include "gf_launch.h"

namespace gfk {

static unsigned nblocks(uint64_t n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

size_t observables_partial_doubles(const Geom& G, uint32_t ncopies) {
  const uint32_t bpu = (G.V3 / 2 + BLOCK - 1) / BLOCK;
  return (size_t)ncopies * G.n[0] * 2 * bpu * 2;
}

template <typename R>
cudaError_t launch_observables(const void* links, const Geom& G, int NS, int gauge, uint32_t ncopies,
                               double* partial, double* out, cudaStream_t st) {
  ObsArgs a;
  a.geom = G;
  a.NS = NS;
  a.gauge = gauge;
  a.ncopies = ncopies;
  a.partial = partial;
  a.blocks_per_unit = (G.V3 / 2 + BLOCK - 1) / BLOCK;
  const uint32_t units = ncopies * (uint32_t)G.n[0] * 2;
  if (units > 65535u) return cudaErrorInvalidConfiguration;
  dim3 grid(a.blocks_per_unit, units);
  observables_kernel<R><<<grid, BLOCK, 0, st>>>(
      static_cast<const typename store_traits<R>::vec*>(links), a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nd = gauge == COULOMB ? 3 : 4;
  const double normF = 1.0 / (3.0 * nd * (double)G.V3);
  const double normT = 1.0 / (3.0 * (double)G.V3);
  const uint32_t ct = ncopies * (uint32_t)G.n[0];
  observables_finish<<<(ct + 127) / 128, 128, 0, st>>>(partial, a.blocks_per_unit, ct, normF, normT, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_reunitarize(void* links, uint32_t Vh, uint64_t nmat, cudaStream_t st) {
  reunitarize_kernel<R><<<nblocks(nmat), BLOCK, 0, st>>>(static_cast<typename store_traits<R>::vec*>(links),
                                                          Vh, nmat);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_import(const double* nat, void* links, const Geom& G, int NS, uint32_t copy, uint32_t t0,
                          uint32_t nt, cudaStream_t st) {
  const uint64_t n = (uint64_t)nt * G.V3 * 4;
  import_kernel<R><<<nblocks(n), BLOCK, 0, st>>>(nat, static_cast<typename store_traits<R>::vec*>(links), G,
                                                  NS, copy, t0, nt);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_export(double* nat, const void* links, const Geom& G, int NS, uint32_t copy, uint32_t t0,
                          uint32_t nt, cudaStream_t st) {
  const uint64_t n = (uint64_t)nt * G.V3 * 4;
  export_kernel<R><<<nblocks(n), BLOCK, 0, st>>>(nat, static_cast<const typename store_traits<R>::vec*>(links),
                                                  G, NS, copy, t0, nt);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_haar_transform(void* links, const Geom& G, int NS, uint32_t ncopies, uint32_t copy0,
                                  uint64_t seed, cudaStream_t st) {
  const uint64_t n = (uint64_t)ncopies * G.Vh;
  for (int p = 0; p < 2; ++p) {
    haar_transform_kernel<R><<<nblocks(n), BLOCK, 0, st>>>(static_cast<typename store_traits<R>::vec*>(links),
                                                            G, NS, p, ncopies, copy0, (uint32_t)seed,
                                                            (uint32_t)(seed >> 32));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_coulomb_fold(void* links, const Geom& G, uint32_t ncopies, cudaStream_t st) {
  const uint64_t n = (uint64_t)ncopies * G.V;
  coulomb_fold_kernel<R><<<nblocks(n), BLOCK, 0, st>>>(static_cast<typename store_traits<R>::vec*>(links), G,
                                                        ncopies);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_identity_slot<R>(links, G, 5, 4, ncopies, st);
}

template <typename R>
cudaError_t launch_identity_slot(void* links, const Geom& G, int NS, int slot, uint32_t ncopies,
                                 cudaStream_t st) {
  const uint64_t n = (uint64_t)ncopies * 2 * G.Vh;
  identity_slot_kernel<R><<<nblocks(n), BLOCK, 0, st>>>(static_cast<typename store_traits<R>::vec*>(links), G,
                                                         NS, slot, ncopies);
  return cudaGetLastError();
}

cudaError_t launch_philox(const void* ctr, void* out, uint64_t n, uint64_t seed, cudaStream_t st) {
  philox_kernel<<<nblocks(n), BLOCK, 0, st>>>(static_cast<const uint4*>(ctr), static_cast<uint4*>(out), n,
                                              (uint32_t)seed, (uint32_t)(seed >> 32));
  return cudaGetLastError();
}

cudaError_t launch_sync_master(void* l32, void* l64, void* gscratch, const Geom& G, int NS32, int NS64,
                               uint32_t ncopies, cudaStream_t st) {
  const uint64_t nsites = (uint64_t)ncopies * 2 * G.Vh;
  prepare_g_kernel<<<nblocks(nsites), BLOCK, 0, st>>>(static_cast<const float4*>(l32),
                                                       static_cast<double2*>(gscratch), G.Vh, NS32, nsites);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint64_t n = (uint64_t)ncopies * G.V * 4;
  sync_master_kernel<<<nblocks(n), BLOCK, 0, st>>>(static_cast<const double2*>(gscratch),
                                                    static_cast<float4*>(l32), static_cast<double2*>(l64), G,
                                                    NS32, NS64, ncopies);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_identity_slot<float>(l32, G, NS32, 4, ncopies, st);
}

cudaError_t launch_demote(const void* l64, void* l32, const Geom& G, int NS64, int NS32, uint32_t ncopies,
                          cudaStream_t st) {
  const uint64_t n = (uint64_t)ncopies * 2 * 4 * G.Vh;
  demote_kernel<<<nblocks(n), BLOCK, 0, st>>>(static_cast<const double2*>(l64), static_cast<float4*>(l32), G.Vh,
                                               NS64, NS32, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_identity_slot<float>(l32, G, NS32, 4, ncopies, st);
}

cudaError_t launch_obs_site_reduce(const void* obs_site, const Geom& G, int gauge, uint32_t ncopies, double* partial,
                                   double* out, cudaStream_t st) {
  const uint32_t bps = (G.V3 / 2 + BLOCK - 1) / BLOCK;  // fits the observables partial buffer
  const uint32_t nct = ncopies * (uint32_t)G.n[0];
  obs_site_reduce<<<dim3(bps, nct), BLOCK, 0, st>>>(static_cast<const double2*>(obs_site), G.V3, bps, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nd = gauge == COULOMB ? 3 : 4;
  obs_site_finish<<<(nct + 127) / 128, 128, 0, st>>>(partial, bps, nct, 1.0 / (3.0 * nd * (double)G.V3),
                                                      1.0 / (3.0 * (double)G.V3), out);
  return cudaGetLastError();
}

#define GF_INST(R)                                                                                         \
  template cudaError_t launch_observables<R>(const void*, const Geom&, int, int, uint32_t, double*, double*, \
                                             cudaStream_t);                                              \
  template cudaError_t launch_reunitarize<R>(void*, uint32_t, uint64_t, cudaStream_t);                     \
  template cudaError_t launch_import<R>(const double*, void*, const Geom&, int, uint32_t, uint32_t,        \
                                        uint32_t, cudaStream_t);                                         \
  template cudaError_t launch_export<R>(double*, const void*, const Geom&, int, uint32_t, uint32_t,        \
                                        uint32_t, cudaStream_t);                                         \
  template cudaError_t launch_haar_transform<R>(void*, const Geom&, int, uint32_t, uint32_t, uint64_t,     \
                                                cudaStream_t);                                           \
  template cudaError_t launch_coulomb_fold<R>(void*, const Geom&, uint32_t, cudaStream_t);                 \
  template cudaError_t launch_identity_slot<R>(void*, const Geom&, int, int, uint32_t, cudaStream_t);
GF_INST(float)
GF_INST(double)

}  // namespace gfk
