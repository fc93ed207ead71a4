// gf_launch.h -- host-side launchers of the device kernels (internal to libgf).
#pragma once
#include <cuda_runtime.h>

#include "gf_device.cuh"

namespace gfk {

template <typename R>
struct SweepArgs;

// One half-sweep of the given gauge/algorithm with lpt links per thread.
template <typename R>
cudaError_t launch_sweep(const SweepArgs<R>& a, int gauge, int algo, int lpt, cudaStream_t st);
// FP32 storage with Step 1 in FP64 (GF_MP).
cudaError_t launch_sweep_mp(const SweepArgs<float>& a, int gauge, int algo, int lpt, cudaStream_t st);

// One half-sweep (overrelaxation) of several lattices in one launch.
template <typename R>
struct GroupArgs;
template <typename R>
cudaError_t launch_group(const GroupArgs<R>& g, int gauge, int lpt, cudaStream_t st);

// Exact F/theta per (copy, slice) into out[ct][2] (device).
template <typename R>
cudaError_t launch_observables(const void* links, const Geom& G, int NS, int gauge, uint32_t ncopies,
                               double* partial, double* out, cudaStream_t st);
size_t observables_partial_doubles(const Geom& G, uint32_t ncopies);

template <typename R>
cudaError_t launch_reunitarize(void* links, uint32_t Vh, uint64_t nmat, cudaStream_t st);

template <typename R>
cudaError_t launch_import(const double* nat, void* links, const Geom& G, int NS, uint32_t copy, uint32_t t0,
                          uint32_t nt, cudaStream_t st);
template <typename R>
cudaError_t launch_export(double* nat, const void* links, const Geom& G, int NS, uint32_t copy, uint32_t t0,
                          uint32_t nt, cudaStream_t st);

template <typename R>
cudaError_t launch_haar_transform(void* links, const Geom& G, int NS, uint32_t ncopies, uint32_t copy0,
                                  uint64_t seed, cudaStream_t st);

template <typename R>
cudaError_t launch_coulomb_fold(void* links, const Geom& G, uint32_t ncopies, cudaStream_t st);

template <typename R>
cudaError_t launch_identity_slot(void* links, const Geom& G, int NS, int slot, uint32_t ncopies,
                                 cudaStream_t st);

// Mixed precision with an FP64 master: apply the FP32-accumulated gauge
// transformation (slot 4) to the FP64 links and re-round the FP32 copy, then
// reset the accumulator; and the plain FP64 -> FP32 copy (accumulator = 1).
cudaError_t launch_sync_master(void* l32, void* l64, void* gscratch, const Geom& G, int NS32, int NS64,
                               uint32_t ncopies, cudaStream_t st);
cudaError_t launch_demote(const void* l64, void* l32, const Geom& G, int NS64, int NS32, uint32_t ncopies,
                          cudaStream_t st);

// Per-(copy, slice) F/theta from the per-site values the fused sweeps wrote.
cudaError_t launch_obs_site_reduce(const void* obs_site, const Geom& G, int gauge, uint32_t ncopies, double* partial,
                                   double* out, cudaStream_t st);

// Record the calling thread's error message (read by gf_last_error).
void set_last_error(const char* msg);

cudaError_t launch_philox(const void* ctr, void* out, uint64_t n, uint64_t seed, cudaStream_t st);

}  // namespace gfk
