// gf_noalloc.cu -- gf_functional_theta_noalloc: the functional / theta
// reduction for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs under a fixed,
// pre-reserved device-memory budget (a serving loop whose pool is sized
// once at start-up, or a host framework that owns every allocation and
// forbids others), or code that must not trigger the allocator's implicit
// synchronisation on its hot path.  gf_functional_theta allocates through a
// context; this entry point needs none: the caller passes the links (device
// memory, natural order) and host pointers for the results, and the partial
// sums of the reduction live in a file-scope device array of fixed size that
// every GPU loading this library holds until the process exits.
#include <cstdio>
#include <mutex>

#include "gf.h"
#include "gf_device.cuh"
#include "gf_launch.h"

namespace {

using namespace gfk;

constexpr int NA_BLOCK = 256;
constexpr int NA_BLOCKS_PER_SLICE = 64;  // grid-stride within a time-slice

// Partial sums: [slice][block][2] doubles, then the per-slice results
// [slice][2].  1 MiB + 16 KiB.
__device__ __align__(256) double g_noalloc_scratch[GF_NOALLOC_MAX_NT * (NA_BLOCKS_PER_SLICE + 1) * 2];

struct NatLinks {
  const double* p;
  __device__ __forceinline__ void get(uint32_t s, int mu, mat3<double>& u) const {
    const double2* q = reinterpret_cast<const double2*>(p + ((size_t)s * 4 + mu) * 18);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = q[k];
      u.e[k / 3][k % 3] = {v.x, v.y};
    }
  }
};

__global__ void __launch_bounds__(NA_BLOCK) noalloc_partials(NatLinks L, Geom G, int gauge, double* scratch) {
  const uint32_t t = blockIdx.y;
  double f = 0, th = 0;
  for (uint32_t i = blockIdx.x * NA_BLOCK + threadIdx.x; i < G.V3; i += NA_BLOCKS_PER_SLICE * NA_BLOCK) {
    const uint32_t s = t * G.V3 + i;
    int c[4];
    c[3] = (int)(s % (uint32_t)G.n[3]);
    c[2] = (int)((s / (uint32_t)G.n[3]) % (uint32_t)G.n[2]);
    c[1] = (int)((s / G.stride[1]) % (uint32_t)G.n[1]);
    c[0] = (int)t;
    if (gauge == MAG) {
      double xr[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
      for (int mu = 0; mu < 4; ++mu) {
        mat3<double> up, dn;
        L.get(s, mu, up);
        L.get(site_minus(G, s, c, mu), mu, dn);
        for (int k = 0; k < 3; ++k) f += up.e[k][k].re * up.e[k][k].re + up.e[k][k].im * up.e[k][k].im;
        for (int sub = 0; sub < 3; ++sub) {
          const int a = sub == 2 ? 1 : 0, b = sub == 0 ? 1 : 2;
          // (W s3 W^dag)_01 + (D^dag s3 D)_01 of the (a,b) blocks
          cx<double> v = cmul2c(up.e[a][a], up.e[b][a], cx<double>{-up.e[a][b].re, -up.e[a][b].im}, up.e[b][b]);
          cx<double> w = cmul2c(dn.e[a][b], dn.e[a][a], cx<double>{-dn.e[b][b].re, -dn.e[b][b].im}, dn.e[b][a]);
          xr[sub] += v.re + w.re;
          xi[sub] += v.im + w.im;
        }
      }
      for (int sub = 0; sub < 3; ++sub) th += xr[sub] * xr[sub] + xi[sub] * xi[sub];
    } else {
      double kr[3][3] = {}, ki[3][3] = {};
      for (int mu = gauge == COULOMB ? 1 : 0; mu < 4; ++mu) {
        mat3<double> up, dn;
        L.get(s, mu, up);
        L.get(site_minus(G, s, c, mu), mu, dn);
        f += up.e[0][0].re + up.e[1][1].re + up.e[2][2].re;
        for (int q = 0; q < 3; ++q)
          for (int r = 0; r < 3; ++r) {
            kr[q][r] += up.e[q][r].re + dn.e[r][q].re;
            ki[q][r] += up.e[q][r].im - dn.e[r][q].im;
          }
      }
      // Delta = traceless part of (K - K^dag)/(2i)
      double dr[3][3], di[3][3];
      for (int q = 0; q < 3; ++q)
        for (int r = 0; r < 3; ++r) {
          dr[q][r] = 0.5 * (ki[q][r] + ki[r][q]);
          di[q][r] = -0.5 * (kr[q][r] - kr[r][q]);
        }
      const double tr3 = (dr[0][0] + dr[1][1] + dr[2][2]) / 3.0;
      for (int q = 0; q < 3; ++q) dr[q][q] -= tr3;
      for (int q = 0; q < 3; ++q)
        for (int r = 0; r < 3; ++r) th += dr[q][r] * dr[q][r] + di[q][r] * di[q][r];
    }
  }
  __shared__ double sf[NA_BLOCK / 32], st[NA_BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_xor_sync(0xffffffffu, f, o);
    th += __shfl_xor_sync(0xffffffffu, th, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sf[threadIdx.x / 32] = f;
    st[threadIdx.x / 32] = th;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0, T = 0;
    for (int k = 0; k < NA_BLOCK / 32; ++k) {
      F += sf[k];
      T += st[k];
    }
    // every (slice, block) entry in use is written by every call
    double* out = scratch + ((size_t)t * NA_BLOCKS_PER_SLICE + blockIdx.x) * 2;
    out[0] = F;
    out[1] = T;
  }
}

__global__ void noalloc_finish(double* scratch, uint32_t Nt, double normF, double normT) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Nt) return;
  double F = 0, T = 0;
  const double* q = scratch + (size_t)t * NA_BLOCKS_PER_SLICE * 2;
  for (int b = 0; b < NA_BLOCKS_PER_SLICE; ++b) {
    F += q[2 * b];
    T += q[2 * b + 1];
  }
  double* res = scratch + (size_t)GF_NOALLOC_MAX_NT * NA_BLOCKS_PER_SLICE * 2;
  res[2 * t] = F * normF;
  res[2 * t + 1] = T * normT;
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side name is only a stand-in for the symbol).
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch_ptr[MAX_DEVICES] = {nullptr};

cudaError_t scratch_for_current_device(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *ptr = g_scratch_ptr[dev];
  return cudaSuccess;
}

int na_fail(int code, const char* what) {
  gfk::set_last_error(what);
  return code;
}

}  // namespace

extern "C" int gf_functional_theta_noalloc(const int dims[4], gf_gauge gauge, const double* device_links,
                                           void* stream, double* F, double* theta, double* F_t,
                                           double* theta_t) {
  if (!dims || !device_links || !F || !theta) return na_fail(GF_EINVAL, "NULL argument");
  if (((uintptr_t)device_links & 15) != 0) return na_fail(GF_EINVAL, "device_links must be 16-byte aligned");
  uint64_t V = 1;
  for (int d = 0; d < 4; ++d) {
    if (dims[d] < 2 || (dims[d] & 1)) return na_fail(GF_EINVAL, "every extent must be even and >= 2");
    V *= (uint64_t)dims[d];
  }
  if (dims[0] > GF_NOALLOC_MAX_NT)
    return na_fail(GF_EINVAL, "Nt exceeds GF_NOALLOC_MAX_NT, the size of the static scratch array");
  if (V >= (1ull << 31)) return na_fail(GF_EINVAL, "lattice volume must be < 2^31");
  if (gauge < GF_LANDAU || gauge > GF_MAG) return na_fail(GF_EINVAL, "bad gauge");
  Geom G;
  for (int d = 0; d < 4; ++d) G.n[d] = dims[d];
  G.V3 = (uint32_t)dims[1] * dims[2] * dims[3];
  G.V = (uint32_t)V;
  G.Vh = G.V / 2;
  G.stride[0] = G.V3;
  G.stride[1] = (uint32_t)dims[2] * dims[3];
  G.stride[2] = (uint32_t)dims[3];
  G.stride[3] = 1;
  G.dz = make_fastdiv((uint32_t)dims[3]);
  G.dy = make_fastdiv((uint32_t)dims[2]);
  G.dx = make_fastdiv((uint32_t)dims[1]);
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return na_fail(e == cudaErrorNoDevice ? GF_ENOSYS : GF_ECUDA, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t Nt = (uint32_t)dims[0];
  noalloc_partials<<<dim3(NA_BLOCKS_PER_SLICE, Nt), NA_BLOCK, 0, st>>>(NatLinks{device_links}, G, gauge, scratch);
  const int nd = gauge == GF_COULOMB ? 3 : 4;
  noalloc_finish<<<(Nt + 127) / 128, 128, 0, st>>>(scratch, Nt, 1.0 / (3.0 * nd * (double)G.V3),
                                                   1.0 / (3.0 * (double)G.V3));
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(GF_ECUDA, cudaGetErrorString(e));
  double res[2 * GF_NOALLOC_MAX_NT];
  e = cudaMemcpyAsync(res, scratch + (size_t)GF_NOALLOC_MAX_NT * NA_BLOCKS_PER_SLICE * 2, 2 * Nt * sizeof(double),
                      cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(GF_ECUDA, cudaGetErrorString(e));
  double Fs = 0, Ts = 0;
  for (uint32_t t = 0; t < Nt; ++t) {
    Fs += res[2 * t];
    Ts += res[2 * t + 1];
    if (F_t) F_t[t] = res[2 * t];
    if (theta_t) theta_t[t] = res[2 * t + 1];
  }
  *F = Fs / Nt;
  *theta = Ts / Nt;
  return GF_OK;
}
