// gf_kernels.cuh -- auxiliary kernels: observables, re-unitarisation,
// precision switch, layout conversion, random gauge transformation and the
// Coulomb final transform.  Included by gf_aux.cu only.
#pragma once
#include "gf_sweep.cuh"

namespace gfk {

// ---------------------------------------------------------------------------
// Observables: exact FP64 functional and theta (Sec. 2.1) from the stored
// links, one thread per site.  Grid: x = blocks within a (copy, slice,
// parity) unit, y = unit.  Each block writes (F, theta) partial sums; a
// second kernel adds them per (copy, slice) in a fixed order.
template <typename R>
__device__ __forceinline__ void load_link_d(const typename store_traits<R>::vec* base, size_t off,
                                            uint32_t Vh, mat3<double>& ud) {
  mat3<R> u;
  load_rows(base + off, Vh, u);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) ud.e[a][b] = {(double)u.e[a][b].re, (double)u.e[a][b].im};
  reconstruct_row2(ud);
}

struct ObsArgs {
  Geom geom;
  int NS;
  int gauge;
  uint32_t ncopies;
  double* partial;  // [unit][blocks_per_unit][2], unit = (copy*Nt + t)*2 + parity
  uint32_t blocks_per_unit;
};

template <typename R>
__global__ void __launch_bounds__(BLOCK) observables_kernel(const typename store_traits<R>::vec* links,
                                                            const ObsArgs a) {
  constexpr int NC = store_traits<R>::NC;
  const Geom& G = a.geom;
  const uint32_t unit = blockIdx.y;
  const int p = (int)(unit & 1);
  const uint32_t ct = unit >> 1;
  const uint32_t copy = ct / (uint32_t)G.n[0];
  const uint32_t t = ct - copy * (uint32_t)G.n[0];
  const uint32_t half3 = G.V3 / 2;
  const uint32_t idx = blockIdx.x * BLOCK + threadIdx.x;
  double f = 0, th = 0;
  if (idx < half3) {
    const uint32_t sp = t * half3 + idx;
    int c[4];
    uint32_t s;
    site_coords(G, sp, p, c, s);
    const int mu0 = a.gauge == COULOMB ? 1 : 0;
    if (a.gauge == MAG) {
      // F: sum |U_ii|^2 over the up links; theta: sum over subgroups |X_01|^2
      double X[3][4] = {};  // per subgroup: X01.re, X01.im (unused), -, -
      double x01r[3] = {0, 0, 0}, x01i[3] = {0, 0, 0};
      for (int mu = 0; mu < 4; ++mu) {
        mat3<double> up, dn;
        load_link_d<R>(links, link_off(copy, p, mu, a.NS, NC, G.Vh, sp), G.Vh, up);
        load_link_d<R>(links, link_off(copy, p ^ 1, mu, a.NS, NC, G.Vh, site_minus(G, s, c, mu) >> 1),
                       G.Vh, dn);
        for (int k = 0; k < 3; ++k) f += up.e[k][k].re * up.e[k][k].re + up.e[k][k].im * up.e[k][k].im;
        for (int sub = 0; sub < 3; ++sub) {
          const int i = sub == 2 ? 1 : 0, j = sub == 0 ? 1 : 2;
          // up: (W s3 W^dag)_01 = W_ii conj(W_ji) - W_ij conj(W_jj)
          cx<double> A = up.e[i][i], B = up.e[i][j], C = up.e[j][i], D = up.e[j][j];
          cx<double> v = cmul2c(A, C, cx<double>{-B.re, -B.im}, D);
          // down: (D^dag s3 D)_01 = conj(D_ii) D_ij - conj(D_ji) D_jj
          cx<double> P = dn.e[i][i], Q = dn.e[i][j], Rr = dn.e[j][i], S = dn.e[j][j];
          cx<double> w = cmul2c(Q, P, cx<double>{-S.re, -S.im}, Rr);
          x01r[sub] += v.re + w.re;
          x01i[sub] += v.im + w.im;
        }
      }
      (void)X;
      for (int sub = 0; sub < 3; ++sub) th += x01r[sub] * x01r[sub] + x01i[sub] * x01i[sub];
    } else {
      mat3<double> K;
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int r = 0; r < 3; ++r) K.e[q][r] = {0.0, 0.0};
      for (int mu = mu0; mu < 4; ++mu) {
        mat3<double> up, dn;
        load_link_d<R>(links, link_off(copy, p, mu, a.NS, NC, G.Vh, sp), G.Vh, up);
        load_link_d<R>(links, link_off(copy, p ^ 1, mu, a.NS, NC, G.Vh, site_minus(G, s, c, mu) >> 1),
                       G.Vh, dn);
        f += up.e[0][0].re + up.e[1][1].re + up.e[2][2].re;
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            K.e[q][r].re += up.e[q][r].re + dn.e[r][q].re;
            K.e[q][r].im += up.e[q][r].im - dn.e[r][q].im;
          }
      }
      // Delta = traceless part of (K - K^dag)/(2i); tr[Delta Delta^dag]
      double d[3][3][2];
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          // (K_qr - conj(K_rq)) / (2i) = ((Im K_qr + Im K_rq) - i (Re K_qr - Re K_rq)) / 2
          d[q][r][0] = 0.5 * (K.e[q][r].im + K.e[r][q].im);
          d[q][r][1] = -0.5 * (K.e[q][r].re - K.e[r][q].re);
        }
      double tr3 = (d[0][0][0] + d[1][1][0] + d[2][2][0]) / 3.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) d[q][q][0] -= tr3;
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int r = 0; r < 3; ++r) th += d[q][r][0] * d[q][r][0] + d[q][r][1] * d[q][r][1];
    }
  }
  // block reduction in a fixed order
  __shared__ double sf[BLOCK / 32], st[BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_xor_sync(FULL, f, o);
    th += __shfl_xor_sync(FULL, th, o);
  }
  const int w = threadIdx.x / 32;
  if ((threadIdx.x & 31) == 0) {
    sf[w] = f;
    st[w] = th;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0, T = 0;
    for (int k = 0; k < BLOCK / 32; ++k) {
      F += sf[k];
      T += st[k];
    }
    double* out = a.partial + ((size_t)unit * a.blocks_per_unit + blockIdx.x) * 2;
    out[0] = F;
    out[1] = T;
  }
}

// Sum the partials of each (copy, slice) and normalise:
// F_t = sum / (3 * nd * V3), theta_t = sum / (3 * V3).
__global__ void observables_finish(const double* partial, uint32_t blocks_per_unit, uint32_t nunits_ct,
                                   double normF, double normT, double* out /* [ct][2] */) {
  const uint32_t ct = blockIdx.x * blockDim.x + threadIdx.x;
  if (ct >= nunits_ct) return;
  double F = 0, T = 0;
  for (int p = 0; p < 2; ++p) {
    const double* q = partial + ((size_t)(ct * 2 + p) * blocks_per_unit) * 2;
    for (uint32_t b = 0; b < blocks_per_unit; ++b) {
      F += q[2 * b];
      T += q[2 * b + 1];
    }
  }
  out[2 * ct] = F * normF;
  out[2 * ct + 1] = T * normT;
}

// ---------------------------------------------------------------------------
// Re-unitarisation of every stored matrix (links and, for Coulomb, the
// accumulated g), computed in FP64 whatever the storage precision.
template <typename R>
__global__ void __launch_bounds__(BLOCK) reunitarize_kernel(typename store_traits<R>::vec* links,
                                                            uint32_t Vh, uint64_t nmat) {
  constexpr int NC = store_traits<R>::NC;
  const uint64_t m = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (m >= nmat) return;
  const uint64_t blk = m / Vh, sp = m - blk * Vh;
  auto* p = links + blk * NC * Vh + sp;
  mat3<R> u;
  load_rows(p, Vh, u);
  mat3<double> d;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) d.e[a][b] = {(double)u.e[a][b].re, (double)u.e[a][b].im};
  gram_schmidt_rows(d);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) u.e[a][b] = {(R)d.e[a][b].re, (R)d.e[a][b].im};
  store_rows(p, Vh, u);
}

// ---------------------------------------------------------------------------
// Layout conversion between the natural order (t,x,y,z,mu,i,j,re/im; 18
// doubles per link) and the parity-split storage, for the time-slices
// [t0, t0 + nt) of one copy.  One thread per (site, mu).
template <typename R>
__global__ void __launch_bounds__(BLOCK) import_kernel(const double* __restrict__ nat,
                                                       typename store_traits<R>::vec* links, Geom G,
                                                       int NS, uint32_t copy, uint32_t t0, uint32_t nt) {
  constexpr int NC = store_traits<R>::NC;
  const uint64_t q = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (q >= (uint64_t)nt * G.V3 * 4) return;
  const uint32_t mu = (uint32_t)(q & 3);
  const uint32_t s = t0 * G.V3 + (uint32_t)(q >> 2);
  const uint32_t z = s % (uint32_t)G.n[3], y = (s / G.n[3]) % G.n[2], x = (s / (G.n[3] * G.n[2])) % G.n[1];
  const uint32_t t = s / G.V3;
  const int p = (int)((t + x + y + z) & 1);
  const double* src = nat + q * 18;
  mat3<R> u;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) u.e[a][b] = {(R)src[(a * 3 + b) * 2], (R)src[(a * 3 + b) * 2 + 1]};
  store_rows(links + link_off(copy, p, (int)mu, NS, NC, G.Vh, s >> 1), G.Vh, u);
}

template <typename R>
__global__ void __launch_bounds__(BLOCK) export_kernel(double* __restrict__ nat,
                                                       const typename store_traits<R>::vec* links, Geom G,
                                                       int NS, uint32_t copy, uint32_t t0, uint32_t nt) {
  constexpr int NC = store_traits<R>::NC;
  const uint64_t q = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (q >= (uint64_t)nt * G.V3 * 4) return;
  const uint32_t mu = (uint32_t)(q & 3);
  const uint32_t s = t0 * G.V3 + (uint32_t)(q >> 2);
  const uint32_t z = s % (uint32_t)G.n[3], y = (s / G.n[3]) % G.n[2], x = (s / (G.n[3] * G.n[2])) % G.n[1];
  const uint32_t t = s / G.V3;
  const int p = (int)((t + x + y + z) & 1);
  mat3<R> u;
  load_rows(links + link_off(copy, p, (int)mu, NS, NC, G.Vh, s >> 1), G.Vh, u);
  reconstruct_row2(u);
  double* dst = nat + q * 18;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      dst[(a * 3 + b) * 2] = (double)u.e[a][b].re;
      dst[(a * 3 + b) * 2 + 1] = (double)u.e[a][b].im;
    }
}

// ---------------------------------------------------------------------------
// Random gauge transformation U_mu(x) -> g(x) U_mu(x) g(x+mu)^dag with Haar
// g(x), done as two passes over the sublattices: sites of one parity apply
// their g(x) from the left to U_mu(x) and from the right (as g^dag) to
// U_mu(x-mu).  Every link has one endpoint of each parity, so after both
// passes it carries g(x) ... g(x+mu)^dag.  One thread per site draws g(x)
// once from the counter-based generator and updates the site's eight links.
template <typename R>
__global__ void __launch_bounds__(BLOCK) haar_transform_kernel(typename store_traits<R>::vec* links, Geom G,
                                                               int NS, int parity, uint32_t ncopies,
                                                               uint32_t copy0, uint32_t k0, uint32_t k1) {
  constexpr int NC = store_traits<R>::NC;
  const uint64_t gsite = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  const uint32_t copy = (uint32_t)(gsite / G.Vh);
  if (copy >= ncopies) return;
  const uint32_t sp = (uint32_t)(gsite - (uint64_t)copy * G.Vh);
  int c[4];
  uint32_t s;
  site_coords(G, sp, parity, c, s);
  Rng rng{k0, k1, s, 0u, copy0 + copy};
  mat3<R> g;
  haar_su3(rng, g);
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int mu = k >> 1;
    const bool down = k & 1;
    const size_t off = down ? link_off(copy, parity ^ 1, mu, NS, NC, G.Vh, site_minus(G, s, c, mu) >> 1)
                            : link_off(copy, parity, mu, NS, NC, G.Vh, sp);
    mat3<R> u, r;
    load_rows(links + off, G.Vh, u);
    reconstruct_row2(u);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        cx<R> acc{R(0), R(0)};
        if (!down) {  // (g u)_ab
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            cx<R> t = cmul(g.e[a][q], u.e[q][b]);
            acc.re += t.re;
            acc.im += t.im;
          }
        } else {  // (u g^dag)_ab = sum_q u_aq conj(g_bq)
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            cx<R> t = cmul(u.e[a][q], cx<R>{g.e[b][q].re, -g.e[b][q].im});
            acc.re += t.re;
            acc.im += t.im;
          }
        }
        r.e[a][b] = acc;
      }
    store_rows(links + off, G.Vh, r);
  }
}

// ---------------------------------------------------------------------------
// Coulomb: fold the accumulated g of the time-slice sweeps into the temporal
// links, U_0(x) <- g(x) U_0(x) g(x+0)^dag (Sec. 5.1: the final g(t) acts on
// U_0(t-1) as well), one thread per site; then reset g to the identity.
template <typename R>
__global__ void __launch_bounds__(BLOCK) coulomb_fold_kernel(typename store_traits<R>::vec* links, Geom G,
                                                             uint32_t ncopies) {
  constexpr int NC = store_traits<R>::NC;
  const uint64_t tid = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  const uint64_t per_copy = (uint64_t)G.V;
  const uint32_t copy = (uint32_t)(tid / per_copy);
  if (copy >= ncopies) return;
  const uint32_t r = (uint32_t)(tid - (uint64_t)copy * per_copy);
  const int p = r >= G.Vh;
  const uint32_t sp = r - (p ? G.Vh : 0);
  int c[4];
  uint32_t s;
  site_coords(G, sp, p, c, s);
  mat3<R> gx, gy, u, t;
  load_rows(links + link_off(copy, p, 4, 5, NC, G.Vh, sp), G.Vh, gx);
  reconstruct_row2(gx);
  load_rows(links + link_off(copy, p ^ 1, 4, 5, NC, G.Vh, site_plus(G, s, c, 0) >> 1), G.Vh, gy);
  reconstruct_row2(gy);
  const size_t off = link_off(copy, p, 0, 5, NC, G.Vh, sp);
  load_rows(links + off, G.Vh, u);
  reconstruct_row2(u);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cx<R> acc{R(0), R(0)};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        cx<R> v = cmul(gx.e[a][q], u.e[q][b]);
        acc.re += v.re;
        acc.im += v.im;
      }
      t.e[a][b] = acc;
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cx<R> acc{R(0), R(0)};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        cx<R> v = cmul(t.e[a][q], cx<R>{gy.e[b][q].re, -gy.e[b][q].im});
        acc.re += v.re;
        acc.im += v.im;
      }
      u.e[a][b] = acc;
    }
  store_rows(links + off, G.Vh, u);
}

// Set slot `slot` of every site to the identity (the Coulomb accumulator).
template <typename R>
__global__ void __launch_bounds__(BLOCK) identity_slot_kernel(typename store_traits<R>::vec* links, Geom G,
                                                              int NS, int slot, uint32_t ncopies) {
  constexpr int NC = store_traits<R>::NC;
  const uint64_t tid = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  const uint64_t per = (uint64_t)2 * G.Vh;
  const uint32_t copy = (uint32_t)(tid / per);
  if (copy >= ncopies) return;
  const uint32_t r = (uint32_t)(tid - (uint64_t)copy * per);
  const int p = r >= G.Vh;
  const uint32_t sp = r - (p ? G.Vh : 0);
  mat3<R> u;
  set_identity(u);
  store_rows(links + link_off(copy, p, slot, NS, NC, G.Vh, sp), G.Vh, u);
}

// Philox4x32-10 on n counters (4 words each) with the key (k0, k1).
__global__ void philox_kernel(const uint4* ctr, uint4* out, uint64_t n, uint32_t k0, uint32_t k1) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint4 c = ctr[i];
  u4 r = philox10(u4{c.x, c.y, c.z, c.w}, k0, k1);
  out[i] = make_uint4(r.x, r.y, r.z, r.w);
}

// ---------------------------------------------------------------------------
// Mixed precision, FP64 master: apply the gauge transformation accumulated by
// the FP32 sweeps (slot 4 of the FP32 array) to the FP64 links,
// U_mu(x) <- G(x) U_mu(x) G(x+mu)^dag in FP64 with G re-unitarised in FP64,
// and write the result back to both arrays (the FP32 copy re-rounded from the
// exact one).  First pass: one thread per site re-unitarises G(x) in FP64
// and keeps the full 3x3 in a scratch array ([copy][parity][9][Vh] double2).
// Second pass: one thread per (site, mu) forms rows 0 and 1 of
// G(x) U G(x+mu)^dag.  The accumulator is reset by a third launch.
__global__ void __launch_bounds__(BLOCK) prepare_g_kernel(const float4* l32, double2* gs, uint32_t Vh, int NS32,
                                                          uint64_t nsites) {
  const uint64_t m = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (m >= nsites) return;
  const uint64_t cp = m / Vh, sp = m - cp * Vh;  // cp = copy*2 + parity
  mat3<float> f;
  load_rows(l32 + ((cp * NS32 + 4) * 3) * Vh + sp, Vh, f);
  mat3<double> g;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) g.e[a][b] = {(double)f.e[a][b].re, (double)f.e[a][b].im};
  gram_schmidt_rows(g);
  reconstruct_row2(g);
  double2* o = gs + cp * 9 * Vh + sp;
#pragma unroll
  for (int k = 0; k < 9; ++k) o[(size_t)k * Vh] = make_double2(g.e[k / 3][k % 3].re, g.e[k / 3][k % 3].im);
}

__device__ __forceinline__ void load_g9(const double2* gs, uint32_t copy, int p, uint32_t Vh, uint32_t sp,
                                        mat3<double>& g) {
  const double2* q = gs + ((size_t)copy * 2 + p) * 9 * Vh + sp;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 v = q[(size_t)k * Vh];
    g.e[k / 3][k % 3] = {v.x, v.y};
  }
}

__global__ void __launch_bounds__(BLOCK) sync_master_kernel(const double2* gs, float4* l32, double2* l64, Geom G,
                                                            int NS32, int NS64, uint32_t ncopies) {
  const uint64_t tid = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  const uint64_t per_copy = (uint64_t)G.V * 4;
  const uint32_t copy = (uint32_t)(tid / per_copy);
  if (copy >= ncopies) return;
  const uint32_t r = (uint32_t)(tid - (uint64_t)copy * per_copy);
  const int mu = (int)(r & 3);
  const uint32_t site = r >> 2;  // 0 .. V-1 over both parities
  const int p = site >= G.Vh;
  const uint32_t sp = site - (p ? G.Vh : 0);
  int c[4];
  uint32_t s;
  site_coords(G, sp, p, c, s);
  mat3<double> gx, gy, u;
  load_g9(gs, copy, p, G.Vh, sp, gx);
  load_g9(gs, copy, p ^ 1, G.Vh, site_plus(G, s, c, mu) >> 1, gy);
  const size_t off64 = link_off(copy, p, mu, NS64, 6, G.Vh, sp);
  load_rows(l64 + off64, G.Vh, u);
  reconstruct_row2(u);
  // rows 0, 1 of G(x) U, then times G(x+mu)^dag
  cx<double> t[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cx<double> acc{0.0, 0.0};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        cx<double> v = cmul(gx.e[a][q], u.e[q][b]);
        acc.re += v.re;
        acc.im += v.im;
      }
      t[a][b] = acc;
    }
  mat3<float> f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cx<double> acc{0.0, 0.0};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        cx<double> v = cmul(t[a][q], cx<double>{gy.e[b][q].re, -gy.e[b][q].im});
        acc.re += v.re;
        acc.im += v.im;
      }
      u.e[a][b] = acc;
      f.e[a][b] = {(float)acc.re, (float)acc.im};
    }
  store_rows(l64 + off64, G.Vh, u);
  store_rows(l32 + link_off(copy, p, mu, NS32, 3, G.Vh, sp), G.Vh, f);
}

// FP32 copy <- FP64 master (links only), for a fresh start of the FP32 sweeps.
__global__ void __launch_bounds__(BLOCK) demote_kernel(const double2* l64, float4* l32, uint32_t Vh, int NS64,
                                                       int NS32, uint64_t nlinks) {
  const uint64_t m = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (m >= nlinks) return;
  const uint64_t sp = m % Vh;
  const uint64_t rest = m / Vh;  // (copy*2 + p)*4 + mu
  const uint64_t mu = rest & 3, cp = rest >> 2;
  mat3<double> d;
  load_rows(l64 + ((cp * NS64 + mu) * 6) * Vh + sp, Vh, d);
  mat3<float> f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) f.e[a][b] = {(float)d.e[a][b].re, (float)d.e[a][b].im};
  store_rows(l32 + ((cp * NS32 + mu) * 3) * Vh + sp, Vh, f);
}

// ---------------------------------------------------------------------------
// Reduction of the per-site observables the fused sweeps wrote
// ([copy][site] double2 (F, theta)): per (copy, time-slice) unit, block
// partials over the slice's contiguous sites, then a fixed-order sum.
__global__ void __launch_bounds__(BLOCK) obs_site_reduce(const double2* obs_site, uint32_t V3, uint32_t bps,
                                                         double* partial) {
  const uint32_t ct = blockIdx.y;
  const double2* q = obs_site + (size_t)ct * V3;
  double f = 0, th = 0;
  for (uint32_t i = blockIdx.x * BLOCK + threadIdx.x; i < V3; i += bps * BLOCK) {
    const double2 v = q[i];
    f += v.x;
    th += v.y;
  }
  __shared__ double sf[BLOCK / 32], st[BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_xor_sync(FULL, f, o);
    th += __shfl_xor_sync(FULL, th, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sf[threadIdx.x / 32] = f;
    st[threadIdx.x / 32] = th;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0, T = 0;
    for (int k = 0; k < BLOCK / 32; ++k) {
      F += sf[k];
      T += st[k];
    }
    partial[((size_t)ct * bps + blockIdx.x) * 2] = F;
    partial[((size_t)ct * bps + blockIdx.x) * 2 + 1] = T;
  }
}

__global__ void obs_site_finish(const double* partial, uint32_t bps, uint32_t nct, double normF, double normT,
                                double* out) {
  const uint32_t ct = blockIdx.x * blockDim.x + threadIdx.x;
  if (ct >= nct) return;
  double F = 0, T = 0;
  for (uint32_t b = 0; b < bps; ++b) {
    F += partial[((size_t)ct * bps + b) * 2];
    T += partial[((size_t)ct * bps + b) * 2 + 1];
  }
  out[2 * ct] = F * normF;
  out[2 * ct + 1] = T * normT;
}

}  // namespace gfk

