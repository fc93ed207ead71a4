// gf_sweep.cuh -- the checkerboard sweep kernel (Alg. 1, one sublattice per
// launch) and the helpers it shares with the auxiliary kernels.
#pragma once
#include "gf_device.cuh"

namespace gfk {

constexpr int BLOCK = 256;
constexpr unsigned FULL = 0xffffffffu;

template <typename R>
struct SweepArgs {
  typename store_traits<R>::vec* links;
  Geom geom;
  int NS;             // slots per site: 4, or 5 with the Coulomb accumulator
  int parity;         // active sublattice
  uint32_t ncopies;   // independent lattices in the batch
  uint32_t copy0;     // Philox copy id of copy 0
  const int* active;  // ncopies * Nt flags (time-slice units), or nullptr
  R param;            // omega (OR), p (SR), T (SA)
  uint32_t k0, k1;    // Philox key (the seed)
  uint32_t sweep;     // sweep index for the random draws
};

// Element offset of (copy, parity, slot, chunk 0, site index).
__device__ __forceinline__ size_t link_off(uint32_t copy, int p, int slot, int NS, int NC, uint32_t Vh,
                                           uint32_t sp) {
  return ((((size_t)copy * 2 + p) * NS + slot) * NC) * Vh + sp;
}

template <typename R>
__device__ __forceinline__ void dagger(mat3<R>& u) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u.e[a][a].im = -u.e[a][a].im;
#pragma unroll
    for (int b = a + 1; b < 3; ++b) {
      cx<R> t = u.e[a][b];
      u.e[a][b] = {u.e[b][a].re, -u.e[b][a].im};
      u.e[b][a] = {t.re, -t.im};
    }
  }
}

template <typename R>
__device__ __forceinline__ void set_identity(mat3<R>& u) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) u.e[a][b] = {R(a == b), R(0)};
}

// Left-multiply rows (i, j) of u by the SU(2) element of quaternion g.
template <typename R>
__device__ __forceinline__ void left_subgroup_mult(mat3<R>& u, int i, int j, const quat<R>& g) {
  cx<R> h00{g.q0, g.q3}, h01{g.q2, g.q1}, h10{-g.q2, g.q1}, h11{g.q0, -g.q3};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cx<R> a = u.e[i][k], b = u.e[j][k];
    u.e[i][k] = cmul2(h00, a, h01, b);
    u.e[j][k] = cmul2(h10, a, h11, b);
  }
}

// ---------------------------------------------------------------------------
// One half-sweep (Alg. 1 for one sublattice).  L = 8/LPT lanes share a site;
// lane l holds slots l*LPT .. l*LPT+LPT-1 of the site's eight links:
// slot k < 4 is U_k(x), slot k >= 4 is U_{k-4}(x - k)^dagger, so that every
// slot's K contribution (Eq. Kx) is its (i,j) block and every update is a
// left multiplication by g.  Per subgroup, the lanes' partial quaternions
// (Landau/Coulomb) or Pauli vectors (MAG) are summed with an xor butterfly of
// warp shuffles, which gives bit-identical sums in all lanes, so all lanes
// compute the same g (Step 1) and apply it to their own slots (Step 2).
// Coulomb: slot 0 holds the accumulated g(x) of the time-slice sweep (updated,
// not gathered) and slot 4 is idle; the temporal links are not touched.
template <typename R, int GAUGE, int ALGO, int LPT>
__global__ void __launch_bounds__(BLOCK) sweep_kernel(const SweepArgs<R> a) {
  using Vec = typename store_traits<R>::vec;
  constexpr int NC = store_traits<R>::NC;
  constexpr int L = 8 / LPT;
  const Geom& G = a.geom;
  const uint32_t Vh = G.Vh;
  const uint64_t tid = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
  const uint64_t gsite = tid / L;
  const int lane = (int)(threadIdx.x % L);
  const uint32_t copy = (uint32_t)(gsite / Vh);
  const uint32_t sp = (uint32_t)(gsite - (uint64_t)copy * Vh);
  bool valid = copy < a.ncopies;
  int c[4] = {0, 0, 0, 0};
  uint32_t s = 0;
  if (valid) {
    site_coords(G, sp, a.parity, c, s);
    if (a.active && !a.active[(size_t)copy * G.n[0] + c[0]]) valid = false;
  }

  mat3<R> u[LPT];
  size_t off[LPT];
  bool use[LPT], gather[LPT], down[LPT];
#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    const int k = lane * LPT + j;
    const int mu = k & 3;
    down[j] = k >= 4;
    gather[j] = !(GAUGE == COULOMB && mu == 0);
    use[j] = valid && !(GAUGE == COULOMB && k == 4);
    int slot = mu;
    uint32_t ssp = sp;
    int par = a.parity;
    if (GAUGE == COULOMB && k == 0) slot = 4;  // the accumulated g(x)
    if (down[j]) {
      ssp = site_minus(G, s, c, mu) >> 1;
      par ^= 1;
    }
    off[j] = link_off(copy, par, slot, a.NS, NC, Vh, ssp);
    if (use[j]) {
      load_rows(a.links + off[j], Vh, u[j]);
      reconstruct_row2(u[j]);
      if (down[j]) dagger(u[j]);
    } else {
      set_identity(u[j]);
    }
  }

  Rng rng{a.k0, a.k1, s, a.sweep, a.copy0 + copy};

#pragma unroll
  for (int sub = 0; sub < 3; ++sub) {
    const int i = sub == 2 ? 1 : 0;
    const int j2 = sub == 0 ? 1 : 2;
    quat<R> g;
    if (GAUGE == MAG) {
      // x = Pauli vector of sum W s3 W^dag over the slots' (i,j) blocks
      R x1 = 0, x2 = 0, x3 = 0;
#pragma unroll
      for (int j = 0; j < LPT; ++j) {
        if (!use[j]) continue;
        cx<R> A = u[j].e[i][i], B = u[j].e[i][j2], C = u[j].e[j2][i], D = u[j].e[j2][j2];
        cx<R> x01 = cmul2c(A, C, cx<R>{-B.re, -B.im}, D);  // A conj(C) - B conj(D)
        x1 += x01.re;
        x2 -= x01.im;
        x3 += R(0.5) * ((A.re * A.re + A.im * A.im) - (B.re * B.re + B.im * B.im) -
                        (C.re * C.re + C.im * C.im) + (D.re * D.re + D.im * D.im));
      }
#pragma unroll
      for (int o = 1; o < L; o <<= 1) {
        x1 += __shfl_xor_sync(FULL, x1, o);
        x2 += __shfl_xor_sync(FULL, x2, o);
        x3 += __shfl_xor_sync(FULL, x3, o);
      }
      R r;
      quat<R> m = mag_max(x1, x2, x3, r);
      if (ALGO == ALG_OR) g = rule_or(m, a.param);
      else if (ALGO == ALG_MICRO) g = mag_micro(x1, x2, x3, r);
      else if (ALGO == ALG_SR) {
        double ua, ub;
        rng.draw2(TAG_SR, (uint32_t)sub, 0, ua, ub);
        g = ((R)ua < a.param) ? mag_micro(x1, x2, x3, r) : rule_or(m, R(1));
      } else {
        g = rule_sa_mag(m, r, a.param, rng, (uint32_t)sub);
      }
    } else {
      // quaternion of the (i,j) block of K (getSubgroupQuaternion, App. A)
      R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
      for (int j = 0; j < LPT; ++j) {
        if (!(use[j] && gather[j])) continue;
        cx<R> W00 = u[j].e[i][i], W01 = u[j].e[i][j2], W10 = u[j].e[j2][i], W11 = u[j].e[j2][j2];
        a0 += W00.re + W11.re;
        a1 += W01.im + W10.im;
        a2 += W01.re - W10.re;
        a3 += W00.im - W11.im;
      }
#pragma unroll
      for (int o = 1; o < L; o <<= 1) {
        a0 += __shfl_xor_sync(FULL, a0, o);
        a1 += __shfl_xor_sync(FULL, a1, o);
        a2 += __shfl_xor_sync(FULL, a2, o);
        a3 += __shfl_xor_sync(FULL, a3, o);
      }
      quat<R> m{a0, -a1, -a2, -a3};  // maximiser of Re tr(g W)
      if (ALGO == ALG_OR) g = rule_or(m, a.param);
      else if (ALGO == ALG_MICRO) g = rule_micro(m);
      else if (ALGO == ALG_SR) {
        double ua, ub;
        rng.draw2(TAG_SR, (uint32_t)sub, 0, ua, ub);
        g = ((R)ua < a.param) ? rule_micro(m) : rule_or(m, R(1));
      } else {
        g = rule_sa_landau(m, a.param, rng, (uint32_t)sub);
      }
    }
#pragma unroll
    for (int j = 0; j < LPT; ++j) left_subgroup_mult(u[j], i, j2, g);
  }

#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    if (!use[j]) continue;
    if (down[j]) dagger(u[j]);
    store_rows(a.links + off[j], Vh, u[j]);
  }
}

}  // namespace gfk
