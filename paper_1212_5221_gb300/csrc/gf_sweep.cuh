// gf_sweep.cuh -- the checkerboard sweep kernel (Alg. 1, one sublattice per
// launch) and the helpers it shares with the auxiliary kernels.
#pragma once
#include <type_traits>

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
  int prefetch;       // 1: prefetch the next tile into L2
  int acc;            // 1: slot 4 accumulates g(x) (mixed precision; never for Coulomb,
                      //    whose slot 0 already does)
  int obs;            // fused observables: 0 none; 1 theta of the gathered K (before any
                      //    update); 2 F and theta of the updated links (odd half-sweep)
  int update;         // 0: read-only pass (with obs = 1): gather, no update, no store
  double2* obs_site;  // [copy][site] (F, theta) contributions written by lane 0
  int* err;           // set to 1 if a shared-memory staging wait ran out (prefetch 2)
  int wait_polls;     // polls of a staging wait before it gives up: < 0 the default
                      // (2^24, about 2 s), 0 none (the wait runs out at once)
  int* sa_trace;      // heat bath only, or nullptr: [copy][site][subgroup] Kennedy-Pendleton
                      // trial counts (0 = none accepted; MAG: 1), written by lane 0
  uint32_t site_offset;  // added to the site index in the Philox counters (time slabs: the
                         // global index of a local site)
  uint32_t sp_lo, sp_n;  // FP64 storage: the launch covers sites [sp_lo, sp_lo + sp_n) of
                         // each copy (0, Vh for all; a time-slab part its slices).  The
                         // FP32 kernels deal whole tiles round-robin over all Vh sites,
                         // which spreads any set of active slices over every block already
};

// Per-site FP64 observables of the MAG form from the slot matrices M
// (M = U_mu(x) for up slots, U_mu(x-mu)^dag for down slots).  Each slot is
// taken as stored: the two stored rows of its link, with the third rebuilt
// as conj(row0 x row1) in FP64 (exactly what a later read of the links
// gives).  theta_site = sum over subgroups |X_01|^2 with X = sum of the
// blocks' W s3 W^dag; F_site = sum of |M_kk|^2.  Each lane adds its own slots
// in FP64; an xor butterfly combines the lanes of the site.
template <typename R>
__device__ __forceinline__ void stored_slot(const mat3<R>& m, bool down, mat3<double>& d) {
  if (!down) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) d.e[a][b] = {(double)m.e[a][b].re, (double)m.e[a][b].im};
    reconstruct_row2(d);
  } else {
    mat3<double> u;  // the stored link is M^dag: rows 0,1 = conj of M's columns 0,1
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) u.e[a][b] = {(double)m.e[b][a].re, -(double)m.e[b][a].im};
    reconstruct_row2(u);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) d.e[a][b] = {u.e[b][a].re, -u.e[b][a].im};
  }
}

template <typename R, int LPT>
__device__ __forceinline__ void site_observables_mag(const mat3<R> (&u)[LPT], const bool (&use)[LPT], int lane,
                                                     double& F, double& theta) {
  constexpr int L = 8 / LPT;
  F = 0.0;
  theta = 0.0;
  double xr[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    if (!use[j]) continue;
    mat3<double> m;
    stored_slot(u[j], (LPT >= 2) ? (j & 1) : ((lane * LPT + j) & 1), m);
#pragma unroll
    for (int k = 0; k < 3; ++k) F += m.e[k][k].re * m.e[k][k].re + m.e[k][k].im * m.e[k][k].im;
#pragma unroll
    for (int sub = 0; sub < 3; ++sub) {
      const int i = sub == 2 ? 1 : 0, i2 = sub == 0 ? 1 : 2;
      const cx<double> A = m.e[i][i], B = m.e[i][i2], C = m.e[i2][i], D = m.e[i2][i2];
      // A conj(C) - B conj(D)
      xr[sub] += A.re * C.re + A.im * C.im - B.re * D.re - B.im * D.im;
      xi[sub] += A.im * C.re - A.re * C.im - B.im * D.re + B.re * D.im;
    }
  }
#pragma unroll
  for (int o = 1; o < L; o <<= 1) {
    F += __shfl_xor_sync(FULL, F, o);
#pragma unroll
    for (int sub = 0; sub < 3; ++sub) {
      xr[sub] += __shfl_xor_sync(FULL, xr[sub], o);
      xi[sub] += __shfl_xor_sync(FULL, xi[sub], o);
    }
  }
#pragma unroll
  for (int sub = 0; sub < 3; ++sub) theta += xr[sub] * xr[sub] + xi[sub] * xi[sub];
}

// Element offset of (copy, parity, slot, chunk 0, site index).
__host__ __device__ __forceinline__ size_t link_off(uint32_t copy, int p, int slot, int NS, int NC, uint32_t Vh,
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
// L2 prefetch of the links a tile of sites will touch: for every slot and
// chunk, one cp.async.bulk.prefetch.L2 of the contiguous range of parity
// indices it covers.  Up-links of sites [sp0, sp0+n) occupy the same range
// of their arrays; the down-link neighbours x - mu of those sites occupy
// [sp0 - d_mu - 1, sp0 + n - d_mu + 1) of the other parity's arrays
// (d_mu = stride_mu / 2 for mu < 3, 0 for z), except for sites on the
// periodic boundary, which are simply not prefetched.  Ranges are clipped to
// [0, Vh), so no prefetch leaves the allocation.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename R, int GAUGE>
__device__ __forceinline__ void prefetch_tile(const SweepArgs<R>& a, uint32_t copy, uint32_t sp0, uint32_t n,
                                              int job) {
  constexpr int NC = store_traits<R>::NC;
  const int chunk = job % NC;
  const int k = job / NC;  // slot 0..7: mu = k >> 1, down = k & 1; 8: the accumulator
  if (k == 8) {  // GF_MIXED's accumulated transformation of the tile's sites (slot 4)
    if (GAUGE == COULOMB || !a.acc) return;
    const auto* base = a.links + link_off(copy, a.parity, 4, a.NS, NC, a.geom.Vh, 0) + (size_t)chunk * a.geom.Vh;
    prefetch_l2(base + sp0, n * 16u);
    return;
  }
  const int mu = k >> 1;
  const bool down = k & 1;
  if (GAUGE == COULOMB && mu == 0 && down) return;  // idle slot
  const int slot = (GAUGE == COULOMB && mu == 0) ? 4 : mu;
  const int64_t Vh = a.geom.Vh;
  int64_t lo = sp0, hi = (int64_t)sp0 + n;
  int par = a.parity;
  if (down) {
    const int64_t d = mu == 3 ? 0 : (int64_t)(a.geom.stride[mu] / 2);
    lo = lo - d - 1;
    hi = hi - d + 1;
    par ^= 1;
  }
  if (lo < 0) lo = 0;
  if (hi > Vh) hi = Vh;
  if (hi <= lo) return;
  const auto* base = a.links + link_off(copy, par, slot, a.NS, NC, (uint32_t)Vh, 0) + (size_t)chunk * Vh;
  prefetch_l2(base + lo, (uint32_t)((hi - lo) * 16));
}

// ---------------------------------------------------------------------------
// Shared-memory staging of a tile (FP32 storage, prefetch mode 2).  While a
// block processes one tile from one of two stage buffers, its next tile's
// links are copied into the other by bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on an mbarrier per buffer).
// Region (k, chunk) of a buffer holds chunk `chunk` of slot k (k = 2 mu + d
// for the links, k = 8 for the mixed-precision accumulator) for the parity
// indices [lo_k, lo_k + extent_k): the tile's own range for up-links and the
// accumulator, the range of prefetch_tile for down-links.  Indices outside
// [0, Vh) are not copied; a site whose neighbour index lies outside the
// copied range (periodic wrap) reads global memory instead.  Each link a
// tile's sites read is written only by those sites (one active endpoint per
// link in a half-sweep), so staged values are never stale.
template <int TILE>
struct StageGeom {
  static constexpr int RS = TILE + 3;  // TILE + 2 rounded up to odd: link regions of the two lanes of a
                                       // site fall 16 banks apart
  static constexpr int ACC0 = 24 * RS;
  static constexpr int VEC = 24 * RS + 3 * TILE;  // float4 per buffer
  static constexpr size_t BYTES = (size_t)VEC * 16;
  __device__ static int base(int k, int chunk) { return k < 8 ? (k * 3 + chunk) * RS : ACC0 + chunk * TILE; }
  __device__ static int stride(int k) { return k < 8 ? RS : TILE; }
};

// Dynamic shared memory of the staged sweep: two buffers and two mbarriers.
template <int LPT>
constexpr size_t stage_smem_bytes() {
  return 2 * StageGeom<BLOCK / (8 / LPT)>::BYTES + 16;
}

// Dynamic shared memory of the non-staged FP32 sweep with GF_MIXED's
// accumulator: the three vectors of every site of a tile.
template <int LPT>
constexpr size_t acc_smem_bytes() {
  return (size_t)3 * (BLOCK / (8 / LPT)) * 16;
}

__device__ __forceinline__ void stage_range(const Geom& G, uint32_t sp0, uint32_t tile, int k, int64_t& lo,
                                            uint32_t& clo, uint32_t& chi) {
  int64_t ext = tile;
  lo = sp0;
  if (k < 8 && (k & 1)) {
    const int mu = k >> 1;
    const uint32_t st = mu == 0 ? G.stride[0] : mu == 1 ? G.stride[1] : mu == 2 ? G.stride[2] : 0u;
    lo = (int64_t)sp0 - (int64_t)(st / 2) - 1;
    ext = (int64_t)tile + 2;
  }
  // clipped to [0, Vh) in signed arithmetic: a down-link range near the start
  // of the lattice can end below zero (empty then)
  int64_t c0 = lo < 0 ? 0 : lo, c1 = lo + ext;
  if (c1 > (int64_t)G.Vh) c1 = G.Vh;
  if (c0 > (int64_t)G.Vh) c0 = G.Vh;
  if (c1 < c0) c1 = c0;
  clo = (uint32_t)c0;
  chi = (uint32_t)c1;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity to complete, for at most about
// two seconds and max_polls polls; false if it did not.
constexpr uint32_t WAIT_POLLS = 1u << 24;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t max_polls = WAIT_POLLS) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t i = 0; i < max_polls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && globaltimer_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Warp 0 of the block: copy the tile at (copy, sp0) into buffer buf and arm
// its mbarrier with the byte count.  Lane r < 24 copies region (r / 3, r % 3),
// lanes 24..26 the accumulator's chunks when the accumulator is in use.
template <int GAUGE, int TILE>
__device__ __forceinline__ void stage_issue(const SweepArgs<float>& a, uint32_t copy, uint32_t sp0, float4* buf,
                                            uint32_t bar, int lane) {
  using SG = StageGeom<TILE>;
  uint32_t bytes = 0, dst = 0;
  const float4* src = nullptr;
  const bool acc = GAUGE != COULOMB && a.acc;
  if (lane < 24 || (acc && lane < 27)) {
    const int k = lane < 24 ? lane / 3 : 8;
    const int chunk = lane < 24 ? lane % 3 : lane - 24;
    if (!(GAUGE == COULOMB && k == 1)) {  // Coulomb: U_0(x - 0) is not touched
      int64_t lo;
      uint32_t clo, chi;
      stage_range(a.geom, sp0, TILE, k, lo, clo, chi);
      if (chi > clo) {
        const int mu = k >> 1;
        const bool down = k < 8 && (k & 1);
        const int par = down ? a.parity ^ 1 : a.parity;
        const int slot = k == 8 ? 4 : (GAUGE == COULOMB && mu == 0) ? 4 : mu;
        src = a.links + link_off(copy, par, slot, a.NS, 3, a.geom.Vh, 0) + (size_t)chunk * a.geom.Vh + clo;
        dst = smem_u32(buf + SG::base(k, chunk) + (int)(clo - lo));
        bytes = (chi - clo) * 16u;
      }
    }
  }
  const uint32_t total = __reduce_add_sync(FULL, bytes);
  if (lane == 0) mbar_arrive_expect_tx(bar, total);
  __syncwarp();
  if (bytes) bulk_g2s(dst, src, bytes, bar);
}

// Rows 0,1 of slot k's link at parity index idx: from the stage buffer when
// it holds that index, else from global memory.
template <typename R, int TILE>
__device__ __forceinline__ void load_slot(const float4* stage, const Geom& G, uint32_t sp0, int k, uint32_t idx,
                                          const typename store_traits<R>::vec* g, uint32_t Vh, mat3<R>& u) {
  if constexpr (sizeof(R) == 4) {
    if (stage) {
      int64_t lo;
      uint32_t clo, chi;
      stage_range(G, sp0, TILE, k, lo, clo, chi);
      if (idx >= clo && idx < chi) {
        using SG = StageGeom<TILE>;
        const float4* p = stage + SG::base(k, 0) + (int)(idx - lo);
        const int rs = SG::stride(k);
        const float4 x = p[0], y = p[rs], z = p[2 * rs];
        u.e[0][0] = {x.x, x.y};
        u.e[0][1] = {x.z, x.w};
        u.e[0][2] = {y.x, y.y};
        u.e[1][0] = {y.z, y.w};
        u.e[1][1] = {z.x, z.y};
        u.e[1][2] = {z.z, z.w};
        return;
      }
    }
  }
  load_rows(g, Vh, u);
}

// ---------------------------------------------------------------------------
// One half-sweep (Alg. 1 for one sublattice), MAG form.  L = 8/LPT lanes
// share a site; lane l holds slots l*LPT .. l*LPT+LPT-1 of the site's eight
// links, slot k = 2 mu + d: d = 0 is U_mu(x), d = 1 is U_mu(x - mu)^dagger,
// so that every update is a left multiplication by g.  MAG's subgroup vector
// is quadratic in the links, so each subgroup is applied to every slot
// before the next subgroup's vector is formed.  Per subgroup, the lanes'
// partial Pauli vectors are summed with an xor butterfly of warp shuffles,
// which gives bit-identical sums in all lanes, so all lanes compute the same
// g (Step 1) and apply it to their own slots (Step 2).  The grid is
// persistent over tiles of BLOCK/L sites.
template <typename R, int ALGO, int LPT, bool OBS, bool MP>
__device__ __forceinline__ void sweep_site_mag(const SweepArgs<R>& a, uint32_t copy, uint32_t sp, bool valid,
                                               int lane, const float4* stage, uint32_t sp0) {
  // S: the precision Step 1 runs in (FP64 for the MP variant of FP32 storage)
  using S = typename std::conditional<MP, double, R>::type;
  constexpr uint32_t TILE = BLOCK / (8 / LPT);
  constexpr int NC = store_traits<R>::NC;
  constexpr int L = 8 / LPT;
  const Geom& G = a.geom;
  const uint32_t Vh = G.Vh;
  int c[4] = {0, 0, 0, 0};
  uint32_t s = 0;
  if (valid) {
    site_coords(G, sp, a.parity, c, s);
    if (a.active && !a.active[(size_t)copy * G.n[0] + c[0]]) valid = false;
  }

  // rows re-projected at load (see reproject_rows): every FP32 kernel, and the
  // FP64 kernels whose rotations stay large (heat bath, microcanonical, SR);
  // FP64 overrelaxation converges to small rotations and is re-unitarised
  // periodically by the driver instead.  A read-only pass leaves them as stored.
  const bool NORM = (sizeof(R) == 4 || ALGO != ALG_OR) && (!OBS || a.update);
  mat3<R> u[LPT];
  uint32_t idx[LPT];  // parity index of each slot's link (its offset is recomputed at the store)
  bool use[LPT];
#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    const int k = lane * LPT + j;
    const int mu = k >> 1;
    const bool down = (LPT >= 2) ? (j & 1) : (k & 1);
    use[j] = valid;
    uint32_t ssp = sp;
    int par = a.parity;
    if (down) {
      // x - mu without dynamic indexing of the coordinate arrays
      const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
      const int nm = mu == 0 ? G.n[0] : mu == 1 ? G.n[1] : mu == 2 ? G.n[2] : G.n[3];
      const uint32_t st = mu == 0 ? G.stride[0] : mu == 1 ? G.stride[1] : mu == 2 ? G.stride[2] : 1u;
      ssp = (cm > 0 ? s - st : s + (uint32_t)(nm - 1) * st) >> 1;
      par ^= 1;
    }
    idx[j] = ssp;
    if (use[j]) {
      load_slot<R, TILE>(stage, G, sp0, k, ssp, a.links + link_off(copy, par, mu, a.NS, NC, Vh, ssp), Vh, u[j]);
      if (NORM) reproject_rows(u[j]);
      reconstruct_row2(u[j]);
      if (down) dagger(u[j]);
    } else {
      set_identity(u[j]);
    }
  }

  // mixed precision: the accumulated gauge transformation of this site (the
  // FP32 working copy only, so FP64 kernels carry no code for it)
  constexpr bool CAN_ACC = sizeof(R) == 4;
  const bool acc = CAN_ACC && a.acc;
  mat3<R> gacc;
  size_t acc_off = 0;
  const bool use_acc = acc && valid && lane == 0;
  if (acc) {
    if (use_acc) {
      acc_off = link_off(copy, a.parity, 4, a.NS, NC, Vh, sp);
      load_slot<R, TILE>(stage, G, sp0, 8, sp, a.links + acc_off, Vh, gacc);
      reproject_rows(gacc);
      reconstruct_row2(gacc);
    } else {
      set_identity(gacc);
    }
  }

  Rng rng{a.k0, a.k1, s + a.site_offset, a.sweep, a.copy0 + copy};

  if (OBS && a.obs == 1) {  // theta of the current links at this site
    double F, th;
    site_observables_mag<R, LPT>(u, use, lane, F, th);
    if (valid && lane == 0) a.obs_site[(size_t)copy * G.V + s] = make_double2(0.0, th);
  }
  if (OBS && !a.update) return;

#pragma unroll
  for (int sub = 0; sub < 3; ++sub) {
    const int i = sub == 2 ? 1 : 0;
    const int j2 = sub == 0 ? 1 : 2;
    // x = Pauli vector of sum W s3 W^dag over the slots' (i,j) blocks
    S x1 = 0, x2 = 0, x3 = 0;
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
      if (!use[j]) continue;
      const cx<S> A{(S)u[j].e[i][i].re, (S)u[j].e[i][i].im}, B{(S)u[j].e[i][j2].re, (S)u[j].e[i][j2].im};
      const cx<S> C{(S)u[j].e[j2][i].re, (S)u[j].e[j2][i].im}, D{(S)u[j].e[j2][j2].re, (S)u[j].e[j2][j2].im};
      cx<S> x01 = cmul2c(A, C, cx<S>{-B.re, -B.im}, D);  // A conj(C) - B conj(D)
      x1 += x01.re;
      x2 -= x01.im;
      x3 += S(0.5) * ((A.re * A.re + A.im * A.im) - (B.re * B.re + B.im * B.im) -
                      (C.re * C.re + C.im * C.im) + (D.re * D.re + D.im * D.im));
    }
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
      x1 += __shfl_xor_sync(FULL, x1, o);
      x2 += __shfl_xor_sync(FULL, x2, o);
      x3 += __shfl_xor_sync(FULL, x3, o);
    }
    S r;
    quat<S> m = mag_max(x1, x2, x3, r);
    quat<S> gs;
    if (ALGO == ALG_OR) gs = rule_or(m, (S)a.param);
    else if (ALGO == ALG_MICRO) gs = mag_micro(x1, x2, x3, r);
    else if (ALGO == ALG_SR) {
      double ua, ub;
      rng.draw2(TAG_SR, (uint32_t)sub, 0, ua, ub);
      gs = ((S)ua < (S)a.param) ? mag_micro(x1, x2, x3, r) : rule_or(m, S(1));
    } else {
      gs = rule_sa_mag(m, r, (S)a.param, rng, (uint32_t)sub);
      if (a.sa_trace && valid && lane == 0) a.sa_trace[((size_t)copy * G.V + s) * 3 + sub] = 1;
    }
    const quat<R> g{(R)gs.q0, (R)gs.q1, (R)gs.q2, (R)gs.q3};
#pragma unroll
    for (int j = 0; j < LPT; ++j) left_subgroup_mult(u[j], i, j2, g);
    if (acc) left_subgroup_mult(gacc, i, j2, g);
  }
  if (use_acc) store_rows(a.links + acc_off, Vh, gacc);
  if (OBS && a.obs == 2) {  // F (every link is written once in a half-sweep) and theta after the update
    double F, th;
    site_observables_mag<R, LPT>(u, use, lane, F, th);
    if (valid && lane == 0) a.obs_site[(size_t)copy * G.V + s] = make_double2(F, th);
  }

#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    if (!use[j]) continue;
    const int k = lane * LPT + j;
    const bool down = (LPT >= 2) ? (j & 1) : (k & 1);
    if (down) dagger(u[j]);
    store_rows(a.links + link_off(copy, a.parity ^ (int)down, k >> 1, a.NS, NC, Vh, idx[j]), Vh, u[j]);
  }
}

// ---------------------------------------------------------------------------
// Landau and Coulomb gauge: the same half-sweep in K form.  Because every
// subgroup step left-multiplies all of a site's slots by the same g, the
// gathered K (Eq. Kx) obeys K <- g K, and the slots need the product
// G = g2 g1 g0 only once (Step 2 of Alg. 1 applied after the three Step-1
// subgroup choices; identical in exact arithmetic to updating the links
// subgroup by subgroup).  The three quaternions are taken from K, of which
// only the entries that a later subgroup reads are kept current.  Up-links
// become G U (rows 0,1, which read all three rows of U), down-links D G^dag
// (rows 0,1 of D only).  FP64 with eight links per lane reads the links
// again for the update (from L2) instead of holding all eight in registers.
template <typename R>
struct su2m {  // [[h00 h01] [h10 h11]] of a unit quaternion (Cayley-Klein form)
  cx<R> h00, h01, h10, h11;
};
template <typename R>
__device__ __forceinline__ su2m<R> su2_of(const quat<R>& g) {
  return {{g.q0, g.q3}, {g.q2, g.q1}, {-g.q2, g.q1}, {g.q0, -g.q3}};
}

// Step 1 for subgroup (i, j) of the current K entries: the maximiser of
// Re tr(g W) and the update rule of the algorithm.
template <typename R, int ALGO>
__device__ __forceinline__ quat<R> choose_k(cx<R> W00, cx<R> W01, cx<R> W10, cx<R> W11, R param, const Rng& rng,
                                            uint32_t sub, int* trace) {
  const quat<R> m{W00.re + W11.re, -(W01.im + W10.im), -(W01.re - W10.re), -(W00.im - W11.im)};
  if (ALGO == ALG_OR) return rule_or(m, param);
  if (ALGO == ALG_MICRO) return rule_micro(m);
  if (ALGO == ALG_SR) {
    double ua, ub;
    rng.draw2(TAG_SR, sub, 0, ua, ub);
    return ((R)ua < param) ? rule_micro(m) : rule_or(m, R(1));
  }
  int trials;
  const quat<R> g = rule_sa_landau(m, param, rng, sub, trials);
  if (trace) trace[sub] = trials;
  return g;
}

// What F and theta need of K = sum of the site's slot matrices M, in FP64:
// the antihermitian part of K, as ah[0..2] = Im K_aa, ah[3..5] = Re(K_ab -
// K_ba) and ah[6..8] = Im(K_ab + K_ba) for (a,b) = (0,1), (0,2), (1,2), and
// ah[9] = Re tr K (10 reals instead of K's 18).  A down slot M = D^dag
// contributes minus the antihermitian part of D and Re tr D.  Each slot is
// taken from its stored rows, row 2 rebuilt in FP64 (what a later read gives).
template <typename R>
__device__ __forceinline__ void add_stored_ah(const mat3<R>& rows, bool down, double (&ah)[10]) {
  mat3<double> d;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) d.e[a][b] = {(double)rows.e[a][b].re, (double)rows.e[a][b].im};
  reconstruct_row2(d);
  const double sg = down ? -1.0 : 1.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) ah[a] += sg * d.e[a][a].im;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int a = p == 2 ? 1 : 0, b = p == 0 ? 1 : 2;
    ah[3 + p] += sg * (d.e[a][b].re - d.e[b][a].re);
    ah[6 + p] += sg * (d.e[a][b].im + d.e[b][a].im);
  }
  ah[9] += d.e[0][0].re + d.e[1][1].re + d.e[2][2].re;
}

// The same ten reals of a gathered K.
template <typename R>
__device__ __forceinline__ void ah_of_k(const mat3<R>& K, double (&ah)[10]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) ah[a] = (double)K.e[a][a].im;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int a = p == 2 ? 1 : 0, b = p == 0 ? 1 : 2;
    ah[3 + p] = (double)K.e[a][b].re - (double)K.e[b][a].re;
    ah[6 + p] = (double)K.e[a][b].im + (double)K.e[b][a].im;
  }
  ah[9] = (double)K.e[0][0].re + (double)K.e[1][1].re + (double)K.e[2][2].re;
}

// theta_site = tr[Delta Delta^dag], Delta = traceless part of (K - K^dag)/(2i):
// its diagonal is Im K_aa minus their mean, its (a,b) and (b,a) entries have
// real part (Im K_ab + Im K_ba)/2 and imaginary parts -/+ (Re K_ab - Re K_ba)/2.
__device__ __forceinline__ double theta_of_ah(const double (&ah)[10]) {
  const double tr3 = (ah[0] + ah[1] + ah[2]) / 3.0;
  double th = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) th += (ah[a] - tr3) * (ah[a] - tr3);
#pragma unroll
  for (int p = 0; p < 3; ++p) th += 0.5 * (ah[3 + p] * ah[3 + p] + ah[6 + p] * ah[6 + p]);
  return th;
}

template <int L>
__device__ __forceinline__ void butterfly_ah(double (&ah)[10]) {
#pragma unroll
  for (int o = 1; o < L; o <<= 1)
#pragma unroll
    for (int k = 0; k < 10; ++k) ah[k] += __shfl_xor_sync(FULL, ah[k], o);
}

// rows 0,1 of G t (t with all three rows)
template <typename R>
__device__ __forceinline__ void apply_left(const mat3<R>& G, const mat3<R>& t, mat3<R>& n) {
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cx<R> x = cmul2(G.e[r][0], t.e[0][c], G.e[r][1], t.e[1][c]);
      n.e[r][c] = {x.re + G.e[r][2].re * t.e[2][c].re - G.e[r][2].im * t.e[2][c].im,
                   x.im + G.e[r][2].re * t.e[2][c].im + G.e[r][2].im * t.e[2][c].re};
    }
}
// rows 0,1 of t G^dag (t's rows 0,1 only)
template <typename R>
__device__ __forceinline__ void apply_right_dag(const mat3<R>& G, const mat3<R>& t, mat3<R>& n) {
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cx<R> x = cmul2c(t.e[r][0], G.e[c][0], t.e[r][1], G.e[c][1]);
      n.e[r][c] = {x.re + t.e[r][2].re * G.e[c][2].re + t.e[r][2].im * G.e[c][2].im,
                   x.im + t.e[r][2].im * G.e[c][2].re - t.e[r][2].re * G.e[c][2].im};
    }
}

// K (in FP64) += the slot's matrix from its stored rows (row 2 rebuilt in FP64).
template <typename R>
__device__ __forceinline__ void add_stored_k64(const mat3<R>& rows, bool down, mat3<double>& K) {
  mat3<double> d;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) d.e[a][b] = {(double)rows.e[a][b].re, (double)rows.e[a][b].im};
  reconstruct_row2(d);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      K.e[a][b].re += down ? d.e[b][a].re : d.e[a][b].re;
      K.e[a][b].im += down ? -d.e[b][a].im : d.e[a][b].im;
    }
}

template <typename R, int GAUGE, int ALGO, int LPT, bool OBS, bool MP>
__device__ __forceinline__ void sweep_site_k(const SweepArgs<R>& a, uint32_t copy, uint32_t sp, bool valid,
                                             int lane, const float4* stage, uint32_t sp0) {
  // S: the precision of Step 1 (the gathered K, the subgroup choices and G);
  // the MP variant of FP32 storage (Sec. 4.5) runs it in FP64, Step 2 in FP32
  using S = typename std::conditional<MP, double, R>::type;
  constexpr uint32_t TILE = BLOCK / (8 / LPT);
  constexpr int NC = store_traits<R>::NC;
  constexpr int L = 8 / LPT;
  // The links are held in registers between the gather and the update, except
  // for FP64 with eight links per lane and the fused-observables variants,
  // which read them again (from L2) instead of spilling
  constexpr bool KEEP = sizeof(R) == 4 ? !OBS : LPT <= 4;
  // FP64 links read again for the update keep the rebuilt third rows of the
  // up-links from the gather in shared memory (48 KB per block): Step 2 then
  // rebuilds none of them (the same values, 96 FP64 operations less per site)
  constexpr bool ROW2C = sizeof(R) == 8 && !KEEP && !MP && LPT == 8;
  const Geom& Gm = a.geom;
  const uint32_t Vh = Gm.Vh;
  int c[4] = {0, 0, 0, 0};
  uint32_t s = 0;
  if (valid) {
    site_coords(Gm, sp, a.parity, c, s);
    if (a.active && !a.active[(size_t)copy * Gm.n[0] + c[0]]) valid = false;
  }
  // rows re-projected at load: every FP32 kernel, and the FP64 kernels whose
  // rotations stay large (heat bath, microcanonical, SR); a read-only pass
  // leaves them as stored
  const bool NORM = (sizeof(R) == 4 || ALGO != ALG_OR) && (!OBS || a.update);

  size_t off[LPT];
  uint32_t idx[LPT];
  bool use[LPT], gather[LPT], dn[LPT];
#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    const int k = lane * LPT + j;
    const int mu = k >> 1;
    const bool down = (LPT >= 2) ? (j & 1) : (k & 1);
    dn[j] = down;
    gather[j] = !(GAUGE == COULOMB && mu == 0);
    use[j] = valid && !(GAUGE == COULOMB && mu == 0 && down);
    const int slot = (GAUGE == COULOMB && mu == 0) ? 4 : mu;
    uint32_t ssp = sp;
    int par = a.parity;
    if (down) {
      const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
      const int nm = mu == 0 ? Gm.n[0] : mu == 1 ? Gm.n[1] : mu == 2 ? Gm.n[2] : Gm.n[3];
      const uint32_t st = mu == 0 ? Gm.stride[0] : mu == 1 ? Gm.stride[1] : mu == 2 ? Gm.stride[2] : 1u;
      ssp = (cm > 0 ? s - st : s + (uint32_t)(nm - 1) * st) >> 1;
      par ^= 1;
    }
    idx[j] = ssp;
    off[j] = link_off(copy, par, slot, a.NS, NC, Vh, ssp);
  }

  // GF_MIXED: the site's accumulated transformation is needed only after Step
  // 1; lane 0 starts copying its three vectors into shared memory now
  // (cp.async, no registers held), so that the load overlaps the gather
  // (the launch gives the non-staged kernel 3 x TILE x 16 bytes of dynamic
  // shared memory for this when the accumulator is in use)
  constexpr bool ACC_ASYNC = sizeof(R) == 4 && GAUGE != COULOMB && !OBS;
  extern __shared__ __align__(128) unsigned char stage_smem[];
  float4* const acc_stage = reinterpret_cast<float4*>(stage_smem);
  const bool acc_async = ACC_ASYNC && a.acc && valid && lane == 0 && stage == nullptr;
  if (acc_async) {
    const float4* src = reinterpret_cast<const float4*>(a.links) + link_off(copy, a.parity, 4, a.NS, NC, Vh, sp);
    const uint32_t dst = smem_u32(&acc_stage[3 * (threadIdx.x / L)]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * k), "l"(src + (size_t)k * Vh)
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  }

  // gather: K = sum of U_mu(x) and U_mu(x - mu)^dag over the lane's slots
  __shared__ cx<R> row2c[ROW2C ? 12 * BLOCK : 1];
  cx<R>* const r2c = row2c + (ROW2C ? threadIdx.x : 0);  // this thread's column: [up-link][entry] stride BLOCK
  mat3<R> u[KEEP ? LPT : 1];
  mat3<S> K;
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) K.e[x][y] = {S(0), S(0)};
  constexpr bool OBS_FP64 = OBS && sizeof(R) == 4;  // FP32 kernels gather the FP64 sums separately
  double ah[10];
  if (OBS) {
#pragma unroll
    for (int k = 0; k < 10; ++k) ah[k] = 0.0;
  }
#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    mat3<R> t;
    if (use[j]) {
      load_slot<R, TILE>(stage, Gm, sp0, lane * LPT + j, idx[j], a.links + off[j], Vh, t);
      if (NORM) reproject_rows(t);
    } else {
      set_identity(t);
    }
    if (KEEP) u[KEEP ? j : 0] = t;
    if (use[j] && gather[j]) {
      if (OBS_FP64 && a.obs == 1) add_stored_ah(t, dn[j], ah);
      if constexpr (MP) {
        add_stored_k64(t, dn[j], K);
      } else {
        reconstruct_row2(t);
        if constexpr (ROW2C) {
          if (!dn[j]) {
#pragma unroll
            for (int y = 0; y < 3; ++y) r2c[((j >> 1) * 3 + y) * BLOCK] = t.e[2][y];
          }
        }
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
          for (int y = 0; y < 3; ++y) {
            const cx<R> v = dn[j] ? cx<R>{t.e[y][x].re, -t.e[y][x].im} : t.e[x][y];
            K.e[x][y].re += v.re;
            K.e[x][y].im += v.im;
          }
      }
    }
  }
#pragma unroll
  for (int o = 1; o < L; o <<= 1)
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int y = 0; y < 3; ++y) {
        K.e[x][y].re += __shfl_xor_sync(FULL, K.e[x][y].re, o);
        K.e[x][y].im += __shfl_xor_sync(FULL, K.e[x][y].im, o);
      }

  if (OBS && a.obs == 1) {  // theta of the current links at this site (K as gathered)
    if (OBS_FP64)
      butterfly_ah<L>(ah);
    else
      ah_of_k(K, ah);
    if (valid && lane == 0) a.obs_site[(size_t)copy * Gm.V + s] = make_double2(0.0, theta_of_ah(ah));
  }
  if (OBS && !a.update) return;

  // Step 1: the three subgroups in the order (0,1), (0,2), (1,2)
  Rng rng{a.k0, a.k1, s + a.site_offset, a.sweep, a.copy0 + copy};
  int* trace = (ALGO == ALG_SA && a.sa_trace && valid && lane == 0) ? a.sa_trace + ((size_t)copy * Gm.V + s) * 3
                                                                     : nullptr;
  const S prm = (S)a.param;
  const su2m<S> h0 = su2_of(choose_k<S, ALGO>(K.e[0][0], K.e[0][1], K.e[1][0], K.e[1][1], prm, rng, 0u, trace));
  {  // K <- g0 K on the entries read later: row 0, and row 1 columns 1, 2
    cx<S> r0[3];
#pragma unroll
    for (int y = 0; y < 3; ++y) r0[y] = cmul2(h0.h00, K.e[0][y], h0.h01, K.e[1][y]);
#pragma unroll
    for (int y = 1; y < 3; ++y) K.e[1][y] = cmul2(h0.h10, K.e[0][y], h0.h11, K.e[1][y]);
#pragma unroll
    for (int y = 0; y < 3; ++y) K.e[0][y] = r0[y];
  }
  const su2m<S> h1 = su2_of(choose_k<S, ALGO>(K.e[0][0], K.e[0][2], K.e[2][0], K.e[2][2], prm, rng, 1u, trace));
#pragma unroll
  for (int y = 1; y < 3; ++y) K.e[2][y] = cmul2(h1.h10, K.e[0][y], h1.h11, K.e[2][y]);  // row 2 of g1 K
  const su2m<S> h2 = su2_of(choose_k<S, ALGO>(K.e[1][1], K.e[1][2], K.e[2][1], K.e[2][2], prm, rng, 2u, trace));

  // G = g2 g1 g0 in the 3x3 embedding
  mat3<S> Gs;
  {
    mat3<S>& G = Gs;
    // g1 g0: rows 0 and 2 mixed, row 1 = row 1 of g0
    const cx<S> r00 = cmul(h1.h00, h0.h00), r01 = cmul(h1.h00, h0.h01);
    const cx<S> r20 = cmul(h1.h10, h0.h00), r21 = cmul(h1.h10, h0.h01);
    G.e[0][0] = r00;
    G.e[0][1] = r01;
    G.e[0][2] = h1.h01;
    // g2 on rows 1 = (h0.h10, h0.h11, 0) and 2 = (r20, r21, h1.h11)
    G.e[1][0] = cmul2(h2.h00, h0.h10, h2.h01, r20);
    G.e[1][1] = cmul2(h2.h00, h0.h11, h2.h01, r21);
    G.e[1][2] = cmul(h2.h01, h1.h11);
    G.e[2][0] = cmul2(h2.h10, h0.h10, h2.h11, r20);
    G.e[2][1] = cmul2(h2.h10, h0.h11, h2.h11, r21);
    G.e[2][2] = cmul(h2.h11, h1.h11);
  }
  // Step 2 runs in the storage precision
  mat3<R> G;
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) G.e[x][y] = {(R)Gs.e[x][y].re, (R)Gs.e[x][y].im};

  // mixed precision: the site's accumulated gauge transformation (FP32 working copy only)
  constexpr bool CAN_ACC = sizeof(R) == 4 && GAUGE != COULOMB;
  if (CAN_ACC && a.acc && valid && lane == 0) {
    const size_t acc_off = link_off(copy, a.parity, 4, a.NS, NC, Vh, sp);
    mat3<R> t, n;
    if (acc_async) {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      const float4* q = &acc_stage[3 * (threadIdx.x / L)];
      const float4 x = q[0], y = q[1], z = q[2];
      t.e[0][0] = {(R)x.x, (R)x.y};
      t.e[0][1] = {(R)x.z, (R)x.w};
      t.e[0][2] = {(R)y.x, (R)y.y};
      t.e[1][0] = {(R)y.z, (R)y.w};
      t.e[1][1] = {(R)z.x, (R)z.y};
      t.e[1][2] = {(R)z.z, (R)z.w};
    } else {
      load_slot<R, TILE>(stage, Gm, sp0, 8, sp, a.links + acc_off, Vh, t);
    }
    reproject_rows(t);
    reconstruct_row2(t);
    apply_left(G, t, n);
    store_rows(a.links + acc_off, Vh, n);
  }

  // Step 2: apply G to the slots; fused F and theta of the written links
  if (OBS && a.obs == 2) {
#pragma unroll
    for (int k = 0; k < 10; ++k) ah[k] = 0.0;
  }
#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    if (!use[j]) continue;
    mat3<R> t, n;
    if (KEEP) {
      t = u[KEEP ? j : 0];
    } else {
      load_slot<R, TILE>(stage, Gm, sp0, lane * LPT + j, idx[j], a.links + off[j], Vh, t);
      if (NORM) reproject_rows(t);
    }
    if (dn[j]) {
      apply_right_dag(G, t, n);
    } else {
      if (ROW2C && gather[j]) {
#pragma unroll
        for (int y = 0; y < 3; ++y) t.e[2][y] = r2c[((j >> 1) * 3 + y) * BLOCK];
      } else {
        reconstruct_row2(t);
      }
      apply_left(G, t, n);
    }
    store_rows(a.links + off[j], Vh, n);
    if (OBS && a.obs == 2 && gather[j]) add_stored_ah(n, dn[j], ah);
  }
  if (OBS && a.obs == 2) {
    butterfly_ah<L>(ah);
    if (valid && lane == 0) a.obs_site[(size_t)copy * Gm.V + s] = make_double2(ah[9], theta_of_ah(ah));
  }
}

// Resident blocks per SM requested from the register allocator (blocks of
// 256 threads; 1 / 2 / 3 / 4 blocks allow 255 / 128 / 80 / 64 registers):
// FP32 1 / 2 / 3 / 4 blocks for 8 / 4 / 2 / 1 links per lane.  FP64 in K form
// 2 / 1 / 1 / 2 (eight links per lane read the links again for the update);
// the per-slot MAG form 1 / 1 / 1 / 2 (FP64 MAG runs eight links per lane as
// four: eight full FP64 matrices per lane do not fit in registers).  (Reading
// the links again in FP32 as well, to fit one more block, measured slower:
// 0.347 against 0.324 ms per 32^3 x 64 sweep.)
template <typename R, int GAUGE, int LPT, bool MP = false>
constexpr int min_blocks() {
  if (MP) return LPT == 8 ? 1 : LPT == 4 ? 1 : LPT == 2 ? 2 : 3;  // FP64 K and G in registers
  if (sizeof(R) == 4) return LPT == 8 ? 1 : LPT == 4 ? 2 : LPT == 2 ? 3 : 4;
  return GAUGE == MAG ? (LPT >= 2 ? 1 : 2) : (LPT == 8 ? 2 : LPT >= 2 ? 1 : 2);
}

template <typename R, int GAUGE, int ALGO, int LPT, bool OBS, bool MP>
__device__ __forceinline__ void site_dispatch(const SweepArgs<R>& a, uint32_t copy, uint32_t sp, bool valid, int lane,
                                              const float4* stage, uint32_t sp0) {
  if constexpr (GAUGE == MAG)
    sweep_site_mag<R, ALGO, LPT, OBS, MP>(a, copy, sp, valid, lane, stage, sp0);
  else
    sweep_site_k<R, GAUGE, ALGO, LPT, OBS, MP>(a, copy, sp, valid, lane, stage, sp0);
}

// Persistent loop with two stage buffers (FP32, prefetch mode 2).  Warp 0
// issues tile i+1's copies before the block waits for tile i's; the
// __syncthreads at the end of an iteration frees the buffer that the next
// iteration refills.  If a wait runs out, the block records the error, waits
// (bounded) for the copies it issued and returns.
template <int GAUGE, int ALGO, int LPT, bool OBS, bool MP>
__device__ __forceinline__ void sweep_staged(const SweepArgs<float>& a) {
  constexpr int L = 8 / LPT;
  constexpr uint32_t TILE = BLOCK / L;
  using SG = StageGeom<TILE>;
  extern __shared__ __align__(128) unsigned char stage_smem[];
  float4* buf[2] = {reinterpret_cast<float4*>(stage_smem), reinterpret_cast<float4*>(stage_smem) + SG::VEC};
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<float4*>(stage_smem) + 2 * SG::VEC);
  const uint32_t bar[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};
  const uint32_t Vh = a.geom.Vh;
  const uint32_t tiles_per_copy = (Vh + TILE - 1) / TILE;
  const uint64_t ntiles = (uint64_t)tiles_per_copy * a.ncopies;
  const int lane = (int)(threadIdx.x % L);
  const uint32_t local = threadIdx.x / L;
  const int warp = (int)(threadIdx.x >> 5), lane32 = (int)(threadIdx.x & 31);
  if (threadIdx.x == 0) {
    mbar_init(bar[0], 1);
    mbar_init(bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](uint64_t t, int b) {
    const uint32_t c = (uint32_t)(t / tiles_per_copy);
    const uint32_t sp0 = (uint32_t)(t - (uint64_t)c * tiles_per_copy) * TILE;
    stage_issue<GAUGE, TILE>(a, c, sp0, buf[b], bar[b], lane32);
  };
  uint32_t phase[2] = {0u, 0u};
  bool pending[2] = {false, false};
  uint64_t tile = blockIdx.x;
  if (tile < ntiles) {
    if (warp == 0) issue(tile, 0);
    pending[0] = true;
  }
  for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    const uint64_t next = tile + gridDim.x;
    if (next < ntiles) {
      if (warp == 0) issue(next, b ^ 1);
      pending[b ^ 1] = true;
    }
    const bool ok = mbar_wait_bounded(bar[b], phase[b], a.wait_polls < 0 ? WAIT_POLLS : (uint32_t)a.wait_polls);
    if (__syncthreads_or(!ok)) {
      // the copies issued for this tile and the next are waited for with the
      // full bound before the block leaves (none may land after it exits)
      if (threadIdx.x == 0) {
        if (a.err) atomicExch(a.err, 1);
        for (int q = 0; q < 2; ++q)
          if (pending[q]) mbar_wait_bounded(bar[q], phase[q]);
      }
      __syncthreads();
      return;
    }
    phase[b] ^= 1u;
    pending[b] = false;
    const uint32_t copy = (uint32_t)(tile / tiles_per_copy);
    const uint32_t sp0 = (uint32_t)(tile - (uint64_t)copy * tiles_per_copy) * TILE;
    const uint32_t sp = sp0 + local;
    site_dispatch<float, GAUGE, ALGO, LPT, OBS, MP>(a, copy, sp, sp < Vh, lane, buf[b], sp0);
    __syncthreads();
  }
}

// OBS: the variant with the fused observables (used for overrelaxation check
// sweeps only, so that the plain kernels keep their register budget).  MP:
// FP32 storage with Step 1 in FP64 (the paper's mixed-precision variant).
template <typename R, int GAUGE, int ALGO, int LPT, bool OBS, bool MP = false>
__global__ void __launch_bounds__(BLOCK, min_blocks<R, GAUGE, LPT, MP>()) sweep_kernel(const SweepArgs<R> a) {
  if constexpr (sizeof(R) == 4) {
    if (a.prefetch == 2) {
      sweep_staged<GAUGE, ALGO, LPT, OBS, MP>(a);
      return;
    }
  }
  constexpr int NC = store_traits<R>::NC;
  constexpr int L = 8 / LPT;
  constexpr uint32_t TILE = BLOCK / L;
  const uint32_t Vh = a.geom.Vh;
  const uint32_t tiles_per_copy = (Vh + TILE - 1) / TILE;
  const uint64_t ntiles = (uint64_t)tiles_per_copy * a.ncopies;
  const int lane = (int)(threadIdx.x % L);
  const uint32_t local = threadIdx.x / L;
  if constexpr (sizeof(R) == 8) {
    // FP64 is ALU-bound: every block takes an equal contiguous range of the
    // (copy, site) indices in tiles of TILE, so that no SM finishes a whole
    // tile before the others (whole tiles dealt round-robin left a 4 % tail).
    // The indices run over the launch's sites [sp_lo, sp_lo + sp_n) of each
    // copy, so that a part of the lattice (a time slab's boundary slice) is
    // spread over every block too.
    const uint32_t span = a.sp_n;
    const uint64_t total = (uint64_t)span * a.ncopies;
    const uint64_t lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
    // (copy, offset in the range) of the tile's first index, advanced by TILE
    // per iteration
    uint32_t c0 = span ? (uint32_t)(lo / span) : 0u;
    uint32_t s0 = (uint32_t)(lo - (uint64_t)c0 * span);
    for (uint64_t base = lo; base < hi; base += TILE) {
      if (a.prefetch && base + TILE < hi && threadIdx.x < 9 * NC) {
        uint32_t nc = c0, ns = s0 + TILE;
        while (ns >= span) ns -= span, ++nc;
        const uint32_t n = (uint32_t)min((uint64_t)min(TILE, span - ns), hi - base - TILE);
        prefetch_tile<R, GAUGE>(a, nc, a.sp_lo + ns, n, (int)threadIdx.x);
      }
      uint32_t copy = c0, sp = s0 + local;
      while (sp >= span) sp -= span, ++copy;
      sp += a.sp_lo;
      site_dispatch<R, GAUGE, ALGO, LPT, OBS, MP>(a, copy, sp, base + local < hi, lane, nullptr, sp);
      s0 += TILE;
      while (s0 >= span) s0 -= span, ++c0;
    }
  } else {
    // FP32 is HBM-bound: whole tiles dealt round-robin keep the blocks' reads
    // within one window of the arrays at a time
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const uint64_t next = tile + gridDim.x;
      if (a.prefetch && next < ntiles && threadIdx.x < 9 * NC) {
        const uint32_t nc = (uint32_t)(next / tiles_per_copy);
        const uint32_t nsp0 = (uint32_t)(next - (uint64_t)nc * tiles_per_copy) * TILE;
        prefetch_tile<R, GAUGE>(a, nc, nsp0, min(TILE, Vh - nsp0), (int)threadIdx.x);
      }
      const uint32_t copy = (uint32_t)(tile / tiles_per_copy);
      const uint32_t sp0 = (uint32_t)(tile - (uint64_t)copy * tiles_per_copy) * TILE;
      site_dispatch<R, GAUGE, ALGO, LPT, OBS, MP>(a, copy, sp0 + local, sp0 + local < Vh, lane, nullptr, sp0);
    }
  }
}

// ---------------------------------------------------------------------------
// Several lattices of different extents (the same gauge and storage) in one
// persistent launch: the tiles of every member are numbered one after the
// other and a block finds the member of a tile by binary search of the
// members' cumulative tile counts.  The members' arguments travel in the
// kernel's parameter space (__grid_constant__, read in place).
constexpr int GROUP_MAX = 48;

template <typename R>
struct GroupArgs {
  SweepArgs<R> m[GROUP_MAX];
  uint64_t tile_end[GROUP_MAX];  // tiles of members 0..k
  uint32_t n;
  uint64_t ntiles;
};

template <typename R>
__device__ __forceinline__ uint32_t group_member(const GroupArgs<R>& g, uint64_t tile) {
  uint32_t lo = 0, hi = g.n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (tile < g.tile_end[mid]) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <typename R, int GAUGE, int ALGO, int LPT>
__global__ void __launch_bounds__(BLOCK, min_blocks<R, GAUGE, LPT>())
    sweep_group_kernel(const __grid_constant__ GroupArgs<R> g) {
  constexpr int NC = store_traits<R>::NC;
  constexpr int L = 8 / LPT;
  constexpr uint32_t TILE = BLOCK / L;
  const int lane = (int)(threadIdx.x % L);
  const uint32_t local = threadIdx.x / L;
  for (uint64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    const uint32_t m = group_member(g, tile);
    const uint64_t next = tile + gridDim.x;
    if (next < g.ntiles && threadIdx.x < 9 * NC) {  // the next tile into L2, as the single-lattice kernel
      const uint32_t mn = group_member(g, next);
      const SweepArgs<R>& an = g.m[mn];
      if (an.prefetch) {
        const uint64_t tn = next - (mn ? g.tile_end[mn - 1] : 0);
        const uint32_t tpc = (an.geom.Vh + TILE - 1) / TILE;
        const uint32_t cn = (uint32_t)(tn / tpc);
        const uint32_t sn = (uint32_t)(tn - (uint64_t)cn * tpc) * TILE;
        prefetch_tile<R, GAUGE>(an, cn, sn, min(TILE, an.geom.Vh - sn), (int)threadIdx.x);
      }
    }
    // the member's arguments by value: the site's loads and stores cannot
    // alias a private copy, so its fields stay in registers across them
    const SweepArgs<R> a = g.m[m];
    const uint64_t t = tile - (m ? g.tile_end[m - 1] : 0);
    const uint32_t Vh = a.geom.Vh;
    const uint32_t tiles_per_copy = (Vh + TILE - 1) / TILE;
    const uint32_t copy = (uint32_t)(t / tiles_per_copy);
    const uint32_t sp0 = (uint32_t)(t - (uint64_t)copy * tiles_per_copy) * TILE;
    site_dispatch<R, GAUGE, ALGO, LPT, false, false>(a, copy, sp0 + local, sp0 + local < Vh, lane, nullptr, sp0);
  }
}

}  // namespace gfk
