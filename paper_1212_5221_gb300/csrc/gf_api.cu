// gf_api.cu -- the C ABI of libgf (declared in include/gf.h): context and
// device-memory management, host<->device layout conversion, the sweep
// sequencing of Alg. 1 and the convergence driver.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gf.h"
#include "gf_sweep.cuh"
#include "gf_launch.h"

using gfk::Geom;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define GF_CUDA(expr)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(GF_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

constexpr size_t ALIGN = 256;
constexpr size_t STAGING_BYTES = (size_t)256 << 20;

size_t round_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// NVTX range around a host phase (shown by Nsight tools; no cost without one)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Launch parameters chosen by gf_autotune, kept for the process per
// (device, gauge, storage is FP64, algorithm, floor(log2(sites x copies))).
struct Tuned {
  int lpt, pmode;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, Tuned> g_tuned;

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  return dev;
}

int volume_class(uint64_t v) {
  int k = 0;
  while (v > 1) {
    v >>= 1;
    ++k;
  }
  return k;
}

struct Layout {
  size_t links32 = 0, links64 = 0, gscratch = 0, obs_site = 0, active = 0, slab = 0, partial = 0, obs = 0,
         err = 0, staging = 0, total = 0;
  int slab_nt = 1;
};

int check_dims(const int dims[4], int ncopies, int gauge, int prec) {
  if (!dims) return fail(GF_EINVAL, "dims is NULL");
  uint64_t V = 1;
  for (int d = 0; d < 4; ++d) {
    if (dims[d] < 2 || (dims[d] & 1))
      return fail(GF_EINVAL, "extent %d of dims is %d: every extent must be even and >= 2", d, dims[d]);
    V *= (uint64_t)dims[d];
  }
  if (V >= (1ull << 31)) return fail(GF_EINVAL, "lattice volume %llu too large (< 2^31)", (unsigned long long)V);
  if (ncopies < 1) return fail(GF_EINVAL, "n_copies must be >= 1");
  if ((uint64_t)ncopies * dims[0] * 2 > 65535) return fail(GF_EINVAL, "n_copies * Nt * 2 must be <= 65535");
  if ((uint64_t)ncopies * V >= (1ull << 40)) return fail(GF_EINVAL, "batch too large");
  if (gauge < GF_LANDAU || gauge > GF_MAG) return fail(GF_EINVAL, "bad gauge %d", gauge);
  if (prec < GF_FP64 || prec > GF_MP) return fail(GF_EINVAL, "bad precision %d", prec);
  return GF_OK;
}

Geom make_geom(const int dims[4]) {
  Geom G;
  for (int d = 0; d < 4; ++d) G.n[d] = dims[d];
  G.V3 = (uint32_t)dims[1] * dims[2] * dims[3];
  G.V = G.V3 * (uint32_t)dims[0];
  G.Vh = G.V / 2;
  G.stride[0] = G.V3;
  G.stride[1] = (uint32_t)dims[2] * dims[3];
  G.stride[2] = (uint32_t)dims[3];
  G.stride[3] = 1;
  G.dz = gfk::make_fastdiv((uint32_t)dims[3]);
  G.dy = gfk::make_fastdiv((uint32_t)dims[2]);
  G.dx = gfk::make_fastdiv((uint32_t)dims[1]);
  return G;
}

Layout make_layout(const int dims[4], int ncopies, int gauge, int prec) {
  Geom G = make_geom(dims);
  Layout L;
  // slot 4: Coulomb's accumulated time-slice transformation, and in GF_MIXED the
  // FP32 sweeps' accumulated transformation awaiting the FP64 master
  const int NS32 = (gauge == GF_COULOMB || prec == GF_MIXED) ? 5 : 4;
  const int NS64 = gauge == GF_COULOMB ? 5 : 4;
  if (prec != GF_FP64) L.links32 = round_up((size_t)ncopies * 2 * NS32 * G.Vh * 3 * sizeof(float4));
  if (prec == GF_FP64 || prec == GF_MIXED)
    L.links64 = round_up((size_t)ncopies * 2 * NS64 * G.Vh * 6 * sizeof(double2));
  // GF_MIXED: the re-unitarised FP64 accumulator, full 3x3, used by the master sync
  if (prec == GF_MIXED) L.gscratch = round_up((size_t)ncopies * 2 * G.Vh * 9 * sizeof(double2));
  L.obs_site = round_up((size_t)ncopies * G.V * sizeof(double2));  // fused per-site F/theta
  L.active = round_up((size_t)ncopies * dims[0] * sizeof(int));
  L.slab = round_up((size_t)3 * dims[0] * sizeof(int));  // time-slab slice masks (all / boundary / inner)
  L.partial = round_up(gfk::observables_partial_doubles(G, ncopies) * sizeof(double));
  L.obs = round_up((size_t)ncopies * dims[0] * 2 * sizeof(double));
  L.err = ALIGN;  // the sweep kernels' error word
  const size_t slice_bytes = (size_t)G.V3 * 4 * 18 * sizeof(double);
  L.slab_nt = (int)std::max<size_t>(1, std::min<size_t>(dims[0], STAGING_BYTES / slice_bytes));
  L.staging = round_up((size_t)L.slab_nt * slice_bytes);
  L.total = L.links32 + L.links64 + L.gscratch + L.obs_site + L.active + L.slab + L.partial + L.obs + L.err +
            L.staging;
  return L;
}

}  // namespace

void gfk::set_last_error(const char* msg) { g_last_error = msg; }

struct gf_ctx {
  int dims[4];
  int ncopies, gauge, prec;
  int device = 0;  // the CUDA device current when the context was created
  int NS32, NS64;  // slots per site in the FP32 / FP64 arrays
  Geom G;
  Layout layout;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  void* owned = nullptr;  // device block allocated by the context (nullptr for gf_create_ext)
  void* links32 = nullptr;
  void* links64 = nullptr;
  void* gscratch = nullptr;
  void* obs_site = nullptr;
  int* active_d = nullptr;
  double* partial = nullptr;
  double* obs_d = nullptr;
  int* err_d = nullptr;      // set by a sweep kernel whose staging wait ran out
  bool err_pending = false;  // a staged sweep ran since err_d was last read
  double* staging = nullptr;
  bool fp64 = false;   // storage the sweeps run on
  bool dirty = false;  // GF_MIXED: FP32 sweeps not yet applied to the FP64 master
  bool all_active = true;
  std::vector<int> active_h;
  uint64_t sweep_index = 0;
  uint32_t copy_base = 0;  // Philox copy id of copy 0
  int prefetch = GF_PREFETCH_L2;  // how the sweep kernels fetch the next tile
  int stage_wait_polls = -1;      // polls of a staging wait (< 0: the kernel's default)
  int fused_obs = 1;       // F/theta fused into the last OR sweep where possible
  int sa_micro = 3;        // microcanonical sweeps after each heat-bath sweep (Sec. 2.3)
  int* sa_trace_d = nullptr;  // caller's device buffer for heat-bath trial counts, or nullptr
  // time-slab mode (Sec. 5): local slice 0 is a halo copy of global slice t0-1,
  // slices 1..Nt-2 are owned (global t0 ..), slice Nt-1 an unused pad
  bool slab = false;
  int slab_t0 = 0, slab_Nt = 0;
  int parity_flip = 0;        // local parity = global parity ^ parity_flip
  uint32_t site_offset = 0;   // global site index = local index + site_offset (Philox counters)
  int* slab_flags_d = nullptr;  // 3 x Nt flags: owned, boundary (first/last owned), inner
  int lpt[2][5] = {{0}};  // [fp64][algo] chosen links per thread, 0 = default
  int pmode[2][5] = {{0}};  // [fp64][algo] tile fetch chosen by gf_autotune + 1, 0 = the context's
  // optional per-kernel timing: CUDA events around every launch of a class
  uint64_t launch_count = 0;  // every kernel this context launched
  bool profiling = false;
  struct Pending {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  uint64_t prof_launches[GF_KERNEL_KINDS] = {0};
  double prof_ms[GF_KERNEL_KINDS] = {0};
  // CUDA graphs of blocks of plain overrelaxation sweeps, keyed by everything
  // their launch arguments depend on
  bool use_graphs = true;
  bool warm = false;  // sweep kernels launched once outside capture (one-time setup done)
  using GraphKey = std::tuple<int, int, int, int, int, int, uint64_t, uint32_t, int>;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  FILE* check_log = nullptr;  // JSON lines, one per convergence check

  void* links() const { return fp64 ? links64 : links32; }
  int NS() const { return fp64 ? NS64 : NS32; }
  // the array that holds the authoritative links: the FP64 master in GF_MIXED
  bool master64() const { return prec == GF_MIXED || fp64; }
  size_t copy_block_bytes(bool f64) const { return (size_t)2 * (f64 ? NS64 : NS32) * G.Vh * (f64 ? 6 : 3) * 16; }
  size_t copy_block_bytes() const { return copy_block_bytes(fp64); }
};

namespace {

cudaEvent_t take_event(gf_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Start / end a timed launch of the given kind (no-ops unless profiling).
cudaEvent_t prof_begin(gf_ctx* c) {
  if (!c->profiling) return nullptr;
  cudaEvent_t e = take_event(c);
  cudaEventRecord(e, c->st);
  return e;
}

void prof_end(gf_ctx* c, cudaEvent_t start, int kind) {
  if (!c->profiling || !start) return;
  cudaEvent_t e = take_event(c);
  cudaEventRecord(e, c->st);
  c->pending.push_back({start, e, kind});
}

// Fold completed event pairs into the per-kind totals (call after a sync).
void prof_collect(gf_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof_ms[p.kind] += ms;
      c->prof_launches[p.kind]++;
    }
    c->event_pool.push_back(p.a);
    c->event_pool.push_back(p.b);
  }
  c->pending.clear();
  cudaGetLastError();
}

int default_lpt(const gf_ctx* c, int algo) {
  int v = c->lpt[c->fp64][algo];
  if (v) return v;
  // fastest on GB300 for the 32^3 x 64 Landau sweep: FP64 (and GF_MP, whose
  // Step 1 is FP64) with one lane per site, so that no lane repeats Step 1;
  // FP32 with two lanes per site
  return (c->fp64 || c->prec == GF_MP) ? 8 : 4;
}

// The kernel arguments of one half-sweep of context c.
template <typename R>
void fill_args(gfk::SweepArgs<R>& a, gf_ctx* c, int kalgo, double param, int parity, uint64_t seed, uint32_t sweep,
               int obs, int update, int prefetch, const int* active_override) {
  a.links = static_cast<typename gfk::store_traits<R>::vec*>(sizeof(R) == 8 ? c->links64 : c->links32);
  a.geom = c->G;
  a.NS = c->NS();
  a.parity = parity;
  a.ncopies = (uint32_t)c->ncopies;
  a.copy0 = c->copy_base;
  a.active = active_override ? active_override : (c->all_active ? nullptr : c->active_d);
  a.param = (R)param;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.sweep = sweep;
  a.prefetch = prefetch;
  a.acc = (update && c->prec == GF_MIXED && !c->fp64 && c->gauge != GF_COULOMB) ? 1 : 0;
  a.obs = obs;
  a.update = update;
  a.obs_site = static_cast<double2*>(c->obs_site);
  a.err = c->err_d;
  a.wait_polls = sizeof(R) == 8 ? -1 : c->stage_wait_polls;
  a.sa_trace = kalgo == gfk::ALG_SA ? c->sa_trace_d : nullptr;
  a.site_offset = c->site_offset;
  a.sp_lo = 0;
  a.sp_n = c->G.Vh;
}

// sp_lo, sp_n: the sites of each copy an FP64 launch covers (all by default).
int launch_half(gf_ctx* c, int kalgo, double param, int parity, uint64_t seed, uint32_t sweep, int lpt,
                int obs = 0, int update = 1, int pmode = -1, const int* active_override = nullptr,
                uint32_t sp_lo = 0, uint32_t sp_n = UINT32_MAX) {
  const int prefetch = pmode >= 0 ? pmode : c->prefetch;
  cudaError_t e;
  if (c->fp64) {
    gfk::SweepArgs<double> a;
    fill_args(a, c, kalgo, param, parity, seed, sweep, obs, update, prefetch, active_override);
    if (sp_n != UINT32_MAX) {
      a.sp_lo = sp_lo;
      a.sp_n = sp_n;
    }
    cudaEvent_t t0 = prof_begin(c);
    e = gfk::launch_sweep<double>(a, c->gauge, kalgo, lpt, c->st);
    prof_end(c, t0, GF_KERNEL_SWEEP_FP64);
    c->launch_count++;
  } else {
    gfk::SweepArgs<float> a;
    fill_args(a, c, kalgo, param, parity, seed, sweep, obs, update, prefetch, active_override);
    if (a.prefetch == GF_PREFETCH_SMEM) c->err_pending = true;
    cudaEvent_t t0 = prof_begin(c);
    e = c->prec == GF_MP ? gfk::launch_sweep_mp(a, c->gauge, kalgo, lpt, c->st)
                         : gfk::launch_sweep<float>(a, c->gauge, kalgo, lpt, c->st);
    prof_end(c, t0, GF_KERNEL_SWEEP_FP32);
    c->launch_count++;
  }
  if (e != cudaSuccess) return fail(GF_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
  return GF_OK;
}

// One full sweep (even, then odd sublattice) of kernel algorithm kalgo; with
// obs_last the odd half also writes F and theta of its sites (fused check).
int full_sweep(gf_ctx* c, int kalgo, int api_algo, double param, uint64_t seed, int lpt_override = 0,
               bool obs_last = false, int pmode_override = -1) {
  const int lpt = lpt_override ? lpt_override : default_lpt(c, api_algo);
  const int pm = pmode_override >= 0 ? pmode_override : c->pmode[c->fp64][api_algo] - 1;
  const uint32_t sw = (uint32_t)c->sweep_index;
  for (int p = 0; p < 2; ++p) {
    int r = launch_half(c, kalgo, param, p, seed, sw, lpt, (obs_last && p == 1) ? 2 : 0, 1, pm);
    if (r) return r;
  }
  if (c->prec == GF_MIXED && !c->fp64) c->dirty = true;
  c->sweep_index++;
  return GF_OK;
}

// A staged sweep whose shared-memory wait ran out records it in err_d; it is
// read at the next point where the host waits for the stream anyway.
int read_sweep_error(gf_ctx* c) {
  if (!c->err_pending) return GF_OK;
  int h = 0;
  GF_CUDA(cudaMemcpyAsync(&h, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  GF_CUDA(cudaStreamSynchronize(c->st));
  c->err_pending = false;
  if (h) {
    GF_CUDA(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st));
    return fail(GF_ETIMEOUT, "a shared-memory staging wait in the sweep kernel ran out");
  }
  return GF_OK;
}

// n plain sweeps of overrelaxation / relaxation (no observables).  These
// draw no random numbers, so every block of GRAPH_SWEEPS sweeps launches the
// same kernels with the same arguments: it is captured once as a CUDA graph
// and replayed, which removes the per-launch host overhead that bounds small
// lattices.  The remainder, the first block ever (one-time kernel setup) and
// profiled runs launch directly.
constexpr int GRAPH_SWEEPS = 16;

int plain_sweeps(gf_ctx* c, int kalgo, int api_algo, double param, int n) {
  while (n >= GRAPH_SWEEPS && c->use_graphs && c->warm && !c->profiling) {
    const int lpt = default_lpt(c, api_algo);
    const int pm = c->pmode[c->fp64][api_algo] - 1;
    const bool acc = c->prec == GF_MIXED && !c->fp64 && c->gauge != GF_COULOMB;
    uint64_t pbits;
    memcpy(&pbits, &param, sizeof pbits);
    const int mode = pm >= 0 ? pm : c->prefetch;
    const gf_ctx::GraphKey key{c->fp64, lpt, mode, kalgo, c->all_active, acc, pbits, c->copy_base,
                               c->stage_wait_polls};
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
      const uint64_t idx = c->sweep_index, nl = c->launch_count;
      if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      int r = GF_OK;
      for (int k = 0; k < GRAPH_SWEEPS && !r; ++k) r = full_sweep(c, kalgo, api_algo, param, 0);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->st, &g);
      c->sweep_index = idx;
      c->launch_count = nl;
      cudaGraphExec_t x = nullptr;
      if (r || e != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->use_graphs = false;  // launch directly from now on
        if (r) return r;
        break;
      }
      cudaGraphDestroy(g);
      it = c->graphs.emplace(key, x).first;
    }
    GF_CUDA(cudaGraphLaunch(it->second, c->st));
    // a replayed staged sweep can record a staging timeout like a direct launch
    if (!c->fp64 && mode == GF_PREFETCH_SMEM) c->err_pending = true;
    c->sweep_index += GRAPH_SWEEPS;
    c->launch_count += 2 * GRAPH_SWEEPS;
    if (c->prec == GF_MIXED && !c->fp64) c->dirty = true;
    n -= GRAPH_SWEEPS;
  }
  for (int k = 0; k < n; ++k) {
    int r = full_sweep(c, kalgo, api_algo, param, 0);
    if (r) return r;
  }
  if (n > 0) c->warm = true;
  return GF_OK;
}

int observables_on(gf_ctx* c, std::vector<double>& per_ct, bool f64) {
  cudaEvent_t t0 = prof_begin(c);
  cudaError_t e = f64 ? gfk::launch_observables<double>(c->links64, c->G, c->NS64, c->gauge, c->ncopies,
                                                         c->partial, c->obs_d, c->st)
                      : gfk::launch_observables<float>(c->links32, c->G, c->NS32, c->gauge, c->ncopies,
                                                        c->partial, c->obs_d, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "observables launch: %s", cudaGetErrorString(e));
  prof_end(c, t0, GF_KERNEL_OBSERVABLES);
  c->launch_count += 2;
  per_ct.resize((size_t)c->ncopies * c->dims[0] * 2);
  GF_CUDA(cudaMemcpyAsync(per_ct.data(), c->obs_d, per_ct.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          c->st));
  GF_CUDA(cudaStreamSynchronize(c->st));
  prof_collect(c);
  return read_sweep_error(c);
}

// observables of the storage the sweeps run on
int observables(gf_ctx* c, std::vector<double>& per_ct) { return observables_on(c, per_ct, c->fp64); }

// Observables from the fused sweeps: the odd half of the last sweep wrote F
// and theta of the odd sites; a read-only pass of the sweep kernel gathers K
// at the even sites; both are summed per (copy, slice).
int fused_observables(gf_ctx* c, std::vector<double>& per_ct) {
  cudaEvent_t t0 = prof_begin(c);
  int r = launch_half(c, gfk::ALG_OR, 1.0, 0, 0, 0, default_lpt(c, GF_OR), 1, 0);
  if (r) return r;
  cudaError_t e = gfk::launch_obs_site_reduce(c->obs_site, c->G, c->gauge, c->ncopies, c->partial, c->obs_d, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "fused observables: %s", cudaGetErrorString(e));
  prof_end(c, t0, GF_KERNEL_OBSERVABLES);
  c->launch_count += 2;
  per_ct.resize((size_t)c->ncopies * c->dims[0] * 2);
  GF_CUDA(cudaMemcpyAsync(per_ct.data(), c->obs_d, per_ct.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          c->st));
  GF_CUDA(cudaStreamSynchronize(c->st));
  prof_collect(c);
  return read_sweep_error(c);
}

void copy_means(const gf_ctx* c, const std::vector<double>& ct, double* F, double* T) {
  const int Nt = c->dims[0];
  for (int k = 0; k < c->ncopies; ++k) {
    double f = 0, t = 0;
    for (int s = 0; s < Nt; ++s) {
      f += ct[2 * ((size_t)k * Nt + s)];
      t += ct[2 * ((size_t)k * Nt + s) + 1];
    }
    if (F) F[k] = f / Nt;
    if (T) T[k] = t / Nt;
  }
}

int upload_active(gf_ctx* c) {
  c->all_active = std::all_of(c->active_h.begin(), c->active_h.end(), [](int v) { return v != 0; });
  GF_CUDA(cudaMemcpyAsync(c->active_d, c->active_h.data(), c->active_h.size() * sizeof(int),
                          cudaMemcpyHostToDevice, c->st));
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int coulomb_fold(gf_ctx* c, bool f64) {
  if (c->gauge != GF_COULOMB) return GF_OK;
  cudaError_t e = f64 ? gfk::launch_coulomb_fold<double>(c->links64, c->G, c->ncopies, c->st)
                      : gfk::launch_coulomb_fold<float>(c->links32, c->G, c->ncopies, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "coulomb fold: %s", cudaGetErrorString(e));
  c->launch_count += 2;
  return GF_OK;
}

// Identity in slots [first, last] of every array the context holds.
int set_identity_slots(gf_ctx* c, int first, int last) {
  for (int f64 = 0; f64 < 2; ++f64) {
    void* l = f64 ? c->links64 : c->links32;
    const int ns = f64 ? c->NS64 : c->NS32;
    if (!l) continue;
    for (int s = first; s <= last && s < ns; ++s) {
      cudaError_t e = f64 ? gfk::launch_identity_slot<double>(l, c->G, ns, s, c->ncopies, c->st)
                          : gfk::launch_identity_slot<float>(l, c->G, ns, s, c->ncopies, c->st);
      if (e != cudaSuccess) return fail(GF_ECUDA, "identity: %s", cudaGetErrorString(e));
      c->launch_count++;
    }
  }
  return GF_OK;
}

// GF_MIXED: apply the FP32 sweeps' accumulated transformation to the FP64
// master and re-round the FP32 copy from it.
int sync_master(gf_ctx* c) {
  if (c->prec != GF_MIXED || c->fp64 || !c->dirty) return GF_OK;
  cudaEvent_t t0 = prof_begin(c);
  cudaError_t e =
      gfk::launch_sync_master(c->links32, c->links64, c->gscratch, c->G, c->NS32, c->NS64, c->ncopies, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "sync: %s", cudaGetErrorString(e));
  prof_end(c, t0, GF_KERNEL_OTHER);
  c->launch_count += 3;
  c->dirty = false;
  return GF_OK;
}

// GF_MIXED: restart the FP32 copy from the FP64 master (accumulator = 1).
int refresh32(gf_ctx* c) {
  if (c->prec != GF_MIXED) return GF_OK;
  cudaError_t e = gfk::launch_demote(c->links64, c->links32, c->G, c->NS64, c->NS32, c->ncopies, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "demote: %s", cudaGetErrorString(e));
  c->launch_count += 2;
  c->fp64 = false;
  c->dirty = false;
  return GF_OK;
}

// Bring the master up to date: pending FP32 transformation applied, and for
// Coulomb the accumulated slice transformation folded into U_0.
int consolidate(gf_ctx* c) {
  int r = sync_master(c);
  if (r) return r;
  return coulomb_fold(c, c->master64());
}

int create_impl(const int dims[4], int ncopies, int gauge, int prec, void* stream, void* buf, size_t bytes,
                gf_ctx** out) {
  if (!out) return fail(GF_EINVAL, "out is NULL");
  *out = nullptr;
  int r = check_dims(dims, ncopies, gauge, prec);
  if (r) return r;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(GF_ENOSYS, "no CUDA device available");
  }
  gf_ctx* c = new (std::nothrow) gf_ctx;
  if (!c) return fail(GF_ENOMEM, "host allocation failed");
  memcpy(c->dims, dims, sizeof c->dims);
  c->ncopies = ncopies;
  c->gauge = gauge;
  c->prec = prec;
  c->device = current_device();
  c->NS32 = (gauge == GF_COULOMB || prec == GF_MIXED) ? 5 : 4;
  c->NS64 = gauge == GF_COULOMB ? 5 : 4;
  c->G = make_geom(dims);
  c->layout = make_layout(dims, ncopies, gauge, prec);
  c->fp64 = prec == GF_FP64;
  c->active_h.assign((size_t)ncopies * dims[0], 1);
  if (stream) {
    c->st = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return fail(GF_ECUDA, "cudaStreamCreate failed");
    }
    c->own_stream = true;
  }
  char* base;
  if (buf) {
    if (((uintptr_t)buf % ALIGN) != 0) {
      gf_destroy(c);
      return fail(GF_EINVAL, "device_buf must be 256-byte aligned");
    }
    if (bytes < c->layout.total) {
      gf_destroy(c);
      return fail(GF_ENOMEM, "device_buf has %zu bytes, %zu needed", bytes, c->layout.total);
    }
    base = static_cast<char*>(buf);
  } else {
    if (cudaMalloc(&c->owned, c->layout.total) != cudaSuccess) {
      cudaGetLastError();
      c->owned = nullptr;
      size_t need = c->layout.total;
      gf_destroy(c);
      return fail(GF_ENOMEM, "cudaMalloc of %zu bytes failed", need);
    }
    base = static_cast<char*>(c->owned);
  }
  const Layout& L = c->layout;
  size_t off = 0;
  if (L.links32) { c->links32 = base + off; off += L.links32; }
  if (L.links64) { c->links64 = base + off; off += L.links64; }
  if (L.gscratch) { c->gscratch = base + off; off += L.gscratch; }
  c->obs_site = base + off; off += L.obs_site;
  c->active_d = reinterpret_cast<int*>(base + off); off += L.active;
  c->slab_flags_d = reinterpret_cast<int*>(base + off); off += L.slab;
  c->partial = reinterpret_cast<double*>(base + off); off += L.partial;
  c->obs_d = reinterpret_cast<double*>(base + off); off += L.obs;
  c->err_d = reinterpret_cast<int*>(base + off); off += L.err;
  c->staging = reinterpret_cast<double*>(base + off); off += L.staging;
  r = upload_active(c);
  if (!r && cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st) != cudaSuccess) r = fail(GF_ECUDA, "init of the error word");
  if (!r) r = set_identity_slots(c, 0, 4);
  if (!r) {
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) r = fail(GF_ECUDA, "init: %s", cudaGetErrorString(e));
  }
  if (r) {
    gf_destroy(c);
    return r;
  }
  {  // start from the launch parameters tuned earlier for this lattice class
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const int vc = volume_class((uint64_t)c->G.V * (uint64_t)c->ncopies);
    for (int f64 = 0; f64 < 2; ++f64)
      for (int a = 0; a < 5; ++a) {
        auto it = g_tuned.find(std::make_tuple(c->device, c->gauge, f64, a, vc));
        if (it != g_tuned.end()) {
          c->lpt[f64][a] = it->second.lpt;
          c->pmode[f64][a] = it->second.pmode + 1;
        }
      }
  }
  *out = c;
  return GF_OK;
}

int check_ctx(gf_ctx* c) { return c ? GF_OK : fail(GF_EINVAL, "context is NULL"); }

// Whole-lattice sweeps would update the halo slices of a time slab.
int check_not_slab(gf_ctx* c, const char* what) {
  return c->slab ? fail(GF_EINVAL, "%s: the context is a time slab; sweep it with gf_sweep_half", what) : GF_OK;
}

int check_copy(gf_ctx* c, int copy, bool allow_all) {
  if (copy == -1 && allow_all) return GF_OK;
  if (copy < 0 || copy >= c->ncopies) return fail(GF_EINVAL, "copy %d out of range [0,%d)", copy, c->ncopies);
  return GF_OK;
}

// Import time-slices [t0, t0+nt) of copy `copy` from natural-order doubles on the device.
// Layout conversion into / out of the master array.
int import_slab(gf_ctx* c, int copy, int t0, int nt, const double* dev) {
  cudaError_t e = c->master64() ? gfk::launch_import<double>(dev, c->links64, c->G, c->NS64, copy, t0, nt, c->st)
                                : gfk::launch_import<float>(dev, c->links32, c->G, c->NS32, copy, t0, nt, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "import: %s", cudaGetErrorString(e));
  c->launch_count++;
  return GF_OK;
}

int export_slab(gf_ctx* c, int copy, int t0, int nt, double* dev) {
  cudaError_t e = c->master64() ? gfk::launch_export<double>(dev, c->links64, c->G, c->NS64, copy, t0, nt, c->st)
                                : gfk::launch_export<float>(dev, c->links32, c->G, c->NS32, copy, t0, nt, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "export: %s", cudaGetErrorString(e));
  c->launch_count++;
  return GF_OK;
}

// A new problem: links go to the master array; pending transformations are
// dropped (slot 4 = 1 in every array).
int begin_load(gf_ctx* c) {
  c->dirty = false;
  if (c->prec == GF_MIXED || c->gauge == GF_COULOMB) return set_identity_slots(c, 4, 4);
  return GF_OK;
}

// After new links reached the master: GF_MIXED restarts its FP32 copy.
int end_load(gf_ctx* c) { return refresh32(c); }

int replicate_copy0(gf_ctx* c) {
  const bool f64 = c->master64();
  const size_t blk = c->copy_block_bytes(f64);
  char* base = static_cast<char*>(f64 ? c->links64 : c->links32);
  for (int k = 1; k < c->ncopies; ++k)
    GF_CUDA(cudaMemcpyAsync(base + k * blk, base, blk, cudaMemcpyDeviceToDevice, c->st));
  return GF_OK;
}

int check_algo_param(int algo, double param) {
  switch (algo) {
    case GF_RELAX:
    case GF_MICRO:
      return GF_OK;
    case GF_OR:
      if (!(param >= 1.0 && param <= 2.0)) return fail(GF_EINVAL, "omega = %g not in [1,2]", param);
      return GF_OK;
    case GF_SR:
      if (!(param >= 0.0 && param <= 1.0)) return fail(GF_EINVAL, "p = %g not in [0,1]", param);
      return GF_OK;
    case GF_SA:
      if (!(param > 0.0) || !std::isfinite(param)) return fail(GF_EINVAL, "T = %g must be > 0", param);
      return GF_OK;
  }
  return fail(GF_EINVAL, "bad algorithm %d", algo);
}

// One API-level sweep: SA = heat bath + sa_micro (3) microcanonical sweeps.
int api_sweep(gf_ctx* c, int algo, double param, uint64_t seed, bool obs_last = false) {
  switch (algo) {
    case GF_RELAX: return full_sweep(c, gfk::ALG_OR, GF_RELAX, 1.0, seed, 0, obs_last);
    case GF_OR: return full_sweep(c, gfk::ALG_OR, GF_OR, param, seed, 0, obs_last);
    case GF_MICRO: return full_sweep(c, gfk::ALG_MICRO, GF_MICRO, 0.0, seed);
    case GF_SR: return full_sweep(c, gfk::ALG_SR, GF_SR, param, seed);
    case GF_SA: {
      int r = full_sweep(c, gfk::ALG_SA, GF_SA, param, seed);
      for (int k = 0; k < c->sa_micro && !r; ++k) r = full_sweep(c, gfk::ALG_MICRO, GF_MICRO, 0.0, seed);
      return r;
    }
  }
  return fail(GF_EINVAL, "bad algorithm %d", algo);
}

// End of a public sweep call: the master is brought up to date (GF_MIXED) and
// the exact observables of the master are returned if asked for.
int finish_public(gf_ctx* c, double* F, double* theta) {
  int r = sync_master(c);
  if (r) return r;
  if (F || theta) {
    std::vector<double> ct;
    if ((r = observables_on(c, ct, c->master64()))) return r;
    copy_means(c, ct, F, theta);
    return GF_OK;
  }
  GF_CUDA(cudaStreamSynchronize(c->st));
  return read_sweep_error(c);
}

int reunitarize(gf_ctx* c) {
  // GF_MIXED with FP32 sweeps: the FP64 master stays unitary; re-rounding the
  // FP32 copy from it (after applying the pending transformation) replaces the
  // re-unitarisation of the FP32 links.
  if (c->prec == GF_MIXED && !c->fp64) {
    c->dirty = true;
    return sync_master(c);
  }
  const uint64_t nmat = (uint64_t)c->ncopies * 2 * c->NS() * c->G.Vh;
  cudaEvent_t t0 = prof_begin(c);
  cudaError_t e = c->fp64 ? gfk::launch_reunitarize<double>(c->links64, c->G.Vh, nmat, c->st)
                          : gfk::launch_reunitarize<float>(c->links32, c->G.Vh, nmat, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "reunitarize: %s", cudaGetErrorString(e));
  prof_end(c, t0, GF_KERNEL_REUNITARIZE);
  c->launch_count++;
  return GF_OK;
}

// GF_MIXED: switch the sweeps to the FP64 master (the FP32 stage's pending
// transformation applied first).
int promote(gf_ctx* c) {
  if (c->fp64) return GF_OK;
  if (c->prec != GF_MIXED) return fail(GF_EINVAL, "gf_promote needs a GF_MIXED context");
  int r = sync_master(c);
  if (r) return r;
  c->fp64 = true;
  return GF_OK;
}

// ---- Groups: several contexts (lattices of different extents) per launch ----

static_assert(GF_GROUP_MAX == gfk::GROUP_MAX, "the group size limit of the ABI and of the kernel");

int check_group(gf_ctx* const* ctxs, int n) {
  if (!ctxs || n < 1 || n > gfk::GROUP_MAX) return fail(GF_EINVAL, "a group has 1..%d contexts", gfk::GROUP_MAX);
  for (int k = 0; k < n; ++k) {
    gf_ctx* c = ctxs[k];
    if (!c) return fail(GF_EINVAL, "context %d of the group is NULL", k);
    if (c->gauge != ctxs[0]->gauge) return fail(GF_EINVAL, "group members differ in gauge");
    if (c->device != ctxs[0]->device) return fail(GF_EINVAL, "group members live on different devices");
    if (c->prec == GF_MP) return fail(GF_EINVAL, "GF_MP contexts cannot be grouped");
    if (c->slab) return fail(GF_EINVAL, "time slabs cannot be grouped");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == c) return fail(GF_EINVAL, "context %d appears twice in the group", k);
  }
  return GF_OK;
}

// n sweeps (overrelaxation, omega) of members that share their storage
// precision, one launch per half-sweep on the first member's stream.  The
// arguments are built once and only the parity and the sweep index change
// between launches; the other members' streams are ordered before the first
// and after the last launch with events (not around every launch).
template <typename R>
int group_sweeps_t(const std::vector<gf_ctx*>& m, double omega, int n) {
  gf_ctx* c0 = m[0];
  int lpt = default_lpt(c0, GF_OR);
  if (c0->gauge == GF_MAG && sizeof(R) == 8 && lpt == 8) lpt = 4;  // as the single-lattice launcher
  const uint32_t tile = gfk::BLOCK / (8 / lpt);
  static thread_local gfk::GroupArgs<R> g;
  uint64_t cum = 0;
  for (size_t k = 0; k < m.size(); ++k) {
    // the group kernel prefetches the next tile into L2 or nothing (it has no staged form)
    fill_args(g.m[k], m[k], gfk::ALG_OR, omega, 0, 0, 0, 0, 1,
              m[k]->prefetch == GF_PREFETCH_NONE ? GF_PREFETCH_NONE : GF_PREFETCH_L2, nullptr);
    cum += (uint64_t)((m[k]->G.Vh + tile - 1) / tile) * (uint64_t)m[k]->ncopies;
    g.tile_end[k] = cum;
  }
  g.n = (uint32_t)m.size();
  g.ntiles = cum;
  std::vector<cudaEvent_t> evs;
  for (size_t k = 1; k < m.size(); ++k)
    if (m[k]->st != c0->st) {
      cudaEvent_t e = take_event(c0);
      GF_CUDA(cudaEventRecord(e, m[k]->st));
      GF_CUDA(cudaStreamWaitEvent(c0->st, e, 0));
      evs.push_back(e);
    }
  for (int s = 0; s < n; ++s)
    for (int parity = 0; parity < 2; ++parity) {
      for (size_t k = 0; k < m.size(); ++k) {
        g.m[k].parity = parity;
        g.m[k].sweep = (uint32_t)(m[k]->sweep_index + s);
      }
      cudaEvent_t t0 = prof_begin(c0);
      cudaError_t e = gfk::launch_group<R>(g, c0->gauge, lpt, c0->st);
      if (e != cudaSuccess) return fail(GF_ECUDA, "group sweep launch: %s", cudaGetErrorString(e));
      prof_end(c0, t0, sizeof(R) == 8 ? GF_KERNEL_SWEEP_FP64 : GF_KERNEL_SWEEP_FP32);
      c0->launch_count++;
    }
  if (!evs.empty()) {
    cudaEvent_t done = take_event(c0);
    GF_CUDA(cudaEventRecord(done, c0->st));
    for (size_t k = 1; k < m.size(); ++k)
      if (m[k]->st != c0->st) GF_CUDA(cudaStreamWaitEvent(m[k]->st, done, 0));
    evs.push_back(done);
  }
  // a wait already enqueued refers to the event's record at the time of the
  // call, so the events can be recorded again right away
  for (cudaEvent_t ev : evs) c0->event_pool.push_back(ev);
  return GF_OK;
}

// n sweeps of every member: members in FP32 storage and members in FP64
// storage (a GF_MIXED member after its switch) go in separate launches.
int group_sweeps(const std::vector<gf_ctx*>& members, double omega, int n) {
  if (n <= 0) return GF_OK;
  std::vector<gf_ctx*> by[2];
  for (gf_ctx* c : members) by[c->fp64 ? 1 : 0].push_back(c);
  for (int f = 0; f < 2; ++f) {
    if (by[f].empty()) continue;
    int r = f ? group_sweeps_t<double>(by[f], omega, n) : group_sweeps_t<float>(by[f], omega, n);
    if (r) return r;
  }
  for (gf_ctx* c : members) {
    c->sweep_index += (uint64_t)n;
    if (c->prec == GF_MIXED && !c->fp64) c->dirty = true;
  }
  return GF_OK;
}

}  // namespace

extern "C" {

int gf_footprint(const int dims[4], int n_copies, gf_gauge gauge, gf_precision prec, size_t* bytes) {
  int r = check_dims(dims, n_copies, gauge, prec);
  if (r) return r;
  if (!bytes) return fail(GF_EINVAL, "bytes is NULL");
  *bytes = make_layout(dims, n_copies, gauge, prec).total;
  return GF_OK;
}

int gf_create(const int dims[4], gf_gauge gauge, gf_precision prec, void* stream, gf_ctx** out) {
  return create_impl(dims, 1, gauge, prec, stream, nullptr, 0, out);
}

int gf_create_batch(const int dims[4], int n_copies, gf_gauge gauge, gf_precision prec, void* stream,
                    gf_ctx** out) {
  return create_impl(dims, n_copies, gauge, prec, stream, nullptr, 0, out);
}

int gf_create_ext(const int dims[4], int n_copies, gf_gauge gauge, gf_precision prec, void* stream,
                  void* device_buf, size_t bytes, gf_ctx** out) {
  if (!device_buf) return fail(GF_EINVAL, "device_buf is NULL");
  return create_impl(dims, n_copies, gauge, prec, stream, device_buf, bytes, out);
}

void gf_destroy(gf_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  prof_collect(c);
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
  if (c->check_log) fclose(c->check_log);
  if (c->owned) cudaFree(c->owned);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

int gf_load_links_slab(gf_ctx* c, int copy, int t0, int nt, const double* host) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_copy(c, copy, true))) return r;
  if (!host) return fail(GF_EINVAL, "host is NULL");
  if (t0 < 0 || nt < 1 || t0 + nt > c->dims[0]) return fail(GF_EINVAL, "slab [%d,%d) outside [0,%d)", t0, t0 + nt, c->dims[0]);
  if (t0 == 0 && nt == c->dims[0] && (r = begin_load(c))) return r;
  const int dst = copy < 0 ? 0 : copy;
  const size_t per_t = (size_t)c->G.V3 * 4 * 18;
  for (int t = t0; t < t0 + nt; t += c->layout.slab_nt) {
    const int n = std::min(c->layout.slab_nt, t0 + nt - t);
    GF_CUDA(cudaMemcpyAsync(c->staging, host + (size_t)(t - t0) * per_t, (size_t)n * per_t * sizeof(double),
                            cudaMemcpyHostToDevice, c->st));
    if ((r = import_slab(c, dst, t, n, c->staging))) return r;
  }
  if (copy < 0 && (r = replicate_copy0(c))) return r;
  if ((r = end_load(c))) return r;
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int gf_load_links(gf_ctx* c, int copy, const double* host) {
  int r = check_ctx(c);
  if (r) return r;
  return gf_load_links_slab(c, copy, 0, c->dims[0], host);
}

int gf_load_links_device(gf_ctx* c, int copy, const double* dev) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_copy(c, copy, true))) return r;
  if (!dev) return fail(GF_EINVAL, "device_src is NULL");
  if ((r = begin_load(c))) return r;
  if ((r = import_slab(c, copy < 0 ? 0 : copy, 0, c->dims[0], dev))) return r;
  if (copy < 0 && (r = replicate_copy0(c))) return r;
  if ((r = end_load(c))) return r;
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int gf_store_links(gf_ctx* c, int copy, double* host) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_copy(c, copy, false))) return r;
  if (!host) return fail(GF_EINVAL, "host is NULL");
  if ((r = consolidate(c))) return r;
  const size_t per_t = (size_t)c->G.V3 * 4 * 18;
  for (int t = 0; t < c->dims[0]; t += c->layout.slab_nt) {
    const int n = std::min(c->layout.slab_nt, c->dims[0] - t);
    if ((r = export_slab(c, copy, t, n, c->staging))) return r;
    GF_CUDA(cudaMemcpyAsync(host + (size_t)t * per_t, c->staging, (size_t)n * per_t * sizeof(double),
                            cudaMemcpyDeviceToHost, c->st));
  }
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int gf_store_links_slab(gf_ctx* c, int copy, int t0, int nt, double* host) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_copy(c, copy, false))) return r;
  if (!host) return fail(GF_EINVAL, "host is NULL");
  if (t0 < 0 || nt < 1 || t0 + nt > c->dims[0]) return fail(GF_EINVAL, "slab [%d,%d) outside [0,%d)", t0, t0 + nt, c->dims[0]);
  if ((r = consolidate(c))) return r;
  const size_t per_t = (size_t)c->G.V3 * 4 * 18;
  for (int t = t0; t < t0 + nt; t += c->layout.slab_nt) {
    const int n = std::min(c->layout.slab_nt, t0 + nt - t);
    if ((r = export_slab(c, copy, t, n, c->staging))) return r;
    GF_CUDA(cudaMemcpyAsync(host + (size_t)(t - t0) * per_t, c->staging, (size_t)n * per_t * sizeof(double),
                            cudaMemcpyDeviceToHost, c->st));
  }
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int gf_store_links_device(gf_ctx* c, int copy, double* dev) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_copy(c, copy, false))) return r;
  if (!dev) return fail(GF_EINVAL, "device_dst is NULL");
  if ((r = consolidate(c))) return r;
  if ((r = export_slab(c, copy, 0, c->dims[0], dev))) return r;
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int gf_random_gauge_transform_async(gf_ctx* c, uint64_t seed) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_not_slab(c, "gf_random_gauge_transform_async"))) return r;
  if ((r = consolidate(c))) return r;
  cudaError_t e = c->master64()
                      ? gfk::launch_haar_transform<double>(c->links64, c->G, c->NS64, c->ncopies, c->copy_base, seed, c->st)
                      : gfk::launch_haar_transform<float>(c->links32, c->G, c->NS32, c->ncopies, c->copy_base, seed, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "random gauge transform: %s", cudaGetErrorString(e));
  c->launch_count += 2;
  return refresh32(c);
}

int gf_random_gauge_transform(gf_ctx* c, uint64_t seed) {
  int r = gf_random_gauge_transform_async(c, seed);
  if (r) return r;
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int gf_sweep_async(gf_ctx* c, gf_algo algo, double param, int n_sweeps, uint64_t seed) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_not_slab(c, "gf_sweep_async"))) return r;
  if ((r = check_algo_param(algo, param))) return r;
  if (n_sweeps < 0) return fail(GF_EINVAL, "n_sweeps < 0");
  if (algo == GF_OR || algo == GF_RELAX) {
    if ((r = plain_sweeps(c, gfk::ALG_OR, algo, algo == GF_RELAX ? 1.0 : param, n_sweeps))) return r;
  } else {
    for (int k = 0; k < n_sweeps; ++k)
      if ((r = api_sweep(c, algo, param, seed))) return r;
  }
  return sync_master(c);  // enqueued, as at the end of gf_sweep
}

int gf_anneal_async(gf_ctx* c, double T0, double T1, int n_steps, uint64_t seed) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_not_slab(c, "gf_anneal_async"))) return r;
  if (!(T0 > 0) || !(T1 > 0) || !std::isfinite(T0) || !std::isfinite(T1))
    return fail(GF_EINVAL, "temperatures must be > 0");
  if (n_steps < 0) return fail(GF_EINVAL, "n_steps < 0");
  for (int k = 0; k < n_steps; ++k) {
    const double T = n_steps > 1 ? T0 + (T1 - T0) * (double)k / (double)(n_steps - 1) : T0;
    if ((r = api_sweep(c, GF_SA, T, seed))) return r;
  }
  return sync_master(c);  // enqueued, as at the end of gf_anneal
}

int gf_synchronize(gf_ctx* c) {
  int r = check_ctx(c);
  if (r) return r;
  GF_CUDA(cudaStreamSynchronize(c->st));
  prof_collect(c);
  return read_sweep_error(c);
}

int gf_sweep(gf_ctx* c, gf_algo algo, double param, int n_sweeps, uint64_t seed, double* F, double* theta) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_not_slab(c, "gf_sweep"))) return r;
  if ((r = check_algo_param(algo, param))) return r;
  if (n_sweeps < 0) return fail(GF_EINVAL, "n_sweeps < 0");
  // fused observables: the odd half of the last sweep writes F/theta of its
  // sites (only when those links are the final ones: not in the FP32 stage of
  // GF_MIXED, whose master is read instead)
  const bool fused = c->fused_obs && (F || theta) && n_sweeps > 0 && (algo == GF_OR || algo == GF_RELAX) &&
                     !(c->prec == GF_MIXED && !c->fp64) && c->prec != GF_MP;
  if ((algo == GF_OR || algo == GF_RELAX) && n_sweeps > 0) {
    const double omega = algo == GF_RELAX ? 1.0 : param;
    if ((r = plain_sweeps(c, gfk::ALG_OR, algo, omega, n_sweeps - 1))) return r;
    if ((r = full_sweep(c, gfk::ALG_OR, algo, omega, seed, 0, fused))) return r;
  } else {
    for (int k = 0; k < n_sweeps; ++k)
      if ((r = api_sweep(c, algo, param, seed, fused && k == n_sweeps - 1))) return r;
  }
  if (fused) {
    std::vector<double> ct;
    if ((r = fused_observables(c, ct))) return r;
    copy_means(c, ct, F, theta);
    return GF_OK;
  }
  return finish_public(c, F, theta);
}

int gf_anneal(gf_ctx* c, double T0, double T1, int n_steps, uint64_t seed, double* F, double* theta) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_not_slab(c, "gf_anneal"))) return r;
  if (!(T0 > 0) || !(T1 > 0) || !std::isfinite(T0) || !std::isfinite(T1))
    return fail(GF_EINVAL, "temperatures must be > 0");
  if (n_steps < 0) return fail(GF_EINVAL, "n_steps < 0");
  for (int k = 0; k < n_steps; ++k) {
    const double T = n_steps > 1 ? T0 + (T1 - T0) * (double)k / (double)(n_steps - 1) : T0;
    if ((r = api_sweep(c, GF_SA, T, seed))) return r;
  }
  return finish_public(c, F, theta);
}

int gf_reunitarize(gf_ctx* c) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = reunitarize(c))) return r;
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int gf_functional_theta(gf_ctx* c, double* F, double* theta) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = sync_master(c))) return r;
  std::vector<double> ct;
  if ((r = observables_on(c, ct, c->master64()))) return r;
  copy_means(c, ct, F, theta);
  return GF_OK;
}

int gf_slice_functional_theta(gf_ctx* c, double* F_t, double* theta_t) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = sync_master(c))) return r;
  std::vector<double> ct;
  if ((r = observables_on(c, ct, c->master64()))) return r;
  for (size_t k = 0; k < ct.size() / 2; ++k) {
    if (F_t) F_t[k] = ct[2 * k];
    if (theta_t) theta_t[k] = ct[2 * k + 1];
  }
  return GF_OK;
}

int gf_promote(gf_ctx* c) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = promote(c))) return r;
  GF_CUDA(cudaStreamSynchronize(c->st));
  return GF_OK;
}

int gf_set_active(gf_ctx* c, const int* flags) {
  int r = check_ctx(c);
  if (r) return r;
  const int Nt = c->dims[0];
  for (int k = 0; k < c->ncopies; ++k) {
    bool all = true;
    for (int t = 0; t < Nt; ++t) {
      const int v = flags ? (flags[(size_t)k * Nt + t] != 0) : 1;
      c->active_h[(size_t)k * Nt + t] = v;
      all = all && v;
    }
    if (c->gauge != GF_COULOMB && !all)
      for (int t = 0; t < Nt; ++t) c->active_h[(size_t)k * Nt + t] = 0;
  }
  return upload_active(c);
}

int gf_get_sweep_index(gf_ctx* c, uint64_t* index) {
  int r = check_ctx(c);
  if (r) return r;
  if (!index) return fail(GF_EINVAL, "index is NULL");
  *index = c->sweep_index;
  return GF_OK;
}

int gf_set_sweep_index(gf_ctx* c, uint64_t index) {
  int r = check_ctx(c);
  if (r) return r;
  c->sweep_index = index;
  return GF_OK;
}

int gf_set_copy_base(gf_ctx* c, uint32_t base) {
  int r = check_ctx(c);
  if (r) return r;
  c->copy_base = base;
  return GF_OK;
}

int gf_set_sa_micro(gf_ctx* c, int n_micro) {
  int r = check_ctx(c);
  if (r) return r;
  if (n_micro < 0 || n_micro > 64) return fail(GF_EINVAL, "n_micro = %d not in [0, 64]", n_micro);
  c->sa_micro = n_micro;
  return GF_OK;
}

int gf_set_sa_trace(gf_ctx* c, int* device_counts) {
  int r = check_ctx(c);
  if (r) return r;
  if (((uintptr_t)device_counts & 3) != 0) return fail(GF_EINVAL, "device_counts must be 4-byte aligned");
  c->sa_trace_d = device_counts;
  return GF_OK;
}

int gf_set_slab(gf_ctx* c, int t0, int Nt_global) {
  int r = check_ctx(c);
  if (r) return r;
  const int nl = c->dims[0];
  if (c->ncopies != 1) return fail(GF_EINVAL, "a time slab holds one lattice (n_copies = %d)", c->ncopies);
  if (c->gauge == GF_COULOMB) return fail(GF_EINVAL, "Coulomb time-slices need no slab exchange: split them as units");
  if (c->prec == GF_MIXED) return fail(GF_EINVAL, "time slabs run in GF_FP64 or GF_FP32 storage");
  if (nl < 4) return fail(GF_EINVAL, "a slab needs at least two owned slices (local Nt = %d)", nl);
  if (Nt_global < nl - 2 || (Nt_global & 1) || t0 < 0 || t0 >= Nt_global)
    return fail(GF_EINVAL, "slab t0 = %d, Nt_global = %d do not fit %d owned slices", t0, Nt_global, nl - 2);
  std::vector<int> flags((size_t)3 * nl, 0);
  for (int t = 1; t <= nl - 2; ++t) {
    flags[t] = 1;                                   // owned
    flags[nl + t] = (t == 1 || t == nl - 2) ? 1 : 0;  // boundary: the first and last owned slice
    flags[2 * nl + t] = 1 - flags[nl + t];          // inner
  }
  GF_CUDA(cudaMemcpyAsync(c->slab_flags_d, flags.data(), flags.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
  GF_CUDA(cudaStreamSynchronize(c->st));
  c->slab = true;
  c->slab_t0 = t0;
  c->slab_Nt = Nt_global;
  c->parity_flip = (t0 - 1) & 1;
  c->site_offset = (uint32_t)((int64_t)(t0 - 1) * (int64_t)c->G.V3);
  return GF_OK;
}

int gf_sweep_half(gf_ctx* c, gf_algo algo, double param, int parity, int part, uint64_t seed) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_algo_param(algo, param))) return r;
  if (parity != 0 && parity != 1) return fail(GF_EINVAL, "parity must be 0 or 1");
  if (part < GF_SLAB_OWNED || part > GF_SLAB_INNER) return fail(GF_EINVAL, "bad part %d", part);
  if (!c->slab && part != GF_SLAB_OWNED) return fail(GF_EINVAL, "boundary/inner parts need a time slab");
  if (c->prec == GF_MIXED && !c->fp64) return fail(GF_EINVAL, "gf_sweep_half runs on FP64 or FP32 storage");
  const int kalgo = algo == GF_MICRO ? gfk::ALG_MICRO : algo == GF_SR ? gfk::ALG_SR : algo == GF_SA ? gfk::ALG_SA
                                                                                            : gfk::ALG_OR;
  const double p = algo == GF_RELAX ? 1.0 : algo == GF_MICRO ? 0.0 : param;
  const int* act = c->slab ? c->slab_flags_d + (size_t)part * c->dims[0] : nullptr;
  const int pm = c->pmode[c->fp64][algo] - 1;
  const int lp = default_lpt(c, algo);
  const uint32_t sw = (uint32_t)c->sweep_index;
  if (!(c->slab && c->fp64))
    return launch_half(c, kalgo, p, parity ^ c->parity_flip, seed, sw, lp, 0, 1, pm, act);
  // FP64 slab: each launch covers its slices' sites only (slice t holds the
  // sites [t, t + 1) x V3/2 of a parity), so that the FP64 kernel's equal
  // ranges spread the part over every block; the flags stay as a guard
  const uint32_t vs = (uint32_t)(c->G.V3 / 2), nl = (uint32_t)c->dims[0];
  if (part == GF_SLAB_BOUNDARY) {
    for (uint32_t t : {1u, nl - 2u})
      if ((r = launch_half(c, kalgo, p, parity ^ c->parity_flip, seed, sw, lp, 0, 1, pm, act, t * vs, vs))) return r;
    return GF_OK;
  }
  const uint32_t t0 = part == GF_SLAB_INNER ? 2u : 1u, t1 = part == GF_SLAB_INNER ? nl - 2u : nl - 1u;  // [t0, t1)
  if (t1 <= t0) return GF_OK;  // two owned slices: no inner slice
  return launch_half(c, kalgo, p, parity ^ c->parity_flip, seed, sw, lp, 0, 1, pm, act, t0 * vs, (t1 - t0) * vs);
}

int gf_slab_bytes(gf_ctx* c, size_t* bytes) {
  int r = check_ctx(c);
  if (r) return r;
  if (!bytes) return fail(GF_EINVAL, "bytes is NULL");
  *bytes = (size_t)(c->fp64 ? 6 : 3) * (c->G.V3 / 2) * 16;
  return GF_OK;
}

// U_0 rows 0,1 of the sites of one parity in one local time-slice: NC chunks
// of V3/2 vectors, contiguous per chunk in the storage (Sec. 5.2's argument
// for a time-slice-major, parity-split layout), moved by one 2-D copy.
static int slab_copy(gf_ctx* c, int slice, int parity, void* buf, bool pack) {
  int r = check_ctx(c);
  if (r) return r;
  if (!buf) return fail(GF_EINVAL, "buffer is NULL");
  if (slice < 0 || slice >= c->dims[0]) return fail(GF_EINVAL, "slice %d outside [0,%d)", slice, c->dims[0]);
  if (parity != 0 && parity != 1) return fail(GF_EINVAL, "parity must be 0 or 1");
  if (c->prec == GF_MIXED && !c->fp64) return fail(GF_EINVAL, "slab exchange runs on FP64 or FP32 storage");
  const int NC = c->fp64 ? 6 : 3;
  const size_t half = c->G.V3 / 2;
  const size_t elem = gfk::link_off(0, parity ^ c->parity_flip, 0, c->NS(), NC, c->G.Vh, (uint32_t)(slice * half));
  char* links = static_cast<char*>(c->links()) + elem * 16;
  const size_t pitch = (size_t)c->G.Vh * 16, width = half * 16;
  cudaError_t e = pack ? cudaMemcpy2DAsync(buf, width, links, pitch, width, NC, cudaMemcpyDefault, c->st)
                       : cudaMemcpy2DAsync(links, pitch, buf, width, width, NC, cudaMemcpyDefault, c->st);
  if (e != cudaSuccess) return fail(GF_ECUDA, "slab %s: %s", pack ? "pack" : "unpack", cudaGetErrorString(e));
  return GF_OK;
}

int gf_slab_pack(gf_ctx* c, int slice, int parity, void* buf) { return slab_copy(c, slice, parity, buf, true); }

int gf_slab_unpack(gf_ctx* c, int slice, int parity, const void* buf) {
  return slab_copy(c, slice, parity, const_cast<void*>(buf), false);
}

int gf_group_sweep(gf_ctx* const* ctxs, int n, gf_algo algo, double param, int n_sweeps) {
  int r = check_group(ctxs, n);
  if (r) return r;
  if (algo != GF_OR && algo != GF_RELAX) return fail(GF_EINVAL, "group sweeps run GF_OR or GF_RELAX");
  if ((r = check_algo_param(algo, param))) return r;
  if (n_sweeps < 0) return fail(GF_EINVAL, "n_sweeps < 0");
  std::vector<gf_ctx*> m(ctxs, ctxs + n);
  const double omega = algo == GF_RELAX ? 1.0 : param;
  if ((r = group_sweeps(m, omega, n_sweeps))) return r;
  for (gf_ctx* c : m) {
    if ((r = sync_master(c))) return r;
    GF_CUDA(cudaStreamSynchronize(c->st));
  }
  return GF_OK;
}

int gf_group_fix(gf_ctx* const* ctxs, int n, const gf_fix_params* P, gf_fix_result* results) {
  int r = check_group(ctxs, n);
  if (r) return r;
  if (!P) return fail(GF_EINVAL, "params is NULL");
  if (P->algo != GF_OR && P->algo != GF_RELAX) return fail(GF_EINVAL, "gf_group_fix runs GF_OR or GF_RELAX");
  if ((r = check_algo_param(P->algo, P->param))) return r;
  if (!(P->theta_target > 0) || P->max_sweeps < 0 || P->check_interval < 1 || P->reunit_interval < 0)
    return fail(GF_EINVAL, "bad fix parameters");
  Range range_fix("gf_group_fix");
  const auto t_start = std::chrono::steady_clock::now();
  const double omega = P->algo == GF_RELAX ? 1.0 : P->param;
  std::vector<gf_fix_result> R(n);
  std::vector<int> since(n, 0);
  std::vector<int> live(n, 1);
  std::vector<uint64_t> units(n, 0);  // sites of a member's active units
  std::vector<double> ct;
  for (auto& x : R) memset(&x, 0, sizeof x);
  for (;;) {
    // every live member: theta per unit (a copy, or a Coulomb time-slice) from the standalone pass
    std::vector<gf_ctx*> sweepers;
    for (int k = 0; k < n; ++k) {
      if (!live[k]) continue;
      gf_ctx* c = ctxs[k];
      if ((r = observables(c, ct))) return r;
      R[k].checks++;
      const int Nt = c->dims[0];
      const bool coul = c->gauge == GF_COULOMB;
      const bool final_phase = c->fp64 || c->prec == GF_FP32;
      double worst = 0, fs = 0, tmax = 0;
      int n_active = 0;
      for (int q = 0; q < c->ncopies; ++q) {
        double tsum = 0;
        for (int t = 0; t < Nt; ++t) {
          fs += ct[2 * ((size_t)q * Nt + t)];
          tsum += ct[2 * ((size_t)q * Nt + t) + 1];
        }
        for (int u = 0; u < (coul ? Nt : 1); ++u) {
          const double th = coul ? ct[2 * ((size_t)q * Nt + u) + 1] : tsum / Nt;
          tmax = std::max(tmax, th);
          const int v = (final_phase && th < P->theta_target) ? 0 : 1;
          if (coul) c->active_h[(size_t)q * Nt + u] = v;
          else
            for (int t = 0; t < Nt; ++t) c->active_h[(size_t)q * Nt + t] = v;
          if (v) {
            n_active++;
            worst = std::max(worst, th);
          }
        }
      }
      R[k].F_mean = fs / ((double)c->ncopies * Nt);
      R[k].theta_max = tmax;
      if ((r = upload_active(c))) return r;
      if (n_active == 0) {
        R[k].converged = 1;
        live[k] = 0;
        continue;
      }
      if (R[k].sweeps >= P->max_sweeps) {
        live[k] = 0;
        continue;
      }
      if (!c->fp64 && c->prec == GF_MIXED && (worst < P->switch_theta || !std::isfinite(worst))) {
        if ((r = promote(c))) return r;
        continue;  // evaluated again in FP64 at the next pass of the loop
      }
      sweepers.push_back(c);
      units[k] = (uint64_t)n_active * (coul ? c->G.V3 : c->G.V);
    }
    if (sweepers.empty()) {
      bool any = false;
      for (int k = 0; k < n; ++k) any = any || live[k];
      if (!any) break;
      continue;  // only promotions in this pass
    }
    // a common interval: the members that are still sweeping
    int steps = P->check_interval;
    for (int k = 0; k < n; ++k)
      if (live[k]) steps = std::min(steps, std::max(1, P->max_sweeps - R[k].sweeps));
    for (int s = 0; s < steps;) {
      // up to the next re-unitarisation of any sweeping member
      int chunk = steps - s;
      if (P->reunit_interval > 0)
        for (int k = 0; k < n; ++k)
          if (live[k] && std::find(sweepers.begin(), sweepers.end(), ctxs[k]) != sweepers.end())
            chunk = std::min(chunk, P->reunit_interval - since[k]);
      if ((r = group_sweeps(sweepers, omega, chunk))) return r;
      s += chunk;
      for (int k = 0; k < n; ++k) {
        if (!live[k] || std::find(sweepers.begin(), sweepers.end(), ctxs[k]) == sweepers.end()) continue;
        gf_ctx* c = ctxs[k];
        if (c->fp64) R[k].sweeps_fp64 += chunk;
        else R[k].sweeps_fp32 += chunk;
        R[k].sweeps += chunk;
        R[k].site_updates += (uint64_t)chunk * units[k];
        since[k] += chunk;
        if (P->reunit_interval > 0 && since[k] >= P->reunit_interval) {
          since[k] = 0;
          if ((r = reunitarize(c))) return r;
        }
      }
    }
  }
  bool all = true;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  for (int k = 0; k < n; ++k) {
    gf_ctx* c = ctxs[k];
    std::fill(c->active_h.begin(), c->active_h.end(), 1);
    if ((r = upload_active(c))) return r;
    if ((r = sync_master(c))) return r;
    R[k].seconds = secs;
    all = all && R[k].converged;
    if (results) results[k] = R[k];
  }
  if (!all) return fail(GF_ENOTCONV, "some group members did not reach theta_target");
  return GF_OK;
}

int gf_set_fused_observables(gf_ctx* c, int on) {
  int r = check_ctx(c);
  if (r) return r;
  c->fused_obs = on ? 1 : 0;
  return GF_OK;
}

int gf_set_check_log(gf_ctx* c, const char* path) {
  int r = check_ctx(c);
  if (r) return r;
  if (c->check_log) fclose(c->check_log);
  c->check_log = nullptr;
  if (!path) return GF_OK;
  c->check_log = fopen(path, "a");
  if (!c->check_log) return fail(GF_EINVAL, "cannot open %s for appending", path);
  return GF_OK;
}

int gf_set_stage_wait_polls(gf_ctx* c, int polls) {
  int r = check_ctx(c);
  if (r) return r;
  c->stage_wait_polls = polls < 0 ? -1 : polls;
  return GF_OK;
}

int gf_set_graphs(gf_ctx* c, int on) {
  int r = check_ctx(c);
  if (r) return r;
  c->use_graphs = on != 0;
  return GF_OK;
}

int gf_set_prefetch(gf_ctx* c, int mode) {
  int r = check_ctx(c);
  if (r) return r;
  if (mode < GF_PREFETCH_NONE || mode > GF_PREFETCH_SMEM) return fail(GF_EINVAL, "bad prefetch mode %d", mode);
  c->prefetch = mode;
  memset(c->pmode, 0, sizeof c->pmode);  // an explicit choice replaces the tuned ones
  return GF_OK;
}

int gf_set_links_per_thread(gf_ctx* c, int lpt) {
  int r = check_ctx(c);
  if (r) return r;
  if (lpt != 0 && lpt != 1 && lpt != 2 && lpt != 4 && lpt != 8) return fail(GF_EINVAL, "lpt must be 0,1,2,4,8");
  for (int p = 0; p < 2; ++p)
    for (int a = 0; a < 5; ++a) c->lpt[p][a] = lpt;
  return GF_OK;
}

int gf_get_links_per_thread(gf_ctx* c, int* lpt) {
  int r = check_ctx(c);
  if (r) return r;
  if (!lpt) return fail(GF_EINVAL, "lpt is NULL");
  *lpt = default_lpt(c, GF_OR);
  return GF_OK;
}

int gf_autotune(gf_ctx* c, gf_algo algo, int* best_lpt, double* ms_best) {
  int r = check_ctx(c);
  if (r) return r;
  if (algo < GF_RELAX || algo > GF_SA) return fail(GF_EINVAL, "bad algorithm %d", algo);
  const size_t bytes = c->copy_block_bytes() * c->ncopies;
  void* backup = nullptr;
  if (cudaMalloc(&backup, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(GF_ENOMEM, "autotune scratch of %zu bytes", bytes);
  }
  GF_CUDA(cudaMemcpyAsync(backup, c->links(), bytes, cudaMemcpyDeviceToDevice, c->st));
  const uint64_t idx0 = c->sweep_index;
  const int kalgo = algo == GF_MICRO ? gfk::ALG_MICRO : algo == GF_SR ? gfk::ALG_SR : algo == GF_SA ? gfk::ALG_SA : gfk::ALG_OR;
  const double param = algo == GF_SR ? 0.5 : algo == GF_SA ? 1.0 : algo == GF_OR ? 1.7 : 1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = 0, best_mode = c->prefetch;
  float best_ms = 1e30f;
  const int cands[4] = {1, 2, 4, 8};
  // FP32 storage: both tile fetches (L2 prefetch, shared-memory staging)
  const int modes[2] = {GF_PREFETCH_L2, GF_PREFETCH_SMEM};
  const int nmodes = c->fp64 ? 1 : 2;
  for (int m = 0; m < nmodes && !r; ++m) {
    const int mode = c->fp64 ? c->prefetch : modes[m];
    for (int lpt : cands) {
      r = full_sweep(c, kalgo, algo, param, 1, lpt, false, mode);  // warm-up
      if (r) break;
      const int reps = 3;
      cudaEventRecord(e0, c->st);
      for (int k = 0; k < reps && !r; ++k) r = full_sweep(c, kalgo, algo, param, 1, lpt, false, mode);
      cudaEventRecord(e1, c->st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (!r && ms < best_ms) {
        best_ms = ms;
        best = lpt;
        best_mode = mode;
      }
      cudaMemcpyAsync(c->links(), backup, bytes, cudaMemcpyDeviceToDevice, c->st);
    }
  }
  cudaStreamSynchronize(c->st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(backup);
  c->sweep_index = idx0;
  if (!r) r = read_sweep_error(c);
  if (r) return r;
  c->lpt[c->fp64][algo] = best;
  c->pmode[c->fp64][algo] = best_mode + 1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[std::make_tuple(c->device, c->gauge, (int)c->fp64, (int)algo,
                            volume_class((uint64_t)c->G.V * (uint64_t)c->ncopies))] = Tuned{best, best_mode};
  }
  if (best_lpt) *best_lpt = best;
  if (ms_best) *ms_best = best_ms;
  return GF_OK;
}

// One JSON line per convergence check (gf_set_check_log).
void log_check(gf_ctx* c, const char* call, int check, int sweeps, double worst, double theta_mean, double F_mean,
               int active, double seconds) {
  if (!c->check_log) return;
  fprintf(c->check_log,
          "{\"call\": \"%s\", \"check\": %d, \"sweeps\": %d, \"storage\": \"%s\", \"theta_worst\": %.6e, "
          "\"theta_mean\": %.6e, \"F_mean\": %.15f, \"active_units\": %d, \"seconds\": %.6f}\n",
          call, check, sweeps, c->fp64 ? "fp64" : "fp32", worst, theta_mean, F_mean, active, seconds);
  fflush(c->check_log);
}

int gf_fix(gf_ctx* c, const gf_fix_params* P, gf_fix_result* res) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_not_slab(c, "gf_fix"))) return r;
  if (!P) return fail(GF_EINVAL, "params is NULL");
  if (P->algo != GF_OR && P->algo != GF_RELAX) return fail(GF_EINVAL, "gf_fix runs GF_OR or GF_RELAX");
  if ((r = check_algo_param(P->algo, P->param))) return r;
  if (!(P->theta_target > 0)) return fail(GF_EINVAL, "theta_target must be > 0");
  if (P->max_sweeps < 0 || P->check_interval < 1 || P->reunit_interval < 0)
    return fail(GF_EINVAL, "bad sweep counts");
  Range range_fix("gf_fix");
  const auto t_start = std::chrono::steady_clock::now();
  gf_fix_result R;
  memset(&R, 0, sizeof R);
  const int Nt = c->dims[0];
  const int units_per_copy = c->gauge == GF_COULOMB ? Nt : 1;
  const uint64_t sites_per_unit = c->gauge == GF_COULOMB ? c->G.V3 : c->G.V;
  std::vector<double> ct;
  std::vector<double> unit_theta((size_t)c->ncopies * units_per_copy);
  double best_fp32 = INFINITY;
  int best_at = 0;  // sweep count when the FP32 stage last improved theta
  // adaptive checks: theta falls geometrically in the tail, so after two
  // checks the next one is scheduled near the predicted crossing
  double prev_worst = -1.0;
  int prev_sweeps = 0;
  bool fused_ready = false;  // the last sweep's odd half wrote F/theta of its sites
  int since_reunit = 0;
  for (;;) {
    // theta after the last sweep: fused into its odd half when nothing has
    // touched the links since, else the standalone pass
    {
      Range range_check("check");
      if ((r = (fused_ready && c->fused_obs) ? fused_observables(c, ct) : observables(c, ct))) return r;
    }
    fused_ready = false;
    R.checks++;
    // theta per unit: a copy (Landau/MAG, mean over slices) or a time-slice (Coulomb)
    double worst = 0;
    int n_active = 0;
    for (int k = 0; k < c->ncopies; ++k) {
      if (c->gauge == GF_COULOMB) {
        for (int t = 0; t < Nt; ++t) unit_theta[(size_t)k * Nt + t] = ct[2 * ((size_t)k * Nt + t) + 1];
      } else {
        double s = 0;
        for (int t = 0; t < Nt; ++t) s += ct[2 * ((size_t)k * Nt + t) + 1];
        unit_theta[k] = s / Nt;
      }
    }
    {  // what the result reports about the last evaluation
      double fs = 0, tm = 0;
      for (int k = 0; k < c->ncopies; ++k)
        for (int t = 0; t < Nt; ++t) fs += ct[2 * ((size_t)k * Nt + t)];
      for (double th : unit_theta) tm = std::max(tm, th);
      R.F_mean = fs / ((double)c->ncopies * Nt);
      R.theta_max = tm;
    }
    const bool final_phase = c->fp64 || c->prec == GF_FP32 || c->prec == GF_MP;
    for (int k = 0; k < c->ncopies; ++k)
      for (int u = 0; u < units_per_copy; ++u) {
        const double th = unit_theta[(size_t)k * units_per_copy + u];
        const bool done = final_phase && th < P->theta_target;
        const int v = done ? 0 : 1;
        if (c->gauge == GF_COULOMB) {
          c->active_h[(size_t)k * Nt + u] = v;
        } else {
          for (int t = 0; t < Nt; ++t) c->active_h[(size_t)k * Nt + t] = v;
        }
        if (v) {
          n_active++;
          worst = std::max(worst, th);
        }
      }
    if (c->check_log) {
      double Fm = 0, Tm = 0;
      int nu = 0;
      for (int k = 0; k < c->ncopies; ++k)
        for (int t = 0; t < Nt; ++t) Fm += ct[2 * ((size_t)k * Nt + t)];
      for (size_t u = 0; u < unit_theta.size(); ++u)
        if (c->gauge == GF_COULOMB ? c->active_h[u] : c->active_h[u * Nt]) {
          Tm += unit_theta[u];
          ++nu;
        }
      log_check(c, "gf_fix", R.checks, R.sweeps, worst, nu ? Tm / nu : 0.0, Fm / ((double)c->ncopies * Nt), n_active,
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
    }
    if ((r = upload_active(c))) return r;
    if (n_active == 0) {
      R.converged = 1;
      break;
    }
    if (R.sweeps >= P->max_sweeps) break;
    if (!c->fp64 && c->prec == GF_MIXED) {
      // switch below switch_theta, or once FP32 has stopped improving theta
      // (its rounding floor) for 25 consecutive checks
      if (worst < best_fp32) {
        best_fp32 = worst;
        best_at = R.sweeps;
      }
      // FP32 "stalls" only near its rounding floor: far above it, slow progress
      // (MAG) is just slow convergence, and FP32 sweeps are the faster way on
      const bool stalled = worst < std::max(100.0 * P->switch_theta, 1e-9) &&
                           R.sweeps - best_at >= 25 * P->check_interval;
      if (worst < P->switch_theta || stalled || !std::isfinite(worst)) {
        Range range_promote("switch to FP64");
        if ((r = promote(c))) return r;
        prev_worst = -1.0;
        continue;  // re-evaluate theta in FP64 (standalone pass)
      }
    }
    const double thr = (!c->fp64 && c->prec == GF_MIXED) ? P->switch_theta : P->theta_target;
    int k = P->check_interval;
    if (prev_worst > 0 && worst < prev_worst && worst > thr && R.sweeps > prev_sweeps) {
      const double rate = std::log(prev_worst / worst) / (double)(R.sweeps - prev_sweeps);
      const double need = std::log(worst / thr) / rate;
      k = (int)std::min<double>(10.0 * P->check_interval, std::max<double>(P->check_interval, 0.7 * need));
    }
    prev_worst = worst;
    prev_sweeps = R.sweeps;
    k = std::min(k, P->max_sweeps - R.sweeps);
    const int kalgo = gfk::ALG_OR;
    const double omega = P->algo == GF_RELAX ? 1.0 : P->param;
    for (int done = 0; done < k;) {
      // up to the next re-unitarisation or the end of the interval, whose
      // last sweep writes the fused observables
      const int seg = std::min(k - done, P->reunit_interval > 0 ? P->reunit_interval - since_reunit : k - done);
      const bool has_last = done + seg == k;
      Range range_sweeps(c->fp64 ? "sweeps fp64" : "sweeps fp32");
      if ((r = plain_sweeps(c, kalgo, P->algo, omega, has_last ? seg - 1 : seg))) return r;
      if (has_last) {
        // the MP kernels have no fused-observables variant: the check reads the links
        const bool fuse = c->prec != GF_MP;
        if ((r = full_sweep(c, kalgo, P->algo, omega, 0, 0, fuse))) return r;
        fused_ready = fuse;
      }
      R.site_updates += (uint64_t)seg * n_active * sites_per_unit;
      if (c->fp64)
        R.sweeps_fp64 += seg;
      else
        R.sweeps_fp32 += seg;
      done += seg;
      // re-unitarise (FP32, FP64) or apply the accumulated transformation to
      // the FP64 master (GF_MIXED's FP32 stage) every reunit_interval sweeps
      since_reunit += seg;
      if (P->reunit_interval > 0 && since_reunit >= P->reunit_interval) {
        since_reunit = 0;
        if ((r = reunitarize(c))) return r;
        fused_ready = false;  // the links changed after the fused half-sweep
      }
    }
    R.sweeps += k;
  }
  // leave every unit active for later calls
  std::fill(c->active_h.begin(), c->active_h.end(), 1);
  if ((r = upload_active(c))) return r;
  R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (res) *res = R;
  if (!R.converged) return fail(GF_ENOTCONV, "theta_target not reached in %d sweeps", R.sweeps);
  return GF_OK;
}

int gf_protocol(gf_ctx* c, const gf_protocol_params* P, gf_fix_result* res) {
  int r = check_ctx(c);
  if (r) return r;
  if ((r = check_not_slab(c, "gf_protocol"))) return r;
  if (!P) return fail(GF_EINVAL, "params is NULL");
  if (P->sa_steps < 0 || P->sr_sweeps < 0) return fail(GF_EINVAL, "negative sweep counts");
  if (P->sa_steps > 0 && (!(P->T_start > 0) || !(P->T_end > 0))) return fail(GF_EINVAL, "temperatures must be > 0");
  if (P->sr_sweeps > 0 && (r = check_algo_param(GF_SR, P->sr_p))) return r;
  const auto t_start = std::chrono::steady_clock::now();
  gf_fix_result R;
  memset(&R, 0, sizeof R);
  const uint64_t sites = (uint64_t)c->ncopies * c->G.V;
  // 1. simulated annealing: heat bath + three microcanonical sweeps per step,
  //    T linear from T_start to T_end (Sec. 2.3)
  Range range_protocol("gf_protocol");
  {
    Range range_sa("simulated annealing");
    for (int k = 0; k < P->sa_steps; ++k) {
      const double T = P->sa_steps > 1 ? P->T_start + (P->T_end - P->T_start) * k / (double)(P->sa_steps - 1)
                                       : P->T_start;
      if ((r = api_sweep(c, GF_SA, T, P->seed))) return r;
      const int per_step = 1 + c->sa_micro;
      R.sweeps += per_step;
      R.site_updates += (uint64_t)per_step * sites;
      if (c->prec != GF_FP64 && !c->fp64) {
        R.sweeps_fp32 += per_step;
        if (P->fix.reunit_interval > 0 && (k + 1) * per_step % P->fix.reunit_interval < per_step &&
            (r = reunitarize(c)))
          return r;
      } else {
        R.sweeps_fp64 += per_step;
      }
    }
  }
  // 2. stochastic relaxation until every copy has theta < sr_theta or
  //    sr_sweeps have run (Sec. 2.2.5, Sec. 6.5)
  int done = 0;
  std::vector<double> ct;
  std::vector<double> Fc(c->ncopies), Tc(c->ncopies);
  // a copy leaves the SR phase at the first check with theta < sr_theta, so a
  // copy's trajectory is the same alone and in a batch
  const int Nt = c->dims[0];
  Range range_sr("stochastic relaxation");
  while (done < P->sr_sweeps) {
    if ((r = observables(c, ct))) return r;
    R.checks++;
    copy_means(c, ct, Fc.data(), Tc.data());
    if (c->check_log) {
      double Fm = 0, Tm = 0, Tw = 0;
      int na = 0;
      for (int k = 0; k < c->ncopies; ++k) {
        Fm += Fc[k];
        if (c->active_h[(size_t)k * Nt] && Tc[k] >= P->sr_theta) {
          Tm += Tc[k];
          Tw = std::max(Tw, Tc[k]);
          ++na;
        }
      }
      log_check(c, "gf_protocol", R.checks, R.sweeps_fp32 + R.sweeps_fp64, Tw, na ? Tm / na : 0.0,
                Fm / c->ncopies, na, std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
    }
    int n_active = 0;
    for (int k = 0; k < c->ncopies; ++k) {
      const int v = (c->active_h[(size_t)k * Nt] && Tc[k] >= P->sr_theta) ? 1 : 0;
      for (int t = 0; t < Nt; ++t) c->active_h[(size_t)k * Nt + t] = v;
      n_active += v;
    }
    if ((r = upload_active(c))) return r;
    if (n_active == 0) break;
    const int k = std::min(P->fix.check_interval > 0 ? P->fix.check_interval : 10, P->sr_sweeps - done);
    for (int i = 0; i < k; ++i) {
      if ((r = api_sweep(c, GF_SR, P->sr_p, P->seed))) return r;
      if (c->prec != GF_FP64 && !c->fp64) {
        R.sweeps_fp32++;
        if (P->fix.reunit_interval > 0 && (R.sweeps_fp32 % P->fix.reunit_interval) == 0 && (r = reunitarize(c)))
          return r;
      } else {
        R.sweeps_fp64++;
      }
    }
    done += k;
    R.sweeps += k;
    R.site_updates += (uint64_t)k * n_active * c->G.V;
  }
  std::fill(c->active_h.begin(), c->active_h.end(), 1);
  if ((r = upload_active(c))) return r;
  // 3. overrelaxation to theta_target
  gf_fix_result F;
  r = gf_fix(c, &P->fix, &F);
  R.sweeps += F.sweeps;
  R.sweeps_fp32 += F.sweeps_fp32;
  R.sweeps_fp64 += F.sweeps_fp64;
  R.checks += F.checks;
  R.site_updates += F.site_updates;
  R.converged = F.converged;
  R.F_mean = F.F_mean;
  R.theta_max = F.theta_max;
  R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (res) *res = R;
  return r;
}

int gf_set_profiling(gf_ctx* c, int on) {
  int r = check_ctx(c);
  if (r) return r;
  GF_CUDA(cudaStreamSynchronize(c->st));
  prof_collect(c);
  c->profiling = on != 0;
  for (int k = 0; k < GF_KERNEL_KINDS; ++k) {
    c->prof_launches[k] = 0;
    c->prof_ms[k] = 0;
  }
  return GF_OK;
}

int gf_launch_count(gf_ctx* c, uint64_t* n) {
  int r = check_ctx(c);
  if (r) return r;
  if (!n) return fail(GF_EINVAL, "n is NULL");
  *n = c->launch_count;
  return GF_OK;
}

int gf_kernel_stats(gf_ctx* c, int kind, uint64_t* launches, double* total_ms) {
  int r = check_ctx(c);
  if (r) return r;
  if (kind < 0 || kind >= GF_KERNEL_KINDS) return fail(GF_EINVAL, "bad kernel kind %d", kind);
  GF_CUDA(cudaStreamSynchronize(c->st));
  prof_collect(c);
  if (launches) *launches = c->prof_launches[kind];
  if (total_ms) *total_ms = c->prof_ms[kind];
  return GF_OK;
}

int gf_get_info(gf_ctx* c, int dims[4], int* n_copies, int* gauge, int* precision, int* storage_fp64) {
  int r = check_ctx(c);
  if (r) return r;
  if (dims) memcpy(dims, c->dims, sizeof c->dims);
  if (n_copies) *n_copies = c->ncopies;
  if (gauge) *gauge = c->gauge;
  if (precision) *precision = c->prec;
  if (storage_fp64) *storage_fp64 = c->fp64;
  return GF_OK;
}

int gf_philox(uint64_t seed, const uint32_t* counters, size_t n, uint32_t* out) {
  if (n == 0) return GF_OK;
  if (!counters || !out) return fail(GF_EINVAL, "NULL array");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(GF_ENOSYS, "no CUDA device available");
  }
  void *dc = nullptr, *dout = nullptr;
  const size_t bytes = n * 4 * sizeof(uint32_t);
  if (cudaMalloc(&dc, bytes) != cudaSuccess || cudaMalloc(&dout, bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dc);
    return fail(GF_ENOMEM, "gf_philox: %zu bytes", 2 * bytes);
  }
  int r = GF_OK;
  cudaError_t e = cudaMemcpy(dc, counters, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = gfk::launch_philox(dc, dout, n, seed, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) r = fail(GF_ECUDA, "gf_philox: %s", cudaGetErrorString(e));
  cudaFree(dc);
  cudaFree(dout);
  return r;
}

const char* gf_strerror(int status) {
  switch (status) {
    case GF_OK: return "GF_OK";
    case GF_EINVAL: return "GF_EINVAL: invalid argument";
    case GF_ENOMEM: return "GF_ENOMEM: out of device memory";
    case GF_ECUDA: return "GF_ECUDA: CUDA error";
    case GF_ETIMEOUT: return "GF_ETIMEOUT: bounded wait expired";
    case GF_ENOTCONV: return "GF_ENOTCONV: not converged";
    case GF_ENOSYS: return "GF_ENOSYS: no CUDA device";
    case GF_ECANCELED: return "GF_ECANCELED: job canceled";
  }
  return "unknown status";
}

const char* gf_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
