/*
 * gf.h -- C ABI of the GB300 lattice gauge-fixing library (libgf.so).
 *
 * The library implements the checkerboard relaxation family of Schroeck &
 * Vogt, "Coulomb, Landau and Maximally Abelian Gauge Fixing in Lattice QCD
 * with Multi-GPUs" (arXiv:1212.5221): the gauge functionals and the gauge
 * precision theta of Sec. 2.1, the local SU(2)-subgroup updates of Sec. 2.2
 * (relaxation, overrelaxation, microcanonical, stochastic relaxation), the
 * simulated annealing of Sec. 2.3 and the sweep of Alg. 1 (Sec. 2.4), on one
 * GPU.
 *
 * Conventions for every entry point:
 *  - The return value is a status code (GF_OK = 0 or one of the GF_E*
 *    codes below); gf_strerror() names it and gf_last_error() gives the
 *    message of the calling thread's last failure.  No C++ exception crosses
 *    this interface.
 *  - dims = {Nt, Nx, Ny, Nz}: every extent even and >= 2, periodic
 *    boundaries, mu = 0 the temporal direction.  A site's index is
 *    s = ((t*Nx + x)*Ny + y)*Nz + z; its parity is (t+x+y+z) mod 2.
 *  - Host link arrays use the natural "StandardPattern" order of Sec. 4.2.1:
 *    t, x, y, z, mu, i, j, re/im -- 18 doubles per link, 72*V doubles per
 *    lattice.  Host pointers are borrowed for the duration of the call only.
 *  - A context owns n_copies independent lattices of the same extents (a
 *    batch of Gribov copies, Sec. 1 and 6.6).  Every F / theta output is an
 *    array of n_copies doubles (per-slice outputs: n_copies*Nt doubles).
 *    Results are FP64 whatever the storage precision.
 *  - Work is issued on the context's CUDA stream; every call returns after
 *    its work on that stream has completed, except the *_async calls, which
 *    return once the work is enqueued (gf_synchronize waits for it).
 *  - A context must not be used from two threads at the same time.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gf_ctx gf_ctx;

/* Target gauge (Sec. 2.1): Landau sums over all four directions, Coulomb over
 * the spatial ones with every time-slice an independent problem, MAG is the
 * maximally Abelian gauge of Eq. MAG_functional. */
typedef enum { GF_LANDAU = 0, GF_COULOMB = 1, GF_MAG = 2 } gf_gauge;

/* Storage/arithmetic precision.  GF_MIXED keeps an FP64 master copy of the
 * links and runs the bulk of the sweeps on an FP32 working copy (12 reals,
 * Sec. 4.2) that also accumulates every site's gauge transformation g(x);
 * the accumulated g, re-unitarised in FP64, is applied to the FP64 master
 * (U_mu(x) <- g(x) U_mu(x) g(x+mu)^dag) every re-unitarisation interval and
 * whenever the links are read, and the FP32 copy is re-rounded from it, so
 * the master never leaves the gauge orbit of the input.  The final sweeps
 * run on the FP64 master (gf_promote / gf_fix).  Reductions are always FP64.
 * GF_MP is the paper's mixed precision "MP" (Sec. 4.5): links stored in FP32
 * (12 reals), the local update (Step 1 of Alg. 1: the gathered K or MAG
 * vector, the subgroup choices and their product) computed in FP64 from
 * them, and its application to the links (Step 2) in FP32; it has no FP64
 * copy and no switch.  Its convergence checks read the links in a separate
 * FP64 pass (no fused variant). */
typedef enum { GF_FP64 = 0, GF_FP32 = 1, GF_MIXED = 2, GF_MP = 3 } gf_precision;

/* Local update (Step 1 of Alg. 1): relaxation (Eq. localsolution per SU(2)
 * subgroup), overrelaxation g -> g^omega to first order (Sec. 2.2.3, in
 * the form of App. A), microcanonical g -> g^2 (Sec. 2.2.4),
 * stochastic relaxation (Sec. 2.2.5), simulated-annealing heat bath
 * (Sec. 2.3). */
typedef enum { GF_RELAX = 0, GF_OR = 1, GF_MICRO = 2, GF_SR = 3, GF_SA = 4 } gf_algo;

enum {
  GF_OK = 0,
  GF_EINVAL = 1,     /* bad argument: odd/zero extent, bad enum, omega not in [1,2], T <= 0, ... */
  GF_ENOMEM = 2,     /* device memory could not be allocated, or an external buffer is too small */
  GF_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  GF_ETIMEOUT = 4,   /* a bounded wait expired */
  GF_ENOTCONV = 5,   /* gf_fix: the sweep limit was reached before theta_target */
  GF_ENOSYS = 6,     /* the library was built without a usable CUDA device */
  GF_ECANCELED = 7   /* a served job removed from the queue by gf_server_cancel */
};

/* Bytes of device memory a context needs (links in the storage layout,
 * reduction scratch, slice flags and a bounded host-transfer staging area).
 * Used for admission by HBM footprint and to size gf_create_ext buffers. */
int gf_footprint(const int dims[4], int n_copies, gf_gauge gauge, gf_precision prec, size_t* bytes);

/* Create a context with one lattice (n_copies = 1).  stream: a cudaStream_t
 * to issue work on, or NULL for a stream the context creates and owns.  The
 * links start as the unit field. */
int gf_create(const int dims[4], gf_gauge gauge, gf_precision prec, void* stream, gf_ctx** out);

/* Create a context with n_copies independent lattices (batched launches). */
int gf_create_batch(const int dims[4], int n_copies, gf_gauge gauge, gf_precision prec, void* stream,
                    gf_ctx** out);

/* As gf_create_batch, but all device storage is carved out of device_buf
 * (at least gf_footprint bytes, 256-byte aligned, owned by the caller, e.g. a
 * PyTorch tensor); the context allocates no device memory. */
int gf_create_ext(const int dims[4], int n_copies, gf_gauge gauge, gf_precision prec, void* stream,
                  void* device_buf, size_t bytes, gf_ctx** out);

/* Release the context and the device memory it allocated. NULL is ignored. */
void gf_destroy(gf_ctx* ctx);

/* Load links from host memory (StandardPattern, 72*V doubles) into copy
 * `copy`, or into every copy when copy = -1.  The first two rows of each
 * link are kept (12-real storage, Sec. 4.2); the third is rebuilt on use.
 * For Coulomb the accumulated time-slice gauge transformation is reset. */
int gf_load_links(gf_ctx* ctx, int copy, const double* host);

/* As gf_load_links for the time-slices [t0, t0+nt) only; host holds
 * nt*Nx*Ny*Nz*4*18 doubles.  Lets very large lattices stream in slab by slab. */
int gf_load_links_slab(gf_ctx* ctx, int copy, int t0, int nt, const double* host);

/* As gf_load_links, from device memory in the same natural order. */
int gf_load_links_device(gf_ctx* ctx, int copy, const double* device_src);

/* Store the links of copy `copy` to host memory (StandardPattern, full 3x3,
 * third row rebuilt as conj(row0 x row1)).  For Coulomb the accumulated
 * time-slice transformation is first folded into the temporal links,
 * U_0(x) <- g(x) U_0(x) g(x+0)^dag (Sec. 5.1). */
int gf_store_links(gf_ctx* ctx, int copy, double* host);

/* As gf_store_links for the time-slices [t0, t0+nt) only (host holds
 * nt*Nx*Ny*Nz*4*18 doubles). */
int gf_store_links_slab(gf_ctx* ctx, int copy, int t0, int nt, double* host);

/* As gf_store_links, to device memory. */
int gf_store_links_device(gf_ctx* ctx, int copy, double* device_dst);

/* Random gauge transformation U_mu(x) <- g(x) U_mu(x) g(x+mu)^dag with
 * Haar-random g(x) in SU(3) (a random point on the gauge orbit, Sec. 6.5):
 * g(x) is drawn from Philox4x32-10 keyed by the seed and counted by (site,
 * copy), so every copy gets a different transformation. */
int gf_random_gauge_transform(gf_ctx* ctx, uint64_t seed);

/* n_sweeps checkerboard sweeps (Alg. 1: even sublattice, then odd; per site
 * the subgroups (0,1), (0,2), (1,2)) over every active unit.  param: omega in
 * [1,2] for GF_OR (GF_RELAX ignores it and uses 1), the probability p in
 * [0,1] for GF_SR, the temperature T > 0 for GF_SA, unused for GF_MICRO.
 * GF_SA: every sweep is one heat-bath sweep followed by three microcanonical
 * sweeps (Sec. 2.3; the count is set by gf_set_sa_micro).  Random draws are
 * keyed by (seed, site, sweep index, copy); the context's sweep index
 * advances by one per sweep (1 + the microcanonical count per SA sweep).  F
 * and theta (may be NULL) receive the exact values after the sweeps, per
 * copy. */
int gf_sweep(gf_ctx* ctx, gf_algo algo, double param, int n_sweeps, uint64_t seed, double* F,
             double* theta);

/* Simulated annealing: n_steps heat-bath sweeps with T falling linearly from
 * T0 to T1, each followed by three microcanonical sweeps (Sec. 2.3). */
int gf_anneal(gf_ctx* ctx, double T0, double T1, int n_steps, uint64_t seed, double* F, double* theta);

/* Microcanonical sweeps after every heat-bath sweep of GF_SA, gf_anneal and
 * gf_protocol: 3 by default, as in Sec. 2.3 ("three microcanonical steps
 * after each change in temperature"); 0 runs the heat bath alone (the form
 * its per-sweep parity is checked in).  GF_EINVAL outside [0, 64]. */
int gf_set_sa_micro(gf_ctx* ctx, int n_micro);

/* Diagnostic record of the Landau/Coulomb heat bath's accept/reject
 * decisions (Kennedy-Pendleton, Sec. 2.3): while set, every heat-bath
 * half-sweep writes, for each updated site and subgroup, the number of
 * trials it took (1..64; 0 when none was accepted and the relaxation value
 * was kept; always 1 for MAG, whose sampler has no rejection step).
 *   device_counts  int32 device memory of n_copies*V*3 entries, layout
 *                  [copy][lexicographic site][subgroup]; owned by the caller,
 *                  who keeps it alive while it is set; NULL turns the record
 *                  off.  Entries of sites not updated are left as they were.
 * GF_EINVAL if the pointer is not 4-byte aligned. */
int gf_set_sa_trace(gf_ctx* ctx, int* device_counts);

/* ---- Time-slab decomposition of one Landau or MAG lattice (Sec. 5) -------
 * The lattice is split along t into slabs of nt consecutive time-slices, one
 * per process (one GPU each).  A site's update reads U_0(x - 0) from the
 * slice below it, so a process also keeps a copy of the slice below its slab
 * and, after every half-sweep, exchanges with its two ring neighbours the
 * temporal links on the slab boundaries that the half-sweep changed
 * (Sec. 5.1): each message is U_0, rows 0 and 1, of the sites of one parity
 * of one slice, 1/12 of a time-slice (Sec. 5.2).  Communication is the
 * caller's (the Python module paper_1212_5221_gb300.slab runs the schedule
 * over torch.distributed); these calls do the device part.
 *
 * gf_set_slab turns a context of local dims (nt + 2, Nx, Ny, Nz), n_copies 1,
 * GF_LANDAU or GF_MAG, GF_FP64 or GF_FP32 storage, into the slab owning the
 * global time-slices [t0, t0 + nt) of a lattice with Nt_global slices (even,
 * >= nt): local slice 0 holds global slice t0 - 1 (mod Nt_global), local
 * slices 1 .. nt the owned ones, local slice nt + 1 is never read.  Load the
 * context with those nt + 2 global slices (natural order) by gf_load_links.
 * Random draws then use global site indices, so every slab draws what the
 * whole lattice would.  Whole-lattice sweeps (gf_sweep, gf_fix, gf_anneal,
 * gf_protocol and their _async forms) and gf_random_gauge_transform return
 * GF_EINVAL on a slab.  GF_EINVAL for any other shape, gauge or storage. */
int gf_set_slab(gf_ctx* ctx, int t0, int Nt_global);

/* Which owned slices gf_sweep_half updates. */
enum { GF_SLAB_OWNED = 0, GF_SLAB_BOUNDARY = 1, GF_SLAB_INNER = 2 };

/* One half-sweep (Alg. 1 for the sites of one parity): the sites of GLOBAL
 * parity `parity` of the owned slices (part GF_SLAB_OWNED), of the first and
 * last owned slice only (GF_SLAB_BOUNDARY), or of the others
 * (GF_SLAB_INNER), so that the boundary can be updated and sent while the
 * inner slices run (Sec. 5.3).  On a context that is not a slab, part must
 * be GF_SLAB_OWNED and the whole lattice is swept.  algo/param as gf_sweep,
 * except that GF_SA is the heat bath alone.  Draws use the context's sweep
 * index, which this call leaves unchanged (advance it with
 * gf_set_sweep_index once both halves are done).  Enqueued on the context's
 * stream; returns without waiting.  In FP64 storage each launch covers only
 * its part's sites (GF_SLAB_BOUNDARY: one launch per boundary slice), spread
 * over the whole grid; FP32 launches cover the slab and skip other slices. */
int gf_sweep_half(gf_ctx* ctx, gf_algo algo, double param, int parity, int part, uint64_t seed);

/* Bytes of one boundary message: 3 (FP32) or 6 (FP64) x Nx*Ny*Nz/2 x 16. */
int gf_slab_bytes(gf_ctx* ctx, size_t* bytes);

/* Copy U_0 (rows 0 and 1, as stored) of the sites of global parity `parity`
 * in local time-slice `slice` into buf (gf_slab_pack) or from buf into the
 * links (gf_slab_unpack).  buf: gf_slab_bytes bytes of device or host memory
 * owned by the caller, layout [chunk][site of that parity in the slice].
 * Enqueued on the context's stream (synchronise before reading buf on the
 * host).  GF_EINVAL for a slice outside [0, local Nt) or a GF_MIXED context
 * in its FP32 stage. */
int gf_slab_pack(gf_ctx* ctx, int slice, int parity, void* buf);
int gf_slab_unpack(gf_ctx* ctx, int slice, int parity, const void* buf);

/* Re-unitarise every stored matrix in FP64: normalise row 0, Gram-Schmidt
 * row 1, normalise; row 2 = conj(row0 x row1) (Sec. 4.5, reprojection). */
int gf_reunitarize(gf_ctx* ctx);

/* Exact FP64 gauge functional and theta per copy (Sec. 2.1).  Coulomb: the
 * means over time-slices of F_t and theta_t. */
int gf_functional_theta(gf_ctx* ctx, double* F, double* theta);

/* Per time-slice F_t and theta_t, arrays of n_copies*Nt (copy-major). */
int gf_slice_functional_theta(gf_ctx* ctx, double* F_t, double* theta_t);

/* GF_MIXED: end the FP32 stage: apply its pending gauge transformation to
 * the FP64 master and run later sweeps on the master.  No-op when the sweeps
 * already run in FP64; GF_EINVAL for other precisions. */
int gf_promote(gf_ctx* ctx);

/* Mark which units take part in sweeps: n_copies*Nt flags (copy-major, one
 * per time-slice); NULL makes every unit active.  For Landau and MAG a copy
 * is swept only if all of its flags are set. */
int gf_set_active(gf_ctx* ctx, const int* flags);

/* Sweep index used to key the random draws (checkpoint / resume). */
int gf_get_sweep_index(gf_ctx* ctx, uint64_t* index);
int gf_set_sweep_index(gf_ctx* ctx, uint64_t index);

/* Philox copy id of the context's copy 0 (default 0): copy k draws with id
 * base + k, so a lattice fixed alone reproduces its run inside a batch. */
int gf_set_copy_base(gf_ctx* ctx, uint32_t base);

/* Links per thread of the sweep kernels: 1, 2, 4 or 8 (8/lpt threads share a
 * site and combine their partial K with warp shuffles); 0 = the tuned
 * default.  gf_autotune times the four on a scratch copy of the links and
 * keeps the fastest for each (precision, algorithm) it is asked about. */
int gf_set_links_per_thread(gf_ctx* ctx, int lpt);

/* The sweep kernels run a persistent grid over tiles of sites; while a block
 * processes one tile, its next tile is fetched:
 *   GF_PREFETCH_NONE  not at all;
 *   GF_PREFETCH_L2    into L2 by bulk prefetches (the default);
 *   GF_PREFETCH_SMEM  FP32 storage: into one of two shared-memory buffers by
 *                     bulk asynchronous copies completing on an mbarrier, from
 *                     which the tile is then processed (FP64 storage falls
 *                     back to GF_PREFETCH_L2).  A wait for a buffer is bounded
 *                     (about 2 s); if one runs out, the kernel stops, records
 *                     it, and the next call that reads results back returns
 *                     GF_ETIMEOUT.
 * Results do not depend on the mode.  GF_EINVAL for any other value. */
enum { GF_PREFETCH_NONE = 0, GF_PREFETCH_L2 = 1, GF_PREFETCH_SMEM = 2 };
int gf_set_prefetch(gf_ctx* ctx, int mode);

/* Polls of a GF_PREFETCH_SMEM staging wait before it gives up: polls < 0
 * restores the default (2^24 polls, about 2 s); polls = 0 makes the first
 * wait of every block run out at once.  The latter exists to exercise the
 * timeout path: the blocks then wait (bounded) for the copies they issued,
 * return without updating their tiles, and the next call that reads results
 * back reports GF_ETIMEOUT; the context stays usable. */
int gf_set_stage_wait_polls(gf_ctx* ctx, int polls);

/* Asynchronous forms of gf_sweep (without F/theta), gf_anneal and
 * gf_random_gauge_transform: the work is enqueued on the context's stream
 * and the call returns without waiting for it (argument errors are still
 * returned at once).  No host buffer is involved.  gf_synchronize waits for
 * everything enqueued on the context and returns GF_ECUDA for a device error
 * or GF_ETIMEOUT for a shared-memory staging wait that ran out.  Every
 * synchronous call of the context orders after the enqueued work.  A context
 * must not be used from two threads at once. */
int gf_sweep_async(gf_ctx* ctx, gf_algo algo, double param, int n_sweeps, uint64_t seed);
int gf_anneal_async(gf_ctx* ctx, double T0, double T1, int n_steps, uint64_t seed);
int gf_random_gauge_transform_async(gf_ctx* ctx, uint64_t seed);
int gf_synchronize(gf_ctx* ctx);

/* Plain overrelaxation/relaxation sweeps of gf_sweep and gf_fix (those with
 * no observables) run in blocks of 16 captured once per launch configuration
 * as a CUDA graph and replayed (on by default; off: every kernel is launched
 * directly; also off while profiling).  The kernels and their arguments are
 * the same either way, and so are the results.  The graphs are captured on
 * the context's stream in thread-local capture mode. */
int gf_set_graphs(gf_ctx* ctx, int on);

/* Append one JSON line per convergence check of gf_fix and gf_protocol to
 * the file at path (created if missing): the call, the check number, sweeps
 * so far, the storage the sweeps ran on ("fp32" / "fp64"), the worst and the
 * mean theta of the units still active, the mean F, the number of active
 * units and the elapsed seconds.  path NULL stops logging.  GF_EINVAL if the
 * file cannot be opened. */
int gf_set_check_log(gf_ctx* ctx, const char* path);

/* F and theta fused into the sweeps (on by default): the odd half of the last
 * overrelaxation/relaxation sweep -- in which every link is written exactly
 * once -- also sums F over the links it writes and theta of its sites from
 * K(x) = sum of the updated links, in FP64; a read-only pass of the sweep
 * kernel gathers K at the even sites; the per-site values are added per
 * (copy, time-slice) in a fixed order.  Used by gf_fix's checks and by
 * gf_sweep(GF_OR / GF_RELAX) when F or theta is requested.  Off: the
 * standalone observables pass (same values up to summation order). */
int gf_set_fused_observables(gf_ctx* ctx, int on);
int gf_get_links_per_thread(gf_ctx* ctx, int* lpt);
/* Time each links-per-thread choice (and, for FP32 storage, both the L2
 * prefetch and the shared-memory staging of tiles) on a scratch copy of the
 * links, restore them, and keep the fastest for (storage precision, algo).
 * A later gf_set_prefetch replaces the tuned tile fetch. */
int gf_autotune(gf_ctx* ctx, gf_algo algo, int* best_lpt, double* ms_per_sweep_best);
/* The choice is also kept for the process, per (CUDA device current at
 * creation, gauge, storage precision, algorithm, lattice class =
 * floor(log2(sites x copies))): contexts created later on the same device
 * start from it (a job server tunes each class once). */

/* Drive the sweeps to theta < theta_target (the while-loop of Alg. 1).
 * theta is evaluated after check_interval sweeps; once two evaluations show
 * theta falling geometrically, the next one is scheduled at 0.7 times the
 * predicted crossing of the current threshold (between 1 and 10
 * check_interval sweeps).  A unit (a copy, or for Coulomb a copy's
 * time-slice) stops as soon as its theta is below target.  The odd half of
 * the sweep before a check also sums F and theta (gf_set_fused_observables).
 * Storage is re-unitarised every reunit_interval sweeps (Sec. 4.5).
 * GF_MIXED runs FP32 sweeps until every active unit has theta < switch_theta
 * (or, once theta is below max(100 switch_theta, 1e-9), it has not improved
 * for 25 check intervals: the FP32 rounding floor), then continues on the
 * FP64 master for the final sweeps; a unit counts as converged only on FP64
 * links.  Blocks of plain sweeps are replayed as CUDA graphs
 * (gf_set_graphs). */
typedef struct {
  gf_algo algo;          /* GF_OR or GF_RELAX */
  double param;          /* omega */
  double theta_target;   /* e.g. 1e-12 */
  int max_sweeps;        /* per run; GF_ENOTCONV beyond */
  int check_interval;    /* sweeps before the first theta evaluations (the base interval), >= 1 */
  int reunit_interval;   /* every this many sweeps re-unitarise the links (GF_FP32, GF_FP64, and
                            GF_MIXED's FP64 stage) or apply the accumulated transformation to the
                            FP64 master (GF_MIXED's FP32 stage); 0 = never */
  double switch_theta;   /* GF_MIXED: FP32 -> FP64 sweeps below this theta (e.g. 1e-8) */
  uint64_t seed;         /* unused by OR/RELAX; kept for symmetry with gf_sweep */
} gf_fix_params;

typedef struct {
  int sweeps;            /* sweeps issued (the slowest unit's count) */
  int sweeps_fp32;       /* of which in FP32 storage */
  int sweeps_fp64;       /* of which in FP64 storage */
  int checks;            /* theta evaluations */
  int converged;         /* 1 if every unit reached theta_target */
  double seconds;        /* host wall time of the call */
  uint64_t site_updates; /* sum over sweeps of the sites actually updated */
  double F_mean;         /* at the last theta evaluation: the functional averaged over the copies */
  double theta_max;      /* ... and the largest theta of any unit (copy, or Coulomb time-slice) */
} gf_fix_result;

int gf_fix(gf_ctx* ctx, const gf_fix_params* params, gf_fix_result* result);

/* The annealing protocol of Sec. 6.5 for every copy of the batch: sa_steps
 * simulated-annealing steps (heat bath + three microcanonical sweeps, T
 * linear from T_start to T_end), then stochastic relaxation (probability
 * sr_p) until every copy has theta < sr_theta or sr_sweeps have run, then
 * overrelaxation to theta_target with the parameters of `fix` (gf_fix).
 * Random draws are keyed by (seed, site, sweep index, copy).  The result
 * counts every sweep (an SA step is four) and reports gf_fix's convergence;
 * gf_functional_theta then gives each copy's functional, from which the
 * best Gribov copy is chosen. */
typedef struct {
  int sa_steps;
  double T_start, T_end;
  int sr_sweeps;
  double sr_p;
  double sr_theta;
  uint64_t seed;
  gf_fix_params fix;
} gf_protocol_params;

int gf_protocol(gf_ctx* ctx, const gf_protocol_params* params, gf_fix_result* result);

/* The device Philox4x32-10 (Salmon et al., SC'11) that keys every random draw
 * of the sweeps and gauge transformations: out[4k..4k+3] = Philox(counters
 * [4k..4k+3], key = (seed low word, seed high word)) for k < n.  Host arrays;
 * the call allocates and frees its own device buffers. */
int gf_philox(uint64_t seed, const uint32_t* counters, size_t n, uint32_t* out);

/* Per-kernel timing.  With profiling on, every launch of the classes below
 * is bracketed by CUDA events on the context's stream; gf_kernel_stats
 * returns the number of launches and their summed device time since
 * profiling was (re)enabled.  gf_set_profiling resets the totals. */
enum {
  GF_KERNEL_SWEEP_FP32 = 0,   /* one half-sweep (one sublattice), FP32 storage */
  GF_KERNEL_SWEEP_FP64 = 1,   /* one half-sweep, FP64 storage */
  GF_KERNEL_OBSERVABLES = 2,  /* exact F/theta pass (both kernels) */
  GF_KERNEL_REUNITARIZE = 3,
  GF_KERNEL_OTHER = 4,        /* FP32 -> FP64 promotion */
  GF_KERNEL_KINDS = 5
};
int gf_set_profiling(gf_ctx* ctx, int on);
int gf_kernel_stats(gf_ctx* ctx, int kind, uint64_t* launches, double* total_ms);

/* Number of kernels this context has launched since it was created. */
int gf_launch_count(gf_ctx* ctx, uint64_t* n);

/* F and theta without any device allocation, for callers that cannot call
 * cudaMalloc (a serving loop confined to a device-memory pool reserved at
 * start-up, a host framework that owns every allocation, or code that must
 * not trigger the allocator's implicit synchronisation).  The paper has no
 * counterpart; this is a deployment aid.
 *   dims, gauge   as for gf_create; Nt = dims[0] <= GF_NOALLOC_MAX_NT.
 *   device_links  the links in device memory, natural order (18 doubles per
 *                 link, full 3x3, 72*V doubles), 16-byte aligned, owned by
 *                 the caller and only read.
 *   stream        the cudaStream_t to run on (NULL: the legacy default stream).
 *   F, theta      host pointers receiving the functional and theta (means
 *                 over time-slices, as gf_functional_theta for one copy).
 *   F_t, theta_t  host arrays of Nt doubles for the per-slice values, or NULL.
 * The reduction's partial sums live in one file-scope device array of about
 * 1 MiB, which every GPU that loads the library holds until the process
 * exits; the call allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).  Every call shares that array and it keeps the last
 * call's contents, so calls that overlap on the GPU race: serialise them.
 * The first call on a device looks up the array's device address (with that
 * device current), so it should come before any CUDA stream capture starts.
 * Every call, the first included, ends by copying its results to the host
 * and synchronising `stream`: it returns only once they are there.
 * Returns GF_EINVAL for sizes beyond the maximum or misaligned input. */
#define GF_NOALLOC_MAX_NT 1024
int gf_functional_theta_noalloc(const int dims[4], gf_gauge gauge, const double* device_links, void* stream,
                                double* F, double* theta, double* F_t, double* theta_t);

/* ---- Several lattices in one launch ---------------------------------------
 * A group is 1..GF_GROUP_MAX contexts of any lattice extents and copy counts,
 * one gauge, on one device (GF_FP32, GF_FP64 or GF_MIXED storage; not GF_MP,
 * not time slabs).  Every half-sweep of all members is a single persistent
 * launch over the union of their tiles (members in FP32 and in FP64 storage
 * go in one launch each), issued on the first member's stream; the other
 * members' streams are ordered before and after it with events.  Small
 * lattices, whose own launches would leave most of the GPU idle, fill it
 * together.  The paper has no counterpart (its batching is over time-slices
 * of one lattice); each member's links come out as if it had been swept
 * alone with the same links-per-thread: bit for bit in FP64 and in the
 * Landau/Coulomb form, to FP32 rounding for FP32 MAG (two separately compiled
 * kernels).
 * gf_group_sweep: n_sweeps sweeps of GF_OR (omega = param) or GF_RELAX, then
 * GF_MIXED members' FP64 masters are brought up to date; synchronous. */
#define GF_GROUP_MAX 48
int gf_group_sweep(gf_ctx* const* ctxs, int n, gf_algo algo, double param, int n_sweeps);

/* gf_fix for every member of a group: theta is evaluated per member every
 * check_interval sweeps (a fixed cadence, by the standalone FP64 pass),
 * each unit (copy or Coulomb time-slice) stops on its own, a GF_MIXED member
 * switches to its FP64 master on its own below switch_theta, and the members
 * still sweeping share the launches; re-unitarisation as in gf_fix.
 * results: n entries (may be NULL).  GF_ENOTCONV if any member did not
 * reach theta_target within max_sweeps. */
int gf_group_fix(gf_ctx* const* ctxs, int n, const gf_fix_params* params, gf_fix_result* results);

/* Job server: many gauge-fixing jobs (different lattices, gauges and
 * precisions) share the GPU.  gf_server_create reserves hbm_bytes of device
 * memory once and starts `slots` worker threads.  A submitted job waits in a
 * FIFO queue; it is admitted as soon as a slot is free and its footprint
 * (gf_footprint) fits in the arena (a job that does not fit yet lets smaller
 * jobs behind it go first, up to 4 x slots times).  Each admitted job gets its
 * own context and CUDA stream carved from the arena (no cudaMalloc), so the
 * kernels of concurrent jobs overlap; when it finishes, its slot and memory
 * go to the next job.  A job: load host_links (natural order; the caller keeps
 * the array alive until the job's result is polled), apply
 * gf_random_gauge_transform(orbit_seed) unless orbit_seed is 0, run gf_fix
 * with `fix` (or gf_protocol with `protocol` when `anneal` is set), then
 * report F/theta and, if host_out is given, store the links there.  Times
 * are seconds since the server was created. */
typedef struct gf_server gf_server;

typedef struct {
  int dims[4];
  gf_gauge gauge;
  gf_precision prec;
  const double* host_links;
  uint64_t orbit_seed;
  gf_fix_params fix;
  double* host_out;
  uint64_t tag;          /* returned with the result */
  int anneal;            /* 1: run gf_protocol with `protocol` instead of gf_fix with `fix` (simulated
                            annealing and stochastic relaxation before the overrelaxation, Sec. 6.5:
                            for MAG, whose overrelaxation alone converges slowly from a random gauge) */
  gf_protocol_params protocol;
} gf_job;

typedef struct {
  uint64_t tag;
  int status;            /* GF_OK, GF_ENOTCONV, GF_ECANCELED (gf_server_cancel), or an error code */
  double F, theta;
  int sweeps, sweeps_fp32, sweeps_fp64;
  uint64_t site_updates;
  size_t footprint;      /* arena bytes the job held */
  double t_submit, t_admit, t_done;
} gf_job_result;

int gf_server_create(size_t hbm_bytes, int slots, gf_server** out);

/* A test double with the same queue, admission and arena logic that runs
 * no device code: each job just holds its memory for seconds_per_gb per GB
 * of footprint. */
int gf_server_create_mock(size_t hbm_bytes, int slots, double seconds_per_gb, gf_server** out);

/* GF_ENOMEM if the job's footprint exceeds the whole arena. */
int gf_server_submit(gf_server* server, const gf_job* job);

/* Up to max_results finished jobs (in completion order), waiting up to
 * wait_ms for the first one; *n_out receives the number returned. */
int gf_server_poll(gf_server* server, gf_job_result* out, int max_results, int wait_ms, int* n_out);

int gf_server_status(gf_server* server, int* queued, int* running, uint64_t* completed, size_t* bytes_in_use);

/* Remove the queued (not yet admitted) jobs with this tag; each is reported
 * by gf_server_poll with status GF_ECANCELED.  A job already running runs to
 * completion.  *n_canceled receives the number removed (0 is not an error). */
int gf_server_cancel(gf_server* server, uint64_t tag, int* n_canceled);

/* Runs every queued job to completion, then releases the arena. */
void gf_server_destroy(gf_server* server);

/* Geometry and state queries. */
int gf_get_info(gf_ctx* ctx, int dims[4], int* n_copies, int* gauge, int* precision, int* storage_fp64);

/* Name of a status code, and the calling thread's last error message. */
const char* gf_strerror(int status);
const char* gf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GF_H */
