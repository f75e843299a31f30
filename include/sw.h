/*
 * sw.h -- C ABI of the GB300 Swendsen-Wang sweep library (libsw_gb300.so).
 *
 * The library advances periodic L x L lattices of the q-state Potts model
 * (Komura & Okabe, arXiv:1202.0635, Sec. 2, Eq. 1; Ising = Potts q = 2 in
 * Ising units) and of the q-state clock model (Sec. 4, Eq. clock) by the
 * Swendsen-Wang multi-cluster update (Sec. 2 steps (i)-(viii); clock: Wolff's
 * embedded clusters, Sec. 4).  Every stage of a sweep runs as a CUDA kernel
 * on the calling thread's current device:
 *   bond activation  -> tile-local cluster labeling in shared memory
 *   -> boundary merge (atomicMin union-find) -> cluster roots, per-cluster
 *   draw and spin write -> integer reductions of the observables.
 *
 * Conventions (identical, by specification, to the CPU oracle's):
 *   site i = y*L + x (row-major); site i owns the bond to (y, x+1 mod L)
 *   ("right", direction 0) and to (y+1 mod L, x) ("down", direction 1).
 *   spins are int8 states 0..q-1 (clock: angle 2*pi*k/q).
 *   Random numbers: Philox-4x32-10, key = (seed lo32, seed hi32), counter =
 *   (index, sweep lo32, tag, sweep hi32); tag 0 bonds (index i>>1, lane
 *   2*(i&1)+direction), tag 1 cluster draw of the Potts model with q > 2
 *   (index = root, lane 0, new state mulhi(u, q)), tag 2 clock mirror axis
 *   (index 0, lane 0), tag 3 random start (index i, sweep 0, lane 0), tag 4
 *   one-bit cluster draw of the q = 2 Potts / Ising new state and of the
 *   clock reflection flag (index = root >> 7; bit root & 31 of lane
 *   (root >> 5) & 3).  "sweep" counts the sweeps completed before the one
 *   drawing.  mulhi(u, q) = (u * q) >> 32.
 *   A bond is active iff its draw u < an integer threshold
 *   floor(p * 2^32) (clamped to 2^32-1), p = -expm1(-x) evaluated in double:
 *     SW_POTTS x = J/T            (Sec. 2 step (ii): p = 1 - e^{-beta})
 *     SW_ISING x = 2J/T           (same chain in Ising units, q = 2)
 *     SW_CLOCK x = (2J/T) * (a*b) with a, b = sin(pi*r/q), r = j mod q the
 *              projection classes j = (2k - m) mod 2q of the two states on
 *              the sweep's mirror axis m; zero unless both j lie strictly on
 *              the same side (0<j<q or q<j<2q).
 *   The label of a cluster is its smallest site index (the "proper label"
 *   of Sec. 2); Potts clusters take state mulhi(u_root, q) (Sec. 2 steps
 *   (v)-(vii)); clock clusters are reflected k -> (m - k) mod q iff the top
 *   bit of u_root is set (Sec. 4).  J = 1.
 *
 * Counters (int64) measured after every sweep, in this order:
 *   n_0 .. n_{q-1}     state counts of the new configuration (Eq. M^2)
 *   class_0 .. class_{C-1}  bond classes of the new configuration
 *                      Potts/Ising: C = 2, class 0 equal pair, 1 unequal;
 *                      clock: C = q/2 + 1, class d = min(dk, q - dk)
 *   active             active bonds of the sweep
 *   clusters           clusters of the sweep
 *   clock only: corr4_0 .. corr4_{C-1}, corr2_0 .. corr2_{C-1}: the classes
 *                      d of the 2N pairs (i, i + r x), (i, i + r y) at
 *                      r = L/4 and r = L/2 (Sec. 4, correlation G(r,T))
 *
 * Errors: every int-returning call returns SW_OK (0) or a negative status;
 * sw_last_error() gives a thread-local message.  The library never exits or
 * aborts.  Device-side failures (a bounded loop that ran out) are sticky per
 * handle and reported by the next sw_sweep/sw_measure/sw_synchronize.
 * Ownership: a handle owns its device buffers (cudaMalloc'd on the device
 * current at sw_create) unless created with sw_create_ext, which borrows
 * caller buffers that must outlive the handle.  Handles are not
 * thread-safe; use one handle per thread or serialise calls.
 */
#ifndef SW_GB300_H
#define SW_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum sw_model { SW_POTTS = 0, SW_CLOCK = 1, SW_ISING = 2 };

enum sw_status {
    SW_OK = 0,
    SW_ERR_ARG = -1,            /* invalid argument                        */
    SW_ERR_OOM = -2,            /* device or host allocation failed        */
    SW_ERR_CUDA = -3,           /* a CUDA runtime call failed              */
    SW_ERR_NOT_CONVERGED = -4,  /* a bounded device loop ran out (sticky)  */
    SW_ERR_STATE = -5           /* call not valid in the handle's state    */
};

enum sw_init_mode { SW_INIT_UP = 0, SW_INIT_RANDOM = 1 };

#define SW_MAX_Q 127
#define SW_MAX_CLOCK_Q 64
#define SW_MAX_COUNTERS (SW_MAX_Q + SW_MAX_Q / 2 + 1 + 2)

typedef struct sw_handle sw_handle;
typedef struct sw_batch sw_batch;

/* Observables after the last sweep plus running means since sw_reset_stats
 * (Sec. 4: energy, magnetisation, moment ratio U = <M^4>/<M^2>^2, Eq. U).
 * Per-site values: e = E/N, m2 = M^2/N^2 with M^2 from Eq. (M^2) (Potts,
 * Ising) or |sum_i S_i|^2 (clock); absm = sqrt(m2); m4 = m2^2. */
typedef struct sw_obs {
    uint64_t sweep;              /* sweeps completed                          */
    int32_t L, q, model, ncounters;
    int64_t counts[SW_MAX_COUNTERS];   /* counters of the last sweep          */
    double e, absm, m2, m4;      /* observables of the last sweep             */
    uint64_t nmeas;              /* sweeps accumulated in the means below     */
    double mean_e, mean_e2, mean_absm, mean_m2, mean_m4;
    double binder_u;             /* mean_m4 / mean_m2^2 (Eq. U)              */
    double mean_active, mean_clusters;
    /* clock model (0 otherwise): G(r) = <cos(theta_i - theta_{i+r})> over the
     * pairs at r = L/4 and L/2 (Sec. 4), last sweep and running means, and
     * R = mean G(L/2) / mean G(L/4) (Sec. 4, R(T)) */
    double g_quarter, g_half, mean_g_quarter, mean_g_half, corr_ratio;
} sw_obs;

/* Number of counters per sweep for (q, model): q + C + 2 (clock: q + 3C + 2). */
int sw_ncounters(int q, int model);

/* Create a lattice on the current device: 4 <= L <= 46340, L % 4 == 0;
 * Potts 2 <= q <= 127; Ising q == 2; clock 2 <= q <= 64; T > 0 finite.
 * Spins start all in state 0; measurement is on.  NULL on error. */
sw_handle *sw_create(int L, int q, int model, double T, uint64_t seed);

/* As sw_create, but borrow caller-owned device buffers (spins: L*L int8,
 * labels: L*L int32, both 16-byte aligned) and run on `stream`
 * (a cudaStream_t, NULL = legacy default stream).  Either buffer may be
 * NULL, in which case the library allocates it. */
sw_handle *sw_create_ext(int L, int q, int model, double T, uint64_t seed,
                         void *d_spins, void *d_labels, void *stream);

/* Release everything the handle owns (NULL-safe).  Synchronises its stream. */
int sw_destroy(sw_handle *h);

/* Thread-local description of the last failure. */
const char *sw_last_error(void);

/* (Re)initialise the spins: SW_INIT_UP (all 0) or SW_INIT_RANDOM
 * (mulhi(u_INIT(i), q)).  Does not change the sweep index. */
int sw_init(sw_handle *h, int mode);

/* Enqueue n >= 0 sweeps on the handle's stream.  Asynchronous, except that
 * the per-sweep counter ring (1024 sweeps) is drained to the host when full.
 * Returns a sticky device error if one was recorded earlier. */
int sw_sweep(sw_handle *h, int n);

/* Wait for the stream, fold every pending sweep's counters into the running
 * means, and fill *out (may be NULL just to drain). */
int sw_measure(sw_handle *h, sw_obs *out);

/* Wait for the handle's stream; report any sticky device error. */
int sw_synchronize(sw_handle *h);

/* Counters on (1, default: the paper's "+ measurement") or off (0,
 * "update only").  Sweeps run with counters off are not accumulated. */
int sw_set_measure(sw_handle *h, int on);

/* Keep (1) or drop (0, default) the per-sweep counter rows on the host;
 * sw_take_counts() returns and clears them. */
int sw_set_record(sw_handle *h, int on);
/* Copy up to max_rows recorded rows (ncounters int64 each, oldest first)
 * into out and drop them; returns the number of rows copied (>= 0). */
int sw_take_counts(sw_handle *h, int64_t *out, int max_rows);

/* Zero the running means. */
int sw_reset_stats(sw_handle *h);

/* Write every site's canonical cluster label (smallest site index) during
 * the sweeps that follow (1), or not (0, default). */
int sw_set_debug_labels(sw_handle *h, int on);

/* Host copies (synchronous on the handle's stream).  n must equal L*L.
 * sw_set_spins checks every state on the device; if any lies outside
 * [0, q) it returns SW_ERR_ARG and leaves all spins in state 0. */
int sw_get_spins(sw_handle *h, int8_t *host, size_t n);
int sw_set_spins(sw_handle *h, const int8_t *host, size_t n);
/* Labels of the last sweep; valid for sweeps run with debug labels on. */
int sw_get_labels(sw_handle *h, int32_t *host, size_t n);

/* Device pointers of the handle's buffers (for zero-copy framework use). */
void *sw_device_spins(sw_handle *h);
void *sw_device_labels(sw_handle *h);

/* Potts/Ising: 1 threshold; clock: the (2q)^2 table, row-major by class j.
 * Returns the number of entries written or a negative status. */
int sw_get_thresholds(sw_handle *h, uint32_t *out, int n);

/* Sweep index (sweeps completed); setting it positions the random stream
 * (checkpoint/resume: spins + sweep index + seed + parameters). */
int sw_get_sweep(sw_handle *h, uint64_t *out);
int sw_set_sweep(sw_handle *h, uint64_t t);

/* Sweep limit: the lattice sweeps only while its sweep index is below
 * `stop` (UINT64_MAX, the default: no limit).  Sweeps requested beyond it
 * are skipped on the device -- in a batch every kernel leaves the lattice
 * as it is -- and its index stays at `stop`, so a batch can be advanced by
 * more sweeps than some of its lattices still need (a job server gives each
 * job its budget this way).  sw_get_sweep_limit reads it back. */
int sw_set_sweep_limit(sw_handle *h, uint64_t stop);
int sw_get_sweep_limit(sw_handle *h, uint64_t *out);

/* Launch shape: resident blocks per SM requested for the kernels of a
 * sweep, shape[4] = {labeling, merge, flip, bonds}, each in [1, 64]
 * (default {11, 12, 10, 16}).  The labeling kernel that draws the bonds
 * itself (batches without a clock lattice) keeps at most 11 blocks per SM,
 * the flip kernel 10 (8 with a clock lattice); the bond figure applies only
 * where the bond kernel runs (a clock lattice in the batch).
 * Results never depend on it.  sw_autotune times every candidate (n real
 * sweeps each, they advance the chain like any others), keeps the fastest
 * per kernel, caches it per (device, work size, measurement, clock lattice)
 * for the process, and writes the choice to shape_out (may be NULL).  A
 * cached choice costs no sweeps. */
int sw_autotune(sw_handle *h, int n, int *shape_out);
int sw_set_launch_shape(sw_handle *h, const int *shape);

/* Cluster labeling of the handle's sweeps.  SW_LABEL_TILED (default) is the
 * library's tile-local labeling plus a boundary merge.  SW_LABEL_HAWICK and
 * SW_LABEL_KALENTEV are the paper's GPU labelings (Sec. 3: Hawick et al.'s
 * label equivalence with a reference array and atomicMin; Kalentev et al.'s
 * refinement with one array and no atomics), kept as comparators: whole-
 * lattice scan/analysis passes until no label changes, the host reading a
 * device flag after each pass.  Every labeling ends at the same canonical
 * labels, so the chain is identical.  The comparators are update only
 * (measurement must be off; SW_ERR_STATE otherwise), need a lattice outside
 * any batch, run without CUDA graphs, and allocate L*L int32 more for
 * Hawick's reference array. */
enum sw_labeling { SW_LABEL_TILED = 0, SW_LABEL_HAWICK = 1, SW_LABEL_KALENTEV = 2 };
int sw_set_labeling(sw_handle *h, int method);
/* Scan passes of the last comparator sweep (0 for the tiled labeling). */
int sw_label_passes(sw_handle *h);

/* Test aid, not needed for simulation.  loop_cap > 0: every data-dependent
 * device loop of the sweep (union-find walks and links in shared and global
 * memory) gives up after loop_cap steps and records a device error, which
 * the next sw_sweep / sw_measure / sw_synchronize reports as the sticky
 * SW_ERR_NOT_CONVERGED (results of that sweep are undefined); no loop can
 * run longer than its cap.  list_cap > 0: a tile's list of union pairs holds
 * at most list_cap pairs; the rest are joined by the threads that found
 * them (same results, the path taken when the list overflows).  0 restores
 * the default of either.  Negative values: SW_ERR_ARG. */
int sw_set_debug_limits(sw_handle *h, int loop_cap, int list_cap);

/* Labeling statistics, the counterpart of the paper's labeling-iteration
 * count (Sec. 4: the passes a whole-lattice labeling needs grow near and
 * below T_c).  on = 1 starts (and zeroes) per-lattice device tallies of the
 * following sweeps, 0 stops and frees them; while on, the merge and flip
 * kernels run variants that tally (slower).  sw_get_labeling_stats writes
 * up to n of these values (per sweep, per tile where stated) and returns
 * how many it wrote:
 *   0 sweeps tallied
 *   1 provisional labels opened by the tile scans, per tile
 *   2 union pairs of the tiles (further run contacts, quadrant seams), per tile
 *   3 tile components (clusters inside a tile + open components), per tile
 *   4 open components (reaching a tile border), per tile
 *   5 unions across tile edges (distinct component pairs), per sweep
 *   6 link attempts per union (atomicMin on a root entry)
 *   7 attempts that found the root linked meanwhile, per attempt
 *   8 walks of the global union-find (merge and root walks), per sweep
 *   9 parent steps per walk
 *   10 the longest walk (steps)
 * Values 1-4 are exact functions of the bonds; 5-10 depend on the order in
 * which the GPU's threads meet.  SW_ERR_STATE if the statistics are off. */
int sw_set_labeling_stats(sw_handle *h, int on);
int sw_get_labeling_stats(sw_handle *h, double *out, int n);

/* Use a different stream for subsequent work (a cudaStream_t). */
int sw_set_stream(sw_handle *h, void *stream);

/* Capture one sweep as a CUDA graph and replay it for every later sweep
 * (1), or launch the kernels directly (0, default).  Same results. */
int sw_set_graph(sw_handle *h, int on);

/* Tracing: run n sweeps with CUDA events recorded on the handle's stream
 * around every kernel (direct launches) and write the mean device time per
 * sweep of each stage in milliseconds to ms[0 .. stages-1]:
 *   0 bond activation (+ bond classes of the incoming configuration),
 *   1 tile-local labeling and closed-cluster draws, 2 merge across tile
 *   edges, 3 open-cluster roots and draws + spin write (+ state counts).
 * The sweeps count like any others.  Returns the number of stages (>0). */
int sw_profile_sweeps(sw_handle *h, int n, float *ms, int max_stages);

/* ------------------------------------------------------------------------
 * Batches: many independent lattices (any mix of L, q, model, T, seed)
 * advanced together, one launch sequence per sweep for all of them.  Every
 * lattice's chain is identical to sweeping it alone (same kernels, same
 * keys).  A batch references handles it does not own; attached handles run
 * on the batch's stream and keep working with every per-handle getter
 * (sw_measure, sw_get_spins, ...).
 * ---------------------------------------------------------------------- */

/* New empty batch on `stream` (a cudaStream_t; NULL: the batch makes one). */
sw_batch *sw_batch_create(void *stream);
/* Detach every lattice (they stay valid) and free the batch.  NULL-safe. */
int sw_batch_destroy(sw_batch *b);
/* Add / remove a lattice.  Attaching waits for the lattice's pending work
 * and moves it to the batch's stream and measurement setting; a lattice
 * can be in one batch at a time.  Detaching gives it a stream of its own.
 * sw_destroy detaches a lattice first. */
int sw_batch_attach(sw_batch *b, sw_handle *h);
int sw_batch_detach(sw_batch *b, sw_handle *h);
int sw_batch_size(sw_batch *b);
/* Enqueue n sweeps of every attached lattice (asynchronous). */
int sw_batch_sweep(sw_batch *b, int n);
/* Wait for the batch's stream; report the first sticky device error. */
int sw_batch_synchronize(sw_batch *b);
/* Measurement on/off, CUDA-graph replay, debug labels: as the per-handle calls. */
int sw_batch_set_measure(sw_batch *b, int on);
int sw_batch_set_graph(sw_batch *b, int on);
int sw_batch_set_debug_labels(sw_batch *b, int on);
/* As sw_profile_sweeps / sw_autotune / sw_set_launch_shape, for the batched
 * launch sequence. */
int sw_batch_profile_sweeps(sw_batch *b, int n, float *ms, int max_stages);
int sw_batch_autotune(sw_batch *b, int n, int *shape_out);
int sw_batch_set_launch_shape(sw_batch *b, const int *shape);

/* ------------------------------------------------------------------------
 * Sweeps without device allocation.  The paper has no counterpart: this is
 * a convenience of the library's interface.
 *
 * Some callers cannot allocate device memory at the point where they want
 * to sweep: a plugin running inside a host framework that hands out all
 * device memory from its own pool (an allocation of its own would fail once
 * the pool holds the memory, or escape the host's accounting), or a
 * latency-bound loop where cudaMalloc / cudaFree could stall on an implicit
 * device synchronisation.  sw_sweep_noalloc serves them: it takes the
 * spins (and, optionally, a counter buffer) from the caller and keeps all
 * its working memory in one fixed array of SW_NOALLOC_SCRATCH_BYTES bytes
 * compiled into the library, which every device that loads the library
 * holds until the process exits.  It calls no allocating routine.
 *
 * It runs n sweeps with the kernels and random streams of sw_sweep: the
 * result equals that of a handle made by sw_create(L, q, model, T, seed)
 * holding the same spins at sweep index sweep0, after sw_sweep(h, n).
 *   d_spins   device, L*L int8 states in [0, q), row-major, 16-byte aligned;
 *             read and overwritten in place.  If any state lies outside
 *             [0, q) the call returns SW_ERR_ARG and changes nothing.
 *   d_counts  device, n * sw_ncounters(q, model) int64, 8-byte aligned, or
 *             NULL: row k receives the counters of sweep sweep0 + k (the
 *             rows sw_take_counts would return).  NULL skips measurement.
 *   sweep0    sweeps completed before this call (positions the random
 *             stream); a chain continues with sweep0 + n on the next call.
 *   stream    cudaStream_t for all work (NULL = legacy default stream).
 * Limits: 4 <= L <= SW_NOALLOC_MAX_L with L % 4 == 0, and the q / model / T
 * rules of sw_create; anything else returns SW_ERR_ARG before any GPU work.
 * The call returns once its work on `stream` is complete (it synchronises
 * the stream, also on an error after work was enqueued).
 *
 * The first call on a device looks up the array's device address (and may
 * load the library's device code onto that device); make that first call
 * before any stream capture begins.  All calls on a device share the array,
 * which keeps the previous call's contents (each call resets what must
 * start from a known value): calls whose work overlaps on the GPU, from
 * several threads or streams, race and corrupt each other's results, so
 * serialise them.
 * ---------------------------------------------------------------------- */
#define SW_NOALLOC_MAX_L 1024
#define SW_NOALLOC_SCRATCH_BYTES (7 * 1024 * 1024)
int sw_sweep_noalloc(int L, int q, int model, double T, uint64_t seed, uint64_t sweep0, int n,
                     int8_t *d_spins, int64_t *d_counts, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SW_GB300_H */
