/*
 * sw_oracle.h -- plain single-threaded CPU Swendsen-Wang sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: its Philox-4x32-10, its bond thresholds, its cluster
 * search and its observables are written here from their definitions.
 *
 * What it computes (Komura & Okabe, arXiv:1202.0635):
 *   - q-state Potts model, Eq. (1), periodic L x L square lattice (Sec. 2);
 *   - the SW update as the CPU procedure (i)-(viii) of Sec. 2: bonds between
 *     equal nearest neighbours with p = 1 - exp(-K), cluster identification,
 *     and a uniformly drawn new state for every cluster;
 *   - the q-state clock model, Eq. (clock, Sec. 4), updated with Wolff's
 *     embedded-cluster idea (Sec. 4): project on a mirror axis, bond aligned
 *     projections, reflect each cluster with probability 1/2;
 *   - the measurement of Sec. 4: state counts n[k] for M^2 of Eq. (M^2),
 *     energy from the bond classes.
 * Cluster identification is a breadth-first search started from every
 * unvisited site in increasing site order, so every cluster's label is its
 * smallest site index (the "proper label" of Sec. 2).
 *
 * Conventions shared with the GPU path by SPECIFICATION only (each side has
 * its own code):
 *   site i = y*L + x; site i owns the bond to its right neighbour
 *   y*L + (x+1)%L (direction 0) and to its down neighbour ((y+1)%L)*L + x
 *   (direction 1).
 *   Philox-4x32-10 key = (seed & 0xffffffff, seed >> 32).
 *   counter = (index, sweep & 0xffffffff, tag, sweep >> 32) with
 *     tag 0 BOND : index = i >> 1; lane 2*(i & 1) + direction is site i's draw
 *     tag 1 STATE: index = cluster root; lane 0 (Potts, q > 2: the new state
 *                  is mulhi(u, q))
 *     tag 2 AXIS : index = 0; lane 0 (clock mirror axis of the sweep)
 *     tag 3 INIT : index = i; lane 0 (random start; sweep field 0)
 *     tag 4 STATE_BIT: index = r >> 7 for cluster root r; the new state
 *                  (Potts / Ising, q = 2) or reflection flag (clock) is bit
 *                  r & 31 of lane (r >> 5) & 3
 *   "sweep" is the number of sweeps completed before the one drawing.
 *   bond active iff the 32-bit draw u < threshold (an integer, see below).
 *   mulhi(u, q) = (u * q) >> 32 maps a draw to [0, q).
 */
#ifndef SW_ORACLE_H
#define SW_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SWO_POTTS = 0, SWO_CLOCK = 1, SWO_ISING = 2 };

typedef struct swo swo;

/* Philox-4x32-10 of one counter under one key. */
void swo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Integer bond threshold floor(p * 2^32), clamped to 2^32-1, p = -expm1(-x). */
uint32_t swo_threshold_from_x(double x);

/* Lifetime.  L >= 2, 2 <= q <= 127, T > 0.  NULL on bad arguments. */
swo *swo_create(int L, int q, int model, double T, uint64_t seed);
void swo_destroy(swo *o);

/* Potts/Ising: one threshold.  Clock: the (2q) x (2q) table, row-major. */
int swo_thresholds(const swo *o, uint32_t *out, int n);

void swo_init_up(swo *o);              /* every spin in state 0 */
void swo_init_random(swo *o);          /* state = mulhi(u_INIT(i), q)  */
void swo_set_spins(swo *o, const int8_t *s);
void swo_get_spins(const swo *o, int8_t *s);
void swo_get_labels(const swo *o, int32_t *lab);   /* last sweep's labels */
void swo_get_bonds(const swo *o, uint8_t *b);      /* bit0 right, bit1 down */
uint64_t swo_get_sweep(const swo *o);
void swo_set_sweep(swo *o, uint64_t t);
int swo_last_axis(const swo *o);

/* Number of int64 counters per measurement: q + nclass + 2, and for the
 * clock model 2 * nclass more. */
int swo_ncounters(int q, int model);

/* Run n sweeps.  If counts != NULL, write the counters measured after
 * every sweep, n rows of swo_ncounters() int64 each:
 *   [n_0 .. n_{q-1}] state counts of the new configuration,
 *   [class_0 .. class_{nc-1}] bond classes of the new configuration
 *       (Potts/Ising: nc = 2, class 0 = equal pair, class 1 = unequal;
 *        clock: nc = q/2 + 1, class d counts bonds with min(dk, q-dk) = d),
 *   [active] active bonds of the sweep, [clusters] clusters of the sweep,
 *   clock only: [corr4_0 .. corr4_{nc-1}] [corr2_0 .. corr2_{nc-1}], the
 *       classes of the 2N pairs (i, i + r x), (i, i + r y) at r = L/4 and
 *       r = L/2 (Sec. 4, G(r,T)). */
void swo_sweep(swo *o, int n, int64_t *counts);

/* Counters of the current configuration (active/clusters of the last sweep). */
void swo_counts(const swo *o, int64_t *counts);

/* FP64 observables from one counter row: out = {E/N, |m|, m^2, m^4}. */
void swo_observables(int L, int q, int model, const int64_t *counts, double *out);

/* Clock model: out = {G(L/4), G(L/2)} from one counter row (Sec. 4). */
void swo_correlations(int L, int q, const int64_t *counts, double *out);

/* Label nsets given bond configurations (N bytes each, bit0 right, bit1
 * down) with the same search the sweep uses; labels: nsets x N. */
void swo_label_bonds(swo *o, const uint8_t *bonds, int64_t nsets, int32_t *labels);

/* One-step transition samples: for s = 0..M-1, set the spins to sigma,
 * set the sweep index to t0 + s, run one sweep and store the result in
 * out[s*N .. s*N+N-1]. */
void swo_sample_one_step(swo *o, const int8_t *sigma, uint64_t t0, int M, int8_t *out);

#ifdef __cplusplus
}
#endif
#endif
