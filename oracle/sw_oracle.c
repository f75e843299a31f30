/*
 * sw_oracle.c -- plain, slow, single-threaded CPU Swendsen-Wang sweep.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers.  Nothing here is shared with the
 * CUDA path.  Conventions (site order, bond ownership, RNG keying, integer
 * thresholds) are described in sw_oracle.h.
 *
 * Every function follows one passage of Komura & Okabe, arXiv:1202.0635:
 *   Sec. 2, Eq. (1)          q-state Potts Hamiltonian, periodic boundaries
 *   Sec. 2, steps (i)-(iii)  bond generation with p = 1 - exp(-beta), beta=J/T
 *   Sec. 2, step (iv)        cluster identification (here: BFS; the label of
 *                            a cluster is its smallest site index, the
 *                            "proper label" of the Hoshen-Kopelman passage)
 *   Sec. 2, steps (v)-(vii)  every cluster gets one of q states, prob. 1/q
 *   Sec. 4, Eq. (clock)      q-state clock model, angles 2 pi p / q
 *   Sec. 4, embedded cluster projection on a mirror axis + reflection
 *   Sec. 4, Eq. (M^2)        Potts order parameter from the counts n[k]
 */
#include "sw_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplications whose high halves are mixed with the other two
 * words and the round key; the key is bumped by the two Weyl constants
 * between rounds.                                                       */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void swo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

enum { TAG_BOND = 0, TAG_STATE = 1, TAG_AXIS = 2, TAG_INIT = 3, TAG_STATE_BIT = 4 };

static uint32_t draw(uint64_t seed, uint32_t index, uint64_t sweep, uint32_t tag, int lane)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {index, (uint32_t)(sweep & 0xffffffffu), tag, (uint32_t)(sweep >> 32)};
    uint32_t out[4];
    swo_philox4x32_10(ctr, key, out);
    return out[lane];
}

/* One uniform bit per index: bit (index & 31) of lane (index >> 5) & 3 of
 * the draw with counter index >> 7 (128 indices share one Philox call). */
static int draw_bit(uint64_t seed, uint32_t index, uint64_t sweep, uint32_t tag)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {index >> 7, (uint32_t)(sweep & 0xffffffffu), tag, (uint32_t)(sweep >> 32)};
    uint32_t out[4];
    swo_philox4x32_10(ctr, key, out);
    return (int)((out[(index >> 5) & 3u] >> (index & 31u)) & 1u);
}

static int mulhi_q(uint32_t u, int q)
{
    return (int)(((uint64_t)u * (uint64_t)q) >> 32);
}

/* ------------------------------------------------------------------ */
/* Bond probabilities as integer thresholds.                           */
/* Sec. 2 step (ii): p = 1 - exp(-beta).  With x the exponent, p is
 * evaluated as -expm1(-x) in double and stored as floor(p * 2^32)
 * clamped to 2^32 - 1; a 32-bit draw u activates the bond iff u < it. */
/* ------------------------------------------------------------------ */
uint32_t swo_threshold_from_x(double x)
{
    if (!(x > 0.0)) return 0u;
    double p = -expm1(-x);
    double s = floor(ldexp(p, 32));
    if (s >= 4294967295.0) return 0xffffffffu;
    if (s <= 0.0) return 0u;
    return (uint32_t)s;
}

/* Clock embedding (Sec. 4, Wolff's embedded cluster).  With mirror axis
 * index m in [0, q), state k has the class j = (2k - m) mod 2q; its
 * projection on the axis normal is proportional to sin(pi j / q): zero for
 * j = 0 and j = q, positive for 0 < j < q, negative for q < j < 2q.  The
 * embedded Ising coupling of a bond is 2 K |s_a| |s_b| when the projections
 * have the same sign, and the bond can only form then. */
static double clock_abs_proj(int j, int q)
{
    int r = j % q;
    return sin((M_PI * (double)r) / (double)q);
}

static int clock_sign(int j, int q)
{
    if (j % q == 0) return 0;
    return j < q ? 1 : -1;
}

struct swo {
    int L, q, model;
    int64_t N;
    double T, K;
    uint64_t seed, sweep;
    int8_t *spin;
    uint8_t *bond;
    int32_t *label;
    int32_t *queue;
    int8_t *newstate;       /* per root: Potts new state / clock reflect flag */
    uint32_t thr;           /* Potts / Ising */
    uint32_t *thr_clock;    /* clock: (2q) x (2q) */
    int axis;
    int64_t active, clusters;
};

swo *swo_create(int L, int q, int model, double T, uint64_t seed)
{
    if (L < 2 || q < 2 || q > 127) return NULL;
    if (model != SWO_POTTS && model != SWO_CLOCK && model != SWO_ISING) return NULL;
    if (model == SWO_ISING && q != 2) return NULL;
    if (!(T > 0.0) || !isfinite(T)) return NULL;
    swo *o = (swo *)calloc(1, sizeof(swo));
    if (!o) return NULL;
    o->L = L; o->q = q; o->model = model; o->T = T; o->seed = seed;
    o->N = (int64_t)L * (int64_t)L;
    o->K = 1.0 / T;    /* J = 1 */
    o->spin = (int8_t *)calloc((size_t)o->N, 1);
    o->bond = (uint8_t *)calloc((size_t)o->N, 1);
    o->label = (int32_t *)calloc((size_t)o->N, sizeof(int32_t));
    o->queue = (int32_t *)calloc((size_t)o->N, sizeof(int32_t));
    o->newstate = (int8_t *)calloc((size_t)o->N, 1);
    if (!o->spin || !o->bond || !o->label || !o->queue || !o->newstate) {
        swo_destroy(o);
        return NULL;
    }
    for (int64_t i = 0; i < o->N; ++i) o->label[i] = (int32_t)i;
    if (model == SWO_POTTS) {
        o->thr = swo_threshold_from_x(o->K);              /* p = 1 - e^{-J/T}  */
    } else if (model == SWO_ISING) {
        o->thr = swo_threshold_from_x(2.0 * o->K);        /* p = 1 - e^{-2J/T} */
    } else {
        int n = 2 * q;
        o->thr_clock = (uint32_t *)calloc((size_t)(n * n), sizeof(uint32_t));
        if (!o->thr_clock) { swo_destroy(o); return NULL; }
        for (int a = 0; a < n; ++a) {
            for (int b = 0; b < n; ++b) {
                int sa = clock_sign(a, q), sb = clock_sign(b, q);
                uint32_t t = 0;
                if (sa != 0 && sa == sb) {
                    double prod = clock_abs_proj(a, q) * clock_abs_proj(b, q);
                    t = swo_threshold_from_x((2.0 * o->K) * prod);
                }
                o->thr_clock[a * n + b] = t;
            }
        }
    }
    return o;
}

void swo_destroy(swo *o)
{
    if (!o) return;
    free(o->spin); free(o->bond); free(o->label); free(o->queue);
    free(o->newstate); free(o->thr_clock);
    free(o);
}

int swo_thresholds(const swo *o, uint32_t *out, int n)
{
    if (o->model == SWO_CLOCK) {
        int m = 4 * o->q * o->q;
        if (n < m) return -1;
        memcpy(out, o->thr_clock, (size_t)m * sizeof(uint32_t));
        return m;
    }
    if (n < 1) return -1;
    out[0] = o->thr;
    return 1;
}

void swo_init_up(swo *o)
{
    memset(o->spin, 0, (size_t)o->N);
}

void swo_init_random(swo *o)
{
    for (int64_t i = 0; i < o->N; ++i)
        o->spin[i] = (int8_t)mulhi_q(draw(o->seed, (uint32_t)i, 0, TAG_INIT, 0), o->q);
}

void swo_set_spins(swo *o, const int8_t *s) { memcpy(o->spin, s, (size_t)o->N); }
void swo_get_spins(const swo *o, int8_t *s) { memcpy(s, o->spin, (size_t)o->N); }
void swo_get_labels(const swo *o, int32_t *lab) { memcpy(lab, o->label, (size_t)o->N * 4); }
void swo_get_bonds(const swo *o, uint8_t *b) { memcpy(b, o->bond, (size_t)o->N); }
uint64_t swo_get_sweep(const swo *o) { return o->sweep; }
void swo_set_sweep(swo *o, uint64_t t) { o->sweep = t; }
int swo_last_axis(const swo *o) { return o->axis; }

int swo_ncounters(int q, int model)
{
    int nclass = (model == SWO_CLOCK) ? q / 2 + 1 : 2;
    /* clock: two more class histograms, pairs at distance L/4 and L/2 */
    return q + nclass + 2 + (model == SWO_CLOCK ? 2 * nclass : 0);
}

static int64_t right_of(const swo *o, int64_t i)
{
    int64_t y = i / o->L, x = i % o->L;
    return y * o->L + (x + 1) % o->L;
}

static int64_t down_of(const swo *o, int64_t i)
{
    int64_t y = i / o->L, x = i % o->L;
    return ((y + 1) % o->L) * o->L + x;
}

static int64_t left_of(const swo *o, int64_t i)
{
    int64_t y = i / o->L, x = i % o->L;
    return y * o->L + (x + o->L - 1) % o->L;
}

static int64_t up_of(const swo *o, int64_t i)
{
    int64_t y = i / o->L, x = i % o->L;
    return ((y + o->L - 1) % o->L) * o->L + x;
}

/* Can the bond between states a and b form, and with which threshold? */
static uint32_t bond_threshold(const swo *o, int a, int b)
{
    if (o->model == SWO_CLOCK) {
        int n = 2 * o->q;
        int ja = ((2 * a - o->axis) % n + n) % n;
        int jb = ((2 * b - o->axis) % n + n) % n;
        return o->thr_clock[ja * n + jb];
    }
    return (a == b) ? o->thr : 0u;   /* Sec. 2 (ii): only equal neighbours */
}

/* Sec. 2 steps (i)-(iii): every site looks at its right and down
 * neighbour; each bond is tested once, by the site that owns it. */
static void make_bonds(swo *o)
{
    o->active = 0;
    for (int64_t i = 0; i < o->N; ++i) {
        int lane = 2 * (int)(i & 1);
        uint32_t u_right = draw(o->seed, (uint32_t)(i >> 1), o->sweep, TAG_BOND, lane);
        uint32_t u_down = draw(o->seed, (uint32_t)(i >> 1), o->sweep, TAG_BOND, lane + 1);
        uint8_t b = 0;
        if (u_right < bond_threshold(o, o->spin[i], o->spin[right_of(o, i)])) b |= 1;
        if (u_down < bond_threshold(o, o->spin[i], o->spin[down_of(o, i)])) b |= 2;
        o->bond[i] = b;
        o->active += (b & 1) + ((b >> 1) & 1);
    }
}

/* Sec. 2 step (iv): label clusters.  A BFS is started from each site that
 * no earlier search reached, in increasing site order; the start site is
 * then the smallest index of its cluster and becomes the label. */
static void label_clusters(swo *o)
{
    for (int64_t i = 0; i < o->N; ++i) o->label[i] = -1;
    o->clusters = 0;
    for (int64_t start = 0; start < o->N; ++start) {
        if (o->label[start] != -1) continue;
        o->clusters++;
        int64_t head = 0, tail = 0;
        o->label[start] = (int32_t)start;
        o->queue[tail++] = (int32_t)start;
        while (head < tail) {
            int64_t i = o->queue[head++];
            int64_t nb[4];
            int has[4];
            nb[0] = right_of(o, i); has[0] = o->bond[i] & 1;
            nb[1] = down_of(o, i);  has[1] = (o->bond[i] >> 1) & 1;
            nb[2] = left_of(o, i);  has[2] = o->bond[nb[2]] & 1;
            nb[3] = up_of(o, i);    has[3] = (o->bond[nb[3]] >> 1) & 1;
            for (int d = 0; d < 4; ++d) {
                if (has[d] && o->label[nb[d]] == -1) {
                    o->label[nb[d]] = (int32_t)start;
                    o->queue[tail++] = (int32_t)nb[d];
                }
            }
        }
    }
}

/* Sec. 2 steps (v)-(vii) (Potts) and the reflection of Sec. 4 (clock):
 * one draw per cluster, keyed on its label.  A uniform new state among q
 * (Potts) or a reflection with probability 1/2 (clock); where there are
 * two outcomes (q = 2, clock) the draw is one uniform bit. */
static void flip_clusters(swo *o)
{
    for (int64_t r = 0; r < o->N; ++r) {
        if (o->label[r] != r) continue;
        if (o->model == SWO_CLOCK || o->q == 2) {
            o->newstate[r] = (int8_t)draw_bit(o->seed, (uint32_t)r, o->sweep, TAG_STATE_BIT);
        } else {
            uint32_t u = draw(o->seed, (uint32_t)r, o->sweep, TAG_STATE, 0);
            o->newstate[r] = (int8_t)mulhi_q(u, o->q);
        }
    }
    for (int64_t i = 0; i < o->N; ++i) {
        int8_t v = o->newstate[o->label[i]];
        if (o->model == SWO_CLOCK) {
            if (v) o->spin[i] = (int8_t)(((o->axis - o->spin[i]) % o->q + o->q) % o->q);
        } else {
            o->spin[i] = v;
        }
    }
}

static void one_sweep(swo *o)
{
    if (o->model == SWO_CLOCK)
        o->axis = mulhi_q(draw(o->seed, 0, o->sweep, TAG_AXIS, 0), o->q);
    make_bonds(o);
    label_clusters(o);
    flip_clusters(o);
    o->sweep++;
}

void swo_counts(const swo *o, int64_t *c)
{
    int q = o->q;
    int nclass = (o->model == SWO_CLOCK) ? q / 2 + 1 : 2;
    memset(c, 0, (size_t)swo_ncounters(q, o->model) * sizeof(int64_t));
    for (int64_t i = 0; i < o->N; ++i) {
        c[o->spin[i]]++;
        int64_t nbs[2] = {right_of(o, i), down_of(o, i)};
        for (int d = 0; d < 2; ++d) {
            int a = o->spin[i], b = o->spin[nbs[d]];
            int cls;
            if (o->model == SWO_CLOCK) {
                int dk = ((a - b) % q + q) % q;
                cls = dk < q - dk ? dk : q - dk;
            } else {
                cls = (a == b) ? 0 : 1;
            }
            c[q + cls]++;
        }
    }
    c[q + nclass] = o->active;
    c[q + nclass + 1] = o->clusters;
    if (o->model == SWO_CLOCK) {
        /* Correlation at distance r = L/4 and L/2 (Sec. 4, G(r,T)): the class
         * min(dk, q - dk) of every pair (i, i + r x) and (i, i + r y). */
        int64_t L = o->L;
        for (int w = 0; w < 2; ++w) {
            int64_t r = (w == 0) ? L / 4 : L / 2;
            int64_t *h = c + q + nclass + 2 + (int64_t)w * nclass;
            for (int64_t y = 0; y < L; ++y) {
                for (int64_t x = 0; x < L; ++x) {
                    int a = o->spin[y * L + x];
                    int bx = o->spin[y * L + (x + r) % L];
                    int by = o->spin[((y + r) % L) * L + x];
                    int dx = ((a - bx) % q + q) % q, dy = ((a - by) % q + q) % q;
                    h[dx < q - dx ? dx : q - dx]++;
                    h[dy < q - dy ? dy : q - dy]++;
                }
            }
        }
    }
}

void swo_sweep(swo *o, int n, int64_t *counts)
{
    int nc = swo_ncounters(o->q, o->model);
    for (int s = 0; s < n; ++s) {
        one_sweep(o);
        if (counts) swo_counts(o, counts + (int64_t)s * nc);
    }
}

/* Observables from one counter row (Sec. 4):
 *   Potts  E = J * (number of unequal neighbour pairs)       (Eq. 1)
 *   Ising  E = -J * (equal pairs - unequal pairs)
 *   clock  E = -J * sum_d class_d cos(2 pi d / q)           (Eq. clock)
 *   Potts/Ising  M^2 = (q sum_k n_k^2 - N^2) / (q - 1)      (Eq. M^2)
 *   clock  M^2 = (sum_k n_k cos th_k)^2 + (sum_k n_k sin th_k)^2
 * The numerator of Eq. (M^2) is formed exactly in 128-bit integers. */
void swo_observables(int L, int q, int model, const int64_t *c, double *out)
{
    int64_t N = (int64_t)L * (int64_t)L;
    double dN = (double)N;
    double E, M2;
    if (model == SWO_CLOCK) {
        int nclass = q / 2 + 1;
        E = 0.0;
        for (int d = 0; d < nclass; ++d) E -= (double)c[q + d] * cos(2.0 * M_PI * (double)d / (double)q);
        double mx = 0.0, my = 0.0;
        for (int k = 0; k < q; ++k) {
            mx += (double)c[k] * cos(2.0 * M_PI * (double)k / (double)q);
            my += (double)c[k] * sin(2.0 * M_PI * (double)k / (double)q);
        }
        M2 = mx * mx + my * my;
    } else {
        if (model == SWO_ISING)
            E = -(double)(c[q] - c[q + 1]);
        else
            E = (double)c[q + 1];
        __int128 s2 = 0;
        for (int k = 0; k < q; ++k) s2 += (__int128)c[k] * (__int128)c[k];
        __int128 num = (__int128)q * s2 - (__int128)N * (__int128)N;
        M2 = (double)num / (double)(q - 1);
    }
    double m2 = M2 / (dN * dN);
    out[0] = E / dN;
    out[1] = sqrt(M2) / dN;
    out[2] = m2;
    out[3] = m2 * m2;
}

/* Clock model: G(L/4) and G(L/2) of one counter row, the mean of
 * cos(theta_i - theta_{i+r}) over the 2N pairs of each distance (x and y
 * displacements): sum_d class_d cos(2 pi d / q) / (2N). */
void swo_correlations(int L, int q, const int64_t *c, double *out)
{
    int nclass = q / 2 + 1;
    double pairs = 2.0 * (double)L * (double)L;
    for (int w = 0; w < 2; ++w) {
        const int64_t *h = c + q + nclass + 2 + (int64_t)w * nclass;
        double g = 0.0;
        for (int d = 0; d < nclass; ++d) g += (double)h[d] * cos(2.0 * M_PI * (double)d / (double)q);
        out[w] = g / pairs;
    }
}

void swo_label_bonds(swo *o, const uint8_t *bonds, int64_t nsets, int32_t *labels)
{
    for (int64_t s = 0; s < nsets; ++s) {
        memcpy(o->bond, bonds + s * o->N, (size_t)o->N);
        label_clusters(o);
        memcpy(labels + s * o->N, o->label, (size_t)o->N * sizeof(int32_t));
    }
}

void swo_sample_one_step(swo *o, const int8_t *sigma, uint64_t t0, int M, int8_t *out)
{
    for (int s = 0; s < M; ++s) {
        memcpy(o->spin, sigma, (size_t)o->N);
        o->sweep = t0 + (uint64_t)s;
        one_sweep(o);
        memcpy(out + (int64_t)s * o->N, o->spin, (size_t)o->N);
    }
}
