// sw_api.cu -- host engine and C ABI of the Swendsen-Wang library.
//
// Owns the device state of each lattice, computes the integer bond
// thresholds (Sec. 2 step (ii) of Komura & Okabe; clock: Sec. 4 embedding),
// enqueues the sweep kernels (directly or as a captured CUDA graph), drains
// the per-sweep counter ring and turns counters into FP64 observables
// (Eq. 1, Eq. clock, Eq. M^2, Eq. U).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sw_internal.h"

using swgb::Batch;
using swgb::BatchSizes;
using swgb::DevState;
using swgb::LaunchShape;
using swgb::Lattice;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(SW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SW_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

// floor(p * 2^32) clamped to 2^32 - 1 with p = -expm1(-x) in double.
uint32_t threshold_of(double x)
{
    if (!(x > 0.0)) return 0u;
    const double p = -std::expm1(-x);
    const double scaled = std::floor(std::ldexp(p, 32));
    if (scaled >= 4294967295.0) return 0xffffffffu;
    if (scaled <= 0.0) return 0u;
    return (uint32_t)scaled;
}

// Clock-model bond thresholds (Sec. 4 embedding, J = 1) of every pair of
// projection classes a, b = (2k - m) mod 2q for the sweep's mirror axis m:
// 1 - exp(-2 K s_a s_b), K = 1 / T, with s = sin(pi (j mod q) / q) when both
// classes project strictly onto the same side of the axis, else 0; (2q)^2
// entries, each rounded as (2 K) (s_a s_b) in double.
std::vector<uint32_t> clock_thresholds(int q, double T)
{
    const double K = 1.0 / T;
    const int n2 = 2 * q;
    std::vector<uint32_t> tab((size_t)n2 * n2, 0u);
    for (int a = 0; a < n2; ++a) {
        for (int b = 0; b < n2; ++b) {
            const int side_a = (a % q == 0) ? 0 : (a < q ? 1 : -1);
            const int side_b = (b % q == 0) ? 0 : (b < q ? 1 : -1);
            if (side_a == 0 || side_a != side_b) continue;
            const double pa = std::sin((M_PI * (double)(a % q)) / (double)q);
            const double pb = std::sin((M_PI * (double)(b % q)) / (double)q);
            tab[(size_t)a * n2 + b] = threshold_of((2.0 * K) * (pa * pb));
        }
    }
    return tab;
}

int nclass_of(int q, int model) { return model == SW_CLOCK ? q / 2 + 1 : 2; }

// Counters per sweep: n_k, bond classes, active bonds, clusters; the clock
// model adds the class histograms of the pairs at distance L/4 and L/2.
int ncounters_of(int q, int model) { return q + nclass_of(q, model) + 2 + (model == SW_CLOCK ? 2 * nclass_of(q, model) : 0); }

}  // namespace

struct sw_handle {
    int L = 0, q = 0, model = 0;
    double T = 0.0;
    uint64_t seed = 0;
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false, own_spin = false, own_label = false;
    int8_t *d_spin = nullptr;
    int32_t *d_label = nullptr;
    uint32_t *d_thr_tab = nullptr;
    uint16_t *d_code = nullptr;
    unsigned long long *d_opar = nullptr;
    uint8_t *d_edge = nullptr;
    int32_t *d_open_count = nullptr;
    unsigned long long *d_stats = nullptr;   // labeling statistics (sw_set_labeling_stats)
    uint32_t *d_cross = nullptr;
    uint32_t *d_bond = nullptr;
    int tiles_x = 0, tiles_y = 0;
    DevState *d_st = nullptr;
    unsigned long long *d_ring = nullptr;
    // Batch-of-one view used by sw_sweep: descriptor, task / merge prefixes, ticket.
    Lattice *d_self = nullptr;
    BatchSizes *d_sizes = nullptr;
    int *d_task_off = nullptr;
    long long *d_merge_off = nullptr;
    unsigned int *d_ticket = nullptr;
    sw_batch *owner = nullptr;   // batch this lattice is attached to, if any
    // Comparator labeling (SW_LABEL_HAWICK / _KALENTEV): reference array,
    // convergence flag (device and pinned host word), passes of the last sweep.
    int labeling = SW_LABEL_TILED;
    int32_t *d_R = nullptr;
    unsigned int *d_flag = nullptr, *h_flag = nullptr;
    // Pinned staging of a counter drain (rows, device state block), so that
    // its copies are asynchronous and one stream synchronisation suffices.
    unsigned long long *h_rows = nullptr;
    size_t h_rows_cap = 0;
    DevState *h_st = nullptr;
    int last_passes = 0;
    uint32_t thr = 0;
    std::vector<uint32_t> thr_tab;
    int ncounters = 0, nclass = 0;
    int dbg_loop_cap = 0, dbg_list_cap = 0;   // test aids (sw_set_debug_limits)
    bool measure = true, labels = false, record = false, use_graph = false;
    LaunchShape shape;
    uint64_t t_host = 0;       // sweep index after all enqueued work
    uint64_t stop = swgb::kNoStop;   // sweeps run only while the index is below this (sw_set_sweep_limit)
    uint64_t t_drained = 0;    // first sweep whose counters are still on the device
    int sticky = SW_OK;
    std::string sticky_msg;
    // host statistics
    std::vector<int64_t> last_counts, history;
    bool have_last = false;
    uint64_t nmeas = 0;
    double sum_e = 0, sum_e2 = 0, sum_absm = 0, sum_m2 = 0, sum_m4 = 0, sum_active = 0, sum_clusters = 0;
    double sum_g4 = 0, sum_g2 = 0;   // clock: correlation at L/4 and L/2
    // captured sweep
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;

    Lattice lattice() const
    {
        Lattice lat{};
        lat.L = L;
        lat.q = q;
        lat.clock = model == SW_CLOCK;
        lat.thr = thr;
        lat.thr_tab = d_thr_tab;
        lat.key0 = (uint32_t)(seed & 0xffffffffu);
        lat.key1 = (uint32_t)(seed >> 32);
        lat.spin = d_spin;
        lat.label = d_label;
        lat.code = d_code;
        lat.opar = d_opar;
        lat.edge = d_edge;
        lat.open_count = d_open_count;
        lat.cross = d_cross;
        lat.bond = d_bond;
        lat.tiles_x = tiles_x;
        lat.tiles_y = tiles_y;
        lat.st = d_st;
        lat.ring = d_ring;
        lat.ring_slots = swgb::kRingSlots;
        lat.ncounters = ncounters;
        lat.nclass = nclass;
        lat.dbg_loop_cap = dbg_loop_cap;
        lat.dbg_list_cap = dbg_list_cap;
        lat.stats = d_stats;
        return lat;
    }

    int ntiles() const { return tiles_x * tiles_y; }
    int ntasks() const { return ntiles(); }
    long long nmerge() const { return (long long)ntiles() * swgb::kMergeItems; }

    Batch self_batch() const
    {
        Batch b{};
        b.dev = d_sizes;
        b.lat = d_self;
        b.task_off = d_task_off;
        b.merge_off = d_merge_off;
        b.ticket = d_ticket;
        b.nrep = 1;
        b.ntasks = ntasks();
        b.nmerge = nmerge();
        b.any_clock = model == SW_CLOCK;
        b.any_stats = d_stats != nullptr;
        return b;
    }
};

// A set of lattices swept together with one launch sequence per sweep.  The
// batch references handles it does not own (sw_batch_attach / _detach).
struct sw_batch {
    std::vector<sw_handle *> reps;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    bool measure = true, labels = false, use_graph = false;
    LaunchShape shape;
    // device descriptor arrays (capacity grows; contents rewritten on change)
    int cap = 0;
    BatchSizes *d_sizes = nullptr;   // the kernels read the sizes here (no recapture when they change)
    Lattice *d_lat = nullptr;
    int *d_task_off = nullptr;
    long long *d_merge_off = nullptr;
    unsigned int *d_ticket = nullptr;
    int ntasks = 0;
    long long nmerge = 0;
    bool any_clock = false, any_stats = false;
    int nrep = 0;                 // lattices in the descriptor arrays
    bool dirty = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;

    Batch view() const
    {
        Batch b{};
        b.dev = d_sizes;
        b.lat = d_lat;
        b.task_off = d_task_off;
        b.merge_off = d_merge_off;
        b.ticket = d_ticket;
        b.full_grid = 1;
        b.nrep = nrep;
        b.ntasks = ntasks;
        b.nmerge = nmerge;
        b.any_clock = any_clock;
        b.any_stats = any_stats;
        return b;
    }
};

namespace {

void drop_graph(sw_handle *h)
{
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
}

// Observables of one counter row (Sec. 4 measurement):
//   Potts E = number of unequal pairs (Eq. 1, J = 1); Ising E = -(equal - unequal);
//   clock E = -sum_d class_d cos(2 pi d / q);
//   Potts/Ising M^2 = (q sum n_k^2 - N^2)/(q - 1) (Eq. M^2), numerator exact;
//   clock M^2 = |sum_k n_k (cos, sin)(2 pi k / q)|^2.
void observables_of(int L, int q, int model, const int64_t *c, double out[4])
{
    const int64_t N = (int64_t)L * L;
    const double dN = (double)N;
    double E, M2;
    if (model == SW_CLOCK) {
        const int nclass = q / 2 + 1;
        E = 0.0;
        for (int d = 0; d < nclass; ++d) E -= (double)c[q + d] * std::cos(2.0 * M_PI * (double)d / (double)q);
        double mx = 0.0, my = 0.0;
        for (int k = 0; k < q; ++k) {
            mx += (double)c[k] * std::cos(2.0 * M_PI * (double)k / (double)q);
            my += (double)c[k] * std::sin(2.0 * M_PI * (double)k / (double)q);
        }
        M2 = mx * mx + my * my;
    } else {
        E = model == SW_ISING ? -(double)(c[q] - c[q + 1]) : (double)c[q + 1];
        __int128 s2 = 0;
        for (int k = 0; k < q; ++k) s2 += (__int128)c[k] * (__int128)c[k];
        const __int128 num = (__int128)q * s2 - (__int128)N * (__int128)N;
        M2 = (double)num / (double)(q - 1);
    }
    const double m2 = M2 / (dN * dN);
    out[0] = E / dN;
    out[1] = std::sqrt(M2) / dN;
    out[2] = m2;
    out[3] = m2 * m2;
}

// Clock model, Sec. 4: G(r) = <cos(theta_i - theta_{i+r})> over the 2N pairs
// at r = L/4 and r = L/2 (x and y displacements), from their class counts.
void correlations_of(int L, int q, const int64_t *c, double g[2])
{
    const int nclass = q / 2 + 1;
    const double pairs = 2.0 * (double)L * (double)L;
    for (int w = 0; w < 2; ++w) {
        const int64_t *hst = c + q + nclass + 2 + w * nclass;
        double s = 0.0;
        for (int d = 0; d < nclass; ++d) s += (double)hst[d] * std::cos(2.0 * M_PI * (double)d / (double)q);
        g[w] = s / pairs;
    }
}

void accumulate(sw_handle *h, const int64_t *row)
{
    double o[4];
    observables_of(h->L, h->q, h->model, row, o);
    h->nmeas++;
    h->sum_e += o[0];
    h->sum_e2 += o[0] * o[0];
    h->sum_absm += o[1];
    h->sum_m2 += o[2];
    h->sum_m4 += o[3];
    h->sum_active += (double)row[h->q + h->nclass];
    h->sum_clusters += (double)row[h->q + h->nclass + 1];
    if (h->model == SW_CLOCK) {
        double g[2];
        correlations_of(h->L, h->q, row, g);
        h->sum_g4 += g[0];
        h->sum_g2 += g[1];
    }
    h->last_counts.assign(row, row + h->ncounters);
    h->have_last = true;
    if (h->record) h->history.insert(h->history.end(), row, row + h->ncounters);
}

// Fold the device state block's error word into the handle's sticky status.
int sticky_from(sw_handle *h, const DevState &st)
{
    if (st.err != swgb::kErrNone && h->sticky == SW_OK) {
        h->sticky = SW_ERR_NOT_CONVERGED;
        char buf[160];
        snprintf(buf, sizeof buf, "device loop bound exceeded (code %d at index %d)", st.err, st.err_where);
        h->sticky_msg = buf;
    }
    if (h->sticky != SW_OK) return fail(h->sticky, "%s", h->sticky_msg.c_str());
    return SW_OK;
}

int check_device_error(sw_handle *h)
{
    DevState st;
    SW_CUDA(cudaMemcpyAsync(&st, h->d_st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    return sticky_from(h, st);
}

// Wait for the stream and fold every pending measured sweep into the host
// statistics, oldest first.
int drain(sw_handle *h)
{
    const uint64_t pending = h->t_host - h->t_drained;
    const bool rows = pending > 0 && h->measure;
    const size_t nc = (size_t)h->ncounters;
    if (!h->h_st) SW_CUDA(cudaHostAlloc(&h->h_st, sizeof(DevState), cudaHostAllocDefault));
    if (rows && h->h_rows_cap < (size_t)pending * nc) {
        if (h->h_rows) cudaFreeHost(h->h_rows);
        h->h_rows = nullptr;
        h->h_rows_cap = 0;
        const size_t cap = std::max((size_t)pending, (size_t)8) * nc;
        SW_CUDA(cudaHostAlloc(&h->h_rows, cap * sizeof(unsigned long long), cudaHostAllocDefault));
        h->h_rows_cap = cap;
    }
    if (rows) {
        // The bond classes of the newest configuration are normally counted
        // by the next sweep's labeling pass; count them now.
        cudaError_t e = swgb::launch_pending_classes(h->lattice(), h->sm_count, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "launch_pending_classes");
        // Copy only the pending rows (at most two contiguous ring segments).
        const size_t first = (size_t)(h->t_drained % swgb::kRingSlots);
        const size_t n1 = std::min((size_t)pending, (size_t)swgb::kRingSlots - first);
        SW_CUDA(cudaMemcpyAsync(h->h_rows, h->d_ring + first * nc, n1 * nc * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, h->stream));
        if (n1 < pending)
            SW_CUDA(cudaMemcpyAsync(h->h_rows + n1 * nc, h->d_ring, ((size_t)pending - n1) * nc *
                                    sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    }
    // The device state block (error word), behind everything enqueued so far.
    SW_CUDA(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    if (rows) {
        std::vector<int64_t> row(nc);
        for (size_t k = 0; k < (size_t)pending; ++k) {
            for (size_t c = 0; c < nc; ++c) row[c] = (int64_t)h->h_rows[k * nc + c];
            accumulate(h, row.data());
        }
    }
    h->t_drained = h->t_host;
    return sticky_from(h, *h->h_st);
}

int reset_device_index(sw_handle *h, uint64_t t)
{
    DevState st{};
    st.sweep = t;
    st.stop = h->stop;
    st.classes_upto = t;   // the current configuration is not a sweep result of this run
    st.next_t = t;
    SW_CUDA(cudaMemcpyAsync(h->d_st, &st, sizeof st, cudaMemcpyHostToDevice, h->stream));
    SW_CUDA(cudaMemsetAsync(h->d_ring, 0, sizeof(unsigned long long) * swgb::kRingSlots * h->ncounters, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    h->t_host = h->t_drained = t;
    h->sticky = SW_OK;
    return SW_OK;
}

// The label array of h, allocated (and zeroed) on first use; the device
// descriptors that hold its address are rewritten.
int ensure_labels(sw_handle *h)
{
    if (h->d_label) return SW_OK;
    const size_t n = (size_t)h->L * h->L * sizeof(int32_t);
    cudaError_t e = cudaMalloc(&h->d_label, n);
    if (e != cudaSuccess) {
        h->d_label = nullptr;
        return fail(SW_ERR_OOM, "cudaMalloc(labels, %zu bytes): %s", n, cudaGetErrorString(e));
    }
    h->own_label = true;
    SW_CUDA(cudaMemsetAsync(h->d_label, 0, n, h->stream));
    const Lattice self = h->lattice();
    SW_CUDA(cudaMemcpyAsync(h->d_self, &self, sizeof self, cudaMemcpyHostToDevice, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    if (h->owner) h->owner->dirty = true;
    return SW_OK;
}

// One sweep of batch view b on stream s, from a captured graph when asked.
int enqueue_sweep(const Batch &b, bool measure, bool labels, int sm_count, const LaunchShape &shape, cudaStream_t s,
                  bool use_graph, cudaGraph_t *graph, cudaGraphExec_t *exec)
{
    if (use_graph) {
        if (!*exec) {
            SW_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            cudaError_t le = swgb::launch_sweep(b, measure, labels, sm_count, shape, s);
            cudaError_t ce = cudaStreamEndCapture(s, graph);
            if (le != cudaSuccess) return cuda_fail(le, "launch_sweep (capture)");
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
            SW_CUDA(cudaGraphInstantiate(exec, *graph, 0));
        }
        SW_CUDA(cudaGraphLaunch(*exec, s));
        return SW_OK;
    }
    cudaError_t e = swgb::launch_sweep(b, measure, labels, sm_count, shape, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch_sweep");
    return SW_OK;
}

// n sweeps of view b with CUDA events around every kernel; per-stage mean
// milliseconds into ms[kMaxStages].  before() runs ahead of every sweep
// (counter drains), after() once it is enqueued (sweep bookkeeping).
template <typename Before, typename After>
int timed_sweeps(const Batch &b, bool measure, bool labels, int sm_count, const LaunchShape &shape, cudaStream_t s,
                 int n, double *ms, Before before, After after)
{
    const int nstages = swgb::kMaxStages;
    cudaEvent_t ev[swgb::kMaxStages + 1];
    for (int k = 0; k <= nstages; ++k) SW_CUDA(cudaEventCreate(&ev[k]));
    for (int k = 0; k < nstages; ++k) ms[k] = 0.0;
    int rc = SW_OK;
    for (int i = 0; i < n && rc == SW_OK; ++i) {
        rc = before();
        if (rc != SW_OK) break;
        cudaError_t e = swgb::launch_sweep(b, measure, labels, sm_count, shape, s, ev);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "launch_sweep");
            break;
        }
        after();
        e = cudaEventSynchronize(ev[nstages]);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cudaEventSynchronize");
            break;
        }
        for (int k = 0; k < nstages; ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            ms[k] += t / n;
        }
    }
    for (int k = 0; k <= nstages; ++k) cudaEventDestroy(ev[k]);
    return rc;
}

// Launch shapes chosen so far, per device and work size (process-wide).
std::mutex g_tune_mu;
std::map<std::string, LaunchShape> g_tune_cache;

std::string tune_key(int nrep, int ntasks, long long nmerge, bool measure, bool any_clock)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    char buf[384];
    snprintf(buf, sizeof buf, "%s|%d|%d|%lld|%d|%d", prop.name, nrep, ntasks, nmerge, (int)measure, (int)any_clock);
    return buf;
}

// Coordinate descent over the blocks per SM of each kernel: every
// candidate runs n timed sweeps (real sweeps of the chain).  The bond
// kernel's figure is tuned only where the sweep launches it (a clock lattice).
template <typename Timer>
int autotune_shape(LaunchShape *best, int n, bool tune_bonds, Timer timer)
{
    static const int cand_label[] = {7, 9, 11};
    static const int cand_other[] = {4, 8, 16, 32};
    double ms[swgb::kMaxStages];
    // Timed stages: 0 bonds, 1 labeling, 2 merge, 3 flip.
    static const int stage_of[4] = {1, 2, 3, 0};   // tuned in the order label, merge, flip, bonds
    for (int k = 0; k < (tune_bonds ? 4 : 3); ++k) {
        const int *cand = k == 0 ? cand_label : cand_other;
        const int ncand = k == 0 ? 3 : 4;
        double best_ms = 1e30;
        LaunchShape pick = *best;
        for (int i = 0; i < ncand; ++i) {
            LaunchShape trial = *best;
            int *field = k == 0 ? &trial.label : k == 1 ? &trial.merge : k == 2 ? &trial.flip : &trial.bonds;
            *field = cand[i];
            int rc = timer(trial, n, ms);
            if (rc != SW_OK) return rc;
            if (ms[stage_of[k]] < best_ms) {
                best_ms = ms[stage_of[k]];
                pick = trial;
            }
        }
        *best = pick;
    }
    return SW_OK;
}

// Upper bound on the passes of a comparator labeling (the paper reports
// fewer than ten at T_c; chains can only shorten, so this never binds for a
// well-formed lattice).
constexpr int kMaxLabelPasses = 100000;

int enqueue_one(sw_handle *h)
{
    if (h->labeling != SW_LABEL_TILED) {
        int passes = 0;
        cudaError_t e = swgb::equivalence_sweep(h->self_batch(), h->lattice(), h->labeling, h->sm_count, h->stream,
                                                h->d_R, h->d_flag, h->h_flag, kMaxLabelPasses, &passes);
        if (e != cudaSuccess) return cuda_fail(e, "equivalence_sweep");
        if (passes < 0) {
            h->sticky = SW_ERR_NOT_CONVERGED;
            h->sticky_msg = "comparator labeling did not converge";
            return fail(h->sticky, "%s", h->sticky_msg.c_str());
        }
        h->last_passes = passes;
        return SW_OK;
    }
    return enqueue_sweep(h->self_batch(), h->measure, h->labels, h->sm_count, h->shape, h->stream, h->use_graph,
                         &h->graph, &h->graph_exec);
}

void free_handle(sw_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    if (h->own_spin && h->d_spin) cudaFree(h->d_spin);
    if (h->own_label && h->d_label) cudaFree(h->d_label);
    if (h->d_thr_tab) cudaFree(h->d_thr_tab);
    if (h->d_code) cudaFree(h->d_code);
    if (h->d_opar) cudaFree(h->d_opar);
    if (h->d_edge) cudaFree(h->d_edge);
    if (h->d_open_count) cudaFree(h->d_open_count);
    if (h->d_cross) cudaFree(h->d_cross);
    if (h->d_R) cudaFree(h->d_R);
    if (h->d_flag) cudaFree(h->d_flag);
    if (h->h_flag) cudaFreeHost(h->h_flag);
    if (h->h_rows) cudaFreeHost(h->h_rows);
    if (h->h_st) cudaFreeHost(h->h_st);
    if (h->d_bond) cudaFree(h->d_bond);
    if (h->d_st) cudaFree(h->d_st);
    if (h->d_ring) cudaFree(h->d_ring);
    if (h->d_stats) cudaFree(h->d_stats);
    if (h->d_self) cudaFree(h->d_self);
    if (h->d_task_off) cudaFree(h->d_task_off);
    if (h->d_sizes) cudaFree(h->d_sizes);
    if (h->d_merge_off) cudaFree(h->d_merge_off);
    if (h->d_ticket) cudaFree(h->d_ticket);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int validate(int L, int q, int model, double T)
{
    if (model != SW_POTTS && model != SW_CLOCK && model != SW_ISING)
        return fail(SW_ERR_ARG, "unknown model %d", model);
    if (L < 4 || L % 4 != 0 || L > 46340)
        return fail(SW_ERR_ARG, "L=%d: need 4 <= L <= 46340 and L %% 4 == 0", L);
    if (model == SW_ISING && q != 2) return fail(SW_ERR_ARG, "Ising needs q = 2 (got %d)", q);
    if (q < 2 || q > SW_MAX_Q) return fail(SW_ERR_ARG, "q=%d out of [2, %d]", q, SW_MAX_Q);
    if (model == SW_CLOCK && q > SW_MAX_CLOCK_Q) return fail(SW_ERR_ARG, "clock q=%d > %d", q, SW_MAX_CLOCK_Q);
    if (!(T > 0.0) || !std::isfinite(T)) return fail(SW_ERR_ARG, "T=%g must be positive and finite", T);
    return SW_OK;
}

sw_handle *create_impl(int L, int q, int model, double T, uint64_t seed, void *d_spins, void *d_labels,
                       void *stream, bool have_stream)
{
    if (validate(L, q, model, T) != SW_OK) return nullptr;
    if ((d_spins && ((uintptr_t)d_spins & 15)) || (d_labels && ((uintptr_t)d_labels & 15))) {
        fail(SW_ERR_ARG, "borrowed buffers must be 16-byte aligned");
        return nullptr;
    }
    sw_handle *h = new (std::nothrow) sw_handle();
    if (!h) {
        fail(SW_ERR_OOM, "host allocation failed");
        return nullptr;
    }
    h->L = L;
    h->q = q;
    h->model = model;
    h->T = T;
    h->seed = seed;
    h->nclass = nclass_of(q, model);
    h->ncounters = ncounters_of(q, model);
    const size_t N = (size_t)L * L;
    auto bail = [&](cudaError_t e, const char *what) -> sw_handle * {
        cuda_fail(e, what);
        free_handle(h);
        return nullptr;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return bail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
        return bail(e, "cudaDeviceGetAttribute");
    if (have_stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e, "cudaStreamCreate");
        h->own_stream = true;
    }
    if (d_spins) {
        h->d_spin = (int8_t *)d_spins;
    } else {
        if ((e = cudaMalloc(&h->d_spin, N)) != cudaSuccess) return bail(e, "cudaMalloc(spins)");
        h->own_spin = true;
    }
    // The label array is only written with debug labels on or by a
    // comparator labeling; it is allocated when one of them is enabled.
    if (d_labels) h->d_label = (int32_t *)d_labels;
    if ((e = cudaMalloc(&h->d_st, sizeof(DevState))) != cudaSuccess) return bail(e, "cudaMalloc(state)");
    h->tiles_x = (L + swgb::kTileW - 1) / swgb::kTileW;
    h->tiles_y = (L + swgb::kTileH - 1) / swgb::kTileH;
    const size_t ntiles = (size_t)h->tiles_x * h->tiles_y;
    if ((e = cudaMalloc(&h->d_code, N * sizeof(uint16_t))) != cudaSuccess) return bail(e, "cudaMalloc(codes)");
    if ((e = cudaMalloc(&h->d_opar, ntiles * swgb::kOpenSlots * sizeof(unsigned long long))) != cudaSuccess)
        return bail(e, "cudaMalloc(open components)");
    if ((e = cudaMalloc(&h->d_edge, ntiles * swgb::kEdgeBytes)) != cudaSuccess) return bail(e, "cudaMalloc(edges)");
    if ((e = cudaMalloc(&h->d_open_count, ntiles * sizeof(int32_t))) != cudaSuccess)
        return bail(e, "cudaMalloc(open counts)");
    if ((e = cudaMalloc(&h->d_cross, ntiles * swgb::kCrossWords * sizeof(uint32_t))) != cudaSuccess)
        return bail(e, "cudaMalloc(crossing bonds)");
    if ((e = cudaMalloc(&h->d_bond, ntiles * swgb::kBondWords * sizeof(uint32_t))) != cudaSuccess)
        return bail(e, "cudaMalloc(bond masks)");
    if ((e = cudaMalloc(&h->d_ring, sizeof(unsigned long long) * swgb::kRingSlots * h->ncounters)) != cudaSuccess)
        return bail(e, "cudaMalloc(ring)");

    // Bond thresholds (Sec. 2 step (ii); clock: Sec. 4 embedding), J = 1.
    const double K = 1.0 / T;
    if (model == SW_POTTS) {
        h->thr = threshold_of(K);
    } else if (model == SW_ISING) {
        h->thr = threshold_of(2.0 * K);
    } else {
        h->thr_tab = clock_thresholds(q, T);
        if ((e = cudaMalloc(&h->d_thr_tab, h->thr_tab.size() * sizeof(uint32_t))) != cudaSuccess)
            return bail(e, "cudaMalloc(thresholds)");
        if ((e = cudaMemcpy(h->d_thr_tab, h->thr_tab.data(), h->thr_tab.size() * sizeof(uint32_t),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "cudaMemcpy(thresholds)");
    }
    // Batch-of-one view.
    {
        const Lattice self = h->lattice();
        const int task_off[2] = {0, h->ntasks()};
        const long long merge_off[2] = {0, h->nmerge()};
        if ((e = cudaMalloc(&h->d_self, sizeof(Lattice))) != cudaSuccess) return bail(e, "cudaMalloc(descriptor)");
        if ((e = cudaMalloc(&h->d_task_off, sizeof task_off)) != cudaSuccess) return bail(e, "cudaMalloc(tasks)");
        if ((e = cudaMalloc(&h->d_merge_off, sizeof merge_off)) != cudaSuccess) return bail(e, "cudaMalloc(merge)");
        if ((e = cudaMalloc(&h->d_ticket, sizeof(unsigned int))) != cudaSuccess) return bail(e, "cudaMalloc(ticket)");
        const BatchSizes sizes{1, h->ntasks(), h->nmerge()};
        if ((e = cudaMalloc(&h->d_sizes, sizeof sizes)) != cudaSuccess) return bail(e, "cudaMalloc(sizes)");
        if ((e = cudaMemcpy(h->d_sizes, &sizes, sizeof sizes, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "cudaMemcpy(sizes)");
        if ((e = cudaMemcpy(h->d_self, &self, sizeof self, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "cudaMemcpy(descriptor)");
        if ((e = cudaMemcpy(h->d_task_off, task_off, sizeof task_off, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "cudaMemcpy(tasks)");
        if ((e = cudaMemcpy(h->d_merge_off, merge_off, sizeof merge_off, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "cudaMemcpy(merge)");
        if ((e = cudaMemset(h->d_ticket, 0, sizeof(unsigned int))) != cudaSuccess) return bail(e, "cudaMemset(ticket)");
    }
    if (reset_device_index(h, 0) != SW_OK) {
        free_handle(h);
        return nullptr;
    }
    if ((e = cudaMemsetAsync(h->d_spin, 0, N, h->stream)) != cudaSuccess) return bail(e, "cudaMemset(spins)");
    if (h->d_label && (e = cudaMemsetAsync(h->d_label, 0, N * sizeof(int32_t), h->stream)) != cudaSuccess)
        return bail(e, "cudaMemset(labels)");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(e, "cudaStreamSynchronize");
    return h;
}

}  // namespace

extern "C" {

int sw_ncounters(int q, int model) { return ncounters_of(q, model); }

const char *sw_last_error(void) { return g_err.c_str(); }

sw_handle *sw_create(int L, int q, int model, double T, uint64_t seed)
{
    return create_impl(L, q, model, T, seed, nullptr, nullptr, nullptr, false);
}

sw_handle *sw_create_ext(int L, int q, int model, double T, uint64_t seed, void *d_spins, void *d_labels,
                         void *stream)
{
    return create_impl(L, q, model, T, seed, d_spins, d_labels, stream, true);
}

int sw_destroy(sw_handle *h)
{
    if (h && h->owner) sw_batch_detach(h->owner, h);
    free_handle(h);
    return SW_OK;
}

int sw_init(sw_handle *h, int mode)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (mode != SW_INIT_UP && mode != SW_INIT_RANDOM) return fail(SW_ERR_ARG, "unknown init mode %d", mode);
    cudaError_t e = swgb::launch_init(h->lattice(), mode == SW_INIT_RANDOM, h->sm_count, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch_init");
    SW_CUDA(cudaStreamSynchronize(h->stream));
    return SW_OK;
}

int sw_sweep(sw_handle *h, int n)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (n < 0) return fail(SW_ERR_ARG, "n=%d < 0", n);
    if (h->sticky != SW_OK) return fail(h->sticky, "%s", h->sticky_msg.c_str());
    for (int s = 0; s < n && h->t_host < h->stop; ++s) {
        if (h->measure && h->t_host - h->t_drained >= (uint64_t)swgb::kRingSlots - 1) {
            int rc = drain(h);
            if (rc != SW_OK) return rc;
        }
        int rc = enqueue_one(h);
        if (rc != SW_OK) return rc;
        h->t_host++;
        if (!h->measure) h->t_drained = h->t_host;
    }
    return SW_OK;
}

int sw_synchronize(sw_handle *h)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    SW_CUDA(cudaStreamSynchronize(h->stream));
    return check_device_error(h);
}

int sw_measure(sw_handle *h, sw_obs *out)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    if (!out) return SW_OK;
    std::memset(out, 0, sizeof *out);
    out->sweep = h->t_host;
    out->L = h->L;
    out->q = h->q;
    out->model = h->model;
    out->ncounters = h->ncounters;
    if (h->have_last) {
        for (int c = 0; c < h->ncounters; ++c) out->counts[c] = h->last_counts[c];
        double o[4];
        observables_of(h->L, h->q, h->model, h->last_counts.data(), o);
        out->e = o[0];
        out->absm = o[1];
        out->m2 = o[2];
        out->m4 = o[3];
        if (h->model == SW_CLOCK) {
            double g[2];
            correlations_of(h->L, h->q, h->last_counts.data(), g);
            out->g_quarter = g[0];
            out->g_half = g[1];
        }
    }
    out->nmeas = h->nmeas;
    if (h->nmeas) {
        const double n = (double)h->nmeas;
        out->mean_e = h->sum_e / n;
        out->mean_e2 = h->sum_e2 / n;
        out->mean_absm = h->sum_absm / n;
        out->mean_m2 = h->sum_m2 / n;
        out->mean_m4 = h->sum_m4 / n;
        out->binder_u = out->mean_m2 > 0 ? out->mean_m4 / (out->mean_m2 * out->mean_m2) : 0.0;
        out->mean_active = h->sum_active / n;
        out->mean_clusters = h->sum_clusters / n;
        if (h->model == SW_CLOCK) {
            out->mean_g_quarter = h->sum_g4 / n;
            out->mean_g_half = h->sum_g2 / n;
            out->corr_ratio = out->mean_g_quarter != 0.0 ? out->mean_g_half / out->mean_g_quarter : 0.0;
        }
    }
    return SW_OK;
}

int sw_set_measure(sw_handle *h, int on)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (on && h->labeling != SW_LABEL_TILED) return fail(SW_ERR_STATE, "the comparator labelings are update only");
    if (h->owner) return fail(SW_ERR_STATE, "lattice is attached to a batch; use sw_batch_set_measure");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    if (h->measure != (on != 0)) drop_graph(h);
    h->measure = on != 0;
    return SW_OK;
}

int sw_set_record(sw_handle *h, int on)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    h->record = on != 0;
    if (!h->record) h->history.clear();
    return SW_OK;
}

int sw_take_counts(sw_handle *h, int64_t *out, int max_rows)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (max_rows < 0 || (max_rows > 0 && !out)) return fail(SW_ERR_ARG, "bad output buffer");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    const size_t have = h->history.size() / h->ncounters;
    const size_t n = std::min(have, (size_t)max_rows);
    std::memcpy(out, h->history.data(), n * h->ncounters * sizeof(int64_t));
    h->history.erase(h->history.begin(), h->history.begin() + n * h->ncounters);
    return (int)n;
}

int sw_reset_stats(sw_handle *h)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    h->nmeas = 0;
    h->sum_e = h->sum_e2 = h->sum_absm = h->sum_m2 = h->sum_m4 = h->sum_active = h->sum_clusters = 0.0;
    h->sum_g4 = h->sum_g2 = 0.0;
    return SW_OK;
}

int sw_set_debug_labels(sw_handle *h, int on)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (on) {
        int rc = drain(h);
        if (rc == SW_OK) rc = ensure_labels(h);
        if (rc != SW_OK) return rc;
    }
    if (h->labels != (on != 0)) drop_graph(h);
    h->labels = on != 0;
    return SW_OK;
}

int sw_get_spins(sw_handle *h, int8_t *host, size_t n)
{
    if (!h || !host) return fail(SW_ERR_ARG, "null argument");
    if (n != (size_t)h->L * h->L) return fail(SW_ERR_ARG, "n=%zu != L*L", n);
    SW_CUDA(cudaMemcpyAsync(host, h->d_spin, n, cudaMemcpyDeviceToHost, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    return SW_OK;
}

int sw_set_spins(sw_handle *h, const int8_t *host, size_t n)
{
    if (!h || !host) return fail(SW_ERR_ARG, "null argument");
    if (n != (size_t)h->L * h->L) return fail(SW_ERR_ARG, "n=%zu != L*L", n);
    SW_CUDA(cudaMemcpyAsync(h->d_spin, host, n, cudaMemcpyHostToDevice, h->stream));
    // Range check on the device: the scratch word of the state block.
    unsigned int *bad = &h->d_st->scratch;
    SW_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), h->stream));
    cudaError_t e = swgb::launch_count_invalid(h->lattice(), bad, h->sm_count, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch_count_invalid");
    unsigned int nbad = 0;
    SW_CUDA(cudaMemcpyAsync(&nbad, bad, sizeof nbad, cudaMemcpyDeviceToHost, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    if (nbad) {
        // Leave a valid configuration behind: every kernel assumes states in [0, q).
        SW_CUDA(cudaMemsetAsync(h->d_spin, 0, n, h->stream));
        SW_CUDA(cudaStreamSynchronize(h->stream));
        return fail(SW_ERR_ARG, "%u spins outside [0, %d); the lattice was reset to state 0", nbad, h->q);
    }
    return SW_OK;
}

int sw_get_labels(sw_handle *h, int32_t *host, size_t n)
{
    if (!h || !host) return fail(SW_ERR_ARG, "null argument");
    if (n != (size_t)h->L * h->L) return fail(SW_ERR_ARG, "n=%zu != L*L", n);
    if (!h->d_label) return fail(SW_ERR_STATE, "no labels: turn debug labels on before sweeping");
    SW_CUDA(cudaMemcpyAsync(host, h->d_label, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    return SW_OK;
}

void *sw_device_spins(sw_handle *h) { return h ? (void *)h->d_spin : nullptr; }
void *sw_device_labels(sw_handle *h) { return h ? (void *)h->d_label : nullptr; }

int sw_get_thresholds(sw_handle *h, uint32_t *out, int n)
{
    if (!h || !out) return fail(SW_ERR_ARG, "null argument");
    if (h->model == SW_CLOCK) {
        const int m = (int)h->thr_tab.size();
        if (n < m) return fail(SW_ERR_ARG, "need %d entries", m);
        std::memcpy(out, h->thr_tab.data(), (size_t)m * sizeof(uint32_t));
        return m;
    }
    if (n < 1) return fail(SW_ERR_ARG, "need 1 entry");
    out[0] = h->thr;
    return 1;
}

int sw_get_sweep(sw_handle *h, uint64_t *out)
{
    if (!h || !out) return fail(SW_ERR_ARG, "null argument");
    *out = h->t_host;
    return SW_OK;
}

int sw_set_sweep(sw_handle *h, uint64_t t)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    return reset_device_index(h, t);
}

int sw_set_stream(sw_handle *h, void *stream)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (h->owner) return fail(SW_ERR_STATE, "lattice is attached to a batch; it runs on the batch's stream");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    if (h->own_stream) cudaStreamDestroy(h->stream);
    h->own_stream = false;
    h->stream = (cudaStream_t)stream;
    drop_graph(h);
    return SW_OK;
}

int sw_profile_sweeps(sw_handle *h, int n, float *ms, int max_stages)
{
    if (!h || !ms) return fail(SW_ERR_ARG, "null argument");
    if (h->labeling != SW_LABEL_TILED) return fail(SW_ERR_STATE, "stage profile needs the tiled labeling");
    if (n < 1 || max_stages < 1) return fail(SW_ERR_ARG, "n and max_stages must be positive");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    double acc[swgb::kMaxStages];
    rc = timed_sweeps(
        h->self_batch(), h->measure, h->labels, h->sm_count, h->shape, h->stream, n, acc,
        [&]() -> int {
            return (h->measure && h->t_host - h->t_drained >= (uint64_t)swgb::kRingSlots - 1) ? drain(h) : (int)SW_OK;
        },
        [&]() {
            if (h->t_host < h->stop) h->t_host++;   // skipped at its limit
            if (!h->measure) h->t_drained = h->t_host;
        });
    if (rc != SW_OK) return rc;
    const int m = std::min(swgb::kMaxStages, max_stages);
    for (int k = 0; k < m; ++k) ms[k] = (float)acc[k];
    rc = drain(h);
    return rc != SW_OK ? rc : m;
}

int sw_autotune(sw_handle *h, int n, int *shape_out)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (h->labeling != SW_LABEL_TILED) return fail(SW_ERR_STATE, "autotuning needs the tiled labeling");
    if (n < 1) return fail(SW_ERR_ARG, "n must be positive");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    const std::string key = tune_key(1, h->ntasks(), h->nmerge(), h->measure, h->model == SW_CLOCK);
    LaunchShape best;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        rc = autotune_shape(&best, n, h->model == SW_CLOCK, [&](const LaunchShape &trial, int nn, double *ms) {
            return timed_sweeps(
                h->self_batch(), h->measure, h->labels, h->sm_count, trial, h->stream, nn, ms,
                [&]() -> int {
                    return (h->measure && h->t_host - h->t_drained >= (uint64_t)swgb::kRingSlots - 1) ? drain(h)
                                                                                                       : (int)SW_OK;
                },
                [&]() {
                    if (h->t_host < h->stop) h->t_host++;   // skipped at its limit
                    if (!h->measure) h->t_drained = h->t_host;
                });
        });
        if (rc != SW_OK) return rc;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    h->shape = best;
    drop_graph(h);
    if (shape_out) {
        shape_out[0] = best.label;
        shape_out[1] = best.merge;
        shape_out[2] = best.flip;
        shape_out[3] = best.bonds;
    }
    return drain(h);
}

int sw_set_launch_shape(sw_handle *h, const int *shape)
{
    if (!h || !shape) return fail(SW_ERR_ARG, "null argument");
    for (int k = 0; k < 4; ++k)
        if (shape[k] < 1 || shape[k] > 64) return fail(SW_ERR_ARG, "blocks per SM must be in [1, 64]");
    h->shape.label = shape[0];
    h->shape.merge = shape[1];
    h->shape.flip = shape[2];
    h->shape.bonds = shape[3];
    drop_graph(h);
    return SW_OK;
}

int sw_set_labeling(sw_handle *h, int method)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (method != SW_LABEL_TILED && method != SW_LABEL_HAWICK && method != SW_LABEL_KALENTEV)
        return fail(SW_ERR_ARG, "unknown labeling %d", method);
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    if (method != SW_LABEL_TILED) {
        if (h->owner) return fail(SW_ERR_STATE, "lattice is attached to a batch");
        if (h->measure) return fail(SW_ERR_STATE, "the comparator labelings are update only: turn measurement off");
        if (!h->d_flag) SW_CUDA(cudaMalloc(&h->d_flag, sizeof(unsigned int)));
        if (!h->h_flag) SW_CUDA(cudaHostAlloc(&h->h_flag, sizeof(unsigned int), cudaHostAllocDefault));
        if (method == SW_LABEL_HAWICK && !h->d_R) SW_CUDA(cudaMalloc(&h->d_R, (size_t)h->L * h->L * sizeof(int32_t)));
        rc = ensure_labels(h);
        if (rc != SW_OK) return rc;
    }
    h->labeling = method;
    h->last_passes = 0;
    return SW_OK;
}

int sw_label_passes(sw_handle *h)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    return h->last_passes;
}

int sw_set_debug_limits(sw_handle *h, int loop_cap, int list_cap)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (loop_cap < 0 || list_cap < 0) return fail(SW_ERR_ARG, "limits must be >= 0 (0: default)");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    h->dbg_loop_cap = loop_cap;
    h->dbg_list_cap = list_cap;
    const Lattice self = h->lattice();
    SW_CUDA(cudaMemcpyAsync(h->d_self, &self, sizeof self, cudaMemcpyHostToDevice, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    if (h->owner) h->owner->dirty = true;
    return SW_OK;
}

int sw_set_labeling_stats(sw_handle *h, int on)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    if (on && !h->d_stats) SW_CUDA(cudaMalloc(&h->d_stats, sizeof(unsigned long long) * swgb::kStatFields));
    if (!on && h->d_stats) {
        cudaFree(h->d_stats);
        h->d_stats = nullptr;
    }
    if (h->d_stats)
        SW_CUDA(cudaMemsetAsync(h->d_stats, 0, sizeof(unsigned long long) * swgb::kStatFields, h->stream));
    const Lattice self = h->lattice();
    SW_CUDA(cudaMemcpyAsync(h->d_self, &self, sizeof self, cudaMemcpyHostToDevice, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    drop_graph(h);   // the kernel variants depend on it
    if (h->owner) h->owner->dirty = true;
    return SW_OK;
}

int sw_get_labeling_stats(sw_handle *h, double *out, int n)
{
    if (!h || !out) return fail(SW_ERR_ARG, "null argument");
    if (!h->d_stats) return fail(SW_ERR_STATE, "labeling statistics are off (sw_set_labeling_stats)");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    unsigned long long a[swgb::kStatFields];
    SW_CUDA(cudaMemcpyAsync(a, h->d_stats, sizeof a, cudaMemcpyDeviceToHost, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    const double sweeps = (double)a[swgb::kStatSweeps];
    const double ts = sweeps * (double)h->ntiles();
    auto ratio = [](double x, double y) { return y > 0.0 ? x / y : 0.0; };
    const double v[11] = {
        sweeps,
        ratio((double)a[swgb::kStatLabels], ts),
        ratio((double)a[swgb::kStatPairs], ts),
        ratio((double)a[swgb::kStatComponents], ts),
        ratio((double)a[swgb::kStatOpen], ts),
        ratio((double)a[swgb::kStatUnions], sweeps),
        ratio((double)a[swgb::kStatLinks], (double)a[swgb::kStatUnions]),
        ratio((double)a[swgb::kStatRetries], (double)a[swgb::kStatLinks]),
        ratio((double)a[swgb::kStatFinds], sweeps),
        ratio((double)a[swgb::kStatHops], (double)a[swgb::kStatFinds]),
        (double)a[swgb::kStatMaxHops],
    };
    const int m = std::min(n, 11);
    for (int i = 0; i < m; ++i) out[i] = v[i];
    return m;
}

int sw_set_sweep_limit(sw_handle *h, uint64_t stop)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    h->stop = stop;
    SW_CUDA(cudaMemcpyAsync(&h->d_st->stop, &h->stop, sizeof h->stop, cudaMemcpyHostToDevice, h->stream));
    SW_CUDA(cudaStreamSynchronize(h->stream));
    return SW_OK;
}

int sw_get_sweep_limit(sw_handle *h, uint64_t *out)
{
    if (!h || !out) return fail(SW_ERR_ARG, "null argument");
    *out = h->stop;
    return SW_OK;
}

int sw_set_graph(sw_handle *h, int on)
{
    if (!h) return fail(SW_ERR_ARG, "null handle");
    if (h->use_graph != (on != 0)) drop_graph(h);
    h->use_graph = on != 0;
    return SW_OK;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
static void drop_batch_graph(sw_batch *b)
{
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
}

static void free_batch_arrays(sw_batch *b)
{
    if (b->d_lat) cudaFree(b->d_lat);
    if (b->d_task_off) cudaFree(b->d_task_off);
    if (b->d_merge_off) cudaFree(b->d_merge_off);
    b->d_lat = nullptr;
    b->d_task_off = nullptr;
    b->d_merge_off = nullptr;
    b->cap = 0;
}

// Rewrite the device descriptor arrays from the attached lattices.
static int rebuild_batch(sw_batch *b)
{
    const int n = (int)b->reps.size();
    if (n > b->cap) {
        drop_batch_graph(b);
        free_batch_arrays(b);
        const int cap = std::max(16, std::max(n, 2 * b->cap));
        SW_CUDA(cudaMalloc(&b->d_lat, sizeof(Lattice) * cap));
        SW_CUDA(cudaMalloc(&b->d_task_off, sizeof(int) * (cap + 1)));
        SW_CUDA(cudaMalloc(&b->d_merge_off, sizeof(long long) * (cap + 1)));
        b->cap = cap;
    }
    std::vector<Lattice> lat(n);
    std::vector<int> task_off(n + 1, 0);
    std::vector<long long> merge_off(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        lat[i] = b->reps[i]->lattice();
        task_off[i + 1] = task_off[i] + b->reps[i]->ntasks();
        merge_off[i + 1] = merge_off[i] + b->reps[i]->nmerge();
    }
    bool any_clock = false, any_stats = false;
    for (int i = 0; i < n; ++i) {
        any_clock = any_clock || b->reps[i]->model == SW_CLOCK;
        any_stats = any_stats || b->reps[i]->d_stats != nullptr;
    }
    // A captured graph holds the kernel parameters of the batch view: the
    // arrays' addresses (reallocated above) and the variant flags; the sizes
    // are read from device memory.
    if (any_clock != b->any_clock || any_stats != b->any_stats) drop_batch_graph(b);
    b->any_stats = any_stats;
    b->ntasks = task_off[n];
    b->nmerge = merge_off[n];
    b->any_clock = any_clock;
    b->nrep = n;
    const BatchSizes sizes{n, task_off[n], merge_off[n]};
    SW_CUDA(cudaMemcpyAsync(b->d_sizes, &sizes, sizeof sizes, cudaMemcpyHostToDevice, b->stream));
    if (n) {
        SW_CUDA(cudaMemcpyAsync(b->d_lat, lat.data(), sizeof(Lattice) * n, cudaMemcpyHostToDevice, b->stream));
        SW_CUDA(cudaMemcpyAsync(b->d_task_off, task_off.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice,
                                b->stream));
        SW_CUDA(cudaMemcpyAsync(b->d_merge_off, merge_off.data(), sizeof(long long) * (n + 1),
                                cudaMemcpyHostToDevice, b->stream));
        SW_CUDA(cudaStreamSynchronize(b->stream));
    }
    b->dirty = false;
    return SW_OK;
}

static int batch_timed_sweeps(sw_batch *b, const LaunchShape &shape, int n, double *ms)
{
    return timed_sweeps(
        b->view(), b->measure, b->labels, b->sm_count, shape, b->stream, n, ms,
        [&]() -> int {
            for (sw_handle *h : b->reps)
                if (b->measure && h->t_host - h->t_drained >= (uint64_t)swgb::kRingSlots - 1) {
                    int rc = drain(h);
                    if (rc != SW_OK) return rc;
                }
            return SW_OK;
        },
        [&]() {
            for (sw_handle *h : b->reps) {
                if (h->t_host < h->stop) h->t_host++;   // skipped at its limit
                if (!b->measure) h->t_drained = h->t_host;
            }
        });
}

sw_batch *sw_batch_create(void *stream)
{
    sw_batch *b = new (std::nothrow) sw_batch();
    if (!b) {
        fail(SW_ERR_OOM, "host allocation failed");
        return nullptr;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if (stream) {
            b->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sizes, sizeof(BatchSizes));
    if (e == cudaSuccess) e = cudaMemset(b->d_sizes, 0, sizeof(BatchSizes));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ticket, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(b->d_ticket, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        cuda_fail(e, "sw_batch_create");
        if (b->d_ticket) cudaFree(b->d_ticket);
        if (b->d_sizes) cudaFree(b->d_sizes);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return nullptr;
    }
    return b;
}

int sw_batch_destroy(sw_batch *b)
{
    if (!b) return SW_OK;
    while (!b->reps.empty()) sw_batch_detach(b, b->reps.back());
    cudaStreamSynchronize(b->stream);
    drop_batch_graph(b);
    free_batch_arrays(b);
    if (b->d_ticket) cudaFree(b->d_ticket);
    if (b->d_sizes) cudaFree(b->d_sizes);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return SW_OK;
}

int sw_batch_attach(sw_batch *b, sw_handle *h)
{
    if (!b || !h) return fail(SW_ERR_ARG, "null argument");
    if (h->owner) return fail(SW_ERR_STATE, "lattice is already attached to a batch");
    if (h->labeling != SW_LABEL_TILED) return fail(SW_ERR_STATE, "a comparator labeling cannot join a batch");
    int rc = drain(h);
    if (rc != SW_OK) return rc;
    if (h->measure != b->measure) {
        drop_graph(h);
        h->measure = b->measure;
    }
    if (b->labels) {
        rc = ensure_labels(h);
        if (rc != SW_OK) return rc;
    }
    if (h->own_stream) cudaStreamDestroy(h->stream);
    h->own_stream = false;
    h->stream = b->stream;
    drop_graph(h);
    h->owner = b;
    b->reps.push_back(h);
    b->dirty = true;   // descriptors rewritten before the next sweep; a captured sweep stays valid
    return SW_OK;
}

int sw_batch_detach(sw_batch *b, sw_handle *h)
{
    if (!b || !h) return fail(SW_ERR_ARG, "null argument");
    auto it = std::find(b->reps.begin(), b->reps.end(), h);
    if (it == b->reps.end()) return fail(SW_ERR_STATE, "lattice is not attached to this batch");
    int rc = drain(h);
    b->reps.erase(it);
    h->owner = nullptr;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess) {
        h->stream = s;
        h->own_stream = true;
    }
    drop_graph(h);
    b->dirty = true;   // descriptors rewritten before the next sweep; a captured sweep stays valid
    return rc;
}

int sw_batch_size(sw_batch *b)
{
    if (!b) return fail(SW_ERR_ARG, "null batch");
    return (int)b->reps.size();
}

int sw_batch_sweep(sw_batch *b, int n)
{
    if (!b) return fail(SW_ERR_ARG, "null batch");
    if (n < 0) return fail(SW_ERR_ARG, "n=%d < 0", n);
    if (b->reps.empty() || n == 0) return SW_OK;
    if (b->dirty) {
        int rc = rebuild_batch(b);
        if (rc != SW_OK) return rc;
    }
    for (int s = 0; s < n; ++s) {
        bool any = false;   // a lattice below its sweep limit
        for (sw_handle *h : b->reps) {
            if (h->sticky != SW_OK) return fail(h->sticky, "%s", h->sticky_msg.c_str());
            if (b->measure && h->t_host - h->t_drained >= (uint64_t)swgb::kRingSlots - 1) {
                int rc = drain(h);
                if (rc != SW_OK) return rc;
            }
            any = any || h->t_host < h->stop;
        }
        if (!any) break;
        int rc = enqueue_sweep(b->view(), b->measure, b->labels, b->sm_count, b->shape, b->stream, b->use_graph,
                               &b->graph, &b->graph_exec);
        if (rc != SW_OK) return rc;
        for (sw_handle *h : b->reps) {
            if (h->t_host < h->stop) h->t_host++;   // the kernels skip a lattice at its limit
            if (!b->measure) h->t_drained = h->t_host;
        }
    }
    return SW_OK;
}

int sw_batch_synchronize(sw_batch *b)
{
    if (!b) return fail(SW_ERR_ARG, "null batch");
    SW_CUDA(cudaStreamSynchronize(b->stream));
    for (sw_handle *h : b->reps) {
        int rc = check_device_error(h);
        if (rc != SW_OK) return rc;
    }
    return SW_OK;
}

int sw_batch_set_measure(sw_batch *b, int on)
{
    if (!b) return fail(SW_ERR_ARG, "null batch");
    for (sw_handle *h : b->reps) {
        int rc = drain(h);
        if (rc != SW_OK) return rc;
        h->measure = on != 0;
        drop_graph(h);
    }
    if (b->measure != (on != 0)) drop_batch_graph(b);
    b->measure = on != 0;
    return SW_OK;
}

int sw_batch_set_graph(sw_batch *b, int on)
{
    if (!b) return fail(SW_ERR_ARG, "null batch");
    if (b->use_graph != (on != 0)) drop_batch_graph(b);
    b->use_graph = on != 0;
    return SW_OK;
}

int sw_batch_set_debug_labels(sw_batch *b, int on)
{
    if (!b) return fail(SW_ERR_ARG, "null batch");
    if (on)
        for (sw_handle *h : b->reps) {
            int rc = ensure_labels(h);
            if (rc != SW_OK) return rc;
        }
    if (b->labels != (on != 0)) drop_batch_graph(b);
    b->labels = on != 0;
    return SW_OK;
}

int sw_batch_profile_sweeps(sw_batch *b, int n, float *ms, int max_stages)
{
    if (!b || !ms) return fail(SW_ERR_ARG, "null argument");
    if (n < 1 || max_stages < 1) return fail(SW_ERR_ARG, "n and max_stages must be positive");
    if (b->reps.empty()) return fail(SW_ERR_STATE, "empty batch");
    if (b->dirty) {
        int rc = rebuild_batch(b);
        if (rc != SW_OK) return rc;
    }
    double acc[swgb::kMaxStages];
    int rc = batch_timed_sweeps(b, b->shape, n, acc);
    if (rc != SW_OK) return rc;
    const int m = std::min(swgb::kMaxStages, max_stages);
    for (int k = 0; k < m; ++k) ms[k] = (float)acc[k];
    return m;
}

int sw_batch_autotune(sw_batch *b, int n, int *shape_out)
{
    if (!b) return fail(SW_ERR_ARG, "null batch");
    if (n < 1) return fail(SW_ERR_ARG, "n must be positive");
    if (b->reps.empty()) return fail(SW_ERR_STATE, "empty batch");
    if (b->dirty) {
        int rc = rebuild_batch(b);
        if (rc != SW_OK) return rc;
    }
    const std::string key = tune_key((int)b->reps.size(), b->ntasks, b->nmerge, b->measure, b->any_clock);
    LaunchShape best;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        int rc = autotune_shape(&best, n, b->any_clock, [&](const LaunchShape &trial, int nn, double *ms) {
            return batch_timed_sweeps(b, trial, nn, ms);
        });
        if (rc != SW_OK) return rc;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    b->shape = best;
    drop_batch_graph(b);
    if (shape_out) {
        shape_out[0] = best.label;
        shape_out[1] = best.merge;
        shape_out[2] = best.flip;
        shape_out[3] = best.bonds;
    }
    return sw_batch_synchronize(b);
}

int sw_batch_set_launch_shape(sw_batch *b, const int *shape)
{
    if (!b || !shape) return fail(SW_ERR_ARG, "null argument");
    for (int k = 0; k < 4; ++k)
        if (shape[k] < 1 || shape[k] > 64) return fail(SW_ERR_ARG, "blocks per SM must be in [1, 64]");
    b->shape.label = shape[0];
    b->shape.merge = shape[1];
    b->shape.flip = shape[2];
    b->shape.bonds = shape[3];
    drop_batch_graph(b);
    return SW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// sw_sweep_noalloc: sweeps of a caller-owned spin array with every piece of
// working memory taken from one fixed device array of this file, so that the
// call allocates nothing.  It runs the same four kernels as sw_sweep, on a
// batch-of-one view whose buffers are carved out of that array.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the working buffers inside the shared array, sized for
// the largest accepted lattice (SW_NOALLOC_MAX_L).
struct NoallocLayout {
    size_t code, opar, edge, open_count, cross, bond, ring, thr_tab, st, lat, sizes, task_off, merge_off, ticket, total;
};
constexpr int kNoallocRingSlots = 128;   // counter rows; longer calls are drained in chunks

constexpr NoallocLayout noalloc_layout()
{
    const size_t sites = (size_t)SW_NOALLOC_MAX_L * SW_NOALLOC_MAX_L;
    const size_t tiles = (size_t)((SW_NOALLOC_MAX_L + swgb::kTileW - 1) / swgb::kTileW) *
                         ((SW_NOALLOC_MAX_L + swgb::kTileH - 1) / swgb::kTileH);
    NoallocLayout o{};
    size_t at = 0;
    o.code = at;       at = align256(at + sites * sizeof(uint16_t));
    o.opar = at;       at = align256(at + tiles * swgb::kOpenSlots * sizeof(unsigned long long));
    o.edge = at;       at = align256(at + tiles * swgb::kEdgeBytes);
    o.open_count = at; at = align256(at + tiles * sizeof(int32_t));
    o.cross = at;      at = align256(at + tiles * swgb::kCrossWords * sizeof(uint32_t));
    o.bond = at;       at = align256(at + tiles * swgb::kBondWords * sizeof(uint32_t));
    o.ring = at;       at = align256(at + (size_t)kNoallocRingSlots * SW_MAX_COUNTERS * sizeof(unsigned long long));
    o.thr_tab = at;    at = align256(at + (size_t)(2 * SW_MAX_CLOCK_Q) * (2 * SW_MAX_CLOCK_Q) * sizeof(uint32_t));
    o.st = at;         at = align256(at + sizeof(DevState));
    o.lat = at;        at = align256(at + sizeof(Lattice));
    o.sizes = at;      at = align256(at + sizeof(BatchSizes));
    o.task_off = at;   at = align256(at + 2 * sizeof(int));
    o.merge_off = at;  at = align256(at + 2 * sizeof(long long));
    o.ticket = at;     at = align256(at + sizeof(unsigned int));
    o.total = at;
    return o;
}
constexpr NoallocLayout kNoalloc = noalloc_layout();
static_assert(kNoalloc.total <= SW_NOALLOC_SCRATCH_BYTES, "SW_NOALLOC_SCRATCH_BYTES is too small for the layout");

}  // namespace

// The working memory of sw_sweep_noalloc.  Each device that loads the
// library holds one copy until the process exits.  Host code must not take
// its address directly (the name is a host-side stand-in); the per-device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SW_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_base[kNoallocMaxDevices];   // device address of the array, per device
int g_noalloc_sms[kNoallocMaxDevices];

// Once per device, with that device current: the array's device address
// and the SM count.  The first lookup may load the library's device code
// onto the device.
int noalloc_setup(int dev, unsigned char **base, int *sms)
{
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(SW_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        g_noalloc_sms[dev] = n;
        g_noalloc_base[dev] = (unsigned char *)p;
    }
    *base = g_noalloc_base[dev];
    *sms = g_noalloc_sms[dev];
    return SW_OK;
}

}  // namespace

extern "C" int sw_sweep_noalloc(int L, int q, int model, double T, uint64_t seed, uint64_t sweep0, int n,
                                int8_t *d_spins, int64_t *d_counts, void *stream)
{
    if (validate(L, q, model, T) != SW_OK) return SW_ERR_ARG;
    if (L > SW_NOALLOC_MAX_L)
        return fail(SW_ERR_ARG, "L=%d exceeds the no-allocation limit L <= %d (%d bytes of scratch per device)", L,
                    SW_NOALLOC_MAX_L, SW_NOALLOC_SCRATCH_BYTES);
    if (n < 0) return fail(SW_ERR_ARG, "n=%d < 0", n);
    if (!d_spins || ((uintptr_t)d_spins & 15)) return fail(SW_ERR_ARG, "spins must be a 16-byte aligned device buffer");
    if (d_counts && ((uintptr_t)d_counts & 7)) return fail(SW_ERR_ARG, "counts must be 8-byte aligned");
    if (n == 0) return SW_OK;

    int dev = 0, sms = 0;
    unsigned char *base = nullptr;
    SW_CUDA(cudaGetDevice(&dev));
    int rc = noalloc_setup(dev, &base, &sms);
    if (rc != SW_OK) return rc;
    const cudaStream_t s = (cudaStream_t)stream;
    const bool measure = d_counts != nullptr;
    const int nclass = nclass_of(q, model), nc = ncounters_of(q, model);
    const int tiles_x = (L + swgb::kTileW - 1) / swgb::kTileW, tiles_y = (L + swgb::kTileH - 1) / swgb::kTileH;

    Lattice lat{};
    lat.L = L;
    lat.q = q;
    lat.clock = model == SW_CLOCK;
    lat.key0 = (uint32_t)(seed & 0xffffffffu);
    lat.key1 = (uint32_t)(seed >> 32);
    lat.spin = d_spins;
    lat.label = nullptr;   // no debug labels here
    lat.code = (uint16_t *)(base + kNoalloc.code);
    lat.opar = (unsigned long long *)(base + kNoalloc.opar);
    lat.edge = base + kNoalloc.edge;
    lat.open_count = (int32_t *)(base + kNoalloc.open_count);
    lat.cross = (uint32_t *)(base + kNoalloc.cross);
    lat.bond = (uint32_t *)(base + kNoalloc.bond);
    lat.tiles_x = tiles_x;
    lat.tiles_y = tiles_y;
    lat.st = (DevState *)(base + kNoalloc.st);
    lat.ring = (unsigned long long *)(base + kNoalloc.ring);
    lat.ring_slots = kNoallocRingSlots;
    lat.ncounters = nc;
    lat.nclass = nclass;
    // Bond thresholds (Sec. 2 step (ii); clock: Sec. 4 embedding), J = 1,
    // built exactly as sw_create builds them.
    std::vector<uint32_t> tab;
    if (model == SW_POTTS) {
        lat.thr = threshold_of(1.0 / T);
    } else if (model == SW_ISING) {
        lat.thr = threshold_of(2.0 / T);
    } else {
        tab = clock_thresholds(q, T);
        lat.thr_tab = (const uint32_t *)(base + kNoalloc.thr_tab);
    }
    const int task_off[2] = {0, tiles_x * tiles_y};
    const long long merge_off[2] = {0, (long long)tiles_x * tiles_y * swgb::kMergeItems};
    Batch b{};
    b.dev = (const BatchSizes *)(base + kNoalloc.sizes);
    b.lat = (const Lattice *)(base + kNoalloc.lat);
    b.task_off = (const int *)(base + kNoalloc.task_off);
    b.merge_off = (const long long *)(base + kNoalloc.merge_off);
    b.ticket = (unsigned int *)(base + kNoalloc.ticket);
    b.nrep = 1;
    b.ntasks = task_off[1];
    b.nmerge = merge_off[1];
    b.any_clock = model == SW_CLOCK;

    // The array keeps whatever the previous call left: reset everything that
    // must start from a known value (sweep index, error word, ticket,
    // counter rows).  Labels, codes and open lists are written before read.
    DevState st{};
    st.sweep = sweep0;
    st.stop = swgb::kNoStop;
    st.classes_upto = sweep0;
    st.next_t = sweep0;
    SW_CUDA(cudaMemcpyAsync(lat.st, &st, sizeof st, cudaMemcpyHostToDevice, s));
    SW_CUDA(cudaMemsetAsync(b.ticket, 0, sizeof(unsigned int), s));
    SW_CUDA(cudaMemsetAsync(lat.ring, 0, sizeof(unsigned long long) * kNoallocRingSlots * nc, s));
    SW_CUDA(cudaMemcpyAsync(base + kNoalloc.lat, &lat, sizeof lat, cudaMemcpyHostToDevice, s));
    const BatchSizes sizes{1, b.ntasks, b.nmerge};
    SW_CUDA(cudaMemcpyAsync(base + kNoalloc.sizes, &sizes, sizeof sizes, cudaMemcpyHostToDevice, s));
    SW_CUDA(cudaMemcpyAsync(base + kNoalloc.task_off, task_off, sizeof task_off, cudaMemcpyHostToDevice, s));
    SW_CUDA(cudaMemcpyAsync(base + kNoalloc.merge_off, merge_off, sizeof merge_off, cudaMemcpyHostToDevice, s));
    if (!tab.empty())
        SW_CUDA(cudaMemcpyAsync(base + kNoalloc.thr_tab, tab.data(), tab.size() * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, s));

    // Every kernel assumes states in [0, q): check them first, change nothing otherwise.
    cudaError_t e = swgb::launch_count_invalid(lat, &lat.st->scratch, sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch_count_invalid");
    unsigned int nbad = 0;
    SW_CUDA(cudaMemcpyAsync(&nbad, &lat.st->scratch, sizeof nbad, cudaMemcpyDeviceToHost, s));
    SW_CUDA(cudaStreamSynchronize(s));
    if (nbad) return fail(SW_ERR_ARG, "%u spins outside [0, %d); nothing was changed", nbad, q);

    // Once sweeps are enqueued, an error return first waits (best effort) for
    // the work already on the stream, so that no later call's work can
    // overlap it in the shared array.
    auto settle_fail = [&](int rc) {
        cudaStreamSynchronize(s);
        return rc;
    };
    // Sweeps in chunks that fit the counter rows; after each chunk the
    // newest configuration's bond classes are completed and the chunk's rows
    // copied to d_counts (row k = sweep sweep0 + k).
    const LaunchShape shape;
    for (int done = 0; done < n;) {
        const int c = std::min(n - done, kNoallocRingSlots - 1);
        for (int k = 0; k < c; ++k) {
            e = swgb::launch_sweep(b, measure, false, sms, shape, s);
            if (e != cudaSuccess) return settle_fail(cuda_fail(e, "launch_sweep"));
        }
        if (measure) {
            e = swgb::launch_pending_classes(lat, sms, s);
            if (e != cudaSuccess) return settle_fail(cuda_fail(e, "launch_pending_classes"));
            const uint64_t t0 = sweep0 + (uint64_t)done;
            const size_t first = (size_t)(t0 % kNoallocRingSlots);
            const size_t n1 = std::min((size_t)c, (size_t)kNoallocRingSlots - first);
            const size_t row = (size_t)nc * sizeof(unsigned long long);
            e = cudaMemcpyAsync(d_counts + (size_t)done * nc, lat.ring + first * nc, n1 * row,
                                cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess && n1 < (size_t)c)
                e = cudaMemcpyAsync(d_counts + ((size_t)done + n1) * nc, lat.ring, ((size_t)c - n1) * row,
                                    cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return settle_fail(cuda_fail(e, "cudaMemcpyAsync(counters)"));
        }
        done += c;
    }
    SW_CUDA(cudaMemcpyAsync(&st, lat.st, sizeof st, cudaMemcpyDeviceToHost, s));
    SW_CUDA(cudaStreamSynchronize(s));
    if (st.err != swgb::kErrNone)
        return fail(SW_ERR_NOT_CONVERGED, "device loop bound exceeded (code %d at index %d)", st.err, st.err_where);
    return SW_OK;
}
