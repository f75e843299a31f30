// sw_device.cuh -- device-side building blocks of the Swendsen-Wang sweep:
// the counter-based generator, the kernel parameter block and the bounded
// union-find primitives.  Written for sm_103a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

// Random-number tags of the counter (index, sweep lo, tag, sweep hi).
enum : uint32_t { kTagBond = 0, kTagState = 1, kTagAxis = 2, kTagInit = 3, kTagStateBit = 4 };

// Error codes stored in the device state word (first error wins).
enum : int { kErrNone = 0, kErrFindCap = 1, kErrUnionCap = 2, kErrTimeBudget = 3, kErrInternal = 4 };

// Wall-clock budget of any single data-dependent device loop (~1 s at the
// GB300's 2.07 GHz maximum SM clock).  A loop that exceeds it records an
// error and returns instead of spinning on.
constexpr long long kLoopBudgetCycles = 2000000000ll;

constexpr unsigned long long kNoStop = ~0ull;

// Sticky per-lattice device state.
struct DevState {
    unsigned long long sweep;          // sweeps completed; read by every kernel of a sweep
    unsigned long long stop;           // the lattice sweeps only while sweep < stop (kNoStop: always)
    unsigned long long classes_upto;   // configurations < this index have their bond classes counted
    unsigned int ticket;               // blocks finished in the sweep's last kernel
    int err;                           // first device error (kErr*)
    int err_where;                     // site or index that hit it
    unsigned int scratch;              // host-side checks (count of invalid spins)
    unsigned int pad;
    unsigned long long next_t;         // sweep index the next labeling kernel will run at (the merge
                                       // kernel writes it; a hint for early bond draws, checked)
};

// Everything a kernel needs about one lattice.  Passed by value.
struct Lattice {
    int L;                      // linear size (L % 4 == 0)
    int q;                      // number of states
    int clock;                  // 1: clock model, 0: Potts / Ising
    uint32_t thr;               // Potts / Ising bond threshold
    const uint32_t *thr_tab;    // clock: (2q) x (2q) thresholds by class
    uint32_t key0, key1;        // Philox key = seed
    int8_t *spin;               // L*L states
    int32_t *label;             // L*L canonical labels (debug labels and the comparator labelings only)
    uint16_t *code;             // L*L per-site codes written by the labeling stage
    unsigned long long *opar;   // tiles x kOpenSlots: union-find over the open components of all tiles
                                // (component id = tile * kOpenSlots + slot), entry = key << 32 | parent id
    uint8_t *edge;              // tiles x kEdgeBytes: open slot of the right-edge sites, then the left-edge sites
    int32_t *open_count;        // tiles
    uint32_t *cross;            // tiles x kCrossWords: active crossing bonds (right edge rows, bottom edge columns)
    uint32_t *bond;             // tiles x 256 words: a tile's right-bond masks (64 rows x 2 words), then
                                // its down-bond masks; bit c of word (row, h) = bond of column 32 h + c
    int tiles_x, tiles_y;
    DevState *st;
    unsigned long long *ring;   // ring_slots x ncounters counters
    int ring_slots;
    int ncounters;
    int nclass;
    // Test aids (0: defaults): every data-dependent device loop gives up
    // after dbg_loop_cap steps (recording kErrFindCap / kErrUnionCap), and a
    // tile's union-pair list holds at most dbg_list_cap pairs.
    int dbg_loop_cap;
    int dbg_list_cap;
    // Labeling statistics (nullptr: not gathered): kStat* accumulators.
    unsigned long long *stats;
};

// Accumulators of the labeling statistics, summed over the sweeps that ran
// with them on.
enum : int {
    kStatLabels = 0,      // provisional labels opened by the tile scans
    kStatPairs = 1,       // union pairs of the tiles (further run contacts and quadrant seams)
    kStatComponents = 2,  // tile components (closed clusters and open components)
    kStatOpen = 3,        // open components (reaching a tile border)
    kStatUnions = 4,      // global unions across tile edges (distinct component pairs of a warp)
    kStatLinks = 5,       // global link attempts (atomicMin of a root entry)
    kStatRetries = 6,     // link attempts that found the root linked meanwhile
    kStatFinds = 7,       // global walks (merge and root walks)
    kStatHops = 8,        // parent steps of those walks
    kStatMaxHops = 9,     // longest walk (steps)
    kStatSweeps = 10,     // sweeps counted
    kStatFields = 11
};

// A set of lattices swept together; a single lattice is a batch of one.
// One block task is one tile of one lattice, processed by kTaskWarps warps.
constexpr int kTaskWarps = 4;
// Sizes of a batch, in device memory: the kernels read them there, so a
// captured sweep stays valid when lattices join or leave.
struct BatchSizes {
    int nrep;
    int ntasks;
    long long nmerge;
};

struct Batch {
    const BatchSizes *dev;         // the sizes below, as the kernels read them (device memory)
    const Lattice *lat;            // [nrep] descriptors (device memory)
    const int *task_off;           // [nrep + 1] prefix sums of the lattices' tile counts
    const long long *merge_off;    // [nrep + 1] prefix sums of the lattices' merge items (kMergeItems a tile)
    unsigned int *ticket;          // blocks finished in the sweep's last kernel
    int nrep;
    int ntasks;
    long long nmerge;
    int any_clock;                 // a clock lattice is present (selects the kernel variant that measures it)
    int any_stats;                 // a lattice gathers labeling statistics (selects the variants that tally)
    int full_grid;                 // size every grid for the whole GPU, not for ntasks / nmerge (batches)
};

// Philox-4x32-10 (Salmon et al., SC'11).  Each round takes two 32x32->64
// products; their high halves are mixed with the other two words and the
// round key, and the key advances by the two Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 draw4(const Lattice &lat, uint32_t index, unsigned long long t, uint32_t tag)
{
    return philox4x32_10(make_uint4(index, (uint32_t)t, tag, (uint32_t)(t >> 32)), lat.key0, lat.key1);
}

__device__ __forceinline__ int mulhi_q(uint32_t u, int q)
{
    return (int)__umulhi(u, (uint32_t)q);
}

// Bit r & 31 of lane (r >> 5) & 3 of the STATE_BIT draw with index r >> 7:
// one uniform bit per index, 128 indices to a Philox call.
__device__ __forceinline__ int draw_bit(const Lattice &lat, uint32_t r, unsigned long long t)
{
    const uint4 u = draw4(lat, r >> 7, t, kTagStateBit);
    const uint32_t l = (r >> 5) & 3u;
    const uint32_t w = l == 0 ? u.x : l == 1 ? u.y : l == 2 ? u.z : u.w;
    return (int)((w >> (r & 31u)) & 1u);
}

// Does the cluster draw take one bit?  Two outcomes: the new state of the
// q = 2 Potts (Ising) model, the reflection flag of the clock model.
__device__ __forceinline__ bool bit_draw(const Lattice &lat)
{
    return lat.clock != 0 || lat.q == 2;
}

// The draw of the cluster rooted at site r (Sec. 2 (v)-(vii), Sec. 4): its
// new state (Potts), uniform in [0, q), or its reflection flag (clock).
__device__ __forceinline__ int cluster_draw(const Lattice &lat, uint32_t r, unsigned long long t)
{
    if (bit_draw(lat)) return draw_bit(lat, r, t);
    return mulhi_q(draw4(lat, r, t, kTagState).x, lat.q);
}

// Mirror axis of the sweep (clock model).
__device__ __forceinline__ int clock_axis(const Lattice &lat, unsigned long long t)
{
    return mulhi_q(draw4(lat, 0u, t, kTagAxis).x, lat.q);
}

// Projection class j = (2k - m) mod 2q.
__device__ __forceinline__ int clock_class(int k, int m, int q)
{
    int j = 2 * k - m;
    return j < 0 ? j + 2 * q : j;
}

__device__ __forceinline__ void record_error(DevState *st, int code, int where)
{
    if (atomicCAS(&st->err, kErrNone, code) == kErrNone) st->err_where = where;
}

// ---------------------------------------------------------------------------
// Global union-find over the open components of every tile (Sec. 2: the
// "proper label" of a cluster is its smallest site).  Node x = tile *
// kOpenSlots + slot; its entry holds its parent's key (the smallest site of
// the parent's tile component) in the high word and the parent's id in the
// low word, so entries order by key.  A root is its own parent.  Roots are
// linked larger key under smaller with a 64-bit atomicMin, so the root of a
// tree is its component with the smallest site; path halving writes only
// ancestors.  Entries are read through the L1 (a load the compiler keeps):
// a stale entry names an older ancestor, which is still an ancestor since
// links only join roots; a root the walk takes for one is checked by the
// link's atomicMin, which hands back the current parent to retry with; and
// while the flip stage walks, no entry of a root changes -- so the many
// walks that end at one large cluster's root mostly hit the L1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_entry(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.global.ca.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Tallies of the global union-find (labeling statistics).
struct OpenTally {
    unsigned int finds = 0, hops = 0, max_hops = 0, links = 0, retries = 0;
};

// Root entry of node x (key << 32 | root id).  Parent steps go to the tally.
__device__ __forceinline__ unsigned long long find_open(unsigned long long *par, uint32_t x, int cap, DevState *st,
                                                        OpenTally &tl)
{
    const long long t0 = clock64();
    ++tl.finds;
    unsigned int steps = 0;
    for (int it = 0; it < cap; ++it) {
        const unsigned long long e = ld_entry(par + x);
        const uint32_t p = (uint32_t)e;
        if (p == x) {
            tl.hops += steps;
            tl.max_hops = max(tl.max_hops, steps);
            return e;
        }
        const unsigned long long ep = ld_entry(par + p);
        const uint32_t gp = (uint32_t)ep;
        ++steps;
        if (gp == p) {
            tl.hops += steps;
            tl.max_hops = max(tl.max_hops, steps);
            return ep;
        }
        ++steps;
        par[x] = ep;   // grandparent: an ancestor of x, safe under concurrent linking
        x = gp;
        if ((it & 255) == 255 && clock64() - t0 > kLoopBudgetCycles) {
            record_error(st, kErrTimeBudget, (int)x);
            return ld_entry(par + x);
        }
    }
    record_error(st, kErrFindCap, (int)x);
    return ld_entry(par + x);
}

__device__ __forceinline__ void union_open(unsigned long long *par, uint32_t a, uint32_t b, int cap, DevState *st,
                                           OpenTally &tl)
{
    const long long t0 = clock64();
    // Both entries in flight at once: most ends are roots already.
    unsigned long long ea = ld_entry(par + a), eb = ld_entry(par + b);
    if ((uint32_t)ea != a) ea = find_open(par, a, cap, st, tl);
    if ((uint32_t)eb != b) eb = find_open(par, b, cap, st, tl);
    for (int it = 0; it < cap; ++it) {
        if (ea == eb) return;
        const unsigned long long hi = ea > eb ? ea : eb;
        const unsigned long long lo = ea > eb ? eb : ea;
        const unsigned long long old = atomicMin(par + (uint32_t)hi, lo);
        ++tl.links;
        if (old == hi) return;   // hi was a root: now under lo
        ++tl.retries;
        // hi had been linked under old meanwhile: join old's tree and lo's.
        ea = find_open(par, (uint32_t)old, cap, st, tl);
        eb = find_open(par, (uint32_t)lo, cap, st, tl);
        if (clock64() - t0 > kLoopBudgetCycles) {
            record_error(st, kErrTimeBudget, (int)(uint32_t)hi);
            return;
        }
    }
    record_error(st, kErrUnionCap, (int)a);
}

// A state outside [0, q) (only possible through a caller writing the spin
// buffer directly) is read as state 0 wherever it would index a table.
__device__ __forceinline__ int valid_state(int s, int q)
{
    return (unsigned)s < (unsigned)q ? s : 0;
}

// Shared-memory union-find of a tile over its nodes v = row * 64 + column,
// one 16-bit word per node (same invariants: a word is never above its
// node, larger root linked under smaller, so a root is its component's
// smallest node).  A link is one 16-bit compare-and-swap that succeeds only
// while the larger root is still a root.  After the roots are settled, a
// root's word is kTileResolved | its cluster's code.
constexpr int kTileResolved = 0x1000;

// Root of x with path halving (writes only ancestors).  Valid while no word
// is resolved.  Returns -1 if the cap is exceeded.
__device__ __forceinline__ int find_t(volatile uint16_t *par, int x, int cap)
{
    for (int it = 0; it < cap; ++it) {
        const int p = par[x];
        if (p == x) return x;
        const int gp = par[p];
        if (gp == p) return p;
        par[x] = (uint16_t)gp;
        x = gp;
    }
    return -1;
}

// Root of x without writing.
__device__ __forceinline__ int find_t_ro(const volatile uint16_t *par, int x, int cap)
{
    for (int it = 0; it < cap; ++it) {
        const int p = par[x];
        if (p == x) return x;
        x = p;
    }
    return -1;
}

__device__ __forceinline__ bool union_t(volatile uint16_t *par, int a, int b, int cap)
{
    for (int it = 0; it < cap; ++it) {
        // Both parents in flight at once: the ends are often roots.
        const int pa = par[a], pb = par[b];
        if (pa != a) a = find_t(par, pa, cap);
        if (pb != b) b = find_t(par, pb, cap);
        if (a < 0 || b < 0) return false;
        if (a == b) return true;
        const int hi = a > b ? a : b;
        const int lo = a > b ? b : a;
        const int old = atomicCAS(const_cast<unsigned short *>(reinterpret_cast<volatile unsigned short *>(par)) + hi,
                                  (unsigned short)hi, (unsigned short)lo);
        if (old == hi) return true;
        a = old;   // hi was linked meanwhile: join its new parent and lo
        b = lo;
    }
    return false;
}

// Block-wide sum of a per-thread value into one global 64-bit counter.
template <int NT>
__device__ __forceinline__ void block_add(unsigned long long *dst, unsigned int v, unsigned int *scratch)
{
    v = __reduce_add_sync(0xffffffffu, v);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;   // blocks may be 2-D
    const int lane = tid & 31;
    const int warp = tid >> 5;
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned int s = (lane < NT / 32) ? scratch[lane] : 0u;
        s = __reduce_add_sync(0xffffffffu, s);
        if (lane == 0 && s) atomicAdd(dst, (unsigned long long)s);
    }
    __syncthreads();
}

// Block-wide flush of the global union-find tallies into a lattice's
// statistics (all threads of the block; no-op without statistics).  unions:
// the thread's unions attempted.
template <int NT>
__device__ __forceinline__ void flush_open_tally(unsigned long long *stats, const OpenTally &tl, unsigned int unions,
                                                 unsigned int *scratch)
{
    if (stats == nullptr) return;   // uniform: one lattice per block call
    block_add<NT>(stats + kStatUnions, unions, scratch);
    block_add<NT>(stats + kStatLinks, tl.links, scratch);
    block_add<NT>(stats + kStatRetries, tl.retries, scratch);
    block_add<NT>(stats + kStatFinds, tl.finds, scratch);
    block_add<NT>(stats + kStatHops, tl.hops, scratch);
    const unsigned int m = __reduce_max_sync(0xffffffffu, tl.max_hops);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(stats + kStatMaxHops, (unsigned long long)m);
}

}  // namespace swgb
