// sw_kernels.cu -- the kernels of one Swendsen-Wang sweep on sm_103a.
//
// One sweep (Komura & Okabe, arXiv:1202.0635, Sec. 2 steps (i)-(viii);
// clock model: Sec. 4 embedded clusters) is three launches over the 64 x 64
// tiles of every lattice of a batch (a single lattice is a batch of one),
// four when the batch holds a clock lattice.  A block owns one tile of one
// lattice at a time ("task"), so per-lattice counters reduce per block.
//
//   k_bonds        (batches with a clock lattice) bonds of every site
//                  (Sec. 2 (ii); Sec. 4): Philox draws against the integer
//                  threshold of the state pair; the masks go to a per-tile
//                  buffer.  With measurement on it also counts the bond
//                  classes of the incoming configuration (the previous
//                  sweep's result) and the active bonds.
//   k_label_tiles  (Potts batches: first the bonds of the tile, as k_bonds
//                  draws them, from packed byte compares of the states)
//                  tile-local clusters by a row-by-row labeling with a
//                  union-find in shared memory (four warps, one 32 x 32
//                  quadrant each).  A component that does not reach the tile
//                  border (or reaches it only through inactive crossing bonds
//                  on the right/bottom edges) is a finished cluster: its root
//                  (smallest site) draws the new state here (Sec. 2 (v)-(vii) /
//                  Sec. 4 reflection) and its sites get a "closed" code.  Open
//                  components enter the global union-find keyed by their
//                  root's site index.
//   k_merge        joins the open roots across every active bond that
//                  crosses a tile edge or the periodic wrap (atomicMin,
//                  larger root under smaller); first it announces the sweep
//                  index of the next labeling launch, which draws its first
//                  bonds before it waits for the flip.
//   k_flip_tiles   finds the cluster root of every open component (the
//                  smallest site index of the cluster, Sec. 2 "proper
//                  label"), which draws the cluster's new state; writes all
//                  spins, counts states and the clusters rooted in the tile;
//                  its last block advances the sweep index of every lattice
//                  of the batch.
#include <type_traits>

#include "sw_internal.h"

namespace swgb {

namespace {

constexpr int TW = kTileW, TH = kTileH, NS = kTileSites, QW = kQuad;
constexpr int kBlockThreads = kTaskWarps * 32;
constexpr int kEnergyThreads = 256;
constexpr unsigned FULL = 0xffffffffu;
// Resident blocks per SM of the flip kernel's variants (its launch bounds);
// its grid never asks for more, so that one wave covers the tiles.
constexpr int kFlipResidentPotts = 10, kFlipResidentClock = 8;
// Resident blocks per SM of the labeling kernel that draws the bonds itself,
// and the bond draws its threads keep in flight.
constexpr int kLabelResidentFused = 11, kFusedDrawUnroll = 16;
// Resolved root word: kTileResolved | the cluster's per-site code, i.e.
// kCodeClosed | new state (Potts) or reflection flag (clock), or the open
// slot.
constexpr int kCodeMask = 0x1FF;
static_assert(SW_MAX_Q <= 0x80 && kOpenSlots <= 0x100 && kCodeClosed == 0x100 && kTileResolved > kCodeMask,
              "resolved words hold a code");

static_assert(QW == 32, "a warp quadrant is 32 x 32: lane r owns row r as a 32-bit mask");
static_assert(TW == 2 * QW && TH == 2 * QW, "a tile is 2 x 2 quadrants");
static_assert(sizeof(Lattice) % 8 == 0, "lattice descriptors are copied in 8-byte words");
static_assert(TW == 64 && kBlockThreads == NS / 32, "lane = column pair; thread t owns labels 32 t .. 32 t + 31");

__device__ __forceinline__ unsigned long long read_u64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ unsigned long long *ring_row(const Lattice &lat, unsigned long long t)
{
    return lat.ring + (size_t)(t % (unsigned long long)lat.ring_slots) * lat.ncounters;
}

__device__ __forceinline__ int tid2d() { return threadIdx.y * blockDim.x + threadIdx.x; }

// Largest r with off[r] <= k, for off[0] = 0 <= k < off[n].
template <typename T>
__device__ __forceinline__ int find_rep(const T *off, int n, T k)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= k) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Copy a lattice descriptor into shared memory (whole block).
__device__ __forceinline__ void load_lattice(Lattice *dst, const Lattice *src)
{
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(Lattice) / 8); i += blockDim.x) d[i] = __ldg(s + i);
}

// Global site index of tile-local node loc (row * 64 + column) in tile (bx, by).
__device__ __forceinline__ int tile_site(int L, int bx, int by, int loc)
{
    return (by * TH + loc / TW) * L + bx * TW + (loc % TW);
}

// Bit k of the result is set iff byte k of x is zero.
__device__ __forceinline__ unsigned zero_bytes4(unsigned x)
{
    const unsigned t = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);   // 0x80 in zero bytes
    return (((t >> 7) * 0x00204081u) >> 21) & 0xFu;
}

__device__ __forceinline__ int byte_at(const uint32_t (&w)[8], int c)
{
    return (int)((w[c >> 2] >> (8 * (c & 3))) & 0xFFu);
}

__device__ __forceinline__ int reflect(int k, int m, int q)
{
    const int v = m - k;
    return v < 0 ? v + q : v;
}

// Clock bond class d = min(dk, q - dk) of states a, b.
__device__ __forceinline__ int clock_bond_class(int a, int b, int q)
{
    int dk = valid_state(a, q) - valid_state(b, q);
    if (dk < 0) dk += q;
    return dk < q - dk ? dk : q - dk;
}

// Shared histogram for any number of bins (warp-aggregated atomics).
// Must be called by all 32 lanes of the warp; invalid lanes add nothing.
__device__ __forceinline__ void add_hist_any(unsigned int *hist, int v, bool valid)
{
    const unsigned int active = __ballot_sync(FULL, valid);
    if (valid) {
        const unsigned int peers = __match_any_sync(active, v);
        if ((tid2d() & 31) == __ffs(peers) - 1) atomicAdd(&hist[v], (unsigned)__popc(peers));
    }
}

// The kernels of a sweep are launched with programmatic stream
// serialization.  pdl_wait: until the previous kernel has completed and its
// writes are visible.  pdl_release: the next kernel of the stream may
// launch, so that its blocks take the SMs this kernel's last blocks leave
// and wait there instead of being launched after the grid drains; a block
// of the next kernel runs only once every block of this one has released
// or exited, i.e. has passed its own wait, so whatever the kernel before
// this one wrote is visible to it before it waits.  (Launched without the
// attribute, both do nothing.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Nothing before this point touches memory.
__device__ __forceinline__ void pdl_begin()
{
    pdl_wait();
    pdl_release();
}

// Per-lattice values every block needs once per task.
struct TaskCtx {
    unsigned long long t;   // sweep index
    int count_classes;      // bond classes of configuration t - 1 are counted now
    int m;                  // clock mirror axis
    int active;             // the lattice sweeps this time (sweep index below its limit)
};

template <bool MEASURE>
__device__ __forceinline__ TaskCtx task_context(const Lattice &lat)
{
    TaskCtx c;
    c.t = read_u64(&lat.st->sweep);
    c.active = c.t < read_u64(&lat.st->stop);
    c.count_classes = c.active && MEASURE && c.t >= 1ull && c.t - 1ull >= read_u64(&lat.st->classes_upto);
    c.m = lat.clock ? clock_axis(lat, c.t) : 0;
    return c;
}

// ---------------------------------------------------------------------------
// k_init: all-up or random start (tag INIT, index = site, sweep field 0).
// ---------------------------------------------------------------------------
__global__ void k_init(Lattice lat, int random)
{
    const long long N4 = (long long)lat.L * lat.L / 4;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N4;
         g += (long long)gridDim.x * blockDim.x) {
        const uint32_t i0 = (uint32_t)(4 * g);
        char4 s = make_char4(0, 0, 0, 0);
        if (random) {
            s.x = (int8_t)mulhi_q(draw4(lat, i0 + 0, 0ull, kTagInit).x, lat.q);
            s.y = (int8_t)mulhi_q(draw4(lat, i0 + 1, 0ull, kTagInit).x, lat.q);
            s.z = (int8_t)mulhi_q(draw4(lat, i0 + 2, 0ull, kTagInit).x, lat.q);
            s.w = (int8_t)mulhi_q(draw4(lat, i0 + 3, 0ull, kTagInit).x, lat.q);
        }
        reinterpret_cast<char4 *>(lat.spin)[g] = s;
    }
}

// The states at distance r to the right (px) and below (py) of the half
// row (y, x0 .. x0 + ncols - 1), four to a word like the row itself.
__device__ __forceinline__ void load_partners(const int8_t *spin, int L, int y, int x0, int r, int ncols, bool rv,
                                              uint32_t (&px)[8], uint32_t (&py)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) px[k] = py[k] = 0u;
    if (!rv) return;
    const int yr = y + r < L ? y + r : y + r - L;   // 0 < r < L
    const uint32_t *prow = reinterpret_cast<const uint32_t *>(spin + (size_t)yr * L + x0);
    const bool whole = (L & 15) == 0 && ncols == 32;   // 16-byte aligned half rows
    if (whole) {
        const uint4 a0 = __ldg(reinterpret_cast<const uint4 *>(prow)), a1 = __ldg(reinterpret_cast<const uint4 *>(prow) + 1);
        py[0] = a0.x; py[1] = a0.y; py[2] = a0.z; py[3] = a0.w;
        py[4] = a1.x; py[5] = a1.y; py[6] = a1.z; py[7] = a1.w;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) py[k] = (4 * k < ncols) ? __ldg(prow + k) : 0u;
    }
    const int cx = x0 + r < L ? x0 + r : x0 + r - L;
    const uint32_t *xrow = reinterpret_cast<const uint32_t *>(spin + (size_t)y * L + cx);
    if (whole && (cx & 15) == 0 && cx + ncols <= L) {
        const uint4 a0 = __ldg(reinterpret_cast<const uint4 *>(xrow)), a1 = __ldg(reinterpret_cast<const uint4 *>(xrow) + 1);
        px[0] = a0.x; px[1] = a0.y; px[2] = a0.z; px[3] = a0.w;
        px[4] = a1.x; px[5] = a1.y; px[6] = a1.z; px[7] = a1.w;
    } else if ((cx & 3) == 0 && cx + ncols <= L) {   // word aligned, no wrap
#pragma unroll
        for (int k = 0; k < 8; ++k) px[k] = (4 * k < ncols) ? __ldg(xrow + k) : 0u;
    } else {   // unrolled: px stays in registers
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j >= ncols) break;
            const int xj = cx + j < L ? cx + j : cx + j - L;
            const uint32_t b = (uint8_t)__ldg(spin + (size_t)y * L + xj);
            px[j >> 2] |= b << (8 * (j & 3));
        }
    }
}

// Bytes of x outside [0, q) set to state 0 (q <= 15): a byte is out of
// range if its top bit is set or its low seven bits reach q.
__device__ __forceinline__ uint32_t clock_valid4(uint32_t x, uint32_t q4)
{
    const uint32_t big = (((x & 0x7F7F7F7Fu) + (0x80808080u - q4)) | x) & 0x80808080u;
    return x & ~((big >> 7) * 0xFFu);
}

// Clock classes min(dk, q - dk), dk = (a - b) mod q, of four state pairs at
// once: the bytes of a and b, states in [0, q), q <= 15 (every class is
// below 8).  Each byte lane works on 128 + value so that no lane borrows
// from its neighbour.
__device__ __forceinline__ uint32_t clock_classes4(uint32_t a, uint32_t b, uint32_t q4)
{
    uint32_t d = (a | 0x80808080u) - b;                              // 128 + a - b
    d += ((~d >> 7) & 0x01010101u) * (q4 & 0xFFu);                    // + q where a < b
    const uint32_t e = d & 0x7F7F7F7Fu;                              // dk
    const uint32_t f = q4 - e;                                       // q - dk, in [1, q]
    const uint32_t ge = ((((e | 0x80808080u) - f) & 0x80808080u) >> 7) * 0xFFu;   // dk >= q - dk
    return e ^ ((e ^ f) & ge);
}

// Tally of pair classes below 2^BITS, four pairs (bytes) at a time: how
// many pairs have each combination of class bits set (bit planes), from
// which the count of every class follows by inclusion-exclusion.
template <int BITS>
struct ClassTally {
    static constexpr int kSets = (1 << BITS) - 1;
    unsigned n = 0;               // pairs
    uint32_t acc[kSets] = {};     // per byte lane: pairs whose class has all bits of S (S = 1 .. 2^BITS - 1)
    // At most 63 calls between flushes (a byte lane holds up to 255, the
    // four lanes' sum is formed in the top byte).
    __device__ __forceinline__ void add4(uint32_t cls)
    {
        n += 4u;
#pragma unroll
        for (int S = 1; S <= kSets; ++S) {
            uint32_t b = 0x01010101u;
#pragma unroll
            for (int j = 0; j < BITS; ++j)
                if ((S >> j) & 1) b &= cls >> j;
            acc[S - 1] += b;
        }
    }
    // Pairs of class d: sum over S containing d of (-1)^|S - d| N_S.
    __device__ __forceinline__ unsigned count(int d) const
    {
        int c = 0;
#pragma unroll
        for (int S = 0; S <= kSets; ++S) {
            if ((S & d) != d) continue;
            const int ns = S ? (int)((acc[S - 1] * 0x01010101u) >> 24) : (int)n;
            c += (__popc(S ^ d) & 1) ? -ns : ns;
        }
        return (unsigned)c;
    }
    // Warp sum of every class count into a shared histogram (all 32 lanes).
    __device__ __forceinline__ void flush(unsigned int *hist, int nclass) const
    {
#pragma unroll
        for (int d = 0; d <= kSets; ++d) {
            const unsigned int v = __reduce_add_sync(FULL, count(d));
            if ((threadIdx.x & 31) == 0 && v && d < nclass) atomicAdd(&hist[d], v);
        }
    }
};

// Clock classes of the pairs (row byte c, px byte c) and (row byte c, py
// byte c), c < ncols, into a shared histogram; the row words hold valid
// states, q <= 15.  All 32 lanes of the warp.
template <int BITS>
__device__ __forceinline__ void tally_pairs(unsigned int *hist, const uint32_t (&wd)[8], const uint32_t (&px)[8],
                                            const uint32_t (&py)[8], int ncols, bool rv, uint32_t q4, int nclass)
{
    ClassTally<BITS> t;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!(rv && 4 * k < ncols)) continue;   // ncols % 4 == 0
        t.add4(clock_classes4(wd[k], clock_valid4(px[k], q4), q4));
        t.add4(clock_classes4(wd[k], clock_valid4(py[k], q4), q4));
    }
    t.flush(hist, nclass);
}

// The same for any q, one pair at a time.
__device__ __forceinline__ void tally_pairs_any(unsigned int *hist, const uint32_t (&wd)[8], const uint32_t (&px)[8],
                                                const uint32_t (&py)[8], int ncols, bool rv, int q)
{
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const bool v = rv && c < ncols;
        const int s0 = byte_at(wd, c);
        add_hist_any(hist, clock_bond_class(s0, byte_at(px, c), q), v);
        add_hist_any(hist, clock_bond_class(s0, byte_at(py, c), q), v);
    }
}

// Clock classes of the incoming configuration seen from one half row of
// k_bonds, q <= 15 (classes below 2^BITS): the nearest-neighbour pairs
// (right, down) into hist_class, and the pairs at distance L/4 and L/2
// (Sec. 4, G(r,T)) into hist4 and hist2.  wd, dn and sr are the row, the
// row below and the state right of the row, all valid states.  All 32
// lanes of the warp.
template <int BITS>
__device__ __forceinline__ void clock_row_classes(unsigned int *hist_class, unsigned int *hist4, unsigned int *hist2,
                                                  const int8_t *spin, int L, int y, int x0, int ncols, bool rv, int q,
                                                  int nclass, const uint32_t (&wd)[8], const uint32_t (&dn)[8],
                                                  uint32_t sr)
{
    const uint32_t q4 = (uint32_t)q * 0x01010101u;
    {
        ClassTally<BITS> t;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (!(rv && 4 * k < ncols)) continue;   // ncols % 4 == 0
            const uint32_t nxt = (k < 7 && 4 * k + 4 < ncols) ? wd[(k + 1) & 7] : sr;
            t.add4(clock_classes4(wd[k], __funnelshift_r(wd[k], nxt, 8), q4));
            t.add4(clock_classes4(wd[k], dn[k], q4));
        }
        t.flush(hist_class, nclass);
    }
#pragma unroll 1
    for (int w = 0; w < 2; ++w) {
        uint32_t px[8], py[8];
        load_partners(spin, L, y, x0, w == 0 ? L / 4 : L / 2, ncols, rv, px, py);
        tally_pairs<BITS>(w == 0 ? hist4 : hist2, wd, px, py, ncols, rv, q4, nclass);
    }
}

// The states of the half row (y, x0 .. x0 + ncols - 1) and of the half row
// below it (periodic), four to a word, and the right neighbour of its last
// site.  Nothing is loaded unless rv (then all are 0).
__device__ __forceinline__ void load_half_rows(const int8_t *spin, int L, int y, int x0, int ncols, bool rv,
                                               uint32_t (&wd)[8], uint32_t (&dn)[8], uint32_t &sr)
{
    const size_t rowbase = (size_t)y * L + x0;
    const int yd = (y + 1 == L) ? 0 : y + 1;
    const uint32_t *row = reinterpret_cast<const uint32_t *>(spin + rowbase);
    const uint32_t *drow = reinterpret_cast<const uint32_t *>(spin + (size_t)yd * L + x0);
    if ((L & 15) == 0 && ncols == QW) {   // whole half row, 16-byte aligned
        const uint4 a0 = rv ? __ldg(reinterpret_cast<const uint4 *>(row)) : make_uint4(0, 0, 0, 0);
        const uint4 a1 = rv ? __ldg(reinterpret_cast<const uint4 *>(row) + 1) : make_uint4(0, 0, 0, 0);
        const uint4 b0 = rv ? __ldg(reinterpret_cast<const uint4 *>(drow)) : make_uint4(0, 0, 0, 0);
        const uint4 b1 = rv ? __ldg(reinterpret_cast<const uint4 *>(drow) + 1) : make_uint4(0, 0, 0, 0);
        wd[0] = a0.x; wd[1] = a0.y; wd[2] = a0.z; wd[3] = a0.w;
        wd[4] = a1.x; wd[5] = a1.y; wd[6] = a1.z; wd[7] = a1.w;
        dn[0] = b0.x; dn[1] = b0.y; dn[2] = b0.z; dn[3] = b0.w;
        dn[4] = b1.x; dn[5] = b1.y; dn[6] = b1.z; dn[7] = b1.w;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool ok = rv && 4 * k < ncols;
            wd[k] = ok ? __ldg(row + k) : 0u;
            dn[k] = ok ? __ldg(drow + k) : 0u;
        }
    }
    sr = 0;
    if (rv) {
        const int xr = (x0 + ncols == L) ? 0 : x0 + ncols;
        sr = (uint8_t)__ldg(spin + (size_t)y * L + xr);
    }
}

// Potts bonds of a half row (Sec. 2 step (ii)) from its states (wd, dn,
// sr as load_half_rows gives them): bit c of R / D is the bond from site c
// to its right / lower neighbour, set iff the two states are equal and the
// bond's lane of the site pair's BOND draw lies below the threshold.  eqR /
// eqD: the equal-neighbour masks.  rowbase: index of the half row's first
// site (even).  UNROLL: draws in flight per thread (registers vs overlap).
// The draws alone (they need no states): bit c of rR / rD is set iff the
// right / lower bond of site c would be active between equal states.
template <int UNROLL>
__device__ __forceinline__ void potts_draws(const Lattice &lat, unsigned long long t, size_t rowbase, int ncols,
                                            bool rv, unsigned &rR, unsigned &rD)
{
    rR = rD = 0u;
    if (rv) {
        const uint32_t pbase = (uint32_t)(rowbase >> 1);
        const uint32_t thr = lat.thr;
#pragma unroll UNROLL
        for (int p = 0; p < 16; ++p) {
            if (2 * p < ncols) {
                const uint4 u = draw4(lat, pbase + (uint32_t)p, t, kTagBond);
                rR |= ((unsigned)(u.x < thr) << (2 * p)) | ((unsigned)(u.z < thr) << (2 * p + 1));
                rD |= ((unsigned)(u.y < thr) << (2 * p)) | ((unsigned)(u.w < thr) << (2 * p + 1));
            }
        }
    }
}

// The equal-neighbour masks of the half row (the states are dead after it,
// before the draws).
__device__ __forceinline__ void potts_equal(int ncols, const uint32_t (&wd)[8], const uint32_t (&dn)[8], uint32_t sr,
                                            unsigned &eqR, unsigned &eqD)
{
    eqR = eqD = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t nxt = (k < 7 && 4 * k + 4 < ncols) ? wd[(k + 1) & 7] : sr;
        eqR |= zero_bytes4(wd[k] ^ __funnelshift_r(wd[k], nxt, 8)) << (4 * k);
        eqD |= zero_bytes4(wd[k] ^ dn[k]) << (4 * k);
    }
}

template <int UNROLL>
__device__ __forceinline__ void potts_bonds(const Lattice &lat, unsigned long long t, size_t rowbase, int ncols,
                                            bool rv, const uint32_t (&wd)[8], const uint32_t (&dn)[8], uint32_t sr,
                                            unsigned &R, unsigned &D, unsigned &eqR, unsigned &eqD)
{
    const unsigned V = ncols >= 32 ? FULL : ((1u << ncols) - 1u);
    potts_equal(ncols, wd, dn, sr, eqR, eqD);
    unsigned rR, rD;
    potts_draws<UNROLL>(lat, t, rowbase, ncols, rv, rR, rD);
    R = rv ? (rR & eqR & V) : 0u;
    D = rv ? (rD & eqD & V) : 0u;
}

// ---------------------------------------------------------------------------
// k_bonds: the bonds of every site (Sec. 2 step (ii); clock: Sec. 4).
// Thread = one 32-site half row of a tile: equal-neighbour masks from packed
// byte compares, one Philox draw per two sites against the integer
// threshold.  The masks of a tile are stored together (right bonds of its 64
// rows, two words a row, then the down bonds), including the bonds that
// cross into the next tile.  With measurement on it also counts the active
// bonds and the bond classes of the incoming configuration (the previous
// sweep's result).
// ---------------------------------------------------------------------------
// ANY_CLOCK: the batch holds a clock lattice; the clock code is compiled in
// (the launches of a sweep use only this variant: Potts-only batches draw
// their bonds in the labeling kernel).  The bounds keep the clock measuring
// variant at 80 registers.
template <bool MEASURE, bool ANY_CLOCK>
__global__ void __launch_bounds__(kBlockThreads, ANY_CLOCK ? (MEASURE ? 6 : 1) : 8) k_bonds(Batch b)
{
    // Clock model: bond threshold of every state pair (a, b) for the sweep's
    // mirror axis, zero unless both project strictly onto the same side.
    __shared__ uint32_t s_thr[SW_MAX_CLOCK_Q * SW_MAX_CLOCK_Q];
    __shared__ unsigned int hist_class[SW_MAX_CLOCK_Q / 2 + 2];
    __shared__ unsigned int hist_corr[2][SW_MAX_CLOCK_Q / 2 + 2];   // clock: pairs at L/4, L/2
    __shared__ unsigned int red[32];
    __shared__ __align__(16) Lattice lat;
    __shared__ TaskCtx ctx;

    pdl_begin();
    unsigned int active = 0, unequal = 0, pairs = 0;
    int cur = -1;
    // Counters of lattice `cur` -> its ring rows (whole block).
    auto flush = [&]() {
        if (MEASURE && cur >= 0) {
            block_add<kBlockThreads>(ring_row(lat, ctx.t) + lat.q + lat.nclass, active, red);
            if (ctx.count_classes) {
                unsigned long long *prev = ring_row(lat, ctx.t - 1);
                if (!lat.clock) {
                    block_add<kBlockThreads>(prev + lat.q + 1, unequal, red);
                    block_add<kBlockThreads>(prev + lat.q + 0, pairs - unequal, red);
                } else if (ANY_CLOCK) {
                    __syncthreads();
                    const int nc = lat.nclass;
                    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
                        if (hist_class[k]) atomicAdd(prev + lat.q + k, (unsigned long long)hist_class[k]);
                        for (int w = 0; w < 2; ++w)
                            if (hist_corr[w][k])
                                atomicAdd(prev + lat.q + nc + 2 + w * nc + k, (unsigned long long)hist_corr[w][k]);
                    }
                }
            }
        }
        active = unequal = pairs = 0;
        __syncthreads();
    };

    const int nrep = __ldg(&b.dev->nrep), ntasks = __ldg(&b.dev->ntasks);
    for (int task = blockIdx.x; task < ntasks; task += gridDim.x) {
        const int rep = find_rep(b.task_off, nrep, task);
        if (rep != cur) {
            flush();
            load_lattice(&lat, b.lat + rep);
            __syncthreads();
            if (threadIdx.x == 0) ctx = task_context<MEASURE>(lat);
            if (MEASURE)
                for (int k = threadIdx.x; k < SW_MAX_CLOCK_Q / 2 + 2; k += blockDim.x)
                    hist_class[k] = hist_corr[0][k] = hist_corr[1][k] = 0u;
            __syncthreads();
            if (lat.clock) {
                // Projection of state k: j = (2k - m) mod 2q, magnitude j mod q,
                // side 1 (j < q) or 2 (j > q), none on the axis (j = 0, q).
                const int q = lat.q;
                for (int i = threadIdx.x; i < q * q; i += blockDim.x) {
                    const int ja = clock_class(i / q, ctx.m, q), jb = clock_class(i % q, ctx.m, q);
                    const int sa = (ja == 0 || ja == q) ? 0 : (ja < q ? 1 : 2);
                    const int sb = (jb == 0 || jb == q) ? 0 : (jb < q ? 1 : 2);
                    s_thr[i] = (sa != 0 && sa == sb) ? __ldg(lat.thr_tab + (ja % q) * (2 * q) + (jb % q)) : 0u;
                }
                __syncthreads();
            }
            cur = rep;
        }
        if (!ctx.active) continue;   // past its sweep limit: left as it is (uniform in the block)
        const int tile = task - __ldg(b.task_off + rep);
        const int L = lat.L, q = lat.q;
        const bool clock = ANY_CLOCK && lat.clock != 0;
        if (!ANY_CLOCK && lat.clock && threadIdx.x == 0) record_error(lat.st, kErrInternal, 0);   // wrong variant
        const unsigned long long t = ctx.t;
        // Clock bond threshold of valid states a, b.
        auto cthr = [&](int a, int c) -> uint32_t { return s_thr[a * q + c]; };
        const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
        const int X0 = bx * TW, Y0 = by * TH;
        const int tw = min(TW, L - X0), th = min(TH, L - Y0);          // valid extent of the tile
        const int ry = threadIdx.x >> 1, hx = threadIdx.x & 1;          // my half row
        const int x0 = X0 + QW * hx, y = Y0 + ry;
        const int ncols = max(0, min(QW, tw - QW * hx));
        const bool rv = ry < th && ncols > 0;
        const unsigned V = ncols >= 32 ? FULL : ((1u << ncols) - 1u);
        uint32_t wd[8], dn[8], sr;
        const size_t rowbase = (size_t)y * L + x0;   // meaningful only if rv
        load_half_rows(lat.spin, L, y, x0, ncols, rv, wd, dn, sr);
        if (clock) {   // states outside [0, q) read as 0: they index the q x q threshold table
            const uint32_t q4 = (uint32_t)q * 0x01010101u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                wd[k] = clock_valid4(wd[k], q4);
                dn[k] = clock_valid4(dn[k], q4);
            }
            sr = (uint32_t)valid_state((int)sr, q);
        }
        unsigned eqR = 0, eqD = 0, R = 0, D = 0;
        if (!clock) {
            potts_bonds<16>(lat, t, rowbase, ncols, rv, wd, dn, sr, R, D, eqR, eqD);
        } else if (rv) {
            unsigned rR = 0, rD = 0;
            const uint32_t pbase = (uint32_t)(rowbase >> 1);
            {
#pragma unroll
                for (int p = 0; p < 16; ++p) {
                    if (2 * p < ncols) {
                        const uint4 u = draw4(lat, pbase + (uint32_t)p, t, kTagBond);
                        const int c0 = 2 * p, c1 = 2 * p + 1;
                        const int s0 = byte_at(wd, c0), s1 = byte_at(wd, c1);
                        const int s2 = (c1 + 1 < ncols) ? byte_at(wd, (c1 + 1) & 31) : (int)sr;
                        rR |= ((unsigned)(u.x < cthr(s0, s1)) << c0) | ((unsigned)(u.z < cthr(s1, s2)) << c1);
                        rD |= ((unsigned)(u.y < cthr(s0, byte_at(dn, c0))) << c0) |
                              ((unsigned)(u.w < cthr(s1, byte_at(dn, c1))) << c1);
                    }
                }
            }
            R = rR & V;
            D = rD & V;
        }
        if (MEASURE) {
            active += __popc(R) + __popc(D);
            if (ctx.count_classes) {
                if (!clock) {
                    if (rv) {
                        unequal += __popc(~eqR & V) + __popc(~eqD & V);
                        pairs += 2u * (unsigned)ncols;
                    }
                } else if (lat.nclass <= 4) {
                    // q <= 7: classes in two bits, four pairs per word,
                    // tallied by bit planes and reduced over the warp.
                    clock_row_classes<2>(hist_class, hist_corr[0], hist_corr[1], lat.spin, L, y, x0, ncols, rv, q,
                                         lat.nclass, wd, dn, sr);
                } else if (lat.nclass <= 8) {   // q <= 15: three bits
                    clock_row_classes<3>(hist_class, hist_corr[0], hist_corr[1], lat.spin, L, y, x0, ncols, rv, q,
                                         lat.nclass, wd, dn, sr);
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const bool v = rv && c < ncols;
                        const int s0 = byte_at(wd, c);
                        const int s1 = (c + 1 < ncols) ? byte_at(wd, (c + 1) & 31) : (int)sr;
                        add_hist_any(hist_class, clock_bond_class(s0, s1, q), v);
                        add_hist_any(hist_class, clock_bond_class(s0, byte_at(dn, c), q), v);
                    }
                    // Correlation pairs at r = L/4 and r = L/2 (Sec. 4, G(r,T)).
#pragma unroll 1
                    for (int w = 0; w < 2; ++w) {
                        uint32_t px[8], py[8];
                        load_partners(lat.spin, L, y, x0, w == 0 ? L / 4 : L / 2, ncols, rv, px, py);
                        tally_pairs_any(hist_corr[w], wd, px, py, ncols, rv, q);
                    }
                }
            }
        }
        uint32_t *tb = lat.bond + (size_t)tile * kBondWords;
        tb[threadIdx.x] = R;                  // word (row ry, half hx) of the right bonds
        tb[kBlockThreads + threadIdx.x] = D;  // ... of the down bonds
    }
    flush();
}

// Segmented prefix OR: bit c of the result is the OR of the bits of x from
// the start of c's segment up to c; segments start at the set bits of m and
// at bit 0.  Five doubling steps.
__device__ __forceinline__ unsigned seg_or(unsigned x, unsigned m)
{
    unsigned p = ~m & ~1u;   // bit c may receive from bit c - 1
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
        x |= (x << sh) & p;
        p &= p << sh;
    }
    return x;
}

// Bit c is set iff bit c of x is set and no lower bit of x lies in c's
// segment (segments as above).
__device__ __forceinline__ unsigned seg_first(unsigned x, unsigned m)
{
    return x & ~((seg_or(x, m) << 1) & ~m);
}

// Run start at or left of column c (0..31) in a row's run-start word.
__device__ __forceinline__ int run_start(unsigned s, int c)
{
    return 31 - __clz(s & (FULL >> (31 - c)));
}

// Per quadrant row, for the scan: run starts, the first down bond from the
// row above into each run ("hook"), and the starts of the hooked runs.
// D: the row's down bonds inside the tile (for the seam between quadrants).
struct RowMasks {
    unsigned S, H, HS, D;
};

// ---------------------------------------------------------------------------
// k_label_tiles
//
// One block labels one 64 x 64 tile; warp w owns the 32 x 32 quadrant
// (qx, qy) = (w & 1, w >> 1).
//   masks    (lane = row) runs are the maximal horizontally bonded segments
//            of a quadrant row, found with bit operations: run starts, the
//            first down bond reaching each run from the row above (its
//            hook), and every further down bond that is the first to join a
//            distinct pair of runs.
//   scan     (lane = column, row by row, as in Hoshen-Kopelman, Sec. 2) a
//            hooked run takes the provisional label of the site above its
//            hook; any other run opens a provisional label, its first node
//            (tile node row * 64 + column, ordered like site indices).
//            Every node's word holds its provisional label; for the first
//            node of a run that opened one, that is the node itself, so the
//            same words serve as the union-find parents of the labels.
//   unions   the further down bonds, the quadrant seams (column 31 | 32,
//            row 31 | 32) join provisional labels in that union-find,
//            larger root under smaller, so a component's root is its
//            smallest site.
//   open     a component reaching the tile border (left and top edges
//            always, right and bottom edges through an active crossing
//            bond) continues in the neighbouring tile.
//   settle   a closed root draws its cluster's new state (Sec. 2 steps
//            (v)-(vii); clock: the reflection flag, Sec. 4); an open root
//            takes a slot and becomes a node of the global union-find; then
//            every other provisional label takes its root's resolved word
//            (with debug labels: points at its root).
//   codes    every site gets its cluster's 2-byte code, 0x100 | new state
//            (closed Potts), 0x100 | reflection flag (closed clock) or the
//            open slot; the open slots of the right and left edge sites go
//            to the tile's edge bytes.
// ---------------------------------------------------------------------------
// FUSED (batches without a clock lattice): the bonds are drawn here, each
// thread its half row (as k_bonds does), instead of read from the bond
// masks; the Philox work then fills the issue slots the labeling leaves.
template <bool MEASURE, bool LABELS, bool FUSED>
__global__ void __launch_bounds__(kBlockThreads, FUSED ? kLabelResidentFused : 11) k_label_tiles(Batch b)
{
    // Node words: provisional label of every node, which for a label's own
    // first node is its union-find parent.
    __shared__ __align__(16) uint16_t X[NS];
    // The union pairs (provisional labels of both ends, packed in a word);
    // then the list of provisional labels.
    __shared__ __align__(16) uint16_t rlist[NS];
    uint32_t *upairs = reinterpret_cast<uint32_t *>(rlist);
    constexpr int kUnionList = NS / 2;
    __shared__ __align__(16) RowMasks sm[TH][2];      // scan masks by (row, half)
    __shared__ unsigned int openw[NS / 32];           // open roots
    __shared__ int s_nroots, s_nopen, s_npairs, s_nclosed;
    __shared__ unsigned int s_cross[kCrossWords];
    __shared__ unsigned int red[32];
    __shared__ __align__(16) Lattice lat;
    __shared__ TaskCtx ctx;
    __shared__ unsigned long long s_pre_t;   // FUSED: sweep index of the first tile's early draws

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qx = warp & 1, qy = warp >> 1;
    const int row = QW * qy + lane;   // my tile row (lane = row phases)
    const int nrep = __ldg(&b.dev->nrep), ntasks = __ldg(&b.dev->ntasks);
    if (FUSED) {
        // Before the wait for the previous kernel: the bond draws of the
        // block's first tile need only the sweep index, which the merge
        // kernel of the previous sweep announced (next_t; that kernel has
        // completed once this block runs).  Kept in the room of the union
        // list until the first masks phase, used there if the index holds.
        if (threadIdx.x == 0) s_pre_t = ~0ull;
        if ((int)blockIdx.x < ntasks) {
            const int rep0 = find_rep(b.task_off, nrep, (int)blockIdx.x);
            load_lattice(&lat, b.lat + rep0);
            __syncthreads();
            const unsigned long long t0 = read_u64(&lat.st->next_t);
            const int tile = (int)blockIdx.x - __ldg(b.task_off + rep0);
            const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
            const int X0 = bx * TW, Y0 = by * TH;
            const int ncols = max(0, min(QW, min(TW, lat.L - X0) - QW * qx));
            const int nrows = max(0, min(QW, min(TH, lat.L - Y0) - QW * qy));
            const bool rv = ncols > 0 && lane < nrows;
            unsigned rR, rD;
            potts_draws<kFusedDrawUnroll>(lat, t0, (size_t)(Y0 + row) * lat.L + X0 + QW * qx, ncols, rv, rR, rD);
            upairs[threadIdx.x] = rR;
            upairs[kBlockThreads + threadIdx.x] = rD;
            if (threadIdx.x == 0) s_pre_t = t0;
        }
    }
    pdl_begin();

    unsigned int closed_roots = 0;
    unsigned int active = 0, unequal = 0, pairs = 0;   // FUSED: k_bonds' counters
    int cur = -1;
    if (threadIdx.x < kCrossWords) s_cross[threadIdx.x] = 0u;   // before the first barrier below
    // Counters of lattice `cur` -> its ring rows (whole block).
    auto flush = [&]() {
        if (MEASURE && cur >= 0) {
            block_add<kBlockThreads>(ring_row(lat, ctx.t) + lat.q + lat.nclass + 1, closed_roots, red);
            if (FUSED) {
                block_add<kBlockThreads>(ring_row(lat, ctx.t) + lat.q + lat.nclass, active, red);
                if (ctx.count_classes) {
                    unsigned long long *prev = ring_row(lat, ctx.t - 1);
                    block_add<kBlockThreads>(prev + lat.q + 1, unequal, red);
                    block_add<kBlockThreads>(prev + lat.q + 0, pairs - unequal, red);
                }
            }
        }
        closed_roots = active = unequal = pairs = 0;
        __syncthreads();
    };

    for (int task = blockIdx.x; task < ntasks; task += gridDim.x) {
        const int rep = find_rep(b.task_off, nrep, task);
        if (rep != cur) {
            flush();
            load_lattice(&lat, b.lat + rep);
            __syncthreads();
            if (threadIdx.x == 0) ctx = task_context<MEASURE>(lat);
            __syncthreads();
            cur = rep;
        }
        if (!ctx.active) continue;   // past its sweep limit: left as it is (uniform in the block)
        const int tile = task - __ldg(b.task_off + rep);
        const int L = lat.L, q = lat.q;
        const unsigned long long t = ctx.t;
        const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
        const int X0 = bx * TW, Y0 = by * TH;
        const int tw = min(TW, L - X0), th = min(TH, L - Y0);          // valid extent of the tile
        const int ncols = max(0, min(QW, tw - QW * qx));
        const int nrows = max(0, min(QW, th - QW * qy));
        const bool qa = ncols > 0 && nrows > 0;                        // quadrant has sites (warp-uniform)
        const bool rv = qa && lane < nrows;                            // my row has sites
        const unsigned V = ncols >= 32 ? FULL : ((1u << ncols) - 1u);
        const bool ext_right = QW * qx + ncols == tw;                   // my right edge is the tile's
        const bool ext_bottom = QW * qy + nrows == th;
        const int cap = lat.dbg_loop_cap > 0 ? lat.dbg_loop_cap : NS + 1;   // loop bound
        const int ulist = lat.dbg_list_cap > 0 ? min(kUnionList, lat.dbg_list_cap) : kUnionList;

        // ===== masks (lane = row; bond masks written by k_bonds or drawn here) ====
        unsigned S = 0u, U2 = 0u;
        bool seam = false;
        {
            unsigned R, D;
            if (FUSED) {
                if (lat.clock && threadIdx.x == 0) record_error(lat.st, kErrInternal, 0);   // wrong variant
                const int y = Y0 + row, x0 = X0 + QW * qx;
                uint32_t wd[8], dn[8], sr;
                load_half_rows(lat.spin, L, y, x0, ncols, rv, wd, dn, sr);
                unsigned eqR, eqD, rR, rD;
                potts_equal(ncols, wd, dn, sr, eqR, eqD);
                if (task == (int)blockIdx.x && t == s_pre_t) {   // the early draws hold (uniform in the block)
                    rR = upairs[threadIdx.x];
                    rD = upairs[kBlockThreads + threadIdx.x];
                } else {
                    potts_draws<kFusedDrawUnroll>(lat, t, (size_t)y * L + x0, ncols, rv, rR, rD);
                }
                R = rv ? (rR & eqR & V) : 0u;
                D = rv ? (rD & eqD & V) : 0u;
                if (MEASURE) {
                    active += __popc(R) + __popc(D);
                    if (ctx.count_classes && rv) {
                        unequal += __popc(~eqR & V) + __popc(~eqD & V);
                        pairs += 2u * (unsigned)ncols;
                    }
                }
            } else {
                const uint32_t *tb = lat.bond + (size_t)tile * kBondWords + row * 2 + qx;
                R = rv ? __ldg(tb) : 0u;
                D = rv ? __ldg(tb + kBlockThreads) : 0u;
            }
            if (qa) {
                const unsigned rc_bits = __ballot_sync(FULL, rv && ((R >> (ncols - 1)) & 1u));   // leaving the right edge
                const unsigned dc_bits = __shfl_sync(FULL, D, nrows - 1) & V;                   // leaving the bottom edge
                if (lane == 0) {
                    if (ext_right) atomicOr(&s_cross[qy], rc_bits);
                    if (ext_bottom) atomicOr(&s_cross[2 + qx], dc_bits);
                }
            }
            const unsigned Rq = R & (V >> 1);                // right bonds with both ends in the quadrant
            S = rv ? (~(Rq << 1) & V) : 0u;                  // run starts (column 0 always starts one)
            const unsigned Din = (rv && row + 1 < th) ? (D & V) : 0u;   // down bonds inside the tile
            // Down bonds from the row above, inside the quadrant.
            const unsigned Dup = __shfl_up_sync(FULL, Din, 1);
            const unsigned Sp = __shfl_up_sync(FULL, S, 1);
            const unsigned Dp = lane > 0 ? Dup : 0u;
            const unsigned H = seg_first(Dp, S);                              // hook of each run
            const unsigned E = (S >> 1) | 0x80000000u;                        // run ends
            const unsigned HS = S & __brev(seg_or(__brev(Dp), __brev(E)));    // starts of hooked runs
            U2 = rv ? (seg_first(Dp, S | Sp) & ~H) : 0u;                      // further run pairs
            seam = rv && qx == 0 && tw > QW && ((R >> 31) & 1u);             // column 31 -> 32
            sm[row][qx] = RowMasks{S, H, HS, Din};
        }
        openw[threadIdx.x] = 0u;
        static_assert(NS / 32 == kBlockThreads, "one open word per thread");
        if (threadIdx.x == 0) s_nroots = s_nopen = s_npairs = s_nclosed = 0;
        __syncthreads();

        // ===== scan (lane = column): provisional labels row by row ============
        // Four rows per step (nrows % 4 == 0): their mask work is independent
        // and overlaps the chain through lab.
        if (qa) {
            const int c = lane;
            int lab = 0;
            uint16_t *pl = X + QW * qy * TW + QW * qx + c;
            const RowMasks *ms = &sm[QW * qy][qx];
            const int nb0 = QW * qy * TW + QW * qx;
            auto scan_row = [&](int r) {
                const RowMasks m = ms[2 * r];
                const int s0 = run_start(m.S, c);
                const bool hooked = (m.HS >> s0) & 1u;
                const int fc = s0 + __ffs(m.H >> s0) - 1;
                const int up = __shfl_sync(FULL, lab, fc & 31);
                lab = hooked ? up : nb0 + r * TW + s0;
                pl[r * TW] = (uint16_t)lab;
            };
            // A whole quadrant unrolled: every row offset is a constant (the
            // kernel that draws the bonds has no registers to spare for it).
            if (!FUSED && nrows == QW) {
#pragma unroll
                for (int r = 0; r < QW; ++r) scan_row(r);
            } else {
                for (int r0 = 0; r0 < nrows; r0 += 4) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) scan_row(r0 + j);
                }
            }
        }
        __syncthreads();

        // ===== unions: further run pairs and the quadrant seams ===============
        // Each lane (row) lists its pairs of provisional labels: further down
        // bonds from the row above, the right bond across column 31 | 32 and,
        // for row 32, the down bonds across row 31 | 32 of its half.  All
        // threads then join the listed pairs; pairs beyond the list's room
        // are joined by their lane.
        {
            const int nb = row * TW + QW * qx;
            // Row 31 | 32 of my half: lane = column, one pair per lane at most.
            bool fs = false;
            if (qy == 1 && qa) {
                const RowMasks above = sm[QW - 1][qx], below = sm[QW][qx];
                fs = (seg_first(above.D, above.S | below.S) >> lane) & 1u;
            }
            const int cnt = __popc(U2) + (int)fs + (int)seam;
            int incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(FULL, incl, d);
                if (lane >= d) incl += o;
            }
            int wbase = 0;
            if (lane == 31 && incl) wbase = atomicAdd(&s_npairs, incl);
            int at = __shfl_sync(FULL, wbase, 31) + incl - cnt;
            // Slots of pairs found redundant stay at 0 | 0 (a no-op union).
            // A pair whose two labels are already the same needs no union.
            auto put = [&](int a, int bn) {
                const uint32_t la = (uint32_t)X[a], lb = (uint32_t)X[bn];
                const uint32_t pr = la == lb ? 0u : (la | (lb << 16));
                if (at < ulist) {
                    upairs[at] = pr;
                } else if (!union_t(X, (int)(pr & 0xFFFFu), (int)(pr >> 16), cap)) {
                    record_error(lat.st, kErrUnionCap, Y0 * L + X0);
                }
                ++at;
            };
            while (U2) {   // the site above and the site itself
                const int c = __ffs(U2) - 1;
                U2 &= U2 - 1;
                put(nb - TW + c, nb + c);
            }
            if (fs) put((QW - 1) * TW + QW * qx + lane, QW * TW + QW * qx + lane);
            if (seam) put(nb + QW - 1, nb + QW);
        }
        __syncthreads();
        {
            // Each thread joins a contiguous run of the list: pairs listed
            // together (neighbouring rows of one quadrant) often share a
            // component, and run one after the other instead of contending
            // for its root at once.
            const int np = min(s_npairs, ulist);
            const int per = (np + (int)blockDim.x - 1) / (int)blockDim.x;
            const int i1 = min(np, ((int)threadIdx.x + 1) * per);
            for (int i = (int)threadIdx.x * per; i < i1; ++i) {
                const uint32_t pr = upairs[i];
                if (pr != 0u && !union_t(X, (int)(pr & 0xFFFFu), (int)(pr >> 16), cap))
                    record_error(lat.st, kErrUnionCap, Y0 * L + X0);
            }
        }
        __syncthreads();

        // ===== open components: left and top edges always, right and bottom
        // edges through an active crossing bond.  Items: left column, top
        // row, right column, bottom row.  Also: the provisional labels listed.
        for (int item = threadIdx.x; item < 4 * TW; item += blockDim.x) {
            const int side = item / TW, k = item % TW;
            int node = -1;
            if (side == 0) {
                if (k < th) node = k * TW;
            } else if (side == 1) {
                if (k < tw) node = k;
            } else if (side == 2) {
                if (k < th && ((s_cross[k >> 5] >> (k & 31)) & 1u)) node = k * TW + tw - 1;
            } else {
                if (k < tw && ((s_cross[2 + (k >> 5)] >> (k & 31)) & 1u)) node = (th - 1) * TW + k;
            }
            int rt = -1;
            if (node >= 0) {
                rt = find_t_ro(X, X[node], cap);
                if (rt < 0) record_error(lat.st, kErrFindCap, Y0 * L + X0);
            }
            const unsigned peers = __match_any_sync(FULL, rt);   // one atomic per distinct root
            if (rt >= 0 && (__ffs(peers) - 1) == lane) atomicOr(&openw[rt >> 5], 1u << (rt & 31));
        }
        {   // provisional labels: the first nodes of the runs that opened one
            const unsigned F = S & ~sm[row][qx].HS;
            const int cnt = __popc(F);
            int incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(FULL, incl, d);
                if (lane >= d) incl += o;
            }
            int wbase = 0;
            if (lane == 31 && incl) wbase = atomicAdd(&s_nroots, incl);
            int at = __shfl_sync(FULL, wbase, 31) + incl - cnt;
            const int nb = row * TW + QW * qx;
            for (unsigned f = F; f; f &= f - 1) rlist[at++] = (uint16_t)(nb + __ffs(f) - 1);
        }
        __syncthreads();

        // ===== settle: a closed root draws, an open root takes a slot; its
        // word becomes resolved.  Then every other provisional label takes
        // the resolved word of its root (debug labels: its root's index, in
        // one pass whose walks stop at a root, settled or not).
        // One-bit cluster draws (bit_draw): the STATE_BIT bits of the tile's
        // sites, eight words per tile row from the two draws that cover the
        // row, in the room of the scan masks (free after the open phase).
        uint32_t *bits = reinterpret_cast<uint32_t *>(&sm[0][0]);
        static_assert(sizeof(sm) == TH * 8 * sizeof(uint32_t) && kBlockThreads == 2 * TH, "two draws per tile row");
        const bool onebit = bit_draw(lat);
        if (onebit) {
            const int r = threadIdx.x >> 1, h = threadIdx.x & 1;
            if (r < th) {
                const uint32_t g0 = (uint32_t)(Y0 + r) * (uint32_t)L + (uint32_t)X0;
                if (h == 0 || (g0 & 127u) + (uint32_t)tw > 128u)
                    reinterpret_cast<uint4 *>(bits)[2 * r + h] = draw4(lat, (g0 >> 7) + (uint32_t)h, t, kTagStateBit);
            }
            __syncthreads();
        }
        {
            const int nlab = s_nroots;
            for (int i = threadIdx.x; i < nlab; i += blockDim.x) {
                const int v = rlist[i];
                int x = v;
                if (LABELS) {
                    bool found = false;
                    for (int it = 0; it < cap; ++it) {   // read-only: stops at a root, settled or not
                        const int p = X[x];
                        if (p == x || p >= kTileResolved) {
                            found = true;
                            break;
                        }
                        x = p;
                    }
                    if (!found) record_error(lat.st, kErrFindCap, Y0 * L + X0);
                    if (x != v) {
                        X[v] = (uint16_t)x;
                        continue;
                    }
                } else if (X[v] != v) {   // not a root: takes its root's word below
                    continue;
                }
                const int g = tile_site(L, bx, by, v);
                int w;
                if ((openw[v >> 5] >> (v & 31)) & 1u) {
                    const int slot = atomicAdd(&s_nopen, 1);
                    if (slot < kOpenSlots) {   // at most 2 * (64 + 64) - 4 open components
                        const uint32_t id = (uint32_t)tile * kOpenSlots + (uint32_t)slot;
                        lat.opar[id] = ((unsigned long long)(uint32_t)g << 32) | id;
                        w = kTileResolved | slot;
                    } else {
                        record_error(lat.st, kErrInternal, g);
                        w = kTileResolved | kCodeClosed;
                    }
                } else {
                    int d;
                    if (onebit) {   // bit g of the draws (draw_bit)
                        const int r = v / TW;
                        const uint32_t g0 = (uint32_t)(Y0 + r) * (uint32_t)L + (uint32_t)X0;
                        d = (int)((bits[8 * r + ((uint32_t)g >> 5) - 4 * (g0 >> 7)] >> (g & 31)) & 1u);
                    } else {
                        d = mulhi_q(draw4(lat, (uint32_t)g, t, kTagState).x, q);
                    }
                    w = kTileResolved | kCodeClosed | d;
                    ++closed_roots;
                    if (lat.stats) atomicAdd(&s_nclosed, 1);
                }
                X[v] = (uint16_t)w;
            }
            if (!LABELS) {
                // Every other label takes its cluster's resolved word, so a
                // node's word leads to it in one step.
                __syncthreads();
                for (int i = threadIdx.x; i < nlab; i += blockDim.x) {
                    const int v = rlist[i];
                    int x = X[v];
                    if (x >= kTileResolved) continue;   // a root
                    bool found = false;
                    for (int it = 0; it < cap; ++it) {   // resolved words: roots, or labels already done
                        const int p = X[x];
                        if (p >= kTileResolved) {
                            x = p;
                            found = true;
                            break;
                        }
                        x = p;
                    }
                    if (!found) {
                        record_error(lat.st, kErrFindCap, Y0 * L + X0);
                        x = kTileResolved | kCodeClosed;
                    }
                    X[v] = (uint16_t)x;
                }
            }
        }
        __syncthreads();

        // ===== codes: warp = quadrant, four rows of 32 columns a step, lane =
        // four columns; a node's word leads to its cluster's resolved word in
        // at most one more step (its label), two with debug labels (label ->
        // root).  Edge slots.
        if (qa) {
            const int c4 = 4 * (lane & 7);
            const bool cv = c4 < ncols;   // ncols % 4 == 0
            // Unrolled (loads of several steps in flight) where registers allow.
#pragma unroll(FUSED ? 1 : 4)
            for (int r = lane >> 3; r < nrows; r += 4) {
                const int row2 = QW * qy + r;
                const int v0 = row2 * TW + QW * qx + c4;
                if (!cv) continue;
                const uint2 w2 = *reinterpret_cast<const uint2 *>(X + v0);
                int wv[4] = {(int)(w2.x & 0xFFFFu), (int)(w2.x >> 16), (int)(w2.y & 0xFFFFu), (int)(w2.y >> 16)};
                int rt[4] = {v0, v0 + 1, v0 + 2, v0 + 3};
                // label -> root -> resolved word: two rounds of independent
                // loads (one where every label holds its resolved word)
#pragma unroll
                for (int it = 0; it < (LABELS ? 2 : 1); ++it) {
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                        if (wv[h] < kTileResolved) {
                            rt[h] = wv[h];
                            wv[h] = X[wv[h]];
                        }
                }
                if (!(wv[0] & wv[1] & wv[2] & wv[3] & kTileResolved)) {   // unreachable for a settled tile
                    record_error(lat.st, kErrInternal, Y0 * L + X0);
                    wv[0] = wv[1] = wv[2] = wv[3] = kTileResolved | kCodeClosed;
                }
                const size_t site = (size_t)(Y0 + row2) * L + X0 + QW * qx + c4;
                *reinterpret_cast<uint2 *>(lat.code + site) =
                    make_uint2(((uint32_t)wv[0] & kCodeMask) | (((uint32_t)wv[1] & kCodeMask) << 16),
                               ((uint32_t)wv[2] & kCodeMask) | (((uint32_t)wv[3] & kCodeMask) << 16));
                if (LABELS) {
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                        if (wv[h] & kCodeClosed) lat.label[site + h] = tile_site(L, bx, by, rt[h]);
                }
                uint8_t *eb = lat.edge + (size_t)tile * kEdgeBytes;
                if (qx == 0 && c4 == 0) eb[TH + row2] = (uint8_t)(wv[0] & 0xFF);   // left edge: column 0
                if (ext_right && c4 + 4 == ncols) eb[row2] = (uint8_t)(wv[3] & 0xFF);   // right edge: column tw - 1
            }
        }
        if (threadIdx.x == 0) {
            lat.open_count[tile] = min(s_nopen, kOpenSlots);
            if (lat.stats) {   // labeling statistics of the tile
                atomicAdd(lat.stats + kStatLabels, (unsigned long long)s_nroots);
                atomicAdd(lat.stats + kStatPairs, (unsigned long long)s_npairs);
                atomicAdd(lat.stats + kStatComponents, (unsigned long long)(s_nopen + s_nclosed));
                atomicAdd(lat.stats + kStatOpen, (unsigned long long)s_nopen);
            }
        }
        if (threadIdx.x < kCrossWords) {
            // Zeroed by its only reader, ready for the next task.
            lat.cross[(size_t)tile * kCrossWords + threadIdx.x] = s_cross[threadIdx.x];
            s_cross[threadIdx.x] = 0u;
        }
        __syncthreads();
    }
    flush();
}

// ---------------------------------------------------------------------------
// k_merge: union of the open components across every active crossing bond.
// Work items of a lattice: kMergeItems per tile, the 64 rows of its right
// edge, then the 64 columns of its bottom edge; a warp takes 32
// consecutive items (one side of one tile).  The slots of both ends come
// from the edge bytes (right edge -> left edge of the next tile) or from
// the codes of the bottom and top rows.
// ---------------------------------------------------------------------------
// STATS: a lattice of the batch gathers labeling statistics (the walk tallies
// are compiled in).
template <bool STATS>
__global__ void __launch_bounds__(256, 8) k_merge(Batch b)
{
    static_assert(kMergeItems == TH + TW, "merge items: right edge rows, then bottom edge columns");
    pdl_wait();
    {   // The sweep index the next labeling kernel runs at, announced before
        // this kernel lets the flip launch (the labeling kernel of this sweep
        // has completed: all its blocks have read the previous value).
        bool wrote = false;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < __ldg(&b.dev->nrep); r += gridDim.x * blockDim.x) {
            DevState *st = b.lat[r].st;
            const unsigned long long t = read_u64(&st->sweep);
            if (t < read_u64(&st->stop)) {
                *reinterpret_cast<volatile unsigned long long *>(&st->next_t) = t + 1;
                wrote = true;
            }
        }
        if (wrote) __threadfence();
    }
    pdl_release();
    long long lo = 0, hi = 0;
    int rep = -1;
    const Lattice *lp = b.lat;   // read through the L1, not copied into registers
    const unsigned lane = threadIdx.x & 31;
    OpenTally tl;           // labeling statistics of the warp's current lattice
    unsigned int unions = 0;
    bool active = true;     // the current lattice sweeps this time
    // A warp's items all belong to one lattice at a time: its tallies go to
    // that lattice's statistics (warp sums) when it moves on or finishes.
    auto flush_warp = [&]() {
        unsigned long long *st = lp->stats;
        if (st != nullptr) {
            const unsigned v[6] = {unions, tl.links, tl.retries, tl.finds, tl.hops, 0u};
            const int f[5] = {kStatUnions, kStatLinks, kStatRetries, kStatFinds, kStatHops};
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const unsigned s = __reduce_add_sync(0xffffffffu, v[i]);
                if (lane == 0 && s) atomicAdd(st + f[i], (unsigned long long)s);
            }
            const unsigned m = __reduce_max_sync(0xffffffffu, tl.max_hops);
            if (lane == 0 && m) atomicMax(st + kStatMaxHops, (unsigned long long)m);
        }
        tl = OpenTally();
        unions = 0;
    };
    // Every lattice has a multiple of kMergeItems items: a warp never spans
    // two lattices, and its trip count is uniform.
    const int nrep = __ldg(&b.dev->nrep);
    const long long nmerge = __ldg(&b.dev->nmerge);
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nmerge;
         base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + lane;
        bool ok = k < nmerge;
        uint32_t a = 0, c2 = 0;
        if (ok) {
            if (k < lo || k >= hi) {
                if (STATS && rep >= 0) flush_warp();   // uniform: the warp's items share a lattice
                rep = find_rep(b.merge_off, nrep, k);
                lo = __ldg(b.merge_off + rep);
                hi = __ldg(b.merge_off + rep + 1);
                lp = b.lat + rep;
                active = read_u64(&lp->st->sweep) < read_u64(&lp->st->stop);
            }
            const Lattice &lat = *lp;
            ok = active;
            const int L = lat.L;
            const int kk = (int)(k - lo);
            const int tile = kk / kMergeItems, e = kk % kMergeItems;
            const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
            const int X0 = bx * TW, Y0 = by * TH;
            const int tw = min(TW, L - X0), th = min(TH, L - Y0);
            const uint32_t *cw = lat.cross + (size_t)tile * kCrossWords;
            int sa = 0, sb = 0, nt;
            if (e < TH) {   // right edge, row e, into the next tile to the right
                ok = ok && e < th && ((__ldg(cw + (e >> 5)) >> (e & 31)) & 1u);
                nt = by * lat.tiles_x + (bx + 1 == lat.tiles_x ? 0 : bx + 1);
                if (ok) {
                    sa = lat.edge[(size_t)tile * kEdgeBytes + e];
                    sb = lat.edge[(size_t)nt * kEdgeBytes + TH + e];
                }
            } else {        // bottom edge, column e - 64, into the next tile below
                const int c = e - TH;
                ok = ok && c < tw && ((__ldg(cw + 2 + (c >> 5)) >> (c & 31)) & 1u);
                const int yn = by + 1 == lat.tiles_y ? 0 : by + 1;
                nt = yn * lat.tiles_x + bx;
                if (ok) {
                    sa = lat.code[(size_t)(Y0 + th - 1) * L + X0 + c];
                    sb = lat.code[(size_t)yn * TH * L + X0 + c];
                    if ((sa | sb) & kCodeClosed) {   // a crossing bond always ends at open sites
                        record_error(lat.st, kErrInternal, (Y0 + th - 1) * L + X0 + c);
                        ok = false;
                    }
                }
            }
            a = (uint32_t)tile * kOpenSlots + (uint32_t)sa;
            c2 = (uint32_t)nt * kOpenSlots + (uint32_t)sb;
        }
        // Bonds of one warp that join the same two open components need one union.
        const unsigned vm = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned long long key = ((unsigned long long)a << 32) | c2;
            const unsigned peers = __match_any_sync(vm, key);
            if ((unsigned)__ffs(peers) - 1u == lane) {
                ++unions;
                union_open(lp->opar, a, c2,
                           lp->dbg_loop_cap > 0 ? lp->dbg_loop_cap : lp->tiles_x * lp->tiles_y * kOpenSlots + 1, lp->st,
                           tl);
            }
        }
    }
    if (STATS && rep >= 0) flush_warp();
}

// Last block of the sweep's final kernel: for every lattice of the batch,
// record that the incoming configuration's classes were counted, zero the
// next counter row and advance the sweep index (every block has read it).
template <bool MEASURE>
__device__ void finish_sweep(const Batch &b)
{
    __shared__ int s_last;
    pdl_wait();   // (the flip kernel waits late; also where a block had no tile to flip)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(b.ticket, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nrep = __ldg(&b.dev->nrep);
    for (int r = threadIdx.x; r < nrep; r += blockDim.x) {
        const Lattice &lt = b.lat[r];
        const unsigned long long t = read_u64(&lt.st->sweep);
        if (t >= read_u64(&lt.st->stop)) continue;   // did not sweep this time
        const bool counted = MEASURE && t >= 1ull && t - 1ull >= read_u64(&lt.st->classes_upto);
        unsigned long long *next = ring_row(lt, t + 1);
        for (int c = 0; c < lt.ncounters; ++c) next[c] = 0ull;
        if (lt.stats) lt.stats[kStatSweeps] += 1ull;
        if (counted) lt.st->classes_upto = t;
        __threadfence();
        *reinterpret_cast<volatile unsigned long long *>(&lt.st->sweep) = t + 1;
    }
    if (threadIdx.x == 0) *b.ticket = 0u;
}

// ---------------------------------------------------------------------------
// k_flip_tiles: the cluster roots and new states of the tile's open
// components, all spin writes, state counts.  One block per tile; a thread
// writes two 16-site chunks (chunk k: row k / 4, columns 16 (k % 4) ..).
// ---------------------------------------------------------------------------
template <bool MEASURE, bool LABELS, bool ANY_CLOCK, bool STATS>
__global__ void __launch_bounds__(kBlockThreads, ANY_CLOCK ? kFlipResidentClock : kFlipResidentPotts) k_flip_tiles(Batch b)
{
    // New state (Potts) or reflection flag (clock) of each open slot; then
    // entry kCodeClosed + s = s, so that a Potts code indexes its new state.
    __shared__ __align__(16) unsigned char tab[2 * kOpenSlots];
    __shared__ int rootg[LABELS ? kOpenSlots : 1];
    __shared__ unsigned int hist_state[SW_MAX_Q + 1];
    __shared__ unsigned int red[32];
    __shared__ __align__(16) Lattice lat;
    __shared__ TaskCtx ctx;

    pdl_release();   // the wait comes after the first codes are loaded
    const int r = threadIdx.x & 31;
    // q <= 8: state counts of this thread, 16 bits per state (states 0-3, 4-7);
    // q == 2: sites in cnt_hi, sites in state 1 in cnt_lo.
    unsigned long long cnt_lo = 0, cnt_hi = 0;
    unsigned int open_roots = 0;   // clusters reaching a tile border, counted at their root
    OpenTally tl;                  // labeling statistics of the root walks
    int cur = -1;
    // Codes are below 2 * kOpenSlots (kCodeMask): entries past the states are never used.
    static_assert(kCodeClosed == kOpenSlots && SW_MAX_Q <= 128 && kCodeMask < 2 * kOpenSlots, "codes index the table");
    for (int k = threadIdx.x; k < kOpenSlots; k += blockDim.x) tab[kOpenSlots + k] = (unsigned char)(k < SW_MAX_Q ? k : 0);
    auto flush = [&]() {
        if (STATS && cur >= 0) flush_open_tally<kBlockThreads>(lat.stats, tl, 0u, red);
        tl = OpenTally();
        if (MEASURE && cur >= 0) {
            block_add<kBlockThreads>(ring_row(lat, ctx.t) + lat.q + lat.nclass + 1, open_roots, red);
            if (lat.q == 2) {
                const unsigned int n1 = __reduce_add_sync(FULL, (unsigned int)cnt_lo);
                const unsigned int n = __reduce_add_sync(FULL, (unsigned int)cnt_hi);
                if (r == 0) {
                    if (n - n1) atomicAdd(&hist_state[0], n - n1);
                    if (n1) atomicAdd(&hist_state[1], n1);
                }
            } else if (lat.q <= 8) {
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const unsigned long long w = s < 4 ? cnt_lo : cnt_hi;
                    const unsigned int v = __reduce_add_sync(FULL, (unsigned int)((w >> (16 * (s & 3))) & 0xFFFFull));
                    if (r == 0 && s < lat.q && v) atomicAdd(&hist_state[s], v);
                }
            }
            __syncthreads();
            unsigned long long *row = ring_row(lat, ctx.t);
            for (int k = threadIdx.x; k < lat.q; k += blockDim.x)
                if (hist_state[k]) atomicAdd(row + k, (unsigned long long)hist_state[k]);
        }
        cnt_lo = cnt_hi = 0;
        open_roots = 0;
        __syncthreads();
    };
    const int nrep = __ldg(&b.dev->nrep), ntasks = __ldg(&b.dev->ntasks);
    for (int task = blockIdx.x; task < ntasks; task += gridDim.x) {
        const int rep = find_rep(b.task_off, nrep, task);
        if (rep != cur) {
            flush();
            load_lattice(&lat, b.lat + rep);
            __syncthreads();
            if (threadIdx.x == 0) ctx = task_context<MEASURE>(lat);
            for (int k = threadIdx.x; k < SW_MAX_Q + 1; k += blockDim.x) hist_state[k] = 0u;
            __syncthreads();
            cur = rep;
        }
        if (!ctx.active) continue;   // past its sweep limit: left as it is (uniform in the block)
        const int tile = task - __ldg(b.task_off + rep);
        const int L = lat.L, q = lat.q;
        const bool clock = ANY_CLOCK && lat.clock != 0;   // ANY_CLOCK: the batch holds a clock lattice
        if (!ANY_CLOCK && lat.clock && threadIdx.x == 0) record_error(lat.st, kErrInternal, 0);
        const int m = ctx.m;
        const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
        const int X0 = bx * TW, Y0 = by * TH;
        const int tw = min(TW, L - X0), th = min(TH, L - Y0);
        // My chunks: rows c0 / 4 and c0 / 4 + 32, columns 16 (c0 % 4) .. + 15.
        const int crow = threadIdx.x >> 2, ccol = 16 * (threadIdx.x & 3);
        const int cn = max(0, min(16, tw - ccol));   // valid columns of my chunks (a multiple of 4)
        const bool vec = (L & 15) == 0;              // 16-byte aligned chunks
        uint4 cwa[2], cwb[2], swv[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int rr = crow + 32 * j;
            const bool v = rr < th && cn > 0;
            const size_t site0 = (size_t)(Y0 + rr) * L + X0 + ccol;
            cwa[j] = cwb[j] = swv[j] = make_uint4(0u, 0u, 0u, 0u);
            if (v) {
                if (vec) {
                    cwa[j] = *reinterpret_cast<const uint4 *>(lat.code + site0);
                    cwb[j] = *reinterpret_cast<const uint4 *>(lat.code + site0 + 8);
                    if (clock) swv[j] = *reinterpret_cast<const uint4 *>(lat.spin + site0);
                } else {
                    const uint2 *cp = reinterpret_cast<const uint2 *>(lat.code + site0);
                    const uint32_t *sp = reinterpret_cast<const uint32_t *>(lat.spin + site0);
                    uint32_t c8[8] = {0, 0, 0, 0, 0, 0, 0, 0}, s4[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        if (4 * g < cn) {
                            const uint2 x = cp[g];
                            c8[2 * g] = x.x;
                            c8[2 * g + 1] = x.y;
                            if (clock) s4[g] = sp[g];
                        }
                    cwa[j] = make_uint4(c8[0], c8[1], c8[2], c8[3]);
                    cwb[j] = make_uint4(c8[4], c8[5], c8[6], c8[7]);
                    swv[j] = make_uint4(s4[0], s4[1], s4[2], s4[3]);
                }
            }
        }
        // The codes above are the labeling kernel's, two launches back; the
        // union-find entries below are the merge's: wait for it here.
        pdl_wait();
        // Every open component of the tile belongs to a cluster whose root
        // (the component with the cluster's smallest site, after the merge)
        // draws the new state (Potts) or the reflection flag (clock), Sec. 2
        // (v)-(vii) / Sec. 4, into the tile's table.  A cluster is counted
        // once, by the tile holding its root.
        {
            const int n = __ldg(lat.open_count + tile);
            const int cap = lat.dbg_loop_cap > 0 ? lat.dbg_loop_cap : lat.tiles_x * lat.tiles_y * kOpenSlots + 1;
            for (int s = threadIdx.x; s < n; s += blockDim.x) {
                const uint32_t x = (uint32_t)tile * kOpenSlots + (uint32_t)s;
                const unsigned long long e = find_open(lat.opar, x, cap, lat.st, tl);
                const uint32_t key = (uint32_t)(e >> 32);
                if (MEASURE && (uint32_t)e == x) ++open_roots;
                tab[s] = (unsigned char)cluster_draw(lat, key, ctx.t);
                if (LABELS) rootg[LABELS ? s : 0] = (int)key;
            }
        }
        __syncthreads();

        // The spin writes, with the state counts the lattice needs compiled
        // into each form (CM 1: q = 2, CM 2: q <= 8, CM 0: none here).
        auto write_chunks = [&](auto cm) {
            constexpr int CM = decltype(cm)::value;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int rr = crow + 32 * j;
                if (!(rr < th && cn > 0)) continue;
                const size_t site0 = (size_t)(Y0 + rr) * L + X0 + ccol;
                const uint32_t cws[8] = {cwa[j].x, cwa[j].y, cwa[j].z, cwa[j].w, cwb[j].x, cwb[j].y, cwb[j].z, cwb[j].w};
                const uint32_t sws[4] = {swv[j].x, swv[j].y, swv[j].z, swv[j].w};
                uint32_t out[4];
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    uint32_t word = 0;
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const uint32_t code = (cws[2 * g + (h >> 1)] >> (16 * (h & 1))) & (uint32_t)kCodeMask;
                        int ns;
                        if (clock) {   // closed: the cluster's flag in the code; open: its root's, in the table
                            const int k0 = valid_state((int)((sws[g] >> (8 * h)) & 0xFFu), q);
                            ns = ((code & kCodeClosed) ? (code & 1u) : tab[code & 0xFFu]) ? reflect(k0, m, q) : k0;
                        } else {
                            ns = tab[code];   // open slot or kCodeClosed | state
                        }
                        if (CM == 2 && 4 * g < cn) {
                            const unsigned long long one = 1ull << (16 * (ns & 3));
                            if (ns < 4) cnt_lo += one;
                            else cnt_hi += one;
                        }
                        if (LABELS && 4 * g < cn && !(code & kCodeClosed))
                            lat.label[site0 + 4 * g + h] = rootg[LABELS ? (code & 0xFF) : 0];
                        word |= (uint32_t)(ns & 0xFF) << (8 * h);
                    }
                    out[g] = word;
                    if (CM == 1 && 4 * g < cn) {   // states are 0 or 1
                        cnt_lo += (unsigned)__popc(word);
                        cnt_hi += 4u;
                    }
                }
                if (vec) {
                    *reinterpret_cast<uint4 *>(lat.spin + site0) = make_uint4(out[0], out[1], out[2], out[3]);
                } else {
                    uint32_t *sp = reinterpret_cast<uint32_t *>(lat.spin + site0);
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        if (4 * g < cn) sp[g] = out[g];
                }
            }
        };
        if (MEASURE && q == 2) write_chunks(std::integral_constant<int, 1>());
        else if (MEASURE && q <= 8) write_chunks(std::integral_constant<int, 2>());
        else write_chunks(std::integral_constant<int, 0>());
        if (MEASURE && q > 8) {
            // Many states: warp-aggregated shared histogram, site by site.
#pragma unroll 1
            for (int j = 0; j < 2; ++j) {
                const int rr = crow + 32 * j;
                const size_t site0 = (size_t)(Y0 + rr) * L + X0 + ccol;
                for (int h = 0; h < 16; ++h) {
                    const bool v = rr < th && h < cn;
                    const int ns = v ? (int)lat.spin[site0 + h] : 0;
                    add_hist_any(hist_state, ns, v && ns >= 0 && ns < q);
                }
            }
        }
        __syncthreads();   // the next tile reuses the open-state table
    }
    flush();
    finish_sweep<MEASURE>(b);
}

// ---------------------------------------------------------------------------
// k_pending_classes: bond classes of the current configuration into the
// last sweep's counter row, when no later labeling pass has counted them.
// ---------------------------------------------------------------------------
template <bool CLOCK>
__global__ void __launch_bounds__(kEnergyThreads) k_pending_classes(Lattice lat)
{
    __shared__ unsigned int hist[SW_MAX_CLOCK_Q / 2 + 2];
    __shared__ unsigned int hist_corr[2][SW_MAX_CLOCK_Q / 2 + 2];   // clock: pairs at L/4, L/2
    __shared__ unsigned int red[32];
    const unsigned long long t = read_u64(&lat.st->sweep);
    if (t == 0ull || t - 1ull < read_u64(&lat.st->classes_upto)) return;   // same for every block
    const int L = lat.L, q = lat.q;
    if (CLOCK)
        for (int k = threadIdx.x; k < lat.nclass; k += blockDim.x) hist[k] = hist_corr[0][k] = hist_corr[1][k] = 0u;
    __syncthreads();
    const long long N4 = (long long)L * L / 4;
    unsigned int unequal = 0, sites = 0;
    // Every thread of a block runs the same number of iterations (warp-wide
    // histogram calls below).
    for (long long base = (long long)blockIdx.x * blockDim.x; base < N4; base += (long long)gridDim.x * blockDim.x) {
        const long long g = base + threadIdx.x;
        const bool v = g < N4;
        int a[8] = {0, 0, 0, 0, 0, 0, 0, 0}, bb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (v) {
            const int i0 = (int)(4 * g);
            const int y = i0 / L, x = i0 - y * L;
            const char4 s = reinterpret_cast<const char4 *>(lat.spin)[g];
            const int yd = (y + 1 == L) ? 0 : y + 1;
            const char4 d = *reinterpret_cast<const char4 *>(lat.spin + (size_t)yd * L + x);
            const int sr = lat.spin[(size_t)y * L + ((x + 4 == L) ? 0 : x + 4)];
            const int aa[8] = {s.x, s.y, s.z, s.w, s.x, s.y, s.z, s.w};
            const int b2[8] = {s.y, s.z, s.w, sr, d.x, d.y, d.z, d.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                a[k] = aa[k];
                bb[k] = b2[k];
            }
            sites += 4;
        }
        if (CLOCK) {
#pragma unroll
            for (int k = 0; k < 8; ++k) add_hist_any(hist, clock_bond_class(a[k], bb[k], q), v);
            // Correlation pairs at r = L/4 and L/2 (Sec. 4, G(r,T)).
            const int i0 = v ? (int)(4 * g) : 0;
            const int y = i0 / L, x = i0 - y * L;
#pragma unroll 1
            for (int w = 0; w < 2; ++w) {
                const int r = w == 0 ? L / 4 : L / 2;
                const size_t yrow = (size_t)((y + r) % L) * L;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int sx = v ? lat.spin[(size_t)y * L + (x + k + r) % L] : 0;
                    const int sy = v ? lat.spin[yrow + x + k] : 0;
                    add_hist_any(hist_corr[w], clock_bond_class(a[k], sx, q), v);
                    add_hist_any(hist_corr[w], clock_bond_class(a[k], sy, q), v);
                }
            }
        } else if (v) {
#pragma unroll
            for (int k = 0; k < 8; ++k) unequal += (a[k] != bb[k]);
        }
    }
    unsigned long long *row = ring_row(lat, t - 1);
    if (CLOCK) {
        __syncthreads();
        const int nc = lat.nclass;
        for (int k = threadIdx.x; k < nc; k += blockDim.x) {
            if (hist[k]) atomicAdd(row + q + k, (unsigned long long)hist[k]);
            for (int w = 0; w < 2; ++w)
                if (hist_corr[w][k]) atomicAdd(row + q + nc + 2 + w * nc + k, (unsigned long long)hist_corr[w][k]);
        }
    } else {
        block_add<kEnergyThreads>(row + q + 1, unequal, red);
        block_add<kEnergyThreads>(row + q + 0, 2u * sites - unequal, red);
    }
}

// The same for the Potts model when rows are 16-byte aligned: sixteen sites
// per thread from one 16-byte load of the row and one of the row below.
__device__ __forceinline__ unsigned int zero_byte_count(uint32_t x)
{
    return __popc(~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu));
}

__global__ void __launch_bounds__(kEnergyThreads) k_pending_unequal(Lattice lat)
{
    __shared__ unsigned int red[32];
    const unsigned long long t = read_u64(&lat.st->sweep);
    if (t == 0ull || t - 1ull < read_u64(&lat.st->classes_upto)) return;   // same for every block
    const int L = lat.L, per_row = L / 16;
    const int n16 = L * per_row;   // L * L < 2^31
    unsigned int unequal = 0, pairs = 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n16; g += gridDim.x * blockDim.x) {
        const int y = g / per_row, xq = g - y * per_row;
        const int yd = y + 1 == L ? 0 : y + 1;
        const uint4 a = reinterpret_cast<const uint4 *>(lat.spin + (size_t)y * L)[xq];
        const uint4 d = reinterpret_cast<const uint4 *>(lat.spin + (size_t)yd * L)[xq];
        const uint32_t r = (uint8_t)lat.spin[(size_t)y * L + (16 * xq + 16 == L ? 0 : 16 * xq + 16)];
        const uint32_t w[5] = {a.x, a.y, a.z, a.w, r};
        const uint32_t dn[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            unequal += 8u - zero_byte_count(w[k] ^ __funnelshift_r(w[k], w[k + 1], 8)) - zero_byte_count(w[k] ^ dn[k]);
        pairs += 32u;
    }
    unsigned long long *row = ring_row(lat, t - 1);
    block_add<kEnergyThreads>(row + lat.q + 1, unequal, red);
    block_add<kEnergyThreads>(row + lat.q + 0, pairs - unequal, red);
}

__global__ void k_mark_classes(DevState *st)
{
    st->classes_upto = st->sweep;
}

// States outside [0, q) (q <= 127) in the spin array: sixteen per 16-byte
// load where the array is aligned (a byte is out of range if its top bit
// is set or its low seven bits reach q), one at a time otherwise.
__device__ __forceinline__ unsigned int out_of_range4(uint32_t x, uint32_t q4)
{
    return __popc((((x & 0x7F7F7F7Fu) + (0x80808080u - q4)) | x) & 0x80808080u);
}

__global__ void k_count_invalid(const int8_t *spin, long long n, int q, unsigned int *bad)
{
    unsigned int c = 0;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if ((reinterpret_cast<uintptr_t>(spin) & 15) == 0) {
        const uint32_t q4 = (uint32_t)q * 0x01010101u;
        const uint4 *v = reinterpret_cast<const uint4 *>(spin);
        const long long n16 = n / 16;
        for (long long i = tid; i < n16; i += stride) {
            const uint4 w = v[i];
            c += out_of_range4(w.x, q4) + out_of_range4(w.y, q4) + out_of_range4(w.z, q4) + out_of_range4(w.w, q4);
        }
        done = n16 * 16;
    }
    for (long long i = done + tid; i < n; i += stride) c += (spin[i] < 0 || spin[i] >= q);
    c = __reduce_add_sync(FULL, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}

// One kernel of a sweep, with programmatic stream serialization (pdl_begin).
template <typename K>
cudaError_t launch_pdl(K kernel, int blocks, int threads, cudaStream_t s, const Batch &b)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, b);
}

template <bool MEASURE, bool LABELS>
cudaError_t sweep_impl(const Batch &b, int sm_count, const LaunchShape &shape, cudaStream_t s, cudaEvent_t *ev)
{
    int nev = 0;
    auto mark = [&]() {
        if (ev) cudaEventRecord(ev[nev++], s);
    };
    cudaError_t e = cudaSuccess;
    auto put = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    mark();
    // Batches take the whole GPU's grid, whatever their current size, so that
    // a captured sweep stays valid when lattices join or leave.
    auto grid = [&](long long work, int per_sm) {
        const long long cap = (long long)sm_count * per_sm;
        return (int)std::max<long long>(1, b.full_grid ? cap : std::min(work, cap));
    };
    if (b.any_clock) {   // bonds in their own kernel (the clock threshold table), then the labeling
        put(launch_pdl(k_bonds<MEASURE, true>, grid(b.ntasks, shape.bonds), kBlockThreads, s, b));
        mark();
        put(launch_pdl(k_label_tiles<MEASURE, LABELS, false>, grid(b.ntasks, shape.label), kBlockThreads, s, b));
    } else {             // bonds drawn by the labeling kernel
        mark();
        put(launch_pdl(k_label_tiles<MEASURE, LABELS, true>, grid(b.ntasks, std::min(shape.label, kLabelResidentFused)),
                       kBlockThreads, s, b));
    }
    mark();
    const int mblocks = grid((b.nmerge + 255) / 256, shape.merge);
    put(launch_pdl(b.any_stats ? k_merge<true> : k_merge<false>, mblocks, 256, s, b));
    mark();
    const int fblocks = grid(b.ntasks, std::min(shape.flip, b.any_clock ? kFlipResidentClock : kFlipResidentPotts));
    if (b.any_clock)
        put(launch_pdl(b.any_stats ? k_flip_tiles<MEASURE, LABELS, true, true> : k_flip_tiles<MEASURE, LABELS, true, false>,
                       fblocks, kBlockThreads, s, b));
    else
        put(launch_pdl(b.any_stats ? k_flip_tiles<MEASURE, LABELS, false, true>
                                   : k_flip_tiles<MEASURE, LABELS, false, false>,
                       fblocks, kBlockThreads, s, b));
    mark();
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t launch_init(const Lattice &lat, int random, int sm_count, cudaStream_t s)
{
    const long long N4 = (long long)lat.L * lat.L / 4;
    const int blocks = (int)std::min<long long>((N4 + 255) / 256, (long long)sm_count * 8);
    k_init<<<blocks, 256, 0, s>>>(lat, random);
    return cudaGetLastError();
}

cudaError_t launch_pending_classes(const Lattice &lat, int sm_count, cudaStream_t s)
{
    const long long N4 = (long long)lat.L * lat.L / 4;
    const int blocks =
        (int)std::min<long long>((N4 + kEnergyThreads - 1) / kEnergyThreads, (long long)sm_count * 8);
    if (lat.clock)
        k_pending_classes<true><<<blocks, kEnergyThreads, 0, s>>>(lat);
    else if (lat.L % 16 == 0 && (reinterpret_cast<uintptr_t>(lat.spin) & 15) == 0)
        k_pending_unequal<<<blocks, kEnergyThreads, 0, s>>>(lat);
    else
        k_pending_classes<false><<<blocks, kEnergyThreads, 0, s>>>(lat);
    k_mark_classes<<<1, 1, 0, s>>>(lat.st);
    return cudaGetLastError();
}

cudaError_t launch_count_invalid(const Lattice &lat, unsigned int *bad, int sm_count, cudaStream_t s)
{
    const long long n = (long long)lat.L * lat.L;
    const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
    k_count_invalid<<<blocks, 256, 0, s>>>(lat.spin, n, lat.q, bad);
    return cudaGetLastError();
}

cudaError_t launch_bonds(const Batch &b, int sm_count, cudaStream_t s)
{
    const int blocks = std::max(1, std::min(b.ntasks, sm_count * kBondBlocksPerSM));
    b.any_clock ? k_bonds<false, true><<<blocks, kBlockThreads, 0, s>>>(b)
                : k_bonds<false, false><<<blocks, kBlockThreads, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const Batch &b, bool measure, bool labels, int sm_count, const LaunchShape &shape,
                         cudaStream_t s, cudaEvent_t *ev)
{
    if (measure)
        return labels ? sweep_impl<true, true>(b, sm_count, shape, s, ev)
                      : sweep_impl<true, false>(b, sm_count, shape, s, ev);
    return labels ? sweep_impl<false, true>(b, sm_count, shape, s, ev)
                  : sweep_impl<false, false>(b, sm_count, shape, s, ev);
}

}  // namespace swgb
