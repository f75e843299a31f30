// sw_kernels.cu -- the kernels of one Swendsen-Wang sweep on sm_103a.
//
// One sweep (Komura & Okabe, arXiv:1202.0635, Sec. 2 steps (i)-(viii);
// clock model: Sec. 4 embedded clusters) is four launches over the 64 x 64
// tiles of every lattice of a batch (a single lattice is a batch of one).
// A block owns one tile of one lattice at a time ("task"), so per-lattice
// counters reduce per block.
//
//   k_bonds        bonds of every site (Sec. 2 (ii)): equal-neighbour masks
//                  from packed byte compares, Philox draws against the
//                  integer threshold; the masks go to a per-tile buffer.
//                  With measurement on it also counts the bond classes of
//                  the incoming configuration (the previous sweep's result)
//                  and the active bonds.
//   k_label_tiles  tile-local clusters by a row-by-row labeling with a
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
//                  larger root under smaller).
//   k_flip_tiles   finds the cluster root of every open component (the
//                  smallest site index of the cluster, Sec. 2 "proper
//                  label"), which draws the cluster's new state; writes all
//                  spins, counts states and the clusters rooted in the tile;
//                  its last block advances the sweep index of every lattice
//                  of the batch.
#include "sw_internal.h"

namespace swgb {

namespace {

constexpr int TW = kTileW, TH = kTileH, NS = kTileSites, QW = kQuad;
constexpr int kBlockThreads = kTaskWarps * 32;
constexpr int kEnergyThreads = 256;
constexpr unsigned FULL = 0xffffffffu;
constexpr int kInfLabel = 1 << 20;      // "no label" (larger than any tile node)
// Queued unions per tile (a row of a quadrant makes at most 31 requests;
// random bonds make about 260 a tile at T_c).  A tile whose requests exceed
// the queue joins all its internal bonds after the scan instead.
constexpr int kMaxPairs = 2048;
constexpr int kFreshList = 2 * kMaxPairs;  // fresh labels listed per tile (more: settled in place)
// Resident blocks per SM of the flip kernel's variants (its launch bounds);
// its grid never asks for more, so that one wave covers the tiles.
constexpr int kFlipResidentPotts = 10, kFlipResidentClock = 8;
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

// Union of labels a and b, queued in slot idx of the tile's list, or done at
// once when the list is full.


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

// Per-lattice values every block needs once per task.
struct TaskCtx {
    unsigned long long t;   // sweep index
    int count_classes;      // bond classes of configuration t - 1 are counted now
    int m;                  // clock mirror axis
};

template <bool MEASURE>
__device__ __forceinline__ TaskCtx task_context(const Lattice &lat)
{
    TaskCtx c;
    c.t = read_u64(&lat.st->sweep);
    c.count_classes = MEASURE && c.t >= 1ull && c.t - 1ull >= read_u64(&lat.st->classes_upto);
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
// ANY_CLOCK: the batch holds a clock lattice; the clock code is compiled in.
// The bounds keep the clock measuring variant at 80 registers and the
// Potts-only variants at 8 resident blocks per SM, without spills.
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

    for (int task = blockIdx.x; task < b.ntasks; task += gridDim.x) {
        const int rep = find_rep(b.task_off, b.nrep, task);
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
        const int tile = task - __ldg(b.task_off + rep);
        const int L = lat.L, q = lat.q;
        const bool clock = ANY_CLOCK && lat.clock != 0;
        if (!ANY_CLOCK && lat.clock && threadIdx.x == 0) record_error(lat.st, kErrInternal, 0);   // wrong variant
        const unsigned long long t = ctx.t;
        const uint32_t thr = lat.thr;
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
        uint32_t wd[8], dn[8], sr = 0;
        const size_t rowbase = (size_t)y * L + x0;   // meaningful only if rv
        {
            const int yd = (y + 1 == L) ? 0 : y + 1;
            const uint32_t *row = reinterpret_cast<const uint32_t *>(lat.spin + rowbase);
            const uint32_t *drow = reinterpret_cast<const uint32_t *>(lat.spin + (size_t)yd * L + x0);
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
            if (rv) {
                const int xr = (x0 + ncols == L) ? 0 : x0 + ncols;
                sr = (uint8_t)__ldg(lat.spin + (size_t)y * L + xr);
            }
        }
        if (clock) {   // states outside [0, q) read as 0: they index the q x q threshold table
            const uint32_t q4 = (uint32_t)q * 0x01010101u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                wd[k] = clock_valid4(wd[k], q4);
                dn[k] = clock_valid4(dn[k], q4);
            }
            sr = (uint32_t)valid_state((int)sr, q);
        }
        unsigned eqR = 0, eqD = 0, rR = 0, rD = 0;
        if (!clock) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t nxt = (k < 7 && 4 * k + 4 < ncols) ? wd[(k + 1) & 7] : sr;
                eqR |= zero_bytes4(wd[k] ^ __funnelshift_r(wd[k], nxt, 8)) << (4 * k);
                eqD |= zero_bytes4(wd[k] ^ dn[k]) << (4 * k);
            }
        }
        if (rv) {
            const uint32_t pbase = (uint32_t)(rowbase >> 1);
            if (!clock) {
#pragma unroll
                for (int p = 0; p < 16; ++p) {
                    if (2 * p < ncols) {
                        const uint4 u = draw4(lat, pbase + (uint32_t)p, t, kTagBond);
                        rR |= ((unsigned)(u.x < thr) << (2 * p)) | ((unsigned)(u.z < thr) << (2 * p + 1));
                        rD |= ((unsigned)(u.y < thr) << (2 * p)) | ((unsigned)(u.w < thr) << (2 * p + 1));
                    }
                }
            } else {
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
        }
        const unsigned R = rv ? (clock ? (rR & V) : (rR & eqR & V)) : 0u;
        const unsigned D = rv ? (clock ? (rD & V) : (rD & eqD & V)) : 0u;
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

// Every bond inside a tile joined in the shared union-find: the fallback of
// a tile whose union requests overflow the queue.  rowR / rowD hold the
// tile-internal right and down bonds of each row (two 32-bit halves).
__device__ __noinline__ void join_tile_bonds(volatile uint16_t *par, const uint16_t *lbl,
                                             const unsigned int (*rowR)[2], const unsigned int (*rowD)[2], int tw,
                                             int th, DevState *st, int where)
{
    for (int item = threadIdx.x; item < 2 * kTileSites; item += blockDim.x) {
        const int node = item >> 1, down = item & 1;
        const int r = node / kTileW, c = node % kTileW;
        if (r >= th || c >= tw) continue;
        const unsigned bits = down ? rowD[r][c >> 5] : rowR[r][c >> 5];
        if (!((bits >> (c & 31)) & 1u)) continue;
        const int other = down ? node + kTileW : node + 1;
        if (!union_t(par, lbl[node], lbl[other], kTileSites + 1)) record_error(st, kErrUnionCap, where);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// k_label_tiles
//
// Per quadrant (warp), lane r holds row r's bond masks.  Phase B labels the
// quadrant row by row (lane = column); queued unions, the seams between
// quadrants and every label's root are then resolved in shared memory,
// components that reach the tile border are marked open, closed roots draw,
// and each site's code is written.
// ---------------------------------------------------------------------------
template <bool MEASURE, bool LABELS>
__global__ void __launch_bounds__(kBlockThreads, 8) k_label_tiles(Batch b)
{
    __shared__ __align__(16) uint16_t par[NS];     // union-find over labels, node v in slot tile_slot(v)
    __shared__ __align__(16) uint16_t lbl[NS];     // label of every node at its row's scan
    __shared__ __align__(16) uint32_t upairs[kMaxPairs];   // queued unions; then the list of roots
    __shared__ __align__(8) unsigned int rowR[TH][2], rowD[TH][2];
    __shared__ unsigned int openw[NS / 32];
    __shared__ int rmin_all[kTaskWarps][QW];                // per-warp run minima of the scan
    __shared__ int s_nopen, s_npairs, s_wsum[kTaskWarps];
    __shared__ unsigned int s_cross[kCrossWords];
    __shared__ unsigned int red[32];
    __shared__ __align__(16) Lattice lat;
    __shared__ TaskCtx ctx;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qx = warp & 1, qy = warp >> 1;

    unsigned int closed_roots = 0;
    int cur = -1;
    if (threadIdx.x < kCrossWords) s_cross[threadIdx.x] = 0u;   // before the first barrier below
    // Counters of lattice `cur` -> its ring row (whole block).
    auto flush = [&]() {
        if (MEASURE && cur >= 0) block_add<kBlockThreads>(ring_row(lat, ctx.t) + lat.q + lat.nclass + 1, closed_roots, red);
        closed_roots = 0;
        __syncthreads();
    };

    for (int task = blockIdx.x; task < b.ntasks; task += gridDim.x) {
        const int rep = find_rep(b.task_off, b.nrep, task);
        if (rep != cur) {
            flush();
            load_lattice(&lat, b.lat + rep);
            __syncthreads();
            if (threadIdx.x == 0) ctx = task_context<MEASURE>(lat);
            __syncthreads();
            cur = rep;
        }
        const int tile = task - __ldg(b.task_off + rep);
        const int L = lat.L, q = lat.q;
        const bool clock = lat.clock != 0;
        const unsigned long long t = ctx.t;
        const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
        const int X0 = bx * TW, Y0 = by * TH;
        const int tw = min(TW, L - X0), th = min(TH, L - Y0);          // valid extent of the tile
        const int ncols = max(0, min(QW, tw - QW * qx));
        const int nrows = max(0, min(QW, th - QW * qy));
        const bool qa = ncols > 0 && nrows > 0;                        // quadrant has sites (warp-uniform)
        const unsigned V = ncols >= 32 ? FULL : ((1u << ncols) - 1u);
        const bool ext_right = QW * qx + ncols == tw;                   // my right edge is the tile's
        const bool ext_bottom = QW * qy + nrows == th;
        unsigned rc_bits = 0, dc_bits = 0;
        unsigned Rq = 0, Dq = 0;   // lane r: row r's bonds inside the quadrant (right, down)

        for (int i = threadIdx.x; i < NS / 32; i += blockDim.x) openw[i] = 0u;
        if (threadIdx.x == 0) s_nopen = 0;
        if (threadIdx.x == 0) s_npairs = 0;

        // ===== bond masks of my quadrant (written by k_bonds), lane = row ======
        if (qa) {
            const int r = lane;
            const bool rv = r < nrows;
            const uint32_t *tb = lat.bond + (size_t)tile * kBondWords + (QW * qy + r) * 2 + qx;
            const unsigned R = rv ? __ldg(tb) : 0u;
            const unsigned D = rv ? __ldg(tb + kBlockThreads) : 0u;
            rc_bits = __ballot_sync(FULL, rv && ((R >> (ncols - 1)) & 1u));   // bonds leaving the right edge
            dc_bits = __shfl_sync(FULL, D, nrows - 1);                       // bonds leaving the bottom edge
            // Tile-internal bonds as 64-bit rows (two 32-bit halves): the
            // right bond of the tile's last column and the down bonds of its
            // last row cross into the neighbouring tiles.
            const unsigned Rin = R & (ext_right ? (V >> 1) : V);
            const unsigned Din = (ext_bottom && r == nrows - 1) ? 0u : D;
            rowR[QW * qy + r][qx] = rv ? Rin : 0u;
            rowD[QW * qy + r][qx] = rv ? Din : 0u;
            Rq = rv ? (R & (V >> 1)) : 0u;             // both ends in the quadrant
            Dq = (r + 1 < nrows) ? D : 0u;
            if (lane == 0) {
                if (ext_right) atomicOr(&s_cross[qy], rc_bits);
                if (ext_bottom) atomicOr(&s_cross[2 + qx], dc_bits);
            }
        } else {
            rowR[QW * qy + lane][qx] = 0u;
            rowD[QW * qy + lane][qx] = 0u;
        }
        __syncthreads();

        // ===== labels, quadrant by quadrant (warp), lane = column ===============
        // Row by row, every site carries the label of the site above it when
        // the two are bonded.  A run (maximal horizontally bonded segment of
        // the row) takes the label carried by its first such site; a run with
        // none opens a fresh label, its first node.  Other labels carried into
        // the run are queued for a union with the run's.  Labels are tile
        // nodes row * 64 + column, which order like global site indices, so
        // with unions linking larger roots under smaller each component's
        // root is its smallest site.
        if (qa) {
            const int c = lane;
            const bool cv = c < ncols;
            const unsigned bit = 1u << c;
            const unsigned upto = FULL >> (31 - c);   // columns <= c
            const int nb = (QW * qy) * TW + QW * qx;  // node of the quadrant's corner
            int *rmin = rmin_all[warp];
            int pl = 0;                               // label of the site above (valid where Dp has my bit)
            uint32_t lastq = 0xFFFFFFFFu;             // pair this lane queued last
            unsigned Dp = 0u, Rp = 0u;
            for (int row = 0; row < nrows; ++row) {
                const unsigned Rr = __shfl_sync(FULL, Rq, row);
                const unsigned S = ~(Rr << 1);                       // run starts
                const int s0 = 31 - __clz(S & upto);                 // my run's first column
                // The run takes the smallest label a bond from above carries
                // into it (collected at its first column), else a fresh
                // label: its first node.
                rmin[c] = kInfLabel;
                __syncwarp();
                if (Dp & bit) atomicMin(&rmin[s0], pl);
                __syncwarp();
                const int node = nb + row * TW + c;
                const int up = rmin[s0];
                const int mlab = up != kInfLabel ? up : node - (c - s0);
                if (cv) {
                    if (mlab == node) par[node ^ row] = (uint16_t)node;   // tile_slot(node): row < 32
                    lbl[node] = (uint16_t)mlab;
                }
                // A bond from above carrying another label queues a union,
                // unless its left neighbour joins the same two runs or this
                // lane queued the same pair last.
                const unsigned E = Dp & ~((Dp & Rp & Rr) << 1);
                const uint32_t pair = (uint32_t)pl | ((uint32_t)mlab << 16);
                const bool u = (E & bit) && pl != mlab && pair != lastq;
                if (u) {   // a slot of its own: no warp vote on the row's path
                    const int idx = atomicAdd(&s_npairs, 1);
                    if (idx < kMaxPairs) upairs[idx] = pair;
                    lastq = pair;
                }
                __syncwarp();
                pl = mlab;
                Rp = Rr;
                Dp = __shfl_sync(FULL, Dq, row);
            }
        }
        __syncthreads();

        // A queue overflow (block-uniform): join every bond inside the tile.
        if (s_npairs > kMaxPairs) join_tile_bonds(par, lbl, rowR, rowD, tw, th, lat.st, Y0 * L + X0);

        // ===== unions: queued pairs, then the seams between the quadrants =====
        {
            const int np = min(s_npairs, kMaxPairs);
            const int nitems = np + TH + TW;
            for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
                int a, c;
                if (i < np) {
                    const uint32_t pr = upairs[i];
                    a = (int)(pr & 0xFFFFu);
                    c = (int)(pr >> 16);
                } else if (i < np + TH) {   // column 31 - 32 of row y
                    const int y = i - np;
                    if (y >= th || tw <= QW || !((rowR[y][0] >> 31) & 1u)) continue;
                    a = lbl[y * TW + QW - 1];
                    c = lbl[y * TW + QW];
                } else {                     // row 31 - 32 of column x
                    const int x = i - np - TH;
                    if (x >= tw || th <= QW || !((rowD[QW - 1][x >> 5] >> (x & 31)) & 1u)) continue;
                    a = lbl[(QW - 1) * TW + x];
                    c = lbl[QW * TW + x];
                }
                if (!union_t(par, a, c, NS + 1)) record_error(lat.st, kErrUnionCap, Y0 * L + X0);
            }
        }
        __syncthreads();

        // ===== fresh labels into one list; components reaching the border ======
        // Fresh labels are the nodes that are their own label.  Thread t owns
        // nodes 32 t .. 32 t + 31 (row t / 2).
        unsigned fresh = 0;
        {
            const int vrow = threadIdx.x >> 1, vcol = 32 * (threadIdx.x & 1);
            if (vrow < th && vcol < tw) {
                const uint4 *lp = reinterpret_cast<const uint4 *>(lbl) + 4 * threadIdx.x;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint4 w4 = lp[k];
                    const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int j = 8 * k + 2 * h;
                        const uint32_t v = 32u * threadIdx.x + (uint32_t)j;
                        fresh |= ((unsigned)((ws[h] & 0xFFFFu) == v) << j) | ((unsigned)((ws[h] >> 16) == v + 1u) << (j + 1));
                    }
                }
                const int ncol = min(32, tw - vcol);
                fresh &= ncol >= 32 ? FULL : ((1u << ncol) - 1u);
            }
        }
        // Left and top edges always make a component open (their bonds belong
        // to the neighbouring tiles); right and bottom edges through an active
        // crossing bond.  Items: top row, left column, right column, bottom row.
        for (int item = threadIdx.x; item < 4 * TW; item += blockDim.x) {
            const int side = item / TW, k = item % TW;
            int node = -1;
            if (side == 0) {
                if (k < tw) node = k;
            } else if (side == 1) {
                if (k < th) node = k * TW;
            } else if (side == 2) {
                if (k < th && ((s_cross[k >> 5] >> (k & 31)) & 1u)) node = k * TW + tw - 1;
            } else {
                if (k < tw && ((s_cross[2 + (k >> 5)] >> (k & 31)) & 1u)) node = (th - 1) * TW + k;
            }
            if (node < 0) continue;
            const int root = find_t(par, lbl[node], NS + 1);
            if (root < 0) {
                record_error(lat.st, kErrFindCap, Y0 * L + X0);
                continue;
            }
            atomicOr(&openw[root >> 5], 1u << (root & 31));
        }
        const int nmine = __popc(fresh);
        int incl = nmine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += o;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        int nfresh = 0, off = incl - nmine;
#pragma unroll
        for (int w = 0; w < kTaskWarps; ++w) {
            off += w < warp ? s_wsum[w] : 0;
            nfresh += s_wsum[w];
        }
        const bool listed = nfresh <= kFreshList;   // block-uniform
        uint16_t *flist = reinterpret_cast<uint16_t *>(upairs);
        if (listed) {
            unsigned f2 = fresh;
            while (f2) {
                const int bit = __ffs(f2) - 1;
                f2 &= f2 - 1;
                flist[off++] = (uint16_t)(32 * threadIdx.x + bit);
            }
        }
        __syncthreads();

        // ===== settle: roots draw (closed) or take an open slot; every other
        // fresh label is pointed straight at its root.  A root's parent word
        // becomes resolved (it carries the outcome).
        auto settle = [&](int v) {
            int x = v;
            for (int it = 0; it <= NS; ++it) {   // read-only chase: stops at a root, settled or not
                const int p = par_ld(par, x);
                if (p == x || p >= kTileResolved) break;
                x = p;
            }
            if (x != v) {
                par[tile_slot(v)] = (uint16_t)x;
                return;
            }
            const int g = tile_site(L, bx, by, v);
            int w;
            if ((openw[v >> 5] >> (v & 31)) & 1u) {
                const int slot = atomicAdd(&s_nopen, 1);
                if (slot < kOpenSlots) {   // at most 2 * (64 + 64) - 4 open components
                    lat.open_list[(size_t)tile * kOpenSlots + slot] = g;
                    lat.label[g] = g;
                    w = kTileResolved | slot;
                } else {
                    record_error(lat.st, kErrInternal, g);
                    w = kTileResolved | kCodeClosed;
                }
            } else {
                const uint32_t u = draw4(lat, (uint32_t)g, t, kTagState).x;
                w = kTileResolved | kCodeClosed | (clock ? (int)(u >> 31) : mulhi_q(u, q));
                ++closed_roots;
            }
            par[tile_slot(v)] = (uint16_t)w;
        };
        if (listed) {
            for (int i = threadIdx.x; i < nfresh; i += blockDim.x) settle(flist[i]);
        } else {
            unsigned f2 = fresh;
            while (f2) {
                const int bit = __ffs(f2) - 1;
                f2 &= f2 - 1;
                settle(32 * threadIdx.x + bit);
            }
        }
        __syncthreads();
        // Every other fresh label takes its root's resolved word, so that a
        // site's label leads to its outcome in one step.  The roots' words
        // are only read here.  (Debug labels keep the root's index instead.)
        auto adopt = [&](int v) {
            const int p = par_ld(par, v);
            if (p < kTileResolved) par[tile_slot(v)] = (uint16_t)par_ld(par, p);
        };
        if (LABELS) {
        } else if (listed) {
            for (int i = threadIdx.x; i < nfresh; i += blockDim.x) adopt(flist[i]);
        } else {
            while (fresh) {
                const int bit = __ffs(fresh) - 1;
                fresh &= fresh - 1;
                adopt(32 * threadIdx.x + bit);
            }
        }
        __syncthreads();

        // ===== codes: lane = four columns, two rows per warp step ==============
        const int c4 = 4 * (lane & 15);
        if (c4 < tw) {   // tw % 4 == 0: all four columns or none
            for (int row = 2 * warp + (lane >> 4); row < th; row += 2 * kTaskWarps) {
                const uint2 lp = reinterpret_cast<const uint2 *>(lbl)[(row * TW + c4) >> 2];
                int xn[4] = {(int)(lp.x & 0xFFFFu), (int)(lp.x >> 16), (int)(lp.y & 0xFFFFu), (int)(lp.y >> 16)};
                int w[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) w[k] = par_ld(par, xn[k]);
                if (LABELS) {   // a label's word is resolved (a root) or names its root
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (w[k] < kTileResolved) {
                            xn[k] = w[k];
                            w[k] = par_ld(par, w[k]);
                        }
                }
                if (!(w[0] & w[1] & w[2] & w[3] & kTileResolved)) {   // unreachable for a settled tile
                    record_error(lat.st, kErrInternal, Y0 * L + X0);
                    w[0] = w[1] = w[2] = w[3] = kTileResolved | kCodeClosed;
                }
                const size_t site = (size_t)(Y0 + row) * L + X0 + c4;
                const uint2 codes = make_uint2(((uint32_t)w[0] | ((uint32_t)w[1] << 16)) & (kCodeMask * 0x10001u),
                                               ((uint32_t)w[2] | ((uint32_t)w[3] << 16)) & (kCodeMask * 0x10001u));
                if (LABELS) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (w[k] & kCodeClosed) lat.label[site + k] = tile_site(L, bx, by, xn[k]);
                }
                *reinterpret_cast<uint2 *>(lat.code + site) = codes;
            }
        }
        if (threadIdx.x == 0) lat.open_count[tile] = min(s_nopen, kOpenSlots);
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
// k_merge: union of the open roots across every active crossing bond.
// Work items of a lattice: kMergeItems per tile, the 64 rows of its right
// edge, then the 64 columns of its bottom edge; a warp takes 32
// consecutive items (one side of one tile).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int open_root_of(const Lattice &lat, int site, int tile, bool &ok)
{
    const int code = lat.code[site];   // open site: slot of its root in the tile's open list
    if (code & kCodeClosed) {
        ok = false;
        return site;
    }
    return __ldg(lat.open_list + (size_t)tile * kOpenSlots + code);
}

__global__ void k_merge(Batch b)
{
    static_assert(kMergeItems == TH + TW, "merge items: right edge rows, then bottom edge columns");
    long long lo = 0, hi = 0;
    int rep = -1;
    Lattice lat;
    const unsigned lane = threadIdx.x & 31;
    // Every lattice has a multiple of kMergeItems items: a warp never spans
    // two lattices, and its trip count is uniform.
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < b.nmerge;
         base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + lane;
        bool ok = k < b.nmerge;
        int a = 0, c2 = 0;
        if (ok) {
            if (k < lo || k >= hi) {
                rep = find_rep(b.merge_off, b.nrep, k);
                lo = __ldg(b.merge_off + rep);
                hi = __ldg(b.merge_off + rep + 1);
                lat = b.lat[rep];
            }
            const int L = lat.L;
            const int kk = (int)(k - lo);
            const int tile = kk / kMergeItems, e = kk % kMergeItems;
            const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
            const int X0 = bx * TW, Y0 = by * TH;
            const int tw = min(TW, L - X0), th = min(TH, L - Y0);
            const uint32_t *cw = lat.cross + (size_t)tile * kCrossWords;
            int i, j, nt;
            if (e < TH) {   // right edge, row e, into the next tile to the right
                ok = e < th && ((__ldg(cw + (e >> 5)) >> (e & 31)) & 1u);
                const int y = Y0 + e, x = X0 + tw - 1;
                i = y * L + x;
                j = y * L + (x + 1 == L ? 0 : x + 1);
                nt = by * lat.tiles_x + (bx + 1 == lat.tiles_x ? 0 : bx + 1);
            } else {        // bottom edge, column e - 64, into the next tile below
                const int c = e - TH;
                ok = c < tw && ((__ldg(cw + 2 + (c >> 5)) >> (c & 31)) & 1u);
                const int x = X0 + c, y = Y0 + th - 1;
                i = y * L + x;
                j = (y + 1 == L ? 0 : y + 1) * L + x;
                nt = (by + 1 == lat.tiles_y ? 0 : by + 1) * lat.tiles_x + bx;
            }
            if (ok) {
                bool open = true;
                a = open_root_of(lat, i, tile, open);
                c2 = open_root_of(lat, j, nt, open);
                if (!open) {   // a crossing bond always ends at open sites
                    record_error(lat.st, kErrInternal, i);
                    ok = false;
                }
            }
        }
        // Bonds of one warp that join the same two open roots need one union.
        const unsigned vm = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const unsigned long long key = ((unsigned long long)(unsigned)a << 32) | (unsigned)c2;
            const unsigned peers = __match_any_sync(vm, key);
            if ((unsigned)__ffs(peers) - 1u == lane) union_roots(lat.label, a, c2, lat.L * lat.L + 1, lat.st);
        }
    }
}

// Last block of the sweep's final kernel: for every lattice of the batch,
// record that the incoming configuration's classes were counted, zero the
// next counter row and advance the sweep index (every block has read it).
template <bool MEASURE>
__device__ void finish_sweep(const Batch &b)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(b.ticket, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int r = threadIdx.x; r < b.nrep; r += blockDim.x) {
        const Lattice &lt = b.lat[r];
        const unsigned long long t = read_u64(&lt.st->sweep);
        const bool counted = MEASURE && t >= 1ull && t - 1ull >= read_u64(&lt.st->classes_upto);
        unsigned long long *next = ring_row(lt, t + 1);
        for (int c = 0; c < lt.ncounters; ++c) next[c] = 0ull;
        if (counted) lt.st->classes_upto = t;
        __threadfence();
        *reinterpret_cast<volatile unsigned long long *>(&lt.st->sweep) = t + 1;
    }
    if (threadIdx.x == 0) *b.ticket = 0u;
}

// ---------------------------------------------------------------------------
// k_flip_tiles: the cluster roots and new states of the tile's open
// components, all spin writes, state counts.  One block per tile, one warp
// per quadrant.
// ---------------------------------------------------------------------------
template <bool MEASURE, bool LABELS, bool ANY_CLOCK>
__global__ void __launch_bounds__(kBlockThreads, ANY_CLOCK ? kFlipResidentClock : kFlipResidentPotts) k_flip_tiles(Batch b)
{
    // New state (Potts) or reflection flag (clock) of each open slot; then
    // entry kCodeClosed + s = s, so that a Potts code indexes its new state.
    __shared__ __align__(16) unsigned char tab[kOpenSlots + SW_MAX_Q];
    __shared__ int rootg[LABELS ? kOpenSlots : 1];
    __shared__ unsigned int hist_state[SW_MAX_Q + 1];
    __shared__ unsigned int red[32];
    __shared__ __align__(16) Lattice lat;
    __shared__ TaskCtx ctx;

    const int warp = threadIdx.x >> 5, r = threadIdx.x & 31;
    const int qx = warp & 1, qy = warp >> 1;
    // q <= 8: state counts of this lane, 16 bits per state (states 0-3, 4-7);
    // q == 2: sites in cnt_hi, sites in state 1 in cnt_lo.
    unsigned long long cnt_lo = 0, cnt_hi = 0;
    unsigned int open_roots = 0;   // clusters reaching a tile border, counted at their root
    int cur = -1;
    static_assert(kCodeClosed == kOpenSlots && SW_MAX_Q <= 128, "codes index the table");
    for (int k = threadIdx.x; k < SW_MAX_Q; k += blockDim.x) tab[kOpenSlots + k] = (unsigned char)k;
    auto flush = [&]() {
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
    for (int task = blockIdx.x; task < b.ntasks; task += gridDim.x) {
        const int rep = find_rep(b.task_off, b.nrep, task);
        if (rep != cur) {
            flush();
            load_lattice(&lat, b.lat + rep);
            __syncthreads();
            if (threadIdx.x == 0) ctx = task_context<MEASURE>(lat);
            for (int k = threadIdx.x; k < SW_MAX_Q + 1; k += blockDim.x) hist_state[k] = 0u;
            __syncthreads();
            cur = rep;
        }
        const int tile = task - __ldg(b.task_off + rep);
        const int L = lat.L, q = lat.q;
        const bool clock = ANY_CLOCK && lat.clock != 0;   // ANY_CLOCK: the batch holds a clock lattice
        if (!ANY_CLOCK && lat.clock && threadIdx.x == 0) record_error(lat.st, kErrInternal, 0);
        const int m = ctx.m;
        const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
        const int X0 = bx * TW, Y0 = by * TH;
        const int x0 = X0 + QW * qx, y0 = Y0 + QW * qy;                 // my quadrant
        const int ncols = max(0, min(QW, min(TW, L - X0) - QW * qx));
        const int nrows = max(0, min(QW, min(TH, L - Y0) - QW * qy));
        // Lane -> 4 consecutive sites: columns cq..cq+3 of row 4 * step + rsub,
        // so every warp access covers whole 32-byte sectors of 4 rows.
        const int cq = (r & 7) * 4, rsub = r >> 3;
        uint2 cw[8];
        uint32_t sw[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int row = 4 * k + rsub;
            const bool v = row < nrows && cq < ncols;
            const size_t site0 = (size_t)(y0 + row) * L + x0 + cq;
            cw[k] = v ? *reinterpret_cast<const uint2 *>(lat.code + site0) : make_uint2(0u, 0u);
            sw[k] = (clock && v) ? *reinterpret_cast<const uint32_t *>(lat.spin + site0) : 0u;
        }
        // Every open component of the tile belongs to a cluster whose root
        // (its smallest site, after the merge) draws the new state (Potts) or
        // the reflection flag (clock), Sec. 2 (v)-(vii) / Sec. 4, into the
        // tile's table.  A cluster is counted once, by the tile holding its root.
        {
            const size_t k0 = (size_t)tile * kOpenSlots;
            // Slot threadIdx.x is read before the count arrives (the list
            // has kOpenSlots entries; those beyond the count are not used).
            const int r0 = __ldg(lat.open_list + k0 + threadIdx.x);
            const int n = __ldg(lat.open_count + tile);
            const int cap = L * L + 1;
            for (int s = threadIdx.x; s < n; s += blockDim.x) {
                const int r = s == (int)threadIdx.x ? r0 : __ldg(lat.open_list + k0 + s);
                const int root = find_root_halving(lat.label, r, cap, lat.st);
                if (MEASURE && root == r) ++open_roots;
                const uint32_t u = draw4(lat, (uint32_t)root, ctx.t, kTagState).x;
                tab[s] = clock ? (unsigned char)(u >> 31) : (unsigned char)mulhi_q(u, q);
                if (LABELS) rootg[LABELS ? s : 0] = root;
            }
        }
        __syncthreads();

#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int row = 4 * k + rsub;
            if (!(row < nrows && cq < ncols)) continue;
            const size_t site0 = (size_t)(y0 + row) * L + x0 + cq;
            uint32_t word = 0;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const uint32_t code = ((h < 2) ? (cw[k].x >> (16 * h)) : (cw[k].y >> (16 * (h - 2)))) & 0xFFFFu;
                int ns;
                if (clock) {   // closed: the cluster's flag in the code; open: its root's, in the table
                    const int k0 = valid_state((int)((sw[k] >> (8 * h)) & 0xFFu), q);
                    ns = ((code & kCodeClosed) ? (code & 1u) : tab[code & 0xFFu]) ? reflect(k0, m, q) : k0;
                } else {
                    ns = tab[min(code, (uint32_t)(kOpenSlots + SW_MAX_Q - 1))];   // open slot or kCodeClosed | state
                }
                if (MEASURE && q > 2 && q <= 8) {
                    const unsigned long long one = 1ull << (16 * (ns & 3));
                    if (ns < 4) cnt_lo += one;
                    else cnt_hi += one;
                }
                if (LABELS && !(code & kCodeClosed))
                    lat.label[site0 + h] = rootg[LABELS ? code : 0];
                word |= (uint32_t)(ns & 0xFF) << (8 * h);
            }
            if (MEASURE && q == 2) {   // states are 0 or 1
                cnt_lo += (unsigned)__popc(word);
                cnt_hi += 4u;
            }
            *reinterpret_cast<uint32_t *>(lat.spin + site0) = word;
        }
        if (MEASURE && q > 8) {
            // Many states: warp-aggregated shared histogram, site by site.
#pragma unroll 1
            for (int k = 0; k < 8; ++k) {
                const int row = 4 * k + rsub;
                const bool v = row < nrows && cq < ncols;
                const size_t site0 = (size_t)(y0 + row) * L + x0 + cq;
                for (int h = 0; h < 4; ++h) {
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

template <bool MEASURE, bool LABELS>
cudaError_t sweep_impl(const Batch &b, int sm_count, const LaunchShape &shape, cudaStream_t s, cudaEvent_t *ev)
{
    int nev = 0;
    auto mark = [&]() {
        if (ev) cudaEventRecord(ev[nev++], s);
    };
    mark();
    const int bblocks = std::max(1, std::min(b.ntasks, sm_count * shape.bonds));
    if (b.any_clock)
        k_bonds<MEASURE, true><<<bblocks, kBlockThreads, 0, s>>>(b);
    else
        k_bonds<MEASURE, false><<<bblocks, kBlockThreads, 0, s>>>(b);
    mark();
    k_label_tiles<MEASURE, LABELS><<<std::max(1, std::min(b.ntasks, sm_count * shape.label)), kBlockThreads, 0, s>>>(b);
    mark();
    const int mblocks =
        (int)std::max<long long>(1, std::min<long long>((b.nmerge + 255) / 256, (long long)sm_count * shape.merge));
    k_merge<<<mblocks, 256, 0, s>>>(b);
    mark();
    const int fblocks = std::max(
        1, std::min(b.ntasks, sm_count * std::min(shape.flip, b.any_clock ? kFlipResidentClock : kFlipResidentPotts)));
    if (b.any_clock)
        k_flip_tiles<MEASURE, LABELS, true><<<fblocks, kBlockThreads, 0, s>>>(b);
    else
        k_flip_tiles<MEASURE, LABELS, false><<<fblocks, kBlockThreads, 0, s>>>(b);
    mark();
    return cudaGetLastError();
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

cudaError_t launch_bonds(const Batch &b, bool measure, int sm_count, cudaStream_t s)
{
    const int blocks = std::max(1, std::min(b.ntasks, sm_count * kBondBlocksPerSM));
    if (measure)
        b.any_clock ? k_bonds<true, true><<<blocks, kBlockThreads, 0, s>>>(b)
                    : k_bonds<true, false><<<blocks, kBlockThreads, 0, s>>>(b);
    else
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
