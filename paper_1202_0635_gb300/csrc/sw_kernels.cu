// sw_kernels.cu -- the kernels of one Swendsen-Wang sweep on sm_103a.
//
// One sweep (Komura & Okabe, arXiv:1202.0635, Sec. 2 steps (i)-(viii);
// clock model: Sec. 4 embedded clusters) is four launches over the 64 x 64
// tiles of every lattice of a batch (a single lattice is a batch of one).
// A block owns one tile of one lattice at a time ("task"); each of its four
// warps owns a 32 x 32 quadrant, so per-lattice counters reduce per block.
//
//   k_label_tiles  bonds of every site (Sec. 2 (ii)): equal-neighbour masks
//                  from packed byte compares, Philox draws against the
//                  integer threshold.  Tile-local clusters by a scanline over
//                  the rows with a union-find in shared memory.  A component
//                  that does not reach the tile border (or reaches it only
//                  through inactive crossing bonds on the right/bottom
//                  edges) is a finished cluster: its root (smallest site)
//                  draws the new state here (Sec. 2 (v)-(vii) / Sec. 4
//                  reflection) and its sites get a "closed" code.  Open
//                  components enter the global union-find keyed by their
//                  root's site index.  With measurement on it also counts
//                  the bond classes of the incoming configuration (the
//                  previous sweep's result) and the active bonds.
//   k_merge        joins the open roots across every active bond that
//                  crosses a tile edge or the periodic wrap (atomicMin,
//                  larger root under smaller).
//   k_flatten      points every open root straight at its cluster root
//                  (the smallest site index of the cluster, Sec. 2 "proper
//                  label") and counts those roots.
//   k_flip_tiles   draws the new state of every open cluster root, writes
//                  all spins, counts states; its last block advances the
//                  sweep index of every lattice of the batch.
#include "sw_internal.h"

namespace swgb {

namespace {

constexpr int TW = kTileW, TH = kTileH, NS = kTileSites, QW = kQuad;
constexpr int kBlockThreads = kTaskWarps * 32;
constexpr int kEnergyThreads = 256;
constexpr unsigned FULL = 0xffffffffu;
constexpr uint16_t kCodeFlip = 0x4000;   // closed clock cluster: reflected
constexpr int kNone = 0x7FFFFFFF;
constexpr int kRootFlag = 0x40000000;   // parent word of a resolved tile root: flag | code

static_assert(QW == 32, "a warp quadrant is 32 x 32: lane r owns row r as a 32-bit mask");
static_assert(TW == 2 * QW && TH == 2 * QW, "a tile is 2 x 2 quadrants");
static_assert(sizeof(Lattice) % 8 == 0, "lattice descriptors are copied in 8-byte words");

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

__device__ __forceinline__ uint32_t clock_thr(const Lattice &lat, int a, int b, int m)
{
    const int n2 = 2 * lat.q;
    return __ldg(lat.thr_tab + clock_class(valid_state(a, lat.q), m, lat.q) * n2 +
                 clock_class(valid_state(b, lat.q), m, lat.q));
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

// ---------------------------------------------------------------------------
// k_label_tiles
//
// Per quadrant (warp):  phase A (lane r = row r) bond masks of the row;
// phase B (lane c = column c) a scanline over the rows: every site's parent
// word holds its run's label, a run of row y+1 takes the smallest root among
// the runs of row y it touches (atomicMin at the run start's slot) and the
// other touched roots are linked under it.  Tile nodes are numbered
// row * 64 + column, which orders them like global site indices, so roots
// stay the smallest site of their component.  Then the block joins the
// quadrants across their inner borders, finds the roots, marks components
// that reach the tile border, draws the closed ones and writes the codes.
// ---------------------------------------------------------------------------
template <bool MEASURE, bool LABELS>
__global__ void __launch_bounds__(kBlockThreads, 8) k_label_tiles(Batch b)
{
    __shared__ int par[NS];
    __shared__ uint16_t roots_all[kTaskWarps][QW * QW];
    __shared__ unsigned int rowS_all[kTaskWarps][32], rowR_all[kTaskWarps][32], rowD_all[kTaskWarps][32];
    __shared__ unsigned int openw[NS / 32];
    __shared__ int s_nopen;
    __shared__ unsigned int s_cross[kCrossWords];
    __shared__ unsigned int hist_class[SW_MAX_CLOCK_Q / 2 + 2];
    __shared__ unsigned int red[32];
    __shared__ __align__(16) Lattice lat;
    __shared__ TaskCtx ctx;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qx = warp & 1, qy = warp >> 1;
    uint16_t *roots = roots_all[warp];
    unsigned int *rowS = rowS_all[warp], *rowR = rowR_all[warp], *rowD = rowD_all[warp];
    const unsigned lanemask_lt = (1u << lane) - 1u;

    unsigned int active = 0, closed_roots = 0, unequal = 0, pairs = 0;
    int cur = -1;
    // Counters of lattice `cur` -> its ring rows (whole block).
    auto flush = [&]() {
        if (MEASURE && cur >= 0) {
            unsigned long long *row = ring_row(lat, ctx.t);
            block_add<kBlockThreads>(row + lat.q + lat.nclass, active, red);
            block_add<kBlockThreads>(row + lat.q + lat.nclass + 1, closed_roots, red);
            if (ctx.count_classes) {
                unsigned long long *prev = ring_row(lat, ctx.t - 1);
                if (!lat.clock) {
                    block_add<kBlockThreads>(prev + lat.q + 1, unequal, red);
                    block_add<kBlockThreads>(prev + lat.q + 0, pairs - unequal, red);
                } else {
                    __syncthreads();
                    for (int k = threadIdx.x; k < lat.nclass; k += blockDim.x)
                        if (hist_class[k]) atomicAdd(prev + lat.q + k, (unsigned long long)hist_class[k]);
                }
            }
        }
        active = closed_roots = unequal = pairs = 0;
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
                for (int k = threadIdx.x; k < SW_MAX_CLOCK_Q / 2 + 2; k += blockDim.x) hist_class[k] = 0u;
            __syncthreads();
            cur = rep;
        }
        const int tile = task - __ldg(b.task_off + rep);
        const int L = lat.L, q = lat.q;
        const bool clock = lat.clock != 0;
        const unsigned long long t = ctx.t;
        const int m = ctx.m;
        const uint32_t thr = lat.thr;
        const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
        const int X0 = bx * TW, Y0 = by * TH;
        const int tw = min(TW, L - X0), th = min(TH, L - Y0);          // valid extent of the tile
        const int x0 = X0 + QW * qx, y0 = Y0 + QW * qy;                // my quadrant
        const int ncols = max(0, min(QW, tw - QW * qx));
        const int nrows = max(0, min(QW, th - QW * qy));
        const bool qa = ncols > 0 && nrows > 0;                        // quadrant has sites (warp-uniform)
        const unsigned V = ncols >= 32 ? FULL : ((1u << ncols) - 1u);
        const bool ext_right = QW * qx + ncols == tw;                   // my right edge is the tile's
        const bool ext_bottom = QW * qy + nrows == th;
        const int nb = (QW * qy) * TW + QW * qx;                        // node of my quadrant's corner
        unsigned rc_bits = 0, dc_bits = 0;

        for (int i = threadIdx.x; i < NS / 32; i += blockDim.x) openw[i] = 0u;
        if (threadIdx.x == 0) s_nopen = 0;
        if (threadIdx.x < kCrossWords) s_cross[threadIdx.x] = 0u;

        // ===== phase A: lane = row ==========================================
        if (qa) {
            const int r = lane;
            const bool rv = r < nrows;
            const int y = y0 + r;
            const size_t rowbase = (size_t)y * L + x0;   // meaningful only if rv
            uint32_t wd[8], dn[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                wd[k] = (rv && 4 * k < ncols) ? __ldg(reinterpret_cast<const uint32_t *>(lat.spin + rowbase) + k) : 0u;
            uint32_t sr = 0;
            if (rv) {
                const int xr = (x0 + ncols == L) ? 0 : x0 + ncols;
                sr = (uint8_t)__ldg(lat.spin + (size_t)y * L + xr);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) dn[k] = __shfl_down_sync(FULL, wd[k], 1);
            if (rv && r == nrows - 1) {
                const int yd = (y + 1 == L) ? 0 : y + 1;
                const uint32_t *drow = reinterpret_cast<const uint32_t *>(lat.spin + (size_t)yd * L + x0);
#pragma unroll
                for (int k = 0; k < 8; ++k) dn[k] = (4 * k < ncols) ? __ldg(drow + k) : 0u;
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
                            rR |= ((unsigned)(u.x < clock_thr(lat, s0, s1, m)) << c0) |
                                  ((unsigned)(u.z < clock_thr(lat, s1, s2, m)) << c1);
                            rD |= ((unsigned)(u.y < clock_thr(lat, s0, byte_at(dn, c0), m)) << c0) |
                                  ((unsigned)(u.w < clock_thr(lat, s1, byte_at(dn, c1), m)) << c1);
                        }
                    }
                }
            }
            const unsigned R = clock ? (rR & V) : (rR & eqR & V);
            const unsigned D = clock ? (rD & V) : (rD & eqD & V);

            if (MEASURE) {
                if (rv) active += __popc(R) + __popc(D);
                if (ctx.count_classes) {
                    if (!clock) {
                        if (rv) {
                            unequal += __popc(~eqR & V) + __popc(~eqD & V);
                            pairs += 2u * (unsigned)ncols;
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const bool v = rv && c < ncols;
                            const int s0 = byte_at(wd, c);
                            const int s1 = (c + 1 < ncols) ? byte_at(wd, (c + 1) & 31) : (int)sr;
                            add_hist_any(hist_class, clock_bond_class(s0, s1, q), v);
                            add_hist_any(hist_class, clock_bond_class(s0, byte_at(dn, c), q), v);
                        }
                    }
                }
            }
            const unsigned Rint = R & (V >> 1);   // both ends inside the quadrant
            rowS[r] = rv ? (V & ~(Rint << 1)) : 0u;
            rowR[r] = Rint;
            rowD[r] = (r + 1 < nrows) ? D : 0u;
            rc_bits = __ballot_sync(FULL, rv && ((R >> (ncols - 1)) & 1u));   // bonds leaving the right edge
            dc_bits = __shfl_sync(FULL, D, nrows - 1);                       // bonds leaving the bottom edge
            __syncwarp();

            // ===== phase B: lane = column, scanline over the rows ============
            const int c = lane;
            const bool cv = c < ncols;
            const unsigned upto_c = FULL >> (31 - c);   // columns <= c
            unsigned S = rowS[0], Rr = rowR[0];
            par[nb + c] = nb + (cv ? 31 - __clz(S & upto_c) : c);
            for (int row = 0; row + 1 < nrows; ++row) {
                const unsigned Sn = rowS[row + 1], Rn = rowR[row + 1], D2 = rowD[row];
                // A vertical bond is implied by its left neighbour column when
                // both rows are joined across that column pair.
                const unsigned E = D2 & ~((D2 & Rr & Rn) << 1);
                const int base1 = nb + (row + 1) * TW;
                const int s = cv ? 31 - __clz(Sn & upto_c) : c;   // start of my run in row + 1
                par[base1 + c] = kNone;
                int cand = kNone;
                if ((E >> c) & 1u) {
                    cand = find_s(par, nb + row * TW + c, NS + 1);
                    if (cand < 0) {
                        record_error(lat.st, kErrFindCap, Y0 * L + X0);
                        cand = kNone;
                    }
                }
                __syncwarp();
                // Smallest root touched by my run, collected at the run start's slot.
                if (cand != kNone) atomicMin(&par[base1 + s], cand);
                __syncwarp();
                int mm = par[base1 + s];
                if (mm == kNone) mm = base1 + s;
                if (cand != kNone && cand != mm && !union_s(par, cand, mm, NS + 1))
                    record_error(lat.st, kErrUnionCap, Y0 * L + X0);
                __syncwarp();
                par[base1 + c] = mm;
                __syncwarp();
                S = Sn;
                Rr = Rn;
            }
        }
        __syncthreads();

        // ===== join the quadrants across their inner borders ==================
        if (qa) {
            if (!ext_right && lane < nrows && ((rc_bits >> lane) & 1u))
                if (!union_s(par, nb + lane * TW + QW - 1, nb + lane * TW + QW, NS + 1))
                    record_error(lat.st, kErrUnionCap, Y0 * L + X0);
            if (!ext_bottom && lane < ncols && ((dc_bits >> lane) & 1u))
                if (!union_s(par, nb + (QW - 1) * TW + lane, nb + QW * TW + lane, NS + 1))
                    record_error(lat.st, kErrUnionCap, Y0 * L + X0);
        }
        __syncthreads();

        // ===== roots, tile-border components, draws, codes ====================
        const int c = lane;
        const bool cv = c < ncols;
        int nroots = 0;
        if (qa) {
            // A node is a root iff its parent word is itself (unions only ever
            // re-point roots).  Collect my quadrant's roots in row order.
            for (int row = 0; row < nrows; ++row) {
                const int x = nb + row * TW + c;
                const bool isroot = cv && par[x] == x;
                const unsigned bal = __ballot_sync(FULL, isroot);
                if (isroot) roots[nroots + __popc(bal & lanemask_lt)] = (uint16_t)x;
                nroots += __popc(bal);
            }
            // Components reaching the tile border.  Left and top edges always
            // count (their bonds belong to the neighbouring tiles); right and
            // bottom edges count through an active crossing bond.
            int site[4];
            bool want[4];
            want[0] = qy == 0 && cv;                                       // top row
            site[0] = nb + c;
            want[1] = qx == 0 && c < nrows;                                // left column
            site[1] = nb + c * TW;
            want[2] = ext_right && c < nrows && ((rc_bits >> c) & 1u);     // right edge, row c
            site[2] = nb + c * TW + ncols - 1;
            want[3] = ext_bottom && cv && ((dc_bits >> c) & 1u);           // bottom edge, column c
            site[3] = nb + (nrows - 1) * TW + c;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!want[k]) continue;
                const int root = find_s(par, site[k], NS + 1);
                if (root < 0) {
                    record_error(lat.st, kErrFindCap, Y0 * L + X0);
                    continue;
                }
                atomicOr(&openw[root >> 5], 1u << (root & 31));
            }
            if (lane == 0) {
                if (ext_right) atomicOr(&s_cross[qy], rc_bits);
                if (ext_bottom) atomicOr(&s_cross[2 + qx], dc_bits);
            }
        }
        __syncthreads();
        // Closed roots draw now; open roots join the global union-find.  The
        // result is stored in the root's own parent word, flagged.
        for (int j = c; j < nroots; j += 32) {
            const int x = roots[j];
            const int g = tile_site(L, bx, by, x);
            int code;
            if ((openw[x >> 5] >> (x & 31)) & 1u) {
                const int slot = atomicAdd(&s_nopen, 1);
                lat.open_list[(size_t)tile * kOpenSlots + slot] = g;
                lat.label[g] = g;
                code = slot;
            } else {
                const uint32_t u = draw4(lat, (uint32_t)g, t, kTagState).x;
                code = clock ? (kCodeClosed | ((u >> 31) ? kCodeFlip : 0)) : (kCodeClosed | mulhi_q(u, q));
                ++closed_roots;
            }
            par[x] = kRootFlag | code;
        }
        __syncthreads();
        if (qa && cv) {
            for (int row = 0; row < nrows; ++row) {
                const size_t site = (size_t)(y0 + row) * L + x0 + c;
                // Follow parents to the flagged root word.
                int x = nb + row * TW + c;
                int p = par[x];
                for (int it = 0; it < NS && !(p & kRootFlag); ++it) {
                    x = p;
                    p = par[x];
                }
                uint32_t code = (uint32_t)p & 0xFFFFu;
                if (clock && (code & kCodeClosed)) {
                    const int k0 = valid_state(__ldg(lat.spin + site), q);
                    code = kCodeClosed | (uint32_t)((code & kCodeFlip) ? reflect(k0, m, q) : k0);
                }
                if (LABELS && (code & kCodeClosed)) lat.label[site] = tile_site(L, bx, by, x);
                lat.code[site] = (uint16_t)code;
            }
        }
        if (threadIdx.x == 0) lat.open_count[tile] = s_nopen;
        if (threadIdx.x < kCrossWords) lat.cross[(size_t)tile * kCrossWords + threadIdx.x] = s_cross[threadIdx.x];
        __syncthreads();
    }
    flush();
}

// ---------------------------------------------------------------------------
// k_merge: union of the open roots across every active crossing bond.
// Work items of a lattice: L * tiles_x right-edge bonds, then L * tiles_y
// bottom-edge bonds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int open_root_of(const Lattice &lat, int site, bool &ok)
{
    const int sy = site / lat.L, sx = site - sy * lat.L;
    const int code = lat.code[site];   // open site: slot of its root in the tile's open list
    if (code & kCodeClosed) {
        ok = false;
        return site;
    }
    const int tile = (sy / TH) * lat.tiles_x + sx / TW;
    return __ldg(lat.open_list + (size_t)tile * kOpenSlots + code);
}

__global__ void k_merge(Batch b)
{
    long long lo = 0, hi = 0;
    Lattice lat;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < b.nmerge;
         k += (long long)gridDim.x * blockDim.x) {
        if (k < lo || k >= hi) {
            const int rep = find_rep(b.merge_off, b.nrep, k);
            lo = __ldg(b.merge_off + rep);
            hi = __ldg(b.merge_off + rep + 1);
            lat = b.lat[rep];
        }
        const int L = lat.L, ncol = lat.tiles_x;
        const long long kk = k - lo;
        const long long nright = (long long)L * ncol;
        int i, j;
        if (kk < nright) {
            const int y = (int)(kk / ncol), c = (int)(kk % ncol);
            const int tile = (y / TH) * ncol + c;
            if (!((__ldg(lat.cross + (size_t)tile * kCrossWords + ((y % TH) >> 5)) >> (y & 31)) & 1u)) continue;
            const int x = min((c + 1) * TW, L) - 1;
            i = y * L + x;
            j = y * L + (x + 1 == L ? 0 : x + 1);
        } else {
            const long long k2 = kk - nright;
            const int rr = (int)(k2 / L), x = (int)(k2 % L);
            const int tile = rr * ncol + x / TW;
            if (!((__ldg(lat.cross + (size_t)tile * kCrossWords + 2 + ((x % TW) >> 5)) >> (x & 31)) & 1u)) continue;
            const int y = min((rr + 1) * TH, L) - 1;
            i = y * L + x;
            j = (y + 1 == L ? 0 : y + 1) * L + x;
        }
        bool ok = true;
        const int a = open_root_of(lat, i, ok), c2 = open_root_of(lat, j, ok);
        if (!ok) {   // a crossing bond always ends at open sites
            record_error(lat.st, kErrInternal, i);
            continue;
        }
        union_roots(lat.label, a, c2, L * L + 1, lat.st);
    }
}

// ---------------------------------------------------------------------------
// k_flatten: every open root -> its cluster root, which draws the cluster's
// new state (Potts) or reflection flag (clock) into the tile's open-state
// table; the open list then holds the cluster roots.  Counts cluster roots.
// One warp per tile.
// ---------------------------------------------------------------------------
template <bool MEASURE>
__global__ void __launch_bounds__(kBlockThreads) k_flatten(Batch b)
{
    __shared__ unsigned int red[32];
    __shared__ __align__(16) Lattice lat;
    __shared__ unsigned long long s_t;
    unsigned int roots = 0;
    int cur = -1;
    auto flush = [&]() {
        if (MEASURE && cur >= 0) block_add<kBlockThreads>(ring_row(lat, s_t) + lat.q + lat.nclass + 1, roots, red);
        roots = 0;
        __syncthreads();
    };
    for (int task = blockIdx.x; task < b.ntasks; task += gridDim.x) {
        const int rep = find_rep(b.task_off, b.nrep, task);
        if (rep != cur) {
            flush();
            load_lattice(&lat, b.lat + rep);
            __syncthreads();
            if (threadIdx.x == 0) s_t = read_u64(&lat.st->sweep);
            __syncthreads();
            cur = rep;
        }
        const int tile = task - __ldg(b.task_off + rep);
        const int cap = lat.L * lat.L + 1;
        const int n = lat.open_count[tile];
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            const size_t k = (size_t)tile * kOpenSlots + s;
            const int r = lat.open_list[k];
            const int root = find_root_halving(lat.label, r, cap, lat.st);
            if (root != r) lat.label[r] = root;
            else ++roots;
            const uint32_t u = draw4(lat, (uint32_t)root, s_t, kTagState).x;
            lat.open_state[k] = lat.clock ? (uint8_t)(u >> 31) : (uint8_t)mulhi_q(u, lat.q);
            lat.open_list[k] = root;
        }
    }
    flush();
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
// k_flip_tiles: new states of open clusters, all spin writes, state counts.
// One block per tile, one warp per quadrant.
// ---------------------------------------------------------------------------
template <bool MEASURE, bool LABELS>
__global__ void __launch_bounds__(kBlockThreads) k_flip_tiles(Batch b)
{
    __shared__ __align__(16) unsigned char tab[kOpenSlots];
    __shared__ int rootg[LABELS ? kOpenSlots : 1];
    __shared__ unsigned int hist_state[SW_MAX_Q + 1];
    __shared__ __align__(16) Lattice lat;
    __shared__ TaskCtx ctx;

    const int warp = threadIdx.x >> 5, r = threadIdx.x & 31;
    const int qx = warp & 1, qy = warp >> 1;
    // q <= 8: state counts of this lane, 16 bits per state (states 0-3, 4-7).
    unsigned long long cnt_lo = 0, cnt_hi = 0;
    int cur = -1;
    auto flush = [&]() {
        if (MEASURE && cur >= 0) {
            if (lat.q <= 8) {
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
        const bool clock = lat.clock != 0;
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
        // The tile's open-state table (kOpenSlots bytes) into shared memory.
        {
            const size_t k0 = (size_t)tile * kOpenSlots;
            for (int i = threadIdx.x; i < kOpenSlots / 4; i += blockDim.x)
                reinterpret_cast<uint32_t *>(tab)[i] = __ldg(reinterpret_cast<const uint32_t *>(lat.open_state + k0) + i);
            if (LABELS)
                for (int s = threadIdx.x; s < kOpenSlots; s += blockDim.x) rootg[LABELS ? s : 0] = lat.open_list[k0 + s];
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
                if (code & kCodeClosed) {
                    ns = (int)(code & 0x7Fu);
                } else if (clock) {
                    const int k0 = valid_state((int)((sw[k] >> (8 * h)) & 0xFFu), q);
                    ns = tab[code] ? reflect(k0, m, q) : k0;
                } else {
                    ns = tab[code];
                }
                if (MEASURE && q <= 8) {
                    const unsigned long long one = 1ull << (16 * (ns & 3));
                    if (ns < 4) cnt_lo += one;
                    else cnt_hi += one;
                }
                if (LABELS && !(code & kCodeClosed))
                    lat.label[site0 + h] = rootg[LABELS ? code : 0];
                word |= (uint32_t)(ns & 0xFF) << (8 * h);
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
    __shared__ unsigned int red[32];
    const unsigned long long t = read_u64(&lat.st->sweep);
    if (t == 0ull || t - 1ull < read_u64(&lat.st->classes_upto)) return;   // same for every block
    const int L = lat.L, q = lat.q;
    if (CLOCK)
        for (int k = threadIdx.x; k < lat.nclass; k += blockDim.x) hist[k] = 0u;
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
        } else if (v) {
#pragma unroll
            for (int k = 0; k < 8; ++k) unequal += (a[k] != bb[k]);
        }
    }
    unsigned long long *row = ring_row(lat, t - 1);
    if (CLOCK) {
        __syncthreads();
        for (int k = threadIdx.x; k < lat.nclass; k += blockDim.x)
            if (hist[k]) atomicAdd(row + q + k, (unsigned long long)hist[k]);
    } else {
        block_add<kEnergyThreads>(row + q + 1, unequal, red);
        block_add<kEnergyThreads>(row + q + 0, 2u * sites - unequal, red);
    }
}

__global__ void k_mark_classes(DevState *st)
{
    st->classes_upto = st->sweep;
}

// Count states outside [0, q) (spins written by the caller).
__global__ void k_count_invalid(const int8_t *spin, long long n, int q, unsigned int *bad)
{
    unsigned int c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += (spin[i] < 0 || spin[i] >= q);
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
    const int blocks = std::max(1, std::min(b.ntasks, sm_count * shape.label));
    mark();
    k_label_tiles<MEASURE, LABELS><<<blocks, kBlockThreads, 0, s>>>(b);
    mark();
    const int mblocks =
        (int)std::max<long long>(1, std::min<long long>((b.nmerge + 255) / 256, (long long)sm_count * shape.merge));
    k_merge<<<mblocks, 256, 0, s>>>(b);
    mark();
    k_flatten<MEASURE><<<std::max(1, std::min(b.ntasks, sm_count * shape.flatten)), kBlockThreads, 0, s>>>(b);
    mark();
    k_flip_tiles<MEASURE, LABELS><<<std::max(1, std::min(b.ntasks, sm_count * shape.flip)), kBlockThreads, 0, s>>>(b);
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
    else
        k_pending_classes<false><<<blocks, kEnergyThreads, 0, s>>>(lat);
    k_mark_classes<<<1, 1, 0, s>>>(lat.st);
    return cudaGetLastError();
}

cudaError_t launch_count_invalid(const Lattice &lat, unsigned int *bad, int sm_count, cudaStream_t s)
{
    const long long n = (long long)lat.L * lat.L;
    const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)sm_count * 4);
    k_count_invalid<<<blocks, 256, 0, s>>>(lat.spin, n, lat.q, bad);
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
