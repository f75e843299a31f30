// sw_kernels.cu -- the kernels of one Swendsen-Wang sweep on sm_103a.
//
// One sweep (Komura & Okabe, arXiv:1202.0635, Sec. 2 steps (i)-(viii);
// clock model: Sec. 4 embedded clusters) is four launches over 32 x 32
// tiles.  A warp owns a tile; lane r owns row r of it as 32-bit masks.
//
//   k_label_tiles  bonds of every site (Sec. 2 (ii)): equal-neighbour masks
//                  from packed byte compares, Philox draws against the
//                  integer threshold.  Horizontal runs of right bonds come
//                  from bit arithmetic; a union-find over run starts in
//                  shared memory joins runs across the vertical bonds that
//                  are not implied by a neighbouring column.  A component
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
//                  sweep index.
#include "sw_internal.h"

namespace swgb {

namespace {

constexpr int TW = kTileW, TH = kTileH, NS = kTileSites;
constexpr int kWarpsLabel = 4;   // tiles in flight per k_label_tiles block
constexpr int kWarpsFlip = 8;    // tiles in flight per k_flip_tiles block
constexpr int kFlatWarps = 8;    // tiles per k_flatten block
constexpr int kEnergyThreads = 256;
constexpr unsigned FULL = 0xffffffffu;
constexpr uint16_t kCodeFlip = 0x4000;   // closed clock cluster: reflected

static_assert(TW == 32 && TH == 32, "the warp-tile layout assumes 32 x 32 tiles");

__device__ __forceinline__ unsigned long long read_u64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ unsigned long long *ring_row(const Lattice &lat, unsigned long long t)
{
    return lat.ring + (size_t)(t % (unsigned long long)lat.ring_slots) * lat.ncounters;
}

__device__ __forceinline__ int tid2d() { return threadIdx.y * blockDim.x + threadIdx.x; }

// Global site index of tile-local index loc (row * 32 + column) in tile (bx, by).
__device__ __forceinline__ int tile_site(const Lattice &lat, int bx, int by, int loc)
{
    return (by * TH + (loc >> 5)) * lat.L + bx * TW + (loc & 31);
}

// Bit k of the result is set iff byte k of x is zero.
__device__ __forceinline__ unsigned zero_bytes4(unsigned x)
{
    const unsigned t = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);   // 0x80 in zero bytes
    return (((t >> 7) * 0x00204081u) >> 21) & 0xFu;
}

// Start column of the run (of right bonds) that contains column c; S holds
// the run starts of the row and always has bit 0 set.
__device__ __forceinline__ int start_of(unsigned S, int c)
{
    return 31 - __clz(S & (FULL >> (31 - c)));
}

// Shared-memory slot of tile-local node x = row * 32 + column.  Lane r
// works on row r, so storing column c at c ^ r puts the 32 lanes' accesses
// to the same column in 32 different banks.
__device__ __forceinline__ int sw_slot(int x)
{
    return x ^ ((x >> 5) & 31);
}

// Union-find over tile-local nodes stored at swizzled slots; same
// invariants as the global one (parent <= node, roots are minima).
__device__ __forceinline__ int find_t(volatile int *par, int x, int cap)
{
    for (int it = 0; it < cap; ++it) {
        const int p = par[sw_slot(x)];
        if (p == x) return x;
        const int gp = par[sw_slot(p)];
        if (gp == p) return p;
        par[sw_slot(x)] = gp;
        x = gp;
    }
    return -1;
}

__device__ __forceinline__ bool union_t(volatile int *par, int a, int b, int cap)
{
    for (int it = 0; it < cap; ++it) {
        a = find_t(par, a, cap);
        b = find_t(par, b, cap);
        if (a < 0 || b < 0) return false;
        if (a == b) return true;
        const int hi = a > b ? a : b;
        const int lo = a > b ? b : a;
        const int old = atomicMin((int *)&par[sw_slot(hi)], lo);
        if (old == hi) return true;
        a = old;
        b = lo;
    }
    return false;
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
// k_label_tiles: one warp per 32 x 32 tile (grid-stride over tiles).
//
// Phase A (lane r = row r): bond masks of the row.  Phase B (lane c =
// column c): a scanline over the rows.  Every site's parent word holds the
// label of its run; a run of row y+1 takes the smallest root among the
// runs of row y it touches (one redux over the run's lanes), and the other
// touched roots are linked under it.  Roots therefore stay the smallest
// site index of their component.  Phase C: resolve every site's root, mark
// components that reach the tile border, draw the closed ones and write
// the per-site codes.
// ---------------------------------------------------------------------------
template <bool CLOCK, bool MEASURE, bool LABELS>
__global__ void __launch_bounds__(kWarpsLabel * 32) k_label_tiles(Lattice lat)
{
    __shared__ int par_all[kWarpsLabel][NS];
    __shared__ uint16_t rcode_all[kWarpsLabel][NS];
    __shared__ uint16_t roots_all[kWarpsLabel][NS];
    __shared__ unsigned int rowS_all[kWarpsLabel][32], rowR_all[kWarpsLabel][32], rowD_all[kWarpsLabel][32];
    __shared__ unsigned int openw_all[kWarpsLabel][32];
    __shared__ int nopen_all[kWarpsLabel];
    __shared__ unsigned int hist_class[SW_MAX_CLOCK_Q / 2 + 2];
    __shared__ unsigned int red[32];
    __shared__ int s_axis;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *par = par_all[warp];
    uint16_t *rcode = rcode_all[warp];
    uint16_t *roots = roots_all[warp];
    unsigned int *rowS = rowS_all[warp], *rowR = rowR_all[warp], *rowD = rowD_all[warp];
    unsigned int *openw = openw_all[warp];
    const int L = lat.L, q = lat.q;
    const unsigned long long t = read_u64(&lat.st->sweep);
    const bool count_classes = MEASURE && t >= 1ull && t - 1ull >= read_u64(&lat.st->classes_upto);
    if (threadIdx.x == 0 && CLOCK) s_axis = clock_axis(lat, t);
    if (MEASURE && CLOCK)
        for (int k = threadIdx.x; k < lat.nclass; k += blockDim.x) hist_class[k] = 0u;
    __syncthreads();
    const int m = CLOCK ? s_axis : 0;
    const uint32_t thr = lat.thr;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    constexpr int kNone = 0x7FFFFFFF;

    unsigned int active = 0, closed_roots = 0, unequal = 0, pairs = 0;
    const int ntiles = lat.tiles_x * lat.tiles_y;
    for (int tile = blockIdx.x * kWarpsLabel + warp; tile < ntiles; tile += gridDim.x * kWarpsLabel) {
        const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
        const int x0 = bx * TW, y0 = by * TH;
        const int ncols = min(TW, L - x0), nrows = min(TH, L - y0);
        const unsigned V = ncols == 32 ? FULL : ((1u << ncols) - 1u);
        unsigned rc_bits, dc_bits;

        // ===== phase A: lane = row ==========================================
        {
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
            if (!CLOCK) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t nxt = (k < 7 && 4 * k + 4 < ncols) ? wd[(k + 1) & 7] : sr;
                    eqR |= zero_bytes4(wd[k] ^ __funnelshift_r(wd[k], nxt, 8)) << (4 * k);
                    eqD |= zero_bytes4(wd[k] ^ dn[k]) << (4 * k);
                }
            }
            if (rv) {
                const uint32_t pbase = (uint32_t)(rowbase >> 1);
#pragma unroll
                for (int p = 0; p < 16; ++p) {
                    if (2 * p < ncols) {
                        const uint4 u = draw4(lat, pbase + (uint32_t)p, t, kTagBond);
                        uint32_t tr0 = thr, tr1 = thr, td0 = thr, td1 = thr;
                        if (CLOCK) {
                            const int c0 = 2 * p, c1 = 2 * p + 1;
                            const int s0 = byte_at(wd, c0), s1 = byte_at(wd, c1);
                            const int s2 = (c1 + 1 < ncols) ? byte_at(wd, (c1 + 1) & 31) : (int)sr;
                            tr0 = clock_thr(lat, s0, s1, m);
                            tr1 = clock_thr(lat, s1, s2, m);
                            td0 = clock_thr(lat, s0, byte_at(dn, c0), m);
                            td1 = clock_thr(lat, s1, byte_at(dn, c1), m);
                        }
                        rR |= ((unsigned)(u.x < tr0) << (2 * p)) | ((unsigned)(u.z < tr1) << (2 * p + 1));
                        rD |= ((unsigned)(u.y < td0) << (2 * p)) | ((unsigned)(u.w < td1) << (2 * p + 1));
                    }
                }
            }
            const unsigned R = CLOCK ? (rR & V) : (rR & eqR & V);
            const unsigned D = CLOCK ? (rD & V) : (rD & eqD & V);

            if (MEASURE) {
                if (rv) active += __popc(R) + __popc(D);
                if (count_classes) {
                    if (!CLOCK) {
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
            const unsigned Rint = R & (V >> 1);   // both ends inside the tile
            rowS[r] = rv ? (V & ~(Rint << 1)) : 0u;
            rowR[r] = Rint;
            rowD[r] = (r + 1 < nrows) ? D : 0u;
            rc_bits = __ballot_sync(FULL, rv && ((R >> (ncols - 1)) & 1u));   // right-edge crossing bonds
            dc_bits = __shfl_sync(FULL, D, nrows - 1);                       // bottom-edge crossing bonds
            openw[r] = 0u;
            if (r == 0) nopen_all[warp] = 0;
        }
        __syncwarp();

        // ===== phase B: lane = column, scanline over the rows ================
        const int c = lane;
        const bool cv = c < ncols;
        const unsigned above_c = ~(FULL >> (31 - c));   // columns > c
        {
            const unsigned S0 = rowS[0];
            par[c] = cv ? start_of(S0, c) : c;
        }
        for (int row = 0; row + 1 < nrows; ++row) {
            const unsigned Sn = rowS[row + 1], D = rowD[row], R = rowR[row], Rn = rowR[row + 1];
            // A vertical bond is implied by its left neighbour column when both
            // rows are joined across that column pair.
            const unsigned E = D & ~((D & R & Rn) << 1);
            int cand = kNone;
            if ((E >> c) & 1u) {
                cand = find_s(par, row * TW + c, NS + 1);
                if (cand < 0) {
                    record_error(lat.st, kErrFindCap, y0 * L + x0);
                    cand = kNone;
                }
            }
            // Smallest candidate of my run: inclusive min-scan within runs,
            // then read it from the run's last lane.
            const int s = cv ? start_of(Sn, c) : c;
            const unsigned nxt = Sn & above_c;
            const int e = cv ? (nxt ? __ffs(nxt) - 1 : ncols) : c + 1;   // run end (exclusive)
            int v = cand;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int u = __shfl_up_sync(FULL, v, d);
                if (c - d >= s) v = min(v, u);
            }
            int mm = __shfl_sync(FULL, v, e - 1);
            if (mm == kNone) mm = (row + 1) * TW + s;
            if (cand != kNone && cand != mm && !union_s(par, cand, mm, NS + 1))
                record_error(lat.st, kErrUnionCap, y0 * L + x0);
            par[(row + 1) * TW + c] = cv ? mm : (row + 1) * TW + c;
            __syncwarp();
        }

        // ===== phase C: roots, border components, codes ======================
        int nroots = 0;
        for (int row = 0; row < nrows; ++row) {
            const int x = row * TW + c;
            int root = x;
            if (cv) {
                root = find_s(par, x, NS + 1);
                if (root < 0) {
                    record_error(lat.st, kErrFindCap, y0 * L + x0);
                    root = x;
                }
                par[x] = root;
                // Left and top edges: the bonds into the tile belong to the
                // neighbouring tiles, so those sites always count as open.
                const bool open = (row == 0) || (c == 0) || (c == ncols - 1 && ((rc_bits >> row) & 1u)) ||
                                  (row == nrows - 1 && ((dc_bits >> c) & 1u));
                if (open) atomicOr(&openw[root >> 5], 1u << (root & 31));
            }
            const bool isroot = cv && root == x;
            const unsigned b = __ballot_sync(FULL, isroot);
            if (isroot) roots[nroots + __popc(b & lanemask_lt)] = (uint16_t)x;
            nroots += __popc(b);
        }
        __syncwarp();
        for (int j = c; j < nroots; j += 32) {
            const int x = roots[j];
            const int g = tile_site(lat, bx, by, x);
            if ((openw[x >> 5] >> (x & 31)) & 1u) {
                const int slot = atomicAdd(&nopen_all[warp], 1);
                lat.open_list[(size_t)tile * kOpenSlots + slot] = g;
                lat.label[g] = g;
                rcode[x] = (uint16_t)x;
            } else {
                const uint32_t u = draw4(lat, (uint32_t)g, t, kTagState).x;
                rcode[x] = CLOCK ? (uint16_t)(kCodeClosed | ((u >> 31) ? kCodeFlip : 0))
                                 : (uint16_t)(kCodeClosed | mulhi_q(u, q));
                ++closed_roots;
            }
        }
        __syncwarp();
        if (cv) {
            for (int row = 0; row < nrows; ++row) {
                const size_t site = (size_t)(y0 + row) * L + x0 + c;
                const int root = par[row * TW + c];
                uint32_t code = rcode[root];
                if (CLOCK && (code & kCodeClosed)) {
                    const int k0 = valid_state(__ldg(lat.spin + site), q);
                    code = kCodeClosed | (uint32_t)((code & kCodeFlip) ? reflect(k0, m, q) : k0);
                }
                if (LABELS && (code & kCodeClosed)) lat.label[site] = tile_site(lat, bx, by, root);
                lat.code[site] = (uint16_t)code;
            }
        }
        if (lane == 0) {
            lat.open_count[tile] = nopen_all[warp];
            lat.cross[(size_t)tile * kCrossWords + 0] = rc_bits;
            lat.cross[(size_t)tile * kCrossWords + 1] = dc_bits;
        }
        __syncwarp();
    }

    if (MEASURE) {
        unsigned long long *row = ring_row(lat, t);
        block_add<kWarpsLabel * 32>(row + q + lat.nclass, active, red);
        block_add<kWarpsLabel * 32>(row + q + lat.nclass + 1, closed_roots, red);
        if (count_classes) {
            unsigned long long *prev = ring_row(lat, t - 1);
            if (!CLOCK) {
                block_add<kWarpsLabel * 32>(prev + q + 1, unequal, red);
                block_add<kWarpsLabel * 32>(prev + q + 0, pairs - unequal, red);
            } else {
                __syncthreads();
                for (int k = threadIdx.x; k < lat.nclass; k += blockDim.x)
                    if (hist_class[k]) atomicAdd(prev + q + k, (unsigned long long)hist_class[k]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_merge: union of the open roots across every active crossing bond.
// Work items: L * tiles_x right-edge bonds, then L * tiles_y bottom-edge bonds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int open_root_of(const Lattice &lat, int site, bool &ok)
{
    const int sy = site / lat.L, sx = site - sy * lat.L;
    const int code = lat.code[site];   // open site: tile-local index of its root
    if (code & kCodeClosed) {
        ok = false;
        return site;
    }
    return tile_site(lat, sx / TW, sy / TH, code);
}

__global__ void k_merge(Lattice lat)
{
    const int L = lat.L, ncol = lat.tiles_x;
    const long long nright = (long long)L * ncol;
    const long long total = nright + (long long)L * lat.tiles_y;
    const int cap = L * L + 1;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        int i, j;
        if (k < nright) {
            const int y = (int)(k / ncol), c = (int)(k % ncol);
            const int tile = (y / TH) * ncol + c;
            if (!((__ldg(lat.cross + (size_t)tile * kCrossWords) >> (y % TH)) & 1u)) continue;
            const int x = min((c + 1) * TW, L) - 1;
            i = y * L + x;
            j = y * L + (x + 1 == L ? 0 : x + 1);
        } else {
            const long long k2 = k - nright;
            const int rr = (int)(k2 / L), x = (int)(k2 % L);
            const int tile = rr * ncol + x / TW;
            if (!((__ldg(lat.cross + (size_t)tile * kCrossWords + 1) >> (x % TW)) & 1u)) continue;
            const int y = min((rr + 1) * TH, L) - 1;
            i = y * L + x;
            j = (y + 1 == L ? 0 : y + 1) * L + x;
        }
        bool ok = true;
        const int a = open_root_of(lat, i, ok), b = open_root_of(lat, j, ok);
        if (!ok) {   // a crossing bond always ends at open sites
            record_error(lat.st, kErrInternal, i);
            continue;
        }
        union_roots(lat.label, a, b, cap, lat.st);
    }
}

// ---------------------------------------------------------------------------
// k_flatten: every open root -> its cluster root; count cluster roots.
// One warp per tile.
// ---------------------------------------------------------------------------
template <bool MEASURE>
__global__ void __launch_bounds__(32 * kFlatWarps) k_flatten(Lattice lat)
{
    __shared__ unsigned int red[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kFlatWarps + warp;
    const int ntiles = lat.tiles_x * lat.tiles_y;
    const int cap = lat.L * lat.L + 1;
    unsigned int roots = 0;
    if (tile < ntiles) {
        const int n = lat.open_count[tile];
        for (int s = lane; s < n; s += 32) {
            const int r = lat.open_list[(size_t)tile * kOpenSlots + s];
            const int root = find_root_halving(lat.label, r, cap, lat.st);
            if (root != r) lat.label[r] = root;
            else ++roots;
        }
    }
    if (MEASURE) {
        const unsigned long long t = read_u64(&lat.st->sweep);
        block_add<32 * kFlatWarps>(ring_row(lat, t) + lat.q + lat.nclass + 1, roots, red);
    }
}

// Last block of the sweep's final kernel: record that the incoming
// configuration's classes were counted, zero the next counter row and
// advance the sweep index (every block has read it by then).
__device__ void finish_sweep(const Lattice &lat, unsigned long long t, bool counted_classes)
{
    __shared__ int s_last;
    __syncthreads();
    const int tid = tid2d();
    if (tid == 0) {
        __threadfence();
        const unsigned int nblk = gridDim.x * gridDim.y;
        const unsigned int prev = atomicAdd(&lat.st->ticket, 1u);
        s_last = (prev == nblk - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        unsigned long long *next = ring_row(lat, t + 1);
        for (int c = tid; c < lat.ncounters; c += blockDim.x * blockDim.y) next[c] = 0ull;
        if (tid == 0) {
            lat.st->ticket = 0u;
            if (counted_classes) lat.st->classes_upto = t;
            *reinterpret_cast<volatile unsigned long long *>(&lat.st->sweep) = t + 1;
        }
    }
}

// ---------------------------------------------------------------------------
// k_flip_tiles: new states of open clusters, all spin writes, state counts.
// One warp per tile (grid-stride); lane r writes row r.
// ---------------------------------------------------------------------------
template <bool CLOCK, bool MEASURE, bool LABELS>
__global__ void __launch_bounds__(kWarpsFlip * 32) k_flip_tiles(Lattice lat)
{
    __shared__ unsigned char tab_all[kWarpsFlip][NS];
    __shared__ int rootg_all[LABELS ? kWarpsFlip : 1][LABELS ? NS : 1];
    __shared__ unsigned int hist_state[SW_MAX_Q + 1];
    __shared__ int s_axis;

    const int warp = threadIdx.x >> 5, r = threadIdx.x & 31;
    unsigned char *tab = tab_all[warp];
    const int L = lat.L, q = lat.q;
    const unsigned long long t = read_u64(&lat.st->sweep);
    const bool counted_classes = MEASURE && t >= 1ull && t - 1ull >= read_u64(&lat.st->classes_upto);
    const int cap = L * L + 1;
    if (threadIdx.x == 0 && CLOCK) s_axis = clock_axis(lat, t);
    if (MEASURE)
        for (int k = threadIdx.x; k < q; k += blockDim.x) hist_state[k] = 0u;
    __syncthreads();
    const int m = CLOCK ? s_axis : 0;

    // q <= 8: state counts of this lane, 16 bits per state (states 0-3, 4-7).
    unsigned long long cnt_lo = 0, cnt_hi = 0;
    const int ntiles = lat.tiles_x * lat.tiles_y;
    for (int tile = blockIdx.x * kWarpsFlip + warp; tile < ntiles; tile += gridDim.x * kWarpsFlip) {
        const int by = tile / lat.tiles_x, bx = tile - by * lat.tiles_x;
        const int x0 = bx * TW, y0 = by * TH;
        const int ncols = min(TW, L - x0), nrows = min(TH, L - y0);
        const bool rv = r < nrows;
        const size_t rowbase = (size_t)(y0 + r) * L + x0;

        // Row codes (and old states for the clock reflection) first, so the
        // loads overlap the root lookups below.
        uint2 cw[8];
        uint32_t sw[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool v = rv && 4 * k < ncols;
            cw[k] = v ? reinterpret_cast<const uint2 *>(lat.code + rowbase)[k] : make_uint2(0u, 0u);
            sw[k] = (CLOCK && v) ? reinterpret_cast<const uint32_t *>(lat.spin + rowbase)[k] : 0u;
        }
        const int n = lat.open_count[tile];
        for (int s = r; s < n; s += 32) {
            const int rg = lat.open_list[(size_t)tile * kOpenSlots + s];
            const int g = find_root_ro(lat.label, rg, cap, lat.st);
            const uint32_t u = draw4(lat, (uint32_t)g, t, kTagState).x;
            const int ry = rg / L, rx = rg - ry * L;
            const int loc = (ry - y0) * TW + (rx - x0);
            tab[loc] = CLOCK ? (unsigned char)(u >> 31) : (unsigned char)mulhi_q(u, q);
            if (LABELS) rootg_all[LABELS ? warp : 0][LABELS ? loc : 0] = g;
        }
        __syncwarp();

        if (rv) {
            uint32_t *dst = reinterpret_cast<uint32_t *>(lat.spin + rowbase);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t word = 0;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const uint32_t code = ((h < 2) ? (cw[k].x >> (16 * h)) : (cw[k].y >> (16 * (h - 2)))) & 0xFFFFu;
                    int ns;
                    if (code & kCodeClosed) {
                        ns = (int)(code & 0x7Fu);
                    } else if (CLOCK) {
                        const int k0 = valid_state((int)((sw[k] >> (8 * h)) & 0xFFu), q);
                        ns = tab[code] ? reflect(k0, m, q) : k0;
                    } else {
                        ns = tab[code];
                    }
                    const bool v = 4 * k + h < ncols;
                    if (MEASURE && q <= 8 && v) {
                        const unsigned long long one = 1ull << (16 * (ns & 3));
                        if (ns < 4) cnt_lo += one;
                        else cnt_hi += one;
                    }
                    if (LABELS && v && !(code & kCodeClosed))
                        lat.label[rowbase + 4 * k + h] = rootg_all[LABELS ? warp : 0][LABELS ? code : 0];
                    word |= (uint32_t)(ns & 0xFF) << (8 * h);
                }
                if (4 * k < ncols) dst[k] = word;
            }
        }
        if (MEASURE && q > 8) {
            // Many states: warp-aggregated shared histogram, site by site.
#pragma unroll 1
            for (int c = 0; c < 32; ++c) {
                const bool v = rv && c < ncols;
                int ns = 0;
                if (v) ns = (int)(lat.spin[rowbase + c]);
                add_hist_any(hist_state, ns, v && ns >= 0 && ns < q);
            }
        }
        __syncwarp();
    }
    if (MEASURE) {
        if (q <= 8) {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const unsigned long long w = s < 4 ? cnt_lo : cnt_hi;
                const unsigned int v = __reduce_add_sync(FULL, (unsigned int)((w >> (16 * (s & 3))) & 0xFFFFull));
                if (r == 0 && s < q && v) atomicAdd(&hist_state[s], v);
            }
        }
        __syncthreads();
        unsigned long long *row = ring_row(lat, t);
        for (int k = threadIdx.x; k < q; k += blockDim.x)
            if (hist_state[k]) atomicAdd(row + k, (unsigned long long)hist_state[k]);
    }
    finish_sweep(lat, t, counted_classes);
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
        int a[8] = {0, 0, 0, 0, 0, 0, 0, 0}, b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (v) {
            const int i0 = (int)(4 * g);
            const int y = i0 / L, x = i0 - y * L;
            const char4 s = reinterpret_cast<const char4 *>(lat.spin)[g];
            const int yd = (y + 1 == L) ? 0 : y + 1;
            const char4 d = *reinterpret_cast<const char4 *>(lat.spin + (size_t)yd * L + x);
            const int sr = lat.spin[(size_t)y * L + ((x + 4 == L) ? 0 : x + 4)];
            const int aa[8] = {s.x, s.y, s.z, s.w, s.x, s.y, s.z, s.w};
            const int bb[8] = {s.y, s.z, s.w, sr, d.x, d.y, d.z, d.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                a[k] = aa[k];
                b[k] = bb[k];
            }
            sites += 4;
        }
        if (CLOCK) {
#pragma unroll
            for (int k = 0; k < 8; ++k) add_hist_any(hist, clock_bond_class(a[k], b[k], q), v);
        } else if (v) {
#pragma unroll
            for (int k = 0; k < 8; ++k) unequal += (a[k] != b[k]);
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

template <bool CLOCK, bool MEASURE, bool LABELS>
cudaError_t sweep_impl(const Lattice &lat, int sm_count, cudaStream_t s, cudaEvent_t *ev)
{
    int nev = 0;
    auto mark = [&]() {
        if (ev) cudaEventRecord(ev[nev++], s);
    };
    const int ntiles = lat.tiles_x * lat.tiles_y;
    mark();
    const int lblocks = std::min((ntiles + kWarpsLabel - 1) / kWarpsLabel, sm_count * 8);
    k_label_tiles<CLOCK, MEASURE, LABELS><<<lblocks, kWarpsLabel * 32, 0, s>>>(lat);
    mark();
    const long long nmerge = (long long)lat.L * (lat.tiles_x + lat.tiles_y);
    const int mblocks = (int)std::min<long long>((nmerge + 255) / 256, (long long)sm_count * 16);
    k_merge<<<mblocks, 256, 0, s>>>(lat);
    mark();
    k_flatten<MEASURE><<<(ntiles + kFlatWarps - 1) / kFlatWarps, 32 * kFlatWarps, 0, s>>>(lat);
    mark();
    const int fblocks = std::min((ntiles + kWarpsFlip - 1) / kWarpsFlip, sm_count * 8);
    k_flip_tiles<CLOCK, MEASURE, LABELS><<<fblocks, kWarpsFlip * 32, 0, s>>>(lat);
    mark();
    return cudaGetLastError();
}

template <bool CLOCK>
cudaError_t sweep_dispatch(const Lattice &lat, bool measure, bool labels, int sm_count, cudaStream_t s,
                           cudaEvent_t *ev)
{
    if (measure)
        return labels ? sweep_impl<CLOCK, true, true>(lat, sm_count, s, ev)
                      : sweep_impl<CLOCK, true, false>(lat, sm_count, s, ev);
    return labels ? sweep_impl<CLOCK, false, true>(lat, sm_count, s, ev)
                  : sweep_impl<CLOCK, false, false>(lat, sm_count, s, ev);
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

cudaError_t launch_sweep(const Lattice &lat, bool measure, bool labels, int sm_count, cudaStream_t s,
                         cudaEvent_t *ev)
{
    if (lat.clock) return sweep_dispatch<true>(lat, measure, labels, sm_count, s, ev);
    return sweep_dispatch<false>(lat, measure, labels, sm_count, s, ev);
}

}  // namespace swgb
