// sw_internal.h -- declarations shared by the host engine and the kernels.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sw.h"
#include "sw_device.cuh"

namespace swgb {

// Tiles: a block labels one 64 x 64 tile (the unit of global work) with
// four warps, each owning a 32 x 32 quadrant whose lane r holds row r as
// 32-bit masks.  Quadrant borders inside the tile are merged in shared
// memory; only components reaching the tile border go global.
constexpr int kTileW = 64;
constexpr int kTileH = 64;
constexpr int kQuad = 32;
constexpr int kTileSites = kTileW * kTileH;
static_assert(kTaskWarps == (kTileW / kQuad) * (kTileH / kQuad), "one warp per quadrant");
// A component that reaches a tile border ("open") owns a border site, so a
// tile has at most 2 * (W + H) - 4 = 252 open components.
constexpr int kOpenSlots = 256;
// Edge bytes per tile: the open slot of the component of each right-edge
// site (rows 0..63), then of each left-edge site.  The merge stage reads
// them for the crossing bonds; the bottom and top edges are read from the
// codes, which are contiguous there.
constexpr int kEdgeBytes = 128;
// Crossing-bond words per tile: [0], [1] bit r = right-edge bond of row
// 32 * w + r; [2], [3] bit c = bottom-edge bond of column 32 * w + c.
constexpr int kCrossWords = 4;
// Merge items per tile: the 64 rows of its right edge, then the 64
// columns of its bottom edge.
constexpr int kMergeItems = 128;
// Per-site code: closed component -> kCodeClosed | new state (Potts, below
// 128) or kCodeClosed | reflection flag (clock); open component -> slot of
// its root in the tile's open list (below 256).  A Potts code thus indexes
// one table: the open slots' new states, then entry kCodeClosed + s = s.
constexpr uint16_t kCodeClosed = 0x100;

// Bond-mask words per tile (right and down bonds of 64 rows, 2 words a row).
constexpr int kBondWords = 2 * kTileH * (kTileW / 32);
// Resident blocks per SM requested for the bond kernel outside a sweep.
constexpr int kBondBlocksPerSM = 16;

// Counter rows kept on the device; the host drains them before the ring
// would wrap onto undrained rows.
constexpr int kRingSlots = 1024;

cudaError_t launch_init(const Lattice &lat, int random, int sm_count, cudaStream_t s);
// Bond classes of the current configuration, if the last sweep's are still
// missing (measurement on, before the host reads the counters).
cudaError_t launch_pending_classes(const Lattice &lat, int sm_count, cudaStream_t s);
// Number of spins outside [0, q) is added to *bad (device word).
cudaError_t launch_count_invalid(const Lattice &lat, unsigned int *bad, int sm_count, cudaStream_t s);
// Launch shape of a sweep: resident blocks per SM requested for the
// labeling, merge, flip and bond kernels (the grids never exceed the work).
// Any shape gives the same results; only the speed differs.
struct LaunchShape {
    int label = 11, merge = 12, flip = 10, bonds = kBondBlocksPerSM;
};
// ev (optional): events recorded before the first and after every kernel of
// the sweep (kMaxStages + 1 entries): bonds, labeling, merge, flip.
constexpr int kMaxStages = 4;
cudaError_t launch_sweep(const Batch &b, bool measure, bool labels, int sm_count, const LaunchShape &shape,
                         cudaStream_t s, cudaEvent_t *ev = nullptr);
// The bond kernel alone, update only (the bonds of the comparator labelings).
cudaError_t launch_bonds(const Batch &b, int sm_count, cudaStream_t s);

// Comparator labelings of the paper's GPU design (Sec. 3), whole-lattice
// iterations until no label changes.
enum : int { kLabelTiled = 0, kLabelHawick = 1, kLabelKalentev = 2 };
// One update-only sweep of lattice `lat` (b: its batch-of-one view) with an
// iterated label-equivalence labeling: bonds, scan/analysis(/relabel)
// passes until the device flag stays clear (the host reads it after every
// pass), new spins from every cluster root's draw, sweep index advanced.
// R: int32[L*L] reference array (Hawick only).  *passes = scan passes, or
// -1 if max_passes ran out (then no spin is updated).
cudaError_t equivalence_sweep(const Batch &b, const Lattice &lat, int method, int sm_count, cudaStream_t s,
                              int32_t *R, unsigned int *d_flag, unsigned int *h_flag, int max_passes, int *passes);

}  // namespace swgb
