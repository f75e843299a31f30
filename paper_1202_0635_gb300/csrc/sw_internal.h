// sw_internal.h -- declarations shared by the host engine and the kernels.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sw.h"
#include "sw_device.cuh"

namespace swgb {

// Tile of the labeling stage: 32 x 32 sites, one warp per tile, lane r
// owning row r of the tile as 32-bit masks.
constexpr int kTileW = 32;
constexpr int kTileH = 32;
constexpr int kTileSites = kTileW * kTileH;
// A component that reaches a tile border ("open") owns a border site, so a
// tile has at most 2 * (W + H) - 4 = 124 open components.
constexpr int kOpenSlots = 128;
// Crossing-bond words per tile: [0] bit r = right-edge bond of row r,
// [1] bit c = bottom-edge bond of column c.
constexpr int kCrossWords = 2;
// Per-site code: closed component -> kCodeClosed | new state; open
// component -> slot of its root in the tile's open list.
constexpr uint16_t kCodeClosed = 0x8000;

// Counter rows kept on the device; the host drains them before the ring
// would wrap onto undrained rows.
constexpr int kRingSlots = 1024;

cudaError_t launch_init(const Lattice &lat, int random, int sm_count, cudaStream_t s);
// Bond classes of the current configuration, if the last sweep's are still
// missing (measurement on, before the host reads the counters).
cudaError_t launch_pending_classes(const Lattice &lat, int sm_count, cudaStream_t s);
// Number of spins outside [0, q) is added to *bad (device word).
cudaError_t launch_count_invalid(const Lattice &lat, unsigned int *bad, int sm_count, cudaStream_t s);
// ev (optional): events recorded before the first and after every kernel of
// the sweep (kMaxStages + 1 entries).
constexpr int kMaxStages = 4;
cudaError_t launch_sweep(const Batch &b, bool measure, bool labels, int sm_count, cudaStream_t s,
                         cudaEvent_t *ev = nullptr);

}  // namespace swgb
