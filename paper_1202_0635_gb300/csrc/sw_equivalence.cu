// sw_equivalence.cu -- the cluster labelings of the paper's own GPU design
// (Komura & Okabe, arXiv:1202.0635, Sec. 3), kept as comparators for the
// tiled labeling of sw_kernels.cu.
//
// Both iterate whole-lattice passes until no label changes, the host reading
// a device flag after each pass:
//   Hawick et al. (label equivalence): a scan lowers, with atomicMin, the
//     reference R[label] of every site to the smallest label among its bonded
//     neighbours; an analysis pass lets every site that is its own label
//     follow the R chain to its end; a relabel pass sets label = R[label].
//   Kalentev et al. (the refinement): a single array; the scan writes the
//     smallest neighbouring label into label[label] without atomics, and the
//     analysis pass follows label chains wherever label[label] != label.
// Labels start as the site index and only take values from the same
// cluster, so both end at the smallest site index of every cluster -- the
// canonical label of the tiled path.  The new spins then come from the same
// per-root draw (Sec. 2 steps (v)-(vii); clock: Sec. 4 reflection), so a
// sweep is bit-identical to the tiled one.  Bonds come from k_bonds.
#include "sw_internal.h"

namespace swgb {

namespace {

constexpr int kEqThreads = 256;

// Bond bit of site (y, x): plane 0 = right bond, plane 1 = down bond.
__device__ __forceinline__ bool bond_at(const Lattice &lat, int y, int x, int plane)
{
    const int tile = (y >> 6) * lat.tiles_x + (x >> 6);
    const uint32_t w = __ldg(lat.bond + (size_t)tile * kBondWords + plane * (kBondWords / 2) + (y & 63) * 2 +
                             ((x & 63) >> 5));
    return (w >> (x & 31)) & 1u;
}

__global__ void k_eq_init(Lattice lat, int32_t *R)
{
    const long long N = (long long)lat.L * lat.L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        lat.label[i] = (int32_t)i;
        if (R) R[i] = (int32_t)i;
    }
}

// Smallest label among site i and its bonded neighbours (periodic).
__device__ __forceinline__ int neighbour_min(const Lattice &lat, int y, int x, int l)
{
    const int L = lat.L;
    const int xr = x + 1 == L ? 0 : x + 1, xl = x == 0 ? L - 1 : x - 1;
    const int yd = y + 1 == L ? 0 : y + 1, yu = y == 0 ? L - 1 : y - 1;
    const volatile int32_t *lab = lat.label;
    int m = l;
    if (bond_at(lat, y, x, 0)) m = min(m, lab[(size_t)y * L + xr]);
    if (bond_at(lat, y, x, 1)) m = min(m, lab[(size_t)yd * L + x]);
    if (bond_at(lat, y, xl, 0)) m = min(m, lab[(size_t)y * L + xl]);
    if (bond_at(lat, yu, x, 1)) m = min(m, lab[(size_t)yu * L + x]);
    return m;
}

template <bool HAWICK>
__global__ void k_eq_scan(Lattice lat, int32_t *R, unsigned int *flag)
{
    const int L = lat.L;
    const long long N = (long long)L * L;
    bool changed = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / L), x = (int)(i - (long long)y * L);
        const int l = reinterpret_cast<const volatile int32_t *>(lat.label)[i];
        const int m = neighbour_min(lat, y, x, l);
        if (m < l) {
            if (HAWICK) atomicMin(R + l, m);
            else lat.label[l] = m;   // no atomic: a lost update is repaired by a later pass
            changed = true;
        }
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) *flag = 1u;
}

// Follow a chain p -> arr[p] to its end (bounded: chains strictly decrease).
__device__ __forceinline__ int chain_end(const volatile int32_t *arr, int p, int cap, DevState *st)
{
    for (int it = 0; it < cap; ++it) {
        const int q = arr[p];
        if (q == p) return p;
        p = q;
    }
    record_error(st, kErrFindCap, p);
    return p;
}

template <bool HAWICK>
__global__ void k_eq_analysis(Lattice lat, int32_t *R)
{
    const long long N = (long long)lat.L * lat.L;
    const int cap = (int)min(N, (long long)0x7FFFFFFF);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (HAWICK) {
            if (lat.label[i] == (int32_t)i) R[i] = chain_end(R, R[i], cap, lat.st);
        } else {
            const int l = lat.label[i];
            if (reinterpret_cast<const volatile int32_t *>(lat.label)[l] != l)
                lat.label[i] = chain_end(lat.label, l, cap, lat.st);
        }
    }
}

__global__ void k_eq_relabel(Lattice lat, const int32_t *R)
{
    const long long N = (long long)lat.L * lat.L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        lat.label[i] = R[lat.label[i]];
}

// New spins: every site takes its cluster root's draw (cluster_draw).  The
// clock reflection uses the sweep's mirror axis.
template <bool CLOCK>
__global__ void k_eq_flip(Lattice lat)
{
    const long long N = (long long)lat.L * lat.L;
    const unsigned long long t = *reinterpret_cast<const volatile unsigned long long *>(&lat.st->sweep);
    const int q = lat.q;
    const int m = CLOCK ? clock_axis(lat, t) : 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int d = cluster_draw(lat, (uint32_t)lat.label[i], t);
        if (CLOCK) {
            const int k = valid_state(lat.spin[i], q);
            int r = m - k;
            if (r < 0) r += q;
            lat.spin[i] = (int8_t)(d ? r : k);
        } else {
            lat.spin[i] = (int8_t)d;
        }
    }
}

// Zero the next counter row (as the tiled sweep does) and advance the index.
__global__ void k_eq_finish(Lattice lat)
{
    const unsigned long long t = lat.st->sweep;
    unsigned long long *next = lat.ring + (size_t)((t + 1) % (unsigned long long)lat.ring_slots) * lat.ncounters;
    for (int c = threadIdx.x; c < lat.ncounters; c += blockDim.x) next[c] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) lat.st->sweep = t + 1;
}

}  // namespace

cudaError_t equivalence_sweep(const Batch &b, const Lattice &lat, int method, int sm_count, cudaStream_t s,
                              int32_t *R, unsigned int *d_flag, unsigned int *h_flag, int max_passes, int *passes)
{
    const bool hawick = method == kLabelHawick;
    const long long N = (long long)lat.L * lat.L;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((N + kEqThreads - 1) / kEqThreads,
                                                                       (long long)sm_count * 8));
    cudaError_t e = launch_bonds(b, sm_count, s);
    if (e != cudaSuccess) return e;
    k_eq_init<<<blocks, kEqThreads, 0, s>>>(lat, hawick ? R : nullptr);
    int n = 0;
    for (;;) {
        if ((e = cudaMemsetAsync(d_flag, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
        if (hawick) {
            k_eq_scan<true><<<blocks, kEqThreads, 0, s>>>(lat, R, d_flag);
            k_eq_analysis<true><<<blocks, kEqThreads, 0, s>>>(lat, R);
            k_eq_relabel<<<blocks, kEqThreads, 0, s>>>(lat, R);
        } else {
            k_eq_scan<false><<<blocks, kEqThreads, 0, s>>>(lat, nullptr, d_flag);
            k_eq_analysis<false><<<blocks, kEqThreads, 0, s>>>(lat, nullptr);
        }
        if ((e = cudaMemcpyAsync(h_flag, d_flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        ++n;
        if (*h_flag == 0u) break;
        if (n >= max_passes) {   // not converged: no spin update, the caller reports it
            *passes = -1;
            return cudaSuccess;
        }
    }
    *passes = n;
    if (lat.clock)
        k_eq_flip<true><<<blocks, kEqThreads, 0, s>>>(lat);
    else
        k_eq_flip<false><<<blocks, kEqThreads, 0, s>>>(lat);
    k_eq_finish<<<1, 128, 0, s>>>(lat);
    return cudaGetLastError();
}

}  // namespace swgb
