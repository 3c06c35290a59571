// nf_plan.cu -- device-side work decomposition of the near-field pass.
//
// Every non-empty cell becomes work items of up to 128 sinks against the
// cell's whole 125-cell neighbourhood: floor(n / 128) full tiles, and the
// remainder r cut into pieces that fill the warp's lanes (64 sinks run with
// 2 per lane, 32 with 1 per lane, <= 16 split the sources over the lanes):
// r > 96 stays one tile; otherwise 64, 32 and 16 are taken while they fit
// and the rest (<= 16) is the last piece.  A piece costs about its lanes x
// neighbourhood, so this cuts the idle lanes of partly filled tiles.  Items are written class
// by class of cell occupancy (>= 4096, >= 512, >= 64, >= 8, >= 1 particles),
// so the persistent kernel takes the longest items first and the short ones
// fill the tail (load imbalance across cells of very different density is
// what the paper names as the cause of its late-time slowdown, Section 2.3).
// Nothing here leaves the device: the item count stays in device memory and
// is read by the pair kernel, so planning needs no host synchronisation.
#include "nf_internal.cuh"

namespace nf {
namespace {

inline int nblocks(int64_t n, int per) { return static_cast<int>((n + per - 1) / per); }

// sizes of the remainder pieces of r (0 < r < 128); returns how many (<= 4)
__device__ __forceinline__ int remainder_pieces(int r, int *out)
{
    int k = 0;
    if (r > 96) {
        out[k++] = r;
        return k;
    }
    if (r >= 64) { out[k++] = 64; r -= 64; }
    if (r >= 32) { out[k++] = 32; r -= 32; }
    if (r > 16) { out[k++] = 16; r -= 16; }
    if (r > 0) out[k++] = r;
    return k;
}

__device__ __forceinline__ int items_of_cell(int n)
{
    int tmp[4];
    const int r = n % kTile;
    return n / kTile + (r ? remainder_pieces(r, tmp) : 0);
}

__global__ void class_counts(const int *__restrict__ cell_start, int ncell, int cls, int *__restrict__ counts)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    if (c == ncell) {
        counts[c] = 0;
        return;
    }
    const int n = cell_start[c + 1] - cell_start[c];
    counts[c] = (n > 0 && occupancy_class(n) == cls) ? items_of_cell(n) : 0;
}

__global__ void emit_items(const int *__restrict__ cell_start, int ncell, int cls, int box,
                           const int *__restrict__ offsets, const int *__restrict__ base_p, Item *__restrict__ items)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int s0 = cell_start[c];
    const int n = cell_start[c + 1] - s0;
    if (n <= 0 || occupancy_class(n) != cls) return;
    int out = *base_p + offsets[c];
    Item it;
    it.box = box;
    it.cell = c;
    int begin = s0;
    for (int t = 0; t < n / kTile; ++t, ++out, begin += kTile) {
        it.sink_begin = begin;
        it.sink_count = kTile;
        items[out] = it;
    }
    const int r = n % kTile;
    if (r) {
        int sz[4];
        const int k = remainder_pieces(r, sz);
        for (int q = 0; q < k; ++q, ++out) {
            it.sink_begin = begin;
            it.sink_count = sz[q];
            items[out] = it;
            begin += sz[q];
        }
    }
}

__global__ void advance_base(int *__restrict__ base_p, const int *__restrict__ offsets, int ncell)
{
    *base_p += offsets[ncell];
}

__global__ void zero_int(int *p) { *p = 0; }

// 5-point periodic window sum along one axis of a cpd^3 array
__global__ void window_sum(const int *__restrict__ in, int *__restrict__ out, int cpd, int axis)
{
    const int64_t ncell = static_cast<int64_t>(cpd) * cpd * cpd;
    const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int z = static_cast<int>(c % cpd), y = static_cast<int>((c / cpd) % cpd);
    const int x = static_cast<int>(c / (static_cast<int64_t>(cpd) * cpd));
    int s = 0;
    for (int d = -kR; d <= kR; ++d) {
        int xx = x, yy = y, zz = z;
        if (axis == 0) xx = (x + d + cpd) % cpd;
        else if (axis == 1) yy = (y + d + cpd) % cpd;
        else zz = (z + d + cpd) % cpd;
        s += in[(static_cast<int64_t>(xx) * cpd + yy) * cpd + zz];
    }
    out[c] = s;
}

__global__ void occupancy(const int *__restrict__ cell_start, int ncell, int *__restrict__ occ)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) occ[c] = cell_start[c + 1] - cell_start[c];
}

__global__ void dot_counts(const int *__restrict__ cell_start, const int *__restrict__ nbr, int ncell,
                           unsigned long long *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (c < ncell)
        v = static_cast<unsigned long long>(cell_start[c + 1] - cell_start[c]) * static_cast<unsigned long long>(nbr[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

}  // namespace

cudaError_t zero_device_int(int *p, cudaStream_t st)
{
    zero_int<<<1, 1, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t plan_items_class(const int *cell_start, int ncell, int box_index, int cls, Item *items, int *n_items,
                             int *scratch_counts, int *scratch_offsets, void *scan_temp, cudaStream_t st)
{
    class_counts<<<nblocks(static_cast<int64_t>(ncell) + 1, 256), 256, 0, st>>>(cell_start, ncell, cls,
                                                                                 scratch_counts);
    cudaError_t e =
        exclusive_scan_i32(scratch_counts, scratch_offsets, static_cast<int64_t>(ncell) + 1, scan_temp, st);
    if (e != cudaSuccess) return e;
    emit_items<<<nblocks(ncell, 256), 256, 0, st>>>(cell_start, ncell, cls, box_index, scratch_offsets, n_items,
                                                    items);
    advance_base<<<1, 1, 0, st>>>(n_items, scratch_offsets, ncell);
    return cudaGetLastError();
}

cudaError_t neighbour_pairs(const int *cell_start, int cpd, unsigned long long *pairs, int *tmp_a, int *tmp_b,
                            cudaStream_t st)
{
    const int ncell = cpd * cpd * cpd;
    occupancy<<<nblocks(ncell, 256), 256, 0, st>>>(cell_start, ncell, tmp_a);
    window_sum<<<nblocks(ncell, 256), 256, 0, st>>>(tmp_a, tmp_b, cpd, 2);
    window_sum<<<nblocks(ncell, 256), 256, 0, st>>>(tmp_b, tmp_a, cpd, 1);
    window_sum<<<nblocks(ncell, 256), 256, 0, st>>>(tmp_a, tmp_b, cpd, 0);
    cudaMemsetAsync(pairs, 0, sizeof(unsigned long long), st);
    dot_counts<<<nblocks(ncell, 256), 256, 0, st>>>(cell_start, tmp_b, ncell, pairs);
    return cudaGetLastError();
}

}  // namespace nf
