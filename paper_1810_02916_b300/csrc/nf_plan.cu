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
// Sparse cells with small neighbourhoods (lane_cell) become lane items instead,
// appended last: runs of consecutive such cells along z with at most 32 sinks,
// one sink per lane, which spares the tail one warp-wide setup per cell.
// Nothing here leaves the device: the item count stays in device memory and
// is read by the pair kernel, so planning needs no host synchronisation.
#include <algorithm>

#include "nf_internal.cuh"

namespace nf {
namespace {

inline int nblocks(int64_t n, int per) { return static_cast<int>((n + per - 1) / per); }

// sizes of the remainder pieces of r (0 < r < 128) under the tile policy (see
// TilePolicy); returns how many (<= 4)
__device__ __forceinline__ int remainder_pieces(int r, const TilePolicy &pol, int *out)
{
    int k = 0;
    if (r > pol.c4) {
        out[k++] = r;
        return k;
    }
    if (r >= 64) { out[k++] = 64; r -= 64; }
    if (r > pol.c2) {
        out[k++] = r;
        return k;
    }
    if (r >= 32) { out[k++] = 32; r -= 32; }
    if (r > pol.c1) {
        out[k++] = r;
        return k;
    }
    if (r > 16) { out[k++] = 16; r -= 16; }
    if (r > 0) out[k++] = r;
    return k;
}

__device__ __forceinline__ int items_of_cell(int n, const TilePolicy &pol)
{
    int tmp[4];
    const int r = n % kTile;
    return n / kTile + (r ? remainder_pieces(r, pol, tmp) : 0);
}

__global__ void class_counts(const int *__restrict__ cell_start, const int *__restrict__ nbr, int ncell, int cls,
                             TilePolicy pol, int *__restrict__ counts)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    if (c == ncell) {
        counts[c] = 0;
        return;
    }
    const int n = cell_start[c + 1] - cell_start[c];
    counts[c] = (!lane_cell(n, nbr[c]) && occupancy_class(n) == cls) ? items_of_cell(n, pol) : 0;
}

__global__ void emit_items(const int *__restrict__ cell_start, const int *__restrict__ nbr, int ncell, int cls,
                           int box, TilePolicy pol, const int *__restrict__ offsets, const int *__restrict__ base_p,
                           Item *__restrict__ items)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int s0 = cell_start[c];
    const int n = cell_start[c + 1] - s0;
    if (lane_cell(n, nbr[c]) || occupancy_class(n) != cls) return;
    int out = *base_p + offsets[c];
    Item it;
    it.cell = c;
    it.piece = -1;
    int begin = s0;
    for (int t = 0; t < n / kTile; ++t, ++out, begin += kTile) {
        it.sink_begin = begin;
        it.box_count = (box << 16) | kTile;
        items[out] = it;
    }
    const int r = n % kTile;
    if (r) {
        int sz[4];
        const int k = remainder_pieces(r, pol, sz);
        for (int q = 0; q < k; ++q, ++out) {
            it.sink_begin = begin;
            it.box_count = (box << 16) | sz[q];
            items[out] = it;
            begin += sz[q];
        }
    }
}

// Lane groups of one z-row of cells (row = x * cpd + y): walking z upwards, a
// group opens at a non-empty lane cell and takes the following cells while each
// is a lane cell (empty ones included), the sinks stay <= 32 and the cells
// <= kLaneMaxCells.  With items == nullptr only counts.
__device__ int lane_row(const int *__restrict__ cs, const int *__restrict__ nbr, int cpd, int row, int box,
                        Item *items, int out)
{
    const int c0 = row * cpd;
    int groups = 0, g0 = -1, total = 0;
    int s = cs[c0];
    for (int z = 0; z <= cpd; ++z) {
        const int c = c0 + z;
        int n = 0;
        bool is_lane = false;
        if (z < cpd) {
            const int s1 = cs[c + 1];
            n = s1 - s;
            s = s1;
            is_lane = lane_cell(n, nbr[c]);
        }
        if (g0 >= 0) {
            if (is_lane && total + n <= 32 && c - g0 < kLaneMaxCells) {
                total += n;
                continue;
            }
            if (items) {
                Item it;
                it.box_count = (box << 16) | total;
                it.cell = g0;
                it.sink_begin = cs[g0];
                it.piece = -1 - (c - g0);
                items[out + groups] = it;
            }
            ++groups;
            g0 = -1;
        }
        if (is_lane && n > 0) {
            g0 = c;
            total = n;
        }
    }
    return groups;
}

__global__ void lane_count(const int *__restrict__ cell_start, const int *__restrict__ nbr, int cpd,
                           int *__restrict__ counts)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int rows = cpd * cpd;
    if (row > rows) return;
    counts[row] = row < rows ? lane_row(cell_start, nbr, cpd, row, 0, nullptr, 0) : 0;
}

__global__ void lane_emit(const int *__restrict__ cell_start, const int *__restrict__ nbr, int cpd, int box,
                          const int *__restrict__ offsets, const int *__restrict__ base_p, Item *__restrict__ items)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= cpd * cpd) return;
    lane_row(cell_start, nbr, cpd, row, box, items, *base_p + offsets[row]);
}

__global__ void advance_base(int *__restrict__ base_p, const int *__restrict__ offsets, int ncell)
{
    *base_p += offsets[ncell];
}

__global__ void zero_int(int *p) { *p = 0; }

// Sum over the 2 radius + 1 cells along z (periodic) of the cell occupancy, read
// straight from cell_start; with n_min > 0 only the cells below n_min (dense = 0)
// or only those at or above it (dense = 1) count.  Indices fit 32 bits (cpd^3 < 2^31).
__global__ void window_z_occ(const int *__restrict__ cell_start, int cpd, int64_t n_min, int dense, int radius,
                             int *__restrict__ out)
{
    const unsigned C = static_cast<unsigned>(cpd);
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C * C * C) return;
    const unsigned row = c / C, z = c - row * C;
    const int *rs = cell_start + row * C;
    int s = 0;
    for (int d = -radius; d <= radius; ++d) {
        int zz = static_cast<int>(z) + d;
        zz += zz < 0 ? cpd : 0;
        zz -= zz >= cpd ? cpd : 0;
        const int n = rs[zz + 1] - rs[zz];
        s += (n_min <= 0 || (n >= n_min) == (dense != 0)) ? n : 0;
    }
    out[c] = s;
}

// Sum over the 2 radius + 1 cells along y (axis 1) or x (axis 0), periodic.
__global__ void window_yx(const int *__restrict__ in, int *__restrict__ out, int cpd, int axis, int radius)
{
    const unsigned C = static_cast<unsigned>(cpd);
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C * C * C) return;
    const unsigned stride = axis == 1 ? C : C * C;
    const unsigned a = axis == 1 ? (c / C) % C : c / (C * C);
    const unsigned base = c - a * stride;
    int s = 0;
    for (int d = -radius; d <= radius; ++d) {
        int aa = static_cast<int>(a) + d;
        aa += aa < 0 ? cpd : 0;
        aa -= aa >= cpd ? cpd : 0;
        s += in[base + static_cast<unsigned>(aa) * stride];
    }
    out[c] = s;
}

__global__ void add_into(int *__restrict__ a, const int *__restrict__ b, int ncell)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) a[c] += b[c];
}

__global__ void dense_flags(const int *__restrict__ cell_start, int ncell, int64_t n_min, int *__restrict__ flags)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    flags[c] = c < ncell && cell_start[c + 1] - cell_start[c] >= n_min;
}

__global__ void dense_slots(const int *__restrict__ cell_start, int ncell, int64_t n_min,
                            const int *__restrict__ rank, int *__restrict__ dslot, int *__restrict__ dense_cells,
                            int *__restrict__ n_dense)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) *n_dense = rank[ncell];
    if (c >= ncell) return;
    const bool dense = cell_start[c + 1] - cell_start[c] >= n_min;
    dslot[c] = dense ? rank[c] : -1;
    if (dense) dense_cells[rank[c]] = c;
}

__global__ void dot_counts(const int *__restrict__ cell_start, const int *__restrict__ nbr, int ncell,
                           unsigned long long *__restrict__ out)
{
    // grid-stride sum per thread, then one atomic per block
    __shared__ unsigned long long part[32];
    unsigned long long v = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x)
        v += static_cast<unsigned long long>(cell_start[c + 1] - cell_start[c]) * static_cast<unsigned long long>(nbr[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && v) atomicAdd(out, v);
    }
}

// ---- source splitting of long items (deterministic: fixed pieces, fixed reduction order)
//
// An item of s sinks whose neighbourhood holds T sources costs s T pairs.  A
// pass of P pairs on W resident warps balances when no item is much longer
// than P / (W F); items with T above T_max(s) = max(t_floor, P / (W F s)) are
// cut into k = ceil(T / T_max) (<= 64) contiguous ranges of the flattened
// neighbourhood.  Each piece writes FP64 partial sums; reduce_partials adds
// them per sink in piece order.  (Sum over split items of (k - 1) <= W F, so
// the extra items and partial slots are bounded by the launch size.)

__global__ void split_count(const Item *__restrict__ items, const int *__restrict__ n_in, int cap,
                            const int *const *__restrict__ nbr, const unsigned long long *__restrict__ total_pairs,
                            long long warps_x_f, int t_floor, int *__restrict__ k, int *__restrict__ p,
                            int *__restrict__ r)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > cap) return;
    int kk = 0, pp = 0, rr = 0;
    if (i < *n_in) {
        const Item it = items[i];
        const long long s = item_count(it);
        const long long T = nbr[item_box(it)][it.cell];
        long long target = static_cast<long long>(*total_pairs) / (warps_x_f > 0 ? warps_x_f : 1);
        long long tmax = target / (s > 0 ? s : 1);
        if (tmax < t_floor) tmax = t_floor;
        kk = 1;
        if (T > tmax && !item_is_lanes(it)) {
            long long q = (T + tmax - 1) / tmax;
            kk = static_cast<int>(q > 64 ? 64 : q);
            pp = kk * static_cast<int>(s);
            rr = 1;
        }
    }
    k[i] = kk;
    p[i] = pp;
    r[i] = rr;
}

// k, p, r hold exclusive scans here; counts are recovered from neighbours
__global__ void split_expand(const Item *__restrict__ items, const int *__restrict__ n_in,
                             const int *const *__restrict__ nbr, const int *__restrict__ k, const int *__restrict__ p,
                             const int *__restrict__ r, Item *__restrict__ out, int *__restrict__ n_out,
                             Piece *__restrict__ pieces, Reduce *__restrict__ reduces, int *__restrict__ n_reduce)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = *n_in;
    if (i == 0) {
        *n_out = k[n];
        *n_reduce = r[n];
    }
    if (i >= n) return;
    const Item it = items[i];
    const int base = k[i];
    const int kk = k[i + 1] - base;
    if (kk == 1) {
        out[base] = it;
        return;
    }
    const int s = item_count(it);
    const int T = nbr[item_box(it)][it.cell];
    for (int j = 0; j < kk; ++j) {
        Item o = it;
        o.piece = base + j;
        out[base + j] = o;
        Piece pc;
        pc.src_lo = static_cast<int>(static_cast<long long>(T) * j / kk);
        pc.src_hi = static_cast<int>(static_cast<long long>(T) * (j + 1) / kk);
        pc.slot = p[i] + j * s;
        pc.pad = 0;
        pieces[base + j] = pc;
    }
    Reduce rd;
    rd.box_count = it.box_count;
    rd.sink_begin = it.sink_begin;
    rd.slot = p[i];
    rd.pieces = kk;
    reduces[r[i]] = rd;
}

// one thread per (reduce record, sink slot); partials summed in piece order
__global__ void reduce_kernel(const BoxDev *__restrict__ boxes, const Reduce *__restrict__ reduces,
                              const int *__restrict__ n_reduce, int adjoint)
{
    const int rec = blockIdx.x;
    if (rec >= *n_reduce) return;
    const Reduce rd = reduces[rec];
    const int s = rd.box_count & 0xffff;
    const int k = threadIdx.x;
    if (k >= s) return;
    const BoxDev &bx = boxes[rd.box_count >> 16];
    double a[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < rd.pieces; ++j) {
        const double *q = bx.partials + 3 * (static_cast<int64_t>(rd.slot) + static_cast<int64_t>(j) * s + k);
        a[0] += q[0];
        a[1] += q[1];
        a[2] += q[2];
    }
    const double scale = adjoint ? bx.grad_scale : bx.acc_scale * kForceUnscale;   // forces: accumulators' scale
    const int idx = rd.sink_begin + k;
    const double gx = a[0] * scale, gy = a[1] * scale, gz = a[2] * scale;
    if (bx.acc64) {
        double *o = bx.acc64 + 3 * static_cast<int64_t>(idx);
        o[0] = gx; o[1] = gy; o[2] = gz;
    }
    if (bx.acc_out)
        bx.acc_out[idx] = make_float4(static_cast<float>(gx), static_cast<float>(gy), static_cast<float>(gz), 0.f);
}

// flags[i] = 1 for a heavy item at i < n, 0 elsewhere (i <= cap)
__global__ void heavy_flags(const Item *__restrict__ items, const int *__restrict__ n_p, int cap, int *__restrict__ flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > cap) return;
    flags[i] = (i < *n_p && !item_is_light(items[i])) ? 1 : 0;
}

// flags hold the exclusive scan of the heavy flags here
__global__ void partition_scatter(const Item *__restrict__ items, int *__restrict__ n_items,
                                  const int *__restrict__ pos, Item *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = n_items[0];
    const int n_heavy = pos[n];
    if (i == 0) n_items[1] = n_heavy;
    if (i >= n) return;
    const Item it = items[i];
    const int h = pos[i];
    out[item_is_light(it) ? n_heavy + (i - h) : h] = it;
}

__global__ void hist_kernel(const int *__restrict__ cell_start, int ncell, unsigned long long *__restrict__ hist)
{
    __shared__ unsigned long long h[kHistBins];
    if (threadIdx.x < kHistBins) h[threadIdx.x] = 0;
    __syncthreads();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const int n = cell_start[c + 1] - cell_start[c];
        if (n > 0) atomicAdd(&h[min(31 - __clz(n), kHistBins - 1)], static_cast<unsigned long long>(n));
    }
    __syncthreads();
    if (threadIdx.x < kHistBins && h[threadIdx.x]) atomicAdd(hist + threadIdx.x, h[threadIdx.x]);
}

}  // namespace

cudaError_t occupancy_hist(const int *cell_start, int ncell, unsigned long long *hist, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kHistBins, st);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(1024, nblocks(ncell, 256)));
    hist_kernel<<<blocks, 256, 0, st>>>(cell_start, ncell, hist);
    return cudaGetLastError();
}

cudaError_t partition_light(const Item *items_in, int *n_items, int cap, int *flags, void *scan_temp,
                            Item *items_out, cudaStream_t st)
{
    const int64_t m = static_cast<int64_t>(cap) + 1;
    heavy_flags<<<nblocks(m, 256), 256, 0, st>>>(items_in, n_items, cap, flags);
    cudaError_t e = exclusive_scan_i32(flags, flags, m, scan_temp, st);
    if (e != cudaSuccess) return e;
    partition_scatter<<<nblocks(m, 256), 256, 0, st>>>(items_in, n_items, flags, items_out);
    return cudaGetLastError();
}

__global__ void sum_kernel(const unsigned long long *const *ptrs, int n, unsigned long long *out)
{
    unsigned long long s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += *ptrs[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ unsigned long long w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) t += w[i];
        *out = t;
    }
}

cudaError_t sum_pair_counts(const unsigned long long *const *ptrs, int n, unsigned long long *out, cudaStream_t st)
{
    sum_kernel<<<1, 256, 0, st>>>(ptrs, n, out);
    return cudaGetLastError();
}

cudaError_t split_items(const Item *items_in, const int *n_in, int item_cap, const int *const *nbr,
                        const unsigned long long *total_pairs, long long warps_x_f, int t_floor, int *k, int *p,
                        int *r, void *scan_temp, Item *items_out, int *n_out, Piece *pieces, Reduce *reduces,
                        int *n_reduce, cudaStream_t st)
{
    const int64_t m = static_cast<int64_t>(item_cap) + 1;
    split_count<<<nblocks(m, 256), 256, 0, st>>>(items_in, n_in, item_cap, nbr, total_pairs, warps_x_f, t_floor, k, p,
                                                 r);
    cudaError_t e;
    if ((e = exclusive_scan_i32(k, k, m, scan_temp, st)) != cudaSuccess) return e;
    if ((e = exclusive_scan_i32(p, p, m, scan_temp, st)) != cudaSuccess) return e;
    if ((e = exclusive_scan_i32(r, r, m, scan_temp, st)) != cudaSuccess) return e;
    split_expand<<<nblocks(m, 256), 256, 0, st>>>(items_in, n_in, nbr, k, p, r, items_out, n_out, pieces, reduces,
                                                  n_reduce);
    return cudaGetLastError();
}

cudaError_t reduce_partials(const BoxDev *boxes, const Reduce *reduces, const int *n_reduce, int max_reduce,
                            int adjoint, cudaStream_t st)
{
    if (max_reduce <= 0) return cudaSuccess;
    reduce_kernel<<<max_reduce, kTile, 0, st>>>(boxes, reduces, n_reduce, adjoint);
    return cudaGetLastError();
}

cudaError_t zero_device_int(int *p, cudaStream_t st)
{
    zero_int<<<1, 1, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t plan_items_class(const int *cell_start, const int *nbr, int ncell, int box_index, int cls, Item *items,
                             int *n_items, int *scratch_counts, int *scratch_offsets, void *scan_temp,
                             TilePolicy pol, cudaStream_t st)
{
    class_counts<<<nblocks(static_cast<int64_t>(ncell) + 1, 256), 256, 0, st>>>(cell_start, nbr, ncell, cls, pol,
                                                                                 scratch_counts);
    cudaError_t e =
        exclusive_scan_i32(scratch_counts, scratch_offsets, static_cast<int64_t>(ncell) + 1, scan_temp, st);
    if (e != cudaSuccess) return e;
    emit_items<<<nblocks(ncell, 256), 256, 0, st>>>(cell_start, nbr, ncell, cls, box_index, pol, scratch_offsets,
                                                    n_items, items);
    advance_base<<<1, 1, 0, st>>>(n_items, scratch_offsets, ncell);
    return cudaGetLastError();
}

cudaError_t plan_dense_cells(const int *cell_start, int ncell, int64_t n_min, int *dslot, int *dense_cells,
                             int *n_dense, int *scratch_counts, int *scratch_offsets, void *scan_temp,
                             cudaStream_t st)
{
    dense_flags<<<nblocks(static_cast<int64_t>(ncell) + 1, 256), 256, 0, st>>>(cell_start, ncell, n_min,
                                                                                scratch_counts);
    cudaError_t e =
        exclusive_scan_i32(scratch_counts, scratch_offsets, static_cast<int64_t>(ncell) + 1, scan_temp, st);
    if (e != cudaSuccess) return e;
    dense_slots<<<nblocks(ncell > 0 ? ncell : 1, 256), 256, 0, st>>>(cell_start, ncell, n_min, scratch_offsets, dslot,
                                                                      dense_cells, n_dense);
    return cudaGetLastError();
}

cudaError_t plan_lane_items(const int *cell_start, const int *nbr, int cpd, int box_index, Item *items, int *n_items,
                            int *scratch_counts, int *scratch_offsets, void *scan_temp, cudaStream_t st)
{
    if (kLaneMaxN <= 0) return cudaSuccess;
    const int rows = cpd * cpd;
    lane_count<<<nblocks(static_cast<int64_t>(rows) + 1, 128), 128, 0, st>>>(cell_start, nbr, cpd, scratch_counts);
    cudaError_t e = exclusive_scan_i32(scratch_counts, scratch_offsets, static_cast<int64_t>(rows) + 1, scan_temp, st);
    if (e != cudaSuccess) return e;
    lane_emit<<<nblocks(rows, 128), 128, 0, st>>>(cell_start, nbr, cpd, box_index, scratch_offsets, n_items, items);
    advance_base<<<1, 1, 0, st>>>(n_items, scratch_offsets, rows);
    return cudaGetLastError();
}

cudaError_t neighbour_pairs(const int *cell_start, int cpd, int64_t n_min, unsigned long long *pairs, int *tmp,
                            int *tmp2, int *nbr, int *nbr_all, cudaStream_t st)
{
    const int ncell = cpd * cpd * cpd;
    const int nb = nblocks(ncell, 256);
    if (n_min > 0) {
        // cut-off mode: every particle of the 125-cell window, dense cells included (the
        // lane-item choice must see a dense far cell, which run_lanes would sum pair by pair)
        window_z_occ<<<nb, 256, 0, st>>>(cell_start, cpd, 0, 0, kR, nbr_all);
        window_yx<<<nb, 256, 0, st>>>(nbr_all, tmp, cpd, 1, kR);
        window_yx<<<nb, 256, 0, st>>>(tmp, nbr_all, cpd, 0, kR);
    }
    // cells summed over the whole 125-cell window (all of them, or those below n_min) ...
    window_z_occ<<<nb, 256, 0, st>>>(cell_start, cpd, n_min, 0, kR, nbr);
    window_yx<<<nb, 256, 0, st>>>(nbr, tmp, cpd, 1, kR);
    window_yx<<<nb, 256, 0, st>>>(tmp, nbr, cpd, 0, kR);
    if (n_min > 0) {
        // ... and, in cut-off mode, the dense cells over the 27 near cells only
        window_z_occ<<<nb, 256, 0, st>>>(cell_start, cpd, n_min, 1, 1, tmp2);
        window_yx<<<nb, 256, 0, st>>>(tmp2, tmp, cpd, 1, 1);
        window_yx<<<nb, 256, 0, st>>>(tmp, tmp2, cpd, 0, 1);
        add_into<<<nb, 256, 0, st>>>(nbr, tmp2, ncell);
    }
    cudaMemsetAsync(pairs, 0, sizeof(unsigned long long), st);
    dot_counts<<<std::max(1, std::min(nb, 148 * 8)), 256, 0, st>>>(cell_start, nbr, ncell, pairs);
    return cudaGetLastError();
}

}  // namespace nf
