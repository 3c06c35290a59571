// nf_sort.cu -- cell binning (Section 2.1: K^3 cells, every particle in one
// cell, positions as offsets from the cell centre), exclusive scan, and a
// stable LSD radix sort used to order particles by cell.
//
// Binning rule (also the re-binning rule after a drift):
//   s = x * (cpd / box)          double, one rounding
//   c = floor(s)                 cell along the axis (wrapped into [0, cpd))
//   x_rel = (s - c) - 1/2        exact; offset from the centre in cell widths
//   x_q = rint(x_rel 2^22) 2^-22 half-to-even; exact in FP32
// Cell id = (cx cpd + cy) cpd + cz.  The sort is stable, so particles of a
// cell keep the order of the input (particle id order).
#include <cfloat>
#include <cmath>

#include "nf_bin.cuh"
#include "nf_internal.cuh"

namespace nf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsThreads * kRsRounds;       // 2048

inline int nblocks(int64_t n, int per) { return static_cast<int>((n + per - 1) / per); }

// block-wide exclusive scan of one int per thread; *total gets the block sum
__device__ int block_exclusive_scan(int v, int *warp_sums, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < nw ? warp_sums[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) warp_sums[lane] = wi - w;
        if (lane == 31) warp_sums[32] = wi;
    }
    __syncthreads();
    const int res = warp_sums[warp] + incl - v;
    *total = warp_sums[32];
    __syncthreads();
    return res;
}

__global__ void scan_reduce(const int *__restrict__ in, int64_t n, int *__restrict__ partials)
{
    __shared__ int ws[33];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    int tot;
    block_exclusive_scan(s, ws, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// exclusive scan of the block partials, one block, in chunks with a carry
__global__ void scan_partials(int *__restrict__ partials, int nb)
{
    __shared__ int ws[33];
    int carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? partials[i] : 0;
        int chunk_total;
        const int ex = block_exclusive_scan(v, ws, &chunk_total);
        if (i < nb) partials[i] = carry + ex;
        carry += chunk_total;
    }
}

// in == out is allowed: every thread reads its own items before any write
__global__ void scan_down(const int *in, int *out, int64_t n, const int *__restrict__ partials)
{
    __shared__ int ws[33];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    int run = block_exclusive_scan(s, ws, &tot) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ---------------------------------------------------------------- radix sort

__global__ void radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift, int nb, int *__restrict__ hist)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile = static_cast<int64_t>(blockIdx.x) * kRsTile;
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t e = tile + r * kRsThreads + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(keys[e] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[static_cast<int64_t>(threadIdx.x) * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: within a tile, elements are ranked in order (round by
// round, warp by warp, lane by lane) among elements of the same digit.  The
// tile is first laid out in shared memory in output order (digit by digit),
// then written so that consecutive threads write consecutive elements of each
// digit's run: the global writes come in runs rather than one element per
// digit and round.
__global__ void radix_scatter(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                              int shift, int nb, const int *__restrict__ hist, const int *__restrict__ offs,
                              uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out)
{
    __shared__ int run[256];                      // running local position of each digit
    __shared__ int lstart[256];                   // the digit's first local position
    __shared__ int gbase[256];                    // the digit's first global position for this tile
    __shared__ int wtot[kRsThreads / 32];
    __shared__ int wcnt[kRsThreads / 32][256];
    __shared__ uint32_t skey[kRsTile], sval[kRsTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile = static_cast<int64_t>(blockIdx.x) * kRsTile;
    const int count = static_cast<int>(n - tile < kRsTile ? n - tile : kRsTile);
    {
        // the tile's digit counts (histogram pass) -> local starts by a block scan
        const int d = threadIdx.x;
        const int c = hist[static_cast<int64_t>(d) * nb + blockIdx.x];
        gbase[d] = offs[static_cast<int64_t>(d) * nb + blockIdx.x];
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wtot[warp] = x;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wtot[w];
        lstart[d] = before + x - c;
        run[d] = before + x - c;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kRsRounds; ++r) {
#pragma unroll
        for (int w = 0; w < kRsThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t e = tile + r * kRsThreads + threadIdx.x;
        const bool valid = e < n;
        const uint32_t key = valid ? keys[e] : 0u;
        const uint32_t val = valid ? vals[e] : 0u;
        const int d = valid ? static_cast<int>((key >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(kFull, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int acc = run[threadIdx.x];
#pragma unroll
            for (int w = 0; w < kRsThreads / 32; ++w) {
                const int c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = acc;
                acc += c;
            }
            run[threadIdx.x] = acc;
        }
        __syncthreads();
        if (valid) {
            const int lpos = wcnt[warp][d] + rank;   // output order within the tile
            skey[lpos] = key;
            sval[lpos] = val;
        }
        __syncthreads();
    }
    // write out in output order: element j of the tile goes to its digit's global run
    for (int j = threadIdx.x; j < count; j += kRsThreads) {
        const uint32_t key = skey[j];
        const int d = static_cast<int>((key >> shift) & 255u);
        const int dest = gbase[d] + (j - lstart[d]);
        keys_out[dest] = key;
        vals_out[dest] = sval[j];
    }
}

// ---------------------------------------------------------------- binning

__device__ __forceinline__ bool bin_axis(double x, double inv_w, int cpd, int &cell, float &xq)
{
    return bin_cell_units(__dmul_rn(x, inv_w), cpd, cell, xq);
}

__global__ void bin_global_kernel(const double *__restrict__ xyz, int n, int cpd, double inv_w,
                                  uint32_t *__restrict__ key, uint32_t *__restrict__ val,
                                  float4 *__restrict__ xq_by_id, int *__restrict__ counts, int *__restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx, cy, cz;
    float qx, qy, qz;
    const double *p = xyz + 3 * static_cast<int64_t>(i);
    const bool ok = bin_axis(p[0], inv_w, cpd, cx, qx) & bin_axis(p[1], inv_w, cpd, cy, qy) &
                    bin_axis(p[2], inv_w, cpd, cz, qz);
    if (!ok) {
        atomicOr(err, 1);
        cx = cy = cz = 0;
        qx = qy = qz = 0.f;
    }
    const uint32_t c = static_cast<uint32_t>((cx * cpd + cy) * cpd + cz);
    key[i] = c;
    val[i] = static_cast<uint32_t>(i);
    xq_by_id[i] = make_float4(qx, qy, qz, 0.f);
    atomicAdd(&counts[c], 1);
}

// w of a stored position: the z index of its cell (cell ids are x-major, z fastest), an
// integer below 2^24 and so exact in FP32; lane items take each source's z offset from it
__device__ __forceinline__ float cell_z(uint32_t cell, int cpd)
{
    return static_cast<float>(cell % static_cast<uint32_t>(cpd));
}

__global__ void gather_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ keys, int cpd,
                              const float4 *__restrict__ xq_by_id, const float4 *__restrict__ vel_by_id,
                              float4 *__restrict__ pos, float4 *__restrict__ vel, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t i = perm[k];
    const float4 q = xq_by_id[i];
    pos[k] = make_float4(q.x, q.y, q.z, cell_z(keys[k], cpd));
    if (vel) vel[k] = vel_by_id ? vel_by_id[i] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// nf_set_particles validation: offsets/counts consistency and offset bounds
__global__ void validate_cells(const int64_t *__restrict__ offsets, const int32_t *__restrict__ counts, int ncell,
                               int n, int *__restrict__ cell_start, int *__restrict__ err)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    const int64_t o = offsets[c];
    if (c == 0 && o != 0) atomicOr(err, 1);
    if (c == ncell) {
        if (o != n) atomicOr(err, 2);
        cell_start[c] = n;
        return;
    }
    const int32_t k = counts[c];
    if (k < 0) atomicOr(err, 4);
    if (offsets[c + 1] - o != k) atomicOr(err, 8);
    if (o < 0 || o > n) atomicOr(err, 16);
    cell_start[c] = static_cast<int>(o < 0 ? 0 : (o > n ? n : o));
}

__global__ void validate_pos(const float4 *__restrict__ pos, int n, float4 *__restrict__ out, int *__restrict__ err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 p = pos[k];
    const float lim = 0.5f * (1.0f + 9.5367431640625e-07f);   // 1/2 (1 + 2^-20)
    bool ok = true;
    float q[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(fabsf(q[a]) <= lim)) ok = false;
        q[a] = static_cast<float>(__dmul_rn(rint(__dmul_rn(static_cast<double>(q[a]), kTwo22)), kTwoM22));
    }
    if (!ok) {
        atomicOr(err, 32);
        q[0] = q[1] = q[2] = 0.f;
    }
    out[k] = make_float4(q[0], q[1], q[2], 0.f);
}

__global__ void cell_ids_kernel(const int *__restrict__ cell_start, int ncell, int n, uint32_t *__restrict__ cell_of,
                                float4 *__restrict__ pos, int cpd)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int lo = 0, hi = ncell;   // cell_start[lo] <= k < cell_start[hi]
    while (hi - lo > 1) {
        const int mid = lo + ((hi - lo) >> 1);
        if (cell_start[mid] <= k) lo = mid; else hi = mid;
    }
    cell_of[k] = static_cast<uint32_t>(lo);
    if (pos) pos[k].w = cell_z(static_cast<uint32_t>(lo), cpd);
}

__global__ void count_keys_kernel(const uint32_t *__restrict__ keys, int n, int *__restrict__ counts)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) atomicAdd(&counts[keys[k]], 1);
}

__global__ void iota_kernel(uint32_t *p, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = static_cast<uint32_t>(k);
}

}  // namespace

size_t scan_temp_bytes(int64_t n) { return sizeof(int) * static_cast<size_t>(nblocks(n, kScanTile) + 1); }

cudaError_t exclusive_scan_i32(const int *in, int *out, int64_t n, void *temp, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int nb = nblocks(n, kScanTile);
    int *partials = static_cast<int *>(temp);
    scan_reduce<<<nb, kScanThreads, 0, st>>>(in, n, partials);
    scan_partials<<<1, 1024, 0, st>>>(partials, nb);
    scan_down<<<nb, kScanThreads, 0, st>>>(in, out, n, partials);
    return cudaGetLastError();
}

size_t radix_temp_bytes(int64_t n)
{
    const int64_t nb = nblocks(n < 1 ? 1 : n, kRsTile);
    const int64_t hist = 256 * nb;
    return sizeof(int) * static_cast<size_t>(2 * hist) + scan_temp_bytes(hist) + 256;
}

cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, int64_t n,
                             int key_bits, void *temp, int *result_in_alt, cudaStream_t st)
{
    *result_in_alt = 0;
    if (n <= 1) return cudaSuccess;
    const int nb = nblocks(n, kRsTile);
    const int64_t hist_n = 256 * static_cast<int64_t>(nb);
    int *hist = static_cast<int *>(temp);
    int *offs = hist + hist_n;
    void *scan_tmp = offs + hist_n;
    uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    int passes = (key_bits + 7) / 8;
    if (passes < 1) passes = 1;
    for (int p = 0; p < passes; ++p) {
        radix_hist<<<nb, kRsThreads, 0, st>>>(ki, n, 8 * p, nb, hist);
        cudaError_t e = exclusive_scan_i32(hist, offs, hist_n, scan_tmp, st);
        if (e != cudaSuccess) return e;
        radix_scatter<<<nb, kRsThreads, 0, st>>>(ki, vi, n, 8 * p, nb, hist, offs, ko, vo);
        uint32_t *t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    *result_in_alt = (passes & 1);
    return cudaGetLastError();
}

cudaError_t bin_global(const double *xyz, int n, int cpd, double inv_w, uint32_t *key, uint32_t *val,
                       float4 *xq_by_id, int *counts, int *err, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    bin_global_kernel<<<nblocks(n, 256), 256, 0, st>>>(xyz, n, cpd, inv_w, key, val, xq_by_id, counts, err);
    return cudaGetLastError();
}

// the drift's records (offset with key bits, velocity) into storage order: one
// 32-byte record read per particle
__global__ void gather_state_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ keys, int cpd,
                                    const float4 *__restrict__ state_by_id, float4 *__restrict__ pos,
                                    float4 *__restrict__ vel, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 *rec = state_by_id + 2 * static_cast<int64_t>(perm[k]);
    const float4 q = rec[0];
    pos[k] = make_float4(q.x, q.y, q.z, cell_z(keys[k], cpd));   // the record's w held the cell id's bits
    vel[k] = rec[1];
}

cudaError_t gather_state(const uint32_t *perm, const uint32_t *keys, int cpd, const float4 *state_by_id, float4 *pos,
                         float4 *vel, int n, cudaStream_t st)
{
    gather_state_kernel<<<nblocks(n, 256), 256, 0, st>>>(perm, keys, cpd, state_by_id, pos, vel, n);
    return cudaGetLastError();
}

cudaError_t gather_sorted(const uint32_t *perm, const uint32_t *keys, int cpd, const float4 *xq_by_id,
                          const float4 *vel_by_id, float4 *pos, float4 *vel, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    gather_kernel<<<nblocks(n, 256), 256, 0, st>>>(perm, keys, cpd, xq_by_id, vel_by_id, pos, vel, n);
    return cudaGetLastError();
}

cudaError_t validate_loaded(const int64_t *offsets, const int32_t *counts, const float4 *pos, int ncell, int n,
                            int *cell_start, float4 *pos_out, int *err, cudaStream_t st)
{
    validate_cells<<<nblocks(static_cast<int64_t>(ncell) + 1, 256), 256, 0, st>>>(offsets, counts, ncell, n,
                                                                                  cell_start, err);
    if (n > 0) validate_pos<<<nblocks(n, 256), 256, 0, st>>>(pos, n, pos_out, err);
    return cudaGetLastError();
}

cudaError_t fill_cell_ids(const int *cell_start, int ncell, int n, uint32_t *cell_of, float4 *pos, int cpd,
                          cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    cell_ids_kernel<<<nblocks(n, 256), 256, 0, st>>>(cell_start, ncell, n, cell_of, pos, cpd);
    return cudaGetLastError();
}

cudaError_t count_keys(const uint32_t *keys, int n, int *counts, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_keys_kernel<<<nblocks(n, 256), 256, 0, st>>>(keys, n, counts);
    return cudaGetLastError();
}

cudaError_t iota_u32(uint32_t *p, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    iota_kernel<<<nblocks(n, 256), 256, 0, st>>>(p, n);
    return cudaGetLastError();
}

}  // namespace nf
