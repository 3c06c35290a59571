// nf_internal.cuh -- shared declarations of the library's translation units.
// Not part of the public ABI (include/nearfield.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nf {

// Scale of the pair kernel's force accumulators: they hold kForceSigma times
// the acceleration (cell units), kForceSigma = -(A - 1) with A = 13981013 *
// 2^-23, the FP32 value nearest 5/3 (so A - 1 = 11184810 * 2^-24 is exact in
// FP32).  The Newtonian tail then needs no separate Newton factor: with y the
// SFU estimate of (r^2)^-1/2 and h = r^2 y^2 = 1 - 2e, one Newton step gives
// r^-3 = y^3 (1 + 3e), and y^3 (h - A) = -y^3 (A - 1 + 2e) equals kForceSigma
// y^3 (1 + 3e) up to a relative 3e (2/(3(A - 1)) - 1) < 2^-43.  Every force
// path (spline and Plummer laws, cut-off moments) accumulates in this scale;
// the FP64 result is multiplied by kForceUnscale.  The adjoint is unscaled.
constexpr float kNewtonA = 1.66666662693023681640625f;
constexpr float kForceSigma = -0.666666626930236816406250f;
constexpr double kForceUnscale = 1.0 / -0.666666626930236816406250;

// Near-field radius supported by the kernels (Section 2.1: R = 2, 125 cells).
constexpr int kR = 2;
constexpr int kNbr = (2 * kR + 1) * (2 * kR + 1) * (2 * kR + 1);   // 125
constexpr int kTile = 128;                                            // sinks per work item (max)

// A source range of one work item whose sink tile is split over several
// warps: flattened neighbourhood sources [src_lo, src_hi), FP64 partial sums
// written at partials[3 * (slot + k)] for the item's k-th sink.
struct Piece {
    int src_lo;
    int src_hi;
    int slot;
    int pad;
};

// One box as the kernels see it.
struct BoxDev {
    const float4 *pos;        // n, cell-relative offsets (cell widths), sorted by cell
    const int *cell_start;    // cpd^3 + 1
    float4 *acc_out;          // n, FP32 output in box units (may be null)
    double *acc64;            // 3 n, FP64 output in box units (may be null)
    const float4 *cot;        // n, cotangent for the adjoint (null for forces)
    const Piece *pieces;      // source ranges of split items (null when nothing is split)
    double *partials;         // FP64 partial sums of split items, cell units
    int cpd;
    int n;
    int zcell;                // 1: pos[k].w holds the z index of particle k's cell (boxes the library loads)
    float a0, a1, a2;         // spline g(r) = a0 + a1 r + a2 r^2 in cell units
    float eps2;               // eps^2 in cell units (spline: adjoint branch test; Plummer: eps_p^2)
    double acc_scale;         // (cpd / box)^2: cell-unit acceleration -> box units
    double grad_scale;        // (cpd / box)^3: cell-unit Jacobian -> box units
    const int *dslot;         // cut-off mode: moment slot of each dense cell, -1 elsewhere (null: exact mode)
    const float *mpole;       // cut-off mode: kCutWords floats per sub-cell, kCutSub sub-cells per dense cell
};

// A work item: up to kTile sinks of one cell against its neighbourhood (or a
// piece of it).  box and sink count share one word: (box << 16) | count.
//
// A lane item instead covers a run of consecutive sparse cells [cell, cell + ng)
// holding at most 32 sinks in all; each lane takes one sink against that sink's
// own neighbourhood (piece = -1 - ng, so piece <= -2 marks a lane item).
struct Item {
    int box_count;
    int cell;
    int sink_begin;
    int piece;                // -1: the whole neighbourhood, final output; >= 0: index into pieces; <= -2: lane item
};
__host__ __device__ inline int item_box(const Item &it) { return it.box_count >> 16; }
__host__ __device__ inline int item_count(const Item &it) { return it.box_count & 0xffff; }
__host__ __device__ inline bool item_is_lanes(const Item &it) { return it.piece <= -2; }
__host__ __device__ inline int item_lane_cells(const Item &it) { return -1 - it.piece; }

// Cells with at most kLaneMaxN particles and at most kLaneMaxT sources in their
// neighbourhood are computed through lane items (runs of at most kLaneMaxCells
// cells and 32 sinks); kLaneMaxN = 0 turns lane items off.
#ifndef NF_LANE_MAX_N
#define NF_LANE_MAX_N 16
#endif
#ifndef NF_LANE_MAX_T
#define NF_LANE_MAX_T 1000
#endif
constexpr int kLaneMaxN = NF_LANE_MAX_N;
constexpr int kLaneMaxT = NF_LANE_MAX_T;
constexpr int kLaneMaxCells = 32;
__host__ __device__ inline bool lane_cell(int n, int nbr) { return n == 0 || (n <= kLaneMaxN && nbr <= kLaneMaxT); }

// Light items: lane items and tiles of at most 16 sinks (the sources split over
// the lanes).  The plan lists them after every heavy item, so the queue runs all
// tiles of more than 16 sinks (largest cells first) before any light item.
__host__ __device__ inline bool item_is_light(const Item &it) { return item_is_lanes(it) || item_count(it) <= 16; }

// Sinks of a split item whose partials are summed (in piece order) by reduce_partials.
struct Reduce {
    int box_count;
    int sink_begin;
    int slot;
    int pieces;
};

// Cut-off acceleration of dense cells: a far cell (Chebyshev distance 2) of
// at least n_min particles acts through the quadrupoles of its kCutK^3
// sub-cells.  Per sub-cell: count, centre of mass (cell units, the cell's own
// frame), traceless Q_xx, Q_xy, Q_xz, Q_yy, Q_yz, Q_zz (cell units^2).
constexpr int kCutK = 4;
constexpr int kCutSub = kCutK * kCutK * kCutK;
constexpr int kCutWords = 10;
// smallest n_min: a dense cell then holds more particles than a lane cell's whole
// 125-cell neighbourhood may (kLaneMaxT), so no lane item has a dense cell in reach
constexpr int kCutMinN = 1024;
static_assert(kLaneMaxT < kCutMinN, "a lane cell's neighbourhood must be smaller than any dense cell");

// How a cell's sinks are cut into work items (its sink tiles): floor(n / 128)
// full tiles of 128 sinks, then the remainder r (0 < r < 128): one tile of r
// sinks if r > c4 (4 sinks per lane); otherwise a piece of 64 while r >= 64,
// then one tile of r if r > c2 (2 per lane); otherwise a piece of 32 while
// r >= 32, then one tile of r if r > c1 (1 per lane); otherwise a piece of 16
// while r > 16, and the rest (<= 16 sinks, the sources split over the lanes).
// c4 in [64, 128], c2 in [32, 64], c1 in [16, 32].  Every piece but the last
// has at least 16 sinks, so a cell of n particles makes at most 1 + n / 16
// items.  split_floor: the shortest source piece of a split item.
struct TilePolicy {
    int c4, c2, c1;
    int split_floor;
};
// default: the tuner's choice on the 512^3 and 256^3 clustered workloads (a remainder of
// 19-31 or 41-63 sinks runs as one partly filled tile rather than split-mode pieces)
constexpr TilePolicy kDefaultTiles{96, 40, 18, 1024};
__host__ __device__ inline bool tile_policy_valid(const TilePolicy &p)
{
    return p.c4 >= 64 && p.c4 <= 128 && p.c2 >= 32 && p.c2 <= 64 && p.c1 >= 16 && p.c1 <= 32 &&
           p.split_floor >= 128 && p.split_floor <= (1 << 20);
}

// Occupancy classes used to order the work queue (largest cells first).
constexpr int kClasses = 5;
__host__ __device__ inline int occupancy_class(int n)
{
    return n >= 4096 ? 0 : n >= 512 ? 1 : n >= 64 ? 2 : n >= 8 ? 3 : 4;
}

// Launch shape of the pair kernel.
struct PairShape {
    int warps;      // warps per block (1..8)
    int stage;      // sources staged per round (128 or 256)
    int blocks;     // persistent grid size (0 = fill the GPU)
};

// Per-class profile of the pair kernel (a diagnostic; off unless a profile
// buffer is passed).  Item classes: kind (0: 4-sink tile, 1: 2-sink, 2: 1-sink,
// 3: <= 16 sinks with the sources split over the lanes, 4: lane item) times
// (whole neighbourhood, source piece): class = 2 kind + (piece >= 0).  Words
// (uint64): [3 cls + 0] summed warp clock cycles spent in the class's items,
// [3 cls + 1] items, [3 cls + 2] pairs (tiled items only; lane items' pairs are
// the pass's total minus the rest); then [kProfWarp + 0] summed warp lifetimes
// (cycles, first grab to exit), [+1] warps, [+2] UINT64_MAX - earliest warp
// start (globaltimer ns), [+3] latest warp exit (globaltimer ns).
constexpr int kProfClasses = 10;
constexpr int kProfWarp = 3 * kProfClasses;
constexpr int kProfWords = kProfWarp + 4;

// ---- pair kernel (nf_pair.cu) ----
// softening: 0 = compact spline (Section 4.3.1), 1 = Plummer (Eq. eqn:plummer)
// prof: kProfWords zero-initialised words, or null (no profile)
cudaError_t launch_pair(const BoxDev *boxes, const Item *items, const int *n_items, int *queue, int compensated,
                        int adjoint, int softening, PairShape shape, int sm_count, cudaStream_t st,
                        unsigned long long *prof = nullptr);
int pair_max_blocks_per_sm(int compensated, int adjoint, int softening, PairShape shape);

// ---- scan / sort / binning (nf_sort.cu) ----
size_t scan_temp_bytes(int64_t n);
cudaError_t exclusive_scan_i32(const int *in, int *out, int64_t n, void *temp, cudaStream_t st);
size_t radix_temp_bytes(int64_t n);
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, int64_t n,
                             int key_bits, void *temp, int *result_in_alt, cudaStream_t st);
cudaError_t bin_global(const double *xyz, int n, int cpd, double inv_w, uint32_t *key, uint32_t *val,
                       float4 *xq_by_id, int *counts, int *err, cudaStream_t st);
// storage order from per-id offsets: pos[k] = (xq_by_id[perm[k]].xyz, z index of cell keys[k])
cudaError_t gather_sorted(const uint32_t *perm, const uint32_t *keys, int cpd, const float4 *xq_by_id,
                          const float4 *vel_by_id, float4 *pos, float4 *vel, int n, cudaStream_t st);
cudaError_t validate_loaded(const int64_t *offsets, const int32_t *counts, const float4 *pos, int ncell, int n,
                            int *cell_start, float4 *pos_out, int *err, cudaStream_t st);
// storage order from the drift's per-id records (state_by_id: 2 float4 per id); pos w as gather_sorted
cudaError_t gather_state(const uint32_t *perm, const uint32_t *keys, int cpd, const float4 *state_by_id, float4 *pos,
                         float4 *vel, int n, cudaStream_t st);
// cell_of[k] = the cell holding storage index k; with pos, also pos[k].w = that cell's z index
cudaError_t fill_cell_ids(const int *cell_start, int ncell, int n, uint32_t *cell_of, float4 *pos, int cpd,
                          cudaStream_t st);
cudaError_t iota_u32(uint32_t *p, int n, cudaStream_t st);
cudaError_t count_keys(const uint32_t *keys, int n, int *counts, cudaStream_t st);

// ---- planner (nf_plan.cu) ----
// Items of one box and one occupancy class, appended at items[*n_items]
// (*n_items is a device int and is advanced).
// nbr: particles in each cell's full 125-cell neighbourhood (neighbour_pairs;
// nbr_all in cut-off mode), which decides the cells left to lane items.
cudaError_t plan_items_class(const int *cell_start, const int *nbr, int ncell, int box_index, int cls, Item *items,
                             int *n_items, int *scratch_counts, int *scratch_offsets, void *scan_temp,
                             TilePolicy pol, cudaStream_t st);
// Lane items of one box (see lane_cell), appended at items[*n_items] after
// every occupancy class.  Scratch: cpd^2 + 1 ints each.
cudaError_t plan_lane_items(const int *cell_start, const int *nbr, int cpd, int box_index, Item *items, int *n_items,
                            int *scratch_counts, int *scratch_offsets, void *scan_temp, cudaStream_t st);
cudaError_t zero_device_int(int *p, cudaStream_t st);
// Split items whose neighbourhood is long against the whole pass into source
// pieces (see nf_plan.cu).  items_in/n_in: the class-ordered list; nbr[box]:
// sources in each cell's neighbourhood of that box; total_pairs: pair count of the pass; warps_x_f:
// resident warps times the balance factor.  Scratch k/p/r: item_cap + 1 ints
// each.  Writes items_out/n_out, pieces, reduces/n_reduce.
cudaError_t split_items(const Item *items_in, const int *n_in, int item_cap, const int *const *nbr,
                        const unsigned long long *total_pairs, long long warps_x_f, int t_floor, int *k, int *p,
                        int *r, void *scan_temp, Item *items_out, int *n_out, Piece *pieces, Reduce *reduces,
                        int *n_reduce, cudaStream_t st);
// Stable partition of items_in[0, n_items[0]) into items_out: heavy items first,
// then light ones (n_items[1] receives the number of heavy items).  flags:
// cap + 1 ints of scratch, scan_temp: scan_temp_bytes(cap + 1).
cudaError_t partition_light(const Item *items_in, int *n_items, int cap, int *flags, void *scan_temp,
                            Item *items_out, cudaStream_t st);
// Occupancy signature of a box: hist[b] (b = 0..kHistBins-1) = particles in
// cells whose occupancy n has floor(log2(n)) = b (the last bin takes the rest).
constexpr int kHistBins = 18;
cudaError_t occupancy_hist(const int *cell_start, int ncell, unsigned long long *hist, cudaStream_t st);
// *out = sum of the n values at ptrs[0..n)
cudaError_t sum_pair_counts(const unsigned long long *const *ptrs, int n, unsigned long long *out, cudaStream_t st);
cudaError_t reduce_partials(const BoxDev *boxes, const Reduce *reduces, const int *n_reduce, int max_reduce,
                            int adjoint, cudaStream_t st);
// sources summed directly in each cell's 125-cell neighbourhood into nbr
// (ncell ints; tmp, tmp2: ncell ints of scratch) and the pass's pair count
// sum_c n_c nbr_c into *pairs.  With n_min > 0 (cut-off mode) far cells of at
// least n_min particles are left out (they act through sub-cell moments), and
// nbr_all (ncell ints) receives the full 125-cell counts, which decide the lane
// cells (a lane item sums every source pair by pair, so it must not border a
// dense cell); with n_min = 0 nbr_all is not touched (may be null).
cudaError_t neighbour_pairs(const int *cell_start, int cpd, int64_t n_min, unsigned long long *pairs, int *tmp,
                            int *tmp2, int *nbr, int *nbr_all, cudaStream_t st);
// cut-off mode: dslot[c] = rank of cell c among the cells of >= n_min particles
// (-1 for the others), dense_cells[rank] = c, *n_dense = their number.
cudaError_t plan_dense_cells(const int *cell_start, int ncell, int64_t n_min, int *dslot, int *dense_cells,
                             int *n_dense, int *scratch_counts, int *scratch_offsets, void *scan_temp,
                             cudaStream_t st);

// ---- kick / drift (nf_step.cu) ----
// kick + drift of every particle into particle-id order: state_by_id[2 id] = new
// offset (w holds the new cell id's bits), state_by_id[2 id + 1] = new velocity;
// drift-limit violations counted in *cap_violations
cudaError_t kick_drift(const float4 *pos, const float4 *vel, const double *acc64, const uint32_t *cell_of,
                       const uint32_t *perm, double dt, double inv_w, int cpd, int n, float4 *state_by_id,
                       int *cap_violations, cudaStream_t st);
// sort keys (new cell ids) and values (ids) from kick_drift's output; counts += cell occupancies
cudaError_t drift_keys(const float4 *state_by_id, int n, uint32_t *keys, uint32_t *vals, int *counts, cudaStream_t st);

// cell multipoles (nf_multipole.cu)
// cut-off mode: the sub-cell moments of the dense cells (mpole, kCutSub * kCutWords floats per dense cell)
cudaError_t subcell_moments(const int *cell_start, const float4 *pos, const int *dense_cells, const int *n_dense,
                            int64_t dense_cap, float *mpole, int sm_count, cudaStream_t st);
int multipole_terms(int order);
cudaError_t cell_multipoles(const int *cell_start, int ncell, const float4 *pos, int order, double *out, int sm_count,
                            cudaStream_t st);

// time-step criteria (nf_step.cu)
size_t dt_temp_bytes(int ncell);
cudaError_t dt_reduce(const int *cell_start, int ncell, const float4 *vel, const double *acc64, void *temp,
                      cudaStream_t st);

}  // namespace nf
