// nf_api.cu -- the C ABI of include/nearfield.h: box state, input
// validation, data movement, and the order of device work for each call.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nearfield.h"
#include "nf_internal.cuh"

using nf::BoxDev;
using nf::Item;
using nf::PairShape;
using nf::Piece;
using nf::Reduce;

static_assert(nf::kProfWords == NF_PROFILE_WORDS, "the header's profile size is out of date");

// Source splitting aims at NF_BALANCE pieces of the pass per warp slot (32 per SM): no item much longer
// than pairs / (SMs x 32 x NF_BALANCE), so the queue's last wave leaves little idle time
#ifndef NF_BALANCE
#define NF_BALANCE 4
#endif

namespace {

thread_local std::string g_create_error;
std::atomic<uint64_t> g_generation{0};   // process-wide, so a reused box address never matches a stale plan

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct nf_box {
    // geometry (Section 2.1)
    int cpd = 0, R = 2, ncell = 0;
    double eps = 0, box = 0, w = 0, inv_w = 0;
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    int acc_mode = NF_ACC_COMPENSATED;
    int softening = NF_SPLINE;
    PairShape shape{8, 128, 0};
    nf::TilePolicy tiles = nf::kDefaultTiles;

    int64_t n = 0, cap = 0, item_cap = 0, split_cap = 0;   // split_cap: items after source splitting
    bool have_particles = false, have_forces = false;
    uint64_t generation = 0;          // changes with the particles
    uint64_t plan_gen = 0;            // changes with every re-plan (particles, cut-off, tiling)

    // particle state, storage order
    float4 *pos = nullptr, *vel = nullptr;
    double *acc64 = nullptr;
    float4 *acc32 = nullptr;          // FP32 output staging for host outputs
    float4 *cot = nullptr;            // cotangent staging
    uint32_t *keys[2] = {nullptr, nullptr}, *vals[2] = {nullptr, nullptr};
    int cur = 0;                      // keys[cur] = cell of each stored particle, vals[cur] = its id
    // per-id scratch used by binning and re-binning
    float4 *xq_by_id = nullptr;       // binned offsets by id (loads)
    float4 *state_by_id = nullptr;    // 2 float4 per id: drifted offset (key bits in w), velocity
    // cells
    int *cell_start = nullptr, *counts = nullptr, *offsets = nullptr;
    void *scan_tmp = nullptr, *radix_tmp = nullptr;
    size_t radix_tmp_bytes = 0;
    // plan: class-ordered items, then the same list with long items split into source pieces
    Item *items_raw = nullptr, *items = nullptr;
    int *n_raw = nullptr, *n_items = nullptr, *queue = nullptr, *err = nullptr;
    Piece *pieces = nullptr;
    Reduce *reduces = nullptr;
    int *n_reduce = nullptr;
    double *partials = nullptr;
    int *split_k = nullptr, *split_p = nullptr, *split_r = nullptr;
    void *split_scan = nullptr;
    int *nbr = nullptr;               // sources in each cell's neighbourhood
    // cut-off mode (dense far cells through sub-cell moments); cut_nmin = 0: exact
    int64_t cut_nmin = 0, dense_cap = 0;
    int *dslot = nullptr, *dense_cells = nullptr, *n_dense = nullptr;
    int *nbr_all = nullptr;           // full 125-cell counts (lane-item choice in cut-off mode)
    float *mpole = nullptr;
    const int **nbr_ptr = nullptr;    // device copy of nbr's address (the split planner reads boxes' tables)
    long long wf = 0;                 // 32 warps per SM x the balance factor NF_BALANCE
    int reduce_cap = 0;
    void *dt_tmp = nullptr;           // time-step reductions
    unsigned long long *pairs = nullptr;
    unsigned long long *hist = nullptr;   // occupancy signature for the tuner's cache key
    BoxDev *d_box = nullptr;
    BoxDev h_box{};                   // host mirror of *d_box
    bool box_dirty = true;
    // staging for host inputs
    DevBuf stage;
    // pointer-kind cache (avoids attribute queries in repeated calls)
    const void *last_ptr[4] = {nullptr, nullptr, nullptr, nullptr};
    bool last_dev[4] = {false, false, false, false};
    // profiling
    bool profile = false;
    bool profile_classes = false;
    unsigned long long *prof_cls = nullptr;   // nf::kProfWords per-class words of the pair kernel
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;

    std::string last_error;
};

namespace {

int fail(nf_t *nf, int code, const std::string &msg)
{
    if (nf) nf->last_error = msg;
    return code;
}

int cuda_fail(nf_t *nf, const char *what, cudaError_t e)
{
    return fail(nf, NF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NF_CK(call)                                                         \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return cuda_fail(nf, #call, e_);             \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// cached per call site (slot) so that repeated calls with the same pointer
// make no attribute query
bool is_device_cached(nf_t *nf, int slot, const void *p)
{
    if (p && p == nf->last_ptr[slot]) return nf->last_dev[slot];
    const bool d = is_device_ptr(p);
    nf->last_ptr[slot] = p;
    nf->last_dev[slot] = d;
    return d;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Allocation-failure injection for tests (nf_fail_allocations): after
// g_fail_skip more successful device allocations, the next g_fail_count fail.
std::mutex g_fail_mu;
int64_t g_fail_skip = 0, g_fail_count = 0;

bool injected_failure()
{
    std::lock_guard<std::mutex> lk(g_fail_mu);
    if (g_fail_count <= 0) return false;
    if (g_fail_skip > 0) {
        --g_fail_skip;
        return false;
    }
    --g_fail_count;
    return true;
}

template <class T>
int dalloc(nf_t *nf, T **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (injected_failure())
        return fail(nf, NF_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(nf, NF_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                       cudaGetErrorString(e));
    }
    return NF_OK;
}

template <class T>
void dfree(T *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

int ensure_stage(nf_t *nf, size_t bytes)
{
    if (nf->stage.bytes >= bytes) return NF_OK;
    if (nf->stage.p) cudaFree(nf->stage.p);
    nf->stage.p = nullptr;
    nf->stage.bytes = 0;
    int rc = dalloc(nf, &nf->stage.p, bytes);
    if (rc == NF_OK) nf->stage.bytes = bytes;
    return rc;
}

// a device copy of a caller input: the pointer itself if it is device memory
// (and 16-byte aligned), else the staging buffer after an async copy
int device_input(nf_t *nf, int slot, const void *src, size_t bytes, const void **out)
{
    if (is_device_cached(nf, slot, src) && aligned16(src)) {
        *out = src;
        return NF_OK;
    }
    int rc = ensure_stage(nf, bytes);
    if (rc != NF_OK) return rc;
    NF_CK(cudaMemcpyAsync(nf->stage.p, src, bytes, cudaMemcpyDefault, nf->stream));
    *out = nf->stage.p;
    return NF_OK;
}

void free_particles(nf_t *nf)
{
    dfree(nf->pos); dfree(nf->vel); dfree(nf->acc64); dfree(nf->acc32); dfree(nf->cot);
    for (int k = 0; k < 2; ++k) { dfree(nf->keys[k]); dfree(nf->vals[k]); }
    dfree(nf->xq_by_id); dfree(nf->state_by_id);
    dfree(nf->items); dfree(nf->items_raw); dfree(nf->pieces); dfree(nf->reduces); dfree(nf->partials);
    dfree(nf->split_k); dfree(nf->split_p); dfree(nf->split_r);
    if (nf->split_scan) cudaFree(nf->split_scan);
    nf->split_scan = nullptr;
    if (nf->radix_tmp) cudaFree(nf->radix_tmp);
    nf->radix_tmp = nullptr;
    nf->radix_tmp_bytes = 0;
    nf->cap = 0;
    nf->item_cap = 0;
}

int ensure_capacity(nf_t *nf, int64_t n)
{
    // items per cell <= 1 + n_c / 16 (full tiles and remainder pieces of >= 16 sinks, plus one)
    const int64_t item_cap = std::min<int64_t>(n, nf->ncell) + n / 16 + 16;
    if (n <= nf->cap && item_cap <= nf->item_cap && nf->pos) return NF_OK;
    // item indices and partial-sum slots are 32-bit on the device
    if (item_cap + 2 * nf->wf + 64 > INT32_MAX || static_cast<int64_t>(nf::kTile) * (2 * nf->wf + 64) + n > INT32_MAX)
        return fail(nf, NF_EINVAL, "too many particles for one box");
    cudaStreamSynchronize(nf->stream);
    // the old particles and plan go with their buffers: until a load completes the
    // box is empty, so no later call can launch on freed or half-built state
    nf->n = 0;
    nf->have_particles = false;
    nf->have_forces = false;
    nf->generation = ++g_generation;
    free_particles(nf);
    const int64_t c = n < 1 ? 1 : n;
    int rc = NF_OK;
    const size_t f4 = sizeof(float4) * static_cast<size_t>(c);
    const size_t u4 = sizeof(uint32_t) * static_cast<size_t>(c);
    if ((rc = dalloc(nf, &nf->pos, f4)) || (rc = dalloc(nf, &nf->vel, f4)) ||
        (rc = dalloc(nf, &nf->acc64, 3 * sizeof(double) * static_cast<size_t>(c))) ||
        (rc = dalloc(nf, &nf->keys[0], u4)) || (rc = dalloc(nf, &nf->keys[1], u4)) ||
        (rc = dalloc(nf, &nf->vals[0], u4)) || (rc = dalloc(nf, &nf->vals[1], u4)) ||
        (rc = dalloc(nf, &nf->xq_by_id, f4)) || (rc = dalloc(nf, &nf->state_by_id, 2 * f4))) {
        free_particles(nf);
        return rc;
    }
    // splitting adds fewer than 2 wf items and reduce records, and at most 128 (2 wf) + n partial slots;
    // items_raw holds the split list's partition too, so both lists have the split capacity
    const int64_t extra = 2 * nf->wf + 64;
    const size_t split_items_cap = static_cast<size_t>(item_cap + extra);
    const size_t slots = static_cast<size_t>(nf::kTile * extra + c);
    const size_t scan_ints = split_items_cap + 1;
    if ((rc = dalloc(nf, &nf->items_raw, sizeof(Item) * split_items_cap)) ||
        (rc = dalloc(nf, &nf->items, sizeof(Item) * split_items_cap)) ||
        (rc = dalloc(nf, &nf->pieces, sizeof(Piece) * split_items_cap)) ||
        (rc = dalloc(nf, &nf->reduces, sizeof(Reduce) * static_cast<size_t>(extra))) ||
        (rc = dalloc(nf, &nf->partials, 3 * sizeof(double) * slots)) ||
        (rc = dalloc(nf, &nf->split_k, sizeof(int) * scan_ints)) ||
        (rc = dalloc(nf, &nf->split_p, sizeof(int) * scan_ints)) ||
        (rc = dalloc(nf, &nf->split_r, sizeof(int) * scan_ints)) ||
        (rc = dalloc(nf, &nf->split_scan, nf::scan_temp_bytes(static_cast<int64_t>(scan_ints))))) {
        free_particles(nf);
        return rc;
    }
    nf->reduce_cap = static_cast<int>(extra);
    nf->radix_tmp_bytes = nf::radix_temp_bytes(c);
    if ((rc = dalloc(nf, &nf->radix_tmp, nf->radix_tmp_bytes))) {
        free_particles(nf);
        return rc;
    }
    nf->cap = c;
    nf->item_cap = item_cap;
    nf->split_cap = static_cast<int64_t>(split_items_cap);
    nf->box_dirty = true;
    return NF_OK;
}

int key_bits(int ncell)
{
    int b = 1;
    while (b < 32 && (1ll << b) < ncell) ++b;
    return b;
}

void fill_box_desc(nf_t *nf, BoxDev &b, float4 *acc_out, double *acc64, const float4 *cot)
{
    const double ec = nf->eps * nf->inv_w;   // eps in cell units
    b.pos = nf->pos;
    b.cell_start = nf->cell_start;
    b.acc_out = acc_out;
    b.acc64 = acc64;
    b.cot = cot;
    b.pieces = nf->pieces;
    b.partials = nf->partials;
    b.cpd = nf->cpd;
    b.n = static_cast<int>(nf->n);
    b.zcell = 1;   // every load and re-binning writes the cell's z index into pos[k].w
    b.a0 = static_cast<float>(10.0 / (ec * ec * ec));
    b.a1 = static_cast<float>(-15.0 / (ec * ec * ec * ec));
    b.a2 = static_cast<float>(6.0 / (ec * ec * ec * ec * ec));
    b.eps2 = static_cast<float>(ec * ec);
    b.acc_scale = nf->inv_w * nf->inv_w;
    b.grad_scale = nf->inv_w * nf->inv_w * nf->inv_w;
    b.dslot = nf->cut_nmin > 0 ? nf->dslot : nullptr;
    b.mpole = nf->cut_nmin > 0 ? nf->mpole : nullptr;
}

int upload_box(nf_t *nf, float4 *acc_out, double *acc64, const float4 *cot)
{
    BoxDev b{};
    fill_box_desc(nf, b, acc_out, acc64, cot);
    if (nf->box_dirty || std::memcmp(&b, &nf->h_box, sizeof(BoxDev)) != 0) {
        nf->h_box = b;
        NF_CK(cudaMemcpyAsync(nf->d_box, &nf->h_box, sizeof(BoxDev), cudaMemcpyHostToDevice, nf->stream));
        nf->box_dirty = false;
    }
    return NF_OK;
}

// cut-off mode buffers: slots for every cell, moments for up to n / n_min dense cells
int ensure_cutoff(nf_t *nf)
{
    int rc = NF_OK;
    if (!nf->dslot && ((rc = dalloc(nf, &nf->dslot, sizeof(int) * (static_cast<size_t>(nf->ncell) + 1))) ||
                       (rc = dalloc(nf, &nf->nbr_all, sizeof(int) * (static_cast<size_t>(nf->ncell) + 2))) ||
                       (rc = dalloc(nf, &nf->n_dense, sizeof(int) * 4)))) {
        dfree(nf->dslot);
        dfree(nf->nbr_all);
        dfree(nf->n_dense);
        return rc;
    }
    const int64_t need = nf->n / nf->cut_nmin + 1;
    if (need <= nf->dense_cap) return NF_OK;
    NF_CK(cudaStreamSynchronize(nf->stream));
    dfree(nf->dense_cells);
    dfree(nf->mpole);
    nf->dense_cap = 0;
    if ((rc = dalloc(nf, &nf->dense_cells, sizeof(int) * static_cast<size_t>(need))) ||
        (rc = dalloc(nf, &nf->mpole, sizeof(float) * nf::kCutSub * nf::kCutWords * static_cast<size_t>(need))))
        return rc;
    nf->dense_cap = need;
    return NF_OK;
}

// items of this box (all classes, largest first) into nf->items
int plan(nf_t *nf)
{
    // neighbourhood sizes and the pass's pair count, the items (occupancy classes, then
    // lane items), then the source split
    if (nf->cut_nmin > 0) {
        int rc = ensure_cutoff(nf);
        if (rc) return rc;
    }
    NF_CK(nf::neighbour_pairs(nf->cell_start, nf->cpd, nf->cut_nmin, nf->pairs, nf->counts, nf->offsets, nf->nbr,
                              nf->nbr_all, nf->stream));
    // lane cells are chosen on the full neighbourhood: the reduced one of cut-off mode
    // hides dense far cells, which a lane item would sum pair by pair
    const int *lane_nbr = nf->cut_nmin > 0 ? nf->nbr_all : nf->nbr;
    NF_CK(nf::zero_device_int(nf->n_raw, nf->stream));
    for (int cls = 0; cls < nf::kClasses; ++cls)
        NF_CK(nf::plan_items_class(nf->cell_start, lane_nbr, nf->ncell, 0, cls, nf->items_raw, nf->n_raw, nf->counts,
                                   nf->offsets, nf->scan_tmp, nf->tiles, nf->stream));
    NF_CK(nf::plan_lane_items(nf->cell_start, lane_nbr, nf->cpd, 0, nf->items_raw, nf->n_raw, nf->counts,
                              nf->offsets, nf->scan_tmp, nf->stream));
    NF_CK(nf::split_items(nf->items_raw, nf->n_raw, static_cast<int>(nf->item_cap), nf->nbr_ptr, nf->pairs, nf->wf,
                          nf->tiles.split_floor, nf->split_k, nf->split_p, nf->split_r, nf->split_scan, nf->items,
                          nf->n_items, nf->pieces, nf->reduces, nf->n_reduce, nf->stream));
    // heavy items first, light ones after
    NF_CK(nf::partition_light(nf->items, nf->n_items, static_cast<int>(nf->split_cap), nf->split_k, nf->split_scan,
                              nf->items_raw, nf->stream));
    std::swap(nf->items, nf->items_raw);
    if (nf->cut_nmin > 0)
        NF_CK(nf::plan_dense_cells(nf->cell_start, nf->ncell, nf->cut_nmin, nf->dslot, nf->dense_cells, nf->n_dense,
                                   nf->counts, nf->offsets, nf->scan_tmp, nf->stream));
    nf->plan_gen = ++g_generation;
    return NF_OK;
}

// counts[0..ncell] -> cell_start (exclusive scan), counts[ncell] must be 0
int counts_to_cell_start(nf_t *nf)
{
    NF_CK(nf::exclusive_scan_i32(nf->counts, nf->cell_start, static_cast<int64_t>(nf->ncell) + 1, nf->scan_tmp,
                                 nf->stream));
    return NF_OK;
}

// sort (keys[src], vals[src]) by key; gather positions (and velocities)
int sort_and_gather(nf_t *nf, int src, bool with_vel)
{
    int in_alt = 0;
    NF_CK(nf::radix_sort_pairs(nf->keys[src], nf->vals[src], nf->keys[1 - src], nf->vals[1 - src], nf->n,
                               key_bits(nf->ncell), nf->radix_tmp, &in_alt, nf->stream));
    nf->cur = in_alt ? 1 - src : src;
    if (with_vel)
        NF_CK(nf::gather_state(nf->vals[nf->cur], nf->keys[nf->cur], nf->cpd, nf->state_by_id, nf->pos, nf->vel,
                               static_cast<int>(nf->n), nf->stream));
    else
        NF_CK(nf::gather_sorted(nf->vals[nf->cur], nf->keys[nf->cur], nf->cpd, nf->xq_by_id, nullptr, nf->pos,
                                nf->vel, static_cast<int>(nf->n), nf->stream));
    return NF_OK;
}

int read_err(nf_t *nf, int *host)
{
    NF_CK(cudaMemcpyAsync(host, nf->err, sizeof(int), cudaMemcpyDeviceToHost, nf->stream));
    NF_CK(cudaStreamSynchronize(nf->stream));
    return NF_OK;
}

int launch_forces(nf_t *nf, const BoxDev *d_boxes, const Item *items, const int *n_items, int *queue, int adjoint)
{
    NF_CK(cudaMemsetAsync(queue, 0, sizeof(int), nf->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (nf->profile) {
        while (nf->ev.size() < nf->ev_used + 2) {
            cudaEvent_t e;
            NF_CK(cudaEventCreate(&e));
            nf->ev.push_back(e);
        }
        e0 = nf->ev[nf->ev_used];
        e1 = nf->ev[nf->ev_used + 1];
        nf->ev_used += 2;
        NF_CK(cudaEventRecord(e0, nf->stream));
    }
    // cut-off mode: this pass's sub-cell moments (inside the profiled interval)
    if (!adjoint && nf->cut_nmin > 0 && d_boxes == nf->d_box)
        NF_CK(nf::subcell_moments(nf->cell_start, nf->pos, nf->dense_cells, nf->n_dense, nf->dense_cap, nf->mpole,
                                  nf->sm_count, nf->stream));
    NF_CK(nf::launch_pair(d_boxes, items, n_items, queue, nf->acc_mode == NF_ACC_COMPENSATED, adjoint, nf->softening,
                          nf->shape, nf->sm_count, nf->stream, nf->profile_classes ? nf->prof_cls : nullptr));
    if (nf->profile) NF_CK(cudaEventRecord(e1, nf->stream));
    return NF_OK;
}

int check_box(nf_t *nf)
{
    if (!nf) return NF_EINVAL;
    cudaError_t e = cudaSetDevice(nf->device);
    if (e != cudaSuccess) return cuda_fail(nf, "cudaSetDevice", e);
    return NF_OK;
}

// widen / reformat state for nf_get_particles
__global__ void k_offsets64(const int *cs, int ncell, int64_t *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c <= ncell) out[c] = cs[c];
}
__global__ void k_counts32(const int *cs, int ncell, int32_t *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) out[c] = cs[c + 1] - cs[c];
}
__global__ void k_perm64(const uint32_t *v, int n, int64_t *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = v[k];
}
__global__ void k_pos_out(const float4 *pos, int n, float4 *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        const float4 p = pos[k];
        out[k] = make_float4(p.x, p.y, p.z, 0.f);
    }
}

inline int nblk(int64_t n) { return static_cast<int>((n + 255) / 256); }

// write `bytes` produced by `produce(dst_device)` into a caller pointer
template <class F>
int produce_out(nf_t *nf, void *dst, size_t bytes, F produce)
{
    if (is_device_ptr(dst) && aligned16(dst)) return produce(dst);
    int rc = ensure_stage(nf, bytes);
    if (rc != NF_OK) return rc;
    rc = produce(nf->stage.p);
    if (rc != NF_OK) return rc;
    NF_CK(cudaMemcpyAsync(dst, nf->stage.p, bytes, cudaMemcpyDefault, nf->stream));
    return NF_OK;
}

std::mutex g_tune_mu;
struct Tuned {
    PairShape shape;
    nf::TilePolicy tiles;
};
std::map<std::string, Tuned> g_tune_cache;
bool g_tune_file_loaded = false;

// Tuning results persist across processes in the text file named by
// NF_TUNE_CACHE (one "key<TAB>warps<TAB>stage<TAB>c4<TAB>c2<TAB>c1<TAB>split_floor"
// line per entry), if set.
void tune_file_load()
{
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char *path = std::getenv("NF_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        char *t1 = std::strchr(line, '\t');
        if (!t1) continue;
        *t1 = 0;
        Tuned t{};
        if (std::sscanf(t1 + 1, "%d\t%d\t%d\t%d\t%d\t%d", &t.shape.warps, &t.shape.stage, &t.tiles.c4, &t.tiles.c2,
                        &t.tiles.c1, &t.tiles.split_floor) == 6 &&
            t.shape.warps >= 1 && t.shape.warps <= 8 && (t.shape.stage == 128 || t.shape.stage == 256) &&
            nf::tile_policy_valid(t.tiles))
            g_tune_cache[line] = t;
    }
    std::fclose(f);
}

void tune_file_append(const std::string &key, const Tuned &t)
{
    const char *path = std::getenv("NF_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s\t%d\t%d\t%d\t%d\t%d\t%d\n", key.c_str(), t.shape.warps, t.shape.stage, t.tiles.c4, t.tiles.c2,
                 t.tiles.c1, t.tiles.split_floor);
    std::fclose(f);
}

}  // namespace

extern "C" {

int nf_create(int cpd, int R, double eps, double box, nf_t **out)
{
    if (!out) return NF_EINVAL;
    *out = nullptr;
    g_create_error.clear();
    if (R != 2) {
        g_create_error = "only R = 2 is supported";
        return NF_EINVAL;
    }
    if (cpd < 2 * R + 1 || static_cast<int64_t>(cpd) * cpd * cpd >= (1ll << 31) - 1) {
        g_create_error = "cpd must satisfy 2R+1 <= cpd and cpd^3 < 2^31";
        return NF_EINVAL;
    }
    if (!(box > 0) || !std::isfinite(box)) {
        g_create_error = "box must be positive and finite";
        return NF_EINVAL;
    }
    if (!(eps >= std::ldexp(box / cpd, -20)) || !(eps < box / cpd)) {
        g_create_error = "eps must satisfy 2^-20 box / cpd <= eps < box / cpd";
        return NF_EINVAL;
    }
    nf_t *nf = new (std::nothrow) nf_box();
    if (!nf) {
        g_create_error = "host allocation failed";
        return NF_ENOMEM;
    }
    nf->cpd = cpd;
    nf->R = R;
    nf->ncell = cpd * cpd * cpd;
    nf->eps = eps;
    nf->box = box;
    nf->w = box / cpd;
    nf->inv_w = static_cast<double>(cpd) / box;
    int rc = NF_OK;
    cudaError_t e = cudaGetDevice(&nf->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nf->sm_count, cudaDevAttrMultiProcessorCount, nf->device);
    if (e != cudaSuccess) {
        g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        cudaGetLastError();
        delete nf;
        return NF_ECUDA;
    }
    const size_t cells = sizeof(int) * (static_cast<size_t>(nf->ncell) + 2);
    if ((rc = dalloc(nf, &nf->cell_start, cells)) || (rc = dalloc(nf, &nf->counts, cells)) ||
        (rc = dalloc(nf, &nf->offsets, cells)) || (rc = dalloc(nf, &nf->nbr, cells)) ||
        (rc = dalloc(nf, &nf->scan_tmp, nf::scan_temp_bytes(static_cast<int64_t>(nf->ncell) + 2))) ||
        (rc = dalloc(nf, &nf->n_items, sizeof(int) * 4)) || (rc = dalloc(nf, &nf->queue, sizeof(int) * 4)) ||
        (rc = dalloc(nf, &nf->n_raw, sizeof(int) * 4)) || (rc = dalloc(nf, &nf->n_reduce, sizeof(int) * 4)) ||
        (rc = dalloc(nf, &nf->nbr_ptr, sizeof(int *))) ||
        (rc = dalloc(nf, &nf->dt_tmp, nf::dt_temp_bytes(nf->ncell))) ||
        (rc = dalloc(nf, &nf->err, sizeof(int) * 4)) || (rc = dalloc(nf, &nf->pairs, sizeof(unsigned long long))) ||
        (rc = dalloc(nf, &nf->d_box, sizeof(BoxDev)))) {
        g_create_error = nf->last_error;
        nf_destroy(nf);
        return rc;
    }
    nf->wf = static_cast<long long>(nf->sm_count) * 32 * NF_BALANCE;
    e = cudaMemset(nf->cell_start, 0, cells);
    if (e == cudaSuccess) e = cudaMemset(nf->n_items, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(nf->n_reduce, 0, sizeof(int) * 4);
    if (e == cudaSuccess) {
        const int *table = nf->nbr;
        e = cudaMemcpy(nf->nbr_ptr, &table, sizeof(table), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        g_create_error = std::string("device initialisation: ") + cudaGetErrorString(e);
        nf_destroy(nf);
        return NF_ECUDA;
    }
    *out = nf;
    return NF_OK;
}

void batch_forget(nf_t *nf);

void nf_destroy(nf_t *nf)
{
    if (!nf) return;
    batch_forget(nf);
    cudaSetDevice(nf->device);
    cudaStreamSynchronize(nf->stream);
    free_particles(nf);
    dfree(nf->cell_start); dfree(nf->counts); dfree(nf->offsets); dfree(nf->nbr);
    dfree(nf->dslot); dfree(nf->dense_cells); dfree(nf->n_dense); dfree(nf->mpole); dfree(nf->nbr_all);
    if (nf->scan_tmp) cudaFree(nf->scan_tmp);
    dfree(nf->n_items); dfree(nf->queue); dfree(nf->err); dfree(nf->pairs); dfree(nf->d_box);
    dfree(nf->n_raw); dfree(nf->n_reduce); dfree(nf->nbr_ptr); dfree(nf->hist);
    if (nf->dt_tmp) cudaFree(nf->dt_tmp);
    dfree(nf->prof_cls);
    if (nf->stage.p) cudaFree(nf->stage.p);
    for (cudaEvent_t e : nf->ev) cudaEventDestroy(e);
    delete nf;
}

const char *nf_last_error(const nf_t *nf)
{
    if (!nf) return g_create_error.c_str();
    return nf->last_error.c_str();
}

int nf_set_stream(nf_t *nf, void *stream)
{
    if (!nf) return NF_EINVAL;
    nf->stream = static_cast<cudaStream_t>(stream);
    return NF_OK;
}

int nf_set_accumulation(nf_t *nf, int mode)
{
    if (!nf) return NF_EINVAL;
    if (mode != NF_ACC_COMPENSATED && mode != NF_ACC_PLAIN) return fail(nf, NF_EINVAL, "unknown accumulation mode");
    nf->acc_mode = mode;
    return NF_OK;
}

int nf_set_softening(nf_t *nf, int mode)
{
    if (!nf) return NF_EINVAL;
    if (mode != NF_SPLINE && mode != NF_PLUMMER) return fail(nf, NF_EINVAL, "unknown softening mode");
    if (mode != NF_SPLINE && nf->cut_nmin > 0)
        return fail(nf, NF_ESTATE, "the cut-off mode applies to the spline law only; set it to 0 first");
    nf->softening = mode;
    return NF_OK;
}

int nf_set_cutoff(nf_t *nf, int64_t n_min)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (n_min < 0 || (n_min > 0 && n_min < nf::kCutMinN))
        return fail(nf, NF_EINVAL, "n_min must be 0 (exact) or at least " + std::to_string(nf::kCutMinN));
    if (n_min > 0 && nf->softening != NF_SPLINE)
        return fail(nf, NF_ESTATE, "the cut-off mode applies to the spline law only");
    if (n_min == nf->cut_nmin) return NF_OK;
    nf->cut_nmin = n_min;
    nf->box_dirty = true;
    if (nf->have_particles) {
        if ((rc = plan(nf))) {
            if (rc == NF_ENOMEM) {
                // the moment buffers could not be had: back to the exact near field
                const std::string why = nf->last_error;
                nf->cut_nmin = 0;
                if (plan(nf) == NF_OK) cudaStreamSynchronize(nf->stream);
                nf->last_error = why + " (the box stays in the exact mode)";
            }
            return rc;
        }
        NF_CK(cudaStreamSynchronize(nf->stream));
    }
    return NF_OK;
}

double nf_spline_eps_from_plummer(double eps_plummer) { return 2.16 * eps_plummer; }

int nf_bin_particles(nf_t *nf, const double *xyz, int64_t n)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (n < 0 || n >= (1ll << 31) - 1) return fail(nf, NF_EINVAL, "n must satisfy 0 <= n < 2^31 - 1");
    if (n > 0 && !xyz) return fail(nf, NF_EINVAL, "xyz is NULL");
    if ((rc = ensure_capacity(nf, n))) return rc;
    const double *dx = nullptr;
    if (n > 0 && (rc = device_input(nf, 0, xyz, sizeof(double) * 3 * static_cast<size_t>(n),
                                    reinterpret_cast<const void **>(&dx))))
        return rc;
    NF_CK(cudaMemsetAsync(nf->counts, 0, sizeof(int) * (static_cast<size_t>(nf->ncell) + 2), nf->stream));
    NF_CK(cudaMemsetAsync(nf->err, 0, sizeof(int), nf->stream));
    const int src = 1 - nf->cur;   // keep the live state untouched until the input is known to be valid
    NF_CK(nf::bin_global(dx, static_cast<int>(n), nf->cpd, nf->inv_w, nf->keys[src], nf->vals[src], nf->xq_by_id,
                         nf->counts, nf->err, nf->stream));
    int herr = 0;
    if ((rc = read_err(nf, &herr))) return rc;
    if (herr) return fail(nf, NF_EINVAL, "non-finite or out-of-range position");
    nf->n = n;
    nf->have_particles = false;
    nf->have_forces = false;
    if (n > 0) {
        if ((rc = sort_and_gather(nf, src, false))) return rc;
    }
    if ((rc = counts_to_cell_start(nf))) return rc;
    NF_CK(cudaMemsetAsync(nf->vel, 0, sizeof(float4) * static_cast<size_t>(n < 1 ? 1 : n), nf->stream));
    if ((rc = plan(nf))) return rc;
    nf->box_dirty = true;
    nf->generation = ++g_generation;
    nf->have_particles = true;
    NF_CK(cudaStreamSynchronize(nf->stream));
    return NF_OK;
}

int nf_set_particles(nf_t *nf, const int64_t *cell_offsets, const int32_t *counts, const float *pos, int64_t n)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (n < 0 || n >= (1ll << 31) - 1) return fail(nf, NF_EINVAL, "n must satisfy 0 <= n < 2^31 - 1");
    if (!cell_offsets || !counts || (n > 0 && !pos)) return fail(nf, NF_EINVAL, "NULL input");
    if ((rc = ensure_capacity(nf, n))) return rc;
    const size_t ob = sizeof(int64_t) * (static_cast<size_t>(nf->ncell) + 1);
    const size_t cb = sizeof(int32_t) * static_cast<size_t>(nf->ncell);
    const size_t pb = sizeof(float4) * static_cast<size_t>(n);
    // stage all three inputs in one device buffer (each part 16-byte aligned)
    const size_t o_off = 0, c_off = (ob + 15) & ~size_t(15), p_off = c_off + ((cb + 15) & ~size_t(15));
    if ((rc = ensure_stage(nf, p_off + pb + 16))) return rc;
    char *sp = static_cast<char *>(nf->stage.p);
    NF_CK(cudaMemcpyAsync(sp + o_off, cell_offsets, ob, cudaMemcpyDefault, nf->stream));
    NF_CK(cudaMemcpyAsync(sp + c_off, counts, cb, cudaMemcpyDefault, nf->stream));
    if (n > 0) NF_CK(cudaMemcpyAsync(sp + p_off, pos, pb, cudaMemcpyDefault, nf->stream));
    NF_CK(cudaMemsetAsync(nf->err, 0, sizeof(int), nf->stream));
    // validated values go to scratch (offsets -> cell starts, xq_by_id -> positions)
    NF_CK(nf::validate_loaded(reinterpret_cast<const int64_t *>(sp + o_off), reinterpret_cast<const int32_t *>(sp + c_off),
                              reinterpret_cast<const float4 *>(sp + p_off), nf->ncell, static_cast<int>(n), nf->offsets,
                              nf->xq_by_id, nf->err, nf->stream));
    int herr = 0;
    if ((rc = read_err(nf, &herr))) return rc;
    if (herr) {
        std::string why;
        if (herr & 3) why += " offsets do not start at 0 / end at n;";
        if (herr & 4) why += " negative count;";
        if (herr & 8) why += " offsets are not the scan of counts;";
        if (herr & 16) why += " offset out of range;";
        if (herr & 32) why += " position non-finite or outside the cell;";
        return fail(nf, NF_EINVAL, "nf_set_particles:" + why);
    }
    std::swap(nf->cell_start, nf->offsets);
    std::swap(nf->pos, nf->xq_by_id);
    nf->n = n;
    NF_CK(nf::iota_u32(nf->vals[nf->cur], static_cast<int>(n), nf->stream));
    NF_CK(nf::fill_cell_ids(nf->cell_start, nf->ncell, static_cast<int>(n), nf->keys[nf->cur], nf->pos, nf->cpd,
                            nf->stream));
    NF_CK(cudaMemsetAsync(nf->vel, 0, sizeof(float4) * static_cast<size_t>(n < 1 ? 1 : n), nf->stream));
    if ((rc = plan(nf))) return rc;
    nf->box_dirty = true;
    nf->generation = ++g_generation;
    nf->have_particles = true;
    nf->have_forces = false;
    NF_CK(cudaStreamSynchronize(nf->stream));
    return NF_OK;
}

int nf_set_velocities(nf_t *nf, const float *vel)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!nf->have_particles) return fail(nf, NF_ESTATE, "no particles loaded");
    if (nf->n == 0) return NF_OK;
    if (!vel) return fail(nf, NF_EINVAL, "vel is NULL");
    NF_CK(cudaMemcpyAsync(nf->vel, vel, sizeof(float4) * static_cast<size_t>(nf->n), cudaMemcpyDefault, nf->stream));
    return NF_OK;
}

int nf_get_particles(nf_t *nf, int64_t *cell_offsets, int32_t *counts, float *pos, float *vel, int64_t *perm)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!nf->have_particles) return fail(nf, NF_ESTATE, "no particles loaded");
    const int ncell = nf->ncell;
    const int n = static_cast<int>(nf->n);
    cudaStream_t st = nf->stream;
    if (cell_offsets) {
        rc = produce_out(nf, cell_offsets, sizeof(int64_t) * (static_cast<size_t>(ncell) + 1), [&](void *d) -> int {
            k_offsets64<<<nblk(static_cast<int64_t>(ncell) + 1), 256, 0, st>>>(nf->cell_start, ncell,
                                                                                static_cast<int64_t *>(d));
            NF_CK(cudaGetLastError());
            return NF_OK;
        });
        if (rc) return rc;
    }
    if (counts) {
        rc = produce_out(nf, counts, sizeof(int32_t) * static_cast<size_t>(ncell), [&](void *d) -> int {
            k_counts32<<<nblk(ncell), 256, 0, st>>>(nf->cell_start, ncell, static_cast<int32_t *>(d));
            NF_CK(cudaGetLastError());
            return NF_OK;
        });
        if (rc) return rc;
    }
    // the stored w holds the cell's z index; the caller gets the documented pad 0
    const bool pos_on_host = pos && n > 0 && !(is_device_ptr(pos) && aligned16(pos));
    if (pos && n > 0) {
        if (pos_on_host) {
            NF_CK(cudaMemcpyAsync(pos, nf->pos, sizeof(float4) * n, cudaMemcpyDefault, st));
        } else {
            k_pos_out<<<nblk(n), 256, 0, st>>>(nf->pos, n, reinterpret_cast<float4 *>(pos));
            NF_CK(cudaGetLastError());
        }
    }
    if (vel && n > 0) NF_CK(cudaMemcpyAsync(vel, nf->vel, sizeof(float4) * n, cudaMemcpyDefault, st));
    if (perm && n > 0) {
        rc = produce_out(nf, perm, sizeof(int64_t) * n, [&](void *d) -> int {
            k_perm64<<<nblk(n), 256, 0, st>>>(nf->vals[nf->cur], n, static_cast<int64_t *>(d));
            NF_CK(cudaGetLastError());
            return NF_OK;
        });
        if (rc) return rc;
    }
    NF_CK(cudaStreamSynchronize(st));
    if (pos_on_host)
        for (int64_t k = 0; k < n; ++k) pos[4 * k + 3] = 0.f;
    return NF_OK;
}

int nf_num_particles(const nf_t *nf, int64_t *n)
{
    if (!nf || !n) return NF_EINVAL;
    *n = nf->n;
    return NF_OK;
}

int nf_generation(const nf_t *nf, uint64_t *gen)
{
    if (!nf || !gen) return NF_EINVAL;
    *gen = nf->generation;
    return NF_OK;
}

int nf_fail_allocations(int64_t skip, int64_t count)
{
    if (skip < 0 || count < 0) return NF_EINVAL;
    std::lock_guard<std::mutex> lk(g_fail_mu);
    g_fail_skip = skip;
    g_fail_count = count;
    return NF_OK;
}

int nf_pair_count(nf_t *nf, int64_t *pairs)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!pairs) return fail(nf, NF_EINVAL, "pairs is NULL");
    if (!nf->have_particles) return fail(nf, NF_ESTATE, "no particles loaded");
    // every change of the particles or of the cut-off re-plans, and the plan keeps its pair
    // count in nf->pairs, so the count is read, not recomputed
    unsigned long long h = 0;
    NF_CK(cudaMemcpyAsync(&h, nf->pairs, sizeof(h), cudaMemcpyDeviceToHost, nf->stream));
    NF_CK(cudaStreamSynchronize(nf->stream));
    *pairs = static_cast<int64_t>(h);
    return NF_OK;
}

int nf_forces(nf_t *nf, float *acc)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!nf->have_particles) return fail(nf, NF_ESTATE, "no particles loaded");
    const size_t bytes = sizeof(float4) * static_cast<size_t>(nf->n);
    float4 *out = nullptr;
    bool copy_back = false;
    if (acc && nf->n > 0) {
        if (is_device_cached(nf, 1, acc) && aligned16(acc)) {
            out = reinterpret_cast<float4 *>(acc);
        } else {
            if (!nf->acc32 && (rc = dalloc(nf, &nf->acc32, sizeof(float4) * static_cast<size_t>(nf->cap)))) return rc;
            out = nf->acc32;
            copy_back = true;
        }
    }
    if ((rc = upload_box(nf, out, nf->acc64, nullptr))) return rc;
    if (nf->n > 0) {
        if ((rc = launch_forces(nf, nf->d_box, nf->items, nf->n_items, nf->queue, 0))) return rc;
        NF_CK(nf::reduce_partials(nf->d_box, nf->reduces, nf->n_reduce, nf->reduce_cap, 0, nf->stream));
    }
    if (copy_back) NF_CK(cudaMemcpyAsync(acc, nf->acc32, bytes, cudaMemcpyDefault, nf->stream));
    nf->have_forces = true;
    return NF_OK;
}

int nf_get_forces64(nf_t *nf, double *acc)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!nf->have_forces) return fail(nf, NF_ESTATE, "no forces computed");
    if (!acc) return fail(nf, NF_EINVAL, "acc is NULL");
    if (nf->n > 0)
        NF_CK(cudaMemcpyAsync(acc, nf->acc64, 3 * sizeof(double) * static_cast<size_t>(nf->n), cudaMemcpyDefault,
                              nf->stream));
    return NF_OK;
}

int nf_vjp(nf_t *nf, const float *w, float *grad)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!nf->have_particles) return fail(nf, NF_ESTATE, "no particles loaded");
    if (nf->cut_nmin > 0) return fail(nf, NF_ESTATE, "the adjoint is exact-only; set the cut-off to 0 first");
    if (nf->n == 0) return NF_OK;
    if (!w || !grad) return fail(nf, NF_EINVAL, "NULL input");
    const size_t bytes = sizeof(float4) * static_cast<size_t>(nf->n);
    const float4 *cot = nullptr;
    if (is_device_cached(nf, 2, w) && aligned16(w)) {
        cot = reinterpret_cast<const float4 *>(w);
    } else {
        if (!nf->cot && (rc = dalloc(nf, &nf->cot, sizeof(float4) * static_cast<size_t>(nf->cap)))) return rc;
        NF_CK(cudaMemcpyAsync(nf->cot, w, bytes, cudaMemcpyDefault, nf->stream));
        cot = nf->cot;
    }
    float4 *out = nullptr;
    bool copy_back = false;
    if (is_device_cached(nf, 3, grad) && aligned16(grad)) {
        out = reinterpret_cast<float4 *>(grad);
    } else {
        if (!nf->acc32 && (rc = dalloc(nf, &nf->acc32, sizeof(float4) * static_cast<size_t>(nf->cap)))) return rc;
        out = nf->acc32;
        copy_back = true;
    }
    if ((rc = upload_box(nf, out, nullptr, cot))) return rc;
    if ((rc = launch_forces(nf, nf->d_box, nf->items, nf->n_items, nf->queue, 1))) return rc;
    NF_CK(nf::reduce_partials(nf->d_box, nf->reduces, nf->n_reduce, nf->reduce_cap, 1, nf->stream));
    if (copy_back) NF_CK(cudaMemcpyAsync(grad, nf->acc32, bytes, cudaMemcpyDefault, nf->stream));
    return NF_OK;
}

int nf_kick_drift(nf_t *nf, double dt)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!nf->have_forces) return fail(nf, NF_ESTATE, "nf_kick_drift needs a previous nf_forces");
    if (!std::isfinite(dt)) return fail(nf, NF_EINVAL, "dt must be finite");
    const int n = static_cast<int>(nf->n);
    if (n == 0) return NF_OK;
    NF_CK(cudaMemsetAsync(nf->err, 0, sizeof(int), nf->stream));
    // the new state goes to scratch (state_by_id), so a refused step changes nothing
    NF_CK(nf::kick_drift(nf->pos, nf->vel, nf->acc64, nf->keys[nf->cur], nf->vals[nf->cur], dt, nf->inv_w, nf->cpd,
                         n, nf->state_by_id, nf->err, nf->stream));
    int viol = 0;
    if ((rc = read_err(nf, &viol))) return rc;
    if (viol)
        return fail(nf, NF_EINVAL, std::to_string(viol) + " particles would drift more than 0.8 cell widths");
    const int src = 1 - nf->cur;
    NF_CK(cudaMemsetAsync(nf->counts, 0, sizeof(int) * (static_cast<size_t>(nf->ncell) + 2), nf->stream));
    NF_CK(nf::drift_keys(nf->state_by_id, n, nf->keys[src], nf->vals[src], nf->counts, nf->stream));
    if ((rc = sort_and_gather(nf, src, true))) return rc;
    if ((rc = counts_to_cell_start(nf))) return rc;
    if ((rc = plan(nf))) return rc;
    nf->box_dirty = true;
    nf->generation = ++g_generation;
    nf->have_forces = false;
    NF_CK(cudaStreamSynchronize(nf->stream));
    return NF_OK;
}

int nf_choose_dt(nf_t *nf, double eta, double dt_max, double *dt, double *parts)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!dt) return fail(nf, NF_EINVAL, "dt is NULL");
    if (!(eta > 0) || !(dt_max > 0)) return fail(nf, NF_EINVAL, "eta and dt_max must be positive");
    if (!nf->have_forces) return fail(nf, NF_ESTATE, "nf_choose_dt needs a previous nf_forces");
    double h[4] = {INFINITY, 0.0, 0.0, 0.0};
    if (nf->n > 0) {
        NF_CK(nf::dt_reduce(nf->cell_start, nf->ncell, nf->vel, nf->acc64, nf->dt_tmp, nf->stream));
        NF_CK(cudaMemcpyAsync(h, nf->dt_tmp, sizeof(h), cudaMemcpyDeviceToHost, nf->stream));
        NF_CK(cudaStreamSynchronize(nf->stream));
    }
    // Section 4.2.1: eta times the larger of (smallest cell v_rms / a_max) and the global v_rms / a_max;
    // a drift of at most 0.8 cell widths; and a cap (TimeStepDlna in an expanding box)
    const double v_rms = nf->n > 0 ? std::sqrt(h[1] / static_cast<double>(nf->n)) : 0.0;
    const double global = h[2] > 0 ? v_rms / h[2] : INFINITY;
    const double dt_acc = eta * std::max(h[0], global);
    const double dt_drift = h[3] > 0 ? 0.8 * nf->w / h[3] : INFINITY;
    *dt = std::min(dt_max, std::min(dt_acc, dt_drift));
    if (parts) {
        parts[0] = dt_acc;
        parts[1] = dt_drift;
        parts[2] = dt_max;
    }
    return NF_OK;
}

int nf_multipoles(nf_t *nf, int order, double *out)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (order < 0 || order > 8) return fail(nf, NF_EINVAL, "multipole order must be 0..8");
    if (!out) return fail(nf, NF_EINVAL, "out is NULL");
    if (!nf->have_particles) return fail(nf, NF_ESTATE, "no particles loaded");
    const size_t bytes = sizeof(double) * static_cast<size_t>(nf->ncell) * nf::multipole_terms(order);
    return produce_out(nf, out, bytes, [&](void *d) -> int {
        NF_CK(nf::cell_multipoles(nf->cell_start, nf->ncell, nf->pos, order, static_cast<double *>(d), nf->sm_count,
                                  nf->stream));
        return NF_OK;
    });
}

int nf_profile(nf_t *nf, int enable)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (enable < 0 || enable > 2) return fail(nf, NF_EINVAL, "enable must be 0, 1 or 2");
    if (enable == 2 && !nf->prof_cls) {
        if ((rc = dalloc(nf, &nf->prof_cls, sizeof(unsigned long long) * nf::kProfWords))) return rc;
        NF_CK(cudaMemsetAsync(nf->prof_cls, 0, sizeof(unsigned long long) * nf::kProfWords, nf->stream));
    }
    nf->profile = enable != 0;
    nf->profile_classes = enable == 2;
    return NF_OK;
}

int nf_profile_classes(nf_t *nf, uint64_t *out, int n_out)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!out || n_out < nf::kProfWords) return fail(nf, NF_EINVAL, "out needs NF_PROFILE_WORDS words");
    if (!nf->prof_cls) {
        std::memset(out, 0, sizeof(uint64_t) * nf::kProfWords);
        return NF_OK;
    }
    NF_CK(cudaMemcpyAsync(out, nf->prof_cls, sizeof(uint64_t) * nf::kProfWords, cudaMemcpyDeviceToHost, nf->stream));
    NF_CK(cudaMemsetAsync(nf->prof_cls, 0, sizeof(uint64_t) * nf::kProfWords, nf->stream));
    NF_CK(cudaStreamSynchronize(nf->stream));
    return NF_OK;
}

int nf_profile_read(nf_t *nf, int64_t *launches, double *ms)
{
    int rc = check_box(nf);
    if (rc) return rc;
    NF_CK(cudaStreamSynchronize(nf->stream));
    double total = 0;
    for (size_t k = 0; k + 1 < nf->ev_used; k += 2) {
        float t = 0;
        NF_CK(cudaEventElapsedTime(&t, nf->ev[k], nf->ev[k + 1]));
        total += t;
    }
    if (launches) *launches = static_cast<int64_t>(nf->ev_used / 2);
    if (ms) *ms = total;
    nf->ev_used = 0;
    return NF_OK;
}

int nf_set_shape(nf_t *nf, int warps, int stage)
{
    if (!nf) return NF_EINVAL;
    if (warps < 1 || warps > 8 || (stage != 128 && stage != 256))
        return fail(nf, NF_EINVAL, "warps must be 1..8 and stage 128 or 256");
    nf->shape.warps = warps;
    nf->shape.stage = stage;
    return NF_OK;
}

int nf_set_tiling(nf_t *nf, int c4, int c2, int c1, int split_floor)
{
    int rc = check_box(nf);
    if (rc) return rc;
    const nf::TilePolicy t{c4, c2, c1, split_floor};
    if (!nf::tile_policy_valid(t))
        return fail(nf, NF_EINVAL, "tiling needs 64 <= c4 <= 128, 32 <= c2 <= 64, 16 <= c1 <= 32, "
                                   "128 <= split_floor <= 2^20");
    nf->tiles = t;
    if (nf->have_particles) {
        if ((rc = plan(nf))) return rc;
        NF_CK(cudaStreamSynchronize(nf->stream));
    }
    return NF_OK;
}

int nf_get_tuning(const nf_t *nf, int32_t *out6)
{
    if (!nf || !out6) return NF_EINVAL;
    out6[0] = nf->shape.warps;
    out6[1] = nf->shape.stage;
    out6[2] = nf->tiles.c4;
    out6[3] = nf->tiles.c2;
    out6[4] = nf->tiles.c1;
    out6[5] = nf->tiles.split_floor;
    return NF_OK;
}

}  // extern "C"

namespace {

// ms per launch of the pair kernel on the current plan and shape (1 untimed + 2 timed launches)
int time_pair(nf_t *nf, cudaEvent_t a, cudaEvent_t b, float *ms)
{
    int rc;
    if ((rc = launch_forces(nf, nf->d_box, nf->items, nf->n_items, nf->queue, 0))) return rc;
    NF_CK(cudaEventRecord(a, nf->stream));
    for (int r = 0; r < 2; ++r)
        if ((rc = launch_forces(nf, nf->d_box, nf->items, nf->n_items, nf->queue, 0))) return rc;
    NF_CK(cudaEventRecord(b, nf->stream));
    NF_CK(cudaEventSynchronize(b));
    float t = 0;
    NF_CK(cudaEventElapsedTime(&t, a, b));
    *ms = t / 2;
    return NF_OK;
}

// Cache key of a box: device, accumulation, law, cut-off, size class and its occupancy
// signature (the share of particles in cells of occupancy 2^b..2^(b+1)-1, b = 0..17, in
// sixteenths), so boxes with different clustering are tuned separately.
int tune_key(nf_t *nf, std::string *key)
{
    cudaDeviceProp prop;
    NF_CK(cudaGetDeviceProperties(&prop, nf->device));
    int rc;
    if (!nf->hist && (rc = dalloc(nf, &nf->hist, sizeof(unsigned long long) * nf::kHistBins))) return rc;
    unsigned long long h[nf::kHistBins] = {};
    NF_CK(nf::occupancy_hist(nf->cell_start, nf->ncell, nf->hist, nf->stream));
    NF_CK(cudaMemcpyAsync(h, nf->hist, sizeof(h), cudaMemcpyDeviceToHost, nf->stream));
    NF_CK(cudaStreamSynchronize(nf->stream));
    std::string sig;
    const double n = nf->n > 0 ? static_cast<double>(nf->n) : 1.0;
    for (int b = 0; b < nf::kHistBins; ++b) sig += "0123456789abcdefg"[static_cast<int>(std::lround(16.0 * h[b] / n))];
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= nf->n) ++lg;
    char k[256];
    std::snprintf(k, sizeof(k), "%s|acc=%d|soft=%d|cut=%lld|log2n=%d|occ=%s", prop.name, nf->acc_mode, nf->softening,
                  static_cast<long long>(nf->cut_nmin), lg, sig.c_str());
    *key = k;
    return NF_OK;
}

}  // namespace

extern "C" {

int nf_tune(nf_t *nf, char *report, int report_len)
{
    int rc = check_box(nf);
    if (rc) return rc;
    if (!nf->have_particles) return fail(nf, NF_ESTATE, "no particles loaded");
    std::string key, summary;
    if ((rc = tune_key(nf, &key))) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_file_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            nf->shape = it->second.shape;
            nf->tiles = it->second.tiles;
            summary = "cached";
        }
    }
    if (!summary.empty()) {
        if ((rc = plan(nf))) return rc;
    } else if (nf->n > 0) {
        // 1. the sink tiling (remainder decomposition) and the split floor at the default launch
        // shape, 2. the launch shape at the best tiling
        const nf::TilePolicy tcand[] = {nf::kDefaultTiles,  {96, 64, 32, 1024}, {80, 48, 24, 1024},
                                        {112, 40, 20, 1024}, {96, 40, 18, 512},  {96, 40, 18, 2048}};
        const PairShape scand[] = {{8, 128, 0}, {4, 128, 0}, {8, 256, 0}, {4, 256, 0}, {2, 128, 0}};
        cudaEvent_t a, b;
        NF_CK(cudaEventCreate(&a));
        NF_CK(cudaEventCreate(&b));
        const bool prof = nf->profile;
        nf->profile = false;
        Tuned best{PairShape{8, 128, 0}, nf::kDefaultTiles};
        float best_ms = 1e30f;
        char part[128];
        if ((rc = upload_box(nf, nullptr, nf->acc64, nullptr))) return rc;
        nf->shape = best.shape;
        for (const nf::TilePolicy &t : tcand) {
            nf->tiles = t;
            float ms = 0;
            if ((rc = plan(nf)) || (rc = time_pair(nf, a, b, &ms))) return rc;
            std::snprintf(part, sizeof(part), "tiles %d/%d/%d/%d:%.3fms ", t.c4, t.c2, t.c1, t.split_floor, ms);
            summary += part;
            if (ms < best_ms) {
                best_ms = ms;
                best.tiles = t;
            }
        }
        nf->tiles = best.tiles;
        if ((rc = plan(nf))) return rc;
        best_ms = 1e30f;
        for (const PairShape &sh : scand) {
            if (nf::pair_max_blocks_per_sm(nf->acc_mode == NF_ACC_COMPENSATED, 0, nf->softening, sh) < 1) continue;
            nf->shape = sh;
            float ms = 0;
            if ((rc = time_pair(nf, a, b, &ms))) return rc;
            std::snprintf(part, sizeof(part), "shape %dx%d:%.3fms ", sh.warps, sh.stage, ms);
            summary += part;
            if (ms < best_ms) {
                best_ms = ms;
                best.shape = sh;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        nf->profile = prof;
        nf->shape = best.shape;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
        tune_file_append(key, best);
        std::snprintf(part, sizeof(part), "-> %dx%d tiles %d/%d/%d/%d", best.shape.warps, best.shape.stage,
                      best.tiles.c4, best.tiles.c2, best.tiles.c1, best.tiles.split_floor);
        summary += part;
    }
    // leave one complete force pass (partials reduced) in the box's FP64 sums
    if (nf->n > 0) {
        if ((rc = upload_box(nf, nullptr, nf->acc64, nullptr)) ||
            (rc = launch_forces(nf, nf->d_box, nf->items, nf->n_items, nf->queue, 0)))
            return rc;
        NF_CK(nf::reduce_partials(nf->d_box, nf->reduces, nf->n_reduce, nf->reduce_cap, 0, nf->stream));
        NF_CK(cudaStreamSynchronize(nf->stream));
    }
    nf->have_forces = true;
    if (report && report_len > 0) std::snprintf(report, static_cast<size_t>(report_len), "%s", summary.c_str());
    return NF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batched

namespace {

// The combined plan of one set of boxes: class-major items over all boxes,
// split into source pieces like a single box's plan, with its own partial
// sums (every box descriptor of the batch points at them).
struct Batch {
    std::vector<nf_t *> boxes;
    std::vector<uint64_t> gens;
    std::vector<BoxDev> h_desc;
    BoxDev *d_desc = nullptr;
    Item *items_raw = nullptr, *items = nullptr;
    Piece *pieces = nullptr;
    Reduce *reduces = nullptr;
    double *partials = nullptr;
    int *split_k = nullptr, *split_p = nullptr, *split_r = nullptr;
    void *split_scan = nullptr;
    const int **nbr_ptrs = nullptr;
    const unsigned long long **pair_ptrs = nullptr;
    unsigned long long *total = nullptr;
    int64_t raw_cap = 0, n_cap = 0, split_cap = 0;
    int nbox_cap = 0, reduce_cap = 0;
    int *n_raw = nullptr, *n_items = nullptr, *n_reduce = nullptr, *queue = nullptr;
    int device = -1;
};

std::mutex g_batch_mu;
Batch g_batch;

}  // namespace

void batch_forget(nf_t *nf)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (nf_t *b : g_batch.boxes)
        if (b == nf) {
            g_batch.boxes.clear();
            g_batch.gens.clear();
            return;
        }
}

namespace {

void batch_release(Batch &b)
{
    void *ps[] = {b.d_desc, b.items_raw, b.items, b.pieces, b.reduces, b.partials, b.split_k, b.split_p,
                  b.split_r, b.split_scan, b.nbr_ptrs, b.pair_ptrs, b.total, b.n_raw, b.n_items, b.n_reduce, b.queue};
    for (void *q : ps)
        if (q) cudaFree(q);
    b = Batch();
}

int batch_alloc(nf_t *nf, Batch &B, int nbox, int64_t raw_cap, int64_t n_total)
{
    batch_release(B);
    const int64_t extra = 2 * nf->wf + 64;
    const size_t items_cap = static_cast<size_t>(raw_cap + extra);
    const size_t scan_ints = items_cap + 1;
    const size_t slots = static_cast<size_t>(nf::kTile * extra + n_total);
    int rc;
    if ((rc = dalloc(nf, &B.d_desc, sizeof(BoxDev) * nbox)) ||
        (rc = dalloc(nf, &B.items_raw, sizeof(Item) * items_cap)) ||
        (rc = dalloc(nf, &B.items, sizeof(Item) * items_cap)) || (rc = dalloc(nf, &B.pieces, sizeof(Piece) * items_cap)) ||
        (rc = dalloc(nf, &B.reduces, sizeof(Reduce) * static_cast<size_t>(extra))) ||
        (rc = dalloc(nf, &B.partials, 3 * sizeof(double) * slots)) ||
        (rc = dalloc(nf, &B.split_k, sizeof(int) * scan_ints)) || (rc = dalloc(nf, &B.split_p, sizeof(int) * scan_ints)) ||
        (rc = dalloc(nf, &B.split_r, sizeof(int) * scan_ints)) ||
        (rc = dalloc(nf, &B.split_scan, nf::scan_temp_bytes(static_cast<int64_t>(scan_ints)))) ||
        (rc = dalloc(nf, &B.nbr_ptrs, sizeof(int *) * nbox)) ||
        (rc = dalloc(nf, &B.pair_ptrs, sizeof(unsigned long long *) * nbox)) ||
        (rc = dalloc(nf, &B.total, sizeof(unsigned long long))) || (rc = dalloc(nf, &B.n_raw, sizeof(int) * 4)) ||
        (rc = dalloc(nf, &B.n_items, sizeof(int) * 4)) || (rc = dalloc(nf, &B.n_reduce, sizeof(int) * 4)) ||
        (rc = dalloc(nf, &B.queue, sizeof(int) * 4))) {
        batch_release(B);
        return rc;
    }
    B.raw_cap = raw_cap;
    B.split_cap = static_cast<int64_t>(items_cap);
    B.n_cap = n_total;
    B.nbox_cap = nbox;
    B.reduce_cap = static_cast<int>(extra);
    B.device = nf->device;
    return NF_OK;
}

}  // namespace

extern "C" int nf_forces_batched(nf_t *const *boxes, int nbox, float *const *acc)
{
    if (!boxes || nbox < 1 || nbox > 4096) return NF_EINVAL;
    nf_t *nf = boxes[0];
    int rc = check_box(nf);
    if (rc) return rc;
    for (int b = 0; b < nbox; ++b) {
        if (!boxes[b]) return fail(nf, NF_EINVAL, "NULL box");
        if (!boxes[b]->have_particles) return fail(nf, NF_ESTATE, "box without particles");
        if (boxes[b]->device != nf->device) return fail(nf, NF_EINVAL, "boxes on different devices");
        if (boxes[b]->softening != nf->softening) return fail(nf, NF_EINVAL, "boxes with different softening");
        if (boxes[b]->cut_nmin > 0) return fail(nf, NF_EINVAL, "the batched launch is exact-only (a box has a cut-off)");
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    Batch &B = g_batch;
    bool same = B.device == nf->device && static_cast<int>(B.boxes.size()) == nbox;
    for (int b = 0; same && b < nbox; ++b) same = B.boxes[b] == boxes[b] && B.gens[b] == boxes[b]->plan_gen;
    if (!same) {
        // (re)plan: one item list over all boxes, class-major (largest cells first), then split
        cudaStreamSynchronize(nf->stream);
        int64_t raw_cap = 16, n_total = 0;
        for (int b = 0; b < nbox; ++b) {
            raw_cap += boxes[b]->item_cap;
            n_total += boxes[b]->n;
        }
        if (B.device != nf->device || raw_cap > B.raw_cap || n_total > B.n_cap || nbox > B.nbox_cap) {
            if ((rc = batch_alloc(nf, B, nbox, raw_cap, n_total))) return rc;
        }
        std::vector<const int *> nbr(nbox);
        std::vector<const unsigned long long *> prs(nbox);
        for (int b = 0; b < nbox; ++b) {
            nf_t *x = boxes[b];
            NF_CK(nf::neighbour_pairs(x->cell_start, x->cpd, 0, x->pairs, x->counts, x->offsets, x->nbr, nullptr,
                                      nf->stream));
            nbr[b] = x->nbr;
            prs[b] = x->pairs;
        }
        NF_CK(nf::zero_device_int(B.n_raw, nf->stream));
        for (int cls = 0; cls < nf::kClasses; ++cls)
            for (int b = 0; b < nbox; ++b)
                NF_CK(nf::plan_items_class(boxes[b]->cell_start, boxes[b]->nbr, boxes[b]->ncell, b, cls, B.items_raw,
                                           B.n_raw, boxes[b]->counts, boxes[b]->offsets, boxes[b]->scan_tmp,
                                           boxes[b]->tiles, nf->stream));
        for (int b = 0; b < nbox; ++b)
            NF_CK(nf::plan_lane_items(boxes[b]->cell_start, boxes[b]->nbr, boxes[b]->cpd, b, B.items_raw, B.n_raw,
                                      boxes[b]->counts, boxes[b]->offsets, boxes[b]->scan_tmp, nf->stream));
        NF_CK(cudaMemcpyAsync(B.nbr_ptrs, nbr.data(), sizeof(int *) * nbox, cudaMemcpyHostToDevice, nf->stream));
        NF_CK(cudaMemcpyAsync(B.pair_ptrs, prs.data(), sizeof(void *) * nbox, cudaMemcpyHostToDevice, nf->stream));
        NF_CK(nf::sum_pair_counts(B.pair_ptrs, nbox, B.total, nf->stream));
        NF_CK(nf::split_items(B.items_raw, B.n_raw, static_cast<int>(B.raw_cap), B.nbr_ptrs, B.total, nf->wf,
                              nf->tiles.split_floor, B.split_k, B.split_p, B.split_r, B.split_scan, B.items, B.n_items, B.pieces,
                              B.reduces, B.n_reduce, nf->stream));
        NF_CK(nf::partition_light(B.items, B.n_items, static_cast<int>(B.split_cap), B.split_k, B.split_scan,
                                  B.items_raw, nf->stream));
        std::swap(B.items, B.items_raw);
        NF_CK(cudaStreamSynchronize(nf->stream));   // the host vectors above must outlive their copies
        B.boxes.assign(boxes, boxes + nbox);
        B.gens.resize(nbox);
        for (int b = 0; b < nbox; ++b) B.gens[b] = boxes[b]->plan_gen;
        B.h_desc.assign(nbox, BoxDev{});
        NF_CK(cudaMemsetAsync(B.d_desc, 0, sizeof(BoxDev) * nbox, nf->stream));
    }
    // descriptors (uploaded only when an output pointer changed)
    bool dirty = false;
    std::vector<int> copy_back(nbox, 0);
    for (int b = 0; b < nbox; ++b) {
        nf_t *x = boxes[b];
        float4 *out = nullptr;
        float *a = acc ? acc[b] : nullptr;
        if (a && x->n > 0) {
            if (is_device_cached(x, 1, a) && aligned16(a)) {
                out = reinterpret_cast<float4 *>(a);
            } else {
                if (!x->acc32 && (rc = dalloc(x, &x->acc32, sizeof(float4) * static_cast<size_t>(x->cap)))) return rc;
                out = x->acc32;
                copy_back[b] = 1;
            }
        }
        BoxDev d{};
        fill_box_desc(x, d, out, x->acc64, nullptr);
        d.pieces = B.pieces;
        d.partials = B.partials;
        if (std::memcmp(&d, &B.h_desc[b], sizeof(BoxDev)) != 0) {
            B.h_desc[b] = d;
            dirty = true;
        }
    }
    if (dirty)
        NF_CK(cudaMemcpyAsync(B.d_desc, B.h_desc.data(), sizeof(BoxDev) * nbox, cudaMemcpyHostToDevice, nf->stream));
    if ((rc = launch_forces(nf, B.d_desc, B.items, B.n_items, B.queue, 0))) return rc;
    NF_CK(nf::reduce_partials(B.d_desc, B.reduces, B.n_reduce, B.reduce_cap, 0, nf->stream));
    for (int b = 0; b < nbox; ++b) {
        boxes[b]->have_forces = true;
        if (copy_back[b])
            NF_CK(cudaMemcpyAsync(acc[b], boxes[b]->acc32, sizeof(float4) * static_cast<size_t>(boxes[b]->n),
                                  cudaMemcpyDefault, nf->stream));
    }
    return NF_OK;
}
