// nf_step.cu -- leapfrog kick and drift (Table 1, rows Kick and Drift) in
// FP64 arithmetic with FP32 storage.
//
// kick:  v' = v + a dt                  (a: the FP64 per-sink sums, box units)
// drift: s = (c + 1/2 + x_rel) + v' dt cpd / box   per axis, in cell units,
//        then the binning rule of nf_bin.cuh gives the new cell and offset.
// One pass does both and writes the new state in particle-id order, the new
// cell id riding in the offset's w word; a second, coalesced pass lays the cell
// ids out as sort keys (values: the ids) and counts the cells.  The stable sort
// that follows then orders every cell by particle id, exactly as a fresh
// binning of the drifted positions would.  The pass writes scratch only, so a
// step refused for its drift limit leaves the box as it was.
#include "nf_bin.cuh"
#include "nf_internal.cuh"

namespace nf {
namespace {

inline int nblocks(int64_t n, int per) { return static_cast<int>((n + per - 1) / per); }

// (c + 1/2 + x_rel) 2^22 for a stored offset x_rel, a multiple of 2^-22 with |x_rel 2^22| <= 2^21 + 2
__device__ __forceinline__ long long scaled_cell_position(int c, float x_rel)
{
    return (static_cast<long long>(c) << 22) + (1LL << 21) + static_cast<long long>(__float2int_rn(x_rel * 4194304.f));
}

__global__ void kick_drift_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                  const double *__restrict__ acc64, const uint32_t *__restrict__ cell_of,
                                  const uint32_t *__restrict__ perm, double dt, double inv_w, int cpd, int n,
                                  float4 *__restrict__ state_by_id, int *__restrict__ violations)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 v = vel[k];
    const double *a = acc64 + 3 * static_cast<int64_t>(k);
    const float vx = static_cast<float>(__dadd_rn(static_cast<double>(v.x), __dmul_rn(a[0], dt)));
    const float vy = static_cast<float>(__dadd_rn(static_cast<double>(v.y), __dmul_rn(a[1], dt)));
    const float vz = static_cast<float>(__dadd_rn(static_cast<double>(v.z), __dmul_rn(a[2], dt)));
    // drift in cell units; at most 0.8 cell widths per axis per step (Section 4.2.1)
    const double mx = __dmul_rn(__dmul_rn(static_cast<double>(vx), dt), inv_w);
    const double my = __dmul_rn(__dmul_rn(static_cast<double>(vy), dt), inv_w);
    const double mz = __dmul_rn(__dmul_rn(static_cast<double>(vz), dt), inv_w);
    const double lim = 0.8;
    const bool capped = fabs(mx) <= lim && fabs(my) <= lim && fabs(mz) <= lim;
    if (!capped) atomicAdd(violations, 1);
    const uint32_t c = cell_of[k];
    const int cz = static_cast<int>(c % cpd), cy = static_cast<int>((c / cpd) % cpd), cx = static_cast<int>(c / (cpd * cpd));
    const float4 p = pos[k];
    int nx = 0, ny = 0, nz = 0;
    float qx = 0.f, qy = 0.f, qz = 0.f;
    if (capped) {
        // The stored position along an axis, s0 = c + 1/2 + x_rel in cell units, is an integer
        // number of 2^-22 quanta (offsets are kept on that grid), so s0 2^22 is formed exactly in
        // integers and S = s 2^22 = (s0 + m) 2^22 takes the drift's one FP64 rounding: m 2^22 is
        // exact, and scaling by 2^22 commutes with rounding.
        const double sx = __dadd_rn(static_cast<double>(scaled_cell_position(cx, p.x)), __dmul_rn(mx, kTwo22));
        const double sy = __dadd_rn(static_cast<double>(scaled_cell_position(cy, p.y)), __dmul_rn(my, kTwo22));
        const double sz = __dadd_rn(static_cast<double>(scaled_cell_position(cz, p.z)), __dmul_rn(mz, kTwo22));
        bin_scaled(sx, cpd, nx, qx);
        bin_scaled(sy, cpd, ny, qy);
        bin_scaled(sz, cpd, nz, qz);
    } else {
        // a drift over the limit (reported): the same rule from s in FP64
        const double sx = __dadd_rn(static_cast<double>(cx) + 0.5 + static_cast<double>(p.x), mx);
        const double sy = __dadd_rn(static_cast<double>(cy) + 0.5 + static_cast<double>(p.y), my);
        const double sz = __dadd_rn(static_cast<double>(cz) + 0.5 + static_cast<double>(p.z), mz);
        bin_cell_units(sx, cpd, nx, qx);
        bin_cell_units(sy, cpd, ny, qy);
        bin_cell_units(sz, cpd, nz, qz);
    }
    const uint32_t id = perm[k];
    const uint32_t key = static_cast<uint32_t>((nx * cpd + ny) * cpd + nz);
    // one 32-byte record per particle (offset with the key bits, then the velocity), written by
    // two adjacent 16-byte stores: the scattered writes fill whole 32-byte sectors
    float4 *rec = state_by_id + 2 * static_cast<int64_t>(id);
    rec[0] = make_float4(qx, qy, qz, __uint_as_float(key));   // key bits: moved, never computed with
    rec[1] = make_float4(vx, vy, vz, 0.f);
}

__global__ void keys_from_state(const float4 *__restrict__ state_by_id, int n, uint32_t *__restrict__ keys,
                                uint32_t *__restrict__ vals, int *__restrict__ counts)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t key = __float_as_uint(state_by_id[2 * static_cast<int64_t>(k)].w);
    keys[k] = key;
    vals[k] = static_cast<uint32_t>(k);
    atomicAdd(&counts[key], 1);
}

}  // namespace

cudaError_t kick_drift(const float4 *pos, const float4 *vel, const double *acc64, const uint32_t *cell_of,
                       const uint32_t *perm, double dt, double inv_w, int cpd, int n, float4 *state_by_id,
                       int *cap_violations, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    kick_drift_kernel<<<nblocks(n, 256), 256, 0, st>>>(pos, vel, acc64, cell_of, perm, dt, inv_w, cpd, n,
                                                       state_by_id, cap_violations);
    return cudaGetLastError();
}

cudaError_t drift_keys(const float4 *state_by_id, int n, uint32_t *keys, uint32_t *vals, int *counts, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    keys_from_state<<<nblocks(n, 256), 256, 0, st>>>(state_by_id, n, keys, vals, counts);
    return cudaGetLastError();
}

}  // namespace nf

// ---------------------------------------------------------------- time step (Section 4.2.1)
//
// Per cell: v_rms = sqrt(mean |v|^2) and a_max = max |a| over its particles;
// per pass: the minimum over cells of v_rms / a_max (cells with a_max = 0
// skipped), the global sum of |v|^2, max |a| and max |v|.  Blocks write their
// partial results; one block combines them in a fixed order, so the result
// does not depend on scheduling.

namespace nf {
namespace {

constexpr int kDtThreads = 256;

struct DtPart {
    double ratio_min;   // min over cells of v_rms / a_max
    double v2_sum;      // sum of |v|^2
    double a_max;       // max |a|
    double v_max;       // max |v|
};

__global__ void dt_cells(const int *__restrict__ cell_start, int ncell, const float4 *__restrict__ vel,
                         const double *__restrict__ acc64, DtPart *__restrict__ parts)
{
    __shared__ DtPart sh[kDtThreads];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    DtPart p{INFINITY, 0.0, 0.0, 0.0};
    if (c < ncell) {
        const int s0 = cell_start[c], s1 = cell_start[c + 1];
        double v2 = 0.0, am = 0.0, vm = 0.0;
        for (int k = s0; k < s1; ++k) {
            const float4 v = vel[k];
            const double vv = static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y +
                              static_cast<double>(v.z) * v.z;
            const double *a = acc64 + 3 * static_cast<int64_t>(k);
            const double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
            v2 += vv;
            am = fmax(am, aa);
            vm = fmax(vm, vv);
        }
        if (s1 > s0) {
            am = sqrt(am);
            if (am > 0.0) p.ratio_min = sqrt(v2 / (s1 - s0)) / am;
            p.v2_sum = v2;
            p.a_max = am;
            p.v_max = sqrt(vm);
        }
    }
    sh[threadIdx.x] = p;
    __syncthreads();
    for (int o = kDtThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            DtPart &a = sh[threadIdx.x];
            const DtPart &b = sh[threadIdx.x + o];
            a.ratio_min = fmin(a.ratio_min, b.ratio_min);
            a.v2_sum += b.v2_sum;
            a.a_max = fmax(a.a_max, b.a_max);
            a.v_max = fmax(a.v_max, b.v_max);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = sh[0];
}

__global__ void dt_combine(const DtPart *__restrict__ parts, int nparts, DtPart *__restrict__ out)
{
    __shared__ DtPart sh[kDtThreads];
    DtPart p{INFINITY, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const DtPart q = parts[i];
        p.ratio_min = fmin(p.ratio_min, q.ratio_min);
        p.v2_sum += q.v2_sum;
        p.a_max = fmax(p.a_max, q.a_max);
        p.v_max = fmax(p.v_max, q.v_max);
    }
    sh[threadIdx.x] = p;
    __syncthreads();
    for (int o = kDtThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            DtPart &a = sh[threadIdx.x];
            const DtPart &b = sh[threadIdx.x + o];
            a.ratio_min = fmin(a.ratio_min, b.ratio_min);
            a.v2_sum += b.v2_sum;
            a.a_max = fmax(a.a_max, b.a_max);
            a.v_max = fmax(a.v_max, b.v_max);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

size_t dt_temp_bytes(int ncell) { return sizeof(DtPart) * (static_cast<size_t>((ncell + kDtThreads - 1) / kDtThreads) + 1); }

// result: 4 doubles {min over cells of v_rms/a_max, sum |v|^2, max |a|, max |v|} at temp[0..3]
cudaError_t dt_reduce(const int *cell_start, int ncell, const float4 *vel, const double *acc64, void *temp,
                      cudaStream_t st)
{
    const int nb = (ncell + kDtThreads - 1) / kDtThreads;
    DtPart *out = static_cast<DtPart *>(temp);
    DtPart *parts = out + 1;
    dt_cells<<<nb, kDtThreads, 0, st>>>(cell_start, ncell, vel, acc64, parts);
    dt_combine<<<1, kDtThreads, 0, st>>>(parts, nb, out);
    return cudaGetLastError();
}

}  // namespace nf
