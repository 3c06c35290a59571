// nf_step.cu -- leapfrog kick and drift (Table 1, rows Kick and Drift) in
// FP64 arithmetic with FP32 storage.
//
// kick:  v' = v + a dt                  (a: the FP64 per-sink sums, box units)
// drift: s = (c + 1/2 + x_rel) + v' dt cpd / box   per axis, in cell units,
//        then the binning rule of nf_bin.cuh gives the new cell and offset.
// The new state is written in particle-id order (key = new cell id), so the
// stable sort that follows orders every cell by particle id, exactly as a
// fresh binning of the drifted positions would.
#include "nf_bin.cuh"
#include "nf_internal.cuh"

namespace nf {
namespace {

inline int nblocks(int64_t n, int per) { return static_cast<int>((n + per - 1) / per); }

__global__ void kick_kernel(const float4 *__restrict__ vel, const double *__restrict__ acc64, double dt, double inv_w,
                            int n, float4 *__restrict__ vel_new, int *__restrict__ violations)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 v = vel[k];
    const double *a = acc64 + 3 * static_cast<int64_t>(k);
    const float vx = static_cast<float>(__dadd_rn(static_cast<double>(v.x), __dmul_rn(a[0], dt)));
    const float vy = static_cast<float>(__dadd_rn(static_cast<double>(v.y), __dmul_rn(a[1], dt)));
    const float vz = static_cast<float>(__dadd_rn(static_cast<double>(v.z), __dmul_rn(a[2], dt)));
    vel_new[k] = make_float4(vx, vy, vz, 0.f);
    // drift limit: at most 0.8 cell widths per axis per step (Section 4.2.1)
    const double lim = 0.8;
    const double mx = fabs(__dmul_rn(__dmul_rn(static_cast<double>(vx), dt), inv_w));
    const double my = fabs(__dmul_rn(__dmul_rn(static_cast<double>(vy), dt), inv_w));
    const double mz = fabs(__dmul_rn(__dmul_rn(static_cast<double>(vz), dt), inv_w));
    if (!(mx <= lim && my <= lim && mz <= lim)) atomicAdd(violations, 1);
}

__global__ void drift_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ vel_new,
                             const uint32_t *__restrict__ cell_of, const uint32_t *__restrict__ perm, double dt,
                             double inv_w, int cpd, int n, uint32_t *__restrict__ key_by_id,
                             uint32_t *__restrict__ val_by_id, float4 *__restrict__ xq_by_id,
                             float4 *__restrict__ vel_by_id)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t c = cell_of[k];
    const int cz = static_cast<int>(c % cpd), cy = static_cast<int>((c / cpd) % cpd), cx = static_cast<int>(c / (cpd * cpd));
    const float4 p = pos[k];
    const float4 v = vel_new[k];
    const double sx = __dadd_rn(static_cast<double>(cx) + 0.5 + static_cast<double>(p.x),
                                __dmul_rn(__dmul_rn(static_cast<double>(v.x), dt), inv_w));
    const double sy = __dadd_rn(static_cast<double>(cy) + 0.5 + static_cast<double>(p.y),
                                __dmul_rn(__dmul_rn(static_cast<double>(v.y), dt), inv_w));
    const double sz = __dadd_rn(static_cast<double>(cz) + 0.5 + static_cast<double>(p.z),
                                __dmul_rn(__dmul_rn(static_cast<double>(v.z), dt), inv_w));
    int nx, ny, nz;
    float qx, qy, qz;
    bin_cell_units(sx, cpd, nx, qx);
    bin_cell_units(sy, cpd, ny, qy);
    bin_cell_units(sz, cpd, nz, qz);
    const uint32_t id = perm[k];
    key_by_id[id] = static_cast<uint32_t>((nx * cpd + ny) * cpd + nz);
    val_by_id[id] = id;
    xq_by_id[id] = make_float4(qx, qy, qz, 0.f);
    vel_by_id[id] = v;
}

}  // namespace

cudaError_t kick(const float4 *vel, const double *acc64, double dt, double inv_w, int n, float4 *vel_new,
                 int *cap_violations, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    kick_kernel<<<nblocks(n, 256), 256, 0, st>>>(vel, acc64, dt, inv_w, n, vel_new, cap_violations);
    return cudaGetLastError();
}

cudaError_t drift(const float4 *pos, const float4 *vel_new, const uint32_t *cell_of, const uint32_t *perm,
                  double dt, double inv_w, int cpd, int n, uint32_t *key_by_id, uint32_t *val_by_id,
                  float4 *xq_by_id, float4 *vel_by_id, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    drift_kernel<<<nblocks(n, 256), 256, 0, st>>>(pos, vel_new, cell_of, perm, dt, inv_w, cpd, n, key_by_id,
                                                  val_by_id, xq_by_id, vel_by_id);
    return cudaGetLastError();
}

}  // namespace nf
