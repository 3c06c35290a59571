// nf_multipole.cu -- Cartesian multipole moments of every cell (Section 2.1:
// the far-field pass computes the multipoles of the particles in every cell,
// order p = 8 in the paper's run, in double precision internally).
//
// For cell c, with offsets x_rel from the cell centre in cell widths and unit
// masses, M_c[a, b, k] = sum_i x_i^a y_i^b z_i^k for a + b + k <= p.
// Terms are ordered by degree n = 0..p, then a = n..0, then b = n-a..0
// (k = n - a - b): (p+1)(p+2)(p+3)/6 terms per cell (165 at p = 8).
//
// One block per cell at a time (grid-stride over cells): the block's threads
// load a chunk of the cell's particles and tabulate their powers in shared
// memory, then thread t accumulates term t over the chunk in FP64.
#include <algorithm>

#include "nf_internal.cuh"

namespace nf {
namespace {

constexpr int kMpThreads = 192;
constexpr int kMaxOrder = 8;
constexpr int kPw = kMaxOrder + 1;   // powers 0..8 per axis

__global__ void __launch_bounds__(kMpThreads) multipole_kernel(const int *__restrict__ cell_start, int ncell,
                                                               const float4 *__restrict__ pos, int order,
                                                               double *__restrict__ out)
{
    __shared__ double pw[kMpThreads][3 * kPw];
    const int nterms = (order + 1) * (order + 2) * (order + 3) / 6;
    // this thread's term (a, b, k)
    int ta = 0, tb = 0, tk = 0;
    {
        int t = threadIdx.x, idx = 0;
        bool found = false;
        for (int n = 0; n <= order && !found; ++n)
            for (int a = n; a >= 0 && !found; --a)
                for (int b = n - a; b >= 0 && !found; --b) {
                    if (idx == t) {
                        ta = a; tb = b; tk = n - a - b;
                        found = true;
                    }
                    ++idx;
                }
    }
    for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int s0 = cell_start[c], s1 = cell_start[c + 1];
        double acc = 0.0;
        for (int base = s0; base < s1; base += kMpThreads) {
            const int m = min(kMpThreads, s1 - base);
            if (threadIdx.x < m) {
                const float4 p = pos[base + threadIdx.x];
                const double x[3] = {static_cast<double>(p.x), static_cast<double>(p.y), static_cast<double>(p.z)};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    double v = 1.0;
                    for (int e = 0; e <= order; ++e) {
                        pw[threadIdx.x][d * kPw + e] = v;
                        v *= x[d];
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x < nterms)
                for (int j = 0; j < m; ++j) acc = fma(pw[j][ta] * pw[j][kPw + tb], pw[j][2 * kPw + tk], acc);
            __syncthreads();
        }
        if (threadIdx.x < nterms) out[static_cast<int64_t>(c) * nterms + threadIdx.x] = acc;
    }
}

// Sub-cell moments of the dense cells (cut-off mode).  One block of kCutSub
// threads per dense cell (grid-stride over the cells); the block stages the
// cell's particles in chunks with their sub-cell index, and thread t sums the
// members of sub-cell t in storage order, in FP64: count and centre of mass in
// a first pass, the traceless quadrupole about that centre in a second.  A
// particle's sub-cell along an axis is floor((x + 1/2) kCutK), kept in
// 0..kCutK-1 (exact on the 2^-22 grid).
constexpr int kCutChunk = 256;

__device__ __forceinline__ int cut_axis(float x)
{
    const int q = __float2int_rd((x + 0.5f) * static_cast<float>(kCutK));
    return q < 0 ? 0 : (q > kCutK - 1 ? kCutK - 1 : q);
}

__global__ void __launch_bounds__(kCutSub) subcell_kernel(const int *__restrict__ cell_start,
                                                          const float4 *__restrict__ pos,
                                                          const int *__restrict__ dense_cells,
                                                          const int *__restrict__ n_dense, float *__restrict__ mpole)
{
    __shared__ float4 sp[kCutChunk];
    __shared__ unsigned char sb[kCutChunk];
    const int t = threadIdx.x;
    const int nd = *n_dense;
    for (int slot = blockIdx.x; slot < nd; slot += gridDim.x) {
        const int c = dense_cells[slot];
        const int j0 = cell_start[c], j1 = cell_start[c + 1];
        double m = 0.0, X[3] = {0.0, 0.0, 0.0}, Q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int pass = 0; pass < 2; ++pass) {
            for (int base = j0; base < j1; base += kCutChunk) {
                const int cnt = min(kCutChunk, j1 - base);
                __syncthreads();
                for (int k = t; k < cnt; k += kCutSub) {
                    const float4 p = pos[base + k];
                    sp[k] = p;
                    sb[k] = static_cast<unsigned char>((cut_axis(p.x) * kCutK + cut_axis(p.y)) * kCutK + cut_axis(p.z));
                }
                __syncthreads();
                for (int k = 0; k < cnt; ++k) {
                    if (sb[k] != t) continue;
                    const float4 p = sp[k];
                    if (pass == 0) {
                        m += 1.0;
                        X[0] += p.x; X[1] += p.y; X[2] += p.z;
                    } else {
                        const double sx = p.x - X[0], sy = p.y - X[1], sz = p.z - X[2];
                        const double s2 = sx * sx + sy * sy + sz * sz;
                        Q[0] += 3.0 * sx * sx - s2; Q[1] += 3.0 * sx * sy; Q[2] += 3.0 * sx * sz;
                        Q[3] += 3.0 * sy * sy - s2; Q[4] += 3.0 * sy * sz; Q[5] += 3.0 * sz * sz - s2;
                    }
                }
            }
            if (pass == 0 && m > 0.0) {
                X[0] /= m; X[1] /= m; X[2] /= m;
            }
        }
        float *o = mpole + (static_cast<int64_t>(slot) * kCutSub + t) * kCutWords;
        o[0] = static_cast<float>(m);
        o[1] = static_cast<float>(X[0]); o[2] = static_cast<float>(X[1]); o[3] = static_cast<float>(X[2]);
        for (int q = 0; q < 6; ++q) o[4 + q] = static_cast<float>(Q[q]);
    }
}

}  // namespace

cudaError_t subcell_moments(const int *cell_start, const float4 *pos, const int *dense_cells, const int *n_dense,
                            int64_t dense_cap, float *mpole, int sm_count, cudaStream_t st)
{
    const int blocks = static_cast<int>(std::min<int64_t>(dense_cap, static_cast<int64_t>(sm_count) * 16));
    if (blocks <= 0) return cudaSuccess;
    subcell_kernel<<<blocks, kCutSub, 0, st>>>(cell_start, pos, dense_cells, n_dense, mpole);
    return cudaGetLastError();
}

int multipole_terms(int order) { return (order + 1) * (order + 2) * (order + 3) / 6; }

cudaError_t cell_multipoles(const int *cell_start, int ncell, const float4 *pos, int order, double *out, int sm_count,
                            cudaStream_t st)
{
    if (order < 0 || order > kMaxOrder) return cudaErrorInvalidValue;
    const int blocks = std::min(ncell, sm_count * 16);
    if (blocks <= 0) return cudaSuccess;
    multipole_kernel<<<blocks, kMpThreads, 0, st>>>(cell_start, ncell, pos, order, out);
    return cudaGetLastError();
}

}  // namespace nf
