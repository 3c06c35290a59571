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

}  // namespace

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
