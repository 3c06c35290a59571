// nf_pair.cu -- the near-field pair kernel (forces and adjoint).
//
// Work: every particle i of a cell takes F(x_j - x_i) from every particle j of
// the 125 cells within R = 2 cells of its own (Section 2.1), with the spline
// law of Section 4.3.1 written branch-free as f = min(r^-3, g(r)),
// g(r) = (10 - 15 r/eps + 6 r^2/eps^2) / eps^3.  The two agree for every
// r > 0: r^3 g(r) = 10u^3 - 15u^4 + 6u^5 (u = r/eps) rises monotonically
// (derivative 30u^2 (1-u)^2) through 1 at u = 1, so g <= r^-3 exactly when
// r <= eps; this is the single `min` of the paper's footnote to Section 4.3.1.
//
// Structure (one persistent grid, one warp per work item):
//   * a work item is up to 128 sinks of one cell; the warp pulls item indices
//     from a device queue (atomic counter), largest cells first;
//   * the warp builds a 125-entry table of its neighbour cells (start, prefix
//     of counts) in shared memory, the 27 near cells (Chebyshev distance <= 1)
//     first, so each round's sources split into a near run and a far run;
//   * sources are streamed in rounds of B particles: each lane gathers B/32
//     float4 with cp.async (16 B each, coalesced along each cell's run) into
//     one of two per-warp shared-memory buffers while the previous round is
//     being computed; once landed, each lane adds its own entries' integer
//     cell offset (dx, dy, dz), so every source is in the sink cell's frame;
//   * sinks live in registers: with > 16 sinks every lane holds S = 1, 2 or 4
//     sinks and reads each staged source as a shared-memory broadcast; with
//     <= 16 sinks the lanes split the sources between them (each sink owns
//     32/P lanes, P = sinks rounded up to a power of two) and the partial
//     sums are combined with a fixed xor-shuffle tree;
//   * pair arithmetic is FP32, rsqrt on the SFU plus one Newton step.  A far
//     source (Chebyshev distance 2, so r >= 1 cell > eps) takes f = r^-3 with
//     the Newton step folded into the cube and the accumulators' scale
//     (kForceSigma): 13 FP32 FMA-pipe operations + 1 SFU.  A near source takes
//     the same 13 unless some sink of the warp lies within eps of it (a warp
//     vote on r^2 < eps^2, which self pairs always trigger); then all of the
//     warp's pairs with it take the branch-free law, 19 operations + 1 min + 1
//     SFU.  Lanes holding 2 or 4 sinks evaluate two
//     sinks per paired FP32 instruction (FADD2 / FMUL2 / FFMA2), which halves
//     the issue slots so the FP32 lanes, not instruction issue, bound the loop;
//   * accumulation: plain FFMA within a round (<= B sources), folded after
//     every round into a (hi, lo) pair with an exact two-sum and reduced to
//     FP64 per sink at the end (compensated mode); or one FP32 running sum
//     per sink (plain mode).  The sums carry the factor kForceSigma, which
//     the FP64 conversion removes.
//
// Exactness of separations: offsets are multiples of 2^-22 cell widths with
// |x| <= 1/2, so x_j + D (|D| <= 2) and (x_j + D) - x_i are exact in FP32.
// Every item owns its sinks and sums its sources in a fixed order, so the
// result does not depend on which warp ran which item (bit-reproducible).
#include <cfloat>
#include <climits>
#include <mutex>

#include "nf_internal.cuh"

namespace nf {
namespace {

#ifndef NF_SRC_UNROLL
#define NF_SRC_UNROLL 4   // staged sources evaluated per unrolled step of the broadcast loop
#endif
#ifndef NF_PACKED
#define NF_PACKED 1   // paired FP32 instructions for two sinks when a lane holds 2 or 4 sinks
#endif
#ifndef NF_STAGE_A
#define NF_STAGE_A 128   // sources staged per round for the launch shape's stage = 128
#endif
#ifndef NF_FAR_LAW
#define NF_FAR_LAW 1   // sources of the 98 far cells take f = r^-3 without the spline branch
#endif
#ifndef NF_NEAR_VOTE
#define NF_NEAR_VOTE 1   // near-cell sources take the Newtonian tail unless a warp lane is within eps
#endif
#ifndef NF_PAIR_SOURCES
#define NF_PAIR_SOURCES 1   // lanes holding one sink evaluate two sources per paired FP32 instruction
#endif
#ifndef NF_LANE_FAR_LAW
#define NF_LANE_FAR_LAW 1   // lane items: columns at |dx| = 2 or |dy| = 2 take the Newtonian law
#endif
#ifndef NF_MIN_BLOCKS
#define NF_MIN_BLOCKS 3   // resident 256-thread blocks per SM the register budget must allow
#endif
#ifndef NF_ADJ_UNROLL
#define NF_ADJ_UNROLL 4   // staged sources per unrolled step of the adjoint
#endif
#ifndef NF_PACKED_ADJ
#define NF_PACKED_ADJ 1   // the adjoint evaluates two sinks per paired FP32 instruction on 2- and 4-sink lanes
#endif
#ifndef NF_STAGE_CONTIG
#define NF_STAGE_CONTIG 1   // each lane stages B/32 consecutive sources (one cell search per lane and round)
#endif
#ifndef NF_LANE_UNROLL
#define NF_LANE_UNROLL 4   // sources per unrolled step of a lane item (independent loads in flight)
#endif
#ifndef NF_PAIR_UNROLL
#define NF_PAIR_UNROLL 2   // source pairs per unrolled step on lanes holding one sink
#endif
#ifndef NF_LANE_PAIRED
#define NF_LANE_PAIRED 1   // lane items of library-loaded boxes: z offsets from w, two sources per paired instruction
#endif
#ifndef NF_LANE_PAIR_UNROLL
#define NF_LANE_PAIR_UNROLL 2   // paired lane items: source pairs per unrolled step (1 or 2)
#endif
#ifndef NF_FOLD_HALVES
#define NF_FOLD_HALVES 1   // one-sink lanes add their two source-pair halves before the compensated fold
#endif
#ifndef NF_PAIRED_FOLD
#define NF_PAIRED_FOLD 1   // lanes with 2 or 4 sinks fold two sinks' partials per paired FP32 instruction
#endif
#ifndef NF_UNROLL_S2
#define NF_UNROLL_S2 NF_SRC_UNROLL   // staged sources per unrolled step on lanes holding two sinks
#endif

constexpr unsigned kFull = 0xffffffffu;
constexpr float kFar = 1.0e18f;   // padding source: y^3 underflows to 0, contributes exactly zero

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// exact sum a + b = s + e (two-sum; no FMA involved)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

struct Comp3 {
    float hx, hy, hz;   // running high parts
    float lx, ly, lz;   // accumulated low parts
};

// combine with the partner lane `o` (xor); both lanes end with the same value
__device__ __forceinline__ void comp_xor_combine(Comp3 &c, int o)
{
    float s, e;
    float h2 = __shfl_xor_sync(kFull, c.hx, o), l2 = __shfl_xor_sync(kFull, c.lx, o);
    two_sum(c.hx, h2, s, e); c.hx = s; c.lx = __fadd_rn(__fadd_rn(c.lx, l2), e);
    h2 = __shfl_xor_sync(kFull, c.hy, o); l2 = __shfl_xor_sync(kFull, c.ly, o);
    two_sum(c.hy, h2, s, e); c.hy = s; c.ly = __fadd_rn(__fadd_rn(c.ly, l2), e);
    h2 = __shfl_xor_sync(kFull, c.hz, o); l2 = __shfl_xor_sync(kFull, c.lz, o);
    two_sum(c.hz, h2, s, e); c.hz = s; c.lz = __fadd_rn(__fadd_rn(c.lz, l2), e);
}

// The rest of a spline-law pair once d and r^2 (FLT_MIN included) are known:
// f = min(r^-3, a0 + a1 r + a2 r^2), rsqrt on the SFU plus one Newton step.
__device__ __forceinline__ void tail_spline(float dx, float dy, float dz, float r2, float &ax, float &ay, float &az,
                                            float a0, float a1, float a2)
{
    float y = rsqrtf(r2);                    // SFU
    const float t = r2 * y;
    const float h = t * y;
    const float e = fmaf(h, -0.5f, 0.5f);
    y = fmaf(y, e, y);                       // one Newton step for r2^-1/2
    const float r = fmaf(t, e, t);           // r2 * y
    const float y3 = y * y * y;
    const float g = fmaf(fmaf(a2, r, a1), r, a0);
    const float f = fminf(y3, g) * kForceSigma;   // the accumulators' scale
    ax = fmaf(f, dx, ax);
    ay = fmaf(f, dy, ay);
    az = fmaf(f, dz, az);
}

// The rest of a pair at r >= eps (law: f = r^-3).  The Newton step is taken on
// r^-3 itself: with y the SFU estimate of (r^2)^-1/2 and h = r^2 y^2, one
// Newton step for (r^2)^-1/2 multiplies y by 1 + e, e = (1 - h) / 2, so
// r^-3 = y^3 (1 + e)^3 = y^3 (1 + 3e) + O(e^2) (|e| < 2^-21, the dropped
// terms below 2^-40 relative).  In the accumulators' scale kForceSigma =
// -(A - 1) that is y^3 (h - A) (nf_internal.cuh): one FFMA forms h - A, so
// the pair costs 7 FP32-pipe operations + 1 SFU, no min.
__device__ __forceinline__ void tail_newton(float dx, float dy, float dz, float r2, float &ax, float &ay, float &az)
{
    const float y = rsqrtf(r2);                   // SFU
    const float yy = y * y;
    const float g = fmaf(r2, yy, -kNewtonA);      // h - A
    const float f = (yy * y) * g;                 // kForceSigma r^-3
    ax = fmaf(f, dx, ax);
    ay = fmaf(f, dy, ay);
    az = fmaf(f, dz, az);
}

// one pair: a += kForceSigma f(r) d.  Spline (SOFT = 0): f = min(r^-3, a0 +
// a1 r + a2 r^2), 21 FP32-pipe operations + 1 SFU.  Plummer (SOFT = 1, Eq.
// eqn:plummer): f = (r^2 + eps_p^2)^-3/2, 13 FP32-pipe operations + 1 SFU
// (eps2 = eps_p^2).
template <int SOFT>
__device__ __forceinline__ void pair_force(const float4 q, float xi, float yi, float zi, float &ax, float &ay,
                                           float &az, float a0, float a1, float a2, float eps2)
{
    const float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
    if (SOFT == 1) {
        // (r^2 + eps_p^2)^-3/2 in the accumulators' scale, the Newton step taken on the cube
        tail_newton(dx, dy, dz, fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2))), ax, ay, az);
        return;
    }
    // + FLT_MIN: below half an ulp of any nonzero r^2 on the 2^-22 grid (r^2 >= 2^-44), so it changes
    // nothing except r = 0 (self pair), where it keeps rsqrt finite: finite g, times d = 0
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, FLT_MIN)));
    tail_spline(dx, dy, dz, r2, ax, ay, az, a0, a1, a2);
}

// tail_spline for two sinks with paired FP32 instructions (same arithmetic per lane)
__device__ __forceinline__ void tail2_spline(const float2 dx, const float2 dy, const float2 dz, const float2 r2,
                                             float2 &ax, float2 &ay, float2 &az, const float2 a0, const float2 a1,
                                             const float2 a2)
{
    const float2 half = make_float2(0.5f, 0.5f), mhalf = make_float2(-0.5f, -0.5f);
    float2 y = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 t = __fmul2_rn(r2, y);
    const float2 h = __fmul2_rn(t, y);
    const float2 e = __ffma2_rn(h, mhalf, half);
    y = __ffma2_rn(y, e, y);
    const float2 r = __ffma2_rn(t, e, t);
    const float2 y3 = __fmul2_rn(__fmul2_rn(y, y), y);
    const float2 g = __ffma2_rn(__ffma2_rn(a2, r, a1), r, a0);
    const float2 f = __fmul2_rn(make_float2(fminf(y3.x, g.x), fminf(y3.y, g.y)),
                                make_float2(kForceSigma, kForceSigma));   // the accumulators' scale
    ax = __ffma2_rn(f, dx, ax);
    ay = __ffma2_rn(f, dy, ay);
    az = __ffma2_rn(f, dz, az);
}

// tail_newton for two sinks with paired FP32 instructions (same arithmetic per lane)
__device__ __forceinline__ void tail2_newton(const float2 dx, const float2 dy, const float2 dz, const float2 r2,
                                             float2 &ax, float2 &ay, float2 &az)
{
    const float2 y = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 yy = __fmul2_rn(y, y);
    const float2 g = __ffma2_rn(r2, yy, make_float2(-kNewtonA, -kNewtonA));   // h - A
    const float2 f = __fmul2_rn(__fmul2_rn(yy, y), g);                         // kForceSigma r^-3
    ax = __ffma2_rn(f, dx, ax);
    ay = __ffma2_rn(f, dy, ay);
    az = __ffma2_rn(f, dz, az);
}

// Two sinks against one source with Blackwell's paired FP32 instructions
// (FADD2 / FMUL2 / FFMA2: one issue slot for two lanes' worth of FP32 work).
// Every lane of a pair follows exactly the scalar pair_force arithmetic
// (round-to-nearest each op, same order), so results are bit-identical.
// nx, ny, nz hold minus the two sinks' offsets.
template <int SOFT>
__device__ __forceinline__ void pair_force2(const float2 qx, const float2 qy, const float2 qz, const float2 nx,
                                            const float2 ny, const float2 nz, float2 &ax, float2 &ay, float2 &az,
                                            const float2 a0, const float2 a1, const float2 a2, const float2 eps2)
{
    const float2 dx = __fadd2_rn(qx, nx), dy = __fadd2_rn(qy, ny), dz = __fadd2_rn(qz, nz);
    if (SOFT == 1) {
        tail2_newton(dx, dy, dz, __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, eps2))), ax, ay, az);
        return;
    }
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, make_float2(FLT_MIN, FLT_MIN))));
    tail2_spline(dx, dy, dz, r2, ax, ay, az, a0, a1, a2);
}

// One pair with a source in a cell at Chebyshev distance 2 from the sink's
// cell: r >= 1 cell width > eps, so the spline law is Newtonian there and the
// pair takes tail_newton: 13 FP32-pipe operations + 1 SFU.
__device__ __forceinline__ void pair_force_far(const float4 q, float xi, float yi, float zi, float &ax, float &ay,
                                               float &az)
{
    const float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
    tail_newton(dx, dy, dz, fmaf(dz, dz, fmaf(dy, dy, dx * dx)), ax, ay, az);
}

// pair_force_far for two sinks with paired FP32 instructions (same arithmetic per lane)
__device__ __forceinline__ void pair_force2_far(const float2 qx, const float2 qy, const float2 qz, const float2 nx,
                                                const float2 ny, const float2 nz, float2 &ax, float2 &ay, float2 &az)
{
    const float2 dx = __fadd2_rn(qx, nx), dy = __fadd2_rn(qy, ny), dz = __fadd2_rn(qz, nz);
    tail2_newton(dx, dy, dz, __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx))), ax, ay, az);
}

// Acceleration from a sub-cell's quadrupole expansion about its centre of mass
// (cut-off mode): R = centre - sink, sum_j 1/|R + s_j| = M/r + (R.Q.R)/(2 r^5)
// + O(s^3), so a += M R/r^3 - Q R/r^5 + (5/2)(R.Q.R) R/r^7 (Newtonian: the
// sub-cell lies beyond eps).  q = Q_xx, Q_xy, Q_xz, Q_yy, Q_yz, Q_zz.
__device__ __forceinline__ void quad_force(float rx, float ry, float rz, float M, const float *q, float &ax,
                                           float &ay, float &az)
{
    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    float y = rsqrtf(r2);
    y = y * fmaf(-0.5f * r2, y * y, 1.5f);   // one Newton step
    const float y2 = y * y, y3 = y2 * y, y5 = y3 * y2, y7 = y5 * y2;
    const float qx = fmaf(q[2], rz, fmaf(q[1], ry, q[0] * rx));
    const float qy = fmaf(q[4], rz, fmaf(q[3], ry, q[1] * rx));
    const float qz = fmaf(q[5], rz, fmaf(q[4], ry, q[2] * rx));
    const float rqr = fmaf(rz, qz, fmaf(ry, qy, rx * qx));
    const float c = fmaf(2.5f * rqr, y7, M * y3);
    ax = fmaf(c, rx, fmaf(-y5, qx, ax));
    ay = fmaf(c, ry, fmaf(-y5, qy, ay));
    az = fmaf(c, rz, fmaf(-y5, qz, az));
}

// one pair of the adjoint: grad += J(d) (w_j - w_k), J = f I + (f'/r) d d^T
template <int SOFT>
__device__ __forceinline__ void pair_adjoint(const float4 q, const float4 wj, float xi, float yi, float zi, float wx,
                                             float wy, float wz, float &gx, float &gy, float &gz, float a0, float a1,
                                             float a2, float eps2)
{
    const float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
    float f, hh;
    if (SOFT == 1) {
        // Plummer: f = s^-3/2, f'/r = -3 s^-5/2, s = r^2 + eps_p^2
        const float s2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
        float y = rsqrtf(s2);
        const float t = s2 * y;
        const float h = t * y;
        const float e = fmaf(h, -0.5f, 0.5f);
        y = fmaf(y, e, y);
        const float y2 = y * y;
        f = y2 * y;
        hh = -3.f * f * y2;
    } else {
        // + FLT_MIN as in the forces: it changes nothing but r = 0, where it keeps rsqrt finite
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, FLT_MIN)));
        const bool inside = r2 < eps2;
        float y = rsqrtf(r2);
        const float t = r2 * y;
        const float h = t * y;
        const float e = fmaf(h, -0.5f, 0.5f);
        y = fmaf(y, e, y);
        const float r = fmaf(t, e, t);
        const float y2 = y * y;
        const float y3 = y2 * y;
        // spline: f = a0 + a1 r + a2 r^2, f'/r = a1 / r + 2 a2 ; Newtonian: f = r^-3, f'/r = -3 r^-5
        f = inside ? fmaf(fmaf(a2, r, a1), r, a0) : y3;
        hh = inside ? fmaf(a1, y, 2.f * a2) : -3.f * y3 * y2;
    }
    const float ux = wj.x - wx, uy = wj.y - wy, uz = wj.z - wz;
    const float du = fmaf(dz, uz, fmaf(dy, uy, dx * ux));
    const float hd = hh * du;
    gx = fmaf(hd, dx, fmaf(f, ux, gx));
    gy = fmaf(hd, dy, fmaf(f, uy, gy));
    gz = fmaf(hd, dz, fmaf(f, uz, gz));
}

// pair_adjoint for two sinks against one source with paired FP32 instructions: every
// lane of a pair follows the scalar arithmetic (same roundings, same order), so results
// are bit-identical.  nx, ny, nz and nwx, nwy, nwz hold minus the sinks'
// offsets and cotangents; a2x2 = 2 a2.
template <int SOFT>
__device__ __forceinline__ void pair_adjoint2(const float2 qx, const float2 qy, const float2 qz, const float2 wjx,
                                              const float2 wjy, const float2 wjz, const float2 nx, const float2 ny,
                                              const float2 nz, const float2 nwx, const float2 nwy, const float2 nwz,
                                              float2 &gx, float2 &gy, float2 &gz, const float2 a0, const float2 a1,
                                              const float2 a2, const float2 a2x2, float eps2)
{
    const float2 dx = __fadd2_rn(qx, nx), dy = __fadd2_rn(qy, ny), dz = __fadd2_rn(qz, nz);
    const float2 half = make_float2(0.5f, 0.5f), mhalf = make_float2(-0.5f, -0.5f);
    float2 f, hh;
    if (SOFT == 1) {
        const float2 e2 = make_float2(eps2, eps2);
        const float2 s2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, e2)));
        float2 y = make_float2(rsqrtf(s2.x), rsqrtf(s2.y));
        const float2 t = __fmul2_rn(s2, y);
        const float2 h = __fmul2_rn(t, y);
        const float2 e = __ffma2_rn(h, mhalf, half);
        y = __ffma2_rn(y, e, y);
        const float2 y2 = __fmul2_rn(y, y);
        f = __fmul2_rn(y2, y);
        hh = __fmul2_rn(__fmul2_rn(make_float2(-3.f, -3.f), f), y2);
    } else {
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, make_float2(FLT_MIN, FLT_MIN))));
        const bool in_x = r2.x < eps2, in_y = r2.y < eps2;
        float2 y = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 t = __fmul2_rn(r2, y);
        const float2 h = __fmul2_rn(t, y);
        const float2 e = __ffma2_rn(h, mhalf, half);
        y = __ffma2_rn(y, e, y);
        const float2 r = __ffma2_rn(t, e, t);
        const float2 y2 = __fmul2_rn(y, y);
        const float2 y3 = __fmul2_rn(y2, y);
        const float2 poly = __ffma2_rn(__ffma2_rn(a2, r, a1), r, a0);
        const float2 hin = __ffma2_rn(a1, y, a2x2);
        const float2 hout = __fmul2_rn(__fmul2_rn(make_float2(-3.f, -3.f), y3), y2);
        f = make_float2(in_x ? poly.x : y3.x, in_y ? poly.y : y3.y);
        hh = make_float2(in_x ? hin.x : hout.x, in_y ? hin.y : hout.y);
    }
    const float2 ux = __fadd2_rn(wjx, nwx), uy = __fadd2_rn(wjy, nwy), uz = __fadd2_rn(wjz, nwz);
    const float2 du = __ffma2_rn(dz, uz, __ffma2_rn(dy, uy, __fmul2_rn(dx, ux)));
    const float2 hd = __fmul2_rn(hh, du);
    gx = __ffma2_rn(hd, dx, __ffma2_rn(f, ux, gx));
    gy = __ffma2_rn(hd, dy, __ffma2_rn(f, uy, gy));
    gz = __ffma2_rn(hd, dz, __ffma2_rn(f, uz, gz));
}

// Order of the neighbour table: the 27 cells within one cell of the sink cell
// (positions 0..26), then the 98 cells at Chebyshev distance 2, each group in
// (dx, dy, dz) lexicographic order.  code[p] = (dx+2)*25 + (dy+2)*5 + (dz+2).
constexpr int kNear = 27;
struct NbrOrder {
    unsigned char code[kNbr];
};
constexpr NbrOrder make_nbr_order()
{
    NbrOrder o{};
    int p = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int t = 0; t < kNbr; ++t) {
            const int dx = t / 25 - 2, dy = (t / 5) % 5 - 2, dz = t % 5 - 2;
            const bool near = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
            if (near == (pass == 0)) o.code[p++] = static_cast<unsigned char>(t);
        }
    return o;
}
__device__ const NbrOrder kNbrOrder = make_nbr_order();

// 125-entry neighbour table of `cell` in kNbrOrder: tstart[p] = first particle,
// tpre[p] = exclusive prefix of counts, tpre[125] = total, so sources
// [tpre[0], tpre[27]) are the near cells' and [tpre[27], total) the far cells'.
__device__ __forceinline__ int build_table(const BoxDev &bx, int cell, int *tstart, int *tpre, int lane)
{
    const int C = bx.cpd;
    const int cz = cell % C, cy = (cell / C) % C, cx = cell / (C * C);
    int cnt[4];
    int local = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int p = 4 * lane + u;
        int c = 0;
        if (p < kNbr) {
            const int t = __ldg(&kNbrOrder.code[p]);
            int nx = cx + t / 25 - 2, ny = cy + (t / 5) % 5 - 2, nz = cz + t % 5 - 2;
            nx += nx < 0 ? C : 0; nx -= nx >= C ? C : 0;
            ny += ny < 0 ? C : 0; ny -= ny >= C ? C : 0;
            nz += nz < 0 ? C : 0; nz -= nz >= C ? C : 0;
            const int n = (nx * C + ny) * C + nz;
            int s0 = __ldg(bx.cell_start + n);
            c = __ldg(bx.cell_start + n + 1) - s0;
            if (bx.dslot != nullptr && p >= kNear) {
                // cut-off mode: a dense far cell acts through its sub-cell moments, not
                // pair by pair; its entry holds -2 - (moment slot) and no sources
                const int ds = __ldg(bx.dslot + n);
                if (ds >= 0) {
                    c = 0;
                    s0 = -2 - ds;
                }
            }
            tstart[p] = s0;
        }
        cnt[u] = c;
        local += c;
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    int run = incl - local;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int p = 4 * lane + u;
        if (p <= kNbr) tpre[p] = run;
        run += cnt[u];
    }
    const int total = __shfl_sync(kFull, incl, 31);
    __syncwarp();
    return total;
}

// neighbour-table position of flat source index f: tpre[p] <= f < tpre[p+1]
__device__ __forceinline__ int find_cell(const int *tpre, int f)
{
    int lo = 0, hi = kNbr;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int mid = (lo + hi) >> 1;
        if (tpre[mid] <= f) lo = mid; else hi = mid;
    }
    return lo;
}

// Gather sources [base, base + B) of the flattened neighbourhood into buf
// (cp.async); entries past `total` become far-away padding.  The neighbour-table
// position of each gathered entry's cell (plus one; 0 = padding) goes to ts[]
// for the shift pass.
template <int B, bool ADJ>
__device__ __forceinline__ void stage_issue(const BoxDev &bx, float4 *buf, float4 *wbuf, const int *tstart,
                                            const int *tpre, int base, int total, int lane, unsigned char *ts)
{
    if (NF_STAGE_CONTIG) {
        // every lane copies B/32 consecutive entries: one search for the first, then the cell
        // only moves forward (entries past the end become far-away padding)
        constexpr int E = B / 32;
        int p = -1;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int slot = lane * E + m;
            const int f = base + slot;
            if (f < total) {
                if (p < 0) {
                    p = find_cell(tpre, f);
                } else {
                    while (tpre[p + 1] <= f) ++p;   // tpre[125] = total > f
                }
                const int src = tstart[p] + (f - tpre[p]);
                cp_async16(buf + slot, bx.pos + src);
                if (ADJ) cp_async16(wbuf + slot, bx.cot + src);
                ts[slot] = static_cast<unsigned char>(p + 1);
            } else {
                buf[slot] = make_float4(kFar, kFar, kFar, 0.f);
                if (ADJ) wbuf[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
                ts[slot] = 0;
            }
        }
        cp_async_commit();
        return;
    }
#pragma unroll
    for (int m = 0; m < B / 32; ++m) {
        const int f = base + m * 32 + lane;
        const int slot = m * 32 + lane;
        if (f < total) {
            const int p = find_cell(tpre, f);
            const int src = tstart[p] + (f - tpre[p]);
            cp_async16(buf + slot, bx.pos + src);
            if (ADJ) cp_async16(wbuf + slot, bx.cot + src);
            ts[slot] = static_cast<unsigned char>(p + 1);
        } else {
            buf[slot] = make_float4(kFar, kFar, kFar, 0.f);
            if (ADJ) wbuf[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
            ts[slot] = 0;
        }
    }
    cp_async_commit();
}

// add the integer cell offset of each of this lane's landed entries, read from
// the per-block table offtab (offtab[p + 1] = offset of neighbour-table position
// p, offtab[0] = 0 for padding); with SOA the round is then rewritten in place
// as three arrays x[B], y[B], z[B] (the layout the source-paired loops read two
// sources at a time from)
template <int B, bool SOA>
__device__ __forceinline__ void stage_shift(float4 *buf, int lane, const unsigned char *ts, const float4 *offtab)
{
    float4 v[B / 32];
#pragma unroll
    for (int m = 0; m < B / 32; ++m) {
        const float4 o = offtab[ts[m * 32 + lane]];
        v[m] = buf[m * 32 + lane];
        v[m].x += o.x;
        v[m].y += o.y;
        v[m].z += o.z;
    }
    if constexpr (SOA) {
        __syncwarp();   // every lane has read its entries before any array entry is written over them
        float *xs = reinterpret_cast<float *>(buf);
#pragma unroll
        for (int m = 0; m < B / 32; ++m) {
            const int slot = m * 32 + lane;
            xs[slot] = v[m].x;
            xs[B + slot] = v[m].y;
            xs[2 * B + slot] = v[m].z;
        }
    } else {
#pragma unroll
        for (int m = 0; m < B / 32; ++m) buf[m * 32 + lane] = v[m];
    }
}

// Compensated sums live in shared memory (per warp: 6 x 128 floats, word
// comp_slot(lane, s) of each array for the lane's sink s), so the registers
// hold only positions and the running FP32 partials of the current round.
// With NF_PAIRED_FOLD the sinks 2k and 2k + 1 of a lane are adjacent words,
// so both fold with paired FP32 instructions (each half exactly the scalar
// two-sum).
__device__ __forceinline__ int comp_slot(int lane, int s)
{
    return NF_PAIRED_FOLD ? 2 * lane + 64 * (s >> 1) + (s & 1) : lane + 32 * s;
}

// a - b with one rounding (b times -1 is exact inside the fused operation)
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    const float2 bp = fsub2(s, a);
    const float2 ap = fsub2(s, bp);
    e = __fadd2_rn(fsub2(a, ap), fsub2(b, bp));
}

// fold the partials of sinks 2k, 2k + 1 (c = comp + comp_slot(lane, 2k))
__device__ __forceinline__ void comp_fold_smem2(float *c, float2 &px, float2 &py, float2 &pz)
{
    float2 *h = reinterpret_cast<float2 *>(c);
    float2 s, e;
    two_sum2(h[0], px, s, e); h[0] = s; h[192] = __fadd2_rn(h[192], e);
    two_sum2(h[64], py, s, e); h[64] = s; h[256] = __fadd2_rn(h[256], e);
    two_sum2(h[128], pz, s, e); h[128] = s; h[320] = __fadd2_rn(h[320], e);
    px = py = pz = make_float2(0.f, 0.f);
}

__device__ __forceinline__ void comp_fold_smem(float *c, float &px, float &py, float &pz)
{
    float s, e;
    two_sum(c[0], px, s, e); c[0] = s; c[384] = __fadd_rn(c[384], e);
    two_sum(c[128], py, s, e); c[128] = s; c[512] = __fadd_rn(c[512], e);
    two_sum(c[256], pz, s, e); c[256] = s; c[640] = __fadd_rn(c[640], e);
    px = py = pz = 0.f;
}

// S = 0: split mode (<= 16 sinks); S = 1, 2, 4: sinks per lane.  Returns the
// number of sources the item evaluated for each of its sinks.
template <int S, int B, bool COMP, bool ADJ, int SOFT>
__device__ int run_item(const BoxDev &bx, const Item &item, float4 *stage, float4 *wstage, int *tstart, int *tpre,
                         float *comp, unsigned char *tslot, const float4 *offtab, int lane)
{
    constexpr bool SPLIT = (S == 0);
    constexpr int SS = SPLIT ? 1 : S;
    const int count = item_count(item);
    int logp = 0;
    if (SPLIT) {
        while ((1 << logp) < count) ++logp;
    }
    const int P = 1 << logp;
    const int my_split = SPLIT ? (lane >> logp) : 0;
    const int splits = SPLIT ? (32 >> logp) : 1;

    float xi[SS], yi[SS], zi[SS], wx[SS], wy[SS], wz[SS];
    float px[SS], py[SS], pz[SS];
#pragma unroll
    for (int s = 0; s < SS; ++s) {
        const int k = SPLIT ? (lane & (P - 1)) : lane + 32 * s;
        const int idx = item.sink_begin + min(k, count - 1);
        const float4 p = __ldg(bx.pos + idx);
        xi[s] = p.x; yi[s] = p.y; zi[s] = p.z;
        if (ADJ) {
            const float4 w = __ldg(bx.cot + idx);
            wx[s] = w.x; wy[s] = w.y; wz[s] = w.z;
        } else {
            wx[s] = wy[s] = wz[s] = 0.f;
        }
        px[s] = py[s] = pz[s] = 0.f;
        if (COMP) {
            float *c = comp + comp_slot(lane, s);
#pragma unroll
            for (int q = 0; q < 6; ++q) c[128 * q] = 0.f;
        }
    }
    const float a0 = bx.a0, a1 = bx.a1, a2 = bx.a2, eps2 = bx.eps2;
    // paired FP32 instructions: lanes with 2 or 4 sinks pair two sinks against one
    // source (PACK); lanes with one sink pair one sink against two sources
    // (PAIRSRC: even and odd sources of a round go to the two halves of a float2
    // partial sum, both folded into the sink's sum)
    constexpr bool PACK = NF_PACKED && !ADJ && SS >= 2;
    constexpr bool PACKA = NF_PACKED_ADJ && ADJ && SS >= 2;   // the adjoint, two sinks per paired instruction
    constexpr bool PAIRSRC = NF_PAIR_SOURCES && !ADJ && SS == 1;
    constexpr int SP = SS >= 2 ? SS / 2 : 1;
    float2 nx2[SP], ny2[SP], nz2[SP], ax2[SP], ay2[SP], az2[SP];
    float2 nwx2[SP], nwy2[SP], nwz2[SP];
    if (PACKA) {
#pragma unroll
        for (int k = 0; k < SP; ++k) {
            nwx2[k] = make_float2(-wx[2 * k], -wx[2 * k + 1]);
            nwy2[k] = make_float2(-wy[2 * k], -wy[2 * k + 1]);
            nwz2[k] = make_float2(-wz[2 * k], -wz[2 * k + 1]);
        }
    }
    if (PACK || PACKA) {
#pragma unroll
        for (int k = 0; k < SP; ++k) {
            nx2[k] = make_float2(-xi[2 * k], -xi[2 * k + 1]);
            ny2[k] = make_float2(-yi[2 * k], -yi[2 * k + 1]);
            nz2[k] = make_float2(-zi[2 * k], -zi[2 * k + 1]);
            ax2[k] = ay2[k] = az2[k] = make_float2(0.f, 0.f);
        }
    }
    if (PAIRSRC) {
        nx2[0] = make_float2(-xi[0], -xi[0]);
        ny2[0] = make_float2(-yi[0], -yi[0]);
        nz2[0] = make_float2(-zi[0], -zi[0]);
        ax2[0] = ay2[0] = az2[0] = make_float2(0.f, 0.f);
    }
    const float2 a02 = make_float2(a0, a0), a12 = make_float2(a1, a1), a22 = make_float2(a2, a2),
                 e22 = make_float2(eps2, eps2);

    const int total = build_table(bx, item.cell, tstart, tpre, lane);
    constexpr bool FARSPLIT = NF_FAR_LAW && SOFT == 0;
    // warp vote in the near cells for lanes holding 2 or 4 sinks, or one sink with
    // source pairs (for one sink and one source the vote costs more issue slots
    // than the spline tail it saves).  eps2 >= 2^-40 by
    // the softening-length bound, so a self pair's r^2 = FLT_MIN is always below it.
    constexpr bool VOTE = NF_NEAR_VOTE && FARSPLIT && !ADJ && SS >= 2;
    constexpr bool VOTE1 = NF_NEAR_VOTE && FARSPLIT && PAIRSRC && !SPLIT;   // one sink, source pairs
    constexpr bool VOTE_SPLIT = NF_NEAR_VOTE && FARSPLIT && PAIRSRC && SPLIT;   // <= 16 sinks, source pairs
    // the whole flattened neighbourhood, or this item's piece of it
    int src_lo = 0, src_hi = total;
    if (item.piece >= 0) {
        src_lo = __ldg(&bx.pieces[item.piece].src_lo);
        src_hi = min(__ldg(&bx.pieces[item.piece].src_hi), total);
    }
    const int rounds = src_hi > src_lo ? (src_hi - src_lo + B - 1) / B : 0;

    if (rounds > 0) stage_issue<B, ADJ>(bx, stage, wstage, tstart, tpre, src_lo, src_hi, lane, tslot);
    for (int r = 0; r < rounds; ++r) {
        const int bsel = r & 1;
        float4 *buf = stage + bsel * B;
        float4 *wbuf = wstage + bsel * B;
        if (r + 1 < rounds) {
            stage_issue<B, ADJ>(bx, stage + ((r + 1) & 1) * B, wstage + ((r + 1) & 1) * B, tstart, tpre,
                                src_lo + (r + 1) * B, src_hi, lane, tslot + ((r + 1) & 1) * B);
            cp_async_wait_1();
        } else {
            cp_async_wait_0();
        }
        // the shift pass reads entries other lanes copied (contiguous staging): their copies are
        // complete once each lane has passed its wait
        if (NF_STAGE_CONTIG) __syncwarp();
        stage_shift<B, PAIRSRC>(buf, lane, tslot + bsel * B, offtab);
        __syncwarp();
        const int nr = min(B, src_hi - src_lo - r * B);
        // this round's entries [0, nn) come from the 27 near cells and take the
        // full law; [nn, nr) come from far cells (spline law only: Plummer
        // softening acts at every distance)
        const int nn = (FARSPLIT && !ADJ) ? max(0, min(nr, tpre[kNear] - (src_lo + r * B))) : nr;
        const float2 *xs2 = reinterpret_cast<const float2 *>(buf);   // PAIRSRC layout: x, y, z arrays
        const float2 *ys2 = xs2 + B / 2, *zs2 = xs2 + B;
        if (SPLIT && PAIRSRC) {
            // Lane group g takes the source pairs g, g + splits, ... (pair m = entries 2m, 2m + 1),
            // two pairs per step.  Every lane runs the same number of steps: pairs past the round's
            // last entry are padding (exact zeros), and a round holds B/2 pairs, a multiple of
            // 2 splits, so the steps stay inside the buffer.  The warp therefore stays converged and
            // votes as the tiled paths do: a near step takes the spline tail only when some lane
            // finds a pair within eps.  The pair holding the last near entry counts as near (the
            // full law is exact for its far partner).
            const int nnp = (nn + 1) >> 1, nrp = (nr + 1) >> 1;
            const int n_near = ((nnp + splits - 1) / splits + 1) & ~1;
            const int n_all = ((nrp + splits - 1) / splits + 1) & ~1;
            for (int i = 0; i < n_near; i += 2) {
                const int m0 = my_split + i * splits, m1 = m0 + splits;
                if (VOTE_SPLIT) {
                    const float2 dx0 = __fadd2_rn(xs2[m0], nx2[0]), dy0 = __fadd2_rn(ys2[m0], ny2[0]),
                                 dz0 = __fadd2_rn(zs2[m0], nz2[0]);
                    const float2 dx1 = __fadd2_rn(xs2[m1], nx2[0]), dy1 = __fadd2_rn(ys2[m1], ny2[0]),
                                 dz1 = __fadd2_rn(zs2[m1], nz2[0]);
                    const float2 fm = make_float2(FLT_MIN, FLT_MIN);
                    const float2 r20 = __ffma2_rn(dz0, dz0, __ffma2_rn(dy0, dy0, __ffma2_rn(dx0, dx0, fm)));
                    const float2 r21 = __ffma2_rn(dz1, dz1, __ffma2_rn(dy1, dy1, __ffma2_rn(dx1, dx1, fm)));
                    if (__any_sync(kFull, fminf(fminf(r20.x, r20.y), fminf(r21.x, r21.y)) < eps2)) {
                        tail2_spline(dx0, dy0, dz0, r20, ax2[0], ay2[0], az2[0], a02, a12, a22);
                        tail2_spline(dx1, dy1, dz1, r21, ax2[0], ay2[0], az2[0], a02, a12, a22);
                    } else {
                        tail2_newton(dx0, dy0, dz0, r20, ax2[0], ay2[0], az2[0]);
                        tail2_newton(dx1, dy1, dz1, r21, ax2[0], ay2[0], az2[0]);
                    }
                } else {
                    pair_force2<SOFT>(xs2[m0], ys2[m0], zs2[m0], nx2[0], ny2[0], nz2[0], ax2[0], ay2[0], az2[0],
                                      a02, a12, a22, e22);
                    pair_force2<SOFT>(xs2[m1], ys2[m1], zs2[m1], nx2[0], ny2[0], nz2[0], ax2[0], ay2[0], az2[0],
                                      a02, a12, a22, e22);
                }
            }
            if (FARSPLIT)
                for (int i = n_near; i < n_all; i += 2) {
                    const int m0 = my_split + i * splits, m1 = m0 + splits;
                    pair_force2_far(xs2[m0], ys2[m0], zs2[m0], nx2[0], ny2[0], nz2[0], ax2[0], ay2[0], az2[0]);
                    pair_force2_far(xs2[m1], ys2[m1], zs2[m1], nx2[0], ny2[0], nz2[0], ax2[0], ay2[0], az2[0]);
                }
        } else if (PAIRSRC) {
            constexpr int U2 = NF_PAIR_UNROLL;
            const int nrp = (nr + 2 * U2 - 1) / (2 * U2) * U2;   // padding pairs add exact zeros
            const int nnp = FARSPLIT ? (nn + 2 * U2 - 1) / (2 * U2) * U2 : nrp;
            for (int m = 0; m < nnp; m += U2) {
#pragma unroll
                for (int u = 0; u < U2; ++u) {
                    const float2 qx = xs2[m + u], qy = ys2[m + u], qz = zs2[m + u];
                    if (VOTE1) {
                        const float2 dx = __fadd2_rn(qx, nx2[0]), dy = __fadd2_rn(qy, ny2[0]),
                                     dz = __fadd2_rn(qz, nz2[0]);
                        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy,
                                                     __ffma2_rn(dx, dx, make_float2(FLT_MIN, FLT_MIN))));
                        if (__any_sync(kFull, fminf(r2.x, r2.y) < eps2))
                            tail2_spline(dx, dy, dz, r2, ax2[0], ay2[0], az2[0], a02, a12, a22);
                        else
                            tail2_newton(dx, dy, dz, r2, ax2[0], ay2[0], az2[0]);
                    } else {
                        pair_force2<SOFT>(qx, qy, qz, nx2[0], ny2[0], nz2[0], ax2[0], ay2[0], az2[0], a02, a12,
                                          a22, e22);
                    }
                }
            }
            if (FARSPLIT)
                for (int m = nnp; m < nrp; m += U2) {
#pragma unroll
                    for (int u = 0; u < U2; ++u)
                        pair_force2_far(xs2[m + u], ys2[m + u], zs2[m + u], nx2[0], ny2[0], nz2[0], ax2[0], ay2[0],
                                        az2[0]);
                }
        } else if (SPLIT) {
            int j = my_split;
            for (; j < nn; j += splits) {
                if (ADJ)
                    pair_adjoint<SOFT>(buf[j], wbuf[j], xi[0], yi[0], zi[0], wx[0], wy[0], wz[0], px[0], py[0], pz[0], a0,
                                 a1, a2, eps2);
                else
                    pair_force<SOFT>(buf[j], xi[0], yi[0], zi[0], px[0], py[0], pz[0], a0, a1, a2, eps2);
            }
            if (FARSPLIT && !ADJ)
                for (; j < nr; j += splits) pair_force_far(buf[j], xi[0], yi[0], zi[0], px[0], py[0], pz[0]);
        } else {
            constexpr int U = ADJ ? NF_ADJ_UNROLL : SS == 2 ? NF_UNROLL_S2 : NF_SRC_UNROLL;
            // padding entries add exact zeros under either law; the near loop's last
            // step may take up to U - 1 far entries, which the full law treats exactly
            const int nru = (nr + U - 1) / U * U;
            const int nnu = (nn + U - 1) / U * U;
            for (int j = 0; j < nnu; j += U) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float4 q = buf[j + u];
                    if (VOTE && PACK) {
                        // a near source takes the spline tail only when some sink of the
                        // warp lies within eps of it (self pairs included: r^2 = FLT_MIN)
                        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                                     qz = make_float2(q.z, q.z);
                        float2 dx[SP], dy[SP], dz[SP], r2[SP];
                        float m = 0.f;
#pragma unroll
                        for (int k = 0; k < SP; ++k) {
                            dx[k] = __fadd2_rn(qx, nx2[k]);
                            dy[k] = __fadd2_rn(qy, ny2[k]);
                            dz[k] = __fadd2_rn(qz, nz2[k]);
                            r2[k] = __ffma2_rn(dz[k], dz[k], __ffma2_rn(dy[k], dy[k],
                                               __ffma2_rn(dx[k], dx[k], make_float2(FLT_MIN, FLT_MIN))));
                            const float mk = fminf(r2[k].x, r2[k].y);
                            m = k == 0 ? mk : fminf(m, mk);
                        }
                        if (__any_sync(kFull, m < eps2)) {
#pragma unroll
                            for (int k = 0; k < SP; ++k)
                                tail2_spline(dx[k], dy[k], dz[k], r2[k], ax2[k], ay2[k], az2[k], a02, a12, a22);
                        } else {
#pragma unroll
                            for (int k = 0; k < SP; ++k) tail2_newton(dx[k], dy[k], dz[k], r2[k], ax2[k], ay2[k], az2[k]);
                        }
                    } else if (VOTE) {
                        float dx[SS], dy[SS], dz[SS], r2[SS];
                        float m = 0.f;
#pragma unroll
                        for (int s = 0; s < SS; ++s) {
                            dx[s] = q.x - xi[s]; dy[s] = q.y - yi[s]; dz[s] = q.z - zi[s];
                            r2[s] = fmaf(dz[s], dz[s], fmaf(dy[s], dy[s], fmaf(dx[s], dx[s], FLT_MIN)));
                            m = s == 0 ? r2[s] : fminf(m, r2[s]);
                        }
                        if (__any_sync(kFull, m < eps2)) {
#pragma unroll
                            for (int s = 0; s < SS; ++s)
                                tail_spline(dx[s], dy[s], dz[s], r2[s], px[s], py[s], pz[s], a0, a1, a2);
                        } else {
#pragma unroll
                            for (int s = 0; s < SS; ++s) tail_newton(dx[s], dy[s], dz[s], r2[s], px[s], py[s], pz[s]);
                        }
                    } else if (PACK) {
                        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                                     qz = make_float2(q.z, q.z);
#pragma unroll
                        for (int k = 0; k < SP; ++k)
                            pair_force2<SOFT>(qx, qy, qz, nx2[k], ny2[k], nz2[k], ax2[k], ay2[k], az2[k], a02, a12,
                                              a22, e22);
                    } else if (PACKA) {
                        const float4 wq = wbuf[j + u];
                        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                                     qz = make_float2(q.z, q.z);
                        const float2 wjx = make_float2(wq.x, wq.x), wjy = make_float2(wq.y, wq.y),
                                     wjz = make_float2(wq.z, wq.z);
                        const float2 a2x2 = make_float2(2.f * a2, 2.f * a2);
#pragma unroll
                        for (int k = 0; k < SP; ++k)
                            pair_adjoint2<SOFT>(qx, qy, qz, wjx, wjy, wjz, nx2[k], ny2[k], nz2[k], nwx2[k], nwy2[k],
                                                nwz2[k], ax2[k], ay2[k], az2[k], a02, a12, a22, a2x2, eps2);
                    } else if (ADJ) {
                        const float4 wq = wbuf[j + u];
#pragma unroll
                        for (int s = 0; s < SS; ++s)
                            pair_adjoint<SOFT>(q, wq, xi[s], yi[s], zi[s], wx[s], wy[s], wz[s], px[s], py[s], pz[s], a0, a1,
                                         a2, eps2);
                    } else {
#pragma unroll
                        for (int s = 0; s < SS; ++s)
                            pair_force<SOFT>(q, xi[s], yi[s], zi[s], px[s], py[s], pz[s], a0, a1, a2, eps2);
                    }
                }
            }
            if (FARSPLIT && !ADJ)
                for (int j = nnu; j < nru; j += U) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const float4 q = buf[j + u];
                        if (PACK) {
                            const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                                         qz = make_float2(q.z, q.z);
#pragma unroll
                            for (int k = 0; k < SP; ++k)
                                pair_force2_far(qx, qy, qz, nx2[k], ny2[k], nz2[k], ax2[k], ay2[k], az2[k]);
                        } else {
#pragma unroll
                            for (int s = 0; s < SS; ++s) pair_force_far(q, xi[s], yi[s], zi[s], px[s], py[s], pz[s]);
                        }
                    }
                }
        }
        if (COMP) {
            if (PAIRSRC) {
                if (NF_FOLD_HALVES) {
                    // the two halves' sum rounds once per round, within the round's FP32 partial error
                    float hx = ax2[0].x + ax2[0].y, hy = ay2[0].x + ay2[0].y, hz = az2[0].x + az2[0].y;
                    comp_fold_smem(comp + comp_slot(lane, 0), hx, hy, hz);
                    ax2[0] = ay2[0] = az2[0] = make_float2(0.f, 0.f);
                } else {
                    comp_fold_smem(comp + comp_slot(lane, 0), ax2[0].x, ay2[0].x, az2[0].x);
                    comp_fold_smem(comp + comp_slot(lane, 0), ax2[0].y, ay2[0].y, az2[0].y);
                }
            } else if (PACK || PACKA) {
#pragma unroll
                for (int k = 0; k < SP; ++k) {
                    if (NF_PAIRED_FOLD) {
                        comp_fold_smem2(comp + comp_slot(lane, 2 * k), ax2[k], ay2[k], az2[k]);
                    } else {
                        comp_fold_smem(comp + comp_slot(lane, 2 * k), ax2[k].x, ay2[k].x, az2[k].x);
                        comp_fold_smem(comp + comp_slot(lane, 2 * k + 1), ax2[k].y, ay2[k].y, az2[k].y);
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < SS; ++s) comp_fold_smem(comp + comp_slot(lane, s), px[s], py[s], pz[s]);
            }
        }
        __syncwarp();
    }
    if (PAIRSRC && !COMP) {
        px[0] = ax2[0].x + ax2[0].y;
        py[0] = ay2[0].x + ay2[0].y;
        pz[0] = az2[0].x + az2[0].y;
    }
    if ((PACK || PACKA) && !COMP) {
#pragma unroll
        for (int k = 0; k < SP; ++k) {
            px[2 * k] = ax2[k].x; py[2 * k] = ay2[k].x; pz[2 * k] = az2[k].x;
            px[2 * k + 1] = ax2[k].y; py[2 * k + 1] = ay2[k].y; pz[2 * k + 1] = az2[k].y;
        }
    }
    // cut-off mode: the dense far cells, once per item (by its first source piece)
    if (SOFT == 0 && !ADJ && bx.mpole != nullptr &&
        (item.piece < 0 || __ldg(&bx.pieces[item.piece].src_lo) == 0)) {
        float sxp[SS], syp[SS], szp[SS], mx[SS], my[SS], mz[SS];
#pragma unroll
        for (int s = 0; s < SS; ++s) {
            const int k = SPLIT ? (lane & (P - 1)) : lane + 32 * s;
            const float4 p = __ldg(bx.pos + item.sink_begin + min(k, count - 1));
            sxp[s] = p.x; syp[s] = p.y; szp[s] = p.z;
            mx[s] = my[s] = mz[s] = 0.f;
        }
        // in split mode the sub-cells are shared out over the lane groups, whose sums
        // the xor tree below adds, so each sub-cell counts once
        const int q0 = SPLIT ? my_split : 0, dq = SPLIT ? splits : 1;
        float *moments = reinterpret_cast<float *>(stage);   // free once the last round is done
        for (int pp = kNear; pp < kNbr; ++pp) {
            const int ts = tstart[pp];
            if (ts > -2) continue;
            const float4 *src = reinterpret_cast<const float4 *>(bx.mpole) +
                                static_cast<int64_t>(-2 - ts) * (kCutSub * kCutWords / 4);
            const int t = __ldg(&kNbrOrder.code[pp]);
            const float ox = static_cast<float>(t / 25 - 2), oy = static_cast<float>((t / 5) % 5 - 2),
                        oz = static_cast<float>(t % 5 - 2);
            // the dense cell's sub-cell words fit the two staging buffers
            static_assert(kCutSub * kCutWords / 4 <= 2 * B, "moments exceed the staging area");
            __syncwarp();
            for (int k = lane; k < kCutSub * kCutWords / 4; k += 32) stage[k] = __ldg(src + k);
            __syncwarp();
            for (int q = q0; q < kCutSub; q += dq) {
                const float *o = moments + q * kCutWords;
                const float M = o[0];
                if (M == 0.f) continue;
                const float cx = o[1] + ox, cy = o[2] + oy, cz = o[3] + oz;
#pragma unroll
                for (int s = 0; s < SS; ++s) quad_force(cx - sxp[s], cy - syp[s], cz - szp[s], M, o + 4, mx[s], my[s], mz[s]);
            }
            // one FP32 partial per dense cell, in the accumulators' scale, folded like a round of sources
#pragma unroll
            for (int s = 0; s < SS; ++s) {
                mx[s] *= kForceSigma; my[s] *= kForceSigma; mz[s] *= kForceSigma;
                if (COMP) {
                    comp_fold_smem(comp + comp_slot(lane, s), mx[s], my[s], mz[s]);
                } else {
                    px[s] += mx[s]; py[s] += my[s]; pz[s] += mz[s];
                    mx[s] = my[s] = mz[s] = 0.f;
                }
            }
        }
        __syncwarp();
    }
    Comp3 acc[SS];
#pragma unroll
    for (int s = 0; s < SS; ++s) {
        if (COMP) {
            const float *c = comp + comp_slot(lane, s);
            acc[s].hx = c[0]; acc[s].hy = c[128]; acc[s].hz = c[256];
            acc[s].lx = c[384]; acc[s].ly = c[512]; acc[s].lz = c[640];
        } else {
            acc[s].hx = px[s]; acc[s].hy = py[s]; acc[s].hz = pz[s];
            acc[s].lx = acc[s].ly = acc[s].lz = 0.f;
        }
    }
    if (SPLIT) {
        for (int o = P; o < 32; o <<= 1) {
            if (COMP) {
                comp_xor_combine(acc[0], o);
            } else {
                acc[0].hx += __shfl_xor_sync(kFull, acc[0].hx, o);
                acc[0].hy += __shfl_xor_sync(kFull, acc[0].hy, o);
                acc[0].hz += __shfl_xor_sync(kFull, acc[0].hz, o);
            }
        }
    }
    if (item.piece >= 0) {
        // a piece of a split item: FP64 partial sums (cell units), reduced later in piece order
        const int slot = __ldg(&bx.pieces[item.piece].slot);
#pragma unroll
        for (int s = 0; s < SS; ++s) {
            const int k = SPLIT ? lane : lane + 32 * s;
            if (k < count) {
                double *o = bx.partials + 3 * (static_cast<int64_t>(slot) + k);
                o[0] = static_cast<double>(acc[s].hx) + static_cast<double>(acc[s].lx);
                o[1] = static_cast<double>(acc[s].hy) + static_cast<double>(acc[s].ly);
                o[2] = static_cast<double>(acc[s].hz) + static_cast<double>(acc[s].lz);
            }
        }
        return src_hi - src_lo;
    }
    const double scale = ADJ ? bx.grad_scale : bx.acc_scale * kForceUnscale;
#pragma unroll
    for (int s = 0; s < SS; ++s) {
        const int k = SPLIT ? lane : lane + 32 * s;
        if (k < count) {
            const int idx = item.sink_begin + k;
            const double gx = (static_cast<double>(acc[s].hx) + static_cast<double>(acc[s].lx)) * scale;
            const double gy = (static_cast<double>(acc[s].hy) + static_cast<double>(acc[s].ly)) * scale;
            const double gz = (static_cast<double>(acc[s].hz) + static_cast<double>(acc[s].lz)) * scale;
            if (bx.acc64) {
                double *o = bx.acc64 + 3 * static_cast<int64_t>(idx);
                o[0] = gx; o[1] = gy; o[2] = gz;
            }
            if (bx.acc_out)
                bx.acc_out[idx] =
                    make_float4(static_cast<float>(gx), static_cast<float>(gy), static_cast<float>(gz), 0.f);
        }
    }
    return src_hi - src_lo;
}

// Forces of a lane item when every stored position carries its cell's z index
// in w (BoxDev::zcell, boxes the library loaded).  Each lane walks its 25
// (dx, dy) columns as run_lanes does, but a source's z offset is w + zoff (an
// exact small integer; zoff is constant over each contiguous run of a column,
// two runs where the column wraps the box in z), so a run needs only its two
// cell boundaries, and each lane evaluates two consecutive sources per paired
// FP32 instruction, two such pairs per step (an odd last source is paired with
// far-away padding, an exact zero; a second pair with no source is skipped).  Separations
// stay exact: (w + zoff) - x_i and x_j + that are sums on the 2^-22 grid below
// 4 in magnitude.  Columns at |dx| = 2 or |dy| = 2 take the Newtonian law;
// in the others a source pair takes the branch-free law only when one of its
// pairs lies within eps (self pairs included: r^2 = FLT_MIN).
template <bool COMP, int SOFT>
__device__ void run_lanes_paired(const BoxDev &bx, const Item &item, int lane)
{
    const int count = item_count(item);
    if (lane >= count) return;
    const int C = bx.cpd;
    const int *cs = bx.cell_start;
    const int g0 = item.cell, ng = item_lane_cells(item);
    const int i = item.sink_begin + lane;
    int c = g0;   // the sink's cell: the last of the run starting at or before i
    for (int k = 1; k < ng; ++k) c += __ldg(cs + g0 + k) <= i;
    const int cz = c % C, cy = (c / C) % C, cx = c / (C * C);
    const float4 p = __ldg(bx.pos + i);
    const float eps2 = bx.eps2;
    const float2 a02 = make_float2(bx.a0, bx.a0), a12 = make_float2(bx.a1, bx.a1), a22 = make_float2(bx.a2, bx.a2);
    const float2 e22 = make_float2(eps2, eps2), fmin2 = make_float2(FLT_MIN, FLT_MIN);
    Comp3 acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool wrap_lo = cz < 2, wrap_hi = cz + 3 > C;   // never both: C >= 5
    for (int col = 0; col < 25; ++col) {
        const int dxi = col / 5 - 2, dyi = col % 5 - 2;
        int nx = cx + dxi, ny = cy + dyi;
        nx += nx < 0 ? C : 0; nx -= nx >= C ? C : 0;
        ny += ny < 0 ? C : 0; ny -= ny >= C ? C : 0;
        const int *row = cs + (nx * C + ny) * C;
        const float ox = static_cast<float>(dxi) - p.x, oy = static_cast<float>(dyi) - p.y;   // exact
        // warp-uniform (every lane walks the columns in the same order)
        const bool far_col = dxi == -2 || dxi == 2 || dyi == -2 || dyi == 2;
        float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
        for (int part = 0; part < 2; ++part) {
            // cells [z0, z1) of the row; a source in cell z lies at z offset z + zoff
            int z0, z1, zoff;
            if (part == 0) {
                z0 = wrap_lo ? cz - 2 + C : cz - 2;
                z1 = wrap_lo ? C : min(cz + 3, C);
                zoff = wrap_lo ? -cz - C : -cz;
            } else {
                if (!wrap_lo && !wrap_hi) break;
                z0 = 0;
                z1 = wrap_lo ? cz + 3 : cz + 3 - C;
                zoff = wrap_lo ? -cz : C - cz;
            }
            const int j0 = __ldg(row + z0), j1 = __ldg(row + z1);
            // one source pair: (w + zoff) is the integer z offset; minus x_i, plus x_j: each step exact
            auto pair = [&](const float4 &q0, const float4 &q1) {
                // scalar adds write each half of the pairs directly: the two sources' words sit in
                // separate float4 registers, so a paired add would first need them moved side by side
                // (6 % faster lane items than paired adds; the same roundings, so the same values)
                const float zf = static_cast<float>(zoff);
                const float2 dx = make_float2(q0.x + ox, q1.x + ox);
                const float2 dy = make_float2(q0.y + oy, q1.y + oy);
                const float2 dz = make_float2(q0.z + ((q0.w + zf) - p.z), q1.z + ((q1.w + zf) - p.z));
                if (SOFT == 1) {
                    tail2_newton(dx, dy, dz, __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, e22))), ax,
                                 ay, az);
                } else {
                    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, fmin2)));
                    if (!far_col && fminf(r2.x, r2.y) < eps2)
                        tail2_spline(dx, dy, dz, r2, ax, ay, az, a02, a12, a22);
                    else
                        tail2_newton(dx, dy, dz, r2, ax, ay, az);
                }
            };
            const float4 pad = make_float4(kFar, kFar, kFar, 0.f);
            if (NF_LANE_PAIR_UNROLL == 2) {
                // two source pairs per step, their four loads issued together; a second pair
                // with no source left is skipped
                for (int j = j0; j < j1; j += 4) {
                    const float4 q0 = __ldg(bx.pos + j);
                    const float4 q1 = j + 1 < j1 ? __ldg(bx.pos + j + 1) : pad;
                    const float4 q2 = j + 2 < j1 ? __ldg(bx.pos + j + 2) : pad;
                    const float4 q3 = j + 3 < j1 ? __ldg(bx.pos + j + 3) : pad;
                    pair(q0, q1);
                    if (j + 2 < j1) pair(q2, q3);
                }
            } else {
                for (int j = j0; j < j1; j += 2) {
                    const float4 q0 = __ldg(bx.pos + j);
                    const float4 q1 = j + 1 < j1 ? __ldg(bx.pos + j + 1) : pad;
                    pair(q0, q1);
                }
            }
        }
        const float px = ax.x + ax.y, py = ay.x + ay.y, pz = az.x + az.y;
        if (COMP) {
            float s, e;
            two_sum(acc.hx, px, s, e); acc.hx = s; acc.lx = __fadd_rn(acc.lx, e);
            two_sum(acc.hy, py, s, e); acc.hy = s; acc.ly = __fadd_rn(acc.ly, e);
            two_sum(acc.hz, pz, s, e); acc.hz = s; acc.lz = __fadd_rn(acc.lz, e);
        } else {
            acc.hx += px; acc.hy += py; acc.hz += pz;
        }
    }
    const double scale = bx.acc_scale * kForceUnscale;
    const double gx = (static_cast<double>(acc.hx) + static_cast<double>(acc.lx)) * scale;
    const double gy = (static_cast<double>(acc.hy) + static_cast<double>(acc.ly)) * scale;
    const double gz = (static_cast<double>(acc.hz) + static_cast<double>(acc.lz)) * scale;
    if (bx.acc64) {
        double *o = bx.acc64 + 3 * static_cast<int64_t>(i);
        o[0] = gx; o[1] = gy; o[2] = gz;
    }
    if (bx.acc_out)
        bx.acc_out[i] = make_float4(static_cast<float>(gx), static_cast<float>(gy), static_cast<float>(gz), 0.f);
}

// A lane item (a run of sparse cells, <= 32 sinks): every lane takes one sink
// against its own neighbourhood, read straight from global memory (L1) as the
// 25 (dx, dy) columns of five z-cells.  The five cells of a column are one
// contiguous particle run (two where the column wraps the box in z), and a
// source's dz follows from the cell boundaries inside the run.  Separations are
// exact as on the staged path: (x_j + D) - x_i on the 2^-22 grid.  Lanes work
// independently (no warp-synchronous step); columns at |dx| = 2 or |dy| = 2
// take the Newtonian law, the others the branch-free law.  Used by the adjoint
// and by boxes whose positions lack the z index (nf_forces_noalloc).
template <bool COMP, bool ADJ, int SOFT>
__device__ void run_lanes(const BoxDev &bx, const Item &item, int lane)
{
    const int count = item_count(item);
    if (lane >= count) return;
    const int C = bx.cpd;
    const int *cs = bx.cell_start;
    const int g0 = item.cell, ng = item_lane_cells(item);
    const int i = item.sink_begin + lane;
    int c = g0;   // the sink's cell: the last of the run starting at or before i
    for (int k = 1; k < ng; ++k) c += __ldg(cs + g0 + k) <= i;
    const int cz = c % C, cy = (c / C) % C, cx = c / (C * C);
    const float4 p = __ldg(bx.pos + i);
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ADJ) w = __ldg(bx.cot + i);
    const float a0 = bx.a0, a1 = bx.a1, a2 = bx.a2, eps2 = bx.eps2;
    Comp3 acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool wrap_lo = cz < 2, wrap_hi = cz + 3 > C;   // never both: C >= 5
    for (int col = 0; col < 25; ++col) {
        const int dxi = col / 5 - 2, dyi = col % 5 - 2;
        int nx = cx + dxi, ny = cy + dyi;
        nx += nx < 0 ? C : 0; nx -= nx >= C ? C : 0;
        ny += ny < 0 ? C : 0; ny -= ny >= C ? C : 0;
        const int *row = cs + (nx * C + ny) * C;
        const float fx = static_cast<float>(dxi), fy = static_cast<float>(dyi);
        const float ox = fx - p.x, oy = fy - p.y;   // exact: the 2^-22 grid, |.| < 3
        // every lane walks the columns in the same order, so this is warp-uniform: a
        // column with |dx| = 2 or |dy| = 2 lies beyond eps and takes the Newtonian law
        const bool far_col = SOFT == 0 && !ADJ && (dxi == -2 || dxi == 2 || dyi == -2 || dyi == 2);
        for (int part = 0; part < 2; ++part) {
            // cells [z0, z1) of the row; the first has z offset dz0
            int z0, z1, dz0;
            if (part == 0) {
                z0 = wrap_lo ? cz - 2 + C : cz - 2;
                z1 = wrap_lo ? C : min(cz + 3, C);
                dz0 = -2;
            } else {
                if (!wrap_lo && !wrap_hi) break;
                z0 = 0;
                z1 = wrap_lo ? cz + 3 : cz + 3 - C;
                dz0 = wrap_lo ? -cz : C - cz;
            }
            const int m = z1 - z0;
            const int j0 = __ldg(row + z0), j1 = __ldg(row + z1);
            if (j0 == j1) continue;
            const int b1 = m > 1 ? __ldg(row + z0 + 1) : INT_MAX;
            const int b2 = m > 2 ? __ldg(row + z0 + 2) : INT_MAX;
            const int b3 = m > 3 ? __ldg(row + z0 + 3) : INT_MAX;
            const int b4 = m > 4 ? __ldg(row + z0 + 4) : INT_MAX;
            float px = 0.f, py = 0.f, pz = 0.f;
            if (ADJ) {
                for (int j = j0; j < j1; ++j) {
                    const float4 q0 = __ldg(bx.pos + j);
                    const int dz = dz0 + (j >= b1) + (j >= b2) + (j >= b3) + (j >= b4);
                    const float4 q = make_float4(q0.x + fx, q0.y + fy, q0.z + static_cast<float>(dz), 0.f);
                    pair_adjoint<SOFT>(q, __ldg(bx.cot + j), p.x, p.y, p.z, w.x, w.y, w.z, px, py, pz, a0, a1, a2,
                                       eps2);
                }
            } else {
                // NF_LANE_UNROLL sources per step, their loads issued together; entries past the
                // run become far-away padding (exact zeros under either law)
                constexpr int LU = NF_LANE_UNROLL;
                const bool newton = NF_LANE_FAR_LAW && far_col;
                for (int j = j0; j < j1; j += LU) {
                    float4 q0[LU];
#pragma unroll
                    for (int u = 0; u < LU; ++u)
                        q0[u] = (u == 0 || j + u < j1) ? __ldg(bx.pos + j + u) : make_float4(kFar, kFar, kFar, 0.f);
#pragma unroll
                    for (int u = 0; u < LU; ++u) {
                        const int ju = j + u;
                        const int dz = dz0 + (ju >= b1) + (ju >= b2) + (ju >= b3) + (ju >= b4);
                        if (newton) {
                            // d = x_j + D - x_i, exact (each sum lies on the 2^-22 grid)
                            const float ddx = q0[u].x + ox, ddy = q0[u].y + oy,
                                        ddz = q0[u].z + (static_cast<float>(dz) - p.z);
                            tail_newton(ddx, ddy, ddz, fmaf(ddz, ddz, fmaf(ddy, ddy, ddx * ddx)), px, py, pz);
                        } else {
                            const float4 q = make_float4(q0[u].x + fx, q0[u].y + fy, q0[u].z + static_cast<float>(dz),
                                                         0.f);
                            pair_force<SOFT>(q, p.x, p.y, p.z, px, py, pz, a0, a1, a2, eps2);
                        }
                    }
                }
            }
            if (COMP) {
                float s, e;
                two_sum(acc.hx, px, s, e); acc.hx = s; acc.lx = __fadd_rn(acc.lx, e);
                two_sum(acc.hy, py, s, e); acc.hy = s; acc.ly = __fadd_rn(acc.ly, e);
                two_sum(acc.hz, pz, s, e); acc.hz = s; acc.lz = __fadd_rn(acc.lz, e);
            } else {
                acc.hx += px; acc.hy += py; acc.hz += pz;
            }
        }
    }
    const double scale = ADJ ? bx.grad_scale : bx.acc_scale * kForceUnscale;
    const double gx = (static_cast<double>(acc.hx) + static_cast<double>(acc.lx)) * scale;
    const double gy = (static_cast<double>(acc.hy) + static_cast<double>(acc.ly)) * scale;
    const double gz = (static_cast<double>(acc.hz) + static_cast<double>(acc.lz)) * scale;
    if (bx.acc64) {
        double *o = bx.acc64 + 3 * static_cast<int64_t>(i);
        o[0] = gx; o[1] = gy; o[2] = gz;
    }
    if (bx.acc_out)
        bx.acc_out[i] = make_float4(static_cast<float>(gx), static_cast<float>(gy), static_cast<float>(gz), 0.f);
}

constexpr int kOffTab = 128;   // entries of the per-block cell-offset table (positions 0..124, plus one)

// per-warp shared memory, in float4 units: staged sources (and cotangents),
// compensated sums, neighbour table (256 ints), table slots (B bytes for each of the two buffers)
template <int B, bool COMP, bool ADJ>
__host__ __device__ constexpr int per_warp_f4()
{
    return (ADJ ? 4 : 2) * B + (COMP ? 192 : 0) + 64 + B / 8;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int B, bool COMP, bool ADJ, int SOFT>
__global__ void __launch_bounds__(256, NF_MIN_BLOCKS) pair_kernel(const BoxDev *__restrict__ boxes,
                                                                  const Item *__restrict__ items,
                                                                  const int *__restrict__ n_items_p,
                                                                  int *__restrict__ queue,
                                                                  unsigned long long *__restrict__ prof)
{
    extern __shared__ __align__(16) float4 smem_f4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *w0 = smem_f4 + warp * per_warp_f4<B, COMP, ADJ>();
    float4 *stage = w0;
    constexpr int SB = (ADJ ? 4 : 2) * B;   // two buffers of staged sources (and cotangents)
    float4 *wstage = stage + 2 * B;
    float *comp = reinterpret_cast<float *>(w0 + SB);
    int *tabs = reinterpret_cast<int *>(w0 + SB + (COMP ? 192 : 0));
    int *tstart = tabs, *tpre = tabs + 128;
    unsigned char *tslot = reinterpret_cast<unsigned char *>(tabs + 256);
    // after every warp's area: the cell offset of each neighbour-table position (index
    // position + 1; 0: padding)
    float4 *offtab = smem_f4 + (blockDim.x >> 5) * per_warp_f4<B, COMP, ADJ>();
    for (int t1 = threadIdx.x; t1 < kOffTab; t1 += blockDim.x) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t1 >= 1 && t1 <= kNbr) {
            const int t = kNbrOrder.code[t1 - 1];
            o = make_float4(static_cast<float>(t / 25 - 2), static_cast<float>((t / 5) % 5 - 2),
                            static_cast<float>(t % 5 - 2), 0.f);
        }
        offtab[t1] = o;
    }
    __syncthreads();
    const int n_items = *n_items_p;
    long long life0 = 0;
    unsigned long long wall0 = 0;
    if (prof) {
        life0 = clock64();
        wall0 = global_ns();
    }
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(queue, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const Item item = items[it];
        const BoxDev &bx = boxes[item_box(item)];
        const int cnt = item_count(item);
        const long long t0 = prof ? clock64() : 0;
        int kind, srcs = 0;
        if (item_is_lanes(item)) {
            if (!ADJ && NF_LANE_PAIRED && bx.zcell)
                run_lanes_paired<COMP, SOFT>(bx, item, lane);
            else
                run_lanes<COMP, ADJ, SOFT>(bx, item, lane);
            kind = 4;
        } else if (cnt <= 16) {
            srcs = run_item<0, B, COMP, ADJ, SOFT>(bx, item, stage, wstage, tstart, tpre, comp, tslot, offtab,
                                                          lane);
            kind = 3;
        } else if (cnt <= 32) {
            srcs = run_item<1, B, COMP, ADJ, SOFT>(bx, item, stage, wstage, tstart, tpre, comp, tslot, offtab,
                                                          lane);
            kind = 2;
        } else if (cnt <= 64) {
            srcs = run_item<2, B, COMP, ADJ, SOFT>(bx, item, stage, wstage, tstart, tpre, comp, tslot, offtab,
                                                          lane);
            kind = 1;
        } else {
            srcs = run_item<4, B, COMP, ADJ, SOFT>(bx, item, stage, wstage, tstart, tpre, comp, tslot, offtab,
                                                          lane);
            kind = 0;
        }
        __syncwarp();
        if (prof && lane == 0) {
            const int cls = 2 * kind + (item.piece >= 0 ? 1 : 0);
            atomicAdd(prof + 3 * cls, static_cast<unsigned long long>(clock64() - t0));
            atomicAdd(prof + 3 * cls + 1, 1ull);
            atomicAdd(prof + 3 * cls + 2, static_cast<unsigned long long>(cnt) * static_cast<unsigned long long>(srcs));
        }
    }
    if (prof && lane == 0) {
        atomicAdd(prof + kProfWarp, static_cast<unsigned long long>(clock64() - life0));
        atomicAdd(prof + kProfWarp + 1, 1ull);
        atomicMax(prof + kProfWarp + 2, ~wall0);
        atomicMax(prof + kProfWarp + 3, global_ns());
    }
}

template <int B, bool COMP, bool ADJ>
size_t smem_bytes(int warps)
{
    return (static_cast<size_t>(warps) * per_warp_f4<B, COMP, ADJ>() + kOffTab) * sizeof(float4);
}

// Occupancy of one instantiation at `warps` warps per block on the current
// device, computed once per device (the dynamic shared-memory limit is raised
// once per device to the 8-warp size), so a later launch makes no attribute or
// occupancy query and can be stream-captured.  Safe to call from several
// threads.
constexpr int kMaxDev = 64;
std::mutex g_occ_mu;

template <int B, bool COMP, bool ADJ, int SOFT>
int blocks_per_sm(int warps)
{
    static int cache[kMaxDev][9];
    static bool attr[kMaxDev] = {};
    static bool init = false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lk(g_occ_mu);
    if (!init) {
        for (int d = 0; d < kMaxDev; ++d)
            for (int w = 0; w < 9; ++w) cache[d][w] = -1;
        init = true;
    }
    auto kern = pair_kernel<B, COMP, ADJ, SOFT>;
    if (!attr[dev]) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem_bytes<B, COMP, ADJ>(8))) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        attr[dev] = true;
    }
    if (cache[dev][warps] < 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem_bytes<B, COMP, ADJ>(warps)) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cache[dev][warps] = per_sm;
    }
    return cache[dev][warps];
}

template <int B, bool COMP, bool ADJ, int SOFT>
cudaError_t launch_t(const BoxDev *boxes, const Item *items, const int *n_items, int *queue, PairShape shape,
                     int sm_count, cudaStream_t st, unsigned long long *prof)
{
    const int per_sm = blocks_per_sm<B, COMP, ADJ, SOFT>(shape.warps);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int blocks = shape.blocks > 0 ? shape.blocks : sm_count * per_sm;
    pair_kernel<B, COMP, ADJ, SOFT><<<blocks, shape.warps * 32, smem_bytes<B, COMP, ADJ>(shape.warps), st>>>(
        boxes, items, n_items, queue, prof);
    return cudaGetLastError();
}

template <int B, bool COMP, bool ADJ, int SOFT>
int max_blocks_t(PairShape shape)
{
    return blocks_per_sm<B, COMP, ADJ, SOFT>(shape.warps);
}

}  // namespace

#define NF_PAIR_DISPATCH_S(FN, SOFT, ...)                                                                          \
    do {                                                                                                            \
        if (shape.stage == 256) {                                                                                   \
            if (adjoint)                                                                                            \
                return compensated ? FN<256, true, true, SOFT>(__VA_ARGS__) : FN<256, false, true, SOFT>(__VA_ARGS__); \
            return compensated ? FN<256, true, false, SOFT>(__VA_ARGS__) : FN<256, false, false, SOFT>(__VA_ARGS__); \
        }                                                                                                           \
        if (adjoint)                                                                                                \
            return compensated ? FN<NF_STAGE_A, true, true, SOFT>(__VA_ARGS__)                                      \
                               : FN<NF_STAGE_A, false, true, SOFT>(__VA_ARGS__);                                    \
        return compensated ? FN<NF_STAGE_A, true, false, SOFT>(__VA_ARGS__)                                         \
                           : FN<NF_STAGE_A, false, false, SOFT>(__VA_ARGS__);                                       \
    } while (0)

#define NF_PAIR_DISPATCH(FN, ...)                                                                                   \
    do {                                                                                                            \
        if (softening == 1) NF_PAIR_DISPATCH_S(FN, 1, __VA_ARGS__);                                                 \
        NF_PAIR_DISPATCH_S(FN, 0, __VA_ARGS__);                                                                     \
    } while (0)

cudaError_t launch_pair(const BoxDev *boxes, const Item *items, const int *n_items, int *queue, int compensated,
                        int adjoint, int softening, PairShape shape, int sm_count, cudaStream_t st,
                        unsigned long long *prof)
{
    if (shape.warps < 1 || shape.warps > 8 || (shape.stage != 128 && shape.stage != 256)) return cudaErrorInvalidValue;
    NF_PAIR_DISPATCH(launch_t, boxes, items, n_items, queue, shape, sm_count, st, prof);
}

int pair_max_blocks_per_sm(int compensated, int adjoint, int softening, PairShape shape)
{
    if (shape.warps < 1 || shape.warps > 8 || (shape.stage != 128 && shape.stage != 256)) return 0;
    NF_PAIR_DISPATCH(max_blocks_t, shape);
}

}  // namespace nf
