// nf_bin.cuh -- the binning rule shared by initial binning and re-binning.
//
// Given a coordinate s in cell units (s = x cpd / box), the particle's cell
// along that axis is c = floor(s) wrapped into [0, cpd), and its offset from
// the cell centre is x_rel = (s - c) - 1/2, rounded once from its exact value
// to a multiple of 2^-22 cell widths (half to even; a negative offset that
// rounds to zero keeps its sign).
//
// The rounding is taken on S = s 2^22, which is exact: in quanta the offset is
// S - K with K = c 2^22 + 2^21, an even integer, and round-half-to-even
// commutes with subtracting an even integer, so q = rint(S) - K.  Forming
// (s - c) - 1/2 in double first would round a second time when -1 < s < 1/4
// and s has bits below 2^-53.  rint(S) and floor(S) come from two conversions
// to int64, floor(s) = floor(S) >> 22, and everything after is integer work.
// FP64 arithmetic is slow on this part, so the drift builds S directly.
#pragma once

#include <cmath>
#include <cstdint>

namespace nf {

constexpr double kTwo22 = 4194304.0;
constexpr double kTwoM22 = 2.384185791015625e-07;
constexpr double kScaledLimit = 4611686018427387904.0;   // 2^62: |S| below it fits the int64 conversions

__device__ __forceinline__ int wrap_cell(long long c, int cpd)
{
    if (c >= -cpd && c < 2LL * cpd) return static_cast<int>(c < 0 ? c + cpd : (c >= cpd ? c - cpd : c));
    const long long r = c % cpd;
    return static_cast<int>(r < 0 ? r + cpd : r);
}

// the rule on S = s 2^22, |S| < 2^62
__device__ __forceinline__ void bin_scaled(double S, int cpd, int &cell, float &xq)
{
    const long long F = __double2ll_rd(S);   // floor(S)
    const long long R = __double2ll_rn(S);   // rint(S), half to even
    const long long c = F >> 22;             // floor(s): arithmetic shift floors
    const int q = static_cast<int>(R - (c << 22) - (1LL << 21));   // in [-2^21, 2^21]
    // q == 0 with S < R (equivalently floor(S) < R) is a negative offset rounded to zero
    xq = (q == 0 && F < R) ? -0.f : static_cast<float>(q) * 2.384185791015625e-07f;
    cell = wrap_cell(c, cpd);
}

__device__ __forceinline__ bool bin_cell_units(double s, int cpd, int &cell, float &xq)
{
    const double S = __dmul_rn(s, kTwo22);
    if (fabs(S) < kScaledLimit) {
        bin_scaled(S, cpd, cell, xq);
        return true;
    }
    if (!(fabs(s) < 4503599627370496.0)) return false;   // non-finite or beyond 2^52
    // 2^40 <= |s| < 2^52: s is a multiple of 2^-12, so (s - c) - 1/2 is exact in double
    const double c = floor(s);
    const double q = rint(__dmul_rn(__dsub_rn(__dsub_rn(s, c), 0.5), kTwo22));
    xq = static_cast<float>(__dmul_rn(q, kTwoM22));
    const double d = static_cast<double>(cpd);
    const double cw = __dsub_rn(c, __dmul_rn(d, floor(__ddiv_rn(c, d))));
    int ci = static_cast<int>(cw);
    ci = ci < 0 ? ci + cpd : (ci >= cpd ? ci - cpd : ci);
    cell = ci;
    return true;
}

}  // namespace nf
