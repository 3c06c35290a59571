// nf_bin.cuh -- the binning rule shared by initial binning and re-binning.
//
// Given a coordinate s in cell units (s = x cpd / box), the particle's cell
// along that axis is c = floor(s) wrapped into [0, cpd), and its offset from
// the cell centre is x_rel = (s - c) - 1/2, rounded to a multiple of 2^-22
// cell widths (half to even).  Both subtractions are exact in double.
#pragma once

#include <cmath>

namespace nf {

constexpr double kTwo22 = 4194304.0;
constexpr double kTwoM22 = 2.384185791015625e-07;

__device__ __forceinline__ bool bin_cell_units(double s, int cpd, int &cell, float &xq)
{
    if (!(fabs(s) < 4503599627370496.0)) return false;   // non-finite or beyond 2^52
    const double c = floor(s);
    const double rel = __dsub_rn(__dsub_rn(s, c), 0.5);
    const double q = rint(__dmul_rn(rel, kTwo22));
    xq = static_cast<float>(__dmul_rn(q, kTwoM22));
    int ci;
    if (c >= -static_cast<double>(cpd) && c < 2.0 * static_cast<double>(cpd)) {
        // within one box of the valid range (always after a drift): the wrap is one integer step,
        // with no FP64 division (slow on this part's FP64 pipe); the same value as below
        ci = static_cast<int>(c);
        ci = ci < 0 ? ci + cpd : (ci >= cpd ? ci - cpd : ci);
    } else {
        const double d = static_cast<double>(cpd);
        const double cw = __dsub_rn(c, __dmul_rn(d, floor(__ddiv_rn(c, d))));
        ci = static_cast<int>(cw);
        ci = ci < 0 ? ci + cpd : (ci >= cpd ? ci - cpd : ci);
    }
    cell = ci;
    return true;
}

}  // namespace nf
