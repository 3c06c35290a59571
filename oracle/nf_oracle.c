/*
 * nf_oracle.c -- plain FP64 CPU oracle for the near-field direct sum.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the test suite, the package's smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header or
 * constant with the CUDA path.
 *
 * What it computes (Abacus near field, Section 2.1 and Section 4.3.1):
 *   every particle i in cell c_i takes the force of every particle j in the
 *   (2R+1)^3 cells whose index differs from c_i by at most R along each axis
 *   (periodic), with the compact spline softening law
 *       F(d) = [10 - 15 u + 6 u^2] d / eps^3      for r <  eps,  u = r/eps
 *       F(d) = d / r^3                            for r >= eps
 *   (Section 4.3.1, unnumbered equation), d = x_j - x_i, G m = 1.
 *   The Plummer law of Eq. (eqn:plummer), F(d) = d / (r^2 + eps_p^2)^(3/2),
 *   is available as the second softening mode.
 *
 * Everything is straight loops in double precision: sinks in parallel
 * (OpenMP), each sink's 125 neighbour cells in (dx, dy, dz) order, each
 * cell's particles in storage order, j == i included (d = 0 adds 0).
 *
 * Positions come in as cell-relative offsets in units of the cell width
 * (the same values the GPU path holds, widened exactly to double).  The
 * oracle converts every separation to box units, d = (x_j + Delta - x_i) w,
 * and returns accelerations in box units.
 *
 * Parity of every function here is pinned by the CPU tests against closed
 * forms, the C^2 spline derivation, brute force over all pairs, Newton's
 * third law, lattice symmetry and finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define SOFT_SPLINE 0
#define SOFT_PLUMMER 1

/* magnitude factor f(r) with F(d) = f(r) d  (Section 4.3.1 / Eq. eqn:plummer) */
static double law_f(double r, double eps, int soft)
{
    if (soft == SOFT_PLUMMER) {
        double s = r * r + eps * eps;
        return 1.0 / (s * sqrt(s));
    }
    if (r < eps) {
        double u = r / eps;
        return (10.0 - 15.0 * u + 6.0 * u * u) / (eps * eps * eps);
    }
    return 1.0 / (r * r * r);
}

/* f'(r)/r, for the Jacobian J(d) = f I + (f'/r) d d^T.  At r = 0 the second
 * term vanishes (it is f'(r) r dhat dhat^T), so 0 is returned there. */
static double law_fprime_over_r(double r, double eps, int soft)
{
    if (r == 0.0) return 0.0;
    if (soft == SOFT_PLUMMER) {
        double s = r * r + eps * eps;
        return -3.0 / (s * s * sqrt(s));
    }
    if (r < eps) {
        double e3 = eps * eps * eps;
        return (-15.0 / (eps * r) + 12.0 / (eps * eps)) / e3;
    }
    double r2 = r * r;
    return -3.0 / (r2 * r2 * r);
}

static inline int64_t wrap(int64_t c, int64_t cpd)
{
    c %= cpd;
    return c < 0 ? c + cpd : c;
}

double nf_oracle_law(double r, double eps, int soft) { return law_f(r, eps, soft) * r; }

/*
 * Near-field acceleration of a list of sinks.
 *   cpd, R       : cells per dimension, near-field radius in cells
 *   w, eps       : cell width and softening length, box units
 *   cell_start   : int64[cpd^3 + 1]; particles of cell c are
 *                  [cell_start[c], cell_start[c+1]) in storage order;
 *                  cell id c = (cx cpd + cy) cpd + cz
 *   xrel         : double[3 n], cell-relative positions in cell widths
 *   sink, sink_cell : the sinks' storage indices and cell ids
 *   acc          : double[3 nsink] out, box units
 *   sumabs       : double[nsink] out (may be NULL): sum_j |F(d_ij)|
 *   pairs        : int64 out (may be NULL): pair evaluations, j == i included
 */
void nf_oracle_forces(int64_t cpd, int R, double w, double eps, int soft,
                      const int64_t *cell_start, const double *xrel,
                      int64_t nsink, const int64_t *sink, const int64_t *sink_cell,
                      double *acc, double *sumabs, int64_t *pairs)
{
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t s = 0; s < nsink; s++) {
        int64_t i = sink[s];
        int64_t c = sink_cell[s];
        int64_t cz = c % cpd, cy = (c / cpd) % cpd, cx = c / (cpd * cpd);
        double xi = xrel[3 * i], yi = xrel[3 * i + 1], zi = xrel[3 * i + 2];
        double ax = 0.0, ay = 0.0, az = 0.0, sa = 0.0;
        int64_t np_ = 0;
        for (int dx = -R; dx <= R; dx++)
            for (int dy = -R; dy <= R; dy++)
                for (int dz = -R; dz <= R; dz++) {
                    int64_t n = (wrap(cx + dx, cpd) * cpd + wrap(cy + dy, cpd)) * cpd + wrap(cz + dz, cpd);
                    for (int64_t j = cell_start[n]; j < cell_start[n + 1]; j++) {
                        double ddx = ((xrel[3 * j] + dx) - xi) * w;
                        double ddy = ((xrel[3 * j + 1] + dy) - yi) * w;
                        double ddz = ((xrel[3 * j + 2] + dz) - zi) * w;
                        double r = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                        double f = law_f(r, eps, soft);
                        ax += f * ddx;
                        ay += f * ddy;
                        az += f * ddz;
                        sa += f * r;
                        np_++;
                    }
                }
        acc[3 * s] = ax;
        acc[3 * s + 1] = ay;
        acc[3 * s + 2] = az;
        if (sumabs) sumabs[s] = sa;
        total += np_;
    }
    if (pairs) *pairs = total;
}

/*
 * Cut-off acceleration of dense cells (the paper leaves trees for dense
 * clusters to future versions, Section 2.1, with the opening rule set by the
 * efficiency-accuracy trade-off; this restates the approximation the library
 * implements, in plain FP64 loops).  For a sink in cell c:
 *   - the 27 cells within one cell of c, and every cell at Chebyshev distance
 *     2 holding fewer than n_min particles, are summed directly with the
 *     spline law, exactly as nf_oracle_forces does;
 *   - a cell at distance 2 holding at least n_min particles is replaced by the
 *     quadrupole expansions of its K^3 sub-cells (K = 4; a particle's sub-cell
 *     along each axis is floor((x_rel + 1/2) K), kept in 0..K-1).  For a
 *     sub-cell with M particles, centre of mass X and traceless quadrupole
 *     Q_ab = sum_j (3 s_a s_b - |s|^2 delta_ab), s = x_j - X, the potential
 *     sum_j 1/|R + s_j| = M/r + (R.Q.R) / (2 r^5) + O(s^3) (R = X - x_i, the
 *     dipole term vanishes about X) gives the acceleration
 *         M R / r^3 - Q R / r^5 + (5/2) (R.Q.R) R / r^7.
 *     Every particle of such a cell is at least one cell width from the sink,
 *     beyond any softening length, so the Newtonian law applies.
 * Arguments as nf_oracle_forces, plus n_min; acc in box units.
 */
#define CUT_K 4
#define CUT_SUB (CUT_K * CUT_K * CUT_K)

static int cut_sub_index(const double *x)
{
    int b[3];
    for (int a = 0; a < 3; a++) {
        int q = (int)floor((x[a] + 0.5) * CUT_K);
        b[a] = q < 0 ? 0 : (q > CUT_K - 1 ? CUT_K - 1 : q);
    }
    return (b[0] * CUT_K + b[1]) * CUT_K + b[2];
}

/* count, centre of mass (cell units) and Q (box units^2) of every sub-cell of cell n; 13 doubles per sub-cell */
static void cut_moments(const int64_t *cell_start, const double *xrel, int64_t n, double w, double *mom)
{
    int64_t j0 = cell_start[n], j1 = cell_start[n + 1];
    for (int sub = 0; sub < CUT_SUB; sub++) {
        double *o = mom + 13 * sub;
        double m = 0.0, X[3] = {0.0, 0.0, 0.0};
        for (int64_t j = j0; j < j1; j++) {
            if (cut_sub_index(xrel + 3 * j) != sub) continue;
            m += 1.0;
            for (int a = 0; a < 3; a++) X[a] += xrel[3 * j + a];
        }
        o[0] = m;
        if (m == 0.0) continue;
        for (int a = 0; a < 3; a++) X[a] /= m;
        double Q[3][3] = {{0.0}};
        for (int64_t j = j0; j < j1; j++) {
            if (cut_sub_index(xrel + 3 * j) != sub) continue;
            double sv[3], s2 = 0.0;
            for (int a = 0; a < 3; a++) {
                sv[a] = (xrel[3 * j + a] - X[a]) * w;
                s2 += sv[a] * sv[a];
            }
            for (int a = 0; a < 3; a++)
                for (int bb = 0; bb < 3; bb++) Q[a][bb] += 3.0 * sv[a] * sv[bb] - (a == bb ? s2 : 0.0);
        }
        for (int a = 0; a < 3; a++) o[1 + a] = X[a];
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++) o[4 + 3 * a + bb] = Q[a][bb];
    }
}

void nf_oracle_cutoff(int64_t cpd, double w, double eps, int64_t n_min,
                      const int64_t *cell_start, const double *xrel,
                      int64_t nsink, const int64_t *sink, const int64_t *sink_cell, double *acc)
{
    const int R = 2;
    const int64_t ncell = cpd * cpd * cpd;
    /* the moments of every cell at or above n_min, computed once */
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t ndense = 0;
    for (int64_t c = 0; c < ncell; c++) slot[c] = cell_start[c + 1] - cell_start[c] >= n_min ? ndense++ : -1;
    double *mom = (double *)malloc(sizeof(double) * 13 * CUT_SUB * (size_t)(ndense > 0 ? ndense : 1));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < ncell; c++)
        if (slot[c] >= 0) cut_moments(cell_start, xrel, c, w, mom + 13 * CUT_SUB * slot[c]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nsink; s++) {
        int64_t i = sink[s];
        int64_t c = sink_cell[s];
        int64_t cz = c % cpd, cy = (c / cpd) % cpd, cx = c / (cpd * cpd);
        double xi = xrel[3 * i], yi = xrel[3 * i + 1], zi = xrel[3 * i + 2];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int dx = -R; dx <= R; dx++)
            for (int dy = -R; dy <= R; dy++)
                for (int dz = -R; dz <= R; dz++) {
                    int64_t n = (wrap(cx + dx, cpd) * cpd + wrap(cy + dy, cpd)) * cpd + wrap(cz + dz, cpd);
                    int far = abs(dx) == 2 || abs(dy) == 2 || abs(dz) == 2;
                    if (!far || slot[n] < 0) {
                        for (int64_t j = cell_start[n]; j < cell_start[n + 1]; j++) {
                            double ddx = ((xrel[3 * j] + dx) - xi) * w;
                            double ddy = ((xrel[3 * j + 1] + dy) - yi) * w;
                            double ddz = ((xrel[3 * j + 2] + dz) - zi) * w;
                            double r = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                            double f = law_f(r, eps, SOFT_SPLINE);
                            ax += f * ddx;
                            ay += f * ddy;
                            az += f * ddz;
                        }
                        continue;
                    }
                    const double *mc = mom + 13 * CUT_SUB * slot[n];
                    for (int sub = 0; sub < CUT_SUB; sub++) {
                        const double *o = mc + 13 * sub;
                        double m = o[0];
                        if (m == 0.0) continue;
                        double Rv[3] = {((o[1] + dx) - xi) * w, ((o[2] + dy) - yi) * w, ((o[3] + dz) - zi) * w};
                        double r2 = Rv[0] * Rv[0] + Rv[1] * Rv[1] + Rv[2] * Rv[2];
                        double r = sqrt(r2);
                        double QR[3], RQR = 0.0;
                        for (int a = 0; a < 3; a++) {
                            QR[a] = o[4 + 3 * a] * Rv[0] + o[5 + 3 * a] * Rv[1] + o[6 + 3 * a] * Rv[2];
                            RQR += Rv[a] * QR[a];
                        }
                        double r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
                        ax += m * Rv[0] / r3 - QR[0] / r5 + 2.5 * RQR * Rv[0] / r7;
                        ay += m * Rv[1] / r3 - QR[1] / r5 + 2.5 * RQR * Rv[1] / r7;
                        az += m * Rv[2] / r3 - QR[2] / r5 + 2.5 * RQR * Rv[2] / r7;
                    }
                }
        acc[3 * s] = ax;
        acc[3 * s + 1] = ay;
        acc[3 * s + 2] = az;
    }
    free(mom);
    free(slot);
}

/*
 * Brute force over all ordered pairs, written without cell lists: particle j
 * acts on particle i through the one periodic image (shift n L, n in
 * {-1,0,1}^3) whose cell lies at most R cells from i's cell along every axis,
 * and not at all if there is none (Section 2.1: near field iff the cells are
 * separated by at most R).  Separations are taken between global positions
 * X = (c + 1/2 + x_rel) w.
 *   cell_xyz : int64[3 n] integer cell coordinates of each particle
 */
void nf_oracle_bruteforce(int64_t cpd, int R, double w, double eps, int soft, int64_t n,
                          const int64_t *cell_xyz, const double *xrel, double *acc)
{
    double L = w * (double)cpd;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double Xi[3], a[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; k++) Xi[k] = ((double)cell_xyz[3 * i + k] + 0.5 + xrel[3 * i + k]) * w;
        for (int64_t j = 0; j < n; j++) {
            double d[3];
            int ok = 1;
            for (int k = 0; k < 3 && ok; k++) {
                int found = 0;
                for (int s = -1; s <= 1; s++) {
                    int64_t dc = cell_xyz[3 * j + k] + s * cpd - cell_xyz[3 * i + k];
                    if (dc >= -R && dc <= R) {
                        double Xj = ((double)cell_xyz[3 * j + k] + 0.5 + xrel[3 * j + k]) * w + s * L;
                        d[k] = Xj - Xi[k];
                        found = 1;
                        break;
                    }
                }
                ok = found;
            }
            if (!ok) continue;
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double f = law_f(r, eps, soft);
            for (int k = 0; k < 3; k++) a[k] += f * d[k];
        }
        for (int k = 0; k < 3; k++) acc[3 * i + k] = a[k];
    }
}

/*
 * Adjoint of the near field: for a cotangent w_k (one 3-vector per
 * particle, in storage order), the gradient of S = sum_i w_i . a_i with
 * respect to the box-unit position of each listed sink k is
 *     g_k = sum_{j in near(k)} J(d_kj) (w_j - w_k),   d_kj = x_j - x_k,
 *     J(d) = f(r) I + (f'(r)/r) d d^T,
 * with cell membership held fixed.  (From a_i = sum_j F(x_j - x_i): x_k
 * enters a_k through every d_kj with sign -1 and every a_j, j near k,
 * through d_jk with sign +1; J is even in d.)
 */
void nf_oracle_vjp(int64_t cpd, int R, double w, double eps, int soft,
                   const int64_t *cell_start, const double *xrel, const double *wv,
                   int64_t nsink, const int64_t *sink, const int64_t *sink_cell, double *grad)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nsink; s++) {
        int64_t i = sink[s];
        int64_t c = sink_cell[s];
        int64_t cz = c % cpd, cy = (c / cpd) % cpd, cx = c / (cpd * cpd);
        double xi = xrel[3 * i], yi = xrel[3 * i + 1], zi = xrel[3 * i + 2];
        double g[3] = {0.0, 0.0, 0.0};
        for (int dx = -R; dx <= R; dx++)
            for (int dy = -R; dy <= R; dy++)
                for (int dz = -R; dz <= R; dz++) {
                    int64_t n = (wrap(cx + dx, cpd) * cpd + wrap(cy + dy, cpd)) * cpd + wrap(cz + dz, cpd);
                    for (int64_t j = cell_start[n]; j < cell_start[n + 1]; j++) {
                        double d[3];
                        d[0] = ((xrel[3 * j] + dx) - xi) * w;
                        d[1] = ((xrel[3 * j + 1] + dy) - yi) * w;
                        d[2] = ((xrel[3 * j + 2] + dz) - zi) * w;
                        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        double f = law_f(r, eps, soft);
                        double h = law_fprime_over_r(r, eps, soft);
                        double dw[3];
                        for (int k = 0; k < 3; k++) dw[k] = wv[3 * j + k] - wv[3 * i + k];
                        double ddw = d[0] * dw[0] + d[1] * dw[1] + d[2] * dw[2];
                        for (int k = 0; k < 3; k++) g[k] += f * dw[k] + h * ddw * d[k];
                    }
                }
        for (int k = 0; k < 3; k++) grad[3 * s + k] = g[k];
    }
}
