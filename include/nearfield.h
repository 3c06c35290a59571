/*
 * nearfield.h -- C ABI of the B300 near-field direct-sum library.
 *
 * The library computes the near-field force of the Abacus N-body method
 * (Garrison, Eisenstein & Pinto, arXiv:1810.02916, Section 2.1): the
 * periodic box is cut into cpd^3 cubic cells, every particle belongs to one
 * cell, and every particle takes the softened Newtonian force of every
 * particle in the (2R+1)^3 cells whose index differs from its own by at most
 * R along each axis (periodic).  The pair law is the compact spline of
 * Section 4.3.1,
 *     F(d) = [10 - 15 u + 6 u^2] d / eps^3   (r < eps, u = r / eps)
 *     F(d) = d / r^3                         (r >= eps),
 * with d = x_j - x_i and G m = 1 (the caller scales by G m).  Positions are
 * stored as offsets from the owning cell's centre (Section 2.1, last
 * paragraph), in units of the cell width w = box / cpd.
 *
 * Conventions for every entry point:
 *  - Return value: an nf_status code.  Nothing aborts the process.  On an
 *    error the box keeps its previous state unless stated otherwise, and
 *    nf_last_error() returns a one-line message.
 *  - Pointers are plain host or device pointers (CUDA unified addressing
 *    tells them apart); the caller owns them and the library copies from or
 *    into them.  Host pointers may be pageable or pinned; pinned ones make
 *    the copies asynchronous on the box's stream.
 *  - All device work is enqueued on the box's stream (nf_set_stream, default
 *    the legacy default stream).  Entry points marked (async) do not wait
 *    for the GPU when their outputs are device pointers; device faults then
 *    surface at the next call that synchronises.
 *  - Particle arrays are in the library's storage order: sorted by cell id
 *    c = (cx cpd + cy) cpd + cz (x-major, z fastest), then by particle id
 *    within the cell (see nf_bin_particles).
 */
#ifndef NEARFIELD_H
#define NEARFIELD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef struct nf_box nf_t;

enum nf_status {
    NF_OK = 0,
    NF_EINVAL = 1,   /* bad argument or input data */
    NF_ENOMEM = 2,   /* device or host allocation failed */
    NF_ECUDA = 3,    /* a CUDA call failed (message in nf_last_error) */
    NF_ETIMEOUT = 4, /* reserved: no call returns it (the kernels of this library
                        make no device-side waits; the work queue is one atomic
                        counter) */
    NF_ESTATE = 5    /* call not valid in the box's current state */
};

/* Pair law (nf_set_softening). */
enum nf_softening {
    NF_SPLINE = 0,  /* compact spline of Section 4.3.1 (default); eps = eps_s */
    NF_PLUMMER = 1  /* F(d) = d / (r^2 + eps_p^2)^(3/2), Eq. (eqn:plummer); eps = eps_p */
};

/* Accumulation of the per-sink force sums (nf_set_accumulation). */
enum nf_accumulation {
    NF_ACC_COMPENSATED = 0, /* FP32 partials over blocks of sources, folded with an
                               exact two-sum into (hi, lo), reduced in FP64 (default) */
    NF_ACC_PLAIN = 1        /* one FP32 running sum per sink (the plain FP32 kernel) */
};

/*
 * nf_create -- make an empty box.
 *   cpd  cells per dimension (K in Section 2.1), cpd >= 2R+1 so that no cell
 *        appears twice in a neighbourhood, cpd^3 < 2^31
 *   R    near-field radius in cells (Section 2.1; the paper uses 2).  This
 *        build supports R = 2 only.
 *   eps  spline softening length eps_s in box units, 2^-20 box/cpd <= eps <
 *        box/cpd (the spline must close inside the near field; the lower
 *        bound keeps the FP32 law coefficients 10/eps^3, 15/eps^4, 6/eps^5 of
 *        cell-unit separations finite and eps^2 far above the r^2 = FLT_MIN
 *        that the kernel gives a self pair)
 *   box  box side length, > 0
 * Errors: NF_EINVAL for any violated bound, NF_ENOMEM, NF_ECUDA.
 * The box owns all of its device buffers; nf_destroy frees them.
 */
int nf_create(int cpd, int R, double eps, double box, nf_t **out);

/* nf_destroy -- free the box and its device memory (NULL is a no-op). */
void nf_destroy(nf_t *nf);

/* nf_last_error -- message of the last failed call on this box ("" if none).
 * With nf == NULL, the message of the last failed nf_create. */
const char *nf_last_error(const nf_t *nf);

/* nf_set_stream -- enqueue all later work of this box on `stream`
 * (a cudaStream_t; NULL = legacy default stream). */
int nf_set_stream(nf_t *nf, void *stream);

/* nf_set_accumulation -- NF_ACC_COMPENSATED (default) or NF_ACC_PLAIN. */
int nf_set_accumulation(nf_t *nf, int mode);

/*
 * nf_set_softening -- pair law of later force and adjoint passes: NF_SPLINE
 * (default) or NF_PLUMMER (Section 4.3.1).  The box's eps is then read as
 * eps_s or eps_p.  Plummer is not compact, but the near field still covers
 * only the 125 cells (the far field would carry the rest).  Boxes of one
 * nf_forces_batched call must share the law.
 */
int nf_set_softening(nf_t *nf, int mode);

/*
 * nf_set_cutoff -- cut-off acceleration of dense cells for later nf_forces
 * calls (the paper leaves trees for dense clusters to future versions, with
 * the opening rule set by the efficiency-accuracy trade-off, Section 2.1; this
 * is one such trade-off, an approximation that changes the results).
 * n_min = 0 (default): the exact near field.  n_min >= 1024: a cell at
 * Chebyshev distance 2 from the sink's cell holding at least n_min particles
 * acts through the quadrupole expansions of its 4^3 sub-cells about their
 * centres of mass (a particle's sub-cell along an axis is
 * floor((x_rel + 1/2) 4)); the 27 near cells and sparser far cells are summed
 * pair by pair as before.  The sub-cell moments are recomputed from the
 * current positions by every nf_forces call.  nf_pair_count then counts the
 * pairs summed directly.
 * Errors: NF_EINVAL for 0 < n_min < 1024; NF_ESTATE with Plummer softening.
 * The adjoint (nf_vjp) and nf_forces_batched stay exact-only and refuse a
 * box in cut-off mode with NF_ESTATE / NF_EINVAL.
 */
int nf_set_cutoff(nf_t *nf, int64_t n_min);

/* nf_spline_eps_from_plummer -- the spline length with the same minimum
 * pairwise dynamical time as a Plummer length: eps_s = 2.16 eps_p
 * (Section 4.3.1). */
double nf_spline_eps_from_plummer(double eps_plummer);

/*
 * nf_bin_particles -- load particles from global positions (device binning).
 *   xyz  n x 3 doubles, box units, any finite values (wrapped periodically);
 *        host or device pointer, particle id = row index
 *   n    number of particles, 0 <= n < 2^31
 * Each particle gets the cell c = floor(s) per axis (wrapped), s = x cpd / box
 * in double, and the offset x_rel = (s - c) - 1/2 in cell widths, rounded once
 * from its exact value to a multiple of 2^-22 (half to even; a negative
 * offset that rounds to zero is -0).  Particles are sorted by cell id, stably
 * in id order.  Velocities are reset to zero.  NF_EINVAL for non-finite
 * positions or |x cpd / box| >= 2^52.  Section 2.1 (cells, cell-centred
 * positions).  Synchronises.
 * A load that needs larger buffers than the box holds frees the old ones
 * first: if it then fails (NF_ENOMEM, or NF_EINVAL for the input), the box
 * is left empty rather than in its previous state.
 */
int nf_bin_particles(nf_t *nf, const double *xyz, int64_t n);

/*
 * nf_set_particles -- load particles that the caller has already binned.
 *   cell_offsets  cpd^3 + 1 int64, cell_offsets[c] = first particle of cell c
 *   counts        cpd^3 int32, particles per cell
 *   pos           n x 4 floats (x, y, z, ignored), cell-relative offsets in
 *                 cell widths, sorted by cell; |x| <= 1/2 (1 + 2^-20)
 *   n             number of particles
 * Offsets are rounded to multiples of 2^-22 cell widths (half to even).
 * Validated on the device: counts >= 0, sum(counts) = n, cell_offsets is the
 * exclusive scan of counts, offsets finite and within bounds; NF_EINVAL
 * otherwise (state unchanged, unless the box had to grow: see
 * nf_bin_particles).  Particle ids are the storage indices.  Velocities are
 * reset to zero.  Synchronises.
 */
int nf_set_particles(nf_t *nf, const int64_t *cell_offsets, const int32_t *counts,
                     const float *pos, int64_t n);

/* nf_set_velocities -- n x 4 floats (vx, vy, vz, ignored), box units per
 * unit time, storage order.  (async) */
int nf_set_velocities(nf_t *nf, const float *vel);

/*
 * nf_get_particles -- read the state back (checkpoint).  Any output may be
 * NULL.  cell_offsets: cpd^3 + 1 int64; counts: cpd^3 int32; pos, vel:
 * n x 4 floats as in nf_set_particles / nf_set_velocities (the fourth word
 * of pos is 0); perm: n int64, perm[k] = id of the particle stored at k.
 * Host or device memory.  Synchronises.
 */
int nf_get_particles(nf_t *nf, int64_t *cell_offsets, int32_t *counts, float *pos,
                     float *vel, int64_t *perm);

/* nf_num_particles -- number of particles held by the box. */
int nf_num_particles(const nf_t *nf, int64_t *n);

/*
 * nf_generation -- a process-wide counter value that changes whenever the
 * box's particles change (nf_bin_particles, nf_set_particles, nf_kick_drift,
 * or a failed load that emptied the box).  A caller that keeps results of an
 * earlier pass (the autograd wrapper's backward, for one) compares it to tell
 * whether the box still holds the positions that pass saw.
 */
int nf_generation(const nf_t *nf, uint64_t *gen);

/*
 * nf_fail_allocations -- failure injection for tests of the NF_ENOMEM paths:
 * after `skip` more successful device allocations made by this library
 * (process-wide, every box), the next `count` allocations fail with NF_ENOMEM
 * before cudaMalloc is called.  nf_fail_allocations(0, 0) turns it off.
 * When a load (nf_bin_particles, nf_set_particles) fails with NF_ENOMEM
 * after its box had to grow, the box is left empty (no particles; load
 * again); nf_set_cutoff failing with NF_ENOMEM leaves the box in the exact
 * mode; nf_create and nf_forces_batched free what they had allocated.
 */
int nf_fail_allocations(int64_t skip, int64_t count);

/*
 * nf_pair_count -- number of ordered (sink, source) evaluations one force
 * pass makes: sum over cells of n_c times the particle count of its
 * (2R+1)^3 neighbourhood (self pairs included).  The count is the one the
 * box's current work plan holds (every load, drift or cut-off change
 * re-plans); reading it copies 8 bytes to the host.  Synchronises.
 */
int nf_pair_count(nf_t *nf, int64_t *pairs);

/*
 * nf_forces -- near-field accelerations (Section 2.1, Section 4.3.1).
 *   acc  n x 4 floats (ax, ay, az, 0), box units, storage order; host or
 *        device pointer, or NULL to keep the result inside the box only
 * The FP64 per-sink sums are kept in the box (nf_get_forces64) and feed
 * nf_kick_drift.  (async for device or NULL acc)
 */
int nf_forces(nf_t *nf, float *acc);

/* nf_get_forces64 -- the FP64 sums of the last nf_forces, n x 3 doubles in
 * box units, storage order.  (async for device acc) */
int nf_get_forces64(nf_t *nf, double *acc);

/*
 * nf_kick_drift -- one leapfrog kick and drift in FP64 arithmetic (Table 1,
 * rows Kick and Drift): v' = fl32(v + a dt) with a the FP64 sums of the last
 * nf_forces, then per axis s = (c + 1/2 + x_rel) + (v' dt) (cpd / box) in cell
 * units with one FP64 rounding, re-binned by the rule of nf_bin_particles
 * (new cells, offsets rounded once to the 2^-22 grid, stable sort by cell in
 * id order).  Velocities and offsets are stored as FP32.  If any particle would move more than 0.8 cell widths
 * along an axis (the drift limit of Section 4.2.1) nothing is changed and
 * NF_EINVAL is returned.  NF_ESTATE without a previous nf_forces.
 * Synchronises.
 */
int nf_kick_drift(nf_t *nf, double dt);

/*
 * nf_choose_dt -- global time step from the criteria of Section 4.2.1, using
 * the box's velocities and the accelerations of the last nf_forces:
 *   dt_acc   = eta * max( min over cells of v_rms,c / a_max,c ,  v_rms / a_max )
 *              (v_rms = sqrt(mean |v|^2), a_max = max |a|; per cell and over
 *              all particles; cells with a_max = 0 are skipped; the global
 *              value guards against abnormally cold cells)
 *   dt_drift = 0.8 cell widths / max |v|
 *   dt       = min(dt_max, dt_acc, dt_drift)
 * dt_max stands in for the TimeStepDlna cap of an expanding box.  eta is
 * TimeStepAccel (the paper uses 0.15 and 0.3).  parts (may be NULL) receives
 * {dt_acc, dt_drift, dt_max}.  With all velocities zero dt_acc is 0.
 * NF_ESTATE without a previous nf_forces.  Synchronises.
 */
int nf_choose_dt(nf_t *nf, double eta, double dt_max, double *dt, double *parts);

/*
 * nf_multipoles -- Cartesian multipole moments of every cell, the per-cell
 * step the far field starts from (Section 2.1; order p = 8 in the paper):
 *   M_c[a, b, k] = sum over the cell's particles of x^a y^b z^k,
 *   a + b + k <= order (0..8), x = offset from the cell centre in cell widths,
 *   unit masses, FP64 arithmetic (the paper computes multipoles in double).
 *   out  cpd^3 x T doubles, T = (p+1)(p+2)(p+3)/6 (165 at p = 8), cell-major;
 *        terms ordered by degree n, then a = n..0, then b = n-a..0.
 * Host or device pointer.  (async for device out)
 */
int nf_multipoles(nf_t *nf, int order, double *out);

/*
 * nf_vjp -- adjoint (vector-Jacobian product) of the accelerations.
 *   w     n x 4 floats (cotangent w_k, storage order; 4th ignored)
 *   grad  n x 4 floats out: d(sum_i w_i . a_i)/dx_k in box units
 *         = sum_{j near k} J(x_j - x_k) (w_j - w_k),
 *         J(d) = f(r) I + (f'(r)/r) d d^T, F(d) = f(r) d,
 *         with cell membership held fixed.
 * The paper has no adjoint; this differentiates its pair law (Section
 * 4.3.1).  (async for device grad)
 */
int nf_vjp(nf_t *nf, const float *w, float *grad);

/*
 * nf_forces_batched -- near-field accelerations of several independent
 * boxes in one persistent launch from one device work queue.
 *   boxes  nbox box handles (all with particles loaded), 1 <= nbox <= 4096
 *   acc    nbox output pointers as in nf_forces (entries may be NULL)
 * Work runs on the first box's stream.  The batch's combined work list is
 * rebuilt when the set of boxes or a box's particles changed since the last
 * call; otherwise the call enqueues only a queue reset and one kernel (plus
 * output copies for host outputs), allocates nothing and does not
 * synchronise.
 */
int nf_forces_batched(nf_t *const *boxes, int nbox, float *const *acc);

/*
 * nf_profile -- timing of the pair kernel.  With enable = 1, later
 * nf_forces / nf_forces_batched / nf_vjp calls bracket the pair kernel with
 * CUDA events on the box's stream; nf_profile_read returns the number of
 * timed launches and their summed duration in milliseconds (synchronises)
 * and resets both.  enable = 2 also makes the pair kernel sum clock cycles
 * per class of work item (a diagnostic: the per-item atomics perturb the
 * timing a little); nf_profile_classes returns and resets those sums.
 */
int nf_profile(nf_t *nf, int enable);
int nf_profile_read(nf_t *nf, int64_t *launches, double *ms);

/*
 * nf_profile_classes -- the per-class sums of enable = 2, NF_PROFILE_WORDS
 * uint64 words (out must hold at least that many).  Item classes cls =
 * 2 kind + piece, kind 0: tiles of 65-128 sinks (4 per lane), 1: 33-64 (2 per
 * lane), 2: 17-32 (1 per lane), 3: <= 16 sinks (sources split over the lanes),
 * 4: lane items (runs of sparse cells, one sink per lane); piece 1 for a
 * source piece of a split item.  out[3 cls] = summed warp clock cycles in the
 * class's items, out[3 cls + 1] = items, out[3 cls + 2] = pairs (0 for lane
 * items); out[30] = summed warp lifetimes (cycles), out[31] = warps,
 * out[32] = UINT64_MAX - earliest warp start, out[33] = latest warp exit
 * (both globaltimer nanoseconds).  Synchronises.
 */
#define NF_PROFILE_WORDS 34
int nf_profile_classes(nf_t *nf, uint64_t *out, int n_out);

/*
 * nf_set_shape -- launch shape of the pair kernel: warps per block (1..8) and
 * sources staged per round (128 or 256).
 */
int nf_set_shape(nf_t *nf, int warps, int stage);

/*
 * nf_set_tiling -- how each cell's sinks are cut into work items (sink tiles)
 * and how long items are split.  A cell of n particles gives floor(n / 128)
 * tiles of 128 sinks (4 per lane); the remainder r (0 < r < 128) becomes one
 * tile of r sinks if r > c4; otherwise a piece of 64 sinks is taken while
 * r >= 64 and the rest becomes one tile (2 sinks per lane) if r > c2;
 * otherwise a piece of 32 while r >= 32 and one tile (1 per lane) if r > c1;
 * otherwise a piece of 16 while r > 16 and the rest (<= 16 sinks, with the
 * sources split over the lanes).  64 <= c4 <= 128, 32 <= c2 <= 64,
 * 16 <= c1 <= 32.  Items whose neighbourhood is long against the whole pass
 * are cut into source pieces of at least split_floor sources
 * (128 <= split_floor <= 2^20).  Default 96 / 40 / 18 / 1024.  Results change
 * only by rounding.  Re-plans the box (synchronises).  NF_EINVAL otherwise.
 */
int nf_set_tiling(nf_t *nf, int c4, int c2, int c1, int split_floor);

/* nf_get_tuning -- out6 = {warps, stage, c4, c2, c1, split_floor} in use. */
int nf_get_tuning(const nf_t *nf, int32_t *out6);

/*
 * nf_tune -- the autotuner: times candidate sink tilings and split floors
 * (nf_set_tiling) at the default launch shape, then candidate launch shapes
 * (nf_set_shape) at the best tiling, on this machine's particles (a few pair
 * passes each), and keeps the fastest.  Results are cached per device,
 * accumulation, pair law, cut-off, size class and occupancy signature (the
 * share of particles in cells of each power-of-two occupancy), in memory and
 * in the text file named by the NF_TUNE_CACHE environment variable when it is
 * set, so later boxes and processes with the same signature reuse them.  The
 * box is left with one complete force pass in its FP64 sums.  report (may be
 * NULL) receives a one-line summary ("cached" for a cache hit).  Synchronises.
 */
int nf_tune(nf_t *nf, char *report, int report_len);

/*
 * nf_forces_noalloc -- nf_forces for callers that cannot allocate device
 * memory (code living inside a memory pool it does not own, plugins whose
 * host forbids new allocations after start-up, loops that must not pay for
 * an allocation's implicit synchronisation).  The paper has no counterpart;
 * it is the same pair kernel as nf_forces, driven without a box handle.
 *   cpd, eps, box  as in nf_create (R = 2); 5 <= cpd <= 64
 *   cell_start     device int32[cpd^3 + 1] on the current device: first
 *                  particle of each cell, a non-decreasing scan from 0 to n
 *   pos            device float[4 n], 16-byte aligned: cell-relative offsets
 *                  in cell widths on the 2^-22 grid (as nf_get_particles
 *                  returns them), sorted by cell
 *   n              0 <= n <= 2^21
 *   acc            device float[4 n], 16-byte aligned, out: accelerations in
 *                  box units (compensated accumulation, as nf_forces)
 *   stream         cudaStream_t for all work (NULL = legacy default stream)
 *   err, err_len   optional buffer for a one-line message
 * No cudaMalloc, cudaFree or other allocating call is made: the work list
 * and counters live in one fixed device array of 9,439,488 bytes that every GPU
 * loading the library holds until exit.  Its device address is looked up on
 * the first call on each device (with that device current), so make that
 * first call before any stream capture.  Calls share that array and it keeps
 * the last call's contents: calls whose GPU work overlaps (other streams,
 * other threads) race and must be serialised by the caller.  Every call
 * validates cell_start on the device and waits for that check on the host (a
 * device-to-host copy of one flag, then a synchronisation of `stream`) before
 * it plans and launches the force pass, which it leaves running (async).
 * pos, acc and cell_start must be device memory of the current device (or
 * managed memory).  NF_EINVAL for sizes beyond the limits above, host
 * pointers or another device's pointers, misaligned arrays or an invalid
 * cell_start; NF_ECUDA otherwise.
 */
int nf_forces_noalloc(int cpd, double eps, double box, const int32_t *cell_start, const float *pos,
                      int64_t n, float *acc, void *stream, char *err, int err_len);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* NEARFIELD_H */
