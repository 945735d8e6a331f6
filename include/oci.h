/*
 * oci.h -- C ABI of the GB300 (sm_103a) one-cell-inversion library for
 * transient slab-geometry S_N transport, discretised with simple corner balance
 * (SCB) in space and multiple balance (MB) in time (arXiv 2305.13555).
 *
 * Problem statement (Sec. "Derivation of MB-SCB", Eq. 1): mono-energetic,
 * isotropic scattering and source, slab [0, X] of n_cells cells of widths dx_j
 * with total / scattering cross sections Sigma_j, Sigma_{s,j}; particle speed
 * v; time step dt; initial angular flux psi_{m,0}; prescribed incident angular
 * flux at x = 0 (mu_m > 0) and x = X (mu_m < 0), or vacuum, or reflection.
 * Angles: n_ord-point Gauss-Legendre quadrature (weights sum to 2), ordinates
 * ascending in mu.  Per cell and ordinate the unknowns are the corner fluxes
 * (k,L) (k,R) (k+1/2,L) (k+1/2,R): time-average (k) and end-of-step (k+1/2)
 * values on the left (L) and right (R) half cells (the vector psi_n of the
 * OCI section).
 *
 * Conventions for every entry point
 *   - Host pointers are read (or written) during the call only; the library
 *     copies what it keeps.  Device pointers are noted as such.
 *   - Array layouts are C row-major, doubles unless stated:
 *       per-cell quantities [n_cells]; sources q[n_cells][4] in component order
 *       (Q_{k,L}, Q_{k,R}, Q_{k+1/2,L}, Q_{k+1/2,R});
 *       scalar-flux moments phi[n_cells][4] in the same order;
 *       time-edge angular flux psi[n_cells][n_ord][2] (L, R);
 *       boundary data bc[n_ord/2][2] = (time moment k, k+1/2) for pair p:
 *       left face -> ordinate n_ord/2 + p (mu > 0), right face -> ordinate
 *       n_ord/2 - 1 - p (mu < 0).
 *   - Every call returns an OCI_* status; none aborts or prints.  On an error
 *     the handle stays usable and its committed state is unchanged, except
 *     after OCI_ECUDA, after which only oci_destroy is meaningful.
 *   - A handle is bound to the CUDA device current at oci_create and to the
 *     stream given there (oci_set_stream changes it).  Calls on one handle
 *     must not overlap; different handles are independent.
 */
#ifndef OCI_GB300_OCI_H
#define OCI_GB300_OCI_H

#include <stddef.h>
#include <stdint.h>

#include "oci_nn.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
    OCI_OK = 0,
    OCI_EINVAL = 1,    /* invalid argument (sizes, signs, NULL where required) */
    OCI_ENOMEM = 2,    /* device or host allocation failed */
    OCI_ECUDA = 3,     /* a CUDA call failed; see oci_last_cuda_error */
    OCI_ENOTCONV = 4,  /* max_iter reached before the tolerance */
    OCI_ENAN = 5,      /* non-finite scalar flux detected in the residual */
    OCI_ETIMEOUT = 6,  /* device-side iteration guard tripped (launch cap) */
    OCI_ESTATE = 7,    /* call not valid in the handle's current state */
    OCI_ESKIPPED = 8   /* oci_run_steps: not run, an earlier step of the call did not commit */
};

enum { OCI_BC_VACUUM = 0, OCI_BC_REFLECT = 1, OCI_BC_INCIDENT = 2 };

/* Arithmetic / storage precision of the angular flux and per-ordinate blocks.
 * OCI_FP64: everything in double.  OCI_FP32: angular flux, per-ordinate 4x4
 * blocks and the scattering-moment sums in float (the sums compensated,
 * TwoSum), the 4x4 capacitance solve and the residual norm in double.
 * OCI_FP32_BF16HALO: OCI_FP32 with oci_set_halo(OCI_HALO_BF16) applied at
 * creation (OCI_EINVAL where that call would refuse). */
enum { OCI_FP64 = 0, OCI_FP32 = 1, OCI_FP32_BF16HALO = 2 };

/* ------------------------------------------------------------- problem */
typedef struct oci_problem {
    int32_t n_cells;           /* J >= 1 */
    int32_t n_ord;             /* N: even, 2 <= N <= 256 */
    const double *dx;          /* host [J], > 0 */
    const double *sigma_t;     /* host [J], >= 0 */
    const double *sigma_s;     /* host [J], 0 <= sigma_s <= sigma_t */
    const double *q;           /* host [J][4] isotropic source moments, or NULL = 0 */
    double v;                  /* speed > 0 (may be +inf: steady state) */
    double dt;                 /* time step > 0 */
    int32_t bc_left, bc_right; /* OCI_BC_* */
    const double *psi_bc_left;  /* host [N/2][2] for OCI_BC_INCIDENT, else ignored */
    const double *psi_bc_right; /* host [N/2][2] for OCI_BC_INCIDENT, else ignored */
    const double *psi0;        /* host [J][N][2] initial angular flux, or NULL = 0 */
    int32_t precision;         /* OCI_FP64 or OCI_FP32 */
    int32_t max_iter;          /* iterations allowed per time step, >= 1 */
    double tol;                /* convergence: ||phi^{l+1}-phi^l||_2/||phi^{l+1}||_2 < tol */
    void *cuda_stream;         /* cudaStream_t to launch on, or NULL (legacy default stream) */
} oci_problem;

/* Per-step statistics. */
typedef struct oci_stats {
    int32_t iters;       /* iterations taken (the one meeting tol included) */
    int32_t status;      /* OCI_OK, OCI_ENOTCONV, OCI_ENAN, OCI_ETIMEOUT (OCI_ESKIPPED: oci_run_steps) */
    double residual;     /* last relative change of phi */
    double seconds;      /* device time of the step (CUDA events on the handle's stream) */
    int32_t committed;   /* 1 if the step advanced the state */
    int32_t nn_accepts;  /* learned guess / corrections kept (0 without a network) */
    int32_t nn_rejects;  /* learned corrections reverted by the safeguard */
    int32_t refined;     /* 1 if the FP32 path finished the step with its refinement (see oci_step) */
    int32_t launches;    /* kernels of this library launched for the step (library GEMMs not counted;
                          * iteration launches that found the step already ended included) */
} oci_stats;

typedef struct oci_handle oci_handle;

/* Create a solver for problem *p (Sec. "Derivation of MB-SCB": the inputs of
 * Eq. 1 plus dx_j, dt and N).  Copies every input, computes the Gauss-Legendre
 * set, the per-material per-ordinate block inverses (the A^+/A^- matrices of
 * the SI section) and the capacitance matrices of the OCI cell system, and
 * allocates all device memory (owned by the handle).  Errors: OCI_EINVAL for
 * out-of-range sizes or values (N odd or > 256, dx <= 0, sigma_s > sigma_t,
 * v or dt <= 0, NULL arrays), OCI_ENOMEM, OCI_ECUDA.  *out is set only on OK. */
int oci_create(const oci_problem *p, oci_handle **out);

/* Release the handle and all its device memory.  NULL is accepted. */
void oci_destroy(oci_handle *h);

/* Replace the source moments used from the next step on (Q_k and Q_{k+1/2}
 * of Eqs. scb-mb-a..d): host [J][4].  The copy is enqueued on the handle's
 * stream: from pageable memory q may be reused when the call returns; from
 * page-locked (pinned) memory the copy is asynchronous, so keep q unchanged
 * until the next call that synchronises (oci_step, si_step, oci_fluxes,
 * oci_step_wait, oci_sync).  While a step started by oci_step_async runs, the
 * copy goes to the handle's copy stream and overlaps that step; the next step
 * applies it.  OCI_EINVAL on NULL. */
int oci_set_source(oci_handle *h, const double *q);

/* Iteration controls: tolerance (>= 0; 0 iterates to max_iter), iteration cap
 * (>= 1), and whether a step that hits the cap still commits its last iterate
 * (1) or leaves the state at the previous step (0, default). */
int oci_set_iteration(oci_handle *h, double tol, int32_t max_iter, int32_t commit_unconverged);

/* Change the stream subsequent calls launch on (cudaStream_t, NULL = legacy). */
int oci_set_stream(oci_handle *h, void *cuda_stream);

/* How oci_step solves each cell's 4N x 4N system (A - S) Psi = c (Sec.
 * "One-Cell Inversion (OCI)").  OCI_SOLVER_WOODBURY (default): the complex
 * 2x2 block inverses plus the rank-4 capacitance correction, in one fused
 * kernel per iteration.  OCI_SOLVER_DENSE: the dense inverse (A - S)^{-1}
 * (the system the paper's CPU code factorises with LAPACK _gesv) is formed
 * once per material on the host in FP64 (Gauss-Jordan, partial pivoting) and
 * every iteration is a right-hand-side kernel, one cuBLAS GEMM per material
 * (DGEMM in OCI_FP64, SGEMM in OCI_FP32) and an output kernel; the iteration
 * loop runs on the host (one status read per iteration).  Both give the same
 * iterates up to rounding.  The dense variant holds n_mat (4N)^2 + 2 J 4N
 * values (OCI_EINVAL above 4 GiB / 16 GiB), does no FP32 stall refinement and
 * ignores a learned corrector (the learned guess still applies).  OCI_EINVAL
 * for an unknown solver or a singular (A - S), OCI_ENOMEM, OCI_ECUDA. */
enum { OCI_SOLVER_WOODBURY = 0, OCI_SOLVER_DENSE = 1 };
int oci_set_solver(oci_handle *h, int32_t solver);

/* How si_step sweeps each ordinate (Sec. "Source Iteration (SI)").
 * OCI_SWEEP_MARCH (default): the paper's sweep, cell by cell in the direction
 * of travel, parallel over ordinates only (a J-long dependent chain).
 * OCI_SWEEP_SCAN: the same recurrence -- the outgoing corner pair of a cell is
 * an affine function of the pair entering it -- evaluated as a parallel prefix
 * over cells (segment compositions, a pass over the segment maps, a pass that
 * applies them), so the sweep's depth is O(log J) and all SMs take part.  Not
 * the paper's method; same fixed point and iterates up to rounding (the
 * association order differs).  Reflecting boundaries keep the march's order
 * (mu < 0 first).  Allocates 2 N/2 ceil(J/2048) x 8 values on first use.
 * OCI_EINVAL for an unknown mode, OCI_ENOMEM, OCI_ECUDA. */
enum { OCI_SWEEP_MARCH = 0, OCI_SWEEP_SCAN = 1 };
int oci_set_sweep(oci_handle *h, int32_t sweep);

/* Time discretisation of oci_step.  OCI_TIME_MB (default): multiple balance,
 * two time moments per corner (the paper's scheme).  OCI_TIME_BE: backward
 * Euler (the paper's disabled section "Backward Euler transient
 * implementation"): one time level per step, total cross section
 * Sigma + 1/(v dt), the previous step's angular flux as a source
 * psi^{n-1}/(v dt); the SCB cell is the same, so the cell system is 2N x 2N and
 * its Woodbury capacitance a scalar.  The source at the new time is Q_{k+1/2}
 * and prescribed incident data its k+1/2 value; oci_fluxes returns the moments
 * (L, R) twice; the state (psi at the end of the last step) carries over when
 * switching.  OCI iteration only (si_step returns OCI_EINVAL under BE); no
 * learned guess, dense solver or FP32 refinement on this path.  OCI_EINVAL for
 * an unknown scheme or a singular capacitance, OCI_ENOMEM, OCI_ECUDA. */
enum { OCI_TIME_MB = 0, OCI_TIME_BE = 1 };
int oci_set_time_scheme(oci_handle *h, int32_t scheme);

/* Storage of the incident-flux halo in the OCI iteration of an OCI_FP32
 * handle (the face buffers that the iteration reads from the neighbours'
 * previous iterate, step a3; the paper stores everything in double).
 * OCI_HALO_FP32 (default): float pairs, 24 bytes per cell-ordinate and
 * iteration.  OCI_HALO_BF16: each OCI step starts with a BF16 phase whose
 * iterations read and write the halo as bfloat16 pairs (16 bytes per
 * cell-ordinate); BF16 rounding (2^-8 relative) stops the relative change of
 * phi near 1e-3, so the phase ends once the change is below 2e-3, after two
 * iterations without a 10% fall, or two iterations before max_iter; one
 * iteration turns the halo back into floats and the FP32 iteration finishes to
 * the tolerance, so the answer keeps the OCI_FP32 accuracy and the last
 * iteration of every step reads float faces.  Applies to oci_step with the
 * Woodbury solver, multiple balance, no corrector and max_iter >= 4 (other
 * steps run the FP32 halo).  OCI_EINVAL for an OCI_FP64 handle, N/2 not a
 * multiple of 4, S_N other than S_32, S_64 or S_128, or no persistent
 * cooperative loop on the device; OCI_ENOMEM; OCI_ECUDA. */
enum { OCI_HALO_FP32 = 0, OCI_HALO_BF16 = 1 };
int oci_set_halo(oci_handle *h, int32_t halo);

/* Initial iterate of the next time step, formed when a multiple-balance OCI
 * step commits (the paper does not state one; a step's iteration starts from
 * some Psi^(0) and converges to the same discrete solution from any).
 * OCI_GUESS_PREVIOUS (default): both time moments of every corner take the
 * committed end-of-step flux psi_{k+1/2}.  OCI_GUESS_EXTRAPOLATE: the linear
 * extrapolation in time through the last two end-of-step fluxes, with
 * d = psi_{k+1/2} - psi_{k-1/2} (the flux the step started from): step-average
 * moment psi_{k+1/2} + d/2, end moment psi_{k+1/2} + d (not the paper's;
 * exact for a flux linear in time; only iteration counts change).  After an
 * OCI step the iterate's scalar-flux moments, which only enter the first
 * iteration's relative change, stay the end-of-step moments, so that change is
 * measured from the previous step's flux; after an SI step, whose iteration
 * starts from them, they are extrapolated the same way (step average
 * phi_{k+1/2} + (phi_{k+1/2} - phi_{k-1/2})/2, end phi_{k+1/2} + (phi_{k+1/2} -
 * phi_{k-1/2})).  A learned guess lifts the iterate, taking its scalar flux as
 * the same extrapolation of the last two committed steps' moments.  Applies
 * to the commits of multiple-balance steps after the call; backward-Euler
 * steps, and a step after oci_set_state or an uncommitted step, start from the
 * end-of-step flux.
 * OCI_EINVAL for an unknown mode, OCI_ESTATE while a step is pending or a
 * decomposed step is open. */
enum { OCI_GUESS_PREVIOUS = 0, OCI_GUESS_EXTRAPOLATE = 1 };
int oci_set_guess(oci_handle *h, int32_t guess);

/* Diagnostics of the bounded waits (the paper has no counterpart).  The
 * persistent FP32 iteration meets the other blocks at a grid barrier once per
 * iteration; every wait there gives up after poll_limit polls (0: the default,
 * about a second) and the step then ends with OCI_ETIMEOUT, the state left at
 * the previous step, the device usable.  barrier_shortfall > 0 makes the
 * barrier wait for that many arrivals more than the grid has -- a wait that
 * nothing satisfies -- so tests can drive the timeout path without a fault;
 * 0 restores normal operation.  Applies from the next step; OCI_EINVAL for a
 * NULL handle or a negative shortfall. */
int oci_set_wait_limits(oci_handle *h, uint32_t poll_limit, int32_t barrier_shortfall);

/* Advance one time step with one-cell inversion (Sec. "One-Cell Inversion"):
 * each iteration every cell solves (A - S) Psi = c for its 4N unknowns with
 * the neighbours' incident fluxes from iterate l, via the block-diagonal plus
 * rank-4 (Woodbury) form; iterate until the relative change of phi < tol.
 * The initial iterate has both time moments equal to psi_{k-1/2}.  Returns
 * OCI_OK, OCI_ENOTCONV (state kept unless commit_unconverged), OCI_ENAN,
 * OCI_ETIMEOUT or OCI_ECUDA.  Synchronises the handle's stream once (more
 * often with a learned corrector or a refinement).
 * FP32 mode: when the relative change stops falling (no 10% improvement in 8
 * iterations while below 1e-5 -- float rounding noise near the tolerance), the
 * step is finished by mixed-precision refinement: the current halo h0 is kept,
 * r0 = G(h0) - h0 and phi(h0) are evaluated once in FP64 (counted as one
 * iteration), and the correction d = B d + r0 (B: the OCI map without sources,
 * homogeneous boundary data) is iterated in FP32 to the same tolerance on the
 * relative change of phi(h0) + phi(d); h0 + d is committed.  Available for
 * N/2 a power of two (the staged kernels); otherwise a stall ends the step with
 * OCI_ENOTCONV at max_iter as usual. */
int oci_step(oci_handle *h, oci_stats *st);

/* Same contract with source iteration (Sec. "Source Iteration (SI)"): the
 * scattering source lags one iteration and every ordinate is swept cell by cell
 * in its direction of travel, mu < 0 first (so a reflecting left face uses the
 * current sweep; a reflecting right face uses the previous iterate). */
int si_step(oci_handle *h, oci_stats *st);

/* Pipelined stepping (no counterpart in the paper; it overlaps the host
 * traffic of consecutive steps with their computation).  oci_step_async
 * enqueues one OCI step -- the oci_step computation -- on the handle's stream and
 * returns without waiting; oci_step_wait waits for it, finishes what needs the
 * host (an FP32 refinement of a stalled step), fills *st (may be NULL) and
 * returns the status oci_step would have returned.  Between the two, the host
 * may call oci_set_source (the next step's source, staged on a copy stream)
 * and oci_fluxes_async; every other call on the handle returns OCI_ESTATE until
 * oci_step_wait.  oci_step_async returns OCI_ESTATE while a step is pending or
 * for a handle whose step takes decisions on the host mid-step (a learned
 * guess attached, the dense solver, backward Euler); use oci_step there. */
int oci_step_async(oci_handle *h);
int oci_step_wait(oci_handle *h, oci_stats *st);

/* Several time steps in one call (no counterpart in the paper; it keeps the
 * device busy across steps): steps k = 0 .. n-1, each with source moments
 * q + k J 4 (host [n][J][4]; NULL: keep the current source), its published
 * moments copied to phi + k J 4 (host [n][J][4], may be NULL) and its
 * statistics to stats[k] (may be NULL).  The results are those of n rounds of
 * oci_set_source / oci_step / oci_fluxes.  For an OCI_FP32 handle whose step
 * runs start to end on the device (the persistent loop; no learned guess,
 * Woodbury solver, multiple balance, FP32 halo or a BF16 phase not in use),
 * the next step is enqueued before the host waits for the current one, the
 * sources go up and the moments come down on two copy streams, and the queued
 * step's prologue holds it (it does nothing) unless the one before it
 * committed; a step that stalls in FP32 is refined on the host and the step
 * behind it is enqueued again.  Other handles run the steps one at a time.
 * Pass page-locked (pinned) q and phi for the copies to overlap.  The call
 * returns when every copy is done.  The first step that does not commit ends
 * the call: its status is returned, later steps are not run (stats status
 * OCI_ESKIPPED; their phi entries are unspecified) and the handle keeps that
 * step's source.  *done (may be NULL)
 * = steps committed.  OCI_OK when all n committed; OCI_EINVAL for n < 0,
 * OCI_ESTATE while a step is pending or a decomposed step is open. */
int oci_run_steps(oci_handle *h, int32_t n, const double *q, double *phi, oci_stats *stats, int32_t *done);

/* Copy the moments published by the last step enqueued before this call (as
 * oci_fluxes, [J][4]) to host memory without waiting: a device snapshot on the
 * handle's stream (so the next step may overwrite the published moments) and
 * the copy to phi on the copy stream, overlapping whatever runs next; phi
 * (page-locked for an asynchronous copy) is complete when the next
 * oci_step_wait or oci_sync returns.  Two snapshots alternate, so at most two
 * such copies are in flight.  OCI_EINVAL on NULL, OCI_ENOMEM, OCI_ECUDA. */
int oci_fluxes_async(oci_handle *h, double *phi);

/* Wait for everything the handle enqueued (its stream and its copy stream). */
int oci_sync(oci_handle *h);

/* Scalar-flux moments phi = sum_n w_n psi_n of the last committed step
 * (Eq. following the SI sweeps): host [J][4]. */
int oci_fluxes(const oci_handle *h, double *phi);

/* Same into device memory: dptr is a device pointer to J*4 doubles.  The copy
 * is enqueued on the handle's stream (no synchronisation). */
int oci_fluxes_device(const oci_handle *h, void *dptr);

/* Checkpoint: the committed time-edge angular flux psi_{k+1/2} -> host
 * [J][N][2]; in OCI_FP32 mode the stored floats are widened. */
int oci_get_state(const oci_handle *h, double *psi_edge);

/* Resume or restart: replace the time-edge angular flux (host [J][N][2]); the
 * next step starts from it.  One host-to-device copy (direct DMA from
 * page-locked memory) and a conversion kernel on the handle's stream; returns
 * with the state in place.  With a network attached, its two previous-step
 * flux inputs restart from the new state's moments. */
int oci_set_state(oci_handle *h, const double *psi_edge);

/* Time the one-cell-inversion iteration alone: run n_iter iterations from the
 * current step's initial iterate (no graph, no convergence exit), after two
 * untimed warm-up iterations, bracketed by CUDA events on the handle's stream,
 * and return the mean device time per iteration in *seconds_per_launch.  The
 * staged FP32 path runs them as one cooperative launch of its persistent loop
 * (as inside a step); other paths as one stream launch per iteration.  With
 * OCI_SOLVER_DENSE an iteration is right-hand sides, GEMMs and outputs; under
 * OCI_TIME_BE it is the backward-Euler iteration kernel.  The
 * committed state (psi_{k-1/2}, published phi) is untouched and the next step
 * restarts from it.  Used by the benchmark's roofline figure. */
int oci_profile_iterations(oci_handle *h, int32_t n_iter, double *seconds_per_launch);

/* ------------------------------------------------- domain decomposition
 * OCI is block Jacobi over cells: within an iteration every cell needs only
 * its neighbours' incident fluxes from the previous iterate, so a slab can be
 * split into cell ranges that iterate independently and exchange only the
 * angular flux crossing each cut, once per iteration, plus two sums for the
 * convergence test (Sec. "GPU Implementations": splitting the problem over
 * several accelerators within an iteration).  A sub-domain is an ordinary
 * handle created for its own cells with OCI_BC_INCIDENT (zero data) on every
 * side that is a cut; the physical faces keep their own conditions.  One time
 * step of a decomposed slab, on every sub-domain:
 *   oci_dd_begin(h);
 *   do {
 *     oci_dd_export(h, out_left, out_right);   (exchange: a sub-domain's
 *     oci_dd_import(h, in_left, in_right);      out_right is its right
 *     oci_dd_iterate(h, sums);                  neighbour's in_left, and
 *     total = sum of sums over sub-domains;     out_left its left
 *     oci_dd_decide(h, total, &done, &stats);   neighbour's in_right)
 *   } while (!done);
 * With the same inputs every cell's arithmetic is that of the undivided
 * slab's iteration (FP64 results agree bit for bit); only the order of the
 * two global sums can differ.  Decomposed steps use the Woodbury solver and
 * the multiple-balance scheme (OCI_EINVAL otherwise), ignore an attached
 * network and the FP32 stall refinement (a step ends at tol or max_iter), and
 * run one launch per iteration.  While a decomposed step is open, every other
 * call on the handle except these returns OCI_ESTATE. */

/* Open a decomposed time step (initial iterate as in oci_step). */
int oci_dd_begin(oci_handle *h);

/* The current iterate's outgoing angular flux at the two faces: out_left gets
 * the mu < 0 flux leaving through the left face, out_right the mu > 0 flux
 * leaving through the right face; DEVICE pointers to [N/2][2] values (time
 * moments k, k+1/2) of the handle's storage type (double in OCI_FP64, float in
 * OCI_FP32), pair p = ordinate pair (mu_p, -mu_p) ascending in mu_p; either
 * may be NULL.  Enqueued on the handle's stream, no synchronisation. */
int oci_dd_export(oci_handle *h, void *out_left, void *out_right);

/* The incident angular flux at the two faces for the next iteration: in_left
 * the mu > 0 flux entering through the left face, in_right the mu < 0 flux
 * entering through the right face; same layout and type as oci_dd_export;
 * NULL keeps a face's own boundary condition.  Enqueued, no synchronisation. */
int oci_dd_import(oci_handle *h, const void *in_left, const void *in_right);

/* One OCI iteration of the sub-domain's cells; sums (HOST double[2]) receives
 * sum (phi^{l+1} - phi^l)^2 and sum (phi^{l+1})^2 over its cells and the four
 * moments.  Synchronises the handle's stream. */
int oci_dd_iterate(oci_handle *h, double *sums);

/* Take the step's decision from the sums totalled over all sub-domains (HOST
 * double[2]): relative change sqrt(sums[0] / sums[1]) < tol ends the step
 * (committed), max_iter iterations end it (committed only with
 * commit_unconverged), a non-finite sum ends it with OCI_ENAN.  *done = 0:
 * iterate again (returns OCI_OK); *done = 1: the step is closed and the
 * return value and *stats (may be NULL) are those oci_step would give. */
int oci_dd_decide(oci_handle *h, const double *sums, int32_t *done, oci_stats *stats);

/* ------------------------------------------------- learned guess (oci_nn.h) */
enum { OCI_NN_OFF = 0, OCI_NN_GUESS = 1, OCI_NN_GUESS_CORRECT = 2, OCI_NN_GUESS_ADAPTIVE = 3 };

/* Attach a trained network (parameters: host FP32 array of
 * oci_nn_param_count() elements, layout in oci_nn.h) to the handle, or detach
 * it (mode OCI_NN_OFF, params may be NULL).  With OCI_NN_GUESS each oci_step
 * first predicts the step's scalar-flux moments phat from the last two
 * committed steps and moves the initial iterate toward them: every incident
 * angular flux gets the isotropic correction (phat - phi)/2 of the upstream
 * corner that feeds it.  With OCI_NN_GUESS_CORRECT the iteration also pauses
 * every k_corr iterations, applies the same correction to the current
 * iterate, iterates min(k_corr, 8) more times and, if the relative change of
 * phi is then larger than before the correction, restores the saved iterate
 * (plain OCI) and makes no further corrections in that step.
 * OCI_NN_GUESS_ADAPTIVE uses the guess only where it pays: after two plain
 * steps (a run often starts with a transient), four steps run plain, guessed,
 * guessed, plain (an order that cancels a linear trend in the iteration
 * counts), and the guess is kept for the following steps only if the two
 * guessed steps took at least 3 % fewer iterations than the two plain ones;
 * the four-step test is repeated every k_corr steps.  The tolerance is unchanged, so the network changes iteration counts
 * only.  The paper has no counterpart; OCI_EINVAL for a bad mode, k_corr < 1
 * or NULL params. */
int oci_nn_attach(oci_handle *h, const float *params, int32_t mode, int32_t k_corr);

/* The handle's static network inputs, as device arrays: stat [J][4] float
 * (log10(sigma_t)/2, c, log10(sigma_t dx), log10(sigma_t v dt)) and qfeat [J]
 * float (v dt (Q_kL + Q_kR)/2), written to caller-owned device memory. */
int oci_nn_static_features(const oci_handle *h, void *stat, void *qfeat);

/* Problem sizes and quadrature of the handle: mu[N], w[N] host (may be NULL). */
int oci_query(const oci_handle *h, int32_t *n_cells, int32_t *n_ord, double *mu, double *w);

/* Message for a status code (static storage). */
const char *oci_strerror(int code);

/* Text of the last CUDA error seen by this handle ("" if none). */
const char *oci_last_cuda_error(const oci_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* OCI_GB300_OCI_H */
