/*
 * lift.h -- C ABI of the GB300 (sm_103a) solver for the sublabel-accurate
 * convex relaxation of Moellenhoff, Laude, Moeller, Lellmann, Cremers,
 * "Sublabel-Accurate Relaxation of Nonconvex Energies" (arXiv 1512.01383).
 *
 * The library minimises the relaxed energy of Sec. 4,
 *     min_u  sum_x rho^**(x, u(x)) + Phi^**(grad u(x)),
 * over the lifted variable u : Omega -> R^k (k = L-1 label intervals) by the
 * preconditioned primal-dual method of Sec. 4 on the saddle-point problem
 * (eq. discrete_saddle_point_final) with the z-splitting of
 * eq. equality_constr_data and its multiplier s.  Each iteration is two
 * fused kernels: a dual step (forward-difference gradient, projection onto
 * the l2 balls of Prop. 5, projection onto the epigraphs of rho_i^*) and a
 * primal step (divergence, primal descent, box clamp, extrapolation).
 *
 * Conventions for every entry point:
 *  - Return value: LIFT_OK (0) or one of the LIFT_ERR_* codes below;
 *    lift_strerror() names it.  A failed call leaves the handle usable
 *    unless it returned LIFT_ERR_CUDA (sticky CUDA error: destroy it).
 *  - All GPU work is issued on the handle's stream, in call order.  Calls
 *    that return host values (lift_energy, lift_gap, lift_solve, and any
 *    call with on_host = 1) synchronise that stream before returning.
 *  - "Device pointer" means memory of the current CUDA device; "host
 *    pointer" means ordinary (pageable or pinned) host memory.
 *  - The handle owns all solver state.  Input buffers are read during the
 *    call that receives them and are not retained.  Output buffers are
 *    allocated by the caller.
 *  - A handle must not be used from two host threads at once.
 */
#ifndef LIFT_H
#define LIFT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
#define LIFT_OK                 0
#define LIFT_ERR_SPEC           1  /* invalid problem description           */
#define LIFT_ERR_OOM            2  /* device allocation failed              */
#define LIFT_ERR_CUDA           3  /* a CUDA call failed                    */
#define LIFT_ERR_NAN            4  /* non-finite energy: iterate diverged   */
#define LIFT_ERR_NOT_CONVERGED  5  /* max_iters reached before gap <= tol   */
#define LIFT_ERR_ARG            6  /* invalid argument (null, size, range)  */
#define LIFT_ERR_TIMEOUT        7  /* a kernel's bounded wait for its bulk
                                      copies gave up; the iterate is invalid
                                      (reported by the next lift_energy /
                                      lift_gap / lift_solve check)          */

/* lift_cuda_error: the name of the CUDA error (as cudaGetErrorName) behind
 * the calling thread's most recent LIFT_ERR_CUDA, or "no error". */
const char *lift_cuda_error(void);

/* Largest supported number of label intervals k = L-1. */
#define LIFT_MAX_K 64

/* ---------------------------------------------------------- data terms */
/* The data term rho(x, t) of eq. general_energy, t in Gamma = [gamma_min,
 * gamma_max]:
 *  LIFT_QUAD       rho = alpha/2 (t - f(x))^2          (Sec. 5.1 ROF)
 *  LIFT_TRUNC_QUAD rho = min(alpha (t - f(x))^2, nu)   (Sec. 5.2)
 *  LIFT_PL_SAMPLED rho = piecewise-linear interpolant of n_samples costs
 *                  at positions sample_min + j (sample_max-sample_min)/
 *                  (n_samples-1)                        (Sec. 5.4 stereo)
 *  LIFT_PERIODIC_QUAD  phase unwrapping (Sec. 5.5): the squared circular
 *                  distance to the wrapped data f(x), approximated on each
 *                  Gamma_i by the parabola alpha/2 (t - c_i)^2 of the
 *                  periodic copy c_i = f + nu m (m integer, nu = the period,
 *                  e.g. 2 pi) nearest to the interval's midpoint; the
 *                  nonconvex energy E_nc evaluates rho itself, alpha/2
 *                  times the squared circular distance of t to f
 * Each interval Gamma_i = [gamma_i, gamma_{i+1}] sees only the convex
 * envelope rho_i^** of rho restricted to it (Prop. 1).  For the two
 * quadratic kinds the envelope is linear-quadratic-linear and is derived in
 * closed form per pixel on the fly; for LIFT_PL_SAMPLED it is the lower
 * convex hull of the samples inside each interval, computed once by
 * lift_create / lift_set_data (the gift-wrapping step of Sec. 5.4). */
#define LIFT_QUAD        0
#define LIFT_TRUNC_QUAD  1
#define LIFT_PL_SAMPLED  2
#define LIFT_PERIODIC_QUAD 3

typedef struct lift_spec {
    int kind;                 /* LIFT_QUAD, LIFT_TRUNC_QUAD, LIFT_PL_SAMPLED,
                                 LIFT_PERIODIC_QUAD                         */
    int H, W;                 /* image size, H*W >= 1 (one slice of a volume) */
    int L;                    /* labels, 2 <= L <= LIFT_MAX_K + 1            */
    double gamma_min;         /* equidistant labels gamma_1 < ... < gamma_L  */
    double gamma_max;         /*   on [gamma_min, gamma_max] (Sec. 3)         */
    double lambda;            /* TV weight >= 0: ball radius lambda*Delta_i  */
    double alpha, nu;         /* QUAD: alpha > 0.  TRUNC: alpha > 0, nu > 0.
                                 PERIODIC: alpha > 0, nu = period > 0      */
    const float *f;           /* QUAD/TRUNC/PERIODIC: N = D*H*W values,
                                 voxel (z*H + y)*W + x (an image: z = 0)    */
    const float *cost;        /* PL: N*n_samples, pixel-major              */
    int n_samples;            /* PL: >= 2                                    */
    double sample_min;        /* PL: sample positions; must cover Gamma      */
    double sample_max;
    int data_on_host;         /* 1: f / cost are host pointers, else device */
    int check_every;          /* lift_solve: iterations between gap checks  */
    double step_balance;      /* theta > 0: every primal step x theta, every
                                 dual step / theta (tau*sigma unchanged);
                                 <= 0 means 1, the diagonal preconditioner  */
    int adaptive_balance;     /* 1: lift_solve re-balances theta at every
                                 check (see lift_solve); 0: theta fixed     */
    int tv_anisotropic;       /* 0: isotropic TV, |nu|_2 in Phi_{i,j} (K = l2
                                 balls, Prop. 5); 1: anisotropic |nu|_1
                                 (K = l-infinity boxes |p_i|_inf <= lambda
                                 Delta, Sec. 5.3)                          */
    int D;                    /* depth: D > 1 makes the domain a D x H x W
                                 volume (the d = 3 Cartesian grid of Sec. 4:
                                 three forward differences, p_i in R^3, and
                                 tau_u = theta/7 instead of theta/5); 0 or 1
                                 is an image.  D*H*W*(L-1) < 2^31.  Batches,
                                 the unrolled solve and lift_energy_noalloc
                                 take images only (LIFT_ERR_SPEC).          */
} lift_spec;

typedef struct lift_ctx *lift_handle;

/* lift_create: validate *spec, allocate the solver state on the current
 * device, upload / convexify the data term and zero the iterate (all primal
 * and dual variables start at 0).  stream: a cudaStream_t (NULL = legacy
 * default stream) on which every later call of this handle runs.
 * Errors: LIFT_ERR_ARG (null pointer), LIFT_ERR_SPEC (see lift_spec),
 * LIFT_ERR_OOM, LIFT_ERR_CUDA. */
int lift_create(const lift_spec *spec, void *stream, lift_handle *out);

/* lift_destroy: free all device memory of the handle (synchronises its
 * stream first).  NULL is ignored. */
void lift_destroy(lift_handle h);

/* lift_set_data: replace the data of an existing handle (same kind and
 * sizes): f (H*W) for the quadratic kinds or cost (H*W*n_samples) for
 * LIFT_PL_SAMPLED, from host (on_host = 1) or device memory.  Re-runs the
 * per-pixel setup.  The iterate is not touched (call lift_reset). */
int lift_set_data(lift_handle h, const float *data, int on_host);

/* lift_reset: set every primal and dual variable to 0. */
int lift_reset(lift_handle h);

/* lift_iterate: run exactly `iters` >= 0 PDHG iterations (Sec. 4), each a
 * dual step from the extrapolated primal followed by a primal step with
 * extrapolation theta = 1.  Whole check intervals (spec->check_every
 * iterations) are replayed from a CUDA graph on a private stream of the
 * handle, ordered after the handle stream's earlier work and before its
 * later work; the rest is launched directly.  Asynchronous: returns after
 * enqueueing. */
int lift_iterate(lift_handle h, int iters);

/* lift_set_bands: the graph that lift_iterate replays for each check
 * interval splits the image (volume) into row (slice) bands of whole tiles,
 * each at least one row (slice) long, and orders each band's half-steps only
 * after those of its own and its adjacent bands that it depends on: the dual
 * step of band j after the primal steps of bands j and j+1, the primal step
 * of band j after the dual steps of bands j and j-1.  Every half-step then
 * reads exactly what it reads in the one-stream order (the iterate is
 * bitwise the same), while the issue-bound dual steps of some bands overlap
 * the memory-bound primal steps of others.  bands = 0 chooses automatically
 * (4 bands from 4096 tiles of 256 threads on, else 1), 1 turns banding off,
 * 2..8 ask for that many (fewer when the bands would be too short).  *used
 * (may be NULL) receives the number that lift_iterate will use.  The
 * cluster-resident path (lift_set_resident) takes precedence where it
 * applies. */
int lift_set_bands(lift_handle h, int bands, int *used);

/* lift_set_resident: small image problems (whole 256-thread tiles, at most 8
 * per CTA on a cluster of at most 16 CTAs, their state within 200 KB of
 * shared memory per CTA: e.g. 64 x 64 pixels with L up to 20) run each call
 * of lift_iterate as one launch of a thread-block cluster that keeps the
 * state in shared memory for all the iterations and reads neighbouring
 * CTAs' halo values through distributed shared memory; the launches and the
 * round trips to L2 between half-steps go away.  The map is the iteration of
 * Sec. 4 as for every other problem (same records, same arithmetic).  This
 * is on by default where the problem fits; enable = 0 makes lift_iterate use
 * the per-half-step kernels (graph replay) instead.  *active (may be NULL)
 * tells whether lift_iterate now takes the resident path.  Volumes never do.
 * lift_dual_step / lift_primal_step always use the per-half-step kernels. */
int lift_set_resident(lift_handle h, int enable, int *active);

/* lift_dual_step / lift_primal_step: one half-step each, the two kernels
 * that lift_iterate runs per iteration (dual first, then primal).  Exposed
 * so that callers can time or interleave them.  Asynchronous. */
int lift_dual_step(lift_handle h);
int lift_primal_step(lift_handle h);

/* lift_solve: iterate until the relative primal-dual gap (see lift_gap) is
 * <= rel_gap_tol, checking every spec->check_every iterations, or until
 * max_iters iterations.  rel_gap_tol <= 0 runs max_iters iterations with no
 * check.  *iters_done (may be NULL) receives the count.  Returns
 * LIFT_ERR_NOT_CONVERGED if the tolerance was not met, LIFT_ERR_NAN if an
 * energy became non-finite.
 * With spec->adaptive_balance, each check also measures how far the primal
 * and the dual iterate moved since the previous check, dx^2 = sum |dx|^2/tau
 * and dy^2 = sum |dy|^2/sigma in the metric of the theta = 1 steps, and moves
 * theta half-way (geometrically) toward dx/dy: the variable that travels
 * farther gets the larger steps (the primal-weight update of Applegate et
 * al.'s PDLP; the paper itself cites adaptive steps of Goldstein and Esser).
 * lift_get_balance returns the current theta. */
int lift_solve(lift_handle h, int max_iters, double rel_gap_tol, int *iters_done);

/* lift_get_balance: the current primal/dual step balance theta. */
int lift_get_balance(lift_handle h, double *theta);

/* lift_energy: evaluate, with FP64 reductions over FP32 per-pixel terms:
 *   primal_relaxed  an upper bound on the relaxed optimum: the relaxed
 *                   energy of the current u projected onto the monotone
 *                   set 1 >= u_1 >= ... >= u_k >= 0, with its data term
 *                   bounded through the decomposition into graph pieces
 *                   whose masses come from the multiplier s (Prop. 1);
 *   dual            a lower bound on the relaxed optimum: the Lagrangian of
 *                   eq. discrete_saddle_point_final minimised over u in
 *                   [0,1]^k at the current p and v, with the smallest q
 *                   allowed by the set C (eq. constraint_C);
 *   e_nonconvex     sum_x rho(x, u~(x)) + lambda sum_x |grad u~(x)|_2 of
 *                   the unlifted image u~ (lift_unlift).
 * Any output pointer may be NULL.  Synchronises the stream. */
int lift_energy(lift_handle h, double *primal_relaxed, double *dual,
                double *e_nonconvex);

/* lift_gap: (primal_relaxed - dual) / max(|primal_relaxed|, |dual|, 1). */
int lift_gap(lift_handle h, double *rel_gap);

/* lift_unlift: u~(x) = gamma_1 + sum_i clamp(u_i(x), 0, 1) Delta_i (the
 * layer-cake formula of Sec. 3) into out[N] (N = D*H*W, voxel order of f), a
 * device pointer
 * (on_host = 0, asynchronous) or a host pointer (on_host = 1). */
int lift_unlift(lift_handle h, float *out, int on_host);

/* Running average of the iterate, for bounds that the last iterate does not
 * give on polyhedral problems (the sampled costs of Sec. 5.4: there the last
 * iterate's dual bound keeps oscillating).  Every iterate is feasible (u in
 * [0,1]^k, p_i in its ball of the set K of Prop. 5, (v_i, z_i) in the scaled
 * epigraph of rho_i^*, eq. constraint_C) and these sets are convex, so the
 * average is feasible and the energies of lift_energy evaluated at it bound
 * the relaxation's optimum as well.
 *
 * lift_average(h, 1) adds the current iterate (x = {u, s}, the dual records
 * y, q, and pz on a volume) to the average, a <- a + (x - a) / n for the n-th
 * iterate added; the first call after creation or after lift_average(h, 0)
 * sets a <- x.  lift_average(h, 0) empties the average (no device work).
 * The averaged records live in the handle (allocated on the first
 * accumulation: 24 bytes per (pixel, interval), 28 on a volume, and 4 per
 * pixel for q; LIFT_ERR_OOM if that fails) and are kept apart from the iterate, which the averaging
 * never changes.  lift_reset, lift_set_data and lift_set_params empty the
 * average too (its points belong to the old start or problem).
 * Asynchronous on the handle's stream.  LIFT_ERR_ARG for a band handle or
 * accumulate other than 0 or 1. */
int lift_average(lift_handle h, int accumulate);

/* The number of iterates in the average (0 after lift_average(h, 0)); -1 for
 * a null handle. */
long long lift_average_count(lift_handle h);

/* lift_energy and lift_unlift evaluated at the averaged iterate (same
 * outputs, same synchronisation).  LIFT_ERR_ARG while the average is empty or
 * for a band handle. */
int lift_energy_average(lift_handle h, double *primal_relaxed, double *dual,
                        double *e_nonconvex);
int lift_unlift_average(lift_handle h, float *out, int on_host);

/* lift_average_restart: the iterate becomes the averaged point (x and x-bar
 * <- the average of x, the dual records and q <- their averages; the average
 * of q is kept with the others) and the average is emptied.  A restart of
 * the iteration from the average, as restarted primal-dual methods do on
 * polyhedral problems; the step balance is kept, a stored unrolled forward
 * pass is dropped.  Asynchronous.  LIFT_ERR_ARG while the average is empty or
 * for a band handle. */
int lift_average_restart(lift_handle h);

/* lift_solve_averaged: lift_solve with certificates from the averaged
 * iterate and restarts from it, for problems whose last iterate's bounds
 * oscillate (the sampled costs of Sec. 5.4).  Epochs of first_epoch,
 * 2 first_epoch, 4 first_epoch, ... iterations (the last clipped to
 * max_iters); within an epoch the iterate is added to the running average
 * (lift_average) after every `every` iterations; at the epoch's end the
 * relative gaps (as lift_gap) of the average and of the last iterate are
 * compared, and when the average's is the smaller the iteration restarts
 * from it (lift_average_restart), so the iterate is always the better of
 * the two points.  Returns LIFT_OK once that gap is <= rel_gap_tol,
 * LIFT_ERR_NOT_CONVERGED after max_iters.  *iters_done: iterations run;
 * *rel_gap: the iterate's relative gap at the last epoch end (either may be
 * NULL).  The step balance stays fixed (adaptive_balance is not applied).
 * Synchronises at every epoch end.  LIFT_ERR_ARG: null or band handle,
 * max_iters < 0, rel_gap_tol <= 0, every < 1 or first_epoch < every. */
int lift_solve_averaged(lift_handle h, int max_iters, double rel_gap_tol, int first_epoch,
                        int every, int *iters_done, double *rel_gap);

/* State image for checkpoint / resume and for tests.  Layout (bytes, in
 * this order, all float32, pixel p = (z*H + y)*W + x, N = D*H*W, interval
 * i = 0..k-1):
 *   primal  [N][k] float2 {u_i, s_i}
 *   xbar    [N][k] float2 {ubar_i, sbar_i}   (extrapolated primal)
 *   dual    [N][k] float4 {v_i, z_i, px_i, py_i}
 *   q       [N]    float
 *   pz      [N][k] float  (volumes only: the z component of p_i)
 * lift_state_bytes returns the total size.  get/set copy exactly that many
 * bytes (bytes must equal it, else LIFT_ERR_ARG). */
size_t lift_state_bytes(lift_handle h);
int lift_get_state(lift_handle h, void *dst, size_t bytes, int on_host);
int lift_set_state(lift_handle h, const void *src, size_t bytes, int on_host);

/* lift_proj_epi: the projection used inside the dual step, exposed for
 * testing: for n points, project (y0[j], h0[j]) onto epi(rho_i^*) of pixel
 * pix[j] and interval interval[j] (0-based), where rho_i^*(y) =
 * sup_{t in Gamma_i} t*y - rho(x, t) (Prop. 1, Fig. 7), writing y[j], h[j].
 * All six arrays are device pointers of length n.  A point whose pixel or
 * interval index is out of range yields NaN outputs.  Asynchronous. */
int lift_proj_epi(lift_handle h, const int *pix, const int *interval,
                  const float *y0, const float *h0, float *y, float *hout,
                  int n);

/* lift_envelope: rho_i^**(t[j]) at n points (device arrays; t[j] is clamped
 * into Gamma_i): the convexified pieces that the relaxation uses.  Out-of-
 * range indices yield NaN. */
int lift_envelope(lift_handle h, const int *pix, const int *interval,
                  const float *t, float *out, int n);

/* ------------------------------------------------------- differentiation */
/* The unrolled solve as a differentiable map (the paper has none): from the
 * zero state, `iters` iterations map (f, lambda, alpha, nu) to the unlifted
 * image u~.  The reverse pass is hand-written (adjoint.cu): it pulls the
 * adjoint back through each half-step, including the clamp, the l2-ball
 * projection and the epigraph projections (derivatives taken on the branch
 * that the forward pass took; the map is piecewise smooth).  Quadratic and
 * truncated-quadratic data terms only. */

/* lift_set_params: change lambda, alpha and nu of an existing handle (the
 * step sizes do not depend on them).  LIFT_ERR_SPEC for invalid values. */
int lift_set_params(lift_handle h, double lambda, double alpha, double nu);

/* lift_unrolled_forward: reset, then run `iters` iterations, storing the
 * state every `checkpoint_every` iterations (ceil(iters/checkpoint_every)
 * state copies of lift_state_bytes each, kept by the handle).  The final
 * state is the handle's state (lift_unlift reads it).  Asynchronous. */
int lift_unrolled_forward(lift_handle h, int iters, int checkpoint_every);

/* lift_unrolled_backward: given grad_u = dL/du~ (device, H*W) for the image
 * of the last lift_unrolled_forward, write dL/df to grad_f (device, H*W; may
 * be NULL) and {dL/dlambda, dL/dalpha, dL/dnu} to grad_scalars (host, 3
 * doubles; may be NULL).  Each segment between checkpoints is recomputed
 * forward into a buffer of checkpoint_every + 1 states, then pulled back.
 * Synchronises when grad_scalars is requested.  LIFT_ERR_ARG if no forward
 * pass is stored, or if lift_set_params, lift_set_data or lift_reset has run
 * since the last one (the stored pass would no longer be this problem's). */
int lift_unrolled_backward(lift_handle h, const float *grad_u, float *grad_f,
                           double *grad_scalars);

/* lift_unrolled_generation: a counter that changes with every
 * lift_unrolled_forward, lift_set_params, lift_set_data and lift_reset of
 * the handle.  A caller that keeps the value of a forward pass (as the
 * autograd wrapper does) can tell, before its reverse pass, whether the
 * handle still holds that forward pass. */
int lift_unrolled_generation(lift_handle h, unsigned long long *generation);

/* ------------------------------------------------------ bands of an image */
/* Spatial decomposition of one image problem over several handles (one per
 * GPU, or several on one GPU): each handle owns a band of consecutive rows.
 * The operator of Sec. 4 couples a pixel only to its forward-difference
 * neighbours (x+1, y+1 in grad, x-1, y-1 in div), so a band needs one row of
 * its neighbours per half-step and exchanges nothing else: per iteration
 *   1. every band but the first exports LIFT_HALO_PRIMAL (its first own
 *      row's x and xbar records); the band above imports it;
 *   2. every band runs lift_dual_step (its own rows only);
 *   3. every band but the last exports LIFT_HALO_DUAL (its last own row's y
 *      records); the band below imports it;
 *   4. every band runs lift_primal_step (its own rows only).
 * The own rows then evolve exactly as in one handle over the whole image
 * (the same arithmetic per record, in the same order).  lift_energy of a
 * band returns the sums over its own pixels; the three sums of the whole
 * image are the sums over the bands (an FP64 allreduce across ranks).  The
 * energies read the row below through the halo, so call it after step 1.
 * lift_unlift writes the band's own rows.  lift_iterate, lift_solve,
 * lift_gap and the unrolled solve return LIFT_ERR_ARG on a band (they would
 * skip the exchanges); the caller runs the loop above. */
#define LIFT_HALO_PRIMAL 0   /* x then xbar records of one row: 2 W k float2 */
#define LIFT_HALO_DUAL   1   /* y records of one row: W k float4             */

/* lift_create_band: a handle for the rows [row0, row1) of the image that
 * *spec describes (its H, W, data pointer and parameters are those of the
 * whole image; the band reads the data rows it needs, its own and the halo
 * rows, at create).  Images only.  Errors as lift_create; LIFT_ERR_ARG for
 * an empty or out-of-range row interval. */
int lift_create_band(const lift_spec *spec, int row0, int row1, void *stream, lift_handle *out);

/* lift_band_halo_bytes: the size of a halo of kind `which` (a row of W
 * pixels).  LIFT_ERR_ARG for a handle that is not a band. */
int lift_band_halo_bytes(lift_handle h, int which, size_t *bytes);

/* lift_band_export: copy the band's halo of kind `which` into dst (device
 * or host per on_host, lift_band_halo_bytes bytes), in stream order on the
 * handle's stream (synchronised when on_host).  LIFT_ERR_ARG when no band
 * receives it (LIFT_HALO_PRIMAL of the first band, LIFT_HALO_DUAL of the
 * last). */
int lift_band_export(lift_handle h, int which, void *dst, int on_host);

/* lift_band_import: copy a neighbour's exported halo from src into this
 * band's halo row (LIFT_HALO_PRIMAL: the row below its own rows;
 * LIFT_HALO_DUAL: the row above), in stream order on the handle's stream.
 * LIFT_ERR_ARG when the band has no such neighbour. */
int lift_band_import(lift_handle h, int which, const void *src, int on_host);

/* --------------------------------------------------------------- batches */
/* A batch solves many independent problems (each its own size, label count
 * and data; one quadratic data-term kind: LIFT_QUAD, LIFT_TRUNC_QUAD or
 * LIFT_PERIODIC_QUAD) together.  Instances too small to fill the GPU share
 * one launch per half-step over all their tiles; an instance with at least
 * big_tiles tiles of 256 threads (two full waves of the GPU by default; see
 * lift_batch_autotune) runs on the single-instance kernels instead, which
 * reach full bandwidth on it alone.  Each check_every iterations (of
 * specs[0]) are replayed as one CUDA graph.  Instances found converged by
 * lift_batch_solve stop iterating (their blocks exit at once, through a
 * device flag) while the others continue.  The iteration of each instance is
 * the same map as a single handle's (the same per-tile arithmetic). */
typedef struct lift_batch_ctx *lift_batch;

/* lift_create_batch: n >= 1 specs (each validated as by lift_create; PL and
 * mixed kinds give LIFT_ERR_SPEC).  stream: cudaStream_t for all work of the
 * batch; NULL makes the batch create (and later destroy) its own
 * non-blocking stream, because graph capture cannot use the legacy default
 * stream; work on that private stream is not ordered with the caller's
 * legacy-default-stream work, so such callers synchronise the device before
 * reading results.  All state lives in one device allocation owned by the
 * batch. */
int lift_create_batch(const lift_spec *specs, int n, void *stream, lift_batch *out);
void lift_batch_destroy(lift_batch b);
int lift_batch_size(lift_batch b);

/* lift_batch_reset: zero every iterate; mark every instance live. */
int lift_batch_reset(lift_batch b);

/* lift_batch_iterate: `iters` iterations of every live instance
 * (asynchronous; whole check intervals run as one graph launch). */
int lift_batch_iterate(lift_batch b, int iters);

/* lift_batch_solve: iterate in check intervals until every instance's
 * relative gap (as lift_gap) is <= rel_gap_tol or max_iters is reached.
 * iters_done (n ints, may be NULL): iterations each instance ran;
 * n_converged (may be NULL).  LIFT_ERR_NOT_CONVERGED if some did not. */
int lift_batch_solve(lift_batch b, int max_iters, double rel_gap_tol, int *iters_done,
                     int *n_converged);

/* lift_batch_energy: out[3*i .. 3*i+2] = {primal_relaxed, dual, e_nonconvex}
 * of instance i (as lift_energy), host array of 3n doubles.  Synchronises. */
int lift_batch_energy(lift_batch b, double *out);

/* lift_batch_unlift: unlifted image of instance i into out (H_i*W_i floats,
 * device or host per on_host). */
int lift_batch_unlift(lift_batch b, int i, float *out, int on_host);

/* lift_batch_get_state: state image of instance i (layout of lift_get_state). */
int lift_batch_get_state(lift_batch b, int i, void *dst, size_t bytes, int on_host);

/* lift_batch_autotune: time `iters` iterations, as the captured graph that
 * lift_batch_iterate replays, for each tile width of the merged primal
 * launch (128, 256, 512 threads), each big-instance threshold (none, 1, 2 or
 * 4 full waves of 256-thread tiles) and each number of streams that the big
 * instances share (1, 2, 4: several big instances run at once) on this
 * batch, and keep the fastest (*threads_chosen, may be NULL).  Resets every
 * iterate to zero. */
int lift_batch_autotune(lift_batch b, int iters, int *threads_chosen);

/* lift_batch_streams: set (set = 1..4; 0 leaves it) and read (*n, may be
 * NULL) the number of streams that the big instances share in a captured
 * interval.  LIFT_ERR_ARG for other values. */
int lift_batch_streams(lift_batch b, int set, int *n);

/* lift_batch_set_schedule: set the schedule by hand: tile width of the
 * merged primal launch (128, 256 or 512 threads, at least k of every
 * instance left in it, else LIFT_ERR_ARG and the schedule is unchanged) and
 * the big-instance threshold in 256-thread tiles (0: every instance merged;
 * 1: every instance on the single-instance kernels).  The iterates are kept.
 * The merged dual steps run each instance in its single handle's strips.
 * With 256-thread primal tiles every instance follows its single handle's
 * map bitwise; other widths change only the association order of the
 * per-pixel sums over intervals in the primal step. */
int lift_batch_set_schedule(lift_batch b, int threads, int big_tiles);

/* lift_batch_schedule: the current schedule: tile width of the merged
 * launch, big-instance threshold in 256-thread tiles (0: none), and how many
 * instances run on the single-instance kernels.  Any pointer may be NULL. */
int lift_batch_schedule(lift_batch b, int *threads, int *big_tiles, int *n_big);

/* ------------------------------------------------ allocation-free variant */
/* lift_energy_noalloc: the energies of lift_energy for a state that the
 * caller holds, computed without allocating any memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: code whose device memory all belongs to another allocator (a
 * framework's caching pool, a fixed memory budget), and code that must not
 * trigger cudaMalloc / cudaFree because those calls can synchronise the whole
 * device.  It needs no handle (lift_create allocates).
 *
 * spec   a LIFT_QUAD or LIFT_TRUNC_QUAD problem with data_on_host = 0:
 *        spec->f is read on the device during the call.
 * state  device pointer, 16-byte aligned, to a state image of this problem
 *        in the layout of lift_get_state (only the primal and dual parts are
 *        read).
 * out    device pointer to 3 doubles: {primal_relaxed, dual, e_nonconvex}.
 * stream cudaStream_t of the current device for the two kernels (a stream
 *        of another device gives LIFT_ERR_ARG); the call is asynchronous and
 *        does not synchronise.
 *
 * The per-block partial sums go to one fixed array in the library's device
 * memory (3 doubles per 256 pixels, 96 KB), which every GPU that loads the
 * library holds until the process exits.  Hence the limit: H*W must not
 * exceed LIFT_NOALLOC_MAX_PIXELS, else LIFT_ERR_ARG (as for null pointers,
 * host-resident data and device ordinals >= 64); other invalid specs give
 * LIFT_ERR_SPEC.  The first call on each device looks up the array's device
 * address (one-time set-up, done with that device current); make that first
 * call before any stream capture.  All calls share the array and each call
 * overwrites every entry it reads, so nothing has to be cleared between
 * calls; but calls whose kernels overlap on the GPU (different streams
 * without ordering between them) race on it and return wrong sums. */
#define LIFT_NOALLOC_MAX_PIXELS (1 << 20)
int lift_energy_noalloc(const lift_spec *spec, const void *state, double *out,
                        void *stream);

const char *lift_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LIFT_H */
