// Internal parameter block of the solver kernels (passed by value) and the
// host-side launchers.  Not part of the public ABI (include/lift.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

// Largest k handled by the per-pixel work arrays (matches LIFT_MAX_K).
#define LIFT_MAXK_DEV 64

namespace lift {

struct LiftParams {
    int H, W, k, N;          // image size, intervals, pixels (voxels: D*H*W)
    int D, HW;               // depth (1: an image) and slice size H*W
    unsigned long long hmul; // slice = (row * hmul) >> hshift for row = pix / W,
    int hshift;              // exact for row < 2^31 (volumes only)
    int kind;                // 0 quadratic, 1 truncated quadratic, 2 PL
    int aniso;               // 1: anisotropic TV (box projection of p_i)
    int ppb;                 // pixels per 256-thread tile in the step kernels
    float inv_k;             // 1/k, for the exact thread -> (pixel, interval) split
    unsigned long long wmul; // row = (pix * wmul) >> wshift, exact for pix < 2^31
    int wshift;
    float delta;             // Delta = gamma_{i+1} - gamma_i (equidistant labels)
    float inv_delta;         // 1/Delta
    float gmin;              // gamma_1
    float lam, alpha, nu;    // TV weight, data-term parameters
    float inv_alpha;         // 1/alpha (quadratic kinds)
    float wtrunc;            // sqrt(nu/alpha): half-width of the parabola
    float tau_u, sigma_q, sigma_p;
    const float4 *icst;      // per interval {gamma_i, tau_s_i, sigma_vz_i, lambda*Delta}
    const float4 *steps;     // {tau_u, sigma_q, sigma_p, 0} in device memory: the step
                             // kernels read these (not the copies above), so a new
                             // primal/dual balance needs no new iteration graph
    const float *f;          // [N] image (quadratic kinds)
    const float *rhat;       // [N][nb] convexified PL values at the breakpoints
    const float *cost;       // [N][ns] raw samples (PL)
    const float *bpos;       // [nb] breakpoint positions (PL)
    const int *bstart;       // [k+1] first breakpoint of each interval (PL)
    int nb, ns;              // breakpoints, samples (PL)
    float smin, sh;          // sample j sits at smin + j*sh (PL)
    int blk_off;             // first block of a band launch (0: the whole grid)
    const int *live;         // batch member run by the single-instance kernels:
                             // their blocks return while *live == 0 (null: run)
    int *err;                // set non-zero by a kernel whose bounded wait for a
                             // bulk copy gave up (null: not recorded)
};

// Device state of one problem instance (all float32, see include/lift.h).
struct LiftState {
    float2 *x;      // [N][k] {u, s}
    float2 *xbar;   // [N][k] {ubar, sbar}
    float4 *y;      // [N][k] {v, z, px, py}
    float *q;       // [N]
    float *pz;      // [N][k] third component of p_i (volumes; null on images)
};

// One instance of a batch: its parameters, its state and its first tile in
// the batch's global tile list.
struct InstDesc {
    LiftParams P;
    LiftState S;
    int tile0, ntiles;      // its tiles in the batch's tile list (primal step)
    int strip0, nstrips;    // its strips in the batch's strip list (dual step)
};

// Adjoint buffers of the differentiable solve (adjoint.cu).
struct AdjState {
    float2 *ax, *axb;   // adjoints of x and xbar
    float4 *ay;         // adjoint of y
    float *aq;          // adjoint of q
    float2 *G, *A;      // per-iteration temporaries for the neighbour gathers
    float *gf;          // dL/df accumulated per pixel
    double *partial;    // per-block scalar partials
    double *acc;        // {dL/dlambda, dL/dalpha, dL/dnu}
};

constexpr int kStepThreads = 256;

// pdhg_step.cu
cudaError_t launch_dual_step(const LiftParams &P, const LiftState &S, cudaStream_t st);
// The half-steps on the tiles [t0, t1) only (t0 even): one band of a banded
// iteration graph.
cudaError_t launch_dual_band(const LiftParams &P, const LiftState &S, int t0, int t1,
                             cudaStream_t st);
cudaError_t launch_primal_band(const LiftParams &P, const LiftState &S, int t0, int t1,
                               cudaStream_t st);
cudaError_t launch_primal_step(const LiftParams &P, const LiftState &S, cudaStream_t st);
// One whole iteration from Sin into Sout (images, quadratic kinds; Sin is not
// modified): bitwise the in-place iteration of Sin.
cudaError_t launch_iteration_into(const LiftParams &P, const LiftState &Sin, const LiftState &Sout,
                                  cudaStream_t st);
// The half-steps on the pixels [p0, p1) of an image.  Tiles (the primal
// step's, and the dual step's of sampled costs) start on the pixels
// congruent to `origin` modulo the tile length, so the
// pixel range of one band of a larger image, given the index that the
// image's first pixel would have, runs its records in the same tile
// positions (and the same scan order) as the whole image.
cudaError_t launch_dual_range(const LiftParams &P, const LiftState &S, int p0, int p1,
                              int origin, cudaStream_t st);
cudaError_t launch_primal_range(const LiftParams &P, const LiftState &S, int p0, int p1,
                                int origin, cudaStream_t st);

// The dual strips of the merged batch members with one CTA shape: threads
// per CTA and dynamic shared bytes (the largest of the group's members),
// and their instance list (device, nstrips entries).
struct StripGroup {
    int threads = 0, bytes = 0, nstrips = 0;
    const int *strip_inst = nullptr;
};

// One iteration of the merged batch members: the dual step in one strip
// launch per group (each member in the strips of a single problem of its
// k), the primal step over their tiles of `threads` threads.  err: set
// non-zero if a bounded wait gave up.
cudaError_t launch_batch_iteration(int threads, const InstDesc *D, const int *tile_inst,
                                   const int *live, int ntiles, const StripGroup *groups,
                                   int ngroups, int *err, cudaStream_t st);
// The strip shape of a single problem with k intervals: threads per CTA and
// dynamic shared bytes.
void strip_shape_of(int k, int *threads, int *bytes, int *pixels);

// adjoint.cu
int adjoint_blocks(const LiftParams &P);
cudaError_t launch_adj_seed(const LiftParams &P, const float *grad_u, float2 *ax, cudaStream_t st);
cudaError_t launch_adj_iteration(const LiftParams &P, const LiftState &Sn, const LiftState &Sn1,
                                 const AdjState &A, cudaStream_t st);
cudaError_t launch_adj_finish(const LiftParams &P, const AdjState &Aj, cudaStream_t st);

// resident.cu: whole check intervals of a small image problem inside one
// thread-block cluster, the state in shared memory.
struct ResidentPlan {
    bool ok = false;
    int ctas = 0;      // CTAs of the cluster (one cluster)
    int ppc = 0;       // pixels per CTA (whole tiles)
    size_t smem = 0;   // dynamic shared memory per CTA
};
bool plan_resident(const LiftParams &P, ResidentPlan &R);
cudaError_t launch_resident(const LiftParams &P, const LiftState &S, int iters,
                            const ResidentPlan &R, cudaStream_t st);

// setup_reduce.cu
cudaError_t launch_pl_setup(const LiftParams &P, float *rhat, cudaStream_t st);
// Writes per-block partial sums {P_hat, D, E_nc} to partial[nblocks] and the
// final sums to out[3]; nblocks = energy_blocks(P).
int energy_blocks(const LiftParams &P);
cudaError_t launch_energy(const LiftParams &P, const LiftState &S, double *partial,
                          double *out, cudaStream_t st);
// The same over the pixels [p0, p1) only (their differences still read the
// neighbours outside); partial holds (p1 - p0 + 255) / 256 blocks' sums.
cudaError_t launch_energy_range(const LiftParams &P, const LiftState &S, int p0, int p1,
                                double *partial, double *out, cudaStream_t st);
cudaError_t launch_unlift(const LiftParams &P, const float2 *x, float *out, cudaStream_t st);
// out[0] = sum |u - u'|^2/tau_u + |s - s'|^2/tau_s, out[1] = sum over the dual
// records |.|^2/sigma, both in the metric of the theta = 1 steps (the
// current steps are those of balance theta).
cudaError_t launch_movement(const LiftParams &P, const LiftState &S, const LiftState &Sprev,
                            float theta, double *partial, double *out, cudaStream_t st);
// a <- a + w (x - a) over the nk records of S.x, S.y (and S.pz when apz is
// not null) and the npix values of S.q; first: a <- x.
cudaError_t launch_average(const LiftState &S, float2 *ax, float4 *ay, float *apz, float *aq,
                           size_t nk, size_t npix, float w, bool first, cudaStream_t st);
cudaError_t launch_proj_epi(const LiftParams &P, const int *pix, const int *interval,
                            const float *y0, const float *h0, float *y, float *h, int n,
                            cudaStream_t st);
cudaError_t launch_envelope(const LiftParams &P, const int *pix, const int *interval,
                            const float *t, float *out, int n, cudaStream_t st);

}  // namespace lift
