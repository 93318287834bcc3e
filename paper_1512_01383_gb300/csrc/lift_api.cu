// Host implementation of the C ABI declared in include/lift.h.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/lift.h"
#include "lift_params.h"

using lift::LiftParams;
using lift::LiftState;

constexpr int kMaxBands = 8;

struct lift_ctx {
    cudaStream_t stream = nullptr;
    int kind = 0;
    int H = 0, W = 0, k = 0, N = 0;
    int check_every = 100;
    LiftParams P{};
    LiftState S{};
    float4 *icst = nullptr;
    float4 *steps = nullptr;   // {tau_u, sigma_q, sigma_p, 0} (see LiftParams::steps)
    float *f = nullptr;        // quadratic kinds
    float *cost = nullptr;     // PL raw samples
    float *rhat = nullptr;     // PL convexified values
    float *bpos = nullptr;     // PL breakpoints
    int *bstart = nullptr;     // PL interval starts
    float *ubuf = nullptr;     // unlift staging for host output
    double *partial = nullptr; // energy partial sums (per block)
    double *dout = nullptr;    // energy sums (device)
    double *hout = nullptr;    // energy sums (pinned host)
    size_t data_elems = 0;     // N (quadratic) or N*ns (PL)
    // differentiable solve
    char *ckpt = nullptr;      // checkpoints: states at iterations 0, C, 2C, ...
    char *seg = nullptr;       // one segment's states, recomputed in the backward pass
    int unrolled_iters = 0, ckpt_every = 0, ckpt_count = 0, seg_cap = 0;
    // bumped by every call that changes what a reverse pass would
    // differentiate (forward, parameters, data, reset)
    unsigned long long generation = 0;
    lift::AdjState adj{};
    void *adj_arena = nullptr;
    // graph replay of whole check intervals (lift_iterate)
    cudaStream_t gstream = nullptr;     // private stream the graph runs on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_iters = 0;
    // banded graph: per band a stream for the dual and one for the primal
    // half-steps, ordered by events (see ensure_iter_graph)
    int bands_req = 0;                  // lift_set_bands: 0 = automatic
    long long l2_bytes = 0;             // the device's L2 size (the automatic band count)
    cudaStream_t band_s[2 * kMaxBands] = {};
    cudaEvent_t band_e[2 * kMaxBands + 1] = {};
    // adaptive primal/dual balance (lift_solve)
    lift_spec spec_copy{};              // data pointers cleared; for re-deriving steps
    double theta = 1.0;
    double adapt_w = 0.5;               // weight of the next re-balancing step
    int adaptive = 0;
    char *prev = nullptr;               // state at the previous check
    bool prev_valid = false;
    // small problems: whole calls of lift_iterate inside one cluster
    lift::ResidentPlan resident{};
    bool resident_on = true;            // caller's preference (lift_set_resident)
    // a band of rows of a larger image (lift_create_band): the own rows are
    // the local pixels [own0, own1), with one halo row above (halo_up) and
    // below (halo_dn) where the image goes on; torg: the local index, modulo
    // the primal tile length, that the image's first pixel would have
    bool band = false;
    int halo_up = 0, halo_dn = 0, own0 = 0, own1 = 0, torg = 0;
    // running average of the iterate (lift_average): x, y (and pz) records,
    // allocated on the first accumulation; avg_count iterates in it
    float2 *avg_x = nullptr;
    float4 *avg_y = nullptr;
    float *avg_pz = nullptr;
    float *avg_q = nullptr;
    long long avg_count = 0;
};

namespace {

// The CUDA error behind the calling thread's last LIFT_ERR_CUDA.
thread_local cudaError_t g_last_cuda_error = cudaSuccess;

#define LIFT_CK(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            g_last_cuda_error = e_;                    \
            return LIFT_ERR_CUDA;                      \
        }                                              \
    } while (0)

int dev_alloc(void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the non-sticky error
        return LIFT_ERR_OOM;
    }
    return e == cudaSuccess ? LIFT_OK : LIFT_ERR_CUDA;
}

void free_ctx(lift_ctx *h)
{
    if (!h) return;
    void *ptrs[] = {h->S.x, h->S.xbar, h->S.y, h->S.q, h->S.pz, h->icst, h->steps, h->f, h->cost,
                    h->rhat, h->bpos, h->bstart, h->ubuf, h->partial, h->dout};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->ckpt) cudaFree(h->ckpt);
    if (h->seg) cudaFree(h->seg);
    if (h->adj_arena) cudaFree(h->adj_arena);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    for (cudaStream_t st : h->band_s)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : h->band_e)
        if (ev) cudaEventDestroy(ev);
    if (h->prev) cudaFree(h->prev);
    if (h->avg_x) cudaFree(h->avg_x);
    if (h->avg_y) cudaFree(h->avg_y);
    if (h->avg_pz) cudaFree(h->avg_pz);
    if (h->avg_q) cudaFree(h->avg_q);
    if (h->hout) cudaFreeHost(h->hout);
    delete h;
}

bool is_finite(double x) { return std::isfinite(x); }

int validate(const lift_spec *s)
{
    if (s->kind < LIFT_QUAD || s->kind > LIFT_PERIODIC_QUAD) return LIFT_ERR_SPEC;
    if (s->H < 1 || s->W < 1 || s->D < 0) return LIFT_ERR_SPEC;
    if (s->L < 2 || s->L > LIFT_MAX_K + 1) return LIFT_ERR_SPEC;
    const long long N = static_cast<long long>(std::max(s->D, 1)) * s->H * s->W;
    if (N * (s->L - 1) > (1LL << 31) - 1) return LIFT_ERR_SPEC;
    if (!is_finite(s->gamma_min) || !is_finite(s->gamma_max) || !(s->gamma_max > s->gamma_min))
        return LIFT_ERR_SPEC;
    if (!is_finite(s->lambda) || s->lambda < 0.0) return LIFT_ERR_SPEC;
    if (!is_finite(s->step_balance)) return LIFT_ERR_SPEC;
    if (s->tv_anisotropic != 0 && s->tv_anisotropic != 1) return LIFT_ERR_SPEC;
    if (s->kind != LIFT_PL_SAMPLED) {
        if (!s->f) return LIFT_ERR_SPEC;
        if (!is_finite(s->alpha) || !(s->alpha > 0.0)) return LIFT_ERR_SPEC;
        if (s->kind != LIFT_QUAD && (!is_finite(s->nu) || !(s->nu > 0.0))) return LIFT_ERR_SPEC;
    } else {
        if (!s->cost || s->n_samples < 2) return LIFT_ERR_SPEC;
        if (!is_finite(s->sample_min) || !is_finite(s->sample_max) || !(s->sample_max > s->sample_min))
            return LIFT_ERR_SPEC;
        const double tol = 1e-9 * (fabs(s->sample_max) + fabs(s->sample_min) + 1.0);
        if (s->sample_min > s->gamma_min + tol || s->sample_max < s->gamma_max - tol)
            return LIFT_ERR_SPEC;
    }
    return LIFT_OK;
}

double label(const lift_spec *s, int j)
{
    const int k = s->L - 1;
    return s->gamma_min + (s->gamma_max - s->gamma_min) * static_cast<double>(j) / k;
}

// Breakpoints of the PL data term: every label and every sample position
// strictly inside Gamma; bstart[i] indexes label gamma_i in the sorted list.
int pl_breakpoints(const lift_spec *s, std::vector<float> &pos, std::vector<int> &bstart)
{
    const int k = s->L - 1;
    const double sh = (s->sample_max - s->sample_min) / (s->n_samples - 1);
    const double eps = 1e-9 * (fabs(s->gamma_max) + fabs(s->gamma_min) + 1.0);
    std::vector<double> p;
    bstart.assign(k + 1, 0);
    int j = 0;
    for (int i = 0; i <= k; ++i) {
        const double g = label(s, i);
        // samples strictly between the previous label and this one
        for (; j < s->n_samples; ++j) {
            const double t = s->sample_min + sh * j;
            if (t >= g - eps) break;
            if (i > 0 && t > label(s, i - 1) + eps) p.push_back(t);
        }
        if (j < s->n_samples && fabs(s->sample_min + sh * j - g) <= eps) ++j;  // coincides
        bstart[i] = static_cast<int>(p.size());
        p.push_back(g);
    }
    for (int i = 0; i < k; ++i)
        if (bstart[i + 1] - bstart[i] + 1 > 512) return LIFT_ERR_SPEC;
    pos.assign(p.begin(), p.end());
    return LIFT_OK;
}

// Kernel parameters of one problem (everything but the device pointers):
// step sizes from the reciprocal absolute row / column sums of the operator,
// scaled by the primal/dual balance theta; per-interval constants in ic.
void make_params(const lift_spec *spec, int threads, LiftParams &P, std::vector<float4> &ic)
{
    const int k = spec->L - 1;
    const double d = label(spec, 1) - label(spec, 0);
    const double gL = label(spec, k);
    const double th = spec->step_balance > 0.0 ? spec->step_balance : 1.0;
    ic.assign(k, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    for (int i = 0; i < k; ++i) {
        const double gi = label(spec, i);
        const double tau_s = th / (1.0 + fabs(gi) + (i + 1) * d);
        const double row_v = 1.0 + fabs(gi) + (gL - label(spec, i + 1));
        const double sig = 1.0 / (th * std::max(row_v, 1.0));
        ic[i] = make_float4(static_cast<float>(gi), static_cast<float>(tau_s),
                            static_cast<float>(sig), static_cast<float>(spec->lambda * d));
    }
    P = LiftParams{};
    P.D = std::max(spec->D, 1);
    P.H = spec->H; P.W = spec->W; P.k = k;
    P.HW = spec->H * spec->W;
    P.N = P.D * P.HW;
    P.kind = spec->kind;
    P.aniso = spec->tv_anisotropic ? 1 : 0;
    P.ppb = threads / k;
    P.inv_k = 1.0f / static_cast<float>(k);
    P.delta = static_cast<float>(d);
    P.inv_delta = static_cast<float>(1.0 / d);
    {
        // exact division by W for 0 <= pix < 2^31: with l = ceil(log2 W) and
        // M = floor(2^(31+l) / W) + 1, floor(pix*M / 2^(31+l)) = floor(pix/W)
        // because the excess pix*(M - 2^(31+l)/W)/2^(31+l) < 2^-l <= 1/W
        int l = 0;
        while ((1LL << l) < spec->W) ++l;
        P.wshift = 31 + l;
        P.wmul = ((1ULL << P.wshift) / static_cast<unsigned long long>(spec->W)) + 1ULL;
        // the same for the slice of a global row index, row / H
        l = 0;
        while ((1LL << l) < spec->H) ++l;
        P.hshift = 31 + l;
        P.hmul = ((1ULL << P.hshift) / static_cast<unsigned long long>(spec->H)) + 1ULL;
    }
    P.gmin = static_cast<float>(spec->gamma_min);
    P.lam = static_cast<float>(spec->lambda);
    P.alpha = static_cast<float>(spec->alpha);
    P.inv_alpha = spec->alpha > 0.0 ? static_cast<float>(1.0 / spec->alpha) : 0.0f;
    P.nu = static_cast<float>(spec->nu);
    P.wtrunc = spec->kind == LIFT_TRUNC_QUAD ? static_cast<float>(sqrt(spec->nu / spec->alpha)) : 0.0f;
    // the column of u holds 1 + 2d entries: 1 + 4 on an image, 1 + 6 on a volume
    P.tau_u = static_cast<float>(th / (P.D > 1 ? 7.0 : 5.0));
    P.sigma_q = static_cast<float>(1.0 / (th * (gL - label(spec, 0))));
    P.sigma_p = static_cast<float>(0.5 / th);
}

int upload_data(lift_handle h, const float *data, int on_host)
{
    float *dst = h->kind == LIFT_PL_SAMPLED ? h->cost : h->f;
    LIFT_CK(cudaMemcpyAsync(dst, data, h->data_elems * sizeof(float),
                            on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            h->stream));
    if (h->kind == LIFT_PL_SAMPLED) LIFT_CK(lift::launch_pl_setup(h->P, h->rhat, h->stream));
    return LIFT_OK;
}

// Re-derive the step sizes for a new balance theta (icst and the scalar
// steps; everything else of the parameters is unchanged).
float4 step_scalars(const LiftParams &P)
{
    return make_float4(P.tau_u, P.sigma_q, P.sigma_p, 0.0f);
}

int set_theta(lift_handle h, double theta)
{
    lift_spec sp = h->spec_copy;
    sp.step_balance = theta;
    LiftParams P2;
    std::vector<float4> ic;
    make_params(&sp, lift::kStepThreads, P2, ic);
    LIFT_CK(cudaMemcpyAsync(h->icst, ic.data(), ic.size() * sizeof(float4), cudaMemcpyHostToDevice,
                            h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));   // ic dies here
    h->P.tau_u = P2.tau_u;
    h->P.sigma_q = P2.sigma_q;
    h->P.sigma_p = P2.sigma_p;
    h->theta = theta;
    // the step kernels read icst and the scalar steps from device memory, so
    // the captured iteration graph stays valid
    const float4 st = step_scalars(h->P);
    LIFT_CK(cudaMemcpyAsync(h->steps, &st, sizeof(float4), cudaMemcpyHostToDevice, h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));   // st dies here
    return LIFT_OK;
}

int save_prev(lift_handle h)
{
    const size_t sb = lift_state_bytes(h);
    if (!h->prev) {
        const int rc = dev_alloc(reinterpret_cast<void **>(&h->prev), (sb + 255) & ~size_t(255));
        if (rc != LIFT_OK) return rc;
    }
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    char *b = h->prev;
    LIFT_CK(cudaMemcpyAsync(b, h->S.x, Nk * sizeof(float2), cudaMemcpyDeviceToDevice, h->stream));
    LIFT_CK(cudaMemcpyAsync(b + 2 * Nk * sizeof(float2), h->S.y, Nk * sizeof(float4),
                            cudaMemcpyDeviceToDevice, h->stream));
    LIFT_CK(cudaMemcpyAsync(b + 2 * Nk * sizeof(float2) + Nk * sizeof(float4), h->S.q,
                            h->N * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    if (h->S.pz)
        LIFT_CK(cudaMemcpyAsync(b + 2 * Nk * sizeof(float2) + Nk * sizeof(float4) +
                                    h->N * sizeof(float),
                                h->S.pz, Nk * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    h->prev_valid = true;
    return LIFT_OK;
}

// log theta <- (1 - w) log theta + w log(dx/dy), dx, dy the movements since
// the previous check in the metric of the theta = 1 steps; the weight w starts
// at 1/2 and shrinks by 0.95 per check, so the steps settle (a decaying
// adaptation, as in the adaptive primal-dual steps the paper cites).
int rebalance(lift_handle h)
{
    if (!h->prev_valid) return LIFT_OK;
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    LiftState Sp;
    Sp.x = reinterpret_cast<float2 *>(h->prev);
    Sp.xbar = nullptr;
    Sp.y = reinterpret_cast<float4 *>(h->prev + 2 * Nk * sizeof(float2));
    Sp.q = reinterpret_cast<float *>(h->prev + 2 * Nk * sizeof(float2) + Nk * sizeof(float4));
    Sp.pz = h->S.pz ? Sp.q + h->N : nullptr;
    LIFT_CK(lift::launch_movement(h->P, h->S, Sp, static_cast<float>(h->theta), h->partial, h->dout,
                                  h->stream));
    LIFT_CK(cudaMemcpyAsync(h->hout, h->dout, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    const double dx = h->hout[0], dy = h->hout[1];
    if (!(dx > 0.0) || !(dy > 0.0) || !is_finite(dx) || !is_finite(dy)) return LIFT_OK;
    const double w = h->adapt_w;
    double th = exp((1.0 - w) * log(h->theta) + w * 0.5 * log(dx / dy));
    th = std::min(std::max(th, 1e-4), 1e6);
    h->adapt_w *= 0.95;
    return set_theta(h, th);
}

}  // namespace

extern "C" {

int lift_create(const lift_spec *spec, void *stream, lift_handle *out)
{
    if (!spec || !out) return LIFT_ERR_ARG;
    *out = nullptr;
    int rc = validate(spec);
    if (rc != LIFT_OK) return rc;

    lift_ctx *h = new (std::nothrow) lift_ctx();
    if (!h) return LIFT_ERR_OOM;
    h->stream = static_cast<cudaStream_t>(stream);
    h->kind = spec->kind;
    h->H = spec->H;
    h->W = spec->W;
    h->k = spec->L - 1;
    h->N = std::max(spec->D, 1) * spec->H * spec->W;
    h->check_every = spec->check_every > 0 ? spec->check_every : 100;
    const int k = h->k;
    const size_t N = static_cast<size_t>(h->N), Nk = N * k;

    std::vector<float4> ic;
    LiftParams &P = h->P;
    make_params(spec, lift::kStepThreads, P, ic);
    h->spec_copy = *spec;
    h->spec_copy.f = nullptr;
    h->spec_copy.cost = nullptr;
    h->theta = spec->step_balance > 0.0 ? spec->step_balance : 1.0;
    h->adaptive = spec->adaptive_balance ? 1 : 0;

    std::vector<float> bp;
    std::vector<int> bs;
    if (spec->kind == LIFT_PL_SAMPLED) {
        rc = pl_breakpoints(spec, bp, bs);
        if (rc != LIFT_OK) { free_ctx(h); return rc; }
        P.nb = static_cast<int>(bp.size());
        P.ns = spec->n_samples;
        P.smin = static_cast<float>(spec->sample_min);
        P.sh = static_cast<float>((spec->sample_max - spec->sample_min) / (spec->n_samples - 1));
    }

#define ALLOC(ptr, bytes)                                              \
    do {                                                               \
        int r_ = dev_alloc(reinterpret_cast<void **>(&(ptr)), (bytes)); \
        if (r_ != LIFT_OK) { free_ctx(h); return r_; }                 \
    } while (0)
#define CUDA_OR_FAIL(call)                                             \
    do {                                                               \
        if ((call) != cudaSuccess) { free_ctx(h); return LIFT_ERR_CUDA; } \
    } while (0)

    ALLOC(h->S.x, Nk * sizeof(float2));
    ALLOC(h->S.xbar, Nk * sizeof(float2));
    ALLOC(h->S.y, Nk * sizeof(float4));
    ALLOC(h->S.q, N * sizeof(float));
    if (P.D > 1) ALLOC(h->S.pz, Nk * sizeof(float));
    ALLOC(h->icst, k * sizeof(float4));
    ALLOC(h->steps, sizeof(float4));
    ALLOC(h->ubuf, N * sizeof(float));
    ALLOC(h->partial, 3 * sizeof(double) * lift::energy_blocks(P));
    // three energy sums and, in the fourth slot, the kernels' error word
    ALLOC(h->dout, 4 * sizeof(double));
    if (cudaMallocHost(reinterpret_cast<void **>(&h->hout), 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        h->hout = nullptr;
        free_ctx(h);
        return LIFT_ERR_OOM;
    }
    if (spec->kind == LIFT_PL_SAMPLED) {
        h->data_elems = N * spec->n_samples;
        ALLOC(h->cost, h->data_elems * sizeof(float));
        ALLOC(h->rhat, N * P.nb * sizeof(float));
        ALLOC(h->bpos, bp.size() * sizeof(float));
        ALLOC(h->bstart, bs.size() * sizeof(int));
        CUDA_OR_FAIL(cudaMemcpyAsync(h->bpos, bp.data(), bp.size() * sizeof(float),
                                     cudaMemcpyHostToDevice, h->stream));
        CUDA_OR_FAIL(cudaMemcpyAsync(h->bstart, bs.data(), bs.size() * sizeof(int),
                                     cudaMemcpyHostToDevice, h->stream));
    } else {
        h->data_elems = N;
        ALLOC(h->f, N * sizeof(float));
    }
#undef ALLOC
    CUDA_OR_FAIL(cudaMemsetAsync(h->dout, 0, 4 * sizeof(double), h->stream));
    P.err = reinterpret_cast<int *>(h->dout + 3);
    P.icst = h->icst;
    P.steps = h->steps;
    P.f = h->f;
    P.rhat = h->rhat;
    P.cost = h->cost;
    P.bpos = h->bpos;
    P.bstart = h->bstart;

    CUDA_OR_FAIL(cudaMemcpyAsync(h->icst, ic.data(), k * sizeof(float4), cudaMemcpyHostToDevice,
                                 h->stream));
    const float4 st0 = step_scalars(P);
    CUDA_OR_FAIL(cudaMemcpyAsync(h->steps, &st0, sizeof(float4), cudaMemcpyHostToDevice, h->stream));
    const float *data = spec->kind == LIFT_PL_SAMPLED ? spec->cost : spec->f;
    rc = upload_data(h, data, spec->data_on_host);
    if (rc != LIFT_OK) { free_ctx(h); return rc; }
    rc = lift_reset(h);
    if (rc != LIFT_OK) { free_ctx(h); return rc; }
    lift::plan_resident(h->P, h->resident);
    {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess)
            h->l2_bytes = l2;
        else
            cudaGetLastError();
    }
    // host-side vectors die with this scope: finish the uploads first
    CUDA_OR_FAIL(cudaStreamSynchronize(h->stream));
#undef CUDA_OR_FAIL
    *out = h;
    return LIFT_OK;
}

int lift_create_band(const lift_spec *spec, int row0, int row1, void *stream, lift_handle *out)
{
    if (!spec || !out) return LIFT_ERR_ARG;
    *out = nullptr;
    int rc = validate(spec);
    if (rc != LIFT_OK) return rc;
    if (spec->D > 1) return LIFT_ERR_SPEC;               // images only
    if (row0 < 0 || row1 > spec->H || row0 >= row1) return LIFT_ERR_ARG;
    const int up = row0 > 0 ? 1 : 0, dn = row1 < spec->H ? 1 : 0;
    // the local image: the own rows and the halo rows, data from the same rows
    lift_spec loc = *spec;
    loc.H = row1 - row0 + up + dn;
    const size_t first = static_cast<size_t>(row0 - up) * spec->W;
    if (spec->kind == LIFT_PL_SAMPLED) {
        if (!spec->cost) return LIFT_ERR_ARG;
        loc.cost = spec->cost + first * static_cast<size_t>(spec->n_samples);
    } else {
        if (!spec->f) return LIFT_ERR_ARG;
        loc.f = spec->f + first;
    }
    rc = lift_create(&loc, stream, out);
    if (rc != LIFT_OK) return rc;
    lift_handle h = *out;
    h->band = true;
    h->halo_up = up;
    h->halo_dn = dn;
    h->own0 = up * spec->W;
    h->own1 = (up + row1 - row0) * spec->W;
    const int ppb = h->P.ppb;
    h->torg = static_cast<int>((static_cast<size_t>(ppb) - first % ppb) % ppb);
    h->resident_on = false;
    return LIFT_OK;
}

int lift_band_halo_bytes(lift_handle h, int which, size_t *bytes)
{
    if (!h || !bytes || !h->band) return LIFT_ERR_ARG;
    const size_t rec = static_cast<size_t>(h->W) * h->k;
    if (which == LIFT_HALO_PRIMAL) *bytes = 2 * rec * sizeof(float2);
    else if (which == LIFT_HALO_DUAL) *bytes = rec * sizeof(float4);
    else return LIFT_ERR_ARG;
    return LIFT_OK;
}

// Rows of the local image: the first and last own row, the halo rows.
static size_t row_rec(lift_handle h, int local_row)
{
    return static_cast<size_t>(local_row) * h->W * h->k;
}

int lift_band_export(lift_handle h, int which, void *dst, int on_host)
{
    if (!h || !dst || !h->band) return LIFT_ERR_ARG;
    const size_t rec = static_cast<size_t>(h->W) * h->k;
    const cudaMemcpyKind kd = on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    char *d = static_cast<char *>(dst);
    if (which == LIFT_HALO_PRIMAL) {            // first own row, for the band above
        if (!h->halo_up) return LIFT_ERR_ARG;
        const size_t o = row_rec(h, h->halo_up);
        LIFT_CK(cudaMemcpyAsync(d, h->S.x + o, rec * sizeof(float2), kd, h->stream));
        LIFT_CK(cudaMemcpyAsync(d + rec * sizeof(float2), h->S.xbar + o, rec * sizeof(float2), kd,
                                h->stream));
    } else if (which == LIFT_HALO_DUAL) {       // last own row, for the band below
        if (!h->halo_dn) return LIFT_ERR_ARG;
        const size_t o = row_rec(h, h->own1 / h->W - 1);
        LIFT_CK(cudaMemcpyAsync(d, h->S.y + o, rec * sizeof(float4), kd, h->stream));
    } else {
        return LIFT_ERR_ARG;
    }
    if (on_host) LIFT_CK(cudaStreamSynchronize(h->stream));
    return LIFT_OK;
}

int lift_band_import(lift_handle h, int which, const void *src, int on_host)
{
    if (!h || !src || !h->band) return LIFT_ERR_ARG;
    const size_t rec = static_cast<size_t>(h->W) * h->k;
    const cudaMemcpyKind kd = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const char *s = static_cast<const char *>(src);
    if (which == LIFT_HALO_PRIMAL) {            // into the halo row below
        if (!h->halo_dn) return LIFT_ERR_ARG;
        const size_t o = row_rec(h, h->own1 / h->W);
        LIFT_CK(cudaMemcpyAsync(h->S.x + o, s, rec * sizeof(float2), kd, h->stream));
        LIFT_CK(cudaMemcpyAsync(h->S.xbar + o, s + rec * sizeof(float2), rec * sizeof(float2), kd,
                                h->stream));
    } else if (which == LIFT_HALO_DUAL) {       // into the halo row above
        if (!h->halo_up) return LIFT_ERR_ARG;
        LIFT_CK(cudaMemcpyAsync(h->S.y, s, rec * sizeof(float4), kd, h->stream));
    } else {
        return LIFT_ERR_ARG;
    }
    // host sources may be reused after return
    if (on_host) LIFT_CK(cudaStreamSynchronize(h->stream));
    return LIFT_OK;
}

void lift_destroy(lift_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_ctx(h);
}

// The stored forward no longer matches the handle: a reverse pass now fails.
static void invalidate_unrolled(lift_handle h)
{
    h->unrolled_iters = 0;
    ++h->generation;
    h->avg_count = 0;   // the running average belongs to the old problem or start
}

int lift_set_data(lift_handle h, const float *data, int on_host)
{
    if (!h || !data) return LIFT_ERR_ARG;
    invalidate_unrolled(h);
    return upload_data(h, data, on_host);
}

int lift_reset(lift_handle h)
{
    if (!h) return LIFT_ERR_ARG;
    invalidate_unrolled(h);
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    LIFT_CK(cudaMemsetAsync(h->S.x, 0, Nk * sizeof(float2), h->stream));
    LIFT_CK(cudaMemsetAsync(h->S.xbar, 0, Nk * sizeof(float2), h->stream));
    LIFT_CK(cudaMemsetAsync(h->S.y, 0, Nk * sizeof(float4), h->stream));
    LIFT_CK(cudaMemsetAsync(h->S.q, 0, h->N * sizeof(float), h->stream));
    if (h->S.pz) LIFT_CK(cudaMemsetAsync(h->S.pz, 0, Nk * sizeof(float), h->stream));
    h->prev_valid = false;
    h->adapt_w = 0.5;
    return LIFT_OK;
}

// Drop the captured check-interval graph (its kernels hold the parameters by
// value, so any parameter change must re-capture).
static void drop_iter_graph(lift_handle h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    h->graph_iters = 0;
}

static int step_tiles(lift_handle h) { return (h->P.N + h->P.ppb - 1) / h->P.ppb; }

// Number of bands of the iteration graph.  By default 4 for problems of at
// least 4096 tiles, where the dual steps of some bands overlap the primal
// steps of others; but 1 where the dual step runs in strips and the state
// exceeds three quarters of L2: there both half-steps stream from DRAM at
// near its bandwidth and overlapping them only makes them contend (512^2,
// L = 20, 160 MB: 74 us per iteration in one band, 87 in four; at L = 10,
// 76 MB, four bands gain 6 %).  Fewer bands (down to 1) while a band would
// hold less than the largest neighbour offset (a row of an image, a slice of
// a volume), so that every halo value lies in the same or an adjacent band.
static int bands_used(lift_handle h)
{
    int B = 1;
    if (h->bands_req > 0) {
        B = std::min(h->bands_req, kMaxBands);
    } else if (step_tiles(h) >= 4096) {
        const bool strips = h->P.D == 1 && h->kind != LIFT_PL_SAMPLED;
        const long long state = static_cast<long long>(lift_state_bytes(h));
        B = strips && h->l2_bytes > 0 && 4 * state > 3 * h->l2_bytes ? 1 : 4;
    }
    const long long span = h->P.D > 1 ? h->P.HW : h->P.W;
    // boundaries fall on even tiles, so a band holds at least T/B - 2 tiles
    while (B > 1 && (static_cast<long long>(step_tiles(h) / B - 2) * h->P.ppb <= span)) --B;
    return B;
}

static int launch_iters(lift_handle h, cudaStream_t st, int iters)
{
    for (int n = 0; n < iters; ++n) {
        LIFT_CK(lift::launch_dual_step(h->P, h->S, st));
        LIFT_CK(lift::launch_primal_step(h->P, h->S, st));
    }
    return LIFT_OK;
}

// Capture check_every iterations once on a private stream; later calls replay
// the graph there, ordered after earlier work of the handle's stream and
// before later work (events), which removes the per-launch host cost that
// dominates small problems.
static int ensure_iter_graph(lift_handle h)
{
    if (h->gexec && h->graph_iters == h->check_every) return LIFT_OK;
    drop_iter_graph(h);
    if (!h->gstream) {
        LIFT_CK(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
        LIFT_CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
        LIFT_CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    }
    const int B = bands_used(h);
    if (B > 1 && !h->band_s[0]) {
        for (int j = 0; j < 2 * kMaxBands; ++j)
            LIFT_CK(cudaStreamCreateWithFlags(&h->band_s[j], cudaStreamNonBlocking));
        for (int j = 0; j < 2 * kMaxBands + 1; ++j)
            LIFT_CK(cudaEventCreateWithFlags(&h->band_e[j], cudaEventDisableTiming));
    }
    LIFT_CK(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal));
    int rc = LIFT_OK;
    if (B == 1) {
        rc = launch_iters(h, h->gstream, h->check_every);
    } else {
        // Rows of tiles in B bands (boundaries on even tiles, each at least a
        // neighbour offset long).  Dual D(j, n) reads ubar of band j and of the
        // first row of band j+1 and overwrites y of band j, which the primal
        // step of band j+1 reads: it follows P(j, n-1) and P(j+1, n-1).  P(j,
        // n) reads p of band j and of the last row of band j-1 and overwrites
        // xbar of band j, which D(j-1, n) reads: it follows D(j, n) and D(j-1,
        // n).  The graph keeps exactly these orders, so every half-step reads
        // what it reads in the one-stream order (the same result, bitwise),
        // while the issue-bound dual steps of some bands run beside the
        // memory-bound primal steps of others.
        const int T = step_tiles(h);
        int b0[kMaxBands + 1];
        for (int j = 0; j <= B; ++j)
            b0[j] = j == B ? T : static_cast<int>(static_cast<long long>(T) * j / B) / 2 * 2;
        cudaStream_t *sD = h->band_s, *sP = h->band_s + kMaxBands;
        cudaEvent_t *eD = h->band_e, *eP = h->band_e + kMaxBands, fork = h->band_e[2 * kMaxBands];
        cudaError_t e = cudaEventRecord(fork, h->gstream);
        for (int j = 0; j < B && e == cudaSuccess; ++j) {
            e = cudaStreamWaitEvent(sD[j], fork, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(sP[j], fork, 0);
        }
        for (int n = 0; n < h->check_every && e == cudaSuccess; ++n) {
            for (int j = 0; j < B && e == cudaSuccess; ++j) {
                if (n > 0) {
                    e = cudaStreamWaitEvent(sD[j], eP[j], 0);
                    if (e == cudaSuccess && j + 1 < B) e = cudaStreamWaitEvent(sD[j], eP[j + 1], 0);
                }
                if (e == cudaSuccess) e = lift::launch_dual_band(h->P, h->S, b0[j], b0[j + 1], sD[j]);
                if (e == cudaSuccess) e = cudaEventRecord(eD[j], sD[j]);
            }
            for (int j = 0; j < B && e == cudaSuccess; ++j) {
                e = cudaStreamWaitEvent(sP[j], eD[j], 0);
                if (e == cudaSuccess && j > 0) e = cudaStreamWaitEvent(sP[j], eD[j - 1], 0);
                if (e == cudaSuccess) e = lift::launch_primal_band(h->P, h->S, b0[j], b0[j + 1], sP[j]);
                if (e == cudaSuccess) e = cudaEventRecord(eP[j], sP[j]);
            }
        }
        // join every band's last primal step into the capture stream
        for (int j = 0; j < B && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(h->gstream, eP[j], 0);
        if (e != cudaSuccess) rc = LIFT_ERR_CUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->gstream, &g);
    if (rc != LIFT_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return LIFT_ERR_CUDA;
    }
    h->graph = g;
    LIFT_CK(cudaGraphInstantiate(&h->gexec, g, 0));
    h->graph_iters = h->check_every;
    return LIFT_OK;
}

int lift_iterate(lift_handle h, int iters)
{
    if (!h || iters < 0 || h->band) return LIFT_ERR_ARG;
    if (iters > 0 && h->resident.ok && h->resident_on) {
        LIFT_CK(lift::launch_resident(h->P, h->S, iters, h->resident, h->stream));
        return LIFT_OK;
    }
    const int reps = iters / h->check_every;
    if (reps > 0) {
        int rc = ensure_iter_graph(h);
        if (rc != LIFT_OK) return rc;
        LIFT_CK(cudaEventRecord(h->ev_in, h->stream));
        LIFT_CK(cudaStreamWaitEvent(h->gstream, h->ev_in, 0));
        for (int r = 0; r < reps; ++r) LIFT_CK(cudaGraphLaunch(h->gexec, h->gstream));
        LIFT_CK(cudaEventRecord(h->ev_out, h->gstream));
        LIFT_CK(cudaStreamWaitEvent(h->stream, h->ev_out, 0));
    }
    return launch_iters(h, h->stream, iters - reps * h->check_every);
}

int lift_dual_step(lift_handle h)
{
    if (!h) return LIFT_ERR_ARG;
    if (h->band) LIFT_CK(lift::launch_dual_range(h->P, h->S, h->own0, h->own1, h->torg, h->stream));
    else LIFT_CK(lift::launch_dual_step(h->P, h->S, h->stream));
    return LIFT_OK;
}

int lift_primal_step(lift_handle h)
{
    if (!h) return LIFT_ERR_ARG;
    if (h->band) LIFT_CK(lift::launch_primal_range(h->P, h->S, h->own0, h->own1, h->torg, h->stream));
    else LIFT_CK(lift::launch_primal_step(h->P, h->S, h->stream));
    return LIFT_OK;
}

int lift_energy(lift_handle h, double *primal_relaxed, double *dual, double *e_nonconvex)
{
    if (!h) return LIFT_ERR_ARG;
    if (h->band)
        LIFT_CK(lift::launch_energy_range(h->P, h->S, h->own0, h->own1, h->partial, h->dout, h->stream));
    else
        LIFT_CK(lift::launch_energy(h->P, h->S, h->partial, h->dout, h->stream));
    LIFT_CK(cudaMemcpyAsync(h->hout, h->dout, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    int err_word = 0;
    memcpy(&err_word, h->hout + 3, sizeof(int));
    if (err_word != 0) return LIFT_ERR_TIMEOUT;
    if (primal_relaxed) *primal_relaxed = h->hout[0];
    if (dual) *dual = h->hout[1];
    if (e_nonconvex) *e_nonconvex = h->hout[2];
    if (!is_finite(h->hout[0]) || !is_finite(h->hout[1]) || !is_finite(h->hout[2])) return LIFT_ERR_NAN;
    return LIFT_OK;
}

int lift_average(lift_handle h, int accumulate)
{
    if (!h || h->band || (accumulate != 0 && accumulate != 1)) return LIFT_ERR_ARG;
    if (!accumulate) {
        h->avg_count = 0;
        return LIFT_OK;
    }
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    if (!h->avg_x) {
        int rc = dev_alloc(reinterpret_cast<void **>(&h->avg_x), Nk * sizeof(float2));
        if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&h->avg_y), Nk * sizeof(float4));
        if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&h->avg_q), h->N * sizeof(float));
        if (rc == LIFT_OK && h->S.pz) rc = dev_alloc(reinterpret_cast<void **>(&h->avg_pz), Nk * sizeof(float));
        if (rc != LIFT_OK) {
            void *ps[] = {h->avg_x, h->avg_y, h->avg_q, h->avg_pz};
            for (void *q : ps)
                if (q) cudaFree(q);
            h->avg_x = nullptr;
            h->avg_y = nullptr;
            h->avg_q = nullptr;
            h->avg_pz = nullptr;
            return rc;
        }
    }
    const long long c = h->avg_count + 1;
    LIFT_CK(lift::launch_average(h->S, h->avg_x, h->avg_y, h->avg_pz, h->avg_q, Nk,
                                 static_cast<size_t>(h->N),
                                 static_cast<float>(1.0 / static_cast<double>(c)), c == 1,
                                 h->stream));
    h->avg_count = c;
    return LIFT_OK;
}

long long lift_average_count(lift_handle h)
{
    return h ? h->avg_count : -1;
}

// The handle's state with the averaged records in place of x, y (and pz).
static int average_state(lift_handle h, lift::LiftState *Sa)
{
    if (!h || h->band || h->avg_count < 1) return LIFT_ERR_ARG;
    *Sa = h->S;
    Sa->x = h->avg_x;
    Sa->xbar = h->avg_x;
    Sa->y = h->avg_y;
    Sa->pz = h->avg_pz;
    return LIFT_OK;
}

int lift_energy_average(lift_handle h, double *primal_relaxed, double *dual, double *e_nonconvex)
{
    lift::LiftState Sa{};
    const int rc = average_state(h, &Sa);
    if (rc != LIFT_OK) return rc;
    LIFT_CK(lift::launch_energy(h->P, Sa, h->partial, h->dout, h->stream));
    LIFT_CK(cudaMemcpyAsync(h->hout, h->dout, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    if (primal_relaxed) *primal_relaxed = h->hout[0];
    if (dual) *dual = h->hout[1];
    if (e_nonconvex) *e_nonconvex = h->hout[2];
    if (!is_finite(h->hout[0]) || !is_finite(h->hout[1]) || !is_finite(h->hout[2])) return LIFT_ERR_NAN;
    return LIFT_OK;
}

int lift_average_restart(lift_handle h)
{
    if (!h || h->band || h->avg_count < 1) return LIFT_ERR_ARG;
    invalidate_unrolled(h);
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    LIFT_CK(cudaMemcpyAsync(h->S.x, h->avg_x, Nk * sizeof(float2), cudaMemcpyDeviceToDevice,
                            h->stream));
    LIFT_CK(cudaMemcpyAsync(h->S.xbar, h->avg_x, Nk * sizeof(float2), cudaMemcpyDeviceToDevice,
                            h->stream));
    LIFT_CK(cudaMemcpyAsync(h->S.y, h->avg_y, Nk * sizeof(float4), cudaMemcpyDeviceToDevice,
                            h->stream));
    LIFT_CK(cudaMemcpyAsync(h->S.q, h->avg_q, h->N * sizeof(float), cudaMemcpyDeviceToDevice,
                            h->stream));
    if (h->S.pz)
        LIFT_CK(cudaMemcpyAsync(h->S.pz, h->avg_pz, Nk * sizeof(float),
                                cudaMemcpyDeviceToDevice, h->stream));
    h->prev_valid = false;
    h->avg_count = 0;
    return LIFT_OK;
}

int lift_unlift_average(lift_handle h, float *out, int on_host)
{
    if (!out) return LIFT_ERR_ARG;
    lift::LiftState Sa{};
    const int rc = average_state(h, &Sa);
    if (rc != LIFT_OK) return rc;
    if (!on_host) {
        LIFT_CK(lift::launch_unlift(h->P, Sa.x, out, h->stream));
        return LIFT_OK;
    }
    LIFT_CK(lift::launch_unlift(h->P, Sa.x, h->ubuf, h->stream));
    LIFT_CK(cudaMemcpyAsync(out, h->ubuf, h->N * sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    return LIFT_OK;
}

int lift_gap(lift_handle h, double *rel_gap)
{
    if (!h || !rel_gap || h->band) return LIFT_ERR_ARG;
    double p = 0.0, d = 0.0;
    const int rc = lift_energy(h, &p, &d, nullptr);
    if (rc != LIFT_OK) return rc;
    *rel_gap = (p - d) / std::max(std::max(fabs(p), fabs(d)), 1.0);
    return LIFT_OK;
}

int lift_solve(lift_handle h, int max_iters, double rel_gap_tol, int *iters_done)
{
    if (!h || max_iters < 0 || h->band) return LIFT_ERR_ARG;
    if (iters_done) *iters_done = 0;
    if (!(rel_gap_tol > 0.0)) {
        const int rc = lift_iterate(h, max_iters);
        if (rc == LIFT_OK && iters_done) *iters_done = max_iters;
        return rc;
    }
    int done = 0;
    while (done < max_iters) {
        if (h->adaptive) {
            const int rc = save_prev(h);
            if (rc != LIFT_OK) return rc;
        }
        const int chunk = std::min(h->check_every, max_iters - done);
        int rc = lift_iterate(h, chunk);
        if (rc != LIFT_OK) return rc;
        done += chunk;
        if (iters_done) *iters_done = done;
        double g = 0.0;
        rc = lift_gap(h, &g);
        if (rc != LIFT_OK) return rc;
        if (g <= rel_gap_tol) return LIFT_OK;
        if (h->adaptive) {
            rc = rebalance(h);
            if (rc != LIFT_OK) return rc;
        }
    }
    return LIFT_ERR_NOT_CONVERGED;
}

int lift_solve_averaged(lift_handle h, int max_iters, double rel_gap_tol, int first_epoch,
                        int every, int *iters_done, double *rel_gap)
{
    if (!h || h->band || max_iters < 0 || !(rel_gap_tol > 0.0) || every < 1 ||
        first_epoch < every)
        return LIFT_ERR_ARG;
    if (iters_done) *iters_done = 0;
    int done = 0;
    long long epoch = first_epoch;
    while (done < max_iters) {
        const int end = static_cast<int>(std::min<long long>(done + epoch, max_iters));
        int rc = lift_average(h, 0);
        if (rc != LIFT_OK) return rc;
        while (done < end) {
            const int step = std::min(every, end - done);
            rc = lift_iterate(h, step);
            if (rc != LIFT_OK) return rc;
            rc = lift_average(h, 1);
            if (rc != LIFT_OK) return rc;
            done += step;
        }
        if (iters_done) *iters_done = done;
        double gl = 0.0, pa = 0.0, da = 0.0;
        rc = lift_gap(h, &gl);
        if (rc != LIFT_OK) return rc;
        rc = lift_energy_average(h, &pa, &da, nullptr);
        if (rc != LIFT_OK) return rc;
        const double ga = (pa - da) / std::max(std::max(fabs(pa), fabs(da)), 1.0);
        if (ga < gl) {
            rc = lift_average_restart(h);     // the iterate becomes the better point
            if (rc != LIFT_OK) return rc;
        }
        const double g = std::min(ga, gl);
        if (rel_gap) *rel_gap = g;
        if (g <= rel_gap_tol) return LIFT_OK;
        epoch *= 2;
    }
    return LIFT_ERR_NOT_CONVERGED;
}

int lift_set_bands(lift_handle h, int bands, int *used)
{
    if (!h || bands < 0) return LIFT_ERR_ARG;
    if (bands != h->bands_req) {
        h->bands_req = bands;
        drop_iter_graph(h);
    }
    if (used) *used = bands_used(h);
    return LIFT_OK;
}

int lift_set_resident(lift_handle h, int enable, int *active)
{
    if (!h) return LIFT_ERR_ARG;
    h->resident_on = enable != 0;
    if (active) *active = h->resident.ok && h->resident_on ? 1 : 0;
    return LIFT_OK;
}

int lift_get_balance(lift_handle h, double *theta)
{
    if (!h || !theta) return LIFT_ERR_ARG;
    *theta = h->theta;
    return LIFT_OK;
}

int lift_unlift(lift_handle h, float *out, int on_host)
{
    if (!h || !out) return LIFT_ERR_ARG;
    // a band unlifts its own rows only
    LiftParams Pu = h->P;
    const float2 *x = h->S.x;
    if (h->band) {
        Pu.N = h->own1 - h->own0;
        x += static_cast<size_t>(h->own0) * h->k;
    }
    if (!on_host) {
        LIFT_CK(lift::launch_unlift(Pu, x, out, h->stream));
        return LIFT_OK;
    }
    LIFT_CK(lift::launch_unlift(Pu, x, h->ubuf, h->stream));
    LIFT_CK(cudaMemcpyAsync(out, h->ubuf, Pu.N * sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    return LIFT_OK;
}

size_t lift_state_bytes(lift_handle h)
{
    if (!h) return 0;
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    return Nk * (2 * sizeof(float2) + sizeof(float4)) + h->N * sizeof(float) +
           (h->S.pz ? Nk * sizeof(float) : 0);
}

static int copy_state(lift_handle h, char *hostdev, size_t bytes, int on_host, bool get)
{
    if (!h || !hostdev || bytes != lift_state_bytes(h)) return LIFT_ERR_ARG;
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    void *parts[5] = {h->S.x, h->S.xbar, h->S.y, h->S.q, h->S.pz};
    const size_t sizes[5] = {Nk * sizeof(float2), Nk * sizeof(float2), Nk * sizeof(float4),
                             h->N * sizeof(float), Nk * sizeof(float)};
    const int nparts = h->S.pz ? 5 : 4;
    cudaMemcpyKind kind = on_host ? (get ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice)
                                  : cudaMemcpyDeviceToDevice;
    size_t off = 0;
    for (int j = 0; j < nparts; ++j) {
        if (get)
            LIFT_CK(cudaMemcpyAsync(hostdev + off, parts[j], sizes[j], kind, h->stream));
        else
            LIFT_CK(cudaMemcpyAsync(parts[j], hostdev + off, sizes[j], kind, h->stream));
        off += sizes[j];
    }
    if (on_host) LIFT_CK(cudaStreamSynchronize(h->stream));
    return LIFT_OK;
}

int lift_get_state(lift_handle h, void *dst, size_t bytes, int on_host)
{
    return copy_state(h, static_cast<char *>(dst), bytes, on_host, true);
}

int lift_set_state(lift_handle h, const void *src, size_t bytes, int on_host)
{
    return copy_state(h, const_cast<char *>(static_cast<const char *>(src)), bytes, on_host, false);
}

int lift_proj_epi(lift_handle h, const int *pix, const int *interval, const float *y0,
                  const float *h0, float *y, float *hout, int n)
{
    if (!h || n < 0 || (n > 0 && (!pix || !interval || !y0 || !h0 || !y || !hout)))
        return LIFT_ERR_ARG;
    LIFT_CK(lift::launch_proj_epi(h->P, pix, interval, y0, h0, y, hout, n, h->stream));
    return LIFT_OK;
}

int lift_envelope(lift_handle h, const int *pix, const int *interval, const float *t,
                  float *out, int n)
{
    if (!h || n < 0 || (n > 0 && (!pix || !interval || !t || !out))) return LIFT_ERR_ARG;
    LIFT_CK(lift::launch_envelope(h->P, pix, interval, t, out, n, h->stream));
    return LIFT_OK;
}

const char *lift_cuda_error(void)
{
    return g_last_cuda_error == cudaSuccess ? "no error" : cudaGetErrorName(g_last_cuda_error);
}

const char *lift_strerror(int code)
{
    switch (code) {
    case LIFT_OK: return "ok";
    case LIFT_ERR_SPEC: return "invalid problem specification";
    case LIFT_ERR_OOM: return "device memory allocation failed";
    case LIFT_ERR_CUDA: return "CUDA error";
    case LIFT_ERR_NAN: return "non-finite energy (iterate diverged)";
    case LIFT_ERR_NOT_CONVERGED: return "gap tolerance not reached within max_iters";
    case LIFT_ERR_ARG: return "invalid argument";
    case LIFT_ERR_TIMEOUT: return "a kernel's bounded wait for its bulk copies gave up";
    default: return "unknown error code";
    }
}

}  // extern "C"

// ===========================================================================
// Batches: many problem instances solved together.  Instances too small to
// fill the GPU share one launch per half-step over all their tiles; an
// instance with at least `big_tiles` 256-thread tiles fills it alone and runs
// on the single-instance kernels (skipped through its live flag once
// converged).  Every check interval is captured in one CUDA graph.
// ===========================================================================
constexpr int kBatchStreams = 4;

struct lift_batch_ctx {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n = 0, kind = 0, check_every = 100, threads = lift::kStepThreads;
    int big_tiles = 0;                  // 0: every instance shares the merged launch
    int nfork = 4;                      // streams the big instances share in a captured interval
    int wave = 1;                       // 256-thread tiles resident on the whole GPU
    std::vector<LiftParams> P;          // host copies (device pointers filled in)
    std::vector<LiftState> S;
    std::vector<LiftParams> Pbig;       // single-kernel parameters of the big instances
    std::vector<int> big;               // indices of the big instances
    std::vector<int> ntiles;            // per instance, for the current tile width
    void *arena = nullptr;              // all per-instance device arrays
    lift::InstDesc *desc = nullptr;     // device [n]
    int *tile_inst = nullptr;           // device [total tiles]: instance of each tile
    int *strip_inst = nullptr;          // device: instance of each dual strip, group by group
    int total_tiles = 0, total_strips = 0;
    std::vector<lift::StripGroup> groups;   // the merged members' dual strips by CTA shape
    int *err = nullptr;                 // device: set by a kernel whose bounded wait gave up
    int *live = nullptr;                // device [n]: 1 = still iterating
    std::vector<int> live_h;
    std::vector<long long> iters_h;     // iterations done per instance
    double *partial = nullptr, *dout = nullptr, *hout = nullptr;
    float *ubuf = nullptr;              // unlift staging for host output
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_iters = 0;
    // the big instances of a captured interval run on these streams (forked
    // from and joined back into `stream`), several instances at once
    cudaStream_t fork_s[kBatchStreams] = {};
    cudaEvent_t fork_e[kBatchStreams + 1] = {};
};

namespace {

void drop_graph(lift_batch b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_iters = 0;
}

void free_batch(lift_batch b)
{
    if (!b) return;
    drop_graph(b);
    void *ptrs[] = {b->arena, b->desc, b->tile_inst, b->strip_inst, b->live,
                    b->partial, b->dout, b->ubuf, b->err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->hout) cudaFreeHost(b->hout);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    for (cudaStream_t st : b->fork_s)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->fork_e)
        if (ev) cudaEventDestroy(ev);
    delete b;
}

// (Re)build the tile list for a tile width of `threads` threads; instances
// with at least big_tiles tiles of kStepThreads threads (big_tiles > 0) leave
// the merged launch for the single-instance kernels.
int batch_set_tiles(lift_batch b, int threads, int big_tiles)
{
    std::vector<lift::InstDesc> d(b->n);
    std::vector<int> ti;
    int t0 = 0;
    b->big.clear();
    b->Pbig.clear();
    // merged members' dual strips, grouped by the CTA threads of their shape
    std::vector<int> gthreads;
    std::vector<std::vector<int>> gstrips;
    std::vector<int> gbytes;
    for (int j = 0; j < b->n; ++j) {
        LiftParams Ps = b->P[j];
        Ps.ppb = lift::kStepThreads / Ps.k;
        Ps.live = b->live + j;
        Ps.err = b->err;
        const int nt_single = (Ps.N + Ps.ppb - 1) / Ps.ppb;
        b->P[j].ppb = threads / b->P[j].k;
        const int nt = (b->P[j].N + b->P[j].ppb - 1) / b->P[j].ppb;
        d[j].P = b->P[j];
        d[j].S = b->S[j];
        if (big_tiles > 0 && nt_single >= big_tiles) {
            b->big.push_back(j);
            b->Pbig.push_back(Ps);
            b->ntiles[j] = 0;
            d[j].tile0 = d[j].ntiles = d[j].strip0 = d[j].nstrips = 0;
            continue;
        }
        b->ntiles[j] = nt;
        d[j].tile0 = t0;
        d[j].ntiles = nt;
        // dual strips of the shape a single problem of this k takes
        int sth = 0, sby = 0, spx = 0;
        lift::strip_shape_of(d[j].P.k, &sth, &sby, &spx);
        size_t g = 0;
        while (g < gthreads.size() && gthreads[g] != sth) ++g;
        if (g == gthreads.size()) {
            gthreads.push_back(sth);
            gstrips.emplace_back();
            gbytes.push_back(0);
        }
        gbytes[g] = std::max(gbytes[g], sby);
        d[j].strip0 = static_cast<int>(gstrips[g].size());
        d[j].nstrips = (d[j].P.N + spx - 1) / spx;
        gstrips[g].insert(gstrips[g].end(), d[j].nstrips, j);
        ti.insert(ti.end(), nt, j);
        t0 += nt;
    }
    std::vector<int> si;
    for (const auto &v : gstrips) si.insert(si.end(), v.begin(), v.end());
    const int ns = static_cast<int>(si.size());
    if (ti.empty()) ti.push_back(0);    // keep valid allocations; the totals stay 0
    if (si.empty()) si.push_back(0);
    if (b->tile_inst) cudaFree(b->tile_inst);
    if (b->strip_inst) cudaFree(b->strip_inst);
    b->tile_inst = b->strip_inst = nullptr;
    int rc = dev_alloc(reinterpret_cast<void **>(&b->tile_inst), ti.size() * sizeof(int));
    if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&b->strip_inst), si.size() * sizeof(int));
    if (rc != LIFT_OK) return rc;
    b->groups.clear();
    int off = 0;
    for (size_t g = 0; g < gthreads.size(); ++g) {
        lift::StripGroup G;
        G.threads = gthreads[g];
        G.bytes = gbytes[g];
        G.nstrips = static_cast<int>(gstrips[g].size());
        G.strip_inst = b->strip_inst + off;
        off += G.nstrips;
        b->groups.push_back(G);
    }
    LIFT_CK(cudaMemcpyAsync(b->tile_inst, ti.data(), ti.size() * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream));
    LIFT_CK(cudaMemcpyAsync(b->strip_inst, si.data(), si.size() * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream));
    LIFT_CK(cudaMemcpyAsync(b->desc, d.data(), d.size() * sizeof(lift::InstDesc),
                            cudaMemcpyHostToDevice, b->stream));
    LIFT_CK(cudaStreamSynchronize(b->stream));   // host vectors die here
    b->total_tiles = t0;
    b->total_strips = ns;
    b->threads = threads;
    b->big_tiles = big_tiles;
    drop_graph(b);
    return LIFT_OK;
}

int batch_launch(lift_batch b, int iters)
{
    for (int it = 0; it < iters; ++it) {
        LIFT_CK(lift::launch_batch_iteration(b->threads, b->desc, b->tile_inst, b->live,
                                             b->total_tiles, b->groups.data(),
                                             static_cast<int>(b->groups.size()), b->err, b->stream));
        for (size_t m = 0; m < b->big.size(); ++m) {
            const LiftState &S = b->S[b->big[m]];
            LIFT_CK(lift::launch_dual_step(b->Pbig[m], S, b->stream));
            LIFT_CK(lift::launch_primal_step(b->Pbig[m], S, b->stream));
        }
    }
    return LIFT_OK;
}

// In a captured interval the merged launches stay on the batch stream and
// the big instances, which share nothing, are spread over nfork (at most kBatchStreams)
// forked streams (all their iterations back to back), so that the dual steps
// of one instance run beside the primal steps of another.
int batch_launch_forked(lift_batch b, int iters)
{
    if (b->big.empty()) return batch_launch(b, iters);
    if (!b->fork_s[0]) {
        for (int j = 0; j < kBatchStreams; ++j)
            LIFT_CK(cudaStreamCreateWithFlags(&b->fork_s[j], cudaStreamNonBlocking));
        for (int j = 0; j <= kBatchStreams; ++j)
            LIFT_CK(cudaEventCreateWithFlags(&b->fork_e[j], cudaEventDisableTiming));
    }
    const int ns = std::min(std::max(1, std::min(b->nfork, kBatchStreams)),
                            static_cast<int>(b->big.size()));
    LIFT_CK(cudaEventRecord(b->fork_e[kBatchStreams], b->stream));
    for (int j = 0; j < ns; ++j) LIFT_CK(cudaStreamWaitEvent(b->fork_s[j], b->fork_e[kBatchStreams], 0));
    for (int it = 0; it < iters; ++it)
        LIFT_CK(lift::launch_batch_iteration(b->threads, b->desc, b->tile_inst, b->live,
                                             b->total_tiles, b->groups.data(),
                                             static_cast<int>(b->groups.size()), b->err, b->stream));
    for (size_t m = 0; m < b->big.size(); ++m) {
        cudaStream_t st = b->fork_s[m % ns];
        const LiftState &S = b->S[b->big[m]];
        for (int it = 0; it < iters; ++it) {
            LIFT_CK(lift::launch_dual_step(b->Pbig[m], S, st));
            LIFT_CK(lift::launch_primal_step(b->Pbig[m], S, st));
        }
    }
    for (int j = 0; j < ns; ++j) {
        LIFT_CK(cudaEventRecord(b->fork_e[j], b->fork_s[j]));
        LIFT_CK(cudaStreamWaitEvent(b->stream, b->fork_e[j], 0));
    }
    return LIFT_OK;
}

int batch_capture(lift_batch b, int iters)
{
    drop_graph(b);
    LIFT_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = batch_launch_forked(b, iters);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != LIFT_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return LIFT_ERR_CUDA;
    }
    b->graph = g;
    LIFT_CK(cudaGraphInstantiate(&b->exec, g, 0));
    b->graph_iters = iters;
    return LIFT_OK;
}

}  // namespace

extern "C" {

int lift_create_batch(const lift_spec *specs, int n, void *stream, lift_batch *out)
{
    if (!specs || !out || n < 1) return LIFT_ERR_ARG;
    *out = nullptr;
    for (int j = 0; j < n; ++j) {
        const int rc = validate(&specs[j]);
        if (rc != LIFT_OK) return rc;
        if (specs[j].kind == LIFT_PL_SAMPLED || specs[j].kind != specs[0].kind) return LIFT_ERR_SPEC;
        if (specs[j].D > 1) return LIFT_ERR_SPEC;      // images only
    }
    lift_batch b = new (std::nothrow) lift_batch_ctx();
    if (!b) return LIFT_ERR_OOM;
    b->n = n;
    b->kind = specs[0].kind;
    b->check_every = specs[0].check_every > 0 ? specs[0].check_every : 100;
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        // graph capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return LIFT_ERR_CUDA;
        }
        b->own_stream = true;
    }
    b->P.resize(n);
    b->S.resize(n);
    b->ntiles.assign(n, 0);
    b->live_h.assign(n, 1);
    b->iters_h.assign(n, 0);

    // one arena: per instance x, xbar, y, q, f, icst (256-byte aligned)
    std::vector<std::vector<float4>> ics(n);
    std::vector<size_t> off(n * 7);
    std::vector<float4> st(n);
    size_t total = 0;
    auto take = [&](size_t bytes) { const size_t o = total; total += (bytes + 255) & ~size_t(255); return o; };
    int max_eblocks = 1;
    size_t max_n = 1;
    for (int j = 0; j < n; ++j) {
        make_params(&specs[j], lift::kStepThreads, b->P[j], ics[j]);
        const size_t N = static_cast<size_t>(b->P[j].N), Nk = N * b->P[j].k;
        off[7 * j + 0] = take(Nk * sizeof(float2));
        off[7 * j + 1] = take(Nk * sizeof(float2));
        off[7 * j + 2] = take(Nk * sizeof(float4));
        off[7 * j + 3] = take(N * sizeof(float));
        off[7 * j + 4] = take(N * sizeof(float));
        off[7 * j + 5] = take(b->P[j].k * sizeof(float4));
        off[7 * j + 6] = take(sizeof(float4));
        st[j] = step_scalars(b->P[j]);
        max_eblocks = std::max(max_eblocks, lift::energy_blocks(b->P[j]));
        max_n = std::max(max_n, N);
    }
    int rc = dev_alloc(&b->arena, total);
    if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&b->desc), n * sizeof(lift::InstDesc));
    if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&b->live), n * sizeof(int));
    if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&b->partial), 3 * sizeof(double) * max_eblocks);
    if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&b->dout), 3 * sizeof(double) * n);
    if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&b->ubuf), max_n * sizeof(float));
    if (rc == LIFT_OK) rc = dev_alloc(reinterpret_cast<void **>(&b->err), sizeof(int));
    if (rc == LIFT_OK && cudaMemsetAsync(b->err, 0, sizeof(int), b->stream) != cudaSuccess)
        rc = LIFT_ERR_CUDA;
    if (rc == LIFT_OK && cudaMallocHost(reinterpret_cast<void **>(&b->hout), 3 * sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        b->hout = nullptr;
        rc = LIFT_ERR_OOM;
    }
    if (rc != LIFT_OK) { free_batch(b); return rc; }
    char *base = static_cast<char *>(b->arena);
    for (int j = 0; j < n; ++j) {
        LiftState &S = b->S[j];
        S.x = reinterpret_cast<float2 *>(base + off[7 * j + 0]);
        S.xbar = reinterpret_cast<float2 *>(base + off[7 * j + 1]);
        S.y = reinterpret_cast<float4 *>(base + off[7 * j + 2]);
        S.q = reinterpret_cast<float *>(base + off[7 * j + 3]);
        float *f = reinterpret_cast<float *>(base + off[7 * j + 4]);
        float4 *ic = reinterpret_cast<float4 *>(base + off[7 * j + 5]);
        b->P[j].f = f;
        b->P[j].icst = ic;
        b->P[j].steps = reinterpret_cast<float4 *>(base + off[7 * j + 6]);
        const size_t N = static_cast<size_t>(b->P[j].N);
        if (cudaMemcpyAsync(f, specs[j].f, N * sizeof(float),
                            specs[j].data_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            b->stream) != cudaSuccess ||
            cudaMemcpyAsync(ic, ics[j].data(), ics[j].size() * sizeof(float4),
                            cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
            cudaMemcpyAsync(base + off[7 * j + 6], &st[j], sizeof(float4), cudaMemcpyHostToDevice,
                            b->stream) != cudaSuccess) {
            free_batch(b);
            return LIFT_ERR_CUDA;
        }
    }
    {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        b->wave = std::max(1, sms * (2048 / lift::kStepThreads));
    }
    rc = batch_set_tiles(b, lift::kStepThreads, 2 * b->wave);   // synchronises (ics die here)
    if (rc == LIFT_OK) rc = lift_batch_reset(b);
    if (rc != LIFT_OK) { free_batch(b); return rc; }
    *out = b;
    return LIFT_OK;
}

void lift_batch_destroy(lift_batch b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
}

int lift_batch_size(lift_batch b)
{
    return b ? b->n : 0;
}

int lift_batch_reset(lift_batch b)
{
    if (!b) return LIFT_ERR_ARG;
    for (int j = 0; j < b->n; ++j) {
        const size_t N = static_cast<size_t>(b->P[j].N), Nk = N * b->P[j].k;
        LIFT_CK(cudaMemsetAsync(b->S[j].x, 0, Nk * sizeof(float2), b->stream));
        LIFT_CK(cudaMemsetAsync(b->S[j].xbar, 0, Nk * sizeof(float2), b->stream));
        LIFT_CK(cudaMemsetAsync(b->S[j].y, 0, Nk * sizeof(float4), b->stream));
        LIFT_CK(cudaMemsetAsync(b->S[j].q, 0, N * sizeof(float), b->stream));
    }
    b->live_h.assign(b->n, 1);
    b->iters_h.assign(b->n, 0);
    LIFT_CK(cudaMemcpyAsync(b->live, b->live_h.data(), b->n * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream));
    LIFT_CK(cudaStreamSynchronize(b->stream));
    return LIFT_OK;
}

int lift_batch_iterate(lift_batch b, int iters)
{
    if (!b || iters < 0) return LIFT_ERR_ARG;
    int done = 0;
    while (iters - done >= b->check_every) {
        if (!b->exec || b->graph_iters != b->check_every) {
            const int rc = batch_capture(b, b->check_every);
            if (rc != LIFT_OK) return rc;
        }
        LIFT_CK(cudaGraphLaunch(b->exec, b->stream));
        done += b->check_every;
    }
    const int rc = batch_launch(b, iters - done);
    if (rc != LIFT_OK) return rc;
    for (int j = 0; j < b->n; ++j)
        if (b->live_h[j]) b->iters_h[j] += iters;
    return LIFT_OK;
}

int lift_batch_energy(lift_batch b, double *out)
{
    if (!b || !out) return LIFT_ERR_ARG;
    for (int j = 0; j < b->n; ++j)
        LIFT_CK(lift::launch_energy(b->P[j], b->S[j], b->partial, b->dout + 3 * j, b->stream));
    LIFT_CK(cudaMemcpyAsync(b->hout, b->dout, 3 * sizeof(double) * b->n, cudaMemcpyDeviceToHost,
                            b->stream));
    int err_word = 0;
    LIFT_CK(cudaMemcpyAsync(&err_word, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    LIFT_CK(cudaStreamSynchronize(b->stream));
    if (err_word != 0) return LIFT_ERR_TIMEOUT;
    memcpy(out, b->hout, 3 * sizeof(double) * b->n);
    for (int j = 0; j < 3 * b->n; ++j)
        if (!is_finite(out[j])) return LIFT_ERR_NAN;
    return LIFT_OK;
}

int lift_batch_solve(lift_batch b, int max_iters, double rel_gap_tol, int *iters_done,
                     int *n_converged)
{
    if (!b || max_iters < 0) return LIFT_ERR_ARG;
    std::vector<double> e(3 * b->n);
    int conv = 0;
    long long done = 0;
    while (done < max_iters) {
        const int chunk = static_cast<int>(std::min<long long>(b->check_every, max_iters - done));
        int rc = lift_batch_iterate(b, chunk);
        if (rc != LIFT_OK) return rc;
        done += chunk;
        rc = lift_batch_energy(b, e.data());
        if (rc != LIFT_OK) return rc;
        conv = 0;
        bool changed = false;
        for (int j = 0; j < b->n; ++j) {
            const double p = e[3 * j], d = e[3 * j + 1];
            const double g = (p - d) / std::max(std::max(fabs(p), fabs(d)), 1.0);
            if (b->live_h[j] && g <= rel_gap_tol) { b->live_h[j] = 0; changed = true; }
            conv += b->live_h[j] ? 0 : 1;
        }
        if (changed)
            LIFT_CK(cudaMemcpyAsync(b->live, b->live_h.data(), b->n * sizeof(int),
                                    cudaMemcpyHostToDevice, b->stream));
        if (conv == b->n) break;
    }
    if (iters_done)
        for (int j = 0; j < b->n; ++j) iters_done[j] = static_cast<int>(b->iters_h[j]);
    if (n_converged) *n_converged = conv;
    return conv == b->n ? LIFT_OK : LIFT_ERR_NOT_CONVERGED;
}

int lift_batch_unlift(lift_batch b, int i, float *out, int on_host)
{
    if (!b || !out || i < 0 || i >= b->n) return LIFT_ERR_ARG;
    const size_t N = static_cast<size_t>(b->P[i].N);
    if (!on_host) {
        LIFT_CK(lift::launch_unlift(b->P[i], b->S[i].x, out, b->stream));
        return LIFT_OK;
    }
    LIFT_CK(lift::launch_unlift(b->P[i], b->S[i].x, b->ubuf, b->stream));
    LIFT_CK(cudaMemcpyAsync(out, b->ubuf, N * sizeof(float), cudaMemcpyDeviceToHost, b->stream));
    LIFT_CK(cudaStreamSynchronize(b->stream));
    return LIFT_OK;
}

int lift_batch_get_state(lift_batch b, int i, void *dst, size_t bytes, int on_host)
{
    if (!b || !dst || i < 0 || i >= b->n) return LIFT_ERR_ARG;
    const size_t N = static_cast<size_t>(b->P[i].N), Nk = N * b->P[i].k;
    const size_t sizes[4] = {Nk * sizeof(float2), Nk * sizeof(float2), Nk * sizeof(float4),
                             N * sizeof(float)};
    if (bytes != sizes[0] + sizes[1] + sizes[2] + sizes[3]) return LIFT_ERR_ARG;
    const void *parts[4] = {b->S[i].x, b->S[i].xbar, b->S[i].y, b->S[i].q};
    size_t o = 0;
    for (int j = 0; j < 4; ++j) {
        LIFT_CK(cudaMemcpyAsync(static_cast<char *>(dst) + o, parts[j], sizes[j],
                                on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                b->stream));
        o += sizes[j];
    }
    if (on_host) LIFT_CK(cudaStreamSynchronize(b->stream));
    return LIFT_OK;
}

int lift_batch_autotune(lift_batch b, int iters, int *threads_chosen)
{
    if (!b || iters < 1) return LIFT_ERR_ARG;
    const int cand[3] = {128, 256, 512};
    // big-instance thresholds: none (all merged), 1, 2 and 4 full waves of
    // 256-thread tiles; the big instances on 1, 2 or 4 streams at once
    const int thr[4] = {0, b->wave, 2 * b->wave, 4 * b->wave};
    const int forks[3] = {1, 2, 4};
    float best_ms = 0.0f;
    int best = lift::kStepThreads, best_big = b->big_tiles, best_fork = b->nfork;
    cudaEvent_t e0, e1;
    LIFT_CK(cudaEventCreate(&e0));
    LIFT_CK(cudaEventCreate(&e1));
    int rc = LIFT_OK;
    for (int t = 0; t < 4 && rc == LIFT_OK; ++t) {
        for (int c = 0; c < 3 && rc == LIFT_OK; ++c) {
            rc = batch_set_tiles(b, cand[c], thr[t]);
            if (rc != LIFT_OK) break;
            // every instance left in the merged launch needs a tile of >= k threads
            bool ok = true;
            for (int j = 0; j < b->n; ++j) ok = ok && (b->ntiles[j] == 0 || cand[c] >= b->P[j].k);
            if (!ok) continue;
            for (int fk = 0; fk < 3 && rc == LIFT_OK; ++fk) {
                if (forks[fk] > 1 && static_cast<int>(b->big.size()) < forks[fk]) continue;
                b->nfork = forks[fk];
                // time the captured interval that a solve would replay
                rc = lift_batch_reset(b);
                if (rc == LIFT_OK) rc = batch_capture(b, iters);
                if (rc != LIFT_OK) break;
                LIFT_CK(cudaGraphLaunch(b->exec, b->stream));           // warm-up
                cudaEventRecord(e0, b->stream);
                LIFT_CK(cudaGraphLaunch(b->exec, b->stream));
                cudaEventRecord(e1, b->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = LIFT_ERR_CUDA; break; }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (best_ms == 0.0f || ms < best_ms) {
                    best_ms = ms;
                    best = cand[c];
                    best_big = thr[t];
                    best_fork = forks[fk];
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LIFT_OK) return rc;
    b->nfork = best_fork;
    rc = batch_set_tiles(b, best, best_big);            // drops the last captured graph
    if (rc == LIFT_OK) rc = lift_batch_reset(b);
    if (rc == LIFT_OK && threads_chosen) *threads_chosen = best;
    return rc;
}

int lift_batch_set_schedule(lift_batch b, int threads, int big_tiles)
{
    if (!b || big_tiles < 0 || (threads != 128 && threads != 256 && threads != 512))
        return LIFT_ERR_ARG;
    const int old_threads = b->threads, old_big = b->big_tiles;
    int rc = batch_set_tiles(b, threads, big_tiles);
    if (rc != LIFT_OK) return rc;
    for (int j = 0; j < b->n; ++j)
        if (b->ntiles[j] > 0 && threads < b->P[j].k) {
            // a merged instance needs a tile of >= k threads: keep the old schedule
            rc = batch_set_tiles(b, old_threads, old_big);
            return rc != LIFT_OK ? rc : LIFT_ERR_ARG;
        }
    return LIFT_OK;
}

int lift_batch_streams(lift_batch b, int set, int *n)
{
    if (!b || set < 0 || set > kBatchStreams) return LIFT_ERR_ARG;
    if (set > 0 && set != b->nfork) {
        b->nfork = set;
        drop_graph(b);
    }
    if (n) *n = b->nfork;
    return LIFT_OK;
}

int lift_batch_schedule(lift_batch b, int *threads, int *big_tiles, int *n_big)
{
    if (!b) return LIFT_ERR_ARG;
    if (threads) *threads = b->threads;
    if (big_tiles) *big_tiles = b->big_tiles;
    if (n_big) *n_big = static_cast<int>(b->big.size());
    return LIFT_OK;
}

}  // extern "C"

// ===========================================================================
// Differentiable unrolled solve (adjoint.cu): checkpointed forward, reverse
// sweep with per-segment recomputation.
// ===========================================================================
namespace {

// Distance between consecutive stored states: the state image rounded up to
// 256 bytes, so that every stored state starts aligned for the float2 /
// float4 records (the image itself ends with N floats).
size_t state_stride(lift_handle h)
{
    return (lift_state_bytes(h) + 255) & ~static_cast<size_t>(255);
}

LiftState state_at(const lift_ctx *h, char *base)
{
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    LiftState S;
    S.x = reinterpret_cast<float2 *>(base);
    S.xbar = reinterpret_cast<float2 *>(base + Nk * sizeof(float2));
    S.y = reinterpret_cast<float4 *>(base + 2 * Nk * sizeof(float2));
    S.q = reinterpret_cast<float *>(base + 2 * Nk * sizeof(float2) + Nk * sizeof(float4));
    return S;
}

int copy_state_dev(lift_handle h, const LiftState &dst, const LiftState &src)
{
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    LIFT_CK(cudaMemcpyAsync(dst.x, src.x, Nk * sizeof(float2), cudaMemcpyDeviceToDevice, h->stream));
    LIFT_CK(cudaMemcpyAsync(dst.xbar, src.xbar, Nk * sizeof(float2), cudaMemcpyDeviceToDevice, h->stream));
    LIFT_CK(cudaMemcpyAsync(dst.y, src.y, Nk * sizeof(float4), cudaMemcpyDeviceToDevice, h->stream));
    LIFT_CK(cudaMemcpyAsync(dst.q, src.q, h->N * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    return LIFT_OK;
}

int iterate_state(lift_handle h, const LiftState &S, int iters)
{
    for (int n = 0; n < iters; ++n) {
        LIFT_CK(lift::launch_dual_step(h->P, S, h->stream));
        LIFT_CK(lift::launch_primal_step(h->P, S, h->stream));
    }
    return LIFT_OK;
}

}  // namespace

extern "C" {

int lift_set_params(lift_handle h, double lambda, double alpha, double nu)
{
    if (!h) return LIFT_ERR_ARG;
    if (!is_finite(lambda) || lambda < 0.0) return LIFT_ERR_SPEC;
    if (h->kind != LIFT_PL_SAMPLED) {
        if (!is_finite(alpha) || !(alpha > 0.0)) return LIFT_ERR_SPEC;
        if (h->kind != LIFT_QUAD && (!is_finite(nu) || !(nu > 0.0))) return LIFT_ERR_SPEC;
    }
    invalidate_unrolled(h);
    std::vector<float4> ic(h->k);
    LIFT_CK(cudaMemcpyAsync(ic.data(), h->icst, h->k * sizeof(float4), cudaMemcpyDeviceToHost, h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < h->k; ++i) ic[i].w = static_cast<float>(lambda * h->P.delta);
    LIFT_CK(cudaMemcpyAsync(h->icst, ic.data(), h->k * sizeof(float4), cudaMemcpyHostToDevice, h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    drop_iter_graph(h);
    h->P.lam = static_cast<float>(lambda);
    if (h->kind != LIFT_PL_SAMPLED) {
        h->P.alpha = static_cast<float>(alpha);
        h->P.inv_alpha = static_cast<float>(1.0 / alpha);
        h->P.nu = static_cast<float>(nu);
        h->P.wtrunc = h->kind == LIFT_TRUNC_QUAD ? static_cast<float>(sqrt(nu / alpha)) : 0.0f;
    }
    return LIFT_OK;
}

int lift_unrolled_forward(lift_handle h, int iters, int checkpoint_every)
{
    if (!h || iters < 1 || checkpoint_every < 1 || h->band) return LIFT_ERR_ARG;
    if (h->kind == LIFT_PL_SAMPLED || h->P.D > 1) return LIFT_ERR_SPEC;
    const size_t sb = state_stride(h);
    const int nck = (iters + checkpoint_every - 1) / checkpoint_every;
    if (nck > h->ckpt_count) {
        if (h->ckpt) cudaFree(h->ckpt);
        h->ckpt = nullptr;
        h->ckpt_count = 0;
        const int rc = dev_alloc(reinterpret_cast<void **>(&h->ckpt), sb * nck);
        if (rc != LIFT_OK) return rc;
        h->ckpt_count = nck;
    }
    int rc = lift_reset(h);
    if (rc != LIFT_OK) return rc;
    for (int c = 0; c < nck; ++c) {
        rc = copy_state_dev(h, state_at(h, h->ckpt + sb * c), h->S);
        if (rc != LIFT_OK) return rc;
        const int len = std::min(checkpoint_every, iters - c * checkpoint_every);
        rc = iterate_state(h, h->S, len);
        if (rc != LIFT_OK) return rc;
    }
    h->unrolled_iters = iters;
    h->ckpt_every = checkpoint_every;
    ++h->generation;
    return LIFT_OK;
}

int lift_unrolled_generation(lift_handle h, unsigned long long *generation)
{
    if (!h || !generation) return LIFT_ERR_ARG;
    *generation = h->generation;
    return LIFT_OK;
}

int lift_unrolled_backward(lift_handle h, const float *grad_u, float *grad_f, double *grad_scalars)
{
    if (!h || !grad_u) return LIFT_ERR_ARG;
    if (h->unrolled_iters < 1) return LIFT_ERR_ARG;
    const size_t sb = state_stride(h);
    const size_t N = static_cast<size_t>(h->N), Nk = N * h->k;
    const int C = h->ckpt_every;
    if (C + 1 > h->seg_cap) {
        if (h->seg) cudaFree(h->seg);
        h->seg = nullptr;
        h->seg_cap = 0;
        const int rc = dev_alloc(reinterpret_cast<void **>(&h->seg), sb * (C + 1));
        if (rc != LIFT_OK) return rc;
        h->seg_cap = C + 1;
    }
    if (!h->adj_arena) {
        const int nb = lift::adjoint_blocks(h->P);
        size_t total = 0;
        auto take = [&](size_t bytes) { const size_t o = total; total += (bytes + 255) & ~size_t(255); return o; };
        const size_t o_ax = take(Nk * sizeof(float2)), o_axb = take(Nk * sizeof(float2));
        const size_t o_ay = take(Nk * sizeof(float4)), o_aq = take(N * sizeof(float));
        const size_t o_G = take(Nk * sizeof(float2)), o_A = take(Nk * sizeof(float2));
        const size_t o_gf = take(N * sizeof(float)), o_p = take(3 * sizeof(double) * nb);
        const size_t o_acc = take(3 * sizeof(double));
        const int rc = dev_alloc(&h->adj_arena, total);
        if (rc != LIFT_OK) return rc;
        char *b = static_cast<char *>(h->adj_arena);
        h->adj.ax = reinterpret_cast<float2 *>(b + o_ax);
        h->adj.axb = reinterpret_cast<float2 *>(b + o_axb);
        h->adj.ay = reinterpret_cast<float4 *>(b + o_ay);
        h->adj.aq = reinterpret_cast<float *>(b + o_aq);
        h->adj.G = reinterpret_cast<float2 *>(b + o_G);
        h->adj.A = reinterpret_cast<float2 *>(b + o_A);
        h->adj.gf = reinterpret_cast<float *>(b + o_gf);
        h->adj.partial = reinterpret_cast<double *>(b + o_p);
        h->adj.acc = reinterpret_cast<double *>(b + o_acc);
    }
    const lift::AdjState &A = h->adj;
    LIFT_CK(lift::launch_adj_seed(h->P, grad_u, A.ax, h->stream));
    LIFT_CK(cudaMemsetAsync(A.axb, 0, Nk * sizeof(float2), h->stream));
    LIFT_CK(cudaMemsetAsync(A.ay, 0, Nk * sizeof(float4), h->stream));
    LIFT_CK(cudaMemsetAsync(A.aq, 0, N * sizeof(float), h->stream));
    LIFT_CK(cudaMemsetAsync(A.gf, 0, N * sizeof(float), h->stream));
    LIFT_CK(cudaMemsetAsync(A.A, 0, Nk * sizeof(float2), h->stream));
    LIFT_CK(cudaMemsetAsync(A.acc, 0, 3 * sizeof(double), h->stream));
    LIFT_CK(cudaMemsetAsync(A.partial, 0, 3 * sizeof(double) * lift::adjoint_blocks(h->P),
                            h->stream));
    const int nck = (h->unrolled_iters + C - 1) / C;
    for (int c = nck - 1; c >= 0; --c) {
        const int len = std::min(C, h->unrolled_iters - c * C);
        // recompute the segment's states from its checkpoint: state 0 is the
        // checkpoint itself, state j + 1 is written by one iteration from
        // state j (no copy; the checkpoint is only read)
        auto seg_state = [&](int j) {
            return state_at(h, j == 0 ? h->ckpt + sb * c : h->seg + sb * j);
        };
        for (int j = 0; j < len; ++j)
            LIFT_CK(lift::launch_iteration_into(h->P, seg_state(j), seg_state(j + 1), h->stream));
        for (int j = len - 1; j >= 0; --j)
            LIFT_CK(lift::launch_adj_iteration(h->P, seg_state(j), seg_state(j + 1), A, h->stream));
    }
    LIFT_CK(lift::launch_adj_finish(h->P, A, h->stream));
    if (grad_f)
        LIFT_CK(cudaMemcpyAsync(grad_f, A.gf, N * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    if (grad_scalars) {
        LIFT_CK(cudaMemcpyAsync(h->hout, A.acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        LIFT_CK(cudaStreamSynchronize(h->stream));
        memcpy(grad_scalars, h->hout, 3 * sizeof(double));
    }
    return LIFT_OK;
}

}  // extern "C"
