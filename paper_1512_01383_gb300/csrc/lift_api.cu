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

struct lift_ctx {
    cudaStream_t stream = nullptr;
    int kind = 0;
    int H = 0, W = 0, k = 0, N = 0;
    int check_every = 100;
    LiftParams P{};
    LiftState S{};
    float4 *icst = nullptr;
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
};

namespace {

#define LIFT_CK(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return LIFT_ERR_CUDA;   \
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
    void *ptrs[] = {h->S.x, h->S.xbar, h->S.y, h->S.q, h->icst, h->f, h->cost, h->rhat,
                    h->bpos, h->bstart, h->ubuf, h->partial, h->dout};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->hout) cudaFreeHost(h->hout);
    delete h;
}

bool is_finite(double x) { return std::isfinite(x); }

int validate(const lift_spec *s)
{
    if (s->kind < LIFT_QUAD || s->kind > LIFT_PL_SAMPLED) return LIFT_ERR_SPEC;
    if (s->H < 1 || s->W < 1) return LIFT_ERR_SPEC;
    if (s->L < 2 || s->L > LIFT_MAX_K + 1) return LIFT_ERR_SPEC;
    const long long N = static_cast<long long>(s->H) * s->W;
    if (N * (s->L - 1) > (1LL << 31) - 1) return LIFT_ERR_SPEC;
    if (!is_finite(s->gamma_min) || !is_finite(s->gamma_max) || !(s->gamma_max > s->gamma_min))
        return LIFT_ERR_SPEC;
    if (!is_finite(s->lambda) || s->lambda < 0.0) return LIFT_ERR_SPEC;
    if (!is_finite(s->step_balance)) return LIFT_ERR_SPEC;
    if (s->kind == LIFT_QUAD || s->kind == LIFT_TRUNC_QUAD) {
        if (!s->f) return LIFT_ERR_SPEC;
        if (!is_finite(s->alpha) || !(s->alpha > 0.0)) return LIFT_ERR_SPEC;
        if (s->kind == LIFT_TRUNC_QUAD && (!is_finite(s->nu) || !(s->nu > 0.0))) return LIFT_ERR_SPEC;
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

int upload_data(lift_handle h, const float *data, int on_host)
{
    float *dst = h->kind == LIFT_PL_SAMPLED ? h->cost : h->f;
    LIFT_CK(cudaMemcpyAsync(dst, data, h->data_elems * sizeof(float),
                            on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            h->stream));
    if (h->kind == LIFT_PL_SAMPLED) LIFT_CK(lift::launch_pl_setup(h->P, h->rhat, h->stream));
    return LIFT_OK;
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
    h->N = spec->H * spec->W;
    h->check_every = spec->check_every > 0 ? spec->check_every : 100;
    const int k = h->k;
    const size_t N = static_cast<size_t>(h->N), Nk = N * k;

    // step sizes: reciprocal absolute row / column sums of the operator
    const double d = label(spec, 1) - label(spec, 0);
    const double gL = label(spec, k);
    // primal/dual balance theta: primal steps x theta, dual steps / theta
    const double th = spec->step_balance > 0.0 ? spec->step_balance : 1.0;
    std::vector<float4> ic(k);
    for (int i = 0; i < k; ++i) {
        const double gi = label(spec, i);
        const double tau_s = th / (1.0 + fabs(gi) + (i + 1) * d);
        const double row_v = 1.0 + fabs(gi) + (gL - label(spec, i + 1));
        const double sig = 1.0 / (th * std::max(row_v, 1.0));
        ic[i] = make_float4(static_cast<float>(gi), static_cast<float>(tau_s),
                            static_cast<float>(sig), static_cast<float>(spec->lambda * d));
    }

    LiftParams &P = h->P;
    P.H = h->H; P.W = h->W; P.k = k; P.N = h->N;
    P.kind = spec->kind;
    P.ppb = lift::kStepThreads / k;

    P.inv_k = 1.0f / static_cast<float>(k);
    P.delta = static_cast<float>(d);
    P.inv_delta = static_cast<float>(1.0 / d);
    {
        // exact division by W for 0 <= pix < 2^31: with l = ceil(log2 W) and
        // M = floor(2^(31+l) / W) + 1, floor(pix*M / 2^(31+l)) = floor(pix/W)
        // because the excess pix*(M - 2^(31+l)/W)/2^(31+l) < 2^-l <= 1/W
        int l = 0;
        while ((1LL << l) < h->W) ++l;
        P.wshift = 31 + l;
        P.wmul = ((1ULL << P.wshift) / static_cast<unsigned long long>(h->W)) + 1ULL;
    }
    P.gmin = static_cast<float>(spec->gamma_min);
    P.lam = static_cast<float>(spec->lambda);
    P.alpha = static_cast<float>(spec->alpha);
    P.nu = static_cast<float>(spec->nu);
    P.wtrunc = spec->kind == LIFT_TRUNC_QUAD ? static_cast<float>(sqrt(spec->nu / spec->alpha)) : 0.0f;
    P.tau_u = static_cast<float>(0.2 * th);
    P.sigma_q = static_cast<float>(1.0 / (th * (gL - label(spec, 0))));
    P.sigma_p = static_cast<float>(0.5 / th);

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
    ALLOC(h->icst, k * sizeof(float4));
    ALLOC(h->ubuf, N * sizeof(float));
    ALLOC(h->partial, 3 * sizeof(double) * lift::energy_blocks(P));
    ALLOC(h->dout, 3 * sizeof(double));
    if (cudaMallocHost(reinterpret_cast<void **>(&h->hout), 3 * sizeof(double)) != cudaSuccess) {
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
    P.icst = h->icst;
    P.f = h->f;
    P.rhat = h->rhat;
    P.cost = h->cost;
    P.bpos = h->bpos;
    P.bstart = h->bstart;

    CUDA_OR_FAIL(cudaMemcpyAsync(h->icst, ic.data(), k * sizeof(float4), cudaMemcpyHostToDevice,
                                 h->stream));
    const float *data = spec->kind == LIFT_PL_SAMPLED ? spec->cost : spec->f;
    rc = upload_data(h, data, spec->data_on_host);
    if (rc != LIFT_OK) { free_ctx(h); return rc; }
    rc = lift_reset(h);
    if (rc != LIFT_OK) { free_ctx(h); return rc; }
    // host-side vectors die with this scope: finish the uploads first
    CUDA_OR_FAIL(cudaStreamSynchronize(h->stream));
#undef CUDA_OR_FAIL
    *out = h;
    return LIFT_OK;
}

void lift_destroy(lift_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_ctx(h);
}

int lift_set_data(lift_handle h, const float *data, int on_host)
{
    if (!h || !data) return LIFT_ERR_ARG;
    return upload_data(h, data, on_host);
}

int lift_reset(lift_handle h)
{
    if (!h) return LIFT_ERR_ARG;
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    LIFT_CK(cudaMemsetAsync(h->S.x, 0, Nk * sizeof(float2), h->stream));
    LIFT_CK(cudaMemsetAsync(h->S.xbar, 0, Nk * sizeof(float2), h->stream));
    LIFT_CK(cudaMemsetAsync(h->S.y, 0, Nk * sizeof(float4), h->stream));
    LIFT_CK(cudaMemsetAsync(h->S.q, 0, h->N * sizeof(float), h->stream));
    return LIFT_OK;
}

int lift_iterate(lift_handle h, int iters)
{
    if (!h || iters < 0) return LIFT_ERR_ARG;
    for (int n = 0; n < iters; ++n) {
        LIFT_CK(lift::launch_dual_step(h->P, h->S, h->stream));
        LIFT_CK(lift::launch_primal_step(h->P, h->S, h->stream));
    }
    return LIFT_OK;
}

int lift_dual_step(lift_handle h)
{
    if (!h) return LIFT_ERR_ARG;
    LIFT_CK(lift::launch_dual_step(h->P, h->S, h->stream));
    return LIFT_OK;
}

int lift_primal_step(lift_handle h)
{
    if (!h) return LIFT_ERR_ARG;
    LIFT_CK(lift::launch_primal_step(h->P, h->S, h->stream));
    return LIFT_OK;
}

int lift_energy(lift_handle h, double *primal_relaxed, double *dual, double *e_nonconvex)
{
    if (!h) return LIFT_ERR_ARG;
    LIFT_CK(lift::launch_energy(h->P, h->S, h->partial, h->dout, h->stream));
    LIFT_CK(cudaMemcpyAsync(h->hout, h->dout, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    if (primal_relaxed) *primal_relaxed = h->hout[0];
    if (dual) *dual = h->hout[1];
    if (e_nonconvex) *e_nonconvex = h->hout[2];
    if (!is_finite(h->hout[0]) || !is_finite(h->hout[1]) || !is_finite(h->hout[2])) return LIFT_ERR_NAN;
    return LIFT_OK;
}

int lift_gap(lift_handle h, double *rel_gap)
{
    if (!h || !rel_gap) return LIFT_ERR_ARG;
    double p = 0.0, d = 0.0;
    const int rc = lift_energy(h, &p, &d, nullptr);
    if (rc != LIFT_OK) return rc;
    *rel_gap = (p - d) / std::max(std::max(fabs(p), fabs(d)), 1.0);
    return LIFT_OK;
}

int lift_solve(lift_handle h, int max_iters, double rel_gap_tol, int *iters_done)
{
    if (!h || max_iters < 0) return LIFT_ERR_ARG;
    if (iters_done) *iters_done = 0;
    if (!(rel_gap_tol > 0.0)) {
        const int rc = lift_iterate(h, max_iters);
        if (rc == LIFT_OK && iters_done) *iters_done = max_iters;
        return rc;
    }
    int done = 0;
    while (done < max_iters) {
        const int chunk = std::min(h->check_every, max_iters - done);
        int rc = lift_iterate(h, chunk);
        if (rc != LIFT_OK) return rc;
        done += chunk;
        if (iters_done) *iters_done = done;
        double g = 0.0;
        rc = lift_gap(h, &g);
        if (rc != LIFT_OK) return rc;
        if (g <= rel_gap_tol) return LIFT_OK;
    }
    return LIFT_ERR_NOT_CONVERGED;
}

int lift_unlift(lift_handle h, float *out, int on_host)
{
    if (!h || !out) return LIFT_ERR_ARG;
    if (!on_host) {
        LIFT_CK(lift::launch_unlift(h->P, h->S.x, out, h->stream));
        return LIFT_OK;
    }
    LIFT_CK(lift::launch_unlift(h->P, h->S.x, h->ubuf, h->stream));
    LIFT_CK(cudaMemcpyAsync(out, h->ubuf, h->N * sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream));
    LIFT_CK(cudaStreamSynchronize(h->stream));
    return LIFT_OK;
}

size_t lift_state_bytes(lift_handle h)
{
    if (!h) return 0;
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    return Nk * (2 * sizeof(float2) + sizeof(float4)) + h->N * sizeof(float);
}

static int copy_state(lift_handle h, char *hostdev, size_t bytes, int on_host, bool get)
{
    if (!h || !hostdev || bytes != lift_state_bytes(h)) return LIFT_ERR_ARG;
    const size_t Nk = static_cast<size_t>(h->N) * h->k;
    void *parts[4] = {h->S.x, h->S.xbar, h->S.y, h->S.q};
    const size_t sizes[4] = {Nk * sizeof(float2), Nk * sizeof(float2), Nk * sizeof(float4),
                             h->N * sizeof(float)};
    cudaMemcpyKind kind = on_host ? (get ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice)
                                  : cudaMemcpyDeviceToDevice;
    size_t off = 0;
    for (int j = 0; j < 4; ++j) {
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
    default: return "unknown error code";
    }
}

}  // extern "C"
