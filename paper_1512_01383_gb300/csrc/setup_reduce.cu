// Per-pixel setup, energies, unlifting and the test entry points of the
// lifted solver (arXiv 1512.01383).
#include <math.h>

#include <mutex>

#include "../../include/lift.h"
#include "lift_device.cuh"
#include "lift_params.h"

namespace lift {

// ---------------------------------------------------------------------------
// PL data term: convexify rho on each interval Gamma_i (Sec. 5.4: "convexify
// the matching cost in each range Gamma_i by numerically computing the
// convex envelope").  One thread per (pixel, interval): evaluate rho at the
// interval's breakpoints (its end labels and the sample positions inside),
// build the lower convex hull by a monotone chain, and store the hull's value
// at every breakpoint.  Breakpoint j of interval i is shared with interval
// i+1 when it is the end label; the hull always passes through the end
// points, so both writers store the same value (only interval k-1 writes the
// last one).
// ---------------------------------------------------------------------------
constexpr int kMaxBreaks = 512;

__global__ void pl_setup_kernel(const LiftParams P, float *__restrict__ rhat)
{
    const long long gid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (gid >= static_cast<long long>(P.N) * P.k) return;
    const int pix = static_cast<int>(gid / P.k);
    const int i = static_cast<int>(gid - static_cast<long long>(pix) * P.k);
    const int b0 = P.bstart[i];
    const int n = P.bstart[i + 1] - b0 + 1;
    const float *t = P.bpos + b0;
    float *out = rhat + static_cast<size_t>(pix) * P.nb + b0;

    int stk[kMaxBreaks];
    float sv[kMaxBreaks];
    int m = 0;
    for (int j = 0; j < n; ++j) {
        const float vj = data_rho(P, pix, t[j]);
        while (m >= 2) {
            const int a = stk[m - 2], b = stk[m - 1];
            // drop b if it lies on or above the segment from a to j
            const float cr = (t[b] - t[a]) * (vj - sv[m - 2]) - (sv[m - 1] - sv[m - 2]) * (t[j] - t[a]);
            if (cr <= 0.0f) --m; else break;
        }
        stk[m] = j;
        sv[m] = vj;
        ++m;
    }
    int s = 0;
    const int last = (i == P.k - 1) ? n : n - 1;
    for (int j = 0; j < last; ++j) {
        while (s < m - 2 && stk[s + 1] <= j) ++s;
        const int a = stk[s], b = stk[s + 1];
        float val;
        if (j == a) val = sv[s];
        else if (j == b) val = sv[s + 1];
        else {
            const float w = (t[j] - t[a]) / (t[b] - t[a]);
            val = (1.0f - w) * sv[s] + w * sv[s + 1];
        }
        out[j] = val;
    }
}

cudaError_t launch_pl_setup(const LiftParams &P, float *rhat, cudaStream_t st)
{
    const long long n = static_cast<long long>(P.N) * P.k;
    const int th = 128;
    pl_setup_kernel<<<static_cast<unsigned>((n + th - 1) / th), th, 0, st>>>(P, rhat);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energies (one thread per pixel; per-pixel terms in FP32, sums in FP64).
// ---------------------------------------------------------------------------
constexpr int kEnergyThreads = 256;

// Projection onto {1 >= w_1 >= ... >= w_k >= 0}: pool adjacent violators for
// the non-increasing order, then clamp to [0,1].
__device__ void monotone_project(const float2 *__restrict__ x, int k, float *w)
{
    float val[LIFT_MAXK_DEV];
    int cnt[LIFT_MAXK_DEV];
    int nb = 0;
    for (int i = 0; i < k; ++i) {
        val[nb] = x[i].x;
        cnt[nb] = 1;
        ++nb;
        while (nb > 1 && val[nb - 2] < val[nb - 1]) {
            const float tot = val[nb - 2] * cnt[nb - 2] + val[nb - 1] * cnt[nb - 1];
            cnt[nb - 2] += cnt[nb - 1];
            val[nb - 2] = tot / static_cast<float>(cnt[nb - 2]);
            --nb;
        }
    }
    int o = 0;
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < cnt[b]; ++c) w[o++] = fminf(fmaxf(val[b], 0.0f), 1.0f);
}

__device__ __forceinline__ float unlift_pixel(const float2 *__restrict__ x, int k, float gmin,
                                              float delta)
{
    float a = 0.0f;
    for (int i = 0; i < k; ++i) a += fminf(fmaxf(x[i].x, 0.0f), 1.0f);
    return gmin + delta * a;
}

// VOL: a D x H x W volume; p_i's third component in pz, and the slice
// neighbours (z + 1 for the forward differences, z - 1 in div p) join.
template <int KIND, bool VOL>
__global__ void __launch_bounds__(kEnergyThreads)
energy_kernel(const LiftParams P, const float2 *__restrict__ x, const float4 *__restrict__ y,
              const float *__restrict__ pz, double *__restrict__ partial, int p0, int p1)
{
    // the pixels [p0, p1) (a band's own rows; the whole problem otherwise)
    const int pix = p0 + blockIdx.x * kEnergyThreads + threadIdx.x;
    double eP = 0.0, eD = 0.0, eE = 0.0;
    if (pix < p1) {
        const int k = P.k;
        const int row = pix / P.W, col = pix - row * P.W;
        const int yy = VOL ? row % P.H : row;
        const size_t o = static_cast<size_t>(pix) * k;
        const size_t sx = static_cast<size_t>(k), sy = static_cast<size_t>(P.W) * k;
        const size_t sz = static_cast<size_t>(P.HW) * k;
        const bool hr = col + 1 < P.W, hd = yy + 1 < P.H, hl = col > 0, hu = yy > 0;
        const bool hb = VOL && pix < P.N - P.HW, hf = VOL && pix >= P.HW;

        // dual bound: sum_i min(0, v_i - div p_i) - max_i (c_i(v) + rho_i^*(v_i/Delta))
        double dsum = 0.0, prefix = 0.0, cmax = -INFINITY;
        for (int i = 0; i < k; ++i) {
            const float4 d = y[o + i];
            float dv = 0.0f;
            if (hr) dv += d.z;
            if (hl) dv -= y[o + i - sx].z;
            if (hd) dv += d.w;
            if (hu) dv -= y[o + i - sy].w;
            if (hb) dv += pz[o + i];
            if (hf) dv -= pz[o + i - sz];
            const float g = d.x - dv;
            dsum += g < 0.0f ? static_cast<double>(g) : 0.0;
            const float gi = P.gmin + P.delta * i;
            const float yv = d.x / P.delta;
            const double ci = prefix - static_cast<double>(gi) * yv +
                              static_cast<double>(piece_conj<KIND>(P, pix, i, gi, yv));
            cmax = ci > cmax ? ci : cmax;
            prefix += d.x;
        }
        eD = dsum - cmax;

        // primal bound on the monotone projection of u
        float w[LIFT_MAXK_DEV], wr[LIFT_MAXK_DEV], wd[LIFT_MAXK_DEV];
        float wb[VOL ? LIFT_MAXK_DEV : 1];
        monotone_project(x + o, k, w);
        if (hr) monotone_project(x + o + sx, k, wr);
        if (hd) monotone_project(x + o + sy, k, wd);
        if (VOL && hb) monotone_project(x + o + sz, k, wb);
        double dat = 0.0, tv = 0.0;
        float tail = 0.0f;
        float Snext = 0.0f;                      // S_{i+1}, starting from S_k = 0
        for (int i = k - 1; i >= 0; --i) {
            float Si;
            if (i == 0) Si = 1.0f;
            else {
                tail += -P.delta * x[o + i].y;
                Si = fminf(fmaxf(tail, w[i]), w[i - 1]);
            }
            const float li = Si - Snext;
            if (li > 0.0f) {
                const float a = fminf(fmaxf((w[i] - Snext) / li, 0.0f), 1.0f);
                const float gi = P.gmin + P.delta * i;
                dat += static_cast<double>(li) *
                       static_cast<double>(piece_envelope<KIND>(P, pix, i, gi, gi + a * P.delta));
            }
            const float ax = hr ? wr[i] - w[i] : 0.0f;
            const float ay = hd ? wd[i] - w[i] : 0.0f;
            const float az = VOL && hb ? wb[VOL ? i : 0] - w[i] : 0.0f;
            tv += static_cast<double>(P.delta * (P.aniso ? fabsf(ax) + fabsf(ay) + fabsf(az)
                                                         : sqrtf(ax * ax + ay * ay + az * az)));
            Snext = Si;
        }
        eP = dat + static_cast<double>(P.lam) * tv;

        // nonconvex energy of the unlifted image
        const float ut = unlift_pixel(x + o, k, P.gmin, P.delta);
        const float ax = hr ? unlift_pixel(x + o + sx, k, P.gmin, P.delta) - ut : 0.0f;
        const float ay = hd ? unlift_pixel(x + o + sy, k, P.gmin, P.delta) - ut : 0.0f;
        const float az = hb ? unlift_pixel(x + o + sz, k, P.gmin, P.delta) - ut : 0.0f;
        eE = static_cast<double>(data_rho(P, pix, ut)) +
             static_cast<double>(P.lam) *
                 static_cast<double>(P.aniso ? fabsf(ax) + fabsf(ay) + fabsf(az)
                                             : sqrtf(ax * ax + ay * ay + az * az));
    }

    // block reduction: warp shuffles, then one value per warp
    __shared__ double red[3][kEnergyThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        eP += __shfl_down_sync(0xffffffffu, eP, off);
        eD += __shfl_down_sync(0xffffffffu, eD, off);
        eE += __shfl_down_sync(0xffffffffu, eE, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = eP; red[1][wid] = eD; red[2][wid] = eE; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int j = 0; j < kEnergyThreads / 32; ++j) { a += red[0][j]; b += red[1][j]; c += red[2][j]; }
        partial[3 * blockIdx.x + 0] = a;
        partial[3 * blockIdx.x + 1] = b;
        partial[3 * blockIdx.x + 2] = c;
    }
}

// Second pass: one block sums the per-block partials in a fixed order.
__global__ void __launch_bounds__(kEnergyThreads)
energy_finish_kernel(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    double a = 0.0, b = 0.0, c = 0.0;
    for (int j = threadIdx.x; j < nblocks; j += kEnergyThreads) {
        a += partial[3 * j]; b += partial[3 * j + 1]; c += partial[3 * j + 2];
    }
    __shared__ double red[3][kEnergyThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
        c += __shfl_down_sync(0xffffffffu, c, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = a; red[1][wid] = b; red[2][wid] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int j = 0; j < kEnergyThreads / 32; ++j) { s0 += red[0][j]; s1 += red[1][j]; s2 += red[2][j]; }
        out[0] = s0; out[1] = s1; out[2] = s2;
    }
}

int energy_blocks(const LiftParams &P)
{
    return (P.N + kEnergyThreads - 1) / kEnergyThreads;
}

cudaError_t launch_energy(const LiftParams &P, const LiftState &S, double *partial, double *out,
                          cudaStream_t st)
{
    return launch_energy_range(P, S, 0, P.N, partial, out, st);
}

cudaError_t launch_energy_range(const LiftParams &P, const LiftState &S, int p0, int p1,
                                double *partial, double *out, cudaStream_t st)
{
    const int nb = (p1 - p0 + kEnergyThreads - 1) / kEnergyThreads;
    if (nb <= 0) return cudaErrorInvalidValue;
    const bool vol = P.D > 1;
    if (P.kind == 2) {
        if (vol) energy_kernel<2, true><<<nb, kEnergyThreads, 0, st>>>(P, S.x, S.y, S.pz, partial, p0, p1);
        else energy_kernel<2, false><<<nb, kEnergyThreads, 0, st>>>(P, S.x, S.y, nullptr, partial, p0, p1);
    } else {
        if (vol) energy_kernel<0, true><<<nb, kEnergyThreads, 0, st>>>(P, S.x, S.y, S.pz, partial, p0, p1);
        else energy_kernel<0, false><<<nb, kEnergyThreads, 0, st>>>(P, S.x, S.y, nullptr, partial, p0, p1);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_finish_kernel<<<1, kEnergyThreads, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Movement of the iterate between two checks (adaptive balance), one thread
// per pixel; the steps of balance theta are converted to those of theta = 1
// (tau / theta, sigma * theta).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEnergyThreads)
movement_kernel(const LiftParams P, const float2 *__restrict__ x, const float4 *__restrict__ y,
                const float *__restrict__ q, const float *__restrict__ pz,
                const float2 *__restrict__ xp, const float4 *__restrict__ yp,
                const float *__restrict__ qp, const float *__restrict__ pzp, float theta,
                double *__restrict__ partial)
{
    const int pix = blockIdx.x * kEnergyThreads + threadIdx.x;
    double mx = 0.0, my = 0.0;
    if (pix < P.N) {
        const size_t o = static_cast<size_t>(pix) * P.k;
        const float itu = theta / P.tau_u;           // 1 / (tau_u / theta)
        const float isp = 1.0f / (P.sigma_p * theta);
        for (int i = 0; i < P.k; ++i) {
            const float4 ic = P.icst[i];
            const float2 a = x[o + i], b = xp[o + i];
            const float du = a.x - b.x, ds = a.y - b.y;
            mx += static_cast<double>(du * du * itu + ds * ds * (theta / ic.y));
            const float4 c = y[o + i], e = yp[o + i];
            const float dv = c.x - e.x, dz = c.y - e.y, dpx = c.z - e.z, dpy = c.w - e.w;
            const float dpz = pz != nullptr ? pz[o + i] - pzp[o + i] : 0.0f;
            my += static_cast<double>((dv * dv + dz * dz) / (ic.z * theta) +
                                      (dpx * dpx + dpy * dpy + dpz * dpz) * isp);
        }
        const float dq = q[pix] - qp[pix];
        my += static_cast<double>(dq * dq / (P.sigma_q * theta));
    }
    __shared__ double red[2][kEnergyThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        mx += __shfl_down_sync(0xffffffffu, mx, off);
        my += __shfl_down_sync(0xffffffffu, my, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = mx; red[1][wid] = my; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < kEnergyThreads / 32; ++j) { a += red[0][j]; b += red[1][j]; }
        partial[3 * blockIdx.x + 0] = a;
        partial[3 * blockIdx.x + 1] = b;
        partial[3 * blockIdx.x + 2] = 0.0;
    }
}

cudaError_t launch_movement(const LiftParams &P, const LiftState &S, const LiftState &Sprev,
                            float theta, double *partial, double *out, cudaStream_t st)
{
    const int nb = energy_blocks(P);
    movement_kernel<<<nb, kEnergyThreads, 0, st>>>(P, S.x, S.y, S.q, S.pz, Sprev.x, Sprev.y,
                                                   Sprev.q, Sprev.pz, theta, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_finish_kernel<<<1, kEnergyThreads, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Unlifting (layer-cake formula, Sec. 3).
// ---------------------------------------------------------------------------
__global__ void unlift_kernel(const LiftParams P, const float2 *__restrict__ x,
                              float *__restrict__ out)
{
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= P.N) return;
    out[pix] = unlift_pixel(x + static_cast<size_t>(pix) * P.k, P.k, P.gmin, P.delta);
}

cudaError_t launch_unlift(const LiftParams &P, const float2 *x, float *out, cudaStream_t st)
{
    unlift_kernel<<<(P.N + 255) / 256, 256, 0, st>>>(P, x, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Test entry points: the projection and the envelope at arbitrary points.
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void proj_epi_kernel(const LiftParams P, const int *__restrict__ pix,
                                const int *__restrict__ itv, const float *__restrict__ y0,
                                const float *__restrict__ h0, float *__restrict__ yo,
                                float *__restrict__ ho, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = itv[j];
    if (pix[j] < 0 || pix[j] >= P.N || i < 0 || i >= P.k) {   // reject, do not read
        yo[j] = ho[j] = __int_as_float(0x7fc00000);
        return;
    }
    float a, b;
    piece_project<KIND>(P, pix[j], i, P.gmin + P.delta * i, y0[j], h0[j], a, b);
    yo[j] = a;
    ho[j] = b;
}

template <int KIND>
__global__ void envelope_kernel(const LiftParams P, const int *__restrict__ pix,
                                const int *__restrict__ itv, const float *__restrict__ t,
                                float *__restrict__ out, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = itv[j];
    if (pix[j] < 0 || pix[j] >= P.N || i < 0 || i >= P.k) {
        out[j] = __int_as_float(0x7fc00000);
        return;
    }
    out[j] = piece_envelope<KIND>(P, pix[j], i, P.gmin + P.delta * i, t[j]);
}

cudaError_t launch_proj_epi(const LiftParams &P, const int *pix, const int *interval,
                            const float *y0, const float *h0, float *y, float *h, int n,
                            cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int nb = (n + 255) / 256;
    if (P.kind == 2)
        proj_epi_kernel<2><<<nb, 256, 0, st>>>(P, pix, interval, y0, h0, y, h, n);
    else
        proj_epi_kernel<0><<<nb, 256, 0, st>>>(P, pix, interval, y0, h0, y, h, n);
    return cudaGetLastError();
}

cudaError_t launch_envelope(const LiftParams &P, const int *pix, const int *interval,
                            const float *t, float *out, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int nb = (n + 255) / 256;
    if (P.kind == 2)
        envelope_kernel<2><<<nb, 256, 0, st>>>(P, pix, interval, t, out, n);
    else
        envelope_kernel<0><<<nb, 256, 0, st>>>(P, pix, interval, t, out, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Running average of the iterate: a <- a + w (x - a) record by record over
// x = {u, s}, y = {v, z, px, py} (and pz on volumes), and pixel by pixel over
// q; first: a <- x (the average of one iterate; the buffers' old contents are
// not read).  A grid-stride loop over the N*k records and the N pixels.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
average_kernel(const float2 *__restrict__ x, const float4 *__restrict__ y,
               const float *__restrict__ pz, const float *__restrict__ q,
               float2 *__restrict__ ax, float4 *__restrict__ ay, float *__restrict__ apz,
               float *__restrict__ aq, size_t nk, size_t npix, float w, int first)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    const size_t t0 = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    for (size_t r = t0; r < nk; r += stride) {
        const float2 a = x[r];
        const float4 b = y[r];
        if (first) {
            ax[r] = a;
            ay[r] = b;
            if (pz) apz[r] = pz[r];
        } else {
            const float2 c = ax[r];
            const float4 d = ay[r];
            ax[r] = make_float2(c.x + w * (a.x - c.x), c.y + w * (a.y - c.y));
            ay[r] = make_float4(d.x + w * (b.x - d.x), d.y + w * (b.y - d.y),
                                d.z + w * (b.z - d.z), d.w + w * (b.w - d.w));
            if (pz) apz[r] = apz[r] + w * (pz[r] - apz[r]);
        }
    }
    for (size_t p = t0; p < npix; p += stride)
        aq[p] = first ? q[p] : aq[p] + w * (q[p] - aq[p]);
}

cudaError_t launch_average(const LiftState &S, float2 *ax, float4 *ay, float *apz, float *aq,
                           size_t nk, size_t npix, float w, bool first, cudaStream_t st)
{
    if (nk == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t need = (nk + 255) / 256;
    const size_t cap = static_cast<size_t>(sms) * 8;          // 8 blocks of 256 per SM
    const unsigned blocks = static_cast<unsigned>(need < cap ? need : cap);
    average_kernel<<<blocks, 256, 0, st>>>(S.x, S.y, apz ? S.pz : nullptr, S.q, ax, ay, apz, aq,
                                           nk, npix, w, first ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace lift

// ---------------------------------------------------------------------------
// Allocation-free energy evaluation (lift_energy_noalloc in include/lift.h).
// The per-block partial sums of energy_kernel go to this fixed array instead
// of a buffer from cudaMalloc.  Host code must not pass the symbol itself to a
// kernel (on the host it names a stand-in, not device memory): its device
// address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoAllocBlocks = (LIFT_NOALLOC_MAX_PIXELS + lift::kEnergyThreads - 1) /
                               lift::kEnergyThreads;
constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_scratch_dev[kNoAllocDevices] = {};
}  // namespace

static __device__ __align__(256) double lift_noalloc_partial[3 * kNoAllocBlocks];

extern "C" int lift_energy_noalloc(const lift_spec *spec, const void *state, double *out,
                                   void *stream)
{
    if (!spec || !state || !out) return LIFT_ERR_ARG;
    if (spec->kind != LIFT_QUAD && spec->kind != LIFT_TRUNC_QUAD) return LIFT_ERR_SPEC;
    if (spec->data_on_host || !spec->f) return LIFT_ERR_ARG;
    if (spec->H < 1 || spec->W < 1 || spec->L < 2 || spec->L > LIFT_MAX_K + 1) return LIFT_ERR_SPEC;
    if (!(spec->gamma_max > spec->gamma_min) || !(spec->lambda >= 0.0) || !(spec->alpha > 0.0))
        return LIFT_ERR_SPEC;
    if (spec->kind == LIFT_TRUNC_QUAD && !(spec->nu > 0.0)) return LIFT_ERR_SPEC;
    if (spec->D > 1) return LIFT_ERR_SPEC;                 // images only
    const long long npix = static_cast<long long>(spec->H) * spec->W;
    if (npix > LIFT_NOALLOC_MAX_PIXELS) return LIFT_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(state) & 15u) != 0) return LIFT_ERR_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LIFT_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocDevices) return LIFT_ERR_ARG;
    // the array's address is the current device's: a stream of another
    // device would run the kernels against the wrong memory
    if (stream) {
        int sdev = -1;
        if (cudaStreamGetDevice(static_cast<cudaStream_t>(stream), &sdev) != cudaSuccess)
            return LIFT_ERR_CUDA;
        if (sdev != dev) return LIFT_ERR_ARG;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_scratch_dev[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, lift_noalloc_partial) != cudaSuccess || !p)
                return LIFT_ERR_CUDA;
            g_noalloc_scratch_dev[dev] = static_cast<double *>(p);
        }
        scratch = g_noalloc_scratch_dev[dev];
    }

    lift::LiftParams P{};
    const int k = spec->L - 1;
    P.H = spec->H; P.W = spec->W; P.k = k; P.N = static_cast<int>(npix);
    P.D = 1; P.HW = P.N;
    P.kind = spec->kind;
    P.aniso = spec->tv_anisotropic ? 1 : 0;
    P.delta = static_cast<float>((spec->gamma_max - spec->gamma_min) / k);
    P.gmin = static_cast<float>(spec->gamma_min);
    P.lam = static_cast<float>(spec->lambda);
    P.alpha = static_cast<float>(spec->alpha);
    P.nu = static_cast<float>(spec->nu);
    P.wtrunc = spec->kind == LIFT_TRUNC_QUAD ? static_cast<float>(sqrt(spec->nu / spec->alpha)) : 0.0f;
    P.f = spec->f;

    const size_t Nk = static_cast<size_t>(npix) * k;
    const float2 *x = static_cast<const float2 *>(state);
    const float4 *y = reinterpret_cast<const float4 *>(static_cast<const char *>(state) +
                                                        2 * Nk * sizeof(float2));
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = lift::energy_blocks(P);
    lift::energy_kernel<0, false><<<nb, lift::kEnergyThreads, 0, st>>>(P, x, y, nullptr, scratch, 0,
                                                                        P.N);
    if (cudaGetLastError() != cudaSuccess) return LIFT_ERR_CUDA;
    lift::energy_finish_kernel<<<1, lift::kEnergyThreads, 0, st>>>(scratch, nb, out);
    if (cudaGetLastError() != cudaSuccess) return LIFT_ERR_CUDA;
    return LIFT_OK;
}
