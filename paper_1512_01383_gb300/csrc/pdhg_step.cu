// The two fused half-steps of the preconditioned primal-dual iteration on the
// lifted saddle-point problem (arXiv 1512.01383, Sec. 4,
// eq. discrete_saddle_point_final with the z-splitting of
// eq. equality_constr_data and its multiplier s):
//
//   dual step   (from the extrapolated primal ubar, sbar)
//     p_i  <- Proj_{|.| <= lambda Delta}(p_i + sigma_p grad ubar_i)        (Prop. 5)
//     v_l  <- v_l + sigma_l (ubar_l + Delta sum_{j>l} sbar_j - gamma_l sbar_l)
//     z_i  <- z_i + sigma_i sbar_i
//     q    <- q - sigma_q (1 + Delta sum_i sbar_i)
//     (v_i, z_i) <- Delta Proj_{epi rho_i^*}((v_i, z_i) / Delta)           (Fig. 7)
//   primal step
//     u_l  <- clamp(u_l - tau_u (v_l - div p_l), 0, 1)
//     s_i  <- s_i - tau_i (z_i - Delta q + Delta sum_{l<i} v_l - gamma_i v_i)
//     ubar <- 2 u_new - u,  sbar <- 2 s_new - s
//
// Memory: label-innermost records, primal float2 {u,s}, extrapolated primal
// float2 {ubar,sbar}, dual float4 {v,z,px,py}, q one float per pixel.  One
// thread owns one (pixel, interval) record, so every warp moves one
// contiguous, fully coalesced run of 8- or 16-byte records.  A block of 256
// threads holds floor(256/k) whole pixels; the per-pixel sums over the k
// intervals (the coupling of v, s and q through the operator of Sec. 4) are
// segmented scans: warp shuffles inside each warp, one shared-memory carry
// for the pixels that straddle a warp boundary.  Halo values (ubar at x+1
// and y+1 in the dual step, p at x-1 and y-1 in the primal step) are re-read
// from L1/L2; the algorithmic DRAM traffic is (20k + 3) floats per pixel and
// iteration (+ f).  On a volume (D > 1, the d = 3 grid of Sec. 4) p_i has a
// third component, kept in its own [N][k] float array pz, and the
// differences add the next / previous slice: (23k + 3) floats per voxel.
#include "lift_device.cuh"
#include "lift_params.h"
#include "lift_tile.cuh"

namespace lift {

// The segmented scan of lift_tile.cuh for two independent values per thread
// (two tiles of the same shape processed by one block), one barrier for both.
struct SegScan2 {
    float2 incl, total;
};

__device__ __forceinline__ SegScan2 block_segmented_scan2(float2 val, int seg, int k, int tid,
                                                          bool active, float2 *s_in, float2 *s_last)
{
    const int lane = tid & 31, warp = tid >> 5;
    const int wbase = warp << 5;
    const int start = seg > wbase ? seg - wbase : 0;
    float2 x = val;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float a = __shfl_up_sync(0xffffffffu, x.x, off);
        const float b = __shfl_up_sync(0xffffffffu, x.y, off);
        if (lane - off >= start) { x.x += a; x.y += b; }
    }
    s_in[tid] = x;
    if (lane == 31) s_last[warp] = x;
    __syncthreads();
    SegScan2 r{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (!active) return r;
    const int sw = seg >> 5;
    float2 carry = make_float2(0.f, 0.f);
    if (sw < warp) {
        carry = s_last[warp - 1];
        if (sw < warp - 1) { carry.x += s_last[warp - 2].x; carry.y += s_last[warp - 2].y; }
    }
    r.incl = make_float2(x.x + carry.x, x.y + carry.y);
    const int e = seg + k - 1, ew = e >> 5;
    float2 ce = make_float2(0.f, 0.f);
    if (sw < ew) {
        ce = s_last[sw];
        if (sw + 1 < ew) { ce.x += s_last[sw + 1].x; ce.y += s_last[sw + 1].y; }
    }
    r.total = make_float2(s_in[e].x + ce.x, s_in[e].y + ce.y);
    return r;
}

// One tile: floor(THREADS/k) whole pixels of one problem instance, one
// thread per (pixel, interval) record; used by the single-instance kernels and
// the batched kernels below.  VOL: a D x H x W volume, whose p_i has a third
// component in pz (Sec. 4 on the d = 3 grid); images take VOL = false and
// never touch pz.
template <int KIND, int THREADS, bool VOL = false>
__device__ __forceinline__ void dual_tile(const LiftParams &P, const float2 *__restrict__ xbar,
                                          float4 *__restrict__ y, float *__restrict__ q,
                                          int tile, float *s_in, float *s_last,
                                          float *__restrict__ pz = nullptr)
{
    const int tid = threadIdx.x;
    int lp, i;
    split_thread(P, tid, lp, i);
    const int pix = tile * P.ppb + lp;
    const bool active = lp < P.ppb && pix < P.N;
    const size_t o = static_cast<size_t>(pix) * P.k + i;

    float2 xb = make_float2(0.0f, 0.0f);
    float4 d = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (active) {
        xb = xbar[o];
        d = y[o];
    }
    const SegScan sc = block_segmented_scan(xb.y, lp * P.k, P.k, tid, active, s_in, s_last);
    if (!active) return;

    const int row = pixel_row(P, pix);
    const int col = pix - row * P.W;
    const int yy = VOL ? row_in_slice(P, row) : row;
    const float4 ic = __ldg(P.icst + i);      // {gamma_i, tau_s, sigma_vz, lambda*Delta}
    const float4 stp = __ldg(P.steps);        // {tau_u, sigma_q, sigma_p, 0}

    // TV dual: forward differences (Neumann), ascent, l2-ball projection
    const float gx = col + 1 < P.W ? xbar[o + P.k].x - xb.x : 0.0f;
    const float gy = yy + 1 < P.H ? xbar[o + static_cast<size_t>(P.W) * P.k].x - xb.x : 0.0f;
    float px = d.z + stp.z * gx;
    float py = d.w + stp.z * gy;
    float pzv = 0.0f;
    if (VOL) {
        const float gz = pix < P.N - P.HW ? xbar[o + static_cast<size_t>(P.HW) * P.k].x - xb.x
                                          : 0.0f;
        pzv = pz[o] + stp.z * gz;
    }
    if (P.aniso) {                              // l-infinity box (anisotropic TV)
        px = fminf(fmaxf(px, -ic.w), ic.w);
        py = fminf(fmaxf(py, -ic.w), ic.w);
        if (VOL) pzv = fminf(fmaxf(pzv, -ic.w), ic.w);
    } else {                                    // l2 ball (isotropic TV)
        const float n2 = px * px + py * py + (VOL ? pzv * pzv : 0.0f);
        if (n2 > ic.w * ic.w) {
            const float sc2 = ic.w * rsqrtf(n2);
            px *= sc2;
            py *= sc2;
            if (VOL) pzv *= sc2;
        }
    }
    if (VOL) pz[o] = pzv;

    // data duals: sum of sbar over the pixel's later intervals = total - inclusive
    const float tail = sc.total - sc.incl;
    float v = d.x + ic.z * (xb.x + P.delta * tail - ic.x * xb.y);
    float z = d.y + ic.z * xb.y;
    if (i == 0) q[pix] -= stp.y * (1.0f + P.delta * sc.total);

    // (v, z) onto Delta * epi(rho_i^*)
    float yo, ho;
    piece_project<KIND>(P, pix, i, ic.x, v * P.inv_delta, z * P.inv_delta, yo, ho);
    v = P.delta * yo;
    z = P.delta * ho;

    y[o] = make_float4(v, z, px, py);
}

// Two consecutive tiles (2 pair, 2 pair + 1) of a quadratic-type problem in
// one block, each thread owning one record of each.  The epigraph projection
// is the only divergent part of the step: after the first iterations only a
// few records per warp leave the epigraph (about 2 of 32 per tile on the
// 512^2, L = 20 denoising problem, yet nearly every warp holds some).  The
// records below the graph of both tiles are packed into one pass of the warp
// through a per-warp queue in shared memory (no block barrier), so a warp runs
// the projection once for two tiles instead of once per tile.  Each record's
// arithmetic is that of dual_tile.
template <int THREADS>
struct PairSmem {
    float2 in[THREADS];
    float2 last[THREADS / 32];
    float4 queue[THREADS / 32][64];
};

// EARLY: q and f are loaded with the records, before the scan's barrier,
// so their latency overlaps it (the single-instance kernel: 61.4 -> 57.4 us
// at 512^2, L = 20, same 48 registers); the batched kernel keeps the late
// loads, which in it would cost 24 registers.
template <int THREADS, bool VOL, bool EARLY = false>
__device__ __forceinline__ void dual_pair(const LiftParams &P, const float2 *__restrict__ xbar,
                                          float4 *__restrict__ y, float *__restrict__ q,
                                          float *__restrict__ pz, int pair, PairSmem<THREADS> &sm)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int lp, i;
    split_thread(P, tid, lp, i);
    int pix[2]; bool act[2]; size_t o[2]; float2 xb[2]; float4 d[2];
    float qo[2], fv[2];   // EARLY: q (interval 0) and f of the record's pixel
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        pix[u] = (2 * pair + u) * P.ppb + lp;
        act[u] = lp < P.ppb && pix[u] < P.N;
        o[u] = static_cast<size_t>(pix[u]) * P.k + i;
        xb[u] = make_float2(0.f, 0.f);
        d[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        qo[u] = fv[u] = 0.f;
        if (act[u]) {
            xb[u] = xbar[o[u]];
            d[u] = y[o[u]];
            if (EARLY) {
                if (i == 0) qo[u] = q[pix[u]];
                fv[u] = __ldg(P.f + pix[u]);
            }
        }
    }
    const SegScan2 sc = block_segmented_scan2(make_float2(xb[0].y, xb[1].y), lp * P.k, P.k, tid,
                                              act[0], sm.in, sm.last);
    const float4 ic = __ldg(P.icst + (lp < P.ppb ? i : 0));  // {gamma_i, tau_s, sigma_vz, lambda*Delta}
    const float4 stp = __ldg(P.steps);                        // {tau_u, sigma_q, sigma_p, 0}
    float px[2], py[2], y0[2], h0[2];
    bool below[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        px[u] = py[u] = y0[u] = h0[u] = 0.0f;
        below[u] = false;
        if (!act[u]) continue;
        const int row = pixel_row(P, pix[u]);
        const int col = pix[u] - row * P.W;
        const int yy = VOL ? row_in_slice(P, row) : row;

        // TV dual: forward differences (Neumann), ascent, ball (or box) projection
        const float gx = col + 1 < P.W ? xbar[o[u] + P.k].x - xb[u].x : 0.0f;
        const float gy = yy + 1 < P.H ? xbar[o[u] + static_cast<size_t>(P.W) * P.k].x - xb[u].x
                                      : 0.0f;
        px[u] = d[u].z + stp.z * gx;
        py[u] = d[u].w + stp.z * gy;
        float pzv = 0.0f;
        if (VOL) {
            const float gz = pix[u] < P.N - P.HW
                                 ? xbar[o[u] + static_cast<size_t>(P.HW) * P.k].x - xb[u].x : 0.0f;
            pzv = pz[o[u]] + stp.z * gz;
        }
        if (P.aniso) {
            px[u] = fminf(fmaxf(px[u], -ic.w), ic.w);
            py[u] = fminf(fmaxf(py[u], -ic.w), ic.w);
            if (VOL) pzv = fminf(fmaxf(pzv, -ic.w), ic.w);
        } else {
            const float n2 = px[u] * px[u] + py[u] * py[u] + (VOL ? pzv * pzv : 0.0f);
            if (n2 > ic.w * ic.w) {
                const float sc2 = ic.w * rsqrtf(n2);
                px[u] *= sc2;
                py[u] *= sc2;
                if (VOL) pzv *= sc2;
            }
        }
        if (VOL) pz[o[u]] = pzv;

        // data duals: sum of sbar over the pixel's later intervals = total - inclusive
        const float total = u == 0 ? sc.total.x : sc.total.y;
        const float tail = total - (u == 0 ? sc.incl.x : sc.incl.y);
        const float v = d[u].x + ic.z * (xb[u].x + P.delta * tail - ic.x * xb[u].y);
        const float z = d[u].y + ic.z * xb[u].y;
        if (i == 0) q[pix[u]] = (EARLY ? qo[u] : q[pix[u]]) - stp.y * (1.0f + P.delta * total);
        y0[u] = v * P.inv_delta;
        h0[u] = z * P.inv_delta;
        // the test of piece_in_epigraph<0>, with f already loaded when EARLY
        below[u] = EARLY ? !(h0[u] >= quad_conj_direct(P, fv[u], ic.x, ic.x + P.delta, y0[u]))
                         : !piece_in_epigraph<0>(P, pix[u], i, ic.x, y0[u], h0[u]);
    }

    // queue slots: tile 0's records below the graph, then tile 1's (at most 64)
    const unsigned m0 = __ballot_sync(0xffffffffu, below[0]);
    const unsigned m1 = __ballot_sync(0xffffffffu, below[1]);
    const int n0 = __popc(m0), n = n0 + __popc(m1);
    const unsigned lt = (1u << lane) - 1u;
    const int e0 = __popc(m0 & lt), e1 = n0 + __popc(m1 & lt);
    float4 *qw = sm.queue[warp];
    if (below[0]) qw[e0] = make_float4(y0[0], h0[0], __int_as_float(pix[0]), __int_as_float(i));
    if (below[1]) qw[e1] = make_float4(y0[1], h0[1], __int_as_float(pix[1]), __int_as_float(i));
    __syncwarp();
    // (v, z) onto Delta * epi(rho_i^*), packed
    for (int j = lane; j < n; j += 32) {
        const float4 e = qw[j];
        const int qp = __float_as_int(e.z), qi = __float_as_int(e.w);
        float yo, ho;
        piece_project_below<0>(P, qp, qi, __ldg(P.icst + qi).x, e.x, e.y, yo, ho);
        qw[j] = make_float4(yo, ho, e.z, e.w);
    }
    __syncwarp();
    if (below[0]) { const float4 r = qw[e0]; y0[0] = r.x; h0[0] = r.y; }
    if (below[1]) { const float4 r = qw[e1]; y0[1] = r.x; h0[1] = r.y; }
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (act[u]) y[o[u]] = make_float4(P.delta * y0[u], P.delta * h0[u], px[u], py[u]);
}

template <int THREADS>
__device__ __forceinline__ void primal_tile(const LiftParams &P, float2 *__restrict__ x,
                                            float2 *__restrict__ xbar,
                                            const float4 *__restrict__ y,
                                            const float *__restrict__ q, int tile, float *s_in,
                                            float *s_last)
{
    const int tid = threadIdx.x;
    int lp, i;
    split_thread(P, tid, lp, i);
    const int pix = tile * P.ppb + lp;
    const bool active = lp < P.ppb && pix < P.N;
    const size_t o = static_cast<size_t>(pix) * P.k + i;

    float4 d = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float2 xo = make_float2(0.0f, 0.0f);
    if (active) {
        d = y[o];
        xo = x[o];
    }
    const SegScan sc = block_segmented_scan(d.x, lp * P.k, P.k, tid, active, s_in, s_last);
    if (!active) return;

    const int row = pixel_row(P, pix);
    const int col = pix - row * P.W;
    const float4 ic = __ldg(P.icst + i);
    const float tau_u = __ldg(P.steps).x;
    const float qq = q[pix];

    // div p = -grad^T p (Neumann forward differences)
    float dv = 0.0f;
    if (col + 1 < P.W) dv += d.z;
    if (col > 0) dv -= y[o - P.k].z;
    if (row + 1 < P.H) dv += d.w;
    if (row > 0) dv -= y[o - static_cast<size_t>(P.W) * P.k].w;

    const float head = sc.incl - d.x;             // sum of v over earlier intervals
    const float un = fminf(fmaxf(xo.x - tau_u * (d.x - dv), 0.0f), 1.0f);
    const float sn = xo.y - ic.y * (d.y - P.delta * qq + P.delta * head - ic.x * d.x);
    x[o] = make_float2(un, sn);
    xbar[o] = make_float2(2.0f * un - xo.x, 2.0f * sn - xo.y);
}

// LIVE: a batch member, whose blocks return while its live flag is 0.
// One tile per block: sampled costs (their projection walks the hull's kinks
// and packing costs more registers than it saves), volumes, and quadratic
// pieces with k < kPairMinK (few records per pixel, little to pack).
template <int KIND, bool VOL, bool LIVE>
__global__ void __launch_bounds__(kStepThreads)
dual_step_kernel(const LiftParams P, const float2 *__restrict__ xbar, float4 *__restrict__ y,
                 float *__restrict__ q, float *__restrict__ pz)
{
    __shared__ float s_in[kStepThreads];
    __shared__ float s_last[kStepThreads / 32];
    if (LIVE && *P.live == 0) return;
    dual_tile<KIND, kStepThreads, VOL>(P, xbar, y, q, blockIdx.x + P.blk_off, s_in, s_last, pz);
}

// Quadratic pieces on an image with k >= kPairMinK: two tiles per block with
// the projections packed (dual_pair).
template <bool LIVE>
__global__ void __launch_bounds__(kStepThreads)
dual_pair_kernel(const LiftParams P, const float2 *__restrict__ xbar, float4 *__restrict__ y,
                 float *__restrict__ q)
{
    __shared__ PairSmem<kStepThreads> sm;
    if (LIVE && *P.live == 0) return;
    dual_pair<kStepThreads, false, true>(P, xbar, y, q, nullptr, blockIdx.x + P.blk_off, sm);
}

// Single-instance primal step: each block takes two consecutive tiles and
// issues the loads of both before the (shared) scan, doubling the bytes in
// flight per thread; the primal step waits on memory rather than on issue.
// On images the neighbours' p (x-1, y-1) and q are loaded before the scan's
// barrier too, so their latency overlaps it (37.3 -> 34.9 us per launch at
// 512^2, L = 20, same registers; on a volume that took 40 -> 46 registers
// and one block per SM, 117 -> 129 us at 128^3, L = 8, so volumes load them
// after the scan).
template <bool VOL, bool LIVE>
__global__ void __launch_bounds__(kStepThreads)
primal_step_kernel(const LiftParams P, float2 *__restrict__ x, float2 *__restrict__ xbar,
                   const float4 *__restrict__ y, const float *__restrict__ q,
                   const float *__restrict__ pz)
{
    __shared__ float2 s_in[kStepThreads];
    __shared__ float2 s_last[kStepThreads / 32];
    if (LIVE && *P.live == 0) return;
    const int tid = threadIdx.x;
    int lp, i;
    split_thread(P, tid, lp, i);
    int pix[2]; bool act[2]; size_t o[2]; float4 d[2]; float2 xo[2];
    int col[2], yy[2];
    float qq[2], px_left[2], py_up[2];   // q and the neighbours' p at x-1, y-1
    auto neighbours = [&](int u) {
        const int row = pixel_row(P, pix[u]);
        col[u] = pix[u] - row * P.W;
        yy[u] = VOL ? row_in_slice(P, row) : row;
        qq[u] = q[pix[u]];
        if (col[u] > 0) px_left[u] = y[o[u] - P.k].z;
        if (yy[u] > 0) py_up[u] = y[o[u] - static_cast<size_t>(P.W) * P.k].w;
    };
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        pix[u] = (2 * (blockIdx.x + P.blk_off) + u) * P.ppb + lp;
        act[u] = lp < P.ppb && pix[u] < P.N;
        o[u] = static_cast<size_t>(pix[u]) * P.k + i;
        d[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        xo[u] = make_float2(0.f, 0.f);
        col[u] = yy[u] = 0;
        qq[u] = px_left[u] = py_up[u] = 0.f;
        if (act[u]) {
            d[u] = y[o[u]];
            xo[u] = x[o[u]];
            // images: the neighbours' loads overlap the scan's barrier; on a
            // volume the extra live registers would cost a block per SM
            if (!VOL) neighbours(u);
        }
    }
    const SegScan2 sc = block_segmented_scan2(make_float2(d[0].x, d[1].x), lp * P.k, P.k, tid,
                                              act[0] || act[1], s_in, s_last);
    const float4 ic = __ldg(P.icst + (lp < P.ppb ? i : 0));
    const float tau_u = __ldg(P.steps).x;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (!act[u]) continue;
        if (VOL) neighbours(u);
        // div p = -grad^T p (Neumann forward differences)
        float dv = 0.0f;
        if (col[u] + 1 < P.W) dv += d[u].z;
        if (col[u] > 0) dv -= px_left[u];
        if (yy[u] + 1 < P.H) dv += d[u].w;
        if (yy[u] > 0) dv -= py_up[u];
        if (VOL) {
            if (pix[u] < P.N - P.HW) dv += pz[o[u]];
            if (pix[u] >= P.HW) dv -= pz[o[u] - static_cast<size_t>(P.HW) * P.k];
        }
        const float head = (u == 0 ? sc.incl.x : sc.incl.y) - d[u].x;
        const float un = fminf(fmaxf(xo[u].x - tau_u * (d[u].x - dv), 0.0f), 1.0f);
        const float sn =
            xo[u].y - ic.y * (d[u].y - P.delta * qq[u] + P.delta * head - ic.x * d[u].x);
        x[o[u]] = make_float2(un, sn);
        xbar[o[u]] = make_float2(2.0f * un - xo[u].x, 2.0f * sn - xo[u].y);
    }
}

// ---------------------------------------------------------------------------
// Batched half-steps: many instances (each its own size, k and data) in one
// launch.  Block b processes tile b - tile0 of instance tile_inst[b]; blocks
// of instances whose flag in `live` is 0 (converged) return at once.
// ---------------------------------------------------------------------------
// The block's instance descriptor is staged once in shared memory, so the
// tile body reads its parameters as broadcast shared loads.
__device__ __forceinline__ void stage_desc(const InstDesc *__restrict__ D, int inst, InstDesc *sd)
{
    constexpr int words = static_cast<int>(sizeof(InstDesc) / sizeof(int));
    static_assert(sizeof(InstDesc) % sizeof(int) == 0, "descriptor size");
    const int *src = reinterpret_cast<const int *>(D + inst);
    int *dst = reinterpret_cast<int *>(sd);
    for (int j = threadIdx.x; j < words; j += blockDim.x) dst[j] = __ldg(src + j);
    __syncthreads();
}

// Batches hold quadratic-type images only.  Instances with k >= kPairMinK
// take their dual step in tile pairs, the others in single tiles, as their
// single-instance kernels do; the two kinds of unit have a list and a kernel
// each (one kernel holding both bodies would compile them differently from
// the single-instance kernels).  Block b takes unit b - pair0 of instance
// unit_inst[b].
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
batch_dual_pair_kernel(const InstDesc *__restrict__ D, const int *__restrict__ unit_inst,
                       const int *__restrict__ live)
{
    __shared__ PairSmem<THREADS> sm;
    __shared__ InstDesc sd;
    const int inst = unit_inst[blockIdx.x];
    if (!live[inst]) return;
    stage_desc(D, inst, &sd);
    dual_pair<THREADS, false>(sd.P, sd.S.xbar, sd.S.y, sd.S.q, nullptr, blockIdx.x - sd.pair0, sm);
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 2048 / THREADS)
batch_dual_tile_kernel(const InstDesc *__restrict__ D, const int *__restrict__ unit_inst,
                       const int *__restrict__ live)
{
    __shared__ float s_in[THREADS];
    __shared__ float s_last[THREADS / 32];
    __shared__ InstDesc sd;
    const int inst = unit_inst[blockIdx.x];
    if (!live[inst]) return;
    stage_desc(D, inst, &sd);
    dual_tile<0, THREADS>(sd.P, sd.S.xbar, sd.S.y, sd.S.q, blockIdx.x - sd.pair0, s_in, s_last);
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 2048 / THREADS)
batch_primal_kernel(const InstDesc *__restrict__ D, const int *__restrict__ tile_inst,
                    const int *__restrict__ live)
{
    __shared__ float s_in[THREADS];
    __shared__ float s_last[THREADS / 32];
    __shared__ InstDesc sd;
    const int inst = tile_inst[blockIdx.x];
    if (!live[inst]) return;
    stage_desc(D, inst, &sd);
    primal_tile<THREADS>(sd.P, sd.S.x, sd.S.xbar, sd.S.y, sd.S.q, blockIdx.x - sd.tile0, s_in,
                         s_last);
}

template <int THREADS>
static cudaError_t launch_batch_t(const InstDesc *D, const int *tile_inst, const int *pair_inst,
                                  const int *single_inst, const int *live, int ntiles, int npairs,
                                  int nsingle, cudaStream_t st)
{
    if (npairs > 0) batch_dual_pair_kernel<THREADS><<<npairs, THREADS, 0, st>>>(D, pair_inst, live);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nsingle > 0)
        batch_dual_tile_kernel<THREADS><<<nsingle, THREADS, 0, st>>>(D, single_inst, live);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_primal_kernel<THREADS><<<ntiles, THREADS, 0, st>>>(D, tile_inst, live);
    return cudaGetLastError();
}

cudaError_t launch_batch_iteration(int threads, const InstDesc *D, const int *tile_inst,
                                   const int *pair_inst, const int *single_inst, const int *live,
                                   int ntiles, int npairs, int nsingle, cudaStream_t st)
{
    if (ntiles <= 0) return cudaSuccess;
    switch (threads) {
    case 128: return launch_batch_t<128>(D, tile_inst, pair_inst, single_inst, live, ntiles, npairs, nsingle, st);
    case 256: return launch_batch_t<256>(D, tile_inst, pair_inst, single_inst, live, ntiles, npairs, nsingle, st);
    case 512: return launch_batch_t<512>(D, tile_inst, pair_inst, single_inst, live, ntiles, npairs, nsingle, st);
    default: return cudaErrorInvalidValue;
    }
}

static inline int step_blocks(const LiftParams &P)
{
    return (P.N + P.ppb - 1) / P.ppb;
}

// Which dual kernel a problem uses, and its unit (tiles per block).
static inline bool dual_in_pairs(const LiftParams &P)
{
    return P.kind != 2 && P.D == 1 && P.k >= kPairMinK;
}

// Dual half-step on the tiles [t0, t1).
cudaError_t launch_dual_band(const LiftParams &P0, const LiftState &S, int t0, int t1,
                             cudaStream_t st)
{
    LiftParams P = P0;
    const bool vol = P.D > 1, live = P.live != nullptr;
    if (dual_in_pairs(P)) {
        // volumes never belong to a batch, so VOL and LIVE do not meet
        P.blk_off = t0 / 2;
        const int nb = (t1 - t0 + 1) / 2;
        if (live) dual_pair_kernel<true><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q);
        else dual_pair_kernel<false><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q);
        return cudaGetLastError();
    }
    P.blk_off = t0;
    const int nb = t1 - t0;
    if (P.kind == 2) {
        if (vol) dual_step_kernel<2, true, false><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, S.pz);
        else if (live) dual_step_kernel<2, false, true><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, nullptr);
        else dual_step_kernel<2, false, false><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, nullptr);
    } else {
        if (vol) dual_step_kernel<0, true, false><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, S.pz);
        else if (live) dual_step_kernel<0, false, true><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, nullptr);
        else dual_step_kernel<0, false, false><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, nullptr);
    }
    return cudaGetLastError();
}

// Primal half-step on the tiles [t0, t1) (two tiles per block).
cudaError_t launch_primal_band(const LiftParams &P0, const LiftState &S, int t0, int t1,
                               cudaStream_t st)
{
    LiftParams P = P0;
    P.blk_off = t0 / 2;
    const int nb = (t1 - t0 + 1) / 2;
    if (P.D > 1)
        primal_step_kernel<true, false><<<nb, kStepThreads, 0, st>>>(P, S.x, S.xbar, S.y, S.q, S.pz);
    else if (P.live != nullptr)
        primal_step_kernel<false, true><<<nb, kStepThreads, 0, st>>>(P, S.x, S.xbar, S.y, S.q, nullptr);
    else
        primal_step_kernel<false, false><<<nb, kStepThreads, 0, st>>>(P, S.x, S.xbar, S.y, S.q, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_dual_step(const LiftParams &P, const LiftState &S, cudaStream_t st)
{
    return launch_dual_band(P, S, 0, step_blocks(P), st);
}

cudaError_t launch_primal_step(const LiftParams &P, const LiftState &S, cudaStream_t st)
{
    return launch_primal_band(P, S, 0, step_blocks(P), st);
}

}  // namespace lift
