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
// float2 {ubar,sbar}, dual float4 {v,z,px,py}, q one float per pixel.
//
// The dual step of an image (dual_strip_kernel) stages strips of consecutive
// pixels in shared memory by bulk copies and lets T threads walk each pixel's
// intervals (see the comment above that kernel).  The primal step, and the
// dual step of a volume, give one thread one (pixel, interval) record, so
// every warp moves one contiguous, fully coalesced run of 8- or 16-byte
// records; a block of 256 threads holds floor(256/k) whole pixels, and the
// per-pixel sums over the k intervals (the coupling of v, s and q through the
// operator of Sec. 4) are segmented scans: warp shuffles inside each warp, one
// shared-memory carry for the pixels that straddle a warp boundary.  Halo
// values (p at x-1 and y-1 in the primal step) are re-read from L1/L2.  The
// algorithmic DRAM traffic is (20k + 3) floats per pixel and iteration (+ f).
// On a volume (D > 1, the d = 3 grid of Sec. 4) p_i has a third component,
// kept in its own [N][k] float array pz, and the differences add the next /
// previous slice: (23k + 3) floats per voxel.
#include "lift_bulk.cuh"
#include "lift_device.cuh"
#include "lift_params.h"
#include "lift_tile.cuh"

#include <algorithm>
#include <mutex>

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
// The tile's pixels start at pbase; only those in [p0, p1) are updated.
template <int KIND, int THREADS, bool VOL = false>
__device__ __forceinline__ void dual_tile(const LiftParams &P, const float2 *__restrict__ xbar,
                                          float4 *__restrict__ y, float *__restrict__ q,
                                          int pbase, int p0, int p1, float *s_in, float *s_last,
                                          float *__restrict__ pz = nullptr)
{
    const int tid = threadIdx.x;
    int lp, i;
    split_thread(P, tid, lp, i);
    const int pix = pbase + lp;
    const bool active = lp < P.ppb && pix >= p0 && pix < p1;
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

// The dual step in tiles, one per block (volumes, and sampled costs on
// images, whose hull walks read per-pixel tables that record-per-thread
// tiles read coalesced).  Block b takes the tile starting at tbase + b ppb;
// only the pixels [p0, p1) are updated.  LIVE: a batch member, whose blocks
// return while its live flag is 0.
template <int KIND, bool VOL, bool LIVE>
__global__ void __launch_bounds__(kStepThreads)
dual_step_kernel(const LiftParams P, const float2 *__restrict__ xbar, float4 *__restrict__ y,
                 float *__restrict__ q, float *__restrict__ pz, int tbase, int p0, int p1)
{
    __shared__ float s_in[kStepThreads];
    __shared__ float s_last[kStepThreads / 32];
    if (LIVE && *P.live == 0) return;
    dual_tile<KIND, kStepThreads, VOL>(P, xbar, y, q, tbase + blockIdx.x * P.ppb, p0, p1, s_in,
                                       s_last, pz);
}

// ---------------------------------------------------------------------------
// Dual step of an image in strips.
//
// The pixels are cut into strips of `spp` consecutive pixels, one per CTA.
// One thread stages by bulk (TMA) copies into shared memory the strip's dual
// records y, its extrapolated primal records xbar together with those of the
// pixel after the strip (the x+1 neighbour of its last pixel), and the xbar
// records of the strip one row below (the y+1 neighbours); the finished y goes
// back by one bulk store.  Several CTAs per SM overlap one another's copies.
//
// T threads share a pixel: thread j of a pixel owns the consecutive intervals
// [j c, (j+1) c), c = ceil(k/T), and walks them from the last to the first,
// so the suffix sum sum_{l>i} sbar_l that the v-update needs is a running sum
// in a register, started from the sums of the later threads' intervals (T-1
// shuffles; no scan over the block).  Records that leave the epigraph of
// rho_i^* (a few per cent after the first iterations) are queued per warp;
// whenever 32 are pending the warp projects them together, one per lane, and
// what is left at the end of the strip (fewer than 32 per warp) is pooled
// over the CTA and projected in as few warp passes as it fills, so the
// divergent projection runs on (nearly) full warps.  The arithmetic of a
// record is that of dual_tile; only the order of the sum over sbar differs.
// T depends on k alone, and single problems and batches run one kernel, so a
// problem gets the same result, bit for bit, whatever the strip length, band
// cut or batch it runs in.
// ---------------------------------------------------------------------------

// log2 of the threads per pixel for k intervals.
__host__ __device__ inline int strip_tshift(int k)
{
    return k >= 12 ? 2 : (k >= 6 ? 1 : 0);
}

// Shared memory of a CTA for strips of `spp` pixels with k records each, run
// by `threads` threads: y, then xbar of the strip and the next pixel (one
// float2 of slack in front for a first record that sits 8 bytes past a
// 16-byte boundary, one behind), then xbar of the row below (same slack), then
// the per-interval constants (k float4), one 64-entry projection ring per
// warp and the CTA's pool of left-over entries (32 per warp), each entry 8
// bytes.  `stage` (the three record arrays) is rounded to 128 bytes.
struct StripSmem {
    int x_off, d_off, stage, ic_off, ring_off, pool_off, bytes;
};

__host__ __device__ inline StripSmem strip_smem(int spp, int k, int threads)
{
    StripSmem L;
    int o = spp * k * 16;
    L.x_off = o;
    o += ((spp + 1) * k + 2) * 8;
    o = (o + 15) & ~15;
    L.d_off = o;
    o += (spp * k + 2) * 8;
    L.stage = (o + 127) & ~127;
    L.ic_off = L.stage;
    L.ring_off = L.ic_off + k * 16;
    L.pool_off = L.ring_off + (threads / 32) * 64 * 8;
    L.bytes = L.pool_off + (threads / 32) * 32 * 8;
    return L;
}

// Records [a, e) of xbar into shared memory, dst[r - a] = record r.  The
// 16-byte aligned middle part moves by one bulk copy: dst starts 8 bytes past
// a 16-byte boundary exactly when record a does in global memory, so aligned
// records land on aligned shared addresses.  A first record that sits 8 bytes
// past a boundary and a last record that starts on one (an 8-byte tail) are
// plain loads.
// L2 prefetch of the 16-byte aligned part of the floats [p, p + n).
__device__ __forceinline__ void prefetch_l2_aligned(const float *p, int n)
{
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
    const uintptr_t e = reinterpret_cast<uintptr_t>(p + n) & ~uintptr_t(15);
    if (e > a) bulk_prefetch_l2(reinterpret_cast<const void *>(a), static_cast<uint32_t>(e - a));
}

struct XRange {
    int a, e, s, e2;   // range, and its bulk part [s, e2) (empty if e2 <= s)
    int ph;            // 1: record a sits 8 bytes past a 16-byte boundary
};

__device__ __forceinline__ XRange x_range(const float2 *xbar, int a, int e)
{
    XRange R;
    R.a = a;
    R.e = e;
    R.ph = static_cast<int>((reinterpret_cast<uintptr_t>(xbar + a) >> 3) & 1);
    R.s = a + R.ph;
    R.e2 = e - static_cast<int>((reinterpret_cast<uintptr_t>(xbar + e) >> 3) & 1);
    return R;
}

__device__ __forceinline__ void x_ragged(const XRange &R, const float2 *__restrict__ xbar,
                                         float2 *dst)
{
    const int s_end = R.s < R.e ? R.s : R.e;
    for (int r = R.a; r < s_end; ++r) dst[r - R.a] = xbar[r];
    int b = R.e2 > R.s ? R.e2 : R.s;
    if (b < R.a) b = R.a;
    for (int r = b; r < R.e; ++r) dst[r - R.a] = xbar[r];
}

// Projection of one queued record onto Delta * epi(rho_i^*), written back into
// the staged y.  e = {record index r in the strip | pixel t in the strip << 16,
// f of the pixel (the quadratic kinds)}; the record holds the unscaled point
// (y0, h0) = (v, z) / Delta until then; sIC: the staged per-interval constants.  Not inlined:
// every record below the graph goes through this one compiled body, whichever
// warp pass (or kernel) handles it, so its result does not depend on how the
// records fall into passes.  Pp: the parameters, in shared memory.
template <int KIND>
__device__ __noinline__ void strip_project(const LiftParams *Pp, float4 *sY, const float4 *sIC,
                                           int pix0, int2 e)
{
    const LiftParams &P = *Pp;
    const int r = e.x & 0xffff, pp = pix0 + (e.x >> 16);
    const int i = r - (pp - pix0) * P.k;
    float2 *rec = reinterpret_cast<float2 *>(sY + r);
    const float2 p0 = rec[0];
    const float l = sIC[i].x;
    float yo, ho;
    if (KIND == 2) {
        piece_project_below<2>(P, pp, i, l, p0.x, p0.y, yo, ho);
    } else {
        const QPiece qp = make_qpiece_f(P, __int_as_float(e.y), l, l + P.delta);
        qpiece_project(qp, p0.x, p0.y, yo, ho);
    }
    rec[0] = make_float2(P.delta * yo, P.delta * ho);
}

// The dual update of one staged record r (interval i of pixel pix) from its
// xbar record xb and tail = sum of sbar over the pixel's later intervals:
// TV dual ascent and ball (or box) projection of p_i; ascent of (v_i, z_i).
// Writes the record back and returns whether (v, z)/Delta lies below the
// graph of rho_i^* (then the record keeps the unscaled point for the
// projection; else it holds the final Delta (y0, h0)).
template <int KIND>
__device__ __forceinline__ bool strip_record(const LiftParams &P, float4 *sY, const float2 *sX,
                                             const float2 *sD, const float4 *sIC, int r, int i,
                                             int pix, float fv, float2 xb, bool hasR, bool hasD,
                                             float sigma_p, float tail)
{
    const int k = P.k;
    const float4 ic = sIC[i];                  // {gamma_i, tau_s, sigma_vz, lambda*Delta}
    const float4 d = sY[r];
    // TV dual: forward differences (Neumann), ascent, ball (or box) projection
    const float gx = hasR ? sX[r + k].x - xb.x : 0.0f;
    const float gy = hasD ? sD[r].x - xb.x : 0.0f;
    float px = d.z + sigma_p * gx;
    float py = d.w + sigma_p * gy;
    if (P.aniso) {
        px = fminf(fmaxf(px, -ic.w), ic.w);
        py = fminf(fmaxf(py, -ic.w), ic.w);
    } else {
        const float n2 = px * px + py * py;
        if (n2 > ic.w * ic.w) {
            const float sc2 = ic.w * rsqrtf(n2);
            px *= sc2;
            py *= sc2;
        }
    }
    const float v = d.x + ic.z * (xb.x + P.delta * tail - ic.x * xb.y);
    const float z = d.y + ic.z * xb.y;
    const float y0 = v * P.inv_delta, h0 = z * P.inv_delta;
    const bool below = KIND == 2 ? !piece_in_epigraph<2>(P, pix, i, ic.x, y0, h0)
                                 : !(h0 >= quad_conj_direct(P, fv, ic.x, ic.x + P.delta, y0));
    sY[r] = below ? make_float4(y0, h0, px, py)
                  : make_float4(P.delta * y0, P.delta * h0, px, py);
    return below;
}

// A warp's ring of queued records: entries [head, head + cnt) (mod 64), each
// {record | pixel in the strip << 16, f of the pixel} (records and pixels of
// a strip fit in 16 bits: at most 256 pixels and 64 intervals).
struct StripRing {
    int2 *e;
    int head, cnt;
};

// Queue this lane's record (if below) and run a warp pass of the projection
// whenever 32 are pending.
template <int KIND>
__device__ __forceinline__ void strip_queue(StripRing &R, bool below, int r, int pix, float fv,
                                            int lane, const LiftParams *sP, float4 *sY,
                                            const float4 *sIC, int pix0)
{
    const unsigned m = __ballot_sync(0xffffffffu, below);
    if (below)
        R.e[(R.head + R.cnt + __popc(m & ((1u << lane) - 1u))) & 63] =
            make_int2(r | ((pix - pix0) << 16), __float_as_int(fv));
    R.cnt += __popc(m);
    if (R.cnt >= 32) {
        __syncwarp();
        strip_project<KIND>(sP, sY, sIC, pix0, R.e[(R.head + lane) & 63]);
        R.head = (R.head + 32) & 63;
        R.cnt -= 32;
        __syncwarp();
    }
}

// This thread's share of a pixel: the C intervals [lo, lo + C) clipped to k
// (C a compile-time length, so the records' loads and arithmetic interleave).
// Returns the sum of sbar over the pixel's intervals from lo on (plus the
// later threads' sums, which it adds first).
template <int KIND, int C>
__device__ __forceinline__ float strip_chunk(const LiftParams &P, const LiftParams *sP, float4 *sY,
                                             const float2 *sX, const float2 *sD,
                                             const float4 *sIC, StripRing &R,
                                             int pix0, int t, int lo, int tshift, bool act,
                                             bool hasR, bool hasD, float fv, float sigma_p,
                                             int lane)
{
    const int k = P.k, pix = pix0 + t;
    float2 xb[C];
    float own = 0.0f;
#pragma unroll
    for (int it = 0; it < C; ++it) {
        const bool ok = act && lo + it < k;
        xb[it] = ok ? sX[t * k + lo + it] : make_float2(0.0f, 0.0f);
        own += xb[it].y;
    }
    // sum of sbar over the intervals of the later threads of this pixel
    float tail = 0.0f;
    const int ppw = 32 >> tshift, T = 1 << tshift, j = lane >> (5 - tshift);
    for (int d = 1; d < T; ++d) {
        const float o = __shfl_down_sync(0xffffffffu, own, d * ppw);
        if (j + d < T) tail += o;
    }
    bool below[C];
#pragma unroll
    for (int it = C - 1; it >= 0; --it) {
        const int i = lo + it;
        below[it] = false;
        if (act && i < k)
            below[it] = strip_record<KIND>(P, sY, sX, sD, sIC, t * k + i, i, pix, fv, xb[it],
                                           hasR, hasD, sigma_p, tail);
        tail += xb[it].y;
    }
#pragma unroll
    for (int it = C - 1; it >= 0; --it)
        strip_queue<KIND>(R, below[it], t * k + lo + it, pix, fv, lane, sP, sY, sIC, pix0);
    return tail;
}

// The same for chunks longer than 8 (k > 32 with four threads per pixel), in
// a loop.
template <int KIND>
__device__ __forceinline__ float strip_chunk_any(const LiftParams &P, const LiftParams *sP,
                                                 float4 *sY, const float2 *sX, const float2 *sD,
                                                 const float4 *sIC, StripRing &R, int pix0, int t, int lo, int c,
                                                 int tshift, bool act, bool hasR, bool hasD,
                                                 float fv, float sigma_p, int lane)
{
    const int k = P.k, pix = pix0 + t;
    float own = 0.0f;
    for (int it = 0; it < c; ++it)
        if (act && lo + it < k) own += sX[t * k + lo + it].y;
    float tail = 0.0f;
    const int ppw = 32 >> tshift, T = 1 << tshift, j = lane >> (5 - tshift);
    for (int d = 1; d < T; ++d) {
        const float o = __shfl_down_sync(0xffffffffu, own, d * ppw);
        if (j + d < T) tail += o;
    }
    for (int it = c - 1; it >= 0; --it) {
        const int i = lo + it;
        bool below = false;
        if (act && i < k) {
            const float2 xb = sX[t * k + i];
            below = strip_record<KIND>(P, sY, sX, sD, sIC, t * k + i, i, pix, fv, xb, hasR,
                                       hasD, sigma_p, tail);
            tail += xb.y;
        }
        strip_queue<KIND>(R, below, t * k + i, pix, fv, lane, sP, sY, sIC, pix0);
    }
    return tail;
}

// One strip per CTA, of a single problem (D == nullptr: the parameters P1 and
// state pointers given, the pixels [p0, p1) in strips of blockDim.x / T) or of
// a batch (strip blockIdx.x belongs to instance strip_inst[blockIdx.x], whose
// descriptor is D[...]; strips of instances whose live flag is 0 return).
// A single problem reads y1, q1 and writes the updated y, q to yout1, qout1:
// the same arrays for the solver's in-place step, the next stored state's for
// the recomputation of the unrolled solve (the arithmetic is the same).
template <int KIND>
__global__ void __launch_bounds__(256, 4)
dual_strip_kernel(const LiftParams P1, const float2 *__restrict__ xbar1, const float4 *y1,
                  const float *__restrict__ q1, float4 *yout1, float *qout1, int p0, int p1,
                  const InstDesc *__restrict__ D, const int *__restrict__ strip_inst,
                  const int *__restrict__ live, int *err, int ahead)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ LiftParams sP;
    __shared__ int s_pool;
    __shared__ __align__(8) uint64_t s_bar;   // completes when the strip's copies land
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the problem's parameters in registers (the loop below reads them
    // there) and, for the projections, in shared memory
    LiftParams P;
    const float2 *xbar;
    const float4 *y;
    const float *q;
    float4 *yout;
    float *qout;
    int s;
    if (D == nullptr) {
        if (P1.live && *P1.live == 0) return;
        P = P1;
        xbar = xbar1;
        y = y1;
        q = q1;
        yout = yout1;
        qout = qout1;
        s = blockIdx.x;
    } else {
        const int inst = strip_inst[blockIdx.x];
        if (!live[inst]) return;
        P = D[inst].P;
        xbar = D[inst].S.xbar;
        yout = D[inst].S.y;
        qout = D[inst].S.q;
        y = yout;
        q = qout;
        s = blockIdx.x - D[inst].strip0;
        p0 = 0;
        p1 = P.N;
    }
    if (tid == 0) {
        sP = P;
        s_pool = 0;
        mbar_init(&s_bar, 1);                 // initialised before any thread waits on it
    }
    __syncthreads();
    const int k = P.k;
    const int tshift = strip_tshift(k);
    const int spp = blockDim.x >> tshift;
    const StripSmem L = strip_smem(spp, k, blockDim.x);
    float4 *sIC = reinterpret_cast<float4 *>(smem + L.ic_off);
    int2 *sRing = reinterpret_cast<int2 *>(smem + L.ring_off) + warp * 64;
    int2 *sPool = reinterpret_cast<int2 *>(smem + L.pool_off);
    uint64_t *bar = &s_bar;

    // where the strip lies (record indices fit in int: N*k < 2^31; pixels are
    // clipped to N first)
    auto clip = [&](long long p) { return static_cast<int>(p < P.N ? p : P.N); };
    const int pix0 = p0 + s * spp;
    const int n = min(spp, p1 - pix0);
    const int ya = pix0 * k;
    const XRange RX = x_range(xbar, ya, clip(pix0 + n + 1LL) * k);
    const XRange RD = x_range(xbar, clip(static_cast<long long>(pix0) + P.W) * k,
                              clip(static_cast<long long>(pix0) + P.W + n) * k);
    float4 *sY = reinterpret_cast<float4 *>(smem);
    float2 *sX = reinterpret_cast<float2 *>(smem + L.x_off) + RX.ph;   // sX[r - RX.a]
    float2 *sD = reinterpret_cast<float2 *>(smem + L.d_off) + RD.ph;   // sD[r - RD.a]

    if (tid == 0) {
        const uint32_t yb = static_cast<uint32_t>(n) * k * 16;
        uint32_t tx = yb + k * 16;
        if (RX.e2 > RX.s) tx += (RX.e2 - RX.s) * 8;
        if (RD.e2 > RD.s) tx += (RD.e2 - RD.s) * 8;
        mbar_arrive_expect_tx(bar, tx);
        bulk_load(sY, y + ya, yb, bar);
        if (RX.e2 > RX.s) bulk_load(sX + (RX.s - RX.a), xbar + RX.s, (RX.e2 - RX.s) * 8, bar);
        if (RD.e2 > RD.s) bulk_load(sD + (RD.s - RD.a), xbar + RD.s, (RD.e2 - RD.s) * 8, bar);
        bulk_load(sIC, P.icst, k * 16, bar);
        // the strip that the CTA taking this one's place `ahead` launches
        // later will stage: its y and xbar into L2 now
        const int s2 = s + ahead;
        if (ahead > 0 && p0 + static_cast<long long>(s2) * spp < p1) {
            const int q0 = p0 + s2 * spp, nq = min(spp, p1 - q0);
            bulk_prefetch_l2(y + q0 * k, static_cast<uint32_t>(nq) * k * 16);
            const XRange RQ = x_range(xbar, q0 * k, clip(q0 + nq + 1LL) * k);
            if (RQ.e2 > RQ.s) bulk_prefetch_l2(xbar + RQ.s, (RQ.e2 - RQ.s) * 8);
            // and its f and q, read with plain loads once the copies land
            // (the 16-byte aligned part of each run)
            if (KIND != 2) prefetch_l2_aligned(P.f + q0, nq);
            prefetch_l2_aligned(q + q0, nq);
        }
    } else if (tid == (blockDim.x > 32 ? 32 : 1)) {   // another warp if there is one
        x_ragged(RX, xbar, sX);
        x_ragged(RD, xbar, sD);
    }

    // this thread: pixel t of the strip (pixels fastest within a warp), and
    // its share j of the pixel's intervals, [lo, lo + c) clipped to k
    const int ppw = 32 >> tshift;
    const int t = warp * ppw + (lane & (ppw - 1));
    const int j = lane >> (5 - tshift);
    const int T = 1 << tshift;
    const int c = (k + T - 1) >> tshift;
    const int lo = j * c;
    const bool act = t < n;
    const int pix = pix0 + t;
    int row = 0, col = 0;
    float fv = 0.0f, qo = 0.0f;
    if (act) {                                 // values that need no staging,
        row = pixel_row(P, pix);               // loaded while the copies fly
        col = pix - row * P.W;
        if (KIND != 2) fv = __ldg(P.f + pix);
        if (j == 0) qo = q[pix];
    }
    const bool hasR = act && col + 1 < P.W, hasD = act && row + 1 < P.H;
    const float4 stp = __ldg(P.steps);         // {tau_u, sigma_q, sigma_p, 0}
    // the copies have landed (and, by the barrier, the plain-loaded records
    // are visible); if any thread's bounded wait gave up, the CTA records the
    // error and leaves
    const bool landed = mbar_wait(bar, 0);
    if (__syncthreads_or(!landed)) {
        if (tid == 0 && err) atomicOr(err, 1);
        return;
    }

    StripRing R{sRing, 0, 0};
    constexpr int PK = KIND == 2 ? 2 : 0;
    float tail;
    switch (c) {
    case 1: tail = strip_chunk<PK, 1>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 2: tail = strip_chunk<PK, 2>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 3: tail = strip_chunk<PK, 3>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 4: tail = strip_chunk<PK, 4>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 5: tail = strip_chunk<PK, 5>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 6: tail = strip_chunk<PK, 6>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 7: tail = strip_chunk<PK, 7>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 8: tail = strip_chunk<PK, 8>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 9: tail = strip_chunk<PK, 9>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    case 10: tail = strip_chunk<PK, 10>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, tshift, act, hasR, hasD, fv, stp.z, lane); break;
    default:
        tail = strip_chunk_any<PK>(P, &sP, sY, sX, sD, sIC, R, pix0, t, lo, c, tshift, act, hasR, hasD, fv,
                                   stp.z, lane);
    }
    // thread 0 of the pixel ends with the sum of sbar over all intervals
    if (act && j == 0) qout[pix] = qo - stp.y * (1.0f + P.delta * tail);

    // the warps' left-overs (fewer than 32 each) into the CTA's pool, then
    // projected in passes of 32 spread over the warps
    int base = 0;
    if (lane == 0 && R.cnt > 0) base = atomicAdd(&s_pool, R.cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lane < R.cnt) sPool[base + lane] = sRing[(R.head + lane) & 63];
    __syncthreads();
    const int pooled = s_pool;
    for (int e0 = warp * 32; e0 < pooled; e0 += blockDim.x)
        if (e0 + lane < pooled) strip_project<PK>(&sP, sY, sIC, pix0, sPool[e0 + lane]);

    fence_proxy_async_smem();                  // the records written above ...
    __syncthreads();
    if (tid == 0) {                            // ... go back by one bulk store
        bulk_store(yout + ya, sY, static_cast<uint32_t>(n) * k * 16);
        bulk_store_commit();
        bulk_wait_read();                      // the shared memory may then go
    }
}

// Single-instance primal step: each block takes two consecutive tiles and
// issues the loads of both before the (shared) scan, doubling the bytes in
// flight per thread; the primal step waits on memory rather than on issue.
// On images the neighbours' p (x-1, y-1) and q are loaded before the scan's
// barrier too, so their latency overlaps it (37.3 -> 34.9 us per launch at
// 512^2, L = 20, same registers; on a volume that took 40 -> 46 registers
// and one block per SM, 117 -> 129 us at 128^3, L = 8, so volumes load them
// after the scan).
// The pixels [p0, p1); block b takes the tiles starting at tbase + 2b ppb
// and tbase + (2b + 1) ppb (tbase <= p0; pixels before p0 are idle).
// ahead > 0 (images): thread 0 also prefetches into L2 the records of block
// blockIdx.x + ahead, the block that takes this one's place on the SM.
// x_out: where the new x goes (x itself for the solver's in-place step, the
// next stored state's x for the recomputation of the unrolled solve).
template <bool VOL, bool LIVE>
__global__ void __launch_bounds__(kStepThreads)
primal_step_kernel(const LiftParams P, float2 *__restrict__ x, float2 *x_out,
                   float2 *__restrict__ xbar,
                   const float4 *__restrict__ y, const float *__restrict__ q,
                   const float *__restrict__ pz, int tbase, int p0, int p1, int ahead)
{
    __shared__ float2 s_in[kStepThreads];
    __shared__ float2 s_last[kStepThreads / 32];
    if (LIVE && *P.live == 0) return;
    const int tid = threadIdx.x;
    if (!VOL && ahead > 0 && tid == 0) {
        const long long b0 = tbase + 2LL * (blockIdx.x + ahead) * P.ppb;
        const long long a = b0 > p0 ? b0 : p0;
        const long long e = b0 + 2LL * P.ppb < p1 ? b0 + 2LL * P.ppb : p1;
        if (a < e) {
            bulk_prefetch_l2(y + a * P.k, static_cast<uint32_t>((e - a) * P.k * 16));
            // the x records' 16-byte aligned part
            const uintptr_t xa = (reinterpret_cast<uintptr_t>(x + a * P.k) + 15) & ~uintptr_t(15);
            const uintptr_t xe = reinterpret_cast<uintptr_t>(x + e * P.k) & ~uintptr_t(15);
            if (xe > xa)
                bulk_prefetch_l2(reinterpret_cast<const void *>(xa), static_cast<uint32_t>(xe - xa));
            prefetch_l2_aligned(q + a, static_cast<int>(e - a));
        }
    }
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
        pix[u] = tbase + (2 * blockIdx.x + u) * P.ppb + lp;
        act[u] = lp < P.ppb && pix[u] >= p0 && pix[u] < p1;
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
        x_out[o[u]] = make_float2(un, sn);
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

// Batches hold quadratic-type images only; their dual step runs in strips
// (batch_dual_strip_kernel above), their primal step in tiles here.
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

// Per device: the SM count, and per strip-kernel shape the CTAs that fit on
// an SM at once, with the kernel's dynamic shared-memory limit raised to
// what the shape needs.  Looked up once per (device, kernel, shape) and kept,
// so a launch costs no device queries (direct launches of small problems are
// host-bound otherwise).
constexpr int kStripSmemCap = 200 * 1024;   // above every strip shape's need

struct StripOcc {
    int dev = -1, kind = -1, threads = 0, bytes = 0, per_sm = 0, sms = 0;
};

template <int KIND>
static cudaError_t strip_occupancy(int threads, int bytes, int *ctas)
{
    static std::mutex mu;
    static StripOcc cache[32];
    static int next = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const StripOcc &c : cache)
            if (c.dev == dev && c.kind == KIND && c.threads == threads && c.bytes == bytes) {
                *ctas = c.per_sm * c.sms;
                return cudaSuccess;
            }
    }
    StripOcc c;
    c.dev = dev;
    c.kind = KIND;
    c.threads = threads;
    c.bytes = bytes;
    e = cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
    // one cap for every shape (each launch still asks for its own bytes): a
    // cap set to one shape's size would refuse a larger shape cached earlier
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(dual_strip_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kStripSmemCap);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.per_sm, dual_strip_kernel<KIND>,
                                                          threads, bytes);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    cache[next] = c;
    next = (next + 1) % 32;
    *ctas = c.per_sm * c.sms;
    return cudaSuccess;
}

template <int THREADS>
static cudaError_t launch_batch_primal(const InstDesc *D, const int *tile_inst, const int *live,
                                       int ntiles, cudaStream_t st)
{
    batch_primal_kernel<THREADS><<<ntiles, THREADS, 0, st>>>(D, tile_inst, live);
    return cudaGetLastError();
}

cudaError_t launch_batch_iteration(int threads, const InstDesc *D, const int *tile_inst,
                                   const int *live, int ntiles, const StripGroup *groups,
                                   int ngroups, int *err, cudaStream_t st)
{
    if (ntiles <= 0) return cudaSuccess;
    for (int g = 0; g < ngroups; ++g) {
        const StripGroup &G = groups[g];
        if (G.nstrips <= 0) continue;
        if (G.bytes > kStripSmemCap) return cudaErrorInvalidValue;
        int resident = 0;
        cudaError_t e = strip_occupancy<0>(G.threads, G.bytes, &resident);
        if (e != cudaSuccess) return e;
        LiftParams none{};
        dual_strip_kernel<0><<<G.nstrips, G.threads, G.bytes, st>>>(
            none, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, D, G.strip_inst, live, err, 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    switch (threads) {
    case 128: return launch_batch_primal<128>(D, tile_inst, live, ntiles, st);
    case 256: return launch_batch_primal<256>(D, tile_inst, live, ntiles, st);
    case 512: return launch_batch_primal<512>(D, tile_inst, live, ntiles, st);
    default: return cudaErrorInvalidValue;
    }
}


static inline int step_blocks(const LiftParams &P)
{
    return (P.N + P.ppb - 1) / P.ppb;
}

// Pixels per strip for k records per pixel on a single problem: 256 / T
// threads' worth, fewer (in steps of one warp's pixels, down to one warp)
// while the staged records exceed kStripStage bytes.
constexpr int kStripStage = 20 * 1024;

static int strip_spp(int k)
{
    const int ts = strip_tshift(k), step = 32 >> ts;
    int spp = 256 >> ts;
    while (spp > step && strip_smem(spp, k, spp << ts).stage > kStripStage) spp -= step;
    return spp;
}

void strip_shape_of(int k, int *threads, int *bytes, int *pixels)
{
    const int spp = strip_spp(k);
    *pixels = spp;
    *threads = spp << strip_tshift(k);
    *bytes = strip_smem(spp, k, *threads).bytes;
}

// The dual step of the pixels [p0, p1) in strips: reads S, writes y and q to
// yout, qout (S.y, S.q for the in-place step).
template <int KIND>
static cudaError_t launch_strips(const LiftParams &P, const LiftState &S, int p0, int p1,
                                 cudaStream_t st, float4 *yout = nullptr, float *qout = nullptr)
{
    const int spp = strip_spp(P.k);
    const int nstrips = (p1 - p0 + spp - 1) / spp;
    if (nstrips <= 0) return cudaSuccess;
    const int threads = spp << strip_tshift(P.k);
    const int bytes = strip_smem(spp, P.k, threads).bytes;
    if (bytes > kStripSmemCap) return cudaErrorInvalidValue;
    // CTAs resident at once: a CTA prefetches the strip of the CTA that will
    // take its place
    int resident = 0;
    const cudaError_t e = strip_occupancy<KIND>(threads, bytes, &resident);
    if (e != cudaSuccess) return e;
    dual_strip_kernel<KIND><<<nstrips, threads, bytes, st>>>(
        P, S.xbar, S.y, S.q, yout ? yout : S.y, qout ? qout : S.q, p0, p1, nullptr, nullptr,
        nullptr, P.err, resident);
    return cudaGetLastError();
}

// Dual half-step in tiles over [p0, p1), tiles aligned to `origin`.
static cudaError_t launch_dual_tiles(const LiftParams &P, const LiftState &S, int p0, int p1,
                                     int origin, cudaStream_t st)
{
    if (p1 <= p0) return cudaSuccess;
    const int r = ((p0 - origin) % P.ppb + P.ppb) % P.ppb;
    const int tbase = p0 - r;
    const int nb = (p1 - tbase + P.ppb - 1) / P.ppb;
    const bool vol = P.D > 1, live = P.live != nullptr;
    if (P.kind == 2) {
        if (vol) dual_step_kernel<2, true, false><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, S.pz, tbase, p0, p1);
        else if (live) dual_step_kernel<2, false, true><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, nullptr, tbase, p0, p1);
        else dual_step_kernel<2, false, false><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, nullptr, tbase, p0, p1);
    } else {
        dual_step_kernel<0, true, false><<<nb, kStepThreads, 0, st>>>(P, S.xbar, S.y, S.q, S.pz, tbase, p0, p1);
    }
    return cudaGetLastError();
}

// Dual half-step on the tiles [t0, t1): quadratic kinds on images in strips
// (the pixels of those tiles), sampled costs and volumes in tiles.
cudaError_t launch_dual_band(const LiftParams &P, const LiftState &S, int t0, int t1,
                             cudaStream_t st)
{
    const int p0 = t0 * P.ppb;
    const int p1 = static_cast<int>(std::min<long long>(static_cast<long long>(t1) * P.ppb, P.N));
    if (P.D == 1 && P.kind != 2) return launch_strips<0>(P, S, p0, p1, st);
    return launch_dual_tiles(P, S, p0, p1, 0, st);
}

// Primal half-step on the tiles [t0, t1) (two tiles per block).
// Blocks of the image primal kernel resident on the current device at once
// (the same for LIVE true and false), looked up once per device.
static cudaError_t primal_resident(int *ctas)
{
    static std::mutex mu;
    static int known[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) { *ctas = 0; return cudaSuccess; }
    std::lock_guard<std::mutex> lock(mu);
    if (known[dev] == 0) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, primal_step_kernel<false, false>,
                                                          kStepThreads, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        known[dev] = per_sm * sms > 0 ? per_sm * sms : -1;
    }
    *ctas = known[dev] > 0 ? known[dev] : 0;
    return cudaSuccess;
}

cudaError_t launch_primal_band(const LiftParams &P, const LiftState &S, int t0, int t1,
                               cudaStream_t st)
{
    const int p1 = static_cast<int>(std::min<long long>(static_cast<long long>(t1) * P.ppb, P.N));
    return launch_primal_range(P, S, t0 * P.ppb, p1, 0, st);
}

cudaError_t launch_primal_range(const LiftParams &P, const LiftState &S, int p0, int p1,
                                int origin, cudaStream_t st)
{
    if (p1 <= p0) return cudaSuccess;
    // the first tile: the largest start <= p0 congruent to origin
    const int r = ((p0 - origin) % P.ppb + P.ppb) % P.ppb;
    const int tbase = p0 - r;
    const int nb = (p1 - tbase + 2 * P.ppb - 1) / (2 * P.ppb);
    if (P.D > 1) {
        primal_step_kernel<true, false><<<nb, kStepThreads, 0, st>>>(P, S.x, S.x, S.xbar, S.y, S.q,
                                                                     S.pz, tbase, p0, p1, 0);
        return cudaGetLastError();
    }
    int ahead = 0;
    const cudaError_t e = primal_resident(&ahead);
    if (e != cudaSuccess) return e;
    if (P.live != nullptr)
        primal_step_kernel<false, true><<<nb, kStepThreads, 0, st>>>(P, S.x, S.x, S.xbar, S.y, S.q,
                                                                     nullptr, tbase, p0, p1, ahead);
    else
        primal_step_kernel<false, false><<<nb, kStepThreads, 0, st>>>(P, S.x, S.x, S.xbar, S.y, S.q,
                                                                      nullptr, tbase, p0, p1, ahead);
    return cudaGetLastError();
}

// One iteration from the state Sin into the state Sout (images, quadratic
// kinds): the dual step reads Sin's xbar, y, q and writes Sout's y, q; the
// primal step reads Sin's x and Sout's y, q and writes Sout's x, xbar.  The
// same kernels and arithmetic as the in-place iteration, so the result is
// bitwise the same; Sin is left unchanged.
cudaError_t launch_iteration_into(const LiftParams &P, const LiftState &Sin, const LiftState &Sout,
                                  cudaStream_t st)
{
    if (P.D != 1 || P.kind == 2 || P.live != nullptr) return cudaErrorInvalidValue;
    cudaError_t e = launch_strips<0>(P, Sin, 0, P.N, st, Sout.y, Sout.q);
    if (e != cudaSuccess) return e;
    const int nb = (P.N + 2 * P.ppb - 1) / (2 * P.ppb);
    int ahead = 0;
    e = primal_resident(&ahead);
    if (e != cudaSuccess) return e;
    primal_step_kernel<false, false><<<nb, kStepThreads, 0, st>>>(P, Sin.x, Sout.x, Sout.xbar, Sout.y,
                                                                  Sout.q, nullptr, 0, 0, P.N, ahead);
    return cudaGetLastError();
}

cudaError_t launch_dual_range(const LiftParams &P, const LiftState &S, int p0, int p1,
                              int origin, cudaStream_t st)
{
    if (P.D != 1) return cudaErrorInvalidValue;     // images only
    if (p1 <= p0) return cudaSuccess;
    if (P.kind != 2) return launch_strips<0>(P, S, p0, p1, st);
    return launch_dual_tiles(P, S, p0, p1, origin, st);
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
