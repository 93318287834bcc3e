// Reverse mode through the unrolled primal-dual iteration (the differentiable
// solve): given the adjoint of the state after iteration n+1, produce the
// adjoint of the state after iteration n and accumulate the gradients with
// respect to the data f, lambda, alpha and nu.  Not part of the paper; it
// differentiates the map of pdhg_step.cu (Sec. 4) exactly, including the
// clamp of u, the l2-ball projection (Prop. 5) and the epigraph projections
// (Fig. 7), whose local Jacobians are written out per branch of the
// projection (ray, kink, parabola arc), with the envelope's dependence on the
// data-term parameters taken from forward-mode dual numbers (lift_ad.cuh).
//
// With x = (u, s), xbar, y = (v, z, px, py), q and adjoints ax, axb, ay, aq,
// one reverse iteration is two kernels:
//   adj_primal_local : completes axb.u with the neighbours' part of grad^T
//                      left by the previous reverse iteration (A), then
//                      g_u = [0 < w < 1](ax.u + 2 axb.u), g_s = ax.s + 2 axb.s
//                      (w = the unclamped primal update), ax <- g - axb
//   adj_dual_strip   : completes ay, aq with the primal step's uses of y, q,
//                      then pulls them back through the dual step: the ball
//                      and epigraph projections, the ascent and the sums over
//                      intervals; writes ay, aq, the own part of axb, the
//                      neighbours' part (A), f's gradient and per-CTA sums of
//                      the scalar gradients
// adj_dual_strip runs on strips of pixels like the forward dual step: T
// threads share a pixel, each owning consecutive intervals, so the sums over
// a pixel's intervals are running sums; the records below the graph of
// rho_i^* are pooled over the CTA and their Jacobians computed on full warps.
// Above 8 intervals per thread (k > 32) the record-per-thread form
// (adj_dual_local, then adj_dual_gather) runs instead.
#include "lift_ad.cuh"
#include "lift_device.cuh"
#include "lift_params.h"

namespace lift {

namespace {

constexpr int kAdjThreads = kStepThreads;

__device__ __forceinline__ void split_thread_adj(const LiftParams &P, int tid, int &lp, int &i)
{
    lp = __float2int_rz((static_cast<float>(tid) + 0.5f) * P.inv_k);
    i = tid - lp * P.k;
}

__device__ __forceinline__ int pixel_row_adj(const LiftParams &P, int pix)
{
    return static_cast<int>((static_cast<unsigned long long>(pix) * P.wmul) >> P.wshift);
}

// Segmented inclusive scan of two values at once over the pixel segments of
// the block (see block_segmented_scan in pdhg_step.cu).  One barrier.
struct Scan2 {
    float2 incl, total;
};

__device__ __forceinline__ Scan2 seg_scan2(float2 val, int seg, int k, int tid, bool active,
                                           float2 *s_in, float2 *s_last)
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
    Scan2 r{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    if (!active) return r;
    float2 c = make_float2(0.0f, 0.0f);
    for (int w = seg >> 5; w < warp; ++w) { c.x += s_last[w].x; c.y += s_last[w].y; }
    r.incl = make_float2(x.x + c.x, x.y + c.y);
    const int e = seg + k - 1, ew = e >> 5;
    float2 ce = make_float2(0.0f, 0.0f);
    for (int w = seg >> 5; w < ew; ++w) { ce.x += s_last[w].x; ce.y += s_last[w].y; }
    r.total = make_float2(s_in[e].x + ce.x, s_in[e].y + ce.y);
    return r;
}

__device__ __forceinline__ float div_p(const LiftParams &P, const float4 *__restrict__ y, size_t o,
                                       int row, int col, float4 d)
{
    // the same expression, in the same order, as the primal step
    float dv = 0.0f;
    if (col + 1 < P.W) dv += d.z;
    if (col > 0) dv -= y[o - P.k].z;
    if (row + 1 < P.H) dv += d.w;
    if (row > 0) dv -= y[o - static_cast<size_t>(P.W) * P.k].w;
    return dv;
}

// The epigraph projection of a record below the graph of rho_i^*, pulled
// back: (y0, h0) = (v^, z^)/Delta, the adjoint (gy, gh) of the projected
// (v', z') = Delta (yo, ho), the pixel's f and the interval's left label l.
// Returns the adjoint of (v^, z^) in (av, az), and Delta times the adjoint's
// derivative with respect to f, alpha and nu in df, dga, dgn.
//
// The branch (ray, kink or arc) is the one the forward step's float code
// takes; its derivative is written out for that branch, with
// L = gy yo + gh ho:
//   ray of slope l:  yo = (y0 + l (h0 + A)) / (1 + l^2), ho = l yo - A, so
//                    with G = (gy + gh l)/(1 + l^2): dL/dy0 = G,
//                    dL/dh0 = G l, dL/dA = G l - gh (the right ray: r, B);
//   kink at m1:      (yo, ho) = (m1, l m1 - A): dL/dm1 = gy + gh l,
//                    dL/dA = -gh (the right kink: m2, r, B);
//   parabola arc:    yo = a d, ho = a d (c + d/2) with d the root of the
//                    cubic F(d) = d^3 + 3c d^2 + (2 + 2c^2 - 2h0/a) d
//                    - 2(c h0 + y0)/a of the stationarity condition, so by
//                    the implicit-function theorem dd = -(dF at fixed d) / F'(d):
//                    with mu = (dL/dd) / F'(d), dL/dy0 = 2 mu / a,
//                    dL/dh0 = 2 mu (d + c)/a, and the partials of F in c and a
//                    (a root clamped to an end of the arc follows that end).
// The piece's own parameters (a, c, A, B, m1, m2, t1, t2) depend on f, alpha
// and nu through the envelope construction of lift_device.cuh, evaluated here
// on dual numbers seeded in those three.
__device__ __forceinline__ void epi_pullback(const LiftParams &P, float y0, float h0, float gy,
                                             float gh, float fv, float l, float &av, float &az,
                                             float &df, float &dga, float &dgn)
{
    using D3 = Dual<3>;
    const float r = l + P.delta;
    const QPiece q = make_qpiece_f(P, fv, l, r);   // the forward step's float piece
    av = gy;
    az = gh;
    df = dga = dgn = 0.0f;
    if (h0 >= qpiece_conj(q, y0)) return;           // in the epigraph: identity
    // adjoints of the piece's parameters
    float La = 0.0f, Lc = 0.0f, LA = 0.0f, LB = 0.0f, Lm1 = 0.0f, Lm2 = 0.0f, Lt1 = 0.0f,
          Lt2 = 0.0f;
    const float ph1 = q.l * q.m1 - q.A;
    const float e1 = fmaxf(ph1 - h0, 0.0f);
    const float ph2 = q.r * q.m2 - q.B;
    const float e2 = fmaxf(ph2 - h0, 0.0f);
    if (q.m1 - y0 + e1 * q.l > 0.0f) {              // left ray
        const float G = (gy + gh * q.l) / (1.0f + q.l * q.l);
        av = G;
        az = G * q.l;
        LA = G * q.l - gh;
    } else if (q.m2 - y0 + e2 * q.r < 0.0f) {       // right ray
        const float G = (gy + gh * q.r) / (1.0f + q.r * q.r);
        av = G;
        az = G * q.r;
        LB = G * q.r - gh;
    } else if (!q.arc || q.m1 - y0 + e1 * q.t1 >= 0.0f) {   // left kink
        av = az = 0.0f;
        Lm1 = gy + gh * q.l;
        LA = -gh;
    } else if (q.m2 - y0 + e2 * q.t2 <= 0.0f) {     // right kink
        av = az = 0.0f;
        Lm2 = gy + gh * q.r;
        LB = -gh;
    } else {                                        // parabola arc
        const float ia = 1.0f / q.a;
        const float p = 2.0f - q.c * q.c - 2.0f * h0 * ia;
        const float qq = -2.0f * (q.c + y0 * ia);
        const float sg = qq <= 0.0f ? 1.0f : -1.0f;
        float w = sg * cubic_outer_root(p, fabsf(qq));
        int wend = 0;                               // 1, 2: w clamped to t1, t2
        if (!(w >= q.t1)) { w = q.t1; wend = 1; }
        if (!(w <= q.t2)) { w = q.t2; wend = 2; }
        float d = w - q.c;
        const float b2 = 3.0f * q.c;
        const float b1 = 2.0f + 2.0f * q.c * q.c - 2.0f * h0 * ia;
        const float b0 = -2.0f * (q.c * h0 + y0) * ia;
        const float F = ((d + b2) * d + b1) * d + b0;
        const float dF = (3.0f * d + 2.0f * b2) * d + b1;
        int dend = -1;                              // -1: no Newton step; 0: interior root
        if (dF > 0.0f) {
            float v = d - F / dF;
            dend = 0;
            if (!(v >= q.t1 - q.c)) { v = q.t1 - q.c; dend = 1; }
            if (!(v <= q.t2 - q.c)) { v = q.t2 - q.c; dend = 2; }
            d = v;
        }
        const float Ld = q.a * (gy + gh * (q.c + d));   // dL/dd
        La = d * (gy + gh * (q.c + 0.5f * d));          // direct dependence on a
        Lc = gh * q.a * d;                               // ... and on c
        av = az = 0.0f;
        if (dend == 0) {
            float Fd = (3.0f * d + 6.0f * q.c) * d + b1;     // F'(d) at the root
            if (!(Fd > 0.0f)) Fd = dF;
            const float mu = Ld / Fd;
            av = 2.0f * mu * ia;
            az = 2.0f * mu * (d + q.c) * ia;
            Lc -= mu * ((3.0f * d + 4.0f * q.c) * d - 2.0f * h0 * ia);
            La -= mu * 2.0f * (h0 * d + q.c * h0 + y0) * ia * ia;
        } else {
            const int end = dend > 0 ? dend : wend;     // d = t - c for the end t
            if (end == 1) Lt1 += Ld;
            if (end == 2) Lt2 += Ld;
            Lc -= Ld;
        }
    }
    // through the envelope construction to (f, alpha, nu)
    QPieceT<D3> Q;
    const D3 f3 = D3::seed(fv, 0), al = D3::seed(P.alpha, 1), nu = D3::seed(P.nu, 2);
    if (P.kind == 3)
        Q = make_quad_piece<D3>(al, f3 + (periodic_center(fv, P.nu, l, r) - fv), l, r);
    else if (P.kind == 0) Q = make_quad_piece<D3>(al, f3, l, r);
    else Q = make_trunc_piece<D3>(al, nu, tsqrt(nu / al), f3, l, r);
    float g[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        g[j] = La * Q.a.d[j] + Lc * Q.c.d[j] + LA * Q.A.d[j] + LB * Q.B.d[j] + Lm1 * Q.m1.d[j] +
               Lm2 * Q.m2.d[j] + Lt1 * Q.t1.d[j] + Lt2 * Q.t2.d[j];
    df = P.delta * g[0];
    dga = P.delta * g[1];
    dgn = P.delta * g[2];
}

}  // namespace

// ---------------------------------------------------------------------------
// A (may be null): the neighbours' part of grad^T from the previous reverse
// iteration's dual kernel, added to axb.u here (the same sum, in the same
// order, as adj_dual_gather).
__global__ void __launch_bounds__(kAdjThreads)
adj_primal_local_kernel(const LiftParams P, const float2 *__restrict__ x_n,
                        const float4 *__restrict__ y_n1, float2 *__restrict__ ax,
                        const float2 *__restrict__ axb, float2 *__restrict__ G,
                        const float2 *__restrict__ A)
{
    int lp, i;
    split_thread_adj(P, threadIdx.x, lp, i);
    const int pix = blockIdx.x * P.ppb + lp;
    if (lp >= P.ppb || pix >= P.N) return;
    const size_t o = static_cast<size_t>(pix) * P.k + i;
    const int row = pixel_row_adj(P, pix), col = pix - row * P.W;
    const float2 xo = x_n[o];
    const float4 d = y_n1[o];
    const float dv = div_p(P, y_n1, o, row, col, d);
    const float w = xo.x - P.tau_u * (d.x - dv);
    const float2 a = ax[o];
    float2 b = axb[o];
    if (A) {
        float add = 0.0f;
        if (col > 0) add += P.sigma_p * A[o - P.k].x;
        if (row > 0) add += P.sigma_p * A[o - static_cast<size_t>(P.W) * P.k].y;
        b.x += add;
    }
    const float gu = (w > 0.0f && w < 1.0f) ? a.x + 2.0f * b.x : 0.0f;
    const float gs = a.y + 2.0f * b.y;
    G[o] = make_float2(gu, gs);
    ax[o] = make_float2(gu - b.x, gs - b.y);
}

// ---------------------------------------------------------------------------
// Four blocks per SM (64 registers).  Records in the epigraph of rho_i^* (the
// forward step's float test) take its identity Jacobian; those below it are
// packed per warp into one pass of the projection's pullback.
template <int KIND>
__global__ void __launch_bounds__(kAdjThreads, 4)
adj_dual_local_kernel(const LiftParams P, const float2 *__restrict__ xbar_n,
                      const float4 *__restrict__ y_n, const float2 *__restrict__ G,
                      float4 *__restrict__ ay, float *__restrict__ aq,
                      float2 *__restrict__ axb, float2 *__restrict__ A,
                      float *__restrict__ gf, double *__restrict__ partial)
{
    __shared__ float2 s_a[kAdjThreads], s_b[kAdjThreads];
    __shared__ float2 s_la[kAdjThreads / 32], s_lb[kAdjThreads / 32];
    __shared__ double red[3][kAdjThreads / 32];
    // per warp: the records below the graph of rho_i^*, packed for the
    // projection's pullback, and its results for their owners
    __shared__ float4 s_qa[kAdjThreads / 32][32];   // {y0, h0, a.x, a.y}
    __shared__ float2 s_qb[kAdjThreads / 32][32];   // {f, gamma_i}
    __shared__ float4 s_qr[kAdjThreads];            // {adj_v, adj_z, df, -} by owner
    __shared__ unsigned char s_qo[kAdjThreads / 32][32];   // owner lane of each entry
    const int tid = threadIdx.x;
    int lp, i;
    split_thread_adj(P, tid, lp, i);
    const int pix = blockIdx.x * P.ppb + lp;
    const bool active = lp < P.ppb && pix < P.N;
    const size_t o = static_cast<size_t>(pix) * P.k + i;
    int row = 0, col = 0;
    float4 ic = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float2 g = make_float2(0.0f, 0.0f), xb = make_float2(0.0f, 0.0f);
    float aq_in = 0.0f;
    if (active) {
        row = pixel_row_adj(P, pix);
        col = pix - row * P.W;
        ic = __ldg(P.icst + i);                 // {gamma_i, tau_s, sigma_vz, lambda*Delta}
        g = G[o];
        xb = xbar_n[o];
        aq_in = aq[pix];                        // read before any write of this kernel
    }
    // scan 1: {tau_s g_s} (the primal step's head sums) and {sbar} (the dual
    // step's tail sums)
    const Scan2 s1 = seg_scan2(make_float2(ic.y * g.y, xb.y), lp * P.k, P.k, tid, active, s_a, s_la);

    double gl = 0.0, ga = 0.0, gn = 0.0;
    float2 scan2_val = make_float2(0.0f, 0.0f);
    float adj_v = 0.0f, adj_z = 0.0f, aq_tot = 0.0f, gfi = 0.0f;
    float2 adj_a = make_float2(0.0f, 0.0f);
    float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float y0f = 0.0f, h0f = 0.0f, fpix = 0.0f;
    bool below = false;
    if (active) {
        // --- complete the adjoint of y_{n+1}, q_{n+1} with the primal step's uses
        a = ay[o];
        const float gr = col + 1 < P.W ? G[o + P.k].x : 0.0f;
        const float gd = row + 1 < P.H ? G[o + static_cast<size_t>(P.W) * P.k].x : 0.0f;
        a.x += -P.tau_u * g.x + ic.y * ic.x * g.y - P.delta * (s1.total.x - s1.incl.x);
        a.y += -ic.y * g.y;
        if (col + 1 < P.W) a.z += P.tau_u * (g.x - gr);
        if (row + 1 < P.H) a.w += P.tau_u * (g.x - gd);
        aq_tot = aq_in + P.delta * s1.total.x;

        // --- recompute the dual step's intermediate values (as in the forward)
        const float4 d = y_n[o];
        const float gx = col + 1 < P.W ? xbar_n[o + P.k].x - xb.x : 0.0f;
        const float gy = row + 1 < P.H ? xbar_n[o + static_cast<size_t>(P.W) * P.k].x - xb.x : 0.0f;
        const float px = d.z + P.sigma_p * gx;
        const float py = d.w + P.sigma_p * gy;
        const float n2 = px * px + py * py;
        adj_a = make_float2(a.z, a.w);
        if (P.aniso) {
            // componentwise clamp to [-R, R]: identity inside, the bound outside
            if (fabsf(px) > ic.w) { gl += static_cast<double>(P.delta * copysignf(1.0f, px) * a.z); adj_a.x = 0.0f; }
            if (fabsf(py) > ic.w) { gl += static_cast<double>(P.delta * copysignf(1.0f, py) * a.w); adj_a.y = 0.0f; }
        } else if (n2 > ic.w * ic.w) {
            // p' = R a/|a|: J = (R/|a|)(I - a a^T/|a|^2), dp'/dR = a/|a|, R = lambda Delta
            const float inv = rsqrtf(n2);
            const float hx = px * inv, hy = py * inv;
            const float dot = hx * a.z + hy * a.w;
            adj_a = make_float2(ic.w * inv * (a.z - hx * dot), ic.w * inv * (a.w - hy * dot));
            gl += static_cast<double>(P.delta * dot);
        }
        const float tail = s1.total.y - s1.incl.y;
        const float vh = d.x + ic.z * (xb.x + P.delta * tail - ic.x * xb.y);
        const float zh = d.y + ic.z * xb.y;

        // --- epigraph projection: in the epigraph it is the identity (the
        // forward step's test, in float); below it, its Jacobian with respect
        // to (y0, h0, f, alpha, nu) comes from the packed pass below
        y0f = vh * P.inv_delta;
        h0f = zh * P.inv_delta;
        fpix = __ldg(P.f + pix);
        below = !(h0f >= quad_conj_direct(P, fpix, ic.x, ic.x + P.delta, y0f));
        adj_v = a.x;
        adj_z = a.y;
    }
    {
        // the warp's records below the graph, one per lane of one pass
        const int lane = tid & 31, wq = tid >> 5;
        const unsigned m = __ballot_sync(0xffffffffu, below);
        const int slot = __popc(m & ((1u << lane) - 1u)), nq = __popc(m);
        if (below) {
            s_qa[wq][slot] = make_float4(y0f, h0f, a.x, a.y);
            s_qb[wq][slot] = make_float2(fpix, ic.x);
            s_qo[wq][slot] = static_cast<unsigned char>(lane);
        }
        __syncwarp();
        if (lane < nq) {
            const float4 e = s_qa[wq][lane];
            const float2 eb = s_qb[wq][lane];
            float av, az, df, dga, dgn;
            epi_pullback(P, e.x, e.y, e.z, e.w, eb.x, eb.y, av, az, df, dga, dgn);
            ga += static_cast<double>(dga);
            gn += static_cast<double>(dgn);
            s_qr[(wq << 5) + s_qo[wq][lane]] = make_float4(av, az, df, 0.0f);   // to its owner
        }
        __syncwarp();
        if (below) {
            const float4 rr = s_qr[tid];
            adj_v = rr.x;
            adj_z = rr.y;
            gfi = rr.z;
        }
    }
    if (active) scan2_val = make_float2(ic.z * adj_v, gfi);
    // scan 2: {sigma adj_v^} (pulled back through the tail sums) and f's
    // gradient summed over the pixel's intervals
    const Scan2 s2 = seg_scan2(scan2_val, lp * P.k, P.k, tid, active, s_b, s_lb);
    if (active) {
        ay[o] = make_float4(adj_v, adj_z, adj_a.x, adj_a.y);
        A[o] = adj_a;
        // own part of grad^T (the neighbours' part is gathered afterwards)
        float au = ic.z * adj_v;
        if (col + 1 < P.W) au -= P.sigma_p * adj_a.x;
        if (row + 1 < P.H) au -= P.sigma_p * adj_a.y;
        const float head = s2.incl.x - scan2_val.x;       // sum over l < i of sigma_l adj_v^_l
        const float as = -ic.z * ic.x * adj_v + ic.z * adj_z + P.delta * head -
                         P.sigma_q * P.delta * aq_tot;
        axb[o] = make_float2(au, as);
        if (i == 0) {
            aq[pix] = aq_tot;
            gf[pix] += s2.total.y;
        }
    }
    // per-block sums of the scalar gradients (fixed order), added to the
    // block's own slot: each slot accumulates over the reverse iterations in
    // their order, and one fixed-order pass sums the slots at the end
    for (int off = 16; off > 0; off >>= 1) {
        gl += __shfl_down_sync(0xffffffffu, gl, off);
        ga += __shfl_down_sync(0xffffffffu, ga, off);
        gn += __shfl_down_sync(0xffffffffu, gn, off);
    }
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) { red[0][wid] = gl; red[1][wid] = ga; red[2][wid] = gn; }
    __syncthreads();
    if (tid == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int j = 0; j < kAdjThreads / 32; ++j) { a0 += red[0][j]; a1 += red[1][j]; a2 += red[2][j]; }
        partial[3 * blockIdx.x + 0] += a0;
        partial[3 * blockIdx.x + 1] += a1;
        partial[3 * blockIdx.x + 2] += a2;
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjThreads)
adj_dual_gather_kernel(const LiftParams P, const float2 *__restrict__ A, float2 *__restrict__ axb)
{
    int lp, i;
    split_thread_adj(P, threadIdx.x, lp, i);
    const int pix = blockIdx.x * P.ppb + lp;
    if (lp >= P.ppb || pix >= P.N) return;
    const size_t o = static_cast<size_t>(pix) * P.k + i;
    const int row = pixel_row_adj(P, pix), col = pix - row * P.W;
    float add = 0.0f;
    if (col > 0) add += P.sigma_p * A[o - P.k].x;
    if (row > 0) add += P.sigma_p * A[o - static_cast<size_t>(P.W) * P.k].y;
    axb[o].x += add;
}

// ---------------------------------------------------------------------------
// The reverse dual step on strips of `spp` consecutive pixels, one strip per
// CTA, 2^ts threads per pixel; thread j of a pixel owns the intervals
// [j c, min((j+1) c, k)), c = ceil(k / 2^ts) <= C.  Shared memory: one queue
// slot per record of the strip ({y0, h0, a_v, a_z} and {f, gamma_i}), filled
// with the records below the graph of rho_i^*; after one barrier the CTA's
// threads take the queue in passes of one entry per thread, each entry's
// results written back into its slot for the owner.
constexpr int kAdjMaxChunk = 8;
constexpr int kAdjStripRecords = 1024;

template <int C>
__global__ void __launch_bounds__(256, 4)
adj_dual_strip_kernel(const LiftParams P, int spp, int ts, const float2 *__restrict__ xbar_n,
                      const float4 *__restrict__ y_n, const float2 *__restrict__ G,
                      float4 *__restrict__ ay, float *__restrict__ aq, float2 *__restrict__ axb,
                      float2 *__restrict__ A, float *__restrict__ gf, double *__restrict__ partial)
{
    extern __shared__ float4 adj_smem[];
    __shared__ int s_n;
    __shared__ double red[3][8];
    const int nrec = spp * P.k;
    float4 *s_qa = adj_smem;                                        // [nrec]
    float2 *s_qb = reinterpret_cast<float2 *>(adj_smem + nrec);     // [nrec]
    const int tid = threadIdx.x, T = 1 << ts, k = P.k;
    const int lp = tid >> ts, j = tid & (T - 1);
    const int c = (k + T - 1) >> ts;
    const int pix = blockIdx.x * spp + lp;
    const bool active = lp < spp && pix < P.N;
    const int lo = j * c, hi = min(lo + c, k);
    const size_t ob = static_cast<size_t>(active ? pix : 0) * k;
    int row = 0, col = 0;
    float aq_in = 0.0f, fpix = 0.0f;
    if (active) {
        row = pixel_row_adj(P, pix);
        col = pix - row * P.W;
        aq_in = aq[pix];                        // read before any write of this kernel
        fpix = __ldg(P.f + pix);
    }
    if (tid == 0) s_n = 0;

    // own sums of tau_s g_s and sbar over this thread's intervals
    float2 g[C], xb[C];
    float own_g = 0.0f, own_s = 0.0f;
#pragma unroll
    for (int it = 0; it < C; ++it) {
        const int i = lo + it;
        const bool ok = active && i < hi;
        g[it] = ok ? G[ob + i] : make_float2(0.0f, 0.0f);
        xb[it] = ok ? xbar_n[ob + i] : make_float2(0.0f, 0.0f);
        if (ok) {
            own_g += __ldg(P.icst + i).y * g[it].y;
            own_s += xb[it].y;
        }
    }
    // the later threads' sums of this pixel, and the pixel's total of tau_s g_s
    float later_g = 0.0f, later_s = 0.0f;
    for (int d = 1; d < T; ++d) {
        const float a = __shfl_down_sync(0xffffffffu, own_g, d, T);
        const float b = __shfl_down_sync(0xffffffffu, own_s, d, T);
        if (j + d < T) { later_g += a; later_s += b; }
    }
    const float total_g = __shfl_sync(0xffffffffu, own_g + later_g, 0, T);
    const float aq_tot = aq_in + P.delta * total_g;
    __syncthreads();                            // s_n initialised

    // per record, from the last interval to the first: complete the adjoint
    // of y with the primal step's uses, recompute the dual step's values,
    // pull back through the ball projection; queue the records below the graph
    float av[C], az[C];
    float2 aa[C];
    int slot[C];
    double gl = 0.0, ga = 0.0, gn = 0.0;
    float run_g = later_g, run_s = later_s;
#pragma unroll
    for (int it = C - 1; it >= 0; --it) {
        const int i = lo + it;
        const bool ok = active && i < hi;
        av[it] = 0.0f; az[it] = 0.0f; aa[it] = make_float2(0.0f, 0.0f); slot[it] = -1;
        if (!ok) continue;
        const size_t o = ob + i;
        const float4 ic = __ldg(P.icst + i);    // {gamma_i, tau_s, sigma_vz, lambda Delta}
        const float after_g = run_g, after_s = run_s;   // sums over l > i
        run_g += ic.y * g[it].y;
        run_s += xb[it].y;
        float4 a = ay[o];
        const float gr = col + 1 < P.W ? G[o + k].x : 0.0f;
        const float gd = row + 1 < P.H ? G[o + static_cast<size_t>(P.W) * k].x : 0.0f;
        a.x += -P.tau_u * g[it].x + ic.y * ic.x * g[it].y - P.delta * after_g;
        a.y += -ic.y * g[it].y;
        if (col + 1 < P.W) a.z += P.tau_u * (g[it].x - gr);
        if (row + 1 < P.H) a.w += P.tau_u * (g[it].x - gd);
        const float4 d = y_n[o];
        const float gx = col + 1 < P.W ? xbar_n[o + k].x - xb[it].x : 0.0f;
        const float gy = row + 1 < P.H ? xbar_n[o + static_cast<size_t>(P.W) * k].x - xb[it].x : 0.0f;
        const float px = d.z + P.sigma_p * gx;
        const float py = d.w + P.sigma_p * gy;
        float2 adj_a = make_float2(a.z, a.w);
        if (P.aniso) {
            // componentwise clamp to [-R, R]: identity inside, the bound outside
            if (fabsf(px) > ic.w) { gl += static_cast<double>(P.delta * copysignf(1.0f, px) * a.z); adj_a.x = 0.0f; }
            if (fabsf(py) > ic.w) { gl += static_cast<double>(P.delta * copysignf(1.0f, py) * a.w); adj_a.y = 0.0f; }
        } else {
            const float n2 = px * px + py * py;
            if (n2 > ic.w * ic.w) {
                // p' = R a/|a|: J = (R/|a|)(I - a a^T/|a|^2), dp'/dR = a/|a|, R = lambda Delta
                const float inv = rsqrtf(n2);
                const float hx = px * inv, hy = py * inv;
                const float dot = hx * a.z + hy * a.w;
                adj_a = make_float2(ic.w * inv * (a.z - hx * dot), ic.w * inv * (a.w - hy * dot));
                gl += static_cast<double>(P.delta * dot);
            }
        }
        aa[it] = adj_a;
        const float vh = d.x + ic.z * (xb[it].x + P.delta * after_s - ic.x * xb[it].y);
        const float zh = d.y + ic.z * xb[it].y;
        const float y0f = vh * P.inv_delta, h0f = zh * P.inv_delta;
        av[it] = a.x;
        az[it] = a.y;
        // in the epigraph (the forward step's test, in float) the projection
        // is the identity; below it the pooled pass computes its Jacobian
        if (!(h0f >= quad_conj_direct(P, fpix, ic.x, ic.x + P.delta, y0f))) {
            const int e = atomicAdd(&s_n, 1);
            s_qa[e] = make_float4(y0f, h0f, a.x, a.y);
            s_qb[e] = make_float2(fpix, ic.x);
            slot[it] = e;
        }
    }
    __syncthreads();
    const int nq = s_n;
    for (int e = tid; e < nq; e += blockDim.x) {
        const float4 q = s_qa[e];
        const float2 qb = s_qb[e];
        float rv, rz, df, dga, dgn;
        epi_pullback(P, q.x, q.y, q.z, q.w, qb.x, qb.y, rv, rz, df, dga, dgn);
        s_qa[e] = make_float4(rv, rz, df, dga);
        s_qb[e] = make_float2(dgn, 0.0f);
    }
    __syncthreads();

    // the pulled-back records, f's gradient, and the prefix sums over l < i of
    // sigma_l adj_v_l for the ascent of s
    float gfi = 0.0f, own_v = 0.0f;
#pragma unroll
    for (int it = 0; it < C; ++it) {
        const int i = lo + it;
        if (!(active && i < hi)) continue;
        if (slot[it] >= 0) {
            const float4 r = s_qa[slot[it]];
            av[it] = r.x;
            az[it] = r.y;
            gfi += r.z;
            ga += static_cast<double>(r.w);
            gn += static_cast<double>(s_qb[slot[it]].x);
        }
        own_v += __ldg(P.icst + i).z * av[it];
    }
    float before_v = 0.0f, tot_f = gfi;
    for (int d = 1; d < T; ++d) {
        const float a = __shfl_up_sync(0xffffffffu, own_v, d, T);
        if (j >= d) before_v += a;
    }
    for (int d = 1; d < T; d <<= 1) tot_f += __shfl_xor_sync(0xffffffffu, tot_f, d, T);
    float run_v = before_v;
#pragma unroll
    for (int it = 0; it < C; ++it) {
        const int i = lo + it;
        if (!(active && i < hi)) continue;
        const size_t o = ob + i;
        const float4 ic = __ldg(P.icst + i);
        const float head = run_v;               // sum over l < i of sigma_l adj_v_l
        run_v += ic.z * av[it];
        ay[o] = make_float4(av[it], az[it], aa[it].x, aa[it].y);
        A[o] = aa[it];
        // own part of grad^T (the neighbours' part is added by the next
        // reverse iteration's primal kernel)
        float au = ic.z * av[it];
        if (col + 1 < P.W) au -= P.sigma_p * aa[it].x;
        if (row + 1 < P.H) au -= P.sigma_p * aa[it].y;
        const float as = -ic.z * ic.x * av[it] + ic.z * az[it] + P.delta * head -
                         P.sigma_q * P.delta * aq_tot;
        axb[o] = make_float2(au, as);
    }
    if (active && j == 0) {
        aq[pix] = aq_tot;
        gf[pix] += tot_f;
    }
    // per-CTA sums of the scalar gradients (fixed order) into the CTA's slot
    for (int off = 16; off > 0; off >>= 1) {
        gl += __shfl_down_sync(0xffffffffu, gl, off);
        ga += __shfl_down_sync(0xffffffffu, ga, off);
        gn += __shfl_down_sync(0xffffffffu, gn, off);
    }
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) { red[0][wid] = gl; red[1][wid] = ga; red[2][wid] = gn; }
    __syncthreads();
    if (tid == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) { a0 += red[0][w]; a1 += red[1][w]; a2 += red[2][w]; }
        partial[3 * blockIdx.x + 0] += a0;
        partial[3 * blockIdx.x + 1] += a1;
        partial[3 * blockIdx.x + 2] += a2;
    }
}

// Sum the per-block scalar partials into acc[3] in a fixed order.
__global__ void adj_finish_kernel(const double *__restrict__ partial, int nblocks,
                                  double *__restrict__ acc)
{
    __shared__ double red[3][8];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int j = threadIdx.x; j < nblocks; j += blockDim.x) {
        a += partial[3 * j]; b += partial[3 * j + 1]; c += partial[3 * j + 2];
    }
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
        for (int j = 0; j < static_cast<int>(blockDim.x / 32); ++j) { s0 += red[0][j]; s1 += red[1][j]; s2 += red[2][j]; }
        acc[0] = s0; acc[1] = s1; acc[2] = s2;
    }
}

// Seed: the adjoint of the final state from dL/du~ (u~ = gamma_1 + Delta sum_i u_i).
__global__ void adj_seed_kernel(const LiftParams P, const float *__restrict__ grad_u,
                                float2 *__restrict__ ax)
{
    const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (t >= static_cast<long long>(P.N) * P.k) return;
    const int pix = static_cast<int>(t / P.k);
    ax[t] = make_float2(P.delta * grad_u[pix], 0.0f);
}

// ---------------------------------------------------------------------------
// Strip geometry of the reverse dual step: 2^ts threads per pixel (as the
// forward strips), c = ceil(k / 2^ts) intervals per thread, at most
// kAdjMaxChunk (else the record-per-thread kernels run: returns false);
// 128 / 2^ts pixels per strip (128 threads: smaller CTAs wait less on one
// another at the barriers around the pooled pass; 56.8 against 58.4 ms for
// the 500-iteration reverse pass at 256^2, L = 16), fewer (in steps of a
// warp's pixels) while the strip holds more than kAdjStripRecords records.
static bool adj_strip_shape(const LiftParams &P, int *spp, int *ts, int *c)
{
    const int t = P.k >= 12 ? 2 : (P.k >= 6 ? 1 : 0);
    const int cc = (P.k + (1 << t) - 1) >> t;
    if (cc > kAdjMaxChunk || P.D > 1) return false;
    int n = 128 >> t;
    while (n > (32 >> t) && n * P.k > kAdjStripRecords) n -= 32 >> t;
    *spp = n;
    *ts = t;
    *c = cc;
    return true;
}

int adjoint_blocks(const LiftParams &P)
{
    int spp, ts, c;
    if (adj_strip_shape(P, &spp, &ts, &c)) return (P.N + spp - 1) / spp;
    return (P.N + P.ppb - 1) / P.ppb;
}

cudaError_t launch_adj_seed(const LiftParams &P, const float *grad_u, float2 *ax, cudaStream_t st)
{
    const long long n = static_cast<long long>(P.N) * P.k;
    adj_seed_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(P, grad_u, ax);
    return cudaGetLastError();
}

template <int C>
static cudaError_t launch_adj_strips(const LiftParams &P, int spp, int ts, const LiftState &Sn,
                                     const AdjState &Aj, cudaStream_t st)
{
    const int nb = (P.N + spp - 1) / spp;
    const size_t bytes = static_cast<size_t>(spp) * P.k * (sizeof(float4) + sizeof(float2));
    if (bytes > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(adj_dual_strip_kernel<C>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(bytes));
        if (e != cudaSuccess) return e;
    }
    adj_dual_strip_kernel<C><<<nb, spp << ts, bytes, st>>>(P, spp, ts, Sn.xbar, Sn.y, Aj.G, Aj.ay,
                                                           Aj.aq, Aj.axb, Aj.A, Aj.gf, Aj.partial);
    return cudaGetLastError();
}

// Aj.A must hold zeros before the first reverse iteration (the primal kernel
// adds the previous iteration's neighbour terms from it).
cudaError_t launch_adj_iteration(const LiftParams &P, const LiftState &Sn, const LiftState &Sn1,
                                 const AdjState &Aj, cudaStream_t st)
{
    const int nb = (P.N + P.ppb - 1) / P.ppb;
    int spp, ts, c;
    const bool strips = adj_strip_shape(P, &spp, &ts, &c);
    adj_primal_local_kernel<<<nb, kAdjThreads, 0, st>>>(P, Sn.x, Sn1.y, Aj.ax, Aj.axb, Aj.G,
                                                        strips ? Aj.A : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (strips) {
        switch (c) {
        case 1: return launch_adj_strips<1>(P, spp, ts, Sn, Aj, st);
        case 2: return launch_adj_strips<2>(P, spp, ts, Sn, Aj, st);
        case 3: return launch_adj_strips<3>(P, spp, ts, Sn, Aj, st);
        case 4: return launch_adj_strips<4>(P, spp, ts, Sn, Aj, st);
        case 5: return launch_adj_strips<5>(P, spp, ts, Sn, Aj, st);
        case 6: return launch_adj_strips<6>(P, spp, ts, Sn, Aj, st);
        case 7: return launch_adj_strips<7>(P, spp, ts, Sn, Aj, st);
        default: return launch_adj_strips<8>(P, spp, ts, Sn, Aj, st);
        }
    }
    adj_dual_local_kernel<0><<<nb, kAdjThreads, 0, st>>>(P, Sn.xbar, Sn.y, Aj.G, Aj.ay, Aj.aq,
                                                         Aj.axb, Aj.A, Aj.gf, Aj.partial);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adj_dual_gather_kernel<<<nb, kAdjThreads, 0, st>>>(P, Aj.A, Aj.axb);
    return cudaGetLastError();
}

cudaError_t launch_adj_finish(const LiftParams &P, const AdjState &Aj, cudaStream_t st)
{
    adj_finish_kernel<<<1, 256, 0, st>>>(Aj.partial, adjoint_blocks(P), Aj.acc);
    return cudaGetLastError();
}

}  // namespace lift
