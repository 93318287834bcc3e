// Reverse mode through the unrolled primal-dual iteration (the differentiable
// solve): given the adjoint of the state after iteration n+1, produce the
// adjoint of the state after iteration n and accumulate the gradients with
// respect to the data f, lambda, alpha and nu.  Not part of the paper; it
// differentiates the map of pdhg_step.cu (Sec. 4) exactly, including the
// clamp of u, the l2-ball projection (Prop. 5) and the epigraph projections
// (Fig. 7), whose local Jacobians come from the same piece / projection code
// evaluated on forward-mode dual numbers (lift_ad.cuh).
//
// With x = (u, s), xbar, y = (v, z, px, py), q and adjoints ax, axb, ay, aq,
// one reverse iteration is three kernels:
//   adj_primal_local : g_u = [0 < w < 1](ax.u + 2 axb.u), g_s = ax.s + 2 axb.s
//                      (w = the unclamped primal update), ax <- g - axb
//   adj_dual_local   : completes ay, aq with the primal step's uses of y, q,
//                      then pulls them back through the dual step: the ball
//                      and epigraph projections, the ascent and the sums over
//                      intervals; writes ay, aq, the own part of axb, f's
//                      gradient and per-block sums of the scalar gradients
//   adj_dual_gather  : adds the neighbours' part of grad^T to axb.u
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

}  // namespace

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjThreads)
adj_primal_local_kernel(const LiftParams P, const float2 *__restrict__ x_n,
                        const float4 *__restrict__ y_n1, float2 *__restrict__ ax,
                        const float2 *__restrict__ axb, float2 *__restrict__ G)
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
    const float2 a = ax[o], b = axb[o];
    const float gu = (w > 0.0f && w < 1.0f) ? a.x + 2.0f * b.x : 0.0f;
    const float gs = a.y + 2.0f * b.y;
    G[o] = make_float2(gu, gs);
    ax[o] = make_float2(gu - b.x, gs - b.y);
}

// ---------------------------------------------------------------------------
// Four blocks per SM (64 registers, a few bytes spilled): the dual-number
// projection below otherwise holds 80 registers and leaves three.  Records in
// the epigraph of rho_i^* (the forward step's float test) take its identity
// Jacobian; those below it are packed per warp into one dual-number pass.
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
    // dual-number projection, and its results for their owners
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
            using D5 = Dual<5>;
            const D5 y0 = D5::seed(e.x, 0), h0 = D5::seed(e.y, 1);
            const D5 f = D5::seed(eb.x, 2), al = D5::seed(P.alpha, 3), nu = D5::seed(P.nu, 4);
            const float l = eb.y, r = eb.y + P.delta;
            QPieceT<D5> qp;
            if (P.kind == 3)
                qp = make_quad_piece<D5>(al, f + (periodic_center(f.v, P.nu, l, r) - f.v), l, r);
            else if (P.kind == 0) qp = make_quad_piece<D5>(al, f, l, r);
            else qp = make_trunc_piece<D5>(al, nu, tsqrt(nu / al), f, l, r);
            D5 yo, ho;
            qpiece_project(qp, y0, h0, yo, ho);
            // (v', z') = Delta (yo, ho)((v^, z^)/Delta)
            const float av = e.z * yo.d[0] + e.w * ho.d[0];
            const float az = e.z * yo.d[1] + e.w * ho.d[1];
            const float df = P.delta * (e.z * yo.d[2] + e.w * ho.d[2]);
            ga += static_cast<double>(P.delta * (e.z * yo.d[3] + e.w * ho.d[3]));
            gn += static_cast<double>(P.delta * (e.z * yo.d[4] + e.w * ho.d[4]));
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
int adjoint_blocks(const LiftParams &P)
{
    return (P.N + P.ppb - 1) / P.ppb;
}

cudaError_t launch_adj_seed(const LiftParams &P, const float *grad_u, float2 *ax, cudaStream_t st)
{
    const long long n = static_cast<long long>(P.N) * P.k;
    adj_seed_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(P, grad_u, ax);
    return cudaGetLastError();
}

cudaError_t launch_adj_iteration(const LiftParams &P, const LiftState &Sn, const LiftState &Sn1,
                                 const AdjState &Aj, cudaStream_t st)
{
    const int nb = adjoint_blocks(P);
    adj_primal_local_kernel<<<nb, kAdjThreads, 0, st>>>(P, Sn.x, Sn1.y, Aj.ax, Aj.axb, Aj.G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
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
