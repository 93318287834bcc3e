// Cluster-resident iteration for small problems (arXiv 1512.01383, Sec. 4).
//
// A problem of a few tens of thousands of records runs each half-step of the
// primal-dual iteration in a couple of microseconds of which most is the
// launch and the round trip to L2, not work: 64 x 64 pixels with L = 2 are 16
// tiles of 256 records.  Here one thread-block cluster (up to 16 CTAs, one per
// SM) keeps the whole state in shared memory for all the iterations of a
// call: CTA c owns a contiguous range of pixels (whole tiles, the same
// 256-thread tiles as the step kernels), loads its state once, and reads its
// neighbours' halo values (ubar at x+1, y+1 in the dual step, p at x-1, y-1 in
// the primal step) from the neighbouring CTA's shared memory through the
// cluster's distributed shared memory.  The hardware cluster barrier separates
// the two half-steps; the state goes back to global memory at the end.  The
// arithmetic of each record is that of dual_tile / primal_tile (pdhg_step.cu).
#include <cooperative_groups.h>

#include "lift_device.cuh"
#include "lift_params.h"
#include "lift_tile.cuh"

namespace cg = cooperative_groups;

namespace lift {

namespace {

constexpr int kResidentMaxCtas = 16;        // a cluster of 16 needs the non-portable size
constexpr int kResidentMaxTilesPerCta = 8;  // beyond that one CTA serialises too much
constexpr size_t kResidentMaxSmem = 200 * 1024;

// The state of one CTA's pixels in shared memory, and where its neighbours'
// state lives.  Every CTA uses the same layout, so a local address maps to
// the same record slot in any other CTA of the cluster.
struct ResMem {
    float4 *y;    // [ppc][k] {v, z, px, py}
    float2 *x;    // [ppc][k] {u, s}
    float2 *xb;   // [ppc][k] {ubar, sbar}
    float *q;     // [ppc]
    int k, ppc, rank, p0, npx;
};

__device__ __forceinline__ int res_owner(const ResMem &M, int pix) { return pix / M.ppc; }

// The cluster barrier in its two halves: every thread arrives when its CTA's
// writes of a phase are done (release), and waits (acquire) only where it is
// about to read another CTA's shared memory or to overwrite what others read,
// so that its own loads and scan overlap the barrier.
__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__device__ __forceinline__ float2 res_xbar(const ResMem &M, cg::cluster_group &cl, int pix, int i)
{
    const int c = res_owner(M, pix);
    const float2 *base = c == M.rank ? M.xb : cl.map_shared_rank(M.xb, c);
    return base[(pix - c * M.ppc) * M.k + i];
}

__device__ __forceinline__ float4 res_y(const ResMem &M, cg::cluster_group &cl, int pix, int i)
{
    const int c = res_owner(M, pix);
    const float4 *base = c == M.rank ? M.y : cl.map_shared_rank(M.y, c);
    return base[(pix - c * M.ppc) * M.k + i];
}

template <int KIND>
__device__ __forceinline__ void res_dual_tile(const LiftParams &P, ResMem &M,
                                              cg::cluster_group &cl, int lt, float *s_in,
                                              float *s_last)
{
    // the previous tile's scan results may still be read from s_in / s_last
    // (the first tile of a phase follows a cluster barrier)
    if (lt > 0) __syncthreads();
    const int tid = threadIdx.x;
    int lp, i;
    split_thread(P, tid, lp, i);
    const int lpix = lt * P.ppb + lp;
    const int pix = M.p0 + lpix;
    const bool active = lp < P.ppb && lpix < M.npx;
    const int lo = lpix * P.k + i;

    float2 xb = make_float2(0.0f, 0.0f);
    float4 d = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (active) {
        xb = M.xb[lo];
        d = M.y[lo];
    }
    // with one interval per pixel every segment is a single record
    const SegScan sc = P.k == 1 ? SegScan{xb.y, xb.y}
                                : block_segmented_scan(xb.y, lp * P.k, P.k, tid, active, s_in, s_last);
    // before the first read of another CTA's xbar (and this phase's writes of
    // y, which the other CTAs read in the previous phase)
    if (lt == 0) cluster_wait();
    if (!active) return;

    const int row = pixel_row(P, pix);
    const int col = pix - row * P.W;
    const float4 ic = __ldg(P.icst + i);      // {gamma_i, tau_s, sigma_vz, lambda*Delta}

    const float gx = col + 1 < P.W ? res_xbar(M, cl, pix + 1, i).x - xb.x : 0.0f;
    const float gy = row + 1 < P.H ? res_xbar(M, cl, pix + P.W, i).x - xb.x : 0.0f;
    float px = d.z + P.sigma_p * gx;
    float py = d.w + P.sigma_p * gy;
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
    const float tail = sc.total - sc.incl;
    float v = d.x + ic.z * (xb.x + P.delta * tail - ic.x * xb.y);
    float z = d.y + ic.z * xb.y;
    if (i == 0) M.q[lpix] -= P.sigma_q * (1.0f + P.delta * sc.total);
    float yo, ho;
    piece_project<KIND>(P, pix, i, ic.x, v * P.inv_delta, z * P.inv_delta, yo, ho);
    v = P.delta * yo;
    z = P.delta * ho;
    M.y[lo] = make_float4(v, z, px, py);
}

__device__ __forceinline__ void res_primal_tile(const LiftParams &P, ResMem &M,
                                                cg::cluster_group &cl, int lt, float *s_in,
                                                float *s_last)
{
    if (lt > 0) __syncthreads();                // as in res_dual_tile
    const int tid = threadIdx.x;
    int lp, i;
    split_thread(P, tid, lp, i);
    const int lpix = lt * P.ppb + lp;
    const int pix = M.p0 + lpix;
    const bool active = lp < P.ppb && lpix < M.npx;
    const int lo = lpix * P.k + i;

    float4 d = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float2 xo = make_float2(0.0f, 0.0f);
    if (active) {
        d = M.y[lo];
        xo = M.x[lo];
    }
    const SegScan sc = P.k == 1 ? SegScan{d.x, d.x}
                                : block_segmented_scan(d.x, lp * P.k, P.k, tid, active, s_in, s_last);
    if (lt == 0) cluster_wait();                 // as in res_dual_tile
    if (!active) return;

    const int row = pixel_row(P, pix);
    const int col = pix - row * P.W;
    const float4 ic = __ldg(P.icst + i);
    const float qq = M.q[lpix];
    float dv = 0.0f;
    if (col + 1 < P.W) dv += d.z;
    if (col > 0) dv -= res_y(M, cl, pix - 1, i).z;
    if (row + 1 < P.H) dv += d.w;
    if (row > 0) dv -= res_y(M, cl, pix - P.W, i).w;
    const float head = sc.incl - d.x;
    const float un = fminf(fmaxf(xo.x - P.tau_u * (d.x - dv), 0.0f), 1.0f);
    const float sn = xo.y - ic.y * (d.y - P.delta * qq + P.delta * head - ic.x * d.x);
    M.x[lo] = make_float2(un, sn);
    M.xb[lo] = make_float2(2.0f * un - xo.x, 2.0f * sn - xo.y);
}

template <int KIND>
__global__ void __launch_bounds__(kStepThreads)
resident_kernel(const LiftParams P, LiftState S, int iters, int ppc)
{
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 res_smem[];
    __shared__ float s_in[kStepThreads];
    __shared__ float s_last[kStepThreads / 32];
    ResMem M;
    M.k = P.k;
    M.ppc = ppc;
    M.rank = static_cast<int>(cl.block_rank());
    M.p0 = M.rank * ppc;
    M.npx = min(ppc, P.N - M.p0);
    const int nrec = ppc * P.k;
    M.y = res_smem;
    M.x = reinterpret_cast<float2 *>(M.y + nrec);
    M.xb = M.x + nrec;
    M.q = reinterpret_cast<float *>(M.xb + nrec);

    const int tid = threadIdx.x;
    const size_t g0 = static_cast<size_t>(M.p0) * P.k;
    const int n = M.npx * P.k;
    for (int r = tid; r < n; r += kStepThreads) {
        M.y[r] = S.y[g0 + r];
        M.x[r] = S.x[g0 + r];
        M.xb[r] = S.xbar[g0 + r];
    }
    for (int r = tid; r < M.npx; r += kStepThreads) M.q[r] = S.q[M.p0 + r];
    // the state is in place; each phase's first tile waits for this (or the
    // previous phase's) arrival of every thread of the cluster
    __syncthreads();
    cluster_arrive();

    const int ntl = (M.npx + P.ppb - 1) / P.ppb;
    for (int it = 0; it < iters; ++it) {
        for (int lt = 0; lt < ntl; ++lt) res_dual_tile<KIND>(P, M, cl, lt, s_in, s_last);
        __syncthreads();
        cluster_arrive();
        for (int lt = 0; lt < ntl; ++lt) res_primal_tile(P, M, cl, lt, s_in, s_last);
        __syncthreads();
        cluster_arrive();
    }
    cluster_wait();

    // every remote read of this CTA's state ended at the last cluster barrier
    for (int r = tid; r < n; r += kStepThreads) {
        S.y[g0 + r] = M.y[r];
        S.x[g0 + r] = M.x[r];
        S.xbar[g0 + r] = M.xb[r];
    }
    for (int r = tid; r < M.npx; r += kStepThreads) S.q[M.p0 + r] = M.q[r];
}

template <int KIND>
cudaLaunchConfig_t resident_config(const ResidentPlan &R, cudaStream_t st,
                                   cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(R.ctas, 1, 1);
    cfg.blockDim = dim3(kStepThreads, 1, 1);
    cfg.dynamicSmemBytes = R.smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = R.ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// The attributes belong to the kernel, not to a handle: they are set to the
// largest request of any handle (every launch asks for at most
// kResidentMaxSmem bytes), so that handles of different sizes can alternate.
template <int KIND>
bool resident_fits(ResidentPlan &R)
{
    if (cudaFuncSetAttribute(resident_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kResidentMaxSmem)) != cudaSuccess ||
        cudaFuncSetAttribute(resident_kernel<KIND>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = resident_config<KIND>(R, nullptr, attr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, resident_kernel<KIND>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

}  // namespace

// Whether the problem fits one cluster: images only, at most 16 CTAs of at
// most 8 tiles each, and their state in the shared memory of one CTA.
bool plan_resident(const LiftParams &P, ResidentPlan &R)
{
    R = ResidentPlan{};
    if (P.D > 1 || P.ppb < 1) return false;
    const int tiles = (P.N + P.ppb - 1) / P.ppb;
    const int tpc = (tiles + kResidentMaxCtas - 1) / kResidentMaxCtas;
    if (tpc > kResidentMaxTilesPerCta) return false;
    R.ppc = tpc * P.ppb;
    R.ctas = (P.N + R.ppc - 1) / R.ppc;
    R.smem = static_cast<size_t>(R.ppc) * P.k * (sizeof(float4) + 2 * sizeof(float2)) +
             static_cast<size_t>(R.ppc) * sizeof(float);
    if (R.smem > kResidentMaxSmem) return false;
    R.ok = P.kind == 2 ? resident_fits<2>(R) : resident_fits<0>(R);
    return R.ok;
}

cudaError_t launch_resident(const LiftParams &P, const LiftState &S, int iters,
                            const ResidentPlan &R, cudaStream_t st)
{
    cudaLaunchAttribute attr[1];
    if (P.kind == 2) {
        const cudaLaunchConfig_t cfg = resident_config<2>(R, st, attr);
        return cudaLaunchKernelEx(&cfg, resident_kernel<2>, P, S, iters, R.ppc);
    }
    const cudaLaunchConfig_t cfg = resident_config<0>(R, st, attr);
    return cudaLaunchKernelEx(&cfg, resident_kernel<0>, P, S, iters, R.ppc);
}

}  // namespace lift
