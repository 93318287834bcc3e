// Device-side data-term pieces of the lifted relaxation (arXiv 1512.01383):
// the convexified pieces rho_i^** on each label interval Gamma_i, their
// conjugates rho_i^* (Prop. 1) and the Euclidean projection onto the
// epigraph of rho_i^* used by the dual step (Sec. 4, Fig. 7).
//
// All arithmetic here is FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lift_params.h"

namespace lift {

// ---------------------------------------------------------------------------
// Quadratic-type piece: rho_i^** on [l, r] is linear on [l, t1], the parabola
// (a/2)(t - c)^2 on [t1, t2] and linear on [t2, r], the linear parts tangent
// to the parabola (C^1).  A = rho_i^**(l), B = rho_i^**(r); m1 = a (t1 - c)
// and m2 = a (t2 - c) are the slopes at t1 and t2.  A piece that is linear on
// the whole interval (a chord, or a constant) has arc = false and m1 = m2.
//
// Its conjugate rho_i^*(y) = sup_{t in [l,r]} t y - rho_i^**(t) is
//   y <= m1 :  l y - A                       (ray of slope l)
//   y >= m2 :  r y - B                       (ray of slope r)
//   between :  c y + y^2 / (2a)              (parabola, slope t = c + y/a)
// with kinks at m1 (slopes l -> t1) and m2 (t2 -> r) when t1 > l, t2 < r.
// ---------------------------------------------------------------------------
// Scalar helpers: T is float on the solver path, or a forward-mode dual
// number (lift_ad.cuh) when the adjoint needs the Jacobian of a projection.
__device__ __forceinline__ float val(float x) { return x; }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }

template <class T>
struct QPieceT {
    T l, r, A, B, m1, m2, t1, t2, a, c;
    bool arc;
};
using QPiece = QPieceT<float>;

// rho = alpha/2 (t - f)^2: the piece is the parabola itself.
template <class T>
__device__ __forceinline__ QPieceT<T> make_quad_piece(T alpha, T f, float l, float r)
{
    QPieceT<T> q;
    q.l = T(l); q.r = T(r); q.a = alpha; q.c = f; q.t1 = T(l); q.t2 = T(r); q.arc = true;
    q.m1 = alpha * (l - f);
    q.m2 = alpha * (r - f);
    q.A = 0.5f * alpha * (l - f) * (l - f);
    q.B = 0.5f * alpha * (r - f) * (r - f);
    return q;
}

// rho = min(alpha (t - f)^2, nu): the parabola 2*alpha/2 (t - f)^2 on
// |t - f| <= w = sqrt(nu/alpha), constant nu outside.  On [l, r] the lower
// convex envelope replaces each constant part adjoining the parabola by the
// tangent from the end point (l, nu) or (r, nu) to the parabola; if the
// tangent point falls outside [l, r] the envelope is the chord between the
// end points, and an interval entirely in a constant part is constant.
// Tangent from (l, nu): with e = f - l > w, the touching point f + d solves
// alpha d^2 + 2 alpha d e + nu = 0, d = -e + sqrt(e^2 - w^2) = -w^2/(e + sqrt(e^2 - w^2)).
template <class T>
__device__ __forceinline__ QPieceT<T> make_trunc_piece(T alpha, T nu, T w, T f, float l, float r)
{
    QPieceT<T> q;
    q.l = T(l); q.r = T(r); q.a = 2.0f * alpha; q.c = f;
    const T kl = f - w, kr = f + w;
    if (r <= val(kl) || l >= val(kr)) {
        q.A = nu; q.B = nu; q.m1 = T(0.0f); q.m2 = T(0.0f); q.t1 = T(l); q.t2 = T(r); q.arc = false;
        return q;
    }
    const T w2 = w * w;
    if (l >= val(kl)) {
        q.t1 = T(l); q.A = alpha * (l - f) * (l - f); q.m1 = 2.0f * alpha * (l - f);
    } else {
        const T e = f - l;
        const T d = -w2 / (e + tsqrt(tmax(e * e - w2, T(0.0f))));
        q.t1 = f + d; q.A = nu; q.m1 = 2.0f * alpha * d;
    }
    if (r <= val(kr)) {
        q.t2 = T(r); q.B = alpha * (r - f) * (r - f); q.m2 = 2.0f * alpha * (r - f);
    } else {
        const T e = r - f;
        const T d = w2 / (e + tsqrt(tmax(e * e - w2, T(0.0f))));
        q.t2 = f + d; q.B = nu; q.m2 = 2.0f * alpha * d;
    }
    q.arc = true;
    if (val(q.t1) > val(q.t2)) {  // the tangent point lies beyond the far end: chord
        const T rl = (l >= val(kl)) ? alpha * (l - f) * (l - f) : nu;
        const T rr = (r <= val(kr)) ? alpha * (r - f) * (r - f) : nu;
        q.A = rl; q.B = rr;
        q.m1 = q.m2 = (rr - rl) / (r - l);
        q.t1 = T(l); q.t2 = T(r);
        q.arc = false;
    }
    return q;
}

template <class T>
__device__ __forceinline__ T qpiece_conj(const QPieceT<T> &q, T y)
{
    if (val(y) <= val(q.m1)) return q.l * y - q.A;
    if (val(y) >= val(q.m2)) return q.r * y - q.B;
    return q.c * y + y * y / (2.0f * q.a);
}

template <class T>
__device__ __forceinline__ T qpiece_envelope(const QPieceT<T> &q, T t)
{
    t = tmin(tmax(t, q.l), q.r);
    if (!q.arc || val(t) <= val(q.t1)) return q.A + q.m1 * (t - q.l);
    if (val(t) >= val(q.t2)) return q.B + q.m2 * (t - q.r);
    const T d = t - q.c;
    return 0.5f * q.a * d * d;
}

// Cube root of x >= 0 from the identity x^(1/3) = 2^(log2(x)/3) on the
// hardware base-2 logarithm / exponential, refined by one Newton step for
// r^3 = x (r <- (2r + x/r^2)/3), which squares the relative error of the
// first estimate.
__device__ __forceinline__ float cube_root(float x)
{
    if (x <= 0.0f) return 0.0f;
    const float r = exp2f(log2f(x) * (1.0f / 3.0f));
    return (2.0f * r + x / (r * r)) * (1.0f / 3.0f);
}

// Largest real root of w^3 + p w - Q = 0 with Q >= 0 (Cardano when one real
// root, trigonometric form when three); written without cancellation.
__device__ __forceinline__ float cubic_outer_root(float p, float Q)
{
    const float p3 = p * (1.0f / 3.0f);
    const float D = 0.25f * Q * Q + p3 * p3 * p3;
    if (D >= 0.0f) {
        const float u1 = cube_root(0.5f * Q + sqrtf(D));
        if (u1 == 0.0f) return 0.0f;
        const float u2 = -p3 / u1;
        // u1^3 + u2^3 = Q and u1 u2 = -p/3, so u1 + u2 = Q / (u1^2 - u1 u2 + u2^2)
        return p >= 0.0f ? Q / (u1 * u1 + p3 + u2 * u2) : u1 + u2;
    }
    const float rr = sqrtf(-p3);
    const float c = fminf(1.0f, 0.5f * Q / (rr * rr * rr));
    return 2.0f * rr * cosf(acosf(c) * (1.0f / 3.0f));
}

// Euclidean projection of (y0, h0) onto epi(rho_i^*) for a quadratic-type
// piece.  The projected abscissa minimises the convex function
//   G(y) = (y - y0)^2 / 2 + max(rho_i^*(y) - h0, 0)^2 / 2,
// whose derivative is increasing; its sign at the two kinks m1, m2 (taken
// from either side) tells which part of the graph receives the point: the
// left ray, the left kink, the parabola, the right kink or the right ray.
// On a ray the projection is onto a line; on the parabola, with
// w = c + y/a, G'(y) = (a/2)(w^3 + p w + q) with p = 2 - c^2 - 2 h0/a,
// q = -2 (c + y0/a), and the projection is its outermost root (the side of
// -q), polished by one Newton step on d = w - c.  (For a dual-number T the
// closed-form root enters as a constant; the Newton step then carries the
// derivative of the root by the implicit-function theorem.)
template <class T>
__device__ __forceinline__ void qpiece_project(const QPieceT<T> &q, T y0, T h0, T &yo, T &ho)
{
    const T phi0 = qpiece_conj(q, y0);
    if (val(h0) >= val(phi0)) { yo = y0; ho = h0; return; }
    const T ph1 = q.l * q.m1 - q.A;             // rho_i^*(m1)
    const T e1 = tmax(ph1 - h0, T(0.0f));
    if (val(q.m1 - y0 + e1 * q.l) > 0.0f) {     // left ray
        const T y = (y0 + q.l * (h0 + q.A)) / (1.0f + q.l * q.l);
        yo = y; ho = q.l * y - q.A; return;
    }
    const T ph2 = q.r * q.m2 - q.B;             // rho_i^*(m2)
    const T e2 = tmax(ph2 - h0, T(0.0f));
    if (val(q.m2 - y0 + e2 * q.r) < 0.0f) {     // right ray
        const T y = (y0 + q.r * (h0 + q.B)) / (1.0f + q.r * q.r);
        yo = y; ho = q.r * y - q.B; return;
    }
    if (!q.arc || val(q.m1 - y0 + e1 * q.t1) >= 0.0f) { yo = q.m1; ho = ph1; return; }
    if (val(q.m2 - y0 + e2 * q.t2) <= 0.0f) { yo = q.m2; ho = ph2; return; }
    // parabola arc: the closed-form root w of the cubic in w
    const T ia = 1.0f / q.a;
    const T p = 2.0f - q.c * q.c - 2.0f * h0 * ia;
    const T qq = -2.0f * (q.c + y0 * ia);
    const float sg = val(qq) <= 0.0f ? 1.0f : -1.0f;
    T w = T(sg * cubic_outer_root(val(p), fabsf(val(qq))));
    w = tmin(tmax(w, q.t1), q.t2);
    // one Newton step on the offset d = w - c = y/a from the centre, whose
    // cubic d^3 + 3c d^2 + (2 + 2c^2 - 2 h0/a) d - 2 (c h0 + y0)/a = 0 is the
    // one above shifted by c; its derivative grows like c^2, so the step is
    // accurate to the rounding of d itself, and y = a d, rho_i^*(y) =
    // y (c + d/2) lose nothing to a centre c far from 0 (periodic pieces sit
    // up to the top of the label range), as w - c and w^2 - c^2 would
    T d = w - q.c;
    const T b2 = 3.0f * q.c;
    const T b1 = 2.0f + 2.0f * q.c * q.c - 2.0f * h0 * ia;
    const T b0 = -2.0f * (q.c * h0 + y0) * ia;
    const T F = ((d + b2) * d + b1) * d + b0;
    const T dF = (3.0f * d + 2.0f * b2) * d + b1;
    if (val(dF) > 0.0f) d = tmin(tmax(d - F / dF, q.t1 - q.c), q.t2 - q.c);
    const T y = q.a * d;
    yo = y;
    ho = y * (q.c + 0.5f * d);
}

// ---------------------------------------------------------------------------
// Piecewise-linear piece: rho_i^** interpolates the values rh[0..n-1] at the
// increasing breakpoints t[0..n-1] of Gamma_i (t[0] = l, t[n-1] = r), with
// non-decreasing slopes (a lower hull).  Its conjugate is
//   rho_i^*(y) = max_j t_j y - rh_j,
// piecewise linear with slope t_j between the kinks y = slope_{j-1} and
// y = slope_j (Sec. 4: the slopes of the conjugate are the sublabel
// positions, its intercepts the function values).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pl_conj(const float *__restrict__ t,
                                         const float *__restrict__ rh, int n, float y)
{
    float best = t[0] * y - rh[0];
    for (int j = 1; j < n; ++j) best = fmaxf(best, t[j] * y - rh[j]);
    return best;
}

__device__ __forceinline__ float pl_envelope(const float *__restrict__ t,
                                             const float *__restrict__ rh, int n, float x)
{
    x = fminf(fmaxf(x, t[0]), t[n - 1]);
    int j = 0;
    while (j < n - 2 && x > t[j + 1]) ++j;
    const float a = (x - t[j]) / (t[j + 1] - t[j]);
    return (1.0f - a) * rh[j] + a * rh[j + 1];
}

// Projection of a point below the graph onto epi(max_j t_j y - rh_j): same
// monotone-derivative test as the quadratic piece, walking the kinks from
// left to right.
__device__ __forceinline__ void pl_project_below(const float *__restrict__ t,
                                                 const float *__restrict__ rh, int n,
                                                 float y0, float h0, float &yo, float &ho)
{
    float tj = t[0], rj = rh[0];
    for (int j = 0; j < n - 1; ++j) {
        const float tn = t[j + 1], rn = rh[j + 1];
        const float m = (rn - rj) / (tn - tj);      // kink of the conjugate
        const float ph = tj * m - rj;
        const float e = fmaxf(ph - h0, 0.0f);
        if (m - y0 + e * tj > 0.0f) {               // segment of slope t_j
            const float y = (y0 + tj * (h0 + rj)) / (1.0f + tj * tj);
            yo = y; ho = tj * y - rj; return;
        }
        if (m - y0 + e * tn >= 0.0f) { yo = m; ho = ph; return; }
        tj = tn; rj = rn;
    }
    const float y = (y0 + tj * (h0 + rj)) / (1.0f + tj * tj);
    yo = y; ho = tj * y - rj;
}

__device__ __forceinline__ void pl_project(const float *__restrict__ t,
                                           const float *__restrict__ rh, int n,
                                           float y0, float h0, float &yo, float &ho)
{
    if (h0 >= pl_conj(t, rh, n, y0)) { yo = y0; ho = h0; return; }
    pl_project_below(t, rh, n, y0, h0, yo, ho);
}

// ---------------------------------------------------------------------------
// Uniform access for the kernels.
// ---------------------------------------------------------------------------
// Phase unwrapping (kind 3): on [l, r] the parabola of the periodic copy
// f + nu*m of the data nearest to the interval's midpoint (nu = period).
__device__ __forceinline__ float periodic_center(float f, float per, float l, float r)
{
    return f + per * floorf((0.5f * (l + r) - f) / per + 0.5f);
}

// The piece on [l, r] of a pixel whose data value is f.
__device__ __forceinline__ QPiece make_qpiece_f(const LiftParams &P, float f, float l, float r)
{
    if (P.kind == 3) return make_quad_piece<float>(P.alpha, periodic_center(f, P.nu, l, r), l, r);
    return P.kind == 0 ? make_quad_piece<float>(P.alpha, f, l, r)
                       : make_trunc_piece<float>(P.alpha, P.nu, P.wtrunc, f, l, r);
}

__device__ __forceinline__ QPiece make_qpiece(const LiftParams &P, int pix, float l, float r)
{
    return make_qpiece_f(P, __ldg(P.f + pix), l, r);
}

// rho_i^*(y) of pixel pix, interval i, for any kind.
template <int KIND>
__device__ __forceinline__ float piece_conj(const LiftParams &P, int pix, int i, float l, float y)
{
    if (KIND == 2) {
        const int b0 = __ldg(P.bstart + i), n = __ldg(P.bstart + i + 1) - b0 + 1;
        return pl_conj(P.bpos + b0, P.rhat + (size_t)pix * P.nb + b0, n, y);
    }
    const QPiece q = make_qpiece(P, pix, l, l + P.delta);
    return qpiece_conj(q, y);
}

// rho_i^*(y) of a quadratic-type interval straight from its definition,
// without building the envelope: for rho = min(alpha (t-f)^2, nu),
// -min(A,B) = max(-A,-B) gives the larger of the clamped-parabola sup and
// max(l y, r y) - nu; for rho = alpha/2 (t-f)^2 only the clamped parabola.
// Branch-free; it lets points that already lie in the epigraph (most of
// them) skip the envelope and the projection.
__device__ __forceinline__ float quad_conj_direct(const LiftParams &P, float f, float l, float r,
                                                  float y)
{
    if (P.kind == 1) {
        const float t = fminf(fmaxf(f + y * (0.5f * P.inv_alpha), l), r);
        const float d = t - f;
        return fmaxf(t * y - P.alpha * d * d, fmaxf(l * y, r * y) - P.nu);
    }
    const float c = P.kind == 3 ? periodic_center(f, P.nu, l, r) : f;
    const float t = fminf(fmaxf(c + y * P.inv_alpha, l), r);
    const float d = t - c;
    return t * y - 0.5f * P.alpha * d * d;
}

template <int KIND>
__device__ __forceinline__ bool piece_in_epigraph(const LiftParams &P, int pix, int i, float l,
                                                  float y0, float h0)
{
    if (KIND == 2) {
        const int b0 = __ldg(P.bstart + i), n = __ldg(P.bstart + i + 1) - b0 + 1;
        return h0 >= pl_conj(P.bpos + b0, P.rhat + (size_t)pix * P.nb + b0, n, y0);
    }
    return h0 >= quad_conj_direct(P, __ldg(P.f + pix), l, l + P.delta, y0);
}

template <int KIND>
__device__ __forceinline__ void piece_project_below(const LiftParams &P, int pix, int i, float l,
                                                    float y0, float h0, float &yo, float &ho)
{
    if (KIND == 2) {
        const int b0 = __ldg(P.bstart + i), n = __ldg(P.bstart + i + 1) - b0 + 1;
        pl_project_below(P.bpos + b0, P.rhat + (size_t)pix * P.nb + b0, n, y0, h0, yo, ho);
        return;
    }
    const QPiece q = make_qpiece(P, pix, l, l + P.delta);
    qpiece_project(q, y0, h0, yo, ho);
}

template <int KIND>
__device__ __forceinline__ void piece_project(const LiftParams &P, int pix, int i, float l,
                                              float y0, float h0, float &yo, float &ho)
{
    if (piece_in_epigraph<KIND>(P, pix, i, l, y0, h0)) { yo = y0; ho = h0; return; }
    piece_project_below<KIND>(P, pix, i, l, y0, h0, yo, ho);
}

template <int KIND>
__device__ __forceinline__ float piece_envelope(const LiftParams &P, int pix, int i, float l,
                                                float t)
{
    if (KIND == 2) {
        const int b0 = __ldg(P.bstart + i), n = __ldg(P.bstart + i + 1) - b0 + 1;
        return pl_envelope(P.bpos + b0, P.rhat + (size_t)pix * P.nb + b0, n, t);
    }
    const QPiece q = make_qpiece(P, pix, l, l + P.delta);
    return qpiece_envelope(q, t);
}

// The data term itself, rho(x, t) (for the nonconvex energy).
__device__ __forceinline__ float data_rho(const LiftParams &P, int pix, float t)
{
    if (P.kind == 2) {
        const float x = (fminf(fmaxf(t, P.smin), P.smin + P.sh * (P.ns - 1)) - P.smin) / P.sh;
        int j = (int)floorf(x);
        j = j < 0 ? 0 : (j > P.ns - 2 ? P.ns - 2 : j);
        const float a = x - (float)j;
        const float *c = P.cost + (size_t)pix * P.ns;
        return (1.0f - a) * __ldg(c + j) + a * __ldg(c + j + 1);
    }
    if (P.kind == 3) {
        // alpha/2 times the squared circular distance to f (period nu): the
        // nearer of the copies f + nu m, m = floor((t - f)/nu), and the next
        const float f = __ldg(P.f + pix);
        const float m = floorf((t - f) / P.nu);
        const float d1 = t - f - P.nu * m, d2 = d1 - P.nu;
        const float d = fabsf(d1) < fabsf(d2) ? d1 : d2;
        return 0.5f * P.alpha * d * d;
    }
    const float d = t - __ldg(P.f + pix);
    if (P.kind == 0) return 0.5f * P.alpha * d * d;
    return fminf(P.alpha * d * d, P.nu);
}

}  // namespace lift
