/*
 * FP64 CPU oracle for the lifted primal-dual (PDHG) solver of
 * "Sublabel-Accurate Relaxation of Nonconvex Energies" (Moellenhoff, Laude,
 * Moeller, Lellmann, Cremers, arXiv 1512.01383).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Every quantity is computed from its definition, in double precision:
 *   - the data term rho(x,t) itself (quadratic, truncated quadratic, or the
 *     piecewise-linear interpolant of sampled costs);
 *   - the per-interval conjugate rho_i^*(y) = sup_{t in Gamma_i} t*y - rho(t)
 *     (Prop. 1, with rho_i = rho + delta_{Gamma_i}), evaluated as an explicit
 *     maximum over the few candidate maximisers of each smooth part;
 *   - the Euclidean projection onto epi(rho_i^*), as the minimiser of the
 *     convex 1-D function  y -> (y-y0)^2/2 + max(rho_i^*(y)-h0, 0)^2/2,
 *     found by bisection on its monotone derivative;
 *   - the convexified piece rho_i^** (t) = sup_y t*y - rho_i^*(y), again by
 *     bisection on a monotone derivative;
 *   - the PDHG iteration on the saddle-point problem of Sec. 4
 *     (eq. discrete_saddle_point_final with the set C of eq. constraint_C,
 *     the z-splitting of eq. equality_constr_data and its multiplier s,
 *     the l2-ball set K of Prop. 5, forward differences on a Cartesian grid
 *     of d = 2 (image) or d = 3 (volume) axes, p_i in R^d),
 *     with the diagonal preconditioning of Pock-Chambolle (alpha = 1).
 *
 * Readings of points the paper leaves open:
 *   c_i(v) = <1_{i-1}, v> - gamma_i v_i / Delta_i (appendix form, proof of
 *   Prop. 1); lambda is the radius factor of K (|p_i| <= lambda*Delta_i);
 *   Neumann forward differences; primal box u in [0,1]^k; fixed steps
 *   (no adaptive step rule) with a constant primal/dual balance theta that
 *   the caller chooses; dual step first from the extrapolated primal,
 *   then primal step, then extrapolation with theta = 1; all variables start
 *   at zero.
 *
 * Parity pins for every function here live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LIFT_ORACLE_MAXK 256

/* ------------------------------------------------------------------------ */
/* Problem description (owned by the caller, read-only here).               */
/* ------------------------------------------------------------------------ */
enum { ORC_QUAD = 0, ORC_TRUNC = 1, ORC_PL = 2, ORC_PERIODIC = 3 };

typedef struct {
    int kind;              /* ORC_QUAD: rho = alpha/2 (t-f)^2
                              ORC_TRUNC: rho = min(alpha (t-f)^2, nu)
                              ORC_PL: rho = PL interpolant of sampled costs
                              ORC_PERIODIC: rho = alpha/2 times the squared
                              circular distance to f (period nu), seen by
                              the relaxation on Gamma_i as alpha/2 (t-c_i)^2,
                              c_i the copy f + nu*m nearest the interval's
                              midpoint (Sec. 5.5) */
    int H, W, L;           /* image size, number of labels (k = L-1)      */
    double gmin, gmax;     /* label range Gamma = [gmin, gmax], equidistant */
    double lam;            /* TV weight lambda                             */
    double alpha, nu;      /* data-term parameters                         */
    const double *f;       /* H*W input image (QUAD, TRUNC)                */
    const double *cost;    /* H*W*ns sampled costs, pixel-major (PL)       */
    int ns;                /* number of samples per pixel (PL)             */
    double smin, smax;     /* sample positions smin + j (smax-smin)/(ns-1)  */
    double theta;          /* primal/dual step balance (<= 0 means 1)      */
    int aniso;             /* 1: phi(nu) = |nu|_1 (anisotropic TV), K is a  */
                           /*    product of l-infinity boxes; 0: |nu|_2     */
    int D;                 /* depth: D > 1 makes the domain a D x H x W     */
                           /* volume (voxel (z*H + y)*W + x, three forward  */
                           /* differences); D <= 1 is the 2-D image         */
} orc_problem;

/* The norm phi of the jump direction in Phi_{i,j} (eq. regularizer_single)
   and the projection onto the dual-norm ball of radius R (Prop. 5 holds for
   any convex one-homogeneous phi, Sec. 5.3).  Three components; a 2-D image
   passes c = 0. */
static double tv_norm(int aniso, double a, double b, double c)
{
    return aniso ? fabs(a) + fabs(b) + fabs(c) : sqrt(a * a + b * b + c * c);
}

static double clamp_abs(double a, double R)
{
    return a > R ? R : (a < -R ? -R : a);
}

static void tv_project(int aniso, double R, double *a, double *b, double *c)
{
    if (aniso) {
        *a = clamp_abs(*a, R);
        *b = clamp_abs(*b, R);
        *c = clamp_abs(*c, R);
        return;
    }
    double nrm = sqrt(*a * *a + *b * *b + *c * *c);
    double sc = nrm > R ? (nrm > 0.0 ? R / nrm : 0.0) : 1.0;
    *a *= sc;
    *b *= sc;
    *c *= sc;
}

/* PDHG state; all arrays caller-allocated, index [pixel*k + i]. */
typedef struct {
    double *u, *s;         /* primal: lifted u and multiplier s            */
    double *ubar, *sbar;   /* extrapolated primal                          */
    double *v, *z;         /* dual: data-term dual and scaled epigraph var */
    double *px, *py;       /* dual: TV dual p_i in R^2                     */
    double *q;             /* dual: epigraph height, one per pixel         */
    double *pz;            /* dual: third component of p_i (D > 1 only)    */
} orc_state;

static int depth(const orc_problem *P) { return P->D > 1 ? P->D : 1; }

static size_t npix(const orc_problem *P)
{
    return (size_t)depth(P) * P->H * P->W;
}

static double gam(const orc_problem *P, int j)   /* gamma_{j+1}, j = 0..k */
{
    int k = P->L - 1;
    return P->gmin + (P->gmax - P->gmin) * (double)j / (double)k;
}

static double clampd(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

/* ------------------------------------------------------------------------ */
/* The data term rho(x, t) (eq. general_energy; Sec. 5.1, 5.2, 5.4).         */
/* ------------------------------------------------------------------------ */
static double pl_pos(const orc_problem *P, int j)
{
    return P->smin + (P->smax - P->smin) * (double)j / (double)(P->ns - 1);
}

/* Phase unwrapping (Sec. 5.5): the squared circular distance d(t, f)^2 is
   approximated on each interval Gamma_i by the parabola of the periodic copy
   of f nearest to the interval's midpoint. */
static double periodic_center(const orc_problem *P, int pix, int i)
{
    double mid = 0.5 * (gam(P, i) + gam(P, i + 1)), f = P->f[pix], per = P->nu;
    return f + per * floor((mid - f) / per + 0.5);
}

static double periodic_piece(const orc_problem *P, int pix, int i, double t)
{
    double d = t - periodic_center(P, pix, i);
    return 0.5 * P->alpha * d * d;
}

/* rho(t) itself (Sec. 5.5): alpha/2 times the squared circular distance of t
   to the data, min over integers m of (t - f - nu m)^2.  The nearest copy is
   f + nu m with m = floor((t - f)/nu) or m + 1, so the minimum over those two
   is the minimum over all m.  Only the nonconvex energy E_nc reads this; the
   relaxation sees the per-interval parabolas above. */
static double periodic_rho(const orc_problem *P, int pix, double t)
{
    double f = P->f[pix], per = P->nu;
    double m = floor((t - f) / per);
    double d1 = t - f - per * m, d2 = t - f - per * (m + 1.0);
    double d = fabs(d1) < fabs(d2) ? d1 : d2;
    return 0.5 * P->alpha * d * d;
}

double orc_rho(const orc_problem *P, int pix, double t)
{
    if (P->kind == ORC_PERIODIC) return periodic_rho(P, pix, t);
    if (P->kind == ORC_QUAD) {
        double d = t - P->f[pix];
        return 0.5 * P->alpha * d * d;
    }
    if (P->kind == ORC_TRUNC) {
        double d = t - P->f[pix];
        double qd = P->alpha * d * d;
        return qd < P->nu ? qd : P->nu;
    }
    /* piecewise-linear interpolation of the samples */
    const double *c = P->cost + (size_t)pix * P->ns;
    double h = (P->smax - P->smin) / (double)(P->ns - 1);
    double x = (clampd(t, P->smin, P->smax) - P->smin) / h;
    int j = (int)floor(x);
    if (j < 0) j = 0;
    if (j > P->ns - 2) j = P->ns - 2;
    double a = x - (double)j;
    return (1.0 - a) * c[j] + a * c[j + 1];
}

/* ------------------------------------------------------------------------ */
/* rho_i^*(y) = sup_{t in [gamma_i, gamma_{i+1}]} t*y - rho(t)  (Prop. 1).   */
/* Returns the value; *tmax receives a maximiser (a subgradient of rho_i^*).  */
/* ------------------------------------------------------------------------ */
double orc_conj(const orc_problem *P, int pix, int i, double y, double *tmax)
{
    double l = gam(P, i), r = gam(P, i + 1);
    double best, bt;
    if (P->kind == ORC_QUAD) {
        /* concave quadratic in t: stationary point f + y/alpha, clamped */
        double t = clampd(P->f[pix] + y / P->alpha, l, r);
        best = t * y - orc_rho(P, pix, t);
        bt = t;
    } else if (P->kind == ORC_PERIODIC) {
        /* the interval's own parabola, centred at c_i */
        double c = periodic_center(P, pix, i);
        double t = clampd(c + y / P->alpha, l, r);
        best = t * y - periodic_piece(P, pix, i, t);
        bt = t;
    } else if (P->kind == ORC_TRUNC) {
        /* -min(A,B) = max(-A,-B): the sup of the max is the max of the sups */
        double f = P->f[pix];
        double tq = clampd(f + y / (2.0 * P->alpha), l, r);
        double vq = tq * y - P->alpha * (tq - f) * (tq - f);
        double tc = y >= 0.0 ? r : l;
        double vc = tc * y - P->nu;
        if (vq >= vc) { best = vq; bt = tq; } else { best = vc; bt = tc; }
    } else {
        /* t*y - rho(t) is piecewise linear in t: the sup is attained at a
           breakpoint of rho inside Gamma_i or at an end of Gamma_i */
        best = l * y - orc_rho(P, pix, l);
        bt = l;
        for (int j = 0; j < P->ns; ++j) {
            double t = pl_pos(P, j);
            if (t > l && t < r) {
                double val = t * y - orc_rho(P, pix, t);
                if (val > best) { best = val; bt = t; }
            }
        }
        double vr = r * y - orc_rho(P, pix, r);
        if (vr > best) { best = vr; bt = r; }
    }
    if (tmax) *tmax = bt;
    return best;
}

/* Lifted conjugate of Prop. 1:  max_i  c_i(v) + rho_i^*(v_i / Delta_i),
   c_i(v) = sum_{l<i} v_l - gamma_i v_i / Delta_i (appendix form). */
double orc_lifted_conj(const orc_problem *P, int pix, const double *v)
{
    int k = P->L - 1;
    double best = -INFINITY, prefix = 0.0;
    for (int i = 0; i < k; ++i) {
        double d = gam(P, i + 1) - gam(P, i);
        double ci = prefix - gam(P, i) * v[i] / d;
        double val = ci + orc_conj(P, pix, i, v[i] / d, NULL);
        if (val > best) best = val;
        prefix += v[i];
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Euclidean projection of (y0, h0) onto epi(rho_i^*) (Sec. 4, Fig. 7).      */
/* Distance to the epigraph:  min_y (y-y0)^2 + max(phi(y)-h0, 0)^2, whose    */
/* objective is convex in y; its derivative is monotone and is bisected.    */
/* ------------------------------------------------------------------------ */
static double epi_deriv(const orc_problem *P, int pix, int i, double y,
                        double y0, double h0)
{
    double t;
    double phi = orc_conj(P, pix, i, y, &t);
    double e = phi - h0;
    if (e < 0.0) e = 0.0;
    return (y - y0) + e * t;
}

void orc_proj_epi(const orc_problem *P, int pix, int i, double y0, double h0,
                  double *y_out, double *h_out)
{
    double phi0 = orc_conj(P, pix, i, y0, NULL);
    if (h0 >= phi0) { *y_out = y0; *h_out = h0; return; }
    /* the minimiser lies within the distance phi0-h0 of y0 */
    double d0 = phi0 - h0;
    double lo = y0 - d0, hi = y0 + d0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (epi_deriv(P, pix, i, mid, y0, h0) > 0.0) hi = mid; else lo = mid;
    }
    double y = 0.5 * (lo + hi);
    double phi = orc_conj(P, pix, i, y, NULL);
    *y_out = y;
    *h_out = phi > h0 ? phi : h0;
}

/* ------------------------------------------------------------------------ */
/* rho_i^**(t) = sup_y t*y - rho_i^*(y), t in Gamma_i: the convexified piece */
/* that the relaxation sees (Prop. 1 and the remark after it).               */
/* ------------------------------------------------------------------------ */
static double slope_bound(const orc_problem *P, int pix, int i)
{
    double l = gam(P, i), r = gam(P, i + 1);
    if (P->kind == ORC_QUAD) {
        double f = P->f[pix];
        return 1.0 + P->alpha * (fabs(l - f) + fabs(r - f));
    }
    if (P->kind == ORC_PERIODIC) {
        double c = periodic_center(P, pix, i);
        return 1.0 + P->alpha * (fabs(l - c) + fabs(r - c));
    }
    if (P->kind == ORC_TRUNC) {
        double f = P->f[pix];
        return 1.0 + 2.0 * P->alpha * (fabs(l - f) + fabs(r - f))
                   + 2.0 * P->nu / (r - l);
    }
    /* PL: no slope of the lower hull exceeds the largest secant slope */
    double m = 0.0, tp = l, rp = orc_rho(P, pix, l);
    for (int j = 0; j <= P->ns; ++j) {
        double t = j < P->ns ? pl_pos(P, j) : r;
        if (j < P->ns && !(t > l && t < r)) continue;
        double rv = orc_rho(P, pix, t);
        double sl = fabs(rv - rp) / (t - tp);
        if (sl > m) m = sl;
        tp = t; rp = rv;
    }
    return 1.0 + 2.0 * m;
}

double orc_biconj(const orc_problem *P, int pix, int i, double t)
{
    double Y = slope_bound(P, pix, i);
    double lo = -Y, hi = Y;
    /* d/dy [t*y - rho_i^*(y)] = t - tmax(y), non-increasing in y */
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double tm;
        orc_conj(P, pix, i, mid, &tm);
        if (t - tm > 0.0) lo = mid; else hi = mid;
    }
    double y = 0.5 * (lo + hi);
    return t * y - orc_conj(P, pix, i, y, NULL);
}

/* ------------------------------------------------------------------------ */
/* Forward differences with Neumann boundary (Sec. 4) and div = -grad^T.     */
/* Arrays are [pixel*k + i].                                                 */
/* ------------------------------------------------------------------------ */
/* A D x H x W volume (D = 1: an image); gz may be NULL when D = 1. */
void orc_grad3(int D, int H, int W, int k, const double *u, double *gx, double *gy,
               double *gz)
{
    size_t row = (size_t)W * k, slice = (size_t)H * W * k;
    for (int zz = 0; zz < D; ++zz)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int i = 0; i < k; ++i) {
                    size_t o = (((size_t)zz * H + y) * W + x) * k + i;
                    gx[o] = x + 1 < W ? u[o + k] - u[o] : 0.0;
                    gy[o] = y + 1 < H ? u[o + row] - u[o] : 0.0;
                    if (gz) gz[o] = zz + 1 < D ? u[o + slice] - u[o] : 0.0;
                }
}

void orc_div3(int D, int H, int W, int k, const double *px, const double *py,
              const double *pz, double *d)
{
    size_t row = (size_t)W * k, slice = (size_t)H * W * k;
    for (int zz = 0; zz < D; ++zz)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int i = 0; i < k; ++i) {
                    size_t o = (((size_t)zz * H + y) * W + x) * k + i;
                    double a = 0.0;
                    if (x + 1 < W) a += px[o];
                    if (x > 0) a -= px[o - k];
                    if (y + 1 < H) a += py[o];
                    if (y > 0) a -= py[o - row];
                    if (pz) {
                        if (zz + 1 < D) a += pz[o];
                        if (zz > 0) a -= pz[o - slice];
                    }
                    d[o] = a;
                }
}

void orc_grad(int H, int W, int k, const double *u, double *gx, double *gy)
{
    orc_grad3(1, H, W, k, u, gx, gy, NULL);
}

void orc_div(int H, int W, int k, const double *px, const double *py,
             double *d)
{
    orc_div3(1, H, W, k, px, py, NULL, d);
}

/* ------------------------------------------------------------------------ */
/* Step sizes: diagonal preconditioning with alpha = 1, i.e. the reciprocal  */
/* absolute row / column sums of the linear operator of the saddle point:   */
/*   v_l : u_l + sum_{j>l} Delta_j s_j - gamma_l s_l                         */
/*   z_i : s_i          q : -sum_i Delta_i s_i        p_i : grad u_i         */
/* The (v_i, z_i) pair is projected jointly, so it shares one step (the      */
/* smaller of its two rows); every component of p_i shares 1/2; the column  */
/* of u uses the interior count 1 + 2 * (number of axes), 1 + 4 on an image */
/* and 1 + 6 on a volume.  A balance theta > 0 then multiplies              */
/* every primal step and divides every dual step: the products tau*sigma,    */
/* and with them the convergence condition of the preconditioned method,    */
/* are unchanged; theta is the primal/dual balance that the adaptive step    */
/* rule cited in Sec. 4 adjusts.                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    double tau_u, sigma_q, sigma_p;
    double *tau_s, *sigma_vz;
} orc_steps;

static void make_steps(const orc_problem *P, orc_steps *S)
{
    int k = P->L - 1;
    S->tau_u = 1.0 / (1.0 + 2.0 * (depth(P) > 1 ? 3.0 : 2.0));
    S->sigma_q = 1.0 / (gam(P, k) - gam(P, 0));
    S->sigma_p = 0.5;
    S->tau_s = (double *)malloc(sizeof(double) * k);
    S->sigma_vz = (double *)malloc(sizeof(double) * k);
    for (int i = 0; i < k; ++i) {
        double d = gam(P, i + 1) - gam(P, i);
        /* column of s_i: (i) entries Delta_i in v_l (l<i), |gamma_i| in v_i,
           1 in z_i, Delta_i in q  (0-based i: i entries with l < i) */
        S->tau_s[i] = 1.0 / (1.0 + fabs(gam(P, i)) + (double)(i + 1) * d);
        double row_v = 1.0 + fabs(gam(P, i)) + (gam(P, k) - gam(P, i + 1));
        double row_z = 1.0;
        S->sigma_vz[i] = 1.0 / (row_v > row_z ? row_v : row_z);
    }
    double th = P->theta > 0.0 ? P->theta : 1.0;
    S->tau_u *= th;
    S->sigma_q /= th;
    S->sigma_p /= th;
    for (int i = 0; i < k; ++i) {
        S->tau_s[i] *= th;
        S->sigma_vz[i] /= th;
    }
}

static void free_steps(orc_steps *S)
{
    free(S->tau_s);
    free(S->sigma_vz);
}

void orc_steps_get(const orc_problem *P, double *tau_u, double *sigma_q,
                   double *sigma_p, double *tau_s, double *sigma_vz)
{
    orc_steps S;
    make_steps(P, &S);
    *tau_u = S.tau_u; *sigma_q = S.sigma_q; *sigma_p = S.sigma_p;
    int k = P->L - 1;
    for (int i = 0; i < k; ++i) { tau_s[i] = S.tau_s[i]; sigma_vz[i] = S.sigma_vz[i]; }
    free_steps(&S);
}

/* ------------------------------------------------------------------------ */
/* PDHG iterations (Sec. 4): dual ascent from the extrapolated primal, then  */
/* the projections onto K (l2 balls, Prop. 5) and onto the scaled epigraphs */
/* of rho_i^* (eq. equality_constr_data), then primal descent on (u, s)     */
/* with u kept in [0,1]^k, then extrapolation with theta = 1.               */
/* ------------------------------------------------------------------------ */
/* The dual half-step: TV dual ascent and projection onto K, data-dual ascent
   and projection onto the scaled epigraphs, q ascent.  gx, gy, gz: Nk work. */
static void dual_half(const orc_problem *P, orc_state *X, const orc_steps *S, double *gx,
                      double *gy, double *gz)
{
    int H = P->H, W = P->W, k = P->L - 1, Dz = depth(P);
    size_t N = npix(P);
    orc_grad3(Dz, H, W, k, X->ubar, gx, gy, gz);
    for (size_t pix = 0; pix < N; ++pix) {
        double *v = X->v + pix * k, *z = X->z + pix * k;
        double *px = X->px + pix * k, *py = X->py + pix * k;
        const double *ub = X->ubar + pix * k, *sb = X->sbar + pix * k;
        /* TV dual: ascent, then projection onto |p_i| <= lambda Delta_i */
        for (int i = 0; i < k; ++i) {
            double d = gam(P, i + 1) - gam(P, i);
            double ax = px[i] + S->sigma_p * gx[pix * k + i];
            double ay = py[i] + S->sigma_p * gy[pix * k + i];
            double az = Dz > 1 ? X->pz[pix * k + i] + S->sigma_p * gz[pix * k + i] : 0.0;
            tv_project(P->aniso, P->lam * d, &ax, &ay, &az);
            px[i] = ax;
            py[i] = ay;
            if (Dz > 1) X->pz[pix * k + i] = az;
        }
        /* data duals: ascent on v, z, q */
        double tot = 0.0;
        for (int i = 0; i < k; ++i) tot += (gam(P, i + 1) - gam(P, i)) * sb[i];
        for (int l = 0; l < k; ++l) {
            double tail = 0.0;
            for (int j = l + 1; j < k; ++j) tail += (gam(P, j + 1) - gam(P, j)) * sb[j];
            v[l] += S->sigma_vz[l] * (ub[l] + tail - gam(P, l) * sb[l]);
            z[l] += S->sigma_vz[l] * sb[l];
        }
        X->q[pix] -= S->sigma_q * (1.0 + tot);
        /* projection of (v_i, z_i) onto Delta_i * epi(rho_i^*) */
        for (int i = 0; i < k; ++i) {
            double d = gam(P, i + 1) - gam(P, i);
            double yo, ho;
            orc_proj_epi(P, (int)pix, i, v[i] / d, z[i] / d, &yo, &ho);
            v[i] = d * yo;
            z[i] = d * ho;
        }
    }
}

/* The primal half-step: descent on (u, s), u clamped to [0,1]^k, then the
   extrapolation (theta = 1).  dv: Nk work. */
static void primal_half(const orc_problem *P, orc_state *X, const orc_steps *S, double *dv)
{
    int H = P->H, W = P->W, k = P->L - 1, Dz = depth(P);
    size_t N = npix(P);
    orc_div3(Dz, H, W, k, X->px, X->py, Dz > 1 ? X->pz : NULL, dv);
    for (size_t pix = 0; pix < N; ++pix) {
        const double *v = X->v + pix * k, *z = X->z + pix * k;
        double *u = X->u + pix * k, *s = X->s + pix * k;
        double *ub = X->ubar + pix * k, *sb = X->sbar + pix * k;
        double q = X->q[pix], prefix = 0.0;
        for (int i = 0; i < k; ++i) {
            double d = gam(P, i + 1) - gam(P, i);
            double un = clampd(u[i] - S->tau_u * (v[i] - dv[pix * k + i]), 0.0, 1.0);
            double sn = s[i] - S->tau_s[i] * (z[i] - d * q + d * prefix - gam(P, i) * v[i]);
            prefix += v[i];
            ub[i] = 2.0 * un - u[i];
            sb[i] = 2.0 * sn - s[i];
            u[i] = un;
            s[i] = sn;
        }
    }
}

int orc_pdhg(const orc_problem *P, orc_state *X, int iters)
{
    int k = P->L - 1, Dz = depth(P);
    size_t Nk = npix(P) * k;
    if (Dz > 1 && !X->pz) return -2;
    orc_steps S;
    make_steps(P, &S);
    double *gx = (double *)malloc(sizeof(double) * Nk);
    double *gy = (double *)malloc(sizeof(double) * Nk);
    double *gz = (double *)malloc(sizeof(double) * Nk);
    double *dv = (double *)malloc(sizeof(double) * Nk);
    if (!gx || !gy || !gz || !dv) {
        free(gx); free(gy); free(gz); free(dv); free_steps(&S); return -1;
    }
    for (int n = 0; n < iters; ++n) {
        dual_half(P, X, &S, gx, gy, gz);
        primal_half(P, X, &S, dv);
    }
    free(gx); free(gy); free(gz); free(dv);
    free_steps(&S);
    return 0;
}

/* One half-step alone (half = 0: dual, 1: primal), for a caller that works
   between the two (the exchange of halo rows between the bands of an image). */
int orc_half_step(const orc_problem *P, orc_state *X, int half)
{
    int k = P->L - 1, Dz = depth(P);
    size_t Nk = npix(P) * k;
    if (Dz > 1 && !X->pz) return -2;
    orc_steps S;
    make_steps(P, &S);
    double *a = (double *)malloc(sizeof(double) * Nk);
    double *b = (double *)malloc(sizeof(double) * Nk);
    double *c = (double *)malloc(sizeof(double) * Nk);
    if (!a || !b || !c) {
        free(a); free(b); free(c); free_steps(&S); return -1;
    }
    if (half == 0) dual_half(P, X, &S, a, b, c);
    else primal_half(P, X, &S, a);
    free(a); free(b); free(c);
    free_steps(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Unlifting by the layer-cake formula (Sec. 3), on the clamped iterate.     */
/* ------------------------------------------------------------------------ */
void orc_unlift(const orc_problem *P, const double *u, double *out)
{
    int k = P->L - 1;
    size_t N = npix(P);
    for (size_t pix = 0; pix < N; ++pix) {
        double a = gam(P, 0);
        for (int i = 0; i < k; ++i)
            a += clampd(u[pix * k + i], 0.0, 1.0) * (gam(P, i + 1) - gam(P, i));
        out[pix] = a;
    }
}

/* Projection onto {1 >= w_1 >= ... >= w_k >= 0}: pool adjacent violators for
   the non-increasing order, then clamp to [0,1]. */
void orc_monotone_proj(int k, const double *u, double *w)
{
    double *val = (double *)malloc(sizeof(double) * k);
    int *cnt = (int *)malloc(sizeof(int) * k);
    int nb = 0;
    for (int i = 0; i < k; ++i) {
        val[nb] = u[i];
        cnt[nb] = 1;
        ++nb;
        while (nb > 1 && val[nb - 2] < val[nb - 1]) {
            double tot = val[nb - 2] * cnt[nb - 2] + val[nb - 1] * cnt[nb - 1];
            cnt[nb - 2] += cnt[nb - 1];
            val[nb - 2] = tot / cnt[nb - 2];
            --nb;
        }
    }
    int o = 0;
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < cnt[b]; ++c) w[o++] = clampd(val[b], 0.0, 1.0);
    free(val);
    free(cnt);
}

/* ------------------------------------------------------------------------ */
/* Energies.                                                                 */
/*  D   : dual bound.  With p in K and q(x) = max_i rho_i^*(v(x)) (the        */
/*        smallest q allowed by C), minimising the Lagrangian over            */
/*        u in [0,1]^k gives sum_x sum_i min(0, v_i - (div p)_i) - q(x).      */
/*  Phat: relaxed energy of an explicit feasible point.  u is projected onto  */
/*        the monotone set; its data term is bounded by a decomposition of    */
/*        u into points of the graph pieces, u = sum_i lam_i 1_i^{a_i}, whose */
/*        tail sums S_i = sum_{j>=i} lam_j must interleave u (S_{i+1} <= u_i  */
/*        <= S_i).  The masses come from the multiplier s (-Delta_i s_i),     */
/*        clamped into the interleaving intervals; the TV term is             */
/*        lambda sum_i Delta_i |grad u_i| (Prop. 5).                          */
/*  Enc : nonconvex energy of the unlifted image,                             */
/*        sum_x rho(x, u~) + lambda sum_x |grad u~|_2.                        */
/* ------------------------------------------------------------------------ */
void orc_energy(const orc_problem *P, const orc_state *X, double *Phat,
                double *Dual, double *Enc)
{
    int H = P->H, W = P->W, k = P->L - 1, Dz = depth(P);
    size_t N = npix(P), Nk = N * k;
    double *dv = (double *)malloc(sizeof(double) * Nk);
    double *uf = (double *)malloc(sizeof(double) * Nk);
    double *gx = (double *)malloc(sizeof(double) * Nk);
    double *gy = (double *)malloc(sizeof(double) * Nk);
    double *gz = (double *)malloc(sizeof(double) * Nk);
    double *ut = (double *)malloc(sizeof(double) * N);
    double *S = (double *)malloc(sizeof(double) * (k + 1));

    /* dual bound */
    orc_div3(Dz, H, W, k, X->px, X->py, Dz > 1 ? X->pz : NULL, dv);
    double D = 0.0;
    for (size_t pix = 0; pix < N; ++pix) {
        double a = 0.0;
        for (int i = 0; i < k; ++i) {
            double g = X->v[pix * k + i] - dv[pix * k + i];
            a += g < 0.0 ? g : 0.0;
        }
        a -= orc_lifted_conj(P, (int)pix, X->v + pix * k);
        D += a;
    }

    /* primal bound */
    double Pd = 0.0;
    for (size_t pix = 0; pix < N; ++pix) {
        const double *s = X->s + pix * k;
        double *w = uf + pix * k;
        orc_monotone_proj(k, X->u + pix * k, w);
        S[0] = 1.0;
        S[k] = 0.0;
        double tail = 0.0;
        for (int i = k - 1; i >= 1; --i) {
            tail += -(gam(P, i + 1) - gam(P, i)) * s[i];
            S[i] = clampd(tail, w[i], w[i - 1]);
        }
        for (int i = 0; i < k; ++i) {
            double li = S[i] - S[i + 1];
            if (li <= 0.0) continue;
            double a = clampd((w[i] - S[i + 1]) / li, 0.0, 1.0);
            double d = gam(P, i + 1) - gam(P, i);
            Pd += li * orc_biconj(P, (int)pix, i, gam(P, i) + a * d);
        }
    }
    orc_grad3(Dz, H, W, k, uf, gx, gy, gz);
    double tv = 0.0;
    for (size_t o = 0; o < Nk; ++o) {
        int i = (int)(o % k);
        tv += (gam(P, i + 1) - gam(P, i)) * tv_norm(P->aniso, gx[o], gy[o], gz[o]);
    }
    Pd += P->lam * tv;

    /* nonconvex energy of the unlifted image (volume) */
    orc_unlift(P, X->u, ut);
    orc_grad3(Dz, H, W, 1, ut, gx, gy, gz);
    double E = 0.0;
    for (size_t pix = 0; pix < N; ++pix)
        E += orc_rho(P, (int)pix, ut[pix]) + P->lam * tv_norm(P->aniso, gx[pix], gy[pix], gz[pix]);

    *Phat = Pd;
    *Dual = D;
    *Enc = E;
    free(dv); free(uf); free(gx); free(gy); free(gz); free(ut); free(S);
}

/* ------------------------------------------------------------------------ */
/* Independent side solver: box-constrained ROF, unlifted,                   */
/*   min_{u in [lo,hi]} sum alpha/2 (u-f)^2 + lambda sum |grad u|_2,         */
/* by the accelerated primal-dual method of Chambolle and Pock (their        */
/* Algorithm 2, strong convexity alpha).  Used only to pin Prop. 3 (L = 2)   */
/* and the tightness of the relaxation for convex data terms.               */
/* Returns the final primal-dual gap.                                        */
/* ------------------------------------------------------------------------ */
static double rof_primal(int D, int H, int W, const double *u, const double *f,
                         double alpha, double lam, int aniso)
{
    size_t N = (size_t)D * H * W;
    double *gx = (double *)malloc(sizeof(double) * N);
    double *gy = (double *)malloc(sizeof(double) * N);
    double *gz = (double *)malloc(sizeof(double) * N);
    orc_grad3(D, H, W, 1, u, gx, gy, gz);
    double e = 0.0;
    for (size_t o = 0; o < N; ++o)
        e += 0.5 * alpha * (u[o] - f[o]) * (u[o] - f[o]) + lam * tv_norm(aniso, gx[o], gy[o], gz[o]);
    free(gx); free(gy); free(gz);
    return e;
}

/* On a D x H x W volume (D = 1: an image); |grad|^2 <= 4 * (number of axes),
   so tau = sigma = 1/sqrt(4 * axes) start the accelerated steps. */
double orc_rof_direct3(int D, int H, int W, const double *f, double alpha, double lam,
                       double lo, double hi, int iters, int aniso, double *u)
{
    size_t N = (size_t)D * H * W;
    double *px = (double *)calloc(N, sizeof(double));
    double *py = (double *)calloc(N, sizeof(double));
    double *pz = (double *)calloc(N, sizeof(double));
    double *ub = (double *)malloc(sizeof(double) * N);
    double *dv = (double *)malloc(sizeof(double) * N);
    double *gx = (double *)malloc(sizeof(double) * N);
    double *gy = (double *)malloc(sizeof(double) * N);
    double *gz = (double *)malloc(sizeof(double) * N);
    for (size_t o = 0; o < N; ++o) { u[o] = clampd(f[o], lo, hi); ub[o] = u[o]; }
    double axes = D > 1 ? 3.0 : 2.0;
    double tau = 1.0 / sqrt(4.0 * axes), sigma = 1.0 / sqrt(4.0 * axes);
    for (int n = 0; n < iters; ++n) {
        orc_grad3(D, H, W, 1, ub, gx, gy, gz);
        for (size_t o = 0; o < N; ++o) {
            double ax = px[o] + sigma * gx[o], ay = py[o] + sigma * gy[o];
            double az = pz[o] + sigma * gz[o];
            tv_project(aniso, lam, &ax, &ay, &az);
            px[o] = ax;
            py[o] = ay;
            pz[o] = az;
        }
        orc_div3(D, H, W, 1, px, py, pz, dv);
        double theta = 1.0 / sqrt(1.0 + 2.0 * alpha * tau);
        for (size_t o = 0; o < N; ++o) {
            double un = (u[o] + tau * dv[o] + tau * alpha * f[o]) / (1.0 + tau * alpha);
            un = clampd(un, lo, hi);
            ub[o] = un + theta * (un - u[o]);
            u[o] = un;
        }
        tau *= theta;
        sigma /= theta;
    }
    /* gap: primal energy minus the dual objective of the box-constrained
       problem, min_{u in box} alpha/2 (u-f)^2 - u*div p, per pixel */
    orc_div3(D, H, W, 1, px, py, pz, dv);
    double dual = 0.0;
    for (size_t o = 0; o < N; ++o) {
        double t = clampd(f[o] + dv[o] / alpha, lo, hi);
        dual += 0.5 * alpha * (t - f[o]) * (t - f[o]) - t * dv[o];
    }
    double gap = rof_primal(D, H, W, u, f, alpha, lam, aniso) - dual;
    free(px); free(py); free(pz); free(ub); free(dv); free(gx); free(gy); free(gz);
    return gap;
}

double orc_rof_energy3(int D, int H, int W, const double *u, const double *f,
                       double alpha, double lam, int aniso)
{
    return rof_primal(D, H, W, u, f, alpha, lam, aniso);
}

/* Image forms, isotropic |grad u|_2 and anisotropic |grad u|_1. */
double orc_rof_direct(int H, int W, const double *f, double alpha, double lam,
                      double lo, double hi, int iters, double *u)
{
    return orc_rof_direct3(1, H, W, f, alpha, lam, lo, hi, iters, 0, u);
}

double orc_rof_energy(int H, int W, const double *u, const double *f,
                      double alpha, double lam)
{
    return rof_primal(1, H, W, u, f, alpha, lam, 0);
}

double orc_rof_direct_aniso(int H, int W, const double *f, double alpha, double lam,
                            double lo, double hi, int iters, double *u)
{
    return orc_rof_direct3(1, H, W, f, alpha, lam, lo, hi, iters, 1, u);
}

double orc_rof_energy_aniso(int H, int W, const double *u, const double *f,
                            double alpha, double lam)
{
    return rof_primal(1, H, W, u, f, alpha, lam, 1);
}

/* ------------------------------------------------------------------------ */
/* Reverse mode through `iters` unrolled PDHG iterations from the zero       */
/* state (the differentiable solve; not part of the paper).  Given           */
/* g_u = dL/du~ of the final unlifted image u~ = gamma_1 + sum_i Delta u_i,   */
/* returns dL/df (per pixel) and dL/d{lambda, alpha, nu}.                     */
/* All states are stored; each step is pulled back in reverse order.  The    */
/* local Jacobians of the epigraph projections (w.r.t. the projected point   */
/* and f, alpha, nu) are taken by central differences of orc_proj_epi in     */
/* FP64; the clamp and the l2-ball projection are differentiated by hand.   */
/* Kinks of the unrolled map (clamp bounds, ball boundary, projection-region */
/* boundaries) are taken as not hit.                                          */
/* ------------------------------------------------------------------------ */
static void proj_jacobian(const orc_problem *P, int pix, int i, double y0, double h0,
                          double J[2][5])
{
    /* columns: y0, h0, f(pix), alpha, nu */
    orc_problem Q = *P;
    double fv = P->f ? P->f[pix] : 0.0;
    double base[5] = {y0, h0, fv, P->alpha, P->nu};
    for (int c = 0; c < 5; ++c) {
        if (c >= 2 && P->kind == ORC_PL) { J[0][c] = J[1][c] = 0.0; continue; }
        if (c == 4 && P->kind != ORC_TRUNC) { J[0][c] = J[1][c] = 0.0; continue; }
        double hstep = 1e-8 * (1.0 + fabs(base[c]));
        double out[2][2];
        for (int sgn = 0; sgn < 2; ++sgn) {
            double a[5] = {base[0], base[1], base[2], base[3], base[4]};
            a[c] += sgn ? hstep : -hstep;
            double fl = a[2];
            Q.f = &fl;
            Q.alpha = a[3];
            Q.nu = a[4];
            double yo, ho;
            orc_proj_epi(&Q, 0, i, a[0], a[1], &yo, &ho);
            out[sgn][0] = yo;
            out[sgn][1] = ho;
        }
        J[0][c] = (out[1][0] - out[0][0]) / (2.0 * hstep);
        J[1][c] = (out[1][1] - out[0][1]) / (2.0 * hstep);
    }
}

int orc_unrolled_grad(const orc_problem *P, int iters, const double *g_u, double *grad_f,
                      double *grad_scal)
{
    int H = P->H, W = P->W, k = P->L - 1;
    size_t N = (size_t)H * W, Nk = N * k;
    if (P->kind == ORC_PL) return -2;
    if (depth(P) > 1) return -3;          /* images only */
    orc_steps S;
    make_steps(P, &S);
    /* stored states: per state u,s,ubar,sbar,v,z,px,py (Nk each) + q (N) */
    size_t per = 8 * Nk + N;
    double *st = (double *)calloc(per * (size_t)(iters + 1), sizeof(double));
    double *ax = (double *)calloc(2 * Nk, sizeof(double));   /* u, s */
    double *axb = (double *)calloc(2 * Nk, sizeof(double));  /* ubar, sbar */
    double *ay = (double *)calloc(4 * Nk, sizeof(double));   /* v, z, px, py */
    double *aq = (double *)calloc(N, sizeof(double));
    double *gu = (double *)calloc(Nk, sizeof(double));
    double *gs = (double *)calloc(Nk, sizeof(double));
    double *Aa = (double *)calloc(2 * Nk, sizeof(double));
    double *dv = (double *)malloc(sizeof(double) * Nk);
    if (!st || !ax || !axb || !ay || !aq || !gu || !gs || !Aa || !dv) {
        free(st); free(ax); free(axb); free(ay); free(aq); free(gu); free(gs); free(Aa); free(dv);
        free_steps(&S);
        return -1;
    }
#define ST(n, f) (st + (size_t)(n) * per + (size_t)(f) * Nk)
    /* forward, keeping every state (state 0 = all zeros) */
    for (int n = 0; n < iters; ++n) {
        memcpy(ST(n + 1, 0), ST(n, 0), sizeof(double) * per);
        orc_state X = {ST(n + 1, 0), ST(n + 1, 1), ST(n + 1, 2), ST(n + 1, 3), ST(n + 1, 4),
                       ST(n + 1, 5), ST(n + 1, 6), ST(n + 1, 7), ST(n + 1, 8), NULL};
        orc_pdhg(P, &X, 1);
    }
    /* seed: dL/du_i = Delta_i dL/du~ */
    for (size_t pix = 0; pix < N; ++pix)
        for (int i = 0; i < k; ++i)
            ax[2 * (pix * k + i)] = (gam(P, i + 1) - gam(P, i)) * g_u[pix];
    for (size_t pix = 0; pix < N; ++pix) grad_f[pix] = 0.0;
    grad_scal[0] = grad_scal[1] = grad_scal[2] = 0.0;

    for (int n = iters - 1; n >= 0; --n) {
        const double *u0 = ST(n, 0), *ub0 = ST(n, 2), *sb0 = ST(n, 3);
        const double *v0 = ST(n, 4), *z0 = ST(n, 5), *px0 = ST(n, 6), *py0 = ST(n, 7);
        const double *v1 = ST(n + 1, 4), *px1 = ST(n + 1, 6), *py1 = ST(n + 1, 7);
        /* ---- primal step: u' = clamp(u - tau_u (v - div p)), s' = ..., xbar' = 2x' - x */
        orc_div(H, W, k, px1, py1, dv);
        for (size_t o = 0; o < Nk; ++o) {
            double w = u0[o] - S.tau_u * (v1[o] - dv[o]);
            double m = (w > 0.0 && w < 1.0) ? 1.0 : 0.0;
            gu[o] = m * (ax[2 * o] + 2.0 * axb[2 * o]);
            gs[o] = ax[2 * o + 1] + 2.0 * axb[2 * o + 1];
            ax[2 * o] = gu[o] - axb[2 * o];
            ax[2 * o + 1] = gs[o] - axb[2 * o + 1];
        }
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t pix = (size_t)y * W + x;
                for (int l = 0; l < k; ++l) {
                    size_t o = pix * k + l;
                    double d = gam(P, l + 1) - gam(P, l);
                    /* s_i uses v_l (l < i) through Delta * sum_{l<i} v_l and v_i through -gamma_i v_i */
                    double acc = -S.tau_u * gu[o] + S.tau_s[l] * gam(P, l) * gs[o];
                    for (int i = l + 1; i < k; ++i)
                        acc -= S.tau_s[i] * (gam(P, i + 1) - gam(P, i)) * gs[pix * k + i];
                    ay[4 * o + 0] += acc;
                    ay[4 * o + 1] += -S.tau_s[l] * gs[o];
                    aq[pix] += S.tau_s[l] * d * gs[o];
                    /* div p = -grad^T p: d u'/d px(x) = tau_u ([x<W-1] g(x) - g(x+1)) */
                    if (x + 1 < W) ay[4 * o + 2] += S.tau_u * (gu[o] - gu[o + k]);
                    if (y + 1 < H) ay[4 * o + 3] += S.tau_u * (gu[o] - gu[o + (size_t)W * k]);
                }
            }
        /* ---- dual step from (xbar_n, y_n, q_n) */
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t pix = (size_t)y * W + x;
                double adjv[LIFT_ORACLE_MAXK];
                for (int i = 0; i < k; ++i) {
                    size_t o = pix * k + i;
                    double d = gam(P, i + 1) - gam(P, i);
                    /* TV part */
                    double gx = x + 1 < W ? ub0[o + k] - ub0[o] : 0.0;
                    double gy = y + 1 < H ? ub0[o + (size_t)W * k] - ub0[o] : 0.0;
                    double a0 = px0[o] + S.sigma_p * gx, a1 = py0[o] + S.sigma_p * gy;
                    double nrm = sqrt(a0 * a0 + a1 * a1), R = P->lam * d;
                    double ap0 = ay[4 * o + 2], ap1 = ay[4 * o + 3];
                    double aa0 = ap0, aa1 = ap1;
                    if (P->aniso) {
                        /* componentwise clamp to [-R, R]: identity inside,
                           the bound (dR/dlambda = Delta) outside */
                        if (fabs(a0) > R) { grad_scal[0] += d * (a0 > 0 ? 1.0 : -1.0) * ap0; aa0 = 0.0; }
                        if (fabs(a1) > R) { grad_scal[0] += d * (a1 > 0 ? 1.0 : -1.0) * ap1; aa1 = 0.0; }
                    } else if (nrm > R) {
                        double h0 = a0 / nrm, h1 = a1 / nrm, dot = h0 * ap0 + h1 * ap1;
                        aa0 = (R / nrm) * (ap0 - h0 * dot);
                        aa1 = (R / nrm) * (ap1 - h1 * dot);
                        grad_scal[0] += d * dot;
                    }
                    Aa[2 * o] = aa0;
                    Aa[2 * o + 1] = aa1;
                    /* data part: v^ = v + sigma (ubar + Delta sum_{j>i} sbar_j - gamma_i sbar_i),
                       z^ = z + sigma sbar, (v', z') = Delta Proj((v^, z^)/Delta) */
                    double tail = 0.0;
                    for (int j = i + 1; j < k; ++j) tail += (gam(P, j + 1) - gam(P, j)) * sb0[pix * k + j];
                    double vh = v0[o] + S.sigma_vz[i] * (ub0[o] + tail - gam(P, i) * sb0[o]);
                    double zh = z0[o] + S.sigma_vz[i] * sb0[o];
                    double J[2][5];
                    proj_jacobian(P, (int)pix, i, vh / d, zh / d, J);
                    double avv = ay[4 * o], avz = ay[4 * o + 1];
                    double adv = avv * J[0][0] + avz * J[1][0];
                    double adz = avv * J[0][1] + avz * J[1][1];
                    grad_f[pix] += d * (avv * J[0][2] + avz * J[1][2]);
                    grad_scal[1] += d * (avv * J[0][3] + avz * J[1][3]);
                    grad_scal[2] += d * (avv * J[0][4] + avz * J[1][4]);
                    adjv[i] = adv;
                    ay[4 * o + 0] = adv;
                    ay[4 * o + 1] = adz;
                    ay[4 * o + 2] = aa0;
                    ay[4 * o + 3] = aa1;
                    /* adjoint of xbar_n: own terms */
                    double au = S.sigma_vz[i] * adv;
                    if (x + 1 < W) au -= S.sigma_p * aa0;
                    if (y + 1 < H) au -= S.sigma_p * aa1;
                    axb[2 * o] = au;
                    axb[2 * o + 1] = -S.sigma_vz[i] * gam(P, i) * adv + S.sigma_vz[i] * adz
                                     - S.sigma_q * d * aq[pix];
                }
                /* sbar_j enters v^_l (l < j) through the tail sums */
                for (int j = 0; j < k; ++j) {
                    double dj = gam(P, j + 1) - gam(P, j), acc = 0.0;
                    for (int l = 0; l < j; ++l) acc += S.sigma_vz[l] * adjv[l];
                    axb[2 * (pix * k + j) + 1] += dj * acc;
                }
            }
        /* neighbours' part of grad^T: a(x-1) and a(x-W) used ubar(x) */
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int i = 0; i < k; ++i) {
                    size_t o = ((size_t)y * W + x) * k + i;
                    if (x > 0) axb[2 * o] += S.sigma_p * Aa[2 * (o - k)];
                    if (y > 0) axb[2 * o] += S.sigma_p * Aa[2 * (o - (size_t)W * k) + 1];
                }
    }
#undef ST
    free(st); free(ax); free(axb); free(ay); free(aq); free(gu); free(gs); free(Aa); free(dv);
    free_steps(&S);
    return 0;
}
