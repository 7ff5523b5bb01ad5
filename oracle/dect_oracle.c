/*
 * FP64 CPU oracle for the dual-energy CT hot path (TEST INFRASTRUCTURE ONLY).
 *
 * Plain, slow, obviously correct restatement of what the paper computes:
 *   - Siddon system matrix A of Eq. (1) (Sec. 2.1; Siddon's method, ref. [42]),
 *   - forward projection A x and its transpose A^T y,
 *   - the backward-difference gradient and isotropic TV of Eq. (2),
 *   - the isotropic shrinkage that solves the z-subproblem, Eq. (8),
 *   - the ADM iteration of Eq. (7)/(9)/(10) with the gradient G_f of Eq. (9),
 *   - the 2x2 material decomposition of Eq. (11)-(12),
 *   - the Prewitt edge map and weights e_ik of Eq. (14) (Sec. 2.3),
 *   - the PLS normal equation of Eq. (13)-(15) solved by Jacobi-preconditioned CG.
 *
 * Only the tests, the package smoke check and the benchmark's CPU-baseline leg
 * load this library.  It shares no code, header or table with the CUDA path.
 * Compile with -ffp-contract=off so that a*b+c is never fused: the same
 * source then gives the same bits on x86-64 and on AArch64.
 *
 * Readings of places where the paper is silent or garbled (each one is also
 * listed with the design notes):
 *   R1 Eq. (8): z = max(|w| - 1/rho, 0) * w/|w| with w = grad f - lambda/rho,
 *      z = 0 where |w| = 0 (the exact minimiser of the z-line of Eq. (7)).
 *   R2 lambda and z have the shape of grad f: two components per pixel.
 *   R3 the TV of Eq. (4) acts on each energy channel separately, so the
 *      stacked problem of Eq. (3) splits into one ADM per channel.  The
 *      other reading, one TV over the stacked image f, is kept as a variant:
 *      the norm at each pixel is taken over both channels' gradients
 *      (orc_adm_joint_*), the z-step shrinks 4-vectors and one step alpha
 *      serves the stacked f.
 *   R5 xi (multiplier step) is a parameter; the default elsewhere is xi = rho.
 *   R6 "BB-like" step: with c(G) = |G|^2 / (mu |A G|^2 + rho |grad G|^2)
 *      (the exact line-search step of the quadratic f-subproblem along -G),
 *      rule BB1 uses alpha^k = c(G^{k-1}) (alpha^0 = c(G^0)), which is the
 *      Barzilai-Borwein step s's/s'y of the previous step; rule CAUCHY uses
 *      alpha^k = c(G^k).  Without the line search of the full method the
 *      lagged step is strongly non-monotone on sparse-view data, so CAUCHY is
 *      the default of the callers; both rules are kept.
 *   R7 Eq. (2) differences with an index outside the image are 0.
 *      i = row (y), j = column (x).
 *   R8 no projection onto x >= 0 (Eq. (10) has none); optionally (nonneg = 1)
 *      f is projected onto f >= 0 right after the f-step.
 *   R10 Siddon segments between consecutive sorted crossing parameters go to
 *      the pixel that holds the segment midpoint; zero-length ones are dropped;
 *      consecutive pieces given to the same pixel (a crossing within rounding
 *      of a grid corner) are summed into one element a_ij.
 *   R13 Eq. (15) with Hessian(R) = 2 L_e reads (I + gamma L_e) u = D^{-1} x.
 *   R14 edges: 3x3 Prewitt magnitude of x_h and x_l (replicate padding), each
 *      divided by its maximum; a pixel is an edge if either exceeds tau;
 *      e_ik = eps if pixel i or k is an edge, else 1.  Magnitudes, maxima
 *      and the comparison with tau are FP64.
 *   R16 PCG: Jacobi preconditioner, initial guess D^{-1} x.
 *   R19 cone-beam geometry (Sec. 2.1, Fig. 1, Sec. 3): circular orbit in the
 *      plane z = 0, flat 2-D detector (rows along z), one ray per detector
 *      cell from the source point to the cell centre; Siddon in 3-D with the
 *      rule of R10 (a ray on a slice boundary goes to the +z voxel).
 *   R20 3-D edge weights: Prewitt in 3-D (each component the difference of
 *      the two neighbours along its axis summed over the 3 x 3 neighbourhood
 *      of the other two axes, replicate padding); N_i of Eq. (14) is the 6
 *      face neighbours of a voxel inside the volume.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Fan-beam slice geometry (Sec. 2.1, Fig. 1; Sec. 3). Units mm and rad. */
typedef struct {
    int n;            /* image n x n */
    double px;        /* pixel side */
    int nv;           /* views */
    int nb;           /* detector bins */
    double pitch;     /* bin pitch */
    double sod;       /* source to isocentre */
    double sdd;       /* source to detector */
    double start;     /* angle of view 0 */
    double arc;       /* angular range covered by the nv views */
    double det_offset;
} orc_geom;

/* ------------------------------------------------------------------------ */
/* Geometry: one ray per bin, from the source point to the bin centre.       */
/* ------------------------------------------------------------------------ */
void orc_ray(const orc_geom *g, int v, int b, double S[2], double D[2])
{
    double th = g->start + (double)v * (g->arc / (double)g->nv);
    double c = cos(th), s = sin(th);
    S[0] = g->sod * c;
    S[1] = g->sod * s;
    double cx = (g->sod - g->sdd) * c, cy = (g->sod - g->sdd) * s;
    double u = ((double)b - 0.5 * (double)(g->nb - 1)) * g->pitch + g->det_offset;
    D[0] = cx - u * s;
    D[1] = cy + u * c;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/*
 * Siddon's method (ref. [42]) for ray (v, b): the ray is P(a) = S + a (D - S),
 * a in [0, 1].  All crossing parameters of the pixel-grid lines inside the
 * image box are collected, sorted, de-duplicated, and each piece between
 * consecutive parameters is given to the pixel holding its midpoint (R10).
 * Writes up to `cap` (pixel index, length in mm) pairs; returns the count.
 * Pixel index = row * n + col, row = y, col = x.
 */
int orc_siddon_ray(const orc_geom *g, int v, int b, int32_t *idx, double *len, int cap)
{
    double S[2], D[2];
    orc_ray(g, v, b, S, D);
    const int n = g->n;
    const double dx = D[0] - S[0], dy = D[1] - S[1];
    const double L = sqrt(dx * dx + dy * dy);
    const double lo = -0.5 * (double)n * g->px;
    const double hi = lo + (double)n * g->px;

    double amin = 0.0, amax = 1.0;
    if (dx != 0.0) {
        double t0 = (lo - S[0]) / dx, t1 = (hi - S[0]) / dx;
        amin = fmax(amin, fmin(t0, t1));
        amax = fmin(amax, fmax(t0, t1));
    } else if (!(S[0] >= lo && S[0] < hi)) {
        return 0;
    }
    if (dy != 0.0) {
        double t0 = (lo - S[1]) / dy, t1 = (hi - S[1]) / dy;
        amin = fmax(amin, fmin(t0, t1));
        amax = fmin(amax, fmax(t0, t1));
    } else if (!(S[1] >= lo && S[1] < hi)) {
        return 0;
    }
    if (!(amin < amax)) return 0;

    double *a = (double *)malloc(sizeof(double) * (size_t)(2 * n + 6));
    int na = 0;
    a[na++] = amin;
    a[na++] = amax;
    for (int k = 0; k <= n; ++k) {
        double plane = lo + (double)k * g->px;
        if (dx != 0.0) {
            double t = (plane - S[0]) / dx;
            if (t > amin && t < amax) a[na++] = t;
        }
        if (dy != 0.0) {
            double t = (plane - S[1]) / dy;
            if (t > amin && t < amax) a[na++] = t;
        }
    }
    qsort(a, (size_t)na, sizeof(double), cmp_double);

    int cnt = 0, last = -1;
    for (int k = 0; k + 1 < na; ++k) {
        double a0 = a[k], a1 = a[k + 1];
        if (!(a1 > a0)) continue;                 /* duplicate (corner) */
        double mid = 0.5 * (a0 + a1);
        double xm = S[0] + mid * dx, ym = S[1] + mid * dy;
        int col = (int)floor((xm - lo) / g->px);
        int row = (int)floor((ym - lo) / g->px);
        if (col < 0 || col >= n || row < 0 || row >= n) continue;
        int pix = row * n + col;
        double seg = (a1 - a0) * L;
        /* a_ij is the whole length of ray i in pixel j: a crossing within
           rounding of a grid corner can split it into two pieces that the
           midpoint rule gives to the same pixel; they are summed. */
        if (cnt > 0 && last == pix) {
            if (cnt - 1 < cap) len[cnt - 1] += seg;
            continue;
        }
        if (cnt < cap) {
            idx[cnt] = pix;
            len[cnt] = seg;
        }
        last = pix;
        ++cnt;
    }
    free(a);
    return cnt;
}

/* Number of (ray, pixel) intersections of the whole geometry. */
int64_t orc_table_nnz(const orc_geom *g)
{
    int cap = 4 * g->n + 8;
    int32_t *ti = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    double *tl = (double *)malloc(sizeof(double) * (size_t)cap);
    int64_t total = 0;
    for (int v = 0; v < g->nv; ++v)
        for (int b = 0; b < g->nb; ++b)
            total += orc_siddon_ray(g, v, b, ti, tl, cap);
    free(ti);
    free(tl);
    return total;
}

/* Ray-major table of A (row r = v * nb + b): rowptr[M + 1], idx[nnz], len[nnz]. */
void orc_table_build(const orc_geom *g, int64_t *rowptr, int32_t *idx, double *len)
{
    int cap = 4 * g->n + 8;
    int64_t pos = 0;
    rowptr[0] = 0;
    for (int v = 0; v < g->nv; ++v)
        for (int b = 0; b < g->nb; ++b) {
            int c = orc_siddon_ray(g, v, b, idx + pos, len + pos, cap);
            pos += c;
            rowptr[(int64_t)v * g->nb + b + 1] = pos;
        }
}

/* y = A x  (Eq. (1)). */
void orc_project(int64_t m, const int64_t *rowptr, const int32_t *idx, const double *len,
                 const double *x, double *y)
{
    for (int64_t r = 0; r < m; ++r) {
        double s = 0.0;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += len[k] * x[idx[k]];
        y[r] = s;
    }
}

/* x = A^T y: the transpose, written as the scatter of each row. */
void orc_backproject(int64_t m, int64_t npix, const int64_t *rowptr, const int32_t *idx,
                     const double *len, const double *y, double *x)
{
    for (int64_t j = 0; j < npix; ++j) x[j] = 0.0;
    for (int64_t r = 0; r < m; ++r)
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) x[idx[k]] += len[k] * y[r];
}

/* ------------------------------------------------------------------------ */
/* Eq. (2): backward differences, gradient layout d[2][n][n]:                */
/*   d[0][i][j] = x[i][j] - x[i-1][j]   (along rows, i = y)                  */
/*   d[1][i][j] = x[i][j] - x[i][j-1]   (along columns, j = x)               */
/* with 0 where i-1 or j-1 is outside the image (R7).                         */
/* ------------------------------------------------------------------------ */
void orc_grad(int n, const double *x, double *d)
{
    int64_t N = (int64_t)n * n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int64_t p = (int64_t)i * n + j;
            d[p] = (i > 0) ? x[p] - x[p - n] : 0.0;
            d[N + p] = (j > 0) ? x[p] - x[p - 1] : 0.0;
        }
}

/* out = grad^T d, the exact transpose of orc_grad. */
void orc_grad_t(int n, const double *d, double *out)
{
    int64_t N = (int64_t)n * n;
    for (int64_t p = 0; p < N; ++p) out[p] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int64_t p = (int64_t)i * n + j;
            if (i > 0) { out[p] += d[p]; out[p - n] -= d[p]; }
            if (j > 0) { out[p] += d[N + p]; out[p - 1] -= d[N + p]; }
        }
}

/* Isotropic TV, Eq. (2): sum over pixels of |grad x|. */
double orc_tv(int n, const double *x)
{
    int64_t N = (int64_t)n * n;
    double *d = (double *)malloc(sizeof(double) * (size_t)(2 * N));
    orc_grad(n, x, d);
    double s = 0.0;
    for (int64_t p = 0; p < N; ++p) s += sqrt(d[p] * d[p] + d[N + p] * d[N + p]);
    free(d);
    return s;
}

/* Eq. (8) under reading R1: per pixel, z = max(|w| - t, 0) w / |w|. */
void orc_shrink(int64_t npix, const double *w, double t, double *z)
{
    for (int64_t p = 0; p < npix; ++p) {
        double a = w[p], b = w[npix + p];
        double nrm = sqrt(a * a + b * b);
        double s = nrm - t;
        if (s > 0.0 && nrm > 0.0) {
            z[p] = s * a / nrm;
            z[npix + p] = s * b / nrm;
        } else {
            z[p] = 0.0;
            z[npix + p] = 0.0;
        }
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* ADM parameters for one channel (Eq. (6)-(10)). */
typedef struct {
    double mu, rho, xi;
    int step_rule;     /* 0 = BB1 (lagged exact step), 1 = CAUCHY (R6) */
    int max_iter;
    double tol;        /* stop when |Phi_{k+1} - Phi_k| / Phi_k < tol; 0 = run max_iter */
    int nonneg;        /* 1: project f onto f >= 0 after the f-step (x in R_+^N, Eq. (1)) */
} orc_adm_params;

/* ADM state of one channel (sizes: f N, z 2N, lam 2N). */
typedef struct {
    double *f, *z, *lam;
    double alpha_prev;  /* c(G^{k-1}) for rule BB1; < 0 before the first step */
} orc_adm_state;

/*
 * One ADM iteration, Eq. (10), for the channel problem
 *   min ||grad f|| + mu/2 ||A f - g||^2:
 *   z^{k+1}  = shrink(grad f^k - lam^k / rho, 1/rho)                      Eq. (8)
 *   G^k      = mu A^T (A f^k - g) + rho grad^T(grad f^k - z^{k+1})
 *              - grad^T lam^k                                             Eq. (9)
 *   alpha^k  = BB-like step (R6)
 *   f^{k+1}  = f^k - alpha^k G^k                                          Eq. (9)
 *   lam^{k+1}= lam^k - xi (grad f^{k+1} - z^{k+1})                        Eq. (7)
 * Returns the step used.  Optional outputs (may be NULL): G (N), and
 * norms[3] = { |G|^2, |A G|^2, |grad G|^2 }.
 */
double orc_adm_iterate(int n, int64_t m, const int64_t *rowptr, const int32_t *idx,
                       const double *len, const double *g, const orc_adm_params *prm,
                       orc_adm_state *st, double *G_out, double *norms)
{
    const int64_t N = (int64_t)n * n;
    const double mu = prm->mu, rho = prm->rho, xi = prm->xi;
    double *gf = (double *)malloc(sizeof(double) * (size_t)(2 * N));
    double *w = (double *)malloc(sizeof(double) * (size_t)(2 * N));
    double *r = (double *)malloc(sizeof(double) * (size_t)m);
    double *t1 = (double *)malloc(sizeof(double) * (size_t)N);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)N);
    double *t3 = (double *)malloc(sizeof(double) * (size_t)N);
    double *G = (double *)malloc(sizeof(double) * (size_t)N);
    double *AG = (double *)malloc(sizeof(double) * (size_t)m);
    double *gG = (double *)malloc(sizeof(double) * (size_t)(2 * N));

    /* z-step, Eq. (8) */
    orc_grad(n, st->f, gf);
    for (int64_t p = 0; p < 2 * N; ++p) w[p] = gf[p] - st->lam[p] / rho;
    orc_shrink(N, w, 1.0 / rho, st->z);

    /* G_f, Eq. (9): three terms */
    orc_project(m, rowptr, idx, len, st->f, r);
    for (int64_t i = 0; i < m; ++i) r[i] -= g[i];
    orc_backproject(m, N, rowptr, idx, len, r, t1);
    for (int64_t p = 0; p < 2 * N; ++p) w[p] = gf[p] - st->z[p];
    orc_grad_t(n, w, t2);
    orc_grad_t(n, st->lam, t3);
    for (int64_t p = 0; p < N; ++p) G[p] = mu * t1[p] + rho * t2[p] - t3[p];

    /* step size (R6) */
    orc_project(m, rowptr, idx, len, G, AG);
    orc_grad(n, G, gG);
    double gg = dot(N, G, G), aa = dot(m, AG, AG), dd = dot(2 * N, gG, gG);
    double den = mu * aa + rho * dd;
    double c = (den > 0.0) ? gg / den : 0.0;
    double alpha;
    if (prm->step_rule == 1 || st->alpha_prev < 0.0) alpha = c;
    else alpha = st->alpha_prev;
    st->alpha_prev = c;

    /* f-step (optionally projected onto f >= 0, since x >= 0 in Eq. (1)) and multiplier step */
    for (int64_t p = 0; p < N; ++p) {
        st->f[p] -= alpha * G[p];
        if (prm->nonneg && st->f[p] < 0.0) st->f[p] = 0.0;
    }
    orc_grad(n, st->f, gf);
    for (int64_t p = 0; p < 2 * N; ++p) st->lam[p] -= xi * (gf[p] - st->z[p]);

    if (G_out) memcpy(G_out, G, sizeof(double) * (size_t)N);
    if (norms) { norms[0] = gg; norms[1] = aa; norms[2] = dd; }
    free(gf); free(w); free(r); free(t1); free(t2); free(t3); free(G); free(AG); free(gG);
    return alpha;
}

/* Phi(f) = ||grad f||_TV + mu/2 ||A f - g||^2, the objective of Eq. (4) per channel. */
double orc_objective(int n, int64_t m, const int64_t *rowptr, const int32_t *idx,
                     const double *len, const double *g, double mu, const double *f)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)m);
    orc_project(m, rowptr, idx, len, f, r);
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) { double e = r[i] - g[i]; s += e * e; }
    free(r);
    return orc_tv(n, f) + 0.5 * mu * s;
}

/*
 * The ADM loop of Eq. (10) for one channel, from f (in/out) with z = lam = 0.
 * phi[0..iters] receives Phi(f^k); alpha[0..iters-1] the steps.
 * Stops after max_iter iterations, or once the relative objective change is
 * below tol (tol > 0).  Returns the number of iterations done.
 */
int orc_adm_run(int n, int64_t m, const int64_t *rowptr, const int32_t *idx, const double *len,
                const double *g, const orc_adm_params *prm, double *f, double *phi, double *alpha)
{
    const int64_t N = (int64_t)n * n;
    orc_adm_state st;
    st.f = f;
    st.z = (double *)calloc((size_t)(2 * N), sizeof(double));
    st.lam = (double *)calloc((size_t)(2 * N), sizeof(double));
    st.alpha_prev = -1.0;
    double prev = orc_objective(n, m, rowptr, idx, len, g, prm->mu, f);
    if (phi) phi[0] = prev;
    int k = 0;
    while (k < prm->max_iter) {
        double a = orc_adm_iterate(n, m, rowptr, idx, len, g, prm, &st, NULL, NULL);
        if (alpha) alpha[k] = a;
        ++k;
        double cur = orc_objective(n, m, rowptr, idx, len, g, prm->mu, f);
        if (phi) phi[k] = cur;
        if (prm->tol > 0.0 && prev > 0.0 && fabs(cur - prev) / prev < prm->tol) break;
        prev = cur;
    }
    free(st.z);
    free(st.lam);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Fan-beam filtered backprojection (the analytic reconstruction of         */
/* Sec. 2.4 and Sec. 3), here the textbook algorithm for a flat detector    */
/* with equally spaced bins over a full 360-degree scan (Kak and Slaney,    */
/* Principles of Computerized Tomographic Imaging, ch. 3).  Steps:          */
/*  1. bins moved to a virtual detector through the isocentre:              */
/*     s_b = u_b SOD / SDD, spacing ds = pitch SOD / SDD;                   */
/*  2. cosine pre-weight q = p SOD / sqrt(SOD^2 + s_b^2);                   */
/*  3. ramp filter, the band-limited (Ram-Lak) kernel sampled at ds:        */
/*     h(0) = 1 / (4 ds^2), h(k) = 0 for even k != 0,                       */
/*     h(k) = -1 / (pi^2 k^2 ds^2) for odd k;  qf(b) = ds sum_k q(k) h(b-k);*/
/*  4. backprojection: for a point P and view v with source S, central-ray  */
/*     direction c and lateral direction e (increasing bin index), with     */
/*     d = P - S, L = d.c, the ray through P meets the virtual detector at  */
/*     s = (d.e) SOD / L; f(P) = sum_v (dtheta / 2) (SOD / L)^2 qf(v, s),   */
/*     qf interpolated linearly between bins and 0 outside them.  The 1/2   */
/*     counts each line twice over 360 degrees.                             */
/* ------------------------------------------------------------------------ */

/* Ramp-filtered, cosine-weighted projections qf [nv][nb] (steps 1-3). */
void orc_fbp_filter(const orc_geom *g, const double *p, double *qf)
{
    const int nb = g->nb;
    const double scale = g->sod / g->sdd, ds = g->pitch * scale;
    double *q = (double *)malloc(sizeof(double) * (size_t)nb);
    double *h = (double *)malloc(sizeof(double) * (size_t)(2 * nb - 1));
    const double pi = 3.14159265358979323846;
    for (int k = -(nb - 1); k <= nb - 1; ++k) {
        double v;
        if (k == 0) v = 1.0 / (4.0 * ds * ds);
        else if (k % 2 == 0) v = 0.0;
        else v = -1.0 / (pi * pi * (double)k * (double)k * ds * ds);
        h[k + nb - 1] = v;
    }
    for (int v = 0; v < g->nv; ++v) {
        for (int b = 0; b < nb; ++b) {
            double u = ((double)b - 0.5 * (double)(nb - 1)) * g->pitch + g->det_offset;
            double sb = u * scale;
            q[b] = p[(int64_t)v * nb + b] * g->sod / sqrt(g->sod * g->sod + sb * sb);
        }
        for (int b = 0; b < nb; ++b) {
            double acc = 0.0;
            for (int k = 0; k < nb; ++k) acc += q[k] * h[b - k + nb - 1];
            qf[(int64_t)v * nb + b] = ds * acc;
        }
    }
    free(q);
    free(h);
}

/* FBP image f [n][n] (row = y, column = x) from projections p [nv][nb]. */
void orc_fbp(const orc_geom *g, const double *p, double *f)
{
    const int n = g->n, nb = g->nb;
    const double scale = g->sod / g->sdd, ds = g->pitch * scale;
    const double s0 = (-0.5 * (double)(nb - 1) * g->pitch + g->det_offset) * scale;
    const double dth = g->arc / (double)g->nv;
    double *qf = (double *)malloc(sizeof(double) * (size_t)g->nv * (size_t)nb);
    orc_fbp_filter(g, p, qf);
    for (int64_t i = 0; i < (int64_t)n * n; ++i) f[i] = 0.0;
    const double lo = -0.5 * (double)n * g->px;
    for (int v = 0; v < g->nv; ++v) {
        double th = g->start + (double)v * dth;
        double cth = cos(th), sth = sin(th);
        double Sx = g->sod * cth, Sy = g->sod * sth;
        double cx = -cth, cy = -sth;      /* central ray, source -> isocentre */
        double ex = -sth, ey = cth;       /* lateral, increasing bin index    */
        for (int i = 0; i < n; ++i) {
            double y = lo + ((double)i + 0.5) * g->px;
            for (int j = 0; j < n; ++j) {
                double x = lo + ((double)j + 0.5) * g->px;
                double dx = x - Sx, dy = y - Sy;
                double L = dx * cx + dy * cy;
                double s = (dx * ex + dy * ey) * g->sod / L;
                double t = (s - s0) / ds;     /* bin coordinate */
                double val = 0.0;
                if (t >= 0.0 && t <= (double)(nb - 1)) {
                    int b0 = (int)floor(t);
                    if (b0 > nb - 2) b0 = nb - 2;
                    double w = t - (double)b0;
                    val = (1.0 - w) * qf[(int64_t)v * nb + b0] + w * qf[(int64_t)v * nb + b0 + 1];
                }
                double wgt = g->sod / L;
                f[(int64_t)i * n + j] += 0.5 * dth * wgt * wgt * val;
            }
        }
    }
    free(qf);
}

/* ------------------------------------------------------------------------ */
/* Joint (channel-coupled) TV on the combined image f = (f_h, f_l), Eq. (4)  */
/* read with the TV norm taken over both channels at every pixel:           */
/*   Phi(f) = sum_p |(grad f_h, grad f_l)_p|_2 + mu/2 sum_c |A f_c - g_c|^2  */
/* The ADM of Eq. (6)-(10) then has one z, lambda in R^{4N} (both channels'  */
/* gradients), one G in R^{2N} and one step alpha for the stacked f.         */
/* ------------------------------------------------------------------------ */

/*
 * Prox of the per-pixel 4-norm, Eq. (8) with the joint reading: for
 * w_p = (wh0, wh1, wl0, wl1), z_p = max(|w_p| - t, 0) w_p / |w_p|.
 * wh, wl, zh, zl: [2][npix] (the two gradient components of each channel).
 */
void orc_shrink4(int64_t npix, const double *wh, const double *wl, double t, double *zh, double *zl)
{
    for (int64_t p = 0; p < npix; ++p) {
        double a = wh[p], b = wh[npix + p], c = wl[p], d = wl[npix + p];
        double nrm = sqrt(a * a + b * b + c * c + d * d);
        double s = nrm - t;
        if (s > 0.0 && nrm > 0.0) {
            zh[p] = s * a / nrm;
            zh[npix + p] = s * b / nrm;
            zl[p] = s * c / nrm;
            zl[npix + p] = s * d / nrm;
        } else {
            zh[p] = zh[npix + p] = zl[p] = zl[npix + p] = 0.0;
        }
    }
}

/* sum_p |(grad f_h, grad f_l)_p|_2 for f = [2][N]. */
double orc_tv_joint(int n, const double *f)
{
    const int64_t N = (int64_t)n * n;
    double *gh = (double *)malloc(sizeof(double) * (size_t)(2 * N));
    double *gl = (double *)malloc(sizeof(double) * (size_t)(2 * N));
    orc_grad(n, f, gh);
    orc_grad(n, f + N, gl);
    double s = 0.0;
    for (int64_t p = 0; p < N; ++p)
        s += sqrt(gh[p] * gh[p] + gh[N + p] * gh[N + p] + gl[p] * gl[p] + gl[N + p] * gl[N + p]);
    free(gh);
    free(gl);
    return s;
}

/* Joint objective; g = [2][m] (g_h then g_l), f = [2][N]. */
double orc_objective_joint(int n, int64_t m, const int64_t *rowptr, const int32_t *idx,
                           const double *len, const double *g, double mu, const double *f)
{
    const int64_t N = (int64_t)n * n;
    double *r = (double *)malloc(sizeof(double) * (size_t)m);
    double s = 0.0;
    for (int c = 0; c < 2; ++c) {
        orc_project(m, rowptr, idx, len, f + c * N, r);
        for (int64_t i = 0; i < m; ++i) { double e = r[i] - g[c * m + i]; s += e * e; }
    }
    free(r);
    return orc_tv_joint(n, f) + 0.5 * mu * s;
}

/*
 * One ADM iteration, Eq. (10), for the joint problem.  State sizes: f 2N
 * ([channel][N]), z and lam 4N ([channel][component][N]).  The steps are
 * those of orc_adm_iterate with the 4-vector shrink in the z-step, and the
 * step c(G) = |G|^2 / (mu |A G|^2 + rho |grad G|^2) taken over both
 * channels (the exact line search of the stacked quadratic).
 * G_out (2N) and norms (3) may be NULL.  Returns the step applied.
 */
double orc_adm_joint_iterate(int n, int64_t m, const int64_t *rowptr, const int32_t *idx,
                             const double *len, const double *g, const orc_adm_params *prm,
                             orc_adm_state *st, double *G_out, double *norms)
{
    const int64_t N = (int64_t)n * n;
    const double mu = prm->mu, rho = prm->rho, xi = prm->xi;
    double *gf = (double *)malloc(sizeof(double) * (size_t)(4 * N));
    double *w = (double *)malloc(sizeof(double) * (size_t)(4 * N));
    double *r = (double *)malloc(sizeof(double) * (size_t)m);
    double *t1 = (double *)malloc(sizeof(double) * (size_t)N);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)N);
    double *t3 = (double *)malloc(sizeof(double) * (size_t)N);
    double *G = (double *)malloc(sizeof(double) * (size_t)(2 * N));
    double *AG = (double *)malloc(sizeof(double) * (size_t)m);
    double *gG = (double *)malloc(sizeof(double) * (size_t)(2 * N));

    /* z-step, Eq. (8), on the 4-vectors of both channels */
    for (int c = 0; c < 2; ++c) orc_grad(n, st->f + c * N, gf + c * 2 * N);
    for (int64_t p = 0; p < 4 * N; ++p) w[p] = gf[p] - st->lam[p] / rho;
    orc_shrink4(N, w, w + 2 * N, 1.0 / rho, st->z, st->z + 2 * N);

    /* G_f, Eq. (9), per channel; norms summed over both channels */
    double gg = 0.0, aa = 0.0, dd = 0.0;
    for (int c = 0; c < 2; ++c) {
        const double *f = st->f + c * N, *z = st->z + c * 2 * N, *lam = st->lam + c * 2 * N;
        double *Gc = G + c * N;
        orc_project(m, rowptr, idx, len, f, r);
        for (int64_t i = 0; i < m; ++i) r[i] -= g[c * m + i];
        orc_backproject(m, N, rowptr, idx, len, r, t1);
        for (int64_t p = 0; p < 2 * N; ++p) w[p] = gf[c * 2 * N + p] - z[p];
        orc_grad_t(n, w, t2);
        orc_grad_t(n, lam, t3);
        for (int64_t p = 0; p < N; ++p) Gc[p] = mu * t1[p] + rho * t2[p] - t3[p];
        orc_project(m, rowptr, idx, len, Gc, AG);
        orc_grad(n, Gc, gG);
        gg += dot(N, Gc, Gc);
        aa += dot(m, AG, AG);
        dd += dot(2 * N, gG, gG);
    }

    /* one step for the stacked f (R6) */
    double den = mu * aa + rho * dd;
    double cst = (den > 0.0) ? gg / den : 0.0;
    double alpha;
    if (prm->step_rule == 1 || st->alpha_prev < 0.0) alpha = cst;
    else alpha = st->alpha_prev;
    st->alpha_prev = cst;

    /* f-step and multiplier step, per channel */
    for (int64_t p = 0; p < 2 * N; ++p) {
        st->f[p] -= alpha * G[p];
        if (prm->nonneg && st->f[p] < 0.0) st->f[p] = 0.0;
    }
    for (int c = 0; c < 2; ++c) orc_grad(n, st->f + c * N, gf + c * 2 * N);
    for (int64_t p = 0; p < 4 * N; ++p) st->lam[p] -= xi * (gf[p] - st->z[p]);

    if (G_out) memcpy(G_out, G, sizeof(double) * (size_t)(2 * N));
    if (norms) { norms[0] = gg; norms[1] = aa; norms[2] = dd; }
    free(gf); free(w); free(r); free(t1); free(t2); free(t3); free(G); free(AG); free(gG);
    return alpha;
}

/* The joint ADM loop from f ([2][N], in/out) with z = lam = 0; as orc_adm_run. */
int orc_adm_joint_run(int n, int64_t m, const int64_t *rowptr, const int32_t *idx, const double *len,
                      const double *g, const orc_adm_params *prm, double *f, double *phi, double *alpha)
{
    const int64_t N = (int64_t)n * n;
    orc_adm_state st;
    st.f = f;
    st.z = (double *)calloc((size_t)(4 * N), sizeof(double));
    st.lam = (double *)calloc((size_t)(4 * N), sizeof(double));
    st.alpha_prev = -1.0;
    double prev = orc_objective_joint(n, m, rowptr, idx, len, g, prm->mu, f);
    if (phi) phi[0] = prev;
    int k = 0;
    while (k < prm->max_iter) {
        double a = orc_adm_joint_iterate(n, m, rowptr, idx, len, g, prm, &st, NULL, NULL);
        if (alpha) alpha[k] = a;
        ++k;
        double cur = orc_objective_joint(n, m, rowptr, idx, len, g, prm->mu, f);
        if (phi) phi[k] = cur;
        if (prm->tol > 0.0 && prev > 0.0 && fabs(cur - prev) / prev < prm->tol) break;
        prev = cur;
    }
    free(st.z);
    free(st.lam);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: decomposition                                                    */
/* ------------------------------------------------------------------------ */

/*
 * d = D^{-1} x per pixel, Eq. (11)-(12).  eta[m*2 + e]: material m (0, 1),
 * energy e (0 = high, 1 = low).  D = [[eta_1H, eta_2H], [eta_1L, eta_2L]].
 */
void orc_direct_decompose(int64_t npix, const double *eta, const double *xh, const double *xl,
                          double *d1, double *d2)
{
    double a = eta[0], b = eta[2];   /* row H: eta_1H, eta_2H */
    double c = eta[1], e = eta[3];   /* row L: eta_1L, eta_2L */
    double det = a * e - b * c;
    for (int64_t p = 0; p < npix; ++p) {
        d1[p] = (e * xh[p] - b * xl[p]) / det;
        d2[p] = (-c * xh[p] + a * xl[p]) / det;
    }
}

/*
 * 3x3 Prewitt gradient magnitude with replicate padding (R14), FP64:
 *   gx = sum over t = -1, 0, 1 of (x[i+t][j+1] - x[i+t][j-1]),
 *   gy = sum over t = -1, 0, 1 of (x[i+1][j+t] - x[i-1][j+t]),
 *   |g| = sqrt(gx^2 + gy^2), indices clamped to the image.
 */
void orc_prewitt(int n, const double *x, double *mag)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double gx = 0.0, gy = 0.0;
            int jl = j - 1 < 0 ? 0 : j - 1, jr = j + 1 >= n ? n - 1 : j + 1;
            int iu = i - 1 < 0 ? 0 : i - 1, id = i + 1 >= n ? n - 1 : i + 1;
            for (int t = -1; t <= 1; ++t) {
                int ii = i + t < 0 ? 0 : (i + t >= n ? n - 1 : i + t);
                int jj = j + t < 0 ? 0 : (j + t >= n ? n - 1 : j + t);
                gx += x[(int64_t)ii * n + jr] - x[(int64_t)ii * n + jl];
                gy += x[(int64_t)id * n + jj] - x[(int64_t)iu * n + jj];
            }
            mag[(int64_t)i * n + j] = sqrt(gx * gx + gy * gy);
        }
}

/*
 * Edge mask (1 = edge) from both energy images (R14), decided in FP64: a
 * pixel is an edge when its Prewitt magnitude divided by the image's largest
 * magnitude exceeds tau in either image.
 */
void orc_edge_mask(int n, const double *xh, const double *xl, double tau, uint8_t *mask)
{
    int64_t N = (int64_t)n * n;
    double *mh = (double *)malloc(sizeof(double) * (size_t)N);
    double *ml = (double *)malloc(sizeof(double) * (size_t)N);
    orc_prewitt(n, xh, mh);
    orc_prewitt(n, xl, ml);
    double Mh = 0.0, Ml = 0.0;
    for (int64_t p = 0; p < N; ++p) {
        if (mh[p] > Mh) Mh = mh[p];
        if (ml[p] > Ml) Ml = ml[p];
    }
    for (int64_t p = 0; p < N; ++p) {
        int eh = Mh > 0.0 && mh[p] / Mh > tau;
        int el = Ml > 0.0 && ml[p] / Ml > tau;
        mask[p] = (uint8_t)(eh || el);
    }
    free(mh);
    free(ml);
}

/* Weight e_ik of Eq. (14) between 4-neighbours p and q. */
static double edge_w(const uint8_t *mask, int64_t p, int64_t q, double eps)
{
    return (mask[p] || mask[q]) ? eps : 1.0;
}

/* out = (I + gamma L_e) u, (L_e u)_i = sum_{k in N_i} e_ik (u_i - u_k) (R13). */
void orc_pls_apply(int n, const uint8_t *mask, double gamma, double eps, const double *u, double *out)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int64_t p = (int64_t)i * n + j;
            double s = 0.0;
            if (i > 0) s += edge_w(mask, p, p - n, eps) * (u[p] - u[p - n]);
            if (i + 1 < n) s += edge_w(mask, p, p + n, eps) * (u[p] - u[p + n]);
            if (j > 0) s += edge_w(mask, p, p - 1, eps) * (u[p] - u[p - 1]);
            if (j + 1 < n) s += edge_w(mask, p, p + 1, eps) * (u[p] - u[p + 1]);
            out[p] = u[p] + gamma * s;
        }
}

/* Jacobi diagonal 1 + gamma sum_k e_ik. */
void orc_pls_diag(int n, const uint8_t *mask, double gamma, double eps, double *diag)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int64_t p = (int64_t)i * n + j;
            double s = 0.0;
            if (i > 0) s += edge_w(mask, p, p - n, eps);
            if (i + 1 < n) s += edge_w(mask, p, p + n, eps);
            if (j > 0) s += edge_w(mask, p, p - 1, eps);
            if (j + 1 < n) s += edge_w(mask, p, p + 1, eps);
            diag[p] = 1.0 + gamma * s;
        }
}

/*
 * Jacobi-preconditioned CG for (I + gamma L_e) u = d (Eq. (15), R13, R16),
 * starting from u = d.  Runs max_iter iterations, or stops once
 * |r| / |d| < tol (tol > 0).  Returns the iterations done; *relres = |r|/|d|.
 */
int orc_pls_pcg(int n, const uint8_t *mask, double gamma, double eps, const double *d,
                double *u, int max_iter, double tol, double *relres)
{
    int64_t N = (int64_t)n * n;
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double *z = (double *)malloc(sizeof(double) * (size_t)N);
    double *p = (double *)malloc(sizeof(double) * (size_t)N);
    double *Ap = (double *)malloc(sizeof(double) * (size_t)N);
    double *M = (double *)malloc(sizeof(double) * (size_t)N);
    orc_pls_diag(n, mask, gamma, eps, M);
    memcpy(u, d, sizeof(double) * (size_t)N);
    orc_pls_apply(n, mask, gamma, eps, u, Ap);
    for (int64_t i = 0; i < N; ++i) r[i] = d[i] - Ap[i];
    double bn = sqrt(dot(N, d, d));
    for (int64_t i = 0; i < N; ++i) { z[i] = r[i] / M[i]; p[i] = z[i]; }
    double rz = dot(N, r, z);
    int it = 0;
    double rn = sqrt(dot(N, r, r));
    while (it < max_iter) {
        if (tol > 0.0 && (bn == 0.0 || rn / bn < tol)) break;
        orc_pls_apply(n, mask, gamma, eps, p, Ap);
        double pAp = dot(N, p, Ap);
        if (pAp <= 0.0) break;
        double a = rz / pAp;
        for (int64_t i = 0; i < N; ++i) { u[i] += a * p[i]; r[i] -= a * Ap[i]; }
        ++it;
        rn = sqrt(dot(N, r, r));
        for (int64_t i = 0; i < N; ++i) z[i] = r[i] / M[i];
        double rz_new = dot(N, r, z);
        double beta = (rz != 0.0) ? rz_new / rz : 0.0;
        rz = rz_new;
        for (int64_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (relres) *relres = (bn > 0.0) ? rn / bn : 0.0;
    free(r); free(z); free(p); free(Ap); free(M);
    return it;
}

/* ======================================================================== */
/* CNN warm start (not in the paper): the encoder-decoder that maps a short */
/* ADM reconstruction to a converged one.  FP64 definition by direct loops; */
/* layout NCHW, one image per batch element, weights [Cout][Cin][3][3].     */
/*                                                                          */
/*   a1 = relu(conv(x/s, W1)),  e1 = relu(conv(a1, W2))           H  x 32   */
/*   p1 = avgpool2(e1); a3 = relu(conv(p1,W3)); e2 = relu(conv(a3,W4)) 64   */
/*   p2 = avgpool2(e2); a5 = relu(conv(p2,W5)); bt = relu(conv(a5,W6)) 128  */
/*   c2 = [up2(bt), e2]; a7 = relu(conv(c2,W7)); d2 = relu(conv(a7,W8)) 64  */
/*   c1 = [up2(d2), e1]; a9 = relu(conv(c1,W9)); d1 = relu(conv(a9,W10)) 32 */
/*   out = x + s (Wh . d1 + bh)     (1x1 head, residual)                     */
/* every conv has a bias; s is the input scale.                              */
/* ======================================================================== */

#define CNN_LAYERS 10
static const int cnn_cin[CNN_LAYERS] = {1, 32, 32, 64, 64, 128, 192, 64, 96, 32};
static const int cnn_cout[CNN_LAYERS] = {32, 32, 64, 64, 128, 128, 64, 64, 32, 32};

/* Parameter vector: for each conv layer W[Cout][Cin][3][3] then b[Cout];
   then the head Wh[32], bh[1]. */
int64_t orc_cnn_num_params(void)
{
    int64_t n = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) n += (int64_t)cnn_cout[l] * cnn_cin[l] * 9 + cnn_cout[l];
    return n + 32 + 1;
}

static void cnn_offsets(int64_t *wo, int64_t *bo, int64_t *ho)
{
    int64_t o = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        wo[l] = o;
        o += (int64_t)cnn_cout[l] * cnn_cin[l] * 9;
        bo[l] = o;
        o += cnn_cout[l];
    }
    *ho = o;
}

/* y[co][h][w] = b[co] + sum_ci sum_kh sum_kw W[co][ci][kh][kw] x[ci][h+kh-1][w+kw-1] (zero padding) */
static void conv3(const double *x, int cin, int H, int W, const double *Wt, const double *b, int cout,
                  double *y)
{
    for (int co = 0; co < cout; ++co)
        for (int h = 0; h < H; ++h)
            for (int w = 0; w < W; ++w) {
                double s = b[co];
                for (int ci = 0; ci < cin; ++ci)
                    for (int kh = 0; kh < 3; ++kh)
                        for (int kw = 0; kw < 3; ++kw) {
                            int hh = h + kh - 1, ww = w + kw - 1;
                            if (hh < 0 || hh >= H || ww < 0 || ww >= W) continue;
                            s += Wt[((int64_t)(co * cin + ci) * 3 + kh) * 3 + kw] *
                                 x[((int64_t)ci * H + hh) * W + ww];
                        }
                y[((int64_t)co * H + h) * W + w] = s;
            }
}

/* gradients of conv3: given dy, accumulate dW, db and (if dx) write dx */
static void conv3_back(const double *x, int cin, int H, int W, const double *Wt, int cout,
                       const double *dy, double *dW, double *db, double *dx)
{
    if (dx)
        for (int64_t i = 0; i < (int64_t)cin * H * W; ++i) dx[i] = 0.0;
    for (int co = 0; co < cout; ++co)
        for (int h = 0; h < H; ++h)
            for (int w = 0; w < W; ++w) {
                double g = dy[((int64_t)co * H + h) * W + w];
                db[co] += g;
                for (int ci = 0; ci < cin; ++ci)
                    for (int kh = 0; kh < 3; ++kh)
                        for (int kw = 0; kw < 3; ++kw) {
                            int hh = h + kh - 1, ww = w + kw - 1;
                            if (hh < 0 || hh >= H || ww < 0 || ww >= W) continue;
                            int64_t wi = ((int64_t)(co * cin + ci) * 3 + kh) * 3 + kw;
                            int64_t xi = ((int64_t)ci * H + hh) * W + ww;
                            dW[wi] += g * x[xi];
                            if (dx) dx[xi] += g * Wt[wi];
                        }
            }
}

static void relu(double *a, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (a[i] < 0.0) a[i] = 0.0;
}

static void relu_mask(const double *y, double *d, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!(y[i] > 0.0)) d[i] = 0.0;
}

static void pool2(const double *x, int C, int H, int W, double *y)
{
    int H2 = H / 2, W2 = W / 2;
    for (int c = 0; c < C; ++c)
        for (int h = 0; h < H2; ++h)
            for (int w = 0; w < W2; ++w) {
                const double *p = x + ((int64_t)c * H + 2 * h) * W + 2 * w;
                y[((int64_t)c * H2 + h) * W2 + w] = 0.25 * (p[0] + p[1] + p[W] + p[W + 1]);
            }
}

static void pool2_back(const double *dy, int C, int H, int W, double *dx_acc)
{
    int H2 = H / 2, W2 = W / 2;
    for (int c = 0; c < C; ++c)
        for (int h = 0; h < H; ++h)
            for (int w = 0; w < W; ++w)
                dx_acc[((int64_t)c * H + h) * W + w] += 0.25 * dy[((int64_t)c * H2 + h / 2) * W2 + w / 2];
}

/* nearest up-sampling by 2 into channels [coff, coff + C) of y (Ctot channels) */
static void up2(const double *x, int C, int H, int W, double *y, int coff)
{
    for (int c = 0; c < C; ++c)
        for (int h = 0; h < 2 * H; ++h)
            for (int w = 0; w < 2 * W; ++w)
                y[((int64_t)(coff + c) * 2 * H + h) * 2 * W + w] = x[((int64_t)c * H + h / 2) * W + w / 2];
}

static void up2_back(const double *dy, int coff, int C, int H, int W, double *dx)
{
    for (int c = 0; c < C; ++c)
        for (int h = 0; h < H; ++h)
            for (int w = 0; w < W; ++w) {
                const double *p = dy + ((int64_t)(coff + c) * 2 * H + 2 * h) * 2 * W + 2 * w;
                dx[((int64_t)c * H + h) * W + w] = p[0] + p[1] + p[2 * W] + p[2 * W + 1];
            }
}

/*
 * Forward, and backward of the loss L = mean over pixels of (out - target)^2
 * when target != NULL (grad receives dL/dparams, *loss the value).  One image
 * x [H][W] (H, W multiples of 4) per call; out [H][W] may be NULL.
 */
void orc_cnn_run(const double *prm, double s, const double *x, int H, int W, double *out,
                 const double *target, double *grad, double *loss)
{
    int64_t wo[CNN_LAYERS], bo[CNN_LAYERS], ho;
    cnn_offsets(wo, bo, &ho);
    const int H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int64_t P = (int64_t)H * W, P2 = (int64_t)H2 * W2, P4 = (int64_t)H4 * W4;
    double *xin = malloc(sizeof(double) * P), *a1 = malloc(sizeof(double) * 32 * P),
           *e1 = malloc(sizeof(double) * 32 * P), *p1 = malloc(sizeof(double) * 32 * P2),
           *a3 = malloc(sizeof(double) * 64 * P2), *e2 = malloc(sizeof(double) * 64 * P2),
           *p2 = malloc(sizeof(double) * 64 * P4), *a5 = malloc(sizeof(double) * 128 * P4),
           *bt = malloc(sizeof(double) * 128 * P4), *c2 = malloc(sizeof(double) * 192 * P2),
           *a7 = malloc(sizeof(double) * 64 * P2), *d2 = malloc(sizeof(double) * 64 * P2),
           *c1 = malloc(sizeof(double) * 96 * P), *a9 = malloc(sizeof(double) * 32 * P),
           *d1 = malloc(sizeof(double) * 32 * P), *o = malloc(sizeof(double) * P);
    for (int64_t i = 0; i < P; ++i) xin[i] = x[i] / s;
    conv3(xin, 1, H, W, prm + wo[0], prm + bo[0], 32, a1); relu(a1, 32 * P);
    conv3(a1, 32, H, W, prm + wo[1], prm + bo[1], 32, e1); relu(e1, 32 * P);
    pool2(e1, 32, H, W, p1);
    conv3(p1, 32, H2, W2, prm + wo[2], prm + bo[2], 64, a3); relu(a3, 64 * P2);
    conv3(a3, 64, H2, W2, prm + wo[3], prm + bo[3], 64, e2); relu(e2, 64 * P2);
    pool2(e2, 64, H2, W2, p2);
    conv3(p2, 64, H4, W4, prm + wo[4], prm + bo[4], 128, a5); relu(a5, 128 * P4);
    conv3(a5, 128, H4, W4, prm + wo[5], prm + bo[5], 128, bt); relu(bt, 128 * P4);
    up2(bt, 128, H4, W4, c2, 0);
    memcpy(c2 + 128 * P2, e2, sizeof(double) * 64 * P2);
    conv3(c2, 192, H2, W2, prm + wo[6], prm + bo[6], 64, a7); relu(a7, 64 * P2);
    conv3(a7, 64, H2, W2, prm + wo[7], prm + bo[7], 64, d2); relu(d2, 64 * P2);
    up2(d2, 64, H2, W2, c1, 0);
    memcpy(c1 + 64 * P, e1, sizeof(double) * 32 * P);
    conv3(c1, 96, H, W, prm + wo[8], prm + bo[8], 32, a9); relu(a9, 32 * P);
    conv3(a9, 32, H, W, prm + wo[9], prm + bo[9], 32, d1); relu(d1, 32 * P);
    const double *Wh = prm + ho, bh = prm[ho + 32];
    for (int64_t i = 0; i < P; ++i) {
        double h = bh;
        for (int c = 0; c < 32; ++c) h += Wh[c] * d1[c * P + i];
        o[i] = x[i] + s * h;
    }
    if (out) memcpy(out, o, sizeof(double) * P);
    if (target) {
        int64_t np = orc_cnn_num_params();
        for (int64_t i = 0; i < np; ++i) grad[i] = 0.0;
        double L = 0.0;
        double *dh = malloc(sizeof(double) * P);
        for (int64_t i = 0; i < P; ++i) {
            double e = o[i] - target[i];
            L += e * e;
            dh[i] = s * 2.0 * e / (double)P;
        }
        *loss = L / (double)P;
        double *dd1 = malloc(sizeof(double) * 32 * P);
        for (int c = 0; c < 32; ++c)
            for (int64_t i = 0; i < P; ++i) {
                grad[ho + c] += dh[i] * d1[c * P + i];
                dd1[c * P + i] = dh[i] * Wh[c];
            }
        for (int64_t i = 0; i < P; ++i) grad[ho + 32] += dh[i];
        relu_mask(d1, dd1, 32 * P);
        double *da9 = malloc(sizeof(double) * 32 * P), *dc1 = malloc(sizeof(double) * 96 * P);
        conv3_back(a9, 32, H, W, prm + wo[9], 32, dd1, grad + wo[9], grad + bo[9], da9);
        relu_mask(a9, da9, 32 * P);
        conv3_back(c1, 96, H, W, prm + wo[8], 32, da9, grad + wo[8], grad + bo[8], dc1);
        double *dd2 = malloc(sizeof(double) * 64 * P2);
        up2_back(dc1, 0, 64, H2, W2, dd2);
        relu_mask(d2, dd2, 64 * P2);
        double *da7 = malloc(sizeof(double) * 64 * P2), *dc2 = malloc(sizeof(double) * 192 * P2);
        conv3_back(a7, 64, H2, W2, prm + wo[7], 64, dd2, grad + wo[7], grad + bo[7], da7);
        relu_mask(a7, da7, 64 * P2);
        conv3_back(c2, 192, H2, W2, prm + wo[6], 64, da7, grad + wo[6], grad + bo[6], dc2);
        double *dbt = malloc(sizeof(double) * 128 * P4);
        up2_back(dc2, 0, 128, H4, W4, dbt);
        relu_mask(bt, dbt, 128 * P4);
        double *da5 = malloc(sizeof(double) * 128 * P4), *dp2 = malloc(sizeof(double) * 64 * P4);
        conv3_back(a5, 128, H4, W4, prm + wo[5], 128, dbt, grad + wo[5], grad + bo[5], da5);
        relu_mask(a5, da5, 128 * P4);
        conv3_back(p2, 64, H4, W4, prm + wo[4], 128, da5, grad + wo[4], grad + bo[4], dp2);
        double *de2 = malloc(sizeof(double) * 64 * P2);
        memcpy(de2, dc2 + 128 * P2, sizeof(double) * 64 * P2);   /* skip path */
        pool2_back(dp2, 64, H2, W2, de2);
        relu_mask(e2, de2, 64 * P2);
        double *da3 = malloc(sizeof(double) * 64 * P2), *dp1 = malloc(sizeof(double) * 32 * P2);
        conv3_back(a3, 64, H2, W2, prm + wo[3], 64, de2, grad + wo[3], grad + bo[3], da3);
        relu_mask(a3, da3, 64 * P2);
        conv3_back(p1, 32, H2, W2, prm + wo[2], 64, da3, grad + wo[2], grad + bo[2], dp1);
        double *de1 = malloc(sizeof(double) * 32 * P);
        memcpy(de1, dc1 + 64 * P, sizeof(double) * 32 * P);      /* skip path */
        pool2_back(dp1, 32, H, W, de1);
        relu_mask(e1, de1, 32 * P);
        double *da1 = malloc(sizeof(double) * 32 * P);
        conv3_back(a1, 32, H, W, prm + wo[1], 32, de1, grad + wo[1], grad + bo[1], da1);
        relu_mask(a1, da1, 32 * P);
        conv3_back(xin, 1, H, W, prm + wo[0], 32, da1, grad + wo[0], grad + bo[0], NULL);
        free(dh); free(dd1); free(da9); free(dc1); free(dd2); free(da7); free(dc2); free(dbt);
        free(da5); free(dp2); free(de2); free(da3); free(dp1); free(de1); free(da1);
    }
    free(xin); free(a1); free(e1); free(p1); free(a3); free(e2); free(p2); free(a5); free(bt);
    free(c2); free(a7); free(d2); free(c1); free(a9); free(d1); free(o);
}

/* ======================================================================== */
/* Cone-beam geometry and 3-D decomposition (Sec. 2.1, Fig. 1: circular    */
/* source orbit, flat 2-D detector; Sec. 2.3, Eq. (14) with the 6          */
/* neighbours of a voxel; Sec. 3)                                           */
/* ======================================================================== */

/*
 * Geometry.  The source turns in the plane z = 0: view v at angle
 * th_v = start + v arc / nv, source S = SOD (cos th, sin th, 0); the flat
 * detector is centred at (SOD - SDD)(cos th, sin th, 0) with axes
 * e_u = (-sin th, cos th, 0) (columns) and e_z = (0, 0, 1) (rows); cell
 * (row r, column c) is centred at u_c = (c - (nc - 1) / 2) pu + off_u,
 * z_r = (r - (nr - 1) / 2) pv + off_v.  One ray per cell, from the source
 * point to the cell centre; ray index (v nr + r) nc + c.  The volume is
 * n x n x nz voxels of px x px x pz, centred on the origin; voxel index
 * (k n + i) n + j with k along z, i along y (row), j along x (column).
 */
typedef struct {
    int n, nz;
    double px, pz;
    int nv, nr, nc;
    double pu, pv;
    double sod, sdd, start, arc, off_u, off_v;
} orc_geom3;

void orc3_ray(const orc_geom3 *g, int v, int r, int c, double S[3], double D[3])
{
    double th = g->start + (double)v * (g->arc / (double)g->nv);
    double ct = cos(th), st = sin(th);
    S[0] = g->sod * ct;
    S[1] = g->sod * st;
    S[2] = 0.0;
    double cx = (g->sod - g->sdd) * ct, cy = (g->sod - g->sdd) * st;
    double u = ((double)c - 0.5 * (double)(g->nc - 1)) * g->pu + g->off_u;
    double z = ((double)r - 0.5 * (double)(g->nr - 1)) * g->pv + g->off_v;
    D[0] = cx - u * st;
    D[1] = cy + u * ct;
    D[2] = z;
}

/*
 * Siddon's method in 3-D (ref. [42]), the same rule as in 2-D (R10): the
 * crossing parameters of the x, y and z grid planes inside the volume box
 * are collected, sorted and de-duplicated; the piece between consecutive
 * parameters goes to the voxel holding its midpoint; consecutive pieces in
 * one voxel are summed.  Writes up to `cap` (voxel, length in mm) pairs;
 * returns the count.
 */
int orc3_siddon_ray(const orc_geom3 *g, int v, int r, int c, int32_t *idx, double *len, int cap)
{
    double S[3], D[3];
    orc3_ray(g, v, r, c, S, D);
    const int n = g->n, nz = g->nz;
    const double d[3] = {D[0] - S[0], D[1] - S[1], D[2] - S[2]};
    const double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double lo[3] = {-0.5 * (double)n * g->px, -0.5 * (double)n * g->px, -0.5 * (double)nz * g->pz};
    const double sz[3] = {g->px, g->px, g->pz};
    const int cnt_ax[3] = {n, n, nz};
    double amin = 0.0, amax = 1.0;
    for (int a = 0; a < 3; ++a) {
        const double hi = lo[a] + (double)cnt_ax[a] * sz[a];
        if (d[a] != 0.0) {
            double t0 = (lo[a] - S[a]) / d[a], t1 = (hi - S[a]) / d[a];
            amin = fmax(amin, fmin(t0, t1));
            amax = fmin(amax, fmax(t0, t1));
        } else if (!(S[a] >= lo[a] && S[a] < hi)) {
            return 0;
        }
    }
    if (!(amin < amax)) return 0;
    double *al = (double *)malloc(sizeof(double) * (size_t)(2 * n + nz + 8));
    int na = 0;
    al[na++] = amin;
    al[na++] = amax;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        for (int k = 0; k <= cnt_ax[a]; ++k) {
            double t = (lo[a] + (double)k * sz[a] - S[a]) / d[a];
            if (t > amin && t < amax) al[na++] = t;
        }
    }
    qsort(al, (size_t)na, sizeof(double), cmp_double);
    int cnt = 0, last = -1;
    for (int k = 0; k + 1 < na; ++k) {
        double a0 = al[k], a1 = al[k + 1];
        if (!(a1 > a0)) continue;
        double mid = 0.5 * (a0 + a1);
        int jj = (int)floor((S[0] + mid * d[0] - lo[0]) / sz[0]);
        int ii = (int)floor((S[1] + mid * d[1] - lo[1]) / sz[1]);
        int kk = (int)floor((S[2] + mid * d[2] - lo[2]) / sz[2]);
        if (jj < 0 || jj >= n || ii < 0 || ii >= n || kk < 0 || kk >= nz) continue;
        int vox = (kk * n + ii) * n + jj;
        double seg = (a1 - a0) * L;
        if (cnt > 0 && last == vox) {
            if (cnt - 1 < cap) len[cnt - 1] += seg;
            continue;
        }
        if (cnt < cap) {
            idx[cnt] = vox;
            len[cnt] = seg;
        }
        last = vox;
        ++cnt;
    }
    free(al);
    return cnt;
}

int64_t orc3_table_nnz(const orc_geom3 *g)
{
    int cap = 2 * g->n + g->nz + 8;
    int32_t *ti = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    double *tl = (double *)malloc(sizeof(double) * (size_t)cap);
    int64_t total = 0;
    for (int v = 0; v < g->nv; ++v)
        for (int r = 0; r < g->nr; ++r)
            for (int c = 0; c < g->nc; ++c) total += orc3_siddon_ray(g, v, r, c, ti, tl, cap);
    free(ti);
    free(tl);
    return total;
}

/* Ray-major table of the cone-beam A: rowptr[M + 1], idx[nnz], len[nnz]. */
void orc3_table_build(const orc_geom3 *g, int64_t *rowptr, int32_t *idx, double *len)
{
    int cap = 2 * g->n + g->nz + 8;
    int64_t pos = 0, row = 0;
    rowptr[0] = 0;
    for (int v = 0; v < g->nv; ++v)
        for (int r = 0; r < g->nr; ++r)
            for (int c = 0; c < g->nc; ++c) {
                pos += orc3_siddon_ray(g, v, r, c, idx + pos, len + pos, cap);
                rowptr[++row] = pos;
            }
}

/*
 * 3-D Prewitt magnitude (reading R14 in 3-D): along each axis the
 * difference of the two neighbours along it, summed over the 3 x 3
 * neighbourhood of the other two axes, indices clamped to the volume;
 * |g| = sqrt(gx^2 + gy^2 + gz^2), FP64.
 */
void orc3_prewitt(int n, int nz, const double *x, double *mag)
{
#define CL(a, m) ((a) < 0 ? 0 : ((a) >= (m) ? (m) - 1 : (a)))
#define X3(k, i, j) x[((int64_t)CL(k, nz) * n + CL(i, n)) * n + CL(j, n)]
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double gx = 0.0, gy = 0.0, gz = 0.0;
                for (int s = -1; s <= 1; ++s)
                    for (int t = -1; t <= 1; ++t) {
                        gx += X3(k + s, i + t, j + 1) - X3(k + s, i + t, j - 1);
                        gy += X3(k + s, i + 1, j + t) - X3(k + s, i - 1, j + t);
                        gz += X3(k + 1, i + s, j + t) - X3(k - 1, i + s, j + t);
                    }
                mag[((int64_t)k * n + i) * n + j] = sqrt(gx * gx + gy * gy + gz * gz);
            }
#undef X3
#undef CL
}

/* Edge mask of the two energy volumes (R14 in 3-D), decided in FP64. */
void orc3_edge_mask(int n, int nz, const double *xh, const double *xl, double tau, uint8_t *mask)
{
    int64_t N = (int64_t)n * n * nz;
    double *mh = (double *)malloc(sizeof(double) * (size_t)N);
    double *ml = (double *)malloc(sizeof(double) * (size_t)N);
    orc3_prewitt(n, nz, xh, mh);
    orc3_prewitt(n, nz, xl, ml);
    double Mh = 0.0, Ml = 0.0;
    for (int64_t p = 0; p < N; ++p) {
        if (mh[p] > Mh) Mh = mh[p];
        if (ml[p] > Ml) Ml = ml[p];
    }
    for (int64_t p = 0; p < N; ++p)
        mask[p] = (uint8_t)((Mh > 0.0 && mh[p] / Mh > tau) || (Ml > 0.0 && ml[p] / Ml > tau));
    free(mh);
    free(ml);
}

/* out = (I + gamma L_e) u over the 6 neighbours of each voxel inside the
   volume (R13 with N_i of Eq. (14) in 3-D); e_ik as in 2-D. */
void orc3_pls_apply(int n, int nz, const uint8_t *mask, double gamma, double eps, const double *u, double *out)
{
    const int64_t plane = (int64_t)n * n;
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                int64_t p = k * plane + (int64_t)i * n + j;
                double s = 0.0;
                if (k > 0) s += edge_w(mask, p, p - plane, eps) * (u[p] - u[p - plane]);
                if (k + 1 < nz) s += edge_w(mask, p, p + plane, eps) * (u[p] - u[p + plane]);
                if (i > 0) s += edge_w(mask, p, p - n, eps) * (u[p] - u[p - n]);
                if (i + 1 < n) s += edge_w(mask, p, p + n, eps) * (u[p] - u[p + n]);
                if (j > 0) s += edge_w(mask, p, p - 1, eps) * (u[p] - u[p - 1]);
                if (j + 1 < n) s += edge_w(mask, p, p + 1, eps) * (u[p] - u[p + 1]);
                out[p] = u[p] + gamma * s;
            }
}

/* Jacobi diagonal 1 + gamma sum_k e_ik over the 6 neighbours. */
void orc3_pls_diag(int n, int nz, const uint8_t *mask, double gamma, double eps, double *diag)
{
    const int64_t plane = (int64_t)n * n;
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                int64_t p = k * plane + (int64_t)i * n + j;
                double s = 0.0;
                if (k > 0) s += edge_w(mask, p, p - plane, eps);
                if (k + 1 < nz) s += edge_w(mask, p, p + plane, eps);
                if (i > 0) s += edge_w(mask, p, p - n, eps);
                if (i + 1 < n) s += edge_w(mask, p, p + n, eps);
                if (j > 0) s += edge_w(mask, p, p - 1, eps);
                if (j + 1 < n) s += edge_w(mask, p, p + 1, eps);
                diag[p] = 1.0 + gamma * s;
            }
}

/* Jacobi PCG for the 3-D system from u = d (as orc_pls_pcg). */
int orc3_pls_pcg(int n, int nz, const uint8_t *mask, double gamma, double eps, const double *d,
                 double *u, int max_iter, double tol, double *relres)
{
    int64_t N = (int64_t)n * n * nz;
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double *z = (double *)malloc(sizeof(double) * (size_t)N);
    double *p = (double *)malloc(sizeof(double) * (size_t)N);
    double *Ap = (double *)malloc(sizeof(double) * (size_t)N);
    double *M = (double *)malloc(sizeof(double) * (size_t)N);
    orc3_pls_diag(n, nz, mask, gamma, eps, M);
    memcpy(u, d, sizeof(double) * (size_t)N);
    orc3_pls_apply(n, nz, mask, gamma, eps, u, Ap);
    for (int64_t i = 0; i < N; ++i) r[i] = d[i] - Ap[i];
    double bn = sqrt(dot(N, d, d));
    for (int64_t i = 0; i < N; ++i) { z[i] = r[i] / M[i]; p[i] = z[i]; }
    double rz = dot(N, r, z);
    int it = 0;
    double rn = sqrt(dot(N, r, r));
    while (it < max_iter) {
        if (tol > 0.0 && (bn == 0.0 || rn / bn < tol)) break;
        orc3_pls_apply(n, nz, mask, gamma, eps, p, Ap);
        double pAp = dot(N, p, Ap);
        if (pAp <= 0.0) break;
        double a = rz / pAp;
        for (int64_t i = 0; i < N; ++i) { u[i] += a * p[i]; r[i] -= a * Ap[i]; }
        ++it;
        rn = sqrt(dot(N, r, r));
        for (int64_t i = 0; i < N; ++i) z[i] = r[i] / M[i];
        double rz_new = dot(N, r, z);
        double beta = (rz != 0.0) ? rz_new / rz : 0.0;
        rz = rz_new;
        for (int64_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (relres) *relres = (bn > 0.0) ? rn / bn : 0.0;
    free(r); free(z); free(p); free(Ap); free(M);
    return it;
}
