/*
 * oracle.c -- plain, slow, FP64 CPU restatement of the selective-segmentation multigrid
 * method of Roberts, Chen and Irion, "A multigrid algorithm with non-standard smoother for
 * two selective models in variational segmentation" (arXiv 1807.02137).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker for the CUDA library.
 * It shares no code, header, table or helper with it.  Only the tests, the package's smoke
 * check and the bench's CPU-baseline leg may load it.  No product code path calls it.
 *
 * Every routine follows one passage of the paper, named in its comment.  Where the paper is
 * silent or ambiguous the reading taken is stated in the comment (the project's design notes
 * list them all).  Conventions:
 *   - an image / grid function is an n x m row-major array of doubles, index [i*m + j],
 *     i = row (downwards), j = column (rightwards), 0-based;
 *   - the four neighbours follow the paper's coefficient names: A <-> (i+1, j) "south",
 *     B <-> (i-1, j) "north", C <-> (i, j+1) "east", D <-> (i, j-1) "west";
 *   - pixel units: the finest grid has spacing h = 1, level l has h = 2^l;
 *   - a marker is (x, y) = (column, row).
 *
 * Parity status of each function is recorded next to it ("pinned by" lists the independent
 * checks in tests/test_oracle_*.py).
 *
 * The "#pragma omp parallel for" lines mark loops whose iterations are independent (each writes
 * its own cells and reads nothing another iteration writes).  The checker is built without
 * OpenMP, where they do nothing; the same file built with -fopenmp is the all-core timing
 * baseline, and gives bitwise the same results (tested).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_CHUNK 32       /* partial-line segments of the parallel ordering are cut at
                             multiples of this many cells along their line */
#define OR_PI 3.14159265358979323846

typedef struct {
    int model;            /* 0 = Spencer-Chen (Sec. 2.2, eq. scfunc), 1 = Rada-Chen (eq. rcfunc) */
    double mu;            /* weight of the (weighted) length term */
    double lambda1, lambda2;   /* intensity-fitting weights */
    double theta;         /* Spencer-Chen distance penalty weight */
    double nu;            /* Rada-Chen area penalty weight */
    double eps;           /* smoothed Heaviside width */
    double beta;          /* |grad phi|_beta regulariser */
    double beta_edge;     /* edge detector g(s) = 1/(1 + beta_edge s) */
    double sigma_blur;    /* Gaussian pre-smoothing of the image before g */
    double sigma_d;       /* distance-function width (px) */
    double Sigma;         /* jump threshold: cell in D iff max(A..D) > Sigma min(A..D) */
    double inv_tau;       /* 1/tau of the implicit pseudo-time step (0 = steady equation) */
    int nu1, nu2;         /* pre/post smoothing outer iterations */
    int levels;           /* number of grids (finest = level 0) */
    int smoother;         /* 0 = Hybrid Smoother 2, parallel ordering (Algorithm 3 on the GPU);
                             1 = Hybrid Smoother 2, lexicographic ordering of Fig. 4;
                             2 = GSLINE-I, columns left to right (Algorithm 1);
                             3 = GSLINE-I, even then odd columns;
                             4 = Hybrid Smoother 1, lexicographic (Algorithm 2);
                             5 = Hybrid Smoother 1, parallel ordering */
    int coarse_maxit;     /* Picard iterations cap of the coarsest solve (AOS: its iterations) */
    double coarse_tol;    /* relative nonlinear-residual target of the coarsest solve */
    int coarse_solver;    /* 0 = Picard + banded Cholesky; 1 = AOS time marching */
    double aos_dt;        /* AOS artificial time step */
} or_params;

/* ------------------------------------------------------------------------------------- */
/* Setup: image-derived data (Sec. 2.2)                                                   */
/* ------------------------------------------------------------------------------------- */

/* Half-sample mirror of an index into [0, n). */
static int mirror(int t, int n)
{
    if (n == 1) return 0;
    while (t < 0 || t >= n) {
        if (t < 0) t = -t - 1;
        if (t >= n) t = 2 * n - t - 1;
    }
    return t;
}

/* G_1 * z: separable Gaussian of width sigma, taps truncated at ceil(3 sigma) and normalised,
 * mirror boundary.  The paper writes g(|grad z|^2) (eq. rcfunc) without saying how z is
 * differentiated; the blur before differencing is the reading fixed for this project.
 * Pinned by: constant image unchanged; symmetric impulse response summing to one. */
void or_gauss_blur(const double *z, int n, int m, double sigma, double *out)
{
    int R = (int)ceil(3.0 * sigma);
    double *wt = malloc(sizeof(double) * (2 * R + 1));
    double s = 0;
    for (int t = -R; t <= R; ++t) { wt[t + R] = exp(-(double)(t * t) / (2 * sigma * sigma)); s += wt[t + R]; }
    for (int t = 0; t <= 2 * R; ++t) wt[t] /= s;
    double *tmp = malloc(sizeof(double) * (size_t)n * m);
    #pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double a = 0;
            for (int t = -R; t <= R; ++t) a += wt[t + R] * z[(size_t)i * m + mirror(j + t, m)];
            tmp[(size_t)i * m + j] = a;
        }
    #pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double a = 0;
            for (int t = -R; t <= R; ++t) a += wt[t + R] * tmp[(size_t)mirror(i + t, n) * m + j];
            out[(size_t)i * m + j] = a;
        }
    free(tmp);
    free(wt);
}

/* Edge detector g(s) = 1/(1 + beta_edge s), s = |grad z|^2 (Sec. 2.2, Rada-Chen model),
 * grad by central differences in pixel units with mirror ghosts.
 * Pinned by: g = 1 on a constant image; closed form on a linear ramp. */
void or_edge_detector(const double *zb, int n, int m, double beta_edge, double *g)
{
    #pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double zx = (zb[(size_t)i * m + mirror(j + 1, m)] - zb[(size_t)i * m + mirror(j - 1, m)]) / 2.0;
            double zy = (zb[(size_t)mirror(i + 1, n) * m + j] - zb[(size_t)mirror(i - 1, n) * m + j]) / 2.0;
            g[(size_t)i * m + j] = 1.0 / (1.0 + beta_edge * (zx * zx + zy * zy));
        }
}

/* Distance function d(x, y) = prod_k (1 - exp(-(x_k-x)^2/(2 s^2)) exp(-(y_k-y)^2/(2 s^2)))
 * (Sec. 2.2, selective models).  Pinned by: zero at a marker on a pixel centre, one far
 * away, product structure for two markers. */
void or_distance(int n, int m, const double *mx, const double *my, int k, double sigma_d, double *d)
{
    #pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double p = 1.0;
            for (int q = 0; q < k; ++q)
                p *= 1.0 - exp(-(mx[q] - j) * (mx[q] - j) / (2 * sigma_d * sigma_d))
                         * exp(-(my[q] - i) * (my[q] - i) / (2 * sigma_d * sigma_d));
            d[(size_t)i * m + j] = p;
        }
}

/* Convex hull (monotone chain) of the markers, counter-clockwise in (x, y).  Returns the
 * number of hull vertices written to hull (x, y pairs; room for 2k + 2 points). */
static int cross_sign_cmp(const void *a, const void *b)
{
    const double *p = a, *q = b;
    if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
    if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
    return 0;
}
static double cross3(const double *o, const double *a, const double *b)
{
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0]);
}
static int convex_hull(const double *mx, const double *my, int k, double *hull)
{
    double *pt = malloc(sizeof(double) * 2 * k);
    for (int q = 0; q < k; ++q) { pt[2 * q] = mx[q]; pt[2 * q + 1] = my[q]; }
    qsort(pt, k, 2 * sizeof(double), cross_sign_cmp);
    int h = 0;
    for (int q = 0; q < k; ++q) {
        while (h >= 2 && cross3(&hull[2 * (h - 2)], &hull[2 * (h - 1)], &pt[2 * q]) <= 0) --h;
        hull[2 * h] = pt[2 * q]; hull[2 * h + 1] = pt[2 * q + 1]; ++h;
    }
    int lower = h + 1;
    for (int q = k - 2; q >= 0; --q) {
        while (h >= lower && cross3(&hull[2 * (h - 2)], &hull[2 * (h - 1)], &pt[2 * q]) <= 0) --h;
        hull[2 * h] = pt[2 * q]; hull[2 * h + 1] = pt[2 * q + 1]; ++h;
    }
    free(pt);
    return h > 1 ? h - 1 : h;
}

/* Initial level set (Sec. 5, choice of initial contour): the contour is the boundary of the
 * polygon formed by the markers.  Reading: the polygon is the convex hull (marker order is not
 * given), phi0 is the signed Euclidean distance to its boundary in px, positive inside.  With
 * fewer than three markers, or collinear ones, phi0 is a disc of radius r0 around their
 * centroid.  Writes the enclosed area (px^2) to *area.  Returns the number of hull vertices
 * (0 for the disc fallback).
 * Pinned by: distances to a square hull checked against hand values; sign = inside test. */
int or_initial_phi(int n, int m, const double *mx, const double *my, int k, double r0,
                   double *phi, double *area)
{
    double *hull = malloc(sizeof(double) * 2 * (2 * k + 2));
    int h = k >= 3 ? convex_hull(mx, my, k, hull) : 0;
    double A = 0;
    for (int q = 0; q < h; ++q) {
        int r = (q + 1) % h;
        A += hull[2 * q] * hull[2 * r + 1] - hull[2 * r] * hull[2 * q + 1];
    }
    A *= 0.5;
    if (h < 3 || A <= 0) {
        double cx = 0, cy = 0;
        for (int q = 0; q < k; ++q) { cx += mx[q]; cy += my[q]; }
        cx /= k; cy /= k;
        #pragma omp parallel for
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < m; ++j)
                phi[(size_t)i * m + j] = r0 - sqrt((j - cx) * (j - cx) + (i - cy) * (i - cy));
        *area = OR_PI * r0 * r0;
        free(hull);
        return 0;
    }
    #pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double px = j, py = i, dmin = INFINITY;
            int inside = 1;
            for (int q = 0; q < h; ++q) {
                int r = (q + 1) % h;
                double ax = hull[2 * q], ay = hull[2 * q + 1], bx = hull[2 * r], by = hull[2 * r + 1];
                double ex = bx - ax, ey = by - ay;
                if (ex * (py - ay) - ey * (px - ax) < 0) inside = 0;
                double t = ((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey);
                if (t < 0) t = 0;
                if (t > 1) t = 1;
                double dx = px - (ax + t * ex), dy = py - (ay + t * ey);
                double dd = sqrt(dx * dx + dy * dy);
                if (dd < dmin) dmin = dd;
            }
            phi[(size_t)i * m + j] = inside ? dmin : -dmin;
        }
    *area = A;
    free(hull);
    return h;
}

/* Smoothed Heaviside H_eps(phi) = 1/2 + atan(phi/eps)/pi (Sec. 2.1). */
static double heaviside(double phi, double eps) { return 0.5 + atan(phi / eps) / OR_PI; }

/* Its derivative delta_eps(phi) = eps / (pi (eps^2 + phi^2)) (Sec. 2.2, after eq. rcel). */
static double dirac(double phi, double eps) { return eps / (OR_PI * (eps * eps + phi * phi)); }

/* Region averages c1, c2 (eq. c1c2) with weights H_eps(phi) and 1 - H_eps(phi).
 * Pinned by: a sharp two-valued phi on a two-valued image returns the two values up to the
 * arctan tails; c1 = c2 = const on a constant image. */
void or_region_means(const double *phi, const double *z, int n, int m, double eps,
                     double *c1, double *c2)
{
    double sh = 0, shz = 0, s1 = 0, s1z = 0;
    for (size_t q = 0; q < (size_t)n * m; ++q) {
        double H = heaviside(phi[q], eps);
        sh += H; shz += H * z[q];
        s1 += 1 - H; s1z += (1 - H) * z[q];
    }
    *c1 = sh > 0 ? shz / sh : 0;
    *c2 = s1 > 0 ? s1z / s1 : 0;
}

/* ------------------------------------------------------------------------------------- */
/* Grid transfers (Sec. 3.1)                                                              */
/* ------------------------------------------------------------------------------------- */

/* One-dimensional full-weighting rule.  Coarse index I sits on fine index 2I+1 (0-based),
 * i.e. 1-based coarse i <-> fine 2i as in the paper's formula; the coarse grid has
 * floor(n/2) cells.  Interior weights (1/4, 1/2, 1/4) on (2I, 2I+1, 2I+2); when n is even the
 * last coarse cell has no fine cell 2I+2 and uses (1/2, 1/2) on (2I, 2I+1), the paper's
 * boundary rule.  Returns the number of taps and fills idx/wt. */
static int fw_taps(int I, int n, int *idx, double *wt)
{
    int q = 2 * I + 1;
    if (q + 1 < n) {
        idx[0] = q - 1; wt[0] = 0.25;
        idx[1] = q;     wt[1] = 0.5;
        idx[2] = q + 1; wt[2] = 0.25;
        return 3;
    }
    idx[0] = q - 1; wt[0] = 0.5;
    idx[1] = q;     wt[1] = 0.5;
    return 2;
}

/* Restriction I_h^{2h} (Sec. 3.1, full weighting): the 2-D operator is the tensor product of
 * the 1-D rule in each direction, which is the paper's 1/16 [1 2 1; 2 4 2; 1 2 1] stencil in
 * the interior.  Pinned by: reproduces linear functions at interior coarse cells, constants
 * everywhere; weights sum to one. */
void or_restrict(const double *f, int n, int m, double *c)
{
    int nc = n / 2, mc = m / 2;
    #pragma omp parallel for
    for (int I = 0; I < nc; ++I) {
        int ri[3], ci[3];
        double rw[3], cw[3];
        int nr = fw_taps(I, n, ri, rw);
        for (int J = 0; J < mc; ++J) {
            int nk = fw_taps(J, m, ci, cw);
            double s = 0;
            for (int a = 0; a < nr; ++a)
                for (int b = 0; b < nk; ++b) s += rw[a] * cw[b] * f[(size_t)ri[a] * m + ci[b]];
            c[(size_t)I * mc + J] = s;
        }
    }
}

/* One-dimensional bilinear rule (Sec. 3.1, interpolation): fine 2I+1 takes coarse I; fine
 * 2I+2 takes the mean of coarse I and I+1; fine 0, and fine n-1 when n is odd, have a single
 * coarse neighbour and take its value (constant extrapolation, consistent with the Neumann
 * condition). */
static int bl_taps(int p, int nc, int *idx, double *wt)
{
    if (p % 2 == 1) { idx[0] = (p - 1) / 2; wt[0] = 1.0; return 1; }
    if (p == 0) { idx[0] = 0; wt[0] = 1.0; return 1; }
    int I = p / 2 - 1;
    if (I + 1 < nc) { idx[0] = I; wt[0] = 0.5; idx[1] = I + 1; wt[1] = 0.5; return 2; }
    idx[0] = I; wt[0] = 1.0;
    return 1;
}

/* Interpolation I_{2h}^h applied to a coarse correction and added: f += P e (Algorithm 1,
 * "correct the fine grid approximation").  Pinned by: reproduces linear functions in the
 * interior, constants everywhere; P = 4 R^T away from the boundary. */
void or_interpolate_add(const double *e, int nc, int mc, double *f, int n, int m)
{
    #pragma omp parallel for
    for (int i = 0; i < n; ++i) {
        int ri[2], ci[2];
        double rw[2], cw[2];
        int nr = bl_taps(i, nc, ri, rw);
        for (int j = 0; j < m; ++j) {
            int nk = bl_taps(j, mc, ci, cw);
            double s = 0;
            for (int a = 0; a < nr; ++a)
                for (int b = 0; b < nk; ++b) s += rw[a] * cw[b] * e[(size_t)ri[a] * mc + ci[b]];
            f[(size_t)i * m + j] += s;
        }
    }
}

/* ------------------------------------------------------------------------------------- */
/* Discretisation (Sec. 2.2, eqs. rcabcd / abcdrc and the Spencer-Chen analogue)          */
/* ------------------------------------------------------------------------------------- */

/* |grad phi|_beta at a cell: central differences with mirror ghosts, grid spacing h,
 * beta under the root. */
static double grad_norm(const double *phi, int n, int m, double h, double beta, int i, int j)
{
    double px = (phi[(size_t)i * m + mirror(j + 1, m)] - phi[(size_t)i * m + mirror(j - 1, m)]) / (2 * h);
    double py = (phi[(size_t)mirror(i + 1, n) * m + j] - phi[(size_t)mirror(i - 1, n) * m + j]) / (2 * h);
    return sqrt(px * px + py * py + beta);
}

/* Frozen coefficients of one grid at a given phi ("global" variant, Sec. 3.2: evaluated once
 * at the start of an outer iteration).  For every cell:
 *   G = w / |grad phi|_beta                                   (eq. abcdrc, with w = g for
 *                                                              Spencer-Chen, d g for Rada-Chen)
 *   A = mu delta(phi) G_{i+1/2,j} / h^2,  B = ... G_{i-1/2,j},
 *   C = mu delta(phi) G_{i,j+1/2} / h^2,  D = ... G_{i,j-1/2}
 * with the face value the arithmetic mean of the two cell values, and a face on the domain
 * boundary carrying no flux (coefficient 0), which is the Neumann condition.
 *   S = A + B + C + D + delta / tau          (the paper's S plus the pseudo-time term)
 *   f = delta (Fn + area + rhs)               (the paper's f, eq. gslexrc, plus the FAS and
 *                                              pseudo-time right-hand sides)
 * delta is the cell's delta_eps(phi).  Fn is the fitting field minus phi^n/tau; area is the
 * Rada-Chen global term 2 nu (|Omega_1| - A1) as area fractions (zero for Spencer-Chen). */
typedef struct {
    int n, m;
    double *A, *B, *C, *D, *S, *f, *delta;
    const double *omega;   /* per-cell relaxation weights of the point updates (NULL = 1) */
} or_coeffs;

static void coeffs_alloc(or_coeffs *k, int n, int m)
{
    size_t N = (size_t)n * m;
    k->n = n; k->m = m;
    k->A = calloc(N, sizeof(double)); k->B = calloc(N, sizeof(double));
    k->C = calloc(N, sizeof(double)); k->D = calloc(N, sizeof(double));
    k->S = calloc(N, sizeof(double)); k->f = calloc(N, sizeof(double));
    k->delta = calloc(N, sizeof(double));
    k->omega = NULL;
}
static void coeffs_free(or_coeffs *k)
{
    free(k->A); free(k->B); free(k->C); free(k->D); free(k->S); free(k->f); free(k->delta);
}

/* Rada-Chen area term 2 nu (h^2 sum_kl H(phi_kl) / |Omega| - A1 / |Omega|) (eq. rcabcd, the
 * sign as in eq. gslexrc, both areas as fractions of the fine image area n0 m0). */
static double area_term(const double *phi, int n, int m, double h, const or_params *p,
                        double n0m0, double A1)
{
    if (p->model != 1) return 0.0;
    double s = 0;
    for (size_t q = 0; q < (size_t)n * m; ++q) s += heaviside(phi[q], p->eps);
    return 2.0 * p->nu * (h * h * s / n0m0 - A1 / n0m0);
}

static void frozen_coeffs(const double *phi, const double *w, const double *Fn, const double *rhs,
                          int n, int m, double h, const or_params *p, double n0m0, double A1,
                          or_coeffs *k)
{
    size_t N = (size_t)n * m;
    double *G = malloc(sizeof(double) * N);
    #pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j)
            G[(size_t)i * m + j] = w[(size_t)i * m + j] / grad_norm(phi, n, m, h, p->beta, i, j);
    double area = area_term(phi, n, m, h, p, n0m0, A1);
    #pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            size_t q = (size_t)i * m + j;
            double dl = dirac(phi[q], p->eps);
            double c = p->mu * dl / (h * h);
            k->A[q] = i + 1 < n ? c * (G[q] + G[q + m]) / 2 : 0.0;
            k->B[q] = i > 0 ? c * (G[q] + G[q - m]) / 2 : 0.0;
            k->C[q] = j + 1 < m ? c * (G[q] + G[q + 1]) / 2 : 0.0;
            k->D[q] = j > 0 ? c * (G[q] + G[q - 1]) / 2 : 0.0;
            k->S[q] = k->A[q] + k->B[q] + k->C[q] + k->D[q] + dl * p->inv_tau;
            k->f[q] = dl * (Fn[q] + area + (rhs ? rhs[q] : 0.0));
            k->delta[q] = dl;
        }
    free(G);
}

/* The nonlinear operator of one pseudo-time step, divided by delta (Sec. 3.1, N^h phi = f^h,
 * eq. syseqns; see the header for the reading):
 *   L(phi)_ij = [A phi_{i+1,j} + B phi_{i-1,j} + C phi_{i,j+1} + D phi_{i,j-1} - S0 phi_ij] / delta_ij
 *               - Fn_ij - area(phi) - phi_ij / tau
 * with A..D evaluated at phi itself and S0 = A + B + C + D.  Multiplying by delta gives the
 * paper's N (eq. rcabcd) plus the implicit time term delta (phi - phi^n) / tau.
 * Pinned by: flux conservation (sum over cells of the diffusion part is zero), symmetry of
 * the frozen matrix, discrete curvature of a cone converging to -1/r. */
void or_apply_L(const double *phi, const double *w, const double *Fn, int n, int m, double h,
                const or_params *p, double n0m0, double A1, double *out)
{
    or_coeffs k;
    coeffs_alloc(&k, n, m);
    frozen_coeffs(phi, w, Fn, NULL, n, m, h, p, n0m0, A1, &k);
    double area = area_term(phi, n, m, h, p, n0m0, A1);
    #pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            size_t q = (size_t)i * m + j;
            double s = -(k.A[q] + k.B[q] + k.C[q] + k.D[q]) * phi[q];
            if (i + 1 < n) s += k.A[q] * phi[q + m];
            if (i > 0) s += k.B[q] * phi[q - m];
            if (j + 1 < m) s += k.C[q] * phi[q + 1];
            if (j > 0) s += k.D[q] * phi[q - 1];
            out[q] = s / k.delta[q] - Fn[q] - area - p->inv_tau * phi[q];
        }
    coeffs_free(&k);
}

/* Fitting field (eq. scel / rcel, the bracket): lambda1 (z - c1)^2 - lambda2 (z - c2)^2, plus
 * theta d for Spencer-Chen, minus phi^n / tau for the pseudo-time step. */
void or_fitting(const double *z, const double *d, const double *phin, int n, int m,
                double c1, double c2, const or_params *p, double *Fn)
{
    #pragma omp parallel for
    for (size_t q = 0; q < (size_t)n * m; ++q) {
        double F = p->lambda1 * (z[q] - c1) * (z[q] - c1) - p->lambda2 * (z[q] - c2) * (z[q] - c2);
        if (p->model == 0) F += p->theta * d[q];
        Fn[q] = F - p->inv_tau * phin[q];
    }
}

/* ------------------------------------------------------------------------------------- */
/* Smoothers (Sec. 3.2 and Sec. 4)                                                        */
/* ------------------------------------------------------------------------------------- */

/* GSLEX-I point update (eq. gslexrc) at one cell with frozen coefficients. */
static double point_update(const or_coeffs *k, const double *phi, int i, int j)
{
    int n = k->n, m = k->m;
    size_t q = (size_t)i * m + j;
    double s = -k->f[q];
    if (i + 1 < n) s += k->A[q] * phi[q + m];
    if (i > 0) s += k->B[q] * phi[q - m];
    if (j + 1 < m) s += k->C[q] * phi[q + 1];
    if (j > 0) s += k->D[q] * phi[q - 1];
    return s / k->S[q];
}

/* Jump classification (Sec. 4.1, definition of the set D; "lag only the smallest coefficient",
 * Sec. 4.1.3).  Returns -1 for a cell outside D, else the index 0..3 of its smallest
 * coefficient (A, B, C, D; ties to the earlier letter).  Only faces inside the domain take
 * part.  Pinned by: hand-made coefficient sets. */
int or_classify(double A, double B, double C, double D, int hasA, int hasB, int hasC, int hasD,
                double Sigma)
{
    double v[4] = {A, B, C, D};
    int has[4] = {hasA, hasB, hasC, hasD};
    double mx = -1, mn = INFINITY;
    int am = -1, cnt = 0;
    for (int t = 0; t < 4; ++t) {
        if (!has[t]) continue;
        ++cnt;
        if (v[t] > mx) mx = v[t];
        if (v[t] < mn) { mn = v[t]; am = t; }
    }
    if (cnt < 2) return -1;
    return mx > Sigma * mn ? am : -1;
}

static int cell_class(const or_coeffs *k, int i, int j, double Sigma)
{
    size_t q = (size_t)i * k->m + j;
    return or_classify(k->A[q], k->B[q], k->C[q], k->D[q], i + 1 < k->n, i > 0, j + 1 < k->m,
                       j > 0, Sigma);
}

/* Membership of the cells of one line piece [lo, hi) in the starred groups of one sweep
 * (Sec. 4.3): starred cells, plus, for each starred cell with no starred neighbour on the line
 * (a "single starred pixel"), its next neighbour on the line (its previous one when it is the
 * last cell of the piece).  Overlapping groups simply merge.  star[] and member[] are indexed
 * by position along the line. */
static void line_members(const int *star, int lo, int hi, int *member)
{
    for (int t = lo; t < hi; ++t) member[t] = star[t];
    for (int t = lo; t < hi; ++t) {
        if (!star[t]) continue;
        int left = t - 1 >= lo && star[t - 1];
        int right = t + 1 < hi && star[t + 1];
        if (left || right) continue;
        if (t + 1 < hi) member[t + 1] = 1;
        else if (t - 1 >= lo) member[t - 1] = 1;
    }
}

/* Partial-line update of the run [a, b] of one line (Sec. 4.3, step III; the tridiagonal
 * system of eq. system restricted to the run).  For a row run (sweeps A, B) the unknowns are
 * phi(i, a..b) coupled through C and D; A and B terms and the two end neighbours are taken
 * from src.  For a column run (sweeps C, D) the unknowns are phi(a..b, j) coupled through A
 * and B.  The result is written to dst.  Thomas algorithm (the system is diagonally dominant,
 * Sec. 3.2). */
static void solve_run(const or_coeffs *k, const double *src, double *dst, int rowwise,
                      int line, int a, int b)
{
    int n = k->n, m = k->m, L = b - a + 1;
    double *lo = malloc(sizeof(double) * L), *di = malloc(sizeof(double) * L);
    double *up = malloc(sizeof(double) * L), *r = malloc(sizeof(double) * L);
    for (int t = 0; t < L; ++t) {
        int i = rowwise ? line : a + t, j = rowwise ? a + t : line;
        size_t q = (size_t)i * m + j;
        double rhs = k->f[q];
        if (rowwise) {
            if (i + 1 < n) rhs -= k->A[q] * src[q + m];
            if (i > 0) rhs -= k->B[q] * src[q - m];
            lo[t] = k->D[q]; up[t] = k->C[q];
            if (t == 0 && j > 0) rhs -= k->D[q] * src[q - 1];
            if (t == L - 1 && j + 1 < m) rhs -= k->C[q] * src[q + 1];
        } else {
            if (j + 1 < m) rhs -= k->C[q] * src[q + 1];
            if (j > 0) rhs -= k->D[q] * src[q - 1];
            lo[t] = k->B[q]; up[t] = k->A[q];
            if (t == 0 && i > 0) rhs -= k->B[q] * src[q - m];
            if (t == L - 1 && i + 1 < n) rhs -= k->A[q] * src[q + m];
        }
        di[t] = -k->S[q];
        r[t] = rhs;
    }
    /* forward elimination */
    for (int t = 1; t < L; ++t) {
        double w = lo[t] / di[t - 1];
        di[t] -= w * up[t - 1];
        r[t] -= w * r[t - 1];
    }
    /* back substitution */
    double x = r[L - 1] / di[L - 1];
    for (int t = L - 1; t >= 0; --t) {
        if (t < L - 1) x = (r[t] - up[t] * x) / di[t];
        int i = rowwise ? line : a + t, j = rowwise ? a + t : line;
        dst[(size_t)i * m + j] = x;
    }
    free(lo); free(di); free(up); free(r);
}


/* Star flags of one sweep k (0..3 = A..D) for every cell: the cell is in D and its smallest
 * coefficient is k (Sec. 4.3, step I). */
static void star_flags(const or_coeffs *k, double Sigma, int sweep, int *star)
{
    #pragma omp parallel for
    for (int i = 0; i < k->n; ++i)
        for (int j = 0; j < k->m; ++j)
            star[(size_t)i * k->m + j] = cell_class(k, i, j, Sigma) == sweep;
}

/* Members of the starred groups of sweep k, with lines cut into pieces of length `piece`
 * (OR_CHUNK for the parallel ordering, the whole line for the lexicographic one). */
static void sweep_members(const or_coeffs *k, const int *star, int sweep, int piece, int *member)
{
    int n = k->n, m = k->m, rowwise = sweep < 2;
    int nl = rowwise ? n : m, len = rowwise ? m : n;
    #pragma omp parallel for
    for (int l = 0; l < nl; ++l) {
        int *sl = malloc(sizeof(int) * len), *ml = malloc(sizeof(int) * len);
        for (int t = 0; t < len; ++t) sl[t] = star[rowwise ? (size_t)l * m + t : (size_t)t * m + l];
        for (int lo = 0; lo < len; lo += piece) {
            int hi = lo + piece < len ? lo + piece : len;
            line_members(sl, lo, hi, ml);
        }
        for (int t = 0; t < len; ++t) member[rowwise ? (size_t)l * m + t : (size_t)t * m + l] = ml[t];
        free(sl); free(ml);
    }
}

/* Hybrid Smoother 2 in the parallel ordering (the ordering the GPU runs, restated plainly).
 * One outer iteration with coefficients frozen at its start (Sec. 4.3, "Implementing Hybrid
 * Smoother 2": four sweeps lagging A, B, C, D in turn).  In sweep k the starred cells are the
 * cells of D whose smallest coefficient is k; their groups lie along rows for k = A, B and
 * along columns for k = C, D, and are cut at multiples of OR_CHUNK along the line.  A sweep:
 *   1. point updates (eq. gslexrc) of the non-member cells of one colour of the checkerboard,
 *      then of the other colour (red = (i+j) even first for A and C, black first for B and D);
 *   2. partial-line updates of all groups on lines of one parity, then of the other parity
 *      (even first for A and C, odd first for B and D).  Within one such phase every group
 *      is solved from the values at the start of the phase.
 * Pinned by: equality with the block Gauss-Seidel error-propagation matrix assembled from the
 * operator; convergence of repeated outer iterations to the direct solution. */
static void hs2_parallel(const or_coeffs *k, double Sigma, double *phi)
{
    int n = k->n, m = k->m;
    size_t N = (size_t)n * m;
    int *star = malloc(sizeof(int) * N), *member = malloc(sizeof(int) * N);
    double *pre = malloc(sizeof(double) * N);
    for (int sweep = 0; sweep < 4; ++sweep) {
        int rowwise = sweep < 2, rev = sweep % 2 == 1;
        star_flags(k, Sigma, sweep, star);
        sweep_members(k, star, sweep, OR_CHUNK, member);
        for (int c = 0; c < 2; ++c) {
            int colour = rev ? 1 - c : c;
            #pragma omp parallel for
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < m; ++j)
                    if ((i + j) % 2 == colour && !member[(size_t)i * m + j]) {
                        size_t q = (size_t)i * m + j;
                        double g = point_update(k, phi, i, j);
                        /* per-cell relaxation weight of the learned-weights extension: phi += omega (g - phi) */
                        phi[q] = k->omega ? phi[q] + k->omega[q] * (g - phi[q]) : g;
                    }
        }
        int nl = rowwise ? n : m, len = rowwise ? m : n;
        for (int c = 0; c < 2; ++c) {
            int parity = rev ? 1 - c : c;
            memcpy(pre, phi, sizeof(double) * N);
            #pragma omp parallel for
            for (int l = parity; l < nl; l += 2)
                for (int lo = 0; lo < len; lo += OR_CHUNK) {
                    int hi = lo + OR_CHUNK < len ? lo + OR_CHUNK : len;
                    int t = lo;
                    while (t < hi) {
                        size_t q = rowwise ? (size_t)l * m + t : (size_t)t * m + l;
                        if (!member[q]) { ++t; continue; }
                        int a = t;
                        while (t < hi && member[rowwise ? (size_t)l * m + t : (size_t)t * m + l]) ++t;
                        solve_run(k, pre, phi, rowwise, l, a, t - 1);
                    }
                }
        }
    }
    free(star); free(member); free(pre);
}

/* Hybrid Smoother 2 in the paper's lexicographic ordering (Sec. 4.3, steps I-VI and the four
 * update orders of Fig. 4).  Sweep A: rows top to bottom, left to right; sweep B: bottom-right
 * to top-left along rows; sweep C: columns left to right, each top to bottom; sweep D:
 * columns right to left, each bottom to top.  Groups run along whole lines.  A cell outside
 * the groups gets a GSLEX-I update when the sweep reaches it; a group is solved as a whole
 * when the sweep reaches its first cell, from the current values around it. */
static void hs2_lexicographic(const or_coeffs *k, double Sigma, double *phi)
{
    int n = k->n, m = k->m;
    size_t N = (size_t)n * m;
    int *star = malloc(sizeof(int) * N), *member = malloc(sizeof(int) * N);
    int *done = malloc(sizeof(int) * N);
    for (int sweep = 0; sweep < 4; ++sweep) {
        int rowwise = sweep < 2, rev = sweep % 2 == 1;
        int len = rowwise ? m : n, nl = rowwise ? n : m;
        star_flags(k, Sigma, sweep, star);
        sweep_members(k, star, sweep, len, member);
        memset(done, 0, sizeof(int) * N);
        for (int lc = 0; lc < nl; ++lc) {
            int l = rev ? nl - 1 - lc : lc;
            for (int tc = 0; tc < len; ++tc) {
                int t = rev ? len - 1 - tc : tc;
                int i = rowwise ? l : t, j = rowwise ? t : l;
                size_t q = (size_t)i * m + j;
                if (!member[q]) { phi[q] = point_update(k, phi, i, j); continue; }
                if (done[q]) continue;
                int a = t, b = t;
#define MEM(tt) member[rowwise ? (size_t)l * m + (tt) : (size_t)(tt) * m + l]
                while (a - 1 >= 0 && MEM(a - 1)) --a;
                while (b + 1 < len && MEM(b + 1)) ++b;
#undef MEM
                solve_run(k, phi, phi, rowwise, l, a, b);
                for (int s = a; s <= b; ++s) done[rowwise ? (size_t)l * m + s : (size_t)s * m + l] = 1;
            }
        }
    }
    free(star); free(member); free(done);
}

/* GSLINE-I (Sec. 3.2, Smoothers 3-4; Algorithm 1): one outer iteration solves the tridiagonal
 * system of eq. system for every column, left to right, with C and D terms from the current
 * values and coefficients frozen at the start of the iteration. */
static void gsline_columns(const or_coeffs *k, double *phi)
{
    for (int j = 0; j < k->m; ++j) solve_run(k, phi, phi, 0, j, 0, k->n - 1);
}

/* GSLINE-I in the zebra ordering (Algorithm 1's smoother restated for parallel hardware): all
 * even columns, each solved exactly as in gsline_columns, then all odd columns.  Columns of one
 * parity are not neighbours, so solving them one after another equals solving them together
 * from the values at the start of the phase.  Pinned by: the block definition. */
static void gsline_zebra(const or_coeffs *k, double *phi)
{
    for (int par = 0; par < 2; ++par)
        for (int j = par; j < k->m; j += 2) solve_run(k, phi, phi, 0, j, 0, k->n - 1);
}

/* Hybrid Smoother 1 block (Sec. 4.2, the schemes with A, B, C or D lagged, eqs. caseAlagged to
 * caseDlagged) at a cell P of the set D whose smallest coefficient is `lag` (0..3 = A..D): P and
 * its neighbours other than the lagged one are updated together by solving their own equations
 * exactly, every other value (the lagged neighbour included) at its current value.  The
 * neighbours are not neighbours of each other, so the system is an arrow matrix; the leaves are
 * eliminated into P's row.  (The paper prints the couplings of the leaf rows with P's
 * coefficients; the rows here keep their own coefficients, A of the north neighbour for its
 * coupling to P and so on, which after division of each row by its delta are the same numbers.)
 * A neighbour outside the grid is not part of the block.  Pinned by: the block definition. */
static void hs1_block(const or_coeffs *k, double *phi, int i, int j, int lag)
{
    int n = k->n, m = k->m;
    size_t q = (size_t)i * m + j;
    /* neighbour offsets and existence in A, B, C, D order */
    int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
    const double *cP[4] = {k->A, k->B, k->C, k->D};
    /* the coefficient of a leaf's row for its neighbour in the opposite direction (P) */
    int opp[4] = {1, 0, 3, 2};
    double rP = k->f[q], num = 0.0, den = -k->S[q];
    double rl[4], cl[4], Sl[4];
    int has[4];
    for (int t = 0; t < 4; ++t) {
        int ii = i + di[t], jj = j + dj[t];
        has[t] = ii >= 0 && ii < n && jj >= 0 && jj < m;
        if (!has[t]) continue;
        size_t ql = (size_t)ii * m + jj;
        if (t == lag) { rP -= cP[t][q] * phi[ql]; has[t] = 0; continue; }
        /* leaf row: c_lP x_P - S_l x_l = f_l - sum over its other neighbours */
        double r = k->f[ql];
        for (int u = 0; u < 4; ++u) {
            if (u == opp[t]) continue;
            int i2 = ii + di[u], j2 = jj + dj[u];
            if (i2 < 0 || i2 >= n || j2 < 0 || j2 >= m) continue;
            r -= cP[u][ql] * phi[(size_t)i2 * m + j2];
        }
        rl[t] = r;
        cl[t] = cP[opp[t]][ql];
        Sl[t] = k->S[ql];
        /* x_l = (c_lP x_P - r_l) / S_l substituted into P's row */
        num += cP[t][q] * r / Sl[t];
        den += cP[t][q] * cl[t] / Sl[t];
    }
    double xP = (rP + num) / den;
    phi[q] = xP;
    for (int t = 0; t < 4; ++t) {
        if (!has[t]) continue;
        size_t ql = (size_t)(i + di[t]) * m + (j + dj[t]);
        phi[ql] = (cl[t] * xP - rl[t]) / Sl[t];
    }
}

/* Hybrid Smoother 1 as Algorithm 2 runs it (Sec. 4.2, steps I-II): GSLINE-I on all columns, then
 * the block of every cell of D in lexicographic order (rows top to bottom, left to right). */
static void hs1_lexicographic(const or_coeffs *k, double Sigma, double *phi)
{
    gsline_columns(k, phi);
    for (int i = 0; i < k->n; ++i)
        for (int j = 0; j < k->m; ++j) {
            int c = cell_class(k, i, j, Sigma);
            if (c >= 0) hs1_block(k, phi, i, j, c);
        }
}

/* Hybrid Smoother 1 in the parallel ordering used on the GPU: GSLINE-I zebra, then the blocks of
 * D in 16 classes (i mod 4, j mod 4), class by class.  Two blocks of one class have centres at
 * least 4 cells apart (Manhattan), so neither reads a cell the other writes: solving a class's
 * blocks one after another equals solving them together.  Pinned by: the block definition. */
static void hs1_parallel(const or_coeffs *k, double Sigma, double *phi)
{
    gsline_zebra(k, phi);
    for (int c = 0; c < 16; ++c)
        for (int i = c / 4; i < k->n; i += 4)
            for (int j = c % 4; j < k->m; j += 4) {
                int cls = cell_class(k, i, j, Sigma);
                if (cls >= 0) hs1_block(k, phi, i, j, cls);
            }
}

/* ------------------------------------------------------------------------------------- */
/* Coarsest-grid solve (Algorithm 1, "compute the exact solution")                        */
/* ------------------------------------------------------------------------------------- */

/* Solves L(phi) = rhs on one small grid.  Picard iteration on the frozen coefficients: each
 * step solves the linear system obtained by freezing A..D, delta and the area term at the
 * current phi, which after division of every row by its delta is
 *     (A+B+C+D)/delta phi_ij - A/delta phi_S - B/delta phi_N - C/delta phi_E - D/delta phi_W
 *        + phi_ij / tau = -(Fn + area + rhs)
 * a symmetric positive definite matrix (face coefficients are shared by the two cells).  It is
 * factorised by banded Cholesky, cells ordered along the shorter side.  Stops when the
 * nonlinear residual falls below coarse_tol times its initial value, when a step changes no
 * value by more than 1e-14 of the largest, or after coarse_maxit steps.  Returns the number of Picard steps, or -1 if a pivot is not positive.
 * Pinned by: dense LU of the same frozen system; the Picard fixed point satisfies L = rhs. */
int or_coarse_solve(double *phi, const double *w, const double *Fn, const double *rhs, int n, int m,
                    double h, const or_params *p, double n0m0, double A1)
{
    size_t N = (size_t)n * m;
    int colmajor = m > n;                /* order along the shorter side */
    int bw = colmajor ? n : m;
    double *band = malloc(sizeof(double) * N * (bw + 1));
    double *x = malloc(sizeof(double) * N), *Lr = malloc(sizeof(double) * N);
    or_coeffs k;
    coeffs_alloc(&k, n, m);
#define IDX(i, j) (colmajor ? (size_t)(j) * n + (i) : (size_t)(i) * m + (j))
#define BAND(r, c) band[(size_t)(r) * (bw + 1) + ((r) - (c))]
    double r0 = 0;
    or_apply_L(phi, w, Fn, n, m, h, p, n0m0, A1, Lr);
    for (size_t q = 0; q < N; ++q) r0 += (rhs[q] - Lr[q]) * (rhs[q] - Lr[q]);
    r0 = sqrt(r0);
    int it = 0;
    while (it < p->coarse_maxit) {
        double res = 0;
        if (it > 0) {
            or_apply_L(phi, w, Fn, n, m, h, p, n0m0, A1, Lr);
            for (size_t q = 0; q < N; ++q) res += (rhs[q] - Lr[q]) * (rhs[q] - Lr[q]);
            res = sqrt(res);
            if (res <= p->coarse_tol * r0 || res == 0) break;
        }
        if (r0 == 0) break;
        frozen_coeffs(phi, w, Fn, rhs, n, m, h, p, n0m0, A1, &k);
        memset(band, 0, sizeof(double) * N * (bw + 1));
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < m; ++j) {
                size_t q = (size_t)i * m + j, r = IDX(i, j);
                double dl = k.delta[q];
                BAND(r, r) = (k.A[q] + k.B[q] + k.C[q] + k.D[q]) / dl + p->inv_tau;
                if (i > 0) { size_t c = IDX(i - 1, j); if (c < r) BAND(r, c) = -k.B[q] / dl; }
                if (i + 1 < n) { size_t c = IDX(i + 1, j); if (c < r) BAND(r, c) = -k.A[q] / dl; }
                if (j > 0) { size_t c = IDX(i, j - 1); if (c < r) BAND(r, c) = -k.D[q] / dl; }
                if (j + 1 < m) { size_t c = IDX(i, j + 1); if (c < r) BAND(r, c) = -k.C[q] / dl; }
                x[r] = -k.f[q] / dl;   /* f = delta (Fn + area + rhs) */
            }
        /* banded Cholesky, lower factor in place */
        for (size_t r = 0; r < N; ++r) {
            size_t c0 = r >= (size_t)bw ? r - bw : 0;
            for (size_t c = c0; c <= r; ++c) {
                double s = BAND(r, c);
                size_t t0 = c >= (size_t)bw ? c - bw : 0;
                if (t0 < c0) t0 = c0;
                for (size_t t = t0; t < c; ++t) s -= BAND(r, t) * BAND(c, t);
                if (c == r) {
                    if (!(s > 0)) { coeffs_free(&k); free(band); free(x); free(Lr); return -1; }
                    BAND(r, r) = sqrt(s);
                } else {
                    BAND(r, c) = s / BAND(c, c);
                }
            }
        }
        for (size_t r = 0; r < N; ++r) {          /* forward: L y = b */
            size_t c0 = r >= (size_t)bw ? r - bw : 0;
            double s = x[r];
            for (size_t c = c0; c < r; ++c) s -= BAND(r, c) * x[c];
            x[r] = s / BAND(r, r);
        }
        for (size_t rr = N; rr-- > 0;) {          /* backward: L^T x = y */
            double s = x[rr];
            size_t c1 = rr + bw < N - 1 ? rr + bw : N - 1;
            for (size_t c = rr + 1; c <= c1; ++c) s -= BAND(c, rr) * x[c];
            x[rr] = s / BAND(rr, rr);
        }
        double dmax = 0, pmax = 1;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < m; ++j) {
                double v = x[IDX(i, j)], o = phi[(size_t)i * m + j];
                if (fabs(v - o) > dmax) dmax = fabs(v - o);
                if (fabs(v) > pmax) pmax = fabs(v);
                phi[(size_t)i * m + j] = v;
            }
        ++it;
        if (dmax <= 1e-14 * pmax) break;     /* stationary to rounding */
    }
#undef IDX
#undef BAND
    coeffs_free(&k);
    free(band); free(x); free(Lr);
    return it;
}

/* ------------------------------------------------------------------------------------- */
/* AOS time marching (Algorithm 1, "using e.g. time-marching or AOS"; Sec. 5: 100 AOS      */
/* iterations on the coarsest grid, and the baseline of Table 6)                          */
/* ------------------------------------------------------------------------------------- */

/* One AOS iteration (additive operator splitting, Weickert, ter Haar Romeny and Viergever,
 * 1998) for the artificial evolution d phi / ds = L(phi) - rhs of one pseudo-time step, with
 * the coefficients frozen at the current phi:
 *   L(phi) - rhs = A_x phi + A_y phi - phi / tau + c,   c = -(Fn + area + rhs)
 * where A_x couples each cell to its east / west neighbours (C, D over delta) and A_y to its
 * south / north neighbours (A, B over delta), and Fn already holds -phi^n / tau.  The reaction
 * term is split evenly between the two directions and kept implicit:
 *   phi <- 1/2 sum_l (I (1 + dt / tau) - 2 dt A_l)^{-1} (phi + dt c),
 * each inverse a set of tridiagonal solves along rows (l = x) or columns (l = y).
 * Pinned by: consistency with L (the step over dt tends to L(phi) - rhs as dt -> 0, with an
 * O(dt) error), the closed form of the reaction-only problem (mu = 0), convergence of the
 * iteration to a fixed point whose residual shrinks with dt. */
void or_aos_iteration(double *phi, const double *w, const double *Fn, const double *rhs, int n, int m,
                      double h, const or_params *p, double n0m0, double A1, double dt)
{
    size_t N = (size_t)n * m;
    or_coeffs k;
    coeffs_alloc(&k, n, m);
    frozen_coeffs(phi, w, Fn, rhs, n, m, h, p, n0m0, A1, &k);
    double area = area_term(phi, n, m, h, p, n0m0, A1);
    double *src = malloc(sizeof(double) * N), *yx = malloc(sizeof(double) * N);
    int L = n > m ? n : m;
    double *lo = malloc(sizeof(double) * L), *di = malloc(sizeof(double) * L);
    double *up = malloc(sizeof(double) * L), *r = malloc(sizeof(double) * L);
    for (size_t q = 0; q < N; ++q) src[q] = phi[q] - dt * (Fn[q] + area + (rhs ? rhs[q] : 0.0));
    const double diag0 = 1.0 + dt * p->inv_tau;
    for (int dir = 0; dir < 2; ++dir) {           /* 0: rows (A_x), 1: columns (A_y) */
        int nl = dir == 0 ? n : m, len = dir == 0 ? m : n;
        for (int line = 0; line < nl; ++line) {
            for (int t = 0; t < len; ++t) {
                int i = dir == 0 ? line : t, j = dir == 0 ? t : line;
                size_t q = (size_t)i * m + j;
                double cp = (dir == 0 ? k.D[q] : k.B[q]) / k.delta[q];   /* previous cell */
                double cn = (dir == 0 ? k.C[q] : k.A[q]) / k.delta[q];   /* next cell */
                lo[t] = -2.0 * dt * cp;
                up[t] = -2.0 * dt * cn;
                di[t] = diag0 + 2.0 * dt * (cp + cn);
                r[t] = src[q];
            }
            for (int t = 1; t < len; ++t) {
                double wgt = lo[t] / di[t - 1];
                di[t] -= wgt * up[t - 1];
                r[t] -= wgt * r[t - 1];
            }
            double x = r[len - 1] / di[len - 1];
            for (int t = len - 1; t >= 0; --t) {
                if (t < len - 1) x = (r[t] - up[t] * x) / di[t];
                int i = dir == 0 ? line : t, j = dir == 0 ? t : line;
                size_t q = (size_t)i * m + j;
                if (dir == 0) yx[q] = x;
                else phi[q] = 0.5 * (yx[q] + x);
            }
        }
    }
    free(src); free(yx); free(lo); free(di); free(up); free(r);
    coeffs_free(&k);
}

/* The coarsest solve by `iters` AOS iterations (the paper's choice: 100). */
static void or_aos_solve(double *phi, const double *w, const double *Fn, const double *rhs, int n, int m,
                         double h, const or_params *p, double n0m0, double A1, int iters, double dt)
{
    for (int it = 0; it < iters; ++it) or_aos_iteration(phi, w, Fn, rhs, n, m, h, p, n0m0, A1, dt);
}

/* ------------------------------------------------------------------------------------- */
/* FAS multigrid (Sec. 3.1, Algorithm 1) and the outer driver (Sec. 5)                    */
/* ------------------------------------------------------------------------------------- */

typedef struct {
    int n, m;
    double h;
    double *phi, *phi0, *rhs, *w, *z, *d, *Fn, *tmp;
    double *omega;          /* relaxation weights of the point updates on this grid (NULL = 1) */
} or_level;

typedef struct {
    or_params p;
    int nlev;
    or_level *lv;
    double c1, c2, A1, n0m0;
    double res0;            /* ||L(phi^n)|| at the start of the current step */
    double *phin;           /* phi at the start of the current step (finest grid) */
    int picard_last;
} or_solver;

/* One outer iteration of smoother `kind` with frozen coefficients k. */
static void run_smoother(const or_coeffs *k, double Sigma, int kind, double *phi)
{
    switch (kind) {
        case 0: hs2_parallel(k, Sigma, phi); break;
        case 1: hs2_lexicographic(k, Sigma, phi); break;
        case 2: gsline_columns(k, phi); break;
        case 3: gsline_zebra(k, phi); break;
        case 4: hs1_lexicographic(k, Sigma, phi); break;
        default: hs1_parallel(k, Sigma, phi); break;
    }
}

/* One outer iteration of the selected smoother on level l (Algorithm 1, "Smoother"). */
static void smooth(or_solver *s, int l)
{
    or_level *L = &s->lv[l];
    or_coeffs k;
    coeffs_alloc(&k, L->n, L->m);
    frozen_coeffs(L->phi, L->w, L->Fn, L->rhs, L->n, L->m, L->h, &s->p, s->n0m0, s->A1, &k);
    k.omega = L->omega;
    run_smoother(&k, s->p.Sigma, s->p.smoother, L->phi);
    coeffs_free(&k);
}

/* r = rhs - L(phi) on level l, into tmp. */
static void residual(or_solver *s, int l)
{
    or_level *L = &s->lv[l];
    or_apply_L(L->phi, L->w, L->Fn, L->n, L->m, L->h, &s->p, s->n0m0, s->A1, L->tmp);
    #pragma omp parallel for
    for (size_t q = 0; q < (size_t)L->n * L->m; ++q) L->tmp[q] = L->rhs[q] - L->tmp[q];
}

/* FASMG (Algorithm 1) with gamma = 1 (a V-cycle). */
static void fas_vcycle(or_solver *s, int l)
{
    or_level *L = &s->lv[l];
    if (l == s->nlev - 1) {
if (s->p.coarse_solver == 1) {
            or_aos_solve(L->phi, L->w, L->Fn, L->rhs, L->n, L->m, L->h, &s->p, s->n0m0, s->A1,
                         s->p.coarse_maxit, s->p.aos_dt);
            s->picard_last = s->p.coarse_maxit;
        } else {
            s->picard_last = or_coarse_solve(L->phi, L->w, L->Fn, L->rhs, L->n, L->m, L->h, &s->p,
                                         s->n0m0, s->A1);
        }
        return;
    }
    or_level *Cg = &s->lv[l + 1];
    size_t Nc = (size_t)Cg->n * Cg->m;
    for (int t = 0; t < s->p.nu1; ++t) smooth(s, l);            /* pre-smoothing */
    residual(s, l);                                             /* r^h = f^h - N^h phi^h */
    or_restrict(L->tmp, L->n, L->m, Cg->rhs);                   /* r^{2h} = I r^h */
    or_restrict(L->phi, L->n, L->m, Cg->phi);                   /* phi^{2h} = I phi^h */
    memcpy(Cg->phi0, Cg->phi, sizeof(double) * Nc);             /* Phi^{2h} = phi^{2h} */
    or_apply_L(Cg->phi0, Cg->w, Cg->Fn, Cg->n, Cg->m, Cg->h, &s->p, s->n0m0, s->A1, Cg->tmp);
    for (size_t q = 0; q < Nc; ++q) Cg->rhs[q] += Cg->tmp[q];   /* f^{2h} = N^{2h} phi^{2h} + r^{2h} */
    fas_vcycle(s, l + 1);
    for (size_t q = 0; q < Nc; ++q) Cg->tmp[q] = Cg->phi[q] - Cg->phi0[q];   /* e^{2h} */
    or_interpolate_add(Cg->tmp, Cg->n, Cg->m, L->phi, L->n, L->m);          /* phi += I e */
    for (int t = 0; t < s->p.nu2; ++t) smooth(s, l);            /* post-smoothing */
}

static double norm2(const double *a, size_t N)
{
    double s = 0;
    for (size_t q = 0; q < N; ++q) s += a[q] * a[q];
    return sqrt(s);
}

/* Builds the solver: image-derived data on every level (Sec. 2.2), initial phi from the
 * markers and initial c1, c2 (Sec. 5, parameter choices). */
or_solver *or_create(const double *image, int n, int m, const double *mx, const double *my, int k,
                     const or_params *p)
{
    or_solver *s = calloc(1, sizeof(or_solver));
    s->p = *p;
    s->nlev = p->levels;
    s->lv = calloc(s->nlev, sizeof(or_level));
    s->n0m0 = (double)n * m;
    int nn = n, mm = m;
    for (int l = 0; l < s->nlev; ++l) {
        or_level *L = &s->lv[l];
        size_t N = (size_t)nn * mm;
        L->n = nn; L->m = mm; L->h = ldexp(1.0, l);
        L->phi = calloc(N, sizeof(double)); L->phi0 = calloc(N, sizeof(double));
        L->rhs = calloc(N, sizeof(double)); L->w = calloc(N, sizeof(double));
        L->z = calloc(N, sizeof(double)); L->d = calloc(N, sizeof(double));
        L->Fn = calloc(N, sizeof(double)); L->tmp = calloc(N, sizeof(double));
        nn /= 2; mm /= 2;
    }
    s->phin = calloc((size_t)n * m, sizeof(double));
    or_level *F = &s->lv[0];
    size_t N = (size_t)n * m;
    memcpy(F->z, image, sizeof(double) * N);
    double *zb = malloc(sizeof(double) * N);
    or_gauss_blur(image, n, m, p->sigma_blur, zb);
    or_edge_detector(zb, n, m, p->beta_edge, F->w);              /* g */
    free(zb);
    or_distance(n, m, mx, my, k, p->sigma_d, F->d);
    if (p->model == 1)
        for (size_t q = 0; q < N; ++q) F->w[q] *= F->d[q];       /* Rada-Chen: d g */
    for (int l = 1; l < s->nlev; ++l) {
        or_level *Pf = &s->lv[l - 1], *Lc = &s->lv[l];
        or_restrict(Pf->w, Pf->n, Pf->m, Lc->w);
        or_restrict(Pf->z, Pf->n, Pf->m, Lc->z);
        or_restrict(Pf->d, Pf->n, Pf->m, Lc->d);
    }
    double r0 = 0.05 * (n > m ? n : m);
    or_initial_phi(n, m, mx, my, k, r0, F->phi, &s->A1);
    or_region_means(F->phi, F->z, n, m, p->eps, &s->c1, &s->c2);
    return s;
}

void or_destroy(or_solver *s)
{
    for (int l = 0; l < s->nlev; ++l) {
        or_level *L = &s->lv[l];
        free(L->phi); free(L->phi0); free(L->rhs); free(L->w); free(L->z); free(L->d);
        free(L->Fn); free(L->tmp); free(L->omega);
    }
    free(s->lv); free(s->phin); free(s);
}

/* Starts one pseudo-time step from the current phi: phi^n = phi, the fitting field of every
 * level from the current c1, c2 and the restricted phi^n, zero right-hand side on the finest
 * grid, and the reference residual ||L(phi^n)||. */
double or_begin_step(or_solver *s)
{
    or_level *F = &s->lv[0];
    size_t N = (size_t)F->n * F->m;
    memcpy(s->phin, F->phi, sizeof(double) * N);
    double *pn = malloc(sizeof(double) * N), *pc = malloc(sizeof(double) * N);
    memcpy(pn, F->phi, sizeof(double) * N);
    for (int l = 0; l < s->nlev; ++l) {
        or_level *L = &s->lv[l];
        if (l > 0) {
            or_restrict(pn, s->lv[l - 1].n, s->lv[l - 1].m, pc);
            memcpy(pn, pc, sizeof(double) * (size_t)L->n * L->m);
        }
        or_fitting(L->z, L->d, pn, L->n, L->m, s->c1, s->c2, &s->p, L->Fn);
        memset(L->rhs, 0, sizeof(double) * (size_t)L->n * L->m);
    }
    free(pn); free(pc);
    residual(s, 0);
    s->res0 = norm2(F->tmp, N);
    return s->res0;
}

/* One V-cycle on the finest grid; returns rho = ||L(phi)|| / ||L(phi^n)||. */
double or_vcycle(or_solver *s)
{
    fas_vcycle(s, 0);
    residual(s, 0);
    double r = norm2(s->lv[0].tmp, (size_t)s->lv[0].n * s->lv[0].m);
    return s->res0 > 0 ? r / s->res0 : r;
}

/* Ends a step: new c1, c2 from the current phi (Sec. 5: updated at the end of each multigrid
 * iteration) and the paper's stopping quantity ||phi^{k+1} - phi^k|| / ||phi^k||. */
double or_end_step(or_solver *s)
{
    or_level *F = &s->lv[0];
    size_t N = (size_t)F->n * F->m;
    or_region_means(F->phi, F->z, F->n, F->m, s->p.eps, &s->c1, &s->c2);
    double dn = 0, pn = 0;
    for (size_t q = 0; q < N; ++q) {
        dn += (F->phi[q] - s->phin[q]) * (F->phi[q] - s->phin[q]);
        pn += s->phin[q] * s->phin[q];
    }
    return pn > 0 ? sqrt(dn / pn) : sqrt(dn);
}

/* AOS on the finest grid for the current pseudo-time step (the AOS method of Table 6): up to
 * max_iter iterations with step dt until the relative change ||phi^{k+1} - phi^k|| / ||phi^k||
 * falls below eta.  Returns the iterations run; *rho gets ||L(phi) - rhs|| / ||L(phi^n)||. */
int or_solver_aos(or_solver *s, double dt, int max_iter, double eta, double *rho)
{
    or_level *F = &s->lv[0];
    size_t N = (size_t)F->n * F->m;
    double *prev = malloc(sizeof(double) * N);
    int it = 0;
    while (it < max_iter) {
        memcpy(prev, F->phi, sizeof(double) * N);
        or_aos_iteration(F->phi, F->w, F->Fn, F->rhs, F->n, F->m, F->h, &s->p, s->n0m0, s->A1, dt);
        ++it;
        double dn = 0, pn = 0;
        for (size_t q = 0; q < N; ++q) {
            dn += (F->phi[q] - prev[q]) * (F->phi[q] - prev[q]);
            pn += prev[q] * prev[q];
        }
        if (sqrt(dn) <= eta * sqrt(pn)) break;
    }
    free(prev);
    residual(s, 0);
    double r = norm2(F->tmp, N);
    if (rho) *rho = s->res0 > 0 ? r / s->res0 : r;
    return it;
}

/* Energy of a level set on the finest grid (the functionals of Sec. 2.2: eq. scfunc for
 * Spencer-Chen, eq. rcfunc for Rada-Chen; Table 7 reports it after each cycle), in pixel units
 * (h = 1, areas summed over cells):
 *   E = sum_ij [ mu w |grad H_eps(phi)| + lambda1 (z - c1)^2 H + lambda2 (z - c2)^2 (1 - H) ]
 *       + theta sum_ij d H                               (Spencer-Chen)
 *       + nu n m (sum_ij H / (n m) - A1 / (n m))^2       (Rada-Chen)
 * with H = H_eps(phi), |grad H_eps(phi)| = delta_eps(phi) |grad phi|_beta (central differences,
 * mirror ghosts, as in the coefficients), w = g (Spencer-Chen) or d g (Rada-Chen).  Reading:
 * the two squared area terms of eq. rcfunc are one term, since |Omega_2| - A2 = -(|Omega_1| - A1);
 * it is written with area fractions and scaled so that its first variation is the area term
 * 2 nu (sum H / (n m) - A1 / (n m)) of the equation solved (the factor of 2 absorbed in nu, as
 * there).  Pinned by: the co-area formula (a straight and a circular contour give mu times
 * their length), the fitting terms of a sharp two-region level set against region variances,
 * the distance term and the area term of a sharp level set against their closed forms. */
double or_energy(const double *phi, const double *z, const double *w, const double *d, int n, int m,
                 double c1, double c2, double A1, const or_params *p)
{
    double E = 0.0, sH = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            size_t q = (size_t)i * m + j;
            double H = heaviside(phi[q], p->eps);
            double len = dirac(phi[q], p->eps) * grad_norm(phi, n, m, 1.0, p->beta, i, j);
            double e = p->mu * w[q] * len + p->lambda1 * (z[q] - c1) * (z[q] - c1) * H
                     + p->lambda2 * (z[q] - c2) * (z[q] - c2) * (1.0 - H);
            if (p->model == 0) e += p->theta * d[q] * H;
            E += e;
            sH += H;
        }
    if (p->model == 1) {
        double nm = (double)n * m, a = sH / nm - A1 / nm;
        E += p->nu * nm * a * a;
    }
    return E;
}

/* The energy of the solver's current finest-grid phi with its current c1, c2. */
double or_solver_energy(const or_solver *s)
{
    const or_level *F = &s->lv[0];
    return or_energy(F->phi, F->z, F->w, F->d, F->n, F->m, s->c1, s->c2, s->A1, &s->p);
}

/* Accessors used by the tests. */
void or_get_phi(const or_solver *s, double *out)
{
    memcpy(out, s->lv[0].phi, sizeof(double) * (size_t)s->lv[0].n * s->lv[0].m);
}
void or_set_phi(or_solver *s, const double *in)
{
    memcpy(s->lv[0].phi, in, sizeof(double) * (size_t)s->lv[0].n * s->lv[0].m);
}
void or_get_level(const or_solver *s, int l, int which, double *out)
{
    const or_level *L = &s->lv[l];
    const double *src = which == 0 ? L->phi : which == 1 ? L->w : which == 2 ? L->z
                      : which == 3 ? L->d : which == 4 ? L->Fn : which == 5 ? L->rhs : L->tmp;
    memcpy(out, src, sizeof(double) * (size_t)L->n * L->m);
}
void or_get_scalars(const or_solver *s, double *out /* c1, c2, A1, res0, picard_last */)
{
    out[0] = s->c1; out[1] = s->c2; out[2] = s->A1; out[3] = s->res0; out[4] = s->picard_last;
}
void or_set_c(or_solver *s, double c1, double c2) { s->c1 = c1; s->c2 = c2; }

/* Sets 1/tau of the following pseudo-time steps (the step-size control of the outer driver
 * halves tau when a step stops contracting; the next or_begin_step folds the new value into
 * the fitting field's -phi^n / tau term). */
void or_set_inv_tau(or_solver *s, double inv_tau) { s->p.inv_tau = inv_tau; }

/* Per-cell relaxation weights of the point updates of the parallel Hybrid Smoother 2 on grid l
 * (NULL: back to 1).  Used by the learned relaxation-weights extension. */
void or_set_omega(or_solver *s, int l, const double *w)
{
    or_level *L = &s->lv[l];
    size_t N = (size_t)L->n * L->m;
    if (!w) { free(L->omega); L->omega = NULL; return; }
    if (!L->omega) L->omega = malloc(sizeof(double) * N);
    memcpy(L->omega, w, sizeof(double) * N);
}

/* Frozen coefficients of an arbitrary grid function, for the tests (A, B, C, D, S, f, delta
 * each n*m, in that order in out). */
void or_frozen_coeffs(const double *phi, const double *w, const double *Fn, const double *rhs,
                      int n, int m, double h, const or_params *p, double n0m0, double A1, double *out)
{
    or_coeffs k;
    coeffs_alloc(&k, n, m);
    frozen_coeffs(phi, w, Fn, rhs, n, m, h, p, n0m0, A1, &k);
    size_t N = (size_t)n * m;
    memcpy(out, k.A, N * sizeof(double)); memcpy(out + N, k.B, N * sizeof(double));
    memcpy(out + 2 * N, k.C, N * sizeof(double)); memcpy(out + 3 * N, k.D, N * sizeof(double));
    memcpy(out + 4 * N, k.S, N * sizeof(double)); memcpy(out + 5 * N, k.f, N * sizeof(double));
    memcpy(out + 6 * N, k.delta, N * sizeof(double));
    coeffs_free(&k);
}

/* One outer smoothing iteration with given frozen coefficients (A..D, S, f as above), for the
 * tests: kind as or_params.smoother. */
void or_smooth_given(const double *coef, int n, int m, double Sigma, int kind, double *phi)
{
    size_t N = (size_t)n * m;
    or_coeffs k;
    k.n = n; k.m = m;
    k.A = (double *)coef; k.B = (double *)coef + N; k.C = (double *)coef + 2 * N;
    k.D = (double *)coef + 3 * N; k.S = (double *)coef + 4 * N; k.f = (double *)coef + 5 * N;
    k.delta = NULL;
    k.omega = NULL;
    run_smoother(&k, Sigma, kind, phi);
}

/* As or_smooth_given, with per-cell relaxation weights of the point updates. */
void or_smooth_given_omega(const double *coef, const double *omega, int n, int m, double Sigma, int kind,
                           double *phi)
{
    size_t N = (size_t)n * m;
    or_coeffs k;
    k.n = n; k.m = m;
    k.A = (double *)coef; k.B = (double *)coef + N; k.C = (double *)coef + 2 * N;
    k.D = (double *)coef + 3 * N; k.S = (double *)coef + 4 * N; k.f = (double *)coef + 5 * N;
    k.delta = NULL;
    k.omega = omega;
    run_smoother(&k, Sigma, kind, phi);
}

/* Member flags of the four sweeps (parallel ordering) for given coefficients: out[k*N + q]. */
void or_members(const double *coef, int n, int m, double Sigma, int piece, int *out)
{
    size_t N = (size_t)n * m;
    or_coeffs k;
    k.n = n; k.m = m;
    k.A = (double *)coef; k.B = (double *)coef + N; k.C = (double *)coef + 2 * N;
    k.D = (double *)coef + 3 * N; k.S = NULL; k.f = NULL; k.delta = NULL; k.omega = NULL;
    int *star = malloc(sizeof(int) * N);
    for (int sweep = 0; sweep < 4; ++sweep) {
        star_flags(&k, Sigma, sweep, star);
        sweep_members(&k, star, sweep, piece > 0 ? piece : (sweep < 2 ? m : n), out + sweep * N);
    }
    free(star);
}
