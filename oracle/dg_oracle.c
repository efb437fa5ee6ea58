/*
 * dg_oracle.c -- plain, slow FP64 CPU oracle for the modal Discontinuous
 * Galerkin discretisation of the rotating shallow water equations on a
 * longitude-latitude mesh of the sphere (arxiv 2303.11767, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path
 * is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Every step is written out in the plainest form that follows the paper:
 *   - nodal values by direct double sums over all modes (no sum factorisation),
 *   - volume, edge and source integrals by direct loops over quadrature points,
 *   - the Rusanov flux literally on the conserved variable U = cos(theta) q,
 *   - the full (p+1)^2 x (p+1)^2 cos(theta)-weighted element mass matrix,
 *     assembled by quadrature and inverted by Cholesky (no Kronecker shortcut),
 *   - explicit Runge-Kutta from the Butcher tableaux (Table "Butcher").
 *
 * Passages followed (paper section / equation):
 *   Eq. (sph3) and the definitions of U, F, G, S that follow it  -> flux_sphere()
 *   Eq. (operators), lat-lon parameterisation                     -> element geometry
 *   Eq. (dg_parts) weak form                                      -> oracle_rhs_element()
 *   Eq. (rusanov) Rusanov flux                                    -> numerical_flux()
 *   Eq. (basis_expansion), bivariate Legendre modal basis         -> basis_phi()
 *   Eq. (ode) and the cos(theta)-weighted mass matrix             -> oracle_mass_matrix()
 *   Table "Butcher" (SSP RK1..RK4)                                -> oracle_rk_step()
 *   Sec. 2, Courant number p c dt / H                             -> oracle_max_dt()
 *   Eq. (lin_adv) planar linear advection (validation problem)    -> flux_advection()
 *   Sec. 4.3 planar shallow water on the f-plane                  -> flux_plane_swe()
 *
 * Readings where the paper is silent:
 *   basis: orthonormal Legendre L_k = sqrt((2k+1)/2) P_k, mode m = b*n + a with
 *     a the lambda-degree; n = p+1 Gauss-Legendre points per direction for the
 *     volume, source and edge integrals; nm = p+9 points for mass matrices,
 *     projections and norms; local Rusanov alpha = max over both sides of the
 *     largest eigenvalue of dF/dU (resp. dG/dU); the whole numerical flux is zero
 *     on the pole edges; integrals in (lambda, theta) without R^2.
 *   well-balanced option: the tendency of the fluid at rest at the
 *     reference depth (the quadrature residual of its constant pressure) is
 *     removed from every tendency, so that rest state is exactly steady.
 *   global Rusanov mode (optional): the one-sided speeds |u| + sqrt(gh) and
 *     |v| + sqrt(gh) of every face are replaced by their maxima over all Gauss
 *     points of the stage input, inside the same eigenvalue (so the lambda
 *     faces keep their 1/(R cos theta) and the theta faces their 1/R).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2
#define ORACLE_ENONPHYSICAL 5

#define PHYS_SPHERE_SWE 0
#define PHYS_PLANE_ADVECTION 1
#define PHYS_PLANE_SWE 2

typedef struct {
    int physics;
    int nx, ny;        /* elements in x (lambda) and y (theta) */
    int p, n, nphi;    /* degree, points per direction, modes per field */
    int nf;            /* fields: 3 for SWE, 1 for advection */
    int nm;            /* points per direction for mass, projection and norms */
    double R, g, omega;
    double fcor;       /* planar shallow water: constant Coriolis parameter (f-plane) */
    double bx, by;     /* advection velocity (planar advection only) */
    int alpha_speed;   /* planar advection: 1 -> alpha = |beta|, 0 -> |beta . n| */
    int alpha_global;  /* sphere: 1 -> the wave speeds of every face are the global maxima */
    /* well-balanced option (sphere): the tendency of the fluid at rest at
     * depth href, per latitude row, is subtracted from every tendency */
    double *rest_res, *rest_mag;   /* ny x nf*nphi, NULL when off */
    double x0, y0, dx, dy;
    double *xg, *wg;   /* n-point Gauss-Legendre rule on [-1, 1] */
    double *xm, *wm;   /* nm-point rule */
    double *minv;      /* per row y-index: nphi*nphi inverse mass matrix */
    /* basis values cached at the quadrature points (plain tables of phi_m):
     * volume nodes q = qy*n + qx: phiv, dphix, dphiy [q][m];
     * edge points of edge e (0 W, 1 E, 2 S, 3 N), point k: phie [e][k][m];
     * nm x nm points: phim [qy*nm + qx][m] */
    double *phiv, *dphix, *dphiy, *phie, *phim;
    int nthreads;
} oracle_ctx;

/* ---------------------------------------------------------------- rules -- */

/* Legendre polynomial P_k(x) and its derivative by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre_pd(int k, double x, double *pk, double *dpk)
{
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (k == 0) { *pk = 1.0; *dpk = 0.0; return; }
    for (int j = 1; j < k; ++j) {
        double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        double d2 = d0 + (2.0 * j + 1.0) * p1; /* P'_{j+1} = P'_{j-1} + (2j+1) P_j */
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    *pk = p1; *dpk = d1;
}

/* Orthonormal Legendre L_k = sqrt((2k+1)/2) P_k on [-1, 1]. */
double oracle_legendre(int k, double x)
{
    double pk, dpk;
    legendre_pd(k, x, &pk, &dpk);
    return sqrt((2.0 * k + 1.0) / 2.0) * pk;
}

double oracle_legendre_deriv(int k, double x)
{
    double pk, dpk;
    legendre_pd(k, x, &pk, &dpk);
    return sqrt((2.0 * k + 1.0) / 2.0) * dpk;
}

/* n-point Gauss-Legendre rule: nodes are the roots of P_n, found by Newton's
 * method; weights 2 / ((1 - x^2) P_n'(x)^2).  Returned in ascending order. */
int oracle_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return ORACLE_EINVAL;
    for (int i = 0; i < n; ++i) {
        double xi = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn, dpn;
            legendre_pd(n, xi, &pn, &dpn);
            double dx = pn / dpn;
            xi -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        double pn, dpn;
        legendre_pd(n, xi, &pn, &dpn);
        /* i = 0 is the largest root; store ascending */
        x[n - 1 - i] = xi;
        w[n - 1 - i] = 2.0 / ((1.0 - xi * xi) * dpn * dpn);
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
    return ORACLE_OK;
}

/* ---------------------------------------------------------------- basis -- */

/* phi_m(xi, eta) = L_a(xi) L_b(eta), m = b*n + a   (Eq. basis_expansion). */
static double basis_phi(int n, int m, double xi, double eta)
{
    return oracle_legendre(m % n, xi) * oracle_legendre(m / n, eta);
}

static double basis_dphi_dxi(int n, int m, double xi, double eta)
{
    return oracle_legendre_deriv(m % n, xi) * oracle_legendre(m / n, eta);
}

static double basis_dphi_deta(int n, int m, double xi, double eta)
{
    return oracle_legendre(m % n, xi) * oracle_legendre_deriv(m / n, eta);
}

/* -------------------------------------------------------------- geometry -- */

/* Mass-matrix weight: cos(theta) on the sphere (conserved U = cos(theta) q),
 * 1 on the plane. */
static double metric_weight(const oracle_ctx *c, double y)
{
    return c->physics == PHYS_SPHERE_SWE ? cos(y) : 1.0;
}

static double elem_x(const oracle_ctx *c, int i, double xi)
{
    return c->x0 + i * c->dx + 0.5 * (1.0 + xi) * c->dx;
}

static double elem_y(const oracle_ctx *c, int j, double eta)
{
    return c->y0 + j * c->dy + 0.5 * (1.0 + eta) * c->dy;
}

/* Solve the symmetric positive definite system by Cholesky and return the
 * full inverse in place of a (size k x k, row major). */
static int cholesky_inverse(int k, double *a)
{
    double *l = calloc((size_t)k * k, sizeof(double));
    double *inv = calloc((size_t)k * k, sizeof(double));
    if (!l || !inv) { free(l); free(inv); return ORACLE_ENOMEM; }
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = a[i * k + j];
            for (int t = 0; t < j; ++t) s -= l[i * k + t] * l[j * k + t];
            if (i == j) {
                if (s <= 0.0) { free(l); free(inv); return ORACLE_EINVAL; }
                l[i * k + i] = sqrt(s);
            } else {
                l[i * k + j] = s / l[j * k + j];
            }
        }
    }
    for (int col = 0; col < k; ++col) {
        double *y = calloc((size_t)k, sizeof(double));
        for (int i = 0; i < k; ++i) {          /* L y = e_col */
            double s = (i == col) ? 1.0 : 0.0;
            for (int t = 0; t < i; ++t) s -= l[i * k + t] * y[t];
            y[i] = s / l[i * k + i];
        }
        for (int i = k - 1; i >= 0; --i) {     /* L^T x = y */
            double s = y[i];
            for (int t = i + 1; t < k; ++t) s -= l[t * k + i] * inv[t * k + col];
            inv[i * k + col] = s / l[i * k + i];
        }
        free(y);
    }
    memcpy(a, inv, sizeof(double) * k * k);
    free(l); free(inv);
    return ORACLE_OK;
}

/* Full element mass matrix of row jy, M_ij = int phi_i phi_j w(y) dx dy, by the
 * nm x nm Gauss-Legendre rule (Eq. ode and the cos(theta)-weighted M). */
void oracle_mass_matrix(const oracle_ctx *c, int jy, double *mass)
{
    int np = c->nphi;
    double jac = 0.25 * c->dx * c->dy;
    for (int r = 0; r < np; ++r)
        for (int s = 0; s < np; ++s) {
            double acc = 0.0;
            for (int qy = 0; qy < c->nm; ++qy)
                for (int qx = 0; qx < c->nm; ++qx) {
                    double xi = c->xm[qx], eta = c->xm[qy];
                    acc += c->wm[qx] * c->wm[qy] * jac * basis_phi(c->n, r, xi, eta) *
                           basis_phi(c->n, s, xi, eta) * metric_weight(c, elem_y(c, jy, eta));
                }
            mass[r * np + s] = acc;
        }
}

/* ---------------------------------------------------------------- setup -- */

void oracle_destroy(oracle_ctx *c)
{
    if (!c) return;
    free(c->xg); free(c->wg); free(c->xm); free(c->wm); free(c->minv);
    free(c->phiv); free(c->dphix); free(c->dphiy); free(c->phie); free(c->phim);
    free(c->rest_res); free(c->rest_mag);
    free(c);
}

/* Reference coordinates of point k of edge e of an element:
 * 0 west (-1, eta_k), 1 east (+1, eta_k), 2 south (xi_k, -1), 3 north (xi_k, +1). */
static void edge_point(const oracle_ctx *c, int e, int k, double *xi, double *eta)
{
    if (e == 0) { *xi = -1.0; *eta = c->xg[k]; }
    else if (e == 1) { *xi = 1.0; *eta = c->xg[k]; }
    else if (e == 2) { *xi = c->xg[k]; *eta = -1.0; }
    else { *xi = c->xg[k]; *eta = 1.0; }
}

static oracle_ctx *ctx_alloc(int physics, int nx, int ny, int p)
{
    if (nx < 1 || ny < 1 || p < 0 || p > 8) return NULL;
    oracle_ctx *c = calloc(1, sizeof(oracle_ctx));
    if (!c) return NULL;
    c->physics = physics;
    c->nx = nx; c->ny = ny; c->p = p; c->n = p + 1; c->nphi = c->n * c->n;
    c->nm = p + 9;
    c->nf = physics == PHYS_PLANE_ADVECTION ? 1 : 3;
    c->nthreads = 1;
    c->xg = malloc(sizeof(double) * c->n); c->wg = malloc(sizeof(double) * c->n);
    c->xm = malloc(sizeof(double) * c->nm); c->wm = malloc(sizeof(double) * c->nm);
    c->minv = malloc(sizeof(double) * (size_t)ny * c->nphi * c->nphi);
    if (!c->xg || !c->wg || !c->xm || !c->wm || !c->minv) { oracle_destroy(c); return NULL; }
    oracle_gauss_legendre(c->n, c->xg, c->wg);
    oracle_gauss_legendre(c->nm, c->xm, c->wm);
    int n = c->n, np = c->nphi, nm = c->nm;
    c->phiv = malloc(sizeof(double) * n * n * np);
    c->dphix = malloc(sizeof(double) * n * n * np);
    c->dphiy = malloc(sizeof(double) * n * n * np);
    c->phie = malloc(sizeof(double) * 4 * n * np);
    c->phim = malloc(sizeof(double) * nm * nm * np);
    if (!c->phiv || !c->dphix || !c->dphiy || !c->phie || !c->phim) { oracle_destroy(c); return NULL; }
    for (int qy = 0; qy < n; ++qy)
        for (int qx = 0; qx < n; ++qx)
            for (int m = 0; m < np; ++m) {
                int q = qy * n + qx;
                c->phiv[q * np + m] = basis_phi(n, m, c->xg[qx], c->xg[qy]);
                c->dphix[q * np + m] = basis_dphi_dxi(n, m, c->xg[qx], c->xg[qy]);
                c->dphiy[q * np + m] = basis_dphi_deta(n, m, c->xg[qx], c->xg[qy]);
            }
    for (int e = 0; e < 4; ++e)
        for (int k = 0; k < n; ++k) {
            double xi, eta;
            edge_point(c, e, k, &xi, &eta);
            for (int m = 0; m < np; ++m) c->phie[(e * n + k) * np + m] = basis_phi(n, m, xi, eta);
        }
    for (int qy = 0; qy < nm; ++qy)
        for (int qx = 0; qx < nm; ++qx)
            for (int m = 0; m < np; ++m)
                c->phim[(qy * nm + qx) * np + m] = basis_phi(n, m, c->xm[qx], c->xm[qy]);
    return c;
}

static int ctx_build_mass(oracle_ctx *c)
{
    size_t np2 = (size_t)c->nphi * c->nphi;
    for (int jy = 0; jy < c->ny; ++jy) {
        double *m = c->minv + jy * np2;
        oracle_mass_matrix(c, jy, m);
        int st = cholesky_inverse(c->nphi, m);
        if (st) return st;
    }
    return ORACLE_OK;
}

/* Sphere: lambda in [0, 2 pi] (nx = nlon columns), theta in [-pi/2, pi/2]
 * (ny = nlat rows), periodic in lambda, zero flux through the pole edges. */
oracle_ctx *oracle_create_sphere(int nlon, int nlat, int p, double R, double g, double omega)
{
    if (R <= 0.0 || g <= 0.0) return NULL;
    oracle_ctx *c = ctx_alloc(PHYS_SPHERE_SWE, nlon, nlat, p);
    if (!c) return NULL;
    c->R = R; c->g = g; c->omega = omega;
    c->x0 = 0.0; c->y0 = -0.5 * M_PI;
    c->dx = 2.0 * M_PI / nlon; c->dy = M_PI / nlat;
    if (ctx_build_mass(c)) { oracle_destroy(c); return NULL; }
    return c;
}

/* Planar shallow water on the f-plane, square domain [0, L]^2, periodic in
 * both directions (the geostrophic adjustment setup of Sec. 4.3). */
oracle_ctx *oracle_create_plane_swe(int nx, int ny, int p, double L, double g, double f)
{
    if (!(L > 0.0) || !(g > 0.0)) return NULL;
    oracle_ctx *c = ctx_alloc(PHYS_PLANE_SWE, nx, ny, p);
    if (!c) return NULL;
    c->g = g; c->fcor = f; c->R = 1.0;
    c->x0 = 0.0; c->y0 = 0.0; c->dx = L / nx; c->dy = L / ny;
    if (ctx_build_mass(c)) { oracle_destroy(c); return NULL; }
    return c;
}

/* Planar scalar advection du/dt + div(beta u) = 0 (Eq. lin_adv) on the unit
 * square, periodic in both directions.  alpha_speed selects the Rusanov alpha:
 * 1 -> |beta|, 0 -> |beta . n|. */
oracle_ctx *oracle_create_plane_advection(int nx, int ny, int p, double bx, double by, int alpha_speed)
{
    oracle_ctx *c = ctx_alloc(PHYS_PLANE_ADVECTION, nx, ny, p);
    if (!c) return NULL;
    c->bx = bx; c->by = by; c->alpha_speed = alpha_speed;
    c->x0 = 0.0; c->y0 = 0.0; c->dx = 1.0 / nx; c->dy = 1.0 / ny;
    if (ctx_build_mass(c)) { oracle_destroy(c); return NULL; }
    return c;
}

void oracle_set_threads(oracle_ctx *c, int nthreads) { c->nthreads = nthreads < 1 ? 1 : nthreads; }

size_t oracle_state_len(const oracle_ctx *c) { return (size_t)c->nx * c->ny * c->nf * c->nphi; }
int oracle_nm(const oracle_ctx *c) { return c->nm; }

/* ---------------------------------------------------------------- physics -- */

/* Sphere fluxes and sources after Eq. (sph3):
 *   F = (1/R) (hu, hu^2 + g h^2/2, huv)
 *   G = (cos(theta)/R) (hv, huv, hv^2 + g h^2/2)
 *   S = (0, (f cos + u sin/R) hv, -g h^2 sin/(2R) - (f cos + u sin/R) hu),
 * with f = 2 Omega sin(theta).  q = (h, hu, hv).  Returns 0 if h <= 0. */
static int flux_sphere(const oracle_ctx *c, const double *q, double theta,
                       double *F, double *G, double *S)
{
    double h = q[0];
    if (!(h > 0.0)) return 0;
    double u = q[1] / h, v = q[2] / h;
    double ct = cos(theta), st = sin(theta);
    double f = 2.0 * c->omega * st;
    double pres = 0.5 * c->g * h * h;
    F[0] = h * u / c->R;
    F[1] = (h * u * u + pres) / c->R;
    F[2] = h * u * v / c->R;
    G[0] = ct * h * v / c->R;
    G[1] = ct * h * u * v / c->R;
    G[2] = ct * (h * v * v + pres) / c->R;
    double cor = f * ct + u * st / c->R;
    S[0] = 0.0;
    S[1] = cor * h * v;
    S[2] = -c->g * h * h * st / (2.0 * c->R) - cor * h * u;
    return 1;
}

/* Planar shallow water on the f-plane (Sec. 4.3, geostrophic adjustment):
 *   F = (hu, hu u + g h^2/2, hu v),  G = (hv, hv u, hv v + g h^2/2),
 *   S = (0, f hv, -f hu).  Returns 0 if h <= 0. */
static int flux_plane_swe(const oracle_ctx *c, const double *q, double *F, double *G, double *S)
{
    double h = q[0];
    if (!(h > 0.0)) return 0;
    double u = q[1] / h, v = q[2] / h;
    double pres = 0.5 * c->g * h * h;
    F[0] = h * u;
    F[1] = h * u * u + pres;
    F[2] = h * u * v;
    G[0] = h * v;
    G[1] = h * v * u;
    G[2] = h * v * v + pres;
    S[0] = 0.0;
    S[1] = c->fcor * h * v;
    S[2] = -c->fcor * h * u;
    return 1;
}

/* Planar linear advection: F = bx u, G = by u, S = 0. */
static int flux_advection(const oracle_ctx *c, const double *q, double *F, double *G, double *S)
{
    F[0] = c->bx * q[0];
    G[0] = c->by * q[0];
    S[0] = 0.0;
    return 1;
}

static int physical_flux(const oracle_ctx *c, const double *q, double y, double *F, double *G, double *S)
{
    if (c->physics == PHYS_SPHERE_SWE) return flux_sphere(c, q, y, F, G, S);
    if (c->physics == PHYS_PLANE_SWE) return flux_plane_swe(c, q, F, G, S);
    return flux_advection(c, q, F, G, S);
}

/* Largest eigenvalue (in magnitude) of the flux Jacobian along the normal
 * (nx, ny) with respect to the conserved variable U:
 *   sphere, lambda direction: dF/dU has eigenvalues (u, u +- c)/(R cos theta)
 *   sphere, theta direction:  dG/dU has eigenvalues (v, v +- c)/R
 * with c = sqrt(g h); planar advection: |beta . n| (the exact upwind value)
 * or, as a global estimate of the largest wave speed, |beta|. */
static double max_eigenvalue(const oracle_ctx *c, const double *q, double y, int nx, int ny)
{
    if (c->physics == PHYS_SPHERE_SWE) {
        double h = q[0];
        double u = q[1] / h, v = q[2] / h, cs = sqrt(c->g * h);
        if (nx != 0) return (fabs(u) + cs) / (c->R * cos(y));
        return (fabs(v) + cs) / c->R;
    }
    if (c->physics == PHYS_PLANE_SWE) {   /* eigenvalues u, u +- c (x) and v, v +- c (y) */
        double h = q[0];
        double u = q[1] / h, v = q[2] / h, cs = sqrt(c->g * h);
        return nx != 0 ? fabs(u) + cs : fabs(v) + cs;
    }
    if (c->alpha_speed) return sqrt(c->bx * c->bx + c->by * c->by);
    return fabs(c->bx * nx + c->by * ny);
}

/* Rusanov flux along the outward normal n of the own element (Eq. rusanov):
 *   f* . n = (f(U_own) . n + f(U_nb) . n) / 2 - alpha/2 (U_nb - U_own)
 * with U = w(y) q the conserved variable and alpha the larger of the two
 * one-sided eigenvalue estimates.  Returns 0 if a state is non-physical. */
static int numerical_flux(const oracle_ctx *c, const double *qown, const double *qnb, double y,
                          int nx, int ny, const double *gspeed, double *fn)
{
    double Fo[3], Go[3], So[3], Fb[3], Gb[3], Sb[3];
    if (!physical_flux(c, qown, y, Fo, Go, So)) return 0;
    if (!physical_flux(c, qnb, y, Fb, Gb, Sb)) return 0;
    double alpha;
    if (gspeed) {
        /* global mode: |u| + c (lambda faces) or |v| + c (theta faces) replaced
         * by its maximum over the whole stage input, in the same eigenvalue */
        alpha = nx != 0 ? gspeed[0] / (c->R * cos(y)) : gspeed[1] / c->R;
    } else {
        double a1 = max_eigenvalue(c, qown, y, nx, ny);
        double a2 = max_eigenvalue(c, qnb, y, nx, ny);
        alpha = a1 > a2 ? a1 : a2;
    }
    double wy = metric_weight(c, y);
    for (int f = 0; f < c->nf; ++f) {
        double fo = Fo[f] * nx + Go[f] * ny;
        double fb = Fb[f] * nx + Gb[f] * ny;
        double Uo = wy * qown[f], Ub = wy * qnb[f];
        fn[f] = 0.5 * (fo + fb) - 0.5 * alpha * (Ub - Uo);
    }
    return 1;
}

/* --------------------------------------------------------------- operator -- */

static const double *elem_modes(const oracle_ctx *c, const double *u, int jy, int ix)
{
    return u + ((size_t)jy * c->nx + ix) * c->nf * c->nphi;
}

/* q_f = sum_m u_m phi_m(point) for every field (direct sum), with the basis
 * values phi_m(point) given as a row of one of the cached tables. */
static void eval_point(const oracle_ctx *c, const double *modes, const double *phi, double *q)
{
    for (int f = 0; f < c->nf; ++f) {
        double acc = 0.0;
        for (int m = 0; m < c->nphi; ++m) acc += modes[f * c->nphi + m] * phi[m];
        q[f] = acc;
    }
}

/* Tendency M^{-1} h(u) of element (jy, ix): the weak form of Eq. (dg_parts)
 *   int dU/dt phi + sum_edges int f*.n phi ds - int (F dphi/dx + G dphi/dy)
 *     = int S phi
 * assembled in (x, y) = (lambda, theta) coordinates and multiplied by the
 * inverse element mass matrix of Eq. (ode).  out: nf * nphi values. */
static int rhs_element_impl(const oracle_ctx *c, const double *u, int jy, int ix, double *out, int mag,
                            const double *gspeed);

/* Global wave speeds of a state for the global Rusanov mode: the maxima of
 * |u| + sqrt(g h) and |v| + sqrt(g h) over all elements and Gauss points. */
static int global_speeds(const oracle_ctx *c, const double *u, double *gs)
{
    double q[3];
    gs[0] = gs[1] = 0.0;
    for (int jy = 0; jy < c->ny; ++jy)
        for (int ix = 0; ix < c->nx; ++ix)
            for (int qi = 0; qi < c->n * c->n; ++qi) {
                eval_point(c, elem_modes(c, u, jy, ix), c->phiv + qi * c->nphi, q);
                if (!(q[0] > 0.0)) return ORACLE_ENONPHYSICAL;
                double cs = sqrt(c->g * q[0]);
                double su = fabs(q[1] / q[0]) + cs, sv = fabs(q[2] / q[0]) + cs;
                if (su > gs[0]) gs[0] = su;
                if (sv > gs[1]) gs[1] = sv;
            }
    return ORACLE_OK;
}

/* Well-balanced option on the sphere (href > 0; href <= 0 turns it off):
 * every tendency has the tendency of the fluid at rest at depth href removed,
 * so that state is exactly steady.  The rest state's tendency is the
 * quadrature residual of its constant pressure (hv modes only); it is the
 * same along a latitude row and is evaluated once per row. */
int oracle_set_well_balanced(oracle_ctx *c, double href)
{
    free(c->rest_res); free(c->rest_mag);
    c->rest_res = c->rest_mag = NULL;
    if (!(href > 0.0)) return ORACLE_OK;
    if (c->physics != PHYS_SPHERE_SWE) return ORACLE_EINVAL;
    const size_t per = (size_t)c->nf * c->nphi;
    double *rest = calloc((size_t)c->nx * c->ny * per, sizeof(double));
    double *res = malloc(sizeof(double) * c->ny * per), *mag = malloc(sizeof(double) * c->ny * per);
    if (!rest || !res || !mag) { free(rest); free(res); free(mag); return ORACLE_ENOMEM; }
    /* h = href: mode 0 of the orthonormal basis is 1/2 everywhere */
    for (size_t e = 0; e < (size_t)c->nx * c->ny; ++e) rest[e * per] = 2.0 * href;
    int st = ORACLE_OK;
    for (int jy = 0; jy < c->ny && st == ORACLE_OK; ++jy) {
        st = rhs_element_impl(c, rest, jy, 0, res + jy * per, 0, NULL);
        if (st == ORACLE_OK) st = rhs_element_impl(c, rest, jy, 0, mag + jy * per, 1, NULL);
    }
    free(rest);
    if (st) { free(res); free(mag); return st; }
    c->rest_res = res;
    c->rest_mag = mag;
    return ORACLE_OK;
}

/* Global Rusanov mode on the sphere: 1 -> every face uses the global speeds
 * of the stage input, 0 (default) -> the larger of the two one-sided ones. */
int oracle_set_alpha_mode(oracle_ctx *c, int mode)
{
    if (mode != 0 && mode != 1) return ORACLE_EINVAL;
    if (mode == 1 && c->physics != PHYS_SPHERE_SWE) return ORACLE_EINVAL;
    c->alpha_global = mode;
    return ORACLE_OK;
}

/* One element's tendency; in the global Rusanov mode the global speeds are
 * taken over the whole state u first (a full pass per call). */
/* Well-balanced option: remove from a tendency (mag = 0) the tendency of the
 * fluid at rest at the reference depth, or add its magnitude bound (mag = 1;
 * the two evaluations round independently). */
static void rest_correct(const oracle_ctx *c, int jy, double *out, int mag)
{
    if (!c->rest_res) return;
    const size_t per = (size_t)c->nf * c->nphi;
    for (size_t m = 0; m < per; ++m)
        out[m] += mag ? c->rest_mag[jy * per + m] : -c->rest_res[jy * per + m];
}

int oracle_rhs_element(const oracle_ctx *c, const double *u, int jy, int ix, double *out)
{
    double gs[2];
    if (c->alpha_global) {
        int st = global_speeds(c, u, gs);
        if (st) return st;
    }
    int st = rhs_element_impl(c, u, jy, ix, out, 0, c->alpha_global ? gs : NULL);
    if (!st) rest_correct(c, jy, out, 0);
    return st;
}

/* Magnitude bound of the tendency of element (jy, ix): the same assembly with
 * every term replaced by its absolute value and the inverse mass matrix by its
 * elementwise absolute value, |M^{-1}| sum |terms|.  Floating-point summation
 * of the tendency errs by at most a small multiple of the unit roundoff times
 * this bound, so it is the scale that tendency tolerances are taken against. */
int oracle_rhs_magnitude_element(const oracle_ctx *c, const double *u, int jy, int ix, double *out)
{
    double gs[2];
    if (c->alpha_global) {
        int st = global_speeds(c, u, gs);
        if (st) return st;
    }
    int st = rhs_element_impl(c, u, jy, ix, out, 1, c->alpha_global ? gs : NULL);
    if (!st) rest_correct(c, jy, out, 1);
    return st;
}

static int rhs_element_impl(const oracle_ctx *c, const double *u, int jy, int ix, double *out, int mag,
                            const double *gspeed)
{
    int n = c->n, np = c->nphi, nf = c->nf;
    double r[3 * 81];
    double q[3], F[3], G[3], S[3], qo[3], qb[3], fn[3];
    memset(r, 0, sizeof(double) * nf * np);
    const double *mo = elem_modes(c, u, jy, ix);
    double jac = 0.25 * c->dx * c->dy;

    /* volume and source integrals, n x n Gauss-Legendre points */
    for (int qy = 0; qy < n; ++qy)
        for (int qx = 0; qx < n; ++qx) {
            int qi = qy * n + qx;
            double y = elem_y(c, jy, c->xg[qy]);
            eval_point(c, mo, c->phiv + qi * np, q);
            if (!physical_flux(c, q, y, F, G, S)) return ORACLE_ENONPHYSICAL;
            double wq = c->wg[qx] * c->wg[qy] * jac;
            for (int m = 0; m < np; ++m) {
                double dpx = c->dphix[qi * np + m] * 2.0 / c->dx;
                double dpy = c->dphiy[qi * np + m] * 2.0 / c->dy;
                double ph = c->phiv[qi * np + m];
                for (int f = 0; f < nf; ++f) {
                    if (mag) r[f * np + m] += fabs(wq * F[f] * dpx) + fabs(wq * G[f] * dpy) + fabs(wq * S[f] * ph);
                    else r[f * np + m] += wq * (F[f] * dpx + G[f] * dpy + S[f] * ph);
                }
            }
        }

    /* edge integrals: west, east, south, north; n Gauss-Legendre points each */
    for (int e = 0; e < 4; ++e) {
        int nxv = (e == 0) ? -1 : (e == 1) ? 1 : 0;
        int nyv = (e == 2) ? -1 : (e == 3) ? 1 : 0;
        int inb = ix, jnb = jy;
        if (e == 0) inb = (ix - 1 + c->nx) % c->nx;
        if (e == 1) inb = (ix + 1) % c->nx;
        if (e == 2) jnb = jy - 1;
        if (e == 3) jnb = jy + 1;
        int pole = 0;
        if (jnb < 0 || jnb >= c->ny) {
            if (c->physics == PHYS_SPHERE_SWE) pole = 1;   /* zero flux through the pole edge */
            else jnb = (jnb + c->ny) % c->ny;              /* plane: periodic */
        }
        double ejac = (nxv != 0) ? 0.5 * c->dy : 0.5 * c->dx;
        int eopp = e ^ 1;   /* the neighbour sees this edge as its opposite edge */
        for (int k = 0; k < n; ++k) {
            double xio, etao;
            edge_point(c, e, k, &xio, &etao);
            const double *phio = c->phie + (e * n + k) * np;
            const double *phib = c->phie + (eopp * n + k) * np;
            double y = elem_y(c, jy, etao);
            if (pole) {
                for (int f = 0; f < nf; ++f) fn[f] = 0.0;
            } else {
                eval_point(c, mo, phio, qo);
                eval_point(c, elem_modes(c, u, jnb, inb), phib, qb);
                if (!numerical_flux(c, qo, qb, y, nxv, nyv, gspeed, fn)) return ORACLE_ENONPHYSICAL;
            }
            double we = c->wg[k] * ejac;
            for (int m = 0; m < np; ++m) {
                double ph = phio[m];
                for (int f = 0; f < nf; ++f) {
                    if (mag) r[f * np + m] += fabs(we * fn[f] * ph);
                    else r[f * np + m] -= we * fn[f] * ph;
                }
            }
        }
    }

    /* apply the inverse of the full element mass matrix of this row */
    const double *mi = c->minv + (size_t)jy * np * np;
    for (int f = 0; f < nf; ++f)
        for (int a = 0; a < np; ++a) {
            double acc = 0.0;
            for (int b = 0; b < np; ++b)
                acc += (mag ? fabs(mi[a * np + b]) : mi[a * np + b]) * r[f * np + b];
            out[f * np + a] = acc;
        }
    return ORACLE_OK;
}

static int rhs_all(const oracle_ctx *c, const double *u, double *tend, int mag)
{
    int status = ORACLE_OK;
    int nel = c->nx * c->ny;
    size_t per = (size_t)c->nf * c->nphi;
    double gs[2];
    const double *gsp = NULL;
    if (c->alpha_global) {
        status = global_speeds(c, u, gs);
        if (status) return status;
        gsp = gs;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(c->nthreads) reduction(max : status)
#endif
    for (int e = 0; e < nel; ++e) {
        int st = rhs_element_impl(c, u, e / c->nx, e % c->nx, tend + (size_t)e * per, mag, gsp);
        if (!st) rest_correct(c, e / c->nx, tend + (size_t)e * per, mag);
        if (st > status) status = st;
    }
    return status;
}

/* du/dt = M^{-1} h(u) for every element (Eq. ode). */
int oracle_rhs(const oracle_ctx *c, const double *u, double *tend)
{
    return rhs_all(c, u, tend, 0);
}

/* The magnitude bound of oracle_rhs_magnitude_element() for every element. */
int oracle_rhs_magnitude(const oracle_ctx *c, const double *u, double *tend)
{
    return rhs_all(c, u, tend, 1);
}

/* ---------------------------------------------------------------- time -- */

typedef int (*oracle_rhs_fn)(void *user, const double *u, double *k);

/* One step of the explicit Runge-Kutta method of order 1..4 given by the
 * Butcher tableaux of Table "Butcher":
 *   k_s = f(u + dt sum_{r<s} a_sr k_r),   u <- u + dt sum_s b_s k_s. */
int oracle_rk_step(int order, double dt, size_t len, double *u, oracle_rhs_fn f, void *user)
{
    static const double A1[1][1] = {{0}};
    static const double B1[1] = {1.0};
    static const double A2[2][2] = {{0, 0}, {1.0, 0}};
    static const double B2[2] = {0.5, 0.5};
    static const double A3[3][3] = {{0, 0, 0}, {1.0, 0, 0}, {0.25, 0.25, 0}};
    static const double B3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
    static const double A4[4][4] = {{0, 0, 0, 0}, {0.5, 0, 0, 0}, {0, 0.5, 0, 0}, {0, 0, 1.0, 0}};
    static const double B4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    if (order < 1 || order > 4) return ORACLE_EINVAL;
    int s = order;
    double *k = malloc(sizeof(double) * len * s);
    double *y = malloc(sizeof(double) * len);
    if (!k || !y) { free(k); free(y); return ORACLE_ENOMEM; }
    int status = ORACLE_OK;
    for (int st = 0; st < s && status == ORACLE_OK; ++st) {
        for (size_t i = 0; i < len; ++i) {
            double acc = u[i];
            for (int r = 0; r < st; ++r) {
                double a = order == 1 ? A1[st][r] : order == 2 ? A2[st][r] : order == 3 ? A3[st][r] : A4[st][r];
                if (a != 0.0) acc += dt * a * k[(size_t)r * len + i];
            }
            y[i] = acc;
        }
        status = f(user, y, k + (size_t)st * len);
    }
    if (status == ORACLE_OK) {
        for (size_t i = 0; i < len; ++i) {
            double acc = 0.0;
            for (int st = 0; st < s; ++st) {
                double b = order == 1 ? B1[st] : order == 2 ? B2[st] : order == 3 ? B3[st] : B4[st];
                acc += b * k[(size_t)st * len + i];
            }
            u[i] += dt * acc;
        }
    }
    free(k); free(y);
    return status;
}

static int rhs_adapter(void *user, const double *u, double *k)
{
    return oracle_rhs((const oracle_ctx *)user, u, k);
}

/* nsteps steps of RK order 1..4 in place. */
int oracle_step(const oracle_ctx *c, double *u, int nsteps, double dt, int order)
{
    size_t len = oracle_state_len(c);
    for (int s = 0; s < nsteps; ++s) {
        int st = oracle_rk_step(order, dt, len, u, rhs_adapter, (void *)c);
        if (st) return st;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------ diagnostics -- */

/* Neumaier compensated summation (Neumaier 1974). */
typedef struct { double s, comp; } nsum;
static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->comp += (a->s - t) + x;
    else a->comp += (x - t) + a->s;
    a->s = t;
}

/* Total mass R^2 sum_k int h cos(theta) dlambda dtheta (sphere; on the plane
 * int u dx dy), by nm x nm quadrature per element and a Neumaier sum. */
double oracle_total_mass(const oracle_ctx *c, const double *u)
{
    nsum acc = {0.0, 0.0};
    double jac = 0.25 * c->dx * c->dy;
    double q[3];
    for (int jy = 0; jy < c->ny; ++jy)
        for (int ix = 0; ix < c->nx; ++ix) {
            const double *mo = elem_modes(c, u, jy, ix);
            for (int qy = 0; qy < c->nm; ++qy)
                for (int qx = 0; qx < c->nm; ++qx) {
                    eval_point(c, mo, c->phim + (qy * c->nm + qx) * c->nphi, q);
                    double w = c->wm[qx] * c->wm[qy] * jac * metric_weight(c, elem_y(c, jy, c->xm[qy]));
                    nsum_add(&acc, w * q[0]);
                }
        }
    double s = acc.s + acc.comp;
    return c->physics == PHYS_SPHERE_SWE ? c->R * c->R * s : s;
}

/* Time step from the Courant number p c dt / H (Sec. 2):
 *   H = min over elements and the n x n nodes of min(R dtheta, R cos(theta) dlambda)
 *   c = max over the nodes of sqrt(u^2 + v^2) + sqrt(g h)
 *   dt = cfl H / (max(p, 1) c).   Sphere only.  Returns a negative value if
 *   the state is non-physical. */
double oracle_max_dt(const oracle_ctx *c, const double *u, double cfl)
{
    double hmin = INFINITY, cmax = 0.0, q[3];
    for (int jy = 0; jy < c->ny; ++jy)
        for (int ix = 0; ix < c->nx; ++ix) {
            const double *mo = elem_modes(c, u, jy, ix);
            for (int qy = 0; qy < c->n; ++qy)
                for (int qx = 0; qx < c->n; ++qx) {
                    double y = elem_y(c, jy, c->xg[qy]);
                    double hl = fmin(c->R * c->dy, c->R * cos(y) * c->dx);
                    if (hl < hmin) hmin = hl;
                    eval_point(c, mo, c->phiv + (qy * c->n + qx) * c->nphi, q);
                    if (!(q[0] > 0.0)) return -1.0;
                    double uu = q[1] / q[0], vv = q[2] / q[0];
                    double sp = sqrt(uu * uu + vv * vv) + sqrt(c->g * q[0]);
                    if (sp > cmax) cmax = sp;
                }
        }
    int pp = c->p > 1 ? c->p : 1;
    return cfl * hmin / (pp * cmax);
}

/* Coordinates of the nm x nm projection / norm points of every element,
 * layout [jy][ix][qy][qx]. */
void oracle_projection_points(const oracle_ctx *c, double *x, double *y)
{
    size_t t = 0;
    for (int jy = 0; jy < c->ny; ++jy)
        for (int ix = 0; ix < c->nx; ++ix)
            for (int qy = 0; qy < c->nm; ++qy)
                for (int qx = 0; qx < c->nm; ++qx, ++t) {
                    x[t] = elem_x(c, ix, c->xm[qx]);
                    y[t] = elem_y(c, jy, c->xm[qy]);
                }
}

/* Weighted L^2 projection onto the modal basis (mass matrix of Eq. ode):
 * u_hat = M^{-1} b, b_m = int f phi_m w(y).  vals layout [jy][ix][f][qy][qx]
 * at the projection points. */
void oracle_project(const oracle_ctx *c, const double *vals, double *modal)
{
    int np = c->nphi, nm = c->nm;
    double jac = 0.25 * c->dx * c->dy;
    double b[81];
    for (int jy = 0; jy < c->ny; ++jy) {
        const double *mi = c->minv + (size_t)jy * np * np;
        for (int ix = 0; ix < c->nx; ++ix)
            for (int f = 0; f < c->nf; ++f) {
                const double *v = vals + (((size_t)jy * c->nx + ix) * c->nf + f) * nm * nm;
                for (int m = 0; m < np; ++m) {
                    double acc = 0.0;
                    for (int qy = 0; qy < nm; ++qy)
                        for (int qx = 0; qx < nm; ++qx)
                            acc += c->wm[qx] * c->wm[qy] * jac * c->phim[(qy * nm + qx) * np + m] *
                                   metric_weight(c, elem_y(c, jy, c->xm[qy])) * v[qy * nm + qx];
                    b[m] = acc;
                }
                double *out = modal + (((size_t)jy * c->nx + ix) * c->nf + f) * np;
                for (int a = 0; a < np; ++a) {
                    double acc = 0.0;
                    for (int m = 0; m < np; ++m) acc += mi[a * np + m] * b[m];
                    out[a] = acc;
                }
            }
    }
}

/* Values of the modal expansion at the projection points, layout
 * [jy][ix][f][qy][qx]. */
void oracle_eval_projection_points(const oracle_ctx *c, const double *modal, double *vals)
{
    int nm = c->nm;
    double q[3];
    for (int jy = 0; jy < c->ny; ++jy)
        for (int ix = 0; ix < c->nx; ++ix) {
            const double *mo = elem_modes(c, modal, jy, ix);
            for (int qy = 0; qy < nm; ++qy)
                for (int qx = 0; qx < nm; ++qx) {
                    eval_point(c, mo, c->phim + (qy * nm + qx) * c->nphi, q);
                    for (int f = 0; f < c->nf; ++f)
                        vals[(((size_t)jy * c->nx + ix) * c->nf + f) * nm * nm + qy * nm + qx] = q[f];
                }
        }
}

/* Continuous L^2 norm of (u_h - exact) for field f with the weight w(y),
 * sqrt(sum_k int (u_h - exact)^2 w(y) dx dy); exact given at the projection
 * points, layout [jy][ix][f][qy][qx]. */
double oracle_l2_error(const oracle_ctx *c, const double *modal, const double *exact, int field)
{
    int nm = c->nm;
    double jac = 0.25 * c->dx * c->dy, q[3];
    nsum acc = {0.0, 0.0};
    for (int jy = 0; jy < c->ny; ++jy)
        for (int ix = 0; ix < c->nx; ++ix) {
            const double *mo = elem_modes(c, modal, jy, ix);
            const double *ex = exact + (((size_t)jy * c->nx + ix) * c->nf + field) * nm * nm;
            for (int qy = 0; qy < nm; ++qy)
                for (int qx = 0; qx < nm; ++qx) {
                    eval_point(c, mo, c->phim + (qy * nm + qx) * c->nphi, q);
                    double d = q[field] - ex[qy * nm + qx];
                    nsum_add(&acc, c->wm[qx] * c->wm[qy] * jac * metric_weight(c, elem_y(c, jy, c->xm[qy])) * d * d);
                }
        }
    return sqrt(acc.s + acc.comp);
}
