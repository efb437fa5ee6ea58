// dg_tables.cpp -- FP64 host precomputation of the constant tables
// (paper Sec. 3.2, "DG solver: precomputation": inverse mass matrices,
// Gauss-Legendre points and weights, basis values at the points).
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "dg_internal.h"

// Orthonormal Legendre polynomials L_k = sqrt((2k+1)/2) P_k by their own
// three-term recurrence
//   L_{k+1}(x) = a_k x L_k(x) - (a_k / a_{k-1}) L_{k-1}(x),
//   a_k = sqrt((2k+1)(2k+3)) / (k+1).
static void legendre_all(int kmax, double x, double *L, double *dL)
{
    L[0] = std::sqrt(0.5);
    dL[0] = 0.0;
    if (kmax == 0) return;
    double a_prev = 0.0;
    for (int k = 0; k < kmax; ++k) {
        double a = std::sqrt((2.0 * k + 1.0) * (2.0 * k + 3.0)) / (k + 1.0);
        double lm = k > 0 ? L[k - 1] : 0.0, dlm = k > 0 ? dL[k - 1] : 0.0;
        double r = k > 0 ? a / a_prev : 0.0;
        L[k + 1] = a * x * L[k] - r * lm;
        dL[k + 1] = a * (L[k] + x * dL[k]) - r * dlm;
        a_prev = a;
    }
}

double dg_legendre(int k, double x)
{
    double L[40], dL[40];
    legendre_all(k, x, L, dL);
    return L[k];
}

double dg_legendre_deriv(int k, double x)
{
    double L[40], dL[40];
    legendre_all(k, x, L, dL);
    return dL[k];
}

// Gauss-Legendre rule: Newton iteration on L_n from Tricomi's asymptotic
// initial guess; weights from the Christoffel function of the orthonormal
// family, w_i = 1 / sum_{k<n} L_k(x_i)^2.  Ascending order.
void dg_gauss_legendre(int n, double *x, double *w)
{
    double L[40], dL[40];
    for (int i = 1; i <= n; ++i) {
        double th = M_PI * (4.0 * i - 1.0) / (4.0 * n + 2.0);
        double r = std::cos(th) * (1.0 - (n - 1.0) / (8.0 * n * n * n));
        for (int it = 0; it < 50; ++it) {
            legendre_all(n, r, L, dL);
            double d = L[n] / dL[n];
            r -= d;
            if (std::fabs(d) < 1e-16) break;
        }
        legendre_all(n, r, L, dL);
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += L[k] * L[k];
        x[n - i] = r;       // i = 1 is the largest root
        w[n - i] = 1.0 / s;
    }
    for (int i = 0; i < n / 2; ++i) {   // exact symmetry of the rule
        double xs = 0.5 * (x[n - 1 - i] - x[i]);
        double ws = 0.5 * (w[n - 1 - i] + w[i]);
        x[i] = -xs; x[n - 1 - i] = xs;
        w[i] = ws; w[n - 1 - i] = ws;
    }
    if (n % 2) x[n / 2] = 0.0;
}

// Gauss-Jordan inversion with partial pivoting (k <= DG_MAXN).
static int invert(int k, const double *a, double *inv)
{
    double m[DG_MAXN][2 * DG_MAXN];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < 2 * k; ++j) m[i][j] = j < k ? a[i * k + j] : (j - k == i ? 1.0 : 0.0);
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int i = c + 1; i < k; ++i)
            if (std::fabs(m[i][c]) > std::fabs(m[piv][c])) piv = i;
        if (m[piv][c] == 0.0) return 1;
        if (piv != c)
            for (int j = 0; j < 2 * k; ++j) std::swap(m[c][j], m[piv][j]);
        double d = 1.0 / m[c][c];
        for (int j = 0; j < 2 * k; ++j) m[c][j] *= d;
        for (int i = 0; i < k; ++i) {
            if (i == c) continue;
            double f = m[i][c];
            if (f != 0.0)
                for (int j = 0; j < 2 * k; ++j) m[i][j] -= f * m[c][j];
        }
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) inv[i * k + j] = m[i][k + j];
    return 0;
}

void dg_free_tables(HostTables &t)
{
    std::free(t.rows);
    std::free(t.C);
    t.rows = nullptr;
    t.C = nullptr;
}

int dg_build_tables(HostTables &t, int nlon, int nlat, int p, double R, double g)
{
    (void)g;
    int n = p + 1;
    t.n = n;
    t.nm = p + 9;
    t.nlon = nlon;
    t.nlat = nlat;
    t.R = R;
    t.dlam = 2.0 * M_PI / nlon;
    t.dth = M_PI / nlat;
    dg_gauss_legendre(n, t.xg, t.wg);
    dg_gauss_legendre(t.nm, t.xm, t.wm);
    std::memset(&t.basis, 0, sizeof(t.basis));
    for (int a = 0; a < n; ++a) {
        t.basis.SE[a] = dg_legendre(a, 1.0);
        t.basis.SW[a] = dg_legendre(a, -1.0);
        for (int q = 0; q < n; ++q) {
            t.basis.LV[a][q] = dg_legendre(a, t.xg[q]);
            t.basis.WLV[a][q] = t.wg[q] * dg_legendre(a, t.xg[q]);
            t.basis.WLD[a][q] = t.wg[q] * dg_legendre_deriv(a, t.xg[q]);
        }
    }
    t.rows = static_cast<RowTab<double> *>(std::calloc(nlat, sizeof(RowTab<double>)));
    t.C = static_cast<double *>(std::calloc((size_t)nlat * n * n, sizeof(double)));
    if (!t.rows || !t.C) return 2;
    // C_j by a Gauss rule of n + 12 points: the integrand is entire and the
    // rule is exact to degree 2n + 23, far past double precision for dth <= pi/2.
    const int nc = n + 12;
    double xc[32], wc[32];
    dg_gauss_legendre(nc, xc, wc);
    const double cG = 2.0 / (R * t.dth);
    for (int j = 0; j < nlat; ++j) {
        RowTab<double> &r = t.rows[j];
        const double tb = -0.5 * M_PI + j * t.dth;
        double *C = t.C + (size_t)j * n * n;
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c) {
                double s = 0.0;
                for (int q = 0; q < nc; ++q)
                    s += wc[q] * dg_legendre(b, xc[q]) * dg_legendre(c, xc[q]) *
                         std::cos(tb + 0.5 * (1.0 + xc[q]) * t.dth);
                C[b * n + c] = s;
            }
        double Ci[DG_MAXN * DG_MAXN];
        if (invert(n, C, Ci)) return 1;
        for (int q = 0; q < n; ++q) {
            const double th = tb + 0.5 * (1.0 + t.xg[q]) * t.dth;
            r.cosn[q] = std::cos(th);
            r.sinn[q] = std::sin(th);
        }
        // the edge between rows j and j + 1 gets one value, whichever row
        // reads it: the two tiles (or bands) that meet there evaluate that
        // edge's flux from the same bits
        r.ce_s = (j == 0) ? 0.0 : std::cos(-0.5 * M_PI + j * t.dth);
        r.ce_n = (j == nlat - 1) ? 0.0 : std::cos(-0.5 * M_PI + (j + 1) * t.dth);
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c) r.Ci[b][c] = Ci[b * n + c];
        for (int b = 0; b < n; ++b)
            for (int q = 0; q < n; ++q) {
                double s = 0.0, sd = 0.0;
                for (int c = 0; c < n; ++c) {
                    s += Ci[b * n + c] * t.basis.WLV[c][q];
                    sd += Ci[b * n + c] * t.basis.WLD[c][q];
                }
                r.Q[b][q] = s;
                r.QT[q][b] = s;
                r.PT[q][b] = sd;
            }
        for (int b = 0; b < n; ++b) {
            double se = 0.0, sw = 0.0;
            for (int c = 0; c < n; ++c) {
                se += Ci[b * n + c] * t.basis.SE[c];
                sw += Ci[b * n + c] * t.basis.SW[c];
            }
            r.CSE[b] = se;
            r.CSW[b] = sw;
        }
        // Unit pressure flux, fluid at rest: G_hv = cG cos(theta) (scaled flux),
        // S_hv = -sin(theta)/R, edge fluxes cG ce; the column contraction gives
        // x2[b], the row contraction with w L_0 = sqrt(2) w, then Ci.
        double x2[DG_MAXN];
        for (int b = 0; b < n; ++b) {
            double s = 0.0;
            for (int q = 0; q < n; ++q)
                s += t.basis.WLD[b][q] * cG * r.cosn[q] - t.basis.WLV[b][q] * r.sinn[q] / R;
            s -= cG * (r.ce_n * t.basis.SE[b] - r.ce_s * t.basis.SW[b]);
            x2[b] = s;
        }
        for (int b = 0; b < n; ++b) {
            double s = 0.0;
            for (int c = 0; c < n; ++c) s += Ci[b * n + c] * x2[c];
            r.rho[b] = std::sqrt(2.0) * s;
        }
    }
    return 0;
}
