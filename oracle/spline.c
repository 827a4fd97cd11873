/*
 * spline.c -- oracle: B-spline basis, quadrature and 1D Galerkin matrices.
 * TEST INFRASTRUCTURE ONLY (see iga_oracle.h).
 *
 * Section 2.1 of the paper: open uniform knot vector, Cox-de Boor recursion
 * with 0/0 := 0, Dirichlet-restricted space S_h^p (dimension m+p-2).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "iga_oracle.h"

/* Section 2.1: xi_1 = ... = xi_{p+1} = 0, xi_{p+i+1} = i/m, xi_{p+m+1} = ... = 1.
 * 0-based: xi[k] is xi_{k+1}. */
void or_knots(int p, int m, double *xi)
{
    for (int k = 0; k < 2 * p + m + 1; ++k) {
        if (k <= p)
            xi[k] = 0.0;
        else if (k >= p + m)
            xi[k] = 1.0;
        else
            xi[k] = (double)(k - p) / (double)m;
    }
}

/* a / b with the paper's convention that a fraction with zero denominator
 * (the 0/0 case of eq. order_spline) contributes nothing. */
static double frac0(double a, double b) { return b == 0.0 ? 0.0 : a / b; }

/* Eqs. (constantspline) and (order_spline).  The degree-0 functions are the
 * indicator functions of the half-open knot spans; at x = 1 the half-open rule
 * leaves every span empty, so the last non-degenerate span [xi_{p+m}, xi_{p+m+1})
 * is taken as closed on the right (N_{m+p}(1) = 1).
 * The derivative uses de Boor's identity
 *   dN_i^p = p/(xi_{i+p}-xi_i) N_i^{p-1} - p/(xi_{i+p+1}-xi_{i+1}) N_{i+1}^{p-1}. */
void or_basis_eval(int p, int m, double x, double *N, double *dN)
{
    const int nk = 2 * p + m + 1;
    double *xi = malloc(sizeof(double) * nk);
    double *B = malloc(sizeof(double) * nk);
    double *Bn = malloc(sizeof(double) * nk);
    or_knots(p, m, xi);

    const int n0 = nk - 1; /* degree-0 functions: m + 2p */
    for (int i = 0; i < n0; ++i)
        B[i] = (xi[i] <= x && x < xi[i + 1]) ? 1.0 : 0.0;
    if (x >= 1.0) {
        for (int i = 0; i < n0; ++i) B[i] = 0.0;
        B[p + m - 1] = 1.0;
    }

    /* raise the degree from 0 to p; at degree k there are n0 - k functions */
    for (int k = 1; k <= p; ++k) {
        if (k == p && dN) {
            for (int i = 0; i < n0 - k; ++i)
                dN[i] = frac0((double)k, xi[i + k] - xi[i]) * B[i]
                      - frac0((double)k, xi[i + k + 1] - xi[i + 1]) * B[i + 1];
        }
        for (int i = 0; i < n0 - k; ++i)
            Bn[i] = frac0(x - xi[i], xi[i + k] - xi[i]) * B[i]
                  + frac0(xi[i + k + 1] - x, xi[i + k + 1] - xi[i + 1]) * B[i + 1];
        memcpy(B, Bn, sizeof(double) * (n0 - k));
    }
    if (p == 0 && dN)
        for (int i = 0; i < n0; ++i) dN[i] = 0.0;
    for (int i = 0; i < m + p; ++i) N[i] = B[i];
    free(xi);
    free(B);
    free(Bn);
}

/* Gauss-Legendre nodes and weights on [-1,1] by Newton's method on the Legendre
 * polynomial P_n, evaluated with the three-term recurrence. */
void or_gauss(int npts, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < npts; ++i) {
        double z = cos(pi * (i + 0.75) / (npts + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= npts; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            /* P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1) */
            dp = npts * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Gauss points of element e of the uniform mesh with m elements, mapped from [-1,1]. */
static void element_points(int m, int e, int nq, const double *gx, const double *gw,
                           double *xq, double *wq)
{
    const double h = 1.0 / m, a = e * h;
    for (int q = 0; q < nq; ++q) {
        xq[q] = a + 0.5 * h * (gx[q] + 1.0);
        wq[q] = 0.5 * h * gw[q];
    }
}

/* Stiffness and mass of the 1D spline space.  The integrands N_i' N_j' and
 * N_i N_j have degree <= 2p on each element, so p+1 Gauss points are exact. */
void or_assemble_1d(int p, int m, int full, double *K, double *M)
{
    const int nf = m + p;
    const int nq = p + 1;
    double *gx = malloc(sizeof(double) * nq), *gw = malloc(sizeof(double) * nq);
    double *xq = malloc(sizeof(double) * nq), *wq = malloc(sizeof(double) * nq);
    double *N = malloc(sizeof(double) * nf), *dN = malloc(sizeof(double) * nf);
    double *Kf = calloc((size_t)nf * nf, sizeof(double));
    double *Mf = calloc((size_t)nf * nf, sizeof(double));
    int *nz = malloc(sizeof(int) * nf);
    or_gauss(nq, gx, gw);

    for (int e = 0; e < m; ++e) {
        element_points(m, e, nq, gx, gw, xq, wq);
        for (int q = 0; q < nq; ++q) {
            or_basis_eval(p, m, xq[q], N, dN);
            /* only the functions that do not vanish at the point contribute */
            int nnz = 0;
            for (int i = 0; i < nf; ++i)
                if (N[i] != 0.0 || dN[i] != 0.0) nz[nnz++] = i;
            for (int a = 0; a < nnz; ++a)
                for (int c = 0; c < nnz; ++c) {
                    const int i = nz[a], j = nz[c];
                    Kf[(size_t)i * nf + j] += wq[q] * dN[i] * dN[j];
                    Mf[(size_t)i * nf + j] += wq[q] * N[i] * N[j];
                }
        }
    }
    if (full) {
        memcpy(K, Kf, sizeof(double) * nf * nf);
        memcpy(M, Mf, sizeof(double) * nf * nf);
    } else {
        /* eq. (splinespace): drop N_1 and N_{m+p} (homogeneous Dirichlet) */
        const int n = nf - 2;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                K[(size_t)i * n + j] = Kf[(size_t)(i + 1) * nf + (j + 1)];
                M[(size_t)i * n + j] = Mf[(size_t)(i + 1) * nf + (j + 1)];
            }
    }
    free(gx); free(gw); free(xq); free(wq); free(N); free(dN); free(Kf); free(Mf); free(nz);
}

/* Section 3.1.2, (M_p^{plow})_{ij} = int phi_i^{plow} phi_j^p.  The product has
 * degree p + plow <= 2p + 1, so p+1 Gauss points are exact. */
void or_mixed_mass_1d(int p, int plow, int m, double *Mx)
{
    const int nfp = m + p, nfl = m + plow;
    const int np = nfp - 2, nl = nfl - 2;
    const int nq = (p > plow ? p : plow) + 1;
    double *gx = malloc(sizeof(double) * nq), *gw = malloc(sizeof(double) * nq);
    double *xq = malloc(sizeof(double) * nq), *wq = malloc(sizeof(double) * nq);
    double *Np = malloc(sizeof(double) * nfp), *Nl = malloc(sizeof(double) * nfl);
    double *dtmp = malloc(sizeof(double) * (nfp > nfl ? nfp : nfl));
    or_gauss(nq, gx, gw);
    memset(Mx, 0, sizeof(double) * (size_t)nl * np);

    for (int e = 0; e < m; ++e) {
        element_points(m, e, nq, gx, gw, xq, wq);
        for (int q = 0; q < nq; ++q) {
            or_basis_eval(p, m, xq[q], Np, dtmp);
            or_basis_eval(plow, m, xq[q], Nl, dtmp);
            for (int i = 0; i < nl; ++i) {
                if (Nl[i + 1] == 0.0) continue; /* vanishing terms contribute nothing */
                for (int j = 0; j < np; ++j)
                    Mx[(size_t)i * np + j] += wq[q] * Nl[i + 1] * Np[j + 1];
            }
        }
    }
    free(gx); free(gw); free(xq); free(wq); free(Np); free(Nl); free(dtmp);
}

static double load_fn(int kind, const double *par, double x)
{
    const double pi = 3.14159265358979323846;
    if (kind == 0) return sin(pi * x);
    double t = (x - par[0]) / par[1];
    return exp(-0.5 * t * t);
}

/* Right-hand side b_p = (f, phi_i) (Section 2) for one factor of a separable f. */
void or_load_1d(int p, int m, int kind, const double *par, int nq, double *g)
{
    const int nf = m + p, n = nf - 2;
    double *gx = malloc(sizeof(double) * nq), *gw = malloc(sizeof(double) * nq);
    double *xq = malloc(sizeof(double) * nq), *wq = malloc(sizeof(double) * nq);
    double *N = malloc(sizeof(double) * nf), *dN = malloc(sizeof(double) * nf);
    or_gauss(nq, gx, gw);
    memset(g, 0, sizeof(double) * n);
    for (int e = 0; e < m; ++e) {
        element_points(m, e, nq, gx, gw, xq, wq);
        for (int q = 0; q < nq; ++q) {
            or_basis_eval(p, m, xq[q], N, dN);
            double fx = load_fn(kind, par, xq[q]);
            for (int i = 0; i < n; ++i) g[i] += wq[q] * fx * N[i + 1];
        }
    }
    free(gx); free(gw); free(xq); free(wq); free(N); free(dN);
}

/* Degree-1 functions are nodal: a coarse function's coefficients in the fine
 * hat basis are its values at the fine interior nodes. */
void or_embed_p1(int mc, double *S)
{
    const int mf = 2 * mc, nf = mf - 1, nc = mc - 1;
    double *N = malloc(sizeof(double) * (mc + 1)), *dN = malloc(sizeof(double) * (mc + 1));
    for (int i = 0; i < nf; ++i) {
        double x = (double)(i + 1) / mf;
        or_basis_eval(1, mc, x, N, dN);
        for (int I = 0; I < nc; ++I) S[(size_t)i * nc + I] = N[I + 1];
    }
    free(N);
    free(dN);
}

/* Embedding of the restricted degree-plow space on mc elements into the one on 2 mc
 * elements (Section 4.1: the standard transfer between spline spaces of equal degree):
 * the coarse space is a subspace of the fine one, so the coefficients are its L2
 * projection, S = (M_f)^{-1} (phi_f, phi_c), exact up to rounding.  Each fine element lies
 * inside one coarse element, where both bases are polynomials of degree plow, so plow + 1
 * Gauss points are exact.  (2 mc + plow - 2) x (mc + plow - 2). */
void or_embed_spline(int plow, int mc, double *S)
{
    const int mf = 2 * mc, nf = mf + plow - 2, nc = mc + plow - 2;
    const int nq = plow + 1;
    double *Kf = malloc(sizeof(double) * (size_t)nf * nf), *Mf = malloc(sizeof(double) * (size_t)nf * nf);
    double *B = calloc((size_t)nf * nc, sizeof(double));
    double *gx = malloc(sizeof(double) * nq), *gw = malloc(sizeof(double) * nq);
    double *xq = malloc(sizeof(double) * nq), *wq = malloc(sizeof(double) * nq);
    double *Nf = malloc(sizeof(double) * (mf + plow)), *Nc = malloc(sizeof(double) * (mc + plow));
    double *dtmp = malloc(sizeof(double) * (mf + plow));
    or_assemble_1d(plow, mf, 0, Kf, Mf);
    or_gauss(nq, gx, gw);
    for (int e = 0; e < mf; ++e) {
        element_points(mf, e, nq, gx, gw, xq, wq);
        for (int q = 0; q < nq; ++q) {
            or_basis_eval(plow, mf, xq[q], Nf, dtmp);
            or_basis_eval(plow, mc, xq[q], Nc, dtmp);
            for (int i = 0; i < nf; ++i) {
                if (Nf[i + 1] == 0.0) continue;
                for (int I = 0; I < nc; ++I) B[(size_t)i * nc + I] += wq[q] * Nf[i + 1] * Nc[I + 1];
            }
        }
    }
    /* S = M_f^{-1} B, column by column (dense Cholesky: test-size problems only) */
    or_cholesky(nf, Mf);
    double *col = malloc(sizeof(double) * nf), *x = malloc(sizeof(double) * nf);
    for (int I = 0; I < nc; ++I) {
        for (int i = 0; i < nf; ++i) col[i] = B[(size_t)i * nc + I];
        or_cholesky_solve(nf, Mf, col, x);
        for (int i = 0; i < nf; ++i) S[(size_t)i * nc + I] = x[i];
    }
    free(Kf); free(Mf); free(B); free(gx); free(gw); free(xq); free(wq); free(Nf); free(Nc); free(dtmp);
    free(col); free(x);
}

/* Section 3.1.2: I_p^{plow} = (M_plow^plow)^{-1} M_p^{plow} with the inverse replaced by
 * the inverse of the row-sum lumped mass; Section 3.3 composes it with the
 * h -> 2h restriction S^T of the degree-plow spaces (the degree-1 embedding is the nodal
 * one, or_embed_p1; degree 2 uses or_embed_spline).  (mr + plow - 2) x n rows, mr = m or m/2. */
void or_restriction_plow(int p, int plow, int m, int aggressive, double *R)
{
    const int n = m + p - 2, n1 = m + plow - 2;
    double *Mx = malloc(sizeof(double) * (size_t)n1 * n);
    double *K1 = malloc(sizeof(double) * (size_t)n1 * n1);
    double *M1 = malloc(sizeof(double) * (size_t)n1 * n1);
    or_mixed_mass_1d(p, plow, m, Mx);
    or_assemble_1d(plow, m, 0, K1, M1);
    /* Rp = D^{-1} M_p^plow with D_ii = sum_j (M_plow^plow)_ij */
    for (int i = 0; i < n1; ++i) {
        double D = 0.0;
        for (int j = 0; j < n1; ++j) D += M1[(size_t)i * n1 + j];
        for (int j = 0; j < n; ++j) Mx[(size_t)i * n + j] /= D;
    }
    if (!aggressive) {
        memcpy(R, Mx, sizeof(double) * (size_t)n1 * n);
    } else {
        const int mc = m / 2, nc = mc + plow - 2;
        double *S = malloc(sizeof(double) * (size_t)n1 * nc);
        if (plow == 1) or_embed_p1(mc, S);
        else or_embed_spline(plow, mc, S);
        for (int I = 0; I < nc; ++I)
            for (int j = 0; j < n; ++j) {
                double acc = 0.0;
                for (int i = 0; i < n1; ++i)
                    if (S[(size_t)i * nc + I] != 0.0) acc += S[(size_t)i * nc + I] * Mx[(size_t)i * n + j];
                R[(size_t)I * n + j] = acc;
            }
        free(S);
    }
    free(Mx);
    free(K1);
    free(M1);
}

void or_restriction_1d(int p, int m, int aggressive, double *R)
{
    or_restriction_plow(p, 1, m, aggressive, R);
}
