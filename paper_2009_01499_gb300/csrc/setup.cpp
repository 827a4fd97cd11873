// setup.cpp -- host-side construction of the solver's tables (run once per handle).
//
// Section 2.1: degree-p, C^{p-1} B-splines on the open uniform knot vector with
// m elements; homogeneous Dirichlet conditions drop the first and last function.
// The basis is evaluated span by span with the triangular form of the Cox-de Boor
// recursion (only the p+1 functions that are nonzero on a span), integrated with
// Gauss-Legendre rules, and stored as band rows.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace iga2l {

namespace {

std::vector<double> open_knots(int p, int m)
{
    std::vector<double> U(2 * p + m + 1);
    for (int k = 0; k < (int)U.size(); ++k) {
        int t = std::min(std::max(k - p, 0), m);   // clamp into 0..m
        U[k] = (double)t / (double)m;
    }
    return U;
}

// Values of the deg+1 B-splines of degree `deg` that are nonzero on the knot span
// [U[k], U[k+1]): out[j] = N_{k-deg+j}^{deg}(x), j = 0..deg.
void span_basis(int deg, const std::vector<double> &U, int k, double x, double *out)
{
    double left[kMaxP + 2], right[kMaxP + 2];
    out[0] = 1.0;
    for (int j = 1; j <= deg; ++j) {
        left[j] = x - U[k + 1 - j];
        right[j] = U[k + j] - x;
        double carry = 0.0;
        for (int t = 0; t < j; ++t) {
            const double w = out[t] / (right[t + 1] + left[j - t]);
            out[t] = carry + right[t + 1] * w;
            carry = left[j - t] * w;
        }
        out[j] = carry;
    }
}

// Values and first derivatives of the p+1 degree-p functions nonzero on span k.
// dN_i^p = p N_i^{p-1}/(U[i+p]-U[i]) - p N_{i+1}^{p-1}/(U[i+p+1]-U[i+1]).
void span_basis_d(int p, const std::vector<double> &U, int k, double x, double *N, double *dN)
{
    span_basis(p, U, k, x, N);
    double low[kMaxP + 2] = {0};
    // low[j] = N_{k-p+j}^{p-1}, j = 0..p; the degree p-1 functions on the span are
    // N_{k-p+1}..N_k, so low[0] = 0.
    double tmp[kMaxP + 2];
    span_basis(p - 1, U, k, x, tmp);
    low[0] = 0.0;
    for (int j = 1; j <= p; ++j) low[j] = tmp[j - 1];
    low[p + 1] = 0.0;
    for (int j = 0; j <= p; ++j) {
        const int i = k - p + j;
        const double d1 = U[i + p] - U[i], d2 = U[i + p + 1] - U[i + 1];
        double v = 0.0;
        if (d1 > 0.0) v += p * low[j] / d1;
        if (d2 > 0.0) v -= p * low[j + 1] / d2;
        dN[j] = v;
    }
}

// Gauss-Legendre points and weights on [0, 1].
void gauss01(int npt, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(npt, 0.0);
    w.assign(npt, 0.0);
    const double pi = 3.141592653589793238462643383279502884;
    for (int i = 0; i < npt; ++i) {
        double t = std::cos(pi * (4.0 * i + 3.0) / (4.0 * npt + 2.0));   // root estimate
        double dP = 1.0;
        for (int it = 0; it < 60; ++it) {
            double Pm1 = 1.0, P = t;
            for (int k = 1; k < npt; ++k) {
                const double Pn = ((2 * k + 1) * t * P - k * Pm1) / (k + 1);
                Pm1 = P;
                P = Pn;
            }
            dP = npt * (Pm1 - t * P) / (1.0 - t * t);
            const double step = P / dP;
            t -= step;
            if (std::fabs(step) <= 4e-17) break;
        }
        x[i] = 0.5 * (1.0 - t);
        w[i] = 1.0 / ((1.0 - t * t) * dP * dP);
    }
}

}  // namespace

int default_block_side(int p)
{
    // Section 4.3: 9-point (3x3) blocks for p = 2,3,4; 25-point for p = 5,6; 49-point for 7,8
    if (p >= 2 && p <= 4) return 3;
    if (p >= 5 && p <= 6) return 5;
    if (p >= 7 && p <= 8) return 7;
    return 0;
}

void default_colouring(int p, int s, int &q, int &g)
{
    // colour period q >= s+p and stride g with gcd(g, q) = 1 (this library's
    // choice; measured to give the smallest two-level factors on 64^2 meshes)
    switch (p) {
    case 2: q = 5; g = 2; break;
    case 3: q = 7; g = 2; break;
    case 4: q = 7; g = 2; break;
    case 5: q = 10; g = 3; break;
    case 6: q = 11; g = 4; break;
    case 7: q = 14; g = 5; break;
    case 8: q = 17; g = 4; break;
    default: q = s + p; g = 1; break;
    }
}

// Stiffness and mass band rows of the restricted degree-p space: row i (DOF i,
// the paper's N_{i+2}), entry a couples DOF i + a - p.  Product integrands have
// degree <= 2p per element, integrated exactly with p+1 Gauss points.
void bspline_band_1d(int p, int m, std::vector<double> &K, std::vector<double> &M)
{
    const int n = m + p - 2, W = 2 * p + 1;
    K.assign((size_t)n * W, 0.0);
    M.assign((size_t)n * W, 0.0);
    const std::vector<double> U = open_knots(p, m);
    std::vector<double> gx, gw;
    gauss01(p + 1, gx, gw);
    const double h = 1.0 / m;
    double N[kMaxP + 2], dN[kMaxP + 2];
    for (int e = 0; e < m; ++e) {
        const int k = p + e;   // span [e h, (e+1) h)
        for (size_t q = 0; q < gx.size(); ++q) {
            const double x = (e + gx[q]) * h, wq = gw[q] * h;
            span_basis_d(p, U, k, x, N, dN);
            for (int a = 0; a <= p; ++a) {
                const int i = e + a - 1;   // restricted index of full function e+a
                if (i < 0 || i >= n) continue;
                for (int b = 0; b <= p; ++b) {
                    const int j = e + b - 1;
                    if (j < 0 || j >= n) continue;
                    K[(size_t)i * W + (j - i + p)] += wq * dN[a] * dN[b];
                    M[(size_t)i * W + (j - i + p)] += wq * N[a] * N[b];
                }
            }
        }
    }
}

bool cholesky_inverse(int N, std::vector<double> &A)
{
    // A = L L^T, then A^{-1} column by column from L y = e_c, L^T x = y
    std::vector<double> L(A);
    for (int j = 0; j < N; ++j) {
        double d = L[(size_t)j * N + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * N + k] * L[(size_t)j * N + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        L[(size_t)j * N + j] = d;
        for (int i = j + 1; i < N; ++i) {
            double v = L[(size_t)i * N + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * N + k] * L[(size_t)j * N + k];
            L[(size_t)i * N + j] = v / d;
        }
    }
    std::vector<double> y(N), x(N);
    for (int c = 0; c < N; ++c) {
        for (int i = 0; i < N; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * N + k] * y[k];
            y[i] = v / L[(size_t)i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double v = y[i];
            for (int k = i + 1; k < N; ++k) v -= L[(size_t)k * N + i] * x[k];
            x[i] = v / L[(size_t)i * N + i];
        }
        for (int i = 0; i < N; ++i) A[(size_t)i * N + c] = x[i];
    }
    return true;
}

// Gauss points, weights and the p+1 nonzero basis values of every element, nq points
// per element: x[e*nq+q], w[e*nq+q], B[(e*nq+q)*(p+1)+a] = N_{e+a}(x) (full index).
void quadrature_tables(int p, int m, int nq, std::vector<double> &x, std::vector<double> &w,
                       std::vector<double> &B)
{
    const std::vector<double> U = open_knots(p, m);
    std::vector<double> gx, gw;
    gauss01(nq, gx, gw);
    const double h = 1.0 / m;
    x.assign((size_t)m * nq, 0.0);
    w.assign((size_t)m * nq, 0.0);
    B.assign((size_t)m * nq * (p + 1), 0.0);
    double N[kMaxP + 2];
    for (int e = 0; e < m; ++e)
        for (int q = 0; q < nq; ++q) {
            const size_t k = (size_t)e * nq + q;
            x[k] = (e + gx[q]) * h;
            w[k] = gw[q] * h;
            span_basis(p, U, p + e, x[k], N);
            for (int a = 0; a <= p; ++a) B[k * (p + 1) + a] = N[a];
        }
}

int build_host_tables(int p, int m, int s, HostTables &ht, std::string &err)
{
    ht.p = p;
    ht.m = m;
    ht.n = m + p - 2;
    ht.s = s;
    ht.r = (s - 1) / 2;
    const int n = ht.n, W = 2 * p + 1;
    bspline_band_1d(p, m, ht.Kb, ht.Mb);

    // residual point classes: rows within 2p-1 of a boundary see non-uniform
    // functions; rows 2p-1 .. n-2p are Toeplitz and share the middle row.  Row x < 2p-1
    // has class x, row x > n-2p (and >= 2p-1) class x-n+4p-1, so on grids with fewer than
    // 4p-1 rows every row keeps its own class and representative (itself), and the classes
    // no row uses still have a row of the grid as representative when n >= 2p-1
    ht.npc = 4 * p - 1;
    if (n < 2 * p - 1) {
        err = "mesh too small for the residual stencil classes";
        return IGA2L_ERR_INVALID_ARG;
    }
    ht.pc_rep.resize(ht.npc);
    for (int c = 0; c < ht.npc; ++c) {
        if (c < 2 * p - 1) ht.pc_rep[c] = c;
        else if (c == 2 * p - 1) ht.pc_rep[c] = n / 2;
        else ht.pc_rep[c] = c + n - (4 * p - 1);
    }
    // block classes: a block is interior if all its DOFs are uniform functions,
    // i.e. its centre lies in [L, n-1-L] with L = p-1+r.  Centre x < L has class x, centre
    // x > n-1-L (and >= L) class 2L-(n-1-x): with fewer than 2L+1 centres no block is
    // interior, every block keeps its own class and representative, and the unused middle
    // class is built from the (boundary) block at n/2
    ht.L = p - 1 + ht.r;
    ht.nbc = 2 * ht.L + 1;
    if (n < ht.L) {
        err = "mesh too small for the Schwarz block classes";
        return IGA2L_ERR_INVALID_ARG;
    }
    ht.bc_rep.resize(ht.nbc);
    for (int c = 0; c < ht.nbc; ++c) {
        if (c < ht.L) ht.bc_rep[c] = c;
        else if (c == ht.L) ht.bc_rep[c] = n / 2;
        else ht.bc_rep[c] = n - 1 - (2 * ht.L - c);
    }

    // ---- restriction (Sections 3.1.2, 3.3) ---------------------------------
    // mixed mass (M_p^1)_{ij} = int phi_i^1 phi_j^p on the h mesh, (m-1) x n
    const int n1 = m - 1;
    std::vector<double> Mx((size_t)n1 * n, 0.0);
    {
        const std::vector<double> Up = open_knots(p, m), U1 = open_knots(1, m);
        std::vector<double> gx, gw;
        gauss01(p + 1, gx, gw);
        const double h = 1.0 / m;
        double Np[kMaxP + 2], N1[4];
        for (int e = 0; e < m; ++e)
            for (size_t q = 0; q < gx.size(); ++q) {
                const double x = (e + gx[q]) * h, wq = gw[q] * h;
                span_basis(p, Up, p + e, x, Np);
                span_basis(1, U1, 1 + e, x, N1);
                for (int a = 0; a <= 1; ++a) {
                    const int i = e + a - 1;
                    if (i < 0 || i >= n1) continue;
                    for (int b = 0; b <= p; ++b) {
                        const int j = e + b - 1;
                        if (j < 0 || j >= n) continue;
                        Mx[(size_t)i * n + j] += wq * N1[a] * Np[b];
                    }
                }
            }
    }
    // row-sum lumped degree-1 mass: D_i = sum_j (M_1^1)_{ij}
    std::vector<double> K1, M1;
    bspline_band_1d(1, m, K1, M1);
    for (int i = 0; i < n1; ++i) {
        const double D = M1[(size_t)i * 3 + 0] + M1[(size_t)i * 3 + 1] + M1[(size_t)i * 3 + 2];
        for (int j = 0; j < n; ++j) Mx[(size_t)i * n + j] /= D;
    }
    // degree-1 restriction h -> 2h: coarse hat I is fine hats 2I, 2I+1, 2I+2 with
    // weights 1/2, 1, 1/2 (exact embedding of nested degree-1 spaces)
    const int nc = m / 2 - 1;
    ht.nc = nc;
    std::vector<double> R((size_t)nc * n, 0.0);
    for (int I = 0; I < nc; ++I)
        for (int j = 0; j < n; ++j)
            R[(size_t)I * n + j] = 0.5 * Mx[(size_t)(2 * I) * n + j] + Mx[(size_t)(2 * I + 1) * n + j]
                                 + 0.5 * Mx[(size_t)(2 * I + 2) * n + j];
    // row band and column band
    ht.Rlo.assign(nc, 0);
    ht.Clo.assign(n, 0);
    std::vector<int> Rhi(nc, -1), Chi(n, -1);
    for (int I = 0; I < nc; ++I) {
        int lo = n, hi = -1;
        for (int j = 0; j < n; ++j)
            if (R[(size_t)I * n + j] != 0.0) { lo = std::min(lo, j); hi = std::max(hi, j); }
        ht.Rlo[I] = lo;
        Rhi[I] = hi;
        ht.wr = std::max(ht.wr, hi - lo + 1);
    }
    for (int j = 0; j < n; ++j) {
        int lo = nc, hi = -1;
        for (int I = 0; I < nc; ++I)
            if (R[(size_t)I * n + j] != 0.0) { lo = std::min(lo, I); hi = std::max(hi, I); }
        if (hi < lo) { lo = 0; hi = -1; }
        ht.Clo[j] = lo;
        Chi[j] = hi;
        ht.wc = std::max(ht.wc, hi - lo + 1);
    }
    ht.Rb.assign((size_t)nc * ht.wr, 0.0);
    ht.Cb.assign((size_t)n * ht.wc, 0.0);
    for (int I = 0; I < nc; ++I)
        for (int t = 0; t < ht.wr; ++t) {
            const int j = ht.Rlo[I] + t;
            if (j < n) ht.Rb[(size_t)I * ht.wr + t] = R[(size_t)I * n + j];
        }
    for (int j = 0; j < n; ++j)
        for (int t = 0; t < ht.wc; ++t) {
            const int I = ht.Clo[j] + t;
            if (I < nc) ht.Cb[(size_t)j * ht.wc + t] = R[(size_t)I * n + j];
        }
    (void)W;
    return IGA2L_OK;
}

}  // namespace iga2l
