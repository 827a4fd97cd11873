/*
 * operators.c -- oracle: the operator A_p, the multiplicative Schwarz step,
 * transfers, the degree-1 V(1,1) cycle, the two-level cycle and the solver.
 * TEST INFRASTRUCTURE ONLY (see iga_oracle.h).
 *
 * Each function follows the definition in the paper without blocking or
 * fusion; terms that are identically zero (outside a band) are skipped.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "iga_oracle.h"

#define OR_MAXLEV 32

static long long ipow(int b, int e)
{
    long long r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}
static int imax(int a, int b) { return a > b ? a : b; }
static int imin(int a, int b) { return a < b ? a : b; }

/* Section 4.3 / Section 5.1: 3x3 blocks for p = 2,3,4, 5x5 for p = 5,6, 7x7 for p = 7,8. */
int or_block_size(int p)
{
    if (p >= 2 && p <= 4) return 3;
    if (p == 5 || p == 6) return 5;
    if (p == 7 || p == 8) return 7;
    return -1;
}

/* Entry A[x][y] of the tensor-product stiffness, x, y given by coordinates. */
static double a_entry(int dim, int n, const double *K, const double *M, const int *x, const int *y)
{
    const double kx = K[(size_t)x[0] * n + y[0]], mx = M[(size_t)x[0] * n + y[0]];
    const double ky = K[(size_t)x[1] * n + y[1]], my = M[(size_t)x[1] * n + y[1]];
    if (dim == 2) return kx * my + mx * ky;
    const double kz = K[(size_t)x[2] * n + y[2]], mz = M[(size_t)x[2] * n + y[2]];
    return kx * my * mz + mx * ky * mz + mx * my * kz;
}

static void coords(int dim, int n, long long idx, int *c)
{
    c[0] = (int)(idx % n);
    c[1] = (int)((idx / n) % n);
    c[2] = dim == 3 ? (int)(idx / ((long long)n * n)) : 0;
}

/* (A u) at one point x: the row of A, restricted to the band |x_k - y_k| <= w. */
static double a_row_apply(int dim, int n, int w, const double *K, const double *M,
                          const int *x, const double *u)
{
    double acc = 0.0;
    int y[3] = {0, 0, 0};
    const int z0 = dim == 3 ? imax(0, x[2] - w) : 0, z1 = dim == 3 ? imin(n - 1, x[2] + w) : 0;
    for (y[2] = z0; y[2] <= z1; ++y[2])
        for (y[1] = imax(0, x[1] - w); y[1] <= imin(n - 1, x[1] + w); ++y[1])
            for (y[0] = imax(0, x[0] - w); y[0] <= imin(n - 1, x[0] + w); ++y[0]) {
                const long long iy = y[0] + (long long)n * (y[1] + (long long)n * y[2]);
                acc += a_entry(dim, n, K, M, x, y) * u[iy];
            }
    return acc;
}

/* A_p = K (x) M + M (x) K (2D); the 3D analogue has three terms. */
void or_apply_A(int dim, int n, int w, const double *K, const double *M,
                const double *u, double *y)
{
    const long long N = ipow(n, dim);
    #pragma omp parallel for schedule(static)
    for (long long i = 0; i < N; ++i) {
        int x[3];
        coords(dim, n, i, x);
        y[i] = a_row_apply(dim, n, w, K, M, x, u);
    }
}

/* Modular inverse of g mod q (gcd(g, q) = 1), by search. */
static int inv_mod(int g, int q)
{
    for (int t = 1; t < q; ++t)
        if ((t * g) % q == 1) return t;
    return q == 1 ? 0 : -1;
}

int or_schedule(int dim, int n, int s, int p, int kind, int tile, int period, int stride,
                int *colour, int *order)
{
    return or_schedule_grouped(dim, n, s, p, kind, tile, period, stride, 1, colour, order);
}

int or_schedule_grouped(int dim, int n, int s, int p, int kind, int tile, int period, int stride,
                        int groups, int *colour, int *order)
{
    if (dim < 2 || dim > 3 || s < 1 || (s % 2) == 0 || n < 1 || groups < 1) return -1;
    const long long N = ipow(n, dim);
    const int q = period;
    if (kind != 0 && (q < s + p || stride < 1 || inv_mod(stride % q, q) < 0)) return -1;
    const int ginv = kind != 0 ? inv_mod(stride % q, q) : 1;
    const long long nlat = kind != 0 ? ipow(q, dim) : 1;
    long long ncol;
    if (kind == 0)
        ncol = N;
    else if (kind == 1)
        ncol = nlat;
    else if (kind == 2) {
        if (tile < q) return -1; /* same-phase tiles must be q-1 or more apart */
        if (groups > nlat) return -1;
        ncol = (long long)groups * ipow(2, dim) * nlat;
    } else
        return -1;

    /* offset o of a centre within its period is visited at position
     * rank(o) = o * stride^{-1} mod q, i.e. offsets in the order 0, g, 2g, ... */
    int c[3];
    for (long long i = 0; i < N; ++i) {
        coords(dim, n, i, c);
        long long col = 0;
        if (kind == 0) {
            col = i;
        } else if (kind == 1) {
            for (int k = dim - 1; k >= 0; --k) col = col * q + ((c[k] % q) * ginv) % q;
        } else {
            long long tp = 0, lc = 0;
            for (int k = dim - 1; k >= 0; --k) {
                tp = tp * 2 + ((c[k] / tile) % 2);
                lc = lc * q + (((c[k] % tile) % q) * ginv) % q;
            }
            /* colour group of the lattice colour: for each group in turn the 2^d tile
             * phases run that group's colours */
            const long long grp = lc * groups / nlat;
            col = (grp * ipow(2, dim) + tp) * nlat + lc;
        }
        colour[i] = (int)col;
    }
    /* ascending colour, ties in index order (counting sort, stable) */
    long long *start = calloc((size_t)ncol + 1, sizeof(long long));
    for (long long i = 0; i < N; ++i) start[colour[i] + 1]++;
    for (long long k = 0; k < ncol; ++k) start[k + 1] += start[k];
    for (long long i = 0; i < N; ++i) order[start[colour[i]]++] = (int)i;
    free(start);
    return (int)ncol;
}

int or_cholesky(int N, double *A)
{
    for (int j = 0; j < N; ++j) {
        double d = A[(size_t)j * N + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * N + k] * A[(size_t)j * N + k];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        A[(size_t)j * N + j] = d;
        for (int i = j + 1; i < N; ++i) {
            double v = A[(size_t)i * N + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * N + k] * A[(size_t)j * N + k];
            A[(size_t)i * N + j] = v / d;
        }
        for (int i = 0; i < j; ++i) A[(size_t)i * N + j] = 0.0;
    }
    return 0;
}

void or_cholesky_solve(int N, const double *L, const double *b, double *x)
{
    double *y = malloc(sizeof(double) * N);
    for (int i = 0; i < N; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= L[(size_t)i * N + k] * y[k];
        y[i] = v / L[(size_t)i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < N; ++k) v -= L[(size_t)k * N + i] * x[k];
        x[i] = v / L[(size_t)i * N + i];
    }
    free(y);
}

/* Scratch of one Schwarz block solve (s^d unknowns at most). */
typedef struct {
    long long *gidx;
    int *gco;
    double *AB, *rB, *eB;
} block_scratch;

static void scratch_alloc(block_scratch *w, int nbmax)
{
    w->gidx = malloc(sizeof(long long) * nbmax);
    w->gco = malloc(sizeof(int) * 3 * nbmax);
    w->AB = malloc(sizeof(double) * nbmax * nbmax);
    w->rB = malloc(sizeof(double) * nbmax);
    w->eB = malloc(sizeof(double) * nbmax);
}

static void scratch_free(block_scratch *w)
{
    free(w->gidx); free(w->gco); free(w->AB); free(w->rB); free(w->eB);
}

/* Section 3.1.1, one block: B_p^j = the s^d box around centre c clipped to the grid,
 * u_B += (A_B)^{-1} (b - A u)_B with A_B = V A V^T by Cholesky. */
static void schwarz_block(int dim, int n, int w, int s, const double *K, const double *M, int centre,
                          const double *b, double *u, block_scratch *ws)
{
    const int r = (s - 1) / 2;
    int c[3];
    coords(dim, n, centre, c);
    /* grid points of the box, lexicographic, x fastest */
    int nb = 0;
    const int oz0 = dim == 3 ? -r : 0, oz1 = dim == 3 ? r : 0;
    for (int oz = oz0; oz <= oz1; ++oz)
        for (int oy = -r; oy <= r; ++oy)
            for (int ox = -r; ox <= r; ++ox) {
                const int x = c[0] + ox, y = c[1] + oy, z = c[2] + oz;
                if (x < 0 || x >= n || y < 0 || y >= n || z < 0 || z >= (dim == 3 ? n : 1)) continue;
                ws->gco[3 * nb] = x;
                ws->gco[3 * nb + 1] = y;
                ws->gco[3 * nb + 2] = z;
                ws->gidx[nb] = x + (long long)n * (y + (long long)n * z);
                ++nb;
            }
    /* A_p^{B_j} = V A V^T and the block residual V (b - A u) */
    for (int a = 0; a < nb; ++a) {
        for (int e = 0; e < nb; ++e)
            ws->AB[a * nb + e] = a_entry(dim, n, K, M, &ws->gco[3 * a], &ws->gco[3 * e]);
        ws->rB[a] = b[ws->gidx[a]] - a_row_apply(dim, n, w, K, M, &ws->gco[3 * a], u);
    }
    or_cholesky(nb, ws->AB);
    or_cholesky_solve(nb, ws->AB, ws->rB, ws->eB);
    for (int a = 0; a < nb; ++a) u[ws->gidx[a]] += ws->eB[a];
}

/* Section 3.1.1: one multiplicative Schwarz iteration, blocks visited in the
 * given order; block j is the s^d box around its grid point clipped to the grid. */
void or_schwarz_sweep(int dim, int n, int w, int s, const double *K, const double *M,
                      const int *order, const double *b, double *u)
{
    const long long N = ipow(n, dim);
    block_scratch ws;
    scratch_alloc(&ws, (int)ipow(s, dim));
    for (long long t = 0; t < N; ++t) schwarz_block(dim, n, w, s, K, M, order[t], b, u, &ws);
    scratch_free(&ws);
}

/* The same sweep with the colour of every centre known: each run of consecutive
 * same-coloured centres in the order is one set of blocks that share no DOF and read
 * none another writes, so with OpenMP the blocks of a run are solved by several threads
 * at once; the result is the sequential sweep's, bit for bit. */
static void schwarz_sweep_colours(int dim, int n, int w, int s, const double *K, const double *M,
                                  const int *order, const int *colour, const double *b, double *u)
{
    const long long N = ipow(n, dim);
    const int nbmax = (int)ipow(s, dim);
    long long t0 = 0;
    while (t0 < N) {
        long long t1 = t0 + 1;
        while (t1 < N && colour[order[t1]] == colour[order[t0]]) ++t1;
        #pragma omp parallel
        {
            block_scratch ws;
            scratch_alloc(&ws, nbmax);
            #pragma omp for schedule(static)
            for (long long t = t0; t < t1; ++t) schwarz_block(dim, n, w, s, K, M, order[t], b, u, &ws);
            scratch_free(&ws);
        }
        t0 = t1;
    }
}

/* Threads used by the parallel loops (only in the OpenMP build of the oracle). */
#ifdef _OPENMP
#include <omp.h>
void or_set_threads(int nthreads) { if (nthreads > 0) omp_set_num_threads(nthreads); }
int or_threads(void) { return omp_get_max_threads(); }
#else
void or_set_threads(int nthreads) { (void)nthreads; }
int or_threads(void) { return 1; }
#endif

/* ------------------------------------------------------------------------ */

struct or_problem {
    int dim, p, m, n, s, w;
    int kind, tile, coarse_kind, aggressive;
    long long N;
    double *K, *M;   /* n x n */
    int *order, *order_rev, *colour;
    int nc;          /* second-level DOFs per axis */
    double *R;       /* nc x n */
    int *Rlo, *Rhi;  /* nonzero column range of each row of R */
    int *Clo, *Chi;  /* nonzero row range of each column of R */
    int nlev;
    int ml[OR_MAXLEV], nl[OR_MAXLEV];
    double *Kl[OR_MAXLEV], *Ml[OR_MAXLEV];
    double *Sl[OR_MAXLEV]; /* embedding level l+1 -> l, nl[l] x nl[l+1] */
    double *Lc;            /* Cholesky factor of the direct level */
};

int or_n(const or_problem *P) { return P->n; }
int or_nc(const or_problem *P) { return P->nc; }
long long or_ndofs(const or_problem *P) { return P->N; }

static double *dense_kron_A(int dim, int n, const double *K, const double *M)
{
    const long long N = ipow(n, dim);
    double *A = malloc(sizeof(double) * N * N);
    int x[3], y[3];
    for (long long i = 0; i < N; ++i) {
        coords(dim, n, i, x);
        for (long long j = 0; j < N; ++j) {
            coords(dim, n, j, y);
            A[i * N + j] = a_entry(dim, n, K, M, x, y);
        }
    }
    return A;
}

or_problem *or_setup(int dim, int p, int m, int s, int sched_kind, int tile,
                     int period, int stride, int coarse_kind, int aggressive)
{
    return or_setup_grouped(dim, p, m, s, sched_kind, tile, period, stride, 1, coarse_kind, aggressive);
}

or_problem *or_setup_grouped(int dim, int p, int m, int s, int sched_kind, int tile,
                             int period, int stride, int groups, int coarse_kind, int aggressive)
{
    return or_setup_plow(dim, p, m, s, sched_kind, tile, period, stride, groups, coarse_kind, aggressive, 1);
}

or_problem *or_setup_plow(int dim, int p, int m, int s, int sched_kind, int tile, int period, int stride,
                          int groups, int coarse_kind, int aggressive, int plow)
{
    if (plow < 1 || plow > 2 || (plow == 2 && coarse_kind != 0)) return NULL;
    if (dim < 2 || dim > 3 || p < 1 || m < 2) return NULL;
    if (s <= 0) s = or_block_size(p);
    if (s <= 0 || (s % 2) == 0) return NULL;
    if (aggressive && (m % 2 != 0 || m < 4)) return NULL;
    or_problem *P = calloc(1, sizeof(or_problem));
    P->dim = dim; P->p = p; P->m = m; P->s = s; P->w = p;
    P->kind = sched_kind; P->tile = tile; P->coarse_kind = coarse_kind; P->aggressive = aggressive;
    P->n = m + p - 2;
    P->N = ipow(P->n, dim);
    const int n = P->n;
    P->K = malloc(sizeof(double) * n * n);
    P->M = malloc(sizeof(double) * n * n);
    or_assemble_1d(p, m, 0, P->K, P->M);
    P->colour = malloc(sizeof(int) * P->N);
    P->order = malloc(sizeof(int) * P->N);
    P->order_rev = malloc(sizeof(int) * P->N);
    if (or_schedule_grouped(dim, n, s, p, sched_kind, tile, period, stride, groups, P->colour, P->order) < 0) {
        or_free(P);
        return NULL;
    }
    for (long long i = 0; i < P->N; ++i) P->order_rev[i] = P->order[P->N - 1 - i];

    /* second level: degree plow on h (m elements) or on 2h (m/2 elements) */
    const int m0 = aggressive ? m / 2 : m;
    P->nc = m0 + plow - 2;
    P->R = malloc(sizeof(double) * (size_t)P->nc * n);
    or_restriction_plow(p, plow, m, aggressive, P->R);
    P->Rlo = malloc(sizeof(int) * P->nc); P->Rhi = malloc(sizeof(int) * P->nc);
    P->Clo = malloc(sizeof(int) * n); P->Chi = malloc(sizeof(int) * n);
    for (int I = 0; I < P->nc; ++I) {
        int lo = n, hi = -1;
        for (int j = 0; j < n; ++j)
            if (P->R[(size_t)I * n + j] != 0.0) { lo = imin(lo, j); hi = imax(hi, j); }
        P->Rlo[I] = lo; P->Rhi[I] = hi;
    }
    for (int j = 0; j < n; ++j) {
        int lo = P->nc, hi = -1;
        for (int I = 0; I < P->nc; ++I)
            if (P->R[(size_t)I * n + j] != 0.0) { lo = imin(lo, I); hi = imax(hi, I); }
        P->Clo[j] = lo; P->Chi[j] = hi;
    }

    /* degree-1 hierarchy for the V(1,1) cycle of Section 3.2; the coarsest level
     * (8 or fewer elements per axis, or an odd count) is solved directly */
    int ml = m0, L = 0;
    for (;;) {
        P->ml[L] = ml;
        P->nl[L] = ml + plow - 2;
        const int nn = ml + plow - 2;
        P->Kl[L] = malloc(sizeof(double) * nn * nn);
        P->Ml[L] = malloc(sizeof(double) * nn * nn);
        or_assemble_1d(plow, ml, 0, P->Kl[L], P->Ml[L]);
        ++L;
        if (coarse_kind == 0 || ml <= 8 || (ml % 2) != 0 || L >= OR_MAXLEV) break;
        ml /= 2;
    }
    P->nlev = L;
    for (int l = 0; l + 1 < L; ++l) {
        P->Sl[l] = malloc(sizeof(double) * (size_t)P->nl[l] * P->nl[l + 1]);
        or_embed_p1(P->ml[l + 1], P->Sl[l]);
    }
    const int nd = P->nl[L - 1];
    P->Lc = dense_kron_A(dim, nd, P->Kl[L - 1], P->Ml[L - 1]);
    if (or_cholesky((int)ipow(nd, dim), P->Lc) != 0) {
        or_free(P);
        return NULL;
    }
    return P;
}

void or_free(or_problem *P)
{
    if (!P) return;
    free(P->K); free(P->M); free(P->order); free(P->order_rev); free(P->colour);
    free(P->R); free(P->Rlo); free(P->Rhi); free(P->Clo); free(P->Chi);
    for (int l = 0; l < P->nlev; ++l) { free(P->Kl[l]); free(P->Ml[l]); free(P->Sl[l]); }
    free(P->Lc);
    free(P);
}

double or_norm2(long long N, const double *v)
{
    double s = 0.0;
    for (long long i = 0; i < N; ++i) s += v[i] * v[i];
    return sqrt(s);
}

/* Algorithm 1: defect d_p = b_p - A_p u_p. */
void or_residual(const or_problem *P, const double *u, const double *b, double *d)
{
    or_apply_A(P->dim, P->n, P->w, P->K, P->M, u, d);
    #pragma omp parallel for schedule(static)
    for (long long i = 0; i < P->N; ++i) d[i] = b[i] - d[i];
}

void or_smooth(const or_problem *P, const double *b, double *u)
{
    schwarz_sweep_colours(P->dim, P->n, P->w, P->s, P->K, P->M, P->order, P->colour, b, u);
}

/* d_c = (R (x) R [(x) R]) d, Kronecker product of the 1D restriction. */
void or_restrict(const or_problem *P, const double *d, double *dc)
{
    const int n = P->n, nc = P->nc, dim = P->dim;
    const double *R = P->R;
    const int Z = dim == 3 ? nc : 1;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int K3 = 0; K3 < Z; ++K3)
        for (int J = 0; J < nc; ++J)
            for (int I = 0; I < nc; ++I) {
                double acc = 0.0;
                const int k0 = dim == 3 ? P->Rlo[K3] : 0, k1 = dim == 3 ? P->Rhi[K3] : 0;
                for (int k = k0; k <= k1; ++k) {
                    const double rz = dim == 3 ? R[(size_t)K3 * n + k] : 1.0;
                    for (int j = P->Rlo[J]; j <= P->Rhi[J]; ++j)
                        for (int i = P->Rlo[I]; i <= P->Rhi[I]; ++i)
                            acc += rz * R[(size_t)J * n + j] * R[(size_t)I * n + i]
                                 * d[i + (long long)n * (j + (long long)n * k)];
                }
                dc[I + (long long)nc * (J + (long long)nc * K3)] = acc;
            }
}

/* u += (R (x) R [(x) R])^T e_c: the prolongation is the adjoint of the restriction (Section 3.1.2). */
void or_prolong_add(const or_problem *P, const double *ec, double *u)
{
    const int n = P->n, nc = P->nc, dim = P->dim;
    const double *R = P->R;
    const int Z = dim == 3 ? n : 1;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < Z; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                const int K0 = dim == 3 ? P->Clo[k] : 0, K1 = dim == 3 ? P->Chi[k] : 0;
                for (int K3 = K0; K3 <= K1; ++K3) {
                    const double rz = dim == 3 ? R[(size_t)K3 * n + k] : 1.0;
                    for (int J = P->Clo[j]; J <= P->Chi[j]; ++J)
                        for (int I = P->Clo[i]; I <= P->Chi[i]; ++I)
                            acc += rz * R[(size_t)J * n + j] * R[(size_t)I * n + i]
                                 * ec[I + (long long)nc * (J + (long long)nc * K3)];
                }
                u[i + (long long)n * (j + (long long)n * k)] += acc;
            }
}

/* One red-black Gauss-Seidel pass on level l (Section 3.2).  Red points have an
 * even coordinate sum, black points an odd one.  On the 9-point (27-point)
 * degree-1 stencil, points of one colour still couple diagonally, so each
 * colour is visited as its parity sub-lattices (x_k mod 2 fixed for every k),
 * none of which contains two coupled points: every red point is relaxed before
 * every black point, each with the latest values of all its neighbours.  The
 * post-smoother visits the sub-lattices in the reverse order. */
static const int gs_seq2[4] = {0, 3, 1, 2};
static const int gs_seq3[8] = {0, 3, 5, 6, 1, 2, 4, 7};

static void gs_level(const or_problem *P, int l, const double *rhs, double *e, int forward)
{
    const int dim = P->dim, nn = P->nl[l];
    const long long Nl = ipow(nn, dim);
    const int ncol = 1 << dim;
    const int *seq = dim == 2 ? gs_seq2 : gs_seq3;
    for (int t = 0; t < ncol; ++t) {
        const int col = seq[forward ? t : ncol - 1 - t];
        /* the points of one sub-lattice do not couple: relaxed by several threads at once */
        #pragma omp parallel for schedule(static)
        for (long long i = 0; i < Nl; ++i) {
            int x[3];
            coords(dim, nn, i, x);
            int c = (x[0] & 1) | ((x[1] & 1) << 1) | (dim == 3 ? ((x[2] & 1) << 2) : 0);
            if (c != col) continue;
            const double diag = a_entry(dim, nn, P->Kl[l], P->Ml[l], x, x);
            const double Ax = a_row_apply(dim, nn, 1, P->Kl[l], P->Ml[l], x, e);
            e[i] += (rhs[i] - Ax) / diag;
        }
    }
}

/* rc = (S^T (x) S^T ...) r and e += (S (x) S ...) ec for the embedding S of level l+1 into l */
static void level_restrict(const or_problem *P, int l, const double *r, double *rc)
{
    const int dim = P->dim, nf = P->nl[l], nc = P->nl[l + 1];
    const double *S = P->Sl[l];
    const long long Nc = ipow(nc, dim);
    #pragma omp parallel for schedule(static)
    for (long long Ic = 0; Ic < Nc; ++Ic) {
        int X[3];
        coords(dim, nc, Ic, X);
        double acc = 0.0;
        /* column I of S is nonzero only on rows 2I .. 2I+2 */
        const int z0 = dim == 3 ? 2 * X[2] : 0, z1 = dim == 3 ? 2 * X[2] + 2 : 0;
        for (int k = z0; k <= z1; ++k)
            for (int j = 2 * X[1]; j <= 2 * X[1] + 2; ++j)
                for (int i = 2 * X[0]; i <= 2 * X[0] + 2; ++i) {
                    double wgt = S[(size_t)i * nc + X[0]] * S[(size_t)j * nc + X[1]];
                    if (dim == 3) wgt *= S[(size_t)k * nc + X[2]];
                    acc += wgt * r[i + (long long)nf * (j + (long long)nf * k)];
                }
        rc[Ic] = acc;
    }
}

static void level_prolong_add(const or_problem *P, int l, const double *ec, double *e)
{
    const int dim = P->dim, nf = P->nl[l], nc = P->nl[l + 1];
    const double *S = P->Sl[l];
    const long long Nf = ipow(nf, dim);
    #pragma omp parallel for schedule(static)
    for (long long i = 0; i < Nf; ++i) {
        int x[3];
        coords(dim, nf, i, x);
        double acc = 0.0;
        /* row x of S is nonzero only on columns (x-2)/2 .. x/2 (rounded inward) */
        int lo[3], hi[3];
        for (int k = 0; k < 3; ++k) {
            lo[k] = imax(0, (x[k] - 1) / 2 - 1);
            hi[k] = imin(nc - 1, x[k] / 2);
        }
        if (dim == 2) { lo[2] = 0; hi[2] = 0; }
        for (int Z = lo[2]; Z <= hi[2]; ++Z)
            for (int Y = lo[1]; Y <= hi[1]; ++Y)
                for (int Xc = lo[0]; Xc <= hi[0]; ++Xc) {
                    double wgt = S[(size_t)x[0] * nc + Xc] * S[(size_t)x[1] * nc + Y];
                    if (dim == 3) wgt *= S[(size_t)x[2] * nc + Z];
                    acc += wgt * ec[Xc + (long long)nc * (Y + (long long)nc * Z)];
                }
        e[i] += acc;
    }
}

/* Section 3.2: one V(1,1) cycle on level l, started from e = 0. */
void or_vcycle_level(const or_problem *P, int l, const double *rhs, double *e)
{
    const int dim = P->dim, nn = P->nl[l];
    const long long Nl = ipow(nn, dim);
    if (l == P->nlev - 1) {
        or_cholesky_solve((int)Nl, P->Lc, rhs, e);
        return;
    }
    memset(e, 0, sizeof(double) * Nl);
    gs_level(P, l, rhs, e, 1);
    double *r = malloc(sizeof(double) * Nl);
    or_apply_A(dim, nn, 1, P->Kl[l], P->Ml[l], e, r);
    for (long long i = 0; i < Nl; ++i) r[i] = rhs[i] - r[i];
    const long long Nc = ipow(P->nl[l + 1], dim);
    double *rc = malloc(sizeof(double) * Nc), *ec = malloc(sizeof(double) * Nc);
    level_restrict(P, l, r, rc);
    or_vcycle_level(P, l + 1, rc, ec);
    level_prolong_add(P, l, ec, e);
    gs_level(P, l, rhs, e, 0);
    free(r); free(rc); free(ec);
}

/* Algorithm 1, "A_{p_low} e_{p_low} = d_{p_low}": exact (Cholesky) or one V(1,1). */
void or_coarse_solve(const or_problem *P, const double *dc, double *ec)
{
    or_vcycle_level(P, 0, dc, ec);
}

static void coarse_correction(const or_problem *P, const double *b, double *u)
{
    const long long Nc = ipow(P->nc, P->dim);
    double *d = malloc(sizeof(double) * P->N);
    double *dc = malloc(sizeof(double) * Nc), *ec = malloc(sizeof(double) * Nc);
    or_residual(P, u, b, d);
    or_restrict(P, d, dc);
    or_coarse_solve(P, dc, ec);
    or_prolong_add(P, ec, u);
    free(d); free(dc); free(ec);
}

/* Algorithm 1: Schwarz step, defect, restriction, coarse solve, prolongation + update. */
void or_cycle(const or_problem *P, const double *b, double *u)
{
    or_smooth(P, b, u);
    coarse_correction(P, b, u);
}

void or_cycle_adjoint(const or_problem *P, const double *b, double *u)
{
    coarse_correction(P, b, u);
    schwarz_sweep_colours(P->dim, P->n, P->w, P->s, P->K, P->M, P->order_rev, P->colour, b, u);
}

/* Section 5: random initial guess, stop when the initial residual is reduced by tol. */
int or_solve(const or_problem *P, const double *b, double tol, int maxc, int adjoint,
             double *u, int *cycles, double *relres, double *hist)
{
    double *d = malloc(sizeof(double) * P->N);
    or_residual(P, u, b, d);
    const double r0 = or_norm2(P->N, d);
    int k = 0, status = 1;
    double rel = 0.0;
    if (r0 == 0.0) status = 0;
    while (status != 0 && k < maxc) {
        if (adjoint) or_cycle_adjoint(P, b, u); else or_cycle(P, b, u);
        ++k;
        or_residual(P, u, b, d);
        rel = or_norm2(P->N, d) / r0;
        if (hist) hist[k - 1] = rel;
        if (rel <= tol) status = 0;
    }
    *cycles = k;
    *relres = rel;
    free(d);
    return status;
}
