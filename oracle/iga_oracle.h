/*
 * iga_oracle.h -- plain, slow, FP64 CPU oracle of the two-level method of
 * de la Riva, Rodrigo and Gaspar, "A two level method for isogeometric
 * discretizations" (arXiv 2009.01499).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this code; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or table generator
 * with the CUDA path.
 *
 * Conventions
 *   - All arithmetic is IEEE binary64, built with -ffp-contract=off.
 *   - Dense 1D matrices are row-major, A[i*ncol + j].
 *   - Grid vectors of a d-dimensional problem with n DOFs per axis are stored
 *     C-order with x fastest: index = i + n*(j + n*k).
 *   - Spline index i (0-based) in a restricted space is the paper's N_{i+2}.
 *
 * Parity status of each function is stated beside it ("pinned by" lists the
 * independent checks in tests/ that fix it).
 */
#ifndef IGA_ORACLE_H
#define IGA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Section 2.1: splines ------------------------------------------------ */

/* Open uniform knot vector Xi_{p,h} (Section 2.1): 2p+m+1 knots. */
void or_knots(int p, int m, double *xi);

/* All m+p functions of the full degree-p basis at x in [0,1] by the Cox-de Boor
 * recursion (eqs. constantspline / order_spline), and their derivatives.
 * Pinned by: partition of unity, non-negativity, finite-difference derivative. */
void or_basis_eval(int p, int m, double x, double *N, double *dN);

/* Gauss-Legendre rule with npts points on [-1,1].
 * Pinned by: exact integration of monomials up to degree 2*npts-1. */
void or_gauss(int npts, double *x, double *w);

/* 1D Galerkin stiffness K_ij = int N_i' N_j' and mass M_ij = int N_i N_j
 * (Section 2, A_p = (a(phi_j, phi_i))).  full=1: all m+p functions;
 * full=0: Dirichlet-restricted space of eq. (splinespace), n = m+p-2.
 * Pinned by: zero row sums of full K, sum of full M = 1, symmetry, interior
 * rows equal to the cardinal B-spline closed form, O(h^{p+1}) L2 convergence. */
void or_assemble_1d(int p, int m, int full, double *K, double *M);

/* Mixed mass (M_p^{plow})_{ij} = int phi_i^{plow} phi_j^p of Section 3.1.2 on the
 * same mesh: (m+plow-2) x (m+p-2), restricted bases on both sides. */
void or_mixed_mass_1d(int p, int plow, int m, double *Mx);

/* 1D load g_i = int f1(x) N_i(x) dx on the restricted space, nq Gauss points
 * per element.  kind 0: f1 = sin(pi x); kind 1: f1 = exp(-(x-c)^2/(2 w^2)),
 * par = {c, w}.  Two-dimensional separable loads are tensor products of these. */
void or_load_1d(int p, int m, int kind, const double *par, int nq, double *g);

/* Degree-1 embedding of the 2h space into the h space (the standard h-transfer
 * between equal-degree spline spaces, Section 4.1): S[i][I] = Phi_I(x_i), the
 * restricted hat I of mesh 1/mc evaluated at interior node i of mesh 1/(2mc).
 * (2mc-1) x (mc-1).  Pinned by: [1/2,1,1/2] stencil, Galerkin identity. */
void or_embed_p1(int mc, double *S);

/* Embedding of the restricted degree-plow spline space on mc elements into the one on
 * 2 mc elements, S = (M_fine)^{-1} (phi_fine, phi_coarse) (exact: nested spaces).
 * (2mc + plow - 2) x (mc + plow - 2).  Pinned by: equal to or_embed_p1 for plow = 1; the
 * quadratic subdivision weights (1/4, 3/4, 3/4, 1/4) in the interior; Galerkin identities
 * S^T M_f S = M_c and S^T K_f S = K_c. */
void or_embed_spline(int plow, int mc, double *S);

/* Restriction of Section 3.1.2 with row-sum lumping to degree plow (1 or 2):
 * aggressive=0: R = D^{-1} M_p^plow, (m+plow-2) x n; aggressive=1: R = S^T D^{-1} M_p^plow,
 * (m/2+plow-2) x n, S the degree-plow 2h -> h embedding.  D = row sums of the restricted
 * degree-plow mass.  Pinned by: scipy mixed mass, interior row sums 1, equal to
 * or_restriction_1d for plow = 1, the dense two-level cycle with it. */
void or_restriction_plow(int p, int plow, int m, int aggressive, double *R);

/* Restriction of Section 3.1.2 with row-sum lumping, plow = 1:
 * aggressive=0: R = D^{-1} M_p^1, (m-1) x n   (same mesh h, Section 3.1.2)
 * aggressive=1: R = S^T D^{-1} M_p^1, (m/2-1) x n   (degree p -> 1, then h -> 2h,
 * Section 3.3).  D = row sums of the restricted degree-1 mass.  Prolongation is R^T. */
void or_restriction_1d(int p, int m, int aggressive, double *R);

/* ---- Section 3.1.1: operator and multiplicative Schwarz ------------------ */

/* Block side s for degree p: 3 (p=2,3,4), 5 (p=5,6), 7 (p=7,8).  Section 4.3. */
int or_block_size(int p);

/* y = A u, A = K(x)M + M(x)K in 2D, K(x)M(x)M + M(x)K(x)M + M(x)M(x)K in 3D, with
 * dense n x n 1D matrices of half bandwidth w.  Pinned by: explicit Kronecker. */
void or_apply_A(int dim, int n, int w, const double *K, const double *M,
                const double *u, double *y);

/* Schedules (block visiting orders); the paper's own colouring is not given,
 * these are this project's.  kind 0 = LEX (index order); 1 = LATTICE: the
 * colour of centre c is sum_k rank(c_k mod q) q^k with period q >= s+p and
 * rank(o) = o * g^{-1} mod q (offsets visited in the order 0, g, 2g, ...,
 * gcd(g, q) = 1); 2 = TILE(T): tile phase sum_k ((c_k/T) mod 2) 2^k (T >= q),
 * then the LATTICE colours anchored at the tile origin.  Blocks of one colour
 * are at least q >= s+p apart along some axis, so they share no DOF and none
 * reads a DOF another writes.  Writes every centre's colour and the processing
 * order (ascending colour, then index); returns the number of colours or -1. */
int or_schedule(int dim, int n, int s, int p, int kind, int tile, int period, int stride,
                int *colour, int *order);
/* TILE(T) with the lattice colours split into `groups` consecutive groups (group of
 * colour rank l: floor(l groups / q^d)): for each group in turn, the 2^d tile phases run
 * that group's colours.  groups = 1 is TILE(T); groups = q^d runs every colour over all
 * tiles before the next, the LATTICE order.  Same colour and order outputs as or_schedule
 * (colour = (group 2^d + tile phase) q^d + lattice colour); the number of colours or -1.
 * Pinned by: brute-force coupling-freedom of every colour; groups = 1 reproduces
 * or_schedule's TILE order and groups = q^d its LATTICE order. */
int or_schedule_grouped(int dim, int n, int s, int p, int kind, int tile, int period, int stride,
                        int groups, int *colour, int *order);

/* One multiplicative Schwarz step (Section 3.1.1): for every centre c in the
 * given order, B = (c + [-r,r]^d) clipped to the grid, r = (s-1)/2, and
 * u_B += (A_B)^{-1} (b - A u)_B with A_B = V_B A V_B^T solved by Cholesky.
 * Pinned by: the product formula prod_j (I - V_j^T A_j^{-1} V_j A) on tiny grids. */
void or_schwarz_sweep(int dim, int n, int w, int s, const double *K, const double *M,
                      const int *order, const double *b, double *u);

/* Threads of the parallel loops.  The oracle is also built with OpenMP (a second shared
 * object): the blocks of one Schwarz colour, the points of one Gauss-Seidel sub-lattice
 * and the outputs of the stencil and transfer loops are independent, so they are split
 * over threads with results identical to the sequential run, bit for bit (sums are never
 * split).  Without OpenMP these are no-ops and or_threads() is 1. */
void or_set_threads(int nthreads);
int or_threads(void);

/* Dense Cholesky A = L L^T in place (lower triangle); returns 0 or -1 (not SPD). */
int or_cholesky(int N, double *A);
void or_cholesky_solve(int N, const double *L, const double *b, double *x);

/* ---- Algorithm 1 and Sections 3.2/3.3: the whole cycle -------------------- */

typedef struct or_problem or_problem;

/* coarse_kind 0 = exact second-level solve (dense Cholesky); 1 = one V(1,1)
 * cycle with red-black Gauss-Seidel (Section 3.2) on the degree-1 hierarchy,
 * direct solve once a level has 8 or fewer elements per axis.  s <= 0 picks
 * or_block_size(p).  Returns NULL on bad arguments. */
or_problem *or_setup(int dim, int p, int m, int s, int sched_kind, int tile,
                     int period, int stride, int coarse_kind, int aggressive);
/* or_setup with a grouped TILE schedule (or_schedule_grouped); groups = 1 is or_setup. */
or_problem *or_setup_grouped(int dim, int p, int m, int s, int sched_kind, int tile,
                             int period, int stride, int groups, int coarse_kind, int aggressive);
/* The same with a second level of degree plow (1 or 2, Section 3: the "linear or
 * quadratic" coarse discretisation): the restriction or_restriction_plow and the Galerkin
 * degree-plow matrix on the second-level mesh.  plow = 2 takes the exact second-level
 * solve only (coarse_kind 0; the V(1,1) of Section 3.2 is for the degree-1 hierarchy). */
or_problem *or_setup_plow(int dim, int p, int m, int s, int sched_kind, int tile, int period, int stride,
                          int groups, int coarse_kind, int aggressive, int plow);
void or_free(or_problem *P);
int  or_n(const or_problem *P);          /* DOFs per axis */
int  or_nc(const or_problem *P);         /* second-level DOFs per axis */
long long or_ndofs(const or_problem *P); /* n^d */

/* Pinned by (problem level): or_residual = b - (explicit Kronecker A) u; or_smooth =
 * the product formula above for the problem's schedule; or_restrict / or_prolong_add =
 * Kronecker products of or_restriction_1d and their adjointness; or_coarse_solve =
 * the dense Cholesky solve (exact kind) or, V-cycle kind, a V(1,1) whose whole
 * approximate inverse equals the dense product of its steps built independently (the
 * sub-lattice Gauss-Seidel sweeps, the level restriction and embedding, the coarsest
 * solve), and which is symmetric and contracts; or_cycle = the dense (I - R^T A_c^{-1} R A) S_E on tiny grids;
 * or_cycle_adjoint = <C x, y> = <x, C^T y> and the dense C^T; or_solve = the stopping
 * rule and the Section 5.1 manufactured solution reached to 1e-8.  In 3D (the paper is
 * 2D only) these are pinned by the same mathematics and parity is unpinned by the
 * paper (no 3D numbers exist); the paper's tables pin the 2D method only softly, its
 * three-colour ordering being unavailable. */
void   or_residual(const or_problem *P, const double *u, const double *b, double *d);
double or_norm2(long long N, const double *v);
void   or_smooth(const or_problem *P, const double *b, double *u);          /* Schwarz step */
void   or_restrict(const or_problem *P, const double *d, double *dc);      /* d_c = R d */
void   or_prolong_add(const or_problem *P, const double *ec, double *u);   /* u += R^T e_c */
void   or_coarse_solve(const or_problem *P, const double *dc, double *ec); /* A_c e_c ~= d_c */
void   or_vcycle_level(const or_problem *P, int level, const double *rhs, double *e);
void   or_cycle(const or_problem *P, const double *b, double *u);          /* Algorithm 1 */
/* Transposed cycle operator: coarse correction first, then the Schwarz step in
 * reversed order.  Used by the adjoint. */
void   or_cycle_adjoint(const or_problem *P, const double *b, double *u);
/* Cycles until ||b - A u||_2 <= tol ||b - A u_0||_2 or maxc cycles; hist gets
 * the relative residual after each cycle (may be NULL).  Returns 0 converged, 1 not. */
int    or_solve(const or_problem *P, const double *b, double tol, int maxc, int adjoint,
                double *u, int *cycles, double *relres, double *hist);

#ifdef __cplusplus
}
#endif
#endif
