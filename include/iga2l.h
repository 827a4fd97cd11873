/*
 * iga2l.h -- C ABI of the GB300 two-level solver for B-spline isogeometric
 * Poisson problems (de la Riva, Rodrigo, Gaspar, "A two level method for
 * isogeometric discretizations", arXiv 2009.01499).
 *
 * Problem (Section 2): -Laplace(u) = f on (0,1)^d, u = 0 on the boundary,
 * Galerkin discretisation with degree-p, C^{p-1} B-splines on a uniform mesh
 * of m elements per axis.  Unknowns are the control points u_p of
 * A_p u_p = b_p (Section 2, A_p = (a(phi_j, phi_i)), b_p = (f, phi_i)).
 *
 * Conventions for every entry point
 *   - Vectors are caller-owned DEVICE pointers to contiguous float64 arrays of
 *     n^d entries, n = m + p - 2 DOFs per axis (the Dirichlet-restricted spline
 *     space of eq. (splinespace)), laid out C-order with x fastest:
 *     index = i + n*(j + n*k).  Second-level vectors have nc^d entries,
 *     nc = m/2 - 1 (degree 1 on the 2h mesh, Section 3.3).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; entry points that return a host scalar synchronise it.
 *   - The handle owns its device tables and workspace, allocated in
 *     iga2l_assemble and released by iga2l_destroy; no other entry point calls
 *     cudaMalloc.  With options.graphs = 1, the first cycle on a new (u, b)
 *     pair captures it into a CUDA graph (the driver keeps its resources until
 *     iga2l_destroy; the handle keeps the four most recently used) and later
 *     cycles replay it; when the caller's stream is itself being captured the
 *     kernels are enqueued directly instead.  A handle must not be used from
 *     two host threads at once, and two calls on one handle must not overlap
 *     on the GPU (they share workspace).
 *   - Return codes: IGA2L_OK, IGA2L_NOT_CONVERGED or a negative error code
 *     (iga2l_strerror; iga2l_last_error gives detail for the calling thread).
 *     Argument checks happen before any work is enqueued.
 */
#ifndef IGA2L_H
#define IGA2L_H

#ifdef __cplusplus
extern "C" {
#endif

#define IGA2L_OK 0
#define IGA2L_NOT_CONVERGED 1
#define IGA2L_ERR_INVALID_ARG (-1)
#define IGA2L_ERR_CUDA (-2)
#define IGA2L_ERR_DEVICE_TIMEOUT (-3)
#define IGA2L_ERR_NONFINITE (-4)
#define IGA2L_ERR_UNSUPPORTED (-5)

/* precision */
#define IGA2L_FP64 0
/* FP64 outer residual, norm and update around an FP32 inner cycle (FP32 storage
 * and FMA; FP64 boundary-block inverses, applied in the FP32 colour kernels as FP32
 * pairs by compensated (Dot2) arithmetic, and an FP64 coarsest solve): iterative
 * refinement */
#define IGA2L_MIXED_FP32 1
/* The same with the boundary-block inverses also applied in FP32 (the Schwarz blocks
 * of p <= 5 have condition numbers below 5e2, so this costs the inner cycle ~3e-5
 * relative at most, which the FP64 refinement removes; coarsest solve still FP64) */
#define IGA2L_MIXED_FP32_ALL 2
/* IGA2L_MIXED_FP32 with the interior blocks of every LATTICE colour computed as one
 * tensor-core GEMM (tcgen05, TF32 operands, FP32 accumulation): e_B = [A_B^-1 | -A_B^-1
 * A_(B,patch)] [b_B ; u_patch], the colour's other (boundary) blocks in FP32 in the same
 * launch; single 2D problems, LATTICE schedule, p <= 5 (IGA2L_ERR_UNSUPPORTED otherwise, or
 * when the lattice period makes a CTA's tile of 128 blocks exceed the shared memory) */
#define IGA2L_MIXED_TF32 3
/* schedule: colour classes of the multiplicative Schwarz step */
#define IGA2L_SCHED_LATTICE 1
#define IGA2L_SCHED_TILE 2
/* second-level solver */
#define IGA2L_COARSE_EXACT 0
#define IGA2L_COARSE_VCYCLE 1
/* right-hand side given to iga2l_solve / iga2l_solve_batch: the B-spline coefficients f
 * of the source (Section 2: b_p = (f, phi_i), formed on the device as (M(x)M) f), or the
 * load vector b_p itself */
#define IGA2L_RHS_COEFFS 0
#define IGA2L_RHS_IS_LOAD 1
/* sweep: how the Schwarz step of the FP32 inner cycle runs in the LATTICE order.  AUTO
 * picks the persistent form for colourings of at least 250 colours (p = 8's default) where
 * it is available (2D single-problem handles with IGA2L_MIXED_FP32 or IGA2L_MIXED_FP32_ALL)
 * and one launch per colour elsewhere;
 * PERSISTENT asks for it (IGA2L_ERR_UNSUPPORTED where it is not available).  Both give
 * the same iterates up to FP32 rounding order. */
#define IGA2L_SWEEP_AUTO 0
#define IGA2L_SWEEP_PER_COLOUR 1
#define IGA2L_SWEEP_PERSISTENT 2
/* WORK_LIST (TILE schedule, 2D, any precision, single or batch handles): the whole TILE sweep
 * of every problem of the handle in one launch.  CTAs claim (colour group, tile phase,
 * problem, tile) items in sweep order; a tile starts once the earlier occurrences of its own
 * and its eight neighbouring tile positions have finished (bounded device waits,
 * IGA2L_ERR_DEVICE_TIMEOUT when one gives up).  Iterates are bitwise those of one launch per tile phase (PER_COLOUR and AUTO with the
 * TILE schedule). */
#define IGA2L_SWEEP_WORK_LIST 3
/* test_flags bits (testing the error paths only; never set in production use):
 * the tensor-core colour kernel does not issue the bulk copy of its block operator, so
 * its bounded wait for that copy runs out (no copy and no MMA is ever in flight), the
 * kernel skips its blocks and the call returns IGA2L_ERR_DEVICE_TIMEOUT */
#define IGA2L_TEST_SKIP_OPERATOR_COPY 1
/* the persistent sweep's first CTA never raises its progress counter, so its neighbours'
 * bounded waits run out (nothing asynchronous is in flight); in the work-list TILE sweep no
 * finished tile is counted, so the first wait for a previous phase runs out; the call
 * returns IGA2L_ERR_DEVICE_TIMEOUT */
#define IGA2L_TEST_WITHHOLD_PROGRESS 2
/* every device buffer of the handle is placed between two 4 KiB guard zones: all-ones bytes
 * (a NaN in FP32 and FP64) around floating-point buffers, zero bytes around integer tables
 * and counters.  A kernel that reads past the end of a floating-point buffer then meets a
 * NaN that reaches its results; one that writes past either end of any buffer changes a
 * zone, which iga2l_guard_check reports.  Results are otherwise unchanged. */
#define IGA2L_TEST_GUARD_ALLOCS 4

typedef struct iga2l_solver *iga2l_handle;

typedef struct {
    int precision;   /* IGA2L_FP64, IGA2L_MIXED_FP32, IGA2L_MIXED_FP32_ALL or IGA2L_MIXED_TF32 */
    int schedule;    /* IGA2L_SCHED_LATTICE or IGA2L_SCHED_TILE */
    int tile;        /* TILE side T >= period (0 = the side compiled for p: 20 for p = 2, 5; 21 for
                        p = 3, 4; 22 for p = 6; the TILE schedule is compiled for p <= 6) */
    int period;      /* colour period q >= s + p (0 = library default for p) */
    int stride;      /* colour stride g, gcd(g, q) = 1 (0 = library default) */
    int coarse;      /* IGA2L_COARSE_VCYCLE (Section 3.2) or IGA2L_COARSE_EXACT */
    int block_side;  /* Schwarz block side s (0 = the paper's choice for p, Section 4.3) */
    int max_cycles;  /* default cap for iga2l_solve when its max_cycles <= 0 */
    int graphs;      /* 1: replay cycles as captured CUDA graphs (default); 0: plain launches */
    int rhs;         /* IGA2L_RHS_COEFFS (default) or IGA2L_RHS_IS_LOAD: what iga2l_solve and
                        iga2l_solve_batch read from their right-hand-side argument */
    int tile_groups; /* TILE: the q^d colours split into this many consecutive groups, each group
                        running the 2^d tile phases in turn (1 = plain TILE, q^d = the LATTICE
                        order; 0 = the library default: 4 for p = 6, else 1).  Capped at q^d. */
    int sweep;       /* IGA2L_SWEEP_AUTO (default), _PER_COLOUR, _PERSISTENT or _WORK_LIST: with
                        LATTICE, the FP32 inner sweep as one persistent launch (all colours;
                        every CTA owns a region, neighbours exchange their boundary bands
                        through L2 under bounded waits) or one launch per colour; with TILE,
                        the work-list sweep (_WORK_LIST) or one launch per tile phase */
    int test_flags;  /* 0, or IGA2L_TEST_* bits (error-path tests only) */
    long long wait_budget_cycles;   /* SM clock cycles a bounded device wait may spin before the
                        kernel gives up, records the failure and returns (the call then reports
                        IGA2L_ERR_DEVICE_TIMEOUT); 0 = 2^31 (about 1 s at 2 GHz) */
} iga2l_options;

/* Fills the defaults: FP64, LATTICE, V(1,1), the paper's block side, 100 cycles,
 * graphs on, right-hand side given as coefficients, default wait budget. */
void iga2l_default_options(iga2l_options *opt);

/* Builds the solver for degree p (2..8 in 2D, 2..4 in 3D), m elements per axis,
 * dimension dim (2 or 3; 3D uses the LATTICE schedule).
 * Host work: 1D B-spline Galerkin tables (Section 2.1), the Schwarz block
 * inverses of every block class (Section 3.1.1), the lumped L2-projection
 * restriction composed with h->2h (Sections 3.1.2, 3.3), the degree-1
 * hierarchy (Section 3.2) and the dense inverse of its coarsest level; then one
 * upload.  m must be even, at least 4 (the 2h level) and at least p + 1 (n >= 2p - 1: the
 * boundary row and block classes); on such small grids every block is a boundary block.
 * 3D handles, IGA2L_MIXED_TF32 and IGA2L_SWEEP_PERSISTENT need m >= 4p + 4 (grids with
 * interior blocks; AUTO then launches one kernel per colour).  The colouring must satisfy
 * q >= s+p, gcd(g,q) = 1, T >= q.
 * *out receives the handle (NULL on error).  opt may be NULL (defaults). */
int iga2l_assemble(int p, int m, int dim, const iga2l_options *opt, iga2l_handle *out);

/* Batch of nbatch independent 2D problems with the same p, m and options (the
 * tables are shared; every problem has its own workspace).  Vectors passed to a
 * batch handle hold all problems back to back: nbatch * n^2 doubles, problem k at
 * offset k * n^2.  The per-step entry points (apply_A, residual without a norm,
 * schwarz_sweep(_reverse), restrict, prolong_add, coarse_solve, cycle,
 * cycle_adjoint, cycles, rhs_from_coeffs) act on every problem; iga2l_solve,
 * iga2l_adjoint_solve, iga2l_unrolled_backward, the bump source and a residual
 * with a norm are single-problem entry points and return IGA2L_ERR_INVALID_ARG. */
int iga2l_assemble_batch(int p, int m, int nbatch, const iga2l_options *opt, iga2l_handle *out);

/* Solves every problem of a batch to its own tolerance (Section 5 stopping rule);
 * `rhs` holds every problem's coefficient vector f (or load vector b with options.rhs =
 * IGA2L_RHS_IS_LOAD), as iga2l_solve:
 * after each cycle a device kernel counts the cycle for each unfinished problem and
 * retires the problems whose relative residual is <= tol; retired problems are
 * skipped by every later kernel, so each problem's iterates and cycle count equal
 * those of a single solve.  With CUDA graphs on (the default) the cycles run inside
 * one graph whose WHILE node that kernel stops once no problem is unfinished or
 * max_cycles ran; otherwise the host polls the number of unfinished problems every
 * 4 cycles.  cycles (int) and relres (double) are host arrays of nbatch entries.
 * Returns IGA2L_OK when all converged, IGA2L_NOT_CONVERGED at the cycle cap,
 * IGA2L_ERR_NONFINITE if a norm is not finite. */
int iga2l_solve_batch(iga2l_handle h, const double *rhs, double tol, int max_cycles, double *u, int *cycles,
                      double *relres, void *stream);

/* Sizes: total fine DOFs, DOFs per axis, total and per-axis second-level DOFs.
 * Any output pointer may be NULL. */
int iga2l_num_dofs(iga2l_handle h, long long *n_total, int *n_axis,
                   long long *nc_total, int *nc_axis);

/* The Schwarz schedule the handle runs (Section 3.1.1 colouring, this library's
 * reading): schedule (IGA2L_SCHED_*), colour period q, stride g, TILE side T (0 for
 * LATTICE), block side s and the TILE order's colour groups (1 for LATTICE), with every
 * default resolved.  Outputs may be NULL. */
int iga2l_schedule_info(iga2l_handle h, int *schedule, int *period, int *stride, int *tile, int *block_side,
                        int *tile_groups);

/* y = A_p u, A_p = K(x)M + M(x)K (Section 2, tensor-product stiffness). */
int iga2l_apply_A(iga2l_handle h, const double *u, double *y, void *stream);

/* Defect d = b - A_p u (Algorithm 1).  d may be NULL (norm only).  If norm is
 * not NULL it receives ||d||_2 on the host (the stream is synchronised). */
int iga2l_residual(iga2l_handle h, const double *u, const double *b, double *d,
                   double *norm, void *stream);

/* One multiplicative Schwarz step u <- u + S_p(b - A_p u) (Section 3.1.1): for
 * every grid point, in the order of the handle's colour schedule, the s^d block
 * around it (clipped to the grid) is corrected by u_B += A_B^{-1} (b - A u)_B. */
int iga2l_schwarz_sweep(iga2l_handle h, double *u, const double *b, void *stream);

/* Same step with the colour order reversed (the transpose of the Schwarz
 * approximate inverse; used by the adjoint cycle). */
int iga2l_schwarz_sweep_reverse(iga2l_handle h, double *u, const double *b, void *stream);

/* The Schwarz step of a mixed-precision handle's inner cycle on FP32 vectors (2D):
 * u <- u + S_p(b - A_p u) in FP32 arithmetic, with the handle's schedule and sweep kernel
 * (reverse != 0: colours in reverse).  u, b: n^2 device floats.  For checking and timing
 * the inner cycle's dominant step; IGA2L_ERR_INVALID_ARG on an FP64 or 3D handle. */
int iga2l_schwarz_sweep_f32(iga2l_handle h, float *u, const float *b, int reverse, void *stream);

/* d_c = I_{p,h}^{1,2h} d (Sections 3.1.2 and 3.3): lumped L2 projection onto
 * the degree-1 space followed by the degree-1 h -> 2h restriction.  dc has nc^d entries. */
int iga2l_restrict(iga2l_handle h, const double *d, double *dc, void *stream);

/* u += I_{1,2h}^{p,h} e_c, the adjoint of iga2l_restrict (Section 3.1.2). */
int iga2l_prolong_add(iga2l_handle h, const double *ec, double *u, void *stream);

/* e_c ~= A_1^{-1} d_c on the second level: one V(1,1) cycle with red-black
 * Gauss-Seidel from e_c = 0 (Section 3.2), or the exact solve (Algorithm 1). */
int iga2l_coarse_solve(iga2l_handle h, const double *dc, double *ec, void *stream);

/* One cycle of Algorithm 1 in place: Schwarz step, defect, restriction,
 * second-level solve, prolongation and update.  With IGA2L_MIXED_FP32: r = b - A u
 * in FP64, the same cycle in FP32 on A delta = r from delta = 0, u += delta in FP64
 * (equal to the FP64 cycle in exact arithmetic, since the cycle is affine in u). */
int iga2l_cycle(iga2l_handle h, double *u, const double *b, void *stream);

/* One transposed cycle: second-level correction first, then the reversed
 * Schwarz step.  Its approximate inverse is the transpose of iga2l_cycle's. */
int iga2l_cycle_adjoint(iga2l_handle h, double *u, const double *b, void *stream);

/* Solves A_p u_p = b_p (Section 2) from the guess in u: cycles until
 * ||b - A u||_2 <= tol ||b - A u_0||_2 (Section 5 stopping rule) or max_cycles (<= 0: the
 * handle's default).  `rhs` is the source's B-spline coefficient vector f (n^d device
 * doubles; b_p = (f, phi_i) = (M(x)M[(x)M]) f is formed on the device into the handle's
 * workspace first), or b_p itself when the handle was built with options.rhs =
 * IGA2L_RHS_IS_LOAD.  Writes the cycle count, the final relative residual and, if hist is
 * not NULL, the relative residual after every cycle (host array of max_cycles).
 * Returns IGA2L_OK, IGA2L_NOT_CONVERGED or an error (IGA2L_ERR_NONFINITE if a
 * residual norm is not finite; IGA2L_ERR_DEVICE_TIMEOUT if a bounded device wait gave
 * up, u then holds unspecified values).  With CUDA graphs on (the default) and max_cycles
 * <= 1024 the cycles and their stopping test run on the device (one graph whose
 * WHILE node repeats cycle + check), and the call synchronises the stream twice
 * (initial residual, result); otherwise once per cycle.  Same results either way. */
int iga2l_solve(iga2l_handle h, const double *rhs, double tol, int max_cycles, double *u,
                int *cycles, double *relres, double *hist, void *stream);

/* iga2l_solve with the load vector b_p given directly (whatever options.rhs says): for
 * right-hand sides that are not a spline, e.g. b_p = (f, phi_i) of a closed-form f by
 * quadrature (Section 5.1).  Same arguments, results and errors otherwise. */
int iga2l_solve_load(iga2l_handle h, const double *b, double tol, int max_cycles, double *u,
                     int *cycles, double *relres, double *hist, void *stream);

/* Solve of A_p lambda = g with the transposed cycle (A_p is symmetric, so the
 * limit is A_p^{-1} g; the iterates are those of the adjoint iteration).  Always
 * FP64 (also on a mixed-precision handle). */
int iga2l_adjoint_solve(iga2l_handle h, const double *g, double tol, int max_cycles,
                        double *lambda, int *cycles, double *relres, void *stream);

/* b = (M(x)M) f (3D: M(x)M(x)M): load vector of f = sum_i f_i phi_i given by its
 * B-spline coefficients (b_p = (f, phi_i), Section 2). */
int iga2l_rhs_from_coeffs(iga2l_handle h, const double *f, double *b, void *stream);

/* ncycles cycles of Algorithm 1 in place, without residual checks (the forward
 * pass of an unrolled solve). */
int iga2l_cycles(iga2l_handle h, double *u, const double *b, int ncycles, void *stream);

/* Reverse pass of ncycles unrolled cycles u_k = u_{k-1} + C (b - A u_{k-1}): given
 * ubar = dL/du_K, writes bbar = dL/db = sum_k C^T (I - A C^T)^{K-k} ubar.  The cycle
 * is affine in u, so no forward states are needed; C^T is the transposed cycle
 * (iga2l_cycle_adjoint from zero).  FP64.  bbar: n^d device doubles (overwritten). */
int iga2l_unrolled_backward(iga2l_handle h, const double *ubar, int ncycles, double *bbar, void *stream);

/* Differentiable 2D source (not in the paper; a parametrised right-hand side for
 * gradient studies): f(x,y) = sum_k a_k exp(-((x-cx_k)^2 + (y-cy_k)^2) / (2 w^2)),
 * theta = device array of nbumps triples (a_k, cx_k, cy_k), 1 <= nbumps <= 64.
 * iga2l_bump_load writes b = (f, phi_ij) (p+3 Gauss points per element and axis).
 * iga2l_bump_grad writes grad = dL/dtheta (nbumps triples, device) given
 * bbar = dL/db.  Both are separable per bump and reduce in a fixed order. */
int iga2l_bump_load(iga2l_handle h, int nbumps, const double *theta, double width, double *b, void *stream);
int iga2l_bump_grad(iga2l_handle h, int nbumps, const double *theta, double width, const double *bbar,
                    double *grad, void *stream);

/* Host copies of the handle's 1D band tables, rows of width 2p+1 (entry a of
 * row i is the coefficient of DOF i + a - p), for tests: K then M, n*(2p+1) each. */
int iga2l_get_bands(iga2l_handle h, double *K, double *M);

/* Host-only helpers (no GPU needed), for checking the library's setup code:
 * the 1D band rows of the degree-p space with m elements (n*(2p+1) each, as in
 * iga2l_get_bands) and the dense 1D aggressive restriction (m/2-1) x n. */
int iga2l_host_bands(int p, int m, double *K, double *M);
int iga2l_host_restriction(int p, int m, double *R);

/* Defect and its squared norm for callers that cannot allocate device memory.
 * (The paper has no counterpart: this is a deployment aid.)  Some callers may
 * not call cudaMalloc at all -- code where the CUDA allocator is off limits, or
 * a host runtime that owns every device allocation and only lends out its own
 * buffers -- so they cannot create a handle (iga2l_assemble allocates).  This
 * entry point needs no handle and allocates nothing: it writes
 * d = b - A_p u (if d is not NULL) and *norm2 = ||d||_2^2, where A_p =
 * K(x)M + M(x)K is given by the caller's DEVICE copies of the 1D band rows Kb, Mb
 * (n x (2p+1) each, the layout of iga2l_host_bands / iga2l_get_bands; n = m+p-2).
 * u, b, d are device vectors of n*n doubles; norm2 is one device double.  All
 * buffers belong to the caller; work is enqueued on `stream`, nothing is
 * synchronised.  p must be 2..5 and n at most 4096 (IGA2L_ERR_INVALID_ARG with
 * a message in iga2l_last_error otherwise).
 * Its only scratch (one partial sum per thread block) is a fixed 512 KiB array
 * inside the library, held by every GPU that loads the library until the
 * process exits.  The first call on each device looks up that array's address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  Every call shares the array: each call overwrites the
 * partials it reads, so nothing has to be cleared, but calls that overlap on the
 * GPU (other streams, other threads) race on it.  The looked-up address belongs to
 * the device's current context: after cudaDeviceReset on a device it is stale, so this
 * entry point must not be called again on that device in the same process. */
int iga2l_residual_norm2_noalloc(int p, int n, const double *Kb, const double *Mb,
                                 const double *u, const double *b, double *d,
                                 double *norm2, void *stream);

/* Releases everything the handle owns (device tables and workspace, captured CUDA
 * graphs, its capture stream, pinned host buffers).  NULL is allowed.  The caller
 * makes sure no work of the handle is still running on the GPU. */
void iga2l_destroy(iga2l_handle h);
/* Static text of a return code (never NULL). */
const char *iga2l_strerror(int code);
/* Detail of the last error on the calling host thread ("" if none). */
const char *iga2l_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all handles and threads).  For benchmarks; no GPU work. */
long long iga2l_kernel_launches(void);

/* For tests: synchronises the device and counts, in *changed, the bytes of the guard zones
 * of a handle assembled with IGA2L_TEST_GUARD_ALLOCS that no longer hold their fill (0: no
 * kernel of the handle wrote outside its buffers).  IGA2L_ERR_INVALID_ARG for a handle built
 * without the flag or a null changed. */
int iga2l_guard_check(iga2l_handle h, long long *changed);

/* For benchmarks (not part of the solver): the throughput of one FMA pipe of the current
 * device in GFLOP/s (an FMA counts 2 flops), measured with dependent-free FMA loops over
 * every SM: kind 0 = FP64, 1 = FP32, 2 = packed FP32 pairs (one instruction, two FMAs).
 * These are the denominators of the ALU rooflines of the FP64 and FP32 kernels.
 * Allocates 16 bytes for the duration of the call and synchronises `stream`. */
int iga2l_fma_peak(int kind, double *gflops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* IGA2L_H */
