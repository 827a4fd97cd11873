// internal.h -- solver state shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/iga2l.h"

namespace iga2l {

constexpr int kMaxP = 8;       // degrees with compiled kernels: 2..8 (2D), 2..4 (3D)
constexpr int kMaxLevels = 24;
constexpr size_t kGuardBytes = 4096;   // IGA2L_TEST_GUARD_ALLOCS: zone before and after each buffer
// Side of the TILE schedule's tiles (block centres) compiled for degree p: a multiple
// of the default colour period, at least 2R + P + 1 so tiles of one phase never interact.
// The TILE kernel keeps a block in one warp, so it exists for blocks up to 5x5 (p <= 6).
constexpr int tile_side(int p) { return p == 2 || p == 5 ? 20 : (p == 6 ? 22 : (p <= 4 ? 21 : 0)); }
// Colour groups of the TILE order by default: degree 6 takes the LATTICE cycle counts with
// its 121 colours split into 4 groups (each group runs the four tile phases in turn); the
// other degrees use one group (p = 2, 3, 5 already match LATTICE; no grouping does for p = 4).
constexpr int tile_groups_default(int p) { return p == 6 ? 4 : 1; }
// 3D TILE side (3x3x3 blocks, p = 2..4): the default colour period, so a colour has one
// block per tile; at least 2R + P, so tiles of one phase never interact.
constexpr int tile_side3d(int p) { return p == 2 ? 5 : 7; }

// Batch addressing passed to 2D kernels: problem z of a batch owns vec (fine vector),
// aux (scratch) and crs (second-level vector) entries starting at z * stride; problems
// with active[z] == 0 are skipped (null: all active).  A single problem has nbatch = 1.
struct BatchRef {
    const int *active;
    long long vec, aux, crs;
};

// Host-side tables built once per handle (setup.cpp); uploaded by api.cu.
struct HostTables {
    int p = 0, m = 0, n = 0, s = 0, r = 0;
    // 1D band rows, n x (2p+1): entry a of row i couples DOF i with DOF i+a-p
    std::vector<double> Kb, Mb;
    // point classes of the residual stencil: rows closer than 2p-1 to a
    // boundary have their own class, the others share the Toeplitz row
    int npc = 0;                       // classes per axis (4p - 1)
    std::vector<int> pc_rep;           // representative row of each class
    // block classes of the Schwarz step: blocks touching the non-uniform
    // boundary functions have their own class
    int L = 0, nbc = 0;                // nbc = 2L + 1 classes per axis
    std::vector<int> bc_rep;           // representative centre of each class
    // aggressive restriction R = S^T D^{-1} M_p^1 as a row band and a column band
    int nc = 0, wr = 0, wc = 0;
    std::vector<double> Rb, Cb;        // nc x wr, n x wc
    std::vector<int> Rlo, Clo;
};

struct Level {                 // degree-1 level of the second-level hierarchy
    int m = 0, n = 0;          // elements, DOFs per axis
    long long N = 0;
    double k[3] = {0, 0, 0};   // 1D stiffness row  (-1, 2, -1)/H
    double mm[3] = {0, 0, 0};  // 1D mass row (1, 4, 1) H/6
    double *e = nullptr, *rhs = nullptr, *r = nullptr;   // device
    double *pre = nullptr;     // pre-smoothed correction (2D V-cycle)
};

// FP32 state of the inner cycle of the mixed-precision form (device pointers).
struct MixedState {
    bool enabled = false;
    float *stencil = nullptr, *binv = nullptr, *Rb = nullptr, *Cb = nullptr;
    float *Kb = nullptr, *Mb = nullptr;   // FP32 band rows (3D kernels)
    // IGA2L_MIXED_TF32: the interior block operator G = [A_B^-1 | -A_B^-1 A_(B,patch)] (rounded
    // to TF32) in the tensor-core operand layout, gtc_n x gtc_k (block DOFs x [b_B; u_patch])
    float *gtc = nullptr;
    int gtc_n = 0, gtc_k = 0;
    // IGA2L_MIXED_FP32 / TF32: the FP64 block inverses as unevaluated pairs binv + binv_lo
    // (binv_lo = fl32(B - binv)), for the compensated FP32 application in the TILE kernel
    float *binv_lo = nullptr;
    // TILE (2D): binv and binv_lo with each class's matrix transposed ([class][f][e]), so that
    // the lanes of a block, one per row e, read consecutive words
    float *binv_t = nullptr, *binv_lo_t = nullptr;
    float *r = nullptr;       // outer residual b - A u, computed in FP64, stored in FP32
    float *delta = nullptr;   // correction of the Schwarz step
    float *d = nullptr, *t = nullptr, *t2 = nullptr, *dc = nullptr, *ec = nullptr;
    std::vector<float *> lev_e, lev_rhs;   // level arrays (index 0 unused: dc / ec)
    std::vector<float *> lev_r;            // level residuals (3D)
    std::vector<float *> lev_pre;          // pre-smoothed corrections (2D)
};

struct Solver {
    int dim = 2, p = 2, m = 0, n = 0, s = 3, r = 1;
    long long N = 0;
    int nbatch = 1;              // problems sharing (p, m, options), stored [problem][...]
    int *active = nullptr;       // per-problem flag (device); null for a single problem
    double *bnorm0 = nullptr, *brel = nullptr;   // batch: initial norms^2, relative residuals
    int *bcycles = nullptr, *bcount = nullptr;   // batch: cycles per problem, active count
    iga2l_options opt{};
    int device = 0;
    int q = 5, g = 1, tile = 0;
    int tile_groups = 1;         // TILE: colour groups (each runs the four tile phases)
    int nsm = 1;                 // SMs of the device (launch balancing)
    HostTables ht;
    // device tables
    double *Kb = nullptr, *Mb = nullptr;
    double *stencil = nullptr;   // npc^dim classes x (2p+1)^dim coefficients
    double *binv = nullptr;      // nbc^dim classes x S*S, S = s^dim
    double *binv_t = nullptr;    // binv with each class transposed ([class][f][e]): TILE and 3D kernels
    int *pcls = nullptr;         // point class of every row index (n)
    int *bcls = nullptr;         // block class of every centre index (n)
    double *Rb = nullptr, *Cb = nullptr;
    int *Rlo = nullptr, *Clo = nullptr;
    int *Mlo = nullptr;          // row starts i - p of the mass band (3D mass apply)
    int nc = 0;
    long long Nc = 0;
    std::vector<Level> lev;      // lev[0] is the second level (nc per axis)
    int ndirect = 0;             // size of the directly solved level
    double *dinv = nullptr;      // dense inverse of the direct level
    // workspace
    double *d = nullptr, *t = nullptr, *dc = nullptr, *ec = nullptr, *t2 = nullptr;
    double *part = nullptr;      // per-CTA partial sums of squares
    unsigned int *rcount = nullptr;   // per problem: residual CTAs done (fused norm), re-armed to 0
    int npart = 0;
    double *bwork = nullptr;     // scratch of the 3D mass apply
    double *rhsb = nullptr;      // b = (M (x) M) f of a solve given the coefficients f
    MixedState mx;
    // differentiable source (2D): 1D quadrature tables, nq = p+3 points per element
    int nq = 0;
    double *qx = nullptr, *qw = nullptr, *qB = nullptr;
    double *adj1 = nullptr, *adj2 = nullptr, *adj3 = nullptr;   // backward workspace (N each)
    double *gbuf = nullptr;      // per-bump 1D loads and their centre derivatives
    int gcap = 0;                // bumps gbuf can hold
    unsigned int *progress = nullptr;   // persistent sweep: colours finished per CTA
    unsigned int *tile_ctr = nullptr;   // work-list TILE sweep: item counter + finished occurrences
                                        // per (problem, tile position); null: one launch per phase
    int tile_work_ctas = 0;             // work-list TILE sweep: resident CTAs (its grid)
    int *wait_status = nullptr;         // device: bounded waits that gave up (tensor-core, persistent)
    int pgx = 0, pgy = 0, prx = 0, pry = 0;   // persistent sweep: regions per axis, largest sides
    unsigned psmem = 0;                       // (pgx = 0: per-colour launches)
    std::vector<void *> allocs;
    // IGA2L_TEST_GUARD_ALLOCS: bytes of the zone before and after every device buffer, and
    // (buffer, size in bytes, fill byte) of each guarded buffer
    size_t guard_bytes = 0;
    struct Guarded { char *p; size_t bytes; unsigned char fill; };
    std::vector<Guarded> guarded;
    // FP64 inverses of the boundary block classes for the FP32 Schwarz kernels, or null
    // when those are applied in FP32 too (IGA2L_MIXED_FP32_ALL)
    const double *boundary64() const
    {
        return opt.precision == IGA2L_MIXED_FP32 || opt.precision == IGA2L_MIXED_TF32 ? binv : nullptr;
    }
    // the same, transposed per class (the 3D kernels)
    const double *boundary64_t() const
    {
        return opt.precision == IGA2L_MIXED_FP32 || opt.precision == IGA2L_MIXED_TF32 ? binv_t : nullptr;
    }
    // the low halves of the FP32 pairs of those inverses, or null likewise
    const float *boundary_lo() const
    {
        return opt.precision == IGA2L_MIXED_FP32 || opt.precision == IGA2L_MIXED_TF32 ? mx.binv_lo : nullptr;
    }
    // the same, transposed per class (the TILE kernels)
    const float *boundary_lo_t() const
    {
        return opt.precision == IGA2L_MIXED_FP32 || opt.precision == IGA2L_MIXED_TF32 ? mx.binv_lo_t : nullptr;
    }
};

// Control block of a device-driven solve (one WHILE graph node runs the cycles): written
// by the host before the launch, updated by the convergence check after every cycle.
struct SolveCtl {
    double r0;     // ||b - A u_0||
    double tol;    // relative residual to reach
    double rel;    // out: last relative residual
    int maxc;      // cycle cap
    int k;         // out: cycles done (0 on entry)
    int status;    // out: 1 converged, 2 non-finite norm, 0 cycle cap reached
};
constexpr int kSolveHistCap = 1024;   // device-driven solves: at most this many cycles

// Number of kernels this library has launched (process-wide), for benchmarks
// that report how many of the timed region's kernels are this library's.
void count_launches(long long k);
long long launches_so_far();

#ifdef __CUDACC__
// Programmatic dependent launch.  The kernels of a cycle are launched with the
// programmatic-serialisation attribute; each reads only constant tables before
// pdl_wait(), which returns once the previous grid has completed and its writes are
// visible, so that part overlaps the previous kernel's completion.  Every thread calls
// pdl_wait() before it exits, so a grid's completion implies its predecessors'.  No kernel
// triggers its dependents early (griddepcontrol.launch_dependents): with early triggers
// the p = 4 FP64 sweep measured 35% slower and four concurrent mixed solves 30% slower
// (the next grid's waiting CTAs are placed on whichever SMs drain first, which likely
// spreads a single-wave colour phase unevenly, and they hold slots other streams need).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename Kernel, typename... Args>
cudaError_t launch_pdl_smem(Kernel kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename Kernel, typename... Args>
cudaError_t launch_pdl(Kernel kernel, dim3 grid, dim3 block, cudaStream_t st, Args... args)
{
    return launch_pdl_smem(kernel, grid, block, 0, st, args...);
}
#endif

// Sets the text returned by iga2l_last_error on the calling thread (api.cu).
void set_last_error(const std::string &msg);

// After a cycle of a device-driven solve: count it, record rel = sqrt(norm2) / r0 in
// hist, and set the WHILE node's condition to 0 once rel <= tol, the norm is not
// finite or maxc cycles are done (kernels_fine.cu).
cudaError_t launch_solve_check(const double *norm2, SolveCtl *ctl, double *hist, cudaGraphConditionalHandle cond,
                               cudaStream_t st);

// setup.cpp
int build_host_tables(int p, int m, int s, HostTables &ht, std::string &err);
void bspline_band_1d(int p, int m, std::vector<double> &K, std::vector<double> &M);
bool cholesky_inverse(int N, std::vector<double> &A);   // in place, SPD
void quadrature_tables(int p, int m, int nq, std::vector<double> &x, std::vector<double> &w,
                       std::vector<double> &B);
int default_block_side(int p);
void default_colouring(int p, int s, int &q, int &g);

// kernels (kernels_fine.cu, kernels_coarse.cu); all enqueue on `st`
cudaError_t launch_residual(const Solver &S, const double *u, const double *b, double *d,
                            double *part, cudaStream_t st);
cudaError_t launch_apply_A(const Solver &S, const double *u, double *y, cudaStream_t st);
cudaError_t launch_norm_finish(const Solver &S, const double *part, double *out, cudaStream_t st);
// residual with its squared norm finished in the same launch (2D) into norm2[problem]
cudaError_t launch_residual_norm(const Solver &S, const double *u, const double *b, double *d, double *norm2,
                                 cudaStream_t st);
cudaError_t launch_outer_residual_norm(const Solver &S, const double *u, const double *b, float *r32,
                                       double *norm2, cudaStream_t st);
cudaError_t launch_schwarz(const Solver &S, double *u, const double *b, bool reverse,
                           cudaStream_t st);
cudaError_t launch_restrict(const Solver &S, const double *d, double *dc, cudaStream_t st);
cudaError_t launch_prolong_add(const Solver &S, const double *ec, double *u, cudaStream_t st);
cudaError_t launch_coarse_solve(const Solver &S, const double *dc, double *ec, cudaStream_t st);
cudaError_t launch_mass2(const Solver &S, const double *f, double *b, cudaStream_t st);
// mixed precision: FP64 outer residual stored in FP32; FP32 inner cycle on A delta = r
// from delta = 0 (fine part, second level, then u += delta + P e_c in FP64)
cudaError_t launch_outer_residual(const Solver &S, const double *u, const double *b, float *r32,
                                  double *part, cudaStream_t st);
cudaError_t launch_inner_fine(const Solver &S, const float *r32, bool reverse, cudaStream_t st);
cudaError_t launch_inner_coarse(const Solver &S, cudaStream_t st);
cudaError_t launch_inner_update(const Solver &S, double *u, cudaStream_t st);
// the FP32 Schwarz step of the inner cycle on caller vectors (2D)
cudaError_t launch_inner_sweep(const Solver &S, float *u, const float *b, bool reverse, cudaStream_t st);
int residual_partials(const Solver &S);
cudaError_t launch_batch_init(const Solver &S, const double *norm2, double *norm0, int *cycles, double *relres,
                              cudaStream_t st);
cudaError_t launch_batch_check(const Solver &S, double tol, const double *norm2, const double *norm0, int *cycles,
                               double *relres, int *count, cudaStream_t st);
// the same inside a device-driven batched solve: tol from ctl, ctl->k counted, and the
// WHILE condition set to continue while a problem is active and fewer than maxc cycles ran
cudaError_t launch_batch_check_loop(const Solver &S, const double *norm2, const double *norm0, int *cycles,
                                    double *relres, int *count, SolveCtl *ctl, cudaGraphConditionalHandle cond,
                                    cudaStream_t st);
// differentiable source (kernels_grad.cu)
constexpr int kMaxBumps = 64;
cudaError_t launch_bump_load(const Solver &S, int nb, const double *theta, double w, double *b, cudaStream_t st);
cudaError_t launch_bump_grad(const Solver &S, int nb, const double *theta, double w, const double *bbar,
                             double *grad, cudaStream_t st);
cudaError_t launch_axpy(long long n, double alpha, const double *x, double *y, cudaStream_t st);

// 3D (kernels_3d.cu)
int residual3d_partials(const Solver &S);
cudaError_t launch3d_residual(const Solver &S, const double *u, const double *b, double *d, double *part,
                              cudaStream_t st);
cudaError_t launch3d_schwarz(const Solver &S, double *u, const double *b, bool reverse, cudaStream_t st);
cudaError_t launch3d_restrict(const Solver &S, const double *d, double *dc, cudaStream_t st);
cudaError_t launch3d_prolong_add(const Solver &S, const double *ec, double *u, cudaStream_t st);
cudaError_t launch3d_coarse_solve(const Solver &S, const double *dc, double *ec, cudaStream_t st);
cudaError_t launch3d_mass(const Solver &S, const double *f, double *b, cudaStream_t st);
cudaError_t launch3d_outer_residual(const Solver &S, const double *u, const double *b, float *r32, double *part,
                                    cudaStream_t st);
cudaError_t launch3d_inner_fine(const Solver &S, const float *r32, cudaStream_t st);
cudaError_t launch3d_inner_coarse(const Solver &S, cudaStream_t st);
cudaError_t launch3d_inner_update(const Solver &S, double *u, cudaStream_t st);
// tensor-core Schwarz (kernels_tc.cu): the colour's block-index range [i0, i0 + ni) along one
// axis whose blocks (and their patches) see only interior rows
void tc_interior_rect(const Solver &S, int o, int nb, int &i0, int &ni);
// checks that the tensor-core colour step's shared memory (set by the lattice period q) fits
// the device and allows it for the kernel (kernels_fine.cu); false: not available
bool tc_colour_prepare(const Solver &S, std::string &why);
// resident CTAs of the work-list TILE sweep for this handle's degree and precision (0: none)
int tile_work_ctas(const Solver &S);
// persistent LATTICE sweep of the FP32 inner cycle (kernels_persist.cu): plans the launch
// (false: not available for this handle, per-colour launches are used) and runs one sweep
bool persist_setup(Solver &S);
cudaError_t launch_schwarz_persist(const Solver &S, float *u, const float *b, bool reverse, cudaStream_t st);
cudaError_t upload_persist_rows(int p, const double *k1, const double *m1);
// the same rows (as FP32 pairs (k, m)) for the 3D FP32 colour kernel, degrees 2..4
cudaError_t upload_rows3d(int p, const double *k1, const double *m1);
// host: G of the interior block in the operand layout (kernels_tc.cu)
void build_gtc(const Solver &S, const std::vector<double> &binv_interior, std::vector<float> &g, int &nrows,
               int &kcols);
constexpr int kTcMaxP = 5;

// The interior 1D rows k = h K_row, m = M_row / h of degree p (h-independent) into
// constant memory; written once per device and degree.
cudaError_t upload_interior_rows(int p, const double *k1, const double *m1);

}  // namespace iga2l
