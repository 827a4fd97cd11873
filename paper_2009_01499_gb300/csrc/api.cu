// api.cu -- the C ABI of include/iga2l.h: handle construction, table upload,
// per-step entry points, Algorithm 1 and the solver loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

using namespace iga2l;

namespace iga2l {
static std::atomic<long long> g_launches{0};
// kernels enqueued while a cycle is being captured into a graph are counted when the
// graph is launched, not when they are recorded
static thread_local bool g_capturing = false;
void count_launches(long long k)
{
    if (!g_capturing) g_launches.fetch_add(k, std::memory_order_relaxed);
}
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace iga2l

struct iga2l_solver : public Solver {
    double *host_norm = nullptr;   // pinned scalar for norm readback
    double *dev_norm = nullptr;
    // Cycles are captured once per (u, b, kind) into CUDA graphs and replayed: one
    // graph launch instead of ~100 small kernel launches per cycle.
    struct CycleGraph {
        const double *u, *b;
        int kind;                  // bit 0: adjoint, bit 1: ends with the residual norm, bit 2: mixed
        cudaGraphExec_t exec;
        long long kernels;
        unsigned long long last_use;
    };
    std::vector<CycleGraph> graphs;
    unsigned long long tick = 0;
    cudaStream_t cap_stream = nullptr;
    // Device-driven solves: per (u, b, kind) one graph whose WHILE node repeats the cycle
    // and its convergence check until the check stops it; 4 most recently used kept.
    struct SolveGraph {
        const double *u, *b;
        int kind;
        cudaGraphExec_t exec;
        long long kernels_per_cycle;
        unsigned long long last_use;
    };
    std::vector<SolveGraph> solve_graphs;
    bool solve_graph_failed = false;   // the driver refused one: use the host-driven loop
    bool cycle_graph_failed = false;   // the driver refused to capture a cycle: plain launches
    SolveCtl *ctl = nullptr, *ctl_host = nullptr;   // device / pinned host copy
    double *dev_hist = nullptr, *host_hist = nullptr;
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(IGA2L_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Every device buffer of a handle comes from here.  Under IGA2L_TEST_GUARD_ALLOCS it sits
// between two zones of guard_bytes bytes: all-ones (a NaN in FP32 and FP64) around
// floating-point buffers, so that a kernel reading past either end meets a NaN that reaches
// its results, and zeros around integer tables and counters, so that a stray read there
// still yields an in-range index; a stray write changes a zone (iga2l_guard_check).  The
// zones are a multiple of 256 bytes, so every buffer keeps cudaMalloc's alignment.
cudaError_t dmalloc(iga2l_solver *S, void **out, size_t bytes, bool floating)
{
    if (bytes == 0) bytes = 1;
    const size_t G = S->guard_bytes;
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes + 2 * G);
    if (e != cudaSuccess) return e;
    S->allocs.push_back(base);
    char *p = static_cast<char *>(base) + G;
    if (G) {
        const unsigned char fill = floating ? 0xFF : 0x00;
        if ((e = cudaMemset(base, fill, G)) != cudaSuccess || (e = cudaMemset(p + bytes, fill, G)) != cudaSuccess)
            return e;
        S->guarded.push_back({p, bytes, fill});
    }
    *out = p;
    return cudaSuccess;
}

template <typename T>
cudaError_t upload(iga2l_solver *S, T **dst, const std::vector<T> &src)
{
    void *p = nullptr;
    cudaError_t e = dmalloc(S, &p, sizeof(T) * src.size(), std::is_floating_point<T>::value);
    if (e != cudaSuccess) return e;
    *dst = static_cast<T *>(p);
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

template <typename T>
cudaError_t alloc(iga2l_solver *S, T **dst, size_t count)
{
    void *p = nullptr;
    cudaError_t e = dmalloc(S, &p, sizeof(T) * count, std::is_floating_point<T>::value);
    if (e == cudaSuccess) *dst = static_cast<T *>(p);
    return e;
}

void release(iga2l_solver *S)
{
    if (!S) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != S->device) cudaSetDevice(S->device);
    for (auto &g : S->graphs) cudaGraphExecDestroy(g.exec);
    S->graphs.clear();
    for (auto &g : S->solve_graphs) cudaGraphExecDestroy(g.exec);
    S->solve_graphs.clear();
    if (S->ctl_host) cudaFreeHost(S->ctl_host);
    if (S->host_hist) cudaFreeHost(S->host_hist);
    if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
    for (void *p : S->allocs) cudaFree(p);
    S->allocs.clear();
    if (S->host_norm) cudaFreeHost(S->host_norm);
    if (cur >= 0 && cur != S->device) cudaSetDevice(cur);
    delete S;
}

int gcd_int(int a, int b)
{
    while (b) { int t = a % b; a = b; b = t; }
    return a;
}

// Kronecker-structured entry A[(x1,y1)][(x2,y2)] from the band rows.
double band(const std::vector<double> &B, int p, int i, int j)
{
    const int off = j - i;
    if (off < -p || off > p) return 0.0;
    return B[(size_t)i * (2 * p + 1) + off + p];
}

int check_handle(iga2l_handle h)
{
    if (!h) return fail(IGA2L_ERR_INVALID_ARG, "null handle");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(IGA2L_ERR_CUDA, "cudaGetDevice failed");
    if (cur != h->device) {
        cudaError_t e = cudaSetDevice(h->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    }
    return IGA2L_OK;
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

int finish(cudaError_t e, const char *where)
{
    if (e != cudaSuccess) return cuda_fail(e, where);
    return IGA2L_OK;
}

// ||b - A u||_2^2 (or ||A u||^2 when b is null) into h->host_norm; synchronises.
int residual_norm2(iga2l_handle h, const double *u, const double *b, double *d, cudaStream_t st,
                   double *out)
{
    cudaError_t e = launch_residual_norm(*h, u, b, d, h->dev_norm, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->host_norm, h->dev_norm, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "residual norm");
    *out = *h->host_norm;
    return IGA2L_OK;
}

int coarse_correction(iga2l_handle h, double *u, const double *b, cudaStream_t st)
{
    cudaError_t e = launch_residual(*h, u, b, h->d, nullptr, st);
    if (e == cudaSuccess) e = launch_restrict(*h, h->d, h->dc, st);
    if (e == cudaSuccess) e = launch_coarse_solve(*h, h->dc, h->ec, st);
    if (e == cudaSuccess) e = launch_prolong_add(*h, h->ec, u, st);
    return finish(e, "coarse correction");
}

// Enqueues one cycle (optionally followed by the residual norm into host_norm).
// Mixed precision (forward cycles only): the FP32 inner cycle on A delta = r from
// delta = 0, then u += delta in FP64, then the FP64 residual r = b - A u (stored in
// FP32 for the next inner cycle) -- r must already hold b - A u on entry.
int enqueue_cycle(iga2l_handle h, double *u, const double *b, cudaStream_t st, bool adjoint, bool norm,
                  bool host_copy = true)
{
    int rc;
    if (h->mx.enabled && !adjoint) {
        cudaError_t e = launch_inner_fine(*h, h->mx.r, false, st);
        if (e == cudaSuccess) e = launch_inner_coarse(*h, st);
        if (e == cudaSuccess) e = launch_inner_update(*h, u, st);
        if (e == cudaSuccess)
            e = norm ? launch_outer_residual_norm(*h, u, b, h->mx.r, h->dev_norm, st)
                     : launch_outer_residual(*h, u, b, h->mx.r, nullptr, st);
        if (e == cudaSuccess && norm && host_copy && !h->active)
            e = cudaMemcpyAsync(h->host_norm, h->dev_norm, sizeof(double), cudaMemcpyDeviceToHost, st);
        return finish(e, "mixed-precision cycle");
    }
    if (!adjoint) {
        cudaError_t e = launch_schwarz(*h, u, b, false, st);
        if (e != cudaSuccess) return cuda_fail(e, "schwarz sweep");
        if ((rc = coarse_correction(h, u, b, st)) != IGA2L_OK) return rc;
    } else {
        if ((rc = coarse_correction(h, u, b, st)) != IGA2L_OK) return rc;
        cudaError_t e = launch_schwarz(*h, u, b, true, st);
        if (e != cudaSuccess) return cuda_fail(e, "reverse schwarz sweep");
    }
    if (norm) {
        cudaError_t e = launch_residual_norm(*h, u, b, nullptr, h->dev_norm, st);
        if (e == cudaSuccess && host_copy && !h->active)
            e = cudaMemcpyAsync(h->host_norm, h->dev_norm, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "residual norm");
    }
    return IGA2L_OK;
}

// One cycle on `st`: replays a captured graph for (u, b, kind), capturing it first if needed.
int run_cycle_graph(iga2l_handle h, double *u, const double *b, cudaStream_t st, bool adjoint, bool norm)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!h->opt.graphs || h->cycle_graph_failed || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
        return enqueue_cycle(h, u, b, st, adjoint, norm);   // plain launches (or the caller is capturing)
    const int kind = (adjoint ? 1 : 0) | (norm ? 2 : 0) | (h->mx.enabled ? 4 : 0);
    iga2l_solver::CycleGraph *g = nullptr;
    for (auto &c : h->graphs)
        if (c.u == u && c.b == b && c.kind == kind) g = &c;
    if (!g) {
        cudaError_t e;
        if (!h->cap_stream && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "capture stream");
        if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "begin capture");
        g_capturing = true;
        int rc = enqueue_cycle(h, u, b, h->cap_stream, adjoint, norm);
        g_capturing = false;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (rc != IGA2L_OK || e != cudaSuccess) {
            // the driver refused to capture one of the cycle's launches: plain launches from now on
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            h->cycle_graph_failed = true;
            return enqueue_cycle(h, u, b, st, adjoint, norm);
        }
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        long long kernels = 0;
        if (nn && cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
            }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        if (h->graphs.size() >= 4) {   // keep the four most recently used
            auto lru = std::min_element(h->graphs.begin(), h->graphs.end(),
                                        [](const auto &x, const auto &y) { return x.last_use < y.last_use; });
            cudaGraphExecDestroy(lru->exec);
            h->graphs.erase(lru);
        }
        h->graphs.push_back({u, b, kind, exec, kernels, 0});
        g = &h->graphs.back();
    }
    g->last_use = ++h->tick;
    cudaError_t e = cudaGraphLaunch(g->exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    count_launches(g->kernels);
    return IGA2L_OK;
}

int run_cycle(iga2l_handle h, double *u, const double *b, cudaStream_t st, bool adjoint)
{
    if (h->mx.enabled && !adjoint) {   // the inner cycle starts from r = b - A u
        cudaError_t e = launch_outer_residual(*h, u, b, h->mx.r, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "outer residual");
    }
    return run_cycle_graph(h, u, b, st, adjoint, false);
}

// The graph of a device-driven solve for (u, b, kind): a WHILE node whose body is one
// cycle, its residual norm and k_solve_check.  Returns null (and remembers it) when the
// driver refuses to build it; the caller then drives the cycles from the host.
iga2l_solver::SolveGraph *solve_graph(iga2l_handle h, double *u, const double *b, bool adjoint)
{
    const bool batch = h->active != nullptr;   // batch handles: k_batch_check stops the loop
    const int kind = (adjoint ? 1 : 0) | (h->mx.enabled ? 4 : 0) | (batch ? 8 : 0);
    for (auto &c : h->solve_graphs)
        if (c.u == u && c.b == b && c.kind == kind) return &c;
    cudaError_t e = cudaSuccess;
    if (!h->cap_stream && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return nullptr;
    cudaGraph_t graph = nullptr, body = nullptr;
    cudaGraphConditionalHandle cond;
    cudaGraphNode_t node;
    cudaGraphNodeParams np = {};
    bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess;
    }
    if (ok) {
        body = np.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            g_capturing = true;
            int rc = enqueue_cycle(h, u, b, h->cap_stream, adjoint, true, false);
            if (rc == IGA2L_OK &&
                (batch ? launch_batch_check_loop(*h, h->dev_norm, h->bnorm0, h->bcycles, h->brel, h->bcount, h->ctl,
                                                 cond, h->cap_stream)
                       : launch_solve_check(h->dev_norm, h->ctl, h->dev_hist, cond, h->cap_stream)) != cudaSuccess)
                rc = IGA2L_ERR_CUDA;
            g_capturing = false;
            cudaGraph_t captured = nullptr;
            ok = cudaStreamEndCapture(h->cap_stream, &captured) == cudaSuccess && rc == IGA2L_OK;
        }
    }
    long long kernels = 0;
    if (ok) {
        size_t nn = 0;
        cudaGraphGetNodes(body, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn && cudaGraphGetNodes(body, nodes.data(), &nn) == cudaSuccess)
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
            }
    }
    cudaGraphExec_t exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();   // a refused build leaves no sticky error
    if (!ok) {
        h->solve_graph_failed = true;
        return nullptr;
    }
    if (h->solve_graphs.size() >= 4) {
        auto lru = std::min_element(h->solve_graphs.begin(), h->solve_graphs.end(),
                                    [](const auto &x, const auto &y) { return x.last_use < y.last_use; });
        cudaGraphExecDestroy(lru->exec);
        h->solve_graphs.erase(lru);
    }
    h->solve_graphs.push_back({u, b, kind, exec, kernels, 0});
    return &h->solve_graphs.back();
}

// b_p = (f, phi_i) of a source given by its B-spline coefficients f (Section 2), into the
// handle's right-hand-side buffer (every problem of a batch)
// every ss x ss class matrix of a [class][e][f] table transposed to [class][f][e]
std::vector<double> transpose_classes(const std::vector<double> &m, int ss)
{
    std::vector<double> t(m.size());
    const size_t sq = (size_t)ss * ss;
    for (size_t c = 0; c + sq <= m.size(); c += sq)
        for (int e = 0; e < ss; ++e)
            for (int f = 0; f < ss; ++f) t[c + (size_t)f * ss + e] = m[c + (size_t)e * ss + f];
    return t;
}

int load_from_coeffs(iga2l_handle h, const double *f, const double *u, cudaStream_t st)
{
    if (!f || !u) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    if (f == h->rhsb) return fail(IGA2L_ERR_INVALID_ARG, "aliased vector");
    return finish(launch_mass2(*h, f, h->rhsb, st), "right-hand side from coefficients");
}

// IGA2L_ERR_DEVICE_TIMEOUT (and the flag cleared) when a bounded device wait gave up since the
// last check: blocks or tiles were left uncorrected
int wait_status_check(iga2l_handle h, cudaStream_t st)
{
    if (!h->wait_status) return IGA2L_OK;
    int bad = 0;
    cudaError_t e = cudaMemcpyAsync(&bad, h->wait_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "wait status");
    if (!bad) return IGA2L_OK;
    e = cudaMemsetAsync(h->wait_status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "wait status");
    return fail(IGA2L_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up (the results are not valid)");
}

int solve_impl(iga2l_handle h, const double *b, double tol, int max_cycles, double *u, int *cycles,
               double *relres, double *hist, void *stream, bool adjoint)
{
    if (!b || !u) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    if (!(tol >= 0.0)) return fail(IGA2L_ERR_INVALID_ARG, "tol must be >= 0");
    if (max_cycles <= 0) max_cycles = h->opt.max_cycles;
    cudaStream_t st = as_stream(stream);
    double r0sq = 0.0;
    int rc;
    if (h->mx.enabled && !adjoint) {   // r_0 in FP64, kept in FP32 for the first inner cycle
        cudaError_t e = launch_outer_residual_norm(*h, u, b, h->mx.r, h->dev_norm, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->host_norm, h->dev_norm, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "initial residual");
        r0sq = *h->host_norm;
    } else if ((rc = residual_norm2(h, u, b, nullptr, st, &r0sq)) != IGA2L_OK) {
        return rc;
    }
    if (!std::isfinite(r0sq)) return fail(IGA2L_ERR_NONFINITE, "initial residual is not finite");
    const double r0 = std::sqrt(r0sq);
    int k = 0;
    double rel = 0.0;
    int status = r0 == 0.0 ? IGA2L_OK : IGA2L_NOT_CONVERGED;
    // Device-driven: one graph launch runs every cycle and its check on the GPU (no host
    // round trip between cycles); one read-back at the end.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    iga2l_solver::SolveGraph *sg = nullptr;
    if (status != IGA2L_OK && h->opt.graphs && !h->solve_graph_failed && max_cycles <= kSolveHistCap &&
        cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
        sg = solve_graph(h, u, b, adjoint);
    if (sg) {
        *h->ctl_host = SolveCtl{r0, tol, 0.0, max_cycles, 0, -1};
        cudaError_t e = cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(SolveCtl), cudaMemcpyHostToDevice, st);
        sg->last_use = ++h->tick;
        if (e == cudaSuccess) e = cudaGraphLaunch(sg->exec, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && hist)
            e = cudaMemcpyAsync(h->host_hist, h->dev_hist, sizeof(double) * max_cycles, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "solve");
        const SolveCtl c = *h->ctl_host;
        k = c.k;
        count_launches(sg->kernels_per_cycle * k);
        if (hist)
            for (int i = 0; i < k; ++i) hist[i] = h->host_hist[i];
        if (c.status == 2) {
            if (cycles) *cycles = k;
            return fail(IGA2L_ERR_NONFINITE, "residual norm is not finite");
        }
        rel = c.rel;
        status = c.status == 1 ? IGA2L_OK : IGA2L_NOT_CONVERGED;
    }
    while (!sg && status != IGA2L_OK && k < max_cycles) {
        // one cycle and its residual norm, read back once per cycle
        rc = run_cycle_graph(h, u, b, st, adjoint, true);
        if (rc != IGA2L_OK) return rc;
        ++k;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "solve");
        const double rsq = *h->host_norm;
        if (!std::isfinite(rsq)) {
            if (cycles) *cycles = k;
            return fail(IGA2L_ERR_NONFINITE, "residual norm is not finite");
        }
        rel = std::sqrt(rsq) / r0;
        if (hist) hist[k - 1] = rel;
        if (rel <= tol) status = IGA2L_OK;
    }
    if (cycles) *cycles = k;
    if (relres) *relres = rel;
    if (status != IGA2L_OK) g_last_error = "cycle cap reached";
    if ((rc = wait_status_check(h, st)) != IGA2L_OK) return rc;
    return status;
}

}  // namespace

void iga2l::set_last_error(const std::string &msg) { g_last_error = msg; }

extern "C" {

void iga2l_default_options(iga2l_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = IGA2L_FP64;
    opt->schedule = IGA2L_SCHED_LATTICE;
    opt->coarse = IGA2L_COARSE_VCYCLE;
    opt->max_cycles = 100;
    opt->graphs = 1;
    opt->rhs = IGA2L_RHS_COEFFS;
    opt->sweep = IGA2L_SWEEP_AUTO;
    opt->test_flags = 0;
    opt->wait_budget_cycles = 0;
}

}  // extern "C"

static int assemble_impl(int p, int m, int dim, int nbatch, bool batch, const iga2l_options *opt_in, iga2l_handle *out)
{
    if (!out) return fail(IGA2L_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    iga2l_options opt;
    if (opt_in) opt = *opt_in; else iga2l_default_options(&opt);
    if (opt.max_cycles <= 0) opt.max_cycles = 100;
    if (dim != 2 && dim != 3) return fail(IGA2L_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (p < 2 || p > kMaxP) return fail(IGA2L_ERR_INVALID_ARG, "p must be in 2..8");
    if (dim == 3 && p > 4) return fail(IGA2L_ERR_UNSUPPORTED, "3D kernels are compiled for p = 2..4");
    // 2D: the boundary row and block classes need n = m + p - 2 >= 2p - 1 DOFs per axis and
    // the aggressive 2h level m >= 4, so grids down to every block being a boundary block
    // are accepted.  The 3D kernels, the tensor-core form and the persistent sweep are built
    // for grids with interior blocks and rows: m >= 4p + 4.
    const bool has_interior = m >= 4 * p + 4;
    if ((m % 2) != 0 || m < 4 || m < p + 1)
        return fail(IGA2L_ERR_INVALID_ARG, "m must be even, >= 4 and >= p + 1");
    if (dim == 3 && !has_interior) return fail(IGA2L_ERR_INVALID_ARG, "3D: m must be even and >= 4p+4");
    if (opt.precision != IGA2L_FP64 && opt.precision != IGA2L_MIXED_FP32 && opt.precision != IGA2L_MIXED_FP32_ALL &&
        opt.precision != IGA2L_MIXED_TF32)
        return fail(IGA2L_ERR_UNSUPPORTED, "precision not available");
    if (opt.precision == IGA2L_MIXED_TF32 &&
        (dim != 2 || batch || opt.schedule != IGA2L_SCHED_LATTICE || p > kTcMaxP || !has_interior))
        return fail(IGA2L_ERR_UNSUPPORTED,
                    "the tensor-core form is compiled for single 2D problems, LATTICE, p <= 5, m >= 4p+4");
    if (opt.schedule != IGA2L_SCHED_LATTICE && opt.schedule != IGA2L_SCHED_TILE)
        return fail(IGA2L_ERR_UNSUPPORTED, "schedule not available");
    if (dim == 3 && opt.schedule == IGA2L_SCHED_TILE) {
        if (opt.tile == 0) opt.tile = tile_side3d(p);
        if (opt.tile != tile_side3d(p)) return fail(IGA2L_ERR_UNSUPPORTED, "3D TILE side not compiled for this degree");
    } else if (opt.schedule == IGA2L_SCHED_TILE) {
        if (opt.tile == 0) opt.tile = tile_side(p);
        if (tile_side(p) == 0) return fail(IGA2L_ERR_UNSUPPORTED, "the TILE schedule is compiled for p <= 6");
        if (opt.tile != tile_side(p)) return fail(IGA2L_ERR_UNSUPPORTED, "TILE side not compiled for this degree");
    }
    if (opt.coarse != IGA2L_COARSE_VCYCLE && opt.coarse != IGA2L_COARSE_EXACT)
        return fail(IGA2L_ERR_INVALID_ARG, "unknown coarse solver");
    if (opt.tile_groups < 0 || opt.tile_groups > 1024) return fail(IGA2L_ERR_INVALID_ARG, "tile_groups must be 0..1024");
    if (opt.sweep != IGA2L_SWEEP_AUTO && opt.sweep != IGA2L_SWEEP_PER_COLOUR && opt.sweep != IGA2L_SWEEP_PERSISTENT &&
        opt.sweep != IGA2L_SWEEP_WORK_LIST)
        return fail(IGA2L_ERR_INVALID_ARG, "unknown sweep kernel choice");
    if (opt.sweep == IGA2L_SWEEP_WORK_LIST && (dim != 2 || opt.schedule != IGA2L_SCHED_TILE))
        return fail(IGA2L_ERR_UNSUPPORTED, "the work-list sweep runs the 2D TILE schedule");
    if (opt.sweep == IGA2L_SWEEP_PERSISTENT && !has_interior)
        return fail(IGA2L_ERR_UNSUPPORTED, "the persistent sweep needs m >= 4p+4");
    if (opt.rhs != IGA2L_RHS_COEFFS && opt.rhs != IGA2L_RHS_IS_LOAD)
        return fail(IGA2L_ERR_INVALID_ARG, "rhs must be IGA2L_RHS_COEFFS or IGA2L_RHS_IS_LOAD");
    if (opt.test_flags & ~(IGA2L_TEST_SKIP_OPERATOR_COPY | IGA2L_TEST_WITHHOLD_PROGRESS | IGA2L_TEST_GUARD_ALLOCS))
        return fail(IGA2L_ERR_INVALID_ARG, "unknown test flag");
    if (opt.wait_budget_cycles < 0) return fail(IGA2L_ERR_INVALID_ARG, "wait_budget_cycles must be >= 0");
    if (opt.wait_budget_cycles == 0) opt.wait_budget_cycles = 1LL << 31;
    const int s = opt.block_side > 0 ? opt.block_side : default_block_side(p);
    if (!((s == 3 && p <= 4) || (s == 5 && (p == 5 || p == 6)) || (s == 7 && (p == 7 || p == 8))))
        return fail(IGA2L_ERR_UNSUPPORTED, "block side not compiled for this degree");
    int q = opt.period, g = opt.stride;
    if (q <= 0) default_colouring(p, s, q, g);
    if (g <= 0) g = 1;
    if (q < s + p) return fail(IGA2L_ERR_INVALID_ARG, "colour period must be >= s + p");
    if (opt.schedule == IGA2L_SCHED_TILE && opt.tile < q)
        return fail(IGA2L_ERR_INVALID_ARG, "TILE side must be >= the colour period");
    if (gcd_int(g % q, q) != 1) return fail(IGA2L_ERR_INVALID_ARG, "colour stride must be coprime to the period");

    iga2l_solver *S = new (std::nothrow) iga2l_solver();
    if (!S) return fail(IGA2L_ERR_CUDA, "host allocation failed");
    S->dim = dim; S->p = p; S->m = m; S->s = s; S->r = (s - 1) / 2;
    S->n = m + p - 2;
    S->N = (long long)S->n * S->n * (dim == 3 ? S->n : 1);
    S->nbatch = nbatch;
    S->opt = opt;
    S->guard_bytes = (opt.test_flags & IGA2L_TEST_GUARD_ALLOCS) ? kGuardBytes : 0;
    S->q = q; S->g = g % q; S->tile = opt.tile;
    S->tile_groups = opt.schedule == IGA2L_SCHED_TILE && dim == 2
                         ? (opt.tile_groups > 0 ? opt.tile_groups : tile_groups_default(p)) : 1;
    if (S->tile_groups > q * q) S->tile_groups = q * q;
    cudaError_t ce = cudaGetDevice(&S->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, S->device);
    if (ce != cudaSuccess) { release(S); return cuda_fail(ce, "cudaGetDevice"); }
    if (S->nsm < 1) S->nsm = 1;

    std::string err;
    int rc = build_host_tables(p, m, s, S->ht, err);
    if (rc != IGA2L_OK) { release(S); return fail(rc, err); }
    const HostTables &ht = S->ht;
    const int n = S->n, W = 2 * p + 1, SS = s * s;

    // residual stencils per (row-class of y, row-class of x) (2D kernels)
    std::vector<double> stencil(dim == 2 ? (size_t)ht.npc * ht.npc * W * W : 1, 0.0);
    for (int cy = 0; dim == 2 && cy < ht.npc; ++cy)
        for (int cx = 0; cx < ht.npc; ++cx) {
            const int xr = ht.pc_rep[cx], yr = ht.pc_rep[cy];
            double *st = &stencil[(size_t)(cy * ht.npc + cx) * W * W];
            for (int b = 0; b < W; ++b)
                for (int a = 0; a < W; ++a)
                    st[b * W + a] = ht.Kb[(size_t)xr * W + a] * ht.Mb[(size_t)yr * W + b]
                                  + ht.Mb[(size_t)xr * W + a] * ht.Kb[(size_t)yr * W + b];
        }
    std::vector<int> pcls(n), bcls(n);
    for (int x = 0; x < n; ++x) {
        pcls[x] = x < 2 * p - 1 ? x : (x > n - 2 * p ? x - n + 4 * p - 1 : 2 * p - 1);
        bcls[x] = x < ht.L ? x : (x > n - 1 - ht.L ? 2 * ht.L - (n - 1 - x) : ht.L);
    }
    // Schwarz block inverses per block class (cz,) cy, cx; block DOF e = ex + s*(ey + s*ez) is
    // (c_x - r + ex, c_y - r + ey, c_z - r + ez); DOFs outside the grid get zero rows
    const int SD = dim == 3 ? s * s * s : s * s;
    const int ncls = dim == 3 ? ht.nbc * ht.nbc * ht.nbc : ht.nbc * ht.nbc;
    std::vector<double> binv((size_t)ncls * SD * SD, 0.0);
    for (int cls = 0; cls < ncls; ++cls) {
        const int bx = cls % ht.nbc, by = (cls / ht.nbc) % ht.nbc, bz = cls / (ht.nbc * ht.nbc);
        const int cx = ht.bc_rep[bx], cy = ht.bc_rep[by], cz = dim == 3 ? ht.bc_rep[bz] : 0;
        std::vector<double> A((size_t)SD * SD, 0.0);
        std::vector<int> valid(SD), X(SD), Y(SD), Z(SD);
        for (int a = 0; a < SD; ++a) {
            X[a] = cx - S->r + a % s;
            Y[a] = cy - S->r + (a / s) % s;
            Z[a] = dim == 3 ? cz - S->r + a / (s * s) : 0;
            valid[a] = X[a] >= 0 && X[a] < n && Y[a] >= 0 && Y[a] < n && (dim == 2 || (Z[a] >= 0 && Z[a] < n));
        }
        for (int a = 0; a < SD; ++a)
            for (int c = 0; c < SD; ++c) {
                if (!valid[a] || !valid[c]) { A[(size_t)a * SD + c] = (a == c) ? 1.0 : 0.0; continue; }
                const double kx = band(ht.Kb, p, X[a], X[c]), mx = band(ht.Mb, p, X[a], X[c]);
                const double ky = band(ht.Kb, p, Y[a], Y[c]), my = band(ht.Mb, p, Y[a], Y[c]);
                if (dim == 2) {
                    A[(size_t)a * SD + c] = kx * my + mx * ky;
                } else {
                    const double kz = band(ht.Kb, p, Z[a], Z[c]), mz = band(ht.Mb, p, Z[a], Z[c]);
                    A[(size_t)a * SD + c] = kx * my * mz + mx * ky * mz + mx * my * kz;
                }
            }
        if (!cholesky_inverse(SD, A)) { release(S); return fail(IGA2L_ERR_INVALID_ARG, "block matrix not SPD"); }
        double *dst = &binv[(size_t)cls * SD * SD];
        for (int a = 0; a < SD; ++a)
            for (int c = 0; c < SD; ++c)
                dst[(size_t)a * SD + c] = (valid[a] && valid[c]) ? A[(size_t)a * SD + c] : 0.0;
    }

    // second-level hierarchy (degree 1 on the 2h mesh, then 4h, ...)
    S->nc = ht.nc;
    S->Nc = (long long)ht.nc * ht.nc * (dim == 3 ? ht.nc : 1);
    for (int ml = m / 2;;) {
        Level L;
        L.m = ml;
        L.n = ml - 1;
        L.N = (long long)L.n * L.n * (dim == 3 ? L.n : 1);
        L.k[0] = -(double)ml; L.k[1] = 2.0 * ml; L.k[2] = -(double)ml;
        L.mm[0] = 1.0 / (6.0 * ml); L.mm[1] = 4.0 / (6.0 * ml); L.mm[2] = 1.0 / (6.0 * ml);
        S->lev.push_back(L);
        if (opt.coarse == IGA2L_COARSE_EXACT || ml <= 8 || (ml % 2) != 0 || (int)S->lev.size() >= kMaxLevels)
            break;
        ml /= 2;
    }
    const Level &D = S->lev.back();
    S->ndirect = (int)D.N;
    if (S->ndirect > 2048) { release(S); return fail(IGA2L_ERR_UNSUPPORTED, "exact second-level solve too large"); }
    std::vector<double> Ad((size_t)S->ndirect * S->ndirect, 0.0);
    {
        const int nd = D.n, nz = dim == 3 ? nd : 1;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < nd; ++y)
                for (int x = 0; x < nd; ++x)
                    for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int x2 = x + dx, y2 = y + dy, z2 = z + dz;
                                if (x2 < 0 || x2 >= nd || y2 < 0 || y2 >= nd || z2 < 0 || z2 >= nz) continue;
                                const size_t row = ((size_t)z * nd + y) * nd + x, col = ((size_t)z2 * nd + y2) * nd + x2;
                                double v;
                                if (dim == 2) v = D.k[dx + 1] * D.mm[dy + 1] + D.mm[dx + 1] * D.k[dy + 1];
                                else
                                    v = D.k[dx + 1] * D.mm[dy + 1] * D.mm[dz + 1] + D.mm[dx + 1] * D.k[dy + 1] * D.mm[dz + 1] +
                                        D.mm[dx + 1] * D.mm[dy + 1] * D.k[dz + 1];
                                Ad[row * S->ndirect + col] = v;
                            }
    }
    if (!cholesky_inverse(S->ndirect, Ad)) { release(S); return fail(IGA2L_ERR_INVALID_ARG, "coarsest matrix not SPD"); }

    // the interior stencil of degree p from a reference mesh, so that every handle of
    // degree p writes identical constant-memory values (2D stencils do not depend on h;
    // the 3D FP32 colour kernel takes the same h-scaled 1D rows)
    {
        HostTables ref;
        std::string rerr;
        const int mref = 8 * p + 16;
        if (build_host_tables(p, mref, s, ref, rerr) != IGA2L_OK) { release(S); return fail(IGA2L_ERR_INVALID_ARG, rerr); }
        const int xr = ref.pc_rep[2 * p - 1];
        std::vector<double> sti((size_t)W * W);
        for (int bb = 0; bb < W; ++bb)
            for (int a = 0; a < W; ++a)
                sti[(size_t)bb * W + a] = ref.Kb[(size_t)xr * W + a] * ref.Mb[(size_t)xr * W + bb]
                                        + ref.Mb[(size_t)xr * W + a] * ref.Kb[(size_t)xr * W + bb];
        // the handle's own interior class uses the same values
        if (dim == 2) {
            double *dst = &stencil[(size_t)((2 * p - 1) * ht.npc + (2 * p - 1)) * W * W];
            for (int i = 0; i < W * W; ++i) dst[i] = sti[i];
        }
        std::vector<double> k1(W), m1(W);
        for (int a = 0; a < W; ++a) {
            k1[a] = ref.Kb[(size_t)xr * W + a] / mref;   // h K_row, h = 1 / mref
            m1[a] = ref.Mb[(size_t)xr * W + a] * mref;   // M_row / h
        }
        if (dim == 2 ? ((ce = upload_interior_rows(p, k1.data(), m1.data())) != cudaSuccess ||
                        (ce = upload_persist_rows(p, k1.data(), m1.data())) != cudaSuccess)
                     : (ce = upload_rows3d(p, k1.data(), m1.data())) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "constant 1D rows upload");
        }
    }
    // upload
    if ((ce = upload(S, &S->Kb, ht.Kb)) != cudaSuccess ||
        (ce = upload(S, &S->Mb, ht.Mb)) != cudaSuccess ||
        (ce = upload(S, &S->stencil, stencil)) != cudaSuccess ||
        (ce = upload(S, &S->binv, binv)) != cudaSuccess ||
        (ce = upload(S, &S->binv_t, transpose_classes(binv, SD))) != cudaSuccess ||
        (ce = upload(S, &S->pcls, pcls)) != cudaSuccess ||
        (ce = upload(S, &S->bcls, bcls)) != cudaSuccess ||
        (ce = upload(S, &S->Rb, ht.Rb)) != cudaSuccess ||
        (ce = upload(S, &S->Cb, ht.Cb)) != cudaSuccess ||
        (ce = upload(S, &S->Rlo, ht.Rlo)) != cudaSuccess ||
        (ce = upload(S, &S->Clo, ht.Clo)) != cudaSuccess ||
        (ce = upload(S, &S->dinv, Ad)) != cudaSuccess) {
        release(S);
        return cuda_fail(ce, "table upload");
    }
    S->npart = residual_partials(*S);
    const size_t B = (size_t)nbatch;   // every per-problem buffer holds nbatch problems
    if ((ce = alloc(S, &S->d, B * S->N)) != cudaSuccess || (ce = alloc(S, &S->bwork, B * S->N)) != cudaSuccess ||
        (ce = alloc(S, &S->rhsb, B * S->N)) != cudaSuccess ||
        (ce = alloc(S, &S->t, B * (dim == 3 ? (size_t)n * n * S->nc : (size_t)n * S->nc))) != cudaSuccess ||
        (ce = alloc(S, &S->t2, B * (dim == 3 ? (size_t)n * S->nc * S->nc : (size_t)n * S->nc))) != cudaSuccess ||
        (ce = alloc(S, &S->dc, B * S->Nc)) != cudaSuccess || (ce = alloc(S, &S->ec, B * S->Nc)) != cudaSuccess ||
        (ce = alloc(S, &S->part, B * S->npart)) != cudaSuccess || (ce = alloc(S, &S->dev_norm, B)) != cudaSuccess) {
        release(S);
        return cuda_fail(ce, "workspace allocation");
    }
    {   // status word of the bounded device waits
        if ((ce = alloc(S, &S->wait_status, 1)) != cudaSuccess ||
            (ce = cudaMemset(S->wait_status, 0, sizeof(int))) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "status word");
        }
    }
    {   // completion counters of the fused residual norm, zero between launches
        if ((ce = alloc(S, &S->rcount, B)) != cudaSuccess ||
            (ce = cudaMemset(S->rcount, 0, sizeof(unsigned int) * B)) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "workspace allocation");
        }
    }
    // differentiable source (2D): quadrature tables and per-bump buffers; backward workspace
    if (dim == 2) {
        std::vector<double> qx, qw, qB;
        S->nq = p + 3;
        quadrature_tables(p, m, S->nq, qx, qw, qB);
        if ((ce = upload(S, &S->qx, qx)) != cudaSuccess || (ce = upload(S, &S->qw, qw)) != cudaSuccess ||
            (ce = upload(S, &S->qB, qB)) != cudaSuccess ||
            (ce = alloc(S, &S->gbuf, (size_t)kMaxBumps * 6 * n)) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "source tables");
        }
        S->gcap = kMaxBumps;
    }
    if ((ce = alloc(S, &S->adj1, S->N)) != cudaSuccess || (ce = alloc(S, &S->adj2, S->N)) != cudaSuccess ||
        (ce = alloc(S, &S->adj3, S->N)) != cudaSuccess) {
        release(S);
        return cuda_fail(ce, "backward workspace");
    }
    {
        std::vector<int> mlo(n);
        for (int i = 0; i < n; ++i) mlo[i] = i - p;
        if ((ce = upload(S, &S->Mlo, mlo)) != cudaSuccess) { release(S); return cuda_fail(ce, "mass band"); }
    }
    for (Level &L : S->lev)
        if ((ce = alloc(S, &L.e, B * L.N)) != cudaSuccess || (ce = alloc(S, &L.rhs, B * L.N)) != cudaSuccess ||
            (dim == 3 && (ce = alloc(S, &L.r, L.N)) != cudaSuccess) ||
            (dim == 2 && (ce = alloc(S, &L.pre, B * L.N)) != cudaSuccess)) {
            release(S);
            return cuda_fail(ce, "level allocation");
        }
    if ((ce = cudaMallocHost(&S->host_norm, sizeof(double))) != cudaSuccess ||
        (ce = cudaMallocHost(&S->ctl_host, sizeof(SolveCtl))) != cudaSuccess ||
        (ce = cudaMallocHost(&S->host_hist, sizeof(double) * kSolveHistCap)) != cudaSuccess) {
        release(S);
        return cuda_fail(ce, "pinned host buffers");
    }
    {
        void *pc = nullptr;
        if ((ce = dmalloc(S, &pc, sizeof(SolveCtl), false)) != cudaSuccess ||
            (ce = alloc(S, &S->dev_hist, kSolveHistCap)) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "solve control block");
        }
        S->ctl = static_cast<SolveCtl *>(pc);
    }
    if (opt.precision == IGA2L_MIXED_FP32 || opt.precision == IGA2L_MIXED_FP32_ALL ||
        opt.precision == IGA2L_MIXED_TF32) {
        // FP32 copies of the tables for the inner cycle (the FP64 block inverses are kept
        // for boundary classes and the FP64 coarsest inverse for the direct solve)
        MixedState &X = S->mx;
        auto to_f = [](const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); };
        auto allocf = [&](float **dst, size_t count) { return alloc(S, dst, count); };
        if ((ce = upload(S, &X.stencil, to_f(stencil))) != cudaSuccess ||
            (ce = upload(S, &X.binv, to_f(binv))) != cudaSuccess ||
            (ce = upload(S, &X.Rb, to_f(ht.Rb))) != cudaSuccess ||
            (ce = upload(S, &X.Cb, to_f(ht.Cb))) != cudaSuccess ||
            (ce = allocf(&X.r, B * S->N)) != cudaSuccess || (ce = allocf(&X.delta, B * S->N)) != cudaSuccess ||
            (ce = upload(S, &X.Kb, to_f(ht.Kb))) != cudaSuccess || (ce = upload(S, &X.Mb, to_f(ht.Mb))) != cudaSuccess ||
            (ce = allocf(&X.d, B * S->N)) != cudaSuccess ||
            (ce = allocf(&X.t, B * (dim == 3 ? (size_t)n * n * S->nc : (size_t)n * S->nc))) != cudaSuccess ||
            (ce = allocf(&X.t2, B * (dim == 3 ? (size_t)n * S->nc * S->nc : (size_t)n * S->nc))) != cudaSuccess ||
            (ce = allocf(&X.dc, B * S->Nc)) != cudaSuccess ||
            (ce = allocf(&X.ec, B * S->Nc)) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "mixed-precision allocation");
        }
        X.lev_e.assign(S->lev.size(), nullptr);
        X.lev_rhs.assign(S->lev.size(), nullptr);
        X.lev_r.assign(S->lev.size(), nullptr);
        X.lev_pre.assign(S->lev.size(), nullptr);
        for (size_t l = 0; l < S->lev.size(); ++l)
            if ((l > 0 && (ce = allocf(&X.lev_e[l], B * S->lev[l].N)) != cudaSuccess) ||
                (l > 0 && (ce = allocf(&X.lev_rhs[l], B * S->lev[l].N)) != cudaSuccess) ||
                (dim == 3 && (ce = allocf(&X.lev_r[l], S->lev[l].N)) != cudaSuccess) ||
                (dim == 2 && (ce = allocf(&X.lev_pre[l], B * S->lev[l].N)) != cudaSuccess)) {
                release(S);
                return cuda_fail(ce, "mixed-precision level allocation");
            }
        if ((ce = upload(S, &X.binv_t, to_f(transpose_classes(binv, SD)))) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "block-inverse upload");
        }
        if (opt.precision == IGA2L_MIXED_FP32 || opt.precision == IGA2L_MIXED_TF32) {
            std::vector<float> lo(binv.size());
            for (size_t i = 0; i < binv.size(); ++i) lo[i] = (float)(binv[i] - (double)(float)binv[i]);
            if ((ce = upload(S, &X.binv_lo, lo)) != cudaSuccess) {
                release(S);
                return cuda_fail(ce, "block-inverse pair upload");
            }
            std::vector<double> bt = transpose_classes(binv, SD);
            for (size_t i = 0; i < bt.size(); ++i) lo[i] = (float)(bt[i] - (double)(float)bt[i]);
            if ((ce = upload(S, &X.binv_lo_t, lo)) != cudaSuccess) {
                release(S);
                return cuda_fail(ce, "block-inverse pair upload");
            }
        }
        if (opt.precision == IGA2L_MIXED_TF32) {
            const int interior = ht.L * ht.nbc + ht.L;
            std::vector<double> ainv(binv.begin() + (size_t)interior * SS * SS,
                                     binv.begin() + (size_t)(interior + 1) * SS * SS);
            std::vector<float> g;
            build_gtc(*S, ainv, g, X.gtc_n, X.gtc_k);
            if ((ce = upload(S, &X.gtc, g)) != cudaSuccess) {
                release(S);
                return cuda_fail(ce, "tensor-core operator upload");
            }
            std::string why;
            if (!tc_colour_prepare(*S, why)) {
                release(S);
                return fail(IGA2L_ERR_UNSUPPORTED, why.c_str());
            }
        }
        X.enabled = true;
        // the persistent LATTICE sweep of the inner cycle (one launch per sweep)
        if (dim == 2 && !batch && opt.schedule == IGA2L_SCHED_LATTICE && opt.precision != IGA2L_MIXED_TF32 &&
            opt.sweep != IGA2L_SWEEP_PER_COLOUR && has_interior) {
            if ((ce = alloc(S, &S->progress, 4096)) != cudaSuccess) {
                release(S);
                return cuda_fail(ce, "progress counters");
            }
            if (!persist_setup(*S) && opt.sweep == IGA2L_SWEEP_PERSISTENT) {
                release(S);
                return fail(IGA2L_ERR_UNSUPPORTED, "no resident launch plan for the persistent sweep");
            }
            // AUTO: measured at 1024^2 (GB300), one persistent launch beats one launch per
            // colour only with the most colours (p = 8, q^2 = 289: 3.85 against 4.23 ms per
            // sweep); with fewer its colour-to-colour hand-off between neighbouring CTAs (about
            // 4.4 us) costs more than a launch (p = 5: 1.20 against 1.11 ms, p = 7: 3.35 against
            // 2.99 ms)
            if (opt.sweep == IGA2L_SWEEP_AUTO && S->q * S->q < 250) S->pgx = 0;
        }
    }
    if (opt.sweep == IGA2L_SWEEP_WORK_LIST) {   // the TILE sweep as one work-list launch
        const size_t nt = (size_t)((S->n + tile_side(p) - 1) / tile_side(p));   // tile positions per axis
        S->tile_work_ctas = tile_work_ctas(*S);
        if (S->tile_work_ctas <= 0) {
            release(S);
            return fail(IGA2L_ERR_UNSUPPORTED, "no resident launch plan for the work-list sweep");
        }
        if ((ce = alloc(S, &S->tile_ctr, 1 + (size_t)nbatch * nt * nt)) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "work-list counters");
        }
    }
    if (opt.sweep == IGA2L_SWEEP_PERSISTENT && S->pgx == 0) {
        release(S);
        return fail(IGA2L_ERR_UNSUPPORTED,
                    "the persistent sweep needs a 2D single-problem handle, IGA2L_MIXED_FP32 or _FP32_ALL, LATTICE, "
                    "m >= 4p+4");
    }
    if (batch) {
        if ((ce = alloc(S, &S->active, B)) != cudaSuccess || (ce = alloc(S, &S->bcycles, B + 1)) != cudaSuccess ||
            (ce = alloc(S, &S->bnorm0, 2 * B)) != cudaSuccess) {
            release(S);
            return cuda_fail(ce, "batch state");
        }
        S->bcount = S->bcycles + B;
        S->brel = S->bnorm0 + B;
    }
    *out = S;
    g_last_error.clear();
    return IGA2L_OK;
}

extern "C" {

int iga2l_assemble(int p, int m, int dim, const iga2l_options *opt, iga2l_handle *out)
{
    return assemble_impl(p, m, dim, 1, false, opt, out);
}

int iga2l_assemble_batch(int p, int m, int nbatch, const iga2l_options *opt, iga2l_handle *out)
{
    if (!out) return fail(IGA2L_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (nbatch < 1 || nbatch > 65535) return fail(IGA2L_ERR_INVALID_ARG, "nbatch must be 1..65535");
    return assemble_impl(p, m, 2, nbatch, true, opt, out);
}

int iga2l_solve_batch(iga2l_handle h, const double *rhs, double tol, int max_cycles, double *u, int *cycles,
                      double *relres, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!rhs || !u || !cycles || !relres) return fail(IGA2L_ERR_INVALID_ARG, "null argument");
    if (!(tol >= 0.0)) return fail(IGA2L_ERR_INVALID_ARG, "tol must be >= 0");
    if (!h->active) return fail(IGA2L_ERR_INVALID_ARG, "handle is not a batch (iga2l_assemble_batch)");
    if (max_cycles <= 0) max_cycles = h->opt.max_cycles;
    cudaStream_t st = as_stream(stream);
    const double *b = rhs;
    if (h->opt.rhs == IGA2L_RHS_COEFFS) {   // every problem's b = (M (x) M) f
        if ((rc = load_from_coeffs(h, rhs, u, st)) != IGA2L_OK) return rc;
        b = h->rhsb;
    }
    const int nb = h->nbatch;
    // initial residuals of every problem (all active while they are computed)
    std::vector<int> ones(nb, 1);
    cudaError_t e = cudaMemcpyAsync(h->active, ones.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        if (h->mx.enabled) e = launch_outer_residual_norm(*h, u, b, h->mx.r, h->dev_norm, st);
        else e = launch_residual_norm(*h, u, b, nullptr, h->dev_norm, st);
    }
    if (e == cudaSuccess) e = launch_batch_init(*h, h->dev_norm, h->bnorm0, h->bcycles, h->brel, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch start");
    int left = nb;
    // device-driven: one graph launch runs the cycles until no problem is active or
    // max_cycles ran (k_batch_check sets the WHILE condition)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    iga2l_solver::SolveGraph *sg = nullptr;
    if (h->opt.graphs && !h->solve_graph_failed && cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
        cs == cudaStreamCaptureStatusNone)
        sg = solve_graph(h, u, b, false);
    if (sg) {
        *h->ctl_host = SolveCtl{0.0, tol, 0.0, max_cycles, 0, -1};
        e = cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(SolveCtl), cudaMemcpyHostToDevice, st);
        sg->last_use = ++h->tick;
        if (e == cudaSuccess) e = cudaGraphLaunch(sg->exec, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "batched solve");
        count_launches(sg->kernels_per_cycle * h->ctl_host->k);
    }
    // host-driven: converged problems are masked on the device, the host polls every 4 cycles
    for (int k = 0; !sg && k < max_cycles && left > 0; ++k) {
        if ((rc = run_cycle_graph(h, u, b, st, false, true)) != IGA2L_OK) return rc;
        e = launch_batch_check(*h, tol, h->dev_norm, h->bnorm0, h->bcycles, h->brel, h->bcount, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch check");
        if ((k % 4) == 3 || k == max_cycles - 1) {
            e = cudaMemcpyAsync(&left, h->bcount, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "batch poll");
        }
    }
    e = cudaMemcpyAsync(cycles, h->bcycles, sizeof(int) * nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(relres, h->brel, sizeof(double) * nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&left, h->bcount, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch results");
    if ((rc = wait_status_check(h, st)) != IGA2L_OK) return rc;
    for (int k = 0; k < nb; ++k)
        if (!std::isfinite(relres[k])) return fail(IGA2L_ERR_NONFINITE, "a residual norm is not finite");
    if (left > 0) { g_last_error = "cycle cap reached"; return IGA2L_NOT_CONVERGED; }
    return IGA2L_OK;
}

int iga2l_num_dofs(iga2l_handle h, long long *n_total, int *n_axis, long long *nc_total, int *nc_axis)
{
    if (!h) return fail(IGA2L_ERR_INVALID_ARG, "null handle");
    if (n_total) *n_total = h->N;
    if (n_axis) *n_axis = h->n;
    if (nc_total) *nc_total = h->Nc;
    if (nc_axis) *nc_axis = h->nc;
    return IGA2L_OK;
}

int iga2l_schedule_info(iga2l_handle h, int *schedule, int *period, int *stride, int *tile, int *block_side,
                        int *tile_groups)
{
    if (!h) return fail(IGA2L_ERR_INVALID_ARG, "null handle");
    if (tile_groups) *tile_groups = h->opt.schedule == IGA2L_SCHED_TILE ? h->tile_groups : 1;
    if (schedule) *schedule = h->opt.schedule;
    if (period) *period = h->q;
    if (stride) *stride = h->g;
    if (tile) *tile = h->opt.schedule == IGA2L_SCHED_TILE ? h->tile : 0;
    if (block_side) *block_side = h->s;
    return IGA2L_OK;
}

int iga2l_apply_A(iga2l_handle h, const double *u, double *y, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!u || !y) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    return finish(launch_apply_A(*h, u, y, as_stream(stream)), "apply_A");
}

int iga2l_residual(iga2l_handle h, const double *u, const double *b, double *d, double *norm, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!u || !b) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    cudaStream_t st = as_stream(stream);
    if (!norm) return finish(launch_residual(*h, u, b, d, nullptr, st), "residual");
    if (h->active) return fail(IGA2L_ERR_INVALID_ARG, "residual norm of a batch: use iga2l_solve_batch");
    double sq = 0.0;
    rc = residual_norm2(h, u, b, d, st, &sq);
    if (rc != IGA2L_OK) return rc;
    *norm = std::sqrt(sq);
    return IGA2L_OK;
}

int iga2l_schwarz_sweep(iga2l_handle h, double *u, const double *b, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!u || !b) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    return finish(launch_schwarz(*h, u, b, false, as_stream(stream)), "schwarz sweep");
}

int iga2l_schwarz_sweep_reverse(iga2l_handle h, double *u, const double *b, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!u || !b) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    return finish(launch_schwarz(*h, u, b, true, as_stream(stream)), "reverse schwarz sweep");
}

int iga2l_schwarz_sweep_f32(iga2l_handle h, float *u, const float *b, int reverse, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!u || !b) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    if (!h->mx.enabled || h->dim != 2)
        return fail(IGA2L_ERR_INVALID_ARG, "the FP32 sweep needs a 2D mixed-precision handle");
    return finish(launch_inner_sweep(*h, u, b, reverse != 0, as_stream(stream)), "FP32 schwarz sweep");
}

int iga2l_restrict(iga2l_handle h, const double *d, double *dc, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!d || !dc) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    return finish(launch_restrict(*h, d, dc, as_stream(stream)), "restrict");
}

int iga2l_prolong_add(iga2l_handle h, const double *ec, double *u, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!ec || !u) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    return finish(launch_prolong_add(*h, ec, u, as_stream(stream)), "prolong_add");
}

int iga2l_coarse_solve(iga2l_handle h, const double *dc, double *ec, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!dc || !ec) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    return finish(launch_coarse_solve(*h, dc, ec, as_stream(stream)), "coarse solve");
}

int iga2l_cycle(iga2l_handle h, double *u, const double *b, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!u || !b) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    return run_cycle(h, u, b, as_stream(stream), false);
}

int iga2l_cycle_adjoint(iga2l_handle h, double *u, const double *b, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!u || !b) return fail(IGA2L_ERR_INVALID_ARG, "null vector");
    return run_cycle(h, u, b, as_stream(stream), true);
}

int iga2l_solve(iga2l_handle h, const double *rhs, double tol, int max_cycles, double *u, int *cycles,
                double *relres, double *hist, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (h->active) return fail(IGA2L_ERR_INVALID_ARG, "single-problem entry point on a batch handle");
    const double *b = rhs;
    if (h->opt.rhs == IGA2L_RHS_COEFFS) {   // b_p = (f, phi_i) = (M (x) M [(x) M]) f
        if ((rc = load_from_coeffs(h, rhs, u, as_stream(stream))) != IGA2L_OK) return rc;
        b = h->rhsb;
    }
    return solve_impl(h, b, tol, max_cycles, u, cycles, relres, hist, stream, false);
}

int iga2l_solve_load(iga2l_handle h, const double *b, double tol, int max_cycles, double *u, int *cycles,
                     double *relres, double *hist, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (h->active) return fail(IGA2L_ERR_INVALID_ARG, "single-problem entry point on a batch handle");
    return solve_impl(h, b, tol, max_cycles, u, cycles, relres, hist, stream, false);
}

int iga2l_adjoint_solve(iga2l_handle h, const double *g, double tol, int max_cycles, double *lambda,
                        int *cycles, double *relres, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (h->active) return fail(IGA2L_ERR_INVALID_ARG, "single-problem entry point on a batch handle");
    return solve_impl(h, g, tol, max_cycles, lambda, cycles, relres, nullptr, stream, true);
}

int iga2l_rhs_from_coeffs(iga2l_handle h, const double *f, double *b, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!f || !b || f == b) return fail(IGA2L_ERR_INVALID_ARG, "null or aliased vector");
    return finish(launch_mass2(*h, f, b, as_stream(stream)), "rhs_from_coeffs");
}

int iga2l_cycles(iga2l_handle h, double *u, const double *b, int ncycles, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!u || !b || ncycles < 0) return fail(IGA2L_ERR_INVALID_ARG, "bad arguments");
    for (int k = 0; k < ncycles; ++k)
        if ((rc = run_cycle(h, u, b, as_stream(stream), false)) != IGA2L_OK) return rc;
    return IGA2L_OK;
}

int iga2l_unrolled_backward(iga2l_handle h, const double *ubar, int ncycles, double *bbar, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (h->active) return fail(IGA2L_ERR_INVALID_ARG, "single-problem entry point on a batch handle");
    if (!ubar || !bbar || ncycles < 0) return fail(IGA2L_ERR_INVALID_ARG, "bad arguments");
    if (bbar == h->adj1 || bbar == h->adj2 || bbar == h->adj3) return fail(IGA2L_ERR_INVALID_ARG, "aliased output");
    cudaStream_t st = as_stream(stream);
    const size_t bytes = sizeof(double) * h->N;
    double *ub = h->adj1, *v = h->adj2, *nx = h->adj3;
    cudaError_t e = cudaMemcpyAsync(ub, ubar, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bbar, 0, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "unrolled backward");
    // u_k = u_{k-1} + C (b - A u_{k-1}):  bbar += C^T ubar,  ubar <- (I - A C^T) ubar
    for (int k = 0; k < ncycles; ++k) {
        if ((e = cudaMemsetAsync(v, 0, bytes, st)) != cudaSuccess) return cuda_fail(e, "unrolled backward");
        if ((rc = run_cycle(h, v, ub, st, true)) != IGA2L_OK) return rc;   // v = C^T ubar
        if ((e = launch_axpy(h->N, 1.0, v, bbar, st)) != cudaSuccess) return cuda_fail(e, "unrolled backward");
        if ((e = launch_residual(*h, v, ub, nx, nullptr, st)) != cudaSuccess) return cuda_fail(e, "unrolled backward");
        double *t = ub; ub = nx; nx = t;
    }
    return IGA2L_OK;
}

int iga2l_bump_load(iga2l_handle h, int nbumps, const double *theta, double width, double *b, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (h->active) return fail(IGA2L_ERR_INVALID_ARG, "single-problem entry point on a batch handle");
    if (h->dim != 2) return fail(IGA2L_ERR_UNSUPPORTED, "the bump source is 2D");
    if (nbumps < 1 || nbumps > h->gcap || !theta || !b || !(width > 0.0))
        return fail(IGA2L_ERR_INVALID_ARG, "bad bump arguments (1 <= nbumps <= 64, width > 0)");
    return finish(launch_bump_load(*h, nbumps, theta, width, b, as_stream(stream)), "bump load");
}

int iga2l_bump_grad(iga2l_handle h, int nbumps, const double *theta, double width, const double *bbar,
                    double *grad, void *stream)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (h->active) return fail(IGA2L_ERR_INVALID_ARG, "single-problem entry point on a batch handle");
    if (h->dim != 2) return fail(IGA2L_ERR_UNSUPPORTED, "the bump source is 2D");
    if (nbumps < 1 || nbumps > h->gcap || !theta || !bbar || !grad || !(width > 0.0))
        return fail(IGA2L_ERR_INVALID_ARG, "bad bump arguments (1 <= nbumps <= 64, width > 0)");
    return finish(launch_bump_grad(*h, nbumps, theta, width, bbar, grad, as_stream(stream)), "bump gradient");
}

int iga2l_get_bands(iga2l_handle h, double *K, double *M)
{
    if (!h || !K || !M) return fail(IGA2L_ERR_INVALID_ARG, "null argument");
    std::memcpy(K, h->ht.Kb.data(), sizeof(double) * h->ht.Kb.size());
    std::memcpy(M, h->ht.Mb.data(), sizeof(double) * h->ht.Mb.size());
    return IGA2L_OK;
}

int iga2l_host_bands(int p, int m, double *K, double *M)
{
    if (p < 1 || p > kMaxP || m < 1 || !K || !M) return fail(IGA2L_ERR_INVALID_ARG, "bad arguments");
    std::vector<double> Kb, Mb;
    bspline_band_1d(p, m, Kb, Mb);
    std::memcpy(K, Kb.data(), sizeof(double) * Kb.size());
    std::memcpy(M, Mb.data(), sizeof(double) * Mb.size());
    return IGA2L_OK;
}

int iga2l_host_restriction(int p, int m, double *R)
{
    if (p < 2 || p > kMaxP || m < 4 || (m % 2) != 0 || !R) return fail(IGA2L_ERR_INVALID_ARG, "bad arguments");
    HostTables ht;
    std::string err;
    const int s = default_block_side(p);
    int rc = build_host_tables(p, m, s, ht, err);
    if (rc != IGA2L_OK) return fail(rc, err);
    const int n = ht.n, nc = ht.nc;
    std::memset(R, 0, sizeof(double) * (size_t)nc * n);
    for (int I = 0; I < nc; ++I)
        for (int t = 0; t < ht.wr; ++t) {
            const int j = ht.Rlo[I] + t;
            if (j < n) R[(size_t)I * n + j] = ht.Rb[(size_t)I * ht.wr + t];
        }
    return IGA2L_OK;
}

void iga2l_destroy(iga2l_handle h) { release(h); }

const char *iga2l_strerror(int code)
{
    switch (code) {
    case IGA2L_OK: return "ok";
    case IGA2L_NOT_CONVERGED: return "not converged";
    case IGA2L_ERR_INVALID_ARG: return "invalid argument";
    case IGA2L_ERR_CUDA: return "CUDA error";
    case IGA2L_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case IGA2L_ERR_NONFINITE: return "non-finite value";
    case IGA2L_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
    }
}

const char *iga2l_last_error(void) { return g_last_error.c_str(); }

long long iga2l_kernel_launches(void) { return launches_so_far(); }

int iga2l_guard_check(iga2l_handle h, long long *changed)
{
    int rc = check_handle(h);
    if (rc != IGA2L_OK) return rc;
    if (!changed) return fail(IGA2L_ERR_INVALID_ARG, "null output");
    *changed = 0;
    if (!h->guard_bytes) return fail(IGA2L_ERR_INVALID_ARG, "the handle was built without IGA2L_TEST_GUARD_ALLOCS");
    cudaError_t ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) return cuda_fail(ce, "guard check");
    std::vector<unsigned char> zone(h->guard_bytes);
    long long bad = 0;
    for (const auto &g : h->guarded)
        for (const char *z : {g.p - h->guard_bytes, g.p + g.bytes}) {
            if ((ce = cudaMemcpy(zone.data(), z, zone.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
                return cuda_fail(ce, "guard check");
            for (unsigned char c : zone) bad += c != g.fill;
        }
    *changed = bad;
    return IGA2L_OK;
}

}  // extern "C"
