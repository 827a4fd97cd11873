// kernels_coarse.cu -- second level of the two-level cycle (2D).
//
// Degree-1 discretisation on the 2h mesh (Section 3.3), approximated by one
// V(1,1) h-multigrid cycle with red-black Gauss-Seidel (Section 3.2), or solved
// exactly (Algorithm 1).  Level operators are the 9-point degree-1 stencils
// k_x m_y + m_x k_y with k = (-1, 2, -1)/H and m = (1, 4, 1) H/6; transfers are
// the exact embedding of nested degree-1 spaces (weights 1/2, 1, 1/2) and its
// transpose; the coarsest level (8 or fewer elements per axis) uses a dense
// inverse computed on the host.  Kernels are templated on the storage type
// (double: FP64 form; float: inner cycle of the mixed form); the coarsest solve
// always accumulates in FP64.
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace iga2l {

namespace {

template <typename T>
struct Stencil9 {
    T c[3][3];   // c[dy][dx], dx, dy in {0,1,2} <-> offsets -1, 0, +1
};

// red-black order of the sub-lattices: red (0,0), (1,1) then black (1,0), (0,1)
__constant__ int kGsSeqDev[4][2] = {{0, 0}, {1, 1}, {1, 0}, {0, 1}};

template <typename T>
Stencil9<T> level_stencil(const Level &L)
{
    Stencil9<T> s;
    for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx) s.c[dy][dx] = (T)(L.k[dx] * L.mm[dy] + L.mm[dx] * L.k[dy]);
    return s;
}

// Relax the sub-lattice {(2a+px, 2b+py)}: e += (rhs - A e) / A_diag.  No two points
// of a sub-lattice are coupled by the 9-point stencil.
template <typename T>
__global__ void k_gs_sublattice(int n, int px, int py, Stencil9<T> st, const T *__restrict__ rhs,
                                T *__restrict__ e, BatchRef bt)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x, bidx = blockIdx.y * blockDim.y + threadIdx.y;
    const int x = 2 * a + px, y = 2 * bidx + py;
    if (x >= n || y >= n || (bt.active && !bt.active[blockIdx.z])) return;
    rhs += blockIdx.z * bt.vec;
    e += blockIdx.z * bt.vec;
    T acc = T(0);
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const int yy = y + dy - 1;
        if (yy < 0 || yy >= n) continue;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            const int xx = x + dx - 1;
            if (xx >= 0 && xx < n) acc = fma(st.c[dy][dx], e[(size_t)yy * n + xx], acc);
        }
    }
    e[(size_t)y * n + x] += (rhs[(size_t)y * n + x] - acc) / st.c[1][1];
}

// First relaxation from e = 0: the first red sub-lattice (0,0) gets e = rhs / A_diag (its
// neighbours are all zero), every other point is zeroed.  Same values as zeroing e and
// relaxing sub-lattice (0,0).
template <typename T>
__global__ void k_gs_first(int n, Stencil9<T> st, const T *__restrict__ rhs, T *__restrict__ e, BatchRef bt)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= n || y >= n || (bt.active && !bt.active[blockIdx.z])) return;
    rhs += blockIdx.z * bt.vec;
    e += blockIdx.z * bt.vec;
    const size_t i = (size_t)y * n + x;
    e[i] = ((x | y) & 1) ? T(0) : (rhs[i] - T(0)) / st.c[1][1];
}

// rc[J][I] = sum_{dy,dx} w_dy w_dx (rhs - A e)[2J+dy][2I+dx], w = (1/2, 1, 1/2): the level
// residual at the 3x3 fine points under coarse hat (I, J), restricted in place.
template <typename T>
__global__ void k_level_residual_restrict(int nf, int nc, Stencil9<T> st, const T *__restrict__ rhs,
                                          const T *__restrict__ e, T *__restrict__ rc, BatchRef bt)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= nc || J >= nc || (bt.active && !bt.active[blockIdx.z])) return;
    rhs += blockIdx.z * bt.vec;
    e += blockIdx.z * bt.vec;
    rc += blockIdx.z * bt.crs;
    const T w[3] = {T(0.5), T(1), T(0.5)};
    T acc = T(0);
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const int y = 2 * J + dy;
        T s = T(0);
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            const int x = 2 * I + dx;
            T a = T(0);
#pragma unroll
            for (int ey = 0; ey < 3; ++ey) {
                const int yy = y + ey - 1;
                if (yy < 0 || yy >= nf) continue;
#pragma unroll
                for (int ex = 0; ex < 3; ++ex) {
                    const int xx = x + ex - 1;
                    if (xx >= 0 && xx < nf) a = fma(st.c[ey][ex], e[(size_t)yy * nf + xx], a);
                }
            }
            const T r = rhs[(size_t)y * nf + x] - a;
            s = fma(w[dx], r, s);
        }
        acc = fma(w[dy], s, acc);
    }
    rc[(size_t)J * nc + I] = acc;
}

// e[y][x] += sum over the coarse points whose hats cover fine node (x, y)
template <typename T>
__global__ void k_level_prolong_add(int nf, int nc, const T *__restrict__ ec, T *__restrict__ e, BatchRef bt)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nf || y >= nf || (bt.active && !bt.active[blockIdx.z])) return;
    ec += blockIdx.z * bt.crs;
    e += blockIdx.z * bt.vec;
    // fine index x is coarse I = (x-1)/2 when odd (weight 1); between I = x/2-1 and x/2 when even
    int Ix[2], Iy[2];
    T wx[2], wy[2];
    int nx, ny;
    if (x & 1) { Ix[0] = (x - 1) / 2; wx[0] = T(1); nx = 1; }
    else { Ix[0] = x / 2 - 1; Ix[1] = x / 2; wx[0] = T(0.5); wx[1] = T(0.5); nx = 2; }
    if (y & 1) { Iy[0] = (y - 1) / 2; wy[0] = T(1); ny = 1; }
    else { Iy[0] = y / 2 - 1; Iy[1] = y / 2; wy[0] = T(0.5); wy[1] = T(0.5); ny = 2; }
    T acc = T(0);
    for (int b = 0; b < ny; ++b) {
        if (Iy[b] < 0 || Iy[b] >= nc) continue;
        T s = T(0);
        for (int a = 0; a < nx; ++a) {
            if (Ix[a] < 0 || Ix[a] >= nc) continue;
            s = fma(wx[a], ec[(size_t)Iy[b] * nc + Ix[a]], s);
        }
        acc = fma(wy[b], s, acc);
    }
    e[(size_t)y * nf + x] += acc;
}

// x = Ainv rhs in FP64, one warp per row (dense inverse of the directly solved level)
template <typename T>
__global__ void k_dense_matvec(int N, const double *__restrict__ Ainv, const T *__restrict__ rhs,
                               T *__restrict__ x, BatchRef bt)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= N || (bt.active && !bt.active[blockIdx.y])) return;
    rhs += blockIdx.y * bt.vec;
    x += blockIdx.y * bt.vec;
    const double *row = Ainv + (size_t)warp * N;
    double s = 0.0;
    for (int j = lane; j < N; j += 32) s = fma(row[j], (double)rhs[j], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) x[warp] = (T)s;
}

// ---- the small levels in one thread block -------------------------------------------
// Levels below a size threshold are cheap but, one kernel per step, launch-bound.  This
// kernel runs the rest of the V(1,1) cycle from level `first` down to the direct solve
// and back in a single CTA whose level vectors live in shared memory, with
// __syncthreads between steps.  Every point update uses the same arithmetic in the same
// order as the per-step kernels above.
constexpr int kTailMaxLevels = 8;

template <typename T>
struct TailArgs {
    const int *active;                // per-problem flags (one CTA per problem) or null
    long long vec0;                   // batch stride of rhs0 / e0
    int nl;                           // levels in the tail (last one solved directly)
    int n[kTailMaxLevels];
    Stencil9<T> st[kTailMaxLevels];
    const T *rhs0;                    // right-hand side of the first tail level (global)
    T *e0;                            // its correction (global, written at the end)
    const double *dinv;
};

template <typename T>
__device__ void tail_gs(int n, const Stencil9<T> &st, const T *rhs, T *e, int px, int py, bool first)
{
    const int half = (n + 1) / 2;
    if (first) {
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
            const int x = i % n, y = i / n;
            e[i] = ((x | y) & 1) ? T(0) : (rhs[i] - T(0)) / st.c[1][1];
        }
        return;
    }
    for (int i = threadIdx.x; i < half * half; i += blockDim.x) {
        const int x = 2 * (i % half) + px, y = 2 * (i / half) + py;
        if (x >= n || y >= n) continue;
        T acc = T(0);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const int yy = y + dy - 1;
            if (yy < 0 || yy >= n) continue;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int xx = x + dx - 1;
                if (xx >= 0 && xx < n) acc = fma(st.c[dy][dx], e[yy * n + xx], acc);
            }
        }
        e[y * n + x] += (rhs[y * n + x] - acc) / st.c[1][1];
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_vcycle_tail(TailArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char tail_smem[];
    if (a.active && !a.active[blockIdx.x]) return;
    a.rhs0 += blockIdx.x * a.vec0;
    a.e0 += blockIdx.x * a.vec0;
    T *E[kTailMaxLevels], *Rh[kTailMaxLevels];
    {
        T *p = reinterpret_cast<T *>(tail_smem);
        for (int l = 0; l < a.nl; ++l) {
            E[l] = p; p += a.n[l] * a.n[l];
            Rh[l] = p; p += a.n[l] * a.n[l];
        }
    }
    for (int i = threadIdx.x; i < a.n[0] * a.n[0]; i += blockDim.x) Rh[0][i] = a.rhs0[i];
    __syncthreads();
    const int last = a.nl - 1;
    for (int l = 0; l < last; ++l) {
        const int n = a.n[l], nc = a.n[l + 1];
        for (int t = 0; t < 4; ++t) {
            tail_gs<T>(n, a.st[l], Rh[l], E[l], kGsSeqDev[t][0], kGsSeqDev[t][1], t == 0);
            __syncthreads();
        }
        const T w[3] = {T(0.5), T(1), T(0.5)};
        for (int i = threadIdx.x; i < nc * nc; i += blockDim.x) {
            const int I = i % nc, J = i / nc;
            T acc = T(0);
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int y = 2 * J + dy;
                T sacc = T(0);
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int x = 2 * I + dx;
                    T aa = T(0);
#pragma unroll
                    for (int ey = 0; ey < 3; ++ey) {
                        const int yy = y + ey - 1;
                        if (yy < 0 || yy >= n) continue;
#pragma unroll
                        for (int ex = 0; ex < 3; ++ex) {
                            const int xx = x + ex - 1;
                            if (xx >= 0 && xx < n) aa = fma(a.st[l].c[ey][ex], E[l][yy * n + xx], aa);
                        }
                    }
                    const T r = Rh[l][y * n + x] - aa;
                    sacc = fma(w[dx], r, sacc);
                }
                acc = fma(w[dy], sacc, acc);
            }
            Rh[l + 1][J * nc + I] = acc;
        }
        __syncthreads();
    }
    {   // direct solve: warp-per-row dot products, the reduction order of k_dense_matvec
        const int N = a.n[last] * a.n[last];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int row = warp; row < N; row += nw) {
            const double *rp = a.dinv + (size_t)row * N;
            double sacc = 0.0;
            for (int j = lane; j < N; j += 32) sacc = fma(rp[j], (double)Rh[last][j], sacc);
            for (int off = 16; off > 0; off >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, off);
            if (lane == 0) E[last][row] = (T)sacc;
        }
        __syncthreads();
    }
    for (int l = last - 1; l >= 0; --l) {
        const int nf = a.n[l], nc = a.n[l + 1];
        for (int i = threadIdx.x; i < nf * nf; i += blockDim.x) {
            const int x = i % nf, y = i / nf;
            int Ix[2], Iy[2];
            T wx[2], wy[2];
            int nx, ny;
            if (x & 1) { Ix[0] = (x - 1) / 2; wx[0] = T(1); nx = 1; }
            else { Ix[0] = x / 2 - 1; Ix[1] = x / 2; wx[0] = T(0.5); wx[1] = T(0.5); nx = 2; }
            if (y & 1) { Iy[0] = (y - 1) / 2; wy[0] = T(1); ny = 1; }
            else { Iy[0] = y / 2 - 1; Iy[1] = y / 2; wy[0] = T(0.5); wy[1] = T(0.5); ny = 2; }
            T acc = T(0);
            for (int bq = 0; bq < ny; ++bq) {
                if (Iy[bq] < 0 || Iy[bq] >= nc) continue;
                T sacc = T(0);
                for (int aq = 0; aq < nx; ++aq) {
                    if (Ix[aq] < 0 || Ix[aq] >= nc) continue;
                    sacc = fma(wx[aq], E[l + 1][Iy[bq] * nc + Ix[aq]], sacc);
                }
                acc = fma(wy[bq], sacc, acc);
            }
            E[l][i] += acc;
        }
        __syncthreads();
        for (int t = 3; t >= 0; --t) {
            tail_gs<T>(nf, a.st[l], Rh[l], E[l], kGsSeqDev[t][0], kGsSeqDev[t][1], false);
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < a.n[0] * a.n[0]; i += blockDim.x) a.e0[i] = E[0][i];
}

dim3 grid2(int nx, int ny, dim3 blk)
{
    return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y);
}

dim3 grid3(int nx, int ny, int nz, dim3 blk)
{
    return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y, nz);
}

// red-black order: red sub-lattices (0,0), (1,1) then black (1,0), (0,1)
constexpr int kGsSeq[4][2] = {{0, 0}, {1, 1}, {1, 0}, {0, 1}};

template <typename T>
cudaError_t gs_pass(const Level &L, const Stencil9<T> &st, const T *rhs, T *e, bool forward,
                    bool from_zero, int nb, const BatchRef &bt, cudaStream_t s)
{
    dim3 blk(32, 4);
    const int half = (L.n + 1) / 2;
    for (int t = 0; t < 4; ++t) {
        const int c = forward ? t : 3 - t;
        if (from_zero && t == 0) {   // forward pass from e = 0: the first colour is (0,0)
            k_gs_first<T><<<grid3(L.n, L.n, nb, blk), blk, 0, s>>>(L.n, st, rhs, e, bt);
            count_launches(1);
            continue;
        }
        k_gs_sublattice<T><<<grid3(half, half, nb, blk), blk, 0, s>>>(L.n, kGsSeq[c][0], kGsSeq[c][1], st, rhs, e, bt);
        count_launches(1);
    }
    return cudaGetLastError();
}

// levE[l], levR[l]: the e and rhs arrays of level l >= 1 in the storage type T
template <typename T>
cudaError_t vcycle(const Solver &S, int l, const T *rhs, T *e, T *const *levE, T *const *levR, cudaStream_t s)
{
    const Level &L = S.lev[l];
    const int last = (int)S.lev.size() - 1;
    const int nb = S.nbatch;
    if (l == last) {
        const int N = S.ndirect;
        k_dense_matvec<T><<<dim3((N * 32 + 255) / 256, nb), 256, 0, s>>>(N, S.dinv, rhs, e,
                                                                         BatchRef{S.active, L.N, 0, 0});
        count_launches(1);
        return cudaGetLastError();
    }
    // small levels: the rest of the cycle in one thread block per problem, in shared memory
    const int tail_n = sizeof(T) == sizeof(float) ? 63 : 31;
    if (L.n <= tail_n && last - l + 1 <= kTailMaxLevels) {
        TailArgs<T> a{};
        a.active = S.active;
        a.vec0 = L.N;
        a.nl = last - l + 1;
        size_t smem = 0;
        for (int k = 0; k < a.nl; ++k) {
            a.n[k] = S.lev[l + k].n;
            a.st[k] = level_stencil<T>(S.lev[l + k]);
            smem += 2 * sizeof(T) * (size_t)a.n[k] * a.n[k];
        }
        if (smem <= 48 * 1024) {
            a.rhs0 = rhs;
            a.e0 = e;
            a.dinv = S.dinv;
            k_vcycle_tail<T><<<nb, 1024, smem, s>>>(a);
            count_launches(1);
            return cudaGetLastError();
        }
    }
    const Level &C = S.lev[l + 1];
    const Stencil9<T> st = level_stencil<T>(L);
    const BatchRef bt{S.active, L.N, 0, C.N};
    dim3 blk(32, 4);
    cudaError_t err;
    if ((err = gs_pass<T>(L, st, rhs, e, true, true, nb, bt, s)) != cudaSuccess) return err;
    k_level_residual_restrict<T><<<grid3(C.n, C.n, nb, blk), blk, 0, s>>>(L.n, C.n, st, rhs, e, levR[l + 1], bt);
    count_launches(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = vcycle<T>(S, l + 1, levR[l + 1], levE[l + 1], levE, levR, s)) != cudaSuccess) return err;
    k_level_prolong_add<T><<<grid3(L.n, L.n, nb, blk), blk, 0, s>>>(L.n, C.n, levE[l + 1], e, bt);
    count_launches(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    return gs_pass<T>(L, st, rhs, e, false, false, nb, bt, s);
}

}  // namespace

cudaError_t launch_coarse_solve(const Solver &S, const double *dc, double *ec, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_coarse_solve(S, dc, ec, st);
    std::vector<double *> E(S.lev.size()), Rr(S.lev.size());
    for (size_t l = 0; l < S.lev.size(); ++l) { E[l] = S.lev[l].e; Rr[l] = S.lev[l].rhs; }
    return vcycle<double>(S, 0, dc, ec, E.data(), Rr.data(), st);
}

cudaError_t launch_inner_coarse(const Solver &S, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_inner_coarse(S, st);
    const MixedState &X = S.mx;
    return vcycle<float>(S, 0, X.dc, X.ec, X.lev_e.data(), X.lev_rhs.data(), st);
}

}  // namespace iga2l
