// kernels_coarse.cu -- second level of the two-level cycle (2D, FP64).
//
// Degree-1 discretisation on the 2h mesh (Section 3.3), approximated by one
// V(1,1) h-multigrid cycle with red-black Gauss-Seidel (Section 3.2), or solved
// exactly (Algorithm 1).  Level operators are the 9-point degree-1 stencils
// k_x m_y + m_x k_y with k = (-1, 2, -1)/H and m = (1, 4, 1) H/6; transfers are
// the exact embedding of nested degree-1 spaces (weights 1/2, 1, 1/2) and its
// transpose; the coarsest level (8 or fewer elements per axis) uses a dense
// inverse computed on the host.
#include <cuda_runtime.h>

#include "internal.h"

namespace iga2l {

namespace {

struct Stencil9 {
    double c[3][3];   // c[dy][dx], dx, dy in {0,1,2} <-> offsets -1, 0, +1
};

Stencil9 level_stencil(const Level &L)
{
    Stencil9 s;
    for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx) s.c[dy][dx] = L.k[dx] * L.mm[dy] + L.mm[dx] * L.k[dy];
    return s;
}

// Relax the sub-lattice {(2a+px, 2b+py)}: e += (rhs - A e) / A_diag.  No two points
// of a sub-lattice are coupled by the 9-point stencil.
__global__ void k_gs_sublattice(int n, int px, int py, Stencil9 st, const double *__restrict__ rhs,
                                double *__restrict__ e)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x, bidx = blockIdx.y * blockDim.y + threadIdx.y;
    const int x = 2 * a + px, y = 2 * bidx + py;
    if (x >= n || y >= n) return;
    double acc = 0.0;
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

// r = rhs - A e on one level
__global__ void k_level_residual(int n, Stencil9 st, const double *__restrict__ rhs,
                                 const double *__restrict__ e, double *__restrict__ r)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= n || y >= n) return;
    double acc = 0.0;
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
    r[(size_t)y * n + x] = rhs[(size_t)y * n + x] - acc;
}

// rc[J][I] = sum w_dy w_dx r[2J+dy][2I+dx], w = (1/2, 1, 1/2)
__global__ void k_level_restrict(int nf, int nc, const double *__restrict__ r, double *__restrict__ rc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= nc || J >= nc) return;
    const double w[3] = {0.5, 1.0, 0.5};
    double acc = 0.0;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const double *row = r + (size_t)(2 * J + dy) * nf + 2 * I;
        double s = 0.0;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) s = fma(w[dx], row[dx], s);
        acc = fma(w[dy], s, acc);
    }
    rc[(size_t)J * nc + I] = acc;
}

// e[y][x] += sum over the coarse points whose hats cover fine node (x, y)
__global__ void k_level_prolong_add(int nf, int nc, const double *__restrict__ ec, double *__restrict__ e)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nf || y >= nf) return;
    // fine index x is coarse I = (x-1)/2 when odd (weight 1); between I = x/2-1 and x/2 when even
    int Ix[2], Iy[2];
    double wx[2], wy[2];
    int nx, ny;
    if (x & 1) { Ix[0] = (x - 1) / 2; wx[0] = 1.0; nx = 1; }
    else { Ix[0] = x / 2 - 1; Ix[1] = x / 2; wx[0] = 0.5; wx[1] = 0.5; nx = 2; }
    if (y & 1) { Iy[0] = (y - 1) / 2; wy[0] = 1.0; ny = 1; }
    else { Iy[0] = y / 2 - 1; Iy[1] = y / 2; wy[0] = 0.5; wy[1] = 0.5; ny = 2; }
    double acc = 0.0;
    for (int b = 0; b < ny; ++b) {
        if (Iy[b] < 0 || Iy[b] >= nc) continue;
        double s = 0.0;
        for (int a = 0; a < nx; ++a) {
            if (Ix[a] < 0 || Ix[a] >= nc) continue;
            s = fma(wx[a], ec[(size_t)Iy[b] * nc + Ix[a]], s);
        }
        acc = fma(wy[b], s, acc);
    }
    e[(size_t)y * nf + x] += acc;
}

// x = Ainv rhs, one warp per row (dense inverse of the directly solved level)
__global__ void k_dense_matvec(int N, const double *__restrict__ Ainv, const double *__restrict__ rhs,
                               double *__restrict__ x)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= N) return;
    const double *row = Ainv + (size_t)warp * N;
    double s = 0.0;
    for (int j = lane; j < N; j += 32) s = fma(row[j], rhs[j], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) x[warp] = s;
}

dim3 grid2(int nx, int ny, dim3 blk)
{
    return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y);
}

// red-black order: red sub-lattices (0,0), (1,1) then black (1,0), (0,1)
constexpr int kGsSeq[4][2] = {{0, 0}, {1, 1}, {1, 0}, {0, 1}};

cudaError_t gs_pass(const Level &L, const Stencil9 &st, const double *rhs, double *e, bool forward,
                    cudaStream_t s)
{
    dim3 blk(32, 4);
    const int half = (L.n + 1) / 2;
    for (int t = 0; t < 4; ++t) {
        const int c = forward ? t : 3 - t;
        k_gs_sublattice<<<grid2(half, half, blk), blk, 0, s>>>(L.n, kGsSeq[c][0], kGsSeq[c][1], st, rhs, e);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t vcycle(const Solver &S, int l, const double *rhs, double *e, cudaStream_t s)
{
    const Level &L = S.lev[l];
    const int last = (int)S.lev.size() - 1;
    if (l == last) {
        const int N = S.ndirect;
        k_dense_matvec<<<(N * 32 + 255) / 256, 256, 0, s>>>(N, S.dinv, rhs, e);
        count_launches(1);
        return cudaGetLastError();
    }
    const Level &C = S.lev[l + 1];
    const Stencil9 st = level_stencil(L);
    dim3 blk(32, 4);
    cudaError_t err = cudaMemsetAsync(e, 0, sizeof(double) * L.N, s);
    if (err != cudaSuccess) return err;
    if ((err = gs_pass(L, st, rhs, e, true, s)) != cudaSuccess) return err;
    k_level_residual<<<grid2(L.n, L.n, blk), blk, 0, s>>>(L.n, st, rhs, e, L.r);
    count_launches(1);
    k_level_restrict<<<grid2(C.n, C.n, blk), blk, 0, s>>>(L.n, C.n, L.r, C.rhs);
    count_launches(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = vcycle(S, l + 1, C.rhs, C.e, s)) != cudaSuccess) return err;
    k_level_prolong_add<<<grid2(L.n, L.n, blk), blk, 0, s>>>(L.n, C.n, C.e, e);
    count_launches(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    return gs_pass(L, st, rhs, e, false, s);
}

}  // namespace

cudaError_t launch_coarse_solve(const Solver &S, const double *dc, double *ec, cudaStream_t st)
{
    return vcycle(S, 0, dc, ec, st);
}

}  // namespace iga2l
