// kernels_fine.cu -- fine-level kernels of the two-level cycle (2D, FP64).
//
//   residual     d = b - A_p u (Algorithm 1) with per-CTA partial sums of d^2
//   schwarz      one colour phase of the multiplicative Schwarz step (Section 3.1.1)
//   restrict     d_c = (R (x) R) d, R = S^T D^{-1} M_p^1 (Sections 3.1.2, 3.3)
//   prolong_add  u += (R (x) R)^T e_c
//   mass2        b = (M (x) M) f
//
// A_p = K (x) M + M (x) K.  The 2D coefficient of DOF (x+a-p, y+b-p) in row
// (x, y) is K[x][a] M[y][b] + M[x][a] K[y][b]; rows 2p-1 .. n-2p of K and M are
// Toeplitz, so the stencil depends only on the (point class of x, point class of y)
// pair and is read from a small table that stays in L1.  On GB300 these FP64
// kernels are bound by the FP64 pipe, not by HBM.
#include <cuda_runtime.h>

#include "internal.h"

namespace iga2l {

namespace {

constexpr int kResTX = 32, kResTY = 8;   // residual tile (outputs per CTA)

// d = b - A u  (b != nullptr)  or  d = A u  (b == nullptr); part[cta] = sum d^2
template <int P>
__global__ void __launch_bounds__(kResTX *kResTY)
k_residual2d(int n, int npc, const double *__restrict__ stencil, const int *__restrict__ pcls,
             const double *__restrict__ u, const double *__restrict__ b, double *__restrict__ d,
             double *__restrict__ part)
{
    constexpr int W = 2 * P + 1;
    constexpr int SX = kResTX + 2 * P, SY = kResTY + 2 * P;
    __shared__ double su[SY][SX];
    __shared__ double red[kResTX * kResTY / 32];
    const int x0 = blockIdx.x * kResTX, y0 = blockIdx.y * kResTY;
    const int tid = threadIdx.x + kResTX * threadIdx.y;
    for (int t = tid; t < SX * SY; t += kResTX * kResTY) {
        const int ly = t / SX, lx = t % SX;
        const int gx = x0 + lx - P, gy = y0 + ly - P;
        su[ly][lx] = (gx >= 0 && gx < n && gy >= 0 && gy < n) ? u[(size_t)gy * n + gx] : 0.0;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    double dv = 0.0;
    if (x < n && y < n) {
        const double *st = stencil + (size_t)(pcls[y] * npc + pcls[x]) * (W * W);
        double acc = 0.0;
#pragma unroll
        for (int bb = 0; bb < W; ++bb)
#pragma unroll
            for (int aa = 0; aa < W; ++aa)
                acc = fma(__ldg(&st[bb * W + aa]), su[threadIdx.y + bb][threadIdx.x + aa], acc);
        dv = b ? b[(size_t)y * n + x] - acc : acc;
        if (d) d[(size_t)y * n + x] = dv;
    }
    if (part) {
        double s = dv * dv;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((tid & 31) == 0) red[tid >> 5] = s;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < kResTX * kResTY / 32; ++w) tot += red[w];
            part[blockIdx.x + gridDim.x * blockIdx.y] = tot;
        }
    }
}

// Fixed-order sum of the partials (deterministic norm).
__global__ void k_sum_partials(const double *__restrict__ part, int np, double *__restrict__ out)
{
    __shared__ double sh[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// One colour of the LATTICE schedule: the blocks centred at (ox + q i, oy + q j).
// S*S threads per Schwarz block: thread e computes the residual at block DOF e,
// then row e of A_B^{-1} times the block residual, and adds it to u.  Blocks of
// one colour neither share DOFs nor read each other's DOFs, so they run in parallel.
template <int P, int S>
__global__ void __launch_bounds__(256)
k_schwarz_lattice2d(int n, int npc, int nbc, int q, int ox, int oy, int nbx, int nblocks,
                    const double *__restrict__ stencil, const int *__restrict__ pcls,
                    const double *__restrict__ binv, const int *__restrict__ bcls,
                    double *__restrict__ u, const double *__restrict__ b)
{
    constexpr int W = 2 * P + 1, SS = S * S, R = (S - 1) / 2;
    constexpr int BPC = 256 / SS;   // Schwarz blocks per CTA
    __shared__ double rs[BPC * SS];
    const int lb = threadIdx.x / SS, e = threadIdx.x % SS;
    const int blk = blockIdx.x * BPC + lb;
    const bool active = lb < BPC && blk < nblocks;
    int cx = 0, cy = 0, x = -1, y = -1;
    bool inside = false;
    if (active) {
        cx = ox + q * (blk % nbx);
        cy = oy + q * (blk / nbx);
        x = cx - R + e % S;
        y = cy - R + e / S;
        inside = x >= 0 && x < n && y >= 0 && y < n;
    }
    double rv = 0.0;
    if (inside) {
        const double *st = stencil + (size_t)(pcls[y] * npc + pcls[x]) * (W * W);
        double acc = 0.0;
#pragma unroll
        for (int bb = 0; bb < W; ++bb) {
            const int yy = y + bb - P;
            if (yy < 0 || yy >= n) continue;
            const double *urow = u + (size_t)yy * n;
#pragma unroll
            for (int aa = 0; aa < W; ++aa) {
                const int xx = x + aa - P;
                if (xx >= 0 && xx < n) acc = fma(__ldg(&st[bb * W + aa]), urow[xx], acc);
            }
        }
        rv = b[(size_t)y * n + x] - acc;
    }
    if (threadIdx.x < BPC * SS) rs[threadIdx.x] = rv;
    __syncthreads();
    if (inside) {
        const double *Bi = binv + ((size_t)(bcls[cy] * nbc + bcls[cx]) * SS + e) * SS;
        const double *rb = rs + lb * SS;
        double ev = 0.0;
#pragma unroll
        for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[f]), rb[f], ev);
        u[(size_t)y * n + x] += ev;
    }
}

// t[j][I] = sum_w Rb[I][w] d[j][Rlo[I]+w]   (x direction, n rows x nc)
__global__ void k_restrict_x(int n, int nc, int wr, const double *__restrict__ Rb,
                             const int *__restrict__ Rlo, const double *__restrict__ d,
                             double *__restrict__ t)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (I >= nc) return;
    const int lo = Rlo[I];
    const double *row = d + (size_t)j * n;
    double acc = 0.0;
    for (int w = 0; w < wr; ++w) {
        const int i = lo + w;
        if (i < n) acc = fma(Rb[(size_t)I * wr + w], row[i], acc);
    }
    t[(size_t)j * nc + I] = acc;
}

// dc[J][I] = sum_w Rb[J][w] t[Rlo[J]+w][I]   (y direction)
__global__ void k_restrict_y(int n, int nc, int wr, const double *__restrict__ Rb,
                             const int *__restrict__ Rlo, const double *__restrict__ t,
                             double *__restrict__ dc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
    if (I >= nc) return;
    const int lo = Rlo[J];
    double acc = 0.0;
    for (int w = 0; w < wr; ++w) {
        const int j = lo + w;
        if (j < n) acc = fma(Rb[(size_t)J * wr + w], t[(size_t)j * nc + I], acc);
    }
    dc[(size_t)J * nc + I] = acc;
}

// t2[J][i] = sum_w Cb[i][w] ec[J][Clo[i]+w]   (x direction of R^T)
__global__ void k_prolong_x(int n, int nc, int wc, const double *__restrict__ Cb,
                            const int *__restrict__ Clo, const double *__restrict__ ec,
                            double *__restrict__ t2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
    if (i >= n) return;
    const int lo = Clo[i];
    double acc = 0.0;
    for (int w = 0; w < wc; ++w) {
        const int I = lo + w;
        if (I < nc) acc = fma(Cb[(size_t)i * wc + w], ec[(size_t)J * nc + I], acc);
    }
    t2[(size_t)J * n + i] = acc;
}

// u[j][i] += sum_w Cb[j][w] t2[Clo[j]+w][i]   (y direction of R^T)
__global__ void k_prolong_y(int n, int nc, int wc, const double *__restrict__ Cb,
                            const int *__restrict__ Clo, const double *__restrict__ t2,
                            double *__restrict__ u)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n) return;
    const int lo = Clo[j];
    double acc = 0.0;
    for (int w = 0; w < wc; ++w) {
        const int J = lo + w;
        if (J < nc) acc = fma(Cb[(size_t)j * wc + w], t2[(size_t)J * n + i], acc);
    }
    u[(size_t)j * n + i] += acc;
}

// b[j][i] = sum_b M[j][b] sum_a M[i][a] f[j+b-p][i+a-p]
template <int P>
__global__ void k_mass2d(int n, const double *__restrict__ Mb, const double *__restrict__ f,
                         double *__restrict__ b)
{
    constexpr int W = 2 * P + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n) return;
    double acc = 0.0;
    for (int bb = 0; bb < W; ++bb) {
        const int jj = j + bb - P;
        if (jj < 0 || jj >= n) continue;
        double s = 0.0;
        for (int aa = 0; aa < W; ++aa) {
            const int ii = i + aa - P;
            if (ii >= 0 && ii < n) s = fma(Mb[(size_t)i * W + aa], f[(size_t)jj * n + ii], s);
        }
        acc = fma(Mb[(size_t)j * W + bb], s, acc);
    }
    b[(size_t)j * n + i] = acc;
}

template <int P>
cudaError_t residual_p(const Solver &S, const double *u, const double *b, double *d, double *part,
                       cudaStream_t st)
{
    dim3 blk(kResTX, kResTY), grd((S.n + kResTX - 1) / kResTX, (S.n + kResTY - 1) / kResTY);
    k_residual2d<P><<<grd, blk, 0, st>>>(S.n, S.ht.npc, S.stencil, S.pcls, u, b, d, part);
    count_launches(1);
    return cudaGetLastError();
}

template <int P, int SB>
cudaError_t schwarz_p(const Solver &S, double *u, const double *b, bool reverse, cudaStream_t st)
{
    constexpr int BPC = 256 / (SB * SB);
    const int q = S.q, ncol = q * q;
    for (int t = 0; t < ncol; ++t) {
        const int c = reverse ? ncol - 1 - t : t;
        // colour c visits offsets (rank_x g mod q, rank_y g mod q)
        const int ox = ((c % q) * S.g) % q, oy = ((c / q) * S.g) % q;
        const int nbx = (S.n - ox + q - 1) / q, nby = (S.n - oy + q - 1) / q;
        const int nblocks = nbx * nby;
        if (nblocks <= 0) continue;
        const int grid = (nblocks + BPC - 1) / BPC;
        k_schwarz_lattice2d<P, SB><<<grid, 256, 0, st>>>(S.n, S.ht.npc, S.ht.nbc, q, ox, oy, nbx,
                                                          nblocks, S.stencil, S.pcls, S.binv,
                                                          S.bcls, u, b);
        count_launches(1);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace

int residual_partials(const Solver &S)
{
    return ((S.n + kResTX - 1) / kResTX) * ((S.n + kResTY - 1) / kResTY);
}

cudaError_t launch_residual(const Solver &S, const double *u, const double *b, double *d,
                            double *part, cudaStream_t st)
{
    switch (S.p) {
    case 2: return residual_p<2>(S, u, b, d, part, st);
    case 3: return residual_p<3>(S, u, b, d, part, st);
    case 4: return residual_p<4>(S, u, b, d, part, st);
    case 5: return residual_p<5>(S, u, b, d, part, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_apply_A(const Solver &S, const double *u, double *y, cudaStream_t st)
{
    return launch_residual(S, u, nullptr, y, nullptr, st);
}

cudaError_t launch_norm_finish(const Solver &S, const double *part, double *out, cudaStream_t st)
{
    k_sum_partials<<<1, 1024, 0, st>>>(part, residual_partials(S), out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_schwarz(const Solver &S, double *u, const double *b, bool reverse,
                           cudaStream_t st)
{
    if (S.s == 3) {
        switch (S.p) {
        case 2: return schwarz_p<2, 3>(S, u, b, reverse, st);
        case 3: return schwarz_p<3, 3>(S, u, b, reverse, st);
        case 4: return schwarz_p<4, 3>(S, u, b, reverse, st);
        default: break;
        }
    } else if (S.s == 5 && S.p == 5) {
        return schwarz_p<5, 5>(S, u, b, reverse, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_restrict(const Solver &S, const double *d, double *dc, cudaStream_t st)
{
    const int nc = S.nc, n = S.n;
    k_restrict_x<<<dim3((nc + 127) / 128, n), 128, 0, st>>>(n, nc, S.ht.wr, S.Rb, S.Rlo, d, S.t);
    count_launches(1);
    k_restrict_y<<<dim3((nc + 127) / 128, nc), 128, 0, st>>>(n, nc, S.ht.wr, S.Rb, S.Rlo, S.t, dc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(const Solver &S, const double *ec, double *u, cudaStream_t st)
{
    const int nc = S.nc, n = S.n;
    k_prolong_x<<<dim3((n + 127) / 128, nc), 128, 0, st>>>(n, nc, S.ht.wc, S.Cb, S.Clo, ec, S.t2);
    count_launches(1);
    k_prolong_y<<<dim3((n + 127) / 128, n), 128, 0, st>>>(n, nc, S.ht.wc, S.Cb, S.Clo, S.t2, u);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mass2(const Solver &S, const double *f, double *b, cudaStream_t st)
{
    dim3 grd((S.n + 127) / 128, S.n);
    switch (S.p) {
    case 2: k_mass2d<2><<<grd, 128, 0, st>>>(S.n, S.Mb, f, b); break;
    count_launches(1);
    case 3: k_mass2d<3><<<grd, 128, 0, st>>>(S.n, S.Mb, f, b); break;
    count_launches(1);
    case 4: k_mass2d<4><<<grd, 128, 0, st>>>(S.n, S.Mb, f, b); break;
    count_launches(1);
    case 5: k_mass2d<5><<<grd, 128, 0, st>>>(S.n, S.Mb, f, b); break;
    count_launches(1);
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace iga2l
