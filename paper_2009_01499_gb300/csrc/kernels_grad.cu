// kernels_grad.cu -- differentiable source for the 2D solve.
//
// f(x, y) = sum_k a_k G(x; cx_k) G(y; cy_k), G(t; c) = exp(-(t - c)^2 / (2 w^2)), so the
// load b = (f, phi_ij) is separable per bump: b[j][i] = sum_k a_k gx_k[i] gy_k[j] with the
// 1D loads g_k[i] = int G(t; c_k) N_i(t) dt (Gauss quadrature, nq points per element).
// Given bbar = dL/db (the adjoint solution), the parameter gradient is
//   dL/da_k  = gy_k^T Bbar gx_k,   dL/dcx_k = a_k gy_k^T Bbar gx'_k,   dL/dcy_k = a_k gy'_k^T Bbar gx_k,
// with g'_k = int dG/dc N_i and Bbar the n x n matrix of bbar (row j, column i).
// All reductions run in a fixed order (deterministic gradients).
#include <cuda_runtime.h>

#include "internal.h"

namespace iga2l {

namespace {

// gbuf[((k*2 + axis)*2 + kind)*n + i]: kind 0 = g, kind 1 = dg/dc; axis 0 uses cx, 1 uses cy
__global__ void k_bump_1d(int m, int p, int nq, int n, const double *__restrict__ qx, const double *__restrict__ qw,
                          const double *__restrict__ qB, int nb, const double *__restrict__ theta, double w,
                          double *__restrict__ gbuf)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nb * 2 * n) return;
    const int i = idx % n, axis = (idx / n) % 2, k = idx / (2 * n);
    const double c = theta[3 * k + 1 + axis];
    const double inv_w2 = 1.0 / (w * w);
    // restricted function i is full function i+1, nonzero on elements e = i+1-p .. i+1
    const int e0 = max(0, i + 1 - p), e1 = min(m - 1, i + 1);
    double g = 0.0, gd = 0.0;
    for (int e = e0; e <= e1; ++e) {
        const int a = i + 1 - e;
        for (int q = 0; q < nq; ++q) {
            const size_t kq = (size_t)e * nq + q;
            const double t = qx[kq] - c;
            const double G = exp(-0.5 * t * t * inv_w2);
            const double wb = qw[kq] * qB[kq * (p + 1) + a];
            g = fma(wb, G, g);
            gd = fma(wb, t * inv_w2 * G, gd);
        }
    }
    gbuf[((size_t)(k * 2 + axis) * 2 + 0) * n + i] = g;
    gbuf[((size_t)(k * 2 + axis) * 2 + 1) * n + i] = gd;
}

__global__ void k_bump_assemble(int n, int nb, const double *__restrict__ theta, const double *__restrict__ gbuf,
                                double *__restrict__ b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n) return;
    double acc = 0.0;
    for (int k = 0; k < nb; ++k) {
        const double gx = gbuf[((size_t)(k * 2 + 0) * 2 + 0) * n + i];
        const double gy = gbuf[((size_t)(k * 2 + 1) * 2 + 0) * n + j];
        acc = fma(theta[3 * k] * gy, gx, acc);
    }
    b[(size_t)j * n + i] = acc;
}

// V[((k*2 + kind)*n + j] = sum_i Bbar[j][i] gx_k^{(kind)}[i]; one warp per (k, j)
__global__ void k_bump_rows(int n, int nb, const double *__restrict__ bbar, const double *__restrict__ gbuf,
                            double *__restrict__ V)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nb * n) return;
    const int j = warp % n, k = warp / n;
    const double *row = bbar + (size_t)j * n;
    const double *g0 = gbuf + ((size_t)(k * 2 + 0) * 2 + 0) * n;
    const double *g1 = gbuf + ((size_t)(k * 2 + 0) * 2 + 1) * n;
    double s0 = 0.0, s1 = 0.0;
    for (int i = lane; i < n; i += 32) {
        s0 = fma(row[i], g0[i], s0);
        s1 = fma(row[i], g1[i], s1);
    }
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, off);
        s1 += __shfl_down_sync(0xffffffffu, s1, off);
    }
    if (lane == 0) {
        V[((size_t)k * 2 + 0) * n + j] = s0;
        V[((size_t)k * 2 + 1) * n + j] = s1;
    }
}

// grad[3k + {0,1,2}] = (dL/da_k, dL/dcx_k, dL/dcy_k); one warp per bump
__global__ void k_bump_final(int n, int nb, const double *__restrict__ theta, const double *__restrict__ gbuf,
                             const double *__restrict__ V, double *__restrict__ grad)
{
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= nb) return;
    const double *gy = gbuf + ((size_t)(k * 2 + 1) * 2 + 0) * n;
    const double *gyd = gbuf + ((size_t)(k * 2 + 1) * 2 + 1) * n;
    const double *v0 = V + ((size_t)k * 2 + 0) * n, *v1 = V + ((size_t)k * 2 + 1) * n;
    double sa = 0.0, sx = 0.0, sy = 0.0;
    for (int j = lane; j < n; j += 32) {
        sa = fma(v0[j], gy[j], sa);
        sx = fma(v1[j], gy[j], sx);
        sy = fma(v0[j], gyd[j], sy);
    }
    for (int off = 16; off > 0; off >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, off);
        sx += __shfl_down_sync(0xffffffffu, sx, off);
        sy += __shfl_down_sync(0xffffffffu, sy, off);
    }
    if (lane == 0) {
        const double a = theta[3 * k];
        grad[3 * k + 0] = sa;
        grad[3 * k + 1] = a * sx;
        grad[3 * k + 2] = a * sy;
    }
}

__global__ void k_axpy(long long n, double alpha, const double *__restrict__ x, double *__restrict__ y)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(alpha, x[i], y[i]);
}

}  // namespace

cudaError_t launch_bump_load(const Solver &S, int nb, const double *theta, double w, double *b, cudaStream_t st)
{
    const int n = S.n;
    k_bump_1d<<<(nb * 2 * n + 127) / 128, 128, 0, st>>>(S.m, S.p, S.nq, n, S.qx, S.qw, S.qB, nb, theta, w, S.gbuf);
    k_bump_assemble<<<dim3((n + 127) / 128, n), 128, 0, st>>>(n, nb, theta, S.gbuf, b);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_bump_grad(const Solver &S, int nb, const double *theta, double w, const double *bbar,
                             double *grad, cudaStream_t st)
{
    const int n = S.n;
    double *V = S.gbuf + (size_t)kMaxBumps * 4 * n;
    k_bump_1d<<<(nb * 2 * n + 127) / 128, 128, 0, st>>>(S.m, S.p, S.nq, n, S.qx, S.qw, S.qB, nb, theta, w, S.gbuf);
    k_bump_rows<<<(nb * n * 32 + 255) / 256, 256, 0, st>>>(n, nb, bbar, S.gbuf, V);
    k_bump_final<<<(nb * 32 + 127) / 128, 128, 0, st>>>(n, nb, theta, S.gbuf, V, grad);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_axpy(long long n, double alpha, const double *x, double *y, cudaStream_t st)
{
    k_axpy<<<(int)((n + 255) / 256), 256, 0, st>>>(n, alpha, x, y);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace iga2l
