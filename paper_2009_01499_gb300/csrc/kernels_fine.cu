// kernels_fine.cu -- fine-level kernels of the two-level cycle (2D).
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
// pair and is read from a small table that stays in L1.
//
// Every kernel is templated on its storage/arithmetic type: double for the FP64
// form, float for the inner cycle of the mixed-precision form (FP32 storage and
// FP32 FMA), whose boundary-class block solves still use the FP64 inverses.  On
// GB300 the FP64 kernels are bound by the FP64 pipe, not by HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>

#include "device_util.cuh"
#include "internal.h"
#include "tc_util.cuh"

namespace iga2l {

namespace {

constexpr int kResTX = 32, kResTY = 8;   // residual tile (outputs per CTA)

// Fixed-order sum of the partials (deterministic norm).
__global__ void k_sum_partials(const double *__restrict__ part, int np, double *__restrict__ out)
{
    __shared__ double sh[1024];
    part += (size_t)blockIdx.x * np;   // one problem per CTA
    out += blockIdx.x;
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
// With T = float, blocks of the interior class use the FP32 inverse and the other
// (boundary) classes the FP64 inverse binv64.  A CTA takes BPC <= 256 / S^2 blocks
// (blockDim = BPC S^2 rounded up to a warp); the launch picks BPC among compiled
// variants so that the colour's CTAs spread evenly over the SMs (lattice_bpc).
template <int P, int S, int BPC, typename T>
__global__ void __launch_bounds__(256)
k_schwarz_lattice2d(int n, int npc, int nbc, int q, int ox, int oy, int nbx, int nblocks,
                    const T *__restrict__ stencil, const int *__restrict__ pcls,
                    const T *__restrict__ binv, const double *__restrict__ binv64, int interior,
                    const int *__restrict__ bcls, T *__restrict__ u, const T *__restrict__ b, BatchRef bt)
{
    constexpr int W = 2 * P + 1, SS = S * S, R = (S - 1) / 2;
    __shared__ T rs[BPC * SS];
    pdl_wait();
    if (bt.active && !bt.active[blockIdx.y]) return;
    u += blockIdx.y * bt.vec;
    b += blockIdx.y * bt.vec;
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
    T rv = T(0);
    if (inside) {
        const T *st = stencil + (size_t)(pcls[y] * npc + pcls[x]) * (W * W);
        T acc = T(0);
#pragma unroll
        for (int bb = 0; bb < W; ++bb) {
            const int yy = y + bb - P;
            if (yy < 0 || yy >= n) continue;
            const T *urow = u + (size_t)yy * n;
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
        const int cls = bcls[cy] * nbc + bcls[cx];
        const T *rb = rs + lb * SS;
        // (binv, binv64: every class's inverse transposed, [class][f][e]: the lanes of a block
        // read consecutive words)
        if (sizeof(T) == sizeof(double) || cls == interior || !binv64) {
            const T *Bi = binv + (size_t)cls * SS * SS + e;
            T ev = T(0);
#pragma unroll
            for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[(size_t)f * SS]), rb[f], ev);
            u[(size_t)y * n + x] += ev;
        } else {
            const double *Bi = binv64 + (size_t)cls * SS * SS + e;
            double ev = 0.0;
#pragma unroll
            for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[(size_t)f * SS]), (double)rb[f], ev);
            u[(size_t)y * n + x] += (T)ev;
        }
    }
}

// Interior rows of the 1D stiffness and mass matrices, scaled to be independent of h
// (k = h K_row, m = M_row / h): the interior 2D coefficient K_y[b] M_x[a] + M_y[b] K_x[a]
// equals k[b] m[a] + m[b] k[a].  Stored as pairs (k[a], m[a]) for the packed y pass and
// (m[a], k[a]) for the packed x pass; written once per device and degree.
__constant__ double2 c_km1d[kMaxP + 1][2 * kMaxP + 1], c_mk1d[kMaxP + 1][2 * kMaxP + 1];
__constant__ float2 c_km1f[kMaxP + 1][2 * kMaxP + 1], c_mk1f[kMaxP + 1][2 * kMaxP + 1];

template <typename T>
__device__ __forceinline__ typename Vec2<T>::type ckm1(int p, int a);
template <typename T>
__device__ __forceinline__ typename Vec2<T>::type cmk1(int p, int a);
template <>
__device__ __forceinline__ double2 ckm1<double>(int p, int a) { return c_km1d[p][a]; }
template <>
__device__ __forceinline__ float2 ckm1<float>(int p, int a) { return c_km1f[p][a]; }
template <>
__device__ __forceinline__ double2 cmk1<double>(int p, int a) { return c_mk1d[p][a]; }
template <>
__device__ __forceinline__ float2 cmk1<float>(int p, int a) { return c_mk1f[p][a]; }

// d = b - A u  (b != nullptr)  or  d = A u  (b == nullptr), arithmetic in T, output
// stored as TO; part[cta] = sum of d^2 (in double) when part != nullptr.  A TX x TY tile
// of outputs per CTA (32 x 8 in FP32, 64 x 8 in FP64) with u (tile + halo p) in shared
// memory and the y-then-x sum factorisation A u = sum_b K_y[b] (sum_a M_x[a] u) + M_y[b]
// (sum_a K_x[a] u): first the pairs (K_y u, M_y u) of every output row at every window
// column, then per output the x sums (2(2p+1)(1 + 2p/TX) + 2(2p+1) FMAs per output instead
// of (2p+1)^2; in interior tiles the symmetric rows make the y pass p adds and 2(p+1)
// FMAs per pair).  Interior tiles take the interior 1D rows from constant memory; boundary
// tiles the 1D rows of their own rows and columns, scaled the same way (h K, M / h).
template <int P, typename T, typename TO, int TX = kResTX, int TY = kResTY>
__global__ void __launch_bounds__(TX *TY)
k_residual2d(int n, const T *__restrict__ kband, const T *__restrict__ mband, const T *__restrict__ u,
             const T *__restrict__ b, TO *__restrict__ d, double *__restrict__ part, unsigned int *__restrict__ done,
             double *__restrict__ norm2, BatchRef bt)
{
    using T2 = typename Vec2<T>::type;
    constexpr int W = 2 * P + 1;
    constexpr int SX = TX + 2 * P, SY = TY + 2 * P;
    __shared__ T su[SY][SX];
    __shared__ T2 yv[TY][SX];
    __shared__ T2 kmy[TY][W], mkx[TX][W];   // boundary tiles
    __shared__ double red[TX * TY / 32];
    const int z = blockIdx.z;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x + TX * threadIdx.y;
    constexpr int NT = TX * TY;
    constexpr int K = (SX * SY + NT - 1) / NT;
    const bool fast = x0 >= 2 * P - 1 && x0 + TX - 1 <= n - 2 * P && y0 >= 2 * P - 1 &&
                      y0 + TY - 1 <= n - 2 * P;
    if (!fast) {   // constant tables: read before the wait
        const T h = T(1) / T(n - P + 2), hinv = T(n - P + 2);
        for (int t = tid; t < (TX + TY) * W; t += NT) {
            const int row = t / W, a = t - row * W;
            if (row < TY) {
                const int gy = y0 + row;
                T2 km;
                km.x = gy < n ? kband[(size_t)gy * W + a] * h : T(0);
                km.y = gy < n ? mband[(size_t)gy * W + a] * hinv : T(0);
                kmy[row][a] = km;
            } else {
                const int gx = x0 + row - TY;
                T2 mk;
                mk.x = gx < n ? mband[(size_t)gx * W + a] * hinv : T(0);
                mk.y = gx < n ? kband[(size_t)gx * W + a] * h : T(0);
                mkx[row - TY][a] = mk;
            }
        }
    }
    pdl_wait();
    if (bt.active && !bt.active[z]) return;
    u += z * bt.vec;
    if (b) b += z * bt.vec;
    if (d) d += z * bt.vec;
    if (part) part += z * bt.aux;
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int t = tid + k * NT;
        const int gx = x0 + t % SX - P, gy = y0 + t / SX - P;
        v[k] = (t < SX * SY && gx >= 0 && gx < n && gy >= 0 && gy < n) ? u[(size_t)gy * n + gx] : T(0);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int t = tid + k * NT;
        if (t < SX * SY) su[t / SX][t % SX] = v[k];
    }
    __syncthreads();
    for (int pt = tid; pt < TY * SX; pt += NT) {
        const int r = pt / SX, c = pt - r * SX;
        T2 y = splat2<T2>(T(0));
        if (fast) {
            // interior rows are symmetric (k[P - j] = k[P + j], the same for m): the two taps
            // at distance j share one multiply-add per half of the pair
            y = fma2(ckm1<T>(P, P), splat2<T2>(su[r + P][c]), y);
#pragma unroll
            for (int j = 1; j <= P; ++j) y = fma2(ckm1<T>(P, P - j), splat2<T2>(su[r + P - j][c] + su[r + P + j][c]), y);
        } else {
#pragma unroll
            for (int bb = 0; bb < W; ++bb) y = fma2(kmy[r][bb], splat2<T2>(su[r + bb][c]), y);
        }
        yv[r][c] = y;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    T dv = T(0);
    if (x < n && y < n) {
        T2 s2 = splat2<T2>(T(0));
        if (fast) {
#pragma unroll
            for (int a = 0; a < W; ++a) s2 = fma2(cmk1<T>(P, a), yv[threadIdx.y][threadIdx.x + a], s2);
        } else {
#pragma unroll
            for (int a = 0; a < W; ++a) s2 = fma2(mkx[threadIdx.x][a], yv[threadIdx.y][threadIdx.x + a], s2);
        }
        const T acc = s2.x + s2.y;
        dv = b ? b[(size_t)y * n + x] - acc : acc;
        if (d) d[(size_t)y * n + x] = (TO)dv;
    }
    if (part) {
        double s = (double)dv * (double)dv;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((tid & 31) == 0) red[tid >> 5] = s;
        __syncthreads();
        __shared__ bool last;
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < TX * TY / 32; ++w) tot += red[w];
            part[blockIdx.x + gridDim.x * blockIdx.y] = tot;
            last = false;
            if (norm2) {   // the last CTA of this problem to finish sums the partials
                __threadfence();
                last = atomicAdd(&done[z], 1u) == gridDim.x * gridDim.y - 1;
            }
        }
        __syncthreads();
        if (last) {
            // fixed-order sum of the partials (deterministic), then re-arm the counter
            __threadfence();
            const int np = gridDim.x * gridDim.y;
            constexpr int NT = TX * TY;
            __shared__ double sh[NT];
            double acc = 0.0;
            for (int i = tid; i < np; i += NT) acc += __ldcg(&part[i]);
            sh[tid] = acc;
            __syncthreads();
            for (int w = NT / 2; w > 0; w >>= 1) {
                if (tid < w) sh[tid] += sh[tid + w];
                __syncthreads();
            }
            if (tid == 0) {
                norm2[z] = sh[0];
                done[z] = 0u;
            }
        }
    }
}

// One colour of the LATTICE schedule with the residual sum-factorised and the work
// packed across lanes (the FP32 sweeps, where the direct form is bound by its loads).  A CTA of 256 threads takes NB
// consecutive blocks of the colour, centres (ox + q i, oy + q j):
//   1. thread (block, window column c) loads the column slice of u (S + 2P values) and
//      forms for each block row r the pair (sum_b K_y[b] u, sum_b M_y[b] u);
//   2. thread per block DOF: the x sums sum_a M_x[a] Y1 + K_x[a] Y2, r = b - A u;
//   3. thread per block DOF: row e of the block's inverse times r, added to u.
// Interior rows/columns take the h-scaled interior 1D rows from constant memory, the
// others their own 1D rows (scaled the same way); with T = float the boundary block
// classes use the FP64 inverses binv64 when given.
// Block (i, j) of a colour's nbx-wide block grid from an index over the grid minus the
// rectangle [ix0, ix0 + nix) x [iy0, iy0 + niy) (the blocks the tensor-core kernel takes);
// with nix = niy = 0 this is the plain row-major order.
__device__ __forceinline__ void frame_block(int f, int nbx, int ix0, int iy0, int nix, int niy, int &i, int &j)
{
    const int top = iy0 * nbx, cnt = nbx - nix;
    if (f < top || niy == 0) { i = f % nbx; j = f / nbx; return; }
    f -= top;
    if (f < niy * cnt) {
        const int row = f / cnt, c = f - row * cnt;
        j = iy0 + row;
        i = c < ix0 ? c : ix0 + nix + (c - ix0);
        return;
    }
    f -= niy * cnt;
    j = iy0 + niy + f / nbx;
    i = f % nbx;
}

// Resident CTAs per SM the register allocation must allow, so that a 1024^2 colour (4.1 to
// 7.7 CTAs of 256 threads per SM for p = 2..6) runs in one wave
constexpr int lattice_sf_minb(int p) { return p == 2 ? 8 : (p == 3 ? 6 : (p == 4 ? 7 : (p <= 6 ? 5 : 4))); }

// Shared memory of one CTA of the per-colour FP32 step (NT threads).
template <int P, int S, typename T, int NT>
struct SfSmem {
    using T2 = typename Vec2<T>::type;
    static constexpr int SS = S * S, WIN = S + 2 * P, NB = NT / WIN, YS = WIN | 1;
    T2 yb[NB][S][YS];
    T rs[NB][SS];
    T sub[NB][SS];   // u at the block's DOFs (from the window columns)
    T sbb[NB][SS];   // b at the block's DOFs
    T sbi[SS * SS];
    int scx[NB], scy[NB], scls[NB];   // block centres and classes (cls < 0: no block)
};

// The work of one CTA of a colour phase: blocks vb NB .. vb NB + NB - 1 of the colour (in the
// numbering of frame_block, which skips the rectangle [ix0, ix0 + nix) x [iy0, iy0 + niy)).
// binv and binv_lo hold every class's inverse transposed ([class][f][e]).
// All NT threads call it; `pre` runs between the constant-table reads and the first
// dependent read (the programmatic-launch wait) and returns whether the CTA goes on (the
// same answer in every thread).
template <int P, int S, typename T, int NT, typename Pre>
__device__ __forceinline__ void schwarz_sf_cta(SfSmem<P, S, T, NT> &sm, int vb, int n, int nbc, int q, int ox,
                                               int oy, int nbx, int ix0, int iy0, int nix, int niy, int nblocks,
                                               const T *__restrict__ kband, const T *__restrict__ mband,
                                               const T *__restrict__ binv, const float *__restrict__ binv_lo,
                                               int interior, T *__restrict__ u, const T *__restrict__ b, Pre pre)
{
    using T2 = typename Vec2<T>::type;
    constexpr int W = 2 * P + 1, SS = S * S, R = (S - 1) / 2, WIN = S + 2 * P, PCI = 2 * P - 1;
    constexpr int NB = SfSmem<P, S, T, NT>::NB, L = P - 1 + R;
    auto &yb = sm.yb;
    auto &rs = sm.rs;
    auto &sub = sm.sub;
    auto &sbb = sm.sbb;
    auto &sbi = sm.sbi;
    auto &scx = sm.scx;
    auto &scy = sm.scy;
    auto &scls = sm.scls;
    const int tid = threadIdx.x;
    for (int i = tid; i < SS * SS; i += NT) sbi[i] = binv[(size_t)interior * SS * SS + i];   // constant table (transposed)
    const int blk0 = vb * NB;
    if (tid < NB) {   // the CTA's blocks, once (frame_block divides by the colour's row length)
        const int blk = blk0 + tid;
        int cls = -1, cx = 0, cy = 0;
        if (blk < nblocks) {
            int bi_, bj_;
            frame_block(blk, nbx, ix0, iy0, nix, niy, bi_, bj_);
            cx = ox + q * bi_;
            cy = oy + q * bj_;
            const int bx = cx < L ? cx : (cx > n - 1 - L ? 2 * L - (n - 1 - cx) : L);
            const int by = cy < L ? cy : (cy > n - 1 - L ? 2 * L - (n - 1 - cy) : L);
            cls = by * nbc + bx;
            if (cls != interior) {   // the class's inverse into L1 now, for phase 3
                constexpr int LINES = (SS * SS * (int)sizeof(T) + 127) / 128;
                const char *m = reinterpret_cast<const char *>(binv + (size_t)cls * SS * SS);
                const char *ml = binv_lo ? reinterpret_cast<const char *>(binv_lo + (size_t)cls * SS * SS) : nullptr;
                for (int l = 0; l < LINES; ++l) {
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(m + 128 * l));
                    if (ml) asm volatile("prefetch.global.L1 [%0];" ::"l"(ml + 128 * l));
                }
            }
        }
        scx[tid] = cx;
        scy[tid] = cy;
        scls[tid] = cls;
    }
    if (!pre()) return;
    __syncthreads();
    const T h = T(1) / T(n - P + 2), hinv = T(n - P + 2);   // boundary rows and columns only
    // 1. thread (block j, window column c): the column's WIN values of u and, for the block's
    //    own columns, its S values of b -- every global load of the launch in one round trip --
    //    then the pairs (sum_b K_y[b] u, sum_b M_y[b] u) of the block's S rows
    if (tid < NB * WIN) {
        const int j = tid / WIN, c = tid - j * WIN;
        if (scls[j] >= 0) {
            const int cx = scx[j], cy = scy[j];
            const int x = cx - R - P + c;
            const bool xin = x >= 0 && x < n, own = c >= P && c < P + S;
            T v[WIN], bv[S];
#pragma unroll
            for (int k = 0; k < WIN; ++k) {
                const int y = cy - R - P + k;
                v[k] = (xin && y >= 0 && y < n) ? u[(size_t)y * n + x] : T(0);
            }
#pragma unroll
            for (int r = 0; r < S; ++r) {
                const int y = cy - R + r;
                bv[r] = (own && xin && y >= 0 && y < n) ? b[(size_t)y * n + x] : T(0);
            }
            if (own)
#pragma unroll
                for (int r = 0; r < S; ++r) {
                    sub[j][r * S + c - P] = v[P + r];
                    sbb[j][r * S + c - P] = bv[r];
                }
            const bool yint = cy - R >= PCI && cy + R <= n - 2 * P;
#pragma unroll
            for (int r = 0; r < S; ++r) {
                T2 acc;
                if (yint) {
                    // interior rows are symmetric: the taps at distance jj share one multiply-add
                    acc = fma2(ckm1<T>(P, P), splat2<T2>(v[r + P]), splat2<T2>(T(0)));
#pragma unroll
                    for (int jj = 1; jj <= P; ++jj)
                        acc = fma2(ckm1<T>(P, P - jj), splat2<T2>(v[r + P - jj] + v[r + P + jj]), acc);
                } else {
                    acc = splat2<T2>(T(0));
                    const int gy = cy - R + r;
                    if (gy >= 0 && gy < n) {
#pragma unroll
                        for (int bb = 0; bb < W; ++bb) {
                            T2 km;
                            km.x = kband[(size_t)gy * W + bb] * h;
                            km.y = mband[(size_t)gy * W + bb] * hinv;
                            acc = fma2(km, splat2<T2>(v[r + bb]), acc);
                        }
                    }
                }
                yb[j][r][c] = acc;
            }
        }
    }
    __syncthreads();
    // 2. x pass and block residuals (shared memory only)
    for (int o = tid; o < NB * SS; o += NT) {
        const int j = o / SS, e = o - j * SS, ey = e / S, ex = e - ey * S;
        if (scls[j] < 0) continue;
        const int cx = scx[j], cy = scy[j];
        const int x = cx - R + ex, y = cy - R + ey;
        T r = T(0);
        if (x >= 0 && x < n && y >= 0 && y < n) {
            const bool xint = cx - R >= PCI && cx + R <= n - 2 * P;
            T2 a0 = splat2<T2>(T(0)), a1 = a0;
            if (xint) {
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    T2 &acc = (a & 1) ? a1 : a0;
                    acc = fma2(cmk1<T>(P, a), yb[j][ey][ex + a], acc);
                }
            } else {
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    T2 mk;
                    mk.x = mband[(size_t)x * W + a] * hinv;
                    mk.y = kband[(size_t)x * W + a] * h;
                    T2 &acc = (a & 1) ? a1 : a0;
                    acc = fma2(mk, yb[j][ey][ex + a], acc);
                }
            }
            const T2 acc = add2(a0, a1);
            r = sbb[j][e] - (acc.x + acc.y);
        }
        rs[j][e] = r;
    }
    __syncthreads();
    // 3. block solves: interior class from shared memory, boundary classes from their own
    //    inverse (FP64 rows as FP32 pairs by compensated arithmetic when binv_lo is given)
    for (int o = tid; o < NB * SS; o += NT) {
        const int j = o / SS, e = o - j * SS;
        const int cls = scls[j];
        if (cls < 0) continue;
        const int x = scx[j] - R + e % S, y = scy[j] - R + e / S;
        if (x < 0 || x >= n || y < 0 || y >= n) continue;
        T ev = T(0);
        if (cls == interior) {
            const T *Bi = sbi + e;
            T e1 = T(0);
#pragma unroll
            for (int f = 0; f < SS; ++f) {
                T &acc = (f & 1) ? e1 : ev;
                acc = fma(Bi[f * SS], rs[j][f], acc);
            }
            ev += e1;
        } else if (sizeof(T) == sizeof(double) || !binv_lo) {
            const T *Bi = binv + (size_t)cls * SS * SS + e;
#pragma unroll
            for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[(size_t)f * SS]), rs[j][f], ev);
        } else if constexpr (sizeof(T) == sizeof(float)) {
            const size_t col = (size_t)cls * SS * SS + e;
            ev = dot2_row<SS, SS>(binv + col, binv_lo + col, &rs[j][0]);
        }
        u[(size_t)y * n + x] = sub[j][e] + ev;
    }
}

template <int P, int S, typename T>
__global__ void __launch_bounds__(256, lattice_sf_minb(P))
k_schwarz_lattice2d_sf(int n, int nbc, int q, int ox, int oy, int nbx, int ix0, int iy0, int nix, int niy,
                       int nblocks,
                       const T *__restrict__ kband, const T *__restrict__ mband,
                       const T *__restrict__ binv, const float *__restrict__ binv_lo, int interior,
                       T *__restrict__ u, const T *__restrict__ b, BatchRef bt)
{
    __shared__ SfSmem<P, S, T, 256> sm;
    u += blockIdx.y * bt.vec;
    b += blockIdx.y * bt.vec;
    schwarz_sf_cta<P, S, T, 256>(sm, blockIdx.x, n, nbc, q, ox, oy, nbx, ix0, iy0, nix, niy, nblocks, kband, mband,
                                 binv, binv_lo, interior, u, b, [&] {
                                     pdl_wait();
                                     return !(bt.active && !bt.active[blockIdx.y]);
                                 });
}

// One LATTICE colour of the FP32 inner cycle with the interior blocks on the tensor cores
// (IGA2L_MIXED_TF32).  The grid's first nfc CTAs take the colour's frame (the blocks outside
// the interior rectangle) with the SIMT step above; each other CTA takes a TBX x TBY tile of
// the interior rectangle (M = 128 blocks) and computes its corrections as D = X G^T:
//   * G (NP x KP, built on the host in the operand layout) arrives by one bulk asynchronous
//     copy (cp.async.bulk, completion on an mbarrier), issued before the wait for the
//     previous grid since G is constant;
//   * the region of u the tile's patches cover (RW x RH, coalesced rows) and the blocks' b
//     values are read once; X = [b_B ; u_patch] is built from shared memory in 16-byte
//     pieces (four consecutive k of one row), rounded to TF32;
//   * one thread issues the tcgen05.mma chain (kind::tf32, FP32 accumulator in tensor
//     memory) and commits it to a second mbarrier; both waits are bounded;
//   * each block's row of D is read back (tcgen05.ld) and u = u_old + e is written, u_old
//     from the staged region.
// Blocks of one colour share no DOF and read no DOF another writes, so all CTAs run
// independently.
struct TcColourArgs {
    int n, nbc, q, ox, oy, nbx, ix0, iy0, nix, niy, ntx, nfc, nframe, interior, skip_copy;
    long long budget;
    const float *kband, *mband, *binv, *binv_lo, *gtc, *b;
    float *u;
    int *status;
};

constexpr int tc_colour_minb(int p) { return p == 2 ? 3 : (p == 5 ? 1 : 2); }

template <int P, int S>
__global__ void __launch_bounds__(256, tc_colour_minb(P)) k_schwarz_tc_colour(const TcColourArgs a)
{
    using G = TcGeom<P, S>;
    constexpr int SS = G::SS, R = G::R, KU = G::KU, KP = G::KP, NP = G::NP, M = G::M;
    constexpr int TBX = G::TBX, TBY = G::TBY;
    constexpr int NT = 256, NWARP = NT / 32;
    extern __shared__ __align__(1024) unsigned char dyn[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if ((int)blockIdx.x < a.nfc) {   // frame blocks: the SIMT step
        auto &sm = *reinterpret_cast<SfSmem<P, S, float, NT> *>(dyn);
        schwarz_sf_cta<P, S, float, NT>(sm, blockIdx.x, a.n, a.nbc, a.q, a.ox, a.oy, a.nbx, a.ix0, a.iy0, a.nix,
                                        a.niy, a.nframe, a.kband, a.mband, a.binv, a.binv_lo, a.interior, a.u, a.b,
                                        [] {
                                            pdl_wait();
                                            return true;
                                        });
        return;
    }
    float *sX = reinterpret_cast<float *>(dyn);
    float *sG = reinterpret_cast<float *>(dyn + G::XB);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(dyn + G::XB + G::GB);   // [0]: MMA, [1]: copy of G
    uint32_t *tslot = reinterpret_cast<uint32_t *>(dyn + G::XB + G::GB + 16);
    int *s_mma = reinterpret_cast<int *>(dyn + G::XB + G::GB + 20);   // 1: G landed, the chain was issued
    int *sOff = reinterpret_cast<int *>(dyn + G::XB + G::GB + G::BARB);   // patch column k -> region offset
    int *sRb = sOff + KP;                                                 // block row r -> region offset
    float *sR = reinterpret_cast<float *>(sRb + M);                       // the region of u
    const int n = a.n, q = a.q, RW = G::RW(q), RH = G::RH(q);
    const int t = blockIdx.x - a.nfc, tx = t % a.ntx, ty = t / a.ntx;
    const int bi0 = a.ix0 + TBX * tx, bj0 = a.iy0 + TBY * ty;   // the tile's first block (lattice indices)
    const int vx = min(TBX, a.ix0 + a.nix - bi0), vy = min(TBY, a.iy0 + a.niy - bj0);   // valid blocks
    const int gx0 = a.ox + q * bi0 - R - P, gy0 = a.oy + q * bj0 - R - P;            // region origin (>= 0)
    const long long drain = a.budget > (1LL << 31) ? a.budget : (1LL << 31);
    pdl_wait();
    // every global load first (b at the blocks' DOFs, then the region of u), the set-up while
    // they are in flight, then the stores to shared memory
    // RB: region loads per thread and batch (one batch for the region of the default period)
    constexpr int NBV = (M * SS + NT - 1) / NT, RB = P == 2 ? 14 : (P == 3 ? 26 : 28);
    float bv[NBV];
#pragma unroll
    for (int i = 0; i < NBV; ++i) {
        const int idx = tid + NT * i, r = idx / SS, k = idx - r * SS;
        const int tbx = r % TBX, tby = r / TBX;
        float v = 0.f;
        if (idx < M * SS && tbx < vx && tby < vy)
            v = __ldg(&a.b[(size_t)(gy0 + q * tby + P + k / S) * n + (gx0 + q * tbx + P + k % S)]);
        bv[i] = v;
    }
    const int nreg = RW * RH;
    const float rcp = 1.0f / (float)RW;   // exact quotient: idx < 2^16 and RW < 2^9
    auto load_region = [&](int base, float (&v)[RB]) {
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int idx = base + NT * i;
            const int ry = (int)(((float)idx + 0.5f) * rcp), rx = idx - ry * RW;
            const int gy = gy0 + ry, gx = gx0 + rx;
            v[i] = (idx < nreg && gy < n && gx < n) ? a.u[(size_t)gy * n + gx] : 0.f;
        }
    };
    float rv[RB];
    load_region(tid, rv);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&mbar[1])),
                     "r"((uint32_t)G::GB)
                     : "memory");
        if (!a.skip_copy)   // (error-path tests leave the copy out, so its wait runs out)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             smem_addr(sG)),
                         "l"(a.gtc), "r"((uint32_t)G::GB), "r"(smem_addr(&mbar[1]))
                         : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(G::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int k = tid; k < KP; k += NT) {
        const int j = k - SS;
        sOff[k] = (k >= SS && k < KU) ? (j / G::PW) * RW + (j % G::PW) : 0;
    }
    for (int r = tid; r < M; r += NT) sRb[r] = q * (r / TBX) * RW + q * (r % TBX);
#pragma unroll
    for (int i = 0; i < RB; ++i)
        if (tid + NT * i < nreg) sR[tid + NT * i] = rv[i];
    for (int base = tid + NT * RB; base < nreg; base += NT * RB) {   // regions above NT RB floats
        load_region(base, rv);
#pragma unroll
        for (int i = 0; i < RB; ++i)
            if (base + NT * i < nreg) sR[base + NT * i] = rv[i];
    }
#pragma unroll
    for (int i = 0; i < NBV; ++i) {
        const int idx = tid + NT * i, r = idx / SS, k = idx - r * SS;
        if (idx < M * SS) sX[tc_off(r, k, KP)] = to_tf32(bv[i]);
    }
    __syncthreads();
    // X's patch columns.  16-byte pieces k = 4 kq .. 4 kq + 3 of one row hold u only for kq in
    // [KQ0, KQ1): warp w builds the 8-row groups w, w + 8 (lane = 8 (kq mod 4) + row in group),
    // U pieces at a time with their loads first.  The pieces that mix b and u, or u and the
    // zero padding, element by element: thread (row, half) one row's head or tail.
    {
        constexpr int KQ0 = (SS + 3) / 4, KQ1 = KU / 4, NQ = KQ1 - KQ0, NIT = (NQ + 3) / 4, U = 4;
        const int r8 = lane & 7, kql = lane >> 3;
        const int4 *off4 = reinterpret_cast<const int4 *>(sOff);
#pragma unroll 1
        for (int rg = warp; rg < M / 8; rg += NWARP) {
            const int r = rg * 8 + r8;
            const float *__restrict__ src = sR + sRb[r];
            float *__restrict__ dst = sX + tc_off(r, 0, KP);
#pragma unroll
            for (int i0 = 0; i0 < NIT; i0 += U) {
                float4 x[U];
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    const int kq = KQ0 + kql + 4 * (i0 + i);
                    if (i0 + i < NIT && kq < KQ1) {
                        const int4 o = off4[kq];
                        x[i] = make_float4(src[o.x], src[o.y], src[o.z], src[o.w]);
                    }
                }
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    const int kq = KQ0 + kql + 4 * (i0 + i);
                    if (i0 + i < NIT && kq < KQ1)
                        *reinterpret_cast<float4 *>(dst + kq * 32) =
                            make_float4(to_tf32(x[i].x), to_tf32(x[i].y), to_tf32(x[i].z), to_tf32(x[i].w));
                }
            }
        }
        constexpr int NH = 4 * KQ0 - SS, NTL = KP - 4 * KQ1;
        static_assert(NT == 2 * M, "one thread per row and half");
        const int r = tid & (M - 1);
        const float *src = sR + sRb[r];
        if (tid < M) {
#pragma unroll
            for (int i = 0; i < NH; ++i) sX[tc_off(r, SS + i, KP)] = to_tf32(src[sOff[SS + i]]);
        } else {
#pragma unroll
            for (int i = 0; i < NTL; ++i) {
                const int k = 4 * KQ1 + i;
                sX[tc_off(r, k, KP)] = k < KU ? to_tf32(src[sOff[k]]) : 0.f;
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> MMA reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        // G has landed (bounded wait), then the MMA chain
        const int gready = mbar_wait_bounded(smem_addr(&mbar[1]), 0, a.budget);
        if (!gready) {
            atomicAdd(a.status, 1);
            // a copy still in flight must land before the CTA may exit (bounded again, by
            // at least the default budget whatever the caller chose)
            if (!a.skip_copy) mbar_wait_bounded(smem_addr(&mbar[1]), 0, drain);
        }
        *s_mma = gready;
        if (gready) {
            constexpr uint32_t idesc = idesc_tf32(M, NP);
            const uint32_t xa = smem_addr(sX), ga = smem_addr(sG);
#pragma unroll 1
            for (int s = 0; s < KP / 8; ++s) {
                const uint64_t da = smem_desc(xa + s * 2 * G::LBO, G::LBO, G::SBO);
                const uint64_t db = smem_desc(ga + s * 2 * G::LBO, G::LBO, G::SBO);
                const uint32_t acc = s > 0 ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                             "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&mbar[0]))
                         : "memory");
        }
    }
    __syncthreads();
    // bounded wait for the MMA chain (phase 0 of the barrier); if it gives up, the chain
    // must still finish before the tensor memory is released (bounded again)
    uint32_t done = 0;
    if (*s_mma) {
        done = mbar_wait_bounded(smem_addr(&mbar[0]), 0, a.budget);
        done = __all_sync(0xffffffffu, done);   // tcgen05.ld below is warp-collective
        if (!done) {
            if (lane == 0) atomicAdd(a.status, 1);
            mbar_wait_bounded(smem_addr(&mbar[0]), 0, drain);
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warp w reads the rows of tensor-memory sub-partition w % 4 (one block per lane), column
    // slices w / 4, w / 4 + 2, ... of 8; the tensor memory is released before the stores
    constexpr int NCS = (NP / 8 + 1) / 2;   // slices per warp
    const int sub = warp & 3, r = sub * 32 + lane;
    uint32_t d[NCS][8];
    if (done) {
#pragma unroll
        for (int j = 0; j < NCS; ++j) {
            const int cs = (warp >> 2) + 2 * j;
            if (cs < NP / 8) {
                const uint32_t taddr = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(cs * 8);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(d[j][0]), "=r"(d[j][1]), "=r"(d[j][2]), "=r"(d[j][3]), "=r"(d[j][4]),
                               "=r"(d[j][5]), "=r"(d[j][6]), "=r"(d[j][7])
                             : "r"(taddr));
            }
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TCOLS));
    const int tbx = r % TBX, tby = r / TBX;
    if (done && tbx < vx && tby < vy) {
        const float *uo = sR + sRb[r] + P * RW + P;   // u_old at the block's first DOF
        float *ug = a.u + (size_t)(gy0 + q * tby + P) * n + (gx0 + q * tbx + P);
#pragma unroll
        for (int j = 0; j < NCS; ++j) {
            const int cs = (warp >> 2) + 2 * j;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = cs * 8 + i, ey = e / S, ex = e - ey * S;
                if (cs < NP / 8 && e < SS) ug[(size_t)ey * n + ex] = uo[ey * RW + ex] + __uint_as_float(d[j][i]);
            }
        }
    }
}

// One colour of the LATTICE schedule in FP64 for 7x7 (or 5x5) blocks, the residual
// sum-factorised with S^2 threads per block in every step (BPC blocks per CTA):
//   0. the block's (S + 2P)^2 window of u into shared memory;
//   1. the S x (S + 2P) pairs (sum_b K_y[b] u, sum_b M_y[b] u) of the block's rows at its
//      window columns, items e, e + S^2, ... of thread e;
//   2. thread e: the x sums of its DOF, r_e = b - A u;
//   3. thread e: row e of the block's inverse times r, added to u.
// Per DOF and colour this is 2W(S + 2P)/S + 2W + S^2 FMAs against W^2 + S^2 for the direct
// stencil (p = 5: 113 against 146; p = 7: 169 against 274), with every step spread evenly
// over the block's threads.  Interior rows/columns use the h-scaled interior 1D rows from
// constant memory, the others their own 1D rows.
template <int P, int S, int BPC>
__global__ void __launch_bounds__(256)
k_schwarz_lattice2d_pd(int n, int nbc, int q, int ox, int oy, int nbx, int nblocks,
                       const double *__restrict__ kband, const double *__restrict__ mband,
                       const double *__restrict__ binv, const int *__restrict__ bcls, double *__restrict__ u,
                       const double *__restrict__ b, BatchRef bt)
{
    constexpr int W = 2 * P + 1, SS = S * S, R = (S - 1) / 2, WIN = S + 2 * P, PCI = 2 * P - 1;
    constexpr int NY = S * WIN;   // y items of a block
    __shared__ double su[BPC][WIN][WIN];
    __shared__ double2 yb[BPC][S][WIN];
    __shared__ double rs[BPC][SS];
    pdl_wait();
    if (bt.active && !bt.active[blockIdx.y]) return;
    u += blockIdx.y * bt.vec;
    b += blockIdx.y * bt.vec;
    const int lb = threadIdx.x / SS, e = threadIdx.x % SS;
    const int blk = blockIdx.x * BPC + lb;
    const bool active = lb < BPC && blk < nblocks;
    const int cx = ox + q * (blk % nbx), cy = oy + q * (blk / nbx);
    const double h = 1.0 / (double)(n - P + 2), hinv = (double)(n - P + 2);
    // 0. window rows cy - R - P .., columns cx - R - P .. (zero outside the grid)
    if (active) {
        constexpr int K = (WIN * WIN + SS - 1) / SS;
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = e + k * SS, wr = i / WIN, wc = i - wr * WIN;
            const int gx = cx - R - P + wc, gy = cy - R - P + wr;
            v[k] = (i < WIN * WIN && gx >= 0 && gx < n && gy >= 0 && gy < n) ? u[(size_t)gy * n + gx] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = e + k * SS;
            if (i < WIN * WIN) su[lb][i / WIN][i % WIN] = v[k];
        }
    }
    __syncthreads();
    // 1. y pass
    if (active) {
        const bool yint = cy - R >= PCI && cy + R <= n - 2 * P;
        for (int i = e; i < NY; i += SS) {
            const int r = i / WIN, c = i - r * WIN;
            double2 acc = make_double2(0.0, 0.0);
            if (yint) {
#pragma unroll
                for (int bb = 0; bb < W; ++bb) acc = fma2(ckm1<double>(P, bb), splat2<double2>(su[lb][r + bb][c]), acc);
            } else {
                const int gy = cy - R + r;
                if (gy >= 0 && gy < n) {
#pragma unroll
                    for (int bb = 0; bb < W; ++bb) {
                        const double2 km =
                            make_double2(kband[(size_t)gy * W + bb] * h, mband[(size_t)gy * W + bb] * hinv);
                        acc = fma2(km, splat2<double2>(su[lb][r + bb][c]), acc);
                    }
                }
            }
            yb[lb][r][c] = acc;
        }
    }
    __syncthreads();
    // 2. x pass and the block residual
    const int ey = e / S, ex = e - ey * S;
    const int x = cx - R + ex, y = cy - R + ey;
    const bool inside = active && x >= 0 && x < n && y >= 0 && y < n;
    if (active) {
        double rv = 0.0;
        if (inside) {
            const bool xint = cx - R >= PCI && cx + R <= n - 2 * P;
            double2 acc = make_double2(0.0, 0.0);
            if (xint) {
#pragma unroll
                for (int a = 0; a < W; ++a) acc = fma2(cmk1<double>(P, a), yb[lb][ey][ex + a], acc);
            } else {
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const double2 mk = make_double2(mband[(size_t)x * W + a] * hinv, kband[(size_t)x * W + a] * h);
                    acc = fma2(mk, yb[lb][ey][ex + a], acc);
                }
            }
            rv = b[(size_t)y * n + x] - (acc.x + acc.y);
        }
        rs[lb][e] = rv;
    }
    __syncthreads();
    // 3. block solve
    if (inside) {
        const int cls = bcls[cy] * nbc + bcls[cx];
        const double *Bi = binv + (size_t)cls * SS * SS + e;   // (transposed per class)
        double ev = 0.0;
#pragma unroll
        for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[(size_t)f * SS]), rs[lb][f], ev);
        u[(size_t)y * n + x] += ev;
    }
}

// Geometry of one CTA of the TILE(TT) schedule.
template <int P, int S, int TT>
struct TileGeom {
    static constexpr int W = 2 * P + 1, SS = S * S, R = (S - 1) / 2, H = R + P;
    static constexpr int SW = TT + 2 * H;                  // staged u: tile + halo R + P
    static constexpr int BW = TT + 2 * R;                  // staged b / rows a tile's blocks cover
    static constexpr int NB1 = (TT + S + P - 1) / (S + P);  // blocks per axis of one colour (q >= S+P)
    static constexpr int NBLK = NB1 * NB1;
    static constexpr int BPW = 32 / SS;                    // blocks per warp (SS lanes each)
    static constexpr int NWARP = (NBLK + BPW - 1) / BPW, NT = 32 * NWARP;
    static constexpr int WIN = S + 2 * P;                  // window columns (and rows) of a block
    // y sums of a block: S rows of YS pairs (K_y u, M_y u); YS and the block stride YB keep
    // the 8-byte reads of each half-warp in the x pass in distinct banks
    static constexpr int YS = S == 5 ? 21 : 19, YB = S * YS;
    static constexpr int RSS = (SS + 3) / 4 * 4;           // residual stride (16-byte loads)
    static constexpr int NB2 = (SS + 1) / 2;               // pairs of one inverse row
    // one block per warp and 2 WIN <= 32 (5 x 5 blocks): the interior y pass takes two lanes
    // per window column, rows 0 .. RA - 1 and RA .. S - 1
    static constexpr bool SPLITY = BPW == 1 && 2 * WIN <= 32;
    static constexpr int RA = (S + 1) / 2;
    // row stride of the staged u: with SPLITY the two halves of a warp read rows RA apart, so
    // the stride is padded until those rows' banks (4-byte words) do not overlap; with 3x3
    // blocks (three per warp, at offsets set by the colour) p = 3 takes 31 for 29: counting the
    // y pass's bank conflicts over every colour offset and candidate stride gave 20% fewer of
    // its load wavefronts (measured sweep 170.2 -> 169.4 us: the y pass is a small part of the
    // kernel's shared-memory traffic), and no better stride for p = 2 or 4
    static constexpr int swp(int w)
    {
        return !SPLITY ? (P == 3 && S == 3 ? SW + 2 : w)
                       : ((RA * w) % 32 >= WIN && (RA * w) % 32 <= 32 - WIN) ? w : swp(w + 1);
    }
    static constexpr int SWP = swp(SW);
    // resident CTAs per SM the register allocation must allow (FP32: a 1024^2 tile phase
    // in one wave; FP64 keeps its registers)
    template <typename T>
    static constexpr int minb() { return sizeof(T) == sizeof(double) ? 1 : (NT >= 128 ? 5 : 4); }
    // the work-list form keeps the per-phase kernel's residency (its item loop would otherwise
    // take more registers)
    template <typename T>
    static constexpr int minb_work() { return sizeof(T) == sizeof(double) ? 1 : (NT >= 128 ? 5 : 8); }
};

// Stages a (tile-local, zero outside the grid) window into shared memory with all loads
// of a thread issued before its stores.
template <int NT, int ROWLEN, int NELEM, typename T, bool L2ONLY = false, int DSTROW = ROWLEN>
__device__ __forceinline__ void stage_window(T *dst, const T *__restrict__ src, int n, int gx0, int gy0, int tid)
{
    constexpr int K = (NELEM + NT - 1) / NT;
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = tid + k * NT;
        const int gx = gx0 + i % ROWLEN, gy = gy0 + i / ROWLEN;
        const bool in = i < NELEM && gx >= 0 && gx < n && gy >= 0 && gy < n;
        if constexpr (L2ONLY)   // written by other CTAs of the same launch: not through L1
            v[k] = in ? __ldcg(&src[(size_t)gy * n + gx]) : T(0);
        else
            v[k] = in ? src[(size_t)gy * n + gx] : T(0);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = tid + k * NT;
        if (i < NELEM) dst[DSTROW == ROWLEN ? i : (i / ROWLEN) * DSTROW + i % ROWLEN] = v[k];
    }
}

// y pass of one block: for window column col (tile-local x = cxl - R - P + col) the
// column slice rows cyl .. cyl + WIN - 1 of the staged u, then for every block row r
//   Y[r][col] = (sum_b K_y[b] u(col, row r + b - P), sum_b M_y[b] u(...)).
// FAST: interior rows (constant 1D rows); else the rows' own 1D rows (km1y: (K, M) pairs).
template <int P, int S, int TT, bool FAST, typename T>
__device__ __forceinline__ void tile_ypass(const T *su, int cxl, int cyl, int lane_e,
                                           typename Vec2<T>::type *yb, const typename Vec2<T>::type *km1y)
{
    using G = TileGeom<P, S, TT>;
    using T2 = typename Vec2<T>::type;
    constexpr int W = G::W, WIN = G::WIN, SW = G::SWP;   // (SW: the staged u's row stride)
    for (int col = lane_e; FAST && col < WIN; col += G::SS) {
        {
            // interior rows are symmetric, so the taps at distance j from the row's centre
            // share one packed multiply-add (K, M) on their sum, held as a (v, v) pair
            T v[WIN];
#pragma unroll
            for (int k = 0; k < WIN; ++k) v[k] = su[(cyl + k) * SW + cxl + col];
#pragma unroll
            for (int r = 0; r < S; ++r) {
                T2 y = fma2(ckm1<T>(P, P), splat2<T2>(v[r + P]), splat2<T2>(T(0)));
#pragma unroll
                for (int j = 1; j <= P; ++j)
                    y = fma2(ckm1<T>(P, P - j), splat2<T2>(v[r + P - j] + v[r + P + j]), y);
                yb[r * G::YS + col] = y;
            }
        }
    }
    if (!FAST) {
        // blocks with boundary rows: per-row coefficients; the S x WIN points are spread
        // over all the block's lanes, u read from shared memory directly
        for (int pt = lane_e; pt < S * WIN; pt += G::SS) {
            const int r = pt / WIN, col = pt - r * WIN;
            const T2 *kr = km1y + (cyl + r) * W;
            const T *uc = su + (cyl + r) * SW + cxl + col;
            T2 y = splat2<T2>(T(0));
#pragma unroll
            for (int bb = 0; bb < W; ++bb) y = fma2(kr[bb], splat2<T2>(uc[bb * SW]), y);
            yb[r * G::YS + col] = y;
        }
    }
}

// y pass with two lanes per window column (SPLITY): lane l < WIN takes rows 0 .. RA - 1 of
// column l, lane WIN + l rows RA .. S - 1.  FASTROW: interior rows (symmetric constant
// rows); otherwise every row's own (K, M) pairs from km1y, read by all lanes at once.
template <int P, int S, int TT, bool FASTROW, typename T>
__device__ __forceinline__ void tile_ypass_split(const T *su, int cxl, int cyl, int lane,
                                                 typename Vec2<T>::type *yb, const typename Vec2<T>::type *km1y)
{
    using G = TileGeom<P, S, TT>;
    using T2 = typename Vec2<T>::type;
    constexpr int W = G::W, WIN = G::WIN, SW = G::SWP, RA = G::RA, RB = S - RA;   // (SW: row stride)
    // one half of the rows per half-warp (lanes 0 .. WIN - 1 and 16 .. 15 + WIN): a half-warp's
    // 8-byte loads then read one contiguous row segment (with the halves mixed in one
    // half-warp, the second half's rows fell on the first half's banks)
    const int half = lane >> 4, col = lane & 15, r0 = half ? RA : 0;
    if (col >= WIN) return;
    const T *up = su + (cyl + r0) * SW + cxl + col;
    T v[RA + 2 * P];
#pragma unroll
    for (int k = 0; k < RB + 2 * P; ++k) v[k] = up[k * SW];
    if (!half)
#pragma unroll
        for (int k = RB + 2 * P; k < RA + 2 * P; ++k) v[k] = up[k * SW];
    T2 *yo = yb + r0 * G::YS + col;
#pragma unroll
    for (int r = 0; r < RA; ++r) {
        if (half && r >= RB) break;
        T2 y;
        if constexpr (FASTROW) {
            y = fma2(ckm1<T>(P, P), splat2<T2>(v[r + P]), splat2<T2>(T(0)));
#pragma unroll
            for (int j = 1; j <= P; ++j)
                y = fma2(ckm1<T>(P, P - j), splat2<T2>(v[r + P - j] + v[r + P + j]), y);
        } else {
            const T2 *kr = km1y + (cyl + r0 + r) * W;
            T2 y1 = splat2<T2>(T(0));
            y = y1;
#pragma unroll
            for (int bb = 0; bb < W; ++bb) {
                T2 &acc = (bb & 1) ? y1 : y;
                acc = fma2(kr[bb], splat2<T2>(v[r + bb]), acc);
            }
            y = add2(y, y1);
        }
        yo[r * G::YS] = y;
    }
}

// x pass of one output (ey, ex) of a block: sum_a M_x[a] Y1[ey][ex + a] + K_x[a] Y2[ey][ex + a]
template <int P, int S, int TT, bool FAST, typename T>
__device__ __forceinline__ T tile_xpass(const typename Vec2<T>::type *yb, int ey, int ex, int xrow,
                                        const typename Vec2<T>::type *mk1x)
{
    using G = TileGeom<P, S, TT>;
    using T2 = typename Vec2<T>::type;
    constexpr int W = G::W;
    const T2 *y = yb + ey * G::YS + ex;
    // two accumulators (even and odd taps): half the dependent chain
    T2 s0 = splat2<T2>(T(0)), s1 = s0;
#pragma unroll
    for (int a = 0; a < W; ++a) {
        T2 &s = (a & 1) ? s1 : s0;
        s = fma2(FAST ? cmk1<T>(P, a) : mk1x[xrow * W + a], y[a], s);
    }
    const T2 s = add2(s0, s1);
    return s.x + s.y;
}

// One tile phase of the TILE(TT) schedule: tiles (tx, ty) with tx = px, px+2, ... and
// ty = py, py+2, ...; each CTA runs all q^2 lattice colours of its tile in order
// (anchored at the tile origin) with u (tile + halo R+P) and b (tile + halo R) staged in
// shared memory, then writes back the DOFs its blocks can change (tile + halo R).  Tiles
// of one phase are 2 TT apart with TT >= 2R + P: none reads what another writes.
//
// Thread (block slot, entry e) owns one DOF of one Schwarz block of the current colour;
// a block's S^2 lanes sit in one warp.  The residual uses the y-then-x sum factorisation
//   (A u)(x, y) = sum_b K_y[b] sum_a M_x[a] u(x+a-P, y+b-P) + M_y[b] sum_a K_x[a] u(...),
// shared by the block's lanes: a y pass over the window columns (each lane slides down
// one column), a warp barrier, then each lane's x pass; the K and M halves run as pairs
// (packed FP32 FMA).  Interior tiles (almost all) take the interior 1D rows from constant
// memory; boundary tiles the 1D rows of their own rows and columns.  After a second warp
// barrier each lane applies row e of its block's inverse (the interior row kept in
// registers; boundary classes with their FP64 inverse, in compensated FP32 arithmetic)
// and adds the result to u in shared memory.  One
// CTA barrier per colour.
// Shared memory of one CTA of the TILE step.
template <int P, int S, int TT, typename T>
struct TileSmem {
    using G = TileGeom<P, S, TT>;
    using T2 = typename Vec2<T>::type;
    T su[G::SW * G::SWP];   // u, rows G::SWP apart (the y passes form the (u, u) pairs of the
                            // packed FMAs in registers)
    T sb[G::BW * G::BW];
    __align__(16) T rs[G::NBLK * G::RSS];
    T2 yb[G::NBLK * G::YB];
    T2 km1y[G::BW * G::W], mk1x[G::BW * G::W];   // boundary tiles: (K, M) of rows, (M, K) of columns
};

// One tile of one TILE phase (tile index ti of the phase's ntpx-wide grid of tiles).  `pre`
// runs after the constant-table reads, before the first read of u or b, and returns whether
// the CTA goes on (the same answer in every thread).  L2ONLY: u is read past L1 (other CTAs
// of the same launch wrote it).  binv and binv_lo hold every class's inverse transposed
// ([class][f][e]): the lanes of a block (one per row e) read consecutive words.
template <int P, int S, int TT, typename T, bool L2ONLY, typename Pre>
__device__ __forceinline__ void schwarz_tile_cta(TileSmem<P, S, TT, T> &sm, int ti, int n, int nbc, int q, int g,
                                                 int rev, int c0, int c1, int px, int py, int ntpx,
                                                 const T *__restrict__ kband, const T *__restrict__ mband,
                                                 const T *__restrict__ binv, const float *__restrict__ binv_lo,
                                                 int interior, T *__restrict__ u, const T *__restrict__ b, Pre pre)
{
    using G = TileGeom<P, S, TT>;
    using T2 = typename Vec2<T>::type;
    constexpr int W = G::W, SS = G::SS, R = G::R, H = G::H, L = P - 1 + R;
    constexpr int SW = G::SW, BW = G::BW, NB1 = G::NB1, NT = G::NT;
    constexpr int PCI = 2 * P - 1;   // first interior row class
    T *su = sm.su;
    T *sb = sm.sb;
    T *rs = sm.rs;
    T2 *yb = sm.yb;
    T2 *km1y = sm.km1y, *mk1x = sm.mk1x;
    const int tid = threadIdx.x;
    const int x0 = (px + 2 * (ti % ntpx)) * TT, y0 = (py + 2 * (ti / ntpx)) * TT;
    const int tw = min(TT, n - x0), th = min(TT, n - y0);   // centres of this tile
    const bool fast = x0 - R >= PCI && x0 + TT - 1 + R <= n - 2 * P && y0 - R >= PCI &&
                      y0 + TT - 1 + R <= n - 2 * P;
    const int lane = tid & 31, bw = lane / SS, e = lane - bw * SS;
    const int ey = e / S, ex = e - ey * S;
    const int slot = (tid >> 5) * G::BPW + bw;
    const bool role = bw < G::BPW && slot < G::NBLK;
    for (int i = tid; i < G::NBLK * G::RSS; i += NT) rs[i] = T(0);   // the padding stays zero
    // constant tables (read before the wait)
    if (!fast) {
        // the rows scaled like the interior constants (h K, M / h), h = 1 / m, so that a
        // block may mix interior and boundary factors
        const T h = T(1) / T(n - P + 2), hinv = T(n - P + 2);
        for (int i = tid; i < BW * W; i += NT) {
            const int row = i / W, a = i - row * W;
            const int gx = x0 - R + row, gy = y0 - R + row;
            const bool inx = gx >= 0 && gx < n, iny = gy >= 0 && gy < n;
            T2 km, mk;
            km.x = iny ? kband[(size_t)gy * W + a] * h : T(0);
            km.y = iny ? mband[(size_t)gy * W + a] * hinv : T(0);
            mk.x = inx ? mband[(size_t)gx * W + a] * hinv : T(0);
            mk.y = inx ? kband[(size_t)gx * W + a] * h : T(0);
            km1y[i] = km;
            mk1x[i] = mk;
        }
    }
    // row e of the interior block inverse as pairs, in registers for the whole tile
    T2 brow[G::NB2];
#pragma unroll
    for (int k = 0; k < G::NB2; ++k) {
        const size_t base = (size_t)interior * SS * SS + e;
        brow[k].x = role ? __ldg(&binv[base + (size_t)(2 * k) * SS]) : T(0);
        brow[k].y = (role && 2 * k + 1 < SS) ? __ldg(&binv[base + (size_t)(2 * k + 1) * SS]) : T(0);
    }
    if (!pre()) return;
    stage_window<NT, SW, SW * SW, T, L2ONLY, G::SWP>(su, u, n, x0 - H, y0 - H, tid);
    stage_window<NT, BW, BW * BW>(sb, b, n, x0 - R, y0 - R, tid);
    __syncthreads();
    const int bi = slot % NB1, bj = slot / NB1;
    T2 *ybs = yb + slot * G::YB;
    T *rsb = rs + slot * G::RSS;
    // colours c0 .. c1 - 1 of the tile's lattice order (all q^2 unless the colours are split
    // into groups), in reverse with rev; colour c visits offsets ((c mod q) g mod q,
    // (c div q) g mod q), advanced incrementally.  The colour loop is compiled twice: FAST
    // (interior tiles: every block of the interior class and inside the grid) and the
    // general form
    const int ncol = c1 - c0, cstart = rev ? c1 - 1 : c0;
    auto colours = [&](auto fast_tag) {
        constexpr bool FAST = decltype(fast_tag)::value;
        int cxr = cstart % q;
        int ox = (cxr * g) % q, oy = ((cstart / q) * g) % q;
        for (int t = 0; t < ncol; ++t) {
            const int cxl = ox + q * bi, cyl = oy + q * bj;   // tile-local centre
            // (q may exceed the minimum period the slots are laid out for, so some slots
            // fall outside the tile in every colour, interior tiles included)
            const bool act = role && cxl < tw && cyl < th;
            const int lx = cxl - R + ex, ly = cyl - R + ey;   // tile-local DOF of this lane
            // are the block's rows / columns all of the interior class?
            const bool yint = FAST || (y0 + cyl - R >= PCI && y0 + cyl + R <= n - 2 * P);
            const bool xint = FAST || (x0 + cxl - R >= PCI && x0 + cxl + R <= n - 2 * P);
            if constexpr (G::SPLITY) {
                (void)yint;
                // the whole warp works on its block's y pass (interior rows); lanes past the
                // block's S^2 carry another slot number, so the warp's own block is used
                const int ws = tid >> 5, wcx = ox + q * (ws % NB1), wcy = oy + q * (ws / NB1);
                if (ws < G::NBLK && wcx < tw && wcy < th) {
                    const bool wyint = FAST || (y0 + wcy - R >= PCI && y0 + wcy + R <= n - 2 * P);
                    if (wyint) tile_ypass_split<P, S, TT, true, T>(su, wcx, wcy, lane, yb + ws * G::YB, km1y);
                    else tile_ypass_split<P, S, TT, false, T>(su, wcx, wcy, lane, yb + ws * G::YB, km1y);
                }
            } else if (act) {
                if (yint) tile_ypass<P, S, TT, true, T>(su, cxl, cyl, e, ybs, km1y);
                else tile_ypass<P, S, TT, false, T>(su, cxl, cyl, e, ybs, km1y);
            }
            __syncwarp();
            const int gx = x0 + lx, gy = y0 + ly;
            const bool in = FAST || (gx >= 0 && gx < n && gy >= 0 && gy < n);
            if (act) {
                const T acc = xint ? tile_xpass<P, S, TT, true, T>(ybs, ey, ex, lx + R, mk1x)
                                   : tile_xpass<P, S, TT, false, T>(ybs, ey, ex, lx + R, mk1x);
                rsb[e] = in ? sb[(ly + R) * BW + (lx + R)] - acc : T(0);
            }
            __syncwarp();
            if (act) {
                int cls = interior;
                if (!FAST) {
                    const int ccx = x0 + cxl, ccy = y0 + cyl;
                    const int bx = ccx < L ? ccx : (ccx > n - 1 - L ? 2 * L - (n - 1 - ccx) : L);
                    const int by = ccy < L ? ccy : (ccy > n - 1 - L ? 2 * L - (n - 1 - ccy) : L);
                    cls = by * nbc + bx;
                }
                T ev = T(0);
                if (cls == interior) {
                    // two pair accumulators: four independent chains
                    T2 acc0 = splat2<T2>(T(0)), acc1 = acc0;
                    const T2 *r2 = reinterpret_cast<const T2 *>(rsb);   // 16-byte aligned, zero padded
    #pragma unroll
                    for (int k = 0; k < G::NB2; ++k) {
                        T2 &acc = (k & 1) ? acc1 : acc0;
                        acc = fma2(brow[k], r2[k], acc);
                    }
                    const T2 acc2 = add2(acc0, acc1);
                    ev = acc2.x + acc2.y;
                } else if (sizeof(T) == sizeof(double) || !binv_lo) {
                    const T *Bi = binv + (size_t)cls * SS * SS + e;
    #pragma unroll
                    for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[(size_t)f * SS]), rsb[f], ev);
                } else if constexpr (sizeof(T) == sizeof(float)) {
                    // FP64 row of a boundary-class inverse (as the pair binv + binv_lo), applied
                    // in compensated FP32 arithmetic: GB300's FP64 pipe is 1/58 of its FP32
                    // rate, and these rows set the boundary tiles' critical path
                    const size_t col = (size_t)cls * SS * SS + e;
                    T rv[2 * G::NB2];
                    const T2 *r2 = reinterpret_cast<const T2 *>(rsb);
    #pragma unroll
                    for (int k = 0; k < G::NB2; ++k) { const T2 v = r2[k]; rv[2 * k] = v.x; rv[2 * k + 1] = v.y; }
                    ev = dot2_row<SS, SS>(binv + col, binv_lo + col, rv);
                }
                if (in) {
                    T &ref = su[(ly + H) * G::SWP + (lx + H)];
                    ref = ref + ev;
                }
            }
            __syncthreads();
            if (!rev) {
                if (++cxr == q) { cxr = 0; ox = 0; oy += g; if (oy >= q) oy -= q; }
                else { ox += g; if (ox >= q) ox -= q; }
            } else {
                if (--cxr < 0) { cxr = q - 1; ox = q - g; oy -= g; if (oy < 0) oy += q; }
                else { ox -= g; if (ox < 0) ox += q; }
            }
        }
    };
    if (fast) colours(std::true_type{});
    else colours(std::false_type{});
    for (int i = tid; i < BW * BW; i += NT) {
        const int gx = x0 - R + i % BW, gy = y0 - R + i / BW;
        if (gx >= 0 && gx < n && gy >= 0 && gy < n) u[(size_t)gy * n + gx] = su[(i / BW + P) * G::SWP + (i % BW + P)];
    }
}

template <int P, int S, int TT, typename T>
__global__ void __launch_bounds__(TileGeom<P, S, TT>::NT, TileGeom<P, S, TT>::template minb<T>())
k_schwarz_tile2d(int n, int nbc, int q, int g, int rev, int c0, int c1, int px, int py, int ntpx,
                 const T *__restrict__ kband, const T *__restrict__ mband,
                 const T *__restrict__ binv, const float *__restrict__ binv_lo, int interior,
                 T *__restrict__ u, const T *__restrict__ b, BatchRef bt)
{
    __shared__ TileSmem<P, S, TT, T> sm;
    u += blockIdx.y * bt.vec;
    b += blockIdx.y * bt.vec;
    schwarz_tile_cta<P, S, TT, T, false>(sm, blockIdx.x, n, nbc, q, g, rev, c0, c1, px, py, ntpx, kband, mband, binv,
                                         binv_lo, interior, u, b, [&] {
                                             pdl_wait();
                                             return !(bt.active && !bt.active[blockIdx.y]);
                                         });
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The TILE sweep of every problem of a handle in one launch (a work list).  Items are
// (colour group, tile phase, problem, tile) in sweep order, claimed one at a time from a
// counter: item ids grow with the sweep order, so an item waits only for items claimed
// before it by CTAs that are running, and the launch cannot deadlock.  A tile reads u within
// H = R + P of its square and writes within R of it; H + R <= TT, so only its eight
// neighbouring tiles (and itself, with colour groups) touch the same DOFs.  It therefore
// starts once the earlier occurrences of those nine tile positions in the sweep order have
// finished: a per-problem, per-position counter of finished occurrences, raised after a
// device-scope fence; each wait is bounded by `budget` cycles and gives up at once after
// any failure.  Every pair of tiles that touch the same DOFs keeps the order of one launch
// per phase, so the iterates are bitwise those of that form, while the tiles of a phase no
// longer wait for its slowest (boundary) tiles unless they are neighbours.  u is read past
// L1, since other SMs wrote it during the launch.  The counters are zeroed on the stream
// before the launch.  withhold (tests only): finished tiles are not counted, so the first
// wait runs out.
struct TileWorkArgs {
    int n, nbc, q, g, rev, interior, nbatch, groups, withhold, nt;
    int tiles[4], ntpx[4];   // tiles and tiles per row of phase (px, py) = (t & 1, t >> 1)
    long long per_group;     // items per colour group: nbatch (tiles[0] + ... + tiles[3])
    long long total;
    unsigned *ctr;           // [0]: next item; [1 + problem nt^2 + J nt + I]: finished
                             // occurrences of tile position (I, J)
    const int *active;
    size_t vec;
    int *status;
    long long budget;
};

template <int P, int S, int TT, typename T>
__global__ void __launch_bounds__(TileGeom<P, S, TT>::NT, TileGeom<P, S, TT>::template minb_work<T>())
k_schwarz_tile2d_work(const __grid_constant__ TileWorkArgs a, const T *__restrict__ kband,
                      const T *__restrict__ mband, const T *__restrict__ binv, const float *__restrict__ binv_lo,
                      T *__restrict__ u, const T *__restrict__ b)
{
    __shared__ TileSmem<P, S, TT, T> sm;
    __shared__ long long s_item;
    __shared__ int s_go;
    const int ncol = a.q * a.q, nt = a.nt;
    pdl_wait();
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.ctr, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= a.total) break;
        // decode: colour group and phase in sweep order, then problem and tile
        const int kseq = (int)(item / a.per_group);
        long long rem = item - (long long)kseq * a.per_group;
        int tseq = 0, ph = a.rev ? 3 : 0;
        while (tseq < 3 && rem >= (long long)a.nbatch * a.tiles[ph]) {
            rem -= (long long)a.nbatch * a.tiles[ph];
            ++tseq;
            ph = a.rev ? 3 - tseq : tseq;
        }
        const int i = (int)(rem / a.tiles[ph]), ti = (int)(rem - (long long)i * a.tiles[ph]);
        const int k = a.rev ? a.groups - 1 - kseq : kseq;
        const int c0 = (k * ncol + a.groups - 1) / a.groups, c1 = ((k + 1) * ncol + a.groups - 1) / a.groups;
        const int I = (ph & 1) + 2 * (ti % a.ntpx[ph]), J = (ph >> 1) + 2 * (ti / a.ntpx[ph]);   // tile position
        unsigned *done = a.ctr + 1 + (size_t)i * nt * nt;   // (every item counts when it is done,
                                                            // converged problems' and empty groups' too)
        if (!(a.active && !a.active[i]) && c1 > c0) {
            schwarz_tile_cta<P, S, TT, T, true>(
                sm, ti, a.n, a.nbc, a.q, a.g, a.rev, c0, c1, ph & 1, ph >> 1, a.ntpx[ph], kband, mband, binv, binv_lo,
                a.interior, u + (size_t)i * a.vec, b + (size_t)i * a.vec, [&] {
                    if (threadIdx.x == 0) {
                        // the earlier occurrences of the nine positions: a position of phase tn
                        // ran kseq times before this colour group, plus once in it if its phase
                        // comes first in the sweep order; relaxed polls (an acquire per poll
                        // would also drop the SM's L1 lines that co-resident tiles are using),
                        // one acquire fence after
                        int go = 1;
                        const long long t0 = clock64();
                        for (int dj = -1; dj <= 1 && go; ++dj)
                            for (int di = -1; di <= 1 && go; ++di) {
                                const int In = I + di, Jn = J + dj;
                                if (In < 0 || In >= nt || Jn < 0 || Jn >= nt) continue;
                                const int tn = (In & 1) + 2 * (Jn & 1);
                                const unsigned need = (unsigned)kseq + ((a.rev ? tn > ph : tn < ph) ? 1u : 0u);
                                if (need == 0) continue;
                                const unsigned *c = done + (size_t)Jn * nt + In;
                                bool ok = ld_relaxed_u32(c) >= need;
                                while (!ok && *(volatile int *)a.status == 0 && clock64() - t0 < a.budget) {
                                    __nanosleep(64);
                                    ok = ld_relaxed_u32(c) >= need;
                                }
                                if (!ok) {
                                    atomicAdd(a.status, 1);
                                    go = 0;
                                }
                            }
                        asm volatile("fence.acq_rel.gpu;" ::: "memory");
                        s_go = go;
                    }
                    __syncthreads();
                    return s_go != 0;
                });
        }
        __syncthreads();   // the tile's writes of u, before it counts as finished
        if (threadIdx.x == 0 && !a.withhold) {
            __threadfence();
            atomicAdd(done + (size_t)J * nt + I, 1u);
        }
        __syncthreads();   // shared memory and s_item are reused by the next item
    }
}

// t[j][I] = sum_w Rb[I][w] d[j][Rlo[I]+w]   (x direction, n rows x nc)
template <typename T>
__global__ void k_restrict_x(int n, int nc, int wr, const T *__restrict__ Rb,
                             const int *__restrict__ Rlo, const T *__restrict__ d,
                             T *__restrict__ t, BatchRef bt)
{
    pdl_wait();
    const int I = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (I >= nc || (bt.active && !bt.active[blockIdx.z])) return;
    d += blockIdx.z * bt.vec;
    t += blockIdx.z * bt.aux;
    const int lo = Rlo[I];
    const T *row = d + (size_t)j * n;
    T acc = T(0);
    for (int w = 0; w < wr; ++w) {
        const int i = lo + w;
        if (i < n) acc = fma(Rb[(size_t)I * wr + w], row[i], acc);
    }
    t[(size_t)j * nc + I] = acc;
}

// dc[J][I] = sum_w Rb[J][w] t[Rlo[J]+w][I]   (y direction)
template <typename T>
__global__ void k_restrict_y(int n, int nc, int wr, const T *__restrict__ Rb,
                             const int *__restrict__ Rlo, const T *__restrict__ t,
                             T *__restrict__ dc, BatchRef bt)
{
    pdl_wait();
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
    if (I >= nc || (bt.active && !bt.active[blockIdx.z])) return;
    t += blockIdx.z * bt.aux;
    dc += blockIdx.z * bt.crs;
    const int lo = Rlo[J];
    T acc = T(0);
    for (int w = 0; w < wr; ++w) {
        const int j = lo + w;
        if (j < n) acc = fma(Rb[(size_t)J * wr + w], t[(size_t)j * nc + I], acc);
    }
    dc[(size_t)J * nc + I] = acc;
}

// t2[J][i] = sum_w Cb[i][w] ec[J][Clo[i]+w]   (x direction of R^T)
template <typename T>
__global__ void k_prolong_x(int n, int nc, int wc, const T *__restrict__ Cb,
                            const int *__restrict__ Clo, const T *__restrict__ ec,
                            T *__restrict__ t2, BatchRef bt)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
    if (i >= n || (bt.active && !bt.active[blockIdx.z])) return;
    ec += blockIdx.z * bt.crs;
    t2 += blockIdx.z * bt.aux;
    const int lo = Clo[i];
    T acc = T(0);
    for (int w = 0; w < wc; ++w) {
        const int I = lo + w;
        if (I < nc) acc = fma(Cb[(size_t)i * wc + w], ec[(size_t)J * nc + I], acc);
    }
    t2[(size_t)J * n + i] = acc;
}

// u[j][i] += sum_w Cb[j][w] t2[Clo[j]+w][i]   (y direction of R^T); with delta != nullptr
// the update is u += delta + (R^T e_c), u in double (end of a mixed-precision inner cycle).
template <typename T, typename TU>
__global__ void k_prolong_y(int n, int nc, int wc, const T *__restrict__ Cb,
                            const int *__restrict__ Clo, const T *__restrict__ t2,
                            const T *__restrict__ delta, TU *__restrict__ u, BatchRef bt)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n || (bt.active && !bt.active[blockIdx.z])) return;
    t2 += blockIdx.z * bt.aux;
    if (delta) delta += blockIdx.z * bt.vec;
    u += blockIdx.z * bt.vec;
    const int lo = Clo[j];
    T acc = T(0);
    for (int w = 0; w < wc; ++w) {
        const int J = lo + w;
        if (J < nc) acc = fma(Cb[(size_t)j * wc + w], t2[(size_t)J * n + i], acc);
    }
    const size_t k = (size_t)j * n + i;
    if (delta) u[k] += (TU)delta[k] + (TU)acc;
    else u[k] += (TU)acc;
}

// One 1D pass of b = (M (x) M) f: along y (AXIS 1, out[j][i] = sum_b M[j][b] in[j+b-p][i])
// or along x (AXIS 0, out[j][i] = sum_a M[i][a] in[j][i+a-p]); the two passes make
// 2(2p+1) multiply-adds per DOF instead of (2p+1)^2.
template <int P, int AXIS>
__global__ void k_mass_pass(int n, const double *__restrict__ Mb, const double *__restrict__ in,
                            double *__restrict__ out, long long vec)
{
    constexpr int W = 2 * P + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n) return;
    in += blockIdx.z * vec;
    out += blockIdx.z * vec;
    const int r = AXIS == 0 ? i : j;
    const double *row = Mb + (size_t)r * W;
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < W; ++a) {
        const int k = r + a - P;
        if (k >= 0 && k < n) acc = fma(__ldg(&row[a]), AXIS == 0 ? in[(size_t)j * n + k] : in[(size_t)k * n + i], acc);
    }
    out[(size_t)j * n + i] = acc;
}

// norm2 != nullptr (with part): the squared norm of every problem is finished inside the
// launch into norm2[problem] (the last CTA of a problem sums its partials)
template <int P, typename T, typename TO>
cudaError_t residual_p(const Solver &S, const T *kband, const T *mband, const T *u, const T *b, TO *d, double *part,
                       double *norm2, cudaStream_t st)
{
    // FP64: 64-wide tiles (the y pass's halo columns are 2p / 64 of its work instead of 2p / 32)
    constexpr int TX = sizeof(T) == sizeof(double) ? 64 : kResTX, TY = kResTY;
    dim3 blk(TX, TY), grd((S.n + TX - 1) / TX, (S.n + TY - 1) / TY, S.nbatch);
    const cudaError_t err = launch_pdl(k_residual2d<P, T, TO, TX, TY>, grd, blk, st, S.n, kband, mband, u, b, d,
                                       part, S.rcount, norm2, BatchRef{S.active, S.N, residual_partials(S), 0});
    count_launches(1);
    return err;
}

template <typename T, typename TO>
cudaError_t residual_any(const Solver &S, const T *kband, const T *mband, const T *u, const T *b, TO *d,
                         double *part, cudaStream_t st, double *norm2 = nullptr)
{
    switch (S.p) {
    case 2: return residual_p<2, T, TO>(S, kband, mband, u, b, d, part, norm2, st);
    case 3: return residual_p<3, T, TO>(S, kband, mband, u, b, d, part, norm2, st);
    case 4: return residual_p<4, T, TO>(S, kband, mband, u, b, d, part, norm2, st);
    case 5: return residual_p<5, T, TO>(S, kband, mband, u, b, d, part, norm2, st);
    case 6: return residual_p<6, T, TO>(S, kband, mband, u, b, d, part, norm2, st);
    case 7: return residual_p<7, T, TO>(S, kband, mband, u, b, d, part, norm2, st);
    case 8: return residual_p<8, T, TO>(S, kband, mband, u, b, d, part, norm2, st);
    default: return cudaErrorInvalidValue;
    }
}

// Blocks per CTA for a colour of nblocks Schwarz blocks of ss DOFs, among bmax, bmax / 2
// and bmax / 4 (bmax = 256 / ss, the compiled variants): the busiest SM holds
// ceil(CTAs / SMs) CTAs, each of ceil(c ss / 32) warps, and every warp costs the same
// FP64 pipe time, so the choice with the fewest warps on the busiest SM wins (a smaller
// CTA only when that is 2% fewer; for a many-wave grid the hardware balances the SMs
// anyway).  A single-wave colour of 772 CTAs on 152 SMs (p = 3, 4 at 1024^2) otherwise
// leaves some SMs with 6 CTAs and the mean at 5.1: 19% above the mean; 64-thread CTAs
// bring that to 4%.
inline int lattice_bpc(long long nblocks, int ss, int nsm)
{
    const int bmax = 256 / ss;
    int best = bmax;
    long long best_load = -1;
    for (int c = bmax; c >= 1 && (c == bmax || c * 2 == bmax || c * 4 == bmax); c /= 2) {
        const long long ncta = (nblocks + c - 1) / c;
        const long long load = (ncta + nsm - 1) / nsm * ((c * ss + 31) / 32);
        if (best_load < 0 || load * 50 < best_load * 49) { best = c; best_load = load; }
    }
    return best;
}

// the block inverses transposed per class, as the TILE and per-colour FP32 kernels read them
template <typename T>
const T *tile_binv(const Solver &S);
template <>
const double *tile_binv<double>(const Solver &S) { return S.binv_t; }
template <>
const float *tile_binv<float>(const Solver &S) { return S.mx.binv_t; }

// launches the compiled variant with bpc blocks per CTA (BPC, BPC / 2 or BPC / 4, the ones
// lattice_bpc offers)
template <int P, int SB, int BPC, typename T>
cudaError_t launch_lattice_direct(const Solver &S, int q, int ox, int oy, int nbx, int nblocks, const T *stencil,
                                  const T *binv, int interior, T *u, const T *b, cudaStream_t st, int bpc)
{
    if constexpr (BPC % 2 == 0) {
        if (bpc < BPC)
            return launch_lattice_direct<P, SB, BPC / 2, T>(S, q, ox, oy, nbx, nblocks, stencil, binv, interior, u, b,
                                                            st, bpc);
    }
    return launch_pdl(k_schwarz_lattice2d<P, SB, BPC, T>, dim3((nblocks + BPC - 1) / BPC, S.nbatch),
                      dim3((BPC * SB * SB + 31) / 32 * 32), st, S.n, S.ht.npc, S.ht.nbc, q, ox, oy, nbx, nblocks,
                      stencil, (const int *)S.pcls, tile_binv<T>(S), S.boundary64_t(), interior,
                      (const int *)S.bcls, u, b, BatchRef{S.active, S.N, 0, 0});
}

// the FP64 sum-factorised colour kernel (5x5 and 7x7 blocks) with bpc blocks per CTA
template <int P, int SB, int BPC>
cudaError_t launch_lattice_pd(const Solver &S, int q, int ox, int oy, int nbx, int nblocks, const double *kband,
                              const double *mband, const double *binv, double *u, const double *b, cudaStream_t st,
                              int bpc)
{
    if constexpr (BPC % 2 == 0) {
        if (bpc < BPC)
            return launch_lattice_pd<P, SB, BPC / 2>(S, q, ox, oy, nbx, nblocks, kband, mband, binv, u, b, st, bpc);
    }
    return launch_pdl(k_schwarz_lattice2d_pd<P, SB, BPC>, dim3((nblocks + BPC - 1) / BPC, S.nbatch),
                      dim3((BPC * SB * SB + 31) / 32 * 32), st, S.n, S.ht.nbc, q, ox, oy, nbx, nblocks, kband, mband,
                      S.binv_t, (const int *)S.bcls, u, b, BatchRef{S.active, S.N, 0, 0});
}

// the colour's dynamic shared memory: the tensor-core tile or the SIMT frame step
template <int P, int S>
size_t tc_colour_smem(int q)
{
    const size_t a = TcGeom<P, S>::smem(q), b = sizeof(SfSmem<P, S, float, 256>);
    return a > b ? a : b;
}

template <int P, int S>
cudaError_t launch_tc_colour(const Solver &S_, int ox, int oy, int nbx, int nby, const float *kband,
                             const float *mband, const float *binv, int interior, float *u, const float *b,
                             cudaStream_t st)
{
    using G = TcGeom<P, S>;
    int ix0 = 0, nix = 0, iy0 = 0, niy = 0;
    tc_interior_rect(S_, ox, nbx, ix0, nix);
    tc_interior_rect(S_, oy, nby, iy0, niy);
    if (nix <= 0 || niy <= 0) ix0 = iy0 = nix = niy = 0;   // no interior block: all frame
    const int ntx = (nix + G::TBX - 1) / G::TBX, nty = (niy + G::TBY - 1) / G::TBY;
    const int nframe = nbx * nby - nix * niy;
    constexpr int NB = SfSmem<P, S, float, 256>::NB;
    const int nfc = (nframe + NB - 1) / NB, grid = nfc + ntx * nty;
    if (grid == 0) return cudaSuccess;
    TcColourArgs a;
    a.n = S_.n;
    a.nbc = S_.ht.nbc;
    a.q = S_.q;
    a.ox = ox;
    a.oy = oy;
    a.nbx = nbx;
    a.ix0 = ix0;
    a.iy0 = iy0;
    a.nix = nix;
    a.niy = niy;
    a.ntx = ntx > 0 ? ntx : 1;
    a.nfc = nfc;
    a.nframe = nframe;
    a.interior = interior;
    a.skip_copy = (S_.opt.test_flags & IGA2L_TEST_SKIP_OPERATOR_COPY) != 0;
    a.budget = S_.opt.wait_budget_cycles;
    a.kband = kband;
    a.mband = mband;
    a.binv = S_.mx.binv_t;
    a.binv_lo = S_.boundary_lo_t();
    a.gtc = S_.mx.gtc;
    a.b = b;
    a.u = u;
    a.status = S_.wait_status;
    return launch_pdl_smem(k_schwarz_tc_colour<P, S>, dim3(grid), dim3(256), tc_colour_smem<P, S>(S_.q), st, a);
}

template <int P, int S>
bool tc_colour_prepare_p(const Solver &S_, std::string &why)
{
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, S_.device);
    const size_t need = tc_colour_smem<P, S>(S_.q);
    using G = TcGeom<P, S>;
    // the region's row index is taken from a float reciprocal, exact while RW < 2^9 and the
    // element index < 2^16
    const bool shape_ok = G::RW(S_.q) < 512 && G::RW(S_.q) * G::RH(S_.q) + 256 * 32 < 65536;
    if (e != cudaSuccess || need > (size_t)optin || !shape_ok) {
        why = "tensor-core colour step: " + std::to_string(need) + " bytes of shared memory for lattice period " +
              std::to_string(S_.q) + " exceed the device's " + std::to_string(optin);
        return false;
    }
    // the largest allowance: handles with other periods share the kernel
    e = cudaFuncSetAttribute(k_schwarz_tc_colour<P, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) {
        why = std::string("tensor-core colour step: ") + cudaGetErrorString(e);
        return false;
    }
    return true;
}

template <int P, int SB, typename T>
cudaError_t schwarz_lattice_p(const Solver &S, const T *stencil, const T *kband, const T *mband, const T *binv, T *u,
                              const T *b, bool reverse, cudaStream_t st)
{
    // FP32: the packed sum-factorised kernel (the direct form is bound by its L1 loads);
    // FP64: the direct form for 3x3 and 5x5 blocks, the per-DOF factorised kernel for 7x7
    // blocks.  Measured at 1024^2: p = 7, 8 sweeps 22% faster factorised (38% fewer FMAs);
    // p = 5, 6 (23% and 20% fewer FMAs) equal or 4% slower, so they keep the direct form,
    // whose FP64 pipe is 96% busy against 87% for the factorised one; with 3x3 blocks the
    // factorised residual needs more FMAs than the stencil.
    constexpr bool SF = sizeof(T) == sizeof(float);
    constexpr int BPC = 256 / (SB * SB), NBSF = 256 / (SB + 2 * P);
    const int q = S.q, ncol = q * q;
    const int interior = S.ht.L * S.ht.nbc + S.ht.L;
    for (int t = 0; t < ncol; ++t) {
        const int c = reverse ? ncol - 1 - t : t;
        // colour c visits offsets (rank_x g mod q, rank_y g mod q)
        const int ox = ((c % q) * S.g) % q, oy = ((c / q) * S.g) % q;
        const int nbx = (S.n - ox + q - 1) / q, nby = (S.n - oy + q - 1) / q;
        const int nblocks = nbx * nby;
        if (nblocks <= 0) continue;
        cudaError_t err;
        if constexpr (SF) {
            if (S.mx.gtc) {   // IGA2L_MIXED_TF32: interior blocks on the tensor cores, same launch
                if constexpr (P <= kTcMaxP)
                    err = launch_tc_colour<P, SB>(S, ox, oy, nbx, nby, kband, mband, binv, interior, u, b, st);
                else
                    err = cudaErrorInvalidValue;
            } else {
                err = launch_pdl(k_schwarz_lattice2d_sf<P, SB, T>, dim3((nblocks + NBSF - 1) / NBSF, S.nbatch),
                                 dim3(256), st, S.n, S.ht.nbc, q, ox, oy, nbx, 0, 0, 0, 0, nblocks, kband, mband,
                                 tile_binv<T>(S), S.boundary_lo_t(), interior, u, b, BatchRef{S.active, S.N, 0, 0});
            }
        } else {
            const int bpc = lattice_bpc((long long)nblocks * S.nbatch, SB * SB, S.nsm);
            if constexpr (SB >= 7)   // sum factorisation pays once the block is as wide as the stencil
                err = launch_lattice_pd<P, SB, BPC>(S, q, ox, oy, nbx, nblocks, kband, mband, binv, u, b, st, bpc);
            else
                err = launch_lattice_direct<P, SB, BPC, T>(S, q, ox, oy, nbx, nblocks, stencil, binv, interior, u, b,
                                                           st, bpc);
        }
        count_launches(1);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// the TILE sweep as one work-list launch over every problem of the handle
template <int P, int SB, typename T>
cudaError_t schwarz_tile_work_p(const Solver &S, const T *kband, const T *mband, const T *binv, T *u, const T *b,
                                bool reverse, cudaStream_t st)
{
    constexpr int TT = tile_side(P);
    using G = TileGeom<P, SB, TT>;
    const int nt = (S.n + TT - 1) / TT;
    TileWorkArgs a;
    a.n = S.n;
    a.nbc = S.ht.nbc;
    a.q = S.q;
    a.g = S.g;
    a.rev = reverse ? 1 : 0;
    a.interior = S.ht.L * S.ht.nbc + S.ht.L;
    a.nbatch = S.nbatch;
    a.groups = S.tile_groups > 1 ? S.tile_groups : 1;
    a.withhold = (S.opt.test_flags & IGA2L_TEST_WITHHOLD_PROGRESS) != 0;
    a.nt = nt;
    long long per = 0, widest = 0;
    for (int t = 0; t < 4; ++t) {
        const int ntpx = (nt - (t & 1) + 1) / 2, ntpy = (nt - (t >> 1) + 1) / 2;
        a.ntpx[t] = ntpx > 0 ? ntpx : 1;
        a.tiles[t] = ntpx > 0 && ntpy > 0 ? ntpx * ntpy : 0;
        per += a.tiles[t];
        widest = std::max(widest, (long long)a.tiles[t] * S.nbatch);
    }
    a.per_group = per * S.nbatch;
    a.total = a.per_group * a.groups;
    if (a.total > (1LL << 31)) return cudaErrorInvalidValue;   // the item counter is 32-bit
    a.ctr = S.tile_ctr;
    a.active = S.active;
    a.vec = S.N;
    a.status = S.wait_status;
    a.budget = S.opt.wait_budget_cycles;
    cudaError_t e = cudaMemsetAsync(S.tile_ctr, 0, sizeof(unsigned) * (1 + (size_t)S.nbatch * nt * nt), st);
    if (e != cudaSuccess) return e;
    // no more CTAs than the largest phase has items: otherwise the CTAs that start last claim
    // the next phase's items at once and the SMs they sit on run fewer tiles of this phase
    // while others run more (measured: p = 5 phase 0 at 1024^2 took 195 us against 153)
    const long long grid = std::min(widest, (long long)S.tile_work_ctas);
    if (grid <= 0) return cudaSuccess;
    k_schwarz_tile2d_work<P, SB, TT, T><<<(unsigned)grid, G::NT, 0, st>>>(a, kband, mband, tile_binv<T>(S),
                                                                          S.boundary_lo_t(), u, b);
    count_launches(1);
    return cudaGetLastError();
}

template <int P, int SB, typename T>
cudaError_t schwarz_tile_p(const Solver &S, const T *kband, const T *mband, const T *binv, T *u, const T *b,
                           bool reverse, cudaStream_t st)
{
    if (S.tile_ctr) return schwarz_tile_work_p<P, SB, T>(S, kband, mband, binv, u, b, reverse, st);
    constexpr int TT = tile_side(P);
    using G = TileGeom<P, SB, TT>;
    const int interior = S.ht.L * S.ht.nbc + S.ht.L;
    const int nt = (S.n + TT - 1) / TT;
    // colour groups: for each group in turn the four tile phases run that group's colours
    // (group k = lattice colours ceil(k q^2 / G) .. ceil((k + 1) q^2 / G) - 1)
    const int ncol = S.q * S.q, G_ = S.tile_groups > 1 ? S.tile_groups : 1;
    for (int kk = 0; kk < G_; ++kk) {
        const int k = reverse ? G_ - 1 - kk : kk;
        const int c0 = (k * ncol + G_ - 1) / G_, c1 = ((k + 1) * ncol + G_ - 1) / G_;
        if (c1 <= c0) continue;
        for (int t = 0; t < 4; ++t) {
            const int ph = reverse ? 3 - t : t;
            const int px = ph & 1, py = ph >> 1;
            const int ntpx = (nt - px + 1) / 2, ntpy = (nt - py + 1) / 2;
            if (ntpx <= 0 || ntpy <= 0) continue;
            const cudaError_t err =
                launch_pdl(k_schwarz_tile2d<P, SB, TT, T>, dim3(ntpx * ntpy, S.nbatch), dim3(G::NT), st, S.n,
                           S.ht.nbc, S.q, S.g, reverse ? 1 : 0, c0, c1, px, py, ntpx, kband, mband,
                           tile_binv<T>(S), S.boundary_lo_t(), interior, u, b, BatchRef{S.active, S.N, 0, 0});
            count_launches(1);
            if (err != cudaSuccess) return err;
        }
    }
    return cudaSuccess;
}

template <int P, int SB, typename T>
cudaError_t schwarz_p(const Solver &S, const T *stencil, const T *kband, const T *mband, const T *binv, T *u,
                      const T *b, bool reverse, cudaStream_t st)
{
    if constexpr (SB * SB <= 32) {   // the TILE kernel keeps a block in one warp
        if (S.opt.schedule == IGA2L_SCHED_TILE)
            return schwarz_tile_p<P, SB, T>(S, kband, mband, binv, u, b, reverse, st);
    }
    return schwarz_lattice_p<P, SB, T>(S, stencil, kband, mband, binv, u, b, reverse, st);
}

template <typename T>
cudaError_t schwarz_any(const Solver &S, const T *stencil, const T *kband, const T *mband, const T *binv, T *u,
                        const T *b, bool reverse, cudaStream_t st)
{
    if (S.s == 3) {
        switch (S.p) {
        case 2: return schwarz_p<2, 3, T>(S, stencil, kband, mband, binv, u, b, reverse, st);
        case 3: return schwarz_p<3, 3, T>(S, stencil, kband, mband, binv, u, b, reverse, st);
        case 4: return schwarz_p<4, 3, T>(S, stencil, kband, mband, binv, u, b, reverse, st);
        default: break;
        }
    } else if (S.s == 5) {
        if (S.p == 5) return schwarz_p<5, 5, T>(S, stencil, kband, mband, binv, u, b, reverse, st);
        if (S.p == 6) return schwarz_p<6, 5, T>(S, stencil, kband, mband, binv, u, b, reverse, st);
    } else if (S.s == 7) {
        if (S.p == 7) return schwarz_p<7, 7, T>(S, stencil, kband, mband, binv, u, b, reverse, st);
        if (S.p == 8) return schwarz_p<8, 7, T>(S, stencil, kband, mband, binv, u, b, reverse, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t restrict_any(const Solver &S, const T *Rb, const T *d, T *t, T *dc, cudaStream_t st)
{
    const int nc = S.nc, n = S.n;
    const BatchRef bt{S.active, S.N, (long long)n * nc, S.Nc};
    cudaError_t err = launch_pdl(k_restrict_x<T>, dim3((nc + 127) / 128, n, S.nbatch), dim3(128), st, n, nc,
                                 S.ht.wr, Rb, (const int *)S.Rlo, d, t, bt);
    count_launches(1);
    if (err != cudaSuccess) return err;
    err = launch_pdl(k_restrict_y<T>, dim3((nc + 127) / 128, nc, S.nbatch), dim3(128), st, n, nc, S.ht.wr, Rb,
                     (const int *)S.Rlo, (const T *)t, dc, bt);
    count_launches(1);
    return err;
}

template <typename T, typename TU>
cudaError_t prolong_any(const Solver &S, const T *Cb, const T *ec, T *t2, const T *delta, TU *u,
                        cudaStream_t st)
{
    const int nc = S.nc, n = S.n;
    const BatchRef bt{S.active, S.N, (long long)n * nc, S.Nc};
    cudaError_t err = launch_pdl(k_prolong_x<T>, dim3((n + 127) / 128, nc, S.nbatch), dim3(128), st, n, nc,
                                 S.ht.wc, Cb, (const int *)S.Clo, ec, t2, bt);
    count_launches(1);
    if (err != cudaSuccess) return err;
    err = launch_pdl(k_prolong_y<T, TU>, dim3((n + 127) / 128, n, S.nbatch), dim3(128), st, n, nc, S.ht.wc, Cb,
                     (const int *)S.Clo, (const T *)t2, delta, u, bt);
    count_launches(1);
    return err;
}

}  // namespace

cudaError_t upload_interior_rows(int p, const double *k1, const double *m1)
{
    static std::mutex mu;
    static bool done[64][kMaxP + 1] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || p < 0 || p > kMaxP) return cudaErrorInvalidValue;
    if (done[dev][p]) return cudaSuccess;
    constexpr int W1 = 2 * kMaxP + 1;
    double2 km64[W1], mk64[W1];
    float2 km32[W1], mk32[W1];
    const int w = 2 * p + 1;
    for (int i = 0; i < w; ++i) {
        km64[i] = make_double2(k1[i], m1[i]);
        mk64[i] = make_double2(m1[i], k1[i]);
        km32[i] = make_float2((float)k1[i], (float)m1[i]);
        mk32[i] = make_float2((float)m1[i], (float)k1[i]);
    }
    e = cudaMemcpyToSymbol(c_km1d, km64, sizeof(double2) * w, sizeof(double2) * W1 * p);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_mk1d, mk64, sizeof(double2) * w, sizeof(double2) * W1 * p);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_km1f, km32, sizeof(float2) * w, sizeof(float2) * W1 * p);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_mk1f, mk32, sizeof(float2) * w, sizeof(float2) * W1 * p);
    if (e == cudaSuccess) done[dev][p] = true;
    return e;
}

int residual_partials(const Solver &S)
{
    if (S.dim == 3) return residual3d_partials(S);
    return ((S.n + kResTX - 1) / kResTX) * ((S.n + kResTY - 1) / kResTY);
}

cudaError_t launch_residual(const Solver &S, const double *u, const double *b, double *d,
                            double *part, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_residual(S, u, b, d, part, st);
    return residual_any<double, double>(S, S.Kb, S.Mb, u, b, d, part, st);
}

cudaError_t launch_residual_norm(const Solver &S, const double *u, const double *b, double *d, double *norm2,
                                 cudaStream_t st)
{
    if (S.dim == 3) {
        cudaError_t e = launch3d_residual(S, u, b, d, S.part, st);
        return e == cudaSuccess ? launch_norm_finish(S, S.part, norm2, st) : e;
    }
    return residual_any<double, double>(S, S.Kb, S.Mb, u, b, d, S.part, st, norm2);
}

cudaError_t launch_apply_A(const Solver &S, const double *u, double *y, cudaStream_t st)
{
    return launch_residual(S, u, nullptr, y, nullptr, st);
}

cudaError_t launch_norm_finish(const Solver &S, const double *part, double *out, cudaStream_t st)
{
    k_sum_partials<<<S.nbatch, 1024, 0, st>>>(part, residual_partials(S), out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_schwarz(const Solver &S, double *u, const double *b, bool reverse,
                           cudaStream_t st)
{
    if (S.dim == 3) return launch3d_schwarz(S, u, b, reverse, st);
    return schwarz_any<double>(S, S.stencil, S.Kb, S.Mb, S.binv, u, b, reverse, st);
}

cudaError_t launch_restrict(const Solver &S, const double *d, double *dc, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_restrict(S, d, dc, st);
    return restrict_any<double>(S, S.Rb, d, S.t, dc, st);
}

cudaError_t launch_prolong_add(const Solver &S, const double *ec, double *u, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_prolong_add(S, ec, u, st);
    return prolong_any<double, double>(S, S.Cb, ec, S.t2, nullptr, u, st);
}

// ---- batch control -----------------------------------------------------------------

// start of a batched solve: problems with a zero initial residual are done at once
__global__ void k_batch_init(int nb, const double *__restrict__ norm2, double *__restrict__ norm0,
                             int *__restrict__ active, int *__restrict__ cycles, double *__restrict__ relres)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    norm0[k] = norm2[k];
    active[k] = norm2[k] > 0.0 ? 1 : 0;
    cycles[k] = 0;
    relres[k] = 0.0;
}

// after a cycle: count it for every active problem and retire those at the tolerance;
// count[0] = number of problems still active (nonfinite norms retire with relres = nan).
// With ctl (a device-driven batched solve): tol comes from ctl, ctl->k counts the cycles
// and the WHILE condition is set to continue while a problem is active and k < maxc.
__global__ void k_batch_check(int nb, double tol, const double *__restrict__ norm2, const double *__restrict__ norm0,
                              int *__restrict__ active, int *__restrict__ cycles, double *__restrict__ relres,
                              int *__restrict__ count, SolveCtl *ctl, cudaGraphConditionalHandle cond)
{
    __shared__ int act;
    if (threadIdx.x == 0) act = 0;
    if (ctl) tol = ctl->tol;
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        if (!active[k]) continue;
        cycles[k] += 1;
        const double rel = sqrt(norm2[k] / norm0[k]);
        relres[k] = rel;
        if (rel <= tol || !(rel == rel)) active[k] = 0;
        else atomicAdd(&act, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        count[0] = act;
        if (ctl) {
            const int k = ctl->k + 1;
            ctl->k = k;
            cudaGraphSetConditional(cond, act > 0 && k < ctl->maxc ? 1u : 0u);
        }
    }
}

cudaError_t launch_batch_init(const Solver &S, const double *norm2, double *norm0, int *cycles, double *relres,
                              cudaStream_t st)
{
    k_batch_init<<<(S.nbatch + 127) / 128, 128, 0, st>>>(S.nbatch, norm2, norm0, S.active, cycles, relres);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batch_check(const Solver &S, double tol, const double *norm2, const double *norm0, int *cycles,
                               double *relres, int *count, cudaStream_t st)
{
    k_batch_check<<<1, 256, 0, st>>>(S.nbatch, tol, norm2, norm0, S.active, cycles, relres, count, nullptr,
                                     cudaGraphConditionalHandle{});
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batch_check_loop(const Solver &S, const double *norm2, const double *norm0, int *cycles,
                                    double *relres, int *count, SolveCtl *ctl, cudaGraphConditionalHandle cond,
                                    cudaStream_t st)
{
    k_batch_check<<<1, 256, 0, st>>>(S.nbatch, 0.0, norm2, norm0, S.active, cycles, relres, count, ctl, cond);
    count_launches(1);
    return cudaGetLastError();
}

// ---- device-driven solve ----------------------------------------------------------

// One thread: the host loop's test after a cycle, on the device (same arithmetic:
// rel = sqrt(norm2) / r0, IEEE square root and quotient), then the WHILE condition.
__global__ void k_solve_check(const double *__restrict__ norm2, SolveCtl *__restrict__ c, double *__restrict__ hist,
                              cudaGraphConditionalHandle cond)
{
    const double rsq = norm2[0];
    const int k = c->k + 1;
    c->k = k;
    unsigned int more = 0;
    if (!isfinite(rsq)) {
        c->status = 2;
    } else {
        const double rel = sqrt(rsq) / c->r0;
        c->rel = rel;
        if (k <= kSolveHistCap) hist[k - 1] = rel;
        if (rel <= c->tol) c->status = 1;
        else if (k >= c->maxc) c->status = 0;
        else more = 1;
    }
    cudaGraphSetConditional(cond, more);
}

cudaError_t launch_solve_check(const double *norm2, SolveCtl *ctl, double *hist, cudaGraphConditionalHandle cond,
                               cudaStream_t st)
{
    k_solve_check<<<1, 1, 0, st>>>(norm2, ctl, hist, cond);
    count_launches(1);
    return cudaGetLastError();
}

// ---- mixed precision -------------------------------------------------------------

cudaError_t launch_outer_residual(const Solver &S, const double *u, const double *b, float *r32,
                                  double *part, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_outer_residual(S, u, b, r32, part, st);
    return residual_any<double, float>(S, S.Kb, S.Mb, u, b, r32, part, st);
}

cudaError_t launch_outer_residual_norm(const Solver &S, const double *u, const double *b, float *r32,
                                       double *norm2, cudaStream_t st)
{
    if (S.dim == 3) {
        cudaError_t e = launch3d_outer_residual(S, u, b, r32, S.part, st);
        return e == cudaSuccess ? launch_norm_finish(S, S.part, norm2, st) : e;
    }
    return residual_any<double, float>(S, S.Kb, S.Mb, u, b, r32, S.part, st, norm2);
}

cudaError_t launch_inner_fine(const Solver &S, const float *r32, bool reverse, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_inner_fine(S, r32, st);
    const MixedState &X = S.mx;
    cudaError_t e = cudaMemsetAsync(X.delta, 0, sizeof(float) * S.N * S.nbatch, st);
    if (e == cudaSuccess)
        e = S.pgx > 0 ? launch_schwarz_persist(S, X.delta, r32, reverse, st)
                      : schwarz_any<float>(S, X.stencil, X.Kb, X.Mb, X.binv, X.delta, r32, reverse, st);
    if (e == cudaSuccess) e = residual_any<float, float>(S, X.Kb, X.Mb, X.delta, r32, X.d, nullptr, st);
    if (e == cudaSuccess) e = restrict_any<float>(S, X.Rb, X.d, X.t, X.dc, st);
    return e;
}

namespace {
template <int P, int SB>
int tile_work_ctas_p(const Solver &S)
{
    constexpr int TT = tile_side(P);
    using G = TileGeom<P, SB, TT>;
    int per_sm = 0;
    cudaError_t e;
    if (S.mx.enabled)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_schwarz_tile2d_work<P, SB, TT, float>, G::NT, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_schwarz_tile2d_work<P, SB, TT, double>, G::NT, 0);
    return e == cudaSuccess ? per_sm * S.nsm : 0;
}
}  // namespace

int tile_work_ctas(const Solver &S)
{
    switch (S.p) {
    case 2: return tile_work_ctas_p<2, 3>(S);
    case 3: return tile_work_ctas_p<3, 3>(S);
    case 4: return tile_work_ctas_p<4, 3>(S);
    case 5: return tile_work_ctas_p<5, 5>(S);
    case 6: return tile_work_ctas_p<6, 5>(S);
    default: return 0;
    }
}

bool tc_colour_prepare(const Solver &S, std::string &why)
{
    switch (S.p) {
    case 2: return tc_colour_prepare_p<2, 3>(S, why);
    case 3: return tc_colour_prepare_p<3, 3>(S, why);
    case 4: return tc_colour_prepare_p<4, 3>(S, why);
    case 5: return tc_colour_prepare_p<5, 5>(S, why);
    default: why = "the tensor-core colour step is compiled for p = 2..5"; return false;
    }
}

cudaError_t launch_inner_sweep(const Solver &S, float *u, const float *b, bool reverse, cudaStream_t st)
{
    const MixedState &X = S.mx;
    return S.pgx > 0 ? launch_schwarz_persist(S, u, b, reverse, st)
                     : schwarz_any<float>(S, X.stencil, X.Kb, X.Mb, X.binv, u, b, reverse, st);
}

cudaError_t launch_inner_update(const Solver &S, double *u, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_inner_update(S, u, st);
    const MixedState &X = S.mx;
    return prolong_any<float, double>(S, X.Cb, X.ec, X.t2, X.delta, u, st);
}

cudaError_t launch_mass2(const Solver &S, const double *f, double *b, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_mass(S, f, b, st);
    // y pass into the workspace d, then the x pass into b
    dim3 grd((S.n + 127) / 128, S.n, S.nbatch);
    switch (S.p) {
#define IGA2L_MASS(PP)                                                                           \
    case PP:                                                                                     \
        k_mass_pass<PP, 1><<<grd, 128, 0, st>>>(S.n, S.Mb, f, S.d, S.N);                         \
        k_mass_pass<PP, 0><<<grd, 128, 0, st>>>(S.n, S.Mb, S.d, b, S.N);                         \
        break;
    IGA2L_MASS(2) IGA2L_MASS(3) IGA2L_MASS(4) IGA2L_MASS(5) IGA2L_MASS(6) IGA2L_MASS(7) IGA2L_MASS(8)
#undef IGA2L_MASS
    default: return cudaErrorInvalidValue;
    }
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace iga2l
