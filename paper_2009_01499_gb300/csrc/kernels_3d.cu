// kernels_3d.cu -- the two-level cycle in 3D (the paper's method on (0,1)^3).
//
// A_p = K(x)M(x)M + M(x)K(x)M + M(x)M(x)K.  Every application of A_p is sum-
// factorised with the exact 1D band rows (row x of K, M couples DOF x with x+a-p):
//   tK = K_x u, tM = M_x u;   S1 = M_y tK + K_y tM, MM = M_y tM;   A u = M_z S1 + K_z MM,
// i.e. 2 + 3 + 2 band passes of width 2p+1 instead of (2p+1)^3 taps per row.
//
//   residual    d = b - A u (+ per-CTA partial sums of d^2), tiles in shared memory
//   schwarz     one LATTICE colour: per block, the patch (s+2p)^3 of u, three band
//               passes, the block residual, the block inverse of its class
//   band_axis   one 1D band along one axis of a 3D array (restriction, prolongation, mass)
//   level_*     degree-1 hierarchy: 27-point stencil, red-black Gauss-Seidel on the 8
//               parity sub-lattices, trilinear transfers, dense coarsest inverse
// Templated on the storage type (double: FP64 form; float: inner cycle of the mixed form).
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace iga2l {

namespace {

constexpr int kR3X = 16, kR3Y = 8, kR3Z = 4;   // residual tile (outputs per CTA)

template <int P>
constexpr int res3d_smem_elems()
{
    return (kR3Z + 2 * P) * (kR3Y + 2 * P) * (kR3X + 2 * P)      // u tile
           + 2 * (kR3Z + 2 * P) * (kR3Y + 2 * P) * kR3X          // tK, tM
           + 2 * (kR3Z + 2 * P) * kR3Y * kR3X;                   // S1, MM
}

// d = b - A u (b != nullptr) or d = A u, arithmetic in T, output TO; part = sum d^2
template <int P, typename T, typename TO>
__global__ void __launch_bounds__(256)
k_residual3d(int n, const T *__restrict__ Kb, const T *__restrict__ Mb, const T *__restrict__ u,
             const T *__restrict__ b, TO *__restrict__ d, double *__restrict__ part)
{
    constexpr int W = 2 * P + 1;
    constexpr int UZ = kR3Z + 2 * P, UY = kR3Y + 2 * P, UX = kR3X + 2 * P;
    extern __shared__ __align__(16) unsigned char smem3[];
    T *su = reinterpret_cast<T *>(smem3);
    T *tK = su + UZ * UY * UX;
    T *tM = tK + UZ * UY * kR3X;
    T *S1 = tM + UZ * UY * kR3X;
    T *MM = S1 + UZ * kR3Y * kR3X;
    __shared__ double red[8];
    const int x0 = blockIdx.x * kR3X, y0 = blockIdx.y * kR3Y, z0 = blockIdx.z * kR3Z;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < UZ * UY * UX; i += nth) {
        const int lx = i % UX, ly = (i / UX) % UY, lz = i / (UX * UY);
        const int gx = x0 + lx - P, gy = y0 + ly - P, gz = z0 + lz - P;
        su[i] = (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n)
                    ? u[((size_t)gz * n + gy) * n + gx] : T(0);
    }
    __syncthreads();
    // x pass on (UZ, UY, kR3X)
    for (int i = tid; i < UZ * UY * kR3X; i += nth) {
        const int lx = i % kR3X, r = i / kR3X;   // r = lz * UY + ly
        const int gx = x0 + lx;
        T k = T(0), m = T(0);
        if (gx < n) {
            const T *kr = Kb + (size_t)gx * W, *mr = Mb + (size_t)gx * W;
            const T *ur = su + r * UX + lx;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                k = fma(kr[a], ur[a], k);
                m = fma(mr[a], ur[a], m);
            }
        }
        tK[i] = k;
        tM[i] = m;
    }
    __syncthreads();
    // y pass on (UZ, kR3Y, kR3X)
    for (int i = tid; i < UZ * kR3Y * kR3X; i += nth) {
        const int lx = i % kR3X, ly = (i / kR3X) % kR3Y, lz = i / (kR3X * kR3Y);
        const int gy = y0 + ly;
        T s1 = T(0), mm = T(0);
        if (gy < n) {
            const T *kr = Kb + (size_t)gy * W, *mr = Mb + (size_t)gy * W;
#pragma unroll
            for (int bb = 0; bb < W; ++bb) {
                const int j = (lz * UY + ly + bb) * kR3X + lx;
                s1 = fma(mr[bb], tK[j], s1);
                s1 = fma(kr[bb], tM[j], s1);
                mm = fma(mr[bb], tM[j], mm);
            }
        }
        S1[i] = s1;
        MM[i] = mm;
    }
    __syncthreads();
    // z pass and output, one thread per output (kR3X * kR3Y * kR3Z = 512 outputs, 2 per thread)
    double sq = 0.0;
    for (int i = tid; i < kR3Z * kR3Y * kR3X; i += nth) {
        const int lx = i % kR3X, ly = (i / kR3X) % kR3Y, lz = i / (kR3X * kR3Y);
        const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
        if (gx >= n || gy >= n || gz >= n) continue;
        const T *kr = Kb + (size_t)gz * W, *mr = Mb + (size_t)gz * W;
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < W; ++c) {
            const int j = ((lz + c) * kR3Y + ly) * kR3X + lx;
            acc = fma(mr[c], S1[j], acc);
            acc = fma(kr[c], MM[j], acc);
        }
        const size_t gi = ((size_t)gz * n + gy) * n + gx;
        const T dv = b ? b[gi] - acc : acc;
        if (d) d[gi] = (TO)dv;
        sq += (double)dv * (double)dv;
    }
    if (part) {
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
        if ((tid & 31) == 0) red[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < nth / 32; ++w) tot += red[w];
            part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = tot;
        }
    }
}

// One LATTICE colour in 3D with NB Schwarz blocks per CTA (256 threads) and every pass
// spread over all threads of the CTA: the patches (S + 2P)^3 of the NB blocks are staged
// together, then the x pass (pairs K_x u, M_x u), the y pass (S1 = M_y tK + K_y tM,
// MM = M_y tM), the z pass with the block residual, and the block solves, each a loop over
// all (block, point) items of the CTA.  Same arithmetic as k_schwarz_lattice3d per item;
// the x and z passes run as pairs (packed FP32 FMA for T = float).
template <typename T>
struct Vec2_3d;
template <>
struct Vec2_3d<float> { using type = float2; };
template <>
struct Vec2_3d<double> { using type = double2; };

__device__ __forceinline__ float2 fma2_3d(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 fma2_3d(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

template <int P, typename T>
struct Lattice3dGeom {
    static constexpr int S = 3, R = 1, W = 2 * P + 1, SS = S * S * S, PW = S + 2 * P;
    static constexpr int NB = sizeof(T) == sizeof(float) ? 4 : 2;   // blocks per CTA (shared memory)
};

template <int P, typename T>
__global__ void __launch_bounds__(256)
k_schwarz_lattice3d_mb(int n, int nbc, int q, int ox, int oy, int oz, int nbx, int nby, int nblocks,
                       const T *__restrict__ Kb, const T *__restrict__ Mb, const T *__restrict__ binv,
                       const double *__restrict__ binv64, int interior, const int *__restrict__ bcls,
                       T *__restrict__ u, const T *__restrict__ b)
{
    using G = Lattice3dGeom<P, T>;
    using T2 = typename Vec2_3d<T>::type;
    constexpr int S = G::S, R = G::R, W = G::W, SS = G::SS, PW = G::PW, NB = G::NB;
    constexpr int NT = 256;
    __shared__ T pu[NB][PW * PW * PW];
    __shared__ T2 tKM[NB][PW * PW * S];     // (K_x u, M_x u)
    __shared__ T2 sMM[NB][PW * S * S];      // (S1, MM)
    __shared__ T rs[NB][SS];
    __shared__ int cen[NB][3];
    const int tid = threadIdx.x;
    const int blk0 = blockIdx.x * NB;
    if (tid < NB) {
        const int blk = blk0 + tid;
        const int bi = blk < nblocks ? blk : 0;
        cen[tid][0] = ox + q * (bi % nbx);
        cen[tid][1] = oy + q * ((bi / nbx) % nby);
        cen[tid][2] = oz + q * (bi / (nbx * nby));
    }
    pdl_wait();   // the previous colour's writes of u
    __syncthreads();
    for (int i = tid; i < NB * PW * PW * PW; i += NT) {
        const int j = i / (PW * PW * PW), k = i - j * (PW * PW * PW);
        const int gx = cen[j][0] - R - P + k % PW, gy = cen[j][1] - R - P + (k / PW) % PW,
                  gz = cen[j][2] - R - P + k / (PW * PW);
        pu[j][k] = (blk0 + j < nblocks && gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n)
                       ? u[((size_t)gz * n + gy) * n + gx] : T(0);
    }
    __syncthreads();
    for (int i = tid; i < NB * PW * PW * S; i += NT) {   // x pass
        const int j = i / (PW * PW * S), k = i - j * (PW * PW * S);
        const int ex = k % S, r = k / S;
        const int gx = cen[j][0] - R + ex;
        T2 acc;
        acc.x = T(0);
        acc.y = T(0);
        if (gx >= 0 && gx < n) {
            const T *kr = Kb + (size_t)gx * W, *mr = Mb + (size_t)gx * W;
            const T *ur = pu[j] + r * PW + ex;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                T2 c, v;
                c.x = kr[a]; c.y = mr[a];
                v.x = ur[a]; v.y = ur[a];
                acc = fma2_3d(c, v, acc);
            }
        }
        tKM[j][k] = acc;
    }
    __syncthreads();
    for (int i = tid; i < NB * PW * S * S; i += NT) {    // y pass
        const int j = i / (PW * S * S), k = i - j * (PW * S * S);
        const int ex = k % S, ey = (k / S) % S, z = k / (S * S);
        const int gy = cen[j][1] - R + ey;
        T s1 = T(0), mm = T(0);
        if (gy >= 0 && gy < n) {
            const T *kr = Kb + (size_t)gy * W, *mr = Mb + (size_t)gy * W;
#pragma unroll
            for (int bb = 0; bb < W; ++bb) {
                const T2 t = tKM[j][(z * PW + ey + bb) * S + ex];
                s1 = fma(mr[bb], t.x, s1);
                s1 = fma(kr[bb], t.y, s1);
                mm = fma(mr[bb], t.y, mm);
            }
        }
        T2 o;
        o.x = s1;
        o.y = mm;
        sMM[j][k] = o;
    }
    __syncthreads();
    for (int i = tid; i < NB * SS; i += NT) {            // z pass and block residual
        const int j = i / SS, e = i - j * SS;
        const int ex = e % S, ey = (e / S) % S, ez = e / (S * S);
        const int gx = cen[j][0] - R + ex, gy = cen[j][1] - R + ey, gz = cen[j][2] - R + ez;
        T rv = T(0);
        if (blk0 + j < nblocks && gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n) {
            const T *kr = Kb + (size_t)gz * W, *mr = Mb + (size_t)gz * W;
            T2 acc;
            acc.x = T(0);
            acc.y = T(0);
#pragma unroll
            for (int c = 0; c < W; ++c) {
                T2 cf;
                cf.x = mr[c]; cf.y = kr[c];
                acc = fma2_3d(cf, sMM[j][((ez + c) * S + ey) * S + ex], acc);
            }
            rv = b[((size_t)gz * n + gy) * n + gx] - (acc.x + acc.y);
        }
        rs[j][e] = rv;
    }
    __syncthreads();
    for (int i = tid; i < NB * SS; i += NT) {            // block solve and update
        const int j = i / SS, e = i - j * SS;
        const int ex = e % S, ey = (e / S) % S, ez = e / (S * S);
        const int cx = cen[j][0], cy = cen[j][1], cz = cen[j][2];
        const int gx = cx - R + ex, gy = cy - R + ey, gz = cz - R + ez;
        if (blk0 + j >= nblocks || gx < 0 || gx >= n || gy < 0 || gy >= n || gz < 0 || gz >= n) continue;
        const int cls = (bcls[cz] * nbc + bcls[cy]) * nbc + bcls[cx];
        if (sizeof(T) == sizeof(double) || cls == interior || !binv64) {
            const T *Bi = binv + (size_t)cls * SS * SS + e;
            T ev = T(0);
#pragma unroll
            for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[(size_t)f * SS]), rs[j][f], ev);
            u[((size_t)gz * n + gy) * n + gx] += ev;
        } else {
            const double *Bi = binv64 + (size_t)cls * SS * SS + e;
            double ev = 0.0;
#pragma unroll
            for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[(size_t)f * SS]), (double)rs[j][f], ev);
            u[((size_t)gz * n + gy) * n + gx] += (T)ev;
        }
    }
}

// Interior rows of the 1D stiffness and mass matrices scaled to be independent of h
// (k = h K_row, m = M_row / h), as pairs (k[a], m[a]); degrees 2..4, written once per
// device and degree.
__constant__ float2 c3_km[5][9];

// One LATTICE colour in 3D for the FP32 inner cycle: one Schwarz block (S = 3) per warp,
// WPC blocks per CTA, each warp on its own without CTA barriers.  With the 1D rows scaled
// as k = h K, m = M / h (interior rows from c3_km, the others from their own band rows):
//   x pass, a lane per patch row (z', y') with the row's PW values of u in registers:
//       tK = sum_a k_x[a] u,  tM = sum_a m_x[a] u          (= h K_x u, M_x u / h)
//   y pass, a lane per (z', x) column of the x pass's output:
//       S1 = sum_b m_y[b] tK + k_y[b] tM,  MM = sum_b m_y[b] tM   (= S1, MM / h^2)
//   z pass, a lane per (y, x) column:  acc = sum_c m_z[c] S1 + k_z[c] MM  (= (A u) / h)
// then r = b - h acc, the block solve e = B^{-1} r (the interior class's inverse staged in
// shared memory once per CTA; a boundary class's FP64 rows as the FP32 pairs binv + binv_lo
// applied by compensated (Dot2) arithmetic, or its FP32 rows when binv_lo is null) and
// u += e.  The arithmetic of the sum factorisation is that of
// the residual kernels, the h factors regrouped.
template <int P>
struct Warp3dGeom {
    static constexpr int S = 3, R = 1, W = 2 * P + 1, SS = S * S * S, PW = S + 2 * P;
    static constexpr int NROW = PW * PW;   // patch rows (z', y') of the x pass
    static constexpr int WPC = 8;          // blocks (warps) per CTA
};

// resident CTAs per SM the register allocation must allow: 6 (40 registers) puts a 128^3
// colour (up to 858 CTAs) in one wave; p = 4 would spill there and keeps 5
constexpr int lattice3d_w_minb(int p) { return p == 4 ? 5 : 6; }

template <int P>
__global__ void __launch_bounds__(256, lattice3d_w_minb(P))
k_schwarz_lattice3d_w(int n, int nbc, int q, int ox, int oy, int oz, int nbx, int nby, int nblocks,
                      const float *__restrict__ Kb, const float *__restrict__ Mb, const float *__restrict__ binv,
                      const float *__restrict__ binv_lo, int interior, const int *__restrict__ bcls,
                      float *__restrict__ u, const float *__restrict__ b)
{
    using G = Warp3dGeom<P>;
    constexpr int S = G::S, R = G::R, W = G::W, SS = G::SS, PW = G::PW, NROW = G::NROW, WPC = G::WPC;
    constexpr int PCI = 2 * P - 1;   // first interior row
    __shared__ float sbi[SS * SS];             // interior inverse, transposed: [f][e]
    __shared__ float2 tkm_s[WPC][NROW * S];    // x pass: [(z' PW + y') S + x]
    __shared__ float2 smm_s[WPC][PW * S * S];  // y pass: [(z' S + y) S + x]
    __shared__ float rs_s[WPC][SS + 1];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < SS * SS; i += 32 * WPC) sbi[i] = binv[(size_t)interior * SS * SS + i];   // constant table
    const int blk = blockIdx.x * WPC + w;
    const int cx = ox + q * (blk % nbx), cy = oy + q * ((blk / nbx) % nby), cz = oz + q * (blk / (nbx * nby));
    const float h = 1.0f / (float)(n - P + 2), hinv = (float)(n - P + 2);
    // are the block's rows along each axis all of the interior class?  is its patch inside?
    const bool xint = cx - R >= PCI && cx + R <= n - 2 * P, yint = cy - R >= PCI && cy + R <= n - 2 * P,
               zint = cz - R >= PCI && cz + R <= n - 2 * P;
    const bool inside = cx - R - P >= 0 && cx + R + P < n && cy - R - P >= 0 && cy + R + P < n &&
                        cz - R - P >= 0 && cz + R + P < n;
    pdl_wait();   // the previous colour's writes of u (and the outer cycle's of b)
    __syncthreads();
    if (blk >= nblocks) return;   // whole warps: no CTA barrier follows
    float2 *tkm = tkm_s[w], *smm = smm_s[w];
    float *rs = rs_s[w];
    // the z pass's values of b, loaded now so that their latency overlaps the x pass
    float bz[S];
    {
        const int ey = lane / S, ex = lane - ey * S;
        const int gx = cx - R + ex, gy = cy - R + ey;
#pragma unroll
        for (int ez = 0; ez < S; ++ez) {
            const int gz = cz - R + ez;
            bz[ez] = (lane < S * S && gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n)
                         ? b[((size_t)gz * n + gy) * n + gx] : 0.0f;
        }
    }
    // x pass (a compile-time number of rounds, so that a round's loads may be issued early)
    constexpr int NR = (NROW + 31) / 32;
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
        const int row = lane + 32 * rr;
        if (row >= NROW) break;
        const int zp = row / PW, yp = row - zp * PW;
        const int gy = cy - R - P + yp, gz = cz - R - P + zp, gx0 = cx - R - P;
        float v[PW];
        if (inside) {
            const float *src = u + ((size_t)gz * n + gy) * n + gx0;
#pragma unroll
            for (int k = 0; k < PW; ++k) v[k] = src[k];
        } else {
            const bool rin = gy >= 0 && gy < n && gz >= 0 && gz < n;
#pragma unroll
            for (int k = 0; k < PW; ++k) {
                const int gx = gx0 + k;
                v[k] = (rin && gx >= 0 && gx < n) ? u[((size_t)gz * n + gy) * n + gx] : 0.0f;
            }
        }
#pragma unroll
        for (int ex = 0; ex < S; ++ex) {
            float2 o = make_float2(0.0f, 0.0f);
            if (xint) {
#pragma unroll
                for (int a = 0; a < W; ++a) o = fma2_3d(c3_km[P][a], make_float2(v[ex + a], v[ex + a]), o);
            } else {
                const int gx = cx - R + ex;
                if (gx >= 0 && gx < n) {
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        const float2 km = make_float2(Kb[(size_t)gx * W + a] * h, Mb[(size_t)gx * W + a] * hinv);
                        o = fma2_3d(km, make_float2(v[ex + a], v[ex + a]), o);
                    }
                }
            }
            tkm[row * S + ex] = o;
        }
    }
    __syncwarp();
    // y pass
    for (int it = lane; it < PW * S; it += 32) {
        const int zp = it / S, ex = it - zp * S;
        float2 t[PW];
#pragma unroll
        for (int yp = 0; yp < PW; ++yp) t[yp] = tkm[(zp * PW + yp) * S + ex];
#pragma unroll
        for (int ey = 0; ey < S; ++ey) {
            const int gy = cy - R + ey;
            float2 acc = make_float2(0.0f, 0.0f);   // (sum m tK, sum m tM)
            float ak = 0.0f;                         // sum k tM
            if (yint) {
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    const float2 c = c3_km[P][bb];
                    acc = fma2_3d(make_float2(c.y, c.y), t[ey + bb], acc);
                    ak = fmaf(c.x, t[ey + bb].y, ak);
                }
            } else if (gy >= 0 && gy < n) {
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    const float k = Kb[(size_t)gy * W + bb] * h, m = Mb[(size_t)gy * W + bb] * hinv;
                    acc = fma2_3d(make_float2(m, m), t[ey + bb], acc);
                    ak = fmaf(k, t[ey + bb].y, ak);
                }
            }
            smm[(zp * S + ey) * S + ex] = make_float2(acc.x + ak, acc.y);
        }
    }
    __syncwarp();
    // z pass and the block residual
    if (lane < S * S) {
        const int ey = lane / S, ex = lane - ey * S;
        const int gx = cx - R + ex, gy = cy - R + ey;
        float2 t[PW];
#pragma unroll
        for (int zp = 0; zp < PW; ++zp) t[zp] = smm[(zp * S + ey) * S + ex];
#pragma unroll
        for (int ez = 0; ez < S; ++ez) {
            const int gz = cz - R + ez;
            float rv = 0.0f;
            if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n) {
                float2 acc = make_float2(0.0f, 0.0f);   // (sum m S1, sum k MM)
                if (zint) {
#pragma unroll
                    for (int c = 0; c < W; ++c) {
                        const float2 km = c3_km[P][c];
                        acc = fma2_3d(make_float2(km.y, km.x), t[ez + c], acc);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < W; ++c) {
                        const float2 mk = make_float2(Mb[(size_t)gz * W + c] * hinv, Kb[(size_t)gz * W + c] * h);
                        acc = fma2_3d(mk, t[ez + c], acc);
                    }
                }
                rv = bz[ez] - h * (acc.x + acc.y);
            }
            rs[(ez * S + ey) * S + ex] = rv;
        }
    }
    __syncwarp();
    // block solve and update
    if (lane < SS) {
        const int e = lane, ex = e % S, ey = (e / S) % S, ez = e / (S * S);
        const int gx = cx - R + ex, gy = cy - R + ey, gz = cz - R + ez;
        if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n) {
            const int cls = (bcls[cz] * nbc + bcls[cy]) * nbc + bcls[cx];
            const size_t k = ((size_t)gz * n + gy) * n + gx;
            if (cls == interior) {
                float e0 = 0.0f, e1 = 0.0f;
#pragma unroll
                for (int f = 0; f < SS; ++f) {
                    float &acc = (f & 1) ? e1 : e0;
                    acc = fmaf(sbi[f * SS + e], rs[f], acc);
                }
                u[k] += e0 + e1;
            } else if (!binv_lo) {
                const float *Bi = binv + (size_t)cls * SS * SS + e;
                float ev = 0.0f;
#pragma unroll
                for (int f = 0; f < SS; ++f) ev = fmaf(__ldg(&Bi[(size_t)f * SS]), rs[f], ev);
                u[k] += ev;
            } else {
                const size_t col = (size_t)cls * SS * SS + e;
                u[k] += dot2_row<SS, SS>(binv + col, binv_lo + col, rs);
            }
        }
    }
}

// One tile phase of the TILE(TT) schedule in 3D: tiles (tx, ty, tz) of the phase's
// parities, each CTA running all q^3 lattice colours of its tile (anchored at the tile
// origin) with u (tile + halo R + P) and b (tile + halo R) in shared memory.  TT is the
// default colour period, so a colour has one block per tile (in general: every block of
// the colour in the tile, one after another).  Per block: the x pass (pairs K_x u, M_x u
// over the (z, y) patch rows), the y pass (S1 = M_y tK + K_y tM, MM = M_y tM), the z pass
// with the block residual, and the block solve, separated by CTA barriers; the 1D rows of
// the tile's output coordinates are staged per axis.  Tiles of one phase are 2 TT apart
// with TT >= 2R + P: none reads what another writes.
template <int P, int TT, typename T>
struct Tile3dGeom {
    static constexpr int S = 3, R = 1, W = 2 * P + 1, SS = S * S * S, H = R + P, PW = S + 2 * P;
    static constexpr int SW = TT + 2 * H, BW = TT + 2 * R;
    static constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }
    // dynamic shared memory layout (bytes)
    static constexpr size_t o_su = 0;
    static constexpr size_t o_sb = align16(o_su + sizeof(T) * SW * SW * SW);
    static constexpr size_t o_tkm = align16(o_sb + sizeof(T) * BW * BW * BW);
    static constexpr size_t o_smm = align16(o_tkm + 2 * sizeof(T) * PW * PW * S);
    static constexpr size_t o_rs = align16(o_smm + 2 * sizeof(T) * PW * S * S);
    static constexpr size_t o_tab = align16(o_rs + sizeof(T) * SS);
    static constexpr size_t o_bi = align16(o_tab + 2 * sizeof(T) * 3 * BW * W);
    static constexpr size_t bytes = align16(o_bi + sizeof(T) * SS * SS);
};

template <int P, int TT, typename T>
__global__ void __launch_bounds__(128)
k_schwarz_tile3d(int n, int nbc, int q, int g, int rev, int px, int py, int pz, int ntpx, int ntpy,
                 const T *__restrict__ Kb, const T *__restrict__ Mb, const T *__restrict__ binv,
                 const double *__restrict__ binv64, int interior, const int *__restrict__ bcls,
                 T *__restrict__ u, const T *__restrict__ b)
{
    using G = Tile3dGeom<P, TT, T>;
    using T2 = typename Vec2_3d<T>::type;
    constexpr int S = G::S, R = G::R, W = G::W, SS = G::SS, H = G::H, PW = G::PW, SW = G::SW, BW = G::BW;
    constexpr int NT = 128;
    extern __shared__ __align__(16) unsigned char smem_t3[];
    T *su = reinterpret_cast<T *>(smem_t3 + G::o_su);
    T *sb = reinterpret_cast<T *>(smem_t3 + G::o_sb);
    T2 *tKM = reinterpret_cast<T2 *>(smem_t3 + G::o_tkm);
    T2 *sMM = reinterpret_cast<T2 *>(smem_t3 + G::o_smm);
    T *rs = reinterpret_cast<T *>(smem_t3 + G::o_rs);
    T *ktab = reinterpret_cast<T *>(smem_t3 + G::o_tab);     // [axis][BW][W]
    T *mtab = ktab + 3 * BW * W;
    T *sbi = reinterpret_cast<T *>(smem_t3 + G::o_bi);
    const int tid = threadIdx.x;
    const int bx = blockIdx.x;
    const int x0 = (px + 2 * (bx % ntpx)) * TT, y0 = (py + 2 * ((bx / ntpx) % ntpy)) * TT,
              z0 = (pz + 2 * (bx / (ntpx * ntpy))) * TT;
    const int org[3] = {x0, y0, z0};
    const int tw = min(TT, n - x0), th = min(TT, n - y0), td = min(TT, n - z0);
    pdl_wait();   // the previous phase's writes of u
    for (int i = tid; i < SW * SW * SW; i += NT) {
        const int gx = x0 - H + i % SW, gy = y0 - H + (i / SW) % SW, gz = z0 - H + i / (SW * SW);
        su[i] = (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n) ? u[((size_t)gz * n + gy) * n + gx]
                                                                               : T(0);
    }
    for (int i = tid; i < BW * BW * BW; i += NT) {
        const int gx = x0 - R + i % BW, gy = y0 - R + (i / BW) % BW, gz = z0 - R + i / (BW * BW);
        sb[i] = (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n) ? b[((size_t)gz * n + gy) * n + gx]
                                                                               : T(0);
    }
    for (int i = tid; i < 3 * BW * W; i += NT) {
        const int ax = i / (BW * W), r = (i / W) % BW, a = i % W;
        const int gc = org[ax] - R + r;
        ktab[i] = (gc >= 0 && gc < n) ? Kb[(size_t)gc * W + a] : T(0);
        mtab[i] = (gc >= 0 && gc < n) ? Mb[(size_t)gc * W + a] : T(0);
    }
    for (int i = tid; i < SS * SS; i += NT) sbi[i] = binv[(size_t)interior * SS * SS + i];
    __syncthreads();
    const int ncol = q * q * q;
    for (int t = 0; t < ncol; ++t) {
        const int c = rev ? ncol - 1 - t : t;
        const int ox = ((c % q) * g) % q, oy = (((c / q) % q) * g) % q, oz = ((c / (q * q)) * g) % q;
        for (int cz = oz; cz < td; cz += q)
            for (int cy = oy; cy < th; cy += q)
                for (int cx = ox; cx < tw; cx += q) {
                    // x pass over the (z, y) patch rows: su rows start at tile-local cx - R - P
                    for (int i = tid; i < PW * PW * S; i += NT) {
                        const int ex = i % S, rr = i / S, yy = rr % PW, zz = rr / PW;
                        const T *ur = su + ((cz + zz) * SW + (cy + yy)) * SW + cx + ex;
                        const T *kr = ktab + (0 * BW + cx + ex) * W, *mr = mtab + (0 * BW + cx + ex) * W;
                        T2 acc;
                        acc.x = T(0);
                        acc.y = T(0);
#pragma unroll
                        for (int a = 0; a < W; ++a) {
                            T2 cf, v;
                            cf.x = kr[a]; cf.y = mr[a];
                            v.x = ur[a]; v.y = ur[a];
                            acc = fma2_3d(cf, v, acc);
                        }
                        tKM[i] = acc;
                    }
                    __syncthreads();
                    for (int i = tid; i < PW * S * S; i += NT) {   // y pass
                        const int ex = i % S, ey = (i / S) % S, z = i / (S * S);
                        const T *kr = ktab + (1 * BW + cy + ey) * W, *mr = mtab + (1 * BW + cy + ey) * W;
                        T s1 = T(0), mm = T(0);
#pragma unroll
                        for (int bb = 0; bb < W; ++bb) {
                            const T2 tv = tKM[(z * PW + ey + bb) * S + ex];
                            s1 = fma(mr[bb], tv.x, s1);
                            s1 = fma(kr[bb], tv.y, s1);
                            mm = fma(mr[bb], tv.y, mm);
                        }
                        T2 o;
                        o.x = s1;
                        o.y = mm;
                        sMM[i] = o;
                    }
                    __syncthreads();
                    if (tid < SS) {                                  // z pass and block residual
                        const int ex = tid % S, ey = (tid / S) % S, ez = tid / (S * S);
                        const int gx = x0 + cx - R + ex, gy = y0 + cy - R + ey, gz = z0 + cz - R + ez;
                        T rv = T(0);
                        if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n) {
                            const T *kr = ktab + (2 * BW + cz + ez) * W, *mr = mtab + (2 * BW + cz + ez) * W;
                            T2 acc;
                            acc.x = T(0);
                            acc.y = T(0);
#pragma unroll
                            for (int cc = 0; cc < W; ++cc) {
                                T2 cf;
                                cf.x = mr[cc]; cf.y = kr[cc];
                                acc = fma2_3d(cf, sMM[((ez + cc) * S + ey) * S + ex], acc);
                            }
                            rv = sb[((cz + ez) * BW + cy + ey) * BW + cx + ex] - (acc.x + acc.y);
                        }
                        rs[tid] = rv;
                    }
                    __syncthreads();
                    if (tid < SS) {                                  // block solve and update
                        const int ex = tid % S, ey = (tid / S) % S, ez = tid / (S * S);
                        const int gcx = x0 + cx, gcy = y0 + cy, gcz = z0 + cz;
                        const int gx = gcx - R + ex, gy = gcy - R + ey, gz = gcz - R + ez;
                        if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n) {
                            const int cls = (bcls[gcz] * nbc + bcls[gcy]) * nbc + bcls[gcx];
                            T ev = T(0);
                            if (cls == interior) {
                                const T *Bi = sbi + tid;
#pragma unroll
                                for (int f = 0; f < SS; ++f) ev = fma(Bi[f * SS], rs[f], ev);
                            } else if (sizeof(T) == sizeof(double) || !binv64) {
                                const T *Bi = binv + (size_t)cls * SS * SS + tid;
#pragma unroll
                                for (int f = 0; f < SS; ++f) ev = fma(__ldg(&Bi[(size_t)f * SS]), rs[f], ev);
                            } else {
                                const double *Bi = binv64 + (size_t)cls * SS * SS + tid;
                                double ed = 0.0;
#pragma unroll
                                for (int f = 0; f < SS; ++f) ed = fma(__ldg(&Bi[(size_t)f * SS]), (double)rs[f], ed);
                                ev = (T)ed;
                            }
                            su[((cz + P + ez) * SW + cy + P + ey) * SW + cx + P + ex] += ev;
                        }
                    }
                    __syncthreads();
                }
    }
    for (int i = tid; i < BW * BW * BW; i += NT) {
        const int lx = i % BW, ly = (i / BW) % BW, lz = i / (BW * BW);
        const int gx = x0 - R + lx, gy = y0 - R + ly, gz = z0 - R + lz;
        if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n)
            u[((size_t)gz * n + gy) * n + gx] = su[((lz + P) * SW + ly + P) * SW + lx + P];
    }
}

// out[z][y][x'] = sum_w B[x'][w] in[z][y][lo[x'] + w] along axis `ax` (0 = x, 1 = y, 2 = z):
// in has dims (nx, ny, nz), out the same with the axis length replaced by nout.  With
// accumulate = 1 the result is added to out (TU) after adding delta (if not null).
template <typename T, typename TU>
__global__ void k_band_axis(int ax, int nx, int ny, int nz, int nout, int nin_axis, int wb,
                            const T *__restrict__ B, const int *__restrict__ lo, const T *__restrict__ in,
                            TU *__restrict__ out, const T *__restrict__ delta, int accumulate)
{
    const long long total = (ax == 0 ? (long long)nout * ny * nz : ax == 1 ? (long long)nx * nout * nz
                                                                            : (long long)nx * ny * nout);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int ox_ = ax == 0 ? nout : nx, oy_ = ax == 1 ? nout : ny;
    const int x = (int)(i % ox_), y = (int)((i / ox_) % oy_), z = (int)(i / ((long long)ox_ * oy_));
    const int o = ax == 0 ? x : ax == 1 ? y : z;    // output index along the axis
    const long long stride = ax == 0 ? 1 : ax == 1 ? nx : (long long)nx * ny;
    const long long base = (long long)(ax == 0 ? 0 : x) + (long long)(ax == 1 ? 0 : y) * nx +
                           (long long)(ax == 2 ? 0 : z) * nx * ny;
    const int l0 = lo[o];
    T acc = T(0);
    for (int w = 0; w < wb; ++w) {
        const int j = l0 + w;
        if (j >= 0 && j < nin_axis) acc = fma(B[(size_t)o * wb + w], in[base + j * stride], acc);
    }
    if (accumulate) {
        if (delta) out[i] += (TU)delta[i] + (TU)acc;
        else out[i] += (TU)acc;
    } else {
        out[i] = (TU)acc;
    }
}

// ---- degree-1 hierarchy in 3D -----------------------------------------------------
template <typename T>
struct Stencil27 {
    T c[27];   // c[(dz*3 + dy)*3 + dx]
};

template <typename T>
Stencil27<T> level_stencil27(const Level &L)
{
    Stencil27<T> s;
    for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy)
            for (int dx = 0; dx < 3; ++dx)
                s.c[(dz * 3 + dy) * 3 + dx] = (T)(L.k[dx] * L.mm[dy] * L.mm[dz] + L.mm[dx] * L.k[dy] * L.mm[dz] +
                                                  L.mm[dx] * L.mm[dy] * L.k[dz]);
    return s;
}

template <typename T>
__device__ __forceinline__ T apply27(int n, const Stencil27<T> &st, const T *e, int x, int y, int z)
{
    T acc = T(0);
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
        const int zz = z + dz - 1;
        if (zz < 0 || zz >= n) continue;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const int yy = y + dy - 1;
            if (yy < 0 || yy >= n) continue;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int xx = x + dx - 1;
                if (xx >= 0 && xx < n) acc = fma(st.c[(dz * 3 + dy) * 3 + dx], e[((size_t)zz * n + yy) * n + xx], acc);
            }
        }
    }
    return acc;
}

// relax the parity sub-lattice (px, py, pz); first = the first pass from e = 0
template <typename T>
__global__ void k_gs3d(int n, int px, int py, int pz, int first, Stencil27<T> st, const T *__restrict__ rhs,
                       T *__restrict__ e)
{
    const int half = (n + 1) / 2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (first) {
        if (i >= (long long)n * n * n) return;
        const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long long)n * n));
        e[i] = ((x | y | z) & 1) ? T(0) : (rhs[i] - T(0)) / st.c[13];
        return;
    }
    if (i >= (long long)half * half * half) return;
    const int x = 2 * (int)(i % half) + px, y = 2 * (int)((i / half) % half) + py,
              z = 2 * (int)(i / ((long long)half * half)) + pz;
    if (x >= n || y >= n || z >= n) return;
    const size_t gi = ((size_t)z * n + y) * n + x;
    e[gi] += (rhs[gi] - apply27<T>(n, st, e, x, y, z)) / st.c[13];
}

template <typename T>
__global__ void k_level_residual3d(int n, Stencil27<T> st, const T *__restrict__ rhs, const T *__restrict__ e,
                                   T *__restrict__ r)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * n * n) return;
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long long)n * n));
    r[i] = rhs[i] - apply27<T>(n, st, e, x, y, z);
}

// rc[K][J][I] = sum w_dz w_dy w_dx r[2K+dz][2J+dy][2I+dx], w = (1/2, 1, 1/2)
template <typename T>
__global__ void k_level_restrict3d(int nf, int nc, const T *__restrict__ r, T *__restrict__ rc)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nc * nc * nc) return;
    const int I = (int)(i % nc), J = (int)((i / nc) % nc), K = (int)(i / ((long long)nc * nc));
    const T w[3] = {T(0.5), T(1), T(0.5)};
    T acc = T(0);
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
        T sy = T(0);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const T *row = r + ((size_t)(2 * K + dz) * nf + (2 * J + dy)) * nf + 2 * I;
            T sx = T(0);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) sx = fma(w[dx], row[dx], sx);
            sy = fma(w[dy], sx, sy);
        }
        acc = fma(w[dz], sy, acc);
    }
    rc[i] = acc;
}

template <typename T>
__global__ void k_level_prolong3d(int nf, int nc, const T *__restrict__ ec, T *__restrict__ e)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nf * nf * nf) return;
    const int c3[3] = {(int)(i % nf), (int)((i / nf) % nf), (int)(i / ((long long)nf * nf))};
    // per axis two coarse slots: odd x -> ((x-1)/2, weight 1), even x -> (x/2-1, x/2,
    // weights 1/2); an unused or out-of-range slot has weight 0 and is skipped
    int I[3][2];
    T w[3][2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int x = c3[k];
        const bool odd = x & 1;
        I[k][0] = odd ? (x - 1) / 2 : x / 2 - 1;
        I[k][1] = x / 2;
        w[k][0] = odd ? T(1) : T(0.5);
        w[k][1] = odd ? T(0) : T(0.5);
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (I[k][c] < 0 || I[k][c] >= nc) w[k][c] = T(0);
    }
    T acc = T(0);
#pragma unroll
    for (int cz = 0; cz < 2; ++cz) {
        if (w[2][cz] == T(0)) continue;
        T sy = T(0);
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            if (w[1][cy] == T(0)) continue;
            T sx = T(0);
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                if (w[0][cx] == T(0)) continue;
                sx = fma(w[0][cx], ec[((size_t)I[2][cz] * nc + I[1][cy]) * nc + I[0][cx]], sx);
            }
            sy = fma(w[1][cy], sx, sy);
        }
        acc = fma(w[2][cz], sy, acc);
    }
    e[i] += acc;
}

template <typename T>
__global__ void k_dense_matvec3(int N, const double *__restrict__ Ainv, const T *__restrict__ rhs, T *__restrict__ x)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= N) return;
    const double *row = Ainv + (size_t)warp * N;
    double s = 0.0;
    for (int j = lane; j < N; j += 32) s = fma(row[j], (double)rhs[j], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) x[warp] = (T)s;
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

// red-black order in 3D: red (0,0,0),(1,1,0),(1,0,1),(0,1,1), black (1,0,0),(0,1,0),(0,0,1),(1,1,1)
constexpr int kGs3Seq[8][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
                               {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 1}};

template <typename T>
cudaError_t vcycle3d(const Solver &S, int l, const T *rhs, T *e, T *const *levE, T *const *levR, T *const *levT,
                     cudaStream_t s)
{
    const Level &L = S.lev[l];
    const int last = (int)S.lev.size() - 1;
    if (l == last) {
        const int N = S.ndirect;
        k_dense_matvec3<T><<<(N * 32 + 255) / 256, 256, 0, s>>>(N, S.dinv, rhs, e);
        count_launches(1);
        return cudaGetLastError();
    }
    const Level &C = S.lev[l + 1];
    const Stencil27<T> st = level_stencil27<T>(L);
    const int n = L.n, half = (n + 1) / 2;
    for (int t = 0; t < 8; ++t) {
        if (t == 0)
            k_gs3d<T><<<blocks_for((long long)n * n * n, 256), 256, 0, s>>>(n, 0, 0, 0, 1, st, rhs, e);
        else
            k_gs3d<T><<<blocks_for((long long)half * half * half, 256), 256, 0, s>>>(n, kGs3Seq[t][0], kGs3Seq[t][1],
                                                                                  kGs3Seq[t][2], 0, st, rhs, e);
        count_launches(1);
    }
    k_level_residual3d<T><<<blocks_for((long long)n * n * n, 256), 256, 0, s>>>(n, st, rhs, e, levT[l]);
    count_launches(1);
    k_level_restrict3d<T><<<blocks_for((long long)C.n * C.n * C.n, 256), 256, 0, s>>>(n, C.n, levT[l], levR[l + 1]);
    count_launches(1);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if ((err = vcycle3d<T>(S, l + 1, levR[l + 1], levE[l + 1], levE, levR, levT, s)) != cudaSuccess) return err;
    k_level_prolong3d<T><<<blocks_for((long long)n * n * n, 256), 256, 0, s>>>(n, C.n, levE[l + 1], e);
    count_launches(1);
    for (int t = 7; t >= 0; --t) {
        k_gs3d<T><<<blocks_for((long long)half * half * half, 256), 256, 0, s>>>(n, kGs3Seq[t][0], kGs3Seq[t][1],
                                                                              kGs3Seq[t][2], 0, st, rhs, e);
        count_launches(1);
    }
    return cudaGetLastError();
}

template <int P, typename T, typename TO>
cudaError_t residual3d_p(const Solver &S, const T *Kb, const T *Mb, const T *u, const T *b, TO *d, double *part,
                         cudaStream_t st)
{
    const size_t smem = sizeof(T) * res3d_smem_elems<P>();
    static bool attr_set = false;   // per instantiation; idempotent
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_residual3d<P, T, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grd((S.n + kR3X - 1) / kR3X, (S.n + kR3Y - 1) / kR3Y, (S.n + kR3Z - 1) / kR3Z);
    k_residual3d<P, T, TO><<<grd, 256, smem, st>>>(S.n, Kb, Mb, u, b, d, part);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, typename TO>
cudaError_t residual3d_any(const Solver &S, const T *Kb, const T *Mb, const T *u, const T *b, TO *d, double *part,
                           cudaStream_t st)
{
    switch (S.p) {
    case 2: return residual3d_p<2, T, TO>(S, Kb, Mb, u, b, d, part, st);
    case 3: return residual3d_p<3, T, TO>(S, Kb, Mb, u, b, d, part, st);
    case 4: return residual3d_p<4, T, TO>(S, Kb, Mb, u, b, d, part, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int P, typename T>
cudaError_t schwarz_tile3d_p(const Solver &S, const T *Kb, const T *Mb, const T *binv, T *u, const T *b,
                             bool reverse, cudaStream_t st)
{
    constexpr int TT = tile_side3d(P);
    using G = Tile3dGeom<P, TT, T>;
    const int nbc = S.ht.nbc;
    const int interior = (S.ht.L * nbc + S.ht.L) * nbc + S.ht.L;
    static bool attr_set[64] = {};   // per device: the dynamic shared memory limit of this instantiation
    if (S.device >= 0 && S.device < 64 && !attr_set[S.device]) {
        cudaError_t e = cudaFuncSetAttribute(k_schwarz_tile3d<P, TT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::bytes);
        if (e != cudaSuccess) return e;
        attr_set[S.device] = true;
    }
    const int nt = (S.n + TT - 1) / TT;
    for (int t = 0; t < 8; ++t) {
        const int ph = reverse ? 7 - t : t;
        const int px = ph & 1, py = (ph >> 1) & 1, pz = ph >> 2;
        const int ntpx = (nt - px + 1) / 2, ntpy = (nt - py + 1) / 2, ntpz = (nt - pz + 1) / 2;
        if (ntpx <= 0 || ntpy <= 0 || ntpz <= 0) continue;
        cudaError_t err = launch_pdl_smem(k_schwarz_tile3d<P, TT, T>, dim3(ntpx * ntpy * ntpz), dim3(128), G::bytes,
                                          st, S.n, nbc, S.q, S.g, reverse ? 1 : 0, px, py, pz, ntpx, ntpy, Kb, Mb,
                                          binv, S.boundary64_t(), interior, (const int *)S.bcls, u, b);
        count_launches(1);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

template <int P, typename T>
cudaError_t schwarz3d_p(const Solver &S, const T *Kb, const T *Mb, const T *binv, T *u, const T *b, bool reverse,
                        cudaStream_t st)
{
    if (S.opt.schedule == IGA2L_SCHED_TILE) return schwarz_tile3d_p<P, T>(S, Kb, Mb, binv, u, b, reverse, st);
    const int q = S.q, ncol = q * q * q, nbc = S.ht.nbc;
    const int interior = (S.ht.L * nbc + S.ht.L) * nbc + S.ht.L;
    for (int t = 0; t < ncol; ++t) {
        const int c = reverse ? ncol - 1 - t : t;
        const int ox = ((c % q) * S.g) % q, oy = (((c / q) % q) * S.g) % q, oz = ((c / (q * q)) * S.g) % q;
        const int nbx = (S.n - ox + q - 1) / q, nby = (S.n - oy + q - 1) / q, nbz = (S.n - oz + q - 1) / q;
        if (nbx <= 0 || nby <= 0 || nbz <= 0) continue;
        // FP64: several blocks per CTA, every pass over all threads (bound by the FP64 pipe;
        // 175 against 180 ms for the 128^3 p=3 solve with one block per CTA); FP32: one block
        // per warp (the one-block-per-CTA form spent ~3.3k warp instructions per block, ncu)
        const int nblocks = nbx * nby * nbz;
        cudaError_t err;
        if constexpr (sizeof(T) == sizeof(double)) {
            constexpr int NB = Lattice3dGeom<P, T>::NB;
            err = launch_pdl(k_schwarz_lattice3d_mb<P, T>, dim3((nblocks + NB - 1) / NB), dim3(256), st, S.n, nbc, q,
                             ox, oy, oz, nbx, nby, nblocks, Kb, Mb, binv, S.boundary64_t(), interior,
                             (const int *)S.bcls, u, b);
        } else {
            constexpr int WPC = Warp3dGeom<P>::WPC;
            err = launch_pdl(k_schwarz_lattice3d_w<P>, dim3((nblocks + WPC - 1) / WPC), dim3(32 * WPC), st, S.n, nbc,
                             q, ox, oy, oz, nbx, nby, nblocks, Kb, Mb, binv, S.boundary_lo_t(), interior,
                             (const int *)S.bcls, u, b);
        }
        count_launches(1);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t schwarz3d_any(const Solver &S, const T *Kb, const T *Mb, const T *binv, T *u, const T *b, bool reverse,
                          cudaStream_t st)
{
    if (S.s != 3) return cudaErrorInvalidValue;
    switch (S.p) {
    case 2: return schwarz3d_p<2, T>(S, Kb, Mb, binv, u, b, reverse, st);
    case 3: return schwarz3d_p<3, T>(S, Kb, Mb, binv, u, b, reverse, st);
    case 4: return schwarz3d_p<4, T>(S, Kb, Mb, binv, u, b, reverse, st);
    default: return cudaErrorInvalidValue;
    }
}

// d (n^3) -> dc (nc^3) by the restriction band along x, y, z; tA, tB hold the passes
template <typename T>
cudaError_t restrict3d(const Solver &S, const T *Rb, const T *d, T *tA, T *tB, T *dc, cudaStream_t st)
{
    const int n = S.n, nc = S.nc, w = S.ht.wr;
    long long c1 = (long long)nc * n * n, c2 = (long long)nc * nc * n, c3 = (long long)nc * nc * nc;
    k_band_axis<T, T><<<blocks_for(c1, 256), 256, 0, st>>>(0, n, n, n, nc, n, w, Rb, S.Rlo, d, tA, nullptr, 0);
    k_band_axis<T, T><<<blocks_for(c2, 256), 256, 0, st>>>(1, nc, n, n, nc, n, w, Rb, S.Rlo, tA, tB, nullptr, 0);
    k_band_axis<T, T><<<blocks_for(c3, 256), 256, 0, st>>>(2, nc, nc, n, nc, n, w, Rb, S.Rlo, tB, dc, nullptr, 0);
    count_launches(3);
    return cudaGetLastError();
}

// u (+= delta) += R^T ec along x, y, z (column band of R)
template <typename T, typename TU>
cudaError_t prolong3d(const Solver &S, const T *Cb, const T *ec, T *tA, T *tB, const T *delta, TU *u,
                      cudaStream_t st)
{
    const int n = S.n, nc = S.nc, w = S.ht.wc;
    long long c1 = (long long)n * nc * nc, c2 = (long long)n * n * nc, c3 = (long long)n * n * n;
    k_band_axis<T, T><<<blocks_for(c1, 256), 256, 0, st>>>(0, nc, nc, nc, n, nc, w, Cb, S.Clo, ec, tB, nullptr, 0);
    k_band_axis<T, T><<<blocks_for(c2, 256), 256, 0, st>>>(1, n, nc, nc, n, nc, w, Cb, S.Clo, tB, tA, nullptr, 0);
    k_band_axis<T, TU><<<blocks_for(c3, 256), 256, 0, st>>>(2, n, n, nc, n, nc, w, Cb, S.Clo, tA, u, delta, 1);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace

// ---- entry points used by the dimension-generic launchers ------------------------------

int residual3d_partials(const Solver &S)
{
    return ((S.n + kR3X - 1) / kR3X) * ((S.n + kR3Y - 1) / kR3Y) * ((S.n + kR3Z - 1) / kR3Z);
}

cudaError_t launch3d_residual(const Solver &S, const double *u, const double *b, double *d, double *part,
                              cudaStream_t st)
{
    return residual3d_any<double, double>(S, S.Kb, S.Mb, u, b, d, part, st);
}

cudaError_t launch3d_schwarz(const Solver &S, double *u, const double *b, bool reverse, cudaStream_t st)
{
    return schwarz3d_any<double>(S, S.Kb, S.Mb, S.binv_t, u, b, reverse, st);
}

cudaError_t launch3d_restrict(const Solver &S, const double *d, double *dc, cudaStream_t st)
{
    return restrict3d<double>(S, S.Rb, d, S.t, S.t2, dc, st);
}

cudaError_t launch3d_prolong_add(const Solver &S, const double *ec, double *u, cudaStream_t st)
{
    return prolong3d<double, double>(S, S.Cb, ec, S.t, S.t2, nullptr, u, st);
}

cudaError_t launch3d_coarse_solve(const Solver &S, const double *dc, double *ec, cudaStream_t st)
{
    std::vector<double *> E(S.lev.size()), Rr(S.lev.size()), Tt(S.lev.size());
    for (size_t l = 0; l < S.lev.size(); ++l) { E[l] = S.lev[l].e; Rr[l] = S.lev[l].rhs; Tt[l] = S.lev[l].r; }
    return vcycle3d<double>(S, 0, dc, ec, E.data(), Rr.data(), Tt.data(), st);
}

cudaError_t launch3d_mass(const Solver &S, const double *f, double *b, cudaStream_t st)
{
    // b = (M (x) M (x) M) f, the band of M as a row band with lo(i) = i - p
    const int n = S.n, W = 2 * S.p + 1;
    long long c = (long long)n * n * n;
    k_band_axis<double, double><<<blocks_for(c, 256), 256, 0, st>>>(0, n, n, n, n, n, W, S.Mb, S.Mlo, f, S.d, nullptr, 0);
    k_band_axis<double, double><<<blocks_for(c, 256), 256, 0, st>>>(1, n, n, n, n, n, W, S.Mb, S.Mlo, S.d, S.bwork, nullptr, 0);
    k_band_axis<double, double><<<blocks_for(c, 256), 256, 0, st>>>(2, n, n, n, n, n, W, S.Mb, S.Mlo, S.bwork, b, nullptr, 0);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch3d_outer_residual(const Solver &S, const double *u, const double *b, float *r32, double *part,
                                    cudaStream_t st)
{
    return residual3d_any<double, float>(S, S.Kb, S.Mb, u, b, r32, part, st);
}

cudaError_t launch3d_inner_fine(const Solver &S, const float *r32, cudaStream_t st)
{
    const MixedState &X = S.mx;
    cudaError_t e = cudaMemsetAsync(X.delta, 0, sizeof(float) * S.N, st);
    if (e == cudaSuccess) e = schwarz3d_any<float>(S, X.Kb, X.Mb, X.binv_t, X.delta, r32, false, st);
    if (e == cudaSuccess) e = residual3d_any<float, float>(S, X.Kb, X.Mb, X.delta, r32, X.d, nullptr, st);
    if (e == cudaSuccess) e = restrict3d<float>(S, X.Rb, X.d, X.t, X.t2, X.dc, st);
    return e;
}

cudaError_t launch3d_inner_coarse(const Solver &S, cudaStream_t st)
{
    const MixedState &X = S.mx;
    return vcycle3d<float>(S, 0, X.dc, X.ec, X.lev_e.data(), X.lev_rhs.data(), X.lev_r.data(), st);
}

cudaError_t launch3d_inner_update(const Solver &S, double *u, cudaStream_t st)
{
    const MixedState &X = S.mx;
    return prolong3d<float, double>(S, X.Cb, X.ec, X.t, X.t2, X.delta, u, st);
}

cudaError_t upload_rows3d(int p, const double *k1, const double *m1)
{
    static std::mutex mu;
    static bool done[64][5] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || p < 2 || p > 4) return cudaErrorInvalidValue;
    if (done[dev][p]) return cudaSuccess;
    float2 km[9] = {};
    for (int i = 0; i < 2 * p + 1; ++i) km[i] = make_float2((float)k1[i], (float)m1[i]);
    e = cudaMemcpyToSymbol(c3_km, km, sizeof(km), sizeof(km) * p);
    if (e == cudaSuccess) done[dev][p] = true;
    return e;
}

}  // namespace iga2l
