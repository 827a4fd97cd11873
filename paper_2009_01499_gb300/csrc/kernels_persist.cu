// kernels_persist.cu -- one multiplicative Schwarz step (Section 3.1.1) in the LATTICE
// colour order as a single persistent launch (2D, one problem).
//
// The LATTICE order runs the q^2 colours one after another; inside a colour the blocks
// are independent (same-coloured centres are q >= s + p apart, so no block reads a DOF
// another writes).  Launching one grid per colour costs a launch and a grid-wide drain per
// colour; here one cooperative launch runs every colour:
//
//   * the centre grid is cut into gx x gy rectangular regions, one per CTA, all CTAs
//     resident at once (cooperative launch);
//   * a CTA keeps its region's window of u (region + H = r + p on each side: every DOF its
//     blocks read) and of b (region + r) in shared memory and runs the colours in order;
//     per colour, three CTA-wide phases over all of the colour's blocks in the region:
//     (A) y pass of the sum-factorised block residual, one thread per (block, window
//     column); (B) x pass and r_B = b_B - (A u)_B, one thread per block DOF; (C) the
//     block solve e_B = A_B^{-1} r_B (interior class: the row in registers; boundary
//     classes: their own inverse, FP64 rows by compensated FP32 arithmetic) and u_B += e_B;
//   * only neighbouring regions interact (region sides >= 2r + p): a block of a region
//     writes DOFs up to r outside it and reads up to r + p outside it.  After colour t a
//     CTA stores to global memory every DOF it changed that a neighbour may read (those
//     within H of a side that has a neighbour, or outside the region), then raises its
//     progress counter to t + 1 (release); before colour t + 1 it waits until each of its
//     8 neighbours has reached t + 1 (acquire, bounded by the handle's wait budget) and
//     reloads from L2 the part of its window a neighbour may have changed (within r of a
//     side that has a neighbour, or outside the region);
//   * at the end each CTA stores the rest of its region (its core).
//
// The arithmetic of every block is the same as in the per-colour kernels, and the result
// equals the LATTICE order exactly: a block of colour t sees every update of colours < t
// in its patch and none of colour > t (a neighbour cannot start colour t + 1 before this
// CTA has finished colour t).  A wait that gives up records it in the status word and the
// CTA leaves its loop; its neighbours then give up too, so the launch always ends.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "device_util.cuh"
#include "internal.h"

namespace iga2l {

namespace {

// h-scaled interior 1D rows as pairs: (k[a], m[a]) for the y pass, (m[a], k[a]) for the x pass
__constant__ float2 c_pkm[kMaxP + 1][2 * kMaxP + 1], c_pmk[kMaxP + 1][2 * kMaxP + 1];

constexpr int kPersistThreads = 512;
constexpr int kPersistMaxCtas = 4096;

template <int P, int S>
struct PGeom {
    static constexpr int W = 2 * P + 1, SS = S * S, R = (S - 1) / 2, H = R + P, WIN = S + 2 * P;
    static constexpr int YS = WIN | 1;                // odd row stride of a block's y sums
    static constexpr int RSS = (SS + 3) / 4 * 4;      // block residual stride (16-byte aligned)
    static constexpr int NB2 = (SS + 1) / 2;          // pairs of an inverse row
    static constexpr bool BREG = SS <= 25;            // interior inverse row kept in registers
    static constexpr int NT = kPersistThreads;
    static constexpr int GA = NT / WIN;               // phase A: groups of WIN threads
    static constexpr int GE = NT / SS;                // phases B, C: groups of SS threads
};

// Shared-memory layout of one CTA (bytes), the same on host and device.
struct PLayout {
    int wx, wy, bx, by, nbmax;
    unsigned off_sb, off_yb, off_rs, off_bi, off_km, off_mk, total;
};

template <int P, int S>
__host__ __device__ inline PLayout persist_layout(int rxmax, int rymax, int q)
{
    using G = PGeom<P, S>;
    PLayout L;
    L.wx = rxmax + 2 * G::H;
    L.wy = rymax + 2 * G::H;
    L.bx = rxmax + 2 * G::R;
    L.by = rymax + 2 * G::R;
    L.nbmax = ((rxmax + q - 1) / q) * ((rymax + q - 1) / q);
    auto up = [](unsigned x) { return (x + 15u) & ~15u; };
    unsigned o = up(sizeof(float) * L.wx * L.wy);                 // su
    L.off_sb = o;
    o = up(o + sizeof(float) * L.bx * L.by);
    L.off_yb = o;
    o = up(o + sizeof(float2) * L.nbmax * S * G::YS);
    L.off_rs = o;
    o = up(o + sizeof(float) * L.nbmax * G::RSS);
    L.off_bi = o;
    o = up(o + (G::BREG ? 0u : sizeof(float) * G::SS * G::SS));
    L.off_km = o;
    o = up(o + sizeof(float2) * L.by * G::W);
    L.off_mk = o;
    o = up(o + sizeof(float2) * L.bx * G::W);
    L.total = o;
    return L;
}

struct PersistArgs {
    int n, q, g, rev, nbc, interior;
    int gx, gy;               // regions per axis
    int rxmax, rymax;         // largest region sides (layout)
    const float *kband, *mband, *binv;
    const float *binv_lo;     // FP64 boundary inverses as pairs binv + binv_lo (Dot2), or null;
                              // both with every class's matrix transposed ([class][f][e])
    float *u;
    const float *b;
    unsigned int *progress;   // per CTA: colours finished in this launch (zeroed before it)
    int *status;              // waits that gave up
    long long budget;         // SM clock cycles per wait
    int withhold;             // error-path tests: CTA 0 never raises its counter
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned int *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int P, int S>
__global__ void __launch_bounds__(kPersistThreads, 2) k_schwarz_persist2d(const __grid_constant__ PersistArgs A)
{
    using G = PGeom<P, S>;
    constexpr int W = G::W, SS = G::SS, R = G::R, H = G::H, WIN = G::WIN, YS = G::YS, NT = G::NT;
    constexpr int PCI = 2 * P - 1;            // first interior row class
    constexpr int L1 = P - 1 + R;             // block classes per side
    constexpr int BIG = 1 << 30;
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ int s_abort;
    const PLayout Lo = persist_layout<P, S>(A.rxmax, A.rymax, A.q);
    float *su = reinterpret_cast<float *>(psm);
    float *sb = reinterpret_cast<float *>(psm + Lo.off_sb);
    float2 *yb = reinterpret_cast<float2 *>(psm + Lo.off_yb);
    float *rs = reinterpret_cast<float *>(psm + Lo.off_rs);
    float *bi = reinterpret_cast<float *>(psm + Lo.off_bi);
    float2 *km1y = reinterpret_cast<float2 *>(psm + Lo.off_km);
    float2 *mk1x = reinterpret_cast<float2 *>(psm + Lo.off_mk);
    const int tid = threadIdx.x, n = A.n, q = A.q;
    const int ci = blockIdx.x % A.gx, cj = blockIdx.x / A.gx;
    const int X0 = (int)((long long)ci * n / A.gx), X1 = (int)((long long)(ci + 1) * n / A.gx);
    const int Y0 = (int)((long long)cj * n / A.gy), Y1 = (int)((long long)(cj + 1) * n / A.gy);
    const bool hasL = ci > 0, hasR = ci + 1 < A.gx, hasD = cj > 0, hasU = cj + 1 < A.gy;
    // core (never read by a neighbour) and exclusive part (never written by one)
    const int cx0 = hasL ? X0 + H : -BIG, cx1 = hasR ? X1 - H : BIG;
    const int cy0 = hasD ? Y0 + H : -BIG, cy1 = hasU ? Y1 - H : BIG;
    const int ex0 = hasL ? X0 + R : -BIG, ex1 = hasR ? X1 - R : BIG;
    const int ey0 = hasD ? Y0 + R : -BIG, ey1 = hasU ? Y1 - R : BIG;
    const int wx0 = X0 - H, wy0 = Y0 - H, nwx = X1 - X0 + 2 * H, nwy = Y1 - Y0 + 2 * H;
    const int bx0 = X0 - R, by0 = Y0 - R, nbx = X1 - X0 + 2 * R, nby = Y1 - Y0 + 2 * R;
    const int WX = Lo.wx, BX = Lo.bx;

    // constant tables: boundary 1D rows (scaled like the interior constants: h K, M / h)
    // and the interior inverse
    {
        const float h = 1.0f / (float)(n - P + 2), hinv = (float)(n - P + 2);
        for (int i = tid; i < nby * W; i += NT) {
            const int row = i / W, a = i - row * W, gy = by0 + row;
            const bool in = gy >= 0 && gy < n;
            km1y[i] = make_float2(in ? A.kband[(size_t)gy * W + a] * h : 0.f, in ? A.mband[(size_t)gy * W + a] * hinv : 0.f);
        }
        for (int i = tid; i < nbx * W; i += NT) {
            const int col = i / W, a = i - col * W, gx = bx0 + col;
            const bool in = gx >= 0 && gx < n;
            mk1x[i] = make_float2(in ? A.mband[(size_t)gx * W + a] * hinv : 0.f, in ? A.kband[(size_t)gx * W + a] * h : 0.f);
        }
        if constexpr (!G::BREG)
            for (int i = tid; i < SS * SS; i += NT) bi[i] = A.binv[(size_t)A.interior * SS * SS + i];   // transposed
    }
    const int gA = tid / WIN, col = tid - gA * WIN;
    const int gB = tid / SS, e = tid - gB * SS;
    const int ey = e / S, ex = e - ey * S;
    float2 brow[G::BREG ? G::NB2 : 1];
    if constexpr (G::BREG) {
        const size_t base = (size_t)A.interior * SS * SS + e;
#pragma unroll
        for (int k = 0; k < G::NB2; ++k) {
            brow[k].x = gB < G::GE ? A.binv[base + (size_t)(2 * k) * SS] : 0.f;
            brow[k].y = (gB < G::GE && 2 * k + 1 < SS) ? A.binv[base + (size_t)(2 * k + 1) * SS] : 0.f;
        }
    }
    // windows of u and b (zero outside the grid); the residual padding stays zero
    for (int i = tid; i < nwx * nwy; i += NT) {
        const int wy = i / nwx, wx = i - wy * nwx, gx = wx0 + wx, gy = wy0 + wy;
        su[wy * WX + wx] = (gx >= 0 && gx < n && gy >= 0 && gy < n) ? __ldcg(&A.u[(size_t)gy * n + gx]) : 0.f;
    }
    for (int i = tid; i < nbx * nby; i += NT) {
        const int yy = i / nbx, xx = i - yy * nbx, gx = bx0 + xx, gy = by0 + yy;
        sb[yy * BX + xx] = (gx >= 0 && gx < n && gy >= 0 && gy < n) ? __ldg(&A.b[(size_t)gy * n + gx]) : 0.f;
    }
    for (int i = tid; i < Lo.nbmax * G::RSS; i += NT) rs[i] = 0.f;
    if (tid == 0) s_abort = 0;
    __syncthreads();

    const int ncol = q * q;
    for (int t = 0; t < ncol; ++t) {
        if (t > 0) {
            // every neighbour has finished colour t - 1: then reload what they may have changed
            if (tid < 9 && tid != 4) {
                const int ni = ci + tid % 3 - 1, nj = cj + tid / 3 - 1;
                if (ni >= 0 && ni < A.gx && nj >= 0 && nj < A.gy) {
                    const unsigned int *pc = A.progress + nj * A.gx + ni;
                    const long long t0 = clock64();
                    bool ok = ld_acquire(pc) >= (unsigned)t;
                    while (!ok && clock64() - t0 < A.budget) ok = ld_acquire(pc) >= (unsigned)t;
                    if (!ok) {
                        atomicAdd(A.status, 1);
                        s_abort = 1;
                    }
                }
            }
            __syncthreads();
            if (s_abort) break;
            // the window minus the exclusive rectangle: four strips
            const int rx0 = max(ex0, wx0), rx1 = min(ex1, wx0 + nwx), ry0 = max(ey0, wy0), ry1 = min(ey1, wy0 + nwy);
            const int ht = ry0 - wy0, hb = wy0 + nwy - ry1, hm = ry1 - ry0;
            const int wl = rx0 - wx0, wr = wx0 + nwx - rx1;
            const int n1 = ht * nwx, n2 = n1 + hb * nwx, n3 = n2 + hm * wl, n4 = n3 + hm * wr;
            // RL loads of a thread in flight before its stores
            constexpr int RL = 8;
            for (int i0 = tid; i0 < n4; i0 += RL * NT) {
                float v[RL];
                int w[RL];
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    const int i = i0 + r * NT;
                    int wx = 0, wy = 0;
                    if (i < n1) { wy = i / nwx; wx = i - wy * nwx; }
                    else if (i < n2) { const int k = i - n1; wy = ry1 - wy0 + k / nwx; wx = k % nwx; }
                    else if (i < n3) { const int k = i - n2; wy = ht + k / wl; wx = k % wl; }
                    else if (i < n4) { const int k = i - n3; wy = ht + k / wr; wx = rx1 - wx0 + k % wr; }
                    const int gx = wx0 + wx, gy = wy0 + wy;
                    const bool ok = i < n4 && gx >= 0 && gx < n && gy >= 0 && gy < n;
                    w[r] = ok ? wy * WX + wx : -1;
                    v[r] = ok ? __ldcg(&A.u[(size_t)gy * n + gx]) : 0.f;
                }
#pragma unroll
                for (int r = 0; r < RL; ++r)
                    if (w[r] >= 0) su[w[r]] = v[r];
            }
            __syncthreads();
        }
        const int c = A.rev ? ncol - 1 - t : t;
        const int ox = ((c % q) * A.g) % q, oy = ((c / q) * A.g) % q;
        // the colour's centres ox + q i, oy + q j inside the region
        const int i0 = X0 > ox ? (X0 - ox + q - 1) / q : 0, j0 = Y0 > oy ? (Y0 - oy + q - 1) / q : 0;
        const int nix = X1 - 1 >= ox + q * i0 ? (X1 - 1 - ox) / q - i0 + 1 : 0;
        const int niy = Y1 - 1 >= oy + q * j0 ? (Y1 - 1 - oy) / q - j0 + 1 : 0;
        const int nbk = nix * niy;
        // (A) y pass: Y[r][col] = (sum_b K_y[b] u, sum_b M_y[b] u) down window column col
        if (gA < G::GA)
            for (int k = gA; k < nbk; k += G::GA) {
                const int cx = ox + q * (i0 + k % nix), cy = oy + q * (j0 + k / nix);
                const float *up = su + (cy - Y0) * WX + (cx - X0) + col;
                float v[WIN];
#pragma unroll
                for (int kk = 0; kk < WIN; ++kk) v[kk] = up[kk * WX];
                float2 *yo = yb + k * (S * YS) + col;
                if (cy - R >= PCI && cy + R <= n - 2 * P) {
#pragma unroll
                    for (int r = 0; r < S; ++r) {
                        float2 y = make_float2(0.f, 0.f);
#pragma unroll
                        for (int bb = 0; bb < W; ++bb) y = fma2(c_pkm[P][bb], splat2<float2>(v[r + bb]), y);
                        yo[r * YS] = y;
                    }
                } else {
                    const float2 *kr = km1y + (cy - R - by0) * W;
#pragma unroll
                    for (int r = 0; r < S; ++r) {
                        float2 y = make_float2(0.f, 0.f);
#pragma unroll
                        for (int bb = 0; bb < W; ++bb) y = fma2(kr[r * W + bb], splat2<float2>(v[r + bb]), y);
                        yo[r * YS] = y;
                    }
                }
            }
        __syncthreads();
        // (B) x pass and the block residual r_B = b_B - (A u)_B
        if (gB < G::GE)
            for (int k = gB; k < nbk; k += G::GE) {
                const int cx = ox + q * (i0 + k % nix), cy = oy + q * (j0 + k / nix);
                const int x = cx - R + ex, y = cy - R + ey;
                const float2 *yr = yb + k * (S * YS) + ey * YS + ex;
                float2 s2 = make_float2(0.f, 0.f);
                if (cx - R >= PCI && cx + R <= n - 2 * P) {
#pragma unroll
                    for (int a = 0; a < W; ++a) s2 = fma2(c_pmk[P][a], yr[a], s2);
                } else {
                    const float2 *mr = mk1x + (x - bx0) * W;
#pragma unroll
                    for (int a = 0; a < W; ++a) s2 = fma2(mr[a], yr[a], s2);
                }
                const bool in = x >= 0 && x < n && y >= 0 && y < n;
                rs[k * G::RSS + e] = in ? sb[(y - by0) * BX + (x - bx0)] - (s2.x + s2.y) : 0.f;
            }
        __syncthreads();
        // (C) block solve and update; DOFs a neighbour may read go to global memory too
        if (gB < G::GE)
            for (int k = gB; k < nbk; k += G::GE) {
                const int cx = ox + q * (i0 + k % nix), cy = oy + q * (j0 + k / nix);
                const int x = cx - R + ex, y = cy - R + ey;
                if (!(x >= 0 && x < n && y >= 0 && y < n)) continue;
                const int bxc = cx < L1 ? cx : (cx > n - 1 - L1 ? 2 * L1 - (n - 1 - cx) : L1);
                const int byc = cy < L1 ? cy : (cy > n - 1 - L1 ? 2 * L1 - (n - 1 - cy) : L1);
                const int cls = byc * A.nbc + bxc;
                const float *rb = rs + k * G::RSS;
                float ev;
                if (cls == A.interior) {
                    const float2 *r2 = reinterpret_cast<const float2 *>(rb);
                    float2 acc = make_float2(0.f, 0.f);
                    if constexpr (G::BREG) {
#pragma unroll
                        for (int kk = 0; kk < G::NB2; ++kk) acc = fma2(brow[kk], r2[kk], acc);
                    } else {
                        const float *br = bi + e;
#pragma unroll
                        for (int f = 0; f < SS; ++f) acc.x = fmaf(br[f * SS], rb[f], acc.x);
                    }
                    ev = acc.x + acc.y;
                } else if (A.binv_lo) {
                    const size_t col = (size_t)cls * SS * SS + e;
                    ev = dot2_row<SS, SS>(A.binv + col, A.binv_lo + col, rb);
                } else {
                    const float *Bi = A.binv + (size_t)cls * SS * SS + e;
                    ev = 0.f;
#pragma unroll
                    for (int f = 0; f < SS; ++f) ev = fmaf(__ldg(&Bi[(size_t)f * SS]), rb[f], ev);
                }
                float &ref = su[(y - wy0) * WX + (x - wx0)];
                const float nv = ref + ev;
                ref = nv;
                if (x < cx0 || x >= cx1 || y < cy0 || y >= cy1) A.u[(size_t)y * n + x] = nv;
            }
        __syncthreads();
        if (tid == 0 && !(A.withhold && blockIdx.x == 0)) {
            __threadfence();
            st_release(A.progress + blockIdx.x, (unsigned)(t + 1));
        }
    }
    if (s_abort) return;
    // the core: DOFs no neighbour reads, stored once at the end
    const int kx0 = max(cx0, max(wx0, 0)), kx1 = min(cx1, min(wx0 + nwx, n));
    const int ky0 = max(cy0, max(wy0, 0)), ky1 = min(cy1, min(wy0 + nwy, n));
    const int kw = kx1 - kx0, kh = ky1 - ky0;
    if (kw > 0 && kh > 0)
        for (int i = tid; i < kw * kh; i += NT) {
            const int yy = ky0 + i / kw, xx = kx0 + i % kw;
            A.u[(size_t)yy * n + xx] = su[(yy - wy0) * WX + (xx - wx0)];
        }
}

// Regions and shared memory of the launch: about two CTAs per SM (then one), region
// sides >= 2r + p, all CTAs resident at once.  Returns false if no such plan exists.
template <int P, int S>
bool persist_plan(Solver &S_)
{
    using G = PGeom<P, S>;
    const int n = S_.n, minside = 2 * G::R + P;
    static std::mutex mu;
    static int smem_set[64] = {};
    for (int per_sm = 2; per_sm >= 1; --per_sm) {
        const int target = per_sm * S_.nsm;
        const int gx = std::max(1, std::min((int)std::sqrt((double)target), n / minside));
        const int gy = std::max(1, std::min(target / gx, n / minside));
        const int rxmax = (n + gx - 1) / gx, rymax = (n + gy - 1) / gy;
        const PLayout L = persist_layout<P, S>(rxmax, rymax, S_.q);
        if (L.total > 227u * 1024u || gx * gy > kPersistMaxCtas) continue;
        cudaError_t e = cudaSuccess;
        {
            std::lock_guard<std::mutex> lock(mu);
            if (S_.device < 0 || S_.device >= 64) return false;
            if (smem_set[S_.device] < (int)L.total) {
                e = cudaFuncSetAttribute(k_schwarz_persist2d<P, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.total);
                if (e == cudaSuccess) smem_set[S_.device] = (int)L.total;
            }
        }
        int occ = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_schwarz_persist2d<P, S>, G::NT, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (occ >= 1 && gx * gy <= occ * S_.nsm) {
            S_.pgx = gx;
            S_.pgy = gy;
            S_.prx = rxmax;
            S_.pry = rymax;
            S_.psmem = L.total;
            return true;
        }
    }
    return false;
}

template <int P, int S>
cudaError_t persist_p(const Solver &S_, float *u, const float *b, bool reverse, cudaStream_t st)
{
    const int nct = S_.pgx * S_.pgy;
    cudaError_t e = cudaMemsetAsync(S_.progress, 0, sizeof(unsigned int) * nct, st);
    if (e != cudaSuccess) return e;
    PersistArgs a;
    a.n = S_.n;
    a.q = S_.q;
    a.g = S_.g;
    a.rev = reverse ? 1 : 0;
    a.nbc = S_.ht.nbc;
    a.interior = S_.ht.L * S_.ht.nbc + S_.ht.L;
    a.gx = S_.pgx;
    a.gy = S_.pgy;
    a.rxmax = S_.prx;
    a.rymax = S_.pry;
    a.kband = S_.mx.Kb;
    a.mband = S_.mx.Mb;
    a.binv = S_.mx.binv_t;
    a.binv_lo = S_.boundary_lo_t();
    a.u = u;
    a.b = b;
    a.progress = S_.progress;
    a.status = S_.wait_status;
    a.budget = S_.opt.wait_budget_cycles;
    a.withhold = (S_.opt.test_flags & IGA2L_TEST_WITHHOLD_PROGRESS) != 0;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nct);
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = S_.psmem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_schwarz_persist2d<P, S>, a);
    count_launches(1);
    return e;
}

}  // namespace

bool persist_setup(Solver &S)
{
    S.pgx = 0;
    if (!(S.dim == 2 && S.nbatch == 1 && S.mx.enabled && S.progress && S.wait_status)) return false;
    if (S.s == 3) {
        switch (S.p) {
        case 2: return persist_plan<2, 3>(S);
        case 3: return persist_plan<3, 3>(S);
        case 4: return persist_plan<4, 3>(S);
        default: return false;
        }
    }
    if (S.s == 5 && S.p == 5) return persist_plan<5, 5>(S);
    if (S.s == 5 && S.p == 6) return persist_plan<6, 5>(S);
    if (S.s == 7 && S.p == 7) return persist_plan<7, 7>(S);
    if (S.s == 7 && S.p == 8) return persist_plan<8, 7>(S);
    return false;
}

cudaError_t launch_schwarz_persist(const Solver &S, float *u, const float *b, bool reverse, cudaStream_t st)
{
    if (S.s == 3) {
        switch (S.p) {
        case 2: return persist_p<2, 3>(S, u, b, reverse, st);
        case 3: return persist_p<3, 3>(S, u, b, reverse, st);
        case 4: return persist_p<4, 3>(S, u, b, reverse, st);
        default: break;
        }
    } else if (S.s == 5) {
        if (S.p == 5) return persist_p<5, 5>(S, u, b, reverse, st);
        if (S.p == 6) return persist_p<6, 5>(S, u, b, reverse, st);
    } else if (S.s == 7) {
        if (S.p == 7) return persist_p<7, 7>(S, u, b, reverse, st);
        if (S.p == 8) return persist_p<8, 7>(S, u, b, reverse, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t upload_persist_rows(int p, const double *k1, const double *m1)
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
    float2 km[W1], mk[W1];
    const int w = 2 * p + 1;
    for (int i = 0; i < w; ++i) {
        km[i] = make_float2((float)k1[i], (float)m1[i]);
        mk[i] = make_float2((float)m1[i], (float)k1[i]);
    }
    e = cudaMemcpyToSymbol(c_pkm, km, sizeof(float2) * w, sizeof(float2) * W1 * p);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_pmk, mk, sizeof(float2) * w, sizeof(float2) * W1 * p);
    if (e == cudaSuccess) done[dev][p] = true;
    return e;
}

}  // namespace iga2l
