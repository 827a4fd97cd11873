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
    T dinv;      // 1 / c[1][1] (rounded once): a Gauss-Seidel update multiplies by it
};

// red-black order of the sub-lattices: red (0,0), (1,1) then black (1,0), (0,1)
__constant__ int kGsSeqDev[4][2] = {{0, 0}, {1, 1}, {1, 0}, {0, 1}};

template <typename T>
Stencil9<T> level_stencil(const Level &L)
{
    Stencil9<T> s;
    for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx) s.c[dy][dx] = (T)(L.k[dx] * L.mm[dy] + L.mm[dx] * L.k[dy]);
    s.dinv = (T)(1.0 / (L.k[1] * L.mm[1] + L.mm[1] * L.k[1]));
    return s;
}

// ---- fused level kernels --------------------------------------------------------------
// One relaxation of the V(1,1) smoother is four sub-lattice sweeps {(2a+px, 2b+py)}, each
// e += (rhs - A e) / A_diag, the quotient taken as a product with the once-rounded
// reciprocal of the diagonal (within about an ulp of the quotient); no two points of a
// sub-lattice are coupled by the 9-point stencil.  A CTA owns a TX x TY tile of the level and stages it with a halo of H >= 4:
// after sweep k every staged point at distance >= k from the staged edge holds exactly the
// value the four global sweeps give (its neighbours were exact after sweep k-1), so the
// tile is exact after four sweeps and one launch replaces four.  Points outside the level
// are zero and never updated.  Each point update uses the arithmetic, in the order, of a
// plain per-sweep kernel.
constexpr int kLvTX = 32, kLvTY = 16;

template <typename T, int RX, int RY>
__device__ __forceinline__ void level_sweeps(int n, int gx0, int gy0, const Stencil9<T> &st, T (*se)[RX],
                                             const T (*sr)[RX], bool forward)
{
    constexpr int HX = RX / 2, HY = RY / 2;   // sub-lattice points per row / column of the region
    for (int t = 0; t < 4; ++t) {
        const int c = forward ? t : 3 - t;
        const int px = kGsSeqDev[c][0], py = kGsSeqDev[c][1];   // region origin is even
        for (int i = threadIdx.x + blockDim.x * threadIdx.y; i < HX * HY; i += blockDim.x * blockDim.y) {
            const int lx = 2 * (i % HX) + px, ly = 2 * (i / HX) + py;
            const int d = min(min(lx, ly), min(RX - 1 - lx, RY - 1 - ly));
            const int gx = gx0 + lx, gy = gy0 + ly;
            if (d < t + 1 || gx < 0 || gx >= n || gy < 0 || gy >= n) continue;
            T acc = T(0);
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int yy = gy + dy - 1;
                if (yy < 0 || yy >= n) continue;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int xx = gx + dx - 1;
                    if (xx >= 0 && xx < n) acc = fma(st.c[dy][dx], se[ly + dy - 1][lx + dx - 1], acc);
                }
            }
            se[ly][lx] += (sr[ly][lx] - acc) * st.dinv;
        }
        __syncthreads();
    }
}

// Pre-smoothing from e = 0, then the level residual restricted to the next level:
//   epre = S_fwd(0; rhs) on the tile,
//   rc[J][I] = sum_{dy,dx} w_dy w_dx (rhs - A epre)[2J+dy][2I+dx], w = (1/2, 1, 1/2),
// for the coarse points whose fine support lies in the tile plus one column / row (halo 6).
template <typename T>
__global__ void __launch_bounds__(kLvTX *kLvTY / 2)
k_level_pre(int nf, int nc, Stencil9<T> st, const T *__restrict__ rhs, T *__restrict__ epre, T *__restrict__ rc,
            BatchRef bt)
{
    constexpr int H = 6, RX = kLvTX + 2 * H, RY = kLvTY + 2 * H;
    __shared__ T se[RY][RX], sr[RY][RX];
    __shared__ T res[kLvTY + 1][kLvTX + 1];
    pdl_wait();
    if (bt.active && !bt.active[blockIdx.z]) return;
    rhs += blockIdx.z * bt.vec;
    epre += blockIdx.z * bt.vec;
    rc += blockIdx.z * bt.crs;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
    const int x0 = blockIdx.x * kLvTX, y0 = blockIdx.y * kLvTY, gx0 = x0 - H, gy0 = y0 - H;
    for (int i = tid; i < RX * RY; i += nt) {
        const int lx = i % RX, ly = i / RX, gx = gx0 + lx, gy = gy0 + ly;
        sr[ly][lx] = (gx >= 0 && gx < nf && gy >= 0 && gy < nf) ? rhs[(size_t)gy * nf + gx] : T(0);
        se[ly][lx] = T(0);
    }
    __syncthreads();
    level_sweeps<T, RX, RY>(nf, gx0, gy0, st, se, sr, true);
    for (int i = tid; i < kLvTX * kLvTY; i += nt) {
        const int x = x0 + i % kLvTX, y = y0 + i / kLvTX;
        if (x < nf && y < nf) epre[(size_t)y * nf + x] = se[y - gy0][x - gx0];
    }
    for (int i = tid; i < (kLvTX + 1) * (kLvTY + 1); i += nt) {
        const int rx = i % (kLvTX + 1), ry = i / (kLvTX + 1), x = x0 + rx, y = y0 + ry;
        T r = T(0);
        if (x < nf && y < nf) {
            T a = T(0);
#pragma unroll
            for (int ey = 0; ey < 3; ++ey) {
                const int yy = y + ey - 1;
                if (yy < 0 || yy >= nf) continue;
#pragma unroll
                for (int ex = 0; ex < 3; ++ex) {
                    const int xx = x + ex - 1;
                    if (xx >= 0 && xx < nf) a = fma(st.c[ey][ex], se[yy - gy0][xx - gx0], a);
                }
            }
            r = sr[y - gy0][x - gx0] - a;
        }
        res[ry][rx] = r;
    }
    __syncthreads();
    const T w[3] = {T(0.5), T(1), T(0.5)};
    for (int i = tid; i < (kLvTX / 2) * (kLvTY / 2); i += nt) {
        const int I = x0 / 2 + i % (kLvTX / 2), J = y0 / 2 + i / (kLvTX / 2);
        if (I >= nc || J >= nc) continue;
        T acc = T(0);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            T sacc = T(0);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) sacc = fma(w[dx], res[2 * J + dy - y0][2 * I + dx - x0], sacc);
            acc = fma(w[dy], sacc, acc);
        }
        rc[(size_t)J * nc + I] = acc;
    }
}

// Coarse correction and post-smoothing: e_out = S_rev(epre + P ec; rhs) on the tile,
// P the exact embedding of the coarse hats (weights 1/2, 1, 1/2) (halo 4).
template <typename T>
__global__ void __launch_bounds__(kLvTX *kLvTY / 2)
k_level_post(int nf, int nc, Stencil9<T> st, const T *__restrict__ rhs, const T *__restrict__ epre,
             const T *__restrict__ ec, T *__restrict__ eout, BatchRef bt)
{
    constexpr int H = 4, RX = kLvTX + 2 * H, RY = kLvTY + 2 * H;
    __shared__ T se[RY][RX], sr[RY][RX];
    pdl_wait();
    if (bt.active && !bt.active[blockIdx.z]) return;
    rhs += blockIdx.z * bt.vec;
    epre += blockIdx.z * bt.vec;
    eout += blockIdx.z * bt.vec;
    ec += blockIdx.z * bt.crs;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
    const int x0 = blockIdx.x * kLvTX, y0 = blockIdx.y * kLvTY, gx0 = x0 - H, gy0 = y0 - H;
    for (int i = tid; i < RX * RY; i += nt) {
        const int lx = i % RX, ly = i / RX, x = gx0 + lx, y = gy0 + ly;
        T ev = T(0), rv = T(0);
        if (x >= 0 && x < nf && y >= 0 && y < nf) {
            rv = rhs[(size_t)y * nf + x];
            // fine x is coarse (x-1)/2 when odd (weight 1); between x/2-1 and x/2 when even
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
                    sacc = fma(wx[aq], ec[(size_t)Iy[bq] * nc + Ix[aq]], sacc);
                }
                acc = fma(wy[bq], sacc, acc);
            }
            ev = epre[(size_t)y * nf + x] + acc;
        }
        se[ly][lx] = ev;
        sr[ly][lx] = rv;
    }
    __syncthreads();
    level_sweeps<T, RX, RY>(nf, gx0, gy0, st, se, sr, false);
    for (int i = tid; i < kLvTX * kLvTY; i += nt) {
        const int x = x0 + i % kLvTX, y = y0 + i / kLvTX;
        if (x < nf && y < nf) eout[(size_t)y * nf + x] = se[y - gy0][x - gx0];
    }
}

// x = Ainv rhs in FP64, one warp per row (dense inverse of the directly solved level)
template <typename T>
__global__ void k_dense_matvec(int N, const double *__restrict__ Ainv, const T *__restrict__ rhs,
                               T *__restrict__ x, BatchRef bt)
{
    pdl_wait();
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
            e[i] = ((x | y) & 1) ? T(0) : (rhs[i] - T(0)) * st.dinv;
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
        e[y * n + x] += (rhs[y * n + x] - acc) * st.dinv;
    }
}

// The arguments are read in place (__grid_constant__: per-level values indexed at run
// time come from the constant bank, not from a per-thread local copy of the struct).
// Level l's correction E and right-hand side Rh lie one after the other in shared
// memory, after those of the levels above it.
template <typename T>
__device__ __forceinline__ T *tail_level(T *base, const TailArgs<T> &a, int l)
{
    for (int k = 0; k < l; ++k) base += 2 * a.n[k] * a.n[k];
    return base;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_vcycle_tail(const __grid_constant__ TailArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char tail_smem[];
    T *const base = reinterpret_cast<T *>(tail_smem);
    pdl_wait();
    if (a.active && !a.active[blockIdx.x]) return;
    const T *rhs0 = a.rhs0 + blockIdx.x * a.vec0;
    T *e0 = a.e0 + blockIdx.x * a.vec0;
    for (int i = threadIdx.x; i < a.n[0] * a.n[0]; i += blockDim.x) base[a.n[0] * a.n[0] + i] = rhs0[i];
    __syncthreads();
    const int last = a.nl - 1;
    for (int l = 0; l < last; ++l) {
        const int n = a.n[l], nc = a.n[l + 1];
        T *E = tail_level(base, a, l), *Rh = E + n * n, *Rc = Rh + n * n + nc * nc;
        const Stencil9<T> st = a.st[l];
        for (int t = 0; t < 4; ++t) {
            tail_gs<T>(n, st, Rh, E, kGsSeqDev[t][0], kGsSeqDev[t][1], t == 0);
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
                            if (xx >= 0 && xx < n) aa = fma(st.c[ey][ex], E[yy * n + xx], aa);
                        }
                    }
                    const T r = Rh[y * n + x] - aa;
                    sacc = fma(w[dx], r, sacc);
                }
                acc = fma(w[dy], sacc, acc);
            }
            Rc[J * nc + I] = acc;
        }
        __syncthreads();
    }
    {   // direct solve: warp-per-row dot products, the reduction order of k_dense_matvec
        const int N = a.n[last] * a.n[last];
        T *El = tail_level(base, a, last), *Rl = El + N;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int row = warp; row < N; row += nw) {
            const double *rp = a.dinv + (size_t)row * N;
            double sacc = 0.0;
            for (int j = lane; j < N; j += 32) sacc = fma(rp[j], (double)Rl[j], sacc);
            for (int off = 16; off > 0; off >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, off);
            if (lane == 0) El[row] = (T)sacc;
        }
        __syncthreads();
    }
    for (int l = last - 1; l >= 0; --l) {
        const int nf = a.n[l], nc = a.n[l + 1];
        T *E = tail_level(base, a, l), *Rh = E + nf * nf, *Ec = Rh + nf * nf;
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
                    sacc = fma(wx[aq], Ec[Iy[bq] * nc + Ix[aq]], sacc);
                }
                acc = fma(wy[bq], sacc, acc);
            }
            E[i] += acc;
        }
        __syncthreads();
        const Stencil9<T> st = a.st[l];
        for (int t = 3; t >= 0; --t) {
            tail_gs<T>(nf, st, Rh, E, kGsSeqDev[t][0], kGsSeqDev[t][1], false);
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < a.n[0] * a.n[0]; i += blockDim.x) e0[i] = base[i];
}

// levE[l], levR[l]: the e and rhs arrays of level l >= 1 in the storage type T; levP[l]:
// the pre-smoothed correction of level l
template <typename T>
cudaError_t vcycle(const Solver &S, int l, const T *rhs, T *e, T *const *levE, T *const *levR, T *const *levP,
                   cudaStream_t s)
{
    const Level &L = S.lev[l];
    const int last = (int)S.lev.size() - 1;
    const int nb = S.nbatch;
    if (l == last) {
        const int N = S.ndirect;
        const cudaError_t err = launch_pdl(k_dense_matvec<T>, dim3((N * 32 + 255) / 256, nb), dim3(256), s, N,
                                           (const double *)S.dinv, rhs, e, BatchRef{S.active, L.N, 0, 0});
        count_launches(1);
        return err;
    }
    // small levels: the rest of the cycle in one thread block per problem, in shared memory
    // larger levels: the fused multi-CTA level kernels are faster (an FP32 tail from 63
    // measured 1% slower per mixed solve)
    const int tail_n = 31;
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
            const cudaError_t err = launch_pdl_smem(k_vcycle_tail<T>, dim3(nb), dim3(1024), smem, s, a);
            count_launches(1);
            return err;
        }
    }
    const Level &C = S.lev[l + 1];
    const Stencil9<T> st = level_stencil<T>(L);
    const BatchRef bt{S.active, L.N, 0, C.N};
    const dim3 blk(kLvTX, kLvTY / 2), grd((L.n + kLvTX - 1) / kLvTX, (L.n + kLvTY - 1) / kLvTY, nb);
    cudaError_t err;
    err = launch_pdl(k_level_pre<T>, grd, blk, s, L.n, C.n, st, rhs, levP[l], levR[l + 1], bt);
    count_launches(1);
    if (err != cudaSuccess) return err;
    if ((err = vcycle<T>(S, l + 1, levR[l + 1], levE[l + 1], levE, levR, levP, s)) != cudaSuccess) return err;
    err = launch_pdl(k_level_post<T>, grd, blk, s, L.n, C.n, st, rhs, (const T *)levP[l], (const T *)levE[l + 1], e,
                     bt);
    count_launches(1);
    return err;
}

}  // namespace

cudaError_t launch_coarse_solve(const Solver &S, const double *dc, double *ec, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_coarse_solve(S, dc, ec, st);
    std::vector<double *> E(S.lev.size()), Rr(S.lev.size()), Pp(S.lev.size());
    for (size_t l = 0; l < S.lev.size(); ++l) { E[l] = S.lev[l].e; Rr[l] = S.lev[l].rhs; Pp[l] = S.lev[l].pre; }
    return vcycle<double>(S, 0, dc, ec, E.data(), Rr.data(), Pp.data(), st);
}

cudaError_t launch_inner_coarse(const Solver &S, cudaStream_t st)
{
    if (S.dim == 3) return launch3d_inner_coarse(S, st);
    const MixedState &X = S.mx;
    return vcycle<float>(S, 0, X.dc, X.ec, X.lev_e.data(), X.lev_rhs.data(), X.lev_pre.data(), st);
}

}  // namespace iga2l
