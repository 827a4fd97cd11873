// kernels_tc.cu -- the interior blocks of one LATTICE colour as a tensor-core GEMM (2D).
//
// Interior Schwarz blocks are translation invariant (Section 3.1.1: every block is the
// s x s box around a grid point; away from the boundary all such blocks see the same
// Toeplitz rows of A), so the correction of block B is
//     e_B = A_B^{-1} (b - A u)_B = G x_B,   G = [A_B^{-1} | -A_B^{-1} A_(B,patch)],
//     x_B = [b_B ; u_patch],   patch = the (s + 2p)^2 DOFs the block's rows couple to,
// one matrix G for every interior block.  For a colour, the interior blocks' corrections
// are D = X G^T with X the (blocks x K) matrix of the x_B: a GEMM with K = s^2 + (s+2p)^2.
// Each CTA takes 128 blocks (M = 128): G arrives by one bulk asynchronous copy
// (cp.async.bulk, completion on an mbarrier), the warps gather X into shared memory in the
// tensor-core operand layout (K-major 8-row x 16-byte core matrices, no swizzle; lanes
// along k, so a patch row is a contiguous run of u), one thread issues the tcgen05.mma
// chain (kind::tf32, FP32 accumulation in tensor memory), completion arrives on a second
// mbarrier (every wait bounded), and each block's row of D is read back (tcgen05.ld) and
// added to u.  Blocks of one colour share no DOF and
// read no DOF another writes, so the CTAs run independently; the colour's remaining
// (boundary) blocks are done by the FP32 SIMT kernel.  Operands are rounded to TF32
// (10-bit mantissa); the FP64 outer refinement of the mixed form absorbs the difference.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

namespace iga2l {

namespace {

template <int P, int S>
struct TcGeom {
    static constexpr int SS = S * S, R = (S - 1) / 2, PW = S + 2 * P, KU = SS + PW * PW;
    static constexpr int KP = (KU + 7) / 8 * 8;        // K padded to the MMA step (8 for TF32)
    static constexpr int NP = (SS + 15) / 16 * 16;     // N padded (M = 128 needs N % 16 == 0)
    static constexpr int M = 128;
    static constexpr int TCOLS = NP < 32 ? 32 : NP;    // tensor-memory columns (power of two >= 32)
    static constexpr int LBO = 128;                    // bytes between the two 16-byte K halves of a step
    static constexpr int SBO = 32 * KP;                // bytes between 8-row groups
    static constexpr size_t XB = (size_t)M * KP * 4, GB = (size_t)NP * KP * 4;
    static constexpr size_t smem = XB + GB + 32;   // + two mbarriers and the TMEM address
};

// float offset of element (row r, k) in the K-major no-swizzle operand layout
__host__ __device__ inline int tc_off(int r, int k, int kp)
{
    return (r / 8) * (8 * kp) + (k / 4) * 32 + (r % 8) * 4 + (k % 4);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Waits for phase `parity` of an mbarrier for at most `budget` SM clock cycles; returns
// whether the phase completed.
__device__ __forceinline__ int mbar_wait_bounded(uint32_t bar, uint32_t parity, long long budget)
{
    const long long t0 = clock64();
    uint32_t ok = 0;
    do {
        asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, q;\n}"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
    } while (!ok && clock64() - t0 < budget);
    return (int)ok;
}

// shared-memory matrix descriptor: start, leading / stride byte offsets, version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int P, int S>
__global__ void __launch_bounds__(512)
k_schwarz_tc(int n, int q, int ox, int oy, int ix0, int iy0, int nix, int niy, int bpc, const float *__restrict__ gtc,
             const float *__restrict__ b, float *__restrict__ u, int *__restrict__ status, long long budget,
             int skip_copy)
{
    using G = TcGeom<P, S>;
    constexpr int SS = G::SS, R = G::R, PW = G::PW, KU = G::KU, KP = G::KP, NP = G::NP, M = G::M;
    constexpr int NT = 512, NWARP = NT / 32;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    float *sX = reinterpret_cast<float *>(tc_smem);
    float *sG = reinterpret_cast<float *>(tc_smem + G::XB);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(tc_smem + G::XB + G::GB);   // [0]: MMA, [1]: copy of G
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tc_smem + G::XB + G::GB + 16);
    __shared__ int s_mma;   // 1: the operator landed and the MMA chain was issued
    const long long drain = budget > (1LL << 31) ? budget : (1LL << 31);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // bpc (<= M) blocks per CTA, chosen so that the grid covers the SMs once; rows beyond are zero
    const int nblk = nix * niy, m0 = blockIdx.x * bpc;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // G (already in the operand layout) by one bulk asynchronous copy
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&mbar[1])),
                     "r"((uint32_t)G::GB)
                     : "memory");
        if (!skip_copy)   // (error-path tests leave the copy out, so its wait runs out)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             smem_addr(sG)),
                         "l"(gtc), "r"((uint32_t)G::GB), "r"(smem_addr(&mbar[1]))
                         : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(G::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // X: warp per block row, lanes along k (the patch rows are contiguous runs of u); RU rows
    // of loads in flight per warp
    constexpr int NK = (KP + 31) / 32, RU = 4;
    for (int r0 = warp * RU; r0 < M; r0 += NWARP * RU) {
        float v[RU][NK];
#pragma unroll
        for (int rr = 0; rr < RU; ++rr) {
            const int m = m0 + r0 + rr;
            const bool valid = r0 + rr < bpc && m < nblk;
            const int cx = valid ? ox + q * (ix0 + m % nix) : 0, cy = valid ? oy + q * (iy0 + m / nix) : 0;
#pragma unroll
            for (int t = 0; t < NK; ++t) {
                const int k = lane + 32 * t;
                float x = 0.f;
                if (valid && k < KU) {
                    if (k < SS) {
                        x = __ldg(&b[(size_t)(cy - R + k / S) * n + (cx - R + k % S)]);
                    } else {
                        const int j = k - SS;
                        x = u[(size_t)(cy - R - P + j / PW) * n + (cx - R - P + j % PW)];
                    }
                }
                v[rr][t] = x;
            }
        }
#pragma unroll
        for (int rr = 0; rr < RU; ++rr)
#pragma unroll
            for (int t = 0; t < NK; ++t) {
                const int k = lane + 32 * t;
                if (k < KP) sX[tc_off(r0 + rr, k, KP)] = to_tf32(v[rr][t]);
            }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> MMA reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        // G has landed (bounded wait), then the MMA chain
        int gready = mbar_wait_bounded(smem_addr(&mbar[1]), 0, budget);
        if (!gready) {
            atomicAdd(status, 1);
            // a copy still in flight must land before the CTA may exit (bounded again, by
            // at least the default budget whatever the caller chose)
            if (!skip_copy) mbar_wait_bounded(smem_addr(&mbar[1]), 0, drain);
        }
        s_mma = gready;
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
    if (s_mma) {
        done = mbar_wait_bounded(smem_addr(&mbar[0]), 0, budget);
        done = __all_sync(0xffffffffu, done);   // tcgen05.ld below is warp-collective
        if (!done) {
            if (lane == 0) atomicAdd(status, 1);
            mbar_wait_bounded(smem_addr(&mbar[0]), 0, drain);
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (done && (warp >> 2) * 8 < NP) {
        // warps w, w + 4, ... read the rows of TMEM sub-partition w % 4, each a slice of the
        // columns (8 at a time; the warps beyond the columns wait)
        constexpr int HALF = 8;
        const int sub = warp & 3, c_base = (warp >> 2) * HALF;
        const int r = sub * 32 + lane, m = m0 + r;
        float e[HALF];
#pragma unroll
        for (int c0 = 0; c0 < HALF; c0 += 8) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(c_base + c0);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j) e[c0 + j] = __uint_as_float(v[j]);
        }
        if (r < bpc && m < nblk) {
            const int cx = ox + q * (ix0 + m % nix), cy = oy + q * (iy0 + m / nix);
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                const int k = c_base + j;
                if (k < SS) u[(size_t)(cy - R + k / S) * n + (cx - R + k % S)] += e[j];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TCOLS));
}

template <int P, int S>
cudaError_t launch_tc_p(const Solver &S_, int ox, int oy, int ix0, int iy0, int nix, int niy, const float *b,
                        float *u, cudaStream_t st)
{
    using G = TcGeom<P, S>;
    static bool attr_set[64] = {};
    if (S_.device >= 0 && S_.device < 64 && !attr_set[S_.device]) {
        cudaError_t e = cudaFuncSetAttribute(k_schwarz_tc<P, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::smem);
        if (e != cudaSuccess) return e;
        attr_set[S_.device] = true;
    }
    const int nblk = nix * niy;
    static int nsm[64] = {};
    if (S_.device >= 0 && S_.device < 64 && nsm[S_.device] == 0)
        cudaDeviceGetAttribute(&nsm[S_.device], cudaDevAttrMultiProcessorCount, S_.device);
    const int sms = (S_.device >= 0 && S_.device < 64 && nsm[S_.device] > 0) ? nsm[S_.device] : 1;
    int bpc = (nblk + sms - 1) / sms;   // one CTA per SM (the operands take most of its shared memory)
    if (bpc > G::M) bpc = G::M;
    if (bpc < 1) bpc = 1;
    k_schwarz_tc<P, S><<<(nblk + bpc - 1) / bpc, 512, G::smem, st>>>(S_.n, S_.q, ox, oy, ix0, iy0, nix, niy, bpc,
                                                                     S_.mx.gtc, b, u, S_.wait_status,
                                                                     S_.opt.wait_budget_cycles,
                                                                     (S_.opt.test_flags & IGA2L_TEST_SKIP_OPERATOR_COPY) != 0);
    count_launches(1);
    return cudaGetLastError();
}

// 1D Galerkin coupling K[a][c] (or M) from the band rows (zero outside the band)
double band_at(const std::vector<double> &B, int p, int a, int c)
{
    const int d = c - a;
    if (d < -p || d > p) return 0.0;
    return B[(size_t)a * (2 * p + 1) + (d + p)];
}

float tf32_host(double x)   // round to nearest (ties away) at the 10th mantissa bit, like cvt.rna
{
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

void tc_interior_rect(const Solver &S, int o, int nb, int &i0, int &ni)
{
    // centres c = o + q i with rows c - R .. c + R of the interior class (the patch is then
    // inside the grid and every coupling is the Toeplitz one)
    const int lo = 2 * S.p - 1 + S.r, hi = S.n - 2 * S.p - S.r;
    i0 = lo <= o ? 0 : (lo - o + S.q - 1) / S.q;
    const int i1 = hi < o ? -1 : (hi - o) / S.q;   // last admissible index
    ni = i1 >= i0 ? (i1 < nb ? i1 : nb - 1) - i0 + 1 : 0;
    if (ni < 0) ni = 0;
}

cudaError_t launch_schwarz_tc(const Solver &S, int ox, int oy, int ix0, int iy0, int nix, int niy, const float *b,
                              float *u, cudaStream_t st)
{
    switch (S.p) {
    case 2: return launch_tc_p<2, 3>(S, ox, oy, ix0, iy0, nix, niy, b, u, st);
    case 3: return launch_tc_p<3, 3>(S, ox, oy, ix0, iy0, nix, niy, b, u, st);
    case 4: return launch_tc_p<4, 3>(S, ox, oy, ix0, iy0, nix, niy, b, u, st);
    case 5: return launch_tc_p<5, 5>(S, ox, oy, ix0, iy0, nix, niy, b, u, st);
    case 6: return launch_tc_p<6, 5>(S, ox, oy, ix0, iy0, nix, niy, b, u, st);
    default: return cudaErrorInvalidValue;
    }
}

void build_gtc(const Solver &S, const std::vector<double> &ainv, std::vector<float> &g, int &nrows, int &kcols)
{
    const int p = S.p, s = S.s, r = S.r, n = S.n;
    const int SS = s * s, PW = s + 2 * p, KU = SS + PW * PW;
    const int KP = (KU + 7) / 8 * 8, NP = (SS + 15) / 16 * 16;
    const std::vector<double> &K = S.ht.Kb, &Mm = S.ht.Mb;
    const int c = n / 2;   // an interior block centre: rows and patch see only Toeplitz couplings
    std::vector<double> ap((size_t)SS * PW * PW);
    for (int f = 0; f < SS; ++f) {
        const int xf = c - r + f % s, yf = c - r + f / s;
        for (int j = 0; j < PW * PW; ++j) {
            const int xj = c - r - p + j % PW, yj = c - r - p + j / PW;
            ap[(size_t)f * PW * PW + j] = band_at(K, p, xf, xj) * band_at(Mm, p, yf, yj) +
                                          band_at(Mm, p, xf, xj) * band_at(K, p, yf, yj);
        }
    }
    g.assign((size_t)NP * KP, 0.0f);
    for (int e = 0; e < SS; ++e)
        for (int k = 0; k < KU; ++k) {
            double v;
            if (k < SS) {
                v = ainv[(size_t)e * SS + k];
            } else {
                v = 0.0;
                for (int f = 0; f < SS; ++f) v -= ainv[(size_t)e * SS + f] * ap[(size_t)f * PW * PW + (k - SS)];
            }
            g[tc_off(e, k, KP)] = tf32_host(v);
        }
    nrows = NP;
    kcols = KP;
}

}  // namespace iga2l
