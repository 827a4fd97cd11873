// kernels_tc.cu -- host side of the tensor-core colour step (2D): the operator G of the
// interior blocks in the MMA operand layout, and the rectangle of a colour's blocks that
// are interior.
//
// Interior Schwarz blocks are translation invariant (Section 3.1.1: every block is the
// s x s box around a grid point; away from the boundary all such blocks see the same
// Toeplitz rows of A), so the correction of block B is
//     e_B = A_B^{-1} (b - A u)_B = G x_B,   G = [A_B^{-1} | -A_B^{-1} A_(B,patch)],
//     x_B = [b_B ; u_patch],   patch = the (s + 2p)^2 DOFs the block's rows couple to,
// one matrix G for every interior block; a colour's interior corrections are D = X G^T
// (k_schwarz_tc_colour in kernels_fine.cu).  G is built here in FP64 and rounded to TF32.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc_util.cuh"

namespace iga2l {

namespace {

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
    g.assign((size_t)(NP / 8) * (8 * KP + 4), 0.0f);   // 8-row groups padded by 16 bytes (tc_off)
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
