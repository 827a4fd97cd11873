// tc_util.cuh -- operand geometry and tcgen05 (kind::tf32) helpers of the tensor-core
// colour step: the interior blocks of a LATTICE colour as one GEMM D = X G^T per CTA of
// M = 128 blocks (Section 3.1.1: interior blocks are translation invariant, so one operator
// G = [A_B^{-1} | -A_B^{-1} A_(B,patch)] serves all of them).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace iga2l {

// X (M x KP) and G (NP x KP) in the K-major, no-swizzle operand layout: 8-row x 16-byte
// core matrices, the two 16-byte halves of one K step LBO bytes apart, 8-row groups SBO
// bytes apart.  SBO is 16 bytes more than a group's 32 KP bytes, so that the core matrices
// of consecutive groups start on different shared-memory banks.  Column k of a block's
// row: k < s^2 the block's b values, then its (s + 2p)^2 patch values of u (row-major),
// then zeros up to KP.
template <int P, int S>
struct TcGeom {
    static constexpr int SS = S * S, R = (S - 1) / 2, PW = S + 2 * P, KU = SS + PW * PW;
    static constexpr int KP = (KU + 7) / 8 * 8;        // K padded to the MMA step (8 for TF32)
    static constexpr int NP = (SS + 15) / 16 * 16;     // N padded (M = 128 needs N % 16 == 0)
    static constexpr int M = 128;
    static constexpr int TBX = 16, TBY = 8;            // a CTA's blocks: TBX x TBY of the colour's lattice
    static constexpr int TCOLS = NP < 32 ? 32 : NP;    // tensor-memory columns (power of two >= 32)
    static constexpr int GS = 8 * KP + 4;              // floats per 8-row group
    static constexpr int LBO = 128;
    static constexpr int SBO = 4 * GS;
    static constexpr size_t XB = (size_t)(M / 8) * GS * 4, GB = (size_t)(NP / 8) * GS * 4;
    static constexpr size_t BARB = 64;                 // two mbarriers, the TMEM address, the MMA flag
    static constexpr size_t TABB = (size_t)(KP + M) * 4;   // patch-offset and block-offset tables
    // the region of u the CTA's blocks read (q the colour lattice's period): RW x RH floats
    __host__ __device__ static constexpr int RW(int q) { return q * (TBX - 1) + PW; }
    __host__ __device__ static constexpr int RH(int q) { return q * (TBY - 1) + PW; }
    __host__ __device__ static constexpr size_t smem(int q)
    {
        return XB + GB + BARB + TABB + (size_t)RW(q) * RH(q) * 4;
    }
};

// float offset of element (row r, k) in the operand layout
__host__ __device__ inline int tc_off(int r, int k, int kp)
{
    return (r / 8) * (8 * kp + 4) + (k / 4) * 32 + (r % 8) * 4 + (k % 4);
}

// instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

#ifdef __CUDACC__
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
#endif

}  // namespace iga2l
