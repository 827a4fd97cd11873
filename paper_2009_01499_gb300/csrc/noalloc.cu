// noalloc.cu -- residual norm for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs where the CUDA
// allocator is off limits (for example a hard real-time loop, or a host
// runtime that owns every device allocation itself and only hands out the
// buffers it manages).  Such a caller cannot create a solver handle, because
// iga2l_assemble allocates the handle's tables and workspace.  This file gives
// it one entry point, iga2l_residual_norm2_noalloc, that computes the defect
// d = b - A_p u and its squared 2-norm from caller-provided buffers only.
//
// The only scratch it needs, one partial sum per thread block, lives in the
// file-scope array g_noalloc_partials below: a fixed 512 KiB that every GPU
// which loads this library holds until the process exits.  Host code cannot
// pass the array's name to a kernel (on the host it is only a stand-in, not a
// device address), so the first call on each device looks up the array's
// device address with cudaGetSymbolAddress while that device is current and
// caches it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace iga2l {

namespace {

constexpr int kNoAllocMaxPartials = 65536;   // 512 KiB of doubles
constexpr int kNoAllocTX = 32, kNoAllocTY = 8;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// d = b - A u with A = K (x) M + M (x) K taken directly from the band rows
// (row x of K, M: Kb[x*(2P+1) + a] couples DOF x with x+a-P).  One partial sum of
// d^2 per thread block into part[].
template <int P>
__global__ void __launch_bounds__(kNoAllocTX *kNoAllocTY)
k_residual2d_bands(int n, const double *__restrict__ Kb, const double *__restrict__ Mb,
                   const double *__restrict__ u, const double *__restrict__ b, double *__restrict__ d,
                   double *__restrict__ part)
{
    constexpr int W = 2 * P + 1;
    constexpr int SX = kNoAllocTX + 2 * P, SY = kNoAllocTY + 2 * P;
    __shared__ double su[SY][SX];
    __shared__ double red[kNoAllocTX * kNoAllocTY / 32];
    const int x0 = blockIdx.x * kNoAllocTX, y0 = blockIdx.y * kNoAllocTY;
    const int tid = threadIdx.x + kNoAllocTX * threadIdx.y;
    for (int t = tid; t < SX * SY; t += kNoAllocTX * kNoAllocTY) {
        const int ly = t / SX, lx = t % SX;
        const int gx = x0 + lx - P, gy = y0 + ly - P;
        su[ly][lx] = (gx >= 0 && gx < n && gy >= 0 && gy < n) ? u[(size_t)gy * n + gx] : 0.0;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    double dv = 0.0;
    if (x < n && y < n) {
        const double *kx = Kb + (size_t)x * W, *mx = Mb + (size_t)x * W;
        const double *ky = Kb + (size_t)y * W, *my = Mb + (size_t)y * W;
        double acc = 0.0;
#pragma unroll
        for (int bb = 0; bb < W; ++bb) {
            double sk = 0.0, sm = 0.0;   // row sums against K and M in x
#pragma unroll
            for (int aa = 0; aa < W; ++aa) {
                const double v = su[threadIdx.y + bb][threadIdx.x + aa];
                sk = fma(kx[aa], v, sk);
                sm = fma(mx[aa], v, sm);
            }
            acc = fma(my[bb], sk, acc);
            acc = fma(ky[bb], sm, acc);
        }
        dv = b[(size_t)y * n + x] - acc;
        if (d) d[(size_t)y * n + x] = dv;
    }
    double s = dv * dv;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < kNoAllocTX * kNoAllocTY / 32; ++w) tot += red[w];
        part[blockIdx.x + gridDim.x * blockIdx.y] = tot;
    }
}

// out[0] = sum of part[0..np), fixed order
__global__ void k_noalloc_sum(const double *__restrict__ part, int np, double *__restrict__ out)
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

// Device address of g_noalloc_partials for the current device (looked up once).
cudaError_t partials_for_current_device(double **ptr)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return cudaSuccess;
}

template <int P>
void launch_noalloc(int n, const double *Kb, const double *Mb, const double *u, const double *b,
                    double *d, double *part, double *norm2, cudaStream_t st)
{
    dim3 blk(kNoAllocTX, kNoAllocTY), grd((n + kNoAllocTX - 1) / kNoAllocTX, (n + kNoAllocTY - 1) / kNoAllocTY);
    k_residual2d_bands<P><<<grd, blk, 0, st>>>(n, Kb, Mb, u, b, d, part);
    count_launches(1);
    k_noalloc_sum<<<1, 1024, 0, st>>>(part, (int)(grd.x * grd.y), norm2);
    count_launches(1);
}

}  // namespace

}  // namespace iga2l

extern "C" int iga2l_residual_norm2_noalloc(int p, int n, const double *Kb, const double *Mb,
                                            const double *u, const double *b, double *d,
                                            double *norm2, void *stream)
{
    using namespace iga2l;
    if (p < 2 || p > 5 || n < 1 || !Kb || !Mb || !u || !b || !norm2) {
        set_last_error("residual_norm2_noalloc: p must be 2..5, n >= 1 and Kb, Mb, u, b, norm2 non-null");
        return IGA2L_ERR_INVALID_ARG;
    }
    // sizes checked in 64-bit arithmetic, so that no n near INT_MAX can wrap around
    const long long nl = n;
    const long long nparts = ((nl + kNoAllocTX - 1) / kNoAllocTX) * ((nl + kNoAllocTY - 1) / kNoAllocTY);
    if (nl > 4096 || nparts > kNoAllocMaxPartials) {
        set_last_error("residual_norm2_noalloc: n = " + std::to_string(n) +
                       " exceeds the fixed scratch (at most 4096 DOFs per axis)");
        return IGA2L_ERR_INVALID_ARG;
    }
    double *part = nullptr;
    cudaError_t e = partials_for_current_device(&part);
    if (e != cudaSuccess) {
        set_last_error(std::string("residual_norm2_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return IGA2L_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (p) {
    case 2: launch_noalloc<2>(n, Kb, Mb, u, b, d, part, norm2, st); break;
    case 3: launch_noalloc<3>(n, Kb, Mb, u, b, d, part, norm2, st); break;
    case 4: launch_noalloc<4>(n, Kb, Mb, u, b, d, part, norm2, st); break;
    default: launch_noalloc<5>(n, Kb, Mb, u, b, d, part, norm2, st); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("residual_norm2_noalloc: ") + cudaGetErrorString(e));
        return IGA2L_ERR_CUDA;
    }
    return IGA2L_OK;
}
