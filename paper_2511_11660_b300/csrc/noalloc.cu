// noalloc.cu -- WNS/TNS reduction of endpoint slacks that allocates nothing.
//
// The regular path (sta_update_timing) folds endpoint slacks in two stages
// through a partial-sums buffer that sta_create allocates with cudaMalloc.
// This file offers the same reduction for callers that cannot allocate
// device memory themselves -- a host flow whose memory is entirely owned by
// another allocator that has already reserved the device, or a loop that
// cannot tolerate the implicit device synchronisation and possible failure
// of a cudaMalloc.  Its partial sums live in a fixed file-scope device array
// instead of a buffer, so it needs neither cudaMalloc nor cudaFree.
#include <atomic>
#include <cstdio>

#include "sta.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 4096;            // endpoints folded by one first-stage block
constexpr int kMaxSlots = 8192;         // chunks x corners held in the scratch array
constexpr int kMaxDevices = 64;

// Six partial values per (chunk, corner): negative-slack sums (setup, hold),
// worst slacks (setup, hold), violation counts (setup, hold).  384 KiB, held
// by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_partial[kMaxSlots * 6];

// Per-device address of g_partial, looked up at the first call on that
// device.  Atomic, so two host threads making their first call on one
// device at once both store the same address without a data race.  The
// cached address belongs to the device's primary context: it does not
// survive cudaDeviceReset (or a release of the primary context).
std::atomic<double *> g_partial_ptr[kMaxDevices] = {};

template <int NT>
__device__ __forceinline__ void fold6(double v[6], double (*sh)[NT])
{
#pragma unroll
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
            sh[3][threadIdx.x] = fmin(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
            sh[4][threadIdx.x] += sh[4][threadIdx.x + w];
            sh[5][threadIdx.x] += sh[5][threadIdx.x + w];
        }
        __syncthreads();
    }
}

// Stage 1: block (b, k) folds endpoints [b*kChunk, (b+1)*kChunk) of corner k.
// Every slot stage 2 reads is written here first, so nothing needs clearing.
__global__ void __launch_bounds__(kThreads)
k_na_chunks(const float *__restrict__ setup, const float *__restrict__ hold, long long E, int K, double *part)
{
    __shared__ double sh[6][kThreads];
    const int b = blockIdx.x, k = blockIdx.y;
    const long long e0 = (long long)b * kChunk, e1 = e0 + kChunk < E ? e0 + kChunk : E;
    double v[6] = {0, 0, INFINITY, INFINITY, 0, 0};
    for (long long e = e0 + threadIdx.x; e < e1; e += kThreads) {
        const double ss = setup[e * K + k], hs = hold[e * K + k];
        v[2] = fmin(v[2], ss);
        v[3] = fmin(v[3], hs);
        if (ss < 0) { v[0] += ss; v[4] += 1; }
        if (hs < 0) { v[1] += hs; v[5] += 1; }
    }
    fold6<kThreads>(v, sh);
    if (threadIdx.x < 6) part[((size_t)b * K + k) * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// Stage 2: one block per corner folds the chunks in a fixed order.
__global__ void __launch_bounds__(kThreads) k_na_final(const double *__restrict__ part, int nb, int K, double *out)
{
    __shared__ double sh[6][kThreads];
    const int k = blockIdx.x;
    double v[6] = {0, 0, INFINITY, INFINITY, 0, 0};
    for (int b = threadIdx.x; b < nb; b += kThreads) {
        const double *p = part + ((size_t)b * K + k) * 6;
        v[0] += p[0];
        v[1] += p[1];
        v[2] = fmin(v[2], p[2]);
        v[3] = fmin(v[3], p[3]);
        v[4] += p[4];
        v[5] += p[5];
    }
    fold6<kThreads>(v, sh);
    if (threadIdx.x == 0) {
        double *o = out + (size_t)k * 8;
        o[0] = fmin(0.0, sh[2][0]);
        o[1] = sh[0][0];
        o[2] = fmin(0.0, sh[3][0]);
        o[3] = sh[1][0];
        o[4] = sh[2][0];
        o[5] = sh[3][0];
        o[6] = sh[4][0];
        o[7] = sh[5][0];
    }
}

// Device address of g_partial on the current device, looked up once per
// device.  The name g_partial in host code is only a host-side stand-in.
cudaError_t partial_ptr(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    double *cached = g_partial_ptr[dev].load(std::memory_order_acquire);
    if (!cached) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partial);
        if (e != cudaSuccess) return e;
        cached = static_cast<double *>(p);
        g_partial_ptr[dev].store(cached, std::memory_order_release);
    }
    *out = cached;
    return cudaSuccess;
}

}  // namespace

extern "C" sta_status sta_reduce_slack_noalloc(const float *setup, const float *hold, int64_t n_endpoints,
                                               int32_t n_corners, double *out, void *stream)
{
    if (!setup || !hold || !out || n_endpoints < 0 || n_corners < 1) return STA_EINVAL;
    // Size check without overflow: bound n_endpoints before rounding it up to
    // chunks, then compare the chunk count against the slots per corner.
    const long long max_endpoints = (long long)kMaxSlots * kChunk;
    const long long nb = n_endpoints <= max_endpoints ? (n_endpoints + kChunk - 1) / kChunk : kMaxSlots + 1LL;
    if (nb > kMaxSlots / n_corners) {
        std::fprintf(stderr,
                     "sta_reduce_slack_noalloc: %lld endpoints x %d corners exceeds the fixed scratch "
                     "(at most %d chunks of %d endpoints times corners)\n",
                     (long long)n_endpoints, n_corners, kMaxSlots, kChunk);
        return STA_EINVAL;
    }
    double *part = nullptr;
    if (partial_ptr(&part) != cudaSuccess) return STA_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Launched through cudaLaunchKernel so that each launch's own status is
    // checked: an error left behind by unrelated earlier work is not taken
    // (or cleared) as this call's failure.
    long long E = n_endpoints;
    int K = n_corners, nbi = (int)nb;
    if (nb > 0) {
        void *args1[] = {(void *)&setup, (void *)&hold, (void *)&E, (void *)&K, (void *)&part};
        if (cudaLaunchKernel((const void *)k_na_chunks, dim3((unsigned)nb, (unsigned)n_corners), dim3(kThreads),
                             args1, 0, st) != cudaSuccess)
            return STA_ECUDA;
    }
    const double *cpart = part;
    void *args2[] = {(void *)&cpart, (void *)&nbi, (void *)&K, (void *)&out};
    if (cudaLaunchKernel((const void *)k_na_final, dim3((unsigned)n_corners), dim3(kThreads), args2, 0, st) !=
        cudaSuccess)
        return STA_ECUDA;
    return STA_OK;
}
