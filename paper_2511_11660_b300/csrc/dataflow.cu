// dataflow.cu -- persistent dataflow schedule of the timing pass.
//
// Instead of one launch per level, each pass is one persistent kernel.  Its
// warps take chunks of at most 8 / KL items of one level in level order (the
// backward pass in reverse level order) from an atomic counter and run each
// item in a slot of 4 * KL lanes (KL = corners side by side) as soon as the
// mailbox entries of the items it reads are complete -- polled without
// blocking, with a bounded number of idle rounds -- and publish its results
// to the mailbox of this pass's epoch parity (item.cuh).  Items are handed
// out in increasing order and an item only waits for earlier ones, so the
// oldest unfinished item can always proceed: no grid barrier and no
// co-residency assumption.  The cell library (tables and per-type
// data) is copied into shared memory once per block.
#include <algorithm>

#include "item.cuh"
#include "kernels.h"

namespace sta {

constexpr int kDfThreads = 256;

static inline size_t df_smem_bytes(int T) { return smem_lib_bytes(T); }

// After an aborted pass the mailboxes hold a mix of parities: reset them
// all to NaN.  (A completed pass leaves the next parity all NaN.)
__global__ void k_df_recover(const DevCtx c)
{
    if (ld_volatile(c.df_state + 3) == 0u) return;
    const float4 nan4 = make_float4(nan_f(), nan_f(), nan_f(), nan_f());
    DF4 nand;
    for (int q = 0; q < 4; ++q) nand.v[q] = nan_df();
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.fbox_len; i += stride) {
        c.fbox_a[i] = nand;
        c.fbox_s[i] = nan4;
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.rbox_len; i += stride) c.rbox[i] = nand;
}

// New epoch, chunk counters at zero, abort cleared.
__global__ void k_df_begin(const DevCtx c)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c.df_state[0] = c.df_state[0] + 1u;
        c.df_state[1] = 0u;
        c.df_state[2] = 0u;
        c.df_state[3] = 0u;
    }
}

// Next chunk for this warp (lane 0 takes it, all lanes get it); -1 when the
// queue is empty or the pass was aborted.
__device__ __forceinline__ int next_chunk(const DevCtx &c, int counter, int n_chunks)
{
    int ch = 0;
    if ((threadIdx.x & 31) == 0) ch = (int)atomicAdd(c.df_state + counter, 1u);
    const unsigned aborted = ld_volatile(c.df_state + 3);   // read while the claim is in flight
    ch = __shfl_sync(0xffffffffu, ch, 0);
    if (ch >= n_chunks) return -1;
    if (aborted) return -1;
    return ch;
}

// The warp's polling loop.  Every pending item of the chunk probes its
// inputs' mailbox entries without blocking; items whose inputs are complete
// run at once, so one late input holds back only its own item.  A warp
// gives up after c.spin_limit idle rounds (timeout bit + abort word), or as
// soon as another warp has aborted.
__device__ __forceinline__ bool warp_idle_round(const DevCtx &c, long long &spins)
{
    if (++spins >= c.spin_limit) {
        if ((threadIdx.x & 31) == 0) {
            atomicOr(c.err, kErrTimeout);
            atomicExch(c.df_state + 3, 1u);
        }
        return false;
    }
    if ((spins & 31) == 0 && __any_sync(0xffffffffu, ld_volatile(c.df_state + 3) != 0u)) return false;
    __nanosleep(32);
    return true;
}

// Two blocks a SM (at most 128 registers a thread): the item slots in flight
// set the pace at 1M cells, so no build may grow past them.
template <bool SMOOTH, bool UNIFORM, bool THRU, class Ctx = DevCtx>
__global__ void __launch_bounds__(kDfThreads, 2) k_df_forward(const Ctx c)
{
    extern __shared__ float smem[];
    const SmemLib L = stage_library(c, smem);
    const int par = (int)(ld_volatile(c.df_state) & 1u);
    const int lane = threadIdx.x & 31, q = lane & 3;
    for (;;) {
        const int ch = next_chunk(c, 1, c.n_fwd_chunks);
        if (ch < 0) break;
        const int x = c.fwd_chunk_lo[ch] + lane / (4 * nKL(c));
        bool pending = x < c.fwd_chunk_hi[ch];
        FwdItem f{};
        if (pending) f = fwd_prep<true>(c, L.nin, L.kind, L.sense, x);
        long long spins = 0;
        FwdIn in;
        unsigned seen = 0;   // inputs found complete (values kept in `in`)
        while (__any_sync(0xffffffffu, pending)) {
            bool ok = false;
            if (pending) ok = fwd_probe<THRU, true>(c, f, par, q, in, &seen);
            if (group_all_warp(c, ok) && pending) {   // the whole warp votes
                fwd_run<SMOOTH, UNIFORM, true, THRU, true>(c, L.lut, f, in, x, q, par);
                pending = false;
            }
            if (__any_sync(0xffffffffu, pending) && !warp_idle_round(c, spins)) break;
        }
    }
}

template <bool UNIFORM, bool THRU, class Ctx = DevCtx>
__global__ void __launch_bounds__(kDfThreads, 2) k_df_backward(const Ctx c)
{
    extern __shared__ float smem[];
    const SmemLib L = stage_library(c, smem);
    const int par = (int)(ld_volatile(c.df_state) & 1u);
    const int lane = threadIdx.x & 31, q = lane & 3;
    for (;;) {
        const int ch = next_chunk(c, 2, c.n_bwd_chunks);
        if (ch < 0) break;
        const int pos = c.bwd_chunk_lo[ch] + lane / (4 * nKL(c));
        bool pending = pos < c.bwd_chunk_hi[ch];
        const int x = pending ? chk(c, c.bwd_order[chk(c, pos, c.I)], c.I) : 0;
        BwdItem b{};
        if (pending) b = bwd_prep(c, L.nin, L.kind, x, q);
        long long spins = 0;
        while (__any_sync(0xffffffffu, pending)) {
            Fold4 fo;
            bool ok = false;
            if (pending) ok = bwd_probe_split<THRU>(c, b, par, q, fo);
            else fold4_clear(fo);
            const bool go = group_all_warp(c, ok) && pending;   // the whole warp votes
            if (__any_sync(0xffffffffu, go)) {
                // every lane folds (full-warp shuffles); the ready groups use it
                const DF Rz = quad_fold(fo, q, 0xffffffffu);
                if (go) {
                    bwd_run<UNIFORM, true, THRU>(c, L.lut, L.sense, b, q, par, Rz);
                    pending = false;
                }
            }
            if (__any_sync(0xffffffffu, pending) && !warp_idle_round(c, spins)) break;
        }
    }
}

template <class F>
static cudaError_t occupancy_blocks(F kernel, size_t smem, int *blocks)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kDfThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *blocks = per_sm * sms;
    return cudaSuccess;
}

size_t dataflow_smem_bytes(int T) { return df_smem_bytes(T); }

// The persistent kernels for a schedule: smoothed merges, shared table axes,
// and -through sets each select a compiled variant.
using DfKernel = void (*)(DevCtx);
static DfKernel df_forward_kernel(bool smooth, bool uniform, bool thru)
{
    if (thru) return smooth ? (uniform ? k_df_forward<true, true, true> : k_df_forward<true, false, true>)
                            : (uniform ? k_df_forward<false, true, true> : k_df_forward<false, false, true>);
    return smooth ? (uniform ? k_df_forward<true, true, false> : k_df_forward<true, false, false>)
                  : (uniform ? k_df_forward<false, true, false> : k_df_forward<false, false, false>);
}
static DfKernel df_backward_kernel(bool uniform, bool thru)
{
    if (thru) return uniform ? k_df_backward<true, true> : k_df_backward<false, true>;
    return uniform ? k_df_backward<true, false> : k_df_backward<false, false>;
}
// the builds for one state a pin (DevCtxOne; no -through sets then)
using DfKernelOne = void (*)(DevCtxOne);
static DfKernelOne df_forward_kernel_one(bool smooth, bool uniform)
{
    return smooth ? (uniform ? k_df_forward<true, true, false, DevCtxOne> : k_df_forward<true, false, false, DevCtxOne>)
                  : (uniform ? k_df_forward<false, true, false, DevCtxOne> : k_df_forward<false, false, false, DevCtxOne>);
}
static DfKernelOne df_backward_kernel_one(bool uniform)
{
    return uniform ? k_df_backward<true, false, DevCtxOne> : k_df_backward<false, false, DevCtxOne>;
}

// Shared-memory attribute and persistent grid sizes, computed outside any
// stream capture.  `requested` > 0 fixes the grid size.
cudaError_t dataflow_prepare(HostSched &h, bool smooth, int requested)
{
    const size_t smem = df_smem_bytes(h.T);
    int bf = 0, bb = 0;
    cudaError_t e;
    if (h.one) {
        e = occupancy_blocks(df_forward_kernel_one(smooth, h.uniform), smem, &bf);
        if (e == cudaSuccess) e = occupancy_blocks(df_backward_kernel_one(h.uniform), smem, &bb);
    } else {
        e = occupancy_blocks(df_forward_kernel(smooth, h.uniform, h.thru), smem, &bf);
        if (e == cudaSuccess) e = occupancy_blocks(df_backward_kernel(h.uniform, h.thru), smem, &bb);
    }
    if (e != cudaSuccess) return e;
    h.df_blocks_fwd = requested > 0 ? std::min(requested, bf) : bf;
    h.df_blocks_bwd = requested > 0 ? std::min(requested, bb) : bb;
    return cudaSuccess;
}

// ------------------------------------------------------- cooperative schedule
//
// Level-synchronous, but without a kernel boundary per level: one launch
// whose blocks are all resident (cooperative launch) walks the forward
// levels, the endpoints and the backward levels, and a grid-wide barrier
// separates consecutive levels.  Inside a level, warp w of W takes items
// (w + r W) * 8/KL + lane / (4 KL), r = 0, 1, ...; the per-item arithmetic is
// that of the level kernels (item.cuh, pin states read from L2).

// Barrier arrivals accumulate in df_state[7] (reset before the launch), so
// the n-th barrier of a pass completes at n * gridDim.x arrivals.  One thread
// per block arrives (after a device-scope fence over the block's writes)
// and polls; the poll is bounded and any block that gives up, or sees that
// another one gave up, raises the abort word and leaves the kernel.
__device__ __forceinline__ bool grid_barrier(const DevCtx &c, unsigned &target, int *abort_flag)
{
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        int ab = 0;
        __threadfence();
        atomicAdd(c.df_state + 7, 1u);
        long long spins = 0;
        while (ld_volatile(c.df_state + 7) < target) {
            if (++spins >= c.spin_limit) {
                atomicOr(c.err, kErrTimeout);
                atomicExch(c.df_state + 3, 1u);
                ab = 1;
                break;
            }
            if ((spins & 15) == 0 && ld_volatile(c.df_state + 3) != 0u) {
                ab = 1;
                break;
            }
        }
        __threadfence();
        *abort_flag = ab;
    }
    __syncthreads();
    return *abort_flag == 0;
}

// Barrier count and abort word at zero.  (The dataflow epoch is left alone:
// its mailbox parities stay consistent across schedule changes.)
__global__ void k_coop_begin(const DevCtx c)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c.df_state[3] = 0u;
        c.df_state[7] = 0u;
    }
}

// Four blocks a SM (64 registers a thread): a level's items are independent
// after the barrier, so more warps in flight hide more load latency (64
// designs x 4 corners: 14.6 -> 11.9 ms an update).
template <bool SMOOTH, bool UNIFORM>
__global__ void __launch_bounds__(kDfThreads, 4) k_coop_pass(const DevCtx c)
{
    extern __shared__ float smem[];
    __shared__ int abort_flag;
    const SmemLib L = stage_library(c, smem);
    const int lane = threadIdx.x & 31, q = lane & 3;
    const int per = 8 / c.KL;                          // items per warp
    const int sub = lane / (4 * c.KL);                 // this lane's item inside the warp's group
    const int W = gridDim.x * (kDfThreads / 32);
    const int w = blockIdx.x * (kDfThreads / 32) + (threadIdx.x >> 5);
    unsigned target = 0;
    for (int s = 0; s < c.S; ++s) {
        const int i0 = __ldg(c.stage_ptr + s), i1 = __ldg(c.stage_ptr + s + 1);
        for (int g = i0 + w * per + sub; g < i1; g += W * per) {
            const FwdItem f = fwd_prep(c, L.nin, L.kind, L.sense, g);
            fwd_run<SMOOTH, UNIFORM, false>(c, L.lut, f, FwdIn{}, g, q, 0);
        }
        if (!grid_barrier(c, target, &abort_flag)) return;
    }
    for (int e = w * per + sub; e < c.E; e += W * per) ep_run<false>(c, ep_prep(c, e), 0.f, 0.f, e, q, 0);
    if (!grid_barrier(c, target, &abort_flag)) return;
    for (int s = c.S - 1; s >= 0; --s) {
        const int i0 = __ldg(c.stage_ptr + s), i1 = __ldg(c.stage_ptr + s + 1);
        for (int g = i0 + w * per + sub; g < i1; g += W * per)
            bwd_run<UNIFORM, false>(c, L.lut, L.sense, bwd_prep(c, L.nin, L.kind, g, q), q, 0, 0.f);
        if (s > 0 && !grid_barrier(c, target, &abort_flag)) return;
    }
}

template <bool SMOOTH, bool UNIFORM>
static cudaError_t coop_launch(const DevCtx &c, int blocks, size_t smem, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kDfThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_coop_pass<SMOOTH, UNIFORM>, c);
}

cudaError_t coop_prepare(HostSched &h, bool smooth, int requested)
{
    const size_t smem = df_smem_bytes(h.T);
    auto k = smooth ? (h.uniform ? k_coop_pass<true, true> : k_coop_pass<true, false>)
                    : (h.uniform ? k_coop_pass<false, true> : k_coop_pass<false, false>);
    int dev = 0, coop = 0, blocks = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess && !coop) e = cudaErrorNotSupported;
    if (e == cudaSuccess) e = occupancy_blocks(k, smem, &blocks);
    if (e != cudaSuccess) return e;
    h.coop_blocks = requested > 0 ? std::min(requested, blocks) : blocks;
    return cudaSuccess;
}

void launch_coop_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev)
{
    const size_t smem = df_smem_bytes(h.T);
    if (ev) cudaEventRecord(ev[0], st);
    k_coop_begin<<<1, 32, 0, st>>>(c);
    launch_net_phase(c, h, st);
    if (ev) cudaEventRecord(ev[1], st);
    if (c.I > 0 || c.E > 0) {
        if (c.gamma > 0.f) {
            if (h.uniform) coop_launch<true, true>(c, h.coop_blocks, smem, st);
            else coop_launch<true, false>(c, h.coop_blocks, smem, st);
        } else {
            if (h.uniform) coop_launch<false, true>(c, h.coop_blocks, smem, st);
            else coop_launch<false, false>(c, h.coop_blocks, smem, st);
        }
    }
    // forward and backward share one launch: the phase events after it
    // coincide (the profile attributes the whole launch to the forward slot)
    if (ev) cudaEventRecord(ev[2], st);
    if (ev) cudaEventRecord(ev[3], st);
    launch_reduce(c, h, st);
    if (ev) cudaEventRecord(ev[4], st);
}

void launch_df_reset(const DevCtx &c, int blocks, cudaStream_t st)
{
    k_df_recover<<<blocks > 0 ? blocks : 1, kDfThreads, 0, st>>>(c);
    k_df_begin<<<1, 32, 0, st>>>(c);
}

void launch_dataflow_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev)
{
    const size_t smem = df_smem_bytes(h.T);
    if (ev) cudaEventRecord(ev[0], st);
    launch_df_reset(c, h.df_blocks_fwd, st);
    launch_net_phase(c, h, st);
    if (ev) cudaEventRecord(ev[1], st);
    const DevCtxOne c1{c};   // the same context, for the one-state builds
    if (c.n_fwd_chunks > 0) {
        if (h.one) df_forward_kernel_one(c.gamma > 0.f, h.uniform)<<<h.df_blocks_fwd, kDfThreads, smem, st>>>(c1);
        else df_forward_kernel(c.gamma > 0.f, h.uniform, h.thru)<<<h.df_blocks_fwd, kDfThreads, smem, st>>>(c);
    }
    launch_endpoints(c, st);   // every driver is final: no polling
    if (ev) cudaEventRecord(ev[2], st);
    if (c.n_bwd_chunks > 0) {
        if (h.one) df_backward_kernel_one(h.uniform)<<<h.df_blocks_bwd, kDfThreads, smem, st>>>(c1);
        else df_backward_kernel(h.uniform, h.thru)<<<h.df_blocks_bwd, kDfThreads, smem, st>>>(c);
    }
    if (ev) cudaEventRecord(ev[3], st);
    launch_reduce(c, h, st);
    if (ev) cudaEventRecord(ev[4], st);
}

}  // namespace sta
