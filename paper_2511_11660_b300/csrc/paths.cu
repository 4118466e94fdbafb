// paths.cu -- top-k path report (Sec. III "Report options": top-k paths with
// a slack threshold and a per-endpoint limit, as flattened CSR path arrays).
//
// Per-endpoint limit 1: the k endpoints of one design with the worst setup
// slack at one corner below a threshold, in increasing slack (ties: lower
// endpoint index), each with its critical path.  The path is traced back from
// the endpoint at the edge with the smaller late slack (ties: rise):
//   a net sink steps to its net's driver with the same edge;
//   a gate output steps to the input arc whose late arrival + NLDM delay
//     (the forward pass's FP32 candidate, same arithmetic) is largest (ties: lower
//     input slot, then rise before fall);
//   a flip-flop Q steps to its CK (rising edge);
//   the trace stops at a PI or CK.
//
// Selection is exact and deterministic: keys are (order-preserving slack bits,
// endpoint index), unique 64-bit integers; a most-significant-digit radix
// select (8 passes of 8 bits, histograms with shared then global atomics,
// the digit chosen on the device) finds the k-th smallest key, the keys up
// to it are compacted and sorted by a bitonic sort in one block.
#include "item.cuh"
#include "kernels.h"

namespace sta {

namespace {

constexpr int kSelThreads = 256;

__device__ __forceinline__ unsigned ordered_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // increasing float -> increasing unsigned
}

__device__ __forceinline__ bool key_of(const DevCtx &c, const PathJob &j, int i, unsigned long long &key)
{
    float s = INFINITY;   // the endpoint's slack at the corner: min over exception tags
    for (int g = 0; g < c.Tg; ++g) s = fminf(s, c.ep_setup[(size_t)(j.e0 + i) * c.K + j.corner * c.Tg + g]);
    if (!(s < j.slack_lt)) return false;   // also drops NaN
    key = ((unsigned long long)ordered_bits(s) << 32) | (unsigned)i;
    return true;
}

// Histogram of digit `pass` (8 bits from the top) of the eligible keys whose
// higher digits equal the prefix found so far.
__global__ void __launch_bounds__(kSelThreads) k_sel_hist(const DevCtx c, const PathJob j, int pass)
{
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int shift = 56 - 8 * pass;
    const unsigned long long prefix = j.sel[0], mask = pass ? (~0ull << (shift + 8)) : 0ull;
    for (int i = blockIdx.x * kSelThreads + threadIdx.x; i < j.n; i += gridDim.x * kSelThreads) {
        unsigned long long key;
        if (key_of(c, j, i, key) && (key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(j.hist + threadIdx.x, h[threadIdx.x]);
}

// One thread: extend the prefix by the digit where the running count reaches
// the remaining rank, and clear the histogram for the next pass.  sel[0]
// prefix, sel[1] remaining rank (1-based), sel[2] keys taken (eligible count
// when it is below k).
__global__ void k_sel_pick(const PathJob j, int pass)
{
    if (threadIdx.x != 0) return;
    const int shift = 56 - 8 * pass;
    unsigned long long rem = j.sel[1], acc = 0;
    int d = 0;
    for (; d < 256; ++d) {
        if (acc + j.hist[d] >= rem) break;
        acc += j.hist[d];
    }
    if (d == 256) d = 255;   // fewer eligible keys than the rank: take them all
    j.sel[0] |= (unsigned long long)d << shift;
    j.sel[1] = rem - acc;
    for (int i = 0; i < 256; ++i) j.hist[i] = 0u;
}

// The eligible keys up to the k-th, appended in any order (sorted next).
__global__ void __launch_bounds__(kSelThreads) k_sel_compact(const DevCtx c, const PathJob j)
{
    for (int i = blockIdx.x * kSelThreads + threadIdx.x; i < j.n; i += gridDim.x * kSelThreads) {
        unsigned long long key;
        if (key_of(c, j, i, key) && key <= j.sel[0]) {
            const unsigned at = atomicAdd(j.count, 1u);
            if (at < (unsigned)j.k) j.keys[at] = key;
        }
    }
}

// Bitonic sort of the selected keys (at most kMaxPaths) in one block.
__global__ void __launch_bounds__(1024) k_sel_sort(const PathJob j)
{
    __shared__ unsigned long long s[kMaxPaths];
    const int m = min((int)*j.count, j.k);
    int n2 = 1;
    while (n2 < m) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) s[i] = i < m ? j.keys[i] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int p = i ^ stride;
                if (p > i) {
                    const bool up = (i & size) == 0;
                    if ((s[i] > s[p]) == up) {
                        const unsigned long long t = s[i];
                        s[i] = s[p];
                        s[p] = t;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < m; i += blockDim.x) j.keys[i] = s[i];
    if (threadIdx.x == 0) *j.count = (unsigned)m;
}

// One step of the trace back from pin p at edge rf in state k; false at a
// startpoint.  Through a -through pin the path may come from the previous
// tag's state: the one whose late arrival is larger (ties: the same tag).
template <bool UNIFORM>
__device__ bool trace_step(const DevCtx &c, const PathJob &j, int &k, int &p, int &rf)
{
    const int K = c.K;
    const int drv = c.drv_of[p];
    if (drv >= 0) {   // net sink
        if (c.pin_adv) {
            const uint32_t adv = c.pin_adv[p];
            const int tg = k % c.Tg;
            const bool stay = !((adv >> tg) & 1u), inflow = tg >= 1 && ((adv >> (tg - 1)) & 1u);
            if (inflow && (!stay || ld_state_df(c.at + (size_t)drv * K + k - 1, 2 + rf) >
                                        ld_state_df(c.at + (size_t)drv * K + k, 2 + rf)))
                --k;
        }
        p = drv;
        return true;
    }
    const int g = j.pin_item[p];
    if (g < 0) return false;
    const int t = c.item_type[g], pin0 = c.item_pin0[g];
    if (t < 0) return false;                        // PI
    const int kind = __ldg(c.type_kind + t), nin = __ldg(c.type_nin + t);
    if (kind == 1) {
        if (p == pin0) return false;                // CK
        p = pin0;                                   // Q -> CK, rising edge
        rf = 0;
        return true;
    }
    const LutGlobal lut{c.lut};
    const float sc = __ldg(c.lut_scale + k);
    const float ld = c.load[(size_t)p * K + k];
    const Seg bl = seg_load<UNIFORM>(c, lut, tab_off(t, 0, 0), ld);
    float best = -INFINITY;
    int bp = -1, brf = 0;
    for (int jn = 0; jn < nin; ++jn) {
        const int a = pin0 + jn;
        const int se = __ldg(c.arc_sense + t * 3 + jn);
        const int tbj = tab_off(t, jn, 0);
        for (int rfi = 0; rfi < 2; ++rfi) {
            if (!arc_on(se, rfi, rf)) continue;
            const float s = ld_state(c.slew + (size_t)a * K + k, 2 + rfi);
            const Seg as = seg_slew<UNIFORM>(c, lut, tbj, s);
            const float dv = lookup<UNIFORM>(lut, tbj + rf * kLutStride, as, bl, s, ld);
            const float cand = ld_state_df(c.at + (size_t)a * K + k, 2 + rfi).hi + sc * dv;
            if (cand > best || bp < 0) {
                best = cand;
                bp = a;
                brf = rfi;
            }
        }
    }
    if (bp < 0) return false;
    p = bp;
    rf = brf;
    return true;
}

// the endpoint, and the (exception tag, edge) state with its smallest late
// slack (ties: lower tag, then rise): the path is traced in that state
__device__ __forceinline__ void path_start(const DevCtx &c, const PathJob &j, int i, int &e, int &p, int &k, int &rf)
{
    e = j.e0 + (int)(j.keys[i] & 0xffffffffu);
    p = c.ep_pin[e];
    float best = INFINITY;
    k = j.corner * c.Tg;
    rf = 0;
    for (int g = 0; g < c.Tg; ++g) {
        const int kk = j.corner * c.Tg + g;
        const size_t o = (size_t)p * c.K + kk;
        const float s0 = ld_state(c.slack + o, 2), s1 = ld_state(c.slack + o, 3);
        const float s = fminf(s0, s1);
        if (s < best) {
            best = s;
            k = kk;
            rf = s0 <= s1 ? 0 : 1;
        }
    }
    if (!(best < INFINITY)) {   // no checked state (cannot be selected): tag 0
        const size_t o = (size_t)p * c.K + k;
        rf = ld_state(c.slack + o, 2) <= ld_state(c.slack + o, 3) ? 0 : 1;
    }
}

// pass 1: path lengths (pins, endpoint and startpoint included)
template <bool UNIFORM>
__global__ void k_path_len(const DevCtx c, const PathJob j)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int)*j.count) return;
    int e, p, k, rf;
    path_start(c, j, i, e, p, k, rf);
    int len = 1;
    while (len < j.max_len && trace_step<UNIFORM>(c, j, k, p, rf)) ++len;
    j.ptr[i + 1] = len;
}

// exclusive scan of the lengths (one block)
__global__ void __launch_bounds__(1024) k_path_scan(const PathJob j)
{
    __shared__ int s[kMaxPaths + 1];
    const int m = (int)*j.count;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s[i] = j.ptr[i + 1];
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        j.ptr[0] = 0;
        for (int i = 0; i < m; ++i) {
            acc += s[i];
            j.ptr[i + 1] = acc;
        }
    }
}

// pass 2: the pins, from the endpoint backwards into [ptr[i], ptr[i+1])
template <bool UNIFORM>
__global__ void k_path_write(const DevCtx c, const PathJob j)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int)*j.count) return;
    int e, p, k, rf;
    path_start(c, j, i, e, p, k, rf);
    const int b = j.ptr[i];
    int w = j.ptr[i + 1] - 1;
    float es = INFINITY;
    for (int g = 0; g < c.Tg; ++g) es = fminf(es, c.ep_setup[(size_t)e * c.K + j.corner * c.Tg + g]);
    j.slack[i] = es;
    j.endpoint[i] = j.caller_pin[p];
    for (;;) {
        if (w < b) break;
        j.pin[w] = j.caller_pin[p];
        j.rf[w] = (int8_t)rf;
        j.at[w] = to_f(ld_state_df(c.at + (size_t)p * c.K + k, 2 + rf));
        --w;
        if (!trace_step<UNIFORM>(c, j, k, p, rf)) break;
    }
}

}  // namespace

void launch_report_paths(const DevCtx &c, const HostSched &h, const PathJob &j, cudaStream_t st)
{
    const int nb = std::max(1, std::min(1024, (j.n + kSelThreads - 1) / kSelThreads));
    if (j.n > 0) {
        for (int pass = 0; pass < 8; ++pass) {
            k_sel_hist<<<nb, kSelThreads, 0, st>>>(c, j, pass);
            k_sel_pick<<<1, 32, 0, st>>>(j, pass);
        }
        k_sel_compact<<<nb, kSelThreads, 0, st>>>(c, j);
    }
    k_sel_sort<<<1, 1024, 0, st>>>(j);
    const int tb = (j.k + 127) / 128;
    if (h.uniform) k_path_len<true><<<tb, 128, 0, st>>>(c, j);
    else k_path_len<false><<<tb, 128, 0, st>>>(c, j);
    k_path_scan<<<1, 1024, 0, st>>>(j);
    if (h.uniform) k_path_write<true><<<tb, 128, 0, st>>>(c, j);
    else k_path_write<false><<<tb, 128, 0, st>>>(c, j);
}

}  // namespace sta
