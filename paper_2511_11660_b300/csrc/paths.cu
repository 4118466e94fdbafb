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

// Fan-in candidates of gate output p at edge rf in state k, in tie order
// (input slot, then rise before fall): the input pin, its edge and its late
// arrival + NLDM delay (the forward pass's FP32 candidate arithmetic).
// Returns how many (at most 6).
template <bool UNIFORM>
__device__ int gate_cands(const DevCtx &c, int k, int t, int pin0, int p, int rf, int *ca, int *crf, float *cv)
{
    const int K = c.K;
    const int nin = __ldg(c.type_nin + t);
    const LutGlobal lut{c.lut, c.lut_scale};
    const float sc = __ldg(c.lut_scale + k);
    const float ld = c.load[(size_t)p * K + k];
    const Seg bl = seg_load<UNIFORM>(c, lut, tab_off(t, 0, 0), ld);
    int n = 0;
    for (int jn = 0; jn < nin; ++jn) {
        const int a = pin0 + jn;
        const int se = __ldg(c.arc_sense + t * 3 + jn);
        const int tbj = tab_off(t, jn, 0);
        for (int rfi = 0; rfi < 2; ++rfi) {
            if (!arc_on(se, rfi, rf)) continue;
            const float s = ld_state(c.slew + (size_t)a * K + k, 2 + rfi);
            const Seg as = seg_slew<UNIFORM>(c, lut, tbj, s);
            const float dv = lookup<UNIFORM>(lut, tbj + rf * kLutStride, as, bl, s, ld);
            ca[n] = a;
            crf[n] = rfi;
            cv[n] = ld_state_df(c.at + (size_t)a * K + k, 2 + rfi).hi + sc * dv;
            ++n;
        }
    }
    return n;
}

// the critical candidate: the largest (the first of equals)
__device__ __forceinline__ int cand_best(const float *cv, int n)
{
    int b = 0;
    for (int i = 1; i < n; ++i)
        if (cv[i] > cv[b]) b = i;
    return b;
}

// Kind of node p for the trace: 0 startpoint, 1 net sink (to the driver),
// 2 flip-flop Q (to CK, rising), 3 gate output (t, pin0 set).
__device__ __forceinline__ int node_kind(const DevCtx &c, const PathJob &j, int p, int &t, int &pin0)
{
    if (c.drv_of[p] >= 0) return 1;
    const int g = j.pin_item[p];
    if (g < 0) return 0;
    t = c.item_type[g];
    pin0 = c.item_pin0[g];
    if (t < 0) return 0;                               // PI
    if (__ldg(c.type_kind + t) == 1) return p == pin0 ? 0 : 2;   // CK / Q
    return 3;
}

// One step of the trace back from pin p at edge rf in state k; false at a
// startpoint.  Through a -through pin the path may come from the previous
// tag's state: the one whose late arrival is larger (ties: the same tag).
template <bool UNIFORM>
__device__ bool trace_step(const DevCtx &c, const PathJob &j, int &k, int &p, int &rf)
{
    const int K = c.K;
    int t = -1, pin0 = 0;
    const int kind = node_kind(c, j, p, t, pin0);
    if (kind == 1) {   // net sink
        const int drv = c.drv_of[p];
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
    if (kind == 0) return false;
    if (kind == 2) {
        p = pin0;                                   // Q -> CK, rising edge
        rf = 0;
        return true;
    }
    int ca[6], crf[6];
    float cv[6];
    const int n = gate_cands<UNIFORM>(c, k, t, pin0, p, rf, ca, crf, cv);
    if (n == 0) return false;
    const int b = cand_best(cv, n);
    p = ca[b];
    rf = crf[b];
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

// ------------------------------------------ per-endpoint limit above 1
//
// A path at an endpoint is its end edge plus the gate outputs where it
// leaves the critical fan-in of trace_step: leaving output (p, rf) for
// candidate i costs dv = cand(critical) - cand(i) >= 0, and the path's slack
// is the end edge's slack plus its dvs.  The "region" of a path is the
// critical chain above its last deviation's input pin (above the endpoint
// for a root), walked from there; its deviations are ordered by (dv, node
// position in the walk, candidate index).  One thread per selected endpoint
// runs a best-first search: both end edges start as roots; popping path x
// (the cheapest pending) accepts it and pushes x's best child (the first
// deviation of x's region) and x's next sibling (the deviation after x's
// own in its parent's region).  Every deviation set is generated once and
// in increasing slack, so the first per_ep pops are the endpoint's
// per_ep worst paths.  A region is re-walked for each push (the walk is
// the critical trace, so nothing is stored per pin).

struct Dev {
    float dv;
    int pos, alt, p, a, rf, rfi;
};

__device__ __forceinline__ bool dev_less(float d1, int p1, int a1, float d2, int p2, int a2)
{
    return d1 < d2 || (d1 == d2 && (p1 < p2 || (p1 == p2 && a1 < a2)));
}

// The deviation of smallest (dv, pos, alt) strictly after (d0, pos0, alt0)
// in the region walked from node (p, rf).
template <bool UNIFORM>
__device__ bool region_next(const DevCtx &c, const PathJob &j, int k, int p, int rf, float d0, int pos0, int alt0,
                            Dev &best)
{
    bool found = false;
    for (int pos = 0; pos < j.max_len; ++pos) {
        int t = -1, pin0 = 0;
        const int kind = node_kind(c, j, p, t, pin0);
        if (kind == 0) break;
        if (kind == 1) {
            p = c.drv_of[p];
            continue;
        }
        if (kind == 2) {
            p = pin0;
            rf = 0;
            continue;
        }
        int ca[6], crf[6];
        float cv[6];
        const int n = gate_cands<UNIFORM>(c, k, t, pin0, p, rf, ca, crf, cv);
        if (n == 0) break;
        const int b = cand_best(cv, n);
        for (int i = 0; i < n; ++i) {
            const float dv = cv[b] - cv[i];
            if (i == b || !(dv >= 0.f)) continue;   // the critical one; NaN (no arrival on either)
            if (dev_less(d0, pos0, alt0, dv, pos, i) && (!found || dev_less(dv, pos, i, best.dv, best.pos, best.alt))) {
                best = Dev{dv, pos, i, p, ca[i], rf, crf[i]};
                found = true;
            }
        }
        p = ca[b];
        rf = crf[b];
    }
    return found;
}

// the search of one selected endpoint (thread i): records and merge keys
template <bool UNIFORM>
__global__ void k_path_nworst(const DevCtx c, const PathJob j)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int)*j.count) return;
    const int L = j.per_ep, k = j.corner;   // one state per corner (no exception tags)
    PathRec *rec = j.recs + (size_t)i * L;
    const int pe = c.ep_pin[j.e0 + (int)(j.keys[i] & 0xffffffffu)];
    PathRec heap[kMaxPerEndpoint + 2];
    int nh = 0;
    for (int rf = 0; rf < 2; ++rf)
        heap[nh++] = PathRec{ld_state(c.slack + (size_t)pe * c.K + k, 2 + rf), 0.f, -1, pe, -1, rf, 0, rf, -1};
    int nrec = 0;
    while (nh > 0 && nrec < L) {
        int b = 0;
        for (int h = 1; h < nh; ++h)
            if (heap[h].cost < heap[b].cost) b = h;
        const PathRec cur = heap[b];
        heap[b] = heap[--nh];
        if (!(cur.cost < j.slack_lt)) break;
        const int r = nrec++;
        rec[r] = cur;
        Dev d;
        const bool root = cur.parent < 0;
        if (region_next<UNIFORM>(c, j, k, root ? cur.p : cur.a, root ? cur.rf : cur.rfi, -INFINITY, -1, -1, d) &&
            nh < kMaxPerEndpoint + 2)
            heap[nh++] = PathRec{cur.cost + d.dv, d.dv, r, d.p, d.a, d.rf, d.rfi, d.pos, d.alt};
        if (!root) {
            const PathRec par = rec[cur.parent];
            const bool proot = par.parent < 0;
            if (region_next<UNIFORM>(c, j, k, proot ? par.p : par.a, proot ? par.rf : par.rfi, cur.dv, cur.pos,
                                     cur.alt, d) &&
                nh < kMaxPerEndpoint + 2)
                heap[nh++] = PathRec{par.cost + d.dv, d.dv, cur.parent, d.p, d.a, d.rf, d.rfi, d.pos, d.alt};
        }
    }
    for (int r = 0; r < L; ++r)
        j.pkeys[(size_t)i * L + r] =
            r < nrec ? ((unsigned long long)ordered_bits(rec[r].cost) << 32) | ((unsigned)i << 5) | (unsigned)r : ~0ull;
}

// Bitonic sort of the selected endpoints' keys in one block (dynamic shared
// memory of a power of two >= their number); the paths reported are the
// first min(k, found) of them.
__global__ void __launch_bounds__(1024) k_nw_sort(const PathJob j)
{
    extern __shared__ unsigned long long s_k[];
    const int m = (int)*j.count * j.per_ep;
    int n2 = 1;
    while (n2 < m) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) s_k[i] = i < m ? j.pkeys[i] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int p = i ^ stride;
                if (p > i) {
                    const bool up = (i & size) == 0;
                    if ((s_k[i] > s_k[p]) == up) {
                        const unsigned long long t = s_k[i];
                        s_k[i] = s_k[p];
                        s_k[p] = t;
                    }
                }
            }
            __syncthreads();
        }
    __shared__ int s_valid;
    if (threadIdx.x == 0) s_valid = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < min(m, j.k); i += blockDim.x) {
        j.pkeys[i] = s_k[i];
        if (s_k[i] != ~0ull) atomicAdd(&s_valid, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *j.count = (unsigned)s_valid;   // valid keys come first
}

// Output path q: its endpoint, end edge, slack and deviations from the
// endpoint upward.
struct NwPath {
    int pe, erf, nd;
    float cost;
    int dp[kMaxPerEndpoint], drf[kMaxPerEndpoint], da[kMaxPerEndpoint], darf[kMaxPerEndpoint];
    float ddv[kMaxPerEndpoint];
};

__device__ void nw_path(const PathJob &j, int q, NwPath &w)
{
    const unsigned long long key = j.pkeys[q];
    const int i = (int)((key >> 5) & 0x7ffffffu), r = (int)(key & 31u);
    const PathRec *rec = j.recs + (size_t)i * j.per_ep;
    w.cost = rec[r].cost;
    int n = 0, x = r;
    while (rec[x].parent >= 0 && n < kMaxPerEndpoint) {   // highest deviation first
        w.dp[n] = rec[x].p;
        w.drf[n] = rec[x].rf;
        w.da[n] = rec[x].a;
        w.darf[n] = rec[x].rfi;
        w.ddv[n] = rec[x].dv;
        ++n;
        x = rec[x].parent;
    }
    for (int a = 0, b = n - 1; a < b; ++a, --b) {   // lowest (nearest the endpoint) first
        const int t0 = w.dp[a], t1 = w.drf[a], t2 = w.da[a], t3 = w.darf[a];
        const float t4 = w.ddv[a];
        w.dp[a] = w.dp[b]; w.drf[a] = w.drf[b]; w.da[a] = w.da[b]; w.darf[a] = w.darf[b]; w.ddv[a] = w.ddv[b];
        w.dp[b] = t0; w.drf[b] = t1; w.da[b] = t2; w.darf[b] = t3; w.ddv[b] = t4;
    }
    w.nd = n;
    w.pe = rec[x].p;
    w.erf = rec[x].rf;
}

// one step of path w from (p, rf): its deviation there, else the critical fan-in
template <bool UNIFORM>
__device__ __forceinline__ bool nw_step(const DevCtx &c, const PathJob &j, const NwPath &w, int &di, int &p, int &rf)
{
    if (di < w.nd && p == w.dp[di] && rf == w.drf[di]) {
        p = w.da[di];
        rf = w.darf[di];
        ++di;
        return true;
    }
    int k = j.corner;
    return trace_step<UNIFORM>(c, j, k, p, rf);
}

template <bool UNIFORM>
__global__ void k_nw_len(const DevCtx c, const PathJob j)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int)*j.count) return;
    NwPath w;
    nw_path(j, q, w);
    int p = w.pe, rf = w.erf, di = 0, len = 1;
    while (len < j.max_len && nw_step<UNIFORM>(c, j, w, di, p, rf)) ++len;
    j.ptr[q + 1] = len;
}

// the pins from the endpoint backwards; the path's arrival at a pin is the
// analysis' late arrival less the deviations taken at or above it
template <bool UNIFORM>
__global__ void k_nw_write(const DevCtx c, const PathJob j)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int)*j.count) return;
    NwPath w;
    nw_path(j, q, w);
    float rem = 0.f;
    for (int i = 0; i < w.nd; ++i) rem += w.ddv[i];
    const int b = j.ptr[q];
    int wpos = j.ptr[q + 1] - 1;
    int p = w.pe, rf = w.erf, di = 0;
    j.slack[q] = w.cost;
    j.endpoint[q] = j.caller_pin[p];
    while (wpos >= b) {
        j.pin[wpos] = j.caller_pin[p];
        j.rf[wpos] = (int8_t)rf;
        j.at[wpos] = to_f(ld_state_df(c.at + (size_t)p * c.K + j.corner, 2 + rf)) - rem;
        --wpos;
        const bool dev = di < w.nd && p == w.dp[di] && rf == w.drf[di];
        const float dvh = dev ? w.ddv[di] : 0.f;
        if (!nw_step<UNIFORM>(c, j, w, di, p, rf)) break;
        rem -= dvh;
    }
}

}  // namespace

static void launch_select(const DevCtx &c, const PathJob &j, cudaStream_t st)
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
}

void launch_report_paths_nworst(const DevCtx &c, const HostSched &h, const PathJob &j, cudaStream_t st)
{
    launch_select(c, j, st);
    const int tb = (j.k + 63) / 64;
    if (h.uniform) k_path_nworst<true><<<tb, 64, 0, st>>>(c, j);
    else k_path_nworst<false><<<tb, 64, 0, st>>>(c, j);
    int n2 = 1;
    while (n2 < j.k * j.per_ep) n2 <<= 1;
    const size_t smem = (size_t)n2 * sizeof(unsigned long long);
    cudaFuncSetAttribute(k_nw_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_nw_sort<<<1, 1024, smem, st>>>(j);
    const int tp = (j.k + 127) / 128;
    if (h.uniform) k_nw_len<true><<<tp, 128, 0, st>>>(c, j);
    else k_nw_len<false><<<tp, 128, 0, st>>>(c, j);
    k_path_scan<<<1, 1024, 0, st>>>(j);
    if (h.uniform) k_nw_write<true><<<tp, 128, 0, st>>>(c, j);
    else k_nw_write<false><<<tp, 128, 0, st>>>(c, j);
}

void launch_report_paths(const DevCtx &c, const HostSched &h, const PathJob &j, cudaStream_t st)
{
    launch_select(c, j, st);
    const int tb = (j.k + 127) / 128;
    if (h.uniform) k_path_len<true><<<tb, 128, 0, st>>>(c, j);
    else k_path_len<false><<<tb, 128, 0, st>>>(c, j);
    k_path_scan<<<1, 1024, 0, st>>>(j);
    if (h.uniform) k_path_write<true><<<tb, 128, 0, st>>>(c, j);
    else k_path_write<false><<<tb, 128, 0, st>>>(c, j);
}

}  // namespace sta
