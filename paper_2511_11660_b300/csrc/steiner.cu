// steiner.cu -- rectilinear Steiner trees of the nets from pin positions
// (Sec. III, "Parasitics (RC) inputs": a placement flow hands over pin
// positions and unit R/C along x and y, and the engine builds Steiner-tree
// RC on the GPU before delay calculation).
//
// Every net is rebuilt at every update from the current positions.  Nets
// come sorted by pin count: nets of at most 8 pins (most of them) take one
// thread each with working storage in shared memory; larger nets take a warp
// each (the lanes share every scan, warp reductions keep the sequential tie
// rules) with working storage in global scratch.  The steps:
//   * integer nm coordinates: the float product x * 1000, rounded to the
//     nearest integer (ties to even), so every decision below is exact;
//   * Prim's rectilinear MST from the driver (keys and sources, O(n^2)):
//     the outside pin with the smallest (distance to the tree, pin index)
//     joins, attached to the earliest-added tree node at that distance;
//   * greedy median insertion (nets of at most kStMaxPins pins), on
//     adjacency bitsets: over every node u (ascending) and every pair of its
//     neighbours v < w, the Steiner point M = (median x, median y) of
//     {u, v, w} gains d(u,v) + d(u,w) - d(M,u) - d(M,v) - d(M,w); the largest
//     gain (the first in that order) is applied while positive, at most
//     2 (n - 1) times -- M at v or w reattaches, else a new node joins the
//     three -- and Steiner nodes left with <= 2 neighbours are removed
//     (lowest index first: a leaf is dropped, a pass-through is bridged);
//   * breadth-first numbering from the driver (neighbours ascending) writes
//     the RC tree that k_net_tree sweeps (a node at the same point as the
//     node it is reached from shares its RC node: no zero-length edges):
//     parent (local, before the child),
//     edge R = rx Lx + ry Ly, wire C = cx Lx + cy Ly split half at each end
//     (Lx, Ly in um), the node of every sink, the live node count and the
//     tree length in nm.
// Working storage per net holds 3 n nodes (pins and at most 2 (n - 1)
// created Steiner points); the tree has at most 2 n - 2 live nodes (every
// live Steiner node has >= 3 neighbours).
// Both bounds are checked at run time: a violation sets kErrBounds and the
// kernel stops writing.
#include <climits>

#include "device.cuh"
#include "kernels.h"

namespace sta {

namespace {

__device__ __forceinline__ long long to_nm(float x) { return __float2ll_rn(__fmul_rn(x, 1000.f)); }

__device__ __forceinline__ long long mdist(long long xa, long long ya, long long xb, long long yb)
{
    return llabs(xa - xb) + llabs(ya - yb);
}

__device__ __forceinline__ long long med3(long long a, long long b, long long c)
{
    return max(min(a, b), min(max(a, b), c));
}

// Working storage of one net: element i of every array at base[i * s]
// (s = 1: a row per net in global scratch; s = threads: a column per thread
// in shared memory, conflict-free).  Coordinates in TX (int64 in global,
// int32 in shared: |x| <= 1e9 nm), small indices in TI, adjacency rows of W
// words, and the RC node capacitances accumulated before they are written.
template <class TX, class TI>
struct Work {
    TX *X, *Y;
    long long *key;
    TI *src, *nid, *queue;
    unsigned *adj;
    float *cap;   // RC node capacitance (fF), 2 m entries
    int s, W;
    __device__ __forceinline__ long long x(int i) const { return X[i * s]; }
    __device__ __forceinline__ long long y(int i) const { return Y[i * s]; }
    __device__ __forceinline__ void set_xy(int i, long long a, long long b) const
    {
        X[i * s] = (TX)a;
        Y[i * s] = (TX)b;
    }
    __device__ __forceinline__ long long &k(int i) const { return key[i * s]; }
    __device__ __forceinline__ int sr(int i) const { return src[i * s]; }
    __device__ __forceinline__ void set_sr(int i, int v) const { src[i * s] = (TI)v; }
    __device__ __forceinline__ int id(int i) const { return nid[i * s]; }
    __device__ __forceinline__ void set_id(int i, int v) const { nid[i * s] = (TI)v; }
    __device__ __forceinline__ int qu(int i) const { return queue[i * s]; }
    __device__ __forceinline__ void set_qu(int i, int v) const { queue[i * s] = (TI)v; }
    __device__ __forceinline__ unsigned &wd(int i, int w) const { return adj[(i * W + w) * s]; }
    __device__ __forceinline__ float &cp(int i) const { return cap[i * s]; }
    __device__ __forceinline__ void link(int i, int j) const
    {
        wd(i, j >> 5) |= 1u << (j & 31);
        wd(j, i >> 5) |= 1u << (i & 31);
    }
    __device__ __forceinline__ void cut(int i, int j) const
    {
        wd(i, j >> 5) &= ~(1u << (j & 31));
        wd(j, i >> 5) &= ~(1u << (i & 31));
    }
    __device__ __forceinline__ int deg(int i) const
    {
        int d = 0;
        for (int w = 0; w < W; ++w) d += __popc(wd(i, w));
        return d;
    }
    __device__ __forceinline__ long long dist(int a, int b) const { return mdist(x(a), y(a), x(b), y(b)); }
};

// Breadth-first numbering from the driver and the RC arrays of item g's
// tree (N working nodes; without Steiner points the MST by its sources).
template <class TX, class TI>
__device__ void write_tree(const DevCtx &c, int g, int f0, int n, int N, bool steinerise, const Work<TX, TI> &w)
{
    const int n0 = c.rc_ptr[g], tcap = c.rc_ptr[g + 1] - n0;   // 2 m nodes
    for (int i = 0; i < N; ++i) w.set_id(i, -1);
    int head = 0, tail = 1, nodes = 1;   // queue of working nodes; RC nodes written
    w.set_qu(0, 0);
    w.set_id(0, 0);
    w.cp(0) = 0.f;
    c.st_parent[n0] = -1;
    c.st_R[n0] = 0.f;
    long long total = 0;
    const float rx = c.r_per_um, ry = c.r_per_um_y, cx = c.c_per_um, cy = c.c_per_um_y;
    // differentiable contexts: which pin carries each coordinate of node b
    // (the lowest one at that value; every coordinate is a pin's), and the
    // sign of b - a along it
    auto src_code = [&](int b, int a, bool along_y) -> int {
        const long long v = along_y ? w.y(b) : w.x(b), u = along_y ? w.y(a) : w.x(a);
        int j = 0;
        while (j < n && (along_y ? w.y(j) : w.x(j)) != v) ++j;
        if (j >= n) {   // not reached: medians of pin coordinates
            atomicOr(c.err, kErrBounds);
            j = 0;
        }
        return (j << 2) | ((v > u) - (v < u) + 1);
    };
    if (c.st_src) c.st_src[n0] = make_int2(1, 1);   // the driver, sign 0
    auto visit = [&](int a, int b) -> bool {
        if (w.id(b) >= 0) return true;
        w.set_qu(tail++, b);   // tail <= N <= cap: each working node is queued once
        const long long ax = llabs(w.x(b) - w.x(a)), ay = llabs(w.y(b) - w.y(a));
        const int ia = w.id(a);
        if (ax + ay == 0) {   // the same point: the same RC node (no zero-length edge)
            w.set_id(b, ia);
            return true;
        }
        if (nodes >= tcap) {   // not reached: <= 2 n - 2 live nodes
            atomicOr(c.err, kErrBounds);
            return false;
        }
        w.set_id(b, nodes);
        total += ax + ay;
        const float lx = 1e-3f * (float)ax, ly = 1e-3f * (float)ay;
        const float half = 0.5f * (cx * lx + cy * ly);
        c.st_parent[n0 + nodes] = ia;
        c.st_R[n0 + nodes] = rx * lx + ry * ly;
        if (c.st_src) c.st_src[n0 + nodes] = make_int2(src_code(b, a, false), src_code(b, a, true));
        w.cp(nodes) = half;
        w.cp(ia) += half;
        ++nodes;
        return true;
    };
    while (head < tail) {
        const int a = w.qu(head++);
        if (steinerise) {
            for (int q = 0; q < w.W; ++q)
                for (unsigned mk = w.wd(a, q); mk; mk &= mk - 1)
                    if (!visit(a, q * 32 + __ffs(mk) - 1)) return;
        } else {   // the MST by its sources: the parent (visited) and the children, ascending
            for (int b = 0; b < n; ++b)
                if (w.sr(b) == a && !visit(a, b)) return;
        }
    }
    for (int i = 0; i < nodes; ++i) c.st_C[n0 + i] = w.cp(i);
    for (int j = 1; j < n; ++j) c.st_fo_node[f0 + j - 1] = w.id(j);
    c.st_nlive[g] = nodes;
    c.st_wl[g] = total;
}

// The tree of item g's net (f0: first sink, m >= 1 sinks) in storage w.
template <class TX, class TI>
__device__ void steiner_net(const DevCtx &c, int g, int f0, int m, const Work<TX, TI> &w)
{
    const int n = m + 1, cap = 3 * n;
    // pins: 0 = the driver, 1..m = the sinks in net order
    {
        const int z = chk(c, item_out_pin(c, chk_type(c, c.item_type[g]), c.item_pin0[g]), c.P);
        const float2 p = pin_pos(c, z);
        w.set_xy(0, to_nm(p.x), to_nm(p.y));
        for (int j = 1; j < n; ++j) {
            const float2 q = pin_pos(c, chk(c, c.fo_pin[f0 + j - 1], c.P));
            w.set_xy(j, to_nm(q.x), to_nm(q.y));
        }
    }
    const bool steinerise = n <= kStMaxPins;
    if (steinerise)
        for (int i = 0; i < cap; ++i)
            for (int k = 0; k < w.W; ++k) w.wd(i, k) = 0u;

    // Prim from the driver; key = distance to the tree (-1 inside it)
    for (int u = 0; u < n; ++u) {
        w.k(u) = LLONG_MAX;
        w.set_sr(u, -1);
    }
    w.k(0) = -1;
    for (int step = 1, t = 0; step < n; ++step) {
        long long best = LLONG_MAX;
        int bu = -1;
        const long long xt = w.x(t), yt = w.y(t);
        for (int u = 0; u < n; ++u) {
            long long ku = w.k(u);
            if (ku < 0) continue;
            const long long d = mdist(w.x(u), w.y(u), xt, yt);
            if (d < ku) {
                ku = d;
                w.k(u) = d;
                w.set_sr(u, t);
            }
            if (ku < best) {
                best = ku;
                bu = u;
            }
        }
        w.k(bu) = -1;
        if (steinerise) w.link(bu, w.sr(bu));
        t = bu;
    }

    int N = n;   // working nodes: pins, then the Steiner points created
    if (steinerise) {
        for (int i = 0; i < n; ++i) w.set_id(i, 1);   // nid doubles as the live flag until the numbering
        for (int it = 0; it < 2 * (n - 1); ++it) {
            long long bg = 0;
            int bu = -1, bv = -1, bw = -1;
            for (int u = 0; u < N; ++u) {
                if (!w.id(u)) continue;
                const long long xu = w.x(u), yu = w.y(u);
                for (int wv = 0; wv < w.W; ++wv) {
                    unsigned mv = w.wd(u, wv);
                    while (mv) {
                        const int v = wv * 32 + __ffs(mv) - 1;
                        mv &= mv - 1;
                        const long long xv = w.x(v), yv = w.y(v);
                        const long long duv = mdist(xu, yu, xv, yv);
                        unsigned mw = mv;   // neighbours above v
                        for (int ww = wv;;) {
                            while (mw) {
                                const int q = ww * 32 + __ffs(mw) - 1;
                                mw &= mw - 1;
                                const long long xq = w.x(q), yq = w.y(q);
                                const long long mx = med3(xu, xv, xq), my = med3(yu, yv, yq);
                                const long long gain = duv + mdist(xu, yu, xq, yq) - mdist(mx, my, xu, yu) -
                                                       mdist(mx, my, xv, yv) - mdist(mx, my, xq, yq);
                                if (gain > bg) {
                                    bg = gain;
                                    bu = u;
                                    bv = v;
                                    bw = q;
                                }
                            }
                            if (++ww >= w.W) break;
                            mw = w.wd(u, ww);
                        }
                    }
                }
            }
            if (bg <= 0) break;
            const long long mx = med3(w.x(bu), w.x(bv), w.x(bw)), my = med3(w.y(bu), w.y(bv), w.y(bw));
            if (mx == w.x(bv) && my == w.y(bv)) {
                w.cut(bu, bw);
                w.link(bv, bw);
            } else if (mx == w.x(bw) && my == w.y(bw)) {
                w.cut(bu, bv);
                w.link(bw, bv);
            } else {
                if (N >= cap) {   // not reached: at most 2 (n - 1) insertions
                    atomicOr(c.err, kErrBounds);
                    return;
                }
                const int s = N++;
                w.set_xy(s, mx, my);
                w.set_id(s, 1);
                w.cut(bu, bv);
                w.cut(bu, bw);
                w.link(s, bu);
                w.link(s, bv);
                w.link(s, bw);
            }
            for (;;) {   // remove Steiner nodes with <= 2 neighbours, lowest index first
                int s = -1, dg = 0;
                for (int i = n; i < N; ++i)
                    if (w.id(i) && (dg = w.deg(i)) <= 2) {
                        s = i;
                        break;
                    }
                if (s < 0) break;
                int nb2[2] = {-1, -1}, k = 0;
                for (int q = 0; q < w.W; ++q)
                    for (unsigned mk = w.wd(s, q); mk; mk &= mk - 1) {
                        const int j = q * 32 + __ffs(mk) - 1;
                        if (k < 2) nb2[k] = j;
                        ++k;
                    }
                for (int q = 0; q < k && q < 2; ++q) w.cut(s, nb2[q]);
                if (dg == 2) w.link(nb2[0], nb2[1]);
                w.set_id(s, 0);
            }
        }
    }

    write_tree(c, g, f0, n, N, steinerise, w);
}

// Nets of at most kSmallPins pins: working storage in shared memory, one
// column per thread.
constexpr int kSmallPins = 8, kSmallCap = 3 * kSmallPins, kSmallThreads = 64;   // kSmallPins: plan.h kSteinerSmallPins

__global__ void __launch_bounds__(kSmallThreads) k_net_steiner_small(const DevCtx c)
{
    __shared__ int32_t s_x[kSmallCap * kSmallThreads], s_y[kSmallCap * kSmallThreads];
    __shared__ long long s_key[kSmallPins * kSmallThreads];
    __shared__ int8_t s_src[kSmallPins * kSmallThreads], s_nid[kSmallCap * kSmallThreads],
        s_q[kSmallCap * kSmallThreads];
    __shared__ unsigned s_adj[kSmallCap * kSmallThreads];
    __shared__ float s_cap[2 * (kSmallPins - 1) * kSmallThreads];
    const int t = threadIdx.x, i = blockIdx.x * kSmallThreads + t;
    if (i >= c.st_small) return;
    const int g = chk(c, c.st_items[i], c.I);
    const int f0 = c.fo_ptr[g], m = c.fo_ptr[g + 1] - f0;
    if (m <= 0 || m + 1 > kSmallPins) return;   // not reached: the plan's split
    const Work<int32_t, int8_t> w{s_x + t, s_y + t, s_key + t, s_src + t, s_nid + t, s_q + t, s_adj + t, s_cap + t,
                                  kSmallThreads, 1};
    steiner_net(c, g, f0, m, w);
}

// Larger nets: one warp per net, working storage in global scratch (one
// row per net).  The lanes share the O(n) scans of every step -- Prim's key
// updates, the gains of every (node, neighbour pair) -- and a warp reduction
// picks the step's choice with the sequential order's tie rule; lane 0
// applies it.  The result is the one steiner_net builds.
constexpr int kWarpNets = 4;   // warps (nets) per block

__device__ __forceinline__ void warp_min_key(long long &k, int &u)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, k, off);
        const int ou = __shfl_xor_sync(0xffffffffu, u, off);
        if (ok < k || (ok == k && ou < u)) {
            k = ok;
            u = ou;
        }
    }
}

// One warp's storage in shared memory, for nets of at most kStMaxPins pins.
constexpr int kWarpCap = 3 * kStMaxPins, kWarpW = (kWarpCap + 31) / 32;
struct WarpSmem {
    int32_t x[kWarpCap], y[kWarpCap];
    long long key[kStMaxPins];
    int16_t src[kStMaxPins], nid[kWarpCap], q[kWarpCap];
    unsigned adj[kWarpCap * kWarpW];
    float cap[2 * kStMaxPins];
};

template <class TX, class TI>
__device__ void warp_net(const DevCtx &c, int g, int f0, int n, int lane, const Work<TX, TI> &w);

__global__ void __launch_bounds__(32 * kWarpNets) k_net_steiner_warp(const DevCtx c)
{
    __shared__ WarpSmem sm[kWarpNets];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int i = c.st_small + blockIdx.x * kWarpNets + wi;
    if (i >= c.st_n_items) return;   // the whole warp
    const int g = chk(c, c.st_items[i], c.I);
    const int f0 = c.fo_ptr[g], m = c.fo_ptr[g + 1] - f0;
    const int n = m + 1, cap = 3 * n;
    if (n <= kStMaxPins) {   // working storage in shared memory
        WarpSmem &S = sm[wi];
        const Work<int32_t, int16_t> w{S.x, S.y, S.key, S.src, S.nid, S.q, S.adj, S.cap, 1, (cap + 31) >> 5};
        warp_net(c, g, f0, n, lane, w);
    } else {                 // the MST of a large net, in global scratch
        const long long nb = c.st_node_ptr[g];
        int32_t *aux = c.st_aux + 3 * nb;
        const Work<long long, int32_t> w{c.st_x + nb, c.st_y + nb, c.st_key + nb, aux, aux + cap, aux + 2 * cap,
                                         nullptr, c.st_capw + nb, 1, (cap + 31) >> 5};
        warp_net(c, g, f0, n, lane, w);
    }
}

template <class TX, class TI>
__device__ void warp_net(const DevCtx &c, int g, int f0, int n, int lane, const Work<TX, TI> &w)
{
    const int cap = 3 * n;
    const bool steinerise = n <= kStMaxPins;
    // pins (0 = the driver, then the sinks in net order), keys, adjacency
    for (int j = lane; j < n; j += 32) {
        const int p = j == 0 ? chk(c, item_out_pin(c, chk_type(c, c.item_type[g]), c.item_pin0[g]), c.P)
                             : chk(c, c.fo_pin[f0 + j - 1], c.P);
        const float2 q = pin_pos(c, p);
        w.set_xy(j, to_nm(q.x), to_nm(q.y));
        w.k(j) = j == 0 ? -1 : LLONG_MAX;
        w.set_sr(j, -1);
    }
    if (steinerise)
        for (int x = lane; x < cap * w.W; x += 32) w.adj[x] = 0u;
    __syncwarp();
    // Prim: lane l owns the pins u = l (mod 32); the next pin by (key, u)
    for (int step = 1, t = 0; step < n; ++step) {
        const long long xt = w.x(t), yt = w.y(t);
        long long best = LLONG_MAX;
        int bu = INT_MAX;
        for (int u = lane; u < n; u += 32) {
            long long ku = w.k(u);
            if (ku < 0) continue;
            const long long d = mdist(w.x(u), w.y(u), xt, yt);
            if (d < ku) {
                ku = d;
                w.k(u) = d;
                w.set_sr(u, t);
            }
            if (ku < best) {
                best = ku;
                bu = u;
            }
        }
        warp_min_key(best, bu);
        if (lane == (bu & 31)) {   // the owner of bu holds its key and source
            w.k(bu) = -1;
            if (steinerise) w.link(bu, w.sr(bu));
        }
        __syncwarp();
        t = bu;
    }
    int N = n;
    if (steinerise) {
        for (int u = lane; u < n; u += 32) w.set_id(u, 1);
        __syncwarp();
        for (int it = 0; it < 2 * (n - 1); ++it) {
            long long bg = 0;
            int bu = INT_MAX, bv = -1, bw = -1;
            for (int u = lane; u < N; u += 32) {
                if (!w.id(u)) continue;
                const long long xu = w.x(u), yu = w.y(u);
                for (int wv = 0; wv < w.W; ++wv) {
                    unsigned mv = w.wd(u, wv);
                    while (mv) {
                        const int v = wv * 32 + __ffs(mv) - 1;
                        mv &= mv - 1;
                        const long long xv = w.x(v), yv = w.y(v);
                        const long long duv = mdist(xu, yu, xv, yv);
                        unsigned mw = mv;
                        for (int ww = wv;;) {
                            while (mw) {
                                const int q = ww * 32 + __ffs(mw) - 1;
                                mw &= mw - 1;
                                const long long xq = w.x(q), yq = w.y(q);
                                const long long mx = med3(xu, xv, xq), my = med3(yu, yv, yq);
                                const long long gain = duv + mdist(xu, yu, xq, yq) - mdist(mx, my, xu, yu) -
                                                       mdist(mx, my, xv, yv) - mdist(mx, my, xq, yq);
                                if (gain > bg) {
                                    bg = gain;
                                    bu = u;
                                    bv = v;
                                    bw = q;
                                }
                            }
                            if (++ww >= w.W) break;
                            mw = w.wd(u, ww);
                        }
                    }
                }
            }
            // the largest gain, ties: the lowest u (each lane's u are ascending)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const long long og = __shfl_xor_sync(0xffffffffu, bg, off);
                const int ou = __shfl_xor_sync(0xffffffffu, bu, off), ov = __shfl_xor_sync(0xffffffffu, bv, off),
                          ow = __shfl_xor_sync(0xffffffffu, bw, off);
                if (og > bg || (og == bg && ou < bu)) {
                    bg = og;
                    bu = ou;
                    bv = ov;
                    bw = ow;
                }
            }
            if (bg <= 0) break;
            int err = 0;
            if (lane == 0) {
                const long long mx = med3(w.x(bu), w.x(bv), w.x(bw)), my = med3(w.y(bu), w.y(bv), w.y(bw));
                if (mx == w.x(bv) && my == w.y(bv)) {
                    w.cut(bu, bw);
                    w.link(bv, bw);
                } else if (mx == w.x(bw) && my == w.y(bw)) {
                    w.cut(bu, bv);
                    w.link(bw, bv);
                } else if (N >= cap) {   // not reached: at most 2 (n - 1) insertions
                    atomicOr(c.err, kErrBounds);
                    err = 1;
                } else {
                    const int s = N++;
                    w.set_xy(s, mx, my);
                    w.set_id(s, 1);
                    w.cut(bu, bv);
                    w.cut(bu, bw);
                    w.link(s, bu);
                    w.link(s, bv);
                    w.link(s, bw);
                }
            }
            N = __shfl_sync(0xffffffffu, N, 0);
            if (__shfl_sync(0xffffffffu, err, 0)) return;
            __syncwarp();
            for (;;) {   // remove Steiner nodes with <= 2 neighbours, lowest index first (lanes scan)
                int s = INT_MAX;
                for (int x = n + lane; x < N; x += 32)
                    if (w.id(x) && w.deg(x) <= 2) {
                        s = x;
                        break;
                    }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) s = min(s, __shfl_xor_sync(0xffffffffu, s, off));
                if (s == INT_MAX) break;
                if (lane == 0) {
                    int nb2[2] = {-1, -1}, k = 0;
                    for (int q = 0; q < w.W; ++q)
                        for (unsigned mk = w.wd(s, q); mk; mk &= mk - 1) {
                            const int j = q * 32 + __ffs(mk) - 1;
                            if (k < 2) nb2[k] = j;
                            ++k;
                        }
                    for (int q = 0; q < k && q < 2; ++q) w.cut(s, nb2[q]);
                    if (k == 2) w.link(nb2[0], nb2[1]);
                    w.set_id(s, 0);
                }
                __syncwarp();
            }
        }
    }
    if (lane == 0) write_tree(c, g, f0, n, N, steinerise, w);   // lane 0, as steiner_net does
}

}  // namespace

void launch_net_steiner(const DevCtx &c, cudaStream_t st)
{
    // the nets by increasing pin count, so that a warp's nets take alike work
    if (c.st_small > 0)
        k_net_steiner_small<<<(c.st_small + kSmallThreads - 1) / kSmallThreads, kSmallThreads, 0, st>>>(c);
    const int big = c.st_n_items - c.st_small;
    if (big > 0) k_net_steiner_warp<<<(big + kWarpNets - 1) / kWarpNets, 32 * kWarpNets, 0, st>>>(c);
}

}  // namespace sta
