// steiner.cu -- rectilinear Steiner trees of the nets from pin positions
// (Sec. III, "Parasitics (RC) inputs": a placement flow hands over pin
// positions and unit R/C along x and y, and the engine builds Steiner-tree
// RC on the GPU before delay calculation).
//
// One thread per net (an item with sinks), rebuilt at every update from the
// current positions:
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
// Working storage per net lives in global scratch sized by the plan (3 n
// nodes: pins and at most 2 (n - 1) created Steiner points); the tree has at
// most 2 n - 2 live nodes (every live Steiner node has >= 3 neighbours).
// Both bounds are checked at run time: a violation sets kErrBounds and the
// kernel stops writing.
#include <climits>

#include "device.cuh"
#include "kernels.h"

namespace sta {

namespace {

constexpr int kSteinerThreads = 128;

__device__ __forceinline__ long long to_nm(float x) { return __float2ll_rn(__fmul_rn(x, 1000.f)); }

__device__ __forceinline__ long long mdist(long long xa, long long ya, long long xb, long long yb)
{
    return llabs(xa - xb) + llabs(ya - yb);
}

__device__ __forceinline__ long long med3(long long a, long long b, long long c)
{
    return max(min(a, b), min(max(a, b), c));
}

// adjacency rows of W words per node
struct Bits {
    unsigned *a;
    int W;
    __device__ __forceinline__ unsigned *row(int i) const { return a + (size_t)i * W; }
    __device__ __forceinline__ void link(int i, int j) const
    {
        row(i)[j >> 5] |= 1u << (j & 31);
        row(j)[i >> 5] |= 1u << (i & 31);
    }
    __device__ __forceinline__ void cut(int i, int j) const
    {
        row(i)[j >> 5] &= ~(1u << (j & 31));
        row(j)[i >> 5] &= ~(1u << (i & 31));
    }
    __device__ __forceinline__ int deg(int i) const
    {
        int d = 0;
        for (int w = 0; w < W; ++w) d += __popc(row(i)[w]);
        return d;
    }
};

__global__ void __launch_bounds__(kSteinerThreads) k_net_steiner(const DevCtx c)
{
    const int g = blockIdx.x * kSteinerThreads + threadIdx.x;
    if (g >= c.I) return;
    const int f0 = c.fo_ptr[g], m = c.fo_ptr[g + 1] - f0;
    if (m <= 0) return;
    const int n = m + 1, cap = 3 * n;
    const long long nb = c.st_node_ptr[g];
    long long *X = c.st_x + nb, *Y = c.st_y + nb, *key = c.st_key + nb;
    int32_t *src = c.st_aux + 3 * nb, *nid = src + cap, *queue = nid + cap;

    // pins: 0 = the driver, 1..m = the sinks in net order
    {
        const int z = chk(c, item_out_pin(c, chk_type(c, c.item_type[g]), c.item_pin0[g]), c.P);
        const float2 p = pin_pos(c, z);
        X[0] = to_nm(p.x);
        Y[0] = to_nm(p.y);
        for (int j = 1; j < n; ++j) {
            const float2 q = pin_pos(c, chk(c, c.fo_pin[f0 + j - 1], c.P));
            X[j] = to_nm(q.x);
            Y[j] = to_nm(q.y);
        }
    }
    const bool steinerise = n <= kStMaxPins;
    const Bits B{steinerise ? c.st_adj + c.st_adj_ptr[g] : nullptr, (cap + 31) >> 5};
    if (steinerise)
        for (int i = 0; i < cap * B.W; ++i) B.a[i] = 0u;

    // Prim from the driver; key = distance to the tree (-1 inside it)
    for (int u = 0; u < n; ++u) {
        key[u] = LLONG_MAX;
        src[u] = -1;
    }
    key[0] = -1;
    for (int step = 1, t = 0; step < n; ++step) {
        long long best = LLONG_MAX;
        int bu = -1;
        for (int u = 0; u < n; ++u) {
            if (key[u] < 0) continue;
            const long long d = mdist(X[u], Y[u], X[t], Y[t]);
            if (d < key[u]) {
                key[u] = d;
                src[u] = t;
            }
            if (key[u] < best) {
                best = key[u];
                bu = u;
            }
        }
        key[bu] = -1;
        if (steinerise) B.link(bu, src[bu]);
        t = bu;
    }

    int N = n;   // working nodes: pins, then the Steiner points created
    if (steinerise) {
        for (int i = 0; i < n; ++i) nid[i] = 1;   // nid doubles as the live flag until the numbering
        for (int it = 0; it < 2 * (n - 1); ++it) {
            long long bg = 0;
            int bu = -1, bv = -1, bw = -1;
            for (int u = 0; u < N; ++u) {
                if (!nid[u]) continue;
                const unsigned *r = B.row(u);
                for (int wv = 0; wv < B.W; ++wv) {
                    unsigned mv = r[wv];
                    while (mv) {
                        const int v = wv * 32 + __ffs(mv) - 1;
                        mv &= mv - 1;
                        const long long duv = mdist(X[u], Y[u], X[v], Y[v]);
                        unsigned mw = mv;   // neighbours above v
                        for (int ww = wv;;) {
                            while (mw) {
                                const int w = ww * 32 + __ffs(mw) - 1;
                                mw &= mw - 1;
                                const long long mx = med3(X[u], X[v], X[w]), my = med3(Y[u], Y[v], Y[w]);
                                const long long gain = duv + mdist(X[u], Y[u], X[w], Y[w]) - mdist(mx, my, X[u], Y[u]) -
                                                       mdist(mx, my, X[v], Y[v]) - mdist(mx, my, X[w], Y[w]);
                                if (gain > bg) {
                                    bg = gain;
                                    bu = u;
                                    bv = v;
                                    bw = w;
                                }
                            }
                            if (++ww >= B.W) break;
                            mw = r[ww];
                        }
                    }
                }
            }
            if (bg <= 0) break;
            const long long mx = med3(X[bu], X[bv], X[bw]), my = med3(Y[bu], Y[bv], Y[bw]);
            if (mx == X[bv] && my == Y[bv]) {
                B.cut(bu, bw);
                B.link(bv, bw);
            } else if (mx == X[bw] && my == Y[bw]) {
                B.cut(bu, bv);
                B.link(bw, bv);
            } else {
                if (N >= cap) {   // not reached: at most 2 (n - 1) insertions
                    atomicOr(c.err, kErrBounds);
                    return;
                }
                const int s = N++;
                X[s] = mx;
                Y[s] = my;
                nid[s] = 1;
                B.cut(bu, bv);
                B.cut(bu, bw);
                B.link(s, bu);
                B.link(s, bv);
                B.link(s, bw);
            }
            for (;;) {   // remove Steiner nodes with <= 2 neighbours, lowest index first
                int s = -1, dg = 0;
                for (int i = n; i < N; ++i)
                    if (nid[i] && (dg = B.deg(i)) <= 2) {
                        s = i;
                        break;
                    }
                if (s < 0) break;
                int nb2[2] = {-1, -1}, k = 0;
                for (int w = 0; w < B.W; ++w)
                    for (unsigned mk = B.row(s)[w]; mk; mk &= mk - 1) {
                        const int j = w * 32 + __ffs(mk) - 1;
                        if (k < 2) nb2[k] = j;
                        ++k;
                    }
                for (int q = 0; q < k && q < 2; ++q) B.cut(s, nb2[q]);
                if (dg == 2) B.link(nb2[0], nb2[1]);
                nid[s] = 0;
            }
        }
    }

    // breadth-first numbering from the driver -> the RC tree of the net
    const int n0 = c.rc_ptr[g], tcap = c.rc_ptr[g + 1] - n0;   // 2 m nodes
    for (int i = 0; i < N; ++i) nid[i] = -1;
    int head = 0, tail = 1, nodes = 1;   // queue of working nodes; RC nodes written
    queue[0] = 0;
    nid[0] = 0;
    c.st_parent[n0] = -1;
    c.st_R[n0] = 0.f;
    c.st_C[n0] = 0.f;
    long long total = 0;
    const float rx = c.r_per_um, ry = c.r_per_um_y, cx = c.c_per_um, cy = c.c_per_um_y;
    auto visit = [&](int a, int b) -> bool {
        if (nid[b] >= 0) return true;
        queue[tail++] = b;   // tail <= N <= cap: each working node is queued once
        const long long ax = llabs(X[b] - X[a]), ay = llabs(Y[b] - Y[a]);
        if (ax + ay == 0) {   // the same point: the same RC node (no zero-length edge)
            nid[b] = nid[a];
            return true;
        }
        if (nodes >= tcap) {   // not reached: <= 2 n - 2 live nodes
            atomicOr(c.err, kErrBounds);
            return false;
        }
        nid[b] = nodes;
        total += ax + ay;
        const float lx = 1e-3f * (float)ax, ly = 1e-3f * (float)ay;
        const float half = 0.5f * (cx * lx + cy * ly);
        c.st_parent[n0 + nodes] = nid[a];
        c.st_R[n0 + nodes] = rx * lx + ry * ly;
        c.st_C[n0 + nodes] = half;
        c.st_C[n0 + nid[a]] += half;
        ++nodes;
        return true;
    };
    while (head < tail) {
        const int a = queue[head++];
        if (steinerise) {
            for (int w = 0; w < B.W; ++w)
                for (unsigned mk = B.row(a)[w]; mk; mk &= mk - 1)
                    if (!visit(a, w * 32 + __ffs(mk) - 1)) return;
        } else {   // the MST by its sources: the parent (visited) and the children, ascending
            for (int b = 0; b < n; ++b)
                if (src[b] == a && !visit(a, b)) return;
        }
    }
    for (int j = 1; j < n; ++j) c.st_fo_node[f0 + j - 1] = nid[j];
    c.st_nlive[g] = nodes;
    c.st_wl[g] = total;
}

}  // namespace

void launch_net_steiner(const DevCtx &c, cudaStream_t st)
{
    if (c.I > 0) k_net_steiner<<<(c.I + kSteinerThreads - 1) / kSteinerThreads, kSteinerThreads, 0, st>>>(c);
}

}  // namespace sta
