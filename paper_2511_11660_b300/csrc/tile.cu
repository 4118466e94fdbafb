// tile.cu -- tile schedule of the timing pass.
//
// Each pass is one co-resident launch of B blocks (one tile each; the
// partition is built on the host, tile.cpp).  A block walks the steps --
// forward: the levels in order, then the endpoints of the last level;
// backward: the levels in reverse -- and at each step runs only the items
// (and endpoints) of its own list, one item per 4 * KL lanes, then waits at
// a block barrier.  The per-item arithmetic is the dataflow schedule's
// (item.cuh), so all schedules agree bit for bit; what changes is where an
// item finds its inputs:
//   * a producer in the same block whose slot is still in the block's
//     shared-memory ring: a shared-memory read after the step barrier (the
//     partition puts an item in the block of its critical fan-in, so most
//     level-to-level dependencies take this path);
//   * any other producer: the parity mailbox of the dataflow schedule,
//     polled without blocking with a bounded number of idle rounds.
// Every item still publishes to the mailbox (other blocks, the other
// corners of a quad, and the -through states read it there).
//
// Latency hiding: a thread's next entry is known in advance (its slot in
// the next wave or step), so its descriptor is fetched one entry ahead and
// the loads that depend on it (net delays and load, and the first poll of
// the mailbox inputs) are issued before the current entry computes.
//
// Progress: a block waits only for entries of earlier steps, every block is
// resident (cooperative launch), and every block finishes the steps in
// order, so every wait ends; the waits are bounded all the same (a timeout
// sets the error word and the abort word, and every block leaves).
#include <algorithm>

#include "item.cuh"
#include "kernels.h"
#include "tile.h"

namespace sta {

constexpr int kTileThreads = 256;
constexpr int kTileRingLanes = 256;   // ring slots x KL quads (R = kTileRingLanes / KL)
constexpr int kTileMaxSteps = 4096;   // steps whose list offsets fit the shared copy

// shared memory after the library: list offsets, item counts and backward
// bases of the block's steps, then the ring
static size_t tile_rows_bytes(int NS) { return ((size_t)3 * (NS + 1) * sizeof(int) + 15) & ~(size_t)15; }
static size_t tile_fwd_smem(int T, int NS)
{
    return ((smem_lib_bytes(T) + 15) & ~(size_t)15) + tile_rows_bytes(NS) + (size_t)kTileRingLanes * 4 * 12;
}
static size_t tile_bwd_smem(int T, int NS)
{
    return ((smem_lib_bytes(T) + 15) & ~(size_t)15) + tile_rows_bytes(NS) + (size_t)kTileRingLanes * 12 * 8;
}

struct TileRows {
    int *ptr, *nit, *rb;   // [NS + 1] / [NS] / [NS]
    char *ring;
};

__device__ __forceinline__ TileRows stage_rows(const DevCtx &c, float *smem)
{
    char *p = reinterpret_cast<char *>(smem) + ((smem_lib_bytes(c.T) + 15) & ~(size_t)15);
    const int NS = c.tl_NS, b = blockIdx.x;
    TileRows r;
    r.ptr = reinterpret_cast<int *>(p);
    r.nit = r.ptr + NS + 1;
    r.rb = r.nit + NS;
    for (int i = threadIdx.x; i <= NS; i += blockDim.x) r.ptr[i] = __ldg(c.tl_ptr + (size_t)b * NS + i);
    for (int i = threadIdx.x; i < NS; i += blockDim.x) {
        r.nit[i] = __ldg(c.tl_nitem + (size_t)b * NS + i);
        r.rb[i] = __ldg(c.tl_rbase + (size_t)b * NS + i);
    }
    r.ring = p + ((3 * (size_t)(NS + 1) * sizeof(int) + 15) & ~(size_t)15);
    return r;
}

// A bounded idle round of a warp waiting on the mailbox: false once the
// wait limit is reached (timeout bit + abort word) or the pass was aborted
// (by any block, or by another warp of this block).
__device__ __forceinline__ bool tile_idle_round(const DevCtx &c, long long &spins, volatile int *s_abort)
{
    if (++spins >= c.spin_limit) {
        if ((threadIdx.x & 31) == 0) {
            atomicOr(c.err, kErrTimeout);
            atomicExch(c.df_state + 3, 1u);
            *s_abort = 1;
        }
        return false;
    }
    if ((spins & 31) == 0 && __any_sync(0xffffffffu, *s_abort != 0 || ld_volatile(c.df_state + 3) != 0u)) {
        if ((threadIdx.x & 31) == 0) *s_abort = 1;
        return false;
    }
    __nanosleep(32);
    return true;
}

// The block-uniform walk over waves: wave (s, x0) holds list entries
// [x0, x0 + W) of step s, lane slot `slot` takes entry x0 + slot if it is
// inside the step.  Empty steps are skipped (their barriers still run).
struct Wave {
    int s, x0;
};

// ------------------------------------------------------------- forward

// One forward list entry as the lane holds it: the descriptor's fields and
// the loads that depend on them.  An endpoint keeps its fields in the
// FwdItem: pin0 = its pin, drv[0] = its driver, Dn0[0] / V0[0] = its net
// delay and variance, tag = 1 for a flip-flop D pin, t = endpoint index.
struct TileFwd {
    int id;          // item g, or I + endpoint
    int ring[3];     // ring slot of each input's driver, -1 = mailbox
    FwdItem f;
    FwdIn in;        // the first corner's component q of the drivers: an early mailbox poll (NaN = not yet)
};

__device__ __forceinline__ void tile_fwd_desc(const DevCtx &c, int x, int4 &d0, int4 &d1)
{
    d0 = __ldg(c.tl_fdesc + 2 * (size_t)x);
    d1 = __ldg(c.tl_fdesc + 2 * (size_t)x + 1);
}

// The loads of an entry that depend on its descriptor: net delays and
// variances, the output load, and a first poll of every mailbox input.
__device__ __forceinline__ void tile_fwd_load(const DevCtx &c, const SmemLib &L, int4 d0, int4 d1, int par, int q,
                                              TileFwd &u)
{
    const int K = c.K, kq = corner_lane(c);
    FwdItem &f = u.f;
    u.id = d0.x;
    if (d0.x < c.I) {
        const int g = chk(c, d0.x, c.I);
        f.t = chk_type(c, d0.z);
        f.pin0 = chk(c, d0.y, c.P);
        f.kind = f.t >= 0 ? L.kind[f.t] : -1;
        f.nin = f.kind == 0 ? L.nin[f.t] : 0;
        f.tag = (c.Tg > 1 && f.kind != 0) ? c.item_tag[g] : 0;
        const int drv[3] = {d0.w, d1.x, d1.y};
        u.ring[0] = (int)(short)(d1.z & 0xffff);
        u.ring[1] = (int)(short)((unsigned)d1.z >> 16);
        u.ring[2] = (int)(short)(d1.w & 0xffff);
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (u.ring[j] >= 0) u.ring[j] = chk(c, u.ring[j], c.tl_R);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool on = j < f.nin;
            f.sense[j] = on ? L.sense[f.t * 3 + j] : -1;
            const int a = on ? chk(c, f.pin0 + j, c.P) : 0;
            f.drv[j] = on ? chk(c, drv[j], c.I) : 0;   // the driver's item (mailbox index)
            f.Dn0[j] = on ? c.netD[(size_t)a * K + kq] : 0.f;
            f.V0[j] = on ? c.netV[(size_t)a * K + kq] : 0.f;
            u.in.at[j] = nan_df();
            u.in.sl[j] = nan_f();
            if (on && u.ring[j] < 0) {
                u.in.at[j] = ld_relaxed_df(fbox_a(c, par, f.drv[j], kq)->v + q);
                u.in.sl[j] = ld_relaxed1(reinterpret_cast<const float *>(fbox_s(c, par, f.drv[j], kq)) + q);
            }
        }
        const int zl = chk(c, f.kind == 1 ? f.pin0 + 1 : f.pin0 + f.nin, c.P);
        f.ld0 = f.t >= 0 ? c.load[(size_t)zl * K + kq] : 0.f;
    } else {
        f.t = chk(c, d1.x, c.E);
        f.pin0 = chk(c, d0.y, c.P);
        f.drv[0] = chk(c, d0.z, c.I);   // the driver's item (mailbox index)
        f.tag = d0.w != 0;
        f.nin = 1;
        f.Dn0[0] = c.netD[(size_t)f.pin0 * K + kq];
        f.V0[0] = c.netV[(size_t)f.pin0 * K + kq];
        u.ring[0] = (int)(short)(d1.z & 0xffff);
        if (u.ring[0] >= 0) u.ring[0] = chk(c, u.ring[0], c.tl_R);
        u.in.at[0] = nan_df();
        u.in.sl[0] = nan_f();
        if (u.ring[0] < 0) {
            u.in.at[0] = ld_relaxed_df(fbox_a(c, par, f.drv[0], kq)->v + q);
            u.in.sl[0] = ld_relaxed1(reinterpret_cast<const float *>(fbox_s(c, par, f.drv[0], kq)) + q);
        }
    }
}

// Are input j's driver values complete?  The ring first (a held test item
// leaves its slot NaN: then the mailbox); a mailbox input keeps its early
// poll if that saw the value, else polls again, and checks the lane's other
// states (every state with -through sets: a path may come in from the
// previous tag).  A ring producer published its other states before the
// step barrier.
template <bool THRU>
__device__ __forceinline__ bool tile_fwd_input(const DevCtx &c, int drv, int ring, int par, int q, const DF *ring_at,
                                               const float *ring_sl, DF &at, float &sl)
{
    const int kq = corner_lane(c);
    if (ring >= 0) {
        const int rs = (ring * c.KL + kq) * 4 + q;
        at = ring_at[rs];
        sl = ring_sl[rs];
        if (real_df(at) && sl == sl) return true;
    }
    if (!(real_df(at) && sl == sl)) {
        at = ld_relaxed_df(fbox_a(c, par, drv, kq)->v + q);
        sl = ld_relaxed1(reinterpret_cast<const float *>(fbox_s(c, par, drv, kq)) + q);
        if (!(real_df(at) && sl == sl)) return false;
    }
    const uint32_t *pin_adv = THRU ? c.pin_adv : nullptr;
    const int k0 = pin_adv ? 0 : kq + c.KL, dk = pin_adv ? 1 : c.KL;
    bool ok = true;
    for (int k = k0; k < c.K && ok; k += dk)
        if (k != kq) ok = complete_df(fbox_a(c, par, drv, k)) && complete(ld_relaxed4(fbox_s(c, par, drv, k)));
    return ok;
}

__device__ __forceinline__ void fwd_wave_next(const int *ptr, int NS, int W, Wave &w)
{
    w.x0 += W;
    while (w.s < NS && w.x0 >= ptr[w.s + 1]) {
        ++w.s;
        if (w.s < NS) w.x0 = ptr[w.s];
    }
}

template <bool SMOOTH, bool UNIFORM, bool THRU>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile_forward(const DevCtx c)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    const SmemLib L = stage_library(c, smem);
    const TileRows rows = stage_rows(c, smem);
    DF *ring_at = reinterpret_cast<DF *>(rows.ring);
    float *ring_sl = reinterpret_cast<float *>(ring_at + kTileRingLanes * 4);
    __syncthreads();
    const int par = (int)(ld_volatile(c.df_state) & 1u);
    const int KL = c.KL, per = 4 * KL, W = blockDim.x / per, slot = threadIdx.x / per;
    const int q = threadIdx.x & 3, kq = corner_lane(c);
    const int NS = c.tl_NS, R = c.tl_R, base = rows.ptr[0];
    const int *ptr = rows.ptr;
    // three waves in flight: w0 computes, w1's dependent loads are issued,
    // w2's descriptor is fetched
    Wave w0{0, ptr[0] - W}, w1, w2;
    fwd_wave_next(ptr, NS, W, w0);
    w1 = w0;
    fwd_wave_next(ptr, NS, W, w1);
    w2 = w1;
    fwd_wave_next(ptr, NS, W, w2);
    auto has = [&](const Wave &w) { return w.s < NS && w.x0 + slot < ptr[w.s + 1]; };
    TileFwd cur, nxt;
    int4 d0, d1, e0 = make_int4(0, 0, 0, 0), e1 = e0;
    if (has(w0)) {
        tile_fwd_desc(c, w0.x0 + slot, d0, d1);
        tile_fwd_load(c, L, d0, d1, par, q, cur);
    }
    if (has(w1)) tile_fwd_desc(c, w1.x0 + slot, e0, e1);
    int cs = 0;          // steps whose barrier has run
    bool bad = false;    // this lane's warp gave up waiting
    while (w0.s < NS) {
        for (; cs < w0.s; ++cs)
            if (__syncthreads_or(bad)) return;
        if (has(w1)) tile_fwd_load(c, L, e0, e1, par, q, nxt);
        if (has(w2)) tile_fwd_desc(c, w2.x0 + slot, e0, e1);
        const int x = w0.x0 + slot;
        bool pending = has(w0) && !bad;
        long long spins = 0;
        while (__any_sync(0xffffffffu, pending)) {
            bool ok = pending;
            if (pending) {
                if (cur.id < c.I) {
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        if (j < cur.f.nin)
                            ok = tile_fwd_input<THRU>(c, cur.f.drv[j], cur.ring[j], par, q, ring_at, ring_sl,
                                                      cur.in.at[j], cur.in.sl[j]) && ok;
                } else {
                    ok = tile_fwd_input<false>(c, cur.f.drv[0], cur.ring[0], par, q, ring_at, ring_sl, cur.in.at[0],
                                               cur.in.sl[0]);
                }
            }
            if (group_all_warp(c, ok) && pending) {   // the whole warp votes
                if (cur.id < c.I) {
                    FwdOut o;
                    fwd_run<SMOOTH, UNIFORM, true, THRU>(c, L.lut, cur.f, cur.in, cur.id, q, par, &o);
                    // a held test item leaves its slot NaN: its consumers then wait on the mailbox
                    const int rs = (((x - base) % R) * KL + kq) * 4 + q;
                    const bool held = cur.id == c.hold_item;
                    ring_at[rs] = held ? nan_df() : o.at;
                    ring_sl[rs] = held ? nan_f() : o.sl;
                } else {
                    EpItem ep;
                    ep.p = cur.f.pin0;
                    ep.d = cur.f.drv[0];
                    ep.isD = cur.f.tag != 0;
                    ep.Dn0 = cur.f.Dn0[0];
                    ep.V0 = cur.f.V0[0];
                    ep_run<true>(c, ep, cur.in.at[0], cur.in.sl[0], cur.f.t, q, par);
                }
                pending = false;
            }
            if (__any_sync(0xffffffffu, pending) && !tile_idle_round(c, spins, &s_abort)) {
                bad = true;
                break;
            }
        }
        w0 = w1;
        w1 = w2;
        fwd_wave_next(ptr, NS, W, w2);
        cur = nxt;
    }
}

// ------------------------------------------------------------- backward
//
// The output's required time is a fold over the net's sinks (item.cuh,
// bwd_probe_split: min (late) / max (early) of RAT - Elmore delay, the first
// extreme in fan-out order wins, and the winner's difference is formed
// exactly).  Here the quad splits the sinks instead of the components:
// lane q folds fan-out entries q, q + 4, q + 8, ... for all four components
// (one 32-byte read per sink), then the quad reduces each component keeping
// the lowest entry among equal extremes -- the same winner as the
// sequential fold, so the same bits -- and lane q takes component q's
// winner.  A driver with many sinks waits for a quarter of the round trips.

// One backward item entry as the lane holds it: the item's loads (states
// of its pins from the forward pass, output load) and the lane's two
// sinks among the first eight (fan-out entries q and q + 4) with their
// ring codes, net delays and an early read of all four components of their
// required times (mailbox or endpoint; NaN = not yet).
struct TileBwd {
    BwdItem b;
    int sk[2], cd[2];
    float nd[2];
    DF m[2][4];
};

__device__ __forceinline__ void tile_bwd_desc(const DevCtx &c, int x, int4 (&d)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = __ldg(c.tl_bdesc + 4 * (size_t)x + i);
}

__device__ __forceinline__ int i4(const int4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// all four components of the required time of sink s (fan-out entry fe) at
// state ks: the ring (first corner, code >= 0), else the mailbox (gate
// input) or the endpoint's required time
__device__ __forceinline__ void sink_rat4(const DevCtx &c, int fe, int s, int code, int ks, int par, const DF *ring_r,
                                          DF (&m)[4])
{
    const int kq = corner_lane(c);
    if (code >= 0 && ks == kq) {
        const DF *r = ring_r + (((code >> 2) * c.KL + kq) * 3 + (code & 3)) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j] = r[j];
    } else if (s < c.ep_begin) {
        ld_relaxed_df4(rbox_at(c, par, fe, ks), m[0], m[1], m[2], m[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j] = ld_state_df(c.rat + (size_t)s * c.K + ks, j);
    }
}

template <bool THRU>
__device__ __forceinline__ void tile_bwd_load(const DevCtx &c, const SmemLib &L, const int4 (&d)[4], int par, int q,
                                              TileBwd &u)
{
    BwdItem &b = u.b;
    const int K = c.K, kq = corner_lane(c);
    b.pin0 = chk(c, d[0].x, c.P);
    b.t = chk_type(c, d[0].y);
    b.kind = b.t >= 0 ? L.kind[b.t] : -1;
    b.nin = b.t >= 0 ? L.nin[b.t] : 0;
    b.z = chk(c, b.t < 0 ? b.pin0 : (b.kind == 1 ? b.pin0 + 1 : b.pin0 + b.nin), c.P);
    b.f0 = chk(c, d[0].z, (long long)c.F + 1);
    b.f1 = chk(c, d[0].w, (long long)c.F + 1);
    b.ld0 = b.t >= 0 ? c.load[(size_t)b.z * K + kq] : 0.f;
    b.az0 = ld_state_df(c.at + (size_t)b.z * K + kq, q);
#pragma unroll
    for (int j = 0; j < 3; ++j)
        b.fin[j] = (b.kind == 0 && j < b.nin) ? chk(c, c.pin_fo[b.pin0 + j], (long long)c.F) : 0;
    const int nread = b.kind == 1 ? 1 : b.kind == 0 ? b.nin : 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const bool on = j < nread;
        const size_t o = (size_t)(b.pin0 + j) * K + kq;
        b.s0[j] = on ? ld_state(c.slew + o, b.kind == 1 ? (q & 2) : q) : 0.f;
        b.a0[j] = on ? ld_state_df(c.at + o, q) : DF(0.f);
    }
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const int e = q + 4 * v;   // fan-out entry of this lane
        const int sk = i4(d[1 + v], q);
        const int cw = i4(d[3], e >> 1);
        const int cd = (int)(short)((e & 1) ? ((unsigned)cw >> 16) : (cw & 0xffff));
        u.sk[v] = sk >= 0 ? chk(c, sk, c.P) : -1;
        u.cd[v] = cd >= 0 ? chk(c, cd, 4 * c.tl_R) : -1;
        u.nd[v] = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) u.m[v][j] = nan_df();
        if (u.sk[v] >= 0) {
            u.nd[v] = __ldg(c.netD + (size_t)u.sk[v] * K + kq);
            // -through sinks pick their state at use; ring sinks are read after the barrier
            if (!THRU && u.cd[v] < 0) sink_rat4(c, b.f0 + e, u.sk[v], -1, kq, par, nullptr, u.m[v]);
        }
    }
}

template <bool THRU>
__device__ __forceinline__ bool tile_bwd_probe(const DevCtx &c, TileBwd &u, int par, int q, const DF *ring_r, Fold4 &f)
{
    const uint32_t *pin_adv = THRU ? c.pin_adv : nullptr;
    const BwdItem &b = u.b;
    const int K = c.K, kq = corner_lane(c);
    fold4_clear(f);
    auto fold = [&](int e, const DF (&m)[4], float nd) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float val = m[j].hi - nd;
            if (j >= 2 ? val < f.v[j] : val > f.v[j]) {
                f.v[j] = val;
                f.idx[j] = e;
                f.rw[j] = m[j];
                f.rd[j] = nd;
            }
        }
    };
    auto state_of = [&](int s) { return (pin_adv && ((pin_adv[s] >> (kq % c.Tg)) & 1u)) ? kq + 1 : kq; };
    bool ok = true;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        if (u.sk[v] < 0) continue;
        const int ks = state_of(u.sk[v]);
        const bool have = real_df(u.m[v][0]) && real_df(u.m[v][1]) && real_df(u.m[v][2]) && real_df(u.m[v][3]);
        if (!have || (u.cd[v] >= 0 && ks == kq)) sink_rat4(c, b.f0 + q + 4 * v, u.sk[v], u.cd[v], ks, par, ring_r, u.m[v]);
        const bool rdy = real_df(u.m[v][0]) && real_df(u.m[v][1]) && real_df(u.m[v][2]) && real_df(u.m[v][3]);
        ok = ok && rdy;
    }
    if (!ok) return false;
#pragma unroll
    for (int v = 0; v < 2; ++v)
        if (u.sk[v] >= 0) fold(q + 4 * v, u.m[v], u.nd[v]);
    // entries beyond the first eight (rare): read at use
    for (int e = 8 + q; b.f0 + e < b.f1; e += 4) {
        const int p = b.f0 + e;
        const int s = chk(c, __ldg(c.fo_pin + p), c.P);
        int code = (int)__ldg(c.tl_fo_ring + p);
        if (code >= 0) code = chk(c, code, 4 * c.tl_R);
        DF m[4];
        sink_rat4(c, p, s, code, state_of(s), par, ring_r, m);
        if (!(real_df(m[0]) && real_df(m[1]) && real_df(m[2]) && real_df(m[3]))) return false;
        fold(e, m, __ldg(c.netD + (size_t)s * K + kq));
    }
    // the lane's other states of mailbox sinks (a ring sink's were
    // published by this block before the step barrier)
    if (K > c.KL || pin_adv) {
        for (int p = b.f0; p < b.f1 && ok; ++p) {
            const int s = chk(c, __ldg(c.fo_pin + p), c.P);
            if (s < c.ep_begin && __ldg(c.tl_fo_ring + p) < 0) {
                const int k0 = pin_adv ? 0 : kq + c.KL, dk = pin_adv ? 1 : c.KL;
                for (int k = k0; k < K && ok; k += dk)
                    if (k != kq) ok = complete_df(rbox_at(c, par, p, k));
            }
        }
    }
    return ok;
}

__device__ __forceinline__ void bwd_wave_next(const int *nit, int W, Wave &w)
{
    w.x0 += W;
    while (w.s >= 0 && w.x0 >= nit[w.s]) {
        --w.s;
        w.x0 = 0;
    }
}

template <bool UNIFORM, bool THRU>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile_backward(const DevCtx c)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    const SmemLib L = stage_library(c, smem);
    const TileRows rows = stage_rows(c, smem);
    DF *ring_r = reinterpret_cast<DF *>(rows.ring);
    __syncthreads();
    const int par = (int)(ld_volatile(c.df_state) & 1u);
    const int KL = c.KL, per = 4 * KL, W = blockDim.x / per, slot = threadIdx.x / per;
    const int q = threadIdx.x & 3, kq = corner_lane(c);
    const int NS = c.tl_NS, R = c.tl_R;
    const int *ptr = rows.ptr, *nit = rows.nit, *rb = rows.rb;
    // waves over the item part of each list, steps in reverse; x0 counts
    // items inside the step
    Wave w0{NS - 1, -W}, w1, w2;
    bwd_wave_next(nit, W, w0);
    w1 = w0;
    bwd_wave_next(nit, W, w1);
    w2 = w1;
    bwd_wave_next(nit, W, w2);
    auto has = [&](const Wave &w) { return w.s >= 0 && w.x0 + slot < nit[w.s]; };
    TileBwd cur, nxt;
    int4 dd[4], de[4];
    if (has(w0)) {
        tile_bwd_desc(c, ptr[w0.s] + w0.x0 + slot, dd);
        tile_bwd_load<THRU>(c, L, dd, par, q, cur);
    }
    if (has(w1)) tile_bwd_desc(c, ptr[w1.s] + w1.x0 + slot, de);
    int cs = NS - 1;     // the next barrier closes step cs
    bool bad = false;
    while (w0.s >= 0) {
        for (; cs > w0.s; --cs)
            if (__syncthreads_or(bad)) return;
        if (has(w1)) tile_bwd_load<THRU>(c, L, de, par, q, nxt);
        if (has(w2)) tile_bwd_desc(c, ptr[w2.s] + w2.x0 + slot, de);
        bool pending = has(w0) && !bad;
        long long spins = 0;
        while (__any_sync(0xffffffffu, pending)) {
            Fold4 fo;
            bool ok = false;
            if (pending) ok = tile_bwd_probe<THRU>(c, cur, par, q, ring_r, fo);
            else fold4_clear(fo);
            const bool go = group_all_warp(c, ok) && pending;   // the whole warp votes
            // every lane folds (full-warp shuffles); the ready groups use it
            const DF Rz = __any_sync(0xffffffffu, go) ? quad_fold(fo, q, 0xffffffffu) : DF(0.f);
            if (go) {
                DF first[3];
                bwd_run<UNIFORM, true, THRU>(c, L.lut, L.sense, cur.b, q, par, Rz, first);
                if (cur.b.kind == 0) {
                    const int rs = ((rb[w0.s] + w0.x0 + slot) % R) * KL + kq;
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        if (j < cur.b.nin) ring_r[(rs * 3 + j) * 4 + q] = first[j];
                }
                pending = false;
            }
            if (__any_sync(0xffffffffu, pending) && !tile_idle_round(c, spins, &s_abort)) {
                bad = true;
                break;
            }
        }
        w0 = w1;
        w1 = w2;
        bwd_wave_next(nit, W, w2);
        cur = nxt;
    }
}

// ------------------------------------------------------------- launches

using TileKernel = void (*)(DevCtx);
static TileKernel tile_forward_kernel(bool smooth, bool uniform, bool thru)
{
    if (thru) return smooth ? (uniform ? k_tile_forward<true, true, true> : k_tile_forward<true, false, true>)
                            : (uniform ? k_tile_forward<false, true, true> : k_tile_forward<false, false, true>);
    return smooth ? (uniform ? k_tile_forward<true, true, false> : k_tile_forward<true, false, false>)
                  : (uniform ? k_tile_forward<false, true, false> : k_tile_forward<false, false, false>);
}
static TileKernel tile_backward_kernel(bool uniform, bool thru)
{
    if (thru) return uniform ? k_tile_backward<true, true> : k_tile_backward<false, true>;
    return uniform ? k_tile_backward<true, false> : k_tile_backward<false, false>;
}

int tile_threads() { return kTileThreads; }
int tile_ring_slots(int KL) { return kTileRingLanes / KL; }
int tile_max_steps() { return kTileMaxSteps; }

// Largest co-resident grid of both tile kernels (blocks), outside capture.
cudaError_t tile_prepare(HostSched &h, bool smooth, int NS, int *max_blocks)
{
    int dev = 0, sms = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess && !coop) e = cudaErrorNotSupported;
    if (e != cudaSuccess) return e;
    const size_t sf = tile_fwd_smem(h.T, NS), sb = tile_bwd_smem(h.T, NS);
    auto kf = tile_forward_kernel(smooth, h.uniform, h.thru);
    auto kb = tile_backward_kernel(h.uniform, h.thru);
    int pf = 0, pb = 0;
    e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, kf, kTileThreads, sf);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pb, kb, kTileThreads, sb);
    if (e != cudaSuccess) return e;
    if (pf < 1 || pb < 1) return cudaErrorInvalidConfiguration;
    *max_blocks = std::min(pf, pb) * sms;
    return cudaSuccess;
}

static void tile_launch(TileKernel k, const DevCtx &c, size_t smem, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.tl_B);
    cfg.blockDim = dim3(kTileThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, c);
}

void launch_tile_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev)
{
    if (ev) cudaEventRecord(ev[0], st);
    launch_df_reset(c, h.tile_blocks, st);
    launch_net_phase(c, h, st);
    if (ev) cudaEventRecord(ev[1], st);
    if (c.I > 0 || c.E > 0) tile_launch(tile_forward_kernel(c.gamma > 0.f, h.uniform, h.thru), c, tile_fwd_smem(h.T, c.tl_NS), st);
    if (ev) cudaEventRecord(ev[2], st);
    if (c.I > 0) tile_launch(tile_backward_kernel(h.uniform, h.thru), c, tile_bwd_smem(h.T, c.tl_NS), st);
    if (ev) cudaEventRecord(ev[3], st);
    launch_reduce(c, h, st);
    if (ev) cudaEventRecord(ev[4], st);
}

}  // namespace sta
