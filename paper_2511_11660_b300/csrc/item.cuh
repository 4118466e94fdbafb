// item.cuh -- the per-item timing math shared by the level kernels and the
// persistent dataflow kernels.
//
// An item is a primary input, a flip-flop (CK -> Q) or a gate with its input
// pins and output pin.  Forward: the gate's input pins take the driver's
// arrival + Elmore delay and slew sqrt(s^2 + var) (net arcs); the output
// merges every arc candidate: arrival = input arrival + NLDM delay(input
// slew, load), slew = NLDM slew(input slew, load), max for late, min for
// early (log-sum-exp when smoothed).  Backward: the output's required time
// is the min (late) / max (early) over its net sinks of RAT - Elmore delay;
// each input's is the min/max over its arcs of output RAT - arc delay.
//
// Four lanes (a "quad") work on one item and corner: lane q owns state
// component q = el*2 + rf (early-rise, early-fall, late-rise, late-fall), so
// a thread's serial chain is a quarter of the item and the four lanes write
// 16 contiguous bytes of every float4.  With several corners, KL quads (a
// power of two, at most 8) share an item, one corner each in turn.
//
// WAIT = true is the dataflow schedule: values produced by other items of
// the same launch are taken from the parity mailboxes once they are
// complete (see below and dataflow.cu) and the item publishes its own
// results there; WAIT = false relies on launch boundaries (level schedule).
//
// Mailboxes.  For epoch parity p, fbox_a[p] / fbox_s[p] hold each item's
// output arrival (double-float) and slew (FP32) and rbox each gate input
// pin's required time (double-float).  Every float is NaN until its producer
// stores the final value with a relaxed store, and a real result is never
// NaN, so a reader that sees all the floats it needs non-NaN has the final
// values: each 32-bit store is single-copy atomic, no fence or flag is
// needed, and the poll is the data load itself.  While it publishes
// parity p, a producer resets its own entries of parity p ^ 1 to NaN for the
// next pass.
#pragma once

#include "device.cuh"

namespace sta {

// ---------------------------------------------------------------- tables

// Table reads: from global memory through the read-only cache, or from a
// shared-memory copy of the packed library.
// sc(k) is state k's table scale (the corner's LUT factor).
constexpr int kSmemScales = 64;   // states whose table scale the shared copy holds
struct LutGlobal {
    const float *base;
    const float *scale;   // [K] in global memory
    __device__ __forceinline__ float operator[](int off) const { return __ldg(base + off); }
    __device__ __forceinline__ float sc(int k) const { return __ldg(scale + k); }
};
struct LutShared {
    const float *base;    // points into shared memory
    const float *scale;   // the first kSmemScales states' scales, in shared memory
    const float *gscale;  // [K] in global memory (states beyond the shared copy)
    __device__ __forceinline__ float operator[](int off) const { return base[off]; }
    __device__ __forceinline__ float sc(int k) const { return k < kSmemScales ? scale[k] : __ldg(gscale + k); }
};

struct Seg {
    int o;     // offset of the segment's first value (i*7 on the slew axis, j on the load axis)
    float t;   // position inside the segment (outside [0, 1] when extrapolating)
};

// Segment = number of interior breakpoints <= x (off-table queries use the
// edge segment); weight = (x - x_i) / (x_{i+1} - x_i) via a stored reciprocal.
template <class L>
__device__ __forceinline__ Seg seg_slew_t(const L &lut, int tb, float s)
{
    const int i = (s >= lut[tb + 1]) + (s >= lut[tb + 2]) + (s >= lut[tb + 3]) + (s >= lut[tb + 4]) +
                  (s >= lut[tb + 5]);
    return Seg{i * 7, (s - lut[tb + i]) * lut[tb + 14 + i]};
}
template <class L>
__device__ __forceinline__ Seg seg_load_t(const L &lut, int tb, float l)
{
    const int j = (l >= lut[tb + 8]) + (l >= lut[tb + 9]) + (l >= lut[tb + 10]) + (l >= lut[tb + 11]) +
                  (l >= lut[tb + 12]);
    return Seg{j, (l - lut[tb + 7 + j]) * lut[tb + 20 + j]};
}

// The same segment rule on the shared axes held in the kernel parameters:
// comparisons and selects only, no memory access.
__device__ __forceinline__ Seg seg_axes(const float *ax, const float *iw, int stride, float x)
{
    const bool b1 = x >= ax[1], b2 = x >= ax[2], b3 = x >= ax[3], b4 = x >= ax[4], b5 = x >= ax[5];
    const int i = b1 + b2 + b3 + b4 + b5;
    const float x0 = b5 ? ax[5] : b4 ? ax[4] : b3 ? ax[3] : b2 ? ax[2] : b1 ? ax[1] : ax[0];
    const float w = b5 ? iw[5] : b4 ? iw[4] : b3 ? iw[3] : b2 ? iw[2] : b1 ? iw[1] : iw[0];
    return Seg{i * stride, (x - x0) * w};
}

template <bool UNIFORM, class L>
__device__ __forceinline__ Seg seg_slew(const DevCtx &c, const L &lut, int tb, float s)
{
    if (UNIFORM) return seg_axes(c.ax1, c.iw1, 7, s);
    return seg_slew_t(lut, tb, s);
}
template <bool UNIFORM, class L>
__device__ __forceinline__ Seg seg_load(const DevCtx &c, const L &lut, int tb, float l)
{
    if (UNIFORM) return seg_axes(c.ax2, c.iw2, 1, l);
    return seg_load_t(lut, tb, l);
}

template <class L>
__device__ __forceinline__ float interp(const L &lut, int tb, Seg a, Seg b)
{
    const int v = tb + 26 + a.o + b.o;
    const float v00 = lut[v], v01 = lut[v + 1], v10 = lut[v + 7], v11 = lut[v + 8];
    const float x = fmaf(b.t, v01 - v00, v00);
    const float y = fmaf(b.t, v11 - v10, v10);
    return fmaf(a.t, y - x, x);
}
// The same bilinear form with its partials: d/ds (per ns) and d/dl (per pF).
template <class L>
__device__ __forceinline__ float interp_d(const L &lut, int tb, Seg a, Seg b, float &ds, float &dl)
{
    const int v = tb + 26 + a.o + b.o;
    const float v00 = lut[v], v01 = lut[v + 1], v10 = lut[v + 7], v11 = lut[v + 8];
    const float x = fmaf(b.t, v01 - v00, v00);
    const float y = fmaf(b.t, v11 - v10, v10);
    ds = (y - x) * lut[tb + 14 + a.o / 7];
    dl = fmaf(a.t, (v11 - v10) - (v01 - v00), v01 - v00) * lut[tb + 20 + b.o];
    return fmaf(a.t, y - x, x);
}

__device__ __forceinline__ int tab_off(int t, int slot, int tb) { return ((t * 3 + slot) * 4 + tb) * kLutStride; }

// value of table tq at (s, l): shared segments when every table has the same
// axes (UNIFORM), else the table's own segments
template <bool UNIFORM, class L>
__device__ __forceinline__ float lookup(const L &lut, int tq, Seg as, Seg bl, float s, float l)
{
    if (UNIFORM) return interp(lut, tq, as, bl);
    return interp(lut, tq, seg_slew_t(lut, tq, s), seg_load_t(lut, tq, l));
}

// The cell library (packed tables and per-type data) in shared memory, one
// copy per block of the persistent kernels.
struct SmemLib {
    LutShared lut;
    const int *nin, *kind, *sense;
};

// tables, then per-type data (5 ints a type), then the states' table scales
__host__ __device__ inline size_t smem_lib_bytes(int T)
{
    return (size_t)T * 3 * 4 * kLutStride * sizeof(float) + (size_t)T * 5 * sizeof(int) +
           (size_t)kSmemScales * sizeof(float);
}

__device__ __forceinline__ SmemLib stage_library(const DevCtx &c, float *smem)
{
    const int nl = c.T * 3 * 4 * kLutStride;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) smem[i] = __ldg(c.lut + i);
    int *ti = reinterpret_cast<int *>(smem + nl);
    for (int i = threadIdx.x; i < c.T; i += blockDim.x) {
        ti[i] = __ldg(c.type_nin + i);
        ti[c.T + i] = __ldg(c.type_kind + i);
    }
    for (int i = threadIdx.x; i < 3 * c.T; i += blockDim.x) ti[2 * c.T + i] = __ldg(c.arc_sense + i);
    float *sc = reinterpret_cast<float *>(ti + 5 * c.T);
    for (int i = threadIdx.x; i < kSmemScales && i < c.K; i += blockDim.x) sc[i] = __ldg(c.lut_scale + i);
    __syncthreads();
    return SmemLib{LutShared{smem, sc, c.lut_scale}, ti, ti + c.T, ti + 2 * c.T};
}

// ------------------------------------------------------ mailbox access

__device__ __forceinline__ float4 ld_relaxed4(const float4 *p)
{
    float4 v;
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}
__device__ __forceinline__ float ld_relaxed1(const float *p)
{
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
// one double-float component (8 bytes) and a whole record (two 16-byte loads)
__device__ __forceinline__ DF ld_relaxed_df(const DF *p)
{
    DF v;
    asm volatile("ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.hi), "=f"(v.lo) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void ld_relaxed_df4(const DF4 *p, DF &x, DF &y, DF &z, DF &w)
{
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(x.hi), "=f"(x.lo), "=f"(y.hi), "=f"(y.lo)
                 : "l"(p->v)
                 : "memory");
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(z.hi), "=f"(z.lo), "=f"(w.hi), "=f"(w.lo)
                 : "l"(p->v + 2)
                 : "memory");
}
// two adjacent double-float components (16 bytes) and two adjacent floats
__device__ __forceinline__ void ld_relaxed_df2(const DF *p, DF &a, DF &b)
{
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(a.hi), "=f"(a.lo), "=f"(b.hi), "=f"(b.lo)
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void ld_relaxed2(const float *p, float &a, float &b)
{
    asm volatile("ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_relaxed(float *p, float v)
{
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_df(DF *p, DF v)
{
    asm volatile("st.relaxed.gpu.global.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.hi), "f"(v.lo) : "memory");
}
__device__ __forceinline__ unsigned ld_volatile(const unsigned *p) { return *(const volatile unsigned *)p; }
__device__ __forceinline__ bool complete(float4 v) { return v.x == v.x && v.y == v.y && v.z == v.z && v.w == v.w; }
// a published double-float: both halves non-NaN (the two 32-bit halves are
// separate single-copy-atomic stores)
__device__ __forceinline__ bool real_df(DF x) { return x.hi == x.hi && x.lo == x.lo; }
__device__ __forceinline__ bool complete_df(const DF4 *p)
{
    DF x, y, z, w;
    ld_relaxed_df4(p, x, y, z, w);
    return real_df(x) && real_df(y) && real_df(z) && real_df(w);
}
__device__ __forceinline__ float nan_f() { return __int_as_float(0x7fffffff); }
__device__ __forceinline__ DF nan_df() { return DF(nan_f(), nan_f()); }

// required-time mailbox records: [pin][state][parity] -- a record's two
// parities side by side, so the reset of parity p ^ 1 falls in the line of
// the store to p (the forward records below stay [parity][item][state]: an
// item's readers are its neighbours' readers too, and interleaving would
// spread them over twice the lines)
template <class Ctx>
__device__ __forceinline__ size_t box_index(const Ctx &c, int par, int pin, int k)
{
    return (((size_t)pin * nK(c) + k) << 1) | (size_t)par;
}
// forward mailbox records: [parity][driver item][state], dense over the
// items (only item outputs are published), so the entries a level polls sit
// close together
template <class Ctx>
__device__ __forceinline__ size_t fbox_index(const Ctx &c, int par, int slot, int k)
{
    return ((size_t)par * c.I + slot) * nK(c) + k;
}
template <class Ctx>
__device__ __forceinline__ DF4 *fbox_a(const Ctx &c, int par, int slot, int k) { return c.fbox_a + fbox_index(c, par, slot, k); }
template <class Ctx>
__device__ __forceinline__ float4 *fbox_s(const Ctx &c, int par, int slot, int k)
{
    return c.fbox_s + fbox_index(c, par, slot, k);
}
// a gate input's required-time record, by its entry fe in its driver's
// fan-out list (c.pin_fo): a driver reads its sinks' records contiguously
template <class Ctx>
__device__ __forceinline__ DF4 *rbox_at(const Ctx &c, int par, int fe, int k) { return c.rbox + box_index(c, par, fe, k); }

// Lane q publishes component q of item g's output arrival and slew for
// parity par and clears the same component of parity par ^ 1.
template <class Ctx>
__device__ __forceinline__ void publish_fwd(const Ctx &c, int par, int g, int k, int q, DF at, float sl)
{
    st_relaxed_df(fbox_a(c, par, g, k)->v + q, at);
    st_relaxed(reinterpret_cast<float *>(fbox_s(c, par, g, k)) + q, sl);
    fbox_a(c, par ^ 1, g, k)->v[q] = nan_df();
    reinterpret_cast<float *>(fbox_s(c, par ^ 1, g, k))[q] = nan_f();
}
template <class Ctx>
__device__ __forceinline__ void publish_rat(const Ctx &c, int par, int fe, int k, int q, DF r)
{
    st_relaxed_df(rbox_at(c, par, fe, k)->v + q, r);
    rbox_at(c, par ^ 1, fe, k)->v[q] = nan_df();
}

// Reads of pin states (arrival, slew, required time) that another item
// produced: L2 only (ld.global.cg), never a line an earlier read left in
// this SM's L1.  Across kernel boundaries plain loads would do; inside one
// persistent launch (the cooperative schedule) the value may have been
// written by another SM after this SM's L1 cached the line.
__device__ __forceinline__ float4 ld_state4(const float4 *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_state(const float4 *p, int q)
{
    return __ldcg(reinterpret_cast<const float *>(p) + q);
}
__device__ __forceinline__ DF ld_state_df(const DF4 *p, int q)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p->v + q));
    return DF(v.x, v.y);
}
__device__ __forceinline__ void st_comp(float4 *p, int q, float v) { reinterpret_cast<float *>(p)[q] = v; }
__device__ __forceinline__ void st_comp_df(DF4 *p, int q, DF v) { p->v[q] = v; }

__device__ __forceinline__ bool arc_on(int sense, int rfi, int rfo)
{
    return sense == kSenseNonC || (sense == kSensePosC && rfi == rfo) || (sense == kSenseNegC && rfi != rfo);
}

// lanes of the quad that owns this lane
__device__ __forceinline__ unsigned quad_mask() { return 0xFu << (threadIdx.x & 28); }

// Corners are spread over c.KL quads: an item owns 4 * KL consecutive lanes,
// and the quad with corner offset kq handles corners kq, kq + KL, ...
template <class Ctx>
__device__ __forceinline__ int corner_lane(const Ctx &c) { return (threadIdx.x >> 2) & (nKL(c) - 1); }
template <class Ctx>
__device__ __forceinline__ unsigned group_mask(const Ctx &c)
{
    const int w = 4 * nKL(c);
    if (w >= 32) return 0xffffffffu;
    return ((1u << w) - 1u) << ((threadIdx.x & 31) & ~(w - 1));
}
// Does every lane of the item's group agree?  One ballot of the whole warp:
// callers keep all 32 lanes converged (lanes without an item vote false).  A
// vote over each group's own lanes (a 4-lane mask) costs many times a
// full-warp ballot when every group of the warp votes at once.
template <class Ctx>
__device__ __forceinline__ bool group_all_warp(const Ctx &c, bool ok)
{
    const unsigned gm = group_mask(c);
    return (__ballot_sync(0xffffffffu, ok) & gm) == gm;
}

// ------------------------------------------------------------- forward

// The slew degraded by a net, sqrt(s^2 + V): the hardware square root
// (sqrt.approx, relative error within 2^-23 by the PTX ISA) in place of the
// IEEE-rounded one, whose longer sequence every level of the pass waits on.
__device__ __forceinline__ float sqrt_hw(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
//
// Each item is processed in three steps: prep (loads that do not depend on
// this pass's results), probe (are the inputs' results complete?  only in
// the dataflow schedule; it returns them) and run (the arithmetic, the
// stores and, in the dataflow schedule, the publication to the mailbox).

struct FwdItem {
    int t, pin0, nin, kind;
    int tag;                    // exception tag of a startpoint item (PI, flip-flop)
    int sense[3];
    int drv[3];                 // each input's driver: its item (BYITEM: the mailbox index) or its pin
    float Dn0[3], V0[3], ld0;   // net values of the lane's first corner, loaded ahead
};

// the drivers' arrival and slew, component q of the lane's first corner, as
// probed, else it comes from the partner lane; with PAIR the probe returns
// both edges of the lane's early/late half instead, rise in at / sl and fall
// in atp / slp (components el*2 and el*2 + 1, as fwd_run takes them)
struct FwdIn {
    DF at[3];
    float sl[3];
    DF atp[3];
    float slp[3];
};

// BYITEM (the schedules that read the drivers from the mailboxes): drv
// holds the driver items; otherwise the driver pins (their pin states).
template <bool BYITEM = false, class Ctx = DevCtx>
__device__ __forceinline__ FwdItem fwd_prep(const Ctx &c, const int *tnin, const int *tkind, const int *tsense,
                                            int g)
{
    FwdItem f;
    g = chk(c, g, c.I);
    f.t = chk_type(c, c.item_type[g]);
    f.pin0 = chk(c, c.item_pin0[g], c.P);
    f.kind = f.t >= 0 ? tkind[f.t] : -1;
    f.nin = f.kind == 0 ? tnin[f.t] : 0;
    f.tag = (c.Tg > 1 && f.kind != 0) ? c.item_tag[g] : 0;
    const int K = nK(c), kq = corner_lane(c);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const bool on = j < f.nin;
        f.sense[j] = on ? tsense[f.t * 3 + j] : -1;
        const int a = on ? chk(c, f.pin0 + j, c.P) : 0;
        f.drv[j] = on ? (BYITEM ? chk(c, c.item_drv[(size_t)g * 3 + j], c.I) : chk(c, c.drv_of[a], c.P)) : 0;
        f.Dn0[j] = on ? c.netD[(size_t)a * K + kq] : 0.f;
        f.V0[j] = on ? c.netV[(size_t)a * K + kq] : 0.f;
    }
    const int zl = chk(c, f.kind == 1 ? f.pin0 + 1 : f.pin0 + f.nin, c.P);
    f.ld0 = f.t >= 0 ? c.load[(size_t)zl * K + kq] : 0.f;
    return f;
}

// Are the drivers' arrivals and slews of the lane's corners complete?  Lane
// q reads component q of its first corner (returned in `in`; with PAIR also
// the other edge of its early/late half); the caller's group vote
// (group_all_warp) over the quad covers the four components.  With `seen`
// (the caller keeps `in` across its polling rounds), an input found complete
// is marked and not read again: a published value is final for the pass, so
// later rounds read only the inputs still pending (one corner per lane group
// and no -through sets, where the first corner's values are all there is).
// THRU = false: the design has no -through sets (c.pin_adv is NULL); the
// kernels compiled so carry none of their code and registers.
template <bool THRU = true, bool PAIR = false, class Ctx = DevCtx>
__device__ __forceinline__ bool fwd_probe(const Ctx &c, const FwdItem &f, int par, int q, FwdIn &in,
                                          unsigned *seen = nullptr)
{
    const uint32_t *pin_adv = THRU ? c.pin_adv : nullptr;
    bool ok = true;
    const int kq = corner_lane(c);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < f.nin) {
            if (seen && ((*seen >> j) & 1u)) continue;   // complete in an earlier round: kept
            if (PAIR) {
                // both edges of the lane's early/late half in one load each
                DF a0, a1;
                float s0, s1;
                ld_relaxed_df2(fbox_a(c, par, f.drv[j], kq)->v + (q & 2), a0, a1);
                ld_relaxed2(reinterpret_cast<const float *>(fbox_s(c, par, f.drv[j], kq)) + (q & 2), s0, s1);
                in.at[j] = a0;
                in.atp[j] = a1;
                in.sl[j] = s0;
                in.slp[j] = s1;
                const bool cj = real_df(a0) && real_df(a1) && s0 == s0 && s1 == s1;
                if (seen && cj && nK(c) == nKL(c) && !pin_adv) *seen |= 1u << j;
                ok = ok && cj;
            } else {
                in.at[j] = ld_relaxed_df(fbox_a(c, par, f.drv[j], kq)->v + q);
                in.sl[j] = ld_relaxed1(reinterpret_cast<const float *>(fbox_s(c, par, f.drv[j], kq)) + q);
                ok = ok && real_df(in.at[j]) && in.sl[j] == in.sl[j];
            }
            // the lane's other states; with -through every state (a path may
            // come in from the previous tag)
            const int k0 = pin_adv ? 0 : kq + nKL(c), dk = pin_adv ? 1 : nKL(c);
            for (int k = k0; k < nK(c) && ok; k += dk)
                if (k != kq)
                    ok = complete_df(fbox_a(c, par, f.drv[j], k)) &&
                         complete(ld_relaxed4(fbox_s(c, par, f.drv[j], k)));
        }
    }
    return ok;
}

// Lane q of the quad computes component q = el*2 + rf of the item's states.
// The lane's results of its first corner (component q of the output's
// arrival and slew), for the tile schedule's shared-memory ring.
struct FwdOut {
    DF at;
    float sl;
};

template <bool SMOOTH, bool UNIFORM, bool WAIT, bool THRU = true, bool PAIR = false, class L, class Ctx = DevCtx>
__device__ __forceinline__ void fwd_run(const Ctx &c, const L &lut, const FwdItem &f, const FwdIn &in, int g,
                                        int q, int par, FwdOut *first = nullptr)
{
    const uint32_t *pin_adv = THRU ? c.pin_adv : nullptr;
    const int K = nK(c), t = f.t, pin0 = f.pin0, nin = f.nin;
    const int el = q >> 1, rfo = q & 1;
    const int kq = corner_lane(c), KL = nKL(c);
    const bool pub = WAIT && g != c.hold_item;
    // a startpoint's arrival exists only in its own exception tag's states
    // (absent elsewhere: -inf late, +inf early); slews are tag-free
    const float absent = el ? -INFINITY : INFINITY;
    if (t < 0) {   // primary input
        for (int k = kq; k < K; k += KL) {
            const DF a((c.Tg == 1 || k % c.Tg == f.tag) ? c.pi_at : absent);
            st_comp_df(c.at + (size_t)pin0 * K + k, q, a);
            st_comp(c.slew + (size_t)pin0 * K + k, q, c.pi_slew);
            if (pub) publish_fwd(c, par, g, k, q, a, c.pi_slew);
            if (first && k == kq) *first = FwdOut{a, c.pi_slew};
        }
        return;
    }
    if (f.kind == 1) {   // flip-flop: ideal clock at CK, arc CK(rise) -> Q for both edges of Q
        const int ck = pin0, qp = pin0 + 1;
        const float cs = c.clk_slew;
        const int tb = tab_off(t, 1, 0);
        for (int k = kq; k < K; k += KL) {
            const float sc = lut.sc(k);
            const float ld = k != kq ? c.load[(size_t)qp * K + k] : f.ld0;
            const DF ck_at((c.Tg == 1 || k % c.Tg == f.tag) ? 0.f : absent);
            st_comp_df(c.at + (size_t)ck * K + k, q, ck_at);
            st_comp(c.slew + (size_t)ck * K + k, q, cs);
            const Seg as = seg_slew<UNIFORM>(c, lut, tb, cs), bl = seg_load<UNIFORM>(c, lut, tb, ld);
            const DF a = ck_at + sc * lookup<UNIFORM>(lut, tb + rfo * kLutStride, as, bl, cs, ld);
            const float sl = sc * lookup<UNIFORM>(lut, tb + (2 + rfo) * kLutStride, as, bl, cs, ld);
            st_comp_df(c.at + (size_t)qp * K + k, q, a);
            st_comp(c.slew + (size_t)qp * K + k, q, sl);
            if (pub) publish_fwd(c, par, g, k, q, a, sl);
            if (first && k == kq) *first = FwdOut{a, sl};
        }
        return;
    }
    const int z = pin0 + nin;
    const float sgn = el ? 1.f : -1.f;   // early merges are mins: max of the negated candidates
    const unsigned qm = quad_mask();
    for (int k = kq; k < K; k += KL) {
        // net arcs into the input pins: this lane needs components el*2 + {0, 1}
        DF ain[3][2];
        float sin[3][2];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j < nin) {
                const int a = pin0 + j;
                DF a0, a1;   // the driver's rise / fall arrival and slew at this lane's el
                float s0, s1;
                const uint32_t adv = pin_adv ? pin_adv[a] : 0u;
                if (adv) {
                    // -through: a path in this state's tag t stays unless a
                    // advances t; one in tag t - 1 comes in when a advances t - 1
                    const int tg = k % c.Tg;
                    const bool stay = !((adv >> tg) & 1u), inflow = tg >= 1 && ((adv >> (tg - 1)) & 1u);
                    auto rd = [&](int kk, int comp) {
                        return WAIT ? ld_relaxed_df(fbox_a(c, par, f.drv[j], kk)->v + comp)
                                    : ld_state_df(c.at + (size_t)f.drv[j] * K + kk, comp);
                    };
                    a0 = a1 = DF(absent);
                    if (stay) {
                        a0 = rd(k, el * 2);
                        a1 = rd(k, el * 2 + 1);
                    }
                    if (inflow) {
                        const DF b0 = rd(k - 1, el * 2), b1 = rd(k - 1, el * 2 + 1);
                        a0 = el ? df_max(a0, b0) : df_min(a0, b0);
                        a1 = el ? df_max(a1, b1) : df_min(a1, b1);
                    }
                    const float4 sd = WAIT ? ld_relaxed4(fbox_s(c, par, f.drv[j], k))
                                           : ld_state4(c.slew + (size_t)f.drv[j] * K + k);
                    s0 = el ? sd.z : sd.x;
                    s1 = el ? sd.w : sd.y;
                } else if (WAIT && PAIR && k == kq) {
                    a0 = in.at[j];
                    a1 = in.atp[j];
                    s0 = in.sl[j];
                    s1 = in.slp[j];
                } else if (WAIT && k == kq) {
                    const DF ap = shfl_xor_df(qm, in.at[j], 1);
                    const float sp = __shfl_xor_sync(qm, in.sl[j], 1);
                    a0 = rfo ? ap : in.at[j];
                    a1 = rfo ? in.at[j] : ap;
                    s0 = rfo ? sp : in.sl[j];
                    s1 = rfo ? in.sl[j] : sp;
                } else {
                    float4 sd;
                    if (!WAIT) {
                        a0 = ld_state_df(c.at + (size_t)f.drv[j] * K + k, el * 2);
                        a1 = ld_state_df(c.at + (size_t)f.drv[j] * K + k, el * 2 + 1);
                        sd = ld_state4(c.slew + (size_t)f.drv[j] * K + k);
                    } else {
                        DF x, y, zz, w;
                        ld_relaxed_df4(fbox_a(c, par, f.drv[j], k), x, y, zz, w);
                        a0 = el ? zz : x;
                        a1 = el ? w : y;
                        sd = ld_relaxed4(fbox_s(c, par, f.drv[j], k));
                    }
                    s0 = el ? sd.z : sd.x;
                    s1 = el ? sd.w : sd.y;
                }
                const float Dn = k != kq ? c.netD[(size_t)a * K + k] : f.Dn0[j];
                const float V = k != kq ? c.netV[(size_t)a * K + k] : f.V0[j];
                ain[j][0] = a0 + Dn;
                ain[j][1] = a1 + Dn;
                sin[j][0] = sqrt_hw(fmaf(s0, s0, V));
                sin[j][1] = sqrt_hw(fmaf(s1, s1, V));
                // lane q stores component q of the input pin: (el, rf = q & 1)
                st_comp_df(c.at + (size_t)a * K + k, q, rfo ? ain[j][1] : ain[j][0]);
                st_comp(c.slew + (size_t)a * K + k, q, rfo ? sin[j][1] : sin[j][0]);
            }
        }
        const float sc = lut.sc(k);
        const float ld = k != kq ? c.load[(size_t)z * K + k] : f.ld0;
        const Seg bl = seg_load<UNIFORM>(c, lut, tab_off(t, 0, 0), ld);
        // Candidates are merged in FP32 -- the input arrival's high part +
        // the arc delay -- and only the winner's sum is formed exactly: a
        // near-tie in FP32 can pick a candidate below the true maximum by at
        // most one FP32 rounding, and that error does not accumulate.
        MaxMerge<SMOOTH> ma, ms;
        DF win(0.f);
        float wd = 0.f, wy = -INFINITY;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j >= nin) continue;
            const int tbj = tab_off(t, j, 0);
            // the input edges with an arc to output edge rfo, in increasing
            // order: the one edge of a unate arc (rfo, or its opposite), both
            // of a non-unate one -- the same candidates in the same order as
            // testing arc_on for rfi = 0, 1, but without lanes of one quad
            // (which differ in rfo) diverging on a unate arc
            const int se = f.sense[j];
            const int n_rfi = se == kSenseNonC ? 2 : (se == kSensePosC || se == kSenseNegC) ? 1 : 0;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (r >= n_rfi) break;
                const int rfi = se == kSenseNonC ? r : (se == kSenseNegC ? 1 - rfo : rfo);
                const float s = rfi ? sin[j][1] : sin[j][0];
                const DF ai = rfi ? ain[j][1] : ain[j][0];
                const Seg as = seg_slew<UNIFORM>(c, lut, tbj, s);
                const float dv = lookup<UNIFORM>(lut, tbj + rfo * kLutStride, as, bl, s, ld);
                const float sv = lookup<UNIFORM>(lut, tbj + (2 + rfo) * kLutStride, as, bl, s, ld);
                const float d = sc * dv;
                const float y = sgn * (ai.hi + d);
                if (y > wy) {
                    wy = y;
                    win = ai;
                    wd = d;
                }
                ma.add(y, c.inv_gamma);
                ms.add(sgn * (sc * sv), c.inv_gamma);
            }
        }
        // the exact winner (no finite candidate: absent, -inf late / +inf
        // early), plus the log-sum-exp excess when smoothed
        DF oa(-sgn * INFINITY);   // no finite candidate
        if (wy > -INFINITY) {
            oa = win + wd;
            if (SMOOTH) oa = oa + sgn * (c.gamma * __logf(ma.s));
        }
        const float os = sgn * ms.get(c.gamma);
        st_comp_df(c.at + (size_t)z * K + k, q, oa);
        st_comp(c.slew + (size_t)z * K + k, q, os);
        if (pub) publish_fwd(c, par, g, k, q, oa, os);
        if (first && k == kq) *first = FwdOut{oa, os};
    }
}

// ------------------------------------------------------------ endpoints

struct EpItem {
    int p, d;   // the endpoint pin; its driver: pin, or (WAIT, the tile schedule) driver item
    bool isD;
    float Dn0, V0;
};

template <class Ctx>
__device__ __forceinline__ EpItem ep_prep(const Ctx &c, int e)
{
    EpItem x;
    e = chk(c, e, c.E);
    x.p = chk(c, c.ep_pin[e], c.P);
    x.d = chk(c, c.drv_of[x.p], c.P);
    x.isD = c.ep_is_d[e] != 0;
    x.Dn0 = c.netD[(size_t)x.p * nK(c) + corner_lane(c)];
    x.V0 = c.netV[(size_t)x.p * nK(c) + corner_lane(c)];
    return x;
}

// Arrival through the net, required times of the ideal clock (D: setup
// capture edge T - setup, hold 0 + hold; PO: T and 0), pin and endpoint
// slacks (min over rise/fall) and violation flags.  Lane q: component q.
template <bool WAIT, class Ctx = DevCtx>
__device__ __forceinline__ void ep_run(const Ctx &c, const EpItem &x, DF at0, float sl0, int e, int q,
                                       int par)
{
    const int K = nK(c), p = x.p, d = x.d;
    const unsigned m = quad_mask();
    const int base = threadIdx.x & 28;   // first lane of the quad
    const int kq = corner_lane(c);
    for (int k = kq; k < K; k += nKL(c)) {
        // requirement of state k: late = M T + off.x (M = 0: off.x alone),
        // early = off.y, from the exception tag's action (false path: no
        // check; multicycle: M; max delay: M = 0, off.x = V - setup; min
        // delay: off.y = V + hold); the default check without exceptions
        float M = 1.f;
        float2 off = make_float2(x.isD ? -c.setup : 0.f, x.isD ? c.hold : 0.f);
        if (c.Tg > 1) {
            M = c.ep_mult[(size_t)e * c.Tg + k % c.Tg];
            off = c.ep_off[(size_t)e * c.Tg + k % c.Tg];
        }
        const DF req = q >= 2 ? (M == 0.f ? DF(off.x) : df_mul(M, c.period) + off.x) : DF(off.y);
        DF ad;
        float sd;
        if (!WAIT) {
            ad = ld_state_df(c.at + (size_t)d * K + k, q);
            sd = ld_state(c.slew + (size_t)d * K + k, q);
        } else if (k == kq) {
            ad = at0;
            sd = sl0;
        } else {
            ad = ld_relaxed_df(fbox_a(c, par, d, k)->v + q);
            sd = ld_relaxed1(reinterpret_cast<const float *>(fbox_s(c, par, d, k)) + q);
        }
        const float Dn = k != kq ? c.netD[(size_t)p * K + k] : x.Dn0, V = k != kq ? c.netV[(size_t)p * K + k] : x.V0;
        const DF A = ad + Dn;
        st_comp_df(c.at + (size_t)p * K + k, q, A);
        st_comp(c.slew + (size_t)p * K + k, q, sqrt_hw(fmaf(sd, sd, V)));
        st_comp_df(c.rat + (size_t)p * K + k, q, req);
        const float sk = q >= 2 ? req - A : A - req;
        st_comp(c.slack + (size_t)p * K + k, q, sk);
        const float worst = fminf(sk, __shfl_xor_sync(m, sk, 1));   // min over the two edges
        const float ss = __shfl_sync(m, worst, base + 2), hs = __shfl_sync(m, worst, base);
        if (q == 0) {
            c.ep_setup[(size_t)e * K + k] = ss;
            c.ep_hold[(size_t)e * K + k] = hs;
            c.viol_setup[(size_t)e * K + k] = ss < 0.f;
            c.viol_hold[(size_t)e * K + k] = hs < 0.f;
        }
    }
}

// ------------------------------------------------------------- backward

struct BwdItem {
    int t, pin0, nin, kind, z, f0, f1;
    float ld0;
    // states of the lane's first corner, component q, loaded ahead (written
    // by the forward pass): arrival of the output, slew and arrival of each
    // input pin (CK: the slew of the rising component of this lane's el)
    DF az0, a0[3];
    float s0[3];
    // sink pins of the fan-out entries q, q + 4, q + 8, q + 12 (-1: none),
    // the ones the lane's probe reads first
    int sk[4];
    // each gate input's entry in its driver's fan-out list: where its
    // required time is published
    int fin[3];
};

template <class Ctx>
__device__ __forceinline__ BwdItem bwd_prep(const Ctx &c, const int *tnin, const int *tkind, int g, int q)
{
    BwdItem b;
    const int K = nK(c), kq = corner_lane(c);
    g = chk(c, g, c.I);
    b.t = chk_type(c, c.item_type[g]);
    b.pin0 = chk(c, c.item_pin0[g], c.P);
    b.kind = b.t >= 0 ? tkind[b.t] : -1;
    b.nin = b.t >= 0 ? tnin[b.t] : 0;
    b.z = chk(c, b.t < 0 ? b.pin0 : (b.kind == 1 ? b.pin0 + 1 : b.pin0 + b.nin), c.P);
    b.f0 = chk(c, c.fo_ptr[g], (long long)c.F + 1);
    b.f1 = chk(c, c.fo_ptr[g + 1], (long long)c.F + 1);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int e = q + 4 * u;
        b.sk[u] = e < b.f1 - b.f0 ? chk(c, __ldg(c.fo_pin + b.f0 + e), c.P) : -1;
    }
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
    return b;
}

// The backward fold split over the quad instead of over components: lane q
// folds fan-out entries q, q + 4, q + 8, ... for all four components (one
// 32-byte read per sink), keeping per component the extreme of RAT - Elmore
// delay, the entry index that holds it (the first on ties, as the sequential
// fold) and the winner's operands; quad_fold then reduces the four lanes.
// A driver with many sinks waits for a quarter of the round trips.
struct Fold4 {
    float v[4];
    int idx[4];
    DF rw[4];
    float rd[4];
};

__device__ __forceinline__ void fold4_clear(Fold4 &f)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        f.v[j] = j >= 2 ? INFINITY : -INFINITY;
        f.idx[j] = 0x7fffffff;
        f.rw[j] = DF(f.v[j]);
        f.rd[j] = 0.f;
    }
}

// Reduce the quad's folds: per component the extreme value, lowest entry on
// ties; lane q returns component q's required time (infinite when no sink
// constrains it).  Every lane of mask m calls it: the quad's own lanes, or
// the whole warp (m = all lanes) when the caller keeps it converged, which
// makes the shuffles cheaper; each quad still reduces only its own lanes.
__device__ __forceinline__ DF quad_fold(Fold4 &f, int q, unsigned m = quad_mask())
{
    const int base = threadIdx.x & 28;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int off = 1; off <= 2; off <<= 1) {
            const float ov = __shfl_xor_sync(m, f.v[j], off);
            const int oi = __shfl_xor_sync(m, f.idx[j], off);
            const bool take = (j >= 2 ? ov < f.v[j] : ov > f.v[j]) || (ov == f.v[j] && oi < f.idx[j]);
            if (take) {
                f.v[j] = ov;
                f.idx[j] = oi;
            }
        }
    }
    DF rw(0.f);
    float rd = 0.f, rf = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int src = base + (f.idx[j] == 0x7fffffff ? 0 : (f.idx[j] & 3));
        const DF w = shfl_df(m, f.rw[j], src);
        const float dd = __shfl_sync(m, f.rd[j], src);
        if (j == q) {
            rw = w;
            rd = dd;
            rf = f.v[j];
        }
    }
    return isfinite(rf) ? rw - rd : DF(rf);
}

// Are the required times of every sink of the item's net complete (all the
// lane's corners)?  The fold split over the quad (Fold4): lane q reads all
// four components of fan-out entries q, q + 4, ... (four at a time, their
// loads in flight together) for the lane's first corner.  The caller's group
// vote covers the quad, then quad_fold gives each lane its component's
// required time: R = min (late) / max (early) over the sinks of RAT - Elmore
// delay, the first extreme in fan-out order, its difference formed exactly.
// Endpoint sinks were set by the forward pass.
template <bool THRU = true, class Ctx = DevCtx>
__device__ __forceinline__ bool bwd_probe_split(const Ctx &c, const BwdItem &b, int par, int q, Fold4 &f)
{
    const uint32_t *pin_adv = THRU ? c.pin_adv : nullptr;
    const int K = nK(c), kq = corner_lane(c);
    fold4_clear(f);
    const int nfo = b.f1 - b.f0;
    for (int e0 = q; e0 < nfo; e0 += 16) {
        int s[4];
        DF m[4][4];
        float nd[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + 4 * u;
            // the first group's sinks were read ahead
            s[u] = e0 == q ? b.sk[u] : e < nfo ? chk(c, __ldg(c.fo_pin + b.f0 + e), c.P) : -1;
            nd[u] = 0.f;
            if (s[u] < 0) continue;
            const int ks = (pin_adv && ((pin_adv[s[u]] >> (kq % c.Tg)) & 1u)) ? kq + 1 : kq;
            if (s[u] < c.ep_begin) {
                ld_relaxed_df4(rbox_at(c, par, b.f0 + e, ks), m[u][0], m[u][1], m[u][2], m[u][3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) m[u][j] = ld_state_df(c.rat + (size_t)s[u] * K + ks, j);
            }
            nd[u] = __ldg(c.netD + (size_t)s[u] * K + kq);
        }
        bool ok = true;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (s[u] >= 0) ok = ok && real_df(m[u][0]) && real_df(m[u][1]) && real_df(m[u][2]) && real_df(m[u][3]);
        if (!ok) return false;   // no arithmetic while waiting
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (s[u] < 0) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float val = m[u][j].hi - nd[u];
                if (j >= 2 ? val < f.v[j] : val > f.v[j]) {
                    f.v[j] = val;
                    f.idx[j] = e0 + 4 * u;
                    f.rw[j] = m[u][j];
                    f.rd[j] = nd[u];
                }
            }
        }
    }
    // the lane's other states of its gate-input sinks
    if (K > nKL(c) || pin_adv) {
        for (int e = q; e < nfo; e += 4) {
            const int s = chk(c, __ldg(c.fo_pin + b.f0 + e), c.P);
            if (s >= c.ep_begin) continue;
            const int k0 = pin_adv ? 0 : kq + nKL(c), dk = pin_adv ? 1 : nKL(c);
            for (int k = k0; k < K; k += dk)
                if (k != kq && !complete_df(rbox_at(c, par, b.f0 + e, k))) return false;
        }
    }
    return true;
}

// Lane q = el*2 + rfi: the output's required time (component q) over its
// net sinks, then each input pin's over its arcs, and pin slacks.  With WAIT
// the first corner's output required time comes folded from the probe (Rpre).
// With `first` (the tile schedule's ring), the lane's first-corner required
// time of each input pin, component q, is returned there as well.
template <bool UNIFORM, bool WAIT, bool THRU = true, class L, class Ctx = DevCtx>
__device__ __forceinline__ void bwd_run(const Ctx &c, const L &lut, const int *tsense, const BwdItem &b, int q,
                                        int par, DF Rpre, DF *first = nullptr)
{
    const uint32_t *pin_adv = THRU ? c.pin_adv : nullptr;
    const int t = b.t, pin0 = b.pin0, z = b.z, K = nK(c);
    const int el = q >> 1, rfi = q & 1;
    const unsigned m = quad_mask();
    const int base = threadIdx.x & 28;
    const int kq = corner_lane(c);
    for (int k = kq; k < K; k += nKL(c)) {
        const bool first_k = k == kq;
        // required time of the output, component q, over its net sinks
        DF R(el ? INFINITY : -INFINITY);
        if (WAIT && first_k) {
            R = Rpre;
        } else {
            float rf = el ? INFINITY : -INFINITY, rd = 0.f;
            DF rw(rf);
            for (int p = b.f0; p < b.f1; ++p) {
                const int s = chk(c, c.fo_pin[p], c.P);
                const int ks = (pin_adv && ((pin_adv[s] >> (k % c.Tg)) & 1u)) ? k + 1 : k;
                const DF rs = (WAIT && s < c.ep_begin) ? ld_relaxed_df(rbox_at(c, par, p, ks)->v + q)
                                                       : ld_state_df(c.rat + (size_t)s * K + ks, q);
                const float nd = c.netD[(size_t)s * K + k];
                const float v = rs.hi - nd;
                if (el ? v < rf : v > rf) {
                    rf = v;
                    rw = rs;
                    rd = nd;
                }
            }
            if (isfinite(rf)) R = rw - rd;
        }
        st_comp_df(c.rat + (size_t)z * K + k, q, R);
        const DF Az = first_k ? b.az0 : ld_state_df(c.at + (size_t)z * K + k, q);
        st_comp(c.slack + (size_t)z * K + k, q, el ? R - Az : Az - R);
        if (t < 0) continue;
        // the output's required times of both edges at this lane's el
        const DF R0 = shfl_df(m, R, base + el * 2), R1 = shfl_df(m, R, base + el * 2 + 1);
        const float sc = lut.sc(k);
        const float ld = first_k ? b.ld0 : c.load[(size_t)z * K + k];
        if (b.kind == 1) {   // CK: only the rising edge has an arc (to both edges of Q)
            const int ck = pin0;
            const float s = first_k ? b.s0[0] : ld_state(c.slew + (size_t)ck * K + k, el * 2);
            const int tb = tab_off(t, 1, 0);
            const Seg as = seg_slew<UNIFORM>(c, lut, tb, s), bl = seg_load<UNIFORM>(c, lut, tb, ld);
            const float d0 = sc * lookup<UNIFORM>(lut, tb, as, bl, s, ld);
            const float d1 = sc * lookup<UNIFORM>(lut, tb + kLutStride, as, bl, s, ld);
            const float c0 = R0.hi - d0, c1 = R1.hi - d1;
            DF Rc = (el ? c1 < c0 : c1 > c0) ? R1 - d1 : R0 - d0;
            if (rfi == 1) Rc = DF(el ? INFINITY : -INFINITY);
            st_comp_df(c.rat + (size_t)ck * K + k, q, Rc);
            const DF Ac = first_k ? b.a0[0] : ld_state_df(c.at + (size_t)ck * K + k, q);
            st_comp(c.slack + (size_t)ck * K + k, q, el ? Rc - Ac : Ac - Rc);
            continue;
        }
        const Seg bl = seg_load<UNIFORM>(c, lut, tab_off(t, 0, 0), ld);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j >= b.nin) continue;
            const int a = pin0 + j;
            const int se = tsense[t * 3 + j];
            const int tbj = tab_off(t, j, 0);
            const float s = first_k ? b.s0[j] : ld_state(c.slew + (size_t)a * K + k, q);
            const Seg as = seg_slew<UNIFORM>(c, lut, tbj, s);
            // FP32 choice between the (at most two) arcs, the winner exactly;
            // the output edges with an arc from input edge rfi in increasing
            // order (one for a unate arc, both for a non-unate one: no lane
            // divergence inside a quad)
            float af = el ? INFINITY : -INFINITY, ad = 0.f;
            DF aw(af);
            const int n_rfo = se == kSenseNonC ? 2 : (se == kSensePosC || se == kSenseNegC) ? 1 : 0;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (r >= n_rfo) break;
                const int rfo = se == kSenseNonC ? r : (se == kSenseNegC ? 1 - rfi : rfi);
                const float d = sc * lookup<UNIFORM>(lut, tbj + rfo * kLutStride, as, bl, s, ld);
                const DF Ro = rfo ? R1 : R0;
                const float v = Ro.hi - d;
                if (el ? v < af : v > af) {
                    af = v;
                    aw = Ro;
                    ad = d;
                }
            }
            const DF acc = isfinite(af) ? aw - ad : DF(af);
            st_comp_df(c.rat + (size_t)a * K + k, q, acc);
            const DF Aa = first_k ? b.a0[j] : ld_state_df(c.at + (size_t)a * K + k, q);
            st_comp(c.slack + (size_t)a * K + k, q, el ? acc - Aa : Aa - acc);
            if (WAIT) publish_rat(c, par, b.fin[j], k, q, acc);
            if (first && first_k) first[j] = acc;
        }
    }
}

}  // namespace sta
