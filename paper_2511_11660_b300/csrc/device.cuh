// device.cuh -- device-side data of a timing context and the per-arc math.
//
// Per-pin state is float4 per (pin, corner): components x, y, z, w =
// early-rise, early-fall, late-rise, late-fall (index el*2 + rf).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sta {

constexpr int kLutStride = 80;   // floats per packed table, see plan.cpp
constexpr int kNetArnoldi = 1;     // DevCtx::net_model of the reduced-order calculator (STA_NET_ARNOLDI)
constexpr int kRcColNodes = 10;    // RC nets up to this size are swept in shared memory (as plan.h)
constexpr int kRcThreads = 128;    // threads (nets) per block of the RC sweep
constexpr int kStMaxPins = 64;     // nets of more pins keep the rectilinear MST (plan.h: kSteinerMaxPins)
constexpr int kRedThreads = 256;   // threads of the reduction kernels
constexpr int kDfStateWords = 16;  // schedule state words (see DevCtx::df_state)
constexpr int kRedChunk = 1024;    // endpoints per first-stage reduction block
static_assert(kRedChunk % kRedThreads == 0, "a reduction thread folds a whole number of endpoints");

// device error word bits (sta_sync maps them to sta_status)
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrBounds = 2u;
constexpr unsigned kErrResize = 4u;

// Arrival and required times are double-float values: an unevaluated sum
// hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2), ~48 significant bits.
// Each level adds a delay to them, and plain FP32 would round at every
// level -- over a deep design the rounding alone reaches the 1e-4 ns parity
// bound once arrivals pass ~20 ns -- while B300's FP64 pipe is too narrow
// for the per-item critical path; these sums run on the FP32 pipe.  Slews,
// slacks and every delay stay FP32.
struct DF {
    float hi, lo;
    DF() = default;
    __host__ __device__ __forceinline__ DF(float x) : hi(x), lo(0.f) {}
    __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
};
// a + b, b an FP32 number: the error-free sum of the high parts (Knuth's
// two-sum), the low parts added, then renormalised (Dekker's fast two-sum).
// Infinite sums (absent arrivals, unconstrained required times) stay exact.
__device__ __forceinline__ DF operator+(DF a, float b)
{
    const float s = __fadd_rn(a.hi, b);
    if (!isfinite(s)) return DF(s, 0.f);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    const float l = __fadd_rn(e, a.lo);
    const float t = __fadd_rn(s, l);
    return DF(t, __fsub_rn(l, __fsub_rn(t, s)));
}
__device__ __forceinline__ DF operator-(DF a, float b) { return a + (-b); }
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
// sign times a value, sign = +1 or -1 (exact)
__device__ __forceinline__ DF operator*(float sgn, DF a) { return DF(sgn * a.hi, sgn * a.lo); }
// a - b rounded to FP32 (slacks, smoothing exponents)
__device__ __forceinline__ float operator-(DF a, DF b)
{
    return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}
__device__ __forceinline__ bool operator>(DF a, DF b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(DF a, DF b) { return b > a; }
__device__ __forceinline__ DF df_max(DF a, DF b) { return b > a ? b : a; }
__device__ __forceinline__ DF df_min(DF a, DF b) { return b < a ? b : a; }
__device__ __forceinline__ float to_f(DF a) { return __fadd_rn(a.hi, a.lo); }
// a * b exactly as a double-float (the product's rounding error by FMA)
__device__ __forceinline__ DF df_mul(float a, float b)
{
    const float p = __fmul_rn(a, b);
    if (!isfinite(p)) return DF(p, 0.f);
    return DF(p) + fmaf(a, b, -p);
}
__device__ __forceinline__ DF shfl_xor_df(unsigned mask, DF v, int lane)
{
    return DF(__shfl_xor_sync(mask, v.hi, lane), __shfl_xor_sync(mask, v.lo, lane));
}
__device__ __forceinline__ DF shfl_df(unsigned mask, DF v, int src)
{
    return DF(__shfl_sync(mask, v.hi, src), __shfl_sync(mask, v.lo, src));
}

struct __align__(32) DF4 {
    DF v[4];
};

struct DevCtx {
    int32_t P, I, S, E, K, T, C, n_designs;
    int32_t KL;                                 // quads per item: states handled side by side (1, 2, 4 or 8)
    int32_t Kc, Tg;                             // corners and exception tags: K = Kc * Tg states, k = corner * Tg + tag
    const int32_t *item_tag;                    // [I] tag of a startpoint item (Tg > 1)
    const float *ep_mult;                       // [E][Tg] setup multiplier per endpoint and tag, 0 = no check (Tg > 1)
    const float2 *ep_off;                       // [E][Tg] late requirement offset, early requirement (Tg > 1)
    const uint32_t *pin_adv;                    // [P] bit t: tag t moves on to t + 1 at this gate input (-through; or NULL)
    int64_t NN;                                 // RC nodes
    int32_t F;                                  // net sinks (fan-out entries)
    int32_t net_model, arnoldi_q;               // STA_NET_ELMORE / STA_NET_ARNOLDI and its order
    float period, clk_slew, pi_at, pi_slew, setup, hold, gamma, inv_gamma;
    float r_per_um, c_per_um;
    const float *lut;          // [T][3][4][80]
    const int32_t *type_nin, *type_kind, *arc_sense;
    const float *lut_scale, *rc_scale;          // [K]
    const int32_t *item_pin0, *item_type, *item_cell;
    const int32_t *item_drv;                    // [I][3] the item driving each gate input (0 where none)
    const int32_t *pin_fo;                      // [P] a gate input's entry in its driver's fan-out list (-1: none)
    const int32_t *fo_ptr, *fo_pin, *fo_node;   // sinks of each item's output net
    const int32_t *fo_item;                     // [F] item of each fan-out entry (differentiable star RC)
    const float *fo_cap;
    const int32_t *rc_ptr, *rc_parent;
    const float *rc_R, *rc_C;
    // Steiner trees from positions (STA_WIRE_STEINER): the tree kernel writes
    // the RC arrays above (through these aliases), the sinks' nodes and the
    // live node count of every item; working storage per item
    int32_t steiner;
    float r_per_um_y, c_per_um_y;
    int32_t *st_parent, *st_fo_node, *st_nlive;
    int2 *st_src;                               // [NN] differentiable contexts: per RC node, for x and y,
                                                // (pin << 2) | (sign of node - parent + 1), pin = the
                                                // lowest net pin (0 = driver) at that coordinate
    float *st_R, *st_C;
    int64_t *st_wl;                             // [I] tree length, nm
    const int64_t *st_node_ptr, *st_adj_ptr;    // [I + 1] working nodes / bitset words per item
    long long *st_x, *st_y, *st_key;            // [working nodes] coordinates (nm), Prim keys
    int32_t *st_aux;                            // [working nodes x 3] Prim source / BFS number / queue
    float *st_capw;                             // [working nodes] RC node capacitances being accumulated
    const int32_t *st_items;                    // items with sinks by increasing sink count
    int32_t st_n_items, st_small;               // their number; the first st_small have <= 8 pins
    int32_t st_adj_tiny, st_adj_small;          // the first st_adj_tiny have <= 5 pins, st_adj_small <= 9 (adjoint)
    unsigned *st_adj;                           // [bitset words] adjacency rows
    const int32_t *drv_of, *pin_cell;
    const float *port_xy, *cell_xy;
    const int32_t *ep_pin, *ep_design_ptr;
    const uint8_t *ep_is_d;
    DF4 *at, *rat;                              // [P*K] arrival and required times (double-float)
    float4 *slew, *slack;                       // [P*K]
    float *netD, *netV, *load;                  // [P*K]
    float *ep_setup, *ep_hold;                  // [E*K]
    uint8_t *viol_setup, *viol_hold;            // [E*K]
    double *report;                             // [n_designs][K][8]
    const int32_t *red_chunk_ptr;               // [n_red_chunks+1] endpoint ranges
    const int32_t *red_design_chunk;            // [n_designs+1] chunk ranges per design
    double *red_partial;                        // [n_red_chunks][K][6] scratch
    unsigned *err;
    float *scratch_a, *scratch_b, *scratch_c;   // [K][NN] RC sweeps of nets larger than kRcColNodes
    // dataflow schedule: mailboxes by epoch parity, NaN until published
    DF4 *fbox_a;                                // [2][P][K] arrival of driver pins
    float4 *fbox_s;                             // [2][P][K] slew of driver pins
    DF4 *rbox;                                  // [F][K][2] required time of gate input pins, by fan-out entry
    size_t fbox_len, rbox_len;                  // records of fbox_a (= of fbox_s) and of rbox
    unsigned *df_state;                         // [kDfStateWords] [0] epoch, [1] forward chunk counter,
                                                // [2] backward counter, [3] abort; adjoint: [4] epoch,
                                                // [5] chunk counter, [6] abort; [7] grid-barrier arrivals
    int32_t ep_begin;                           // first endpoint pin (endpoints are the last E pins)
    int32_t hold_item;                          // test hook: item whose forward flag is never published (-1 none)
    long long spin_limit;                       // polls before a wait gives up
    int32_t n_fwd_chunks, n_bwd_chunks;
    const int32_t *stage_ptr;                   // [S+1] item offsets of the levels (cooperative schedule)
    const int32_t *fwd_chunk_lo, *fwd_chunk_hi;   // forward work: items by level, then endpoints (index I + e)
    const int32_t *bwd_chunk_lo, *bwd_chunk_hi;   // backward work: positions of bwd_order, deepest level first
    const int32_t *bwd_order;                   // [I] items in backward work order
    // tile schedule (tile.cu): per-block lists of items and endpoints by step
    int32_t tl_B, tl_NS, tl_R;                  // tiles, steps, ring slots per block
    const int32_t *tl_ptr;                      // [B*NS + 1] list (b, s) = entries [tl_ptr[b*NS+s], ...+1)
    const int32_t *tl_nitem;                    // [B*NS] items at the front of list (b, s), endpoints after
    const int32_t *tl_rbase;                    // [B*NS] backward ring position of list (b, s)'s first item
    const int4 *tl_fdesc;                       // [(I + E) * 2] forward descriptor of every list entry
    const int4 *tl_bdesc;                       // [(I + E) * 4] backward descriptor of every item entry
    const int16_t *tl_fo_ring;                  // [F] backward ring code of a fan-out entry, -1 = mailbox
    // differentiable pass (sta_backward)
    float4 *adj;                                // [P][K] late adjoints: dJ/dAT rise, fall, dJ/dslew rise, fall
    float4 *abox;                               // [P][K][2] the same for gate input pins, parity mailbox
    size_t abox_len;
    double *obj;                                // [K][4] max(-s/g), sum exp(-s/g - max), TNS_g, WNS_g; [4K] J
    float *aload;                               // [I][K] dJ/dload of each item's output net
    double *grad;                               // [C][2] dJ/d(x, y)
    float *st_abuf;                             // [kAdjArrays][NN] Steiner adjoint storage of trees above
                                                // kAdjColNodes nodes
    double w_tns, w_wns;
    // shared table axes (valid when every table has the same ones): slew and
    // load breakpoints and reciprocal segment widths
    float ax1[7], ax2[7], iw1[6], iw2[6];
};

// A context with one state per pin and one corner per lane group (K = KL =
// 1: one corner, no exception tags), known at compile time.  The per-item
// functions read the state counts through nK / nKL, so the kernels built for
// this type carry no other-states loops, checks or index arithmetic: a
// polling round and an item's run issue fewer instructions.  Made by copying
// a DevCtx whose K and KL are 1.
struct DevCtxOne : DevCtx {};
__device__ __forceinline__ int nK(const DevCtx &c) { return c.K; }
__device__ __forceinline__ int nK(const DevCtxOne &) { return 1; }
__device__ __forceinline__ int nKL(const DevCtx &c) { return c.KL; }
__device__ __forceinline__ int nKL(const DevCtxOne &) { return 1; }

// Debug builds (-DSTA_CHECKS) range-check every index a kernel derives from
// plan data: out of range records kErrBounds in the device error word and
// yields 0 (or -1 for a cell type), so the access that follows stays in
// bounds.  In normal builds both are the identity.
__device__ __forceinline__ int chk(const DevCtx &c, long long i, long long n)
{
#ifdef STA_CHECKS
    if (i < 0 || i >= n) {
        atomicOr(c.err, kErrBounds);
        return 0;
    }
#endif
    return (int)i;
}
__device__ __forceinline__ int chk_type(const DevCtx &c, int t)
{
#ifdef STA_CHECKS
    if (t < -1 || t >= c.T) {
        atomicOr(c.err, kErrBounds);
        return -1;
    }
#endif
    return t;
}

// arc senses as the kernels see them
constexpr int kSensePosC = 0, kSenseNegC = 1, kSenseNonC = 2, kSenseRiseC = 3;

__device__ __forceinline__ float comp(const float4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Running max of candidates y (callers pass y = x for a late max and y = -x
// for an early min, and negate the result back).  SMOOTH replaces the max by
// gamma * log-sum-exp(y / gamma), accumulated max-shifted.
template <bool SMOOTH, class T = float>
struct MaxMerge {
    T m = -INFINITY;
    float s = 0.f;
    __device__ __forceinline__ void add(T y, float inv_g)
    {
        if (!SMOOTH) {
            m = y > m ? y : m;
        } else if (!(y > -INFINITY)) {
            // an absent candidate (another exception tag's arrival): no term
        } else {
            // one exponential of -|y - m| / gamma, whichever of the two is
            // larger, and selects: no branch on the values, which differ
            // between the lanes of a warp (-|y - m| is m - y, or y - m,
            // exactly: IEEE subtraction rounds symmetrically).  The hardware
            // exponential (__expf) errs by a few ulp near 0 and more only
            // where the term is negligible beside s >= 1.
            const float e = __expf(-fabsf((float)(y - m)) * inv_g);
            const bool up = y > m;
            s = up ? s * e + 1.f : s + e;
            m = up ? y : m;
        }
    }
    // __logf of s in [1, candidates]: absolute error below 1e-6, times gamma
    __device__ __forceinline__ T get(float g) const { return SMOOTH ? m + g * __logf(s) : m; }
};

__device__ __forceinline__ int item_out_pin(const DevCtx &c, int t, int pin0)
{
    if (t < 0) return pin0;
    return __ldg(c.type_kind + t) == 1 ? pin0 + 1 : pin0 + __ldg(c.type_nin + t);
}

// position of a pin (um): its cell's, or its port's for a PI / PO
__device__ __forceinline__ float2 pin_pos(const DevCtx &c, int p)
{
    const int pc = c.pin_cell[chk(c, p, c.P)];
    if (pc >= 0) {
        const int cc = chk(c, pc, c.C);
        return make_float2(c.cell_xy[2 * (size_t)cc], c.cell_xy[2 * (size_t)cc + 1]);
    }
    const int q = -pc - 1;
    return make_float2(c.port_xy[2 * (size_t)q], c.port_xy[2 * (size_t)q + 1]);
}

}  // namespace sta
