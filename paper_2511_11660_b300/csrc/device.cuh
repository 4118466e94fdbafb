// device.cuh -- device-side data of a timing context and the per-arc math.
//
// Per-pin state is float4 per (pin, corner): components x, y, z, w =
// early-rise, early-fall, late-rise, late-fall (index el*2 + rf).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sta {

constexpr int kLutStride = 80;   // floats per packed table, see plan.cpp
constexpr int kRcTileNodes = 2048;
constexpr int kRcTileNets = 128;
constexpr int kRedThreads = 256;   // threads of the reduction kernels
constexpr int kRedChunk = 4096;    // endpoints per first-stage reduction block

// device error word bits (sta_sync maps them to sta_status)
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrBounds = 2u;

struct DevCtx {
    int32_t P, I, S, E, K, T, C, n_designs;
    float period, clk_slew, pi_at, pi_slew, setup, hold, gamma, inv_gamma;
    float r_per_um, c_per_um;
    const float *lut;          // [T][3][4][80]
    const int32_t *type_nin, *type_kind, *arc_sense;
    const float *lut_scale, *rc_scale;          // [K]
    const int32_t *item_pin0, *item_type, *item_cell;
    const int32_t *fo_ptr, *fo_pin, *fo_node;   // sinks of each item's output net
    const float *fo_cap;
    const int32_t *rc_ptr, *rc_parent, *tile_item;
    const float *rc_R, *rc_C;
    const int32_t *drv_of, *pin_cell;
    const float *port_xy, *cell_xy;
    const int32_t *ep_pin, *ep_design_ptr;
    const uint8_t *ep_is_d;
    float4 *at, *slew, *rat, *slack;            // [P*K]
    float *netD, *netV, *load;                  // [P*K]
    float *ep_setup, *ep_hold;                  // [E*K]
    uint8_t *viol_setup, *viol_hold;            // [E*K]
    double *report;                             // [n_designs][K][8]
    const int32_t *red_chunk_ptr;               // [n_red_chunks+1] endpoint ranges
    const int32_t *red_design_chunk;            // [n_designs+1] chunk ranges per design
    double *red_partial;                        // [n_red_chunks][K][6] scratch
    unsigned *err;
    float *scratch_a, *scratch_b;               // RC sweeps of nets larger than a tile
};

__device__ __forceinline__ float comp(const float4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// NLDM bilinear lookup (segment = number of interior breakpoints <= query,
// so queries off the table extrapolate from the edge segment).  Packed table:
// idx1[0..6] idx2[7..13] 1/width1[14..19] 1/width2[20..25] val[26..74].
__device__ __forceinline__ float lut_eval(const float *__restrict__ tb, float s, float l)
{
    const int i = (s >= __ldg(tb + 1)) + (s >= __ldg(tb + 2)) + (s >= __ldg(tb + 3)) + (s >= __ldg(tb + 4)) +
                  (s >= __ldg(tb + 5));
    const int j = (l >= __ldg(tb + 8)) + (l >= __ldg(tb + 9)) + (l >= __ldg(tb + 10)) + (l >= __ldg(tb + 11)) +
                  (l >= __ldg(tb + 12));
    const float t = (s - __ldg(tb + i)) * __ldg(tb + 14 + i);
    const float u = (l - __ldg(tb + 7 + j)) * __ldg(tb + 20 + j);
    const float *v = tb + 26 + i * 7 + j;
    const float v00 = __ldg(v), v01 = __ldg(v + 1), v10 = __ldg(v + 7), v11 = __ldg(v + 8);
    const float a = fmaf(u, v01 - v00, v00);
    const float b = fmaf(u, v11 - v10, v10);
    return fmaf(t, b - a, a);
}

// Same lookup, also returning d/ds and d/dl.
__device__ __forceinline__ float lut_eval_d(const float *__restrict__ tb, float s, float l, float &ds, float &dl)
{
    const int i = (s >= __ldg(tb + 1)) + (s >= __ldg(tb + 2)) + (s >= __ldg(tb + 3)) + (s >= __ldg(tb + 4)) +
                  (s >= __ldg(tb + 5));
    const int j = (l >= __ldg(tb + 8)) + (l >= __ldg(tb + 9)) + (l >= __ldg(tb + 10)) + (l >= __ldg(tb + 11)) +
                  (l >= __ldg(tb + 12));
    const float w1 = __ldg(tb + 14 + i), w2 = __ldg(tb + 20 + j);
    const float t = (s - __ldg(tb + i)) * w1;
    const float u = (l - __ldg(tb + 7 + j)) * w2;
    const float *v = tb + 26 + i * 7 + j;
    const float v00 = __ldg(v), v01 = __ldg(v + 1), v10 = __ldg(v + 7), v11 = __ldg(v + 8);
    const float a = fmaf(u, v01 - v00, v00);
    const float b = fmaf(u, v11 - v10, v10);
    ds = (b - a) * w1;
    dl = ((1.f - t) * (v01 - v00) + t * (v11 - v10)) * w2;
    return fmaf(t, b - a, a);
}

// Running merge of candidates: LATE keeps the max, early the min; SMOOTH
// replaces both by gamma * log-sum-exp (max-shifted).
template <bool LATE, bool SMOOTH>
struct Merge {
    float m, s;
    __device__ __forceinline__ Merge() : m(LATE ? -INFINITY : INFINITY), s(0.f) {}
    __device__ __forceinline__ void add(float x, float inv_g)
    {
        if (!SMOOTH) {
            m = LATE ? fmaxf(m, x) : fminf(m, x);
        } else {
            const float y = LATE ? x : -x, mm = LATE ? m : -m;
            if (y > mm) {
                s = s * expf((mm - y) * inv_g) + 1.f;
                m = x;
            } else {
                s += expf((y - mm) * inv_g);
            }
        }
    }
    __device__ __forceinline__ float get(float g) const
    {
        if (!SMOOTH) return m;
        return LATE ? m + g * logf(s) : m - g * logf(s);
    }
};

__device__ __forceinline__ int item_out_pin(const DevCtx &c, int t, int pin0)
{
    if (t < 0) return pin0;
    return __ldg(c.type_kind + t) == 1 ? pin0 + 1 : pin0 + __ldg(c.type_nin + t);
}

__device__ __forceinline__ const float *table(const DevCtx &c, int t, int slot, int tb)
{
    return c.lut + ((size_t)(t * 3 + slot) * 4 + tb) * kLutStride;
}

}  // namespace sta
