// adjoint.cu -- gradient of the smoothed WNS/TNS objective with respect to
// every cell position, by a hand-written reverse sweep of the forward pass.
//
// Objective (per corner k, summed over corners): endpoint setup slack
//   s_e = smin_g over rise/fall of (RAT_e - AT_late,e),
//   TNS_g = -sum_e g softplus(-s_e / g),   WNS_g = -g log sum_e exp(-s_e / g),
//   J = w_tns TNS_g + w_wns WNS_g.
// The forward pass in differentiable mode merges with g log-sum-exp, so J is
// smooth almost everywhere.  The reverse sweep walks the levels backwards:
// an item gathers the adjoints of its net's sinks (Elmore delay and the
// sqrt(s^2 + var) slew law), differentiates its output merges (softmax
// weights) and NLDM lookups (bilinear partials in slew and load), writes
// its input pins' adjoints, and scatters the derivative of every star
// segment length L = |dx| + |dy| to the two cells it joins:
//   dJ/dL = D_bar 1e-6 dD/dL + var_bar 1e-12 2 D dD/dL + load_bar 1e-3 c,
//   D = r L (c L / 2 + Cpin) [Ohm fF], dD/dL = r (c L + Cpin).
// The objective sums are FP64; the gradient accumulates with FP64 atomics.
// Placement-driven timing optimisation consumes such gradients (the paper's
// DREAMPlace integration uses pin slacks, Sec. IV-C); the paper itself has
// no differentiable mode.
#include "item.cuh"
#include "kernels.h"

namespace sta {

static inline int nblk2(long long n, int t) { return (int)((n + t - 1) / t); }

// smooth min of the two edges' setup margins of endpoint e at corner k (FP64)
__device__ __forceinline__ double ep_smooth_slack(const DevCtx &c, int e, int k, double y[2])
{
    const int p = c.ep_pin[e];
    const double req = c.ep_is_d[e] ? (double)c.period - c.setup : (double)c.period;
    const float4 a = c.at[(size_t)p * c.K + k];
    y[0] = req - a.z;
    y[1] = req - a.w;
    const double g = c.gamma, m = fmin(y[0], y[1]);
    return m - g * log(exp((m - y[0]) / g) + exp((m - y[1]) / g));
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}
template <int NT>
__device__ __forceinline__ double block_max(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// stage 1: per chunk and corner, max of -s_e / g
__global__ void __launch_bounds__(kRedThreads) k_obj_max_chunks(const DevCtx c)
{
    __shared__ double sh[kRedThreads];
    const int b = blockIdx.x, k = blockIdx.y;
    double v = -INFINITY;
    for (int e = c.red_chunk_ptr[b] + threadIdx.x; e < c.red_chunk_ptr[b + 1]; e += kRedThreads) {
        double y[2];
        v = fmax(v, -ep_smooth_slack(c, e, k, y) / c.gamma);
    }
    v = block_max<kRedThreads>(v, sh);
    if (threadIdx.x == 0) c.red_partial[((size_t)b * c.K + k) * 6] = v;
}

// stage 2: per corner, the global max
__global__ void __launch_bounds__(kRedThreads) k_obj_max_final(const DevCtx c, int nb)
{
    __shared__ double sh[kRedThreads];
    const int k = blockIdx.x;
    double v = -INFINITY;
    for (int b = threadIdx.x; b < nb; b += kRedThreads) v = fmax(v, c.red_partial[((size_t)b * c.K + k) * 6]);
    v = block_max<kRedThreads>(v, sh);
    if (threadIdx.x == 0) c.obj[k * 4 + 0] = v;
}

// stage 3: per chunk and corner, sum exp(-s/g - max) and the TNS terms
__global__ void __launch_bounds__(kRedThreads) k_obj_sum_chunks(const DevCtx c)
{
    __shared__ double sh[kRedThreads];
    const int b = blockIdx.x, k = blockIdx.y;
    const double mx = c.obj[k * 4 + 0], g = c.gamma;
    double se = 0, st = 0;
    for (int e = c.red_chunk_ptr[b] + threadIdx.x; e < c.red_chunk_ptr[b + 1]; e += kRedThreads) {
        double y[2];
        const double s = ep_smooth_slack(c, e, k, y);
        se += exp(-s / g - mx);
        const double z = -s / g;   // softplus(z) = max(z, 0) + log1p(exp(-|z|))
        st += -g * (fmax(z, 0.0) + log1p(exp(-fabs(z))));
    }
    se = block_sum<kRedThreads>(se, sh);
    st = block_sum<kRedThreads>(st, sh);
    if (threadIdx.x == 0) {
        c.red_partial[((size_t)b * c.K + k) * 6 + 1] = se;
        c.red_partial[((size_t)b * c.K + k) * 6 + 2] = st;
    }
}

// stage 4: per corner lse and TNS_g, WNS_g; then J
__global__ void __launch_bounds__(kRedThreads) k_obj_final(const DevCtx c, int nb)
{
    __shared__ double sh[kRedThreads];
    const int k = blockIdx.x;
    double se = 0, st = 0;
    for (int b = threadIdx.x; b < nb; b += kRedThreads) {
        se += c.red_partial[((size_t)b * c.K + k) * 6 + 1];
        st += c.red_partial[((size_t)b * c.K + k) * 6 + 2];
    }
    se = block_sum<kRedThreads>(se, sh);
    st = block_sum<kRedThreads>(st, sh);
    if (threadIdx.x == 0) {
        c.obj[k * 4 + 1] = se;
        c.obj[k * 4 + 2] = st;
        c.obj[k * 4 + 3] = se > 0 ? -(double)c.gamma * (c.obj[k * 4 + 0] + log(se)) : 0.0;
    }
}

__global__ void k_obj_total(const DevCtx c)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double J = 0;
        for (int k = 0; k < c.K; ++k) J += c.w_tns * c.obj[k * 4 + 2] + c.w_wns * c.obj[k * 4 + 3];
        c.obj[c.K * 4] = J;
    }
}

// dJ/dAT_late at every endpoint (slew adjoints are zero there)
__global__ void k_adj_seed(const DevCtx c)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.E) return;
    const int p = c.ep_pin[e];
    const double g = c.gamma;
    for (int k = 0; k < c.K; ++k) {
        double y[2];
        const double s = ep_smooth_slack(c, e, k, y);
        const double z = -s / g;
        const double sig = z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
        const double dj = c.w_tns * sig + c.w_wns * exp(-s / g - c.obj[k * 4 + 0]) / c.obj[k * 4 + 1];
        const double w0 = exp((s - y[0]) / g), w1 = exp((s - y[1]) / g);
        c.adj[(size_t)p * c.K + k] = make_float4((float)(-dj * w0), (float)(-dj * w1), 0.f, 0.f);
    }
}

__device__ __forceinline__ float2 pos_of(const DevCtx &c, int p)
{
    const int pc = c.pin_cell[p];
    if (pc >= 0) return make_float2(c.cell_xy[2 * (size_t)pc], c.cell_xy[2 * (size_t)pc + 1]);
    const int q = -pc - 1;
    return make_float2(c.port_xy[2 * (size_t)q], c.port_xy[2 * (size_t)q + 1]);
}

// One item of the reverse sweep (one thread per item, all corners).
template <bool UNIFORM>
__device__ void adj_item(const DevCtx &c, int g)
{
    const LutGlobal lut{c.lut};
    const int t = c.item_type[g];
    const int pin0 = c.item_pin0[g];
    const int kind = t >= 0 ? __ldg(c.type_kind + t) : -1;
    const int nin = kind == 0 ? __ldg(c.type_nin + t) : 0;
    const int z = t < 0 ? pin0 : (kind == 1 ? pin0 + 1 : pin0 + nin);
    const int f0 = c.fo_ptr[g], f1 = c.fo_ptr[g + 1];
    const int K = c.K;
    const float ig = c.inv_gamma;
    const float2 pz = pos_of(c, z);
    const int cz = c.pin_cell[z];
    for (int k = 0; k < K; ++k) {
        const float fk = __ldg(c.rc_scale + k);
        const float r = fk * c.r_per_um, cc = fk * c.c_per_um;
        const float4 Sz = c.slew[(size_t)z * K + k];
        // gather the sinks' adjoints through the net arcs
        float aA[2] = {0.f, 0.f}, aS[2] = {0.f, 0.f};
        for (int q = f0; q < f1; ++q) {
            const int s = c.fo_pin[q];
            const float4 as = c.adj[(size_t)s * K + k];
            const float4 Ss = c.slew[(size_t)s * K + k];
            aA[0] += as.x;
            aA[1] += as.y;
            aS[0] += as.z * Sz.z / Ss.z;
            aS[1] += as.w * Sz.w / Ss.w;
        }
        // through the output merges and the NLDM lookups
        float aload = 0.f;
        if (t >= 0) {
            const float sc = __ldg(c.lut_scale + k);
            const float ld = c.load[(size_t)z * K + k];
            if (kind == 1) {
                const float cs = c.slew[(size_t)pin0 * K + k].z;
                const int tb = tab_off(t, 1, 0);
                for (int rfo = 0; rfo < 2; ++rfo) {
                    float dds, ddl, sds, sdl;
                    const int td = tb + rfo * kLutStride, ts = tb + (2 + rfo) * kLutStride;
                    interp_d(lut, td, seg_slew<UNIFORM>(c, lut, td, cs), seg_load<UNIFORM>(c, lut, td, ld), dds, ddl);
                    interp_d(lut, ts, seg_slew<UNIFORM>(c, lut, ts, cs), seg_load<UNIFORM>(c, lut, ts, ld), sds, sdl);
                    aload += aA[rfo] * sc * ddl + aS[rfo] * sc * sdl;
                }
            } else {
                float aAin[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                float aSin[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                float4 Ain[3], Sin[3];
                int sense[3];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (j < nin) {
                        Ain[j] = c.at[(size_t)(pin0 + j) * K + k];
                        Sin[j] = c.slew[(size_t)(pin0 + j) * K + k];
                        sense[j] = __ldg(c.arc_sense + t * 3 + j);
                    }
                }
#pragma unroll
                for (int rfo = 0; rfo < 2; ++rfo) {
                    float xa[6], xs[6], dds[6], ddl[6], sds[6], sdl[6];
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        xa[i] = xs[i] = -INFINITY;
                        dds[i] = ddl[i] = sds[i] = sdl[i] = 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        if (j >= nin) continue;
                        const int tbj = tab_off(t, j, 0);
#pragma unroll
                        for (int rfi = 0; rfi < 2; ++rfi) {
                            const bool on = arc_on(sense[j], rfi, rfo);
                            const float s = comp(Sin[j], 2 + rfi);
                            const int td = tbj + rfo * kLutStride, ts = tbj + (2 + rfo) * kLutStride;
                            float dv = 0.f, sv = 0.f, a = 0.f, b = 0.f, e2 = 0.f, f2 = 0.f;
                            if (on) {
                                dv = interp_d(lut, td, seg_slew<UNIFORM>(c, lut, td, s), seg_load<UNIFORM>(c, lut, td, ld), a, b);
                                sv = interp_d(lut, ts, seg_slew<UNIFORM>(c, lut, ts, s), seg_load<UNIFORM>(c, lut, ts, ld), e2, f2);
                            }
                            const int i = j * 2 + rfi;
                            xa[i] = on ? comp(Ain[j], 2 + rfi) + sc * dv : -INFINITY;
                            xs[i] = on ? sc * sv : -INFINITY;
                            dds[i] = a;
                            ddl[i] = b;
                            sds[i] = e2;
                            sdl[i] = f2;
                        }
                    }
                    // softmax weights of the log-sum-exp merges
                    float ma = -INFINITY, ms = -INFINITY;
#pragma unroll
                    for (int i = 0; i < 6; ++i) { ma = fmaxf(ma, xa[i]); ms = fmaxf(ms, xs[i]); }
                    float za = 0.f, zs = 0.f;
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        za += xa[i] > -INFINITY ? expf((xa[i] - ma) * ig) : 0.f;
                        zs += xs[i] > -INFINITY ? expf((xs[i] - ms) * ig) : 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        if (!(xa[i] > -INFINITY)) continue;
                        const float wa = expf((xa[i] - ma) * ig) / za, ws = expf((xs[i] - ms) * ig) / zs;
                        const int j = i >> 1, rfi = i & 1;
                        aAin[j][rfi] += aA[rfo] * wa;
                        aSin[j][rfi] += aA[rfo] * wa * sc * dds[i] + aS[rfo] * ws * sc * sds[i];
                        aload += aA[rfo] * wa * sc * ddl[i] + aS[rfo] * ws * sc * sdl[i];
                    }
                }
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < nin)
                        c.adj[(size_t)(pin0 + j) * K + k] = make_float4(aAin[j][0], aAin[j][1], aSin[j][0], aSin[j][1]);
            }
        }
        // star segments of the item's net: dJ/dL to the cells at both ends
        for (int q = f0; q < f1; ++q) {
            const int s = c.fo_pin[q];
            const float4 as = c.adj[(size_t)s * K + k];
            const float4 Ss = c.slew[(size_t)s * K + k];
            const float2 ps = pos_of(c, s);
            const float dx = pz.x - ps.x, dy = pz.y - ps.y;
            const float L = fabsf(dx) + fabsf(dy);
            const float cp = 1e3f * c.fo_cap[q];
            const double Draw = (double)r * L * (0.5 * cc * L + cp);
            const double dDdL = (double)r * (cc * L + cp);
            const double Dbar = (double)as.x + as.y;
            const double Vbar = (double)as.z / (2.0 * Ss.z) + (double)as.w / (2.0 * Ss.w);
            const double dJdL = Dbar * 1e-6 * dDdL + Vbar * 1e-12 * 2.0 * Draw * dDdL + (double)aload * 1e-3 * cc;
            const double gx = dJdL * (double)((dx > 0.f) - (dx < 0.f)), gy = dJdL * (double)((dy > 0.f) - (dy < 0.f));
            const int cs = c.pin_cell[s];
            if (cz >= 0) {
                atomicAdd(c.grad + 2 * (size_t)cz, gx);
                atomicAdd(c.grad + 2 * (size_t)cz + 1, gy);
            }
            if (cs >= 0) {
                atomicAdd(c.grad + 2 * (size_t)cs, -gx);
                atomicAdd(c.grad + 2 * (size_t)cs + 1, -gy);
            }
        }
    }
}

template <bool UNIFORM>
__global__ void k_adj_level(const DevCtx c, int i0, int i1)
{
    const int g = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (g < i1) adj_item<UNIFORM>(c, g);
}

void launch_adjoint(const DevCtx &c, const HostSched &h, cudaStream_t st)
{
    const int nb = h.n_red_chunks;
    if (nb > 0) {
        k_obj_max_chunks<<<dim3(nb, c.K), kRedThreads, 0, st>>>(c);
        k_obj_max_final<<<c.K, kRedThreads, 0, st>>>(c, nb);
        k_obj_sum_chunks<<<dim3(nb, c.K), kRedThreads, 0, st>>>(c);
        k_obj_final<<<c.K, kRedThreads, 0, st>>>(c, nb);
    }
    k_obj_total<<<1, 32, 0, st>>>(c);
    cudaMemsetAsync(c.grad, 0, std::max<size_t>(1, 2 * (size_t)c.C) * sizeof(double), st);
    if (c.E > 0) k_adj_seed<<<nblk2(c.E, 128), 128, 0, st>>>(c);
    for (int s = h.S - 1; s >= 0; --s) {
        const int i0 = h.stage_ptr[s], i1 = h.stage_ptr[s + 1];
        if (i1 <= i0) continue;
        if (h.uniform) k_adj_level<true><<<nblk2(i1 - i0, 128), 128, 0, st>>>(c, i0, i1);
        else k_adj_level<false><<<nblk2(i1 - i0, 128), 128, 0, st>>>(c, i0, i1);
    }
}

}  // namespace sta
