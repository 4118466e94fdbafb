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
// Per-endpoint and per-segment terms are FP32; the objective sums are FP64
// and the gradient accumulates with FP64 atomics.
// Placement-driven timing optimisation consumes such gradients (the paper's
// DREAMPlace integration uses pin slacks, Sec. IV-C); the paper itself has
// no differentiable mode.
#include "item.cuh"
#include "kernels.h"

namespace sta {

static inline int nblk2(long long n, int t) { return (int)((n + t - 1) / t); }

constexpr int kDfThreadsA = 256;

// Smooth min of the two edges' setup margins of endpoint e at corner k.
// Per-endpoint terms are FP32 (margins formed from the double-float
// arrivals, then rounded once); the sums over endpoints and over the
// gradient are FP64.
__device__ __forceinline__ float ep_smooth_slack(const DevCtx &c, int e, int k, float y[2])
{
    const int p = chk(c, c.ep_pin[e], c.P);
    const DF req = c.ep_is_d[e] ? DF(c.period) - c.setup : DF(c.period);
    const DF4 &a = c.at[(size_t)p * c.K + k];
    y[0] = req - a.v[2];
    y[1] = req - a.v[3];
    const float m = fminf(y[0], y[1]);
    return m - c.gamma * logf(expf((m - y[0]) * c.inv_gamma) + expf((m - y[1]) * c.inv_gamma));
}

// softplus(z) = max(z, 0) + log1p(exp(-|z|))
// x / y by the hardware's approximate division (div.approx: within 2 ulp for
// |y| below 2^126; the divisors here are slews in ns and softmax sums >= 1).
// An IEEE division costs many times more on a path that every level waits
// on.  The quotient is an asm result, so the compiler cannot fuse it into a
// later add: every schedule rounds it alike.
__device__ __forceinline__ float div_hw(float x, float y)
{
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(y));
    return r;
}

__device__ __forceinline__ float softplus_f(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

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
    float v = -INFINITY;
    for (int e = c.red_chunk_ptr[b] + threadIdx.x; e < c.red_chunk_ptr[b + 1]; e += kRedThreads) {
        float y[2];
        v = fmaxf(v, -ep_smooth_slack(c, e, k, y) * c.inv_gamma);
    }
    const double vm = block_max<kRedThreads>((double)v, sh);
    if (threadIdx.x == 0) c.red_partial[((size_t)b * c.K + k) * 6] = vm;
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
    const float mx = (float)c.obj[k * 4 + 0], g = c.gamma;
    double se = 0, st = 0;
    for (int e = c.red_chunk_ptr[b] + threadIdx.x; e < c.red_chunk_ptr[b + 1]; e += kRedThreads) {
        float y[2];
        const float z = -ep_smooth_slack(c, e, k, y) * c.inv_gamma;
        se += (double)expf(z - mx);
        st += (double)(-g * softplus_f(z));
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
    const int p = chk(c, c.ep_pin[e], c.P);
    const float ig = c.inv_gamma;
    const float wt = (float)c.w_tns, ww = (float)c.w_wns;
    for (int k = 0; k < c.K; ++k) {
        float y[2];
        const float s = ep_smooth_slack(c, e, k, y);
        const float z = -s * ig;
        const float sig = z >= 0.f ? 1.f / (1.f + expf(-z)) : expf(z) / (1.f + expf(z));
        const float dj = wt * sig + ww * expf(z - (float)c.obj[k * 4 + 0]) / (float)c.obj[k * 4 + 1];
        const float w0 = expf((s - y[0]) * ig), w1 = expf((s - y[1]) * ig);
        c.adj[(size_t)p * c.K + k] = make_float4(-dj * w0, -dj * w1, 0.f, 0.f);
    }
}

template <class Ctx>
__device__ __forceinline__ float4 *abox_at(const Ctx &c, int par, int pin, int k)
{
    return c.abox + ((((size_t)pin * nK(c) + k) << 1) | (size_t)par);   // [pin][state][parity], as rbox
}

struct AdjItem {
    int t, pin0, kind, nin, z, f0, f1;
    // the lane's first corner, loaded ahead (written by the forward pass):
    // the output's late slews (rise, fall), its load, the clock slew
    // (flip-flop) or the late arrival and slew of each input pin
    float sz0[2], ld0, sin0[3][2];
    DF ain0[3][2];
};

template <class Ctx>
__device__ __forceinline__ AdjItem adj_prep(const Ctx &c, const int *tnin, const int *tkind, int g, int q)
{
    AdjItem a;
    const int K = nK(c), kq = corner_lane(c);
    g = chk(c, g, c.I);
    a.t = chk_type(c, c.item_type[g]);
    a.pin0 = chk(c, c.item_pin0[g], c.P);
    a.kind = a.t >= 0 ? tkind[a.t] : -1;
    a.nin = a.kind == 0 ? tnin[a.t] : 0;
    a.z = a.t < 0 ? a.pin0 : (a.kind == 1 ? a.pin0 + 1 : a.pin0 + a.nin);
    a.z = chk(c, a.z, c.P);
    a.f0 = chk(c, c.fo_ptr[g], (long long)c.F + 1);
    a.f1 = chk(c, c.fo_ptr[g + 1], (long long)c.F + 1);
    a.sz0[0] = ld_state(c.slew + (size_t)a.z * K + kq, 2);
    a.sz0[1] = ld_state(c.slew + (size_t)a.z * K + kq, 3);
    a.ld0 = a.t >= 0 ? c.load[(size_t)a.z * K + kq] : 0.f;
    const int nread = a.kind == 1 ? 1 : a.nin;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const bool on = j < nread;
        const size_t o = (size_t)(a.pin0 + j) * K + kq;
        a.ain0[j][0] = on ? ld_state_df(c.at + o, 2) : DF(0.f);
        a.ain0[j][1] = on ? ld_state_df(c.at + o, 3) : DF(0.f);
        a.sin0[j][0] = on ? ld_state(c.slew + o, 2) : 0.f;
        a.sin0[j][1] = on ? ld_state(c.slew + o, 3) : 0.f;
    }
    return a;
}

// Lane q of a quad works on output edge rf = q >> 1, arrivals (q & 1 == 0)
// or slews (q & 1 == 1); its adjoint of the output is the sum over the net's
// sinks of dJ/dAT (arrival lanes) or of dJ/dslew * slew_z / slew_sink (slew
// lanes, through slew_sink = sqrt(slew_z^2 + var)).  Every schedule sums in
// one order: the entries of each residue class mod 4 in increasing order,
// then (class 0 + class 1) + (class 2 + class 3).
// A gate input's mailbox record (`scaled`) carries dJ/dslew / slew_sink
// already, divided by the item that published it: the gather then needs
// neither the sink's slew nor a division.  From the adjoint array (endpoints,
// the level sweep) the same quotient is formed here from the same operands.
template <class Ctx>
__device__ __forceinline__ float4 adj_sink_terms(const Ctx &c, int s, int k, float4 as, float szr, float szf,
                                                 bool scaled)
{
    if (!scaled) {
        as.z = div_hw(as.z, ld_state(c.slew + (size_t)s * nK(c) + k, 2));
        as.w = div_hw(as.w, ld_state(c.slew + (size_t)s * nK(c) + k, 3));
    }
    return make_float4(as.x, as.y, __fmul_rn(as.z, szr), __fmul_rn(as.w, szf));
}

// Are the adjoints of every gate-input sink of the item's net complete (all
// the lane's corners)?  The quad splits the sinks: lane q reads the whole
// adjoint record of fan-out entries q, q + 4, ... (first corner) and sums
// each component over them (`part`, its residue class); adj_quad_sum then
// combines the classes.  Endpoint sinks were seeded by an earlier launch.
template <class Ctx>
__device__ __forceinline__ bool adj_probe(const Ctx &c, const AdjItem &a, int par, int q, float4 &part)
{
    const int K = nK(c), kq = corner_lane(c);
    const int nfo = a.f1 - a.f0;
    bool ok = true;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e0 = q; e0 < nfo && ok; e0 += 16) {
        int s[4];
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + 4 * u;
            s[u] = e < nfo ? chk(c, __ldg(c.fo_pin + a.f0 + e), c.P) : -1;
            if (s[u] < 0) continue;
            v[u] = s[u] < c.ep_begin ? ld_relaxed4(abox_at(c, par, s[u], kq)) : c.adj[(size_t)s[u] * K + kq];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (s[u] >= 0) ok = ok && complete(v[u]);
        if (!ok) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (s[u] < 0) continue;
            const float4 tm = adj_sink_terms(c, s[u], kq, v[u], a.sz0[0], a.sz0[1], s[u] < c.ep_begin);
            acc.x += tm.x;
            acc.y += tm.y;
            acc.z += tm.z;
            acc.w += tm.w;
        }
    }
    for (int e = q; e < nfo && ok; e += 4) {
        const int s = chk(c, __ldg(c.fo_pin + a.f0 + e), c.P);
        if (s < c.ep_begin)
            for (int k = kq + nKL(c); k < K && ok; k += nKL(c)) ok = complete(ld_relaxed4(abox_at(c, par, s, k)));
    }
    part = acc;
    return ok;
}

// The quad's residue-class sums combined, lane q's component.  Every lane
// of mask m calls it: the quad's own lanes, or the whole warp when the
// caller keeps it converged (cheaper shuffles; each quad still sums only
// its own lanes).
__device__ __forceinline__ float adj_quad_sum(float4 part, int q, unsigned m = quad_mask())
{
    const int base = threadIdx.x & 28;
    float r = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float pj = j == 0 ? part.x : j == 1 ? part.y : j == 2 ? part.z : part.w;
        const float c0 = __shfl_sync(m, pj, base), c1 = __shfl_sync(m, pj, base + 1);
        const float c2 = __shfl_sync(m, pj, base + 2), c3 = __shfl_sync(m, pj, base + 3);
        const float tot = (c0 + c1) + (c2 + c3);
        if (j == (q >> 1) + 2 * (q & 1)) r = tot;
    }
    return r;
}

__device__ __forceinline__ float quad_sum(float v)
{
    const unsigned m = quad_mask();
    v += __shfl_xor_sync(m, v, 1);
    v += __shfl_xor_sync(m, v, 2);
    return v;
}

// One item of the reverse sweep.  Lane q of a quad differentiates the merge
// of output edge rf = q >> 1, of the arrivals (q & 1 == 0, delay tables) or
// of the slews (q & 1 == 1, slew tables), for the quad's corners; the quad
// sums the partials.  The segment gradients are summed over corners (and the
// driver's over all its segments) before the FP64 atomics.
// The lane's partials of one item for its first corner, before the quad
// sums: the load adjoint and the adjoints of each input candidate's arrival
// (aAin) and slew (aSin).
struct AdjPart {
    float aload, aAin[6], aSin[6];
};

// SPLIT (one corner per lane group, K == KL, with WAIT): adj_run stops
// before the quad sums and returns the lane's partials in *part; the caller
// sums them over the quad with the whole warp converged (adj_part_sum) and
// stores them (adj_store).  The sums and the stores are the ones adj_run
// makes itself otherwise.
template <bool UNIFORM, bool WAIT, bool SPLIT = false, class Lut, class Ctx = DevCtx>
__device__ __forceinline__ void adj_run(const Ctx &c, const Lut &lut, const int *tsense, const AdjItem &a, int g,
                                        int q, int par, float abar0, AdjPart *part = nullptr)
{
    const int t = a.t, pin0 = a.pin0, z = a.z, K = nK(c), nin = a.nin;
    const int kq = corner_lane(c), KL = nKL(c);
    const float ig = c.inv_gamma;
    const int rfo = q >> 1;
    const bool slew_lane = (q & 1) != 0;
    for (int k = kq; k < K; k += KL) {
        const bool first = k == kq;
        // the lane's adjoint of the output, gathered from the sinks through
        // the net arcs (folded by adj_probe for the first corner when WAIT)
        float abar;
        if (WAIT && first) {
            abar = abar0;
        } else {
            const float szr = first ? a.sz0[0] : ld_state(c.slew + (size_t)z * K + k, 2);
            const float szf = first ? a.sz0[1] : ld_state(c.slew + (size_t)z * K + k, 3);
            const int j = rfo + 2 * (slew_lane ? 1 : 0);   // component: dJ/dAT rise, fall, dJ/dslew rise, fall
            float cls[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                cls[r] = 0.f;
                for (int p = a.f0 + r; p < a.f1; p += 4) {
                    const int s = chk(c, c.fo_pin[p], c.P);
                    const float4 as = (WAIT && s < c.ep_begin) ? ld_relaxed4(abox_at(c, par, s, k)) : c.adj[(size_t)s * K + k];
                    const float4 tm = adj_sink_terms(c, s, k, as, szr, szf, WAIT && s < c.ep_begin);
                    cls[r] += j == 0 ? tm.x : j == 1 ? tm.y : j == 2 ? tm.z : tm.w;
                }
            }
            abar = (cls[0] + cls[1]) + (cls[2] + cls[3]);
        }
        // through the output merges and the NLDM lookups
        float aload = 0.f;
        float aAin[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, aSin[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (t >= 0) {
            const float sc = __ldg(c.lut_scale + k);
            const float ld = first ? a.ld0 : c.load[(size_t)z * K + k];
            if (a.kind == 1) {
                const float cs = first ? a.sin0[0][0] : ld_state(c.slew + (size_t)pin0 * K + k, 2);
                const int tq = tab_off(t, 1, slew_lane ? 2 + rfo : rfo);
                float ds, dl;
                interp_d(lut, tq, seg_slew<UNIFORM>(c, lut, tq, cs), seg_load<UNIFORM>(c, lut, tq, ld), ds, dl);
                aload = abar * sc * dl;
            } else {
                float x[6];   // candidates (FP32, as the forward merge forms them)
                float dds[6], ddl[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    x[i] = -INFINITY;
                    dds[i] = ddl[i] = 0.f;
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (j >= nin) continue;
                    const int se = tsense[t * 3 + j];
                    const int tq = tab_off(t, j, slew_lane ? 2 + rfo : rfo);
                    DF Ain[2];
                    float Sin[2];
                    if (first) {
                        Ain[0] = a.ain0[j][0];
                        Ain[1] = a.ain0[j][1];
                        Sin[0] = a.sin0[j][0];
                        Sin[1] = a.sin0[j][1];
                    } else {
                        const size_t o = (size_t)(pin0 + j) * K + k;
                        Ain[0] = ld_state_df(c.at + o, 2);
                        Ain[1] = ld_state_df(c.at + o, 3);
                        Sin[0] = ld_state(c.slew + o, 2);
                        Sin[1] = ld_state(c.slew + o, 3);
                    }
                    // the input edges with an arc to rfo (one for a unate arc,
                    // both for a non-unate one): no divergence between the
                    // quad's lanes of different rfo
                    const int n_rfi = se == kSenseNonC ? 2 : (se == kSensePosC || se == kSenseNegC) ? 1 : 0;
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        if (r >= n_rfi) break;
                        const int rfi = se == kSenseNonC ? r : (se == kSenseNegC ? 1 - rfo : rfo);
                        const float s = rfi ? Sin[1] : Sin[0];
                        float ds, dl;
                        const float v = interp_d(lut, tq, seg_slew<UNIFORM>(c, lut, tq, s),
                                                 seg_load<UNIFORM>(c, lut, tq, ld), ds, dl);
                        const float xv = slew_lane ? sc * v : (rfi ? Ain[1] : Ain[0]).hi + sc * v;
                        if (rfi) {
                            x[j * 2 + 1] = xv;
                            dds[j * 2 + 1] = ds;
                            ddl[j * 2 + 1] = dl;
                        } else {
                            x[j * 2] = xv;
                            dds[j * 2] = ds;
                            ddl[j * 2] = dl;
                        }
                    }
                }
                // softmax weights of the log-sum-exp merge
                float m = -INFINITY;
#pragma unroll
                for (int i = 0; i < 6; ++i) m = fmaxf(m, x[i]);
                float zsum = 0.f, ex[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    ex[i] = x[i] > -INFINITY ? expf((float)(x[i] - m) * ig) : 0.f;
                    zsum += ex[i];
                }
                const float az = div_hw(abar, zsum);   // zsum >= 1 (the max's own term)
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    if (!(x[i] > -INFINITY)) continue;
                    const float w = az * ex[i];
                    if (!slew_lane) aAin[i] = w;
                    aSin[i] = w * sc * dds[i];
                    aload += w * sc * ddl[i];
                }
            }
        }
        if (SPLIT) {
            part->aload = aload;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                part->aAin[i] = aAin[i];
                part->aSin[i] = aSin[i];
            }
            return;
        }
        aload = quad_sum(aload);
        if (q == 0) c.aload[(size_t)g * K + k] = aload;
        if (a.kind == 0) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                aAin[i] = quad_sum(aAin[i]);
                aSin[i] = quad_sum(aSin[i]);
            }
            for (int j = 0; j < nin; ++j) {
                const float v = q == 0 ? aAin[j * 2] : q == 1 ? aAin[j * 2 + 1] : q == 2 ? aSin[j * 2] : aSin[j * 2 + 1];
                reinterpret_cast<float *>(c.adj + (size_t)(pin0 + j) * K + k)[q] = v;
                if (WAIT) {
                    // the slew lanes publish dJ/dslew / slew of the pin (adj_sink_terms)
                    const float pv = q >= 2 ? div_hw(v, ld_state(c.slew + (size_t)(pin0 + j) * K + k, q)) : v;
                    float *n = reinterpret_cast<float *>(abox_at(c, par, pin0 + j, k));
                    float *o = reinterpret_cast<float *>(abox_at(c, par ^ 1, pin0 + j, k));
                    st_relaxed(n + q, pv);
                    o[q] = __int_as_float(0x7fffffff);
                }
            }
        }
    }
}

// The quad sums of the partials (every lane of mask m calls it: the whole
// warp, converged), in quad_sum's order.
__device__ __forceinline__ void adj_part_sum(AdjPart &p, unsigned m)
{
    p.aload += __shfl_xor_sync(m, p.aload, 1);
    p.aload += __shfl_xor_sync(m, p.aload, 2);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        p.aAin[i] += __shfl_xor_sync(m, p.aAin[i], 1);
        p.aAin[i] += __shfl_xor_sync(m, p.aAin[i], 2);
        p.aSin[i] += __shfl_xor_sync(m, p.aSin[i], 1);
        p.aSin[i] += __shfl_xor_sync(m, p.aSin[i], 2);
    }
}

// adj_run's stores of the summed partials (first corner; the dataflow sweep)
template <class Ctx>
__device__ __forceinline__ void adj_store(const Ctx &c, const AdjItem &a, int g, int q, int par, const AdjPart &p)
{
    const int K = nK(c), k = corner_lane(c);
    if (q == 0) c.aload[(size_t)g * K + k] = p.aload;
    if (a.kind != 0) return;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j >= a.nin) continue;
        const float v = q == 0 ? p.aAin[j * 2] : q == 1 ? p.aAin[j * 2 + 1] : q == 2 ? p.aSin[j * 2] : p.aSin[j * 2 + 1];
        reinterpret_cast<float *>(c.adj + (size_t)(a.pin0 + j) * K + k)[q] = v;
        // the slew lanes publish dJ/dslew / slew of the pin (adj_sink_terms)
        const float pv = q >= 2 ? div_hw(v, q == 2 ? a.sin0[j][0] : a.sin0[j][1]) : v;
        float *n = reinterpret_cast<float *>(abox_at(c, par, a.pin0 + j, k));
        float *o = reinterpret_cast<float *>(abox_at(c, par ^ 1, a.pin0 + j, k));
        st_relaxed(n + q, pv);
        o[q] = __int_as_float(0x7fffffff);
    }
}

// Star segments, after the sweep: dJ/dL of every driver-sink segment from
// the sink's adjoints (arrival and slew, through the segment's Elmore delay
// D = r L (c L / 2 + Cpin) and variance D^2) and the driver's load adjoint
// (load = sum of c L + Cpin), summed over corners, then to the two cells'
// positions through L = |dx| + |dy| (sign 0 at dx = 0).  One thread per
// fan-out entry (segment); each segment adds its share to both cells.
__global__ void k_adj_star(const DevCtx c)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.F) return;
    const int K = c.K;
    // every input of this kernel is read-only here (read-only loads)
    auto pos = [&](int cell_or_port) -> float2 {
        if (cell_or_port >= 0) {
            const int cc = chk(c, cell_or_port, c.C);
            return make_float2(__ldg(c.cell_xy + 2 * (size_t)cc), __ldg(c.cell_xy + 2 * (size_t)cc + 1));
        }
        const int q = -cell_or_port - 1;
        return make_float2(__ldg(c.port_xy + 2 * (size_t)q), __ldg(c.port_xy + 2 * (size_t)q + 1));
    };
    const int g = chk(c, __ldg(c.fo_item + p), c.I);
    const int s = chk(c, __ldg(c.fo_pin + p), c.P);
    const int z = chk(c, __ldg(c.drv_of + s), c.P);   // the net's driver: the item's output pin
    const int cz = __ldg(c.pin_cell + z), csp = __ldg(c.pin_cell + s);
    const float2 pz = pos(cz), ps = pos(csp);
    const float dx = pz.x - ps.x, dy = pz.y - ps.y;
    const float L = fabsf(dx) + fabsf(dy);
    const float cp = 1e3f * __ldg(c.fo_cap + p);
    float dJdL = 0.f;
    for (int k = 0; k < K; ++k) {
        const float fk = __ldg(c.rc_scale + k);
        const float r = fk * c.r_per_um, cc = fk * c.c_per_um;
        const float4 as = __ldg(c.adj + (size_t)s * K + k);
        const float2 Ss = __ldg(reinterpret_cast<const float2 *>(c.slew + (size_t)s * K + k) + 1);   // late
        const float Draw = r * L * (0.5f * cc * L + cp);
        const float dDdL = r * (cc * L + cp);
        const float Dbar = as.x + as.y;
        const float Vbar = as.z / (2.f * Ss.x) + as.w / (2.f * Ss.y);
        dJdL += Dbar * 1e-6f * dDdL + Vbar * 1e-12f * 2.f * Draw * dDdL + __ldg(c.aload + (size_t)g * K + k) * 1e-3f * cc;
    }
    // the sign products are exact in FP32 (a sign is -1, 0 or 1)
    const double gx = (double)(dJdL * (float)((dx > 0.f) - (dx < 0.f)));
    const double gy = (double)(dJdL * (float)((dy > 0.f) - (dy < 0.f)));
    if (csp >= 0) {
        const int cs = chk(c, csp, c.C);
        atomicAdd(c.grad + 2 * (size_t)cs, -gx);
        atomicAdd(c.grad + 2 * (size_t)cs + 1, -gy);
    }
    if (cz >= 0) {
        const int cd = chk(c, cz, c.C);
        atomicAdd(c.grad + 2 * (size_t)cd, gx);
        atomicAdd(c.grad + 2 * (size_t)cd + 1, gy);
    }
}

// Steiner trees, after the sweep: the tree of the update held fixed.  Per
// corner, the reverse mode of the tree's Elmore recurrences (those of
// k_net_tree, taken back in the opposite order)
//   var_i = 2 beta_i - D_i^2       betabar = 2 varbar, summed up the subtree
//   beta_i = beta_p + R_i M_i      Rbar_i += betabar_i M_i; Mbar = betabar R,
//                                  summed down from the root
//   M_i = C_i D_i + sum children   Cbar_i += Mbar_i D_i, Dbar_i += Mbar_i C_i
//   D_i = D_p + R_i Cdown_i        Dbar summed up the subtree; Rbar_i +=
//                                  Dbar_i Cdown_i; Cdownbar_i = Dbar_i R_i,
//                                  summed down from the root (root: loadbar)
//   Cdown_i = C_i + sum children   Cbar_i += Cdownbar_i
// from the sinks' adjoints (Dbar = 1e-6 (dJ/dAT rise + fall), varbar =
// 1e-12 sum over edges of dJ/dslew / (2 slew)) and the driver's load
// adjoint (1e-3 dJ/dload); then dJ/dLx_i = f (rx Rbar_i + cx (Cbar_i +
// Cbar_p) / 2), likewise for y, summed over corners.  Every node coordinate
// is a pin's (Steiner points take medians); the tree writer recorded the
// lowest net pin at it and the sign of node - parent, so Lx_i moves by +-1
// per um of the two carrying pins' cells (nm rounding taken as the
// identity, sign 0 at equal coordinates).  One thread per net.  The tree
// (parents, R), the pin caps and every per-node sum sit in a shared-memory
// column of COLN nodes, where the gradient is also summed per net pin (up to
// COLP pins) before one FP64 atomic per pin and axis: nets of at most 5 pins
// take 8-node columns and nets of 6-9 pins 16-node columns, 64 threads a
// block; larger ones 128-node columns, 8 threads a block, largest first.  Trees beyond a column work in global
// scratch with an atomic per contribution.
enum { kA_PAR, kA_R, kA_PC, kA_CN, kA_CD, kA_D, kA_M, kA_DB, kA_RB, kA_BB, kAdjArrays };

// Node arrays of one net: a shared-memory column (element i of array a at
// s_col[(a COLN + i) NT + thread]) or a row of the global scratch.
template <int COLN, int NT>
struct ColNodes {
    float *p;   // s_col + thread
    __device__ __forceinline__ float &operator()(int arr, int i) const { return p[(arr * COLN + i) * NT]; }
};
struct RowNodes {
    float *p;       // scratch + first node
    long long a;    // array stride
    __device__ __forceinline__ float &operator()(int arr, int i) const { return p[arr * a + i]; }
};

// The sweeps of one net (n tree nodes from n0, m sinks from f0); scatter(j,
// axis, g) takes dJ/d(coordinate of net pin j).  Every input is read-only
// here and goes through the read-only path.  Per corner: Cdown (up), D and
// M = C D (down), the sinks' seeds, then in one upward sweep the subtree
// sums of M and betabar with Rbar += betabar M, in one downward sweep Mbar
// with Cbar and Dbar's M term, in one upward sweep Dbar with Rbar += Dbar
// Cdown, and in one downward sweep Cdownbar, Cbar and the scatter.
template <class V, class S>
__device__ __forceinline__ void steiner_adjoint_net(const DevCtx &c, const V &v, const S &scatter, int g, int f0,
                                                    int m, int n0, int n)
{
    auto par = [&](int i) { return __float_as_int(v(kA_PAR, i)); };
#pragma unroll 4
    for (int i = 0; i < n; ++i) {
        v(kA_PAR, i) = __int_as_float(i ? chk(c, __ldg(c.st_parent + n0 + i), i) : -1);
        v(kA_R, i) = __ldg(c.st_R + n0 + i);
        v(kA_PC, i) = 0.f;
    }
#pragma unroll 4
    for (int p = f0; p < f0 + m; ++p) v(kA_PC, chk(c, __ldg(c.st_fo_node + p), n)) += 1e3f * __ldg(c.fo_cap + p);
    const float rx = c.r_per_um, ry = c.r_per_um_y, cx = c.c_per_um, cy = c.c_per_um_y;
    const int K = c.K;
    for (int k = 0; k < K; ++k) {
        const float f = __ldg(c.rc_scale + k);
#pragma unroll 4
        for (int i = 0; i < n; ++i) {
            const float cn = f * __ldg(c.st_C + n0 + i) + v(kA_PC, i);
            v(kA_CN, i) = cn;
            v(kA_CD, i) = cn;
            v(kA_DB, i) = 0.f;
            v(kA_BB, i) = 0.f;
        }
        for (int i = n - 1; i >= 1; --i) v(kA_CD, par(i)) += v(kA_CD, i);
        v(kA_D, 0) = 0.f;
        v(kA_M, 0) = 0.f;
        for (int i = 1; i < n; ++i) {
            const float Di = v(kA_D, par(i)) + f * v(kA_R, i) * v(kA_CD, i);
            v(kA_D, i) = Di;
            v(kA_M, i) = v(kA_CN, i) * Di;
        }
#pragma unroll 4
        for (int p = f0; p < f0 + m; ++p) {   // Dbar with its -2 D varbar term; BB = 2 varbar
            const int s = chk(c, __ldg(c.fo_pin + p), c.P), q = chk(c, __ldg(c.st_fo_node + p), n);
            const float4 as = __ldg(c.adj + (size_t)s * K + k), Ss = __ldg(c.slew + (size_t)s * K + k);
            const float bb = 2e-12f * (as.z / (2.f * Ss.z) + as.w / (2.f * Ss.w));
            v(kA_DB, q) += 1e-6f * (as.x + as.y) - v(kA_D, q) * bb;
            v(kA_BB, q) += bb;
        }
        for (int i = n - 1; i >= 1; --i) {   // M and betabar summed up the subtree
            const int pi = par(i);
            const float Mi = v(kA_M, i), bi = v(kA_BB, i);
            v(kA_M, pi) += Mi;
            v(kA_RB, i) = bi * Mi;
            v(kA_BB, pi) += bi;
        }
        v(kA_M, 0) = 0.f;    // M becomes Mbar, BB becomes Cbar
        v(kA_BB, 0) = 0.f;
        for (int i = 1; i < n; ++i) {
            const float mb = v(kA_BB, i) * f * v(kA_R, i) + v(kA_M, par(i));
            v(kA_M, i) = mb;
            v(kA_BB, i) = mb * v(kA_D, i);
            v(kA_DB, i) += mb * v(kA_CN, i);
        }
        for (int i = n - 1; i >= 1; --i) {
            const float db = v(kA_DB, i);
            v(kA_RB, i) += db * v(kA_CD, i);
            v(kA_DB, par(i)) += db;
        }
        v(kA_CD, 0) = 1e-3f * __ldg(c.aload + (size_t)g * K + k);   // CD becomes Cdownbar
        v(kA_BB, 0) += v(kA_CD, 0);
        for (int i = 1; i < n; ++i) {
            const int pi = par(i);
            const float cdb = v(kA_DB, i) * f * v(kA_R, i) + v(kA_CD, pi);
            v(kA_CD, i) = cdb;
            const float cbi = v(kA_BB, i) + cdb;
            v(kA_BB, i) = cbi;
            const float rb = v(kA_RB, i), cb = cbi + v(kA_BB, pi);
            const float gl[2] = {f * (rx * rb + 0.5f * cx * cb), f * (ry * rb + 0.5f * cy * cb)};
            const int2 ci = __ldg(c.st_src + n0 + i), cp = __ldg(c.st_src + n0 + pi);
            const int own[2] = {ci.x, ci.y}, up[2] = {cp.x, cp.y};
            for (int ax = 0; ax < 2; ++ax) {
                const int sg = (own[ax] & 3) - 1;
                if (sg == 0) continue;
                scatter(own[ax] >> 2, ax, sg * gl[ax]);
                scatter(up[ax] >> 2, ax, -sg * gl[ax]);
            }
        }
    }
}

// Items i0 .. i1 - 1 of the Steiner list (by increasing pin count), the
// last first.
template <int COLN, int COLP, int NT>
__global__ void __launch_bounds__(NT) k_adj_steiner(const DevCtx c, int i0, int i1)
{
    __shared__ float s_col[kAdjArrays * COLN * NT];
    __shared__ float s_pin[2 * COLP * NT];
    const int t = threadIdx.x, it = blockIdx.x * NT + t;
    if (it >= i1 - i0) return;
    const int g = chk(c, __ldg(c.st_items + i1 - 1 - it), c.I);
    const int f0 = __ldg(c.fo_ptr + g), m = __ldg(c.fo_ptr + g + 1) - f0;
    const int n0 = __ldg(c.rc_ptr + g), n = chk(c, __ldg(c.st_nlive + g), __ldg(c.rc_ptr + g + 1) - n0 + 1);
    if (m <= 0 || n <= 1) return;
    const int z = chk(c, item_out_pin(c, chk_type(c, __ldg(c.item_type + g)), __ldg(c.item_pin0 + g)), c.P);
    auto cell_of = [&](int j) -> int {
        const int p = j ? chk(c, __ldg(c.fo_pin + f0 + chk(c, j - 1, m)), c.P) : z;
        const int cc = __ldg(c.pin_cell + p);
        return cc >= 0 ? chk(c, cc, c.C) : -1;
    };
    if (n <= COLN && m + 1 <= COLP) {
        for (int j = 0; j < 2 * (m + 1); ++j) s_pin[j * NT + t] = 0.f;
        steiner_adjoint_net(
            c, ColNodes<COLN, NT>{s_col + t},
            [&](int j, int ax, float gv) { s_pin[(2 * chk(c, j, m + 1) + ax) * NT + t] += gv; }, g, f0, m, n0, n);
        for (int j = 0; j <= m; ++j) {
            const int cc = cell_of(j);
            if (cc < 0) continue;
            for (int ax = 0; ax < 2; ++ax) {
                const float gv = s_pin[(2 * j + ax) * NT + t];
                if (gv != 0.f) atomicAdd(c.grad + 2 * (size_t)cc + ax, (double)gv);
            }
        }
    } else {
        steiner_adjoint_net(
            c, RowNodes{c.st_abuf + n0, c.NN},
            [&](int j, int ax, float gv) {
                const int cc = cell_of(j);
                if (cc >= 0) atomicAdd(c.grad + 2 * (size_t)cc + ax, (double)gv);
            },
            g, f0, m, n0, n);
    }
}

template <bool UNIFORM>
__global__ void k_adj_level(const DevCtx c, int i0, int i1)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = i0 + tid / (4 * c.KL);
    if (g < i1)
        adj_run<UNIFORM, false>(c, LutGlobal{c.lut, c.lut_scale}, c.arc_sense, adj_prep(c, c.type_nin, c.type_kind, g, tid & 3), g,
                                tid & 3, 0, 0.f);
}

// ----------------------------------------------------- dataflow adjoint

// After an aborted adjoint pass: reset its mailbox to NaN.
__global__ void k_adj_recover(const DevCtx c)
{
    if (ld_volatile(c.df_state + 6) == 0u) return;
    const float4 nan4 = make_float4(__int_as_float(0x7fffffff), __int_as_float(0x7fffffff),
                                    __int_as_float(0x7fffffff), __int_as_float(0x7fffffff));
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.abox_len; i += stride) c.abox[i] = nan4;
}

__global__ void k_adj_begin(const DevCtx c)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c.df_state[4] = c.df_state[4] + 1u;
        c.df_state[5] = 0u;
        c.df_state[6] = 0u;
    }
}

template <bool UNIFORM, class Ctx = DevCtx>
__global__ void __launch_bounds__(kDfThreadsA) k_df_adjoint(const Ctx c)
{
    extern __shared__ float smem[];
    const int nl = c.T * 3 * 4 * kLutStride;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) smem[i] = __ldg(c.lut + i);
    int *ti = reinterpret_cast<int *>(smem + nl);
    for (int i = threadIdx.x; i < c.T; i += blockDim.x) {
        ti[i] = __ldg(c.type_nin + i);
        ti[c.T + i] = __ldg(c.type_kind + i);
    }
    for (int i = threadIdx.x; i < 3 * c.T; i += blockDim.x) ti[2 * c.T + i] = __ldg(c.arc_sense + i);
    __syncthreads();
    const LutShared lut{smem, c.lut_scale, c.lut_scale};   // table scales read from global memory here
    const int par = (int)(ld_volatile(c.df_state + 4) & 1u);
    const int lane = threadIdx.x & 31, q = lane & 3;
    for (;;) {
        int ch = 0;
        if (lane == 0) ch = (int)atomicAdd(c.df_state + 5, 1u);
        ch = __shfl_sync(0xffffffffu, ch, 0);
        if (ch >= c.n_bwd_chunks || ld_volatile(c.df_state + 6)) break;
        const int pos = c.bwd_chunk_lo[ch] + lane / (4 * nKL(c));
        bool pending = pos < c.bwd_chunk_hi[ch];
        const int x = pending ? chk(c, c.bwd_order[chk(c, pos, c.I)], c.I) : 0;
        AdjItem it{};
        if (pending) it = adj_prep(c, ti, ti + c.T, x, q);
        long long spins = 0;
        // the lane's share of the sinks summed (`part`), kept once every one
        // of them was complete: a published adjoint is final for the sweep
        float4 part = make_float4(0.f, 0.f, 0.f, 0.f);
        bool lane_done = false;
        while (__any_sync(0xffffffffu, pending)) {
            bool ok = false;
            if (pending) {
                ok = lane_done || adj_probe(c, it, par, q, part);
                lane_done = ok;
            }
            const bool go = group_all_warp(c, ok) && pending;   // the whole warp votes
            if (__any_sync(0xffffffffu, go)) {
                // every lane sums (full-warp shuffles); the ready groups use it
                const float sum = adj_quad_sum(part, q, 0xffffffffu);
                if (nK(c) == nKL(c)) {
                    // one corner per group: the quad sums of the item's
                    // partials also run converged
                    AdjPart ap{};
                    if (go) adj_run<UNIFORM, true, true>(c, lut, ti + 2 * c.T, it, x, q, par, sum, &ap);
                    adj_part_sum(ap, 0xffffffffu);
                    if (go) {
                        adj_store(c, it, x, q, par, ap);
                        pending = false;
                    }
                } else if (go) {
                    adj_run<UNIFORM, true>(c, lut, ti + 2 * c.T, it, x, q, par, sum);
                    pending = false;
                }
            }
            if (__any_sync(0xffffffffu, pending)) {
                if (++spins >= c.spin_limit) {
                    if (lane == 0) {
                        atomicOr(c.err, kErrTimeout);
                        atomicExch(c.df_state + 6, 1u);
                    }
                    break;
                }
                if ((spins & 31) == 0 && __any_sync(0xffffffffu, ld_volatile(c.df_state + 6) != 0u)) break;
                __nanosleep(32);
            }
        }
    }
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
    if (h.adj_blocks > 0) {
        k_adj_recover<<<h.adj_blocks, kDfThreadsA, 0, st>>>(c);
        k_adj_begin<<<1, 32, 0, st>>>(c);
        const size_t smem = adjoint_smem_bytes(h.T);
        if (h.one) {
            const DevCtxOne c1{c};   // the same context, for the one-state builds
            if (h.uniform) k_df_adjoint<true, DevCtxOne><<<h.adj_blocks, kDfThreadsA, smem, st>>>(c1);
            else k_df_adjoint<false, DevCtxOne><<<h.adj_blocks, kDfThreadsA, smem, st>>>(c1);
        } else if (h.uniform) {
            k_df_adjoint<true><<<h.adj_blocks, kDfThreadsA, smem, st>>>(c);
        } else {
            k_df_adjoint<false><<<h.adj_blocks, kDfThreadsA, smem, st>>>(c);
        }
    } else {
        for (int s = h.S - 1; s >= 0; --s) {
            const int i0 = h.stage_ptr[s], i1 = h.stage_ptr[s + 1];
            if (i1 <= i0) continue;
            if (h.uniform) k_adj_level<true><<<nblk2(4LL * c.KL * (i1 - i0), 128), 128, 0, st>>>(c, i0, i1);
            else k_adj_level<false><<<nblk2(4LL * c.KL * (i1 - i0), 128), 128, 0, st>>>(c, i0, i1);
        }
    }
    if (c.steiner) {
        const int nt = c.st_adj_tiny, ns = c.st_adj_small, nl = c.st_n_items - ns;
        if (nt > 0) k_adj_steiner<kAdjTinyColNodes, kAdjTinyPins, 64><<<nblk2(nt, 64), 64, 0, st>>>(c, 0, nt);
        if (ns > nt)
            k_adj_steiner<kAdjColNodes, kAdjSmallPins, 64><<<nblk2(ns - nt, 64), 64, 0, st>>>(c, nt, ns);
        if (nl > 0)
            k_adj_steiner<kAdjBigColNodes, 64, 8><<<nblk2(nl, 8), 8, 0, st>>>(c, ns, c.st_n_items);
    } else if (c.I > 0) {
        if (c.F > 0) k_adj_star<<<nblk2(c.F, 256), 256, 0, st>>>(c);
    }
}

size_t steiner_adjoint_floats(int64_t NN) { return (size_t)kAdjArrays * (size_t)std::max<int64_t>(1, NN); }

size_t adjoint_smem_bytes(int T) { return (size_t)T * 3 * 4 * kLutStride * sizeof(float) + (size_t)T * 5 * sizeof(int); }

cudaError_t adjoint_prepare(HostSched &h)
{
    const size_t smem = adjoint_smem_bytes(h.T);
    if (h.adj_level || smem > 200 * 1024) {   // chosen, or the library is too large for the shared copy
        h.adj_blocks = 0;
        return cudaSuccess;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto occ = [&](auto k) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kDfThreadsA, smem);
    };
    if (h.one) occ(h.uniform ? k_df_adjoint<true, DevCtxOne> : k_df_adjoint<false, DevCtxOne>);
    else occ(h.uniform ? k_df_adjoint<true> : k_df_adjoint<false>);
    if (e != cudaSuccess) return e;
    h.adj_blocks = std::max(1, per_sm) * sms;
    return cudaSuccess;
}

}  // namespace sta
