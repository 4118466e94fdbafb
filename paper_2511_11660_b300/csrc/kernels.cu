// kernels.cu -- level-schedule kernels of the STA pass.
//
// One update = net delay calculation (Elmore + second moment on RC trees,
// or star trees from positions), forward arrival/slew propagation level by
// level, endpoint required times and slacks, backward required-time
// propagation level by level (with pin slacks), and an FP64 WNS/TNS
// reduction.  HeteroSTA names these steps (delay calculation and graph
// propagation, Sec. I; Elmore delay, Sec. III "Delay models"; WNS/TNS and
// pin slacks, Sec. III "Report options") without formulas; the formulas are
// the textbook ones stated in include/sta.h.
#include "kernels.h"

namespace sta {

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ nets

// RC trees.  One block per tile of consecutive items whose nodes fit in
// shared memory (one thread per net); a tile holding a single larger net
// sweeps it in global scratch instead.  Per corner: Cdown (reverse sweep),
// Elmore D (forward), M = C*D summed over the subtree (reverse), beta
// (forward), var = 2*beta - D^2.  Units: Ohm*fF -> 1e-6 ns.
__global__ void __launch_bounds__(kRcTileNets) k_net_tree(const DevCtx c)
{
    __shared__ int32_t s_par[kRcTileNodes];
    __shared__ float s_R[kRcTileNodes], s_C[kRcTileNodes], s_A[kRcTileNodes], s_B[kRcTileNodes];
    const int g0 = c.tile_item[blockIdx.x], g1 = c.tile_item[blockIdx.x + 1];
    const int n0 = c.rc_ptr[g0], nn = c.rc_ptr[g1] - n0;
    const bool big = nn > kRcTileNodes;
    if (!big) {
        for (int i = threadIdx.x; i < nn; i += blockDim.x) {
            s_par[i] = c.rc_parent[n0 + i];
            s_R[i] = c.rc_R[n0 + i];
            s_C[i] = c.rc_C[n0 + i];
        }
    }
    __syncthreads();
    const int g = g0 + threadIdx.x;
    if (g >= g1) return;
    const int b = c.rc_ptr[g] - n0, e = c.rc_ptr[g + 1] - n0;
    if (e == b) return;
    const int32_t *par = big ? c.rc_parent + n0 : s_par;
    const float *R = big ? c.rc_R + n0 : s_R;
    const float *Cw = big ? c.rc_C + n0 : s_C;
    float *A = big ? c.scratch_a + n0 : s_A;
    float *B = big ? c.scratch_b + n0 : s_B;
    const int t = c.item_type[g];
    const int z = item_out_pin(c, t, c.item_pin0[g]);
    const int f0 = c.fo_ptr[g], f1 = c.fo_ptr[g + 1];
    const int K = c.K;
    for (int k = 0; k < K; ++k) {
        const float f = __ldg(c.rc_scale + k);
        for (int i = b; i < e; ++i) A[i] = f * Cw[i];
        for (int q = f0; q < f1; ++q) A[b + c.fo_node[q]] += 1e3f * c.fo_cap[q];
        for (int i = b; i < e; ++i) B[i] = A[i];                       // node capacitance
        for (int i = e - 1; i > b; --i) A[b + par[i]] += A[i];          // Cdown
        c.load[(size_t)z * K + k] = 1e-3f * A[b];
        A[b] = 0.f;
        for (int i = b + 1; i < e; ++i) A[i] = A[b + par[i]] + f * R[i] * A[i];   // Elmore D
        for (int i = b; i < e; ++i) B[i] *= A[i];                      // C_i D_i
        for (int i = e - 1; i > b; --i) B[b + par[i]] += B[i];          // M
        B[b] = 0.f;
        for (int i = b + 1; i < e; ++i) B[i] = B[b + par[i]] + f * R[i] * B[i];   // beta
        for (int q = f0; q < f1; ++q) {
            const int node = b + c.fo_node[q];
            const int s = c.fo_pin[q];
            const float Dn = A[node];
            c.netD[(size_t)s * K + k] = 1e-6f * Dn;
            c.netV[(size_t)s * K + k] = 1e-12f * fmaxf(2.f * B[node] - Dn * Dn, 0.f);
        }
    }
}

__device__ __forceinline__ float2 pin_pos(const DevCtx &c, int p)
{
    const int pc = c.pin_cell[p];
    if (pc >= 0) return make_float2(c.cell_xy[2 * (size_t)pc], c.cell_xy[2 * (size_t)pc + 1]);
    const int q = -pc - 1;
    return make_float2(c.port_xy[2 * (size_t)q], c.port_xy[2 * (size_t)q + 1]);
}

// Star trees from positions: segment R = r L, C = c L (half at each end),
// D = R (C/2 + Cpin), var = D^2 (the second moment of a single RC).
__global__ void k_net_star(const DevCtx c)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= c.I) return;
    const int f0 = c.fo_ptr[g], f1 = c.fo_ptr[g + 1];
    if (f0 == f1) return;
    const int z = item_out_pin(c, c.item_type[g], c.item_pin0[g]);
    const float2 pz = pin_pos(c, z);
    const int K = c.K;
    for (int k = 0; k < K; ++k) {
        const float f = __ldg(c.rc_scale + k);
        const float r = f * c.r_per_um, cc = f * c.c_per_um;
        float ld = 0.f;
        for (int q = f0; q < f1; ++q) {
            const int s = c.fo_pin[q];
            const float2 ps = pin_pos(c, s);
            const float L = fabsf(pz.x - ps.x) + fabsf(pz.y - ps.y);
            const float cp = 1e3f * c.fo_cap[q];
            const float Dr = r * L * fmaf(0.5f * cc, L, cp);
            const float Dn = 1e-6f * Dr;
            c.netD[(size_t)s * K + k] = Dn;
            c.netV[(size_t)s * K + k] = Dn * Dn;
            ld += fmaf(cc, L, cp);
        }
        c.load[(size_t)z * K + k] = 1e-3f * ld;
    }
}

// --------------------------------------------------------------- forward

template <bool SMOOTH>
__device__ __forceinline__ void fwd_item(const DevCtx &c, int g)
{
    const int t = c.item_type[g];
    const int pin0 = c.item_pin0[g];
    const int K = c.K;
    if (t < 0) {   // primary input
        const float4 a = make_float4(c.pi_at, c.pi_at, c.pi_at, c.pi_at);
        const float4 s = make_float4(c.pi_slew, c.pi_slew, c.pi_slew, c.pi_slew);
        for (int k = 0; k < K; ++k) {
            c.at[(size_t)pin0 * K + k] = a;
            c.slew[(size_t)pin0 * K + k] = s;
        }
        return;
    }
    if (__ldg(c.type_kind + t) == 1) {   // flip-flop: ideal clock at CK, arc CK(rise) -> Q
        const int ck = pin0, q = pin0 + 1;
        const float cs = c.clk_slew;
        const float *tb = table(c, t, 1, 0);
        for (int k = 0; k < K; ++k) {
            const float sc = __ldg(c.lut_scale + k);
            const float ld = c.load[(size_t)q * K + k];
            c.at[(size_t)ck * K + k] = make_float4(0.f, 0.f, 0.f, 0.f);
            c.slew[(size_t)ck * K + k] = make_float4(cs, cs, cs, cs);
            const float dr = sc * lut_eval(tb, cs, ld), df = sc * lut_eval(tb + kLutStride, cs, ld);
            const float sr = sc * lut_eval(tb + 2 * kLutStride, cs, ld), sf = sc * lut_eval(tb + 3 * kLutStride, cs, ld);
            c.at[(size_t)q * K + k] = make_float4(dr, df, dr, df);
            c.slew[(size_t)q * K + k] = make_float4(sr, sf, sr, sf);
        }
        return;
    }
    const int nin = __ldg(c.type_nin + t);
    const int z = pin0 + nin;
    int sense[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) sense[j] = j < nin ? __ldg(c.arc_sense + t * 3 + j) : -1;
    for (int k = 0; k < K; ++k) {
        float4 A[3], S[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j < nin) {
                const int a = pin0 + j;
                const int d = c.drv_of[a];
                const float4 ad = c.at[(size_t)d * K + k], sd = c.slew[(size_t)d * K + k];
                const float Dn = c.netD[(size_t)a * K + k], V = c.netV[(size_t)a * K + k];
                A[j] = make_float4(ad.x + Dn, ad.y + Dn, ad.z + Dn, ad.w + Dn);
                S[j] = make_float4(sqrtf(fmaf(sd.x, sd.x, V)), sqrtf(fmaf(sd.y, sd.y, V)), sqrtf(fmaf(sd.z, sd.z, V)),
                                   sqrtf(fmaf(sd.w, sd.w, V)));
                c.at[(size_t)a * K + k] = A[j];
                c.slew[(size_t)a * K + k] = S[j];
            }
        }
        const float sc = __ldg(c.lut_scale + k);
        const float ld = c.load[(size_t)z * K + k];
        float oa[4], os[4];
#pragma unroll
        for (int rfo = 0; rfo < 2; ++rfo) {
            Merge<true, SMOOTH> la, ls;
            Merge<false, SMOOTH> ea, es;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (j >= nin) continue;
                const float *td = table(c, t, j, rfo), *ts = table(c, t, j, 2 + rfo);
#pragma unroll
                for (int rfi = 0; rfi < 2; ++rfi) {
                    const bool on = sense[j] == 2 || (sense[j] == 0 && rfi == rfo) || (sense[j] == 1 && rfi != rfo);
                    if (!on) continue;
                    const float se = comp(S[j], rfi), sl = comp(S[j], 2 + rfi);
                    ea.add(comp(A[j], rfi) + sc * lut_eval(td, se, ld), c.inv_gamma);
                    es.add(sc * lut_eval(ts, se, ld), c.inv_gamma);
                    la.add(comp(A[j], 2 + rfi) + sc * lut_eval(td, sl, ld), c.inv_gamma);
                    ls.add(sc * lut_eval(ts, sl, ld), c.inv_gamma);
                }
            }
            oa[rfo] = ea.get(c.gamma);
            os[rfo] = es.get(c.gamma);
            oa[2 + rfo] = la.get(c.gamma);
            os[2 + rfo] = ls.get(c.gamma);
        }
        c.at[(size_t)z * K + k] = make_float4(oa[0], oa[1], oa[2], oa[3]);
        c.slew[(size_t)z * K + k] = make_float4(os[0], os[1], os[2], os[3]);
    }
}

template <bool SMOOTH>
__global__ void k_fwd_level(const DevCtx c, int i0, int i1)
{
    const int g = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (g < i1) fwd_item<SMOOTH>(c, g);
}

// ------------------------------------------------------------- endpoints

// Arrival at the endpoint through its net, the required times of the ideal
// clock (D: setup capture edge T - setup, hold edge 0 + hold; PO: T and 0),
// pin slack, and the endpoint slacks (min over rise/fall) with violation
// flags.
__global__ void k_endpoints(const DevCtx c)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.E) return;
    const int p = c.ep_pin[e];
    const int d = c.drv_of[p];
    const bool isD = c.ep_is_d[e] != 0;
    const int K = c.K;
    const float rl = isD ? c.period - c.setup : c.period;
    const float re = isD ? c.hold : 0.f;
    for (int k = 0; k < K; ++k) {
        const float4 ad = c.at[(size_t)d * K + k], sd = c.slew[(size_t)d * K + k];
        const float Dn = c.netD[(size_t)p * K + k], V = c.netV[(size_t)p * K + k];
        const float4 A = make_float4(ad.x + Dn, ad.y + Dn, ad.z + Dn, ad.w + Dn);
        const float4 S = make_float4(sqrtf(fmaf(sd.x, sd.x, V)), sqrtf(fmaf(sd.y, sd.y, V)),
                                     sqrtf(fmaf(sd.z, sd.z, V)), sqrtf(fmaf(sd.w, sd.w, V)));
        c.at[(size_t)p * K + k] = A;
        c.slew[(size_t)p * K + k] = S;
        c.rat[(size_t)p * K + k] = make_float4(re, re, rl, rl);
        const float4 sk = make_float4(A.x - re, A.y - re, rl - A.z, rl - A.w);
        c.slack[(size_t)p * K + k] = sk;
        const float ss = fminf(sk.z, sk.w), hs = fminf(sk.x, sk.y);
        c.ep_setup[(size_t)e * K + k] = ss;
        c.ep_hold[(size_t)e * K + k] = hs;
        c.viol_setup[(size_t)e * K + k] = ss < 0.f;
        c.viol_hold[(size_t)e * K + k] = hs < 0.f;
    }
}

// -------------------------------------------------------------- backward

__device__ __forceinline__ void bwd_item(const DevCtx &c, int g)
{
    const int t = c.item_type[g];
    const int pin0 = c.item_pin0[g];
    const int z = item_out_pin(c, t, pin0);
    const int f0 = c.fo_ptr[g], f1 = c.fo_ptr[g + 1];
    const int K = c.K;
    const int kind = t >= 0 ? __ldg(c.type_kind + t) : -1;
    const int nin = t >= 0 ? __ldg(c.type_nin + t) : 0;
    for (int k = 0; k < K; ++k) {
        float4 R = make_float4(-INFINITY, -INFINITY, INFINITY, INFINITY);
        for (int q = f0; q < f1; ++q) {
            const int s = c.fo_pin[q];
            const float4 r = c.rat[(size_t)s * K + k];
            const float Dn = c.netD[(size_t)s * K + k];
            R.x = fmaxf(R.x, r.x - Dn);
            R.y = fmaxf(R.y, r.y - Dn);
            R.z = fminf(R.z, r.z - Dn);
            R.w = fminf(R.w, r.w - Dn);
        }
        const float4 Az = c.at[(size_t)z * K + k];
        c.rat[(size_t)z * K + k] = R;
        c.slack[(size_t)z * K + k] = make_float4(Az.x - R.x, Az.y - R.y, R.z - Az.z, R.w - Az.w);
        if (t < 0) continue;
        const float sc = __ldg(c.lut_scale + k);
        const float ld = c.load[(size_t)z * K + k];
        if (kind == 1) {
            const int ck = pin0;
            const float4 S = c.slew[(size_t)ck * K + k];
            const float *tb = table(c, t, 1, 0);
            const float er = fmaxf(R.x - sc * lut_eval(tb, S.x, ld), R.y - sc * lut_eval(tb + kLutStride, S.x, ld));
            const float lr = fminf(R.z - sc * lut_eval(tb, S.z, ld), R.w - sc * lut_eval(tb + kLutStride, S.z, ld));
            const float4 Rc = make_float4(er, -INFINITY, lr, INFINITY);
            const float4 Ac = c.at[(size_t)ck * K + k];
            c.rat[(size_t)ck * K + k] = Rc;
            c.slack[(size_t)ck * K + k] = make_float4(Ac.x - Rc.x, Ac.y - Rc.y, Rc.z - Ac.z, Rc.w - Ac.w);
            continue;
        }
        for (int j = 0; j < nin; ++j) {
            const int a = pin0 + j;
            const int se = __ldg(c.arc_sense + t * 3 + j);
            const float4 S = c.slew[(size_t)a * K + k];
            float r[4];
#pragma unroll
            for (int el = 0; el < 2; ++el) {
#pragma unroll
                for (int rfi = 0; rfi < 2; ++rfi) {
                    float acc = el ? INFINITY : -INFINITY;
                    const float s_in = comp(S, el * 2 + rfi);
#pragma unroll
                    for (int rfo = 0; rfo < 2; ++rfo) {
                        const bool on = se == 2 || (se == 0 && rfi == rfo) || (se == 1 && rfi != rfo);
                        if (!on) continue;
                        const float cand = comp(R, el * 2 + rfo) - sc * lut_eval(table(c, t, j, rfo), s_in, ld);
                        acc = el ? fminf(acc, cand) : fmaxf(acc, cand);
                    }
                    r[el * 2 + rfi] = acc;
                }
            }
            const float4 Ra = make_float4(r[0], r[1], r[2], r[3]);
            const float4 Aa = c.at[(size_t)a * K + k];
            c.rat[(size_t)a * K + k] = Ra;
            c.slack[(size_t)a * K + k] = make_float4(Aa.x - Ra.x, Aa.y - Ra.y, Ra.z - Aa.z, Ra.w - Aa.w);
        }
    }
}

__global__ void k_bwd_level(const DevCtx c, int i0, int i1)
{
    const int g = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (g < i1) bwd_item(c, g);
}

// ------------------------------------------------------------- reduction

// Two-stage FP64 reduction of the endpoint slacks, deterministic (fixed
// thread-to-element assignment and fixed tree order).  Stage 1: block b of
// corner k reduces endpoint chunk b (chunks never straddle designs) into six
// partials (TNS setup, TNS hold, worst setup, worst hold, violation counts).
// Stage 2: one block per (design, corner) folds that design's chunks into
// WNS = min(0, worst), TNS = sum of negatives.
template <int NT>
__device__ __forceinline__ void block_fold6(double v[6], double (*sh)[NT])
{
#pragma unroll
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
            sh[3][threadIdx.x] = fmin(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
            sh[4][threadIdx.x] += sh[4][threadIdx.x + w];
            sh[5][threadIdx.x] += sh[5][threadIdx.x + w];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_chunks(const DevCtx c)
{
    __shared__ double sh[6][kRedThreads];
    const int b = blockIdx.x, k = blockIdx.y, K = c.K;
    const int e0 = c.red_chunk_ptr[b], e1 = c.red_chunk_ptr[b + 1];
    double v[6] = {0, 0, INFINITY, INFINITY, 0, 0};
    for (int e = e0 + threadIdx.x; e < e1; e += kRedThreads) {
        const double ss = c.ep_setup[(size_t)e * K + k], hs = c.ep_hold[(size_t)e * K + k];
        v[2] = fmin(v[2], ss);
        v[3] = fmin(v[3], hs);
        if (ss < 0) { v[0] += ss; v[4] += 1; }
        if (hs < 0) { v[1] += hs; v[5] += 1; }
    }
    block_fold6<kRedThreads>(v, sh);
    if (threadIdx.x < 6) c.red_partial[((size_t)b * K + k) * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const DevCtx c)
{
    __shared__ double sh[6][kRedThreads];
    const int d = blockIdx.x / c.K, k = blockIdx.x % c.K, K = c.K;
    const int b0 = c.red_design_chunk[d], b1 = c.red_design_chunk[d + 1];
    double v[6] = {0, 0, INFINITY, INFINITY, 0, 0};
    for (int b = b0 + threadIdx.x; b < b1; b += kRedThreads) {
        const double *p = c.red_partial + ((size_t)b * K + k) * 6;
        v[0] += p[0];
        v[1] += p[1];
        v[2] = fmin(v[2], p[2]);
        v[3] = fmin(v[3], p[3]);
        v[4] += p[4];
        v[5] += p[5];
    }
    block_fold6<kRedThreads>(v, sh);
    if (threadIdx.x == 0) {
        double *o = c.report + ((size_t)d * K + k) * 8;
        o[0] = fmin(0.0, sh[2][0]);
        o[1] = sh[0][0];
        o[2] = fmin(0.0, sh[3][0]);
        o[3] = sh[1][0];
        o[4] = sh[2][0];
        o[5] = sh[3][0];
        o[6] = sh[4][0];
        o[7] = sh[5][0];
    }
}

void launch_reduce(const DevCtx &c, const HostSched &h, cudaStream_t st)
{
    if (h.n_red_chunks > 0) k_reduce_chunks<<<dim3(h.n_red_chunks, c.K), kRedThreads, 0, st>>>(c);
    k_reduce_final<<<c.n_designs * c.K, kRedThreads, 0, st>>>(c);
}

// ------------------------------------------------------------- gathers

// out[p] = arr[gpu_of[p]] for every caller pin p (K float4 each).
__global__ void k_gather_pins(const float4 *__restrict__ arr, const int32_t *__restrict__ gpu_of, float4 *out,
                              int P, int K)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)P * K) return;
    const size_t p = i / K, k = i % K;
    out[i] = arr[(size_t)gpu_of[p] * K + k];
}

// dst[r] = src[idx[r]]
__global__ void k_gather_f32(const float *__restrict__ src, const int32_t *__restrict__ idx, float *dst, int n)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) dst[r] = src[idx[r]];
}

// ------------------------------------------------------------- launchers

void launch_level_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev)
{
    if (ev) cudaEventRecord(ev[0], st);
    if (h.placed) {
        if (c.I > 0) k_net_star<<<nblk(c.I, 128), 128, 0, st>>>(c);
    } else if (h.n_tiles > 0) {
        k_net_tree<<<h.n_tiles, kRcTileNets, 0, st>>>(c);
    }
    if (ev) cudaEventRecord(ev[1], st);
    const int tpb = h.threads > 0 ? h.threads : 128;
    for (int s = 0; s < h.S; ++s) {
        const int i0 = h.stage_ptr[s], i1 = h.stage_ptr[s + 1];
        if (i1 <= i0) continue;
        if (c.gamma > 0.f) k_fwd_level<true><<<nblk(i1 - i0, tpb), tpb, 0, st>>>(c, i0, i1);
        else k_fwd_level<false><<<nblk(i1 - i0, tpb), tpb, 0, st>>>(c, i0, i1);
    }
    if (c.E > 0) k_endpoints<<<nblk(c.E, 256), 256, 0, st>>>(c);
    if (ev) cudaEventRecord(ev[2], st);
    for (int s = h.S - 1; s >= 0; --s) {
        const int i0 = h.stage_ptr[s], i1 = h.stage_ptr[s + 1];
        if (i1 <= i0) continue;
        k_bwd_level<<<nblk(i1 - i0, tpb), tpb, 0, st>>>(c, i0, i1);
    }
    if (ev) cudaEventRecord(ev[3], st);
    launch_reduce(c, h, st);
    if (ev) cudaEventRecord(ev[4], st);
}

void launch_gather_pins(const float4 *arr, const int32_t *gpu_of, float4 *out, int P, int K, cudaStream_t st)
{
    if ((long long)P * K > 0) k_gather_pins<<<nblk((long long)P * K, 256), 256, 0, st>>>(arr, gpu_of, out, P, K);
}

void launch_gather_f32(const float *src, const int32_t *idx, float *dst, int n, cudaStream_t st)
{
    if (n > 0) k_gather_f32<<<nblk(n, 256), 256, 0, st>>>(src, idx, dst, n);
}

}  // namespace sta
