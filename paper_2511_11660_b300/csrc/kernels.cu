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
#include "item.cuh"
#include "kernels.h"

namespace sta {

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ nets

// RC trees, one thread per (item's net, corner): the K threads of a net are
// adjacent, so their per-sink outputs (corner innermost) are written side by
// side.  A net of at most kRcColNodes nodes
// lives in a shared-memory column of its thread: node i at [i * kRcThreads +
// thread], so every access of the sweeps -- the parent's entry included --
// falls in the thread's own bank.  The loads that fill the column are
// unrolled over the column height (predicated on the net size), so all of a
// thread's loads are in flight together.  Larger nets sweep the same way in
// global scratch at their node offsets (one copy of the scratch per corner).  Per corner (node capacitance =
// scaled wire C + sink pin caps, Ohm * fF -> 1e-6 ns):
//   Cdown (reverse sweep), load = Cdown at the root;
//   D_i = D_parent + R_i Cdown_i and, in the same sweep, C_i D_i;
//   M = subtree sums of C D (reverse sweep);
//   beta_i = beta_parent + R_i M_i; var = 2 beta - D^2 at the sinks.
struct ColRef {
    float *base;
    int stride;
    __device__ __forceinline__ float &operator[](int i) const { return base[i * stride]; }
};

// Symmetric 3x3 (or smaller) eigen-decomposition by cyclic Jacobi rotations
// (a row-major, overwritten; eigenvectors in the columns of v).
__device__ __forceinline__ void jacobi3(int q, float a[9], float lam[3], float v[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = (i % 4 == 0) ? 1.f : 0.f;
    for (int sweep = 0; sweep < 8; ++sweep) {
        const float off = fabsf(a[1]) + fabsf(a[2]) + fabsf(a[5]);
        if (!(off > 1e-7f * (fabsf(a[0]) + fabsf(a[4]) + fabsf(a[8])))) break;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int r = p + 1; r < 3; ++r) {
                if (r >= q) continue;
                const float apr = a[p * 3 + r];
                if (fabsf(apr) < 1e-30f) continue;
                const float theta = (a[r * 3 + r] - a[p * 3 + p]) / (2.f * apr);
                const float tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
                const float cs = rsqrtf(tt * tt + 1.f), sn = tt * cs;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float akp = a[k * 3 + p], akr = a[k * 3 + r];
                    a[k * 3 + p] = cs * akp - sn * akr;
                    a[k * 3 + r] = sn * akp + cs * akr;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float apk = a[p * 3 + k], ark = a[r * 3 + k];
                    a[p * 3 + k] = cs * apk - sn * ark;
                    a[r * 3 + k] = sn * apk + cs * ark;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float vkp = v[k * 3 + p], vkr = v[k * 3 + r];
                    v[k * 3 + p] = cs * vkp - sn * vkr;
                    v[k * 3 + r] = sn * vkp + cs * vkr;
                }
            }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) lam[i] = a[i * 4];
}

// The Arnoldi reduced-order delays of one net at one corner (STA_NET_ARNOLDI),
// the same steps as the FP64 reference in FP32 with q <= 3:
//   Krylov basis of G^-1 Cn from v1 = 1/sqrt(m) (implicit) -- each new
//   direction by one tree solve (subtree sums, then path sums of R times
//   them), modified Gram-Schmidt, and the basis stops when the orthogonal
//   part is below 1e-5 of the direction (space exhausted); v2 in A, v3 in B;
//   G_r = sum over edges of dv dv / R, C_r = sum Cn v v, b_r = sum over the
//   driver's edges of v / R; C_r = L L^T, M = L^-1 G_r L^-T = W diag(l) W^T;
//   sink s: v_s(t) = sum_k a_k (1 - exp(-l_k t)) with a_k = (h^T w_k)
//   (w_k^T M^-1 L^-1 b_r), h = L^-1 V^T e_s; netD = the 50% crossing,
//   bracketed by doubling, then safeguarded Newton steps inside the bracket
//   (bisection wherever a step would leave it) to FP32 resolution.
template <class Par, class Rf>
__device__ void arnoldi_delays(const DevCtx &c, int n, float f, int q_req, const ColRef &A, const ColRef &B,
                               const ColRef &Cn, Par par, Rf Rv, int f0, int f1, int K, int k)
{
    const int m = n - 1;
    const int qmax = min(q_req, m);
    const float c1 = rsqrtf((float)m);
    int qq = 1;
    // direction 2 from v1, direction 3 from v2
    for (int j = 1; j < qmax; ++j) {
        const ColRef &X = j == 1 ? A : B;   // the new direction's column
        for (int i = 1; i < n; ++i) X[i] = Cn[i] * (j == 1 ? c1 : A[i]);
        X[0] = 0.f;
        for (int i = n - 1; i > 0; --i) {
            const int p = par(i);
            if (p > 0) X[p] += X[i];
        }
        for (int i = 1; i < n; ++i) X[i] = (par(i) > 0 ? X[par(i)] : 0.f) + f * Rv(i) * X[i];
        float len = 0.f, d1 = 0.f;
        for (int i = 1; i < n; ++i) {
            len += X[i] * X[i];
            d1 += c1 * X[i];
        }
        len = sqrtf(len);
        for (int i = 1; i < n; ++i) X[i] -= d1 * c1;
        if (j == 2) {
            float d2 = 0.f;
            for (int i = 1; i < n; ++i) d2 += A[i] * X[i];
            for (int i = 1; i < n; ++i) X[i] -= d2 * A[i];
        }
        float nrm = 0.f;
        for (int i = 1; i < n; ++i) nrm += X[i] * X[i];
        nrm = sqrtf(nrm);
        if (!(nrm > 1e-5f * len)) break;
        const float inv = 1.f / nrm;
        for (int i = 1; i < n; ++i) X[i] *= inv;
        qq = j + 1;
    }
    // projected matrices
    float Gr[9] = {}, Cr[9] = {}, br[3] = {};
    for (int i = 1; i < n; ++i) {
        const int p = par(i);
        const float g = 1.f / (f * Rv(i));
        const float v[3] = {c1, qq > 1 ? A[i] : 0.f, qq > 2 ? B[i] : 0.f};
        const float vp[3] = {p > 0 ? c1 : 0.f, (qq > 1 && p > 0) ? A[p] : 0.f, (qq > 2 && p > 0) ? B[p] : 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (p == 0) br[a] += v[a] * g;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Gr[a * 3 + b] += (v[a] - vp[a]) * (v[b] - vp[b]) * g;
                Cr[a * 3 + b] += Cn[i] * v[a] * v[b];
            }
        }
    }
    // Cholesky of C_r, M = L^-1 G_r L^-T, eigen-decomposition, modal steady state
    float L[9] = {}, T[9] = {}, M[9] = {}, W[9], lam[3], cc[3] = {}, yinf[3] = {};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            if (i >= qq) continue;
            float s = Cr[i * 3 + j];
#pragma unroll
            for (int t = 0; t < j; ++t) s -= L[i * 3 + t] * L[j * 3 + t];
            if (i == j) L[i * 4] = sqrtf(fmaxf(s, 1e-30f));
            else L[i * 3 + j] = s / L[j * 4];
        }
#pragma unroll
    for (int col = 0; col < 3; ++col)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i >= qq || col >= qq) continue;
            float s = Gr[i * 3 + col];
#pragma unroll
            for (int t = 0; t < i; ++t) s -= L[i * 3 + t] * T[t * 3 + col];
            T[i * 3 + col] = s / L[i * 4];
        }
#pragma unroll
    for (int row = 0; row < 3; ++row)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i >= qq || row >= qq) continue;
            float s = T[row * 3 + i];
#pragma unroll
            for (int t = 0; t < i; ++t) s -= L[i * 3 + t] * M[row * 3 + t];
            M[row * 3 + i] = s / L[i * 4];
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i + 1; j < 3; ++j) M[i * 3 + j] = M[j * 3 + i] = 0.5f * (M[i * 3 + j] + M[j * 3 + i]);
    jacobi3(qq, M, lam, W);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i >= qq) continue;
        float s = br[i];
#pragma unroll
        for (int t = 0; t < i; ++t) s -= L[i * 3 + t] * cc[t];
        cc[i] = s / L[i * 4];
    }
    float lmin = INFINITY;
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        if (kk >= qq) continue;
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i < qq) s += W[i * 3 + kk] * cc[i];
        yinf[kk] = s / lam[kk];
        lmin = fminf(lmin, lam[kk]);
    }
    // every sink: its modal weights and its 50% crossing
    for (int q = f0; q < f1; ++q) {
        const int node = chk(c, __ldg(c.fo_node + q), n);
        const int s = chk(c, __ldg(c.fo_pin + q), c.P);
        float t50 = 0.f;
        if (node > 0) {
            const float e[3] = {c1, qq > 1 ? A[node] : 0.f, qq > 2 ? B[node] : 0.f};
            float h[3] = {}, a[3] = {};
            float vinf = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i >= qq) continue;
                float sum = e[i];
#pragma unroll
                for (int t = 0; t < i; ++t) sum -= L[i * 3 + t] * h[t];
                h[i] = sum / L[i * 4];
            }
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                if (kk >= qq) continue;
                float sum = 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    if (i < qq) sum += h[i] * W[i * 3 + kk];
                a[kk] = sum * yinf[kk];
                vinf += a[kk];
            }
            // v(t) - vinf/2 and its derivative (one exponential per pole)
            auto resp = [&](float t, float &dv) {
                float v = -0.5f * vinf;
                dv = 0.f;
#pragma unroll
                for (int kk = 0; kk < 3; ++kk)
                    if (kk < qq) {
                        const float ex = expf(-lam[kk] * t);
                        v += a[kk] * (1.f - ex);
                        dv += a[kk] * lam[kk] * ex;
                    }
                return v;
            };
            float dv;
            float lo = 0.f, hi = 1.f / lmin;
            for (int it = 0; it < 64 && resp(hi, dv) < 0.f; ++it) {
                lo = hi;
                hi *= 2.f;
            }
            // safeguarded Newton inside [lo, hi], from the dominant pole's ln 2 / l
            float t = fminf(fmaxf(0.69314718f / lmin, lo), hi);
            for (int it = 0; it < 24 && hi - lo > 1e-7f * hi; ++it) {
                const float v = resp(t, dv);
                if (v >= 0.f) hi = t;
                else lo = t;
                float tn = t - v / dv;
                if (!(dv > 0.f) || !(tn > lo && tn < hi)) tn = 0.5f * (lo + hi);
                t = tn;
            }
            t50 = t;
        }
        c.netD[(size_t)s * K + k] = 1e-6f * t50;
    }
}

// the net values of state k (a corner's first exception tag) copied to the
// corner's other tags
__device__ __forceinline__ void copy_to_tags(const DevCtx &c, int z, int f0, int f1, int k)
{
    const int K = c.K;
    const float ld = c.load[(size_t)z * K + k];
    for (int g = 1; g < c.Tg; ++g) c.load[(size_t)z * K + k + g] = ld;
    for (int q = f0; q < f1; ++q) {
        const int s = chk(c, __ldg(c.fo_pin + q), c.P);
        const float Dn = c.netD[(size_t)s * K + k], Vn = c.netV[(size_t)s * K + k];
        for (int g = 1; g < c.Tg; ++g) {
            c.netD[(size_t)s * K + k + g] = Dn;
            c.netV[(size_t)s * K + k + g] = Vn;
        }
    }
}

// The Elmore sweeps of one net (load, D, second moment, variance).  Node
// columns A and B and the net's parents, R and C sit in shared memory (node
// i at element i * kRcThreads of each column) when the net fits there
// (col), else in global memory (the scratch columns, the plan's RC arrays).
// SH: every net of the warp fits, so the sweeps use shared-memory accesses
// only; otherwise each thread picks its own columns (generic accesses, the
// warp's nets of both kinds in one pass).
template <bool SH>
__device__ __forceinline__ void rc_elmore(const DevCtx &c, float *sA, float *sB, const int8_t *spar, const float *sR,
                                          const float *sC, float *gA, float *gB, bool col, int n0, int n, int f0,
                                          int f1, int z, int k, float f)
{
    constexpr int S = kRcThreads;
    const int K = c.K;
    const bool sh = SH || col;
    auto A = [&](int i) -> float & { return sh ? sA[i * S] : gA[i]; };
    auto B = [&](int i) -> float & { return sh ? sB[i * S] : gB[i]; };
    auto par = [&](int i) -> int { return sh ? spar[i * S] : chk(c, __ldg(c.rc_parent + n0 + i), i); };
    auto Rv = [&](int i) -> float { return sh ? sR[i * S] : __ldg(c.rc_R + n0 + i); };
    auto Cv = [&](int i) -> float { return sh ? sC[i * S] : __ldg(c.rc_C + n0 + i); };
    // every rounding is spelled out (products, sums, one FMA per node in
    // the D and beta sweeps), not left to the compiler's contraction
    for (int i = 0; i < n; ++i) {
        const float ci = __fmul_rn(f, Cv(i));
        A(i) = ci;
        B(i) = ci;
    }
    for (int q0 = f0; q0 < f1; q0 += 4) {
        int nd[4];
        float cp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (q0 + u < f1) {
                nd[u] = chk(c, __ldg(c.fo_node + q0 + u), n);
                cp[u] = __fmul_rn(1e3f, __ldg(c.fo_cap + q0 + u));
            }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (q0 + u < f1) {
                A(nd[u]) = __fadd_rn(A(nd[u]), cp[u]);
                B(nd[u]) = __fadd_rn(B(nd[u]), cp[u]);             // node capacitance
            }
    }
    for (int i = n - 1; i > 0; --i) A(par(i)) = __fadd_rn(A(par(i)), A(i));   // Cdown
    c.load[(size_t)z * K + k] = __fmul_rn(1e-3f, A(0));
    A(0) = 0.f;
    B(0) = 0.f;
    for (int i = 1; i < n; ++i) {
        const float d = fmaf(__fmul_rn(f, Rv(i)), A(i), A(par(i)));   // Elmore D
        A(i) = d;
        B(i) = __fmul_rn(B(i), d);                                     // C_i D_i
    }
    for (int i = n - 1; i > 0; --i) B(par(i)) = __fadd_rn(B(par(i)), B(i));   // M
    B(0) = 0.f;
    for (int i = 1; i < n; ++i) B(i) = fmaf(__fmul_rn(f, Rv(i)), B(i), B(par(i)));   // beta
    for (int q0 = f0; q0 < f1; q0 += 4) {
        int nd[4], sp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (q0 + u < f1) {
                nd[u] = chk(c, __ldg(c.fo_node + q0 + u), n);
                sp[u] = chk(c, __ldg(c.fo_pin + q0 + u), c.P);
            }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (q0 + u < f1) {
                const float Dn = A(nd[u]);
                c.netD[(size_t)sp[u] * K + k] = __fmul_rn(1e-6f, Dn);
                c.netV[(size_t)sp[u] * K + k] = __fmul_rn(1e-12f, fmaxf(fmaf(-Dn, Dn, __fmul_rn(2.f, B(nd[u]))), 0.f));
            }
    }
}

__global__ void __launch_bounds__(kRcThreads) k_net_tree(const DevCtx c)
{
    __shared__ int8_t s_par[kRcColNodes * kRcThreads];
    __shared__ float s_R[kRcColNodes * kRcThreads], s_C[kRcColNodes * kRcThreads];
    __shared__ float s_A[kRcColNodes * kRcThreads], s_B[kRcColNodes * kRcThreads];
    const int t = threadIdx.x;
    // one thread per (net, corner); the exception tags of a corner share
    // its net values, computed at the corner's first state and copied
    const long long gk = (long long)blockIdx.x * kRcThreads + t;
    if (gk >= (long long)c.I * c.Kc) return;
    // (net, corner) from the thread index: I * Kc < 2^31 (checked at set-up)
    const unsigned u = (unsigned)gk, nk = (unsigned)c.Kc;
    const int g = nk == 1u ? (int)u : (int)(u / nk), kc = nk == 1u ? 0 : (int)(u % nk), k = kc * c.Tg;
    const int n0 = chk(c, c.rc_ptr[g], c.NN + 1);
    const int n = c.steiner ? chk(c, c.st_nlive[g], chk(c, c.rc_ptr[g + 1], c.NN + 1) - n0 + 1)
                            : chk(c, c.rc_ptr[g + 1], c.NN + 1) - n0;
    const int f0 = chk(c, c.fo_ptr[g], (long long)c.F + 1), f1 = chk(c, c.fo_ptr[g + 1], (long long)c.F + 1);
    if (n <= 0) return;
    const bool col = n <= kRcColNodes;
    if (col) {
        int8_t pv[kRcColNodes];
        float rv[kRcColNodes], cv[kRcColNodes];
#pragma unroll
        for (int i = 0; i < kRcColNodes; ++i)
            if (i < n) {
                pv[i] = (int8_t)(i ? chk(c, __ldg(c.rc_parent + n0 + i), i) : 0);
                rv[i] = __ldg(c.rc_R + n0 + i);
                cv[i] = __ldg(c.rc_C + n0 + i);
            }
#pragma unroll
        for (int i = 0; i < kRcColNodes; ++i)
            if (i < n) {
                s_par[i * kRcThreads + t] = pv[i];
                s_R[i * kRcThreads + t] = rv[i];
                s_C[i * kRcThreads + t] = cv[i];
            }
    }
    const size_t so = (size_t)kc * c.NN + n0;   // global scratch: one copy per corner
    const int z = chk(c, item_out_pin(c, chk_type(c, c.item_type[g]), c.item_pin0[g]), c.P);
    const float f = __ldg(c.rc_scale + k);
    if (__all_sync(__activemask(), col))
        rc_elmore<true>(c, s_A + t, s_B + t, s_par + t, s_R + t, s_C + t, nullptr, nullptr, true, n0, n, f0, f1, z, k, f);
    else
        rc_elmore<false>(c, s_A + t, s_B + t, s_par + t, s_R + t, s_C + t, c.scratch_a + so, c.scratch_b + so, col, n0,
                         n, f0, f1, z, k, f);
    if (c.net_model == kNetArnoldi && n > 1) {
        const ColRef A = col ? ColRef{s_A + t, kRcThreads} : ColRef{c.scratch_a + so, 1};
        const ColRef B = col ? ColRef{s_B + t, kRcThreads} : ColRef{c.scratch_b + so, 1};
        auto par = [&](int i) -> int { return col ? s_par[i * kRcThreads + t] : chk(c, __ldg(c.rc_parent + n0 + i), i); };
        auto Rv = [&](int i) -> float { return col ? s_R[i * kRcThreads + t] : __ldg(c.rc_R + n0 + i); };
        auto Cv = [&](int i) -> float { return col ? s_C[i * kRcThreads + t] : __ldg(c.rc_C + n0 + i); };
        // node capacitance again (wire * f + sink pins), in the C column
        const ColRef Cn = col ? ColRef{s_C + t, kRcThreads} : ColRef{c.scratch_c + so, 1};
        for (int i = 0; i < n; ++i) Cn[i] = f * Cv(i);
        for (int q = f0; q < f1; ++q) Cn[chk(c, __ldg(c.fo_node + q), n)] += 1e3f * __ldg(c.fo_cap + q);
        arnoldi_delays(c, n, f, c.arnoldi_q, A, B, Cn, par, Rv, f0, f1, c.K, k);
    }
    if (c.Tg > 1) copy_to_tags(c, z, f0, f1, k);
}

// Star trees from positions: segment R = r L, C = c L (half at each end),
// D = R (C/2 + Cpin), var = D^2 (the second moment of a single RC).
__global__ void k_net_star(const DevCtx c)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= c.I) return;
    const int f0 = chk(c, c.fo_ptr[g], (long long)c.F + 1), f1 = chk(c, c.fo_ptr[g + 1], (long long)c.F + 1);
    if (f0 >= f1) return;
    const int z = chk(c, item_out_pin(c, chk_type(c, c.item_type[g]), c.item_pin0[g]), c.P);
    const float2 pz = pin_pos(c, z);
    const int K = c.K;
    for (int k = 0; k < K; k += c.Tg) {   // a corner's first exception tag, copied to the others
        const float f = __ldg(c.rc_scale + k);
        const float r = f * c.r_per_um, cc = f * c.c_per_um;
        float ld = 0.f;
        // four sinks at a time, their (read-only) loads in flight together;
        // the load is summed in net order as before
        for (int q0 = f0; q0 < f1; q0 += 4) {
            int s[4];
            float L[4], cp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                s[u] = q0 + u < f1 ? chk(c, __ldg(c.fo_pin + q0 + u), c.P) : -1;
                cp[u] = q0 + u < f1 ? 1e3f * __ldg(c.fo_cap + q0 + u) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                L[u] = 0.f;
                if (s[u] < 0) continue;
                const int pc = __ldg(c.pin_cell + s[u]);
                float2 ps;
                if (pc >= 0) {
                    const int cl = chk(c, pc, c.C);
                    ps = make_float2(__ldg(c.cell_xy + 2 * (size_t)cl), __ldg(c.cell_xy + 2 * (size_t)cl + 1));
                } else {
                    const int pq = -pc - 1;
                    ps = make_float2(__ldg(c.port_xy + 2 * (size_t)pq), __ldg(c.port_xy + 2 * (size_t)pq + 1));
                }
                L[u] = fabsf(pz.x - ps.x) + fabsf(pz.y - ps.y);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (s[u] < 0) continue;
                const float Dr = r * L[u] * fmaf(0.5f * cc, L[u], cp[u]);
                const float Dn = 1e-6f * Dr;
                c.netD[(size_t)s[u] * K + k] = Dn;
                c.netV[(size_t)s[u] * K + k] = Dn * Dn;
                ld += fmaf(cc, L[u], cp[u]);
            }
        }
        c.load[(size_t)z * K + k] = 1e-3f * ld;
        if (c.Tg > 1) copy_to_tags(c, z, f0, f1, k);
    }
}

// ------------------------------------------------- level-schedule passes

// One launch per level: four lanes per item run fwd_run / bwd_run
// (item.cuh), reading tables through the read-only cache.
// The level kernels run one wave of independent items per launch and wait on
// their loads: capped at 64 registers (a few spilled values) they keep 32
// warps a SM in flight instead of 18 (64 designs x 4 corners: 14.5 -> 12.3 ms
// an update).
template <bool SMOOTH, bool UNIFORM>
__global__ void __maxnreg__(64) k_fwd_level(const DevCtx c, int i0, int i1)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = i0 + tid / (4 * c.KL);
    if (g < i1) {
        const FwdItem f = fwd_prep(c, c.type_nin, c.type_kind, c.arc_sense, g);
        fwd_run<SMOOTH, UNIFORM, false>(c, LutGlobal{c.lut, c.lut_scale}, f, FwdIn{}, g, tid & 3, 0);
    }
}

__global__ void k_endpoints(const DevCtx c)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = tid / (4 * c.KL);
    if (e < c.E) ep_run<false>(c, ep_prep(c, e), 0.f, 0.f, e, tid & 3, 0);
}

void launch_endpoints(const DevCtx &c, cudaStream_t st)
{
    if (c.E > 0) k_endpoints<<<nblk(4LL * c.KL * c.E, 256), 256, 0, st>>>(c);
}

template <bool UNIFORM>
__global__ void __maxnreg__(64) k_bwd_level(const DevCtx c, int i0, int i1)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = i0 + tid / (4 * c.KL);
    if (g < i1) bwd_run<UNIFORM, false>(c, LutGlobal{c.lut, c.lut_scale}, c.arc_sense,
                                        bwd_prep(c, c.type_nin, c.type_kind, g, tid & 3), tid & 3, 0, 0.f);
}

// ------------------------------------------------------------- reduction

// Two-stage FP64 reduction of the endpoint slacks, deterministic (fixed
// thread-to-element assignment and fixed tree order).  Stage 1: block b of
// corner k reduces endpoint chunk b (chunks never straddle designs) into six
// partials (TNS setup, TNS hold, worst setup, worst hold, violation counts).
// Stage 2: one block per (design, corner) folds that design's chunks into
// WNS = min(0, worst), TNS = sum of negatives.
// The partials of a reduction: TNS setup and hold (FP64 sums of FP32
// slacks), worst setup and hold (FP32, exact), violation counts (integers).
// Only the sums take FP64 arithmetic, B300's FP64 pipe being narrow.
struct Fold6 {
    double ts, th;
    float ms, mh;
    int ns, nh;
};
__device__ __forceinline__ Fold6 fold6_init() { return Fold6{0.0, 0.0, INFINITY, INFINITY, 0, 0}; }
__device__ __forceinline__ void fold6_add(Fold6 &a, const Fold6 &b)
{
    a.ts += b.ts;
    a.th += b.th;
    a.ms = fminf(a.ms, b.ms);
    a.mh = fminf(a.mh, b.mh);
    a.ns += b.ns;
    a.nh += b.nh;
}
// A block's partials folded in a fixed order: a butterfly across each warp
// (every lane ends with the same value: each step combines the same two
// operands), then thread 0 folds the warps' values in warp order; its
// return value is the block's result.
template <int NT>
__device__ __forceinline__ Fold6 block_fold6(Fold6 f, Fold6 *sh)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Fold6 o;
        o.ts = __shfl_xor_sync(0xffffffffu, f.ts, off);
        o.th = __shfl_xor_sync(0xffffffffu, f.th, off);
        o.ms = __shfl_xor_sync(0xffffffffu, f.ms, off);
        o.mh = __shfl_xor_sync(0xffffffffu, f.mh, off);
        o.ns = __shfl_xor_sync(0xffffffffu, f.ns, off);
        o.nh = __shfl_xor_sync(0xffffffffu, f.nh, off);
        fold6_add(f, o);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = f;
    __syncthreads();
    Fold6 r = sh[0];
    if (threadIdx.x == 0)
        for (int w = 1; w < NT / 32; ++w) fold6_add(r, sh[w]);
    return r;
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_chunks(const DevCtx c)
{
    __shared__ Fold6 sh[kRedThreads / 32];
    const int b = blockIdx.x, k = blockIdx.y, K = c.Kc;
    const int e0 = c.red_chunk_ptr[b], e1 = c.red_chunk_ptr[b + 1];
    // thread t folds endpoints e0 + t + i * kRedThreads in increasing i; every
    // slack is loaded first, so the loads are in flight together
    constexpr int kPer = kRedChunk / kRedThreads;
    float fsv[kPer], fhv[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int e = e0 + threadIdx.x + i * kRedThreads;
        // the endpoint's slack at corner k: min over its exception tags
        float fs = INFINITY, fh = INFINITY;
        if (e < e1)
            for (int g = 0; g < c.Tg; ++g) {
                fs = fminf(fs, c.ep_setup[(size_t)e * c.K + k * c.Tg + g]);
                fh = fminf(fh, c.ep_hold[(size_t)e * c.K + k * c.Tg + g]);
            }
        fsv[i] = fs;
        fhv[i] = fh;
    }
    Fold6 f = fold6_init();
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        if (e0 + (int)threadIdx.x + i * kRedThreads >= e1) break;
        const float fs = fsv[i], fh = fhv[i];
        f.ms = fminf(f.ms, fs);
        f.mh = fminf(f.mh, fh);
        if (fs < 0.f) { f.ts += (double)fs; ++f.ns; }
        if (fh < 0.f) { f.th += (double)fh; ++f.nh; }
    }
    f = block_fold6<kRedThreads>(f, sh);
    if (threadIdx.x == 0) {
        double *o = c.red_partial + ((size_t)b * K + k) * 6;
        o[0] = f.ts;
        o[1] = f.th;
        o[2] = f.ms;
        o[3] = f.mh;
        o[4] = f.ns;
        o[5] = f.nh;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const DevCtx c)
{
    __shared__ Fold6 sh[kRedThreads / 32];
    const int d = blockIdx.x / c.Kc, k = blockIdx.x % c.Kc, K = c.Kc;
    const int b0 = c.red_design_chunk[d], b1 = c.red_design_chunk[d + 1];
    Fold6 f = fold6_init();
    for (int b = b0 + threadIdx.x; b < b1; b += kRedThreads) {
        const double *p = c.red_partial + ((size_t)b * K + k) * 6;
        // minima and counts were stored from FP32 values and integers: exact
        fold6_add(f, Fold6{p[0], p[1], (float)p[2], (float)p[3], (int)p[4], (int)p[5]});
    }
    f = block_fold6<kRedThreads>(f, sh);
    if (threadIdx.x == 0) {
        double *o = c.report + ((size_t)d * K + k) * 8;
        o[0] = fmin(0.0, (double)f.ms);
        o[1] = f.ts;
        o[2] = fmin(0.0, (double)f.mh);
        o[3] = f.th;
        o[4] = f.ms;
        o[5] = f.mh;
        o[6] = f.ns;
        o[7] = f.nh;
    }
}

void launch_reduce(const DevCtx &c, const HostSched &h, cudaStream_t st)
{
    if (h.n_red_chunks > 0) k_reduce_chunks<<<dim3(h.n_red_chunks, c.Kc), kRedThreads, 0, st>>>(c);
    k_reduce_final<<<c.n_designs * c.Kc, kRedThreads, 0, st>>>(c);
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

// Resize cells: new type per cell (same input count and kind), and the pin
// capacitance of its input pins in the fan-out lists of their nets.
__global__ void k_resize(const DevCtx c, const int32_t *__restrict__ item_of_cell, const int32_t *__restrict__ fo_of_pin,
                         const float *__restrict__ type_pin_cap, const int32_t *__restrict__ cells,
                         const int32_t *__restrict__ types, int n, int32_t *item_type)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cell = cells[i], t = types[i];
    if (cell < 0 || cell >= c.C || t < 0 || t >= c.T) {
        atomicOr(c.err, kErrResize);
        return;
    }
    const int g = item_of_cell[cell];
    const int old = item_type[g];
    if (c.type_nin[t] != c.type_nin[old] || c.type_kind[t] != c.type_kind[old]) {
        atomicOr(c.err, kErrResize);
        return;
    }
    item_type[g] = t;
    const int pin0 = c.item_pin0[g];
    if (c.type_kind[t] == 1) return;   // a flip-flop's D pin: see the endpoint entry below
    for (int s = 0; s < c.type_nin[t]; ++s) {
        const int q = fo_of_pin[pin0 + s];
        if (q >= 0) const_cast<float *>(c.fo_cap)[q] = type_pin_cap[t * 4 + s];
    }
}

// Flip-flops: the D pin lives in the endpoint region; its fan-out entry is
// found through the caller pin map.
__global__ void k_resize_dff(const DevCtx c, const int32_t *__restrict__ item_of_cell,
                             const int32_t *__restrict__ d_pin_of_cell, const int32_t *__restrict__ fo_of_pin,
                             const float *__restrict__ type_pin_cap, const int32_t *__restrict__ cells,
                             const int32_t *__restrict__ types, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cell = cells[i], t = types[i];
    if (cell < 0 || cell >= c.C || t < 0 || t >= c.T || c.type_kind[t] != 1) return;
    const int dp = d_pin_of_cell[cell];
    if (dp < 0) return;
    const int q = fo_of_pin[dp];
    if (q >= 0) const_cast<float *>(c.fo_cap)[q] = type_pin_cap[t * 4];
}

void launch_resize(const DevCtx &c, const int32_t *item_of_cell, const int32_t *d_pin_of_cell,
                   const int32_t *fo_of_pin, const float *type_pin_cap, const int32_t *cells, const int32_t *types,
                   int n, int32_t *item_type, cudaStream_t st)
{
    if (n <= 0) return;
    k_resize<<<nblk(n, 256), 256, 0, st>>>(c, item_of_cell, fo_of_pin, type_pin_cap, cells, types, n, item_type);
    k_resize_dff<<<nblk(n, 256), 256, 0, st>>>(c, item_of_cell, d_pin_of_cell, fo_of_pin, type_pin_cap, cells,
                                               types, n);
}

// dst[r] = src[idx[r]]
__global__ void k_gather_f32(const float *__restrict__ src, const int32_t *__restrict__ idx, float *dst, int n)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) dst[r] = src[idx[r]];
}

// ------------------------------------------------------------- launchers

void launch_net_star(const DevCtx &c, cudaStream_t st) { k_net_star<<<nblk(c.I, 128), 128, 0, st>>>(c); }

void launch_net_tree(const DevCtx &c, cudaStream_t st)
{
    if (c.I > 0) k_net_tree<<<nblk((long long)c.I * c.Kc, kRcThreads), kRcThreads, 0, st>>>(c);
}

void launch_net_phase(const DevCtx &c, const HostSched &h, cudaStream_t st)
{
    if (h.steiner) {
        launch_net_steiner(c, st);
        launch_net_tree(c, st);
    } else if (h.placed) {
        if (c.I > 0) launch_net_star(c, st);
    } else if (h.rc) {
        launch_net_tree(c, st);
    }
}

__global__ void k_gather_i64(const int64_t *src, const int32_t *idx, int64_t *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = src[idx[i]];
}

void launch_gather_i64(const int64_t *src, const int32_t *idx, int64_t *out, int n, cudaStream_t st)
{
    if (n > 0) k_gather_i64<<<nblk(n, 256), 256, 0, st>>>(src, idx, out, n);
}

void launch_level_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev)
{
    if (ev) cudaEventRecord(ev[0], st);
    launch_net_phase(c, h, st);
    if (ev) cudaEventRecord(ev[1], st);
    const int tpb = h.threads > 0 ? h.threads : 128;
    for (int s = 0; s < h.S; ++s) {
        const int i0 = h.stage_ptr[s], i1 = h.stage_ptr[s + 1];
        if (i1 <= i0) continue;
        const dim3 grid(nblk(4LL * c.KL * (i1 - i0), tpb));
        if (c.gamma > 0.f) {
            if (h.uniform) k_fwd_level<true, true><<<grid, tpb, 0, st>>>(c, i0, i1);
            else k_fwd_level<true, false><<<grid, tpb, 0, st>>>(c, i0, i1);
        } else {
            if (h.uniform) k_fwd_level<false, true><<<grid, tpb, 0, st>>>(c, i0, i1);
            else k_fwd_level<false, false><<<grid, tpb, 0, st>>>(c, i0, i1);
        }
    }
    launch_endpoints(c, st);
    if (ev) cudaEventRecord(ev[2], st);
    for (int s = h.S - 1; s >= 0; --s) {
        const int i0 = h.stage_ptr[s], i1 = h.stage_ptr[s + 1];
        if (i1 <= i0) continue;
        if (h.uniform) k_bwd_level<true><<<nblk(4LL * c.KL * (i1 - i0), tpb), tpb, 0, st>>>(c, i0, i1);
        else k_bwd_level<false><<<nblk(4LL * c.KL * (i1 - i0), tpb), tpb, 0, st>>>(c, i0, i1);
    }
    if (ev) cudaEventRecord(ev[3], st);
    launch_reduce(c, h, st);
    if (ev) cudaEventRecord(ev[4], st);
}

void launch_gather_pins(const float4 *arr, const int32_t *gpu_of, float4 *out, int P, int K, cudaStream_t st)
{
    if ((long long)P * K > 0) k_gather_pins<<<nblk((long long)P * K, 256), 256, 0, st>>>(arr, gpu_of, out, P, K);
}

// The same for a double-float array (arrival or required times), rounded to FP32.
__global__ void k_gather_pins_d(const DF4 *__restrict__ arr, const int32_t *__restrict__ gpu_of, float4 *out, int P,
                                int K)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)P * K) return;
    const size_t p = i / K, k = i % K;
    const DF4 v = arr[(size_t)gpu_of[p] * K + k];
    out[i] = make_float4(to_f(v.v[0]), to_f(v.v[1]), to_f(v.v[2]), to_f(v.v[3]));
}

void launch_gather_pins_d(const DF4 *arr, const int32_t *gpu_of, float4 *out, int P, int K, cudaStream_t st)
{
    if ((long long)P * K > 0) k_gather_pins_d<<<nblk((long long)P * K, 256), 256, 0, st>>>(arr, gpu_of, out, P, K);
}

__global__ void k_collapse_tags(const DevCtx c, float *ep, uint8_t *viol)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t EK = (size_t)c.E * c.Kc;
    if (i >= EK) return;
    const size_t e = i / c.Kc, k = i % c.Kc;
    float s = INFINITY, h = INFINITY;
    for (int g = 0; g < c.Tg; ++g) {
        s = fminf(s, c.ep_setup[e * c.K + k * c.Tg + g]);
        h = fminf(h, c.ep_hold[e * c.K + k * c.Tg + g]);
    }
    ep[i] = s;
    ep[EK + i] = h;
    viol[i] = s < 0.f;
    viol[EK + i] = h < 0.f;
}

void launch_collapse_tags(const DevCtx &c, float *ep, uint8_t *viol, cudaStream_t st)
{
    if ((long long)c.E * c.Kc > 0) k_collapse_tags<<<nblk((long long)c.E * c.Kc, 256), 256, 0, st>>>(c, ep, viol);
}

void launch_gather_f32(const float *src, const int32_t *idx, float *dst, int n, cudaStream_t st)
{
    if (n > 0) k_gather_f32<<<nblk(n, 256), 256, 0, st>>>(src, idx, dst, n);
}

}  // namespace sta
