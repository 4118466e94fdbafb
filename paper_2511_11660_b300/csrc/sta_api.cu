// sta_api.cu -- the C ABI of libsta.so (see include/sta.h).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "plan.h"
#include "sta.h"
#include "tile.h"

using sta::DevCtx;
using sta::HostSched;
using sta::Plan;

struct sta_ctx {
    int device = 0;
    Plan plan;
    DevCtx dc{};
    HostSched hs;
    std::vector<void *> allocs;
    size_t bytes = 0;
    int32_t *d_gpu_of = nullptr;
    // device-side resizing (allocated at the first sta_resize_cells)
    int32_t *d_item_of_cell = nullptr, *d_d_pin_of_cell = nullptr, *d_fo_of_pin = nullptr;
    float *d_type_pin_cap = nullptr;
    int32_t *d_resize_tmp = nullptr;
    int32_t resize_cap = 0;
    int32_t *d_rc_src = nullptr;
    int32_t *d_item_of_net = nullptr;   // Steiner contexts: driving item of every caller net
    int64_t *d_wl_tmp = nullptr;        // staging of sta_get_net_wirelength to the host
    float *d_rc_tmp = nullptr;
    // sta_set_rc_async: two staging buffers (R then C), copy-done and
    // buffer-free events, the buffer the next update applies (-1: none)
    float *d_stage[2] = {nullptr, nullptr};
    cudaEvent_t stage_copied[2] = {nullptr, nullptr}, stage_free[2] = {nullptr, nullptr};
    int stage_next = 0, stage_pending = -1;
    float4 *d_gather_tmp = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    int schedule = STA_SCHED_LEVEL;
    int sched_param = 0;
    bool updated = false;
    bool profiling = false;
    cudaEvent_t ev[5] = {};
    float last_ms[4] = {0, 0, 0, 0};
    std::string msg;
    // caller pin -> (cell, slot) for resizing
    std::vector<int32_t> pin_cell_c, pin_slot_c;
    // endpoint slacks collapsed over exception tags (allocated at first use)
    float *d_ep_collapse = nullptr;
    uint8_t *d_viol_collapse = nullptr;
    // path reports (allocated at the first sta_report_paths)
    sta::PathJob pj{};
    int32_t path_cap = 0;   // pins the path buffers hold
    // tile schedule: the partition's device arrays (rebuilt when the tile
    // count changes) and its statistics
    std::vector<void *> tile_allocs;
    size_t tile_bytes = 0;
    sta::TilePlan tile_stats;   // sizes and statistics only (vectors cleared after the upload)
};

namespace {

thread_local std::string g_plan_err;

// quads per item: states handled side by side (1, 2, 4 or 8)
int32_t quads_per_item(int32_t K) { return K >= 8 ? 8 : K >= 4 ? 4 : K >= 2 ? 2 : 1; }

struct CudaFail {
    cudaError_t e;
    const char *what;
};

#define CK(call)                                        \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) throw CudaFail{_e, #call}; \
    } while (0)

sta_status fail(sta_ctx *c, sta_status st, const std::string &m)
{
    if (c) c->msg = m;
    return st;
}

sta_status from_cuda(sta_ctx *c, const CudaFail &f)
{
    const sta_status st = (f.e == cudaErrorMemoryAllocation) ? STA_ENOMEM : STA_ECUDA;
    return fail(c, st, std::string(f.what) + ": " + cudaGetErrorString(f.e));
}

template <class T>
T *dev_alloc(sta_ctx *c, size_t n)
{
    void *p = nullptr;
    const size_t b = std::max<size_t>(n * sizeof(T), 16);
    CK(cudaMalloc(&p, b));
    c->allocs.push_back(p);
    c->bytes += b;
    return static_cast<T *>(p);
}

template <class T>
T *upload(sta_ctx *c, const std::vector<T> &v)
{
    T *p = dev_alloc<T>(c, v.size());
    if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

void drop_graph(sta_ctx *c)
{
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
}

void record_pass(sta_ctx *c, cudaStream_t st, cudaEvent_t *ev = nullptr)
{
    if (c->schedule == STA_SCHED_DATAFLOW) sta::launch_dataflow_pass(c->dc, c->hs, st, ev);
    else if (c->schedule == STA_SCHED_COOP) sta::launch_coop_pass(c->dc, c->hs, st, ev);
    else if (c->schedule == STA_SCHED_TILE) sta::launch_tile_pass(c->dc, c->hs, st, ev);
    else sta::launch_level_pass(c->dc, c->hs, st, ev);
}

void free_tiles(sta_ctx *c)
{
    for (void *p : c->tile_allocs) cudaFree(p);
    c->tile_allocs.clear();
    c->bytes -= c->tile_bytes;
    c->tile_bytes = 0;
    c->dc.tl_B = 0;
}

template <class T>
T *tile_upload(sta_ctx *c, const std::vector<T> &v)
{
    void *p = nullptr;
    const size_t b = std::max<size_t>(v.size() * sizeof(T), 16);
    CK(cudaMalloc(&p, b));
    c->tile_allocs.push_back(p);
    c->tile_bytes += b;
    c->bytes += b;
    if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return static_cast<T *>(p);
}

// Partition the graph into B tiles and upload the lists, descriptors and
// ring codes (tile.cpp).
void build_tiles(sta_ctx *c, int B)
{
    if (c->dc.tl_B == B) return;
    free_tiles(c);
    sta::TilePlan tp;
    const int W = sta::tile_threads() / (4 * c->dc.KL);
    sta::build_tile_plan(c->plan, B, W, sta::tile_ring_slots(c->dc.KL), tp);
    sta::DevCtx &d = c->dc;
    d.tl_ptr = tile_upload(c, tp.ptr);
    d.tl_nitem = tile_upload(c, tp.nitem);
    d.tl_rbase = tile_upload(c, tp.rbase);
    d.tl_fdesc = reinterpret_cast<const int4 *>(tile_upload(c, tp.fdesc));
    d.tl_bdesc = reinterpret_cast<const int4 *>(tile_upload(c, tp.bdesc));
    d.tl_fo_ring = tile_upload(c, tp.fo_ring);
    d.tl_NS = tp.NS;
    d.tl_R = tp.R;
    d.tl_B = B;
    c->hs.tile_blocks = B;
    tp.ptr.clear();
    tp.nitem.clear();
    tp.rbase.clear();
    tp.item.clear();
    tp.fdesc.clear();
    tp.bdesc.clear();
    tp.fo_ring.clear();
    tp.tile_of.clear();
    c->tile_stats = std::move(tp);
}

void ensure_graph(sta_ctx *c)
{
    if (c->exec) return;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    record_pass(c, c->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) throw CudaFail{e, "cudaStreamEndCapture"};
    c->graph = g;
    CK(cudaGraphInstantiate(&c->exec, c->graph, 0));
}

sta_status create_from_plan(sta_ctx *c, int device)
{
    Plan &pl = c->plan;
    c->device = device;
    // the RC sweep numbers its (net, corner) threads in 32 bits
    if ((long long)pl.I * pl.Kc >= (1LL << 31))
        return fail(c, STA_EINVAL, "too many items x corners (must be below 2^31)");
    CK(cudaSetDevice(device));
    CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    DevCtx &d = c->dc;
    d.P = pl.P;
    d.I = pl.I;
    d.S = pl.S;
    d.E = pl.E;
    d.K = pl.K;
    d.Kc = pl.Kc;
    d.Tg = pl.Tg;
    d.NN = pl.NN;
    d.F = (int32_t)pl.F;
    d.net_model = pl.net_model;
    d.arnoldi_q = pl.arnoldi_q;
    d.T = pl.T;
    d.C = pl.C;
    d.n_designs = pl.n_designs;
    d.period = pl.period;
    d.clk_slew = pl.clk_slew;
    d.pi_at = pl.pi_at;
    d.pi_slew = pl.pi_slew;
    d.setup = pl.setup;
    d.hold = pl.hold;
    d.gamma = pl.gamma;
    d.inv_gamma = pl.gamma > 0 ? 1.f / pl.gamma : 0.f;
    d.r_per_um = pl.r_per_um;
    d.c_per_um = pl.c_per_um;
    d.lut = upload(c, pl.lut);
    d.type_nin = upload(c, pl.type_nin);
    d.type_kind = upload(c, pl.type_kind);
    d.arc_sense = upload(c, pl.arc_sense);
    d.lut_scale = upload(c, pl.lut_scale);
    d.rc_scale = upload(c, pl.rc_scale);
    d.item_pin0 = upload(c, pl.item_pin0);
    d.item_type = upload(c, pl.item_type);
    d.item_cell = upload(c, pl.item_cell);
    d.fo_ptr = upload(c, pl.fo_ptr);
    d.fo_pin = upload(c, pl.fo_pin);
    d.fo_node = upload(c, pl.fo_node);
    d.fo_cap = upload(c, pl.fo_cap);
    d.rc_ptr = upload(c, pl.rc_ptr);
    d.rc_parent = upload(c, pl.rc_parent);
    d.rc_R = upload(c, pl.rc_R);
    d.rc_C = upload(c, pl.rc_C);
    d.drv_of = upload(c, pl.drv_of);
    d.pin_cell = upload(c, pl.pin_cell);
    d.port_xy = upload(c, pl.port_xy);
    d.cell_xy = upload(c, pl.cell_xy.empty() ? std::vector<float>(2 * (size_t)pl.C, 0.f) : pl.cell_xy);
    d.ep_pin = upload(c, pl.ep_pin);
    d.ep_is_d = upload(c, pl.ep_is_d);
    d.ep_design_ptr = upload(c, pl.ep_design_ptr);
    c->d_gpu_of = upload(c, pl.gpu_of);
    {
        std::vector<int32_t> src(pl.rc_src.begin(), pl.rc_src.end());
        c->d_rc_src = upload(c, src);
    }
    const size_t PK = (size_t)pl.P * pl.K;
    d.at = dev_alloc<sta::DF4>(c, PK);
    d.slew = dev_alloc<float4>(c, PK);
    d.rat = dev_alloc<sta::DF4>(c, PK);
    d.slack = dev_alloc<float4>(c, PK);
    d.netD = dev_alloc<float>(c, PK);
    d.netV = dev_alloc<float>(c, PK);
    d.load = dev_alloc<float>(c, PK);
    CK(cudaMemset(d.netD, 0, PK * sizeof(float)));
    CK(cudaMemset(d.netV, 0, PK * sizeof(float)));
    CK(cudaMemset(d.load, 0, PK * sizeof(float)));
    const size_t EK = (size_t)pl.E * pl.K;
    d.ep_setup = dev_alloc<float>(c, EK);
    d.ep_hold = dev_alloc<float>(c, EK);
    d.viol_setup = dev_alloc<uint8_t>(c, EK);
    d.viol_hold = dev_alloc<uint8_t>(c, EK);
    d.report = dev_alloc<double>(c, (size_t)pl.n_designs * pl.Kc * 8);
    if (pl.Tg > 1) {
        d.item_tag = upload(c, pl.item_tag);
        d.ep_mult = upload(c, pl.ep_mult);
        d.ep_off = reinterpret_cast<const float2 *>(upload(c, pl.ep_off));
        d.pin_adv = pl.pin_adv.empty() ? nullptr : upload(c, pl.pin_adv);
    }
    {
        // reduction chunks: <= kRedChunk endpoints, never straddling designs
        std::vector<int32_t> cp{0}, dc{0};
        for (int32_t dd = 0; dd < pl.n_designs; ++dd) {
            for (int32_t e = pl.ep_design_ptr[dd]; e < pl.ep_design_ptr[dd + 1]; e += sta::kRedChunk)
                cp.push_back(std::min(e + sta::kRedChunk, pl.ep_design_ptr[dd + 1]));
            dc.push_back((int32_t)cp.size() - 1);
        }
        c->hs.n_red_chunks = (int)cp.size() - 1;
        d.red_chunk_ptr = upload(c, cp);
        d.red_design_chunk = upload(c, dc);
        d.red_partial = dev_alloc<double>(c, std::max<size_t>(1, cp.size() - 1) * pl.Kc * 6);
    }
    d.err = dev_alloc<unsigned>(c, 1);
    CK(cudaMemset(d.err, 0, sizeof(unsigned)));
    if (pl.steiner) {
        // Steiner trees: the RC arrays are written on the device at every update
        d.steiner = 1;
        d.r_per_um_y = pl.r_per_um_y;
        d.c_per_um_y = pl.c_per_um_y;
        const size_t NN = std::max<int64_t>(1, pl.NN), WN = std::max<int64_t>(1, pl.st_node_ptr[pl.I]);
        d.st_parent = dev_alloc<int32_t>(c, NN);
        d.st_R = dev_alloc<float>(c, NN);
        d.st_C = dev_alloc<float>(c, NN);
        d.st_fo_node = dev_alloc<int32_t>(c, std::max<int64_t>(1, pl.F));
        d.st_nlive = dev_alloc<int32_t>(c, std::max(1, pl.I));
        d.st_wl = dev_alloc<int64_t>(c, std::max(1, pl.I));
        CK(cudaMemset(d.st_nlive, 0, std::max(1, pl.I) * sizeof(int32_t)));
        CK(cudaMemset(d.st_wl, 0, std::max(1, pl.I) * sizeof(int64_t)));
        CK(cudaMemset(d.st_fo_node, 0, std::max<int64_t>(1, pl.F) * sizeof(int32_t)));
        d.st_node_ptr = upload(c, pl.st_node_ptr);
        d.st_adj_ptr = upload(c, pl.st_adj_ptr);
        d.st_x = dev_alloc<long long>(c, WN);
        d.st_y = dev_alloc<long long>(c, WN);
        d.st_key = dev_alloc<long long>(c, WN);
        d.st_aux = dev_alloc<int32_t>(c, 3 * WN);
        d.st_capw = dev_alloc<float>(c, WN);
        d.st_items = upload(c, pl.st_items);
        d.st_n_items = (int32_t)pl.st_items.size();
        d.st_small = pl.st_small;
        d.st_adj_tiny = 0;
        while (d.st_adj_tiny < d.st_n_items &&
               pl.fo_ptr[pl.st_items[d.st_adj_tiny] + 1] - pl.fo_ptr[pl.st_items[d.st_adj_tiny]] + 1 <=
                   sta::kAdjTinyPins)
            ++d.st_adj_tiny;
        d.st_adj_small = d.st_adj_tiny;
        while (d.st_adj_small < d.st_n_items &&
               pl.fo_ptr[pl.st_items[d.st_adj_small] + 1] - pl.fo_ptr[pl.st_items[d.st_adj_small]] + 1 <=
                   sta::kAdjSmallPins)
            ++d.st_adj_small;
        d.st_adj = dev_alloc<unsigned>(c, std::max<int64_t>(1, pl.st_adj_ptr[pl.I]));
        if (pl.gamma > 0.f) d.st_src = dev_alloc<int2>(c, NN);   // read by sta_backward
        d.rc_parent = d.st_parent;
        d.rc_R = d.st_R;
        d.rc_C = d.st_C;
        d.fo_node = d.st_fo_node;
        std::vector<int32_t> item_of_net(std::max(1, pl.n_nets), -1);
        for (int32_t g = 0; g < pl.I; ++g)
            if (pl.net_of_item[g] >= 0) item_of_net[pl.net_of_item[g]] = g;
        c->d_item_of_net = upload(c, item_of_net);
    }
    if (pl.n_big_nets > 0) {
        d.scratch_a = dev_alloc<float>(c, (size_t)pl.NN * pl.Kc);
        d.scratch_b = dev_alloc<float>(c, (size_t)pl.NN * pl.Kc);
        if (pl.net_model == STA_NET_ARNOLDI) d.scratch_c = dev_alloc<float>(c, (size_t)pl.NN * pl.Kc);
    }
    HostSched &h = c->hs;
    h.S = pl.S;
    h.stage_ptr = pl.stage_ptr;
    h.rc = !pl.placed && pl.NN > 0;
    h.placed = pl.placed;
    h.steiner = pl.steiner;
    h.thru = !pl.pin_adv.empty();
    h.threads = 128;
    h.uniform = pl.uniform_axes;
    if (pl.uniform_axes) {
        for (int i = 0; i < 7; ++i) {
            d.ax1[i] = pl.axes[i];
            d.ax2[i] = pl.axes[7 + i];
        }
        for (int i = 0; i < 6; ++i) {
            d.iw1[i] = pl.axes[14 + i];
            d.iw2[i] = pl.axes[20 + i];
        }
    }
    h.T = pl.T;
    // dataflow schedule: parity mailboxes (all NaN), epoch state, work chunks
    d.fbox_len = 2 * (size_t)pl.I * pl.K;   // forward mailboxes: one record per item output
    d.rbox_len = 2 * (size_t)std::max<int64_t>(pl.F, 1) * pl.K;   // one record per fan-out entry
    d.fbox_a = dev_alloc<sta::DF4>(c, d.fbox_len);
    d.fbox_s = dev_alloc<float4>(c, d.fbox_len);
    d.rbox = dev_alloc<sta::DF4>(c, d.rbox_len);
    CK(cudaMemset(d.fbox_a, 0xFF, std::max<size_t>(1, d.fbox_len) * sizeof(sta::DF4)));   // all NaN
    CK(cudaMemset(d.fbox_s, 0xFF, std::max<size_t>(1, d.fbox_len) * sizeof(float4)));
    CK(cudaMemset(d.rbox, 0xFF, std::max<size_t>(1, d.rbox_len) * sizeof(sta::DF4)));
    d.df_state = dev_alloc<unsigned>(c, sta::kDfStateWords);
    CK(cudaMemset(d.df_state, 0, sta::kDfStateWords * sizeof(unsigned)));
    d.stage_ptr = upload(c, pl.stage_ptr);
    d.ep_begin = pl.P - pl.E;
    d.hold_item = -1;
    d.spin_limit = 1LL << 23;
    {
        // a warp works on 8 / KL items, 4 * KL lanes each (KL corners side by side)
        d.KL = quads_per_item(pl.K);
        h.one = d.K == 1 && d.KL == 1 && !h.thru;
        const int32_t kChunkItems = 8 / d.KL;
        // Forward work list: the item chunks of each level.  The endpoints
        // are not in it: one launch after the pass computes them all at once
        // (every driver is final by then), where chunks of them in the list
        // held warps that the items needed (1M cells: forward 0.537 ->
        // 0.453 ms without them).
        std::vector<int32_t> out_item(pl.P, -1);
        for (int32_t g = 0; g < pl.I; ++g) {
            const int32_t t = pl.item_type[g], p0 = pl.item_pin0[g];
            out_item[t < 0 ? p0 : (pl.type_kind[t] == 1 ? p0 + 1 : p0 + pl.type_nin[t])] = g;
        }
        {   // the mailbox index (driver item) of every gate input
            std::vector<int32_t> idrv((size_t)pl.I * 3, 0);
            for (int32_t g = 0; g < pl.I; ++g) {
                const int32_t t = pl.item_type[g];
                if (t < 0 || pl.type_kind[t] != 0) continue;
                for (int32_t j = 0; j < pl.type_nin[t] && j < 3; ++j) {
                    const int32_t dp = pl.drv_of[pl.item_pin0[g] + j];
                    idrv[(size_t)g * 3 + j] = dp >= 0 && out_item[dp] >= 0 ? out_item[dp] : 0;
                }
            }
            d.item_drv = upload(c, idrv);
            // the required-time mailbox of a gate input is its entry in its
            // driver's fan-out list: a driver's sinks are then contiguous
            std::vector<int32_t> pfo(pl.P, -1);
            for (int64_t q = 0; q < pl.F; ++q)
                if (pl.fo_pin[q] < pl.P - pl.E) pfo[pl.fo_pin[q]] = (int32_t)q;
            for (int32_t g = 0; g < pl.I; ++g) {   // every gate input is driven (the plan requires it)
                const int32_t t = pl.item_type[g];
                if (t < 0 || pl.type_kind[t] != 0) continue;
                for (int32_t j = 0; j < pl.type_nin[t]; ++j)
                    if (pfo[pl.item_pin0[g] + j] < 0) return fail(c, STA_EINVAL, "internal: an undriven gate input");
            }
            d.pin_fo = upload(c, pfo);
        }
        std::vector<int32_t> flo, fhi, blo, bhi;
        for (int32_t s = 0; s < pl.S; ++s)
            for (int32_t g = pl.stage_ptr[s]; g < pl.stage_ptr[s + 1]; g += kChunkItems) {
                flo.push_back(g);
                fhi.push_back(std::min(g + kChunkItems, pl.stage_ptr[s + 1]));
            }
        // Backward work order: levels deepest first; inside a level the items
        // by cell type (a warp's lanes take the same table branch), then by
        // the position of their last sink item (the one taken last, whose
        // required time completes last; items whose sinks are all endpoints
        // first), so that a chunk's items tend to become ready together.
        std::vector<int32_t> pin_item(pl.P, -1), bpos(pl.I, -1), bord;
        bord.reserve(pl.I);
        for (int32_t g = 0; g < pl.I; ++g) {
            const int32_t t = pl.item_type[g], p0 = pl.item_pin0[g];
            const int32_t z = t < 0 ? p0 : (pl.type_kind[t] == 1 ? p0 + 1 : p0 + pl.type_nin[t]);
            for (int32_t p = p0; p <= z; ++p) pin_item[p] = g;
        }
        std::vector<std::pair<int64_t, int32_t>> key;
        for (int32_t s = pl.S - 1; s >= 0; --s) {
            key.clear();
            for (int32_t g = pl.stage_ptr[s]; g < pl.stage_ptr[s + 1]; ++g) {
                int32_t k = -1;
                for (int32_t q = pl.fo_ptr[g]; q < pl.fo_ptr[g + 1]; ++q) {
                    const int32_t sp = pl.fo_pin[q];
                    if (sp < pl.P - pl.E && pin_item[sp] >= 0) k = std::max(k, bpos[pin_item[sp]]);
                }
                key.emplace_back(((int64_t)(pl.item_type[g] + 1) << 32) + (k + 1), g);
            }
            std::stable_sort(key.begin(), key.end(),
                             [](const std::pair<int64_t, int32_t> &a, const std::pair<int64_t, int32_t> &b) {
                                 return a.first < b.first;
                             });
            const int32_t first = (int32_t)bord.size();
            for (const auto &kg : key) {
                bpos[kg.second] = (int32_t)bord.size();
                bord.push_back(kg.second);
            }
            const int32_t last = (int32_t)bord.size();
            for (int32_t x = first; x < last; x += kChunkItems) {
                blo.push_back(x);
                bhi.push_back(std::min(x + kChunkItems, last));
            }
        }
        d.bwd_order = upload(c, bord);
        d.n_fwd_chunks = (int32_t)flo.size();
        d.n_bwd_chunks = (int32_t)blo.size();
        d.fwd_chunk_lo = upload(c, flo);
        d.fwd_chunk_hi = upload(c, fhi);
        d.bwd_chunk_lo = upload(c, blo);
        d.bwd_chunk_hi = upload(c, bhi);
    }
    for (auto &e : c->ev) CK(cudaEventCreate(&e));
    CK(cudaDeviceSynchronize());
    return STA_OK;
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

// Kernel launches of one update under the current schedule.
int32_t launches_per_update(const sta_ctx *c)
{
    const Plan &pl = c->plan;
    int32_t n = 0;
    if (pl.steiner)   // Steiner trees (small nets, larger nets), then the RC sweep
        n += (pl.st_small > 0) + ((int32_t)pl.st_items.size() > pl.st_small) + (pl.I > 0);
    else if (pl.placed) n += pl.I > 0;
    else n += pl.NN > 0 && pl.I > 0;
    if (c->schedule == STA_SCHED_DATAFLOW) {
        n += 2;                                  // mailbox recovery, epoch / counter reset
        n += c->dc.n_fwd_chunks > 0;
        n += pl.E > 0;                           // the endpoints, after the forward pass
        n += c->dc.n_bwd_chunks > 0;
        n += (c->hs.n_red_chunks > 0) + 1;       // two-stage reduction
        return n;
    }
    if (c->schedule == STA_SCHED_COOP) {
        n += 2;                                  // barrier reset, all levels in one launch
        n += (c->hs.n_red_chunks > 0) + 1;       // two-stage reduction
        return n;
    }
    if (c->schedule == STA_SCHED_TILE) {
        n += 2;                                  // mailbox recovery, epoch reset
        n += (pl.I > 0 || pl.E > 0) + (pl.I > 0);   // forward, backward
        n += (c->hs.n_red_chunks > 0) + 1;       // two-stage reduction
        return n;
    }
    int32_t levels = 0;
    for (int32_t s = 0; s < pl.S; ++s) levels += pl.stage_ptr[s + 1] > pl.stage_ptr[s];
    n += 2 * levels;
    n += pl.E > 0;
    n += (c->hs.n_red_chunks > 0) + 1;   // two-stage reduction
    return n;
}

// Kernel launches of one sta_backward under the current reverse-sweep schedule.
int32_t launches_per_backward(const sta_ctx *c)
{
    const Plan &pl = c->plan;
    if (!(pl.gamma > 0.f) || !pl.placed) return 0;
    int32_t n = 0;
    n += c->hs.n_red_chunks > 0 ? 4 : 0;        // objective: max and sums, two stages each
    n += 1;                                      // objective total
    n += pl.E > 0;                               // endpoint seed
    const bool dataflow = !c->hs.adj_level && sta::adjoint_smem_bytes(pl.T) <= 200 * 1024;
    if (dataflow) {
        n += 3;                                  // mailbox recovery, epoch, persistent sweep
    } else {
        for (int32_t s = 0; s < pl.S; ++s) n += pl.stage_ptr[s + 1] > pl.stage_ptr[s];
    }
    if (pl.steiner)   // Steiner trees: three column sizes
        n += (c->dc.st_adj_tiny > 0) + (c->dc.st_adj_small > c->dc.st_adj_tiny) + (c->dc.st_n_items > c->dc.st_adj_small);
    else n += pl.I > 0;                                    // star segments
    return n;
}

sta_status check_device_error(sta_ctx *c)
{
    unsigned err = 0;
    CK(cudaMemcpy(&err, c->dc.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) {
        CK(cudaMemset(c->dc.err, 0, sizeof(unsigned)));
        if (err & sta::kErrTimeout) return fail(c, STA_ETIMEOUT, "a device-side wait reached its limit");
        if (err & sta::kErrResize)
            return fail(c, STA_EINVAL, "sta_resize_cells: a cell index or type was out of range, or a new type "
                                       "changes the input count or kind (those cells were left unchanged)");
        return fail(c, STA_ECUDA, "device-side bounds check failed");
    }
    return STA_OK;
}

}  // namespace

extern "C" {

const char *sta_status_string(sta_status s)
{
    switch (s) {
    case STA_OK: return "ok";
    case STA_EINVAL: return "invalid argument";
    case STA_ECYCLE: return "combinational cycle";
    case STA_ENOMEM: return "out of memory";
    case STA_ECUDA: return "CUDA error";
    case STA_ETIMEOUT: return "device wait timed out";
    case STA_ESTATE: return "call out of order";
    }
    return "unknown status";
}

sta_status sta_plan(const sta_design_desc *desc, sta_plan_info *out)
{
    Plan pl;
    std::string err;
    const sta_status st = sta::build_plan(desc, pl, err);
    if (st != STA_OK) {
        g_plan_err = err;
        return st;
    }
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->n_pins = pl.P;
        out->n_cells = pl.C;
        out->n_nets = desc->n_nets;
        out->n_items = pl.I;
        out->n_cell_arcs = pl.cell_arcs;
        out->n_net_arcs = pl.F;
        out->n_rc_nodes = pl.placed ? pl.F + desc->n_nets : pl.NN;
        out->n_endpoints = pl.E;
        out->n_levels = pl.S;
        out->n_corners = pl.Kc;
        out->n_tags = pl.Tg;
        out->max_level_width = pl.max_width;
        out->n_designs = 1;
        out->device_bytes = 0;
    }
    return STA_OK;
}

const char *sta_plan_error(void) { return g_plan_err.c_str(); }

namespace {
void fill_tile_info(const sta::TilePlan &tp, sta_tile_info *out)
{
    std::memset(out, 0, sizeof(*out));
    out->n_tiles = tp.B;
    out->n_steps = tp.NS;
    out->wave_items = tp.W;
    out->ring_slots = tp.R;
    out->max_step_entries = tp.max_step_items;
    out->fwd_edges = tp.fwd_edges;
    out->fwd_local = tp.fwd_local;
    out->bwd_edges = tp.bwd_edges;
    out->bwd_local = tp.bwd_local;
    out->crit_edges = tp.crit_edges;
    out->crit_local = tp.crit_local;
}
}  // namespace

sta_status sta_plan_tiles(const sta_design_desc *desc, int32_t n_tiles, sta_tile_info *out)
{
    if (n_tiles < 1) {
        g_plan_err = "n_tiles must be >= 1";
        return STA_EINVAL;
    }
    Plan pl;
    std::string err;
    const sta_status st = sta::build_plan(desc, pl, err);
    if (st != STA_OK) {
        g_plan_err = err;
        return st;
    }
    const int32_t KL = quads_per_item(pl.K);
    sta::TilePlan tp;
    sta::build_tile_plan(pl, n_tiles, sta::tile_threads() / (4 * KL), sta::tile_ring_slots(KL), tp);
    const std::string bad = sta::check_tile_plan(pl, tp);
    if (!bad.empty()) {
        g_plan_err = "tile partition check failed: " + bad;
        return STA_EINVAL;
    }
    if (out) fill_tile_info(tp, out);
    return STA_OK;
}

sta_status sta_get_tile_info(const sta_ctx *c, sta_tile_info *out)
{
    if (!c || !out) return STA_EINVAL;
    if (c->schedule != STA_SCHED_TILE) {
        std::memset(out, 0, sizeof(*out));
        return STA_OK;
    }
    fill_tile_info(c->tile_stats, out);
    return STA_OK;
}

sta_status sta_plan_levels(const sta_design_desc *desc, int32_t *cell_level)
{
    if (!cell_level) return STA_EINVAL;
    Plan pl;
    std::string err;
    const sta_status st = sta::build_plan(desc, pl, err);
    if (st != STA_OK) {
        g_plan_err = err;
        return st;
    }
    for (int32_t c = 0; c < pl.C; ++c) cell_level[c] = pl.cell_level[c];
    return STA_OK;
}

static sta_status finish_create(sta_ctx *c, int device, sta_ctx **out)
{
    try {
        const sta_status st = create_from_plan(c, device);
        if (st != STA_OK) {
            g_plan_err = c->msg;
            sta_destroy(c);
            return st;
        }
    } catch (const CudaFail &f) {
        const sta_status st = from_cuda(c, f);
        g_plan_err = c->msg;
        sta_destroy(c);
        return st;
    } catch (const std::bad_alloc &) {
        g_plan_err = "host allocation failed";
        sta_destroy(c);
        return STA_ENOMEM;
    }
    *out = c;
    return STA_OK;
}

static void keep_pin_maps(sta_ctx *c, const sta_design_desc *const *descs, int32_t n)
{
    int64_t P = 0;
    for (int32_t i = 0; i < n; ++i) P += descs[i]->n_pins;
    c->pin_cell_c.assign(P, -1);
    c->pin_slot_c.assign(P, -1);
    int64_t p0 = 0, c0 = 0;
    for (int32_t i = 0; i < n; ++i) {
        const sta_design_desc &d = *descs[i];
        for (int32_t cc = 0; cc < d.n_cells; ++cc)
            for (int32_t k = d.cell_pin_ptr[cc]; k < d.cell_pin_ptr[cc + 1]; ++k) {
                c->pin_cell_c[p0 + d.cell_pin[k]] = (int32_t)(c0 + cc);
                c->pin_slot_c[p0 + d.cell_pin[k]] = k - d.cell_pin_ptr[cc];
            }
        p0 += d.n_pins;
        c0 += d.n_cells;
    }
}

sta_status sta_create(const sta_design_desc *desc, int device, sta_ctx **out)
{
    if (!out) return STA_EINVAL;
    *out = nullptr;
    sta_ctx *c = new (std::nothrow) sta_ctx();
    if (!c) return STA_ENOMEM;
    std::string err;
    const sta_status st = sta::build_plan(desc, c->plan, err);
    if (st != STA_OK) {
        g_plan_err = err;
        delete c;
        return st;
    }
    keep_pin_maps(c, &desc, 1);
    return finish_create(c, device, out);
}

sta_status sta_create_batch(const sta_design_desc *const *descs, int32_t n_designs, int device, sta_ctx **out)
{
    if (!out) return STA_EINVAL;
    *out = nullptr;
    sta_ctx *c = new (std::nothrow) sta_ctx();
    if (!c) return STA_ENOMEM;
    std::string err;
    const sta_status st = sta::build_batch_plan(descs, n_designs, c->plan, err);
    if (st != STA_OK) {
        g_plan_err = err;
        delete c;
        return st;
    }
    keep_pin_maps(c, descs, n_designs);
    return finish_create(c, device, out);
}

void sta_destroy(sta_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    drop_graph(c);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (int b = 0; b < 2; ++b) {
        if (c->stage_copied[b]) cudaEventDestroy(c->stage_copied[b]);
        if (c->stage_free[b]) cudaEventDestroy(c->stage_free[b]);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (void *p : c->allocs) cudaFree(p);
    for (void *p : c->tile_allocs) cudaFree(p);
    delete c;
}

const char *sta_last_error(const sta_ctx *c) { return c ? c->msg.c_str() : "NULL context"; }

sta_status sta_set_corners(sta_ctx *c, const float *lut_scale, const float *rc_scale)
{
    if (!c || !lut_scale || !rc_scale) return STA_EINVAL;
    const int Kc = c->plan.Kc, Tg = c->plan.Tg, K = c->plan.K;
    for (int k = 0; k < Kc; ++k)
        if (!std::isfinite(lut_scale[k]) || !(lut_scale[k] > 0) || !std::isfinite(rc_scale[k]) || !(rc_scale[k] > 0))
            return fail(c, STA_EINVAL, "corner scales must be finite and > 0");
    std::vector<float> ls(K), rs(K);   // every exception tag of a corner shares its scales
    for (int k = 0; k < K; ++k) {
        ls[k] = lut_scale[k / Tg];
        rs[k] = rc_scale[k / Tg];
    }
    try {
        CK(cudaSetDevice(c->device));
        CK(cudaMemcpy(const_cast<float *>(c->dc.lut_scale), ls.data(), K * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(const_cast<float *>(c->dc.rc_scale), rs.data(), K * sizeof(float), cudaMemcpyHostToDevice));
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    c->plan.lut_scale = ls;
    c->plan.rc_scale = rs;
    return STA_OK;
}

sta_status sta_set_clock(sta_ctx *c, float period_ns)
{
    if (!c) return STA_EINVAL;
    if (!std::isfinite(period_ns)) return fail(c, STA_EINVAL, "period must be finite");
    try {
        CK(cudaSetDevice(c->device));
        drop_graph(c);   // the context is passed to the kernels by value
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    c->plan.period = period_ns;
    c->dc.period = period_ns;
    return STA_OK;
}

sta_status sta_set_schedule(sta_ctx *c, int32_t schedule, int32_t param)
{
    if (!c) return STA_EINVAL;
    if (schedule != STA_SCHED_LEVEL && schedule != STA_SCHED_DATAFLOW && schedule != STA_SCHED_COOP &&
        schedule != STA_SCHED_TILE)
        return fail(c, STA_EINVAL, "unknown schedule");
    if (schedule == STA_SCHED_TILE && c->plan.S + 1 > sta::tile_max_steps())
        return fail(c, STA_EINVAL, "too many levels for the tile schedule");
    if (schedule == STA_SCHED_LEVEL && param != 0 && (param < 32 || param > 1024 || param % 32))
        return fail(c, STA_EINVAL, "threads per block must be a multiple of 32 in [32, 1024]");
    if (schedule != STA_SCHED_LEVEL && (param < 0 || param > 65535))
        return fail(c, STA_EINVAL, "persistent grid size must be in [0, 65535] (0 = from occupancy)");
    if (schedule != STA_SCHED_LEVEL && sta::dataflow_smem_bytes(c->plan.T) > 200 * 1024)
        return fail(c, STA_EINVAL, "cell library too large for the persistent schedules' shared-memory copy");
    try {
        CK(cudaSetDevice(c->device));
        drop_graph(c);
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    c->schedule = schedule;
    c->sched_param = param;
    if (schedule == STA_SCHED_LEVEL) {
        c->hs.threads = param ? param : 128;
    } else if (schedule == STA_SCHED_COOP) {
        const cudaError_t e = sta::coop_prepare(c->hs, c->dc.gamma > 0.f, param);
        if (e != cudaSuccess) {
            c->schedule = STA_SCHED_LEVEL;
            return fail(c, STA_ECUDA, std::string("cooperative set-up: ") + cudaGetErrorString(e));
        }
    } else if (schedule == STA_SCHED_TILE) {
        int max_blocks = 0, sms = 0;
        cudaError_t e = sta::tile_prepare(c->hs, c->dc.gamma > 0.f, c->plan.S + 1, &max_blocks);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        if (e != cudaSuccess) {
            c->schedule = STA_SCHED_LEVEL;
            return fail(c, STA_ECUDA, std::string("tile set-up: ") + cudaGetErrorString(e));
        }
        const int B = param > 0 ? param : std::min(sms, max_blocks);
        if (B > max_blocks) {
            c->schedule = STA_SCHED_LEVEL;
            return fail(c, STA_EINVAL, "more tiles than co-resident blocks of the tile kernels (" +
                                           std::to_string(max_blocks) + ")");
        }
        try {
            build_tiles(c, B);
        } catch (const CudaFail &f) {
            c->schedule = STA_SCHED_LEVEL;
            free_tiles(c);
            return from_cuda(c, f);
        }
    } else {
        const cudaError_t e = sta::dataflow_prepare(c->hs, c->dc.gamma > 0.f, param);
        if (e != cudaSuccess) {
            c->schedule = STA_SCHED_LEVEL;
            return fail(c, STA_ECUDA, std::string("dataflow set-up: ") + cudaGetErrorString(e));
        }
    }
    return STA_OK;
}

sta_status sta_set_adjoint_schedule(sta_ctx *c, int32_t schedule)
{
    if (!c) return STA_EINVAL;
    if (schedule != STA_SCHED_LEVEL && schedule != STA_SCHED_DATAFLOW)
        return fail(c, STA_EINVAL, "adjoint schedule must be STA_SCHED_LEVEL or STA_SCHED_DATAFLOW");
    c->hs.adj_level = schedule == STA_SCHED_LEVEL;
    c->hs.adj_ready = false;
    return STA_OK;
}

sta_status sta_set_wait_limit(sta_ctx *c, int64_t polls)
{
    if (!c) return STA_EINVAL;
    if (polls < 1) return fail(c, STA_EINVAL, "wait limit must be >= 1 poll");
    try {
        CK(cudaSetDevice(c->device));
        drop_graph(c);
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    c->dc.spin_limit = polls;
    return STA_OK;
}

sta_status sta_debug_hold_cell(sta_ctx *c, int32_t cell)
{
    if (!c) return STA_EINVAL;
    if (cell < -1 || cell >= c->plan.C) return fail(c, STA_EINVAL, "cell index out of range");
    try {
        CK(cudaSetDevice(c->device));
        drop_graph(c);
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    c->dc.hold_item = cell < 0 ? -1 : c->plan.item_of_cell[cell];
    return STA_OK;
}

namespace {
struct TuneKey {
    int device;
    int64_t P, I, S, K, T, E;
    bool uniform, placed, smooth, steiner;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(device, P, I, S, K, T, E, uniform, placed, smooth, steiner) <
               std::tie(o.device, o.P, o.I, o.S, o.K, o.T, o.E, o.uniform, o.placed, o.smooth, o.steiner);
    }
};
struct TuneChoice {
    int schedule, param;
    float ms;
    int adj_schedule;   // reverse sweep of sta_backward (differentiable contexts), -1 = not tuned
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;
}  // namespace

sta_status sta_autotune(sta_ctx *c, void *stream, int32_t trials, int32_t force, int32_t *schedule_out,
                        int32_t *param_out, float *ms_out)
{
    if (!c) return STA_EINVAL;
    if (trials < 1) trials = 1;
    const Plan &pl = c->plan;
    const TuneKey key{c->device, pl.P, pl.I, pl.S, pl.K, pl.T, pl.E, pl.uniform_axes, pl.placed, pl.gamma > 0.f,
                      pl.steiner};
    TuneChoice best{-1, 0, 0.f, -1};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (!force && it != g_tune_cache.end()) best = it->second;
    }
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        if (best.schedule < 0) {
            int sms = 0;
            CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
            std::vector<std::pair<int, int>> cand = {{STA_SCHED_LEVEL, 64}, {STA_SCHED_LEVEL, 128},
                                                     {STA_SCHED_LEVEL, 256}, {STA_SCHED_DATAFLOW, 0},
                                                     {STA_SCHED_DATAFLOW, sms}, {STA_SCHED_DATAFLOW, 2 * sms},
                                                     {STA_SCHED_COOP, 0}, {STA_SCHED_COOP, sms},
                                                     {STA_SCHED_TILE, sms}, {STA_SCHED_TILE, 2 * sms}};
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            for (auto &cs : cand) {
                if (sta_set_schedule(c, cs.first, cs.second) != STA_OK) continue;   // e.g. library too large
                CK(cudaSetDevice(c->device));
                if (sta_update_timing(c, stream) != STA_OK) continue;            // warm-up, captures the graph
                CK(cudaEventRecord(e0, st));
                for (int i = 0; i < trials; ++i) sta_update_timing(c, stream);
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                ms /= trials;
                if (check_device_error(c) != STA_OK) continue;
                if (best.schedule < 0 || ms < best.ms) best = TuneChoice{cs.first, cs.second, ms, -1};
            }
            if (best.schedule < 0) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return fail(c, STA_ECUDA, "no schedule could run");
            }
            // differentiable contexts: the reverse sweep of sta_backward too
            if (pl.gamma > 0.f && pl.placed) {
                float best_adj = 0.f;
                if (sta_set_schedule(c, best.schedule, best.param) != STA_OK || sta_update_timing(c, stream) != STA_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return fail(c, STA_ECUDA, "the chosen schedule failed to run again");
                }
                for (int as : {STA_SCHED_DATAFLOW, STA_SCHED_LEVEL}) {
                    if (sta_set_adjoint_schedule(c, as) != STA_OK) continue;
                    if (sta_backward(c, 1.0, 1.0, nullptr, nullptr, nullptr, STA_DEVICE, stream) != STA_OK) continue;
                    CK(cudaSetDevice(c->device));
                    CK(cudaEventRecord(e0, st));
                    for (int i = 0; i < trials; ++i) sta_backward(c, 1.0, 1.0, nullptr, nullptr, nullptr, STA_DEVICE, stream);
                    CK(cudaEventRecord(e1, st));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    ms /= trials;
                    if (check_device_error(c) != STA_OK) continue;
                    if (best.adj_schedule < 0 || ms < best_adj) {
                        best.adj_schedule = as;
                        best_adj = ms;
                    }
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[key] = best;
        }
        const sta_status st2 = sta_set_schedule(c, best.schedule, best.param);
        if (st2 != STA_OK) return st2;
        if (best.adj_schedule >= 0) {
            const sta_status st4 = sta_set_adjoint_schedule(c, best.adj_schedule);
            if (st4 != STA_OK) return st4;
        }
        const sta_status st3 = sta_update_timing(c, stream);
        if (st3 != STA_OK) return st3;
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    if (schedule_out) *schedule_out = best.schedule;
    if (param_out) *param_out = best.param;
    if (ms_out) *ms_out = best.ms;
    return STA_OK;
}

sta_status sta_update_timing(sta_ctx *c, void *stream)
{
    if (!c) return STA_EINVAL;
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        if (c->stage_pending >= 0) {   // RC values staged by sta_set_rc_async: wait for the copy, reorder
            const int b = c->stage_pending;
            const size_t NN = (size_t)c->plan.NN;
            CK(cudaStreamWaitEvent(st, c->stage_copied[b], 0));
            sta::launch_gather_f32(c->d_stage[b], c->d_rc_src, const_cast<float *>(c->dc.rc_R), (int)NN, st);
            sta::launch_gather_f32(c->d_stage[b] + NN, c->d_rc_src, const_cast<float *>(c->dc.rc_C), (int)NN, st);
            CK(cudaEventRecord(c->stage_free[b], st));
            c->stage_pending = -1;
        }
        if (c->profiling) {
            // eager launches with events at the phase boundaries
            record_pass(c, st, c->ev);
        } else {
            ensure_graph(c);
            CK(cudaGraphLaunch(c->exec, st));
        }
        CK(cudaGetLastError());
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    c->updated = true;
    return STA_OK;
}

sta_status sta_sync(sta_ctx *c, void *stream)
{
    if (!c) return STA_EINVAL;
    try {
        CK(cudaSetDevice(c->device));
        CK(cudaStreamSynchronize(as_stream(stream)));
        CK(cudaGetLastError());
        if (c->profiling && c->updated) {
            for (int i = 0; i < 4; ++i) {
                float ms = 0;
                if (cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]) == cudaSuccess) c->last_ms[i] = ms;
            }
        }
        return check_device_error(c);
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
}

sta_status sta_report_slack_design(sta_ctx *c, int32_t d, void *stream, sta_corner_report *rep)
{
    if (!c || !rep) return STA_EINVAL;
    if (!c->updated) return fail(c, STA_ESTATE, "sta_report_slack before sta_update_timing");
    if (d < 0 || d >= c->plan.n_designs) return fail(c, STA_EINVAL, "design index out of range");
    sta_status st = sta_sync(c, stream);
    if (st != STA_OK) return st;
    const int K = c->plan.Kc;
    std::vector<double> h((size_t)K * 8);
    try {
        CK(cudaMemcpy(h.data(), c->dc.report + (size_t)d * K * 8, h.size() * sizeof(double),
                      cudaMemcpyDeviceToHost));
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    for (int k = 0; k < K; ++k) {
        const double *o = h.data() + (size_t)k * 8;
        rep[k].wns_setup = o[0];
        rep[k].tns_setup = o[1];
        rep[k].wns_hold = o[2];
        rep[k].tns_hold = o[3];
        rep[k].worst_setup = o[4];
        rep[k].worst_hold = o[5];
        rep[k].n_viol_setup = (int64_t)o[6];
        rep[k].n_viol_hold = (int64_t)o[7];
    }
    return STA_OK;
}

sta_status sta_report_slack(sta_ctx *c, void *stream, sta_corner_report *rep)
{
    return sta_report_slack_design(c, 0, stream, rep);
}

sta_status sta_get_pin_state(sta_ctx *c, int32_t which, float *out, sta_mem mem, void *stream)
{
    if (!c || !out) return STA_EINVAL;
    if (!c->updated) return fail(c, STA_ESTATE, "no analysis yet");
    const sta::DF4 *srcd = which == STA_AT ? c->dc.at : which == STA_RAT ? c->dc.rat : nullptr;
    const float4 *src = which == STA_SLEW ? c->dc.slew : which == STA_SLACK ? c->dc.slack : nullptr;
    if (!src && !srcd) return fail(c, STA_EINVAL, "unknown array id");
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        const size_t PK = (size_t)c->plan.P * c->plan.K;
        auto gather = [&](float4 *dst) {
            if (srcd) sta::launch_gather_pins_d(srcd, c->d_gpu_of, dst, c->plan.P, c->plan.K, st);
            else sta::launch_gather_pins(src, c->d_gpu_of, dst, c->plan.P, c->plan.K, st);
        };
        if (mem == STA_DEVICE) {
            gather(reinterpret_cast<float4 *>(out));
            CK(cudaGetLastError());
        } else {
            if (!c->d_gather_tmp) c->d_gather_tmp = dev_alloc<float4>(c, PK);
            gather(c->d_gather_tmp);
            CK(cudaMemcpyAsync(out, c->d_gather_tmp, PK * sizeof(float4), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

sta_status sta_get_endpoint_slack(sta_ctx *c, float *setup, float *hold, uint8_t *vs, uint8_t *vh, sta_mem mem,
                                  void *stream)
{
    if (!c) return STA_EINVAL;
    if (!c->updated) return fail(c, STA_ESTATE, "no analysis yet");
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        const size_t EK = (size_t)c->plan.E * c->plan.Kc;
        const cudaMemcpyKind kind = mem == STA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const float *es = c->dc.ep_setup, *eh = c->dc.ep_hold;
        const uint8_t *evs = c->dc.viol_setup, *evh = c->dc.viol_hold;
        if (c->plan.Tg > 1) {   // per corner: min over the exception tags
            if (!c->d_ep_collapse) {
                c->d_ep_collapse = dev_alloc<float>(c, 2 * std::max<size_t>(1, EK));
                c->d_viol_collapse = dev_alloc<uint8_t>(c, 2 * std::max<size_t>(1, EK));
            }
            sta::launch_collapse_tags(c->dc, c->d_ep_collapse, c->d_viol_collapse, st);
            es = c->d_ep_collapse;
            eh = c->d_ep_collapse + EK;
            evs = c->d_viol_collapse;
            evh = c->d_viol_collapse + EK;
        }
        if (setup) CK(cudaMemcpyAsync(setup, es, EK * sizeof(float), kind, st));
        if (hold) CK(cudaMemcpyAsync(hold, eh, EK * sizeof(float), kind, st));
        if (vs) CK(cudaMemcpyAsync(vs, evs, EK, kind, st));
        if (vh) CK(cudaMemcpyAsync(vh, evh, EK, kind, st));
        if (mem == STA_HOST) CK(cudaStreamSynchronize(st));
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

static sta_status report_paths_impl(sta_ctx *c, int32_t design, int32_t corner, int32_t k, int32_t per_ep,
                                    float slack_lt, int32_t *n_paths, int32_t *n_pins, int32_t *path_ptr,
                                    int32_t *path_pin, int8_t *path_rf, float *path_at, float *path_slack,
                                    int32_t *path_endpoint, int32_t pin_capacity, sta_mem mem, void *stream)
{
    if (!c || !n_paths || !n_pins) return STA_EINVAL;
    if (!c->updated) return fail(c, STA_ESTATE, "no analysis yet");
    const Plan &pl = c->plan;
    if (design < 0 || design >= pl.n_designs) return fail(c, STA_EINVAL, "design index out of range");
    if (corner < 0 || corner >= pl.Kc) return fail(c, STA_EINVAL, "corner index out of range");
    if (k < 0 || k > sta::kMaxPaths) return fail(c, STA_EINVAL, "k must be in 0..4096");
    if (std::isnan(slack_lt)) return fail(c, STA_EINVAL, "slack threshold is NaN");
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        sta::PathJob &j = c->pj;
        if (!j.sel) {
            // item of every item pin, caller id of every internal pin
            std::vector<int32_t> pin_item(pl.P, -1), caller(pl.P, 0);
            for (int32_t g = 0; g < pl.I; ++g) {
                const int32_t t = pl.item_type[g], p0 = pl.item_pin0[g];
                const int32_t np = t < 0 ? 1 : (pl.type_kind[t] == 1 ? 2 : pl.type_nin[t] + 1);
                for (int32_t i = 0; i < np; ++i) pin_item[p0 + i] = g;
            }
            for (int32_t p = 0; p < pl.P; ++p) caller[pl.gpu_of[p]] = p;
            j.pin_item = upload(c, pin_item);
            j.caller_pin = upload(c, caller);
            j.max_len = 2 * pl.S + 3;
            c->path_cap = sta::kMaxPaths * j.max_len;
            j.sel = dev_alloc<unsigned long long>(c, 3);
            j.hist = dev_alloc<unsigned>(c, 256);
            j.count = dev_alloc<unsigned>(c, 1);
            j.keys = dev_alloc<unsigned long long>(c, sta::kMaxPaths);
            j.ptr = dev_alloc<int32_t>(c, sta::kMaxPaths + 1);
            j.pin = dev_alloc<int32_t>(c, (size_t)c->path_cap);
            j.rf = dev_alloc<int8_t>(c, (size_t)c->path_cap);
            j.at = dev_alloc<float>(c, (size_t)c->path_cap);
            j.slack = dev_alloc<float>(c, sta::kMaxPaths);
            j.endpoint = dev_alloc<int32_t>(c, sta::kMaxPaths);
        }
        if (per_ep > 1 && !j.recs) {
            j.recs = dev_alloc<sta::PathRec>(c, sta::kMaxNworst);
            j.pkeys = dev_alloc<unsigned long long>(c, sta::kMaxNworst);
        }
        j.per_ep = per_ep;
        j.e0 = pl.ep_design_ptr[design];
        j.n = pl.ep_design_ptr[design + 1] - j.e0;
        j.corner = corner;
        j.k = k;
        j.slack_lt = slack_lt;
        const unsigned long long sel0[3] = {0ull, (unsigned long long)k, 0ull};
        CK(cudaMemcpyAsync(j.sel, sel0, sizeof(sel0), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(j.hist, 0, 256 * sizeof(unsigned), st));
        CK(cudaMemsetAsync(j.count, 0, sizeof(unsigned), st));
        CK(cudaMemsetAsync(j.ptr, 0, sizeof(int32_t), st));
        if (k > 0 && per_ep > 1) sta::launch_report_paths_nworst(c->dc, c->hs, j, st);
        else if (k > 0) sta::launch_report_paths(c->dc, c->hs, j, st);
        CK(cudaGetLastError());
        unsigned cnt = 0;
        CK(cudaMemcpyAsync(&cnt, j.count, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (k == 0) cnt = 0;
        int32_t total = 0;
        if (cnt > 0) CK(cudaMemcpy(&total, j.ptr + cnt, sizeof(int32_t), cudaMemcpyDeviceToHost));
        *n_paths = (int32_t)cnt;
        *n_pins = total;
        if (total > pin_capacity && (path_pin || path_rf || path_at))
            return fail(c, STA_EINVAL, "pin arrays too small for the report (n_pins holds the size needed)");
        const cudaMemcpyKind kind = mem == STA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (path_ptr) CK(cudaMemcpyAsync(path_ptr, j.ptr, (cnt + 1) * sizeof(int32_t), kind, st));
        if (path_pin && total) CK(cudaMemcpyAsync(path_pin, j.pin, total * sizeof(int32_t), kind, st));
        if (path_rf && total) CK(cudaMemcpyAsync(path_rf, j.rf, total * sizeof(int8_t), kind, st));
        if (path_at && total) CK(cudaMemcpyAsync(path_at, j.at, total * sizeof(float), kind, st));
        if (path_slack && cnt) CK(cudaMemcpyAsync(path_slack, j.slack, cnt * sizeof(float), kind, st));
        if (path_endpoint && cnt) CK(cudaMemcpyAsync(path_endpoint, j.endpoint, cnt * sizeof(int32_t), kind, st));
        CK(cudaStreamSynchronize(st));
        const sta_status se = check_device_error(c);
        if (se != STA_OK) return se;
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

sta_status sta_report_paths(sta_ctx *c, int32_t design, int32_t corner, int32_t k, float slack_lt, int32_t *n_paths,
                            int32_t *n_pins, int32_t *path_ptr, int32_t *path_pin, int8_t *path_rf, float *path_at,
                            float *path_slack, int32_t *path_endpoint, int32_t pin_capacity, sta_mem mem,
                            void *stream)
{
    return report_paths_impl(c, design, corner, k, 1, slack_lt, n_paths, n_pins, path_ptr, path_pin, path_rf, path_at,
                             path_slack, path_endpoint, pin_capacity, mem, stream);
}

sta_status sta_report_paths_nworst(sta_ctx *c, int32_t design, int32_t corner, int32_t k, int32_t per_endpoint,
                                   float slack_lt, int32_t *n_paths, int32_t *n_pins, int32_t *path_ptr,
                                   int32_t *path_pin, int8_t *path_rf, float *path_at, float *path_slack,
                                   int32_t *path_endpoint, int32_t pin_capacity, sta_mem mem, void *stream)
{
    if (!c) return STA_EINVAL;
    if (per_endpoint < 1 || per_endpoint > sta::kMaxPerEndpoint)
        return fail(c, STA_EINVAL, "per_endpoint must be in 1..32");
    if (per_endpoint > 1 && (int64_t)k * per_endpoint > sta::kMaxNworst)
        return fail(c, STA_EINVAL, "k * per_endpoint must be at most 16384");
    if (per_endpoint > 1 && c->plan.Tg > 1)
        return fail(c, STA_EINVAL, "a per-endpoint limit above 1 needs a design without timing exceptions");
    return report_paths_impl(c, design, corner, k, per_endpoint, slack_lt, n_paths, n_pins, path_ptr, path_pin,
                             path_rf, path_at, path_slack, path_endpoint, pin_capacity, mem, stream);
}

sta_status sta_set_rc(sta_ctx *c, const float *R, const float *Cc, sta_mem mem)
{
    if (!c || !R || !Cc) return STA_EINVAL;
    if (c->plan.placed) return fail(c, STA_ESTATE, "context uses positions, not RC trees");
    const size_t NN = (size_t)c->plan.NN;
    try {
        CK(cudaSetDevice(c->device));
        if (!c->d_rc_tmp) c->d_rc_tmp = dev_alloc<float>(c, NN);
        const cudaMemcpyKind kind = mem == STA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CK(cudaMemcpy(c->d_rc_tmp, R, NN * sizeof(float), kind));
        sta::launch_gather_f32(c->d_rc_tmp, c->d_rc_src, const_cast<float *>(c->dc.rc_R), (int)NN, 0);
        CK(cudaMemcpy(c->d_rc_tmp, Cc, NN * sizeof(float), kind));
        sta::launch_gather_f32(c->d_rc_tmp, c->d_rc_src, const_cast<float *>(c->dc.rc_C), (int)NN, 0);
        CK(cudaDeviceSynchronize());
        c->stage_pending = -1;   // these values replace any staged ones
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

sta_status sta_set_rc_async(sta_ctx *c, const float *R, const float *Cc, sta_mem mem, void *stream)
{
    if (!c || !R || !Cc) return STA_EINVAL;
    if (c->plan.placed) return fail(c, STA_ESTATE, "context uses positions, not RC trees");
    const size_t NN = (size_t)c->plan.NN;
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        if (!c->d_stage[0]) {
            for (int b = 0; b < 2; ++b) {
                c->d_stage[b] = dev_alloc<float>(c, 2 * std::max<size_t>(1, NN));
                CK(cudaEventCreateWithFlags(&c->stage_copied[b], cudaEventDisableTiming));
                CK(cudaEventCreateWithFlags(&c->stage_free[b], cudaEventDisableTiming));
                CK(cudaEventRecord(c->stage_free[b], st));
            }
        }
        // a buffer staged but not applied yet is replaced: reuse it
        const int b = c->stage_pending >= 0 ? c->stage_pending : c->stage_next;
        CK(cudaStreamWaitEvent(st, c->stage_free[b], 0));   // its last reorder has read it
        const cudaMemcpyKind kind = mem == STA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CK(cudaMemcpyAsync(c->d_stage[b], R, NN * sizeof(float), kind, st));
        CK(cudaMemcpyAsync(c->d_stage[b] + NN, Cc, NN * sizeof(float), kind, st));
        CK(cudaEventRecord(c->stage_copied[b], st));
        c->stage_pending = b;
        c->stage_next = b ^ 1;
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

sta_status sta_set_positions(sta_ctx *c, const float *cell_xy, sta_mem mem, void *stream)
{
    if (!c || !cell_xy) return STA_EINVAL;
    if (!c->plan.placed) return fail(c, STA_ESTATE, "context uses RC trees, not positions");
    try {
        CK(cudaSetDevice(c->device));
        const cudaMemcpyKind kind = mem == STA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CK(cudaMemcpyAsync(const_cast<float *>(c->dc.cell_xy), cell_xy, 2 * (size_t)c->plan.C * sizeof(float), kind,
                           as_stream(stream)));
        if (mem == STA_HOST) CK(cudaStreamSynchronize(as_stream(stream)));
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

sta_status sta_get_net_wirelength(sta_ctx *c, int64_t *wl_nm, sta_mem mem, void *stream)
{
    if (!c || !wl_nm) return STA_EINVAL;
    if (!c->plan.steiner) return fail(c, STA_ESTATE, "context does not build Steiner trees");
    if (!c->updated) return fail(c, STA_ESTATE, "sta_get_net_wirelength before sta_update_timing");
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        const int32_t N = c->plan.n_nets;
        if (N == 0) return STA_OK;
        if (mem == STA_DEVICE) {
            sta::launch_gather_i64(c->dc.st_wl, c->d_item_of_net, wl_nm, N, st);
        } else {
            if (!c->d_wl_tmp) c->d_wl_tmp = dev_alloc<int64_t>(c, N);
            sta::launch_gather_i64(c->dc.st_wl, c->d_item_of_net, c->d_wl_tmp, N, st);
            CK(cudaMemcpyAsync(wl_nm, c->d_wl_tmp, (size_t)N * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
        CK(cudaGetLastError());
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

sta_status sta_set_cell_types(sta_ctx *c, const int32_t *cell_type)
{
    if (!c || !cell_type) return STA_EINVAL;
    Plan &pl = c->plan;
    for (int32_t i = 0; i < pl.C; ++i) {
        const int32_t t = cell_type[i], o = pl.cell_type[i];
        if (t < 0 || t >= pl.T) return fail(c, STA_EINVAL, "cell type out of range");
        if (pl.type_nin[t] != pl.type_nin[o] || pl.type_kind[t] != pl.type_kind[o])
            return fail(c, STA_EINVAL, "resizing must keep the input count and kind");
    }
    for (int32_t i = 0; i < pl.C; ++i) {
        pl.cell_type[i] = cell_type[i];
        pl.item_type[pl.item_of_cell[i]] = cell_type[i];
    }
    for (int64_t q = 0; q < pl.F; ++q) {
        const int32_t s = pl.fo_src[q];
        const int32_t cc = c->pin_cell_c[s];
        if (cc >= 0) pl.fo_cap[q] = pl.type_pin_cap[(size_t)pl.cell_type[cc] * 4 + c->pin_slot_c[s]];
    }
    try {
        CK(cudaSetDevice(c->device));
        CK(cudaMemcpy(const_cast<int32_t *>(c->dc.item_type), pl.item_type.data(), pl.item_type.size() * 4,
                      cudaMemcpyHostToDevice));
        if (pl.F)
            CK(cudaMemcpy(const_cast<float *>(c->dc.fo_cap), pl.fo_cap.data(), pl.fo_cap.size() * 4,
                          cudaMemcpyHostToDevice));
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

sta_status sta_resize_cells(sta_ctx *c, const int32_t *cells, const int32_t *types, int32_t n, sta_mem mem,
                            void *stream)
{
    if (!c) return STA_EINVAL;
    if (n < 0 || (n > 0 && (!cells || !types))) return fail(c, STA_EINVAL, "bad resize arguments");
    if (n == 0) return STA_OK;
    Plan &pl = c->plan;
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        if (!c->d_item_of_cell) {
            c->d_item_of_cell = upload(c, pl.item_of_cell);
            std::vector<int32_t> fo_of_pin(pl.P, -1), dpin(pl.C, -1);
            for (int64_t q = 0; q < pl.F; ++q) fo_of_pin[pl.fo_pin[q]] = (int32_t)q;
            for (size_t p = 0; p < c->pin_cell_c.size(); ++p) {
                const int32_t cc = c->pin_cell_c[p];
                if (cc >= 0 && c->pin_slot_c[p] == 0 && pl.type_kind[pl.cell_type[cc]] == 1) dpin[cc] = pl.gpu_of[p];
            }
            c->d_fo_of_pin = upload(c, fo_of_pin);
            c->d_d_pin_of_cell = upload(c, dpin);
            c->d_type_pin_cap = upload(c, pl.type_pin_cap);
        }
        const int32_t *dc = cells, *dt = types;
        if (mem == STA_HOST) {
            if (n > c->resize_cap) {
                c->d_resize_tmp = dev_alloc<int32_t>(c, 2 * (size_t)n);
                c->resize_cap = n;
            }
            CK(cudaMemcpyAsync(c->d_resize_tmp, cells, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(c->d_resize_tmp + n, types, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            dc = c->d_resize_tmp;
            dt = c->d_resize_tmp + n;
        }
        sta::launch_resize(c->dc, c->d_item_of_cell, c->d_d_pin_of_cell, c->d_fo_of_pin, c->d_type_pin_cap, dc, dt,
                           n, const_cast<int32_t *>(c->dc.item_type), st);
        CK(cudaGetLastError());
        if (mem == STA_HOST) CK(cudaStreamSynchronize(st));
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

sta_status sta_get_arrays(sta_ctx *c, sta_views *out)
{
    if (!c || !out) return STA_EINVAL;
    out->at = reinterpret_cast<const float *>(c->dc.at);
    out->slew = reinterpret_cast<const float *>(c->dc.slew);
    out->rat = reinterpret_cast<const float *>(c->dc.rat);
    out->slack = reinterpret_cast<const float *>(c->dc.slack);
    out->gpu_pin_of = c->d_gpu_of;
    return STA_OK;
}

sta_status sta_stats(const sta_ctx *c, sta_plan_info *out)
{
    if (!c || !out) return STA_EINVAL;
    const Plan &pl = c->plan;
    std::memset(out, 0, sizeof(*out));
    out->n_pins = pl.P;
    out->n_cells = pl.C;
    // every caller net (as sta_plan; sta_get_net_wirelength writes one value
    // per net), sinkless ones included
    out->n_nets = pl.n_nets;
    int64_t nets_with_sinks = 0;
    for (int32_t g = 0; g < pl.I; ++g) nets_with_sinks += pl.fo_ptr[g + 1] > pl.fo_ptr[g];
    out->n_items = pl.I;
    out->n_cell_arcs = pl.cell_arcs;
    out->n_net_arcs = pl.F;
    out->n_rc_nodes = pl.placed ? pl.F + nets_with_sinks : pl.NN;
    out->n_endpoints = pl.E;
    out->n_levels = pl.S;
    out->n_corners = pl.Kc;
    out->n_tags = pl.Tg;
    out->max_level_width = pl.max_width;
    out->n_designs = pl.n_designs;
    out->device_bytes = (int64_t)c->bytes;
    out->launches_per_update = launches_per_update(c);
    out->launches_per_backward = launches_per_backward(c);
    return STA_OK;
}

sta_status sta_set_profiling(sta_ctx *c, int32_t on)
{
    if (!c) return STA_EINVAL;
    c->profiling = on != 0;
    return STA_OK;
}

sta_status sta_last_timings(sta_ctx *c, float *ms4)
{
    if (!c || !ms4) return STA_EINVAL;
    for (int i = 0; i < 4; ++i) ms4[i] = c->last_ms[i];
    return STA_OK;
}

sta_status sta_backward(sta_ctx *c, double w_tns, double w_wns, double *J_out, double *terms, double *grad_xy,
                        sta_mem mem, void *stream)
{
    if (!c) return STA_EINVAL;
    if (!c->updated) return fail(c, STA_ESTATE, "sta_backward before sta_update_timing");
    if (!(c->plan.gamma > 0.f) || !c->plan.placed)
        return fail(c, STA_ESTATE, "sta_backward needs a differentiable context (gamma_ns > 0, positions)");
    if (!std::isfinite(w_tns) || !std::isfinite(w_wns)) return fail(c, STA_EINVAL, "weights must be finite");
    if (c->plan.steiner && c->plan.net_model != STA_NET_ELMORE)
        return fail(c, STA_ESTATE, "sta_backward on Steiner trees needs the Elmore net model");
    try {
        CK(cudaSetDevice(c->device));
        cudaStream_t st = as_stream(stream);
        DevCtx &d = c->dc;
        const int K = c->plan.K;
        if (!d.adj) {
            d.adj = dev_alloc<float4>(c, (size_t)c->plan.P * K);
            d.obj = dev_alloc<double>(c, 4 * (size_t)K + 1);
            d.grad = dev_alloc<double>(c, 2 * (size_t)c->plan.C);
            d.aload = dev_alloc<float>(c, (size_t)c->plan.I * K);
            if (!c->plan.steiner) {   // the star segments' kernel runs one thread per fan-out entry
                std::vector<int32_t> fo_item(c->plan.F);
                for (int32_t g = 0; g < c->plan.I; ++g)
                    for (int64_t p = c->plan.fo_ptr[g]; p < c->plan.fo_ptr[g + 1]; ++p) fo_item[p] = g;
                d.fo_item = upload(c, fo_item);
            }
            d.abox_len = 2 * (size_t)c->plan.P * K;
            d.abox = dev_alloc<float4>(c, d.abox_len);
            CK(cudaMemset(d.abox, 0xFF, std::max<size_t>(1, d.abox_len) * sizeof(float4)));
            if (c->plan.steiner) {   // node storage for trees too large for the shared-memory column
                int64_t big = 0;
                for (int32_t g = 0; g < c->plan.I; ++g)
                    big = std::max<int64_t>(big, c->plan.rc_ptr[g + 1] - c->plan.rc_ptr[g]);
                if (big >= sta::kAdjBigColNodes) d.st_abuf = dev_alloc<float>(c, sta::steiner_adjoint_floats(c->plan.NN));
            }
        }
        if (!c->hs.adj_ready) {
            const cudaError_t e = sta::adjoint_prepare(c->hs);
            if (e != cudaSuccess) throw CudaFail{e, "adjoint set-up"};
            c->hs.adj_ready = true;
        }
        d.w_tns = w_tns;
        d.w_wns = w_wns;
        sta::launch_adjoint(d, c->hs, st);
        CK(cudaGetLastError());
        const cudaMemcpyKind kind = mem == STA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (J_out) CK(cudaMemcpyAsync(J_out, d.obj + 4 * K, sizeof(double), kind, st));
        if (terms)
            CK(cudaMemcpy2DAsync(terms, 2 * sizeof(double), d.obj + 2, 4 * sizeof(double), 2 * sizeof(double), K,
                                 kind, st));
        if (grad_xy && c->plan.C > 0)
            CK(cudaMemcpyAsync(grad_xy, d.grad, 2 * (size_t)c->plan.C * sizeof(double), kind, st));
        if (mem == STA_HOST) {
            CK(cudaStreamSynchronize(st));
            return check_device_error(c);
        }
    } catch (const CudaFail &f) {
        return from_cuda(c, f);
    }
    return STA_OK;
}

}  // extern "C"
