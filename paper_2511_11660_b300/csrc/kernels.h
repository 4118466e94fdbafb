// kernels.h -- host entry points of the device passes.
#pragma once

#include <algorithm>
#include <vector>

#include "device.cuh"

namespace sta {

// Host-side description of the launch sequence.
struct HostSched {
    int S = 0;
    std::vector<int32_t> stage_ptr;   // host copy of the level offsets
    bool rc = false;                  // RC trees to sweep (tree mode with nodes)
    bool placed = false;
    bool steiner = false;             // Steiner trees built from positions before the RC sweep
    bool thru = false;                // -through exception sets (the dataflow kernels' variant)
    int threads = 128;                // threads per block of the level kernels
    int n_red_chunks = 0;             // first-stage reduction blocks
    bool uniform = false;             // every table shares the same slew and load axes
    int T = 0;                        // cell types (shared-memory table size)
    int df_blocks_fwd = 0;            // persistent grids of the dataflow kernels
    int df_blocks_bwd = 0;
    int adj_blocks = 0;               // persistent grid of the dataflow adjoint (0 = level sweep)
    bool adj_level = false;           // reverse sweep forced to one launch per level
    bool adj_ready = false;           // adjoint_prepare has run for the current choice
    bool one = false;                 // one state a pin, one corner a lane group: the DevCtxOne kernels
    int coop_blocks = 0;              // co-resident grid of the cooperative schedule
    int tile_blocks = 0;              // tiles (co-resident blocks) of the tile schedule
};

// Net delays, forward levels, endpoints, backward levels, reduction.  With
// `ev` (5 events) the phase boundaries are recorded: ev[0] start, ev[1] after
// net delays, ev[2] after forward + endpoints, ev[3] after backward, ev[4]
// after the reduction.
void launch_level_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev = nullptr);

// Net delay calculation: RC trees (one thread per net) or star trees.
void launch_net_tree(const DevCtx &c, cudaStream_t st);
// Every endpoint at once, after a forward pass (the level and dataflow schedules).
void launch_endpoints(const DevCtx &c, cudaStream_t st);
void launch_net_star(const DevCtx &c, cudaStream_t st);
// Steiner trees from positions (steiner.cu): writes the RC arrays the tree sweep reads.
void launch_net_steiner(const DevCtx &c, cudaStream_t st);
// The net phase of a pass: Steiner trees + RC sweep, star trees, or RC sweep.
void launch_net_phase(const DevCtx &c, const HostSched &h, cudaStream_t st);
// out[i] = src[idx[i]] (int64), n entries
void launch_gather_i64(const int64_t *src, const int32_t *idx, int64_t *out, int n, cudaStream_t st);

// Dataflow schedule: one persistent kernel per pass (see dataflow.cu).
// dataflow_prepare sizes the persistent grids (at most `requested` blocks
// when > 0, else every block the occupancy allows) and must run before the
// first launch and outside stream capture.
size_t dataflow_smem_bytes(int T);
cudaError_t dataflow_prepare(HostSched &h, bool smooth, int requested);
void launch_dataflow_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev = nullptr);

// Cooperative schedule: one co-resident launch runs every forward level,
// the endpoints and every backward level, with a grid-wide barrier between
// levels (see dataflow.cu).  coop_prepare sizes the grid (at most `requested`
// blocks when > 0) outside stream capture.
cudaError_t coop_prepare(HostSched &h, bool smooth, int requested);
void launch_coop_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev = nullptr);

// Tile schedule (tile.cu): one co-resident launch per pass, each block
// walking its own tile of the partition (tile.cpp) step by step.
// tile_prepare gives the largest co-resident grid of the tile kernels
// (outside stream capture); the DevCtx tl_* arrays must hold a partition
// for c.tl_B <= that many tiles.
int tile_threads();
int tile_ring_slots(int KL);
int tile_max_steps();
cudaError_t tile_prepare(HostSched &h, bool smooth, int NS, int *max_blocks);
void launch_tile_pass(const DevCtx &c, const HostSched &h, cudaStream_t st, cudaEvent_t *ev = nullptr);
// Mailbox recovery after an aborted pass and a new epoch (dataflow and tile
// schedules), on a grid of `blocks` blocks.
void launch_df_reset(const DevCtx &c, int blocks, cudaStream_t st);

// Smoothed objective and its reverse sweep to cell positions (adjoint.cu):
// a persistent dataflow sweep when adjoint_prepare gave it a grid
// (h.adj_blocks > 0), else one launch per level.
void launch_adjoint(const DevCtx &c, const HostSched &h, cudaStream_t st);
size_t adjoint_smem_bytes(int T);
cudaError_t adjoint_prepare(HostSched &h);
// Steiner contexts: the adjoint of a net's tree works in a shared-memory
// column of kAdjColNodes nodes (nets of at most kAdjSmallPins pins) or
// kAdjBigColNodes nodes (larger nets, at most 64 pins); trees beyond that
// keep their node arrays in a device buffer of steiner_adjoint_floats(NN)
// floats, needed when some net has room for kAdjBigColNodes nodes or more.
constexpr int kAdjColNodes = 16, kAdjSmallPins = 9, kAdjBigColNodes = 128;
constexpr int kAdjTinyColNodes = 8, kAdjTinyPins = 5;   // nets of <= 5 pins: <= 8 tree nodes
size_t steiner_adjoint_floats(int64_t NN);

// The two-stage FP64 WNS/TNS reduction.
void launch_reduce(const DevCtx &c, const HostSched &h, cudaStream_t st);

// Top-k path report of one design (paths.cu): selection of the k worst
// endpoints below a slack threshold and the trace of their critical paths.
constexpr int kMaxPaths = 4096;   // paths one report returns at most
// One path at an endpoint: its end edge and deviations from the critical
// fan-in, as a chain of records (parent = the same path without its last,
// highest deviation).
struct PathRec {
    float cost;                   // the path's setup slack
    float dv;                     // its last deviation's cost (0 at a root)
    int parent;                   // record of the parent path, -1 at a root
    int p, a;                     // deviation: gate output p at edge rf takes input a at edge rfi
    int rf, rfi;                  // (root: p = the endpoint, rf = the end edge)
    int pos, alt;                 // place of the deviation in its parent's region order
};
struct PathJob {
    int e0, n;                    // the design's endpoints [e0, e0 + n)
    int corner, k, max_len;       // max_len: pins a path can hold
    float slack_lt;
    const int32_t *pin_item;      // [P] item of an item pin, -1 for endpoint pins
    const int32_t *caller_pin;    // [P] internal pin -> caller pin id
    unsigned long long *sel;      // [3] selection state: key prefix, remaining rank
    unsigned *hist;               // [256] digit histogram (zero between passes)
    unsigned *count;              // keys selected
    unsigned long long *keys;     // [kMaxPaths] selected keys, sorted
    int32_t *ptr;                 // [kMaxPaths + 1] CSR offsets
    int32_t *pin;                 // [kMaxPaths * max_len] caller pin ids
    int8_t *rf;                   // edges
    float *at;                    // late arrivals
    float *slack;                 // [kMaxPaths] setup slack of each path
    int32_t *endpoint;            // [kMaxPaths] caller pin id of each endpoint
    // per-endpoint limit above 1 (sta_report_paths_nworst)
    int per_ep;                   // paths per endpoint at most
    PathRec *recs;                // [kMaxNworst] paths found, per_ep slots per selected endpoint
    unsigned long long *pkeys;    // [kMaxNworst] (slack, endpoint order, rank) keys, then sorted
};
constexpr int kMaxPerEndpoint = 32, kMaxNworst = 16384;   // per_ep, k * per_ep
void launch_report_paths_nworst(const DevCtx &c, const HostSched &h, const PathJob &j, cudaStream_t st);
void launch_report_paths(const DevCtx &c, const HostSched &h, const PathJob &j, cudaStream_t st);

// Device-side resizing (sta_resize_cells).
void launch_resize(const DevCtx &c, const int32_t *item_of_cell, const int32_t *d_pin_of_cell,
                   const int32_t *fo_of_pin, const float *type_pin_cap, const int32_t *cells, const int32_t *types,
                   int n, int32_t *item_type, cudaStream_t st);

void launch_gather_pins(const float4 *arr, const int32_t *gpu_of, float4 *out, int P, int K, cudaStream_t st);
void launch_gather_pins_d(const DF4 *arr, const int32_t *gpu_of, float4 *out, int P, int K, cudaStream_t st);
// Endpoint slacks and violation flags per corner, min over the exception
// tags: ep[0 .. E*Kc) setup, ep[E*Kc ..) hold; viol likewise.
void launch_collapse_tags(const DevCtx &c, float *ep, uint8_t *viol, cudaStream_t st);
void launch_gather_f32(const float *src, const int32_t *idx, float *dst, int n, cudaStream_t st);

}  // namespace sta
