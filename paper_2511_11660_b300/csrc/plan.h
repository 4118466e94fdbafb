// plan.h -- host-side validation, levelisation and device layout of a design.
//
// The netlist arrives as flattened CSR (cells -> pins, nets -> pins), the
// form HeteroSTA accepts from a host flow (Sec. III, "Heterogeneous netlist
// database").  Graph propagation (Sec. I) needs a dependency order; this
// file computes one by Kahn's algorithm over "items" (a primary input or a
// cell with its input pins and output pin) and lays every per-pin array out
// level-major so that one level's writes are contiguous.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "sta.h"

namespace sta {

constexpr int kNldm = 7;          // 7x7 NLDM tables
constexpr int kMaxSlot = 3;       // at most three inputs per cell
constexpr int kTabStride = 80;    // floats per packed table (see packLut)
constexpr int kColNodes = 10;     // RC nets up to this many nodes are swept in shared memory
constexpr int kSteinerMaxPins = 64;  // nets of more pins keep the rectilinear MST (no Steiner points)
constexpr int kSteinerSmallPins = 8; // nets of at most this many pins are built in shared memory

enum { kPinPI = 0, kPinPO = 1, kPinIN = 2, kPinOUT = 3, kPinD = 4, kPinCK = 5, kPinQ = 6 };
enum { kSenseNone = -1, kSensePos = 0, kSenseNeg = 1, kSenseNon = 2, kSenseRise = 3 };

struct Plan {
    // sizes
    int32_t P = 0, I = 0, S = 0, E = 0, K = 1, T = 0, C = 0;
    int64_t NN = 0;                // RC nodes
    int64_t F = 0;                 // net sinks (= net arcs)
    int64_t cell_arcs = 0;
    int32_t max_width = 0;
    int32_t n_designs = 1;
    bool placed = false;
    bool steiner = false;                    // positions mode with Steiner trees (STA_WIRE_STEINER)
    float r_per_um_y = 0.f, c_per_um_y = 0.f; // Steiner: unit R/C along y (the x values when <= 0 on input)
    std::vector<int64_t> st_node_ptr;        // [I + 1] Steiner working nodes per item: 3 n (n = sinks + 1), 0 without sinks
    std::vector<int64_t> st_adj_ptr;         // [I + 1] adjacency bitset words per item: 3 n x ceil(3 n / 32) (n <= 64)
    std::vector<int32_t> net_of_item;        // [I] caller net driven by the item, -1 if none
    std::vector<int32_t> st_items;           // items with sinks by increasing sink count (a warp's nets alike)
    int32_t st_small = 0;                    // how many of them have at most kSteinerSmallPins pins
    int32_t n_nets = 0;
    float gamma = 0.f;
    int32_t net_model = STA_NET_ELMORE;      // net delay calculator
    int32_t Kc = 1, Tg = 1;                  // corners and exception tags; K = Kc * Tg states
    std::vector<int32_t> item_tag;           // [I] exception tag of a startpoint item (PI, flip-flop), else 0
    std::vector<float> ep_mult;              // [E][Tg] setup multiplier of each endpoint and tag, 0 = no check
    std::vector<float> ep_off;               // [E][Tg][2] late requirement offset and early requirement (ns)
    std::vector<uint32_t> pin_adv;           // [P] bit t: tag t moves on to t + 1 at this gate input (empty: no -through)
    int32_t arnoldi_q = 3;                   // order of STA_NET_ARNOLDI
    // constraints
    float period = 1.f, clk_slew = 0.02f, pi_at = 0.f, pi_slew = 0.02f;
    float setup = 0.f, hold = 0.f, po_cap = 0.f;
    float r_per_um = 0.f, c_per_um = 0.f;
    std::vector<float> lut_scale, rc_scale;
    // library (packed tables: idx1[7] idx2[7] inv1[6] inv2[6] val[49] pad)
    std::vector<float> lut;                  // [T][3][4][80]
    std::vector<int32_t> type_nin, type_kind, arc_sense;
    std::vector<float> type_pin_cap;         // [T][4]
    // items (level-major)
    std::vector<int32_t> stage_ptr;          // [S+1]
    std::vector<int32_t> item_pin0;          // [I]
    std::vector<int32_t> item_type;          // [I] cell type, -1 = primary input
    std::vector<int32_t> item_cell;          // [I] caller cell id, -1 = primary input
    std::vector<int32_t> fo_ptr;             // [I+1] sinks of the item's output net
    std::vector<int32_t> fo_pin;             // [F]   internal sink pin
    std::vector<int32_t> fo_node;            // [F]   local RC node of the sink
    std::vector<float> fo_cap;               // [F]   sink pin capacitance, pF
    std::vector<int32_t> fo_src;             // [F]   caller pin id of the sink (for set_cell_types)
    // RC trees, nets in item order (items without a net own no nodes)
    std::vector<int32_t> rc_ptr;             // [I+1]
    std::vector<int32_t> rc_parent;          // [NN] local parent
    std::vector<float> rc_R, rc_C;           // [NN]
    std::vector<int64_t> rc_src;             // [NN] caller node index
    int32_t n_big_nets = 0;                  // RC nets of more than kColNodes nodes (swept in global scratch)
    // pins
    std::vector<int32_t> drv_of;             // [P] internal driver of a sink pin, -1
    std::vector<int32_t> gpu_of;             // [P] caller pin -> internal pin
    std::vector<int32_t> pin_cell;           // [P] internal pin -> caller cell, or -(port+1)
    std::vector<float> port_xy;              // [n_ports*2]
    std::vector<float> cell_xy;              // [C*2]
    // endpoints, ascending caller pin id
    std::vector<int32_t> ep_pin;             // [E] internal pin
    std::vector<uint8_t> ep_is_d;            // [E]
    std::vector<int32_t> ep_design_ptr;      // [n_designs+1]
    // caller cell types (for resizing) and the item of each cell
    std::vector<int32_t> cell_type;          // [C]
    std::vector<int32_t> item_of_cell;       // [C]
    std::vector<int32_t> cell_level;         // [C] propagation level of each cell
    bool uniform_axes = false;               // all tables share one slew axis and one load axis
    float axes[26] = {};                     // those axes: idx1[7] idx2[7] 1/width1[6] 1/width2[6]
};

// Validate `desc` and fill `plan`.  On failure returns the status and sets
// `err`.  Pure host code: safe to call without a GPU.
sta_status build_plan(const sta_design_desc *desc, Plan &plan, std::string &err);

// Pack several designs into one plan (levels aligned by index).
sta_status build_batch_plan(const sta_design_desc *const *descs, int32_t n, Plan &plan,
                            std::string &err);

}  // namespace sta
