// tile.h -- partition of the levelised timing graph into per-block tiles.
//
// The tile schedule (tile.cu) runs each propagation pass as one resident
// block per tile.  A block walks "steps" -- the levels in order, forward; in
// reverse order, backward -- and at each step processes only its own items.
// Results a block consumes from itself come through a shared-memory ring,
// one barrier per step; results from other blocks come through the parity
// mailboxes of the dataflow schedule.  The partition below decides which
// block owns each item so that most dependencies on the previous level stay
// inside a block: an item goes to the block of its critical fan-in (the
// driver item with the highest level) unless that block's step is full.
//
// Pure host code.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "plan.h"

namespace sta {

// Ring codes: a dependency read from the shared ring carries its slot; -1
// means "through the mailbox".  Forward slots hold an item's output arrival
// and slew (or nothing for endpoints, which are leaves); backward slots hold
// the required times of an item's input pins (slot * 4 + pin slot).
struct TilePlan {
    int32_t B = 0;        // tiles (resident blocks)
    int32_t NS = 0;       // steps: levels 0 .. S-1, then one step of endpoints driven by the last level
    int32_t W = 0;        // items one wave of a block processes (threads / (4 KL))
    int32_t R = 0;        // ring slots (items) of a block
    // Lists, tile-major then step: list (b, s) = item[ptr[b*NS + s] .. ptr[b*NS + s + 1]),
    // items (id g) first, then endpoints (id I + e).
    std::vector<int32_t> ptr;       // [B*NS + 1]
    std::vector<int32_t> nitem;     // [B*NS] items at the front of list (b, s)
    std::vector<int32_t> rbase;     // [B*NS] backward position of the first item of list (b, s)
    std::vector<int32_t> item;      // [I + E] list entries
    // forward descriptor of each list entry: two int4 (see tile.cu)
    std::vector<int32_t> fdesc;     // [(I + E) * 8]
    // backward descriptor of each item entry: four int4 (see tile.cu)
    std::vector<int32_t> bdesc;     // [(I + E) * 16]
    std::vector<int16_t> fo_ring;   // [F] backward ring code of each fan-out entry (slot * 4 + pin slot) or -1
    std::vector<int32_t> tile_of;   // [I] owning tile of every item
    // statistics of the partition (tests and design notes)
    int64_t fwd_edges = 0, fwd_local = 0;   // fan-in edges item -> item, and those read from the ring
    int64_t bwd_edges = 0, bwd_local = 0;   // fan-out entries to item pins, and those read from the ring
    int64_t crit_edges = 0, crit_local = 0; // critical fan-in edges, and those inside one tile
    int32_t max_step_items = 0;             // largest list (b, s)
};

// Build the partition of `pl` into B tiles of W items per wave with rings of
// R slots.  Deterministic.
void build_tile_plan(const Plan &pl, int32_t B, int32_t W, int32_t R, TilePlan &tp);

// Check a partition against the plan by replaying what the kernels do:
// every item and endpoint sits in exactly one list, at its step; the lists
// respect the step capacities; and, walking each tile's lists step by step
// with the ring written as the kernels write it, every ring read finds its
// producer's value whether it comes before or after the other writes of
// its step.  Returns an empty string, or the first violation.
std::string check_tile_plan(const Plan &pl, const TilePlan &tp);

}  // namespace sta
