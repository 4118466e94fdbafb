// tile.cpp -- partition of the levelised timing graph into per-block tiles
// (see tile.h).  Pure host code.
//
// Steps.  Forward step s < S processes the items of level s, plus
// endpoints whose driver item sits at a level below s; step S the
// endpoints left over.  The backward pass walks the steps in reverse and
// processes items only (endpoint required times are set by the forward
// pass).
//
// Assignment, step by step: every step has a capacity per tile of
// W * ceil(n / (B W)) entries (n = the level's items), so every tile runs the
// same number of waves.  An item whose critical fan-in (the driver with the
// highest level; the first such input on ties) sits in a tile with room goes
// there; the rest fill the tiles with room in turn.  Endpoints have no
// consumer in the forward pass, so they only fill the slots the items leave
// free: in their driver's tile, oldest first, from the step after their
// driver on; the last step takes whatever is left.  An item's critical fan-in is at
// the previous level whenever the item's level is set by it, so this keeps
// most level-to-level dependencies inside a tile, where they cost a ring
// read after a block barrier instead of an L2 round trip.
//
// Rings.  A tile's list positions number its entries in processing order;
// an entry's ring slot is its position mod R.  A consumer reads a
// producer's slot only if no later entry can have overwritten it by the
// end of the consumer's step: producer position >= end of the consumer's
// step - R.  Otherwise (or across tiles) it reads the mailbox.
#include "tile.h"

#include <algorithm>
#include <string>

namespace sta {

namespace {

int32_t out_pin_of(const Plan &pl, int32_t g)
{
    const int32_t t = pl.item_type[g], p0 = pl.item_pin0[g];
    if (t < 0) return p0;
    return pl.type_kind[t] == 1 ? p0 + 1 : p0 + pl.type_nin[t];
}

int32_t nin_of(const Plan &pl, int32_t g)
{
    const int32_t t = pl.item_type[g];
    return (t >= 0 && pl.type_kind[t] == 0) ? pl.type_nin[t] : 0;
}

}  // namespace

void build_tile_plan(const Plan &pl, int32_t B, int32_t W, int32_t R, TilePlan &tp)
{
    tp = TilePlan{};
    const int32_t I = pl.I, E = pl.E, S = pl.S, P = pl.P;
    const int32_t NS = S + 1;
    tp.B = B;
    tp.NS = NS;
    tp.W = W;
    tp.R = R;
    std::vector<int32_t> level(I), out_item(P, -1), item_of_in(P, -1);
    for (int32_t s = 0; s < S; ++s)
        for (int32_t g = pl.stage_ptr[s]; g < pl.stage_ptr[s + 1]; ++g) level[g] = s;
    for (int32_t g = 0; g < I; ++g) {
        out_item[out_pin_of(pl, g)] = g;
        for (int32_t j = 0; j < nin_of(pl, g); ++j) item_of_in[pl.item_pin0[g] + j] = g;
    }
    auto drv_item = [&](int32_t pin) {
        const int32_t d = pl.drv_of[pin];
        return d >= 0 ? out_item[d] : -1;
    };
    // critical fan-in of every item
    std::vector<int32_t> crit(I, -1);
    for (int32_t g = 0; g < I; ++g) {
        int32_t best = -1;
        for (int32_t j = 0; j < nin_of(pl, g); ++j) {
            const int32_t h = drv_item(pl.item_pin0[g] + j);
            if (h >= 0 && (best < 0 || level[h] > level[best])) best = h;
        }
        crit[g] = best;
    }
    // endpoints by step
    std::vector<int32_t> ep_drv(E), ep_step(E), ep_ptr(NS + 1, 0), ep_by_step(E);
    for (int32_t e = 0; e < E; ++e) {
        ep_drv[e] = drv_item(pl.ep_pin[e]);
        ep_step[e] = ep_drv[e] >= 0 ? std::min(level[ep_drv[e]] + 1, S) : 0;
        ++ep_ptr[ep_step[e] + 1];
    }
    for (int32_t s = 0; s < NS; ++s) ep_ptr[s + 1] += ep_ptr[s];
    {
        std::vector<int32_t> fill(ep_ptr.begin(), ep_ptr.end() - 1);
        for (int32_t e = 0; e < E; ++e) ep_by_step[fill[ep_step[e]]++] = e;
    }
    // assignment: items by critical fan-in within the step capacity;
    // endpoints (leaves of the forward pass, no consumer in it) fill the
    // slots the items leave free, in their tile's driver order, from the step
    // after their driver on; whatever is left runs in the last step
    tp.tile_of.assign(I, -1);
    std::vector<int32_t> ep_tile(E, -1), ep_at(E, -1);
    std::vector<int32_t> cnt((size_t)B * NS, 0), cnt_item((size_t)B * NS, 0);
    std::vector<std::vector<int32_t>> pending(B);   // per tile: endpoints waiting for a free slot, FIFO
    std::vector<size_t> head(B, 0);
    int32_t rr = 0;   // round-robin pointer over tiles
    std::vector<int32_t> deferred;
    for (int32_t s = 0; s < NS; ++s) {
        const int32_t i0 = s < S ? pl.stage_ptr[s] : I, i1 = s < S ? pl.stage_ptr[s + 1] : I;
        const int64_t n = i1 - i0;
        const int64_t waves = std::max<int64_t>(1, (n + (int64_t)B * W - 1) / ((int64_t)B * W));
        const int32_t cap = (int32_t)(W * waves);
        int32_t *cs = cnt.data() + (size_t)s;   // cnt[b * NS + s] = cs[b * NS]
        deferred.clear();
        for (int32_t g = i0; g < i1; ++g) {
            const int32_t pref = crit[g] >= 0 ? tp.tile_of[crit[g]] : -1;
            if (pref >= 0 && cs[(size_t)pref * NS] < cap) {
                tp.tile_of[g] = pref;
                ++cs[(size_t)pref * NS];
            } else {
                deferred.push_back(g);
            }
        }
        for (int32_t g : deferred) {
            while (cs[(size_t)rr * NS] >= cap) rr = (rr + 1) % B;
            tp.tile_of[g] = rr;
            ++cs[(size_t)rr * NS];
            rr = (rr + 1) % B;
        }
        for (int32_t b = 0; b < B; ++b) cnt_item[(size_t)b * NS + s] = cs[(size_t)b * NS];
        // endpoints that became ready at this step join their driver tile's queue
        for (int32_t k = ep_ptr[s]; k < ep_ptr[s + 1]; ++k) {
            const int32_t e = ep_by_step[k];
            const int32_t b = ep_drv[e] >= 0 ? tp.tile_of[ep_drv[e]] : (int32_t)(e % B);
            pending[b].push_back(e);
        }
        auto take = [&](int32_t from, int32_t to) {
            const int32_t e = pending[from][head[from]++];
            ep_tile[e] = to;
            ep_at[e] = s;
            ++cs[(size_t)to * NS];
        };
        // own queue first (the driver's value may still be in the ring) ...
        for (int32_t b = 0; b < B; ++b)
            while (head[b] < pending[b].size() && cs[(size_t)b * NS] < cap) take(b, b);
        // ... then endpoints waiting for two steps or more, from any tile
        // (their driver's value has long been published to the mailbox)
        auto aged = [&](int32_t b) {
            return head[b] < pending[b].size() && ep_step[pending[b][head[b]]] <= s - 2;
        };
        int32_t donor = 0, idle = 0;
        for (int32_t b = 0; b < B && idle < B; ++b) {
            while (cs[(size_t)b * NS] < cap && idle < B) {
                if (aged(donor)) {
                    take(donor, b);
                    idle = 0;
                } else {
                    donor = (donor + 1) % B;
                    ++idle;
                }
            }
        }
        if (s == NS - 1) {   // the last step: everything left, spread evenly
            int32_t to = 0;
            for (int32_t b = 0; b < B; ++b)
                while (head[b] < pending[b].size()) {
                    int32_t best = to;
                    for (int32_t k = 0; k < B; ++k)
                        if (cs[(size_t)k * NS] < cs[(size_t)best * NS]) best = k;
                    take(b, best);
                    to = best;
                }
        }
    }
    // lists, tile-major: items of (b, s) by id, then endpoints by id
    tp.ptr.assign((size_t)B * NS + 1, 0);
    tp.nitem.assign((size_t)B * NS, 0);
    for (size_t i = 0; i < (size_t)B * NS; ++i) {
        tp.ptr[i + 1] = tp.ptr[i] + cnt[i];
        tp.nitem[i] = cnt_item[i];
        tp.max_step_items = std::max(tp.max_step_items, cnt[i]);
    }
    tp.item.assign((size_t)I + E, -1);
    std::vector<int32_t> pos((size_t)I + E, -1);   // absolute list index of each item / endpoint
    {
        std::vector<int32_t> fill(tp.ptr.begin(), tp.ptr.end() - 1);
        for (int32_t g = 0; g < I; ++g) {
            const size_t k = (size_t)tp.tile_of[g] * NS + level[g];
            pos[g] = fill[k]++;
            tp.item[pos[g]] = g;
        }
        for (int32_t e = 0; e < E; ++e) {
            const size_t k = (size_t)ep_tile[e] * NS + ep_at[e];
            pos[(size_t)I + e] = fill[k]++;
            tp.item[pos[(size_t)I + e]] = I + e;
        }
    }
    // tile-relative positions and step ends
    auto tile_base = [&](int32_t b) { return tp.ptr[(size_t)b * NS]; };
    auto step_end = [&](int32_t b, int32_t s) { return tp.ptr[(size_t)b * NS + s + 1] - tile_base(b); };
    auto fwd_code = [&](int32_t h, int32_t b, int32_t s) -> int32_t {
        if (h < 0 || tp.tile_of[h] != b) return -1;
        const int32_t lp = pos[h] - tile_base(b);
        return lp >= step_end(b, s) - R ? lp % R : -1;
    };
    // forward descriptors
    tp.fdesc.assign(((size_t)I + E) * 8, 0);
    for (int32_t g = 0; g < I; ++g) {
        int32_t *dsc = tp.fdesc.data() + (size_t)pos[g] * 8;
        const int32_t b = tp.tile_of[g], s = level[g], nin = nin_of(pl, g);
        int32_t ring[3] = {-1, -1, -1};
        dsc[0] = g;
        dsc[1] = pl.item_pin0[g];
        dsc[2] = pl.item_type[g];
        for (int32_t j = 0; j < 3; ++j) {
            const int32_t a = pl.item_pin0[g] + j;
            const int32_t h0 = j < nin ? drv_item(a) : -1;
            dsc[3 + j] = h0 >= 0 ? h0 : 0;   // the driver's item: its mailbox index
            if (j < nin) {
                const int32_t h = h0;
                ring[j] = fwd_code(h, b, s);
                ++tp.fwd_edges;
                tp.fwd_local += ring[j] >= 0;
            }
        }
        dsc[6] = (int32_t)(((uint32_t)(uint16_t)ring[0]) | ((uint32_t)(uint16_t)ring[1] << 16));
        dsc[7] = (int32_t)(uint32_t)(uint16_t)ring[2];
        if (crit[g] >= 0) {
            ++tp.crit_edges;
            tp.crit_local += tp.tile_of[crit[g]] == b;
        }
    }
    for (int32_t e = 0; e < E; ++e) {
        int32_t *dsc = tp.fdesc.data() + (size_t)pos[(size_t)I + e] * 8;
        const int32_t p = pl.ep_pin[e];
        dsc[0] = I + e;
        dsc[1] = p;
        dsc[2] = ep_drv[e] >= 0 ? ep_drv[e] : 0;   // the driver's item
        dsc[3] = pl.ep_is_d[e];
        dsc[4] = e;
        const int32_t ring = fwd_code(ep_drv[e], ep_tile[e], ep_at[e]);
        dsc[6] = (int32_t)(uint32_t)(uint16_t)ring;
        dsc[7] = (int32_t)(uint32_t)(uint16_t)-1;
    }
    // backward positions: steps in reverse, items only
    tp.rbase.assign((size_t)B * NS, 0);
    for (int32_t b = 0; b < B; ++b) {
        int32_t acc = 0;
        for (int32_t s = NS - 1; s >= 0; --s) {
            tp.rbase[(size_t)b * NS + s] = acc;
            acc += tp.nitem[(size_t)b * NS + s];
        }
    }
    auto rpos = [&](int32_t h) {
        const int32_t b = tp.tile_of[h], s = level[h];
        return tp.rbase[(size_t)b * NS + s] + (pos[h] - tp.ptr[(size_t)b * NS + s]);
    };
    tp.fo_ring.assign(pl.F, (int16_t)-1);
    tp.bdesc.assign(((size_t)I + E) * 16, 0);
    for (int32_t g = 0; g < I; ++g) {
        const int32_t b = tp.tile_of[g], s = level[g];
        const int32_t rend = tp.rbase[(size_t)b * NS + s] + tp.nitem[(size_t)b * NS + s];
        for (int32_t p = pl.fo_ptr[g]; p < pl.fo_ptr[g + 1]; ++p) {
            const int32_t sp = pl.fo_pin[p];
            const int32_t h = sp < P - E ? item_of_in[sp] : -1;
            if (h < 0) continue;   // endpoint sink: its required time is set by the forward pass
            ++tp.bwd_edges;
            if (tp.tile_of[h] != b) continue;
            const int32_t rp = rpos(h);
            if (rp >= rend - R) {
                tp.fo_ring[p] = (int16_t)((rp % R) * 4 + (sp - pl.item_pin0[h]));
                ++tp.bwd_local;
            }
        }
        // backward descriptor: first pin, type, fan-out range, and the first
        // eight sinks with their ring codes (the rest are read from the
        // fan-out arrays)
        int32_t *dsc = tp.bdesc.data() + (size_t)pos[g] * 16;
        const int32_t f0 = pl.fo_ptr[g], f1 = pl.fo_ptr[g + 1];
        int32_t cd[8];
        dsc[0] = pl.item_pin0[g];
        dsc[1] = pl.item_type[g];
        dsc[2] = f0;
        dsc[3] = f1;
        for (int32_t u = 0; u < 8; ++u) {
            dsc[4 + u] = f0 + u < f1 ? pl.fo_pin[f0 + u] : -1;
            cd[u] = f0 + u < f1 ? tp.fo_ring[f0 + u] : -1;
        }
        for (int32_t u = 0; u < 4; ++u)
            dsc[12 + u] = (int32_t)(((uint32_t)(uint16_t)cd[2 * u]) | ((uint32_t)(uint16_t)cd[2 * u + 1] << 16));
    }
}

std::string check_tile_plan(const Plan &pl, const TilePlan &tp)
{
    const int32_t I = pl.I, E = pl.E, S = pl.S, P = pl.P, B = tp.B, NS = tp.NS, R = tp.R;
    if (NS != S + 1 || (int64_t)tp.ptr.size() != (int64_t)B * NS + 1 || tp.ptr[(size_t)B * NS] != I + E)
        return "list sizes";
    std::vector<int32_t> level(I), out_item(P, -1), item_of_in(P, -1);
    for (int32_t s = 0; s < S; ++s)
        for (int32_t g = pl.stage_ptr[s]; g < pl.stage_ptr[s + 1]; ++g) level[g] = s;
    for (int32_t g = 0; g < I; ++g) {
        out_item[out_pin_of(pl, g)] = g;
        for (int32_t j = 0; j < nin_of(pl, g); ++j) item_of_in[pl.item_pin0[g] + j] = g;
    }
    // the mailbox index a descriptor holds for a driven pin: the driver's item
    auto drv_mbox = [&](int32_t pin) {
        const int32_t d = pl.drv_of[pin];
        return d >= 0 && out_item[d] >= 0 ? out_item[d] : 0;
    };
    std::vector<char> seen((size_t)I + E, 0);
    for (int32_t b = 0; b < B; ++b)
        for (int32_t s = 0; s < NS; ++s) {
            const size_t k = (size_t)b * NS + s;
            const int32_t lo = tp.ptr[k], hi = tp.ptr[k + 1], ni = tp.nitem[k];
            if (hi < lo || ni > hi - lo) return "list bounds";
            for (int32_t x = lo; x < hi; ++x) {
                const int32_t id = tp.fdesc[(size_t)x * 8];
                if (id < 0 || id >= I + E || seen[id]) return "entry missing or repeated";
                seen[id] = 1;
                if ((x - lo < ni) != (id < I)) return "items must precede endpoints";
                if (id < I && level[id] != s) return "item at the wrong step";
                if (id >= I) {
                    const int32_t dp = pl.drv_of[pl.ep_pin[id - I]];
                    const int32_t h = dp >= 0 ? out_item[dp] : -1;
                    if (h >= 0 && level[h] >= s) return "endpoint before its driver";
                }
                if (id < I && tp.tile_of[id] != b) return "item in the wrong tile";
            }
        }
    for (char v : seen)
        if (!v) return "entry missing";
    // forward replay: ring[slot] = item whose output it holds
    for (int32_t b = 0; b < B; ++b) {
        std::vector<int32_t> ring(R, -1);
        const int32_t base = tp.ptr[(size_t)b * NS];
        for (int32_t s = 0; s < NS; ++s) {
            const size_t k = (size_t)b * NS + s;
            const int32_t lo = tp.ptr[k], hi = tp.ptr[k + 1];
            std::vector<int32_t> after = ring;
            for (int32_t x = lo; x < hi; ++x) {
                const int32_t id = tp.fdesc[(size_t)x * 8];
                if (id < I) after[(x - base) % R] = id;
            }
            for (int32_t x = lo; x < hi; ++x) {
                const int32_t *d = tp.fdesc.data() + (size_t)x * 8;
                const int32_t id = d[0];
                int32_t codes[3], drv[3], n = 0;
                if (id < I) {
                    n = nin_of(pl, id);
                    codes[0] = (int16_t)(d[6] & 0xffff);
                    codes[1] = (int16_t)((uint32_t)d[6] >> 16);
                    codes[2] = (int16_t)(d[7] & 0xffff);
                    for (int32_t j = 0; j < n; ++j) {
                        drv[j] = d[3 + j];
                        if (drv[j] != drv_mbox(pl.item_pin0[id] + j)) return "descriptor driver";
                    }
                } else {
                    n = 1;
                    codes[0] = (int16_t)(d[6] & 0xffff);
                    drv[0] = d[2];
                    if (drv[0] != drv_mbox(pl.ep_pin[id - I])) return "endpoint driver";
                }
                for (int32_t j = 0; j < n; ++j) {
                    if (codes[j] < 0) continue;
                    if (codes[j] >= R) return "ring code out of range";
                    const int32_t h = drv[j];
                    if (ring[codes[j]] != h || after[codes[j]] != h) return "forward ring read of a stale slot";
                }
            }
            ring.swap(after);
        }
    }
    // backward replay: items only, steps in reverse; ring[slot] = item whose input required times it holds
    for (int32_t b = 0; b < B; ++b) {
        std::vector<int32_t> ring(R, -1);
        for (int32_t s = NS - 1; s >= 0; --s) {
            const size_t k = (size_t)b * NS + s;
            const int32_t lo = tp.ptr[k], ni = tp.nitem[k], rb = tp.rbase[k];
            std::vector<int32_t> after = ring;
            for (int32_t i = 0; i < ni; ++i) after[(rb + i) % R] = tp.fdesc[(size_t)(lo + i) * 8];
            for (int32_t i = 0; i < ni; ++i) {
                const int32_t g = tp.fdesc[(size_t)(lo + i) * 8];
                const int32_t *bd = tp.bdesc.data() + (size_t)(lo + i) * 16;
                if (bd[0] != pl.item_pin0[g] || bd[1] != pl.item_type[g] || bd[2] != pl.fo_ptr[g] ||
                    bd[3] != pl.fo_ptr[g + 1])
                    return "backward descriptor";
                for (int32_t u = 0; u < 8; ++u) {
                    const int32_t p = pl.fo_ptr[g] + u;
                    const int32_t want_s = p < pl.fo_ptr[g + 1] ? pl.fo_pin[p] : -1;
                    const int32_t want_c = p < pl.fo_ptr[g + 1] ? tp.fo_ring[p] : -1;
                    const int32_t got_c = (int16_t)((uint32_t)bd[12 + u / 2] >> (16 * (u & 1)));
                    if (bd[4 + u] != want_s || got_c != want_c) return "backward descriptor sinks";
                }
                for (int32_t p = pl.fo_ptr[g]; p < pl.fo_ptr[g + 1]; ++p) {
                    const int32_t code = tp.fo_ring[p];
                    if (code < 0) continue;
                    const int32_t slot = code >> 2, j = code & 3, sp = pl.fo_pin[p];
                    if (slot >= R) return "backward ring code out of range";
                    const int32_t h = item_of_in[sp];
                    if (h < 0 || sp != pl.item_pin0[h] + j) return "backward ring pin";
                    if (ring[slot] != h || after[slot] != h) return "backward ring read of a stale slot";
                }
            }
            ring.swap(after);
        }
    }
    return std::string();
}

}  // namespace sta
