// plan.cpp -- validation, Kahn levelisation and level-major layout (host).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

namespace sta {
namespace {

bool finite(float x) { return std::isfinite(x); }

struct Fail {
    sta_status code;
    std::string msg;
};

#define REQUIRE(cond, code, ...)                                   \
    do {                                                           \
        if (!(cond)) {                                             \
            char _b[256];                                          \
            std::snprintf(_b, sizeof(_b), __VA_ARGS__);            \
            throw Fail{code, std::string(_b)};                     \
        }                                                          \
    } while (0)

void pack_library(const sta_library *L, Plan &pl)
{
    const int T = L->n_types;
    REQUIRE(T >= 1 && T <= 4096, STA_EINVAL, "n_types %d out of range [1, 4096]", T);
    REQUIRE(L->type_nin && L->type_kind && L->arc_sense && L->lut_idx1 && L->lut_idx2 && L->lut_val &&
                L->pin_cap,
            STA_EINVAL, "library array is NULL");
    REQUIRE(finite(L->setup_ns) && finite(L->hold_ns) && finite(L->po_cap_pf) && L->po_cap_pf >= 0,
            STA_EINVAL, "setup/hold/po_cap not finite");
    pl.T = T;
    pl.type_nin.assign(L->type_nin, L->type_nin + T);
    pl.type_kind.assign(L->type_kind, L->type_kind + T);
    pl.arc_sense.assign((size_t)T * kMaxSlot, kSenseNone);
    pl.type_pin_cap.assign((size_t)T * 4, 0.f);
    pl.lut.assign((size_t)T * kMaxSlot * 4 * kTabStride, 0.f);
    for (int t = 0; t < T; ++t) {
        const int nin = L->type_nin[t], kind = L->type_kind[t];
        REQUIRE(nin >= 1 && nin <= kMaxSlot, STA_EINVAL, "type %d: %d inputs (1..3 allowed)", t, nin);
        REQUIRE(kind == 0 || kind == 1, STA_EINVAL, "type %d: kind %d", t, kind);
        if (kind == 1)
            REQUIRE(nin == 2 && L->arc_sense[t * 3] == kSenseNone && L->arc_sense[t * 3 + 1] == kSenseRise,
                    STA_EINVAL, "type %d: a flip-flop needs inputs (D: NONE, CK: RISE)", t);
        for (int s = 0; s < nin; ++s) {
            const int se = L->arc_sense[t * 3 + s];
            if (kind == 0)
                REQUIRE(se == kSensePos || se == kSenseNeg || se == kSenseNon, STA_EINVAL,
                        "type %d slot %d: sense %d (POS/NEG/NON required)", t, s, se);
            pl.arc_sense[(size_t)t * 3 + s] = se;
            const float cap = L->pin_cap[(size_t)t * 4 + s];
            REQUIRE(finite(cap) && cap >= 0, STA_EINVAL, "type %d slot %d: bad pin cap", t, s);
            pl.type_pin_cap[(size_t)t * 4 + s] = cap;
            if (se == kSenseNone) continue;
            for (int tb = 0; tb < 4; ++tb) {
                const size_t src = (((size_t)t * 3 + s) * 4 + tb);
                const float *i1 = L->lut_idx1 + src * kNldm;
                const float *i2 = L->lut_idx2 + src * kNldm;
                const float *v = L->lut_val + src * kNldm * kNldm;
                float *o = pl.lut.data() + src * kTabStride;
                for (int k = 0; k < kNldm; ++k) {
                    REQUIRE(finite(i1[k]) && finite(i2[k]), STA_EINVAL, "type %d: table axis not finite", t);
                    if (k) REQUIRE(i1[k] > i1[k - 1] && i2[k] > i2[k - 1], STA_EINVAL,
                                   "type %d slot %d table %d: axis not strictly increasing", t, s, tb);
                    o[k] = i1[k];
                    o[7 + k] = i2[k];
                }
                for (int k = 0; k < kNldm - 1; ++k) {
                    o[14 + k] = 1.0f / (i1[k + 1] - i1[k]);
                    o[20 + k] = 1.0f / (i2[k + 1] - i2[k]);
                }
                for (int k = 0; k < kNldm * kNldm; ++k) {
                    REQUIRE(finite(v[k]), STA_EINVAL, "type %d slot %d table %d: value not finite", t, s, tb);
                    o[26 + k] = v[k];
                }
            }
        }
    }
    // do all active tables share the same axes?  Then one segment search per
    // (slew, load) query serves every table.
    pl.uniform_axes = true;
    const float *ref = nullptr;
    for (int t = 0; t < T && pl.uniform_axes; ++t)
        for (int s = 0; s < pl.type_nin[t] && pl.uniform_axes; ++s) {
            if (pl.arc_sense[(size_t)t * 3 + s] == kSenseNone) continue;
            for (int tb = 0; tb < 4; ++tb) {
                const float *o = pl.lut.data() + (((size_t)t * 3 + s) * 4 + tb) * kTabStride;
                if (!ref) {
                    ref = o;
                    std::memcpy(pl.axes, o, sizeof(pl.axes));
                }
                else if (std::memcmp(o, ref, 26 * sizeof(float)) != 0) { pl.uniform_axes = false; break; }
            }
        }
    pl.setup = L->setup_ns;
    pl.hold = L->hold_ns;
    pl.po_cap = L->po_cap_pf;
}

void build(const sta_design_desc *d, Plan &pl)
{
    REQUIRE(d != nullptr && d->lib != nullptr, STA_EINVAL, "NULL descriptor or library");
    pack_library(d->lib, pl);
    const int32_t C = d->n_cells, P = d->n_pins, N = d->n_nets;
    REQUIRE(C >= 0 && P >= 0 && N >= 0, STA_EINVAL, "negative size");
    REQUIRE(d->n_corners >= 1 && d->n_corners <= 16, STA_EINVAL, "n_corners %d out of [1, 16]", d->n_corners);
    const int Kc = d->n_corners;
    REQUIRE(d->n_exc >= 0 && d->n_exc <= 7, STA_EINVAL, "n_exc %d out of [0, 7]", d->n_exc);
    REQUIRE(d->n_exc == 0 || (d->exc_from_ptr && d->exc_to_ptr && d->exc_action && d->exc_mult &&
                              (d->exc_from || d->exc_from_ptr[d->n_exc] == 0) &&
                              (d->exc_to || d->exc_to_ptr[d->n_exc] == 0)),
            STA_EINVAL, "exception arrays NULL");
    REQUIRE(d->n_exc == 0 || d->gamma_ns == 0.f, STA_EINVAL, "timing exceptions need gamma_ns = 0");
    // tags: 0 = no group; group g owns 1 + (its through sets) tags, one per
    // stage of its -through sequence
    int Tg = 1;
    if (d->n_exc > 0 && d->exc_thru_ptr) {
        REQUIRE(d->exc_thru_set_ptr && (d->exc_thru_pin || d->exc_thru_set_ptr[d->exc_thru_ptr[d->n_exc]] == 0) &&
                    d->exc_thru_ptr[0] == 0,
                STA_EINVAL, "exception through arrays NULL or not starting at 0");
        for (int g = 0; g < d->n_exc; ++g)
            REQUIRE(d->exc_thru_ptr[g + 1] >= d->exc_thru_ptr[g], STA_EINVAL, "exception group %d: through offsets", g);
    }
    for (int g = 0; g < d->n_exc; ++g) Tg += 1 + (d->exc_thru_ptr ? d->exc_thru_ptr[g + 1] - d->exc_thru_ptr[g] : 0);
    REQUIRE(Tg <= 32, STA_EINVAL, "%d exception tags (groups + their through sets) exceed 32", Tg);
    const int K = Kc * Tg;   // states: corner * Tg + tag
    pl.Kc = Kc;
    pl.Tg = Tg;
    pl.K = K;
    pl.C = C;
    pl.P = P;
    pl.lut_scale.assign(K, 1.f);
    pl.rc_scale.assign(K, 1.f);
    for (int k = 0; k < Kc; ++k) {
        const float ls = d->lut_scale ? d->lut_scale[k] : 1.f, rs = d->rc_scale ? d->rc_scale[k] : 1.f;
        REQUIRE(finite(ls) && ls > 0 && finite(rs) && rs > 0, STA_EINVAL, "corner %d: scales must be finite and > 0",
                k);
        for (int g = 0; g < Tg; ++g) {
            pl.lut_scale[k * Tg + g] = ls;
            pl.rc_scale[k * Tg + g] = rs;
        }
    }
    REQUIRE(finite(d->period_ns) && finite(d->clk_slew_ns) && d->clk_slew_ns >= 0 && finite(d->pi_at_ns) &&
                finite(d->pi_slew_ns) && d->pi_slew_ns >= 0,
            STA_EINVAL, "clock / input constraints not finite or negative slew");
    REQUIRE(finite(d->gamma_ns) && d->gamma_ns >= 0, STA_EINVAL, "gamma_ns must be finite and >= 0");
    REQUIRE(d->net_model == STA_NET_ELMORE || d->net_model == STA_NET_ARNOLDI, STA_EINVAL,
            "net_model must be STA_NET_ELMORE or STA_NET_ARNOLDI");
    REQUIRE(d->wire_model == STA_WIRE_STAR || d->wire_model == STA_WIRE_STEINER, STA_EINVAL,
            "wire_model must be STA_WIRE_STAR or STA_WIRE_STEINER");
    REQUIRE(d->wire_model == STA_WIRE_STAR || !d->rc_ptr, STA_EINVAL,
            "STA_WIRE_STEINER builds RC from positions (rc_ptr must be NULL)");
    REQUIRE(d->net_model == STA_NET_ELMORE || d->rc_ptr || d->wire_model == STA_WIRE_STEINER, STA_EINVAL,
            "STA_NET_ARNOLDI needs RC trees (rc_ptr) or Steiner trees");
    REQUIRE(d->net_model == STA_NET_ELMORE || (d->arnoldi_order >= 0 && d->arnoldi_order <= 3), STA_EINVAL,
            "arnoldi_order must be in 0..3");
    pl.net_model = d->net_model;
    pl.arnoldi_q = d->arnoldi_order > 0 ? d->arnoldi_order : 3;
    pl.period = d->period_ns;
    pl.clk_slew = d->clk_slew_ns;
    pl.pi_at = d->pi_at_ns;
    pl.pi_slew = d->pi_slew_ns;
    pl.gamma = d->gamma_ns;
    pl.placed = (d->rc_ptr == nullptr);
    pl.r_per_um = d->r_per_um;
    pl.c_per_um = d->c_per_um;
    pl.steiner = pl.placed && d->wire_model == STA_WIRE_STEINER;
    pl.n_nets = N;
    if (pl.steiner) {
        REQUIRE(finite(d->r_per_um_y) && finite(d->c_per_um_y), STA_EINVAL, "unit R/C along y must be finite");
        pl.r_per_um_y = d->r_per_um_y > 0.f ? d->r_per_um_y : d->r_per_um;
        pl.c_per_um_y = d->c_per_um_y > 0.f ? d->c_per_um_y : d->c_per_um;
        REQUIRE(d->net_model == STA_NET_ELMORE || (d->r_per_um > 0.f && pl.r_per_um_y > 0.f), STA_EINVAL,
                "STA_NET_ARNOLDI on Steiner trees needs unit R > 0");
    }
    if (P > 0) REQUIRE(d->pin_role != nullptr, STA_EINVAL, "pin_role is NULL");
    if (C > 0) REQUIRE(d->cell_type && d->cell_pin_ptr && d->cell_pin, STA_EINVAL, "cell arrays NULL");
    if (N > 0) REQUIRE(d->net_pin_ptr && d->net_pin, STA_EINVAL, "net arrays NULL");
    if (pl.placed) {
        REQUIRE(finite(d->r_per_um) && finite(d->c_per_um) && d->r_per_um >= 0 && d->c_per_um >= 0, STA_EINVAL,
                "unit R/C must be finite and >= 0");
        if (C > 0) REQUIRE(d->cell_xy != nullptr, STA_EINVAL, "positions mode needs cell_xy");
    } else if (N > 0) {
        REQUIRE(d->rc_parent && d->rc_R && d->rc_C && d->rc_pin_node, STA_EINVAL, "RC arrays NULL");
    }

    // ---- pins and cells
    for (int32_t p = 0; p < P; ++p)
        REQUIRE(d->pin_role[p] >= 0 && d->pin_role[p] <= 6, STA_EINVAL, "pin %d: role %d", p, d->pin_role[p]);
    std::vector<int32_t> pin_cell(P, -1), pin_slot(P, -1);
    if (C > 0) REQUIRE(d->cell_pin_ptr[0] == 0, STA_EINVAL, "cell_pin_ptr[0] != 0");
    pl.cell_type.assign(d->cell_type, d->cell_type + C);
    for (int32_t c = 0; c < C; ++c) {
        const int32_t t = d->cell_type[c];
        REQUIRE(t >= 0 && t < pl.T, STA_EINVAL, "cell %d: type %d out of range", c, t);
        const int nin = pl.type_nin[t];
        REQUIRE(d->cell_pin_ptr[c + 1] - d->cell_pin_ptr[c] == nin + 1, STA_EINVAL,
                "cell %d: %d pins, type needs %d", c, d->cell_pin_ptr[c + 1] - d->cell_pin_ptr[c], nin + 1);
        for (int s = 0; s <= nin; ++s) {
            const int32_t p = d->cell_pin[d->cell_pin_ptr[c] + s];
            REQUIRE(p >= 0 && p < P, STA_EINVAL, "cell %d: pin id %d out of range", c, p);
            REQUIRE(pin_cell[p] < 0, STA_EINVAL, "pin %d belongs to two cells", p);
            pin_cell[p] = c;
            pin_slot[p] = s;
            int want;
            if (pl.type_kind[t] == 1) want = (s == 0) ? kPinD : (s == 1) ? kPinCK : kPinQ;
            else want = (s == nin) ? kPinOUT : kPinIN;
            REQUIRE(d->pin_role[p] == want, STA_EINVAL, "cell %d slot %d: pin %d has role %d, expected %d", c, s, p,
                    d->pin_role[p], want);
        }
    }
    for (int32_t p = 0; p < P; ++p)
        if (pin_cell[p] < 0)
            REQUIRE(d->pin_role[p] == kPinPI || d->pin_role[p] == kPinPO, STA_EINVAL,
                    "pin %d: role %d but on no cell", p, d->pin_role[p]);

    // ---- nets
    std::vector<int32_t> drv_net(P, -1), sink_net(P, -1), sink_entry(P, -1);
    if (N > 0) REQUIRE(d->net_pin_ptr[0] == 0, STA_EINVAL, "net_pin_ptr[0] != 0");
    for (int32_t n = 0; n < N; ++n) {
        const int32_t b = d->net_pin_ptr[n], e = d->net_pin_ptr[n + 1];
        REQUIRE(e > b, STA_EINVAL, "net %d: no driver", n);
        const int32_t drv = d->net_pin[b];
        REQUIRE(drv >= 0 && drv < P, STA_EINVAL, "net %d: driver id %d out of range", n, drv);
        const int r = d->pin_role[drv];
        REQUIRE(r == kPinPI || r == kPinOUT || r == kPinQ, STA_EINVAL, "net %d: driver pin %d has role %d", n, drv, r);
        REQUIRE(drv_net[drv] < 0, STA_EINVAL, "pin %d drives two nets", drv);
        drv_net[drv] = n;
        for (int32_t k = b + 1; k < e; ++k) {
            const int32_t s = d->net_pin[k];
            REQUIRE(s >= 0 && s < P, STA_EINVAL, "net %d: sink id %d out of range", n, s);
            const int rs = d->pin_role[s];
            REQUIRE(rs == kPinIN || rs == kPinD || rs == kPinPO, STA_EINVAL, "net %d: sink pin %d has role %d", n, s, rs);
            REQUIRE(sink_net[s] < 0, STA_EINVAL, "pin %d is a sink of two nets", s);
            sink_net[s] = n;
            sink_entry[s] = k;
        }
    }
    for (int32_t p = 0; p < P; ++p) {
        const int r = d->pin_role[p];
        if (r == kPinIN || r == kPinD || r == kPinPO)
            REQUIRE(sink_net[p] >= 0, STA_EINVAL, "pin %d (role %d) is driven by no net", p, r);
    }
    // ---- RC
    if (!pl.placed) {
        REQUIRE(d->rc_ptr[0] == 0, STA_EINVAL, "rc_ptr[0] != 0");
        for (int32_t n = 0; n < N; ++n) {
            const int32_t b = d->rc_ptr[n], e = d->rc_ptr[n + 1];
            REQUIRE(e > b, STA_EINVAL, "net %d: RC tree has no node", n);
            REQUIRE(d->rc_parent[b] == -1, STA_EINVAL, "net %d: RC node 0 must be the root", n);
            for (int32_t i = b; i < e; ++i) {
                if (i > b)
                    REQUIRE(d->rc_parent[i] >= 0 && d->rc_parent[i] < i - b, STA_EINVAL,
                            "net %d: RC node %d parent %d not before it", n, i - b, d->rc_parent[i]);
                REQUIRE(finite(d->rc_R[i]) && d->rc_R[i] >= 0 && finite(d->rc_C[i]) && d->rc_C[i] >= 0,
                        STA_EINVAL, "net %d: negative or non-finite R/C at node %d", n, i - b);
                if (i > b && d->net_model == STA_NET_ARNOLDI)
                    REQUIRE(d->rc_R[i] > 0, STA_EINVAL, "net %d: STA_NET_ARNOLDI needs R > 0 (node %d)", n, i - b);
            }
            REQUIRE(d->rc_pin_node[d->net_pin_ptr[n]] == 0, STA_EINVAL, "net %d: driver must sit on node 0", n);
            for (int32_t k = d->net_pin_ptr[n] + 1; k < d->net_pin_ptr[n + 1]; ++k)
                REQUIRE(d->rc_pin_node[k] >= 0 && d->rc_pin_node[k] < e - b, STA_EINVAL,
                        "net %d: sink node %d out of range", n, d->rc_pin_node[k]);
        }
        pl.NN = N ? d->rc_ptr[N] : 0;
    } else {
        for (int64_t i = 0; i < 2LL * C; ++i)
            REQUIRE(finite(d->cell_xy[i]), STA_EINVAL, "cell_xy[%lld] not finite", (long long)i);
        if (pl.steiner) {   // integer nm coordinates must fit: |x|, |y| <= 1e6 um
            for (int64_t i = 0; i < 2LL * C; ++i)
                REQUIRE(std::fabs(d->cell_xy[i]) <= 1e6f, STA_EINVAL, "cell_xy[%lld] beyond 1e6 um", (long long)i);
            if (d->port_xy)
                for (int32_t p = 0; p < P; ++p)
                    if (d->pin_role[p] == kPinPI || d->pin_role[p] == kPinPO)
                        REQUIRE(finite(d->port_xy[2 * (size_t)p]) && finite(d->port_xy[2 * (size_t)p + 1]) &&
                                    std::fabs(d->port_xy[2 * (size_t)p]) <= 1e6f &&
                                    std::fabs(d->port_xy[2 * (size_t)p + 1]) <= 1e6f,
                                STA_EINVAL, "port_xy of pin %d not finite or beyond 1e6 um", p);
        }
    }

    // ---- items: primary inputs (ascending pin id), then cells
    std::vector<int32_t> pis;
    for (int32_t p = 0; p < P; ++p)
        if (d->pin_role[p] == kPinPI) pis.push_back(p);
    const int32_t nPI = (int32_t)pis.size();
    const int32_t I = nPI + C;
    pl.I = I;
    auto item_of_driver = [&](int32_t drvpin) -> int32_t {
        return d->pin_role[drvpin] == kPinPI ? -1 : nPI + pin_cell[drvpin];
    };
    std::vector<int32_t> pi_item(P, -1);
    for (int32_t i = 0; i < nPI; ++i) pi_item[pis[i]] = i;
    auto item_of = [&](int32_t drvpin) -> int32_t {
        int32_t it = item_of_driver(drvpin);
        return it >= 0 ? it : pi_item[drvpin];
    };
    // successors and in-degrees (every input of a combinational cell)
    std::vector<int32_t> indeg(I, 0), succ_ptr(I + 1, 0);
    for (int32_t c = 0; c < C; ++c) {
        const int32_t t = d->cell_type[c];
        if (pl.type_kind[t] == 1) continue;
        for (int s = 0; s < pl.type_nin[t]; ++s) {
            const int32_t a = d->cell_pin[d->cell_pin_ptr[c] + s];
            const int32_t drv = d->net_pin[d->net_pin_ptr[sink_net[a]]];
            succ_ptr[item_of(drv) + 1]++;
            indeg[nPI + c]++;
        }
    }
    std::partial_sum(succ_ptr.begin(), succ_ptr.end(), succ_ptr.begin());
    std::vector<int32_t> succ(succ_ptr[I]), fill(succ_ptr.begin(), succ_ptr.end() - 1);
    for (int32_t c = 0; c < C; ++c) {
        const int32_t t = d->cell_type[c];
        if (pl.type_kind[t] == 1) continue;
        for (int s = 0; s < pl.type_nin[t]; ++s) {
            const int32_t a = d->cell_pin[d->cell_pin_ptr[c] + s];
            const int32_t drv = d->net_pin[d->net_pin_ptr[sink_net[a]]];
            succ[fill[item_of(drv)]++] = nPI + c;
        }
    }
    // Kahn by layers: level = longest path from a source item
    std::vector<int32_t> level(I, -1), order;
    order.reserve(I);
    for (int32_t i = 0; i < I; ++i)
        if (indeg[i] == 0) { order.push_back(i); level[i] = 0; }
    size_t head = 0;
    pl.stage_ptr.assign(1, 0);
    while (head < order.size()) {
        const size_t layer_end = order.size();
        const int32_t lv = level[order[head]];
        for (; head < layer_end; ++head) {
            const int32_t it = order[head];
            for (int32_t k = succ_ptr[it]; k < succ_ptr[it + 1]; ++k) {
                const int32_t v = succ[k];
                if (--indeg[v] == 0) { level[v] = lv + 1; order.push_back(v); }
            }
        }
        pl.stage_ptr.push_back((int32_t)layer_end);
    }
    if ((int32_t)order.size() != I) {
        int32_t bad = -1;
        for (int32_t i = 0; i < I; ++i)
            if (level[i] < 0) { bad = i - nPI; break; }
        throw Fail{STA_ECYCLE, "combinational loop through cell " + std::to_string(bad)};
    }
    pl.S = (int32_t)pl.stage_ptr.size() - 1;
    // Items inside one level are grouped by cell type (primary inputs first):
    // the kernels run 8 / KL consecutive items per warp, and items of one type
    // take the same branches (input count, arc senses), so a warp does not
    // pay for the arcs of every type in the level.  Within a type, items are
    // ordered by the position of their critical fan-in (the driver item of
    // the highest level) in the previous levels' order, then by original
    // index: items whose inputs complete together share a warp.
    std::vector<int32_t> pos_of(I, -1);
    for (int32_t s = 0; s < pl.S; ++s) {
        std::vector<int32_t> key(pl.stage_ptr[s + 1] - pl.stage_ptr[s]);
        for (int32_t i = pl.stage_ptr[s]; i < pl.stage_ptr[s + 1]; ++i) {
            const int32_t it = order[i];
            int32_t best = -1, best_lv = -1;
            if (it >= nPI) {
                const int32_t c = it - nPI, t = d->cell_type[c];
                if (pl.type_kind[t] != 1)
                    for (int sl = 0; sl < pl.type_nin[t]; ++sl) {
                        const int32_t a = d->cell_pin[d->cell_pin_ptr[c] + sl];
                        const int32_t h = item_of(d->net_pin[d->net_pin_ptr[sink_net[a]]]);
                        if (level[h] > best_lv) {
                            best_lv = level[h];
                            best = pos_of[h];
                        }
                    }
            }
            key[i - pl.stage_ptr[s]] = best;
        }
        std::vector<int32_t> idx(key.size());
        for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int32_t)i;
        const int32_t base = pl.stage_ptr[s];
        std::sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
            const int32_t a = order[base + x], b = order[base + y];
            const int32_t ta = a < nPI ? -1 : d->cell_type[a - nPI];
            const int32_t tb = b < nPI ? -1 : d->cell_type[b - nPI];
            if (ta != tb) return ta < tb;
            if (key[x] != key[y]) return key[x] < key[y];
            return a < b;
        });
        std::vector<int32_t> sorted(idx.size());
        for (size_t i = 0; i < idx.size(); ++i) sorted[i] = order[base + idx[i]];
        for (size_t i = 0; i < idx.size(); ++i) {
            order[base + i] = sorted[i];
            pos_of[sorted[i]] = base + (int32_t)i;
        }
    }
    pl.max_width = 0;
    for (int32_t s = 0; s < pl.S; ++s) pl.max_width = std::max(pl.max_width, pl.stage_ptr[s + 1] - pl.stage_ptr[s]);

    // ---- internal pin numbering: item groups level-major, then endpoints
    pl.gpu_of.assign(P, -1);
    pl.item_pin0.resize(I);
    pl.item_type.resize(I);
    pl.item_cell.resize(I);
    pl.item_of_cell.assign(C, -1);
    int32_t next = 0;
    std::vector<int32_t> out_pin_of_item(I);
    for (int32_t g = 0; g < I; ++g) {
        const int32_t it = order[g];
        pl.item_pin0[g] = next;
        if (it < nPI) {
            pl.item_type[g] = -1;
            pl.item_cell[g] = -1;
            pl.gpu_of[pis[it]] = next++;
            out_pin_of_item[g] = pis[it];
        } else {
            const int32_t c = it - nPI, t = d->cell_type[c];
            pl.item_type[g] = t;
            pl.item_cell[g] = c;
            pl.item_of_cell[c] = g;
            const int32_t *cp = d->cell_pin + d->cell_pin_ptr[c];
            if (pl.type_kind[t] == 1) {          // flip-flop group: CK, Q (D is an endpoint)
                pl.gpu_of[cp[1]] = next++;
                pl.gpu_of[cp[2]] = next++;
                out_pin_of_item[g] = cp[2];
            } else {
                for (int s = 0; s <= pl.type_nin[t]; ++s) pl.gpu_of[cp[s]] = next++;
                out_pin_of_item[g] = cp[pl.type_nin[t]];
            }
        }
    }
    for (int32_t p = 0; p < P; ++p) {
        const int r = d->pin_role[p];
        if (r == kPinD || r == kPinPO) {
            pl.ep_pin.push_back(next);
            pl.ep_is_d.push_back(r == kPinD ? 1 : 0);
            pl.gpu_of[p] = next++;
        }
    }
    REQUIRE(next == P, STA_EINVAL, "internal: numbered %d of %d pins", next, P);
    pl.E = (int32_t)pl.ep_pin.size();
    // level of each cell as the launch schedule sees it (the stage holding its item)
    pl.cell_level.assign(C, -1);
    for (int32_t s = 0; s < pl.S; ++s)
        for (int32_t g = pl.stage_ptr[s]; g < pl.stage_ptr[s + 1]; ++g)
            if (pl.item_cell[g] >= 0) pl.cell_level[pl.item_cell[g]] = s;
    pl.ep_design_ptr = {0, pl.E};

    // ---- per-pin maps
    pl.drv_of.assign(P, -1);
    pl.pin_cell.assign(P, 0);
    std::vector<int32_t> port_index(P, -1);
    int32_t n_ports = 0;
    for (int32_t p = 0; p < P; ++p)
        if (pin_cell[p] < 0) port_index[p] = n_ports++;
    pl.port_xy.assign((size_t)n_ports * 2, 0.f);
    for (int32_t p = 0; p < P; ++p) {
        const int32_t g = pl.gpu_of[p];
        if (sink_net[p] >= 0) pl.drv_of[g] = pl.gpu_of[d->net_pin[d->net_pin_ptr[sink_net[p]]]];
        if (pin_cell[p] >= 0) pl.pin_cell[g] = pin_cell[p];
        else {
            pl.pin_cell[g] = -(port_index[p] + 1);
            if (d->port_xy) {
                pl.port_xy[2 * (size_t)port_index[p]] = d->port_xy[2 * (size_t)p];
                pl.port_xy[2 * (size_t)port_index[p] + 1] = d->port_xy[2 * (size_t)p + 1];
            }
        }
    }
    if (pl.placed && C > 0) pl.cell_xy.assign(d->cell_xy, d->cell_xy + 2 * (size_t)C);

    // ---- fan-out (net sinks) per item, RC nodes per item, pin caps
    auto sink_cap = [&](int32_t s) -> float {
        if (d->pin_role[s] == kPinPO) return pl.po_cap;
        return pl.type_pin_cap[(size_t)d->cell_type[pin_cell[s]] * 4 + pin_slot[s]];
    };
    pl.fo_ptr.assign(I + 1, 0);
    pl.rc_ptr.assign(I + 1, 0);
    pl.net_of_item.assign(I, -1);
    if (pl.steiner) {
        pl.st_node_ptr.assign(I + 1, 0);
        pl.st_adj_ptr.assign(I + 1, 0);
    }
    for (int32_t g = 0; g < I; ++g) {
        const int32_t n = drv_net[out_pin_of_item[g]];
        pl.net_of_item[g] = n;
        const int32_t m = n >= 0 ? d->net_pin_ptr[n + 1] - d->net_pin_ptr[n] - 1 : 0;   // sinks
        pl.fo_ptr[g + 1] = pl.fo_ptr[g] + m;
        if (!pl.placed) pl.rc_ptr[g + 1] = pl.rc_ptr[g] + (n >= 0 ? d->rc_ptr[n + 1] - d->rc_ptr[n] : 0);
        if (pl.steiner) {
            // tree capacity 2 m nodes (m + 1 pins, at most m - 1 Steiner points);
            // working storage 3 (m + 1) nodes, bitset rows for nets of <= 64 pins
            const int64_t w = m > 0 ? 3LL * (m + 1) : 0;
            pl.rc_ptr[g + 1] = pl.rc_ptr[g] + 2 * m;
            pl.st_node_ptr[g + 1] = pl.st_node_ptr[g] + w;
            pl.st_adj_ptr[g + 1] = pl.st_adj_ptr[g] + (m > 0 && m + 1 <= kSteinerMaxPins ? w * ((w + 31) / 32) : 0);
        }
    }
    if (pl.steiner) {
        pl.NN = pl.rc_ptr[I];
        pl.st_items.clear();
        for (int32_t g = 0; g < I; ++g)
            if (pl.fo_ptr[g + 1] > pl.fo_ptr[g]) pl.st_items.push_back(g);
        std::stable_sort(pl.st_items.begin(), pl.st_items.end(), [&](int32_t a, int32_t b) {
            return pl.fo_ptr[a + 1] - pl.fo_ptr[a] < pl.fo_ptr[b + 1] - pl.fo_ptr[b];
        });
        pl.st_small = 0;
        while (pl.st_small < (int32_t)pl.st_items.size() &&
               pl.fo_ptr[pl.st_items[pl.st_small] + 1] - pl.fo_ptr[pl.st_items[pl.st_small]] + 1 <= kSteinerSmallPins)
            ++pl.st_small;
    }
    pl.F = pl.fo_ptr[I];
    pl.fo_pin.resize(pl.F);
    pl.fo_node.resize(pl.F);
    pl.fo_cap.resize(pl.F);
    pl.fo_src.resize(pl.F);
    if (!pl.placed) {
        pl.rc_parent.resize(pl.rc_ptr[I]);
        pl.rc_R.resize(pl.rc_ptr[I]);
        pl.rc_C.resize(pl.rc_ptr[I]);
        pl.rc_src.resize(pl.rc_ptr[I]);
    }
    for (int32_t g = 0; g < I; ++g) {
        const int32_t n = drv_net[out_pin_of_item[g]];
        if (n < 0) continue;
        int32_t o = pl.fo_ptr[g];
        for (int32_t k = d->net_pin_ptr[n] + 1; k < d->net_pin_ptr[n + 1]; ++k, ++o) {
            const int32_t s = d->net_pin[k];
            pl.fo_pin[o] = pl.gpu_of[s];
            pl.fo_cap[o] = sink_cap(s);
            pl.fo_node[o] = pl.placed ? (k - d->net_pin_ptr[n]) : d->rc_pin_node[k];
            pl.fo_src[o] = s;
        }
        if (!pl.placed) {
            int32_t r = pl.rc_ptr[g];
            for (int32_t i = d->rc_ptr[n]; i < d->rc_ptr[n + 1]; ++i, ++r) {
                pl.rc_parent[r] = d->rc_parent[i];
                pl.rc_R[r] = d->rc_R[i];
                pl.rc_C[r] = d->rc_C[i];
                pl.rc_src[r] = i;
            }
        }
    }
    // ---- timing exceptions: the tag of every startpoint item (its PI or CK
    // pin's first group) and the setup multiplier of every (endpoint, tag)
    pl.item_tag.clear();
    pl.ep_mult.clear();
    pl.ep_off.clear();
    pl.pin_adv.clear();
    if (pl.Tg > 1) {
        const int32_t G = d->n_exc;
        std::vector<int32_t> base(G + 1, 1), nthru(G, 0);   // first tag and through sets of each group
        for (int32_t g = 0; g < G; ++g) {
            nthru[g] = d->exc_thru_ptr ? d->exc_thru_ptr[g + 1] - d->exc_thru_ptr[g] : 0;
            base[g + 1] = base[g] + nthru[g] + 1;
        }
        std::vector<int8_t> tag_of(P, 0);
        std::vector<int32_t> caller_of(P, 0);
        for (int32_t p = 0; p < P; ++p) caller_of[pl.gpu_of[p]] = p;
        for (int32_t g = 0; g < G; ++g) {
            REQUIRE(d->exc_from_ptr[g] >= 0 && d->exc_from_ptr[g] <= d->exc_from_ptr[g + 1] && d->exc_to_ptr[g] >= 0 &&
                        d->exc_to_ptr[g] <= d->exc_to_ptr[g + 1],
                    STA_EINVAL, "exception group %d: offsets not monotone", g);
            for (int32_t i = d->exc_from_ptr[g]; i < d->exc_from_ptr[g + 1]; ++i) {
                const int32_t p = d->exc_from[i];
                REQUIRE(p >= 0 && p < P && (d->pin_role[p] == kPinPI || d->pin_role[p] == kPinCK), STA_EINVAL,
                        "exception group %d: startpoint %d is not a PI or CK pin", g, p);
                if (!tag_of[p]) tag_of[p] = (int8_t)base[g];
            }
            for (int32_t i = d->exc_to_ptr[g]; i < d->exc_to_ptr[g + 1]; ++i) {
                const int32_t p = d->exc_to[i];
                REQUIRE(p >= 0 && p < P && (d->pin_role[p] == kPinD || d->pin_role[p] == kPinPO), STA_EINVAL,
                        "exception group %d: endpoint %d is not a D or PO pin", g, p);
            }
            REQUIRE(d->exc_action[g] >= 0 && d->exc_action[g] <= 3 && finite(d->exc_mult[g]) &&
                        (d->exc_action[g] != 1 || d->exc_mult[g] >= 1.f),
                    STA_EINVAL,
                    "exception group %d: action must be 0 (false path), 1 (multicycle, M >= 1), 2 (max delay) or "
                    "3 (min delay) with a finite value", g);
            // through set j + 1: the group's tag base + j moves on to base + j + 1 at its pins
            for (int32_t j = 0; j < nthru[g]; ++j) {
                const int32_t s = d->exc_thru_ptr[g] + j;
                REQUIRE(d->exc_thru_set_ptr[s] >= 0 && d->exc_thru_set_ptr[s] <= d->exc_thru_set_ptr[s + 1], STA_EINVAL,
                        "exception group %d: through set offsets not monotone", g);
                for (int32_t i = d->exc_thru_set_ptr[s]; i < d->exc_thru_set_ptr[s + 1]; ++i) {
                    const int32_t p = d->exc_thru_pin[i];
                    REQUIRE(p >= 0 && p < P && d->pin_role[p] == kPinIN, STA_EINVAL,
                            "exception group %d: through pin %d is not a gate input pin", g, p);
                    if (pl.pin_adv.empty()) pl.pin_adv.assign(P, 0u);
                    pl.pin_adv[pl.gpu_of[p]] |= 1u << (base[g] + j);
                }
            }
        }
        pl.item_tag.assign(pl.I, 0);
        for (int32_t g = 0; g < pl.I; ++g) {
            const int32_t t = pl.item_type[g];
            if (t < 0) pl.item_tag[g] = tag_of[caller_of[pl.item_pin0[g]]];
            else if (pl.type_kind[t] == 1) pl.item_tag[g] = tag_of[d->cell_pin[d->cell_pin_ptr[pl.item_cell[g]] + 1]];
        }
        // requirement of (endpoint, tag): late = mult * T + off[0] (mult = 0: off[0] alone), early = off[1];
        // default: flip-flop D T - setup and hold, output port T and 0
        pl.ep_mult.assign((size_t)pl.E * pl.Tg, 1.f);
        pl.ep_off.assign((size_t)pl.E * pl.Tg * 2, 0.f);
        for (int32_t e = 0; e < pl.E; ++e)
            for (int32_t t = 0; t < pl.Tg; ++t) {
                pl.ep_off[((size_t)e * pl.Tg + t) * 2] = pl.ep_is_d[e] ? -pl.setup : 0.f;
                pl.ep_off[((size_t)e * pl.Tg + t) * 2 + 1] = pl.ep_is_d[e] ? pl.hold : 0.f;
            }
        std::vector<uint8_t> in_to(P, 0);
        for (int32_t g = 0; g < G; ++g) {
            const bool all = d->exc_to_ptr[g] == d->exc_to_ptr[g + 1];
            const double v = d->exc_mult[g];
            for (int32_t i = d->exc_to_ptr[g]; i < d->exc_to_ptr[g + 1]; ++i) in_to[d->exc_to[i]] = 1;
            for (int32_t e = 0; e < pl.E; ++e) {   // the fully matched tag gets the action
                if (!all && !in_to[caller_of[pl.ep_pin[e]]]) continue;
                const size_t x = (size_t)e * pl.Tg + base[g] + nthru[g];
                const bool isd = pl.ep_is_d[e];
                switch (d->exc_action[g]) {
                case 0:   // false path: no check
                    pl.ep_mult[x] = 0.f;
                    pl.ep_off[2 * x] = INFINITY;
                    pl.ep_off[2 * x + 1] = -INFINITY;
                    break;
                case 1:   // multicycle: setup capture edge at M * T
                    pl.ep_mult[x] = (float)v;
                    break;
                case 2:   // max delay: setup capture edge at v
                    pl.ep_mult[x] = 0.f;
                    pl.ep_off[2 * x] = (float)(isd ? v - pl.setup : v);
                    break;
                default:  // min delay: hold edge at v
                    pl.ep_off[2 * x + 1] = (float)(isd ? v + pl.hold : v);
                    break;
                }
            }
            for (int32_t i = d->exc_to_ptr[g]; i < d->exc_to_ptr[g + 1]; ++i) in_to[d->exc_to[i]] = 0;
        }
    }
    // ---- RC nets too large for the shared-memory sweep
    pl.n_big_nets = 0;
    if (!pl.placed || pl.steiner)
        for (int32_t g = 0; g < I; ++g) pl.n_big_nets += pl.rc_ptr[g + 1] - pl.rc_ptr[g] > kColNodes;
    // ---- arc count
    pl.cell_arcs = 0;
    for (int32_t c = 0; c < C; ++c) {
        const int32_t t = d->cell_type[c];
        for (int s = 0; s < pl.type_nin[t]; ++s) pl.cell_arcs += pl.arc_sense[(size_t)t * 3 + s] != kSenseNone;
    }
}

}  // namespace

sta_status build_plan(const sta_design_desc *desc, Plan &plan, std::string &err)
{
    try {
        plan = Plan();
        build(desc, plan);
        return STA_OK;
    } catch (const Fail &f) {
        err = f.msg;
        return f.code;
    } catch (const std::bad_alloc &) {
        err = "host allocation failed";
        return STA_ENOMEM;
    }
}

namespace {

template <class T>
bool same_array(const T *a, const T *b, size_t n)
{
    if (a == b) return true;
    if (!a || !b) return false;
    return std::memcmp(a, b, n * sizeof(T)) == 0;
}

bool same_library(const sta_library &a, const sta_library &b)
{
    if (a.n_types != b.n_types || a.setup_ns != b.setup_ns || a.hold_ns != b.hold_ns || a.po_cap_pf != b.po_cap_pf)
        return false;
    const size_t T = (size_t)a.n_types;
    return same_array(a.type_nin, b.type_nin, T) && same_array(a.type_kind, b.type_kind, T) &&
           same_array(a.arc_sense, b.arc_sense, T * 3) && same_array(a.lut_idx1, b.lut_idx1, T * 84) &&
           same_array(a.lut_idx2, b.lut_idx2, T * 84) && same_array(a.lut_val, b.lut_val, T * 588) &&
           same_array(a.pin_cap, b.pin_cap, T * 4);
}

}  // namespace

sta_status build_batch_plan(const sta_design_desc *const *descs, int32_t n, Plan &plan, std::string &err)
{
    if (n < 1 || !descs) { err = "empty batch"; return STA_EINVAL; }
    for (int32_t i = 0; i < n; ++i) {
        if (!descs[i] || !descs[i]->lib) { err = "NULL descriptor in batch"; return STA_EINVAL; }
    }
    // timing exceptions: the groups of every design, pins offset, in one list
    // (a group's tag only travels on paths from its own design's startpoints,
    // so an empty endpoint list still reaches only that design's endpoints)
    int32_t G = 0;
    bool any_thru = false;
    for (int32_t i = 0; i < n; ++i) {
        if (descs[i]->n_exc < 0) { err = "negative n_exc"; return STA_EINVAL; }
        G += descs[i]->n_exc;
        any_thru = any_thru || (descs[i]->n_exc > 0 && descs[i]->exc_thru_ptr);
    }
    if (G > 7) { err = "at most 7 timing-exception groups over the whole batch"; return STA_EINVAL; }
    const sta_design_desc &d0 = *descs[0];
    const bool placed = d0.rc_ptr == nullptr;
    const int K = d0.n_corners;
    int64_t C = 0, P = 0, N = 0, NN = 0, NP = 0, CP = 0;
    for (int32_t i = 0; i < n; ++i) {
        const sta_design_desc &di = *descs[i];
        const bool ok = same_library(*di.lib, *d0.lib) && di.n_corners == K && (di.rc_ptr == nullptr) == placed &&
                        di.period_ns == d0.period_ns && di.clk_slew_ns == d0.clk_slew_ns &&
                        di.pi_at_ns == d0.pi_at_ns && di.pi_slew_ns == d0.pi_slew_ns &&
                        di.gamma_ns == d0.gamma_ns && di.r_per_um == d0.r_per_um && di.c_per_um == d0.c_per_um &&
                        di.net_model == d0.net_model && di.arnoldi_order == d0.arnoldi_order &&
                        di.wire_model == d0.wire_model && di.r_per_um_y == d0.r_per_um_y &&
                        di.c_per_um_y == d0.c_per_um_y &&
                        (K < 1 || K > 16 || (same_array(di.lut_scale, d0.lut_scale, (size_t)K) &&
                                             same_array(di.rc_scale, d0.rc_scale, (size_t)K)));
        if (!ok) {
            err = "design " + std::to_string(i) +
                  " differs from design 0 in library, corners, clock, parasitic kind or net model";
            return STA_EINVAL;
        }
        if (di.n_cells < 0 || di.n_pins < 0 || di.n_nets < 0) { err = "negative size"; return STA_EINVAL; }
        if ((di.n_cells > 0 && !di.cell_pin_ptr) || (di.n_nets > 0 && !di.net_pin_ptr) ||
            (!placed && di.n_nets > 0 && !di.rc_ptr)) {
            err = "NULL array in design " + std::to_string(i);
            return STA_EINVAL;
        }
        C += di.n_cells;
        P += di.n_pins;
        N += di.n_nets;
        CP += di.n_cells ? di.cell_pin_ptr[di.n_cells] : 0;
        NP += di.n_nets ? di.net_pin_ptr[di.n_nets] : 0;
        if (!placed) NN += di.n_nets ? di.rc_ptr[di.n_nets] : 0;
    }
    if (P > INT32_MAX / 2 || NP > INT32_MAX / 2 || NN > INT32_MAX / 2) { err = "batch too large"; return STA_EINVAL; }
    try {
        std::vector<int32_t> cell_type(C), cell_pin_ptr(C + 1, 0), cell_pin(CP), net_pin_ptr(N + 1, 0), net_pin(NP);
        std::vector<int8_t> pin_role(P);
        std::vector<int32_t> rc_ptr, rc_parent, rc_pin_node;
        std::vector<float> rc_R, rc_C, cell_xy, port_xy;
        if (!placed) {
            rc_ptr.assign(N + 1, 0);
            rc_parent.resize(NN);
            rc_R.resize(NN);
            rc_C.resize(NN);
            rc_pin_node.resize(NP);
        } else {
            cell_xy.resize(2 * C);
            port_xy.assign(2 * P, 0.f);
        }
        std::vector<int64_t> pin_off(n + 1, 0);
        std::vector<int32_t> xf_ptr(1, 0), xf, xt_ptr(1, 0), xt, xact, xth_ptr(1, 0), xth_set(1, 0), xth_pin;
        std::vector<float> xmult;
        int64_t c0 = 0, p0 = 0, n0 = 0, cp0 = 0, np0 = 0, r0 = 0;
        for (int32_t i = 0; i < n; ++i) {
            const sta_design_desc &di = *descs[i];
            if (di.n_exc > 0) {   // the checks build_plan makes, before the arrays are read here
                bool ok = di.exc_from_ptr && di.exc_to_ptr && di.exc_action && di.exc_mult &&
                          (!di.exc_thru_ptr || di.exc_thru_set_ptr);
                for (int32_t g = 0; ok && g < di.n_exc; ++g)
                    ok = di.exc_from_ptr[g] >= 0 && di.exc_from_ptr[g] <= di.exc_from_ptr[g + 1] &&
                         di.exc_to_ptr[g] >= 0 && di.exc_to_ptr[g] <= di.exc_to_ptr[g + 1] &&
                         (!di.exc_thru_ptr || (di.exc_thru_ptr[g] >= 0 && di.exc_thru_ptr[g] <= di.exc_thru_ptr[g + 1]));
                ok = ok && (di.exc_from || di.exc_from_ptr[di.n_exc] == 0) && (di.exc_to || di.exc_to_ptr[di.n_exc] == 0);
                if (ok && di.exc_thru_ptr)
                    for (int32_t sset = di.exc_thru_ptr[0]; ok && sset < di.exc_thru_ptr[di.n_exc]; ++sset)
                        ok = di.exc_thru_set_ptr[sset] >= 0 && di.exc_thru_set_ptr[sset] <= di.exc_thru_set_ptr[sset + 1] &&
                             (di.exc_thru_pin || di.exc_thru_set_ptr[sset + 1] == di.exc_thru_set_ptr[sset]);
                if (!ok) {
                    err = "exception arrays NULL or offsets not monotone in design " + std::to_string(i);
                    return STA_EINVAL;
                }
            }
            for (int32_t g = 0; g < di.n_exc; ++g) {
                for (int32_t k = di.exc_from_ptr[g]; k < di.exc_from_ptr[g + 1]; ++k)
                    xf.push_back((int32_t)(p0 + di.exc_from[k]));
                xf_ptr.push_back((int32_t)xf.size());
                for (int32_t k = di.exc_to_ptr[g]; k < di.exc_to_ptr[g + 1]; ++k) xt.push_back((int32_t)(p0 + di.exc_to[k]));
                xt_ptr.push_back((int32_t)xt.size());
                xact.push_back(di.exc_action[g]);
                xmult.push_back(di.exc_mult[g]);
                if (di.exc_thru_ptr)
                    for (int32_t sset = di.exc_thru_ptr[g]; sset < di.exc_thru_ptr[g + 1]; ++sset) {
                        for (int32_t k = di.exc_thru_set_ptr[sset]; k < di.exc_thru_set_ptr[sset + 1]; ++k)
                            xth_pin.push_back((int32_t)(p0 + di.exc_thru_pin[k]));
                        xth_set.push_back((int32_t)xth_pin.size());
                    }
                xth_ptr.push_back((int32_t)xth_set.size() - 1);
            }
            for (int32_t c = 0; c < di.n_cells; ++c) {
                cell_type[c0 + c] = di.cell_type[c];
                cell_pin_ptr[c0 + c + 1] = (int32_t)(cp0 + di.cell_pin_ptr[c + 1]);
            }
            for (int32_t k = 0; k < (di.n_cells ? di.cell_pin_ptr[di.n_cells] : 0); ++k)
                cell_pin[cp0 + k] = (int32_t)(p0 + di.cell_pin[k]);
            for (int32_t p = 0; p < di.n_pins; ++p) pin_role[p0 + p] = di.pin_role[p];
            for (int32_t m = 0; m < di.n_nets; ++m) net_pin_ptr[n0 + m + 1] = (int32_t)(np0 + di.net_pin_ptr[m + 1]);
            const int32_t np = di.n_nets ? di.net_pin_ptr[di.n_nets] : 0;
            for (int32_t k = 0; k < np; ++k) net_pin[np0 + k] = (int32_t)(p0 + di.net_pin[k]);
            if (!placed) {
                for (int32_t m = 0; m < di.n_nets; ++m) rc_ptr[n0 + m + 1] = (int32_t)(r0 + di.rc_ptr[m + 1]);
                const int32_t nn = di.n_nets ? di.rc_ptr[di.n_nets] : 0;
                for (int32_t k = 0; k < nn; ++k) {
                    rc_parent[r0 + k] = di.rc_parent[k];
                    rc_R[r0 + k] = di.rc_R[k];
                    rc_C[r0 + k] = di.rc_C[k];
                }
                for (int32_t k = 0; k < np; ++k) rc_pin_node[np0 + k] = di.rc_pin_node[k];
                r0 += nn;
            } else {
                for (int64_t k = 0; k < 2LL * di.n_cells; ++k) cell_xy[2 * c0 + k] = di.cell_xy ? di.cell_xy[k] : 0.f;
                if (di.port_xy)
                    for (int64_t k = 0; k < 2LL * di.n_pins; ++k) port_xy[2 * p0 + k] = di.port_xy[k];
            }
            c0 += di.n_cells;
            p0 += di.n_pins;
            n0 += di.n_nets;
            cp0 += di.n_cells ? di.cell_pin_ptr[di.n_cells] : 0;
            np0 += np;
            pin_off[i + 1] = p0;
        }
        sta_design_desc m = d0;
        m.n_cells = (int32_t)C;
        m.cell_type = cell_type.data();
        m.cell_pin_ptr = cell_pin_ptr.data();
        m.cell_pin = cell_pin.data();
        m.n_pins = (int32_t)P;
        m.pin_role = pin_role.data();
        m.n_nets = (int32_t)N;
        m.net_pin_ptr = net_pin_ptr.data();
        m.net_pin = net_pin.data();
        if (!placed) {
            m.rc_ptr = rc_ptr.data();
            m.rc_parent = rc_parent.data();
            m.rc_R = rc_R.data();
            m.rc_C = rc_C.data();
            m.rc_pin_node = rc_pin_node.data();
        } else {
            m.cell_xy = cell_xy.data();
            m.port_xy = port_xy.data();
        }
        m.n_exc = G;
        m.exc_from_ptr = xf_ptr.data();
        m.exc_from = xf.data();
        m.exc_to_ptr = xt_ptr.data();
        m.exc_to = xt.data();
        m.exc_action = xact.data();
        m.exc_mult = xmult.data();
        m.exc_thru_ptr = any_thru ? xth_ptr.data() : nullptr;
        m.exc_thru_set_ptr = any_thru ? xth_set.data() : nullptr;
        m.exc_thru_pin = any_thru ? xth_pin.data() : nullptr;
        sta_status st = build_plan(&m, plan, err);
        if (st != STA_OK) return st;
        // endpoints are in ascending merged pin id: split them by design
        plan.n_designs = n;
        plan.ep_design_ptr.assign(n + 1, 0);
        std::vector<int32_t> ep_caller(plan.E);
        {
            std::vector<int32_t> caller_of(P);
            for (int64_t p = 0; p < P; ++p) caller_of[plan.gpu_of[p]] = (int32_t)p;
            for (int32_t e = 0; e < plan.E; ++e) ep_caller[e] = caller_of[plan.ep_pin[e]];
        }
        for (int32_t i = 0, e = 0; i < n; ++i) {
            while (e < plan.E && ep_caller[e] < pin_off[i + 1]) ++e;
            plan.ep_design_ptr[i + 1] = e;
        }
        return STA_OK;
    } catch (const std::bad_alloc &) {
        err = "host allocation failed";
        return STA_ENOMEM;
    }
}

}  // namespace sta
