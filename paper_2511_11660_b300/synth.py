"""Seeded synthetic timing designs (inputs only; no timing arithmetic here).

The paper's benchmarks (TAU 2015 designs moved to 14 nm, ICCAD 2015
superblue, ISPD 2025; HeteroSTA Sec. IV, Tab. I-IV) are not available, so
every workload is generated from a seed with the shape the experiments use:
gate-level netlists of 10^3 - 10^7 cells, a flattened CSR netlist (Sec. III,
"Heterogeneous netlist database"), NLDM 7x7 tables per cell arc, RC trees
per net or pin positions plus unit R/C (Sec. III, "Parasitics (RC) inputs").

This module only draws numbers and lays them out; it computes no delay,
load, arrival or slack.  Both the GPU library and the FP64 oracle read the
dict it returns, which is why it lives on its own.

Design dict keys (all arrays numpy, C-contiguous):
  library  n_types, type_nin[T], type_kind[T], arc_sense[T*3],
           lut_idx1/lut_idx2[T*3*4*7] (slew ns / load pF axes),
           lut_val[T*3*4*49] (value[i_slew*7 + j_load]),
           pin_cap[T*4] pF, setup_ns, hold_ns, po_cap_pf
  netlist  n_cells, cell_type[n_cells], cell_pin_ptr[n_cells+1], cell_pin[],
           n_pins, pin_role[n_pins] (int8), n_nets, net_pin_ptr[n_nets+1],
           net_pin[] (driver first)
  RC       rc_ptr[n_nets+1], rc_parent[] (local, -1 at root), rc_R[] Ohm,
           rc_C[] fF, rc_pin_node[len(net_pin)] (local node of each entry)
  place    cell_xy[n_cells*2] um, port_xy[n_pins*2] um, r_per_um, c_per_um
  timing   period_ns, clk_slew_ns, pi_at_ns, pi_slew_ns, n_corners,
           lut_scale[K], rc_scale[K], gamma_ns
"""
from __future__ import annotations

import numpy as np

# pin roles
PI, PO, IN, OUT, D, CK, Q = 0, 1, 2, 3, 4, 5, 6
# arc senses
NONE, POS, NEG, NON, RISE = -1, 0, 1, 2, 3

TYPE_NAMES = ["INV", "BUF", "NAND2", "NOR2", "AOI21", "XOR2", "MUX2", "DFF"]
TYPE_NIN = [1, 1, 2, 2, 3, 2, 3, 2]
TYPE_KIND = [0, 0, 0, 0, 0, 0, 0, 1]
TYPE_SENSE = [
    [NEG, NONE, NONE],   # INV
    [POS, NONE, NONE],   # BUF
    [NEG, NEG, NONE],    # NAND2
    [NEG, NEG, NONE],    # NOR2
    [NEG, NEG, NEG],     # AOI21
    [NON, NON, NONE],    # XOR2
    [POS, POS, NON],     # MUX2 (A, B, select)
    [NONE, RISE, NONE],  # DFF (D check pin, CK -> Q on the rising edge)
]
N_BASE = len(TYPE_NAMES)
DFF_TYPE = 7

SLEW_AXIS = np.geomspace(0.005, 1.0, 7)   # ns
LOAD_AXIS = np.geomspace(0.001, 0.5, 7)   # pF


def make_library(seed: int = 0, noise: float = 0.02, fixed_delay: bool = False,
                 strengths: int = 1, strength_factor: float = 0.7) -> dict:
    """Eight cell types with 7x7 rise/fall delay and slew tables per arc.

    Each table holds a + b*slew + c*load + d*slew*load at the axis points,
    times (1 + U(-noise, noise)).  a > 0 and b, c, d >= 0, so tables are
    positive and non-decreasing in both axes.  ``fixed_delay`` zeroes b and d
    of the delay tables and the noise, so every cell delay depends on load
    only.  ``strengths`` > 1 appends copies of the eight types whose table
    values are multiplied by ``strength_factor`` per step (drive strengths)."""
    rng = np.random.default_rng(seed)
    T = N_BASE * strengths
    idx1 = np.zeros((T, 3, 4, 7), np.float32)
    idx2 = np.zeros((T, 3, 4, 7), np.float32)
    val = np.zeros((T, 3, 4, 49), np.float32)
    idx1[:] = SLEW_AXIS.astype(np.float32)
    idx2[:] = LOAD_AXIS.astype(np.float32)
    s = SLEW_AXIS.astype(np.float32).astype(np.float64)[:, None]
    l = LOAD_AXIS.astype(np.float32).astype(np.float64)[None, :]
    base = np.zeros((N_BASE, 3, 4, 49), np.float64)
    for t in range(N_BASE):
        for slot in range(3):
            if TYPE_SENSE[t][slot] == NONE:
                continue
            for tb in range(4):
                if tb < 2:   # delay tables
                    a = rng.uniform(0.040, 0.080) if t == DFF_TYPE else rng.uniform(0.010, 0.030)
                    b, c, d = rng.uniform(0.05, 0.20), rng.uniform(1.0, 3.0), rng.uniform(0.1, 0.5)
                    if fixed_delay:
                        b = d = 0.0
                else:        # output slew tables
                    a = rng.uniform(0.005, 0.015)
                    b, c, d = rng.uniform(0.02, 0.10), rng.uniform(2.0, 5.0), rng.uniform(0.1, 0.5)
                v = a + b * s + c * l + d * s * l
                if noise > 0 and not fixed_delay:
                    v = v * (1.0 + rng.uniform(-noise, noise, size=v.shape))
                base[t, slot, tb] = v.reshape(-1)
    for k in range(strengths):
        val[k * N_BASE:(k + 1) * N_BASE] = (base * (strength_factor ** k)).astype(np.float32)
    pin_cap = np.zeros((T, 4), np.float32)
    caps = rng.uniform(0.001, 0.004, size=(N_BASE, 4))
    for t in range(N_BASE):
        for slot in range(TYPE_NIN[t]):
            pin_cap[[t + k * N_BASE for k in range(strengths)], slot] = caps[t, slot]
    sense = np.array(TYPE_SENSE * strengths, np.int32).reshape(-1)
    return dict(
        n_types=T,
        type_nin=np.array(TYPE_NIN * strengths, np.int32),
        type_kind=np.array(TYPE_KIND * strengths, np.int32),
        arc_sense=sense,
        lut_idx1=idx1.reshape(-1), lut_idx2=idx2.reshape(-1), lut_val=val.reshape(-1),
        pin_cap=pin_cap.reshape(-1),
        setup_ns=0.03, hold_ns=0.01, po_cap_pf=0.002,
    )


def _csr_from_groups(keys: np.ndarray, n_groups: int):
    order = np.argsort(keys, kind="stable")
    counts = np.bincount(keys, minlength=n_groups)
    ptr = np.zeros(n_groups + 1, np.int64)
    np.cumsum(counts, out=ptr[1:])
    return order, ptr


def make_design(n_cells: int, depth: int, seed: int = 0, lib: dict | None = None,
                rc_nodes: tuple[int, int] = (2, 12), fanout_mean: float = 2.5,
                dff_frac: float = 0.10, pi_frac: float = 0.02, po_frac: float = 0.2, placed: bool = False,
                die_um: float = 1000.0, r_per_um: float = 0.1, c_per_um: float = 0.2,
                period_ns: float = 1.0, n_corners: int = 1, lut_scale=None, rc_scale=None,
                gamma_ns: float = 0.0, base_types_only: bool = True, placement: str = "uniform",
                local_um: float = 20.0) -> dict:
    """A random levelised netlist of ``n_cells`` cells and logic depth ``depth``.

    * 10% of cells are DFFs; the rest draw uniformly from the 7 gate types.
    * Gates are spread evenly over levels 1..depth.  Input 0 of a gate at
      level k is driven from level k-1 (which fixes the depth); the other
      inputs from any level below k.  Level 0 holds the primary inputs and
      the DFF Q pins.  DFF D pins are driven from any level.
    * Every driver draws a weight from a geometric law of mean
      ``fanout_mean`` and is picked with probability proportional to it.
    * A cell output nobody picked drives a primary output (all last-level
      outputs become POs); ``po_frac * n_cells`` further cell outputs get an
      extra primary output (observation points).  No primary output is fed
      straight from a primary input (its hold slack would be the bare net
      delay, inside the tolerance of zero); a primary input nobody picked
      has no sinks.
    * RC per net: ``rc_nodes`` inclusive node-count range, parent of node i
      uniform in [0, i), R ~ U(5, 50) Ohm (root 0), C ~ U(0.5, 5) fF; each
      sink sits on a uniform non-root node.
    * ``placed`` draws cell and port positions uniformly in the die
      (``placement="uniform"``: every net spans the die, so path delays run
      to ~100 ns); ``placement="local"`` then places, level by level, each
      gate at the mean of its input drivers plus N(0, local_um^2) per axis
      and each primary output at its driver plus the same noise (flip-flops
      and primary inputs stay uniform), so nets are tens of um long.
    Cell ids are shuffled, so id order says nothing about level order."""
    rng = np.random.default_rng(seed)
    if lib is None:
        lib = make_library(seed)
    n_dff = int(round(dff_frac * n_cells)) if n_cells >= 10 else min(1, n_cells // 2)
    n_comb = n_cells - n_dff
    depth = max(1, min(depth, n_comb)) if n_comb > 0 else 0
    n_pi = max(1, int(round(pi_frac * n_cells)))

    comb_type = rng.integers(0, 7, size=n_comb).astype(np.int32)
    comb_level = (1 + (np.arange(n_comb, dtype=np.int64) * depth) // max(n_comb, 1)).astype(np.int64)

    # drivers in level order: PIs, DFF Qs (level 0), then gate outputs
    n_drv = n_pi + n_dff + n_comb
    drv_level = np.concatenate([np.zeros(n_pi + n_dff, np.int64), comb_level])
    w = rng.geometric(1.0 / fanout_mean, size=n_drv).astype(np.float64)
    cum = np.cumsum(w)
    lvl_end = np.searchsorted(drv_level, np.arange(depth + 1), side="right")  # drivers with level <= k
    lvl_beg = np.concatenate([[0], lvl_end[:-1]])

    def cum_at(i):  # total weight of drivers [0, i)
        i = np.asarray(i)
        return np.where(i > 0, cum[np.maximum(i - 1, 0)], 0.0)

    def pick(lo_idx, hi_idx):  # weighted draw of one driver in [lo_idx, hi_idx) per row
        lo, hi = cum_at(lo_idx), cum_at(hi_idx)
        u = lo + rng.random(len(lo)) * (hi - lo)
        return np.minimum(np.searchsorted(cum, u, side="right"), np.asarray(hi_idx) - 1)

    nin_comb = np.array(TYPE_NIN, np.int64)[comb_type]
    # gate input slots: (gate, slot)
    g_of_slot = np.repeat(np.arange(n_comb), nin_comb)
    slot_of = np.arange(len(g_of_slot)) - np.repeat(np.cumsum(nin_comb) - nin_comb, nin_comb)
    k_of = comb_level[g_of_slot]
    first = slot_of == 0
    lo = np.where(first, lvl_beg[np.maximum(k_of - 1, 0)], 0)
    hi = lvl_end[np.maximum(k_of - 1, 0)]
    slot_drv = pick(lo, hi) if len(g_of_slot) else np.zeros(0, np.int64)
    d_drv = pick(np.zeros(n_dff, np.int64), np.full(n_dff, n_drv, np.int64)) if n_dff else np.zeros(0, np.int64)

    # ---- cells, shuffled ids; pins contiguous per cell (inputs, then output)
    cell_type_lin = np.concatenate([np.full(n_dff, DFF_TYPE, np.int32), comb_type])
    perm = rng.permutation(n_cells)           # linear cell index -> cell id
    cell_type = np.empty(n_cells, np.int32)
    cell_type[perm] = cell_type_lin
    npins_cell = np.array(TYPE_NIN, np.int64)[cell_type] + 1
    cell_pin_ptr = np.zeros(n_cells + 1, np.int64)
    np.cumsum(npins_cell, out=cell_pin_ptr[1:])
    n_cell_pins = int(cell_pin_ptr[-1])
    lin_pin0 = cell_pin_ptr[perm]             # first pin of each linear cell
    # DFF linear cells 0..n_dff-1: pins D, CK, Q; gates n_dff.. : inputs, output
    dff_pin0 = lin_pin0[:n_dff]
    gate_pin0 = lin_pin0[n_dff:]
    gate_out = gate_pin0 + nin_comb
    drv_pin = np.concatenate([
        n_cell_pins + np.arange(n_pi),        # PI pins follow the cell pins
        dff_pin0 + 2,                         # DFF Q
        gate_out,
    ]).astype(np.int64)

    # sinks: gate inputs, DFF D pins, then POs for unpicked drivers
    sink_pin = np.concatenate([gate_pin0[g_of_slot] + slot_of, dff_pin0]).astype(np.int64)
    sink_drv = np.concatenate([slot_drv, d_drv]).astype(np.int64)
    fan = np.bincount(sink_drv, minlength=n_drv)
    # A cell output nobody picked drives a primary output; a primary input
    # nobody picked stays a port without sinks.  No primary output hangs
    # straight off a primary input: such a feed-through's hold slack would be
    # its net delay alone (~1e-4 ns), inside the FP32 tolerance of zero, and
    # its hold violation flag would not be well defined.
    lonely = np.nonzero(fan[n_pi:] == 0)[0] + n_pi
    # observation points: extra primary outputs on random cell outputs
    n_tap = int(round(po_frac * n_cells))
    n_cell_drv = n_drv - n_pi
    taps = (rng.choice(n_cell_drv, size=min(n_tap, n_cell_drv), replace=False) + n_pi if n_tap > 0 and n_cell_drv > 0
            else np.zeros(0, np.int64))
    lonely = np.concatenate([lonely, np.setdiff1d(taps, lonely)])
    n_po = len(lonely)
    po_pin = n_cell_pins + n_pi + np.arange(n_po)
    sink_pin = np.concatenate([sink_pin, po_pin])
    sink_drv = np.concatenate([sink_drv, lonely])
    n_pins = n_cell_pins + n_pi + n_po

    pin_role = np.empty(n_pins, np.int8)
    slot_in_cell = np.arange(n_cell_pins) - np.repeat(cell_pin_ptr[:-1], npins_cell)
    ctype_of_pin = np.repeat(cell_type, npins_cell)
    is_dff_pin = ctype_of_pin == DFF_TYPE
    nin_of_pin = np.array(TYPE_NIN, np.int64)[ctype_of_pin]
    role_cell = np.where(slot_in_cell == nin_of_pin, OUT, IN)
    role_cell = np.where(is_dff_pin & (slot_in_cell == 0), D, role_cell)
    role_cell = np.where(is_dff_pin & (slot_in_cell == 1), CK, role_cell)
    role_cell = np.where(is_dff_pin & (slot_in_cell == 2), Q, role_cell)
    pin_role[:n_cell_pins] = role_cell
    pin_role[n_cell_pins:n_cell_pins + n_pi] = PI
    pin_role[n_cell_pins + n_pi:] = PO

    # nets: one per driver, in shuffled order; sinks shuffled inside a net
    net_of_drv = rng.permutation(n_drv)
    key = net_of_drv[sink_drv]
    shuffle = rng.permutation(len(sink_pin))
    key_s, sink_s = key[shuffle], sink_pin[shuffle]
    order, _ = _csr_from_groups(key_s, n_drv)
    sinks_sorted = sink_s[order]
    fan_net = np.bincount(key_s, minlength=n_drv)
    net_pin_ptr = np.zeros(n_drv + 1, np.int64)
    np.cumsum(fan_net + 1, out=net_pin_ptr[1:])
    net_pin = np.empty(int(net_pin_ptr[-1]), np.int64)
    drv_of_net = np.empty(n_drv, np.int64)
    drv_of_net[net_of_drv] = drv_pin
    net_pin[net_pin_ptr[:-1]] = drv_of_net
    is_sink_slot = np.ones(len(net_pin), bool)
    is_sink_slot[net_pin_ptr[:-1]] = False
    net_pin[is_sink_slot] = sinks_sorted

    cell_pin = np.arange(n_cell_pins, dtype=np.int64)
    d = dict(lib)
    d.update(n_cells=n_cells, cell_type=cell_type, cell_pin_ptr=cell_pin_ptr.astype(np.int32),
             cell_pin=cell_pin.astype(np.int32), n_pins=n_pins, pin_role=pin_role,
             n_nets=n_drv, net_pin_ptr=net_pin_ptr.astype(np.int32), net_pin=net_pin.astype(np.int32))

    # ---- RC trees
    lo_n, hi_n = rc_nodes
    nn = rng.integers(lo_n, hi_n + 1, size=n_drv).astype(np.int64)
    rc_ptr = np.zeros(n_drv + 1, np.int64)
    np.cumsum(nn, out=rc_ptr[1:])
    tot = int(rc_ptr[-1])
    local = np.arange(tot) - np.repeat(rc_ptr[:-1], nn)
    parent = np.floor(rng.random(tot) * local).astype(np.int64)
    parent[local == 0] = -1
    R = rng.uniform(5.0, 50.0, size=tot).astype(np.float32)
    R[local == 0] = 0.0
    Cw = rng.uniform(0.5, 5.0, size=tot).astype(np.float32)
    net_of_entry = np.repeat(np.arange(n_drv), np.diff(net_pin_ptr))
    nn_entry = nn[net_of_entry]
    pin_node = 1 + np.floor(rng.random(len(net_pin)) * (nn_entry - 1)).astype(np.int64)
    pin_node[net_pin_ptr[:-1]] = 0
    d.update(rc_ptr=rc_ptr.astype(np.int32), rc_parent=parent.astype(np.int32), rc_R=R, rc_C=Cw,
             rc_pin_node=pin_node.astype(np.int32))

    # ---- placement (always drawn so the stream of draws does not depend on it)
    cell_xy = rng.uniform(0.0, die_um, size=(n_cells, 2)).astype(np.float32)
    port_xy = np.zeros((n_pins, 2), np.float32)
    ports = np.nonzero((pin_role == PI) | (pin_role == PO))[0]
    port_xy[ports] = rng.uniform(0.0, die_um, size=(len(ports), 2)).astype(np.float32)
    if placement == "local":
        # driver positions: PIs (ports), DFF Qs (their cells), gate outputs (their cells)
        cell_of_lin = perm                                     # linear cell -> cell id
        drv_xy = np.concatenate([port_xy[n_cell_pins:n_cell_pins + n_pi],
                                 cell_xy[cell_of_lin[:n_dff]],
                                 cell_xy[cell_of_lin[n_dff:]]]).astype(np.float64)
        noise = rng.normal(0.0, local_um, size=(n_comb + n_po, 2))
        gate_first = np.cumsum(nin_comb) - nin_comb
        for k in range(1, depth + 1):
            gs = np.nonzero(comb_level == k)[0]
            if len(gs) == 0:
                continue
            acc = np.zeros((len(gs), 2))
            for j in range(3):
                has = nin_comb[gs] > j
                acc[has] += drv_xy[slot_drv[gate_first[gs[has]] + j]]
            drv_xy[n_pi + n_dff + gs] = np.clip(acc / nin_comb[gs][:, None] + noise[gs], 0.0, die_um)
        cell_xy[cell_of_lin[n_dff:]] = drv_xy[n_pi + n_dff:].astype(np.float32)
        port_xy[po_pin] = np.clip(drv_xy[lonely] + noise[n_comb:], 0.0, die_um).astype(np.float32)
    d.update(cell_xy=cell_xy.reshape(-1), port_xy=port_xy.reshape(-1), r_per_um=r_per_um,
             c_per_um=c_per_um, placed=placed)
    if placed:
        for k in ("rc_ptr", "rc_parent", "rc_R", "rc_C", "rc_pin_node"):
            d[k] = None

    d.update(period_ns=period_ns, clk_slew_ns=0.02, pi_at_ns=0.0, pi_slew_ns=0.02,
             n_corners=n_corners,
             lut_scale=np.asarray(lut_scale if lut_scale is not None else [1.0] * n_corners, np.float32),
             rc_scale=np.asarray(rc_scale if rc_scale is not None else [1.0] * n_corners, np.float32),
             gamma_ns=gamma_ns, depth=depth, seed=seed)
    return d


def exception_groups(d: dict, rng, n_groups: int, div_from: int = 3, div_to: int = 2, max_thru: int = 0,
                     div_thru: int = 8, actions=None) -> dict:
    """Random timing-exception groups for design ``d``: each group takes a
    random 1/div_from of the startpoints (PI and CK pins) and, with probability
    0.7, a random 1/div_to of the endpoints (D and PO pins; otherwise an empty
    list, i.e. every endpoint); its action is a false path or a multicycle
    with M in {2, 3}.  With max_thru > 0 each group also gets 0..max_thru
    ordered through sets, each a random 1/div_thru of the gate input pins.
    With ``actions`` (a tuple of codes) each group draws its action from it
    instead: 0 false path, 1 multicycle (M in {2, 3}), 2 max delay (a value
    uniform in [0.5, 1.5] periods), 3 min delay (uniform in [0, 0.3]
    periods; the period is d["period_ns"], else 1 ns).  Returned as the
    design keys exc_*."""
    role = np.asarray(d["pin_role"])
    starts = np.nonzero((role == PI) | (role == CK))[0]
    ends = np.nonzero((role == D) | (role == PO))[0]
    ins = np.nonzero(role == IN)[0]
    fp, fr, tp, to, act, mult = [0], [], [0], [], [], []
    thp, tsp, tpin = [0], [0], []
    for _ in range(n_groups):
        for _ in range(int(rng.integers(0, max_thru + 1)) if max_thru > 0 else 0):
            tpin += list(rng.choice(ins, size=max(1, len(ins) // div_thru), replace=False))
            tsp.append(len(tpin))
        thp.append(len(tsp) - 1)
        fr += list(rng.choice(starts, size=max(1, len(starts) // div_from), replace=False))
        fp.append(len(fr))
        if rng.random() < 0.7:
            to += list(rng.choice(ends, size=max(1, len(ends) // div_to), replace=False))
        tp.append(len(to))
        if actions is None:
            act.append(int(rng.random() < 0.5))
            mult.append(float(rng.integers(2, 4)))
        else:
            a = int(actions[int(rng.integers(0, len(actions)))])
            T = float(d.get("period_ns", 1.0))
            act.append(a)
            mult.append(float(rng.integers(2, 4)) if a == 1 else
                        T * float(rng.uniform(0.5, 1.5)) if a == 2 else T * float(rng.uniform(0.0, 0.3)) if a == 3
                        else 1.0)
    out = dict(exc_from_ptr=np.array(fp, np.int32), exc_from=np.array(fr, np.int32),
               exc_to_ptr=np.array(tp, np.int32), exc_to=np.array(to, np.int32),
               exc_action=np.array(act, np.int32), exc_mult=np.array(mult, np.float32))
    if max_thru > 0:
        out.update(exc_thru_ptr=np.array(thp, np.int32), exc_thru_set_ptr=np.array(tsp, np.int32),
                   exc_thru_pin=np.array(tpin, np.int32))
    return out


def design_stats(d: dict) -> dict:
    """Counts of the realised design (arcs are counted once, any rf/el/corner)."""
    role = np.asarray(d["pin_role"])
    nin = np.asarray(d["type_nin"])[np.asarray(d["cell_type"])]
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)[np.asarray(d["cell_type"])]
    cell_arcs = int((sense != NONE).sum())
    net_arcs = int(len(d["net_pin"]) - d["n_nets"])
    n_rc = int(d["rc_ptr"][-1]) if d.get("rc_ptr") is not None else int(len(d["net_pin"]))
    return dict(cells=int(d["n_cells"]), pins=int(d["n_pins"]), nets=int(d["n_nets"]),
                cell_arcs=cell_arcs, net_arcs=net_arcs, arcs=cell_arcs + net_arcs,
                rc_nodes=n_rc, endpoints=int(((role == D) | (role == PO)).sum()),
                pis=int((role == PI).sum()), pos=int((role == PO).sum()),
                mean_fanout=float(net_arcs / max(int(d["n_nets"]), 1)), cell_inputs=int(nin.sum()))


# ---------------------------------------------------------------- workloads

def lut_corners():
    """Four corners: LUT values x {0.9, 1.0, 1.1, 1.25}, wire R and C x
    {0.95, 1.0, 1.05, 1.15}."""
    return [0.9, 1.0, 1.1, 1.25], [0.95, 1.0, 1.05, 1.15]


def workload(name: str, seed: int = 0, **over) -> dict:
    """Named workloads: 'tiny' (2,000 cells, depth 30, RC trees of 2-12
    nodes), 'scale' (1M cells, depth 150, 2-10 nodes), 'mid' (the same at
    200k cells, for profiler captures), 'diff' (200k cells
    placed in a 1000 um die, star RC from positions, gamma 0.01 ns),
    'steiner' / 'steiner_mid' (1M / 200k cells placed locally in a 1000 um
    die, Steiner-tree RC from positions) and 'large' (10M cells, depth 400,
    placed, 4 corners, 2 drive strengths)."""
    steiner = name in ("steiner", "steiner_mid")
    if name == "tiny":
        kw = dict(n_cells=2000, depth=30, rc_nodes=(2, 12))
    elif name == "scale":
        kw = dict(n_cells=1_000_000, depth=150, rc_nodes=(2, 10))
    elif name == "mid":
        kw = dict(n_cells=200_000, depth=150, rc_nodes=(2, 10))
    elif name == "diff":
        kw = dict(n_cells=200_000, depth=150, rc_nodes=(2, 10), placed=True, gamma_ns=0.01)
    elif steiner:
        kw = dict(n_cells=1_000_000 if name == "steiner" else 200_000, depth=150, placed=True, placement="local")
    elif name == "large":
        ls, rs = lut_corners()
        kw = dict(n_cells=10_000_000, depth=400, rc_nodes=(2, 10), placed=True, gamma_ns=0.01,
                  n_corners=4, lut_scale=ls, rc_scale=rs, lib=make_library(seed, strengths=2))
    else:
        raise ValueError(name)
    kw.update(over)
    d = make_design(seed=seed, **kw)
    if steiner:
        d["wire_model"] = 1   # rectilinear Steiner trees rebuilt from the positions at every update
    return d


def batch_workload(seed: int = 0, n_designs: int = 64, lo: int = 5_000, hi: int = 500_000, depth: int = 150,
                   n_corners: int = 4, period_ns: float = 11.0) -> list:
    """Independent designs with cell counts log-uniform in [lo, hi], all on
    one library, with the four corners of ``lut_corners`` and one clock."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_designs)).astype(np.int64)
    lib = make_library(seed)
    ls, rs = lut_corners()
    ls, rs = ls[:n_corners], rs[:n_corners]
    return [make_design(int(n), depth, seed=seed * 1000 + i + 1, lib=lib, rc_nodes=(2, 10), n_corners=n_corners,
                        lut_scale=ls, rc_scale=rs, period_ns=period_ns) for i, n in enumerate(sizes)]


class Builder:
    """Hand-built netlists for small exact cases.

    >>> b = Builder(make_library(0))
    >>> a = b.pi(); x = b.cell("INV", [a]); b.po(x)
    >>> d = b.design(period_ns=1.0)
    Each ``cell`` input names a driver pin; ``rc`` per net defaults to a
    two-node tree (root + one node holding all sinks) with the given R, C."""

    def __init__(self, lib: dict):
        self.lib = lib
        self.cells = []      # (type, [driver pins])
        self.pins_role = []
        self.cell_pins = []
        self.drv_sinks = {}  # driver pin -> list of sink pins
        self.net_rc = {}     # driver pin -> (parent, R, C, node_of_sink dict)
        self.xy = {}

    def _new_pin(self, role):
        self.pins_role.append(role)
        return len(self.pins_role) - 1

    def pi(self, xy=(0.0, 0.0)):
        p = self._new_pin(PI)
        self.xy[p] = xy
        return p

    def po(self, drv, xy=(0.0, 0.0)):
        p = self._new_pin(PO)
        self.drv_sinks.setdefault(drv, []).append(p)
        self.xy[p] = xy
        return p

    def cell(self, tname, inputs, xy=(0.0, 0.0)):
        t = TYPE_NAMES.index(tname) if isinstance(tname, str) else int(tname)
        nin = int(self.lib["type_nin"][t])
        pins = []
        if t % N_BASE == DFF_TYPE:
            dpin, ck, q = self._new_pin(D), self._new_pin(CK), self._new_pin(Q)
            pins = [dpin, ck, q]
            self.drv_sinks.setdefault(inputs[0], []).append(dpin)
            out = q
        else:
            assert len(inputs) == nin
            for drv in inputs:
                p = self._new_pin(IN)
                pins.append(p)
                self.drv_sinks.setdefault(drv, []).append(p)
            out = self._new_pin(OUT)
            pins.append(out)
        self.cells.append(t)
        self.cell_pins.append(pins)
        self.xy[("cell", len(self.cells) - 1)] = xy
        return out

    def set_rc(self, drv, parent, R, C, node_of_sink):
        self.net_rc[drv] = (list(parent), list(R), list(C), dict(node_of_sink))

    def design(self, period_ns=1.0, default_R=10.0, default_C=1.0, n_corners=1, lut_scale=None,
               rc_scale=None, gamma_ns=0.0, placed=False, r_per_um=0.1, c_per_um=0.2) -> dict:
        d = dict(self.lib)
        n_cells = len(self.cells)
        cell_pin_ptr = np.zeros(n_cells + 1, np.int32)
        cell_pin_ptr[1:] = np.cumsum([len(p) for p in self.cell_pins])
        cell_pin = np.array([p for ps in self.cell_pins for p in ps], np.int32)
        drivers = [p for p in range(len(self.pins_role)) if p in self.drv_sinks]
        net_pin_ptr = [0]
        net_pin, rc_ptr, rc_parent, rc_R, rc_C, rc_pin_node = [], [0], [], [], [], []
        for drv in drivers:
            sinks = self.drv_sinks[drv]
            net_pin += [drv] + sinks
            net_pin_ptr.append(len(net_pin))
            if drv in self.net_rc:
                par, R, Cc, nos = self.net_rc[drv]
            else:
                par, R, Cc, nos = [-1, 0], [0.0, default_R], [0.0, default_C], {s: 1 for s in sinks}
            rc_parent += par
            rc_R += R
            rc_C += Cc
            rc_ptr.append(rc_ptr[-1] + len(par))
            rc_pin_node += [0] + [nos[s] for s in sinks]
        n_pins = len(self.pins_role)
        cell_xy = np.array([self.xy[("cell", c)] for c in range(n_cells)], np.float32).reshape(-1)
        port_xy = np.zeros((n_pins, 2), np.float32)
        for p in range(n_pins):
            if p in self.xy:
                port_xy[p] = self.xy[p]
        d.update(n_cells=n_cells, cell_type=np.array(self.cells, np.int32), cell_pin_ptr=cell_pin_ptr,
                 cell_pin=cell_pin, n_pins=n_pins, pin_role=np.array(self.pins_role, np.int8),
                 n_nets=len(drivers), net_pin_ptr=np.array(net_pin_ptr, np.int32),
                 net_pin=np.array(net_pin, np.int32),
                 rc_ptr=np.array(rc_ptr, np.int32), rc_parent=np.array(rc_parent, np.int32),
                 rc_R=np.array(rc_R, np.float32), rc_C=np.array(rc_C, np.float32),
                 rc_pin_node=np.array(rc_pin_node, np.int32),
                 cell_xy=cell_xy, port_xy=port_xy.reshape(-1), r_per_um=r_per_um, c_per_um=c_per_um,
                 period_ns=period_ns, clk_slew_ns=0.02, pi_at_ns=0.0, pi_slew_ns=0.02,
                 n_corners=n_corners,
                 lut_scale=np.asarray(lut_scale or [1.0] * n_corners, np.float32),
                 rc_scale=np.asarray(rc_scale or [1.0] * n_corners, np.float32),
                 gamma_ns=gamma_ns, placed=placed)
        if placed:
            for k in ("rc_ptr", "rc_parent", "rc_R", "rc_C", "rc_pin_node"):
                d[k] = None
        return d
