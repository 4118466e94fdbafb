"""Independent re-derivations used to pin the oracle (tests only).

Nothing here calls the oracle or the GPU library.  Each routine computes a
quantity from a different formula than the oracle uses:

* Elmore delay and second moment from shared-path resistances
  (D_i = sum_j R_ij C_j, beta_i = sum_j R_ij C_j D_j, R_ij = resistance of the
  common part of the root->i and root->j paths) instead of the oracle's
  two-sweep recurrences;
* loads as plain sums of capacitances;
* NLDM values by direct bilinear interpolation written out here;
* arrival times by enumerating every path (no max/min merge until the end).
"""
from __future__ import annotations

import numpy as np

PI, PO, IN, OUT, D, CK, Q = 0, 1, 2, 3, 4, 5, 6
NONE, POS, NEG, NON, RISE = -1, 0, 1, 2, 3


def shared_path_moments(parent, R, C):
    """Elmore D and beta of every node by the shared-resistance sums."""
    n = len(parent)
    anc = []
    for i in range(n):
        path, k = set(), i
        while k > 0:
            path.add(k)
            k = parent[k]
        anc.append(path)
    Rsh = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            Rsh[i, j] = sum(R[k] for k in anc[i] & anc[j])
    Dm = Rsh @ np.asarray(C, float)
    beta = Rsh @ (np.asarray(C, float) * Dm)
    return Dm, beta


def bilinear(idx1, idx2, val, s, l):
    idx1 = np.asarray(idx1, float)
    idx2 = np.asarray(idx2, float)
    v = np.asarray(val, float).reshape(7, 7)
    i = int(np.clip(np.searchsorted(idx1, s, side="right") - 1, 0, 5))
    j = int(np.clip(np.searchsorted(idx2, l, side="right") - 1, 0, 5))
    t = (s - idx1[i]) / (idx1[i + 1] - idx1[i])
    u = (l - idx2[j]) / (idx2[j + 1] - idx2[j])
    return ((1 - t) * (1 - u) * v[i, j] + t * (1 - u) * v[i + 1, j]
            + (1 - t) * u * v[i, j + 1] + t * u * v[i + 1, j + 1])


class Net:
    """Per-net parasitic quantities computed independently."""

    def __init__(self, d, corner=0):
        f = float(np.asarray(d["rc_scale"])[corner])
        role = np.asarray(d["pin_role"])
        cell_of = -np.ones(d["n_pins"], int)
        slot_of = -np.ones(d["n_pins"], int)
        cpp = np.asarray(d["cell_pin_ptr"])
        cp = np.asarray(d["cell_pin"])
        for c in range(d["n_cells"]):
            for k in range(cpp[c], cpp[c + 1]):
                cell_of[cp[k]] = c
                slot_of[cp[k]] = k - cpp[c]
        self.cell_of, self.slot_of = cell_of, slot_of
        pin_cap = np.asarray(d["pin_cap"]).reshape(-1, 4)
        ctype = np.asarray(d["cell_type"])

        def cap(p):
            if role[p] == PO:
                return float(d["po_cap_pf"])
            return float(pin_cap[ctype[cell_of[p]], slot_of[p]])

        self.cap = cap
        if d.get("cell_xy") is not None:
            cxy = np.asarray(d["cell_xy"]).reshape(-1, 2)
            pxy_ = np.asarray(d["port_xy"]).reshape(-1, 2)
            self.pos = lambda p: tuple(float(v) for v in (cxy[cell_of[p]] if cell_of[p] >= 0 else pxy_[p]))
        self.load, self.Dns, self.Vns, self.driver = {}, {}, {}, {}
        npp = np.asarray(d["net_pin_ptr"])
        npn = np.asarray(d["net_pin"])
        for n in range(d["n_nets"]):
            b, e = npp[n], npp[n + 1]
            drv = int(npn[b])
            sinks = [int(s) for s in npn[b + 1:e]]
            if d.get("rc_ptr") is not None:
                r0, r1 = d["rc_ptr"][n], d["rc_ptr"][n + 1]
                par = [int(x) for x in d["rc_parent"][r0:r1]]
                R = [0.0] + [f * float(x) for x in d["rc_R"][r0 + 1:r1]]
                Cn = [f * float(x) for x in d["rc_C"][r0:r1]]
                node = {s: int(d["rc_pin_node"][b + 1 + k]) for k, s in enumerate(sinks)}
                for s in sinks:
                    Cn[node[s]] += 1e3 * cap(s)
            else:
                xy = np.asarray(d["cell_xy"]).reshape(-1, 2)
                pxy = np.asarray(d["port_xy"]).reshape(-1, 2)

                def pos(p):
                    return xy[cell_of[p]] if cell_of[p] >= 0 else pxy[p]

                par, R, Cn, node = [-1], [0.0], [0.0], {}
                for k, s in enumerate(sinks):
                    L = float(np.abs(pos(drv).astype(float) - pos(s).astype(float)).sum())
                    par.append(0)
                    R.append(f * d["r_per_um"] * L)
                    Cn.append(0.5 * f * d["c_per_um"] * L + 1e3 * cap(s))
                    Cn[0] += 0.5 * f * d["c_per_um"] * L
                    node[s] = k + 1
            Dm, beta = shared_path_moments(par, R, Cn)
            self.load[drv] = 1e-3 * sum(Cn)
            for s in sinks:
                self.Dns[s] = 1e-6 * Dm[node[s]]
                self.Vns[s] = 1e-12 * (2 * beta[node[s]] - Dm[node[s]] ** 2)
                self.driver[s] = drv


def rf_in_of(sense, rf_out):
    return {POS: [rf_out], NEG: [1 - rf_out], NON: [0, 1], RISE: [0]}.get(sense, [])


def enumerate_paths(d, corner=0, with_slew=False):
    """All (arrival, slew, rf) path values at every pin, by exhaustive
    enumeration.  Cell delays are evaluated per path at the path's own slew
    (path-based analysis)."""
    net = Net(d, corner)
    sc = float(np.asarray(d["lut_scale"])[corner])
    role = np.asarray(d["pin_role"])
    ctype = np.asarray(d["cell_type"])
    cpp = np.asarray(d["cell_pin_ptr"])
    cp = np.asarray(d["cell_pin"])
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    nin = np.asarray(d["type_nin"])
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    memo = {}

    def paths(p):
        if p in memo:
            return memo[p]
        r = role[p]
        if r == PI:
            out = [(float(d["pi_at_ns"]), float(d["pi_slew_ns"]), rf) for rf in (0, 1)]
        elif r == CK:
            out = [(0.0, float(d["clk_slew_ns"]), rf) for rf in (0, 1)]
        elif r in (IN, D, PO):
            drv = net.driver[p]
            out = [(a + net.Dns[p], np.sqrt(s * s + net.Vns[p]), rf) for a, s, rf in paths(drv)]
        else:
            c = net.cell_of[p]
            t = ctype[c]
            l = net.load.get(p, 0.0)
            out = []
            for slot in range(nin[t]):
                se = sense[t, slot]
                if se == NONE:
                    continue
                a_pin = cp[cpp[c] + slot]
                for a, s, rf in paths(a_pin):
                    if r == Q and rf != 0:
                        continue
                    for rfo in (0, 1):
                        if rf not in rf_in_of(se, rfo):
                            continue
                        dl = sc * bilinear(i1[t, slot, rfo], i2[t, slot, rfo], vv[t, slot, rfo], s, l)
                        sl = sc * bilinear(i1[t, slot, 2 + rfo], i2[t, slot, 2 + rfo], vv[t, slot, 2 + rfo], s, l)
                        out.append((a + dl, sl, rfo))
        memo[p] = out
        return out

    return {p: paths(p) for p in range(d["n_pins"])}


def enumerate_suffixes(d, corner=0, with_pins=False):
    """Every path from each pin to an endpoint, for slew-independent cell
    delays: {pin: [(delay to the endpoint, rf at the pin, endpoint pin)]}.
    Cell delays are read at the driven net's load (the tables do not depend
    on slew); net delays are the independent Elmore sums of ``Net``.  With
    with_pins each tuple also carries the gate input pins after the pin,
    in order."""
    net = Net(d, corner)
    sc = float(np.asarray(d["lut_scale"])[corner])
    role = np.asarray(d["pin_role"])
    ctype = np.asarray(d["cell_type"])
    cpp = np.asarray(d["cell_pin_ptr"])
    cp = np.asarray(d["cell_pin"])
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    nin = np.asarray(d["type_nin"])
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    sinks_of = {}
    for s, drv in net.driver.items():
        sinks_of.setdefault(drv, []).append(s)
    memo = {}

    def suf(p):
        if p in memo:
            return memo[p]
        r = role[p]
        out = []
        if r in (D, PO):
            out = [(0.0, rf, p, ()) for rf in (0, 1)]
        elif r in (PI, OUT, Q):
            for s in sinks_of.get(p, []):
                head = (s,) if role[s] == IN else ()
                out += [(dl + net.Dns[s], rf, e, head + ps) for dl, rf, e, ps in suf(s)]
        elif r in (IN, CK):
            c = net.cell_of[p]
            t = ctype[c]
            slot = net.slot_of[p]
            se = sense[t, slot]
            z = cp[cpp[c] + nin[t]]
            l = net.load.get(int(z), 0.0)
            for dl, rfo, e, ps in suf(int(z)):
                dc = sc * bilinear(i1[t, slot, rfo], i2[t, slot, rfo], vv[t, slot, rfo], 0.0, l)
                for rf in rf_in_of(se, rfo):
                    out.append((dl + dc, rf, e, ps))
        memo[p] = out
        return out

    alls = {p: suf(p) for p in range(d["n_pins"])}
    if with_pins:
        return alls
    return {p: [(dl, rf, e) for dl, rf, e, _ in v] for p, v in alls.items()}


def enumerate_paths_from(d, corner=0, with_pins=False):
    """Every path's (arrival, edge, startpoint pin) at every pin, for
    slew-independent cell delays (read at the driven net's load).  With
    with_pins each tuple also carries the gate input pins the path passes,
    in order."""
    net = Net(d, corner)
    sc = float(np.asarray(d["lut_scale"])[corner])
    role = np.asarray(d["pin_role"])
    ctype = np.asarray(d["cell_type"])
    cpp = np.asarray(d["cell_pin_ptr"])
    cp = np.asarray(d["cell_pin"])
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    nin = np.asarray(d["type_nin"])
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    memo = {}

    def paths(p):
        if p in memo:
            return memo[p]
        r = role[p]
        if r == PI:
            out = [(float(d["pi_at_ns"]), rf, p, ()) for rf in (0, 1)]
        elif r == CK:
            out = [(0.0, rf, p, ()) for rf in (0, 1)]
        elif r in (IN, D, PO):
            out = [(a + net.Dns[p], rf, s, ps + ((p,) if r == IN else ()))
                   for a, rf, s, ps in paths(net.driver[p])]
        else:
            c = net.cell_of[p]
            t = ctype[c]
            l = net.load.get(p, 0.0)
            out = []
            for slot in range(nin[t]):
                se = sense[t, slot]
                if se == NONE:
                    continue
                for a, rf, s, ps in paths(cp[cpp[c] + slot]):
                    if r == Q and rf != 0:
                        continue
                    for rfo in (0, 1):
                        if rf in rf_in_of(se, rfo):
                            dl = sc * bilinear(i1[t, slot, rfo], i2[t, slot, rfo], vv[t, slot, rfo], 0.0, l)
                            out.append((a + dl, rfo, s, ps))
        memo[p] = out
        return out

    allp = {p: paths(p) for p in range(d["n_pins"])}
    if with_pins:
        return allp
    return {p: [(a, rf, s) for a, rf, s, _ in v] for p, v in allp.items()}


def _lse(xs, gamma, late):
    """gamma * log sum exp(x / gamma) (late) or its mirror -gamma * log sum
    exp(-x / gamma) (early), by numpy's logaddexp over the listed values."""
    x = np.asarray(xs, np.float64)
    return gamma * np.logaddexp.reduce(x / gamma) if late else -gamma * np.logaddexp.reduce(-x / gamma)


def smoothed_forward(d, gamma, corner=0):
    """Arrival and slew of every pin, [pin][4] with index el*2 + rf, when every
    fan-in merge (arrival and slew) is the smooth max / min of the
    differentiable reading: each gate output lists all its arc candidates
    (input arrival + NLDM delay at the input slew and the output load, and
    the NLDM slew) and merges them at once with ``_lse``; net arcs add the
    shared-path Elmore delay and combine slews as sqrt(s^2 + var)."""
    net = Net(d, corner)
    sc = float(np.asarray(d["lut_scale"])[corner])
    role = np.asarray(d["pin_role"])
    ctype = np.asarray(d["cell_type"])
    cpp = np.asarray(d["cell_pin_ptr"])
    cp = np.asarray(d["cell_pin"])
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    nin = np.asarray(d["type_nin"])
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    memo = {}

    def st(p):
        if p in memo:
            return memo[p]
        r = role[p]
        if r == PI:
            out = (np.full(4, float(d["pi_at_ns"])), np.full(4, float(d["pi_slew_ns"])))
        elif r == CK:
            out = (np.zeros(4), np.full(4, float(d["clk_slew_ns"])))
        elif r in (IN, D, PO):
            a, s = st(net.driver[p])
            out = (a + net.Dns[p], np.sqrt(s * s + net.Vns[p]))
        else:
            c = net.cell_of[p]
            t = ctype[c]
            l = net.load.get(p, 0.0)
            at, sl = np.zeros(4), np.zeros(4)
            for el in (0, 1):
                for rfo in (0, 1):
                    ca, cs = [], []
                    for slot in range(nin[t]):
                        se = sense[t, slot]
                        if se == NONE:
                            continue
                        aa, ss = st(int(cp[cpp[c] + slot]))
                        for rfi in rf_in_of(se, rfo):
                            s_in = ss[el * 2 + rfi]
                            ca.append(aa[el * 2 + rfi] + sc * bilinear(i1[t, slot, rfo], i2[t, slot, rfo],
                                                                       vv[t, slot, rfo], s_in, l))
                            cs.append(sc * bilinear(i1[t, slot, 2 + rfo], i2[t, slot, 2 + rfo],
                                                    vv[t, slot, 2 + rfo], s_in, l))
                    at[el * 2 + rfo] = _lse(ca, gamma, el == 1)
                    sl[el * 2 + rfo] = _lse(cs, gamma, el == 1)
            out = (at, sl)
        memo[p] = out
        return out

    res = [st(p) for p in range(d["n_pins"])]
    return np.array([r[0] for r in res]), np.array([r[1] for r in res])


def enumerate_paths_at_slews(d, slew, corner=0):
    """Every path's (late arrival, edge) at every pin when each cell arc's
    delay is read at the slew the analysis computed for the arc's input pin
    and edge (``slew`` [pin][4], late components used) and the output load:
    path delays are then additive, and the latest path to a pin is its
    graph-based arrival."""
    net = Net(d, corner)
    sc = float(np.asarray(d["lut_scale"])[corner])
    role = np.asarray(d["pin_role"])
    ctype = np.asarray(d["cell_type"])
    cpp = np.asarray(d["cell_pin_ptr"])
    cp = np.asarray(d["cell_pin"])
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    nin = np.asarray(d["type_nin"])
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    slew = np.asarray(slew, np.float64)
    memo = {}

    def paths(p):
        if p in memo:
            return memo[p]
        r = role[p]
        if r == PI:
            out = [(float(d["pi_at_ns"]), rf) for rf in (0, 1)]
        elif r == CK:
            out = [(0.0, rf) for rf in (0, 1)]
        elif r in (IN, D, PO):
            out = [(a + net.Dns[p], rf) for a, rf in paths(net.driver[p])]
        else:
            c = net.cell_of[p]
            t = ctype[c]
            l = net.load.get(p, 0.0)
            out = []
            for slot in range(nin[t]):
                se = sense[t, slot]
                if se == NONE:
                    continue
                a_pin = int(cp[cpp[c] + slot])
                for a, rf in paths(a_pin):
                    if r == Q and rf != 0:
                        continue
                    for rfo in (0, 1):
                        if rf not in rf_in_of(se, rfo):
                            continue
                        dl = sc * bilinear(i1[t, slot, rfo], i2[t, slot, rfo], vv[t, slot, rfo],
                                           slew[a_pin, 2 + rf], l)
                        out.append((a + dl, rfo))
        memo[p] = out
        return out

    return {p: paths(p) for p in range(d["n_pins"])}
