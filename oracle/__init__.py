"""FP64 CPU reference STA (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library: ``sta_oracle.c`` is compiled on its own with
gcc into ``liboracle.so`` and driven through ctypes here.

Every function follows the textbook reading of the terms HeteroSTA
(arXiv 2511.11660) uses without formulas: NLDM tables (Sec. IV-A), Elmore
delay on RC trees (Sec. III, "Delay models"), RC from positions and unit R/C
(Sec. III, "Parasitics (RC) inputs"), pin slacks and WNS/TNS (Sec. III,
"Report options").  ``sta_oracle.c`` states each formula.

A design is a plain ``dict`` of numpy arrays and scalars (the layout that
``paper_2511_11660_b300.synth`` writes); see ``_Design`` for the keys.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sta_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ERRORS = {0: "ok", 1: "invalid input", 2: "combinational cycle", 3: "out of memory"}


def build(force: bool = False) -> str:
    """Compile ``sta_oracle.c`` into ``liboracle.so`` (gcc -O3, plain C; OpenMP
    only in the timed baseline ``orc_sta_timed``)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_lut_eval.argtypes = [P, P, P, C.c_double, C.c_double, P]
        _lib.orc_rc_tree.argtypes = [C.c_int32, P, P, P, P, P, P, P]
        _lib.orc_rc_tree_adjoint.argtypes = [C.c_int32, P, P, P, P, P, C.c_double, P, P]
        _lib.orc_arnoldi_t50.argtypes = [C.c_int32, P, P, P, C.c_int32, P]
        _lib.orc_net_delays.argtypes = [P, C.c_int32, P, P, P]
        _lib.orc_topo_order.argtypes = [P, P]
        _lib.orc_sta.argtypes = [P, P, P, P, P, P, P, P]
        _lib.orc_sta_timed.argtypes = [P, C.c_int32, C.c_int32, P, P]
        _lib.orc_objective_grad.argtypes = [P, C.c_double, C.c_double, P, P, P]
        _lib.orc_objective.argtypes = [P, C.c_double, C.c_double, P]
        _lib.orc_steiner_tree.argtypes = [C.c_int32, P, P, P, P, P, P, P, P]
        _lib.orc_nm.argtypes = [C.c_float]
        _lib.orc_net_wirelengths.argtypes = [P, P]
        _lib.orc_nm.restype = C.c_int64
        for f in ("orc_lut_eval", "orc_rc_tree", "orc_rc_tree_adjoint", "orc_arnoldi_t50", "orc_net_delays", "orc_topo_order", "orc_sta",
                  "orc_sta_timed",
                  "orc_objective_grad", "orc_objective", "orc_steiner_tree", "orc_net_wirelengths"):
            getattr(_lib, f).restype = C.c_int
    return _lib


class _Design(C.Structure):
    _fields_ = [
        ("n_types", C.c_int32), ("type_nin", C.c_void_p), ("type_kind", C.c_void_p),
        ("arc_sense", C.c_void_p), ("lut_idx1", C.c_void_p), ("lut_idx2", C.c_void_p),
        ("lut_val", C.c_void_p), ("pin_cap", C.c_void_p),
        ("setup_ns", C.c_double), ("hold_ns", C.c_double), ("po_cap_pf", C.c_double),
        ("n_cells", C.c_int32), ("cell_type", C.c_void_p), ("cell_pin_ptr", C.c_void_p),
        ("cell_pin", C.c_void_p), ("n_pins", C.c_int32), ("pin_role", C.c_void_p),
        ("n_nets", C.c_int32), ("net_pin_ptr", C.c_void_p), ("net_pin", C.c_void_p),
        ("rc_ptr", C.c_void_p), ("rc_parent", C.c_void_p), ("rc_pin_node", C.c_void_p),
        ("rc_R", C.c_void_p), ("rc_C", C.c_void_p), ("cell_xy", C.c_void_p), ("port_xy", C.c_void_p),
        ("r_per_um", C.c_double), ("c_per_um", C.c_double),
        ("period_ns", C.c_double), ("clk_slew_ns", C.c_double), ("pi_at_ns", C.c_double),
        ("pi_slew_ns", C.c_double), ("n_corners", C.c_int32), ("lut_scale", C.c_void_p),
        ("rc_scale", C.c_void_p), ("gamma_ns", C.c_double),
        ("net_model", C.c_int32), ("arnoldi_order", C.c_int32),
        ("n_exc", C.c_int32), ("exc_from_ptr", C.c_void_p), ("exc_from", C.c_void_p), ("exc_to_ptr", C.c_void_p),
        ("exc_to", C.c_void_p), ("exc_action", C.c_void_p), ("exc_mult", C.c_void_p),
        ("exc_thru_ptr", C.c_void_p), ("exc_thru_set_ptr", C.c_void_p), ("exc_thru_pin", C.c_void_p),
        ("wire_model", C.c_int32), ("r_per_um_y", C.c_double), ("c_per_um_y", C.c_double),
    ]


_ARRAYS = {
    "type_nin": np.int32, "type_kind": np.int32, "arc_sense": np.int32, "lut_idx1": np.float32,
    "lut_idx2": np.float32, "lut_val": np.float32, "pin_cap": np.float32, "cell_type": np.int32,
    "cell_pin_ptr": np.int32, "cell_pin": np.int32, "pin_role": np.int8, "net_pin_ptr": np.int32,
    "net_pin": np.int32, "rc_ptr": np.int32, "rc_parent": np.int32, "rc_pin_node": np.int32,
    "rc_R": np.float32, "rc_C": np.float32, "cell_xy": np.float32, "port_xy": np.float32,
    "lut_scale": np.float32, "rc_scale": np.float32,
    "exc_from_ptr": np.int32, "exc_from": np.int32, "exc_to_ptr": np.int32, "exc_to": np.int32,
    "exc_action": np.int32, "exc_mult": np.float32,
    "exc_thru_ptr": np.int32, "exc_thru_set_ptr": np.int32, "exc_thru_pin": np.int32,
}
_SCALARS = ("setup_ns", "hold_ns", "po_cap_pf", "r_per_um", "c_per_um", "period_ns", "clk_slew_ns",
            "pi_at_ns", "pi_slew_ns", "gamma_ns", "r_per_um_y", "c_per_um_y")


def _marshal(d: dict, use_rc: bool | None = None):
    """Build the ctypes struct; returns (struct, keep-alive list)."""
    keep = []
    s = _Design()
    if use_rc is None:
        use_rc = d.get("rc_ptr") is not None
    for k, dt in _ARRAYS.items():
        v = d.get(k)
        if k.startswith("rc_") and k not in ("rc_scale",) and not use_rc:
            v = None
        if v is None:
            setattr(s, k, None)
            continue
        a = np.ascontiguousarray(np.asarray(v), dtype=dt)
        keep.append(a)
        setattr(s, k, a.ctypes.data)
    for k in _SCALARS:
        setattr(s, k, float(d.get(k, 0.0)))
    s.n_types = int(d["n_types"])
    s.n_cells = int(d["n_cells"])
    s.n_pins = int(d["n_pins"])
    s.n_nets = int(d["n_nets"])
    s.n_corners = int(d.get("n_corners", 1))
    s.net_model = int(d.get("net_model", 0))
    s.wire_model = int(d.get("wire_model", 0))
    s.n_exc = int(len(d["exc_action"])) if d.get("exc_action") is not None else 0
    s.arnoldi_order = int(d.get("arnoldi_order", 3))
    if d.get("lut_scale") is None:
        a = np.ones(s.n_corners, np.float32); keep.append(a); s.lut_scale = a.ctypes.data
    if d.get("rc_scale") is None:
        a = np.ones(s.n_corners, np.float32); keep.append(a); s.rc_scale = a.ctypes.data
    return s, keep


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError("oracle %s failed: %s" % (what, ERRORS.get(rc, rc)))


def _ptr(a: np.ndarray):
    return a.ctypes.data


def lut_eval(idx1, idx2, val, s: float, l: float):
    """O1: bilinear lookup -> (value, d/d slew, d/d load)."""
    lib = _load()
    i1 = np.ascontiguousarray(idx1, np.float32)
    i2 = np.ascontiguousarray(idx2, np.float32)
    v = np.ascontiguousarray(val, np.float32).reshape(-1)
    out = np.zeros(3, np.float64)
    _check(lib.orc_lut_eval(_ptr(i1), _ptr(i2), _ptr(v), float(s), float(l), _ptr(out)), "lut_eval")
    return float(out[0]), float(out[1]), float(out[2])


def rc_tree(parent, R, C_):
    """O3 on one tree (double inputs): returns (Cdown, D, beta, var)."""
    lib = _load()
    par = np.ascontiguousarray(parent, np.int32)
    r = np.ascontiguousarray(R, np.float64)
    c = np.ascontiguousarray(C_, np.float64)
    n = len(par)
    outs = [np.zeros(n, np.float64) for _ in range(4)]
    _check(lib.orc_rc_tree(n, _ptr(par), _ptr(r), _ptr(c), *[_ptr(o) for o in outs]), "rc_tree")
    return tuple(outs)


def rc_tree_adjoint(parent, R, C_, Dbar, Vbar, Lbar: float):
    """Reverse mode of O3 on one tree: dJ/dR and dJ/dC from dJ/dD, dJ/dvar
    (per node) and dJ/dload (the root's downstream capacitance)."""
    lib = _load()
    par = np.ascontiguousarray(parent, np.int32)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (R, C_, Dbar, Vbar)]
    n = len(par)
    Rb, Cb = np.zeros(n, np.float64), np.zeros(n, np.float64)
    _check(lib.orc_rc_tree_adjoint(n, _ptr(par), *[_ptr(a) for a in arrs], float(Lbar), _ptr(Rb), _ptr(Cb)),
           "rc_tree_adjoint")
    return Rb, Cb


def arnoldi_t50(parent, R, C_, q: int):
    """O7 on one tree (double inputs, Ohm and fF): the 50% step-response delay
    of every node under an order-q Arnoldi reduced model (node 0: 0)."""
    lib = _load()
    par = np.ascontiguousarray(parent, np.int32)
    r = np.ascontiguousarray(R, np.float64)
    c = np.ascontiguousarray(C_, np.float64)
    out = np.zeros(len(par), np.float64)
    _check(lib.orc_arnoldi_t50(len(par), _ptr(par), _ptr(r), _ptr(c), int(q), _ptr(out)), "arnoldi_t50")
    return out


def nm(x_um: float) -> int:
    """O9 coordinate: the float product x * 1000 rounded to the nearest
    integer (ties to even), in nm."""
    return int(_load().orc_nm(float(x_um)))


def steiner_tree(X, Y) -> dict:
    """O9 on one net: integer nm pin coordinates (pin 0 = the driver) ->
    the rectilinear Steiner tree in breadth-first order: parent (root -1),
    node coordinates nx, ny, pin_node (node of each pin) and the total
    wirelength wl (nm)."""
    lib = _load()
    X = np.ascontiguousarray(X, np.int64)
    Y = np.ascontiguousarray(Y, np.int64)
    n = len(X)
    cap = max(1, 2 * n - 2)
    par = np.zeros(cap, np.int32)
    nx = np.zeros(cap, np.int64)
    ny = np.zeros(cap, np.int64)
    pn = np.zeros(max(n, 1), np.int32)
    n_out = C.c_int32(0)
    wl = C.c_int64(0)
    _check(lib.orc_steiner_tree(n, _ptr(X), _ptr(Y), C.byref(n_out), _ptr(par), _ptr(nx), _ptr(ny), _ptr(pn),
                                C.byref(wl)), "steiner_tree")
    k = n_out.value
    return {"parent": par[:k], "nx": nx[:k], "ny": ny[:k], "pin_node": pn[:n], "wl": int(wl.value)}


def net_wirelengths(d: dict) -> np.ndarray:
    """O9 tree length (int64 nm) of every net of a placed design."""
    lib = _load()
    s, keep = _marshal(d, use_rc=False)
    wl = np.zeros(max(int(d["n_nets"]), 1), np.int64)
    _check(lib.orc_net_wirelengths(C.byref(s), _ptr(wl)), "net_wirelengths")
    return wl[: int(d["n_nets"])]


def net_delays(d: dict, corner: int = 0, use_rc: bool | None = None):
    """Per pin: driver load (pF), sink Elmore delay (ns), sink variance (ns^2)."""
    lib = _load()
    s, keep = _marshal(d, use_rc)
    P = int(d["n_pins"])
    outs = [np.zeros(max(P, 1), np.float64) for _ in range(3)]
    _check(lib.orc_net_delays(C.byref(s), int(corner), *[_ptr(o) for o in outs]), "net_delays")
    return tuple(o[:P] for o in outs)


def topo_order(d: dict):
    lib = _load()
    s, keep = _marshal(d)
    out = np.zeros(max(int(d["n_pins"]), 1), np.int32)
    _check(lib.orc_topo_order(C.byref(s), _ptr(out)), "topo_order")
    return out[: int(d["n_pins"])]


def endpoints(d: dict) -> np.ndarray:
    """Endpoint pins (DFF D and PO) in ascending pin id, the oracle's order."""
    role = np.asarray(d["pin_role"])
    return np.nonzero((role == 4) | (role == 1))[0].astype(np.int32)


def tag_layout(d: dict):
    """O8 tags of an exception-group design: the first tag of each group and
    the advance mask of every pin (bit t: tag t moves on to t + 1 there)."""
    G = len(d["exc_action"]) if d.get("exc_action") is not None else 0
    tp = d.get("exc_thru_ptr")
    base, t = [], 1
    for g in range(G):
        base.append(t)
        t += (int(tp[g + 1]) - int(tp[g]) if tp is not None else 0) + 1
    adv = {}
    if tp is not None:
        tsp, tpin = d["exc_thru_set_ptr"], d["exc_thru_pin"]
        for g in range(G):
            for jj in range(int(tp[g + 1]) - int(tp[g])):
                s = int(tp[g]) + jj
                for p in tpin[tsp[s]:tsp[s + 1]]:
                    adv[int(p)] = adv.get(int(p), 0) | (1 << (base[g] + jj))
    return base, adv


def n_tags(d: dict) -> int:
    """O8 tags per corner: 1 + sum over exception groups of (through sets + 1)."""
    if d.get("exc_action") is None:
        return 1
    G = len(d["exc_action"])
    tp = d.get("exc_thru_ptr")
    return 1 + sum((int(tp[g + 1]) - int(tp[g]) if tp is not None else 0) + 1 for g in range(G))


def sta_timed(d: dict, n_threads: int = 1, reps: int = 3):
    """The plain analysis (no exception groups) timed ``reps`` times on
    ``n_threads`` host threads (OpenMP over the nets and over the pins of a
    level; the serial result).  Only net delays through WNS/TNS are timed:
    validation, the topological order and its levels are prepared once
    outside.  Returns (seconds per run [reps], summary [n_corners][8] as in
    ``sta``)."""
    lib = _load()
    s, keep = _marshal(d, None)
    K = int(d.get("n_corners", 1))
    secs = np.zeros(max(int(reps), 1), np.float64)
    summ = np.zeros((K, 8), np.float64)
    rc = lib.orc_sta_timed(C.byref(s), int(n_threads), int(reps), _ptr(secs), _ptr(summ))
    _check(rc, "sta_timed")
    return secs, summ


def sta(d: dict, use_rc: bool | None = None) -> dict:
    """Full FP64 analysis; see ``orc_sta`` for the array layouts.  With
    timing-exception groups (keys exc_from_ptr, exc_from, exc_to_ptr,
    exc_to, exc_action, exc_mult) the per-pin arrays hold one state per
    (corner, tag): index corner * (groups + 1) + tag."""
    lib = _load()
    s, keep = _marshal(d, use_rc)
    P, K = int(d["n_pins"]), int(d.get("n_corners", 1))
    Ks = K * n_tags(d)   # states: corner * tags + tag
    E = len(endpoints(d))
    arr = {k: np.zeros((max(P, 1), Ks, 4), np.float64) for k in ("at", "slew", "rat", "slack")}
    eps = np.zeros((max(E, 1), K), np.float64)
    eph = np.zeros((max(E, 1), K), np.float64)
    summ = np.zeros((K, 8), np.float64)
    rc = lib.orc_sta(C.byref(s), _ptr(arr["at"]), _ptr(arr["slew"]), _ptr(arr["rat"]),
                     _ptr(arr["slack"]), _ptr(eps), _ptr(eph), _ptr(summ))
    _check(rc, "sta")
    out = {k: v[:P] for k, v in arr.items()}
    out["ep_setup"] = eps[:E]
    out["ep_hold"] = eph[:E]
    out["endpoints"] = endpoints(d)
    out["wns_setup"] = summ[:, 0].copy()
    out["tns_setup"] = summ[:, 1].copy()
    out["wns_hold"] = summ[:, 2].copy()
    out["tns_hold"] = summ[:, 3].copy()
    out["worst_setup"] = summ[:, 4].copy()
    out["worst_hold"] = summ[:, 5].copy()
    out["n_viol_setup"] = summ[:, 6].astype(np.int64)
    out["n_viol_hold"] = summ[:, 7].astype(np.int64)
    return out


def objective_grad(d: dict, w_tns: float = 1.0, w_wns: float = 1.0):
    """O6: smoothed J, per-corner (TNS_g, WNS_g) and dJ/d(cell x, y) in FP64
    (star or Steiner parasitics from positions; Steiner with the Elmore model)."""
    lib = _load()
    s, keep = _marshal(d, use_rc=False)
    K = int(d.get("n_corners", 1))
    J = np.zeros(1, np.float64)
    terms = np.zeros((K, 2), np.float64)
    g = np.zeros((max(int(d["n_cells"]), 1), 2), np.float64)
    _check(lib.orc_objective_grad(C.byref(s), float(w_tns), float(w_wns), _ptr(J), _ptr(terms), _ptr(g)),
           "objective_grad")
    return float(J[0]), terms, g[: int(d["n_cells"])]


def objective(d: dict, w_tns: float = 1.0, w_wns: float = 1.0) -> float:
    lib = _load()
    s, keep = _marshal(d, use_rc=False)
    J = np.zeros(1, np.float64)
    _check(lib.orc_objective(C.byref(s), float(w_tns), float(w_wns), _ptr(J)), "objective")
    return float(J[0])


def report_paths(d: dict, k: int, slack_lt: float = float("inf"), corner: int = 0, res: dict | None = None):
    """Top-k path report (Sec. III "Report options": top-k, per-endpoint
    limit, slack threshold, CSR path arrays), per-endpoint limit 1.

    The endpoints whose setup slack at ``corner`` is below ``slack_lt``, in
    increasing slack (ties: lower endpoint index), the first ``k``; for each
    its critical path, traced back from the endpoint at the edge with the
    smaller late slack (ties: rise): a net sink steps to its net's driver with
    the same edge; a gate output steps to the input arc whose late arrival +
    NLDM delay (at that input's late slew and the output's load) is largest
    (ties: lower input slot, then rise before fall); a flip-flop Q steps to
    its CK (rising edge); the trace stops at a PI or CK.  Returns a list of
    dicts: endpoint pin, slack, and the pins, edges and late arrivals from the
    startpoint to the endpoint.  FP64, from this package's own analysis.

    With timing exceptions the endpoint's slack is its minimum over the
    exception tags, and the path is traced in the (tag, edge) state with the
    smallest late slack (ties: lower tag, then rise) -- the path of the
    startpoint group that sets the endpoint's slack."""
    res = res if res is not None else sta(d)
    K = int(d.get("n_corners", 1))
    Tg = n_tags(d)
    _, adv = tag_layout(d)
    sc = float(np.asarray(d["lut_scale"] if d.get("lut_scale") is not None else np.ones(K))[corner])
    load, _, _ = net_delays(d, corner)
    role = np.asarray(d["pin_role"])
    cpp, cp = np.asarray(d["cell_pin_ptr"]), np.asarray(d["cell_pin"])
    ctype, nin = np.asarray(d["cell_type"]), np.asarray(d["type_nin"])
    kind = np.asarray(d["type_kind"])
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    cell_of = -np.ones(d["n_pins"], int)
    slot_of = -np.ones(d["n_pins"], int)
    for c in range(d["n_cells"]):
        for j in range(cpp[c], cpp[c + 1]):
            cell_of[cp[j]] = c
            slot_of[cp[j]] = j - cpp[c]
    npp, npn = np.asarray(d["net_pin_ptr"]), np.asarray(d["net_pin"])
    driver = -np.ones(d["n_pins"], int)
    for n in range(d["n_nets"]):
        driver[npn[npp[n] + 1:npp[n + 1]]] = npn[npp[n]]
    eps, es = res["endpoints"], res["ep_setup"][:, corner]
    order = sorted((e for e in range(len(eps)) if es[e] < slack_lt), key=lambda e: (es[e], e))[:k]
    arcs_on = {0: lambda i, o: i == o, 1: lambda i, o: i != o, 2: lambda i, o: True}
    out = []
    for e in order:
        p = int(eps[e])
        best_s, st, rf = np.inf, corner * Tg, 0
        for g in range(Tg):
            sl = res["slack"][p, corner * Tg + g]
            if min(sl[2], sl[3]) < best_s:
                best_s, st, rf = min(sl[2], sl[3]), corner * Tg + g, 0 if sl[2] <= sl[3] else 1
        pins, rfs, ats = [], [], []
        while True:
            if len(pins) > d["n_pins"]:
                raise RuntimeError("oracle report_paths: path longer than the design")
            at, slew = res["at"][:, st], res["slew"][:, st]
            pins.append(p)
            rfs.append(rf)
            ats.append(at[p, 2 + rf])
            if driver[p] >= 0:                       # net sink: to the driver, same edge
                # through a -through pin the path may come from the previous
                # tag's state: the one with the larger late arrival (ties: same)
                tg = st - corner * Tg
                a = adv.get(p, 0)
                stay, inflow = not (a >> tg) & 1, tg >= 1 and (a >> (tg - 1)) & 1
                dp = int(driver[p])
                if inflow and (not stay or res["at"][dp, st - 1, 2 + rf] > res["at"][dp, st, 2 + rf]):
                    st -= 1
                p = dp
                continue
            if role[p] in (0, 5):                    # PI or CK: the startpoint
                break
            c = cell_of[p]
            t = ctype[c]
            if kind[t] == 1:                         # Q: to CK (the rising-edge input slot)
                p, rf = int(cp[cpp[c] + int(np.nonzero(sense[t] == 3)[0][0])]), 0
                continue
            best, arg = -np.inf, None
            for j in range(nin[t]):
                a = int(cp[cpp[c] + j])
                for rfi in (0, 1):
                    if sense[t, j] < 0 or not arcs_on[int(sense[t, j])](rfi, rf):
                        continue
                    dl = lut_eval(i1[t, j, rf], i2[t, j, rf], vv[t, j, rf], slew[a, 2 + rfi], load[p])[0]
                    cand = at[a, 2 + rfi] + sc * dl
                    if cand > best:
                        best, arg = cand, (a, rfi)
            p, rf = arg
        pins.reverse()
        rfs.reverse()
        ats.reverse()
        out.append({"endpoint": int(eps[e]), "slack": float(es[e]), "pins": np.array(pins),
                    "rf": np.array(rfs, np.int8), "at": np.array(ats)})
    return out


def report_paths_nworst(d: dict, k: int, per_endpoint: int, slack_lt: float = float("inf"), corner: int = 0,
                        res: dict | None = None):
    """Top-k path report with a per-endpoint limit (Sec. III "Report
    options": top-k, per-endpoint report limit, slack-less-than threshold):
    the k paths of smallest setup slack at ``corner`` below ``slack_lt``,
    at most ``per_endpoint`` of them ending at any one endpoint.

    A path runs from a startpoint (PI or CK) to an endpoint through timing
    arcs; its late arrival adds, along the path, each cell arc's NLDM delay
    at the analysis' own input slew and output load, and each net's delay.
    Relative to the critical path of report_paths (same tie rules), a path
    is the endpoint edge it ends on plus the gate outputs where it leaves the
    critical fan-in: leaving it at output (p, rf) for input arc (a, rfi)
    costs dev = cand(critical) - cand(a, rfi) >= 0 with cand = late arrival
    of (a, rfi) + arc delay, and the path's slack is the endpoint edge's
    slack plus the sum of its devs.  Each endpoint's paths come from a
    best-first search over these deviation sets, every set generated once:
    a path's children leave the critical fan-in at or above its last
    deviation's input pin.  The endpoints considered are the k worst (no
    other can hold one of the k worst paths); their paths are merged by
    (slack, endpoint order, rank at the endpoint).  Returns dicts like
    report_paths, with the pins, edges and the path's own late arrivals.
    Without timing exceptions only."""
    import heapq
    if n_tags(d) != 1:
        raise ValueError("per-endpoint limit above 1 needs a design without timing exceptions")
    res = res if res is not None else sta(d)
    K = int(d.get("n_corners", 1))
    sc = float(np.asarray(d["lut_scale"] if d.get("lut_scale") is not None else np.ones(K))[corner])
    load, _, _ = net_delays(d, corner)
    role = np.asarray(d["pin_role"])
    cpp, cp = np.asarray(d["cell_pin_ptr"]), np.asarray(d["cell_pin"])
    ctype, nin = np.asarray(d["cell_type"]), np.asarray(d["type_nin"])
    kind = np.asarray(d["type_kind"])
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    cell_of = -np.ones(d["n_pins"], int)
    for c in range(d["n_cells"]):
        cell_of[cp[cpp[c]:cpp[c + 1]]] = c
    npp, npn = np.asarray(d["net_pin_ptr"]), np.asarray(d["net_pin"])
    driver = -np.ones(d["n_pins"], int)
    for n in range(d["n_nets"]):
        driver[npn[npp[n] + 1:npp[n + 1]]] = npn[npp[n]]
    at, slew = res["at"][:, corner], res["slew"][:, corner]
    arcs_on = {0: lambda i, o: i == o, 1: lambda i, o: i != o, 2: lambda i, o: True}

    def fanin(p, rf):
        """Candidates of node (p, rf): [(a, rfi, cand)] in tie order, or one
        (driver / CK) step, or [] at a startpoint; and whether p is a gate output."""
        if driver[p] >= 0:
            return [(int(driver[p]), rf, None)], False
        if role[p] in (0, 5):
            return [], False
        c = cell_of[p]
        t = ctype[c]
        if kind[t] == 1:
            return [(int(cp[cpp[c] + int(np.nonzero(sense[t] == 3)[0][0])]), 0, None)], False
        out = []
        for j in range(nin[t]):
            a = int(cp[cpp[c] + j])
            for rfi in (0, 1):
                if sense[t, j] < 0 or not arcs_on[int(sense[t, j])](rfi, rf):
                    continue
                dl = lut_eval(i1[t, j, rf], i2[t, j, rf], vv[t, j, rf], slew[a, 2 + rfi], load[p])[0]
                out.append((a, rfi, at[a, 2 + rfi] + sc * dl))
        return out, True

    def critical(cands):
        best = 0
        for i in range(1, len(cands)):
            if cands[i][2] > cands[best][2]:
                best = i
        return best

    def region(p, rf):
        """Deviations at or above node (p, rf) along the critical fan-in:
        [(dev, (p, rf, a, rfi))]."""
        out = []
        while True:
            cands, gate = fanin(p, rf)
            if not cands:
                return out
            b = critical(cands) if gate else 0
            if gate:
                for i, (a, rfi, cand) in enumerate(cands):
                    if i != b:
                        out.append((cands[b][2] - cand, (p, rf, a, rfi)))
            p, rf = cands[b][0], cands[b][1]

    eps, es = res["endpoints"], res["ep_setup"][:, corner]
    order = sorted((e for e in range(len(eps)) if es[e] < slack_lt), key=lambda e: (es[e], e))[:k]
    found = []
    for oi, e in enumerate(order):
        p = int(eps[e])
        sl = res["slack"][p, corner]
        heap, seq = [], 0
        for rf in (0, 1):
            heapq.heappush(heap, (float(sl[2 + rf]), seq, rf, ()))
            seq += 1
        rank = 0
        while heap and rank < per_endpoint:
            cost, _, rf, devs = heapq.heappop(heap)
            if not cost < slack_lt:
                break
            found.append((cost, oi, rank, p, rf, devs))
            rank += 1
            start = (p, rf) if not devs else (devs[-1][2], devs[-1][3])
            for dv, dev in region(*start):
                heapq.heappush(heap, (cost + dv, seq, rf, devs + (dev,)))
                seq += 1
    found.sort(key=lambda f: (f[0], f[1], f[2]))
    out = []
    for cost, _, _, p, rf, devs in found[:k]:
        pins, rfs, ats, dsum = [], [], [], []
        q, qrf, di, acc = p, rf, 0, 0.0
        while True:
            pins.append(q)
            rfs.append(qrf)
            cands, gate = fanin(q, qrf)
            if not cands:
                break
            if gate and di < len(devs) and devs[di][0] == q and devs[di][1] == qrf:
                b = critical(cands)
                alt = [x for x in cands if x[0] == devs[di][2] and x[1] == devs[di][3]][0]
                dsum.append(cands[b][2] - alt[2])
                q, qrf = alt[0], alt[1]
                di += 1
                continue
            dsum.append(0.0)
            b = critical(cands) if gate else 0
            q, qrf = cands[b][0], cands[b][1]
        dsum.append(0.0)
        # the path's arrival at a pin: the analysis' arrival less the devs taken at or above it
        up = np.cumsum(dsum[::-1])[::-1]
        ats = [at[x, 2 + r] - u for x, r, u in zip(pins, rfs, up[:len(pins)])]
        out.append({"endpoint": p, "slack": cost, "pins": np.array(pins[::-1]),
                    "rf": np.array(rfs[::-1], np.int8), "at": np.array(ats[::-1])})
    return out
