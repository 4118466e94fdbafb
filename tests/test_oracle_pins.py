"""Pins for the FP64 oracle: hand-worked values, closed forms, brute force
and invariants (no GPU).  Each test names the reading it checks; HeteroSTA
(arXiv 2511.11660) prints no formula, so the readings are the textbook STA
definitions of the terms it uses (NLDM Sec. IV-A, Elmore Sec. III "Delay
models", pin slacks and WNS/TNS Sec. III "Report options")."""
import os

import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import synth
from tests import _indep

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_lut_golden():
    idx1 = idx2 = None
    rows, qs = [], []
    for line in open(os.path.join(GOLD, "lut_hand.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "idx1":
            idx1 = [float(x) for x in line[1:]]
        elif line[0] == "idx2":
            idx2 = [float(x) for x in line[1:]]
        elif line[0] == "row":
            rows.append([float(x) for x in line[1:]])
        elif line[0] == "q":
            qs.append(tuple(float(x) for x in line[1:]))
    return np.array(idx1), np.array(idx2), np.array(rows), qs


# ------------------------------------------------------------------ O1 NLDM

def test_lut_hand_worked_values():
    idx1, idx2, val, qs = _read_lut_golden()
    assert len(qs) >= 5
    for s, l, want in qs:
        got, _, _ = oracle.lut_eval(idx1, idx2, val, s, l)
        # tables are stored in fp32, so compare at fp32 resolution
        assert got == pytest.approx(want, abs=2e-7), (s, l)


def test_lut_reproduces_bilinear_function_exactly():
    """A noise-free table of a + b s + c l + d s l is reproduced everywhere,
    inside the table and when extrapolating from its edge segments."""
    rng = np.random.default_rng(1)
    idx1 = np.geomspace(0.005, 1.0, 7)
    idx2 = np.geomspace(0.001, 0.5, 7)
    # fp32-exact grid so the table holds the function's exact values
    idx1 = np.round(idx1 * 2 ** 8) / 2 ** 8
    idx2 = np.round(idx2 * 2 ** 10) / 2 ** 10
    a, b, c, d = 0.25, 0.5, 2.0, 0.75
    val = a + b * idx1[:, None] + c * idx2[None, :] + d * idx1[:, None] * idx2[None, :]
    assert np.all(val.astype(np.float32) == val)
    for s, l in zip(rng.uniform(-0.2, 1.6, 300), rng.uniform(-0.1, 0.9, 300)):
        got, ds, dl = oracle.lut_eval(idx1, idx2, val, s, l)
        assert got == pytest.approx(a + b * s + c * l + d * s * l, rel=1e-12, abs=1e-13)
        assert ds == pytest.approx(b + d * l, rel=1e-10, abs=1e-12)
        assert dl == pytest.approx(c + d * s, rel=1e-10, abs=1e-12)


def test_lut_partials_match_independent_bilinear():
    lib = synth.make_library(3)
    i1 = lib["lut_idx1"].reshape(-1, 3, 4, 7)[2, 0, 1]
    i2 = lib["lut_idx2"].reshape(-1, 3, 4, 7)[2, 0, 1]
    v = lib["lut_val"].reshape(-1, 3, 4, 49)[2, 0, 1]
    rng = np.random.default_rng(2)
    for s, l in zip(rng.uniform(0.0, 1.2, 200), rng.uniform(0.0, 0.6, 200)):
        got, ds, dl = oracle.lut_eval(i1, i2, v, s, l)
        assert got == pytest.approx(_indep.bilinear(i1, i2, v, s, l), rel=1e-12, abs=1e-14)
        h = 1e-7
        # derivative inside the segment: one-sided towards the segment interior
        fd_s = (_indep.bilinear(i1, i2, v, s + h, l) - _indep.bilinear(i1, i2, v, s - h, l)) / (2 * h)
        fd_l = (_indep.bilinear(i1, i2, v, s, l + h) - _indep.bilinear(i1, i2, v, s, l - h)) / (2 * h)
        near_bp = np.min(np.abs(i1[1:6] - s)) < 2 * h or np.min(np.abs(i2[1:6] - l)) < 2 * h
        if not near_bp:
            assert ds == pytest.approx(fd_s, rel=1e-5, abs=1e-7)
            assert dl == pytest.approx(fd_l, rel=1e-5, abs=1e-7)


# ---------------------------------------------------------------- O3 Elmore

def test_elmore_chain_hand_worked():
    rows = {}
    for line in open(os.path.join(GOLD, "elmore_chain.txt")):
        line = line.split("#")[0].split()
        if line:
            rows[line[0]] = [float(x) for x in line[1:]]
    par = [int(x) for x in rows["parent"]]
    cd, Dm, beta, var = oracle.rc_tree(par, rows["R"], rows["C"])
    np.testing.assert_allclose(Dm, rows["D"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(beta, rows["beta"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(var, rows["var"], rtol=0, atol=1e-9)


def test_elmore_single_rc_closed_form():
    for R, Cc in [(5.0, 0.5), (50.0, 5.0), (17.0, 2.25)]:
        _, Dm, beta, var = oracle.rc_tree([-1, 0], [0.0, R], [0.0, Cc])
        assert Dm[1] == pytest.approx(R * Cc, rel=1e-14)
        assert beta[1] == pytest.approx((R * Cc) ** 2, rel=1e-14)
        assert var[1] == pytest.approx((R * Cc) ** 2, rel=1e-12)


@pytest.mark.parametrize("n", [1, 2, 5, 11])
def test_elmore_uniform_chain_closed_form(n):
    R, Cc = 7.0, 1.5
    par = [-1] + list(range(n))
    _, Dm, _, _ = oracle.rc_tree(par, [0.0] + [R] * n, [0.0] + [Cc] * n)
    for k in range(1, n + 1):
        assert Dm[k] == pytest.approx(R * Cc * (k * n - k * (k - 1) / 2), rel=1e-13)


def test_elmore_random_trees_vs_shared_path_sums():
    rng = np.random.default_rng(5)
    for _ in range(30):
        n = int(rng.integers(2, 14))
        par = [-1] + [int(rng.integers(0, i)) for i in range(1, n)]
        R = [0.0] + list(rng.uniform(5, 50, n - 1))
        Cc = list(rng.uniform(0.5, 5, n))
        cd, Dm, beta, var = oracle.rc_tree(par, R, Cc)
        D2, b2 = _indep.shared_path_moments(par, R, Cc)
        np.testing.assert_allclose(Dm, D2, rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(beta, b2, rtol=1e-12, atol=1e-6)
        assert cd[0] == pytest.approx(sum(Cc), rel=1e-13)
        assert np.all(var >= -1e-9 * np.maximum(1, beta))   # a variance


def test_net_delays_match_shared_path_on_generated_design():
    d = synth.make_design(300, 8, seed=11)
    load, Dn, Vn = oracle.net_delays(d)
    ind = _indep.Net(d)
    for p, L in ind.load.items():
        assert load[p] == pytest.approx(L, rel=1e-12)
    for p, v in ind.Dns.items():
        assert Dn[p] == pytest.approx(v, rel=1e-11, abs=1e-18)
        assert Vn[p] == pytest.approx(ind.Vns[p], rel=1e-9, abs=1e-20)


def test_star_tree_closed_form():
    """Star RC from positions: D = R (C/2 + Cpin), var = D^2, load = sum
    over sinks of (c L + Cpin), R = r L, C = c L."""
    lib = synth.make_library(0)
    b = synth.Builder(lib)
    a = b.pi(xy=(0.0, 0.0))
    x = b.cell("BUF", [a], xy=(30.0, 40.0))
    y = b.cell("INV", [x], xy=(130.0, 10.0))
    b.po(x, xy=(0.0, 500.0))
    b.po(y, xy=(10.0, 10.0))
    d = b.design(placed=True)
    load, Dn, Vn = oracle.net_delays(d)
    r, c = 0.1, 0.2
    capin = lib["pin_cap"].reshape(-1, 4).astype(np.float64)
    # net of x: sinks = INV input (|100|+|30| = 130 um) and PO (30 + 460 = 490 um)
    pins = d["net_pin"][d["net_pin_ptr"][1]:d["net_pin_ptr"][2]]
    assert pins[0] == x
    want_load = 0.0
    for s in pins[1:]:
        if d["pin_role"][s] == synth.PO:
            L, cp = 490.0, 1e3 * lib["po_cap_pf"]
        else:
            L, cp = 130.0, 1e3 * float(capin[synth.TYPE_NAMES.index("INV"), 0])
        Dr = r * L * (c * L / 2 + cp)
        assert Dn[s] == pytest.approx(1e-6 * Dr, rel=1e-12)
        assert Vn[s] == pytest.approx((1e-6 * Dr) ** 2, rel=1e-9)
        want_load += 1e-3 * (c * L + cp)
    assert load[x] == pytest.approx(want_load, rel=1e-12)


# ------------------------------------------------- O2/O4 propagation, slack

def _fixed_design(seed, n_cells=9, depth=4):
    lib = synth.make_library(seed, fixed_delay=True)
    return synth.make_design(n_cells, depth, seed=seed, lib=lib, rc_nodes=(2, 5), pi_frac=0.3)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_paths_fixed_delay(seed):
    """With slew-independent delays, arrival times are exactly the longest /
    shortest path sums over every enumerated path."""
    d = _fixed_design(seed)
    r = oracle.sta(d)
    allp = _indep.enumerate_paths(d)
    checked = 0
    for p, lst in allp.items():
        for rf in (0, 1):
            vals = [a for a, _, f in lst if f == rf]
            if not vals:
                continue
            assert r["at"][p, 0, 2 + rf] == pytest.approx(max(vals), abs=1e-12), (p, rf)
            assert r["at"][p, 0, rf] == pytest.approx(min(vals), abs=1e-12), (p, rf)
            checked += 1
    assert checked > 20


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_required_times_fixed_delay(seed):
    """With slew-independent delays, the late required time of a pin is the
    minimum over every path from it to an endpoint of (endpoint requirement
    - path delay) and the early one the maximum (setup requirement T - t_setup
    at a D pin and T at a PO; hold requirement t_hold at a D pin and 0 at a
    PO); pins with no path to an endpoint have +-inf."""
    d = _fixed_design(seed)
    d["period_ns"] = 0.7
    r = oracle.sta(d)
    role = np.asarray(d["pin_role"])
    req_late = {synth.D: d["period_ns"] - d["setup_ns"], synth.PO: d["period_ns"]}
    req_early = {synth.D: d["hold_ns"], synth.PO: 0.0}
    checked = 0
    for p, lst in _indep.enumerate_suffixes(d).items():
        for rf in (0, 1):
            late = [req_late[role[e]] - dl for dl, f, e in lst if f == rf]
            early = [req_early[role[e]] - dl for dl, f, e in lst if f == rf]
            want_l = min(late) if late else np.inf
            want_e = max(early) if early else -np.inf
            assert r["rat"][p, 0, 2 + rf] == pytest.approx(want_l, abs=1e-12), (p, rf)
            assert r["rat"][p, 0, rf] == pytest.approx(want_e, abs=1e-12), (p, rf)
            checked += bool(late)
    assert checked > 20


@pytest.mark.parametrize("seed", range(4))
def test_gba_bounds_pba(seed):
    """Slew-dependent mode with monotone tables: graph-based late arrival is
    no smaller than any path-based arrival, early no larger, and equal to it
    where a pin is reached by a single path (every Q pin: its CK source, at
    the clock slew).  The clock slew and the PI arrival/slew differ so that
    each source's own value is the one that propagates."""
    lib = synth.make_library(seed, noise=0.0)
    d = synth.make_design(10, 4, seed=seed, lib=lib, rc_nodes=(2, 6), pi_frac=0.3)
    d.update(clk_slew_ns=0.07, pi_slew_ns=0.02, pi_at_ns=0.013)
    r = oracle.sta(d)
    allp = _indep.enumerate_paths(d)
    role = np.asarray(d["pin_role"])
    n_tight = n_single = 0
    for p, lst in allp.items():
        for rf in (0, 1):
            vals = [a for a, _, f in lst if f == rf]
            slews = [s for _, s, f in lst if f == rf]
            if not vals:
                continue
            assert r["at"][p, 0, 2 + rf] >= max(vals) - 1e-12
            assert r["at"][p, 0, rf] <= min(vals) + 1e-12
            n_tight += abs(r["at"][p, 0, 2 + rf] - max(vals)) < 1e-12
            if len(vals) == 1:
                n_single += 1
                for el in (0, 2):
                    assert r["at"][p, 0, el + rf] == pytest.approx(vals[0], abs=1e-12), (p, rf)
                    assert r["slew"][p, 0, el + rf] == pytest.approx(slews[0], abs=1e-12), (p, rf)
    assert n_tight > 0 and n_single > 0
    assert np.any(role == synth.Q)


def test_single_gate_hand_case():
    """PI -> INV -> DFF D with a noise-free library, worked in closed form."""
    lib = synth.make_library(0, noise=0.0)
    coef = {}
    # INV slot 0: set known coefficients for the 4 tables
    s_ax = lib["lut_idx1"].reshape(-1, 3, 4, 7)[0, 0, 0].astype(float)
    l_ax = lib["lut_idx2"].reshape(-1, 3, 4, 7)[0, 0, 0].astype(float)
    val = lib["lut_val"].reshape(-1, 3, 4, 49).astype(np.float64)
    for tb, (a, b_, c, dd) in enumerate([(0.02, 0.1, 2.0, 0.3), (0.015, 0.12, 1.5, 0.2),
                                         (0.01, 0.05, 3.0, 0.4), (0.012, 0.06, 2.5, 0.1)]):
        coef[tb] = (a, b_, c, dd)
        val[0, 0, tb] = (a + b_ * s_ax[:, None] + c * l_ax[None, :] + dd * s_ax[:, None] * l_ax[None, :]).reshape(-1)
    lib["lut_val"] = val.astype(np.float32).reshape(-1)
    b = synth.Builder(lib)
    a = b.pi()
    z = b.cell("INV", [a])
    b.cell("DFF", [z])
    d = b.design(period_ns=0.5, default_R=20.0, default_C=2.0)
    r = oracle.sta(d)
    capin = lib["pin_cap"].reshape(-1, 4).astype(np.float64)
    inv_in, inv_out = d["cell_pin"][0], d["cell_pin"][1]
    dpin = d["cell_pin"][2]
    # net PI -> INV input: two-node tree, R = 20, C = 2 fF + pin cap
    Cn = 2.0 + 1e3 * capin[0, 0]
    Dn = 1e-6 * 20.0 * Cn
    Vn = (1e-6 * 20.0 * Cn) ** 2
    s_in = np.sqrt(0.02 ** 2 + Vn)
    # net INV -> DFF D
    Cz = 2.0 + 1e3 * capin[7, 0]
    load = 1e-3 * Cz
    Dz = 1e-6 * 20.0 * Cz

    def f(tb, s, l):
        a_, b_, c_, d_ = coef[tb]
        return a_ + b_ * s + c_ * l + d_ * s * l

    # inverter: output rise from input fall and vice versa; PI AT 0 both
    at_out = {0: Dn + f(0, s_in, load), 1: Dn + f(1, s_in, load)}
    for rf in (0, 1):
        assert r["at"][inv_in, 0, 2 + rf] == pytest.approx(Dn, abs=1e-12)
        assert r["slew"][inv_in, 0, 2 + rf] == pytest.approx(s_in, abs=1e-12)
        # fp32 table values: allow their rounding
        assert r["at"][inv_out, 0, 2 + rf] == pytest.approx(at_out[rf], abs=1e-7)
        assert r["slew"][inv_out, 0, 2 + rf] == pytest.approx(f(2 + rf, s_in, load), abs=1e-7)
        assert r["at"][dpin, 0, 2 + rf] == pytest.approx(at_out[rf] + Dz, abs=1e-7)
    want_setup = 0.5 - 0.03 - max(at_out[0], at_out[1]) - Dz
    assert r["ep_setup"][0, 0] == pytest.approx(want_setup, abs=1e-7)
    assert r["ep_hold"][0, 0] == pytest.approx(min(at_out[0], at_out[1]) + Dz - 0.01, abs=1e-7)
    # required time at the PI: back through the net and the inverter
    rat_out = {rf: 0.5 - 0.03 - Dz for rf in (0, 1)}
    assert r["rat"][inv_in, 0, 2 + 1] == pytest.approx(rat_out[0] - f(0, s_in, load), abs=1e-7)
    assert r["rat"][a, 0, 2 + 0] == pytest.approx(rat_out[1] - f(1, s_in, load) - Dn, abs=1e-7)


@pytest.mark.parametrize("seed", [0, 1])
def test_invariants_on_generated_design(seed):
    # early <= late for slews needs tables non-decreasing in slew: noise-free
    d = synth.make_design(3000, 25, seed=seed, period_ns=1.5, lib=synth.make_library(seed, noise=0.0))
    r = oracle.sta(d)
    at, sl, rat, sk = r["at"][:, 0], r["slew"][:, 0], r["rat"][:, 0], r["slack"][:, 0]
    fin = np.isfinite(rat)
    # slack = RAT - AT (late), AT - RAT (early)
    np.testing.assert_array_equal(sk[:, 2:][fin[:, 2:]], (rat[:, 2:] - at[:, 2:])[fin[:, 2:]])
    np.testing.assert_array_equal(sk[:, :2][fin[:, :2]], (at[:, :2] - rat[:, :2])[fin[:, :2]])
    # early <= late
    assert np.all(at[:, :2] <= at[:, 2:] + 1e-15)
    assert np.all(sl[:, :2] <= sl[:, 2:] + 1e-15)
    assert np.all(sl > 0)
    # WNS / TNS definitions over the endpoint slacks
    e = r["ep_setup"][:, 0]
    assert r["wns_setup"][0] == pytest.approx(min(0.0, e.min()), abs=0)
    assert r["tns_setup"][0] == pytest.approx(np.minimum(e, 0).sum(), rel=1e-12)
    assert r["tns_setup"][0] <= 0
    assert r["n_viol_setup"][0] == int((e < 0).sum())
    # the critical path carries the worst slack: no pin is worse, and some
    # source pin (its start) has exactly the worst slack
    late = sk[:, 2:][np.isfinite(sk[:, 2:])]
    assert late.min() == pytest.approx(e.min(), abs=1e-12)
    src = np.isin(np.asarray(d["pin_role"]), [synth.PI, synth.CK])
    assert np.min(sk[src][:, 2:][np.isfinite(sk[src][:, 2:])]) == pytest.approx(e.min(), abs=1e-12)
    # endpoints listed in ascending pin id, DFF D and PO only
    ep = r["endpoints"]
    assert np.all(np.diff(ep) > 0)
    assert set(np.unique(np.asarray(d["pin_role"])[ep])) <= {synth.D, synth.PO}


def test_topological_order_is_valid():
    d = synth.make_design(500, 12, seed=4)
    order = oracle.topo_order(d)
    pos = np.empty(d["n_pins"], int)
    pos[order] = np.arange(d["n_pins"])
    assert sorted(order.tolist()) == list(range(d["n_pins"]))
    npp, npn = d["net_pin_ptr"], d["net_pin"]
    for n in range(d["n_nets"]):
        drv = npn[npp[n]]
        assert np.all(pos[npn[npp[n] + 1:npp[n + 1]]] > pos[drv])
    cpp, cp = d["cell_pin_ptr"], d["cell_pin"]
    for c in range(d["n_cells"]):
        pins = cp[cpp[c]:cpp[c + 1]]
        if d["cell_type"][c] == synth.DFF_TYPE:
            assert pos[pins[2]] > pos[pins[1]]
        else:
            assert np.all(pos[pins[-1]] > pos[pins[:-1]])


def test_cycle_is_rejected():
    lib = synth.make_library(0)
    b = synth.Builder(lib)
    a = b.pi()
    z1 = b.cell("NAND2", [a, a])
    z2 = b.cell("INV", [z1])
    b.po(z2)
    d = b.design()
    # re-wire NAND2 input 1 to be driven by z2: INV out -> NAND2 -> INV loop
    npn = d["net_pin"].copy()
    nand_in1 = d["cell_pin"][1]
    # move nand_in1 from the PI net to the z2 net
    nets = [list(npn[d["net_pin_ptr"][n]:d["net_pin_ptr"][n + 1]]) for n in range(d["n_nets"])]
    for net in nets:
        if nand_in1 in net[1:]:
            net.remove(nand_in1)
    for net in nets:
        if net[0] == z2:
            net.append(nand_in1)
    d["net_pin"] = np.array([p for n in nets for p in n], np.int32)
    d["net_pin_ptr"] = np.concatenate([[0], np.cumsum([len(n) for n in nets])]).astype(np.int32)
    d["rc_pin_node"] = np.array([0 if i == 0 else 1 for n in nets for i in range(len(n))], np.int32)
    with pytest.raises(RuntimeError, match="cycle"):
        oracle.sta(d)


def test_corner_scaling_is_per_corner():
    """A corner with LUT scale 1 and RC scale 1 equals the single-corner run;
    scaling wire R and C by f scales every wire-only Elmore delay by f^2."""
    d1 = synth.make_design(400, 10, seed=8)
    d4 = dict(d1)
    d4.update(n_corners=3, lut_scale=np.array([1.0, 0.9, 1.25], np.float32),
              rc_scale=np.array([1.0, 1.1, 0.95], np.float32))
    r1, r4 = oracle.sta(d1), oracle.sta(d4)
    np.testing.assert_array_equal(r4["at"][:, 0], r1["at"][:, 0])
    np.testing.assert_array_equal(r4["slack"][:, 0], r1["slack"][:, 0])
    assert not np.allclose(r4["at"][:, 1], r1["at"][:, 0])


@pytest.mark.parametrize("placed", [False, True])
def test_corner_equals_prescaled_single_corner(placed):
    """Corner k with LUT scale s_k and RC scale f_k equals a single-corner
    design whose table values are multiplied by s_k and whose wire R and C
    (tree values, or per-um values for positions) are multiplied by f_k.
    Powers of two keep the pre-scaled fp32 inputs exact."""
    d = synth.make_design(300, 9, seed=12, placed=placed, period_ns=0.8)
    ls, rs = [1.0, 0.5, 2.0], [1.0, 2.0, 0.5]
    dk = dict(d)
    dk.update(n_corners=3, lut_scale=np.array(ls, np.float32), rc_scale=np.array(rs, np.float32))
    rk = oracle.sta(dk)
    for k in range(3):
        d1 = dict(d)
        d1["lut_val"] = (np.asarray(d["lut_val"], np.float32) * np.float32(ls[k])).astype(np.float32)
        if placed:
            d1["r_per_um"] = d["r_per_um"] * rs[k]
            d1["c_per_um"] = d["c_per_um"] * rs[k]
        else:
            d1["rc_R"] = (np.asarray(d["rc_R"], np.float32) * np.float32(rs[k])).astype(np.float32)
            d1["rc_C"] = (np.asarray(d["rc_C"], np.float32) * np.float32(rs[k])).astype(np.float32)
        r1 = oracle.sta(d1)
        for key in ("at", "slew", "rat", "slack"):
            np.testing.assert_allclose(rk[key][:, k], r1[key][:, 0], rtol=1e-13, atol=1e-15, err_msg=key)
        assert rk["tns_setup"][k] == pytest.approx(r1["tns_setup"][0], rel=1e-12)
        assert rk["tns_hold"][k] == pytest.approx(r1["tns_hold"][0], rel=1e-12)


# ----------------------------------------------------------- O6 the adjoint

def _single_path_design(x, y, gamma):
    lib = synth.make_library(0, fixed_delay=True)
    b = synth.Builder(lib)
    a = b.pi(xy=(0.0, 0.0))
    z = b.cell("BUF", [a], xy=(x, y))
    b.po(z, xy=(100.0, 0.0))
    return b.design(period_ns=0.05, placed=True, gamma_ns=gamma), lib


def test_adjoint_single_path_closed_form():
    """PI(0,0) -> BUF(x,y) -> PO(100,0), delays linear in load: J and dJ/dx
    written out by hand along the one path."""
    x, y, g = 37.0, 21.0, 0.01
    d, lib = _single_path_design(x, y, g)
    r_, c_ = 0.1, 0.2
    cap_buf = 1e3 * float(lib["pin_cap"].reshape(-1, 4)[1, 0])
    cap_po = 1e3 * float(lib["po_cap_pf"])
    val = lib["lut_val"].reshape(-1, 3, 4, 49)[1, 0].astype(float)
    l_ax = lib["lut_idx2"].reshape(-1, 3, 4, 7)[1, 0, 0].astype(float)

    def J_of(xx):
        L1 = abs(xx) + abs(y)
        L2 = abs(100.0 - xx) + abs(y)
        D1 = 1e-6 * r_ * L1 * (c_ * L1 / 2 + cap_buf)
        D2 = 1e-6 * r_ * L2 * (c_ * L2 / 2 + cap_po)
        load = 1e-3 * (c_ * L2 + cap_po)
        ats = []
        for tb in (0, 1):
            row = val[tb].reshape(7, 7)[0]
            j = int(np.clip(np.searchsorted(l_ax, load, side="right") - 1, 0, 5))
            dl = row[j] + (row[j + 1] - row[j]) * (load - l_ax[j]) / (l_ax[j + 1] - l_ax[j])
            ats.append(D1 + dl + D2)
        ys = [0.05 - at for at in ats]
        s = -g * np.log(sum(np.exp(-v / g) for v in ys))
        tns = -g * np.log1p(np.exp(-s / g)) if -s / g < 30 else s
        wns = s   # one endpoint: the smooth min over one value is itself
        return tns + wns

    J, terms, grad = oracle.objective_grad(d)
    assert J == pytest.approx(J_of(x), rel=1e-12)
    h = 1e-4
    fd = (J_of(x + h) - J_of(x - h)) / (2 * h)
    assert grad[0, 0] == pytest.approx(fd, rel=1e-6)


def _multi_fanin_design(gamma):
    """Gates with two to four arc candidates per output edge: NAND2 (two
    inputs, negative unate), XOR2 (non-unate: two edges per input), AOI21,
    MUX2 (unate data inputs, non-unate select) and a NOR2 after a flip-flop;
    slew-dependent tables (noise on)."""
    lib = synth.make_library(3)
    b = synth.Builder(lib)
    a, bb, c0 = b.pi(), b.pi(), b.pi()
    n1 = b.cell("NAND2", [a, bb])
    x1 = b.cell("XOR2", [n1, c0])
    o1 = b.cell("AOI21", [x1, n1, a])
    m1 = b.cell("MUX2", [o1, x1, bb])
    q = b.cell("DFF", [m1])
    z = b.cell("NOR2", [q, o1])
    b.po(z)
    b.po(m1)
    return b.design(period_ns=1.0, gamma_ns=gamma, default_R=40.0, default_C=3.0)


@pytest.mark.parametrize("gamma", [0.01, 0.003])
def test_smoothed_merges_match_independent_log_sum_exp(gamma):
    """Reading (differentiable mode, gamma > 0): every fan-in merge of
    arrivals and of slews is gamma log-sum-exp over the arc candidates
    (late; early the mirror).  Recomputed on gates with two to four
    candidates per edge by listing every candidate with the independent net
    sums and bilinear form and merging all at once with numpy's logaddexp --
    not the oracle's running max-shifted sum -- on a hand-built design and a
    generated one.  The smoothing is visible: the hard merges differ by far
    more than the tolerance."""
    for d in (_multi_fanin_design(gamma), synth.make_design(300, 10, seed=4, gamma_ns=gamma)):
        r = oracle.sta(d)
        at, sl = _indep.smoothed_forward(d, gamma)
        np.testing.assert_allclose(r["at"][:, 0, :], at, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(r["slew"][:, 0, :], sl, rtol=1e-12, atol=1e-14)
        hard = oracle.sta(dict(d, gamma_ns=0.0))
        assert np.max(np.abs(hard["at"][:, 0, :] - r["at"][:, 0, :])) > 1e-3


@pytest.mark.parametrize("resistive", [False, True])
def test_adjoint_matches_central_differences(resistive):
    """dJ/d(x, y) of the oracle's adjoint against central differences of its
    own smoothed objective, h = 1e-3 um, on random cells of a placed design.
    With resistive wires (R per um raised 10x) the wire variance is
    comparable to the slews, so the wire-slew terms of the adjoint carry a
    visible share of the gradient."""
    d = synth.make_design(400, 12, seed=21, placed=True, gamma_ns=0.01, period_ns=0.6)
    if resistive:
        d["r_per_um"] = 1.0
        d["gamma_ns"] = 0.0
        d["period_ns"] = 0.0
        req = -oracle.sta(d)["ep_setup"][:, 0]
        d["period_ns"] = float(np.quantile(req, 0.7))
        d["gamma_ns"] = 0.01
    J, _, g = oracle.objective_grad(d)
    rng = np.random.default_rng(0)
    cells = rng.choice(d["n_cells"], 40, replace=False)
    h = 1e-3
    bad = 0
    scale = np.abs(g).max()
    for c in cells:
        for ax in (0, 1):
            xy = d["cell_xy"].astype(np.float64).copy()

            def Jat(v):
                dd = dict(d)
                xy2 = xy.copy()
                xy2[2 * c + ax] = v
                dd["cell_xy"] = xy2.astype(np.float32)
                return oracle.objective(dd)
            v0 = float(d["cell_xy"][2 * c + ax])
            # fp32 positions: use a step the fp32 grid represents exactly
            vp, vm = np.float32(v0 + h), np.float32(v0 - h)
            fd = (Jat(vp) - Jat(vm)) / (float(vp) - float(vm))
            if abs(fd - g[c, ax]) > 1e-5 * abs(g[c, ax]) + 1e-6 * scale:
                bad += 1
    # a cell may straddle a breakpoint or a |dx| = 0 kink inside +-h: allow one
    assert bad <= 1, bad
    assert scale > 0


# ------------------------------------------------ O7 Arnoldi reduced order

def _random_tree(rng, n):
    par = [-1] + [int(rng.integers(0, i)) for i in range(1, n)]
    R = np.concatenate([[0.0], rng.uniform(5, 50, n - 1)])
    C_ = rng.uniform(0.5, 5, n)
    return par, R, C_


def _exact_t50(par, R, C_):
    """Unreduced step response of the RC tree, written out independently:
    nodal G (conductance, root grounded) and diagonal C, generalized
    eigenvectors with phi^T C phi = I, v(t) = 1 - Phi exp(-L t) Phi^T C 1,
    and the 50% crossing of every node by root bracketing."""
    import scipy.linalg
    import scipy.optimize
    n = len(par)
    m = n - 1
    G = np.zeros((m, m))
    for i in range(1, n):
        g = 1.0 / R[i]
        G[i - 1, i - 1] += g
        if par[i] > 0:
            p = par[i] - 1
            G[p, p] += g
            G[i - 1, p] -= g
            G[p, i - 1] -= g
    Cm = np.diag(np.asarray(C_[1:], float))
    lam, phi = scipy.linalg.eigh(G, Cm)
    coef = phi.T @ Cm @ np.ones(m)
    out = np.zeros(n)
    for i in range(1, n):
        w = phi[i - 1] * coef

        def v(t):
            return 1.0 - np.sum(w * np.exp(-lam * t)) - 0.5
        hi = 1.0 / lam.min()
        while v(hi) < 0:
            hi *= 2
        out[i] = scipy.optimize.brentq(v, 0.0, hi, xtol=1e-14, rtol=1e-14)
    return out


def test_arnoldi_single_rc_closed_form():
    """One R, one C: v(t) = 1 - exp(-t / RC), so t50 = RC ln 2 at any order."""
    for q in (1, 2, 3):
        t = oracle.arnoldi_t50([-1, 0], [0.0, 12.5], [0.0, 3.2], q)
        assert t[1] == pytest.approx(12.5 * 3.2 * np.log(2), rel=1e-12)
    # identical branches off the driver: each is that single RC, and the
    # Krylov space stops at one direction (the exhausted-space path)
    t = oracle.arnoldi_t50([-1, 0, 0, 0], [0.0, 12.5, 12.5, 12.5], [0.0, 3.2, 3.2, 3.2], 3)
    np.testing.assert_allclose(t[1:], 12.5 * 3.2 * np.log(2), rtol=1e-12)


def test_arnoldi_first_order_is_the_lumped_pole():
    """q = 1 projects on the DC vector (all ones): one pole G_r / C_r =
    (sum of the root's edge conductances) / (total capacitance), the same
    t50 = ln 2 / pole at every node."""
    rng = np.random.default_rng(3)
    for n in (3, 7, 12):
        par, R, C_ = _random_tree(rng, n)
        g = sum(1.0 / R[i] for i in range(1, n) if par[i] == 0)
        want = np.log(2) * C_[1:].sum() / g
        np.testing.assert_allclose(oracle.arnoldi_t50(par, R, C_, 1)[1:], want, rtol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 6, 11, 16])
def test_arnoldi_full_order_is_the_exact_response(n):
    """With q = n - 1 the Krylov space is the whole space: the reduced model
    is the unreduced network, so t50 matches the independent generalized
    eigen-solution."""
    rng = np.random.default_rng(n)
    par, R, C_ = _random_tree(rng, n)
    np.testing.assert_allclose(oracle.arnoldi_t50(par, R, C_, n - 1), _exact_t50(par, R, C_), rtol=1e-9, atol=1e-12)


def test_arnoldi_bounded_by_elmore_and_converging():
    """The Elmore delay bounds the exact 50% step delay of an RC tree from
    above.  The reduced model approaches the exact response as q grows,
    measured against each net's largest delay.  Nodes next to the driver see
    fast poles a low order cannot resolve, so per-node relative error is not
    the measure.  Over 40 random trees of 4-16 nodes the worst error falls
    with q, order 3 is below 12% and order 5 below 3%, and order 3 is never
    worse than order 1 on any tree."""
    rng = np.random.default_rng(11)
    worst = np.zeros(5)
    for _ in range(40):
        n = int(rng.integers(4, 17))
        par, R, C_ = _random_tree(rng, n)
        exact = _exact_t50(par, R, C_)
        elm = oracle.rc_tree(par, R, C_)[1]
        assert np.all(exact[1:] <= elm[1:] * (1 + 1e-12))
        err = [np.abs(oracle.arnoldi_t50(par, R, C_, q)[1:] - exact[1:]).max() / exact.max() for q in (1, 2, 3, 4, 5)]
        assert err[2] <= err[0]
        worst = np.maximum(worst, err)
    assert np.all(np.diff(worst) < 0)
    assert worst[2] < 0.12 and worst[4] < 0.03


def test_arnoldi_net_model_in_the_analysis():
    """net_model = 1 replaces each sink's Elmore delay by the tree's t50 of
    the chosen order; loads and variances are unchanged."""
    d = synth.make_design(200, 8, seed=6, rc_nodes=(2, 12))
    da = dict(d, net_model=1, arnoldi_order=3)
    L0, D0, V0 = oracle.net_delays(d)
    L1, D1, V1 = oracle.net_delays(da)
    np.testing.assert_array_equal(L0, L1)
    np.testing.assert_array_equal(V0, V1)
    npp, npn = d["net_pin_ptr"], d["net_pin"]
    pins_cap = np.asarray(d["pin_cap"]).reshape(-1, 4)
    net = _indep.Net(d)
    for n in range(0, d["n_nets"], 17):
        r0, r1 = d["rc_ptr"][n], d["rc_ptr"][n + 1]
        C_ = np.asarray(d["rc_C"][r0:r1], float).copy()
        R = np.asarray(d["rc_R"][r0:r1], float)
        par = np.asarray(d["rc_parent"][r0:r1])
        for k in range(npp[n] + 1, npp[n + 1]):
            s = npn[k]
            role = d["pin_role"][s]
            cap = d["po_cap_pf"] if role == synth.PO else pins_cap[d["cell_type"][net.cell_of[s]], net.slot_of[s]]
            C_[d["rc_pin_node"][k]] += 1e3 * float(cap)
        t = oracle.arnoldi_t50(par, R, C_, 3)
        for k in range(npp[n] + 1, npp[n + 1]):
            assert D1[npn[k]] == pytest.approx(1e-6 * t[d["rc_pin_node"][k]], rel=1e-12)
    assert np.all(D1[D0 > 0] < D0[D0 > 0])
    r = oracle.sta(da)
    assert np.isfinite(r["tns_setup"][0])


# ------------------------------------------------------- top-k path report

def _arc_ok(d, net, u, ru, v, rv):
    """u -> v is a timing arc with edges ru -> rv (net arc: same edge)."""
    role = np.asarray(d["pin_role"])
    if net.driver.get(v) == u:
        return ru == rv
    c = net.cell_of[v]
    if c < 0 or net.cell_of[u] != c:
        return False
    t = d["cell_type"][c]
    se = np.asarray(d["arc_sense"]).reshape(-1, 3)[t, net.slot_of[u]]
    if role[v] == synth.Q:
        return se == _indep.RISE and ru == 0
    return ru in _indep.rf_in_of(se, rv)


@pytest.mark.parametrize("seed", range(4))
def test_paths_are_longest_paths_fixed_delay(seed):
    """With slew-independent delays every reported path is made of timing
    arcs with consistent edges, and it is a longest path: its arrival at the
    endpoint equals the maximum over all enumerated paths ending there with
    that edge, and the late arrival along it is the path's own prefix sum."""
    d = _fixed_design(seed, n_cells=12, depth=5)
    d["period_ns"] = 0.3
    res = oracle.sta(d)
    allp = _indep.enumerate_paths(d)
    net = _indep.Net(d)
    paths = oracle.report_paths(d, 50, res=res)
    assert len(paths) > 0
    for pth in paths:
        pins, rfs, at = pth["pins"], pth["rf"], pth["at"]
        e = pins[-1]
        assert e == pth["endpoint"]
        assert np.asarray(d["pin_role"])[pins[0]] in (synth.PI, synth.CK)
        for (u, ru), (v, rv) in zip(zip(pins[:-1], rfs[:-1]), zip(pins[1:], rfs[1:])):
            assert _arc_ok(d, net, int(u), int(ru), int(v), int(rv)), (u, v)
        best = max(a for a, _, f in allp[e] if f == rfs[-1])
        assert at[-1] == pytest.approx(best, abs=1e-12)
        # every prefix is tight: arrival = predecessor's arrival + arc delay
        for i in range(1, len(pins)):
            v, u = int(pins[i]), int(pins[i - 1])
            if net.driver.get(v) == u:
                assert at[i] == pytest.approx(at[i - 1] + net.Dns[v], abs=1e-12)
        assert pth["slack"] == pytest.approx(res["rat"][e, 0, 2 + rfs[-1]] - at[-1], abs=1e-12)


def test_paths_order_threshold_and_count():
    """Endpoints by increasing setup slack (ties by index), only those below
    the threshold, at most k of them."""
    d = synth.make_design(800, 12, seed=3, period_ns=0.9)
    res = oracle.sta(d)
    es = res["ep_setup"][:, 0]
    for k, thr in ((10, np.inf), (1000, 0.0), (5, -0.2)):
        paths = oracle.report_paths(d, k, slack_lt=thr, res=res)
        want = sorted((e for e in range(len(es)) if es[e] < thr), key=lambda e: (es[e], e))[:k]
        assert [p["endpoint"] for p in paths] == [int(res["endpoints"][e]) for e in want]
        assert all(p["slack"] < thr for p in paths)


# ------------------------------------------------------- O8 timing exceptions

@pytest.mark.parametrize("seed,actions", [(0, None), (1, None), (2, None), (3, None), (4, None),
                                          (5, (0, 1, 2, 3)), (6, (2, 3)), (7, (1, 2, 3))])
def test_exceptions_brute_force_fixed_delay(seed, actions):
    """Every path tagged by its startpoint's first group: an endpoint's setup
    slack is the minimum over the paths ending there of (requirement -
    arrival) and its hold slack the minimum of (arrival - requirement), with
    the tag's requirement -- the group's action when the endpoint is in its
    list (or the list is empty): false path removes the check, multicycle M
    moves the setup capture edge to M * T, max delay V moves it to V, min
    delay V moves the hold edge to V -- and the default otherwise."""
    rng = np.random.default_rng(seed)
    d = _fixed_design(seed, n_cells=14, depth=5)
    d["period_ns"] = 0.35
    d.update(synth.exception_groups(d, rng, 3, actions=actions))
    res = oracle.sta(d)
    role = np.asarray(d["pin_role"])
    first = {}
    for g in range(3):
        for p in d["exc_from"][d["exc_from_ptr"][g]:d["exc_from_ptr"][g + 1]]:
            first.setdefault(int(p), g)
    T = d["period_ns"]
    allp = _indep.enumerate_paths_from(d)
    for e, p in enumerate(res["endpoints"]):
        setup = hold = np.inf
        for a, rf, s in allp[p]:
            late = T - d["setup_ns"] if role[p] == synth.D else T
            early = d["hold_ns"] if role[p] == synth.D else 0.0
            g = first.get(s)
            if g is not None:
                lst = d["exc_to"][d["exc_to_ptr"][g]:d["exc_to_ptr"][g + 1]]
                if len(lst) == 0 or p in lst:
                    act, v = d["exc_action"][g], float(d["exc_mult"][g])
                    if act == 0:
                        late, early = np.inf, -np.inf
                    elif act == 1:
                        late = v * T - d["setup_ns"] if role[p] == synth.D else v * T
                    elif act == 2:
                        late = v - d["setup_ns"] if role[p] == synth.D else v
                    else:
                        early = v + d["hold_ns"] if role[p] == synth.D else v
            setup = min(setup, late - a)
            hold = min(hold, a - early)
        assert res["ep_setup"][e, 0] == pytest.approx(setup, abs=1e-12), (e, p)
        assert res["ep_hold"][e, 0] == pytest.approx(hold, abs=1e-12), (e, p)
    assert res["at"].shape[1] == 4                     # one corner x (3 groups + 1) tags


def test_exceptions_all_false_and_all_multicycle():
    """Every startpoint in one false-path group: no check anywhere, WNS = TNS
    = 0.  Every startpoint in one multicycle-M group: every setup slack moves
    by exactly (M - 1) * T, hold slacks do not move."""
    d = synth.make_design(600, 10, seed=5, period_ns=0.7)
    role = np.asarray(d["pin_role"])
    starts = np.nonzero((role == synth.PI) | (role == synth.CK))[0].astype(np.int32)
    base = oracle.sta(d)
    grp = dict(exc_from_ptr=np.array([0, len(starts)], np.int32), exc_from=starts,
               exc_to_ptr=np.array([0, 0], np.int32), exc_to=np.zeros(0, np.int32))
    r = oracle.sta(dict(d, exc_action=np.array([0], np.int32), exc_mult=np.array([1], np.float32), **grp))
    assert np.all(np.isinf(r["ep_setup"])) and np.all(np.isinf(r["ep_hold"]))
    assert r["wns_setup"][0] == 0 and r["tns_setup"][0] == 0 and r["tns_hold"][0] == 0
    r = oracle.sta(dict(d, exc_action=np.array([1], np.int32), exc_mult=np.array([3], np.float32), **grp))
    np.testing.assert_allclose(r["ep_setup"], base["ep_setup"] + 2 * d["period_ns"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(r["ep_hold"], base["ep_hold"])
    # every startpoint in one max-delay-V group: setup slacks move by V - T; one min-delay-V group: hold by -V
    V = np.float32(0.45)
    r = oracle.sta(dict(d, exc_action=np.array([2], np.int32), exc_mult=np.array([V], np.float32), **grp))
    np.testing.assert_allclose(r["ep_setup"], base["ep_setup"] + float(V) - d["period_ns"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(r["ep_hold"], base["ep_hold"])
    r = oracle.sta(dict(d, exc_action=np.array([3], np.int32), exc_mult=np.array([V], np.float32), **grp))
    np.testing.assert_allclose(r["ep_hold"], base["ep_hold"] - float(V), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(r["ep_setup"], base["ep_setup"])


@pytest.mark.parametrize("seed,max_thru", [(0, 0), (1, 0), (2, 0), (3, 2), (4, 2)])
def test_exception_paths_fixed_delay(seed, max_thru):
    """With exceptions the reported path is the one that sets the endpoint's
    slack: it starts at a startpoint s, its arrival at the endpoint is an
    enumerated path arrival from s, and (late requirement of its group's
    match at the endpoint) - arrival equals the endpoint's slack, the minimum
    over every enumerated tagged path.  With -through sets, a path's match
    also needs its gate input pins to pass the group's sets in order."""
    rng = np.random.default_rng(50 + seed)
    d = _fixed_design(seed, n_cells=14, depth=5)
    d["period_ns"] = 0.35
    d.update(synth.exception_groups(d, rng, 3, max_thru=max_thru, div_thru=3))
    res = oracle.sta(d)
    role = np.asarray(d["pin_role"])
    first = {}
    for g in range(3):
        for p in d["exc_from"][d["exc_from_ptr"][g]:d["exc_from_ptr"][g + 1]]:
            first.setdefault(int(p), g)
    T = d["period_ns"]

    def late_req(p, s, ins):
        base = T - d["setup_ns"] if role[p] == synth.D else T
        g = first.get(int(s))
        if g is None or (max_thru and not _through_matched(d, g, ins)):
            return base
        lst = d["exc_to"][d["exc_to_ptr"][g]:d["exc_to_ptr"][g + 1]]
        if len(lst) and p not in lst:
            return base
        if d["exc_action"][g] == 0:
            return np.inf
        M = float(d["exc_mult"][g])
        return M * T - d["setup_ns"] if role[p] == synth.D else M * T

    allp = _indep.enumerate_paths_from(d, with_pins=True)
    paths = oracle.report_paths(d, 100, res=res)
    assert len(paths) == int(np.sum(res["ep_setup"][:, 0] < np.inf))
    for pth in paths:
        e, s, rf = int(pth["endpoint"]), int(pth["pins"][0]), int(pth["rf"][-1])
        want = min(late_req(e, s2, ins) - a for a, _, s2, ins in allp[e])
        assert pth["slack"] == pytest.approx(want, abs=1e-12)
        ins = tuple(int(q) for q in pth["pins"] if role[q] == synth.IN)
        arrivals = [a for a, f, s2, ins2 in allp[e] if s2 == s and f == rf and ins2 == ins]
        assert min(abs(a - pth["at"][-1]) for a in arrivals) <= 1e-12
        assert late_req(e, s, ins) - pth["at"][-1] == pytest.approx(want, abs=1e-12)


# --------------------------------------------------- O9 Steiner RC from positions

def _read_steiner_golden():
    g = {"nm": []}
    for line in open(os.path.join(GOLD, "steiner_hand.txt")):
        f = line.split("#")[0].split()
        if not f:
            continue
        if f[0] == "nm":
            g["nm"].append((float(f[1]), int(f[2])))
        else:
            g[f[0]] = [float(x) for x in f[1:]]
    return g


def _hanan_rsmt(X, Y):
    """Exact rectilinear Steiner minimal tree length by brute force: by
    Hanan's theorem some RSMT has its Steiner points on the Hanan grid and
    needs at most n - 2 of them, so the minimum over those subsets of the
    rectilinear MST length (scipy) is the RSMT length."""
    from itertools import combinations

    from scipy.sparse.csgraph import minimum_spanning_tree
    pts = sorted(set(zip(X, Y)))   # coincident pins join at no cost
    grid = [(x, y) for x in sorted(set(X)) for y in sorted(set(Y)) if (x, y) not in pts]

    def mst(ps):
        a = np.array(ps, np.float64)
        dm = np.abs(a[:, None, 0] - a[None, :, 0]) + np.abs(a[:, None, 1] - a[None, :, 1])
        return float(minimum_spanning_tree(dm).sum())

    best = mst(pts)
    for k in range(1, len(pts) - 1):
        for sub in combinations(grid, k):
            best = min(best, mst(pts + list(sub)))
    return best


def _tree_checks(X, Y, t):
    """A tree on the pins: breadth-first numbering, every pin on its own
    node, Steiner nodes with at least three neighbours on the Hanan grid,
    and wl the sum of the edges' Manhattan lengths."""
    par, nx, ny, pn = t["parent"], t["nx"], t["ny"], t["pin_node"]
    n = len(X)
    assert par[0] == -1 and all(0 <= par[i] < i for i in range(1, len(par)))
    assert pn[0] == 0
    for j in range(n):
        assert (nx[pn[j]], ny[pn[j]]) == (X[j], Y[j])
    for i in range(n):   # pins share a node exactly when they sit at the same point
        for j in range(i + 1, n):
            assert (pn[i] == pn[j]) == ((X[i], Y[i]) == (X[j], Y[j]))
    deg = np.bincount(par[1:], minlength=len(par)) + (np.arange(len(par)) > 0)
    steiner = sorted(set(range(len(par))) - set(pn.tolist()))
    assert all(deg[s] >= 3 for s in steiner)
    assert all(nx[s] in set(X) and ny[s] in set(Y) for s in steiner)
    assert len(par) <= max(1, 2 * n - 2)
    wl = sum(abs(nx[i] - nx[par[i]]) + abs(ny[i] - ny[par[i]]) for i in range(1, len(par)))
    assert wl == t["wl"]
    # a Steiner node never sits on a neighbour, and no median insertion or
    # reattachment can shorten the final tree (the greedy stops at zero gain)
    nbr = [[] for _ in par]
    for i in range(1, len(par)):
        nbr[i].append(par[i])
        nbr[par[i]].append(i)
    dist = lambda a, b: abs(int(nx[a]) - int(nx[b])) + abs(int(ny[a]) - int(ny[b]))  # noqa: E731
    assert all(dist(i, par[i]) > 0 for i in range(1, len(par)))   # no zero-length edge
    if n <= 64:
        for u in range(len(par)):
            for i, v in enumerate(nbr[u]):
                for w in nbr[u][i + 1:]:
                    mx = sorted([nx[u], nx[v], nx[w]])[1]
                    my = sorted([ny[u], ny[v], ny[w]])[1]
                    m = lambda a: abs(int(nx[a]) - int(mx)) + abs(int(ny[a]) - int(my))  # noqa: E731
                    assert dist(u, v) + dist(u, w) - m(u) - m(v) - m(w) <= 0


def test_steiner_nm_rounding():
    g = _read_steiner_golden()
    assert len(g["nm"]) >= 5
    for x, want in g["nm"]:
        assert oracle.nm(x) == want, x


def test_steiner_hand_worked_T_net():
    """The T net of the golden file: tree, wirelength, and the Elmore delay,
    variance and load of its RC with different unit R/C along x and y."""
    g = _read_steiner_golden()
    p = [int(v) for v in g["tpins"]]
    X, Y = p[0::2], p[1::2]
    t = oracle.steiner_tree(X, Y)
    np.testing.assert_array_equal(t["parent"], np.array(g["tparent"], int))
    nodes = [int(v) for v in g["tnodes"]]
    np.testing.assert_array_equal(t["nx"], nodes[0::2])
    np.testing.assert_array_equal(t["ny"], nodes[1::2])
    np.testing.assert_array_equal(t["pin_node"], np.array(g["tpinnode"], int))
    assert t["wl"] == int(g["twl"][0])
    rx, ry, cx, cy, cpo = g["tunits"]
    lib = synth.make_library(0)
    b = synth.Builder(lib)
    a = b.pi(xy=(0.0, 0.0))
    s1 = b.po(a, xy=(100.0, 40.0))
    s2 = b.po(a, xy=(100.0, -40.0))
    d = b.design(placed=True, r_per_um=rx, c_per_um=cx)
    d.update(wire_model=1, r_per_um_y=ry, c_per_um_y=cy, po_cap_pf=cpo)
    load, Dn, Vn = oracle.net_delays(d)
    assert load[a] == pytest.approx(g["tload"][0], rel=1e-12)
    for s in (s1, s2):
        assert Dn[s] == pytest.approx(g["tdelay"][0], rel=1e-12)
        assert Vn[s] == pytest.approx(g["tvar"][0], rel=1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_steiner_two_and_three_pins_optimal(seed):
    """Two pins: the Manhattan distance.  Three pins: the half perimeter of
    the bounding box (the RSMT of three points), also on a small grid where
    distance ties and coincident pins are common."""
    rng = np.random.default_rng(seed)
    for hi in (5, 1000):
        for _ in range(300):
            X, Y = rng.integers(0, hi, 2), rng.integers(0, hi, 2)
            t = oracle.steiner_tree(X, Y)
            _tree_checks(X, Y, t)
            assert t["wl"] == abs(X[0] - X[1]) + abs(Y[0] - Y[1])
            X, Y = rng.integers(0, hi, 3), rng.integers(0, hi, 3)
            t = oracle.steiner_tree(X, Y)
            _tree_checks(X, Y, t)
            assert t["wl"] == (X.max() - X.min()) + (Y.max() - Y.min())


def test_steiner_bounded_by_rsmt_and_rmst():
    """RSMT <= WL <= RMST (so WL <= 1.5 RSMT, Hwang's bound on the RMST);
    the RSMT by brute force over the Hanan grid, the RMST by scipy.  Also
    reports how close the construction gets on 4- and 5-pin nets."""
    from scipy.sparse.csgraph import minimum_spanning_tree
    rng = np.random.default_rng(7)
    ratios = []
    for n, reps in ((4, 100), (5, 12)):
        for _ in range(reps):
            X, Y = rng.integers(0, 50, n), rng.integers(0, 50, n)
            t = oracle.steiner_tree(X, Y)
            _tree_checks(X, Y, t)
            u = np.array(sorted(set(zip(X.tolist(), Y.tolist()))), np.float64)
            dm = np.abs(u[:, None, 0] - u[None, :, 0]) + np.abs(u[:, None, 1] - u[None, :, 1])
            rmst = round(float(minimum_spanning_tree(dm).sum()))
            rsmt = _hanan_rsmt(X.tolist(), Y.tolist())
            assert rsmt - 1e-6 <= t["wl"] <= rmst
            ratios.append(t["wl"] / rsmt)
    assert max(ratios) <= 1.5
    assert np.mean(ratios) < 1.03   # close to optimal on small nets


def test_steiner_large_nets_valid():
    """Nets up to 64 pins are Steinerised (WL below the RMST on random
    points); larger nets keep the MST."""
    from scipy.sparse.csgraph import minimum_spanning_tree
    rng = np.random.default_rng(3)
    for _ in range(150):   # small grids: distance ties, coincident pins, reattachments
        n = int(rng.integers(6, 13))
        X, Y = rng.integers(0, 12, n), rng.integers(0, 12, n)
        _tree_checks(X, Y, oracle.steiner_tree(X, Y))
    for n in (10, 37, 64, 65, 90):
        X, Y = rng.integers(0, 10**6, n), rng.integers(0, 10**6, n)
        t = oracle.steiner_tree(X, Y)
        _tree_checks(X, Y, t)
        dm = (np.abs(X[:, None] - X[None, :]) + np.abs(Y[:, None] - Y[None, :])).astype(float)
        rmst = round(float(minimum_spanning_tree(dm).sum()))
        if n <= 64:
            assert t["wl"] < rmst
        else:
            assert t["wl"] == rmst and len(t["parent"]) == n


def test_steiner_rc_matches_shared_path_and_corner_prescale():
    """Steiner RC in a generated placed design: every sink's Elmore delay and
    variance equal the shared-path sums over an RC tree rebuilt here from the
    O9 tree (edge R = rx Lx + ry Ly, wire C split half at each end), and
    corner k equals a single-corner design with unit R/C pre-scaled by
    rc_scale[k]."""
    d = synth.make_design(400, 8, seed=12, placed=True)
    d.update(wire_model=1, r_per_um_y=0.13, c_per_um_y=0.25, n_corners=2,
             lut_scale=np.array([1.0, 1.0], np.float32), rc_scale=np.array([1.0, 1.3], np.float32))
    rx, cx, ry, cy = d["r_per_um"], d["c_per_um"], 0.13, 0.25
    load, Dn, Vn = oracle.net_delays(d, 0)
    net = _indep.Net(dict(d, wire_model=0))   # pin positions and caps only
    npp, npn = d["net_pin_ptr"], d["net_pin"]
    checked = 0
    for m in range(d["n_nets"]):
        pins = npn[npp[m]:npp[m + 1]]
        if len(pins) < 3:
            continue
        xy = [net.pos(int(p)) for p in pins]
        X = [oracle.nm(x) for x, _ in xy]
        Y = [oracle.nm(y) for _, y in xy]
        t = oracle.steiner_tree(X, Y)
        par, nx, ny = t["parent"], t["nx"], t["ny"]
        k = len(par)
        R, Cc = np.zeros(k), np.zeros(k)
        for i in range(1, k):
            lx, ly = abs(nx[i] - nx[par[i]]) * 1e-3, abs(ny[i] - ny[par[i]]) * 1e-3
            R[i] = rx * lx + ry * ly
            Cc[i] += 0.5 * (cx * lx + cy * ly)
            Cc[par[i]] += 0.5 * (cx * lx + cy * ly)
        for j, p in enumerate(pins[1:], 1):
            Cc[t["pin_node"][j]] += 1e3 * net.cap(int(p))
        Dm, beta = _indep.shared_path_moments(par, R, Cc)
        assert load[pins[0]] == pytest.approx(1e-3 * Cc.sum(), rel=1e-12)
        for j, p in enumerate(pins[1:], 1):
            nd = t["pin_node"][j]
            assert Dn[p] == pytest.approx(1e-6 * Dm[nd], rel=1e-11)
            assert Vn[p] == pytest.approx(1e-12 * (2 * beta[nd] - Dm[nd] ** 2), rel=1e-8, abs=1e-22)
        checked += 1
        if checked > 60:
            break
    assert checked > 20
    f = float(np.float32(1.3))   # the corner's scale as stored
    d1 = dict(d, n_corners=1, lut_scale=np.ones(1, np.float32), rc_scale=np.ones(1, np.float32),
              r_per_um=f * rx, c_per_um=f * cx, r_per_um_y=f * ry, c_per_um_y=f * cy)
    l1, D1, V1 = oracle.net_delays(d, 1)
    l2, D2, V2 = oracle.net_delays(d1, 0)
    np.testing.assert_allclose(l1, l2, rtol=1e-12)
    np.testing.assert_allclose(D1, D2, rtol=1e-12)
    np.testing.assert_allclose(V1, V2, rtol=1e-9, atol=1e-24)


def test_net_wirelengths_match_per_net_trees():
    """The per-net tree lengths of a placed design equal the single-net
    trees built from its pins' nm coordinates (driver first)."""
    d = synth.make_design(300, 6, seed=2, placed=True)
    wl = oracle.net_wirelengths(d)
    net = _indep.Net(d)
    npp, npn = d["net_pin_ptr"], d["net_pin"]
    for m in range(d["n_nets"]):
        xy = [net.pos(int(p)) for p in npn[npp[m]:npp[m + 1]]]
        t = oracle.steiner_tree([oracle.nm(x) for x, _ in xy], [oracle.nm(y) for _, y in xy])
        assert wl[m] == t["wl"]


def _through_matched(d, g, ins_pins):
    """The path's gate input pins pass group g's through sets in order
    (greedy earliest match, which decides a subsequence of sets)."""
    tp, tsp, tpin = d["exc_thru_ptr"], d["exc_thru_set_ptr"], d["exc_thru_pin"]
    j, r = 0, tp[g + 1] - tp[g]
    for p in ins_pins:
        if j < r:
            s = tp[g] + j
            if p in set(int(x) for x in tpin[tsp[s]:tsp[s + 1]]):
                j += 1
    return j == r


@pytest.mark.parametrize("seed", range(6))
def test_exceptions_through_brute_force(seed):
    """-through: a path of group g (its startpoint's first group) gets g's
    action only if its gate input pins pass g's through sets in order and it
    ends in g's list; every endpoint's setup and hold slack is the minimum
    over its enumerated paths of that path's requirement - arrival."""
    rng = np.random.default_rng(200 + seed)
    d = _fixed_design(seed, n_cells=16, depth=5)
    d["period_ns"] = 0.35
    d.update(synth.exception_groups(d, rng, 3, max_thru=2, div_thru=3))
    assert d["exc_thru_ptr"][-1] > 0
    res = oracle.sta(d)
    assert res["at"].shape[1] == oracle.n_tags(d)
    role = np.asarray(d["pin_role"])
    first = {}
    for g in range(3):
        for p in d["exc_from"][d["exc_from_ptr"][g]:d["exc_from_ptr"][g + 1]]:
            first.setdefault(int(p), g)
    T = d["period_ns"]
    allp = _indep.enumerate_paths_from(d, with_pins=True)
    matched_any = 0
    for e, p in enumerate(res["endpoints"]):
        setup = hold = np.inf
        for a, rf, s, ins in allp[p]:
            late = T - d["setup_ns"] if role[p] == synth.D else T
            early = d["hold_ns"] if role[p] == synth.D else 0.0
            g = first.get(s)
            if g is not None and _through_matched(d, g, ins):
                lst = d["exc_to"][d["exc_to_ptr"][g]:d["exc_to_ptr"][g + 1]]
                if len(lst) == 0 or p in lst:
                    matched_any += 1
                    if d["exc_action"][g] == 0:
                        late, early = np.inf, -np.inf
                    else:
                        late = float(d["exc_mult"][g]) * T - d["setup_ns"] if role[p] == synth.D \
                            else float(d["exc_mult"][g]) * T
            setup = min(setup, late - a)
            hold = min(hold, a - early)
        assert res["ep_setup"][e, 0] == pytest.approx(setup, abs=1e-12), (e, p)
        assert res["ep_hold"][e, 0] == pytest.approx(hold, abs=1e-12), (e, p)
    assert matched_any > 0


def test_exceptions_through_every_pin_equals_plain_group():
    """A through set holding every gate input pin is passed by every path
    that crosses a gate: with one such set, the group acts exactly like the
    group without -through on every endpoint reached through a gate."""
    d = synth.make_design(500, 8, seed=6, period_ns=0.7)
    rng = np.random.default_rng(1)
    g1 = synth.exception_groups(d, rng, 2)
    role = np.asarray(d["pin_role"])
    ins = np.nonzero(role == synth.IN)[0].astype(np.int32)
    thru = dict(exc_thru_ptr=np.array([0, 1, 1], np.int32), exc_thru_set_ptr=np.array([0, len(ins)], np.int32),
                exc_thru_pin=ins)
    r0 = oracle.sta(dict(d, **g1))
    r1 = oracle.sta(dict(d, **g1, **thru))
    # endpoints driven straight from a startpoint (no gate) may differ; all others agree
    npp, npn = d["net_pin_ptr"], d["net_pin"]
    drv = {int(s): int(npn[npp[n]]) for n in range(d["n_nets"]) for s in npn[npp[n] + 1:npp[n + 1]]}
    direct = np.array([role[drv[int(p)]] in (synth.PI, synth.Q) for p in r0["endpoints"]])
    assert (~direct).sum() > 10
    np.testing.assert_allclose(r1["ep_setup"][~direct], r0["ep_setup"][~direct], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r1["ep_hold"][~direct], r0["ep_hold"][~direct], rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_exceptions_through_required_times_brute_force(seed):
    """Required times per tag with -through: at every pin and tag t, the late
    required time is the minimum over the path suffixes to an endpoint of
    (requirement of the tag the suffix ends in - suffix delay), the tag
    advancing at each gate input of the suffix that is in its group's next
    through set (the early one the maximum, likewise)."""
    rng = np.random.default_rng(300 + seed)
    d = _fixed_design(seed, n_cells=14, depth=5)
    d["period_ns"] = 0.35
    d.update(synth.exception_groups(d, rng, 2, max_thru=2, div_thru=3))
    res = oracle.sta(d)
    base, _ = oracle.tag_layout(d)
    tp, tsp, tpin = d["exc_thru_ptr"], d["exc_thru_set_ptr"], d["exc_thru_pin"]
    role = np.asarray(d["pin_role"])
    T = d["period_ns"]
    Tg = oracle.n_tags(d)
    group_of = {}
    for g in range(2):
        for j in range(tp[g + 1] - tp[g] + 1):
            group_of[base[g] + j] = (g, j)

    def final(t, ins):   # (group, fully matched) after the suffix's gate inputs
        if t == 0:
            return None, False
        g, j = group_of[t]
        r = tp[g + 1] - tp[g]
        for p in ins:
            if j < r and p in set(int(x) for x in tpin[tsp[tp[g] + j]:tsp[tp[g] + j + 1]]):
                j += 1
        return g, j == r

    def reqs(e, t, ins):
        late = T - d["setup_ns"] if role[e] == synth.D else T
        early = d["hold_ns"] if role[e] == synth.D else 0.0
        g, full = final(t, ins)
        if full:
            lst = d["exc_to"][d["exc_to_ptr"][g]:d["exc_to_ptr"][g + 1]]
            if len(lst) == 0 or e in lst:
                if d["exc_action"][g] == 0:
                    return np.inf, -np.inf
                M = float(d["exc_mult"][g])
                late = M * T - d["setup_ns"] if role[e] == synth.D else M * T
        return late, early

    suf = _indep.enumerate_suffixes(d, with_pins=True)
    for p in range(d["n_pins"]):
        for t in range(Tg):
            for rf in (0, 1):
                late = min([reqs(e, t, ins)[0] - dl for dl, r, e, ins in suf[p] if r == rf], default=np.inf)
                early = max([reqs(e, t, ins)[1] - dl for dl, r, e, ins in suf[p] if r == rf], default=-np.inf)
                assert res["rat"][p, t, 2 + rf] == pytest.approx(late, abs=1e-12), (p, t, rf)
                assert res["rat"][p, t, rf] == pytest.approx(early, abs=1e-12), (p, t, rf)


# ------------------------------------------- O6 on Steiner trees (O9 + O3)

def test_rc_tree_adjoint_matches_central_differences():
    """dJ/dR and dJ/dC of orc_rc_tree_adjoint against central differences of
    J = sum_i (Dbar_i D_i + Vbar_i var_i) + Lbar Cdown_0 through the forward
    orc_rc_tree, on random trees of 1-24 nodes (a chain and a star among
    them).  J is quadratic in any single R_i or C_i, so a central difference
    is exact up to rounding at any step."""
    rng = np.random.default_rng(5)
    shapes = [None] * 20 + ["chain", "star"]
    for k, shape in enumerate(shapes):
        n = int(rng.integers(1, 25)) if shape is None else 9
        par, R, C_ = _random_tree(rng, n)
        if shape == "chain":
            par = [-1] + list(range(n - 1))
        elif shape == "star":
            par = [-1] + [0] * (n - 1)
        Db, Vb = rng.normal(size=n), rng.normal(size=n)
        Lb = float(rng.normal())

        def J(R_, C2):
            cd, D, _, var = oracle.rc_tree(par, R_, C2)
            return float(Db @ D + Vb @ var + Lb * cd[0])
        Rb, Cb = oracle.rc_tree_adjoint(par, R, C_, Db, Vb, Lb)
        assert Rb[0] == 0.0
        for i in range(n):
            for arr, bar, skip0 in ((R, Rb, True), (C_, Cb, False)):
                if skip0 and i == 0:
                    continue
                h = 0.1 * arr[i]
                up, dn = arr.copy(), arr.copy()
                up[i] += h
                dn[i] -= h
                fd = (J(up, C_) - J(dn, C_)) / (2 * h) if arr is R else (J(R, up) - J(R, dn)) / (2 * h)
                assert bar[i] == pytest.approx(fd, rel=1e-7, abs=1e-9), (k, i)


def _pin_positions(d):
    """um position of every pin (cell pins at their cell, ports at port_xy)."""
    P = int(d["n_pins"])
    cell_of = np.full(P, -1, np.int64)
    cp = np.asarray(d["cell_pin_ptr"])
    for c in range(int(d["n_cells"])):
        cell_of[np.asarray(d["cell_pin"])[cp[c]:cp[c + 1]]] = c
    xy = np.asarray(d["cell_xy"], np.float32).reshape(-1, 2)
    pxy = np.asarray(d["port_xy"], np.float32).reshape(-1, 2)
    out = np.where(cell_of[:, None] >= 0, xy[np.maximum(cell_of, 0)], pxy[:P])
    return out.astype(np.float32), cell_of


def _net_trees(d, nets):
    pos, _ = _pin_positions(d)
    ptr, pins = np.asarray(d["net_pin_ptr"]), np.asarray(d["net_pin"])
    out = []
    for n in nets:
        q = pins[ptr[n]:ptr[n + 1]]
        X = [oracle.nm(float(v)) for v in pos[q, 0]]
        Y = [oracle.nm(float(v)) for v in pos[q, 1]]
        out.append(oracle.steiner_tree(X, Y))
    return out


@pytest.mark.parametrize("ry", [None, 0.3])
def test_steiner_adjoint_matches_central_differences(ry):
    """dJ/d(x, y) of the oracle's adjoint on Steiner-tree RC against central
    differences of its own smoothed objective.  Positions sit at (integer +
    1/4) nm so that a step of h = 20 nm moves every nm coordinate by exactly
    20; a cell is checked only where the trees of all its nets keep their
    topology at both steps (parents and pin nodes equal, every node
    coordinate moving linearly), which is where the tree-held-fixed gradient
    is the derivative.  With ry, unit R and C along y differ from x."""
    d = synth.make_design(400, 12, seed=23, placed=True, placement="local", gamma_ns=0.01, period_ns=0.6)
    d["wire_model"] = 1
    d["r_per_um"] = 0.5
    if ry is not None:
        d["r_per_um_y"], d["c_per_um_y"] = ry, 0.35
    for key in ("cell_xy", "port_xy"):
        v = np.asarray(d[key], np.float64)
        d[key] = ((np.round(v * 1000.0) + 0.25) / 1000.0).astype(np.float32)
    d["gamma_ns"], d["period_ns"] = 0.0, 0.0
    req = -oracle.sta(d)["ep_setup"][:, 0]
    d["period_ns"], d["gamma_ns"] = float(np.quantile(req, 0.7)), 0.01
    J, _, g = oracle.objective_grad(d)
    _, cell_of = _pin_positions(d)
    ptr, pins = np.asarray(d["net_pin_ptr"]), np.asarray(d["net_pin"])
    net_of_pin = np.repeat(np.arange(int(d["n_nets"])), np.diff(ptr))
    pin_net = np.full(int(d["n_pins"]), -1)
    pin_net[pins] = net_of_pin
    rng = np.random.default_rng(1)
    cells = rng.choice(d["n_cells"], 60, replace=False)
    h = 0.020
    scale = np.abs(g).max()
    checked = bad = 0
    for c in cells:
        nets = sorted(set(pin_net[np.nonzero(cell_of == c)[0]]) - {-1})
        base = _net_trees(d, nets)
        for ax in (0, 1):
            dd = {}
            for sgn in (1, -1):
                dd[sgn] = dict(d)
                xy = np.asarray(d["cell_xy"], np.float64).copy()
                xy[2 * c + ax] += sgn * h
                dd[sgn]["cell_xy"] = xy.astype(np.float32)
            tp, tm = _net_trees(dd[1], nets), _net_trees(dd[-1], nets)
            same = all(len(a["parent"]) == len(b["parent"]) == len(o["parent"]) and
                       np.array_equal(a["parent"], o["parent"]) and np.array_equal(b["parent"], o["parent"]) and
                       np.array_equal(a["pin_node"], o["pin_node"]) and np.array_equal(b["pin_node"], o["pin_node"]) and
                       np.array_equal(a["nx"] + b["nx"], 2 * o["nx"]) and np.array_equal(a["ny"] + b["ny"], 2 * o["ny"])
                       for a, b, o in zip(tp, tm, base))
            if not same:
                continue
            checked += 1
            fd = (oracle.objective(dd[1]) - oracle.objective(dd[-1])) / (2 * h)
            if abs(fd - g[c, ax]) > 1e-5 * abs(g[c, ax]) + 1e-6 * scale:
                bad += 1
    assert checked >= 60, checked
    # a cell may straddle a table breakpoint inside +-h: allow one
    assert bad <= 1, (bad, checked)
    assert scale > 0


# --------------------------------------- N4 top-k paths, per-endpoint limit

@pytest.mark.parametrize("seed", range(4))
def test_nworst_paths_match_brute_force_fixed_delay(seed):
    """With slew-independent delays the report with a per-endpoint limit L is
    fixed by exhaustive enumeration: per endpoint, every path's slack
    (required time of its end edge - its arrival), the L smallest of each of
    the k worst endpoints, merged by (slack, endpoint order, rank), the first
    k.  Every reported path is made of timing arcs, distinct from the others,
    its arrivals are its own prefix sums and its slack is required - arrival."""
    d = _fixed_design(seed, n_cells=14, depth=5)
    d["period_ns"] = 0.3
    res = oracle.sta(d)
    allp = _indep.enumerate_paths(d)
    net = _indep.Net(d)
    eps, es = res["endpoints"], res["ep_setup"][:, 0]
    for k, L in ((50, 3), (12, 8), (40, 1), (5, 30)):
        paths = oracle.report_paths_nworst(d, k, L, res=res)
        order = sorted(range(len(eps)), key=lambda e: (es[e], e))[:k]
        want = []
        for oi, e in enumerate(order):
            p = int(eps[e])
            sl = sorted(res["rat"][p, 0, 2 + rf] - a for a, _, rf in allp[p])
            want += [(s, oi, r, p) for r, s in enumerate(sl[:L])]
        want.sort()
        want = want[:k]
        assert len(paths) == len(want)
        for pth, (s, _, _, p) in zip(paths, want):
            assert pth["slack"] == pytest.approx(s, abs=1e-12)
            assert pth["endpoint"] == p
        seen = set()
        for pth in paths:
            pins, rfs, at = pth["pins"], pth["rf"], pth["at"]
            key = (tuple(pins.tolist()), tuple(rfs.tolist()))
            assert key not in seen
            seen.add(key)
            assert pins[-1] == pth["endpoint"]
            assert np.asarray(d["pin_role"])[pins[0]] in (synth.PI, synth.CK)
            for (u, ru), (v, rv) in zip(zip(pins[:-1], rfs[:-1]), zip(pins[1:], rfs[1:])):
                assert _arc_ok(d, net, int(u), int(ru), int(v), int(rv)), (u, v)
            for i in range(1, len(pins)):
                v, u = int(pins[i]), int(pins[i - 1])
                if net.driver.get(v) == u:
                    assert at[i] == pytest.approx(at[i - 1] + net.Dns[v], abs=1e-12)
                else:
                    assert at[i] >= at[i - 1]
            assert any(abs(a - at[-1]) < 1e-12 and rf == rfs[-1] for a, _, rf in allp[int(pins[-1])])
            e = int(pins[-1])
            assert pth["slack"] == pytest.approx(res["rat"][e, 0, 2 + rfs[-1]] - at[-1], abs=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_nworst_paths_match_brute_force_slew_dependent(seed):
    """Reading 15 on slew-dependent tables: a path's arrival adds each cell
    arc's delay at the analysis' own input slew (late, the path's edge at
    the arc's input) and the output load, so path delays are additive and
    plain enumeration fixes the report: every path to each endpoint, summed
    with the independent net sums and bilinear form, ranked per endpoint,
    the L smallest of each of the k worst endpoints merged by (slack,
    endpoint order, rank).  The best-first search of the oracle must give
    the same slacks and endpoints rank by rank."""
    d = synth.make_design(14, 5, seed=seed, rc_nodes=(2, 5), pi_frac=0.3)
    d["period_ns"] = 0.3
    res = oracle.sta(d)
    allp = _indep.enumerate_paths_at_slews(d, res["slew"][:, 0])
    eps, es = res["endpoints"], res["ep_setup"][:, 0]
    # the graph-based arrival is the latest enumerated path at every endpoint edge
    for e in range(len(eps)):
        p = int(eps[e])
        for rf in (0, 1):
            vals = [a for a, r in allp[p] if r == rf]
            if vals:
                assert res["at"][p, 0, 2 + rf] == pytest.approx(max(vals), abs=1e-12)
    for k, L in ((50, 3), (12, 8), (40, 1), (5, 30)):
        paths = oracle.report_paths_nworst(d, k, L, res=res)
        order = sorted(range(len(eps)), key=lambda e: (es[e], e))[:k]
        want = []
        for oi, e in enumerate(order):
            p = int(eps[e])
            sl = sorted(res["rat"][p, 0, 2 + rf] - a for a, rf in allp[p])
            want += [(s, oi, r, p) for r, s in enumerate(sl[:L])]
        want.sort()
        want = want[:k]
        assert len(paths) == len(want)
        for pth, (s, _, _, p) in zip(paths, want):
            assert pth["slack"] == pytest.approx(s, abs=1e-12)
            assert pth["endpoint"] == p


def test_nworst_limit_one_is_the_plain_report():
    d = synth.make_design(800, 12, seed=3, period_ns=0.9)
    res = oracle.sta(d)
    for k, thr in ((10, np.inf), (60, 0.0)):
        a = oracle.report_paths(d, k, slack_lt=thr, res=res)
        b = oracle.report_paths_nworst(d, k, 1, slack_lt=thr, res=res)
        assert [p["endpoint"] for p in a] == [p["endpoint"] for p in b]
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x["pins"], y["pins"])
            np.testing.assert_allclose(x["at"], y["at"], atol=1e-12)
            assert x["slack"] == pytest.approx(y["slack"], abs=1e-12)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_timed_baseline_is_the_same_analysis(threads):
    """The timed CPU baseline (net delays through WNS/TNS over level buckets,
    OpenMP over a level's pins) reports exactly what the serial analysis
    reports, for any thread count, on one and several corners."""
    ls, rs = synth.lut_corners()
    for d in (synth.workload("tiny", seed=1),
              synth.make_design(3000, 20, seed=4, n_corners=4, lut_scale=ls, rc_scale=rs, period_ns=1.7),
              synth.make_design(2000, 15, seed=5, placed=True)):
        r = oracle.sta(d)
        secs, summ = oracle.sta_timed(d, threads, 2)
        assert len(secs) == 2 and np.all(secs > 0)
        keys = ("wns_setup", "tns_setup", "wns_hold", "tns_hold", "worst_setup", "worst_hold")
        for k in range(int(d.get("n_corners", 1))):
            want = [r[x][k] for x in keys] + [r["n_viol_setup"][k], r["n_viol_hold"][k]]
            np.testing.assert_array_equal(summ[k], np.array(want, np.float64))
