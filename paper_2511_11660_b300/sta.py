"""Thin ctypes binding of ``libsta.so`` (names follow ``include/sta.h``).

Argument marshalling only: every step of the timing pass runs in the CUDA
kernels of the library.  There is no CPU fallback; if ``libsta.so`` is missing
or no CUDA device is present the calls raise.

PyTorch serves as the device allocator and stream source: device outputs are
``torch`` tensors whose ``data_ptr()`` is handed to the library, and the
stream defaults to ``torch.cuda.current_stream()``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

OK, EINVAL, ECYCLE, ENOMEM, ECUDA, ETIMEOUT, ESTATE = range(7)
HOST, DEVICE = 0, 1
AT, SLEW, RAT, SLACK = 0, 1, 2, 3
SCHED_LEVEL, SCHED_DATAFLOW, SCHED_COOP, SCHED_TILE = 0, 1, 2, 3
NET_ELMORE, NET_ARNOLDI = 0, 1
WIRE_STAR, WIRE_STEINER = 0, 1


class StaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d): %s" % (_status_name(status), status, msg))
        self.status = status


class sta_library(C.Structure):
    _fields_ = [("n_types", C.c_int32), ("type_nin", C.c_void_p), ("type_kind", C.c_void_p),
                ("arc_sense", C.c_void_p), ("lut_idx1", C.c_void_p), ("lut_idx2", C.c_void_p),
                ("lut_val", C.c_void_p), ("pin_cap", C.c_void_p), ("setup_ns", C.c_float),
                ("hold_ns", C.c_float), ("po_cap_pf", C.c_float)]


class sta_design_desc(C.Structure):
    _fields_ = [("lib", C.POINTER(sta_library)), ("n_cells", C.c_int32), ("cell_type", C.c_void_p),
                ("cell_pin_ptr", C.c_void_p), ("cell_pin", C.c_void_p), ("n_pins", C.c_int32),
                ("pin_role", C.c_void_p), ("n_nets", C.c_int32), ("net_pin_ptr", C.c_void_p),
                ("net_pin", C.c_void_p), ("rc_ptr", C.c_void_p), ("rc_parent", C.c_void_p),
                ("rc_pin_node", C.c_void_p), ("rc_R", C.c_void_p), ("rc_C", C.c_void_p),
                ("cell_xy", C.c_void_p), ("port_xy", C.c_void_p), ("r_per_um", C.c_float),
                ("c_per_um", C.c_float), ("period_ns", C.c_float), ("clk_slew_ns", C.c_float),
                ("pi_at_ns", C.c_float), ("pi_slew_ns", C.c_float), ("n_corners", C.c_int32),
                ("lut_scale", C.c_void_p), ("rc_scale", C.c_void_p), ("gamma_ns", C.c_float),
                ("net_model", C.c_int32), ("arnoldi_order", C.c_int32), ("n_exc", C.c_int32),
                ("exc_from_ptr", C.c_void_p), ("exc_from", C.c_void_p), ("exc_to_ptr", C.c_void_p),
                ("exc_to", C.c_void_p), ("exc_action", C.c_void_p), ("exc_mult", C.c_void_p),
                ("exc_thru_ptr", C.c_void_p), ("exc_thru_set_ptr", C.c_void_p), ("exc_thru_pin", C.c_void_p),
                ("wire_model", C.c_int32), ("r_per_um_y", C.c_float), ("c_per_um_y", C.c_float)]


class sta_plan_info(C.Structure):
    _fields_ = [("n_pins", C.c_int64), ("n_cells", C.c_int64), ("n_nets", C.c_int64), ("n_items", C.c_int64),
                ("n_cell_arcs", C.c_int64), ("n_net_arcs", C.c_int64), ("n_rc_nodes", C.c_int64),
                ("n_endpoints", C.c_int64), ("n_levels", C.c_int32), ("n_corners", C.c_int32),
                ("max_level_width", C.c_int32), ("n_designs", C.c_int32), ("device_bytes", C.c_int64),
                ("launches_per_update", C.c_int32), ("launches_per_backward", C.c_int32), ("n_tags", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sta_tile_info(C.Structure):
    _fields_ = [("n_tiles", C.c_int32), ("n_steps", C.c_int32), ("wave_items", C.c_int32),
                ("ring_slots", C.c_int32), ("max_step_entries", C.c_int32), ("pad", C.c_int32),
                ("fwd_edges", C.c_int64), ("fwd_local", C.c_int64), ("bwd_edges", C.c_int64),
                ("bwd_local", C.c_int64), ("crit_edges", C.c_int64), ("crit_local", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class sta_corner_report(C.Structure):
    _fields_ = [("wns_setup", C.c_double), ("tns_setup", C.c_double), ("wns_hold", C.c_double),
                ("tns_hold", C.c_double), ("worst_setup", C.c_double), ("worst_hold", C.c_double),
                ("n_viol_setup", C.c_int64), ("n_viol_hold", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sta_views(C.Structure):
    _fields_ = [("at", C.c_void_p), ("slew", C.c_void_p), ("rat", C.c_void_p), ("slack", C.c_void_p),
                ("gpu_pin_of", C.c_void_p)]


# every entry point of include/sta.h: name -> (restype, argtypes)
_V, _P = C.c_void_p, C.c_void_p
SIGNATURES = {
    "sta_plan": (C.c_int, [_P, C.POINTER(sta_plan_info)]),
    "sta_plan_error": (C.c_char_p, []),
    "sta_plan_levels": (C.c_int, [_P, _P]),
    "sta_plan_tiles": (C.c_int, [_P, C.c_int32, C.POINTER(sta_tile_info)]),
    "sta_get_tile_info": (C.c_int, [_V, C.POINTER(sta_tile_info)]),
    "sta_create": (C.c_int, [_P, C.c_int, C.POINTER(C.c_void_p)]),
    "sta_create_batch": (C.c_int, [_P, C.c_int32, C.c_int, C.POINTER(C.c_void_p)]),
    "sta_set_rc": (C.c_int, [_V, _P, _P, C.c_int]),
    "sta_set_positions": (C.c_int, [_V, _P, C.c_int, _V]),
    "sta_set_cell_types": (C.c_int, [_V, _P]),
    "sta_set_clock": (C.c_int, [_V, C.c_float]),
    "sta_resize_cells": (C.c_int, [_V, _P, _P, C.c_int32, C.c_int, _V]),
    "sta_set_corners": (C.c_int, [_V, _P, _P]),
    "sta_set_schedule": (C.c_int, [_V, C.c_int32, C.c_int32]),
    "sta_autotune": (C.c_int, [_V, _V, C.c_int32, C.c_int32, _P, _P, _P]),
    "sta_set_wait_limit": (C.c_int, [_V, C.c_int64]),
    "sta_set_adjoint_schedule": (C.c_int, [_V, C.c_int32]),
    "sta_debug_hold_cell": (C.c_int, [_V, C.c_int32]),
    "sta_update_timing": (C.c_int, [_V, _V]),
    "sta_sync": (C.c_int, [_V, _V]),
    "sta_report_slack": (C.c_int, [_V, _V, _P]),
    "sta_report_slack_design": (C.c_int, [_V, C.c_int32, _V, _P]),
    "sta_get_pin_state": (C.c_int, [_V, C.c_int32, _P, C.c_int, _V]),
    "sta_get_endpoint_slack": (C.c_int, [_V, _P, _P, _P, _P, C.c_int, _V]),
    "sta_get_net_wirelength": (C.c_int, [_V, _P, C.c_int, _V]),
    "sta_set_rc_async": (C.c_int, [_V, _P, _P, C.c_int, _V]),
    "sta_report_paths": (C.c_int, [_V, C.c_int32, C.c_int32, C.c_int32, C.c_float, _P, _P, _P, _P, _P, _P, _P, _P,
                                   C.c_int32, C.c_int, _V]),
    "sta_report_paths_nworst": (C.c_int, [_V, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_float, _P, _P, _P, _P,
                                          _P, _P, _P, _P, C.c_int32, C.c_int, _V]),
    "sta_backward": (C.c_int, [_V, C.c_double, C.c_double, _P, _P, _P, C.c_int, _V]),
    "sta_get_arrays": (C.c_int, [_V, C.POINTER(sta_views)]),
    "sta_stats": (C.c_int, [_V, C.POINTER(sta_plan_info)]),
    "sta_set_profiling": (C.c_int, [_V, C.c_int32]),
    "sta_last_timings": (C.c_int, [_V, _P]),
    "sta_last_error": (C.c_char_p, [_V]),
    "sta_status_string": (C.c_char_p, [C.c_int]),
    "sta_destroy": (None, [_V]),
    "sta_reduce_slack_noalloc": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, _V]),
}

_lib = None


def load(path: str | None = None):
    """Load ``libsta.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = path or LIB
        if not os.path.exists(path):
            raise ImportError("libsta.so not built: run `python -m paper_2511_11660_b300.build`")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _status_name(s: int) -> str:
    try:
        return load().sta_status_string(s).decode()
    except Exception:
        return str(s)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _mem_of(t) -> int:
    return DEVICE if hasattr(t, "is_cuda") and t.is_cuda else HOST


class Design:
    """ctypes view of a design dict (see ``synth``); keeps its arrays alive."""

    _ARR = {"type_nin": np.int32, "type_kind": np.int32, "arc_sense": np.int32, "lut_idx1": np.float32,
            "lut_idx2": np.float32, "lut_val": np.float32, "pin_cap": np.float32, "cell_type": np.int32,
            "cell_pin_ptr": np.int32, "cell_pin": np.int32, "pin_role": np.int8, "net_pin_ptr": np.int32,
            "net_pin": np.int32, "rc_ptr": np.int32, "rc_parent": np.int32, "rc_pin_node": np.int32,
            "rc_R": np.float32, "rc_C": np.float32, "cell_xy": np.float32, "port_xy": np.float32,
            "lut_scale": np.float32, "rc_scale": np.float32, "exc_from_ptr": np.int32, "exc_from": np.int32,
            "exc_to_ptr": np.int32, "exc_to": np.int32, "exc_action": np.int32, "exc_mult": np.float32,
            "exc_thru_ptr": np.int32, "exc_thru_set_ptr": np.int32, "exc_thru_pin": np.int32}

    def __init__(self, d: dict):
        self.src = d
        self.keep = {}
        for k, dt in self._ARR.items():
            v = d.get(k)
            self.keep[k] = None if v is None else np.ascontiguousarray(np.asarray(v), dtype=dt)
        a = self.keep
        self.lib = sta_library(int(d["n_types"]), _ptr(a["type_nin"]), _ptr(a["type_kind"]), _ptr(a["arc_sense"]),
                               _ptr(a["lut_idx1"]), _ptr(a["lut_idx2"]), _ptr(a["lut_val"]), _ptr(a["pin_cap"]),
                               float(d["setup_ns"]), float(d["hold_ns"]), float(d["po_cap_pf"]))
        placed = d.get("rc_ptr") is None
        self.desc = sta_design_desc(
            C.pointer(self.lib), int(d["n_cells"]), _ptr(a["cell_type"]), _ptr(a["cell_pin_ptr"]),
            _ptr(a["cell_pin"]), int(d["n_pins"]), _ptr(a["pin_role"]), int(d["n_nets"]), _ptr(a["net_pin_ptr"]),
            _ptr(a["net_pin"]), None if placed else _ptr(a["rc_ptr"]), None if placed else _ptr(a["rc_parent"]),
            None if placed else _ptr(a["rc_pin_node"]), None if placed else _ptr(a["rc_R"]),
            None if placed else _ptr(a["rc_C"]), _ptr(a["cell_xy"]), _ptr(a["port_xy"]),
            float(d.get("r_per_um", 0.0)), float(d.get("c_per_um", 0.0)), float(d["period_ns"]),
            float(d["clk_slew_ns"]), float(d["pi_at_ns"]), float(d["pi_slew_ns"]), int(d.get("n_corners", 1)),
            _ptr(a["lut_scale"]), _ptr(a["rc_scale"]), float(d.get("gamma_ns", 0.0)),
            int(d.get("net_model", 0)), int(d.get("arnoldi_order", 0)),
            0 if a["exc_action"] is None else len(a["exc_action"]), _ptr(a["exc_from_ptr"]), _ptr(a["exc_from"]),
            _ptr(a["exc_to_ptr"]), _ptr(a["exc_to"]), _ptr(a["exc_action"]), _ptr(a["exc_mult"]),
            _ptr(a["exc_thru_ptr"]), _ptr(a["exc_thru_set_ptr"]), _ptr(a["exc_thru_pin"]),
            int(d.get("wire_model", 0)), float(d.get("r_per_um_y", 0.0)), float(d.get("c_per_um_y", 0.0)))

    @property
    def n_pins(self):
        return int(self.src["n_pins"])

    @property
    def n_corners(self):
        return int(self.src.get("n_corners", 1))


def sta_plan(design) -> dict:
    """Host-only validation and levelisation (no GPU)."""
    lib = load()
    dd = design if isinstance(design, Design) else Design(design)
    info = sta_plan_info()
    st = lib.sta_plan(C.byref(dd.desc), C.byref(info))
    if st != OK:
        raise StaError(st, lib.sta_plan_error().decode())
    return info.as_dict()


def sta_plan_tiles(design, n_tiles: int) -> dict:
    """Host-only: the tile schedule's partition into ``n_tiles`` tiles,
    checked by replaying the kernels' ring use; its statistics."""
    lib = load()
    dd = design if isinstance(design, Design) else Design(design)
    info = sta_tile_info()
    st = lib.sta_plan_tiles(C.byref(dd.desc), int(n_tiles), C.byref(info))
    if st != OK:
        raise StaError(st, lib.sta_plan_error().decode())
    return info.as_dict()


def sta_plan_levels(design) -> np.ndarray:
    """Host-only: propagation level of every cell."""
    lib = load()
    dd = design if isinstance(design, Design) else Design(design)
    out = np.zeros(max(int(dd.src["n_cells"]), 1), np.int32)
    st = lib.sta_plan_levels(C.byref(dd.desc), _ptr(out))
    if st != OK:
        raise StaError(st, lib.sta_plan_error().decode())
    return out[: int(dd.src["n_cells"])]


class Context:
    """One timing context (``sta_create`` / ``sta_create_batch``)."""

    def __init__(self, design, device: int = 0, batch=None):
        self.lib = load()
        self.h = C.c_void_p()
        if batch is not None:
            self.designs = [d if isinstance(d, Design) else Design(d) for d in batch]
            arr = (C.c_void_p * len(self.designs))(*[C.addressof(d.desc) for d in self.designs])
            self._arr = arr
            st = self.lib.sta_create_batch(arr, len(self.designs), device, C.byref(self.h))
        else:
            self.designs = [design if isinstance(design, Design) else Design(design)]
            st = self.lib.sta_create(C.byref(self.designs[0].desc), device, C.byref(self.h))
        if st != OK:
            raise StaError(st, self.lib.sta_plan_error().decode())
        info = self.stats()
        self.P, self.K, self.E, self.C = info["n_pins"], info["n_corners"], info["n_endpoints"], info["n_cells"]
        self.T = info["n_tags"]
        self.device = device

    def _chk(self, st):
        if st != OK:
            raise StaError(st, self.lib.sta_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.lib.sta_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        info = sta_plan_info()
        self._chk(self.lib.sta_stats(self.h, C.byref(info)))
        return info.as_dict()

    def tile_info(self) -> dict:
        """Statistics of the current tile partition (zeros unless SCHED_TILE)."""
        info = sta_tile_info()
        self._chk(self.lib.sta_get_tile_info(self.h, C.byref(info)))
        return info.as_dict()

    def set_schedule(self, schedule: int, param: int = 0):
        self._chk(self.lib.sta_set_schedule(self.h, schedule, param))

    def autotune(self, trials: int = 5, force: bool = False, stream=None):
        """Time the candidate schedules, select the fastest; returns
        (schedule, param, ms per update)."""
        sch, par, ms = C.c_int32(), C.c_int32(), C.c_float()
        self._chk(self.lib.sta_autotune(self.h, _stream(stream), int(trials), int(force), C.byref(sch),
                                        C.byref(par), C.byref(ms)))
        return sch.value, par.value, ms.value

    def set_wait_limit(self, polls: int):
        self._chk(self.lib.sta_set_wait_limit(self.h, int(polls)))

    def set_adjoint_schedule(self, schedule: int):
        """Reverse sweep of backward(): SCHED_DATAFLOW (default) or SCHED_LEVEL."""
        self._chk(self.lib.sta_set_adjoint_schedule(self.h, schedule))

    def debug_hold_cell(self, cell: int):
        self._chk(self.lib.sta_debug_hold_cell(self.h, int(cell)))

    def set_corners(self, lut_scale, rc_scale):
        a = np.ascontiguousarray(lut_scale, np.float32)
        b = np.ascontiguousarray(rc_scale, np.float32)
        assert len(a) == self.K and len(b) == self.K
        self._chk(self.lib.sta_set_corners(self.h, _ptr(a), _ptr(b)))

    def set_clock(self, period_ns: float):
        self._chk(self.lib.sta_set_clock(self.h, float(period_ns)))

    def set_profiling(self, on: bool):
        self._chk(self.lib.sta_set_profiling(self.h, int(on)))

    def last_timings(self):
        ms = (C.c_float * 4)()
        self._chk(self.lib.sta_last_timings(self.h, ms))
        return list(ms)

    def set_rc(self, R, Cc):
        self._chk(self.lib.sta_set_rc(self.h, _ptr(R), _ptr(Cc), _mem_of(R)))

    def set_rc_async(self, R, Cc, stream=None):
        """Stage R/C for the next update_timing; the copy runs on ``stream``
        (page-locked host tensors or device tensors) and may overlap an
        update in flight.  The caller keeps R and Cc unchanged until then."""
        self._chk(self.lib.sta_set_rc_async(self.h, _ptr(R), _ptr(Cc), _mem_of(R), _stream(stream)))

    def set_positions(self, cell_xy, stream=None):
        mem = _mem_of(cell_xy)
        if mem == HOST:
            cell_xy = np.ascontiguousarray(cell_xy, np.float32)
        self._chk(self.lib.sta_set_positions(self.h, _ptr(cell_xy), mem, _stream(stream) if mem == DEVICE else None))

    def set_cell_types(self, cell_type):
        a = np.ascontiguousarray(cell_type, np.int32)
        self._chk(self.lib.sta_set_cell_types(self.h, _ptr(a)))

    def resize_cells(self, cells, types, stream=None):
        """Give cells[i] the type types[i] (int32; torch CUDA tensors stay on
        the device, numpy arrays are copied)."""
        mem = _mem_of(cells)
        if mem == HOST:
            cells = np.ascontiguousarray(cells, np.int32)
            types = np.ascontiguousarray(types, np.int32)
        self._chk(self.lib.sta_resize_cells(self.h, _ptr(cells), _ptr(types), int(len(cells)), mem,
                                            _stream(stream)))

    def update_timing(self, stream=None):
        self._chk(self.lib.sta_update_timing(self.h, _stream(stream)))

    def sync(self, stream=None):
        self._chk(self.lib.sta_sync(self.h, _stream(stream)))

    def report_slack(self, design: int = 0, stream=None):
        reps = (sta_corner_report * self.K)()
        self._chk(self.lib.sta_report_slack_design(self.h, design, _stream(stream), reps))
        return [r.as_dict() for r in reps]

    def get_pin_state(self, which: int, out=None, stream=None):
        """[n_pins, n_corners * n_tags, 4] float32 in caller pin order (state
        = corner * n_tags + exception tag); a torch CUDA tensor ``out``
        receives it on the device, else a numpy array."""
        if out is None:
            out = np.empty((self.P, self.K * self.T, 4), np.float32)
        self._chk(self.lib.sta_get_pin_state(self.h, which, _ptr(out), _mem_of(out), _stream(stream)))
        return out

    def report_paths(self, k: int, slack_lt: float = float("inf"), corner: int = 0, design: int = 0, stream=None,
                     per_endpoint: int = 1):
        """Top-k path report (host arrays): a list of dicts with the endpoint
        pin, the path's setup slack and the path's pins, edges and late
        arrivals from the startpoint to the endpoint.  per_endpoint > 1:
        sta_report_paths_nworst (up to that many paths per endpoint)."""
        n_paths, n_pins = C.c_int32(0), C.c_int32(0)
        cap = max(1, k) * (2 * self.stats()["n_levels"] + 3)
        ptr = np.zeros(max(1, k) + 1, np.int32)
        pin = np.zeros(cap, np.int32)
        rf = np.zeros(cap, np.int8)
        at = np.zeros(cap, np.float32)
        slack = np.zeros(max(1, k), np.float32)
        ep = np.zeros(max(1, k), np.int32)
        if per_endpoint == 1:
            self._chk(self.lib.sta_report_paths(self.h, design, corner, k, float(slack_lt), C.byref(n_paths),
                                                C.byref(n_pins), _ptr(ptr), _ptr(pin), _ptr(rf), _ptr(at),
                                                _ptr(slack), _ptr(ep), cap, HOST, _stream(stream)))
        else:
            self._chk(self.lib.sta_report_paths_nworst(self.h, design, corner, k, int(per_endpoint), float(slack_lt),
                                                       C.byref(n_paths), C.byref(n_pins), _ptr(ptr), _ptr(pin),
                                                       _ptr(rf), _ptr(at), _ptr(slack), _ptr(ep), cap, HOST,
                                                       _stream(stream)))
        out = []
        for i in range(n_paths.value):
            b, e = ptr[i], ptr[i + 1]
            out.append({"endpoint": int(ep[i]), "slack": float(slack[i]), "pins": pin[b:e].copy(),
                        "rf": rf[b:e].copy(), "at": at[b:e].copy()})
        return out

    def get_net_wirelength(self, device: bool = False, stream=None):
        """Steiner wirelength (int64 nm) of every net at the last update, in
        caller net order; a torch CUDA tensor with ``device``, else numpy."""
        n = self.stats()["n_nets"]   # every caller net: the count the library writes
        if device:
            import torch
            out = torch.empty(n, dtype=torch.int64, device=torch.device("cuda", self.device))
        else:
            out = np.empty(n, np.int64)
        self._chk(self.lib.sta_get_net_wirelength(self.h, _ptr(out), DEVICE if device else HOST, _stream(stream)))
        return out

    def get_endpoint_slack(self, device: bool = False, stream=None, out=None):
        """Endpoint setup and hold slacks [E, corners] and violation flags.
        ``out``: four preallocated arrays (setup, hold, setup flags, hold
        flags) to fill instead -- page-locked host memory makes the copies
        direct DMA."""
        if out is not None:
            s, h, vs, vh = out
            self._chk(self.lib.sta_get_endpoint_slack(self.h, _ptr(s), _ptr(h), _ptr(vs), _ptr(vh), _mem_of(s),
                                                      _stream(stream)))
            return s, h, vs, vh
        if device:
            import torch
            dev = torch.device("cuda", self.device)
            s = torch.empty((self.E, self.K), dtype=torch.float32, device=dev)
            h = torch.empty_like(s)
            vs = torch.empty((self.E, self.K), dtype=torch.uint8, device=dev)
            vh = torch.empty_like(vs)
        else:
            s = np.empty((self.E, self.K), np.float32)
            h = np.empty_like(s)
            vs = np.empty((self.E, self.K), np.uint8)
            vh = np.empty_like(vs)
        self._chk(self.lib.sta_get_endpoint_slack(self.h, _ptr(s), _ptr(h), _ptr(vs), _ptr(vh),
                                                  DEVICE if device else HOST, _stream(stream)))
        return s, h, vs, vh

    def backward(self, w_tns: float = 1.0, w_wns: float = 1.0, grad_out=None, stream=None):
        """Smoothed objective J and dJ/d(cell x, y) (float64).  With a torch
        CUDA ``grad_out`` of shape [n_cells, 2] everything stays on the
        device; returns (J, per-corner (TNS_g, WNS_g), grad)."""
        if grad_out is not None and _mem_of(grad_out) == DEVICE:
            import torch
            J = torch.empty(1 + 2 * self.K, dtype=torch.float64, device=grad_out.device)
            self._chk(self.lib.sta_backward(self.h, w_tns, w_wns, _ptr(J), J.data_ptr() + 8, _ptr(grad_out),
                                            DEVICE, _stream(stream)))
            return J[0], J[1:].view(self.K, 2), grad_out
        J = np.zeros(1, np.float64)
        terms = np.zeros((self.K, 2), np.float64)
        g = np.zeros((self.C, 2), np.float64) if grad_out is None else grad_out
        self._chk(self.lib.sta_backward(self.h, w_tns, w_wns, _ptr(J), _ptr(terms), _ptr(g), HOST,
                                        _stream(stream)))
        return float(J[0]), terms, g

    def views(self) -> dict:
        """Device pointers in the library's pin order: at and rat point to
        [n_pins][states][4][2] float32 double-float pairs (value hi + lo),
        slew and slack to [n_pins][states][4] float32."""
        v = sta_views()
        self._chk(self.lib.sta_get_arrays(self.h, C.byref(v)))
        return {k: getattr(v, k) for k, _ in v._fields_}


def reduce_slack_noalloc(setup, hold, out, stream=None):
    """WNS/TNS of device endpoint slacks ``setup``/``hold`` ([E, K] float32
    CUDA tensors) into ``out`` ([K, 8] float64 CUDA tensor) without any device
    allocation (``sta_reduce_slack_noalloc``)."""
    import torch
    lib = load()
    for name, t, dt in (("setup", setup, torch.float32), ("hold", hold, torch.float32), ("out", out, torch.float64)):
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if setup.dim() != 2 or setup.shape != hold.shape:
        raise ValueError("setup and hold must both be [n_endpoints, n_corners]")
    if setup.device != hold.device or setup.device != out.device:
        raise ValueError("setup, hold and out must sit on one CUDA device")
    E, K = int(setup.shape[0]), int(setup.shape[1])
    if K < 1 or out.numel() < 8 * K:
        raise ValueError("out must hold n_corners x 8 float64 values")
    # the C entry point runs on the current device: make it the tensors' one
    with torch.cuda.device(setup.device):
        s = _stream(stream) if stream is not None else torch.cuda.current_stream(setup.device).cuda_stream
        st = lib.sta_reduce_slack_noalloc(_ptr(setup), _ptr(hold), E, K, _ptr(out), s)
    if st != OK:
        raise StaError(st, "sta_reduce_slack_noalloc failed")
    return out
