/*
 * sta.h -- C ABI of libsta.so, a B300 (sm_103a) graph-based static timing
 * analysis library.
 *
 * What it computes follows HeteroSTA (arXiv 2511.11660):
 *   - inputs are a flattened CSR netlist handed over by a host flow instead
 *     of parsed files (Sec. III, "Heterogeneous netlist database"), a cell
 *     library of NLDM tables (Sec. IV-A), parasitics either as flattened RC
 *     trees or as pin positions plus unit R/C (Sec. III, "Parasitics (RC)
 *     inputs") and one ideal clock;
 *   - delay calculation uses the Elmore calculator (Sec. III, "Delay
 *     models"), extended with the second moment for the output slew;
 *   - outputs are pin slacks and WNS/TNS (Sec. III, "Report options"),
 *     left on the GPU or copied to the host at the caller's choice.
 * The paper gives no formulas; the library implements the textbook readings
 * (NLDM bilinear interpolation with edge extrapolation; Elmore delay and
 * slew = sqrt(s^2 + 2*m2 - D^2); max/min propagation of arrival times over
 * rise/fall x early/late; required times propagated backwards; setup slack
 * = RAT - AT, hold slack = AT - RAT; WNS = min(0, worst endpoint slack),
 * TNS = sum of negative endpoint slacks).
 *
 * Conventions shared by every entry point:
 *   - Every call returns sta_status; no C++ exception crosses the ABI.
 *   - Pointers in sta_design_desc are HOST pointers, read during the call
 *     only and copied; the caller keeps ownership.
 *   - Arguments typed with sta_mem say where a caller buffer lives
 *     (STA_HOST or STA_DEVICE, device = the context's device).
 *   - Streams are cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that take a stream are asynchronous unless they return host data.
 *   - Asynchronous device errors, and the device-side error word set by the
 *     kernels' own bounds / wait-limit checks, are reported by the next call
 *     that synchronises (sta_report_slack, sta_sync, sta_backward with host
 *     output).
 *   - Units: ns, pF for tables and loads; Ohm, fF for RC; um for positions.
 *   - Per-pin arrays use the layout [n_pins][n_corners][4] with the inner
 *     index el*2 + rf: el 0 = early (hold), 1 = late (setup); rf 0 = rise,
 *     1 = fall.  Endpoints are the DFF D pins and primary outputs in
 *     ascending pin id.
 */
#ifndef STA_H
#define STA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sta_ctx sta_ctx;   /* opaque, owned by the library */

typedef enum {
    STA_OK = 0,
    STA_EINVAL = 1,    /* malformed input (message in sta_last_error) */
    STA_ECYCLE = 2,    /* combinational loop in the timing graph */
    STA_ENOMEM = 3,    /* device or host allocation failed */
    STA_ECUDA = 4,     /* CUDA runtime error */
    STA_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    STA_ESTATE = 6     /* call out of order (e.g. report before update) */
} sta_status;

typedef enum { STA_HOST = 0, STA_DEVICE = 1 } sta_mem;

/* pin roles */
enum { STA_PIN_PI = 0, STA_PIN_PO = 1, STA_PIN_IN = 2, STA_PIN_OUT = 3,
       STA_PIN_D = 4, STA_PIN_CK = 5, STA_PIN_Q = 6 };
/* timing sense of the arc from an input slot to the cell output */
enum { STA_SENSE_NONE = -1, STA_SENSE_POS = 0, STA_SENSE_NEG = 1,
       STA_SENSE_NON = 2, STA_SENSE_RISE = 3 /* clock rising edge -> Q */ };
/* which per-pin array sta_get_pin_state copies */
enum { STA_AT = 0, STA_SLEW = 1, STA_RAT = 2, STA_SLACK = 3 };
/* propagation schedules (sta_set_schedule) */
enum { STA_SCHED_LEVEL = 0,      /* one kernel launch per level, graph-captured */
       STA_SCHED_DATAFLOW = 1,   /* one persistent kernel per pass, per-item ready flags */
       STA_SCHED_COOP = 2,       /* one co-resident launch for both passes, a grid barrier per level */
       STA_SCHED_TILE = 3 };     /* one co-resident launch per pass; each block walks its own tile of the
                                    graph level by level, block-local dependencies through shared memory */

/*
 * Cell library.  Per type: type_nin inputs (1..3) followed by one output.
 * A flip-flop (type_kind 1) has exactly two inputs, D (slot 0, sense NONE,
 * a setup/hold check pin) and CK (slot 1, sense RISE, arc CK -> Q).
 * Tables: per (type, slot) four 7x7 NLDM tables in the order delay rise,
 * delay fall, slew rise, slew fall; idx1 = input slew axis (ns), idx2 = load
 * axis (pF), both strictly increasing; val[i_slew * 7 + j_load].
 * Array shapes: type_nin/type_kind [n_types]; arc_sense [n_types*3];
 * lut_idx1/lut_idx2 [n_types*3*4*7]; lut_val [n_types*3*4*49];
 * pin_cap [n_types*4] (pF, by slot).
 */
typedef struct {
    int32_t n_types;
    const int32_t *type_nin;
    const int32_t *type_kind;
    const int32_t *arc_sense;
    const float *lut_idx1;
    const float *lut_idx2;
    const float *lut_val;
    const float *pin_cap;
    float setup_ns, hold_ns;   /* flip-flop setup / hold against the ideal clock */
    float po_cap_pf;           /* load of a primary output pin */
} sta_library;

/*
 * One design.  Cells: cell c owns pins cell_pin[cell_pin_ptr[c] ..
 * cell_pin_ptr[c+1]) in slot order (inputs, then the output), roles IN..OUT
 * or D, CK, Q.  Pins that belong to no cell are ports (PI or PO).  Nets:
 * net n lists net_pin[net_pin_ptr[n] .. net_pin_ptr[n+1]) with its driver
 * (PI, OUT or Q) first, then its sinks (IN, D or PO).  Every IN, D and PO pin
 * is the sink of exactly one net; CK pins are on no net (ideal clock).
 *
 * Parasitics, one of:
 *   RC trees: net n has nodes rc_ptr[n] .. rc_ptr[n+1) listed parent before
 *     child; rc_parent is the local parent index (-1 at node 0, the driver);
 *     rc_R (Ohm, node to parent; node 0 ignored), rc_C (fF, wire);
 *     rc_pin_node[k] is the local node of the pin net_pin[k] (0 for the
 *     driver).  Sink pin capacitances are added at their nodes.
 *   Positions (rc_ptr == NULL): a star tree per net from the driver to each
 *     sink, segment R = r_per_um * L, C = c_per_um * L split half to each
 *     end, L = Manhattan distance; pins sit at their cell's cell_xy[2c..],
 *     ports at port_xy[2p..] (port_xy may be NULL: ports at the origin).
 * Corners: n_corners >= 1; corner k multiplies every table value by
 * lut_scale[k] and every wire R and C by rc_scale[k] (NULL = all 1).
 * gamma_ns > 0 selects log-sum-exp smoothed max/min merges (differentiable
 * mode, required for sta_backward); 0 = exact max/min.
 * Net delay calculator (Sec. III "Delay models": an Elmore calculator and
 * an Arnoldi-based reduced-order model), the latter on RC trees (rc_ptr)
 * or Steiner trees (STA_WIRE_STEINER), not on stars, and with every edge
 * R > 0 (rc_R of non-root nodes; unit R for Steiner trees, whose points at
 * the same position share one node):
 *   STA_NET_ELMORE:  sink delay = Elmore delay (first moment of the impulse
 *     response);
 *   STA_NET_ARNOLDI: sink delay = the time the step response of an
 *     order-q reduced model reaches 50%.  The model projects the tree's
 *     nodal equations C v' + G v = b u (driver node held at u) onto an
 *     orthonormal basis of the Krylov space of G^-1 C started at the DC
 *     solution (congruence, so it stays passive); q = arnoldi_order (1..3,
 *     0 = 3), capped by the number of non-driver nodes.
 *   Both keep the slew law slew_sink = sqrt(slew_drv^2 + 2 beta - D^2) with
 *   the tree's second moment (an order >= 2 model matches it exactly).
 */
typedef struct {
    const sta_library *lib;
    int32_t n_cells;
    const int32_t *cell_type;
    const int32_t *cell_pin_ptr;
    const int32_t *cell_pin;
    int32_t n_pins;
    const int8_t *pin_role;
    int32_t n_nets;
    const int32_t *net_pin_ptr;
    const int32_t *net_pin;
    const int32_t *rc_ptr;
    const int32_t *rc_parent;
    const int32_t *rc_pin_node;
    const float *rc_R;
    const float *rc_C;
    const float *cell_xy;
    const float *port_xy;
    float r_per_um, c_per_um;
    float period_ns;      /* ideal clock period: setup capture edge */
    float clk_slew_ns;    /* slew at every CK pin (arrival 0, rising edge) */
    float pi_at_ns, pi_slew_ns;
    int32_t n_corners;
    const float *lut_scale;
    const float *rc_scale;
    float gamma_ns;
    int32_t net_model;      /* STA_NET_ELMORE (0) or STA_NET_ARNOLDI (1) */
    int32_t arnoldi_order;  /* q of STA_NET_ARNOLDI: 1..3, 0 = 3 */
    /* Timing exceptions (Sec. III: an SDC exceptions manager; Sec. IV-B
     * lists false and multicycle paths and min/max delays; this is the
     * reading of set_false_path / set_multicycle_path -setup /
     * set_max_delay / set_min_delay with -from startpoints and -to
     * endpoints).  Group g (0 <= g < n_exc <= 7):
     * startpoint pins exc_from[exc_from_ptr[g] .. exc_from_ptr[g+1]) (PI or
     * CK), endpoint pins exc_to[exc_to_ptr[g] .. exc_to_ptr[g+1]) (D or PO;
     * an empty list means every endpoint), exc_action[g] (0 false path, 1
     * multicycle, 2 max delay, 3 min delay) and exc_mult[g] (multicycle:
     * the setup multiplier M >= 1; max/min delay: the value V in ns).  Every
     * path carries the tag of its startpoint's first group (0 = none);
     * arrivals and required times are propagated per (corner, tag) state,
     * slews are tag-free; endpoint e checks tag g with g's action when it is
     * in g's list -- false path: no check; multicycle: setup capture edge at
     * M * T, hold unchanged; max delay: setup capture edge at V (a
     * flip-flop's setup time still applies), hold unchanged; min delay: hold
     * edge at V (plus a flip-flop's hold time), setup unchanged -- and the
     * default check otherwise.  Endpoint slacks,
     * WNS and TNS take the min over tags; per-pin arrays (sta_get_pin_state)
     * hold n_corners * (n_exc + 1) states, state = corner * (n_exc + 1) +
     * tag.  Not with gamma_ns > 0.  In a batch the groups of every design
     * count together (at most 7 groups and 32 tags over the batch; a group
     * acts only on its own design's paths).  n_exc = 0: none.
     * -through (Sec. IV-B: false paths through pin sequences): group g may
     * have ordered through sets exc_thru_ptr[g] .. exc_thru_ptr[g+1]; set s
     * lists gate input pins exc_thru_pin[exc_thru_set_ptr[s] ..
     * exc_thru_set_ptr[s+1]).  A path of group g moves to the next stage at
     * a pin of its next set, and only a path through every set, in order,
     * gets the group's action (else the default check).  Tags are then one
     * per stage: n_tags = 1 + sum over groups of (sets + 1) <= 32.
     * exc_thru_ptr NULL: no through sets. */
    int32_t n_exc;
    const int32_t *exc_from_ptr, *exc_from, *exc_to_ptr, *exc_to, *exc_action;
    const float *exc_mult;
    const int32_t *exc_thru_ptr, *exc_thru_set_ptr, *exc_thru_pin;
    /* RC from positions (rc_ptr == NULL; Sec. III "Parasitics (RC) inputs":
     * pin positions and unit R/C along x and y).  wire_model:
     *   STA_WIRE_STAR (0): one segment per sink of Manhattan length L,
     *     R = r_per_um L, C = c_per_um L split half at each end;
     *   STA_WIRE_STEINER (1): a rectilinear Steiner tree per net, rebuilt at
     *     every update from the current positions -- coordinates rounded to
     *     integer nm (the float product x * 1000, nearest, ties to even),
     *     Prim's rectilinear MST from the driver (ties: smaller distance,
     *     then lower pin index in net order, then the earlier-attached tree
     *     node), then greedy median insertion: over every node u and pair of
     *     its neighbours v < w, the Steiner point M = (median x, median y) of
     *     {u, v, w} gains d(u,v) + d(u,w) - d(M,u) - d(M,v) - d(M,w); the
     *     largest gain (first in (u, v, w) order) is applied while positive,
     *     at most 2 (n - 1) times for n pins; nets of more than 64 pins keep
     *     the MST.  Each tree edge of lengths Lx, Ly (um) has R = r_per_um Lx
     *     + r_per_um_y Ly and wire C = c_per_um Lx + c_per_um_y Ly split half
     *     at each end (r_per_um_y, c_per_um_y <= 0: the x values).
     *     Positions must satisfy |x|, |y| <= 1e6 um.  Elmore or Arnoldi
     *     (net_model) on the tree.  Not differentiable (no sta_backward). */
    int32_t wire_model;
    float r_per_um_y, c_per_um_y;
} sta_design_desc;

/* parasitics built from positions (sta_design_desc.wire_model) */
enum { STA_WIRE_STAR = 0, STA_WIRE_STEINER = 1 };

/* net delay calculators (sta_design_desc.net_model) */
enum { STA_NET_ELMORE = 0, STA_NET_ARNOLDI = 1 };

/* Sizes of a levelised design (sta_plan / sta_stats). */
typedef struct {
    int64_t n_pins, n_cells, n_nets, n_items;    /* items: PIs + cells */
    int64_t n_cell_arcs, n_net_arcs, n_rc_nodes, n_endpoints;
    int32_t n_levels;                            /* propagation levels (items) */
    int32_t n_corners;
    int32_t max_level_width;
    int32_t n_designs;                           /* 1, or the batch size */
    int64_t device_bytes;                        /* device memory the context holds */
    int32_t launches_per_update;                 /* kernels one sta_update_timing launches */
    int32_t launches_per_backward;               /* kernels one sta_backward launches (differentiable
                                                    contexts, current reverse-sweep schedule; else 0) */
    int32_t n_tags;                              /* exception tags (1 + sum over groups of (through
                                                    sets + 1)); per-pin states = n_corners * n_tags */
} sta_plan_info;

/* Per-corner summary returned by sta_report_slack. */
typedef struct {
    double wns_setup, tns_setup;   /* WNS = min(0, worst), TNS = sum of negatives */
    double wns_hold, tns_hold;
    double worst_setup, worst_hold;   /* raw worst endpoint slacks (may be > 0) */
    int64_t n_viol_setup, n_viol_hold;
} sta_corner_report;

/* Host only, no GPU needed: validate a design and levelise its timing graph.
 * Fills *out.  Returns STA_EINVAL (message via sta_plan_error) or
 * STA_ECYCLE.  Defined by the CSR database of Sec. III plus the level
 * ordering that graph propagation (Sec. I) needs. */
sta_status sta_plan(const sta_design_desc *desc, sta_plan_info *out);
/* Host only: the propagation level of every cell, cell_level[n_cells]
 * (flip-flops 0; a gate 1 + the highest level among the cells driving its
 * inputs, primary inputs counting as level 0).  Errors as sta_plan. */
sta_status sta_plan_levels(const sta_design_desc *desc, int32_t *cell_level);

/* Partition of the graph for the tile schedule (STA_SCHED_TILE): sizes and
 * how many dependencies stay inside a tile. */
typedef struct {
    int32_t n_tiles, n_steps;        /* tiles (resident blocks), steps (levels + 1) */
    int32_t wave_items, ring_slots;  /* entries one wave of a block runs; shared-memory ring slots */
    int32_t max_step_entries;        /* largest list of one tile at one step */
    int32_t pad;
    int64_t fwd_edges, fwd_local;    /* gate-input -> driver dependencies, and those read from the ring */
    int64_t bwd_edges, bwd_local;    /* driver -> gate-input dependencies, and those read from the ring */
    int64_t crit_edges, crit_local;  /* critical fan-in edges, and those inside one tile */
} sta_tile_info;

/* Host only, no GPU needed: build the tile schedule's partition of a design
 * into n_tiles tiles (as sta_set_schedule(STA_SCHED_TILE, n_tiles) would),
 * check it by replaying the kernels' ring use on the host (every entry in
 * exactly one list at its level, every ring read finds its producer), and
 * report its statistics.  Errors: as sta_plan; STA_EINVAL also for
 * n_tiles < 1 or a failed check (message via sta_plan_error). */
sta_status sta_plan_tiles(const sta_design_desc *desc, int32_t n_tiles, sta_tile_info *out);

/* Statistics of the context's current tile partition (zeros unless the
 * schedule is STA_SCHED_TILE). */
sta_status sta_get_tile_info(const sta_ctx *ctx, sta_tile_info *out);

/* Message of the last failed sta_plan / sta_create on this thread. */
const char *sta_plan_error(void);

/* Validate, levelise, renumber pins level-major and upload everything to
 * `device`.  The context owns its device memory (cudaMalloc) until
 * sta_destroy.  Errors: STA_EINVAL, STA_ECYCLE, STA_ENOMEM, STA_ECUDA. */
sta_status sta_create(const sta_design_desc *desc, int device, sta_ctx **out);

/* Many independent designs in one context: they are packed into one graph
 * whose levels are the union of the designs' levels, so one launch sequence
 * times all of them.  Every design must use the same library (same pointer
 * contents), the same n_corners and the same parasitic kind.  Reports are per
 * design (sta_report_slack_design).  Errors as sta_create. */
sta_status sta_create_batch(const sta_design_desc *const *descs, int32_t n_designs, int device,
                            sta_ctx **out);

/* Replace RC values (same topology): R and C as in sta_design_desc, in the
 * caller's node order, total n_rc_nodes floats each.  Takes effect at the
 * next sta_update_timing. */
sta_status sta_set_rc(sta_ctx *ctx, const float *R, const float *C, sta_mem mem);

/* Stage new RC values for the next sta_update_timing without waiting: R and
 * C (host, page-locked for the copies to overlap, or device; the caller's
 * node order, n_rc_nodes floats each) are copied on `stream` into one of two
 * staging buffers, and the next sta_update_timing, on its own stream, waits
 * for that copy and reorders the values into place before its pass.  So the
 * copy of the next step's parasitics can run while the current update
 * computes.  The source buffers must stay unchanged until the copy has run
 * (synchronise `stream`, or wait for the next update).  A later call before
 * the next update replaces the staged values.  Errors: STA_ESTATE if the
 * context uses positions. */
sta_status sta_set_rc_async(sta_ctx *ctx, const float *R, const float *C, sta_mem mem, void *stream);

/* Replace cell positions (positions mode): cell_xy[n_cells*2] um, copied on
 * `stream`.  Errors: STA_ESTATE if the context uses RC trees. */
sta_status sta_set_positions(sta_ctx *ctx, const float *cell_xy, sta_mem mem, void *stream);

/* Replace cell types (resizing), host array [n_cells]; each new type must
 * have the same number of inputs and the same kind as the old one. */
sta_status sta_set_cell_types(sta_ctx *ctx, const int32_t *cell_type);

/* Replace the corner scale factors (n_corners host floats each; see
 * sta_design_desc).  Takes effect at the next sta_update_timing. */
sta_status sta_set_corners(sta_ctx *ctx, const float *lut_scale, const float *rc_scale);

/* Pick the fastest schedule for this context: times `trials` graph launches
 * of each candidate (level schedule with 64, 128 and 256 threads per block;
 * dataflow schedule with a persistent grid from occupancy, one block per SM
 * and two per SM; cooperative schedule with a grid from occupancy and one
 * block per SM) on `stream`, keeps the best and selects it.  In a
 * differentiable context it also times sta_backward with each reverse-sweep
 * schedule (sta_set_adjoint_schedule) and selects the faster.  Choices are
 * cached per (device, graph shape); a cached choice is reused unless `force`.
 * Outputs (nullable): the chosen schedule, its parameter and its ms per
 * update.  Runs full timing updates (the context's results are those of the
 * last one). */
sta_status sta_autotune(sta_ctx *ctx, void *stream, int32_t trials, int32_t force, int32_t *schedule,
                        int32_t *param, float *ms);

/* Change the ideal clock period (ns) used by the next sta_update_timing. */
sta_status sta_set_clock(sta_ctx *ctx, float period_ns);

/* Resize n cells: cell_type of cells[i] becomes types[i] (both arrays in
 * `mem`, int32).  Each new type must keep the cell's input count and kind
 * (checked on the device; a violation sets the device error word, reported
 * as STA_EINVAL by the next synchronising call, and leaves that cell
 * unchanged).  Updates the cell's type and the capacitance its input pins
 * present to their nets, on `stream`, without touching other cells. */
sta_status sta_resize_cells(sta_ctx *ctx, const int32_t *cells, const int32_t *types, int32_t n, sta_mem mem,
                            void *stream);

/* Select the propagation schedule (STA_SCHED_*) and its parameter: threads
 * per block for LEVEL (0 = 128); for DATAFLOW and COOP the persistent grid
 * size in blocks (0 = every block the occupancy allows on this device); for
 * TILE the number of tiles (0 = one per SM), at most the co-resident
 * blocks of its kernels.  TILE partitions the graph on the host (every item
 * goes to the tile of its critical fan-in while that tile's level has room,
 * so that most level-to-level dependencies stay inside one block and pass
 * through shared memory) and uploads the partition; it needs at most 4095
 * levels.  Errors: STA_EINVAL (unknown schedule, parameter out of range,
 * library too large for the shared-memory copy, too many levels or tiles),
 * STA_ECUDA / STA_ENOMEM (set-up on the device). */
sta_status sta_set_schedule(sta_ctx *ctx, int32_t schedule, int32_t param);

/* Reverse sweep of sta_backward: STA_SCHED_DATAFLOW (one persistent kernel,
 * the default; used only when the cell library fits its shared-memory copy)
 * or STA_SCHED_LEVEL (one launch per level).  Both compute the same
 * gradient. */
sta_status sta_set_adjoint_schedule(sta_ctx *ctx, int32_t schedule);

/* Dataflow and cooperative schedules: polls a wait (on a ready flag, or on
 * the grid barrier between levels) may spend before the pass gives up and
 * the next synchronising call returns STA_ETIMEOUT (default 2^23, seconds of
 * waiting; a real wait ends in microseconds). */
sta_status sta_set_wait_limit(sta_ctx *ctx, int64_t polls);

/* Failure-detection test hook (dataflow schedule): while `cell` >= 0, the
 * forward pass of that cell never publishes its results to the items that
 * read them, so their bounded waits run out and the update reports
 * STA_ETIMEOUT with the context still usable; -1 restores normal
 * operation. */
sta_status sta_debug_hold_cell(sta_ctx *ctx, int32_t cell);

/* Full analysis on `stream` (Sec. III: the engine's graph-based analysis
 * with the "Delay models" paragraph's NLDM cell delays and Elmore or
 * Arnoldi net delays): net delay calculation, forward arrival/slew
 * propagation, endpoint required times, backward required-time propagation,
 * pin and endpoint slacks, FP64 WNS/TNS.  Asynchronous; errors of the
 * device work surface at the next synchronising call. */
sta_status sta_update_timing(sta_ctx *ctx, void *stream);

/* Wait for the context's work on `stream` and surface device errors. */
sta_status sta_sync(sta_ctx *ctx, void *stream);

/* Synchronise and fill reports[n_corners] (design 0 of a batch): WNS/TNS
 * and worst slacks per corner, the WNS/TNS of Sec. III "Report options".
 * Caller owns `reports` (host memory). */
sta_status sta_report_slack(sta_ctx *ctx, void *stream, sta_corner_report *reports);
/* Same for design `d` of a batch context. */
sta_status sta_report_slack_design(sta_ctx *ctx, int32_t d, void *stream, sta_corner_report *reports);

/* Copy one per-pin array (STA_AT, STA_SLEW, STA_RAT or STA_SLACK) into
 * out[n_pins][n_corners][4] in the caller's pin numbering, on `stream`.
 * For a batch, pins of design d follow those of design d-1. */
sta_status sta_get_pin_state(sta_ctx *ctx, int32_t which, float *out, sta_mem mem, void *stream);

/* Steiner wirelength of every net at the last sta_update_timing:
 * wl_nm[n_nets] (int64, nm) in the caller's net order (for a batch, nets of
 * design d follow those of design d-1), the sum of the Manhattan lengths of
 * the tree's edges on integer nm coordinates.  Errors: STA_ESTATE unless the
 * context builds Steiner trees (STA_WIRE_STEINER) and has been updated. */
sta_status sta_get_net_wirelength(sta_ctx *ctx, int64_t *wl_nm, sta_mem mem, void *stream);

/* Endpoint slacks: setup[n_endpoints][n_corners] = min over rise/fall of the
 * late slack, hold likewise with the early slack, viol_* = slack < 0 as
 * 0/1 bytes.  Any output may be NULL. */
sta_status sta_get_endpoint_slack(sta_ctx *ctx, float *setup, float *hold, uint8_t *viol_setup,
                                  uint8_t *viol_hold, sta_mem mem, void *stream);

/* Differentiable mode (gamma_ns > 0, positions; the timing feedback a
 * timing-driven placer takes from the engine, Sec. IV-C): after
 * sta_update_timing, compute the smoothed objective
 *   J = w_tns * TNS_g + w_wns * WNS_g,  summed over corners, with
 *   s_e   = smooth min over rise/fall of (RAT_e - AT_late,e),
 *   TNS_g = -sum_e g * softplus(-s_e / g),  WNS_g = -g * log sum_e exp(-s_e / g)
 * and its gradient with respect to every cell position by a hand-written
 * adjoint of the forward pass (LSE merges, NLDM interpolation, Elmore delay
 * and variance of the star or of the Steiner tree).  On Steiner trees the
 * gradient is that of the update's trees held fixed: every tree node sits at
 * pin coordinates (a Steiner point takes medians) and moves with the lowest
 * pin of the net (driver first, then the sinks in net order) at that x or
 * y; the nm rounding of positions counts as the identity.
 * J_out: 1 double (+ per-corner TNS_g, WNS_g pairs if terms != NULL);
 * grad_xy: n_cells*2 doubles.  All three in `mem`; host outputs synchronise.
 * Errors: STA_ESTATE (no prior update, not differentiable, or Steiner trees
 * with STA_NET_ARNOLDI). */
sta_status sta_backward(sta_ctx *ctx, double w_tns, double w_wns, double *J_out, double *terms,
                        double *grad_xy, sta_mem mem, void *stream);

/* Top-k path report (Sec. III "Report options": top-k paths with a slack
 * threshold and a per-endpoint limit, as flattened CSR path pin arrays).
 * Per-endpoint limit 1: the endpoints of design `design` whose setup slack
 * at `corner` is below slack_lt (ns; +inf for no threshold), in increasing
 * slack (ties: lower endpoint index), the first k (k <= 4096); for each its
 * critical path, traced back from the endpoint at the edge with the smaller
 * late slack (ties: rise): a net sink steps to its net's driver (same
 * edge), a gate output to the input arc whose late arrival + NLDM delay is
 * largest (ties: lower input slot, then rise), a flip-flop Q to its CK
 * (rising edge); the path starts at a PI or CK.  Outputs (in `mem`, any of
 * the array pointers may be NULL):
 *   n_paths, n_pins      host int32: paths reported, pins over all paths;
 *   path_ptr[n_paths+1]  offsets of each path in the pin arrays;
 *   path_pin[n_pins]     caller pin ids, startpoint first, endpoint last;
 *   path_rf[n_pins]      edge at each pin (0 rise, 1 fall);
 *   path_at[n_pins]      late arrival at each pin (ns);
 *   path_slack[n_paths]  setup slack of each path's endpoint (ns);
 *   path_endpoint[n_paths] caller pin id of each endpoint.
 * Pin arrays hold pin_capacity entries; if the report needs more, returns
 * STA_EINVAL with n_pins set to the size needed.  Synchronises `stream`.
 * For a batch, pin ids follow sta_get_pin_state's numbering. */
sta_status sta_report_paths(sta_ctx *ctx, int32_t design, int32_t corner, int32_t k, float slack_lt,
                            int32_t *n_paths, int32_t *n_pins, int32_t *path_ptr, int32_t *path_pin,
                            int8_t *path_rf, float *path_at, float *path_slack, int32_t *path_endpoint,
                            int32_t pin_capacity, sta_mem mem, void *stream);

/* Top-k path report with a per-endpoint report limit (Sec. III "Report
 * options": top-k, per-endpoint report limit, slack-less-than threshold):
 * the k paths of design `design` with the smallest setup slack at `corner`
 * below slack_lt, at most per_endpoint (1..32) of them ending at any one
 * endpoint, in increasing slack (ties: the endpoint's place in the
 * per-endpoint-1 order, then the path's rank there).  A path's late
 * arrival adds, along the path, each cell arc's NLDM delay at the
 * analysis' input slew and output load and each net's delay; relative to
 * the critical path of sta_report_paths, a path leaves the critical fan-in
 * at some gate outputs, each costing (critical candidate - its candidate),
 * and its slack is its end edge's late slack plus those costs.  Only the k
 * worst endpoints can hold one of the k worst paths; each of them is
 * searched best-first over these deviations.  path_at holds the path's own
 * arrivals (the analysis' arrival less the deviation costs at or above the
 * pin); path_slack the path's slack; the other outputs as sta_report_paths
 * (an endpoint may appear several times).  per_endpoint = 1 is
 * sta_report_paths.  Errors: STA_EINVAL also when k * per_endpoint > 16384
 * or, with per_endpoint > 1, the design has timing exceptions. */
sta_status sta_report_paths_nworst(sta_ctx *ctx, int32_t design, int32_t corner, int32_t k, int32_t per_endpoint,
                                   float slack_lt, int32_t *n_paths, int32_t *n_pins, int32_t *path_ptr,
                                   int32_t *path_pin, int8_t *path_rf, float *path_at, float *path_slack,
                                   int32_t *path_endpoint, int32_t pin_capacity, sta_mem mem, void *stream);

/* Device views in the library's internal (level-major) pin order; valid
 * until the next sta_update_timing or sta_destroy.  gpu_pin_of[p] maps a
 * caller pin id to its internal index (device int32 array). */
typedef struct {
    const float *at;      /* [n_pins][n_corners][4][2] internal order: double-float (hi, lo), value hi + lo */
    const float *slew;    /* [n_pins][n_corners][4] */
    const float *rat;     /* [n_pins][n_corners][4][2] like at */
    const float *slack;   /* [n_pins][n_corners][4] */
    const int32_t *gpu_pin_of;              /* [n_pins] */
} sta_views;
sta_status sta_get_arrays(sta_ctx *ctx, sta_views *out);

/* Sizes and the device bytes held. */
sta_status sta_stats(const sta_ctx *ctx, sta_plan_info *out);

/* Wall time of the last update's passes measured with CUDA events when
 * enabled by sta_set_profiling(ctx, 1); ms[0..3] = net delays, forward,
 * backward (incl. endpoints and slack), reduction. */
sta_status sta_set_profiling(sta_ctx *ctx, int32_t on);
sta_status sta_last_timings(sta_ctx *ctx, float *ms4);

/* WNS/TNS of endpoint slacks without allocating anything.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc -- a flow whose
 * device memory is already reserved by another allocator, or a loop that must
 * not pay cudaMalloc's implicit synchronisation -- and so cannot create the
 * partial-sums buffer the regular reduction uses.  It computes what
 * sta_report_slack reports for a single design, from device arrays
 * setup[n_endpoints][n_corners] and hold[...] (as sta_get_endpoint_slack writes
 * them), into device out[n_corners][8] doubles in sta_corner_report field
 * order (violation counts as doubles), asynchronously on `stream`.
 * Its partial sums live in one fixed 384 KiB device array inside the library,
 * held on every GPU that loads it until the process exits; the limit is
 * ceil(n_endpoints / 4096) * n_corners <= 8192 (about 33.5 million
 * endpoint-corners), larger inputs return STA_EINVAL with a message on
 * stderr.  The kernels run on the current device, which must own setup,
 * hold, out and the stream.  The first call on a device looks the array's
 * address up (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  The cached address does not
 * survive cudaDeviceReset.  Every call shares the array: calls whose
 * kernels overlap on the GPU race, so serialise them (one stream).  Errors:
 * STA_EINVAL (NULL pointer, bad size), STA_ECUDA (a launch of this call
 * failed). */
sta_status sta_reduce_slack_noalloc(const float *setup, const float *hold, int64_t n_endpoints,
                                    int32_t n_corners, double *out, void *stream);

/* Message for the last failed call on this context (never NULL). */
const char *sta_last_error(const sta_ctx *ctx);
const char *sta_status_string(sta_status s);

/* Free the context and its device memory.  NULL is accepted. */
void sta_destroy(sta_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* STA_H */
