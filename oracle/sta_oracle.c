/*
 * sta_oracle.c -- plain, slow, FP64 reference static timing analysis.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that tests/, the smoke check and the CPU
 * baseline leg of the benchmark can compare the GPU library against an
 * independent computation.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * What it computes (HeteroSTA, arXiv 2511.11660): the graph-based part of
 * the STA engine the paper accelerates -- delay calculation followed by
 * graph propagation (Sec. I lists these among the engine's steps), with the
 * Elmore net delay calculator (Sec. III, "Delay models"), NLDM cell tables
 * (Sec. IV-A names the NLDM delay model), RC supplied as a
 * flattened tree or built from pin positions and unit R/C (Sec. III,
 * "Parasitics (RC) inputs") and WNS/TNS plus pin slacks as reports (Sec. III,
 * "Report options").  The paper prints no formula; it defers the STA
 * definitions to the textbook it cites (Bhasker & Chadha, "Static Timing
 * Analysis for Nanometer Designs").  Every formula below is therefore the
 * textbook / TAU-contest reading of those terms:
 *
 *   O1  NLDM bilinear interpolation, linear extrapolation off the table edge;
 *   O2  cell arcs with unateness, rise/fall x early/late, worst-slew merge;
 *   O3  Elmore delay and second moment on RC trees, slew = sqrt(s^2 + var);
 *   O4  endpoint required times, back-propagated required times, slack,
 *       WNS = min(0, worst endpoint slack), TNS = sum of negative slacks;
 *   O7  Arnoldi reduced-order net model (the paper's second delay
 *       calculator, Sec. III "Delay models"): sink delay = 50% crossing of
 *       the step response of an order-q congruence-projected model of the
 *       RC tree; the slew law of O3 is kept;
 *   O8  timing exceptions (Sec. III names an SDC exceptions manager, Sec.
 *       IV-B lists false and multicycle paths and min/max delays; the
 *       reading is SDC's set_false_path / set_multicycle_path -setup /
 *       set_max_delay / set_min_delay with -from startpoints and -to
 *       endpoints): every path carries the tag of its startpoint's group
 *       (0 = none); arrivals and required times are propagated per tag
 *       (slews are tag-free); an endpoint checks tag g with group g's action
 *       when it is in the group's endpoint list (or the list is empty) --
 *       false path: no check; multicycle M: setup capture edge at M * T,
 *       hold unchanged; max delay V: setup capture edge at V (the library
 *       setup time still applies at a flip-flop), hold unchanged; min delay
 *       V: hold edge at V (plus the hold time), setup unchanged -- and the
 *       default check otherwise; endpoint slack = min over tags.  With -through, a group
 *       has ordered through sets of gate input pins and one tag per stage:
 *       a path of the group moves to the next stage at a pin of the next
 *       set, and only a path through every set gets the group's action;
 *   O9  rectilinear Steiner tree RC from pin positions (Sec. III,
 *       "Parasitics (RC) inputs"): Prim MST on integer nm coordinates,
 *       greedy median Steiner insertion, breadth-first RC tree;
 *   O6  log-sum-exp smoothed objective and its hand-written FP64 adjoint
 *       with respect to cell (x, y) (not in the paper; it feeds a placer the
 *       way the paper's DREAMPlace integration consumes pin slacks, Sec. IV-C).
 *
 * Order of evaluation is a memoised depth-first topological order of the pin
 * graph (no levelisation), single threaded, every value in double.
 *
 * Units: ns, pF for library tables and loads; Ohm and fF for RC
 * (Ohm * fF = 1e-6 ns); um for positions.
 *
 * Parity pins (tests/test_oracle_*.py) fix: hand-worked LUT values, exact
 * reproduction of noise-free bilinear tables, closed-form Elmore / second
 * moment on single RC, uniform chains and star trees, brute-force path
 * enumeration on tiny DAGs, the GBA >= PBA invariant, slack = RAT - AT,
 * early <= late, WNS/TNS definitions, and the adjoint against central finite
 * differences of this file's own smoothed forward pass.
 */
#define _POSIX_C_SOURCE 200809L   /* clock_gettime */
#include <math.h>
#include <time.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* pin roles (the netlist description uses the same integer codes) */
enum { R_PI = 0, R_PO = 1, R_IN = 2, R_OUT = 3, R_D = 4, R_CK = 5, R_Q = 6 };
/* arc sense per (cell type, input slot) */
enum { S_NONE = -1, S_POS = 0, S_NEG = 1, S_NON = 2, S_RISE = 3 };
/* table order inside one arc: delay rise, delay fall, slew rise, slew fall */
enum { TB_DR = 0, TB_DF = 1, TB_SR = 2, TB_SF = 3 };

#define NLDM 7          /* 7 x 7 tables */
#define MAXSLOT 3       /* at most three inputs per cell */

enum { OK = 0, ERR_INVAL = 1, ERR_CYCLE = 2, ERR_NOMEM = 3 };

typedef struct {
    /* cell library */
    int32_t n_types;
    const int32_t *type_nin;   /* input pins per type (a DFF has D and CK) */
    const int32_t *type_kind;  /* 0 combinational, 1 flip-flop */
    const int32_t *arc_sense;  /* [n_types * 3] */
    const float *lut_idx1;     /* [n_types][3][4][7] input slew, ns */
    const float *lut_idx2;     /* [n_types][3][4][7] load, pF */
    const float *lut_val;      /* [n_types][3][4][49] value[i_slew * 7 + j_load] */
    const float *pin_cap;      /* [n_types * 4] pF by pin slot */
    double setup_ns, hold_ns, po_cap_pf;
    /* netlist */
    int32_t n_cells;
    const int32_t *cell_type;
    const int32_t *cell_pin_ptr; /* [n_cells + 1] */
    const int32_t *cell_pin;     /* pins of each cell, slot order, output last */
    int32_t n_pins;
    const int8_t *pin_role;
    int32_t n_nets;
    const int32_t *net_pin_ptr;  /* [n_nets + 1] */
    const int32_t *net_pin;      /* driver first, then sinks */
    /* parasitics: an RC tree per net, or positions (star tree) */
    const int32_t *rc_ptr;       /* [n_nets + 1] node ranges */
    const int32_t *rc_parent;    /* local parent index, -1 at the root (node 0) */
    const int32_t *rc_pin_node;  /* per net_pin entry: local node it sits on */
    const float *rc_R;           /* Ohm, per node (root ignored) */
    const float *rc_C;           /* fF wire capacitance, per node */
    const float *cell_xy;        /* [n_cells * 2] um; used when rc_ptr == NULL */
    const float *port_xy;        /* [n_pins * 2] um; read for PI/PO pins only */
    double r_per_um, c_per_um;   /* Ohm/um, fF/um */
    /* constraints */
    double period_ns, clk_slew_ns, pi_at_ns, pi_slew_ns;
    int32_t n_corners;
    const float *lut_scale;      /* [n_corners] */
    const float *rc_scale;       /* [n_corners] */
    double gamma_ns;             /* 0: hard max/min merges; > 0: log-sum-exp */
    int32_t net_model;           /* 0 Elmore; 1 Arnoldi reduced order (O7, RC trees only) */
    int32_t arnoldi_order;       /* Krylov dimension q of O7 (>= 1) */
    /* O8 timing exceptions: group g lists startpoint pins (PI or CK)
     * exc_from[exc_from_ptr[g] ..), endpoint pins (D or PO)
     * exc_to[exc_to_ptr[g] ..) (none = every endpoint), an action
     * (0 false path, 1 multicycle setup) and a multiplier */
    int32_t n_exc;
    const int32_t *exc_from_ptr, *exc_from, *exc_to_ptr, *exc_to, *exc_action;
    const float *exc_mult;
    /* O8 -through: group g's ordered through sets are sets
     * exc_thru_ptr[g] .. exc_thru_ptr[g+1]; set s lists gate input pins
     * exc_thru_pin[exc_thru_set_ptr[s] .. exc_thru_set_ptr[s+1]).  NULL: none. */
    const int32_t *exc_thru_ptr, *exc_thru_set_ptr, *exc_thru_pin;
    /* O9: RC from positions as a star (0) or a Steiner tree (1); unit R/C
     * along y for the Steiner tree (<= 0: the x values r_per_um, c_per_um) */
    int32_t wire_model;
    double r_per_um_y, c_per_um_y;
} orc_design;

/* ------------------------------------------------------------------ O1 */

/* Bilinear NLDM lookup at (s, l) with partial derivatives.
 * Segment i = largest index with idx1[i] <= s, clamped to [0, 5]; t is not
 * clamped, so inputs off the table extrapolate linearly from the edge
 * segment.  Same for the load axis. */
int orc_lut_eval(const float *idx1, const float *idx2, const float *val,
                 double s, double l, double *out3)
{
    int i = 0, j = 0;
    for (int k = 1; k <= NLDM - 2; ++k) {
        if ((double)idx1[k] <= s) i = k;
        if ((double)idx2[k] <= l) j = k;
    }
    double x0 = idx1[i], x1 = idx1[i + 1], y0 = idx2[j], y1 = idx2[j + 1];
    double t = (s - x0) / (x1 - x0);
    double u = (l - y0) / (y1 - y0);
    double v00 = val[i * NLDM + j], v10 = val[(i + 1) * NLDM + j];
    double v01 = val[i * NLDM + j + 1], v11 = val[(i + 1) * NLDM + j + 1];
    out3[0] = (1 - t) * (1 - u) * v00 + t * (1 - u) * v10 + (1 - t) * u * v01 + t * u * v11;
    out3[1] = ((1 - u) * (v10 - v00) + u * (v11 - v01)) / (x1 - x0);
    out3[2] = ((1 - t) * (v01 - v00) + t * (v11 - v10)) / (y1 - y0);
    return OK;
}

/* ------------------------------------------------------------------ O3 */

/* Elmore delay and second moment of one RC tree whose nodes are listed
 * parent before child (parent[0] = -1, R[0] ignored).
 *   Cdown_i = C_i + sum over children Cdown
 *   D_i     = D_parent + R_i Cdown_i
 *   M_i     = C_i D_i + sum over children M
 *   beta_i  = beta_parent + R_i M_i
 *   var_i   = 2 beta_i - D_i^2 */
int orc_rc_tree(int32_t n, const int32_t *parent, const double *R, const double *C,
                double *cdown, double *D, double *beta, double *var)
{
    if (n <= 0 || parent[0] != -1) return ERR_INVAL;
    for (int32_t i = 1; i < n; ++i)
        if (parent[i] < 0 || parent[i] >= i) return ERR_INVAL;
    double *M = (double *)malloc(sizeof(double) * (size_t)n);
    if (!M) return ERR_NOMEM;
    for (int32_t i = 0; i < n; ++i) cdown[i] = C[i];
    for (int32_t i = n - 1; i >= 1; --i) cdown[parent[i]] += cdown[i];
    D[0] = 0.0;
    for (int32_t i = 1; i < n; ++i) D[i] = D[parent[i]] + R[i] * cdown[i];
    for (int32_t i = 0; i < n; ++i) M[i] = C[i] * D[i];
    for (int32_t i = n - 1; i >= 1; --i) M[parent[i]] += M[i];
    beta[0] = 0.0;
    for (int32_t i = 1; i < n; ++i) beta[i] = beta[parent[i]] + R[i] * M[i];
    for (int32_t i = 0; i < n; ++i) var[i] = 2.0 * beta[i] - D[i] * D[i];
    free(M);
    return OK;
}

/* Reverse mode of orc_rc_tree: given Dbar_i = dJ/dD_i, Vbar_i = dJ/dvar_i
 * and Lbar = dJ/dCdown_0 (the load), the derivatives Rbar_i = dJ/dR_i
 * (Rbar_0 = 0) and Cbar_i = dJ/dC_i.  Each forward recurrence is taken
 * back in the opposite order:
 *   var_i = 2 beta_i - D_i^2          -> betabar_i = 2 Vbar_i, Dbar_i -= 2 D_i Vbar_i
 *   beta_i = beta_parent + R_i M_i    -> betabar summed up the subtree;
 *                                        Rbar_i += betabar_i M_i, Mbar_i = betabar_i R_i
 *   M_i = C_i D_i + sum children M    -> Mbar summed down from the root;
 *                                        Cbar_i += Mbar_i D_i, Dbar_i += Mbar_i C_i
 *   D_i = D_parent + R_i Cdown_i      -> Dbar summed up the subtree;
 *                                        Rbar_i += Dbar_i Cdown_i, Cdbar_i = Dbar_i R_i
 *   Cdown_i = C_i + sum children      -> Cdbar summed down from the root
 *                                        (Cdbar_0 = Lbar); Cbar_i += Cdbar_i. */
int orc_rc_tree_adjoint(int32_t n, const int32_t *parent, const double *R, const double *C, const double *Dbar,
                        const double *Vbar, double Lbar, double *Rbar, double *Cbar)
{
    if (n <= 0) return ERR_INVAL;
    double *cd = (double *)malloc(sizeof(double) * (size_t)n), *D = (double *)malloc(sizeof(double) * (size_t)n);
    double *be = (double *)malloc(sizeof(double) * (size_t)n), *va = (double *)malloc(sizeof(double) * (size_t)n);
    double *M = (double *)malloc(sizeof(double) * (size_t)n), *bb = (double *)malloc(sizeof(double) * (size_t)n);
    double *mb = (double *)malloc(sizeof(double) * (size_t)n), *db = (double *)malloc(sizeof(double) * (size_t)n);
    double *cb = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = (!cd || !D || !be || !va || !M || !bb || !mb || !db || !cb) ? ERR_NOMEM : OK;
    if (!rc) rc = orc_rc_tree(n, parent, R, C, cd, D, be, va);
    if (!rc) {
        for (int32_t i = 0; i < n; ++i) M[i] = C[i] * D[i];
        for (int32_t i = n - 1; i >= 1; --i) M[parent[i]] += M[i];
        for (int32_t i = 0; i < n; ++i) {
            Rbar[i] = 0.0;
            Cbar[i] = 0.0;
            bb[i] = 2.0 * Vbar[i];
        }
        for (int32_t i = n - 1; i >= 1; --i) {
            Rbar[i] += bb[i] * M[i];
            bb[parent[i]] += bb[i];
        }
        for (int32_t i = 0; i < n; ++i) mb[i] = (i ? bb[i] * R[i] : 0.0) + (i ? mb[parent[i]] : 0.0);
        for (int32_t i = 0; i < n; ++i) {
            Cbar[i] += mb[i] * D[i];
            db[i] = Dbar[i] - 2.0 * D[i] * Vbar[i] + mb[i] * C[i];
        }
        for (int32_t i = n - 1; i >= 1; --i) {
            Rbar[i] += db[i] * cd[i];
            db[parent[i]] += db[i];
        }
        for (int32_t i = 0; i < n; ++i) cb[i] = (i ? db[i] * R[i] + cb[parent[i]] : Lbar);
        for (int32_t i = 0; i < n; ++i) Cbar[i] += cb[i];
    }
    free(cd); free(D); free(be); free(va); free(M); free(bb); free(mb); free(db); free(cb);
    return rc;
}

/* ------------------------------------------------------------------ O7 */

/* Solve G x = y for an RC tree whose root (node 0) is held at 0 V: G is the
 * nodal conductance matrix of nodes 1..n-1.  The current through the edge
 * above node i is the sum of y over i's subtree, so x_i = x_parent + R_i *
 * (subtree sum of y).  x[0] = 0; y[0] is ignored. */
static void tree_solve(int32_t n, const int32_t *parent, const double *R, const double *y, double *x)
{
    for (int32_t i = 0; i < n; ++i) x[i] = i ? y[i] : 0.0;
    for (int32_t i = n - 1; i >= 1; --i) if (parent[i] > 0) x[parent[i]] += x[i];
    x[0] = 0.0;
    for (int32_t i = 1; i < n; ++i) x[i] = x[parent[i]] + R[i] * x[i];
}

/* Symmetric eigen-decomposition by cyclic Jacobi rotations: a (q x q, row
 * major) is overwritten, eigenvalues in w, eigenvectors in the columns of v. */
static void jacobi_eig(int q, double *a, double *w, double *v)
{
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) v[i * q + j] = i == j;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < q; ++i)
            for (int j = i + 1; j < q; ++j) off += a[i * q + j] * a[i * q + j];
        if (off < 1e-30) break;
        for (int p = 0; p < q; ++p)
            for (int r = p + 1; r < q; ++r) {
                const double apr = a[p * q + r];
                if (fabs(apr) < 1e-300) continue;
                const double theta = (a[r * q + r] - a[p * q + p]) / (2.0 * apr);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < q; ++k) {   /* A <- A J (columns p, r) */
                    const double akp = a[k * q + p], akr = a[k * q + r];
                    a[k * q + p] = c * akp - s * akr;
                    a[k * q + r] = s * akp + c * akr;
                }
                for (int k = 0; k < q; ++k) {   /* A <- J^T A (rows p, r) */
                    const double apk = a[p * q + k], ark = a[r * q + k];
                    a[p * q + k] = c * apk - s * ark;
                    a[r * q + k] = s * apk + c * ark;
                }
                for (int k = 0; k < q; ++k) {   /* V <- V J */
                    const double vkp = v[k * q + p], vkr = v[k * q + r];
                    v[k * q + p] = c * vkp - s * vkr;
                    v[k * q + r] = s * vkp + c * vkr;
                }
            }
    }
    for (int i = 0; i < q; ++i) w[i] = a[i * q + i];
}

/* Arnoldi reduced-order model of an RC tree driven by a unit step at node 0
 * (R in Ohm, C in fF, nodes parent before child; C[0] ignored).  The node
 * voltages v of nodes 1..m (m = n - 1) obey C v' + G v = b u, u the root
 * voltage, so the DC solution is v = 1.  The order-q Krylov space of
 * A = G^-1 C started at G^-1 b = 1 is spanned by an orthonormal basis V
 * (modified Gram-Schmidt, each new direction A v_j by one tree solve); the
 * congruence projection G_r = V^T G V, C_r = V^T C V, b_r = V^T b keeps a
 * passive model whose sink voltage is v_s(t) = sum_k a_sk (1 - exp(-l_k t))
 * with l_k the eigenvalues of C_r^-1 G_r (through the Cholesky factor of
 * C_r and a symmetric eigensolve).  t50[i] = the time v_i(t) first reaches
 * half its final value (bisection), for every node (t50[0] = 0).  q is
 * capped at m; q = m reproduces the unreduced response.  The basis stops
 * growing when a new direction's part orthogonal to the basis is below
 * 1e-5 of its length (the Krylov space is exhausted, e.g. by symmetric
 * branches): what is left is rounding, not a direction. */
int orc_arnoldi_t50(int32_t n, const int32_t *parent, const double *R, const double *C, int32_t q_in, double *t50)
{
    if (n <= 0 || parent[0] != -1 || q_in < 1) return ERR_INVAL;
    for (int32_t i = 1; i < n; ++i)
        if (parent[i] < 0 || parent[i] >= i || !(R[i] > 0.0)) return ERR_INVAL;   /* G needs every R > 0 */
    t50[0] = 0.0;
    const int32_t m = n - 1;
    if (m == 0) return OK;
    const int q = q_in < m ? q_in : m;
    double *V = (double *)calloc((size_t)q * n, sizeof(double));   /* V[j*n + i], entries 1..m used */
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *Gr = (double *)calloc((size_t)q * q, sizeof(double)), *Cr = (double *)calloc((size_t)q * q, sizeof(double));
    double *L = (double *)calloc((size_t)q * q, sizeof(double)), *M = (double *)calloc((size_t)q * q, sizeof(double));
    double *T = (double *)calloc((size_t)q * q, sizeof(double)), *W = (double *)calloc((size_t)q * q, sizeof(double));
    double *lam = (double *)calloc((size_t)q, sizeof(double)), *br = (double *)calloc((size_t)q, sizeof(double));
    double *c = (double *)calloc((size_t)q, sizeof(double)), *yinf = (double *)calloc((size_t)q, sizeof(double));
    double *h = (double *)calloc((size_t)q, sizeof(double)), *a = (double *)calloc((size_t)q, sizeof(double));
    int rc = OK;
    if (!V || !y || !x || !Gr || !Cr || !L || !M || !T || !W || !lam || !br || !c || !yinf || !h || !a) {
        rc = ERR_NOMEM;
        goto done;
    }
    /* Krylov basis */
    for (int32_t i = 1; i < n; ++i) V[i] = 1.0 / sqrt((double)m);
    int qq = 1;
    for (int j = 1; j < q; ++j) {
        for (int32_t i = 0; i < n; ++i) y[i] = i ? C[i] * V[(j - 1) * n + i] : 0.0;
        tree_solve(n, parent, R, y, x);
        double len = 0.0;
        for (int32_t i = 1; i < n; ++i) len += x[i] * x[i];
        len = sqrt(len);
        for (int p = 0; p < j; ++p) {   /* modified Gram-Schmidt */
            double dot = 0.0;
            for (int32_t i = 1; i < n; ++i) dot += V[p * n + i] * x[i];
            for (int32_t i = 1; i < n; ++i) x[i] -= dot * V[p * n + i];
        }
        double nrm = 0.0;
        for (int32_t i = 1; i < n; ++i) nrm += x[i] * x[i];
        nrm = sqrt(nrm);
        if (!(nrm > 1e-5 * len)) break;   /* the Krylov space is exhausted (to 1e-5 of the new direction) */
        for (int32_t i = 1; i < n; ++i) V[j * n + i] = x[i] / nrm;
        qq = j + 1;
    }
    /* projected matrices: v^T G w = sum over edges of dv dw / R (root at 0 V);
     * b = G * 1, so b_r = V^T G 1 = sum over the root's edges of v / R */
    for (int p = 0; p < qq; ++p)
        for (int r = 0; r < qq; ++r) {
            double g = 0.0, cc = 0.0;
            for (int32_t i = 1; i < n; ++i) {
                const double dp = V[p * n + i] - (parent[i] ? V[p * n + parent[i]] : 0.0);
                const double dr = V[r * n + i] - (parent[i] ? V[r * n + parent[i]] : 0.0);
                g += dp * dr / R[i];
                cc += C[i] * V[p * n + i] * V[r * n + i];
            }
            Gr[p * qq + r] = g;
            Cr[p * qq + r] = cc;
        }
    for (int p = 0; p < qq; ++p) {
        double s = 0.0;
        for (int32_t i = 1; i < n; ++i) if (parent[i] == 0) s += V[p * n + i] / R[i];
        br[p] = s;
    }
    /* Cholesky C_r = L L^T */
    for (int i = 0; i < qq; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = Cr[i * qq + j];
            for (int k = 0; k < j; ++k) s -= L[i * qq + k] * L[j * qq + k];
            if (i == j) {
                if (!(s > 0.0)) { rc = ERR_INVAL; goto done; }   /* a zero-capacitance subspace */
                L[i * qq + i] = sqrt(s);
            } else {
                L[i * qq + j] = s / L[j * qq + j];
            }
        }
    /* M = L^-1 G_r L^-T: T = L^-1 G_r (forward substitution per column), M = T L^-T */
    for (int col = 0; col < qq; ++col)
        for (int i = 0; i < qq; ++i) {
            double s = Gr[i * qq + col];
            for (int k = 0; k < i; ++k) s -= L[i * qq + k] * T[k * qq + col];
            T[i * qq + col] = s / L[i * qq + i];
        }
    for (int row = 0; row < qq; ++row)
        for (int i = 0; i < qq; ++i) {
            double s = T[row * qq + i];
            for (int k = 0; k < i; ++k) s -= L[i * qq + k] * M[row * qq + k];
            M[row * qq + i] = s / L[i * qq + i];
        }
    for (int i = 0; i < qq; ++i)   /* symmetrise rounding */
        for (int j = i + 1; j < qq; ++j) M[i * qq + j] = M[j * qq + i] = 0.5 * (M[i * qq + j] + M[j * qq + i]);
    jacobi_eig(qq, M, lam, W);
    /* y' + M y = c with c = L^-1 b_r, y = L^T z; y_inf = M^-1 c = W diag(1/l) W^T c */
    for (int i = 0; i < qq; ++i) {
        double s = br[i];
        for (int k = 0; k < i; ++k) s -= L[i * qq + k] * c[k];
        c[i] = s / L[i * qq + i];
    }
    for (int k = 0; k < qq; ++k) {
        double s = 0.0;
        for (int i = 0; i < qq; ++i) s += W[i * qq + k] * c[i];
        yinf[k] = s / lam[k];   /* modal coordinates of y_inf */
    }
    for (int32_t node = 1; node < n; ++node) {
        /* v_node = e^T V z = h^T y with h = L^-1 V^T e_node; in modal form
         * v(t) = sum_k (h^T w_k) yinf_k (1 - exp(-l_k t)) */
        for (int i = 0; i < qq; ++i) {
            double s = V[i * n + node];
            for (int k = 0; k < i; ++k) s -= L[i * qq + k] * h[k];
            h[i] = s / L[i * qq + i];
        }
        double vinf = 0.0;
        for (int k = 0; k < qq; ++k) {
            double s = 0.0;
            for (int i = 0; i < qq; ++i) s += h[i] * W[i * qq + k];
            a[k] = s * yinf[k];
            vinf += a[k];
        }
        /* bracket the first time v reaches vinf / 2, then bisect */
        double lmin = lam[0];
        for (int k = 1; k < qq; ++k) lmin = fmin(lmin, lam[k]);
        double hi = 1.0 / lmin, lo = 0.0;
        for (int it = 0; it < 200; ++it) {
            double v = 0.0;
            for (int k = 0; k < qq; ++k) v += a[k] * (1.0 - exp(-lam[k] * hi));
            if (v >= 0.5 * vinf) break;
            lo = hi;
            hi *= 2.0;
        }
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            double v = 0.0;
            for (int k = 0; k < qq; ++k) v += a[k] * (1.0 - exp(-lam[k] * mid));
            if (v >= 0.5 * vinf) hi = mid;
            else lo = mid;
        }
        t50[node] = 0.5 * (lo + hi);
    }
done:
    free(V); free(y); free(x); free(Gr); free(Cr); free(L); free(M); free(T); free(W);
    free(lam); free(br); free(c); free(yinf); free(h); free(a);
    return rc;
}

/* --------------------------------------------------------- helpers */

typedef struct {
    int32_t *cell, *slot;     /* per pin: owning cell (-1 for ports) and slot */
    int32_t *drv_net;         /* per pin: net it drives, -1 */
    int32_t *sink_net;        /* per pin: net it is a sink of, -1 */
    int32_t *sink_entry;      /* per pin: index into net_pin of that sink entry */
} pin_info;

static void free_info(pin_info *pi)
{
    free(pi->cell); free(pi->slot); free(pi->drv_net); free(pi->sink_net); free(pi->sink_entry);
}

static int build_info_checked(const orc_design *d, pin_info *pi);

static int build_info(const orc_design *d, pin_info *pi)
{
    memset(pi, 0, sizeof(*pi));
    int rc = build_info_checked(d, pi);
    if (rc) free_info(pi);
    return rc;
}

static int build_info_checked(const orc_design *d, pin_info *pi)
{
    size_t P = (size_t)d->n_pins;
    pi->cell = (int32_t *)malloc(P * 4); pi->slot = (int32_t *)malloc(P * 4);
    pi->drv_net = (int32_t *)malloc(P * 4); pi->sink_net = (int32_t *)malloc(P * 4);
    pi->sink_entry = (int32_t *)malloc(P * 4);
    if (!pi->cell || !pi->slot || !pi->drv_net || !pi->sink_net || !pi->sink_entry) return ERR_NOMEM;
    for (size_t p = 0; p < P; ++p) {
        pi->cell[p] = -1; pi->slot[p] = -1; pi->drv_net[p] = -1;
        pi->sink_net[p] = -1; pi->sink_entry[p] = -1;
    }
    for (int32_t c = 0; c < d->n_cells; ++c) {
        int32_t t = d->cell_type[c];
        if (t < 0 || t >= d->n_types) return ERR_INVAL;
        if (d->cell_pin_ptr[c + 1] - d->cell_pin_ptr[c] != d->type_nin[t] + 1) return ERR_INVAL;
        for (int32_t k = d->cell_pin_ptr[c]; k < d->cell_pin_ptr[c + 1]; ++k) {
            int32_t p = d->cell_pin[k];
            if (p < 0 || p >= d->n_pins || pi->cell[p] != -1) return ERR_INVAL;
            pi->cell[p] = c; pi->slot[p] = k - d->cell_pin_ptr[c];
        }
    }
    for (int32_t n = 0; n < d->n_nets; ++n) {
        int32_t b = d->net_pin_ptr[n], e = d->net_pin_ptr[n + 1];
        if (e - b < 1) return ERR_INVAL;
        int32_t drv = d->net_pin[b];
        if (drv < 0 || drv >= d->n_pins || pi->drv_net[drv] != -1) return ERR_INVAL;
        int r = d->pin_role[drv];
        if (r != R_PI && r != R_OUT && r != R_Q) return ERR_INVAL;
        pi->drv_net[drv] = n;
        for (int32_t k = b + 1; k < e; ++k) {
            int32_t s = d->net_pin[k];
            if (s < 0 || s >= d->n_pins || pi->sink_net[s] != -1) return ERR_INVAL;
            int rs = d->pin_role[s];
            if (rs != R_IN && rs != R_D && rs != R_PO) return ERR_INVAL;
            pi->sink_net[s] = n; pi->sink_entry[s] = k;
        }
    }
    /* every pin that needs a driver has one */
    for (int32_t p = 0; p < d->n_pins; ++p) {
        int r = d->pin_role[p];
        if ((r == R_IN || r == R_D || r == R_PO) && pi->sink_net[p] < 0) return ERR_INVAL;
    }
    return OK;
}

static const float *tab_base(const float *arr, int32_t t, int32_t slot, int tb, int per)
{
    return arr + (((size_t)t * MAXSLOT + (size_t)slot) * 4 + (size_t)tb) * (size_t)per;
}

static double lut(const orc_design *d, int32_t t, int32_t slot, int tb, double s, double l,
                  double *ds, double *dl)
{
    double o[3];
    orc_lut_eval(tab_base(d->lut_idx1, t, slot, tb, NLDM), tab_base(d->lut_idx2, t, slot, tb, NLDM),
                 tab_base(d->lut_val, t, slot, tb, NLDM * NLDM), s, l, o);
    if (ds) *ds = o[1];
    if (dl) *dl = o[2];
    return o[0];
}

/* rf_in values that reach rf_out through an arc of the given sense */
static int rf_inputs(int sense, int rf_out, int *rf_in)
{
    switch (sense) {
    case S_POS: rf_in[0] = rf_out; return 1;
    case S_NEG: rf_in[0] = 1 - rf_out; return 1;
    case S_NON: rf_in[0] = 0; rf_in[1] = 1; return 2;
    case S_RISE: rf_in[0] = 0; return 1;
    default: return 0;
    }
}

/* merge: late = max, early = min; gamma > 0 replaces them by
 * gamma * log sum exp(x / gamma) (and its mirror for min). */
static double merge(const double *x, int n, int late, double gamma)
{
    if (n == 0) return late ? -INFINITY : INFINITY;
    double m = x[0];
    for (int i = 1; i < n; ++i) m = late ? fmax(m, x[i]) : fmin(m, x[i]);
    if (gamma <= 0.0 || isinf(m)) return m;   /* no finite candidate (another tag's arrivals) */
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp((late ? (x[i] - m) : (m - x[i])) / gamma);
    return late ? m + gamma * log(s) : m - gamma * log(s);
}

static double pin_cap_of(const orc_design *d, const pin_info *pi, int32_t p)
{
    if (d->pin_role[p] == R_PO) return d->po_cap_pf;
    int32_t c = pi->cell[p];
    return d->pin_cap[(size_t)d->cell_type[c] * 4 + (size_t)pi->slot[p]];
}

static void pin_xy(const orc_design *d, const pin_info *pi, int32_t p, double *x, double *y)
{
    int32_t c = pi->cell[p];
    if (c >= 0) { *x = d->cell_xy[2 * (size_t)c]; *y = d->cell_xy[2 * (size_t)c + 1]; }
    else if (d->port_xy) { *x = d->port_xy[2 * (size_t)p]; *y = d->port_xy[2 * (size_t)p + 1]; }
    else { *x = 0.0; *y = 0.0; }
}

/* ------------------------------------------------------------------ O9 */

/* Rectilinear Steiner tree of one net from its pin positions (Sec. III,
 * "Parasitics (RC) inputs": the placement flow sends pin positions and unit
 * R/C along x and y and the engine builds Steiner-tree RC).  The paper's
 * tree builder (GPU FLUTE) is not reproduced; this is the reading:
 *
 *   coordinates  x, y in um (float) -> integer nm, X = round-to-nearest-even
 *                of the float product x * 1000 (every geometric decision
 *                below is then exact integer arithmetic);
 *   distance     d(a, b) = |Xa - Xb| + |Ya - Yb|;
 *   1. MST       Prim from pin 0 (the driver): each step attaches the
 *                outside pin u and tree node v with the smallest
 *                (d(u, v), u, rank of v), rank = order of attachment;
 *   2. Steiner   greedy median insertion, at most 2 (n - 1) times: over
 *                every live node u (ascending index) and every pair v < w
 *                of u's neighbours, M = (median of X, median of Y) of
 *                {u, v, w} and gain = d(u,v) + d(u,w) - d(M,u) - d(M,v) -
 *                d(M,w); take the largest gain (ties: the first in that
 *                order); stop when it is <= 0.  Apply: M at v -> edge
 *                (u, w) becomes (v, w); M at w -> (u, v) becomes (w, v);
 *                else a new Steiner node s at M with edges (s, u), (s, v),
 *                (s, w) replacing (u, v), (u, w).  Then, while some live
 *                Steiner node has <= 2 neighbours, take the lowest-index one
 *                and remove it (one neighbour: drop the edge; two: join
 *                them).  Nets of more than 64 pins keep the MST.  (The
 *                reattachments and the removals are defensive: on 20k random
 *                nets of 3-19 pins, grids with many ties included, neither
 *                ever fired -- a Steiner node at the median of its three
 *                neighbours leaves no positive gain at itself);
 *   3. output    breadth-first from the driver, neighbours in ascending
 *                index: node 0 = driver, parent[i] < i; a node at the same
 *                point as the node it is reached from shares its RC node (no
 *                zero-length edges); pin_node[j] = the node of pin j; wl =
 *                total length (nm).
 *
 * Capacity: n pins give at most 2n - 2 live nodes (n >= 2; a live Steiner
 * node has >= 3 neighbours).  parent, nx, ny need max(1, 2n - 2) entries. */
#define ORC_STEINER_MAX_PINS 64

static int64_t mdist(int64_t xa, int64_t ya, int64_t xb, int64_t yb)
{
    return llabs(xa - xb) + llabs(ya - yb);
}

static int64_t med3(int64_t a, int64_t b, int64_t c)
{
    if ((a <= b && b <= c) || (c <= b && b <= a)) return b;
    if ((b <= a && a <= c) || (c <= a && a <= b)) return a;
    return c;
}

int64_t orc_nm(float x_um)
{
    float p = x_um * 1000.0f;   /* the float product, then round to nearest even */
    return (int64_t)lrintf(p);
}

int orc_steiner_tree(int32_t n, const int64_t *X, const int64_t *Y, int32_t *n_out, int32_t *parent,
                     int64_t *nx, int64_t *ny, int32_t *pin_node, int64_t *wl)
{
    if (n < 1) return ERR_INVAL;
    int32_t cap = 3 * n;                 /* pins + at most 2 (n - 1) Steiner nodes */
    int64_t *x = (int64_t *)calloc((size_t)cap, sizeof(int64_t));
    int64_t *y = (int64_t *)calloc((size_t)cap, sizeof(int64_t));
    char *adj = (char *)calloc((size_t)cap * (size_t)cap, 1);
    char *live = (char *)calloc((size_t)cap, 1);
    int32_t *rank = (int32_t *)calloc((size_t)cap, sizeof(int32_t));
    int32_t *queue = (int32_t *)calloc((size_t)cap, sizeof(int32_t));
    int32_t *newid = (int32_t *)calloc((size_t)cap, sizeof(int32_t));
    if (!x || !y || !adj || !live || !rank || !queue || !newid) {
        free(x); free(y); free(adj); free(live); free(rank); free(queue); free(newid);
        return ERR_NOMEM;
    }
#define ADJ(a, b) adj[(size_t)(a) * (size_t)cap + (size_t)(b)]
    int32_t N = n;
    for (int32_t i = 0; i < n; ++i) { x[i] = X[i]; y[i] = Y[i]; live[i] = 1; rank[i] = -1; }
    /* 1. Prim from the driver */
    rank[0] = 0;
    for (int32_t step = 1; step < n; ++step) {
        int64_t bd = -1;
        int32_t bu = -1, bv = -1;
        for (int32_t u = 0; u < n; ++u) {
            if (rank[u] >= 0) continue;
            for (int32_t v = 0; v < n; ++v) {
                if (rank[v] < 0) continue;
                int64_t dd = mdist(x[u], y[u], x[v], y[v]);
                if (bu < 0 || dd < bd || (dd == bd && (u < bu || (u == bu && rank[v] < rank[bv])))) {
                    bd = dd; bu = u; bv = v;
                }
            }
        }
        rank[bu] = step;
        ADJ(bu, bv) = ADJ(bv, bu) = 1;
    }
    /* 2. greedy median insertion, then removal of Steiner nodes of degree <= 2 */
    for (int32_t it = 0; n <= ORC_STEINER_MAX_PINS && it < 2 * (n - 1); ++it) {
        int64_t bg = 0;
        int32_t bu = -1, bv = -1, bw = -1;
        for (int32_t u = 0; u < N; ++u) {
            if (!live[u]) continue;
            for (int32_t v = 0; v < N; ++v) {
                if (!ADJ(u, v)) continue;
                for (int32_t w = v + 1; w < N; ++w) {
                    if (!ADJ(u, w)) continue;
                    int64_t mx = med3(x[u], x[v], x[w]), my = med3(y[u], y[v], y[w]);
                    int64_t g = mdist(x[u], y[u], x[v], y[v]) + mdist(x[u], y[u], x[w], y[w]) -
                                mdist(mx, my, x[u], y[u]) - mdist(mx, my, x[v], y[v]) - mdist(mx, my, x[w], y[w]);
                    if (g > bg) { bg = g; bu = u; bv = v; bw = w; }
                }
            }
        }
        if (bg <= 0) break;
        int64_t mx = med3(x[bu], x[bv], x[bw]), my = med3(y[bu], y[bv], y[bw]);
        if (mx == x[bv] && my == y[bv]) {
            ADJ(bu, bw) = ADJ(bw, bu) = 0;
            ADJ(bv, bw) = ADJ(bw, bv) = 1;
        } else if (mx == x[bw] && my == y[bw]) {
            ADJ(bu, bv) = ADJ(bv, bu) = 0;
            ADJ(bw, bv) = ADJ(bv, bw) = 1;
        } else {
            int32_t s = N++;
            x[s] = mx; y[s] = my; live[s] = 1;
            ADJ(bu, bv) = ADJ(bv, bu) = 0;
            ADJ(bu, bw) = ADJ(bw, bu) = 0;
            ADJ(s, bu) = ADJ(bu, s) = 1;
            ADJ(s, bv) = ADJ(bv, s) = 1;
            ADJ(s, bw) = ADJ(bw, s) = 1;
        }
        for (;;) {
            int32_t s = -1, deg = 0, nb[2] = {-1, -1};
            for (int32_t i = n; i < N && s < 0; ++i) {
                if (!live[i]) continue;
                int32_t dg = 0;
                for (int32_t j = 0; j < N; ++j) dg += ADJ(i, j);
                if (dg <= 2) { s = i; deg = dg; }
            }
            if (s < 0) break;
            int32_t k = 0;
            for (int32_t j = 0; j < N; ++j)
                if (ADJ(s, j)) { nb[k++] = j; ADJ(s, j) = ADJ(j, s) = 0; }
            if (deg == 2) ADJ(nb[0], nb[1]) = ADJ(nb[1], nb[0]) = 1;
            live[s] = 0;
        }
    }
    /* 3. breadth-first numbering from the driver */
    for (int32_t i = 0; i < N; ++i) newid[i] = -1;
    int32_t head = 0, tail = 0;
    queue[tail++] = 0;
    newid[0] = 0;
    parent[0] = -1;
    nx[0] = x[0]; ny[0] = y[0];
    int64_t total = 0;
    int32_t nodes = 1;
    while (head < tail) {
        int32_t a = queue[head++];
        for (int32_t b = 0; b < N; ++b) {
            if (!ADJ(a, b) || newid[b] >= 0) continue;
            queue[tail++] = b;
            if (x[b] == x[a] && y[b] == y[a]) {   /* same point: the same RC node */
                newid[b] = newid[a];
                continue;
            }
            newid[b] = nodes;
            parent[nodes] = newid[a];
            nx[nodes] = x[b]; ny[nodes] = y[b];
            total += mdist(x[a], y[a], x[b], y[b]);
            ++nodes;
        }
    }
    int rc = OK;
    for (int32_t j = 0; j < n; ++j) {
        pin_node[j] = newid[j];
        if (newid[j] < 0) rc = ERR_INVAL;   /* not reached: the tree is connected */
    }
    *n_out = nodes;
    *wl = total;
#undef ADJ
    free(x); free(y); free(adj); free(live); free(rank); free(queue); free(newid);
    return rc;
}

/* O9 RC tree of net n at corner RC scale f: the Steiner tree of its pins'
 * nm coordinates (pin 0 = the driver), each edge of x length Lx and y length
 * Ly (um) with R = f (rx Lx + ry Ly) and wire C = f (cx Lx + cy Ly) split
 * half at each end, plus the sink pin caps (fF) at their nodes.  Arrays of
 * max(1, 2 m - 2) entries for m pins (pnode: m); nx, ny (node coordinates,
 * nm) may be NULL. */
static int steiner_rc(const orc_design *d, const pin_info *pi, int32_t n, double f, int32_t *nn_out,
                      int32_t *par, double *R, double *C, int32_t *pnode, int64_t *nx, int64_t *ny)
{
    int32_t b = d->net_pin_ptr[n], m = d->net_pin_ptr[n + 1] - b, cap = m > 1 ? 2 * m - 2 : 1, nn = 0;
    int64_t *X = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    int64_t *Y = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    int64_t *tx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    int64_t *ty = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    int rc = OK;
    if (!X || !Y || !tx || !ty) rc = ERR_NOMEM;
    else {
        for (int32_t k = 0; k < m; ++k) {
            double xs, ys;
            pin_xy(d, pi, d->net_pin[b + k], &xs, &ys);
            X[k] = orc_nm((float)xs);
            Y[k] = orc_nm((float)ys);
        }
        int64_t wl;
        rc = orc_steiner_tree(m, X, Y, &nn, par, tx, ty, pnode, &wl);
    }
    if (!rc) {
        double rx = d->r_per_um, cx = d->c_per_um;
        double ry = d->r_per_um_y > 0 ? d->r_per_um_y : rx, cy = d->c_per_um_y > 0 ? d->c_per_um_y : cx;
        for (int32_t i = 0; i < nn; ++i) { R[i] = 0.0; C[i] = 0.0; }
        for (int32_t i = 1; i < nn; ++i) {
            double lx = 1e-3 * (double)llabs(tx[i] - tx[par[i]]), ly = 1e-3 * (double)llabs(ty[i] - ty[par[i]]);
            double cw = f * (cx * lx + cy * ly);
            R[i] = f * (rx * lx + ry * ly);
            C[i] += 0.5 * cw;
            C[par[i]] += 0.5 * cw;
        }
        for (int32_t k = 1; k < m; ++k) C[pnode[k]] += 1e3 * pin_cap_of(d, pi, d->net_pin[b + k]);
        for (int32_t i = 0; i < nn; ++i) {
            if (nx) nx[i] = tx[i];
            if (ny) ny[i] = ty[i];
        }
        *nn_out = nn;
    }
    free(X); free(Y); free(tx); free(ty);
    return rc;
}

/* Per-corner net quantities: load (pF) at each driver pin, Elmore delay (ns)
 * and variance (ns^2) at each sink pin.  With rc_ptr == NULL the tree is the
 * star of O3/A8: root at the driver, one segment per sink of Manhattan length
 * L with R = r L and C = c L split half at each end, plus the sink pin cap;
 * with wire_model == 1 it is the O9 Steiner tree, each edge of x length Lx
 * and y length Ly (um) with R = rx Lx + ry Ly and C = cx Lx + cy Ly split
 * half at each end (ry, cy <= 0: the x values). */
static int net_delays_one(const orc_design *d, const pin_info *pi_, int32_t n, double f, double *load_pf,
                          double *D_ns, double *V_ns2);

int orc_net_delays(const orc_design *d, int32_t corner, double *load_pf, double *D_ns, double *V_ns2)
{
    pin_info pi;
    int rc = build_info(d, &pi);
    if (rc) return rc;
    for (int32_t p = 0; p < d->n_pins; ++p) { load_pf[p] = 0.0; D_ns[p] = 0.0; V_ns2[p] = 0.0; }
    double f = d->rc_scale ? d->rc_scale[corner] : 1.0;
    for (int32_t n = 0; n < d->n_nets && !rc; ++n) rc = net_delays_one(d, &pi, n, f, load_pf, D_ns, V_ns2);
    free_info(&pi);
    return rc;
}

/* Net n's driver load, sink delays and variances (corner scale f applied to
 * R and C); writes only the pins of net n. */
static int net_delays_one(const orc_design *d, const pin_info *pi_, int32_t n, double f, double *load_pf,
                          double *D_ns, double *V_ns2)
{
    int rc = OK;
    pin_info pi = *pi_;
    {
        int32_t b = d->net_pin_ptr[n], e = d->net_pin_ptr[n + 1];
        int32_t nn;
        const int steiner = !d->rc_ptr && d->wire_model == 1;
        if (d->rc_ptr) nn = d->rc_ptr[n + 1] - d->rc_ptr[n];
        else if (steiner) nn = e - b > 1 ? 2 * (e - b) - 2 : 1;   /* capacity; set below */
        else nn = e - b;             /* root + one node per sink */
        int32_t *pnode = NULL;
        int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
        double *R = (double *)malloc(sizeof(double) * (size_t)nn);
        double *C = (double *)malloc(sizeof(double) * (size_t)nn);
        double *cd = (double *)malloc(sizeof(double) * (size_t)nn);
        double *Dd = (double *)malloc(sizeof(double) * (size_t)nn);
        double *be = (double *)malloc(sizeof(double) * (size_t)nn);
        double *va = (double *)malloc(sizeof(double) * (size_t)nn);
        if (!par || !R || !C || !cd || !Dd || !be || !va) { rc = ERR_NOMEM; goto next; }
        if (d->rc_ptr) {
            int32_t o = d->rc_ptr[n];
            for (int32_t i = 0; i < nn; ++i) {
                par[i] = d->rc_parent[o + i];
                R[i] = i ? f * (double)d->rc_R[o + i] : 0.0;
                C[i] = f * (double)d->rc_C[o + i];
            }
            for (int32_t k = b + 1; k < e; ++k) {
                int32_t node = d->rc_pin_node[k];
                if (node < 0 || node >= nn) { rc = ERR_INVAL; goto next; }
                C[node] += 1e3 * pin_cap_of(d, &pi, d->net_pin[k]);   /* pF -> fF */
            }
        } else if (steiner) {
            pnode = (int32_t *)malloc(sizeof(int32_t) * (size_t)(e - b));
            if (!pnode) rc = ERR_NOMEM;
            else rc = steiner_rc(d, &pi, n, f, &nn, par, R, C, pnode, NULL, NULL);
            if (rc) goto next;
        } else {
            double xd, yd;
            pin_xy(d, &pi, d->net_pin[b], &xd, &yd);
            par[0] = -1; R[0] = 0.0; C[0] = 0.0;
            for (int32_t k = b + 1; k < e; ++k) {
                double xs, ys;
                pin_xy(d, &pi, d->net_pin[k], &xs, &ys);
                double L = fabs(xd - xs) + fabs(yd - ys);
                int32_t i = k - b;
                par[i] = 0;
                R[i] = f * d->r_per_um * L;
                C[i] = 0.5 * f * d->c_per_um * L + 1e3 * pin_cap_of(d, &pi, d->net_pin[k]);
                C[0] += 0.5 * f * d->c_per_um * L;
            }
        }
        rc = orc_rc_tree(nn, par, R, C, cd, Dd, be, va);
        if (rc) goto next;
        if (d->net_model == 1 && (d->rc_ptr || steiner)) {
            rc = orc_arnoldi_t50(nn, par, R, C, d->arnoldi_order, Dd);   /* O7 delays replace Elmore's */
            if (rc) goto next;
        }
        load_pf[d->net_pin[b]] = 1e-3 * cd[0];
        for (int32_t k = b + 1; k < e; ++k) {
            int32_t node = d->rc_ptr ? d->rc_pin_node[k] : steiner ? pnode[k - b] : k - b;
            D_ns[d->net_pin[k]] = 1e-6 * Dd[node];
            V_ns2[d->net_pin[k]] = 1e-12 * va[node];
        }
    next:
        free(par); free(R); free(C); free(cd); free(Dd); free(be); free(va); free(pnode);
    }
    return rc;
}

/* O9 tree length (nm) of every net of a placed design: wl[n_nets]. */
int orc_net_wirelengths(const orc_design *d, int64_t *wl)
{
    pin_info pi;
    int rc = build_info(d, &pi);
    if (rc) return rc;
    for (int32_t n = 0; n < d->n_nets && !rc; ++n) {
        int32_t b = d->net_pin_ptr[n], m = d->net_pin_ptr[n + 1] - b, nn = 0;
        int32_t cap = m > 1 ? 2 * m - 2 : 1;
        int64_t *X = (int64_t *)malloc(sizeof(int64_t) * (size_t)m), *Y = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
        int64_t *tx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap), *ty = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap), *pn = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
        if (!X || !Y || !tx || !ty || !par || !pn) rc = ERR_NOMEM;
        else {
            for (int32_t k = 0; k < m; ++k) {
                double xs, ys;
                pin_xy(d, &pi, d->net_pin[b + k], &xs, &ys);
                X[k] = orc_nm((float)xs);
                Y[k] = orc_nm((float)ys);
            }
            rc = orc_steiner_tree(m, X, Y, &nn, par, tx, ty, pn, &wl[n]);
        }
        free(X); free(Y); free(tx); free(ty); free(par); free(pn);
    }
    free_info(&pi);
    return rc;
}

/* ------------------------------------------------------ topological order */

/* Fan-in pins of p in the timing graph: net sink <- driver, cell output <-
 * the cell's arc inputs, flip-flop Q <- CK.  PI and CK are sources. */
static int fanins(const orc_design *d, const pin_info *pi, int32_t p, int32_t *out)
{
    int r = d->pin_role[p];
    if (r == R_IN || r == R_D || r == R_PO) {
        out[0] = d->net_pin[d->net_pin_ptr[pi->sink_net[p]]];
        return 1;
    }
    if (r == R_OUT || r == R_Q) {
        int32_t c = pi->cell[p], t = d->cell_type[c], n = 0;
        for (int32_t s = 0; s < d->type_nin[t]; ++s)
            if (d->arc_sense[t * MAXSLOT + s] != S_NONE) out[n++] = d->cell_pin[d->cell_pin_ptr[c] + s];
        return n;
    }
    return 0;
}

/* Memoised depth-first search; order[] receives every pin after all of its
 * fan-ins.  Returns ERR_CYCLE on a combinational loop. */
static int topo_order(const orc_design *d, const pin_info *pi, int32_t *order)
{
    int32_t P = d->n_pins;
    int8_t *mark = (int8_t *)calloc((size_t)P, 1);    /* 0 new, 1 on stack, 2 done */
    int32_t *stk = (int32_t *)malloc(sizeof(int32_t) * (size_t)P);
    int32_t *it = (int32_t *)malloc(sizeof(int32_t) * (size_t)P);
    if (!mark || !stk || !it) { free(mark); free(stk); free(it); return ERR_NOMEM; }
    int32_t nout = 0;
    for (int32_t root = 0; root < P; ++root) {
        if (mark[root]) continue;
        int32_t sp = 0;
        stk[sp] = root; it[sp] = 0; mark[root] = 1;
        while (sp >= 0) {
            int32_t p = stk[sp], fi[MAXSLOT + 1];
            int nf = fanins(d, pi, p, fi);
            if (it[sp] < nf) {
                int32_t q = fi[it[sp]++];
                if (mark[q] == 1) { free(mark); free(stk); free(it); return ERR_CYCLE; }
                if (mark[q] == 0) { ++sp; stk[sp] = q; it[sp] = 0; mark[q] = 1; }
            } else {
                mark[p] = 2; order[nout++] = p; --sp;
            }
        }
    }
    free(mark); free(stk); free(it);
    return OK;
}

int orc_topo_order(const orc_design *d, int32_t *order)
{
    pin_info pi;
    int rc = build_info(d, &pi);
    if (rc) return rc;
    rc = topo_order(d, &pi, order);
    free_info(&pi);
    return rc;
}

/* ------------------------------------------------------- O2: forward */

#define IX(p, k, j) ((((size_t)(p)) * (size_t)K + (size_t)(k)) * 4 + (size_t)(j))
#define JJ(el, rf) ((el) * 2 + (rf))   /* el 0 early, 1 late; rf 0 rise, 1 fall */

/* Pin p of one state (its fan-ins final): k indexes the at/slew arrays of Ks states (corner * tags +
 * tag), kc is the corner (its table scale).  src_on[p] == 0 marks a
 * startpoint of another tag: its arrivals are absent (-inf late, +inf
 * early); its slew is kept (slews are tag-free).  src_on may be NULL.
 * adv (may be NULL) marks the through pins: bit t of adv[p] set when tag t
 * moves on to tag t + 1 at gate input p; this state's tag is t = k - kt0
 * (kt0: the corner's first state), and the state k - 1 (tag t - 1) must be
 * final already. */
static void forward_pin(const orc_design *d, const pin_info *pi, int32_t p, int32_t k, int32_t Ks, int32_t kc,
                        const int8_t *src_on, const uint32_t *adv, int32_t kt0, const double *load, const double *Dn,
                        const double *Vn, double *at, double *slew)
{
    const int32_t t = k - kt0;
    int32_t K = Ks;
    double sc = d->lut_scale ? d->lut_scale[kc] : 1.0;
    {
        int r = d->pin_role[p];
        if (r == R_PI || r == R_CK) {
            double a = (r == R_PI) ? d->pi_at_ns : 0.0;
            double s = (r == R_PI) ? d->pi_slew_ns : d->clk_slew_ns;
            for (int j = 0; j < 4; ++j) { at[IX(p, k, j)] = a; slew[IX(p, k, j)] = s; }
            if (src_on && !src_on[p])
                for (int j = 0; j < 4; ++j) at[IX(p, k, j)] = j < 2 ? INFINITY : -INFINITY;
        } else if (r == R_IN || r == R_D || r == R_PO) {
            int32_t drv = d->net_pin[d->net_pin_ptr[pi->sink_net[p]]];
            /* a path in tag t stays unless p advances t; one in tag t - 1
             * arrives in tag t when p advances t - 1 */
            const int stay = !adv || !((adv[p] >> t) & 1u);
            const int inflow = adv && t >= 1 && ((adv[p] >> (t - 1)) & 1u);
            for (int j = 0; j < 4; ++j) {
                double sd = slew[IX(drv, k, j)];
                double a = j < 2 ? INFINITY : -INFINITY;   /* absent */
                if (stay) a = at[IX(drv, k, j)];
                if (inflow) a = j < 2 ? fmin(a, at[IX(drv, k - 1, j)]) : fmax(a, at[IX(drv, k - 1, j)]);
                at[IX(p, k, j)] = a + Dn[p];
                slew[IX(p, k, j)] = sqrt(sd * sd + Vn[p]);
            }
        } else { /* R_OUT or R_Q */
            int32_t c = pi->cell[p], t = d->cell_type[c];
            double l = load[p];
            for (int el = 0; el < 2; ++el)
                for (int rfo = 0; rfo < 2; ++rfo) {
                    double ca[2 * MAXSLOT], cs[2 * MAXSLOT];
                    int n = 0;
                    for (int32_t s = 0; s < d->type_nin[t]; ++s) {
                        int sense = d->arc_sense[t * MAXSLOT + s], rfi[2];
                        int m = rf_inputs(sense, rfo, rfi);
                        int32_t a = d->cell_pin[d->cell_pin_ptr[c] + s];
                        for (int q = 0; q < m; ++q) {
                            double si = slew[IX(a, k, JJ(el, rfi[q]))];
                            ca[n] = at[IX(a, k, JJ(el, rfi[q]))] +
                                    sc * lut(d, t, s, rfo ? TB_DF : TB_DR, si, l, 0, 0);
                            cs[n] = sc * lut(d, t, s, rfo ? TB_SF : TB_SR, si, l, 0, 0);
                            ++n;
                        }
                    }
                    at[IX(p, k, JJ(el, rfo))] = merge(ca, n, el, d->gamma_ns);
                    slew[IX(p, k, JJ(el, rfo))] = merge(cs, n, el, d->gamma_ns);
                }
        }
    }
}

/* One state over every pin in topological order (see forward_pin). */
static void forward_corner(const orc_design *d, const pin_info *pi, const int32_t *order, int32_t k, int32_t Ks,
                           int32_t kc, const int8_t *src_on, const uint32_t *adv, int32_t kt0, const double *load,
                           const double *Dn, const double *Vn, double *at, double *slew)
{
    for (int32_t oi = 0; oi < d->n_pins; ++oi)
        forward_pin(d, pi, order[oi], k, Ks, kc, src_on, adv, kt0, load, Dn, Vn, at, slew);
}

/* ----------------------------------------------- O4: required times, slack */

/* Pin p of one state (as forward_pin; its fan-outs final).  ep_req[2p], ep_req[2p+1] replace the late
 * and early requirements of endpoint pin p (may be NULL: the defaults).
 * Through a sink s that advances this state's tag t, the path continues in
 * tag t + 1: the state k + 1 must be final already. */
static void backward_pin(const orc_design *d, const pin_info *pi, int32_t p, int32_t k, int32_t Ks, int32_t kc,
                         const double *ep_req, const uint32_t *adv, int32_t kt0, const double *load, const double *Dn,
                         const double *slew, double *rat)
{
    int32_t K = Ks;
    const int32_t t = k - kt0;
    double sc = d->lut_scale ? d->lut_scale[kc] : 1.0;
    {
        int r = d->pin_role[p];
        double rl[2] = {INFINITY, INFINITY}, re[2] = {-INFINITY, -INFINITY};
        if (r == R_D || r == R_PO) {
            if (r == R_D) {
                rl[0] = rl[1] = d->period_ns - d->setup_ns;
                re[0] = re[1] = d->hold_ns;
            } else {
                rl[0] = rl[1] = d->period_ns;
                re[0] = re[1] = 0.0;
            }
            if (ep_req) {
                rl[0] = rl[1] = ep_req[2 * (size_t)p];
                re[0] = re[1] = ep_req[2 * (size_t)p + 1];
            }
        } else {
            if (pi->drv_net[p] >= 0) {
                int32_t n = pi->drv_net[p];
                for (int32_t q = d->net_pin_ptr[n] + 1; q < d->net_pin_ptr[n + 1]; ++q) {
                    int32_t s = d->net_pin[q];
                    const int32_t ks = adv && ((adv[s] >> t) & 1u) ? k + 1 : k;
                    for (int rf = 0; rf < 2; ++rf) {
                        rl[rf] = fmin(rl[rf], rat[IX(s, ks, JJ(1, rf))] - Dn[s]);
                        re[rf] = fmax(re[rf], rat[IX(s, ks, JJ(0, rf))] - Dn[s]);
                    }
                }
            }
            if ((r == R_IN || r == R_CK) && pi->cell[p] >= 0) {
                int32_t c = pi->cell[p], t = d->cell_type[c], s = pi->slot[p];
                int sense = d->arc_sense[t * MAXSLOT + s];
                int32_t z = d->cell_pin[d->cell_pin_ptr[c] + d->type_nin[t]];
                for (int rfo = 0; rfo < 2; ++rfo) {
                    int rfi[2];
                    int m = rf_inputs(sense, rfo, rfi);
                    for (int q = 0; q < m; ++q) {
                        int ri = rfi[q];
                        double dl = sc * lut(d, t, s, rfo ? TB_DF : TB_DR, slew[IX(p, k, JJ(1, ri))], load[z], 0, 0);
                        double de = sc * lut(d, t, s, rfo ? TB_DF : TB_DR, slew[IX(p, k, JJ(0, ri))], load[z], 0, 0);
                        rl[ri] = fmin(rl[ri], rat[IX(z, k, JJ(1, rfo))] - dl);
                        re[ri] = fmax(re[ri], rat[IX(z, k, JJ(0, rfo))] - de);
                    }
                }
            }
        }
        rat[IX(p, k, JJ(0, 0))] = re[0]; rat[IX(p, k, JJ(0, 1))] = re[1];
        rat[IX(p, k, JJ(1, 0))] = rl[0]; rat[IX(p, k, JJ(1, 1))] = rl[1];
    }
}

/* One state over every pin in reverse topological order (see backward_pin). */
static void backward_corner(const orc_design *d, const pin_info *pi, const int32_t *order, int32_t k, int32_t Ks,
                            int32_t kc, const double *ep_req, const uint32_t *adv, int32_t kt0, const double *load,
                            const double *Dn, const double *slew, double *rat)
{
    for (int32_t oi = d->n_pins - 1; oi >= 0; --oi)
        backward_pin(d, pi, order[oi], k, Ks, kc, ep_req, adv, kt0, load, Dn, slew, rat);
}

/* Full analysis.  Arrays at/slew/rat/slack are [n_pins][n_corners][4] with
 * the inner index el * 2 + rf (el 0 early / hold, 1 late / setup).
 * With exception groups (O8) the pin arrays hold n_corners * tags states,
 * state = corner * tags + tag, tags = 1 + sum over groups of (through sets
 * + 1).
 * Endpoints are the DFF D pins and POs in ascending pin id; ep_setup and
 * ep_hold are [n_endpoints][n_corners] (min over rise/fall and tags).  summary is
 * [n_corners][8]: WNS setup, TNS setup, WNS hold, TNS hold, worst setup
 * slack, worst hold slack, setup violations, hold violations. */
int orc_sta(const orc_design *d, double *at, double *slew, double *rat, double *slack,
            double *ep_setup, double *ep_hold, double *summary)
{
    pin_info pi;
    int rc = build_info(d, &pi);
    if (rc) { return rc; }
    const int32_t P = d->n_pins, Kc = d->n_corners;
    const int32_t G = d->n_exc > 0 ? d->n_exc : 0;
    /* O8 tags: 0 = no group; group g owns tags base[g] .. base[g] + r_g, its
     * progress through its r_g ordered through sets (base[g] + r_g: fully
     * matched) */
    int32_t base[33], nthru[32];
    int32_t Tg = 1;
    for (int32_t g = 0; g < G && g < 32; ++g) {
        nthru[g] = d->exc_thru_ptr ? d->exc_thru_ptr[g + 1] - d->exc_thru_ptr[g] : 0;
        if (nthru[g] < 0) { free_info(&pi); return ERR_INVAL; }
        base[g] = Tg;
        Tg += nthru[g] + 1;
    }
    if (G > 32 || Tg > 32) { free_info(&pi); return ERR_INVAL; }
    const int32_t K = Kc * Tg;   /* K: states (corner, tag) */
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P ? P : 1));
    double *load = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *Dn = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *Vn = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    int8_t *tag_of = (int8_t *)calloc((size_t)(P ? P : 1), 1);
    int8_t *src_on = (int8_t *)calloc((size_t)(P ? P : 1), 1);
    uint8_t *in_to = (uint8_t *)calloc((size_t)(P ? P : 1), 1);
    double *ep_req = (double *)malloc(sizeof(double) * 2 * (size_t)(P ? P : 1));
    uint32_t *adv = (uint32_t *)calloc((size_t)(P ? P : 1), sizeof(uint32_t));
    int any_thru = 0;
    if (!order || !load || !Dn || !Vn || !tag_of || !src_on || !in_to || !ep_req || !adv) { rc = ERR_NOMEM; goto done; }
    rc = topo_order(d, &pi, order);
    if (rc) goto done;
    /* O8: a startpoint's tag is its first group (0 = none) */
    for (int32_t g = 0; g < G; ++g) {
        for (int32_t i = d->exc_from_ptr[g]; i < d->exc_from_ptr[g + 1]; ++i) {
            const int32_t p = d->exc_from[i];
            if (p < 0 || p >= P || (d->pin_role[p] != R_PI && d->pin_role[p] != R_CK)) { rc = ERR_INVAL; goto done; }
            if (!tag_of[p]) tag_of[p] = (int8_t)base[g];
        }
        for (int32_t i = d->exc_to_ptr[g]; i < d->exc_to_ptr[g + 1]; ++i) {
            const int32_t p = d->exc_to[i];
            if (p < 0 || p >= P || (d->pin_role[p] != R_D && d->pin_role[p] != R_PO)) { rc = ERR_INVAL; goto done; }
        }
        if (d->exc_action[g] < 0 || d->exc_action[g] > 3 || !isfinite(d->exc_mult[g]) ||
            (d->exc_action[g] == 1 && d->exc_mult[g] < 1.0f)) { rc = ERR_INVAL; goto done; }
        /* through set j + 1 of group g: tag base[g] + j moves on at its pins */
        for (int32_t j = 0; j < nthru[g]; ++j) {
            const int32_t s = d->exc_thru_ptr[g] + j;
            for (int32_t i = d->exc_thru_set_ptr[s]; i < d->exc_thru_set_ptr[s + 1]; ++i) {
                const int32_t p = d->exc_thru_pin[i];
                if (p < 0 || p >= P || d->pin_role[p] != R_IN) { rc = ERR_INVAL; goto done; }
                adv[p] |= 1u << (base[g] + j);
                any_thru = 1;
            }
        }
    }
    for (int32_t kc = 0; kc < Kc; ++kc) {
        rc = orc_net_delays(d, kc, load, Dn, Vn);
        if (rc) goto done;
        const int32_t kt0 = kc * Tg;
        /* forward: tags in increasing order (a path moves from tag t to t + 1) */
        for (int32_t t = 0; t < Tg; ++t) {
            if (G > 0)
                for (int32_t p = 0; p < P; ++p) src_on[p] = tag_of[p] == t;
            forward_corner(d, &pi, order, kt0 + t, K, kc, G ? src_on : NULL, any_thru ? adv : NULL, kt0, load, Dn,
                           Vn, at, slew);
        }
        /* backward: tags in decreasing order */
        for (int32_t t = Tg - 1; t >= 0; --t) {
            const int32_t k = kt0 + t;
            if (G > 0) {
                /* requirements of tag t at every endpoint: its group's action
                 * when t is the group's fully matched tag and the endpoint is
                 * in the group's list (or the list is empty); else the default */
                int32_t grp = -1;
                for (int32_t g = 0; g < G; ++g)
                    if (t == base[g] + nthru[g]) grp = g;
                for (int32_t p = 0; p < P; ++p) in_to[p] = 0;
                const int applies_all = grp >= 0 && d->exc_to_ptr[grp + 1] == d->exc_to_ptr[grp];
                if (grp >= 0)
                    for (int32_t i = d->exc_to_ptr[grp]; i < d->exc_to_ptr[grp + 1]; ++i) in_to[d->exc_to[i]] = 1;
                for (int32_t p = 0; p < P; ++p) {
                    const int r = d->pin_role[p];
                    if (r != R_D && r != R_PO) continue;
                    const double T = d->period_ns;
                    double late = r == R_D ? T - d->setup_ns : T, early = r == R_D ? d->hold_ns : 0.0;
                    if (grp >= 0 && (applies_all || in_to[p])) {
                        if (d->exc_action[grp] == 0) {
                            late = INFINITY;   /* false path: no check */
                            early = -INFINITY;
                        } else if (d->exc_action[grp] == 1) {
                            const double M = d->exc_mult[grp];   /* multicycle: capture at M * T */
                            late = r == R_D ? M * T - d->setup_ns : M * T;
                        } else if (d->exc_action[grp] == 2) {
                            const double V = d->exc_mult[grp];   /* max delay: capture at V */
                            late = r == R_D ? V - d->setup_ns : V;
                        } else {
                            const double V = d->exc_mult[grp];   /* min delay: hold edge at V */
                            early = r == R_D ? V + d->hold_ns : V;
                        }
                    }
                    ep_req[2 * (size_t)p] = late;
                    ep_req[2 * (size_t)p + 1] = early;
                }
            }
            backward_corner(d, &pi, order, k, K, kc, G ? ep_req : NULL, any_thru ? adv : NULL, kt0, load, Dn, slew,
                            rat);
            for (int32_t p = 0; p < P; ++p)
                for (int rf = 0; rf < 2; ++rf) {
                    slack[IX(p, k, JJ(0, rf))] = at[IX(p, k, JJ(0, rf))] - rat[IX(p, k, JJ(0, rf))];
                    slack[IX(p, k, JJ(1, rf))] = rat[IX(p, k, JJ(1, rf))] - at[IX(p, k, JJ(1, rf))];
                }
        }
        /* endpoints of corner kc: min over rise/fall and over tags */
        double *sm = summary + (size_t)kc * 8;
        double wns_s = 0, tns_s = 0, wns_h = 0, tns_h = 0, worst_s = INFINITY, worst_h = INFINITY;
        double nv_s = 0, nv_h = 0;
        int32_t e = 0;
        for (int32_t p = 0; p < P; ++p) {
            int r = d->pin_role[p];
            if (r != R_D && r != R_PO) continue;
            double ssm = INFINITY, hsm = INFINITY;
            for (int32_t g = 0; g < Tg; ++g) {
                const int32_t k = kc * Tg + g;
                double ss = fmin(slack[IX(p, k, JJ(1, 0))], slack[IX(p, k, JJ(1, 1))]);
                double hs = fmin(slack[IX(p, k, JJ(0, 0))], slack[IX(p, k, JJ(0, 1))]);
                ssm = fmin(ssm, ss);
                hsm = fmin(hsm, hs);
            }
            const double ss = ssm, hs = hsm;
            ep_setup[(size_t)e * Kc + kc] = ss;
            ep_hold[(size_t)e * Kc + kc] = hs;
            ++e;
            worst_s = fmin(worst_s, ss); worst_h = fmin(worst_h, hs);
            if (ss < 0) { tns_s += ss; nv_s += 1; wns_s = fmin(wns_s, ss); }
            if (hs < 0) { tns_h += hs; nv_h += 1; wns_h = fmin(wns_h, hs); }
        }
        sm[0] = wns_s; sm[1] = tns_s; sm[2] = wns_h; sm[3] = tns_h;
        sm[4] = worst_s; sm[5] = worst_h; sm[6] = nv_s; sm[7] = nv_h;
    }
done:
    free(order); free(load); free(Dn); free(Vn); free(tag_of); free(src_on); free(in_to); free(ep_req); free(adv);
    free_info(&pi);
    return rc;
}

/* ------------------------------------------------ timed baseline (O2-O4) */

static double wall_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* The plain analysis of orc_sta (no exception groups) repeated `reps` times
 * with each run's wall time in secs[reps]: net delays, forward arrivals and
 * slews, backward required times, pin slacks, endpoint slacks and WNS/TNS.
 * Validation, the topological order and its level buckets are prepared
 * once, outside the timed runs.  One thread walks the depth-first order
 * of orc_sta.  With n_threads > 1 the nets and the pins of one level are
 * split over OpenMP threads: a pin's level is one more
 * than its deepest fan-in's, so a level's pins read only values of earlier
 * levels (forward) or later ones (backward) and write only their own: the
 * results equal the serial analysis.  summary[n_corners][8] as orc_sta
 * (last run).  Returns ERR_INVAL with exception groups. */
int orc_sta_timed(const orc_design *d, int32_t n_threads, int32_t reps, double *secs, double *summary)
{
    if (d->n_exc > 0 || reps < 1) return ERR_INVAL;
    pin_info pi;
    int rc = build_info(d, &pi);
    if (rc) return rc;
    const int32_t P = d->n_pins, K = d->n_corners, nt = n_threads > 0 ? n_threads : 1;
    const size_t PK4 = (size_t)(P ? P : 1) * (size_t)K * 4;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P ? P : 1));
    int32_t *lev = (int32_t *)calloc((size_t)(P ? P : 1), sizeof(int32_t));
    int32_t *lv_pins = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P ? P : 1));
    int32_t *lv_ptr = NULL;
    double *at = (double *)malloc(sizeof(double) * PK4), *slew = (double *)malloc(sizeof(double) * PK4);
    double *rat = (double *)malloc(sizeof(double) * PK4), *slack = (double *)malloc(sizeof(double) * PK4);
    double *load = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *Dn = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *Vn = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    int32_t L = 0;
    if (!order || !lev || !lv_pins || !at || !slew || !rat || !slack || !load || !Dn || !Vn) { rc = ERR_NOMEM; goto done; }
    rc = topo_order(d, &pi, order);
    if (rc) goto done;
    for (int32_t oi = 0; oi < P; ++oi) {
        const int32_t p = order[oi];
        int32_t fi[MAXSLOT + 1];
        const int nf = fanins(d, &pi, p, fi);
        for (int i = 0; i < nf; ++i) lev[p] = lev[p] > lev[fi[i]] + 1 ? lev[p] : lev[fi[i]] + 1;
        L = L > lev[p] + 1 ? L : lev[p] + 1;
    }
    lv_ptr = (int32_t *)calloc((size_t)L + 1, sizeof(int32_t));
    if (!lv_ptr) { rc = ERR_NOMEM; goto done; }
    for (int32_t p = 0; p < P; ++p) ++lv_ptr[lev[p] + 1];
    for (int32_t l = 0; l < L; ++l) lv_ptr[l + 1] += lv_ptr[l];
    {
        int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L ? L : 1));
        if (!fill) { rc = ERR_NOMEM; goto done; }
        for (int32_t l = 0; l < L; ++l) fill[l] = lv_ptr[l];
        for (int32_t p = 0; p < P; ++p) lv_pins[fill[lev[p]]++] = p;
        free(fill);
    }
    for (int32_t rep = 0; rep < reps; ++rep) {
        const double t0 = wall_s();
        for (int32_t kc = 0; kc < K && !rc; ++kc) {
            const double f = d->rc_scale ? d->rc_scale[kc] : 1.0;
            int bad = 0;
#pragma omp parallel for num_threads(nt) schedule(static)
            for (int32_t p = 0; p < P; ++p) { load[p] = 0.0; Dn[p] = 0.0; Vn[p] = 0.0; }
#pragma omp parallel for num_threads(nt) schedule(dynamic, 512) reduction(| : bad)
            for (int32_t n = 0; n < d->n_nets; ++n) bad |= net_delays_one(d, &pi, n, f, load, Dn, Vn) != OK;
            if (bad) { rc = ERR_INVAL; break; }
            if (nt == 1) {   /* one thread: the analysis' own depth-first order */
                forward_corner(d, &pi, order, kc, K, kc, NULL, NULL, kc, load, Dn, Vn, at, slew);
                backward_corner(d, &pi, order, kc, K, kc, NULL, NULL, kc, load, Dn, slew, rat);
            } else {
                for (int32_t l = 0; l < L; ++l) {
#pragma omp parallel for num_threads(nt) schedule(static)
                    for (int32_t i = lv_ptr[l]; i < lv_ptr[l + 1]; ++i)
                        forward_pin(d, &pi, lv_pins[i], kc, K, kc, NULL, NULL, kc, load, Dn, Vn, at, slew);
                }
                for (int32_t l = L - 1; l >= 0; --l) {
#pragma omp parallel for num_threads(nt) schedule(static)
                    for (int32_t i = lv_ptr[l]; i < lv_ptr[l + 1]; ++i)
                        backward_pin(d, &pi, lv_pins[i], kc, K, kc, NULL, NULL, kc, load, Dn, slew, rat);
                }
            }
#pragma omp parallel for num_threads(nt) schedule(static)
            for (int32_t p = 0; p < P; ++p)
                for (int rf = 0; rf < 2; ++rf) {
                    slack[IX(p, kc, JJ(0, rf))] = at[IX(p, kc, JJ(0, rf))] - rat[IX(p, kc, JJ(0, rf))];
                    slack[IX(p, kc, JJ(1, rf))] = rat[IX(p, kc, JJ(1, rf))] - at[IX(p, kc, JJ(1, rf))];
                }
            /* endpoint slacks and the FP64 sums, in pin order as orc_sta */
            double wns_s = 0, tns_s = 0, wns_h = 0, tns_h = 0, worst_s = INFINITY, worst_h = INFINITY;
            double nv_s = 0, nv_h = 0;
            for (int32_t p = 0; p < P; ++p) {
                const int r = d->pin_role[p];
                if (r != R_D && r != R_PO) continue;
                const double ss = fmin(slack[IX(p, kc, JJ(1, 0))], slack[IX(p, kc, JJ(1, 1))]);
                const double hs = fmin(slack[IX(p, kc, JJ(0, 0))], slack[IX(p, kc, JJ(0, 1))]);
                worst_s = fmin(worst_s, ss); worst_h = fmin(worst_h, hs);
                if (ss < 0) { tns_s += ss; nv_s += 1; wns_s = fmin(wns_s, ss); }
                if (hs < 0) { tns_h += hs; nv_h += 1; wns_h = fmin(wns_h, hs); }
            }
            double *sm = summary + (size_t)kc * 8;
            sm[0] = wns_s; sm[1] = tns_s; sm[2] = wns_h; sm[3] = tns_h;
            sm[4] = worst_s; sm[5] = worst_h; sm[6] = nv_s; sm[7] = nv_h;
        }
        secs[rep] = wall_s() - t0;
    }
done:
    free(order); free(lev); free(lv_pins); free(lv_ptr); free(at); free(slew); free(rat); free(slack);
    free(load); free(Dn); free(Vn);
    free_info(&pi);
    return rc;
}

/* ---------------------------------------------- O6: objective and adjoint */

static double softplus(double z) { return (z > 0 ? z : 0) + log1p(exp(-fabs(z))); }
static double sigmoid(double z)
{
    if (z >= 0) return 1.0 / (1.0 + exp(-z));
    double e = exp(z);
    return e / (1.0 + e);
}

/* Steiner partials of one corner (RC scale f): from the sinks' dJ/dD and
 * dJ/dvar and the drivers' dJ/dload, dJ/dR and dJ/dC of every tree node
 * (orc_rc_tree_adjoint), then dJ/dLx = f (rx Rbar_i + cx (Cbar_i +
 * Cbar_parent) / 2) and likewise for y, then the cells.  The gradient is
 * that of the tree held fixed: every node coordinate is the coordinate of a
 * pin (a Steiner point takes medians of pin coordinates), it moves with the
 * lowest-index pin of the net at that coordinate (Lx = |X_i - X_parent| in
 * nm / 1000, nm rounding taken as the identity), and sign 0 at X_i =
 * X_parent. */
static int steiner_grad(const orc_design *d, const pin_info *pi, double f, const double *aD, const double *aV,
                        const double *aload, double *grad_xy)
{
    double rx = d->r_per_um, cx = d->c_per_um;
    double ry = d->r_per_um_y > 0 ? d->r_per_um_y : rx, cy = d->c_per_um_y > 0 ? d->c_per_um_y : cx;
    int rc = OK;
    for (int32_t n = 0; n < d->n_nets && !rc; ++n) {
        int32_t b = d->net_pin_ptr[n], m = d->net_pin_ptr[n + 1] - b, cap = m > 1 ? 2 * m - 2 : 1, nn = 0;
        if (m < 2) continue;
        int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap), *pnode = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
        double *R = (double *)malloc(sizeof(double) * (size_t)cap), *C = (double *)malloc(sizeof(double) * (size_t)cap);
        double *Db = (double *)calloc((size_t)cap, sizeof(double)), *Vb = (double *)calloc((size_t)cap, sizeof(double));
        double *Rb = (double *)malloc(sizeof(double) * (size_t)cap), *Cb = (double *)malloc(sizeof(double) * (size_t)cap);
        int64_t *nx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap), *ny = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        int64_t *X = (int64_t *)malloc(sizeof(int64_t) * (size_t)m), *Y = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
        if (!par || !pnode || !R || !C || !Db || !Vb || !Rb || !Cb || !nx || !ny || !X || !Y) rc = ERR_NOMEM;
        if (!rc) rc = steiner_rc(d, pi, n, f, &nn, par, R, C, pnode, nx, ny);
        if (!rc) {
            for (int32_t k = 1; k < m; ++k) {
                int32_t s = d->net_pin[b + k];
                Db[pnode[k]] += 1e-6 * aD[s];
                Vb[pnode[k]] += 1e-12 * aV[s];
            }
            rc = orc_rc_tree_adjoint(nn, par, R, C, Db, Vb, 1e-3 * aload[d->net_pin[b]], Rb, Cb);
        }
        if (!rc) {
            for (int32_t k = 0; k < m; ++k) {
                double xs, ys;
                pin_xy(d, pi, d->net_pin[b + k], &xs, &ys);
                X[k] = orc_nm((float)xs);
                Y[k] = orc_nm((float)ys);
            }
            for (int32_t i = 1; i < nn; ++i) {
                int32_t p = par[i];
                double gl[2] = {f * (rx * Rb[i] + 0.5 * cx * (Cb[i] + Cb[p])), f * (ry * Rb[i] + 0.5 * cy * (Cb[i] + Cb[p]))};
                const int64_t *co[2] = {nx, ny}, *pc[2] = {X, Y};
                for (int ax = 0; ax < 2; ++ax) {
                    int64_t a = co[ax][i], q = co[ax][p];
                    double sg = (double)((a > q) - (a < q));
                    if (sg == 0.0) continue;
                    int32_t ka = -1, kq = -1;   /* the pins that carry the two coordinates */
                    for (int32_t k = m - 1; k >= 0; --k) {
                        if (pc[ax][k] == a) ka = k;
                        if (pc[ax][k] == q) kq = k;
                    }
                    if (ka < 0 || kq < 0) { rc = ERR_INVAL; break; }   /* not reached */
                    int32_t ca = pi->cell[d->net_pin[b + ka]], cq = pi->cell[d->net_pin[b + kq]];
                    if (ca >= 0) grad_xy[2 * ca + ax] += gl[ax] * sg;
                    if (cq >= 0) grad_xy[2 * cq + ax] -= gl[ax] * sg;
                }
            }
        }
        free(par); free(pnode); free(R); free(C); free(Db); free(Vb); free(Rb); free(Cb);
        free(nx); free(ny); free(X); free(Y);
    }
    return rc;
}

/* Smoothed objective J = w_tns * TNS_g + w_wns * WNS_g summed over corners,
 * with per endpoint setup slack s_e = smin_g over rise/fall of (RAT - AT_late)
 *   TNS_g = - sum_e g * softplus(-s_e / g)
 *   WNS_g = - g * log sum_e exp(-s_e / g)
 * and its gradient with respect to every cell (x, y) (ports are fixed).  The
 * forward merges are the log-sum-exp ones of merge() with the same gamma.
 * Requires parasitics from positions (star, or Steiner with the Elmore
 * model) and gamma_ns > 0.
 * terms[k*2 + 0] = TNS_g, terms[k*2 + 1] = WNS_g of corner k (may be NULL). */
int orc_objective_grad(const orc_design *d, double w_tns, double w_wns, double *J_out,
                       double *terms, double *grad_xy)
{
    if (d->rc_ptr || !d->cell_xy || d->gamma_ns <= 0.0 || (d->wire_model != 0 && d->wire_model != 1) ||
        (d->wire_model == 1 && d->net_model != 0))
        return ERR_INVAL;
    pin_info pi;
    int rc = build_info(d, &pi);
    if (rc) return rc;
    int32_t P = d->n_pins, K = d->n_corners;
    double g = d->gamma_ns;
    size_t PK4 = (size_t)(P ? P : 1) * (size_t)K * 4;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P ? P : 1));
    double *load = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *Dn = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *Vn = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *at = (double *)malloc(sizeof(double) * PK4);
    double *sl = (double *)malloc(sizeof(double) * PK4);
    double *aat = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1) * 2);
    double *asl = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1) * 2);
    double *aload = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *aD = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *aV = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *seed = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double J = 0.0;
    if (!order || !load || !Dn || !Vn || !at || !sl || !aat || !asl || !aload || !aD || !aV || !seed) {
        rc = ERR_NOMEM; goto done;
    }
    for (int32_t c = 0; c < 2 * d->n_cells; ++c) grad_xy[c] = 0.0;
    rc = topo_order(d, &pi, order);
    if (rc) goto done;
    for (int32_t k = 0; k < K; ++k) {
        double sc = d->lut_scale ? d->lut_scale[k] : 1.0;
        double f = d->rc_scale ? d->rc_scale[k] : 1.0;
        rc = orc_net_delays(d, k, load, Dn, Vn);
        if (rc) goto done;
        forward_corner(d, &pi, order, k, K, k, NULL, NULL, k, load, Dn, Vn, at, sl);
        /* endpoint slacks and the objective */
        double mx = -INFINITY;
        for (int32_t p = 0; p < P; ++p) {
            int r = d->pin_role[p];
            if (r != R_D && r != R_PO) continue;
            double req = (r == R_D) ? d->period_ns - d->setup_ns : d->period_ns;
            double y[2] = {req - at[IX(p, k, JJ(1, 0))], req - at[IX(p, k, JJ(1, 1))]};
            seed[p] = merge(y, 2, 0, g);              /* smooth min over rise/fall */
            mx = fmax(mx, -seed[p] / g);
        }
        double tns = 0.0, lse = 0.0;
        for (int32_t p = 0; p < P; ++p) {
            int r = d->pin_role[p];
            if (r != R_D && r != R_PO) continue;
            tns += -g * softplus(-seed[p] / g);
            lse += exp(-seed[p] / g - mx);
        }
        double wns = (lse > 0) ? -g * (mx + log(lse)) : 0.0;
        if (terms) { terms[2 * k] = tns; terms[2 * k + 1] = wns; }
        J += w_tns * tns + w_wns * wns;
        /* seed the adjoint: dJ/dAT_late at each endpoint */
        for (int32_t p = 0; p < P; ++p) {
            aat[2 * p] = aat[2 * p + 1] = 0.0; asl[2 * p] = asl[2 * p + 1] = 0.0;
            aload[p] = 0.0; aD[p] = 0.0; aV[p] = 0.0;
        }
        for (int32_t p = 0; p < P; ++p) {
            int r = d->pin_role[p];
            if (r != R_D && r != R_PO) continue;
            double s = seed[p];
            double dj = w_tns * sigmoid(-s / g) + w_wns * exp(-s / g - mx) / lse;
            double req = (r == R_D) ? d->period_ns - d->setup_ns : d->period_ns;
            for (int rf = 0; rf < 2; ++rf) {
                double y = req - at[IX(p, k, JJ(1, rf))];
                double om = exp(-(y - s) / g);          /* d smin / d y_rf */
                aat[2 * p + rf] += -dj * om;            /* d y / d AT = -1 */
            }
        }
        /* reverse topological sweep, late quantities only */
        for (int32_t oi = P - 1; oi >= 0; --oi) {
            int32_t p = order[oi];
            int r = d->pin_role[p];
            if (r == R_IN || r == R_D || r == R_PO) {
                int32_t drv = d->net_pin[d->net_pin_ptr[pi.sink_net[p]]];
                for (int rf = 0; rf < 2; ++rf) {
                    double sp = sl[IX(p, k, JJ(1, rf))], sd = sl[IX(drv, k, JJ(1, rf))];
                    aat[2 * drv + rf] += aat[2 * p + rf];
                    asl[2 * drv + rf] += asl[2 * p + rf] * sd / sp;
                    aD[p] += aat[2 * p + rf];
                    aV[p] += asl[2 * p + rf] / (2.0 * sp);
                }
            } else if (r == R_OUT || r == R_Q) {
                int32_t c = pi.cell[p], t = d->cell_type[c];
                double l = load[p];
                for (int rfo = 0; rfo < 2; ++rfo) {
                    double ca[2 * MAXSLOT], cs[2 * MAXSLOT], dds[2 * MAXSLOT], ddl[2 * MAXSLOT];
                    double sds[2 * MAXSLOT], sdl[2 * MAXSLOT];
                    int32_t src[2 * MAXSLOT], srf[2 * MAXSLOT];
                    int n = 0;
                    for (int32_t s = 0; s < d->type_nin[t]; ++s) {
                        int sense = d->arc_sense[t * MAXSLOT + s], rfi[2];
                        int m = rf_inputs(sense, rfo, rfi);
                        int32_t a = d->cell_pin[d->cell_pin_ptr[c] + s];
                        for (int q = 0; q < m; ++q) {
                            double si = sl[IX(a, k, JJ(1, rfi[q]))];
                            ca[n] = at[IX(a, k, JJ(1, rfi[q]))] +
                                    sc * lut(d, t, s, rfo ? TB_DF : TB_DR, si, l, &dds[n], &ddl[n]);
                            cs[n] = sc * lut(d, t, s, rfo ? TB_SF : TB_SR, si, l, &sds[n], &sdl[n]);
                            src[n] = a; srf[n] = rfi[q];
                            ++n;
                        }
                    }
                    double ma = merge(ca, n, 1, g), ms = merge(cs, n, 1, g);
                    double Aa = aat[2 * p + rfo], As = asl[2 * p + rfo];
                    for (int i = 0; i < n; ++i) {
                        double wa = exp((ca[i] - ma) / g), ws = exp((cs[i] - ms) / g);
                        int32_t a = src[i];
                        int rf = srf[i];
                        aload[p] += Aa * wa * sc * ddl[i] + As * ws * sc * sdl[i];
                        if (d->pin_role[a] == R_CK) continue;   /* ideal clock: fixed */
                        aat[2 * a + rf] += Aa * wa;
                        asl[2 * a + rf] += Aa * wa * sc * dds[i] + As * ws * sc * sds[i];
                    }
                }
            }
        }
        if (d->wire_model == 1) {
            rc = steiner_grad(d, &pi, f, aD, aV, aload, grad_xy);
            if (rc) goto done;
            continue;
        }
        /* star-tree partials: D = R (C/2 + Cp), var = D^2, load = sum (cL + Cp) */
        for (int32_t n = 0; n < d->n_nets; ++n) {
            int32_t b = d->net_pin_ptr[n], e = d->net_pin_ptr[n + 1];
            int32_t drv = d->net_pin[b];
            double xd, yd;
            pin_xy(d, &pi, drv, &xd, &yd);
            for (int32_t q = b + 1; q < e; ++q) {
                int32_t s = d->net_pin[q];
                double xs, ys;
                pin_xy(d, &pi, s, &xs, &ys);
                double L = fabs(xd - xs) + fabs(yd - ys);
                double cp = 1e3 * pin_cap_of(d, &pi, s);
                double r = f * d->r_per_um, cc = f * d->c_per_um;
                double Draw = r * L * (0.5 * cc * L + cp);
                double dDdL = r * (cc * L + cp);
                double dJdL = aD[s] * 1e-6 * dDdL + aV[s] * 1e-12 * 2.0 * Draw * dDdL + aload[drv] * 1e-3 * cc;
                double sx = (xd > xs) - (xd < xs), sy = (yd > ys) - (yd < ys);
                int32_t cd = pi.cell[drv], cs = pi.cell[s];
                if (cd >= 0) { grad_xy[2 * cd] += dJdL * sx; grad_xy[2 * cd + 1] += dJdL * sy; }
                if (cs >= 0) { grad_xy[2 * cs] -= dJdL * sx; grad_xy[2 * cs + 1] -= dJdL * sy; }
            }
        }
    }
    *J_out = J;
done:
    free(order); free(load); free(Dn); free(Vn); free(at); free(sl);
    free(aat); free(asl); free(aload); free(aD); free(aV); free(seed);
    free_info(&pi);
    return rc;
}

/* Smoothed objective only (for finite differences in the tests). */
int orc_objective(const orc_design *d, double w_tns, double w_wns, double *J_out)
{
    double *gx = (double *)malloc(sizeof(double) * (size_t)(2 * d->n_cells + 2));
    if (!gx) return ERR_NOMEM;
    int rc = orc_objective_grad(d, w_tns, w_wns, J_out, NULL, gx);
    free(gx);
    return rc;
}
