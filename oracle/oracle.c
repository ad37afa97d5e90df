/*
 * oracle.c -- plain FP64 CPU reference for short-range pair-force molecular dynamics.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load this library.  It shares no code, header, table or helper with the CUDA
 * library; it is written from the definitions in Rapaport, "GPU molecular dynamics: Algorithms
 * and performance" (arXiv 2003.14061), and from the textbook definitions that paper relies on.
 *
 * What each function follows:
 *   orc_pair            -- the Lennard-Jones / WCA pair potential and force (Sec. 3.1 gives the
 *                          cutoffs r_c = 2^{1/6} for the soft-sphere fluid and 2.5 for LJ).
 *   orc_forces_brute    -- the plain definition F_i = sum_{j != i, r_ij < r_c} f(r_ij) with the
 *                          minimum-image convention, O(N^2).  U and the virial are pair sums.
 *   orc_cells           -- step N1 of Sec. 2.3 (atom -> cell by position).
 *   orc_cell_order      -- steps N2-N4 of Sec. 2.3 and the reorder vector s of Sec. 2.4 item 4:
 *                          cell occupancy counts k_c, their prefix sum, and the atoms of each
 *                          cell listed in ascending index order.
 *   orc_forces_cells    -- step F1 evaluated over the 27 neighbouring cells (cell side >= r_c).
 *                          Reaches the plain definition exactly up to summation order.
 *   orc_neighbours      -- step N5 of Sec. 2.3: for every atom, the atoms in the 27 neighbouring
 *                          cells that lie within r_c + delta.  The decision r^2 < (r_c+delta)^2
 *                          is taken in the precision the caller names (FP32 or FP64), from
 *                          cell-local coordinates, as the reading of the criterion states.
 *   orc_run             -- leapfrog (kick-drift-kick) integration, Sec. 4.3 item 1 names the
 *                          symplectic leapfrog; forces from the definition at every step; the
 *                          neighbour-refresh rule of Sec. 2.3 (maximum velocity) is tracked so
 *                          that rebuild counts can be compared.
 *   orc_props           -- the measured quantities of Sec. 2.3 (U from the u_i sum, kinetic
 *                          energy, maximum speed) plus virial, pressure and momentum.
 *   orc_force_jvp       -- the force Jacobian-vector product (J lambda)_i = dF_i/dx . lambda.
 *   orc_param_grads     -- dF/d(eps), dF/d(sigma), dU/d(eps), dU/d(sigma).
 *   orc_adjoint         -- reverse-mode derivative of the trajectory loss
 *                          L = (1/S) sum_{n=1..S} U(x_n) + |v_S|^2 through the leapfrog steps,
 *                          with every state stored (no checkpointing).
 *   orc_chain_forces    -- polymer chains (Sec. 4.3 item 2): FENE bonds, bending and dihedral
 *                          terms along chains of consecutive ids, forces as -dU/dr per term;
 *   orc_run_chains      -- orc_run with the chain terms added.
 *   orc_dynamics        -- velocity autocorrelation and mean-square displacement of atoms
 *                          followed by identity (Sec. 4.1 items 1 and 7), from orc_run's
 *                          trajectory, over several time origins.
 *
 * Parity notes: the potential, forces, energies, integrator and adjoint are pinned by closed
 * forms, brute force, lattice sums, invariants and finite differences in the CPU test suite.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (the -ffp-contract=off flag keeps the
 * criterion arithmetic of orc_neighbours exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Pair potential parameters. */
typedef struct {
    double eps;      /* well depth epsilon */
    double sigma;    /* length scale sigma */
    double rc;       /* interaction cutoff r_c (absolute length) */
    int32_t shift;   /* 1: u(r) shifted by a constant so that u(r_c) = 0 */
    int32_t rc_scales_with_sigma; /* 1: r_c = (r_c/sigma) * sigma moves with sigma (WCA) */
} orc_pot;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_BOX = -2, ORC_ERR_MEM = -3 };

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Pair potential (Sec. 3.1): u(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - u_c for r < r_c.     */
/* The force on atom i from j is g(r^2) (x_i - x_j) with g = 24 eps [2 (sigma/r)^12 -          */
/* (sigma/r)^6] / r^2.  Also returned: dg/d(r^2) (for the Jacobian) and the sigma-derivatives. */
/* ------------------------------------------------------------------------------------------ */
static double orc_shift_const(const orc_pot* p)
{
    if (!p->shift) return 0.0;
    double q2 = (p->sigma * p->sigma) / (p->rc * p->rc);
    double q6 = q2 * q2 * q2;
    return 4.0 * p->eps * (q6 * q6 - q6);
}

void orc_pair(const orc_pot* p, double r2, double* u, double* g)
{
    double rc2 = p->rc * p->rc;
    if (!(r2 < rc2)) { *u = 0.0; *g = 0.0; return; }
    double s2 = (p->sigma * p->sigma) / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    *u = 4.0 * p->eps * (s12 - s6) - orc_shift_const(p);
    *g = 24.0 * p->eps * (2.0 * s12 - s6) / r2;
}

/* dg/d(r^2) with g as above: g = 24 eps (2 sigma^12 s^-7 - sigma^6 s^-4), s = r^2. */
static double orc_dg_ds(const orc_pot* p, double r2)
{
    double s2 = (p->sigma * p->sigma) / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    return 24.0 * p->eps * (-14.0 * s12 + 4.0 * s6) / (r2 * r2);
}

/* dg/d(sigma) and du/d(sigma) at fixed r. */
static void orc_sigma_derivs(const orc_pot* p, double r2, double* dg_dsig, double* du_dsig)
{
    double sig = p->sigma;
    double s2 = (sig * sig) / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    /* g = 24 eps (2 s12 - s6) / r2 ; d(s12)/dsig = 12 s12/sig ; d(s6)/dsig = 6 s6/sig */
    *dg_dsig = 24.0 * p->eps * (24.0 * s12 - 6.0 * s6) / (sig * r2);
    double du = 4.0 * p->eps * (12.0 * s12 - 6.0 * s6) / sig;
    if (p->shift && !p->rc_scales_with_sigma) {
        /* u_c = 4 eps ((sigma/r_c)^12 - (sigma/r_c)^6) moves with sigma at fixed r_c. */
        double q2 = (sig * sig) / (p->rc * p->rc);
        double q6 = q2 * q2 * q2;
        du -= 4.0 * p->eps * (12.0 * q6 * q6 - 6.0 * q6) / sig;
    }
    /* With r_c proportional to sigma the shift constant does not depend on sigma, and the
     * moving cutoff adds nothing because u(r_c) = 0 and g(r_c) = 0 for the shifted WCA form. */
    *du_dsig = du;
}

/* Minimum-image displacement along one axis of a periodic box of side L. */
static double orc_min_image(double d, double L)
{
    return d - L * round(d / L);
}

/* ------------------------------------------------------------------------------------------ */
/* Plain definition, O(N^2): F_i = sum_{j != i, r_ij < r_c} g (x_i - x_j); U and the virial     */
/* W = sum_{i<j} r_ij . f_ij are sums over pairs i < j.  u_atom[i] = sum_{j != i} u(r_ij).     */
/* ------------------------------------------------------------------------------------------ */
int orc_forces_brute(int64_t n, const double* x, const double* box, const orc_pot* p,
                     double* f, double* u_atom, double* U_out, double* W_out)
{
    if (n < 0 || !x || !box || !p) return ORC_ERR_ARG;
    double U = 0.0, W = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0, ui = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = orc_min_image(x[3 * i + 0] - x[3 * j + 0], box[0]);
            double dy = orc_min_image(x[3 * i + 1] - x[3 * j + 1], box[1]);
            double dz = orc_min_image(x[3 * i + 2] - x[3 * j + 2], box[2]);
            double r2 = dx * dx + dy * dy + dz * dz;
            double u, g;
            orc_pair(p, r2, &u, &g);
            fx += g * dx; fy += g * dy; fz += g * dz;
            ui += u;
            if (j > i) { U += u; W += g * r2; }
        }
        if (f) { f[3 * i + 0] = fx; f[3 * i + 1] = fy; f[3 * i + 2] = fz; }
        if (u_atom) u_atom[i] = ui;
    }
    if (U_out) *U_out = U;
    if (W_out) *W_out = W;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* N1 (Sec. 2.3): cell grid with n_a = floor(L_a / r_cell) cells per axis, cell side            */
/* w_a = L_a / n_a, and c_a = floor(x_a * (n_a / L_a)) clamped to [0, n_a - 1].  Positions are  */
/* first wrapped into [0, L_a).  Linear cell id = (c_z n_y + c_y) n_x + c_x.                    */
/* ------------------------------------------------------------------------------------------ */
static double orc_wrap(double xa, double L)
{
    if (xa < 0.0) xa += L;
    if (xa >= L) xa -= L;
    return xa;
}

static int orc_grid(const double* box, double r_cell, int32_t nc[3])
{
    for (int a = 0; a < 3; ++a) {
        double q = floor(box[a] / r_cell);
        if (!(q >= 3.0)) return ORC_ERR_BOX;
        if (q > 1.0e6) return ORC_ERR_BOX;
        nc[a] = (int32_t)q;
    }
    return ORC_OK;
}

static void orc_cell_coords(const double* xi, const double* box, const int32_t nc[3], int32_t c[3])
{
    for (int a = 0; a < 3; ++a) {
        double s = (double)nc[a] / box[a];
        double xa = orc_wrap(xi[a], box[a]);
        int32_t ca = (int32_t)floor(xa * s);
        if (ca < 0) ca = 0;
        if (ca > nc[a] - 1) ca = nc[a] - 1;
        c[a] = ca;
    }
}

int orc_cells(int64_t n, const double* x, const double* box, double r_cell,
              int32_t* nc_out, int32_t* cell)
{
    if (n < 0 || !x || !box || !nc_out || !cell) return ORC_ERR_ARG;
    int32_t nc[3];
    int rc = orc_grid(box, r_cell, nc);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) {
        int32_t c[3];
        orc_cell_coords(&x[3 * i], box, nc, c);
        cell[i] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
    }
    nc_out[0] = nc[0]; nc_out[1] = nc[1]; nc_out[2] = nc[2];
    return ORC_OK;
}

/* N2-N4 and the reorder vector s: start[c] = sum_{c' < c} k_{c'} (start has ncells+1 entries),
 * order[start[c] .. start[c+1]) = the atoms of cell c in ascending index order. */
int orc_cell_order(int64_t n, const int32_t* cell, int64_t ncells, int64_t* start, int64_t* order)
{
    if (n < 0 || ncells <= 0 || !cell || !start || !order) return ORC_ERR_ARG;
    for (int64_t c = 0; c <= ncells; ++c) start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (cell[i] < 0 || cell[i] >= ncells) return ORC_ERR_ARG;
        start[cell[i] + 1] += 1;                      /* k_c */
    }
    for (int64_t c = 0; c < ncells; ++c) start[c + 1] += start[c];   /* prefix sum */
    int64_t* fill = (int64_t*)calloc((size_t)ncells, sizeof(int64_t));
    if (!fill) return ORC_ERR_MEM;
    for (int64_t i = 0; i < n; ++i) {                 /* ascending i keeps the order stable */
        int64_t c = cell[i];
        order[start[c] + fill[c]] = i;
        fill[c] += 1;
    }
    free(fill);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* F1 over cells of side >= r_c: the same sums as orc_forces_brute, visiting only the atoms in  */
/* the 27 cells around each atom's cell (with n_a >= 3 these are 27 distinct cells).  Falls     */
/* back to the O(N^2) definition when the box holds fewer than 3 cells per axis.               */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t nc[3];
    int64_t ncells;
    int32_t* cell;
    int64_t* start;
    int64_t* order;
} orc_cell_list;

static void orc_cell_list_free(orc_cell_list* cl)
{
    free(cl->cell); free(cl->start); free(cl->order);
    cl->cell = NULL; cl->start = NULL; cl->order = NULL;
}

static int orc_cell_list_build(int64_t n, const double* x, const double* box, double r_cell,
                               orc_cell_list* cl)
{
    memset(cl, 0, sizeof(*cl));
    int rc = orc_grid(box, r_cell, cl->nc);
    if (rc) return rc;
    cl->ncells = (int64_t)cl->nc[0] * cl->nc[1] * cl->nc[2];
    cl->cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    cl->start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cl->ncells + 1));
    cl->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cl->cell || !cl->start || !cl->order) { orc_cell_list_free(cl); return ORC_ERR_MEM; }
    int32_t nc_dummy[3];
    rc = orc_cells(n, x, box, r_cell, nc_dummy, cl->cell);
    if (!rc) rc = orc_cell_order(n, cl->cell, cl->ncells, cl->start, cl->order);
    if (rc) orc_cell_list_free(cl);
    return rc;
}

/* The 27 cells around cell (c_x, c_y, c_z), periodic; distinct because n_a >= 3. */
static void orc_cells27(const orc_cell_list* cl, const int32_t ci[3], int64_t cc[27])
{
    int q = 0;
    for (int oz = -1; oz <= 1; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
    for (int ox = -1; ox <= 1; ++ox) {
        int32_t cx = (ci[0] + ox + cl->nc[0]) % cl->nc[0];
        int32_t cy = (ci[1] + oy + cl->nc[1]) % cl->nc[1];
        int32_t cz = (ci[2] + oz + cl->nc[2]) % cl->nc[2];
        cc[q++] = ((int64_t)cz * cl->nc[1] + cy) * cl->nc[0] + cx;
    }
}

static void orc_decode_cell(int32_t c, const int32_t nc[3], int32_t out[3])
{
    out[0] = c % nc[0];
    out[1] = (c / nc[0]) % nc[1];
    out[2] = c / (nc[0] * nc[1]);
}

int orc_forces_cells(int64_t n, const double* x, const double* box, const orc_pot* p,
                     double* f, double* u_atom, double* U_out, double* W_out)
{
    if (n < 0 || !x || !box || !p) return ORC_ERR_ARG;
    orc_cell_list cl;
    int rc = orc_cell_list_build(n, x, box, p->rc, &cl);
    if (rc == ORC_ERR_BOX) return orc_forces_brute(n, x, box, p, f, u_atom, U_out, W_out);
    if (rc) return rc;
    double* upair = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* wpair = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!upair || !wpair) { free(upair); free(wpair); orc_cell_list_free(&cl); return ORC_ERR_MEM; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int32_t ci[3];
        orc_decode_cell(cl.cell[i], cl.nc, ci);
        double fx = 0.0, fy = 0.0, fz = 0.0, ui = 0.0, uh = 0.0, wh = 0.0;
        int64_t cc[27];
        orc_cells27(&cl, ci, cc);
        for (int q = 0; q < 27; ++q)
        for (int64_t k = cl.start[cc[q]]; k < cl.start[cc[q] + 1]; ++k) {
            int64_t j = cl.order[k];
            if (j == i) continue;
            double dx = orc_min_image(x[3 * i + 0] - x[3 * j + 0], box[0]);
            double dy = orc_min_image(x[3 * i + 1] - x[3 * j + 1], box[1]);
            double dz = orc_min_image(x[3 * i + 2] - x[3 * j + 2], box[2]);
            double r2 = dx * dx + dy * dy + dz * dz;
            double u, g;
            orc_pair(p, r2, &u, &g);
            fx += g * dx; fy += g * dy; fz += g * dz;
            ui += u;
            if (j > i) { uh += u; wh += g * r2; }
        }
        if (f) { f[3 * i + 0] = fx; f[3 * i + 1] = fy; f[3 * i + 2] = fz; }
        if (u_atom) u_atom[i] = ui;
        upair[i] = uh;
        wpair[i] = wh;
    }
    double U = 0.0, W = 0.0;
    for (int64_t i = 0; i < n; ++i) { U += upair[i]; W += wpair[i]; }   /* fixed order */
    if (U_out) *U_out = U;
    if (W_out) *W_out = W;
    free(upair); free(wpair);
    orc_cell_list_free(&cl);
    return ORC_OK;
}

/* Force on a single atom i from the definition over cells (for sampled checks on big inputs).
 * cell/start/order come from orc_cells + orc_cell_order with r_cell >= r_c. */
int orc_force_on_atoms(int64_t n, const double* x, const double* box, const orc_pot* p,
                       const int32_t* nc, const int32_t* cell, const int64_t* start,
                       const int64_t* order, int64_t nsample, const int64_t* atoms,
                       double* f, double* u_atom)
{
    if (n < 0 || !x || !box || !p || !nc || !cell || !start || !order || !atoms) return ORC_ERR_ARG;
    orc_cell_list cl;
    cl.nc[0] = nc[0]; cl.nc[1] = nc[1]; cl.nc[2] = nc[2];
    cl.ncells = (int64_t)nc[0] * nc[1] * nc[2];
    cl.cell = (int32_t*)cell; cl.start = (int64_t*)start; cl.order = (int64_t*)order;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < nsample; ++s) {
        int64_t i = atoms[s];
        int32_t ci[3];
        orc_decode_cell(cl.cell[i], cl.nc, ci);
        double fx = 0.0, fy = 0.0, fz = 0.0, ui = 0.0;
        int64_t cc[27];
        orc_cells27(&cl, ci, cc);
        for (int q = 0; q < 27; ++q)
        for (int64_t k = cl.start[cc[q]]; k < cl.start[cc[q] + 1]; ++k) {
            int64_t j = cl.order[k];
            if (j == i) continue;
            double dx = orc_min_image(x[3 * i + 0] - x[3 * j + 0], box[0]);
            double dy = orc_min_image(x[3 * i + 1] - x[3 * j + 1], box[1]);
            double dz = orc_min_image(x[3 * i + 2] - x[3 * j + 2], box[2]);
            double r2 = dx * dx + dy * dy + dz * dz;
            double u, g;
            orc_pair(p, r2, &u, &g);
            fx += g * dx; fy += g * dy; fz += g * dz;
            ui += u;
        }
        if (f) { f[3 * s + 0] = fx; f[3 * s + 1] = fy; f[3 * s + 2] = fz; }
        if (u_atom) u_atom[s] = ui;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* N5 (Sec. 2.3): neighbour sets.  Cells of side w_a = L_a / n_a with n_a = floor(L_a/(r_c+d)). */
/* Criterion (the reading of "within r_c + delta" made exact):                                  */
/*   l_a   = x_a - c_a * w_a                     (FP64: product rounded, then difference)       */
/*   FP32: lf_a = (float) l_a, wf_a = (float) w_a,                                              */
/*         d_a  = (lf_{j,a} - lf_{i,a}) + o_a * wf_a   (o_a in {-1,0,1}: the periodic offset of */
/*                                                    j's cell from i's cell; two roundings)   */
/*         r2   = fmaf(d_z, d_z, fmaf(d_y, d_y, d_x * d_x))                                   */
/*         j is a neighbour iff r2 < (float)((r_c + delta)^2)                                   */
/*   FP64: the same expression in double, compared with (r_c + delta)^2.                       */
/* Output: counts[i]; if nbrs != NULL, offsets[i] .. offsets[i+1] hold i's neighbours in        */
/* ascending index order (offsets has n+1 entries and must be filled by a first counting call). */
/* ------------------------------------------------------------------------------------------ */
static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Neighbours of atom i under the criterion above; writes up to cap of them (ascending) to out
 * and returns the full count. */
static int64_t orc_nbrs_of_atom(const orc_cell_list* cl, const double* loc, const double w[3],
                                const float wf[3], double rl2, float rl2f, int32_t use_fp32,
                                int64_t i, int64_t* out, int64_t cap)
{
    int32_t ci[3];
    orc_decode_cell(cl->cell[i], cl->nc, ci);
    int64_t m = 0;
    for (int oz = -1; oz <= 1; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
    for (int ox = -1; ox <= 1; ++ox) {
        int o[3] = {ox, oy, oz};
        int32_t cx = (ci[0] + ox + cl->nc[0]) % cl->nc[0];
        int32_t cy = (ci[1] + oy + cl->nc[1]) % cl->nc[1];
        int32_t cz = (ci[2] + oz + cl->nc[2]) % cl->nc[2];
        int64_t cc = ((int64_t)cz * cl->nc[1] + cy) * cl->nc[0] + cx;
        for (int64_t k = cl->start[cc]; k < cl->start[cc + 1]; ++k) {
            int64_t j = cl->order[k];
            if (j == i) continue;
            int inside;
            if (use_fp32) {
                float d[3];
                for (int a = 0; a < 3; ++a) {
                    float t = (float)loc[3 * j + a] - (float)loc[3 * i + a];
                    float off = (float)o[a] * wf[a];
                    d[a] = t + off;
                }
                float r2 = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
                inside = r2 < rl2f;
            } else {
                double d[3];
                for (int a = 0; a < 3; ++a) {
                    double t = loc[3 * j + a] - loc[3 * i + a];
                    double off = (double)o[a] * w[a];
                    d[a] = t + off;
                }
                double r2 = fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
                inside = r2 < rl2;
            }
            if (inside) {
                if (out && m < cap) out[m] = j;
                ++m;
            }
        }
    }
    if (out) qsort(out, (size_t)(m < cap ? m : cap), sizeof(int64_t), cmp_i64);
    return m;
}

/* Cell list of side r_c + skin and the cell-local FP64 coordinates of every atom. */
static int orc_nbr_setup(int64_t n, const double* x, const double* box, double rl, orc_cell_list* cl,
                         double** loc_out, double w[3], float wf[3])
{
    int rcode = orc_cell_list_build(n, x, box, rl, cl);
    if (rcode) return rcode;
    for (int a = 0; a < 3; ++a) { w[a] = box[a] / (double)cl->nc[a]; wf[a] = (float)w[a]; }
    double* loc = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!loc) { orc_cell_list_free(cl); return ORC_ERR_MEM; }
    for (int64_t i = 0; i < n; ++i) {
        int32_t ci[3];
        orc_decode_cell(cl->cell[i], cl->nc, ci);
        for (int a = 0; a < 3; ++a) {
            double xa = orc_wrap(x[3 * i + a], box[a]);
            double origin = (double)ci[a] * w[a];
            loc[3 * i + a] = xa - origin;
        }
    }
    *loc_out = loc;
    return ORC_OK;
}

int orc_neighbours(int64_t n, const double* x, const double* box, double rc, double skin,
                   int32_t use_fp32, int32_t* nc_out, int64_t* counts, const int64_t* offsets,
                   int64_t* nbrs)
{
    if (n < 0 || !x || !box || !nc_out || !counts) return ORC_ERR_ARG;
    double rl = rc + skin, w[3], *loc = NULL;
    float wf[3];
    orc_cell_list cl;
    int rcode = orc_nbr_setup(n, x, box, rl, &cl, &loc, w, wf);
    if (rcode) return rcode;
    double rl2 = rl * rl;
    float rl2f = (float)rl2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t* out = (nbrs && offsets) ? &nbrs[offsets[i]] : NULL;
        int64_t cap = (nbrs && offsets) ? offsets[i + 1] - offsets[i] : 0;
        counts[i] = orc_nbrs_of_atom(&cl, loc, w, wf, rl2, rl2f, use_fp32, i, out, cap);
    }
    nc_out[0] = cl.nc[0]; nc_out[1] = cl.nc[1]; nc_out[2] = cl.nc[2];
    free(loc);
    orc_cell_list_free(&cl);
    return ORC_OK;
}

/* Neighbour sets of the listed atoms only: counts[s] and nbrs[s * cap ..] (ascending, truncated). */
int orc_neighbours_sample(int64_t n, const double* x, const double* box, double rc, double skin,
                          int32_t use_fp32, int64_t nsample, const int64_t* atoms, int64_t cap,
                          int64_t* counts, int64_t* nbrs)
{
    if (n < 0 || !x || !box || !atoms || !counts || !nbrs || cap <= 0) return ORC_ERR_ARG;
    double rl = rc + skin, w[3], *loc = NULL;
    float wf[3];
    orc_cell_list cl;
    int rcode = orc_nbr_setup(n, x, box, rl, &cl, &loc, w, wf);
    if (rcode) return rcode;
    double rl2 = rl * rl;
    float rl2f = (float)rl2;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < nsample; ++s)
        counts[s] = orc_nbrs_of_atom(&cl, loc, w, wf, rl2, rl2f, use_fp32, atoms[s], &nbrs[s * cap], cap);
    free(loc);
    orc_cell_list_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Measured quantities: U (pair sum), K = (m/2) sum v^2, virial W, P = (2K + W) / (3V),         */
/* momentum m sum v, max |v|.  props layout: [U, K, W, P, px, py, pz, vmax].                    */
/* ------------------------------------------------------------------------------------------ */
enum { ORC_NPROPS = 8 };

static void orc_fill_props(int64_t n, const double* v, const double* box, double mass,
                           double U, double W, double* props)
{
    double K = 0.0, px = 0.0, py = 0.0, pz = 0.0, vmax2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double vx = v[3 * i + 0], vy = v[3 * i + 1], vz = v[3 * i + 2];
        double v2 = vx * vx + vy * vy + vz * vz;
        K += v2;
        px += vx; py += vy; pz += vz;
        if (v2 > vmax2) vmax2 = v2;
    }
    K *= 0.5 * mass;
    double V = box[0] * box[1] * box[2];
    props[0] = U;
    props[1] = K;
    props[2] = W;
    props[3] = (2.0 * K + W) / (3.0 * V);
    props[4] = mass * px; props[5] = mass * py; props[6] = mass * pz;
    props[7] = sqrt(vmax2);
}

int orc_props(int64_t n, const double* x, const double* v, const double* box, const orc_pot* p,
              double mass, double* props)
{
    if (n < 0 || !x || !v || !box || !p || !props) return ORC_ERR_ARG;
    double U, W;
    int rc = orc_forces_cells(n, x, box, p, NULL, NULL, &U, &W);
    if (rc) return rc;
    orc_fill_props(n, v, box, mass, U, W, props);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Leapfrog in kick-drift-kick form, c = dt / (2 m):                                            */
/*   v_{n+1/2} = v_n + c F(x_n);  x_{n+1} = wrap(x_n + dt v_{n+1/2});  v_{n+1} = v_{n+1/2} +    */
/*   c F(x_{n+1}).                                                                              */
/* Neighbour-refresh bookkeeping (the list itself is not needed for the forces, which are the  */
/* definition at every step):                                                                   */
/*   rule 0: none; rule 1: D += dt max_i |v_{n+1/2,i}|, rebuild when D > delta/2 (Sec. 2.3,     */
/*   maximum velocity); rule 2: rebuild when max_i |x_{n+1,i} - x_ref,i| > delta/2.             */
/*   A rebuild resets D = 0 and x_ref = x_{n+1}.                                                */
/* props_out (if not NULL) receives ORC_NPROPS values for every step 0..nsteps.                 */
/* ------------------------------------------------------------------------------------------ */
int orc_run(int64_t n, double* x, double* v, const double* box, const orc_pot* p, double mass,
            double dt, int64_t nsteps, int32_t rule, double skin, double* props_out,
            int64_t* rebuilds_out)
{
    if (n < 0 || !x || !v || !box || !p || nsteps < 0 || mass <= 0.0) return ORC_ERR_ARG;
    size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
    double* f = (double*)malloc(sizeof(double) * n3);
    double* xref = (double*)malloc(sizeof(double) * n3);
    if (!f || !xref) { free(f); free(xref); return ORC_ERR_MEM; }
    double U, W;
    int rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
    if (rc) { free(f); free(xref); return rc; }
    if (props_out) orc_fill_props(n, v, box, mass, U, W, &props_out[0]);
    memcpy(xref, x, sizeof(double) * 3 * (size_t)n);
    double c = dt / (2.0 * mass);
    double D = 0.0;
    int64_t rebuilds = 0;
    for (int64_t step = 0; step < nsteps; ++step) {
        double vmax2 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double v2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double vh = v[3 * i + a] + c * f[3 * i + a];
                v[3 * i + a] = vh;
                v2 += vh * vh;
                x[3 * i + a] = orc_wrap(x[3 * i + a] + dt * vh, box[a]);
            }
            if (v2 > vmax2) vmax2 = v2;
        }
        if (rule == 1) {
            D += dt * sqrt(vmax2);
            if (D > 0.5 * skin) { ++rebuilds; D = 0.0; }
        } else if (rule == 2) {
            double dmax2 = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double d = orc_min_image(x[3 * i + a] - xref[3 * i + a], box[a]);
                    d2 += d * d;
                }
                if (d2 > dmax2) dmax2 = d2;
            }
            if (sqrt(dmax2) > 0.5 * skin) {
                ++rebuilds;
                memcpy(xref, x, sizeof(double) * 3 * (size_t)n);
            }
        }
        rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
        if (rc) { free(f); free(xref); return rc; }
        for (int64_t i = 0; i < 3 * n; ++i) v[i] += c * f[i];
        if (props_out) orc_fill_props(n, v, box, mass, U, W, &props_out[ORC_NPROPS * (step + 1)]);
    }
    if (rebuilds_out) *rebuilds_out = rebuilds;
    free(f); free(xref);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Force Jacobian-vector product.  With d = x_i - x_j and s = |d|^2 the pair force on i is      */
/* g(s) d, whose derivative with respect to d is A = g I + 2 g'(s) d d^T, so                     */
/*   (J lam)_i = sum_j A_ij (lam_i - lam_j).                                                    */
/* ------------------------------------------------------------------------------------------ */
int orc_force_jvp(int64_t n, const double* x, const double* box, const orc_pot* p,
                  const double* lam, double* out)
{
    if (n < 0 || !x || !box || !p || !lam || !out) return ORC_ERR_ARG;
    orc_cell_list cl;
    int rc = orc_cell_list_build(n, x, box, p->rc, &cl);
    int brute = (rc == ORC_ERR_BOX);
    if (rc && !brute) return rc;
    double rc2 = p->rc * p->rc;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
#define ORC_JVP_BODY                                                                            \
        {                                                                                       \
            double d[3], dl[3];                                                                 \
            for (int a = 0; a < 3; ++a) {                                                       \
                d[a] = orc_min_image(x[3 * i + a] - x[3 * j + a], box[a]);                      \
                dl[a] = lam[3 * i + a] - lam[3 * j + a];                                        \
            }                                                                                   \
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];                                \
            if (r2 < rc2) {                                                                     \
                double u, g;                                                                    \
                orc_pair(p, r2, &u, &g);                                                        \
                double gp = orc_dg_ds(p, r2);                                                   \
                double ddl = d[0] * dl[0] + d[1] * dl[1] + d[2] * dl[2];                        \
                for (int a = 0; a < 3; ++a) acc[a] += g * dl[a] + 2.0 * gp * ddl * d[a];        \
            }                                                                                   \
        }
        if (brute) {
            for (int64_t j = 0; j < n; ++j) { if (j == i) continue; ORC_JVP_BODY }
        } else {
            int32_t ci[3];
            orc_decode_cell(cl.cell[i], cl.nc, ci);
            int64_t cc[27];
            orc_cells27(&cl, ci, cc);
            for (int q = 0; q < 27; ++q)
            for (int64_t k = cl.start[cc[q]]; k < cl.start[cc[q] + 1]; ++k) {
                int64_t j = cl.order[k];
                if (j == i) continue; ORC_JVP_BODY
            }
        }
#undef ORC_JVP_BODY
        out[3 * i + 0] = acc[0]; out[3 * i + 1] = acc[1]; out[3 * i + 2] = acc[2];
    }
    if (!brute) orc_cell_list_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Parameter derivatives: dF/deps = F/eps, dU/deps = U/eps (everything is proportional to eps); */
/* dF_i/dsigma = sum_j dg/dsigma (x_i - x_j), dU/dsigma = sum_{i<j} du/dsigma.                   */
/* ------------------------------------------------------------------------------------------ */
int orc_param_grads(int64_t n, const double* x, const double* box, const orc_pot* p,
                    double* dF_deps, double* dF_dsig, double* dU_deps, double* dU_dsig)
{
    if (n < 0 || !x || !box || !p) return ORC_ERR_ARG;
    if (p->rc_scales_with_sigma && p->shift) {
        /* allowed only when g(r_c) = 0 (WCA): the moving cutoff then adds no boundary term */
        double u, g;
        orc_pair(p, p->rc * p->rc * (1.0 - 1e-15), &u, &g);
        if (fabs(g) > 1e-6 * p->eps) return ORC_ERR_ARG;
    }
    double* f = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!f) return ORC_ERR_MEM;
    double U, W;
    int rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
    if (rc) { free(f); return rc; }
    if (dF_deps) for (int64_t i = 0; i < 3 * n; ++i) dF_deps[i] = f[i] / p->eps;
    if (dU_deps) *dU_deps = U / p->eps;
    free(f);
    orc_cell_list cl;
    rc = orc_cell_list_build(n, x, box, p->rc, &cl);
    int brute = (rc == ORC_ERR_BOX);
    if (rc && !brute) return rc;
    double rc2 = p->rc * p->rc;
    double* dus = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!dus) { if (!brute) orc_cell_list_free(&cl); return ORC_ERR_MEM; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0}, du_half = 0.0;
#define ORC_SIG_BODY                                                                            \
        {                                                                                       \
            double d[3];                                                                        \
            for (int a = 0; a < 3; ++a) d[a] = orc_min_image(x[3 * i + a] - x[3 * j + a], box[a]); \
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];                                \
            if (r2 < rc2) {                                                                     \
                double dg, du;                                                                  \
                orc_sigma_derivs(p, r2, &dg, &du);                                              \
                for (int a = 0; a < 3; ++a) acc[a] += dg * d[a];                                \
                if (j > i) du_half += du;                                                       \
            }                                                                                   \
        }
        if (brute) {
            for (int64_t j = 0; j < n; ++j) { if (j == i) continue; ORC_SIG_BODY }
        } else {
            int32_t ci[3];
            orc_decode_cell(cl.cell[i], cl.nc, ci);
            int64_t cc[27];
            orc_cells27(&cl, ci, cc);
            for (int q = 0; q < 27; ++q)
            for (int64_t k = cl.start[cc[q]]; k < cl.start[cc[q] + 1]; ++k) {
                int64_t j = cl.order[k];
                if (j == i) continue; ORC_SIG_BODY
            }
        }
#undef ORC_SIG_BODY
        if (dF_dsig) { dF_dsig[3 * i + 0] = acc[0]; dF_dsig[3 * i + 1] = acc[1]; dF_dsig[3 * i + 2] = acc[2]; }
        dus[i] = du_half;
    }
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += dus[i];
    if (dU_dsig) *dU_dsig = s;
    free(dus);
    if (!brute) orc_cell_list_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Reverse mode through S leapfrog steps, c = dt/(2m), with h_n = v_n + c F(x_n),               */
/* x_{n+1} = x_n + dt h_n, v_{n+1} = h_n + c F(x_{n+1}) and                                      */
/* L = (1/S) sum_{n=1..S} U(x_n) + |v_S|^2.  Adjoints (J symmetric, dU/dx = -F):                 */
/*   lv_S = 2 v_S ;  lx_S = c J(x_S) lv_S - F(x_S)/S                                             */
/*   for n = S-1 .. 0:  lh_n = lv_{n+1} + dt lx_{n+1}                                            */
/*                      lv_n = lh_n                                                              */
/*                      n >= 1: lx_n = lx_{n+1} + c J(x_n) (lh_n + lv_n) - F(x_n)/S              */
/*   dL/dv_0 = lv_0.                                                                            */
/*   dL/dtheta = sum_{n=0}^{S-1} c dF(x_n)/dtheta . lh_n + sum_{k=1}^{S} c dF(x_k)/dtheta . lv_k  */
/*             + (1/S) sum_{k=1}^{S} dU(x_k)/dtheta,   theta in {eps, sigma}.                    */
/* ------------------------------------------------------------------------------------------ */
static double orc_dot(int64_t m, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

int orc_adjoint(int64_t n, const double* x0, const double* v0, const double* box, const orc_pot* p,
                double mass, double dt, int64_t S, double* loss_out, double* dL_deps,
                double* dL_dsig, double* dL_dv0, double* xS_out, double* vS_out)
{
    if (n <= 0 || S <= 0 || !x0 || !v0 || !box || !p || mass <= 0.0) return ORC_ERR_ARG;
    size_t n3 = 3 * (size_t)n;
    double* X = (double*)malloc(sizeof(double) * n3 * (size_t)(S + 1));
    double* v = (double*)malloc(sizeof(double) * n3);
    double* f = (double*)malloc(sizeof(double) * n3);
    double* lx = (double*)malloc(sizeof(double) * n3);
    double* lv = (double*)malloc(sizeof(double) * n3);
    double* lh = (double*)malloc(sizeof(double) * n3);
    double* tmp = (double*)malloc(sizeof(double) * n3);
    double* fe = (double*)malloc(sizeof(double) * n3);
    double* fs = (double*)malloc(sizeof(double) * n3);
    if (!X || !v || !f || !lx || !lv || !lh || !tmp || !fe || !fs) {
        free(X); free(v); free(f); free(lx); free(lv); free(lh); free(tmp); free(fe); free(fs);
        return ORC_ERR_MEM;
    }
    int rc = ORC_OK;
    double c = dt / (2.0 * mass);
    double loss = 0.0;
    memcpy(X, x0, sizeof(double) * n3);
    memcpy(v, v0, sizeof(double) * n3);
    double U, W;
    rc = orc_forces_cells(n, X, box, p, f, NULL, &U, &W);
    for (int64_t s = 0; s < S && !rc; ++s) {
        double* xs = X + n3 * (size_t)s;
        double* xn = X + n3 * (size_t)(s + 1);
        for (size_t k = 0; k < n3; ++k) {
            double h = v[k] + c * f[k];
            v[k] = h;
            xn[k] = orc_wrap(xs[k] + dt * h, box[k % 3]);
        }
        rc = orc_forces_cells(n, xn, box, p, f, NULL, &U, &W);
        for (size_t k = 0; k < n3; ++k) v[k] += c * f[k];
        loss += U / (double)S;
    }
    if (rc) goto done;
    loss += orc_dot((int64_t)n3, v, v);
    if (xS_out) memcpy(xS_out, X + n3 * (size_t)S, sizeof(double) * n3);
    if (vS_out) memcpy(vS_out, v, sizeof(double) * n3);

    double geps = 0.0, gsig = 0.0, dUe, dUs;
    /* terminal step k = S */
    for (size_t k = 0; k < n3; ++k) lv[k] = 2.0 * v[k];
    {
        const double* xS = X + n3 * (size_t)S;
        rc = orc_force_jvp(n, xS, box, p, lv, tmp);
        if (!rc) rc = orc_forces_cells(n, xS, box, p, f, NULL, &U, &W);
        if (!rc) rc = orc_param_grads(n, xS, box, p, fe, fs, &dUe, &dUs);
        if (rc) goto done;
        for (size_t k = 0; k < n3; ++k) lx[k] = c * tmp[k] - f[k] / (double)S;
        geps += c * orc_dot((int64_t)n3, fe, lv) + dUe / (double)S;
        gsig += c * orc_dot((int64_t)n3, fs, lv) + dUs / (double)S;
    }
    for (int64_t s = S - 1; s >= 0; --s) {
        const double* xs = X + n3 * (size_t)s;
        for (size_t k = 0; k < n3; ++k) lh[k] = lv[k] + dt * lx[k];
        rc = orc_param_grads(n, xs, box, p, fe, fs, &dUe, &dUs);
        if (rc) goto done;
        /* h_n depends on F(x_n) */
        geps += c * orc_dot((int64_t)n3, fe, lh);
        gsig += c * orc_dot((int64_t)n3, fs, lh);
        for (size_t k = 0; k < n3; ++k) lv[k] = lh[k];
        if (s >= 1) {
            /* v_n = h_{n-1} + c F(x_n) and the loss term U(x_n)/S */
            geps += c * orc_dot((int64_t)n3, fe, lv) + dUe / (double)S;
            gsig += c * orc_dot((int64_t)n3, fs, lv) + dUs / (double)S;
            for (size_t k = 0; k < n3; ++k) tmp[k] = lh[k] + lv[k];
            double* jv = fe;   /* reuse as output buffer */
            rc = orc_force_jvp(n, xs, box, p, tmp, jv);
            if (!rc) rc = orc_forces_cells(n, xs, box, p, f, NULL, &U, &W);
            if (rc) goto done;
            for (size_t k = 0; k < n3; ++k) lx[k] = lx[k] + c * jv[k] - f[k] / (double)S;
        }
    }
    if (loss_out) *loss_out = loss;
    if (dL_deps) *dL_deps = geps;
    if (dL_dsig) *dL_dsig = gsig;
    if (dL_dv0) memcpy(dL_dv0, lv, sizeof(double) * n3);
done:
    free(X); free(v); free(f); free(lx); free(lv); free(lh); free(tmp); free(fe); free(fs);
    return rc;
}

/* Forward loss only (for finite differences). */
int orc_loss(int64_t n, const double* x0, const double* v0, const double* box, const orc_pot* p,
             double mass, double dt, int64_t S, double* loss_out)
{
    if (n <= 0 || S <= 0 || !x0 || !v0 || !box || !p || !loss_out) return ORC_ERR_ARG;
    size_t n3 = 3 * (size_t)n;
    double* x = (double*)malloc(sizeof(double) * n3);
    double* v = (double*)malloc(sizeof(double) * n3);
    double* f = (double*)malloc(sizeof(double) * n3);
    if (!x || !v || !f) { free(x); free(v); free(f); return ORC_ERR_MEM; }
    memcpy(x, x0, sizeof(double) * n3);
    memcpy(v, v0, sizeof(double) * n3);
    double c = dt / (2.0 * mass), U, W, loss = 0.0;
    int rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
    for (int64_t s = 0; s < S && !rc; ++s) {
        for (size_t k = 0; k < n3; ++k) {
            v[k] += c * f[k];
            x[k] = orc_wrap(x[k] + dt * v[k], box[k % 3]);
        }
        rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
        for (size_t k = 0; k < n3; ++k) v[k] += c * f[k];
        loss += U / (double)S;
    }
    if (!rc) *loss_out = loss + orc_dot((int64_t)n3, v, v);
    free(x); free(v); free(f);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Velocity autocorrelation and mean-square displacement of atoms followed by their permanent  */
/* ids (Sec. 4.1 item 1: atoms keep identities through reordering; Sec. 4.1 item 7: the VACF   */
/* of the SP fluid at rho = 1.0, whose oscillations show the atoms are caged).                 */
/* The trajectory is orc_run's (KDK leapfrog, forces from the definition).  A sample is taken  */
/* at step 0 and after every `every` steps, at integer-step velocities.  Sample s starts a new  */
/* time origin when s is a multiple of origin_every, and every origin is followed for nlag     */
/* samples (lags 0 .. nlag-1):                                                                 */
/*   vacf[k] = sum over origins t0 reaching lag k, and atoms i, of v_i(t0) . v_i(t0 + k T)     */
/*   msd[k]  = the same sum of |r_i(t0 + k T) - r_i(t0)|^2,   T = every dt,                    */
/* with r_i unwrapped: r_i(t) - r_i(t0) is the sum of the drifts dt v_{n+1/2} in between.      */
/* counts[k] = number of origins that reached lag k; the averages per atom are                 */
/* vacf[k] / (n counts[k]) and msd[k] / (n counts[k]).  nsamples = samples taken in total.     */
/* ------------------------------------------------------------------------------------------ */
int orc_dynamics(int64_t n, const double* x0, const double* v0, const double* box, const orc_pot* p,
                 double mass, double dt, int64_t nsamples, int32_t every, int32_t nlag,
                 int32_t origin_every, double* vacf, double* msd, int64_t* counts)
{
    if (n <= 0 || !x0 || !v0 || !box || !p || mass <= 0.0 || nsamples <= 0 || every <= 0 || nlag <= 0 ||
        origin_every <= 0 || !vacf || !msd || !counts)
        return ORC_ERR_ARG;
    size_t n3 = 3 * (size_t)n;
    int32_t norg = (nlag + origin_every - 1) / origin_every;     /* origins alive at once */
    double* x = (double*)malloc(sizeof(double) * n3);
    double* v = (double*)malloc(sizeof(double) * n3);
    double* f = (double*)malloc(sizeof(double) * n3);
    double* dr = (double*)calloc(n3 * (size_t)norg, sizeof(double));    /* displacement since origin */
    double* vo = (double*)calloc(n3 * (size_t)norg, sizeof(double));    /* velocity at the origin */
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)norg);   /* sample index of the origin */
    if (!x || !v || !f || !dr || !vo || !start) {
        free(x); free(v); free(f); free(dr); free(vo); free(start);
        return ORC_ERR_MEM;
    }
    for (int32_t b = 0; b < norg; ++b) start[b] = -1;
    for (int32_t k = 0; k < nlag; ++k) { vacf[k] = 0.0; msd[k] = 0.0; counts[k] = 0; }
    memcpy(x, x0, sizeof(double) * n3);
    memcpy(v, v0, sizeof(double) * n3);
    double c = dt / (2.0 * mass), U, W;
    int rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
    for (int64_t s = 0; s < nsamples && !rc; ++s) {
        if (s > 0) {
            for (int32_t q = 0; q < every && !rc; ++q) {
                for (size_t k = 0; k < n3; ++k) {
                    v[k] += c * f[k];
                    double drift = dt * v[k];
                    for (int32_t b = 0; b < norg; ++b) dr[(size_t)b * n3 + k] += drift;
                    x[k] = orc_wrap(x[k] + drift, box[k % 3]);
                }
                rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
                for (size_t k = 0; k < n3; ++k) v[k] += c * f[k];
            }
            if (rc) break;
        }
        if (s % origin_every == 0) {                   /* a new origin in the oldest slot */
            int32_t b = (int32_t)((s / origin_every) % norg);
            start[b] = s;
            memcpy(&vo[(size_t)b * n3], v, sizeof(double) * n3);
            memset(&dr[(size_t)b * n3], 0, sizeof(double) * n3);
        }
        for (int32_t b = 0; b < norg; ++b) {
            if (start[b] < 0) continue;
            int64_t lag = s - start[b];
            if (lag >= nlag) continue;
            double cv = 0.0, cm = 0.0;
            for (size_t k = 0; k < n3; ++k) {
                cv += v[k] * vo[(size_t)b * n3 + k];
                cm += dr[(size_t)b * n3 + k] * dr[(size_t)b * n3 + k];
            }
            vacf[lag] += cv;
            msd[lag] += cm;
            counts[lag] += 1;
        }
    }
    free(x); free(v); free(f); free(dr); free(vo); free(start);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Polymer chains (Sec. 4.3 item 2): atoms linked by elastic bonds, a bond-angle term that     */
/* depends on adjacent bonds, and an optional dihedral term on three consecutive bonds; the    */
/* pair potential acts between all atoms, bonded ones included.  The chains are consecutive    */
/* ids: atom c*len + k (k = 0..len-1) of a system of n atoms, the last chain shorter if len     */
/* does not divide n.  With b_k = r_{k+1} - r_k (minimum image):                               */
/*   bond      U = -(1/2) kb R0^2 ln(1 - (|b|/R0)^2)          (FENE)                           */
/*   angle     U = ka (1 - cos t),  cos t = b_k . b_{k+1} / (|b_k| |b_{k+1}|)  (0: straight)   */
/*   dihedral  U = kd (1 - cos p),  cos p = m1 . m2 / (|m1| |m2|),  m1 = b_k x b_{k+1},        */
/*             m2 = b_{k+1} x b_{k+2}                                                          */
/* The forces are -dU/dr, from the derivatives of |b|, cos t and cos p written out per term;   */
/* U and the virial W = sum over terms of sum_a r_a . f_a (positions of the term's atoms       */
/* relative to its first atom) are accumulated.  A dihedral whose bonds are collinear to 1e-12 */
/* (m1 or m2 of length below 1e-6 |b_{k+1}|^2) contributes nothing.                            */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t len;       /* atoms per chain (0: no chains) */
    int32_t pad;
    double kb, r0;     /* FENE stiffness and maximum extension */
    double ka;         /* bending constant */
    double kd;         /* dihedral constant */
} orc_chains;

static void orc_cross(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double orc_dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

int orc_chain_forces(int64_t n, const double* x, const double* box, const orc_chains* ch, double* f,
                     double* U_out, double* W_out)
{
    if (n < 0 || !x || !box || !ch) return ORC_ERR_ARG;
    double U = 0.0, W = 0.0;
    if (ch->len >= 2) {
        for (int64_t s = 0; s < n; s += ch->len) {
            int64_t e = s + ch->len < n ? s + ch->len : n;       /* chain atoms s .. e-1 */
            for (int64_t k = s; k + 1 < e; ++k) {               /* bonds (k, k+1) */
                double b[3];
                for (int a = 0; a < 3; ++a) b[a] = orc_min_image(x[3 * (k + 1) + a] - x[3 * k + a], box[a]);
                double r2 = orc_dot3(b, b), q = 1.0 - r2 / (ch->r0 * ch->r0);
                if (!(q > 0.0)) return ORC_ERR_ARG;                /* a bond beyond R0 */
                U += -0.5 * ch->kb * ch->r0 * ch->r0 * log(q);
                double g = ch->kb / q;                              /* f_{k+1} = -g b, f_k = +g b */
                for (int a = 0; a < 3; ++a) {
                    if (f) { f[3 * (k + 1) + a] -= g * b[a]; f[3 * k + a] += g * b[a]; }
                }
                W += -g * r2;                                       /* b . f_{k+1} */
            }
            for (int64_t k = s; k + 2 < e; ++k) {               /* angles (k, k+1, k+2) */
                double b1[3], b2[3];
                for (int a = 0; a < 3; ++a) {
                    b1[a] = orc_min_image(x[3 * (k + 1) + a] - x[3 * k + a], box[a]);
                    b2[a] = orc_min_image(x[3 * (k + 2) + a] - x[3 * (k + 1) + a], box[a]);
                }
                double l1 = sqrt(orc_dot3(b1, b1)), l2 = sqrt(orc_dot3(b2, b2));
                double c = orc_dot3(b1, b2) / (l1 * l2);
                U += ch->ka * (1.0 - c);
                /* dc/db1 = b2/(l1 l2) - c b1/l1^2, dc/db2 = b1/(l1 l2) - c b2/l2^2; F = ka dc/dr */
                double g1[3], g2[3], fr[3][3];
                for (int a = 0; a < 3; ++a) {
                    g1[a] = b2[a] / (l1 * l2) - c * b1[a] / (l1 * l1);
                    g2[a] = b1[a] / (l1 * l2) - c * b2[a] / (l2 * l2);
                    fr[0][a] = -ch->ka * g1[a];                     /* r_k enters b1 with a minus */
                    fr[1][a] = ch->ka * (g1[a] - g2[a]);
                    fr[2][a] = ch->ka * g2[a];
                }
                for (int a = 0; a < 3; ++a) {
                    if (f) { f[3 * k + a] += fr[0][a]; f[3 * (k + 1) + a] += fr[1][a]; f[3 * (k + 2) + a] += fr[2][a]; }
                }
                W += orc_dot3(b1, fr[1]) + (orc_dot3(b1, fr[2]) + orc_dot3(b2, fr[2]));
            }
            for (int64_t k = s; k + 3 < e && ch->kd != 0.0; ++k) {   /* dihedrals (k .. k+3) */
                double b1[3], b2[3], b3[3], m1[3], m2[3];
                for (int a = 0; a < 3; ++a) {
                    b1[a] = orc_min_image(x[3 * (k + 1) + a] - x[3 * k + a], box[a]);
                    b2[a] = orc_min_image(x[3 * (k + 2) + a] - x[3 * (k + 1) + a], box[a]);
                    b3[a] = orc_min_image(x[3 * (k + 3) + a] - x[3 * (k + 2) + a], box[a]);
                }
                orc_cross(b1, b2, m1);
                orc_cross(b2, b3, m2);
                double q1 = sqrt(orc_dot3(m1, m1)), q2 = sqrt(orc_dot3(m2, m2)), bb = orc_dot3(b2, b2);
                if (q1 < 1e-6 * bb || q2 < 1e-6 * bb) continue;
                double c = orc_dot3(m1, m2) / (q1 * q2);
                U += ch->kd * (1.0 - c);
                /* dc/dm1 = m2/(q1 q2) - c m1/q1^2 (and 1 <-> 2); G . (db1 x b2) = db1 . (b2 x G),  */
                /* G . (b1 x db2) = db2 . (G x b1): dc/db1 = b2 x G1, dc/db2 = G1 x b1 + b3 x G2,    */
                /* dc/db3 = G2 x b2                                                                  */
                double G1[3], G2[3], d1[3], d2a[3], d2b[3], d3[3], fr[4][3];
                for (int a = 0; a < 3; ++a) {
                    G1[a] = m2[a] / (q1 * q2) - c * m1[a] / (q1 * q1);
                    G2[a] = m1[a] / (q1 * q2) - c * m2[a] / (q2 * q2);
                }
                orc_cross(b2, G1, d1);
                orc_cross(G1, b1, d2a);
                orc_cross(b3, G2, d2b);
                orc_cross(G2, b2, d3);
                for (int a = 0; a < 3; ++a) {
                    double d2 = d2a[a] + d2b[a];
                    fr[0][a] = -ch->kd * d1[a];
                    fr[1][a] = ch->kd * (d1[a] - d2);
                    fr[2][a] = ch->kd * (d2 - d3[a]);
                    fr[3][a] = ch->kd * d3[a];
                }
                for (int q = 0; q < 4; ++q)
                    for (int a = 0; a < 3; ++a)
                        if (f) f[3 * (k + q) + a] += fr[q][a];
                double r2[3], r3[3];
                for (int a = 0; a < 3; ++a) { r2[a] = b1[a] + b2[a]; r3[a] = r2[a] + b3[a]; }
                W += orc_dot3(b1, fr[1]) + orc_dot3(r2, fr[2]) + orc_dot3(r3, fr[3]);
            }
        }
    }
    if (U_out) *U_out = U;
    if (W_out) *W_out = W;
    return ORC_OK;
}

/* orc_run with the chain terms added to the pair forces (same KDK steps, props with the chain
 * energy in U and its virial in W; rule 0 only). */
int orc_run_chains(int64_t n, double* x, double* v, const double* box, const orc_pot* p, const orc_chains* ch,
                   double mass, double dt, int64_t nsteps, double* props_out)
{
    if (n < 0 || !x || !v || !box || !p || !ch || nsteps < 0 || mass <= 0.0) return ORC_ERR_ARG;
    size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
    double* f = (double*)malloc(sizeof(double) * n3);
    if (!f) return ORC_ERR_MEM;
    double U, W, Uc, Wc;
    int rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
    if (!rc) rc = orc_chain_forces(n, x, box, ch, f, &Uc, &Wc);
    if (!rc && props_out) orc_fill_props(n, v, box, mass, U + Uc, W + Wc, &props_out[0]);
    double c = dt / (2.0 * mass);
    for (int64_t step = 0; step < nsteps && !rc; ++step) {
        for (int64_t i = 0; i < 3 * n; ++i) {
            v[i] += c * f[i];
            x[i] = orc_wrap(x[i] + dt * v[i], box[i % 3]);
        }
        rc = orc_forces_cells(n, x, box, p, f, NULL, &U, &W);
        if (!rc) rc = orc_chain_forces(n, x, box, ch, f, &Uc, &Wc);
        if (rc) break;
        for (int64_t i = 0; i < 3 * n; ++i) v[i] += c * f[i];
        if (props_out) orc_fill_props(n, v, box, mass, U + Uc, W + Wc, &props_out[ORC_NPROPS * (step + 1)]);
    }
    free(f);
    return rc;
}
