/*
 * gbmd.h -- C ABI of libgbmd.so, a GB300 (sm_103a) library for short-range pair-force molecular
 * dynamics with cell and neighbour lists in periodic boxes.
 *
 * The method is the one of Rapaport, "GPU molecular dynamics: Algorithms and performance"
 * (arXiv 2003.14061): atoms are assigned to cells and cell layers (Sec. 2.3, steps N1-N4), a
 * neighbour matrix W is built from the 27 surrounding cells (N5), forces are accumulated per atom
 * from W without Newton's third law (F1), the energy is a reduction of per-atom terms (F2), the
 * state is advanced by the leapfrog integrator (Sec. 4.3 item 1), W is refreshed when the maximum
 * velocity says atoms may have moved by half the shell (Sec. 2.3), and atoms are periodically
 * reordered by cell (Sec. 2.4 item 4, Sec. 4.1 item 1).
 *
 * Conventions
 *   - Every function returns an int: MD_OK (0) or a negative md_status.  Nothing throws across
 *     this boundary.  md_last_error() gives a message for the last failure on this thread.
 *   - Device memory: the caller allocates one workspace of md_workspace_bytes() bytes (device
 *     memory, 256-byte aligned) and passes it to md_create / md_create_batch; the library carves
 *     all its arrays out of it and allocates nothing else on the device.  The caller frees the
 *     workspace after md_destroy.
 *   - Host arrays passed in are owned by the caller and are only read or written during the call.
 *     Pointers named "host or device" may point to either (unified addressing decides).
 *   - Streams: every call is ordered on the stream given at creation (a cudaStream_t passed as
 *     void*).  Only md_reduce_props, md_get_state, md_get_cells, md_get_neighbours, md_check and
 *     md_adjoint wait for the stream; the others return after queueing work.
 *   - Atoms carry permanent ids 0..n-1 (the order of the arrays given at creation), which survive
 *     reordering (Sec. 4.1 item 1).  All state exchanged through this ABI is in id order.
 *   - Errors detected on the device (neighbour-capacity overflow, non-finite values) are latched
 *     in device memory and returned by the next call that waits for the stream.
 */
#ifndef GBMD_H
#define GBMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_system md_system;   /* opaque; owned by the library */

/* Arithmetic of the pair forces and of the state (Sec. 4.1 item 7 discusses s.p. and d.p.).
 *   MD_FP64  : pair forces, positions and velocities in FP64.
 *   MD_MIXED : pair forces in FP32; positions, velocities and all reductions beyond a 32-lane
 *              warp in FP64.
 *   MD_FP32  : pair forces, positions and velocities in FP32; reductions in FP64. */
typedef enum { MD_FP64 = 0, MD_MIXED = 1, MD_FP32 = 2 } md_precision;

/* When the neighbour matrix is rebuilt (Sec. 2.3 reduces the largest atom speed for this
 * decision).
 *   MD_REBUILD_VMAX  : D += dt * max_i |v_i| after every position update; rebuild when
 *                      D > skin/2, then D = 0.
 *   MD_REBUILD_DISP  : rebuild when max_i |x_i - x_i(at last rebuild)| > skin/2.
 *   MD_REBUILD_EVERY : rebuild before every force evaluation (a plain cell list when skin = 0). */
typedef enum { MD_REBUILD_VMAX = 0, MD_REBUILD_DISP = 1, MD_REBUILD_EVERY = 2 } md_rebuild_rule;

typedef enum {
    MD_OK = 0,
    MD_ERR_INVALID_ARG = -1,   /* bad pointer, size or parameter */
    MD_ERR_BOX_TOO_SMALL = -2, /* fewer than 3 cells of side >= r_c + skin along an axis */
    MD_ERR_NBR_OVERFLOW = -3,  /* an atom had more neighbours than nbr_capacity */
    MD_ERR_CELL_OVERFLOW = -4, /* more than 1023 cells along an axis, or too many atoms */
    MD_ERR_NONFINITE = -5,     /* a non-finite position, velocity or force was produced */
    MD_ERR_TIMEOUT = -6,       /* a bounded device wait gave up */
    MD_ERR_CUDA = -7,          /* a CUDA runtime call failed */
    MD_ERR_WORKSPACE = -8      /* workspace missing, misaligned or smaller than required */
} md_status;

/* Parameters shared by all replicas of a system (the paper keeps them in one constant-memory
 * struct, Sec. 2.4 item 2).  Lengths in units of sigma, energies of eps, masses of m. */
typedef struct {
    int64_t n;             /* atoms (md_create); ignored by md_create_batch */
    double box[3];         /* periodic box sides (md_create); ignored by md_create_batch */
    double eps;            /* Lennard-Jones epsilon */
    double sigma;          /* Lennard-Jones sigma */
    double mass;           /* atom mass */
    double rc;             /* interaction cutoff r_c (absolute; WCA: 2^(1/6) sigma) */
    double skin;           /* neighbour shell thickness delta (Sec. 4.1 item 5); 0 = cell list */
    double dt;             /* time step */
    int32_t shift_energy;  /* 1: u(r) shifted so that u(r_c) = 0 (the forces are unchanged) */
    int32_t precision;     /* md_precision */
    int32_t reorder_every; /* reorder atoms by cell at the first rebuild at least this many steps
                              after the last reorder (Sec. 4.1 item 1: 100); 0 = every rebuild */
    int32_t nbr_capacity;  /* rows of W, i.e. maximum neighbours per atom; 0 = automatic */
    int32_t rebuild_rule;  /* md_rebuild_rule */
    int32_t props_every;   /* >0: accumulate props every this many steps inside md_integrate into
                              a device time series (md_get_series); 0: only on md_reduce_props */
    int32_t cell_block;    /* cell order: rows of cells (fixed y, z) are numbered in blocks of b z
                              planes, (z / b, y, z % b), x fastest within a row, so that slot
                              ranges are compact in 3D; b = this value rounded down to a power of
                              two; 1 = plain (z, y) order, 0 = chosen from the system size and
                              the SM count.  Performance only: results
                              agree with any other choice to rounding (the summation order of a
                              force follows the within-cell order), cells and neighbour sets
                              exactly. */
} md_params;

/* Measured quantities of one replica (Sec. 2.3: total interaction energy from the reduction of
 * the u_i, kinetic energy, maximal velocity), plus the virial and pressure. */
typedef struct {
    double U;              /* potential energy sum_{i<j} u(r_ij) = (1/2) sum_i u_i */
    double K;              /* kinetic energy (m/2) sum_i |v_i|^2, velocities at the integer step */
    double E_per_atom;     /* (U + K) / n */
    double virial;         /* W = sum_{i<j} r_ij . f_ij */
    double pressure;       /* (2K + W) / (3V) */
    double P[3];           /* total momentum m sum_i v_i */
    double vmax;           /* max_i |v_i| */
    double mean_nbrs;      /* mean neighbour count at the last rebuild */
    int64_t step;          /* steps taken since creation or md_set_state */
    int64_t rebuilds;      /* neighbour-matrix rebuilds since creation or md_set_state */
    int32_t max_cell_occ;  /* N_l = max_c k_c at the last rebuild (Sec. 2.3 step N3) */
    int32_t max_nbrs;      /* max_i m_i at the last rebuild */
    int64_t reorders;      /* reorders by cell since creation or md_set_state (both reorder) */
} md_props;

/* Size of the workspace for one system (md_create) or a batch (md_create_batch); 0 on error. */
size_t md_workspace_bytes(const md_params* p);
size_t md_workspace_bytes_batch(const md_params* p, int32_t nrep, const int64_t* n_rep,
                                const double* box_rep);

/* Create one system of p->n atoms in box p->box.  x0, v0: host or device, [n][3] FP64 in id
 * order; positions are wrapped into the box (any number of box lengths away).  The call bins the
 * atoms, reorders them by cell and builds the neighbour matrix (N1-N5).  A non-finite x0 or v0
 * component fails with MD_ERR_NONFINITE.  stream: cudaStream_t (NULL = legacy default stream). */
int md_create(const md_params* p, void* d_workspace, size_t workspace_bytes, const double* x0,
              const double* v0, void* stream, md_system** out);

/* Create nrep independent systems advanced together (Sec. 4.3 item 2: independent simulations
 * carried out simultaneously in a single run).  n_rep[r] atoms, box_rep[3r..3r+2]; x0/v0 hold
 * the replicas' atoms concatenated in replica order ([sum n_rep][3], FP64, host or device).
 * Replica r's atoms have ids sum_{q<r} n_rep[q] + 0 .. n_rep[r]-1. */
int md_create_batch(const md_params* p, int32_t nrep, const int64_t* n_rep, const double* box_rep,
                    void* d_workspace, size_t workspace_bytes, const double* x0, const double* v0,
                    void* stream, md_system** out);

/* N1-N4 (Sec. 2.3) and the reorder of Sec. 2.4 item 4: bin every atom into its cell, count the
 * cell occupancies k_c, prefix-sum them and list each cell's atoms in ascending slot order; if a
 * reorder is due (or reorder_every == 0), permute the atoms into that order. */
int md_bin_cells(md_system* s);

/* N5 (Sec. 2.3): rebuild the neighbour matrix W from the current binning.  Each W entry holds the
 * neighbour's slot and its cell's periodic offset; neighbours are within r_c + skin by the
 * FP32 (MD_MIXED, MD_FP32) or FP64 (MD_FP64) criterion on cell-local coordinates. */
int md_build_neighbours(md_system* s);

/* F1 (Sec. 2.3): forces f_i and per-atom energies u_i at the current positions from W, without
 * advancing the state (read them with md_get_state). */
int md_compute_forces(md_system* s);

/* Advance every replica by nsteps leapfrog steps (kick-drift-kick, Sec. 4.3 item 1), evaluating
 * forces from W each step and rebuilding W (with a reorder when due) whenever the rebuild rule
 * fires.  Stream-ordered; does not wait. */
int md_integrate(md_system* s, int32_t nsteps);

/* F2 (Sec. 2.3) and the other measured quantities at the current state, one md_props per replica
 * (out must hold md_nrep(s) entries; host pointer).  Waits for the stream. */
int md_reduce_props(md_system* s, md_props* out);

/* Time series written by md_integrate when props_every > 0 (a ring of the last 1024 rows): up to
 * max_rows of the most recent rows of [step, U, K, W, P, px, py, pz, vmax] (9 doubles) per
 * replica, replica-major, oldest first.  Returns the number of rows written per replica through
 * *rows.  Host pointer.  Waits. */
int md_get_series(md_system* s, double* out, int32_t max_rows, int32_t* rows);
int md_clear_series(md_system* s);

/* Queue (without waiting) a copy of the most recent time-series row of every replica,
 * [nrep][9] doubles as in md_get_series, to dst (pinned host or device memory; pageable host
 * memory makes the copy synchronous).  The row is the props of the last props step issued by
 * md_integrate: the energies of that step's positions and integer-step velocities.  Errors with
 * MD_ERR_INVALID_ARG if no props step has been issued. */
int md_props_latest(md_system* s, double* dst);

/* State in id order.  x: positions wrapped into the box; v: velocities at the current integer
 * step; f: forces at the current positions (computed by this call).  Each may be NULL; host or
 * device; [n_total][3] FP64.  Waits for the stream. */
int md_get_state(md_system* s, double* x, double* v, double* f);

/* Replace positions and velocities (id order, [n_total][3] FP64, host or device), resetting the
 * step and rebuild counters, then bin, reorder and rebuild W as md_create does.  A non-finite
 * component fails with MD_ERR_NONFINITE (the state is then unusable until the next successful
 * md_set_state). */
int md_set_state(md_system* s, const double* x, const double* v);

/* Diagnostics in id order (host pointers), from the last binning / rebuild:
 *   md_get_cells      : cell[n_total] = linear cell id (c_z n_y + c_y) n_x + c_x in the replica.
 *   md_get_neighbours : counts[n_total] = m_i; nbr_ids[n_total * cap] = the neighbours' ids
 *                       (row i, first counts[i] entries, unordered; rows truncated at cap). */
int md_get_cells(md_system* s, int32_t* cell);
int md_get_neighbours(md_system* s, int32_t* counts, int32_t* nbr_ids, int32_t cap);

/* Polymer chains (Sec. 4.3 item 2: atoms linked by elastic bonds, a bond-angle term from adjacent
 * bonds and an optional dihedral term on three consecutive bonds, all other interactions as
 * before).  In every replica the atoms of local ids c*length .. c*length + length - 1 form chain
 * c (the last chain shorter when length does not divide the replica's atoms).  With b the bond
 * vectors between consecutive atoms of a chain (minimum image):
 *   bond      U = -(1/2) fene_k fene_r0^2 ln(1 - |b|^2 / fene_r0^2)     (FENE)
 *   bend      U = bend_k (1 - cos t),  t the angle between consecutive bonds (0 = straight)
 *   dihedral  U = dihedral_k (1 - cos p),  p the angle between the normals b1 x b2 and b2 x b3
 *             (skipped while the bonds are collinear to 1e-6)
 * The pair potential still acts between all atoms, bonded ones included.  Each thread computes
 * the force on its own atom from every term the atom belongs to (positions of up to three
 * chain neighbours on each side, found through the permanent ids); U and the virial include the
 * terms.  FP32 arithmetic as the pair forces; MD_MIXED and MD_FP32 only.  length 0 removes the
 * chains.  A bond stretched to fene_r0 or beyond gives non-finite forces (MD_ERR_NONFINITE).
 * md_adjoint refuses systems with chains. */
typedef struct {
    int32_t length;        /* atoms per chain (0: no chains) */
    int32_t pad;
    double fene_k;         /* FENE stiffness (30 in the usual bead-spring units) */
    double fene_r0;        /* FENE maximum extension (1.5) */
    double bend_k;
    double dihedral_k;
} md_chains;
int md_set_chains(md_system* s, const md_chains* c);

/* Waits for the stream and returns the first latched device error (then clears it).  A
 * non-finite value is reported before a neighbour overflow it may have caused. */
int md_check(md_system* s);

/* Test hook for the error-reporting path (the paper has no counterpart): queues, on the system's
 * stream, a one-thread kernel that sets the device error word as a kernel meeting the condition
 * would.  status: MD_ERR_NBR_OVERFLOW, MD_ERR_NONFINITE or MD_ERR_TIMEOUT (else
 * MD_ERR_INVALID_ARG).  The next call that waits (md_check, md_reduce_props, ...) returns that
 * status and clears it, so conditions a healthy run never meets -- a bounded device wait giving
 * up -- can be tested without making any kernel fail. */
int md_debug_set_error(md_system* s, int32_t status);

/* Sizes: replicas, total atoms, rows of W, cells per axis of replica r (nc[3]). */
int32_t md_nrep(const md_system* s);
int64_t md_natoms(const md_system* s);
int32_t md_nbr_capacity(const md_system* s);
int md_cells_per_axis(const md_system* s, int32_t r, int32_t* nc);

/* Launch shapes chosen by the autotuner (paper_2003_14061_gb300.tune): the paper found block
 * size mattered little on its GPU and warned that this need not hold in general (Sec. 4.1
 * item 2).  A field left 0 keeps its current value. */
typedef struct {
    int32_t ctas_per_sm;     /* persistent CTAs per SM of the step kernel and the other per-step
                                tile loops (1..64); the step kernel is also compiled to fit 4, 8,
                                12 or 16 CTAs per SM (the largest not above this) and its grid is
                                capped at residency.  The rebuild kernels (binning, scatter,
                                reorder, neighbour build) always run at their full residency */
    int32_t nbr_batch;       /* W entries each thread loads together in the pair loop: 2, 4 or 8 */
    int32_t build_batch;     /* neighbour build: 2 or 4 = one thread per atom loading that many
                                candidates together; 32 = one warp per cell, each row of
                                candidates staged once in shared memory (for cells of tens of
                                atoms); 1 = one thread per atom over half-side sub-cells, the
                                atoms counting-sorted by sub-cell and only the sub-cells within
                                reach scanned (about half the candidates).  The neighbour sets
                                are the same for every choice; the order within a column of W
                                (and so the summation order of a force) follows the choice */
    int32_t use_graph;       /* 1: md_integrate replays captured CUDA graphs; 2: direct launches */
    int32_t step_kernel;     /* fused step kernel (MD_MIXED, MD_FP32): 1 = each thread loads its
                                atom's state and W column; warps take 32-atom warp-tiles from
                                the slot range of the SM they run on, the next one prefetched
                                into L2;
                                2 = the tile's state and W rows copied into a two-stage
                                shared-memory ring by cp.async.bulk, completing on mbarriers;
                                3 = as 1 but on 128-atom tiles per CTA, with each tile's
                                neighbour positions first copied into
                                shared memory by cp.async.bulk (one slot window per row of
                                neighbour cells; compact when atoms are reordered at every
                                rebuild, reorder_every = 0);
                                4 = no neighbour matrix (the cell-block alternative of Sec. 4.2
                                item 1): every atom of the 27 cells around an atom is tested
                                against r_c each step, two at a time in packed FP32x2; atoms are
                                then reordered by cell at every rebuild and W is not built
                                (md_get_neighbours reports the last W built; md_adjoint refuses
                                this kernel);
                                5 = the half neighbour list with Newton's third law (the variant
                                Sec. 2.3 rejects): W keeps each pair once, at its lower slot; a
                                first kernel evaluates each pair once and adds the force to both
                                atoms (the partner by vector atomic adds into FP32 buffers), the
                                step kernel then reads and clears the buffers.  The atomics add
                                in no fixed order, so repeat runs differ in the last bits;
                                md_get_neighbours reports the half sets; md_adjoint refuses it */
    int32_t build_stage;     /* neighbour build (build_batch 1, 2, 4): 1 = each thread appends its
                                column of W in shared memory and the warps write whole rows (128
                                contiguous bytes per row for 32 atoms; for matrices far larger
                                than L2), 2 = each entry written to W as found */
    int32_t reorder_every;   /* the reorder of atoms by cell (Sec. 4.1 item 1): at the first rebuild
                                at least this many steps after the last reorder, or -1 = at
                                every rebuild; starts as md_params.reorder_every (0 there reads
                                as -1 here); 0 keeps the current value in md_set_tuning */
} md_tuning;
int md_set_tuning(md_system* s, const md_tuning* t);
int md_get_tuning(const md_system* s, md_tuning* t);

/* Reverse-mode derivative of a trajectory loss (the paper has no adjoint; this differentiates
 * its method: the leapfrog of Sec. 4.3 item 1 and the pair force of Sec. 2.3).  Starting from
 * the system's current state (x_0, v_0), S = nsteps kick-drift-kick steps are taken and
 *     L = (1/S) sum_{n=1..S} U(x_n) + |v_S|^2
 * is differentiated with respect to eps, sigma and every initial velocity.  The trajectory is run
 * as segments of ckpt_every steps, each restarted from an FP64 checkpoint of (x, v); the reverse
 * pass recomputes one segment at a time from its checkpoint (checkpoint-and-recompute) and walks
 * it backwards with one force-Jacobian-vector-product kernel per step (FP32 pair arithmetic, FP64
 * accumulation).  sigma moves the cutoff with it when r_c = 2^(1/6) sigma (WCA); otherwise r_c is
 * held fixed.  The segments run from CUDA graphs captured on first use and cached per (d_work,
 * nsteps, ckpt_every, segment shape); md_set_tuning and md_destroy release them, and a call
 * with another workspace or horizon captures its own.
 *   d_work     : device scratch of md_adjoint_workspace_bytes(s, nsteps, ckpt_every) bytes,
 *                256-byte aligned, owned by the caller (snapshots of one segment, checkpoints,
 *                adjoint vectors).
 *   loss, dL_deps, dL_dsigma : host doubles (each may be NULL).
 *   dL_dv0     : [n][3] FP64 in id order, host or device (may be NULL).
 * Needs nrep == 1 and MD_MIXED or MD_FP32.  Waits for the stream.  On return the system is back
 * at (x_0, v_0) with its step and rebuild counters reset, as after md_set_state. */
size_t md_adjoint_workspace_bytes(const md_system* s, int32_t nsteps, int32_t ckpt_every);
int md_adjoint(md_system* s, void* d_work, size_t work_bytes, int32_t nsteps, int32_t ckpt_every, double* loss,
               double* dL_deps, double* dL_dsigma, double* dL_dv0);

/* Velocity autocorrelation and mean-square displacement of atoms followed by their permanent
 * ids (Sec. 4.1 item 1: ids survive the reorders; Sec. 4.1 item 7: the VACF of the soft-sphere
 * fluid at density 1.0 oscillates as atoms are caged).  md_dyn_begin starts a measurement in a
 * caller-owned device buffer; every md_dyn_sample takes one sample at the current state (wrapped
 * positions, velocities at the integer step; it evaluates the forces for them), the caller
 * advancing the system between samples by a fixed number of steps T.  Sample s starts a new
 * time origin when s is a multiple of origin_every, and each origin is followed for nlag samples
 * (lags 0 .. nlag-1, at most 8 origins at once: ceil(nlag / origin_every) <= 8).  md_dyn_get
 * returns, for each lag k,
 *     vacf[k] = < v_i(t0) . v_i(t0 + k T) >,   msd[k] = < |r_i(t0 + k T) - r_i(t0)|^2 >
 * averaged over all atoms (of all replicas) and over the origins that reached lag k
 * (counts[k]).  r is unwrapped from consecutive samples by the minimum image, so an atom must
 * move less than half a box side between two samples.  Sums are per CTA in FP64, added in a
 * fixed order.  The self-diffusion coefficient is the slope of msd / 6 at long lags.
 *   d_work : md_dyn_workspace_bytes(s, nlag, origin_every) bytes of device memory, 256-byte
 *            aligned, owned by the caller and untouched by other calls (per-atom velocities and
 *            displacements of every origin, indexed by id).
 *   vacf, msd : host [nlag] doubles (may be NULL); counts: host [nlag] int64 (may be NULL).
 * md_dyn_sample queues work and does not wait; md_dyn_get waits.  A new md_dyn_begin restarts the
 * measurement. */
size_t md_dyn_workspace_bytes(const md_system* s, int32_t nlag, int32_t origin_every);
int md_dyn_begin(md_system* s, void* d_work, size_t work_bytes, int32_t nlag, int32_t origin_every);
int md_dyn_sample(md_system* s);
int md_dyn_get(md_system* s, double* vacf, double* msd, int64_t* counts);

/* Per-phase timing (the breakdown of Table 2 of the paper: neighbour matrix, forces +
 * integration, layer/cell assignment, reorder, energy).  With timing enabled, every phase is
 * bracketed by CUDA events on the system's stream.  md_get_timing waits for the stream, then
 * returns for each phase the summed milliseconds and the number of timed intervals they add up
 * (both 0 while timing is off), and the number of kernels launched (counted whether or not
 * timing is on), and resets the counters.  Arrays hold MD_NPHASE entries (host pointers, each
 * may be NULL). */
#define MD_NPHASE 6
enum {
    MD_PHASE_STEP = 0,     /* F1 fused with the leapfrog update (and F2 when props_every hits) */
    MD_PHASE_BIN = 1,      /* N1-N4: cells, occupancy counts, prefix sum, cell order */
    MD_PHASE_REORDER = 2,  /* reorder of the atoms by cell (Sec. 4.1 item 1) */
    MD_PHASE_BUILD = 3,    /* N5: neighbour matrix */
    MD_PHASE_PROPS = 4,    /* md_reduce_props: forces and reductions at the current state */
    MD_PHASE_OTHER = 5     /* state exchange and standalone force passes */
};
int md_set_timing(md_system* s, int32_t enable);
int md_get_timing(md_system* s, double* ms, int64_t* calls, int64_t* launches);

/* Release the system (host-side bookkeeping and graphs).  The workspace stays the caller's. */
int md_destroy(md_system* s);

/* Forces for a small system without any device allocation (the paper has no counterpart).
 * For callers that cannot allocate device memory where they need forces -- code inside another
 * runtime or framework that owns the device allocator and hands out only pre-planned buffers,
 * plug-ins running between someone else's kernels where the synchronisation of cudaMalloc/
 * cudaFree is not allowed, code with no workspace to hand -- this computes f_i and u_i as
 * md_compute_forces does (FP32 pair arithmetic on cell-local coordinates), over a plain cell
 * list of side >= rc (skin is ignored) kept in one file-scope device array of 1.75 MiB that
 * every GPU loading the library holds until exit.  The atoms of each cell are visited in index
 * order, so repeated calls on the same input return the same bits.
 *   p      : eps, sigma, rc, shift_energy and box are used; the rest is ignored.
 *   n      : 1..65536 atoms; the box may hold at most 65536 cells of side >= rc
 *            (MD_ERR_INVALID_ARG otherwise, before any work is queued; md_last_error says which).
 *   x      : device, [n][3] FP64 positions, any number of box lengths from the box (wrapped
 *            into it on the fly).
 *   f      : device, [n][3] FP64 output forces;  u: device, [n] FP64 output u_i, or NULL.
 *   stream : cudaStream_t as void*; the call only queues work and does not wait.
 * The array is shared by all calls and keeps the last call's contents (each call clears what it
 * needs to start at zero); calls whose work overlaps on the GPU race on it and must not be
 * issued.  The first call on each device looks up the array's device address with that device
 * current, so it should come before any stream capture; the address is kept until the process
 * exits, so the call must not be used on a device after cudaDeviceReset.  A launch error left
 * pending by earlier, unrelated work is cleared on entry rather than reported.  Calls no
 * cudaMalloc or cudaFree. */
int md_forces_static(const md_params* p, int64_t n, const double* x, double* f, double* u, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* md_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GBMD_H */
