// gbmd_internal.cuh -- device data layout and helpers shared by the kernels of libgbmd.so.
//
// Layout in HBM (all arrays carved from the caller's workspace):
//   * Atoms live in "slots".  Replica r owns slots [slot0_r, slot0_r + n_r); slot0_r is a
//     multiple of TILE, so every tile of TILE slots belongs to exactly one replica and the tail
//     of a replica's last tile is padding.  One tile is the work unit of one CTA iteration.
//   * Positions used by the pair loops are cell-local: pos = (x - origin(cell), packed cell),
//     float4 for MD_MIXED/MD_FP32 and double4_32a for MD_FP64, double-buffered (read A, write B).
//     The cell coordinates (c_x, c_y, c_z) are packed as c_x | c_y << 10 | c_z << 20 in .w.
//     Cell-local coordinates keep FP32 pair distances at ~1e-7 absolute in any box size.
//   * MD_MIXED/MD_FP64 keep the master state in FP64 SoA streams: xl[3] (cell-local position)
//     and v[3].  MD_FP32 keeps pos (float4) and v32[3] as its master state.
//   * The neighbour matrix W is row-major, W[m * nslots + slot] (Sec. 2.3: the m-th neighbours of
//     consecutive atoms are adjacent, so the per-atom loop reads it coalesced).  An entry holds
//     (o_x+1) | (o_y+1) << 2 | (o_z+1) << 4 in bits 0..5 and the neighbour slot in bits 6..31,
//     o being the periodic offset of the neighbour's cell relative to the atom's cell.
//   * Cells are numbered globally: replica r's cells are cell0_r + row_pos(c_y, c_z) n_x + c_x,
//     the rows of cells in blocks of kz planes (row_pos below).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbmd.h"

namespace gbmd {

constexpr int TILE = 128;                 // slots per tile
constexpr int NPROP = 8;                  // U, K, W, px, py, pz, (spare), vmax^2
constexpr int SM_RANGES = 256;            // slot ranges of the step kernel's per-SM schedule
constexpr int SERIES_COLS = 9;            // step, U, K, W, P, px, py, pz, vmax
constexpr int IDX_SHIFT = 6;              // W entry: slot << 6 | (o_z+1) << 4 | (o_y+1) << 2 | (o_x+1)
constexpr int64_t MAX_SLOTS = int64_t(1) << 26;
constexpr int MAX_NC = 1023;
constexpr int SCAN_CHUNK = 2048;          // cells per block of the prefix sum
constexpr int PROPS_SPLIT_MAX = 2048;     // CTAs per replica in the first level of the final sums
constexpr int ADJ_VPART = 128;            // blocks of the |v_S|^2 partial sums

// entries of psort past the last atom, so that a build batch may read past a row's end
constexpr int PSORT_PAD = 8;

enum ErrBits { ERR_NBR_OVERFLOW = 1, ERR_NONFINITE = 2, ERR_TIMEOUT = 4 };

struct Rep {                  // per replica, fixed after creation
    int64_t slot0;            // first slot
    int32_t n;                // atoms
    int32_t tile0;            // first tile
    int32_t ntiles;
    int32_t cell0;            // first global cell id
    int32_t ncells;
    int32_t id0;              // first permanent id
    int32_t nc[3];            // cells per axis
    int32_t kz;               // z planes per block of the cell order, a power of two (1: rows in
                              // plain (z, y) order)
    double L[3];              // box sides
    double w[3];              // cell sides L / n_c
    double s[3];              // n_c / L
    float wf[3];              // (float) w
    float wlo[3];             // (float) (w - wf): the FP32 pair displacement adds o wf, then o wlo,
                              // so that the rounding of w does not bias every cross-cell distance
                              // of an axis the same way
    float pad2[2];
};

struct RepState {             // per replica, mutable on the device
    double D;                 // accumulated displacement bound (rule VMAX)
    unsigned int vmax2;       // max |v|^2 or |dx|^2 of this step, as float bits
    int32_t rebuild;          // 1: rebuild before the next force evaluation
    int32_t reorder;          // 1: the pending rebuild reorders too
    int32_t vhalf;            // 1: v holds v_{n-1/2}; 0: v holds v_n
    int32_t tiles_done;       // last-tile-done counter of the step kernel
    int32_t max_nbrs;         // max m_i at the last rebuild
    int32_t max_occ;          // max k_c at the last rebuild
    int32_t series_rows;      // rows written to the time series
    int64_t step;
    int64_t rebuilds;
    int64_t last_reorder;     // step of the last reorder
    int64_t sum_nbrs;         // sum m_i at the last rebuild
    int64_t reorders;         // reorders since creation or md_set_state
    int32_t props_done;       // CTAs of the props reduction that have stored their slice
    unsigned int pvmax2;      // props step (MD_MIXED / MD_FP32): max |v_n|^2, as float bits
    long long pacc[NPROP - 1];// props step: the sums in fixed point (2^-24), added by every warp
    double pbig[NPROP - 1];   // props step: warp sums too large for the fixed point (FP64 atomics)
};

struct Global {               // device-wide words
    int32_t any_rebuild;      // some replica needs a rebuild before the next force pass
    int32_t any_reorder;      // some rebuilding replica reorders
    int32_t err;              // ErrBits, latched
    int32_t max_nbr_seen;     // largest m_i that overflowed
    int32_t n_rb_tiles;       // entries of rb_tiles for the rebuild in progress
    int32_t pad;
    long long graph_rebuilds; // rebuild sequences that ran inside captured graphs
};

struct Arrays {
    // per slot
    float4* pos32[2];
    double4_32a* pos64[2];
    double* xl[3];
    double* v[3];
    float* v32[3];
    double4_32a* f;               // forces and u_i (md_compute_forces)
    double* wvir;             // per-atom virial sum_j r_ij . f_ij (md_compute_forces)
    int32_t* id;
    int32_t* slot_of_id;      // [n_total] the inverse of id (chain neighbours are found by id)
    int32_t* cell;
    int32_t* layer;
    int32_t* nbr_count;
    uint32_t* W;
    float4* xref;             // positions at the last rebuild (rule DISP)
    int32_t* perm;            // cell-ordered slots (the matrix H of Sec. 2.3, flattened)
    float4* psort;            // FP32 positions in cell order, slot in .w (MD_MIXED, MD_FP32)
    float4* fbuf;             // step kernel 5: FP32 force and u_i accumulated over the half list
    float* wbuf;              //   and the per-atom virial (zero between steps)
    float4* psub;             // FP32 positions sorted by half-side sub-cell, slot in .w (sub-cell build)
    int32_t* scount;          // per sub-cell (8 per cell): occupancy, then zero again after the scan
    int32_t* sstart;          // per sub-cell + 1: start in psub
    int32_t* schunk;          // per SCAN_CHUNK sub-cells
    int2* tile_win;           // [ntiles][9] slot window (lo, hi) of each tile's W entries per
                              // (o_y, o_z) row, periodic-wrap entries excluded (MD_MIXED, MD_FP32)
    // reorder scratch, per slot
    double* tmp_d[3];
    double* tmp_v[3];
    int32_t* tmp_i[2];
    float4* tmp_p32;
    double4_32a* tmp_p64;
    // per cell
    int32_t* ccount;
    int32_t* cstart;
    int2* ckeep;              // per cell: [start, end) in its replica's cell order at that replica's
                              // last rebuild (the list-free step kernel reads it every step; cstart
                              // is recomputed for all cells when any replica rebuilds)
    int32_t* chunk;           // per SCAN_CHUNK cells
    // per tile
    int32_t* tile_rep;
    int32_t* rb_tiles;        // tiles of the replicas rebuilding in this step
    int32_t* cell_rep;        // replica of every (global) cell
    int32_t* rb_base;         // per replica: its first entry in rb_tiles
    double* warp_part;        // NPROP per warp of every tile (32 slots): the props partials
    double* slice_part;       // NPROP per (replica, slice) of the final sums, props_split per replica
    // per replica
    Rep* rep;
    RepState* rs;
    md_props* props;          // per replica, output of the props reduction
    double* series;           // [nrep][series_cap][SERIES_COLS]
    Global* g;
    int32_t* sm_claim;        // [SM_RANGES] warp-tiles claimed per range in this step, then warps done
    // id-ordered exchange buffers (3 doubles per atom)
    double* xchg[3];
};

struct Scal {
    int64_t nslots;
    int32_t ntiles;
    int32_t nrep;
    int32_t ncells;
    int32_t nchunks;
    int32_t cap;              // rows of W
    int32_t mode;             // md_precision
    int32_t rule;             // md_rebuild_rule
    int32_t reorder_every;
    int32_t series_cap;
    int32_t shift;
    int32_t props_split;      // CTAs per replica of the props reduction (1..PROPS_SPLIT_MAX)
    int32_t half_list;        // 1: W keeps each pair once, at the lower slot (step kernel 5)
    int32_t chain_len;        // polymer chains (md_set_chains): atoms per chain, 0 = none
    float ch_kb, ch_r0sq, ch_ka, ch_kd;   // FENE stiffness, R0^2, bend and dihedral constants
    int64_t nsub;             // half-side sub-cells (8 per cell) of the sub-cell build
    int32_t nschunks;
    double dt, mass, c;       // c = dt / (2 m)
    double half_skin;
    double disp_margin;       // rounding margin of a displacement measured on FP32 positions
    double rc2d, rl2d, sig2d, eps4d, eps48d, ucd;
    float rc2f, rl2f, sig2f, eps4f, eps48f, ucf;
    float adj_eps144_over_sig, adj_eps24_over_sig, adj_ducf;   // sigma-derivative constants
};

// adjoint workspace (md_adjoint), carved from the caller's second buffer
struct AdjView {
    float4* pos_snap;         // [K+1][nslots] positions of the segment's steps
    int32_t* cnt_snap;        // [K+1][nslots] neighbour counts
    uint32_t* W_snap;         // [K+1][cap][nslots] neighbour matrices
    int32_t* id_snap;         // [nslots] permanent id of each slot during the segment
    double* lx[2][3];         // adjoint of positions, slot order, ping-pong
    double* lv[2][3];         // adjoint of velocities
    double* mu[2][3];         // kappa (lv + dt lx) of the reverse step that reads buffer b
    double* tile_acc;         // [ntiles][4] running sums of the parameter terms and the loss
    double* ck_x;             // [nseg+1][n][3] FP64 checkpoints, id order
    double* ck_v;
    double* lam_x;            // [n][3] adjoint state in id order between segments
    double* lam_v;
    double* vnorm_part;       // [ADJ_VPART]
    double* out;              // [8]
};

// velocity autocorrelation / mean-square displacement measurement (md_dyn_*), in the caller's
// buffer; per-atom arrays are indexed by permanent id
constexpr int DYN_MAX_ORG = 8;            // time origins followed at once
constexpr int DYN_BLOCKS = 1024;          // CTAs of the sample kernel (partial sums per CTA)
struct DynView {
    int64_t n;                // atoms (all replicas)
    double* xprev;            // [n][3] wrapped positions of the previous sample
    double* v0;               // [DYN_MAX_ORG][n][3] velocities at each origin
    double* dr;               // [DYN_MAX_ORG][n][3] displacements since each origin
    double* part;             // [DYN_BLOCKS][2 DYN_MAX_ORG] per-CTA sums of one sample
    double* vacf;             // [nlag] sums over origins and atoms
    double* msd;              // [nlag]
};
struct DynStep {              // one sample: which origin slot starts here, each slot's lag
    int norg;
    int start;                // slot whose origin is this sample (-1: none)
    int lag[DYN_MAX_ORG];     // lag of each slot at this sample, -1 when not followed
};

// ------------------------------------------------------------------------------------------
// small device helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_cell(int cx, int cy, int cz)
{
    return uint32_t(cx) | (uint32_t(cy) << 10) | (uint32_t(cz) << 20);
}

// Cell order.  Cells are numbered x fastest, so each row of cells (fixed y, z) is a contiguous
// run of the cell-ordered arrays.  The rows go in blocks of kz planes, ordered (z / kz, y, z % kz),
// so that a contiguous range of cells (and of slots, after a reorder) is compact along all three
// axes; kz = 1 is the plain (z, y) row order.  kz is a power of two, so the block of a plane is a
// shift (the build looks up 9 rows per atom).
__host__ __device__ __forceinline__ int row_pos(const Rep& R, int ny, int nz)
{
#ifdef __CUDA_ARCH__
    const int sh = __ffs(R.kz) - 1;
#else
    const int sh = __builtin_ffs(R.kz) - 1;
#endif
    const int z0 = (nz >> sh) << sh;
    const int hb = min(R.kz, R.nc[2] - z0);
    return z0 * R.nc[1] + ny * hb + (nz - z0);
}

__host__ __device__ __forceinline__ int cell_index(const Rep& R, int cx, int cy, int cz)
{
    return R.cell0 + row_pos(R, cy, cz) * R.nc[0] + cx;
}

// (cx, cy, cz) of the replica-local cell number cl
__host__ __device__ __forceinline__ void cell_coords(const Rep& R, int cl, int& cx, int& cy, int& cz)
{
    cx = cl % R.nc[0];
    const int p = cl / R.nc[0];
    const int z0 = (p / (R.kz * R.nc[1])) * R.kz;
    const int hb = min(R.kz, R.nc[2] - z0);
    const int rel = p - z0 * R.nc[1];
    cy = rel / hb;
    cz = z0 + rel % hb;
}

__device__ __forceinline__ void unpack_cell(uint32_t p, int& cx, int& cy, int& cz)
{
    cx = int(p & 1023u);
    cy = int((p >> 10) & 1023u);
    cz = int((p >> 20) & 1023u);
}

__device__ __forceinline__ uint32_t cell_bits(float w) { return __float_as_uint(w); }
__device__ __forceinline__ uint32_t cell_bits(double w) { return uint32_t(__double2uint_rz(w)); }
__device__ __forceinline__ float cell_word_f(uint32_t p) { return __uint_as_float(p); }
__device__ __forceinline__ double cell_word_d(uint32_t p) { return double(p); }

// FP32 <-> FP64 conversions (round to nearest even).  The hardware conversions issue to the FP64
// pipe (1/64 of the FP32 rate on GB300); versions that edit the IEEE-754 fields with 32-bit
// integer operations returned the same bits but made the step kernel 3.5 % slower (more issue
// slots for fewer FP64-pipe cycles, the FP64 pipe not being the bound), so these are the
// hardware ones.
__device__ __forceinline__ double f32_to_f64(float f) { return double(f); }
__device__ __forceinline__ float f64_to_f32(double x) { return __double2float_rn(x); }

// Warp-wide sums and maxima.
__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ float warp_max(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

__device__ __forceinline__ int warp_max_i(int x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

__device__ __forceinline__ long long warp_sum_ll(long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ------------------------------------------------------------------------------------------
// bulk asynchronous copies global -> shared (cp.async.bulk, the TMA engine's linear mode)
// completing on an mbarrier in shared memory
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes initialised mbarriers visible to the asynchronous proxy (the copy engine)
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// one arrival that also raises the transaction count the phase waits for by `bytes`
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of the given parity to complete, for one second at most; false if it
// gave up (the caller latches ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

// `bytes` (a multiple of 16) from global src to shared dst, both 16-byte aligned; completes as
// transactions on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// One stage of the step kernel's shared-memory ring: a tile's FP32 positions, its velocity
// (and, MD_MIXED, FP64 position) streams, its neighbour counts and `rows` rows of W.  Every
// offset is a multiple of 512 bytes.
struct StageLayout {
    uint32_t pos, xl, v, cnt, w, bytes;
};

__host__ __device__ inline StageLayout stage_layout(int mode, int rows)
{
    StageLayout L;
    uint32_t o = 0;
    L.pos = o;
    o += TILE * 16u;
    L.xl = o;
    if (mode == MD_MIXED) o += 3u * TILE * 8u;
    L.v = o;
    o += 3u * TILE * ((mode == MD_MIXED) ? 8u : 4u);
    L.cnt = o;
    o += TILE * 4u;
    L.w = o;
    o += uint32_t(rows) * TILE * 4u;
    L.bytes = o;
    return L;
}

// ------------------------------------------------------------------------------------------
// host-side launch wrappers (defined in the .cu files)
// ------------------------------------------------------------------------------------------
struct Launch {
    cudaStream_t stream;
    int grid;                 // persistent CTAs for tile loops
    int nsm;                  // SMs of the device
    int grid_step;            // persistent CTAs of the step kernel (capped at its occupancy)
    int step_block;
    int build_block;
    int nbr_batch;            // W entries loaded together per thread in the pair loop (2, 4, 8)
    int ctas_req;             // requested resident CTAs/SM (register bound of the step kernel)
    int build_stage;          // 1: the thread-per-atom builds stage their columns in shared memory
    int build_batch;          // candidates loaded together per thread in the build (2, 4; 32 = warp per cell;
                              // 1 = thread per atom over half-side sub-cells)
    int step_kernel;          // 1: per-thread loads with L2 prefetch; 2: bulk-copy shared-memory ring;
                              // 3: as 1, with each tile's neighbour positions staged in shared memory
    int bulk_rows;            // rows of W staged per tile by the ring (step_kernel 2)
    int bulk_smem;            // dynamic shared memory of the ring kernel, bytes
    int stage_cap;            // neighbour positions staged per tile (step_kernel 3)
    int stage_smem;           // dynamic shared memory of the staged step kernel, bytes
    cudaGraphConditionalHandle cond;   // IF node of the rebuild (inside a captured graph)
    int use_cond;             // 1 while capturing md_integrate into a graph
    int in_graph;             // 1 while capturing an IF-node body (counts rebuild sequences)
};

// records msg for md_last_error() on this thread and returns code (api.cu)
int set_last_error(int code, const char* msg);

// md_debug_set_error: ORs ErrBits into the device error word as a kernel meeting the condition
// would (kernels_step.cu)
cudaError_t launch_debug_error(const Arrays& A, const Launch& L, int bits, int nbr_seen);

// rebuild path (kernels_rebuild.cu)
cudaError_t launch_force_rebuild(const Arrays& A, const Scal& S, const Launch& L, int reorder);
void prime_rebuild_grids(const Scal& S, const Launch& L);
cudaError_t launch_rebuild(const Arrays& A, const Scal& S, const Launch& L, int cur, bool from_set);
cudaError_t launch_bin_only(const Arrays& A, const Scal& S, const Launch& L, int cur, bool from_set);
cudaError_t launch_bin_order(const Arrays& A, const Scal& S, const Launch& L, int cur, bool from_set);   // 7 kernels
cudaError_t launch_reorder(const Arrays& A, const Scal& S, const Launch& L, int cur);                    // 2 kernels
cudaError_t launch_build_only(const Arrays& A, const Scal& S, const Launch& L, int cur);                // 3 kernels
constexpr int REBUILD_KERNELS = 12;       // kernels of one rebuild sequence (bin/order 7, reorder 2, build 3)
int build_kernels(const Scal& S, const Launch& L);   // kernels of launch_build_only (2, 3 or 9)

// adjoint (kernels_adjoint.cu)
cudaError_t launch_adj_reverse(const Arrays& A, const Scal& S, const Launch& L, const AdjView& V, int q, double kappa,
                               double w_U, int in_buf, double kappa_next);
// to_slot: kappa is that of the segment's first reverse step (its mu is written)
cudaError_t launch_adj_permute(const Arrays& A, const Scal& S, const Launch& L, const AdjView& V, int buf, bool to_slot,
                               double kappa);
cudaError_t launch_adj_init(const AdjView& V, const Launch& L, int64_t n, const double* vS);
cudaError_t launch_adj_final(const AdjView& V, const Launch& L, int ntiles);

// measurement (kernels_dyn.cu): one VACF / MSD sample (the forces must be current)
cudaError_t launch_dyn_sample(const Arrays& A, const Scal& S, const Launch& L, const DynView& D, const DynStep& P,
                              int cur);

// step path (kernels_step.cu)
// launches per step without the props: the half-list pairs and the chain terms run before the step
inline int step_kernels(const Scal& S, const Launch& L)
{
    return (L.step_kernel == 5 ? 2 : 1) + ((S.chain_len && S.mode != MD_FP64) ? 1 : 0);
}
cudaError_t launch_step(const Arrays& A, const Scal& S, const Launch& L, int cur, bool props);
int step_ctas_per_sm(const Scal& S, const Launch& L);     // resident CTAs/SM of the chosen k_step
// rows of W and dynamic shared memory of the ring kernel for ctas_per_sm resident CTAs/SM
void bulk_shape(const Scal& S, int ctas_per_sm, int smem_per_sm, int smem_per_cta, int* rows, int* smem_bytes);
// neighbour positions staged per tile and dynamic shared memory of step kernel 3
void stage_shape(int ctas_per_sm, int smem_per_sm, int* cap, int* smem_bytes);
cudaError_t launch_forces(const Arrays& A, const Scal& S, const Launch& L, int cur);
cudaError_t launch_props(const Arrays& A, const Scal& S, const Launch& L, int cur, bool from_forces,
                         bool to_series);
cudaError_t launch_get_state(const Arrays& A, const Scal& S, const Launch& L, int cur, bool want_v,
                             bool want_f);
cudaError_t launch_set_state(const Arrays& A, const Scal& S, const Launch& L, int cur);
cudaError_t launch_get_cells(const Arrays& A, const Scal& S, const Launch& L, int32_t* out_by_id);
cudaError_t launch_get_neighbours(const Arrays& A, const Scal& S, const Launch& L, int32_t* counts_by_id,
                                  int32_t* nbr_by_id, int32_t cap_out, int64_t id_lo, int64_t id_hi);

}  // namespace gbmd
