// kernels_rebuild.cu -- cell binning, cell ordering, reordering and neighbour-matrix build.
//
// Sec. 2.3 of the paper lists the steps N1-N5; Sec. 2.4 item 4 the reorder vector s obtained
// there by a serial host pass over H and, as the GPU alternative it names, by a prefix sum of
// the cell occupancies k_c.  Here everything runs on the GPU:
//   k_bin          N1 + N2: cell of every atom from its FP64 position, layer l_i = atomic slot
//                  in the cell (the occupancy counter k_c); max k_c (N3) per replica.
//   k_scan_*       prefix sum of k_c -> cstart (the row offsets of H, Sec. 2.4 item 4).
//   k_scatter      N4: H flattened: perm[cstart[c] + l_i] = i.
//   k_sort_cells   the atomic layer order is indeterminate (Sec. 2.3 notes the resulting
//                  irreproducibility); sorting each cell's slots makes the order, and every
//                  result after it, deterministic.  It also writes psort, the FP32 positions in
//                  that order with each slot in .w, which the FP32 builds read.
//   k_reorder_*    Sec. 4.1 item 1: permute the atoms into cell order (gather through scratch).
//   k_build_sorted N5 in FP32: W from the 27 neighbouring cells, one thread per atom, each row of
//                  3 cells read as a contiguous run of psort; W stored row-major for coalescing
//                  (Sec. 4.1 item 6).  k_build_cw: the same W with one warp per cell (cells of
//                  tens of atoms).  k_build<double>: MD_FP64 through perm.
//   k_tile_windows the slot window of each tile's W entries per row of neighbour cells, read by
//                  the step kernel that stages neighbour positions (step kernel 3 only).
// Only replicas whose rebuild flag is set do work; kernels return at once when none is set, so
// the whole sequence can sit in every step of md_integrate.
#include <algorithm>

#include "gbmd_internal.cuh"

namespace gbmd {

// ------------------------------------------------------------------------------------------
// Per-replica statistics (N3: max occupancy; neighbour counts) are accumulated per thread over a
// CTA's contiguous run of tiles and folded in once per replica: one block reduction and one
// atomic, instead of an atomic per warp on the same address.  All threads of the CTA call this.
// ------------------------------------------------------------------------------------------
__device__ void flush_stats(int64_t* sum_dst, int* max_dst, long long sum, int mx)
{
    __shared__ long long sh_sum[TILE / 32];
    __shared__ int sh_max[TILE / 32];
    sum = warp_sum_ll(sum);
    mx = warp_max_i(mx);
    if ((threadIdx.x & 31) == 0) {
        sh_sum[threadIdx.x >> 5] = sum;
        sh_max[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        int m = 0;
        for (int w = 0; w < TILE / 32; ++w) { tot += sh_sum[w]; m = max(m, sh_max[w]); }
        if (sum_dst && tot) atomicAdd(reinterpret_cast<unsigned long long*>(sum_dst), static_cast<unsigned long long>(tot));
        if (max_dst && m > 0) atomicMax(max_dst, m);
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// The tiles of the replicas that rebuild in this step, listed contiguously so that the rebuild
// kernels share them evenly among their CTAs (in a batch only some replicas rebuild per step).
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_rebuild_list(Arrays A, Scal S)
{
    if (!A.g->any_rebuild) return;
    __shared__ int sh[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (int r0 = 0; r0 < S.nrep; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        const int v = (r < S.nrep && A.rs[r].rebuild) ? A.rep[r].ntiles : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) sh[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int wv = sh[lane];
            int wi = wv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            sh[lane] = wi - wv;
            if (lane == 31) sh[32] = wi;
        }
        __syncthreads();
        if (r < S.nrep) A.rb_base[r] = carry + sh[wid] + incl - v;
        carry += sh[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) A.g->n_rb_tiles = carry;
    // fill: replica by replica, all threads writing its consecutive tiles
    for (int r = 0; r < S.nrep; ++r) {
        if (!A.rs[r].rebuild) continue;
        const int base = A.rb_base[r], t0 = A.rep[r].tile0, nt = A.rep[r].ntiles;
        for (int k = threadIdx.x; k < nt; k += blockDim.x) A.rb_tiles[base + k] = t0 + k;
    }
}

// ------------------------------------------------------------------------------------------
// N1 + N2
// ------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(TILE) k_bin(Arrays A, Scal S, int cur, int from_set)
{
    if (!A.g->any_rebuild) return;
    const int nrb = A.g->n_rb_tiles;                  // tiles of the rebuilding replicas
    const int per = (nrb + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * per, t_end = min(nrb, t_begin + per);
    int run_r = -1, run_occ = 0;
    for (int it = t_begin; it < t_end; ++it) {
        const int t = A.rb_tiles[it];
        const int r = A.tile_rep[t];
        if (r != run_r) {
            if (run_r >= 0) flush_stats(nullptr, &A.rs[run_r].max_occ, 0, run_occ);
            run_r = r;
            run_occ = 0;
        }
        const Rep& R = A.rep[r];
        if (t == R.tile0 && threadIdx.x == 0) {
            A.rs[r].sum_nbrs = 0;
            A.rs[r].max_nbrs = 0;
        }
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const int64_t j = slot - R.slot0;
        int occ = 0;
        int cell_bin = -1;            // this lane's cell, -1 for padding slots
        if (j < R.n && from_set) {
            // exact binning of a global position (the definition the oracle follows):
            // wrap into [0, L), c = floor(x n_c / L) clamped, local = x - c w, all in FP64
            double x[3] = {A.xl[0][slot], A.xl[1][slot], A.xl[2][slot]};
            int c[3];
            double loc[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double xa = x[a];
                if (!isfinite(xa)) {                  // reported; the atom goes to cell 0
                    atomicOr(&A.g->err, ERR_NONFINITE);
                    xa = 0.0;
                }
                if (xa < 0.0) xa = __dadd_rn(xa, R.L[a]);
                if (xa >= R.L[a]) xa = __dsub_rn(xa, R.L[a]);
                if (!(xa >= 0.0 && xa < R.L[a])) {    // more than one period away: whole periods
                    xa = __dsub_rn(xa, __dmul_rn(R.L[a], floor(xa / R.L[a])));
                    if (xa < 0.0) xa = __dadd_rn(xa, R.L[a]);
                    if (xa >= R.L[a]) xa = __dsub_rn(xa, R.L[a]);
                }
                int ca = int(floor(__dmul_rn(xa, R.s[a])));
                ca = min(max(ca, 0), R.nc[a] - 1);
                c[a] = ca;
                loc[a] = __dsub_rn(xa, __dmul_rn(double(ca), R.w[a]));
            }
            const uint32_t packed = pack_cell(c[0], c[1], c[2]);
            if (MODE == MD_FP64) {
                A.pos64[cur][slot] = make_double4_32a(loc[0], loc[1], loc[2], cell_word_d(packed));
            } else {
                A.pos32[cur][slot] = make_float4(__double2float_rn(loc[0]), __double2float_rn(loc[1]),
                                                 __double2float_rn(loc[2]), cell_word_f(packed));
            }
            if (MODE != MD_FP32) {
                A.xl[0][slot] = loc[0]; A.xl[1][slot] = loc[1]; A.xl[2][slot] = loc[2];
            }
            const int cell = cell_index(R, c[0], c[1], c[2]);
            A.cell[slot] = cell;
            cell_bin = cell;
        } else if (j < R.n) {
            // during a run every atom is within skin/2 < w of its cell: it stays or moves to the
            // adjacent cell along each axis; its local coordinate shifts by -s w (s in -1, 0, 1)
            int c[3], sh[3];
            bool moved = false;
            if (MODE == MD_FP64) {
                const double4_32a p = A.pos64[cur][slot];
                unpack_cell(cell_bits(p.w), c[0], c[1], c[2]);
                const double l[3] = {p.x, p.y, p.z};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    sh[a] = (l[a] < 0.0) ? -1 : ((l[a] >= R.w[a]) ? 1 : 0);
                    moved |= sh[a] != 0;
                    if (!(l[a] >= -R.w[a] && l[a] < 2.0 * R.w[a])) atomicOr(&A.g->err, ERR_NONFINITE);
                }
                if (moved) {
                    double nl[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        nl[a] = sh[a] ? __dsub_rn(l[a], double(sh[a]) * R.w[a]) : l[a];
                        int ca = c[a] + sh[a];
                        ca += (ca < 0) ? R.nc[a] : 0;
                        ca -= (ca >= R.nc[a]) ? R.nc[a] : 0;
                        c[a] = ca;
                        A.xl[a][slot] = nl[a];
                    }
                    A.pos64[cur][slot] = make_double4_32a(nl[0], nl[1], nl[2], cell_word_d(pack_cell(c[0], c[1], c[2])));
                }
            } else {
                const float4 p = A.pos32[cur][slot];
                unpack_cell(__float_as_uint(p.w), c[0], c[1], c[2]);
                const float l[3] = {p.x, p.y, p.z};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    sh[a] = (l[a] < 0.0f) ? -1 : ((l[a] >= R.wf[a]) ? 1 : 0);
                    moved |= sh[a] != 0;
                    if (!(l[a] >= -R.wf[a] && l[a] < 2.0f * R.wf[a])) atomicOr(&A.g->err, ERR_NONFINITE);
                }
                if (moved) {
                    float nl[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (MODE == MD_MIXED) {
                            const double x = sh[a] ? __dsub_rn(A.xl[a][slot], double(sh[a]) * R.w[a]) : A.xl[a][slot];
                            if (sh[a]) A.xl[a][slot] = x;
                            nl[a] = __double2float_rn(x);
                        } else {
                            nl[a] = sh[a] ? __fsub_rn(l[a], float(sh[a]) * R.wf[a]) : l[a];
                        }
                        int ca = c[a] + sh[a];
                        ca += (ca < 0) ? R.nc[a] : 0;
                        ca -= (ca >= R.nc[a]) ? R.nc[a] : 0;
                        c[a] = ca;
                    }
                    A.pos32[cur][slot] = make_float4(nl[0], nl[1], nl[2], cell_word_f(pack_cell(c[0], c[1], c[2])));
                }
            }
            const int cell = cell_index(R, c[0], c[1], c[2]);
            if (moved) A.cell[slot] = cell;
            cell_bin = cell;
        }
        // N2 layer slots: lanes of a warp that share a cell (common, the atoms are cell-sorted)
        // take consecutive layers from one atomic on the cell's counter
        {
            const unsigned peers = __match_any_sync(0xffffffffu, cell_bin);
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(peers) - 1;
            const int rank = __popc(peers & ((1u << lane) - 1u));
            int base = 0;
            if (cell_bin >= 0 && lane == leader) base = atomicAdd(&A.ccount[cell_bin], __popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (cell_bin >= 0) {
                A.layer[slot] = base + rank;
                occ = base + rank + 1;
            }
        }
        run_occ = max(run_occ, occ);
    }
    if (run_r >= 0) flush_stats(nullptr, &A.rs[run_r].max_occ, 0, run_occ);
}

// ------------------------------------------------------------------------------------------
// prefix sum of the cell occupancies (three passes, no inter-block waiting)
// ------------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER_THREAD = SCAN_CHUNK / SCAN_THREADS;

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh_warp, int& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (blockDim.x >> 5)) ? sh_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (blockDim.x >> 5)) sh_warp[lane] = wi - w;
        if (lane == (blockDim.x >> 5) - 1) sh_warp[32] = wi;
    }
    __syncthreads();
    total = sh_warp[32];
    const int r = sh_warp[wid] + incl - v;
    __syncthreads();
    return r;
}

// The scan of n counters `count` into `start` (n + 1 entries), through per-chunk totals in
// `chunk`; the counters are left at zero for the next binning.  Serves the cells and the half-side
// sub-cells of the sub-cell neighbour build.
struct ScanArgs {
    int32_t* count;
    int32_t* start;
    int32_t* chunk;
    int64_t n;
    int32_t nchunks;
};

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_chunks(Arrays A, ScanArgs C)
{
    if (!A.g->any_rebuild) return;
    __shared__ int sh[33];
    const int64_t base = int64_t(blockIdx.x) * SCAN_CHUNK + threadIdx.x * SCAN_PER_THREAD;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        const int64_t c = base + k;
        if (c < C.n) s += C.count[c];
    }
    int total;
    block_exclusive_scan(s, sh, total);
    if (threadIdx.x == 0) C.chunk[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(Arrays A, ScanArgs C)
{
    if (!A.g->any_rebuild) return;
    __shared__ int sh[33];
    int carry = 0;
    for (int b0 = 0; b0 < C.nchunks; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const int v = (b < C.nchunks) ? C.chunk[b] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sh, total);
        if (b < C.nchunks) C.chunk[b] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(Arrays A, ScanArgs C)
{
    if (!A.g->any_rebuild) return;
    __shared__ int sh[33];
    const int64_t base = int64_t(blockIdx.x) * SCAN_CHUNK + threadIdx.x * SCAN_PER_THREAD;
    int v[SCAN_PER_THREAD];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        const int64_t c = base + k;
        v[k] = (c < C.n) ? C.count[c] : 0;
        s += v[k];
    }
    int total;
    int run = C.chunk[blockIdx.x] + block_exclusive_scan(s, sh, total);
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        const int64_t c = base + k;
        if (c < C.n) {
            C.start[c] = run;
            C.count[c] = 0;               // ready for the next binning
            run += v[k];
            if (c == C.n - 1) C.start[C.n] = run;
        }
    }
}

static void launch_scan(const Arrays& A, const ScanArgs& C, cudaStream_t st)
{
    k_scan_chunks<<<C.nchunks, SCAN_THREADS, 0, st>>>(A, C);
    k_scan_top<<<1, 1024, 0, st>>>(A, C);
    k_scan_apply<<<C.nchunks, SCAN_THREADS, 0, st>>>(A, C);
}

// ------------------------------------------------------------------------------------------
// N4 and the deterministic order within cells
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE) k_scatter(Arrays A, Scal S)
{
    if (!A.g->any_rebuild) return;
    const int nrb = A.g->n_rb_tiles;
    for (int it = blockIdx.x; it < nrb; it += gridDim.x) {
        const int t = A.rb_tiles[it];
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 < R.n) A.perm[A.cstart[A.cell[slot]] + A.layer[slot]] = int32_t(slot);
    }
}

__global__ void __launch_bounds__(256) k_sort_cells(Arrays A, Scal S, int cur)
{
    if (!A.g->any_rebuild) return;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < S.ncells;
         c += int64_t(gridDim.x) * blockDim.x) {
        const int b = A.cstart[c], e = A.cstart[c + 1];
        for (int k = b + 1; k < e; ++k) {            // insertion sort, cells hold a few atoms
            const int32_t key = A.perm[k];
            int q = k - 1;
            while (q >= b && A.perm[q] > key) {
                A.perm[q + 1] = A.perm[q];
                --q;
            }
            A.perm[q + 1] = key;
        }
        if (A.ckeep && A.rs[A.cell_rep[c]].rebuild) {
            const int base = A.cstart[A.rep[A.cell_rep[c]].cell0];
            A.ckeep[c] = make_int2(b - base, e - base);
        }
        // the cell-ordered copy of the FP32 positions read by the neighbour build, slot in .w
        if (A.psort && A.rs[A.cell_rep[c]].rebuild) {
            const float4* __restrict__ pos = A.pos32[cur];
            for (int k = b; k < e; ++k) {
                const int32_t j = A.perm[k];
                const float4 p = pos[j];
                A.psort[k] = make_float4(p.x, p.y, p.z, __int_as_float(j));
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// reorder (Sec. 4.1 item 1): new slot slot0 + j takes the j-th atom in cell order
// ------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(TILE) k_reorder_gather(Arrays A, Scal S, int cur)
{
    if (!A.g->any_reorder) return;
    const int nrb = A.g->n_rb_tiles;
    for (int it = blockIdx.x; it < nrb; it += gridDim.x) {
        const int t = A.rb_tiles[it];
        const int r = A.tile_rep[t];
        if (!A.rs[r].reorder) continue;
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const int64_t j = slot - R.slot0;
        if (j >= R.n) continue;
        const int32_t src = A.perm[A.cstart[R.cell0] + j];
        if (MODE == MD_FP32) {
            A.tmp_p32[slot] = A.pos32[cur][src];
            for (int a = 0; a < 3; ++a) A.tmp_v[a][slot] = double(A.v32[a][src]);
        } else {
            if (MODE == MD_FP64) A.tmp_p64[slot] = A.pos64[cur][src];
            else A.tmp_p32[slot] = A.pos32[cur][src];
            for (int a = 0; a < 3; ++a) {
                A.tmp_d[a][slot] = A.xl[a][src];
                A.tmp_v[a][slot] = A.v[a][src];
            }
        }
        A.tmp_i[0][slot] = A.id[src];
        A.tmp_i[1][slot] = A.cell[src];
    }
}

template <int MODE>
__global__ void __launch_bounds__(TILE) k_reorder_copy(Arrays A, Scal S, int cur)
{
    if (!A.g->any_reorder) return;
    const int nrb = A.g->n_rb_tiles;
    for (int it = blockIdx.x; it < nrb; it += gridDim.x) {
        const int t = A.rb_tiles[it];
        const int r = A.tile_rep[t];
        if (!A.rs[r].reorder) continue;
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const int64_t j = slot - R.slot0;
        if (j >= R.n) continue;
        if (MODE == MD_FP32) {
            A.pos32[cur][slot] = A.tmp_p32[slot];
            for (int a = 0; a < 3; ++a) A.v32[a][slot] = float(A.tmp_v[a][slot]);
        } else {
            if (MODE == MD_FP64) A.pos64[cur][slot] = A.tmp_p64[slot];
            else A.pos32[cur][slot] = A.tmp_p32[slot];
            for (int a = 0; a < 3; ++a) {
                A.xl[a][slot] = A.tmp_d[a][slot];
                A.v[a][slot] = A.tmp_v[a][slot];
            }
        }
        A.id[slot] = A.tmp_i[0][slot];
        A.slot_of_id[A.tmp_i[0][slot]] = int32_t(slot);
        A.cell[slot] = A.tmp_i[1][slot];
        const int k = A.cstart[R.cell0] + int(j);
        A.perm[k] = int32_t(slot);
        if (MODE != MD_FP64) reinterpret_cast<float*>(A.psort + k)[3] = __int_as_float(int(slot));
    }
}

// ------------------------------------------------------------------------------------------
// N5: neighbour matrix.  Criterion (exact, shared with nothing): with lf the cell-local
// coordinates and o the periodic cell offset, d = (lf_j - lf_i) + o * wf (two roundings),
// r2 = fma(d_z, d_z, fma(d_y, d_y, d_x * d_x)), neighbour iff r2 < (r_c + skin)^2.
// ------------------------------------------------------------------------------------------
template <typename T> struct PosT;
template <> struct PosT<float> { using type = float4; };
template <> struct PosT<double> { using type = double4_32a; };

__device__ __forceinline__ uint32_t word_of(const float4& p) { return __float_as_uint(p.w); }
__device__ __forceinline__ uint32_t word_of(const double4_32a& p) { return cell_bits(p.w); }

__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T, int BB>
__global__ void __launch_bounds__(TILE) k_build(Arrays A, Scal S, int cur)
{
    using P4 = typename PosT<T>::type;
    if (!A.g->any_rebuild) return;
    const P4* __restrict__ pos = nullptr;
    if constexpr (sizeof(T) == 8) pos = reinterpret_cast<const P4*>(A.pos64[cur]);
    else pos = reinterpret_cast<const P4*>(A.pos32[cur]);
    const T rl2 = (sizeof(T) == 8) ? T(S.rl2d) : T(S.rl2f);
    const int nrb = A.g->n_rb_tiles;                  // tiles of the rebuilding replicas
    const int per = (nrb + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * per, t_end = min(nrb, t_begin + per);
    int run_r = -1, run_max = 0;
    long long run_sum = 0;
    for (int it = t_begin; it < t_end; ++it) {
        const int t = A.rb_tiles[it];
        const int r = A.tile_rep[t];
        if (r != run_r) {
            if (run_r >= 0) flush_stats(&A.rs[run_r].sum_nbrs, &A.rs[run_r].max_nbrs, run_sum, run_max);
            run_r = r;
            run_sum = 0;
            run_max = 0;
        }
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const bool active = slot - R.slot0 < R.n;
        int m = 0;
        if (active) {
            const P4 pi = pos[slot];
            int cx, cy, cz;
            unpack_cell(word_of(pi), cx, cy, cz);
            T w[3];
            if constexpr (sizeof(T) == 8) { w[0] = R.w[0]; w[1] = R.w[1]; w[2] = R.w[2]; }
            else { w[0] = R.wf[0]; w[1] = R.wf[1]; w[2] = R.wf[2]; }
            const int xm = (cx == 0) ? R.nc[0] - 1 : cx - 1;
            const int xp = (cx == R.nc[0] - 1) ? 0 : cx + 1;
            uint32_t* wp = A.W + slot;         // next free entry of this atom's column of W
            // Squared distance from the atom to the lower and upper faces of its cell, per axis:
            // a neighbouring cell whose nearest point is farther than r_c + skin cannot hold a
            // neighbour.  The relative margin keeps this strictly looser than the criterion below.
            const T lc[3] = {pi.x, pi.y, pi.z};
            T dlo2[3], dhi2[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dlo2[a] = lc[a] * lc[a];
                dhi2[a] = (w[a] - lc[a]) * (w[a] - lc[a]);
            }
            const T skip2 = rl2 * ((sizeof(T) == 8) ? T(1.0 + 1e-12) : T(1.0f + 1e-5f));
            for (int oz = -1; oz <= 1; ++oz) {
                int nz = cz + oz; nz += (nz < 0) ? R.nc[2] : 0; nz -= (nz >= R.nc[2]) ? R.nc[2] : 0;
                const T offz = T(oz) * w[2];
                for (int oy = -1; oy <= 1; ++oy) {
                    int ny = cy + oy; ny += (ny < 0) ? R.nc[1] : 0; ny -= (ny >= R.nc[1]) ? R.nc[1] : 0;
                    const T offy = T(oy) * w[1];
                    const T dyz = ((oy < 0) ? dlo2[1] : ((oy > 0) ? dhi2[1] : T(0))) +
                                  ((oz < 0) ? dlo2[2] : ((oz > 0) ? dhi2[2] : T(0)));
                    if (dyz > skip2) continue;
                    const bool use_l = dyz + dlo2[0] <= skip2, use_r = dyz + dhi2[0] <= skip2;
                    const int row = R.cell0 + row_pos(R, ny, nz) * R.nc[0];
                    const uint32_t codeyz = (uint32_t(oy + 1) << 2) | (uint32_t(oz + 1) << 4);
                    // the three cells of this row, as [b0,e0) [b1,e1) [b2,e2) in perm; without a
                    // periodic wrap in x they are one contiguous range [b0, e2) split at b1, b2
                    const int b0 = A.cstart[row + xm], e0 = use_l ? A.cstart[row + xm + 1] : b0;
                    const int b1 = A.cstart[row + cx], e1 = A.cstart[row + cx + 1];
                    const int b2 = A.cstart[row + xp], e2 = use_r ? A.cstart[row + xp + 1] : b2;
                    if (cx > 0 && cx < R.nc[0] - 1) {
                        // consecutive cells: one range, starting past the left cell if it is skipped
                        const int kb = use_l ? b0 : b1;
                        for (int k0 = kb; k0 < e2; k0 += BB) {
                            int32_t js[BB];
#pragma unroll
                            for (int u = 0; u < BB; ++u) js[u] = A.perm[min(k0 + u, e2 - 1)];
                            P4 pj[BB];
#pragma unroll
                            for (int u = 0; u < BB; ++u) pj[u] = pos[js[u]];
#pragma unroll
                            for (int u = 0; u < BB; ++u) {
                                const int k = k0 + u;
                                const int ox = int(k >= b1) + int(k >= b2) - 1;
                                const T offx = (ox < 0) ? -w[0] : ((ox > 0) ? w[0] : T(0));
                                const T dx = add_rn(sub_rn(pj[u].x, pi.x), offx);
                                const T dy = add_rn(sub_rn(pj[u].y, pi.y), offy);
                                const T dz = add_rn(sub_rn(pj[u].z, pi.z), offz);
                                const T r2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
                                if (k < e2 && r2 < rl2 && js[u] != slot) {
                                    if (m < S.cap) {
                                        *wp = (uint32_t(js[u]) << IDX_SHIFT) | codeyz | uint32_t(ox + 1);
                                        wp += S.nslots;
                                    }
                                    ++m;
                                }
                            }
                        }
                        continue;
                    }
                    const int n0 = e0 - b0, n01 = n0 + (e1 - b1), ntot = n01 + (e2 - b2);
                    for (int q0 = 0; q0 < ntot; q0 += BB) {
                        int32_t js[BB];
#pragma unroll
                        for (int u = 0; u < BB; ++u) {
                            const int q = q0 + u;
                            const int k = (q < n0) ? b0 + q : ((q < n01) ? b1 + (q - n0) : b2 + (q - n01));
                            js[u] = (q < ntot) ? A.perm[k] : -1;
                        }
                        P4 pj[BB];
#pragma unroll
                        for (int u = 0; u < BB; ++u) pj[u] = (js[u] >= 0) ? pos[js[u]] : pi;
#pragma unroll
                        for (int u = 0; u < BB; ++u) {
                            const int q = q0 + u;
                            if (js[u] < 0 || js[u] == slot) continue;
                            const int ox = (q < n0) ? -1 : ((q < n01) ? 0 : 1);
                            const T offx = T(ox) * w[0];
                            const T dx = add_rn(sub_rn(pj[u].x, pi.x), offx);
                            const T dy = add_rn(sub_rn(pj[u].y, pi.y), offy);
                            const T dz = add_rn(sub_rn(pj[u].z, pi.z), offz);
                            const T r2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
                            if (r2 < rl2) {
                                if (m < S.cap) {
                                    *wp = (uint32_t(js[u]) << IDX_SHIFT) | codeyz | uint32_t(ox + 1);
                                    wp += S.nslots;
                                }
                                ++m;
                            }
                        }
                    }
                }
            }
            A.nbr_count[slot] = m;
            if (S.rule == MD_REBUILD_DISP) {
                A.xref[slot] = make_float4(float(pi.x), float(pi.y), float(pi.z), 0.0f);
            }
            if (m > S.cap) {
                atomicOr(&A.g->err, ERR_NBR_OVERFLOW);
                atomicMax(&A.g->max_nbr_seen, m);
            }
        }
        if (active) {
            run_sum += m;
            run_max = max(run_max, m);
        }
    }
    if (run_r >= 0) flush_stats(&A.rs[run_r].sum_nbrs, &A.rs[run_r].max_nbrs, run_sum, run_max);
}


// N5 in FP32 from the cell-ordered copy of the positions: psort[k] is the k-th atom of the cell
// order (the order of perm) with its slot in .w, so the candidates of a 3-cell row are one
// contiguous run of psort (three separate runs at a periodic wrap in x), read in order with no
// load through perm.  x and y of a candidate are adjacent in its float4 and go through packed
// FP32x2 adds; each lane rounds as the scalar criterion does (a - b is a + (-b)), and the rows,
// cells and candidates are visited in k_build's order, so W is entry for entry k_build's.
// With half = 1 (the half list of step kernel 5) only partners of a higher slot are kept: the
// criterion is exactly antisymmetric in i and j (IEEE subtraction and negation), so every pair
// is kept once.
__device__ __forceinline__ void nbr_test(const float4& p, const float2& npxy, float npz, float offx, float offy,
                                         float offz, bool valid, uint32_t code, int me, float rl2, uint32_t*& wp,
                                         int& m, int cap, int64_t stride, int half)
{
    const float2 dxy = __fadd2_rn(__fadd2_rn(make_float2(p.x, p.y), npxy), make_float2(offx, offy));
    const float dz = __fadd_rn(__fadd_rn(p.z, npz), offz);
    const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dxy.y, dxy.y, __fmul_rn(dxy.x, dxy.x)));
    const int j = __float_as_int(p.w);
    if (valid && r2 < rl2 && (half ? j > me : j != me)) {
        if (m < cap) {
            *wp = (uint32_t(j) << IDX_SHIFT) | code;
            wp += stride;
        }
        ++m;
    }
}

// The order in which a CTA of a neighbour build takes the rebuild tiles: chunks of BUILD_CHUNK
// consecutive tiles dealt to the CTAs in turn, so that the CTAs resident at one time work on one
// stretch of consecutive slots (grid x BUILD_CHUNK tiles) and the candidate rows they read stay
// in L2; contiguous runs per CTA spread them over the whole system (measured in the build A/B).
constexpr int BUILD_CHUNK = 4;
#define build_tile(q) ((((q) / BUILD_CHUNK) * int(gridDim.x) + int(blockIdx.x)) * BUILD_CHUNK + (q) % BUILD_CHUNK)

// Two candidates of a row in one pass of packed FP32x2 operations (candidate a in lane x, b in
// lane y); each lane rounds as nbr_test does, and a is appended before b, so W is the same entry
// for entry.
__device__ __forceinline__ void nbr_test2(const float4& pa, const float4& pb, float2 nx, float2 ny, float2 nz,
                                          float2 offx, float offy, float offz, bool va, bool vb, uint32_t ca,
                                          uint32_t cb, int me, float rl2, uint32_t*& wp, int& m, int cap,
                                          int64_t stride, int half)
{
    const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(pa.x, pb.x), nx), offx);
    const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(pa.y, pb.y), ny), make_float2(offy, offy));
    const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(pa.z, pb.z), nz), make_float2(offz, offz));
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const int ja = __float_as_int(pa.w), jb = __float_as_int(pb.w);
    if (va && r2.x < rl2 && (half ? ja > me : ja != me)) {
        if (m < cap) {
            *wp = (uint32_t(ja) << IDX_SHIFT) | ca;
            wp += stride;
        }
        ++m;
    }
    if (vb && r2.y < rl2 && (half ? jb > me : jb != me)) {
        if (m < cap) {
            *wp = (uint32_t(jb) << IDX_SHIFT) | cb;
            wp += stride;
        }
        ++m;
    }
}

// STAGE: a thread appends its column of W to shared memory (stride TILE) instead of W itself,
// and each warp then writes its columns row by row: 32 consecutive slots of a row are 128
// contiguous bytes, where entries written as found land one at a time in partly written sectors.
// Every thread reads back only its own column, so no block barrier is needed.
__device__ __forceinline__ void flush_columns(const Arrays& A, const Scal& S, const uint32_t* sW, int64_t slot, int mc)
{
    const int mw = int(__reduce_max_sync(0xffffffffu, unsigned(mc)));
    for (int q = 0; q < mw; ++q)
        if (q < mc) A.W[int64_t(q) * S.nslots + slot] = sW[q * TILE + threadIdx.x];
}

template <int BB, bool STAGE>
__global__ void __launch_bounds__(TILE) k_build_sorted(Arrays A, Scal S, int cur)
{
    static_assert(BB % 2 == 0, "candidates are tested in pairs");
    extern __shared__ uint32_t sW[];                 // STAGE: [cap][TILE] columns of this tile
    if (!A.g->any_rebuild) return;
    const int64_t wstride = STAGE ? int64_t(TILE) : S.nslots;
    const float4* __restrict__ pos = A.pos32[cur];
    const float4* __restrict__ ps = A.psort;
    const int32_t* __restrict__ cs = A.cstart;
    const float rl2 = S.rl2f;
    const float skip2 = rl2 * (1.0f + 1e-5f);
    const int nrb = A.g->n_rb_tiles;
    int run_r = -1, run_max = 0;
    long long run_sum = 0;
    for (int q = 0;; ++q) {
        const int it = build_tile(q);
        if (it >= nrb) break;
        const int t = A.rb_tiles[it];
        const int r = A.tile_rep[t];
        if (r != run_r) {
            if (run_r >= 0) flush_stats(&A.rs[run_r].sum_nbrs, &A.rs[run_r].max_nbrs, run_sum, run_max);
            run_r = r;
            run_sum = 0;
            run_max = 0;
        }
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const bool active = slot - R.slot0 < R.n;
        int m = 0;
        if (active) {
            const float4 pi = pos[slot];
            int cx, cy, cz;
            unpack_cell(__float_as_uint(pi.w), cx, cy, cz);
            const float w0 = R.wf[0], w1 = R.wf[1], w2 = R.wf[2];
            const int ncx = R.nc[0];
            const bool inner = cx > 0 && cx < ncx - 1;
            const int me = int(slot);
            uint32_t* wp = STAGE ? sW + threadIdx.x : A.W + slot;
            // neighbouring cells whose nearest point is beyond r_c + skin are skipped (as k_build)
            const float dlo2[3] = {pi.x * pi.x, pi.y * pi.y, pi.z * pi.z};
            const float dhi2[3] = {(w0 - pi.x) * (w0 - pi.x), (w1 - pi.y) * (w1 - pi.y), (w2 - pi.z) * (w2 - pi.z)};
            const float2 npxy = make_float2(-pi.x, -pi.y);
            const float npz = -pi.z;
            const float2 nx2 = make_float2(-pi.x, -pi.x), ny2 = make_float2(-pi.y, -pi.y), nz2 = make_float2(-pi.z, -pi.z);
            for (int oz = -1; oz <= 1; ++oz) {
                int nz = cz + oz; nz += (nz < 0) ? R.nc[2] : 0; nz -= (nz >= R.nc[2]) ? R.nc[2] : 0;
                const float offz = float(oz) * w2;
                for (int oy = -1; oy <= 1; ++oy) {
                    int ny = cy + oy; ny += (ny < 0) ? R.nc[1] : 0; ny -= (ny >= R.nc[1]) ? R.nc[1] : 0;
                    const float offy = float(oy) * w1;
                    const float dyz = ((oy < 0) ? dlo2[1] : ((oy > 0) ? dhi2[1] : 0.0f)) +
                                      ((oz < 0) ? dlo2[2] : ((oz > 0) ? dhi2[2] : 0.0f));
                    if (dyz > skip2) continue;
                    const bool use_l = dyz + dlo2[0] <= skip2, use_r = dyz + dhi2[0] <= skip2;
                    const int row = R.cell0 + row_pos(R, ny, nz) * ncx;
                    const uint32_t codeyz = (uint32_t(oy + 1) << 2) | (uint32_t(oz + 1) << 4);
                    if (inner) {
                        // cells cx-1, cx, cx+1 are adjacent runs [b0,b1) [b1,b2) [b2,b3) of psort
                        const int b0 = cs[row + cx - 1], b1 = cs[row + cx], b2 = cs[row + cx + 1];
                        const int kb = use_l ? b0 : b1;
                        const int ke = use_r ? cs[row + cx + 2] : b2;
                        // psort has PSORT_PAD entries past its end, so the last batch reads
                        // past ke unclamped (those lanes are invalid)
                        for (int k0 = kb; k0 < ke; k0 += BB) {
                            float4 pj[BB];
#pragma unroll
                            for (int u = 0; u < BB; ++u) pj[u] = ps[k0 + u];
#pragma unroll
                            for (int u = 0; u < BB; u += 2) {
                                const int ka = k0 + u, kb2 = ka + 1;
                                const uint32_t ca = uint32_t(ka >= b1) + uint32_t(ka >= b2);   // o_x + 1
                                const uint32_t cb = uint32_t(kb2 >= b1) + uint32_t(kb2 >= b2);
                                const float2 offx = make_float2((ka < b1) ? -w0 : ((ka < b2) ? 0.0f : w0),
                                                                (kb2 < b1) ? -w0 : ((kb2 < b2) ? 0.0f : w0));
                                nbr_test2(pj[u], pj[u + 1], nx2, ny2, nz2, offx, offy, offz, ka < ke, kb2 < ke,
                                          codeyz | ca, codeyz | cb, me, rl2, wp, m, S.cap, wstride, S.half_list);
                            }
                        }
                    } else {
                        // a periodic wrap in x: the three cells are separate runs, in the same order
                        const int xs[3] = {(cx == 0) ? ncx - 1 : cx - 1, cx, (cx == ncx - 1) ? 0 : cx + 1};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            if ((c == 0 && !use_l) || (c == 2 && !use_r)) continue;
                            const int b = cs[row + xs[c]], e = cs[row + xs[c] + 1];
                            const float offx = float(c - 1) * w0;
                            for (int k0 = b; k0 < e; k0 += BB) {
                                float4 pj[BB];
#pragma unroll
                                for (int u = 0; u < BB; ++u) pj[u] = ps[min(k0 + u, e - 1)];
#pragma unroll
                                for (int u = 0; u < BB; ++u)
                                    nbr_test(pj[u], npxy, npz, offx, offy, offz, k0 + u < e, codeyz | uint32_t(c), me,
                                             rl2, wp, m, S.cap, wstride, S.half_list);
                            }
                        }
                    }
                }
            }
            A.nbr_count[slot] = m;
            if (S.rule == MD_REBUILD_DISP) A.xref[slot] = make_float4(pi.x, pi.y, pi.z, 0.0f);
            if (m > S.cap) {
                atomicOr(&A.g->err, ERR_NBR_OVERFLOW);
                atomicMax(&A.g->max_nbr_seen, m);
            }
            run_sum += m;
            run_max = max(run_max, m);
        }
        if (STAGE) flush_columns(A, S, sW, slot, active ? min(m, S.cap) : 0);
    }
    if (run_r >= 0) flush_stats(&A.rs[run_r].sum_nbrs, &A.rs[run_r].max_nbrs, run_sum, run_max);
}

// ------------------------------------------------------------------------------------------
// N5 over half-side sub-cells.  Every cell of side w >= r_c + skin is split into 2 x 2 x 2
// sub-cells of side w / 2 (an atom's sub-cell along an axis is 2 c + (l >= w / 2)), and the atoms
// are counting-sorted by sub-cell into psub (rows of sub-cells along x contiguous, ascending slot
// within a sub-cell).  A neighbour lies at most 2 sub-cells away along each axis, and of the
// 5 x 5 x 5 sub-cells around an atom only those whose nearest point is within r_c + skin are
// scanned: a row (fixed y, z) at a time, as one contiguous run of psub.  That tests about half
// the candidates of the 27 cells (WCA) and 40 % of them at the LJ cutoff.  The test itself is
// the criterion's expression, d = (lf_j - lf_i) + o * wf with o the offset of j's cell, so the
// sets are those of k_build_sorted (the order within a column follows the sub-cell rows).
// The sub-cell slot of an atom is kept in A.layer (free once the cell order is built).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int sub_of(float l, float w, int c) { return 2 * c + ((l >= 0.5f * w) ? 1 : 0); }

__device__ __forceinline__ int64_t sub_index(const Rep& R, int sx, int sy, int sz)
{
    return int64_t(8) * R.cell0 + (int64_t(sz) * (2 * R.nc[1]) + sy) * (2 * R.nc[0]) + sx;
}

__device__ __forceinline__ int64_t sub_of_atom(const Rep& R, const float4& p)
{
    int cx, cy, cz;
    unpack_cell(__float_as_uint(p.w), cx, cy, cz);
    return sub_index(R, sub_of(p.x, R.wf[0], cx), sub_of(p.y, R.wf[1], cy), sub_of(p.z, R.wf[2], cz));
}

__global__ void __launch_bounds__(TILE) k_sub_bin(Arrays A, Scal S, int cur)
{
    if (!A.g->any_rebuild) return;
    const int nrb = A.g->n_rb_tiles;
    for (int it = blockIdx.x; it < nrb; it += gridDim.x) {
        const int t = A.rb_tiles[it];
        const Rep& R = A.rep[A.tile_rep[t]];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const bool active = slot - R.slot0 < R.n;
        const long long sub = active ? sub_of_atom(R, A.pos32[cur][slot]) : -1;
        // lanes of a warp that share a sub-cell take consecutive slots from one atomic
        const unsigned peers = __match_any_sync(0xffffffffu, sub);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int base = 0;
        if (active && lane == leader) base = atomicAdd(&A.scount[sub], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (active) A.layer[slot] = base + rank;
    }
}

__global__ void __launch_bounds__(TILE) k_sub_scatter(Arrays A, Scal S, int cur)
{
    if (!A.g->any_rebuild) return;
    const int nrb = A.g->n_rb_tiles;
    for (int it = blockIdx.x; it < nrb; it += gridDim.x) {
        const int t = A.rb_tiles[it];
        const Rep& R = A.rep[A.tile_rep[t]];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        const float4 p = A.pos32[cur][slot];
        A.psub[A.sstart[sub_of_atom(R, p)] + A.layer[slot]] = make_float4(p.x, p.y, p.z, __int_as_float(int(slot)));
    }
}

// ascending slot within each sub-cell (the atomic slots leave the order to chance)
__global__ void __launch_bounds__(256) k_sub_sort(Arrays A, Scal S)
{
    if (!A.g->any_rebuild) return;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < S.nsub; c += int64_t(gridDim.x) * blockDim.x) {
        const int b = A.sstart[c], e = A.sstart[c + 1];
        for (int k = b + 1; k < e; ++k) {
            const float4 key = A.psub[k];
            int q = k - 1;
            while (q >= b && __float_as_int(A.psub[q].w) > __float_as_int(key.w)) {
                A.psub[q + 1] = A.psub[q];
                --q;
            }
            A.psub[q + 1] = key;
        }
    }
}

// squared distance from l to the sub-cell interval [j h, (j + 1) h) of the atom's cell frame
__device__ __forceinline__ float sub_gap2(float l, int j, float h)
{
    const float lo = float(j) * h, hi = lo + h;
    const float d = (l < lo) ? lo - l : ((l > hi) ? l - hi : 0.0f);
    return d * d;
}

template <int BB, bool STAGE>
__global__ void __launch_bounds__(TILE) k_build_sub(Arrays A, Scal S, int cur)
{
    extern __shared__ uint32_t sW[];                 // STAGE: [cap][TILE] columns of this tile
    if (!A.g->any_rebuild) return;
    const int64_t wstride = STAGE ? int64_t(TILE) : S.nslots;
    const float4* __restrict__ pos = A.pos32[cur];
    const float4* __restrict__ ps = A.psub;
    const int32_t* __restrict__ ss = A.sstart;
    const float rl2 = S.rl2f;
    const float skip2 = rl2 * (1.0f + 1e-5f);
    const int nrb = A.g->n_rb_tiles;
    int run_r = -1, run_max = 0;
    long long run_sum = 0;
    for (int q = 0;; ++q) {
        const int it = build_tile(q);
        if (it >= nrb) break;
        const int t = A.rb_tiles[it];
        const int r = A.tile_rep[t];
        if (r != run_r) {
            if (run_r >= 0) flush_stats(&A.rs[run_r].sum_nbrs, &A.rs[run_r].max_nbrs, run_sum, run_max);
            run_r = r;
            run_sum = 0;
            run_max = 0;
        }
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const bool active = slot - R.slot0 < R.n;
        int m = 0;
        if (active) {
            const float4 pi = pos[slot];
            int cx, cy, cz;
            unpack_cell(__float_as_uint(pi.w), cx, cy, cz);
            const float w0 = R.wf[0], w1 = R.wf[1], w2 = R.wf[2];
            const float h0 = 0.5f * w0, h1 = 0.5f * w1, h2 = 0.5f * w2;
            // the atom's half along each axis; sub-cell j = b + d (d = -2..2) of the cell frame
            const int bx = (pi.x >= h0) ? 1 : 0, by = (pi.y >= h1) ? 1 : 0, bz = (pi.z >= h2) ? 1 : 0;
            const int nsx = 2 * R.nc[0], nsy = 2 * R.nc[1], nsz = 2 * R.nc[2];
            float gx[5];
#pragma unroll
            for (int d = 0; d < 5; ++d) gx[d] = sub_gap2(pi.x, bx + d - 2, h0);
            const int me = int(slot);
            uint32_t* wp = STAGE ? sW + threadIdx.x : A.W + slot;
            const float2 npxy = make_float2(-pi.x, -pi.y);
            const float npz = -pi.z;
            for (int dz = 0; dz < 5; ++dz) {
                const int jz = bz + dz - 2;
                const float gz = sub_gap2(pi.z, jz, h2);
                if (gz > skip2) continue;
                const int oz = jz >> 1;                            // offset of the sub-cell's cell
                int sz = 2 * cz + jz; sz += (sz < 0) ? nsz : 0; sz -= (sz >= nsz) ? nsz : 0;
                const float offz = float(oz) * w2;
                for (int dy = 0; dy < 5; ++dy) {
                    const int jy = by + dy - 2;
                    const float gyz = sub_gap2(pi.y, jy, h1) + gz;
                    if (gyz > skip2) continue;
                    // the sub-cells of this row within reach form one range d = lo .. hi
                    int lo = 5, hi = -1;
#pragma unroll
                    for (int d = 0; d < 5; ++d) {
                        if (gyz + gx[d] <= skip2) {
                            lo = min(lo, d);
                            hi = d;
                        }
                    }
                    if (hi < 0) continue;
                    const int oy = jy >> 1;
                    int sy = 2 * cy + jy; sy += (sy < 0) ? nsy : 0; sy -= (sy >= nsy) ? nsy : 0;
                    const float offy = float(oy) * w1;
                    const uint32_t codeyz = (uint32_t(oy + 1) << 2) | (uint32_t(oz + 1) << 4);
                    const int64_t row = sub_index(R, 0, sy, sz);
                    const int sxl = 2 * cx + bx + lo - 2, sxh = 2 * cx + bx + hi - 2;
                    if (sxl >= 0 && sxh < nsx) {
                        // one run of psub; the cells change at sub-cells 2 cx and 2 cx + 2
                        const int kb = ss[row + sxl], ke = ss[row + sxh + 1];
                        const int b1 = ss[row + min(max(2 * cx, sxl), sxh + 1)];
                        const int b2 = ss[row + min(max(2 * cx + 2, sxl), sxh + 1)];
                        for (int k0 = kb; k0 < ke; k0 += BB) {
                            float4 pj[BB];
#pragma unroll
                            for (int u = 0; u < BB; ++u) pj[u] = ps[min(k0 + u, ke - 1)];
#pragma unroll
                            for (int u = 0; u < BB; ++u) {
                                const int k = k0 + u;
                                const uint32_t c = uint32_t(k >= b1) + uint32_t(k >= b2);   // o_x + 1
                                const float offx = (k < b1) ? -w0 : ((k < b2) ? 0.0f : w0);
                                nbr_test(pj[u], npxy, npz, offx, offy, offz, k < ke, codeyz | c, me, rl2, wp, m,
                                         S.cap, wstride, S.half_list);
                            }
                        }
                    } else {
                        // a periodic wrap in x: sub-cell by sub-cell
                        for (int d = lo; d <= hi; ++d) {
                            const int jx = bx + d - 2;
                            const int ox = jx >> 1;
                            int sx = 2 * cx + jx; sx += (sx < 0) ? nsx : 0; sx -= (sx >= nsx) ? nsx : 0;
                            const int b = ss[row + sx], e = ss[row + sx + 1];
                            const float offx = float(ox) * w0;
                            for (int k0 = b; k0 < e; k0 += BB) {
                                float4 pj[BB];
#pragma unroll
                                for (int u = 0; u < BB; ++u) pj[u] = ps[min(k0 + u, e - 1)];
#pragma unroll
                                for (int u = 0; u < BB; ++u)
                                    nbr_test(pj[u], npxy, npz, offx, offy, offz, k0 + u < e, codeyz | uint32_t(ox + 1), me,
                                             rl2, wp, m, S.cap, wstride, S.half_list);
                            }
                        }
                    }
                }
            }
            A.nbr_count[slot] = m;
            if (S.rule == MD_REBUILD_DISP) A.xref[slot] = make_float4(pi.x, pi.y, pi.z, 0.0f);
            if (m > S.cap) {
                atomicOr(&A.g->err, ERR_NBR_OVERFLOW);
                atomicMax(&A.g->max_nbr_seen, m);
            }
            run_sum += m;
            run_max = max(run_max, m);
        }
        if (STAGE) flush_columns(A, S, sW, slot, active ? min(m, S.cap) : 0);
    }
    if (run_r >= 0) flush_stats(&A.rs[run_r].sum_nbrs, &A.rs[run_r].max_nbrs, run_sum, run_max);
}

// ------------------------------------------------------------------------------------------
// N5 for dense cells (tens of atoms per cell, e.g. the LJ liquid at r_c + skin = 2.8): one warp
// per cell, one lane per atom of it.  The candidates of each 3-cell row of the 27-cell
// neighbourhood are staged once in the warp's shared memory (coalesced loads, double-buffered:
// the next row is loaded while the current one is tested), and every lane tests them with
// broadcast reads, so no candidate is fetched per lane and no lane diverges.  The displacement
// is the criterion's expression (p_j - p_i) + o w, o constant per cell.  Rows and cells no lane
// of the warp can reach are skipped by a warp vote.
// ------------------------------------------------------------------------------------------
constexpr int CW_WARPS = TILE / 32;
constexpr int CW_ROW = 128;                    // candidates of one row staged at a time
constexpr int CW_PER_LANE = CW_ROW / 32;

struct CwRow {
    int b[3], n[3];                           // the three cells of the row as perm ranges
    int tot;
};

__device__ __forceinline__ int cw_index(const CwRow& R, int q)
{
    return (q < R.n[0]) ? R.b[0] + q : ((q < R.n[0] + R.n[1]) ? R.b[1] + (q - R.n[0]) : R.b[2] + (q - R.n[0] - R.n[1]));
}

__global__ void __launch_bounds__(TILE) k_build_cw(Arrays A, Scal S, int cur)
{
    if (!A.g->any_rebuild) return;
    __shared__ float4 s_p[CW_WARPS][2][CW_ROW];
    const float4* __restrict__ ps = A.psort;
    const float rl2 = S.rl2f;
    const float skip2 = rl2 * (1.0f + 1e-5f);
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int run_r = -1, run_max = 0;
    long long run_sum = 0;
    // cells in chunks of 2 dealt to the warps in turn (as build_tile does for tiles)
    for (int q = 0;; ++q) {
        const int c = ((q >> 1) * nw + gw) * 2 + (q & 1);
        if (c >= S.ncells) break;
        const int r = A.cell_rep[c];
        if (r != run_r) {
            if (run_r >= 0) {
                const long long ws = warp_sum_ll(run_sum);
                const int wm = warp_max_i(run_max);
                if (lane == 0) {
                    if (ws) atomicAdd(reinterpret_cast<unsigned long long*>(&A.rs[run_r].sum_nbrs),
                                      static_cast<unsigned long long>(ws));
                    if (wm > 0) atomicMax(&A.rs[run_r].max_nbrs, wm);
                }
            }
            run_r = r;
            run_sum = 0;
            run_max = 0;
        }
        if (!A.rs[r].rebuild) continue;
        const Rep& R = A.rep[r];
        const int cl = c - R.cell0;
        int cx, cy, cz;
        cell_coords(R, cl, cx, cy, cz);
        const int xs[3] = {(cx == 0) ? R.nc[0] - 1 : cx - 1, cx, (cx == R.nc[0] - 1) ? 0 : cx + 1};
        const float w0 = R.wf[0], w1 = R.wf[1], w2 = R.wf[2];
        const int ab = A.cstart[c], ae = A.cstart[c + 1];
        for (int a0 = ab; a0 < ae; a0 += 32) {
            const bool have = a0 + lane < ae;
            const float4 pi = have ? ps[a0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int i = have ? __float_as_int(pi.w) : -1;
            const float dl[3] = {pi.x * pi.x, pi.y * pi.y, pi.z * pi.z};
            const float dh[3] = {(w0 - pi.x) * (w0 - pi.x), (w1 - pi.y) * (w1 - pi.y), (w2 - pi.z) * (w2 - pi.z)};
            int m = 0;
            uint32_t* wp = A.W + (have ? i : 0);
            // the 9 rows (oy, oz) and their cells, with the ones no lane can reach removed
            auto row_of = [&](int rr, CwRow& Q) {
                const int oy = rr % 3 - 1, oz = rr / 3 - 1;
                int ny = cy + oy; ny += (ny < 0) ? R.nc[1] : 0; ny -= (ny >= R.nc[1]) ? R.nc[1] : 0;
                int nz = cz + oz; nz += (nz < 0) ? R.nc[2] : 0; nz -= (nz >= R.nc[2]) ? R.nc[2] : 0;
                const float dyz = ((oy < 0) ? dl[1] : ((oy > 0) ? dh[1] : 0.f)) + ((oz < 0) ? dl[2] : ((oz > 0) ? dh[2] : 0.f));
                const int rowc = R.cell0 + row_pos(R, ny, nz) * R.nc[0];
                Q.tot = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float dd = dyz + ((k == 0) ? dl[0] : ((k == 2) ? dh[0] : 0.f));
                    const bool need = __any_sync(0xffffffffu, have && dd <= skip2);
                    const int gc = rowc + xs[k];
                    Q.b[k] = A.cstart[gc];
                    Q.n[k] = need ? A.cstart[gc + 1] - Q.b[k] : 0;
                    Q.tot += Q.n[k];
                }
            };
            CwRow cur_row, nxt_row;
            float4 rp[CW_PER_LANE];                 // a candidate's slot is in .w
            auto load_regs = [&](const CwRow& Q, int q0) {
#pragma unroll
                for (int u = 0; u < CW_PER_LANE; ++u) {
                    const int q = q0 + lane + 32 * u;
                    if (q < Q.tot) rp[u] = ps[cw_index(Q, q)];
                }
            };
            auto store_regs = [&](const CwRow& Q, int q0, int buf) {
#pragma unroll
                for (int u = 0; u < CW_PER_LANE; ++u) {
                    const int q = lane + 32 * u;
                    if (q0 + q < Q.tot) s_p[wl][buf][q] = rp[u];
                }
            };
            auto test_row = [&](const CwRow& Q, int q0, int buf, int rr) {
                const int oy = rr % 3 - 1, oz = rr / 3 - 1;
                const float offy = float(oy) * w1, offz = float(oz) * w2;
                const uint32_t codeyz = (uint32_t(oy + 1) << 2) | (uint32_t(oz + 1) << 4);
                const int qend = min(Q.tot, q0 + CW_ROW);
                int seg_end = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int seg_beg = seg_end;
                    seg_end += Q.n[k];
                    const int lo = max(seg_beg, q0), hi = min(seg_end, qend);
                    const float offx = float(k - 1) * w0;
                    const uint32_t code = codeyz | uint32_t(k);
                    for (int q = lo; q < hi; ++q) {
                        const float4 pj = s_p[wl][buf][q - q0];
                        const int j = __float_as_int(pj.w);
                        const float dx = __fadd_rn(__fsub_rn(pj.x, pi.x), offx);
                        const float dy = __fadd_rn(__fsub_rn(pj.y, pi.y), offy);
                        const float dz = __fadd_rn(__fsub_rn(pj.z, pi.z), offz);
                        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                        if (have && r2 < rl2 && (S.half_list ? j > i : j != i)) {
                            if (m < S.cap) {
                                *wp = (uint32_t(j) << IDX_SHIFT) | code;
                                wp += S.nslots;
                            }
                            ++m;
                        }
                    }
                }
            };
            // software pipeline over the rows: stage row rr+1 while testing row rr
            int buf = 0;
            row_of(0, cur_row);
            load_regs(cur_row, 0);
            store_regs(cur_row, 0, buf);
            __syncwarp();
            for (int rr = 0; rr < 9; ++rr) {
                // rows longer than the staging buffer are walked in chunks without overlap
                for (int q0 = CW_ROW; q0 < cur_row.tot; q0 += CW_ROW) {
                    test_row(cur_row, q0 - CW_ROW, buf, rr);
                    __syncwarp();
                    load_regs(cur_row, q0);
                    store_regs(cur_row, q0, buf);
                    __syncwarp();
                }
                const int qlast = (cur_row.tot > 0) ? ((cur_row.tot - 1) / CW_ROW) * CW_ROW : 0;
                if (rr + 1 < 9) {
                    row_of(rr + 1, nxt_row);
                    load_regs(nxt_row, 0);
                }
                test_row(cur_row, qlast, buf, rr);
                if (rr + 1 < 9) {
                    store_regs(nxt_row, 0, buf ^ 1);
                    __syncwarp();
                    buf ^= 1;
                    cur_row = nxt_row;
                }
            }
            __syncwarp();
            if (have) {
                A.nbr_count[i] = m;
                if (S.rule == MD_REBUILD_DISP) A.xref[i] = make_float4(pi.x, pi.y, pi.z, 0.0f);
                if (m > S.cap) {
                    atomicOr(&A.g->err, ERR_NBR_OVERFLOW);
                    atomicMax(&A.g->max_nbr_seen, m);
                }
                run_sum += m;
                run_max = max(run_max, m);
            }
        }
    }
    if (run_r >= 0) {
        const long long ws = warp_sum_ll(run_sum);
        const int wm = warp_max_i(run_max);
        if (lane == 0) {
            if (ws) atomicAdd(reinterpret_cast<unsigned long long*>(&A.rs[run_r].sum_nbrs), static_cast<unsigned long long>(ws));
            if (wm > 0) atomicMax(&A.rs[run_r].max_nbrs, wm);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Slot windows of each rebuilt tile's neighbours, for the step kernel that stages neighbour
// positions in shared memory: for every (o_y, o_z) row code, the smallest and largest slot among
// the tile's W entries of that code whose neighbour cell is reached without a periodic wrap
// (wrapped entries are gathered from global memory).  With atoms in cell order (reorder at every
// rebuild) each window spans the tile's cells plus one halo cell at either end, in one row of
// cells; otherwise windows can be wide, and the step kernel then stages what fits its budget.
// One CTA per tile; empty rows get lo > hi.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE) k_tile_windows(Arrays A, Scal S, int cur, int enabled)
{
    __shared__ int sh_lo[9], sh_hi[9];
    if (!enabled || !A.g->any_rebuild || !A.tile_win) return;
    const int nrb = A.g->n_rb_tiles;
    for (int it = blockIdx.x; it < nrb; it += gridDim.x) {
        const int t = A.rb_tiles[it];
        const Rep& R = A.rep[A.tile_rep[t]];
        if (threadIdx.x < 9) {
            sh_lo[threadIdx.x] = INT32_MAX;
            sh_hi[threadIdx.x] = -1;
        }
        __syncthreads();
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 < R.n) {
            int cx, cy, cz;
            unpack_cell(__float_as_uint(A.pos32[cur][slot].w), cx, cy, cz);
            // codes whose neighbour cell lies across the periodic boundary for this atom
            const bool wxl = cx == 0, wxh = cx == R.nc[0] - 1, wyl = cy == 0, wyh = cy == R.nc[1] - 1;
            const bool wzl = cz == 0, wzh = cz == R.nc[2] - 1;
            int lo[9], hi[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                lo[q] = INT32_MAX;
                hi[q] = -1;
            }
            const int mm = min(A.nbr_count[slot], S.cap);
            constexpr int B = 4;                 // rows of W loaded together
            for (int m0 = 0; m0 < mm; m0 += B) {
              uint32_t eb[B];
#pragma unroll
              for (int u = 0; u < B; ++u) eb[u] = (m0 + u < mm) ? __ldcs(A.W + int64_t(m0 + u) * S.nslots + slot) : 0u;
#pragma unroll
              for (int u = 0; u < B; ++u) {
                if (m0 + u >= mm) break;
                const uint32_t e = eb[u];
                const uint32_t ox = e & 3u, oy = (e >> 2) & 3u, oz = (e >> 4) & 3u;
                const bool wrap = (ox == 0 && wxl) || (ox == 2 && wxh) || (oy == 0 && wyl) || (oy == 2 && wyh) ||
                                  (oz == 0 && wzl) || (oz == 2 && wzh);
                if (wrap) continue;
                const int j = int(e >> IDX_SHIFT);
                const int q = int(oy + 3 * oz);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    if (k == q) {
                        lo[k] = min(lo[k], j);
                        hi[k] = max(hi[k], j);
                    }
                }
              }
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                if (hi[k] >= 0) {
                    atomicMin(&sh_lo[k], lo[k]);
                    atomicMax(&sh_hi[k], hi[k]);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < 9) A.tile_win[int64_t(t) * 9 + threadIdx.x] = make_int2(sh_lo[threadIdx.x], sh_hi[threadIdx.x]);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// bookkeeping after a rebuild
// ------------------------------------------------------------------------------------------
__global__ void k_rebuild_finish(Arrays A, Scal S, int in_graph)
{
    if (!A.g->any_rebuild) return;
    for (int r = threadIdx.x; r < S.nrep; r += blockDim.x) {
        RepState& st = A.rs[r];
        if (!st.rebuild) continue;
        if (st.reorder) {
            st.last_reorder = st.step;
            st.reorders += 1;
        }
        st.reorder = 0;
        st.rebuild = 0;
        st.D = 0.0;
        st.rebuilds += 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        A.g->any_rebuild = 0;
        A.g->any_reorder = 0;
        if (in_graph) A.g->graph_rebuilds += 1;
    }
}

// Mark every replica for a rebuild (creation, md_set_state, md_bin_cells).
__global__ void k_force_rebuild(Arrays A, Scal S, int reorder)
{
    for (int r = threadIdx.x; r < S.nrep; r += blockDim.x) {
        A.rs[r].rebuild = 1;
        A.rs[r].reorder = reorder;
        A.rs[r].max_occ = 0;
    }
    if (threadIdx.x == 0) {
        A.g->any_rebuild = 1;
        A.g->any_reorder = reorder;
    }
}

// ------------------------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------------------------
static int tile_grid(const Scal& S, const Launch& L)
{
    return std::max(1, std::min(L.grid, S.ntiles));
}

// Grid of a per-tile rebuild kernel that holds nothing across tiles (binning, scatter, reorder,
// the neighbour build): every CTA the device can keep resident.  Binning, scatter and reorder wait
// on memory and atomics, so each resident warp adds requests in flight; the build gains warps to
// issue from (9 CTAs per SM instead of the step kernel's 8: 3 % less build time on the 4M-atom
// fluid).  The occupancy of each kernel is looked up once.
template <auto Kernel>
static int resident_grid(const Scal& S, const Launch& L)
{
    static const int per_sm = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, Kernel, TILE, 0) != cudaSuccess) b = 0;
        return b;
    }();
    const int g = (per_sm > 0) ? L.nsm * per_sm : L.grid;
    return std::max(1, std::min(g, S.ntiles));
}

// looks the occupancies up outside any stream capture
void prime_rebuild_grids(const Scal& S, const Launch& L)
{
    (void)resident_grid<k_bin<MD_FP64>>(S, L);
    (void)resident_grid<k_bin<MD_MIXED>>(S, L);
    (void)resident_grid<k_bin<MD_FP32>>(S, L);
    (void)resident_grid<k_scatter>(S, L);
    (void)resident_grid<k_build_sorted<2, false>>(S, L);
    (void)resident_grid<k_build_sorted<4, false>>(S, L);
    (void)resident_grid<k_build_sub<2, false>>(S, L);
    (void)resident_grid<k_sub_bin>(S, L);
    (void)resident_grid<k_sub_scatter>(S, L);
    (void)resident_grid<k_reorder_gather<MD_FP64>>(S, L);
    (void)resident_grid<k_reorder_gather<MD_MIXED>>(S, L);
    (void)resident_grid<k_reorder_gather<MD_FP32>>(S, L);
    (void)resident_grid<k_reorder_copy<MD_FP64>>(S, L);
    (void)resident_grid<k_reorder_copy<MD_MIXED>>(S, L);
    (void)resident_grid<k_reorder_copy<MD_FP32>>(S, L);
}

cudaError_t launch_force_rebuild(const Arrays& A, const Scal& S, const Launch& L, int reorder)
{
    k_force_rebuild<<<1, 256, 0, L.stream>>>(A, S, reorder);
    return cudaGetLastError();
}

cudaError_t launch_bin_order(const Arrays& A, const Scal& S, const Launch& L, int cur, bool from_set)
{
    k_rebuild_list<<<1, 1024, 0, L.stream>>>(A, S);
    const int fs = from_set ? 1 : 0;
    if (S.mode == MD_FP64) k_bin<MD_FP64><<<resident_grid<k_bin<MD_FP64>>(S, L), TILE, 0, L.stream>>>(A, S, cur, fs);
    else if (S.mode == MD_MIXED) k_bin<MD_MIXED><<<resident_grid<k_bin<MD_MIXED>>(S, L), TILE, 0, L.stream>>>(A, S, cur, fs);
    else k_bin<MD_FP32><<<resident_grid<k_bin<MD_FP32>>(S, L), TILE, 0, L.stream>>>(A, S, cur, fs);
    launch_scan(A, ScanArgs{A.ccount, A.cstart, A.chunk, S.ncells, S.nchunks}, L.stream);
    k_scatter<<<resident_grid<k_scatter>(S, L), TILE, 0, L.stream>>>(A, S);
    const int gs = int(std::min<int64_t>((S.ncells + 255) / 256, int64_t(L.grid) * 8));
    k_sort_cells<<<std::max(gs, 1), 256, 0, L.stream>>>(A, S, cur);
    return cudaGetLastError();
}

cudaError_t launch_reorder(const Arrays& A, const Scal& S, const Launch& L, int cur)
{
#define GBMD_REORDER(M)                                                                               \
    {                                                                                                 \
        k_reorder_gather<M><<<resident_grid<k_reorder_gather<M>>(S, L), TILE, 0, L.stream>>>(A, S, cur); \
        k_reorder_copy<M><<<resident_grid<k_reorder_copy<M>>(S, L), TILE, 0, L.stream>>>(A, S, cur);     \
    }
    if (S.mode == MD_FP64) GBMD_REORDER(MD_FP64)
    else if (S.mode == MD_MIXED) GBMD_REORDER(MD_MIXED)
    else GBMD_REORDER(MD_FP32)
#undef GBMD_REORDER
    return cudaGetLastError();
}

cudaError_t launch_bin_only(const Arrays& A, const Scal& S, const Launch& L, int cur, bool from_set)
{
    cudaError_t e = launch_bin_order(A, S, L, cur, from_set);
    if (e != cudaSuccess) return e;
    return launch_reorder(A, S, L, cur);
}

// the list-free step kernel reads no neighbour matrix; it is built only where the exact
// displacement rule needs the positions at the rebuild (written by the build)
static bool skip_w(const Scal& S, const Launch& L) { return L.step_kernel == 4 && S.rule != MD_REBUILD_DISP; }

int build_kernels(const Scal& S, const Launch& L) { return skip_w(S, L) ? 2 : (L.build_batch == 1 ? 9 : 3); }

// Grid of a staged build kernel: every CTA resident with `smem` bytes of columns each (the
// occupancy is looked up again when the size changes)
template <auto Kernel>
static int staged_grid(const Scal& S, const Launch& L, int smem)
{
    static int last_smem = -1, per_sm = 0;
    if (smem != last_smem) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, std::min(optin, smem));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kernel, TILE, smem) != cudaSuccess) per_sm = 1;
        last_smem = smem;
    }
    return std::max(1, std::min(L.nsm * std::max(per_sm, 1), S.ntiles));
}

// staging the columns needs cap x TILE x 4 bytes per CTA: at most 160 KB (cap <= 320)
static bool stage_w(const Scal& S, const Launch& L) { return L.build_stage && S.cap * TILE * 4 <= 160 * 1024; }

cudaError_t launch_build_only(const Arrays& A, const Scal& S, const Launch& L, int cur)
{
    const int g = tile_grid(S, L);
    if (S.mode == MD_FP64) k_build<double, 1><<<g, TILE, 0, L.stream>>>(A, S, cur);
    else if (skip_w(S, L)) {
    } else if (L.build_batch == 1) {
        k_sub_bin<<<resident_grid<k_sub_bin>(S, L), TILE, 0, L.stream>>>(A, S, cur);
        launch_scan(A, ScanArgs{A.scount, A.sstart, A.schunk, S.nsub, S.nschunks}, L.stream);
        k_sub_scatter<<<resident_grid<k_sub_scatter>(S, L), TILE, 0, L.stream>>>(A, S, cur);
        const int gs = int(std::min<int64_t>((S.nsub + 255) / 256, int64_t(L.grid) * 8));
        k_sub_sort<<<std::max(gs, 1), 256, 0, L.stream>>>(A, S);
        if (stage_w(S, L)) {
            const int sm = S.cap * TILE * 4;
            k_build_sub<2, true><<<staged_grid<k_build_sub<2, true>>(S, L, sm), TILE, sm, L.stream>>>(A, S, cur);
        } else {
            k_build_sub<2, false><<<resident_grid<k_build_sub<2, false>>(S, L), TILE, 0, L.stream>>>(A, S, cur);
        }
    }
    else if (L.build_batch >= 32) k_build_cw<<<std::max(1, L.grid), TILE, 0, L.stream>>>(A, S, cur);
    else if (stage_w(S, L)) {
        const int sm = S.cap * TILE * 4;
        if (L.build_batch >= 4)
            k_build_sorted<4, true><<<staged_grid<k_build_sorted<4, true>>(S, L, sm), TILE, sm, L.stream>>>(A, S, cur);
        else
            k_build_sorted<2, true><<<staged_grid<k_build_sorted<2, true>>(S, L, sm), TILE, sm, L.stream>>>(A, S, cur);
    }
    else if (L.build_batch >= 4)
        k_build_sorted<4, false><<<resident_grid<k_build_sorted<4, false>>(S, L), TILE, 0, L.stream>>>(A, S, cur);
    else k_build_sorted<2, false><<<resident_grid<k_build_sorted<2, false>>(S, L), TILE, 0, L.stream>>>(A, S, cur);
    k_tile_windows<<<g, TILE, 0, L.stream>>>(A, S, cur, L.step_kernel == 3 ? 1 : 0);   // used by step kernel 3
    k_rebuild_finish<<<1, 256, 0, L.stream>>>(A, S, L.in_graph);
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const Arrays& A, const Scal& S, const Launch& L, int cur, bool from_set)
{
    cudaError_t e = launch_bin_only(A, S, L, cur, from_set);
    if (e != cudaSuccess) return e;
    return launch_build_only(A, S, L, cur);
}

}  // namespace gbmd
