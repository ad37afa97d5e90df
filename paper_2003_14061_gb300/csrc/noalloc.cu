// noalloc.cu -- md_forces_static: pair forces for a small system without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need forces: host code
// inside another runtime or framework that hands out only pre-planned buffers and owns the
// device allocator, plug-ins that run between someone else's kernels where a cudaMalloc/cudaFree
// would take the device-wide synchronisation these calls can imply, or code that has no
// workspace to hand.  For them this entry point keeps its cell-list scratch (occupancy counts,
// prefix sums, cell order, cell-local positions) in one file-scope __device__ array of fixed
// size, instead of a caller-provided workspace.  The computation is the force pass of
// md_compute_forces on a plain cell list of side >= r_c (no neighbour matrix): FP32 pair
// arithmetic on cell-local coordinates, per-atom sums in a fixed order (the atoms of each cell
// ascending), so repeated calls on the same input give the same bits.
//
// Limits and sharing:
//   * at most NA_MAX_ATOMS atoms and NA_MAX_CELLS cells (both 65536); larger requests fail with
//     MD_ERR_INVALID_ARG before any work is queued;
//   * every GPU that loads the library keeps the NA_BYTES array until the process exits;
//   * all calls share the array and it keeps the last call's contents: each call clears the
//     occupancy counters itself, and calls whose work overlaps on the GPU (different streams
//     without ordering between them) race on the array and must not be issued;
//   * the host needs the array's device address: the first call on each device looks it up
//     (cudaGetSymbolAddress) with that device current, so that first call should come before any
//     stream capture; the address is kept for the life of the process, so the entry point must
//     not be used after cudaDeviceReset on that device.
#include <mutex>
#include <string>

#include "gbmd_internal.cuh"

namespace {

constexpr int NA_MAX_ATOMS = 1 << 16;
constexpr int NA_MAX_CELLS = 1 << 16;
constexpr int NA_THREADS = 128;
constexpr size_t NA_COUNT_OFF = 0;                                              // int32[cells]
constexpr size_t NA_START_OFF = NA_COUNT_OFF + sizeof(int32_t) * NA_MAX_CELLS;  // int32[cells+1]
constexpr size_t NA_PERM_OFF = NA_START_OFF + sizeof(int32_t) * (NA_MAX_CELLS + 64);
constexpr size_t NA_CELL_OFF = NA_PERM_OFF + sizeof(int32_t) * NA_MAX_ATOMS;
constexpr size_t NA_LAYER_OFF = NA_CELL_OFF + sizeof(int32_t) * NA_MAX_ATOMS;
constexpr size_t NA_POS_OFF = NA_LAYER_OFF + sizeof(int32_t) * NA_MAX_ATOMS;     // float4[atoms]
constexpr size_t NA_BYTES = NA_POS_OFF + sizeof(float4) * NA_MAX_ATOMS;          // 1.75 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NaView {
    int32_t* count;
    int32_t* start;
    int32_t* perm;
    int32_t* cell;
    int32_t* layer;
    float4* pos;
};

struct NaGeom {
    double L[3], w[3], s[3];
    float wf[3];
    float wlo[3];          // (float) (w - wf), added after o wf to keep the distances unbiased
    int nc[3];
    int ncells;
    int n;
    float rc2f, sig2f, eps4f, eps48f, ucf;
};

NaView view_of(void* base)
{
    unsigned char* b = static_cast<unsigned char*>(base);
    return NaView{reinterpret_cast<int32_t*>(b + NA_COUNT_OFF), reinterpret_cast<int32_t*>(b + NA_START_OFF),
                  reinterpret_cast<int32_t*>(b + NA_PERM_OFF), reinterpret_cast<int32_t*>(b + NA_CELL_OFF),
                  reinterpret_cast<int32_t*>(b + NA_LAYER_OFF), reinterpret_cast<float4*>(b + NA_POS_OFF)};
}

// cell of each atom, cell-local FP32 position, layer slot in its cell
__global__ void __launch_bounds__(NA_THREADS) k_na_bin(NaView V, NaGeom G, const double* __restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    int c[3];
    float l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double xa = x[3 * i + a];
        if (xa < 0.0) xa += G.L[a];
        if (xa >= G.L[a]) xa -= G.L[a];
        if (!(xa >= 0.0 && xa < G.L[a])) {           // more than one period away: whole periods
            xa -= G.L[a] * floor(xa / G.L[a]);
            if (xa < 0.0) xa += G.L[a];
            if (xa >= G.L[a]) xa -= G.L[a];
        }
        int ca = int(floor(xa * G.s[a]));
        ca = min(max(ca, 0), G.nc[a] - 1);
        c[a] = ca;
        l[a] = __double2float_rn(xa - double(ca) * G.w[a]);
    }
    const int cell = (c[2] * G.nc[1] + c[1]) * G.nc[0] + c[0];
    V.pos[i] = make_float4(l[0], l[1], l[2], __uint_as_float(gbmd::pack_cell(c[0], c[1], c[2])));
    V.cell[i] = cell;
    V.layer[i] = atomicAdd(&V.count[cell], 1);
}

// exclusive prefix sum of the occupancies, one block
__global__ void __launch_bounds__(1024) k_na_scan(NaView V, NaGeom G)
{
    __shared__ int sh[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (int c0 = 0; c0 < G.ncells; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int v = (c < G.ncells) ? V.count[c] : 0;
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
        if (c < G.ncells) V.start[c] = carry + sh[wid] + incl - v;
        carry += sh[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) V.start[G.ncells] = carry;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_scatter(NaView V, NaGeom G)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < G.n) V.perm[V.start[V.cell[i]] + V.layer[i]] = i;
}

// the atomic layer slots leave the order inside a cell to chance; sorting each cell's atoms by
// index fixes the summation order of every force, so repeated calls give identical bits
__global__ void __launch_bounds__(NA_THREADS) k_na_sort(NaView V, NaGeom G)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.ncells) return;
    const int b = V.start[c], e = V.start[c + 1];
    for (int k = b + 1; k < e; ++k) {                // insertion sort: cells hold a few atoms
        const int key = V.perm[k];
        int q = k - 1;
        while (q >= b && V.perm[q] > key) {
            V.perm[q + 1] = V.perm[q];
            --q;
        }
        V.perm[q + 1] = key;
    }
}

// F1 over the 27 cells around each atom; force on i is g (x_i - x_j)
__global__ void __launch_bounds__(NA_THREADS) k_na_forces(NaView V, NaGeom G, double* __restrict__ f,
                                                          double* __restrict__ u)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    const float4 pi = V.pos[i];
    int cx, cy, cz;
    gbmd::unpack_cell(__float_as_uint(pi.w), cx, cy, cz);
    float fx = 0.f, fy = 0.f, fz = 0.f, ui = 0.f;
    for (int oz = -1; oz <= 1; ++oz) {
        int nz = cz + oz; nz += (nz < 0) ? G.nc[2] : 0; nz -= (nz >= G.nc[2]) ? G.nc[2] : 0;
        for (int oy = -1; oy <= 1; ++oy) {
            int ny = cy + oy; ny += (ny < 0) ? G.nc[1] : 0; ny -= (ny >= G.nc[1]) ? G.nc[1] : 0;
            for (int ox = -1; ox <= 1; ++ox) {
                int nx = cx + ox; nx += (nx < 0) ? G.nc[0] : 0; nx -= (nx >= G.nc[0]) ? G.nc[0] : 0;
                const int c = (nz * G.nc[1] + ny) * G.nc[0] + nx;
                for (int k = V.start[c]; k < V.start[c + 1]; ++k) {
                    const int j = V.perm[k];
                    if (j == i) continue;
                    const float4 pj = V.pos[j];
                    const float dx = fmaf(float(ox), G.wlo[0], fmaf(float(ox), G.wf[0], pj.x - pi.x));
                    const float dy = fmaf(float(oy), G.wlo[1], fmaf(float(oy), G.wf[1], pj.y - pi.y));
                    const float dz = fmaf(float(oz), G.wlo[2], fmaf(float(oz), G.wf[2], pj.z - pi.z));
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    if (r2 < G.rc2f) {
                        const float ri2 = __frcp_rn(r2);
                        const float sr2 = G.sig2f * ri2;
                        const float sr6 = sr2 * sr2 * sr2;
                        const float fs = G.eps48f * sr6 * (sr6 - 0.5f) * ri2;
                        fx = fmaf(-fs, dx, fx);
                        fy = fmaf(-fs, dy, fy);
                        fz = fmaf(-fs, dz, fz);
                        ui += fmaf(G.eps4f * sr6, sr6 - 1.0f, -G.ucf);
                    }
                }
            }
        }
    }
    f[3 * i + 0] = fx;
    f[3 * i + 1] = fy;
    f[3 * i + 2] = fz;
    if (u) u[i] = ui;
}

std::mutex g_na_mutex;
void* g_na_addr[256] = {nullptr};

int na_fail(int code, const std::string& msg) { return gbmd::set_last_error(code, msg.c_str()); }

}  // namespace

extern "C" {

int md_forces_static(const md_params* p, int64_t n, const double* x, double* f, double* u, void* stream)
{
    if (!p || !x || !f) return na_fail(MD_ERR_INVALID_ARG, "params, x and f are required");
    if (n <= 0 || n > NA_MAX_ATOMS)
        return na_fail(MD_ERR_INVALID_ARG, "md_forces_static handles 1.." + std::to_string(NA_MAX_ATOMS) + " atoms, got " +
                                               std::to_string(n));
    if (!(p->rc > 0.0) || !(p->eps > 0.0) || !(p->sigma > 0.0)) return na_fail(MD_ERR_INVALID_ARG, "bad potential");
    NaGeom G;
    G.ncells = 1;
    for (int a = 0; a < 3; ++a) {
        const double L = p->box[a];
        if (!(L > 0.0)) return na_fail(MD_ERR_INVALID_ARG, "box sides must be > 0");
        const double q = std::floor(L / p->rc);
        if (q < 3.0) return na_fail(MD_ERR_BOX_TOO_SMALL, "fewer than 3 cells of side >= rc");
        if (q > gbmd::MAX_NC) return na_fail(MD_ERR_INVALID_ARG, "more than 1023 cells along an axis");
        G.nc[a] = int(q);
        G.L[a] = L;
        G.w[a] = L / q;
        G.s[a] = q / L;
        G.wf[a] = float(G.w[a]);
        G.wlo[a] = float(G.w[a] - double(G.wf[a]));
        if (int64_t(G.ncells) * G.nc[a] > NA_MAX_CELLS)
            return na_fail(MD_ERR_INVALID_ARG, "md_forces_static handles at most " + std::to_string(NA_MAX_CELLS) +
                                                   " cells of side >= rc");
        G.ncells *= G.nc[a];
    }
    G.n = int(n);
    const double rc2 = p->rc * p->rc, sig2 = p->sigma * p->sigma;
    double uc = 0.0;
    if (p->shift_energy) {
        const double q2 = sig2 / rc2, q6 = q2 * q2 * q2;
        uc = 4.0 * p->eps * (q6 * q6 - q6);
    }
    G.rc2f = float(rc2);
    G.sig2f = float(sig2);
    G.eps4f = float(4.0 * p->eps);
    G.eps48f = float(48.0 * p->eps);
    G.ucf = float(uc);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(MD_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return na_fail(MD_ERR_CUDA, "device ordinal out of range");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_addr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr)
                return na_fail(MD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_addr[dev] = ptr;
        }
        base = g_na_addr[dev];
    }
    const NaView V = view_of(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    (void)cudaGetLastError();        // an earlier, unrelated launch error is not this call's failure
    e = cudaMemsetAsync(V.count, 0, sizeof(int32_t) * size_t(G.ncells), st);
    if (e != cudaSuccess) return na_fail(MD_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int blocks = int((n + NA_THREADS - 1) / NA_THREADS);
    k_na_bin<<<blocks, NA_THREADS, 0, st>>>(V, G, x);
    k_na_scan<<<1, 1024, 0, st>>>(V, G);
    k_na_scatter<<<blocks, NA_THREADS, 0, st>>>(V, G);
    k_na_sort<<<(G.ncells + NA_THREADS - 1) / NA_THREADS, NA_THREADS, 0, st>>>(V, G);
    k_na_forces<<<blocks, NA_THREADS, 0, st>>>(V, G, f, u);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(MD_ERR_CUDA, cudaGetErrorString(e));
    return MD_OK;
}

}  // extern "C"
