// api.cu -- the C ABI of libgbmd.so (declared in include/gbmd.h): parameter checks, the plan of
// slots / tiles / cells, the carving of the caller's workspace, and the host sequence of kernel
// launches for each entry point.  No device memory is allocated here.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gbmd_internal.cuh"

using namespace gbmd;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

#define GBMD_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(MD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

struct Plan {
    int32_t nrep = 0;
    std::vector<Rep> reps;
    std::vector<int32_t> tile_rep;
    std::vector<int32_t> cell_rep;
    int64_t nslots = 0;
    int32_t ntiles = 0;
    int32_t ncells = 0;
    int32_t nchunks = 0;
    int32_t cap = 0;
    int32_t series_cap = 0;
    int64_t n_total = 0;
    int mode = MD_MIXED;
    int rule = MD_REBUILD_VMAX;
};

struct Carver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += std::max<size_t>(count, 1) * sizeof(T);
        return p;
    }
};

int check_params(const md_params* p)
{
    if (!p) return fail(MD_ERR_INVALID_ARG, "params is NULL");
    auto pos = [](double x) { return std::isfinite(x) && x > 0.0; };
    if (!pos(p->eps) || !pos(p->sigma) || !pos(p->mass) || !pos(p->rc) || !pos(p->dt))
        return fail(MD_ERR_INVALID_ARG, "eps, sigma, mass, rc and dt must be finite and > 0");
    if (!std::isfinite(p->skin) || p->skin < 0.0) return fail(MD_ERR_INVALID_ARG, "skin must be >= 0");
    if (p->precision < MD_FP64 || p->precision > MD_FP32) return fail(MD_ERR_INVALID_ARG, "bad precision");
    if (p->rebuild_rule < MD_REBUILD_VMAX || p->rebuild_rule > MD_REBUILD_EVERY)
        return fail(MD_ERR_INVALID_ARG, "bad rebuild_rule");
    if (p->reorder_every < 0 || p->nbr_capacity < 0 || p->props_every < 0 || p->cell_block < 0)
        return fail(MD_ERR_INVALID_ARG, "reorder_every, nbr_capacity, props_every and cell_block must be >= 0");
    return MD_OK;
}

// the largest power of two not above v (v >= 1)
int pow2_floor(int v)
{
    int k = 1;
    while (2 * k <= v) k *= 2;
    return k;
}

int make_plan(const md_params* p, int32_t nrep, const int64_t* n_rep, const double* box_rep, Plan* P)
{
    int rc = check_params(p);
    if (rc) return rc;
    if (nrep <= 0 || !n_rep || !box_rep) return fail(MD_ERR_INVALID_ARG, "need nrep > 0, n_rep and box_rep");
    const double rl = p->rc + p->skin;
    P->nrep = nrep;
    P->mode = p->precision;
    P->rule = p->rebuild_rule;
    P->reps.resize(nrep);
    int64_t slot = 0, cells = 0, ids = 0;
    double rho_max = 0.0;
    for (int32_t r = 0; r < nrep; ++r) {
        Rep& R = P->reps[r];
        std::memset(&R, 0, sizeof(R));
        if (n_rep[r] <= 0) return fail(MD_ERR_INVALID_ARG, "every replica needs at least one atom");
        int64_t nc_tot = 1;
        for (int a = 0; a < 3; ++a) {
            const double L = box_rep[3 * r + a];
            if (!(std::isfinite(L) && L > 0.0)) return fail(MD_ERR_INVALID_ARG, "box sides must be > 0");
            const double q = std::floor(L / rl);
            if (q < 3.0)
                return fail(MD_ERR_BOX_TOO_SMALL, "replica " + std::to_string(r) +
                                                      ": fewer than 3 cells of side >= rc + skin");
            if (q > MAX_NC) return fail(MD_ERR_CELL_OVERFLOW, "more than 1023 cells along an axis");
            R.nc[a] = int32_t(q);
            R.L[a] = L;
            R.w[a] = L / double(R.nc[a]);
            R.s[a] = double(R.nc[a]) / L;
            R.wf[a] = float(R.w[a]);
            R.wlo[a] = float(R.w[a] - double(R.wf[a]));
            nc_tot *= R.nc[a];
        }
        R.kz = p->cell_block > 0 ? pow2_floor(std::min(p->cell_block, R.nc[2])) : 0;   // 0: chosen in md_create
        R.n = int32_t(n_rep[r]);
        R.slot0 = slot;
        R.tile0 = int32_t(slot / TILE);
        R.ntiles = int32_t((n_rep[r] + TILE - 1) / TILE);
        R.cell0 = int32_t(cells);
        R.ncells = int32_t(nc_tot);
        R.id0 = int32_t(ids);
        slot += int64_t(R.ntiles) * TILE;
        cells += nc_tot;
        ids += n_rep[r];
        rho_max = std::max(rho_max, double(n_rep[r]) / (R.L[0] * R.L[1] * R.L[2]));
        if (slot > MAX_SLOTS || cells > (int64_t(1) << 30))
            return fail(MD_ERR_CELL_OVERFLOW, "more than 2^26 atom slots or 2^30 cells");
    }
    P->nslots = slot;
    P->ntiles = int32_t(slot / TILE);
    P->ncells = int32_t(cells);
    P->nchunks = int32_t((cells + SCAN_CHUNK - 1) / SCAN_CHUNK);
    P->n_total = ids;
    P->tile_rep.resize(P->ntiles);
    for (int32_t r = 0; r < nrep; ++r)
        for (int32_t k = 0; k < P->reps[r].ntiles; ++k) P->tile_rep[P->reps[r].tile0 + k] = r;
    P->cell_rep.resize(size_t(P->ncells));
    for (int32_t r = 0; r < nrep; ++r)
        for (int32_t k = 0; k < P->reps[r].ncells; ++k) P->cell_rep[size_t(P->reps[r].cell0) + k] = r;
    if (p->nbr_capacity > 0) {
        P->cap = p->nbr_capacity;
    } else {
        const double mean = 4.0 / 3.0 * M_PI * rl * rl * rl * rho_max;
        P->cap = std::max(8, int(std::ceil(1.5 * mean + 16.0)));
        P->cap = (P->cap + 3) & ~3;
    }
    if (P->cap > 4096) return fail(MD_ERR_INVALID_ARG, "nbr_capacity above 4096");
    P->series_cap = 1024;
    return MD_OK;
}

// CTAs per replica of the props reduction: one warp partial per thread of the first pass (32
// tiles of 4 warps per CTA of 128 threads), so the pass is one memory round
int32_t props_split(const Plan& P)
{
    int32_t max_tiles = 1;
    for (const Rep& R : P.reps) max_tiles = std::max(max_tiles, R.ntiles);
    return std::max(1, std::min(PROPS_SPLIT_MAX, (max_tiles + 31) / 32));
}

size_t carve(const Plan& P, char* base, Arrays* A)
{
    Carver c{base};
    Arrays a;
    std::memset(&a, 0, sizeof(a));
    const size_t ns = size_t(P.nslots);
    const bool f64 = P.mode == MD_FP64, f32 = P.mode == MD_FP32;
    for (int b = 0; b < 2; ++b) {
        if (f64) a.pos64[b] = c.take<double4_32a>(ns);
        else a.pos32[b] = c.take<float4>(ns);
    }
    for (int q = 0; q < 3; ++q) a.xl[q] = c.take<double>(ns);
    for (int q = 0; q < 3; ++q) {
        if (f32) a.v32[q] = c.take<float>(ns);
        else a.v[q] = c.take<double>(ns);
    }
    a.f = c.take<double4_32a>(ns);
    a.wvir = c.take<double>(ns);
    a.id = c.take<int32_t>(ns);
    a.slot_of_id = c.take<int32_t>(size_t(P.n_total));
    a.cell = c.take<int32_t>(ns);
    a.layer = c.take<int32_t>(ns);
    a.nbr_count = c.take<int32_t>(ns);
    a.W = c.take<uint32_t>(ns * size_t(P.cap));
    if (P.rule == MD_REBUILD_DISP) a.xref = c.take<float4>(ns);
    a.perm = c.take<int32_t>(ns);
    if (!f64) a.psort = c.take<float4>(ns + PSORT_PAD);       // readable past the last atom
    if (!f64) a.tile_win = c.take<int2>(size_t(P.ntiles) * 9);
    if (!f64) {
        a.fbuf = c.take<float4>(ns);
        a.wbuf = c.take<float>(ns);
    }
    if (!f64) {
        const size_t nsub = size_t(8) * size_t(P.ncells);
        a.psub = c.take<float4>(ns);
        a.scount = c.take<int32_t>(nsub);
        a.sstart = c.take<int32_t>(nsub + 1);
        a.schunk = c.take<int32_t>((nsub + SCAN_CHUNK - 1) / SCAN_CHUNK);
    }
    if (!f32) for (int q = 0; q < 3; ++q) a.tmp_d[q] = c.take<double>(ns);
    for (int q = 0; q < 3; ++q) a.tmp_v[q] = c.take<double>(ns);
    for (int q = 0; q < 2; ++q) a.tmp_i[q] = c.take<int32_t>(ns);
    if (f64) a.tmp_p64 = c.take<double4_32a>(ns);
    else a.tmp_p32 = c.take<float4>(ns);
    a.ccount = c.take<int32_t>(size_t(P.ncells));
    a.cstart = c.take<int32_t>(size_t(P.ncells) + 1);
    if (!f64) a.ckeep = c.take<int2>(size_t(P.ncells));
    a.chunk = c.take<int32_t>(size_t(P.nchunks));
    a.tile_rep = c.take<int32_t>(size_t(P.ntiles));
    a.rb_tiles = c.take<int32_t>(size_t(P.ntiles));
    a.cell_rep = c.take<int32_t>(size_t(P.ncells));
    a.rb_base = c.take<int32_t>(size_t(P.nrep));
    a.warp_part = c.take<double>(size_t(P.ntiles) * (TILE / 32) * NPROP);
    a.slice_part = c.take<double>(size_t(P.nrep) * props_split(P) * NPROP);
    a.rep = c.take<Rep>(size_t(P.nrep));
    a.rs = c.take<RepState>(size_t(P.nrep));
    a.props = c.take<md_props>(size_t(P.nrep));
    a.series = c.take<double>(size_t(P.nrep) * P.series_cap * SERIES_COLS);
    a.g = c.take<Global>(1);
    a.sm_claim = c.take<int32_t>(size_t(SM_RANGES) + 1);
    for (int q = 0; q < 3; ++q) a.xchg[q] = c.take<double>(size_t(P.n_total) * 3);
    if (A) *A = a;
    return (c.off + 255) & ~size_t(255);
}

}  // namespace

namespace gbmd {
// lets other translation units of the library report through md_last_error
int set_last_error(int code, const char* msg)
{
    g_last_error = msg ? msg : "";
    return code;
}
}  // namespace gbmd

struct md_system {
    struct EvPair {
        cudaEvent_t a, b;
        int phase;
    };
    md_params p;
    Plan plan;
    Arrays A;
    Scal S;
    Launch L;
    int cur = 0;
    int nsm = 0;
    int smem_per_sm = 0;          // shared memory per SM and the per-CTA opt-in maximum, bytes
    int smem_per_cta = 0;
    int64_t host_step = 0;
    bool binned_fresh = false;
    md_tuning tune;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // per-phase timers (CUDA events on the system's stream) and kernel-launch counts
    bool timing = false;
    long long graph_rebuilds_seen = 0;
    std::vector<EvPair> pending;
    std::vector<cudaEvent_t> pool;
    double ms[MD_NPHASE] = {0};
    int64_t calls[MD_NPHASE] = {0};
    int64_t launches[MD_NPHASE] = {0};

    // CUDA graphs of GRAPH_STEPS steps each (one per starting position buffer)
    static constexpr int GRAPH_STEPS = 16;
    struct GraphEntry {
        int cur0, steps;
        uint32_t props_mask;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    struct AdjGraph {                 // captured segments of md_adjoint (kind 0 forward, 1 recompute
        const void* work;             // with snapshots, 2 reverse), for one adjoint workspace
        int32_t nsteps, ckpt, kind, steps, buf0, flags;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
    };
    std::vector<AdjGraph> adj_graphs;
    int64_t host_series_rows = 0;     // series rows issued (props steps since creation/clear)
    // VACF / MSD measurement (md_dyn_*): buffers in the caller's d_work, origins kept on the host
    bool dyn_on = false;
    DynView dyn{};
    int32_t dyn_nlag = 0, dyn_every = 0, dyn_norg = 0;
    int64_t dyn_samples = 0;
    int64_t dyn_start[DYN_MAX_ORG] = {0};
    std::vector<int64_t> dyn_counts;
    cudaStream_t aux = nullptr;       // captures the IF-node bodies
    cudaStream_t gstream = nullptr;   // captures and replays the graphs (the caller's stream may be
                                      // the legacy default stream, which cannot be captured)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaStream_t rstream = nullptr;   // md_adjoint's reverse walks, overlapping the recomputes
    cudaEvent_t ev_rc[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};

    void drop_graphs()
    {
        for (auto& g : graphs) {
            cudaGraphExecDestroy(g.exec);
            cudaGraphDestroy(g.graph);
        }
        graphs.clear();
        for (auto& g : adj_graphs) {
            cudaGraphExecDestroy(g.exec);
            cudaGraphDestroy(g.graph);
        }
        adj_graphs.clear();
    }

    cudaEvent_t take_event()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    ~md_system()
    {
        for (auto& pr : pending) { cudaEventDestroy(pr.a); cudaEventDestroy(pr.b); }
        for (auto e : pool) cudaEventDestroy(e);
        drop_graphs();
        if (aux) cudaStreamDestroy(aux);
        if (gstream) cudaStreamDestroy(gstream);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (rstream) cudaStreamDestroy(rstream);
        for (int k = 0; k < 2; ++k) {
            if (ev_rc[k]) cudaEventDestroy(ev_rc[k]);
            if (ev_rev[k]) cudaEventDestroy(ev_rev[k]);
        }
    }
};

namespace {

// Brackets one phase of work: counts its kernel launches and, with timing on, records a pair
// of events around it on the system's stream.
struct Phase {
    md_system* s;
    int ph;
    cudaEvent_t b = nullptr;
    Phase(md_system* s_, int ph_, int nlaunch) : s(s_), ph(ph_)
    {
        s->launches[ph] += nlaunch;
        if (s->timing) {
            s->calls[ph] += 1;            // timed intervals: the divisor of the summed milliseconds
            cudaEvent_t a = s->take_event();
            b = s->take_event();
            cudaEventRecord(a, s->L.stream);
            s->pending.push_back({a, b, ph});
        }
    }
    ~Phase()
    {
        if (b) cudaEventRecord(b, s->L.stream);
    }
};

}  // namespace

namespace {

void fill_scal(md_system* s)
{
    const md_params& p = s->p;
    const Plan& P = s->plan;
    Scal& S = s->S;
    std::memset(&S, 0, sizeof(S));
    S.nslots = P.nslots;
    S.ntiles = P.ntiles;
    S.nrep = P.nrep;
    S.ncells = P.ncells;
    S.nchunks = P.nchunks;
    S.cap = P.cap;
    S.mode = P.mode;
    S.rule = P.rule;
    S.reorder_every = p.reorder_every;
    S.series_cap = P.series_cap;
    S.shift = p.shift_energy;
    S.nsub = int64_t(8) * P.ncells;
    S.nschunks = int32_t((S.nsub + SCAN_CHUNK - 1) / SCAN_CHUNK);
    S.props_split = props_split(P);
    S.dt = p.dt;
    S.mass = p.mass;
    S.c = p.dt / (2.0 * p.mass);
    S.half_skin = 0.5 * p.skin;
    {
        // |fl(a) - fl(b) - (a - b)| for cell-local coordinates |a|, |b| < 2 (w + skin): two
        // roundings of the positions plus one of the difference, per axis, summed over 3 axes
        double wmax = 0.0;
        for (const Rep& R : P.reps) for (int a = 0; a < 3; ++a) wmax = std::max(wmax, R.w[a]);
        const double ulp = (P.mode == MD_FP64) ? std::ldexp(1.0, -52) : std::ldexp(1.0, -23);
        S.disp_margin = 3.0 * 3.0 * ulp * 2.0 * (wmax + p.skin);
    }
    const double rl = p.rc + p.skin;
    S.rc2d = p.rc * p.rc;
    S.rl2d = rl * rl;
    S.sig2d = p.sigma * p.sigma;
    S.eps4d = 4.0 * p.eps;
    S.eps48d = 48.0 * p.eps;
    double uc = 0.0;
    if (p.shift_energy) {
        const double q2 = S.sig2d / S.rc2d, q6 = q2 * q2 * q2;
        uc = 4.0 * p.eps * (q6 * q6 - q6);
    }
    S.ucd = uc;
    S.adj_eps144_over_sig = float(144.0 * p.eps / p.sigma);
    S.adj_eps24_over_sig = float(24.0 * p.eps / p.sigma);
    {
        // du_c/dsigma: zero when r_c moves with sigma (the WCA cutoff 2^(1/6) sigma)
        const bool scales = std::fabs(p.rc / p.sigma - std::pow(2.0, 1.0 / 6.0)) < 1e-9;
        double duc = 0.0;
        if (p.shift_energy && !scales) {
            const double q2 = S.sig2d / S.rc2d, q6 = q2 * q2 * q2;
            duc = 24.0 * p.eps * q6 * (2.0 * q6 - 1.0) / p.sigma;
        }
        S.adj_ducf = float(duc);
    }
    S.rc2f = float(S.rc2d);
    S.rl2f = float(S.rl2d);
    S.sig2f = float(S.sig2d);
    S.eps4f = float(S.eps4d);
    S.eps48f = float(S.eps48d);
    S.ucf = float(uc);
}

int apply_tuning(md_system* s)
{
    const int per_sm = std::max(1, s->tune.ctas_per_sm);
    s->L.grid = std::max(1, s->nsm * per_sm);
    s->L.nsm = std::max(1, s->nsm);
    prime_rebuild_grids(s->S, s->L);
    s->L.step_block = TILE;
    s->L.build_block = TILE;
    s->L.nbr_batch = s->tune.nbr_batch;
    s->L.build_batch = s->tune.build_batch;
    s->L.build_stage = s->tune.build_stage == 1 ? 1 : 0;
    s->L.step_kernel = (s->S.mode == MD_FP64) ? 1 : s->tune.step_kernel;
    // the list-free kernel reads each row of cells as a run of slots: atoms reorder at every rebuild
    // tune.reorder_every: -1 = at every rebuild, else every that many steps
    s->S.reorder_every = (s->L.step_kernel == 4 || s->tune.reorder_every < 0) ? 0 : s->tune.reorder_every;
    s->S.half_list = (s->L.step_kernel == 5) ? 1 : 0;      // W keeps each pair once
    bulk_shape(s->S, per_sm, s->smem_per_sm, s->smem_per_cta, &s->L.bulk_rows, &s->L.bulk_smem);
    stage_shape(per_sm, s->smem_per_sm, &s->L.stage_cap, &s->L.stage_smem);
    s->L.ctas_req = per_sm;
    // a persistent grid larger than what can be resident would run as a trailing second wave
    s->L.grid_step = s->nsm * std::min(per_sm, step_ctas_per_sm(s->S, s->L));
    return MD_OK;
}

int latch_error(md_system* s)
{
    Global g;
    GBMD_CUDA(cudaMemcpyAsync(&g, s->A.g, sizeof(Global), cudaMemcpyDeviceToHost, s->L.stream));
    GBMD_CUDA(cudaStreamSynchronize(s->L.stream));
    if (g.err == 0) return MD_OK;
    const int zero = 0;
    GBMD_CUDA(cudaMemcpyAsync(&s->A.g->err, &zero, sizeof(int), cudaMemcpyHostToDevice, s->L.stream));
    GBMD_CUDA(cudaStreamSynchronize(s->L.stream));
    // a non-finite input or state is the root cause of anything else it triggers (a NaN position
    // binned to cell 0 can overflow that cell's neighbours), so it is reported first
    if (g.err & ERR_NONFINITE) return fail(MD_ERR_NONFINITE, "non-finite position, velocity or displacement");
    if (g.err & ERR_NBR_OVERFLOW)
        return fail(MD_ERR_NBR_OVERFLOW, "neighbour capacity " + std::to_string(s->plan.cap) +
                                             " exceeded (an atom had " + std::to_string(g.max_nbr_seen) + ")");
    if (g.err & ERR_TIMEOUT) return fail(MD_ERR_TIMEOUT, "a bounded device wait gave up");
    return fail(MD_ERR_CUDA, "unknown device error word");
}

int load_state(md_system* s, const double* x, const double* v)
{
    const size_t bytes = size_t(s->plan.n_total) * 3 * sizeof(double);
    GBMD_CUDA(cudaMemcpyAsync(s->A.xchg[0], x, bytes, cudaMemcpyDefault, s->L.stream));
    GBMD_CUDA(cudaMemcpyAsync(s->A.xchg[1], v, bytes, cudaMemcpyDefault, s->L.stream));
    s->cur = 0;
    GBMD_CUDA(launch_set_state(s->A, s->S, s->L, s->cur));
    GBMD_CUDA(launch_force_rebuild(s->A, s->S, s->L, 1));
    GBMD_CUDA(launch_rebuild(s->A, s->S, s->L, s->cur, true));
    s->host_step = 0;
    s->host_series_rows = 0;
    s->binned_fresh = false;
    return MD_OK;
}

cudaError_t ensure_graph_streams(md_system* s)
{
    cudaError_t e = cudaSuccess;
    if (!s->aux) e = cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess && !s->gstream) e = cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !s->ev_in) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess && !s->ev_out) e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming);
    return e;
}

cudaError_t ensure_adj_streams(md_system* s)
{
    cudaError_t e = ensure_graph_streams(s);
    if (e == cudaSuccess && !s->rstream) e = cudaStreamCreateWithFlags(&s->rstream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (!s->ev_rc[k]) e = cudaEventCreateWithFlags(&s->ev_rc[k], cudaEventDisableTiming);
        if (e == cudaSuccess && !s->ev_rev[k]) e = cudaEventCreateWithFlags(&s->ev_rev[k], cudaEventDisableTiming);
    }
    return e;
}

// Inside a capture on stream st: the fused step kernel from position buffer cur (with S), then an
// IF node whose body (captured on s->aux) is the rebuild sequence for the new buffer.  The step
// kernel opens the node only when some replica's refresh criterion fired.
cudaError_t capture_step_and_rebuild(md_system* s, const Scal& S, cudaStream_t st, int cur, bool props)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    cudaError_t err = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd);
    cudaGraphConditionalHandle h = 0;
    if (err == cudaSuccess) err = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    Launch L = s->L;
    L.stream = st;
    L.cond = h;
    L.use_cond = 1;
    if (err == cudaSuccess) err = launch_step(s->A, S, L, cur, props);
    const int nxt = cur ^ 1;
    if (err == cudaSuccess) err = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (err == cudaSuccess) err = cudaGraphAddNode(&node, g, deps, ed, nd, &cp);
    if (err == cudaSuccess) err = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (err == cudaSuccess)
        err = cudaStreamBeginCaptureToGraph(s->aux, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        Launch Lb = s->L;
        Lb.stream = s->aux;
        Lb.use_cond = 0;
        Lb.in_graph = 1;
        cudaError_t e2 = launch_bin_order(s->A, S, Lb, nxt, false);
        if (e2 == cudaSuccess) e2 = launch_reorder(s->A, S, Lb, nxt);
        if (e2 == cudaSuccess) e2 = launch_build_only(s->A, S, Lb, nxt);
        cudaGraph_t body = nullptr;
        err = cudaStreamEndCapture(s->aux, &body);
        if (err == cudaSuccess) err = e2;
    }
    return err;
}

// Captures what body(st) issues on the library's capture stream into an instantiated graph.
template <class F>
int capture_exec(md_system* s, F body, cudaGraph_t* g_out, cudaGraphExec_t* e_out)
{
    GBMD_CUDA(ensure_graph_streams(s));
    cudaStream_t st = s->gstream;
    GBMD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = body(st);
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(st, &graph);
    if (err == cudaSuccess) err = e_end;
    if (err != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(MD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(err));
    }
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiate(&exec, graph, 0);
    if (err != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(MD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(err));
    }
    *g_out = graph;
    *e_out = exec;
    return MD_OK;
}

// Replays a graph on the capture stream, ordered after and before the caller's stream.
int replay(md_system* s, cudaGraphExec_t exec)
{
    GBMD_CUDA(cudaEventRecord(s->ev_in, s->L.stream));
    GBMD_CUDA(cudaStreamWaitEvent(s->gstream, s->ev_in, 0));
    GBMD_CUDA(cudaGraphLaunch(exec, s->gstream));
    GBMD_CUDA(cudaEventRecord(s->ev_out, s->gstream));
    GBMD_CUDA(cudaStreamWaitEvent(s->L.stream, s->ev_out, 0));
    return MD_OK;
}

// Capture `steps` steps starting from position buffer cur0 (bit j of props_mask: step j also
// reduces the props into the time series).  Steps without a rebuild launch one kernel.
int capture_graph(md_system* s, int cur0, int steps, uint32_t props_mask, cudaGraphExec_t* out_exec)
{
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int rc = capture_exec(
        s,
        [&](cudaStream_t st) {
            cudaError_t err = cudaSuccess;
            int cur = cur0;
            for (int k = 0; k < steps && err == cudaSuccess; ++k) {
                err = capture_step_and_rebuild(s, s->S, st, cur, (props_mask >> k) & 1u);
                cur ^= 1;
            }
            return err;
        },
        &graph, &exec);
    if (rc) return rc;
    s->graphs.push_back({cur0, steps, props_mask, graph, exec});
    *out_exec = exec;
    return MD_OK;
}

}  // namespace

extern "C" {

const char* md_last_error(void) { return g_last_error.c_str(); }

size_t md_workspace_bytes_batch(const md_params* p, int32_t nrep, const int64_t* n_rep, const double* box_rep)
{
    Plan P;
    if (make_plan(p, nrep, n_rep, box_rep, &P) != MD_OK) return 0;
    return carve(P, nullptr, nullptr);
}

size_t md_workspace_bytes(const md_params* p)
{
    if (!p) return 0;
    const int64_t n = p->n;
    return md_workspace_bytes_batch(p, 1, &n, p->box);
}

int md_create_batch(const md_params* p, int32_t nrep, const int64_t* n_rep, const double* box_rep,
                    void* d_workspace, size_t workspace_bytes, const double* x0, const double* v0,
                    void* stream, md_system** out)
{
    if (!out) return fail(MD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!x0 || !v0) return fail(MD_ERR_INVALID_ARG, "x0 and v0 are required");
    Plan P;
    int rc = make_plan(p, nrep, n_rep, box_rep, &P);
    if (rc) return rc;
    const size_t need = carve(P, nullptr, nullptr);
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return fail(MD_ERR_WORKSPACE, "workspace missing or not 256-byte aligned");
    if (workspace_bytes < need)
        return fail(MD_ERR_WORKSPACE, "workspace has " + std::to_string(workspace_bytes) + " bytes, needs " +
                                          std::to_string(need));
    cudaPointerAttributes attr;
    GBMD_CUDA(cudaPointerGetAttributes(&attr, d_workspace));
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(MD_ERR_WORKSPACE, "workspace is not device memory");
    int dev = 0;
    GBMD_CUDA(cudaGetDevice(&dev));
    if (attr.device != dev) return fail(MD_ERR_WORKSPACE, "workspace lives on another device than the current one");

    md_system* s = new (std::nothrow) md_system();
    if (!s) return fail(MD_ERR_INVALID_ARG, "out of host memory");
    s->p = *p;
    s->plan = std::move(P);
    s->ws = d_workspace;
    s->ws_bytes = workspace_bytes;
    carve(s->plan, static_cast<char*>(d_workspace), &s->A);
    fill_scal(s);
    s->L.stream = static_cast<cudaStream_t>(stream);
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) { delete s; return fail(MD_ERR_CUDA, cudaGetErrorString(e)); }
    s->nsm = prop.multiProcessorCount;
    // blocks of the cell order: about sqrt(rows of cells per SM's slot range) planes, rounded down
    // to a power of two, at most 8 (measured on the 4M-atom WCA fluid: 4 and 8 equally fast, 12
    // slower, 1 slowest)
    for (Rep& R : s->plan.reps) {
        if (R.kz > 0) continue;
        const double rows = double(R.nc[1]) * double(R.nc[2]);
        const double per_range = double(s->plan.nslots) / double(std::max(1, s->nsm)) * rows / double(R.n);
        const int kz = int(std::lround(std::sqrt(per_range)));
        R.kz = pow2_floor(std::max(1, std::min(std::min(kz, 8), int(R.nc[2]))));
    }
    s->smem_per_sm = int(prop.sharedMemPerMultiprocessor);
    s->smem_per_cta = int(prop.sharedMemPerBlockOptin);
    s->tune.ctas_per_sm = 8;            // the measured best for the 4M-atom fluid (the tuner searches 4-16)
    s->tune.nbr_batch = 2;
    s->tune.build_batch = 2;
    s->tune.use_graph = 1;
    s->tune.step_kernel = 1;
    s->tune.reorder_every = s->p.reorder_every == 0 ? -1 : s->p.reorder_every;
    s->tune.build_stage = 2;            // 2 = off (0 keeps the current value in md_set_tuning)
    apply_tuning(s);

    auto bail = [&](int code) { delete s; return code; };
    if (cudaMemsetAsync(d_workspace, 0, need, s->L.stream) != cudaSuccess) return bail(fail(MD_ERR_CUDA, "memset"));
    if (cudaMemcpyAsync(s->A.rep, s->plan.reps.data(), sizeof(Rep) * s->plan.nrep, cudaMemcpyHostToDevice,
                        s->L.stream) != cudaSuccess ||
        cudaMemcpyAsync(s->A.tile_rep, s->plan.tile_rep.data(), sizeof(int32_t) * s->plan.ntiles,
                        cudaMemcpyHostToDevice, s->L.stream) != cudaSuccess ||
        cudaMemcpyAsync(s->A.cell_rep, s->plan.cell_rep.data(), sizeof(int32_t) * s->plan.ncells,
                        cudaMemcpyHostToDevice, s->L.stream) != cudaSuccess)
        return bail(fail(MD_ERR_CUDA, "upload of the replica table"));
    rc = load_state(s, x0, v0);
    if (rc) return bail(rc);
    rc = latch_error(s);
    if (rc) return bail(rc);
    *out = s;
    return MD_OK;
}

int md_create(const md_params* p, void* d_workspace, size_t workspace_bytes, const double* x0, const double* v0,
              void* stream, md_system** out)
{
    if (!p) return fail(MD_ERR_INVALID_ARG, "params is NULL");
    const int64_t n = p->n;
    return md_create_batch(p, 1, &n, p->box, d_workspace, workspace_bytes, x0, v0, stream, out);
}

int md_destroy(md_system* s)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    cudaStreamSynchronize(s->L.stream);
    delete s;
    return MD_OK;
}

int md_bin_cells(md_system* s)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    GBMD_CUDA(launch_force_rebuild(s->A, s->S, s->L, s->S.reorder_every == 0 ? 1 : 0));
    GBMD_CUDA(launch_bin_only(s->A, s->S, s->L, s->cur, false));
    s->binned_fresh = true;
    return MD_OK;
}

int md_build_neighbours(md_system* s)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    if (!s->binned_fresh) {
        GBMD_CUDA(launch_force_rebuild(s->A, s->S, s->L, 0));
        GBMD_CUDA(launch_bin_only(s->A, s->S, s->L, s->cur, false));
    }
    GBMD_CUDA(launch_build_only(s->A, s->S, s->L, s->cur));
    s->binned_fresh = false;
    return MD_OK;
}

int md_compute_forces(md_system* s)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    Phase t(s, MD_PHASE_OTHER, 1);
    GBMD_CUDA(launch_forces(s->A, s->S, s->L, s->cur));
    return MD_OK;
}

int md_integrate(md_system* s, int32_t nsteps)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    if (nsteps < 0) return fail(MD_ERR_INVALID_ARG, "nsteps < 0");
    if (s->binned_fresh) {      // a md_bin_cells without md_build_neighbours: finish the rebuild
        Phase t(s, MD_PHASE_BUILD, build_kernels(s->S, s->L));
        GBMD_CUDA(launch_build_only(s->A, s->S, s->L, s->cur));
        s->binned_fresh = false;
    }
    int32_t k = 0;
    if (s->tune.use_graph == 1) {
        // replay cached graphs of 16 steps, or of 1 step for the remainder; a graph is keyed by
        // its starting buffer, length and which of its steps reduce the props
        while (k < nsteps) {
            const int G = (nsteps - k >= md_system::GRAPH_STEPS) ? md_system::GRAPH_STEPS : 1;
            uint32_t mask = 0;
            for (int j = 0; j < G; ++j)
                if (s->p.props_every > 0 && ((s->host_step + j) % s->p.props_every == 0)) mask |= 1u << j;
            cudaGraphExec_t exec = nullptr;
            for (auto& g : s->graphs)
                if (g.cur0 == s->cur && g.steps == G && g.props_mask == mask) exec = g.exec;
            if (!exec) {
                const int rc = capture_graph(s, s->cur, G, mask, &exec);
                if (rc) return rc;
            }
            Phase t(s, MD_PHASE_STEP,
                    G * step_kernels(s->S, s->L) + (s->S.mode == MD_FP64 ? __builtin_popcount(mask) : 0));
            const int rc = replay(s, exec);
            if (rc) return rc;
            k += G;
            s->host_step += G;
            s->host_series_rows += __builtin_popcount(mask);
            if (G & 1) s->cur ^= 1;
        }
    }
    for (; k < nsteps; ++k) {
        const bool props = s->p.props_every > 0 && (s->host_step % s->p.props_every == 0);
        if (props) s->host_series_rows += 1;
        {
            Phase t(s, MD_PHASE_STEP, step_kernels(s->S, s->L) + (props && s->S.mode == MD_FP64 ? 1 : 0));
            GBMD_CUDA(launch_step(s->A, s->S, s->L, s->cur, props));
        }
        s->cur ^= 1;
        {
            Phase t(s, MD_PHASE_BIN, 7);
            GBMD_CUDA(launch_bin_order(s->A, s->S, s->L, s->cur, false));
        }
        {
            Phase t(s, MD_PHASE_REORDER, 2);
            GBMD_CUDA(launch_reorder(s->A, s->S, s->L, s->cur));
        }
        {
            Phase t(s, MD_PHASE_BUILD, build_kernels(s->S, s->L));
            GBMD_CUDA(launch_build_only(s->A, s->S, s->L, s->cur));
        }
        s->host_step += 1;
    }
    return MD_OK;
}

int md_set_timing(md_system* s, int32_t enable)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    s->timing = enable != 0;
    return MD_OK;
}

int md_get_timing(md_system* s, double* ms, int64_t* calls, int64_t* launches)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    GBMD_CUDA(cudaStreamSynchronize(s->L.stream));
    {
        // rebuild sequences inside graphs ran only when their IF node opened: count them here
        long long gr = 0;
        GBMD_CUDA(cudaMemcpy(&gr, &s->A.g->graph_rebuilds, sizeof(gr), cudaMemcpyDeviceToHost));
        s->launches[MD_PHASE_BUILD] += (REBUILD_KERNELS - 3 + build_kernels(s->S, s->L)) * (gr - s->graph_rebuilds_seen);
        s->graph_rebuilds_seen = gr;
    }
    for (auto& pr : s->pending) {
        float t = 0.0f;
        GBMD_CUDA(cudaEventElapsedTime(&t, pr.a, pr.b));
        s->ms[pr.phase] += double(t);
        s->pool.push_back(pr.a);
        s->pool.push_back(pr.b);
    }
    s->pending.clear();
    for (int k = 0; k < MD_NPHASE; ++k) {
        if (ms) ms[k] = s->ms[k];
        if (calls) calls[k] = s->calls[k];
        if (launches) launches[k] = s->launches[k];
        s->ms[k] = 0.0;
        s->calls[k] = 0;
        s->launches[k] = 0;
    }
    return MD_OK;
}

int md_reduce_props(md_system* s, md_props* out)
{
    if (!s || !out) return fail(MD_ERR_INVALID_ARG, "system or out is NULL");
    {
        Phase t(s, MD_PHASE_PROPS, 3);
        GBMD_CUDA(launch_props(s->A, s->S, s->L, s->cur, true, false));
    }
    GBMD_CUDA(cudaMemcpyAsync(out, s->A.props, sizeof(md_props) * s->plan.nrep, cudaMemcpyDeviceToHost,
                              s->L.stream));
    return latch_error(s);
}

int md_get_series(md_system* s, double* out, int32_t max_rows, int32_t* rows)
{
    if (!s || !out || !rows || max_rows < 0) return fail(MD_ERR_INVALID_ARG, "bad arguments");
    GBMD_CUDA(cudaStreamSynchronize(s->L.stream));
    const int64_t written = s->host_series_rows;
    const int64_t cap = s->plan.series_cap;
    const int32_t nr = int32_t(std::min<int64_t>(std::min<int64_t>(written, cap), max_rows));
    const int nrep = s->plan.nrep;
    // the last nr rows, oldest first: ring rows (written - nr + q) % cap, [row][replica][col]
    for (int32_t q = 0; q < nr; ++q) {
        const int64_t row = (written - nr + q) % cap;
        GBMD_CUDA(cudaMemcpy2DAsync(out + size_t(q) * SERIES_COLS, sizeof(double) * SERIES_COLS * max_rows,
                                    s->A.series + size_t(row) * nrep * SERIES_COLS, sizeof(double) * SERIES_COLS,
                                    sizeof(double) * SERIES_COLS, nrep, cudaMemcpyDeviceToHost, s->L.stream));
    }
    *rows = nr;
    return latch_error(s);
}

int md_clear_series(md_system* s)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    std::vector<RepState> st(s->plan.nrep);
    GBMD_CUDA(cudaMemcpyAsync(st.data(), s->A.rs, sizeof(RepState) * st.size(), cudaMemcpyDeviceToHost,
                              s->L.stream));
    GBMD_CUDA(cudaStreamSynchronize(s->L.stream));
    for (auto& x : st) x.series_rows = 0;
    GBMD_CUDA(cudaMemcpyAsync(s->A.rs, st.data(), sizeof(RepState) * st.size(), cudaMemcpyHostToDevice,
                              s->L.stream));
    GBMD_CUDA(cudaStreamSynchronize(s->L.stream));
    s->host_series_rows = 0;
    return MD_OK;
}

int md_props_latest(md_system* s, double* dst)
{
    if (!s || !dst) return fail(MD_ERR_INVALID_ARG, "system or dst is NULL");
    if (s->host_series_rows == 0) return fail(MD_ERR_INVALID_ARG, "no props step has been issued (props_every = 0?)");
    const int64_t row = (s->host_series_rows - 1) % s->plan.series_cap;
    const size_t bytes = sizeof(double) * SERIES_COLS * s->plan.nrep;
    GBMD_CUDA(cudaMemcpyAsync(dst, s->A.series + size_t(row) * s->plan.nrep * SERIES_COLS, bytes, cudaMemcpyDefault,
                              s->L.stream));
    return MD_OK;
}

int md_get_state(md_system* s, double* x, double* v, double* f)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    if (!x && !v && !f) return MD_OK;
    {
        Phase t(s, MD_PHASE_OTHER, (v || f) ? 2 : 1);
        if (v || f) GBMD_CUDA(launch_forces(s->A, s->S, s->L, s->cur));
        GBMD_CUDA(launch_get_state(s->A, s->S, s->L, s->cur, v != nullptr, f != nullptr));
    }
    const size_t bytes = size_t(s->plan.n_total) * 3 * sizeof(double);
    if (x) GBMD_CUDA(cudaMemcpyAsync(x, s->A.xchg[0], bytes, cudaMemcpyDefault, s->L.stream));
    if (v) GBMD_CUDA(cudaMemcpyAsync(v, s->A.xchg[1], bytes, cudaMemcpyDefault, s->L.stream));
    if (f) GBMD_CUDA(cudaMemcpyAsync(f, s->A.xchg[2], bytes, cudaMemcpyDefault, s->L.stream));
    return latch_error(s);
}

int md_set_state(md_system* s, const double* x, const double* v)
{
    if (!s || !x || !v) return fail(MD_ERR_INVALID_ARG, "system, x and v are required");
    int rc = load_state(s, x, v);
    if (rc) return rc;
    return latch_error(s);
}

int md_get_cells(md_system* s, int32_t* cell)
{
    if (!s || !cell) return fail(MD_ERR_INVALID_ARG, "system or cell is NULL");
    int32_t* tmp = reinterpret_cast<int32_t*>(s->A.xchg[0]);
    GBMD_CUDA(launch_get_cells(s->A, s->S, s->L, tmp));
    GBMD_CUDA(cudaMemcpyAsync(cell, tmp, sizeof(int32_t) * s->plan.n_total, cudaMemcpyDefault, s->L.stream));
    return latch_error(s);
}

int md_get_neighbours(md_system* s, int32_t* counts, int32_t* nbr_ids, int32_t cap)
{
    if (!s || !counts || !nbr_ids || cap <= 0) return fail(MD_ERR_INVALID_ARG, "bad arguments");
    // counts staged in xchg[0]; rows staged in xchg[1] (6 int32 per atom) one id window at a time
    const int64_t n = s->plan.n_total;
    int32_t* dcounts = reinterpret_cast<int32_t*>(s->A.xchg[0]);
    int32_t* drows = reinterpret_cast<int32_t*>(s->A.xchg[1]);
    const int64_t window = std::max<int64_t>(1, (n * 6) / cap);
    for (int64_t lo = 0; lo < n; lo += window) {
        const int64_t hi = std::min(n, lo + window);
        GBMD_CUDA(launch_get_neighbours(s->A, s->S, s->L, dcounts, drows, cap, lo, hi));
        GBMD_CUDA(cudaMemcpyAsync(nbr_ids + lo * cap, drows, sizeof(int32_t) * (hi - lo) * cap, cudaMemcpyDefault,
                                  s->L.stream));
    }
    GBMD_CUDA(cudaMemcpyAsync(counts, dcounts, sizeof(int32_t) * n, cudaMemcpyDefault, s->L.stream));
    return latch_error(s);
}

int md_check(md_system* s)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    GBMD_CUDA(cudaGetLastError());
    return latch_error(s);
}

int md_set_chains(md_system* s, const md_chains* c)
{
    if (!s || !c) return fail(MD_ERR_INVALID_ARG, "system and chains are required");
    if (c->length < 0) return fail(MD_ERR_INVALID_ARG, "chain length must be >= 0");
    if (c->length > 0) {
        if (s->S.mode == MD_FP64) return fail(MD_ERR_INVALID_ARG, "chains need MD_MIXED or MD_FP32");
        if (!(std::isfinite(c->fene_k) && c->fene_k >= 0.0 && std::isfinite(c->fene_r0) && c->fene_r0 > 0.0 &&
              std::isfinite(c->bend_k) && std::isfinite(c->dihedral_k)))
            return fail(MD_ERR_INVALID_ARG, "fene_k >= 0, fene_r0 > 0 and finite bend_k, dihedral_k are required");
    }
    s->S.chain_len = c->length;
    s->S.ch_kb = float(c->fene_k);
    s->S.ch_r0sq = float(c->fene_r0 * c->fene_r0);
    s->S.ch_ka = float(c->bend_k);
    s->S.ch_kd = float(c->dihedral_k);
    s->drop_graphs();          // the parameters are baked into captured graphs
    return MD_OK;
}

int md_debug_set_error(md_system* s, int32_t status)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    int bits = 0;
    if (status == MD_ERR_NBR_OVERFLOW) bits = ERR_NBR_OVERFLOW;
    else if (status == MD_ERR_NONFINITE) bits = ERR_NONFINITE;
    else if (status == MD_ERR_TIMEOUT) bits = ERR_TIMEOUT;
    else return fail(MD_ERR_INVALID_ARG, "status must be MD_ERR_NBR_OVERFLOW, MD_ERR_NONFINITE or MD_ERR_TIMEOUT");
    GBMD_CUDA(launch_debug_error(s->A, s->L, bits, s->plan.cap + 1));
    return MD_OK;
}

// ---- VACF / MSD measurement ----------------------------------------------------------------
namespace {
int dyn_shape(const md_system* s, int32_t nlag, int32_t origin_every, int32_t* norg)
{
    if (!s || nlag <= 0 || origin_every <= 0) return fail(MD_ERR_INVALID_ARG, "need nlag > 0 and origin_every > 0");
    const int32_t k = (nlag + origin_every - 1) / origin_every;
    if (k > DYN_MAX_ORG)
        return fail(MD_ERR_INVALID_ARG, "nlag / origin_every may be at most " + std::to_string(DYN_MAX_ORG) +
                                            " (origins followed at once)");
    *norg = k;
    return MD_OK;
}

size_t dyn_carve(int64_t n, int32_t nlag, char* base, DynView* V)
{
    Carver c{base};
    DynView d{};
    d.n = n;
    d.xprev = c.take<double>(size_t(n) * 3);
    d.v0 = c.take<double>(size_t(DYN_MAX_ORG) * n * 3);
    d.dr = c.take<double>(size_t(DYN_MAX_ORG) * n * 3);
    d.part = c.take<double>(size_t(DYN_BLOCKS) * 2 * DYN_MAX_ORG);
    d.vacf = c.take<double>(size_t(nlag));
    d.msd = c.take<double>(size_t(nlag));
    if (V) *V = d;
    return (c.off + 255) & ~size_t(255);
}
}  // namespace

size_t md_dyn_workspace_bytes(const md_system* s, int32_t nlag, int32_t origin_every)
{
    int32_t norg = 0;
    if (dyn_shape(s, nlag, origin_every, &norg) != MD_OK) return 0;
    return dyn_carve(s->plan.n_total, nlag, nullptr, nullptr);
}

int md_dyn_begin(md_system* s, void* d_work, size_t work_bytes, int32_t nlag, int32_t origin_every)
{
    int32_t norg = 0;
    int rc = dyn_shape(s, nlag, origin_every, &norg);
    if (rc) return rc;
    const size_t need = dyn_carve(s->plan.n_total, nlag, nullptr, nullptr);
    if (!d_work || (reinterpret_cast<uintptr_t>(d_work) & 255u) || work_bytes < need)
        return fail(MD_ERR_WORKSPACE, "measurement buffer missing, misaligned or smaller than " + std::to_string(need) +
                                          " bytes");
    dyn_carve(s->plan.n_total, nlag, static_cast<char*>(d_work), &s->dyn);
    GBMD_CUDA(cudaMemsetAsync(s->dyn.vacf, 0, sizeof(double) * size_t(nlag), s->L.stream));
    GBMD_CUDA(cudaMemsetAsync(s->dyn.msd, 0, sizeof(double) * size_t(nlag), s->L.stream));
    s->dyn_on = true;
    s->dyn_nlag = nlag;
    s->dyn_every = origin_every;
    s->dyn_norg = norg;
    s->dyn_samples = 0;
    for (int b = 0; b < DYN_MAX_ORG; ++b) s->dyn_start[b] = -1;
    s->dyn_counts.assign(size_t(nlag), 0);
    return MD_OK;
}

int md_dyn_sample(md_system* s)
{
    if (!s || !s->dyn_on) return fail(MD_ERR_INVALID_ARG, "no measurement begun (md_dyn_begin)");
    const int64_t k = s->dyn_samples;
    DynStep P{};
    P.norg = s->dyn_norg;
    P.start = -1;
    if (k % s->dyn_every == 0) {                     // a new origin in the oldest slot
        const int b = int((k / s->dyn_every) % s->dyn_norg);
        s->dyn_start[b] = k;
        P.start = b;
    }
    for (int b = 0; b < DYN_MAX_ORG; ++b) {
        const int64_t lag = (b < s->dyn_norg && s->dyn_start[b] >= 0) ? k - s->dyn_start[b] : -1;
        P.lag[b] = (lag >= 0 && lag < s->dyn_nlag) ? int(lag) : -1;
        if (P.lag[b] >= 0) s->dyn_counts[size_t(P.lag[b])] += 1;
    }
    {
        Phase t(s, MD_PHASE_OTHER, 3);
        GBMD_CUDA(launch_forces(s->A, s->S, s->L, s->cur));
        GBMD_CUDA(launch_dyn_sample(s->A, s->S, s->L, s->dyn, P, s->cur));
    }
    s->dyn_samples = k + 1;
    return MD_OK;
}

int md_dyn_get(md_system* s, double* vacf, double* msd, int64_t* counts)
{
    if (!s || !s->dyn_on) return fail(MD_ERR_INVALID_ARG, "no measurement begun (md_dyn_begin)");
    const size_t nl = size_t(s->dyn_nlag);
    std::vector<double> a(nl), b(nl);
    GBMD_CUDA(cudaMemcpyAsync(a.data(), s->dyn.vacf, sizeof(double) * nl, cudaMemcpyDeviceToHost, s->L.stream));
    GBMD_CUDA(cudaMemcpyAsync(b.data(), s->dyn.msd, sizeof(double) * nl, cudaMemcpyDeviceToHost, s->L.stream));
    const int rc = latch_error(s);
    if (rc) return rc;
    const double n = double(s->plan.n_total);
    for (size_t k = 0; k < nl; ++k) {
        const double cnt = double(s->dyn_counts[k]);
        if (vacf) vacf[k] = cnt > 0 ? a[k] / (n * cnt) : 0.0;
        if (msd) msd[k] = cnt > 0 ? b[k] / (n * cnt) : 0.0;
        if (counts) counts[k] = s->dyn_counts[k];
    }
    return MD_OK;
}

int32_t md_nrep(const md_system* s) { return s ? s->plan.nrep : 0; }
int64_t md_natoms(const md_system* s) { return s ? s->plan.n_total : 0; }
int32_t md_nbr_capacity(const md_system* s) { return s ? s->plan.cap : 0; }

int md_cells_per_axis(const md_system* s, int32_t r, int32_t* nc)
{
    if (!s || !nc || r < 0 || r >= s->plan.nrep) return fail(MD_ERR_INVALID_ARG, "bad arguments");
    for (int a = 0; a < 3; ++a) nc[a] = s->plan.reps[r].nc[a];
    return MD_OK;
}

int md_set_tuning(md_system* s, const md_tuning* t)
{
    if (!s || !t) return fail(MD_ERR_INVALID_ARG, "bad arguments");
    if (t->ctas_per_sm < 0 || t->ctas_per_sm > 64) return fail(MD_ERR_INVALID_ARG, "ctas_per_sm in 0..64");
    if (t->nbr_batch && t->nbr_batch != 2 && t->nbr_batch != 4 && t->nbr_batch != 8)
        return fail(MD_ERR_INVALID_ARG, "nbr_batch must be 2, 4 or 8");
    if (t->build_batch && t->build_batch != 1 && t->build_batch != 2 && t->build_batch != 4 && t->build_batch != 32)
        return fail(MD_ERR_INVALID_ARG, "build_batch must be 1, 2, 4 or 32");
    if (t->use_graph < 0 || t->use_graph > 2) return fail(MD_ERR_INVALID_ARG, "use_graph must be 0, 1 or 2");
    if (t->step_kernel < 0 || t->step_kernel > 5) return fail(MD_ERR_INVALID_ARG, "step_kernel must be 0..5");
    if (t->build_stage < 0 || t->build_stage > 2) return fail(MD_ERR_INVALID_ARG, "build_stage must be 0, 1 or 2");
    if (t->reorder_every < -1) return fail(MD_ERR_INVALID_ARG, "reorder_every must be >= -1");
    const int old_kernel = s->L.step_kernel;
    if (t->ctas_per_sm) s->tune.ctas_per_sm = t->ctas_per_sm;
    if (t->nbr_batch) s->tune.nbr_batch = t->nbr_batch;
    if (t->build_batch) s->tune.build_batch = t->build_batch;
    if (t->use_graph) s->tune.use_graph = t->use_graph;
    if (t->step_kernel) s->tune.step_kernel = t->step_kernel;
    if (t->build_stage) s->tune.build_stage = t->build_stage;
    if (t->reorder_every) s->tune.reorder_every = t->reorder_every;
    s->drop_graphs();          // launch shapes are baked into captured graphs
    int rc = apply_tuning(s);
    if (rc) return rc;
    if ((s->L.step_kernel == 4) != (old_kernel == 4) || (s->L.step_kernel == 5) != (old_kernel == 5)) {
        // into the list-free kernel: atoms reordered by cell now; out of it: W built now; into or
        // out of the half list: W rebuilt with the other half rule
        GBMD_CUDA(launch_force_rebuild(s->A, s->S, s->L, s->L.step_kernel == 4 ? 1 : 0));
        GBMD_CUDA(launch_rebuild(s->A, s->S, s->L, s->cur, false));
        s->binned_fresh = false;
    }
    return MD_OK;
}

int md_get_tuning(const md_system* s, md_tuning* t)
{
    if (!s || !t) return fail(MD_ERR_INVALID_ARG, "bad arguments");
    *t = s->tune;
    return MD_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// adjoint driver
// ------------------------------------------------------------------------------------------
namespace {

struct AdjPlan {
    int K, S, nseg;
};

// Two sets of segment snapshots: segment k uses set k & 1, so the recompute of segment k-1 can
// run while segment k is walked back.
struct AdjSets {
    float4* pos[2];
    int32_t* cnt[2];
    uint32_t* W[2];
    int32_t* id[2];
};

// the adjoint view with snapshot set `set` as its snapshot arrays
AdjView adj_view_of(const AdjView& V, const AdjSets& Z, int set)
{
    AdjView v = V;
    v.pos_snap = Z.pos[set];
    v.cnt_snap = Z.cnt[set];
    v.W_snap = Z.W[set];
    v.id_snap = Z.id[set];
    return v;
}

size_t carve_adj(const md_system* s, const AdjPlan& P, char* base, AdjView* V, AdjSets* Z = nullptr)
{
    Carver c{base};
    AdjView v;
    std::memset(&v, 0, sizeof(v));
    AdjSets z;
    const size_t ns = size_t(s->plan.nslots), n3 = size_t(s->plan.n_total) * 3;
    for (int set = 0; set < 2; ++set) {
        z.pos[set] = c.take<float4>(ns * (P.K + 1));
        z.cnt[set] = c.take<int32_t>(ns * (P.K + 1));
        z.W[set] = c.take<uint32_t>(ns * size_t(s->plan.cap) * (P.K + 1));
        z.id[set] = c.take<int32_t>(ns);
    }
    v.pos_snap = z.pos[0];
    v.cnt_snap = z.cnt[0];
    v.W_snap = z.W[0];
    v.id_snap = z.id[0];
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 3; ++a) {
            v.lx[b][a] = c.take<double>(ns);
            v.lv[b][a] = c.take<double>(ns);
            v.mu[b][a] = c.take<double>(ns);
        }
    v.tile_acc = c.take<double>(size_t(s->plan.ntiles) * 4);
    v.ck_x = c.take<double>(n3 * (P.nseg + 1));
    v.ck_v = c.take<double>(n3 * (P.nseg + 1));
    v.lam_x = c.take<double>(n3);
    v.lam_v = c.take<double>(n3);
    v.vnorm_part = c.take<double>(ADJ_VPART);
    v.out = c.take<double>(8);
    if (V) *V = v;
    if (Z) *Z = z;
    return (c.off + 255) & ~size_t(255);
}

int adj_plan(const md_system* s, int32_t nsteps, int32_t ckpt_every, AdjPlan* P)
{
    if (!s) return fail(MD_ERR_INVALID_ARG, "system is NULL");
    if (s->plan.nrep != 1) return fail(MD_ERR_INVALID_ARG, "md_adjoint needs a single system (nrep == 1)");
    if (s->plan.mode == MD_FP64) return fail(MD_ERR_INVALID_ARG, "md_adjoint runs on MD_MIXED or MD_FP32 systems");
    if (nsteps < 1 || ckpt_every < 1 || ckpt_every > nsteps)
        return fail(MD_ERR_INVALID_ARG, "need nsteps >= 1 and 1 <= ckpt_every <= nsteps");
    P->K = ckpt_every;
    P->S = nsteps;
    P->nseg = (nsteps + ckpt_every - 1) / ckpt_every;
    return MD_OK;
}

// positions and integer-step velocities (id order) into device buffers x, v
int adj_save(md_system* s, const Scal& S, int cur, double* x, double* v)
{
    GBMD_CUDA(launch_forces(s->A, S, s->L, cur));
    GBMD_CUDA(launch_get_state(s->A, S, s->L, cur, true, false));
    const size_t bytes = size_t(s->plan.n_total) * 3 * sizeof(double);
    GBMD_CUDA(cudaMemcpyAsync(x, s->A.xchg[0], bytes, cudaMemcpyDeviceToDevice, s->L.stream));
    GBMD_CUDA(cudaMemcpyAsync(v, s->A.xchg[1], bytes, cudaMemcpyDeviceToDevice, s->L.stream));
    return MD_OK;
}

// restart from a checkpoint: exact binning, reorder by cell, neighbour build
int adj_load(md_system* s, const Scal& S, const double* x, const double* v)
{
    const size_t bytes = size_t(s->plan.n_total) * 3 * sizeof(double);
    GBMD_CUDA(cudaMemcpyAsync(s->A.xchg[0], x, bytes, cudaMemcpyDeviceToDevice, s->L.stream));
    GBMD_CUDA(cudaMemcpyAsync(s->A.xchg[1], v, bytes, cudaMemcpyDeviceToDevice, s->L.stream));
    GBMD_CUDA(launch_set_state(s->A, S, s->L, 0));
    GBMD_CUDA(launch_force_rebuild(s->A, S, s->L, 1));
    GBMD_CUDA(launch_rebuild(s->A, S, s->L, 0, true));
    return MD_OK;
}

cudaError_t adj_snapshot(md_system* s, const AdjView& V, int q, int cur, cudaStream_t st)
{
    const size_t ns = size_t(s->plan.nslots);
    cudaError_t e = cudaMemcpyAsync(V.pos_snap + ns * q, s->A.pos32[cur], ns * sizeof(float4), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(V.cnt_snap + ns * q, s->A.nbr_count, ns * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(V.W_snap + ns * size_t(s->plan.cap) * q, s->A.W, ns * size_t(s->plan.cap) * sizeof(uint32_t),
                            cudaMemcpyDeviceToDevice, st);
    return e;
}

// The graphs of md_adjoint's segments, captured once per (workspace, horizon, segment shape,
// snapshot set) and replayed: kind 0 runs `steps` forward steps from buffer 0; kind 1 also
// records the slot -> id map and snapshots the positions, counts and W before the first and after
// every step; kind 2 walks the segment back (reverse steps `steps`..1, plus step 0 in the first
// segment; flags bit 0: the segment ends at the horizon, bit 1: it is the first).  Each step's
// rebuild sits behind an IF node as in md_integrate.
int adj_graph(md_system* s, const Scal& Sa, const AdjView& V0, const AdjSets& Z, int set, const void* work, int nsteps,
              int ckpt, int kind, int steps, int buf0, int flags, cudaGraphExec_t* out)
{
    const AdjView V = adj_view_of(V0, Z, set);
    flags |= set << 8;                            // the snapshot set is part of the key
    for (auto& g : s->adj_graphs)
        if (g.work == work && g.nsteps == nsteps && g.ckpt == ckpt && g.kind == kind && g.steps == steps &&
            g.buf0 == buf0 && g.flags == flags) {
            *out = g.exec;
            return MD_OK;
        }
    // a bounded cache: callers that vary workspaces or horizons start it over
    constexpr size_t ADJ_GRAPH_CACHE = 32;
    if (s->adj_graphs.size() >= ADJ_GRAPH_CACHE) {
        GBMD_CUDA(cudaStreamSynchronize(s->L.stream));
        for (auto& g : s->adj_graphs) {
            cudaGraphExecDestroy(g.exec);
            cudaGraphDestroy(g.graph);
        }
        s->adj_graphs.clear();
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int rc = capture_exec(
        s,
        [&](cudaStream_t st) {
            cudaError_t err = cudaSuccess;
            if (kind == 0 || kind == 1) {
                int cur = 0;
                if (kind == 1)                    // the segment's slot -> id map, then snapshot 0
                    err = cudaMemcpyAsync(V.id_snap, s->A.id, size_t(s->plan.nslots) * sizeof(int32_t),
                                          cudaMemcpyDeviceToDevice, st);
                if (kind == 1 && err == cudaSuccess) err = adj_snapshot(s, V, 0, cur, st);
                for (int q = 1; q <= steps && err == cudaSuccess; ++q) {
                    err = capture_step_and_rebuild(s, Sa, st, cur, false);
                    cur ^= 1;
                    if (err == cudaSuccess && kind == 1) err = adj_snapshot(s, V, q, cur, st);
                }
            } else {
                Launch L = s->L;
                L.stream = st;
                int buf = buf0;
                // kappa of reverse step q: 1 at the horizon and at n = 0, else 2
                auto kappa_of = [&](int q) { return (((flags & 1) && q == steps) || q == 0) ? 1.0 : 2.0; };
                err = launch_adj_permute(s->A, Sa, L, V, buf, true, kappa_of(steps));
                for (int q = steps; q >= 1 && err == cudaSuccess; --q) {
                    err = launch_adj_reverse(s->A, Sa, L, V, q, kappa_of(q), 1.0 / double(nsteps), buf, kappa_of(q - 1));
                    buf ^= 1;
                }
                if (err == cudaSuccess && (flags & 2)) {
                    err = launch_adj_reverse(s->A, Sa, L, V, 0, 1.0, 0.0, buf, 1.0);
                    buf ^= 1;
                }
                if (err == cudaSuccess) err = launch_adj_permute(s->A, Sa, L, V, buf, false, 0.0);
            }
            return err;
        },
        &graph, &exec);
    if (rc) return rc;
    s->adj_graphs.push_back({work, nsteps, ckpt, kind, steps, buf0, flags, graph, exec});
    *out = exec;
    return MD_OK;
}

}  // namespace

extern "C" {

size_t md_adjoint_workspace_bytes(const md_system* s, int32_t nsteps, int32_t ckpt_every)
{
    AdjPlan P;
    if (adj_plan(s, nsteps, ckpt_every, &P) != MD_OK) return 0;
    return carve_adj(s, P, nullptr, nullptr);
}

int md_adjoint(md_system* s, void* d_work, size_t work_bytes, int32_t nsteps, int32_t ckpt_every, double* loss,
               double* dL_deps, double* dL_dsigma, double* dL_dv0)
{
    AdjPlan P;
    int rc = adj_plan(s, nsteps, ckpt_every, &P);
    if (rc) return rc;
    if (s->L.step_kernel >= 4)
        return fail(MD_ERR_INVALID_ARG, "the adjoint walks the full neighbour matrix: select step kernel 1, 2 or 3");
    if (s->S.chain_len) return fail(MD_ERR_INVALID_ARG, "the adjoint covers the pair forces only: no chains");
    const size_t need = carve_adj(s, P, nullptr, nullptr);
    if (!d_work || (reinterpret_cast<uintptr_t>(d_work) & 255u) || work_bytes < need)
        return fail(MD_ERR_WORKSPACE, "adjoint workspace missing, misaligned or below " + std::to_string(need) + " bytes");
    AdjView V;
    AdjSets Z;
    carve_adj(s, P, static_cast<char*>(d_work), &V, &Z);
    if (s->binned_fresh) {
        GBMD_CUDA(launch_build_only(s->A, s->S, s->L, s->cur));
        s->binned_fresh = false;
    }
    // inside a segment the slot order must stay fixed: no reorder (the restart reorders)
    Scal Sa = s->S;
    Sa.reorder_every = 0x7fffffff;
    const size_t n3 = size_t(s->plan.n_total) * 3;
    cudaStream_t st = s->L.stream;
    Phase tph(s, MD_PHASE_OTHER, 0);

    // forward: checkpoints of (x, v) at the start of every segment and at the end
    rc = adj_save(s, s->S, s->cur, V.ck_x, V.ck_v);
    if (rc) return rc;
    for (int k = 0; k < P.nseg; ++k) {
        rc = adj_load(s, Sa, V.ck_x + n3 * k, V.ck_v + n3 * k);
        if (rc) return rc;
        const int steps = std::min(P.K, P.S - k * P.K);
        cudaGraphExec_t g = nullptr;
        rc = adj_graph(s, Sa, V, Z, 0, d_work, nsteps, ckpt_every, 0, steps, 0, 0, &g);
        if (!rc) rc = replay(s, g);
        if (rc) return rc;
        rc = adj_save(s, Sa, steps & 1, V.ck_x + n3 * (k + 1), V.ck_v + n3 * (k + 1));
        if (rc) return rc;
    }
    // terminal conditions and the |v_S|^2 part of the loss
    GBMD_CUDA(launch_adj_init(V, s->L, s->plan.n_total, V.ck_v + n3 * P.nseg));
    GBMD_CUDA(cudaMemsetAsync(V.tile_acc, 0, sizeof(double) * 4 * size_t(s->plan.ntiles), st));
    // reverse, one segment at a time: recompute it from its checkpoint into snapshot set k & 1 (on
    // the system's stream), then walk it back on the reverse stream, so the recompute of segment
    // k-1 overlaps the walk of segment k; a set is refilled only after its previous walk ended
    GBMD_CUDA(ensure_adj_streams(s));
    GBMD_CUDA(cudaEventRecord(s->ev_rc[0], st));          // the terminal conditions are in place
    GBMD_CUDA(cudaStreamWaitEvent(s->rstream, s->ev_rc[0], 0));
    bool set_used[2] = {false, false};
    int buf = 0;
    for (int k = P.nseg - 1; k >= 0; --k) {
        const int set = k & 1;
        if (set_used[set]) GBMD_CUDA(cudaStreamWaitEvent(st, s->ev_rev[set], 0));
        rc = adj_load(s, Sa, V.ck_x + n3 * k, V.ck_v + n3 * k);
        if (rc) return rc;
        const int steps = std::min(P.K, P.S - k * P.K);
        const int flags = (k == P.nseg - 1 ? 1 : 0) | (k == 0 ? 2 : 0);
        cudaGraphExec_t gr = nullptr, gb = nullptr;
        rc = adj_graph(s, Sa, V, Z, set, d_work, nsteps, ckpt_every, 1, steps, 0, 0, &gr);
        if (!rc) rc = replay(s, gr);
        if (!rc) rc = adj_graph(s, Sa, V, Z, set, d_work, nsteps, ckpt_every, 2, steps, buf, flags, &gb);
        if (rc) return rc;
        GBMD_CUDA(cudaEventRecord(s->ev_rc[set], st));
        GBMD_CUDA(cudaStreamWaitEvent(s->rstream, s->ev_rc[set], 0));
        GBMD_CUDA(cudaGraphLaunch(gb, s->rstream));
        GBMD_CUDA(cudaEventRecord(s->ev_rev[set], s->rstream));
        set_used[set] = true;
        buf ^= (steps + (k == 0 ? 1 : 0)) & 1;
    }
    GBMD_CUDA(cudaStreamWaitEvent(st, s->ev_rev[0], 0));   // segment 0 (set 0) is walked last
    GBMD_CUDA(launch_adj_final(V, s->L, s->plan.ntiles));
    double out[8];
    GBMD_CUDA(cudaMemcpyAsync(out, V.out, sizeof(double) * 5, cudaMemcpyDeviceToHost, st));
    if (dL_dv0) GBMD_CUDA(cudaMemcpyAsync(dL_dv0, V.lam_v, sizeof(double) * n3, cudaMemcpyDefault, st));
    // leave the system at its initial state
    rc = load_state(s, V.ck_x, V.ck_v);
    if (rc) return rc;
    GBMD_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = out[2] + out[4];
    if (dL_deps) *dL_deps = (out[0] + out[2]) / s->p.eps;
    if (dL_dsigma) *dL_dsigma = out[1] + out[3];
    return latch_error(s);
}

}  // extern "C"
