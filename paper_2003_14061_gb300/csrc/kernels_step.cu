// kernels_step.cu -- per-step kernels: fused force + leapfrog, standalone forces, reductions,
// and the id-ordered state exchange.
//
//   k_step     F1 (Sec. 2.3) fused with the leapfrog update (Sec. 4.3 item 1).  One thread per
//              atom walks its column of W (coalesced rows, Sec. 4.1 item 6), gathers neighbour
//              positions from the other position buffer, accumulates f_i without Newton's third
//              law (Sec. 2.3), then kicks and drifts its own FP64 state and writes its next
//              cell-local position.  Per tile, the maximum speed (or displacement) is reduced;
//              the CTA that completes a replica's last tile (the "last block" pattern of
//              Sec. 2.3, an atomic counter after a memory fence) updates the refresh criterion
//              and raises the rebuild flag.  With PROPS, the tile also writes FP64 partial sums
//              of U, K, virial and momentum (F2).
//   k_forces   F1 alone: f_i, u_i and the per-atom virial at the current positions.
//   k_props_*  F2 and the other measured quantities: per-tile FP64 partials, then one CTA per
//              replica sums them in a fixed order (deterministic).
#include <algorithm>

#include "gbmd_internal.cuh"

namespace gbmd {

// offset code (0, 1, 2) of one axis -> (code - 1) as an exact float, without a conversion op
__device__ __forceinline__ float offset_f(uint32_t code2)
{
    return __uint_as_float(0x4B000000u | code2) - 8388609.0f;
}

// ------------------------------------------------------------------------------------------
// pair loops
// ------------------------------------------------------------------------------------------
struct AccF { float fx, fy, fz, u, w; };
struct AccD { double fx, fy, fz, u, w; };

// One thread per atom over its column of W, NB entries at a time: the NB row loads are issued
// together, then the NB position gathers, so each thread keeps 2 NB loads in flight.
template <int NB>
__device__ __forceinline__ AccF force_f32(const Arrays& A, const Scal& S, const Rep& R,
                                          const float4* __restrict__ pos, int64_t slot, float4 pi)
{
    AccF a{0.f, 0.f, 0.f, 0.f, 0.f};
    const int mm = min(__ldcs(A.nbr_count + slot), S.cap);
    const uint32_t* __restrict__ Wc = A.W + slot;
    const float wx = R.wf[0], wy = R.wf[1], wz = R.wf[2];
    for (int m0 = 0; m0 < mm; m0 += NB) {
        uint32_t e[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k)
            e[k] = (m0 + k < mm) ? __ldcs(Wc + int64_t(m0 + k) * S.nslots) : 0u;
        float4 pj[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k)
            pj[k] = (m0 + k < mm) ? __ldg(pos + (e[k] & IDX_MASK)) : pi;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const uint32_t ek = e[k];
            const float dx = fmaf(offset_f((ek >> 26) & 3u), wx, pj[k].x - pi.x);
            const float dy = fmaf(offset_f((ek >> 28) & 3u), wy, pj[k].y - pi.y);
            const float dz = fmaf(offset_f(ek >> 30), wz, pj[k].z - pi.z);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (m0 + k < mm && r2 < S.rc2f) {
                const float ri2 = __frcp_rn(r2);
                const float sr2 = S.sig2f * ri2;
                const float sr6 = sr2 * sr2 * sr2;
                const float fs = S.eps48f * sr6 * (sr6 - 0.5f) * ri2;   // g(r^2)
                a.fx = fmaf(-fs, dx, a.fx);                              // f_i = g (x_i - x_j)
                a.fy = fmaf(-fs, dy, a.fy);
                a.fz = fmaf(-fs, dz, a.fz);
                a.u += fmaf(S.eps4f * sr6, sr6 - 1.0f, -S.ucf);
                a.w = fmaf(fs, r2, a.w);
            }
        }
    }
    return a;
}

__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ AccD force_f64(const Arrays& A, const Scal& S, const Rep& R,
                                          const double4_32a* __restrict__ pos, int64_t slot, double4_32a pi)
{
    AccD a{0.0, 0.0, 0.0, 0.0, 0.0};
    const int mm = min(A.nbr_count[slot], S.cap);
    const uint32_t* __restrict__ Wc = A.W + slot;
    for (int m = 0; m < mm; ++m) {
        const uint32_t e = Wc[int64_t(m) * S.nslots];
        const double4_32a pj = pos[e & IDX_MASK];
        const double dx = fma(double(int((e >> 26) & 3u) - 1), R.w[0], pj.x - pi.x);
        const double dy = fma(double(int((e >> 28) & 3u) - 1), R.w[1], pj.y - pi.y);
        const double dz = fma(double(int(e >> 30) - 1), R.w[2], pj.z - pi.z);
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        if (r2 < S.rc2d) {
            const double ri2 = 1.0 / r2;
            const double sr2 = S.sig2d * ri2;
            const double sr6 = sr2 * sr2 * sr2;
            const double fs = S.eps48d * sr6 * (sr6 - 0.5) * ri2;
            a.fx -= fs * dx;
            a.fy -= fs * dy;
            a.fz -= fs * dz;
            a.u += S.eps4d * sr6 * (sr6 - 1.0) - S.ucd;
            a.w += fs * r2;
        }
    }
    return a;
}

// ------------------------------------------------------------------------------------------
// block reductions over one tile (TILE threads)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float tile_max(float v, float* sh)
{
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = sh[0];
#pragma unroll
    for (int k = 1; k < TILE / 32; ++k) m = fmaxf(m, sh[k]);
    return m;
}

__device__ __forceinline__ void tile_partials(double (&p)[NPROP], double (*sh)[NPROP], double* out)
{
#pragma unroll
    for (int q = 0; q < NPROP - 1; ++q) p[q] = warp_sum(p[q]);
    {
        double x = p[NPROP - 1];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        p[NPROP - 1] = x;
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < NPROP; ++q) sh[threadIdx.x >> 5][q] = p[q];
    }
    __syncthreads();
    if (threadIdx.x < NPROP) {
        const int q = threadIdx.x;
        double s = sh[0][q];
        for (int k = 1; k < TILE / 32; ++k) s = (q == NPROP - 1) ? fmax(s, sh[k][q]) : s + sh[k][q];
        out[q] = s;
    }
}

// Refresh criterion and step bookkeeping, run by one thread of the CTA that completed the last
// tile of replica r in this launch.
__device__ void finish_replica_step(const Arrays& A, const Scal& S, int r, cudaGraphConditionalHandle cond,
                                    int use_cond)
{
    RepState& st = A.rs[r];
    st.tiles_done = 0;
    const float m2 = __uint_as_float(atomicExch(&st.vmax2, 0u));
    if (!(m2 <= 3.0e38f)) atomicOr(&A.g->err, ERR_NONFINITE);
    st.step += 1;
    st.vhalf = 1;
    bool rebuild;
    if (S.rule == MD_REBUILD_VMAX) {
        // D bounds every atom's displacement since the last rebuild (triangle inequality);
        // the factor covers the FP32 rounding of |v|.
        st.D += S.dt * sqrt(double(m2)) * (1.0 + 1e-6);
        rebuild = st.D > S.half_skin;
    } else if (S.rule == MD_REBUILD_DISP) {
        rebuild = sqrt(double(m2)) * (1.0 + 1e-6) > S.half_skin;
    } else {
        rebuild = true;
    }
    if (rebuild) {
        const int reorder = (S.reorder_every == 0) || (st.step - st.last_reorder >= S.reorder_every);
        st.rebuild = 1;
        st.reorder = reorder;
        st.max_occ = 0;
        if (reorder) A.g->any_reorder = 1;
        // the first replica to ask for a rebuild in this step opens the graph's IF node (one
        // caller per step: concurrent cudaGraphSetConditional calls are not allowed)
        if (atomicExch(&A.g->any_rebuild, 1) == 0 && use_cond) cudaGraphSetConditional(cond, 1u);
    }
}

// ------------------------------------------------------------------------------------------
// fused force + leapfrog step
// ------------------------------------------------------------------------------------------
template <int MODE, bool PROPS, int NB>
__global__ void __launch_bounds__(TILE) k_step(Arrays A, Scal S, int cur, cudaGraphConditionalHandle cond,
                                                 int use_cond)
{
    __shared__ float sh_max[TILE / 32];
    __shared__ double sh_part[PROPS ? TILE / 32 : 1][NPROP];
    __shared__ int sh_last;
    const int nxt = cur ^ 1;
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const bool active = slot - R.slot0 < R.n;
        const int vhalf = A.rs[r].vhalf;
        float metric = 0.0f;                     // |v|^2 (VMAX) or |x - x_ref|^2 (DISP)
        double part[NPROP];
#pragma unroll
        for (int q = 0; q < NPROP; ++q) part[q] = 0.0;
        if (active) {
            if (MODE == MD_FP64) {
                const double4_32a* pos = A.pos64[cur];
                const double4_32a pi = pos[slot];
                const AccD a = force_f64(A, S, R, pos, slot, pi);
                const double f[3] = {a.fx, a.fy, a.fz};
                double xl[3] = {pi.x, pi.y, pi.z};
                const double kick = vhalf ? 2.0 * S.c : S.c;
                double vn2 = 0.0, vv[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    double v = A.v[q][slot];
                    if (PROPS) {
                        const double vn = vhalf ? fma(S.c, f[q], v) : v;
                        vn2 = fma(vn, vn, vn2);
                        part[3 + q] = S.mass * vn;
                    }
                    v = fma(kick, f[q], v);
                    xl[q] = fma(S.dt, v, xl[q]);
                    A.v[q][slot] = v;
                    A.xl[q][slot] = xl[q];
                    vv[q] = v;
                }
                A.pos64[nxt][slot] = make_double4_32a(xl[0], xl[1], xl[2], pi.w);
                if (S.rule == MD_REBUILD_DISP) {
                    const float4 xr = A.xref[slot];
                    const float d0 = float(xl[0] - double(xr.x)), d1 = float(xl[1] - double(xr.y)),
                                d2 = float(xl[2] - double(xr.z));
                    metric = d0 * d0 + d1 * d1 + d2 * d2;
                } else {
                    metric = float(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
                }
                if (PROPS) {
                    part[0] = 0.5 * a.u;
                    part[1] = 0.5 * S.mass * vn2;
                    part[2] = 0.5 * a.w;
                    part[NPROP - 1] = vn2;
                }
            } else {
                const float4* pos = A.pos32[cur];
                const float4 pi = __ldg(pos + slot);
                if (MODE == MD_MIXED) {
                    // bring the FP64 state towards L2 while the pair loop runs
#pragma unroll
                    for (int q = 0; q < 3; ++q) { prefetch_l2(A.v[q] + slot); prefetch_l2(A.xl[q] + slot); }
                } else {
#pragma unroll
                    for (int q = 0; q < 3; ++q) prefetch_l2(A.v32[q] + slot);
                }
                const AccF a = force_f32<NB>(A, S, R, pos, slot, pi);
                const float f[3] = {a.fx, a.fy, a.fz};
                float pn[3];
                double vn2 = 0.0;
                if (MODE == MD_MIXED) {
                    const double kick = vhalf ? 2.0 * S.c : S.c;
                    float vf[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        double v = __ldcs(A.v[q] + slot);
                        const double fq = double(f[q]);
                        if (PROPS) {
                            const double vn = vhalf ? fma(S.c, fq, v) : v;
                            vn2 = fma(vn, vn, vn2);
                            part[3 + q] = S.mass * vn;
                        }
                        v = fma(kick, fq, v);
                        const double x = fma(S.dt, v, __ldcs(A.xl[q] + slot));
                        __stcs(A.v[q] + slot, v);
                        __stcs(A.xl[q] + slot, x);
                        pn[q] = __double2float_rn(x);
                        vf[q] = __double2float_rn(v);
                    }
                    if (S.rule != MD_REBUILD_DISP) metric = fmaf(vf[2], vf[2], fmaf(vf[1], vf[1], vf[0] * vf[0]));
                } else {
                    const float kick = float(vhalf ? 2.0 * S.c : S.c);
                    const float cf = float(S.c), dtf = float(S.dt);
                    const float pc[3] = {pi.x, pi.y, pi.z};
                    float vf[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        float v = A.v32[q][slot];
                        if (PROPS) {
                            const float vn = vhalf ? fmaf(cf, f[q], v) : v;
                            vn2 = fma(double(vn), double(vn), vn2);
                            part[3 + q] = S.mass * double(vn);
                        }
                        v = fmaf(kick, f[q], v);
                        A.v32[q][slot] = v;
                        pn[q] = fmaf(dtf, v, pc[q]);
                        vf[q] = v;
                    }
                    if (S.rule != MD_REBUILD_DISP) metric = fmaf(vf[2], vf[2], fmaf(vf[1], vf[1], vf[0] * vf[0]));
                }
                A.pos32[nxt][slot] = make_float4(pn[0], pn[1], pn[2], pi.w);
                if (S.rule == MD_REBUILD_DISP) {
                    const float4 xr = A.xref[slot];
                    const float d0 = pn[0] - xr.x, d1 = pn[1] - xr.y, d2 = pn[2] - xr.z;
                    metric = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
                }
                if (PROPS) {
                    part[0] = 0.5 * double(a.u);
                    part[1] = 0.5 * S.mass * vn2;
                    part[2] = 0.5 * double(a.w);
                    part[NPROP - 1] = vn2;
                }
            }
            if (!(metric <= 3.0e38f)) metric = __uint_as_float(0x7f800000u);   // +inf marks non-finite
        }
        const float tmax = tile_max(metric, sh_max);
        if (PROPS) tile_partials(part, sh_part, A.tile_part + int64_t(t) * NPROP);
        if (threadIdx.x == 0) {
            atomicMax(&A.rs[r].vmax2, __float_as_uint(tmax));
            __threadfence();
            sh_last = (atomicAdd(&A.rs[r].tiles_done, 1) == R.ntiles - 1);
            if (sh_last) {
                __threadfence();
                finish_replica_step(A, S, r, cond, use_cond);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// forces only (F1): f, u_i, per-atom virial
// ------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(TILE) k_forces(Arrays A, Scal S, int cur)
{
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        if (MODE == MD_FP64) {
            const double4_32a pi = A.pos64[cur][slot];
            const AccD a = force_f64(A, S, R, A.pos64[cur], slot, pi);
            A.f[slot] = make_double4_32a(a.fx, a.fy, a.fz, a.u);
            A.wvir[slot] = a.w;
        } else {
            const float4 pi = A.pos32[cur][slot];
            const AccF a = force_f32<4>(A, S, R, A.pos32[cur], slot, pi);
            A.f[slot] = make_double4_32a(a.fx, a.fy, a.fz, a.u);
            A.wvir[slot] = a.w;
        }
    }
}

// per-tile FP64 partials from stored forces and the state's velocities (closed to step n)
template <int MODE>
__global__ void __launch_bounds__(TILE) k_props_tiles(Arrays A, Scal S)
{
    __shared__ double sh_part[TILE / 32][NPROP];
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        double part[NPROP];
#pragma unroll
        for (int q = 0; q < NPROP; ++q) part[q] = 0.0;
        if (slot - R.slot0 < R.n) {
            const double4_32a f = A.f[slot];
            const int vhalf = A.rs[r].vhalf;
            const double fq[3] = {f.x, f.y, f.z};
            double vn2 = 0.0;
            for (int q = 0; q < 3; ++q) {
                double v = (MODE == MD_FP32) ? double(A.v32[q][slot]) : A.v[q][slot];
                double vn;
                if (MODE == MD_FP32) vn = vhalf ? double(fmaf(float(S.c), float(fq[q]), float(v))) : v;
                else vn = vhalf ? fma(S.c, fq[q], v) : v;
                vn2 = fma(vn, vn, vn2);
                part[3 + q] = S.mass * vn;
            }
            part[0] = 0.5 * f.w;
            part[1] = 0.5 * S.mass * vn2;
            part[2] = 0.5 * A.wvir[slot];
            part[NPROP - 1] = vn2;
        }
        tile_partials(part, sh_part, A.tile_part + int64_t(t) * NPROP);
        __syncthreads();
    }
}

// one CTA per replica: fixed-order sum of its tile partials
__global__ void __launch_bounds__(256) k_props_finalize(Arrays A, Scal S, int to_series, int step_lag)
{
    __shared__ double sh[256][NPROP];
    const int r = blockIdx.x;
    const Rep& R = A.rep[r];
    double acc[NPROP];
#pragma unroll
    for (int q = 0; q < NPROP; ++q) acc[q] = 0.0;
    for (int k = threadIdx.x; k < R.ntiles; k += blockDim.x) {
        const double* p = A.tile_part + int64_t(R.tile0 + k) * NPROP;
#pragma unroll
        for (int q = 0; q < NPROP - 1; ++q) acc[q] += p[q];
        acc[NPROP - 1] = fmax(acc[NPROP - 1], p[NPROP - 1]);
    }
#pragma unroll
    for (int q = 0; q < NPROP; ++q) sh[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
#pragma unroll
            for (int q = 0; q < NPROP - 1; ++q) sh[threadIdx.x][q] += sh[threadIdx.x + h][q];
            sh[threadIdx.x][NPROP - 1] = fmax(sh[threadIdx.x][NPROP - 1], sh[threadIdx.x + h][NPROP - 1]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const RepState& st = A.rs[r];
        const double U = sh[0][0], K = sh[0][1], W = sh[0][2];
        const double V = R.L[0] * R.L[1] * R.L[2];
        md_props pr;
        pr.U = U;
        pr.K = K;
        pr.E_per_atom = (U + K) / double(R.n);
        pr.virial = W;
        pr.pressure = (2.0 * K + W) / (3.0 * V);
        pr.P[0] = sh[0][3]; pr.P[1] = sh[0][4]; pr.P[2] = sh[0][5];
        pr.vmax = sqrt(sh[0][NPROP - 1]);
        pr.mean_nbrs = double(st.sum_nbrs) / double(R.n);
        pr.step = st.step - step_lag;
        pr.rebuilds = st.rebuilds;
        pr.max_cell_occ = st.max_occ;
        pr.max_nbrs = st.max_nbrs;
        A.props[r] = pr;
        if (to_series) {
            RepState& sw = A.rs[r];
            const int row = sw.series_rows;
            if (row < S.series_cap) {
                double* o = A.series + (int64_t(r) * S.series_cap + row) * SERIES_COLS;
                o[0] = double(pr.step); o[1] = U; o[2] = K; o[3] = W; o[4] = pr.pressure;
                o[5] = pr.P[0]; o[6] = pr.P[1]; o[7] = pr.P[2]; o[8] = pr.vmax;
                sw.series_rows = row + 1;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// state exchange in id order
// ------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(TILE) k_set_state(Arrays A, Scal S, int cur)
{
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const int64_t j = slot - R.slot0;
        if (threadIdx.x == 0 && t == R.tile0) {
            RepState& st = A.rs[r];
            st.D = 0.0; st.vmax2 = 0u; st.rebuild = 0; st.reorder = 0; st.vhalf = 0;
            st.tiles_done = 0; st.max_nbrs = 0; st.max_occ = 0; st.series_rows = 0;
            st.step = 0; st.rebuilds = 0; st.last_reorder = 0; st.sum_nbrs = 0;
        }
        if (j >= R.n) continue;
        const int64_t id = R.id0 + j;
        A.id[slot] = int32_t(id);
        for (int a = 0; a < 3; ++a) {
            A.xl[a][slot] = A.xchg[0][id * 3 + a];     // global position, origin cell (0,0,0)
            const double v = A.xchg[1][id * 3 + a];
            if (MODE == MD_FP32) A.v32[a][slot] = float(v);
            else A.v[a][slot] = v;
        }
        if (MODE == MD_FP64) A.pos64[cur][slot] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        else A.pos32[cur][slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int MODE>
__global__ void __launch_bounds__(TILE) k_get_state(Arrays A, Scal S, int cur, int want_v, int want_f)
{
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        const int64_t id = A.id[slot];
        uint32_t pw;
        double loc[3];
        if (MODE == MD_FP64) {
            const double4_32a p = A.pos64[cur][slot];
            pw = cell_bits(p.w);
            loc[0] = A.xl[0][slot]; loc[1] = A.xl[1][slot]; loc[2] = A.xl[2][slot];
        } else {
            const float4 p = A.pos32[cur][slot];
            pw = __float_as_uint(p.w);
            if (MODE == MD_FP32) { loc[0] = p.x; loc[1] = p.y; loc[2] = p.z; }
            else { loc[0] = A.xl[0][slot]; loc[1] = A.xl[1][slot]; loc[2] = A.xl[2][slot]; }
        }
        int c[3];
        unpack_cell(pw, c[0], c[1], c[2]);
        const int vhalf = A.rs[r].vhalf;
        const double4_32a f = (want_f || (want_v && vhalf)) ? A.f[slot] : make_double4_32a(0, 0, 0, 0);
        const double fq[3] = {f.x, f.y, f.z};
        for (int a = 0; a < 3; ++a) {
            double x = __dadd_rn(__dmul_rn(double(c[a]), R.w[a]), loc[a]);
            if (x < 0.0) x += R.L[a];
            if (x >= R.L[a]) x -= R.L[a];
            A.xchg[0][id * 3 + a] = x;
            if (want_v) {
                double v = (MODE == MD_FP32) ? double(A.v32[a][slot]) : A.v[a][slot];
                if (vhalf) {
                    if (MODE == MD_FP32) v = double(fmaf(float(S.c), float(fq[a]), float(v)));
                    else v = fma(S.c, fq[a], v);
                }
                A.xchg[1][id * 3 + a] = v;
            }
            if (want_f) A.xchg[2][id * 3 + a] = fq[a];
        }
    }
}

__global__ void __launch_bounds__(TILE) k_get_cells(Arrays A, Scal S, int32_t* out)
{
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        out[A.id[slot]] = A.cell[slot] - R.cell0;
    }
}

__global__ void __launch_bounds__(TILE) k_get_nbrs(Arrays A, Scal S, int32_t* counts, int32_t* nbrs,
                                                   int32_t cap_out, int64_t id_lo, int64_t id_hi)
{
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        const int64_t id = A.id[slot];
        const int m = A.nbr_count[slot];
        counts[id] = m;
        if (id < id_lo || id >= id_hi) continue;
        const int mm = min(min(m, S.cap), cap_out);
        for (int k = 0; k < mm; ++k) {
            const uint32_t e = A.W[int64_t(k) * S.nslots + slot];
            nbrs[(id - id_lo) * cap_out + k] = A.id[e & IDX_MASK];
        }
    }
}

// ------------------------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------------------------
static int tile_grid(const Scal& S, const Launch& L)
{
    return std::max(1, std::min(L.grid, S.ntiles));
}

cudaError_t launch_step(const Arrays& A, const Scal& S, const Launch& L, int cur, bool props)
{
    const int g = tile_grid(S, L);
#define GBMD_STEP(M, NB)                                                                             \
    if (props) k_step<M, true, NB><<<g, TILE, 0, L.stream>>>(A, S, cur, L.cond, L.use_cond);        \
    else k_step<M, false, NB><<<g, TILE, 0, L.stream>>>(A, S, cur, L.cond, L.use_cond);
    if (S.mode == MD_FP64) {
        GBMD_STEP(MD_FP64, 1)
    } else if (S.mode == MD_MIXED) {
        if (L.nbr_batch >= 8) { GBMD_STEP(MD_MIXED, 8) }
        else if (L.nbr_batch >= 4) { GBMD_STEP(MD_MIXED, 4) }
        else { GBMD_STEP(MD_MIXED, 2) }
    } else {
        if (L.nbr_batch >= 8) { GBMD_STEP(MD_FP32, 8) }
        else if (L.nbr_batch >= 4) { GBMD_STEP(MD_FP32, 4) }
        else { GBMD_STEP(MD_FP32, 2) }
    }
#undef GBMD_STEP
    if (props) k_props_finalize<<<S.nrep, 256, 0, L.stream>>>(A, S, 1, 1);
    return cudaGetLastError();
}

cudaError_t launch_forces(const Arrays& A, const Scal& S, const Launch& L, int cur)
{
    const int g = tile_grid(S, L);
    if (S.mode == MD_FP64) k_forces<MD_FP64><<<g, TILE, 0, L.stream>>>(A, S, cur);
    else if (S.mode == MD_MIXED) k_forces<MD_MIXED><<<g, TILE, 0, L.stream>>>(A, S, cur);
    else k_forces<MD_FP32><<<g, TILE, 0, L.stream>>>(A, S, cur);
    return cudaGetLastError();
}

cudaError_t launch_props(const Arrays& A, const Scal& S, const Launch& L, int cur, bool from_forces,
                         bool to_series)
{
    cudaError_t e = cudaSuccess;
    if (from_forces) e = launch_forces(A, S, L, cur);
    if (e != cudaSuccess) return e;
    const int g = tile_grid(S, L);
    if (S.mode == MD_FP64) k_props_tiles<MD_FP64><<<g, TILE, 0, L.stream>>>(A, S);
    else if (S.mode == MD_MIXED) k_props_tiles<MD_MIXED><<<g, TILE, 0, L.stream>>>(A, S);
    else k_props_tiles<MD_FP32><<<g, TILE, 0, L.stream>>>(A, S);
    k_props_finalize<<<S.nrep, 256, 0, L.stream>>>(A, S, to_series ? 1 : 0, 0);
    return cudaGetLastError();
}

cudaError_t launch_get_state(const Arrays& A, const Scal& S, const Launch& L, int cur, bool want_v,
                             bool want_f)
{
    const int g = tile_grid(S, L);
    if (S.mode == MD_FP64) k_get_state<MD_FP64><<<g, TILE, 0, L.stream>>>(A, S, cur, want_v, want_f);
    else if (S.mode == MD_MIXED) k_get_state<MD_MIXED><<<g, TILE, 0, L.stream>>>(A, S, cur, want_v, want_f);
    else k_get_state<MD_FP32><<<g, TILE, 0, L.stream>>>(A, S, cur, want_v, want_f);
    return cudaGetLastError();
}

cudaError_t launch_set_state(const Arrays& A, const Scal& S, const Launch& L, int cur)
{
    const int g = tile_grid(S, L);
    if (S.mode == MD_FP64) k_set_state<MD_FP64><<<g, TILE, 0, L.stream>>>(A, S, cur);
    else if (S.mode == MD_MIXED) k_set_state<MD_MIXED><<<g, TILE, 0, L.stream>>>(A, S, cur);
    else k_set_state<MD_FP32><<<g, TILE, 0, L.stream>>>(A, S, cur);
    return cudaGetLastError();
}

cudaError_t launch_get_cells(const Arrays& A, const Scal& S, const Launch& L, int32_t* out_by_id)
{
    k_get_cells<<<tile_grid(S, L), TILE, 0, L.stream>>>(A, S, out_by_id);
    return cudaGetLastError();
}

cudaError_t launch_get_neighbours(const Arrays& A, const Scal& S, const Launch& L, int32_t* counts_by_id,
                                  int32_t* nbr_by_id, int32_t cap_out, int64_t id_lo, int64_t id_hi)
{
    k_get_nbrs<<<tile_grid(S, L), TILE, 0, L.stream>>>(A, S, counts_by_id, nbr_by_id, cap_out, id_lo, id_hi);
    return cudaGetLastError();
}

}  // namespace gbmd
