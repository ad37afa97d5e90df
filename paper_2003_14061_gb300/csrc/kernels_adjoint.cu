// kernels_adjoint.cu -- reverse mode through the leapfrog trajectory and the pair force.
//
// Loss (time-averaged potential energy plus the squared final velocity norm):
//     L = (1/S) sum_{n=1..S} U(x_n) + |v_S|^2.
// Kick-drift-kick steps h_n = v_n + c F(x_n), x_{n+1} = x_n + dt h_n, v_{n+1} = h_n + c F(x_{n+1})
// (c = dt / 2m) give, with J = dF/dx symmetric and dU/dx = -F, the adjoint recursion
//     lv_S = 2 v_S,  lx_S = c J(x_S) lv_S - F(x_S) / S,
//     lh_n = lv_{n+1} + dt lx_{n+1},  lv_n = lh_n,
//     lx_n = lx_{n+1} + c J(x_n) (2 lh_n) - F(x_n) / S          (1 <= n <= S-1)
// and dL/dv_0 = lv_0.  Parameter gradients collect c (dF/dtheta . mu) at every force evaluation
// and (1/S) dU/dtheta at every loss term.  One kernel per reverse step covers all three cases
// with (kappa, w_U): mu = kappa lh, lx_out = lx + c J mu - w_U F, lv_out = lh, where the
// terminal step is kappa = 1, w_U = 1/S with lx_in = 0; interior steps kappa = 2, w_U = 1/S;
// the first step (n = 0) kappa = 1, w_U = 0.
//
// Pair terms (r the distance, s = r^2, d the displacement, sr6 = (sigma^2/s)^3):
//     g  = 48 eps sr6 (sr6 - 1/2) / s           force on i is g (x_i - x_j)
//     g' = dg/ds = 48 eps sr6 (2 - 7 sr6) / s^2
//     dg/dsigma = 144 eps sr6 (4 sr6 - 1) / (sigma s)
//     du/dsigma = 24 eps sr6 (2 sr6 - 1) / sigma  (minus du_c/dsigma when r_c is fixed)
//     (J mu)_i = sum_j [g (mu_i - mu_j) + 2 g' (d . (mu_i - mu_j)) d]
// dF/deps = F/eps and dU/deps = U/eps.  Pair arithmetic is FP32 on cell-local coordinates;
// every accumulation of adjoint quantities is FP64.
#include <algorithm>

#include "gbmd_internal.cuh"

namespace gbmd {

__device__ __forceinline__ float offx_a(uint32_t e) { return __uint_as_float(0x4B000000u | (e & 3u)) - 8388609.0f; }
__device__ __forceinline__ float offy4_a(uint32_t e) { return __uint_as_float(0x4B000000u | (e & 12u)) - 8388612.0f; }
__device__ __forceinline__ float offz16_a(uint32_t e) { return __uint_as_float(0x4B000000u | (e & 48u)) - 8388624.0f; }

// One reverse step at the snapshot q of the current segment.  mu[in_buf] holds every atom's
// mu = kappa lh of this step (written by the previous step or by the permute into slot order),
// so a neighbour costs one FP64 3-vector gather; this step writes mu[out_buf] = kappa_next lh'
// for the next one.  The neighbour loop runs NB entries at a time: their W rows, positions and mu
// are loaded together.
constexpr int ADJ_NB = 4;

__global__ void __launch_bounds__(TILE) k_adj_reverse(Arrays A, Scal S, AdjView V, int q, double kappa, double w_U,
                                                      int in_buf, double kappa_next)
{
    __shared__ double sh[TILE / 32][4];
    const int out_buf = in_buf ^ 1;
    const float4* __restrict__ pos = V.pos_snap + int64_t(q) * S.nslots;
    const int32_t* __restrict__ cnt = V.cnt_snap + int64_t(q) * S.nslots;
    const uint32_t* __restrict__ W = V.W_snap + int64_t(q) * S.cap * S.nslots;
    const double* lxi[3] = {V.lx[in_buf][0], V.lx[in_buf][1], V.lx[in_buf][2]};
    const double* lvi[3] = {V.lv[in_buf][0], V.lv[in_buf][1], V.lv[in_buf][2]};
    const double* mu[3] = {V.mu[in_buf][0], V.mu[in_buf][1], V.mu[in_buf][2]};
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const Rep& R = A.rep[A.tile_rep[t]];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        double part[4] = {0.0, 0.0, 0.0, 0.0};
        if (slot - R.slot0 < R.n) {
            const float4 pi = pos[slot];
            double lh[3], mui[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lh[a] = fma(S.dt, lxi[a][slot], lvi[a][slot]);
                mui[a] = mu[a][slot];                                      // = kappa lh
            }
            double jm[3] = {0.0, 0.0, 0.0};
            float f[3] = {0.f, 0.f, 0.f}, fs[3] = {0.f, 0.f, 0.f};
            float u = 0.f, us = 0.f;
            const int mm = min(cnt[slot], S.cap);
            const float wx = R.wf[0], wy4 = 0.25f * R.wf[1], wz16 = 0.0625f * R.wf[2];
            const float wxl = R.wlo[0], wy4l = 0.25f * R.wlo[1], wz16l = 0.0625f * R.wlo[2];
            for (int m0 = 0; m0 < mm; m0 += ADJ_NB) {
                uint32_t e[ADJ_NB];
                float4 pj[ADJ_NB];
                double mj[ADJ_NB][3];
#pragma unroll
                for (int k = 0; k < ADJ_NB; ++k) e[k] = (m0 + k < mm) ? W[int64_t(m0 + k) * S.nslots + slot] : 0u;
#pragma unroll
                for (int k = 0; k < ADJ_NB; ++k) {
                    const bool ok = m0 + k < mm;
                    const int64_t j = ok ? int64_t(e[k] >> IDX_SHIFT) : slot;
                    pj[k] = pos[j];
#pragma unroll
                    for (int a = 0; a < 3; ++a) mj[k][a] = mu[a][j];
                }
#pragma unroll
                for (int k = 0; k < ADJ_NB; ++k) {
                    const uint32_t ek = e[k];
                    const float ox = offx_a(ek), oy = offy4_a(ek), oz = offz16_a(ek);
                    const float dx = fmaf(ox, wxl, fmaf(ox, wx, pj[k].x - pi.x));      // d = x_j - x_i
                    const float dy = fmaf(oy, wy4l, fmaf(oy, wy4, pj[k].y - pi.y));
                    const float dz = fmaf(oz, wz16l, fmaf(oz, wz16, pj[k].z - pi.z));
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    if (m0 + k < mm && r2 < S.rc2f) {
                        const float ri2 = 1.0f / r2;
                        const float sr2 = S.sig2f * ri2;
                        const float sr6 = sr2 * sr2 * sr2;
                        const float g = S.eps48f * sr6 * (sr6 - 0.5f) * ri2;
                        const float gp = S.eps48f * sr6 * (2.0f - 7.0f * sr6) * ri2 * ri2;
                        const float gsg = S.adj_eps144_over_sig * sr6 * (4.0f * sr6 - 1.0f) * ri2;
                        f[0] = fmaf(-g, dx, f[0]); f[1] = fmaf(-g, dy, f[1]); f[2] = fmaf(-g, dz, f[2]);
                        fs[0] = fmaf(-gsg, dx, fs[0]); fs[1] = fmaf(-gsg, dy, fs[1]); fs[2] = fmaf(-gsg, dz, fs[2]);
                        u += fmaf(S.eps4f * sr6, sr6 - 1.0f, -S.ucf);
                        us += fmaf(S.adj_eps24_over_sig * sr6, 2.0f * sr6 - 1.0f, -S.adj_ducf);
                        // mu_i - mu_j in FP64, then FP32 for the pair arithmetic
                        float dm[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) dm[a] = f64_to_f32(mui[a] - mj[k][a]);
                        const float proj = 2.0f * gp * fmaf(dz, dm[2], fmaf(dy, dm[1], dx * dm[0]));
                        jm[0] += f32_to_f64(fmaf(g, dm[0], proj * dx));
                        jm[1] += f32_to_f64(fmaf(g, dm[1], proj * dy));
                        jm[2] += f32_to_f64(fmaf(g, dm[2], proj * dz));
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double fa = f32_to_f64(f[a]);
                const double lxo = fma(S.c, jm[a], lxi[a][slot]) - w_U * fa;
                V.lx[out_buf][a][slot] = lxo;
                V.lv[out_buf][a][slot] = lh[a];
                V.mu[out_buf][a][slot] = kappa_next * fma(S.dt, lxo, lh[a]);
                part[0] += fa * mui[a];
                part[1] += f32_to_f64(fs[a]) * mui[a];
            }
            part[0] *= S.c;
            part[1] *= S.c;
            part[2] = 0.5 * w_U * f32_to_f64(u);
            part[3] = 0.5 * w_U * f32_to_f64(us);
        }
        // tile sums (4 FP64 values), added to this tile's running accumulators
#pragma unroll
        for (int k = 0; k < 4; ++k) part[k] = warp_sum(part[k]);
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) sh[threadIdx.x >> 5][k] = part[k];
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double s = 0.0;
            for (int w = 0; w < TILE / 32; ++w) s += sh[w][threadIdx.x];
            V.tile_acc[int64_t(t) * 4 + threadIdx.x] += s;
        }
        __syncthreads();
    }
}

// adjoint vectors between id order (kept across segments) and this segment's slot order (the
// segment's slot -> id map is a snapshot, so the next segment may already be re-binned)
// (to slot order, also mu = kappa (lv + dt lx) for the segment's first reverse step)
__global__ void __launch_bounds__(TILE) k_adj_to_slot(Arrays A, Scal S, AdjView V, int buf, double kappa)
{
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const Rep& R = A.rep[A.tile_rep[t]];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        const int64_t id = V.id_snap[slot];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double lx = V.lam_x[id * 3 + a], lv = V.lam_v[id * 3 + a];
            V.lx[buf][a][slot] = lx;
            V.lv[buf][a][slot] = lv;
            V.mu[buf][a][slot] = kappa * fma(S.dt, lx, lv);
        }
    }
}

__global__ void __launch_bounds__(TILE) k_adj_to_id(Arrays A, Scal S, AdjView V, int buf)
{
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const Rep& R = A.rep[A.tile_rep[t]];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        const int64_t id = V.id_snap[slot];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            V.lam_x[id * 3 + a] = V.lx[buf][a][slot];
            V.lam_v[id * 3 + a] = V.lv[buf][a][slot];
        }
    }
}

// terminal conditions in id order: lv_S = 2 v_S, lx_S = 0; partial |v_S|^2 per block
__global__ void __launch_bounds__(256) k_adj_init(AdjView V, int64_t n3, const double* __restrict__ vS)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n3; k += int64_t(gridDim.x) * blockDim.x) {
        const double v = vS[k];
        V.lam_v[k] = 2.0 * v;
        V.lam_x[k] = 0.0;
        s = fma(v, v, s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) V.vnorm_part[blockIdx.x] = sh[0];
}

// fixed-order sums: out = [sum c F.mu, sum c F_sigma.mu, sum w_U U, sum w_U dU/dsigma, |v_S|^2]
__global__ void __launch_bounds__(256) k_adj_final(AdjView V, int ntiles, int nvpart)
{
    __shared__ double sh[256][5];
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        for (int k = 0; k < 4; ++k) acc[k] += V.tile_acc[int64_t(t) * 4 + k];
    for (int b = threadIdx.x; b < nvpart; b += blockDim.x) acc[4] += V.vnorm_part[b];
    for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + h][k];
        __syncthreads();
    }
    if (threadIdx.x < 5) V.out[threadIdx.x] = sh[0][threadIdx.x];
}

static int tile_grid(const Scal& S, const Launch& L) { return std::max(1, std::min(L.grid, S.ntiles)); }

cudaError_t launch_adj_reverse(const Arrays& A, const Scal& S, const Launch& L, const AdjView& V, int q, double kappa,
                               double w_U, int in_buf, double kappa_next)
{
    k_adj_reverse<<<tile_grid(S, L), TILE, 0, L.stream>>>(A, S, V, q, kappa, w_U, in_buf, kappa_next);
    return cudaGetLastError();
}

cudaError_t launch_adj_permute(const Arrays& A, const Scal& S, const Launch& L, const AdjView& V, int buf, bool to_slot,
                               double kappa)
{
    if (to_slot) k_adj_to_slot<<<tile_grid(S, L), TILE, 0, L.stream>>>(A, S, V, buf, kappa);
    else k_adj_to_id<<<tile_grid(S, L), TILE, 0, L.stream>>>(A, S, V, buf);
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const AdjView& V, const Launch& L, int64_t n, const double* vS)
{
    k_adj_init<<<ADJ_VPART, 256, 0, L.stream>>>(V, n * 3, vS);
    return cudaGetLastError();
}

cudaError_t launch_adj_final(const AdjView& V, const Launch& L, int ntiles)
{
    k_adj_final<<<1, 256, 0, L.stream>>>(V, ntiles, ADJ_VPART);
    return cudaGetLastError();
}

}  // namespace gbmd
