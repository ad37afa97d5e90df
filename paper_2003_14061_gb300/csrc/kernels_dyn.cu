// kernels_dyn.cu -- velocity autocorrelation and mean-square displacement of atoms followed by
// their permanent ids (Sec. 4.1 item 1: atoms keep their identities through the reorders;
// Sec. 4.1 item 7: the VACF of the dense soft-sphere fluid shows caging).
//
//   k_dyn_sample  one sample at the current state: per atom (indexed by permanent id) the
//                 displacement since the previous sample by the minimum image (unwrapping the
//                 periodic positions), the integer-step velocity v_n = v + c f (the forces were
//                 just evaluated), and for every time origin that is being followed the products
//                 v_i(t0) . v_i(t) and |r_i(t) - r_i(t0)|^2, summed per CTA in FP64.
//   k_dyn_finish  adds the CTAs' sums in CTA order into the per-lag accumulators (deterministic).
#include <algorithm>

#include "gbmd_internal.cuh"

namespace gbmd {

__global__ void __launch_bounds__(TILE) k_dyn_sample(Arrays A, Scal S, DynView D, DynStep P, int cur)
{
    __shared__ double sh[TILE / 32][2 * DYN_MAX_ORG];
    double acc[2 * DYN_MAX_ORG];
#pragma unroll
    for (int q = 0; q < 2 * DYN_MAX_ORG; ++q) acc[q] = 0.0;
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        const int64_t id = A.id[slot];
        // wrapped global position and integer-step velocity, as md_get_state returns them
        uint32_t pw;
        double loc[3];
        if (S.mode == MD_FP64) {
            pw = cell_bits(A.pos64[cur][slot].w);
            loc[0] = A.xl[0][slot]; loc[1] = A.xl[1][slot]; loc[2] = A.xl[2][slot];
        } else {
            const float4 p = A.pos32[cur][slot];
            pw = __float_as_uint(p.w);
            if (S.mode == MD_FP32) { loc[0] = p.x; loc[1] = p.y; loc[2] = p.z; }
            else { loc[0] = A.xl[0][slot]; loc[1] = A.xl[1][slot]; loc[2] = A.xl[2][slot]; }
        }
        int c[3];
        unpack_cell(pw, c[0], c[1], c[2]);
        const int vhalf = A.rs[r].vhalf;
        const double4_32a f = vhalf ? A.f[slot] : make_double4_32a(0, 0, 0, 0);
        const double fq[3] = {f.x, f.y, f.z};
        double vn[3], d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double xa = __dadd_rn(__dmul_rn(double(c[a]), R.w[a]), loc[a]);
            if (xa < 0.0) xa += R.L[a];
            if (xa >= R.L[a]) xa -= R.L[a];
            double v = (S.mode == MD_FP32) ? double(A.v32[a][slot]) : A.v[a][slot];
            if (vhalf) {
                if (S.mode == MD_FP32) v = double(fmaf(float(S.c), float(fq[a]), float(v)));
                else v = fma(S.c, fq[a], v);
            }
            vn[a] = v;
            // displacement since the previous sample: the minimum image of the wrapped difference
            const double dd = xa - D.xprev[id * 3 + a];
            d[a] = dd - R.L[a] * rint(dd / R.L[a]);
            D.xprev[id * 3 + a] = xa;
        }
#pragma unroll
        for (int b = 0; b < DYN_MAX_ORG; ++b) {
            if (b >= P.norg) break;
            double* v0 = D.v0 + (int64_t(b) * D.n + id) * 3;
            double* dr = D.dr + (int64_t(b) * D.n + id) * 3;
            if (b == P.start) {
                v0[0] = vn[0]; v0[1] = vn[1]; v0[2] = vn[2];
                dr[0] = 0.0; dr[1] = 0.0; dr[2] = 0.0;
            } else if (P.lag[b] >= 0) {
                dr[0] += d[0]; dr[1] += d[1]; dr[2] += d[2];
            }
            if (P.lag[b] >= 0) {
                acc[2 * b] += vn[0] * v0[0] + vn[1] * v0[1] + vn[2] * v0[2];
                acc[2 * b + 1] += dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
            }
        }
    }
    // CTA sums in a fixed order: warp butterflies, then the warps in order
#pragma unroll
    for (int q = 0; q < 2 * DYN_MAX_ORG; ++q) {
        const double w = warp_sum(acc[q]);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][q] = w;
    }
    __syncthreads();
    if (threadIdx.x < 2 * P.norg) {
        double s = 0.0;
        for (int k = 0; k < TILE / 32; ++k) s += sh[k][threadIdx.x];
        D.part[int64_t(blockIdx.x) * 2 * DYN_MAX_ORG + threadIdx.x] = s;
    }
}

__global__ void k_dyn_finish(DynView D, DynStep P, int nblocks)
{
    const int q = threadIdx.x;                       // 2 b + (0: VACF, 1: MSD)
    if (q >= 2 * P.norg) return;
    const int b = q >> 1;
    if (P.lag[b] < 0) return;
    double s = 0.0;
    for (int k = 0; k < nblocks; ++k) s += D.part[int64_t(k) * 2 * DYN_MAX_ORG + q];
    double* dst = (q & 1) ? D.msd : D.vacf;
    dst[P.lag[b]] += s;                              // one origin per lag per sample: no race
}

cudaError_t launch_dyn_sample(const Arrays& A, const Scal& S, const Launch& L, const DynView& D, const DynStep& P,
                              int cur)
{
    const int g = std::max(1, std::min(std::min(L.grid, DYN_BLOCKS), S.ntiles));
    k_dyn_sample<<<g, TILE, 0, L.stream>>>(A, S, D, P, cur);
    k_dyn_finish<<<1, 2 * DYN_MAX_ORG, 0, L.stream>>>(D, P, g);
    return cudaGetLastError();
}

}  // namespace gbmd
