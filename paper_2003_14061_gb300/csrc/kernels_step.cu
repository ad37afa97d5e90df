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
//              and raises the rebuild flag.  With PROPS, the step also forms F2 (U, K, virial,
//              momentum): MD_FP64 tiles write FP64 partial sums for k_props_reduce; the MD_MIXED
//              and MD_FP32 kernels add their warp sums in fixed point and the warp that completes
//              a replica writes its props (no further launch).
//   k_step_sm  the same for MD_MIXED and MD_FP32 (step kernel 1): warps take 32-slot warp-tiles
//              from the slot range of the SM they run on, so the warps of an SM gather from one
//              neighbourhood held in its L1.  k_step runs MD_FP64 and step kernel 3.
//   k_step<..., STG = true>  the same with each tile's neighbour positions staged in shared
//              memory by cp.async.bulk first (step kernel 3).
//   k_step_bulk  the same arithmetic with the tile's state and W rows in a two-stage shared-memory
//              ring filled by cp.async.bulk (step kernel 2).  The four forms share the pair loop
//              and the kick-drift, so they give bit-identical trajectories.
//   k_forces   F1 alone: f_i, u_i and the per-atom virial at the current positions.
//   k_props_*  F2 outside the step (and for MD_FP64 steps): per-warp FP64 partials, then CTA
//              slices per replica summed in a fixed order (deterministic).
#include <algorithm>
#include <type_traits>

#include "gbmd_internal.cuh"

namespace gbmd {

// Periodic offsets of a W entry as exact floats without conversion ops: OR-ing the code bits into
// the mantissa of 2^23 gives 2^23 + code (the *_raw values); subtracting 2^23 + (the code of
// offset 0) leaves o_x, 4 o_y and 16 o_z, which multiply w_x, w_y / 4 and w_z / 16 (exact
// power-of-two scalings).
__device__ __forceinline__ float offx_raw(uint32_t e) { return __uint_as_float(0x4B000000u | (e & 3u)); }
__device__ __forceinline__ float offy_raw(uint32_t e) { return __uint_as_float(0x4B000000u | (e & 12u)); }
__device__ __forceinline__ float offz_raw(uint32_t e) { return __uint_as_float(0x4B000000u | (e & 48u)); }

// reciprocal to ~1 ulp (the force tolerance is 1e-5 relative)
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/r^2 for the pair terms: the approximation above refined by one Newton-Raphson step for the
// reciprocal, y <- y + y (1 - x y), which leaves about half an ulp of error with no bias (u(r)
// takes the error of 1/r^2 six times over, r^-12 = (r^-2)^6, and the energy sums millions of
// such terms).  Lanes whose r^2 is 0 (padding, masked afterwards) give NaN here, never used.
__device__ __forceinline__ float2 rcp2_nr(float2 x)
{
    const float2 y = make_float2(rcp_approx(x.x), rcp_approx(x.y));
    const float2 e = __ffma2_rn(make_float2(-x.x, -x.y), y, make_float2(1.0f, 1.0f));
    return __ffma2_rn(y, e, y);
}
__device__ __forceinline__ float rcp_nr(float x)
{
    const float y = rcp_approx(x);
    return __fmaf_rn(y, __fmaf_rn(-x, y, 1.0f), y);
}

// ------------------------------------------------------------------------------------------
// pair loops
// ------------------------------------------------------------------------------------------
struct AccF { float fx, fy, fz, u, w; };
struct AccD { double fx, fy, fz, u, w; };

// With polymer chains the chain terms of every atom are first added into the FP32 buffers
// fbuf / wbuf by k_chain_terms; the force passes add the buffers in and clear them.
__device__ __forceinline__ void add_buffer(const Arrays& A, int64_t slot, AccF& a)
{
    const float4 b = A.fbuf[slot];
    a.fx += b.x; a.fy += b.y; a.fz += b.z; a.u += b.w;
    a.w += A.wbuf[slot];
    A.fbuf[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    A.wbuf[slot] = 0.f;
}

// One thread per atom over its column of W, NB entries at a time; wr(m) returns the m-th entry
// and pr(e) the FP32 cell-local position of the neighbour an entry names.
// The entries of batch b+1 are read together with the position gathers of batch b, so each
// thread keeps 2 NB loads in flight and a batch waits for one memory latency, not two.  The
// arithmetic runs on packed FP32x2 operations (one instruction for two lanes, each lane rounded as
// the scalar operation): entries 2k and 2k+1 of the column go to lanes x and y, and the two
// lanes' sums are added at the end, so the summation order is the same for every NB and every
// source of the entries.
template <int NB, class WRead, class PRead>
__device__ __forceinline__ AccF pair_loop_f32(const Scal& S, const Rep& R, float4 pi, int mm, WRead wr, PRead pr)
{
    static_assert(NB % 2 == 0, "W entries are processed in pairs");
    const float2 wx = make_float2(R.wf[0], R.wf[0]);
    const float2 wy4 = make_float2(0.25f * R.wf[1], 0.25f * R.wf[1]);
    const float2 wz16 = make_float2(0.0625f * R.wf[2], 0.0625f * R.wf[2]);
    const float2 wxl = make_float2(R.wlo[0], R.wlo[0]);
    const float2 wy4l = make_float2(0.25f * R.wlo[1], 0.25f * R.wlo[1]);
    const float2 wz16l = make_float2(0.0625f * R.wlo[2], 0.0625f * R.wlo[2]);
    const float2 npx = make_float2(-pi.x, -pi.x), npy = make_float2(-pi.y, -pi.y), npz = make_float2(-pi.z, -pi.z);
    const float2 sig2 = make_float2(S.sig2f, S.sig2f), eps48 = make_float2(S.eps48f, S.eps48f);
    float2 fx = make_float2(0.f, 0.f), fy = fx, fz = fx, u = fx, w = fx;
    uint32_t e[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) e[k] = (k < mm) ? wr(k) : 0u;
    for (int m0 = 0; m0 < mm; m0 += NB) {
        float4 pj[NB];
#pragma unroll
        // entries past mm are 0 (slot 0, a valid address) and masked below; with 4 or 8 entries
        // per batch the unconditional gathers measured faster (LJ, 8 per batch: 2.61 against
        // 2.73 ms), with 2 slower (0.227 against 0.206 ms), so the select stays there
        for (int k = 0; k < NB; ++k) pj[k] = (NB >= 4 || m0 + k < mm) ? pr(e[k]) : pi;
        uint32_t en[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) en[k] = (m0 + NB + k < mm) ? wr(m0 + NB + k) : 0u;
#pragma unroll
        for (int k = 0; k < NB; k += 2) {
            const uint32_t e0 = e[k], e1 = e[k + 1];
            const float2 ox = __fadd2_rn(make_float2(offx_raw(e0), offx_raw(e1)), make_float2(-8388609.0f, -8388609.0f));
            const float2 oy = __fadd2_rn(make_float2(offy_raw(e0), offy_raw(e1)), make_float2(-8388612.0f, -8388612.0f));
            const float2 oz = __fadd2_rn(make_float2(offz_raw(e0), offz_raw(e1)), make_float2(-8388624.0f, -8388624.0f));
            const float2 dx = __ffma2_rn(ox, wxl, __ffma2_rn(ox, wx, __fadd2_rn(make_float2(pj[k].x, pj[k + 1].x), npx)));
            const float2 dy = __ffma2_rn(oy, wy4l, __ffma2_rn(oy, wy4, __fadd2_rn(make_float2(pj[k].y, pj[k + 1].y), npy)));
            const float2 dz = __ffma2_rn(oz, wz16l, __ffma2_rn(oz, wz16, __fadd2_rn(make_float2(pj[k].z, pj[k + 1].z), npz)));
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const bool in0 = (m0 + k < mm) && r2.x < S.rc2f;
            const bool in1 = (m0 + k + 1 < mm) && r2.y < S.rc2f;
            const float2 ri2 = rcp2_nr(r2);
            const float2 sr2 = __fmul2_rn(sig2, ri2);
            const float2 sr6 = __fmul2_rn(__fmul2_rn(sr2, sr2), sr2);
            float2 fs = __fmul2_rn(__fmul2_rn(__fmul2_rn(eps48, sr6), __fadd2_rn(sr6, make_float2(-0.5f, -0.5f))), ri2);
            fs.x = in0 ? fs.x : 0.0f;                                      // g(r^2), zero outside r_c
            fs.y = in1 ? fs.y : 0.0f;
            fx = __ffma2_rn(fs, dx, fx);                                   // sum g (x_j - x_i)
            fy = __ffma2_rn(fs, dy, fy);
            fz = __ffma2_rn(fs, dz, fz);
            float2 ut = __ffma2_rn(__fmul2_rn(make_float2(S.eps4f, S.eps4f), sr6),
                                   __fadd2_rn(sr6, make_float2(-1.0f, -1.0f)), make_float2(-S.ucf, -S.ucf));
            ut.x = in0 ? ut.x : 0.0f;
            ut.y = in1 ? ut.y : 0.0f;
            u = __fadd2_rn(u, ut);
            w = __ffma2_rn(fs, r2, w);
        }
#pragma unroll
        for (int k = 0; k < NB; ++k) e[k] = en[k];
    }
    // f_i = sum g (x_i - x_j) = -(sum g (x_j - x_i))
    return AccF{-(fx.x + fx.y), -(fy.x + fy.y), -(fz.x + fz.y), u.x + u.y, w.x + w.y};
}

// the pair loop with W read from global memory, over the first mm rows of the atom's column
template <int NB>
__device__ __forceinline__ AccF force_f32_rows(const Arrays& A, const Scal& S, const Rep& R,
                                               const float4* __restrict__ pos, int64_t slot, float4 pi, int mm)
{
    const uint32_t* __restrict__ Wc = A.W + slot;
    const int64_t ns = S.nslots;
    return pair_loop_f32<NB>(S, R, pi, mm, [=](int m) { return __ldcs(Wc + int64_t(m) * ns); },
                             [=](uint32_t e) { return __ldg(pos + (e >> IDX_SHIFT)); });
}

template <int NB>
__device__ __forceinline__ AccF force_f32(const Arrays& A, const Scal& S, const Rep& R,
                                          const float4* __restrict__ pos, int64_t slot, float4 pi)
{
    return force_f32_rows<NB>(A, S, R, pos, slot, pi, min(__ldcs(A.nbr_count + slot), S.cap));
}

// Two pairs (lanes x and y) of the FP32 pair loop: g(r^2) with the in-range masks, accumulated
// into f (sum g (x_j - x_i)), u_i and the virial.
__device__ __forceinline__ void pair2(const Scal& S, float2 dx, float2 dy, float2 dz, bool in0, bool in1,
                                      float2& fx, float2& fy, float2& fz, float2& u, float2& w)
{
    const float2 sig2 = make_float2(S.sig2f, S.sig2f), eps48 = make_float2(S.eps48f, S.eps48f);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    in0 = in0 && r2.x < S.rc2f;
    in1 = in1 && r2.y < S.rc2f;
    const float2 ri2 = rcp2_nr(r2);
    const float2 sr2 = __fmul2_rn(sig2, ri2);
    const float2 sr6 = __fmul2_rn(__fmul2_rn(sr2, sr2), sr2);
    float2 fs = __fmul2_rn(__fmul2_rn(__fmul2_rn(eps48, sr6), __fadd2_rn(sr6, make_float2(-0.5f, -0.5f))), ri2);
    fs.x = in0 ? fs.x : 0.0f;
    fs.y = in1 ? fs.y : 0.0f;
    fx = __ffma2_rn(fs, dx, fx);
    fy = __ffma2_rn(fs, dy, fy);
    fz = __ffma2_rn(fs, dz, fz);
    float2 ut = __ffma2_rn(__fmul2_rn(make_float2(S.eps4f, S.eps4f), sr6), __fadd2_rn(sr6, make_float2(-1.0f, -1.0f)),
                           make_float2(-S.ucf, -S.ucf));
    ut.x = in0 ? ut.x : 0.0f;
    ut.y = in1 ? ut.y : 0.0f;
    u = __fadd2_rn(u, ut);
    w = __ffma2_rn(fs, r2, w);
}

// F1 without a neighbour matrix (step kernel 4, the cell-block alternative of Sec. 4.2 item 1).
// The atoms are in cell order (reordered at every rebuild), so the 3 cells of each row around the
// atom are one contiguous run of slots; every atom of the 27 cells is tested against r_c at the
// current positions.  The cells, of side >= r_c + skin, were binned at the last rebuild and no
// atom has moved more than skin/2 since, so no pair within r_c is missed.  Two candidates at a
// time go through the packed pair arithmetic; the offset of a candidate's cell is o w, as in
// the neighbour-matrix loop.
__device__ __forceinline__ AccF force_f32_cells(const Arrays& A, const Scal& S, const Rep& R,
                                                const float4* __restrict__ pos, int64_t slot, float4 pi)
{
    int cx, cy, cz;
    unpack_cell(__float_as_uint(pi.w), cx, cy, cz);
    const int2* __restrict__ ck = A.ckeep;                  // [start, end) of each cell in the replica
    const int64_t sbase = R.slot0;                          // slot of replica cell-order position k
    const int ncx = R.nc[0];
    const float wx = R.wf[0], wxl = R.wlo[0];
    const float2 npx = make_float2(-pi.x, -pi.x), npy = make_float2(-pi.y, -pi.y), npz = make_float2(-pi.z, -pi.z);
    float2 fx = make_float2(0.f, 0.f), fy = fx, fz = fx, u = fx, w = fx;
    const int xs[3] = {(cx == 0) ? ncx - 1 : cx - 1, cx, (cx == ncx - 1) ? 0 : cx + 1};
    const bool inner = cx > 0 && cx < ncx - 1;
    for (int oz = -1; oz <= 1; ++oz) {
        int nz = cz + oz; nz += (nz < 0) ? R.nc[2] : 0; nz -= (nz >= R.nc[2]) ? R.nc[2] : 0;
        const float2 offz = make_float2(float(oz) * R.wf[2], float(oz) * R.wf[2]);
        const float2 offzl = make_float2(float(oz) * R.wlo[2], float(oz) * R.wlo[2]);
        for (int oy = -1; oy <= 1; ++oy) {
            int ny = cy + oy; ny += (ny < 0) ? R.nc[1] : 0; ny -= (ny >= R.nc[1]) ? R.nc[1] : 0;
            const float2 offy = make_float2(float(oy) * R.wf[1], float(oy) * R.wf[1]);
            const float2 offyl = make_float2(float(oy) * R.wlo[1], float(oy) * R.wlo[1]);
            const int row = R.cell0 + row_pos(R, ny, nz) * ncx;
            // runs [b, e) with their x offsets: one run of three cells, or three at a wrap in x
            const int nrun = inner ? 1 : 3;
            for (int q = 0; q < nrun; ++q) {
                const int b = inner ? ck[row + cx - 1].x : ck[row + xs[q]].x;
                const int e = inner ? ck[row + cx + 1].y : ck[row + xs[q]].y;
                const int b1 = inner ? ck[row + cx].x : e, b2 = inner ? ck[row + cx + 1].x : e;
                const float oq = inner ? -1.0f : float(q - 1);
                for (int k0 = b; k0 < e; k0 += 2) {
                    const int k1 = k0 + 1;
                    const bool v1 = k1 < e;
                    const int64_t j0 = sbase + k0, j1 = sbase + (v1 ? k1 : k0);
                    const float4 p0 = __ldg(pos + j0), p1 = __ldg(pos + j1);
                    // o_x of each candidate: the run's first cell, +1 past b1, +2 past b2
                    const float o0 = oq + float(k0 >= b1) + float(k0 >= b2);
                    const float o1 = oq + float(k1 >= b1) + float(k1 >= b2);
                    const float2 dx = __ffma2_rn(make_float2(o0, o1), make_float2(wxl, wxl),
                                                 __ffma2_rn(make_float2(o0, o1), make_float2(wx, wx),
                                                            __fadd2_rn(make_float2(p0.x, p1.x), npx)));
                    const float2 dy = __fadd2_rn(__fadd2_rn(__fadd2_rn(make_float2(p0.y, p1.y), npy), offy), offyl);
                    const float2 dz = __fadd2_rn(__fadd2_rn(__fadd2_rn(make_float2(p0.z, p1.z), npz), offz), offzl);
                    pair2(S, dx, dy, dz, j0 != slot, v1 && j1 != slot, fx, fy, fz, u, w);
                }
            }
        }
    }
    return AccF{-(fx.x + fx.y), -(fy.x + fy.y), -(fz.x + fz.y), u.x + u.y, w.x + w.y};
}

// Step kernel 5, first pass: forces over the half neighbour list with Newton's third law (the
// paper keeps the full list so that F1 reads W coalesced and writes nothing scattered, Sec. 2.3).
// Every pair is evaluated once, by the atom of the lower slot: its force, energy and virial go to
// that atom in registers and to the partner by one vector atomic add (force and u) and one scalar
// atomic add (virial) into fbuf / wbuf; each atom then adds its own sums the same way.  u_i and
// the virial keep the full-list convention (each pair counted at both atoms).  The atomics add in
// no fixed order, so results vary between runs in the last bits.
template <int NB>
__global__ void __launch_bounds__(TILE) k_half_pairs(Arrays A, Scal S, int cur)
{
    const float4* __restrict__ pos = A.pos32[cur];
    const int64_t ns = S.nslots;
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const Rep& R = A.rep[A.tile_rep[t]];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        const float4 pi = __ldg(pos + slot);
        const int mm = min(__ldcs(A.nbr_count + slot), S.cap);
        const uint32_t* __restrict__ Wc = A.W + slot;
        const float wx = R.wf[0], wy4 = 0.25f * R.wf[1], wz16 = 0.0625f * R.wf[2];
        const float wxl = R.wlo[0], wy4l = 0.25f * R.wlo[1], wz16l = 0.0625f * R.wlo[2];
        float fx = 0.f, fy = 0.f, fz = 0.f, u = 0.f, w = 0.f;
        for (int m0 = 0; m0 < mm; m0 += NB) {
            uint32_t e[NB];
            float4 pj[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) e[k] = (m0 + k < mm) ? __ldcs(Wc + int64_t(m0 + k) * ns) : 0u;
#pragma unroll
            for (int k = 0; k < NB; ++k) pj[k] = (m0 + k < mm) ? __ldg(pos + (e[k] >> IDX_SHIFT)) : pi;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const float ox = offx_raw(e[k]) - 8388609.0f, oy = offy_raw(e[k]) - 8388612.0f;
                const float oz = offz_raw(e[k]) - 8388624.0f;
                const float dx = fmaf(ox, wxl, fmaf(ox, wx, pj[k].x - pi.x));
                const float dy = fmaf(oy, wy4l, fmaf(oy, wy4, pj[k].y - pi.y));
                const float dz = fmaf(oz, wz16l, fmaf(oz, wz16, pj[k].z - pi.z));
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (m0 + k < mm && r2 < S.rc2f) {
                    const float ri2 = rcp_nr(r2);
                    const float sr2 = S.sig2f * ri2;
                    const float sr6 = sr2 * sr2 * sr2;
                    const float fs = S.eps48f * sr6 * (sr6 - 0.5f) * ri2;     // g(r^2)
                    const float ut = fmaf(S.eps4f * sr6, sr6 - 1.0f, -S.ucf);
                    const float wt = fs * r2;
                    fx = fmaf(fs, dx, fx);                                  // sum g (x_j - x_i)
                    fy = fmaf(fs, dy, fy);
                    fz = fmaf(fs, dz, fz);
                    u += ut;
                    w += wt;
                    const int64_t j = e[k] >> IDX_SHIFT;
                    atomicAdd(A.fbuf + j, make_float4(fs * dx, fs * dy, fs * dz, ut));   // on j: +g (x_j - x_i)
                    atomicAdd(A.wbuf + j, wt);
                }
            }
        }
        atomicAdd(A.fbuf + slot, make_float4(-fx, -fy, -fz, u));
        atomicAdd(A.wbuf + slot, w);
    }
}

// md_compute_forces / md_get_state with step kernel 5: the accumulated half-list forces into the
// FP64 force array, the buffers cleared for the next step
__global__ void __launch_bounds__(TILE) k_half_to_f(Arrays A, Scal S)
{
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const Rep& R = A.rep[A.tile_rep[t]];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        const float4 b = A.fbuf[slot];
        const AccF a{b.x, b.y, b.z, b.w, A.wbuf[slot]};
        A.f[slot] = make_double4_32a(a.fx, a.fy, a.fz, a.u);
        A.wvir[slot] = a.w;
        A.fbuf[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
        A.wbuf[slot] = 0.f;
    }
}

// ------------------------------------------------------------------------------------------
// polymer chains (md_set_chains; Sec. 4.3 item 2): one thread per atom and all its interactions
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void cross3(const float* a, const float* b, float* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot3(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Adds to a the force on the atom at `slot` from the chain terms that contain it (the bonds to
// its chain neighbours, the bends centred on it and on them, the dihedrals through it), its share
// of their energy (a bond's energy to both atoms, a bend's 2/3 to each of three, a dihedral's 1/2
// to each of four, so that (1/2) sum_i u_i counts every term once) and of their virial
// (2 (r_i - r_first) . f_i, r_first the term's first atom).  Positions are relative to the atom:
// a chain neighbour's cell-local position, found through its permanent id, plus its cell's offset
// (the nearest periodic image of the cell difference) times the cell side.
__device__ __forceinline__ void chain_terms(const Arrays& A, const Scal& S, const Rep& R, const float4* pos, int64_t slot,
                                         float4 pi, AccF& acc)
{
    const int q = A.id[slot] - R.id0;
    const int c0 = (q / S.chain_len) * S.chain_len;
    const int c1 = min(c0 + S.chain_len, R.n);              // the chain: local ids c0 .. c1-1
    int ci[3];
    unpack_cell(__float_as_uint(pi.w), ci[0], ci[1], ci[2]);
    const float pc[3] = {pi.x, pi.y, pi.z};
    float r[7][3];                                          // chain atoms q-3 .. q+3
    bool ok[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) {
        const int qq = q + d - 3;
        ok[d] = qq >= c0 && qq < c1;
        r[d][0] = r[d][1] = r[d][2] = 0.0f;
        if (d != 3 && ok[d]) {
            const float4 pj = pos[A.slot_of_id[R.id0 + qq]];
            int cj[3];
            unpack_cell(__float_as_uint(pj.w), cj[0], cj[1], cj[2]);
            const float pp[3] = {pj.x, pj.y, pj.z};
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                int dc = cj[x] - ci[x];
                if (2 * dc > R.nc[x]) dc -= R.nc[x];
                if (2 * dc < -R.nc[x]) dc += R.nc[x];
                r[d][x] = fmaf(float(dc), R.wlo[x], (pp[x] - pc[x]) + float(dc) * R.wf[x]);
            }
        }
    }
    float f[3] = {0.f, 0.f, 0.f}, u = 0.f, w = 0.f;
    // bonds (i-1, i) and (i, i+1): f_i = -g (r_i - r_{i-1}) and +g (r_{i+1} - r_i)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        if (!ok[side ? 4 : 2]) continue;
        const float* o = r[side ? 4 : 2];
        const float b2 = dot3(o, o), qf = 1.0f - b2 / S.ch_r0sq;
        const float g = S.ch_kb / qf;
#pragma unroll
        for (int x = 0; x < 3; ++x) f[x] += g * o[x];       // towards the partner either way
        u += -0.5f * S.ch_kb * S.ch_r0sq * logf(qf);
        if (!side) w += -2.0f * g * b2;                     // r_i - r_first = r_i - r_{i-1}
    }
    // bends with first atom s = i-2, i-1, i (the atom is term atom t = i - s)
    if (S.ch_ka != 0.0f) {
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int s0 = 3 - t;                             // index of the term's first atom in r
            if (!(ok[s0] && ok[s0 + 1] && ok[s0 + 2])) continue;
            float b1[3], b2[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                b1[x] = r[s0 + 1][x] - r[s0][x];
                b2[x] = r[s0 + 2][x] - r[s0 + 1][x];
            }
            const float l1 = sqrtf(dot3(b1, b1)), l2 = sqrtf(dot3(b2, b2));
            const float c = dot3(b1, b2) / (l1 * l2);
            float fr[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const float g1 = b2[x] / (l1 * l2) - c * b1[x] / (l1 * l1);
                const float g2 = b1[x] / (l1 * l2) - c * b2[x] / (l2 * l2);
                fr[x] = S.ch_ka * (t == 0 ? -g1 : (t == 1 ? g1 - g2 : g2));
                f[x] += fr[x];
            }
            u += (2.0f / 3.0f) * S.ch_ka * (1.0f - c);
            w += -2.0f * dot3(r[s0], fr);
        }
    }
    // dihedrals with first atom s = i-3 .. i
    if (S.ch_kd != 0.0f) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int s0 = 3 - t;
            if (!(ok[s0] && ok[s0 + 1] && ok[s0 + 2] && ok[s0 + 3])) continue;
            float b1[3], b2[3], b3[3], m1[3], m2[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                b1[x] = r[s0 + 1][x] - r[s0][x];
                b2[x] = r[s0 + 2][x] - r[s0 + 1][x];
                b3[x] = r[s0 + 3][x] - r[s0 + 2][x];
            }
            cross3(b1, b2, m1);
            cross3(b2, b3, m2);
            const float q1 = sqrtf(dot3(m1, m1)), q2 = sqrtf(dot3(m2, m2)), bb = dot3(b2, b2);
            if (q1 < 1e-6f * bb || q2 < 1e-6f * bb) continue;
            const float c = dot3(m1, m2) / (q1 * q2);
            float G1[3], G2[3], d1[3], d2a[3], d2b[3], d3[3], fr[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                G1[x] = m2[x] / (q1 * q2) - c * m1[x] / (q1 * q1);
                G2[x] = m1[x] / (q1 * q2) - c * m2[x] / (q2 * q2);
            }
            cross3(b2, G1, d1);
            cross3(G1, b1, d2a);
            cross3(b3, G2, d2b);
            cross3(G2, b2, d3);
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const float d2 = d2a[x] + d2b[x];
                fr[x] = S.ch_kd * (t == 0 ? -d1[x] : (t == 1 ? d1[x] - d2 : (t == 2 ? d2 - d3[x] : d3[x])));
                f[x] += fr[x];
            }
            u += 0.5f * S.ch_kd * (1.0f - c);
            w += -2.0f * dot3(r[s0], fr);
        }
    }
    acc.fx += f[0];
    acc.fy += f[1];
    acc.fz += f[2];
    acc.u += u;
    acc.w += w;
}

// The chain terms of every atom into fbuf / wbuf (one thread per atom, its own slot only; run
// before the force pass that adds the buffers, or after k_half_pairs on the same stream)
__global__ void __launch_bounds__(TILE) k_chain_terms(Arrays A, Scal S, int cur)
{
    const float4* __restrict__ pos = A.pos32[cur];
    for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
        const Rep& R = A.rep[A.tile_rep[t]];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        if (slot - R.slot0 >= R.n) continue;
        AccF a{0.f, 0.f, 0.f, 0.f, 0.f};
        chain_terms(A, S, R, pos, slot, pos[slot], a);
        const float4 b = A.fbuf[slot];
        A.fbuf[slot] = make_float4(b.x + a.fx, b.y + a.fy, b.z + a.fz, b.w + a.u);
        A.wbuf[slot] += a.w;
    }
}

// Leapfrog kick and drift of one atom (Sec. 4.3 item 1) from its force a: MD_MIXED advances the
// FP64 state (v, x), MD_FP32 the FP32 velocity v32 and position pi; pn receives the FP32
// cell-local position of step n+1.  FP32<->FP64 conversions round to nearest.  Returns
// |x_{n+1} - x_n|^2 measured on the FP32 positions (the refresh metric unless the rule is DISP).
// With PROPS, part receives this atom's terms of the props at step n in FP32 -- u_i, |v_n|^2,
// the virial and v_n -- which the warp sums in FP32 and beyond the warp exactly (fixed point; the
// MD_MIXED contract allows FP64 there): v_n = v + c f from the FP32 rounding of the stored
// velocity, so the props cost no FP64 arithmetic (1/64 of the FP32 rate on GB300).
template <int MODE, bool PROPS>
__device__ __forceinline__ float kick_drift(const Scal& S, int vhalf, const float4& pi, const AccF& a,
                                            double (&v)[3], double (&x)[3], float (&v32)[3], float (&pn)[3],
                                            float (&part)[NPROP])
{
    const float f[3] = {a.fx, a.fy, a.fz};
    const float cf = float(S.c);
    float vn2 = 0.0f;
    if (MODE == MD_MIXED) {
        const double kick = vhalf ? 2.0 * S.c : S.c;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double fq = f32_to_f64(f[q]);
            if (PROPS) {
                const float vf = f64_to_f32(v[q]);
                const float vn = vhalf ? fmaf(cf, f[q], vf) : vf;
                vn2 = fmaf(vn, vn, vn2);
                part[3 + q] = vn;
            }
            v[q] = fma(kick, fq, v[q]);
            x[q] = fma(S.dt, v[q], x[q]);
            pn[q] = f64_to_f32(x[q]);
        }
    } else {
        const float kick = float(vhalf ? 2.0 * S.c : S.c);
        const float dtf = float(S.dt);
        const float pc[3] = {pi.x, pi.y, pi.z};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (PROPS) {
                const float vn = vhalf ? fmaf(cf, f[q], v32[q]) : v32[q];
                vn2 = fmaf(vn, vn, vn2);
                part[3 + q] = vn;
            }
            v32[q] = fmaf(kick, f[q], v32[q]);
            pn[q] = fmaf(dtf, v32[q], pc[q]);
        }
    }
    if (PROPS) {
        part[0] = a.u;
        part[1] = vn2;
        part[2] = a.w;
        part[NPROP - 1] = vn2;
    }
    // |x_{n+1} - x_n| = dt |v_{n+1/2}| from the FP32 copies of both positions (same cell frame);
    // the per-step rounding margin is added in the finish
    const float d0 = pn[0] - pi.x, d1 = pn[1] - pi.y, d2 = pn[2] - pi.z;
    return fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
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
        const double4_32a pj = pos[e >> IDX_SHIFT];
        const double dx = fma(double(int(e & 3u) - 1), R.w[0], pj.x - pi.x);
        const double dy = fma(double(int((e >> 2) & 3u) - 1), R.w[1], pj.y - pi.y);
        const double dz = fma(double(int((e >> 4) & 3u) - 1), R.w[2], pj.z - pi.z);
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

// Per-tile FP64 sums of the 7 additive quantities and the FP32 maximum of |v|^2.  The 8 values
// (FP64 for MD_FP64 and the standalone reduction, FP32 in the MD_MIXED / MD_FP32 step kernels)
// of each lane are reduced across the warp by reduce-scatter (each exchange halves the number of
// quantities a lane carries, 4 + 2 + 1 adds, then 2 more over the last 4 lanes): 9 FP64 adds per
// lane instead of 35 for a butterfly per quantity (FP64 runs at 1/64-1/72 of the FP32 rate on
// GB300).
// The in-warp part: lane 4q (q < NPROP - 1) ends with the warp's sum of quantity q, lane 0 also
// with the warp's maximum of |v|^2 (returned in vm).
template <class T>
__device__ __forceinline__ T warp_partials(T (&p)[NPROP], int& q, float& vm)
{
    const int lane = threadIdx.x & 31;
    vm = warp_max(float(p[NPROP - 1]));
    p[NPROP - 1] = T(0);
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    T a4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T keep = h16 ? p[4 + k] : p[k], give = h16 ? p[k] : p[4 + k];
        a4[k] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
    T a2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const T keep = h8 ? a4[2 + k] : a4[k], give = h8 ? a4[k] : a4[2 + k];
        a2[k] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    T a1 = (h4 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? a2[0] : a2[1], 4);
    a1 += __shfl_xor_sync(0xffffffffu, a1, 2);
    a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
    q = (h16 ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0);
    return a1;
}

// the NPROP values of one warp into dst[0..NPROP) (FP64; from FP32 lanes the warp's sums are
// formed in FP32 and widened exactly)
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x) { return f32_to_f64(x); }

template <class T>
__device__ __forceinline__ void warp_partials_store(T (&p)[NPROP], double* dst)
{
    const int lane = threadIdx.x & 31;
    int q;
    float vm;
    const T a1 = warp_partials(p, q, vm);
    if ((lane & 3) == 0 && q != NPROP - 1) dst[q] = widen(a1);
    if (lane == 0) dst[NPROP - 1] = widen(vm);
}

// Each warp of a tile stores its NPROP values at warp_part[(t * TILE / 32 + warp) * NPROP]; the
// props kernel adds a tile's warps in warp order.  No fence or counter is needed between the
// step kernel and that kernel (the launch boundary orders them), so a warp never waits for its
// own stores.
__device__ __forceinline__ double* warp_slot(const Arrays& A, int64_t warp_tile) { return A.warp_part + warp_tile * NPROP; }

// The props of replica r from its sums (acc[0] = sum u_i, acc[1] = sum |v|^2, acc[2] = sum w_i,
// acc[3..5] = sum v, acc[NPROP-1] = max |v|^2), with the constant factors U = sum u_i / 2,
// K = m sum v^2 / 2, W = sum w_i / 2, P = m sum v; with to_series also the time-series row.  One
// thread.
__device__ void write_props(const Arrays& A, const Scal& S, int r, const double (&acc)[NPROP], int step_lag,
                            int to_series)
{
    const Rep& R = A.rep[r];
    RepState& st = A.rs[r];
    const double U = 0.5 * acc[0], K = 0.5 * S.mass * acc[1], W = 0.5 * acc[2];
    const double V = R.L[0] * R.L[1] * R.L[2];
    md_props pr;
    pr.U = U;
    pr.K = K;
    pr.E_per_atom = (U + K) / double(R.n);
    pr.virial = W;
    pr.pressure = (2.0 * K + W) / (3.0 * V);
    pr.P[0] = S.mass * acc[3]; pr.P[1] = S.mass * acc[4]; pr.P[2] = S.mass * acc[5];
    pr.vmax = sqrt(acc[NPROP - 1]);
    pr.mean_nbrs = double(st.sum_nbrs) / double(R.n);
    pr.step = st.step - step_lag;
    pr.rebuilds = st.rebuilds;
    pr.max_cell_occ = st.max_occ;
    pr.max_nbrs = st.max_nbrs;
    pr.reorders = st.reorders;
    A.props[r] = pr;
    if (to_series) {
        // ring of series_cap rows laid out [row][replica][column]: the latest row of every
        // replica is contiguous (one copy reads it)
        const int row = st.series_rows % S.series_cap;
        double* o = A.series + (int64_t(row) * S.nrep + r) * SERIES_COLS;
        o[0] = double(pr.step); o[1] = U; o[2] = K; o[3] = W; o[4] = pr.pressure;
        o[5] = pr.P[0]; o[6] = pr.P[1]; o[7] = pr.P[2]; o[8] = pr.vmax;
        st.series_rows += 1;
    }
}

// Props fused into the MD_MIXED / MD_FP32 step kernels, in fixed point: each warp-tile's FP32
// warp sums (lane 4q holds quantity q) are rounded to multiples of 2^-24 and added to one int64
// per lane; each warp adds its totals to the replica's int64 sums with atomics, and the warp that
// completes the replica writes the props.  Integer sums do not depend on the order, so the props
// are the same bits whichever warp computed which warp-tile, in every step kernel.  The step
// 2^-24 is below the rounding of the FP32 warp sums themselves (for a sum of order 1, half an ulp
// is 6e-8); the range, 2^39 = 5.5e11 per replica, is hundreds of times what a 1e9-atom state at
// T = 1 sums to.  A warp sum of 2^31 or more (overlapping atoms) is added in FP64 instead, so it
// cannot wrap the integers.  The largest |v|^2 goes through an atomic maximum.
constexpr float PROPS_FIX = 16777216.0f;            // 2^24
constexpr float PROPS_FIX_MAX = 2147483648.0f;      // 2^31: larger warp sums go to pbig
struct PropsAcc {
    long long a;                                    // this lane's quantity (lane 4q: quantity q)
    float vm;                                       // max |v|^2 seen by the warp
};

__device__ __forceinline__ void props_warp_add(const Arrays& A, int r, float (&p)[NPROP], PropsAcc& pa)
{
    int q;
    float vm;
    const float a1 = warp_partials(p, q, vm);
    if ((threadIdx.x & 3) == 0 && q != NPROP - 1) {
        if (fabsf(a1) < PROPS_FIX_MAX) pa.a += __float2ll_rn(a1 * PROPS_FIX);
        else atomicAdd(&A.rs[r].pbig[q], double(a1));   // also NaN, which then shows in the props
    }
    pa.vm = fmaxf(pa.vm, vm);
}

// the warp's sums into replica r (all lanes; each lane fences its atomics)
__device__ __forceinline__ void props_warp_flush(const Arrays& A, int r, PropsAcc& pa)
{
    const int lane = threadIdx.x & 31;
    if ((lane & 3) == 0 && (lane >> 2) < NPROP - 1 && pa.a != 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(&A.rs[r].pacc[lane >> 2]), static_cast<unsigned long long>(pa.a));
    if (lane == 0) atomicMax(&A.rs[r].pvmax2, __float_as_uint(pa.vm));
    __threadfence();
    pa.a = 0;
    pa.vm = 0.0f;
}

// The same with the warp's sums in shared memory (acc[q] for quantity q, vm the maximum; each
// entry touched by one lane only), which keeps them out of the registers of the per-SM step
// kernel, whose pair loop runs at the register bound.
__device__ __forceinline__ void props_warp_add_sh(const Arrays& A, int r, float (&p)[NPROP], long long* acc, float* vm)
{
    int q;
    float m;
    const float a1 = warp_partials(p, q, m);
    if ((threadIdx.x & 3) == 0 && q != NPROP - 1) {
        if (fabsf(a1) < PROPS_FIX_MAX) acc[q] += __float2ll_rn(a1 * PROPS_FIX);
        else atomicAdd(&A.rs[r].pbig[q], double(a1));
    }
    if ((threadIdx.x & 31) == 0) *vm = fmaxf(*vm, m);
}

__device__ __forceinline__ void props_warp_flush_sh(const Arrays& A, int r, long long* acc, float* vm)
{
    const int lane = threadIdx.x & 31;
    if ((lane & 3) == 0 && (lane >> 2) < NPROP - 1) {
        const long long a = acc[lane >> 2];
        if (a != 0) atomicAdd(reinterpret_cast<unsigned long long*>(&A.rs[r].pacc[lane >> 2]), static_cast<unsigned long long>(a));
        acc[lane >> 2] = 0;
    }
    if (lane == 0) {
        atomicMax(&A.rs[r].pvmax2, __float_as_uint(*vm));
        *vm = 0.0f;
    }
    __threadfence();
}

// one warp-tile's props: FP64 lanes (MD_FP64) store the warp's partials for k_props_reduce, FP32
// lanes add them to the warp's fixed-point sums
__device__ __forceinline__ void props_take(const Arrays&, int, double (&p)[NPROP], PropsAcc&, double* dst)
{
    warp_partials_store(p, dst);
}
__device__ __forceinline__ void props_take(const Arrays& A, int r, float (&p)[NPROP], PropsAcc& pa, double*)
{
    props_warp_add(A, r, p, pa);
}

// Refresh criterion and step bookkeeping, run by one thread of the CTA that completed the last
// tile of replica r in this launch.  With props (fixed-point path), first the props of the step.
__device__ void finish_replica_step(const Arrays& A, const Scal& S, int r, cudaGraphConditionalHandle cond,
                                    int use_cond, int props = 0)
{
    RepState& st = A.rs[r];
    if (props) {
        double acc[NPROP];
#pragma unroll
        for (int q = 0; q < NPROP - 1; ++q) {
            acc[q] = double(static_cast<long long>(atomicExch(reinterpret_cast<unsigned long long*>(&st.pacc[q]), 0ull))) *
                         (1.0 / 16777216.0) +
                     __ldcg(&st.pbig[q]);
            st.pbig[q] = 0.0;
        }
        acc[NPROP - 1] = double(__uint_as_float(atomicExch(&st.pvmax2, 0u)));
        write_props(A, S, r, acc, 0, 1);
    }
    st.tiles_done = 0;
    const float m2 = __uint_as_float(atomicExch(&st.vmax2, 0u));
    if (!(m2 <= 3.0e38f)) atomicOr(&A.g->err, ERR_NONFINITE);
    st.step += 1;
    st.vhalf = 1;
    bool rebuild;
    if (S.rule == MD_REBUILD_VMAX) {
        // D bounds every atom's displacement since the last rebuild (triangle inequality):
        // max_i |x_{n+1} - x_n| = dt max_i |v_{n+1/2}|, measured on the FP32 position copies,
        // plus a margin covering their rounding
        st.D += sqrt(double(m2)) * (1.0 + 1e-6) + S.disp_margin;
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

// Fold one CTA's contribution to replica r: the maximum of the refresh metric over its tiles
// and the number of tiles it completed.  The CTA that brings the count to the replica's tile
// total runs the refresh bookkeeping (the last-block pattern).  All threads of the CTA call this.
__device__ __forceinline__ void flush_replica(const Arrays& A, const Scal& S, int r, float run_max, int tiles,
                                              float* sh, cudaGraphConditionalHandle cond, int use_cond,
                                              PropsAcc* pa = nullptr)
{
    if (pa) props_warp_flush(A, r, *pa);
    const float m = tile_max(run_max, sh);
    if (threadIdx.x == 0) {
        atomicMax(&A.rs[r].vmax2, __float_as_uint(m));
        __threadfence();
        const int done = atomicAdd(&A.rs[r].tiles_done, tiles) + tiles;
        if (done == A.rep[r].ntiles) {
            __threadfence();
            finish_replica_step(A, S, r, cond, use_cond, pa ? 1 : 0);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// fused force + leapfrog step
// ------------------------------------------------------------------------------------------
//
// With STG (MD_MIXED, MD_FP32), the positions of each tile's neighbours are staged in shared
// memory first: the tile's slot window per (o_y, o_z) row of W codes (k_tile_windows) is copied
// by cp.async.bulk, as many windows as `stage_cap` positions hold, and the pair loop reads a
// neighbour from shared memory when its slot lies in its row's staged window (which then holds
// exactly that slot's position), else from global memory.  The arithmetic is unchanged.
template <int MODE, bool PROPS, int NB, int MINB, bool STG>
__global__ void __launch_bounds__(TILE, MINB) k_step(Arrays A, Scal S, int cur, cudaGraphConditionalHandle cond,
                                                 int use_cond, int stage_cap)
{
    __shared__ float sh_max[TILE / 32];
    extern __shared__ __align__(16) float4 s_nb[];       // STG: staged neighbour positions
    __shared__ int4 sh_win[16];          // STG: per (o_y+1) + 4 (o_z+1): first slot, length, s_nb offset
    __shared__ uint64_t sh_bar;
    __shared__ int sh_staged;
    uint32_t stg_parity = 0;
    bool stg_timeout = false;
    if (STG) {
        if (threadIdx.x == 0) {
            mbar_init(&sh_bar, 1);
            mbar_fence_init();
        }
        __syncthreads();
    }
    const int nxt = cur ^ 1;
    // Each CTA takes a contiguous run of tiles.  Software pipeline over them: while tile t is
    // computed, tile t+1's state and the rows of W below each atom's count are prefetched into
    // L2 (the counts are read one tile earlier still), so the next tile's HBM traffic is in
    // flight without holding registers.
    const int per = (S.ntiles + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * per;
    const int t_end = min(S.ntiles, t_begin + per);
    int c_ahead = 0;
    if (MODE != MD_FP64 && t_begin + 1 < t_end)
        c_ahead = __ldcs(A.nbr_count + int64_t(t_begin + 1) * TILE + threadIdx.x);
    // the refresh metric is kept per thread across this CTA's tiles of one replica and folded
    // into the replica's counters once per replica (one fence per CTA, not per tile)
    int run_r = -1, run_tiles = 0;
    float run_max = 0.0f;
    PropsAcc pa{0, 0.0f};
    PropsAcc* const pfix = (PROPS && MODE != MD_FP64) ? &pa : nullptr;
    for (int t = t_begin; t < t_end; ++t) {
        if (MODE != MD_FP64) {
            if (t + 1 < t_end) {
                // one prefetch per 128-byte line, spread over the warp's lanes: the warp's 32
                // slots span 4 lines of positions, 2 lines of each FP64 stream (1 of each FP32
                // stream) and 1 line per row of W below the warp's largest count
                const int lane = threadIdx.x & 31;
                const int64_t w1 = int64_t(t + 1) * TILE + (threadIdx.x & ~31);
                const int mw = min(__reduce_max_sync(0xffffffffu, unsigned(c_ahead)), unsigned(S.cap));
                constexpr int NSTATE = (MODE == MD_MIXED) ? 12 : 3;      // lines of the state streams
                const int nref = (S.rule == MD_REBUILD_DISP) ? 4 : 0;     // positions at the last rebuild
                for (int k = lane; k < 4 + NSTATE + nref + mw; k += 32) {
                    const void* p;
                    if (k < 4) {
                        p = A.pos32[cur] + w1 + 8 * k;
                    } else if (k < 4 + NSTATE) {
                        const int q = k - 4;
                        if (MODE == MD_MIXED) p = ((q & 1) ? A.v[q >> 2] : A.xl[q >> 2]) + w1 + 16 * ((q >> 1) & 1);
                        else p = A.v32[q] + w1;
                    } else if (k < 4 + NSTATE + nref) {
                        p = A.xref + w1 + 8 * (k - 4 - NSTATE);
                    } else {
                        p = A.W + int64_t(k - 4 - NSTATE - nref) * S.nslots + w1;
                    }
                    prefetch_l2(p);
                }
            }
            c_ahead = (t + 2 < t_end) ? __ldcs(A.nbr_count + int64_t(t + 2) * TILE + threadIdx.x) : 0;
        }
        {
            const int r_t = A.tile_rep[t];
            if (r_t != run_r) {
                if (run_r >= 0) flush_replica(A, S, run_r, run_max, run_tiles, sh_max, cond, use_cond, pfix);
                run_r = r_t;
                run_tiles = 0;
                run_max = 0.0f;
            }
        }
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const bool active = slot - R.slot0 < R.n;
        const int vhalf = A.rs[r].vhalf;
        if (STG) {
            // every thread is past its reads of the previous tile's staged positions
            __syncthreads();
            if (threadIdx.x == 0) {
                // windows in row order while they fit; a window that does not fit (or is empty)
                // gets length 0 and its neighbours are read from global memory
                const int2* wv = A.tile_win + int64_t(t) * 9;
                int off = 0;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int2 w = wv[q];
                    const int len = w.y - w.x + 1;
                    const bool fit = len > 0 && w.x >= 0 && int64_t(w.y) < S.nslots && off + len <= stage_cap;
                    sh_win[(q % 3) + 4 * (q / 3)] = make_int4(w.x, fit ? len : 0, off, 0);
                    if (fit) off += len;
                }
                if (off > 0) {
                    mbar_arrive_expect_tx(&sh_bar, uint32_t(off) * 16u);
                    const float4* pos = A.pos32[cur];
#pragma unroll 1
                    for (int q = 0; q < 9; ++q) {
                        const int4 w = sh_win[(q % 3) + 4 * (q / 3)];
                        if (w.y > 0) bulk_load(s_nb + w.z, pos + w.x, uint32_t(w.y) * 16u, &sh_bar);
                    }
                }
                sh_staged = off > 0;
            }
            __syncthreads();
            if (sh_staged) {
                if (!stg_timeout && !mbar_wait_bounded(&sh_bar, stg_parity)) stg_timeout = true;
                stg_parity ^= 1u;
            }
        }
        float metric = 0.0f;                     // |v|^2 (VMAX) or |x - x_ref|^2 (DISP)
        using PT = typename std::conditional<MODE == MD_FP64, double, float>::type;
        PT part[NPROP];
#pragma unroll
        for (int q = 0; q < NPROP; ++q) part[q] = PT(0);
        if (active) {
            if constexpr (MODE == MD_FP64) {
                const double4_32a* pos = A.pos64[cur];
                const double4_32a pi = pos[slot];
                const AccD a = force_f64(A, S, R, pos, slot, pi);
                const double f[3] = {a.fx, a.fy, a.fz};
                double xl[3] = {pi.x, pi.y, pi.z};
                const double kick = vhalf ? 2.0 * S.c : S.c;
                double vn2 = 0.0;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    double v = A.v[q][slot];
                    if (PROPS) {
                        const double vn = vhalf ? fma(S.c, f[q], v) : v;
                        vn2 = fma(vn, vn, vn2);
                        part[3 + q] = vn;
                    }
                    v = fma(kick, f[q], v);
                    xl[q] = fma(S.dt, v, xl[q]);
                    A.v[q][slot] = v;
                    A.xl[q][slot] = xl[q];
                }
                A.pos64[nxt][slot] = make_double4_32a(xl[0], xl[1], xl[2], pi.w);
                if (S.rule == MD_REBUILD_DISP) {
                    const float4 xr = A.xref[slot];
                    const float d0 = float(xl[0] - double(xr.x)), d1 = float(xl[1] - double(xr.y)),
                                d2 = float(xl[2] - double(xr.z));
                    metric = d0 * d0 + d1 * d1 + d2 * d2;
                } else {
                    const double d0 = xl[0] - pi.x, d1 = xl[1] - pi.y, d2 = xl[2] - pi.z;
                    metric = float(d0 * d0 + d1 * d1 + d2 * d2);
                }
                if (PROPS) {
                    part[0] = a.u;
                    part[1] = vn2;
                    part[2] = a.w;
                    part[NPROP - 1] = vn2;
                }
            } else {
                const float4* pos = A.pos32[cur];
                const float4 pi = __ldg(pos + slot);
                if (t == t_begin) {                      // first tile of this CTA: nothing prefetched yet
                    if (MODE == MD_MIXED) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) { prefetch_l2(A.v[q] + slot); prefetch_l2(A.xl[q] + slot); }
                    } else {
#pragma unroll
                        for (int q = 0; q < 3; ++q) prefetch_l2(A.v32[q] + slot);
                    }
                }
                AccF a;
                if (STG) {
                    // a neighbour inside its row's staged window is read from shared memory (the
                    // window holds exactly those slots); any other from global memory
                    const bool use_smem = !stg_timeout;
                    const int mm = min(__ldcs(A.nbr_count + slot), S.cap);
                    const uint32_t* __restrict__ Wc = A.W + slot;
                    const int64_t ns = S.nslots;
                    a = pair_loop_f32<NB>(
                        S, R, pi, mm, [=](int m) { return __ldcs(Wc + int64_t(m) * ns); },
                        [=](uint32_t e) {
                            const int j = int(e >> IDX_SHIFT);
                            const int4 w = sh_win[(e >> 2) & 15u];
                            const uint32_t d = uint32_t(j - w.x);
                            const bool in = use_smem && d < uint32_t(w.y);
                            const int si = in ? w.z + int(d) : 0;      // inside the staged range either way
                            float4 r;
                            if (in) r = s_nb[si];
                            else r = __ldg(pos + j);
                            return r;
                        });
                } else {
                    a = force_f32<NB>(A, S, R, pos, slot, pi);
                }
                if (S.chain_len) add_buffer(A, slot, a);
                double v[3], x[3];
                float v32[3], pn[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (MODE == MD_MIXED) {
                        v[q] = __ldcs(A.v[q] + slot);
                        x[q] = __ldcs(A.xl[q] + slot);
                    } else {
                        v32[q] = A.v32[q][slot];
                    }
                }
                metric = kick_drift<MODE, PROPS>(S, vhalf, pi, a, v, x, v32, pn, part);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (MODE == MD_MIXED) {
                        __stcs(A.v[q] + slot, v[q]);
                        __stcs(A.xl[q] + slot, x[q]);
                    } else {
                        A.v32[q][slot] = v32[q];
                    }
                }
                A.pos32[nxt][slot] = make_float4(pn[0], pn[1], pn[2], pi.w);
                if (S.rule == MD_REBUILD_DISP) {
                    const float4 xr = A.xref[slot];
                    const float d0 = pn[0] - xr.x, d1 = pn[1] - xr.y, d2 = pn[2] - xr.z;
                    metric = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
                }
            }
            if (!(metric <= 3.0e38f)) metric = __uint_as_float(0x7f800000u);   // +inf marks non-finite
        }
        run_max = fmaxf(run_max, metric);
        run_tiles += 1;
        if (PROPS) props_take(A, run_r, part, pa, warp_slot(A, int64_t(t) * (TILE / 32) + (threadIdx.x >> 5)));
    }
    if (run_r >= 0) flush_replica(A, S, run_r, run_max, run_tiles, sh_max, cond, use_cond, pfix);
    if (STG && stg_timeout) atomicOr(&A.g->err, ERR_TIMEOUT);
}

// ------------------------------------------------------------------------------------------
// fused force + leapfrog step on a per-SM schedule (MD_MIXED, MD_FP32)
// ------------------------------------------------------------------------------------------
// The slots are cut into SM_RANGES-bounded contiguous ranges, one per SM id, and each warp takes
// 32-slot warp-tiles from the range of the SM it runs on (an atomic counter per range), in
// order.  All warps of an SM therefore compute neighbouring atoms at the same time, and since
// slots are in cell order with the rows of cells blocked in z (row_pos), their neighbour
// gathers share one compact region in the SM's L1 instead of one region per CTA.  A warp whose
// range is exhausted takes warp-tiles from any range with some left, so every warp-tile is
// computed exactly once whatever the placement of the CTAs.  The last warp to finish resets the
// counters for the next step.  Per atom the arithmetic is k_step's, bit for bit, and so are the
// props: the fixed-point sums do not depend on which warp took which warp-tile.
__device__ __forceinline__ int ld_relaxed_gpu(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Fold one warp's contribution to replica r (k_step's flush_replica for a warp): the maximum of
// the refresh metric and the number of warp-tiles; the warp that completes the replica's
// warp-tiles runs the refresh bookkeeping.
__device__ __forceinline__ void flush_replica_warp(const Arrays& A, const Scal& S, int r, float run_max, int wtiles,
                                                   cudaGraphConditionalHandle cond, int use_cond,
                                                   long long* pacc = nullptr, float* pvm = nullptr)
{
    if (pacc) {
        props_warp_flush_sh(A, r, pacc, pvm);
        __syncwarp();
    }
    const float m = warp_max(run_max);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&A.rs[r].vmax2, __float_as_uint(m));
        __threadfence();
        const int done = atomicAdd(&A.rs[r].tiles_done, wtiles) + wtiles;
        if (done == A.rep[r].ntiles * (TILE / 32)) {
            __threadfence();
            finish_replica_step(A, S, r, cond, use_cond, pacc ? 1 : 0);
        }
    }
    __syncwarp();
}

// SRC: where the forces come from -- 0 the neighbour matrix W, 1 the 27 cells (step kernel 4),
// 2 the half-list buffers filled by k_half_pairs (step kernel 5; read and cleared here)
template <int MODE, bool PROPS, int NB, int MINB, int SRC = 0>
__global__ void __launch_bounds__(TILE, MINB) k_step_sm(Arrays A, Scal S, int cur, cudaGraphConditionalHandle cond,
                                                      int use_cond)
{
    static_assert(MODE != MD_FP64, "MD_FP64 steps run k_step");
    const int nxt = cur ^ 1;
    const int lane = threadIdx.x & 31;
    uint32_t smid, nsmid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
    const int nr = max(1, min(int(nsmid), SM_RANGES));
    const int home = int(smid) % nr;
    const int nwt = S.ntiles * (TILE / 32);
    const int per = (nwt + nr - 1) / nr;
    int* const claimc = A.sm_claim;
    const float4* __restrict__ pos = A.pos32[cur];
    auto range_len = [&](int q) { return max(0, min(nwt - q * per, per)); };

    bool home_open = true;
    // a warp-tile of any range with some left, or -1 when all are done.  Every failed claim
    // leaves its range exhausted for the rest of the launch, so nr + 1 scans always suffice.
    auto steal = [&]() -> int {
        for (int iter = 0; iter <= nr + 1; ++iter) {
            int sel = -1;
            for (int i = 0; i * 32 < nr && sel < 0; ++i) {
                const int q = i * 32 + lane;
                const int rr = (home + 1 + q) % nr;
                const bool avail = q < nr && ld_relaxed_gpu(claimc + rr) < range_len(rr);
                const unsigned b = __ballot_sync(0xffffffffu, avail);
                if (b) sel = (home + 1 + i * 32 + __ffs(b) - 1) % nr;
            }
            if (sel < 0) return -1;
            int k = 0;
            if (lane == 0) k = atomicAdd(claimc + sel, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k < range_len(sel)) return sel * per + k;
        }
        if (lane == 0) atomicOr(&A.g->err, ERR_TIMEOUT);     // unreachable: the scan is bounded
        return -1;
    };
    auto claim_now = [&]() -> int {
        if (home_open) {
            int k = 0;
            if (lane == 0) k = atomicAdd(claimc + home, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k < range_len(home)) return home * per + k;
            home_open = false;
        }
        return steal();
    };

    // w0 is computed while w1, the next warp-tile, has its positions and state prefetched into
    // L2 and the claim of the one after it is in flight
    int w0 = claim_now();
    int w1 = (w0 >= 0) ? claim_now() : -1;
    int c0 = (w0 >= 0 && SRC == 0) ? __ldcs(A.nbr_count + int64_t(w0) * 32 + lane) : 0;   // w0's counts
    int run_r = -1, run_cnt = 0;
    float run_max = 0.0f;
    __shared__ long long s_pacc[TILE / 32][8];
    __shared__ float s_pvm[TILE / 32];
    long long* const pacc = PROPS ? s_pacc[threadIdx.x >> 5] : nullptr;
    float* const pvm = PROPS ? &s_pvm[threadIdx.x >> 5] : nullptr;
    if (PROPS) {
        if (lane < 8) pacc[lane] = 0;
        if (lane == 0) *pvm = 0.0f;
        __syncwarp();
    }
    while (w0 >= 0) {
        int pend = 0;
        const bool pending = home_open && w1 >= 0;
        if (pending && lane == 0) pend = atomicAdd(claimc + home, 1);
        int c1 = 0;
        if (w1 >= 0) {
            // one prefetch per 128-byte line: 4 lines of positions, 2 of each FP64 stream (1 of
            // each FP32 stream), 4 of positions at the last rebuild (rule DISP)
            const int64_t s1 = int64_t(w1) * 32;
            constexpr int NSTATE = (MODE == MD_MIXED) ? 12 : 3;
            const int nref = (S.rule == MD_REBUILD_DISP) ? 4 : 0;
            if (lane < 4 + NSTATE + nref) {
                const void* p;
                if (lane < 4) {
                    p = A.pos32[cur] + s1 + 8 * lane;
                } else if (lane < 4 + NSTATE) {
                    const int q = lane - 4;
                    if (MODE == MD_MIXED) p = ((q & 1) ? A.v[q >> 2] : A.xl[q >> 2]) + s1 + 16 * ((q >> 1) & 1);
                    else p = A.v32[q] + s1;
                } else {
                    p = A.xref + s1 + 8 * (lane - 4 - NSTATE);
                }
                prefetch_l2(p);
            }
            if (SRC == 0) c1 = __ldcs(A.nbr_count + s1 + lane);
        }
        const int t = w0 / (TILE / 32);
        const int r = A.tile_rep[t];
        if (r != run_r) {
            if (run_r >= 0) flush_replica_warp(A, S, run_r, run_max, run_cnt, cond, use_cond, pacc, pvm);
            run_r = r;
            run_cnt = 0;
            run_max = 0.0f;
        }
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(w0) * 32 + lane;
        const bool active = slot - R.slot0 < R.n;
        const int vhalf = A.rs[r].vhalf;
        float metric = 0.0f;                     // |v|^2 (VMAX) or |x - x_ref|^2 (DISP)
        float part[NPROP];
#pragma unroll
        for (int q = 0; q < NPROP; ++q) part[q] = 0.0f;
        if (active) {
            const float4 pi = __ldg(pos + slot);
            AccF a;
            if (SRC == 1) {
                a = force_f32_cells(A, S, R, pos, slot, pi);
            } else if (SRC == 2) {
                const float4 fb = __ldcs(A.fbuf + slot);
                a = AccF{fb.x, fb.y, fb.z, fb.w, __ldcs(A.wbuf + slot)};
                A.fbuf[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
                A.wbuf[slot] = 0.f;
            } else {
                a = force_f32_rows<NB>(A, S, R, pos, slot, pi, min(c0, S.cap));
            }
            if (S.chain_len && SRC != 2) add_buffer(A, slot, a);
            double v[3], x[3];
            float v32[3], pn[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (MODE == MD_MIXED) {
                    v[q] = __ldcs(A.v[q] + slot);
                    x[q] = __ldcs(A.xl[q] + slot);
                } else {
                    v32[q] = A.v32[q][slot];
                }
            }
            metric = kick_drift<MODE, PROPS>(S, vhalf, pi, a, v, x, v32, pn, part);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (MODE == MD_MIXED) {
                    __stcs(A.v[q] + slot, v[q]);
                    __stcs(A.xl[q] + slot, x[q]);
                } else {
                    A.v32[q][slot] = v32[q];
                }
            }
            A.pos32[nxt][slot] = make_float4(pn[0], pn[1], pn[2], pi.w);
            if (S.rule == MD_REBUILD_DISP) {
                const float4 xr = A.xref[slot];
                const float d0 = pn[0] - xr.x, d1 = pn[1] - xr.y, d2 = pn[2] - xr.z;
                metric = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
            }
            if (!(metric <= 3.0e38f)) metric = __uint_as_float(0x7f800000u);   // +inf marks non-finite
        }
        run_max = fmaxf(run_max, metric);
        run_cnt += 1;
        if (PROPS) props_warp_add_sh(A, r, part, pacc, pvm);
        int w2 = -1;
        if (w1 >= 0) {
            // the rows of W below the next warp-tile's largest count into L2
            const int mw = min(__reduce_max_sync(0xffffffffu, unsigned(c1)), unsigned(S.cap));
            if (SRC == 0)
                for (int k = lane; k < mw; k += 32) prefetch_l2(A.W + int64_t(k) * S.nslots + int64_t(w1) * 32);
            if (pending) {
                const int k = __shfl_sync(0xffffffffu, pend, 0);
                if (k < range_len(home)) w2 = home * per + k;
                else home_open = false;
            }
            if (w2 < 0 && !home_open) w2 = steal();
        }
        w0 = w1;
        w1 = w2;
        c0 = c1;                                 // read one warp-tile ahead
    }
    if (run_r >= 0) flush_replica_warp(A, S, run_r, run_max, run_cnt, cond, use_cond, pacc, pvm);
    // the last warp of the launch resets the counters; the next launch is ordered after this one
    if (lane == 0) {
        __threadfence();
        const int total = int(gridDim.x) * (TILE / 32);
        if (atomicAdd(claimc + SM_RANGES, 1) == total - 1) {
            for (int q = 0; q < nr; ++q) claimc[q] = 0;
            claimc[SM_RANGES] = 0;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------------------------------
// fused force + leapfrog step through a shared-memory ring (MD_MIXED, MD_FP32)
// ------------------------------------------------------------------------------------------
// Each CTA takes a contiguous run of tiles and keeps two of them in a two-stage ring in shared
// memory.  One thread issues a tile's cp.async.bulk copies (positions, velocity and position
// streams, neighbour counts, and the rows of W below the tile's largest count, up to `rows`);
// they complete on the stage's mbarrier.  The CTA waits on it, runs the same pair loop and
// kick-drift as k_step with W and the state read from shared memory (only the neighbour
// positions are gathered from global memory, through L1), and releases the stage, into which the
// copies of the tile two ahead then go.  The HBM reads of the next tile are in flight while the
// current one computes, without registers held for them.
template <int MODE, bool PROPS, int NB>
__global__ void __launch_bounds__(TILE, 2) k_step_bulk(Arrays A, Scal S, int cur, int rows,
                                                       cudaGraphConditionalHandle cond, int use_cond)
{
    extern __shared__ __align__(128) unsigned char ring[];
    __shared__ uint64_t bar[2];
    __shared__ float sh_max[TILE / 32];
    __shared__ int sh_mm[2][TILE / 32];
    const StageLayout SL = stage_layout(MODE, rows);
    const int nxt = cur ^ 1;
    const int per = (S.ntiles + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * per;
    const int t_end = min(S.ntiles, t_begin + per);
    if (t_begin >= t_end) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4* __restrict__ pos = A.pos32[cur];

    // the copies of tile t into stage st (thread 0); mmax = the tile's largest neighbour count
    auto issue = [&](int t, int st, int mmax) {
        unsigned char* sb = ring + size_t(st) * SL.bytes;
        const int64_t s0 = int64_t(t) * TILE;
        const int nr = min(min(mmax, S.cap), rows);
        const uint32_t state = (MODE == MD_MIXED) ? 6u * TILE * 8u : 3u * TILE * 4u;
        mbar_arrive_expect_tx(&bar[st], TILE * 16u + state + TILE * 4u + uint32_t(nr) * TILE * 4u);
        bulk_load(sb + SL.pos, pos + s0, TILE * 16u, &bar[st]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (MODE == MD_MIXED) {
                bulk_load(sb + SL.xl + q * TILE * 8, A.xl[q] + s0, TILE * 8u, &bar[st]);
                bulk_load(sb + SL.v + q * TILE * 8, A.v[q] + s0, TILE * 8u, &bar[st]);
            } else {
                bulk_load(sb + SL.v + q * TILE * 4, A.v32[q] + s0, TILE * 4u, &bar[st]);
            }
        }
        bulk_load(sb + SL.cnt, A.nbr_count + s0, TILE * 4u, &bar[st]);
        for (int m = 0; m < nr; ++m)
            bulk_load(sb + SL.w + uint32_t(m) * TILE * 4u, A.W + int64_t(m) * S.nslots + s0, TILE * 4u, &bar[st]);
    };
    auto block_mmax = [&](int st) {
        int m = sh_mm[st][0];
#pragma unroll
        for (int k = 1; k < TILE / 32; ++k) m = max(m, sh_mm[st][k]);
        return m;
    };

    // prologue: barriers, then the first two tiles
    {
        const int c0 = __ldcs(A.nbr_count + int64_t(t_begin) * TILE + threadIdx.x);
        const int c1 = (t_begin + 1 < t_end) ? __ldcs(A.nbr_count + int64_t(t_begin + 1) * TILE + threadIdx.x) : 0;
        const int m0 = warp_max_i(c0), m1 = warp_max_i(c1);
        if (lane == 0) {
            sh_mm[0][warp] = m0;
            sh_mm[1][warp] = m1;
        }
        if (threadIdx.x == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            mbar_fence_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            issue(t_begin, 0, block_mmax(0));
            if (t_begin + 1 < t_end) issue(t_begin + 1, 1, block_mmax(1));
        }
    }
    uint32_t parity = 0;                          // bit st: parity of stage st's next phase
    bool timed_out = false;
    int run_r = -1, run_tiles = 0;
    float run_max = 0.0f;
    PropsAcc pa{0, 0.0f};
    PropsAcc* const pfix = PROPS ? &pa : nullptr;
    for (int t = t_begin; t < t_end; ++t) {
        const int st = (t - t_begin) & 1;
        const int c2 = (t + 2 < t_end) ? __ldcs(A.nbr_count + int64_t(t + 2) * TILE + threadIdx.x) : 0;
        {
            const int r_t = A.tile_rep[t];
            if (r_t != run_r) {
                if (run_r >= 0) flush_replica(A, S, run_r, run_max, run_tiles, sh_max, cond, use_cond, pfix);
                run_r = r_t;
                run_tiles = 0;
                run_max = 0.0f;
            }
        }
        const int r = A.tile_rep[t];
        const Rep& R = A.rep[r];
        const int64_t slot = int64_t(t) * TILE + threadIdx.x;
        const bool active = slot - R.slot0 < R.n;
        const int vhalf = A.rs[r].vhalf;
        // after a wait that gave up the stage holds no valid data: this thread stops computing
        // and waiting (its W entries would index garbage), and the error is latched at exit
        if (!timed_out && !mbar_wait_bounded(&bar[st], (parity >> st) & 1u)) timed_out = true;
        parity ^= 1u << st;
        const unsigned char* sb = ring + size_t(st) * SL.bytes;
        float metric = 0.0f;
        float part[NPROP];
#pragma unroll
        for (int q = 0; q < NPROP; ++q) part[q] = 0.0f;
        if (active && !timed_out) {
            const float4 pi = reinterpret_cast<const float4*>(sb + SL.pos)[threadIdx.x];
            const int mm = min(reinterpret_cast<const int32_t*>(sb + SL.cnt)[threadIdx.x], S.cap);
            const uint32_t* sw = reinterpret_cast<const uint32_t*>(sb + SL.w) + threadIdx.x;
            const uint32_t* __restrict__ gw = A.W + slot;
            const int64_t ns = S.nslots;
            AccF a = pair_loop_f32<NB>(
                S, R, pi, mm, [=](int m) { return (m < rows) ? sw[m * TILE] : __ldcs(gw + int64_t(m) * ns); },
                [=](uint32_t e) { return __ldg(pos + (e >> IDX_SHIFT)); });
            if (S.chain_len) add_buffer(A, slot, a);
            double v[3], x[3];
            float v32[3], pn[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (MODE == MD_MIXED) {
                    v[q] = reinterpret_cast<const double*>(sb + SL.v)[q * TILE + threadIdx.x];
                    x[q] = reinterpret_cast<const double*>(sb + SL.xl)[q * TILE + threadIdx.x];
                } else {
                    v32[q] = reinterpret_cast<const float*>(sb + SL.v)[q * TILE + threadIdx.x];
                }
            }
            metric = kick_drift<MODE, PROPS>(S, vhalf, pi, a, v, x, v32, pn, part);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (MODE == MD_MIXED) {
                    __stcs(A.v[q] + slot, v[q]);
                    __stcs(A.xl[q] + slot, x[q]);
                } else {
                    __stcs(A.v32[q] + slot, v32[q]);
                }
            }
            A.pos32[nxt][slot] = make_float4(pn[0], pn[1], pn[2], pi.w);
            if (S.rule == MD_REBUILD_DISP) {
                const float4 xr = A.xref[slot];
                const float d0 = pn[0] - xr.x, d1 = pn[1] - xr.y, d2 = pn[2] - xr.z;
                metric = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
            }
            if (!(metric <= 3.0e38f)) metric = __uint_as_float(0x7f800000u);   // +inf marks non-finite
        }
        run_max = fmaxf(run_max, metric);
        run_tiles += 1;
        if (PROPS) props_warp_add(A, run_r, part, pa);
        // release the stage (every thread is past its reads of it), then refill it with tile t+2
        const int wm = warp_max_i(c2);
        if (lane == 0) sh_mm[st][warp] = wm;
        __syncthreads();
        if (threadIdx.x == 0 && t + 2 < t_end && !timed_out) issue(t + 2, st, block_mmax(st));
    }
    if (run_r >= 0) flush_replica(A, S, run_r, run_max, run_tiles, sh_max, cond, use_cond, pfix);
    if (timed_out) atomicOr(&A.g->err, ERR_TIMEOUT);
}

// ------------------------------------------------------------------------------------------
// forces only (F1): f, u_i, per-atom virial
// ------------------------------------------------------------------------------------------
template <int MODE, bool CELLS = false>
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
            AccF a = CELLS ? force_f32_cells(A, S, R, A.pos32[cur], slot, pi)
                           : force_f32<4>(A, S, R, A.pos32[cur], slot, pi);
            if (S.chain_len) add_buffer(A, slot, a);
            A.f[slot] = make_double4_32a(a.fx, a.fy, a.fz, a.u);
            A.wvir[slot] = a.w;
        }
    }
}

// per-tile FP64 partials from stored forces and the state's velocities (closed to step n)
template <int MODE>
__global__ void __launch_bounds__(TILE) k_props_tiles(Arrays A, Scal S)
{
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
                part[3 + q] = vn;
            }
            part[0] = f.w;
            part[1] = vn2;
            part[2] = A.wvir[slot];
            part[NPROP - 1] = vn2;
        }
        warp_partials_store(part, warp_slot(A, int64_t(t) * (TILE / 32) + (threadIdx.x >> 5)));
    }
}

// Final sums, in a fixed order, in one launch: S.props_split CTAs per replica each add a
// contiguous slice of the replica's warp partials (thread t the rows t, t + 128, ...; then a
// tree over the threads in shared memory), store the slice's sums, and count themselves in; the
// CTA that completes the replica (the last-block pattern of Sec. 2.3's reductions: a fence,
// then an atomic counter) adds the slices the same way and writes the props, applying the
// constant factors (U = sum u_i / 2, K = m sum v^2 / 2, W = sum w_i / 2, P = m sum v), and the
// time-series row.
constexpr int PROPS_THREADS = 128;

__device__ __forceinline__ void props_tree(double (*sh)[NPROP], double (&acc)[NPROP])
{
#pragma unroll
    for (int q = 0; q < NPROP; ++q) sh[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int h = PROPS_THREADS / 2; h > 0; h >>= 1) {
        if (int(threadIdx.x) < h) {
#pragma unroll
            for (int q = 0; q < NPROP - 1; ++q) sh[threadIdx.x][q] += sh[threadIdx.x + h][q];
            sh[threadIdx.x][NPROP - 1] = fmax(sh[threadIdx.x][NPROP - 1], sh[threadIdx.x + h][NPROP - 1]);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(PROPS_THREADS) k_props_reduce(Arrays A, Scal S, int to_series, int step_lag)
{
    __shared__ double sh[PROPS_THREADS][NPROP];
    __shared__ int sh_last;
    const int split = S.props_split;
    const int r = blockIdx.x / split, b = blockIdx.x % split;
    const Rep& R = A.rep[r];
    const int64_t rows = int64_t(R.ntiles) * (TILE / 32);            // warp partials of the replica
    const int64_t per = (rows + split - 1) / split;
    const int64_t w0 = int64_t(R.tile0) * (TILE / 32) + b * per;
    const int64_t w1 = int64_t(R.tile0) * (TILE / 32) + min(rows, (b + 1) * per);
    double acc[NPROP];
#pragma unroll
    for (int q = 0; q < NPROP; ++q) acc[q] = 0.0;
    for (int64_t w = w0 + threadIdx.x; w < w1; w += PROPS_THREADS) {
        const double* p = A.warp_part + w * NPROP;
#pragma unroll
        for (int q = 0; q < NPROP - 1; ++q) acc[q] += p[q];
        acc[NPROP - 1] = fmax(acc[NPROP - 1], p[NPROP - 1]);
    }
    props_tree(sh, acc);
    if (threadIdx.x < NPROP) A.slice_part[int64_t(blockIdx.x) * NPROP + threadIdx.x] = sh[0][threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(&A.rs[r].props_done, 1) == split - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NPROP; ++q) acc[q] = 0.0;
    for (int k = threadIdx.x; k < split; k += PROPS_THREADS) {
        const double* p = A.slice_part + (int64_t(r) * split + k) * NPROP;
#pragma unroll
        for (int q = 0; q < NPROP - 1; ++q) acc[q] += __ldcg(p + q);
        acc[NPROP - 1] = fmax(acc[NPROP - 1], __ldcg(p + NPROP - 1));
    }
    __syncthreads();
    props_tree(sh, acc);
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int q = 0; q < NPROP; ++q) acc[q] = sh[0][q];
    A.rs[r].props_done = 0;                          // ready for the next reduction
    write_props(A, S, r, acc, step_lag, to_series);
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
            st.step = 0; st.rebuilds = 0; st.last_reorder = 0; st.sum_nbrs = 0; st.reorders = 0;
            st.props_done = 0; st.pvmax2 = 0u;
            for (int q = 0; q < NPROP - 1; ++q) { st.pacc[q] = 0; st.pbig[q] = 0.0; }
        }
        if (j >= R.n) continue;
        const int64_t id = R.id0 + j;
        A.id[slot] = int32_t(id);
        A.slot_of_id[id] = int32_t(slot);
        for (int a = 0; a < 3; ++a) {
            A.xl[a][slot] = A.xchg[0][id * 3 + a];     // global position, origin cell (0,0,0)
            double v = A.xchg[1][id * 3 + a];
            if (!isfinite(v)) {                        // reported by the call; the atom is held still
                atomicOr(&A.g->err, ERR_NONFINITE);
                v = 0.0;
            }
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
        int cx, cy, cz;
        cell_coords(R, A.cell[slot] - R.cell0, cx, cy, cz);
        out[A.id[slot]] = (cz * R.nc[1] + cy) * R.nc[0] + cx;
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
            nbrs[(id - id_lo) * cap_out + k] = A.id[e >> IDX_SHIFT];
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

template <int M, int NB, int MINB, bool STG = false>
static int occ_of(int dyn_smem = 0)
{
    int a = 0, b = 0;
    if constexpr (M != MD_FP64 && !STG) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_step_sm<M, false, NB, MINB>, TILE, dyn_smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_sm<M, true, NB, MINB>, TILE, dyn_smem);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_step<M, false, NB, MINB, STG>, TILE, dyn_smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step<M, true, NB, MINB, STG>, TILE, dyn_smem);
    }
    return std::max(1, std::min(a, b));
}

// register bound from the requested residency: __launch_bounds__(TILE, MINB)
static int minb_of(int ctas_per_sm)
{
    return ctas_per_sm >= 16 ? 16 : ctas_per_sm >= 12 ? 12 : ctas_per_sm >= 8 ? 8 : 4;
}

#define GBMD_DISPATCH_NB_MINB(M, FN)                                                      \
    {                                                                                     \
        const int mb = minb_of(L.ctas_req);                                               \
        const int nb = L.nbr_batch >= 8 ? 8 : L.nbr_batch >= 4 ? 4 : 2;                    \
        if (nb == 8) {                                                                    \
            if (mb == 16) FN(M, 8, 16) else if (mb == 12) FN(M, 8, 12) else if (mb == 8) FN(M, 8, 8) else FN(M, 8, 4) \
        } else if (nb == 4) {                                                             \
            if (mb == 16) FN(M, 4, 16) else if (mb == 12) FN(M, 4, 12) else if (mb == 8) FN(M, 4, 8) else FN(M, 4, 4) \
        } else {                                                                          \
            if (mb == 16) FN(M, 2, 16) else if (mb == 12) FN(M, 2, 12) else if (mb == 8) FN(M, 2, 8) else FN(M, 2, 4) \
        }                                                                                 \
    }

// The dynamic shared-memory limit is a per-function setting: it is raised to the device's opt-in
// maximum less the function's static shared memory, so systems with different ring sizes can
// share the kernels.
template <class K>
static void raise_dyn_smem(K kernel)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(fa.sharedSizeBytes));
}

template <int M, int NB>
static int occ_bulk(int smem)
{
    int a = 0, b = 0;
    raise_dyn_smem(k_step_bulk<M, false, NB>);
    raise_dyn_smem(k_step_bulk<M, true, NB>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_step_bulk<M, false, NB>, TILE, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_bulk<M, true, NB>, TILE, smem);
    return std::max(1, std::min(a, b));
}

#define GBMD_DISPATCH_NB(M, FN)                                                           \
    {                                                                                     \
        const int nb = L.nbr_batch >= 8 ? 8 : L.nbr_batch >= 4 ? 4 : 2;                    \
        if (nb == 8) FN(M, 8) else if (nb == 4) FN(M, 4) else FN(M, 2)                    \
    }

void bulk_shape(const Scal& S, int ctas_per_sm, int smem_per_sm, int smem_per_cta, int* rows, int* smem_bytes)
{
    // per CTA: the ring, its static shared memory (under 1 KB) and the 1 KB the runtime reserves
    const int per_cta = std::min(smem_per_sm / std::max(1, ctas_per_sm) - 2048, smem_per_cta - 1024);
    const int state = int(stage_layout(S.mode, 0).bytes);
    int nr = (per_cta / 2 - state) / int(TILE * 4);
    nr = std::max(1, std::min(nr, S.cap));
    *rows = nr;
    *smem_bytes = 2 * int(stage_layout(S.mode, nr).bytes);
}

template <int M, int NB, int MINB>
static int occ_staged(int dyn_smem)
{
    raise_dyn_smem(k_step<M, false, NB, MINB, true>);
    raise_dyn_smem(k_step<M, true, NB, MINB, true>);
    return occ_of<M, NB, MINB, true>(dyn_smem);
}

void stage_shape(int ctas_per_sm, int smem_per_sm, int* cap, int* smem_bytes)
{
    // per CTA: the staged positions, the kernel's static shared memory and the runtime's 1 KB
    const int per_cta = smem_per_sm / std::max(1, ctas_per_sm) - 2048;
    const int c = std::max(256, std::min(per_cta / 16, 8192));
    *cap = c;
    *smem_bytes = c * 16;
}

template <int M, int MINB, int SRC>
static int occ_src()
{
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_step_sm<M, false, 2, MINB, SRC>, TILE, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_sm<M, true, 2, MINB, SRC>, TILE, 0);
    return std::max(1, std::min(a, b));
}

template <int M, int SRC>
static int occ_src_mb(int mb)
{
    return mb == 16 ? occ_src<M, 16, SRC>() : mb == 12 ? occ_src<M, 12, SRC>() : mb == 8 ? occ_src<M, 8, SRC>()
                                                                                       : occ_src<M, 4, SRC>();
}

int step_ctas_per_sm(const Scal& S, const Launch& L)
{
    int occ = 1;
    if (S.mode == MD_FP64) return occ_of<MD_FP64, 2, 4>();
    if (L.step_kernel == 4 || L.step_kernel == 5) {
        const int mb = minb_of(L.ctas_req);
        if (L.step_kernel == 4) return S.mode == MD_MIXED ? occ_src_mb<MD_MIXED, 1>(mb) : occ_src_mb<MD_FP32, 1>(mb);
        return S.mode == MD_MIXED ? occ_src_mb<MD_MIXED, 2>(mb) : occ_src_mb<MD_FP32, 2>(mb);
    }
    if (L.step_kernel == 3) {
#define GBMD_OCC(M, NB, MB) { occ = occ_staged<M, NB, MB>(L.stage_smem); }
        if (S.mode == MD_MIXED) GBMD_DISPATCH_NB_MINB(MD_MIXED, GBMD_OCC)
        else GBMD_DISPATCH_NB_MINB(MD_FP32, GBMD_OCC)
#undef GBMD_OCC
        return occ;
    }
    if (L.step_kernel == 2) {
#define GBMD_OCC(M, NB) { occ = occ_bulk<M, NB>(L.bulk_smem); }
        if (S.mode == MD_MIXED) GBMD_DISPATCH_NB(MD_MIXED, GBMD_OCC)
        else GBMD_DISPATCH_NB(MD_FP32, GBMD_OCC)
#undef GBMD_OCC
        return occ;
    }
#define GBMD_OCC(M, NB, MB) { occ = occ_of<M, NB, MB>(); }
    if (S.mode == MD_MIXED) GBMD_DISPATCH_NB_MINB(MD_MIXED, GBMD_OCC)
    else GBMD_DISPATCH_NB_MINB(MD_FP32, GBMD_OCC)
#undef GBMD_OCC
    return occ;
}

cudaError_t launch_step(const Arrays& A, const Scal& S, const Launch& L, int cur, bool props)
{
    const int g = std::max(1, std::min(L.grid_step, S.ntiles));
    if (S.chain_len && S.mode != MD_FP64)
        k_chain_terms<<<std::max(1, std::min(L.grid, S.ntiles)), TILE, 0, L.stream>>>(A, S, cur);
    if (S.mode != MD_FP64 && L.step_kernel == 2) {
#define GBMD_STEP_BULK(M, NB)                                                                               \
    {                                                                                                       \
        if (props) k_step_bulk<M, true, NB><<<g, TILE, L.bulk_smem, L.stream>>>(A, S, cur, L.bulk_rows, L.cond, L.use_cond); \
        else k_step_bulk<M, false, NB><<<g, TILE, L.bulk_smem, L.stream>>>(A, S, cur, L.bulk_rows, L.cond, L.use_cond);     \
    }
        if (S.mode == MD_MIXED) GBMD_DISPATCH_NB(MD_MIXED, GBMD_STEP_BULK)
        else GBMD_DISPATCH_NB(MD_FP32, GBMD_STEP_BULK)
#undef GBMD_STEP_BULK
    } else if (S.mode != MD_FP64 && (L.step_kernel == 4 || L.step_kernel == 5)) {
        if (L.step_kernel == 5) {
            // the half-list pairs into the buffers, then the step reads them
            const int gp = std::max(1, std::min(L.grid, S.ntiles));
            if (L.nbr_batch >= 4) k_half_pairs<4><<<gp, TILE, 0, L.stream>>>(A, S, cur);
            else k_half_pairs<2><<<gp, TILE, 0, L.stream>>>(A, S, cur);
        }
#define GBMD_STEP_SRC(M, MB, SRC)                                                                           \
    {                                                                                                       \
        if (props) k_step_sm<M, true, 2, MB, SRC><<<g, TILE, 0, L.stream>>>(A, S, cur, L.cond, L.use_cond);    \
        else k_step_sm<M, false, 2, MB, SRC><<<g, TILE, 0, L.stream>>>(A, S, cur, L.cond, L.use_cond);         \
    }
#define GBMD_SRC_MB(M, SRC)                                                                                 \
    {                                                                                                       \
        const int mb = minb_of(L.ctas_req);                                                                 \
        if (mb == 16) GBMD_STEP_SRC(M, 16, SRC) else if (mb == 12) GBMD_STEP_SRC(M, 12, SRC)                \
        else if (mb == 8) GBMD_STEP_SRC(M, 8, SRC) else GBMD_STEP_SRC(M, 4, SRC)                            \
    }
        if (L.step_kernel == 4) {
            if (S.mode == MD_MIXED) GBMD_SRC_MB(MD_MIXED, 1)
            else GBMD_SRC_MB(MD_FP32, 1)
        } else {
            if (S.mode == MD_MIXED) GBMD_SRC_MB(MD_MIXED, 2)
            else GBMD_SRC_MB(MD_FP32, 2)
        }
#undef GBMD_SRC_MB
#undef GBMD_STEP_SRC
    } else if (S.mode != MD_FP64 && L.step_kernel == 3) {
#define GBMD_STEP_STG(M, NB, MB)                                                                       \
    {                                                                                                  \
        if (props)                                                                                     \
            k_step<M, true, NB, MB, true><<<g, TILE, L.stage_smem, L.stream>>>(A, S, cur, L.cond, L.use_cond, L.stage_cap); \
        else                                                                                           \
            k_step<M, false, NB, MB, true><<<g, TILE, L.stage_smem, L.stream>>>(A, S, cur, L.cond, L.use_cond, L.stage_cap); \
    }
        if (S.mode == MD_MIXED) GBMD_DISPATCH_NB_MINB(MD_MIXED, GBMD_STEP_STG)
        else GBMD_DISPATCH_NB_MINB(MD_FP32, GBMD_STEP_STG)
#undef GBMD_STEP_STG
    } else {
#define GBMD_STEP(M, NB, MB)                                                                           \
    {                                                                                                  \
        if (props) k_step_sm<M, true, NB, MB><<<g, TILE, 0, L.stream>>>(A, S, cur, L.cond, L.use_cond);         \
        else k_step_sm<M, false, NB, MB><<<g, TILE, 0, L.stream>>>(A, S, cur, L.cond, L.use_cond);               \
    }
        if (S.mode == MD_FP64) {
            if (props) k_step<MD_FP64, true, 2, 4, false><<<g, TILE, 0, L.stream>>>(A, S, cur, L.cond, L.use_cond, 0);
            else k_step<MD_FP64, false, 2, 4, false><<<g, TILE, 0, L.stream>>>(A, S, cur, L.cond, L.use_cond, 0);
        }
        else if (S.mode == MD_MIXED) GBMD_DISPATCH_NB_MINB(MD_MIXED, GBMD_STEP)
        else GBMD_DISPATCH_NB_MINB(MD_FP32, GBMD_STEP)
#undef GBMD_STEP
    }
    if (props && S.mode == MD_FP64) {
        // MD_MIXED / MD_FP32 step kernels write the props themselves (fixed-point sums)
        k_props_reduce<<<S.nrep * S.props_split, PROPS_THREADS, 0, L.stream>>>(A, S, 1, 1);
    }
    return cudaGetLastError();
}

cudaError_t launch_forces(const Arrays& A, const Scal& S, const Launch& L, int cur)
{
    const int g = tile_grid(S, L);
    // with the list-free step kernel there is no current W: the forces come from the cells too;
    // with the half list, from its pairs
    const bool cells = L.step_kernel == 4;
    if (S.mode != MD_FP64 && L.step_kernel == 5) {
        k_half_pairs<2><<<g, TILE, 0, L.stream>>>(A, S, cur);
        if (S.chain_len) k_chain_terms<<<g, TILE, 0, L.stream>>>(A, S, cur);
        k_half_to_f<<<g, TILE, 0, L.stream>>>(A, S);
        return cudaGetLastError();
    }
    if (S.chain_len && S.mode != MD_FP64) k_chain_terms<<<g, TILE, 0, L.stream>>>(A, S, cur);
    if (S.mode == MD_FP64) k_forces<MD_FP64><<<g, TILE, 0, L.stream>>>(A, S, cur);
    else if (S.mode == MD_MIXED && cells) k_forces<MD_MIXED, true><<<g, TILE, 0, L.stream>>>(A, S, cur);
    else if (S.mode == MD_MIXED) k_forces<MD_MIXED><<<g, TILE, 0, L.stream>>>(A, S, cur);
    else if (cells) k_forces<MD_FP32, true><<<g, TILE, 0, L.stream>>>(A, S, cur);
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
    k_props_reduce<<<S.nrep * S.props_split, PROPS_THREADS, 0, L.stream>>>(A, S, to_series ? 1 : 0, 0);
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

__global__ void k_debug_error(Arrays A, int bits, int nbr_seen)
{
    atomicOr(&A.g->err, bits);
    if (bits & ERR_NBR_OVERFLOW) atomicMax(&A.g->max_nbr_seen, nbr_seen);
}

cudaError_t launch_debug_error(const Arrays& A, const Launch& L, int bits, int nbr_seen)
{
    k_debug_error<<<1, 1, 0, L.stream>>>(A, bits, nbr_seen);
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
