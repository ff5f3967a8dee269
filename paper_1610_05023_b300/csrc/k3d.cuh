// 3D stage kernel: volume term, upwind surface flux + lift, LSERK update and
// new face traces of the tetrahedra (Sec. 3.2, eq. dgLocalRhs, eqs.
// timeStepProc1-2, Algorithm 2), fused into one pass over the cells.
//
// B300 design
//  * Cell-interleaved layouts: q, res [K/32][field][node][32]; the incoming
//    face traces of every cell [K/32][face][Nfp][32][p, n.u] (one 8-byte pair
//    per face node and cell); geometry [K/32][GEO3][32]; connectivity
//    [K/32][4][32].  A 32-cell block of each is one contiguous chunk.
//  * Traces are pushed, not pulled: after its update a cell writes (p, -n.u)
//    of each face straight into the incoming slots of the neighbour (in the
//    neighbour's face-node order), with fire-and-forget 8-byte stores.  The next stage
//    then reads its own incoming traces as one contiguous block -- no
//    dependent gathers on the critical path.  Boundary faces write their own
//    traces to a per-boundary-face array read by the 2D (face HABC) kernel,
//    which in turn writes the exterior state (2 r^-, 0) into the incoming slots.
//  * A CTA owns 32 cells (lane e = cell e) and NW warps; warp w computes the
//    w-th chunk of C output nodes, so derivative / lift rows are warp-uniform
//    shared-memory broadcasts read four at a time.
//  * The input blocks (q, incoming traces, geometry, connectivity) of the next
//    tile are fetched with TMA bulk copies (cp.async.bulk + mbarrier) into a
//    second buffer while the current tile is computed; res is prefetched into L2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgh {

constexpr int GEO3 = 16;  // per cell (interleaved [16][32]): drdx[9], Z of the 4 neighbours, rho c^2, 1/rho, Z
constexpr unsigned long long kWaitLimit = 1ull << 24;   // mbarrier polls before reporting a timeout
constexpr int kPadConn = (int)0x80000000;               // connectivity of padding cells (no pushes)

template <int N>
struct Cfg3 {
    static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6;
    static constexpr int NFP = (N + 1) * (N + 2) / 2;
    static constexpr int NF = 4 * NFP;
    static constexpr int NW = N == 1 ? 1 : N == 2 ? 2 : N == 3 ? 5 : N == 4 ? 9 : N == 5 ? 14 : 7;  // warps per CTA
    static constexpr int C = (NP + NW - 1) / NW;       // output nodes per warp
    static constexpr int CP = (C + 3) / 4 * 4;         // padded to float4
    static constexpr int MAXSLOT = 3;                  // a node lies on at most 3 faces
    static constexpr int QS = 4 * NP * 32;             // q of one block (floats)
    static constexpr int TI = 2 * NF * 32;             // incoming traces of one block
    static constexpr int GS = GEO3 * 32;               // geometry of one block
    static constexpr int CS = 4 * 32;                  // connectivity of one block (ints)
    static constexpr int STAGE = QS + TI + GS + CS;    // one pipeline stage (4-byte words)
    static constexpr int SPW = (NF + NW - 1) / NW;     // face slots per warp
    static constexpr int NSTAGE = (N >= 6 || N == 3) ? 1 : 2;   // input pipeline depth (N = 6: no room for two; N = 3: one more CTA per SM instead)
    static constexpr bool PQ = N == 4 || N == 5;      // (p, f_r, f_s, f_t) interleaved per lane: one float4 load per node
    static constexpr int SF = (PQ ? 4 : 3) * NP * 32;  // contravariant fluxes (N = 3: spills at 4 CTAs per SM; N = 6: no room)
    static constexpr int SM_WORDS = NP * 3 * NW * CP + NF * NW * CP + NSTAGE * STAGE + SF + NF + 6 * NFP + NP * MAXSLOT;
    static constexpr size_t SMEM = 16 + sizeof(float) * SM_WORDS;  // 16: two mbarriers
    static constexpr int MINB = N <= 3 ? 4 : N == 4 ? 2 : 1;
};

struct Args3 {
    float *q, *res;          // [K32][4][Np][32]
    const float *tin;        // incoming traces read this stage  [K32][4][Nfp][32][2] (p, n.u) pairs
    float *tout;             // incoming traces written for the next stage
    float *trb;              // own traces of boundary faces [Fb][2][Nfp]
    const float *geo;        // [K32][GEO3][32]
    const int *conn;         // [K32][4][32]: >=0 (k'*4+f')<<3 | sigma ; <0: -1 - (bidx<<1 | dirichlet)
    const float *D;          // [Np(m)][3][NW][CP]
    const float *LIFT;       // [NF][NW][CP]
    const int *fmask;        // [4][Nfp]
    const int *fperm;        // [6][Nfp]
    const int *nslot;        // [Np][3] face slots (f*Nfp+m) of every node, -1 padded
    int *err;                // device error word (bounded waits)
    int64_t blk_begin;       // 32-cell blocks [blk_begin, blk_end) handled by this launch
    int64_t blk_end;
    int64_t kcells, nbfaces;       // bounds of pushed cell and boundary-face ids (checked build)
    unsigned long long *tile_ctr;  // zeroed before the launch; CTAs claim blocks from it
    int max_tiles;                 // blocks per CTA at most (CTAs retire regularly so that
                                   // concurrent kernels of the HABC chain get SMs)
    SrcParams src;
};

// outward unit normal and Fscale = |grad zeta_f| of face f from the metric
__device__ __forceinline__ void face_normal(const float *g, int f, float &nx, float &ny, float &nz, float &fs) {
    // zeta: f0 -t, f1 -s, f2 +(r+s+t), f3 -r   (g[3j+i] = d r_j / d x_i)
    float a, b, c;
    if (f == 0) { a = -g[6]; b = -g[7]; c = -g[8]; }
    else if (f == 1) { a = -g[3]; b = -g[4]; c = -g[5]; }
    else if (f == 2) { a = g[0] + g[3] + g[6]; b = g[1] + g[4] + g[7]; c = g[2] + g[5] + g[8]; }
    else { a = -g[0]; b = -g[1]; c = -g[2]; }
    fs = sqrtf(a * a + b * b + c * c);
    const float inv = 1.0f / fs;
    nx = a * inv;
    ny = b * inv;
    nz = c * inv;
}

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// bounded wait on an mbarrier phase; returns false (and sets *err) on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          unsigned long long limit = kWaitLimit) {
    const uint32_t a = smem_addr(bar);
    for (unsigned long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    atomicExch(err, 1);
    return false;
}

template <int N>
__device__ __forceinline__ void issue_tile(const Args3 &A, float *stage, uint64_t *bar, int64_t blk) {
    using G = Cfg3<N>;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, (G::QS + G::TI + G::GS + G::CS) * 4);
    bulk_g2s(stage, A.q + blk * G::QS, G::QS * 4, bar);
    bulk_g2s(stage + G::QS, A.tin + blk * G::TI, G::TI * 4, bar);
    bulk_g2s(stage + G::QS + G::TI, A.geo + blk * G::GS, G::GS * 4, bar);
    bulk_g2s(stage + G::QS + G::TI + G::GS, A.conn + blk * G::CS, G::CS * 4, bar);
}

template <int N>
__global__ void __launch_bounds__(Cfg3<N>::NW * 32, Cfg3<N>::MINB) k3d_stage(Args3 A, StageCoef sc) {
    using G = Cfg3<N>;
    constexpr int NP = G::NP, NFP = G::NFP, NF = G::NF, NW = G::NW, C = G::C, CP = G::CP;
    constexpr int QS = G::QS, TI = G::TI, GS = G::GS;
    extern __shared__ __align__(16) unsigned char smraw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smraw);
    float *sD = reinterpret_cast<float *>(smraw + 16);  // NP*3*NW*CP
    float *sL = sD + NP * 3 * NW * CP;                  // NF*NW*CP
    float *sS = sL + NF * NW * CP;                      // NSTAGE pipeline stages
    float *sF = sS + G::NSTAGE * G::STAGE;              // [NP][32](p, f_r, f_s, f_t) (N = 4, 5), else [3][NP][32] fluxes
    int *sFm = reinterpret_cast<int *>(sF + G::SF);
    int *sFp = sFm + NF;
    int *sNs = sFp + 6 * NFP;
    const int tid = threadIdx.x, nth = NW * 32;
    const int w = tid >> 5, e = tid & 31;
    const int64_t ntiles = A.blk_end;

    // blocks are claimed dynamically (one atomic per block), so CTAs that start
    // late -- e.g. behind a concurrent kernel of the HABC chain -- simply take
    // fewer blocks
    __shared__ int64_t s_blk[2];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int q = 0; q < G::NSTAGE; ++q) {
            const int64_t b = q < A.max_tiles ? A.blk_begin + (int64_t)atomicAdd(A.tile_ctr, 1ull) : ntiles;
            s_blk[q] = b;
            if (b < ntiles) issue_tile<N>(A, sS + q * G::STAGE, &bar[q], b);
        }
    }
    for (int i = tid; i < NP * 3 * NW * CP; i += nth) sD[i] = A.D[i];
    for (int i = tid; i < NF * NW * CP; i += nth) sL[i] = A.LIFT[i];
    for (int i = tid; i < NF; i += nth) sFm[i] = A.fmask[i];
    for (int i = tid; i < 6 * NFP; i += nth) sFp[i] = A.fperm[i];
    for (int i = tid; i < NP * 3; i += nth) sNs[i] = A.nslot[i];
    double tstage = 0.0;
    if (A.src.n > 0) tstage = sc.time[0] + sc.c_dt;
    __syncthreads();

    for (int it = 0;; ++it) {
        const int st = G::NSTAGE == 2 ? (it & 1) : 0;
        const int64_t blk = s_blk[st];
        if (blk >= ntiles) break;
        float *sQ = sS + st * G::STAGE;
        float *sTi = sQ + QS;       // incoming traces, overwritten in place by the flux terms
        const float *sG = sTi + TI;
        const int *sC = reinterpret_cast<const int *>(sG + GS);
        if (!mbar_wait(&bar[st], (G::NSTAGE == 2 ? (it >> 1) : it) & 1, A.err)) return;
        const float *__restrict__ rgc = A.res + blk * QS;
        float rpre[C][4];   // this warp's res values, fetched now and used by the update
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int n = w * C + c;
#pragma unroll
            for (int fl = 0; fl < 4; ++fl) rpre[c][fl] = (C * NW == NP || n < NP) ? __ldg(rgc + (fl * NP + n) * 32 + e) : 0.f;
        }
        float g[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) g[q] = sG[q * 32 + e];
        const float Zm = sG[15 * 32 + e];
        float nrm[4][4];    // outward normal and Fscale of the 4 faces
#pragma unroll
        for (int f = 0; f < 4; ++f) face_normal(g, f, nrm[f][0], nrm[f][1], nrm[f][2], nrm[f][3]);
        // ---------------- face fluxes (slots f*NFP+m split over the warps; per-face terms hoisted)
        {
            const int s0 = w * G::SPW, s1 = (s0 + G::SPW < NF) ? s0 + G::SPW : NF;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (f * NFP >= s1 || (f + 1) * NFP <= s0) continue;
                const float nx = nrm[f][0], ny = nrm[f][1], nz = nrm[f][2], fsc = nrm[f][3];
                const float Zp = sG[(9 + f) * 32 + e];
                const float izs = 1.0f / (Zm + Zp);
                const float wm = Zm * izs, zz = Zm * Zp * izs;
                const int c = sC[f * 32 + e];
                const bool dir = c < 0 && ((-1 - c) & 1);
                const int m0 = (s0 > f * NFP) ? s0 - f * NFP : 0;
                const int m1 = (s1 < (f + 1) * NFP) ? s1 - f * NFP : NFP;
                for (int m = m0; m < m1; ++m) {
                    const int n = sFm[f * NFP + m];
                    const float pm = sQ[n * 32 + e];
                    const float unm = nx * sQ[(NP + n) * 32 + e] + ny * sQ[(2 * NP + n) * 32 + e] + nz * sQ[(3 * NP + n) * 32 + e];
                    float2 *x_slot = reinterpret_cast<float2 *>(sTi) + (f * NFP + m) * 32 + e;   // (p, n.u) -> Fscale (dP, dUn)
                    const float2 xin = *x_slot;
                    float pp = xin.x, unp = xin.y;
                    if (dir) {   // p = 0 face: mirror state
                        pp = -pm;
                        unp = unm;
                    }
                    const float dP = wm * (pp - pm) + zz * (unm - unp);
                    const float dUn = (1.0f - wm) * (unp - unm) + izs * (pm - pp);
                    *x_slot = make_float2(fsc * dP, fsc * dUn);
                }
            }
        }
        // ---------------- contravariant fluxes f_j = sum_i dr_j/dx_i u_i (same phase:
        // the flux terms are read only by the lift, after the volume term)
        for (int n = w; n < NP; n += NW) {
            const float u = sQ[(NP + n) * 32 + e], v = sQ[(2 * NP + n) * 32 + e], ww = sQ[(3 * NP + n) * 32 + e];
            const float fr = g[0] * u + g[1] * v + g[2] * ww, fs = g[3] * u + g[4] * v + g[5] * ww,
                        ft = g[6] * u + g[7] * v + g[8] * ww;
            if (G::PQ) {
                reinterpret_cast<float4 *>(sF)[n * 32 + e] = make_float4(sQ[n * 32 + e], fr, fs, ft);
            } else {
                sF[n * 32 + e] = fr;
                sF[(NP + n) * 32 + e] = fs;
                sF[(2 * NP + n) * 32 + e] = ft;
            }
        }
        __syncthreads();
        // ---------------- volume term for the chunk of warp w
        // Output nodes in pairs: packed FP32x2 FMAs (each half an ordinary
        // round-to-nearest FP32 FMA) on the pairs of a float4 row.
        float2 div2[CP / 2], dr2[CP / 2], ds2[CP / 2], dt2[CP / 2];
#pragma unroll
        for (int c = 0; c < CP / 2; ++c) div2[c] = dr2[c] = ds2[c] = dt2[c] = make_float2(0.f, 0.f);
        const float4 *D4 = reinterpret_cast<const float4 *>(sD) + w * (CP / 4);
#pragma unroll 5
        for (int m = 0; m < NP; ++m) {
            float p, fr, fs, ft;
            if (G::PQ) {
                const float4 v = reinterpret_cast<const float4 *>(sF)[m * 32 + e];
                p = v.x;
                fr = v.y;
                fs = v.z;
                ft = v.w;
            } else {
                p = sQ[m * 32 + e];
                fr = sF[m * 32 + e];
                fs = sF[(NP + m) * 32 + e];
                ft = sF[(2 * NP + m) * 32 + e];
            }
            const float2 p2 = make_float2(p, p), fr2 = make_float2(fr, fr), fs2 = make_float2(fs, fs), ft2 = make_float2(ft, ft);
            const float4 *Dm = D4 + m * 3 * NW * (CP / 4);
#pragma unroll
            for (int c4 = 0; c4 < CP / 4; ++c4) {
                const float4 a = Dm[c4], b = Dm[NW * (CP / 4) + c4], d = Dm[2 * NW * (CP / 4) + c4];
                const float2 a2[2] = {make_float2(a.x, a.y), make_float2(a.z, a.w)};
                const float2 b2[2] = {make_float2(b.x, b.y), make_float2(b.z, b.w)};
                const float2 d2[2] = {make_float2(d.x, d.y), make_float2(d.z, d.w)};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = 2 * c4 + h;
                    div2[c] = __ffma2_rn(a2[h], fr2, div2[c]);
                    div2[c] = __ffma2_rn(b2[h], fs2, div2[c]);
                    div2[c] = __ffma2_rn(d2[h], ft2, div2[c]);
                    dr2[c] = __ffma2_rn(a2[h], p2, dr2[c]);
                    ds2[c] = __ffma2_rn(b2[h], p2, ds2[c]);
                    dt2[c] = __ffma2_rn(d2[h], p2, dt2[c]);
                }
            }
        }
        float div[CP], dr[CP], ds[CP], dt[CP];
#pragma unroll
        for (int c = 0; c < CP / 2; ++c) {
            div[2 * c] = div2[c].x;
            div[2 * c + 1] = div2[c].y;
            dr[2 * c] = dr2[c].x;
            dr[2 * c + 1] = dr2[c].y;
            ds[2 * c] = ds2[c].x;
            ds[2 * c + 1] = ds2[c].y;
            dt[2 * c] = dt2[c].x;
            dt[2 * c + 1] = dt2[c].y;
        }
        // gradient of p in physical coordinates; reuse dr/ds/dt as the velocity right-hand sides
#pragma unroll
        for (int c = 0; c < CP; ++c) {
            const float a = dr[c], b = ds[c], d = dt[c];
            dr[c] = g[0] * a + g[3] * b + g[6] * d;
            ds[c] = g[1] * a + g[4] * b + g[7] * d;
            dt[c] = g[2] * a + g[5] * b + g[8] * d;
        }
        // ---------------- lift of the face terms
        const float4 *L4 = reinterpret_cast<const float4 *>(sL) + w * (CP / 4);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            float2 lp2[CP / 2], dv2[CP / 2];
#pragma unroll
            for (int c = 0; c < CP / 2; ++c) {
                lp2[c] = make_float2(0.f, 0.f);
                dv2[c] = make_float2(div[2 * c], div[2 * c + 1]);
            }
#pragma unroll 5
            for (int m = 0; m < NFP; ++m) {
                const int fm = f * NFP + m;
                const float2 xpu = reinterpret_cast<const float2 *>(sTi)[(f * NFP + m) * 32 + e];
                const float xu = xpu.y, xp = xpu.x;
                const float2 xu2 = make_float2(xu, xu), xp2 = make_float2(xp, xp);
                const float4 *Lm = L4 + fm * NW * (CP / 4);
#pragma unroll
                for (int c4 = 0; c4 < CP / 4; ++c4) {
                    const float4 l = Lm[c4];
                    const float2 l2[2] = {make_float2(l.x, l.y), make_float2(l.z, l.w)};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        dv2[2 * c4 + h] = __ffma2_rn(l2[h], xu2, dv2[2 * c4 + h]);
                        lp2[2 * c4 + h] = __ffma2_rn(l2[h], xp2, lp2[2 * c4 + h]);
                    }
                }
            }
            float lp[CP];
#pragma unroll
            for (int c = 0; c < CP / 2; ++c) {
                div[2 * c] = dv2[c].x;
                div[2 * c + 1] = dv2[c].y;
                lp[2 * c] = lp2[c].x;
                lp[2 * c + 1] = lp2[c].y;
            }
            const float nx = nrm[f][0], ny = nrm[f][1], nz = nrm[f][2];
#pragma unroll
            for (int c = 0; c < CP; ++c) {
                dr[c] += nx * lp[c];
                ds[c] += ny * lp[c];
                dt[c] += nz * lp[c];
            }
        }
        // ---------------- update, then push the new traces
        const float rc2 = sG[13 * 32 + e], irho = sG[14 * 32 + e];
        const int64_t k = blk * 32 + e;
        float *qg = A.q + blk * QS;
        float *rg = A.res + blk * QS;
        const int cf0 = sC[e], cf1 = sC[32 + e], cf2 = sC[64 + e], cf3 = sC[96 + e];
        bool has_src = false;   // one scan of the source list per tile, not per node
        for (int s = 0; s < A.src.n; ++s) has_src |= A.src.cell[s] == k;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int n = w * C + c;
            if (C * NW != NP && n >= NP) break;
            float rhs[4];
            rhs[0] = -rc2 * div[c];
            rhs[1] = -irho * dr[c];
            rhs[2] = -irho * ds[c];
            rhs[3] = -irho * dt[c];
            if (has_src)
                for (int s = 0; s < A.src.n; ++s)
                    if (A.src.cell[s] == k)
                        rhs[0] += (float)(A.src.amp[s] * ricker_integral_d(tstage, A.src.f_peak[s], A.src.t_s[s])) *
                                  A.src.vec[s * NP + n];
            float qn[4];
#pragma unroll
            for (int fl = 0; fl < 4; ++fl) {
                const int idx = (fl * NP + n) * 32 + e;
                const float r = sc.a * rpre[c][fl] + sc.dt * rhs[fl];
                rg[idx] = r;
                qn[fl] = sQ[idx] + sc.b * r;
                qg[idx] = qn[fl];
            }
#pragma unroll
            for (int s = 0; s < G::MAXSLOT; ++s) {
                const int slot = sNs[n * G::MAXSLOT + s];
                if (slot < 0) break;
                const int f = slot / NFP, m = slot % NFP;
                const float nx = f == 0 ? nrm[0][0] : f == 1 ? nrm[1][0] : f == 2 ? nrm[2][0] : nrm[3][0];
                const float ny = f == 0 ? nrm[0][1] : f == 1 ? nrm[1][1] : f == 2 ? nrm[2][1] : nrm[3][1];
                const float nz = f == 0 ? nrm[0][2] : f == 1 ? nrm[1][2] : f == 2 ? nrm[2][2] : nrm[3][2];
                const float un = nx * qn[1] + ny * qn[2] + nz * qn[3];
                const int cc = f == 0 ? cf0 : f == 1 ? cf1 : f == 2 ? cf2 : cf3;
                if (cc == kPadConn) break;   // padding cell: nothing to push
                if (cc >= 0) {   // neighbour face (k', f'): its node order, its normal
                    const int nb = cc >> 3;
                    const int64_t kn = nb >> 2;
                    const int fn = nb & 3;
                    const int mn = sFp[(cc & 7) * NFP + m];
                    if (DGH_IN_RANGE(A.err, kn, A.kcells))
                        reinterpret_cast<float2 *>(A.tout)[(((kn >> 5) * 4 + fn) * NFP + mn) * 32 + (kn & 31)] = make_float2(qn[0], -un);
                } else {         // boundary face: own trace for the face HABC solver
                    const int64_t b = (-1 - cc) >> 1;
                    if (DGH_IN_RANGE(A.err, b, A.nbfaces)) {
                        A.trb[b * 2 * NFP + m] = qn[0];
                        A.trb[b * 2 * NFP + NFP + m] = un;
                    }
                }
            }
        }
        __syncthreads();   // stage st (with the flux terms) is free again
        if (tid == 0) {
            const int64_t b = it + G::NSTAGE < A.max_tiles ? A.blk_begin + (int64_t)atomicAdd(A.tile_ctr, 1ull) : ntiles;
            s_blk[st] = b;
            if (b < ntiles) issue_tile<N>(A, sS + st * G::STAGE, &bar[st], b);
        }
        // With two stages, s_blk[st] is next read two iterations later, after
        // the barrier of the iteration in between; one stage needs a barrier.
        if (G::NSTAGE == 1) __syncthreads();
    }
}

// Push the traces of the current fields (initialisation of the boundary algebra).
template <int N>
__global__ void __launch_bounds__(128) k3d_traces(const float *q, const float *geo, const int *conn, const int *fmask,
                                                  const int *fperm, float *tout, float *trb, int64_t K) {
    using G = Cfg3<N>;
    constexpr int NP = G::NP, NFP = G::NFP;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= K * 4 * NFP) return;
    const int64_t k = i / (4 * NFP);
    const int fm = (int)(i % (4 * NFP)), f = fm / NFP, m = fm % NFP;
    const int64_t blk = k / 32;
    const int e = (int)(k % 32);
    const int n = fmask[fm];
    float g[9];
    for (int q = 0; q < 9; ++q) g[q] = geo[(blk * GEO3 + q) * 32 + e];
    float nx, ny, nz, fsc;
    face_normal(g, f, nx, ny, nz, fsc);
    const float *qt = q + blk * (4 * NP * 32);
    const float p = qt[n * 32 + e];
    const float un = nx * qt[(NP + n) * 32 + e] + ny * qt[(2 * NP + n) * 32 + e] + nz * qt[(3 * NP + n) * 32 + e];
    const int cc = conn[(blk * 4 + f) * 32 + e];
    if (cc == kPadConn) return;
    if (cc >= 0) {
        const int nb = cc >> 3;
        const int64_t kn = nb >> 2;
        const int fn = nb & 3;
        const int mn = fperm[(cc & 7) * NFP + m];
        reinterpret_cast<float2 *>(tout)[(((kn >> 5) * 4 + fn) * NFP + mn) * 32 + (kn & 31)] = make_float2(p, -un);
    } else {
        const int64_t b = (-1 - cc) >> 1;
        trb[b * 2 * NFP + m] = p;
        trb[b * 2 * NFP + NFP + m] = un;
    }
}

}  // namespace dgh
