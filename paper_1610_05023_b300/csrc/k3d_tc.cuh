// 3D stage kernel on the 5th-generation tensor cores (tcgen05): the volume
// term and the lift of the surface fluxes (Sec. 3.2, eq. dgLocalRhs) as
// BF16 / FP16 matrix products with FP32 accumulation in tensor memory, the
// flux, LSERK update (eqs. timeStepProc1-2) and trace pushes on the CUDA
// cores.  Same global layouts, arguments and results as k3d_stage.
//
// Products per tile of 128 cells (M = 128, one TMEM lane per cell):
//   acc_j   = P D_j^T + sum_f c_fj dP_f LIFT_f^T          (j = r, s, t)
//   acc_div = sum_j F_j D_j^T + XU LIFT^T
// with P the pressure, F_j = sum_i dr_j/dx_i u_i the contravariant fluxes,
// dP / XU the pressure / normal-velocity flux differences of the faces
// (XU scaled by Fscale), c_fj the reference-space outward normals of the
// faces scaled by Fscale (f0: -t, f1: -s, f2: r+s+t, f3: -r), so that
// Fscale_f n_f = sum_j c_fj grad r_j and the velocity lift folds into the
// reference-space gradient:
//   rhs_p = -rho c^2 acc_div,   rhs_u_i = -(1/rho) sum_j dr_j/dx_i acc_j.
// The signs of c_fj are folded into dP (faces 0, 1, 3 negated), so that
// every product is a plain accumulate.
//
// B operands (D_j and LIFT, rows = output nodes) stay in shared memory for
// the whole launch (one TMA bulk copy per CTA); A operands (cell data) are
// written by the threads in slabs of 16 K-values into a two-slot ring,
// whose slots are released by tcgen05.commit arrivals.  The split variant
// stores x = hi + lo (both BF16) for data and operators and accumulates
// hi*hi + lo*hi + hi*lo (three products; ~16 significant bits).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "k3d.cuh"

namespace dgh {

enum { TC_BF16 = 0, TC_FP16 = 1, TC_SPLIT_BF16 = 2 };

template <int N, int PREC>
struct CfgTC {
    static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6;
    static constexpr int NFP = (N + 1) * (N + 2) / 2;
    static constexpr int NF = 4 * NFP;
    static constexpr int NPAD = (NP + 15) / 16 * 16;        // output nodes (MMA N) and volume K
    static constexpr int FPAD = (NFP + 15) / 16 * 16;       // face nodes padded to whole K-steps
    static constexpr int KL = 4 * FPAD;                     // lift K
    static constexpr int NSV = NPAD / 16;                   // volume slabs per tile
    static constexpr int NSF = KL / 16;                     // flux slabs per tile
    static constexpr int CELLS = 128;                       // cells per tile (MMA M)
    static constexpr int NTHR = 256;                        // 8 warps: warp w -> 32-cell block w%4, half w/4
    static constexpr int NCOPY = PREC == TC_SPLIT_BF16 ? 2 : 1;
    static constexpr int LBO_B = (NPAD / 8) * 128;          // K-adjacent core matrices of a B operand
    static constexpr int BD = NPAD * NPAD * 2;              // one D_j (bytes)
    static constexpr int BL = NPAD * KL * 2;                // LIFT (bytes)
    static constexpr int BOPS = 3 * BD + BL;                // one copy of all operators
    static constexpr int LBO_A = (CELLS / 8) * 128;         // 2048
    static constexpr int CH = CELLS * 16 * 2;               // one A chunk (128 cells x 16 K), one copy
    static constexpr int SLOT = 4 * CH * NCOPY;             // a ring slot: 4 chunks (hi, then lo)
    static constexpr int OFF_OPS = 1024;                    // after barriers / scalars
    static constexpr int OFF_RING = OFF_OPS + BOPS * NCOPY;
    static constexpr int OFF_TAB = OFF_RING + 2 * SLOT;
    static constexpr int TAB_INTS = NF + 6 * NFP + 3 * NP;
    static constexpr size_t SMEM = OFF_TAB + 4 * TAB_INTS + 128;   // + 128: base alignment slack
    static constexpr int TC4 = 4 * NPAD;
    static constexpr int TCOLS = TC4 <= 32 ? 32 : TC4 <= 64 ? 64 : TC4 <= 128 ? 128 : TC4 <= 256 ? 256 : 512;
    static_assert(NPAD <= 256 && TC4 <= 512, "accumulators exceed tensor memory");
    // kind::f16 instruction descriptor: D = F32, A = B = BF16 (1) or F16 (0),
    // both K-major, N = NPAD, M = 128
    static constexpr uint32_t AB = PREC == TC_FP16 ? 0u : 1u;
    static constexpr uint32_t IDESC = (1u << 4) | (AB << 7) | (AB << 10) | (uint32_t(NPAD >> 3) << 17) | (uint32_t(128 >> 4) << 24);
};

// ------------------------------------------------------------ tcgen05 helpers
// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// 8-row x 16-byte core matrices, LBO = distance of K-adjacent core
// matrices, SBO = distance of row-adjacent (8-row group) core matrices.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8 consecutive K-values of one A row (16 bytes), hi (and lo) parts
template <int PREC>
__device__ __forceinline__ void tc_pack8(const float (&x)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (PREC == TC_FP16) {
            __half2 v = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
            h[i] = *reinterpret_cast<uint32_t *>(&v);
            l[i] = 0u;
        } else {
            __nv_bfloat162 v = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
            h[i] = *reinterpret_cast<uint32_t *>(&v);
            if (PREC == TC_SPLIT_BF16) {
                const float r0 = x[2 * i] - __bfloat162float(v.x), r1 = x[2 * i + 1] - __bfloat162float(v.y);
                __nv_bfloat162 w = __floats2bfloat162_rn(r0, r1);
                l[i] = *reinterpret_cast<uint32_t *>(&w);
            } else {
                l[i] = 0u;
            }
        }
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Bounded wait; a timeout sets the error word and the calling thread's
// flag.  The flags are combined at the next barrier with __syncthreads_or,
// so that all threads of the CTA take the same decision to stop.
__device__ __forceinline__ void tc_wait(uint64_t *bar, uint32_t parity, int *err, bool &bad) {
    if (bad) return;
    if (!mbar_wait(bar, parity, err)) bad = true;
}

template <int N, int PREC>
__global__ void __launch_bounds__(256, 1) k3d_tc(Args3 A, StageCoef sc, const uint8_t *ops) {
    using G = CfgTC<N, PREC>;
    constexpr int NP = G::NP, NFP = G::NFP, NF = G::NF, NPAD = G::NPAD, FPAD = G::FPAD;
    constexpr int QS = 4 * NP * 32, TI = 2 * NF * 32, GS = GEO3 * 32, CS = 4 * 32;
    extern __shared__ unsigned char smraw_tc[];
    // 1024-byte aligned base (descriptor addresses are taken from it)
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw_tc) + 127) & ~uintptr_t(127));
    uint64_t *bar_slot = reinterpret_cast<uint64_t *>(sm);        // [2]
    uint64_t *bar_acc = bar_slot + 2;
    uint64_t *bar_ops = bar_slot + 3;
    uint64_t *bar_fin = bar_slot + 4;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(sm + 64);
    int64_t *s_tile = reinterpret_cast<int64_t *>(sm + 128);     // [2]: current, next
    unsigned char *s_ops = sm + G::OFF_OPS;
    unsigned char *s_ring = sm + G::OFF_RING;
    int *sFm = reinterpret_cast<int *>(sm + G::OFF_TAB);
    int *sFp = sFm + NF;
    int *sNs = sFp + 6 * NFP;

    const int tid = threadIdx.x;
    const int w = tid >> 5, lane = tid & 31;
    const int bw = w & 3, hh = w >> 2;       // 32-cell block within the tile, half of the K-values
    const int cell = 32 * bw + lane;         // row of the A operand = TMEM lane
    const int64_t nblk = A.blk_end - A.blk_begin;
    const int64_t ntiles = (nblk + 3) / 4;

    if (tid == 0) {
        mbar_init(&bar_slot[0], 1);
        mbar_init(&bar_slot[1], 1);
        mbar_init(bar_acc, 1);
        mbar_init(bar_ops, 1);
        mbar_init(bar_fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // operators: one bulk copy per matrix and copy
        mbar_expect_tx(bar_ops, G::BOPS * G::NCOPY);
        for (int c = 0; c < G::NCOPY; ++c) {
            for (int j = 0; j < 3; ++j)
                bulk_g2s(s_ops + c * G::BOPS + j * G::BD, ops + c * G::BOPS + j * G::BD, G::BD, bar_ops);
            bulk_g2s(s_ops + c * G::BOPS + 3 * G::BD, ops + c * G::BOPS + 3 * G::BD, G::BL, bar_ops);
        }
        const int64_t t0 = (int64_t)atomicAdd(A.tile_ctr, 1ull);
        s_tile[0] = t0;
        s_tile[1] = ntiles;
    }
    if (w == 0) {   // tensor memory for the four accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"((uint32_t)G::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < NF; i += G::NTHR) sFm[i] = A.fmask[i];
    for (int i = tid; i < 6 * NFP; i += G::NTHR) sFp[i] = A.fperm[i];
    for (int i = tid; i < 3 * NP; i += G::NTHR) {   // face slots of every node, decoded to (f << 8 | m)
        const int v = A.nslot[i];
        sNs[i] = v < 0 ? -1 : ((v / NFP) << 8) | (v % NFP);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *s_tmem;
    double tstage = 0.0;
    if (A.src.n > 0) tstage = sc.time[0] + sc.c_dt;
    const uint32_t ops_addr = smem_addr(s_ops), ring_addr = smem_addr(s_ring);
    bool ops_ready = false;
    bool bad = false;          // this thread saw a timed-out wait
    bool stop = false;         // some thread of the CTA did (same value in all threads)
    uint32_t slab_ctr = 0;     // slabs issued so far (ring position, across tiles)
    uint32_t tile_iter = 0;

    for (;;) {
        const int64_t tile = s_tile[0];
        if (tile >= ntiles || stop) break;
        // claim the next tile now and pull its blocks into L2
        if (tid == 0) {
            const int64_t nt = (int64_t)atomicAdd(A.tile_ctr, 1ull);
            s_tile[1] = nt;
            if (nt < ntiles)
                for (int b = 0; b < 4; ++b) {
                    const int64_t gb = A.blk_begin + nt * 4 + b;
                    if (gb >= A.blk_end) break;
                    prefetch_l2(A.q + gb * QS, QS * 4);
                    prefetch_l2(A.res + gb * QS, QS * 4);
                    prefetch_l2(A.tin + gb * TI, TI * 4);
                    prefetch_l2(A.geo + gb * GS, GS * 4);
                    prefetch_l2(A.conn + gb * CS, CS * 4);
                }
        }
        const int64_t gb = A.blk_begin + tile * 4 + bw;    // this thread's 32-cell block
        const bool valid = gb < A.blk_end;
        const float *__restrict__ qb = A.q + (valid ? gb : 0) * QS;
        float g[9], nrm[4][4];
        float Zm = 1.f, rc2 = 0.f, irho = 0.f;
        int cf[4] = {kPadConn, kPadConn, kPadConn, kPadConn};
        float Zp[4] = {1.f, 1.f, 1.f, 1.f};
        if (valid) {
            const float *gg = A.geo + gb * GS;
#pragma unroll
            for (int q = 0; q < 9; ++q) g[q] = gg[q * 32 + lane];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                Zp[f] = gg[(9 + f) * 32 + lane];
                cf[f] = A.conn[gb * CS + f * 32 + lane];
            }
            rc2 = gg[13 * 32 + lane];
            irho = gg[14 * 32 + lane];
            Zm = gg[15 * 32 + lane];
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) g[q] = (q == 0 || q == 4 || q == 8) ? 1.f : 0.f;
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) face_normal(g, f, nrm[f][0], nrm[f][1], nrm[f][2], nrm[f][3]);

        // ---------------- A operands slab by slab, products issued per slab.
        // The global loads of slab s + 1 are issued before slab s is
        // converted, stored and handed to the tensor core, so that their
        // latency overlaps the barrier and the products of slab s.
        const float *__restrict__ tb = A.tin + (valid ? gb : 0) * TI;
        auto load_slab = [&](int s, float (&v)[48]) {
            if (s < G::NSV) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int n = 16 * s + 8 * hh + k;
                    const bool ok = valid && n < NP;
#pragma unroll
                    for (int fl = 0; fl < 4; ++fl) v[4 * k + fl] = ok ? qb[(fl * NP + n) * 32 + lane] : 0.f;
                }
            } else {
                const int sf = s - G::NSV;
                const int f = (sf * 16) / FPAD, hf = sf - f * (FPAD / 16);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int m = 16 * hf + 8 * hh + k;
                    const bool ok = valid && m < NFP;
                    const int n = ok ? sFm[f * NFP + m] : 0;
#pragma unroll
                    for (int fl = 0; fl < 4; ++fl) v[6 * k + fl] = ok ? qb[(fl * NP + n) * 32 + lane] : 0.f;
                    const float2 pu = ok ? reinterpret_cast<const float2 *>(tb)[(f * NFP + m) * 32 + lane] : make_float2(0.f, 0.f);
                    v[6 * k + 4] = pu.x;
                    v[6 * k + 5] = pu.y;
                }
            }
        };
        // returns true (in every thread) when the CTA must stop
        auto process_slab = [&](int s, const float (&v)[48]) -> bool {
            const uint32_t slot = slab_ctr & 1u;
            if (slab_ctr >= 2) tc_wait(&bar_slot[slot], ((slab_ctr >> 1) + 1u) & 1u, A.err, bad);
            unsigned char *sb = s_ring + slot * G::SLOT;
            const int rowoff = hh * G::LBO_A + (cell >> 3) * 128 + (cell & 7) * 16;
            auto put = [&](int chunk, const float (&x)[8]) {
                uint4 hi, lo;
                tc_pack8<PREC>(x, hi, lo);
                *reinterpret_cast<uint4 *>(sb + chunk * G::CH + rowoff) = hi;
                if (G::NCOPY == 2) *reinterpret_cast<uint4 *>(sb + (4 + chunk) * G::CH + rowoff) = lo;
            };
            if (s < G::NSV) {
                // volume slab: p and the contravariant fluxes F_r, F_s, F_t
                float xp[8], xr[8], xs[8], xt[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float u = v[4 * k + 1], vv = v[4 * k + 2], ww = v[4 * k + 3];
                    xp[k] = v[4 * k];
                    xr[k] = g[0] * u + g[1] * vv + g[2] * ww;
                    xs[k] = g[3] * u + g[4] * vv + g[5] * ww;
                    xt[k] = g[6] * u + g[7] * vv + g[8] * ww;
                }
                put(0, xp);
                put(1, xr);
                put(2, xs);
                put(3, xt);
            } else {
                // flux slab: XU = Fscale dUn and the signed dP of face f
                const int sf = s - G::NSV;
                const int f = (sf * 16) / FPAD, hf = sf - f * (FPAD / 16);
                const float nx = f == 0 ? nrm[0][0] : f == 1 ? nrm[1][0] : f == 2 ? nrm[2][0] : nrm[3][0];
                const float ny = f == 0 ? nrm[0][1] : f == 1 ? nrm[1][1] : f == 2 ? nrm[2][1] : nrm[3][1];
                const float nz = f == 0 ? nrm[0][2] : f == 1 ? nrm[1][2] : f == 2 ? nrm[2][2] : nrm[3][2];
                const float fsc = f == 0 ? nrm[0][3] : f == 1 ? nrm[1][3] : f == 2 ? nrm[2][3] : nrm[3][3];
                const float zp = f == 0 ? Zp[0] : f == 1 ? Zp[1] : f == 2 ? Zp[2] : Zp[3];
                const int cc = f == 0 ? cf[0] : f == 1 ? cf[1] : f == 2 ? cf[2] : cf[3];
                const bool dir = cc < 0 && cc != kPadConn && ((-1 - cc) & 1);
                const float izs = 1.0f / (Zm + zp);
                const float wm = Zm * izs, zz = Zm * zp * izs;
                const float sgn = f == 2 ? 1.f : -1.f;
                float xu[8], xd[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int m = 16 * hf + 8 * hh + k;
                    const float pm = v[6 * k];
                    const float unm = nx * v[6 * k + 1] + ny * v[6 * k + 2] + nz * v[6 * k + 3];
                    float pp = v[6 * k + 4], unp = v[6 * k + 5];
                    if (dir) {
                        pp = -pm;
                        unp = unm;
                    }
                    const float dP = wm * (pp - pm) + zz * (unm - unp);
                    const float dUn = (1.0f - wm) * (unp - unm) + izs * (pm - pp);
                    const bool ok = valid && m < NFP;
                    xu[k] = ok ? fsc * dUn : 0.f;
                    xd[k] = ok ? sgn * dP : 0.f;
                }
                put(0, xu);
                put(1, xd);
            }
            if (tid == 0 && !ops_ready) {   // operators in shared memory before the first product
                tc_wait(bar_ops, 0, A.err, bad);
                ops_ready = true;
            }
            fence_async_smem();
            if (__syncthreads_or(bad)) return true;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t a0 = ring_addr + slot * G::SLOT;
                const uint32_t alo = a0 + 4 * G::CH;
                const uint32_t blo = ops_addr + G::BOPS;
                auto ad = [&](uint32_t base, int chunk) { return tc_desc(base + chunk * G::CH, G::LBO_A, 128); };
                auto bd = [&](uint32_t base, int mat, int kstep) {
                    return tc_desc(base + mat * G::BD + kstep * 2 * G::LBO_B, G::LBO_B, 128);
                };
                // one product (plus the two correction products of the split variant)
                auto prod = [&](uint32_t acc_col, int chunk, int mat, int kstep, uint32_t accumulate) {
                    const uint32_t d = tbase + acc_col;
                    tc_mma(d, ad(a0, chunk), bd(ops_addr, mat, kstep), G::IDESC, accumulate);
                    if (G::NCOPY == 2) {
                        tc_mma(d, ad(alo, chunk), bd(ops_addr, mat, kstep), G::IDESC, 1u);
                        tc_mma(d, ad(a0, chunk), bd(blo, mat, kstep), G::IDESC, 1u);
                    }
                };
                if (s < G::NSV) {
                    const uint32_t first = s == 0 ? 0u : 1u;
#pragma unroll
                    for (int j = 0; j < 3; ++j) prod(j * NPAD, 0, j, s, first);
#pragma unroll
                    for (int j = 0; j < 3; ++j) prod(3 * NPAD, 1 + j, j, s, (s == 0 && j == 0) ? 0u : 1u);
                } else {
                    // LIFT is stored after the three D_j (mat index 3), K-step = flux slab index
                    const int sf = s - G::NSV;
                    const int f = (sf * 16) / FPAD;
                    prod(3 * NPAD, 0, 3, sf, 1u);
                    if (f == 2) {
#pragma unroll
                        for (int j = 0; j < 3; ++j) prod(j * NPAD, 1, 3, sf, 1u);
                    } else {
                        const int j = f == 0 ? 2 : f == 1 ? 1 : 0;   // f0: -t, f1: -s, f3: -r
                        prod(j * NPAD, 1, 3, sf, 1u);
                    }
                }
                tc_commit(&bar_slot[slot]);
                if (s == G::NSV + G::NSF - 1) tc_commit(bar_acc);
            }
            ++slab_ctr;
            return false;
        };
        {
            // one call site of each (instruction-cache footprint); the next
            // slab's values are copied into place after the current one is done
            constexpr int NS = G::NSV + G::NSF;
            float va[48], vb[48];
            load_slab(0, va);
#pragma unroll 1
            for (int s = 0; s < NS; ++s) {
                if (s + 1 < NS) load_slab(s + 1, vb);
                if ((stop = process_slab(s, va))) break;
#pragma unroll
                for (int i = 0; i < 48; ++i) va[i] = vb[i];
            }
        }
        if (stop) break;
        // ---------------- epilogue: accumulators -> right-hand sides, update, pushes
        tc_wait(bar_acc, tile_iter & 1u, A.err, bad);
        tc_fence_after();
        // warp-uniform: tcgen05.ld is executed by whole warps only
        if (__all_sync(0xffffffffu, valid && !bad)) {
            const int64_t kcell = gb * 32 + lane;
            bool has_src = false;
            for (int si = 0; si < A.src.n; ++si) has_src |= A.src.cell[si] == kcell;
            float *__restrict__ qg = A.q + gb * QS;
            float *__restrict__ rg = A.res + gb * QS;
            float *__restrict__ tout = A.tout;
            float *__restrict__ trb = A.trb;
            const uint32_t tl = tbase + ((uint32_t)(32 * bw) << 16);
            for (int j = hh; j < NPAD / 16; j += 2) {
                float ar[16], as_[16], at[16], adv[16];
                tmem_ld16(tl + 0 * NPAD + 16 * j, ar);
                tmem_ld16(tl + 1 * NPAD + 16 * j, as_);
                tmem_ld16(tl + 2 * NPAD + 16 * j, at);
                tmem_ld16(tl + 3 * NPAD + 16 * j, adv);
#pragma unroll
                for (int sub = 0; sub < 2; ++sub) {
                    // all loads of 8 nodes first, then the arithmetic and the stores
                    float qo[8][4], ro[8][4];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int n = 16 * j + 8 * sub + c;
                        const bool ok = n < NP;
#pragma unroll
                        for (int fl = 0; fl < 4; ++fl) {
                            const int idx = (fl * NP + (ok ? n : 0)) * 32 + lane;
                            ro[c][fl] = ok ? __ldg(rg + idx) : 0.f;
                            qo[c][fl] = ok ? qg[idx] : 0.f;
                        }
                    }
                    if (sub == 0) tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int cc16 = 8 * sub + c;
                        const int n = 16 * j + cc16;
                        if (n >= NP) break;
                        float rhs[4];
                        rhs[0] = -rc2 * adv[cc16];
                        rhs[1] = -irho * (g[0] * ar[cc16] + g[3] * as_[cc16] + g[6] * at[cc16]);
                        rhs[2] = -irho * (g[1] * ar[cc16] + g[4] * as_[cc16] + g[7] * at[cc16]);
                        rhs[3] = -irho * (g[2] * ar[cc16] + g[5] * as_[cc16] + g[8] * at[cc16]);
                        if (has_src)
                            for (int si = 0; si < A.src.n; ++si)
                                if (A.src.cell[si] == kcell)
                                    rhs[0] += (float)(A.src.amp[si] * ricker_integral_d(tstage, A.src.f_peak[si], A.src.t_s[si])) *
                                              A.src.vec[si * NP + n];
                        float qn[4];
#pragma unroll
                        for (int fl = 0; fl < 4; ++fl) {
                            const int idx = (fl * NP + n) * 32 + lane;
                            const float r = sc.a * ro[c][fl] + sc.dt * rhs[fl];
                            rg[idx] = r;
                            qn[fl] = qo[c][fl] + sc.b * r;
                            qg[idx] = qn[fl];
                        }
#pragma unroll 1
                        for (int sl = 0; sl < 3; ++sl) {
                            const int slotn = sNs[n * 3 + sl];
                            if (slotn < 0) break;
                            const int f = slotn >> 8, m = slotn & 255;
                            const float nx = f == 0 ? nrm[0][0] : f == 1 ? nrm[1][0] : f == 2 ? nrm[2][0] : nrm[3][0];
                            const float ny = f == 0 ? nrm[0][1] : f == 1 ? nrm[1][1] : f == 2 ? nrm[2][1] : nrm[3][1];
                            const float nz = f == 0 ? nrm[0][2] : f == 1 ? nrm[1][2] : f == 2 ? nrm[2][2] : nrm[3][2];
                            const float un = nx * qn[1] + ny * qn[2] + nz * qn[3];
                            const int cc = f == 0 ? cf[0] : f == 1 ? cf[1] : f == 2 ? cf[2] : cf[3];
                            if (cc == kPadConn) break;
                            if (cc >= 0) {
                                const int nb = cc >> 3;
                                const int64_t kn = nb >> 2;
                                const int fn = nb & 3;
                                const int mn = sFp[(cc & 7) * NFP + m];
                                if (DGH_IN_RANGE(A.err, kn, A.kcells))
                                    reinterpret_cast<float2 *>(tout)[(((kn >> 5) * 4 + fn) * NFP + mn) * 32 + (kn & 31)] =
                                        make_float2(qn[0], -un);
                            } else {
                                const int64_t b = (-1 - cc) >> 1;
                                if (DGH_IN_RANGE(A.err, b, A.nbfaces)) {
                                    trb[b * 2 * NFP + m] = qn[0];
                                    trb[b * 2 * NFP + NFP + m] = un;
                                }
                            }
                        }
                    }
                }
            }
        }
        tc_fence_before();
        stop = __syncthreads_or(bad);   // accumulators read: the next tile may overwrite them
        if (tid == 0) s_tile[0] = s_tile[1];
        ++tile_iter;
        __syncthreads();
    }
    // all issued products have completed before tensor memory is released
    __syncthreads();
    if (tid == 0) {
        tc_commit(bar_fin);
        mbar_wait(bar_fin, 0, A.err);
        if (!ops_ready) mbar_wait(bar_ops, 0, A.err);   // no bulk copy may still target shared memory
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"((uint32_t)G::TCOLS)
                     : "memory");
}

}  // namespace dgh
