// 3D stage kernel with the volume and lift contractions on the tcgen05
// tensor cores at FP32-grade accuracy (split TF32), warp-specialised.
// Same global layouts, arguments and results as k3d_stage: the volume term
// and upwind surface flux + lift of eq. dgLocalRhs (Sec. 3.2), the LSERK
// update of eqs. timeStepProc1-2 and the new face traces (Algorithm 2).
//
// Products per tile of 128 cells (M = 128, one TMEM lane per cell), with
// the same reference-space folding as k3d_tc:
//   acc_j   = P D_j^T + sum_f c_fj dP_f LIFT_f^T          (j = r, s, t)
//   acc_div = sum_j F_j D_j^T + XU LIFT^T
//   rhs_p = -rho c^2 acc_div,   rhs_u_i = -(1/rho) sum_j dr_j/dx_i acc_j,
// c_fj in {0, +-1} the reference normals (f0: -t, f1: -s, f2: r+s+t, f3: -r),
// their signs folded into dP.  P D_j^T for the three j is one product
// against the stacked operator [D_r; D_s; D_t].
//
// Split TF32 (x = hi + lo, both TF32 = FP32 with 13 zero low bits): every
// product is hi_a*hi_b + lo_a*hi_b + hi_a*lo_b in kind::tf32 with FP32
// accumulation.  Each operand is represented to 2^-22 relative and the
// dropped lo*lo term is below 2^-22 of the product, so the contractions are
// within a few units of FP32 rounding (Ootomo & Yokota 2022 on TF32 error
// correction; the tensor core truncates the 13 low bits of its FP32
// inputs, so hi and lo are rounded explicitly before they reach it).
//
// B300 design: one persistent CTA per SM, 18 warps in four roles.
//   warp 0     producer: claims tiles, TMA bulk-copies each tile's q and
//              geometry into one of two shared-memory stages (a stage is
//              held until the converters and the epilogue of its tile are
//              done with it);
//   warp 1     MMA issuer (one thread) and tensor-memory owner;
//   warps 2-9  converters, two warps per 32-cell block taking alternate
//              slabs (thread = cell): flux differences (incoming traces read
//              from L2 one slab ahead), contravariant fluxes, hi/lo split;
//              the A operands go straight into tensor memory (tcgen05.st) in
//              a ring of four 32-column slabs, so no shared-memory bandwidth
//              is spent on them.  The store of a slab completes while the
//              warp computes its next one;
//   warps 10-17 epilogue, two warps per 32-cell block (thread = cell):
//              accumulators (tcgen05.ld) and the old state (from the stage)
//              -> right-hand sides, LSERK update (each warp every other
//              2-node chunk, res read from L2 one chunk ahead), the new state
//              written to global memory and over the old one in the stage;
//              then the trace pushes read from the stage, each warp two
//              faces, node after node of the face.
// The work per cell is latency-bound, so the roles get as many warps as
// the register file allows (18 warps: 96 registers each, as four
// sub-partitions hold at most five warps of 96); the per-thread state is
// kept small enough for that without spills (with most of the SM's memory
// given to shared memory, a spilled register would be reloaded from L2).
// An M = 128 tcgen05.mma costs about the same issue time for any N up to
// 256 on this part, so products are grouped into as few instructions as
// the accumulator layout allows (P D_j^T for all three j in one N = 3 NPAD
// product).
// Two accumulator sets in tensor memory let the epilogue of tile i run
// beside the products of tile i + 1.  The B operands (D stack and LIFT,
// hi and lo) stay in shared memory for the whole launch.  Every wait is
// bounded: a timeout sets the error word and the CTA's abort flag, every
// role leaves its loop, in-flight products and copies are drained and
// tensor memory is freed.
#pragma once
#include "k3d_tc.cuh"

namespace dgh {

template <int N>
struct CfgTF {
    static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6;
    static constexpr int NFP = (N + 1) * (N + 2) / 2;
    static constexpr int NF = 4 * NFP;
    static constexpr int NPAD = (NP + 15) / 16 * 16;        // output nodes per accumulator (MMA N)
    static constexpr int KV = (NP + 7) / 8 * 8;             // volume K (TF32 K-step = 8)
    static constexpr int FK = (NFP + 7) / 8 * 8;            // K of one face
    static constexpr int NKV = KV / 8, NKF = FK / 8;
    static constexpr int NSLAB = 2 * NKV + 4 * NKF;         // ring slabs per tile
    static constexpr int QS = 4 * NP * 32, TI = 2 * NF * 32, GS = GEO3 * 32, CS = 4 * 32;   // floats per 32-cell block
    // B operand images (TF32, K-major, no swizzle; rows = output nodes)
    static constexpr int RD = 3 * NPAD;                     // [D_r; D_s; D_t]
    static constexpr int LBO_D = (RD / 8) * 128, LBO_L = (NPAD / 8) * 128;
    static constexpr int BD = RD * KV * 4, BL = NPAD * 4 * FK * 4;
    static constexpr int BOPS = BD + BL;                    // one copy (hi or lo), bytes
    // shared memory (16-byte aligned): barriers and scalars, operators (hi,
    // lo), two stages of q and geometry, tables
    static constexpr int OFF_OPS = 256;
    static constexpr int STAGE = 4 * (QS + GS) * 4;
    static constexpr int OFF_STAGE = OFF_OPS + 2 * BOPS;
    static constexpr int OFF_TAB = OFF_STAGE + 2 * STAGE;
    static constexpr int TAB_INTS = NF + 6 * NFP + 4 * NP;  // fmask, fperm, node -> face position
    static constexpr int SMEM_USED = OFF_TAB + 4 * TAB_INTS;
    // at least 116 KB so that one CTA runs per SM (it allocates all 512 TMEM columns)
    static constexpr size_t SMEM = SMEM_USED > 118784 ? SMEM_USED : 118784;
    static_assert(SMEM_USED <= 232448, "shared memory");
    // tensor memory: two accumulator sets, then the A ring
    static constexpr int ACC = 4 * NPAD;                    // acc_r | acc_s | acc_t | acc_div
    static constexpr int RING_COL = 2 * ACC;
    static_assert(RING_COL + 32 * 4 <= 512, "tensor memory");
    static_assert(RD <= 256 && NPAD % 16 == 0, "MMA N");
    static constexpr int NTHR = 576;   // 18 warps
    static constexpr int NCONV = 8;    // converter warps (two per 32-cell block)
    static constexpr int NEPI = 8;     // epilogue warps (two per 32-cell block)
    // kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128
    __host__ __device__ static constexpr uint32_t idesc(int n) {
        return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
    }
};

__device__ __forceinline__ void tf_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float (&v)[2]) {
    uint32_t r[2];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
    v[0] = __uint_as_float(r[0]);
    v[1] = __uint_as_float(r[1]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Nearest TF32 value of a finite float (ties away from zero): add half of
// the last kept place to the magnitude bits, clear the 13 dropped bits.
// Integer ops run at full rate on the ALU pipe.
__device__ __forceinline__ uint32_t tf32_rna_bits(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// x = hi + lo, hi and lo TF32 (round to nearest): x - hi is exact in FP32,
// |x - (hi + lo)| <= 2^-22 |x|.
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_rna_bits(x);
    lo = tf32_rna_bits(x - __uint_as_float(hi));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kTfWaitNs = 2000000000ull;   // a role gives up after 2 s without progress
constexpr uint32_t kTfSuspendNs = 200000u;      // longest sleep per try (wakes at once when the phase completes)

// Bounded wait on an mbarrier phase.  The waiting thread sleeps inside
// try_wait (suspend-time hint) instead of spinning, so waiting warps leave
// the issue slots to the working ones.  Gives up -- setting the error word
// and the CTA's abort flag -- after kTfWaitNs, or at once when another role
// has aborted.
__device__ __forceinline__ bool tf_wait(uint64_t *bar, uint32_t parity, int *err, volatile int *abort_flag) {
    const uint32_t a = smem_addr(bar);
    uint64_t t0 = 0;
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(a), "r"(parity), "r"(kTfSuspendNs)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
        const uint64_t now = global_ns();
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > kTfWaitNs) {
            atomicExch(err, 1);
            *abort_flag = 1;
            return false;
        }
    }
}

// Incoming traces (p, n.u) of face slab kl (face f = kl / NKF, nodes 8 h ..).
// K positions past the face's last node repeat its last node: the operator
// rows there are zero, so any finite value contributes nothing, and the
// loads need no branch.
template <int N>
__device__ __forceinline__ void tf_load_tin(const float2 *__restrict__ tb, int kl, int lane, float2 (&t)[8]) {
    using G = CfgTF<N>;
    const int f = kl / G::NKF, h = kl - f * G::NKF;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int m = min(8 * h + k, G::NFP - 1);
        t[k] = tb[(f * G::NFP + m) * 32 + lane];
    }
}

template <int N>
__global__ void __launch_bounds__(576, 1) k3d_tf32(Args3 A, StageCoef sc, const uint8_t *ops) {
    using G = CfgTF<N>;
    constexpr int NP = G::NP, NFP = G::NFP, NF = G::NF, NPAD = G::NPAD, QS = G::QS, TI = G::TI, GS = G::GS, CS = G::CS;
    extern __shared__ __align__(16) unsigned char sm_tf[];
    unsigned char *sm = sm_tf;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm);
    uint64_t *stage_full = bars + 0, *stage_empty = bars + 2;    // [2] each
    uint64_t *ring_full = bars + 4, *ring_empty = bars + 8;      // [4] each
    uint64_t *acc_full = bars + 12, *acc_empty = bars + 14;      // [2] each
    uint64_t *ops_bar = bars + 16, *fin_bar = bars + 17;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(sm + 160);
    volatile int *s_abort = reinterpret_cast<volatile int *>(sm + 164);
    volatile int64_t *s_tiles = reinterpret_cast<volatile int64_t *>(sm + 192);   // [8]
    unsigned char *s_ops = sm + G::OFF_OPS;
    // stage st: q of the four blocks [4][QS], then their geometry [4][GS]
    auto stage_q = [&](int st) { return reinterpret_cast<float *>(sm + G::OFF_STAGE + st * G::STAGE); };
    auto stage_g = [&](int st) { return reinterpret_cast<float *>(sm + G::OFF_STAGE + st * G::STAGE) + 4 * QS; };
    int *sFm = reinterpret_cast<int *>(sm + G::OFF_TAB);
    int *sFp = sFm + NF;
    int *sNf = sFp + 6 * NFP;   // [4][NP]: position m of node n on face f, or -1

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int64_t nblk = A.blk_end - A.blk_begin;
    const int64_t ntiles = (nblk + 3) / 4;

    if (tid == 0) {
        for (int st = 0; st < 2; ++st) {
            mbar_init(&stage_full[st], 1);
            mbar_init(&stage_empty[st], 32 * (G::NCONV + G::NEPI));   // converters and epilogue
            mbar_init(&acc_full[st], 2);      // the products' commit + the issuing thread's release
            mbar_init(&acc_empty[st], 32 * G::NEPI);
        }
        for (int r = 0; r < 4; ++r) {
            mbar_init(&ring_full[r], 128);
            mbar_init(&ring_empty[r], 1);
        }
        mbar_init(ops_bar, 1);
        mbar_init(fin_bar, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(ops_bar, 2 * G::BOPS);
        bulk_g2s(s_ops, ops, 2 * G::BOPS, ops_bar);
    }
    if (w == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(s_tmem)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < NF; i += G::NTHR) sFm[i] = A.fmask[i];
    for (int i = tid; i < 6 * NFP; i += G::NTHR) sFp[i] = A.fperm[i];
    for (int i = tid; i < 4 * NP; i += G::NTHR) {
        const int f = i / NP, n = i % NP;
        int pos = -1;
        for (int m = 0; m < NFP; ++m)
            if (A.fmask[f * NFP + m] == n) pos = m;
        sNf[i] = pos;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *s_tmem;
    int last_issued = -1;       // producer: last tile iteration whose stage copies were issued
    bool reached_end = false;   // producer: the end of the work was signalled (every issued copy consumed)

    if (w == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            auto claim = [&](int i) -> int64_t {
                return i < A.max_tiles ? (int64_t)atomicAdd(A.tile_ctr, 1ull) : ntiles;
            };
            // No L2 prefetch of the next tile here: its stage copy runs about a tile
            // period later, by when a prefetched line has often been evicted (the
            // DRAM reads grew by a third with it).  The converters request the
            // incoming traces and res of their own block closer to their use.
            int64_t next = claim(0);
            for (int i = 0;; ++i) {
                const int64_t t = next;
                next = t < ntiles ? claim(i + 1) : ntiles;
                s_tiles[i & 7] = t < ntiles ? t : ntiles;
                const int st = i & 1;
                // stage st is free once both consumers of tile i - 2 are done with it
                if (i >= 2 && !tf_wait(&stage_empty[st], ((i >> 1) + 1) & 1, A.err, s_abort)) break;
                if (t >= ntiles) {
                    mbar_arrive(&stage_full[st]);   // end of the work: releases the converters
                    reached_end = true;
                    break;
                }
                int nv = 0;
                for (int b = 0; b < 4; ++b) nv += (A.blk_begin + 4 * t + b < A.blk_end) ? 1 : 0;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&stage_full[st], nv * (QS + GS) * 4);
                for (int b = 0; b < nv; ++b) {
                    const int64_t gb = A.blk_begin + 4 * t + b;
                    bulk_g2s(stage_q(st) + b * QS, A.q + gb * QS, QS * 4, &stage_full[st]);
                    bulk_g2s(stage_g(st) + b * GS, A.geo + gb * GS, GS * 4, &stage_full[st]);
                }
                last_issued = i;
            }
        }
    } else if (w == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t ops_hi = smem_addr(s_ops), ops_lo = ops_hi + G::BOPS;
            auto bdesc_d = [&](uint32_t base, int kv, int row0) {
                return tc_desc(base + kv * 2 * G::LBO_D + (row0 / 8) * 128, G::LBO_D, 128);
            };
            auto bdesc_l = [&](uint32_t base, int kl) { return tc_desc(base + G::BD + kl * 2 * G::LBO_L, G::LBO_L, 128); };
            // hi*hi + lo*hi + hi*lo into D
            auto prod3 = [&](uint32_t dcol, uint32_t acol, uint64_t bhi, uint64_t blo, uint32_t id, uint32_t accum) {
                tf_mma(tbase + dcol, tbase + acol, bhi, id, accum);
                tf_mma(tbase + dcol, tbase + acol + 8, bhi, id, 1u);
                tf_mma(tbase + dcol, tbase + acol, blo, id, 1u);
            };
            constexpr uint32_t ID1 = G::idesc(NPAD), ID3 = G::idesc(3 * NPAD);
            bool ops_ready = false;
            uint32_t rc = 0;   // slabs consumed
            for (int i = 0;; ++i) {
                const int a = i & 1;
                const uint32_t ab = a * G::ACC;
                bool stop = false;
                for (int s = 0; s < G::NSLAB; ++s, ++rc) {
                    const int slot = rc & 3;
                    if (!tf_wait(&ring_full[slot], (rc >> 2) & 1, A.err, s_abort)) { stop = true; break; }
                    if (s == 0) {
                        // accumulator set a is free once the epilogue of tile i - 2 has read it
                        // (also before the end signal, so that no phase of acc_full[a] is skipped)
                        if (i >= 2 && !tf_wait(&acc_empty[a], ((i >> 1) + 1) & 1, A.err, s_abort)) { stop = true; break; }
                        if (s_tiles[i & 7] >= ntiles) {   // end: release the epilogue
                            mbar_arrive(&acc_full[a]);
                            mbar_arrive(&acc_full[a]);
                            stop = true;
                            break;
                        }
                        if (!ops_ready) {
                            if (!tf_wait(ops_bar, 0, A.err, s_abort)) { stop = true; break; }
                            ops_ready = true;
                        }
                    }
                    tc_fence_after();
                    const uint32_t rs = G::RING_COL + 32 * slot;
                    if (s < 2 * G::NKV) {
                        const int kv = s >> 1;
                        const uint32_t first = kv == 0 ? 0u : 1u;
                        if ((s & 1) == 0) {   // (P, F_r)
                            prod3(ab, rs, bdesc_d(ops_hi, kv, 0), bdesc_d(ops_lo, kv, 0), ID3, first);
                            prod3(ab + 3 * NPAD, rs + 16, bdesc_d(ops_hi, kv, 0), bdesc_d(ops_lo, kv, 0), ID1, first);
                        } else {              // (F_s, F_t)
                            prod3(ab + 3 * NPAD, rs, bdesc_d(ops_hi, kv, NPAD), bdesc_d(ops_lo, kv, NPAD), ID1, 1u);
                            prod3(ab + 3 * NPAD, rs + 16, bdesc_d(ops_hi, kv, 2 * NPAD), bdesc_d(ops_lo, kv, 2 * NPAD), ID1, 1u);
                        }
                    } else {                  // (XU, signed dP) of face f, K-step h
                        const int kl = s - 2 * G::NKV;
                        const int f = kl / G::NKF;
                        const uint64_t bh = bdesc_l(ops_hi, kl), bl = bdesc_l(ops_lo, kl);
                        prod3(ab + 3 * NPAD, rs, bh, bl, ID1, 1u);
                        if (f == 2) {
#pragma unroll
                            for (int j = 0; j < 3; ++j) prod3(ab + j * NPAD, rs + 16, bh, bl, ID1, 1u);
                        } else {
                            const int j = f == 0 ? 2 : f == 1 ? 1 : 0;   // f0: -t, f1: -s, f3: -r
                            prod3(ab + j * NPAD, rs + 16, bh, bl, ID1, 1u);
                        }
                    }
                    tc_commit(&ring_empty[slot]);
                }
                if (stop) break;
                tc_commit(&acc_full[a]);
                mbar_arrive(&acc_full[a]);
            }
        }
    } else if (w < 2 + G::NCONV) {
        // ------------------------------------------------------------ converters
        const int b = w & 3, hc = (w - 2) >> 2;   // 32-cell block; this warp's slabs are those of parity hc
        const uint32_t trow = tbase + ((uint32_t)(32 * b) << 16);
        for (int i = 0;; ++i) {
            const int st = i & 1;
            if (!tf_wait(&stage_full[st], (i >> 1) & 1, A.err, s_abort)) break;
            const int64_t t = s_tiles[i & 7];
            uint32_t rc = (uint32_t)i * G::NSLAB + hc;   // ring position of this warp's first slab of the tile
            if (t >= ntiles) {   // end: one empty slab (the tile's first) tells the MMA issuer
                if (hc == 0) {
                    const int slot = rc & 3;
                    if (rc >= 4 && !tf_wait(&ring_empty[slot], ((rc >> 2) + 1) & 1, A.err, s_abort)) break;
                    mbar_arrive(&ring_full[slot]);
                }
                break;
            }
            const int64_t gb = A.blk_begin + 4 * t + b;
            const bool valid = gb < A.blk_end;
            const float *sQ = stage_q(st) + b * QS;
            const float *sG = stage_g(st) + b * GS;
            const float2 *__restrict__ tb = reinterpret_cast<const float2 *>(A.tin) + (valid ? gb : 0) * (TI / 2);
            // this block's incoming traces are read from the first face slab on
            if (hc == 0 && valid && lane == 0) prefetch_l2(tb, TI * 4);
            // A block past the end of the launch range computes on whatever its stage
            // slot holds: its rows of the products are never read (each output row
            // depends on its own A row only) and its tensor-memory rows are not stored.
            float g[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) g[q] = sG[q * 32 + lane];
            const float Zm = sG[15 * 32 + lane];
            int cf[4];        // connectivity words (p = 0 faces)
#pragma unroll
            for (int f = 0; f < 4; ++f) cf[f] = A.conn[(valid ? gb : 0) * CS + f * 32 + lane];
            float2 tnxt[8];   // incoming traces of this warp's next face slab
            tf_load_tin<N>(tb, hc, lane, tnxt);
            bool bad = false;
            int prev_slot = -1;   // ring slot stored but not yet signalled
            for (int s = hc; s < G::NSLAB; s += 2, rc += 2) {
                uint32_t v[32];
                if (s < 2 * G::NKV) {
                    const int kv = s >> 1;
                    // (P, F_r) on even slabs, (F_s, F_t) on odd ones; K positions past the
                    // last node repeat it (zero operator rows there)
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int n = min(8 * kv + k, NP - 1);
                        const float u = sQ[(NP + n) * 32 + lane], vv = sQ[(2 * NP + n) * 32 + lane],
                                    ww = sQ[(3 * NP + n) * 32 + lane];
                        const float x0 = hc ? g[3] * u + g[4] * vv + g[5] * ww : sQ[n * 32 + lane];
                        const float x1 = hc ? g[6] * u + g[7] * vv + g[8] * ww : g[0] * u + g[1] * vv + g[2] * ww;
                        tf32_split(x0, v[k], v[8 + k]);
                        tf32_split(x1, v[16 + k], v[24 + k]);
                    }
                } else {
                    const int kl = s - 2 * G::NKV;
                    const int f = kl / G::NKF, h = kl - f * G::NKF;
                    float2 tcur[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) tcur[k] = tnxt[k];
                    if (kl + 2 < 4 * G::NKF) tf_load_tin<N>(tb, kl + 2, lane, tnxt);
                    float nx, ny, nz, fsc;
                    face_normal(g, f, nx, ny, nz, fsc);
                    const float zp = sG[(9 + f) * 32 + lane];
                    const int cc = f == 0 ? cf[0] : f == 1 ? cf[1] : f == 2 ? cf[2] : cf[3];
                    const bool dir = cc < 0 && cc != kPadConn && ((-1 - cc) & 1);
                    const float izs = 1.0f / (Zm + zp);
                    const float wm = Zm * izs, zz = Zm * zp * izs;
                    const float sgn = f == 2 ? 1.f : -1.f;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int m = min(8 * h + k, NFP - 1);   // past the last face node: repeat it
                        const int n = sFm[f * NFP + m];
                        const float pm = sQ[n * 32 + lane];
                        const float unm = nx * sQ[(NP + n) * 32 + lane] + ny * sQ[(2 * NP + n) * 32 + lane] +
                                          nz * sQ[(3 * NP + n) * 32 + lane];
                        const float pp = dir ? -pm : tcur[k].x, unp = dir ? unm : tcur[k].y;   // p = 0 face: mirror state
                        const float dP = wm * (pp - pm) + zz * (unm - unp);
                        const float dUn = (1.0f - wm) * (unp - unm) + izs * (pm - pp);
                        tf32_split(fsc * dUn, v[k], v[8 + k]);
                        tf32_split(sgn * dP, v[16 + k], v[24 + k]);
                    }
                    // the epilogue of this tile reads res after the products; request it now
                    if (kl == 0 && valid && lane == 0) prefetch_l2(A.res + gb * QS, QS * 4);
                }
                if (s + 2 >= G::NSLAB) mbar_arrive(&stage_empty[st]);   // this warp's last read of the stage
                // the previous slab's store has had this slab's arithmetic to complete
                if (prev_slot >= 0) {
                    if (valid) tmem_wait_st();
                    tc_fence_before();
                    mbar_arrive(&ring_full[prev_slot]);
                }
                const int slot = rc & 3;
                if (rc >= 4 && !tf_wait(&ring_empty[slot], ((rc >> 2) + 1) & 1, A.err, s_abort)) { bad = true; break; }
                tc_fence_after();
                if (valid) tmem_st32(trow + G::RING_COL + 32 * slot, v);
                prev_slot = slot;
            }
            if (bad) break;
            if (valid) tmem_wait_st();   // the warp's last slab of the tile
            tc_fence_before();
            mbar_arrive(&ring_full[prev_slot]);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int b = w & 3, h = (w - 2 - G::NCONV) >> 2;   // 32-cell block; this warp's half of the work
        const uint32_t trow = tbase + ((uint32_t)(32 * b) << 16);
        double tstage = 0.0;
        if (A.src.n > 0) tstage = sc.time[0] + sc.c_dt;
        for (int i = 0;; ++i) {
            const int a = i & 1, st = i & 1;
            if (!tf_wait(&acc_full[a], (i >> 1) & 1, A.err, s_abort)) break;
            const int64_t t = s_tiles[i & 7];
            if (t >= ntiles) break;
            tc_fence_after();
            // the stage of tile i (complete since its converters ran; held until this arrival)
            if (!tf_wait(&stage_full[st], (i >> 1) & 1, A.err, s_abort)) break;
            const int64_t gb = A.blk_begin + 4 * t + b;
            const bool valid = gb < A.blk_end;
            float *sQw = stage_q(st) + b * QS;   // old state in; the new state is written over it
            const float *sG = stage_g(st) + b * GS;
            float g[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) g[q] = sG[q * 32 + lane];
            if (valid) {
                // ---- update: NC-node chunks, this warp every other one; res of the warp's
                // next chunk is requested before the current chunk is processed
                const float rc2 = sG[13 * 32 + lane], irho = sG[14 * 32 + lane];
                const int64_t kcell = gb * 32 + lane;
                bool has_src = false;
                for (int si = 0; si < A.src.n; ++si) has_src |= A.src.cell[si] == kcell;
                float *__restrict__ qg = A.q + gb * QS;
                float *__restrict__ rg = A.res + gb * QS;
                const uint32_t tacc = trow + a * G::ACC;
                constexpr int NC = 2;
                constexpr int NCH = (NP + NC - 1) / NC;
                float rcur[NC][4], rnxt[NC][4];
                auto load_res = [&](int j, float (&rv)[NC][4]) {   // past the last node: repeat it (unused)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int n = min(NC * j + c, NP - 1);
#pragma unroll
                        for (int fl = 0; fl < 4; ++fl) rv[c][fl] = rg[(fl * NP + n) * 32 + lane];
                    }
                };
                if (h < NCH) load_res(h, rnxt);
#pragma unroll 1
                for (int j = h; j < NCH; j += 2) {
#pragma unroll
                    for (int c = 0; c < NC; ++c)
#pragma unroll
                        for (int fl = 0; fl < 4; ++fl) rcur[c][fl] = rnxt[c][fl];
                    if (j + 2 < NCH) load_res(j + 2, rnxt);
                    float ar[NC], as_[NC], at[NC], adv[NC];
                    tmem_ld2(tacc + NC * j, ar);
                    tmem_ld2(tacc + NPAD + NC * j, as_);
                    tmem_ld2(tacc + 2 * NPAD + NC * j, at);
                    tmem_ld2(tacc + 3 * NPAD + NC * j, adv);
                    tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int n = NC * j + c;
                        if (n >= NP) break;
                        float rhs[4];
                        rhs[0] = -rc2 * adv[c];
                        rhs[1] = -irho * (g[0] * ar[c] + g[3] * as_[c] + g[6] * at[c]);
                        rhs[2] = -irho * (g[1] * ar[c] + g[4] * as_[c] + g[7] * at[c]);
                        rhs[3] = -irho * (g[2] * ar[c] + g[5] * as_[c] + g[8] * at[c]);
                        if (has_src)
                            for (int si = 0; si < A.src.n; ++si)
                                if (A.src.cell[si] == kcell)
                                    rhs[0] += (float)(A.src.amp[si] * ricker_integral_d(tstage, A.src.f_peak[si], A.src.t_s[si])) *
                                              A.src.vec[si * NP + n];
#pragma unroll
                        for (int fl = 0; fl < 4; ++fl) {
                            const int idx = (fl * NP + n) * 32 + lane;
                            const float r = sc.a * rcur[c][fl] + sc.dt * rhs[fl];
                            rg[idx] = r;
                            const float qn = sQw[idx] + sc.b * r;
                            qg[idx] = qn;
                            sQw[idx] = qn;
                        }
                    }
                }
            }
            // the accumulators of tile i are read: the products of tile i + 2 may start
            tc_fence_before();
            mbar_arrive(&acc_empty[a]);
            if (valid) {
                // both epilogue warps of this block have written their nodes' new state
                asm volatile("bar.sync %0, %1;" ::"r"(1 + b), "r"(64) : "memory");
                // ---- new traces, face by face (this warp: faces 2h and 2h + 1), read from the stage
#pragma unroll 1
                for (int ff = 0; ff < 2; ++ff) {
                    const int f = 2 * h + ff;
                    const int cc = A.conn[gb * CS + f * 32 + lane];
                    if (cc == kPadConn) continue;
                    float nx, ny, nz, fs_unused;
                    face_normal(g, f, nx, ny, nz, fs_unused);
                    // neighbour face (k', f'): float2 slot of (k', f', node 0) and its node order;
                    // boundary face: own trace for the face HABC solver
                    const bool inner = cc >= 0;
                    const int nb = cc >> 3;
                    const int64_t kn = nb >> 2;
                    const int64_t base = inner ? (((kn >> 5) * 4 + (nb & 3)) * NFP) * 32 + (kn & 31) : 0;
                    const int pofs = (cc & 7) * NFP;
                    const int64_t bf = inner ? 0 : (-1 - cc) >> 1;
                    const bool ok = inner ? DGH_IN_RANGE(A.err, kn, A.kcells) : DGH_IN_RANGE(A.err, bf, A.nbfaces);
                    float *__restrict__ tb = A.trb + bf * 2 * NFP;
                    float2 *__restrict__ tout = reinterpret_cast<float2 *>(A.tout);
#pragma unroll
                    for (int m = 0; m < NFP; ++m) {
                        const int n = sFm[f * NFP + m];
                        const float p = sQw[n * 32 + lane];
                        const float un = nx * sQw[(NP + n) * 32 + lane] + ny * sQw[(2 * NP + n) * 32 + lane] +
                                         nz * sQw[(3 * NP + n) * 32 + lane];
                        if (ok) {
                            if (inner) {
                                tout[base + sFp[pofs + m] * 32] = make_float2(p, -un);
                            } else {
                                tb[m] = p;
                                tb[NFP + m] = un;
                            }
                        }
                    }
                }
            }
            // the stage was written through the generic proxy; the next copy into it is a TMA write
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&stage_empty[st]);
        }
    }

    // ---------------------------------------------------------------- drain
    __syncthreads();
    if (tid == 32) {   // every product issued by this thread has completed
        tc_commit(fin_bar);
        mbar_wait(fin_bar, 0, A.err);
    }
    if (tid == 0) {    // no bulk copy may still target shared memory
        mbar_wait(ops_bar, 0, A.err);
        // After an abort the last two stage copies may still be in flight: each
        // completes the barrier phase of its iteration (no later phase of its
        // stage was started).  In a normal run the converters consumed them
        // before the end was signalled.
        if (!reached_end)
            for (int j = last_issued - 1; j <= last_issued; ++j)
                if (j >= 0) mbar_wait(&stage_full[j & 1], (j >> 1) & 1, A.err);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
}

}  // namespace dgh
