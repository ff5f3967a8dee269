// Device kernels of one LSERK4 stage of the multidimensional DG + HABC solver.
//
// Per stage (Algorithm 1, with the volume/surface/update work of each level
// fused into one kernel):
//   k3d_stage  3D volume term, upwind surface flux + lift, LSERK update, new
//              3D traces (Sec. 3.2, eq. dgLocalRhs, eqs. timeStepProc1-2)
//   k2d_stage  2D face systems (eqs. proc:2Dpvsyst1-3) for all P sets, then
//              the face BC: r^+_3D from the new 3D traces, r^-_3D =
//              (1/M) sum c_a p*_a (eq. proc:faceBC), q0 = r^- + r^+,
//              p_a = p*_a + q0 (eq. proc:pi00Star), new 2D traces
//   k1d_stage  1D edge systems (eqs. proc:1Dpvsyst1-2) for all P^2 sets, then
//              the edge BCs (eqs. proc:edgeBC1-2) through the precomputed
//              solution operator, p_ab (eq. proc:pij0Star), new 1D traces
//   k0d_stage  corner BCs (eqs. proc:cornerBC1-3) through the precomputed
//              solution operator
// Traces are double-buffered (read tr_in, write tr_out); q and res are
// updated in place because cells only read their neighbours' traces.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgh {

template <int N>
struct Ord {
    static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6;
    static constexpr int NFP = (N + 1) * (N + 2) / 2;
    static constexpr int NP2 = (N + 1) * (N + 2) / 2;
    static constexpr int NFP2 = N + 1;
    static constexpr int NP1 = N + 1;
};

constexpr int GEO2 = 28;   // per tri: drdx[4], 3 x (nx,ny,fscale,wm,zz,iz), rho c^2, 1/rho, Z, pad[3]
constexpr int GEO1 = 16;   // per line: rx, fscale, rho c^2, 1/rho, Z, ZA, ZB, 2 x (wm,zz,iz), pad[3]
constexpr int MAXP = 12;
constexpr int MAXSRC = 64;

// Checked build (compiled with -DDGH_CHECKED): every index that a stage
// kernel gathers through or pushes to is tested against its array; a
// violation writes 2 into the device error word and the access is skipped
// (the host reports DGH_EBOUNDS).  In the normal build the test is compiled
// out.  This stands in for a memory checker that this platform lacks.
#ifdef DGH_CHECKED
__device__ __forceinline__ bool in_range_checked(int *err, int64_t i, int64_t n) {
    if (i >= 0 && i < n) return true;
    if (err) atomicExch(err, 2);
    return false;
}
#define DGH_IN_RANGE(err, i, n) ::dgh::in_range_checked((err), (int64_t)(i), (int64_t)(n))
#else
#define DGH_IN_RANGE(err, i, n) true
#endif

struct SrcParams {
    int n;
    int64_t cell[MAXSRC];
    double f_peak[MAXSRC], t_s[MAXSRC], amp[MAXSRC];
    const float *vec;       // [MAXSRC][Np]
};

struct StageCoef {
    float a, b, dt;
    double c_dt;            // C_s * dt (stage time offset)
    const double *time;     // device: time at the start of the step
};

struct Args2 {
    float *q, *res;         // [T][P][3][Np2]
    const float *tr_in;     // [T][P][3][2][Nfp2]
    float *tr_out;
    const float *geo;       // [T][GEO2]
    const int *conn;        // >=0: (t'*3+e')<<1 | flip ; -1: HABC edge (qb2) ; -2: Dirichlet edge
    const float *qb;        // [T][3][P][Nfp2]  incoming 2D characteristic at domain-edge nodes
    float *q0;              // [T][Np2]         r^- + r^+ of the 3D field at the triangle nodes
    float *tin3;            // out: 3D incoming traces [K32][4][Nfp][32][2], exterior state (2 r^-, 0); NULL: not written
    float *feat;            // out (optional): closure features per triangle node [T][Np2][6]
    float *rm_out;          // out (optional): r^- per triangle node [T][Np2]
    const float *trb;       // own 3D traces of the boundary faces [Fb][2][Nfp]
    const int *tri_face;    // [T] global face id k*4+f of the owning tet face
    const int *tri_bface;   // [T] boundary face index
    const float *D;         // [2][Np2(m)][Np2(n)]
    const float *LIFT;      // [3Nfp2][Np2]
    const int *fmask;       // [3][Nfp2]
    const float *cP;        // [P] Pade coefficients
    float invM;
    int P;
    int64_t T;
    int *err;               // device error word (checked build)
    int64_t kcells, nbfaces;   // bounds of tri_face cells and tri_bface (checked build)
    unsigned *tile_ctr;     // [2]: tiles claimed, CTAs done; zero at launch, reset to zero by the last CTA
};

struct Args1 {
    float *q, *res;         // [L][P^2][2][Np1]
    const float *tr_in;     // [L][P^2][2 ends][2]
    float *tr_out;
    const float *geo;       // [L][GEO1]
    const int *conn;        // [L][2] >=0: l'*2+e' ; -1: HABC corner (qb1) ; -2: Dirichlet corner
    const float *qb;        // [L][2][P^2]  incoming 1D characteristic at corner ends
    float *q0;              // [L][2][P][Np1] r^- + r^+ of the 2D fields of faces A, B at the line nodes
    float *qb2;             // out: incoming 2D characteristic [T][3][P][Nfp2]
    const float *tr2;       // new 2D traces [T][P][3][2][Nfp2]
    const int *lmap;        // [L][6]: triA, edgeA, revA, triB, edgeB, revB
    const float *D;         // [Np1(m)][Np1(n)]
    const float *LIFT;      // [2][Np1]
    const float *H1;        // [2P][2P]
    const float *H2;        // [2P][P^2]
    const float *cP;
    float invM;
    int P;
    int64_t L;
    int *err;               // device error word (checked build)
    int64_t T;              // bound of the triangle ids in lmap (checked build)
};

struct Args0 {
    const float *tr1;       // new 1D traces
    float *qb1;             // [L][2][P^2]
    const int *corner;      // [C][6]: (line, end) x 3 slots (YZ, XZ, XY)
    const float *cornerZ;   // [C][3]
    const float *Hc;        // [3P^2][3P^2]
    int P;
    int C;
    int *err;               // device error word (checked build)
    int64_t L;              // bound of the line ids in corner (checked build)
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double ricker_integral_d(double t, double f, double ts) {
    const double a = 3.14159265358979323846 * f * (t - ts);
    return (t - ts) * exp(-a * a);
}

}  // namespace dgh
#include "k3d.cuh"
#include "k3d_tc.cuh"
#include "k3d_tf32.cuh"
#include "closure.cuh"
namespace dgh {

// ==================================================================== 2D
// One thread per (triangle, set) item: its p*, v1, v2 at the NP2 nodes live in
// registers, the volume and lift operators are read as broadcast float4 rows
// from shared memory, and every global array of a tile (fields, residuals,
// traces) is a contiguous block moved by the whole CTA with 16-byte
// asynchronous copies / vector stores.  A CTA handles tile_tris triangles at a
// time (tile_tris * P <= blockDim.x).
// Small-integer division s / P for s < 2^12, P <= 12: the fractional part of
// (s + 0.5) / P lies in [0.5 / P, 1 - 0.5 / P], far from the float rounding.
__device__ __forceinline__ int div_small(int s, float inv) { return __float2int_rz((float(s) + 0.5f) * inv); }

// Asynchronous global -> shared copies (no register round trip): a tile's
// loads are all in flight at once; cp_async_wait_all before the barrier.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copies g[start, start + count) to s[sh, sh + count), sh = start mod 4, so
// that global and shared addresses agree mod 16 bytes and the body moves
// float4s (s is 16-byte aligned, with 4 floats of slack).  Returns sh.
__device__ __forceinline__ int block_load_async(float *s, const float *g, int64_t start, int count, int tid, int nth) {
    const int sh = (int)(start & 3);
    const int head = min(count, (4 - sh) & 3);
    const int body = (count - head) >> 2;
    const int tail = count - head - 4 * body;
    float *d = s + sh;
    const float *src = g + start;
    if (tid < head) cp_async4(d + tid, src + tid);
    for (int i = tid; i < body; i += nth) cp_async16(d + head + 4 * i, src + head + 4 * i);
    if (tid < tail) cp_async4(d + head + 4 * body + tid, src + head + 4 * body + tid);
    return sh;
}

// The reverse of block_load_async: s[sh, sh + count) -> g[start, ...).
__device__ __forceinline__ void block_store(float *g, const float *s, int64_t start, int count, int tid, int nth) {
    const int sh = (int)(start & 3);
    const int head = min(count, (4 - sh) & 3);
    const int body = (count - head) >> 2;
    const int tail = count - head - 4 * body;
    const float *src = s + sh;
    float *d = g + start;
    if (tid < head) d[tid] = src[tid];
    for (int i = tid; i < body; i += nth)
        *reinterpret_cast<float4 *>(d + head + 4 * i) = *reinterpret_cast<const float4 *>(src + head + 4 * i);
    if (tid < tail) d[head + 4 * body + tid] = src[head + 4 * body + tid];
}

template <int N>
struct Cfg2 {
    static constexpr int NP2 = Ord<N>::NP2, NFP2 = Ord<N>::NFP2, NE = 3 * NFP2;
    static constexpr int NPP = (NP2 + 3) / 4 * 4;   // operator rows padded to float4
    static constexpr int NEP = (NE + 3) / 4 * 4;
    static constexpr int F = 3 * NP2;                 // (p*, v1, v2) of one item
    static constexpr int TR = 6 * NFP2;               // traces of one item: [3 edges][p, v.n][Nfp2]
};

// Shared-memory carve-up of k2d_stage (float offsets; every array 16-byte aligned).
struct Smem2 {
    int dt, lt, cp, q, res, g, q0, trb, r, face, fm, total;
    __host__ __device__ Smem2(int NP2, int NFP2, int P, int tile) {
        auto al = [](int x) { return (x + 3) & ~3; };
        const int NE = 3 * NFP2, NPP = al(NP2), NEP = al(NE), F = 3 * NP2;
        dt = 0;
        lt = dt + 2 * NP2 * NPP;
        cp = lt + NP2 * NEP;
        q = cp + 2 * 16;                       // c_a (a < MAXP), the claimed tile, 1 / (1 + c_a)
        res = q + al(tile * P * F + 4);
        g = res + al(tile * P * F + 4);
        q0 = g + tile * GEO2;
        trb = q0 + al(tile * NP2 + 4);
        r = trb + al(tile * 2 * NP2);
        face = r + al(tile * 2 * NP2);
        fm = face + al(tile);
        total = fm + al(NE);
    }
};

template <int N, bool UPDATE>
__global__ void __launch_bounds__(256) k2d_stage(Args2 A, StageCoef sc, int tile_tris) {
    using C = Cfg2<N>;
    constexpr int NP2 = C::NP2, NFP2 = C::NFP2, NE = C::NE, NPP = C::NPP, NEP = C::NEP, F = C::F, TR = C::TR;
    const int P = A.P;
    const float invP = 1.0f / float(P);
    extern __shared__ float4 sm4[];
    float *sm = reinterpret_cast<float *>(sm4);
    const Smem2 L(NP2, NFP2, P, tile_tris);
    float *sDT = sm + L.dt;                           // [2][n][m]: D[d][m][n] (output row n)
    float *sLT = sm + L.lt;                           // [n][em]: LIFT[em][n]
    float *scp = sm + L.cp;                           // c_a, then 1 / (1 + c_a)
    float *sqb = sm + L.q;                            // fields of the tile (+ alignment shift), updated in place
    float *srb = sm + L.res;                          // residuals of the tile (same shift), updated in place
    float *sg = sm + L.g;                             // tile*GEO2
    float *s0b = sm + L.q0;                           // q0 (+ shift)
    float *strb = sm + L.trb;                         // tile*2*NP2 own 3D traces of the triangle
    float *sr = sm + L.r;                             // tile*2*NP2 dp*/dt of sets 0, 1 (closure features)
    int *sface = reinterpret_cast<int *>(sm + L.face);
    int *sfm = reinterpret_cast<int *>(sm + L.fm);
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = (nth + 31) >> 5;
    if (UPDATE) {
        for (int i = tid; i < 2 * NP2 * NPP; i += nth) {
            const int d = i / (NP2 * NPP), r = i % (NP2 * NPP), n = r / NPP, m = r % NPP;
            sDT[i] = m < NP2 ? A.D[(d * NP2 + m) * NP2 + n] : 0.f;
        }
        for (int i = tid; i < NP2 * NEP; i += nth) {
            const int n = i / NEP, em = i % NEP;
            sLT[i] = em < NE ? A.LIFT[em * NP2 + n] : 0.f;
        }
    }
    for (int i = tid; i < P; i += nth) {
        scp[i] = A.cP[i];
        scp[16 + i] = 1.0f / (1.0f + A.cP[i]);
    }
    for (int i = tid; i < NE; i += nth) sfm[i] = A.fmask[i];
    const int64_t ntiles = (A.T + tile_tris - 1) / tile_tris;
    // Tiles are claimed from a device counter: a CTA that finishes early takes
    // the next tile, so the CTAs of an SM drift out of step (one loads while
    // another computes) and the last tiles spread over all CTAs.
    volatile unsigned *s_tile = reinterpret_cast<unsigned *>(scp + MAXP);   // a free word after c_a
    for (;;) {
        if (tid == 0) *s_tile = atomicAdd(&A.tile_ctr[0], 1u);
        __syncthreads();   // also: the previous tile's shared-memory reads are done
        const int64_t tile = *s_tile;
        if (tile >= ntiles) break;
        const int64_t t0 = tile * tile_tris;
        const int nt = (int)((A.T - t0) < tile_tris ? (A.T - t0) : tile_tris);
        const int nitem = nt * P;
        // every global input of the tile in one phase: contiguous blocks by the
        // whole CTA, the exterior states at the edge nodes by each item thread
        const int shq = block_load_async(sqb, A.q, t0 * P * F, nitem * F, tid, nth);
        if (UPDATE) block_load_async(srb, A.res, t0 * P * F, nitem * F, tid, nth);
        const int sh0 = block_load_async(s0b, A.q0, t0 * NP2, nt * NP2, tid, nth);
        block_load_async(sg, A.geo, t0 * GEO2, nt * GEO2, tid, nth);   // GEO2 = 28: no shift
        if (A.tin3 && tid < nt) cp_async4(sface + tid, A.tri_face + t0 + tid);
        for (int i = tid; i < nt * 2 * NP2; i += nth) {
            const int t = i / (2 * NP2), r = i % (2 * NP2);
            const int bf = A.tri_bface[t0 + t];
            if (DGH_IN_RANGE(A.err, bf, A.nbfaces)) cp_async4(strb + i, A.trb + (int64_t)bf * 2 * NP2 + r);
        }
        float *sq = sqb + shq, *sres = srb + shq, *s0 = s0b + sh0;
        const bool act = tid < nitem;
        const int t = act ? div_small(tid, invP) : 0, a = tid - t * P;
        float xp[NE], xv[NE];   // exterior (p, v.n) at the edge nodes
        int ce[3];
        if (UPDATE && act) {
            const int64_t tg = t0 + t;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const int c = A.conn[tg * 3 + e];
                ce[e] = c;
                if (c >= 0) {
                    const int nb = c >> 1, tn0 = nb / 3, en = nb - 3 * tn0;
                    const int tn = DGH_IN_RANGE(A.err, tn0, A.T) ? tn0 : 0;
                    const float *tr = A.tr_in + (((int64_t)tn * P + a) * 3 + en) * 2 * NFP2;
#pragma unroll
                    for (int m = 0; m < NFP2; ++m) {
                        const int mm = (c & 1) ? (NFP2 - 1 - m) : m;
                        xp[e * NFP2 + m] = tr[mm];
                        xv[e * NFP2 + m] = -tr[NFP2 + mm];
                    }
                } else {
                    const float *qb = A.qb + ((tg * 3 + e) * P + a) * NFP2;
#pragma unroll
                    for (int m = 0; m < NFP2; ++m) {
                        xp[e * NFP2 + m] = c != -2 ? 2.0f * qb[m] : 0.f;
                        xv[e * NFP2 + m] = 0.f;
                    }
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
        if (UPDATE && act) {
            const float *g = sg + t * GEO2;
            float *qa = sq + tid * F;
            float *ra = sres + tid * F;
            const float *q0t = s0 + t * NP2;
            float p[NP2], w1[NP2], w2[NP2];
            const float g0 = g[0], g1 = g[1], g2 = g[2], g3 = g[3];
#pragma unroll
            for (int n = 0; n < NP2; ++n) {
                p[n] = qa[n] + q0t[n];
                const float v1 = qa[NP2 + n], v2 = qa[2 * NP2 + n];
                w1[n] = g0 * v1 + g1 * v2;
                w2[n] = g2 * v1 + g3 * v2;
            }
            // upwind flux differences at the edge nodes, scaled by the edge Fscale
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const float nx = g[4 + 6 * e], ny = g[5 + 6 * e], fs = g[6 + 6 * e];
                const float wm = g[7 + 6 * e], zz = g[8 + 6 * e], iz = g[9 + 6 * e];
#pragma unroll
                for (int m = 0; m < NFP2; ++m) {
                    const int em = e * NFP2 + m, n = sfm[em];
                    const float pm = qa[n] + q0t[n];
                    const float vnm = nx * qa[NP2 + n] + ny * qa[2 * NP2 + n];
                    float pp = xp[em], vnp = xv[em];
                    if (ce[e] == -2) {   // p = 0 edge: mirror state
                        pp = -pm;
                        vnp = vnm;
                    }
                    const float dP = wm * (pp - pm) + zz * (vnm - vnp);
                    const float dVn = (1.0f - wm) * (vnp - vnm) + iz * (pm - pp);
                    xv[em] = fs * dVn;
                    xp[em] = fs * dP;
                }
            }
            const float rc2 = g[22], irho = g[23];
            const float cw = -rc2 * scp[16 + a];
            const float nx0 = g[4], ny0 = g[5], nx1 = g[10], ny1 = g[11], nx2 = g[16], ny2 = g[17];
#pragma unroll 1
            for (int n = 0; n < NP2; ++n) {
                const float4 *dr4 = reinterpret_cast<const float4 *>(sDT + n * NPP);
                const float4 *ds4 = reinterpret_cast<const float4 *>(sDT + (NP2 + n) * NPP);
                float div = 0.f, dpr = 0.f, dps = 0.f;
#pragma unroll
                for (int k = 0; k < NPP / 4; ++k) {
                    const float4 r4 = dr4[k], s4 = ds4[k];
                    const float rv[4] = {r4.x, r4.y, r4.z, r4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int m = 4 * k + j;
                        if (m < NP2) {
                            div += rv[j] * w1[m] + sv[j] * w2[m];
                            dpr += rv[j] * p[m];
                            dps += sv[j] * p[m];
                        }
                    }
                }
                const float4 *l4 = reinterpret_cast<const float4 *>(sLT + n * NEP);
                float lvn = 0.f, lp0 = 0.f, lp1 = 0.f, lp2 = 0.f;
#pragma unroll
                for (int k = 0; k < NEP / 4; ++k) {
                    const float4 L4 = l4[k];
                    const float lv[4] = {L4.x, L4.y, L4.z, L4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int em = 4 * k + j;
                        if (em < NE) {
                            lvn += lv[j] * xv[em];
                            if (em < NFP2) lp0 += lv[j] * xp[em];
                            else if (em < 2 * NFP2) lp1 += lv[j] * xp[em];
                            else lp2 += lv[j] * xp[em];
                        }
                    }
                }
                float rhs[3];
                rhs[0] = cw * (div + lvn);
                rhs[1] = -irho * (g0 * dpr + g2 * dps + nx0 * lp0 + nx1 * lp1 + nx2 * lp2);
                rhs[2] = -irho * (g1 * dpr + g3 * dps + ny0 * lp0 + ny1 * lp1 + ny2 * lp2);
                if (a < 2) sr[t * 2 * NP2 + a * NP2 + n] = rhs[0];
#pragma unroll
                for (int fl = 0; fl < 3; ++fl) {
                    const float rr = sc.a * ra[fl * NP2 + n] + sc.dt * rhs[fl];
                    ra[fl * NP2 + n] = rr;
                    qa[fl * NP2 + n] += sc.b * rr;
                }
            }
        }
        __syncthreads();
        // face BC: r^+ from the new 3D traces, r^- = (1/M) sum c_a p*_a, q0 = r^- + r^+
        for (int i = tid; i < nt * NP2; i += nth) {
            const int tt = i / NP2, n = i % NP2;
            const int64_t tg = t0 + tt;
            const float *tr = strb + tt * 2 * NP2;   // own tet face traces (Nfp == Np2)
            const float Z = sg[tt * GEO2 + 24];
            const float rp = 0.5f * (tr[n] + Z * tr[NP2 + n]);
            float rm = 0.f;
            const float *qn = sq + tt * P * F + n;
#pragma unroll
            for (int b = 0; b < MAXP; ++b)
                if (b < P) rm += scp[b] * qn[b * F];
            rm *= A.invM;
            if (A.tin3) {
                const int64_t gf = sface[tt], kc = gf >> 2;
                const int fc = (int)(gf & 3);
                if (DGH_IN_RANGE(A.err, kc, A.kcells))
                    A.tin3[((((kc >> 5) * 4 + fc) * NP2 + n) * 32 + (kc & 31)) * 2] = 2.0f * rm;   // exterior p; n.u = 0
            }
            const float q0 = rm + rp;
            if (A.rm_out) A.rm_out[tg * NP2 + n] = rm;
            if (A.feat) {   // (p, n.u, p_1, p_2, dp*_1/dt, dp*_2/dt) at this face node
                float *f = A.feat + (tg * NP2 + n) * 6;
                f[0] = tr[n];
                f[1] = tr[NP2 + n];
                f[2] = P >= 1 ? sq[(tt * P + 0) * F + n] + q0 : 0.f;
                f[3] = P >= 2 ? sq[(tt * P + 1) * F + n] + q0 : 0.f;
                f[4] = (UPDATE && P >= 1) ? sr[tt * 2 * NP2 + n] : 0.f;
                f[5] = (UPDATE && P >= 2) ? sr[tt * 2 * NP2 + NP2 + n] : 0.f;
            }
            s0[tt * NP2 + n] = q0;
        }
        __syncthreads();
        // write-back: fields, residuals and q0 (contiguous blocks), new 2D
        // traces (full pressure, in-plane normal velocity), one warp per item
        // over its contiguous [3][2][Nfp2] block
        if (UPDATE) {
            block_store(A.q, sqb, t0 * P * F, nitem * F, tid, nth);
            block_store(A.res, srb, t0 * P * F, nitem * F, tid, nth);
        }
        block_store(A.q0, s0b, t0 * NP2, nt * NP2, tid, nth);
        for (int r = lane; r < TR; r += 32) {   // lane-constant part of the trace slot r
            const int e = r / (2 * NFP2), k = r % (2 * NFP2), isp = k < NFP2;
            const int n = sfm[e * NFP2 + (isp ? k : k - NFP2)];
            const float *ge = sg + 4 + 6 * e;
            float *gt = A.tr_out + t0 * P * TR + r;
            for (int s = warp; s < nitem; s += nwarp) {
                const int tt = div_small(s, invP);
                const float *qa = sq + s * F + n;
                gt[s * TR] = isp ? qa[0] + s0[tt * NP2 + n] : ge[tt * GEO2] * qa[NP2] + ge[tt * GEO2 + 1] * qa[2 * NP2];
            }
        }
    }
    // the last CTA to finish leaves the counters at zero for the next launch
    // (every CTA has made its last claim before it counts itself done)
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&A.tile_ctr[1], 1u) == gridDim.x - 1) {
            atomicExch(&A.tile_ctr[0], 0u);
            atomicExch(&A.tile_ctr[1], 0u);
        }
    }
}

inline size_t k2d_smem(int N, int P, int tile) {
    return sizeof(float) * (size_t)Smem2((N + 1) * (N + 2) / 2, N + 1, P, tile).total;
}

// Triangles per CTA of the 2D kernel: one thread per (triangle, set).
inline int k2d_tile_max(int P, int thr) { return P > 0 ? (thr / P > 0 ? thr / P : 1) : 1; }

// ==================================================================== 1D
template <int N, bool UPDATE>
__global__ void __launch_bounds__(256) k1d_stage(Args1 A, StageCoef sc, int tile_lines) {
    constexpr int NP1 = N + 1;
    const int P = A.P, S = P * P;
    extern __shared__ float sm[];
    float *sD = sm;                                   // NP1*NP1
    float *sL = sD + NP1 * NP1;                       // 2*NP1
    float *sq = sL + 2 * NP1;                         // tile*S*2*NP1
    float *sp = sq + tile_lines * S * 2 * NP1;        // tile*S*NP1 full p
    float *sx = sp + tile_lines * S * NP1;            // tile*S*2*2
    float *s0 = sx + tile_lines * S * 4;              // tile*2*P*NP1
    float *sg = s0 + tile_lines * 2 * P * NP1;        // tile*GEO1
    float *sn = sg + tile_lines * GEO1;               // tile*S*2*NP1 new (p*, w)
    float *sH = sn + tile_lines * S * 2 * NP1;        // 2P*2P + 2P*S
    float *srp = sH + 4 * P * P + 2 * P * S;          // tile*NP1*2P  r^+ of the 2D fields of faces A, B
    float *sres = srp + tile_lines * NP1 * 2 * P;     // tile*S*2*NP1 residuals (update only)
    float *sxe = sres + tile_lines * S * 2 * NP1;     // tile*S*2*2   exterior (p, w.n) at the two ends (update only)
    int *smp = reinterpret_cast<int *>(sxe + tile_lines * S * 4);   // tile*6 line map
    int *scn = smp + tile_lines * 6;                  // tile*2 end connectivity
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < NP1 * NP1; i += nth) sD[i] = A.D[i];
    for (int i = tid; i < 2 * NP1; i += nth) sL[i] = A.LIFT[i];
    for (int i = tid; i < 4 * P * P; i += nth) sH[i] = A.H1[i];
    for (int i = tid; i < 2 * P * S; i += nth) sH[4 * P * P + i] = A.H2[i];
    const int64_t ntiles = (A.L + tile_lines - 1) / tile_lines;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t l0 = tile * tile_lines;
        const int nl = (int)((A.L - l0) < tile_lines ? (A.L - l0) : tile_lines);
        __syncthreads();
        for (int i = tid; i < nl * S * 2 * NP1; i += nth) sq[i] = A.q[l0 * S * 2 * NP1 + i];
        for (int i = tid; i < nl * 2 * P * NP1; i += nth) s0[i] = A.q0[l0 * 2 * P * NP1 + i];
        for (int i = tid; i < nl * GEO1; i += nth) sg[i] = A.geo[l0 * GEO1 + i];
        for (int i = tid; i < nl * 6; i += nth) smp[i] = A.lmap[l0 * 6 + i];
        if (UPDATE) {
            for (int i = tid; i < nl * S * 2 * NP1; i += nth) sres[i] = A.res[l0 * S * 2 * NP1 + i];
            for (int i = tid; i < nl * 2; i += nth) scn[i] = A.conn[l0 * 2 + i];
        }
        __syncthreads();
        // gathers through the index arrays (one more memory round trip): r^+ of
        // the faces' new 2D traces at the line nodes, exterior states at the ends
        for (int i = tid; i < nl * NP1 * 2 * P; i += nth) {
            const int l = i / (NP1 * 2 * P), r = i % (NP1 * 2 * P), n = r / (2 * P), j = r % (2 * P);
            const int side = j >= P, a = j - side * P;
            const int *mp = smp + l * 6 + 3 * side;
            const int m = mp[2] ? (N - n) : n;
            const float Z = sg[l * GEO1 + 5 + side];
            const int tri = DGH_IN_RANGE(A.err, mp[0], A.T) ? mp[0] : 0;
            const float *tr = A.tr2 + (((int64_t)tri * P + a) * 3 + mp[1]) * 2 * NP1;
            srp[i] = 0.5f * (tr[m] + Z * tr[NP1 + m]);
        }
        if (UPDATE)
            for (int i = tid; i < nl * S * 2; i += nth) {
                const int l = i / (S * 2), r = i % (S * 2), s2 = r / 2, e = r % 2;
                const int c = scn[l * 2 + e];
                float pp = 0.f, wnp = 0.f;
                if (c >= 0 && DGH_IN_RANGE(A.err, c >> 1, A.L)) {
                    const float *tr = A.tr_in + ((int64_t)(c >> 1) * S + s2) * 4 + (c & 1) * 2;
                    pp = tr[0];
                    wnp = -tr[1];
                } else if (c != -2) {
                    pp = 2.0f * A.qb[((l0 + l) * 2 + e) * S + s2];
                }
                sxe[2 * i] = pp;
                sxe[2 * i + 1] = wnp;
            }
        __syncthreads();
        if (UPDATE) {
            // full p_ab = p*_ab + C_ba q0_A,a + C_ab q0_B,b
            for (int i = tid; i < nl * S * NP1; i += nth) {
                const int l = i / (S * NP1), r = i % (S * NP1), s = r / NP1, n = r % NP1;
                const int a = s % P, b = s / P;
                const float ca = A.cP[a], cb = A.cP[b], den = 1.0f / (1.0f + ca + cb);
                sp[i] = sq[(l * S + s) * 2 * NP1 + n] + (1.0f + cb) * den * s0[(l * 2 + 0) * P * NP1 + a * NP1 + n] +
                        (1.0f + ca) * den * s0[(l * 2 + 1) * P * NP1 + b * NP1 + n];
            }
            __syncthreads();
            for (int i = tid; i < nl * S * 2; i += nth) {
                const int l = i / (S * 2), r = i % (S * 2), s = r / 2, e = r % 2;
                const float *g = sg + l * GEO1;
                const int nd = e ? N : 0;
                const float tau = e ? 1.0f : -1.0f;
                const float pm = sp[(l * S + s) * NP1 + nd];
                const float wnm = tau * sq[(l * S + s) * 2 * NP1 + NP1 + nd];
                float pp = sxe[2 * i], wnp = sxe[2 * i + 1];
                if (scn[l * 2 + e] == -2) {   // p = 0 end: mirror state
                    pp = -pm;
                    wnp = wnm;
                }
                const float wm = g[7 + 3 * e], zz = g[8 + 3 * e], iz = g[9 + 3 * e];
                const float dP = wm * (pp - pm) + zz * (wnm - wnp);
                const float dWn = (1.0f - wm) * (wnp - wnm) + iz * (pm - pp);
                sx[(l * S + s) * 4 + e] = g[1] * dWn;
                sx[(l * S + s) * 4 + 2 + e] = g[1] * tau * dP;
            }
            __syncthreads();
            for (int i = tid; i < nl * S * NP1; i += nth) {
                const int l = i / (S * NP1), r = i % (S * NP1), s = r / NP1, n = r % NP1;
                const int a = s % P, b = s / P;
                const float *g = sg + l * GEO1;
                const float *qs = sq + (l * S + s) * 2 * NP1;
                const float *ps = sp + (l * S + s) * NP1;
                float dw = 0.f, dp = 0.f;
                for (int m = 0; m < NP1; ++m) {
                    const float d = sD[m * NP1 + n];
                    dw += d * qs[NP1 + m];
                    dp += d * ps[m];
                }
                const float *xs = sx + (l * S + s) * 4;
                const float lw = sL[n] * xs[0] + sL[NP1 + n] * xs[1];
                const float lpp = sL[n] * xs[2] + sL[NP1 + n] * xs[3];
                const float wab = 1.0f / (1.0f + A.cP[a] + A.cP[b]);
                float rhs[2];
                rhs[0] = -g[2] * wab * (g[0] * dw + lw);
                rhs[1] = -g[3] * (g[0] * dp + lpp);
                const int64_t base = ((l0 + l) * S + s) * 2 * NP1;
                for (int fl = 0; fl < 2; ++fl) {
                    const float rr = sc.a * sres[(l * S + s) * 2 * NP1 + fl * NP1 + n] + sc.dt * rhs[fl];
                    A.res[base + fl * NP1 + n] = rr;
                    const float qv = qs[fl * NP1 + n] + sc.b * rr;
                    A.q[base + fl * NP1 + n] = qv;
                    sn[(l * S + s) * 2 * NP1 + fl * NP1 + n] = qv;
                }
            }
            __syncthreads();
            for (int i = tid; i < nl * S * 2 * NP1; i += nth) sq[i] = sn[i];
            __syncthreads();
        }
        // edge BCs: one thread per (line, node, row) of the solution operator
        for (int i = tid; i < nl * NP1 * 2 * P; i += nth) {
            const int l = i / (NP1 * 2 * P), r = i % (NP1 * 2 * P), n = r / (2 * P), row = r % (2 * P);
            const int64_t lg = l0 + l;
            const float *rp = srp + (l * NP1 + n) * 2 * P;
            const float *H1 = sH + row * 2 * P, *H2 = sH + 4 * P * P + row * S;
            const float *qn = sq + l * S * 2 * NP1 + n;
            float x = 0.f;
            for (int col = 0; col < 2 * P; ++col) x += H1[col] * rp[col];
            for (int s2 = 0; s2 < S; ++s2) x += H2[s2] * qn[s2 * 2 * NP1];
            const int side = row >= P, a = row - side * P;
            const int *mp = smp + l * 6 + 3 * side;
            const int m = mp[2] ? (N - n) : n;
            if (DGH_IN_RANGE(A.err, mp[0], A.T)) A.qb2[(((int64_t)mp[0] * 3 + mp[1]) * P + a) * NP1 + m] = x;
            const float q0 = x + rp[row];
            A.q0[(lg * 2 + side) * P * NP1 + a * NP1 + n] = q0;
            s0[(l * 2 + side) * P * NP1 + a * NP1 + n] = q0;
        }
        __syncthreads();
        // new 1D traces (full p_ab, tangential velocity along the outward end direction)
        for (int i = tid; i < nl * S * 2; i += nth) {
            const int l = i / (S * 2), r = i % (S * 2), s = r / 2, e = r % 2;
            const int a = s % P, b = s / P;
            const int nd = e ? N : 0;
            const float ca = A.cP[a], cb = A.cP[b], den = 1.0f / (1.0f + ca + cb);
            const float *qs = sq + (l * S + s) * 2 * NP1;
            const float p = qs[nd] + (1.0f + cb) * den * s0[(l * 2 + 0) * P * NP1 + a * NP1 + nd] +
                            (1.0f + ca) * den * s0[(l * 2 + 1) * P * NP1 + b * NP1 + nd];
            float *dst = A.tr_out + ((l0 + l) * S + s) * 4 + e * 2;
            dst[0] = p;
            dst[1] = (e ? 1.0f : -1.0f) * qs[NP1 + nd];
        }
    }
}

inline size_t k1d_smem(int N, int P, int tile) {
    const int NP1 = N + 1, S = P * P;
    return sizeof(float) * (NP1 * NP1 + 2 * NP1 + tile * (2 * S * 2 * NP1 + S * NP1 + S * 4 + 2 * P * NP1 + GEO1) +
                            4 * P * P + 2 * P * S + tile * NP1 * 2 * P + tile * S * 2 * NP1 + tile * S * 4) +
           sizeof(int) * tile * 8;
}

// ==================================================================== 0D
// One CTA per (corner, block of K0D_ROWS rows of the 3P^2 x 3P^2 solution
// operator): the CTA forms the corner's r^+ (3P^2 values) in shared memory,
// then each warp takes rows two at a time -- coalesced row loads, shuffle
// sums -- so that the operator (746 KB at P = 12) streams through many SMs.
constexpr int K0D_ROWS = 32;

__global__ void __launch_bounds__(256) k0d_stage(Args0 A) {
    const int c = blockIdx.x;
    const int P = A.P, S = P * P, R = 3 * S;
    extern __shared__ float rp[];
    const int *cd = A.corner + c * 6;
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        const int slot = i / S, s = i % S;
        const int l0 = cd[2 * slot], e = cd[2 * slot + 1];
        const int l = DGH_IN_RANGE(A.err, l0, A.L) ? l0 : 0;
        const float *tr = A.tr1 + ((int64_t)l * S + s) * 4 + e * 2;
        rp[i] = 0.5f * (tr[0] + A.cornerZ[c * 3 + slot] * tr[1]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int r0 = blockIdx.y * K0D_ROWS, r1 = min(R, r0 + K0D_ROWS);
    for (int i = r0 + 2 * warp; i < r1; i += 2 * nwarp) {
        const bool two = i + 1 < r1;
        const float *h0 = A.Hc + (int64_t)i * R, *h1 = h0 + R;
        float x0 = 0.f, x1 = 0.f;
        for (int j = lane; j < R; j += 32) {
            const float r = rp[j];
            x0 += h0[j] * r;
            if (two) x1 += h1[j] * r;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x0 += __shfl_xor_sync(0xffffffffu, x0, o);
            x1 += __shfl_xor_sync(0xffffffffu, x1, o);
        }
        if (lane == 0)
            for (int k = 0; k < (two ? 2 : 1); ++k) {
                const int row = i + k, slot = row / S, s = row % S;
                const int l = cd[2 * slot], e = cd[2 * slot + 1];
                if (DGH_IN_RANGE(A.err, l, A.L)) A.qb1[((int64_t)l * 2 + e) * S + s] = k ? x1 : x0;
            }
    }
}

__global__ void k_advance_time(double *time, int64_t *step, double dt) {
    time[0] += dt;
    step[0] += 1;
}

// ==================================================================== misc
// Gaussian pressure at the nodes (FP64 node coordinates from the tet vertices).
template <int N>
__global__ void k_init_gaussian(float *q, const double *cellv, const double *rst, int64_t K, double x0, double y0,
                                double z0, double w, double amp) {
    constexpr int NP = Ord<N>::NP;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= K * NP) return;
    const int64_t k = i / NP;
    const int n = (int)(i % NP);
    const double r = rst[3 * n], s = rst[3 * n + 1], t = rst[3 * n + 2];
    const double l0 = -(1.0 + r + s + t) * 0.5, l1 = (1.0 + r) * 0.5, l2 = (1.0 + s) * 0.5, l3 = (1.0 + t) * 0.5;
    const double *v = cellv + 12 * k;
    const double x = l0 * v[0] + l1 * v[3] + l2 * v[6] + l3 * v[9];
    const double y = l0 * v[1] + l1 * v[4] + l2 * v[7] + l3 * v[10];
    const double z = l0 * v[2] + l1 * v[5] + l2 * v[8] + l3 * v[11];
    const double d2 = (x - x0) * (x - x0) + (y - y0) * (y - y0) + (z - z0) * (z - z0);
    float *qk = q + (k / 32) * (4 * NP * 32) + (k % 32);   // cell-interleaved [K/32][4][Np][32]
    qk[n * 32] = (float)(amp * exp(-d2 / (w * w)));
    qk[(NP + n) * 32] = 0.f;
    qk[(2 * NP + n) * 32] = 0.f;
    qk[(3 * NP + n) * 32] = 0.f;
}

// Energy: per cell |J| [p^T M p /(2 rho c^2) + rho/2 sum u^T M u] (Sec. 4.1,
// energy of the pressure-velocity system), all in FP64: the FP32 fields are
// widened, the mass-matrix product uses the FP64 mass matrix Md (dynamic
// shared memory, NP*NP doubles) and the sums are FP64.
template <int N>
__global__ void __launch_bounds__(256) k_energy_partial(const float *q, const double *Md, const double *ew, int64_t K,
                                                        double *partial) {
    constexpr int NP = Ord<N>::NP;
    extern __shared__ double sMe[];
    __shared__ double red[256];
    for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) sMe[i] = Md[i];
    __syncthreads();
    double acc = 0.0;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < K * 4; it += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = it / 4;
        const int fl = (int)(it % 4);
        const float *x = q + (k / 32) * (4 * NP * 32) + fl * NP * 32 + (k % 32);   // stride 32 between nodes
        double s = 0.0;
        for (int n = 0; n < NP; ++n) {
            double y = 0.0;
            for (int m = 0; m < NP; ++m) y += sMe[n * NP + m] * (double)x[m * 32];
            s += (double)x[n * 32] * y;
        }
        acc += s * ew[2 * k + (fl == 0 ? 0 : 1)];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Dynamic shared memory of the energy kernels (the FP64 mass matrix).
inline size_t energy_smem(int N) {
    const int np = (N + 1) * (N + 2) * (N + 3) / 6;
    return sizeof(double) * np * np;
}

__global__ void k_sum_partials(const double *partial, int n, double *out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Full auxiliary pressures for read-back.
__global__ void k_full2(const float *q2, const float *q0, float *out, int64_t T, int P, int NP2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = T * P * 3 * NP2;
    if (i >= total) return;
    const int64_t t = i / (P * 3 * NP2);
    const int r = (int)(i % (3 * NP2));
    const int fl = r / NP2, n = r % NP2;
    out[i] = q2[i] + (fl == 0 ? q0[t * NP2 + n] : 0.f);
}

__global__ void k_full1(const float *q1, const float *q0, const float *cP, float *out, int64_t L, int P, int NP1) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int S = P * P;
    const int64_t total = L * S * 2 * NP1;
    if (i >= total) return;
    const int64_t l = i / (S * 2 * NP1);
    const int r = (int)(i % (S * 2 * NP1));
    const int s = r / (2 * NP1), fl = (r / NP1) % 2, n = r % NP1;
    float v = q1[i];
    if (fl == 0) {
        const int a = s % P, b = s / P;
        const float ca = cP[a], cb = cP[b], den = 1.0f / (1.0f + ca + cb);
        v += (1.0f + cb) * den * q0[(l * 2 + 0) * P * NP1 + a * NP1 + n] + (1.0f + ca) * den * q0[(l * 2 + 1) * P * NP1 + b * NP1 + n];
    }
    out[i] = v;
}

}  // namespace dgh
