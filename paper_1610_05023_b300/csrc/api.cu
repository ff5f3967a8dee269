// C ABI of the solver (include/dgh.h): set-up, device layout, stage launches,
// CUDA-graph replay of the step, read-back, energy, checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dgh.h"
#include "kernels.cuh"
#include "setup.h"

using namespace dgh;

namespace {

// NVTX range over one API call, so that a profiler's timeline groups the
// kernels of a call under its name (no cost without an attached tool).
struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
};


// Carpenter & Kennedy (1994) 5-stage 2N-storage RK4 coefficients.
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};
const double kRkC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                        2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

thread_local std::string g_create_error = "no error";

// No C++ exception crosses the C ABI: every int entry point runs its body
// through dgh_guarded.  A failed host allocation returns DGH_ENOMEM and any
// other exception DGH_EINVAL; the message goes to the object's last-error
// string (err_slot), or to the thread's creation error when there is none.
template <class T>
static std::string *err_slot(const T *obj) {
    return obj ? &const_cast<T *>(obj)->err : nullptr;
}

template <class F>
static int dgh_guarded(std::string *err, F &&body) noexcept {
    std::string &slot = err ? *err : g_create_error;
    try {
        return body();
    } catch (const std::bad_alloc &) {
        try { slot = "internal error: host memory exhausted"; } catch (...) {}
        return DGH_ENOMEM;
    } catch (const std::exception &e) {
        try { slot = std::string("internal error: ") + e.what(); } catch (...) {}
        return DGH_EINVAL;
    } catch (...) {
        try { slot = "internal error: unknown C++ exception"; } catch (...) {}
        return DGH_EINVAL;
    }
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct dgh_ctx {
    std::string err = "no error";
    cudaStream_t stream = nullptr;
    int device = 0;
    int N = 0, P = 0, Np = 0, Nfp = 0, Np2 = 0, Np1 = 0;
    int64_t K = 0, K32 = 0, T = 0, L = 0, Fb = 0;
    int64_t Ki32 = 0, Kb32 = 0;       // 32-cell blocks of interior cells, then of cells with HABC faces
    bool no_overlap = false;          // union of a batch: one launch over all cells, no side stream
    std::vector<int64_t> part_blk0;   // first 32-cell block of every part (batch problem), + end
    std::vector<int64_t> can2dev;     // canonical cell -> device cell slot
    int *can2dev_d = nullptr;         // the same map on the device (state transfers)
    cudaStream_t side = nullptr;      // HABC chain stream (overlaps the interior 3D work)
    cudaEvent_t ev3d[5] = {}, ev2d[5] = {}, evjoin = nullptr;
    cudaEvent_t ev_order = nullptr;   // orders a caller's stream after the context's work (no-allocation energy)
    void *xfer = nullptr;             // staging buffer of the 3D state transfers (grown on demand)
    size_t xfer_bytes = 0;
    int C = 0;
    int M = 1;
    double dt = 0.0, t0 = 0.0;
    double cfl = 1.0;                 // time-step rule factor of the description
    bool dt_fixed = false;            // dt given in the description (kept by dgh_set_material)
    int64_t step_count = 0;
    int64_t wd_every = 0;     // energy watchdog: check every wd_every steps (0 = off)
    double wd_limit = 0.0;    // energy bound (<= 0: finiteness only)
    int cur = 0;              // trace buffer holding the current traces
    bool dirty = true;        // boundary algebra must be recomputed
    std::vector<DevBuf> bufs;
    int64_t device_bytes = 0;
    // 3D
    float *q3 = nullptr, *res3 = nullptr, *tin3[2] = {nullptr, nullptr}, *trb = nullptr, *geo3 = nullptr;
    int *d_err = nullptr;
    int *conn3 = nullptr;
    float *D3 = nullptr, *L3 = nullptr, *M3 = nullptr;
    double *M3d = nullptr;            // FP64 mass matrix (error reductions)
    int *fmask3 = nullptr, *fperm3 = nullptr, *nslot3 = nullptr;
    double *cellv = nullptr, *rst = nullptr, *ew = nullptr;
    // 2D
    float *q2 = nullptr, *res2 = nullptr, *tr2[2] = {nullptr, nullptr}, *geo2 = nullptr, *qb2 = nullptr, *q0_3 = nullptr;
    int *conn2 = nullptr, *tri_face = nullptr, *tri_bface = nullptr, *fmask2 = nullptr;
    float *D2 = nullptr, *L2 = nullptr;
    // 1D
    float *q1 = nullptr, *res1 = nullptr, *tr1[2] = {nullptr, nullptr}, *geo1 = nullptr, *qb1 = nullptr, *q0_2 = nullptr;
    int *conn1 = nullptr, *lmap = nullptr;
    float *D1 = nullptr, *L1 = nullptr, *H1 = nullptr, *H2 = nullptr, *cP = nullptr;
    // 0D
    int *corner = nullptr;
    float *cornerZ = nullptr, *Hc = nullptr;
    // time
    double *d_time = nullptr;
    int64_t *d_step = nullptr;
    // energy scratch
    double *partial = nullptr, *d_energy = nullptr;
    int energy_blocks = 0;
    // sources
    SrcParams src{};
    float *srcvec = nullptr;
    std::vector<int64_t> src_k;       // canonical cell of every source
    std::vector<float> src_vec_h;     // host copy of the source vectors [n][Np]
    // launch shapes
    int grid3 = 1, grid2 = 1, grid1 = 1, tile2 = 1, tile1 = 1, occ3 = 0, sms = 1;
    int cta3_per_sm = 0;              // tunable: persistent 3D CTAs per SM (0 = occupancy limit)
    int sm3_div = 1;                  // tunable: the 3D grid covers sms / sm3_div SMs (concurrent batch groups)
    int split3 = 1;                   // tunable: 1 = interior and HABC-face cells as two 3D launches per stage
    int thr2 = 128, thr1 = 256;       // tunable: threads per CTA of the 2D / 1D kernels
    int precision = DGH_PREC_FP32;    // arithmetic of the 3D contractions (DGH_PREC_*)
    uint8_t *tcops = nullptr;         // tensor-core operand images of D_r, D_s, D_t, LIFT (hi, then lo)
    unsigned long long *tile_ctr = nullptr;   // [16] block counters of the 3D launches of a step
    unsigned *tile_ctr2 = nullptr;            // [4] tile counters of the 2D kernel: main chain, shadow chain
    size_t smem3 = 0, smem2 = 0, smem1 = 0, smem0 = 0;
    int smem_optin = 0;
    // learned closure (inference on this context's chain)
    bool cl_on = false;
    bool cl_homog = false;            // homogeneous form: 7 scales follow the weights
    float *cl_w = nullptr;            // MLP weights (BF16-rounded, stored FP32) [MLP_NPARAM], 7 FP32 scales, MLP(0)
    float *cl_feat = nullptr;         // [T][Np2][6]
    float *cl_rm = nullptr;           // [T][Np2] r^- of this chain
    // shadow chain of another HABC order driven one-way by the 3D traces (sample recording)
    struct Shadow {
        int P = 0, M = 1, tile2 = 1, tile1 = 1, grid2 = 1, grid1 = 1;
        size_t smem2 = 0, smem1 = 0, smem0 = 0;
        HabcOps habc;
        float *q2 = nullptr, *res2 = nullptr, *tr2[2] = {nullptr, nullptr}, *qb2 = nullptr, *q0_3 = nullptr;
        float *q1 = nullptr, *res1 = nullptr, *tr1[2] = {nullptr, nullptr}, *qb1 = nullptr, *q0_2 = nullptr;
        float *H1 = nullptr, *H2 = nullptr, *Hc = nullptr, *cP = nullptr;
        float *feat = nullptr, *rm = nullptr, *rm_main = nullptr;
        float *samples = nullptr;
        unsigned long long *count = nullptr;
        int64_t max_samples = 0;
        int every = 1;
        uint32_t threshold = 0;
        uint64_t seed = 0;
    };
    Shadow *sh = nullptr;
    // graphs (one per trace parity)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // host copies needed by read-back
    HostMesh mesh;
    RefTet ref3;
    RefTri ref2;
    RefLine ref1;
    HabcOps habc;
};

#define CK(call)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            return DGH_ECUDA;                                                    \
        }                                                                        \
    } while (0)

namespace {

template <class T>
int dalloc(dgh_ctx *ctx, T *&ptr, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DGH_ENOMEM : DGH_ECUDA;
    }
    cudaMemset(p, 0, bytes);
    ctx->bufs.push_back({p, bytes});
    ctx->device_bytes += int64_t(bytes);
    ptr = static_cast<T *>(p);
    return DGH_OK;
}

template <class T>
int upload(dgh_ctx *ctx, T *&ptr, const std::vector<T> &h) {
    int rc = dalloc(ctx, ptr, h.size());
    if (rc) return rc;
    if (!h.empty()) CK(cudaMemcpy(ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return DGH_OK;
}

std::vector<float> to_f(const Mat &A) {
    std::vector<float> v(A.a.size());
    for (size_t i = 0; i < v.size(); ++i) v[i] = float(A.a[i]);
    return v;
}

// ------------------------------------------------------------ dispatch on N
template <template <int> class F, class... Args>
int dispatchN(int N, Args &&...args) {
    switch (N) {
        case 1: return F<1>::run(args...);
        case 2: return F<2>::run(args...);
        case 3: return F<3>::run(args...);
        case 4: return F<4>::run(args...);
        case 5: return F<5>::run(args...);
        case 6: return F<6>::run(args...);
        default: return DGH_EUNSUPPORTED;
    }
}

Args3 args3(dgh_ctx *c, int cur) {
    Args3 A;
    A.q = c->q3;
    A.res = c->res3;
    A.tin = c->tin3[cur];
    A.tout = c->tin3[cur ^ 1];
    A.trb = c->trb;
    A.geo = c->geo3;
    A.conn = c->conn3;
    A.err = c->d_err;
    A.kcells = c->K32 * 32;
    A.nbfaces = c->Fb;
    A.blk_begin = 0;
    A.blk_end = c->K32;
    A.D = c->D3;
    A.LIFT = c->L3;
    A.fmask = c->fmask3;
    A.fperm = c->fperm3;
    A.nslot = c->nslot3;
    A.src = c->src;
    A.src.vec = c->srcvec;
    return A;
}

Args2 args2(dgh_ctx *c, int cur, bool update, bool shadow = false) {
    if (shadow) {   // same geometry, the shadow chain's order and state; no exterior state written
        const dgh_ctx::Shadow *h = c->sh;
        Args2 A = args2(c, cur, update, false);
        A.q = h->q2;
        A.res = h->res2;
        A.tr_in = h->tr2[cur];
        A.tr_out = update ? h->tr2[cur ^ 1] : h->tr2[cur];
        A.qb = h->qb2;
        A.q0 = h->q0_3;
        A.tin3 = nullptr;
        A.feat = h->feat;
        A.rm_out = h->rm;
        A.cP = h->cP;
        A.invM = 1.0f / float(h->M);
        A.P = h->P;
        A.tile_ctr = c->tile_ctr2 + 2;
        return A;
    }
    Args2 A;
    A.q = c->q2;
    A.res = c->res2;
    A.tr_in = c->tr2[cur];
    A.tr_out = update ? c->tr2[cur ^ 1] : c->tr2[cur];
    A.geo = c->geo2;
    A.conn = c->conn2;
    A.qb = c->qb2;
    A.q0 = c->q0_3;
    A.tin3 = c->cl_on ? nullptr : (update ? c->tin3[cur ^ 1] : c->tin3[cur]);   // the closure writes it instead
    A.feat = c->cl_on ? c->cl_feat : nullptr;
    A.rm_out = c->cl_on ? c->cl_rm : (c->sh ? c->sh->rm_main : nullptr);
    A.trb = c->trb;
    A.tri_face = c->tri_face;
    A.tri_bface = c->tri_bface;
    A.D = c->D2;
    A.LIFT = c->L2;
    A.fmask = c->fmask2;
    A.cP = c->cP;
    A.invM = 1.0f / float(c->M);
    A.P = c->P;
    A.T = c->T;
    A.err = c->d_err;
    A.kcells = c->K32 * 32;
    A.nbfaces = c->Fb;
    A.tile_ctr = c->tile_ctr2;
    return A;
}

Args1 args1(dgh_ctx *c, int cur, bool update, bool shadow = false) {
    if (shadow) {
        const dgh_ctx::Shadow *h = c->sh;
        Args1 A = args1(c, cur, update, false);
        A.q = h->q1;
        A.res = h->res1;
        A.tr_in = h->tr1[cur];
        A.tr_out = update ? h->tr1[cur ^ 1] : h->tr1[cur];
        A.qb = h->qb1;
        A.q0 = h->q0_2;
        A.qb2 = h->qb2;
        A.tr2 = update ? h->tr2[cur ^ 1] : h->tr2[cur];
        A.H1 = h->H1;
        A.H2 = h->H2;
        A.cP = h->cP;
        A.invM = 1.0f / float(h->M);
        A.P = h->P;
        return A;
    }
    Args1 A;
    A.q = c->q1;
    A.res = c->res1;
    A.tr_in = c->tr1[cur];
    A.tr_out = update ? c->tr1[cur ^ 1] : c->tr1[cur];
    A.geo = c->geo1;
    A.conn = c->conn1;
    A.qb = c->qb1;
    A.q0 = c->q0_2;
    A.qb2 = c->qb2;
    A.tr2 = update ? c->tr2[cur ^ 1] : c->tr2[cur];
    A.lmap = c->lmap;
    A.D = c->D1;
    A.LIFT = c->L1;
    A.H1 = c->H1;
    A.H2 = c->H2;
    A.cP = c->cP;
    A.invM = 1.0f / float(c->M);
    A.P = c->P;
    A.L = c->L;
    A.err = c->d_err;
    A.T = c->T;
    return A;
}

int tc_code(int precision) {
    return precision == DGH_PREC_BF16_TC ? TC_BF16 : precision == DGH_PREC_FP16_TC ? TC_FP16 : TC_SPLIT_BF16;
}

// Which 3D kernel a context runs: the split-TF32 tensor-core kernel
// (DGH_PREC_SPLIT_TF32, and DGH_PREC_FP32 where it is the faster one), the
// BF16/FP16 tensor-core kernel (the precision form) or the FP32 CUDA-core
// kernel.  Measured on B300 (whole steps, tuned shapes): at N = 4 the
// split-TF32 kernel is the faster one from about 80 k cells (10-18% per
// step at 83 k - 384 k cells, 20% at 663 k), while on small meshes its
// per-launch prologue (operator images, tensor memory) and its 128-cell
// tiles, one CTA per SM, cost more than they save; at N = 1, 2, 3 the
// CUDA-core kernel is faster at every size (1.2-2.2x per 3D launch at
// 384 k cells), their contractions being too short for the tensor core to
// pay for the operand conversion.
enum Kern3 { K3_CUDA = 0, K3_TF32 = 1, K3_TC = 2 };
constexpr int kMaxTf32Order = 4;   // largest N whose operators and stage fit one CTA's shared memory
constexpr int64_t kTf32MinCells = 65536;   // DGH_PREC_FP32 at N = 4: split TF32 from this many cells
int kern3_of(int precision, int N, int64_t K) {
    if (precision == DGH_PREC_SPLIT_TF32) return K3_TF32;
    if (precision == DGH_PREC_FP32) return (N == kMaxTf32Order && K >= kTf32MinCells) ? K3_TF32 : K3_CUDA;
    if (precision == DGH_PREC_FP32_CUDA) return K3_CUDA;
    return K3_TC;
}

// Round to the nearest TF32 value (13 low bits of the FP32 significand
// cleared, ties to even); finite inputs.
float tf32_round(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

// Operator images of the split-TF32 kernel: B operands with rows = output
// nodes, K-major canonical layout without swizzle (8-row x 16-byte core
// matrices of 4 TF32 values; element (n, k) of a matrix with R rows at byte
// (k/4)(R/8)128 + (n/8)128 + (n%8)16 + (k%4)4), zero padding.
//   [D_r; D_s; D_t]: 3 NPAD rows x KV (D_j in rows j NPAD .. j NPAD + Np - 1)
//   LIFT: NPAD rows x 4 FK (face f's nodes at K = f FK + m)
// hi = TF32 rounding of the FP64 entry, lo = TF32 rounding of the rest; the
// hi image is followed by the lo image.
std::vector<uint8_t> tf32_operator_images(const RefTet &T3) {
    const int Np = T3.Np, Nfp = T3.Nfp;
    const int NPAD = (Np + 15) / 16 * 16, KV = (Np + 7) / 8 * 8, FK = (Nfp + 7) / 8 * 8;
    const size_t BD = size_t(3) * NPAD * KV * 4, BL = size_t(NPAD) * 4 * FK * 4, BOPS = BD + BL;
    std::vector<uint8_t> img(2 * BOPS, 0);
    auto put = [&](size_t base, int R, int n, int k, double x) {
        const size_t off = base + size_t(k / 4) * (R / 8) * 128 + size_t(n / 8) * 128 + (n % 8) * 16 + (k % 4) * 4;
        const float hi = tf32_round(float(x));
        const float lo = tf32_round(float(x - double(hi)));
        std::memcpy(&img[off], &hi, 4);
        std::memcpy(&img[BOPS + off], &lo, 4);
    };
    const Mat *Dj[3] = {&T3.Dr, &T3.Ds, &T3.Dt};
    for (int j = 0; j < 3; ++j)
        for (int n = 0; n < Np; ++n)
            for (int k = 0; k < Np; ++k) put(0, 3 * NPAD, j * NPAD + n, k, (*Dj[j])(n, k));
    for (int n = 0; n < Np; ++n)
        for (int f = 0; f < 4; ++f)
            for (int m = 0; m < Nfp; ++m) put(BD, NPAD, n, f * FK + m, T3.LIFT(n, f * Nfp + m));
    return img;
}

// Operator images of the tensor-core kernel: the B operands D_r, D_s, D_t
// (NPAD x NPAD) and LIFT (NPAD x 4 FPAD, face f's nodes at K = f FPAD + m),
// rows = output nodes, in the K-major canonical layout without swizzle:
// 8-row x 16-byte core matrices, element (n, k) of a matrix with R rows at
// byte (k/8)(R/8)128 + (n/8)128 + (n%8)16 + (k%8)2; zero padding.  The
// split variant appends the BF16 residuals x - hi(x) of every entry.
std::vector<uint8_t> tc_operator_images(const RefTet &T3, int precision) {
    const int Np = T3.Np, Nfp = T3.Nfp;
    const int NPAD = (Np + 15) / 16 * 16, FPAD = (Nfp + 15) / 16 * 16, KL = 4 * FPAD;
    const bool split = precision == DGH_PREC_SPLIT_BF16, half = precision == DGH_PREC_FP16_TC;
    const size_t BD = size_t(NPAD) * NPAD * 2, BL = size_t(NPAD) * KL * 2, BOPS = 3 * BD + BL;
    std::vector<uint8_t> img(BOPS * (split ? 2 : 1), 0);
    auto put = [&](size_t base, int n, int k, double x) {
        const size_t off = base + size_t(k / 8) * (NPAD / 8) * 128 + size_t(n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
        uint16_t hi = 0, lo = 0;
        if (half) {
            const __half h = __float2half_rn(float(x));
            std::memcpy(&hi, &h, 2);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(float(x));
            std::memcpy(&hi, &h, 2);
            if (split) {
                const __nv_bfloat16 l = __float2bfloat16_rn(float(x - double(__bfloat162float(h))));
                std::memcpy(&lo, &l, 2);
            }
        }
        std::memcpy(&img[off], &hi, 2);
        if (split) std::memcpy(&img[BOPS + off], &lo, 2);
    };
    const Mat *Dj[3] = {&T3.Dr, &T3.Ds, &T3.Dt};
    for (int j = 0; j < 3; ++j)
        for (int n = 0; n < Np; ++n)
            for (int k = 0; k < Np; ++k) put(j * BD, n, k, (*Dj[j])(n, k));
    for (int n = 0; n < Np; ++n)
        for (int f = 0; f < 4; ++f)
            for (int m = 0; m < Nfp; ++m) put(3 * BD, n, f * FPAD + m, T3.LIFT(n, f * Nfp + m));
    return img;
}

// part: 0 = all cells, 1 = interior blocks, 2 = blocks with HABC faces
template <int N>
struct Launch3 {
    static int run(dgh_ctx *c, int cur, int stage, bool update, int part = 0, cudaStream_t st = nullptr) {
        if (!st) st = c->stream;
        if (!update) {
            const int64_t total = c->K32 * 32 * 4 * Cfg3<N>::NFP;
            k3d_traces<N><<<int((total + 127) / 128), 128, 0, st>>>(c->q3, c->geo3, c->conn3, c->fmask3, c->fperm3,
                                                                    c->tin3[cur], c->trb, c->K32 * 32);
            return DGH_OK;
        }
        StageCoef sc;
        sc.a = float(kRkA[stage]);
        sc.b = float(kRkB[stage]);
        sc.dt = float(c->dt);
        sc.c_dt = kRkC[stage] * c->dt;
        sc.time = c->d_time;
        Args3 A = args3(c, cur);
        // counters: parts 1, 2 of stage s at 2s, 2s+1, part 3 at 10+s (zeroed once per step), part 0 at 15
        A.tile_ctr = c->tile_ctr + (part == 0 ? 15 : part == 3 ? 10 + stage : stage * 2 + (part - 1));
        if (part == 0) cudaMemsetAsync(A.tile_ctr, 0, sizeof(unsigned long long), st);
        if (part == 1) A.blk_end = c->Ki32;
        if (part == 2) A.blk_begin = c->Ki32;
        const int64_t nblk = A.blk_end - A.blk_begin;
        if (nblk <= 0) return DGH_OK;
        A.max_tiles = int(std::min<int64_t>(nblk, int64_t(1) << 30));
        const int kern = kern3_of(c->precision, N, c->K);
        if (kern == K3_TF32) {   // split-TF32 tensor-core kernel: tiles of four 32-cell blocks, one CTA per SM
            if constexpr (N <= kMaxTf32Order) {
                const int grid = (int)std::min<int64_t>((nblk + 3) / 4, c->grid3);
                k3d_tf32<N><<<grid, CfgTF<N>::NTHR, CfgTF<N>::SMEM, st>>>(A, sc, c->tcops);
                return DGH_OK;
            } else {
                return DGH_EUNSUPPORTED;
            }
        }
        if (kern == K3_TC) {   // tensor-core kernel: tiles of four 32-cell blocks
            const int grid = (int)std::min<int64_t>((nblk + 3) / 4, c->grid3);
            switch (tc_code(c->precision)) {
                case TC_BF16: k3d_tc<N, TC_BF16><<<grid, 256, CfgTC<N, TC_BF16>::SMEM, st>>>(A, sc, c->tcops); break;
                case TC_FP16: k3d_tc<N, TC_FP16><<<grid, 256, CfgTC<N, TC_FP16>::SMEM, st>>>(A, sc, c->tcops); break;
                default: k3d_tc<N, TC_SPLIT_BF16><<<grid, 256, CfgTC<N, TC_SPLIT_BF16>::SMEM, st>>>(A, sc, c->tcops); break;
            }
            return DGH_OK;
        }
        const int grid = (int)std::min<int64_t>(nblk, c->grid3);   // persistent CTAs, blocks claimed dynamically
        k3d_stage<N><<<grid, Cfg3<N>::NW * 32, Cfg3<N>::SMEM, st>>>(A, sc);
        return DGH_OK;
    }
};

template <int N>
struct Launch2 {
    static int run(dgh_ctx *c, int cur, int stage, bool update, cudaStream_t st = nullptr, bool shadow = false) {
        if (!st) st = c->stream;
        if (c->T == 0 || (!shadow && c->P == 0)) return DGH_OK;
        StageCoef sc;
        sc.a = float(kRkA[stage]);
        sc.b = float(kRkB[stage]);
        sc.dt = float(c->dt);
        sc.c_dt = 0.0;
        sc.time = c->d_time;
        Args2 A = args2(c, cur, update, shadow);
        // the kernel moves these arrays with 16-byte copies from 16-byte aligned bases
        if ((reinterpret_cast<uintptr_t>(A.q) | reinterpret_cast<uintptr_t>(A.res) | reinterpret_cast<uintptr_t>(A.q0) |
             reinterpret_cast<uintptr_t>(A.geo)) & 15u) {
            c->err = "2D level arrays are not 16-byte aligned";
            return DGH_EINVAL;
        }
        const int grid = shadow ? c->sh->grid2 : c->grid2, tile = shadow ? c->sh->tile2 : c->tile2;
        const int thr = shadow ? 256 : c->thr2;
        const size_t smem = shadow ? c->sh->smem2 : c->smem2;
        if (update)
            k2d_stage<N, true><<<grid, thr, smem, st>>>(A, sc, tile);
        else
            k2d_stage<N, false><<<grid, thr, smem, st>>>(A, sc, tile);
        // Learned closure: exterior state 2 (r^- + MLP(features)) by its own
        // kernel, at full occupancy.  Evaluated inside the face kernel's
        // boundary loop instead, the MLP (4.5 k multiply-adds per node, 7.5
        // nodes per thread of that kernel at P = 2) ran at 8 warps per SM and
        // made the closed step 1.9 times as long as the plain one.
        if (!shadow && c->cl_on) {
            const int64_t rows = c->T * c->Np2;
            const int blocks = (int)std::min<int64_t>((rows + 255) / 256, int64_t(4) * c->sms);
            k_closure_apply<<<blocks, 256, 0, st>>>(c->cl_w, c->cl_homog ? c->cl_w + MLP_NPARAM : nullptr,
                                                    c->cl_w + CL_MLP0, c->cl_feat,
                                                    c->cl_rm, rows, c->Np2, c->tri_face,
                                                    update ? c->tin3[cur ^ 1] : c->tin3[cur], nullptr);
        }
        return DGH_OK;
    }
};

template <int N>
struct Launch1 {
    static int run(dgh_ctx *c, int cur, int stage, bool update, cudaStream_t st = nullptr, bool shadow = false) {
        if (!st) st = c->stream;
        if (c->L == 0 || (!shadow && c->P == 0)) return DGH_OK;
        StageCoef sc;
        sc.a = float(kRkA[stage]);
        sc.b = float(kRkB[stage]);
        sc.dt = float(c->dt);
        sc.c_dt = 0.0;
        sc.time = c->d_time;
        Args1 A = args1(c, cur, update, shadow);
        const int grid = shadow ? c->sh->grid1 : c->grid1, tile = shadow ? c->sh->tile1 : c->tile1;
        const int thr = shadow ? 256 : c->thr1;
        const size_t smem = shadow ? c->sh->smem1 : c->smem1;
        if (update)
            k1d_stage<N, true><<<grid, thr, smem, st>>>(A, sc, tile);
        else
            k1d_stage<N, false><<<grid, thr, smem, st>>>(A, sc, tile);
        return DGH_OK;
    }
};

void launch0(dgh_ctx *c, int cur_traces, cudaStream_t st = nullptr, bool shadow = false) {
    if (!st) st = c->stream;
    if (c->C == 0 || (!shadow && c->P == 0)) return;
    Args0 A;
    A.tr1 = shadow ? c->sh->tr1[cur_traces] : c->tr1[cur_traces];
    A.qb1 = shadow ? c->sh->qb1 : c->qb1;
    A.corner = c->corner;
    A.cornerZ = c->cornerZ;
    A.Hc = shadow ? c->sh->Hc : c->Hc;
    A.P = shadow ? c->sh->P : c->P;
    A.C = c->C;
    A.err = c->d_err;
    A.L = c->L;
    const int R = 3 * A.P * A.P;
    k0d_stage<<<dim3(c->C, (R + K0D_ROWS - 1) / K0D_ROWS), 256, shadow ? c->sh->smem0 : c->smem0, st>>>(A);
}

// The shadow chain of one stage (2D, 1D, 0D of the shadow order; no
// exterior state) and, after stage 0, the sample recorder.  part 1 is the
// 2D kernel (it reads the 3D boundary traces, so it must finish before the
// next 3D launch of the boundary cells), part 2 the rest.
int launch_shadow(dgh_ctx *c, int cur, int stage, bool update, cudaStream_t st, int part = 0) {
    if (!c->sh) return DGH_OK;
    int rc = DGH_OK;
    if (part != 2 && (rc = dispatchN<Launch2>(c->N, c, cur, stage, update, st, true))) return rc;
    if (part == 1) return DGH_OK;
    rc = dispatchN<Launch1>(c->N, c, cur, stage, update, st, true);
    if (rc) return rc;
    launch0(c, update ? cur ^ 1 : cur, st, true);
    if (update && stage == 0 && c->T > 0) {
        dgh_ctx::Shadow *h = c->sh;
        const int64_t rows = c->T * c->Np2;
        const int blocks = (int)std::min<int64_t>((rows + 255) / 256, int64_t(4) * c->sms);
        // With the closure on, the rows are closed-loop: this chain's features
        // and r^-_shadow - r^-_this, the correction that the shadow order
        // implies on the trajectory the closure itself produces.
        const bool cl = c->cl_on;
        k_record_samples<<<blocks, 256, 0, st>>>(cl ? c->cl_feat : h->feat, cl ? c->cl_rm : h->rm, cl ? h->rm : h->rm_main,
                                                 rows, c->d_step, h->every, h->threshold, h->seed, h->samples, h->count,
                                                 h->max_samples);
    }
    return DGH_OK;
}

template <int N>
struct SetAttrs {
    static int run(dgh_ctx *c) {
        c->smem3 = Cfg3<N>::SMEM;
        // The limit is a property of the kernel, shared by every context of
        // this N (whatever P and tile): the 2D/1D kernels get the device's
        // opt-in maximum once, so that no context lowers it below another's need.
        // A refused attribute would otherwise surface only later, as a failed
        // launch: the first failure is reported here.
        cudaError_t first = cudaSuccess;
        auto chk = [&](cudaError_t r) {
            if (r != cudaSuccess && first == cudaSuccess) first = r;
        };
        int optin = 0;
        chk(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
        chk(cudaFuncSetAttribute(k3d_stage<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem3));
        chk(cudaFuncSetAttribute(k2d_stage<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        chk(cudaFuncSetAttribute(k2d_stage<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        chk(cudaFuncSetAttribute(k1d_stage<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        chk(cudaFuncSetAttribute(k1d_stage<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        c->smem_optin = optin;
        int nb = 0;
        const int kern = kern3_of(c->precision, N, c->K);
        if (kern == K3_CUDA) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k3d_stage<N>, Cfg3<N>::NW * 32, c->smem3);
        } else if (kern == K3_TF32) {
            if constexpr (N <= kMaxTf32Order) {
                // one CTA per SM: it owns all 512 tensor-memory columns
                chk(cudaFuncSetAttribute(k3d_tf32<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgTF<N>::SMEM));
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k3d_tf32<N>, CfgTF<N>::NTHR, CfgTF<N>::SMEM);
                nb = std::min(nb, 1);
                c->smem3 = CfgTF<N>::SMEM;
            }
        } else {
            // one CTA owns TCOLS tensor-memory columns (512 per SM)
            auto occ = [&](auto kern, size_t smem, int tcols) {
                chk(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, smem);
                nb = std::min(nb, 512 / tcols);
                c->smem3 = smem;
            };
            switch (tc_code(c->precision)) {
                case TC_BF16: occ(k3d_tc<N, TC_BF16>, CfgTC<N, TC_BF16>::SMEM, CfgTC<N, TC_BF16>::TCOLS); break;
                case TC_FP16: occ(k3d_tc<N, TC_FP16>, CfgTC<N, TC_FP16>::SMEM, CfgTC<N, TC_FP16>::TCOLS); break;
                default: occ(k3d_tc<N, TC_SPLIT_BF16>, CfgTC<N, TC_SPLIT_BF16>::SMEM, CfgTC<N, TC_SPLIT_BF16>::TCOLS); break;
            }
        }
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        c->occ3 = nb;
        c->sms = sms;
        if (first != cudaSuccess) {
            cudaGetLastError();   // a non-sticky error: clear it so that a later call is not blamed
            c->err = std::string("kernel shared-memory attributes: ") + cudaGetErrorString(first);
            return DGH_ECUDA;
        }
        return DGH_OK;
    }
};

// Launch shapes from the tunables: triangles / lines per CTA of the 2D / 1D
// kernels (tile2, tile1) and the number of persistent 3D CTAs per SM
// (cta3_per_sm, 0 = as many as fit).  Returns DGH_EINVAL for a tile whose
// shared memory does not fit.
template <int N>
struct Shapes {
    static int run(dgh_ctx *c) {
        const int P = c->P;
        c->smem2 = P ? k2d_smem(N, P, c->tile2) : 0;
        c->smem1 = P ? k1d_smem(N, P, c->tile1) : 0;
        c->smem0 = sizeof(float) * 3 * P * P;
        if ((int64_t)c->smem2 > c->smem_optin || (int64_t)c->smem1 > c->smem_optin) return DGH_EINVAL;
        if (P && c->tile2 * P > c->thr2) return DGH_EINVAL;   // one thread per (triangle, set)
        const int sms = c->sms;
        const int per_sm = c->cta3_per_sm > 0 ? std::min(c->cta3_per_sm, std::max(c->occ3, 1)) : std::max(c->occ3, 1);
        const int sms3 = std::max(1, c->sms / std::max(c->sm3_div, 1));
        const int64_t tiles3 = kern3_of(c->precision, N, c->K) == K3_CUDA ? c->K32 : (c->K32 + 3) / 4;
        c->grid3 = (int)std::max<int64_t>(1, std::min<int64_t>(tiles3, (int64_t)per_sm * sms3));
        int nb2 = 0, nb1 = 0;
        if (c->T) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k2d_stage<N, true>, c->thr2, c->smem2);
        if (c->L) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, k1d_stage<N, true>, c->thr1, c->smem1);
        const int64_t tiles2 = (c->T + c->tile2 - 1) / c->tile2;
        const int64_t tiles1 = (c->L + c->tile1 - 1) / c->tile1;
        c->grid2 = (int)std::max<int64_t>(1, std::min<int64_t>(tiles2, (int64_t)std::max(nb2, 1) * sms));
        c->grid1 = (int)std::max<int64_t>(1, std::min<int64_t>(tiles1, (int64_t)std::max(nb1, 1) * sms));
        return DGH_OK;
    }
};

// Boundary algebra of Algorithm 1 from the current fields (no time advance).
int run_closure(dgh_ctx *c) {
    const int cur = c->cur;
    int rc = dispatchN<Launch3>(c->N, c, cur, 0, false);
    if (rc) return rc;
    rc = dispatchN<Launch2>(c->N, c, cur, 0, false);
    if (rc) return rc;
    rc = dispatchN<Launch1>(c->N, c, cur, 0, false);
    if (rc) return rc;
    launch0(c, cur);
    if ((rc = launch_shadow(c, cur, 0, false, c->stream))) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("closure launch: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    c->dirty = false;
    return DGH_OK;
}

// The stage launches of one step plus the time advance; cur flips once per
// stage, so a step starting from cur ends with cur ^ 1.  With overlap, the
// HABC chain of stage s (2D, 1D, 0D kernels) runs on the side stream while
// the interior cells of stage s+1 are computed on the main stream; the cells
// with HABC faces of stage s+1 wait for the 2D kernel of stage s (it writes
// their exterior states), and the 2D kernel of stage s+1 waits for them.
// ms overrides the context's stream (a batch enqueues each group on its own).
int enqueue_step(dgh_ctx *c, int cur, bool overlap, cudaStream_t ms = nullptr) {
    if (!ms) ms = c->stream;
    overlap = overlap && !c->no_overlap;
    cudaStream_t ss = overlap ? c->side : ms;
    cudaMemsetAsync(c->tile_ctr, 0, 15 * sizeof(unsigned long long), ms);
    // split3 = 0: one 3D launch per stage over all cells (after the 2D kernel of
    // the previous stage), no tail of a separate launch of the HABC-face cells
    const bool split = overlap && c->split3 != 0 && c->T > 0;
    for (int s = 0; s < 5; ++s) {
        int rc = DGH_OK;
        if (split) {
            rc = dispatchN<Launch3>(c->N, c, cur, s, true, 1, ms);
            if (rc) return rc;
        }
        if (overlap && s > 0) cudaStreamWaitEvent(ms, c->ev2d[s - 1], 0);
        rc = dispatchN<Launch3>(c->N, c, cur, s, true, split ? 2 : 3, ms);
        if (rc) return rc;
        if (overlap) {
            cudaEventRecord(c->ev3d[s], ms);
            cudaStreamWaitEvent(ss, c->ev3d[s], 0);
        }
        rc = dispatchN<Launch2>(c->N, c, cur, s, true, ss);
        if (rc) return rc;
        if ((rc = launch_shadow(c, cur, s, true, ss, 1))) return rc;
        if (overlap) cudaEventRecord(c->ev2d[s], ss);
        rc = dispatchN<Launch1>(c->N, c, cur, s, true, ss);
        if (rc) return rc;
        launch0(c, cur ^ 1, ss);
        if ((rc = launch_shadow(c, cur, s, true, ss, 2))) return rc;
        cur ^= 1;
    }
    k_advance_time<<<1, 1, 0, ms>>>(c->d_time, c->d_step, c->dt);
    if (overlap) {
        cudaEventRecord(c->evjoin, ss);
        cudaStreamWaitEvent(ms, c->evjoin, 0);
    }
    return DGH_OK;
}

void drop_graphs(dgh_ctx *c) {
    for (int i = 0; i < 2; ++i)
        if (c->graph[i]) {
            cudaGraphExecDestroy(c->graph[i]);
            c->graph[i] = nullptr;
        }
}

int build_graph(dgh_ctx *c, int cur) {
    cudaGraph_t g = nullptr;
    cudaStream_t cs = c->stream;   // never the legacy stream (dgh_step enqueues directly then)
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c->err = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    int rc = enqueue_step(c, cur, true);
    e = cudaStreamEndCapture(cs, &g);
    if (rc) return rc;
    if (e != cudaSuccess) {
        c->err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    e = cudaGraphInstantiate(&c->graph[cur], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    return DGH_OK;
}

int level_count(const dgh_ctx *c, int level, size_t &n) {
    if (level == 3) n = size_t(c->K) * 4 * c->Np;
    else if (level == 2) n = size_t(c->T) * c->P * 3 * c->Np2;
    else if (level == 1) n = size_t(c->L) * c->P * c->P * 2 * c->Np1;
    else return DGH_EINVAL;
    return DGH_OK;
}

float *level_ptr(dgh_ctx *c, int level, bool res) {
    if (level == 3) return res ? c->res3 : c->q3;
    if (level == 2) return res ? c->res2 : c->q2;
    return res ? c->res1 : c->q1;
}

// State transfers convert and reorder on the device: the host copies plain
// FP64 (or FP32) arrays in canonical order, the kernels below map them to and
// from the FP32 device layouts (cell-interleaved for the 3D fields).
template <typename H>
__global__ void k_scatter3(const H *src, float *q, const int *c2d, int64_t n, int per) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / per;
        const int r = (int)(i % per);
        const int64_t kd = c2d[k];
        q[((kd >> 5) * per + r) * 32 + (kd & 31)] = (float)src[i];
    }
}

template <typename H>
__global__ void k_gather3(const float *q, H *dst, const int *c2d, int64_t n, int per) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / per;
        const int r = (int)(i % per);
        const int64_t kd = c2d[k];
        dst[i] = (H)q[((kd >> 5) * per + r) * 32 + (kd & 31)];
    }
}

__global__ void k_d2f(const double *a, float *b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

__global__ void k_f2d(const float *a, double *b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

int xfer_grid(const dgh_ctx *c, size_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)((n + 255) / 256), int64_t(8) * std::max(c->sms, 1)));
}

// Device staging buffer of the 3D state transfers (canonical order on the
// host, cell-interleaved on the device): kept by the context and grown when a
// larger one is needed, so repeated transfers of a large state do not map
// and unmap hundreds of MB on every call.  Callers synchronise the context's
// stream before returning, so one buffer serves every transfer.
cudaError_t xfer_buffer(dgh_ctx *c, size_t bytes, void **p) {
    if (c->xfer_bytes < bytes) {
        if (c->xfer) {
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return e;
            cudaFree(c->xfer);
            c->xfer = nullptr;
            c->xfer_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&c->xfer, bytes);
        if (e != cudaSuccess) {
            c->xfer = nullptr;
            return e;
        }
        c->xfer_bytes = bytes;
    }
    *p = c->xfer;
    return cudaSuccess;
}

// device array dptr (level layout) -> host doubles out (canonical), n values
int copy_out_level(dgh_ctx *c, int level, const float *dptr, double *out, size_t n) {
    if (n == 0) return DGH_OK;
    double *tmp = nullptr;
    cudaError_t e = xfer_buffer(c, n * sizeof(double), (void **)&tmp);
    if (e == cudaSuccess) {
        if (level == 3)
            k_gather3<<<xfer_grid(c, n), 256, 0, c->stream>>>(dptr, tmp, c->can2dev_d, (int64_t)n, 4 * c->Np);
        else
            k_f2d<<<xfer_grid(c, n), 256, 0, c->stream>>>(dptr, tmp, (int64_t)n);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        c->err = std::string("device to host transfer: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    return DGH_OK;
}

// host doubles in (canonical), n values -> device array dptr (level layout)
int copy_in_level(dgh_ctx *c, int level, const double *in, float *dptr, size_t n) {
    if (n == 0) return DGH_OK;
    double *tmp = nullptr;
    cudaError_t e = xfer_buffer(c, n * sizeof(double), (void **)&tmp);
    if (e == cudaSuccess) {
        e = cudaMemcpyAsync(tmp, in, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) {
            if (level == 3)
                k_scatter3<<<xfer_grid(c, n), 256, 0, c->stream>>>(tmp, dptr, c->can2dev_d, (int64_t)n, 4 * c->Np);
            else
                k_d2f<<<xfer_grid(c, n), 256, 0, c->stream>>>(tmp, dptr, (int64_t)n);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        c->err = std::string("host to device transfer: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    return DGH_OK;
}

// FP32 host arrays (canonical order) in the device precision: half the bytes
// of the FP64 transfers.  Levels 2 and 1 have the canonical layout on the
// device as well and are copied straight into the state; level 3 goes
// through the staging buffer and the layout scatter / gather.
int copy_in_level_f32(dgh_ctx *c, int level, const float *in, float *dptr, size_t n) {
    if (n == 0) return DGH_OK;
    cudaError_t e = cudaSuccess;
    if (level != 3) {
        e = cudaMemcpyAsync(dptr, in, n * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    } else {
        float *tmp = nullptr;
        e = xfer_buffer(c, n * sizeof(float), (void **)&tmp);
        if (e == cudaSuccess) {
            e = cudaMemcpyAsync(tmp, in, n * sizeof(float), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) {
                k_scatter3<<<xfer_grid(c, n), 256, 0, c->stream>>>(tmp, dptr, c->can2dev_d, (int64_t)n, 4 * c->Np);
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("host to device transfer: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    return DGH_OK;
}

int copy_out_level_f32(dgh_ctx *c, int level, const float *dptr, float *out, size_t n) {
    if (n == 0) return DGH_OK;
    cudaError_t e = cudaSuccess;
    if (level != 3) {
        e = cudaMemcpyAsync(out, dptr, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    } else {
        float *tmp = nullptr;
        e = xfer_buffer(c, n * sizeof(float), (void **)&tmp);
        if (e == cudaSuccess) {
            k_gather3<<<xfer_grid(c, n), 256, 0, c->stream>>>(dptr, tmp, c->can2dev_d, (int64_t)n, 4 * c->Np);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("device to host transfer: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    return DGH_OK;
}

// Energy of the difference between the 3D fields and a reference field given
// in canonical order (FP64), per cell |J| [d_p^T M d_p / (2 rho c^2) +
// (rho/2) sum_i d_u_i^T M d_u_i], all in FP64 with the FP64 mass matrix.
template <int N>
__global__ void __launch_bounds__(256) k_energy_diff_partial(const float *q, const double *ref, const double *Md,
                                                             const double *ew, const int *c2d, int64_t K,
                                                             double *partial) {
    constexpr int NP = Ord<N>::NP;
    extern __shared__ double sMd[];
    __shared__ double red[256];
    for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) sMd[i] = Md[i];
    __syncthreads();
    double acc = 0.0;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < K * 4; it += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = it / 4;
        const int fl = (int)(it % 4);
        const int64_t kd = c2d[k];
        const float *x = q + (kd >> 5) * (4 * NP * 32) + fl * NP * 32 + (kd & 31);
        const double *r = ref + it * NP;
        double sacc = 0.0;
        for (int n = 0; n < NP; ++n) {
            double y = 0.0;
            for (int m = 0; m < NP; ++m) y += sMd[n * NP + m] * ((double)x[m * 32] - r[m]);
            sacc += ((double)x[n * 32] - r[n]) * y;
        }
        acc += sacc * ew[2 * kd + (fl == 0 ? 0 : 1)];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Energy partial sums of the 3D fields (FP64 throughout), nb blocks on st.
template <int N>
struct EnergyPartial {
    static int run(const float *q, const double *Md, const double *ew, int64_t K, double *partial, int nb, cudaStream_t st) {
        const size_t smem = energy_smem(N);
        cudaFuncSetAttribute(k_energy_partial<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_energy_partial<N><<<nb, 256, smem, st>>>(q, Md, ew, K, partial);
        return DGH_OK;
    }
};

template <int N>
struct EnergyDiff {
    static int run(dgh_ctx *c, const double *dref) {
        constexpr int NP = Ord<N>::NP;
        const size_t smem = sizeof(double) * NP * NP;
        cudaFuncSetAttribute(k_energy_diff_partial<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_energy_diff_partial<N><<<c->energy_blocks, 256, smem, c->stream>>>(c->q3, dref, c->M3d, c->ew, c->can2dev_d,
                                                                            c->K, c->partial);
        return DGH_OK;
    }
};

}  // namespace

// ============================================================================
extern "C" {

const char *dgh_last_error(const dgh_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void dgh_destroy(dgh_ctx *ctx) {
    if (!ctx) return;
    drop_graphs(ctx);
    for (int i = 0; i < 5; ++i) {
        if (ctx->ev3d[i]) cudaEventDestroy(ctx->ev3d[i]);
        if (ctx->ev2d[i]) cudaEventDestroy(ctx->ev2d[i]);
    }
    if (ctx->evjoin) cudaEventDestroy(ctx->evjoin);
    if (ctx->ev_order) cudaEventDestroy(ctx->ev_order);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    for (auto &b : ctx->bufs) cudaFree(b.p);
    if (ctx->xfer) cudaFree(ctx->xfer);
    delete ctx->sh;
    delete ctx;
}

static int validate_desc(const dgh_desc *d) {
    if (!d || !d->vertices || !d->cells || !d->c || !d->rho || d->n_vertices < 4 || d->n_cells < 1) {
        g_create_error = "invalid description (null pointer or empty mesh)";
        return DGH_EINVAL;
    }
    if (d->order < 1 || d->order > 6 || d->habc_order < 0 || d->habc_order > MAXP) {
        g_create_error = "order N must be 1..6 and HABC order P 0..12";
        return DGH_EUNSUPPORTED;
    }
    if (d->precision != DGH_PREC_FP32 && d->precision != DGH_PREC_BF16_TC && d->precision != DGH_PREC_FP16_TC &&
        d->precision != DGH_PREC_SPLIT_BF16 && d->precision != DGH_PREC_FP32_CUDA && d->precision != DGH_PREC_SPLIT_TF32) {
        g_create_error = "unknown precision code";
        return DGH_EUNSUPPORTED;
    }
    if (d->precision == DGH_PREC_SPLIT_TF32 && d->order > kMaxTf32Order) {
        g_create_error = "split-TF32 products are built for N <= 4 (operators and stage exceed shared memory above)";
        return DGH_EUNSUPPORTED;
    }
    if (d->n_cells > (int64_t(1) << 26)) {
        g_create_error = "too many cells for the 32-bit connectivity encoding (max 2^26)";
        return DGH_EUNSUPPORTED;
    }
    for (int f = 0; f < 6; ++f)
        if (d->bc[f] != DGH_BC_HABC && d->bc[f] != DGH_BC_DIRICHLET) {
            g_create_error = "unknown boundary condition code";
            return DGH_EINVAL;
        }
    for (int64_t k = 0; k < d->n_cells; ++k)
        if (!(d->c[k] > 0.0) || !(d->rho[k] > 0.0)) {
            g_create_error = "c and rho must be positive";
            return DGH_EINVAL;
        }
    return DGH_OK;
}

static int host_setup(const dgh_desc *d, HostMesh &m, RefTet &T3, RefTri &T2, RefLine &T1, HabcOps &habc) {
    std::string err;
    const int N = d->order, P = d->habc_order;
    if (!build_tet(N, T3, err)) {
        g_create_error = err;
        return DGH_EINVAL;
    }
    build_tri(N, warp_alpha_tet(N), T2);
    build_line(N, T1);
    m.N = N;
    m.P = P;
    for (int f = 0; f < 6; ++f) m.bc[f] = d->bc[f];
    m.K = d->n_cells;
    m.Nv = d->n_vertices;
    m.VX.assign(d->vertices, d->vertices + 3 * m.Nv);
    m.EToV.assign(d->cells, d->cells + 4 * m.K);
    m.c.assign(d->c, d->c + m.K);
    m.rho.assign(d->rho, d->rho + m.K);
    if (!build_mesh(m, T3, T2, T1, err) || !build_habc(P, habc, err)) {
        g_create_error = err;
        return DGH_EINVAL;
    }
    return DGH_OK;
}

int dgh_plan(const dgh_desc *d, dgh_info *o) {
    return dgh_guarded(nullptr, [&]() -> int {
        if (!o) {
            g_create_error = "out is NULL";
            return DGH_EINVAL;
        }
        int rc = validate_desc(d);
        if (rc) return rc;
        HostMesh m;
        RefTet T3;
        RefTri T2;
        RefLine T1;
        HabcOps habc;
        if ((rc = host_setup(d, m, T3, T2, T1, habc))) return rc;
        std::memset(o, 0, sizeof(*o));
        o->order = d->order;
        o->habc_order = d->habc_order;
        o->Np = T3.Np;
        o->Np2 = T2.Np;
        o->Np1 = T1.Np;
        o->n_corners = int(m.corners.size());
        o->n_cells = m.K;
        o->n_tris = m.Ktri;
        o->n_lines = m.Klin;
        o->n_bfaces = int64_t(m.bface.size());
        const int64_t P = d->habc_order;
        o->ndof = 4 * int64_t(T3.Np) * m.K + 3 * P * T2.Np * m.Ktri + 2 * P * P * T1.Np * m.Klin;
        o->dt = d->dt > 0.0 ? d->dt : dt_rule(m, d->cfl > 0.0 ? d->cfl : 1.0);
        return DGH_OK;
    });
}

}  // extern "C"

// Device arrays of a context whose host set-up (mesh, reference elements,
// HABC operators, dt) is complete.  parts lists the cell offsets of the
// independent problems the mesh is made of ({0, K} for one problem); each
// problem gets its own range of 32-cell blocks.  With one problem the cells
// without HABC faces come first and the cells with HABC faces (whose exterior
// state the 2D kernel writes) last, each group padded to whole blocks, so
// that the two groups can be launched separately; a batch union launches all
// blocks at once (no_overlap).  m.dtCell, when present, holds each cell's own
// time step, which is folded into the rho c^2 and 1/rho coefficients of all
// levels (every right-hand side is proportional to one of them), so that the
// stage kernels advance with dt = 1.
static int build_context(dgh_ctx *ctx, const std::vector<int64_t> &parts) {
    auto fail = [&](int rc, const std::string &msg) {
        if (!msg.empty()) ctx->err = msg;
        return rc;
    };
    const int N = ctx->N, P = ctx->P;
    HostMesh &m = ctx->mesh;
    const RefTet &T3 = ctx->ref3;
    const RefTri &T2 = ctx->ref2;
    const RefLine &T1 = ctx->ref1;
    ctx->Np = T3.Np;
    ctx->Nfp = T3.Nfp;
    ctx->Np2 = T2.Np;
    ctx->Np1 = T1.Np;
    ctx->K = m.K;
    ctx->T = m.Ktri;
    ctx->L = m.Klin;
    ctx->Fb = int64_t(m.bface.size());
    ctx->C = int(m.corners.size());
    ctx->M = ctx->habc.M;
    const int64_t K = m.K;
    const int Np = T3.Np, Nfp = T3.Nfp, Np2 = T2.Np, Np1 = T1.Np;
    auto fold = [&](int64_t k) { return m.dtCell.empty() ? 1.0 : m.dtCell[size_t(k)]; };
    int rc;
    // ---------------------------------------------------------------- 3D
    // Cell-interleaved tiles of 32 cells: q, res [K32][4][Np][32], geometry
    // [K32][GEO3][32], connectivity [K32][4][32]; traces [K32*32][4][2][Nfp].
    {
        const int nparts = int(parts.size()) - 1;
        std::vector<char> habc_cell(size_t(K), 0);
        for (int64_t t = 0; t < m.Ktri; ++t) habc_cell[m.bface[m.triBface[t]] / 4] = 1;
        ctx->can2dev.assign(size_t(K), -1);
        ctx->part_blk0.assign(size_t(nparts) + 1, 0);
        int64_t blk = 0;
        for (int pp = 0; pp < nparts; ++pp) {
            int64_t ni = 0, nb = 0;
            for (int64_t k = parts[pp]; k < parts[pp + 1]; ++k) (habc_cell[k] ? nb : ni)++;
            const int64_t bi = (ni + 31) / 32, bb = (nb + 31) / 32;
            int64_t pi = blk * 32, pb = (blk + bi) * 32;
            for (int64_t k = parts[pp]; k < parts[pp + 1]; ++k) ctx->can2dev[k] = habc_cell[k] ? pb++ : pi++;
            ctx->part_blk0[pp] = blk;
            if (nparts == 1) {
                ctx->Ki32 = bi;
                ctx->Kb32 = bb;
            }
            blk += bi + bb;
        }
        ctx->part_blk0[nparts] = blk;
        ctx->K32 = blk;
        if (nparts != 1) {
            ctx->Ki32 = blk;
            ctx->Kb32 = 0;
            ctx->no_overlap = true;
        }
    }
    if (ctx->K32 * 32 * 4 >= (int64_t(1) << 28)) return fail(DGH_EUNSUPPORTED, "too many cells for the 32-bit connectivity encoding");
    {
        const int64_t K32 = ctx->K32, Kp = K32 * 32;
        int NW = 1, C = 1, CP = 4;
        switch (N) {
            case 1: NW = Cfg3<1>::NW; C = Cfg3<1>::C; CP = Cfg3<1>::CP; break;
            case 2: NW = Cfg3<2>::NW; C = Cfg3<2>::C; CP = Cfg3<2>::CP; break;
            case 3: NW = Cfg3<3>::NW; C = Cfg3<3>::C; CP = Cfg3<3>::CP; break;
            case 4: NW = Cfg3<4>::NW; C = Cfg3<4>::C; CP = Cfg3<4>::CP; break;
            case 5: NW = Cfg3<5>::NW; C = Cfg3<5>::C; CP = Cfg3<5>::CP; break;
            case 6: NW = Cfg3<6>::NW; C = Cfg3<6>::C; CP = Cfg3<6>::CP; break;
        }
        std::vector<float> geo(size_t(Kp) * GEO3, 0.f);
        std::vector<int> conn(size_t(Kp) * 4, kPadConn);
        std::vector<double> cellv(size_t(Kp) * 12, 0.0), ew(size_t(Kp) * 2, 0.0);
        auto G = [&](int64_t kd, int q) -> float & { return geo[(size_t(kd / 32) * GEO3 + q) * 32 + (kd % 32)]; };
        auto CN = [&](int64_t kd, int f) -> int & { return conn[(size_t(kd / 32) * 4 + f) * 32 + (kd % 32)]; };
        // padding cells: identity metric, unit impedance (their results are never read)
        for (int64_t kd = 0; kd < Kp; ++kd) {
            G(kd, 0) = G(kd, 4) = G(kd, 8) = 1.f;
            for (int f = 0; f < 4; ++f) G(kd, 9 + f) = 1.f;
            G(kd, 13) = G(kd, 14) = G(kd, 15) = 1.f;
        }
        for (int64_t k = 0; k < K; ++k) {
            const int64_t kd = ctx->can2dev[k];
            for (int q = 0; q < 9; ++q) G(kd, q) = float(m.drdx[9 * k + q]);
            const double Z = m.rho[k] * m.c[k];
            for (int f = 0; f < 4; ++f) {
                const int64_t nb = m.nbr[4 * k + f];
                double Zp = Z;
                if (nb >= 0) Zp = m.rho[nb / 4] * m.c[nb / 4];
                G(kd, 9 + f) = float(Zp);
                if (nb >= 0) {
                    CN(kd, f) = int(((ctx->can2dev[nb / 4] * 4 + nb % 4) << 3) | m.nbrSigma[4 * k + f]);
                } else {
                    const int64_t b = m.bfaceOf[4 * k + f];
                    const int dir = m.bfaceDir[b] ? 1 : 0;
                    CN(kd, f) = int(-1 - ((b << 1) | dir));
                }
            }
            G(kd, 13) = float(m.rho[k] * m.c[k] * m.c[k] * fold(k));
            G(kd, 14) = float(fold(k) / m.rho[k]);
            G(kd, 15) = float(Z);
            for (int v = 0; v < 4; ++v)
                for (int dd = 0; dd < 3; ++dd) cellv[12 * kd + 3 * v + dd] = m.VX[3 * m.EToV[4 * k + v] + dd];
            ew[2 * kd] = std::fabs(m.J[k]) / (2.0 * m.rho[k] * m.c[k] * m.c[k]);
            ew[2 * kd + 1] = std::fabs(m.J[k]) * 0.5 * m.rho[k];
        }
        // D rows of output chunk w (nodes w*C .. w*C+C-1), padded to CP: [m][j][w][CP]
        std::vector<float> D(size_t(Np) * 3 * NW * CP, 0.f), Lf(size_t(4) * Nfp * NW * CP, 0.f), Mf(size_t(Np) * Np);
        const Mat *Dj[3] = {&T3.Dr, &T3.Ds, &T3.Dt};
        for (int mm = 0; mm < Np; ++mm)
            for (int j = 0; j < 3; ++j)
                for (int w = 0; w < NW; ++w)
                    for (int c = 0; c < C; ++c) {
                        const int n = w * C + c;
                        if (n < Np) D[((size_t(mm) * 3 + j) * NW + w) * CP + c] = float((*Dj[j])(n, mm));
                    }
        for (int fm = 0; fm < 4 * Nfp; ++fm)
            for (int w = 0; w < NW; ++w)
                for (int c = 0; c < C; ++c) {
                    const int n = w * C + c;
                    if (n < Np) Lf[(size_t(fm) * NW + w) * CP + c] = float(T3.LIFT(n, fm));
                }
        for (size_t i = 0; i < Mf.size(); ++i) Mf[i] = float(T3.M.a[i]);
        std::vector<int> fmask(4 * Nfp), fperm(6 * Nfp), nslot(size_t(Np) * 3, -1);
        for (int f = 0; f < 4; ++f)
            for (int q = 0; q < Nfp; ++q) {
                const int n = T3.Fmask[f][q];
                fmask[f * Nfp + q] = n;
                for (int sl = 0; sl < 3; ++sl)
                    if (nslot[3 * n + sl] < 0) {
                        nslot[3 * n + sl] = f * Nfp + q;
                        break;
                    }
            }
        for (int sg = 0; sg < 6; ++sg)
            for (int q = 0; q < Nfp; ++q) fperm[sg * Nfp + q] = T3.facePerm[sg][q];
        std::vector<double> rst(size_t(3) * Np);
        for (int n = 0; n < Np; ++n) {
            rst[3 * n] = T3.r[n];
            rst[3 * n + 1] = T3.s[n];
            rst[3 * n + 2] = T3.t[n];
        }
        if ((rc = dalloc(ctx, ctx->q3, size_t(Kp) * 4 * Np)) || (rc = dalloc(ctx, ctx->res3, size_t(Kp) * 4 * Np)) ||
            (rc = dalloc(ctx, ctx->tin3[0], size_t(Kp) * 8 * Nfp)) || (rc = dalloc(ctx, ctx->tin3[1], size_t(Kp) * 8 * Nfp)) ||
            (rc = dalloc(ctx, ctx->trb, size_t(std::max<int64_t>(ctx->Fb, 1)) * 2 * Nfp)) ||
            (rc = dalloc(ctx, ctx->d_err, 1)) || (rc = upload(ctx, ctx->geo3, geo)) ||
            (rc = upload(ctx, ctx->conn3, conn)) || (rc = upload(ctx, ctx->D3, D)) || (rc = upload(ctx, ctx->L3, Lf)) ||
            (rc = upload(ctx, ctx->M3, Mf)) || (rc = upload(ctx, ctx->fmask3, fmask)) ||
            (rc = upload(ctx, ctx->fperm3, fperm)) || (rc = upload(ctx, ctx->nslot3, nslot)) ||
            (rc = upload(ctx, ctx->cellv, cellv)) || (rc = upload(ctx, ctx->rst, rst)) || (rc = upload(ctx, ctx->ew, ew)))
            return fail(rc, "");
        const int kern = kern3_of(ctx->precision, N, ctx->K);
        if (kern == K3_TC && (rc = upload(ctx, ctx->tcops, tc_operator_images(T3, ctx->precision)))) return fail(rc, "");
        if (kern == K3_TF32 && (rc = upload(ctx, ctx->tcops, tf32_operator_images(T3)))) return fail(rc, "");
        std::vector<int> c2d(ctx->can2dev.begin(), ctx->can2dev.end());
        if ((rc = upload(ctx, ctx->can2dev_d, c2d)) || (rc = upload(ctx, ctx->M3d, T3.M.a))) return fail(rc, "");
    }
    // ---------------------------------------------------------------- 2D
    const int64_t Tn = m.Ktri;
    {
        std::vector<float> geo(size_t(Tn) * GEO2, 0.f);
        std::vector<int> conn(size_t(Tn) * 3), tface(Tn), tb(Tn);
        for (int64_t t = 0; t < Tn; ++t) {
            float *g = &geo[size_t(t) * GEO2];
            for (int q = 0; q < 4; ++q) g[q] = float(m.drdx2[4 * t + q]);
            const int64_t gf = m.bface[m.triBface[t]];
            const int64_t k = gf / 4;
            const double Z = m.rho[k] * m.c[k];
            for (int e = 0; e < 3; ++e) {
                float *ge = g + 4 + 6 * e;
                ge[0] = float(m.nrm2[6 * t + 2 * e]);
                ge[1] = float(m.nrm2[6 * t + 2 * e + 1]);
                ge[2] = float(m.fscale2[3 * t + e]);
                const int64_t nb = m.nbr2[3 * t + e];
                double Zp = Z;
                if (nb >= 0) {
                    const int64_t kn = m.bface[m.triBface[nb / 3]] / 4;
                    Zp = m.rho[kn] * m.c[kn];
                    conn[3 * t + e] = int((nb << 1) | m.flip2[3 * t + e]);
                } else {
                    conn[3 * t + e] = m.edgeDir[3 * t + e] ? -2 : -1;
                }
                ge[3] = float(Z / (Z + Zp));
                ge[4] = float(Z * Zp / (Z + Zp));
                ge[5] = float(1.0 / (Z + Zp));
            }
            g[22] = float(m.rho[k] * m.c[k] * m.c[k] * fold(k));
            g[23] = float(fold(k) / m.rho[k]);
            g[24] = float(Z);
            tface[t] = int(ctx->can2dev[gf / 4] * 4 + gf % 4);
            tb[t] = int(m.triBface[t]);
        }
        std::vector<float> D(size_t(2) * Np2 * Np2), Lf(size_t(3) * (N + 1) * Np2);
        for (int n = 0; n < Np2; ++n)
            for (int mm = 0; mm < Np2; ++mm) {
                D[size_t(mm) * Np2 + n] = float(T2.Dr(n, mm));
                D[(size_t(Np2) + mm) * Np2 + n] = float(T2.Ds(n, mm));
            }
        for (int n = 0; n < Np2; ++n)
            for (int em = 0; em < 3 * (N + 1); ++em) Lf[size_t(em) * Np2 + n] = float(T2.LIFT(n, em));
        std::vector<int> fmask(3 * (N + 1));
        for (int e = 0; e < 3; ++e)
            for (int q = 0; q <= N; ++q) fmask[e * (N + 1) + q] = T2.Fmask[e][q];
        const size_t nq = size_t(Tn) * P * 3 * Np2;
        if ((rc = dalloc(ctx, ctx->q2, nq)) || (rc = dalloc(ctx, ctx->res2, nq)) ||
            (rc = dalloc(ctx, ctx->tr2[0], size_t(Tn) * P * 3 * 2 * (N + 1))) ||
            (rc = dalloc(ctx, ctx->tr2[1], size_t(Tn) * P * 3 * 2 * (N + 1))) ||
            (rc = dalloc(ctx, ctx->qb2, size_t(Tn) * 3 * P * (N + 1))) || (rc = dalloc(ctx, ctx->q0_3, size_t(Tn) * Np2)) ||
            (rc = upload(ctx, ctx->geo2, geo)) || (rc = upload(ctx, ctx->conn2, conn)) ||
            (rc = upload(ctx, ctx->tri_face, tface)) || (rc = upload(ctx, ctx->tri_bface, tb)) ||
            (rc = upload(ctx, ctx->D2, D)) || (rc = upload(ctx, ctx->L2, Lf)) || (rc = upload(ctx, ctx->fmask2, fmask)))
            return fail(rc, "");
    }
    // ---------------------------------------------------------------- 1D
    const int64_t Ln = m.Klin;
    {
        std::vector<float> geo(size_t(Ln) * GEO1, 0.f);
        std::vector<int> conn(size_t(Ln) * 2), lmap(size_t(Ln) * 6);
        for (int64_t l = 0; l < Ln; ++l) {
            float *g = &geo[size_t(l) * GEO1];
            const int64_t tA = m.linTri[0][l], tB = m.linTri[1][l];
            const int64_t kA = m.bface[m.triBface[tA]] / 4, kB = m.bface[m.triBface[tB]] / 4;
            const double ZA = m.rho[kA] * m.c[kA], ZB = m.rho[kB] * m.c[kB];
            const double Z = ZA;   // a line cell takes the material of its face-A triangle
            g[0] = float(1.0 / m.J1[l]);
            g[1] = float(1.0 / std::fabs(m.J1[l]));
            g[2] = float(m.rho[kA] * m.c[kA] * m.c[kA] * fold(kA));
            g[3] = float(fold(kA) / m.rho[kA]);
            g[4] = float(Z);
            g[5] = float(ZA);
            g[6] = float(ZB);
            for (int e = 0; e < 2; ++e) {
                const int64_t nb = m.nbr1[2 * l + e];
                double Zp = Z;
                if (nb >= 0) {
                    const int64_t kn = m.bface[m.triBface[m.linTri[0][nb / 2]]] / 4;
                    Zp = m.rho[kn] * m.c[kn];
                    conn[2 * l + e] = int(nb);
                } else {
                    conn[2 * l + e] = m.endDir[2 * l + e] ? -2 : -1;
                }
                g[7 + 3 * e] = float(Z / (Z + Zp));
                g[8 + 3 * e] = float(Z * Zp / (Z + Zp));
                g[9 + 3 * e] = float(1.0 / (Z + Zp));
            }
            for (int s = 0; s < 2; ++s) {
                lmap[6 * l + 3 * s] = int(m.linTri[s][l]);
                lmap[6 * l + 3 * s + 1] = m.linEdge[s][l];
                lmap[6 * l + 3 * s + 2] = m.linRev[s][l];
            }
        }
        std::vector<float> D(size_t(Np1) * Np1), Lf(size_t(2) * Np1);
        for (int n = 0; n < Np1; ++n)
            for (int mm = 0; mm < Np1; ++mm) D[size_t(mm) * Np1 + n] = float(T1.Dr(n, mm));
        for (int n = 0; n < Np1; ++n) {
            Lf[n] = float(T1.LIFT(n, 0));
            Lf[Np1 + n] = float(T1.LIFT(n, 1));
        }
        const size_t nq = size_t(Ln) * P * P * 2 * Np1;
        std::vector<float> cP(std::max(P, 1), 0.f);
        for (int a = 0; a < P; ++a) cP[a] = float(ctx->habc.c[a]);
        if ((rc = dalloc(ctx, ctx->q1, nq)) || (rc = dalloc(ctx, ctx->res1, nq)) ||
            (rc = dalloc(ctx, ctx->tr1[0], size_t(Ln) * P * P * 4)) || (rc = dalloc(ctx, ctx->tr1[1], size_t(Ln) * P * P * 4)) ||
            (rc = dalloc(ctx, ctx->qb1, size_t(Ln) * 2 * P * P)) || (rc = dalloc(ctx, ctx->q0_2, size_t(Ln) * 2 * P * Np1)) ||
            (rc = upload(ctx, ctx->geo1, geo)) || (rc = upload(ctx, ctx->conn1, conn)) || (rc = upload(ctx, ctx->lmap, lmap)) ||
            (rc = upload(ctx, ctx->D1, D)) || (rc = upload(ctx, ctx->L1, Lf)) || (rc = upload(ctx, ctx->cP, cP)))
            return fail(rc, "");
        if (P >= 1) {
            if ((rc = upload(ctx, ctx->H1, to_f(ctx->habc.H1))) || (rc = upload(ctx, ctx->H2, to_f(ctx->habc.H2))) ||
                (rc = upload(ctx, ctx->Hc, to_f(ctx->habc.Hc))))
                return fail(rc, "");
        }
    }
    // ---------------------------------------------------------------- 0D
    {
        std::vector<int> cor(size_t(ctx->C) * 6);
        std::vector<float> cz(size_t(ctx->C) * 3);
        for (int c = 0; c < ctx->C; ++c)
            for (int sl = 0; sl < 3; ++sl) {
                const int64_t l = m.corners[c].line[sl];
                cor[6 * c + 2 * sl] = int(l);
                cor[6 * c + 2 * sl + 1] = m.corners[c].end[sl];
                const int64_t kA = m.bface[m.triBface[m.linTri[0][l]]] / 4;
                cz[3 * c + sl] = float(m.rho[kA] * m.c[kA]);
            }
        if ((rc = upload(ctx, ctx->corner, cor)) || (rc = upload(ctx, ctx->cornerZ, cz))) return fail(rc, "");
    }
    // ---------------------------------------------------------------- misc
    if ((rc = dalloc(ctx, ctx->tile_ctr, 16)) || (rc = dalloc(ctx, ctx->tile_ctr2, 4)) ||
        (rc = dalloc(ctx, ctx->d_time, 1)) || (rc = dalloc(ctx, ctx->d_step, 1)) ||
        (rc = dalloc(ctx, ctx->srcvec, size_t(MAXSRC) * Np)) || (rc = dalloc(ctx, ctx->d_energy, 1)))
        return fail(rc, "");
    ctx->energy_blocks = 2 * 148;
    if ((rc = dalloc(ctx, ctx->partial, ctx->energy_blocks))) return fail(rc, "");
    // launch shapes
    ctx->thr2 = 128;
    ctx->tile2 = k2d_tile_max(P, ctx->thr2);
    ctx->tile1 = std::max(1, 256 / std::max(1, P * P * Np1));
    if ((rc = dispatchN<SetAttrs>(N, ctx))) return fail(rc, "");
    if ((rc = dispatchN<Shapes>(N, ctx))) return fail(DGH_EUNSUPPORTED, "2D/1D tile does not fit in shared memory");
    {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, hi) != cudaSuccess) return fail(DGH_ECUDA, "side stream");

    }
    for (int i = 0; i < 5; ++i)
        if (cudaEventCreateWithFlags(&ctx->ev3d[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev2d[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(DGH_ECUDA, "events");
    if (cudaEventCreateWithFlags(&ctx->evjoin, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_order, cudaEventDisableTiming) != cudaSuccess)
        return fail(DGH_ECUDA, "events");
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(DGH_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
    return DGH_OK;
}

extern "C" {

int dgh_create(const dgh_desc *d, void *stream, dgh_ctx **out) {
    return dgh_guarded(nullptr, [&]() -> int {
        ApiRange nvtx_range("dgh_create");
        if (!out) {
            g_create_error = "out is NULL";
            return DGH_EINVAL;
        }
        *out = nullptr;
        int vrc = validate_desc(d);
        if (vrc) return vrc;
        struct Owner {   // destroys the partly built context on every failure, thrown or returned
            dgh_ctx *c;
            ~Owner() { if (c) dgh_destroy(c); }
        } owner{new dgh_ctx()};
        dgh_ctx *ctx = owner.c;
        ctx->stream = static_cast<cudaStream_t>(stream);
        cudaGetDevice(&ctx->device);
        ctx->N = d->order;
        ctx->P = d->habc_order;
        ctx->precision = d->precision;
        int rc = host_setup(d, ctx->mesh, ctx->ref3, ctx->ref2, ctx->ref1, ctx->habc);
        if (rc) return rc;
        ctx->cfl = d->cfl > 0.0 ? d->cfl : 1.0;
        ctx->dt_fixed = d->dt > 0.0;
        ctx->dt = d->dt > 0.0 ? d->dt : dt_rule(ctx->mesh, ctx->cfl);
        rc = build_context(ctx, {0, ctx->mesh.K});
        if (rc) {
            g_create_error = ctx->err;
            return rc;
        }
        *out = ctx;
        owner.c = nullptr;
        return DGH_OK;
    });
}

int dgh_get_info(const dgh_ctx *ctx, dgh_info *o) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !o) return DGH_EINVAL;
        o->order = ctx->N;
        o->habc_order = ctx->P;
        o->Np = ctx->Np;
        o->Np2 = ctx->Np2;
        o->Np1 = ctx->Np1;
        o->n_corners = ctx->C;
        o->n_cells = ctx->K;
        o->n_tris = ctx->T;
        o->n_lines = ctx->L;
        o->n_bfaces = ctx->Fb;
        o->ndof = 4 * int64_t(ctx->Np) * ctx->K + 3 * int64_t(ctx->P) * ctx->Np2 * ctx->T +
                  2 * int64_t(ctx->P) * ctx->P * ctx->Np1 * ctx->L;
        o->step_count = ctx->step_count;
        o->dt = ctx->dt;
        o->time = ctx->t0 + ctx->step_count * 0.0;
        o->device_bytes = ctx->device_bytes;
        double t = 0.0;
        if (cudaMemcpy(&t, ctx->d_time, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess) o->time = t;
        return DGH_OK;
    });
}

int dgh_get_nodes(const dgh_ctx *ctx, int level, double *xyz, size_t count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !xyz) return DGH_EINVAL;
        const HostMesh &m = ctx->mesh;
        if (level == 3) {
            if (count != size_t(ctx->K) * ctx->Np * 3) return DGH_EINVAL;
            for (int64_t k = 0; k < ctx->K; ++k)
                for (int n = 0; n < ctx->Np; ++n) {
                    const double r = ctx->ref3.r[n], s = ctx->ref3.s[n], t = ctx->ref3.t[n];
                    const double l[4] = {-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2};
                    for (int d = 0; d < 3; ++d) {
                        double x = 0;
                        for (int v = 0; v < 4; ++v) x += l[v] * m.VX[3 * m.EToV[4 * k + v] + d];
                        xyz[(size_t(k) * ctx->Np + n) * 3 + d] = x;
                    }
                }
            return DGH_OK;
        }
        if (level == 2) {
            if (count != size_t(ctx->T) * ctx->Np2 * 3) return DGH_EINVAL;
            for (int64_t t = 0; t < ctx->T; ++t)
                for (int n = 0; n < ctx->Np2; ++n) {
                    const double r = ctx->ref2.r[n], s = ctx->ref2.s[n];
                    const double l[3] = {-(r + s) / 2, (1 + r) / 2, (1 + s) / 2};
                    for (int d = 0; d < 3; ++d) {
                        double x = 0;
                        for (int v = 0; v < 3; ++v) x += l[v] * m.VX[3 * m.triV[3 * t + v] + d];
                        xyz[(size_t(t) * ctx->Np2 + n) * 3 + d] = x;
                    }
                }
            return DGH_OK;
        }
        if (level == 1) {
            if (count != size_t(ctx->L) * ctx->Np1 * 3) return DGH_EINVAL;
            for (int64_t l = 0; l < ctx->L; ++l)
                for (int n = 0; n < ctx->Np1; ++n) {
                    const double r = ctx->ref1.r[n];
                    for (int d = 0; d < 3; ++d)
                        xyz[(size_t(l) * ctx->Np1 + n) * 3 + d] =
                            (1 - r) / 2 * m.VX[3 * m.linV[2 * l] + d] + (1 + r) / 2 * m.VX[3 * m.linV[2 * l + 1] + d];
                }
            return DGH_OK;
        }
        const_cast<dgh_ctx *>(ctx)->err = "level must be 3, 2 or 1";
        return DGH_EINVAL;
    });
}

int dgh_set_time(dgh_ctx *ctx, double t) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx) return DGH_EINVAL;
        CK(cudaMemcpyAsync(ctx->d_time, &t, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return DGH_OK;
    });
}

int dgh_init_gaussian(dgh_ctx *ctx, const double x0[3], double width, double amp) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !x0 || !(width > 0.0)) return DGH_EINVAL;
        for (int lv = 1; lv <= 3; ++lv) {
            size_t n;
            level_count(ctx, lv, n);
            if (lv == 3) n = size_t(ctx->K32) * 32 * 4 * ctx->Np;
            CK(cudaMemsetAsync(level_ptr(ctx, lv, false), 0, n * sizeof(float), ctx->stream));
            CK(cudaMemsetAsync(level_ptr(ctx, lv, true), 0, n * sizeof(float), ctx->stream));
        }
        if (ctx->sh) {   // shadow chain restarts at zero with the fields
            dgh_ctx::Shadow *h = ctx->sh;
            const size_t n2 = size_t(ctx->T) * h->P * 3 * ctx->Np2, n1 = size_t(ctx->L) * h->P * h->P * 2 * ctx->Np1;
            CK(cudaMemsetAsync(h->q2, 0, std::max<size_t>(n2, 1) * sizeof(float), ctx->stream));
            CK(cudaMemsetAsync(h->res2, 0, std::max<size_t>(n2, 1) * sizeof(float), ctx->stream));
            CK(cudaMemsetAsync(h->q1, 0, std::max<size_t>(n1, 1) * sizeof(float), ctx->stream));
            CK(cudaMemsetAsync(h->res1, 0, std::max<size_t>(n1, 1) * sizeof(float), ctx->stream));
        }
        const int64_t total = ctx->K32 * 32 * ctx->Np;
        const int blocks = int((total + 255) / 256);
        switch (ctx->N) {
            case 1: k_init_gaussian<1><<<blocks, 256, 0, ctx->stream>>>(ctx->q3, ctx->cellv, ctx->rst, ctx->K32 * 32, x0[0], x0[1], x0[2], width, amp); break;
            case 2: k_init_gaussian<2><<<blocks, 256, 0, ctx->stream>>>(ctx->q3, ctx->cellv, ctx->rst, ctx->K32 * 32, x0[0], x0[1], x0[2], width, amp); break;
            case 3: k_init_gaussian<3><<<blocks, 256, 0, ctx->stream>>>(ctx->q3, ctx->cellv, ctx->rst, ctx->K32 * 32, x0[0], x0[1], x0[2], width, amp); break;
            case 4: k_init_gaussian<4><<<blocks, 256, 0, ctx->stream>>>(ctx->q3, ctx->cellv, ctx->rst, ctx->K32 * 32, x0[0], x0[1], x0[2], width, amp); break;
            case 5: k_init_gaussian<5><<<blocks, 256, 0, ctx->stream>>>(ctx->q3, ctx->cellv, ctx->rst, ctx->K32 * 32, x0[0], x0[1], x0[2], width, amp); break;
            case 6: k_init_gaussian<6><<<blocks, 256, 0, ctx->stream>>>(ctx->q3, ctx->cellv, ctx->rst, ctx->K32 * 32, x0[0], x0[1], x0[2], width, amp); break;
        }
        CK(cudaGetLastError());
        ctx->step_count = 0;
        ctx->t0 = 0.0;
        CK(cudaMemsetAsync(ctx->d_time, 0, sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(ctx->d_step, 0, sizeof(int64_t), ctx->stream));
        ctx->dirty = true;
        CK(cudaStreamSynchronize(ctx->stream));
        return DGH_OK;
    });
}

int dgh_init_fields(dgh_ctx *ctx, const double *q3d, size_t count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !q3d) return DGH_EINVAL;
        size_t n;
        level_count(ctx, 3, n);
        if (count != n) {
            ctx->err = "state size mismatch";
            return DGH_EINVAL;
        }
        const double x0[3] = {0.0, 0.0, 0.0};
        int rc = dgh_init_gaussian(ctx, x0, 1.0, 0.0);   // every level and the clock to zero
        if (rc) return rc;
        return dgh_set_state(ctx, 3, q3d, count);
    });
}

int dgh_set_material(dgh_ctx *ctx, const double *c, const double *rho, size_t count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !c || !rho) return DGH_EINVAL;
        if (count != size_t(ctx->mesh.K)) {
            ctx->err = "material: one (c, rho) per cell";
            return DGH_EINVAL;
        }
        if (ctx->no_overlap || ctx->part_blk0.size() > 2) {
            ctx->err = "material: not for a batch group";
            return DGH_ESTATE;
        }
        for (size_t k = 0; k < count; ++k)
            if (!(c[k] > 0.0) || !(rho[k] > 0.0) || !std::isfinite(c[k]) || !std::isfinite(rho[k])) {
                ctx->err = "material: c and rho must be positive and finite";
                return DGH_EINVAL;
            }
        // the state (all levels, time, step count) moves through a checkpoint blob
        size_t sz = 0;
        int rc = dgh_save_state(ctx, nullptr, &sz);
        if (rc) return rc;
        std::vector<char> blob(sz);
        if ((rc = dgh_save_state(ctx, blob.data(), &sz))) return rc;
        dgh_ctx *n = new dgh_ctx();
        n->stream = ctx->stream;
        n->device = ctx->device;
        n->N = ctx->N;
        n->P = ctx->P;
        n->precision = ctx->precision;
        n->mesh = ctx->mesh;
        n->mesh.c.assign(c, c + count);
        n->mesh.rho.assign(rho, rho + count);
        n->ref3 = ctx->ref3;
        n->ref2 = ctx->ref2;
        n->ref1 = ctx->ref1;
        n->habc = ctx->habc;
        n->cfl = ctx->cfl;
        n->dt_fixed = ctx->dt_fixed;
        n->dt = ctx->dt_fixed ? ctx->dt : dt_rule(n->mesh, ctx->cfl);
        n->t0 = ctx->t0;
        auto give_up = [&](int code) {
            ctx->err = n->err;
            dgh_destroy(n);
            return code;
        };
        if ((rc = build_context(n, {0, n->mesh.K}))) return give_up(rc);
        // sources, launch shapes and the watchdog carry over; the closure and a
        // recording shadow chain do not (set them again)
        n->src = ctx->src;
        if (ctx->src.n > 0 && cudaMemcpy(n->srcvec, ctx->srcvec, sizeof(float) * MAXSRC * ctx->Np,
                                         cudaMemcpyDeviceToDevice) != cudaSuccess)
            return give_up(DGH_ECUDA);
        n->tile2 = ctx->tile2;
        n->tile1 = ctx->tile1;
        n->cta3_per_sm = ctx->cta3_per_sm;
        n->sm3_div = ctx->sm3_div;
        n->split3 = ctx->split3;
        n->thr2 = ctx->thr2;
        n->thr1 = ctx->thr1;
        if (dispatchN<Shapes>(n->N, n) != DGH_OK) return give_up(DGH_EINVAL);
        n->wd_every = ctx->wd_every;
        n->wd_limit = ctx->wd_limit;
        if ((rc = dgh_load_state(n, blob.data(), sz))) return give_up(rc);
        std::swap(*ctx, *n);   // the handle keeps its address; n now holds the old context
        dgh_destroy(n);
        return DGH_OK;
    });
}

int dgh_set_material_layers(dgh_ctx *ctx, int nlayers, const double *z_top, const double *c, const double *rho) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || nlayers < 1 || !c || !rho || (nlayers > 1 && !z_top)) return DGH_EINVAL;
        for (int l = 0; l + 2 < nlayers; ++l)
            if (!(z_top[l] < z_top[l + 1])) {
                ctx->err = "material layers: z_top must increase";
                return DGH_EINVAL;
            }
        const HostMesh &m = ctx->mesh;
        std::vector<double> cc(size_t(m.K)), rr(size_t(m.K));
        for (int64_t k = 0; k < m.K; ++k) {
            double z = 0.0;
            for (int v = 0; v < 4; ++v) z += m.VX[size_t(m.EToV[size_t(k) * 4 + v]) * 3 + 2];
            z *= 0.25;
            int l = 0;
            while (l < nlayers - 1 && z_top[l] <= z) ++l;   // layer l holds z < z_top[l]
            cc[size_t(k)] = c[l];
            rr[size_t(k)] = rho[l];
        }
        return dgh_set_material(ctx, cc.data(), rr.data(), cc.size());
    });
}

int dgh_set_state(dgh_ctx *ctx, int level, const double *in, size_t count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        ApiRange nvtx_range("dgh_set_state");
        if (!ctx || (!in && count)) return DGH_EINVAL;
        size_t n;
        if (level_count(ctx, level, n) || n != count) {
            if (ctx) ctx->err = "state size mismatch";
            return DGH_EINVAL;
        }
        if (n == 0) return DGH_OK;
        int rc = copy_in_level(ctx, level, in, level_ptr(ctx, level, false), n);
        if (rc) return rc;
        ctx->dirty = true;
        return DGH_OK;
    });
}

int dgh_get_state(dgh_ctx *ctx, int level, double *out, size_t count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        ApiRange nvtx_range("dgh_get_state");
        if (!ctx || (!out && count)) return DGH_EINVAL;
        size_t n;
        if (level_count(ctx, level, n) || n != count) {
            ctx->err = "state size mismatch";
            return DGH_EINVAL;
        }
        return copy_out_level(ctx, level, level_ptr(ctx, level, false), out, n);
    });
}

int dgh_set_state_f32(dgh_ctx *ctx, int level, const float *in, size_t count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        ApiRange nvtx_range("dgh_set_state_f32");
        if (!ctx || (!in && count)) return DGH_EINVAL;
        size_t n;
        if (level_count(ctx, level, n) || n != count) {
            ctx->err = "state size mismatch";
            return DGH_EINVAL;
        }
        if (n == 0) return DGH_OK;
        int rc = copy_in_level_f32(ctx, level, in, level_ptr(ctx, level, false), n);
        if (rc) return rc;
        ctx->dirty = true;
        return DGH_OK;
    });
}

int dgh_get_state_f32(dgh_ctx *ctx, int level, float *out, size_t count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        ApiRange nvtx_range("dgh_get_state_f32");
        if (!ctx || (!out && count)) return DGH_EINVAL;
        size_t n;
        if (level_count(ctx, level, n) || n != count) {
            ctx->err = "state size mismatch";
            return DGH_EINVAL;
        }
        return copy_out_level_f32(ctx, level, level_ptr(ctx, level, false), out, n);
    });
}

int dgh_get_fields(dgh_ctx *ctx, int level, double *out, size_t count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || (!out && count)) return DGH_EINVAL;
        size_t n;
        if (level_count(ctx, level, n) || n != count) {
            ctx->err = "field size mismatch";
            return DGH_EINVAL;
        }
        if (level == 3) return copy_out_level(ctx, 3, ctx->q3, out, n);
        if (n == 0) return DGH_OK;
        if (ctx->dirty) {
            int rc = run_closure(ctx);
            if (rc) return rc;
        }
        float *tmp = nullptr;
        CK(cudaMallocAsync((void **)&tmp, n * sizeof(float), ctx->stream));
        const int blocks = int((n + 255) / 256);
        if (level == 2)
            k_full2<<<blocks, 256, 0, ctx->stream>>>(ctx->q2, ctx->q0_3, tmp, ctx->T, ctx->P, ctx->Np2);
        else
            k_full1<<<blocks, 256, 0, ctx->stream>>>(ctx->q1, ctx->q0_2, ctx->cP, tmp, ctx->L, ctx->P, ctx->Np1);
        int rc = copy_out_level(ctx, level, tmp, out, n);
        cudaFreeAsync(tmp, ctx->stream);
        return rc;
    });
}

int dgh_add_point_source(dgh_ctx *ctx, const double xs[3], double f_peak, double t_s, double amp) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !xs) return DGH_EINVAL;
        if (ctx->src.n >= MAXSRC) {
            ctx->err = "too many sources";
            return DGH_EINVAL;
        }
        const HostMesh &m = ctx->mesh;
        for (int64_t k = 0; k < m.K; ++k) {
            const double *v0 = &m.VX[3 * m.EToV[4 * k]];
            double c0[3];
            for (int d = 0; d < 3; ++d)
                c0[d] = 0.5 * (m.VX[3 * m.EToV[4 * k + 1] + d] + m.VX[3 * m.EToV[4 * k + 2] + d] + m.VX[3 * m.EToV[4 * k + 3] + d] - v0[d]);
            double rst[3] = {0, 0, 0};
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i) rst[j] += m.drdx[9 * k + 3 * j + i] * (xs[i] - c0[i]);
            if (rst[0] >= -1 - 1e-12 && rst[1] >= -1 - 1e-12 && rst[2] >= -1 - 1e-12 && rst[0] + rst[1] + rst[2] <= -1 + 1e-12) {
                std::vector<double> row = tet_interp_row(ctx->ref3, rst[0], rst[1], rst[2]);
                // M_k^{-1} l(xs) = V V^T l(xs) / |J_k|
                const Mat &V = ctx->ref3.V;
                const int Np = ctx->Np;
                std::vector<double> tmp(Np, 0.0);
                std::vector<float> vec(Np);
                for (int j = 0; j < Np; ++j)
                    for (int n = 0; n < Np; ++n) tmp[j] += V(n, j) * row[n];
                for (int n = 0; n < Np; ++n) {
                    double s = 0;
                    for (int j = 0; j < Np; ++j) s += V(n, j) * tmp[j];
                    vec[n] = float(s / std::fabs(m.J[k]));
                }
                const int s = ctx->src.n;
                CK(cudaMemcpy(ctx->srcvec + size_t(s) * Np, vec.data(), Np * sizeof(float), cudaMemcpyHostToDevice));
                ctx->src.cell[s] = ctx->can2dev[k];
                ctx->src.f_peak[s] = f_peak;
                ctx->src.t_s[s] = t_s;
                ctx->src.amp[s] = amp;
                ctx->src.n = s + 1;
                ctx->src_k.push_back(k);
                ctx->src_vec_h.insert(ctx->src_vec_h.end(), vec.begin(), vec.end());
                drop_graphs(ctx);
                return DGH_OK;
            }
        }
        ctx->err = "source point outside the mesh";
        return DGH_EINVAL;
    });
}

int dgh_step(dgh_ctx *ctx, int64_t nsteps) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        ApiRange nvtx_range("dgh_step");
        if (!ctx || nsteps < 0) return DGH_EINVAL;
        if (ctx->dirty) {
            int rc = run_closure(ctx);
            if (rc) return rc;
        }
        const bool use_graph = ctx->stream != nullptr;
        for (int64_t i = 0; i < nsteps; ++i) {
            if (use_graph) {
                if (!ctx->graph[ctx->cur]) {
                    int rc = build_graph(ctx, ctx->cur);
                    if (rc) return rc;
                }
                CK(cudaGraphLaunch(ctx->graph[ctx->cur], ctx->stream));
            } else {
                int rc = enqueue_step(ctx, ctx->cur, false);
                if (rc) return rc;
            }
            ctx->cur ^= 1;   // 5 stages: odd number of trace swaps
            ctx->step_count++;
            if (ctx->wd_every > 0 && ctx->step_count % ctx->wd_every == 0) {
                double E = 0.0;
                int rc = dgh_get_energy(ctx, &E);
                if (rc) return rc;
                if (!std::isfinite(E) || (ctx->wd_limit > 0.0 && E > ctx->wd_limit)) {
                    char msg[160];
                    std::snprintf(msg, sizeof msg, "watchdog: energy %.6e at step %lld (limit %.6e)", E,
                                  (long long)ctx->step_count, ctx->wd_limit);
                    ctx->err = msg;
                    return DGH_EUNSTABLE;
                }
            }
        }
        CK(cudaGetLastError());
        return DGH_OK;
    });
}

int dgh_set_watchdog(dgh_ctx *ctx, int64_t every, double energy_limit) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx) return DGH_EINVAL;
        if (every < 0 || !std::isfinite(energy_limit)) {
            ctx->err = "watchdog: every >= 0 and a finite energy limit";
            return DGH_EINVAL;
        }
        ctx->wd_every = every;
        ctx->wd_limit = energy_limit;
        return DGH_OK;
    });
}

int dgh_time_kernels(dgh_ctx *ctx, int64_t nsteps, double out_ms[5]) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !out_ms || nsteps < 1) return DGH_EINVAL;
        if (ctx->dirty) {
            int rc = run_closure(ctx);
            if (rc) return rc;
        }
        const int per_step = 5 * 4;
        std::vector<cudaEvent_t> ev(size_t(2 * per_step) * nsteps + 2);
        for (auto &e : ev) CK(cudaEventCreate(&e));
        double acc[4] = {0, 0, 0, 0};
        int cnt[4] = {0, 0, 0, 0};
        size_t ie = 0;
        CK(cudaEventRecord(ev[ie++], ctx->stream));
        int cur = ctx->cur;
        std::vector<std::pair<int, size_t>> marks;
        for (int64_t i = 0; i < nsteps; ++i) {
            for (int s = 0; s < 5; ++s) {
                for (int lv = 0; lv < 4; ++lv) {
                    const bool present = lv == 0 || (lv == 1 && ctx->T) || (lv == 2 && ctx->L) || (lv == 3 && ctx->C);
                    if (!present) continue;
                    CK(cudaEventRecord(ev[ie], ctx->stream));
                    int rc = DGH_OK;
                    if (lv == 0) rc = dispatchN<Launch3>(ctx->N, ctx, cur, s, true);
                    if (lv == 1) rc = dispatchN<Launch2>(ctx->N, ctx, cur, s, true);
                    if (lv == 2) rc = dispatchN<Launch1>(ctx->N, ctx, cur, s, true);
                    if (lv == 3) launch0(ctx, cur ^ 1);
                    if (rc) return rc;
                    CK(cudaEventRecord(ev[ie + 1], ctx->stream));
                    marks.push_back({lv, ie});
                    ie += 2;
                }
                cur ^= 1;
            }
            k_advance_time<<<1, 1, 0, ctx->stream>>>(ctx->d_time, ctx->d_step, ctx->dt);
            ctx->cur ^= 1;
            ctx->step_count++;
        }
        CK(cudaEventRecord(ev[ie], ctx->stream));
        CK(cudaEventSynchronize(ev[ie]));
        for (auto &mk : marks) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[mk.second], ev[mk.second + 1]));
            acc[mk.first] += ms;
            cnt[mk.first]++;
        }
        float total = 0.f;
        CK(cudaEventElapsedTime(&total, ev[0], ev[ie]));
        for (int lv = 0; lv < 4; ++lv) out_ms[lv] = cnt[lv] ? acc[lv] / cnt[lv] : 0.0;
        out_ms[4] = total / double(nsteps);
        for (auto &e : ev) cudaEventDestroy(e);
        return DGH_OK;
    });
}

int dgh_sync(dgh_ctx *ctx) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx) return DGH_EINVAL;
        CK(cudaStreamSynchronize(ctx->stream));
        int err = 0;
        CK(cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err == 2) {
            ctx->err = "checked build: an index outside its array (the access was skipped)";
            return DGH_EBOUNDS;
        }
        if (err) {
            ctx->err = "a device-side wait timed out (stage kernel aborted)";
            return DGH_ETIMEOUT;
        }
        return DGH_OK;
    });
}

int dgh_is_checked_build(void) {
    return dgh_guarded(nullptr, [&]() -> int {
    #ifdef DGH_CHECKED
        return 1;
    #else
        return 0;
    #endif
    });
}

int dgh_get_energy(dgh_ctx *ctx, double *E) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !E) return DGH_EINVAL;
        const int nb = ctx->energy_blocks;
        dispatchN<EnergyPartial>(ctx->N, (const float *)ctx->q3, (const double *)ctx->M3d, (const double *)ctx->ew,
                                 ctx->K32 * 32, ctx->partial, nb, ctx->stream);
        k_sum_partials<<<1, 256, 0, ctx->stream>>>(ctx->partial, nb, ctx->d_energy);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(E, ctx->d_energy, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return DGH_OK;
    });
}

int dgh_get_error_energy(dgh_ctx *ctx, const double *ref, size_t count, double *E) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !ref || !E) return DGH_EINVAL;
        size_t n = 0;
        level_count(ctx, 3, n);
        if (count != n) {
            ctx->err = "reference size mismatch";
            return DGH_EINVAL;
        }
        double *dref = nullptr;
        CK(cudaMallocAsync((void **)&dref, n * sizeof(double), ctx->stream));
        cudaError_t e = cudaMemcpyAsync(dref, ref, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) {
            dispatchN<EnergyDiff>(ctx->N, ctx, (const double *)dref);
            k_sum_partials<<<1, 256, 0, ctx->stream>>>(ctx->partial, ctx->energy_blocks, ctx->d_energy);
            e = cudaGetLastError();
        }
        cudaFreeAsync(dref, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(E, ctx->d_energy, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            ctx->err = std::string("error energy: ") + cudaGetErrorString(e);
            return DGH_ECUDA;
        }
        return DGH_OK;
    });
}

// Checkpoint blob: header (magic, sizes, time, step) then q/res of levels 3, 2, 1.
int dgh_save_state(dgh_ctx *ctx, void *buf, size_t *size) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !size) return DGH_EINVAL;
        size_t n3, n2, n1;
        n3 = size_t(ctx->K32) * 32 * 4 * ctx->Np;   // raw interleaved arrays
        level_count(ctx, 2, n2);
        level_count(ctx, 1, n1);
        const size_t header = 8 * sizeof(int64_t);
        const size_t need = header + 2 * (n3 + n2 + n1) * sizeof(float);
        if (!buf) {
            *size = need;
            return DGH_OK;
        }
        if (*size < need) {
            ctx->err = "checkpoint buffer too small";
            return DGH_EINVAL;
        }
        double t = 0.0;
        CK(cudaMemcpyAsync(&t, ctx->d_time, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        int64_t h[8] = {0x4447484350543031LL, int64_t(n3), int64_t(n2), int64_t(n1), ctx->step_count, 0, 0, 0};
        std::memcpy(&h[5], &t, sizeof(double));
        char *p = static_cast<char *>(buf);
        std::memcpy(p, h, header);
        p += header;
        const size_t ns[3] = {n3, n2, n1};
        for (int i = 0; i < 3; ++i)
            for (int r = 0; r < 2; ++r) {
                if (ns[i]) CK(cudaMemcpyAsync(p, level_ptr(ctx, 3 - i, r), ns[i] * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
                p += ns[i] * sizeof(float);
            }
        CK(cudaStreamSynchronize(ctx->stream));
        *size = need;
        return DGH_OK;
    });
}

int dgh_load_state(dgh_ctx *ctx, const void *buf, size_t size) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !buf) return DGH_EINVAL;
        size_t n3, n2, n1;
        n3 = size_t(ctx->K32) * 32 * 4 * ctx->Np;
        level_count(ctx, 2, n2);
        level_count(ctx, 1, n1);
        const size_t header = 8 * sizeof(int64_t);
        const size_t need = header + 2 * (n3 + n2 + n1) * sizeof(float);
        int64_t h[8];
        if (size != need) {
            ctx->err = "checkpoint size mismatch";
            return DGH_EINVAL;
        }
        std::memcpy(h, buf, header);
        if (h[0] != 0x4447484350543031LL || h[1] != int64_t(n3) || h[2] != int64_t(n2) || h[3] != int64_t(n1)) {
            ctx->err = "checkpoint does not match this context";
            return DGH_EINVAL;
        }
        double t;
        std::memcpy(&t, &h[5], sizeof(double));
        const char *p = static_cast<const char *>(buf) + header;
        const size_t ns[3] = {n3, n2, n1};
        for (int i = 0; i < 3; ++i)
            for (int r = 0; r < 2; ++r) {
                if (ns[i]) CK(cudaMemcpyAsync(level_ptr(ctx, 3 - i, r), p, ns[i] * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
                p += ns[i] * sizeof(float);
            }
        CK(cudaMemcpyAsync(ctx->d_time, &t, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_step, &h[4], sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->step_count = h[4];
        ctx->dirty = true;
        return DGH_OK;
    });
}


// ---------------------------------------------------------------- launch shapes and tuning
static int dispatch_kern3(const dgh_ctx *c) { return kern3_of(c->precision, c->N, c->K); }

int dgh_get_launch(const dgh_ctx *ctx, dgh_launch *o) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !o) return DGH_EINVAL;
        o->tile2 = ctx->tile2;
        o->tile1 = ctx->tile1;
        o->cta3_per_sm = ctx->cta3_per_sm;
        o->grid3 = ctx->grid3;
        o->grid2 = ctx->grid2;
        o->grid1 = ctx->grid1;
        o->occ3 = ctx->occ3;
        o->sms = ctx->sms;
        o->thr2 = ctx->thr2;
        o->thr1 = ctx->thr1;
        o->sm3_div = ctx->sm3_div;
        o->split3 = ctx->split3;
        o->kern3 = dispatch_kern3(ctx);
        return DGH_OK;
    });
}

int dgh_set_launch(dgh_ctx *ctx, const dgh_launch *in) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        auto thr_ok = [](int t) { return t == 32 || t == 64 || t == 128 || t == 256; };
        if (!ctx || !in || in->tile2 < 1 || in->tile1 < 1 || in->cta3_per_sm < 0 || !thr_ok(in->thr2) ||
            !thr_ok(in->thr1) || in->sm3_div < 1 || in->sm3_div > 16 || (in->split3 != 0 && in->split3 != 1)) {
            if (ctx)
                ctx->err = "tile2, tile1 must be >= 1, cta3_per_sm >= 0, thr2 / thr1 one of 32, 64, 128, 256, "
                           "sm3_div in 1..16, split3 0 or 1";
            return DGH_EINVAL;
        }
        const int t2 = ctx->tile2, t1 = ctx->tile1, c3 = ctx->cta3_per_sm, h2 = ctx->thr2, h1 = ctx->thr1;
        const int d3 = ctx->sm3_div, s3 = ctx->split3;
        ctx->tile2 = in->tile2;
        ctx->tile1 = in->tile1;
        ctx->cta3_per_sm = in->cta3_per_sm;
        ctx->thr2 = in->thr2;
        ctx->thr1 = in->thr1;
        ctx->sm3_div = in->sm3_div;
        ctx->split3 = in->split3;
        if (dispatchN<Shapes>(ctx->N, ctx) != DGH_OK) {
            ctx->tile2 = t2;
            ctx->tile1 = t1;
            ctx->cta3_per_sm = c3;
            ctx->thr2 = h2;
            ctx->thr1 = h1;
            ctx->sm3_div = d3;
            ctx->split3 = s3;
            dispatchN<Shapes>(ctx->N, ctx);
            ctx->err = "launch shape does not fit (shared memory, or tile2 * P > thr2)";
            return DGH_EINVAL;
        }
        drop_graphs(ctx);
        return DGH_OK;
    });
}

}  // extern "C"

namespace {

// Milliseconds per step of run(steps) on stream st (after two untimed steps),
// best of two repetitions.
template <class Run>
int time_per_step(cudaStream_t st, int steps, Run run, double &ms, std::string &err) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        err = "cudaEventCreate failed";
        return DGH_ECUDA;
    }
    int rc = run(2);   // both trace parities: any graph is built before the timed region
    ms = 1e300;
    for (int rep = 0; rep < 2 && rc == DGH_OK; ++rep) {
        cudaEventRecord(a, st);
        rc = run(steps);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            err = "tuning run failed";
            rc = DGH_ECUDA;
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        ms = std::min(ms, double(t) / steps);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

// Coordinate search over the launch shape of every context (2D threads and
// triangles per CTA, 1D threads and lines per CTA, persistent 3D CTAs per
// SM), the paper's tuning of
// elements per block (K_blk) carried over to these kernels: each candidate
// is timed on whole steps and kept if it is at least 1% faster.  The fields
// are saved before and restored after, so the search changes no result.
template <class Run, class Invalidate>
int tune_contexts(const std::vector<dgh_ctx *> &cs, cudaStream_t st, int steps, Run run, Invalidate invalidate,
                  double *ms_before, double *ms_after, std::string &err) {
    std::vector<std::vector<char>> saved(cs.size());
    for (size_t i = 0; i < cs.size(); ++i) {
        size_t sz = 0;
        int rc = dgh_save_state(cs[i], nullptr, &sz);
        if (rc) return rc;
        saved[i].resize(sz);
        if ((rc = dgh_save_state(cs[i], saved[i].data(), &sz))) {
            err = cs[i]->err;
            return rc;
        }
    }
    double best = 0.0;
    int rc = time_per_step(st, steps, run, best, err);
    if (rc) return rc;
    if (ms_before) *ms_before = best;
    // concurrent contexts (the groups of a batch): first the SM share of every
    // group's 3D grid at once, since one group alone leaving SMs free gains
    // nothing while the others still take all of them
    if (cs.size() > 1) {
        int keep = cs[0]->sm3_div;
        for (int v = 2; v <= 8 && rc == DGH_OK; v *= 2) {
            for (dgh_ctx *c : cs) {
                c->sm3_div = v;
                dispatchN<Shapes>(c->N, c);
            }
            invalidate();
            double ms = 0.0;
            if ((rc = time_per_step(st, steps, run, ms, err))) break;
            if (ms < 0.99 * best) {
                best = ms;
                keep = v;
            }
        }
        for (dgh_ctx *c : cs) {
            c->sm3_div = keep;
            dispatchN<Shapes>(c->N, c);
        }
        invalidate();
    }
    for (dgh_ctx *c : cs) {
        for (int param = 0; param < 7 && rc == DGH_OK; ++param) {
            int *slot = param == 0 ? &c->thr2 : param == 1 ? &c->tile2 : param == 2 ? &c->thr1 : param == 3 ? &c->tile1
                        : param == 4 ? &c->cta3_per_sm : param == 5 ? &c->sm3_div : &c->split3;
            std::vector<int> cand;
            if ((param == 0 && c->T > 0) || (param == 2 && c->L > 0))
                for (int v = 32; v <= 256; v *= 2) cand.push_back(v);
            if (param == 1 && c->T > 0)
                for (int v = 1; v <= 32 && v <= c->T; v *= 2) cand.push_back(v);
            if (param == 3 && c->L > 0)
                for (int v = 1; v <= 32 && v <= c->L; v *= 2) cand.push_back(v);
            if (param == 4)
                for (int v = 0; v <= c->occ3; ++v) cand.push_back(v);
            if (param == 5 && cs.size() > 1)   // SM share of the 3D grid: only concurrent contexts can use the rest
                for (int v = 1; v <= 4; v *= 2) cand.push_back(v);
            if (param == 6 && c->T > 0 && !c->no_overlap) cand = {1, 0};
            if (param == 1 && c->T > 0) cand.push_back(k2d_tile_max(c->P, c->thr2));
            int keep = *slot, keep_tile2 = c->tile2;
            for (int v : cand) {
                if (v == keep) continue;
                *slot = v;
                if (param == 0) c->tile2 = k2d_tile_max(c->P, v);   // a 2D thread count comes with its largest tile
                if (dispatchN<Shapes>(c->N, c) != DGH_OK) continue;
                invalidate();
                double ms = 0.0;
                if ((rc = time_per_step(st, steps, run, ms, err))) break;
                if (ms < 0.99 * best) {
                    best = ms;
                    keep = v;
                    keep_tile2 = c->tile2;
                }
            }
            *slot = keep;
            c->tile2 = param == 1 ? keep : keep_tile2;
            dispatchN<Shapes>(c->N, c);
            invalidate();
        }
        if (rc) break;
    }
    for (size_t i = 0; i < cs.size(); ++i) {
        int rc2 = dgh_load_state(cs[i], saved[i].data(), saved[i].size());
        if (rc2 && !rc) {
            err = cs[i]->err;
            rc = rc2;
        }
    }
    if (ms_after) *ms_after = best;
    return rc;
}

}  // namespace

extern "C" int dgh_tune(dgh_ctx *ctx, int steps, double *ms_before, double *ms_after) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        ApiRange nvtx_range("dgh_tune");
        if (!ctx || steps < 1) return DGH_EINVAL;
        const int64_t sc0 = ctx->step_count;
        int rc = tune_contexts(
            {ctx}, ctx->stream, steps, [&](int n) { return dgh_step(ctx, n); }, [&]() { drop_graphs(ctx); }, ms_before,
            ms_after, ctx->err);
        ctx->step_count = sc0;
        return rc;
    });
}

// ============================================================================
// Batching form: independent problems stepped together.
//
// The problems are grouped by (N, P).  Each group is one union context whose
// mesh is the disjoint union of its problems' meshes (every problem keeps its
// own range of 32-cell blocks, triangles, lines and corners), with every
// problem's time step folded into its cells' coefficients.  One CUDA graph
// per step forks one branch per group; inside a branch the stage kernels of
// Algorithm 1 run over all problems of the group at once, the 3D kernel
// claiming 32-cell blocks from a device counter (the work queue), so small
// problems share the GPU instead of each under-filling it.
struct dgh_batch {
    std::string err = "no error";
    int device = 0;
    cudaStream_t stream = nullptr;   // capture / replay stream (non-blocking)
    std::vector<dgh_ctx *> groups;
    std::vector<cudaStream_t> gstream;
    std::vector<cudaEvent_t> gjoin;
    cudaEvent_t fork = nullptr;
    struct Prob {
        int group = 0, part = 0, N = 0, P = 0;
        int64_t cell0 = 0, K = 0, tri0 = 0, T = 0, lin0 = 0, L = 0, C = 0, Fb = 0;
        double dt = 0.0, t0 = 0.0;
        int64_t step0 = 0;
    };
    std::vector<Prob> probs;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t step_count = 0;
};

namespace {

void batch_drop_graphs(dgh_batch *b) {
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
}

int batch_build_graph(dgh_batch *b) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        b->err = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    int rc = DGH_OK;
    cudaEventRecord(b->fork, b->stream);
    for (size_t i = 0; i < b->groups.size() && rc == DGH_OK; ++i) {
        cudaStreamWaitEvent(b->gstream[i], b->fork, 0);
        rc = enqueue_step(b->groups[i], b->groups[i]->cur, false, b->gstream[i]);
        if (rc) b->err = b->groups[i]->err;
        cudaEventRecord(b->gjoin[i], b->gstream[i]);
        cudaStreamWaitEvent(b->stream, b->gjoin[i], 0);
    }
    e = cudaStreamEndCapture(b->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        b->err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    e = cudaGraphInstantiate(&b->graph[b->cur], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        return DGH_ECUDA;
    }
    return DGH_OK;
}

// Host-only grouping of problems by (N, P), in order of first appearance.
std::vector<int> group_by_order(const std::vector<std::pair<int, int>> &np, int &ngroups) {
    std::vector<std::pair<int, int>> keys;   // (N, P * 8 + precision) in order of first appearance
    std::vector<int> g(np.size());
    for (size_t i = 0; i < np.size(); ++i) {
        size_t j = 0;
        while (j < keys.size() && keys[j] != np[i]) ++j;
        if (j == keys.size()) keys.push_back(np[i]);
        g[i] = int(j);
    }
    ngroups = int(keys.size());
    return g;
}

}  // namespace

extern "C" {

const char *dgh_batch_last_error(const dgh_batch *b) { return b ? b->err.c_str() : g_create_error.c_str(); }

void dgh_batch_destroy(dgh_batch *b) {
    if (!b) return;
    batch_drop_graphs(b);
    for (dgh_ctx *c : b->groups) dgh_destroy(c);
    for (cudaStream_t s : b->gstream)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->gjoin)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int dgh_batch_plan(const dgh_desc *descs, int count, int *group_of, dgh_info *group_info, int *n_groups) {
    return dgh_guarded(nullptr, [&]() -> int {
        if (!descs || count < 1 || !group_of || !group_info || !n_groups) {
            g_create_error = "invalid batch plan arguments";
            return DGH_EINVAL;
        }
        std::vector<std::pair<int, int>> np(static_cast<size_t>(count));
        for (int i = 0; i < count; ++i) {
            int rc = validate_desc(&descs[i]);
            if (rc) return rc;
            np[i] = {descs[i].order, descs[i].habc_order * 8 + descs[i].precision};
        }
        int ng = 0;
        std::vector<int> g = group_by_order(np, ng);
        for (int gi = 0; gi < ng; ++gi) {
            std::vector<HostMesh> parts;
            RefTet T3;
            RefTri T2;
            RefLine T1;
            HabcOps habc;
            for (int i = 0; i < count; ++i) {
                if (g[i] != gi) continue;
                parts.emplace_back();
                int rc = host_setup(&descs[i], parts.back(), T3, T2, T1, habc);
                if (rc) return rc;
            }
            HostMesh u;
            merge_meshes(parts, u);
            dgh_info &o = group_info[gi];
            std::memset(&o, 0, sizeof(o));
            o.order = u.N;
            o.habc_order = u.P;
            o.Np = T3.Np;
            o.Np2 = T2.Np;
            o.Np1 = T1.Np;
            o.n_corners = int(u.corners.size());
            o.n_cells = u.K;
            o.n_tris = u.Ktri;
            o.n_lines = u.Klin;
            o.n_bfaces = int64_t(u.bface.size());
            const int64_t P = u.P;
            o.ndof = 4 * int64_t(T3.Np) * u.K + 3 * P * T2.Np * u.Ktri + 2 * P * P * T1.Np * u.Klin;
        }
        for (int i = 0; i < count; ++i) group_of[i] = g[i];
        *n_groups = ng;
        return DGH_OK;
    });
}

int dgh_batch_create(dgh_ctx *const *problems, int count, dgh_batch **out) {
    return dgh_guarded(nullptr, [&]() -> int {
        if (!out || !problems || count < 1) {
            g_create_error = "invalid batch arguments";
            return DGH_EINVAL;
        }
        *out = nullptr;
        int dev = 0;
        cudaGetDevice(&dev);
        std::vector<std::pair<int, int>> np(static_cast<size_t>(count));
        for (int i = 0; i < count; ++i) {
            if (!problems[i]) {
                g_create_error = "null problem context";
                return DGH_EINVAL;
            }
            if (problems[i]->device != dev) {
                g_create_error = "all problems must live on the current device";
                return DGH_EINVAL;
            }
            if (problems[i]->cl_on || problems[i]->sh) {
                g_create_error = "a learned closure or sample recording is not supported in a batch";
                return DGH_EUNSUPPORTED;
            }
            np[i] = {problems[i]->N, problems[i]->P * 8 + problems[i]->precision};
        }
        int ng = 0;
        std::vector<int> gof = group_by_order(np, ng);
        struct Owner {   // destroys the partly built batch on every failure, thrown or returned
            dgh_batch *b;
            ~Owner() { if (b) dgh_batch_destroy(b); }
        } owner{new dgh_batch()};
        dgh_batch *b = owner.b;
        b->device = dev;
        auto fail = [&](int rc, const std::string &msg) {
            g_create_error = msg;
            return rc;
        };
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
            return fail(DGH_ECUDA, "batch stream / event");
        b->probs.resize(size_t(count));
        for (int gi = 0; gi < ng; ++gi) {
            std::vector<int> members;
            for (int i = 0; i < count; ++i)
                if (gof[i] == gi) members.push_back(i);
            b->groups.push_back(nullptr);
            dgh_ctx *u = b->groups.back() = new dgh_ctx();
            const dgh_ctx *first = problems[members[0]];
            u->stream = b->stream;
            u->device = dev;
            u->N = first->N;
            u->P = first->P;
            u->precision = first->precision;
            u->ref3 = first->ref3;
            u->ref2 = first->ref2;
            u->ref1 = first->ref1;
            u->habc = first->habc;
            u->dt = 1.0;   // time steps folded into the coefficients: the clock counts steps
            std::vector<HostMesh> parts;
            std::vector<int64_t> offs{0};
            int64_t t0 = 0, l0 = 0;
            for (size_t j = 0; j < members.size(); ++j) {
                dgh_ctx *pc = problems[members[j]];
                double tnow = 0.0;
                if (cudaStreamSynchronize(pc->stream) != cudaSuccess ||
                    cudaMemcpy(&tnow, pc->d_time, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
                    return fail(DGH_ECUDA, "reading a problem's time");
                parts.push_back(pc->mesh);
                parts.back().dtCell.assign(size_t(pc->mesh.K), pc->dt);
                dgh_batch::Prob &pr = b->probs[size_t(members[j])];
                pr.group = gi;
                pr.part = int(j);
                pr.N = pc->N;
                pr.P = pc->P;
                pr.cell0 = offs.back();
                pr.K = pc->K;
                pr.tri0 = t0;
                pr.T = pc->T;
                pr.lin0 = l0;
                pr.L = pc->L;
                pr.C = pc->C;
                pr.Fb = pc->Fb;
                pr.dt = pc->dt;
                pr.t0 = tnow;
                pr.step0 = pc->step_count;
                offs.push_back(offs.back() + pc->K);
                t0 += pc->T;
                l0 += pc->L;
            }
            merge_meshes(parts, u->mesh);
            parts.clear();
            int rc = build_context(u, offs);
            if (rc) return fail(rc, u->err);
            // sources: time measured in steps of the problem's own dt
            for (size_t j = 0; j < members.size(); ++j) {
                const dgh_ctx *pc = problems[members[j]];
                const dgh_batch::Prob &pr = b->probs[size_t(members[j])];
                for (int s = 0; s < pc->src.n; ++s) {
                    const int d = u->src.n;
                    if (d >= MAXSRC) return fail(DGH_EINVAL, "more than MAXSRC point sources in one (N, P) group");
                    const std::vector<float> vec(pc->src_vec_h.begin() + size_t(s) * pc->Np,
                                                 pc->src_vec_h.begin() + size_t(s + 1) * pc->Np);
                    if (cudaMemcpy(u->srcvec + size_t(d) * u->Np, vec.data(), vec.size() * sizeof(float),
                                   cudaMemcpyHostToDevice) != cudaSuccess)
                        return fail(DGH_ECUDA, "source upload");
                    u->src.cell[d] = u->can2dev[size_t(pr.cell0 + pc->src_k[size_t(s)])];
                    u->src.f_peak[d] = pc->src.f_peak[s] * pr.dt;
                    u->src.t_s[d] = (pc->src.t_s[s] - pr.t0) / pr.dt;
                    u->src.amp[d] = pc->src.amp[s] * pr.dt * pr.dt;
                    u->src.n = d + 1;
                    u->src_k.push_back(pr.cell0 + pc->src_k[size_t(s)]);
                    u->src_vec_h.insert(u->src_vec_h.end(), vec.begin(), vec.end());
                }
            }
            // current fields of every problem, concatenated in canonical order
            for (int lv = 3; lv >= 1; --lv) {
                size_t ntot = 0;
                level_count(u, lv, ntot);
                std::vector<double> all(ntot);
                size_t at = 0;
                for (int i : members) {
                    size_t n = 0;
                    level_count(problems[i], lv, n);
                    if (n && dgh_get_state(problems[i], lv, all.data() + at, n) != DGH_OK)
                        return fail(DGH_ECUDA, std::string("reading a problem's state: ") + problems[i]->err);
                    at += n;
                }
                if (ntot && (rc = dgh_set_state(u, lv, all.data(), ntot))) return fail(rc, u->err);
            }
            cudaStream_t gs = nullptr;
            cudaEvent_t ge = nullptr;
            if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess) return fail(DGH_ECUDA, "group stream");
            b->gstream.push_back(gs);
            if (cudaEventCreateWithFlags(&ge, cudaEventDisableTiming) != cudaSuccess) return fail(DGH_ECUDA, "group event");
            b->gjoin.push_back(ge);
        }
        *out = b;
        owner.b = nullptr;
        return DGH_OK;
    });
}

int dgh_batch_stream(const dgh_batch *b, void **stream) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        if (!b || !stream) return DGH_EINVAL;
        *stream = static_cast<void *>(b->stream);
        return DGH_OK;
    });
}

int dgh_batch_count(const dgh_batch *b, int *n_problems, int *n_groups) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        if (!b) return DGH_EINVAL;
        if (n_problems) *n_problems = int(b->probs.size());
        if (n_groups) *n_groups = int(b->groups.size());
        return DGH_OK;
    });
}

int dgh_batch_step(dgh_batch *b, int64_t nsteps) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        ApiRange nvtx_range("dgh_batch_step");
        if (!b || nsteps < 0) return DGH_EINVAL;
        for (dgh_ctx *u : b->groups)
            if (u->dirty) {
                int rc = run_closure(u);
                if (rc) {
                    b->err = u->err;
                    return rc;
                }
            }
        for (int64_t i = 0; i < nsteps; ++i) {
            if (!b->graph[b->cur]) {
                int rc = batch_build_graph(b);
                if (rc) return rc;
            }
            cudaError_t e = cudaGraphLaunch(b->graph[b->cur], b->stream);
            if (e != cudaSuccess) {
                b->err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
                return DGH_ECUDA;
            }
            b->cur ^= 1;
            for (dgh_ctx *u : b->groups) {
                u->cur ^= 1;
                u->step_count++;
            }
            b->step_count++;
        }
        return DGH_OK;
    });
}

int dgh_batch_sync(dgh_batch *b) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        if (!b) return DGH_EINVAL;
        for (dgh_ctx *u : b->groups) {
            int rc = dgh_sync(u);
            if (rc) {
                b->err = u->err;
                return rc;
            }
        }
        return DGH_OK;
    });
}

int dgh_batch_get_info(const dgh_batch *b, int i, dgh_info *o) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        if (!b || !o || i < 0 || i >= int(b->probs.size())) return DGH_EINVAL;
        const dgh_batch::Prob &p = b->probs[size_t(i)];
        const dgh_ctx *u = b->groups[size_t(p.group)];
        std::memset(o, 0, sizeof(*o));
        o->order = p.N;
        o->habc_order = p.P;
        o->Np = u->Np;
        o->Np2 = u->Np2;
        o->Np1 = u->Np1;
        o->n_corners = int(p.C);
        o->n_cells = p.K;
        o->n_tris = p.T;
        o->n_lines = p.L;
        o->n_bfaces = p.Fb;
        o->ndof = 4 * int64_t(u->Np) * p.K + 3 * int64_t(p.P) * u->Np2 * p.T + 2 * int64_t(p.P) * p.P * u->Np1 * p.L;
        o->step_count = p.step0 + b->step_count;
        o->dt = p.dt;
        o->time = p.t0 + double(b->step_count) * p.dt;
        o->device_bytes = u->device_bytes;
        return DGH_OK;
    });
}

int dgh_batch_get_state(dgh_batch *b, int i, int level, double *out, size_t count) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        if (!b || i < 0 || i >= int(b->probs.size()) || (!out && count)) return DGH_EINVAL;
        const dgh_batch::Prob &p = b->probs[size_t(i)];
        dgh_ctx *u = b->groups[size_t(p.group)];
        size_t per = 0, off = 0, n = 0;
        if (level == 3) {
            per = size_t(4) * u->Np;
            off = size_t(p.cell0) * per;
            n = size_t(p.K) * per;
        } else if (level == 2) {
            per = size_t(p.P) * 3 * u->Np2;
            off = size_t(p.tri0) * per;
            n = size_t(p.T) * per;
        } else if (level == 1) {
            per = size_t(p.P) * p.P * 2 * u->Np1;
            off = size_t(p.lin0) * per;
            n = size_t(p.L) * per;
        } else {
            b->err = "level must be 3, 2 or 1";
            return DGH_EINVAL;
        }
        if (n != count) {
            b->err = "state size mismatch";
            return DGH_EINVAL;
        }
        if (n == 0) return DGH_OK;
        size_t ntot = 0;
        level_count(u, level, ntot);
        std::vector<double> all(ntot);
        int rc = dgh_get_state(u, level, all.data(), ntot);
        if (rc) {
            b->err = u->err;
            return rc;
        }
        std::memcpy(out, all.data() + off, n * sizeof(double));
        return DGH_OK;
    });
}

int dgh_batch_get_energy(dgh_batch *b, int i, double *E) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        if (!b || !E || i < 0 || i >= int(b->probs.size())) return DGH_EINVAL;
        const dgh_batch::Prob &p = b->probs[size_t(i)];
        dgh_ctx *u = b->groups[size_t(p.group)];
        const int64_t blk0 = u->part_blk0[size_t(p.part)], nblk = u->part_blk0[size_t(p.part) + 1] - blk0;
        const float *q = u->q3 + blk0 * 4 * u->Np * 32;
        const double *ew = u->ew + blk0 * 32 * 2;
        const int nb = u->energy_blocks;
        cudaStream_t st = u->stream;
        dispatchN<EnergyPartial>(u->N, q, (const double *)u->M3d, ew, nblk * 32, u->partial, nb, st);
        k_sum_partials<<<1, 256, 0, st>>>(u->partial, nb, u->d_energy);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(E, u->d_energy, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            b->err = std::string("energy: ") + cudaGetErrorString(e);
            return DGH_ECUDA;
        }
        return DGH_OK;
    });
}

int dgh_batch_get_launch(const dgh_batch *b, int group, dgh_launch *o) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        if (!b || group < 0 || group >= int(b->groups.size())) return DGH_EINVAL;
        return dgh_get_launch(b->groups[size_t(group)], o);
    });
}

int dgh_batch_tune(dgh_batch *b, int steps, double *ms_before, double *ms_after) {
    return dgh_guarded(err_slot(b), [&]() -> int {
        ApiRange nvtx_range("dgh_batch_tune");
        if (!b || steps < 1) return DGH_EINVAL;
        const int64_t sc0 = b->step_count;
        std::vector<int64_t> gsc;
        for (dgh_ctx *u : b->groups) gsc.push_back(u->step_count);
        int rc = tune_contexts(
            b->groups, b->stream, steps, [&](int n) { return dgh_batch_step(b, n); }, [&]() { batch_drop_graphs(b); },
            ms_before, ms_after, b->err);
        b->step_count = sc0;
        for (size_t i = 0; i < b->groups.size(); ++i) b->groups[i]->step_count = gsc[i];
        return rc;
    });
}


// ---------------------------------------------------------------- learned closure
int dgh_closure_set_weights(dgh_ctx *ctx, const float *w, size_t n) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx) return DGH_EINVAL;
        if (!w) {   // disable
            ctx->cl_on = false;
            ctx->dirty = true;
            drop_graphs(ctx);
            return DGH_OK;
        }
        if (n != size_t(MLP_NPARAM) && n != size_t(MLP_NPARAM + MLP_IN + 1)) {
            ctx->err = "closure weights: expected " + std::to_string(MLP_NPARAM) + " values (or " +
                       std::to_string(MLP_NPARAM + MLP_IN + 1) + " for the homogeneous form)";
            return DGH_EINVAL;
        }
        if (ctx->P < 1 || ctx->T == 0) {
            ctx->err = "closure needs HABC faces (P >= 1)";
            return DGH_EINVAL;
        }
        std::vector<float> wb(n);   // BF16 weights (FP32 arithmetic); the scales of the homogeneous form stay FP32
        for (size_t i = 0; i < n; ++i) wb[i] = i < size_t(MLP_NPARAM) ? __bfloat162float(__float2bfloat16_rn(w[i])) : w[i];
        int rc = DGH_OK;
        if (!ctx->cl_w && ((rc = dalloc(ctx, ctx->cl_w, size_t(CL_MLP0 + 1))) || (rc = dalloc(ctx, ctx->cl_feat, size_t(ctx->T) * ctx->Np2 * MLP_IN)) ||
                           (rc = dalloc(ctx, ctx->cl_rm, size_t(ctx->T) * ctx->Np2))))
            return rc;
        CK(cudaMemcpy(ctx->cl_w, wb.data(), n * sizeof(float), cudaMemcpyHostToDevice));
        k_mlp_zero<<<1, 256, 0, ctx->stream>>>(ctx->cl_w, ctx->cl_w + CL_MLP0);   // once per weight set
        CK(cudaGetLastError());
        ctx->cl_on = true;
        ctx->cl_homog = n != size_t(MLP_NPARAM);
        ctx->dirty = true;   // the exterior state is rebuilt with the closure before the next step
        drop_graphs(ctx);
        return DGH_OK;
    });
}

int dgh_closure_record(dgh_ctx *ctx, int shadow_order, int every, double fraction, int64_t max_samples, uint64_t seed) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx) return DGH_EINVAL;
        if (ctx->sh) {
            ctx->err = "recording is already enabled on this context";
            return DGH_ESTATE;
        }
        if (shadow_order < 1 || shadow_order > MAXP || every < 1 || !(fraction > 0.0 && fraction <= 1.0) || max_samples < 1) {
            ctx->err = "record: shadow order 1..12, every >= 1, 0 < fraction <= 1, max_samples >= 1";
            return DGH_EINVAL;
        }
        if (ctx->P < 1 || ctx->T == 0) {
            ctx->err = "record needs HABC faces (P >= 1)";
            return DGH_EINVAL;
        }
        auto *h = new dgh_ctx::Shadow();
        ctx->sh = h;
        h->P = shadow_order;
        std::string err;
        if (!build_habc(h->P, h->habc, err)) {
            ctx->err = err;
            return DGH_EINVAL;
        }
        h->M = h->habc.M;
        const int P = h->P, N = ctx->N, Np2 = ctx->Np2, Np1 = ctx->Np1;
        const int64_t T = ctx->T, L = ctx->L;
        std::vector<float> cP(static_cast<size_t>(P));
        for (int a = 0; a < P; ++a) cP[a] = float(h->habc.c[a]);
        int rc;
        if ((rc = dalloc(ctx, h->q2, size_t(T) * P * 3 * Np2)) || (rc = dalloc(ctx, h->res2, size_t(T) * P * 3 * Np2)) ||
            (rc = dalloc(ctx, h->tr2[0], size_t(T) * P * 3 * 2 * (N + 1))) || (rc = dalloc(ctx, h->tr2[1], size_t(T) * P * 3 * 2 * (N + 1))) ||
            (rc = dalloc(ctx, h->qb2, size_t(T) * 3 * P * (N + 1))) || (rc = dalloc(ctx, h->q0_3, size_t(T) * Np2)) ||
            (rc = dalloc(ctx, h->q1, size_t(L) * P * P * 2 * Np1)) || (rc = dalloc(ctx, h->res1, size_t(L) * P * P * 2 * Np1)) ||
            (rc = dalloc(ctx, h->tr1[0], size_t(L) * P * P * 4)) || (rc = dalloc(ctx, h->tr1[1], size_t(L) * P * P * 4)) ||
            (rc = dalloc(ctx, h->qb1, size_t(L) * 2 * P * P)) || (rc = dalloc(ctx, h->q0_2, size_t(L) * 2 * P * Np1)) ||
            (rc = upload(ctx, h->H1, to_f(h->habc.H1))) || (rc = upload(ctx, h->H2, to_f(h->habc.H2))) ||
            (rc = upload(ctx, h->Hc, to_f(h->habc.Hc))) || (rc = upload(ctx, h->cP, cP)) ||
            (rc = dalloc(ctx, h->feat, size_t(T) * Np2 * MLP_IN)) || (rc = dalloc(ctx, h->rm, size_t(T) * Np2)) ||
            (rc = dalloc(ctx, h->rm_main, size_t(T) * Np2)) || (rc = dalloc(ctx, h->samples, size_t(max_samples) * SAMPLE_W)) ||
            (rc = dalloc(ctx, h->count, 1)))
            return rc;
        h->max_samples = max_samples;
        h->every = every;
        h->threshold = fraction >= 1.0 ? 0xFFFFFFFFu : uint32_t(fraction * 4294967296.0);
        h->seed = seed;
        h->tile2 = k2d_tile_max(P, 256);
        h->tile1 = std::max(1, 256 / std::max(1, P * P * Np1));
        h->smem2 = k2d_smem(N, P, h->tile2);
        h->smem1 = k1d_smem(N, P, h->tile1);
        h->smem0 = sizeof(float) * 3 * P * P;
        if ((int64_t)h->smem2 > ctx->smem_optin || (int64_t)h->smem1 > ctx->smem_optin) {
            ctx->err = "shadow chain tile does not fit in shared memory";
            return DGH_EUNSUPPORTED;
        }
        h->grid2 = (int)std::max<int64_t>(1, std::min<int64_t>((T + h->tile2 - 1) / h->tile2, int64_t(8) * ctx->sms));
        h->grid1 = (int)std::max<int64_t>(1, std::min<int64_t>((L + h->tile1 - 1) / h->tile1, int64_t(8) * ctx->sms));
        ctx->dirty = true;
        drop_graphs(ctx);
        return DGH_OK;
    });
}

int dgh_closure_samples(dgh_ctx *ctx, float *out, int64_t max_rows, int64_t *count) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !count || (!out && max_rows > 0)) return DGH_EINVAL;
        if (!ctx->sh) {
            ctx->err = "recording is not enabled on this context";
            return DGH_ESTATE;
        }
        unsigned long long c = 0;
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaMemcpy(&c, ctx->sh->count, sizeof(c), cudaMemcpyDeviceToHost));
        const int64_t have = std::min<int64_t>((int64_t)c, ctx->sh->max_samples);
        *count = have;
        const int64_t rows = std::min<int64_t>(have, max_rows);
        if (rows > 0) CK(cudaMemcpy(out, ctx->sh->samples, size_t(rows) * SAMPLE_W * sizeof(float), cudaMemcpyDeviceToHost));
        return DGH_OK;
    });
}

}  // extern "C"

namespace {
int closure_train_rows(dgh_ctx *ctx, bool homogeneous, const dgh_train_cfg *cfg, float *w_out, double *loss_hist,
                       double *final_mse) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !cfg || !w_out) return DGH_EINVAL;
        int64_t n = 0;
        int rc = dgh_closure_samples(ctx, nullptr, 0, &n);
        if (rc) return rc;
        if (n < 2) {
            ctx->err = "closure train: fewer than 2 recorded rows";
            return DGH_ESTATE;
        }
        std::vector<float> rows(static_cast<size_t>(n) * SAMPLE_W), X(static_cast<size_t>(n) * MLP_IN),
            Y(static_cast<size_t>(n));
        if ((rc = dgh_closure_samples(ctx, rows.data(), n, &n))) return rc;
        for (int64_t r = 0; r < n; ++r) {
            for (int i = 0; i < MLP_IN; ++i) X[size_t(r) * MLP_IN + i] = rows[size_t(r) * SAMPLE_W + i];
            Y[size_t(r)] = rows[size_t(r) * SAMPLE_W + MLP_IN];
        }
        rc = homogeneous ? dgh_closure_fit_homogeneous(X.data(), Y.data(), n, cfg, w_out, loss_hist, final_mse)
                         : dgh_mlp_train(X.data(), Y.data(), n, cfg, w_out, loss_hist, final_mse);
        if (rc) ctx->err = dgh_last_error(nullptr);
        return rc;
    });
}
}  // namespace

extern "C" {

int dgh_closure_train(dgh_ctx *ctx, const dgh_train_cfg *cfg, float *w_out, double *loss_hist, double *final_mse) {
    return closure_train_rows(ctx, false, cfg, w_out, loss_hist, final_mse);
}

int dgh_closure_train_homogeneous(dgh_ctx *ctx, const dgh_train_cfg *cfg, float *w_out, double *loss_hist,
                                  double *final_mse) {
    return closure_train_rows(ctx, true, cfg, w_out, loss_hist, final_mse);
}

}  // extern "C"

namespace {

// scoped device buffers of the context-free MLP calls
struct DevScratch {
    std::vector<void *> ptrs;
    ~DevScratch() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    T *get(size_t count) {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
};

int mlp_fail(const std::string &msg, int rc) {
    g_create_error = msg;
    return rc;
}

// loss and gradient on the device: rows idx (or 0..n-1), weights already on the device
int mlp_loss_grad_dev(const float *dw, const float *dX, const float *dY, const int64_t *didx, int64_t n, float *dpart,
                      int nblocks, float *dgrad, double *dloss) {
    k_mlp_grad<<<nblocks, MLP_BS, mlp_grad_smem()>>>(dw, dX, dY, didx, n, 1.0 / double(n), dpart);
    k_mlp_reduce<<<(MLP_NPARAM + 1 + 255) / 256, 256>>>(dpart, nblocks, dgrad, dloss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DGH_OK : mlp_fail(std::string("mlp kernels: ") + cudaGetErrorString(e), DGH_ECUDA);
}

int mlp_setup(int &sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_grad_smem()) != cudaSuccess)
        return mlp_fail("mlp: shared memory attribute", DGH_ECUDA);
    return DGH_OK;
}

}  // namespace

extern "C" {

int dgh_closure_eval(const float *w, size_t nw, const float *X, int64_t n, float *y) {
    return dgh_guarded(nullptr, [&]() -> int {
        if (!w || (n > 0 && (!X || !y)) || n < 0 || (nw != size_t(MLP_NPARAM) && nw != size_t(MLP_NPARAM + MLP_IN + 1)))
            return mlp_fail("closure eval: invalid arguments", DGH_EINVAL);
        if (n == 0) return DGH_OK;
        std::vector<float> wb(nw);
        for (size_t i = 0; i < nw; ++i) wb[i] = i < size_t(MLP_NPARAM) ? __bfloat162float(__float2bfloat16_rn(w[i])) : w[i];
        DevScratch d;
        float *dw = d.get<float>(nw), *dX = d.get<float>(size_t(n) * MLP_IN), *dy = d.get<float>(size_t(n));
        float *d0 = d.get<float>(1);
        if (!dw || !dX || !dy || !d0) return mlp_fail("closure eval: device allocation failed", DGH_ENOMEM);
        cudaMemcpy(dw, wb.data(), nw * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(dX, X, size_t(n) * MLP_IN * sizeof(float), cudaMemcpyHostToDevice);
        k_mlp_zero<<<1, 256>>>(dw, d0);
        const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
        k_closure_apply<<<blocks, 256>>>(dw, nw == size_t(MLP_NPARAM) ? nullptr : dw + MLP_NPARAM, d0, dX, nullptr, n, 1,
                                         nullptr, nullptr, dy);
        cudaError_t e = cudaMemcpy(y, dy, size_t(n) * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return mlp_fail(std::string("closure eval: ") + cudaGetErrorString(e), DGH_ECUDA);
        return DGH_OK;
    });
}

int dgh_mlp_loss_grad(const float *w, const float *X, const float *Y, int64_t n, double *loss, float *grad) {
    return dgh_guarded(nullptr, [&]() -> int {
        if (!w || !X || !Y || n < 1 || !loss || !grad) return mlp_fail("mlp loss/grad: invalid arguments", DGH_EINVAL);
        int sms = 1, rc = mlp_setup(sms);
        if (rc) return rc;
        const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + MLP_BS - 1) / MLP_BS, int64_t(2) * sms));
        DevScratch d;
        float *dw = d.get<float>(MLP_NPARAM), *dX = d.get<float>(size_t(n) * MLP_IN), *dY = d.get<float>(size_t(n));
        float *dpart = d.get<float>(size_t(nblocks) * (MLP_NPARAM + 1)), *dg = d.get<float>(MLP_NPARAM);
        double *dl = d.get<double>(1);
        if (!dw || !dX || !dY || !dpart || !dg || !dl) return mlp_fail("mlp loss/grad: device allocation failed", DGH_ENOMEM);
        cudaMemcpy(dw, w, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(dX, X, size_t(n) * MLP_IN * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(dY, Y, size_t(n) * sizeof(float), cudaMemcpyHostToDevice);
        if ((rc = mlp_loss_grad_dev(dw, dX, dY, nullptr, n, dpart, nblocks, dg, dl))) return rc;
        cudaMemcpy(grad, dg, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
        cudaError_t e = cudaMemcpy(loss, dl, sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return mlp_fail(std::string("mlp loss/grad: ") + cudaGetErrorString(e), DGH_ECUDA);
        return DGH_OK;
    });
}

int dgh_closure_fit_homogeneous(const float *X, const float *Y, int64_t n, const dgh_train_cfg *cfg, float *w_out,
                                double *loss_hist, double *final_mse) {
    return dgh_guarded(nullptr, [&]() -> int {
        if (!X || !Y || n < 2 || !cfg || !w_out) return mlp_fail("closure fit: invalid arguments", DGH_EINVAL);
        // per-feature RMS scales sigma_i and the target's sigma_y (FP64)
        double sx[MLP_IN] = {0}, sy = 0.0;
        for (int64_t r = 0; r < n; ++r) {
            for (int i = 0; i < MLP_IN; ++i) sx[i] += double(X[r * MLP_IN + i]) * X[r * MLP_IN + i];
            sy += double(Y[r]) * Y[r];
        }
        for (int i = 0; i < MLP_IN; ++i) {
            sx[i] = std::sqrt(sx[i] / double(n));
            if (!(sx[i] > 0.0)) sx[i] = 1.0;
        }
        sy = std::sqrt(sy / double(n));
        if (!(sy > 0.0)) sy = 1.0;
        // directions u = x~ / |x~| (x~ = x / sigma) and relative targets y / (sigma_y |x~|);
        // rows with zero features carry no direction and are dropped
        std::vector<float> U, V;
        U.reserve(size_t(n) * MLP_IN);
        V.reserve(size_t(n));
        for (int64_t r = 0; r < n; ++r) {
            double xt[MLP_IN], s2 = 0.0;
            for (int i = 0; i < MLP_IN; ++i) {
                xt[i] = X[r * MLP_IN + i] / sx[i];
                s2 += xt[i] * xt[i];
            }
            const double sn = std::sqrt(s2);
            if (!(sn > 0.0)) continue;
            for (int i = 0; i < MLP_IN; ++i) U.push_back(float(xt[i] / sn));
            V.push_back(float(Y[r] / (sy * sn)));
        }
        const int64_t m = int64_t(V.size());
        if (m < 2) return mlp_fail("closure fit: fewer than 2 rows with non-zero features", DGH_EINVAL);
        int rc = dgh_mlp_train(U.data(), V.data(), m, cfg, w_out, loss_hist, final_mse);
        if (rc) return rc;
        for (int i = 0; i < MLP_IN; ++i) w_out[MLP_NPARAM + i] = float(1.0 / sx[i]);
        w_out[MLP_NPARAM + MLP_IN] = float(sy);
        return DGH_OK;
    });
}

int dgh_mlp_train(const float *X, const float *Y, int64_t n, const dgh_train_cfg *cfg, float *w_out, double *loss_hist,
                  double *final_mse) {
    return dgh_guarded(nullptr, [&]() -> int {
        ApiRange nvtx_range("dgh_mlp_train");
        if (!X || !Y || n < 2 || !cfg || !w_out || cfg->steps < 0 || cfg->batch < 1 || !(cfg->lr > 0.f))
            return mlp_fail("mlp train: invalid arguments", DGH_EINVAL);
        int sms = 1, rc = mlp_setup(sms);
        if (rc) return rc;
        // standardise inputs and target (folded back into the weights at the end)
        double mu[MLP_IN + 1] = {0}, sd[MLP_IN + 1] = {0};
        for (int64_t r = 0; r < n; ++r) {
            for (int i = 0; i < MLP_IN; ++i) mu[i] += X[r * MLP_IN + i];
            mu[MLP_IN] += Y[r];
        }
        for (int i = 0; i <= MLP_IN; ++i) mu[i] /= double(n);
        for (int64_t r = 0; r < n; ++r) {
            for (int i = 0; i < MLP_IN; ++i) sd[i] += (X[r * MLP_IN + i] - mu[i]) * (X[r * MLP_IN + i] - mu[i]);
            sd[MLP_IN] += (Y[r] - mu[MLP_IN]) * (Y[r] - mu[MLP_IN]);
        }
        for (int i = 0; i <= MLP_IN; ++i) sd[i] = std::sqrt(sd[i] / double(n)) > 1e-30 ? std::sqrt(sd[i] / double(n)) : 1.0;
        std::vector<float> Xn(static_cast<size_t>(n) * MLP_IN), Yn(static_cast<size_t>(n));
        for (int64_t r = 0; r < n; ++r) {
            for (int i = 0; i < MLP_IN; ++i) Xn[r * MLP_IN + i] = float((X[r * MLP_IN + i] - mu[i]) / sd[i]);
            Yn[r] = float((Y[r] - mu[MLP_IN]) / sd[MLP_IN]);
        }
        // Glorot-uniform initial weights (splitmix64 stream), zero biases
        std::vector<float> w(MLP_NPARAM, 0.f);
        uint64_t st = cfg->seed;
        auto uni = [&]() {
            st += 0x9E3779B97F4A7C15ull;
            uint64_t z = st;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            return double(z >> 11) / double(1ull << 53);
        };
        auto glorot = [&](int off, int fan_in, int fan_out, int count) {
            const double a = std::sqrt(6.0 / (fan_in + fan_out));
            for (int i = 0; i < count; ++i) w[off + i] = float((2.0 * uni() - 1.0) * a);
        };
        glorot(MLP_OW1, MLP_IN, MLP_H, MLP_H * MLP_IN);
        glorot(MLP_OW2, MLP_H, MLP_H, MLP_H * MLP_H);
        glorot(MLP_OW3, MLP_H, 1, MLP_H);
        const int64_t bs = std::min<int64_t>(cfg->batch, n);
        const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>((bs + MLP_BS - 1) / MLP_BS, int64_t(2) * sms));
        DevScratch d;
        float *dw = d.get<float>(MLP_NPARAM), *dX = d.get<float>(size_t(n) * MLP_IN), *dY = d.get<float>(size_t(n));
        float *dm = d.get<float>(MLP_NPARAM), *dv = d.get<float>(MLP_NPARAM), *dg = d.get<float>(MLP_NPARAM);
        float *dpart = d.get<float>(size_t(2 * sms) * (MLP_NPARAM + 1));
        int64_t *didx = d.get<int64_t>(size_t(bs));
        double *dl = d.get<double>(size_t(std::max<int64_t>(cfg->steps, 1)) + 1);
        if (!dw || !dX || !dY || !dm || !dv || !dg || !dpart || !didx || !dl)
            return mlp_fail("mlp train: device allocation failed", DGH_ENOMEM);
        cudaMemcpy(dw, w.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(dX, Xn.data(), Xn.size() * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(dY, Yn.data(), Yn.size() * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemset(dm, 0, MLP_NPARAM * sizeof(float));
        cudaMemset(dv, 0, MLP_NPARAM * sizeof(float));
        const float b1 = cfg->beta1 > 0.f ? cfg->beta1 : 0.9f, b2 = cfg->beta2 > 0.f ? cfg->beta2 : 0.999f;
        const float eps = cfg->eps > 0.f ? cfg->eps : 1e-8f;
        double pb1 = 1.0, pb2 = 1.0;
        for (int64_t it = 0; it < cfg->steps; ++it) {
            k_batch_indices<<<(int)((bs + 255) / 256), 256>>>(didx, bs, n, cfg->seed * 0x100000001B3ull + uint64_t(it));
            if ((rc = mlp_loss_grad_dev(dw, dX, dY, didx, bs, dpart, nblocks, dg, dl + it))) return rc;
            pb1 *= b1;
            pb2 *= b2;
            k_adam<<<(MLP_NPARAM + 255) / 256, 256>>>(dw, dg, dm, dv, MLP_NPARAM, cfg->lr, b1, b2, eps, float(1.0 - pb1),
                                                      float(1.0 - pb2));
        }
        // final loss on all rows (normalised units)
        const int nbf = (int)std::max<int64_t>(1, std::min<int64_t>((n + MLP_BS - 1) / MLP_BS, int64_t(2) * sms));
        if ((rc = mlp_loss_grad_dev(dw, dX, dY, nullptr, n, dpart, nbf, dg, dl + cfg->steps))) return rc;
        std::vector<double> hist(size_t(cfg->steps) + 1);
        cudaMemcpy(w.data(), dw, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
        cudaError_t e = cudaMemcpy(hist.data(), dl, hist.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return mlp_fail(std::string("mlp train: ") + cudaGetErrorString(e), DGH_ECUDA);
        // losses are 0.5 * mean squared error of the standardised target
        if (loss_hist)
            for (int64_t it = 0; it < cfg->steps; ++it) loss_hist[it] = 2.0 * hist[size_t(it)] * sd[MLP_IN] * sd[MLP_IN];
        if (final_mse) *final_mse = 2.0 * hist[size_t(cfg->steps)] * sd[MLP_IN] * sd[MLP_IN];
        // fold the standardisation into the weights: raw features in, raw target out
        for (int j = 0; j < MLP_H; ++j) {
            double b = w[MLP_OB1 + j];
            for (int i = 0; i < MLP_IN; ++i) {
                const double wi = w[MLP_OW1 + j * MLP_IN + i] / sd[i];
                b -= wi * mu[i];
                w_out[MLP_OW1 + j * MLP_IN + i] = float(wi);
            }
            w_out[MLP_OB1 + j] = float(b);
        }
        for (int i = MLP_OW2; i < MLP_OW3; ++i) w_out[i] = w[i];
        for (int j = 0; j < MLP_H; ++j) w_out[MLP_OW3 + j] = float(w[MLP_OW3 + j] * sd[MLP_IN]);
        w_out[MLP_OB3] = float(w[MLP_OB3] * sd[MLP_IN] + mu[MLP_IN]);
        return DGH_OK;
    });
}


}  // extern "C"

namespace {

// One thread waits, with the kernels' bounded-wait helper and a short limit,
// on an mbarrier phase that nothing completes; it gives up, sets the error
// word and returns.
__global__ void k_selftest_wait(int *err, unsigned long long limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait(&bar, 0, err, limit);
    }
}

}  // namespace

namespace {

// FP32 throughput probes: 8 independent FMA chains per thread (scalar or
// packed FP32x2), enough CTAs to fill every SM; the result is stored only
// under a condition that never holds, so the chains stay live.
__global__ void __launch_bounds__(256) k_probe_ffma(float *out, int iters, float sink) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 1e-7f + j;
    const float b = 0.999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == sink) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_ffma2(float *out, int iters, float sink) {
    float2 a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = make_float2(threadIdx.x * 1e-7f + j, threadIdx.x * 2e-7f + j);
    const float2 b = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = __ffma2_rn(a[j], b, c);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j].x + a[j].y;
    if (s == sink) out[blockIdx.x] = s;
}

}  // namespace

extern "C" int dgh_fp32_probe(double *tflops_ffma, double *tflops_ffma2) {
    return dgh_guarded(nullptr, [&]() -> int {
        if (!tflops_ffma || !tflops_ffma2) return mlp_fail("fp32 probe: null output", DGH_EINVAL);
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        DevScratch d;
        float *out = d.get<float>(size_t(sms) * 64);
        cudaEvent_t e0, e1;
        if (!out || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            return mlp_fail("fp32 probe: set-up failed", DGH_ECUDA);
        const int blocks = sms * 8, iters = 1 << 14;
        double best[2] = {0.0, 0.0};
        for (int kind = 0; kind < 2; ++kind)
            for (int rep = 0; rep < 4; ++rep) {   // first repetition warms up
                cudaEventRecord(e0);
                if (kind == 0) k_probe_ffma<<<blocks, 256>>>(out, iters, -1.f);
                else k_probe_ffma2<<<blocks, 256>>>(out, iters, -1.f);
                cudaEventRecord(e1);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                const double fma = double(blocks) * 256 * iters * 8 * (kind == 0 ? 1 : 2);
                if (rep > 0) best[kind] = std::max(best[kind], 2.0 * fma / (ms * 1e-3) / 1e12);
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return mlp_fail(std::string("fp32 probe: ") + cudaGetErrorString(e), DGH_ECUDA);
        *tflops_ffma = best[0];
        *tflops_ffma2 = best[1];
        return DGH_OK;
    });
}

extern "C" int dgh_selftest_throw(int kind) {
    return dgh_guarded(nullptr, [&]() -> int {
        if (kind == 0) throw std::bad_alloc();
        if (kind == 1) throw std::runtime_error("self-test exception");
        if (kind == 2) throw kind;
        return DGH_OK;
    });
}

extern "C" int dgh_selftest_wait(dgh_ctx *ctx, int64_t limit) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || limit < 1) return DGH_EINVAL;
        k_selftest_wait<<<1, 32, 0, ctx->stream>>>(ctx->d_err, (unsigned long long)limit);
        CK(cudaGetLastError());
        return dgh_sync(ctx);
    });
}

extern "C" int dgh_clear_error(dgh_ctx *ctx) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx) return DGH_EINVAL;
        CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return DGH_OK;
    });
}

extern "C" {
}  // extern "C"

// ============================================================================
// Energy without any device allocation.
//
// Some callers cannot allocate device memory at the moment they want the
// energy: code embedded in a host framework whose memory pool owns the whole
// device and forbids allocations outside it, or a monitoring loop on a
// latency-critical path where cudaMalloc's implicit device synchronisation is
// not acceptable.  This entry point therefore keeps its per-block partial
// sums in a fixed file-scope device array instead of allocating them.  The
// array is kNoAllocMaxPartials doubles (512 KiB) and stays resident on every
// GPU that loads the library until the process exits.
namespace {

constexpr int64_t kNoAllocMaxPartials = 65536;
constexpr int kNoAllocBlock = 256;
__device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[256] = {};   // device address of g_noalloc_partials, per device ordinal

// Per-device look-up of the array's device address (host code cannot use
// the symbol itself as a device pointer).
int noalloc_scratch(dgh_ctx *ctx, double **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        ctx->err = "device ordinal out of range for the static scratch table";
        return DGH_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) {
            ctx->err = std::string("cudaGetSymbolAddress(static energy scratch): ") + cudaGetErrorString(e);
            return DGH_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return DGH_OK;
}

// One block per kNoAllocBlock (cell, field) items; block b writes partial[b].
// FP64 throughout, as k_energy_partial: widened fields, FP64 mass matrix
// (dynamic shared memory), FP64 sums.
template <int N>
__global__ void __launch_bounds__(kNoAllocBlock) k_energy_partial_fixed(const float *q, const double *Md, const double *ew,
                                                                        int64_t K, double *partial) {
    constexpr int NP = Ord<N>::NP;
    extern __shared__ double sMf[];
    __shared__ double red[kNoAllocBlock];
    for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) sMf[i] = Md[i];
    __syncthreads();
    const int64_t it = blockIdx.x * (int64_t)kNoAllocBlock + threadIdx.x;
    double acc = 0.0;
    if (it < K * 4) {
        const int64_t k = it / 4;
        const int fl = (int)(it % 4);
        const float *x = q + (k / 32) * (4 * NP * 32) + fl * NP * 32 + (k % 32);
        for (int n = 0; n < NP; ++n) {
            double y = 0.0;
            for (int m = 0; m < NP; ++m) y += sMf[n * NP + m] * (double)x[m * 32];
            acc += (double)x[n * 32] * y;
        }
        acc *= ew[2 * k + (fl == 0 ? 0 : 1)];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kNoAllocBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

template <int N>
struct EnergyFixed {
    static int run(dgh_ctx *ctx, double *scratch, int nb, cudaStream_t s) {
        const size_t smem = energy_smem(N);
        cudaFuncSetAttribute(k_energy_partial_fixed<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_energy_partial_fixed<N><<<nb, kNoAllocBlock, smem, s>>>(ctx->q3, ctx->M3d, ctx->ew, ctx->K32 * 32, scratch);
        return DGH_OK;
    }
};

}  // namespace

extern "C" int dgh_get_energy_noalloc(dgh_ctx *ctx, double *d_energy, void *stream) {
    return dgh_guarded(err_slot(ctx), [&]() -> int {
        if (!ctx || !d_energy) return DGH_EINVAL;
        const int64_t nblocks = (ctx->K32 * 32 * 4 + kNoAllocBlock - 1) / kNoAllocBlock;
        if (nblocks > kNoAllocMaxPartials) {
            ctx->err = "dgh_get_energy_noalloc: " + std::to_string(ctx->K) + " cells need " + std::to_string(nblocks) +
                       " partial sums, more than the static scratch holds (" + std::to_string(kNoAllocMaxPartials) +
                       ", i.e. at most " + std::to_string(kNoAllocMaxPartials * kNoAllocBlock / 4) + " cells)";
            return DGH_EINVAL;
        }
        double *scratch = nullptr;
        int rc = noalloc_scratch(ctx, &scratch);
        if (rc) return rc;
        cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
        if (s != ctx->stream) {   // the fields are written on the context's stream: read them after that work
            CK(cudaEventRecord(ctx->ev_order, ctx->stream));
            CK(cudaStreamWaitEvent(s, ctx->ev_order, 0));
        }
        const int nb = (int)nblocks;
        dispatchN<EnergyFixed>(ctx->N, ctx, scratch, nb, s);
        k_sum_partials<<<1, 256, 0, s>>>(scratch, nb, d_energy);
        CK(cudaGetLastError());
        return DGH_OK;
    });
}
