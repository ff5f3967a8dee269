/*
 * dgh.h -- C ABI of the B300 nodal DG acoustic solver with high-order
 * absorbing boundary conditions (HABC) and edge/corner compatibility
 * (Modave, Atle, Chan, Warburton, arXiv 1610.05023).
 *
 * One context = one problem on one GPU: a conforming tetrahedral mesh of a
 * cuboid, the 3D pressure-velocity system (Sec. 2, eqs. pressureEqn /
 * velocityEqn) discretised by nodal DG with upwind fluxes (Sec. 3.2), and the
 * Pade HABC of order P on the boundary faces with its 2D face, 1D edge and
 * 0D corner solvers (Sec. 2.3, Sec. 3.1, Algorithm 1), advanced by the
 * 5-stage low-storage RK4 (eqs. timeStepProc1-2).
 *
 * Conventions shared by every call
 *  - Status: every int-returning call returns DGH_OK (0) or a negative code;
 *    dgh_last_error() gives a message.  No call aborts or throws: a C++
 *    exception inside a call is caught at the boundary (a failed host
 *    allocation returns DGH_ENOMEM, anything else DGH_EINVAL, with a message
 *    starting "internal error:"), and a create call that fails for any reason
 *    frees everything it had built.
 *  - Memory: arrays passed in are HOST arrays owned by the caller and only
 *    read during the call (copied).  Arrays passed out are HOST arrays owned
 *    by the caller, of the size stated, written during the call.  All device
 *    memory is owned by the context and freed by dgh_destroy().
 *  - Streams: all device work of a context runs on the stream given to
 *    dgh_create (NULL = the legacy default stream).  dgh_step() is
 *    asynchronous; errors of launched work surface at the next synchronising
 *    call (dgh_sync, read-backs) as DGH_ECUDA.
 *  - Notation: N = polynomial degree (the paper's P), P = HABC order (the
 *    paper's N, number of auxiliary fields per face).  Np = (N+1)(N+2)(N+3)/6,
 *    Np2 = (N+1)(N+2)/2, Np1 = N+1.
 *
 * Canonical layouts (read-back order; independent of the device layout)
 *  - Level 3 (tetrahedra): [K][4][Np], fields (p, u, v, w).
 *  - Level 2 (triangles = cell faces on HABC faces, P >= 1): [Ktri][P][3][Np2],
 *    fields (p_a, v1, v2): the auxiliary pressure of set a and the velocity
 *    components along the two in-plane axes in increasing axis order.
 *    Triangles are the HABC boundary cell faces in increasing order of
 *    (cell, local face); a triangle's nodes are the face nodes of its cell.
 *  - Level 1 (line cells on edges between two HABC faces A < B):
 *    [Klin][P*P][2][Np1], fields (p_ab, w) with set s = a + P*b and w the
 *    velocity along the edge axis.  Lines are enumerated by their face-A
 *    triangle, then the triangle's local edge; nodes run along +axis.
 *  - Reference nodes: Warp & Blend (Warburton 2006); node order = lattice
 *    order (tet: t outer, s middle, r inner; triangle: s outer, r inner).
 *  - Local faces of a tet (v0..v3): (v0,v1,v2), (v0,v1,v3), (v1,v2,v3),
 *    (v0,v2,v3), i.e. t=-1, s=-1, r+s+t=-1, r=-1 of the reference tet.
 *  - Domain faces d = 0..5: -x, +x, -y, +y, -z, +z.
 *  - "state" read/write gives the time-stepped variables: for levels 2 and 1
 *    the temporary fields p* of eqs. proc:pi00Star / proc:pij0Star instead
 *    of the full auxiliary pressure; "fields" give the full pressures.
 */
#ifndef DGH_H
#define DGH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define DGH_OK            0
#define DGH_EINVAL       -1   /* invalid argument (null pointer, bad size, bad mesh) */
#define DGH_ENOMEM       -2   /* device or host allocation failed */
#define DGH_ECUDA        -3   /* CUDA runtime error (launch or asynchronous) */
#define DGH_EUNSTABLE    -4   /* non-finite energy, or energy above the watchdog bound (dgh_set_watchdog) */
#define DGH_ETIMEOUT     -5   /* a bounded device-side wait gave up (reported by dgh_sync) */
#define DGH_ESTATE       -6   /* call not valid in the current state */
#define DGH_EUNSUPPORTED -7   /* feature / order not compiled in */
#define DGH_EBOUNDS      -8   /* checked build: an index outside its array, access skipped (reported by dgh_sync) */

/* Boundary condition of a domain face. */
#define DGH_BC_HABC       0   /* Pade HABC of order P (P = 0: basic ABC, Sec. 3.2) */
#define DGH_BC_DIRICHLET  1   /* p = 0 (free surface, Sec. 2.4, Sec. 3.2)         */

/* Arithmetic of the 3D volume / lift contractions (the products
 * D_j x and LIFT x of eq. dgLocalRhs); everything else (fluxes, update,
 * 2D/1D/0D levels) is FP32 in every mode.  The tensor-core modes run the
 * products on tcgen05 tensor cores with FP32 accumulation in tensor memory.
 * DGH_PREC_FP32 is the plain path held to the FP32 contract (relative L2
 * error <= 1e-5 per field against the FP64 oracle) and picks the faster of
 * its two kernels: at N = 4 with at least 65,536 cells the split-TF32
 * tensor-core kernel (each operand to 2^-22, three products, a few units of
 * FP32 rounding), otherwise the FP32 CUDA-core kernel (measured faster at
 * N = 1, 2, 3 at every size, and at N = 4 on small meshes; N >= 5 has no
 * split-TF32 kernel).  DGH_PREC_FP32_CUDA forces the CUDA-core kernel at
 * every order and size (packed FP32 FMAs, no tensor cores);
 * DGH_PREC_SPLIT_TF32 forces the split-TF32 kernel (N <= 4 only:
 * DGH_EUNSUPPORTED otherwise). */
#define DGH_PREC_FP32        0   /* FP32 contract: split TF32 (N = 4, >= 65,536 cells), else CUDA cores */
#define DGH_PREC_BF16_TC     1   /* BF16 operands, one product                    */
#define DGH_PREC_FP16_TC     2   /* FP16 operands, one product                    */
#define DGH_PREC_SPLIT_BF16  3   /* x = hi + lo in BF16, hi*hi + lo*hi + hi*lo    */
#define DGH_PREC_FP32_CUDA   4   /* FP32 CUDA cores at every order (the fallback)  */
#define DGH_PREC_SPLIT_TF32  5   /* x = hi + lo in TF32, hi*hi + lo*hi + hi*lo (N <= 4) */

typedef struct dgh_ctx dgh_ctx;

/* Problem description (all pointers: host, read during dgh_create only). */
typedef struct dgh_desc {
    int32_t        order;        /* N, 1..6                                     */
    int32_t        habc_order;   /* P, 0..12 (common to all HABC faces)          */
    int32_t        bc[6];        /* DGH_BC_* per domain face                     */
    int32_t        precision;    /* DGH_PREC_* (batches group problems by N, P and precision) */
    int32_t        reserved0;
    int64_t        n_vertices;
    int64_t        n_cells;
    const double  *vertices;     /* [n_vertices][3]                              */
    const int32_t *cells;        /* [n_cells][4] 0-based vertex ids              */
    const double  *c;            /* [n_cells] wave speed (constant per cell)     */
    const double  *rho;          /* [n_cells] density                            */
    double         dt;           /* > 0: time step; <= 0: cfl * min_k 1/(c_k (N+1)^2 Fscale_k) */
    double         cfl;          /* used when dt <= 0 (eq. validBench:timeStep, min over cells) */
} dgh_desc;

typedef struct dgh_info {
    int32_t order, habc_order, Np, Np2, Np1, n_corners;
    int64_t n_cells, n_tris, n_lines, n_bfaces;
    int64_t ndof;                /* 4 Np K + 3 P Np2 Ktri + 2 P^2 Np1 Klin (Table 3 convention) */
    int64_t step_count;
    double  dt, time;
    int64_t device_bytes;        /* device memory held by the context            */
} dgh_info;

/* Builds the reference elements (Sec. 3.2), the volume / surface / line meshes
 * and their node maps (Sec. 3.2, Table 1), the geometric factors, the Pade
 * coefficients c_i = tan^2(i pi / M) (eq. approxRoot2) and the precomputed
 * solution operators of the edge and corner systems (Sec. 3.1, item 2), then
 * uploads everything.  All state starts at zero.  stream: a cudaStream_t or
 * NULL.  *out receives a new context (NULL on failure).
 * Errors: DGH_EINVAL for an invalid mesh (non-conforming, degenerate cell,
 * boundary face off the cuboid), DGH_EUNSUPPORTED for N or P out of range,
 * DGH_ENOMEM, DGH_ECUDA. */
int dgh_create(const dgh_desc *desc, void *stream, dgh_ctx **out);

/* Host-only dry run of dgh_create: validates the description, builds the
 * reference elements and the meshes on the CPU and fills *out (sizes, ndof,
 * time step) without touching any GPU.  device_bytes is left 0.  Same errors
 * as dgh_create except DGH_ENOMEM / DGH_ECUDA. */
int dgh_plan(const dgh_desc *desc, dgh_info *out);

/* Frees all device and host memory of the context (NULL is accepted). */
void dgh_destroy(dgh_ctx *ctx);

/* Message of the last failing call on this context (or of the last failing
 * dgh_create when ctx is NULL).  Never NULL; valid until the next call. */
const char *dgh_last_error(const dgh_ctx *ctx);

int dgh_get_info(const dgh_ctx *ctx, dgh_info *out);

/* Node coordinates of a level (3, 2 or 1) in the canonical order:
 * [K][Np][3], [Ktri][Np2][3] or [Klin][Np1][3].  count = number of doubles. */
int dgh_get_nodes(const dgh_ctx *ctx, int level, double *xyz, size_t count);

/* Sets the 3D pressure to amp * exp(-|x - x0|^2 / width^2) at the nodes
 * (nodal interpolation, computed on the GPU), the 3D velocity to zero and
 * every auxiliary field to zero; time and step count restart at 0. */
int dgh_init_gaussian(dgh_ctx *ctx, const double x0[3], double width, double amp);

/* Writes (set) or reads (get) the time-stepped variables of a level in the
 * canonical layout (FP64 on the host, FP32 on the device).  count = number of
 * doubles (level 3: K*4*Np; level 2: Ktri*P*3*Np2; level 1: Klin*P*P*2*Np1).
 * After a set the boundary algebra of Algorithm 1 is recomputed before the
 * next step. */
int dgh_set_state(dgh_ctx *ctx, int level, const double *in, size_t count);
int dgh_get_state(dgh_ctx *ctx, int level, double *out, size_t count);

/* dgh_set_state / dgh_get_state with FP32 host arrays, the precision of the
 * device state: the same canonical layout and counts (count = number of
 * floats), half the bytes over the host link, and the values pass unchanged
 * (a get after a set returns the floats that were set; dgh_set_state rounds
 * FP64 input to the same floats).  Synchronising; the host array may be
 * pageable or pinned (pinned memory transfers at the full link rate).
 * DGH_EINVAL on a size mismatch or a NULL array, DGH_ECUDA on a failed
 * transfer. */
int dgh_set_state_f32(dgh_ctx *ctx, int level, const float *in, size_t count);
int dgh_get_state_f32(dgh_ctx *ctx, int level, float *out, size_t count);

/* Like dgh_get_state but levels 2 and 1 return the full auxiliary pressures
 * p_a = p*_a + (r^- + r^+) (eq. proc:pi00Star) and
 * p_ab = p*_ab + C_ba Q_A,a + C_ab Q_B,b (eq. proc:pij0Star). */
int dgh_get_fields(dgh_ctx *ctx, int level, double *out, size_t count);

/* Initial state from 3D fields: q3d [K][4][Np] in canonical order (as
 * dgh_get_state level 3); every auxiliary field, the time and the step count
 * are set to zero, as by dgh_init_gaussian.  DGH_EINVAL on a size mismatch. */
int dgh_init_fields(dgh_ctx *ctx, const double *q3d, size_t count);

/* Changes the material: c, rho per cell (count = number of cells, positive
 * and finite).  The set-up that depends on it (impedances, upwind
 * coefficients of every level, time step unless the description fixed dt) is
 * rebuilt; the fields of all levels, the time, the step count, the point
 * sources, the launch shape and the watchdog carry over (the handle stays
 * valid).  A learned closure and a recording shadow chain are removed.  On
 * an error the context is unchanged.  DGH_ESTATE for a batch group. */
int dgh_set_material(dgh_ctx *ctx, const double *c, const double *rho, size_t count);

/* Horizontal layers, bottom to top: layer l holds the cells whose centroid
 * has z < z_top[l] (z_top increasing, nlayers - 1 values); the last layer
 * takes the rest.  Then as dgh_set_material. */
int dgh_set_material_layers(dgh_ctx *ctx, int nlayers, const double *z_top, const double *c, const double *rho);

/* Sets the simulated time (the step count is unchanged). */
int dgh_set_time(dgh_ctx *ctx, double t);

/* Adds a point source delta(x - xs) S(t) to the pressure equation, with S the
 * integral of the Ricker wavelet of peak frequency f_peak and delay t_s
 * (Sec. 4.1, eq. validBench:ricker), scaled by amp; discretised as
 * S(t) M_k^{-1} l(xs) in the cell k containing xs (lowest id on ties) and
 * evaluated at every RK stage time.  At most 64 sources per context.
 * Errors: DGH_EINVAL if xs lies outside the mesh. */
int dgh_add_point_source(dgh_ctx *ctx, const double xs[3], double f_peak, double t_s, double amp);

/* Advances nsteps LSERK4 steps on the context's stream (asynchronous unless
 * the watchdog is on).  With the watchdog on, returns DGH_EUNSTABLE after the
 * first checked step whose energy fails the check; the steps up to and
 * including it have been taken. */
int dgh_step(dgh_ctx *ctx, int64_t nsteps);

/* Energy watchdog.  The Pade HABC has a known slow error growth over long
 * times (Sec. 4.1); this guards long runs against it and against non-finite
 * values.  With every > 0, dgh_step computes the 3D energy (as dgh_get_energy)
 * after every step whose step count is a multiple of `every` and stops with
 * DGH_EUNSTABLE if it is not finite, or if energy_limit > 0 and the energy
 * exceeds energy_limit (the message in dgh_last_error gives the step and the
 * energy).  Each check synchronises the stream.  every = 0 turns it off.
 * DGH_EINVAL if every < 0 or energy_limit is not finite. */
int dgh_set_watchdog(dgh_ctx *ctx, int64_t every, double energy_limit);

/* Profiling aid: advances nsteps steps with direct launches (no graph),
 * bracketing every kernel launch with CUDA events on the context's stream.
 * out_ms[0..3] = mean duration of one launch of the 3D / 2D / 1D / 0D stage
 * kernels in milliseconds (0 for an absent level), out_ms[4] = mean duration
 * of a whole step.  Synchronising. */
int dgh_time_kernels(dgh_ctx *ctx, int64_t nsteps, double out_ms[5]);

/* Waits for the context's stream; reports asynchronous CUDA errors. */
int dgh_sync(dgh_ctx *ctx);

/* 1 in the checked build (libdgh_checked.so, compiled with -DDGH_CHECKED),
 * else 0.  In the checked build the stage kernels test every index they
 * gather through or push to against its array; a violation skips the access
 * and dgh_sync returns DGH_EBOUNDS.  Results are otherwise identical. */
int dgh_is_checked_build(void);

/* Discrete energy of the 3D fields,
 * E = sum_k |J_k| [p^T M p / (2 rho c^2) + (rho/2) sum_i u_i^T M u_i],
 * (Sec. 4.1, energy of the pressure-velocity system) reduced on the GPU in
 * FP64 throughout: the FP32 fields are widened, M is the FP64 mass matrix
 * and every product and sum is FP64 (synchronising). */
int dgh_get_energy(dgh_ctx *ctx, double *E);

/* Error reduction (Error(t)^2 = E(q - ref) / E_ref of the paper's accuracy
 * study, Sec. 4.1): *E = the discrete energy of the difference between the
 * 3D fields and ref, a HOST array [K][4][Np] in the canonical order of
 * dgh_get_state (count = K*4*Np doubles), with the FP64 mass matrix and FP64
 * arithmetic on the device (synchronising). */
int dgh_get_error_energy(dgh_ctx *ctx, const double *ref, size_t count, double *E);

/* Energy as dgh_get_energy, but the call allocates no memory at all: the
 * per-block partial sums live in a fixed static device array of the library
 * (65,536 doubles = 512 KiB, held on every GPU that loads the library until
 * the process exits).  Meant for callers that cannot allocate device memory
 * when they need the value: code inside a framework whose memory pool owns
 * the whole device, or a monitoring loop on a latency-critical path where
 * cudaMalloc's implicit device synchronisation is not acceptable.  The paper
 * has no counterpart; it is a service of this library.
 *  d_energy: DEVICE pointer to one double, owned by the caller, written on
 *            `stream` (NULL = the context's stream); asynchronous, read it
 *            after synchronising that stream.
 *  Ordering: when `stream` is not the context's stream, the call first makes
 *            `stream` wait (event record + stream wait) for all work enqueued
 *            on the context's stream so far, so the energy is that of the
 *            fields after the last dgh_step.
 *  Limit: at most 4,194,304 cells (65,536 partial sums of 256 (cell, field)
 *         items); larger contexts get DGH_EINVAL with a message.
 *  Arithmetic: FP64 throughout (FP64 mass matrix, FP64 sums), as dgh_get_energy.
 *  The first call on each device looks up the array's device address with
 *  cudaGetSymbolAddress, once per device.
 *  All calls share the one array (every partial sum is rewritten by each
 *  call, nothing needs clearing), so calls whose kernels overlap on the GPU
 *  -- e.g. on two streams at once -- race and must be serialised. */
int dgh_get_energy_noalloc(dgh_ctx *ctx, double *d_energy, void *stream);

/* FP32 CUDA-core throughput probe on the current device (the roofline's
 * compute bound for the FP32 path): TFLOP/s of scalar FFMA and of packed
 * FP32x2 FMA chains (8 independent chains per thread, all SMs, best of
 * three timed launches).  Errors via dgh_last_error(NULL). */
int dgh_fp32_probe(double *tflops_ffma, double *tflops_ffma2);

/* Failure-detection self-test: a one-thread kernel waits, with the bounded
 * wait of the stage kernels and a limit of `limit` polls, on an mbarrier
 * phase that nothing completes; it gives up and sets the context's error
 * word, and the call returns what dgh_sync then reports (DGH_ETIMEOUT).  No
 * fault, trap or endless wait is involved; the context stays usable.
 * dgh_clear_error resets the error word (synchronising). */
int dgh_selftest_wait(dgh_ctx *ctx, int64_t limit);
int dgh_clear_error(dgh_ctx *ctx);

/* Boundary self-test (host only, no GPU): throws inside the guard every entry
 * point runs under -- kind 0 std::bad_alloc (returns DGH_ENOMEM), 1 a
 * std::runtime_error, 2 a non-standard exception (both DGH_EINVAL); the
 * message ("internal error: ...") is in dgh_last_error(NULL).  Any other
 * kind throws nothing and returns DGH_OK. */
int dgh_selftest_throw(int kind);

/* Serialises the complete time-stepping state (all levels, residuals,
 * boundary algebra, time, step count) into buf.  Call with buf == NULL to
 * query the size in *size.  dgh_load_state restores it into a context
 * created from the same description.  DGH_EINVAL on size mismatch. */
int dgh_save_state(dgh_ctx *ctx, void *buf, size_t *size);
int dgh_load_state(dgh_ctx *ctx, const void *buf, size_t size);

/* ---------------------------------------------------------------- launch shapes
 * Launch shape of the stage kernels: the number of elements a CTA handles,
 * which the paper tunes per kernel as K_blk (Sec. 3.3, Tables 4-5), and the
 * number of persistent 3D CTAs.  tile2 = triangles per CTA of the 2D kernel
 * (one thread per triangle and HABC set: tile2 * P <= thr2), tile1 = line cells per CTA of the 1D kernel, cta3_per_sm = persistent 3D
 * CTAs per SM (0 = as many as fit).  grid3/grid2/grid1 (CTAs per launch),
 * occ3 (3D CTAs that fit on one SM) and sms are derived, read only.  A 3D
 * CTA always handles 32-cell blocks (one cell per lane). */
typedef struct dgh_launch {
    int32_t tile2, tile1, cta3_per_sm;
    int32_t grid3, grid2, grid1, occ3, sms;
    int32_t thr2, thr1;      /* threads per CTA of the 2D / 1D kernels: 32, 64, 128 or 256 */
    int32_t sm3_div;         /* the persistent 3D grid covers sms / sm3_div SMs (1..16; 1 = all) */
    int32_t split3;          /* 1: cells without and with HABC faces as two 3D launches per stage, so that
                                the HABC chain may overlap the first; 0: one 3D launch per stage */
    int32_t kern3;           /* read only: the 3D kernel, 0 FP32 CUDA cores, 1 split TF32, 2 BF16/FP16 */
} dgh_launch;

int dgh_get_launch(const dgh_ctx *ctx, dgh_launch *out);

/* Sets tile2, tile1, cta3_per_sm, thr2, thr1, sm3_div and split3 (the other fields are ignored).  No
 * result changes: every element's arithmetic is the same whatever the shape.
 * DGH_EINVAL if a value is out of range, tile2 * P > thr2, or a tile does not
 * fit in shared memory (the previous shape is kept). */
int dgh_set_launch(dgh_ctx *ctx, const dgh_launch *in);

/* Autotuner: coordinate search over thr2, tile2, thr1, tile1, cta3_per_sm, split3
 * (and, for the groups of a batch, which run concurrently, sm3_div), each
 * candidate timed with CUDA events over `steps` whole steps (best of two),
 * kept when at least 1% faster.  The fields, time and step count are saved
 * before and restored after (host copy of the state), so the search changes
 * no result.  ms_before / ms_after (may be NULL) receive the time of one
 * step before and after.  Synchronising; takes roughly
 * (3 + number of candidates) * 2 * steps steps of GPU time. */
int dgh_tune(dgh_ctx *ctx, int steps, double *ms_before, double *ms_after);

/* ---------------------------------------------------------------- batching
 * A batch steps many independent problems (each with its own mesh, material,
 * N, P, time step and sources) together: the problems are grouped by (N, P);
 * each group becomes one union context over all its problems' cells,
 * triangles, lines and corners, with each problem's time step folded into
 * its cells' coefficients, and one CUDA graph per step runs all groups
 * concurrently (one branch per group).  This is the paper's method applied
 * per problem (Algorithm 1 with eqs. timeStepProc1-2); the paper itself runs
 * one problem at a time. */
typedef struct dgh_batch dgh_batch;

/* Snapshots `count` problem contexts (mesh, material, N, P, time step,
 * sources, current fields, time, step count) into a new batch on the current
 * device.  The problem contexts are only read and stay valid and
 * independent: stepping the batch does not advance them.  Device memory of
 * the batch is separate from theirs.  At most 64 point sources per (N, P)
 * group.  Errors: DGH_EINVAL (null arguments, problems on another device, too
 * many sources), DGH_ENOMEM, DGH_ECUDA. */
int dgh_batch_create(dgh_ctx *const *problems, int count, dgh_batch **out);

/* Host-only dry run of the grouping: for the descriptions descs[0..count),
 * group_of[i] receives the group of problem i (groups numbered in order of
 * first appearance of their (N, P)), group_info[g] (room for `count`
 * entries) the sizes of the union mesh of group g (dt, time, step_count and
 * device_bytes are 0), *n_groups the number of groups.  No GPU is used. */
int dgh_batch_plan(const dgh_desc *descs, int count, int *group_of, dgh_info *group_info, int *n_groups);

void dgh_batch_destroy(dgh_batch *b);
const char *dgh_batch_last_error(const dgh_batch *b);   /* NULL: last failing dgh_batch_create */
int dgh_batch_count(const dgh_batch *b, int *n_problems, int *n_groups);

/* *stream receives the batch's own non-blocking cudaStream_t, on which all its
 * device work runs (owned by the batch, valid until dgh_batch_destroy): record
 * events on it, or make other streams wait on it. */
int dgh_batch_stream(const dgh_batch *b, void **stream);

/* Advances every problem by nsteps steps of its own time step (asynchronous,
 * on the batch's own stream; one graph launch per step). */
int dgh_batch_step(dgh_batch *b, int64_t nsteps);

/* Waits for the batch; reports asynchronous errors and timed-out waits
 * (DGH_ETIMEOUT) of any group. */
int dgh_batch_sync(dgh_batch *b);

/* Problem i (0-based, the order given to dgh_batch_create): sizes, its own
 * dt, time t0 + steps * dt and step count, in the layout and units of
 * dgh_get_info (device_bytes = those of its group). */
int dgh_batch_get_info(const dgh_batch *b, int i, dgh_info *out);

/* Problem i's time-stepped variables of a level in the canonical layout of
 * dgh_get_state (count as there, for that problem alone).  Synchronising. */
int dgh_batch_get_state(dgh_batch *b, int i, int level, double *out, size_t count);

/* Problem i's 3D energy as dgh_get_energy.  Synchronising. */
int dgh_batch_get_energy(dgh_batch *b, int i, double *E);

/* Launch shape of group g (0 <= g < n_groups). */
int dgh_batch_get_launch(const dgh_batch *b, int group, dgh_launch *out);

/* Autotuner of dgh_tune over the launch shapes of all groups, timed on whole
 * batch steps; fields, times and step counts are restored afterwards. */
int dgh_batch_tune(dgh_batch *b, int steps, double *ms_before, double *ms_after);

/* ---------------------------------------------------------------- learned closure
 * A learned correction of the face condition of a low-order HABC chain:
 * the exterior state seen by the 3D flux at a boundary face node becomes
 * 2 (r^- + MLP(x) - MLP(0)) instead of 2 r^- (eq. proc:pi00Star, r^- = (1/M) sum c_a p*_a;
 * the fields enter linearly, so zero fields give exactly zero correction),
 * with x = (p, n.u, p_1, p_2, dp*_1/dt, dp*_2/dt) at that node: the 3D trace
 * pressure and outward normal velocity, the full auxiliary pressures of sets
 * 1 and 2 (p_a = p*_a + r^- + r^+) and the time derivatives of p*_1, p*_2 of
 * the stage just computed (0 for sets beyond P).  The chain's own algebra
 * keeps the uncorrected r^-.  The paper has no learned component.
 * MLP 6 -> 64 (tanh) -> 64 (tanh) -> 1, DGH_MLP_NPARAM = 4673 parameters:
 * W1 [64][6], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 (row-major, in
 * that order).  Inference uses the weights rounded to BF16, FP32 arithmetic. */
#define DGH_MLP_NPARAM 4673

/* Enables the closure on this context with the given weights, or disables
 * it (w = NULL).  n = 4673: correction MLP(x) - MLP(0).  n = 4680: the
 * homogeneous form sigma_y |x~| MLP(x~ / |x~|) with x~_i = x_i / sigma_i,
 * the 4673 weights followed by 1/sigma_1..6 and sigma_y (kept FP32); it is of
 * degree one in the fields, as the linear equations require, and zero at
 * zero fields.  DGH_EINVAL without HABC faces (P = 0).  Not supported inside
 * a batch. */
int dgh_closure_set_weights(dgh_ctx *ctx, const float *w, size_t n);

/* Training data: adds a shadow HABC chain of order shadow_order (its own 2D
 * face, 1D edge and 0D corner fields, zero at start and after
 * dgh_init_gaussian) driven one-way by this context's 3D traces, and records
 * on every step that is a multiple of `every` (at its first stage) the rows
 * (x of the shadow chain, r^-_this - r^-_shadow) of a hashed fraction of the
 * boundary face nodes into a device buffer of max_samples rows (further rows
 * are dropped).  With the closure enabled on this context (a low order here,
 * a high shadow order), the rows are closed-loop instead: (x of this chain,
 * r^-_shadow - r^-_this), the correction the shadow order implies on the
 * trajectory the closure produces.  The shadow chain never changes this
 * context's solution. */
int dgh_closure_record(dgh_ctx *ctx, int shadow_order, int every, double fraction, int64_t max_samples, uint64_t seed);

/* Copies up to max_rows recorded rows [row][7] (6 features, target) into out
 * (host, caller-owned); *count = rows recorded (at most max_samples). */
int dgh_closure_samples(dgh_ctx *ctx, float *out, int64_t max_rows, int64_t *count);

/* Context-free device calls (current device; errors via dgh_last_error(NULL)).
 * dgh_closure_eval: the correction y[r] of the inference kernel for the
 * weights w of nw = 4673 or 4680 values (as dgh_closure_set_weights;
 * BF16-rounded network weights), X [n][6] host, y [n] host.
 * dgh_mlp_loss_grad: FP32 weights w, loss = (1/2n) sum (MLP(X_r) - Y_r)^2 and
 * its gradient with respect to w (host arrays), by the training kernels.
 * dgh_mlp_train: minibatch Adam (Kingma & Ba) on the GPU from seeded
 * Glorot-uniform weights, on standardised inputs and target; the returned
 * weights w_out take raw features and return the raw target.  loss_hist
 * (cfg->steps entries, or NULL) receives each minibatch's mean-squared error
 * and *final_mse (or NULL) that of all rows, both in target units. */
typedef struct dgh_train_cfg {
    int64_t steps;        /* Adam steps                                 */
    int64_t batch;        /* samples per step (drawn with replacement)  */
    float   lr;           /* learning rate                              */
    float   beta1, beta2; /* <= 0: 0.9, 0.999                           */
    float   eps;          /* <= 0: 1e-8                                 */
    uint64_t seed;        /* initial weights and batches                */
} dgh_train_cfg;

int dgh_closure_eval(const float *w, size_t nw, const float *X, int64_t n, float *y);
int dgh_mlp_loss_grad(const float *w, const float *X, const float *Y, int64_t n, double *loss, float *grad);
int dgh_mlp_train(const float *X, const float *Y, int64_t n, const dgh_train_cfg *cfg, float *w_out, double *loss_hist,
                  double *final_mse);

/* dgh_closure_fit_homogeneous: the homogeneous form of the closure, fitted
 * to raw features X [n][6] and targets Y [n] (host): per-feature RMS scales
 * sigma_i and the target's sigma_y (FP64), directions u = x~ / |x~| with
 * x~ = x / sigma and relative targets y / (sigma_y |x~|) (rows with zero
 * features dropped), then dgh_mlp_train on (u, relative target).  w_out
 * (host, 4680 floats) receives the 4673 network weights, 1/sigma_i and
 * sigma_y: the layout dgh_closure_set_weights takes for this form.  The
 * fitted correction sigma_y |x~| MLP(x~ / |x~|) is of degree one in the
 * fields, as the linear equations require.  loss_hist and final_mse are in
 * relative-target units.  DGH_EINVAL with fewer than 2 non-zero rows. */
int dgh_closure_fit_homogeneous(const float *X, const float *Y, int64_t n, const dgh_train_cfg *cfg, float *w_out,
                                double *loss_hist, double *final_mse);

/* Trains the closure on the rows this context has recorded
 * (dgh_closure_record): the same training as dgh_mlp_train on their
 * features and targets.  DGH_ESTATE without recording or with fewer than 2
 * rows. */
int dgh_closure_train(dgh_ctx *ctx, const dgh_train_cfg *cfg, float *w_out, double *loss_hist, double *final_mse);

/* The same rows fitted in the homogeneous form (dgh_closure_fit_homogeneous;
 * w_out: 4680 floats). */
int dgh_closure_train_homogeneous(dgh_ctx *ctx, const dgh_train_cfg *cfg, float *w_out, double *loss_hist,
                                  double *final_mse);

#ifdef __cplusplus
}
#endif

#endif /* DGH_H */
