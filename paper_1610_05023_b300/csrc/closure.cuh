// Learned boundary closure: a small MLP that corrects the incoming
// characteristic of a low-order HABC chain,
//   r^-_used = r^-_P + MLP(x) - MLP(0),  x = (p, n.u, p_1, p_2, dp*_1/dt, dp*_2/dt),
// or its homogeneous form sigma_y |x~| MLP(x~ / |x~|), x~ = x / sigma,
// evaluated per boundary face node; the data pipeline that records training
// samples from a high-order run with a low-order shadow chain; and the
// training kernels (forward, backward, gradient reduction, Adam).  The paper
// has no learned component: this extends its Pade chain (Sec. 2.1, eq.
// approxRoot2) with a correction of the face condition of eq. proc:pi00Star.
//
// MLP: 6 -> 64 (tanh) -> 64 (tanh) -> 1.  Parameter vector (4673 floats):
//   W1 [64][6], b1 [64], W2 [64][64], b2 [64], w3 [64], b3.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgh {

constexpr int MLP_IN = 6, MLP_H = 64;
constexpr int MLP_OW1 = 0, MLP_OB1 = MLP_OW1 + MLP_H * MLP_IN, MLP_OW2 = MLP_OB1 + MLP_H,
              MLP_OB2 = MLP_OW2 + MLP_H * MLP_H, MLP_OW3 = MLP_OB2 + MLP_H, MLP_OB3 = MLP_OW3 + MLP_H;
constexpr int MLP_NPARAM = MLP_OB3 + 1;   // 4673
constexpr int SAMPLE_W = MLP_IN + 1;      // recorded sample: 6 features, target
constexpr int CL_MLP0 = MLP_NPARAM + MLP_IN + 1;   // device weight block: weights, 7 scales, then MLP(0)

// Forward pass of one sample with the weights in shared memory, arranged for
// throughput: the hidden activations as (h[k], h[k+1]) register pairs, each
// W2 row read as float4s (w 16-byte aligned), packed FP32x2 FMAs over the even
// and odd k of a row.
__device__ __forceinline__ float mlp_forward(const float *w, const float (&x)[MLP_IN]) {
    float2 h[MLP_H / 2];
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) {
        float z = w[MLP_OB1 + j];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) z += w[MLP_OW1 + j * MLP_IN + i] * x[i];
        if (j & 1) h[j >> 1].y = tanhf(z);
        else h[j >> 1].x = tanhf(z);
        asm volatile("" ::: "memory");   // one activation at a time (register pressure)
    }
    float y = w[MLP_OB3];
    const float4 *w2 = reinterpret_cast<const float4 *>(w + MLP_OW2);
#pragma unroll 1
    for (int j = 0; j < MLP_H; ++j) {
        float2 z2 = make_float2(0.f, 0.f);   // (sum over even k, sum over odd k)
#pragma unroll
        for (int k4 = 0; k4 < MLP_H / 4; ++k4) {
            const float4 a = w2[j * (MLP_H / 4) + k4];
            z2 = __ffma2_rn(make_float2(a.x, a.y), h[2 * k4], z2);
            z2 = __ffma2_rn(make_float2(a.z, a.w), h[2 * k4 + 1], z2);
        }
        y += w[MLP_OW3 + j] * tanhf(w[MLP_OB2 + j] + (z2.x + z2.y));
    }
    return y;
}
static_assert(MLP_OW2 % 4 == 0 && MLP_H % 4 == 0, "W2 rows must be float4-aligned");

// MLP(0) with the inference code and the weights in shared memory, as
// k_closure_apply evaluates every row (one block; the value goes to *y0).
__global__ void k_mlp_zero(const float *wts, float *y0) {
    __shared__ __align__(16) float sw[MLP_NPARAM];
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) sw[i] = wts[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        const float z[MLP_IN] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        *y0 = mlp_forward(sw, z);
    }
}

// The correction y of one feature row x (overwritten): MLP(x) - y0 with y0 =
// MLP(0), or, with the homogeneous form (ssc = 1/sigma of the 6 features,
// then sigma_y), sigma_y |x~| MLP(x~ / |x~|), x~ = x / sigma, 0 at x~ = 0.
// w: the weights in shared memory.
__device__ __forceinline__ float closure_y(const float *w, const float *ssc, bool homog, float y0,
                                           float (&x)[MLP_IN]) {
    float amp = 1.f, off = y0;   // y = amp * MLP(x') - off
    if (homog) {
        float s2 = 0.f;
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) {
            x[i] *= ssc[i];
            s2 += x[i] * x[i];
        }
        const float sn = sqrtf(s2);
        const float inv = sn > 1e-30f ? 1.0f / sn : 0.f;
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) x[i] *= inv;
        amp = sn > 1e-30f ? ssc[MLP_IN] * sn : 0.f;
        off = 0.f;
    }
    const float m = mlp_forward(w, x);
    return amp == 0.f ? 0.f : amp * m - off;
}

// Inference: the correction y = MLP(feat) - MLP(0) for n feature rows (the
// fields enter linearly, so no fields must give no correction; MLP(0) comes
// from k_mlp_zero, the same code with the same weights, so y(0) = 0 exactly).
// When tin3 is given, the corrected exterior state 2 (r^- + y) of every
// boundary face node of the chain goes to the 3D incoming traces (rows =
// triangle nodes t * NP2 + node).
// Homogeneous form (scales != NULL: 1/sigma_i of the 6 features, then
// sigma_y): x~ = x / sigma, s = |x~|, y = sigma_y s MLP(x~ / s), 0 at s = 0 --
// the correction is then of degree one in the fields, as the linear wave
// equation requires, and the network sees only the direction of x.
__global__ void __launch_bounds__(256) k_closure_apply(const float *wts, const float *scales, const float *mlp0,
                                                       const float *feat, const float *rm, int64_t n, int np2,
                                                       const int *tri_face, float *tin3, float *y_out) {
    __shared__ __align__(16) float sw[MLP_NPARAM];
    __shared__ float ssc[MLP_IN + 1];
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) sw[i] = wts[i];
    if (threadIdx.x <= MLP_IN) ssc[threadIdx.x] = scales ? scales[threadIdx.x] : 1.f;
    const float y0 = scales ? 0.f : mlp0[0];   // MLP(0) (not used by the homogeneous form)
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        float x[MLP_IN];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) x[i] = feat[r * MLP_IN + i];
        const float y = closure_y(sw, ssc, scales != nullptr, y0, x);
        if (y_out) y_out[r] = y;
        if (tin3) {
            const int64_t t = r / np2;
            const int node = (int)(r % np2);
            const int64_t gf = tri_face[t], kc = gf >> 2;
            const int fc = (int)(gf & 3);
            tin3[((((kc >> 5) * 4 + fc) * np2 + node) * 32 + (kc & 31)) * 2] = 2.0f * (rm[r] + y);
        }
    }
}

// splitmix64 finaliser (Steele, Lea, Flood 2014): hashed sampling decisions
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Records (features of the shadow chain, r^-_main - r^-_shadow) of a hashed
// subset of boundary face nodes, on steps that are multiples of `every`
// (called after the stage-0 chains; the step counter is final by then).
__global__ void k_record_samples(const float *feat_s, const float *rm_s, const float *rm_main, int64_t n,
                                 const int64_t *step, int every, uint32_t threshold, uint64_t seed, float *out,
                                 unsigned long long *count, int64_t max_samples) {
    const int64_t st = step[0];
    if (every <= 0 || st % every != 0) return;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t h = (uint32_t)(mix64(seed ^ mix64((uint64_t)st * 0x100000001B3ull + (uint64_t)r)) >> 32);
        if (h >= threshold) continue;
        const unsigned long long slot = atomicAdd(count, 1ull);
        if ((int64_t)slot >= max_samples) continue;
        float *o = out + slot * SAMPLE_W;
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) o[i] = feat_s[r * MLP_IN + i];
        o[MLP_IN] = rm_main[r] - rm_s[r];
    }
}

// ------------------------------------------------------------ training
constexpr int MLP_BS = 128;   // samples per chunk = threads per block

// Loss 0.5/n sum (y - t)^2 -> the mean-squared error is twice it.  Each
// block accumulates its partial gradient over chunks of MLP_BS samples
// (sample indices from idx, or rows b0.. b0+n when idx is NULL) and writes
// it to partial[block][MLP_NPARAM + 1] (last entry: partial loss).
__global__ void __launch_bounds__(MLP_BS) k_mlp_grad(const float *wts, const float *X, const float *Y, const int64_t *idx,
                                                     int64_t n, double inv_n, float *partial) {
    extern __shared__ float sm_mlp[];
    float *sw = sm_mlp;                         // MLP_NPARAM
    float *sx = sw + MLP_NPARAM;                // BS * IN
    float *sh1 = sx + MLP_BS * MLP_IN;          // BS * H
    float *sh2 = sh1 + MLP_BS * MLP_H;          // BS * H
    float *sd2 = sh2 + MLP_BS * MLP_H;          // BS * H  dL/dz2
    float *sd1 = sd2 + MLP_BS * MLP_H;          // BS * H  dL/dz1
    float *sdy = sd1 + MLP_BS * MLP_H;          // BS      dL/dy
    const int tid = threadIdx.x;
    for (int i = tid; i < MLP_NPARAM; i += MLP_BS) sw[i] = wts[i];
    // this thread's parameters: p = tid + MLP_BS * q
    constexpr int PPT = (MLP_NPARAM + MLP_BS - 1) / MLP_BS;
    float g[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) g[q] = 0.f;
    double loss = 0.0;
    __syncthreads();
    const int64_t nchunks = (n + MLP_BS - 1) / MLP_BS;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t s = c * MLP_BS + tid;
        const bool ok = s < n;
        const int64_t row = ok ? (idx ? idx[s] : s) : 0;
        float x[MLP_IN];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) {
            x[i] = ok ? X[row * MLP_IN + i] : 0.f;
            sx[tid * MLP_IN + i] = x[i];
        }
        float h1[MLP_H];
#pragma unroll
        for (int j = 0; j < MLP_H; ++j) {
            float z = sw[MLP_OB1 + j];
#pragma unroll
            for (int i = 0; i < MLP_IN; ++i) z += sw[MLP_OW1 + j * MLP_IN + i] * x[i];
            h1[j] = tanhf(z);
            sh1[tid * MLP_H + j] = h1[j];
        }
        float y = sw[MLP_OB3];
        for (int j = 0; j < MLP_H; ++j) {
            float z = sw[MLP_OB2 + j];
#pragma unroll
            for (int k = 0; k < MLP_H; ++k) z += sw[MLP_OW2 + j * MLP_H + k] * h1[k];
            const float h = tanhf(z);
            sh2[tid * MLP_H + j] = h;
            y += sw[MLP_OW3 + j] * h;
        }
        const float e = ok ? y - Y[row] : 0.f;
        loss += 0.5 * (double)e * (double)e * inv_n;
        const float dy = (float)(e * inv_n);
        sdy[tid] = dy;
        // dz2_j = dy w3_j (1 - h2_j^2);  dh1_k = sum_j W2[j][k] dz2_j;  dz1_k = dh1_k (1 - h1_k^2)
        float dh1[MLP_H];
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) dh1[k] = 0.f;
        for (int j = 0; j < MLP_H; ++j) {
            const float h = sh2[tid * MLP_H + j];
            const float d2 = dy * sw[MLP_OW3 + j] * (1.f - h * h);
            sd2[tid * MLP_H + j] = d2;
#pragma unroll
            for (int k = 0; k < MLP_H; ++k) dh1[k] += sw[MLP_OW2 + j * MLP_H + k] * d2;
        }
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) sd1[tid * MLP_H + k] = dh1[k] * (1.f - h1[k] * h1[k]);
        __syncthreads();
        // parameter gradients summed over the chunk's samples
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int p = tid + MLP_BS * q;
            if (p >= MLP_NPARAM) break;
            float acc = 0.f;
            if (p < MLP_OB1) {                       // W1[j][i]
                const int j = p / MLP_IN, i = p % MLP_IN;
                for (int t = 0; t < MLP_BS; ++t) acc += sd1[t * MLP_H + j] * sx[t * MLP_IN + i];
            } else if (p < MLP_OW2) {                // b1[j]
                const int j = p - MLP_OB1;
                for (int t = 0; t < MLP_BS; ++t) acc += sd1[t * MLP_H + j];
            } else if (p < MLP_OB2) {                // W2[j][k]
                const int j = (p - MLP_OW2) / MLP_H, k = (p - MLP_OW2) % MLP_H;
                for (int t = 0; t < MLP_BS; ++t) acc += sd2[t * MLP_H + j] * sh1[t * MLP_H + k];
            } else if (p < MLP_OW3) {                // b2[j]
                const int j = p - MLP_OB2;
                for (int t = 0; t < MLP_BS; ++t) acc += sd2[t * MLP_H + j];
            } else if (p < MLP_OB3) {                // w3[j]
                const int j = p - MLP_OW3;
                for (int t = 0; t < MLP_BS; ++t) acc += sdy[t] * sh2[t * MLP_H + j];
            } else {                                 // b3
                for (int t = 0; t < MLP_BS; ++t) acc += sdy[t];
            }
            g[q] += acc;
        }
        __syncthreads();
    }
    float *out = partial + (int64_t)blockIdx.x * (MLP_NPARAM + 1);
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int p = tid + MLP_BS * q;
        if (p < MLP_NPARAM) out[p] = g[q];
    }
    // block loss: reduce in shared memory (reuse sdy)
    __shared__ double red[MLP_BS];
    red[tid] = loss;
    __syncthreads();
    for (int w = MLP_BS / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) out[MLP_NPARAM] = (float)red[0];
}

inline size_t mlp_grad_smem() {
    return sizeof(float) * (MLP_NPARAM + MLP_BS * MLP_IN + 4 * MLP_BS * MLP_H + MLP_BS);
}

// grad[p] = sum over blocks (fixed order: deterministic); loss likewise (FP64)
__global__ void k_mlp_reduce(const float *partial, int nblocks, float *grad, double *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > MLP_NPARAM) return;
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += (double)partial[(int64_t)b * (MLP_NPARAM + 1) + p];
    if (p < MLP_NPARAM) grad[p] = (float)acc;
    else loss[0] = acc;
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void k_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float gg = g[p];
    const float mm = b1 * m[p] + (1.f - b1) * gg;
    const float vv = b2 * v[p] + (1.f - b2) * gg * gg;
    m[p] = mm;
    v[p] = vv;
    w[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
}

// minibatch of sample indices drawn with replacement by hashing (epoch, batch, i)
__global__ void k_batch_indices(int64_t *idx, int64_t bs, int64_t n, uint64_t key) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= bs) return;
    idx[i] = (int64_t)(mix64(key ^ mix64((uint64_t)i)) % (uint64_t)n);
}

}  // namespace dgh
