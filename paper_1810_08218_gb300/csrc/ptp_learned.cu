// Learned iteration schedule: a small MLP (6 -> 32 -> 32 -> 1, FP16 weights,
// FP32 accumulation) predicts, for every topleset window V_i, how many
// iterations the band's lower bound stays at i.  The window kernel then runs
// that many iterations without the relative-change test of Eq. lower_band,
// tests once, and falls back to tested iterations if V_i has not converged,
// so with predictions that do not exceed the plain method's counts the
// result is the plain method's.  The paper notes that the iterations needed
// grow as the toplesets diverge from the distance isocurves (Sec. 5.2); the
// features describe that per window.
//
// Window features (per topleset r, computed on the device):
//   0: log2(|V_r| + 1) / 20                       vertex count
//   1: mean ring-edge length over V_r / mesh mean  edge-length mean
//   2: std of those lengths / mesh mean            edge-length std
//   3: smallest triangle angle at V_r's vertices   minimum angle (radians)
//   4: std / mean of |x - x_s| over V_r, x_s the   front spread: how far the
//      first source                                topleset is from a sphere
//   5: r / rho                                     window position
//
// Parameters, one flat FP32 array (MLP_NPARAM): W1[32][6], b1[32],
// W2[32][32], b2[32], W3[32], b3.
#include <cuda_fp16.h>
#include <math.h>

#include "ptp_internal.cuh"

namespace {

constexpr int H = 32;
constexpr int NIN = 6;
constexpr int OW1 = 0, OB1 = OW1 + H * NIN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H;
constexpr int NPARAM = OB3 + 1;
static_assert(NPARAM == PTP_MLP_NPARAM, "parameter count");

unsigned blocks_for(int64_t work, int threads, int device) {
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)ptp_num_sms(device) * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

__device__ __forceinline__ int level_of(const int *__restrict__ off, int rho, int u) {
    int lo = 0, hi = rho;  // largest r with off[r] <= u
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Per-topleset sums: acc[r] = {count, sum e, sum e^2, sum rad, sum rad^2,
// min angle bits, pad, pad}; acc[n] holds the mesh's edge sum and count.
__global__ void window_sums(int n, const int *__restrict__ off, const int *__restrict__ info,
                            const float4 *__restrict__ pos, const int *__restrict__ meta,
                            const float4 *__restrict__ tgeom, const float4 *__restrict__ elen, float *__restrict__ acc) {
    const int rho = info[0];
    const int reached = info[1];
    const float4 xs = pos[0];  // V_0 comes first: a source
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < reached; u += gridDim.x * blockDim.x) {
        const int r = level_of(off, rho, u);
        const int m = __ldg(meta + u);
        const int cnt = (m & PTP_META_GENERAL) ? 0 : (m & PTP_META_CNT);
        const float4 l0 = __ldg(elen + u), l1 = __ldg(elen + n + u);
        const float el[PTP_RING] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
        float es = 0.0f, eq = 0.0f, amin = 3.14159265f;
#pragma unroll
        for (int t = 0; t < PTP_RING; ++t) {
            if (t < cnt) {
                es += el[t];
                eq += el[t] * el[t];
            }
        }
#pragma unroll
        for (int t = 0; t < PTP_TRI; ++t) {
            if (t < cnt - 1) {
                const float4 g = __ldg(tgeom + (size_t)t * n + u);
                const float den = el[t] * el[t + 1];
                if (den > 0.0f) amin = fminf(amin, acosf(fmaxf(-1.0f, fminf(1.0f, g.x / den))));
            }
        }
        const float4 p = pos[u];
        const float dx = p.x - xs.x, dy = p.y - xs.y, dz = p.z - xs.z;
        const float rad = sqrtf(dx * dx + dy * dy + dz * dz);
        float *a = acc + (size_t)r * 8;
        atomicAdd(a + 0, 1.0f);
        atomicAdd(a + 1, es);
        atomicAdd(a + 2, eq);
        atomicAdd(a + 3, rad);
        atomicAdd(a + 4, rad * rad);
        atomicMin((int *)(a + 5), __float_as_int(amin));
        atomicAdd(a + 6, (float)cnt);
        atomicAdd(acc + (size_t)n * 8 + 0, es);
        atomicAdd(acc + (size_t)n * 8 + 1, (float)cnt);
    }
}

__global__ void init_sums(int n, float *acc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 8 * (n + 1); i += gridDim.x * blockDim.x)
        acc[i] = (i % 8 == 5) ? 3.14159265f : 0.0f;
}

__global__ void window_finalize(int n, const int *__restrict__ info, const float *__restrict__ acc,
                                float *__restrict__ feat) {
    const int rho = info[0];
    const float emean = acc[(size_t)n * 8 + 0] / fmaxf(acc[(size_t)n * 8 + 1], 1.0f);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rho; r += gridDim.x * blockDim.x) {
        const float *a = acc + (size_t)r * 8;
        const float c = a[0], ne = fmaxf(a[6], 1.0f);
        const float em = a[1] / ne;
        const float ev = fmaxf(a[2] / ne - em * em, 0.0f);
        const float rm = a[3] / fmaxf(c, 1.0f);
        const float rv = fmaxf(a[4] / fmaxf(c, 1.0f) - rm * rm, 0.0f);
        float *f = feat + (size_t)r * NIN;
        f[0] = log2f(c + 1.0f) / 20.0f;
        f[1] = emean > 0.0f ? em / emean : 0.0f;
        f[2] = emean > 0.0f ? sqrtf(ev) / emean : 0.0f;
        f[3] = a[5];
        f[4] = rm > 0.0f ? sqrtf(rv) / rm : 0.0f;
        f[5] = (float)r / (float)(rho > 1 ? rho : 1);
    }
}

// Forward pass of one sample with FP16 weights from shared memory and FP32
// accumulation; keeps the hidden activations for the backward pass.
__device__ __forceinline__ float mlp_forward(const __half *w, const float x[NIN], float h1[H], float h2[H]) {
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
        float z = __half2float(w[OB1 + j]);
#pragma unroll
        for (int i = 0; i < NIN; ++i) z = fmaf(__half2float(w[OW1 + j * NIN + i]), x[i], z);
        h1[j] = fmaxf(z, 0.0f);
    }
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
        float z = __half2float(w[OB2 + j]);
#pragma unroll
        for (int i = 0; i < H; ++i) z = fmaf(__half2float(w[OW2 + j * H + i]), h1[i], z);
        h2[j] = fmaxf(z, 0.0f);
    }
    float y = __half2float(w[OB3]);
#pragma unroll
    for (int i = 0; i < H; ++i) y = fmaf(__half2float(w[OW3 + i]), h2[i], y);
    return y;
}

__global__ void __launch_bounds__(256) mlp_infer(const __half *__restrict__ wh, const float *__restrict__ feat,
                                                 const int *__restrict__ count_dev, int count, float margin, int cap,
                                                 int *__restrict__ sched) {
    __shared__ __half w[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = wh[i];
    __syncthreads();
    if (count_dev) count = *count_dev;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
        float x[NIN], h1[H], h2[H];
#pragma unroll
        for (int i = 0; i < NIN; ++i) x[i] = feat[(size_t)s * NIN + i];
        const float y = mlp_forward(w, x, h1, h2);
        const float nh = exp2f(fminf(y - margin, 24.0f));
        int v = nh >= 1.0f ? (int)nh : 1;
        sched[s] = v < cap ? v : cap;
    }
}

// Fused forward + backward over the samples: loss sum((y - t)^2) / count and
// its gradient accumulated in shared memory (FP32), then added to `grad`.
__global__ void __launch_bounds__(256) mlp_grad(const __half *__restrict__ wh, const float *__restrict__ X,
                                                const float *__restrict__ Y, int count, float *__restrict__ grad,
                                                float *__restrict__ loss) {
    __shared__ __half w[NPARAM];
    __shared__ float g[NPARAM];
    __shared__ float s_loss;
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
        w[i] = wh[i];
        g[i] = 0.0f;
    }
    if (threadIdx.x == 0) s_loss = 0.0f;
    __syncthreads();
    const float inv = 1.0f / (float)count;
    float my_loss = 0.0f;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < count; s += gridDim.x * blockDim.x) {
        float x[NIN], h1[H], h2[H];
#pragma unroll
        for (int i = 0; i < NIN; ++i) x[i] = X[(size_t)s * NIN + i];
        const float y = mlp_forward(w, x, h1, h2);
        const float err = y - Y[s];
        my_loss += err * err * inv;
        const float gy = 2.0f * err * inv;
        atomicAdd(&g[OB3], gy);
        float dz2[H];
#pragma unroll
        for (int j = 0; j < H; ++j) {
            atomicAdd(&g[OW3 + j], gy * h2[j]);
            dz2[j] = h2[j] > 0.0f ? gy * __half2float(w[OW3 + j]) : 0.0f;
        }
        float dh1[H];
#pragma unroll
        for (int i = 0; i < H; ++i) dh1[i] = 0.0f;
        for (int j = 0; j < H; ++j) {
            if (dz2[j] == 0.0f) continue;
            atomicAdd(&g[OB2 + j], dz2[j]);
#pragma unroll
            for (int i = 0; i < H; ++i) {
                atomicAdd(&g[OW2 + j * H + i], dz2[j] * h1[i]);
                dh1[i] = fmaf(__half2float(w[OW2 + j * H + i]), dz2[j], dh1[i]);
            }
        }
        for (int i = 0; i < H; ++i) {
            const float dz1 = h1[i] > 0.0f ? dh1[i] : 0.0f;
            if (dz1 == 0.0f) continue;
            atomicAdd(&g[OB1 + i], dz1);
#pragma unroll
            for (int k = 0; k < NIN; ++k) atomicAdd(&g[OW1 + i * NIN + k], dz1 * x[k]);
        }
    }
    atomicAdd(&s_loss, my_loss);
    __syncthreads();
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
        if (g[i] != 0.0f) atomicAdd(&grad[i], g[i]);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, s_loss);
}

// Adam on the FP32 master weights; refreshes the FP16 copy and clears grad.
__global__ void mlp_adam(float *__restrict__ wmaster, __half *__restrict__ wh, float *__restrict__ m,
                         float *__restrict__ v, float *__restrict__ grad, float lr, float b1t, float b2t) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = wmaster[i] - lr * (mi / (1.0f - b1t)) / (sqrtf(vi / (1.0f - b2t)) + eps);
        wmaster[i] = w;
        wh[i] = __float2half(w);
        grad[i] = 0.0f;
    }
}

__global__ void to_half(const float *__restrict__ w, __half *__restrict__ wh) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) wh[i] = __float2half(w[i]);
}

}  // namespace

extern "C" ptp_status ptp_window_features(ptp_toplesets_t *t, float *feat_out, void *stream) {
    if (!t || !feat_out) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)t->n;
    float *acc = nullptr;
    PTP_TRY(ptp_malloc_async((void **)&acc, sizeof(float) * 8 * ((size_t)n + 1), s));
    init_sums<<<blocks_for(8 * ((int64_t)n + 1), 256, t->device), 256, 0, s>>>(n, acc);
    window_sums<<<blocks_for(n, 256, t->device), 256, 0, s>>>(n, t->off, t->info, t->pos, t->meta, t->tgeom, t->elen,
                                                              acc);
    window_finalize<<<blocks_for(n, 256, t->device), 256, 0, s>>>(n, t->info, acc, feat_out);
    ptp_count_launches(3);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(acc, s);
    return e == cudaSuccess ? PTP_OK : ptp_internal_cuda_status(e);
}

extern "C" ptp_status ptp_mlp_infer(const uint16_t *w_half, const float *feat, int32_t count, const int32_t *count_dev,
                                    float margin, int32_t cap, int32_t *sched_out, void *stream) {
    if (!w_half || !feat || !sched_out || (count < 0 && !count_dev) || cap < 1) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    PTP_TRY(cudaGetDevice(&dev));
    const int work = count_dev ? ptp_num_sms(dev) * 256 : (count > 0 ? count : 1);
    mlp_infer<<<blocks_for(work, 256, dev), 256, 0, s>>>((const __half *)w_half, feat, count_dev, count, margin, cap,
                                                          sched_out);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

extern "C" ptp_status ptp_mlp_grad(const uint16_t *w_half, const float *X, const float *Y, int32_t count, float *grad,
                                   float *loss, void *stream) {
    if (!w_half || !X || !Y || count < 1 || !grad) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    PTP_TRY(cudaGetDevice(&dev));
    mlp_grad<<<blocks_for(count, 256, dev), 256, 0, s>>>((const __half *)w_half, X, Y, count, grad, loss);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

extern "C" ptp_status ptp_mlp_adam(float *w_master, uint16_t *w_half, float *m, float *v, float *grad, float lr,
                                   int32_t step, void *stream) {
    if (!w_master || !w_half || !m || !v || !grad || step < 1) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float b1t = powf(0.9f, (float)step), b2t = powf(0.999f, (float)step);
    mlp_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(w_master, (__half *)w_half, m, v, grad, lr, b1t, b2t);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

extern "C" ptp_status ptp_mlp_to_half(const float *w, uint16_t *w_half, void *stream) {
    if (!w || !w_half) return PTP_ERR_ARG;
    to_half<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, (__half *)w_half);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}
