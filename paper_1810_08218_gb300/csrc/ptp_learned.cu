// Learned window schedule: a small MLP (6 -> 32 -> 32 -> 1, FP16 weights,
// FP32 accumulation) predicts, for every topleset window V_r, the log2 of the
// number of iterations after it enters the band (at iteration r) until it has
// converged.  The window kernel uses the prediction in the learned
// multi-advance band (band_mode 2): toplesets whose predicted time has come
// are tested as one group besides the bottom topleset of Eq. lower_band, and
// when both pass the band's lower bound moves past all of them at once.  The
// paper notes that the iterations needed grow as the toplesets diverge from
// the distance isocurves (Sec. 5.2); the features describe that per window
// (ptp_schedule.cuh).  In band_mode 0 a schedule only delays the first test
// of each bottom topleset.
//
// This file: the features of a toplesets handle, inference, and training
// (fused forward + backward, Adam).  Parameters, one flat FP32 array
// (PTP_MLP_NPARAM): W1[32][6], b1[32], W2[32][32], b2[32], W3[32], b3.
#include <cuda_fp16.h>
#include <math.h>

#include "ptp_internal.cuh"
#include "ptp_schedule.cuh"

namespace {

constexpr int H = MLP_H;
constexpr int NIN = MLP_NIN;
constexpr int OW1 = MLP_OW1, OB1 = MLP_OB1, OW2 = MLP_OW2, OB2 = MLP_OB2, OW3 = MLP_OW3, OB3 = MLP_OB3;
constexpr int NPARAM = MLP_NPARAM_;

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

// Per-topleset sums of the window features (ptp_schedule.cuh):
// acc[r * FEAT_WORDS ...], the same integers the fused launch accumulates
// while it copies each topleset.  A warp's positions are consecutive, so its
// lanes are grouped by topleset and each group adds its sums once.
__global__ void window_sums(int n, const int *__restrict__ off, const int *__restrict__ info,
                            const float4 *__restrict__ pos, const int *__restrict__ meta,
                            const float4 *__restrict__ tgeom, const float4 *__restrict__ elen, double scale,
                            double scale2, unsigned long long *__restrict__ acc) {
    const int rho = info[0];
    const int reached = info[1];
    const float4 s0 = pos[0];  // V_0 comes first: a source
    const float3 xs = make_float3(s0.x, s0.y, s0.z);
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < reached; base += stride) {
        const int u = base + lane;
        const bool ok = u < reached;
        int r = -1;
        FeatTerms f = {};
        if (ok) {
            r = level_of(off, rho, u);
            const float4 l0 = __ldg(elen + u), l1 = __ldg(elen + n + u);
            const float el[PTP_RING] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
            float gb[PTP_TRI];
#pragma unroll
            for (int t = 0; t < PTP_TRI; ++t) gb[t] = __ldg(tgeom + (size_t)t * n + u).x;
            const float4 p = __ldg(pos + u);
            f = feat_terms(__ldg(meta + u), el, gb, make_float3(p.x, p.y, p.z), xs, scale, scale2);
        }
        bool todo = ok;
        while (__any_sync(0xffffffffu, todo)) {  // warp-uniform
            const int lead = __ffs(__ballot_sync(0xffffffffu, todo)) - 1;
            const int rl = __shfl_sync(0xffffffffu, r, lead);
            const bool mine = todo && r == rl;
            feat_warp_add(acc + (size_t)rl * FEAT_WORDS, f, mine);
            todo = todo && !mine;
        }
    }
}

__global__ void window_finalize(int n, const int *__restrict__ off, const int *__restrict__ info,
                                const unsigned long long *__restrict__ acc, float *__restrict__ feat) {
    const int rho = info[0];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rho; r += gridDim.x * blockDim.x) {
        const int count = off[r + 1] - off[r];
        const int prev = r > 0 ? off[r] - off[r - 1] : 1;
        float x[NIN];
        feat_finalize(acc + (size_t)r * FEAT_WORDS, count, prev, r, n, x);
#pragma unroll
        for (int q = 0; q < NIN; ++q) feat[(size_t)r * NIN + q] = x[q];
    }
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
        sched[s] = sched_from_y(mlp_forward(w, x, h1, h2), margin, cap);
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
    unsigned long long *acc = nullptr;
    const size_t bytes = sizeof(unsigned long long) * FEAT_WORDS * ((size_t)n + 1);
    PTP_TRY(ptp_malloc_async((void **)&acc, bytes, s));
    cudaError_t e = cudaMemsetAsync(acc, 0, bytes, s);
    if (e == cudaSuccess) {
        const double diam = t->mesh->diameter > 0.0 ? t->mesh->diameter : 1.0;
        window_sums<<<blocks_for(n, 256, t->device), 256, 0, s>>>(n, t->off, t->info, t->pos, t->meta, t->tgeom,
                                                                  t->elen, 1073741824.0 / diam,
                                                                  1073741824.0 / (diam * diam), acc);
        window_finalize<<<blocks_for(n, 256, t->device), 256, 0, s>>>(n, t->off, t->info, acc, feat_out);
        ptp_count_launches(2);
        e = cudaGetLastError();
    }
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
