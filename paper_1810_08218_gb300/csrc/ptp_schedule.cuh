// Device side of the learned window schedule, shared by the fused launch's
// copy CTAs (features summed while they copy each topleset into place, the
// MLP run right after) and by ptp_window_features / ptp_mlp_infer (the same
// features and the same forward pass for a toplesets handle), so that both
// paths infer bit-identical schedules.
//
// Window features of topleset V_r (six inputs of the 6 -> 32 -> 32 -> 1 MLP):
//   0: log2(|V_r| + 1) / 20                          vertex count
//   1: min(|V_r| / |V_{r-1}|, 4) / 4                  growth of the front
//   2: std / mean of the ring-edge lengths over V_r   edge-length spread
//   3: smallest triangle angle at V_r's vertices      minimum angle (radians)
//   4: std / mean of |x - x_s| over V_r, x_s the      front spread: how far the
//      first source                                   topleset is from a sphere
//   5: min(r / sqrt(n), 4) / 4                        window position
// All are scale-free and computable from V_r, |V_{r-1}| and n alone, so the
// fused launch can evaluate them while the BFS is still running.  The sums
// behind them are fixed-point integers (quantities in units of the mesh
// diameter times 2^30), so accumulating them with atomics in any order gives
// the same bits.
#pragma once

#include <cuda_fp16.h>
#include <math.h>

#include "ptp_internal.cuh"

namespace {

constexpr int MLP_H = 32;
constexpr int MLP_NIN = 6;
constexpr int MLP_OW1 = 0, MLP_OB1 = MLP_OW1 + MLP_H * MLP_NIN, MLP_OW2 = MLP_OB1 + MLP_H,
              MLP_OB2 = MLP_OW2 + MLP_H * MLP_H, MLP_OW3 = MLP_OB2 + MLP_H, MLP_OB3 = MLP_OW3 + MLP_H;
constexpr int MLP_NPARAM_ = MLP_OB3 + 1;
static_assert(MLP_NPARAM_ == PTP_MLP_NPARAM, "parameter count");

// The ring of per-topleset feature accumulators a fused launch keeps (a copy
// round takes at most this many toplesets).
constexpr int FEAT_RING = 64;
constexpr int FEAT_WORDS = 8;  // per topleset: se, se2, sr, sr2, edges, count, amin bits, pad
static_assert(FEAT_RING * FEAT_WORDS == PTP_FEAT_RING_WORDS, "feature ring size");

// Iteration from which topleset r, entering the band at iteration r, may
// join the tested group of the learned multi-advance band: its predicted
// delay after entry (at least one iteration).  In a fused launch the
// schedule of V_r is written before V_r is published to the window, so it
// is known by then.
__host__ __device__ __forceinline__ long long sched_due(int r, int sched) {
    return (long long)r + (sched > 1 ? sched : 1);
}

__device__ __forceinline__ long long fixq(double v, double scale) { return llrint(v * scale); }

// One vertex's contribution to its topleset's sums: ring-edge lengths and
// their squares, the distance to the first source and its square (fixed
// point, scales 2^30 / diameter and 2^30 / diameter^2), the ring-edge count
// and the largest cosine of an angle at the vertex between consecutive ring
// neighbours (the smallest angle is its arc cosine, taken once per topleset).
// el: the ring-edge lengths, gb: the dot products e_t . e_{t+1} of the ring
// triangles (the first component of the ring geometry).
struct FeatTerms {
    long long se, se2, sr, sr2;
    int edges;
    float cmax;  // largest cosine of an angle at the vertex (-1: none)
};

__device__ __forceinline__ FeatTerms feat_terms(int meta, const float el[PTP_RING], const float gb[PTP_TRI], float3 x,
                                                float3 xs, double scale, double scale2) {
    const int cnt = (meta & PTP_META_GENERAL) ? 0 : (meta & PTP_META_CNT);
    float es = 0.0f, eq = 0.0f, cmax = -1.0f;  // the smallest angle has the largest cosine
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
            const float den = el[t] * el[t + 1];
            if (den > 0.0f) cmax = fmaxf(cmax, fmaxf(-1.0f, fminf(1.0f, gb[t] / den)));
        }
    }
    const float dx = x.x - xs.x, dy = x.y - xs.y, dz = x.z - xs.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float rad = sqrtf(r2);
    FeatTerms f;
    f.se = fixq((double)es, scale);
    f.se2 = fixq((double)eq, scale2);
    f.sr = fixq((double)rad, scale);
    f.sr2 = fixq((double)r2, scale2);
    f.edges = cnt;
    f.cmax = cmax;
    return f;
}

// Adds a warp's terms into acc[0..FEAT_WORDS) (lanes with have = false add
// nothing); every lane of the warp must call it.
__device__ __forceinline__ void feat_warp_add(unsigned long long *acc, const FeatTerms &f, bool have) {
    long long se = have ? f.se : 0, se2 = have ? f.se2 : 0, sr = have ? f.sr : 0, sr2 = have ? f.sr2 : 0;
    int ed = have ? f.edges : 0, cnt = have ? 1 : 0;
    float cm = have ? f.cmax : -1.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_xor_sync(0xffffffffu, se, o);
        se2 += __shfl_xor_sync(0xffffffffu, se2, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        sr2 += __shfl_xor_sync(0xffffffffu, sr2, o);
        ed += __shfl_xor_sync(0xffffffffu, ed, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    }
    if ((threadIdx.x & 31) == 0 && cnt > 0) {
        atomicAdd(acc + 0, (unsigned long long)se);
        atomicAdd(acc + 1, (unsigned long long)se2);
        atomicAdd(acc + 2, (unsigned long long)sr);
        atomicAdd(acc + 3, (unsigned long long)sr2);
        atomicAdd(acc + 4, (unsigned long long)ed);
        atomicAdd(acc + 5, (unsigned long long)cnt);
        // 1 + cos lies in [0, 2], where floats order like their bit patterns
        // (a fresh slot, 0, reads as cos = -1)
        atomicMax(acc + 6, (unsigned long long)__float_as_uint(1.0f + cm));
    }
}

// The six MLP inputs of topleset r from its sums (acc as written by
// feat_warp_add), |V_r|, |V_{r-1}| and the vertex count n.
__device__ __forceinline__ void feat_finalize(const unsigned long long *acc, int count, int count_prev, int r,
                                              long long n, float x[MLP_NIN]) {
    const double se = (double)(long long)acc[0], se2 = (double)(long long)acc[1];
    const double sr = (double)(long long)acc[2], sr2 = (double)(long long)acc[3];
    const double ed = (double)acc[4], c = (double)acc[5];
    const float amin = acosf(fmaxf(-1.0f, fminf(1.0f, __uint_as_float((unsigned)acc[6]) - 1.0f)));
    double cv_e = 0.0, cv_r = 0.0;
    if (ed > 0.0 && se > 0.0) {
        // both sums are scaled by 2^30 / diameter (squares by its square), so
        // the ratio std / mean comes out scale-free after one factor 2^30
        const double m = se / ed, q = se2 / ed * 1073741824.0;
        cv_e = sqrt(fmax(q - m * m, 0.0)) / m;
    }
    if (c > 0.0 && sr > 0.0) {
        const double m = sr / c, q = sr2 / c * 1073741824.0;
        cv_r = sqrt(fmax(q - m * m, 0.0)) / m;
    }
    x[0] = log2f((float)count + 1.0f) / 20.0f;
    x[1] = fminf((float)count / (float)(count_prev > 0 ? count_prev : 1), 4.0f) / 4.0f;
    x[2] = (float)cv_e;
    x[3] = amin;
    x[4] = (float)cv_r;
    x[5] = fminf((float)((double)r / sqrt((double)n)), 4.0f) / 4.0f;
}

// Forward pass of one sample, FP16 weights, FP32 accumulation in a fixed
// order; keeps the hidden activations (for the backward pass).
__device__ __forceinline__ float mlp_forward(const __half *w, const float x[MLP_NIN], float h1[MLP_H],
                                             float h2[MLP_H]) {
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        float z = __half2float(w[MLP_OB1 + j]);
#pragma unroll
        for (int i = 0; i < MLP_NIN; ++i) z = fmaf(__half2float(w[MLP_OW1 + j * MLP_NIN + i]), x[i], z);
        h1[j] = fmaxf(z, 0.0f);
    }
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        float z = __half2float(w[MLP_OB2 + j]);
#pragma unroll
        for (int i = 0; i < MLP_H; ++i) z = fmaf(__half2float(w[MLP_OW2 + j * MLP_H + i]), h1[i], z);
        h2[j] = fmaxf(z, 0.0f);
    }
    float y = __half2float(w[MLP_OB3]);
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) y = fmaf(__half2float(w[MLP_OW3 + i]), h2[i], y);
    return y;
}

// The same forward pass as mlp_forward for one sample, spread over a warp
// (lane j computes hidden unit j of both layers in the same order; the output
// sums the units in order, as mlp_forward does), with no per-thread arrays.
// Every lane returns y.  x must be the same on every lane.
__device__ __forceinline__ float mlp_forward_warp(const __half *w, const float x[MLP_NIN]) {
    const int j = threadIdx.x & 31;
    float z = __half2float(w[MLP_OB1 + j]);
#pragma unroll
    for (int i = 0; i < MLP_NIN; ++i) z = fmaf(__half2float(w[MLP_OW1 + j * MLP_NIN + i]), x[i], z);
    const float h1 = fmaxf(z, 0.0f);
    z = __half2float(w[MLP_OB2 + j]);
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) z = fmaf(__half2float(w[MLP_OW2 + j * MLP_H + i]), __shfl_sync(0xffffffffu, h1, i), z);
    const float h2 = fmaxf(z, 0.0f);
    float y = __half2float(w[MLP_OB3]);
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) y = fmaf(__half2float(w[MLP_OW3 + i]), __shfl_sync(0xffffffffu, h2, i), y);
    return y;
}

// Schedule entry from the MLP output y (a log2 iteration count).
__device__ __forceinline__ int sched_from_y(float y, float margin, int cap) {
    const float nh = exp2f(fminf(y - margin, 24.0f));
    const int v = nh >= 1.0f ? (int)nh : 1;
    return v < cap ? v : cap;
}

}  // namespace
