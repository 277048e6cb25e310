// Device side of the window update shared by the single-map and batched
// window kernels: the update step of Sec. 3.2 on one triangle, the fan
// update of one vertex, work-skipping stamps and small reductions.  Every
// definition lives in an unnamed namespace, so each translation unit that
// includes this header gets its own copy.
#pragma once

#include <math.h>

#include "ptp_internal.cuh"

namespace {

constexpr int DIST_THREADS = 512;
constexpr int ROUND_CHUNKS = 8;                                 // chunks per warp per round
constexpr int P1_BATCH = 4;                                     // chunks whose state loads overlap
constexpr int QUEUE_CAP = ROUND_CHUNKS * DIST_THREADS;         // queue entries per CTA
#define INF __int_as_float(0x7f800000)

struct DistArgs {
    int n;
    const float4 *__restrict__ pos;
    const int4 *__restrict__ ring;
    const float4 *__restrict__ tgeom;
    const float4 *__restrict__ elen;
    const int *__restrict__ meta;
    const int *__restrict__ row;
    const int2 *__restrict__ pairs;
    const int *__restrict__ off;
    const int *__restrict__ info;
    float *d0;
    float *d1;
    int *nstamp;
    int *chg;
    ptp_ctrl *ctrl;
    ptp_trace_rec *trace;
    long long trace_cap;
    double eps;
    double eps_abs;
    long long max_iter;
    const int *perm;  // band position -> vertex, when the data stay in the original order
    int *lab0;        // Voronoi labels, double-buffered like d (optional)
    int *lab1;
    int band_mode;    // 0: Eq. lower_band; 1: fixed band, i_k = ceil(k / 2)
    const int *sched; // learned schedule per topleset, or NULL
    // BFS inside the launch (fused window): the last `producers` CTAs, and
    // in topleset order the `copiers` CTAs before them, which put each
    // topleset into place once the BFS has published it
    int producers;
    int copiers;
    int *level;       // [n] BFS level, -1 unvisited
    int *queue_w;     // the BFS queue (= perm), written by the producers
    int *off_w;       // topleset offsets, written by the producers
    int *info_w;      // [0] rho, [1] vertices reached
    // ... reading the mesh in its original numbering
    const float4 *opos;
    const int4 *oring;
    const int *ometa;
    const float4 *otgeom;
    const float4 *oelen;
    // ... and, when they also renumber, writing the topleset-ordered copies
    // that pos / ring / meta / tgeom / elen point to, plus the map
    // original -> position (then row / pairs are the original corner lists)
    float4 *pos_w;
    int4 *ring_w;
    int *meta_w;
    float4 *tgeom_w;
    float4 *elen_w;
    int *iperm;
    const int *gmap;  // renumbered fused launch: original vertex -> position for the corner lists (= iperm)
    int coherent;     // the renumbered arrays are written during the launch: load them through L2
    // learned multi-advance band (band_mode 2; sched above is then the due delays)
    int *sched_w;                  // fused: the schedule the launch infers, one entry per topleset
    unsigned long long *facc;      // fused: ring of per-topleset feature sums (ptp_schedule.cuh)
    const void *mlp_w;             // fused: FP16 MLP weights
    float mlp_margin;
    double feat_scale, feat_scale2;  // 2^30 / diameter and its square over the diameter
    int *conv_trace;               // optional [rho]: last iteration a topleset failed the test
};

__device__ __forceinline__ float fsqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// FP64 solve of the planar update for vertex x0 of triangle (x0, x1, x2),
// given e1 = x1 - x0, e2 = x2 - x0 (FP32 differences of nearby coordinates,
// exact or nearly so) and finite d1, d2.
__device__ __noinline__ float tri_solve_fp64(float3 e1f, float3 e2f, float d1f, float d2f, float fb) {
    const double e1x = e1f.x, e1y = e1f.y, e1z = e1f.z;
    const double e2x = e2f.x, e2y = e2f.y, e2z = e2f.z;
    const double a = e1x * e1x + e1y * e1y + e1z * e1z;
    const double c = e2x * e2x + e2y * e2y + e2z * e2z;
    const double b = e1x * e2x + e1y * e2y + e1z * e2z;
    const double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
    const double det = cx * cx + cy * cy + cz * cz;
    if (!(det > 1e-12 * a * c)) return fb;
    const double fx = e2x - e1x, fy = e2y - e1y, fz = e2z - e1z;  // x2 - x1
    const double A = fx * fx + fy * fy + fz * fz;
    const double d1 = d1f, delta = (double)d2f - d1;
    const double L = sqrt(A), ad = fabs(delta);
    if (!(ad < L)) return fb;
    const double disc = (L - ad) * (L + ad);
    const double amb = -(e1x * fx + e1y * fy + e1z * fz);  // a - b
    const double cmb = e2x * fx + e2y * fy + e2z * fz;     // c - b
    const double q = (delta * amb + sqrt(det * disc)) / A;
    if (cmb * q + b * delta > 0.0 && amb * q - a * delta > 0.0) {
        const float p = (float)(d1 + q);
        return p < fb ? p : fb;
    }
    return fb;
}

// Update step (Sec. 3.2) for vertex x0 from triangle (x0, x1, x2), with
// e1 = x1 - x0, e2 = x2 - x0, a1 = |e1|^2, l1 = |e1|, likewise a2, l2.
// Returns the candidate distance: the planar solution when it exists and
// satisfies the monotonicity condition Q X^T n < 0, else
// min(d1 + l1, d2 + l2).
__device__ __forceinline__ float tri_update(float3 e1, float3 e2, float d1, float d2, float a1, float l1, float a2,
                                            float l2, unsigned &nfp64) {
    const float fb = fminf(d1 + l1, d2 + l2);
    if (!(fmaxf(d1, d2) < INF)) return fb;  // at most one finite neighbour: edge only
    const float3 e12 = sub3(e2, e1);
    const float b = dot3(e1, e2);
    const float3 cr = cross3(e1, e2);
    const float det = dot3(cr, cr);
    const float A = dot3(e12, e12);
    const float big = fmaxf(a1 * a2, A * fmaxf(a1, a2));
    const float delta = d2 - d1;
    const float ad = fabsf(delta);
    const float L = fsqrt(A);
    if (det < 1e-6f * big) {
        ++nfp64;
        return tri_solve_fp64(e1, e2, d1, d2, fb);
    }
    if (!(ad < L)) return fb;
    const float disc = (L - ad) * (L + ad);
    // The planar solution is causal only if
    //   disc > A det / (max((a-b)^2, (c-b)^2) + det),
    // and since (a-b)^2, (c-b)^2 <= big, a triangle that passed the test
    // above (det >= 1e-6 big) needs disc > ~1e-6 A.  A computed disc below
    // 2^-22 A (where its own rounding error becomes large) is therefore
    // certainly non-causal: the edge fallback is exact here, no FP64 needed.
    if (disc < 0x1p-22f * A) return fb;
    const float amb = -dot3(e1, e12);  // a - b
    const float cmb = dot3(e2, e12);   // c - b
    const float q = __fdividef(fmaf(delta, amb, fsqrt(det * disc)), A);
    const bool causal = (fmaf(cmb, q, b * delta) > 0.0f) && (fmaf(amb, q, -a1 * delta) > 0.0f);
    return causal ? fminf(d1 + q, fb) : fb;
}

__device__ __forceinline__ float3 xyz(float4 p) { return make_float3(p.x, p.y, p.z); }

// Update step (Sec. 3.2) for vertex u from ring triangle (u, x1, x2) with
// the triangle's precomputed geometry g = (b, L, alpha, beta) and edge
// lengths l1 = |x1 - x_u|, l2 = |x2 - x_u|: q = delta * alpha + beta *
// sqrt(disc) is the planar solution shifted by d1, kept when both
// monotonicity conditions hold, else min(d1 + l1, d2 + l2).
__device__ __forceinline__ float tri_update_geom(float4 g, float d1, float d2, float l1, float l2) {
    const float fb = fminf(d1 + l1, d2 + l2);
    if (!(fmaxf(d1, d2) < INF)) return fb;  // at most one finite neighbour: edge only
    const float delta = d2 - d1;
    const float ad = fabsf(delta);
    const float L = g.y;
    if (!(ad < L)) return fb;
    const float disc = (L - ad) * (L + ad);
    if (disc < 0x1p-22f * (L * L)) return fb;  // provably non-causal, see tri_update
    const float q = fmaf(delta, g.z, g.w * fsqrt(disc));
    const float b = g.x, a1 = l1 * l1, c = l2 * l2;
    const bool causal = (fmaf(c - b, q, b * delta) > 0.0f) && (fmaf(a1 - b, q, -a1 * delta) > 0.0f);
    return causal ? fminf(d1 + q, fb) : fb;
}

// Near-degenerate ring triangle: solve from the positions in FP64.
__device__ __noinline__ float tri_update_degenerate(const DistArgs &a, int u, int id1, int id2, float d1, float d2,
                                                    float l1, float l2) {
    const float fb = fminf(d1 + l1, d2 + l2);
    if (!(fmaxf(d1, d2) < INF)) return fb;
    auto ld = [&](int x) { return xyz(a.coherent ? __ldcg(a.pos + x) : __ldg(a.pos + x)); };
    const float3 x0 = ld(u);
    return tri_solve_fp64(sub3(ld(id1), x0), sub3(ld(id2), x0), d1, d2, fb);
}

// New value of a ring-slot vertex: min of the old value and the update over
// its fan.  The geometry was loaded with the ring (one round trip); here
// only the neighbours' distances are gathered (the second).  Triangles whose
// two neighbours are both no closer than the current best are skipped: the
// update never returns less than min(d1, d2).  With LABELS the new value
// carries the label of the winning triangle's closer neighbour (Voronoi
// regions, Sec. 5.3).
template <bool LABELS>
__device__ __forceinline__ float update_ring(const DistArgs &a, int u, const int ids[PTP_RING], const float el[PTP_RING],
                                             const float4 g[PTP_TRI], int m, float best, const float *__restrict__ dp,
                                             const int *__restrict__ lp, int &label, unsigned &nfp64) {
    float dn[PTP_RING];
#pragma unroll
    for (int t = 0; t < PTP_RING; ++t) dn[t] = t < m ? __ldcg(dp + ids[t]) : INF;
#pragma unroll
    for (int t = 0; t < PTP_TRI; ++t) {
        if (t < m - 1 && fminf(dn[t], dn[t + 1]) < best) {
            float c;
            if (g[t].w >= 0.0f) {
                c = tri_update_geom(g[t], dn[t], dn[t + 1], el[t], el[t + 1]);
            } else {
                ++nfp64;
                c = tri_update_degenerate(a, u, ids[t], ids[t + 1], dn[t], dn[t + 1], el[t], el[t + 1]);
            }
            if (c < best) {
                best = c;
                if (LABELS) label = __ldcg(lp + (dn[t] <= dn[t + 1] ? ids[t] : ids[t + 1]));
            }
        }
    }
    return best;
}

// New value of a GENERAL vertex from its corner list.
__device__ __noinline__ float update_general(const DistArgs &a, int u, float best, const float *__restrict__ dp,
                                             const int *__restrict__ lp, int *label, unsigned &nfp64) {
    // With a.gmap (fused, renumbered) the corner lists are the original ones:
    // vertex u is original vertex perm[u] and a corner's ids map through iperm.
    const bool fmap = a.gmap != nullptr;
    const int v = fmap ? __ldcg(a.perm + u) : u;
    const float3 x0 = xyz(fmap ? __ldg(a.opos + v) : __ldg(a.pos + u));
    const int cb = __ldg(a.row + v), ce = __ldg(a.row + v + 1);
    for (int c = cb; c < ce; ++c) {
        const int2 pr = __ldg(a.pairs + c);
        const int p1 = fmap ? __ldcg(a.gmap + pr.x) : pr.x, p2 = fmap ? __ldcg(a.gmap + pr.y) : pr.y;
        const float d1 = __ldcg(dp + p1), d2 = __ldcg(dp + p2);
        if (!(fminf(d1, d2) < best)) continue;
        const float3 x1 = xyz(fmap ? __ldg(a.opos + pr.x) : __ldg(a.pos + pr.x));
        const float3 x2 = xyz(fmap ? __ldg(a.opos + pr.y) : __ldg(a.pos + pr.y));
        const float3 e1 = sub3(x1, x0), e2 = sub3(x2, x0);
        const float a1 = dot3(e1, e1), a2 = dot3(e2, e2);
        const float cand = tri_update(e1, e2, d1, d2, a1, fsqrt(a1), a2, fsqrt(a2), nfp64);
        if (cand < best) {
            best = cand;
            if (label) *label = __ldcg(lp + (d1 <= d2 ? p1 : p2));
        }
    }
    return best;
}

__device__ __noinline__ void stamp_general(const DistArgs &a, int u, int k) {
    const bool fmap = a.gmap != nullptr;
    const int v = fmap ? __ldcg(a.perm + u) : u;
    const int cb = __ldg(a.row + v), ce = __ldg(a.row + v + 1);
    for (int c = cb; c < ce; ++c) {
        const int2 pr = __ldg(a.pairs + c);
        a.nstamp[fmap ? __ldcg(a.gmap + pr.x) : pr.x] = k;
        a.nstamp[fmap ? __ldcg(a.gmap + pr.y) : pr.y] = k;
    }
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

#ifndef PTP_DIST_MIN_BLOCKS
#define PTP_DIST_MIN_BLOCKS 1
#endif

// Threads per CTA of a window launch: 0 selects DIST_THREADS; otherwise a
// multiple of 32 in [64, DIST_THREADS] (the kernels index by blockDim and
// size their shared arrays for DIST_THREADS); -1 if invalid.
inline int window_block(int32_t requested) {
    if (requested == 0) return DIST_THREADS;
    if (requested < 64 || requested > DIST_THREADS || requested % 32 != 0) return -1;
    return requested;
}

// Band bounds of one iteration.
struct Band {
    int copy_lo;  // start of the topleset retired after the previous iteration
    int lo;       // off[i]
    int vi_end;   // off[i + 1]
    int vj_beg;   // off[j]
    int hi;       // off[j + 1]
};

}  // namespace
