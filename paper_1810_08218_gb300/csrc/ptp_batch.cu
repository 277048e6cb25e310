// Batched PTP: up to 32 independent maps (different meshes and sources) in
// one persistent cooperative launch.  Every map keeps its own window
// (i_k, j_k of Eq. lower_band / upper_band, Sec. 4.2) and its own iteration
// count K_b; the maps advance in lockstep under one grid barrier per
// iteration, so the barrier and the dependent-load latency of an iteration
// are paid once for the whole batch, while each map's iterates are exactly
// the ones it has when run alone.  A map whose window has passed its last
// topleset drops out of the band enumeration; the launch ends when every
// map has.
//
// The maps' renumbered layouts are concatenated into one vertex range (map
// b occupies [base_b, base_b + n_b), its neighbour and corner ids offset by
// base_b), so the update step and its stored geometry are the single-map
// ones and a map's vertices only ever read and stamp vertices of the same
// map.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ptp_update.cuh"

namespace {

constexpr int MAXB = PTP_BATCH_MAX;  // maps per batch: one lane of warp 0 each
constexpr int MAPINFO = 8;   // ints per map in the map table
constexpr int NBITS = 26;    // band positions below 2^26 (queue encoding)

}  // namespace

// Device arrays of a batch: the maps' renumbered layouts concatenated into
// one vertex range, every vertex and corner id offset by its map's base.
struct ptp_batch_layout {
    float4 *pos;    // [N]
    int4 *ring;     // [2 N]
    int *meta;      // [N]
    float4 *tgeom;  // [PTP_TRI N]
    float4 *elen;   // [2 N]
    int *row;       // [N + 1] corner lists of GENERAL vertices
    int2 *pairs;    // [C]
    int *off;       // map b's topleset offsets at [offstart_b, offstart_b + rho_b], + base_b
    int *perm;      // [N] position -> original vertex index within its mesh
    int *mapinfo;   // [count][MAPINFO]: base, n, offstart, rho, number of source positions
};

struct ptp_batch_s {
    int device;
    cudaStream_t stream;
    int count;
    int64_t N;  // total vertices
    int64_t C;  // total corners
    ptp_batch_layout L;
    int64_t n[PTP_BATCH_MAX];  // vertices per map
};

namespace {

unsigned blocks_for(int64_t work, int threads, int device) {
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)ptp_num_sms(device) * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Copy map b's renumbered layout into the batch at vertex base `base` and
// corner base `cbase`.
__global__ void batch_copy(int N, int nb, int base, int cbase, int ncorner, int offstart, int b,
                           const float4 *__restrict__ pos, const int4 *__restrict__ ring, const int *__restrict__ meta,
                           const float4 *__restrict__ tgeom, const float4 *__restrict__ elen,
                           const int *__restrict__ row, const int2 *__restrict__ pairs, const int *__restrict__ off,
                           const int *__restrict__ info, const int *__restrict__ perm, ptp_batch_layout L) {
    const int rho = info[0];
    auto sh = [base](int x) { return x >= 0 ? x + base : x; };  // -1 pads the ring slots
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nb; u += gridDim.x * blockDim.x) {
        L.pos[base + u] = pos[u];
        L.meta[base + u] = meta[u];
        L.perm[base + u] = perm[u];
        const int4 r0 = ring[u], r1 = ring[nb + u];
        L.ring[base + u] = make_int4(sh(r0.x), sh(r0.y), sh(r0.z), sh(r0.w));
        L.ring[N + base + u] = make_int4(sh(r1.x), sh(r1.y), sh(r1.z), sh(r1.w));
        for (int t = 0; t < PTP_TRI; ++t) L.tgeom[(size_t)t * N + base + u] = tgeom[(size_t)t * nb + u];
        L.elen[base + u] = elen[u];
        L.elen[N + base + u] = elen[nb + u];
        L.row[base + u] = row[u] + cbase;
        if (u == nb - 1) L.row[base + nb] = row[nb] + cbase;
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncorner; c += gridDim.x * blockDim.x) {
        const int2 pr = pairs[c];
        L.pairs[cbase + c] = make_int2(pr.x + base, pr.y + base);
    }
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r <= rho; r += gridDim.x * blockDim.x)
        L.off[offstart + r] = off[r] + base;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int *mi = L.mapinfo + b * MAPINFO;
        mi[0] = base;
        mi[1] = nb;
        mi[2] = offstart;
        mi[3] = rho;
        mi[4] = off[1];
    }
}

struct BatchArgs {
    DistArgs a;         // n = N and the concatenated arrays, scratch and control block (zeroed by the host)
    int count;
    const int *mapinfo;
    unsigned *fmask;    // [3] rotating per-iteration masks: bit b = some vertex of map b's V_i failed
    long long *kres;    // [count] K_b
    long long *bures;   // [count] band updates of map b
    int *sres;          // [count] status of map b
};

// Largest b with pre[b] <= c: the map owning chunk c (maps that enumerate no
// chunk have pre[b] == pre[b + 1] and are skipped).
__device__ __forceinline__ int owner_of(const int *pre, int count, int c) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The batched window kernel.  An iteration enumerates the union of the live
// maps' bands as one sequence of 32-position chunks (map b owns chunks
// [pre_b, pre_{b+1})), interleaved over the warps of all CTAs as in the
// single-map kernel; pass 1 queues the vertices to recompute, tagged with
// their map, and pass 2 recomputes them.  Lane b of warp 0 in every CTA holds
// map b's window state; all CTAs apply the same per-map decisions after the
// barrier, so the copies never diverge.
__global__ void __launch_bounds__(DIST_THREADS, 1) ptp_window_batch(BatchArgs ba) {
    const DistArgs &a = ba.a;
    const int count = ba.count;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gwarp = wid * gridDim.x + blockIdx.x;
    const int nwarps = (blockDim.x >> 5) * gridDim.x;
    unsigned tot_active = 0, tot_changed = 0, nfp64 = 0;
    unsigned long long prev_hi[2] = {0ull, 0ull};
    __shared__ int2 s_queue[QUEUE_CAP];  // (position | map << 26 | in V_i << 31, bits of d_{k-1})
    __shared__ int s_nq;
    __shared__ int s_pre[MAXB + 1];
    __shared__ int s_abase[MAXB], s_start[MAXB], s_lo[MAXB], s_hi[MAXB], s_vi_end[MAXB], s_vj_beg[MAXB];
    __shared__ int s_src_end[MAXB], s_entering[MAXB];
    __shared__ unsigned s_mask;
    __shared__ int s_alldone;

    // map `lane`'s window state (warp 0 only)
    int rho = 0, src_end = 0, os = 0, i = 0;
    bool done = true;
    long long maxit = 0, bu = 0;
    Band bd = {0, 0, 0, 0, 0};
    if (wid == 0 && lane < count) {
        const int *mi = ba.mapinfo + lane * MAPINFO;
        os = mi[2];
        rho = mi[3];
        src_end = mi[0] + mi[4];
        maxit = a.max_iter > 0 ? a.max_iter : 8LL * rho + 64;
        done = false;
        // iteration 1: i_0 = 0, j_1 = min(1, rho - 1)
        const int j1 = rho > 1 ? 1 : 0;
        bd.lo = __ldcg(a.off + os);
        bd.copy_lo = bd.lo;
        bd.vi_end = __ldcg(a.off + os + 1);
        bd.vj_beg = __ldcg(a.off + os + j1);
        bd.hi = __ldcg(a.off + os + j1 + 1);
    }
    auto off_at = [&](int r) { return __ldcg(a.off + os + (r < rho ? r : rho)); };

    long long k = 1;
    for (;; ++k) {
        // this iteration's ranges of the live maps and the chunk prefix sums
        if (wid == 0) {
            int chunks = 0;
            if (lane < count && !done) {
                const int j = k < rho ? (int)k : rho - 1;
                const int first = bd.lo > src_end ? bd.lo : src_end;
                const int start = bd.copy_lo < first ? bd.copy_lo : first;
                const int abase = start & ~31;
                chunks = bd.hi > abase ? (bd.hi - abase + 31) >> 5 : 0;
                s_abase[lane] = abase;
                s_start[lane] = start;
                s_lo[lane] = bd.lo;
                s_hi[lane] = bd.hi;
                s_vi_end[lane] = bd.vi_end;
                s_vj_beg[lane] = bd.vj_beg;
                s_src_end[lane] = src_end;
                s_entering[lane] = (long long)j == k;
            }
            int incl = chunks;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane < count) s_pre[lane + 1] = incl;
            if (lane == 0) {
                s_pre[0] = 0;
                s_mask = 0u;
            }
        }
        __syncthreads();
        const float *dp = (k & 1) ? a.d0 : a.d1;  // d_{k-1} lives in buffer (k-1) % 2
        float *dnx = (k & 1) ? a.d1 : a.d0;
        const int nchunks = s_pre[count];
        int n_active = 0, n_changed = 0;
        unsigned fail = 0u;
        const int rounds_m = nchunks > gwarp ? (nchunks - gwarp + nwarps - 1) / nwarps : 0;
        const int cta_m = (nchunks > (int)blockIdx.x) ? (nchunks - (int)blockIdx.x + nwarps - 1) / nwarps : 0;
        for (int m0 = 0; m0 < cta_m; m0 += ROUND_CHUNKS) {
            if (threadIdx.x == 0) s_nq = 0;
            __syncthreads();
            // pass 1, P1_BATCH chunks' state in flight at once
            for (int m = m0; m < m0 + ROUND_CHUNKS && m < rounds_m; m += P1_BATCH) {
                int pp[P1_BATCH], bb[P1_BATCH], ns[P1_BATCH], cg[P1_BATCH];
                float dold[P1_BATCH];
                bool ok[P1_BATCH], live[P1_BATCH];
#pragma unroll
                for (int q = 0; q < P1_BATCH; ++q) {
                    const int c = gwarp + (m + q) * nwarps;  // warp-uniform
                    const bool valid = m + q < rounds_m;
                    const int b = valid ? owner_of(s_pre, count, c) : 0;
                    bb[q] = b;
                    pp[q] = s_abase[b] + (c - s_pre[b]) * 32 + lane;
                    ok[q] = valid && pp[q] >= s_start[b] && pp[q] < s_hi[b] && pp[q] >= s_src_end[b];
                    live[q] = ok[q] && pp[q] >= s_lo[b];
                }
#pragma unroll
                for (int q = 0; q < P1_BATCH; ++q) {
                    dold[q] = ok[q] ? __ldcg(dp + pp[q]) : 0.0f;
                    ns[q] = live[q] ? __ldcg(a.nstamp + pp[q]) : -2;
                    cg[q] = live[q] ? __ldcg(a.chg + pp[q]) : -2;
                    if (ok[q] && !live[q]) dnx[pp[q]] = dold[q];  // retired after the previous iteration
                }
#pragma unroll
                for (int q = 0; q < P1_BATCH; ++q) {
                    const int b = bb[q];
                    const bool need = live[q] && ((s_entering[b] && pp[q] >= s_vj_beg[b]) || ns[q] >= k - 1);
                    if (live[q] && !need && cg[q] == k - 1) dnx[pp[q]] = dold[q];
                    const unsigned bal = __ballot_sync(0xffffffffu, need);
                    if (bal) {
                        int at = 0;
                        if (lane == 0) at = atomicAdd(&s_nq, __popc(bal));
                        at = __shfl_sync(0xffffffffu, at, 0);
                        if (need)
                            s_queue[at + __popc(bal & ((1u << lane) - 1u))] =
                                make_int2(pp[q] | (b << NBITS) | (pp[q] < s_vi_end[b] ? (int)0x80000000 : 0),
                                          __float_as_int(dold[q]));
                    }
                }
            }
            __syncthreads();
            // pass 2: recompute the queued vertices
            const int nq = s_nq;
            for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                const int2 ent = s_queue[q];
                const int u = ent.x & ((1 << NBITS) - 1);
                const int b = (ent.x >> NBITS) & 31;
                const bool in_vi = ent.x < 0;
                const float dold = __int_as_float(ent.y);
                // through L2 only, as in the single-map kernel
                const int meta = __ldcg(a.meta + u);
                const int4 r0 = __ldcg(a.ring + u), r1 = __ldcg(a.ring + a.n + u);
                const float4 l0 = __ldcg(a.elen + u), l1 = __ldcg(a.elen + a.n + u);
                const int mm = meta & PTP_META_CNT;
                float4 g[PTP_TRI];
#pragma unroll
                for (int t = 0; t < PTP_TRI; ++t)
                    g[t] = __ldcg(a.tgeom + (size_t)t * a.n + u);  // every slot is written: no wait on meta
                const int ids[PTP_RING] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                const float el[PTP_RING] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
                int label = 0;
                float dnew;
                if (meta & PTP_META_GENERAL) dnew = update_general(a, u, dold, dp, nullptr, nullptr, nfp64);
                else dnew = update_ring<false>(a, u, ids, el, g, mm, dold, dp, nullptr, label, nfp64);
                ++n_active;
                dnx[u] = dnew;
                if (dnew != dold) {
                    ++n_changed;
                    a.chg[u] = (int)k;
                    if (meta & PTP_META_GENERAL) {
                        stamp_general(a, u, (int)k);
                    } else {
#pragma unroll
                        for (int t = 0; t < PTP_RING; ++t)
                            if (t < mm) a.nstamp[ids[t]] = (int)k;
                    }
                    if (in_vi) {
                        // relative-change test of Eq. lower_band, in FP64
                        const double o = dold, delta = o - (double)dnew;
                        if (!(isfinite(o) && delta < __dadd_rn(__dmul_rn(a.eps, o), a.eps_abs))) fail |= 1u << b;
                    }
                }
            }
            // the next round refills the queue; after the last one the CTA
            // barrier below comes first
            if (m0 + ROUND_CHUNKS < cta_m) __syncthreads();
        }
        tot_active += n_active;
        tot_changed += n_changed;
        if (fail) atomicOr(&s_mask, fail);
        // the bounds the next iteration may need are static: fetch them now
        int o_i2 = 0, o_jn = 0, o_jn1 = 0;
        if (wid == 0 && lane < count && !done) {
            const int jn = k + 1 < rho ? (int)(k + 1) : rho - 1;
            o_i2 = off_at(i + 2);
            o_jn = off_at(jn);
            o_jn1 = off_at(jn + 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_mask) atomicOr(&ba.fmask[k % 3], s_mask);
            // slot (k + 1) % 3 was last read after barrier k - 2, before every
            // CTA arrived at barrier k - 1; it is next written after barrier k
            if (blockIdx.x == 0) ba.fmask[(k + 1) % 3] = 0u;
        }
        if (ptp_grid_sync(a.ctrl->bar, k, 0u, &a.ctrl->abort, &a.ctrl->status, prev_hi) < 0) break;
        if (threadIdx.x == 0) s_mask = *(volatile unsigned *)&ba.fmask[k % 3];
        __syncthreads();
        if (wid == 0) {
            bool fin = true;
            if (lane < count && !done) {
                // Eq. lower_band, or the fixed band whose lower bound is ceil(k / 2)
                const bool advance = a.band_mode == 1 ? (int)((k + 1) >> 1) > i : !((s_mask >> lane) & 1u);
                bu += s_hi[lane] - (s_lo[lane] > src_end ? s_lo[lane] : src_end);
                int st = -1;
                if (advance) {
                    ++i;
                    if (i > rho - 1) st = PTP_OK;
                    bd.copy_lo = i >= 2 ? bd.lo : bd.vi_end;
                    bd.lo = bd.vi_end;
                    bd.vi_end = o_i2;
                } else {
                    bd.copy_lo = bd.lo;
                }
                bd.vj_beg = o_jn;
                bd.hi = o_jn1;
                if (st < 0 && k >= maxit) st = PTP_ERR_NOT_CONVERGED;
                if (st >= 0) {
                    done = true;
                    if (blockIdx.x == 0) {
                        ba.kres[lane] = k;
                        ba.bures[lane] = bu;
                        ba.sres[lane] = st;
                    }
                }
                fin = done;
            }
            const bool all = __all_sync(0xffffffffu, fin);
            if (lane == 0) s_alldone = all ? 1 : 0;
        }
        __syncthreads();
        if (s_alldone) break;
    }

    __shared__ unsigned long long s_tot[3];
    if (threadIdx.x == 0) s_tot[0] = s_tot[1] = s_tot[2] = 0ull;
    __syncthreads();
    if (tot_active) atomicAdd(&s_tot[0], (unsigned long long)tot_active);
    if (tot_changed) atomicAdd(&s_tot[1], (unsigned long long)tot_changed);
    if (nfp64) atomicAdd(&s_tot[2], (unsigned long long)nfp64);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&a.ctrl->active, s_tot[0]);
        atomicAdd(&a.ctrl->changed, s_tot[1]);
        atomicAdd(&a.ctrl->fp64, s_tot[2]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->iterations = k;
}

// The map holding vertex u: largest b with base_b <= u.
__device__ __forceinline__ int map_of(const int *__restrict__ mapinfo, int count, int u) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(mapinfo + mid * MAPINFO) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void batch_init(int N, int count, const int *__restrict__ mapinfo, float *__restrict__ d0,
                           float *__restrict__ d1, int *__restrict__ nstamp, int *__restrict__ chg) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        const int *mi = mapinfo + map_of(mapinfo, count, u) * MAPINFO;
        const float v = u < __ldg(mi) + __ldg(mi + 4) ? 0.0f : INF;
        d0[u] = v;
        d1[u] = v;
        nstamp[u] = -2;
        chg[u] = -2;
    }
}

// outs[b][perm[u]] = d_{K_b}[u]; map b's final iterate lives in buffer K_b % 2.
__global__ void batch_scatter(int N, int count, const int *__restrict__ mapinfo, const int *__restrict__ perm,
                              const long long *__restrict__ kres, const float *__restrict__ d0,
                              const float *__restrict__ d1, float *const *__restrict__ outs) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        const int b = map_of(mapinfo, count, u);
        const float *d = (kres[b] & 1) ? d1 : d0;
        outs[b][perm[u]] = d[u];
    }
}

void free_layout(ptp_batch_layout &L, cudaStream_t s) {
    void *ptrs[] = {L.pos, L.ring, L.meta, L.tgeom, L.elen, L.row, L.pairs, L.off, L.perm, L.mapinfo};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, s);
    memset(&L, 0, sizeof(L));
}

}  // namespace

ptp_status ptp_internal_batch_shape(const ptp_batch_t *bt, int *device, int *count, int64_t *sizes) {
    if (!bt) return PTP_ERR_ARG;
    *device = bt->device;
    *count = bt->count;
    if (sizes)
        for (int b = 0; b < bt->count; ++b) sizes[b] = bt->n[b];
    return PTP_OK;
}

ptp_status ptp_internal_window_occupancy_batch(int block, int *per_sm) {
    *per_sm = 0;
    PTP_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, ptp_window_batch, block, 0));
    return PTP_OK;
}

extern "C" ptp_status ptp_batch_create(ptp_toplesets_t *const *tops, int32_t count, void *stream, ptp_batch_t **out) {
    if (!out) return PTP_ERR_ARG;
    *out = nullptr;
    if (!tops || count < 1 || count > MAXB) return PTP_ERR_ARG;
    for (int b = 0; b < count; ++b)
        if (!tops[b] || tops[b]->device != tops[0]->device) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t N = 0, C = 0, O = 0;
    for (int b = 0; b < count; ++b) {
        N += tops[b]->n;
        C += tops[b]->ncorner;
        O += tops[b]->n + 2;
    }
    if (N >= (1LL << NBITS) || C >= (1LL << 31) || O >= (1LL << 31)) return PTP_ERR_TOO_LARGE;
    ptp_batch_s *bt = new ptp_batch_s();
    memset(&bt->L, 0, sizeof(bt->L));
    bt->device = tops[0]->device;
    bt->stream = s;
    bt->count = count;
    bt->N = N;
    bt->C = C;
    ptp_batch_layout &L = bt->L;
    void **ptrs[] = {(void **)&L.pos,  (void **)&L.ring,  (void **)&L.meta, (void **)&L.tgeom, (void **)&L.elen,
                     (void **)&L.row,  (void **)&L.pairs, (void **)&L.off,  (void **)&L.perm,  (void **)&L.mapinfo};
    const size_t sizes[] = {sizeof(float4) * N,     sizeof(int4) * 2 * N,  sizeof(int) * N,
                            sizeof(float4) * PTP_TRI * N, sizeof(float4) * 2 * N, sizeof(int) * (N + 1),
                            sizeof(int2) * (C > 0 ? C : 1), sizeof(int) * O, sizeof(int) * N,
                            sizeof(int) * MAPINFO * count};
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 10 && e == cudaSuccess; ++q) e = ptp_malloc_async(ptrs[q], sizes[q], s);
    int64_t base = 0, cbase = 0, ostart = 0;
    for (int b = 0; b < count && e == cudaSuccess; ++b) {
        const ptp_toplesets_t *t = tops[b];
        bt->n[b] = t->n;
        const int64_t work = t->n > t->ncorner ? t->n : t->ncorner;
        batch_copy<<<blocks_for(work, 256, bt->device), 256, 0, s>>>(
            (int)N, (int)t->n, (int)base, (int)cbase, (int)t->ncorner, (int)ostart, b, t->pos, t->ring, t->meta,
            t->tgeom, t->elen, t->row, t->pairs, t->off, t->info, t->perm, L);
        ptp_count_launches(1);
        e = cudaGetLastError();
        base += t->n;
        cbase += t->ncorner;
        ostart += t->n + 2;
    }
    // wait for the copy, so the toplesets handles (possibly built on other
    // streams) may be destroyed as soon as this returns
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_layout(L, s);
        cudaStreamSynchronize(s);
        delete bt;
        return ptp_internal_cuda_status(e);
    }
    *out = bt;
    return PTP_OK;
}

extern "C" ptp_status ptp_batch_destroy(ptp_batch_t *bt) {
    if (!bt) return PTP_ERR_ARG;
    free_layout(bt->L, bt->stream);
    const cudaError_t e = cudaStreamSynchronize(bt->stream);
    delete bt;
    return e == cudaSuccess ? PTP_OK : ptp_internal_cuda_status(e);
}

extern "C" ptp_status ptp_distance_batch(ptp_batch_t *bt, const ptp_params *params, float *const *d_out, void *stream,
                                         ptp_stats *stats) {
    if (!bt || !params || !d_out) return PTP_ERR_ARG;
    for (int b = 0; b < bt->count; ++b)
        if (!d_out[b]) return PTP_ERR_ARG;
    if (!(params->eps >= 0.0) || !(params->eps_abs >= 0.0) || params->max_iter < 0) return PTP_ERR_ARG;
    if (params->band_mode != 0 && params->band_mode != 1) return PTP_ERR_ARG;
    const int block = window_block(params->block);
    if (block < 0) return PTP_ERR_ARG;
    if (params->trace || params->schedule) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = bt->N;
    const int count = bt->count;
    const int dev = bt->device;
    // scratch: d0, d1, nstamp, chg [N] | ctrl | fmask[3] | kres, bures [MAXB] | sres [MAXB] | outs [MAXB]
    const size_t ctrl_bytes = (sizeof(ptp_ctrl) + 255) & ~(size_t)255;
    const size_t tail_bytes = 64 + 16 * MAXB + 4 * MAXB + sizeof(float *) * MAXB;
    const size_t head_bytes = ((16 * (size_t)N) + 255) & ~(size_t)255;
    char *scr = nullptr;
    PTP_TRY(ptp_malloc_async((void **)&scr, head_bytes + ctrl_bytes + tail_bytes, s));
    float *d0 = (float *)scr;
    float *d1 = d0 + N;
    int *nstamp = (int *)(d1 + N);
    int *chg = nstamp + N;
    ptp_ctrl *ctrl = (ptp_ctrl *)(scr + head_bytes);
    char *tail = scr + head_bytes + ctrl_bytes;
    unsigned *fmask = (unsigned *)tail;
    long long *kres = (long long *)(tail + 64);
    long long *bures = kres + MAXB;
    int *sres = (int *)(bures + MAXB);
    float **outs = (float **)(sres + MAXB);
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(ptp_ctrl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tail, 0, 64 + 16 * MAXB + 4 * MAXB, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(outs, d_out, sizeof(float *) * count, cudaMemcpyHostToDevice, s);
    ptp_status st = PTP_OK;
    if (e == cudaSuccess) {
        batch_init<<<blocks_for(N, 256, dev), 256, 0, s>>>((int)N, count, bt->L.mapinfo, d0, d1, nstamp, chg);
        ptp_count_launches(1);
        e = cudaGetLastError();
    }
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ptp_window_batch, block, 0);
    if (e == cudaSuccess && per_sm < 1) st = PTP_ERR_CUDA;
    if (e == cudaSuccess && st == PTP_OK) {
        int grid = per_sm * ptp_num_sms(dev);
        if (params->grid > 0 && params->grid < grid) grid = params->grid;
        BatchArgs ba;
        memset(&ba, 0, sizeof(ba));
        ba.a.n = (int)N;
        ba.a.pos = bt->L.pos;
        ba.a.ring = bt->L.ring;
        ba.a.tgeom = bt->L.tgeom;
        ba.a.elen = bt->L.elen;
        ba.a.meta = bt->L.meta;
        ba.a.row = bt->L.row;
        ba.a.pairs = bt->L.pairs;
        ba.a.off = bt->L.off;
        ba.a.d0 = d0;
        ba.a.d1 = d1;
        ba.a.nstamp = nstamp;
        ba.a.chg = chg;
        ba.a.ctrl = ctrl;
        ba.a.eps = params->eps;
        ba.a.eps_abs = params->eps_abs;
        ba.a.max_iter = params->max_iter;
        ba.a.band_mode = params->band_mode;
        ba.count = count;
        ba.mapinfo = bt->L.mapinfo;
        ba.fmask = fmask;
        ba.kres = kres;
        ba.bures = bures;
        ba.sres = sres;
        void *args[] = {(void *)&ba};
        if (params->ev_begin) e = cudaEventRecord((cudaEvent_t)params->ev_begin, s);
        if (e == cudaSuccess) {
            e = cudaLaunchCooperativeKernel((const void *)ptp_window_batch, dim3(grid), dim3(block), args, 0, s);
            ptp_count_launches(1);
        }
        if (e == cudaSuccess && params->ev_end) e = cudaEventRecord((cudaEvent_t)params->ev_end, s);
        if (e == cudaSuccess) {
            batch_scatter<<<blocks_for(N, 256, dev), 256, 0, s>>>((int)N, count, bt->L.mapinfo, bt->L.perm, kres, d0,
                                                                  d1, outs);
            ptp_count_launches(1);
            e = cudaGetLastError();
        }
    }
    // per-map status (always) and statistics
    if (e == cudaSuccess && st == PTP_OK) {
        std::vector<long long> hk(count), hb(count);
        std::vector<int> hs(count), info((size_t)count * MAPINFO);
        ptp_ctrl hc;
        e = cudaMemcpyAsync(hk.data(), kres, 8 * count, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), bures, 8 * count, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), sres, 4 * count, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(info.data(), bt->L.mapinfo, 4 * MAPINFO * count, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctrl, sizeof(hc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) {
            for (int b = 0; b < count; ++b) {
                const int sb = hc.status == PTP_ERR_TIMEOUT ? (int)PTP_ERR_TIMEOUT : hs[b];
                if (sb == PTP_ERR_TIMEOUT || (sb != PTP_OK && st == PTP_OK)) st = (ptp_status)sb;
                if (!stats) continue;
                stats[b].iterations = hk[b];
                stats[b].band_updates = hb[b];
                stats[b].active_updates = (int64_t)hc.active;  // batch totals
                stats[b].changed = (int64_t)hc.changed;
                stats[b].fp64_solves = (int64_t)hc.fp64;
                stats[b].rho = info[(size_t)b * MAPINFO + 3];
                stats[b].status = sb;
                stats[b].checks = hk[b];
            }
        }
    }
    cudaFreeAsync(scr, s);
    if (e != cudaSuccess) return ptp_internal_cuda_status(e);
    return st;
}
