// The PTP iteration (Sec. 4.2) over the sliding update band, as one
// persistent cooperative kernel with the window control on the device.
//
// Iteration k recomputes every non-source vertex of the band
// B = V_{i_{k-1}} u ... u V_{j_k} from d_{k-1} (Jacobi: two distance buffers,
// read d_{k-1}, write d_k), then a grid barrier, then every CTA applies
// Eq. lower_band from a per-iteration "some vertex of V_{i_{k-1}} failed the
// relative-change test" flag; j_k = min(k, rho - 1) is Eq. upper_band.
//
// Work skipping (exact): a vertex's new value depends only on its own and its
// neighbours' previous values, so when no neighbour changed in iteration k-1
// its recomputation would return d_{k-1}(u) unchanged.  Every vertex that
// changes stamps its neighbours with k (nstamp); only vertices stamped k-1,
// or entering the band, are recomputed.  Distances of skipped vertices that
// changed in k-1 are copied forward so both buffers stay Jacobi-consistent.
//
// The update step (Sec. 3.2) is evaluated in FP32 in a form shifted by d1
// (the unknown is q = p - d1, a local quantity of the order of an edge), with
// the discriminant written as det * (L - |d2-d1|) (L + |d2-d1|), L = |x2-x1|,
// so neither the magnitude of d nor the front's alignment with an edge
// cancels digits.  Near-degenerate triangles (some angle with squared sine
// below 1e-6) are solved in FP64; when the discriminant itself is too small
// for FP32 the triangle is provably non-causal (see tri_update).  The
// relative-change test of Eq. lower_band is evaluated in FP64.
#include <math.h>
#include <stdlib.h>

#include "ptp_internal.cuh"

#include "ptp_schedule.cuh"
#include "ptp_update.cuh"

namespace {

// BFS CTAs of the fused window launch: the toplesets (Sec. 4.1) level by
// level into the queue.  Level L's entries (positions off[L] .. off[L+1])
// are dealt out one per producer thread and round (warps interleaved across
// the producer CTAs).  Every queued vertex has a record at its position in
// the topleset-ordered meta and ring arrays (meta, and the one-ring slots
// as original vertex ids, -1 past the count), written when it was claimed,
// so a lane reads its entry's vertex, meta and slots in one coalesced round
// trip and claims every unvisited ring neighbour with atomicCAS (level -1
// -> L+1).  A warp stages its claims in shared memory; while one atomicAdd
// on the shared tail reserves their positions, its lanes load the claims'
// records from the original mesh, then write each claim's queue entry, iperm
// and record.  The producers' own barrier sums what each CTA appended, so
// after it one thread writes off[L+2] (the end of V_{L+1}) and publishes it
// with a release store of ctrl->ready = L + 2 (PTP_LEVELS_DONE once a level
// comes out empty), which the window CTAs acquire before they read those
// offsets, queue entries and records; they remap the slots through iperm
// when they copy the level.  Producers never wait for the window CTAs.
__device__ __noinline__ void bfs_producer(const DistArgs &a, int *stage_smem) {
    const int P = a.producers;
    const int n = a.n;
    const int pid = (int)blockIdx.x - ((int)gridDim.x - P);
    const int lane = threadIdx.x & 31;
    const int pwarp = (int)(threadIdx.x >> 5) * P + pid;  // warps interleaved across the producer CTAs
    const int nthr = (int)blockDim.x * P;
    const int ptid = pwarp * 32 + lane;
    int *const stage = stage_smem + (threadIdx.x >> 5) * (32 * PTP_RING);  // this warp's claims
    __shared__ int s_app[2];  // vertices this CTA appended in level L: s_app[L & 1]
    if (threadIdx.x == 0) s_app[0] = s_app[1] = 0;
    __syncthreads();
    unsigned long long prev_hi[2] = {0ull, 0ull};
    // queue entry, iperm and record of the vertex w claimed at position at
    auto put = [&](int w, int at, int wm, int4 w0, int4 w1) {
        const int vc = (wm & PTP_META_GENERAL) ? 0 : (wm & PTP_META_CNT);
        a.queue_w[at] = w;
        a.iperm[w] = at;
        a.meta_w[at] = wm;
        a.ring_w[at] = make_int4(vc > 0 ? w0.x : -1, vc > 1 ? w0.y : -1, vc > 2 ? w0.z : -1, vc > 3 ? w0.w : -1);
        a.ring_w[n + at] = make_int4(vc > 4 ? w1.x : -1, vc > 5 ? w1.y : -1, vc > 6 ? w1.z : -1, vc > 7 ? w1.w : -1);
    };
    int fbeg = 0;
    int total = __ldcg(a.off + 1);  // V_0: the (unique) sources, queued with their records
    for (int L = 0;; ++L) {
        int *const app = &s_app[L & 1];
        const int rounds = (total + nthr - 1) / nthr;
        for (int r = 0; r < rounds; ++r) {  // warp-uniform
            const int t = r * nthr + ptid;
            const bool ok = t < total;
            const int p = fbeg + t;
            const int u = ok ? __ldcg(a.queue_w + p) : -1;
            const int m = ok ? __ldcg(a.meta_w + p) : PTP_META_GENERAL;
            const int4 r0 = ok ? __ldcg(a.ring_w + p) : make_int4(-1, -1, -1, -1);
            const int4 r1 = ok ? __ldcg(a.ring_w + n + p) : make_int4(-1, -1, -1, -1);
            const int ids[PTP_RING] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            unsigned claimed = 0;
            if (u >= 0 && !(m & PTP_META_GENERAL)) {
                const int cnt = m & PTP_META_CNT;
                int old[PTP_RING];
#pragma unroll
                for (int q = 0; q < PTP_RING; ++q) old[q] = q < cnt ? atomicCAS(a.level + ids[q], -1, L + 1) : 0;
#pragma unroll
                for (int q = 0; q < PTP_RING; ++q)
                    if (q < cnt && old[q] == -1) claimed |= 1u << q;
            } else if (u >= 0) {
                // vertex without a ring slot: claim from its corner lists
                const int cb = __ldg(a.row + u), ce = __ldg(a.row + u + 1);
                for (int c = cb; c < ce; ++c) {
                    const int2 pr = __ldg(a.pairs + c);
                    const int ww[2] = {pr.x, pr.y};
                    for (int e = 0; e < 2; ++e)
                        if (atomicCAS(a.level + ww[e], -1, L + 1) == -1) {
                            const int at = atomicAdd(&a.ctrl->tail, 1);
                            put(ww[e], at, __ldg(a.ometa + ww[e]), __ldg(a.oring + ww[e]), __ldg(a.oring + n + ww[e]));
                            atomicAdd(app, 1);
                        }
                }
            }
            // the claimed ring neighbours: stage them, reserve their positions
            // and load their records at once, then write them
            const int cntc = __popc(claimed);
            int incl = cntc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int wtot = __shfl_sync(0xffffffffu, incl, 31);
            if (wtot) {
                int idx = incl - cntc;
#pragma unroll
                for (int q = 0; q < PTP_RING; ++q)
                    if (claimed >> q & 1u) stage[idx++] = ids[q];
                __syncwarp();
                int at = 0;
                if (lane == 31) {
                    at = atomicAdd(&a.ctrl->tail, wtot);
                    atomicAdd(app, wtot);
                }
                const int w0 = lane < wtot ? stage[lane] : -1;
                const int w1 = lane + 32 < wtot ? stage[lane + 32] : -1;
                const int4 none = make_int4(-1, -1, -1, -1);
                const int m0 = w0 >= 0 ? __ldg(a.ometa + w0) : 0, m1 = w1 >= 0 ? __ldg(a.ometa + w1) : 0;
                const int4 a0 = w0 >= 0 ? __ldg(a.oring + w0) : none, b0 = w0 >= 0 ? __ldg(a.oring + n + w0) : none;
                const int4 a1 = w1 >= 0 ? __ldg(a.oring + w1) : none, b1 = w1 >= 0 ? __ldg(a.oring + n + w1) : none;
                const int base = __shfl_sync(0xffffffffu, at, 31);
                if (w0 >= 0) put(w0, base + lane, m0, a0, b0);
                if (w1 >= 0) put(w1, base + lane + 32, m1, a1, b1);
                for (int e = lane + 64; e < wtot; e += 32) {
                    const int w = stage[e];
                    put(w, base + e, __ldg(a.ometa + w), __ldg(a.oring + w), __ldg(a.oring + n + w));
                }
                __syncwarp();  // the stage is reused in the next round
            }
        }
        __syncthreads();  // every append of this CTA is counted in *app
        const unsigned val = (unsigned)*app;
        if (threadIdx.x == 0) s_app[(L + 1) & 1] = 0;  // last read before the previous barrier
        const long long next = ptp_grid_sync(a.ctrl->pbar, L + 1, val, &a.ctrl->abort, &a.ctrl->status, prev_hi,
                                             (unsigned)P, PTP_WAIT_CYCLES, true);
        if (next < 0) return;
        const int end = fbeg + total + (int)next;
        if (pid == 0 && threadIdx.x == 0) {
            a.off_w[L + 2] = end;
            if (next == 0) {
                a.info_w[0] = L + 1;  // rho
                a.info_w[1] = end;    // vertices reached
                ptp_st_release_s32(&a.ctrl->ready, PTP_LEVELS_DONE);
            } else {
                ptp_st_release_s32(&a.ctrl->ready, L + 2);
            }
        }
        if (next == 0) return;
        fbeg += total;
        total = (int)next;
    }
}

// Band position p of a topleset-ordered fused launch into place: the
// producers' record there (meta, raw slots as original ids) gets its slots
// remapped through iperm and the vertex's geometry copied from the original
// mesh.  Every slot's vertex must have its position (iperm) by then.  With
// ft, also the vertex's window-feature terms (ptp_schedule.cuh) from the
// values just copied: the same inputs ptp_window_features reads from a
// toplesets handle, so the sums come out the same.
__device__ __forceinline__ void copy_position(const DistArgs &a, int p, FeatTerms *ft, float3 xs) {
    const int n = a.n;
    const int v = __ldcg(a.perm + p);
    const int4 s0 = __ldcg(a.ring_w + p), s1 = __ldcg(a.ring_w + n + p);
    float4 g[PTP_TRI];
#pragma unroll
    for (int q = 0; q < PTP_TRI; ++q) g[q] = __ldg(a.otgeom + (size_t)q * n + v);
    const float4 e0 = __ldg(a.oelen + v), e1 = __ldg(a.oelen + n + v), x = __ldg(a.opos + v);
    auto mp = [&](int id) { return id >= 0 ? __ldcg(a.iperm + id) : -1; };
    a.ring_w[p] = make_int4(mp(s0.x), mp(s0.y), mp(s0.z), mp(s0.w));
    a.ring_w[n + p] = make_int4(mp(s1.x), mp(s1.y), mp(s1.z), mp(s1.w));
    a.pos_w[p] = x;
#pragma unroll
    for (int q = 0; q < PTP_TRI; ++q) a.tgeom_w[(size_t)q * n + p] = g[q];
    a.elen_w[p] = e0;
    a.elen_w[n + p] = e1;
    if (ft) {
        const float el[PTP_RING] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
        float gb[PTP_TRI];
#pragma unroll
        for (int q = 0; q < PTP_TRI; ++q) gb[q] = g[q].x;
        *ft = feat_terms(__ldcg(a.meta + p), el, gb, make_float3(x.x, x.y, x.z), xs, a.feat_scale, a.feat_scale2);
    }
}

// Learned multi-advance band in a fused launch: the schedule of topleset r
// (one warp, in a copy CTA), from the feature sums its copy accumulated
// (ptp_schedule.cuh) and the MLP whose FP16 weights are in `w`; the sums'
// ring slot is cleared for reuse.  Toplesets at or past `lim` are skipped,
// and V_0 (the sources) needs no schedule.
__device__ __noinline__ void infer_one(const DistArgs &a, const __half *w, int r, int lim) {
    if (r >= lim) return;
    const int lane = threadIdx.x & 31;
    unsigned long long *acc = a.facc + (size_t)(r % FEAT_RING) * FEAT_WORDS;
    if (r >= 1) {
        const int om = __ldcg(a.off + r - 1), o0 = __ldcg(a.off + r), o1 = __ldcg(a.off + r + 1);
        unsigned long long v[FEAT_WORDS];
#pragma unroll
        for (int q = 0; q < FEAT_WORDS; ++q) v[q] = __ldcg(acc + q);
        float x[MLP_NIN];
        feat_finalize(v, o1 - o0, o0 - om, r, a.n, x);
        const float y = mlp_forward_warp(w, x);
        if (lane == 0) a.sched_w[r] = sched_from_y(y, a.mlp_margin, 1 << 20);
    }
    __syncwarp();
    // the slot serves topleset r + FEAT_RING next (V_0's sums are never used)
    if (lane < FEAT_WORDS) acc[lane] = 0ull;
}

// Copy CTAs of a topleset-ordered fused launch: the a.copiers CTAs before
// the producers put the toplesets into place as the BFS publishes them, so
// that the window CTAs spend no iteration time on it.  Topleset V_r can be
// copied once every vertex of its one-ring has a position, that is once
// V_{r+1} is complete (ctrl->ready >= r + 2).  A round copies V_done ..
// V_{upto-1}: every copy CTA waits (thread 0, acquire) until ctrl->ready
// >= upto + 1, the positions are dealt to the copy threads in 32-position
// chunks (warps interleaved across the copy CTAs, so a small topleset still
// spreads over all of them), the copy CTAs pass their own grid barrier and
// one thread publishes ctrl->copied = upto with a release store.  Every copy
// CTA must copy the same range (each position exactly once: a second copy
// would remap slots that are already positions), so the next range comes
// from the barrier: copy CTA 0 adds how far the latest ctrl->ready it saw
// is past upto + 1 (or a flag once the BFS has ended) and the others 0, and
// the sum, the same in every CTA, sets the next upto (every topleset
// copyable by then, at least one more).  When the BFS is ahead, a round
// takes many toplesets.  Once ctrl->ready is PTP_LEVELS_DONE the next
// round ends at rho, which every copy CTA reads after its own wait, and
// ctrl->copied becomes PTP_LEVELS_DONE.  The window CTAs acquire
// ctrl->copied before they read the copied toplesets and the offsets;
// ctrl->copied >= r + 1 implies ctrl->ready >= r + 2, so off[0 .. r+2] are
// published as well.  Copy CTAs never wait for the window CTAs.
//
// LEARN (the learned multi-advance band): the copy also sums each
// topleset's window features (one topleset at a time, so that a warp adds
// to one feature slot), a round takes at most FEAT_RING toplesets (their
// slots), and after the barrier one warp per topleset infers its schedule
// (infer_one); a second barrier precedes the publication, so ctrl->copied
// >= r + 1 also means that schedule[r] is written.
template <bool LEARN>
__device__ __noinline__ void level_copier(const DistArgs &a) {
    const int C = a.copiers;
    const int cid = (int)blockIdx.x - ((int)gridDim.x - a.producers - C);
    const int lane = threadIdx.x & 31;
    const int cwarp = (int)(threadIdx.x >> 5) * C + cid;  // warps interleaved across the copy CTAs
    const int ncw = (int)(blockDim.x >> 5) * C;
    constexpr int TO_RHO = 0x7fffffff;  // the round ends at rho (the BFS has ended)
    constexpr unsigned BFS_ENDED = 1u << 30;
    __shared__ int s_now[2];
    __shared__ __half s_w[LEARN ? MLP_NPARAM_ : 1];      // MLP weights
    __shared__ int s_off[LEARN ? FEAT_RING + 1 : 1];     // the round's offsets
    __shared__ float s_xs[3];                            // the first source's position
    float3 xs = make_float3(0.0f, 0.0f, 0.0f);
    if constexpr (LEARN) {
        const __half *wg = (const __half *)a.mlp_w;
        for (int q = threadIdx.x; q < MLP_NPARAM_; q += blockDim.x) s_w[q] = wg[q];
        if (threadIdx.x == 0) {
            const float4 x0 = __ldg(a.opos + __ldcg(a.perm));
            s_xs[0] = x0.x;
            s_xs[1] = x0.y;
            s_xs[2] = x0.z;
        }
        __syncthreads();
        xs = make_float3(s_xs[0], s_xs[1], s_xs[2]);
    }
    unsigned long long prev_hi[2] = {0ull, 0ull};
    long long e = 1;         // the copy CTAs' barrier epoch
    int done = 0, upto = 1;  // the first round copies V_0
    while (true) {
        if (threadIdx.x == 0) {
            int now = 0, ok = 1;
            const long long t0 = clock64();
            unsigned spins = 0;
            while (true) {
                now = ptp_ld_acquire_s32(&a.ctrl->ready);
                if (now >= (upto == TO_RHO ? PTP_LEVELS_DONE : upto + 1)) break;
                if ((++spins & 63u) == 0) {
                    if (*(volatile int *)&a.ctrl->abort) { ok = 0; break; }
                    if (clock64() - t0 > PTP_WAIT_CYCLES) {
                        atomicExch(&a.ctrl->status, (int)PTP_ERR_TIMEOUT);
                        atomicExch(&a.ctrl->abort, 1);
                        ok = 0;
                        break;
                    }
                }
            }
            s_now[0] = ok;
            s_now[1] = (ok && now == PTP_LEVELS_DONE) ? __ldcg(a.info) : TO_RHO;  // rho once known
        }
        __syncthreads();
        if (!s_now[0]) return;
        const int rho_seen = s_now[1];  // s_now is rewritten in the next round
        if (upto == TO_RHO) upto = rho_seen;  // every copy CTA has seen the BFS end
        if (LEARN && upto - done > FEAT_RING) upto = done + FEAT_RING;
        if constexpr (LEARN) {
            for (int q = threadIdx.x; q <= upto - done; q += blockDim.x) s_off[q] = __ldcg(a.off + done + q);
            __syncthreads();
            int cbase = 0;  // chunks of the round's earlier toplesets
            for (int r = done; r < upto; ++r) {
                const int pb = s_off[r - done], pe = s_off[r - done + 1];
                const int cb = pb & ~31;
                const int rch = pe > cb ? (pe - cb + 31) >> 5 : 0;
                unsigned long long *acc = a.facc + (size_t)(r % FEAT_RING) * FEAT_WORDS;
                int c0 = (cwarp - cbase) % ncw;
                if (c0 < 0) c0 += ncw;
                for (int c = c0; c < rch; c += ncw) {  // warp-uniform
                    const int p = cb + c * 32 + lane;
                    const bool have = p >= pb && p < pe;
                    FeatTerms ft = {};
                    if (have) copy_position(a, p, &ft, xs);
                    feat_warp_add(acc, ft, have);
                }
                cbase += rch;
            }
        } else {
            const int pb = __ldcg(a.off + done), pe = __ldcg(a.off + upto);
            const int cb = pb & ~31;
            const int rch = pe > cb ? (pe - cb + 31) >> 5 : 0;
            for (int c = cwarp; c < rch; c += ncw) {
                const int p = cb + c * 32 + lane;
                if (p >= pb && p < pe) copy_position(a, p, nullptr, xs);
            }
        }
        // the BFS's progress for the next range, from copy CTA 0 only: how
        // many toplesets past upto are copyable, or BFS_ENDED (the barrier
        // sums the values of all its epochs in 32 bits, so they stay small)
        unsigned seen = 0;
        if (cid == 0 && threadIdx.x == 0) {
            const int rd = ptp_ld_acquire_s32(&a.ctrl->ready);  // >= upto + 1, seen above
            seen = rd == PTP_LEVELS_DONE ? BFS_ENDED : (unsigned)min(rd - (upto + 1), 1 << 20);
        }
        const long long sum = ptp_grid_sync(a.ctrl->cbar, e++, seen, &a.ctrl->abort, &a.ctrl->status, prev_hi,
                                            (unsigned)C);
        if (sum < 0) return;
        if constexpr (LEARN) {
            // every feature sum of the round is complete: the schedules
            for (int r = done + cwarp; r < upto; r += ncw) infer_one(a, s_w, r, upto);  // warp-uniform
            if (ptp_grid_sync(a.ctrl->cbar, e++, 0u, &a.ctrl->abort, &a.ctrl->status, prev_hi, (unsigned)C) < 0)
                return;
        }
        const bool last = upto == rho_seen;  // V_{rho-1} is in place
        if (cid == 0 && threadIdx.x == 0) ptp_st_release_s32(&a.ctrl->copied, last ? PTP_LEVELS_DONE : upto);
        if (last) return;
        done = upto;
        upto = sum >= BFS_ENDED ? TO_RHO : done + (sum > 0 ? (int)sum : 1);
    }
}

// Topleset of band position p (two-step path, convergence traces only).
__device__ __forceinline__ int topleset_of(const int *__restrict__ off, int rho, int p) {
    int lo = 0, hi = rho;  // largest r with off[r] <= p
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldcg(off + mid) <= p) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The persistent window kernel.  Each iteration walks the band in chunks of
// 32 consecutive band positions (coalesced), chunk c to warp c mod W with
// the warps numbered across CTAs first, so even a narrow band spreads over
// all SMs.  Pass 1 reads each vertex's own distance and change stamps and
// queues, in shared memory, the vertices some neighbour of which changed in
// the previous iteration; pass 2 recomputes the queued vertices with every
// lane busy.  Long bands are handled in rounds that fit the queue.  The next
// iteration's band bounds are fetched before the barrier, so after it only
// distances written in this iteration are on the critical path.
//
// PERM: the vertex data stay in the original order and band position p holds
// vertex perm[p] (multi-source maps, where the paper also skips the
// rearrangement, Sec. 5.1); otherwise position p is vertex p of the
// renumbered mesh.  LABELS: also carry a label per vertex (Voronoi regions).
//
// FUSED (ptp_distance_from_sources): the toplesets are built inside this
// launch.  The last a.producers CTAs run the BFS (bfs_producer).  In
// topleset order the a.copiers CTAs before them put each topleset into
// place (level_copier): the producers write each vertex's meta and raw
// slots at its position when they claim it, the copiers remap the slots
// through iperm and copy the geometry from the original mesh.  The other
// CTAs run the iteration.  Before iteration k a window CTA waits until
// V_0 .. V_k are copied (ctrl->copied >= k + 1, which implies that off[0 ..
// k+2] are published); in the original order, until off[0 .. k+3] are
// published (ctrl->ready >= k + 3).  rho is unknown until the BFS ends;
// until then V_{k+1} is known to be non-empty, so rho > k + 1 and j_k = k,
// the same decision the known rho would give.
template <bool PERM, bool LABELS, bool FUSED = false, bool MULTI = false>
__global__ void __launch_bounds__(DIST_THREADS, PTP_DIST_MIN_BLOCKS) ptp_window(DistArgs a) {
    static_assert(!(MULTI && PERM), "the learned multi-advance band runs in topleset order");
    static_assert(!(FUSED && LABELS && !PERM), "labels are carried in the original order");
    __shared__ int2 s_queue[QUEUE_CAP];  // (vertex | in V_i << 31, bits of d_{k-1})
    if constexpr (FUSED) {
        // the producers stage their claims in the window's queue, 256 ints a warp
        static_assert(2 * QUEUE_CAP >= (DIST_THREADS / 32) * 32 * PTP_RING, "producer stage");
        if ((int)blockIdx.x >= (int)gridDim.x - a.producers) {
            bfs_producer(a, reinterpret_cast<int *>(s_queue));
            return;
        }
        if constexpr (!PERM) {
            if ((int)blockIdx.x >= (int)gridDim.x - a.producers - a.copiers) {
                level_copier<MULTI>(a);
                return;
            }
        }
    }
    constexpr int RHO_UNKNOWN = 0x3fffffff;
    const int ncta = FUSED ? (int)gridDim.x - a.producers - (PERM ? 0 : a.copiers) : (int)gridDim.x;  // window CTAs
    int rho = FUSED ? RHO_UNKNOWN : __ldcg(a.info);
    const int nsrc = __ldcg(a.off + 1);
    long long max_iter = a.max_iter > 0 ? a.max_iter : (FUSED ? (1LL << 40) : 8LL * rho + 64);
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gwarp = wid * ncta + blockIdx.x;
    const int nwarps = (blockDim.x >> 5) * ncta;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned tot_active = 0, tot_changed = 0, nfp64 = 0;
    unsigned long long prev_hi[2] = {0ull, 0ull};
    long long band_updates = 0;
    int i = 0;  // i_{k-1}
    long long k = 1;
    long long check_from = 1;  // first iteration that tests V_i (learned schedule)
    long long checks = 0;
    int status = PTP_ERR_NOT_CONVERGED;
    __shared__ float s_max[DIST_THREADS / 32];
    __shared__ double s_sum[DIST_THREADS / 32];
    __shared__ int s_cnt[2][DIST_THREADS / 32];
    __shared__ int s_nq;

    auto off_at = [&](int r) { return __ldcg(a.off + (r < rho ? r : rho)); };
    // the queue is written during a fused launch: read it through L2 there
    auto vertex_at = [&](int pos) { return PERM ? (FUSED ? __ldcg(a.perm + pos) : __ldg(a.perm + pos)) : pos; };
    // FUSED: wait until the progress word (ctrl->copied in topleset order,
    // ctrl->ready in the original order) reaches `need` (or the BFS has
    // ended); afterwards rho is set if known.  Called by every thread of the
    // CTA.
    // Returns false when a wait timed out or another CTA aborted.
    // Every thread keeps the progress its CTA has seen (`seen`, updated by
    // all threads from the same shared value after the barrier below, so it
    // is uniform), and when the BFS is already far enough ahead (the common
    // case) the CTA passes no barrier here; the word is polled, by thread 0,
    // only when it is not.  rho becomes known at the first poll after the
    // BFS has ended, in every CTA before it needs it (need > rho by then).
    // Consecutive calls are separated by a CTA barrier (the grid barrier),
    // which keeps s_wait from being rewritten before every thread read it.
    __shared__ int s_wait[3];
    int *const progress = PERM ? &a.ctrl->ready : &a.ctrl->copied;
    int seen = PERM ? 1 : 0;  // off[0], off[1] are set before launch
    auto wait_levels = [&](int need) -> bool {
        if (seen >= need) return true;
        if (threadIdx.x == 0) {
            int ok = 1;
            int now = seen;
            const long long t0 = clock64();
            unsigned spins = 0;
            while (true) {
                now = ptp_ld_acquire_s32(progress);
                if (now >= need) break;
                if ((++spins & 63u) == 0) {
                    if (*(volatile int *)&a.ctrl->abort) { ok = 0; break; }
                    if (clock64() - t0 > PTP_WAIT_CYCLES) {
                        atomicExch(&a.ctrl->status, (int)PTP_ERR_TIMEOUT);
                        atomicExch(&a.ctrl->abort, 1);
                        ok = 0;
                        break;
                    }
                }
            }
            s_wait[0] = ok;
            s_wait[1] = (ok && now == PTP_LEVELS_DONE) ? __ldcg(a.info) : RHO_UNKNOWN;
            s_wait[2] = now;
        }
        __syncthreads();
        const bool ok = s_wait[0] != 0;
        seen = s_wait[2];
        if (s_wait[1] != RHO_UNKNOWN && rho == RHO_UNKNOWN) {
            rho = s_wait[1];
            if (a.max_iter <= 0) max_iter = 8LL * rho + 64;
        }
        return ok;
    };
    // what iteration k needs: V_0 .. V_k in place (topleset order), or the
    // offsets off[0 .. k+3] (original order)
    auto need_for = [](long long kk) { return (int)kk + (PERM ? 3 : 1); };
    if constexpr (FUSED) {
        if (!wait_levels(need_for(1))) {
            status = PTP_ERR_TIMEOUT;
            k = 0;  // the loop below does not run
        }
    }
    Band bd;  // iteration 1: i_0 = 0, j_1 = min(1, rho - 1)
    {
        const int j1 = rho > 1 ? 1 : 0;
        bd.lo = 0;
        bd.copy_lo = 0;
        bd.vi_end = off_at(1);
        bd.vj_beg = off_at(j1);
        bd.hi = off_at(j1 + 1);
    }

    // Learned multi-advance band (band_mode 2): the group of iteration k is
    // the toplesets V_{i+1} .. V_{gend-1} that are due (sched_due), band
    // positions [bd.vi_end, g_hi) with g_hi = off[gend].
    constexpr bool multi = MULTI;
    // The group state is CTA-uniform: every thread computes the same values
    // and writes them to shared memory (s_mg = gend, g_hi), where they cost the
    // iteration no registers; the next write comes only after a CTA barrier
    // that every reader of the previous values has passed.
    __shared__ int s_mg[2];
    // The group's test result of iteration k: set to 1 by any thread whose
    // group vertex failed, read and cleared by thread 0 after the CTA
    // barrier that ends the iteration's work; two slots by parity, so a slot
    // is written again only two barriers after thread 0 cleared it.
    __shared__ int s_gfail[2];
    if constexpr (MULTI) {
        if (threadIdx.x == 0) {
            s_mg[0] = 1;
            s_mg[1] = 0;
            s_gfail[0] = s_gfail[1] = 0;
        }
        __syncthreads();
    }
    __shared__ int s_pf[2][MULTI ? 9 : 1];
    const int slim = FUSED ? a.n + 8 : rho;  // entries of the schedule array

    for (; k >= 1 && k <= max_iter; ++k) {
        if constexpr (FUSED) {
            if (!wait_levels(need_for(k))) {
                status = PTP_ERR_TIMEOUT;
                break;
            }
        }
        const int j = k < rho ? (int)k : rho - 1;
        const float *dp = (k & 1) ? a.d0 : a.d1;  // d_{k-1} lives in buffer (k-1) % 2
        float *dnx = (k & 1) ? a.d1 : a.d0;
        const int *lp = (k & 1) ? a.lab0 : a.lab1;
        int *lnx = (k & 1) ? a.lab1 : a.lab0;
        const bool entering = (long long)j == k;
        const int first = bd.lo > nsrc ? bd.lo : nsrc;
        const int start = bd.copy_lo < first ? bd.copy_lo : first;
        const bool testing = multi || k >= check_from;
        // multi: what the next group end needs (schedule and offsets from gend
        // on), one value per thread 0..8, copied into shared memory with
        // cp.async now and waited for just before the CTA barrier at the end
        // of the iteration (no register holds it across the band's work)
        int *const pf = s_pf[k & 1];
        if constexpr (multi) {
            const int q = threadIdx.x, ge = s_mg[0];
            const int *src = nullptr;
            if (q < 4) {
                if (ge + q < slim) src = a.sched + ge + q;
                else pf[q] = 0x3fffffff;
            } else if (q < 9) {
                const int r = ge + q - 4 < a.n + 1 ? ge + q - 4 : a.n + 1;
                src = a.off + (r < rho ? r : rho);
            }
            if (src) {
                const unsigned dst = (unsigned)__cvta_generic_to_shared(pf + q);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" : : "r"(dst), "l"(src) : "memory");
            }
        }

        int notconv = 0, n_active = 0, n_changed = 0;
        float maxrel = 0.0f;
        double errsum = 0.0;
        const int base = start & ~31;
        const int nchunks = bd.hi > base ? (bd.hi - base + 31) >> 5 : 0;

        // Recompute band vertex u from d_{k-1}, given its one-ring slots and
        // geometry: write d_k (and its label), stamp the neighbours if it
        // changed, and apply the relative-change test to V_{i_{k-1}}.
        auto recompute = [&](int u, bool in_vi, float dold, int meta, int4 r0, int4 r1, float4 l0, float4 l1,
                             const float4 *g) {
            const int ids[PTP_RING] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            const float el[PTP_RING] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
            const int m = meta & PTP_META_CNT;
            int label = LABELS ? __ldcg(lp + u) : 0;
            float dnew;
            if (meta & PTP_META_GENERAL) dnew = update_general(a, u, dold, dp, lp, LABELS ? &label : nullptr, nfp64);
            else dnew = update_ring<LABELS>(a, u, ids, el, g, m, dold, dp, lp, label, nfp64);
            ++n_active;
            dnx[u] = dnew;
            if (LABELS) lnx[u] = label;
            if (dnew != dold) {
                ++n_changed;
                a.chg[u] = (int)k;
                if (meta & PTP_META_GENERAL) {
                    stamp_general(a, u, (int)k);
                } else {
#pragma unroll
                    for (int t = 0; t < PTP_RING; ++t)
                        if (t < m) a.nstamp[ids[t]] = (int)k;
                }
                // multi: the group's test, for its vertices (u is the band
                // position here; the group is [bd.vi_end, s_mg[1]))
                const bool in_g = multi && u >= bd.vi_end && u < s_mg[1];
                if ((in_vi && testing) || in_g || a.conv_trace) {
                    // relative-change test of Eq. lower_band, in FP64 (the
                    // difference of two floats is exact in double)
                    const double o = dold, delta = o - (double)dnew;
                    const bool fail = !(isfinite(o) && delta < __dadd_rn(__dmul_rn(a.eps, o), a.eps_abs));
                    if (fail && in_g) s_gfail[k & 1] = 1;
                    if (fail && a.conv_trace) atomicMax(a.conv_trace + topleset_of(a.off, rho, u), (int)k);
                    if (in_vi && testing) {
                    if (fail) notconv = 1;
                    if (a.trace) {
                        const double rel = isfinite(o) ? (o > 0.0 ? delta / o : 0.0) : (double)INF;
                        maxrel = fmaxf(maxrel, (float)rel);
                        errsum += rel;
                    }
                    }
                }
            }
        };
        // The geometry of every slot is loaded whatever the vertex's count:
        // every slot is written, and the loads need not wait for meta.  The
        // loads go through L2 only: a fused launch writes these arrays while
        // it runs, and with the read-only cache the unfused kernel was no
        // faster (a vertex is rarely recomputed on the same SM twice).
        auto load_slots = [&](int u, int &meta, int4 &r0, int4 &r1, float4 &l0, float4 &l1, float4 *g) {
            meta = __ldcg(a.meta + u);
            r0 = __ldcg(a.ring + u);
            r1 = __ldcg(a.ring + a.n + u);
            l0 = __ldcg(a.elen + u);
            l1 = __ldcg(a.elen + a.n + u);
#pragma unroll
            for (int t = 0; t < PTP_TRI; ++t) g[t] = __ldcg(a.tgeom + (size_t)t * a.n + u);
        };

        if (nchunks <= nwarps) {
            // Narrow band: at most one chunk per warp (c = gwarp).  The warp
            // loads its chunk's state, one-ring slots and geometry in one round
            // trip and recomputes in place, with no queue and no CTA barrier
            // between the passes; the extra geometry read for vertices that
            // turn out not to need an update is small at this band width.
            if (gwarp < nchunks) {
                const int p = base + gwarp * 32 + lane;
                const bool ok = p >= start && p < bd.hi && p >= nsrc;
                const bool live = ok && p >= bd.lo;
                const int u = ok ? vertex_at(p) : 0;
                const float dold = ok ? __ldcg(dp + u) : 0.0f;
                const int ns = live ? __ldcg(a.nstamp + u) : -2;
                const int cg = live ? __ldcg(a.chg + u) : -2;
                int meta = 0;
                int4 r0 = make_int4(-1, -1, -1, -1), r1 = r0;
                float4 l0 = make_float4(0.f, 0.f, 0.f, 0.f), l1 = l0;
                float4 g[PTP_TRI];
#pragma unroll
                for (int t = 0; t < PTP_TRI; ++t) g[t] = l0;
                if (live) load_slots(u, meta, r0, r1, l0, l1, g);
                if (ok && !live) {  // retired after the previous iteration
                    dnx[u] = dold;
                    if (LABELS) lnx[u] = __ldcg(lp + u);
                }
                const bool need = live && ((entering && p >= bd.vj_beg) || ns >= k - 1);
                if (live && !need && cg == k - 1) {
                    dnx[u] = dold;
                    if (LABELS) lnx[u] = __ldcg(lp + u);
                }
                if (need) recompute(u, p < bd.vi_end, dold, meta, r0, r1, l0, l1, g);
            }
        } else {
            // chunks of this CTA's warps: c = gwarp + m * nwarps, m = 0, 1, ...
            const int rounds_m = nchunks > gwarp ? (nchunks - gwarp + nwarps - 1) / nwarps : 0;
            // every warp of the CTA must run the same number of rounds
            const int cta_m = (nchunks > (int)blockIdx.x) ? (nchunks - (int)blockIdx.x + nwarps - 1) / nwarps : 0;
            for (int m0 = 0; m0 < cta_m; m0 += ROUND_CHUNKS) {
                if (threadIdx.x == 0) s_nq = 0;
                __syncthreads();
                // pass 1: state of each band vertex; queue the ones to recompute.
                // The state of P1_BATCH chunks is loaded before any is used.
                for (int m = m0; m < m0 + ROUND_CHUNKS && m < rounds_m; m += P1_BATCH) {
                    int pp[P1_BATCH], uu[P1_BATCH], ns[P1_BATCH], cg[P1_BATCH];
                    float dold[P1_BATCH];
                    bool live[P1_BATCH];
#pragma unroll
                    for (int q = 0; q < P1_BATCH; ++q) {
                        pp[q] = base + (gwarp + (m + q) * nwarps) * 32 + lane;
                        const bool ok = m + q < rounds_m && pp[q] >= start && pp[q] < bd.hi && pp[q] >= nsrc;
                        live[q] = ok && pp[q] >= bd.lo;
                        uu[q] = ok ? vertex_at(pp[q]) : 0;
                    }
#pragma unroll
                    for (int q = 0; q < P1_BATCH; ++q) {
                        const bool ok = m + q < rounds_m && pp[q] >= start && pp[q] < bd.hi && pp[q] >= nsrc;
                        dold[q] = ok ? __ldcg(dp + uu[q]) : 0.0f;
                        ns[q] = live[q] ? __ldcg(a.nstamp + uu[q]) : -2;
                        cg[q] = live[q] ? __ldcg(a.chg + uu[q]) : -2;
                        if (ok && !live[q]) {  // retired after the previous iteration
                            dnx[uu[q]] = dold[q];
                            if (LABELS) lnx[uu[q]] = __ldcg(lp + uu[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < P1_BATCH; ++q) {
                        const bool need = live[q] && ((entering && pp[q] >= bd.vj_beg) || ns[q] >= k - 1);
                        if (live[q] && !need && cg[q] == k - 1) {
                            dnx[uu[q]] = dold[q];
                            if (LABELS) lnx[uu[q]] = __ldcg(lp + uu[q]);
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, need);
                        if (bal) {
                            int at = 0;
                            if (lane == 0) at = atomicAdd(&s_nq, __popc(bal));
                            at = __shfl_sync(0xffffffffu, at, 0);
                            if (need)
                                s_queue[at + __popc(bal & ((1u << lane) - 1u))] =
                                    make_int2(uu[q] | (pp[q] < bd.vi_end ? (int)0x80000000 : 0), __float_as_int(dold[q]));
                        }
                    }
                }
                __syncthreads();
                // pass 2: recompute the queued vertices
                const int nq = s_nq;
                for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                    const int2 ent = s_queue[q];
                    const int u = ent.x & 0x7fffffff;
                    int meta;
                    int4 r0, r1;
                    float4 l0, l1, g[PTP_TRI];
                    load_slots(u, meta, r0, r1, l0, l1, g);
                    recompute(u, ent.x < 0, __int_as_float(ent.y), meta, r0, r1, l0, l1, g);
                }
                // the queue is refilled by the next round; after the last one
                // only in the next iteration, behind the grid barrier
                if (m0 + ROUND_CHUNKS < cta_m) __syncthreads();
            }
        }
        tot_active += n_active;
        tot_changed += n_changed;

        if (a.trace && k - 1 < a.trace_cap) {
            const float wm = warp_max_f(maxrel);
            const double ws = warp_sum_d(errsum);
            const int wa = warp_sum_i(n_active), wc = warp_sum_i(n_changed);
            if (lane == 0) {
                s_max[wid] = wm;
                s_sum[wid] = ws;
                s_cnt[0][wid] = wa;
                s_cnt[1][wid] = wc;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                float bm = 0.0f;
                double bs = 0.0;
                int ba = 0, bc = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    bm = fmaxf(bm, s_max[w]);
                    bs += s_sum[w];
                    ba += s_cnt[0][w];
                    bc += s_cnt[1][w];
                }
                ptp_trace_rec *rec = a.trace + (k - 1);
                if (ba) atomicAdd(&rec->active, ba);
                if (bc) atomicAdd(&rec->changed, bc);
                if (bs != 0.0) atomicAdd(&rec->errsum, bs);
                if (bm > 0.0f) atomicMax((int *)&rec->maxrel, __float_as_int(bm));
            }
        }

        // the bounds the next iteration may need are static: fetch them now
        const int jn = k + 1 < rho ? (int)(k + 1) : rho - 1;
        const int o_i2 = off_at(i + 2);
        const int o_jn = off_at(jn), o_jn1 = off_at(jn + 1);
        const int sched_next = (a.sched && !multi && i + 1 < rho) ? __ldcg(a.sched + i + 1) : 1;
        // multi: every thread reads the prefetched values after the grid
        // barrier, whose last step is a CTA barrier (two buffers by iteration
        // parity, so the next write waits a barrier)
        if constexpr (multi) {
            if (threadIdx.x < 9) asm volatile("cp.async.wait_all;" : : : "memory");
        }

        const int any = __syncthreads_or(notconv);
        int anyg = 0;
        if constexpr (multi) {
            if (threadIdx.x == 0) {  // only thread 0's value enters the grid barrier
                anyg = s_gfail[k & 1];
                s_gfail[k & 1] = 0;
            }
        }
        const long long failed = ptp_grid_sync(a.ctrl->bar, k, (any ? 1u : 0u) | (anyg ? 0x10000u : 0u),
                                               &a.ctrl->abort, &a.ctrl->status, prev_hi, (unsigned)ncta,
                                               PTP_WAIT_CYCLES, true);
        if (failed < 0) {
            status = PTP_ERR_TIMEOUT;
            break;
        }
        // Eq. lower_band (applied from iteration check_from on), or the fixed
        // band whose lower bound is ceil(k / 2)
        const bool bottom_ok = (failed & 0xffff) == 0, group_ok = (failed >> 16) == 0;
        const bool advance = a.band_mode == 1 ? (int)((k + 1) >> 1) > i : (testing && bottom_ok);
        // multi: the bottom and every due topleset above it passed: retire them all
        const int gend = multi ? s_mg[0] : 1;
        const bool jump = multi && advance && gend > i + 1 && group_ok;
        if (leader) {
            band_updates += bd.hi - first;
            checks += testing ? 1 : 0;
            if (a.trace && k - 1 < a.trace_cap) {
                ptp_trace_rec *rec = a.trace + (k - 1);
                rec->i = i;
                rec->j = j;
                rec->advanced = jump ? gend - i : (advance ? 1 : 0);
            }
        }
        if (jump) {
            // V_{i_{k-1}} .. V_{gend-1} retire together and are copied forward
            // in the next iteration (V_0 never changes)
            bd.copy_lo = i >= 1 ? bd.lo : bd.vi_end;
            i = gend;
            if (i > rho - 1) {
                status = PTP_OK;
                break;
            }
            bd.lo = pf[4];
            bd.vi_end = pf[5];
        } else if (advance) {
            // i_k = i_{k-1} + 1: V_{i_{k-1}} retires and is copied forward in
            // the next iteration (V_0 never changes)
            ++i;
            if (i > rho - 1) {
                status = PTP_OK;
                break;
            }
            // V_i is the new bottom from iteration k + 1 on; with a schedule
            // its first test comes after the predicted number of iterations
            check_from = k + (sched_next > 1 ? sched_next : 1);
            bd.copy_lo = i >= 2 ? bd.lo : bd.vi_end;
            bd.lo = bd.vi_end;
            bd.vi_end = o_i2;
        } else {
            bd.copy_lo = bd.lo;
        }
        if constexpr (multi) {
            // the next group: from V_{i+1} on, every topleset due by iteration
            // k + 1 (at most four more per iteration, from the prefetch)
            int g = gend > i + 1 ? gend : i + 1;
            while (g - gend < 4 && g < rho && sched_due(g, pf[g - gend]) <= k + 1) ++g;
            const int ghi = pf[4 + g - gend];
            __syncwarp();
            s_mg[0] = g;  // the same values from every thread
            s_mg[1] = ghi;
        }
        bd.vj_beg = o_jn;
        bd.hi = o_jn1;
    }
    if (status == PTP_ERR_NOT_CONVERGED) k = max_iter;

    // per-CTA totals
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
    if (leader) {
        a.ctrl->iterations = k;
        a.ctrl->band_updates = band_updates;
        a.ctrl->checks = checks;
        if (status != PTP_ERR_TIMEOUT) atomicCAS(&a.ctrl->status, 0, status);
    }
}

__global__ void init_distances(const int *__restrict__ off, int n, float *__restrict__ d0, float *__restrict__ d1,
                               int *__restrict__ nstamp, int *__restrict__ chg) {
    const int nsrc = off[1];
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const float v = u < nsrc ? 0.0f : INF;
        d0[u] = v;
        d1[u] = v;
        nstamp[u] = -2;
        chg[u] = -2;
    }
}

// d_out[perm[u]] = d_K[u]; the final iterate lives in buffer K % 2.
__global__ void scatter_out(const int *__restrict__ perm, int n, const float *__restrict__ d0, const float *__restrict__ d1,
                            const ptp_ctrl *__restrict__ ctrl, float *__restrict__ out) {
    const float *d = (ctrl->iterations & 1) ? d1 : d0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) out[perm[u]] = d[u];
}

// Multi-source runs in the original order: distances +inf and labels
// "none" everywhere, then the sources.
__global__ void init_multi(int n, float *__restrict__ d0, float *__restrict__ d1, int *__restrict__ nstamp,
                           int *__restrict__ chg, int *__restrict__ lab0, int *__restrict__ lab1) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        d0[u] = INF;
        d1[u] = INF;
        nstamp[u] = -2;
        chg[u] = -2;
        if (lab0) {
            lab0[u] = 0x7fffffff;
            lab1[u] = 0x7fffffff;
        }
    }
}

__global__ void seed_multi(const int *__restrict__ src, int m, const int *__restrict__ m_dev, float *__restrict__ d0,
                           float *__restrict__ d1, int *__restrict__ lab0, int *__restrict__ lab1) {
    if (m_dev) m = *m_dev;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        const int v = src[q];
        d0[v] = 0.0f;
        d1[v] = 0.0f;
        if (lab0) {
            atomicMin(&lab0[v], q);  // a repeated seed keeps its first index
            atomicMin(&lab1[v], q);
        }
    }
}

unsigned blocks_for(int64_t work, int threads, int device) {
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)ptp_num_sms(device) * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

ptp_status ptp_internal_window_multi(const ptp_mesh *mesh, ptp_multi_bufs *b, const ptp_params *params,
                                     const int *src, const int *m_dev, int m_max, bool labels, cudaStream_t s) {
    const int n = b->n;
    const int dev = mesh->device;
    PTP_TRY(cudaMemsetAsync(b->ctrl, 0, sizeof(ptp_ctrl), s));
    init_multi<<<blocks_for(n, 256, dev), 256, 0, s>>>(n, b->d0, b->d1, b->nstamp, b->chg, labels ? b->lab0 : nullptr,
                                                        labels ? b->lab1 : nullptr);
    seed_multi<<<blocks_for(m_max, 256, dev), 256, 0, s>>>(src, m_max, m_dev, b->d0, b->d1, labels ? b->lab0 : nullptr,
                                                           labels ? b->lab1 : nullptr);
    ptp_count_launches(2);
    PTP_TRY(cudaGetLastError());
    const void *fn = labels ? (const void *)ptp_window<true, true> : (const void *)ptp_window<true, false>;
    const int block = window_block(params->block);
    if (block < 0) return PTP_ERR_ARG;
    int per_sm = 0;
    PTP_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0));
    if (per_sm < 1) return PTP_ERR_CUDA;
    int grid = per_sm * ptp_num_sms(dev);
    if (params->grid > 0 && params->grid < grid) grid = params->grid;
    DistArgs a = {};
    a.n = n;
    a.pos = mesh->pos;
    a.ring = mesh->ring;
    a.tgeom = mesh->tgeom;
    a.elen = mesh->elen;
    a.meta = mesh->meta;
    a.row = mesh->row;
    a.pairs = mesh->pairs;
    a.off = b->off;
    a.info = b->info;
    a.d0 = b->d0;
    a.d1 = b->d1;
    a.nstamp = b->nstamp;
    a.chg = b->chg;
    a.ctrl = b->ctrl;
    a.trace = (ptp_trace_rec *)params->trace;
    a.trace_cap = params->trace ? params->trace_cap : 0;
    a.eps = params->eps;
    a.eps_abs = params->eps_abs;
    a.max_iter = params->max_iter;
    a.perm = b->queue;
    a.lab0 = labels ? b->lab0 : nullptr;
    a.lab1 = labels ? b->lab1 : nullptr;
    a.band_mode = params->band_mode;
    a.sched = params->schedule;
    if (params->trace && params->trace_cap > 0)
        PTP_TRY(cudaMemsetAsync(params->trace, 0, sizeof(ptp_trace_rec) * params->trace_cap, s));
    void *args[] = {(void *)&a};
    PTP_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, s));
    ptp_count_launches(1);
    return PTP_OK;
}

ptp_status ptp_internal_window_occupancy(int block, int *per_sm) {
    *per_sm = 0;
    PTP_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, ptp_window<false, false>, block, 0));
    return PTP_OK;
}

namespace {

// V_0 of a fused launch: off[0..1], the BFS state the producers start from,
// and the sources' positions.
__global__ void fused_setup(ptp_ctrl *ctrl, int *off, const int *info, const int *queue, int *iperm, int n,
                            const int *__restrict__ ometa, const int4 *__restrict__ oring, int *meta_w, int4 *ring_w) {
    const int m0 = info[3];  // unique sources, queued by the seeding kernel
    for (int q = threadIdx.x; q < m0; q += blockDim.x) {
        // position q, with the record the producers read (meta, raw slots)
        const int v = queue[q];
        iperm[v] = q;
        const int vm = ometa[v];
        const int vc = (vm & PTP_META_GENERAL) ? 0 : (vm & PTP_META_CNT);
        const int4 w0 = oring[v], w1 = oring[n + v];
        meta_w[q] = vm;
        ring_w[q] = make_int4(vc > 0 ? w0.x : -1, vc > 1 ? w0.y : -1, vc > 2 ? w0.z : -1, vc > 3 ? w0.w : -1);
        ring_w[n + q] = make_int4(vc > 4 ? w1.x : -1, vc > 5 ? w1.y : -1, vc > 6 ? w1.z : -1, vc > 7 ? w1.w : -1);
    }
    if (threadIdx.x != 0) return;
    off[0] = 0;
    off[1] = m0;
    ctrl->tail = m0;
    ctrl->ready = 1;
}

// Distances of a renumbered fused run, back to the original order:
// d_out[v] = d_K[iperm[v]] for reached vertices, +inf for the others.
__global__ void fused_gather(const ptp_ctrl *__restrict__ ctrl, int n, const int *__restrict__ level,
                             const int *__restrict__ iperm, const float *__restrict__ d0, const float *__restrict__ d1,
                             float *__restrict__ d_out) {
    const float *d = (ctrl->iterations & 1) ? d1 : d0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        d_out[v] = level[v] >= 0 ? d[iperm[v]] : INF;
}

// The fused window kernel: renumbered (topleset order, the single-map
// path) or in the original order (multi-source maps, with or without labels).
const void *fused_kernel(bool perm, bool labels, bool multi) {
    if (!perm) return multi ? (const void *)ptp_window<false, false, true, true> : (const void *)ptp_window<false, false, true>;
    return labels ? (const void *)ptp_window<true, true, true> : (const void *)ptp_window<true, false, true>;
}

// Launch shape of a fused run: CTAs in all, how many run the BFS and how
// many copy the toplesets into place (topleset order only: as many as run
// the BFS, whose levels they copy, one position per thread when a level
// fits the producers' threads).  A
// level's frontier grows like sqrt(n) on these meshes from one source (a few
// thousand vertices at a million), and like n / rho from many: 2 sqrt(n m)
// producer threads for m sources, from 2048 up to 8192 for one source and
// 16384 for several, at most a quarter of the grid (0 when the grid cannot
// split).  From one source the BFS paces the window only while the band is
// narrow, when the frontier is still small, so the largest levels may take
// two rounds and every CTA spared from the BFS runs the window, whose wide
// bands are throughput-bound; a multi-source map (K close to rho, wide
// frontiers from the first level) is paced by the BFS throughout.
ptp_status fused_shape(const ptp_mesh *mesh, const ptp_params *params, int m, bool perm, bool labels, int *block,
                       int *grid, int *producers, int *copiers) {
    *block = window_block(params->block);
    if (*block < 0) return PTP_ERR_ARG;
    int per_sm = 0;
    PTP_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel(perm, labels, params->band_mode == 2),
                                                          *block, 0));
    if (per_sm < 1) return PTP_ERR_CUDA;
    *grid = per_sm * ptp_num_sms(mesh->device);
    if (params->grid > 0 && params->grid < *grid) *grid = params->grid;
    double th = 2.0 * sqrt((double)mesh->n * (double)(m > 1 ? m : 1));
    const double th_max = m > 1 ? 16384.0 : 8192.0;
    th = th < 2048.0 ? 2048.0 : (th > th_max ? th_max : th);
    int p = ((int)th + *block - 1) / *block;
    if (p > *grid / 4) p = *grid / 4;
    *producers = p > 0 ? p : 0;
    *copiers = perm ? 0 : *producers;
    return PTP_OK;
}

}  // namespace

int ptp_internal_fused_producers(const ptp_mesh *mesh, const ptp_params *params, int m, bool perm, bool labels) {
    int block = 0, grid = 0, producers = 0, copiers = 0;
    if (fused_shape(mesh, params, m, perm, labels, &block, &grid, &producers, &copiers) != PTP_OK) return 0;
    return producers;
}

ptp_status ptp_internal_fused_gather(const ptp_mesh *mesh, const ptp_multi_bufs *b, const ptp_renum_bufs *rb,
                                     float *d_out, cudaStream_t s) {
    fused_gather<<<blocks_for(b->n, 256, mesh->device), 256, 0, s>>>(b->ctrl, b->n, b->level, rb->iperm, b->d0, b->d1,
                                                                     d_out);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

ptp_status ptp_internal_fused(const ptp_mesh *mesh, ptp_multi_bufs *b, const ptp_params *params, const int *src,
                              const int *m_dev, int m_max, bool perm, bool labels, const ptp_renum_bufs *rb,
                              cudaStream_t s) {
    const int n = b->n;
    const int dev = mesh->device;
    int block = 0, grid = 0, producers = 0, copiers = 0;
    PTP_CHECK(fused_shape(mesh, params, m_max, perm, labels, &block, &grid, &producers, &copiers));
    if (producers < 1) return PTP_ERR_TOO_LARGE;  // callers check ptp_internal_fused_producers first
    PTP_CHECK(ptp_internal_bfs_seed(mesh, b, src, m_dev, m_max, s));
    PTP_TRY(cudaMemsetAsync(b->ctrl, 0, sizeof(ptp_ctrl), s));
    fused_setup<<<1, 256, 0, s>>>(b->ctrl, b->off, b->info, b->queue, rb->iperm, n, mesh->meta, mesh->ring, rb->meta,
                                  rb->ring);
    if (perm) {
        // distances (and labels) in the original order
        init_multi<<<blocks_for(n, 256, dev), 256, 0, s>>>(n, b->d0, b->d1, b->nstamp, b->chg,
                                                            labels ? b->lab0 : nullptr, labels ? b->lab1 : nullptr);
        seed_multi<<<blocks_for(m_max, 256, dev), 256, 0, s>>>(src, m_max, m_dev, b->d0, b->d1,
                                                               labels ? b->lab0 : nullptr, labels ? b->lab1 : nullptr);
        ptp_count_launches(3);
    } else {
        // distances by position: the sources are positions [0, off[1])
        init_distances<<<blocks_for(n, 256, dev), 256, 0, s>>>(b->off, n, b->d0, b->d1, b->nstamp, b->chg);
        ptp_count_launches(2);
    }
    PTP_TRY(cudaGetLastError());
    DistArgs a = {};
    a.n = n;
    if (perm) {
        // the window reads the original mesh; rb holds only the BFS's records
        a.pos = mesh->pos;
        a.ring = mesh->ring;
        a.tgeom = mesh->tgeom;
        a.elen = mesh->elen;
        a.meta = mesh->meta;
        a.lab0 = labels ? b->lab0 : nullptr;
        a.lab1 = labels ? b->lab1 : nullptr;
    } else {
        a.pos = rb->pos;
        a.ring = rb->ring;
        a.tgeom = rb->tgeom;
        a.elen = rb->elen;
        a.meta = rb->meta;
        a.gmap = rb->iperm;  // original corner lists: GENERAL vertices map through iperm
        a.coherent = 1;
    }
    a.row = mesh->row;
    a.pairs = mesh->pairs;
    a.off = b->off;
    a.info = b->info;
    a.d0 = b->d0;
    a.d1 = b->d1;
    a.nstamp = b->nstamp;
    a.chg = b->chg;
    a.ctrl = b->ctrl;
    a.trace = (ptp_trace_rec *)params->trace;
    a.trace_cap = params->trace ? params->trace_cap : 0;
    a.eps = params->eps;
    a.eps_abs = params->eps_abs;
    a.max_iter = params->max_iter;
    a.perm = b->queue;
    a.band_mode = params->band_mode;
    a.sched = nullptr;  // band_mode 0: a schedule needs the whole toplesets first
    const bool multi = params->band_mode == 2;
    if (multi) {
        // the learned multi-advance band: the launch infers the schedule
        if (perm || !rb->sched || !rb->facc || !params->mlp_half) return PTP_ERR_ARG;
        PTP_TRY(cudaMemsetAsync(rb->facc, 0, sizeof(unsigned long long) * FEAT_RING * FEAT_WORDS, s));
        a.sched = rb->sched;
        a.sched_w = rb->sched;
        a.facc = rb->facc;
        a.mlp_w = params->mlp_half;
        a.mlp_margin = params->mlp_margin;
        const double diam = mesh->diameter > 0.0 ? mesh->diameter : 1.0;
        a.feat_scale = 1073741824.0 / diam;
        a.feat_scale2 = 1073741824.0 / (diam * diam);
    }
    a.producers = producers;
    a.copiers = copiers;
    a.level = b->level;
    a.queue_w = b->queue;
    a.off_w = b->off;
    a.info_w = b->info;
    a.opos = mesh->pos;
    a.oring = mesh->ring;
    a.ometa = mesh->meta;
    a.otgeom = mesh->tgeom;
    a.oelen = mesh->elen;
    a.pos_w = rb->pos;
    a.ring_w = rb->ring;
    a.meta_w = rb->meta;
    a.tgeom_w = rb->tgeom;
    a.elen_w = rb->elen;
    a.iperm = rb->iperm;
    if (params->trace && params->trace_cap > 0)
        PTP_TRY(cudaMemsetAsync(params->trace, 0, sizeof(ptp_trace_rec) * params->trace_cap, s));
    void *args[] = {(void *)&a};
    if (params->ev_begin) PTP_TRY(cudaEventRecord((cudaEvent_t)params->ev_begin, s));
    PTP_TRY(cudaLaunchCooperativeKernel(fused_kernel(perm, labels, multi), dim3(grid), dim3(block), args, 0, s));
    ptp_count_launches(1);
    if (params->ev_end) PTP_TRY(cudaEventRecord((cudaEvent_t)params->ev_end, s));
    return PTP_OK;
}

namespace {

// Validation shared by ptp_distance and ptp_distance_noalloc.
ptp_status check_distance_args(const ptp_toplesets_t *t, const ptp_params *params, const float *d_out) {
    if (!t || !params || !d_out) return PTP_ERR_ARG;
    if (!(params->eps >= 0.0) || !(params->eps_abs >= 0.0) || params->max_iter < 0 || params->trace_cap < 0)
        return PTP_ERR_ARG;
    if (window_block(params->block) < 0) return PTP_ERR_ARG;
    if (params->band_mode < 0 || params->band_mode > 2) return PTP_ERR_ARG;
    if (params->band_mode == 2 && !params->schedule) return PTP_ERR_ARG;  // the learned band needs its schedule
    if (params->reserved != 0 || params->reserved2 != 0 || params->mlp_half) return PTP_ERR_ARG;
    if (t->n >= 0x40000000) return PTP_ERR_TOO_LARGE;  // queue entries carry two flag bits
    return PTP_OK;
}

// One window run of toplesets t on stream s with the given scratch: dbuf
// holds d0, d1 (2n floats), ibuf nstamp, chg (2n ints), ctrl the control
// block.  Clears the control block (and the trace), initialises the
// scratch, launches the window kernel and scatters d_K to d_out.
// ptp_distance and ptp_distance_noalloc differ only in where the scratch
// and the control block come from.
ptp_status run_window(const ptp_toplesets_t *t, const ptp_params *params, float *dbuf, int *ibuf, ptp_ctrl *ctrl,
                      float *d_out, cudaStream_t s) {
    const int64_t n = t->n;
    const int dev = t->device;
    const int block = window_block(params->block);
    PTP_TRY(cudaMemsetAsync(ctrl, 0, sizeof(ptp_ctrl), s));
    if (params->trace && params->trace_cap > 0)
        PTP_TRY(cudaMemsetAsync(params->trace, 0, sizeof(ptp_trace_rec) * params->trace_cap, s));
    init_distances<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->off, (int)n, dbuf, dbuf + n, ibuf, ibuf + n);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    const void *fn = params->band_mode == 2 ? (const void *)ptp_window<false, false, false, true>
                                            : (const void *)ptp_window<false, false>;
    int per_sm = 0;
    PTP_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0));
    if (per_sm < 1) return PTP_ERR_CUDA;
    int grid = per_sm * ptp_num_sms(dev);
    if (params->grid > 0 && params->grid < grid) grid = params->grid;

    DistArgs a = {};
    a.n = (int)n;
    a.pos = t->pos;
    a.ring = t->ring;
    a.tgeom = t->tgeom;
    a.elen = t->elen;
    a.meta = t->meta;
    a.row = t->row;
    a.pairs = t->pairs;
    a.off = t->off;
    a.info = t->info;
    a.d0 = dbuf;
    a.d1 = dbuf + n;
    a.nstamp = ibuf;
    a.chg = ibuf + n;
    a.ctrl = ctrl;
    a.trace = (ptp_trace_rec *)params->trace;
    a.trace_cap = params->trace ? params->trace_cap : 0;
    a.eps = params->eps;
    a.eps_abs = params->eps_abs;
    a.max_iter = params->max_iter;
    a.perm = nullptr;
    a.lab0 = a.lab1 = nullptr;
    a.band_mode = params->band_mode;
    a.sched = params->schedule;
    a.conv_trace = params->conv_trace;
    void *args[] = {(void *)&a};
    if (params->ev_begin) PTP_TRY(cudaEventRecord((cudaEvent_t)params->ev_begin, s));
    PTP_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, s));
    ptp_count_launches(1);
    if (params->ev_end) PTP_TRY(cudaEventRecord((cudaEvent_t)params->ev_end, s));
    scatter_out<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->perm, (int)n, dbuf, dbuf + n, ctrl, d_out);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

// Statistics of the run whose control block is ctrl (blocks on s).
ptp_status read_stats(const ptp_ctrl *ctrl, const int *info_dev, cudaStream_t s, ptp_stats *st) {
    ptp_ctrl h;
    int info[4];
    PTP_TRY(cudaMemcpyAsync(&h, ctrl, sizeof(ptp_ctrl), cudaMemcpyDeviceToHost, s));
    PTP_TRY(cudaMemcpyAsync(info, info_dev, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    PTP_TRY(cudaStreamSynchronize(s));
    st->iterations = h.iterations;
    st->band_updates = h.band_updates;
    st->active_updates = (int64_t)h.active;
    st->changed = (int64_t)h.changed;
    st->fp64_solves = (int64_t)h.fp64;
    st->rho = info[0];
    st->status = h.status;
    st->checks = h.checks;
    return (ptp_status)h.status;
}

}  // namespace

extern "C" ptp_status ptp_distance(ptp_toplesets_t *t, const ptp_params *params, float *d_out, void *stream,
                                   ptp_stats *stats) {
    PTP_CHECK(check_distance_args(t, params, d_out));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = t->n;
    float *dbuf = nullptr;
    int *ibuf = nullptr;
    PTP_TRY(ptp_malloc_async((void **)&dbuf, sizeof(float) * 2 * n, s));
    cudaError_t ce = ptp_malloc_async((void **)&ibuf, sizeof(int) * 2 * n, s);
    if (ce != cudaSuccess) {
        cudaFreeAsync(dbuf, s);
        return ptp_internal_cuda_status(ce);
    }
    const ptp_status st = run_window(t, params, dbuf, ibuf, t->ctrl, d_out, s);
    cudaFreeAsync(dbuf, s);
    cudaFreeAsync(ibuf, s);
    if (st != PTP_OK) return st;
    if (stats) return read_stats(t->ctrl, t->info, s, stats);
    return PTP_OK;
}

extern "C" ptp_status ptp_last_stats(ptp_toplesets_t *t, void *stream, ptp_stats *st) {
    if (!t || !st) return PTP_ERR_ARG;
    return read_stats(t->ctrl, t->info, (cudaStream_t)stream, st);
}

extern "C" ptp_status ptp_geodesic(const float *xyz, int64_t n_verts, const int32_t *faces, int64_t n_faces,
                                   const int32_t *sources, int32_t m, int ptr_kind, const ptp_params *params,
                                   float *d_out, void *stream, ptp_stats *stats) {
    if (!d_out || !params) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ptp_mesh *mesh = nullptr;
    PTP_CHECK(ptp_mesh_create(xyz, n_verts, faces, n_faces, ptr_kind, stream, &mesh));
    float *dev_out = d_out;
    if (ptr_kind == PTP_HOST) {
        cudaError_t ce = ptp_malloc_async((void **)&dev_out, sizeof(float) * n_verts, s);
        if (ce != cudaSuccess) {
            ptp_mesh_destroy(mesh);
            return ptp_internal_cuda_status(ce);
        }
    }
    ptp_stats local;
    ptp_status st;
    if (!params->schedule) {
        // toplesets built inside the window launch
        st = ptp_distance_from_sources(mesh, sources, m, ptr_kind, params, dev_out, stream, &local);
    } else {
        // a learned schedule needs the whole toplesets first
        ptp_toplesets_t *tops = nullptr;
        st = ptp_toplesets(mesh, sources, m, ptr_kind, stream, &tops);
        if (st == PTP_OK) {
            st = ptp_distance(tops, params, dev_out, stream, &local);
            ptp_toplesets_destroy(tops);
        }
    }
    if (ptr_kind == PTP_HOST) {
        cudaError_t ce = cudaSuccess;
        if (st == PTP_OK || st == PTP_ERR_NOT_CONVERGED)
            ce = cudaMemcpyAsync(d_out, dev_out, sizeof(float) * n_verts, cudaMemcpyDeviceToHost, s);
        cudaFreeAsync(dev_out, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess && (st == PTP_OK || st == PTP_ERR_NOT_CONVERGED)) st = ptp_internal_cuda_status(ce);
    }
    if (stats && (st == PTP_OK || st == PTP_ERR_NOT_CONVERGED)) *stats = local;
    ptp_mesh_destroy(mesh);
    return st;
}

// ---------------------------------------------------------------------------
// ptp_distance_noalloc: the same window kernel with its per-call scratch in a
// file-scope device array instead of a stream-ordered allocation.
// ---------------------------------------------------------------------------

namespace {

// Layout: [0, 256) control block, then d0[n], d1[n], nstamp[n], chg[n].
constexpr size_t NOALLOC_HEADER = 256;
static_assert(sizeof(ptp_ctrl) <= NOALLOC_HEADER, "control block must fit the header");
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_HEADER + (size_t)PTP_NOALLOC_MAX_VERTS * 16];

constexpr int NOALLOC_MAX_DEVICES = 64;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES];
bool g_noalloc_ready[NOALLOC_MAX_DEVICES];

// Device address of the scratch array for the current device.  The array's
// name is only a host-side stand-in in host code, so its address is looked up
// once per device, with that device current, and cached per ordinal: the
// cache is valid as long as the device's primary context lives (not across
// cudaDeviceReset).
ptp_status noalloc_scratch(int dev, unsigned char **out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return PTP_ERR_ARG;
    if (!__atomic_load_n(&g_noalloc_ready[dev], __ATOMIC_ACQUIRE)) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return ptp_internal_cuda_status(e);
        g_noalloc_addr[dev] = p;
        __atomic_store_n(&g_noalloc_ready[dev], true, __ATOMIC_RELEASE);
    }
    *out = (unsigned char *)g_noalloc_addr[dev];
    return PTP_OK;
}

}  // namespace

extern "C" ptp_status ptp_distance_noalloc(ptp_toplesets_t *t, const ptp_params *params, float *d_out, void *stream,
                                           ptp_stats *stats) {
    PTP_CHECK(check_distance_args(t, params, d_out));
    if (t->n > (int64_t)PTP_NOALLOC_MAX_VERTS) return PTP_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = t->n;
    int dev = 0;
    PTP_TRY(cudaGetDevice(&dev));
    if (dev != t->device) return PTP_ERR_ARG;
    unsigned char *base = nullptr;
    PTP_CHECK(noalloc_scratch(dev, &base));
    ptp_ctrl *ctrl = (ptp_ctrl *)base;
    float *dbuf = (float *)(base + NOALLOC_HEADER);
    int *ibuf = (int *)(dbuf + 2 * n);
    // the array keeps the previous call's contents: run_window clears the
    // control block and init_distances rewrites all 4n scratch words
    PTP_CHECK(run_window(t, params, dbuf, ibuf, ctrl, d_out, s));
    if (!stats) return PTP_OK;
    return read_stats(ctrl, t->info, s, stats);
}
