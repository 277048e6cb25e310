// Internal declarations shared by the CUDA translation units of the PTP
// library.  Nothing here is part of the public ABI (include/ptp.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ptp.h"

#define PTP_TRY(call)                                                                    \
    do {                                                                                 \
        cudaError_t e__ = (call);                                                        \
        if (e__ != cudaSuccess) return ptp_internal_cuda_status(e__);                    \
    } while (0)

#define PTP_CHECK(expr)                                                                  \
    do {                                                                                 \
        ptp_status s__ = (expr);                                                         \
        if (s__ != PTP_OK) return s__;                                                   \
    } while (0)

ptp_status ptp_internal_cuda_status(cudaError_t e);

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------

struct ptp_mesh {
    int device;
    cudaStream_t stream;  // creating stream; the handle's memory is freed on it
    int64_t n, nf;
    float4 *pos;          // [n] xyz, w = 0
    int *row;             // [n + 1] corner offsets
    int2 *pairs;          // [3 nf] per corner: the other two vertices of the face,
                          //        in the face's cyclic order
    int4 *ring;           // [2 n] one-ring slots, original numbering (layout below)
    int *meta;            // [n]
    float4 *tgeom;        // ring geometry in the original numbering, built on the
    float4 *elen;         //   first multi-source call (NULL until then)
    double diameter;      // bounding-box diagonal
};

// Device control block of one distance run.
struct ptp_ctrl {
    unsigned long long bar[2];   // grid-barrier words (ptp_grid_sync)
    int status;                  // PTP_OK / PTP_ERR_NOT_CONVERGED / PTP_ERR_TIMEOUT
    int abort;                   // set by a CTA whose wait timed out
    long long iterations;        // K
    long long band_updates;      // sum_k |B_k minus S|
    unsigned long long active;   // recomputed vertex updates
    unsigned long long changed;  // updates that lowered d
    unsigned long long fp64;     // triangle solves taken in FP64
    long long checks;            // iterations that applied the test of Eq. lower_band
    // BFS running inside the window launch (ptp_distance_from_sources):
    unsigned long long pbar[2];  // barrier words of the BFS CTAs
    int tail;                    // BFS queue length so far
    int ready;                   // levels published: off[0 .. ready] and the queue entries,
                                 // records and iperm of V_0 .. V_{ready-1} are final
                                 // (PTP_LEVELS_DONE once the BFS has ended)
    unsigned long long cbar[2];  // barrier words of the copy CTAs (topleset order)
    int copied;                  // toplesets in place: V_0 .. V_{copied-1} copied into
                                 // topleset order (PTP_LEVELS_DONE once all are)
};

#define PTP_LEVELS_DONE 0x7fffffff

// One-ring slot layout of a renumbered vertex: its neighbours in cyclic
// order in ring[2u], ring[2u+1] (8 int32, -1 padded).  meta[u] holds the
// entry count m (low 4 bits), CLOSED for a closed fan (then the last entry
// repeats the first) and GENERAL for vertices not stored this way.  Triangle
// t of u is (u, ring[t], ring[t+1]) for t < m - 1.  GENERAL vertices (a link
// that is not one simple path or cycle, or one longer than the slot) are
// updated from the corner lists (row, pairs).
#define PTP_RING 8
#define PTP_META_CNT 0xF
#define PTP_META_CLOSED 0x10
#define PTP_META_GENERAL 0x20

// Static per-triangle geometry of the one-ring slots, precomputed in FP64
// and stored structure-of-arrays (component t of vertex u at [t * n + u]):
//   tgeom[t] = (b, L, alpha, beta) of triangle t = (u, ring[t], ring[t+1]):
//     e1 = x_ring[t] - x_u, e2 = x_ring[t+1] - x_u, a = |e1|^2, c = |e2|^2,
//     b = e1.e2, A = |e2 - e1|^2, L = sqrt(A), det = |e1 x e2|^2,
//     alpha = (a - b) / A, beta = sqrt(det) / A; beta < 0 marks a
//     near-degenerate triangle (some angle with sin^2 < 1e-6), solved in FP64
//     from the positions instead;
//   elen[0], elen[1] = |x_ring[t] - x_u| for t = 0..3 and 4..7.
#define PTP_TRI 7

struct ptp_toplesets_s {
    ptp_mesh *mesh;
    int device;
    cudaStream_t stream;
    int64_t n;
    int64_t ncorner;
    int *level;      // [n] original order, -1 = unreachable
    int *perm;       // [n] renumbered -> original
    int *iperm;      // [n] original -> renumbered
    int *off;        // [n + 2] topleset offsets in renumbered order, [0 .. rho]
    int *info;       // [4]: rho, n_reached, bfs status, number of unique sources
    float4 *pos;     // [n] renumbered positions
    int *row;        // [n + 1] renumbered corner offsets
    int2 *pairs;     // [3 nf] renumbered corner pairs
    int4 *ring;      // [2 n] one-ring slots (ring[u], ring[n + u])
    int *meta;       // [n]
    float4 *tgeom;   // [PTP_TRI n] per-triangle geometry, structure of arrays
    float4 *elen;    // [2 n] edge lengths to the ring neighbours
    ptp_ctrl *ctrl;  // control block of the last ptp_distance run
};

// Scratch of one multi-source run in the original vertex order (Voronoi, FPS).
struct ptp_multi_bufs {
    int n;
    int *level;                 // [n]
    int *queue;                 // [n] BFS queue: band position -> vertex
    int *off;                   // [n + 2]
    int *info;                  // [4]
    int *spill;                 // [2 n]
    int *cnt;                   // [16] BFS counters
    float *d0, *d1;             // [n] each
    int *nstamp, *chg;          // [n] each
    int *lab0, *lab1;           // [n] each, or NULL without labels
    ptp_ctrl *ctrl;
};

// ---------------------------------------------------------------------------
// Helpers shared by the translation units (host side)
// ---------------------------------------------------------------------------

// One-off kernel attributes (the BFS cluster kernel's shared memory); call
// before any stream capture.
ptp_status ptp_internal_prepare();
// Toplesets of the sources src[0 .. *m_dev) into b->level / queue / off / info
// (BFS queue order, no renumbering).  Resets the per-run BFS state itself.
ptp_status ptp_internal_bfs(const ptp_mesh *mesh, ptp_multi_bufs *b, const int *src, const int *m_dev, int m_max,
                            cudaStream_t s);
// Only the reset and V_0 of that BFS: level = -1 except the sources (0),
// queue[0 .. info[3]) = the unique sources.
ptp_status ptp_internal_bfs_seed(const ptp_mesh *mesh, ptp_multi_bufs *b, const int *src, const int *m_dev, int m_max,
                                 cudaStream_t s);
// Ring geometry of the mesh in the original numbering (cached in the mesh).
ptp_status ptp_internal_mesh_geometry(ptp_mesh *mesh, cudaStream_t s);
// Initialise distances (0 on the sources, which get labels 0..m-1) and run
// the window kernel over b->queue in the original order.
ptp_status ptp_internal_window_multi(const ptp_mesh *mesh, ptp_multi_bufs *b, const ptp_params *params,
                                     const int *src, const int *m_dev, int m_max, bool labels, cudaStream_t s);
// The same map with the BFS running inside the window launch
// (ptp_window<false, false, true>): seeds the sources, initialises the
// distances by position and launches; the last CTAs build the toplesets
// level by level into b->queue / off / level and rb->iperm while the others
// copy each level into topleset order (rb) and iterate on it.  The
// distances in b follow the positions (ptp_internal_fused_gather maps them
// back).  PTP_ERR_TOO_LARGE when the grid is too small to split: callers
// check ptp_internal_fused_producers first.
struct ptp_renum_bufs {
    float4 *pos;    // [n]
    int4 *ring;     // [2 n]
    int *meta;      // [n]
    float4 *tgeom;  // [PTP_TRI n]
    float4 *elen;   // [2 n]
    int *iperm;     // [n] original vertex -> position
    // learned multi-advance band (band_mode 2) only, else NULL:
    int *sched;                // [n + 8] schedule the launch infers, per topleset
    unsigned long long *facc;  // [PTP_FEAT_RING_WORDS] ring of per-topleset window-feature sums
};
// Words of that ring (64 toplesets x 8; ptp_schedule.cuh)
#define PTP_FEAT_RING_WORDS 512
// perm: the window runs in the original order (multi-source maps; with
// labels, Voronoi regions) and rb needs only meta, ring and iperm (the BFS
// records); otherwise the renumbered single-map path (d by position).
ptp_status ptp_internal_fused(const ptp_mesh *mesh, ptp_multi_bufs *b, const ptp_params *params, const int *src,
                              const int *m_dev, int m_max, bool perm, bool labels, const ptp_renum_bufs *rb,
                              cudaStream_t s);
// BFS CTAs a fused launch for m sources gets (0: the grid is too small).
int ptp_internal_fused_producers(const ptp_mesh *mesh, const ptp_params *params, int m, bool perm, bool labels);
// d_out (original order) from a fused run.
ptp_status ptp_internal_fused_gather(const ptp_mesh *mesh, const ptp_multi_bufs *b, const ptp_renum_bufs *rb,
                                     float *d_out, cudaStream_t s);
// The final distance (and label) buffer of the last window run in b.
__host__ __device__ inline int ptp_final_buffer(long long iterations) { return (int)(iterations & 1); }

int ptp_num_sms(int device);

// Stream-ordered allocation from the library's own memory pool of the
// current device (created on first use).  The pool keeps freed memory
// mapped, so repeated calls do not map and unmap their buffers every time;
// ptp_release_memory() returns it.  Freed with cudaFreeAsync.
cudaError_t ptp_malloc_async(void **p, size_t bytes, cudaStream_t s);

// Co-resident CTAs per SM of the single-map / batched window kernel
// launched with `block` threads; 0 when it cannot launch.
ptp_status ptp_internal_window_occupancy(int block, int *per_sm);
ptp_status ptp_internal_window_occupancy_batch(int block, int *per_sm);

// Device of a batch handle and its maps' vertex counts (sizes may be NULL).
ptp_status ptp_internal_batch_shape(const ptp_batch_t *batch, int *device, int *count, int64_t *sizes);

// Counts kernel launches issued by the library (ptp_kernel_launches).
void ptp_count_launches(int n);

// Exclusive scan of n int32 values: out[0..n] with out[n] = total.
// `tmp` must hold ptp_scan_tmp_ints(n) ints.
int64_t ptp_scan_tmp_ints(int64_t n);
ptp_status ptp_exclusive_scan(const int *in, int *out, int64_t n, int *tmp, cudaStream_t s);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// A wait gives up after this many SM clock cycles (about 4 s at 2 GHz), then
// flags PTP_ERR_TIMEOUT and the kernel returns.
#define PTP_WAIT_CYCLES 8000000000LL

__device__ __forceinline__ unsigned long long ptp_ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ptp_ld_acquire_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void ptp_st_release_s32(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ptp_atom_add_release_u64(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.release.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

// Grid-wide barrier for a co-resident (cooperative) grid that also sums one
// value per CTA.  Two 64-bit words alternate between epochs; each CTA adds
// 1 + (value << 32) with release semantics, and the low half counts
// arrivals.  A word is reused only two epochs later, which no CTA can reach
// before every CTA has left this epoch, so all CTAs read the same final
// word: its high half minus the high half seen at the word's previous use
// is the sum of this epoch's values.  `prev_hi` (two entries, thread 0 only)
// carries those previous high halves.  Returns the sum, or -1 when the wait
// timed out here (PTP_ERR_TIMEOUT is written to *status) or another CTA
// flagged an abort; the caller must then leave its loop.  epoch starts at 1.
// `parts` is the number of CTAs that take part (0: the whole grid);
// `limit` the wait's limit in SM clock cycles; `synced`: the caller has just
// passed a CTA barrier (e.g. __syncthreads_or) after its last writes, so the
// one on entry is skipped.
__device__ __forceinline__ long long ptp_grid_sync(unsigned long long *words, long long epoch, unsigned value,
                                                   int *abort_flag, int *status, unsigned long long *prev_hi,
                                                   unsigned parts = 0, long long limit = PTP_WAIT_CYCLES,
                                                   bool synced = false) {
    __shared__ long long result_s;
    if (!synced) __syncthreads();
    if (threadIdx.x == 0) {
        const int w = (int)(epoch & 1);
        unsigned long long *word = words + w;
        const unsigned target = (unsigned)((epoch + 1) >> 1) * (parts ? parts : gridDim.x);
        const unsigned long long add = 1ull + ((unsigned long long)value << 32);
        unsigned long long v = ptp_atom_add_release_u64(word, add) + add;
        long long res = 0;
        if ((unsigned)v < target) {
            const long long t0 = clock64();
            unsigned spins = 0;
            do {
                v = ptp_ld_acquire_u64(word);
                if ((unsigned)v >= target) break;
                if ((++spins & 63u) == 0) {
                    if (*(volatile int *)abort_flag) { res = -1; break; }
                    if (clock64() - t0 > limit) {
                        atomicExch(status, (int)PTP_ERR_TIMEOUT);
                        atomicExch(abort_flag, 1);
                        res = -1;
                        break;
                    }
                }
            } while (true);
        }
        if (res == 0) {
            const unsigned long long hi = v >> 32;
            res = (long long)(hi - prev_hi[w]);
            prev_hi[w] = hi;
        }
        result_s = res;
    }
    __syncthreads();
    return result_s;
}
