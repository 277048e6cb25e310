// Toplesets (Sec. 3.1, Definition: V_0 = S, V_r = the not yet visited
// neighbours of V_{r-1}) by a level-synchronous breadth-first search in one
// persistent cooperative kernel, and the renumbering of the mesh in topleset
// order (Sec. 3.3): the BFS queue itself is the new vertex order, so V_r
// occupies the index range [off[r], off[r+1]).  The renumbered mesh is also
// packed into fixed-size one-ring slots (cyclic neighbour order) for the
// window kernel.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ptp_internal.cuh"

namespace {

constexpr int BFS_THREADS = 512;

__global__ void bfs_seed(const int *__restrict__ src, int m, int *__restrict__ level, int *__restrict__ queue,
                         int *__restrict__ info, int *__restrict__ tail) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x) {
        const int v = src[s];
        if (atomicCAS(&level[v], -1, 0) == -1) {
            queue[atomicAdd(&info[3], 1)] = v;
            atomicAdd(tail, 1);
        }
    }
}

// Level-synchronous BFS.  Level r's frontier is queue[off[r] .. off[r+1]).
// One lane per frontier vertex: it loads its corners, then the levels of all
// corner vertices, then claims the unvisited ones (atomicCAS on level), all
// as independent loads / atomics in flight together.  A warp appends its
// claims with one atomicAdd on the queue tail, and the grid barrier returns
// the number of vertices added, i.e. the size of the next frontier.
__global__ void __launch_bounds__(BFS_THREADS) bfs_levels(const int *__restrict__ row, const int2 *__restrict__ pairs,
                                                          int *__restrict__ level, int *__restrict__ queue,
                                                          int *__restrict__ off, int *__restrict__ info,
                                                          unsigned long long *bar, int *tail, int *abort_flag) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int nwarps = (blockDim.x >> 5) * gridDim.x;
    __shared__ unsigned s_added;
    unsigned long long prev_hi[2] = {0ull, 0ull};
    int fbeg = 0;
    int fend = __ldcg(&info[3]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        off[0] = 0;
        off[1] = fend;
    }
    for (int r = 0;; ++r) {
        if (threadIdx.x == 0) s_added = 0;
        __syncthreads();
        const int base = fbeg & ~31;
        unsigned my_added = 0;
        for (int ch = gwarp;; ch += nwarps) {
            const int p0 = base + ch * 32;
            if (p0 >= fend) break;
            const int p = p0 + lane;
            const bool valid = p >= fbeg && p < fend;
            const int u = valid ? __ldcg(&queue[p]) : 0;
            const int cb = valid ? __ldg(row + u) : 0;
            const int deg = valid ? __ldg(row + u + 1) - cb : 0;
            int w[2 * PTP_RING];
            unsigned claimed = 0;
            if (deg <= PTP_RING) {
                int lv[2 * PTP_RING];
#pragma unroll
                for (int t = 0; t < PTP_RING; ++t) {
                    const int2 pr = t < deg ? __ldg(pairs + cb + t) : make_int2(0, 0);
                    w[2 * t] = pr.x;
                    w[2 * t + 1] = pr.y;
                }
#pragma unroll
                for (int t = 0; t < 2 * PTP_RING; ++t) lv[t] = t < 2 * deg ? __ldcg(level + w[t]) : 0;
#pragma unroll
                for (int t = 0; t < 2 * PTP_RING; ++t)
                    if (lv[t] < 0 && atomicCAS(&level[w[t]], -1, r + 1) == -1) claimed |= 1u << t;
            } else {
                // rare high-valence vertex: claim and append one at a time
                for (int c = cb; c < cb + deg; ++c) {
                    const int2 pr = __ldg(pairs + c);
                    const int ww[2] = {pr.x, pr.y};
                    for (int e = 0; e < 2; ++e)
                        if (__ldcg(level + ww[e]) < 0 && atomicCAS(&level[ww[e]], -1, r + 1) == -1) {
                            queue[atomicAdd(tail, 1)] = ww[e];
                            ++my_added;
                        }
                }
            }
            // warp-aggregated append of the claimed vertices
            const int cnt = __popc(claimed);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (total) {
                int at = 0;
                if (lane == 31) at = atomicAdd(tail, total);
                at = __shfl_sync(0xffffffffu, at, 31) + incl - cnt;
#pragma unroll
                for (int t = 0; t < 2 * PTP_RING; ++t)
                    if (claimed >> t & 1u) queue[at++] = w[t];
                if (lane == 0) my_added += (unsigned)total;
            }
        }
        if (my_added) atomicAdd(&s_added, my_added);
        __syncthreads();
        const long long added = ptp_grid_sync(bar, r + 1, s_added, abort_flag, &info[2], prev_hi);
        if (added < 0) return;
        if (added == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                info[0] = r + 1;  // rho
                info[1] = fend;   // reached
            }
            return;
        }
        fbeg = fend;
        fend += (int)added;
        if (blockIdx.x == 0 && threadIdx.x == 0) off[r + 2] = fend;
    }
}

// Append the vertices the BFS did not reach after the last topleset.
__global__ void append_unreached(const int *__restrict__ level, int n, int *__restrict__ queue,
                                 const int *__restrict__ info, int *__restrict__ counter) {
    const int lane = threadIdx.x & 31;
    const int reached = info[1];
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < n; base += gridDim.x * blockDim.x) {
        const int v = base + lane;
        const bool un = v < n && level[v] < 0;
        const unsigned bal = __ballot_sync(0xffffffffu, un);
        if (bal) {
            int at = 0;
            if (lane == 0) at = atomicAdd(counter, __popc(bal));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (un) queue[reached + at + __popc(bal & ((1u << lane) - 1u))] = v;
        }
    }
}

__global__ void invert_perm(const int *__restrict__ perm, int n, int *__restrict__ iperm, const float4 *__restrict__ pos,
                            float4 *__restrict__ npos, const int *__restrict__ row, int *__restrict__ ndeg) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int v = perm[u];
        iperm[v] = u;
        npos[u] = pos[v];
        ndeg[u] = row[v + 1] - row[v];
    }
}

__global__ void renumber_corners(const int *__restrict__ perm, const int *__restrict__ iperm, int n,
                                 const int *__restrict__ row, const int2 *__restrict__ pairs,
                                 const int *__restrict__ nrow, int2 *__restrict__ npairs) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int v = perm[u];
        const int cb = row[v], ce = row[v + 1], nb = nrow[u];
        for (int c = cb; c < ce; ++c) {
            const int2 pr = pairs[c];
            npairs[nb + (c - cb)] = make_int2(iperm[pr.x], iperm[pr.y]);
        }
    }
}

// Order each vertex's incident triangles into a fan.  The link of u (the
// edges {a, b} over its corners) must be one simple path (open fan, boundary
// vertex) or one simple cycle (closed fan).  The walk along it gives deg + 1
// entries r[0..deg]; for a cycle r[deg] == r[0], so in both cases triangle t
// is (u, r[t], r[t+1]) for t < deg.  Vertices whose walk does not fit in
// PTP_RING entries, or whose link is anything else (non-manifold, repeated
// faces), are marked GENERAL and use the corner lists instead.
__global__ void build_rings(int n, const int *__restrict__ nrow, const int2 *__restrict__ npairs, int4 *__restrict__ ring,
                            int *__restrict__ meta) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int cb = nrow[u];
        const int deg = nrow[u + 1] - cb;
        int r[PTP_RING];
#pragma unroll
        for (int q = 0; q < PTP_RING; ++q) r[q] = -1;
        int m = 0;
        if (deg + 1 > PTP_RING) {
            m = PTP_META_GENERAL;
        } else if (deg > 0) {
            int pa[PTP_RING], pb[PTP_RING];
            for (int q = 0; q < deg; ++q) {
                const int2 pr = npairs[cb + q];
                pa[q] = pr.x;
                pb[q] = pr.y;
            }
            bool bad = false, open = false;
            int start = 0, first = pa[0];
            for (int q = 0; q < deg && !bad; ++q) {
                for (int e = 0; e < 2; ++e) {
                    const int x = e ? pb[q] : pa[q];
                    int occ = 0;
                    for (int t = 0; t < deg; ++t) occ += (pa[t] == x) + (pb[t] == x);
                    if (occ > 2) bad = true;
                    if (occ == 1 && !open) {
                        open = true;
                        start = q;
                        first = x;
                    }
                }
            }
            if (!bad) {
                unsigned used = 1u << start;
                r[0] = first;
                r[1] = pa[start] == first ? pb[start] : pa[start];
                for (int step = 1; step < deg; ++step) {
                    const int last = r[step];
                    int found = -1;
                    for (int t = 0; t < deg; ++t)
                        if (!(used >> t & 1u) && (pa[t] == last || pb[t] == last)) { found = t; break; }
                    if (found < 0) { bad = true; break; }
                    used |= 1u << found;
                    r[step + 1] = pa[found] == last ? pb[found] : pa[found];
                }
            }
            if (!bad) {
                // distinct entries, except that a cycle closes on r[0]
                const int distinct = open ? deg + 1 : deg;
                if (!open && r[deg] != r[0]) bad = true;
                if (open && r[deg] == r[0]) bad = true;
                for (int a = 0; a < distinct && !bad; ++a)
                    for (int b = a + 1; b < distinct; ++b)
                        if (r[a] == r[b]) { bad = true; break; }
            }
            if (bad) {
                m = PTP_META_GENERAL;
#pragma unroll
                for (int q = 0; q < PTP_RING; ++q) r[q] = -1;
            } else {
                m = (deg + 1) | (open ? 0 : PTP_META_CLOSED);
            }
        }
        ring[u] = make_int4(r[0], r[1], r[2], r[3]);
        ring[n + u] = make_int4(r[4], r[5], r[6], r[7]);
        meta[u] = m;
    }
}


// Precompute the static geometry of every ring triangle in FP64 (see the
// layout comment in ptp_internal.cuh), so the window kernel's update step
// needs only the two neighbour distances per triangle.
__global__ void build_geometry(int n, const float4 *__restrict__ pos, const int4 *__restrict__ ring,
                               const int *__restrict__ meta, float4 *__restrict__ tgeom, float4 *__restrict__ elen) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int m = meta[u];
        const int4 r0 = ring[u], r1 = ring[n + u];
        const int ids[PTP_RING] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const int cnt = (m & PTP_META_GENERAL) ? 0 : (m & PTP_META_CNT);
        const float4 p0 = pos[u];
        double ex[PTP_RING], ey[PTP_RING], ez[PTP_RING];
        float el[PTP_RING];
        for (int t = 0; t < PTP_RING; ++t) {
            if (t < cnt) {
                const float4 p = pos[ids[t]];
                ex[t] = (double)p.x - p0.x;
                ey[t] = (double)p.y - p0.y;
                ez[t] = (double)p.z - p0.z;
                el[t] = (float)sqrt(ex[t] * ex[t] + ey[t] * ey[t] + ez[t] * ez[t]);
            } else {
                ex[t] = ey[t] = ez[t] = 0.0;
                el[t] = 0.0f;
            }
        }
        elen[u] = make_float4(el[0], el[1], el[2], el[3]);
        elen[n + u] = make_float4(el[4], el[5], el[6], el[7]);
        for (int t = 0; t < PTP_TRI; ++t) {
            float4 g = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
            if (t < cnt - 1) {
                const double a = ex[t] * ex[t] + ey[t] * ey[t] + ez[t] * ez[t];
                const double c = ex[t + 1] * ex[t + 1] + ey[t + 1] * ey[t + 1] + ez[t + 1] * ez[t + 1];
                const double b = ex[t] * ex[t + 1] + ey[t] * ey[t + 1] + ez[t] * ez[t + 1];
                const double fx = ex[t + 1] - ex[t], fy = ey[t + 1] - ey[t], fz = ez[t + 1] - ez[t];
                const double A = fx * fx + fy * fy + fz * fz;
                const double cx = ey[t] * ez[t + 1] - ez[t] * ey[t + 1];
                const double cy = ez[t] * ex[t + 1] - ex[t] * ez[t + 1];
                const double cz = ex[t] * ey[t + 1] - ey[t] * ex[t + 1];
                const double det = cx * cx + cy * cy + cz * cz;
                const double big = fmax(a * c, A * fmax(a, c));
                const double amb = -(ex[t] * fx + ey[t] * fy + ez[t] * fz);  // a - b
                if (A > 0.0 && det >= 1e-6 * big)
                    g = make_float4((float)b, (float)sqrt(A), (float)(amb / A), (float)(sqrt(det) / A));
                else
                    g = make_float4((float)b, (float)sqrt(A), 0.0f, -1.0f);
            }
            tgeom[(size_t)t * n + u] = g;
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

extern "C" ptp_status ptp_toplesets(ptp_mesh *mesh, const int32_t *sources, int32_t m, int ptr_kind, void *stream,
                                    ptp_toplesets_t **out) {
    if (!out) return PTP_ERR_ARG;
    *out = nullptr;
    if (!mesh || !sources || m < 1 || (ptr_kind != PTP_HOST && ptr_kind != PTP_DEVICE)) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = mesh->n;
    const int dev = mesh->device;

    // validate the sources on the host
    std::vector<int32_t> hsrc((size_t)m);
    if (ptr_kind == PTP_DEVICE) {
        PTP_TRY(cudaMemcpyAsync(hsrc.data(), sources, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
        PTP_TRY(cudaStreamSynchronize(s));
    } else {
        memcpy(hsrc.data(), sources, sizeof(int32_t) * m);
    }
    for (int32_t q = 0; q < m; ++q)
        if (hsrc[q] < 0 || hsrc[q] >= n) return PTP_ERR_INDEX;

    ptp_toplesets_t *t = (ptp_toplesets_t *)calloc(1, sizeof(ptp_toplesets_t));
    if (!t) return PTP_ERR_NOMEM;
    t->mesh = mesh;
    t->device = dev;
    t->stream = s;
    t->n = n;
    t->ncorner = 3 * mesh->nf;

    int *work = nullptr, *src_d = nullptr;
    ptp_status st = PTP_OK;
    cudaError_t ce = cudaSuccess;
#define TOPS_TRY(call)                                   \
    do {                                                 \
        ce = (call);                                     \
        if (ce != cudaSuccess) {                         \
            st = ptp_internal_cuda_status(ce);           \
            goto fail;                                   \
        }                                                \
    } while (0)
    {
        TOPS_TRY(cudaMallocAsync((void **)&t->level, sizeof(int) * n, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->perm, sizeof(int) * n, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->iperm, sizeof(int) * n, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->off, sizeof(int) * (n + 2), s));
        TOPS_TRY(cudaMallocAsync((void **)&t->info, sizeof(int) * 4, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->pos, sizeof(float4) * n, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->row, sizeof(int) * (n + 1), s));
        TOPS_TRY(cudaMallocAsync((void **)&t->pairs, sizeof(int2) * t->ncorner, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->ring, sizeof(int4) * 2 * n, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->meta, sizeof(int) * n, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->tgeom, sizeof(float4) * PTP_TRI * n, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->elen, sizeof(float4) * 2 * n, s));
        TOPS_TRY(cudaMallocAsync((void **)&t->ctrl, sizeof(ptp_ctrl), s));
        // work: [0..n) degree in new order, then scan temp, then bfs counters
        const int64_t scan_tmp = ptp_scan_tmp_ints(n);
        TOPS_TRY(cudaMallocAsync((void **)&work, sizeof(int) * (n + scan_tmp + 16), s));
        // counters first so the 64-bit barrier words are 8-byte aligned:
        // [0] queue tail, [3] abort, [4] unreached counter, [8..11] barrier words
        int *bfs_cnt = work;
        unsigned long long *bfs_bar = (unsigned long long *)(bfs_cnt + 8);
        int *ndeg = work + 16;
        int *tmp = ndeg + n;

        TOPS_TRY(cudaMallocAsync((void **)&src_d, sizeof(int) * m, s));
        TOPS_TRY(cudaMemcpyAsync(src_d, hsrc.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
        TOPS_TRY(cudaMemsetAsync(t->level, 0xFF, sizeof(int) * n, s));
        TOPS_TRY(cudaMemsetAsync(t->info, 0, sizeof(int) * 4, s));
        TOPS_TRY(cudaMemsetAsync(t->off, 0, sizeof(int) * (n + 2), s));
        TOPS_TRY(cudaMemsetAsync(bfs_cnt, 0, sizeof(int) * 16, s));
        TOPS_TRY(cudaMemsetAsync(t->ctrl, 0, sizeof(ptp_ctrl), s));
        bfs_seed<<<blocks_for(m, 256, dev), 256, 0, s>>>(src_d, m, t->level, t->perm, t->info, bfs_cnt);
        ptp_count_launches(1);
        TOPS_TRY(cudaGetLastError());

        // persistent BFS: every CTA co-resident
        int per_sm = 0;
        TOPS_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_levels, BFS_THREADS, 0));
        if (per_sm < 1) { st = PTP_ERR_CUDA; goto fail; }
        int nblk = per_sm * ptp_num_sms(dev);
        {
            const int *row_c = mesh->row;
            const int2 *pairs_c = mesh->pairs;
            int *tail = bfs_cnt;
            int *abort_flag = bfs_cnt + 3;
            void *args[] = {(void *)&row_c, (void *)&pairs_c, (void *)&t->level, (void *)&t->perm, (void *)&t->off,
                            (void *)&t->info, (void *)&bfs_bar, (void *)&tail, (void *)&abort_flag};
            TOPS_TRY(cudaLaunchCooperativeKernel((const void *)bfs_levels, dim3(nblk), dim3(BFS_THREADS), args, 0, s));
            ptp_count_launches(1);
        }
        append_unreached<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->level, (int)n, t->perm, t->info, bfs_cnt + 4);
        invert_perm<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->perm, (int)n, t->iperm, mesh->pos, t->pos, mesh->row, ndeg);
        ptp_count_launches(2);
        TOPS_TRY(cudaGetLastError());
        st = ptp_exclusive_scan(ndeg, t->row, n, tmp, s);
        if (st != PTP_OK) goto fail;
        renumber_corners<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->perm, t->iperm, (int)n, mesh->row, mesh->pairs, t->row,
                                                                t->pairs);
        build_rings<<<blocks_for(n, 128, dev), 128, 0, s>>>((int)n, t->row, t->pairs, t->ring, t->meta);
        build_geometry<<<blocks_for(n, 128, dev), 128, 0, s>>>((int)n, t->pos, t->ring, t->meta, t->tgeom, t->elen);
        ptp_count_launches(3);
        TOPS_TRY(cudaGetLastError());
        cudaFreeAsync(work, s);
        cudaFreeAsync(src_d, s);
    }
    *out = t;
    return PTP_OK;
fail:
    if (work) cudaFreeAsync(work, s);
    if (src_d) cudaFreeAsync(src_d, s);
    {
        void *ptrs[] = {t->level, t->perm, t->iperm, t->off, t->info, t->pos, t->row, t->pairs, t->ring, t->meta,
                        t->tgeom, t->elen, t->ctrl};
        for (void *p : ptrs)
            if (p) cudaFreeAsync(p, s);
    }
    cudaStreamSynchronize(s);
    free(t);
    return st;
#undef TOPS_TRY
}

extern "C" ptp_status ptp_toplesets_info(ptp_toplesets_t *t, void *stream, int32_t *rho, int32_t *n_reached,
                                         const int32_t **off_dev, const int32_t **perm_dev) {
    if (!t) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int h[4] = {0, 0, 0, 0};
    PTP_TRY(cudaMemcpyAsync(h, t->info, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    PTP_TRY(cudaStreamSynchronize(s));
    if (rho) *rho = h[0];
    if (n_reached) *n_reached = h[1];
    if (off_dev) *off_dev = t->off;
    if (perm_dev) *perm_dev = t->perm;
    return h[2] != 0 ? (ptp_status)h[2] : PTP_OK;
}

extern "C" ptp_status ptp_toplesets_destroy(ptp_toplesets_t *t) {
    if (!t) return PTP_ERR_ARG;
    void *ptrs[] = {t->level, t->perm, t->iperm, t->off, t->info, t->pos, t->row, t->pairs, t->ring, t->meta,
                    t->tgeom, t->elen, t->ctrl};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, t->stream);
    const cudaError_t e = cudaStreamSynchronize(t->stream);
    free(t);
    return e == cudaSuccess ? PTP_OK : ptp_internal_cuda_status(e);
}
