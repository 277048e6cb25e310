// Toplesets (Sec. 4.1, Definition: V_0 = S, V_r = the not yet visited
// neighbours of V_{r-1}) by a level-synchronous breadth-first search inside
// one thread-block cluster, and the renumbering of the mesh in topleset
// order (Sec. 4.3): the BFS queue itself is the new vertex order, so V_r
// occupies the index range [off[r], off[r+1]).  The renumbered mesh gets
// one-ring slots (remapped from the mesh's), corner lists for the vertices
// that have no slot, and the precomputed geometry of every ring triangle.
#include <cooperative_groups.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ptp_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int BC_CLUSTER = 8;     // CTAs in the BFS cluster (portable maximum)
constexpr int BC_THREADS = 1024;  // threads per CTA
constexpr int BC_CAP = 12288;     // frontier entries per CTA list (two lists: 96 KiB)

// V_0: claim the sources (duplicates once).  The count is m, or *m_dev when
// m_dev is given (device-side source lists, e.g. farthest-point sampling).
__global__ void bfs_seed(const int *__restrict__ src, int m, const int *__restrict__ m_dev, int *__restrict__ level,
                         int *__restrict__ queue, int *__restrict__ info) {
    if (m_dev) m = *m_dev;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x) {
        const int v = src[s];
        if (atomicCAS(&level[v], -1, 0) == -1) queue[atomicAdd(&info[3], 1)] = v;
    }
}

// Level-synchronous BFS in one cluster.  Level r's frontier is V_r, held as
// the concatenation of the CTAs' lists in shared memory (level 0 and any
// overflow are in global memory).  Frontier entries are dealt out in groups
// of 32 to warps interleaved across the CTAs, so every SM shares the work
// whichever CTA discovered the entries; a lane reads its entry from the
// owner's list through distributed shared memory, writes it to its
// renumbered position queue[off[r] + t], loads the vertex's one-ring slot,
// reads its neighbours' levels and claims the unvisited ones with
// atomicCAS; claimed vertices (V_{r+1}) are appended to the lane's own CTA
// list.  After the hardware cluster barrier every CTA reads all list
// lengths through distributed shared memory; their prefix sums locate the
// next level's entries.
__global__ void __cluster_dims__(BC_CLUSTER, 1, 1) __launch_bounds__(BC_THREADS, 1)
    bfs_cluster(const int4 *__restrict__ ring, const int *__restrict__ meta, const int *__restrict__ row,
                const int2 *__restrict__ pairs, int n, int *__restrict__ level, int *__restrict__ queue,
                int *__restrict__ off, int *__restrict__ info, int *__restrict__ spill, int *__restrict__ spill_cnt) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ int s_list[];  // [2][BC_CAP]
    __shared__ int s_cnt[2];
    __shared__ int s_pref[BC_CLUSTER + 1];
    __shared__ int s_spill;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwarps_cl = BC_CLUSTER * (BC_THREADS / 32);
    const int gw = wid * BC_CLUSTER + rank;  // warps interleaved across the CTAs
    const bool leader = rank == 0 && threadIdx.x == 0;
    int fbeg = 0;
    int total = __ldcg(&info[3]);  // V_0 = the unique sources, queue[0, m0)
    int nsmem = 0;                 // frontier entries held in the CTAs' lists
    if (leader) {
        off[0] = 0;
        off[1] = total;
        spill_cnt[0] = spill_cnt[1] = spill_cnt[2] = 0;
    }
    if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0;
    cl.sync();
    for (int r = 0;; ++r) {
        const int b = r & 1;  // V_{r+1} goes to list b; V_r (r >= 1) is in list b ^ 1
        if (threadIdx.x == 0) s_cnt[b] = 0;
        if (leader) spill_cnt[(r + 1) % 3] = 0;  // last read before the previous barrier
        __syncthreads();
        const int *spill_in = spill + (size_t)(b ^ 1) * n;
        int *spill_out = spill + (size_t)b * n;
        int *lst_out = s_list + b * BC_CAP;
        const int steps = (total + 32 * nwarps_cl - 1) / (32 * nwarps_cl);
        for (int step = 0; step < steps; ++step) {
            const int t = (step * nwarps_cl + gw) * 32 + lane;
            int u = -1;
            if (t < total) {
                if (r == 0) {
                    u = __ldcg(&queue[t]);  // the sources are already in place
                } else {
                    if (t < nsmem) {
                        int q = 0;
                        while (q + 1 < BC_CLUSTER && s_pref[q + 1] <= t) ++q;
                        const int *lst = cl.map_shared_rank(s_list + (b ^ 1) * BC_CAP, q);
                        u = lst[t - s_pref[q]];
                    } else {
                        u = __ldcg(&spill_in[t - nsmem]);
                    }
                    queue[fbeg + t] = u;  // renumbered position of u
                }
            }
            int w[PTP_RING];
            unsigned claimed = 0;
            const int m = u >= 0 ? __ldg(meta + u) : PTP_META_GENERAL;
            const int4 r0 = u >= 0 ? __ldg(ring + u) : make_int4(-1, -1, -1, -1);
            const int4 r1 = u >= 0 ? __ldg(ring + n + u) : make_int4(-1, -1, -1, -1);
            if (u >= 0 && !(m & PTP_META_GENERAL)) {
                const int ids[PTP_RING] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                const int cnt = m & PTP_META_CNT;
                // read the neighbours' levels first (plain loads, all in
                // flight), then claim only the unvisited ones
                int lv[PTP_RING];
#pragma unroll
                for (int q = 0; q < PTP_RING; ++q) {
                    w[q] = ids[q];
                    lv[q] = q < cnt ? __ldcg(&level[ids[q]]) : 0;
                }
                int old[PTP_RING];
#pragma unroll
                for (int q = 0; q < PTP_RING; ++q) old[q] = lv[q] < 0 ? atomicCAS(&level[ids[q]], -1, r + 1) : 0;
#pragma unroll
                for (int q = 0; q < PTP_RING; ++q)
                    if (lv[q] < 0 && old[q] == -1) claimed |= 1u << q;
            } else if (u >= 0) {
                // vertex without a ring slot: claim from its corner list, one at a time
                const int cb = __ldg(row + u), ce = __ldg(row + u + 1);
                for (int c = cb; c < ce; ++c) {
                    const int2 pr = __ldg(pairs + c);
                    const int ww[2] = {pr.x, pr.y};
                    for (int e = 0; e < 2; ++e) {
                        if (atomicCAS(&level[ww[e]], -1, r + 1) == -1) {
                            const int at = atomicAdd(&s_cnt[b], 1);
                            if (at < BC_CAP) lst_out[at] = ww[e];
                            else spill_out[atomicAdd(&spill_cnt[r % 3], 1)] = ww[e];
                        }
                    }
                }
            }
            // append the claimed ring neighbours, one shared atomic per warp
            const int cntc = __popc(claimed);
            int incl = cntc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int wtot = __shfl_sync(0xffffffffu, incl, 31);
            if (wtot) {
                int at = 0;
                if (lane == 31) at = atomicAdd(&s_cnt[b], wtot);
                at = __shfl_sync(0xffffffffu, at, 31) + incl - cntc;
#pragma unroll
                for (int q = 0; q < PTP_RING; ++q) {
                    if (claimed >> q & 1u) {
                        if (at < BC_CAP) lst_out[at] = w[q];
                        else spill_out[atomicAdd(&spill_cnt[r % 3], 1)] = w[q];
                        ++at;
                    }
                }
            }
        }
        cl.sync();  // V_{r+1} complete in the lists and the spill buffer
        if (threadIdx.x < 32) {
            // one lane per cluster CTA reads its list length (distributed shared memory)
            const int c = lane < BC_CLUSTER ? *cl.map_shared_rank(&s_cnt[b], lane) : 0;
            const int over = __any_sync(0xffffffffu, c > BC_CAP);
            int incl = c < BC_CAP ? c : BC_CAP;
#pragma unroll
            for (int o = 1; o < BC_CLUSTER; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane < BC_CLUSTER) s_pref[lane + 1] = incl;
            if (lane == 0) {
                s_pref[0] = 0;
                s_spill = over ? __ldcg(&spill_cnt[r % 3]) : 0;
            }
        }
        __syncthreads();
        const int next = s_pref[BC_CLUSTER] + s_spill;
        if (next == 0) {
            if (leader) {
                info[0] = r + 1;          // rho
                info[1] = fbeg + total;   // reached
            }
            break;
        }
        fbeg += total;
        total = next;
        nsmem = s_pref[BC_CLUSTER];
        if (leader) off[r + 2] = fbeg + total;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
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

__global__ void invert_perm(const int *__restrict__ perm, int n, int *__restrict__ iperm) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) iperm[perm[u]] = u;
}

// Renumbered positions, one-ring slots (ids remapped) and metadata; corner
// counts only for the vertices without a slot (their corner lists are kept).
__global__ void renumber_vertices(const int *__restrict__ perm, const int *__restrict__ iperm, int n,
                                  const float4 *__restrict__ pos, const int4 *__restrict__ ring,
                                  const int *__restrict__ meta, const int *__restrict__ row, float4 *__restrict__ npos,
                                  int4 *__restrict__ nring, int *__restrict__ nmeta, int *__restrict__ ndeg) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int v = perm[u];
        npos[u] = pos[v];
        const int m = meta[v];
        nmeta[u] = m;
        const int4 r0 = ring[v], r1 = ring[n + v];
        const int cnt = (m & PTP_META_GENERAL) ? 0 : (m & PTP_META_CNT);
        auto mp = [&](int q, int x) { return q < cnt ? iperm[x] : -1; };
        nring[u] = make_int4(mp(0, r0.x), mp(1, r0.y), mp(2, r0.z), mp(3, r0.w));
        nring[n + u] = make_int4(mp(4, r1.x), mp(5, r1.y), mp(6, r1.z), mp(7, r1.w));
        ndeg[u] = (m & PTP_META_GENERAL) ? row[v + 1] - row[v] : 0;
    }
}

__global__ void renumber_corners(const int *__restrict__ perm, const int *__restrict__ iperm, int n,
                                 const int *__restrict__ row, const int2 *__restrict__ pairs,
                                 const int *__restrict__ nrow, int2 *__restrict__ npairs) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int nb = nrow[u];
        if (nrow[u + 1] == nb) continue;
        const int v = perm[u];
        const int cb = row[v], ce = row[v + 1];
        for (int c = cb; c < ce; ++c) {
            const int2 pr = pairs[c];
            npairs[nb + (c - cb)] = make_int2(iperm[pr.x], iperm[pr.y]);
        }
    }
}

// Precompute the static geometry of every ring triangle (see the layout
// comment in ptp_internal.cuh), so the window kernel's update step needs only
// the two neighbour distances per triangle.  Edge vectors are FP32
// differences of nearby coordinates; the dot products, the cross product
// and the derived terms are FP32, accurate to a few ulps for triangles that
// are not near-degenerate (the update's own result is rounded to FP32
// anyway); triangles close to the degeneracy threshold are classified in
// FP64.
__global__ void build_geometry(int n, const float4 *__restrict__ pos, const int4 *__restrict__ ring,
                               const int *__restrict__ meta, float4 *__restrict__ tgeom, float4 *__restrict__ elen) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int m = meta[u];
        const int4 r0 = ring[u], r1 = ring[n + u];
        const int ids[PTP_RING] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const int cnt = (m & PTP_META_GENERAL) ? 0 : (m & PTP_META_CNT);
        const float4 p0 = pos[u];
        float3 e[PTP_RING];
        float el[PTP_RING];
#pragma unroll
        for (int t = 0; t < PTP_RING; ++t) {
            if (t < cnt) {
                const float4 p = pos[ids[t]];
                e[t] = make_float3(p.x - p0.x, p.y - p0.y, p.z - p0.z);
                el[t] = sqrtf(e[t].x * e[t].x + e[t].y * e[t].y + e[t].z * e[t].z);
            } else {
                e[t] = make_float3(0.0f, 0.0f, 0.0f);
                el[t] = 0.0f;
            }
        }
        elen[u] = make_float4(el[0], el[1], el[2], el[3]);
        elen[n + u] = make_float4(el[4], el[5], el[6], el[7]);
#pragma unroll
        for (int t = 0; t < PTP_TRI; ++t) {
            float4 g = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
            if (t < cnt - 1) {
                const float3 e1 = e[t], e2 = e[t + 1];
                const float3 f = make_float3(e2.x - e1.x, e2.y - e1.y, e2.z - e1.z);
                const float a = e1.x * e1.x + e1.y * e1.y + e1.z * e1.z;
                const float c = e2.x * e2.x + e2.y * e2.y + e2.z * e2.z;
                const float b = e1.x * e2.x + e1.y * e2.y + e1.z * e2.z;
                const float A = f.x * f.x + f.y * f.y + f.z * f.z;
                const float cx = e1.y * e2.z - e1.z * e2.y, cy = e1.z * e2.x - e1.x * e2.z, cz = e1.x * e2.y - e1.y * e2.x;
                const float det = cx * cx + cy * cy + cz * cz;
                const float big = fmaxf(a * c, A * fmaxf(a, c));
                bool ok = A > 0.0f && det >= 1e-6f * big;
                if (A > 0.0f && det < 1e-4f * big) {
                    // close to the threshold: decide it in FP64
                    const double dx = (double)e1.y * e2.z - (double)e1.z * e2.y;
                    const double dy = (double)e1.z * e2.x - (double)e1.x * e2.z;
                    const double dz = (double)e1.x * e2.y - (double)e1.y * e2.x;
                    const double dd = dx * dx + dy * dy + dz * dz;
                    const double ad = (double)e1.x * e1.x + (double)e1.y * e1.y + (double)e1.z * e1.z;
                    const double cd = (double)e2.x * e2.x + (double)e2.y * e2.y + (double)e2.z * e2.z;
                    const double fx = (double)e2.x - e1.x, fy = (double)e2.y - e1.y, fz = (double)e2.z - e1.z;
                    const double Ad = fx * fx + fy * fy + fz * fz;
                    ok = dd >= 1e-6 * fmax(ad * cd, Ad * fmax(ad, cd));
                }
                const float amb = -(e1.x * f.x + e1.y * f.y + e1.z * f.z);  // a - b
                const float L = sqrtf(A);
                g = ok ? make_float4(b, L, amb / A, sqrtf(det) / A) : make_float4(b, L, 0.0f, -1.0f);
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

ptp_status ptp_internal_prepare() {
    PTP_TRY(cudaFuncSetAttribute(bfs_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(int) * 2 * BC_CAP)));
    return PTP_OK;
}

ptp_status ptp_internal_bfs_seed(const ptp_mesh *mesh, ptp_multi_bufs *b, const int *src, const int *m_dev, int m_max,
                                 cudaStream_t s) {
    const int n = b->n;
    PTP_TRY(cudaMemsetAsync(b->level, 0xFF, sizeof(int) * n, s));
    PTP_TRY(cudaMemsetAsync(b->info, 0, sizeof(int) * 4, s));
    PTP_TRY(cudaMemsetAsync(b->cnt, 0, sizeof(int) * 16, s));
    bfs_seed<<<blocks_for(m_max, 256, mesh->device), 256, 0, s>>>(src, m_max, m_dev, b->level, b->queue, b->info);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

ptp_status ptp_internal_bfs(const ptp_mesh *mesh, ptp_multi_bufs *b, const int *src, const int *m_dev, int m_max,
                            cudaStream_t s) {
    const int n = b->n;
    PTP_CHECK(ptp_internal_bfs_seed(mesh, b, src, m_dev, m_max, s));
    bfs_cluster<<<BC_CLUSTER, BC_THREADS, sizeof(int) * 2 * BC_CAP, s>>>(mesh->ring, mesh->meta, mesh->row, mesh->pairs,
                                                                         n, b->level, b->queue, b->off, b->info, b->spill,
                                                                         b->cnt);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

ptp_status ptp_internal_mesh_geometry(ptp_mesh *mesh, cudaStream_t s) {
    if (mesh->tgeom) return PTP_OK;
    const int64_t n = mesh->n;
    float4 *tg = nullptr, *el = nullptr;
    PTP_TRY(ptp_malloc_async((void **)&tg, sizeof(float4) * PTP_TRI * n, s));
    cudaError_t e = ptp_malloc_async((void **)&el, sizeof(float4) * 2 * n, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(tg, s);
        return ptp_internal_cuda_status(e);
    }
    build_geometry<<<blocks_for(n, 128, mesh->device), 128, 0, s>>>((int)n, mesh->pos, mesh->ring, mesh->meta, tg, el);
    ptp_count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(tg, s);
        cudaFreeAsync(el, s);
        return ptp_internal_cuda_status(e);
    }
    mesh->tgeom = tg;
    mesh->elen = el;
    return PTP_OK;
}

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
        TOPS_TRY(ptp_malloc_async((void **)&t->level, sizeof(int) * n, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->perm, sizeof(int) * n, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->iperm, sizeof(int) * n, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->off, sizeof(int) * (n + 2), s));
        TOPS_TRY(ptp_malloc_async((void **)&t->info, sizeof(int) * 4, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->pos, sizeof(float4) * n, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->row, sizeof(int) * (n + 1), s));
        TOPS_TRY(ptp_malloc_async((void **)&t->ring, sizeof(int4) * 2 * n, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->meta, sizeof(int) * n, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->tgeom, sizeof(float4) * PTP_TRI * n, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->elen, sizeof(float4) * 2 * n, s));
        TOPS_TRY(ptp_malloc_async((void **)&t->ctrl, sizeof(ptp_ctrl), s));
        // work: counters [0..15], degrees [n], scan temp, BFS spill lists [2n]
        const int64_t scan_tmp = ptp_scan_tmp_ints(n);
        TOPS_TRY(ptp_malloc_async((void **)&work, sizeof(int) * (16 + n + scan_tmp + 2 * n), s));
        int *cnt = work;  // [0..2] spill counters, [4] unreached counter
        int *ndeg = work + 16;
        int *tmp = ndeg + n;
        int *spill = tmp + scan_tmp;

        TOPS_TRY(ptp_malloc_async((void **)&src_d, sizeof(int) * m, s));
        TOPS_TRY(cudaMemcpyAsync(src_d, hsrc.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
        TOPS_TRY(cudaMemsetAsync(t->level, 0xFF, sizeof(int) * n, s));
        TOPS_TRY(cudaMemsetAsync(t->info, 0, sizeof(int) * 4, s));
        TOPS_TRY(cudaMemsetAsync(t->off, 0, sizeof(int) * (n + 2), s));
        TOPS_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * 16, s));
        TOPS_TRY(cudaMemsetAsync(t->ctrl, 0, sizeof(ptp_ctrl), s));
        bfs_seed<<<blocks_for(m, 256, dev), 256, 0, s>>>(src_d, m, nullptr, t->level, t->perm, t->info);
        ptp_count_launches(1);
        TOPS_TRY(cudaGetLastError());
        {
            const size_t smem = sizeof(int) * 2 * BC_CAP;
            st = ptp_internal_prepare();
            if (st != PTP_OK) goto fail;
            bfs_cluster<<<BC_CLUSTER, BC_THREADS, smem, s>>>(mesh->ring, mesh->meta, mesh->row, mesh->pairs, (int)n,
                                                             t->level, t->perm, t->off, t->info, spill, cnt);
            ptp_count_launches(1);
            TOPS_TRY(cudaGetLastError());
        }
        append_unreached<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->level, (int)n, t->perm, t->info, cnt + 4);
        invert_perm<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->perm, (int)n, t->iperm);
        renumber_vertices<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->perm, t->iperm, (int)n, mesh->pos, mesh->ring,
                                                                 mesh->meta, mesh->row, t->pos, t->ring, t->meta, ndeg);
        ptp_count_launches(3);
        TOPS_TRY(cudaGetLastError());
        st = ptp_exclusive_scan(ndeg, t->row, n, tmp, s);
        if (st != PTP_OK) goto fail;
        // corner lists, filled only for the vertices without a ring slot
        TOPS_TRY(ptp_malloc_async((void **)&t->pairs, sizeof(int2) * t->ncorner, s));
        renumber_corners<<<blocks_for(n, 256, dev), 256, 0, s>>>(t->perm, t->iperm, (int)n, mesh->row, mesh->pairs,
                                                                t->row, t->pairs);
        build_geometry<<<blocks_for(n, 128, dev), 128, 0, s>>>((int)n, t->pos, t->ring, t->meta, t->tgeom, t->elen);
        ptp_count_launches(2);
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
