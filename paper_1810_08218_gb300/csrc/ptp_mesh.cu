// Mesh construction: validation, the vertex -> incident-triangle lists
// ("corner lists"), the one-ring slots (fans in cyclic order), positions and
// the bounding-box diameter.  The paper keeps the mesh as a compact half-edge
// structure (Sec. 4.3); the update step only needs, per vertex, the
// triangles around it, which is what this builds.
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "ptp_internal.cuh"

ptp_status ptp_internal_cuda_status(cudaError_t e) {
    cudaGetLastError();  // clear a sticky launch error so later calls can proceed
    return e == cudaErrorMemoryAllocation ? PTP_ERR_NOMEM : PTP_ERR_CUDA;
}

extern "C" const char *ptp_status_str(ptp_status s) {
    switch (s) {
        case PTP_OK: return "PTP_OK";
        case PTP_ERR_ARG: return "PTP_ERR_ARG";
        case PTP_ERR_INDEX: return "PTP_ERR_INDEX";
        case PTP_ERR_DEGENERATE_FACE: return "PTP_ERR_DEGENERATE_FACE";
        case PTP_ERR_CUDA: return "PTP_ERR_CUDA";
        case PTP_ERR_NOT_CONVERGED: return "PTP_ERR_NOT_CONVERGED";
        case PTP_ERR_TIMEOUT: return "PTP_ERR_TIMEOUT";
        case PTP_ERR_NOMEM: return "PTP_ERR_NOMEM";
        case PTP_ERR_TOO_LARGE: return "PTP_ERR_TOO_LARGE";
    }
    return "PTP_ERR_UNKNOWN";
}

extern "C" ptp_status ptp_params_default(ptp_params *p) {
    if (!p) return PTP_ERR_ARG;
    p->eps = 1e-3;
    p->eps_abs = 0.0;
    p->max_iter = 0;
    p->block = 0;
    p->grid = 0;
    p->band_mode = 0;
    p->reserved = 0;
    p->trace = nullptr;
    p->trace_cap = 0;
    p->ev_begin = nullptr;
    p->ev_end = nullptr;
    p->schedule = nullptr;
    p->mlp_half = nullptr;
    p->mlp_margin = 0.0f;
    p->reserved2 = 0;
    p->conv_trace = nullptr;
    return PTP_OK;
}

static unsigned long long g_launches = 0;

void ptp_count_launches(int n) { __atomic_fetch_add(&g_launches, (unsigned long long)(long long)n, __ATOMIC_RELAXED); }

extern "C" int64_t ptp_kernel_launches(void) { return (int64_t)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int ptp_num_sms(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}

namespace {

constexpr int POOL_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[POOL_DEVICES] = {};

}  // namespace

cudaError_t ptp_malloc_async(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= POOL_DEVICES) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pools[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            e = cudaMemPoolCreate(&np, &props);
            if (e != cudaSuccess) return e;
            unsigned long long keep = ~0ull;  // keep freed memory until ptp_release_memory
            e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(np);
                return e;
            }
            g_pools[dev] = np;
        }
        pool = g_pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

extern "C" ptp_status ptp_release_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d = 0; d < POOL_DEVICES; ++d) {
        if (!g_pools[d]) continue;
        const cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
        if (e != cudaSuccess) return ptp_internal_cuda_status(e);
    }
    return PTP_OK;
}

// ---------------------------------------------------------------------------
// Exclusive scan (three passes: tile sums, scan of the tile sums, tiles)
// ---------------------------------------------------------------------------

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int block_exclusive_scan(int v, int *excl) {
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    const int before = wid > 0 ? warp_tot[wid - 1] : 0;
    *excl = before + x - v;
    const int total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_sums(const int *__restrict__ in, int64_t n,
                                                               int *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q)
        if (base + q < n) s += in[base + q];
    int excl;
    const int tot = block_exclusive_scan(s, &excl);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One CTA scans the tile sums in place (exclusive), in chunks of SCAN_THREADS.
__global__ void __launch_bounds__(SCAN_THREADS) scan_sums(int *sums, int64_t nt) {
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t b = 0; b < nt; b += SCAN_THREADS) {
        const int64_t idx = b + threadIdx.x;
        const int v = idx < nt ? sums[idx] : 0;
        int excl;
        const int tot = block_exclusive_scan(v, &excl);
        const int carry = carry_s;
        if (idx < nt) sums[idx] = carry + excl;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles(const int *__restrict__ in, int64_t n,
                                                           const int *__restrict__ sums, int *__restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = base + q < n ? in[base + q] : 0;
        s += v[q];
    }
    int excl;
    const int tot = block_exclusive_scan(s, &excl);
    int run = sums[blockIdx.x] + excl;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[blockIdx.x] + tot;
}

}  // namespace

int64_t ptp_scan_tmp_ints(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

ptp_status ptp_exclusive_scan(const int *in, int *out, int64_t n, int *tmp, cudaStream_t s) {
    if (n <= 0) {
        PTP_TRY(cudaMemsetAsync(out, 0, sizeof(int), s));
        return PTP_OK;
    }
    const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    scan_tile_sums<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, tmp);
    scan_sums<<<1, SCAN_THREADS, 0, s>>>(tmp, nt);
    scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, tmp, out);
    ptp_count_launches(3);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

// ---------------------------------------------------------------------------
// Mesh kernels
// ---------------------------------------------------------------------------

namespace {

__global__ void validate_faces(const int *__restrict__ F, int64_t nf, int64_t n, int *__restrict__ err) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
        if (a < 0 || a >= n || b < 0 || b >= n || c < 0 || c >= n) atomicOr(err, 1);
        else if (a == b || b == c || a == c) atomicOr(err, 2);
    }
}

__global__ void count_corners(const int *__restrict__ F, int64_t nc, int *__restrict__ deg) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[F[c]], 1);
}

__global__ void fill_corners(const int *__restrict__ F, int64_t nf, const int *__restrict__ row,
                             int *__restrict__ cursor, int2 *__restrict__ pairs) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const int t[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int v = t[s];
            const int slot = row[v] + atomicAdd(&cursor[v], 1);
            pairs[slot] = make_int2(t[(s + 1) % 3], t[(s + 2) % 3]);
        }
    }
}

// float32 xyz -> float4; also a per-block bounding box into bb[6] using the
// order-preserving integer image of each float.
__device__ __forceinline__ int float_key(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__global__ void pack_positions(const float *__restrict__ xyz, int64_t n, float4 *__restrict__ pos, int *__restrict__ bb) {
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const float x = xyz[3 * v], y = xyz[3 * v + 1], z = xyz[3 * v + 2];
        pos[v] = make_float4(x, y, z, 0.0f);
        mn[0] = fminf(mn[0], x); mn[1] = fminf(mn[1], y); mn[2] = fminf(mn[2], z);
        mx[0] = fmaxf(mx[0], x); mx[1] = fmaxf(mx[1], y); mx[2] = fmaxf(mx[2], z);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[q] = fminf(mn[q], __shfl_xor_sync(0xffffffffu, mn[q], o));
            mx[q] = fmaxf(mx[q], __shfl_xor_sync(0xffffffffu, mx[q], o));
        }
    }
    // then across the CTA's warps, so that only one atomic per CTA and key
    // reaches the six shared words
    __shared__ float s_mn[3][32], s_mx[3][32];
    const int wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            s_mn[q][wid] = mn[q];
            s_mx[q][wid] = mx[q];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float a = s_mn[q][0], b = s_mx[q][0];
            for (int w = 1; w < nw; ++w) {
                a = fminf(a, s_mn[q][w]);
                b = fmaxf(b, s_mx[q][w]);
            }
            atomicMin(&bb[q], float_key(a));
            atomicMax(&bb[3 + q], float_key(b));
        }
    }
}

__global__ void init_bbox(int *bb) {
    if (threadIdx.x < 3) bb[threadIdx.x] = 0x7fffffff;
    else if (threadIdx.x < 6) bb[threadIdx.x] = (int)0x80000000;
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
            // the corner lists are filled by atomics in arbitrary order; sort
            // them so the fan (and every FP32 result) is the same each run
            for (int q = 1; q < deg; ++q) {
                const int xa = pa[q], xb = pb[q];
                int z = q - 1;
                while (z >= 0 && (pa[z] > xa || (pa[z] == xa && pb[z] > xb))) {
                    pa[z + 1] = pa[z];
                    pb[z + 1] = pb[z];
                    --z;
                }
                pa[z + 1] = xa;
                pb[z + 1] = xb;
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


unsigned grid_for(int64_t work, int threads, int device) {
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)ptp_num_sms(device) * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

extern "C" ptp_status ptp_mesh_create(const float *xyz, int64_t n_verts, const int32_t *faces, int64_t n_faces,
                                      int ptr_kind, void *stream, ptp_mesh **out) {
    if (!out) return PTP_ERR_ARG;
    *out = nullptr;
    if (!xyz || !faces || n_verts < 3 || n_faces < 1 || (ptr_kind != PTP_HOST && ptr_kind != PTP_DEVICE))
        return PTP_ERR_ARG;
    if (3 * n_faces > 2147483647LL || n_verts > 2147483646LL) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    PTP_TRY(cudaGetDevice(&dev));

    ptp_mesh *m = (ptp_mesh *)calloc(1, sizeof(ptp_mesh));
    if (!m) return PTP_ERR_NOMEM;
    m->device = dev;
    m->stream = s;
    m->n = n_verts;
    m->nf = n_faces;
    const int64_t nc = 3 * n_faces;

    float *xyz_d = nullptr;
    int *F_d = nullptr, *deg = nullptr, *tmp = nullptr, *err = nullptr;
    ptp_status st = PTP_OK;
    int herr[8] = {0};
    cudaError_t ce = cudaSuccess;
#define MESH_TRY(call)                                   \
    do {                                                 \
        ce = (call);                                     \
        if (ce != cudaSuccess) {                         \
            st = ptp_internal_cuda_status(ce);           \
            goto fail;                                   \
        }                                                \
    } while (0)

    MESH_TRY(ptp_malloc_async((void **)&m->pos, sizeof(float4) * n_verts, s));
    MESH_TRY(ptp_malloc_async((void **)&m->row, sizeof(int) * (n_verts + 1), s));
    MESH_TRY(ptp_malloc_async((void **)&m->pairs, sizeof(int2) * nc, s));
    MESH_TRY(ptp_malloc_async((void **)&m->ring, sizeof(int4) * 2 * n_verts, s));
    MESH_TRY(ptp_malloc_async((void **)&m->meta, sizeof(int) * n_verts, s));
    MESH_TRY(ptp_malloc_async((void **)&deg, sizeof(int) * (2 * n_verts + 8), s));
    MESH_TRY(ptp_malloc_async((void **)&tmp, sizeof(int) * ptp_scan_tmp_ints(n_verts), s));
    err = deg + 2 * n_verts;  // [0] face errors, [2..7] bbox keys
    if (ptr_kind == PTP_HOST) {
        MESH_TRY(ptp_malloc_async((void **)&xyz_d, sizeof(float) * 3 * n_verts, s));
        MESH_TRY(ptp_malloc_async((void **)&F_d, sizeof(int) * nc, s));
        MESH_TRY(cudaMemcpyAsync(xyz_d, xyz, sizeof(float) * 3 * n_verts, cudaMemcpyHostToDevice, s));
        MESH_TRY(cudaMemcpyAsync(F_d, faces, sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    } else {
        xyz_d = (float *)xyz;
        F_d = (int *)faces;
    }
    MESH_TRY(cudaMemsetAsync(deg, 0, sizeof(int) * (2 * n_verts + 8), s));
    init_bbox<<<1, 32, 0, s>>>(err + 2);
    validate_faces<<<grid_for(n_faces, 256, dev), 256, 0, s>>>(F_d, n_faces, n_verts, err);
    pack_positions<<<grid_for(n_verts, 256, dev), 256, 0, s>>>(xyz_d, n_verts, m->pos, err + 2);
    ptp_count_launches(3);
    MESH_TRY(cudaGetLastError());
    MESH_TRY(cudaMemcpyAsync(herr, err, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
    MESH_TRY(cudaStreamSynchronize(s));
    if (herr[0] & 1) { st = PTP_ERR_INDEX; goto fail; }
    if (herr[0] & 2) { st = PTP_ERR_DEGENERATE_FACE; goto fail; }
    {
        double d2 = 0.0;
        for (int q = 0; q < 3; ++q) {
            auto kf = [](int k) { unsigned u = (unsigned)(k >= 0 ? k : k ^ 0x7fffffff); float f; memcpy(&f, &u, 4); return f; };
            const double e = (double)kf(herr[5 + q]) - (double)kf(herr[2 + q]);
            d2 += e * e;
        }
        m->diameter = sqrt(d2);
    }
    count_corners<<<grid_for(nc, 256, dev), 256, 0, s>>>(F_d, nc, deg);
    ptp_count_launches(1);
    MESH_TRY(cudaGetLastError());
    st = ptp_exclusive_scan(deg, m->row, n_verts, tmp, s);
    if (st != PTP_OK) goto fail;
    MESH_TRY(cudaMemsetAsync(deg + n_verts, 0, sizeof(int) * n_verts, s));
    fill_corners<<<grid_for(n_faces, 256, dev), 256, 0, s>>>(F_d, n_faces, m->row, deg + n_verts, m->pairs);
    build_rings<<<grid_for(n_verts, 128, dev), 128, 0, s>>>((int)n_verts, m->row, m->pairs, m->ring, m->meta);
    ptp_count_launches(2);
    MESH_TRY(cudaGetLastError());
    if (ptr_kind == PTP_HOST) {
        cudaFreeAsync(xyz_d, s);
        cudaFreeAsync(F_d, s);
    }
    cudaFreeAsync(deg, s);
    cudaFreeAsync(tmp, s);
    *out = m;
    return PTP_OK;

fail:
    if (ptr_kind == PTP_HOST) {
        if (xyz_d) cudaFreeAsync(xyz_d, s);
        if (F_d) cudaFreeAsync(F_d, s);
    }
    if (deg) cudaFreeAsync(deg, s);
    if (tmp) cudaFreeAsync(tmp, s);
    if (m->pos) cudaFreeAsync(m->pos, s);
    if (m->row) cudaFreeAsync(m->row, s);
    if (m->pairs) cudaFreeAsync(m->pairs, s);
    if (m->ring) cudaFreeAsync(m->ring, s);
    if (m->meta) cudaFreeAsync(m->meta, s);
    cudaStreamSynchronize(s);
    free(m);
    return st;
#undef MESH_TRY
}

extern "C" ptp_status ptp_mesh_info(const ptp_mesh *m, int64_t *n_verts, int64_t *n_faces, double *diameter) {
    if (!m) return PTP_ERR_ARG;
    if (n_verts) *n_verts = m->n;
    if (n_faces) *n_faces = m->nf;
    if (diameter) *diameter = m->diameter;
    return PTP_OK;
}

extern "C" ptp_status ptp_mesh_destroy(ptp_mesh *m) {
    if (!m) return PTP_ERR_ARG;
    cudaFreeAsync(m->pos, m->stream);
    cudaFreeAsync(m->row, m->stream);
    cudaFreeAsync(m->pairs, m->stream);
    cudaFreeAsync(m->ring, m->stream);
    cudaFreeAsync(m->meta, m->stream);
    if (m->tgeom) cudaFreeAsync(m->tgeom, m->stream);
    if (m->elen) cudaFreeAsync(m->elen, m->stream);
    const cudaError_t e = cudaStreamSynchronize(m->stream);
    free(m);
    return e == cudaSuccess ? PTP_OK : ptp_internal_cuda_status(e);
}

// ---------------------------------------------------------------------------
// Self-test of the device-side wait limit: every CTA of a cooperative launch
// arrives at a grid barrier that counts one CTA more than the grid has, so
// it can never complete; the wait gives up after `cycles` SM clock cycles,
// flags PTP_ERR_TIMEOUT and the kernel returns.
// ---------------------------------------------------------------------------

namespace {

__global__ void wait_selftest(ptp_ctrl *ctrl, long long cycles) {
    unsigned long long prev_hi[2] = {0ull, 0ull};
    ptp_grid_sync(ctrl->bar, 1, 0u, &ctrl->abort, &ctrl->status, prev_hi, gridDim.x + 1, cycles);
}

}  // namespace

extern "C" ptp_status ptp_selftest_wait_limit(int64_t cycles, void *stream) {
    if (cycles < 1000 || cycles > 4000000000LL) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ptp_ctrl *ctrl = nullptr;
    PTP_TRY(ptp_malloc_async((void **)&ctrl, sizeof(ptp_ctrl), s));
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(ptp_ctrl), s);
    long long c = cycles;
    void *args[] = {(void *)&ctrl, (void *)&c};
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void *)wait_selftest, dim3(2), dim3(32), args, 0, s);
    if (e == cudaSuccess) ptp_count_launches(1);
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(ctrl, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ptp_internal_cuda_status(e);
    return (ptp_status)status;
}
