// Multi-source maps in the original vertex order: geodesic Voronoi regions
// and farthest-point sampling (Sec. 5.3, App. A).  The paper's multi-source
// GPU runs skip the rearrangement of the vertices (Sec. 5.1); here the band
// is walked through the BFS queue instead, with every per-vertex array in the
// original order, so a new source set costs one BFS and one window run and
// no renumbering pass.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ptp_internal.cuh"

namespace {

#define INF_BITS 0x7f800000u

unsigned blocks_for(int64_t work, int threads, int device) {
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)ptp_num_sms(device) * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Final distance / label buffers of the last window run -> caller's arrays.
__global__ void multi_out(const ptp_ctrl *__restrict__ ctrl, int n, const float *__restrict__ d0,
                          const float *__restrict__ d1, const int *__restrict__ lab0, const int *__restrict__ lab1,
                          float *__restrict__ d_out, int *__restrict__ lab_out) {
    const int w = ptp_final_buffer(ctrl->iterations);
    const float *d = w ? d1 : d0;
    const int *l = w ? lab1 : lab0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const float v = d[u];
        if (d_out) d_out[u] = v;
        if (lab_out) lab_out[u] = (v < __int_as_float(INF_BITS) && l) ? l[u] : -1;
    }
}

// argmax_v d(v) as one 64-bit key: distance bits (d >= 0, so they order like
// the floats; +inf is largest) above the complemented vertex index, so among
// equal distances the smallest index wins.
__global__ void argmax_key(const ptp_ctrl *__restrict__ ctrl, int n, const float *__restrict__ d0,
                           const float *__restrict__ d1, unsigned long long *__restrict__ slot) {
    const float *d = ptp_final_buffer(ctrl->iterations) ? d1 : d0;
    unsigned long long best = 0ull;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const unsigned long long key = ((unsigned long long)__float_as_uint(d[u]) << 32) | (unsigned)(~u);
        best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
        best = y > best ? y : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(slot, best);
}

// Totals over the maps of one sampling run.
struct FpsAccum {
    unsigned long long slot;  // argmax key of the current map
    long long iterations;
    long long band_updates;
    long long active;
    long long changed;
    long long fp64;
    int status;
    int rho;
};

// Append the chosen sample (the next source) and fold the map's statistics.
__global__ void fps_append(FpsAccum *acc, const ptp_ctrl *__restrict__ ctrl, const int *__restrict__ info,
                           int *__restrict__ samples, int *__restrict__ m_dev, int n_samples) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = *m_dev;
    if (m < n_samples) {
        samples[m] = (int)(~(unsigned)(acc->slot & 0xffffffffull));
        *m_dev = m + 1;
    }
    acc->slot = 0ull;
    acc->iterations += ctrl->iterations;
    acc->band_updates += ctrl->band_updates;
    acc->active += (long long)ctrl->active;
    acc->changed += (long long)ctrl->changed;
    acc->fp64 += (long long)ctrl->fp64;
    if (ctrl->status > acc->status) acc->status = ctrl->status;
    acc->rho = info[0];
}

__global__ void fps_fold(FpsAccum *acc, const ptp_ctrl *__restrict__ ctrl, const int *__restrict__ info) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    acc->iterations += ctrl->iterations;
    acc->band_updates += ctrl->band_updates;
    acc->active += (long long)ctrl->active;
    acc->changed += (long long)ctrl->changed;
    acc->fp64 += (long long)ctrl->fp64;
    if (ctrl->status > acc->status) acc->status = ctrl->status;
    acc->rho = info[0];
}

__global__ void fps_init(FpsAccum *acc, int *samples, int *m_dev, int first) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    memset(acc, 0, sizeof(FpsAccum));
    samples[0] = first;
    *m_dev = 1;
}

// All scratch of a multi-source run in one allocation (stream-ordered).
struct MultiAlloc {
    ptp_multi_bufs b;
    void *base = nullptr;
    cudaStream_t s = nullptr;
    ptp_status alloc(int n, bool labels, size_t extra, void **extra_out, cudaStream_t st) {
        s = st;
        const size_t N = (size_t)n;
        const size_t sizes[] = {sizeof(ptp_ctrl), extra,         4 * N,         4 * N, 4 * N,
                                4 * N,            4 * (N + 2),   16,            8 * N, 64,
                                4 * N,            4 * N,         labels ? 4 * N : 0, labels ? 4 * N : 0};
        size_t bytes = 0;
        for (size_t z : sizes) bytes += (z + 255) & ~(size_t)255;
        PTP_TRY(ptp_malloc_async(&base, bytes + 256, st));
        char *p = (char *)base;
        int q = 0;
        auto take = [&]() {
            char *r = p;
            p += (sizes[q++] + 255) & ~(size_t)255;
            return (void *)r;
        };
        b.n = n;
        b.ctrl = (ptp_ctrl *)take();
        void *ex = take();
        if (extra_out) *extra_out = ex;
        b.d0 = (float *)take();
        b.d1 = (float *)take();
        b.level = (int *)take();
        b.queue = (int *)take();
        b.off = (int *)take();
        b.info = (int *)take();
        b.spill = (int *)take();
        b.cnt = (int *)take();
        b.nstamp = (int *)take();
        b.chg = (int *)take();
        b.lab0 = labels ? (int *)take() : nullptr;
        b.lab1 = labels ? (int *)take() : nullptr;
        return PTP_OK;
    }
    ~MultiAlloc() {
        if (base) cudaFreeAsync(base, s);
    }
};

// The topleset-ordered copy a fused run writes (ptp_renum_bufs), in one
// stream-ordered allocation freed with the object.
struct RenumAlloc {
    ptp_renum_bufs rb;
    void *base = nullptr;
    cudaStream_t s = nullptr;
    // records_only: just what the BFS CTAs of an original-order run write
    // (meta, slots, iperm)
    // multi: also the schedule and feature sums of the learned multi-advance band
    ptp_status alloc(int n, cudaStream_t st, bool records_only = false, bool multi = false) {
        s = st;
        const size_t N = (size_t)n;
        const size_t R = records_only ? 0 : N;
        const size_t parts[] = {sizeof(float4) * R, sizeof(int4) * 2 * N, sizeof(int) * N,
                                sizeof(float4) * PTP_TRI * R, sizeof(float4) * 2 * R, sizeof(int) * N,
                                multi ? sizeof(int) * (N + 8) : 0,
                                multi ? sizeof(unsigned long long) * PTP_FEAT_RING_WORDS : 0};
        size_t bytes = 0;
        for (size_t z : parts) bytes += (z + 255) & ~(size_t)255;
        PTP_TRY(ptp_malloc_async(&base, bytes, st));
        char *q = (char *)base;
        int i = 0;
        auto take = [&]() {
            char *r = q;
            q += (parts[i++] + 255) & ~(size_t)255;
            return (void *)r;
        };
        rb.pos = (float4 *)take();
        rb.ring = (int4 *)take();
        rb.meta = (int *)take();
        rb.tgeom = (float4 *)take();
        rb.elen = (float4 *)take();
        rb.iperm = (int *)take();
        rb.sched = multi ? (int *)take() : nullptr;
        rb.facc = multi ? (unsigned long long *)take() : nullptr;
        return PTP_OK;
    }
    ~RenumAlloc() {
        if (base) cudaFreeAsync(base, s);
    }
};

// allow_multi: the entry point runs the learned multi-advance band (band_mode 2)
ptp_status check_params(const ptp_params *p, bool allow_multi = false) {
    if (!p) return PTP_ERR_ARG;
    if (!(p->eps >= 0.0) || !(p->eps_abs >= 0.0) || p->max_iter < 0 || p->trace_cap < 0) return PTP_ERR_ARG;
    if (p->reserved != 0 || p->reserved2 != 0 || p->conv_trace) return PTP_ERR_ARG;
    if (p->band_mode == 2 ? !(allow_multi && p->mlp_half && !p->schedule) : (p->band_mode != 0 && p->band_mode != 1))
        return PTP_ERR_ARG;
    if (p->band_mode != 2 && p->mlp_half) return PTP_ERR_ARG;
    if (p->block != 0 && (p->block < 64 || p->block > 512 || p->block % 32 != 0)) return PTP_ERR_ARG;
    return PTP_OK;
}

void fill_stats(ptp_stats *st, const ptp_ctrl &h, int rho) {
    st->iterations = h.iterations;
    st->band_updates = h.band_updates;
    st->active_updates = (int64_t)h.active;
    st->changed = (int64_t)h.changed;
    st->fp64_solves = (int64_t)h.fp64;
    st->rho = rho;
    st->status = h.status;
    st->checks = h.checks;
}

}  // namespace

extern "C" ptp_status ptp_distance_from_sources(ptp_mesh *mesh, const int32_t *sources, int32_t m, int ptr_kind,
                                               const ptp_params *params, float *d_out, void *stream,
                                               ptp_stats *stats) {
    if (!mesh || !sources || m < 1 || !d_out || (ptr_kind != PTP_HOST && ptr_kind != PTP_DEVICE)) return PTP_ERR_ARG;
    PTP_CHECK(check_params(params, true));
    if (params->schedule) return PTP_ERR_ARG;
    const bool multi = params->band_mode == 2;
    if (multi && mesh->n >= 0x40000000) return PTP_ERR_TOO_LARGE;  // queue entries carry two flag bits
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)mesh->n;
    std::vector<int32_t> h((size_t)m);
    if (ptr_kind == PTP_DEVICE) {
        PTP_TRY(cudaMemcpyAsync(h.data(), sources, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
        PTP_TRY(cudaStreamSynchronize(s));
    } else {
        memcpy(h.data(), sources, sizeof(int32_t) * m);
    }
    for (int32_t q = 0; q < m; ++q)
        if (h[q] < 0 || h[q] >= n) return PTP_ERR_INDEX;
    PTP_CHECK(ptp_internal_prepare());
    PTP_CHECK(ptp_internal_mesh_geometry(mesh, s));
    MultiAlloc ma;
    void *src_v = nullptr;
    PTP_CHECK(ma.alloc(n, false, sizeof(int) * (size_t)m, &src_v, s));
    int *src = (int *)src_v;
    PTP_TRY(cudaMemcpyAsync(src, h.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    if (ptp_internal_fused_producers(mesh, params, m, false, false) > 0) {
        // topleset-ordered copy written during the launch (200 B per vertex)
        RenumAlloc ra;
        PTP_CHECK(ra.alloc(n, s, false, multi));
        PTP_CHECK(ptp_internal_fused(mesh, &ma.b, params, src, nullptr, m, false, false, &ra.rb, s));
        PTP_CHECK(ptp_internal_fused_gather(mesh, &ma.b, &ra.rb, d_out, s));
    } else if (multi) {
        // the learned band infers its schedule inside the split launch
        return PTP_ERR_ARG;
    } else {
        // too few CTAs to split the launch: BFS, then the window in the original order
        PTP_CHECK(ptp_internal_bfs(mesh, &ma.b, src, nullptr, m, s));
        PTP_CHECK(ptp_internal_window_multi(mesh, &ma.b, params, src, nullptr, m, false, s));
        multi_out<<<blocks_for(n, 256, mesh->device), 256, 0, s>>>(ma.b.ctrl, n, ma.b.d0, ma.b.d1, nullptr, nullptr,
                                                                    d_out, nullptr);
        ptp_count_launches(1);
        PTP_TRY(cudaGetLastError());
    }
    if (!stats) return PTP_OK;
    ptp_ctrl hc;
    int info[4];
    PTP_TRY(cudaMemcpyAsync(&hc, ma.b.ctrl, sizeof(ptp_ctrl), cudaMemcpyDeviceToHost, s));
    PTP_TRY(cudaMemcpyAsync(info, ma.b.info, sizeof(info), cudaMemcpyDeviceToHost, s));
    PTP_TRY(cudaStreamSynchronize(s));
    fill_stats(stats, hc, info[0]);
    return (ptp_status)hc.status;
}

extern "C" ptp_status ptp_voronoi(ptp_mesh *mesh, const int32_t *seeds, int32_t m, int ptr_kind,
                                  const ptp_params *params, float *d_out, int32_t *label_out, void *stream,
                                  ptp_stats *stats) {
    if (!mesh || !seeds || m < 1 || (!d_out && !label_out) || (ptr_kind != PTP_HOST && ptr_kind != PTP_DEVICE))
        return PTP_ERR_ARG;
    PTP_CHECK(check_params(params));
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)mesh->n;
    std::vector<int32_t> h((size_t)m);
    if (ptr_kind == PTP_DEVICE) {
        PTP_TRY(cudaMemcpyAsync(h.data(), seeds, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
        PTP_TRY(cudaStreamSynchronize(s));
    } else {
        memcpy(h.data(), seeds, sizeof(int32_t) * m);
    }
    for (int32_t q = 0; q < m; ++q)
        if (h[q] < 0 || h[q] >= n) return PTP_ERR_INDEX;
    PTP_CHECK(ptp_internal_prepare());
    PTP_CHECK(ptp_internal_mesh_geometry(mesh, s));
    MultiAlloc ma;
    void *src_v = nullptr;
    PTP_CHECK(ma.alloc(n, true, sizeof(int) * (size_t)m, &src_v, s));
    int *src = (int *)src_v;
    PTP_TRY(cudaMemcpyAsync(src, h.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    RenumAlloc ra;  // the BFS records of a fused run
    if (ptp_internal_fused_producers(mesh, params, m, true, true) > 0) {
        PTP_CHECK(ra.alloc(n, s, true));
        PTP_CHECK(ptp_internal_fused(mesh, &ma.b, params, src, nullptr, m, true, true, &ra.rb, s));
    } else {
        PTP_CHECK(ptp_internal_bfs(mesh, &ma.b, src, nullptr, m, s));
        PTP_CHECK(ptp_internal_window_multi(mesh, &ma.b, params, src, nullptr, m, true, s));
    }
    multi_out<<<blocks_for(n, 256, mesh->device), 256, 0, s>>>(ma.b.ctrl, n, ma.b.d0, ma.b.d1, ma.b.lab0, ma.b.lab1,
                                                                d_out, label_out);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());
    if (!stats) return PTP_OK;
    ptp_ctrl hc;
    int info[4];
    PTP_TRY(cudaMemcpyAsync(&hc, ma.b.ctrl, sizeof(ptp_ctrl), cudaMemcpyDeviceToHost, s));
    PTP_TRY(cudaMemcpyAsync(info, ma.b.info, sizeof(info), cudaMemcpyDeviceToHost, s));
    PTP_TRY(cudaStreamSynchronize(s));
    fill_stats(stats, hc, info[0]);
    return (ptp_status)hc.status;
}

namespace {

// One sampling step: map from samples[0 .. *m_dev), then append its argmax.
// With rb (the BFS records) the map is one fused launch in the original
// order (the toplesets built while the window runs, no copy into topleset
// order: the paper also keeps multi-source maps in place, Sec. 5.1);
// without, the BFS and the window run one after the other.
ptp_status fps_step(ptp_mesh *mesh, ptp_multi_bufs *b, const ptp_params *params, int *samples, int *m_dev,
                    int n_samples, FpsAccum *acc, const ptp_renum_bufs *rb, cudaStream_t s) {
    const int n = b->n;
    if (rb) {
        PTP_CHECK(ptp_internal_fused(mesh, b, params, samples, m_dev, n_samples, true, false, rb, s));
    } else {
        PTP_CHECK(ptp_internal_bfs(mesh, b, samples, m_dev, n_samples, s));
        PTP_CHECK(ptp_internal_window_multi(mesh, b, params, samples, m_dev, n_samples, false, s));
    }
    argmax_key<<<blocks_for(n, 256, mesh->device), 256, 0, s>>>(b->ctrl, n, b->d0, b->d1, &acc->slot);
    fps_append<<<1, 32, 0, s>>>(acc, b->ctrl, b->info, samples, m_dev, n_samples);
    ptp_count_launches(2);
    PTP_TRY(cudaGetLastError());
    return PTP_OK;
}

}  // namespace

extern "C" ptp_status ptp_fps(ptp_mesh *mesh, int32_t first, int32_t n_samples, const ptp_params *params,
                              int32_t *samples_out, float *d_out, int use_graph, void *stream, ptp_stats *stats) {
    if (!mesh || !samples_out || n_samples < 1) return PTP_ERR_ARG;
    if (first < 0 || first >= mesh->n) return PTP_ERR_INDEX;
    PTP_CHECK(check_params(params));
    ptp_params p = *params;
    p.trace = nullptr;  // one trace per map would overwrite itself
    p.trace_cap = 0;
    p.schedule = nullptr;  // a schedule is per source set
    cudaStream_t us = (cudaStream_t)stream;
    const int n = (int)mesh->n;
    PTP_CHECK(ptp_internal_prepare());
    PTP_CHECK(ptp_internal_mesh_geometry(mesh, us));
    MultiAlloc ma;
    void *ex = nullptr;
    PTP_CHECK(ma.alloc(n, false, sizeof(FpsAccum) + 256 + sizeof(int) * 4, &ex, us));
    FpsAccum *acc = (FpsAccum *)ex;
    int *m_dev = (int *)((char *)ex + ((sizeof(FpsAccum) + 255) & ~(size_t)255));

    RenumAlloc ra;  // the BFS records of the fused sampling maps
    const bool fused = ptp_internal_fused_producers(mesh, &p, n_samples, true, false) > 0;
    if (fused) PTP_CHECK(ra.alloc(n, us, true));

    fps_init<<<1, 32, 0, us>>>(acc, samples_out, m_dev, first);
    ptp_count_launches(1);
    PTP_TRY(cudaGetLastError());

    ptp_status st = PTP_OK;
    if (n_samples > 1) {
        if (use_graph) {
            // capture one step on a private stream and relaunch it
            cudaStream_t cs = nullptr;
            cudaEvent_t ev = nullptr;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(ev, us);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            int64_t per_step = 0;
            if (e == cudaSuccess) {
                const int64_t c0 = ptp_kernel_launches();
                st = fps_step(mesh, &ma.b, &p, samples_out, m_dev, n_samples, acc, fused ? &ra.rb : nullptr, cs);
                per_step = ptp_kernel_launches() - c0;
                const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
                if (st == PTP_OK && e2 != cudaSuccess) e = e2;
            }
            ptp_count_launches((int)-per_step);  // recorded into the graph, not launched
            if (st == PTP_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            for (int i = 1; st == PTP_OK && e == cudaSuccess && i < n_samples; ++i) {
                e = cudaGraphLaunch(exec, cs);
                ptp_count_launches((int)per_step);  // the kernels captured in one step
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(us, ev, 0);
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            if (cs) {
                cudaStreamSynchronize(cs);
                cudaStreamDestroy(cs);
            }
            if (ev) cudaEventDestroy(ev);
            if (st == PTP_OK && e != cudaSuccess) st = ptp_internal_cuda_status(e);
        } else {
            for (int i = 1; st == PTP_OK && i < n_samples; ++i)
                st = fps_step(mesh, &ma.b, &p, samples_out, m_dev, n_samples, acc, fused ? &ra.rb : nullptr, us);
        }
    }
    if (st != PTP_OK) return st;
    if (d_out) {
        PTP_CHECK(ptp_internal_bfs(mesh, &ma.b, samples_out, m_dev, n_samples, us));
        PTP_CHECK(ptp_internal_window_multi(mesh, &ma.b, &p, samples_out, m_dev, n_samples, false, us));
        multi_out<<<blocks_for(n, 256, mesh->device), 256, 0, us>>>(ma.b.ctrl, n, ma.b.d0, ma.b.d1, nullptr, nullptr,
                                                                     d_out, nullptr);
        ptp_count_launches(1);
        fps_fold<<<1, 32, 0, us>>>(acc, ma.b.ctrl, ma.b.info);
        ptp_count_launches(1);
        PTP_TRY(cudaGetLastError());
    }
    if (!stats) return PTP_OK;
    FpsAccum h;
    PTP_TRY(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, us));
    PTP_TRY(cudaStreamSynchronize(us));
    stats->iterations = h.iterations;
    stats->band_updates = h.band_updates;
    stats->active_updates = h.active;
    stats->changed = h.changed;
    stats->fp64_solves = h.fp64;
    stats->rho = h.rho;
    stats->status = h.status;
    stats->checks = 0;
    return (ptp_status)h.status;
}
