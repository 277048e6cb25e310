// Launch-shape autotuner for the window kernels.  The iteration of Sec. 4.2
// fixes what every launch computes (bands, tests, iterates); threads per CTA
// and the number of CTAs only decide how the band's chunks are spread over
// the GPU and how many CTAs meet at each iteration's grid barrier, and the
// maps are bit-identical for every shape.  Small meshes (a band of a few
// hundred vertices) favour few CTAs (a cheaper barrier), large ones all SMs;
// the tuner times each candidate on the caller's own problem and keeps the
// fastest.
#include <string.h>

#include <algorithm>
#include <vector>

#include "ptp_internal.cuh"

namespace {

struct Shape {
    int block, grid;
};

// Candidates: CTAs of 512, 256 and 128 threads; per CTA size, all
// co-resident CTAs, one per SM, and 1/2, 1/4, 1/8 of the SMs, and 8 CTAs.
ptp_status candidates(int device, bool batch, std::vector<Shape> &out) {
    const int sms = ptp_num_sms(device);
    const int blocks[] = {512, 256, 128};
    for (int block : blocks) {
        int per_sm = 0;
        const ptp_status st = batch ? ptp_internal_window_occupancy_batch(block, &per_sm)
                                    : ptp_internal_window_occupancy(block, &per_sm);
        if (st != PTP_OK) return st;
        if (per_sm < 1) continue;
        const int full = per_sm * sms;
        int grids[] = {full, sms, sms / 2, sms / 4, sms / 8, 8};
        std::vector<int> g;
        for (int x : grids)
            if (x >= 1 && x <= full && std::find(g.begin(), g.end(), x) == g.end()) g.push_back(x);
        for (int x : g) out.push_back({block, x});
    }
    return out.empty() ? PTP_ERR_CUDA : PTP_OK;
}

}  // namespace

extern "C" ptp_status ptp_autotune(ptp_toplesets_t *tops, ptp_batch_t *batch, ptp_params *params, int32_t reps,
                                   void *stream, ptp_tune_result *result) {
    if (!params || (!tops == !batch)) return PTP_ERR_ARG;
    if (reps <= 0) reps = 3;
    if (reps > 100) return PTP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int device = 0, count = 1;
    int64_t sizes[PTP_BATCH_MAX];
    if (batch) {
        PTP_CHECK(ptp_internal_batch_shape(batch, &device, &count, sizes));
    } else {
        device = tops->device;
        sizes[0] = tops->n;
    }
    std::vector<Shape> cand;
    PTP_CHECK(candidates(device, batch != nullptr, cand));

    // outputs for the trial runs (the caller's buffers are not touched)
    int64_t total = 0;
    for (int b = 0; b < count; ++b) total += sizes[b];
    float *scratch = nullptr;
    PTP_TRY(ptp_malloc_async((void **)&scratch, sizeof(float) * (total > 0 ? total : 1), s));
    float *outs[PTP_BATCH_MAX];
    {
        int64_t o = 0;
        for (int b = 0; b < count; ++b) {
            outs[b] = scratch + o;
            o += sizes[b];
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);

    ptp_params trial = *params;
    trial.ev_begin = e0;
    trial.ev_end = e1;
    ptp_status st = ce == cudaSuccess ? PTP_OK : ptp_internal_cuda_status(ce);
    Shape best = cand[0];
    float best_ms = 0.0f, default_ms = 0.0f;
    int tried = 0;
    std::vector<float> t(reps);
    for (size_t c = 0; c < cand.size() && st == PTP_OK; ++c) {
        trial.block = cand[c].block;
        trial.grid = cand[c].grid;
        for (int r = 0; r < reps && st == PTP_OK; ++r) {
            ptp_status rs = batch ? ptp_distance_batch(batch, &trial, outs, stream, nullptr)
                                  : ptp_distance(tops, &trial, outs[0], stream, nullptr);
            if (rs != PTP_OK && rs != PTP_ERR_NOT_CONVERGED) {
                st = rs;
                break;
            }
            ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t[r], e0, e1);
            if (ce != cudaSuccess) st = ptp_internal_cuda_status(ce);
        }
        if (st != PTP_OK) break;
        std::sort(t.begin(), t.end());
        const float med = t[reps / 2];
        ++tried;
        if (c == 0) default_ms = med;
        if (c == 0 || med < best_ms) {
            best_ms = med;
            best = cand[c];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(scratch, s);
    if (st != PTP_OK) return st;
    params->block = best.block;
    params->grid = best.grid;
    if (result) {
        result->block = best.block;
        result->grid = best.grid;
        result->ms = best_ms;
        result->ms_default = default_ms;
        result->tried = tried;
    }
    return PTP_OK;
}
