// Launch autotuner of the fused path: timed trial frames over the launch configurations that do
// not change any result (the fused kernel's grid and whether a frame is one CUDA graph launch).

#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/letkf.h"
#include "internal.hpp"

namespace {

// The grid with the fewest CTAs that still takes ceil(n_dom / SMs) rounds of domains.
int balanced_grid(const letkf_ctx* c) {
    const int rounds = (c->n_dom + c->sms - 1) / c->sms;
    return (c->n_dom + rounds - 1) / rounds;
}

}  // namespace

extern "C" {

int letkf_get_tuning(const letkf_ctx* c, letkf_tuning* t) {
    if (!c || !t) return LETKF_EINVAL;
    t->fused_grid = c->fused_grid;
    t->graph = c->graph_on;
    return LETKF_OK;
}

int letkf_set_tuning(letkf_ctx* c, const letkf_tuning* t) {
    if (!c || !t) return LETKF_EINVAL;
    if (c->path != LETKF_PATH_FUSED) return (t->fused_grid == 0 && t->graph == 0) ? LETKF_OK : LETKF_EINVAL;
    if (t->fused_grid < 0 || t->fused_grid > c->sms || (t->graph != 0 && t->graph != 1)) return LETKF_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) return LETKF_ECUDA;
    letkf::fused_graph_reset(c);
    c->fused_grid = t->fused_grid > 0 ? std::min(t->fused_grid, c->n_dom) : std::min(c->sms, c->n_dom);
    c->graph_on = t->graph;
    return LETKF_OK;
}

int letkf_autotune(letkf_ctx* c, const void* y, int frames, letkf_tuning* best, double* best_ms) {
    if (!c || !y || frames < 1 || frames > 10000) return LETKF_EINVAL;
    if (c->path != LETKF_PATH_FUSED) {
        if (best) best->fused_grid = best->graph = 0;
        return LETKF_OK;
    }
    if (c->phase != 0) return LETKF_ESTATE;
    if (cudaSetDevice(c->device) != cudaSuccess) return LETKF_ECUDA;
    // the filter's state is saved and put back: trial frames leave no trace
    const size_t bytes = (size_t)c->n * c->m_pad * letkf::state_bytes(c);
    void* saved = nullptr;
    void* xpred = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LETKF_OK;
    const int cur0 = c->cur;
    const unsigned long long frame0 = c->frame;
    const double sigma0 = c->sigma;
    letkf_tuning keep;
    letkf_get_tuning(c, &keep);
    std::vector<letkf_tuning> cand;
    for (int g : {std::min(c->sms, c->n_dom), balanced_grid(c)})
        for (int gr = 0; gr < 2; ++gr) {
            bool dup = false;
            for (const letkf_tuning& t : cand) dup = dup || (t.fused_grid == g && t.graph == gr);
            if (!dup) cand.push_back({g, gr});
        }
    double t_best = 1e300;
    letkf_tuning w_best = keep;
    int st0 = 0;    // the caller's latched status survives the trials
    if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(&st0, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return LETKF_ECUDA;
    if (cudaMalloc(&saved, bytes) != cudaSuccess || cudaMalloc(&xpred, (size_t)c->n_act * 8) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = LETKF_ENOMEM;
    } else if (cudaMemcpyAsync(saved, c->X[cur0], bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        rc = LETKF_ECUDA;
    }
    for (size_t k = 0; k < cand.size() && rc == LETKF_OK; ++k) {
        if ((rc = letkf_set_tuning(c, &cand[k]))) break;
        for (int w = 0; w < 3 && rc == LETKF_OK; ++w) rc = letkf_step(c, y, 0.0, xpred);
        if (rc) break;
        cudaEventRecord(e0, c->stream);
        for (int f = 0; f < frames && rc == LETKF_OK; ++f) rc = letkf_step(c, y, 0.0, xpred);
        cudaEventRecord(e1, c->stream);
        if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = rc ? rc : LETKF_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / frames < t_best) {
            t_best = ms / frames;
            w_best = cand[k];
        }
        // back to the saved state before the next configuration
        if (cudaMemcpyAsync(c->X[cur0], saved, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) rc = LETKF_ECUDA;
        c->cur = cur0;
        c->frame = frame0;
        c->phase = 0;
    }
    if (saved) {
        cudaStreamSynchronize(c->stream);
        if (c->side) cudaStreamSynchronize(c->side);
        cudaMemcpy(c->X[cur0], saved, bytes, cudaMemcpyDeviceToDevice);
    }
    c->cur = cur0;
    c->frame = frame0;
    c->phase = 0;
    c->sigma = sigma0;
    c->v_frame[0] = c->v_frame[1] = ~0ull;     // noise blocks drawn during the trials are stale
    const int rc2 = letkf_set_tuning(c, rc == LETKF_OK ? &w_best : &keep);
    if (saved) cudaFree(saved);
    if (xpred) cudaFree(xpred);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // what the trial frames latched belongs to them
    cudaMemcpy(c->d_status, &st0, sizeof(int), cudaMemcpyHostToDevice);
    if (rc) return rc;
    if (rc2) return rc2;
    if (best) *best = w_best;
    if (best_ms) *best_ms = t_best;
    return LETKF_OK;
}

}  // extern "C"
