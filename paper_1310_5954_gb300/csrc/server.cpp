// Serving loop: many AO systems resident on one GPU, frames batched continuously into single
// launches of the fused kernel (one work queue over the domains of every system in the batch).

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "../../include/letkf_serve.h"
#include "internal.hpp"

namespace {

struct Waiting {
    int buf;                 // index of the pinned slope buffer holding the frame
    double sigma;
    long long t_arrival;
};

struct System {
    bool used = false;
    letkf_ctx* c = nullptr;
    cudaStream_t stream = nullptr;    // the context's stream (owned by the server)
    unsigned long long bytes = 0;     // budget charged
    int p = 0, n_act = 0;
    float* y_pinned = nullptr;        // (max_pending + 1) x p
    std::vector<int> free_bufs;
    std::deque<Waiting> waiting;
    float* y_dev = nullptr;           // slopes of the frame on the device
    float* xpred_dev = nullptr;
    float* pred_pinned = nullptr;     // prediction of the frame in flight
    int* bad_pinned = nullptr;        // its rejection flag
    int busy_slot = -1;
    Waiting inflight{};
    unsigned long long inflight_frame = 0;
    float* out = nullptr;             // caller's prediction ring
    int out_frames = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr;      // the batch's first operation on the stream (device clock)
    cudaEvent_t done = nullptr;       // its last
    int* queue = nullptr;             // 4 ints: the fused kernel's work-queue counters
    bool busy = false;
    long long t_launch = 0;
    std::vector<int> systems;
};

long long now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

struct letkf_server {
    letkf_server_params prm{};
    cudaEvent_t ref = nullptr;        // device-clock origin of the records' device times
    unsigned long long used = 0;
    std::vector<System> sys;
    std::vector<Slot> slots;
    std::deque<letkf_frame_record> records;
    unsigned long long frames_done = 0, batches = 0, batched = 0;
};

namespace {

unsigned long long server_bytes_per_system(int p, int n_act) {
    // y and x_hat on the device
    return (unsigned long long)p * 4 + (unsigned long long)n_act * 4;
}

void drop_system(System& s) {
    if (s.c) letkf_destroy(s.c);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.y_pinned) cudaFreeHost(s.y_pinned);
    if (s.pred_pinned) cudaFreeHost(s.pred_pinned);
    if (s.bad_pinned) cudaFreeHost(s.bad_pinned);
    if (s.y_dev) cudaFree(s.y_dev);
    if (s.xpred_dev) cudaFree(s.xpred_dev);
    s = System();
}

// Retire every finished batch; returns the number of frames completed (or a negative status).
int retire(letkf_server* S) {
    int done = 0;
    for (size_t k = 0; k < S->slots.size(); ++k) {
        Slot& sl = S->slots[k];
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return LETKF_ECUDA;
        const long long t = now_ns();
        // device-clock interval of the batch, relative to the server's reference event
        float ms0 = 0.f, ms1 = 0.f;
        if (cudaEventElapsedTime(&ms0, S->ref, sl.start) != cudaSuccess ||
            cudaEventElapsedTime(&ms1, S->ref, sl.done) != cudaSuccess)
            return LETKF_ECUDA;
        for (int id : sl.systems) {
            System& s = S->sys[id];
            letkf_frame_record r;
            r.system = id;
            r.status = *s.bad_pinned ? LETKF_ENONFINITE : LETKF_OK;
            r.frame = s.inflight_frame;
            r.t_arrival_ns = s.inflight.t_arrival;
            r.t_launch_ns = sl.t_launch;
            r.t_done_ns = t;
            r.batch_systems = (int)sl.systems.size();
            r.slot = (int)k;
            r.t_dev_start_ns = (long long)((double)ms0 * 1e6);
            r.t_dev_end_ns = (long long)((double)ms1 * 1e6);
            S->records.push_back(r);
            if (s.out && s.out_frames > 0)
                std::memcpy(s.out + (size_t)(s.inflight_frame % (unsigned long long)s.out_frames) * s.n_act,
                            s.pred_pinned, (size_t)s.n_act * 4);
            s.free_bufs.push_back(s.inflight.buf);
            s.busy_slot = -1;
            ++done;
        }
        S->frames_done += sl.systems.size();
        sl.systems.clear();
        sl.busy = false;
    }
    return done;
}

// Launch one batch into a free slot if any system has a frame waiting and none in flight.
// Returns 1 if a batch was launched, 0 if not, or a negative status.
int launch(letkf_server* S) {
    int k = -1;
    for (size_t i = 0; i < S->slots.size(); ++i)
        if (!S->slots[i].busy) {
            k = (int)i;
            break;
        }
    if (k < 0) return 0;
    // the oldest waiting frames first
    std::vector<int> ready;
    for (size_t id = 0; id < S->sys.size(); ++id) {
        const System& s = S->sys[id];
        if (s.used && s.busy_slot < 0 && !s.waiting.empty()) ready.push_back((int)id);
    }
    if (ready.empty()) return 0;
    std::stable_sort(ready.begin(), ready.end(), [&](int a, int b) {
        return S->sys[a].waiting.front().t_arrival < S->sys[b].waiting.front().t_arrival;
    });
    if ((int)ready.size() > S->prm.max_batch) ready.resize(S->prm.max_batch);
    Slot& sl = S->slots[k];
    if (cudaEventRecord(sl.start, sl.stream) != cudaSuccess) return LETKF_ECUDA;
    std::vector<letkf::FusedFrame> frames;
    for (int id : ready) {
        System& s = S->sys[id];
        const Waiting w = s.waiting.front();
        if (cudaMemcpyAsync(s.y_dev, s.y_pinned + (size_t)w.buf * s.p, (size_t)s.p * 4, cudaMemcpyHostToDevice,
                            sl.stream) != cudaSuccess)
            return LETKF_ECUDA;
        frames.push_back({s.c, s.y_dev, w.sigma, s.c->piston != LETKF_PISTON_OFF ? s.c->xhat : s.xpred_dev, 1});
    }
    sl.t_launch = now_ns();
    int rc = letkf::fused_batch(frames.data(), (int)frames.size(), sl.queue, sl.stream);
    if (rc) return rc;
    for (int id : ready) {
        System& s = S->sys[id];
        // differential pistons: the new state is the context's other buffer until the swap below
        if ((rc = letkf::piston_launch(s.c, s.y_dev, s.xpred_dev, s.c->X[s.c->cur ^ 1], sl.stream))) return rc;
        if (cudaMemcpyAsync(s.pred_pinned, s.xpred_dev, (size_t)s.n_act * 4, cudaMemcpyDeviceToHost, sl.stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(s.bad_pinned, s.c->d_frame_bad, sizeof(int), cudaMemcpyDeviceToHost, sl.stream) !=
                cudaSuccess)
            return LETKF_ECUDA;
        s.inflight = s.waiting.front();
        s.waiting.pop_front();
        s.inflight_frame = s.c->frame;
        s.busy_slot = k;
        // the context's own bookkeeping, as letkf_step does
        s.c->cur ^= 1;
        s.c->frame += 1;
        s.c->phase = 0;
    }
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return LETKF_ECUDA;
    sl.systems = ready;
    sl.busy = true;
    S->batches += 1;
    S->batched += ready.size();
    return 1;
}

bool anything_left(const letkf_server* S) {
    for (const Slot& sl : S->slots)
        if (sl.busy) return true;
    for (const System& s : S->sys)
        if (s.used && !s.waiting.empty()) return true;
    return false;
}

}  // namespace

extern "C" {

long long letkf_now_ns(void) { return now_ns(); }

int letkf_server_create(const letkf_server_params* p, letkf_server** out) {
    if (!out) return LETKF_EINVAL;
    *out = nullptr;
    if (!p || p->max_systems < 1 || p->max_systems > 1024 || p->slots < 1 || p->slots > 8 || p->max_pending < 1 ||
        p->max_pending > 4096 || p->max_batch < 1 || p->max_batch > letkf::FUSED_MAX_BATCH)
        return LETKF_EINVAL;
    if (cudaSetDevice(p->device) != cudaSuccess) return LETKF_ECUDA;
    letkf_server* S = new (std::nothrow) letkf_server();
    if (!S) return LETKF_ENOMEM;
    S->prm = *p;
    if (S->prm.hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete S;
            return LETKF_ECUDA;
        }
        S->prm.hbm_budget = (unsigned long long)(0.9 * (double)fr);
    }
    S->sys.resize(p->max_systems);
    S->slots.resize(p->slots);
    int rc = LETKF_OK;
    for (Slot& sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&sl.start) != cudaSuccess || cudaEventCreate(&sl.done) != cudaSuccess) {
            rc = LETKF_ECUDA;
            break;
        }
        if (cudaMalloc(&sl.queue, 4 * sizeof(int)) != cudaSuccess || cudaMemset(sl.queue, 0, 4 * sizeof(int)) != cudaSuccess) {
            rc = LETKF_ENOMEM;
            break;
        }
    }
    if (!rc && (cudaEventCreate(&S->ref) != cudaSuccess || cudaEventRecord(S->ref, S->slots[0].stream) != cudaSuccess ||
                cudaEventSynchronize(S->ref) != cudaSuccess))
        rc = LETKF_ECUDA;
    if (rc) {
        letkf_server_destroy(S);
        return rc;
    }
    *out = S;
    return LETKF_OK;
}

int letkf_server_destroy(letkf_server* S) {
    if (!S) return LETKF_OK;
    cudaSetDevice(S->prm.device);
    for (Slot& sl : S->slots)
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    for (System& s : S->sys)
        if (s.used) drop_system(s);
    for (Slot& sl : S->slots) {
        if (sl.queue) cudaFree(sl.queue);
        if (sl.start) cudaEventDestroy(sl.start);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (S->ref) cudaEventDestroy(S->ref);
    delete S;
    return LETKF_OK;
}

int letkf_server_admit(letkf_server* S, const letkf_params* params, int* id) {
    if (!S || !params || !id) return LETKF_EINVAL;
    *id = -1;
    if (params->path != LETKF_PATH_FUSED) return LETKF_EINVAL;
    letkf_params p = *params;
    p.device = S->prm.device;
    p.stream = nullptr;
    unsigned long long fp = 0;
    int rc = letkf_footprint(&p, &fp);
    if (rc) return rc;
    int slot = -1;
    for (size_t i = 0; i < S->sys.size(); ++i)
        if (!S->sys[i].used) {
            slot = (int)i;
            break;
        }
    if (slot < 0) return LETKF_EBUSY;
    if (cudaSetDevice(S->prm.device) != cudaSuccess) return LETKF_ECUDA;
    if (S->used + fp > S->prm.hbm_budget) return LETKF_EBUSY;
    System s;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) return LETKF_ECUDA;
    p.stream = s.stream;
    rc = letkf_create(&p, &s.c);
    if (rc) {
        drop_system(s);
        return rc;
    }
    s.used = true;
    letkf_info info;
    letkf_get_info(s.c, &info);
    s.p = info.p;
    s.n_act = info.n_act;
    s.bytes = fp + server_bytes_per_system(s.p, s.n_act);
    if (S->used + s.bytes > S->prm.hbm_budget) {
        drop_system(s);
        return LETKF_EBUSY;
    }
    const int nb = S->prm.max_pending + 1;
    if (cudaMallocHost((void**)&s.y_pinned, (size_t)nb * s.p * 4) != cudaSuccess ||
        cudaMallocHost((void**)&s.pred_pinned, (size_t)s.n_act * 4) != cudaSuccess ||
        cudaMallocHost((void**)&s.bad_pinned, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&s.y_dev, (size_t)s.p * 4) != cudaSuccess ||
        cudaMalloc((void**)&s.xpred_dev, (size_t)s.n_act * 4) != cudaSuccess) {
        drop_system(s);
        return LETKF_ENOMEM;
    }
    for (int b = nb - 1; b >= 0; --b) s.free_bufs.push_back(b);
    S->used += s.bytes;
    S->sys[slot] = std::move(s);
    *id = slot;
    return LETKF_OK;
}

int letkf_server_release(letkf_server* S, int id) {
    if (!S || id < 0 || id >= (int)S->sys.size() || !S->sys[id].used) return LETKF_EINVAL;
    System& s = S->sys[id];
    cudaSetDevice(S->prm.device);
    while (s.busy_slot >= 0) {
        cudaStreamSynchronize(S->slots[s.busy_slot].stream);
        const int rc = retire(S);
        if (rc < 0) return rc;
    }
    S->used -= s.bytes;
    drop_system(s);
    return LETKF_OK;
}

int letkf_server_set_output(letkf_server* S, int id, float* host, int n_frames) {
    if (!S || id < 0 || id >= (int)S->sys.size() || !S->sys[id].used || (host && n_frames < 1)) return LETKF_EINVAL;
    S->sys[id].out = host;
    S->sys[id].out_frames = host ? n_frames : 0;
    return LETKF_OK;
}

int letkf_server_submit(letkf_server* S, int id, const float* y, double sigma, long long t_arrival) {
    if (!S || !y || id < 0 || id >= (int)S->sys.size() || !S->sys[id].used) return LETKF_EINVAL;
    System& s = S->sys[id];
    if ((int)s.waiting.size() >= S->prm.max_pending || s.free_bufs.empty()) return LETKF_EBUSY;
    const int b = s.free_bufs.back();
    s.free_bufs.pop_back();
    std::memcpy(s.y_pinned + (size_t)b * s.p, y, (size_t)s.p * 4);
    s.waiting.push_back({b, sigma, t_arrival ? t_arrival : now_ns()});
    return LETKF_OK;
}

int letkf_server_pump(letkf_server* S, int* n_done) {
    if (n_done) *n_done = 0;
    if (!S) return LETKF_EINVAL;
    if (cudaSetDevice(S->prm.device) != cudaSuccess) return LETKF_ECUDA;
    const int d = retire(S);
    if (d < 0) return d;
    if (n_done) *n_done = d;
    for (;;) {
        const int l = launch(S);
        if (l < 0) return l;
        if (l == 0) break;
    }
    return LETKF_OK;
}

int letkf_server_drain(letkf_server* S) {
    if (!S) return LETKF_EINVAL;
    while (anything_left(S)) {
        const int rc = letkf_server_pump(S, nullptr);
        if (rc) return rc;
    }
    return LETKF_OK;
}

int letkf_server_records(letkf_server* S, letkf_frame_record* out, int max, int* n) {
    if (!S || !n || (max > 0 && !out)) return LETKF_EINVAL;
    int k = 0;
    while (k < max && !S->records.empty()) {
        out[k++] = S->records.front();
        S->records.pop_front();
    }
    *n = k;
    return LETKF_OK;
}

int letkf_server_context(letkf_server* S, int id, letkf_ctx** ctx) {
    if (!S || !ctx || id < 0 || id >= (int)S->sys.size() || !S->sys[id].used) return LETKF_EINVAL;
    *ctx = S->sys[id].c;
    return LETKF_OK;
}

int letkf_server_get_info(const letkf_server* S, letkf_server_info* o) {
    if (!S || !o) return LETKF_EINVAL;
    o->hbm_budget = S->prm.hbm_budget;
    o->hbm_used = S->used;
    o->systems = 0;
    o->frames_waiting = 0;
    o->frames_in_flight = 0;
    for (const System& s : S->sys) {
        if (!s.used) continue;
        o->systems += 1;
        o->frames_waiting += (int)s.waiting.size();
        o->frames_in_flight += s.busy_slot >= 0 ? 1 : 0;
    }
    o->frames_done = S->frames_done;
    o->batches = S->batches;
    o->batched_systems = S->batched;
    return LETKF_OK;
}

int letkf_server_replay(letkf_server* S, int n, const int* sys, const long long* t_ns, const float* const* y,
                        const double* sigma, int* n_refused) {
    if (n_refused) *n_refused = 0;
    if (!S || n < 0 || (n > 0 && (!sys || !t_ns || !y))) return LETKF_EINVAL;
    for (int i = 1; i < n; ++i)
        if (t_ns[i] < t_ns[i - 1]) return LETKF_EINVAL;
    const long long t0 = now_ns();
    int i = 0, refused = 0;
    while (i < n || anything_left(S)) {
        const long long t = now_ns();
        while (i < n && t0 + t_ns[i] <= t) {
            const int rc = letkf_server_submit(S, sys[i], y[i], sigma ? sigma[i] : 0.0, t0 + t_ns[i]);
            if (rc == LETKF_EBUSY) {
                ++refused;
            } else if (rc) {
                return rc;
            }
            ++i;
        }
        const int rc = letkf_server_pump(S, nullptr);
        if (rc) return rc;
    }
    if (n_refused) *n_refused = refused;
    return LETKF_OK;
}

}  // extern "C"
