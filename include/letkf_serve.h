/*
 * letkf_serve.h - serving loop for many adaptive-optics systems on one GPU.
 *
 * The paper runs one AO system per machine (Sect. 4).  A server keeps the
 * ensembles of many systems resident on the device at once, each one a
 * fused-path letkf_ctx (letkf.h).  The server:
 *   - admits a system only while its device footprint (letkf_footprint) fits in
 *     what is left of the server's HBM budget, else refuses it with LETKF_EBUSY
 *     (nothing allocated; admit again once a release has freed memory);
 *   - queues each submitted frame (slopes copied into pinned host memory);
 *   - batches continuously: whenever one of its `slots` (a CUDA stream each) is
 *     free, the oldest waiting frame of every system that has no frame on the
 *     device (up to max_batch systems) goes into ONE launch of the fused kernel,
 *     whose work queue holds the domains of all of them.  Systems of different
 *     sizes and ensemble sizes share the launch.  Frames that arrive while batches
 *     run wait for the next free slot, and batches in different slots overlap on
 *     the device.  A system has at most one frame in flight, so its frames run in
 *     order and every frame's result is the one letkf_step would give it alone.
 *   - copies each frame's prediction x_hat(k+1|k) (n_act floats) and rejection
 *     flag back to pinned host memory and timestamps arrival, launch and host-
 *     observed completion.
 *
 * Threading: a server and its systems are driven from one host thread at a time.
 * Times are nanoseconds of letkf_now_ns (a monotonic host clock).
 * Every function returns a letkf_status (letkf.h).
 */
#ifndef LETKF_SERVE_H
#define LETKF_SERVE_H

#include "letkf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct letkf_server letkf_server;

typedef struct letkf_server_params {
    int device;                     /* CUDA device ordinal */
    unsigned long long hbm_budget;  /* device bytes the systems may hold in total (footprints plus the
                                       server's per-system buffers); 0: 90 % of the free memory */
    int max_systems;                /* 1 .. 1024 */
    int slots;                      /* batches in flight at once, one CUDA stream each: 1 .. 8 */
    int max_pending;                /* frames a system may have waiting: 1 .. 4096 */
    int max_batch;                  /* systems per launch: 1 .. 32 */
} letkf_server_params;

typedef struct letkf_frame_record {
    int system;                     /* id from letkf_server_admit */
    int status;                     /* LETKF_OK, or LETKF_ENONFINITE: frame rejected, state unchanged */
    unsigned long long frame;       /* the system's frame index */
    long long t_arrival_ns;         /* arrival time given to letkf_server_submit */
    long long t_launch_ns;          /* launch of the batch that carried it */
    long long t_done_ns;            /* completion seen by the host (prediction in host memory) */
    int batch_systems;              /* systems in that batch */
    int slot;                       /* stream slot of that batch */
    long long t_dev_start_ns;       /* device clock (CUDA events, from the server's creation): the
                                       batch's first operation on its slot's stream (slope copy) */
    long long t_dev_end_ns;         /* and its last (prediction copied out); batches in different
                                       slots whose intervals intersect ran on the device together */
} letkf_frame_record;

typedef struct letkf_server_info {
    unsigned long long hbm_budget, hbm_used;
    int systems;                    /* admitted */
    int frames_waiting, frames_in_flight;
    unsigned long long frames_done, batches, batched_systems;   /* batched_systems / batches = mean batch */
} letkf_server_info;

/* Monotonic host clock in nanoseconds. */
long long letkf_now_ns(void);

/* Create a server (creates `slots` streams on `device`).  *out is NULL on failure. */
int letkf_server_create(const letkf_server_params* params, letkf_server** out);

/* Wait for every batch in flight, release every system and the server.  NULL is accepted. */
int letkf_server_destroy(letkf_server* server);

/*
 * Admit a system: `params` as for letkf_create, with path LETKF_PATH_FUSED (else LETKF_EINVAL);
 * params->device and params->stream are ignored (the server's device; the context gets a
 * stream of its own).  LETKF_EBUSY if its footprint plus the server's buffers for it do not
 * fit in the budget left, or max_systems are admitted.  *id >= 0 on success.
 */
int letkf_server_admit(letkf_server* server, const letkf_params* params, int* id);

/* Release a system (waits for its frame in flight; drops its waiting frames). */
int letkf_server_release(letkf_server* server, int id);

/* Optional per-frame prediction output: from now on, frame k's x_hat(k+1|k) (n_act floats) is
 * copied to host + (k % n_frames) * n_act when the frame completes.  host = NULL turns it off.
 * The buffer is the caller's and must stay valid while it is registered. */
int letkf_server_set_output(letkf_server* server, int id, float* host, int n_frames);

/*
 * Queue one frame of system `id`: y_host holds its p slopes (FP32, letkf.h order), copied before
 * the call returns.  sigma > 0 replaces the noise std from this frame on.  t_arrival_ns is the
 * frame's arrival time (0: now).  LETKF_EBUSY if max_pending frames are already waiting.
 */
int letkf_server_submit(letkf_server* server, int id, const float* y_host, double sigma, long long t_arrival_ns);

/* One scheduler pass without blocking: retire finished batches, then launch batches into the
 * free slots.  *n_done (may be NULL) = frames completed in this pass. */
int letkf_server_pump(letkf_server* server, int* n_done);

/* Pump until no frame waits or runs. */
int letkf_server_drain(letkf_server* server);

/* Move up to `max` completion records (oldest first) to out; *n = how many. */
int letkf_server_records(letkf_server* server, letkf_frame_record* out, int max, int* n);

/* The system's context, for letkf_get_state / letkf_set_state / letkf_get_info between frames
 * (after letkf_server_drain).  Owned by the server. */
int letkf_server_context(letkf_server* server, int id, letkf_ctx** ctx);

int letkf_server_get_info(const letkf_server* server, letkf_server_info* out);

/*
 * Replay an arrival trace in real time on the calling thread: event i submits y[i] for system
 * sys[i] at t0 + t_ns[i] (t0 = the call's start; t_ns non-decreasing), with sigma[i] (sigma
 * may be NULL: keep), pumping in between, then drains.  An event refused with LETKF_EBUSY is
 * dropped and counted in *n_refused (may be NULL).
 */
int letkf_server_replay(letkf_server* server, int n, const int* sys, const long long* t_ns, const float* const* y,
                        const double* sigma, int* n_refused);

#ifdef __cplusplus
}
#endif

#endif /* LETKF_SERVE_H */
