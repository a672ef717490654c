/*
 * fhash_serve.h - continuous-batching serving loop for trained F-Hash models on one GPU.
 *
 * The paper renders pretrained F-Hash INRs by sample streaming with adaptive ray marching (Section
 * 3.3, Algorithm 1) and supports temporal super-resolution at unseen time steps (Section 3.3).  This
 * server runs many such requests at once: render requests (images of any size, any camera, any
 * fractional time) and time-slice decode requests (the model on a grid over the Feature Bounding Box
 * at any fractional time, upsampled 1x-8x), over one or more device-resident models.
 *
 * Each fhash_server_tick:
 *  1. admits queued requests in arrival order while fewer than max_live requests are live and their
 *     scratch fits in the memory budget (a pool carved once at creation; no allocation per request);
 *  2. packs samples from every live request into one buffer of tick_samples slots: each render
 *     contributes one ARM round (its alive rays x its pace N_s, Algorithm 1), each decode its next
 *     chunk of grid points;
 *  3. evaluates each model's packed segment with one persistent encode+MLP launch, captured once in a
 *     CUDA graph at creation and replayed every tick (the segment offset and count are read from
 *     device memory);
 *  4. composites render samples and copies decode values to the requests' outputs, then reads every
 *     request's progress back with one copy and one synchronisation.
 * Steps 2 and 4 are one kernel launch each over all live requests (a per-tick work table gives every
 * request its range of threads), and the rays of all renders admitted in a tick are set up by one more
 * launch: a tick makes a number of launches that does not grow with the number of live requests.
 * A render's w*h may not exceed tick_samples (one round of all its rays must fit in a tick).
 * Requests that arrive while others are on the GPU join at the next tick.  Per-sample arithmetic does
 * not depend on where a sample sits in the packed buffer and the image does not depend on the pace,
 * so every result is bit-identical to the same request run alone through fhash_render / fhash_decode.
 *
 * Calls on one server are serialised by an internal lock.  The server does not own the models, which
 * must outlive it and must not be trained while it serves them.
 */
#ifndef FHASH_SERVE_H
#define FHASH_SERVE_H

#include "fhash.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fhash_server fhash_server;

enum { FHASH_REQ_RENDER = 0, FHASH_REQ_DECODE = 1 };
enum { FHASH_REQ_QUEUED = 0, FHASH_REQ_LIVE = 1, FHASH_REQ_DONE = 2, FHASH_REQ_CANCELLED = 3 };

/*
 * One request.  kind FHASH_REQ_RENDER: cam, w, h, max_pace (1..64 per Algorithm 1), tf (device
 * [256][4]), out = device [h][w][4] float32, counts = device [h][w] int32 or NULL - as fhash_render.
 * kind FHASH_REQ_DECODE: upsample (1..8), out = device [dims z][y][x] float32 - as fhash_decode.
 * model indexes the list given to fhash_server_create; t_norm in [0,1].  Output buffers are owned by
 * the caller and must stay valid until the request is done or cancelled.
 */
typedef struct {
    int32_t kind;
    int32_t model;
    float t_norm;
    fhash_camera cam;
    int32_t w, h, max_pace;
    const float* tf;
    int32_t upsample;
    float* out;
    int32_t* counts;
} fhash_request;

typedef struct {
    int64_t ticks;          /* ticks run */
    int64_t samples;        /* sample slots evaluated */
    int64_t model_launches; /* graph replays of the packed encode+MLP launch */
    int64_t live, queued;   /* current request counts */
    uint64_t pool_bytes;    /* request scratch pool */
    uint64_t pool_used;
    int64_t packed_launches; /* the other kernel launches: one ray initialisation per admission tick,
                                one sample generation and one compositing launch per tick, each over
                                every live request */
} fhash_server_stats;

/*
 * Create a server over n_models resident models.  budget_bytes bounds the device memory of the models'
 * parameters (+ bf16 shadows and occupancy grids), the packed buffers (20 bytes per tick sample) and
 * the request scratch pool, which takes the rest and is allocated here once.  Render requests need
 * about 64 bytes per pixel of scratch; decode requests none.  max_live: requests admitted at once.
 * Errors: FHASH_EINVAL if the models and buffers alone exceed the budget; FHASH_ENOMEM.
 */
fhash_status fhash_server_create(fhash_model* const* models, int32_t n_models, uint64_t budget_bytes, int32_t max_live,
                                 int64_t tick_samples, fhash_stream stream, fhash_server** out);

/* Queue a request (validated now; FHASH_EINVAL if malformed or larger than the whole pool).
 * *id identifies it for poll and cancel.  Does not touch the GPU. */
fhash_status fhash_server_submit(fhash_server* srv, const fhash_request* req, uint64_t* id);

/* Run one tick on `stream` (synchronises it once, or twice when requests are admitted).
 * *n_completed (may be NULL) receives the number of requests finished in this tick. */
fhash_status fhash_server_tick(fhash_server* srv, fhash_stream stream, int32_t* n_completed);

/* State of a request (FHASH_REQ_*) and, once done, its latency from submission to completion in ms
 * (measured on the host clock at the end of the tick that finished it). */
fhash_status fhash_server_poll(fhash_server* srv, uint64_t id, int32_t* state, double* latency_ms);

/* Cancel a queued or live request; its scratch is released at the next tick. */
fhash_status fhash_server_cancel(fhash_server* srv, uint64_t id);

fhash_status fhash_server_get_stats(fhash_server* srv, fhash_server_stats* out);

/* Destroy the server (synchronises the device; the models are not touched). */
void fhash_server_destroy(fhash_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* FHASH_SERVE_H */
