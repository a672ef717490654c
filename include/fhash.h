/*
 * fhash.h - C ABI of the F-Hash hot path for one GB300 GPU (sm_103a).
 *
 * F-Hash (feature-based multi-resolution Tesseract encoding, arXiv 2507.03836) learns an implicit
 * neural representation of a time-varying volume: given the volume's dimensions, its time steps,
 * a feature mask and a level schedule (Section 3.1, Section 3.2.1-3.2.2), every (x, y, z, t)
 * query is encoded per level by locating its 4D cell, mapping the cell's 16 corners through the
 * collision-free F-Hash of Eq. 9 to rows of compact per-level embedding tables and interpolating
 * the F embeddings quadrilinearly (Section 3.2.4, Eqs. 10-12); a shallow MLP decodes the
 * concatenated levels (Section 3.2.4, Section 4.2), trained with Adam (Section 5.1.3), and the
 * trained model is rendered by sample streaming with adaptive ray marching (Section 3.3,
 * Algorithm 1).
 *
 * Conventions shared by every call:
 *  - Pointers marked "device" must be device memory of the model's GPU; pointers marked
 *    "host or device" are inspected with cudaPointerGetAttributes and host memory is staged
 *    through the model's own device buffers (pinned host memory avoids a bounce copy).
 *  - The caller owns every input and output buffer.  The model owns its tables, MLP, Adam state,
 *    occupancy grid and scratch buffers (device memory allocated by fhash_build and grown on
 *    demand), and frees them in fhash_destroy.
 *  - Work is enqueued on `stream` (a cudaStream_t; 0 = legacy default stream) and is
 *    asynchronous unless stated otherwise.  Calls on one model must not overlap in time on
 *    different streams: the model's scratch buffers are shared.
 *  - Arguments are validated on the host before any launch; a bad argument returns FHASH_EINVAL
 *    and launches nothing.  Nothing aborts or traps.  fhash_last_error() returns a
 *    thread-local message for the last failing call on the calling thread.
 *  - Coordinates are FBB-normalised points u in [0,1]^4, stored [n][4] float32 as (x, y, z, t):
 *    u = 0 / 1 are the first / last vertex of the Feature Bounding Box on x, y, z and the first /
 *    last time step on t.  Values outside [0,1] are clamped and NaN is read as 0 (a documented
 *    behaviour, not an error).
 *  - Table rows are stored level after level (coarsest first); within level l the row of grid
 *    vertex (x, y, z, t) is base[l] + F-Hash^l(t, x, y, z) (Eq. 9), each row holding F values.
 *    The flat parameter vector is [rows * F table values | MLP parameters], the MLP stored
 *    layer by layer as W[out][in] followed by b[out].
 */
#ifndef FHASH_H
#define FHASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fhash_model fhash_model;
typedef void* fhash_stream; /* cudaStream_t */

typedef enum {
    FHASH_OK = 0,
    FHASH_EINVAL = 1,   /* invalid argument or unsupported configuration; nothing launched */
    FHASH_ENOMEM = 2,   /* device or host allocation failed */
    FHASH_ECUDA = 3,    /* a CUDA runtime call failed (message in fhash_last_error) */
    FHASH_EDEVICE = 4,  /* a kernel reported an error through the model's device error word */
    FHASH_ETIMEOUT = 5, /* a bounded device wait ran out */
    FHASH_EBUSY = 6,    /* serving: no slot or memory budget free for the request right now */
    FHASH_EIO = 7       /* checkpoint file could not be read or written */
} fhash_status;

enum { FHASH_FP32 = 0, FHASH_BF16 = 1 };
enum { FHASH_SCHED_FOLD = 0, FHASH_SCHED_EXPLICIT = 1, FHASH_SCHED_GEOMETRIC = 2 };
enum { FHASH_LEVELS_MAX = 0, FHASH_LEVELS_MIN = 1 };

#define FHASH_MAX_LEVELS 24
#define FHASH_MAX_HIDDEN 4

/*
 * Level schedule (Section 3.2.1-3.2.2).  All levels are listed COARSE -> FINE and count grid
 * vertices per axis (a level with R vertices has R-1 cells; vertex j sits at u = j/(R-1)).
 *  FHASH_SCHED_FOLD: the fold policy of Eqs. 4-8 on the Feature Bounding Box size S (Eq. 4),
 *    L_d = ceil(log_fold S_d) (Eq. 5), L_s = max_d L_d (Eq. 6; levels_rule FHASH_LEVELS_MAX) or
 *    min_d L_d (the level counts Table 3 prints; FHASH_LEVELS_MIN); each coarser level divides the
 *    previous one by fold, rounding up, while it exceeds fold, else takes 2 (Eqs. 7-8).  The time
 *    axis follows the same recursion from nt (Section 3.2.2).
 *  FHASH_SCHED_EXPLICIT: res[0..n_levels-1] = (Rx, Ry, Rz, Rt) per level.
 *  FHASH_SCHED_GEOMETRIC: R_l = floor(r0 * (r1/r0)^(l/(n_levels-1)) + 0.5) per axis in double.
 */
typedef struct {
    int32_t mode;
    int32_t fold;
    int32_t levels_rule;
    int32_t n_levels;
    int32_t res[FHASH_MAX_LEVELS][4];
    int32_t r0[4];
    int32_t r1[4];
} fhash_schedule;

/*
 * Model description for fhash_build (Section 3.1 and 3.2).
 *  nx, ny, nz: volume vertex counts (>= 2); nt: number of time steps / key frames (>= 1).
 *  mask: HOST pointer to [nt][nz][ny][nx] bytes, nonzero where a vertex belongs to the extracted
 *    feature; NULL means every vertex.  It is read during the call only.  The build dilates it
 *    by the 26-neighbourhood per time step (feature dilation, Section 3.1), takes the union of
 *    the per-frame boxes as the Feature Bounding Box and keeps the dilated mask as the bit
 *    occupancy grid used by the renderer.  An all-zero mask is FHASH_EINVAL.
 *  F: embedding size, 1, 2, 4 or 8 (L*F at most 64).  dtype: FHASH_FP32, or FHASH_BF16 (tables and MLP read as bf16
 *    shadows of float32 master weights; MLP on the tensor cores with float32 accumulation).
 *  mlp_hidden_layers (1..FHASH_MAX_HIDDEN) hidden layers of mlp_width (16, 32 or 64) with ReLU,
 *    then a linear scalar output; every layer has a bias.
 *  seed, init_range: tables start U(-init_range, init_range) (Section 3.2.4: uniform
 *    initialisation); the MLP starts with PyTorch's nn.Linear bounds U(-1/sqrt(fan_in),
 *    1/sqrt(fan_in)).  Values come from SplitMix64 used as a counter-based generator: element i
 *    of the table is output i of SplitMix64 seeded with key = output 200 of SplitMix64 seeded
 *    with `seed`, top 24 bits as U in [0,1), value = (float)(lo + (hi - lo) * U) in double; MLP
 *    layer k uses streams 300 + 2k (W) and 301 + 2k (b).
 */
/* Row order of a level's vertices.  LINEAR is Eq. 9: t*Rx*Ry*Rz + z*Rx*Ry + y*Rx + x.  BRICK is a
 * locality-preserving linearisation, which Section 3.2.3 allows in place of Eq. 9: each time slice is
 * cut into 4x4x4 spatial bricks (narrower at the high end of an axis when R is not a multiple of 4),
 * bricks in (bz, by, bx) order and vertices inside a brick in (iz, iy, ix) order.  With b = v / 4,
 * i = v % 4 and w(b) = min(4, R - 4b) per axis the row is
 *   t*Rx*Ry*Rz + 4*bz*Rx*Ry + wz*4*by*Rx + wz*wy*4*bx + (iz*wy + iy)*wx + ix,
 * a bijection onto [0, Rx*Ry*Rz*Rt) like Eq. 9.  The 16 corners of a cell then lie in 1 to 8 bricks
 * per time slice, which cuts the random memory accesses of the gathers at HBM-resident levels.
 *
 * MASKED keeps rows only for the vertices near the features: the irregular multi-resolution grids
 * that Section 3.1 describes as a smaller-model variant of the coreset.  Active vertices come from the
 * dilated mask of every time step:
 *   - Footprint of dilated voxel v (FBB-relative) on a spatial axis of S voxels: u*(S-1) in
 *     [v - 1/2, v + 1/2], the points whose nearest voxel is v.  On the time axis (nt steps), step k
 *     covers t*(nt-1) in [k - 1, k + 1].  In level units p = u*(R-1) the footprint is widened by
 *     1/64 on each side.
 *   - A vertex is active when it is a corner of a cell that the float32 cell step assigns to a point
 *     of some footprint.  Per axis these are the vertices clamp(floor(p_lo), 0, R-2) ..
 *     clamp(floor(p_hi), 0, R-2) + 1, in exact integer arithmetic.  An axis whose FBB has one voxel
 *     keeps all its vertices.
 *   - A level's rows are its active vertices in Eq. 9 order; base[l] adds up the active counts of the
 *     coarser levels.
 * An inactive corner contributes 0 to the encoding and receives no gradient.  Every sample whose
 * nearest voxel is in the dilated feature (coreset samples, rendered samples at occupied voxels) sees
 * only active corners.  There its encoding equals that of the rectangular table with the same vertex
 * values.  MASKED needs dtype FHASH_FP32 and a mask; the allocation-free gradient entry point does not
 * take it. */
enum { FHASH_LAYOUT_LINEAR = 0, FHASH_LAYOUT_BRICK = 1, FHASH_LAYOUT_MASKED = 2 };

typedef struct {
    int64_t nx, ny, nz, nt;
    const uint8_t* mask;
    fhash_schedule sched;
    int32_t F;
    int32_t dtype;
    int32_t mlp_hidden_layers;
    int32_t mlp_width;
    uint64_t seed;
    float init_range;
    int32_t layout;  /* FHASH_LAYOUT_LINEAR (Eq. 9, the default), _BRICK or _MASKED */
    /* Several features in one model (Section 3.1 merges the occupancy grids of several features for
     * rendering): n_masks > 0 host masks of the same shape as `mask` (which must then be NULL).  Each is
     * dilated on its own and the dilated regions are OR-merged: the Feature Bounding Box is the box of
     * the union, the occupancy grid its bits, and the masked layout keeps the vertices near any of
     * them.  0 means the single `mask` (or none). */
    const uint8_t* const* masks;
    int32_t n_masks;
} fhash_build_desc;

/* Read-only description of a built model. */
typedef struct {
    int32_t n_levels, F, dtype, n_mlp_layers;
    int32_t mlp_dims[FHASH_MAX_HIDDEN + 2];  /* L*F, width, ..., width, 1 */
    int32_t res[FHASH_MAX_LEVELS][4];        /* (Rx, Ry, Rz, Rt), coarse -> fine */
    uint64_t base[FHASH_MAX_LEVELS];         /* first row of each level */
    uint64_t total_rows;                     /* sum of Rx*Ry*Rz*Rt (MASKED: of the active counts) */
    uint64_t n_table_params;                 /* total_rows * F */
    uint64_t n_mlp_params;
    int64_t fbb_lo[3], fbb_size[3];          /* Feature Bounding Box, vertices, (x, y, z) */
    int64_t nt;                              /* time steps of the occupancy grid */
    int64_t step;                            /* Adam steps taken */
    uint64_t device_bytes;                   /* device memory held by the model */
} fhash_info;

/* Adam hyper-parameters (Section 5.1.3 uses lr = 0.01).  PyTorch semantics: dense update of every
 * parameter, bias correction, eps added to sqrt of the corrected second moment, no weight decay. */
typedef struct {
    float lr, beta1, beta2, eps;
} fhash_adam;

/*
 * Build a model (Section 3.1 feature dilation, bounding box and temporal fusion, occupancy grid;
 * Section 3.2.1-3.2.3 schedule and table sizing) on the current CUDA device and initialise its
 * parameters.  Synchronous: returns after the model is ready.  *out receives the model (owned by
 * the caller, released with fhash_destroy).  Errors: FHASH_EINVAL for bad dimensions, schedule,
 * F, MLP shape or an empty mask; FHASH_ENOMEM if the device cannot hold tables, gradients and the
 * two Adam moments (4 x rows x F x 4 bytes, plus bf16 shadows in FHASH_BF16).
 */
fhash_status fhash_build(const fhash_build_desc* desc, fhash_stream stream, fhash_model** out);

/*
 * Capacity planning without a build (host only: no CUDA call, so it also runs on a machine without a
 * GPU).  For a Feature Bounding Box of fbb[3] = (Sx, Sy, Sz) vertices and nt time steps it returns what
 * fhash_build would use with the same schedule, F, dtype and MLP shape in the rectangular layouts
 * (Eq. 9 or bricks; a masked layout keeps a subset of these rows):
 *  - *n_levels and res[0 .. *n_levels - 1] = (Rx, Ry, Rz, Rt), coarse -> fine (res may hold
 *    FHASH_MAX_LEVELS rows);
 *  - *table_rows = sum of Rx*Ry*Rz*Rt and *n_params = table_rows * F + the MLP's weights and biases;
 *  - *state_bytes = 16 bytes per parameter (parameter, gradient, two Adam moments), plus 2 more for
 *    the bf16 shadow of FHASH_BF16.
 * Any output pointer may be NULL.  Errors (FHASH_EINVAL) as fhash_build reports them for the same
 * arguments: bad schedule, F, dtype, MLP shape, L*F above 64, or a level too large to index.
 */
fhash_status fhash_plan(const fhash_schedule* sched, const int64_t fbb[3], int64_t nt, int32_t F, int32_t dtype,
                        int32_t mlp_hidden_layers, int32_t mlp_width, int32_t* n_levels, int32_t (*res)[4],
                        uint64_t* table_rows, uint64_t* n_params, uint64_t* state_bytes);

/* Release every device and host resource of the model (synchronises the device first). */
void fhash_destroy(fhash_model* model);

/* Thread-local text of the last error returned to this thread ("" if none). */
const char* fhash_last_error(void);

fhash_status fhash_get_info(const fhash_model* model, fhash_info* out);

/*
 * Level schedule and Feature Bounding Box of a model (the subset of fhash_get_info that defines
 * the Eq. 9 rows): *L levels; res[l] = (Rx, Ry, Rz, Rt) and base[l] = first row of level l,
 * coarse to fine; fbb = (lo_x, lo_y, lo_z, size_x, size_y, size_z).  The arrays need room for L
 * levels (at most FHASH_MAX_LEVELS); any output pointer may be NULL.
 */
fhash_status fhash_level_info(const fhash_model* model, int32_t* L, int32_t (*res)[4], uint64_t* base, int64_t fbb[6]);

/*
 * The model's float32 master parameters in two caller-owned buffers, host or device: tables
 * [total_rows][F] (Eq. 9 rows, levels concatenated coarse to fine) and the MLP vector
 * [n_mlp_params] (per layer W[out][in] then b[out]).  Either pointer may be NULL.  Returns after the
 * copy when a buffer is host memory.  fhash_set_params writes them (and refreshes the bf16 shadows of
 * FHASH_BF16 models).  Equivalent to fhash_read_state / fhash_write_state of FHASH_STATE_PARAM over
 * the two ranges.
 */
fhash_status fhash_get_params(fhash_model* model, float* tables, float* mlp, fhash_stream stream);
fhash_status fhash_set_params(fhash_model* model, const float* tables, const float* mlp, fhash_stream stream);

/*
 * Encoding steps 1-3 of Section 3.2.4 for inspection: per sample and level, the 16 corner rows
 * through Eq. 9 (with level base) and their quadrilinear weights (Eqs. 10-12), corner index
 * c = i + 2j + 4k + 8s (i, j, k: upper corner on x, y, z; s = 1 for t_Next).  In a
 * FHASH_LAYOUT_MASKED model an inactive corner's row is UINT64_MAX.
 *  coords: device [n][4]; rows: device [n][L][16] uint64; weights: device [n][L][16] float or NULL.
 */
fhash_status fhash_lookup(fhash_model* model, const float* coords, int64_t n, uint64_t* rows, float* weights,
                          fhash_stream stream);

/* Multi-resolution Tesseract encoding (Section 3.2.4, Eqs. 9-12): enc[n][L*F] float32, level 0
 * (coarsest) first.  coords: device [n][4]; enc: device.  n = 0 is a no-op. */
fhash_status fhash_encode(fhash_model* model, const float* coords, int64_t n, float* enc, fhash_stream stream);

/*
 * Backward of fhash_encode.  Eqs. 10-12 are linear in the table, so for every sample n, level l,
 * corner c (Eq. 9 row r) and feature f it adds w_c(n) * d_enc[n][l*F + f] to the gradient of
 * table element [r][f].  The sums ACCUMULATE in the model's gradient buffer (the table part of
 * FHASH_STATE_GRAD), which fhash_apply_adam consumes and clears; the MLP part is not touched.
 * Weights are recomputed from the coordinates, not stored.
 *  coords: device [n][4], the coordinates given to fhash_encode; d_enc: device [n][L*F] float32,
 *  row-major like fhash_encode's output.  Both stay owned by the caller.  n = 0 is a no-op; host
 *  pointers are FHASH_EINVAL.  Additions are float32 atomics: their order, and so the last bits
 *  of the sums, is not deterministic.
 */
fhash_status fhash_encode_backward(fhash_model* model, const float* coords, const float* d_enc, int64_t n,
                                   fhash_stream stream);

/*
 * No counterpart in the paper (an implementation choice of the bf16 precision form): how
 * fhash_forward, fhash_render and fhash_decode evaluate FHASH_BF16 models (float32 models have one
 * path).  FUSED: one kernel encodes each 128-sample tile into shared memory and runs the MLP on
 * it.  SPLIT: per chunk of up to 2^20 samples, one kernel writes the bf16 encoding rows and a second
 * one runs the MLP on the tensor cores, fed by TMA from those rows.  Both give bit-identical outputs;
 * they differ only in speed.  AUTO (the default) takes FUSED, the faster of the two on GB300 at every
 * batch size measured.  The serving loop always uses the fused kernel.  Unknown values are
 * FHASH_EINVAL.
 */
enum { FHASH_FORWARD_AUTO = 0, FHASH_FORWARD_FUSED = 1, FHASH_FORWARD_SPLIT = 2 };
fhash_status fhash_set_forward_path(fhash_model* model, int32_t path);

/* Encoding fused with the MLP decoder (Section 3.2.4): out[n] float32.
 * coords: host or device [n][4]; out: host or device [n]. */
fhash_status fhash_forward(fhash_model* model, const float* coords, int64_t n, float* out, fhash_stream stream);

/*
 * Forward + MSE loss + backward without the optimiser: leaves d(loss)/d(parameter) in the model's
 * gradient buffer (read it with fhash_read_state(FHASH_STATE_GRAD)).  loss = mean((y - target)^2)
 * reduced in float64 (host or device double*, may be NULL).  coords, target: host or device.
 */
fhash_status fhash_compute_grads(fhash_model* model, const float* coords, const float* target, int64_t n,
                                 double* loss, fhash_stream stream);

/* One Adam step (Section 5.1.3) over every parameter using the gradient buffer, which it then
 * clears to zero; increments the step count.  In float32: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * d = sqrt(v) * (1 / sqrt(bc2)) + eps, p = p - (lr / bc1) * (m / d), each line one rounded multiply and
 * one fused multiply-add, with the GPU's approximate square root and division (a few ulp); lr / bc1,
 * 1 / sqrt(bc2) and 1 - beta are computed in double from the step count and rounded to float32. */
fhash_status fhash_apply_adam(fhash_model* model, const fhash_adam* adam, fhash_stream stream);

/* One full training step: the result of fhash_compute_grads followed by fhash_apply_adam, bit for bit.
 * For models with deferred levels (fhash_set_adam_deferral) the Adam update of those levels' rows is
 * deferred to the next step that reads them, or to the next call that reads or writes the model's
 * state, whichever comes first; no call can observe the difference. */
fhash_status fhash_train_step(fhash_model* model, const float* coords, const float* target, int64_t n,
                              const fhash_adam* adam, double* loss, fhash_stream stream);

/*
 * Deferred Adam (an implementation of Section 5.1.3's dense Adam, not a different optimiser).  A step
 * whose gradient is zero moves every parameter by a fixed float32 map of (parameter, first moment,
 * second moment) that depends only on that step's scalars.  In fhash_train_step the table levels with
 * at least min_level_rows rows (and every finer level) do not take that map every step: each group of
 * 32 consecutive parameters remembers the last step applied to it, and when a batch is about to read
 * it (or any other call touches the state) it replays the missed steps, the first with its pending
 * gradient and the others with a zero gradient, with the same float32 operations in the same order as
 * the dense update.  Parameters, gradients and moments are therefore bit-identical to dense Adam at
 * every point a caller can observe, while a step streams only the groups its batch touches instead of
 * every parameter.  Coarser levels and the MLP take the dense update every step.
 *  min_level_rows: 0 turns deferral off; the default is 2^25 (33,554,432 rows).  Changing it first
 *  brings every group to the current step (a kernel on `stream`).  The state costs 4 bytes per 32
 *  deferred parameters (allocated at the first deferred step) and 32 bytes per step taken.
 */
#define FHASH_ADAM_DEFER_DEFAULT_ROWS (1ull << 25)
fhash_status fhash_set_adam_deferral(fhash_model* model, uint64_t min_level_rows, fhash_stream stream);

/* Measurement aid (no counterpart in the paper): with enable != 0, fhash_train_step records CUDA events
 * on its stream around its phases, read back by fhash_get_adam_stats. */
fhash_status fhash_set_timing(fhash_model* model, int32_t enable);

typedef struct {
    int32_t first_deferred_level;    /* -1 when no level is deferred */
    uint64_t deferred_params;        /* parameters in deferred groups */
    int64_t step, clean_step;        /* Adam steps taken; every deferred group is current at least at clean_step */
    uint64_t last_replayed_groups;   /* last training step: groups brought up to date before its gathers */
    uint64_t last_replayed_steps;    /* ... and the group-steps replayed for them */
    float last_ms[7];                /* with timing on, the last training step's phases (ms): claim and
                                        sort of the catch-up, its replay, the gathers (bf16: the fused
                                        forward), MLP forward + loss + backward, table scatter, weight
                                        gradients, dense Adam (with deferred levels: only the recording
                                        of the step's scalars; see last_side_ms) */
    uint32_t group_params;           /* parameters per deferral group (one stamp, caught up together) */
    float last_side_ms;              /* with timing on and deferred levels: the dense update of the levels
                                        below the deferred ones and the MLP, which a deferred step leaves to
                                        the next step; that step runs it on a second stream beside its
                                        replay and waits for it before its gathers.  0 otherwise */
} fhash_adam_stats;

/* Deferral state and the last training step's counters; synchronises with the last training step. */
fhash_status fhash_get_adam_stats(fhash_model* model, fhash_adam_stats* out);

/*
 * Feature-based coreset (Section 3.1).  The training samples are the vertices of the dilated feature
 * d_k at each key frame t_k (the occupancy the model built from the mask in fhash_build), each
 * labelled with the volume value there; the coreset is their union over the key frames.  The samples
 * stay on the device (12 bytes each) in key-frame order, then (z, y, x) order inside the Feature
 * Bounding Box, and replace any previous coreset of the model.
 *  volume: host or device float32 [nt][nz][ny][nx] (the build dimensions), read during the call only;
 *  key_frames: host int32 [n_key], strictly increasing time steps in [0, nt).
 *  count (host, may be NULL) receives the number of samples N.  Dimensions above 65535 are
 *  FHASH_EINVAL.  The call synchronises the stream.
 */
fhash_status fhash_coreset_build(fhash_model* model, const float* volume, const int32_t* key_frames, int32_t n_key,
                                 int64_t* count, fhash_stream stream);

/*
 * Batch `batch` of epoch `epoch` over the coreset.  Epoch e visits every sample once, in the order of a
 * keyed permutation pi_e of [0, N): a balanced 4-round Feistel network on k-bit integers
 * (k = max(2, ceil(log2 N)) rounded up to even; round function SplitMix64's output function of the
 * right half XOR round key r, keys r = 0..3 = SplitMix64 outputs 0..3 seeded with value `epoch` of
 * stream 400 of `seed`), applied again while the result is >= N.  The batch holds the samples at
 * positions batch*B .. batch*B + B - 1 of pi_e (fewer in the last batch; ceil(N / B) batches per
 * epoch).  Writes their FBB-normalised coordinates u = ((x - lo) / (S - 1), ..., t / (nt - 1)) in
 * float32 to coords (device [n][4]) and labels to target (device [n]), and n to *n_out (host, may be
 * NULL).  No coreset, B <= 0 or a batch past the end is FHASH_EINVAL.
 */
fhash_status fhash_coreset_batch(fhash_model* model, uint64_t seed, int64_t epoch, int64_t batch, int64_t batch_size,
                                 float* coords, float* target, int64_t* n_out, fhash_stream stream);

/* fhash_train_step on batch `batch` of epoch `epoch` of the coreset (as fhash_coreset_batch). */
fhash_status fhash_coreset_train_step(fhash_model* model, uint64_t seed, int64_t epoch, int64_t batch,
                                      int64_t batch_size, const fhash_adam* adam, double* loss, fhash_stream stream);

enum { FHASH_STATE_PARAM = 0, FHASH_STATE_GRAD = 1, FHASH_STATE_ADAM_M = 2, FHASH_STATE_ADAM_V = 3 };

/* Copy n float32 elements starting at flat element `offset` of a state vector ([table | MLP]
 * layout above) to / from `buf` (host or device).  Writing FHASH_STATE_PARAM refreshes the bf16
 * shadows of FHASH_BF16 models.  Offsets beyond the vector are FHASH_EINVAL. */
fhash_status fhash_read_state(fhash_model* model, int32_t which, uint64_t offset, uint64_t n, float* buf,
                              fhash_stream stream);
fhash_status fhash_write_state(fhash_model* model, int32_t which, uint64_t offset, uint64_t n, const float* buf,
                               fhash_stream stream);

/* Occupancy grid of time step t (Section 3.1) over the Feature Bounding Box as bytes 0/1,
 * out: host or device [Sz][Sy][Sx]. */
fhash_status fhash_read_occupancy(fhash_model* model, int64_t t, uint8_t* out, fhash_stream stream);

/* The rule FHASH_LAYOUT_MASKED builds with, for inspection (host only, no CUDA call): the vertices
 * [*lo, *hi] of a level axis with R vertices that the footprint of voxel v of the S voxels of the FBB
 * on that axis makes active (is_time = 0), or that time step v of S makes active (is_time = 1); see
 * the layout description above.  FHASH_EINVAL unless 0 <= v < S, 1 <= S <= 2^24 and 1 <= R <= 2^24. */
fhash_status fhash_active_range(int64_t v, int64_t S, int64_t R, int32_t is_time, int64_t* lo, int64_t* hi);

/* Active-vertex bits of level l of a FHASH_LAYOUT_MASKED model: word w holds the vertices with Eq. 9
 * rows 64w .. 64w+63 of the level (bit i = row 64w + i), words [word0, word0 + n_words) into `bits`
 * (host or device).  Synchronous for host buffers.  FHASH_EINVAL for another layout, a level out of
 * range or words past ceil(Rx*Ry*Rz*Rt / 64). */
fhash_status fhash_read_active(fhash_model* model, int32_t level, uint64_t word0, uint64_t n_words, uint64_t* bits,
                               fhash_stream stream);

/*
 * Checkpoints (the paper pretrains the INR before visualisation, Section 3.3).  fhash_save writes the
 * model description, level schedule, Feature Bounding Box, Adam step count, every state vector
 * (parameters, gradients, both Adam moments) and the occupancy grid to `path`; fhash_load rebuilds an
 * identical model on the current device (bf16 shadows recomputed).  Both are synchronous; the file is
 * specific to this library version and byte order.  Errors: FHASH_EIO for unreadable, truncated or
 * foreign files; FHASH_ENOMEM.
 */
fhash_status fhash_save(const fhash_model* model, const char* path);
fhash_status fhash_load(const char* path, fhash_stream stream, fhash_model** out);

/* Diagnostic of the failure path: launches one CTA that waits, with the bounded wait every
 * tensor-core kernel uses, on an mbarrier that nothing arrives on.  After limit_ns (at most 10 s) the
 * wait gives up, the kernel records the timeout in the model's device error word and returns; the
 * next fhash_check reports FHASH_EDEVICE.  Nothing traps or hangs.  Asynchronous. */
fhash_status fhash_diag_wait_timeout(fhash_model* model, uint64_t limit_ns, fhash_stream stream);

/* Measurement aid with no counterpart in the paper: the ceiling of the encoding's access pattern.
 * It performs n gathers of `width` bytes (4, 8 or 16) at uniformly random aligned positions of a
 * device table of `bytes` bytes (16-byte aligned), 8 independent loads in flight per thread, and adds
 * a float checksum into *sum (device).  Time it with events on `stream`: for a table that fits in L2
 * it gives the L2 random-gather rate, and for one far larger than L2 the HBM rate at 32-byte
 * sectors.  Asynchronous; bad arguments are FHASH_EINVAL. */
fhash_status fhash_diag_random_gather(const void* table, uint64_t bytes, int32_t width, int64_t n, uint64_t seed,
                                      float* sum, fhash_stream stream);

/* Synchronise `stream` and report FHASH_EDEVICE if a kernel of this model raised the device
 * error word since the last check (the word is then cleared). */
fhash_status fhash_check(fhash_model* model, fhash_stream stream);

/*
 * Camera of fhash_render, in the world space of the Feature Bounding Box scaled to [-1,1]^3
 * (Section 3.1, Eqs. 1-2).  Pixel (i, j) of a W x H image (row 0 at the top) looks from eye along
 * fwd + sx*right + sy*up with sx = (2i+1)/W - 1 and sy = 1 - (2j+1)/H; right and up already carry
 * the half extents of the image plane at unit distance (field of view and aspect ratio).
 */
typedef struct {
    float eye[3], right[3], up[3], fwd[3];
} fhash_camera;

typedef struct {
    int64_t rounds;             /* ARM rounds (Algorithm 1 iterations) */
    int64_t samples_evaluated;  /* sample slots sent through the encode+MLP kernel */
    int64_t samples_composited; /* samples used by compositing (before early termination) */
    int64_t steps_marched;      /* sample positions visited, occupied or not */
} fhash_render_stats;

/*
 * Render one image of the model at normalised time t_norm in [0,1] by sample streaming with
 * adaptive ray marching (Section 3.3, Algorithm 1).  Every round, each alive ray contributes up to
 * N_s = max(min(N_r / N_a, max_pace), 1) samples (N_r = w*h rays, N_a alive; the paper uses 64 as
 * the pace limit), all samples of the round go through the fused encode+MLP kernel in one launch,
 * then each ray applies the transfer function and composites front to back and leaves when it exits
 * the box or its opacity exceeds 0.99.  Samples lie at spacing 1/(S_max - 1) world units from the
 * box entry and are evaluated only where the occupancy grid (Section 3.1) is set at the nearest voxel
 * (at an unseen t: set at either neighbouring key frame).  The image does not depend on max_pace.
 *  tf: device [256][4] RGBA float32, indexed by the value clamped to [0,1] times 255 with linear
 *      interpolation; alpha is per sample (already corrected for the spacing).
 *  rgba: device [h][w][4] float32 = (accumulated colour, opacity); rays missing the box give 0.
 *  counts: device [h][w] int32 composited samples per pixel, or NULL.  stats: host, or NULL.
 * Synchronous.  Each round's kernels read the alive count from device memory, so rounds are issued
 * in batches of 1, 2, 4, ... up to 64 with one read-back of the alive count per batch instead of one
 * per round.
 */
fhash_status fhash_render(fhash_model* model, const fhash_camera* cam, float t_norm, const float* tf, int32_t w,
                          int32_t h, int32_t max_pace, float* rgba, int32_t* counts, fhash_render_stats* stats,
                          fhash_stream stream);

/* Points per axis of fhash_decode's grid: dims[a] = upsample * (S_a - 1) + 1, (x, y, z). */
fhash_status fhash_decode_dims(const fhash_model* model, int32_t upsample, int64_t dims[3]);

/*
 * Time-slice decode: the model evaluated on a regular grid over the Feature Bounding Box at
 * normalised time t_norm (any value in [0,1], including times between key frames: temporal
 * super-resolution, Section 3.3), upsample = 1..8 points per voxel edge.  Point (x, y, z) is
 * u = (x/(dims[0]-1), y/(dims[1]-1), z/(dims[2]-1), t_norm); out: device [dims[2]][dims[1]][dims[0]].
 */
fhash_status fhash_decode(fhash_model* model, float t_norm, int32_t upsample, float* out, fhash_stream stream);

/*
 * Gradient computation that allocates nothing (the paper has no counterpart to this call).
 *
 * Same result as fhash_compute_grads on float32 models (forward, MSE loss, backward, gradients added
 * to the model's gradient buffer); for FHASH_BF16 models, the float32-form loss and gradients of the
 * float32 master weights (fhash_compute_grads evaluates those models' bf16 forward).  Its working memory is a fixed array of FHASH_NOALLOC_SCRATCH_BYTES that the
 * library holds in device global memory from load to exit, on every GPU that loads it.  For callers
 * that cannot call cudaMalloc: for example an application that has handed all device memory to its
 * own pool, or a latency-critical loop that cannot afford the implicit device synchronisation of
 * cudaMalloc/cudaFree (fhash_compute_grads grows its scratch buffers with them).  This call makes no
 * cudaMalloc, cudaFree or other allocating call.
 *  - coords [n][4] and target [n] must be DEVICE memory (they are not staged); loss is host or
 *    device double* or NULL.
 *  - n must be in 1..FHASH_NOALLOC_MAX_SAMPLES; a model/n combination whose working set exceeds the
 *    array is rejected with FHASH_EINVAL before anything is launched.  FHASH_LAYOUT_MASKED models are
 *    rejected with FHASH_EINVAL (they take fhash_compute_grads).
 *  - The first call on a device, made with that device current, looks up the array's device address
 *    (cudaGetSymbolAddress) once and keeps it for the life of the process; make that first call
 *    before any stream capture.  cudaDeviceReset invalidates the kept address (the array may be
 *    reloaded elsewhere): do not call this entry point on a device after resetting it.
 *  - Every call shares the one array, which keeps the previous call's contents: every scratch byte
 *    this call reads it has written earlier in the same call, so nothing needs clearing, but calls
 *    that overlap on the GPU (other streams, other threads, other models) race and must be ordered
 *    by the caller.
 */
#define FHASH_NOALLOC_MAX_SAMPLES 4096
#define FHASH_NOALLOC_SCRATCH_BYTES (12u << 20)
fhash_status fhash_compute_grads_noalloc(fhash_model* model, const float* coords, const float* target, int64_t n,
                                         double* loss, fhash_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* FHASH_H */
