// Internal definitions shared by the library's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "fhash.h"

namespace fh {

// NVTX range around an entry point (header-only NVTX 3): visible to Nsight Systems and to
// `ncu --nvtx --nvtx-include`; without a tool attached each push and pop is a no-op call.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define FH_RANGE(name) ::fh::NvtxRange fh_nvtx_range_(name)


// ------------------------------------------------------------------ errors
fhash_status set_error(fhash_status s, const char* fmt, ...);
fhash_status cuda_error(cudaError_t e, const char* what);
#define FH_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::fh::cuda_error(e_, #call);      \
    } while (0)
#define FH_TRY(call)                                                    \
    do {                                                                \
        fhash_status s_ = (call);                                       \
        if (s_ != FHASH_OK) return s_;                                  \
    } while (0)

// ------------------------------------------------------------------ level table
// One level of the Tesseract grid.  Rows of the level: base + t*st + z*sz + y*sy + x (Eq. 9).
struct Level {
    int32_t R[4];     // vertices per axis (x, y, z, t)
    float Rm1[4];     // (float)(R - 1), the scale of the float32 cell step
    uint32_t sy, sz;  // Rx, Rx*Ry
    uint64_t st;      // Rx*Ry*Rz
    uint64_t base;    // first row of the level
    uint64_t nrows;   // rows of the level: Rx*Ry*Rz*Rt, or its active vertices (FHASH_LAYOUT_MASKED)
    const uint4* dir; // masked levels: per 64 Eq. 9 rows {active bits lo, hi, active rows before lo, hi}
    int32_t layout;   // FHASH_LAYOUT_LINEAR (Eq. 9), _BRICK (4x4x4 bricks per time slice) or _MASKED
};

struct Levels {
    int32_t L, F;
    Level lv[FHASH_MAX_LEVELS];
};

// MLP shape: dims[0] = L*F, dims[1..nh] = width, dims[nh+1] = 1.  Flat offsets into the MLP block.
struct MlpShape {
    int32_t in, width, nh;  // nh hidden layers
    int32_t n_params;
    int32_t w_off[FHASH_MAX_HIDDEN + 1], b_off[FHASH_MAX_HIDDEN + 1];
};

// ------------------------------------------------------------------ model
struct Scratch {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace fh

struct fhash_model {
    int device = 0;
    fhash_build_desc desc{};
    fh::Levels lv{};
    fh::MlpShape mlp{};
    uint64_t total_rows = 0, n_table = 0, n_params = 0;  // n_params = n_table + mlp params
    int64_t fbb_lo[3]{}, fbb_size[3]{};
    int64_t nt = 1;
    int64_t step = 0;

    // flat state vectors [n_params] float32 (table values then MLP)
    float* param = nullptr;
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* shadow = nullptr;  // bf16 copy of param (FHASH_BF16 only)

    // occupancy over the FBB: bricks of 8^3 voxels, 16 x u32 words each (Morton order inside)
    uint32_t* occ = nullptr;
    uint8_t* occ_any = nullptr;  // per brick: any bit set
    int64_t nbx = 0, nby = 0, nbz = 0;

    // FHASH_LAYOUT_MASKED: the active-vertex directories of all levels, one record per 64 Eq. 9 rows
    uint4* dir = nullptr;
    uint64_t dir_words = 0;

    int* err_word = nullptr;  // device error word (0 = ok)

    // scratch (grown on demand; owned by the model)
    fh::Scratch s_coords, s_target, s_out, s_acts, s_gacts, s_partial, s_loss, s_misc, s_render, s_enc;
    fh::Scratch s_cs_ent, s_cs_val;  // coreset samples: packed (x, y, z, t) and labels
    int64_t cs_n = 0;
    uint64_t device_bytes = 0;
    int32_t forward_path = 0;  // FHASH_FORWARD_* (precision form only)

    // deferred Adam (csrc/adam.cu): levels from defer_level on (those with at least defer_min_rows
    // rows) hold groups of 32 floats [defer_lo/32, defer_hi/32) of the flat vectors, each with a stamp: the
    // step its p, m, v are current at; every group is at least clean_step-current; dirty when some
    // group is behind `step`.
    uint64_t defer_min_rows = 1ull << 25;
    int32_t defer_level = -1;
    uint64_t defer_lo = 0, defer_hi = 0;
    uint64_t planned_lo = 0, planned_hi = 0;  // the range the last deferred step used (what a flush covers)
    uint32_t* stamp = nullptr;
    uint64_t stamp_groups = 0;
    int64_t clean_step = 0;
    bool dirty = false;
    void* adam_tab = nullptr;  // per-step Adam scalars, indexed by step
    int64_t adam_tab_cap = 0;
    fh::Scratch s_defer;       // counters, claim list and its bucket-sorted copy
    // the dense-range Adam update of step pend_k (hyper-parameters pend_ad) not run yet: the next
    // training step runs it on `side` beside its catch-up; anything else runs it first
    bool dense_pending = false;
    fhash_adam pend_ad{};
    int64_t pend_k = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    void* last_ctr = nullptr;  // counters of the last step's catch-up (device), or null
    // phase timing of fhash_train_step (fhash_set_timing): events at the phase boundaries fh::TEV_*
    bool timing = false, tev_init = false;
    cudaEvent_t tev[8]{};
    cudaEvent_t tev_side[2]{};  // around the dense-range update on `side`
    bool side_timed = false;    // the last training step recorded them
};

namespace fh {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output i of the generator seeded with s is
// mix(s + (i + 1) * gamma).
#define FH_GAMMA 0x9E3779B97F4A7C15ULL
__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm_at(uint64_t seed, uint64_t i) { return sm_mix(seed + (i + 1) * FH_GAMMA); }

// Phase boundaries of a training step, recorded on its stream when timing is on: start, after the
// claim and sort of the deferred catch-up, after its replay, after the gathers (the fused forward in
// the precision form), after the MLP forward, loss and backward, after the table scatter, after the
// weight gradients, after Adam.
enum { TEV_START = 0, TEV_CLAIM, TEV_REPLAY, TEV_ENCODE, TEV_MLP, TEV_SCATTER, TEV_DW, TEV_ADAM, TEV_N };
inline void tev_record(fhash_model* m, int i, cudaStream_t st) {
    if (m->timing) cudaEventRecord(m->tev[i], st);
}

fhash_status grow(fhash_model* m, Scratch& s, size_t bytes);
bool is_device_ptr(const void* p);
// Copies a host-or-device input into `s` when it is host memory; returns the device pointer to use.
fhash_status stage_in(fhash_model* m, Scratch& s, const void* p, size_t bytes, cudaStream_t st, const void** dev);

// ------------------------------------------------------------------ device helpers
// Float32 cell step (Section 3.2.4 steps 1-2): c = clamp(floor(u*(R-1)), 0, R-2), w = u*(R-1) - c,
// upper corner min(c+1, R-1).  u is clamped to [0,1] first, NaN -> 0.  Round-to-nearest multiply,
// no contraction, so rows are bit-identical to any IEEE float32 evaluation of the same steps.
__device__ __forceinline__ void cell(float u, int R, float Rm1, int& c, int& d1, float& w) {
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    float p = __fmul_rn(u, Rm1);
    int ci = (int)floorf(p);
    ci = min(ci, R - 2);
    ci = max(ci, 0);
    w = __fsub_rn(p, (float)ci);
    c = ci;
    d1 = (ci + 1 <= R - 1) ? 1 : 0;  // 0 only on single-vertex axes
}

// Per-level corner geometry of one sample: base row (lower corner at t_Previous), the row offsets of
// the upper corners on each axis, and the four axis fractions.  In the brick layout r0 is the first
// row of the t_Previous slice, ot the slice stride or 0, ox/oy/oz the upper-corner steps (1 or 0) and
// (cx, cy, cz) the lower cell corner; corner rows then come from brick_row3.
struct Corners {
    uint64_t r0;
    uint32_t ox, oy, oz;
    uint64_t ot;
    float wx, wy, wz, wt;
    uint32_t layout, cx, cy, cz, Rx, Ry, Rz;
    const uint4* dir;  // masked levels: r0 is the Eq. 9 row within the level, mapped through dir
    uint64_t mbase;
};

// Row returned for an inactive corner of a masked level: it reads 0 and takes no gradient.
constexpr uint64_t kInactiveRow = ~0ull;

// Row of the vertex with Eq. 9 row r (within a masked level): the level's base plus the number of
// active rows before r (the record's prefix count and a popcount inside its 64-row word), or
// kInactiveRow when the vertex is not active.
__device__ __forceinline__ uint64_t masked_row(const uint4* __restrict__ dir, uint64_t base, uint64_t r) {
    const uint4 d = __ldg(dir + (r >> 6));
    const uint64_t bits = ((uint64_t)d.y << 32) | d.x;
    const uint32_t i = (uint32_t)r & 63u;
    if (!((bits >> i) & 1ull)) return kInactiveRow;
    return base + ((((uint64_t)d.w) << 32) | d.z) + (uint64_t)__popcll(bits & ((1ull << i) - 1ull));
}

// Row of vertex (x, y, z) inside a time slice in the brick layout (Section 3.2.3 allows other
// linearisations than Eq. 9): 4x4x4 bricks in (bz, by, bx) order, vertices in (iz, iy, ix) order
// inside a brick, bricks narrower at the high end of an axis (w = min(4, R - 4b)); a bijection onto
// [0, Rx*Ry*Rz).  The build keeps Rx*Ry*Rz below 2^32.
__device__ __forceinline__ uint32_t brick_row3(uint32_t x, uint32_t y, uint32_t z, uint32_t Rx, uint32_t Ry, uint32_t Rz) {
    const uint32_t bx = x >> 2, by = y >> 2, bz = z >> 2;
    const uint32_t wx = min(4u, Rx - 4u * bx), wy = min(4u, Ry - 4u * by), wz = min(4u, Rz - 4u * bz);
    return 4u * bz * Rx * Ry + wz * (4u * by * Rx + wy * 4u * bx) + ((z & 3u) * wy + (y & 3u)) * wx + (x & 3u);
}

// Rows of the x-neighbours with Eq. 9 rows r and r + ox (ox = 0 or 1) of a masked level, from one
// directory record unless r + 1 starts the next 64-row word.  The rank of r + 1 is that of r plus one
// when r is active.
__device__ __forceinline__ void masked_pair(const uint4* __restrict__ dir, uint64_t base, uint64_t r, uint32_t ox,
                                            uint64_t& a, uint64_t& b) {
    const uint4 d = __ldg(dir + (r >> 6));
    const uint64_t bits = ((uint64_t)d.y << 32) | d.x;
    const uint32_t i = (uint32_t)r & 63u;
    const uint64_t at = base + ((((uint64_t)d.w) << 32) | d.z) + (uint64_t)__popcll(bits & ((1ull << i) - 1ull));
    const bool act0 = (bits >> i) & 1ull;
    a = act0 ? at : kInactiveRow;
    if (ox == 0u) {
        b = a;
    } else if (i < 63u) {
        b = ((bits >> (i + 1u)) & 1ull) ? at + (act0 ? 1ull : 0ull) : kInactiveRow;
    } else {
        b = masked_row(dir, base, r + 1);
    }
}

// LAYOUT: 0 = Eq. 9, 1 = bricks, 2 = masked, -1 = read from the level (kernels over one level per thread
// take the runtime form; kernels that walk all levels of a sample are instantiated per layout, so that
// no branch sits between the gathers of consecutive levels).
template <int LAYOUT = -1>
__device__ __forceinline__ Corners corners(const Level& L, float4 u) {
    int cx, cy, cz, ct, dx, dy, dz, dt;
    Corners k;
    cell(u.x, L.R[0], L.Rm1[0], cx, dx, k.wx);
    cell(u.y, L.R[1], L.Rm1[1], cy, dy, k.wy);
    cell(u.z, L.R[2], L.Rm1[2], cz, dz, k.wz);
    cell(u.w, L.R[3], L.Rm1[3], ct, dt, k.wt);
    k.ot = dt ? L.st : 0ull;
    const int lay = LAYOUT < 0 ? L.layout : LAYOUT;
    k.layout = (uint32_t)lay;
    k.dir = L.dir;
    k.mbase = L.base;
    if (lay == 1) {
        k.r0 = L.base + (uint64_t)ct * L.st;
        k.ox = dx; k.oy = dy; k.oz = dz;
        k.cx = cx; k.cy = cy; k.cz = cz;
        k.Rx = L.R[0]; k.Ry = L.R[1]; k.Rz = L.R[2];
    } else {
        k.r0 = (lay == 2 ? 0ull : L.base) + (uint64_t)ct * L.st + (uint64_t)cz * L.sz + (uint64_t)cy * L.sy + (uint64_t)cx;
        k.ox = dx;
        k.oy = dy ? L.sy : 0u;
        k.oz = dz ? L.sz : 0u;
        k.cx = k.cy = k.cz = k.Rx = k.Ry = k.Rz = 0;
    }
    return k;
}

// Row of corner c = i + 2j + 4k + 8s (i, j, k: upper corner on x, y, z; s = 1 for t_Next); kInactiveRow
// for an inactive corner of a masked level.
template <int LAYOUT = -1>
__device__ __forceinline__ uint64_t corner_row(const Corners& k, int c) {
    const int lay = LAYOUT < 0 ? (int)k.layout : LAYOUT;
    if (lay == 1)
        return k.r0 + ((c & 8) ? k.ot : 0ull) +
               brick_row3(k.cx + ((c & 1) ? k.ox : 0u), k.cy + ((c & 2) ? k.oy : 0u), k.cz + ((c & 4) ? k.oz : 0u),
                          k.Rx, k.Ry, k.Rz);
    const uint64_t r = k.r0 + ((c & 8) ? k.ot : 0ull) + ((c & 4) ? k.oz : 0u) + ((c & 2) ? k.oy : 0u) + ((c & 1) ? k.ox : 0u);
    if (lay == 2) return masked_row(k.dir, k.mbase, r);
    return r;
}

// Rows of corners c (even: lower x) and c + 1 (upper x) of a masked level: one directory record per pair.
__device__ __forceinline__ void masked_corner_pair(const Corners& k, int c, uint64_t& a, uint64_t& b) {
    const uint64_t r = k.r0 + ((c & 8) ? k.ot : 0ull) + ((c & 4) ? k.oz : 0u) + ((c & 2) ? k.oy : 0u);
    masked_pair(k.dir, k.mbase, r, k.ox, a, b);
}

__device__ __forceinline__ void raise_error(int* word, int code) {
    if (word) atomicCAS(word, 0, code);
}

// Vector reductions to global memory (no return value); addresses aligned to the vector size.
__device__ __forceinline__ void red_add(float* a, float v) { atomicAdd(a, v); }
__device__ __forceinline__ void red_add2(float* a, float x, float y) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(a), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ void red_add4(float* a, float x, float y, float z, float w) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(x), "f"(y), "f"(z), "f"(w)
                 : "memory");
}

inline int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// ------------------------------------------------------------------ launchers (encode.cu)
fhash_status launch_lookup(fhash_model* m, const float* coords, int64_t n, uint64_t* rows, float* w, cudaStream_t st);
fhash_status launch_encode(fhash_model* m, const float* coords, int64_t n, float* enc, cudaStream_t st);
fhash_status launch_forward(fhash_model* m, const float* coords, int64_t n, float* out, cudaStream_t st);
// Precision form, split evaluation: bf16 encoding rows, then the TMA-fed tensor-core MLP (csrc/mlp_split.cu).
fhash_status launch_forward_split(fhash_model* m, const float* coords, int64_t n, float* out, cudaStream_t st);
fhash_status launch_forward_seg(fhash_model* m, const float* coords, float* out, const int64_t* seg, int64_t max_n,
                                cudaStream_t st);
// Forward + loss + backward into the gradient buffer (csrc/train.cu).
fhash_status launch_grads2(fhash_model* m, const float* coords, const float* target, int64_t n, double* loss_dev,
                           cudaStream_t st);
// Table-gradient scatter of the encoding alone, d(encoding) row-major [n][L*F] (csrc/train.cu).
fhash_status launch_encode_backward(fhash_model* m, const float* coords, int64_t n, const float* denc, cudaStream_t st);
fhash_status launch_adam(fhash_model* m, const fhash_adam* a, cudaStream_t st);
// Training step (forward, loss, backward, Adam), deferred where the model has deferred levels (csrc/adam.cu).
fhash_status launch_train_step(fhash_model* m, const float* coords, const float* target, int64_t n,
                               const fhash_adam* a, double* loss_dev, cudaStream_t st);
// Brings every deferred group to the current step; a no-op unless a deferred training step left some
// behind.  Every entry point that reads or writes the model's state outside fhash_train_step calls it.
fhash_status settle_deferred(fhash_model* m, cudaStream_t st);
fhash_status refresh_shadow(fhash_model* m, uint64_t off, uint64_t n, cudaStream_t st);

}  // namespace fh
