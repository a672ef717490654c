// Adam (Section 5.1.3; PyTorch semantics: dense, bias-corrected, eps added outside the square root, no
// weight decay) in two forms with bit-identical results.
//
// Dense: k_adam streams every parameter once per step (28 bytes per parameter; HBM-bound).
//
// Deferred: a step whose gradient is zero is a fixed float32 map of (p, m, v) that depends only on
// that step's scalars (beta1, beta2, lr / bc1, 1 / sqrt(bc2), eps).  For the table levels whose rows a
// batch rarely touches (the HBM-resident fine levels), that map is not applied every step: each group
// of kGroup consecutive floats keeps a stamp s, meaning "p, m, v are current at step s and the gradient buffer holds
// the gradient of step s + 1".  Before the gathers of step k, every group the batch will read is
// brought to step k - 1 by replaying, with the same float32 operations in the same order, step s + 1
// with its pending gradient and steps s + 2 .. k - 1 with a zero gradient (the scalars of every step
// are kept in a small device table); the step's backward then adds its gradient, which stays pending.
// Coarse levels, the level boundaries and the MLP take the dense update every step.  Anything that
// reads or writes the state outside the training step first replays every group to the current step
// (settle_deferred), so no caller can observe the difference.
//
// Work of a deferred step: claim (one atomicMax per touched group decides which thread replays it),
// a counting sort of the claimed groups by replay length (so a warp's lanes loop the same number of
// times), the replay, then the usual gradient pass and the dense update of the rest.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "kernels.cuh"

namespace fh {

// One step's scalars: beta1, 1 - beta1, beta2, 1 - beta2, -lr / bc1, 1 / sqrt(bc2) (bc = 1 - beta^k; both
// computed in double and rounded once), eps.
struct AdamScal {
    float b1, omb1, b2, omb2, neg_step, inv_sqrt_bc2, eps, pad;
};

// The GPU's approximate square root and division (one special-function instruction each, relative error
// of a few ulp), in place of the correctly rounded sequences, which cost several times more issue slots
// and left Adam's arithmetic, not its memory traffic, as the limit of the replay.  Deterministic: the same
// inputs give the same bits in every kernel.
// Subnormal inputs are flushed to zero here: a subnormal v gives sqrt(v) below 1e-19, far under eps, and a
// subnormal m an update below 1e-30 lr; either way the step is unchanged at float32 precision.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float div_approx(float x, float y) {
    float q;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(q) : "f"(x), "f"(y));
    return q;
}

// One Adam step of one parameter:
//   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;  p = p - (lr / bc1) m / (sqrt(v) / sqrt(bc2) + eps),
// every multiply-add rounded to nearest with no further contraction, so the same call gives the same bits
// wherever it is compiled (the dense kernel, the replay, the flush).
__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, const AdamScal& s) {
    m = __fmaf_rn(s.b1, m, __fmul_rn(s.omb1, g));
    v = __fmaf_rn(s.b2, v, __fmul_rn(s.omb2, __fmul_rn(g, g)));
    const float denom = __fmaf_rn(sqrt_approx(v), s.inv_sqrt_bc2, s.eps);
    p = __fmaf_rn(s.neg_step, div_approx(m, denom), p);
}

// adam1 with g = +0, bit for bit: (1 - beta) is positive and finite, so (1 - beta) * (+0) and
// (1 - beta) * (+0)^2 are +0 and the fused multiply-adds receive the same +0 addend.  Saves the two
// multiplies by the zero gradient in the replay of steps without a gradient.
__device__ __forceinline__ void adam1_zero(float& p, float& m, float& v, const AdamScal& s) {
    m = __fmaf_rn(s.b1, m, 0.0f);
    v = __fmaf_rn(s.b2, v, 0.0f);
    const float denom = __fmaf_rn(sqrt_approx(v), s.inv_sqrt_bc2, s.eps);
    p = __fmaf_rn(s.neg_step, div_approx(m, denom), p);
}

__device__ __forceinline__ void adam4_zero(float4& p, float4& m, float4& v, const AdamScal& s) {
    adam1_zero(p.x, m.x, v.x, s);
    adam1_zero(p.y, m.y, v.y, s);
    adam1_zero(p.z, m.z, v.z, s);
    adam1_zero(p.w, m.w, v.w, s);
}

__device__ __forceinline__ void adam4(float4& p, const float4& g, float4& m, float4& v, const AdamScal& s) {
    adam1(p.x, g.x, m.x, v.x, s);
    adam1(p.y, g.y, m.y, v.y, s);
    adam1(p.z, g.z, m.z, v.z, s);
    adam1(p.w, g.w, m.w, v.w, s);
}

// Dense update of n parameters (one thread per float4, plus one per leftover parameter): streams p, g,
// m, v once, 16 bytes read + 12 written per parameter (+2 for the bf16 shadow); the gradient is cleared
// by writing zeros only where it is not zero already (a step's scatter touches few table rows, and
// untouched sectors then cost no DRAM write).  With tab != nullptr the step's scalars are recorded at
// tab[k] for later replays.
template <bool SHADOW>
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ P, float* __restrict__ G, float* __restrict__ M,
                                              float* __restrict__ V, uint64_t n, const AdamScal s,
                                              __nv_bfloat16* __restrict__ shadow, AdamScal* __restrict__ tab,
                                              int64_t k) {
    if (tab && blockIdx.x == 0 && threadIdx.x == 0) tab[k] = s;
    const uint64_t n4 = n / 4;
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n4) {
        float4* P4 = reinterpret_cast<float4*>(P);
        float4* G4 = reinterpret_cast<float4*>(G);
        float4* M4 = reinterpret_cast<float4*>(M);
        float4* V4 = reinterpret_cast<float4*>(V);
        float4 p = __ldcs(P4 + i), g = __ldcs(G4 + i), m = __ldcs(M4 + i), v = __ldcs(V4 + i);
        const bool touched = (g.x != 0.0f) | (g.y != 0.0f) | (g.z != 0.0f) | (g.w != 0.0f);
        adam4(p, g, m, v, s);
        __stcs(P4 + i, p);
        if (touched) __stcs(G4 + i, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
        __stcs(M4 + i, m);
        __stcs(V4 + i, v);
        if (SHADOW) {
            __nv_bfloat162* s2 = reinterpret_cast<__nv_bfloat162*>(shadow) + 2 * i;
            s2[0] = __floats2bfloat162_rn(p.x, p.y);
            s2[1] = __floats2bfloat162_rn(p.z, p.w);
        }
    } else if (i - n4 < n - 4 * n4) {
        const uint64_t e = 4 * n4 + (i - n4);
        float p = P[e], m = M[e], v = V[e];
        adam1(p, G[e], m, v, s);
        P[e] = p; M[e] = m; V[e] = v;
        G[e] = 0.0f;
        if (SHADOW) shadow[e] = __float2bfloat16_rn(p);
    }
}

// ------------------------------------------------------------------ deferred form
// Floats per deferral group (one stamp each; a claim catches up the whole group).  32 floats = one
// 128-byte line of each state vector: a batch's corners then fall into about half as many groups as
// with 8-float groups, and the replay's random accesses (p, g, m, v read, p, m, v, g written) move whole
// lines, which a random access costs nearly the same as one sector.  kLanes lanes replay a group, 8
// floats each.
constexpr uint32_t kGroup = 32;
constexpr uint32_t kLanes = kGroup / 8;
constexpr int kBuckets = 64;

// Counters of one deferred step (device memory, cleared before the claim).
struct DeferCtr {
    uint32_t count;              // groups claimed for replay
    uint32_t hist[kBuckets];     // per replay-length bucket
    uint32_t cursor[kBuckets];   // placement cursors of the counting sort
    uint32_t pad;
    unsigned long long steps;    // replayed group-steps (sum of replay lengths)
};

// Quarter-octave bucket of a replay length >= 1: 4 floor(log2 len) + the next two bits.
__device__ __forceinline__ uint32_t len_bucket(uint32_t len) {
    const uint32_t e = 31u - __clz(len);
    const uint32_t frac = e >= 2u ? (len >> (e - 2u)) & 3u : (len << (2u - e)) & 3u;
    return min(4u * e + frac, (uint32_t)kBuckets - 1u);
}

struct DeferArgs {
    uint32_t* stamp;     // per group of the deferred range
    uint64_t q0, q1;     // deferred groups [q0, q1) (group q = floats kGroup q .. kGroup q + kGroup - 1)
    uint32_t target;     // k - 1: the step every read group must reach
    uint32_t clean;      // every group is at least this current
    int32_t l0;          // first deferred level
    uint2* items;        // claimed groups {q - q0, replay start s}
    DeferCtr* ctr;
};

// One thread per (deferred level, sample): the 16 corner rows of the sample's cell (Eq. 9 or the
// model's layout), their groups, and one atomicMax per distinct group.  The thread that raises a stamp
// below k - 1 replays that group; it appends {group, start} to the claim list (block-aggregated).
template <int F, int LAYOUT>
__global__ void __launch_bounds__(256) k_defer_claim(const __grid_constant__ Levels lv, const float* __restrict__ coords,
                                                     int64_t n, const DeferArgs d) {
    __shared__ uint32_t sh_hist[kBuckets];
    __shared__ uint32_t warp_off[8];
    __shared__ uint32_t blk_base;
    __shared__ unsigned long long blk_steps;
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) sh_hist[i] = 0;
    if (threadIdx.x == 0) blk_steps = 0;
    __syncthreads();
    const int nd = lv.L - d.l0;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    uint32_t q[16], st[16];
    bool ok[16];
    uint32_t cnt = 0, steps = 0;
#pragma unroll
    for (int c = 0; c < 16; ++c) ok[c] = false;
    if (idx < n * nd) {
        const int l = d.l0 + (int)(idx / n);
        const int64_t s = idx - (int64_t)(l - d.l0) * n;
        const Corners k = corners<LAYOUT>(lv.lv[l], load_coord(coords, s));
        uint64_t prev = ~0ull;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const uint64_t r = corner_row<LAYOUT>(k, c);
            if (LAYOUT == 2 && r == kInactiveRow) continue;
            const uint64_t g = (r * (uint64_t)F) / kGroup;
            if (g == prev || g < d.q0 || g >= d.q1) continue;
            prev = g;
            const uint32_t old = atomicMax(d.stamp + (g - d.q0), d.target);
            if (old < d.target) {
                const uint32_t from = max(old, d.clean);
                if (from < d.target) {
                    ok[c] = true;
                    q[c] = (uint32_t)(g - d.q0);
                    st[c] = from;
                    ++cnt;
                    steps += d.target - from;
                    atomicAdd(&sh_hist[len_bucket(d.target - from)], 1u);
                }
            }
        }
    }
    // block-aggregated append: warp scan of the per-thread counts, one global atomic per block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_off[warp] = incl;
    unsigned long long ws = steps;
#pragma unroll
    for (int o = 16; o; o >>= 1) ws += __shfl_down_sync(0xffffffffu, ws, o);
    if (lane == 0 && ws) atomicAdd(&blk_steps, ws);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const uint32_t x = warp_off[w];
            warp_off[w] = t;
            t += x;
        }
        blk_base = t ? atomicAdd(&d.ctr->count, t) : 0u;
        if (blk_steps) atomicAdd(&d.ctr->steps, blk_steps);
    }
    __syncthreads();
    uint32_t pos = blk_base + warp_off[warp] + incl - cnt;
#pragma unroll
    for (int c = 0; c < 16; ++c)
        if (ok[c]) d.items[pos++] = make_uint2(q[c], st[c]);
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
        if (sh_hist[i]) atomicAdd(&d.ctr->hist[i], sh_hist[i]);
}

// Counting sort of the claim list by replay-length bucket (order inside a bucket is arbitrary).  A block
// of 256 threads takes 256 kBinPer items, so few blocks contend for the 64 bucket cursors.
constexpr int kBinPer = 8;
__global__ void __launch_bounds__(256) k_defer_bin(const uint2* __restrict__ items, uint2* __restrict__ binned,
                                                   DeferCtr* __restrict__ ctr, uint32_t target) {
    static_assert(kBuckets == 64, "the offset scan below takes two warps");
    __shared__ uint32_t off[kBuckets], loc[kBuckets], base[kBuckets];
    __shared__ uint32_t w0;
    const uint32_t n = ctr->count;
    const uint32_t i0 = blockIdx.x * (256u * kBinPer);
    if (i0 >= n) return;  // the grid is sized for the largest possible list
    // bucket offsets: exclusive prefix sum of the histogram, one bucket per thread of the first two warps
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < kBuckets) {
        const uint32_t hv = ctr->hist[threadIdx.x];
        uint32_t inc = hv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        off[threadIdx.x] = inc - hv;
        loc[threadIdx.x] = 0;
        if (threadIdx.x == 31) w0 = inc;
    }
    __syncthreads();
    if (threadIdx.x >= 32 && threadIdx.x < kBuckets) off[threadIdx.x] += w0;
    uint2 it[kBinPer];
    uint32_t bk[kBinPer], rk[kBinPer];
#pragma unroll
    for (int k = 0; k < kBinPer; ++k) {
        const uint32_t i = i0 + k * 256u + threadIdx.x;
        if (i < n) {
            it[k] = items[i];
            bk[k] = len_bucket(target - it[k].y);
            rk[k] = atomicAdd(&loc[bk[k]], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < kBuckets && loc[threadIdx.x]) base[threadIdx.x] = atomicAdd(&ctr->cursor[threadIdx.x], loc[threadIdx.x]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBinPer; ++k) {
        const uint32_t i = i0 + k * 256u + threadIdx.x;
        if (i < n) binned[off[bk[k]] + base[bk[k]] + rk[k]] = it[k];
    }
}

// Replays steps from + 1 .. to of the 8 floats starting at float index f: the first with the
// pending gradient, the rest with a zero gradient; clears the gradient (where it is not zero already)
// and refreshes the bf16 shadow.
template <bool SHADOW>
__device__ __forceinline__ void replay_group(float* __restrict__ P, float* __restrict__ G, float* __restrict__ M,
                                             float* __restrict__ V, __nv_bfloat16* __restrict__ shadow, uint64_t f,
                                             uint32_t from, uint32_t to, const AdamScal* __restrict__ tab) {
    float4* P4 = reinterpret_cast<float4*>(P + f);
    float4* G4 = reinterpret_cast<float4*>(G + f);
    float4* M4 = reinterpret_cast<float4*>(M + f);
    float4* V4 = reinterpret_cast<float4*>(V + f);
    float4 p0 = P4[0], p1 = P4[1], m0 = M4[0], m1 = M4[1], v0 = V4[0], v1 = V4[1];
    const float4 g0 = G4[0], g1 = G4[1];
    const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    {
        const AdamScal s = tab[from + 1];
        adam4(p0, g0, m0, v0, s);
        adam4(p1, g1, m1, v1, s);
    }
    if (from + 2 <= to) {
        // the next step's scalars are loaded while this step's eight independent chains run
        AdamScal sn = tab[from + 2];
#pragma unroll 1
        for (uint32_t j = from + 2; j < to; ++j) {
            const AdamScal s = sn;
            sn = tab[j + 1];
            adam4_zero(p0, m0, v0, s);
            adam4_zero(p1, m1, v1, s);
        }
        adam4_zero(p0, m0, v0, sn);
        adam4_zero(p1, m1, v1, sn);
    }
    P4[0] = p0; P4[1] = p1;
    M4[0] = m0; M4[1] = m1;
    V4[0] = v0; V4[1] = v1;
    const bool touched = (g0.x != 0.0f) | (g0.y != 0.0f) | (g0.z != 0.0f) | (g0.w != 0.0f) | (g1.x != 0.0f) |
                         (g1.y != 0.0f) | (g1.z != 0.0f) | (g1.w != 0.0f);
    if (touched) { G4[0] = z; G4[1] = z; }
    if (SHADOW) {
        __nv_bfloat162* s2 = reinterpret_cast<__nv_bfloat162*>(shadow + f);
        s2[0] = __floats2bfloat162_rn(p0.x, p0.y);
        s2[1] = __floats2bfloat162_rn(p0.z, p0.w);
        s2[2] = __floats2bfloat162_rn(p1.x, p1.y);
        s2[3] = __floats2bfloat162_rn(p1.z, p1.w);
    }
}

// The claimed groups in bucket order, kLanes consecutive threads per group, 8 floats each (a persistent
// grid walks the list).
template <bool SHADOW>
__global__ void __launch_bounds__(256, 3) k_defer_replay(const uint2* __restrict__ binned, const DeferCtr* __restrict__ ctr,
                                                      float* __restrict__ P, float* __restrict__ G, float* __restrict__ M,
                                                      float* __restrict__ V, __nv_bfloat16* __restrict__ shadow,
                                                      uint64_t f0, const AdamScal* __restrict__ tab, uint32_t target) {
    const uint64_t n = (uint64_t)ctr->count * kLanes;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 it = binned[i / kLanes];
        replay_group<SHADOW>(P, G, M, V, shadow, f0 + (uint64_t)kGroup * it.x + 8 * (i % kLanes), it.y, target, tab);
    }
}

// Every deferred group brought to step k (before anything outside the training step reads the state).
template <bool SHADOW>
__global__ void __launch_bounds__(256, 3) k_defer_flush(const uint32_t* __restrict__ stamp, uint64_t ngroups,
                                                     float* __restrict__ P, float* __restrict__ G, float* __restrict__ M,
                                                     float* __restrict__ V, __nv_bfloat16* __restrict__ shadow,
                                                     uint64_t f0, const AdamScal* __restrict__ tab, uint32_t clean,
                                                     uint32_t k) {
    const uint64_t n = ngroups * kLanes;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = i / kLanes;
        const uint32_t from = max(stamp[q], clean);
        if (from < k) replay_group<SHADOW>(P, G, M, V, shadow, f0 + (uint64_t)kGroup * q + 8 * (i % kLanes), from, k, tab);
    }
}

// ------------------------------------------------------------------ host side
static AdamScal scalars(const fhash_adam* ad, int64_t step) {
    const double k = (double)step;
    const double bc1 = 1.0 - pow((double)ad->beta1, k), bc2 = 1.0 - pow((double)ad->beta2, k);
    AdamScal s{};
    s.b1 = ad->beta1;
    s.omb1 = (float)(1.0 - (double)ad->beta1);
    s.b2 = ad->beta2;
    s.omb2 = (float)(1.0 - (double)ad->beta2);
    s.neg_step = (float)(-(double)ad->lr / bc1);
    s.inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
    s.eps = ad->eps;
    return s;
}

// Dense update of n parameters from flat offset off (a multiple of 4).
__global__ void k_set_tab(AdamScal* tab, int64_t k, const AdamScal s) { tab[k] = s; }

static cudaError_t dense_range(fhash_model* m, uint64_t off, uint64_t n, const AdamScal& s, AdamScal* tab, int64_t k,
                               cudaStream_t st) {
    if (n == 0) {
        if (tab) k_set_tab<<<1, 1, 0, st>>>(tab, k, s);
        return cudaGetLastError();
    }
    // one thread per float4 (plus one per leftover parameter), no grid-stride loop: measured fastest on
    // GB300 at this size (every thread issues its four 16-byte loads at once)
    const uint64_t n4 = n / 4, threads = n4 + (n - 4 * n4);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, (threads + 255) / 256);
    if (m->shadow)
        k_adam<true><<<grid, 256, 0, st>>>(m->param + off, m->grad + off, m->adam_m + off, m->adam_v + off, n, s,
                                           m->shadow + off, tab, k);
    else
        k_adam<false><<<grid, 256, 0, st>>>(m->param + off, m->grad + off, m->adam_m + off, m->adam_v + off, n, s,
                                            nullptr, tab, k);
    return cudaGetLastError();
}

fhash_status launch_adam(fhash_model* m, const fhash_adam* ad, cudaStream_t st) {
    FH_TRY(settle_deferred(m, st));
    m->step += 1;
    FH_CUDA(dense_range(m, 0, m->n_params, scalars(ad, m->step), nullptr, m->step, st));
    m->clean_step = m->step;
    return FHASH_OK;
}

// Levels from the first one whose rows (and every finer level's) reach min_rows; the deferred range is
// the kGroup-float groups wholly inside those levels' tables.
static void plan_deferral(fhash_model* m) {
    m->defer_level = -1;
    m->defer_lo = m->defer_hi = 0;
    if (m->defer_min_rows == 0) return;
    int l0 = m->lv.L;
    while (l0 > 0 && m->lv.lv[l0 - 1].nrows >= m->defer_min_rows) --l0;
    if (l0 >= m->lv.L) return;
    const uint64_t F = (uint64_t)m->lv.F;
    const uint64_t lo = (m->lv.lv[l0].base * F + kGroup - 1) / kGroup * kGroup, hi = m->n_table / kGroup * kGroup;
    if (lo >= hi) return;
    m->defer_level = l0;
    m->defer_lo = lo;
    m->defer_hi = hi;
}

static fhash_status ensure_tab(fhash_model* m, int64_t k) {
    if (k < m->adam_tab_cap) return FHASH_OK;
    int64_t cap = std::max<int64_t>(4096, m->adam_tab_cap);
    while (cap <= k) cap *= 2;
    void* p = nullptr;
    FH_CUDA(cudaMalloc(&p, (size_t)cap * sizeof(AdamScal)));
    if (m->adam_tab) {
        FH_CUDA(cudaMemcpy(p, m->adam_tab, (size_t)m->adam_tab_cap * sizeof(AdamScal), cudaMemcpyDeviceToDevice));
        cudaFree(m->adam_tab);
    }
    m->adam_tab = p;
    m->adam_tab_cap = cap;
    m->device_bytes += (size_t)cap * sizeof(AdamScal);
    return FHASH_OK;
}

// The pending dense-range update (levels below the deferred ones and the MLP) of step pend_k, on st.
static fhash_status apply_pending_dense(fhash_model* m, cudaStream_t st) {
    const AdamScal s = scalars(&m->pend_ad, m->pend_k);
    FH_CUDA(dense_range(m, 0, m->planned_lo, s, nullptr, m->pend_k, st));
    FH_CUDA(dense_range(m, m->planned_hi, m->n_params - m->planned_hi, s, nullptr, m->pend_k, st));
    m->dense_pending = false;
    return FHASH_OK;
}

// The pending dense-range update on the side stream, after everything issued on st so far; ev_join marks
// its end.
static fhash_status fork_pending_dense(fhash_model* m, cudaStream_t st) {
    if (!m->side) {
        FH_CUDA(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
        FH_CUDA(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
        FH_CUDA(cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming));
    }
    FH_CUDA(cudaEventRecord(m->ev_fork, st));
    FH_CUDA(cudaStreamWaitEvent(m->side, m->ev_fork, 0));
    if (m->timing) FH_CUDA(cudaEventRecord(m->tev_side[0], m->side));
    FH_TRY(apply_pending_dense(m, m->side));
    if (m->timing) FH_CUDA(cudaEventRecord(m->tev_side[1], m->side));
    m->side_timed = m->timing;
    FH_CUDA(cudaEventRecord(m->ev_join, m->side));
    return FHASH_OK;
}

fhash_status settle_deferred(fhash_model* m, cudaStream_t st) {
    if (m->dense_pending) FH_TRY(apply_pending_dense(m, st));
    if (!m->dirty) return FHASH_OK;
    const uint64_t ng = (m->planned_hi - m->planned_lo) / kGroup;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((ng * kLanes + 255) / 256, (uint64_t)num_sms() * 64));
    const AdamScal* tab = (const AdamScal*)m->adam_tab;
    if (m->shadow)
        k_defer_flush<true><<<grid, 256, 0, st>>>(m->stamp, ng, m->param, m->grad, m->adam_m, m->adam_v, m->shadow,
                                                  m->planned_lo, tab, (uint32_t)m->clean_step, (uint32_t)m->step);
    else
        k_defer_flush<false><<<grid, 256, 0, st>>>(m->stamp, ng, m->param, m->grad, m->adam_m, m->adam_v, nullptr,
                                                   m->planned_lo, tab, (uint32_t)m->clean_step, (uint32_t)m->step);
    FH_CUDA(cudaGetLastError());
    m->dirty = false;
    m->clean_step = m->step;
    return FHASH_OK;
}

template <int F, int LAYOUT>
static void claim_launch(fhash_model* m, unsigned grid, const float* coords, int64_t n, const DeferArgs& d,
                         cudaStream_t st) {
    k_defer_claim<F, LAYOUT><<<grid, 256, 0, st>>>(m->lv, coords, n, d);
}

template <int F>
static void claim_any(fhash_model* m, unsigned grid, const float* coords, int64_t n, const DeferArgs& d, cudaStream_t st) {
    switch (m->lv.lv[0].layout) {
        case FHASH_LAYOUT_BRICK: claim_launch<F, 1>(m, grid, coords, n, d, st); break;
        case FHASH_LAYOUT_MASKED: claim_launch<F, 2>(m, grid, coords, n, d, st); break;
        default: claim_launch<F, 0>(m, grid, coords, n, d, st); break;
    }
}

static fhash_status fork_pending_dense(fhash_model* m, cudaStream_t st);

// Brings every group that a batch's gathers will read to step m->step (deferred step m->step + 1).  A
// pending dense-range update is forked onto the side stream once the claim list is sorted, so that it
// runs beside the replay (which is bound by its arithmetic) rather than beside the claim (whose random
// stamp accesses compete with it for memory).
static fhash_status catch_up(fhash_model* m, const float* coords, int64_t n, cudaStream_t st, bool* forked) {
    const uint32_t target = (uint32_t)m->step;
    if (target == (uint32_t)m->clean_step) return FHASH_OK;  // nothing is behind the previous step
    const int nd = m->lv.L - m->defer_level;
    const uint64_t ng = (m->defer_hi - m->defer_lo) / kGroup;
    const uint64_t cap = std::min<uint64_t>((uint64_t)n * nd * 16, ng);
    const size_t ctr_bytes = (sizeof(DeferCtr) + 255) / 256 * 256;
    FH_TRY(grow(m, m->s_defer, ctr_bytes + 2 * cap * sizeof(uint2)));
    DeferCtr* ctr = (DeferCtr*)m->s_defer.p;
    uint2* items = (uint2*)((char*)m->s_defer.p + ctr_bytes);
    uint2* binned = items + cap;
    FH_CUDA(cudaMemsetAsync(ctr, 0, sizeof(DeferCtr), st));
    DeferArgs d{};
    d.stamp = m->stamp;
    d.q0 = m->defer_lo / kGroup;
    d.q1 = m->defer_hi / kGroup;
    d.target = target;
    d.clean = (uint32_t)m->clean_step;
    d.l0 = m->defer_level;
    d.items = items;
    d.ctr = ctr;
    const unsigned cg = (unsigned)(((uint64_t)n * nd + 255) / 256);
    switch (m->lv.F) {
        case 1: claim_any<1>(m, cg, coords, n, d, st); break;
        case 2: claim_any<2>(m, cg, coords, n, d, st); break;
        case 4: claim_any<4>(m, cg, coords, n, d, st); break;
        case 8: claim_any<8>(m, cg, coords, n, d, st); break;
        default: return set_error(FHASH_EINVAL, "F=%d unsupported", m->lv.F);
    }
    FH_CUDA(cudaGetLastError());
    k_defer_bin<<<(unsigned)((cap + 256 * kBinPer - 1) / (256 * kBinPer)), 256, 0, st>>>(items, binned, ctr, target);
    FH_CUDA(cudaGetLastError());
    tev_record(m, TEV_CLAIM, st);
    if (m->dense_pending) {
        FH_TRY(fork_pending_dense(m, st));
        *forked = true;
    }
    const unsigned rg = (unsigned)num_sms() * 3;  // resident blocks (three per SM at this register use)
    const AdamScal* tab = (const AdamScal*)m->adam_tab;
    if (m->shadow)
        k_defer_replay<true><<<rg, 256, 0, st>>>(binned, ctr, m->param, m->grad, m->adam_m, m->adam_v, m->shadow,
                                                 m->defer_lo, tab, target);
    else
        k_defer_replay<false><<<rg, 256, 0, st>>>(binned, ctr, m->param, m->grad, m->adam_m, m->adam_v, nullptr,
                                                  m->defer_lo, tab, target);
    FH_CUDA(cudaGetLastError());
    m->last_ctr = ctr;
    return FHASH_OK;
}

// One training step: forward, loss, backward and Adam, with the deferred form when the model has
// deferred levels.
fhash_status launch_train_step(fhash_model* m, const float* coords, const float* target, int64_t n,
                               const fhash_adam* ad, double* loss_dev, cudaStream_t st) {
    plan_deferral(m);
    const bool defer = m->defer_level >= 0 && m->step + 1 < (int64_t)UINT32_MAX;
    tev_record(m, TEV_START, st);
    m->last_ctr = nullptr;
    m->side_timed = false;
    if (!defer) {
        FH_TRY(settle_deferred(m, st));
        tev_record(m, TEV_CLAIM, st);
        tev_record(m, TEV_REPLAY, st);
        FH_TRY(launch_grads2(m, coords, target, n, loss_dev, st));
        FH_TRY(launch_adam(m, ad, st));
        tev_record(m, TEV_ADAM, st);
        return FHASH_OK;
    }
    if (!m->stamp || m->stamp_groups != (m->defer_hi - m->defer_lo) / kGroup) {
        FH_TRY(settle_deferred(m, st));  // the deferred range changed: start from current state
        if (m->stamp) {
            cudaFree(m->stamp);
            m->device_bytes -= m->stamp_groups * 4;
            m->stamp = nullptr;
        }
        m->stamp_groups = (m->defer_hi - m->defer_lo) / kGroup;
        FH_CUDA(cudaMalloc(&m->stamp, std::max<uint64_t>(4, m->stamp_groups * 4)));
        m->device_bytes += m->stamp_groups * 4;
        FH_CUDA(cudaMemsetAsync(m->stamp, 0, m->stamp_groups * 4, st));
    }
    FH_TRY(ensure_tab(m, m->step + 2));
    // The previous step's dense-range update runs on a second stream beside this step's catch-up (they
    // touch disjoint parameters) and is joined before the gathers, which read those parameters.
    bool forked = false;
    FH_TRY(catch_up(m, coords, n, st, &forked));
    if (!m->last_ctr) tev_record(m, TEV_CLAIM, st);
    if (m->dense_pending && !forked) {
        FH_TRY(fork_pending_dense(m, st));
        forked = true;
    }
    if (forked) FH_CUDA(cudaStreamWaitEvent(st, m->ev_join, 0));
    m->planned_lo = m->defer_lo;  // the range this step defers (the pending update above used the last one)
    m->planned_hi = m->defer_hi;
    tev_record(m, TEV_REPLAY, st);
    FH_TRY(launch_grads2(m, coords, target, n, loss_dev, st));
    const int64_t k = m->step + 1;
    k_set_tab<<<1, 1, 0, st>>>((AdamScal*)m->adam_tab, k, scalars(ad, k));  // for later replays
    FH_CUDA(cudaGetLastError());
    m->pend_ad = *ad;
    m->pend_k = k;
    m->dense_pending = true;
    m->step = k;
    m->dirty = true;
    tev_record(m, TEV_ADAM, st);
    return FHASH_OK;
}

}  // namespace fh

using namespace fh;

extern "C" {

fhash_status fhash_set_adam_deferral(fhash_model* m, uint64_t min_level_rows, fhash_stream stream) {
    if (!m) return set_error(FHASH_EINVAL, "fhash_set_adam_deferral: null model");
    FH_TRY(settle_deferred(m, (cudaStream_t)stream));
    m->defer_min_rows = min_level_rows;
    plan_deferral(m);
    return FHASH_OK;
}

fhash_status fhash_set_timing(fhash_model* m, int32_t enable) {
    if (!m) return set_error(FHASH_EINVAL, "fhash_set_timing: null model");
    if (enable && !m->tev_init) {
        for (int i = 0; i < TEV_N; ++i) FH_CUDA(cudaEventCreate(&m->tev[i]));
        for (int i = 0; i < 2; ++i) FH_CUDA(cudaEventCreate(&m->tev_side[i]));
        m->tev_init = true;
    }
    m->timing = enable != 0;
    return FHASH_OK;
}

fhash_status fhash_get_adam_stats(fhash_model* m, fhash_adam_stats* out) {
    if (!m || !out) return set_error(FHASH_EINVAL, "fhash_get_adam_stats: null argument");
    memset(out, 0, sizeof *out);
    plan_deferral(m);
    out->first_deferred_level = m->defer_level;
    out->deferred_params = m->defer_hi - m->defer_lo;
    out->clean_step = m->clean_step;
    out->step = m->step;
    out->group_params = kGroup;
    if (m->last_ctr) {
        DeferCtr c;
        FH_CUDA(cudaMemcpy(&c, m->last_ctr, sizeof c, cudaMemcpyDeviceToHost));
        out->last_replayed_groups = c.count;
        out->last_replayed_steps = c.steps;
    }
    if (m->timing && m->tev_init) {
        FH_CUDA(cudaEventSynchronize(m->tev[TEV_ADAM]));
        for (int i = 0; i + 1 < TEV_N; ++i) FH_CUDA(cudaEventElapsedTime(&out->last_ms[i], m->tev[i], m->tev[i + 1]));
        if (m->side_timed) FH_CUDA(cudaEventElapsedTime(&out->last_side_ms, m->tev_side[0], m->tev_side[1]));
    }
    return FHASH_OK;
}

}  // extern "C"
