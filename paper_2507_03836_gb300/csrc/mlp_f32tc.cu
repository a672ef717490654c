// Float32 MLP of a training step on the tensor cores: forward, MSE loss and the backward data path of
// one 128-sample tile in one CTA, every layer a tcgen05.mma kind::tf32 GEMM with the error-compensated
// 3xTF32 split (hi*hi + hi*lo + lo*hi, Ootomo and Yokota 2022), so the results keep float32 accuracy.
//
// A tile's samples are the TMEM lanes.  Two threads share a sample: warps 0-3 take columns 0-31 of
// its rows and warps 4-7 columns 32-63 (warp w reads TMEM lane quarter w % 4), so an accumulator row
// is two threads' registers after tcgen05.ld, and 8 warps per SM hide the epilogues' latency.  Every
// GEMM has the samples as M = 128 and K-major operands in the 128-byte swizzle layout:
//   forward layer j:   z[s][o] = sum_c a[s][c] W_j[o][c]     A = activations, B = W_j as stored;
//   backward layer j:  p[s][c] = sum_o d[s][o] W_j[o][c]     A = deltas,      B = W_j transposed.
// The weights of every hidden layer, both ways and split into hi and lo, are staged once per CTA; the
// A operand of each GEMM is written by its producing epilogue (each thread its own row: the encoding
// read from its feature-major columns, the activations, the deltas), split into hi and lo.  The ReLU
// masks stay in registers (one bit per unit), so the backward needs no activation reloads.  Global
// outputs are the ones the split kernels write, feature-major [row][n] and coalesced across the
// threads: the hidden activations (for the weight gradients), the deltas of every layer and
// d(loss)/d(encoding) (for the table scatter), plus one loss partial per CTA.
//
// The precision (bf16) form runs its own forward kernel and uses the backward data path alone (the BWD
// instantiation: masks from the stored activations).
//
// Shapes: encoding width IN in {16, 32, 64}, hidden width 64, up to kTcMaxHidden hidden layers (the
// weights of both directions must fit in shared memory); others take the float32 SIMT kernels.
#include <stdint.h>

#include <algorithm>

#include "kernels.cuh"
#include "tc.cuh"

namespace fh {

constexpr int kMt = 128;         // samples per tile = TMEM lanes
constexpr int kMthreads = 256;   // two threads per sample, 32 columns each
constexpr int kMw = 64;          // hidden width handled here
constexpr int kTcMaxHidden = 2;  // hidden layers whose weights (both directions, hi and lo) fit

// Shared-memory layout (bytes from the 1024-aligned base).  A K-major operand of R rows and K floats is
// ceil(K / 32) blocks of R x 128 bytes (8-row swizzle atoms of 1024 bytes); hi and lo copies are
// separate regions of the same shape.
struct TcMlpLayout {
    int a_hi, a_lo;                                   // A: 128 rows x 64 floats (two blocks)
    int wf_hi[kTcMaxHidden], wf_lo[kTcMaxHidden];     // forward B of layer j: 64 rows x fi_j floats
    int wb_hi[kTcMaxHidden], wb_lo[kTcMaxHidden];     // backward B of layer j: fi_j rows x 64 floats
    int bias, wout, ypart, bar, slot, total;
};

__host__ __device__ inline int tc_blocks(int k) { return (k + 31) / 32; }

__host__ __device__ inline TcMlpLayout tc_mlp_layout(int in, int nh) {
    TcMlpLayout L{};
    int o = 0;
    L.a_hi = o; o += 2 * kMt * 128;
    L.a_lo = o; o += 2 * kMt * 128;
    for (int j = 0; j < nh; ++j) {
        const int fi = j == 0 ? in : kMw;
        const int wf = tc_blocks(fi) * kMw * 128, wb = tc_blocks(kMw) * fi * 128;
        L.wf_hi[j] = o; o += wf;
        L.wf_lo[j] = o; o += wf;
        L.wb_hi[j] = o; o += wb;
        L.wb_lo[j] = o; o += wb;
    }
    L.bias = o; o += kTcMaxHidden * kMw * 4;
    L.wout = o; o += kMw * 4 + 16;
    L.ypart = o; o += 2 * kMt * 4;  // the two column halves' partial output sums
    L.bar = o; o += 16;
    L.slot = o; o += 16;
    L.total = o + 1024;  // alignment slack of the dynamic shared-memory base
    return L;
}

// Byte offset of element (row r, k) in a K-major 128-byte-swizzled operand of R rows.
__device__ __forceinline__ int sw128_off(int R, int r, int k) {
    return (k >> 5) * R * 128 + r * 128 + ((((k & 31) >> 2) ^ (r & 7)) << 4) + ((k & 3) << 2);
}


// Round to the nearest tf32 value (10 explicit mantissa bits, ties to even), kept as float32.
__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t u = __float_as_uint(x);
    u += 0xFFFu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xFFFFE000u);
}

// Writes values [h K/2, (h + 1) K/2) of row r of an A operand of K floats (hi and lo), 16 bytes at a time.
template <int K>
__device__ __forceinline__ void put_half(uint8_t* hi, uint8_t* lo, int r, int h, const float (&v)[K / 2]) {
#pragma unroll
    for (int q = 0; q < K / 8; ++q) {
        const int c = h * (K / 8) + q;  // 16-byte chunk along K
        const int off = (c >> 3) * kMt * 128 + r * 128 + (((c & 7) ^ (r & 7)) << 4);
        float4 a, b;
        a.x = tf32_hi(v[4 * q + 0]); b.x = v[4 * q + 0] - a.x;
        a.y = tf32_hi(v[4 * q + 1]); b.y = v[4 * q + 1] - a.y;
        a.z = tf32_hi(v[4 * q + 2]); b.z = v[4 * q + 2] - a.z;
        a.w = tf32_hi(v[4 * q + 3]); b.w = v[4 * q + 3] - a.w;
        *reinterpret_cast<float4*>(hi + off) = a;
        *reinterpret_cast<float4*>(lo + off) = b;
    }
}

// Columns [h N/2, (h + 1) N/2) of this thread's accumulator lane (N = 16, 32 or 64; 64 are allocated).
template <int N>
__device__ __forceinline__ void read_half(uint32_t taddr, int h, float (&v)[N / 2]) {
    float part[32];
    tc::tmem_ld32(taddr + h * (N / 2), part);
    tc::tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < N / 2; ++q) v[q] = part[q];
}

// Every hidden layer's weights, split into hi and lo, in both operand forms; biases and output weights.
__device__ __forceinline__ void stage_tc_weights(uint8_t* sm, const TcMlpLayout& L, const MlpShape& sh,
                                                 const float* __restrict__ Pm, int in) {
    for (int j = 0; j < sh.nh; ++j) {
        const int fi = j == 0 ? in : kMw;
        const float* W = Pm + sh.w_off[j];  // [64][fi]
        for (int e = threadIdx.x; e < kMw * fi; e += blockDim.x) {
            const int o = e / fi, c = e % fi;
            const float w = W[e], hw = tf32_hi(w), lw = w - hw;
            const int f = sw128_off(kMw, o, c), b = sw128_off(fi, c, o);
            *reinterpret_cast<float*>(sm + L.wf_hi[j] + f) = hw;
            *reinterpret_cast<float*>(sm + L.wf_lo[j] + f) = lw;
            *reinterpret_cast<float*>(sm + L.wb_hi[j] + b) = hw;
            *reinterpret_cast<float*>(sm + L.wb_lo[j] + b) = lw;
        }
        for (int o = threadIdx.x; o < kMw; o += blockDim.x)
            reinterpret_cast<float*>(sm + L.bias)[j * kMw + o] = Pm[sh.b_off[j] + o];
    }
    float* wout = reinterpret_cast<float*>(sm + L.wout);
    for (int o = threadIdx.x; o < kMw; o += blockDim.x) wout[o] = Pm[sh.w_off[sh.nh] + o];
    if (threadIdx.x == 0) wout[kMw] = Pm[sh.b_off[sh.nh]];
}

// acts rows [0, IN) hold the encoding; the kernel writes rows IN + j*64 + o (hidden activations), dl
// (deltas: row j*64 + o of hidden layer j, row nh*64 the output's dL/dy) and denc (IN rows), all
// feature-major with row stride n, and one loss partial (sum of squared errors) per CTA.
// BWD: the backward data path alone, after the precision form's forward kernel has stored the hidden
// activations in acts and dL/dy in gyin (ReLU masks from the stored activations; no loss partials).
template <int IN, bool BWD>
__global__ void __launch_bounds__(kMthreads, 1) k_mlp_f32tc(const __grid_constant__ MlpShape sh, const float* __restrict__ Pm,
                                                         const float* __restrict__ target, const float* __restrict__ gyin,
                                                         int64_t n, float two_over_n,
                                                         float* __restrict__ acts, float* __restrict__ dl,
                                                         float* __restrict__ denc, double* __restrict__ partial,
                                                         int* __restrict__ err) {
    constexpr int HI = IN / 2;  // encoding values per thread
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    const int nh = sh.nh, t = threadIdx.x, warp = t >> 5;
    const int h = warp >> 2;                      // column half: 0 -> columns 0-31, 1 -> 32-63
    const int r = (warp & 3) * 32 + (t & 31);     // sample of the tile = TMEM lane
    const TcMlpLayout L = tc_mlp_layout(IN, nh);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + L.slot);
    const float* bias = reinterpret_cast<const float*>(sm + L.bias);
    const float* wout = reinterpret_cast<const float*>(sm + L.wout);
    float* ypart = reinterpret_cast<float*>(sm + L.ypart);
    uint8_t* a_hi = sm + L.a_hi;
    uint8_t* a_lo = sm + L.a_lo;
    if (warp == 0) tc::tmem_alloc(slot, 64);
    if (t == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    stage_tc_weights(sm, L, sh, Pm, IN);
    tc::fence_async_smem();  // the staged weights become visible to the tensor cores
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this thread's lane quarter
    const uint32_t ah0 = tc::smem_addr(a_hi), al0 = tc::smem_addr(a_lo);
    const float bo = wout[kMw];
    uint32_t phase = 0;
    bool bad = false;
    double lsum = 0.0;

    // D = A * B^T over K (3xTF32), B of N rows at (off_hi, off_lo); every thread has written its A half-row.
    auto gemm = [&](int off_hi, int off_lo, int N, int K) -> bool {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
            const uint32_t idesc = tc::idesc_tf32(kMt, N);
            const uint32_t bh0 = tc::smem_addr(sm + off_hi), bl0 = tc::smem_addr(sm + off_lo);
            for (int kk = 0; kk < K / 8; ++kk) {
                const uint32_t ka = (kk >> 2) * kMt * 128 + (kk & 3) * 32, kb = (kk >> 2) * N * 128 + (kk & 3) * 32;
                const uint64_t ah = tc::sdesc_sw128(ah0 + ka), al = tc::sdesc_sw128(al0 + ka);
                const uint64_t bh = tc::sdesc_sw128(bh0 + kb), bl = tc::sdesc_sw128(bl0 + kb);
                tc::mma_tf32(tmem, ah, bh, idesc, kk > 0 ? 1u : 0u);
                tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                tc::mma_tf32(tmem, al, bh, idesc, 1u);
            }
            tc::mma_commit(bar);
        }
        const bool ok = tc::mbar_wait(bar, phase);
        phase ^= 1u;
        tc::fence_after_sync();
        return !__syncthreads_or(!ok);
    };

    const int64_t ntiles = (n + kMt - 1) / kMt;
    float x[HI];
    auto load_x = [&](int64_t tl) {
        const int64_t i = tl * kMt + r;
        const bool in_range = tl < ntiles && i < n;
#pragma unroll
        for (int k = 0; k < HI; ++k) x[k] = in_range ? acts[(int64_t)(h * HI + k) * n + i] : 0.0f;
    };
    if (!BWD) load_x(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * kMt + r;
        const bool valid = i < n;
        float v[32];
        uint32_t mk[kTcMaxHidden] = {};  // ReLU masks of this thread's 32 units per hidden layer
        float gy = 0.0f;
        if constexpr (BWD) {
#pragma unroll
            for (int j = 0; j < kTcMaxHidden; ++j) {
                if (j >= nh) break;
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    if (valid && acts[(int64_t)(IN + j * kMw + 32 * h + q) * n + i] > 0.0f) mk[j] |= 1u << q;
            }
            if (valid) {
                gy = gyin[i];
                if (h == 0) dl[(int64_t)(nh * kMw) * n + i] = gy;
            }
        } else {
        put_half<IN>(a_hi, a_lo, r, h, x);
        load_x(tile + gridDim.x);  // the next tile's encoding stays in flight during this one
        // forward: z = W a + b, a = ReLU(z)
#pragma unroll
        for (int j = 0; j < kTcMaxHidden; ++j) {
            if (j >= nh) break;
            const bool ok = j == 0 ? gemm(L.wf_hi[0], L.wf_lo[0], kMw, IN) : gemm(L.wf_hi[j], L.wf_lo[j], kMw, kMw);
            if (!ok) { bad = true; break; }
            read_half<kMw>(taddr, h, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int o = 32 * h + q;
                const float z = v[q] + bias[j * kMw + o];
                if (z > 0.0f) mk[j] |= 1u << q;
                v[q] = fmaxf(z, 0.0f);
                if (valid) acts[(int64_t)(IN + j * kMw + o) * n + i] = v[q];
            }
            if (j + 1 < nh) put_half<kMw>(a_hi, a_lo, r, h, v);
        }
        if (bad) break;
        // output unit: the two halves' partial sums, added in a fixed order; dL/dy = 2 (y - target) / N
        float part = h == 0 ? bo : 0.0f;
#pragma unroll
        for (int q = 0; q < 32; ++q) part = fmaf(wout[32 * h + q], v[q], part);
        ypart[h * kMt + r] = part;
        __syncthreads();
        const float y = ypart[r] + ypart[kMt + r];
        if (valid) {
            const float d = y - target[i];
            gy = two_over_n * d;
            if (h == 0) {
                lsum += (double)d * (double)d;
                dl[(int64_t)(nh * kMw) * n + i] = gy;
            }
        }
        }
        // delta of the last hidden layer: wout * dL/dy where its unit was active
        uint32_t ml = 0u;
#pragma unroll
        for (int j = 0; j < kTcMaxHidden; ++j)
            if (j == nh - 1) ml = mk[j];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int o = 32 * h + q;
            v[q] = ((ml >> q) & 1u) ? wout[o] * gy : 0.0f;
            if (valid) dl[(int64_t)((nh - 1) * kMw + o) * n + i] = v[q];
        }
        // backward: p = W^T delta; below a hidden layer, delta = p where that layer was active
#pragma unroll
        for (int j = kTcMaxHidden - 1; j >= 0; --j) {
            if (j >= nh) continue;
            put_half<kMw>(a_hi, a_lo, r, h, v);
            if (j > 0) {
                if (!gemm(L.wb_hi[j], L.wb_lo[j], kMw, kMw)) { bad = true; break; }
                read_half<kMw>(taddr, h, v);
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    v[q] = ((mk[j - 1] >> q) & 1u) ? v[q] : 0.0f;
                    if (valid) dl[(int64_t)((j - 1) * kMw + 32 * h + q) * n + i] = v[q];
                }
            } else {
                if (!gemm(L.wb_hi[0], L.wb_lo[0], IN, kMw)) { bad = true; break; }
                float p[HI];
                read_half<IN>(taddr, h, p);
                if (valid) {
#pragma unroll
                    for (int q = 0; q < HI; ++q) denc[(int64_t)(h * HI + q) * n + i] = p[q];
                }
            }
        }
        if (bad) break;
    }
    tc::fence_before_sync();
    const double tot = block_sum(lsum);  // synchronises the CTA
    if (t == 0) {
        if (!BWD) partial[blockIdx.x] = tot;
        if (bad) raise_error(err, 0x7C0A);
    }
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}
template <int IN, bool BWD>
static cudaError_t launch_in(const MlpShape& sh, int g, int smem, const float* Pm, const float* target,
                             const float* gyin, int64_t n, float* acts, float* dl, float* denc, double* partial,
                             int* err, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_mlp_f32tc<IN, BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_mlp_f32tc<IN, BWD><<<g, kMthreads, smem, st>>>(sh, Pm, target, gyin, n, 2.0f / (float)n, acts, dl, denc, partial, err);
    return cudaGetLastError();
}

// The fused float32 MLP pass over n samples (one CTA per SM, persistent over 128-sample tiles): forward,
// loss and backward data path, or with gyin != nullptr the backward data path alone (the precision
// form, whose forward kernel stored the activations and dL/dy = gyin).  Returns false, launching
// nothing, when the model's shape is not handled here; otherwise *grid receives the number of CTAs
// (the loss partials written by the full pass, at most max_partials).
bool launch_mlp_f32tc(fhash_model* m, const float* target, const float* gyin, int64_t n, float* acts, float* dl,
                      float* denc, double* partial, int max_partials, int* grid, cudaStream_t st, cudaError_t* err) {
    *err = cudaSuccess;
    const MlpShape& sh = m->mlp;
    if (sh.width != kMw || sh.nh < 1 || sh.nh > kTcMaxHidden || (sh.in != 16 && sh.in != 32 && sh.in != 64) ||
        n < 1 || max_partials < 1)
        return false;
    const TcMlpLayout L = tc_mlp_layout(sh.in, sh.nh);
    if (L.total > 227 * 1024) return false;
    const int64_t ntiles = (n + kMt - 1) / kMt;
    const int g = (int)std::min<int64_t>(std::min<int64_t>(ntiles, num_sms()), max_partials);
    const float* Pm = m->param + m->n_table;
    const bool bwd = gyin != nullptr;
    cudaError_t e;
    switch (sh.in) {
        case 16: e = bwd ? launch_in<16, true>(sh, g, L.total, Pm, target, gyin, n, acts, dl, denc, partial, m->err_word, st)
                         : launch_in<16, false>(sh, g, L.total, Pm, target, gyin, n, acts, dl, denc, partial, m->err_word, st); break;
        case 32: e = bwd ? launch_in<32, true>(sh, g, L.total, Pm, target, gyin, n, acts, dl, denc, partial, m->err_word, st)
                         : launch_in<32, false>(sh, g, L.total, Pm, target, gyin, n, acts, dl, denc, partial, m->err_word, st); break;
        default: e = bwd ? launch_in<64, true>(sh, g, L.total, Pm, target, gyin, n, acts, dl, denc, partial, m->err_word, st)
                         : launch_in<64, false>(sh, g, L.total, Pm, target, gyin, n, acts, dl, denc, partial, m->err_word, st); break;
    }
    *grid = g;
    *err = e;
    return true;
}

}  // namespace fh
