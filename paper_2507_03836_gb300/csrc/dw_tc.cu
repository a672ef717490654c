// MLP weight gradients on the tensor cores, fed by TMA: tf32 inputs for the precision form, the
// error-compensated 3xTF32 split for the float32 form.
//
// dW_j[o][c] = sum over samples s of delta_j[o][s] * a_j[c][s].  The backward keeps deltas and
// activations as float32 columns [feature][n], so both operands are already K-major with the samples
// as K: TMA copies 32-sample boxes (128 bytes per feature row, 128-byte swizzle, zero fill past the
// ends) straight into shared memory, and one thread issues tcgen05.mma kind::tf32 (M=128 with the
// output rows zero-padded, N=64, K=8 per instruction) accumulating the CTA's whole chunk of samples in
// 64 TMEM columns.  A 4-stage mbarrier pipeline keeps the copies ahead of the MMAs.  The four warps
// then read the accumulator lanes back and write the CTA's partial dW; a reduction adds the partials
// into the gradient.  Waits are bounded (2 s) and report through the model's error word.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "kernels.cuh"
#include "tc.cuh"

namespace fh {

constexpr int kDwStages = 4;
constexpr int kDwTileA = 128 * 128;  // bytes: 128 rows (padded outputs) x 32 float32
constexpr int kDwTileB = 64 * 128;   // bytes: 64 rows (inputs) x 32 float32

struct alignas(64) DwMaps {
    CUtensorMap a[FHASH_MAX_HIDDEN + 1];
    CUtensorMap b[FHASH_MAX_HIDDEN + 1];
    int32_t fi[FHASH_MAX_HIDDEN + 1], fo[FHASH_MAX_HIDDEN + 1];
};

// Round to the nearest tf32 value (10 explicit mantissa bits, ties to even), kept as float32.
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t u = __float_as_uint(x);
    u += 0xFFFu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xFFFFE000u);
}

// SPLIT3 (the float32 form): every staged value a is split in shared memory into hi = tf32(a) and
// lo = a - hi (exact in float32), and each K step issues hi*hi + hi*lo + lo*hi (the lo*lo term is below
// float32 rounding): the error-compensated "3xTF32" product of Ootomo and Yokota (2022), which keeps the
// weight gradients at float32 accuracy on the tensor cores.  Without it (the precision form) the
// tensor cores read the float32 inputs as tf32.
template <bool SPLIT3>
__global__ void __launch_bounds__(128) k_dw_tc(const __grid_constant__ DwMaps M, int64_t n, int64_t chunk,
                                               float* __restrict__ partial, int* __restrict__ err) {
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    uint8_t* tileA = sm;
    uint8_t* tileB = sm + kDwStages * kDwTileA;
    uint8_t* loA = tileB + kDwStages * kDwTileB;             // SPLIT3 only
    uint8_t* loB = loA + (SPLIT3 ? kDwStages * kDwTileA : 0);
    uint64_t* full = reinterpret_cast<uint64_t*>(loB + (SPLIT3 ? kDwStages * kDwTileB : 0));
    uint64_t* empty = full + kDwStages;
    uint32_t* slot = reinterpret_cast<uint32_t*>(empty + kDwStages);
    const int t = threadIdx.x, warp = t >> 5, layer = blockIdx.y;
    const int fi = M.fi[layer], fo = M.fo[layer];
    const int64_t s0 = blockIdx.x * chunk, s1 = min(n, s0 + chunk);
    const int nk = s1 > s0 ? (int)((s1 - s0 + 31) / 32) : 0;

    if (warp == 0) tc::tmem_alloc(slot, 64);
    if (t == 0) {
        for (int s = 0; s < kDwStages; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    bool bad = false;
    const void* mapA = &M.a[layer];
    const void* mapB = &M.b[layer];
    auto load = [&](int kt) {
        const int s = kt % kDwStages;
        tc::mbar_expect_tx(&full[s], kDwTileA + kDwTileB);
        const int x = (int)(s0 + 32 * (int64_t)kt);
        tc::tma_load_2d(tileA + s * kDwTileA, mapA, x, 0, &full[s]);
        tc::tma_load_2d(tileB + s * kDwTileB, mapB, x, 0, &full[s]);
    };
    constexpr uint32_t idesc = tc::idesc_tf32(128, 64);
    const uint32_t a0 = tc::smem_addr(tileA), b0 = tc::smem_addr(tileB);
    if (!SPLIT3) {
        if (t == 0 && nk > 0) {
            for (int kt = 0; kt < nk && kt < kDwStages; ++kt) load(kt);
            for (int kt = 0; kt < nk && !bad; ++kt) {
                const int s = kt % kDwStages;
                const uint32_t ph = (uint32_t)(kt / kDwStages) & 1u;
                if (!tc::mbar_wait(&full[s], ph)) { bad = true; break; }
                tc::fence_after_sync();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_tf32(tmem, tc::sdesc_sw128(a0 + s * kDwTileA + kk * 32), tc::sdesc_sw128(b0 + s * kDwTileB + kk * 32),
                                 idesc, (kt > 0 || kk > 0) ? 1u : 0u);
                tc::mma_commit(&empty[s]);
                if (kt + kDwStages < nk) {
                    if (!tc::mbar_wait(&empty[s], ph)) { bad = true; break; }
                    load(kt + kDwStages);
                }
            }
            if (!bad) {  // every MMA has completed once the last commit has arrived
                const int kl = nk - 1;
                if (!tc::mbar_wait(&empty[kl % kDwStages], (uint32_t)(kl / kDwStages) & 1u)) bad = true;
            }
            if (bad) raise_error(err, 0x7C06);
        }
    } else if (nk > 0) {
        const uint32_t la0 = tc::smem_addr(loA), lb0 = tc::smem_addr(loB);
        int loaded = 0, consumed = 0, issued = 0;  // copies issued, copies waited for, MMA batches committed
        if (t == 0)
            for (; loaded < nk && loaded < kDwStages; ++loaded) load(loaded);
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % kDwStages;
            const uint32_t ph = (uint32_t)(kt / kDwStages) & 1u;
            const bool ok = tc::mbar_wait(&full[s], ph);
            if (__syncthreads_or(!ok)) { bad = true; break; }
            consumed = kt + 1;
            // split the stage in place: tile <- hi, lo buffer <- a - hi (same swizzled positions)
            float4* ha = reinterpret_cast<float4*>(tileA + s * kDwTileA);
            float4* hb = reinterpret_cast<float4*>(tileB + s * kDwTileB);
            float4* la = reinterpret_cast<float4*>(loA + s * kDwTileA);
            float4* lb = reinterpret_cast<float4*>(loB + s * kDwTileB);
            for (int e = t; e < (kDwTileA + kDwTileB) / 16; e += blockDim.x) {
                float4* h = e < kDwTileA / 16 ? ha + e : hb + (e - kDwTileA / 16);
                float4* l = e < kDwTileA / 16 ? la + e : lb + (e - kDwTileA / 16);
                const float4 v = *h;
                const float4 hi = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
                *h = hi;
                *l = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
            }
            tc::fence_async_smem();  // the generic-proxy stores become visible to the tensor cores
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (t == 0) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ah = tc::sdesc_sw128(a0 + s * kDwTileA + kk * 32), bh = tc::sdesc_sw128(b0 + s * kDwTileB + kk * 32);
                    const uint64_t al = tc::sdesc_sw128(la0 + s * kDwTileA + kk * 32), bl = tc::sdesc_sw128(lb0 + s * kDwTileB + kk * 32);
                    tc::mma_tf32(tmem, ah, bh, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
                    tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                    tc::mma_tf32(tmem, al, bh, idesc, 1u);
                }
                tc::mma_commit(&empty[s]);
                issued = kt + 1;
                if (loaded < nk) {
                    if (!tc::mbar_wait(&empty[s], ph)) bad = true;  // stage s free again: refill it
                    else load(loaded++);
                }
            }
            if (__syncthreads_or(bad)) { bad = true; break; }
        }
        if (t == 0) {
            // wait (bounded) for the last committed batch, so that no MMA is in flight when TMEM is freed,
            // and for every copy issued but not waited for, so that none lands after the CTA has left
            if (issued > 0) {
                const int kl = issued - 1;
                if (!tc::mbar_wait(&empty[kl % kDwStages], (uint32_t)(kl / kDwStages) & 1u)) bad = true;
            }
            for (int k = consumed; k < loaded; ++k) tc::mbar_wait(&full[k % kDwStages], (uint32_t)(k / kDwStages) & 1u);
            if (bad) raise_error(err, 0x7C06);
        }
    }
    tc::fence_before_sync();
    const int any_bad = __syncthreads_or(bad);
    tc::fence_after_sync();
    float* out = partial + ((int64_t)blockIdx.x * gridDim.y + layer) * 4096;
    if (!any_bad) {
        const int o = warp * 32 + (t & 31);  // TMEM lane = output row
        float v[32];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32 * h, v);
            tc::tmem_ld_wait();
            if (o < fo) {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int c = 32 * h + q;
                    if (c < fi) out[o * fi + c] = nk > 0 ? v[q] : 0.0f;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// grad[e] += sum over chunks of partial[chunk][layer][e], e < fo*fi.
__global__ void k_dw_tc_reduce(const float* __restrict__ partial, int nchunk, int nlayers, int layer, int ne,
                               float* __restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    float s = 0.0f;
    for (int c = 0; c < nchunk; ++c) s += partial[((int64_t)c * nlayers + layer) * 4096 + e];
    grad[e] += s;
}

// Bias gradients, two deterministic stages: part[o][c] = sum of delta[o][s] over chunk c (64 chunks),
// then grad[o] += sum over c.
constexpr int kRowChunks = 64;
__global__ void k_rowsum_part(const float* __restrict__ d, int64_t n, float* __restrict__ part) {
    const int o = blockIdx.x, c = blockIdx.y;
    const int64_t per = (n + kRowChunks - 1) / kRowChunks, s0 = c * per, s1 = min(n, s0 + per);
    float acc = 0.0f;
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) acc += d[(int64_t)o * n + s];
    __shared__ float red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[o * kRowChunks + c] = red[0];
}
__global__ void k_rowsum_final(const float* __restrict__ part, int fo, float* __restrict__ grad) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= fo) return;
    float s = 0.0f;
    for (int c = 0; c < kRowChunks; ++c) s += part[o * kRowChunks + c];
    grad[o] += s;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    }
    return fn;
}

// Column-major float32 rows [rows][n] as a 2D tensor (x = sample, y = row) with 32 x box_rows boxes.
static bool make_map(CUtensorMap* m, const float* base, int64_t n, int rows, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)n * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Weight and bias gradients of every layer from activations `acts` and deltas `dl` (column-major,
// n samples).  Returns false (nothing launched) when the tensor-core path does not apply: n not a
// multiple of 4 (row strides must be 16-byte multiples) or no tensor-map encoder.
bool launch_dw_tc(fhash_model* m, const float* acts, const float* dl, int64_t n, float* wpart, size_t wpart_bytes,
                  cudaStream_t st, cudaError_t* err, bool split3) {
    *err = cudaSuccess;
    const MlpShape& sh = m->mlp;
    const int W = sh.width, nl = sh.nh + 1;
    if (n % 4 != 0 || n < 32 || !tensor_map_encoder()) return false;
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>((n + 2047) / 2048, (int64_t)num_sms()));
    const int64_t chunk = ((n + nchunk - 1) / nchunk + 31) / 32 * 32;
    const size_t dw_floats = (size_t)nchunk * nl * 4096;
    if ((dw_floats + (size_t)64 * kRowChunks) * 4 > wpart_bytes) return false;
    float* rpart = wpart + dw_floats;
    DwMaps M;
    memset(&M, 0, sizeof M);
    for (int j = 0; j < nl; ++j) {
        const int fi = j == 0 ? sh.in : W, fo = j == sh.nh ? 1 : W;
        const float* aj = (j == 0) ? acts : acts + (int64_t)(sh.in + (j - 1) * W) * n;
        const float* dj = dl + (int64_t)j * W * n;
        if (!make_map(&M.a[j], dj, n, fo, 128) || !make_map(&M.b[j], aj, n, fi, 64)) return false;
        M.fi[j] = fi;
        M.fo[j] = fo;
    }
    const int smem = 1024 + (split3 ? 2 : 1) * kDwStages * (kDwTileA + kDwTileB) + 2 * kDwStages * 8 + 16;
    const void* fn = split3 ? (const void*)k_dw_tc<true> : (const void*)k_dw_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        if (split3)
            k_dw_tc<true><<<dim3(nchunk, nl), 128, smem, st>>>(M, n, chunk, wpart, m->err_word);
        else
            k_dw_tc<false><<<dim3(nchunk, nl), 128, smem, st>>>(M, n, chunk, wpart, m->err_word);
        e = cudaGetLastError();
    }
    float* gm = m->grad + m->n_table;
    for (int j = 0; j < nl && e == cudaSuccess; ++j) {
        const int fi = j == 0 ? sh.in : W, fo = j == sh.nh ? 1 : W;
        k_dw_tc_reduce<<<(fo * fi + 255) / 256, 256, 0, st>>>(wpart, nchunk, nl, j, fo * fi, gm + sh.w_off[j]);
        k_rowsum_part<<<dim3(fo, kRowChunks), 256, 0, st>>>(dl + (int64_t)j * W * n, n, rpart);
        k_rowsum_final<<<1, 64, 0, st>>>(rpart, fo, gm + sh.b_off[j]);
        e = cudaGetLastError();
    }
    *err = e;
    return true;
}

}  // namespace fh
