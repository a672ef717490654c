// MLP weight and bias gradients on the tensor cores, fed by TMA: tf32 inputs for the precision form,
// the error-compensated 3xTF32 split for the float32 form.
//
// dW_j[o][c] = sum over samples s of delta_j[o][s] * a_j[c][s] and db_j[o] = sum over s of delta_j[o][s].
// The backward keeps deltas and activations as float32 columns [feature][n], so both operands are
// already K-major with the samples as K: TMA copies 32-sample boxes (128 bytes per feature row, 128-byte
// swizzle, zero fill past the ends) straight into shared memory, and one thread issues tcgen05.mma
// kind::tf32 (M=64: the outputs, zero-padded to 64 by the box; N = the inputs rounded up to 16; K=8 per
// instruction) accumulating the CTA's whole chunk of samples in TMEM.  A deep mbarrier ring (10 stages
// of 16 KB in the float32 form, 6 in the precision form) keeps enough copies in flight for HBM; a stage
// is refilled one k-tile after its MMAs were issued, so the issuing thread never waits on the MMAs it
// has just issued.  While a stage is resident every thread adds its share of the
// delta rows into the bias sums, and in the float32 form splits its share of the rows for the 3xTF32
// product.  A layer with a single output (the last) is a dot product per input: its CTAs accumulate it
// on the CUDA cores in float32 and issue no MMA.  Each CTA writes its partial weight and bias gradients
// (kDwStride layout); one reduction adds the partials into the gradient.  Waits are bounded (2 s) and
// report through the model's error word.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "kernels.cuh"
#include "tc.cuh"

namespace fh {

constexpr int kDwTileA = 64 * 128;  // bytes: 64 rows (outputs, zero-padded) x 32 float32
constexpr int kDwTileB = 64 * 128;  // bytes: 64 rows (inputs, zero-padded) x 32 float32
constexpr int kDwLo = 2;            // lo tiles of the float32 form: k-tile kt uses lo buffer kt % 2
constexpr int kDwThreads = 512;     // 16 warps: the per-stage split and sums are latency-bound per warp
constexpr int kDwPer = kDwTileA / 16 / kDwThreads;  // float4 chunks of each tile per thread
template <bool SPLIT3>
__host__ __device__ constexpr int dw_stages() { return SPLIT3 ? 10 : 6; }
template <bool SPLIT3>
constexpr int dw_smem() {
    return 1024 + dw_stages<SPLIT3>() * (kDwTileA + kDwTileB) + (SPLIT3 ? kDwLo * (kDwTileA + kDwTileB) : 0) +
           2 * dw_stages<SPLIT3>() * 8 + 16;
}

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

// hi = tf32(v) written back in place, lo = v - hi (exact in float32) to the lo buffer.
__device__ __forceinline__ void split4(float4* h, float4* l, const float4 v) {
    const float4 hi = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
    *h = hi;
    *l = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
}

// Sum over the 8 consecutive lanes that share a staged row (lanes differing in bits 0-2).
__device__ __forceinline__ float sum8(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}

// SPLIT3 (the float32 form): every staged value a is split in shared memory into hi = tf32(a) (in place)
// and lo = a - hi (into the k-tile's lo buffer), and each K step issues hi*hi + hi*lo + lo*hi (the lo*lo term is below float32 rounding):
// the error-compensated "3xTF32" product of Ootomo and Yokota (2022), which keeps the weight gradients
// at float32 accuracy on the tensor cores.  Without it (the precision form) the tensor cores read the
// float32 inputs as tf32.
//
// Staged rows: a tile row is 128 bytes (8 float4 chunks, permuted within the row by the swizzle), so
// float4 number e of a tile lies in row e / 8, and thread t visits float4s t + kDwThreads i (i < kDwPer),
// rows t/8 + (kDwThreads/8) i, of each tile; the 8 lanes sharing a row are consecutive.
// TMEM: with M = 64, row r of the accumulator is lane 32 (r / 16) + r % 16.
template <bool SPLIT3>
__global__ void __launch_bounds__(kDwThreads) k_dw_tc(const __grid_constant__ DwMaps M, int64_t n, int64_t chunk,
                                               float* __restrict__ partial, int* __restrict__ err) {
    constexpr int kDwStages = dw_stages<SPLIT3>();
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    uint8_t* tileA = sm;
    uint8_t* tileB = sm + kDwStages * kDwTileA;
    uint8_t* loA = tileB + kDwStages * kDwTileB;  // SPLIT3 only: kDwLo tiles each
    uint8_t* loB = loA + (SPLIT3 ? kDwLo * kDwTileA : 0);
    uint64_t* full = reinterpret_cast<uint64_t*>(loB + (SPLIT3 ? kDwLo * kDwTileB : 0));
    uint64_t* empty = full + kDwStages;
    uint32_t* slot = reinterpret_cast<uint32_t*>(empty + kDwStages);
    const int t = threadIdx.x, warp = t >> 5, layer = blockIdx.y;
    const int fi = M.fi[layer], fo = M.fo[layer];
    const bool simt = fo == 1;         // a dot product per input on the CUDA cores, no MMA
    const int nN = (fi + 15) / 16 * 16;  // MMA N
    const int64_t s0 = blockIdx.x * chunk, s1 = min(n, s0 + chunk);
    const int nk = s1 > s0 ? (int)((s1 - s0 + 31) / 32) : 0;

    if (!simt && warp == 0) tc::tmem_alloc(slot, 64);
    if (t == 0) {
        for (int s = 0; s < kDwStages; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        tc::fence_mbar_init();
    }
    if (SPLIT3 && !simt) {
        // the lo halves of the padding rows (A rows >= fo, B rows >= fi), which the split never writes
        const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int s = 0; s < kDwLo; ++s) {
            float4* la = reinterpret_cast<float4*>(loA + s * kDwTileA);
            float4* lb = reinterpret_cast<float4*>(loB + s * kDwTileB);
            for (int e = fo * 8 + t; e < kDwTileA / 16; e += kDwThreads) la[e] = z;
            for (int e = fi * 8 + t; e < kDwTileB / 16; e += kDwThreads) lb[e] = z;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = simt ? 0u : *slot;
    const void* mapA = &M.a[layer];
    const void* mapB = &M.b[layer];
    auto load = [&](int kt) {
        const int s = kt % kDwStages;
        tc::mbar_expect_tx(&full[s], kDwTileA + kDwTileB);
        const int x = (int)(s0 + 32 * (int64_t)kt);
        tc::tma_load_2d(tileA + s * kDwTileA, mapA, x, 0, &full[s]);
        tc::tma_load_2d(tileB + s * kDwTileB, mapB, x, 0, &full[s]);
    };
    const uint32_t idesc = tc::idesc_tf32(64, nN);
    const uint32_t a0 = tc::smem_addr(tileA), b0 = tc::smem_addr(tileB);
    const uint32_t la0 = tc::smem_addr(loA), lb0 = tc::smem_addr(loB);
    float bsum[kDwPer] = {};  // bias sums of the thread's A rows
    float dot[kDwPer] = {};   // simt: dW of the thread's B rows
    bool bad = false;
    int loaded = 0, consumed = 0, issued = 0;  // thread 0: copies issued, waited for; MMA batches committed
    if (t == 0)
        for (; loaded < nk && loaded < kDwStages; ++loaded) load(loaded);
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % kDwStages;
        const uint32_t ph = (uint32_t)(kt / kDwStages) & 1u;
        const bool ok = tc::mbar_wait(&full[s], ph);
        if (__syncthreads_or(!ok || bad)) { bad = true; break; }
        consumed = kt + 1;
        float4* ha = reinterpret_cast<float4*>(tileA + s * kDwTileA);
        float4* hb = reinterpret_cast<float4*>(tileB + s * kDwTileB);
        const int lo = kt % kDwLo;
        float4* la = reinterpret_cast<float4*>(loA + lo * kDwTileA);
        float4* lb = reinterpret_cast<float4*>(loB + lo * kDwTileB);
        // delta rows (< fo): bias sums, and the split
#pragma unroll
        for (int i = 0; i < kDwPer; ++i) {
            const int e = t + kDwThreads * i;
            if (e < fo * 8) {
                const float4 v = ha[e];
                bsum[i] += (v.x + v.y) + (v.z + v.w);
                if (SPLIT3 && !simt) split4(ha + e, la + e, v);
            }
        }
        // activation rows (< fi): the split, or the single output's dot products
#pragma unroll
        for (int i = 0; i < kDwPer; ++i) {
            const int e = t + kDwThreads * i;
            if (e < fi * 8) {
                const float4 v = hb[e];
                if (simt) {
                    // stored chunk e & 7 of row r holds samples 4j .. 4j+3, j = (e & 7) ^ (r & 7); the delta
                    // row is row 0 of A, whose chunks are not permuted
                    const float4 d = ha[(e & 7) ^ ((e >> 3) & 7)];
                    dot[i] = fmaf(v.x, d.x, fmaf(v.y, d.y, fmaf(v.z, d.z, fmaf(v.w, d.w, dot[i]))));
                } else if (SPLIT3) {
                    split4(hb + e, lb + e, v);
                }
            }
        }
        if (SPLIT3 && !simt) tc::fence_async_smem();  // the generic-proxy stores become visible to the MMAs
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
            if (!simt) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ah = tc::sdesc_sw128(a0 + s * kDwTileA + kk * 32), bh = tc::sdesc_sw128(b0 + s * kDwTileB + kk * 32);
                    tc::mma_tf32(tmem, ah, bh, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
                    if (SPLIT3) {
                        const uint64_t al = tc::sdesc_sw128(la0 + lo * kDwTileA + kk * 32), bl = tc::sdesc_sw128(lb0 + lo * kDwTileB + kk * 32);
                        tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                        tc::mma_tf32(tmem, al, bh, idesc, 1u);
                    }
                }
                tc::mma_commit(&empty[s]);
                issued = kt + 1;
                // the previous k-tile's MMAs (issued a whole stage ago) have completed before its stage is
                // refilled and before the next k-tile's split overwrites its lo buffer
                if (kt > 0) {
                    const int kp = kt - 1;
                    if (!tc::mbar_wait(&empty[kp % kDwStages], (uint32_t)(kp / kDwStages) & 1u)) bad = true;
                    else if (loaded < nk) load(loaded++);
                }
            } else if (loaded < nk) {
                load(loaded++);  // every thread has read stage s
            }
        }
    }
    if (t == 0) {
        // wait (bounded) for the last committed batch, so that no MMA is in flight when TMEM is freed, and
        // for every copy issued but not waited for, so that none lands after the CTA has left
        if (issued > 0) {
            const int kl = issued - 1;
            if (!tc::mbar_wait(&empty[kl % kDwStages], (uint32_t)(kl / kDwStages) & 1u)) bad = true;
        }
        for (int k = consumed; k < loaded; ++k) tc::mbar_wait(&full[k % kDwStages], (uint32_t)(k / kDwStages) & 1u);
        if (bad) raise_error(err, 0x7C06);
    }
    tc::fence_before_sync();
    const int any_bad = __syncthreads_or(bad);
    tc::fence_after_sync();
    float* out = partial + ((int64_t)blockIdx.x * gridDim.y + layer) * kDwStride;
    if (!any_bad) {
#pragma unroll
        for (int i = 0; i < kDwPer; ++i) {
            const int r = (t >> 3) + (kDwThreads / 8) * i;
            const float b = sum8(bsum[i]);
            if ((t & 7) == 0 && r < fo) out[fo * fi + r] = b;
            if (simt) {
                const float d = sum8(dot[i]);
                if ((t & 7) == 0 && r < fi) out[r] = d;
            }
        }
        if (!simt && warp < 4) {  // warp w reads TMEM lane quarter w
            const int o = warp * 16 + (t & 31);  // lanes 0-15 of the warp's quarter hold rows 16 warp + 0..15
            float v[32];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (32 * h >= nN) break;
                tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32 * h, v);
                tc::tmem_ld_wait();
                if ((t & 31) < 16 && o < fo) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int c = 32 * h + q;
                        if (c < fi) out[o * fi + c] = nk > 0 ? v[q] : 0.0f;
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (!simt && warp == 0) tc::tmem_dealloc(tmem, 64);
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

// Partial weight and bias gradients of every layer (kDwStride layout, *nchunk_out chunks) from
// activations `acts` and deltas `dl` (column-major, n samples).  Returns false (nothing launched) when
// the tensor-core path does not apply: n not a multiple of 4 (row strides must be 16-byte multiples),
// fewer than 32 samples, a layer wider than 64 or no tensor-map encoder.
bool launch_dw_tc(fhash_model* m, const float* acts, const float* dl, int64_t n, float* wpart, size_t wpart_bytes,
                  int* nchunk_out, cudaStream_t st, cudaError_t* err, bool split3) {
    *err = cudaSuccess;
    const MlpShape& sh = m->mlp;
    const int W = sh.width, nl = sh.nh + 1;
    if (n % 4 != 0 || n < 32 || W > 64 || sh.in > 64 || !tensor_map_encoder()) return false;
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>((n + 2047) / 2048, (int64_t)num_sms()));
    const int64_t chunk = ((n + nchunk - 1) / nchunk + 31) / 32 * 32;
    if ((size_t)nchunk * nl * kDwStride * 4 > wpart_bytes) return false;
    DwMaps M;
    memset(&M, 0, sizeof M);
    for (int j = 0; j < nl; ++j) {
        const int fi = j == 0 ? sh.in : W, fo = j == sh.nh ? 1 : W;
        const float* aj = (j == 0) ? acts : acts + (int64_t)(sh.in + (j - 1) * W) * n;
        const float* dj = dl + (int64_t)j * W * n;
        if (!make_map(&M.a[j], dj, n, fo, 64) || !make_map(&M.b[j], aj, n, fi, 64)) return false;
        M.fi[j] = fi;
        M.fo[j] = fo;
    }
    const int smem = split3 ? dw_smem<true>() : dw_smem<false>();
    const void* fn = split3 ? (const void*)k_dw_tc<true> : (const void*)k_dw_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        if (split3)
            k_dw_tc<true><<<dim3(nchunk, nl), kDwThreads, smem, st>>>(M, n, chunk, wpart, m->err_word);
        else
            k_dw_tc<false><<<dim3(nchunk, nl), kDwThreads, smem, st>>>(M, n, chunk, wpart, m->err_word);
        e = cudaGetLastError();
    }
    *nchunk_out = nchunk;
    *err = e;
    return true;
}

}  // namespace fh
