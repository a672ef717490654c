// Precision form: bf16 tables and MLP on the tcgen05 tensor cores with float32 accumulation in TMEM.
//
// One CTA of 128 threads owns a tile of 128 samples (the MMA's M).  Each thread encodes its sample
// from the bf16 shadow of the tables (Section 3.2.4; interpolation weights and accumulation in
// float32) and writes it as one 128-byte bf16 row of the A operand in shared memory (K-major,
// 128-byte swizzle).  One thread then issues the layer's tcgen05.mma instructions (M=128, N=64,
// K=64 as 4 x K=16) against the layer's weight tile, also bf16 in shared memory, accumulating float32
// in 64 TMEM columns; tcgen05.commit arrives on an mbarrier when they are done.  Each warp reads its
// 32 TMEM lanes back (tcgen05.ld), adds the bias, applies ReLU and writes the next layer's A rows.
// The scalar output layer runs on the CUDA cores in float32.  Widths below 64 and inputs below 64 are
// zero-padded to 64 (the padding multiplies zeros).  Every mbarrier wait is bounded: on timeout the
// kernel reports through the model's error word, waits once more for its MMAs and frees its TMEM.
#include <math.h>

#include <algorithm>

#include "kernels.cuh"
#include "tc.cuh"

namespace fh {

template <int F>
__device__ __forceinline__ void load_row_bf16(const __nv_bfloat16* __restrict__ T, uint64_t r, float (&v)[F]) {
    const __nv_bfloat16* p = T + r * F;
    if constexpr (F == 1) {
        v[0] = __bfloat162float(p[0]);
    } else if constexpr (F == 2) {
        uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(p));
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&w);
        float2 f = __bfloat1622float2(b);
        v[0] = f.x; v[1] = f.y;
    } else if constexpr (F == 4) {
        uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
        uint4 w = __ldg(reinterpret_cast<const uint4*>(p));
        uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&ws[q]));
            v[2 * q] = a.x; v[2 * q + 1] = a.y;
        }
    }
}

template <int F>
__device__ __forceinline__ void interp_level_bf16(const __nv_bfloat16* __restrict__ T, const Corners& k, float* out) {
    float v[16][F];
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
        uint64_t r = k.r0 + ((c & 8) ? k.ot : 0ull) + ((c & 4) ? k.oz : 0u) + ((c & 2) ? k.oy : 0u);
        load_row_bf16<F>(T, r, v[c]);
        load_row_bf16<F>(T, r + k.ox, v[c + 1]);
    }
#pragma unroll
    for (int f = 0; f < F; ++f) {
        float vt[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            float vz[2];
#pragma unroll
            for (int kz = 0; kz < 2; ++kz) {
                const int c = 8 * s + 4 * kz;
                float y0 = fmaf(k.wx, v[c + 1][f] - v[c][f], v[c][f]);
                float y1 = fmaf(k.wx, v[c + 3][f] - v[c + 2][f], v[c + 2][f]);
                vz[kz] = fmaf(k.wy, y1 - y0, y0);
            }
            vt[s] = fmaf(k.wz, vz[1] - vz[0], vz[0]);
        }
        out[f] = fmaf(k.wt, vt[1] - vt[0], vt[0]);
    }
}

// enc[64] (zero beyond L*F) from the bf16 tables.
template <int F>
__device__ __forceinline__ void encode64_bf16(const Levels& lv, const __nv_bfloat16* __restrict__ T, float4 u,
                                              float (&enc)[64]) {
#pragma unroll
    for (int i = 0; i < 64; ++i) enc[i] = 0.0f;
#pragma unroll
    for (int l = 0; l < 64 / F; ++l) {
        if (l < lv.L) {
            Corners k = corners(lv.lv[l], u);
            float o[F];
            interp_level_bf16<F>(T, k, o);
#pragma unroll
            for (int f = 0; f < F; ++f) enc[l * F + f] = o[f];
        }
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b);

// Encodes one sample straight into its bf16 row t of the A tile (column l*F + f for level l, zeros
// beyond L*F), without holding the whole encoding in registers; in training also stores the float32
// encoding to the activation columns.
// Shared-memory stores as explicit st.shared without a memory clobber: the compiler knows they cannot
// alias the global gathers and keeps issuing the next level's loads ahead of them.
__device__ __forceinline__ void sts32(uint32_t a, uint32_t v) { asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v)); }
__device__ __forceinline__ void sts16(uint32_t a, unsigned short v) { asm volatile("st.shared.b16 [%0], %1;" ::"r"(a), "h"(v)); }
__device__ __forceinline__ void sts64(uint32_t a, uint32_t x, uint32_t y) {
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(x), "r"(y));
}
__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w));
}

// Encodes one sample straight into its bf16 row t of the A tile (column l*F + f for level l, zeros
// beyond L*F), without holding the whole encoding in registers; in training also stores the float32
// encoding to the activation columns.
template <int F, bool TRAIN>
__device__ __forceinline__ void encode_row_bf16(const Levels& lv, const __nv_bfloat16* __restrict__ T, float4 u,
                                                uint8_t* tile, int t, float* acts, int64_t n) {
    const uint32_t rowa = tc::smem_addr(tile) + (t >> 3) * 1024 + (t & 7) * 128;
#pragma unroll
    for (int c = 0; c < 8; ++c) sts128(rowa + ((c ^ (t & 7)) << 4), 0u, 0u, 0u, 0u);
#pragma unroll
    for (int l = 0; l < 64 / F; ++l) {
        if (l < lv.L) {
            Corners k = corners(lv.lv[l], u);
            float o[F];
            interp_level_bf16<F>(T, k, o);
            if (TRAIN && acts) {
#pragma unroll
                for (int f = 0; f < F; ++f) acts[(int64_t)(l * F + f) * n] = o[f];
            }
            const int byte = l * F * 2;  // column l*F
            const uint32_t dst = rowa + (((byte >> 4) ^ (t & 7)) << 4) + (byte & 15);
            if constexpr (F == 1) {
                __nv_bfloat16 h = __float2bfloat16_rn(o[0]);
                sts16(dst, *reinterpret_cast<unsigned short*>(&h));
            } else if constexpr (F == 2) {
                sts32(dst, pack_bf16x2(o[0], o[1]));
            } else if constexpr (F == 4) {
                sts64(dst, pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]));
            } else {
                sts128(dst, pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]), pack_bf16x2(o[4], o[5]),
                       pack_bf16x2(o[6], o[7]));
            }
        }
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Columns 32h .. 32h+31 of row r of a 128 x 64 bf16 A tile (128-byte swizzle) from 32 floats.
__device__ __forceinline__ void write_half_row(uint8_t* tile, int r, int h, const float (&x)[32]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = 4 * h + q;
        uint4 w = make_uint4(pack_bf16x2(x[8 * q + 0], x[8 * q + 1]), pack_bf16x2(x[8 * q + 2], x[8 * q + 3]),
                             pack_bf16x2(x[8 * q + 4], x[8 * q + 5]), pack_bf16x2(x[8 * q + 6], x[8 * q + 7]));
        *reinterpret_cast<uint4*>(tile + tc::sw128_off(r, c)) = w;
    }
}

// Row r of a 128 x 64 bf16 A tile (128-byte swizzle) from 64 floats.
__device__ __forceinline__ void write_row(uint8_t* tile, int r, const float (&x)[64]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint4 w = make_uint4(pack_bf16x2(x[8 * c + 0], x[8 * c + 1]), pack_bf16x2(x[8 * c + 2], x[8 * c + 3]),
                             pack_bf16x2(x[8 * c + 4], x[8 * c + 5]), pack_bf16x2(x[8 * c + 6], x[8 * c + 7]));
        *reinterpret_cast<uint4*>(tile + tc::sw128_off(r, c)) = w;
    }
}

// Shared memory of a CTA with R sample tiles: R A tiles (128 x 64 bf16, 16 KB each), the layer weight
// tiles (64 x 64 bf16, 8 KB each), biases, output layer, mbarrier and TMEM slot.
struct TcSmem {
    __host__ __device__ static int W(int R) { return R * 16384; }
    __host__ __device__ static int bias(int R, int nh) { return W(R) + nh * 8192; }
    __host__ __device__ static int wout(int R, int nh) { return bias(R, nh) + nh * 64 * 4; }
    __host__ __device__ static int bout(int R, int nh) { return wout(R, nh) + 64 * 4; }
    __host__ __device__ static int mbar(int R, int nh) { return bout(R, nh) + 16; }
    __host__ __device__ static int slot(int R, int nh) { return mbar(R, nh) + 8; }
    __host__ __device__ static int bytes(int R, int nh) { return slot(R, nh) + 8 + 1024; }  // + alignment slack
};

// R = samples per thread: the CTA holds R tiles of 128 samples (R MMA tiles, R x 64 TMEM columns),
// so every thread keeps the gathers of R samples in flight.
template <int F, bool TRAIN, int R>
__global__ void __launch_bounds__(128) k_forward_tc(const __grid_constant__ Levels lv, const __grid_constant__ MlpShape sh,
                                                    const __nv_bfloat16* __restrict__ Tb,
                                                    const __nv_bfloat16* __restrict__ Pmb, const float* __restrict__ Pm,
                                                    const float* __restrict__ coords, const float* __restrict__ target,
                                                    int64_t n, float* __restrict__ out, float* __restrict__ acts,
                                                    float* __restrict__ gy, double* __restrict__ partial, float two_over_n,
                                                    int* __restrict__ err, const int64_t* __restrict__ seg) {
    if (!TRAIN && seg) {  // packed serving buffers: {offset, count} read at run time
        coords += 4 * seg[0];
        out += seg[0];
        n = seg[1];
    }
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    const int nh = sh.nh, Wd = sh.width;
    uint8_t* Wt = sm + TcSmem::W(R);
    float* bias = reinterpret_cast<float*>(sm + TcSmem::bias(R, nh));
    float* wout = reinterpret_cast<float*>(sm + TcSmem::wout(R, nh));
    float* bout = reinterpret_cast<float*>(sm + TcSmem::bout(R, nh));
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + TcSmem::mbar(R, nh));
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + TcSmem::slot(R, nh));
    const int t = threadIdx.x, warp = t >> 5;
    constexpr uint32_t kCols = 64 * R;

    if (warp == 0) tc::tmem_alloc(slot, kCols);
    if (t == 0) {
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
    }
    // weights of the hidden-producing layers as 64 x 64 bf16 tiles (rows = outputs, K = inputs)
    for (int j = 0; j < nh; ++j) {
        const int fi = j == 0 ? sh.in : Wd;
        for (int e = t; e < 64 * 8; e += 128) {
            const int r = e >> 3, c = e & 7;
            uint32_t w4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k0 = 8 * c + 2 * q;
                __nv_bfloat16 lo = __float2bfloat16_rn(0.0f), hi = lo;
                if (r < Wd && k0 < fi) lo = Pmb[sh.w_off[j] + r * fi + k0];
                if (r < Wd && k0 + 1 < fi) hi = Pmb[sh.w_off[j] + r * fi + k0 + 1];
                __nv_bfloat162 h2 = __halves2bfloat162(lo, hi);
                w4[q] = *reinterpret_cast<uint32_t*>(&h2);
            }
            *reinterpret_cast<uint4*>(Wt + j * 8192 + tc::sw128_off(r, c)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        for (int o = t; o < 64; o += 128) bias[j * 64 + o] = (o < Wd) ? Pm[sh.b_off[j] + o] : 0.0f;
    }
    for (int o = t; o < 64; o += 128) wout[o] = (o < Wd) ? Pm[sh.w_off[nh] + o] : 0.0f;
    if (t == 0) bout[0] = Pm[sh.b_off[nh]];
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    constexpr uint32_t idesc = tc::idesc_bf16(128, 64);
    const uint32_t a_addr = tc::smem_addr(sm), w_addr = tc::smem_addr(Wt);

    uint32_t phase = 0;
    bool bad = false;
    double lsum = 0.0;
    for (int64_t tile = blockIdx.x; tile * (128 * R) < n && !bad; tile += gridDim.x) {
        int64_t idx[R];
        bool valid[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            idx[r] = tile * (128 * R) + r * 128 + t;
            valid[r] = idx[r] < n;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float4 u = valid[r] ? load_coord(coords, idx[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
            encode_row_bf16<F, TRAIN>(lv, Tb, u, sm + r * 16384, t, valid[r] ? acts + idx[r] : nullptr, n);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        float y[R];
#pragma unroll
        for (int r = 0; r < R; ++r) y[r] = bout[0];
        for (int j = 0; j < nh; ++j) {
            if (t == 0) {
                tc::fence_after_sync();
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(tmem + 64 * r, tc::sdesc_sw128(a_addr + r * 16384 + kk * 32),
                                     tc::sdesc_sw128(w_addr + j * 8192 + kk * 32), idesc, kk > 0 ? 1u : 0u);
                tc::mma_commit(mbar);
            }
            const bool ok = tc::mbar_wait(mbar, phase);
            phase ^= 1;
            if (__syncthreads_or(!ok)) { bad = true; break; }
            tc::fence_after_sync();
            const bool last = j + 1 == nh;
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {  // 32 accumulator columns at a time
                    float v[32];
                    tc::tmem_ld32(lane_base + 64 * r + 32 * h, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = fmaxf(v[q] + bias[j * 64 + 32 * h + q], 0.0f);
                    if (TRAIN && valid[r]) {
                        float* a = acts + (int64_t)(sh.in + j * Wd) * n + idx[r];
#pragma unroll
                        for (int q = 0; q < 32; ++q)
                            if (32 * h + q < Wd) a[(int64_t)(32 * h + q) * n] = v[q];
                    }
                    if (!last) {
                        write_half_row(sm + r * 16384, t, h, v);
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; ++q) y[r] = fmaf(wout[32 * h + q], v[q], y[r]);  // scalar output layer
                    }
                }
            }
            if (!last) tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
        }
        if (bad) break;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!valid[r]) continue;
            if (TRAIN) {
                const float d = y[r] - __ldg(target + idx[r]);
                gy[idx[r]] = two_over_n * d;
                lsum += (double)d * (double)d;
            } else {
                out[idx[r]] = y[r];
            }
        }
    }
    if (TRAIN) {
        const double s = block_sum(lsum);
        if (t == 0) partial[blockIdx.x] = s;
    }
    if (bad && t == 0) {
        raise_error(err, 0x7C05);
        tc::mbar_wait(mbar, phase ^ 1);  // one more bounded wait for the MMAs in flight
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// Samples per thread (the kernel supports R tiles per CTA; one measured fastest).
constexpr int kRInfer = 1, kRTrain = 1;

// Launches the tensor-core forward over a.n samples (the largest segment for segment launches) on a
// persistent grid of kCtasPerSm CTAs per SM with half the unified L1/shared memory as shared memory.
// Measured on GB300 (1024^2 renders and 4M uniform points, advect-128^3x32): the gathers depend on L1
// capacity (the maximum shared carve-out halves throughput) and 3 CTAs of 4 warps per SM are as fast
// as 6 or 8; 2 samples per thread (more registers, fewer warps) is slower.  3 x 64 TMEM columns per SM
// never approach the 512 available.  a.grid returns the grid used.
constexpr int kCtasPerSm = 3;
template <int F>
static cudaError_t run_tc(fhash_model* m, bool train, FusedArgs& a) {
    const int R = train ? kRTrain : kRInfer;
    const int smem = TcSmem::bytes(R, m->mlp.nh);
    const void* fn = train ? (const void*)k_forward_tc<F, true, kRTrain> : (const void*)k_forward_tc<F, false, kRInfer>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 50);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (std::max<int64_t>(a.n, 1) + 128 * R - 1) / (128 * R);
    a.grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * kCtasPerSm));
    const __nv_bfloat16* Tb = m->shadow;
    const __nv_bfloat16* Pmb = m->shadow + m->n_table;
    const float* Pm = m->param + m->n_table;
    if (train)
        k_forward_tc<F, true, kRTrain><<<a.grid, 128, smem, a.st>>>(m->lv, m->mlp, Tb, Pmb, Pm, a.coords, a.target, a.n,
                                                                    nullptr, a.acts, a.gy, a.partial, 2.0f / (float)a.n,
                                                                    m->err_word, nullptr);
    else
        k_forward_tc<F, false, kRInfer><<<a.grid, 128, smem, a.st>>>(m->lv, m->mlp, Tb, Pmb, Pm, a.coords, nullptr, a.n,
                                                                     a.out, nullptr, nullptr, nullptr, 0.0f, m->err_word,
                                                                     a.seg);
    return cudaGetLastError();
}

cudaError_t run_tc_any(fhash_model* m, bool train, FusedArgs& a) {
    switch (m->lv.F) {
        case 1: return run_tc<1>(m, train, a);
        case 2: return run_tc<2>(m, train, a);
        case 4: return run_tc<4>(m, train, a);
        case 8: return run_tc<8>(m, train, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fh

namespace fh {
// One CTA waits on an mbarrier that nothing arrives on, with the same bounded wait the tensor-core
// kernels use; when the limit runs out it reports through the model's error word and returns.
__global__ void k_diag_wait(uint64_t limit_ns, int* __restrict__ err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit_ns)) raise_error(err, 0x7C07);
}
}  // namespace fh

extern "C" fhash_status fhash_diag_wait_timeout(fhash_model* m, uint64_t limit_ns, fhash_stream stream) {
    if (!m || limit_ns == 0 || limit_ns > 10000000000ull)
        return fh::set_error(FHASH_EINVAL, "fhash_diag_wait_timeout: limit must be in (0, 10 s]");
    fh::k_diag_wait<<<1, 32, 0, (cudaStream_t)stream>>>(limit_ns, m->err_word);
    FH_CUDA(cudaGetLastError());
    return FHASH_OK;
}
