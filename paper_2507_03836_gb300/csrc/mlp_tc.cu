// Precision form: bf16 tables and MLP on the tcgen05 tensor cores with float32 accumulation in TMEM.
//
// One CTA of 128 threads owns a tile of 128 samples (the MMA's M).  Each thread encodes its sample
// from the bf16 shadow of the tables (Section 3.2.4; interpolation weights and accumulation in
// float32) and writes it as one 128-byte bf16 row of the A operand in shared memory (K-major,
// 128-byte swizzle).  One thread then issues the layer's tcgen05.mma instructions (M=128, N=64,
// K=64 as 4 x K=16) against the layer's weight tile, also bf16 in shared memory, accumulating float32
// in 64 TMEM columns; tcgen05.commit arrives on an mbarrier when they are done.  Each warp reads its
// 32 TMEM lanes back (tcgen05.ld), adds the bias, applies ReLU and writes the next layer's A rows.
// The scalar output layer is an M=128, N=16 MMA of the last hidden rows against a 16-row weight tile
// whose row 0 holds the output weights (rows 1-15 zero) into 16 more TMEM columns; column 0 plus the
// float32 output bias is the result.  Widths below 64 and inputs below 64 are zero-padded to 64 (the
// padding multiplies zeros).  Every mbarrier wait is bounded: on timeout the
// kernel reports through the model's error word, waits once more for its MMAs and frees its TMEM.
#include <math.h>

#include <algorithm>

#include "bf16.cuh"

namespace fh {

// Shared memory of a CTA with R sample tiles: R A tiles (128 x 64 bf16, 16 KB each), the hidden layer
// weight tiles (64 x 64 bf16, 8 KB each), the output weight tile (16 x 64 bf16, 2 KB), biases,
// mbarrier and TMEM slot.
struct TcSmem {
    __host__ __device__ static int W(int R) { return R * 16384; }
    __host__ __device__ static int wout(int R, int nh) { return W(R) + nh * 8192; }
    __host__ __device__ static int bias(int R, int nh) { return wout(R, nh) + 2048; }
    __host__ __device__ static int bout(int R, int nh) { return bias(R, nh) + nh * 64 * 4; }
    __host__ __device__ static int mbar(int R, int nh) { return bout(R, nh) + 16; }
    __host__ __device__ static int slot(int R, int nh) { return mbar(R, nh) + 8; }
    __host__ __device__ static int bytes(int R, int nh) { return slot(R, nh) + 8 + 1024; }  // + alignment slack
};

// R = samples per thread: the CTA holds R tiles of 128 samples (R MMA tiles, R x 64 TMEM columns),
// so every thread keeps the gathers of R samples in flight.
template <int F, bool TRAIN, int R, int LAYOUT>
__global__ void __launch_bounds__(128, 3) k_forward_tc(const __grid_constant__ Levels lv, const __grid_constant__ MlpShape sh,
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
    uint8_t* Wo = sm + TcSmem::wout(R, nh);
    float* bias = reinterpret_cast<float*>(sm + TcSmem::bias(R, nh));
    float* bout = reinterpret_cast<float*>(sm + TcSmem::bout(R, nh));
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + TcSmem::mbar(R, nh));
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + TcSmem::slot(R, nh));
    const int t = threadIdx.x, warp = t >> 5;
    constexpr uint32_t kOut = 64 * R;                               // first output column (16 per tile)
    constexpr uint32_t kCols = (kOut + 16 * R) <= 128 ? 128 : 256;  // power of two for tcgen05.alloc

    if (warp == 0) tc::tmem_alloc(slot, kCols);
    if (t == 0) {
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
    }
    // hidden-producing layers as 64 x 64 bf16 tiles (rows = outputs, K = inputs); output weights as
    // row 0 of a 16 x 64 tile
    for (int j = 0; j < nh; ++j) {
        load_wtile(Wt + j * 8192, Pmb + sh.w_off[j], Wd, j == 0 ? sh.in : Wd, 64, 64);
        for (int o = t; o < 64; o += 128) bias[j * 64 + o] = (o < Wd) ? Pm[sh.b_off[j] + o] : 0.0f;
    }
    load_wtile(Wo, Pmb + sh.w_off[nh], 1, Wd, 16, 64);
    if (t == 0) bout[0] = Pm[sh.b_off[nh]];
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    constexpr uint32_t idesc = tc::idesc_bf16(128, 64), idesc_out = tc::idesc_bf16(128, 16);
    const uint32_t a_addr = tc::smem_addr(sm), w_addr = tc::smem_addr(Wt), wo_addr = tc::smem_addr(Wo);
    const int nk_in = (sh.in + 15) / 16, nk_w = (Wd + 15) / 16;  // K steps that are not all zero
#pragma unroll
    for (int r = 0; r < R; ++r) store_bias64(lane_base + 64 * r, bias);  // layer 0 starts from its bias
    tc::tmem_st_wait();

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
            encode_row_bf16<F, TRAIN, LAYOUT>(lv, Tb, u, sm + r * 16384, t, valid[r] ? acts + idx[r] : nullptr, n);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        float y[R];
        for (int j = 0; j <= nh; ++j) {  // hidden layers onto their bias, then the output layer (j == nh)
            if (t == 0) {
                tc::fence_after_sync();
                const int nk = j == 0 ? nk_in : nk_w;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    for (int kk = 0; kk < nk; ++kk) {
                        if (j < nh)
                            tc::mma_bf16(tmem + 64 * r, tc::sdesc_sw128(a_addr + r * 16384 + kk * 32),
                                         tc::sdesc_sw128(w_addr + j * 8192 + kk * 32), idesc, 1u);
                        else
                            tc::mma_bf16(tmem + kOut + 16 * r, tc::sdesc_sw128(a_addr + r * 16384 + kk * 32),
                                         tc::sdesc_sw128(wo_addr + kk * 32), idesc_out, kk > 0 ? 1u : 0u);
                    }
                tc::mma_commit(mbar);
            }
            const bool ok = tc::mbar_wait(mbar, phase);
            phase ^= 1;
            if (__syncthreads_or(!ok)) { bad = true; break; }
            tc::fence_after_sync();
            if (j == nh) {
#pragma unroll
                for (int r = 0; r < R; ++r) y[r] = tc::tmem_ld1(lane_base + kOut + 16 * r);
                tc::tmem_ld_wait();
#pragma unroll
                for (int r = 0; r < R; ++r) y[r] += bout[0];
                break;
            }
            const float* next_bias = bias + (j + 1 < nh ? (j + 1) * 64 : 0);  // the next tile starts at layer 0
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float* a = (TRAIN && valid[r]) ? acts + (int64_t)(sh.in + j * Wd) * n + idx[r] : nullptr;
                hidden_epilogue(lane_base + 64 * r, sm + r * 16384, t, a, n, Wd);
                store_bias64(lane_base + 64 * r, next_bias);
            }
            tc::tmem_st_wait();
            tc::fence_async_smem();
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
template <int F, int LAYOUT>
static cudaError_t run_tc(fhash_model* m, bool train, FusedArgs& a) {
    const int R = train ? kRTrain : kRInfer;
    const int smem = TcSmem::bytes(R, m->mlp.nh);
    const void* fn = train ? (const void*)k_forward_tc<F, true, kRTrain, LAYOUT>
                           : (const void*)k_forward_tc<F, false, kRInfer, LAYOUT>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 50);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (std::max<int64_t>(a.n, 1) + 128 * R - 1) / (128 * R);
    a.grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * kCtasPerSm));
    const __nv_bfloat16* Tb = m->shadow;
    const __nv_bfloat16* Pmb = m->shadow + m->n_table;
    const float* Pm = m->param + m->n_table;
    if (train)
        k_forward_tc<F, true, kRTrain, LAYOUT><<<a.grid, 128, smem, a.st>>>(
            m->lv, m->mlp, Tb, Pmb, Pm, a.coords, a.target, a.n, nullptr, a.acts, a.gy, a.partial, 2.0f / (float)a.n,
            m->err_word, nullptr);
    else
        k_forward_tc<F, false, kRInfer, LAYOUT><<<a.grid, 128, smem, a.st>>>(
            m->lv, m->mlp, Tb, Pmb, Pm, a.coords, nullptr, a.n, a.out, nullptr, nullptr, nullptr, 0.0f, m->err_word, a.seg);
    return cudaGetLastError();
}

// All levels of a model share one layout; the kernel is instantiated for each.
template <int F>
static cudaError_t run_tc_f(fhash_model* m, bool train, FusedArgs& a) {
    return m->lv.lv[0].layout == FHASH_LAYOUT_BRICK ? run_tc<F, 1>(m, train, a) : run_tc<F, 0>(m, train, a);
}

cudaError_t run_tc_any(fhash_model* m, bool train, FusedArgs& a) {
    switch (m->lv.F) {
        case 1: return run_tc_f<1>(m, train, a);
        case 2: return run_tc_f<2>(m, train, a);
        case 4: return run_tc_f<4>(m, train, a);
        case 8: return run_tc_f<8>(m, train, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fh
