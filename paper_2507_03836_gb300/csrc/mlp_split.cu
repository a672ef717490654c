// Split evaluation of the precision form: the encoding and the MLP as two kernels, chunk by chunk.
//
//   k_encode_rows_bf16  one thread per (level, sample): 16 gathers from the bf16 shadow tables and the
//                       quadrilinear interpolation in float32 (Section 3.2.4, Eqs. 9-12), stored as F bf16
//                       values of row s of an [n][E] bf16 buffer (E = 32 or 64 columns, zero beyond L*F).
//                       It holds no shared memory or TMEM, so it runs at full occupancy.
//   k_mlp_tc            the MLP on the tensor cores, fed by TMA.  128-row boxes of the encoding buffer
//                       (64-byte swizzle for E = 32, 128-byte for E = 64) arrive in an S-stage mbarrier
//                       ring.  Per tile, the layer-0 MMAs read the box, each hidden epilogue writes a bf16
//                       tile H, and an N = 16 MMA gives the output.  The per-layer arithmetic is the fused
//                       kernel's (bias stored into TMEM first, MMAs over the same K steps, ReLU, bf16
//                       rounding, output bias added in float32), so the two paths give bit-identical
//                       outputs.
// One chunk of at most 2^20 samples (64 MB of bf16 encoding at E = 32) stays in L2 between the two
// kernels.  Every mbarrier wait is bounded (2 s); on a timeout the kernel reports through the model's
// error word, waits once more for its MMAs and its copies in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "bf16.cuh"

namespace fh {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();  // csrc/dw_tc.cu

template <int F>
__global__ void __launch_bounds__(256) k_encode_rows_bf16(const __grid_constant__ Levels lv,
                                                          const __nv_bfloat16* __restrict__ T,
                                                          const float* __restrict__ coords, int64_t n, int E,
                                                          __nv_bfloat16* __restrict__ enc) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * lv.L) return;
    const int l = (int)(idx / n);
    const int64_t s = idx - (int64_t)l * n;
    Corners k = corners(lv.lv[l], load_coord(coords, s));
    float o[F];
    interp_level_bf16<F>(T, k, o);
    __nv_bfloat16* row = enc + s * E;
    if constexpr (F == 1) {
        row[l] = __float2bfloat16_rn(o[0]);
    } else if constexpr (F == 2) {
        *reinterpret_cast<uint32_t*>(row + 2 * l) = pack_bf16x2(o[0], o[1]);
    } else if constexpr (F == 4) {
        *reinterpret_cast<uint2*>(row + 4 * l) = make_uint2(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]));
    } else {
        *reinterpret_cast<uint4*>(row + 8 * l) = make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]),
                                                            pack_bf16x2(o[4], o[5]), pack_bf16x2(o[6], o[7]));
    }
    if (l == 0)
        for (int c = lv.L * F; c < E; ++c) row[c] = __float2bfloat16_rn(0.0f);
}

// Shared memory of k_mlp_tc: the box ring, H, the layer-0 weight tile (64 x E), the other hidden
// weight tiles (64 x 64), the output tile (16 x 64), biases, mbarriers and the TMEM slot.
template <int E>
struct SplitSmem {
    static constexpr int S = E == 32 ? 4 : 2;  // ring stages
    static constexpr int kBox = 128 * E * 2;   // bytes of one box: 128 rows x E bf16
    __host__ __device__ static int H() { return S * kBox; }
    __host__ __device__ static int W0() { return H() + 16384; }
    __host__ __device__ static int Wh() { return W0() + 64 * E * 2; }
    __host__ __device__ static int Wo(int nh) { return Wh() + (nh - 1) * 8192; }
    __host__ __device__ static int bias(int nh) { return Wo(nh) + 2048; }
    __host__ __device__ static int bout(int nh) { return bias(nh) + nh * 64 * 4; }
    __host__ __device__ static int bars(int nh) { return bout(nh) + 16; }
    __host__ __device__ static int slot(int nh) { return bars(nh) + (S + 1) * 8; }
    __host__ __device__ static int bytes(int nh) { return slot(nh) + 8 + 1024; }  // + alignment slack
};

template <int E>
__global__ void __launch_bounds__(128, 1) k_mlp_tc(const __grid_constant__ CUtensorMap map,
                                                   const __grid_constant__ MlpShape sh,
                                                   const __nv_bfloat16* __restrict__ Pmb, const float* __restrict__ Pm,
                                                   int64_t n, float* __restrict__ out, int* __restrict__ err) {
    using C = SplitSmem<E>;
    constexpr int S = C::S;
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    const int nh = sh.nh, Wd = sh.width;
    uint8_t* H = sm + C::H();
    uint8_t* W0 = sm + C::W0();
    uint8_t* Wh = sm + C::Wh();
    uint8_t* Wo = sm + C::Wo(nh);
    float* bias = reinterpret_cast<float*>(sm + C::bias(nh));
    float* bout = reinterpret_cast<float*>(sm + C::bout(nh));
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::bars(nh));
    uint64_t* mbar = full + S;
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + C::slot(nh));
    const int t = threadIdx.x, warp = t >> 5;

    if (warp == 0) tc::tmem_alloc(slot, 128);
    if (t == 0) {
        for (int s = 0; s < S; ++s) tc::mbar_init(&full[s], 1);
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
    }
    load_wtile(W0, Pmb + sh.w_off[0], Wd, sh.in, 64, E);
    for (int j = 1; j < nh; ++j) load_wtile(Wh + (j - 1) * 8192, Pmb + sh.w_off[j], Wd, Wd, 64, 64);
    load_wtile(Wo, Pmb + sh.w_off[nh], 1, Wd, 16, 64);
    for (int e = t; e < nh * 64; e += 128) bias[e] = (e % 64 < Wd) ? Pm[sh.b_off[e / 64] + e % 64] : 0.0f;
    if (t == 0) bout[0] = Pm[sh.b_off[nh]];
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
    const int64_t ntiles = (n + 127) / 128;
    const int64_t mine = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    int64_t issued = 0;  // boxes requested so far (thread 0)
    auto request = [&](int64_t q) {
        const int s = (int)(q % S);
        tc::mbar_expect_tx(&full[s], C::kBox);
        tc::tma_load_2d(sm + s * C::kBox, &map, 0, (int)((blockIdx.x + q * gridDim.x) * 128), &full[s]);
    };
    if (t == 0)
        for (; issued < mine && issued < S; ++issued) request(issued);
    store_bias64(lane, bias);  // layer 0 starts from its bias
    tc::tmem_st_wait();
    tc::fence_before_sync();
    __syncthreads();

    constexpr uint32_t idesc = tc::idesc_bf16(128, 64), idesc_out = tc::idesc_bf16(128, 16);
    const uint32_t a0 = tc::smem_addr(sm), h0 = tc::smem_addr(H), w0 = tc::smem_addr(W0), wh = tc::smem_addr(Wh),
                   wo = tc::smem_addr(Wo);
    const int nk_in = (sh.in + 15) / 16, nk_w = (Wd + 15) / 16;
    uint32_t phase = 0;
    bool bad = false;
    int64_t i = 0;
    for (; i < mine; ++i) {
        const int s = (int)(i % S);
        for (int j = 0; j <= nh; ++j) {
            bool ok = true;
            if (t == 0) {
                if (j == 0) ok = tc::mbar_wait(&full[s], (uint32_t)(i / S) & 1u);
                if (ok) {
                    tc::fence_after_sync();
                    if (j == 0) {
                        for (int kk = 0; kk < nk_in; ++kk) {
                            const uint32_t a = a0 + s * C::kBox + kk * 32, b = w0 + kk * 32;
                            tc::mma_bf16(tmem, E == 32 ? tc::sdesc_sw64(a) : tc::sdesc_sw128(a),
                                         E == 32 ? tc::sdesc_sw64(b) : tc::sdesc_sw128(b), idesc, 1u);
                        }
                    } else if (j < nh) {
                        for (int kk = 0; kk < nk_w; ++kk)
                            tc::mma_bf16(tmem, tc::sdesc_sw128(h0 + kk * 32), tc::sdesc_sw128(wh + (j - 1) * 8192 + kk * 32),
                                         idesc, 1u);
                    } else {
                        for (int kk = 0; kk < nk_w; ++kk)
                            tc::mma_bf16(tmem + 64, tc::sdesc_sw128(h0 + kk * 32), tc::sdesc_sw128(wo + kk * 32), idesc_out,
                                         kk > 0 ? 1u : 0u);
                    }
                    tc::mma_commit(mbar);
                }
            }
            if (j == 0 && __syncthreads_or(!ok)) { bad = true; break; }  // the box never arrived
            ok = tc::mbar_wait(mbar, phase);
            phase ^= 1;
            if (__syncthreads_or(!ok)) { bad = true; break; }
            tc::fence_after_sync();
            if (j == 0 && t == 0 && issued < mine) request(issued++);  // stage s has been read: refill it
            if (j == nh) {
                float y = tc::tmem_ld1(lane + 64);
                tc::tmem_ld_wait();
                const int64_t idx = (blockIdx.x + i * gridDim.x) * 128 + t;
                if (idx < n) out[idx] = y + bout[0];
                break;
            }
            hidden_epilogue(lane, H, t, nullptr, 0, Wd);
            store_bias64(lane, bias + (j + 1 < nh ? (j + 1) * 64 : 0));  // the next tile starts at layer 0
            tc::tmem_st_wait();
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
        }
        if (bad) break;
    }
    if (bad && t == 0) {
        raise_error(err, 0x7C08);
        tc::mbar_wait(mbar, phase ^ 1);  // MMAs possibly in flight
        for (int64_t q = i; q < issued; ++q) tc::mbar_wait(&full[q % S], (uint32_t)(q / S) & 1u);  // copies in flight
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// Rows [rows][E] bf16 as a 2D tensor (x = column, y = row) with E x 128 boxes, zero fill past the end.
static bool make_enc_map(CUtensorMap* m, const void* base, int64_t rows, int E) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)E, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)E * 2};
    cuuint32_t box[2] = {(cuuint32_t)E, 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, E == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int E>
static fhash_status mlp_chunk(fhash_model* m, const void* enc, int64_t cnt, float* out, cudaStream_t st) {
    const int smem = SplitSmem<E>::bytes(m->mlp.nh);
    const void* fn = (const void*)k_mlp_tc<E>;
    FH_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FH_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    // at most 3 CTAs (3 x 128 TMEM columns) per SM; shared memory never admits more than 4
    const int per_sm = std::max(1, std::min(3, (227 * 1024) / smem));
    CUtensorMap map;
    if (!make_enc_map(&map, enc, cnt, E)) return set_error(FHASH_ECUDA, "split forward: tensor map encoding failed");
    const int64_t tiles = (cnt + 127) / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * per_sm));
    k_mlp_tc<E><<<grid, 128, smem, st>>>(map, m->mlp, m->shadow + m->n_table, m->param + m->n_table, cnt, out,
                                         m->err_word);
    FH_CUDA(cudaGetLastError());
    return FHASH_OK;
}

fhash_status launch_forward_split(fhash_model* m, const float* coords, int64_t n, float* out, cudaStream_t st) {
    if (n <= 0) return FHASH_OK;
    if (!m->shadow) return set_error(FHASH_EINVAL, "split forward: the model has no bf16 form");
    const int E = m->mlp.in <= 32 ? 32 : 64;
    const int64_t chunk = E == 32 ? (1 << 20) : (1 << 19);  // 64 MB of encoding per chunk
    FH_TRY(grow(m, m->s_enc, (size_t)std::min(n, chunk) * E * 2));
    __nv_bfloat16* enc = (__nv_bfloat16*)m->s_enc.p;
    const int L = m->lv.L;
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t cnt = std::min(chunk, n - c0);
        const unsigned g = (unsigned)((cnt * L + 255) / 256);
        const float* c = coords + 4 * c0;
        switch (m->lv.F) {
            case 1: k_encode_rows_bf16<1><<<g, 256, 0, st>>>(m->lv, m->shadow, c, cnt, E, enc); break;
            case 2: k_encode_rows_bf16<2><<<g, 256, 0, st>>>(m->lv, m->shadow, c, cnt, E, enc); break;
            case 4: k_encode_rows_bf16<4><<<g, 256, 0, st>>>(m->lv, m->shadow, c, cnt, E, enc); break;
            case 8: k_encode_rows_bf16<8><<<g, 256, 0, st>>>(m->lv, m->shadow, c, cnt, E, enc); break;
            default: return set_error(FHASH_EINVAL, "F=%d unsupported", m->lv.F);
        }
        FH_CUDA(cudaGetLastError());
        FH_TRY(E == 32 ? mlp_chunk<32>(m, enc, cnt, out + c0, st) : mlp_chunk<64>(m, enc, cnt, out + c0, st));
    }
    return FHASH_OK;
}

}  // namespace fh
