// Split evaluation of the precision form: the encoding and the MLP as two kernels, chunk by chunk.
//
//   k_encode_rows_bf16  one thread per (level, sample): 16 gathers from the bf16 shadow tables and the
//                       quadrilinear interpolation in float32 (Section 3.2.4, Eqs. 9-12), stored as F bf16
//                       values of row s of an [n][E] bf16 buffer (E = 32 or 64 columns, zero beyond L*F).
//                       It holds no shared memory or TMEM, so it runs at full occupancy; blocks
//                       interleave the levels.
//   k_mlp_tc            the MLP on the tensor cores, fed by TMA.  128-row boxes of the encoding buffer
//                       (64-byte swizzle for E = 32, 128-byte for E = 64) arrive in an S-stage mbarrier
//                       ring.  Per tile, the layer-0 MMAs read the box, each hidden epilogue writes a bf16
//                       tile H, and an N = 16 MMA gives the output; warp roles below.  The per-layer
//                       arithmetic is the fused kernel's (bias stored into TMEM first, MMAs over the same
//                       K steps, ReLU, bf16 rounding, output bias added in float32), so the two paths give
//                       bit-identical outputs.
// One chunk of at most 2^20 samples (64 MB of bf16 encoding at E = 32) stays in L2 between the two
// kernels.  Every mbarrier wait is bounded (2 s); on a timeout the kernel reports through the model's
// error word, waits (bounded) for its MMAs and its copies in flight, frees its TMEM and returns.
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
    // block b serves level b % L, so resident blocks mix L2-resident and HBM-resident levels
    const int l = (int)(blockIdx.x % (unsigned)lv.L);
    const int64_t s = (int64_t)(blockIdx.x / (unsigned)lv.L) * blockDim.x + threadIdx.x;
    if (s >= n) return;
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

// k_mlp_tc is warp-specialised: warps 0-3 run the epilogues (warp w owns TMEM lanes 32w..32w+31, the
// rule for tcgen05.ld/st), warp 4 allocates TMEM and its lane 0 issues every MMA, warp 5's lane 0 issues
// the TMA copies.  Two tiles are in flight per CTA in two TMEM slots of 128 columns (64 hidden
// accumulator columns, 16 output columns) with one bf16 tile H each, so one tile's MMAs run while the
// other tile's epilogue reads TMEM and writes H.  Tiles are taken in pairs, and both the MMA issuer
// and the epilogue warps walk each pair layer by layer, slot 0 then slot 1.  mbarriers:
//   a_full[s]    the box in stage s has landed (TMA transaction count)
//   a_empty[s]   the layer-0 MMAs reading stage s are done (tcgen05.commit), so it can be refilled
//   acc_full[i]  the MMAs of slot i's current layer are done (tcgen05.commit)
//   h_full[i]    the four epilogue warps wrote H[i] and the next layer's bias into slot i's TMEM
//   acc_empty[i] the four epilogue warps read slot i's output column, so the slot takes a new tile
// Every wait is bounded and also gives up once any role has given up (a shared abort flag).
constexpr int kWsEpiWarps = 4, kWsMmaWarp = 4, kWsTmaWarp = 5, kWsThreads = 192;

template <int E>
struct SplitSmem {
    static constexpr int S = E == 32 ? 6 : 3;  // ring stages
    static constexpr int kBox = 128 * E * 2;   // bytes of one box: 128 rows x E bf16
    static constexpr int kBars = 2 * S + 7;    // a_full, a_empty, acc_full[2], h_full[2], acc_empty[2], fin
    __host__ __device__ static int H() { return S * kBox; }
    __host__ __device__ static int W0() { return H() + 2 * 16384; }
    __host__ __device__ static int Wh() { return W0() + 64 * E * 2; }
    __host__ __device__ static int Wo(int nh) { return Wh() + (nh - 1) * 8192; }
    __host__ __device__ static int bias(int nh) { return Wo(nh) + 2048; }
    __host__ __device__ static int bout(int nh) { return bias(nh) + nh * 64 * 4; }
    __host__ __device__ static int bars(int nh) { return bout(nh) + 16; }
    __host__ __device__ static int flag(int nh) { return bars(nh) + kBars * 8; }
    __host__ __device__ static int slot(int nh) { return flag(nh) + 8; }
    __host__ __device__ static int bytes(int nh) { return slot(nh) + 8 + 1024; }  // + alignment slack
};

template <int E>
__global__ void __launch_bounds__(kWsThreads, 1) k_mlp_tc(const __grid_constant__ CUtensorMap map,
                                                          const __grid_constant__ MlpShape sh,
                                                          const __nv_bfloat16* __restrict__ Pmb,
                                                          const float* __restrict__ Pm, int64_t n,
                                                          float* __restrict__ out, int* __restrict__ err) {
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
    uint64_t* a_full = reinterpret_cast<uint64_t*>(sm + C::bars(nh));
    uint64_t* a_empty = a_full + S;
    uint64_t* acc_full = a_empty + S;
    uint64_t* h_full = acc_full + 2;
    uint64_t* acc_empty = h_full + 2;
    uint64_t* fin = acc_empty + 2;
    volatile int* abort = reinterpret_cast<volatile int*>(sm + C::flag(nh));
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + C::slot(nh));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == kWsMmaWarp) tc::tmem_alloc(slot, 256);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&a_full[s], 1);
            tc::mbar_init(&a_empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&h_full[i], kWsEpiWarps);
            tc::mbar_init(&acc_empty[i], kWsEpiWarps);
        }
        tc::mbar_init(fin, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    load_wtile(W0, Pmb + sh.w_off[0], Wd, sh.in, 64, E);
    for (int j = 1; j < nh; ++j) load_wtile(Wh + (j - 1) * 8192, Pmb + sh.w_off[j], Wd, Wd, 64, 64);
    load_wtile(Wo, Pmb + sh.w_off[nh], 1, Wd, 16, 64);
    for (int e = threadIdx.x; e < nh * 64; e += blockDim.x) bias[e] = (e % 64 < Wd) ? Pm[sh.b_off[e / 64] + e % 64] : 0.0f;
    if (threadIdx.x == 0) bout[0] = Pm[sh.b_off[nh]];
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    if (warp < kWsEpiWarps) {  // both slots start at layer 0 from its bias
        store_bias64(tmem + ((uint32_t)(warp * 32) << 16), bias);
        store_bias64(tmem + 128 + ((uint32_t)(warp * 32) << 16), bias);
        tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const int64_t ntiles = (n + 127) / 128;
    const int64_t mine = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int nk_in = (sh.in + 15) / 16, nk_w = (Wd + 15) / 16;
    if (warp == kWsTmaWarp) {
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t k = 0; k < mine; ++k) {
                const int s = (int)(k % S);
                if (k >= S && !tc::mbar_wait_or_abort(&a_empty[s], (uint32_t)((k / S) - 1) & 1u, abort)) break;
                tc::mbar_expect_tx(&a_full[s], C::kBox);
                tc::tma_load_2d(sm + s * C::kBox, &map, 0, (int)((blockIdx.x + k * gridDim.x) * 128), &a_full[s]);
                issued = k + 1;
            }
            // no copy may still be landing when the CTA leaves: wait (bounded) for the last ones
            for (int64_t k = issued > S ? issued - S : 0; k < issued; ++k)
                tc::mbar_wait(&a_full[k % S], (uint32_t)(k / S) & 1u);
        }
    } else if (warp == kWsMmaWarp) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16(128, 64), idesc_out = tc::idesc_bf16(128, 16);
            const uint32_t a0 = tc::smem_addr(sm), h0 = tc::smem_addr(H), w0 = tc::smem_addr(W0),
                           wh = tc::smem_addr(Wh), wo = tc::smem_addr(Wo);
            bool ok = true;
            for (int64_t k0 = 0; k0 < mine && ok; k0 += 2) {
                const int np = mine - k0 < 2 ? (int)(mine - k0) : 2;
                for (int j = 0; j <= nh && ok; ++j) {
                    for (int sl = 0; sl < np && ok; ++sl) {
                        const int64_t k = k0 + sl, u = k >> 1;
                        const uint32_t acc = tmem + sl * 128, hs = h0 + sl * 16384;
                        if (j == 0) {
                            const int s = (int)(k % S);
                            if (u > 0 && !(ok = tc::mbar_wait_or_abort(&acc_empty[sl], (uint32_t)(u - 1) & 1u, abort))) break;
                            if (!(ok = tc::mbar_wait_or_abort(&a_full[s], (uint32_t)(k / S) & 1u, abort))) break;
                            tc::fence_after_sync();
                            for (int kk = 0; kk < nk_in; ++kk) {
                                const uint32_t a = a0 + s * C::kBox + kk * 32, b = w0 + kk * 32;
                                tc::mma_bf16(acc, E == 32 ? tc::sdesc_sw64(a) : tc::sdesc_sw128(a),
                                             E == 32 ? tc::sdesc_sw64(b) : tc::sdesc_sw128(b), idesc, 1u);
                            }
                            tc::mma_commit(&a_empty[s]);
                        } else {
                            if (!(ok = tc::mbar_wait_or_abort(&h_full[sl], (uint32_t)(u * nh + j - 1) & 1u, abort))) break;
                            tc::fence_after_sync();
                            if (j < nh) {
                                for (int kk = 0; kk < nk_w; ++kk)
                                    tc::mma_bf16(acc, tc::sdesc_sw128(hs + kk * 32),
                                                 tc::sdesc_sw128(wh + (j - 1) * 8192 + kk * 32), idesc, 1u);
                            } else {
                                for (int kk = 0; kk < nk_w; ++kk)
                                    tc::mma_bf16(acc + 64, tc::sdesc_sw128(hs + kk * 32), tc::sdesc_sw128(wo + kk * 32),
                                                 idesc_out, kk > 0 ? 1u : 0u);
                            }
                        }
                        tc::mma_commit(&acc_full[sl]);
                    }
                }
            }
            tc::mma_commit(fin);     // arrives when every MMA issued above has completed
            tc::mbar_wait(fin, 0u);  // so none is in flight when TMEM is freed
        }
    } else {  // epilogue warps
        const int row = warp * 32 + lane;
        const uint32_t lanes = (uint32_t)(warp * 32) << 16;
        bool ok = true;
        for (int64_t k0 = 0; k0 < mine && ok; k0 += 2) {
            const int np = mine - k0 < 2 ? (int)(mine - k0) : 2;
            for (int j = 0; j <= nh && ok; ++j) {
                for (int sl = 0; sl < np && ok; ++sl) {
                    const int64_t k = k0 + sl, u = k >> 1;
                    const uint32_t acc = tmem + sl * 128 + lanes;
                    // warp-uniform outcome: tcgen05.ld/st and __syncwarp below need the whole warp
                    ok = __all_sync(0xffffffffu, tc::mbar_wait_or_abort(&acc_full[sl], (uint32_t)(u * (nh + 1) + j) & 1u, abort));
                    if (!ok) break;
                    tc::fence_after_sync();
                    if (j < nh) {
                        hidden_epilogue(acc, H + sl * 16384, row, nullptr, 0, Wd);
                        store_bias64(acc, bias + (j + 1 < nh ? (j + 1) * 64 : 0));  // the next tile starts at layer 0
                        tc::tmem_st_wait();
                        tc::fence_async_smem();
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&h_full[sl]);
                    } else {
                        const float y = tc::tmem_ld1(acc + 64);
                        tc::tmem_ld_wait();
                        const int64_t idx = (blockIdx.x + k * gridDim.x) * 128 + row;
                        if (idx < n) out[idx] = y + bout[0];
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&acc_empty[sl]);
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0 && *abort) raise_error(err, 0x7C08);
    if (warp == kWsMmaWarp) {
        __syncwarp();
        tc::tmem_dealloc(tmem, 256);
    }
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
    // at most two CTAs (2 x 256 TMEM columns) per SM; shared memory (over 76 KB each) never admits a third
    const int per_sm = std::max(1, std::min(2, (227 * 1024) / smem));
    CUtensorMap map;
    if (!make_enc_map(&map, enc, cnt, E)) return set_error(FHASH_ECUDA, "split forward: tensor map encoding failed");
    const int64_t tiles = (cnt + 127) / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * per_sm));
    k_mlp_tc<E><<<grid, kWsThreads, smem, st>>>(map, m->mlp, m->shadow + m->n_table, m->param + m->n_table, cnt, out,
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
        const unsigned g = (unsigned)(((cnt + 255) / 256) * L);
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
