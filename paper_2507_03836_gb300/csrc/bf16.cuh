// bf16 helpers shared by the precision-form kernels (csrc/mlp_tc.cu, csrc/mlp_split.cu): table
// gathers and quadrilinear interpolation from the bf16 shadow tables (Section 3.2.4, Eqs. 10-12, with
// float32 weights and accumulation), packing, swizzled shared-memory tiles, and the per-layer pieces
// of the tensor-core MLP that both kernels run with identical arithmetic.
#pragma once
#include "kernels.cuh"
#include "tc.cuh"

namespace fh {

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

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

template <int F, int LAYOUT = -1>
__device__ __forceinline__ void interp_level_bf16(const __nv_bfloat16* __restrict__ T, const Corners& k, float* out) {
    float v[16][F];
    if (LAYOUT < 0 ? k.layout == 1u : LAYOUT == 1) {  // masked levels never reach the bf16 form
#pragma unroll
        for (int c = 0; c < 16; ++c) load_row_bf16<F>(T, corner_row<1>(k, c), v[c]);
    } else {
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
            uint64_t r = k.r0 + ((c & 8) ? k.ot : 0ull) + ((c & 4) ? k.oz : 0u) + ((c & 2) ? k.oy : 0u);
            load_row_bf16<F>(T, r, v[c]);
            load_row_bf16<F>(T, r + k.ox, v[c + 1]);
        }
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
template <int F, bool TRAIN, int LAYOUT>
__device__ __forceinline__ void encode_row_bf16(const Levels& lv, const __nv_bfloat16* __restrict__ T, float4 u,
                                                uint8_t* tile, int t, float* acts, int64_t n) {
    const uint32_t rowa = tc::smem_addr(tile) + (t >> 3) * 1024 + (t & 7) * 128;
#pragma unroll
    for (int c = 0; c < 8; ++c) sts128(rowa + ((c ^ (t & 7)) << 4), 0u, 0u, 0u, 0u);
#pragma unroll
    for (int l = 0; l < 64 / F; ++l) {
        if (l < lv.L) {
            Corners k = corners<LAYOUT>(lv.lv[l], u);
            float o[F];
            interp_level_bf16<F, LAYOUT>(T, k, o);
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


// Weight tile of one layer as bf16 rows o < rows (outputs; zero for o >= fo) by `cols` K columns
// (inputs; zero for k >= fi), W row-major [fo][fi].  cols = 64: 128-byte swizzle; cols = 32:
// 64-byte swizzle.  Called by every thread of the CTA.
__device__ inline void load_wtile(uint8_t* dst, const __nv_bfloat16* __restrict__ W, int fo, int fi, int rows, int cols) {
    const int chunks = cols / 8;
    for (int e = threadIdx.x; e < rows * chunks; e += blockDim.x) {
        const int r = e / chunks, c = e % chunks;
        uint32_t w4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k0 = 8 * c + 2 * q;
            __nv_bfloat16 lo = __float2bfloat16_rn(0.0f), hi = lo;
            if (r < fo && k0 < fi) lo = W[r * fi + k0];
            if (r < fo && k0 + 1 < fi) hi = W[r * fi + k0 + 1];
            __nv_bfloat162 h2 = __halves2bfloat162(lo, hi);
            w4[q] = *reinterpret_cast<uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(dst + (cols == 64 ? tc::sw128_off(r, c) : tc::sw64_off(r, c))) =
            make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
}

// Every warp writes bias[0..63] into 64 TMEM columns of its 32 lanes starting at lane_taddr, so that
// the layer's MMAs accumulate onto the bias.  `bias` is 16-byte aligned shared memory.  The caller
// waits (tcgen05.wait::st) before the barrier that precedes the MMAs.
__device__ __forceinline__ void store_bias64(uint32_t lane_taddr, const float* bias) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float b[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 v = reinterpret_cast<const float4*>(bias + 32 * h)[q];
            b[4 * q] = v.x; b[4 * q + 1] = v.y; b[4 * q + 2] = v.z; b[4 * q + 3] = v.w;
        }
        tc::tmem_st32(lane_taddr + 32 * h, b);
    }
}

// max(a, 0) and max(b, 0) rounded to bf16 (nearest even) and packed, b in the upper half: one
// cvt.rn.relu.bf16x2.f32.  For finite inputs this equals pack_bf16x2(fmaxf(b, 0), fmaxf(a, 0))
// with the halves swapped back, since rounding keeps the sign.
__device__ __forceinline__ uint32_t relu_pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Hidden-layer epilogue of one sample row: the 64 accumulator columns of this thread's lane (bias +
// products) -> ReLU -> bf16 row r of the 128-byte-swizzled tile H.  With `a` non-null, also stores the
// float32 activations a[o * stride] for o < width (training keeps them for the backward pass).
__device__ __forceinline__ void hidden_epilogue(uint32_t lane_taddr, uint8_t* H, int r, float* a, int64_t stride,
                                                int width) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[32];
        tc::tmem_ld32(lane_taddr + 32 * h, v);
        tc::tmem_ld_wait();
        if (a) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (32 * h + q < width) a[(int64_t)(32 * h + q) * stride] = fmaxf(v[q], 0.0f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 w = make_uint4(relu_pack_bf16x2(v[8 * q + 0], v[8 * q + 1]), relu_pack_bf16x2(v[8 * q + 2], v[8 * q + 3]),
                                       relu_pack_bf16x2(v[8 * q + 4], v[8 * q + 5]), relu_pack_bf16x2(v[8 * q + 6], v[8 * q + 7]));
            *reinterpret_cast<uint4*>(H + tc::sw128_off(r, 4 * h + q)) = w;
        }
    }
}

}  // namespace fh
