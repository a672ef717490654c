// Device templates of the float32 path: encoding (Section 3.2.4, Eqs. 9-12), the fused MLP decoder
// and its backward with the table scatter-add.  Instantiated per embedding size in inst_f*.cu.
#pragma once
#include <math.h>

#include "common.cuh"

namespace fh {

// ------------------------------------------------------------------ gathers
template <int F>
__device__ __forceinline__ void load_row(const float* __restrict__ T, uint64_t r, float (&v)[F]) {
    const float* p = T + r * F;
    if constexpr (F == 2) {
        float2 a = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = a.x; v[1] = a.y;
    } else if constexpr (F == 4) {
        float4 a = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (F == 8) {
        float4 a = __ldg(reinterpret_cast<const float4*>(p));
        float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int f = 0; f < F; ++f) v[f] = __ldg(p + f);
    }
}

// Steps 3-4 of Section 3.2.4 for one level: the 16 look-ups, trilinear interpolation inside the cells
// at t_Previous and t_Next (Eqs. 10-11) and the linear blend in time (Eq. 12).
template <int F, int LAYOUT = -1>
__device__ __forceinline__ void interp_level(const float* __restrict__ T, const Corners& k, float* out) {
    float v[16][F];
    const int lay = LAYOUT < 0 ? (int)k.layout : LAYOUT;
    if (lay == 1) {
#pragma unroll
        for (int c = 0; c < 16; ++c) load_row<F>(T, corner_row<1>(k, c), v[c]);
    } else if (lay == 2) {
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
            uint64_t r[2];
            masked_corner_pair(k, c, r[0], r[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (r[h] != kInactiveRow) {
                    load_row<F>(T, r[h], v[c + h]);
                } else {
#pragma unroll
                    for (int f = 0; f < F; ++f) v[c + h][f] = 0.0f;  // an inactive corner reads 0
                }
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
            uint64_t r = k.r0 + ((c & 8) ? k.ot : 0ull) + ((c & 4) ? k.oz : 0u) + ((c & 2) ? k.oy : 0u);
            load_row<F>(T, r, v[c]);
            load_row<F>(T, r + k.ox, v[c + 1]);
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

// Weight of corner c = i + 2j + 4k + 8s: product of the per-axis linear weights.
__device__ __forceinline__ float corner_weight(const Corners& k, int c) {
    float a = (c & 1) ? k.wx : 1.0f - k.wx;
    float b = (c & 2) ? k.wy : 1.0f - k.wy;
    float d = (c & 4) ? k.wz : 1.0f - k.wz;
    float e = (c & 8) ? k.wt : 1.0f - k.wt;
    return ((e * d) * b) * a;
}


__device__ __forceinline__ float4 load_coord(const float* __restrict__ coords, int64_t n) {
    return __ldg(reinterpret_cast<const float4*>(coords) + n);
}

// ------------------------------------------------------------------ lookup / encode (thread per sample-level)
template <int F>
__global__ void k_encode(const __grid_constant__ Levels lv, const float* __restrict__ T, const float* __restrict__ coords,
                         int64_t n, float* __restrict__ enc) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * lv.L) return;
    int64_t s = idx / lv.L;
    int l = (int)(idx % lv.L);
    Corners k = corners(lv.lv[l], load_coord(coords, s));
    float o[F];
    interp_level<F>(T, k, o);
#pragma unroll
    for (int f = 0; f < F; ++f) enc[idx * F + f] = o[f];
}

// ------------------------------------------------------------------ MLP with per-thread smem columns
// Thread t of a block owns sample t of the block's tile; its activations live in shared-memory
// column t ([feature][blockDim] layout: consecutive threads hit consecutive banks), so layer shapes
// are runtime values and no thread reads another thread's column (no barriers between layers).
// Weights are staged once per block, transposed (Wt[in][out]) for the forward pass and row-major
// (W[out][in]) for the backward pass, so both inner loops read float4 broadcasts.
// Weight-gradient partials: partial[(chunk * layers + layer) * kDwStride + e], e < fo*fi the weights
// (row-major [fo][fi]), fo*fi + o the biases.
constexpr int kDwStride = 64 * 64 + 64;

constexpr int TB = 128;  // threads (= samples) per block

struct MlpSmemLayout {
    int wt[FHASH_MAX_HIDDEN + 1];  // offsets of the transposed weights per layer
    int wr[FHASH_MAX_HIDDEN + 1];  // offsets of the row-major weights per layer (backward only)
    int b[FHASH_MAX_HIDDEN + 1];
    int acts;                      // offset of the activation columns
    int floats;                    // total
};

__host__ __device__ inline MlpSmemLayout mlp_layout(const MlpShape& sh, bool rowmajor, int ncols) {
    MlpSmemLayout L{};
    int off = 0;
    for (int k = 0; k <= sh.nh; ++k) {
        int fi = k == 0 ? sh.in : sh.width, fo = k == sh.nh ? 1 : sh.width;
        L.wt[k] = off; off += (fi * fo + 3) / 4 * 4;
        if (rowmajor) { L.wr[k] = off; off += fo * ((fi + 3) / 4 * 4); } else L.wr[k] = -1;
        L.b[k] = off; off += (fo + 3) / 4 * 4;
    }
    L.acts = off;
    L.floats = off + ncols * TB;
    return L;
}

__device__ inline void load_mlp(const float* __restrict__ g, const MlpShape& sh, const MlpSmemLayout& L, float* s) {
    for (int k = 0; k <= sh.nh; ++k) {
        int fi = k == 0 ? sh.in : sh.width, fo = k == sh.nh ? 1 : sh.width;
        const int fi4 = (fi + 3) / 4 * 4;  // row-major rows padded with zeros to a multiple of 4
        for (int e = threadIdx.x; e < fi4 * fo; e += blockDim.x) {
            int o = e / fi4, i = e % fi4;
            float w = (i < fi) ? g[sh.w_off[k] + o * fi + i] : 0.0f;
            if (i < fi) s[L.wt[k] + i * fo + o] = w;
            if (L.wr[k] >= 0) s[L.wr[k] + e] = w;
        }
        for (int e = threadIdx.x; e < fo; e += blockDim.x) s[L.b[k] + e] = g[sh.b_off[k] + e];
    }
}

// y[o] = act(sum_i Wt[i][o] x[i] + b[o]) on this thread's column; fo a multiple of 4.
template <bool RELU>
__device__ __forceinline__ void layer_fwd(const float* __restrict__ Wt, const float* __restrict__ b, int fi, int fo,
                                          const float* __restrict__ x, float* __restrict__ y) {
    for (int o = 0; o < fo; o += 4) {
        float a0 = b[o], a1 = b[o + 1], a2 = b[o + 2], a3 = b[o + 3];
#pragma unroll 8
        for (int i = 0; i < fi; ++i) {
            float xv = x[i * TB];
            float4 w = *reinterpret_cast<const float4*>(Wt + i * fo + o);
            a0 = fmaf(w.x, xv, a0);
            a1 = fmaf(w.y, xv, a1);
            a2 = fmaf(w.z, xv, a2);
            a3 = fmaf(w.w, xv, a3);
        }
        if (RELU) { a0 = fmaxf(a0, 0.0f); a1 = fmaxf(a1, 0.0f); a2 = fmaxf(a2, 0.0f); a3 = fmaxf(a3, 0.0f); }
        y[(o + 0) * TB] = a0;
        y[(o + 1) * TB] = a1;
        y[(o + 2) * TB] = a2;
        y[(o + 3) * TB] = a3;
    }
}

// Scalar output layer: w[fi], b[0].
__device__ __forceinline__ float layer_out(const float* __restrict__ w, const float* __restrict__ b, int fi,
                                           const float* __restrict__ x) {
    float a = b[0];
#pragma unroll 8
    for (int i = 0; i < fi; ++i) a = fmaf(w[i], x[i * TB], a);
    return a;
}

// Encodes one sample into column x (x[(l*F + f) * TB]).
template <int F, int LAYOUT>
__device__ __forceinline__ void encode_to_col(const Levels& lv, const float* __restrict__ T, float4 u, float* x) {
    for (int l = 0; l < lv.L; ++l) {
        Corners k = corners<LAYOUT>(lv.lv[l], u);
        float o[F];
        interp_level<F, LAYOUT>(T, k, o);
#pragma unroll
        for (int f = 0; f < F; ++f) x[(l * F + f) * TB] = o[f];
    }
}

// Full MLP forward on this thread's column; bufA holds the input (in rows), bufB/bufC are scratch
// columns of width rows.  Returns y.  When `acts` is given, each hidden output is also written to
// the global column-major activation store.
__device__ __forceinline__ float mlp_fwd_col(const MlpShape& sh, const MlpSmemLayout& L, const float* s, float* bufA,
                                             float* bufB, float* bufC, float* acts, int64_t n, int64_t i) {
    const float* x = bufA;
    float* y = bufB;
    for (int k = 0; k < sh.nh; ++k) {
        int fi = k == 0 ? sh.in : sh.width;
        layer_fwd<true>(s + L.wt[k], s + L.b[k], fi, sh.width, x, y);
        if (acts) {
            float* a = acts + (int64_t)(sh.in + k * sh.width) * n + i;
            for (int o = 0; o < sh.width; ++o) a[(int64_t)o * n] = y[o * TB];
        }
        x = y;
        y = (y == bufB) ? bufC : bufB;
    }
    return layer_out(s + L.wt[sh.nh], s + L.b[sh.nh], sh.width, x);
}

// ------------------------------------------------------------------ forward (inference)
// seg (optional, device): {offset, count} read at run time, so that one captured launch can serve
// batches of any size placed anywhere in a packed buffer (the serving loop replays it every tick).
template <int F, int LAYOUT>
__global__ void __launch_bounds__(TB) k_forward(const __grid_constant__ Levels lv, const __grid_constant__ MlpShape sh,
                                                const float* __restrict__ T, const float* __restrict__ Pm,
                                                const float* __restrict__ coords, int64_t n, float* __restrict__ out,
                                                const int64_t* __restrict__ seg) {
    if (seg) {
        coords += 4 * seg[0];
        out += seg[0];
        n = seg[1];
    }
    extern __shared__ float4 smem4[];
    float* s = reinterpret_cast<float*>(smem4);
    const MlpSmemLayout L = mlp_layout(sh, false, sh.in + 2 * sh.width);
    load_mlp(Pm, sh, L, s);
    __syncthreads();
    float* bufA = s + L.acts + threadIdx.x;
    float* bufB = bufA + sh.in * TB;
    float* bufC = bufB + sh.width * TB;
    for (int64_t i = blockIdx.x * (int64_t)TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        encode_to_col<F, LAYOUT>(lv, T, load_coord(coords, i), bufA);
        out[i] = mlp_fwd_col(sh, L, s, bufA, bufB, bufC, nullptr, n, i);
    }
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// ------------------------------------------------------------------ training forward
// Stores what the backward needs, column-major [feature][n]: acts = enc (sh.in rows) then each
// hidden layer's output (width rows each); gy[n] = dL/dy = 2 (y - target) / N (MSE mean);
// per-block float64 partial sums of (y - target)^2.
template <int F, int LAYOUT>
__global__ void __launch_bounds__(TB) k_train_fwd(const __grid_constant__ Levels lv, const __grid_constant__ MlpShape sh,
                                                  const float* __restrict__ T, const float* __restrict__ Pm,
                                                  const float* __restrict__ coords, const float* __restrict__ target,
                                                  int64_t n, float two_over_n, float* __restrict__ acts,
                                                  float* __restrict__ gy, double* __restrict__ partial) {
    extern __shared__ float4 smem4[];
    float* s = reinterpret_cast<float*>(smem4);
    const MlpSmemLayout L = mlp_layout(sh, false, sh.in + 2 * sh.width);
    load_mlp(Pm, sh, L, s);
    __syncthreads();
    float* bufA = s + L.acts + threadIdx.x;
    float* bufB = bufA + sh.in * TB;
    float* bufC = bufB + sh.width * TB;
    double lsum = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        encode_to_col<F, LAYOUT>(lv, T, load_coord(coords, i), bufA);
        for (int c = 0; c < sh.in; ++c) acts[(int64_t)c * n + i] = bufA[c * TB];
        float y = mlp_fwd_col(sh, L, s, bufA, bufB, bufC, acts, n, i);
        float r = y - __ldg(target + i);
        gy[i] = two_over_n * r;
        lsum += (double)r * (double)r;
    }
    double t = block_sum(lsum);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// ------------------------------------------------------------------ training backward (data path + scatter)
// Thread per sample.  delta_j = dL/dz_{j+1} of layer j is stored column-major at dl[(j*W + o) * n + i]
// (the output layer's at dl[(nh*W) * n + i]); then d_enc = W_0^T delta_0 is scattered into the table
// gradient: every corner row of every level receives weight * d_enc (weights recomputed, not stored).
// p[c] = sum_o W[o][c] d[o] over this thread's columns, c < fi4 = fi rounded up to a multiple of 4
// (row stride fi4; padded columns are zero).
__device__ __forceinline__ void layer_bwd(const float* __restrict__ Wr, int fi4, int fo, const float* __restrict__ d,
                                          float* __restrict__ p) {
    for (int c = 0; c < fi4; c += 4) {
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll 8
        for (int o = 0; o < fo; ++o) {
            float dv = d[o * TB];
            float4 w = *reinterpret_cast<const float4*>(Wr + o * fi4 + c);
            a0 = fmaf(w.x, dv, a0);
            a1 = fmaf(w.y, dv, a1);
            a2 = fmaf(w.z, dv, a2);
            a3 = fmaf(w.w, dv, a3);
        }
        p[(c + 0) * TB] = a0;
        p[(c + 1) * TB] = a1;
        p[(c + 2) * TB] = a2;
        p[(c + 3) * TB] = a3;
    }
}

template <int F, int LAYOUT>
__device__ __forceinline__ void scatter_sample(const Levels& lv, float* __restrict__ G, float4 u, const float* de) {
    for (int l = 0; l < lv.L; ++l) {
        Corners k = corners<LAYOUT>(lv.lv[l], u);
        float g[F];
#pragma unroll
        for (int f = 0; f < F; ++f) g[f] = de[(l * F + f) * TB];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float w = corner_weight(k, c);
            const uint64_t r = corner_row<LAYOUT>(k, c);
            if (LAYOUT == 2 && r == kInactiveRow) continue;  // inactive corners take no gradient
            float* dst = G + r * F;
            if constexpr (F == 2) {
                red_add2(dst, w * g[0], w * g[1]);
            } else if constexpr (F == 4) {
                red_add4(dst, w * g[0], w * g[1], w * g[2], w * g[3]);
            } else if constexpr (F == 8) {
                red_add4(dst, w * g[0], w * g[1], w * g[2], w * g[3]);
                red_add4(dst + 4, w * g[4], w * g[5], w * g[6], w * g[7]);
            } else {
#pragma unroll
                for (int f = 0; f < F; ++f) red_add(dst + f, w * g[f]);
            }
        }
    }
}

template <int F, int LAYOUT>
__global__ void __launch_bounds__(TB) k_train_bwd(const __grid_constant__ Levels lv, const __grid_constant__ MlpShape sh,
                                                  float* __restrict__ G, const float* __restrict__ Pm,
                                                  const float* __restrict__ coords, int64_t n,
                                                  const float* __restrict__ acts, const float* __restrict__ gy,
                                                  float* __restrict__ dl) {
    extern __shared__ float4 smem4[];
    float* s = reinterpret_cast<float*>(smem4);
    const int W = sh.width;
    const int cols = ((sh.in > W ? sh.in : W) + 3) / 4 * 4 + W;
    const MlpSmemLayout L = mlp_layout(sh, true, cols);
    load_mlp(Pm, sh, L, s);
    __syncthreads();
    float* d = s + L.acts + threadIdx.x;  // current delta (W rows)
    float* p = d + W * TB;                // propagated (max(in, W) rows)
    for (int64_t i = blockIdx.x * (int64_t)TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        const float g = gy[i];
        dl[(int64_t)(sh.nh * W) * n + i] = g;
        const float* wout = s + L.wt[sh.nh];  // output layer weights [W] (same in both layouts)
        const float* a = acts + (int64_t)(sh.in + (sh.nh - 1) * W) * n + i;
        for (int o = 0; o < W; ++o) d[o * TB] = (a[(int64_t)o * n] > 0.0f) ? wout[o] * g : 0.0f;
        for (int j = sh.nh - 1; j >= 0; --j) {
            float* dst = dl + (int64_t)j * W * n + i;
            for (int o = 0; o < W; ++o) dst[(int64_t)o * n] = d[o * TB];
            const int fi4 = ((j == 0 ? sh.in : W) + 3) / 4 * 4;
            layer_bwd(s + L.wr[j], fi4, W, d, p);
            if (j > 0) {
                const float* aj = acts + (int64_t)(sh.in + (j - 1) * W) * n + i;
                for (int c = 0; c < W; ++c) d[c * TB] = (aj[(int64_t)c * n] > 0.0f) ? p[c * TB] : 0.0f;
            }
        }
        scatter_sample<F, LAYOUT>(lv, G, load_coord(coords, i), p);  // p now holds d_enc (sh.in rows)
    }
}

// Host-side launch of the fused kernels for one embedding size.
struct FusedArgs {
    const Levels* lv;
    const MlpShape* sh;
    const float* T;
    float* G;
    const float* Pm;
    const float* coords;
    const float* target;
    int64_t n;
    float* out;
    float* acts;
    float* gy;
    float* dl;
    double* partial;
    int grid;
    cudaStream_t st;
    const int64_t* seg;  // optional device {offset, count} for the forward kernels
};

template <int F, int LAYOUT>
cudaError_t run_fused_layout(int which, const FusedArgs& a) {
    const MlpShape& sh = *a.sh;
    const int W = sh.width;
    const int cols_f = sh.in + 2 * W, cols_b = ((sh.in > W ? sh.in : W) + 3) / 4 * 4 + W;
    const int smem = (which == 2 ? mlp_layout(sh, true, cols_b).floats : mlp_layout(sh, false, cols_f).floats) * 4;
    const void* fn = which == 0   ? (const void*)k_forward<F, LAYOUT>
                     : which == 1 ? (const void*)k_train_fwd<F, LAYOUT>
                                  : (const void*)k_train_bwd<F, LAYOUT>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (which == 0)
        k_forward<F, LAYOUT><<<a.grid, TB, smem, a.st>>>(*a.lv, sh, a.T, a.Pm, a.coords, a.n, a.out, a.seg);
    else if (which == 1)
        k_train_fwd<F, LAYOUT><<<a.grid, TB, smem, a.st>>>(*a.lv, sh, a.T, a.Pm, a.coords, a.target, a.n,
                                                           2.0f / (float)a.n, a.acts, a.gy, a.partial);
    else
        k_train_bwd<F, LAYOUT><<<a.grid, TB, smem, a.st>>>(*a.lv, sh, a.G, a.Pm, a.coords, a.n, a.acts, a.gy, a.dl);
    return cudaGetLastError();
}

// All levels of a model share one layout; the per-sample kernels are instantiated for each.
template <int F>
cudaError_t run_fused(int which, const FusedArgs& a) {
    switch (a.lv->lv[0].layout) {
        case FHASH_LAYOUT_BRICK: return run_fused_layout<F, 1>(which, a);
        case FHASH_LAYOUT_MASKED: return run_fused_layout<F, 2>(which, a);
        default: return run_fused_layout<F, 0>(which, a);
    }
}

}  // namespace fh
