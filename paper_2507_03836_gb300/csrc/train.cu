// Training pass split by access pattern (float32 and the backward of the bf16 form):
//   k_encode_cols   level-major gathers (thread per level and sample), encoding to global columns;
//   k_mlp_fwd_t     MLP forward + MSE from those columns on 128-sample tiles (weights and activation
//                   tiles in shared memory, register-tiled GEMMs), dL/dy and float64 loss partials;
//   k_mlp_bwd_t     MLP backward data path on the same tiles: deltas per layer and d(loss)/d(encoding)
//                   to global columns;
//   k_scatter_cols  backward of Eqs. 10-12: level-major vector reductions into the table gradient, with
//                   coarse levels accumulated in shared memory first (privatised) to avoid thousands of
//                   same-address atomics per row;
//   k_dw_tiles      weight gradients over the batch, 4 x 4 register tiles per thread.
// The gather and scatter kernels carry no MLP state, so they run at full occupancy.
#include <math.h>

#include <algorithm>

#include "kernels.cuh"

namespace fh {

// ------------------------------------------------------------------ gathers / scatters (level-major)
// LAYOUT: the model's row layout (all levels share it), fixed per instantiation.
template <int F, int LAYOUT>
__global__ void __launch_bounds__(256) k_encode_cols(const __grid_constant__ Levels lv, const float* __restrict__ T,
                                                     const float* __restrict__ coords, int64_t n, float* __restrict__ enc) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * lv.L) return;
    const int l = (int)(idx / n);
    const int64_t s = idx - (int64_t)l * n;
    Corners k = corners<LAYOUT>(lv.lv[l], load_coord(coords, s));
    float o[F];
    interp_level<F, LAYOUT>(T, k, o);
#pragma unroll
    for (int f = 0; f < F; ++f) enc[(int64_t)(l * F + f) * n + s] = o[f];
}

template <int F>
__device__ __forceinline__ void red_row(float* dst, float w, const float (&g)[F]) {
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

// Blocks [first[l], first[l+1]) serve level l, `per[l]` samples each; priv[l] = 1 when the whole level
// table (rows*F floats) is accumulated in shared memory by each block before one flush.
struct ScatterPlan {
    int32_t first[FHASH_MAX_LEVELS + 1];
    int64_t per[FHASH_MAX_LEVELS];
    int32_t priv[FHASH_MAX_LEVELS];
};

template <int F, int LAYOUT>
__global__ void __launch_bounds__(256) k_scatter_cols(const __grid_constant__ Levels lv, const __grid_constant__ ScatterPlan P,
                                                      float* __restrict__ G, const float* __restrict__ coords, int64_t n,
                                                      const float* __restrict__ denc, int64_t dsf, int64_t dss) {
    extern __shared__ float acc[];
    int l = 0;
    while (l + 1 < lv.L && (int)blockIdx.x >= P.first[l + 1]) ++l;
    const int64_t s0 = (int64_t)(blockIdx.x - P.first[l]) * P.per[l];
    const int64_t s1 = min(n, s0 + P.per[l]);
    const Level& L = lv.lv[l];
    if (P.priv[l]) {
        const int64_t nrow = (int64_t)L.nrows;
        for (int64_t e = threadIdx.x; e < nrow * F; e += blockDim.x) acc[e] = 0.0f;
        __syncthreads();
        for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
            Corners k = corners<LAYOUT>(L, load_coord(coords, s));
            float g[F];
#pragma unroll
            for (int f = 0; f < F; ++f) g[f] = denc[(int64_t)(l * F + f) * dsf + s * dss];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float w = corner_weight(k, c);
                const uint64_t r = corner_row<LAYOUT>(k, c);
                if (LAYOUT == 2 && r == kInactiveRow) continue;  // masked: inactive corners take no gradient
                float* dst = acc + (r - L.base) * F;
#pragma unroll
                for (int f = 0; f < F; ++f) atomicAdd(dst + f, w * g[f]);
            }
        }
        __syncthreads();
        float* Gl = G + L.base * F;
        for (int64_t e = threadIdx.x; e < nrow * F; e += blockDim.x)
            if (acc[e] != 0.0f) red_add(Gl + e, acc[e]);
    } else {
        const int64_t s = s0 + threadIdx.x;
        if (s >= s1) return;
        Corners k = corners<LAYOUT>(L, load_coord(coords, s));
        float g[F];
#pragma unroll
        for (int f = 0; f < F; ++f) g[f] = denc[(int64_t)(l * F + f) * dsf + s * dss];
        if constexpr (F == 2) {
            // x-neighbours are consecutive rows: when the lower row is even the pair is one aligned 16-byte
            // reduction instead of two 8-byte ones (fewer L2 atomic operations)
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                uint64_t r, r1;
                if constexpr (LAYOUT == 2) {
                    masked_corner_pair(k, c, r, r1);
                } else {
                    r = corner_row<LAYOUT>(k, c);
                    r1 = corner_row<LAYOUT>(k, c + 1);
                }
                const float w0 = corner_weight(k, c), w1 = corner_weight(k, c + 1);
                // (kInactiveRow is odd, so an inactive lower row never takes the paired form)
                if (r1 == r + 1 && (r & 1u) == 0u) {
                    red_add4(G + r * 2, w0 * g[0], w0 * g[1], w1 * g[0], w1 * g[1]);
                } else {
                    if (LAYOUT != 2 || r != kInactiveRow) red_add2(G + r * 2, w0 * g[0], w0 * g[1]);
                    if (LAYOUT != 2 || r1 != kInactiveRow) red_add2(G + r1 * 2, w1 * g[0], w1 * g[1]);
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                uint64_t r[2];
                if constexpr (LAYOUT == 2) {
                    masked_corner_pair(k, c, r[0], r[1]);
                } else {
                    r[0] = corner_row<LAYOUT>(k, c);
                    r[1] = corner_row<LAYOUT>(k, c + 1);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (LAYOUT != 2 || r[h] != kInactiveRow) red_row<F>(G + r[h] * F, corner_weight(k, c + h), g);
            }
        }
    }
}

// ------------------------------------------------------------------ MLP on 128-sample tiles (float32 SIMT)
// A block of 256 threads takes 128 samples at a time.  Layer inputs and outputs live in shared memory
// feature-major, X[k][s] (k < 64 features, s < 128 samples), and every layer is a small GEMM: thread
// (to = tid / 32, ts = tid % 32) owns outputs o = 8 to .. 8 to + 7 of samples s = 4 ts .. 4 ts + 3,
// reading per k one float4 of X (a warp reads 512 contiguous bytes) and two float4 of the weights
// (the same address across the warp): 32 FMAs per 3 shared loads.  Weights are staged once per block,
// zero-padded to 64 outputs.
constexpr int kTileS = 128, kTileF = 64;

// acc[u][v] += sum over k < K of Wk[k][8 to + u] * X[k][4 ts + v] (row strides 64 and 128 floats).
__device__ __forceinline__ void tile_gemm(const float* __restrict__ X, const float* __restrict__ Wk, int K,
                                          float (&acc)[8][4]) {
    const int ts = threadIdx.x & 31, to = threadIdx.x >> 5;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 x = *reinterpret_cast<const float4*>(X + k * kTileS + 4 * ts);
        const float4 w0 = *reinterpret_cast<const float4*>(Wk + k * kTileF + 8 * to);
        const float4 w1 = *reinterpret_cast<const float4*>(Wk + k * kTileF + 8 * to + 4);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(w[u], xv[v], acc[u][v]);
    }
}

// Rows [r][c] of a layer's weights in shared memory with row stride 64: transposed (Wt[in][out], the
// forward's Wk) or as stored (W[out][in], the backward's Wk); zero outside fo x fi.
__device__ inline void stage_weights(float* dst, const float* __restrict__ W, int fo, int fi, bool transpose) {
    for (int e = threadIdx.x; e < kTileF * kTileF; e += blockDim.x) {
        const int r = e / kTileF, c = e % kTileF;
        float v = 0.0f;
        if (transpose) { if (r < fi && c < fo) v = W[c * fi + r]; }
        else if (r < fo && c < fi) v = W[r * fi + c];
        dst[e] = v;
    }
}

// Global column rows [rows][n] of a tile into X[k][s] (zero past n).
__device__ inline void load_tile(float* X, const float* __restrict__ cols, int rows, int64_t n, int64_t t0) {
    for (int e = threadIdx.x; e < rows * kTileS; e += blockDim.x) {
        const int k = e / kTileS, sidx = e % kTileS;
        X[e] = (t0 + sidx < n) ? cols[(int64_t)k * n + t0 + sidx] : 0.0f;
    }
}

// Shared memory (floats): nh weight blocks of 64 x 64, biases [nh][64], output weights [64], two tiles.
__host__ __device__ inline int tile_smem_floats(int nh) { return nh * kTileF * kTileF + nh * kTileF + kTileF + 2 * kTileF * kTileS; }

__global__ void __launch_bounds__(256) k_mlp_fwd_t(const __grid_constant__ MlpShape sh, const float* __restrict__ Pm,
                                                   const float* __restrict__ target, int64_t n, float two_over_n,
                                                   float* __restrict__ acts, float* __restrict__ gy,
                                                   double* __restrict__ partial) {
    extern __shared__ float4 sm4[];
    float* Wk = reinterpret_cast<float*>(sm4);
    const int nh = sh.nh, Wd = sh.width;
    float* bias = Wk + nh * kTileF * kTileF;
    float* wout = bias + nh * kTileF;
    float* T0 = wout + kTileF;
    float* T1 = T0 + kTileF * kTileS;
    for (int j = 0; j < nh; ++j) {
        stage_weights(Wk + j * kTileF * kTileF, Pm + sh.w_off[j], Wd, j == 0 ? sh.in : Wd, true);
        for (int o = threadIdx.x; o < kTileF; o += blockDim.x) bias[j * kTileF + o] = o < Wd ? Pm[sh.b_off[j] + o] : 0.0f;
    }
    for (int o = threadIdx.x; o < kTileF; o += blockDim.x) wout[o] = o < Wd ? Pm[sh.w_off[nh] + o] : 0.0f;
    const float bo = Pm[sh.b_off[nh]];
    const int ts = threadIdx.x & 31, to = threadIdx.x >> 5;
    double lsum = 0.0;
    for (int64_t t0 = (int64_t)blockIdx.x * kTileS; t0 < n; t0 += (int64_t)gridDim.x * kTileS) {
        __syncthreads();  // weights staged / the previous tile consumed
        load_tile(T0, acts, sh.in, n, t0);
        __syncthreads();
        float* src = T0;
        float* dst = T1;
        const bool vec = (n & 3) == 0 && t0 + kTileS <= n;  // whole tile, 16-byte aligned rows
        for (int j = 0; j < nh; ++j) {
            float acc[8][4];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = bias[j * kTileF + 8 * to + u];
            tile_gemm(src, Wk + j * kTileF * kTileF, j == 0 ? sh.in : Wd, acc);
            float* arow = acts + (int64_t)(sh.in + j * Wd) * n;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int o = 8 * to + u;
                float r[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) r[v] = fmaxf(acc[u][v], 0.0f);
                *reinterpret_cast<float4*>(dst + o * kTileS + 4 * ts) = make_float4(r[0], r[1], r[2], r[3]);
                if (o < Wd) {
                    float* a4 = arow + (int64_t)o * n + t0 + 4 * ts;
                    if (vec) {
                        *reinterpret_cast<float4*>(a4) = make_float4(r[0], r[1], r[2], r[3]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (t0 + 4 * ts + v < n) a4[v] = r[v];
                    }
                }
            }
            __syncthreads();
            float* t = src; src = dst; dst = t;
        }
        if (threadIdx.x < kTileS && t0 + threadIdx.x < n) {  // scalar output layer on the last hidden tile
            float y = bo;
            for (int o = 0; o < Wd; ++o) y = fmaf(wout[o], src[o * kTileS + threadIdx.x], y);
            const int64_t i = t0 + threadIdx.x;
            const float d = y - __ldg(target + i);
            gy[i] = two_over_n * d;
            lsum += (double)d * (double)d;
        }
    }
    const double t = block_sum(lsum);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// dl[(j*W + o) * n + i] = delta of layer j's output (the output layer's at row nh*W); denc[c * n + i] =
// d(loss)/d(encoding c).  Delta tiles stay in shared memory from layer to layer.
__global__ void __launch_bounds__(256) k_mlp_bwd_t(const __grid_constant__ MlpShape sh, const float* __restrict__ Pm,
                                                   int64_t n, const float* __restrict__ acts, const float* __restrict__ gy,
                                                   float* __restrict__ dl, float* __restrict__ denc) {
    extern __shared__ float4 sm4[];
    float* Wk = reinterpret_cast<float*>(sm4);
    const int nh = sh.nh, Wd = sh.width;
    float* wout = Wk + nh * kTileF * kTileF + nh * kTileF;
    float* T0 = wout + kTileF;
    float* T1 = T0 + kTileF * kTileS;
    for (int j = 0; j < nh; ++j) stage_weights(Wk + j * kTileF * kTileF, Pm + sh.w_off[j], Wd, j == 0 ? sh.in : Wd, false);
    for (int o = threadIdx.x; o < kTileF; o += blockDim.x) wout[o] = o < Wd ? Pm[sh.w_off[nh] + o] : 0.0f;
    const int ts = threadIdx.x & 31, to = threadIdx.x >> 5;
    for (int64_t t0 = (int64_t)blockIdx.x * kTileS; t0 < n; t0 += (int64_t)gridDim.x * kTileS) {
        __syncthreads();
        // output layer: delta of the last hidden layer = (a > 0) * wout * dL/dy
        const float* alast = acts + (int64_t)(sh.in + (nh - 1) * Wd) * n;
        float* dlast = dl + (int64_t)((nh - 1) * Wd) * n;
        for (int e = threadIdx.x; e < kTileF * kTileS; e += blockDim.x) {
            const int o = e / kTileS, sidx = e % kTileS;
            const int64_t i = t0 + sidx;
            float d = 0.0f;
            if (o < Wd && i < n) {
                const float g = gy[i];
                d = alast[(int64_t)o * n + i] > 0.0f ? wout[o] * g : 0.0f;
                dlast[(int64_t)o * n + i] = d;
                if (o == 0) dl[(int64_t)(nh * Wd) * n + i] = g;
            }
            T0[e] = d;
        }
        __syncthreads();
        float* src = T0;
        float* dst = T1;
        const bool vec = (n & 3) == 0 && t0 + kTileS <= n;  // whole tile, 16-byte aligned rows
        for (int j = nh - 1; j >= 0; --j) {
            const int fi = j == 0 ? sh.in : Wd;
            float acc[8][4] = {};
            tile_gemm(src, Wk + j * kTileF * kTileF, Wd, acc);  // p[c][s] = sum_o W_j[o][c] delta_j[o][s]
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = 8 * to + u;
                const int64_t i0 = t0 + 4 * ts;
                if (j > 0) {
                    const float* arow = acts + (int64_t)(sh.in + (j - 1) * Wd + c) * n;
                    float* drow = dl + (int64_t)((j - 1) * Wd + c) * n;
                    float r[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    if (c < Wd && vec) {
                        const float4 a = *reinterpret_cast<const float4*>(arow + i0);
                        r[0] = a.x > 0.0f ? acc[u][0] : 0.0f;
                        r[1] = a.y > 0.0f ? acc[u][1] : 0.0f;
                        r[2] = a.z > 0.0f ? acc[u][2] : 0.0f;
                        r[3] = a.w > 0.0f ? acc[u][3] : 0.0f;
                        *reinterpret_cast<float4*>(drow + i0) = make_float4(r[0], r[1], r[2], r[3]);
                    } else if (c < Wd) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            if (i0 + v >= n) continue;
                            r[v] = arow[i0 + v] > 0.0f ? acc[u][v] : 0.0f;
                            drow[i0 + v] = r[v];
                        }
                    }
                    *reinterpret_cast<float4*>(dst + c * kTileS + 4 * ts) = make_float4(r[0], r[1], r[2], r[3]);
                } else if (c < fi) {
                    float* e4 = denc + (int64_t)c * n + i0;
                    if (vec) {
                        *reinterpret_cast<float4*>(e4) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (i0 + v < n) e4[v] = acc[u][v];
                    }
                }
            }
            __syncthreads();
            float* t = src; src = dst; dst = t;
        }
    }
}

// Weight-gradient partials of every layer over chunks of samples (blockIdx.y = layer).  Thread (ob, ib)
// owns dW[4ob..4ob+3][4ib..4ib+3] and, when ib == 0, db of its rows.  Slabs of 32 samples are staged in
// shared memory sample-major (sd[c][o], sa[c][i]), double-buffered through registers, so each thread
// reads one float4 of deltas and one float4 of activations per sample: 16 FMAs per 2 shared loads.
// Partials in the kDwStride layout.
struct DwLayers {
    const float* a[FHASH_MAX_HIDDEN + 1];
    const float* d[FHASH_MAX_HIDDEN + 1];
    int32_t fi[FHASH_MAX_HIDDEN + 1], fo[FHASH_MAX_HIDDEN + 1];
};

__global__ void __launch_bounds__(256) k_dw_tiles(const __grid_constant__ DwLayers Ls, int64_t n, int64_t chunk,
                                                  float* __restrict__ partial) {
    constexpr int TS = 32, LD = 68, KS = 16;  // KS = staged values per thread: 128 rows x 32 samples / 256
    __shared__ __align__(16) float sa[TS][LD];
    __shared__ __align__(16) float sd[TS][LD];
    const int layer = blockIdx.y;
    const float* __restrict__ a = Ls.a[layer];
    const float* __restrict__ d = Ls.d[layer];
    const int fi = Ls.fi[layer], fo = Ls.fo[layer], rows = fi + fo;
    const int nig = (fi + 3) / 4, nob = (fo + 3) / 4;
    const int ob = threadIdx.x / nig, ib = threadIdx.x % nig;
    const bool active = (int)threadIdx.x < nob * nig;
    const int64_t n0 = blockIdx.x * chunk, n1 = min(n, n0 + chunk);
    float stage[KS];
    auto fetch = [&](int64_t t0) {
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int q = threadIdx.x + 256 * k, r = q / TS, c = q % TS;
            const int64_t smp = t0 + c;
            float v = 0.0f;
            if (r < rows && smp < n1) v = r < fi ? a[(int64_t)r * n + smp] : d[(int64_t)(r - fi) * n + smp];
            stage[k] = v;
        }
    };
    float acc[4][4] = {}, bacc[4] = {};
    if (n0 < n1) fetch(n0);
    for (int64_t t0 = n0; t0 < n1; t0 += TS) {
        __syncthreads();  // the previous slab has been read
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int q = threadIdx.x + 256 * k, r = q / TS, c = q % TS;
            if (r < fi) sa[c][r] = stage[k];
            else if (r < rows) sd[c][r - fi] = stage[k];
        }
        __syncthreads();
        if (t0 + TS < n1) fetch(t0 + TS);  // the next slab's loads stay in flight during the FMAs
        if (active) {
#pragma unroll 8
            for (int c = 0; c < TS; ++c) {
                const float4 dv = *reinterpret_cast<const float4*>(&sd[c][4 * ob]);
                const float4 av = *reinterpret_cast<const float4*>(&sa[c][4 * ib]);
                const float dd[4] = {dv.x, dv.y, dv.z, dv.w}, aa[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(dd[u], aa[v], acc[u][v]);
                    bacc[u] += dd[u];
                }
            }
        }
    }
    if (!active) return;
    float* out = partial + ((int64_t)blockIdx.x * gridDim.y + layer) * kDwStride;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int o = 4 * ob + u;
        if (o >= fo) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = 4 * ib + v;
            if (i < fi) out[o * fi + i] = acc[u][v];
        }
        if (ib == 0) out[fo * fi + o] = bacc[u];
    }
}

// grad[off[layer] + e] += sum over chunks of the partials (weights then biases, contiguous per layer).
__global__ void k_dw_reduce2(const float* __restrict__ partial, int nchunk, const __grid_constant__ DwLayers Ls,
                             const __grid_constant__ MlpShape sh, float* __restrict__ gm) {
    const int layer = blockIdx.y, e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Ls.fo[layer] * Ls.fi[layer] + Ls.fo[layer]) return;
    float s = 0.0f;
    for (int c = 0; c < nchunk; ++c) s += partial[((int64_t)c * gridDim.y + layer) * kDwStride + e];
    gm[sh.w_off[layer] + e] += s;
}

__global__ void k_loss2(const double* __restrict__ partial, int nb, int64_t n, double* __restrict__ loss) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (double)n;
}

cudaError_t run_tc_any(fhash_model* m, bool train, FusedArgs& a);
bool launch_mlp_f32tc(fhash_model* m, const float* target, const float* gyin, int64_t n, float* acts, float* dl,
                      float* denc, double* partial, int max_partials, int* grid, cudaStream_t st, cudaError_t* err);
bool launch_dw_tc(fhash_model* m, const float* acts, const float* dl, int64_t n, float* wpart, size_t wpart_bytes,
                  int* nchunk_out, cudaStream_t st, cudaError_t* err, bool split3);

template <int F, int LAYOUT>
static cudaError_t scatter_run(fhash_model* m, const ScatterPlan& Pp, const ScatterPlan& Pf, int bp, int bf,
                               int64_t priv_floats, const float* coords, int64_t n, const float* denc, int64_t dsf,
                               int64_t dss, cudaStream_t st) {
    if (bp > 0) {
        const int smem = (int)(priv_floats * 4);
        cudaError_t e = cudaFuncSetAttribute((const void*)k_scatter_cols<F, LAYOUT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(smem, 1));
        if (e != cudaSuccess) return e;
        k_scatter_cols<F, LAYOUT><<<bp, 256, smem, st>>>(m->lv, Pp, m->grad, coords, n, denc, dsf, dss);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (bf > 0) k_scatter_cols<F, LAYOUT><<<bf, 256, 0, st>>>(m->lv, Pf, m->grad, coords, n, denc, dsf, dss);
    return cudaGetLastError();
}

template <int F>
static cudaError_t scatter_launch(fhash_model* m, const float* coords, int64_t n, const float* denc, int64_t dsf,
                                  int64_t dss, cudaStream_t st) {
    constexpr int64_t kPrivMax = 32768;  // floats of a level accumulated in shared memory (128 KB)
    // Two launches: the privatised coarse levels (shared memory sized for the largest of them) and the
    // fine levels (no shared memory, so their blocks run at full occupancy).
    ScatterPlan Pp{}, Pf{};
    int bp = 0, bf = 0;
    int64_t priv_floats = 0;
    for (int l = 0; l < m->lv.L; ++l) {
        const Level& L = m->lv.lv[l];
        const int64_t fl = (int64_t)L.nrows * F;
        Pp.first[l] = bp;
        Pf.first[l] = bf;
        if (fl <= kPrivMax) {
            Pp.priv[l] = 1;
            Pp.per[l] = std::max<int64_t>(2048, (n + 63) / 64);  // at most 64 flushes of the level
            priv_floats = std::max(priv_floats, fl);
            bp += (int)((n + Pp.per[l] - 1) / Pp.per[l]);
        } else {
            Pf.priv[l] = 0;
            Pf.per[l] = 256;
            bf += (int)((n + 255) / 256);
        }
    }
    Pp.first[m->lv.L] = bp;
    Pf.first[m->lv.L] = bf;
    switch (m->lv.lv[0].layout) {
        case FHASH_LAYOUT_BRICK: return scatter_run<F, 1>(m, Pp, Pf, bp, bf, priv_floats, coords, n, denc, dsf, dss, st);
        case FHASH_LAYOUT_MASKED: return scatter_run<F, 2>(m, Pp, Pf, bp, bf, priv_floats, coords, n, denc, dsf, dss, st);
        default: return scatter_run<F, 0>(m, Pp, Pf, bp, bf, priv_floats, coords, n, denc, dsf, dss, st);
    }
}

template <int F>
static void encode_cols(fhash_model* m, unsigned grid, const float* coords, int64_t n, float* acts, cudaStream_t st) {
    switch (m->lv.lv[0].layout) {
        case FHASH_LAYOUT_BRICK: k_encode_cols<F, 1><<<grid, 256, 0, st>>>(m->lv, m->param, coords, n, acts); break;
        case FHASH_LAYOUT_MASKED: k_encode_cols<F, 2><<<grid, 256, 0, st>>>(m->lv, m->param, coords, n, acts); break;
        default: k_encode_cols<F, 0><<<grid, 256, 0, st>>>(m->lv, m->param, coords, n, acts); break;
    }
}

// Backward of the encoding alone: d(encoding) given row-major [n][L*F] (the layout of fhash_encode).
fhash_status launch_encode_backward(fhash_model* m, const float* coords, int64_t n, const float* denc, cudaStream_t st) {
    const int64_t LF = (int64_t)m->lv.L * m->lv.F;
    switch (m->lv.F) {
        case 1: FH_CUDA(scatter_launch<1>(m, coords, n, denc, 1, LF, st)); break;
        case 2: FH_CUDA(scatter_launch<2>(m, coords, n, denc, 1, LF, st)); break;
        case 4: FH_CUDA(scatter_launch<4>(m, coords, n, denc, 1, LF, st)); break;
        case 8: FH_CUDA(scatter_launch<8>(m, coords, n, denc, 1, LF, st)); break;
        default: return set_error(FHASH_EINVAL, "F=%d unsupported", m->lv.F);
    }
    return FHASH_OK;
}

fhash_status launch_grads2(fhash_model* m, const float* coords, const float* target, int64_t n, double* loss_dev,
                           cudaStream_t st) {
    const MlpShape& sh = m->mlp;
    const int W = sh.width, F = m->lv.F;
    const int64_t A = sh.in + (int64_t)sh.nh * W;  // activation rows
    const int64_t D = (int64_t)sh.nh * W + 1;       // delta rows
    FH_TRY(grow(m, m->s_acts, (size_t)(A * n * 4)));
    FH_TRY(grow(m, m->s_gacts, (size_t)((D + 1 + sh.in) * n * 4)));
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, (int64_t)num_sms() * 8));  // loss partials
    const int nl = sh.nh + 1;
    // weight-gradient chunks: about 4 blocks per SM over all layers, at least 512 samples each
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>((n + 511) / 512, (int64_t)num_sms() * 4 / nl));
    const int64_t chunk = ((n + nchunk - 1) / nchunk + 31) / 32 * 32;
    const size_t tc_part = (size_t)num_sms() * nl * kDwStride * 4;
    FH_TRY(grow(m, m->s_partial, std::max((size_t)nchunk * nl * kDwStride * 4, tc_part) + (size_t)nb * 8 + 64));
    float* acts = (float*)m->s_acts.p;
    float* gy = (float*)m->s_gacts.p;
    float* dl = gy + n;
    float* denc = dl + D * n;
    double* lpart = (double*)m->s_partial.p;
    const size_t wpart_off = ((size_t)nb * 8 + 63) / 64 * 64;  // fixed before nb shrinks to the grid used
    float* wpart = (float*)((char*)m->s_partial.p + wpart_off);
    const float* Pm = m->param + m->n_table;
    const int tsmem = tile_smem_floats(sh.nh) * 4;
    // resident blocks only: each stages the weights once and then walks its share of the tiles
    const int tile_grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + kTileS - 1) / kTileS,
                                                                       (int64_t)num_sms() * std::max(1, (227 * 1024) / tsmem)));

    // forward: encoding + MLP (bf16 form: one tensor-core kernel writes the same activations)
    bool fused_mlp = false;
    if (m->shadow) {
        FusedArgs a{};
        a.coords = coords; a.target = target; a.n = n; a.acts = acts; a.gy = gy; a.partial = lpart; a.st = st;
        FH_CUDA(run_tc_any(m, true, a));
        nb = a.grid;  // at most one loss partial per CTA, never more than the buffer holds
        tev_record(m, TEV_ENCODE, st);
    } else {
        const unsigned eg = (unsigned)((n * m->lv.L + 255) / 256);
        switch (F) {
            case 1: encode_cols<1>(m, eg, coords, n, acts, st); break;
            case 2: encode_cols<2>(m, eg, coords, n, acts, st); break;
            case 4: encode_cols<4>(m, eg, coords, n, acts, st); break;
            case 8: encode_cols<8>(m, eg, coords, n, acts, st); break;
            default: return set_error(FHASH_EINVAL, "F=%d unsupported", F);
        }
        FH_CUDA(cudaGetLastError());
        tev_record(m, TEV_ENCODE, st);
        // the MLP's forward, loss and backward data path fused on the tensor cores (3xTF32), where the
        // shape allows; otherwise the float32 SIMT tile kernels
        int g = 0;
        cudaError_t e = cudaSuccess;
        if (launch_mlp_f32tc(m, target, nullptr, n, acts, dl, denc, lpart, nb, &g, st, &e)) {
            FH_CUDA(e);
            nb = g;
            fused_mlp = true;
        } else {
            FH_CUDA(cudaFuncSetAttribute((const void*)k_mlp_fwd_t, cudaFuncAttributeMaxDynamicSharedMemorySize, tsmem));
            nb = std::min(nb, tile_grid);  // one loss partial per block
            k_mlp_fwd_t<<<nb, 256, tsmem, st>>>(sh, Pm, target, n, 2.0f / (float)n, acts, gy, lpart);
            FH_CUDA(cudaGetLastError());
        }
    }
    k_loss2<<<1, 256, 0, st>>>(lpart, nb, n, loss_dev);
    FH_CUDA(cudaGetLastError());
    // backward: MLP data path, table scatter, weight gradients
    if (!fused_mlp && m->shadow) {
        // precision form: the backward data path on the tensor cores from the stored activations and dL/dy
        int g = 0;
        cudaError_t e = cudaSuccess;
        if (launch_mlp_f32tc(m, target, gy, n, acts, dl, denc, lpart, nb, &g, st, &e)) {
            FH_CUDA(e);
            fused_mlp = true;
        }
    }
    if (!fused_mlp) {
        const int bb = tile_grid;
        FH_CUDA(cudaFuncSetAttribute((const void*)k_mlp_bwd_t, cudaFuncAttributeMaxDynamicSharedMemorySize, tsmem));
        k_mlp_bwd_t<<<bb, 256, tsmem, st>>>(sh, Pm, n, acts, gy, dl, denc);
        FH_CUDA(cudaGetLastError());
    }
    tev_record(m, TEV_MLP, st);
    switch (F) {
        case 1: FH_CUDA(scatter_launch<1>(m, coords, n, denc, n, 1, st)); break;
        case 2: FH_CUDA(scatter_launch<2>(m, coords, n, denc, n, 1, st)); break;
        case 4: FH_CUDA(scatter_launch<4>(m, coords, n, denc, n, 1, st)); break;
        case 8: FH_CUDA(scatter_launch<8>(m, coords, n, denc, n, 1, st)); break;
    }
    tev_record(m, TEV_SCATTER, st);
    // weight and bias gradients on the tensor cores (TMA + tcgen05 kind::tf32): tf32 inputs for the bf16
    // form, the 3xTF32 split (float32 accuracy) for the float32 form; float32 SIMT tiles when the batch
    // does not suit the tensor maps (n not a multiple of 4, or below 32); then one reduction of the partials
    DwLayers Ls{};
    for (int j = 0; j < nl; ++j) {
        Ls.fi[j] = j == 0 ? sh.in : W;
        Ls.fo[j] = j == sh.nh ? 1 : W;
        Ls.a[j] = (j == 0) ? acts : acts + (int64_t)(sh.in + (j - 1) * W) * n;
        Ls.d[j] = dl + (int64_t)j * W * n;
    }
    int nparts = nchunk;
    cudaError_t e = cudaSuccess;
    if (launch_dw_tc(m, acts, dl, n, wpart, m->s_partial.bytes - wpart_off, &nparts, st, &e, m->shadow == nullptr)) {
        FH_CUDA(e);
    } else {
        nparts = nchunk;
        k_dw_tiles<<<dim3(nchunk, nl), 256, 0, st>>>(Ls, n, chunk, wpart);
        FH_CUDA(cudaGetLastError());
    }
    k_dw_reduce2<<<dim3((kDwStride + 255) / 256, nl), 256, 0, st>>>(wpart, nparts, Ls, sh, m->grad + m->n_table);
    FH_CUDA(cudaGetLastError());
    tev_record(m, TEV_DW, st);
    return FHASH_OK;
}

}  // namespace fh
