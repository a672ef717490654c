// Sample-streaming renderer with adaptive ray marching (Section 3.3, Algorithm 1) and the time-slice
// decode (temporal super-resolution at fractional t, Section 3.3).
//
// Each ARM round: every alive ray marches on from where it stopped and emits up to N_s samples that lie
// in occupied space (empty-space skipping with the occupancy grid); all emitted samples are evaluated
// by the fused encode+MLP kernel in one launch; each ray then composites its samples front to back and
// rays that exited the box or became opaque leave the alive list.  N_s = max(min(N_r / N_a, pace), 1).
// Which samples a ray takes and in what order does not depend on the pace, so neither does the image.
//
// The ray geometry decides integer sample indices, so it is written with explicit round-to-nearest
// intrinsics (no contraction into fused multiply-adds): any IEEE float32 evaluation of the same steps
// gives the same samples.
#include <math.h>

#include <algorithm>

#include "render.cuh"

namespace fh {

cudaError_t run_fused_any(int F, int which, const FusedArgs& a);

__device__ __forceinline__ bool occ_bit(const RenderGeo& g, int t, int x, int y, int z) {
    int64_t b = ((int64_t)(z >> 3) * g.nby + (y >> 3)) * g.nbx + (x >> 3);
    if (!g.occ_any[(int64_t)t * g.nbrick + b]) return false;
    int lx = x & 7, ly = y & 7, lz = z & 7;
    int mi = (lx & 1) | ((ly & 1) << 1) | ((lz & 1) << 2) | ((lx & 2) << 2) | ((ly & 2) << 3) | ((lz & 2) << 4) |
             ((lx & 4) << 4) | ((ly & 4) << 5) | ((lz & 4) << 6);
    return (g.occ[((int64_t)t * g.nbrick + b) * 16 + (mi >> 5)] >> (mi & 31)) & 1u;
}

// Occupancy of the sample at model coordinate u (nearest voxel), at t_norm.
__device__ __forceinline__ bool sample_occupied(const RenderGeo& g, const float u[3]) {
    int v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float q = __fmul_rn(u[a], (float)(g.S[a] - 1));
        v[a] = (int)floorf(__fadd_rn(q, 0.5f));
        if (v[a] < 0 || v[a] >= g.S[a]) return false;
    }
    if (occ_bit(g, g.tp, v[0], v[1], v[2])) return true;
    return g.use_tn && occ_bit(g, g.tn, v[0], v[1], v[2]);
}

__global__ void k_ray_init(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs, int* __restrict__ alive,
                           int* __restrict__ n_alive, float4* __restrict__ rgba, int* __restrict__ counts) {
    int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= g.W * g.H) return;
    int i = pix % g.W, j = pix / g.W;
    float sx = __fsub_rn(__fdiv_rn((float)(2 * i + 1), (float)g.W), 1.0f);
    float sy = __fsub_rn(1.0f, __fdiv_rn((float)(2 * j + 1), (float)g.H));
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = __fadd_rn(__fadd_rn(g.fwd[a], __fmul_rn(sx, g.right[a])), __fmul_rn(sy, g.up[a]));
    float ln = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])), __fmul_rn(d[2], d[2])));
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = __fdiv_rn(d[a], ln);
    float tn = -INFINITY, tf = INFINITY;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0f) {
            float t0 = __fdiv_rn(__fsub_rn(-1.0f, g.eye[a]), d[a]);
            float t1 = __fdiv_rn(__fsub_rn(1.0f, g.eye[a]), d[a]);
            tn = fmaxf(tn, fminf(t0, t1));
            tf = fminf(tf, fmaxf(t0, t1));
        } else if (g.eye[a] < -1.0f || g.eye[a] > 1.0f) {
            hit = false;
        }
    }
    float tmin = fmaxf(tn, 0.0f), tmax = tf;
    hit = hit && (tmin <= tmax);
    RayState s;
    s.d[0] = d[0]; s.d[1] = d[1]; s.d[2] = d[2];
    s.tmin = tmin; s.tmax = tmax; s.k = 0; s.flags = hit ? 0 : 1;
    s.C[0] = s.C[1] = s.C[2] = 0.0f; s.T = 1.0f; s.count = 0;
    rs[pix] = s;
    if (hit) {
        alive[atomicAdd(n_alive, 1)] = pix;
    } else {
        rgba[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (counts) counts[pix] = 0;
    }
}

// Index of the last sample that surely still lies in the empty 8^3 brick holding voxel v, for a ray
// whose sample k is in it.  The brick holds the samples whose nearest voxel is in [8b, 8b + 7] on each
// axis, that is model coordinate q = u (S - 1) in [8b - 0.5, 8b + 7.5); the ray parameter where q
// reaches that box's far faces, pulled in by 0.01 voxel (far more than the float32 rounding of q and of
// this bound, about 1e-4 voxel), limits the samples that can be skipped.  Samples never evaluated there
// are unoccupied, so the set of samples (and the image) is the same as stepping through them one by one.
// Float32 throughout: the FP64 rate of this GPU is a small fraction of its FP32 rate.
__device__ __forceinline__ int empty_brick_last_sample(const RenderGeo& g, const RayState& s, const int v[3], int k) {
    float t_exit = 3.0e38f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float d = s.d[ax];
        if (d == 0.0f) continue;
        const int b8 = (v[ax] >> 3) * 8;
        const float qf = d > 0.0f ? (float)b8 + 7.49f : (float)b8 - 0.49f;  // the face the ray runs to
        const float uf = qf / (float)(g.S[ax] - 1);
        t_exit = fminf(t_exit, ((2.0f * uf - 1.0f) - g.eye[ax]) / d);  // u = (eye + t d + 1) / 2
    }
    const float kl = floorf((t_exit - s.tmin) / g.delta);
    return kl > (float)k ? (int)fminf(kl, (float)(1 << 24)) : k;
}

// Marches each alive ray on until it has up to Ns occupied samples (or leaves the box); writes their
// model coordinates to slots [a*Ns, a*Ns + cnt).  A sample in an 8^3 brick that is empty at both time
// steps in use jumps the ray to the last sample inside that brick (empty-space skipping).
__global__ void k_arm_generate(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs,
                               const int* __restrict__ alive, int na, int ns, float4* __restrict__ coords,
                               int* __restrict__ cnt, unsigned long long* __restrict__ marched) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= na) return;
    int pix = alive[a];
    RayState s = rs[pix];
    int c = 0, k = s.k;
    long long steps = 0;
    while (c < ns) {
        if (k >= (1 << 24)) { s.flags |= 1; break; }
        float sk = __fadd_rn(s.tmin, __fmul_rn((float)k, g.delta));
        if (!(sk <= s.tmax)) { s.flags |= 1; break; }
        float u[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) u[ax] = __fmul_rn(__fadd_rn(__fadd_rn(g.eye[ax], __fmul_rn(sk, s.d[ax])), 1.0f), 0.5f);
        ++steps;
        int v[3];
        bool inside = true;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            v[ax] = (int)floorf(__fadd_rn(__fmul_rn(u[ax], (float)(g.S[ax] - 1)), 0.5f));
            inside = inside && v[ax] >= 0 && v[ax] < g.S[ax];
        }
        if (!inside) { ++k; continue; }
        const int64_t b = ((int64_t)(v[2] >> 3) * g.nby + (v[1] >> 3)) * g.nbx + (v[0] >> 3);
        const bool any_p = g.occ_any[(int64_t)g.tp * g.nbrick + b] != 0;
        const bool any_n = g.use_tn && g.occ_any[(int64_t)g.tn * g.nbrick + b] != 0;
        if (!any_p && !any_n) {
            k = empty_brick_last_sample(g, s, v, k) + 1;  // samples up to the returned one are empty
            continue;
        }
        ++k;
        if ((any_p && occ_bit(g, g.tp, v[0], v[1], v[2])) || (any_n && occ_bit(g, g.tn, v[0], v[1], v[2])))
            coords[(int64_t)a * ns + c++] = make_float4(u[0], u[1], u[2], g.t_norm);
    }
    rs[pix].k = k;
    rs[pix].flags = s.flags;
    cnt[a] = c;
    if (marched) atomicAdd(marched, (unsigned long long)steps);
}

// Transfer function lookup (256 RGBA entries, linear interpolation) and front-to-back compositing;
// rays that are done write their pixel, the others are appended to the next alive list.
__global__ void k_arm_composite(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs,
                                const int* __restrict__ alive, int na, int ns, const int* __restrict__ cnt,
                                const float* __restrict__ vals, const float4* __restrict__ tf,
                                int* __restrict__ next, int* __restrict__ n_next, float4* __restrict__ rgba,
                                int* __restrict__ counts, unsigned long long* __restrict__ used) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= na) return;
    int pix = alive[a];
    RayState s = rs[pix];
    int c = cnt[a];
    bool opaque = false;
    int u = 0;
    for (int j = 0; j < c && !opaque; ++j) {
        float v = vals[(int64_t)a * ns + j];
        float x = fminf(fmaxf(v, 0.0f), 1.0f) * 255.0f;
        int i0 = min((int)floorf(x), 254);
        float f = x - (float)i0;
        float4 p = __ldg(tf + i0), q = __ldg(tf + i0 + 1);
        float r = p.x + f * (q.x - p.x), gg = p.y + f * (q.y - p.y), b = p.z + f * (q.z - p.z), al = p.w + f * (q.w - p.w);
        float w = s.T * al;
        s.C[0] += w * r; s.C[1] += w * gg; s.C[2] += w * b;
        s.T *= (1.0f - al);
        ++u;
        if (1.0f - s.T > 0.99f) opaque = true;
    }
    s.count += u;
    if (used) atomicAdd(used, (unsigned long long)u);
    if (opaque || (s.flags & 1)) {
        rgba[pix] = make_float4(s.C[0], s.C[1], s.C[2], 1.0f - s.T);
        if (counts) counts[pix] = s.count;
        rs[pix].flags = s.flags | 2;
    } else {
        next[atomicAdd(n_next, 1)] = pix;
    }
    rs[pix].C[0] = s.C[0]; rs[pix].C[1] = s.C[1]; rs[pix].C[2] = s.C[2];
    rs[pix].T = s.T;
    rs[pix].count = s.count;
}

RenderGeo make_geo(const fhash_model* m, const fhash_camera* cam, float t_norm, int w, int h) {
    RenderGeo g{};
    for (int a = 0; a < 3; ++a) {
        g.eye[a] = cam->eye[a]; g.right[a] = cam->right[a]; g.up[a] = cam->up[a]; g.fwd[a] = cam->fwd[a];
        g.S[a] = (int)m->fbb_size[a];
    }
    int64_t smax = std::max(m->fbb_size[0], std::max(m->fbb_size[1], m->fbb_size[2]));
    g.delta = (float)(1.0 / (double)(smax - 1));
    g.t_norm = t_norm;
    g.W = w; g.H = h;
    g.nt = (int)m->nt;
    // time steps of the occupancy used at t_norm (same float32 steps as the sample test)
    const float tq = t_norm * (float)(g.nt - 1);  // host code is built without FP contraction
    int tp = (int)floorf(tq);
    tp = std::min(std::max(tp, 0), g.nt - 1);
    const float wt = tq - (float)tp;
    g.tp = tp;
    g.tn = std::min(tp + 1, g.nt - 1);
    g.use_tn = wt > 0.0f ? 1 : 0;
    g.nbx = m->nbx; g.nby = m->nby; g.nbrick = m->nbx * m->nby * m->nbz;
    g.occ = m->occ; g.occ_any = m->occ_any;

    return g;
}

// Decode: the model on a regular grid over the FBB at fractional t (n'_d = up*(S_d-1)+1 points per
// axis, u_d = j/(n'_d - 1)), out[z][y][x].
template <int F>
__global__ void __launch_bounds__(TB) k_decode(const __grid_constant__ Levels lv, const __grid_constant__ MlpShape sh,
                                               const float* __restrict__ T, const float* __restrict__ Pm, int nx,
                                               int ny, int nz, float t_norm, float* __restrict__ out) {
    extern __shared__ float4 smem4[];
    float* s = reinterpret_cast<float*>(smem4);
    const MlpSmemLayout L = mlp_layout(sh, false, sh.in + 2 * sh.width);
    load_mlp(Pm, sh, L, s);
    __syncthreads();
    float* bufA = s + L.acts + threadIdx.x;
    float* bufB = bufA + sh.in * TB;
    float* bufC = bufB + sh.width * TB;
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        float4 u = make_float4(__fdiv_rn((float)x, (float)(nx - 1)), __fdiv_rn((float)y, (float)(ny - 1)),
                               __fdiv_rn((float)z, (float)(nz - 1)), t_norm);
        encode_to_col<F, -1>(lv, T, u, bufA);
        out[i] = mlp_fwd_col(sh, L, s, bufA, bufB, bufC, nullptr, n, i);
    }
}

template <int F>
static cudaError_t run_decode(fhash_model* m, int nx, int ny, int nz, float t, float* out, cudaStream_t st) {
    const MlpShape& sh = m->mlp;
    const int smem = mlp_layout(sh, false, sh.in + 2 * sh.width).floats * 4;
    cudaError_t e = cudaFuncSetAttribute((const void*)k_decode<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int64_t n = (int64_t)nx * ny * nz;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + TB - 1) / TB, (int64_t)num_sms() * 16));
    k_decode<F><<<grid, TB, smem, st>>>(m->lv, sh, m->param, m->param + m->n_table, nx, ny, nz, t, out);
    return cudaGetLastError();
}

int64_t decode_points(int64_t S, int up) { return (int64_t)up * (S - 1) + 1; }

// Grid coordinates of points [i0, i0 + cnt) of the decode grid (same float32 steps as k_decode).
__global__ void k_grid_coords(int nx, int ny, int nz, float t_norm, int64_t i0, int64_t cnt, float4* __restrict__ co) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    int64_t i = i0 + q;
    int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
    co[q] = make_float4(__fdiv_rn((float)x, (float)(nx - 1)), __fdiv_rn((float)y, (float)(ny - 1)),
                        __fdiv_rn((float)z, (float)(nz - 1)), t_norm);
}

}  // namespace fh

using namespace fh;

extern "C" {

fhash_status fhash_decode_dims(const fhash_model* m, int32_t upsample, int64_t dims[3]) {
    if (!m || !dims || upsample < 1 || upsample > 8) return set_error(FHASH_EINVAL, "fhash_decode_dims: bad arguments");
    for (int a = 0; a < 3; ++a) dims[a] = decode_points(m->fbb_size[a], upsample);
    return FHASH_OK;
}

fhash_status fhash_decode(fhash_model* m, float t_norm, int32_t upsample, float* out, fhash_stream stream) {
    FH_RANGE("fhash_decode");
    if (!m || !out || upsample < 1 || upsample > 8 || !(t_norm >= 0.0f && t_norm <= 1.0f))
        return set_error(FHASH_EINVAL, "fhash_decode: bad arguments (upsample 1..8, t_norm in [0,1])");
    if (!is_device_ptr(out)) return set_error(FHASH_EINVAL, "fhash_decode: out must be device memory");
    int64_t d[3];
    for (int a = 0; a < 3; ++a) d[a] = decode_points(m->fbb_size[a], upsample);
    if (d[0] * d[1] * d[2] >= (1ll << 40)) return set_error(FHASH_EINVAL, "fhash_decode: grid too large");
    cudaStream_t st = (cudaStream_t)stream;
    FH_TRY(settle_deferred(m, st));
    if (m->shadow) {  // precision form: coordinates in chunks, then the tensor-core forward
        const int64_t total = d[0] * d[1] * d[2], chunk = 1 << 23;
        FH_TRY(grow(m, m->s_misc, (size_t)chunk * 16));
        for (int64_t i0 = 0; i0 < total; i0 += chunk) {
            const int64_t cnt = std::min(chunk, total - i0);
            k_grid_coords<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>((int)d[0], (int)d[1], (int)d[2], t_norm, i0, cnt,
                                                                         (float4*)m->s_misc.p);
            FH_CUDA(cudaGetLastError());
            FH_TRY(launch_forward(m, (const float*)m->s_misc.p, cnt, out + i0, st));
        }
        return FHASH_OK;
    }
    cudaError_t e;
    switch (m->lv.F) {
        case 1: e = run_decode<1>(m, (int)d[0], (int)d[1], (int)d[2], t_norm, out, st); break;
        case 2: e = run_decode<2>(m, (int)d[0], (int)d[1], (int)d[2], t_norm, out, st); break;
        case 4: e = run_decode<4>(m, (int)d[0], (int)d[1], (int)d[2], t_norm, out, st); break;
        case 8: e = run_decode<8>(m, (int)d[0], (int)d[1], (int)d[2], t_norm, out, st); break;
        default: return set_error(FHASH_EINVAL, "fhash_decode: F=%d unsupported", m->lv.F);
    }
    FH_CUDA(e);
    return FHASH_OK;
}

fhash_status fhash_render(fhash_model* m, const fhash_camera* cam, float t_norm, const float* tf, int32_t w, int32_t h,
                          int32_t max_pace, float* rgba, int32_t* counts, fhash_render_stats* stats,
                          fhash_stream stream) {
    FH_RANGE("fhash_render");
    if (!m || !cam || !tf || !rgba || w < 1 || h < 1 || (int64_t)w * h > (1 << 26) || max_pace < 1 ||
        !(t_norm >= 0.0f && t_norm <= 1.0f))
        return set_error(FHASH_EINVAL, "fhash_render: bad arguments");
    if (!is_device_ptr(tf) || !is_device_ptr(rgba) || (counts && !is_device_ptr(counts)))
        return set_error(FHASH_EINVAL, "fhash_render: tf, rgba and counts must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    FH_TRY(settle_deferred(m, st));
    const RenderGeo g = make_geo(m, cam, t_norm, w, h);
    const int64_t NR = (int64_t)w * h;
    // scratch: ray states, two alive lists, sample coords and values, per-ray counts, counters
    const size_t o_rs = 0;
    const size_t o_al0 = (o_rs + NR * sizeof(RayState) + 255) / 256 * 256;
    const size_t o_al1 = (o_al0 + NR * 4 + 255) / 256 * 256;
    const size_t o_cnt = (o_al1 + NR * 4 + 255) / 256 * 256;
    const size_t o_co = (o_cnt + NR * 4 + 255) / 256 * 256;
    const size_t o_val = (o_co + NR * 16 + 255) / 256 * 256;
    const size_t o_ctr = (o_val + NR * 4 + 255) / 256 * 256;
    const size_t total = o_ctr + 64;
    FH_TRY(grow(m, m->s_render, total));
    char* b = (char*)m->s_render.p;
    RayState* rs = (RayState*)(b + o_rs);
    int* al[2] = {(int*)(b + o_al0), (int*)(b + o_al1)};
    int* cnt = (int*)(b + o_cnt);
    float4* co = (float4*)(b + o_co);
    float* val = (float*)(b + o_val);
    int* ctr = (int*)(b + o_ctr);                                     // [0], [1]: alive counters
    unsigned long long* acc = (unsigned long long*)(b + o_ctr + 16);  // marched, used
    FH_CUDA(cudaMemsetAsync(ctr, 0, 64, st));
    k_ray_init<<<(unsigned)((NR + 255) / 256), 256, 0, st>>>(g, rs, al[0], ctr, (float4*)rgba, counts);
    FH_CUDA(cudaGetLastError());
    int na = 0;
    FH_CUDA(cudaMemcpyAsync(&na, ctr, 4, cudaMemcpyDeviceToHost, st));
    FH_CUDA(cudaStreamSynchronize(st));
    int64_t rounds = 0, slots = 0;
    int cur = 0;
    while (na > 0) {
        if (rounds > (1 << 24)) return set_error(FHASH_ETIMEOUT, "fhash_render: round limit exceeded");
        int ns = (int)std::max<int64_t>(1, std::min<int64_t>(NR / na, max_pace));
        k_arm_generate<<<(na + 127) / 128, 128, 0, st>>>(g, rs, al[cur], na, ns, co, cnt, stats ? acc : nullptr);
        FH_CUDA(cudaGetLastError());
        const int64_t nslots = (int64_t)na * ns;
        FH_TRY(launch_forward(m, (const float*)co, nslots, val, st));
        FH_CUDA(cudaMemsetAsync(ctr + 1 - cur, 0, 4, st));
        k_arm_composite<<<(na + 127) / 128, 128, 0, st>>>(g, rs, al[cur], na, ns, cnt, val, (const float4*)tf,
                                                          al[1 - cur], ctr + 1 - cur, (float4*)rgba, counts,
                                                          stats ? acc + 1 : nullptr);
        FH_CUDA(cudaGetLastError());
        FH_CUDA(cudaMemcpyAsync(&na, ctr + 1 - cur, 4, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
        cur = 1 - cur;
        ++rounds;
        slots += nslots;
    }
    if (stats) {
        unsigned long long h2[2];
        FH_CUDA(cudaMemcpyAsync(h2, acc, 16, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
        stats->rounds = rounds;
        stats->samples_evaluated = slots;
        stats->samples_composited = (int64_t)h2[1];
        stats->steps_marched = (int64_t)h2[0];
    }
    return FHASH_OK;
}

}  // extern "C"
