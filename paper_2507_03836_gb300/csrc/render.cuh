// Internal declarations of the renderer shared with the serving loop (not part of the C ABI).
#pragma once
#include "kernels.cuh"

namespace fh {

struct RenderGeo {
    float eye[3], right[3], up[3], fwd[3];
    float delta;      // sample spacing in world units
    float t_norm;
    int W, H;
    int S[3];         // FBB vertices per axis
    int nt;
    int tp, tn;       // time steps whose occupancy is used
    int use_tn;       // 1 when t lies strictly between key frames
    int64_t nbx, nby, nbrick;
    const uint32_t* occ;
    const uint8_t* occ_any;
};

struct RayState {
    float d[3];
    float tmin, tmax;
    int k;       // next sample index
    int flags;   // 1 = exited
    float C[3], T;
    int count;   // composited samples
};

// ------------------------------------------------------------------ per-ray steps of Algorithm 1
// Device functions shared by fhash_render's kernels and the serving loop's packed kernels, so that a
// ray's samples and pixel are the same bits in both.
// Morton index of voxel (x, y, z) inside its 8^3 brick: bit 3k from x, 3k + 1 from y, 3k + 2 from z.
__device__ __forceinline__ int morton9(int lx, int ly, int lz) {
    return (lx & 1) | ((ly & 1) << 1) | ((lz & 1) << 2) | ((lx & 2) << 2) | ((ly & 2) << 3) | ((lz & 2) << 4) |
           ((lx & 4) << 4) | ((ly & 4) << 5) | ((lz & 4) << 6);
}

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

// Ray of pixel pix: direction, entry and exit of the box; appended to the alive list when it hits the
// box, else its pixel is written as (0, 0, 0, 0).
__device__ __forceinline__ void ray_init_px(const RenderGeo& g, int pix, RayState* __restrict__ rs, int* __restrict__ alive,
                                            int* __restrict__ n_alive, float4* __restrict__ rgba, int* __restrict__ counts) {
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

// Index of the last sample that surely still lies in the empty aligned block of 2^lg voxels per axis
// (lg = 3: an 8^3 occupancy brick; 2 and 1: its 4^3 and 2^3 Morton sub-blocks) holding voxel v, for a
// ray whose sample k is in it.  The block holds the samples whose nearest voxel is in [b, b + 2^lg - 1]
// on each axis, that is model coordinate q = u (S - 1) in [b - 0.5, b + 2^lg - 0.5); the ray parameter
// where q reaches that box's far faces, pulled in by 0.01 voxel (far more than the float32 rounding of
// q and of this bound, about 1e-4 voxel), limits the samples that can be skipped.  Samples never
// evaluated there are unoccupied, so the set of samples (and the image) is the same as stepping through
// them one by one.  Float32 throughout: the FP64 rate of this GPU is a small fraction of its FP32 rate.
__device__ __forceinline__ int empty_block_last_sample(const RenderGeo& g, const RayState& s, const int v[3], int k,
                                                       int lg) {
    float t_exit = 3.0e38f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float d = s.d[ax];
        if (d == 0.0f) continue;
        const int b0 = (v[ax] >> lg) << lg;
        const float qf = d > 0.0f ? (float)(b0 + (1 << lg) - 1) + 0.49f : (float)b0 - 0.49f;  // the far face
        const float uf = qf / (float)(g.S[ax] - 1);
        t_exit = fminf(t_exit, ((2.0f * uf - 1.0f) - g.eye[ax]) / d);  // u = (eye + t d + 1) / 2
    }
    const float kl = floorf((t_exit - s.tmin) / g.delta);
    return kl > (float)k ? (int)fminf(kl, (float)(1 << 24)) : k;
}

// Marches each alive ray on until it has up to Ns occupied samples (or leaves the box); writes their
// model coordinates to slots [a*Ns, a*Ns + cnt).  Empty-space skipping over an occupancy hierarchy at
// both time steps in use: an empty 8^3 brick (its "any" byte), else an empty 4^3 sub-block of the brick
// (64 consecutive Morton bits: two words), else an empty 2^3 sub-block (8 consecutive bits: one byte)
// jumps the ray to the last sample inside that block; otherwise the voxel's own bit decides.
__device__ __forceinline__ void arm_generate_ray(const RenderGeo& g, RayState* __restrict__ rs, int pix, int a, int ns,
                                                 float4* __restrict__ coords, int* __restrict__ cnt,
                                                 unsigned long long* __restrict__ marched) {
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
            k = empty_block_last_sample(g, s, v, k, 3) + 1;  // samples up to the returned one are empty
            continue;
        }
        const int mi = morton9(v[0] & 7, v[1] & 7, v[2] & 7);
        uint2 q = make_uint2(0u, 0u);  // the 4^3 sub-block's 64 bits at either time step
        if (any_p) {
            const uint2 w = __ldg(reinterpret_cast<const uint2*>(g.occ + ((int64_t)g.tp * g.nbrick + b) * 16) + (mi >> 6));
            q.x |= w.x; q.y |= w.y;
        }
        if (any_n) {
            const uint2 w = __ldg(reinterpret_cast<const uint2*>(g.occ + ((int64_t)g.tn * g.nbrick + b) * 16) + (mi >> 6));
            q.x |= w.x; q.y |= w.y;
        }
        if ((q.x | q.y) == 0u) {
            k = empty_block_last_sample(g, s, v, k, 2) + 1;
            continue;
        }
        const uint32_t byte = (((mi >> 5) & 1) ? q.y : q.x) >> (mi & 24) & 0xffu;  // the 2^3 sub-block
        if (byte == 0u) {
            k = empty_block_last_sample(g, s, v, k, 1) + 1;
            continue;
        }
        ++k;
        if ((byte >> (mi & 7)) & 1u) coords[(int64_t)a * ns + c++] = make_float4(u[0], u[1], u[2], g.t_norm);
    }
    rs[pix].k = k;
    rs[pix].flags = s.flags;
    cnt[a] = c;
    if (marched) atomicAdd(marched, (unsigned long long)steps);
}

// Transfer function lookup (256 RGBA entries, linear interpolation) and front-to-back compositing;
// rays that are done write their pixel, the others are appended to the next alive list.
__device__ __forceinline__ void arm_composite_ray(const RenderGeo& g, RayState* __restrict__ rs, int pix, int a, int ns,
                                                  const int* __restrict__ cnt, const float* __restrict__ vals,
                                                  const float4* __restrict__ tf, int* __restrict__ next,
                                                  int* __restrict__ n_next, float4* __restrict__ rgba,
                                                  int* __restrict__ counts, unsigned long long* __restrict__ used) {
    RayState s = rs[pix];
    int c = cnt[a];
    bool opaque = false;
    int u = 0;
    for (int j = 0; j < c && !opaque; ++j) {
        float v = vals[(int64_t)a * ns + j];
        float x = __fmul_rn(fminf(fmaxf(v, 0.0f), 1.0f), 255.0f);
        int i0 = min((int)floorf(x), 254);
        float f = __fsub_rn(x, (float)i0);
        float4 p = __ldg(tf + i0), q = __ldg(tf + i0 + 1);
        float r = __fmaf_rn(f, __fsub_rn(q.x, p.x), p.x), gg = __fmaf_rn(f, __fsub_rn(q.y, p.y), p.y);
        float b = __fmaf_rn(f, __fsub_rn(q.z, p.z), p.z), al = __fmaf_rn(f, __fsub_rn(q.w, p.w), p.w);
        float w = __fmul_rn(s.T, al);
        s.C[0] = __fmaf_rn(w, r, s.C[0]); s.C[1] = __fmaf_rn(w, gg, s.C[1]); s.C[2] = __fmaf_rn(w, b, s.C[2]);
        s.T = __fmul_rn(s.T, __fsub_rn(1.0f, al));
        ++u;
        if (__fsub_rn(1.0f, s.T) > 0.99f) opaque = true;
    }
    s.count += u;
    if (used) atomicAdd(used, (unsigned long long)u);
    if (opaque || (s.flags & 1)) {
        rgba[pix] = make_float4(s.C[0], s.C[1], s.C[2], __fsub_rn(1.0f, s.T));
        if (counts) counts[pix] = s.count;
        rs[pix].flags = s.flags | 2;
    } else {
        next[atomicAdd(n_next, 1)] = pix;
    }
    rs[pix].C[0] = s.C[0]; rs[pix].C[1] = s.C[1]; rs[pix].C[2] = s.C[2];
    rs[pix].T = s.T;
    rs[pix].count = s.count;
}

// Host: geometry of one render of model m (camera, time, image size) - the same float32 steps as the
// sample test on the device.
RenderGeo make_geo(const fhash_model* m, const fhash_camera* cam, float t_norm, int w, int h);

__global__ void k_ray_init(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs, int* __restrict__ alive,
                           int* __restrict__ n_alive, float4* __restrict__ rgba, int* __restrict__ counts);
__global__ void k_arm_generate(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs,
                               const int* __restrict__ alive, int na, int ns, float4* __restrict__ coords,
                               int* __restrict__ cnt, unsigned long long* __restrict__ marched);
__global__ void k_arm_composite(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs,
                                const int* __restrict__ alive, int na, int ns, const int* __restrict__ cnt,
                                const float* __restrict__ vals, const float4* __restrict__ tf,
                                int* __restrict__ next, int* __restrict__ n_next, float4* __restrict__ rgba,
                                int* __restrict__ counts, unsigned long long* __restrict__ used);
__global__ void k_grid_coords(int nx, int ny, int nz, float t_norm, int64_t i0, int64_t cnt, float4* __restrict__ co);
int64_t decode_points(int64_t S, int up);

}  // namespace fh
