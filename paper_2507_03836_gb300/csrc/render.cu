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

__global__ void k_ray_init(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs, int* __restrict__ alive,
                           int* __restrict__ n_alive, float4* __restrict__ rgba, int* __restrict__ counts) {
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix < g.W * g.H) ray_init_px(g, pix, rs, alive, n_alive, rgba, counts);
}

__global__ void k_arm_generate(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs,
                               const int* __restrict__ alive, int na, int ns, float4* __restrict__ coords,
                               int* __restrict__ cnt, unsigned long long* __restrict__ marched) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < na) arm_generate_ray(g, rs, alive[a], a, ns, coords, cnt, marched);
}

__global__ void k_arm_composite(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs,
                                const int* __restrict__ alive, int na, int ns, const int* __restrict__ cnt,
                                const float* __restrict__ vals, const float4* __restrict__ tf,
                                int* __restrict__ next, int* __restrict__ n_next, float4* __restrict__ rgba,
                                int* __restrict__ counts, unsigned long long* __restrict__ used) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < na) arm_composite_ray(g, rs, alive[a], a, ns, cnt, vals, tf, next, n_next, rgba, counts, used);
}

// The same round with its sizes read on the device, so that fhash_render issues rounds without waiting
// for the alive count: N_a = *n_alive, N_s = max(min(N_r / N_a, pace), 1) (Algorithm 1); thread 0
// publishes N_s and the round's sample count {0, N_a N_s} (the segment the persistent encode+MLP launch
// reads), clears the next list's counter and counts the round.  A round issued after the last ray left
// (N_a = 0) does nothing.
__global__ void k_arm_generate_dev(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs,
                                   const int* __restrict__ alive, const int* __restrict__ n_alive, int max_pace,
                                   int* __restrict__ ns_out, int64_t* __restrict__ seg, int* __restrict__ n_next,
                                   int* __restrict__ rounds, float4* __restrict__ coords, int* __restrict__ cnt,
                                   unsigned long long* __restrict__ acc) {
    const int na = *n_alive;
    const int64_t NR = (int64_t)g.W * g.H;
    const int ns = (int)max((int64_t)1, min(na > 0 ? NR / na : (int64_t)1, (int64_t)max_pace));
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a == 0) {
        *ns_out = ns;
        seg[0] = 0;
        seg[1] = (int64_t)na * ns;
        *n_next = 0;
        if (na > 0) {
            *rounds += 1;
            if (acc) acc[2] += (unsigned long long)na * ns;
        }
    }
    if (a < na) arm_generate_ray(g, rs, alive[a], a, ns, coords, cnt, acc);
}

__global__ void k_arm_composite_dev(const __grid_constant__ RenderGeo g, RayState* __restrict__ rs,
                                    const int* __restrict__ alive, const int* __restrict__ n_alive,
                                    const int* __restrict__ ns_in, const int* __restrict__ cnt,
                                    const float* __restrict__ vals, const float4* __restrict__ tf,
                                    int* __restrict__ next, int* __restrict__ n_next, float4* __restrict__ rgba,
                                    int* __restrict__ counts, unsigned long long* __restrict__ used) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < *n_alive) arm_composite_ray(g, rs, alive[a], a, *ns_in, cnt, vals, tf, next, n_next, rgba, counts, used);
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
    int* ctr = (int*)(b + o_ctr);  // [0], [1]: alive counters; [2]: the round's N_s; [3]: rounds with rays
    int64_t* seg = (int64_t*)(b + o_ctr + 16);                         // the round's {offset, count}
    unsigned long long* acc = (unsigned long long*)(b + o_ctr + 32);  // marched, used, evaluated
    FH_CUDA(cudaMemsetAsync(ctr, 0, 64, st));
    const unsigned gr = (unsigned)((NR + 127) / 128);
    k_ray_init<<<gr, 128, 0, st>>>(g, rs, al[0], ctr, (float4*)rgba, counts);
    FH_CUDA(cudaGetLastError());
    // Rounds are issued in batches of 1, 2, 4, ... 64 with no host wait inside a batch: every launch reads
    // the alive count from device memory.  After a batch the host reads the count once; a round issued
    // after the last ray has left does nothing.
    int cur = 0, na = 1;
    int64_t issued = 0;
    for (int batch = 1; na > 0; batch = std::min(2 * batch, 64)) {
        if (issued > (1 << 24)) return set_error(FHASH_ETIMEOUT, "fhash_render: round limit exceeded");
        for (int r = 0; r < batch; ++r) {
            k_arm_generate_dev<<<gr, 128, 0, st>>>(g, rs, al[cur], ctr + cur, max_pace, ctr + 2, seg, ctr + 1 - cur,
                                                   ctr + 3, co, cnt, stats ? acc : nullptr);
            FH_CUDA(cudaGetLastError());
            FH_TRY(launch_forward_seg(m, (const float*)co, val, seg, NR, st));
            k_arm_composite_dev<<<gr, 128, 0, st>>>(g, rs, al[cur], ctr + cur, ctr + 2, cnt, val, (const float4*)tf,
                                                    al[1 - cur], ctr + 1 - cur, (float4*)rgba, counts,
                                                    stats ? acc + 1 : nullptr);
            FH_CUDA(cudaGetLastError());
            cur = 1 - cur;
        }
        issued += batch;
        FH_CUDA(cudaMemcpyAsync(&na, ctr + cur, 4, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
    }
    if (stats) {
        unsigned long long h2[3];
        int hr[4];
        FH_CUDA(cudaMemcpyAsync(h2, acc, 24, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaMemcpyAsync(hr, ctr, 16, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
        stats->rounds = hr[3];
        stats->samples_evaluated = (int64_t)h2[2];
        stats->samples_composited = (int64_t)h2[1];
        stats->steps_marched = (int64_t)h2[0];
    }
    return FHASH_OK;
}

}  // extern "C"
