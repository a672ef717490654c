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
