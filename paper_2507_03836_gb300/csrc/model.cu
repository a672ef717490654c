// Model construction and state access: feature dilation, Feature Bounding Box, occupancy grid
// (Section 3.1), level schedule and table sizing (Section 3.2.1-3.2.3), parameter initialisation
// (Section 3.2.4), and the C-ABI entry points that move state in and out of the model.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>

#include "common.cuh"

namespace fh {

static thread_local std::string g_err;

fhash_status set_error(fhash_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

fhash_status cuda_error(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(FHASH_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(FHASH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static fhash_status dev_alloc(fhash_model* m, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(FHASH_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    m->device_bytes += bytes;
    return FHASH_OK;
}

fhash_status grow(fhash_model* m, Scratch& s, size_t bytes) {
    if (s.bytes >= bytes) return FHASH_OK;
    if (s.p) {
        FH_CUDA(cudaDeviceSynchronize());  // buffer may still be read by queued work
        cudaFree(s.p);
        m->device_bytes -= s.bytes;
        s.p = nullptr;
        s.bytes = 0;
    }
    size_t want = bytes + bytes / 4;
    FH_TRY(dev_alloc(m, &s.p, want));
    s.bytes = want;
    return FHASH_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

fhash_status stage_in(fhash_model* m, Scratch& s, const void* p, size_t bytes, cudaStream_t st, const void** dev) {
    if (bytes == 0 || is_device_ptr(p)) {
        *dev = p;
        return FHASH_OK;
    }
    FH_TRY(grow(m, s, bytes));
    FH_CUDA(cudaMemcpyAsync(s.p, p, bytes, cudaMemcpyHostToDevice, st));
    *dev = s.p;
    return FHASH_OK;
}

// ------------------------------------------------------------------ SplitMix64 uniforms (device + host)
// (float)(lo + (hi - lo) * U) with the multiply and the add rounded separately (no FMA contraction).
__host__ __device__ __forceinline__ float sm_uniform(uint64_t key, uint64_t i, double lo, double hi) {
    double u = (double)(sm_at(key, i) >> 40) * (1.0 / 16777216.0);
#ifdef __CUDA_ARCH__
    return (float)__dadd_rn(lo, __dmul_rn(hi - lo, u));
#else
    volatile double t = (hi - lo) * u;
    return (float)(lo + t);
#endif
}

__global__ void k_init_uniform(float* p, uint64_t n, uint64_t key, double lo, double hi) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = sm_uniform(key, i, lo, hi);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        q[i] = __float2bfloat16_rn(p[i]);
}

fhash_status refresh_shadow(fhash_model* m, uint64_t off, uint64_t n, cudaStream_t st) {
    if (!m->shadow || n == 0) return FHASH_OK;
    k_to_bf16<<<num_sms() * 8, 256, 0, st>>>(m->param + off, m->shadow + off, n);
    FH_CUDA(cudaGetLastError());
    return FHASH_OK;
}

// ------------------------------------------------------------------ feature dilation + boxes
// d(v) = OR of f over the 3x3x3 spatial neighbourhood of v, clipped at the border (Section 3.1); with
// merge, d(v) |= that instead (the union of several features' dilated regions, whose occupancy grids
// Section 3.1 merges for rendering).  Also folds the per-frame bounding box of this feature's dilated
// region into box[6] = (minx, miny, minz, maxx, maxy, maxz).
__global__ void k_dilate(const uint8_t* __restrict__ f, uint8_t* __restrict__ d, int nx, int ny, int nz, int* box,
                         int merge) {
    __shared__ int sb[6];
    if (threadIdx.x < 6) sb[threadIdx.x] = (threadIdx.x < 3) ? INT32_MAX : -1;
    __syncthreads();
    int64_t n3 = (int64_t)nx * ny * nz;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n3) {
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        uint8_t v = 0;
        for (int dz = -1; dz <= 1 && !v; ++dz) {
            int zz = z + dz;
            if (zz < 0 || zz >= nz) continue;
            for (int dy = -1; dy <= 1 && !v; ++dy) {
                int yy = y + dy;
                if (yy < 0 || yy >= ny) continue;
                const uint8_t* row = f + ((int64_t)zz * ny + yy) * nx;
                for (int dx = -1; dx <= 1; ++dx) {
                    int xx = x + dx;
                    if (xx >= 0 && xx < nx && row[xx]) { v = 1; break; }
                }
            }
        }
        d[i] = merge ? (uint8_t)(d[i] | v) : v;
        if (v) {
            atomicMin(&sb[0], x); atomicMin(&sb[1], y); atomicMin(&sb[2], z);
            atomicMax(&sb[3], x); atomicMax(&sb[4], y); atomicMax(&sb[5], z);
        }
    }
    __syncthreads();
    if (threadIdx.x < 3 && sb[threadIdx.x] != INT32_MAX) atomicMin(&box[threadIdx.x], sb[threadIdx.x]);
    if (threadIdx.x >= 3 && threadIdx.x < 6 && sb[threadIdx.x] >= 0) atomicMax(&box[threadIdx.x], sb[threadIdx.x]);
}

// Morton index inside an 8^3 brick: bit 3k+0 from x, 3k+1 from y, 3k+2 from z.
__host__ __device__ __forceinline__ void morton_decode(int mi, int& x, int& y, int& z) {
    x = (mi & 1) | ((mi >> 2) & 2) | ((mi >> 4) & 4);
    y = ((mi >> 1) & 1) | ((mi >> 3) & 2) | ((mi >> 5) & 4);
    z = ((mi >> 2) & 1) | ((mi >> 4) & 2) | ((mi >> 6) & 4);
}

// One block (512 threads) per brick of one time step: 16 ballots -> 16 words, plus the any-bit.
__global__ void k_occupancy(const uint8_t* __restrict__ d, int nx, int ny, int lx, int ly, int lz, int sx, int sy,
                            int sz, int nbx, int nby, uint32_t* __restrict__ words, uint8_t* __restrict__ any) {
    int b = blockIdx.x;
    int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    int mi = threadIdx.x, x, y, z;
    morton_decode(mi, x, y, z);
    x += bx * 8; y += by * 8; z += bz * 8;
    int v = 0;
    if (x < sx && y < sy && z < sz) v = d[((int64_t)(lz + z) * ny + (ly + y)) * nx + (lx + x)] != 0;
    unsigned word = __ballot_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) words[(int64_t)b * 16 + (threadIdx.x >> 5)] = word;
    int a = __syncthreads_or(v);
    if (threadIdx.x == 0) any[b] = (uint8_t)a;
}

__global__ void k_occ_read(const uint32_t* __restrict__ words, int sx, int sy, int sz, int nbx, int nby,
                           uint8_t* __restrict__ out) {
    int64_t n = (int64_t)sx * sy * sz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(i % sx), y = (int)((i / sx) % sy), z = (int)(i / ((int64_t)sx * sy));
        int b = ((z >> 3) * nby + (y >> 3)) * nbx + (x >> 3);
        int lx = x & 7, ly = y & 7, lz = z & 7, mi = 0;
        for (int k = 0; k < 3; ++k) mi |= (((lx >> k) & 1) << (3 * k)) | (((ly >> k) & 1) << (3 * k + 1)) | (((lz >> k) & 1) << (3 * k + 2));
        out[i] = (uint8_t)((words[(int64_t)b * 16 + (mi >> 5)] >> (mi & 31)) & 1u);
    }
}

// ------------------------------------------------------------------ masked compact tables
// FHASH_LAYOUT_MASKED keeps table rows only for the vertices near the features (the irregular grids
// of Section 3.1's feature-only coreset).  The active vertices of a level are the corners of the cells
// that the float32 cell step assigns to the footprint of some dilated-feature voxel.  Footprint and
// cells are products over the axes, so the active grid is the dilated mask over the FBB resampled
// axis by axis with OR over the voxels whose footprint reaches each vertex.

// The dilated mask over the Feature Bounding Box, [nt][sz][sy][sx] bytes 0/1.
__global__ void k_fbb_copy(const uint8_t* __restrict__ dil, int64_t nx, int64_t ny, int64_t nz, int64_t lx,
                           int64_t ly, int64_t lz, int64_t sx, int64_t sy, int64_t sz, int64_t nt,
                           uint8_t* __restrict__ out) {
    const int64_t n = sx * sy * sz * nt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = e % sx, y = (e / sx) % sy, z = (e / (sx * sy)) % sz, t = e / (sx * sy * sz);
        out[e] = dil[((t * nz + lz + z) * ny + ly + y) * nx + lx + x] != 0 ? 1 : 0;
    }
}

// out[o][X][i] = OR of in[o][v][i] over the voxels v in range[X] (one axis of the active grid);
// range[X] lies inside [0, S) or is empty (x > y).
__global__ void k_or_resample(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int64_t n_outer, int S,
                              int R, int64_t n_inner, const int2* __restrict__ range) {
    const int64_t n = n_outer * R * n_inner;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n_inner, q = e / n_inner;
        const int X = (int)(q % R);
        const int64_t o = q / R;
        const int2 ab = range[X];
        const uint8_t* p = in + o * S * n_inner + i;
        uint8_t a = 0;
        for (int v = ab.x; v <= ab.y && !a; ++v) a = p[(int64_t)v * n_inner];
        out[e] = a ? 1 : 0;
    }
}

// Bit i of 64-bit word w = grid[64 w + i] (0 past n), one 32-bit ballot per warp.  The loop bound is a
// multiple of 32, so the lanes of a warp stay in the loop together.
__global__ void k_pack_active(const uint8_t* __restrict__ grid, uint64_t n, uint64_t nwords, uint32_t* __restrict__ bits) {
    const uint64_t total = nwords * 64;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < total; r += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned b = __ballot_sync(0xffffffffu, r < n && grid[r] != 0);
        if ((threadIdx.x & 31) == 0) bits[r >> 5] = b;
    }
}

static int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Active vertices [lo, hi] of a level axis with R vertices for voxel v of the S voxels of the FBB on a
// spatial axis (footprint u*(S-1) in [v - 1/2, v + 1/2]) or for step v of S on the time axis
// (t*(S-1) in [v - 1, v + 1]); in level units p = u*(R-1), widened by 1/64, cells
// clamp(floor(p), 0, R-2), vertices up to the last cell + 1.  Exact integer arithmetic.
static void active_range(int64_t v, int64_t S, int64_t R, bool time, int64_t& lo, int64_t& hi) {
    if (R == 1) { lo = hi = 0; return; }
    if (S == 1) { lo = 0; hi = R - 1; return; }
    const int64_t den = 64 * (S - 1);
    const int64_t nlo = time ? (v - 1) * (R - 1) * 64 - (S - 1) : (2 * v - 1) * (R - 1) * 32 - (S - 1);
    const int64_t nhi = time ? (v + 1) * (R - 1) * 64 + (S - 1) : (2 * v + 1) * (R - 1) * 32 + (S - 1);
    lo = std::min(std::max(floor_div(nlo, den), (int64_t)0), R - 2);
    hi = std::min(std::max(floor_div(nhi, den), (int64_t)0), R - 2) + 1;
}

// For every vertex X of an axis, the voxels whose active range holds X.  Both ends of the range grow
// with v, so these voxels form an interval; an empty one is (1, 0).
static std::vector<int2> inverse_ranges(int64_t S, int64_t R, bool time) {
    std::vector<int2> r((size_t)R, make_int2(INT32_MAX, -1));
    for (int64_t v = 0; v < S; ++v) {
        int64_t lo, hi;
        active_range(v, S, R, time, lo, hi);
        for (int64_t X = lo; X <= hi; ++X) {
            r[X].x = std::min<int>(r[X].x, (int)v);
            r[X].y = std::max<int>(r[X].y, (int)v);
        }
    }
    for (auto& e : r)
        if (e.y < 0) e = make_int2(1, 0);
    return r;
}

static uint64_t level_dense_rows(const Level& v) { return v.st * (uint64_t)v.R[3]; }

// Points each masked level at its directory inside m->dir (records of the levels back to back).
static void link_dirs(fhash_model* m) {
    uint64_t off = 0;
    for (int l = 0; l < m->lv.L; ++l) {
        Level& v = m->lv.lv[l];
        v.dir = m->dir ? m->dir + off : nullptr;
        off += (level_dense_rows(v) + 63) / 64;
    }
}

struct DevTmp {
    void* p = nullptr;
    ~DevTmp() { if (p) cudaFree(p); }
};

// Builds the active-vertex directories and the compact bases (levels' R, sy, sz, st already set).
// dil: the dilated mask of the whole volume on the device, or null (no mask: every vertex active).
static fhash_status build_masked(fhash_model* m, const uint8_t* dil, cudaStream_t st) {
    const int L = m->lv.L;
    const int64_t sx = m->fbb_size[0], sy = m->fbb_size[1], sz = m->fbb_size[2], T = m->nt;
    uint64_t words = 0, max_words = 0;
    size_t cap = 1;
    int64_t max_axis = 1;
    for (int l = 0; l < L; ++l) {
        const Level& v = m->lv.lv[l];
        const int64_t Rx = v.R[0], Ry = v.R[1], Rz = v.R[2], Rt = v.R[3];
        const uint64_t nw = (level_dense_rows(v) + 63) / 64;
        words += nw;
        max_words = std::max(max_words, nw);
        cap = std::max<size_t>(cap, (size_t)std::max({T * sz * sy * Rx, T * sz * Ry * Rx, T * Rz * Ry * Rx, Rt * Rz * Ry * Rx}));
        max_axis = std::max({max_axis, Rx, Ry, Rz, Rt});
    }
    m->dir_words = words;
    FH_TRY(dev_alloc(m, (void**)&m->dir, (size_t)words * sizeof(uint4)));
    link_dirs(m);
    DevTmp fbb, P, Q, bits, rng;
    if (dil) {
        FH_CUDA(cudaMalloc(&fbb.p, (size_t)(sx * sy * sz * T)));
        k_fbb_copy<<<num_sms() * 8, 256, 0, st>>>(dil, m->desc.nx, m->desc.ny, m->desc.nz, m->fbb_lo[0], m->fbb_lo[1],
                                                  m->fbb_lo[2], sx, sy, sz, T, (uint8_t*)fbb.p);
        FH_CUDA(cudaGetLastError());
        FH_CUDA(cudaMalloc(&P.p, cap));
    }
    FH_CUDA(cudaMalloc(&Q.p, cap));
    FH_CUDA(cudaMalloc(&bits.p, (size_t)max_words * 8));
    FH_CUDA(cudaMalloc(&rng.p, (size_t)max_axis * 4 * sizeof(int2)));
    std::vector<uint64_t> hb((size_t)max_words);
    std::vector<uint4> rec((size_t)max_words);
    const unsigned grid = (unsigned)(num_sms() * 8);
    uint64_t acc = 0;
    for (int l = 0; l < L; ++l) {
        Level& v = m->lv.lv[l];
        const int64_t Rx = v.R[0], Ry = v.R[1], Rz = v.R[2], Rt = v.R[3];
        const uint64_t n = level_dense_rows(v), nw = (n + 63) / 64;
        uint8_t* g = (uint8_t*)Q.p;
        if (dil) {
            std::vector<int2> ax[4] = {inverse_ranges(sx, Rx, false), inverse_ranges(sy, Ry, false),
                                       inverse_ranges(sz, Rz, false), inverse_ranges(T, Rt, true)};
            int2* dr = (int2*)rng.p;
            const int64_t off[4] = {0, max_axis, 2 * max_axis, 3 * max_axis};
            for (int a = 0; a < 4; ++a)
                FH_CUDA(cudaMemcpyAsync(dr + off[a], ax[a].data(), ax[a].size() * sizeof(int2), cudaMemcpyHostToDevice, st));
            uint8_t *A = (uint8_t*)fbb.p, *B = (uint8_t*)P.p, *C = (uint8_t*)Q.p;
            k_or_resample<<<grid, 256, 0, st>>>(A, B, T * sz * sy, (int)sx, (int)Rx, 1, dr + off[0]);
            k_or_resample<<<grid, 256, 0, st>>>(B, C, T * sz, (int)sy, (int)Ry, Rx, dr + off[1]);
            k_or_resample<<<grid, 256, 0, st>>>(C, B, T, (int)sz, (int)Rz, Ry * Rx, dr + off[2]);
            k_or_resample<<<grid, 256, 0, st>>>(B, C, 1, (int)T, (int)Rt, Rz * Ry * Rx, dr + off[3]);
            FH_CUDA(cudaGetLastError());
        } else {
            FH_CUDA(cudaMemsetAsync(g, 1, (size_t)n, st));
        }
        k_pack_active<<<grid, 256, 0, st>>>(g, n, nw, (uint32_t*)bits.p);
        FH_CUDA(cudaGetLastError());
        FH_CUDA(cudaMemcpyAsync(hb.data(), bits.p, (size_t)nw * 8, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));  // also retires the range uploads before ax goes away
        uint64_t cnt = 0;
        for (uint64_t w = 0; w < nw; ++w) {
            rec[w] = make_uint4((uint32_t)hb[w], (uint32_t)(hb[w] >> 32), (uint32_t)cnt, (uint32_t)(cnt >> 32));
            cnt += (uint64_t)__builtin_popcountll(hb[w]);
        }
        FH_CUDA(cudaMemcpyAsync((void*)v.dir, rec.data(), (size_t)nw * sizeof(uint4), cudaMemcpyHostToDevice, st));
        FH_CUDA(cudaStreamSynchronize(st));
        v.base = acc;
        v.nrows = cnt;
        acc += cnt;
    }
    m->total_rows = acc;
    return FHASH_OK;
}

// ------------------------------------------------------------------ schedule (host)
static int ceil_log(int f, int64_t s) {
    int L = 0;
    int64_t p = 1;
    while (p < s) { p *= f; ++L; }
    return L;
}

static fhash_status make_schedule(const fhash_schedule& sc, const int64_t S[3], int64_t nt,
                                  std::vector<std::array<int64_t, 4>>& out) {
    out.clear();
    if (sc.mode == FHASH_SCHED_EXPLICIT) {
        if (sc.n_levels < 1 || sc.n_levels > FHASH_MAX_LEVELS) return set_error(FHASH_EINVAL, "explicit schedule: n_levels %d", sc.n_levels);
        for (int l = 0; l < sc.n_levels; ++l) out.push_back({sc.res[l][0], sc.res[l][1], sc.res[l][2], sc.res[l][3]});
    } else if (sc.mode == FHASH_SCHED_GEOMETRIC) {
        int L = sc.n_levels;
        if (L < 1 || L > FHASH_MAX_LEVELS) return set_error(FHASH_EINVAL, "geometric schedule: n_levels %d", L);
        for (int d = 0; d < 4; ++d)
            if (sc.r0[d] < 1 || sc.r1[d] < 1) return set_error(FHASH_EINVAL, "geometric schedule: r0/r1 must be >= 1");
        for (int l = 0; l < L; ++l) {
            std::array<int64_t, 4> r;
            for (int d = 0; d < 4; ++d)
                r[d] = (L == 1) ? sc.r1[d]
                                : (int64_t)floor(sc.r0[d] * pow((double)sc.r1[d] / sc.r0[d], (double)l / (L - 1)) + 0.5);
            out.push_back(r);
        }
    } else if (sc.mode == FHASH_SCHED_FOLD) {
        int f = sc.fold;
        if (f < 2) return set_error(FHASH_EINVAL, "fold must be >= 2");
        int Ld[3] = {ceil_log(f, S[0]), ceil_log(f, S[1]), ceil_log(f, S[2])};
        int L = (sc.levels_rule == FHASH_LEVELS_MIN) ? std::min(Ld[0], std::min(Ld[1], Ld[2]))
                                                     : std::max(Ld[0], std::max(Ld[1], Ld[2]));
        L = std::max(L, 1);
        if (L > FHASH_MAX_LEVELS) return set_error(FHASH_EINVAL, "fold schedule needs %d levels (max %d)", L, FHASH_MAX_LEVELS);
        std::vector<std::array<int64_t, 4>> fine;  // paper order: level 1 = native FBB resolution
        fine.push_back({S[0], S[1], S[2], nt});
        for (int l = 2; l <= L; ++l) {
            std::array<int64_t, 4> r = fine.back();
            for (int d = 0; d < 4; ++d) r[d] = (r[d] > f) ? (r[d] + f - 1) / f : 2;
            fine.push_back(r);
        }
        out.assign(fine.rbegin(), fine.rend());
    } else {
        return set_error(FHASH_EINVAL, "unknown schedule mode %d", sc.mode);
    }
    for (auto& r : out)
        for (int d = 0; d < 4; ++d)
            if (r[d] < 1 || r[d] > (1 << 24)) return set_error(FHASH_EINVAL, "level resolution %lld out of range", (long long)r[d]);
    return FHASH_OK;
}

static void destroy_model(fhash_model* m) {
    if (!m) return;
    cudaDeviceSynchronize();
    void* ps[] = {m->param, m->grad, m->adam_m, m->adam_v, m->shadow, m->occ, m->occ_any, m->dir, m->err_word,
                  m->s_coords.p, m->s_target.p, m->s_out.p, m->s_acts.p, m->s_gacts.p, m->s_partial.p,
                  m->s_loss.p, m->s_misc.p, m->s_render.p, m->s_enc.p, m->s_cs_ent.p, m->s_cs_val.p,
                  m->stamp, m->adam_tab, m->s_defer.p};
    for (void* p : ps)
        if (p) cudaFree(p);
    if (m->tev_init) {
        for (cudaEvent_t e : m->tev) cudaEventDestroy(e);
        for (cudaEvent_t e : m->tev_side) cudaEventDestroy(e);
    }
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    if (m->ev_join) cudaEventDestroy(m->ev_join);
    if (m->side) cudaStreamDestroy(m->side);
    delete m;
}

}  // namespace fh

using namespace fh;

extern "C" {

const char* fhash_last_error(void) { return g_err.c_str(); }

void fhash_destroy(fhash_model* m) { destroy_model(m); }

fhash_status fhash_build(const fhash_build_desc* d, fhash_stream stream, fhash_model** out) {
    FH_RANGE("fhash_build");
    if (!d || !out) return set_error(FHASH_EINVAL, "fhash_build: null argument");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (d->nx < 2 || d->ny < 2 || d->nz < 2 || d->nt < 1 || d->nx > (1 << 20) || d->ny > (1 << 20) || d->nz > (1 << 20))
        return set_error(FHASH_EINVAL, "volume dims must be >= 2 (space) and >= 1 (time)");
    if (d->F != 1 && d->F != 2 && d->F != 4 && d->F != 8) return set_error(FHASH_EINVAL, "F must be 1, 2, 4 or 8");
    if (d->dtype != FHASH_FP32 && d->dtype != FHASH_BF16) return set_error(FHASH_EINVAL, "dtype");
    if (d->mlp_hidden_layers < 1 || d->mlp_hidden_layers > FHASH_MAX_HIDDEN)
        return set_error(FHASH_EINVAL, "mlp_hidden_layers must be in 1..%d", FHASH_MAX_HIDDEN);
    if (d->mlp_width != 16 && d->mlp_width != 32 && d->mlp_width != 64)
        return set_error(FHASH_EINVAL, "mlp_width must be 16, 32 or 64");
    if (!(d->init_range >= 0.0f)) return set_error(FHASH_EINVAL, "init_range");
    if (d->layout != FHASH_LAYOUT_LINEAR && d->layout != FHASH_LAYOUT_BRICK && d->layout != FHASH_LAYOUT_MASKED)
        return set_error(FHASH_EINVAL, "layout must be FHASH_LAYOUT_LINEAR, _BRICK or _MASKED");
    if (d->layout == FHASH_LAYOUT_MASKED && d->dtype != FHASH_FP32)
        return set_error(FHASH_EINVAL, "FHASH_LAYOUT_MASKED takes dtype FHASH_FP32");
    const bool masked = d->layout == FHASH_LAYOUT_MASKED;
    if (d->n_masks < 0 || d->n_masks > 64 || (d->n_masks > 0 && (!d->masks || d->mask)))
        return set_error(FHASH_EINVAL, "n_masks must be 0..64; with n_masks > 0 give masks[] and leave mask NULL");
    for (int k = 0; k < d->n_masks; ++k)
        if (!d->masks[k]) return set_error(FHASH_EINVAL, "masks[%d] is NULL", k);
    const int n_feat = d->n_masks > 0 ? d->n_masks : (d->mask ? 1 : 0);

    fhash_model* m = new fhash_model();
    m->desc = *d;
    m->desc.mask = nullptr;
    m->desc.masks = nullptr;
    cudaGetDevice(&m->device);
    m->nt = d->nt;
    struct Guard {
        fhash_model*& m;
        ~Guard() { if (m) destroy_model(m); }
    } guard{m};

    FH_TRY(dev_alloc(m, (void**)&m->err_word, sizeof(int)));
    FH_CUDA(cudaMemsetAsync(m->err_word, 0, sizeof(int), st));

    // ---- feature dilation, per-frame boxes, FBB (Section 3.1)
    const int64_t nx = d->nx, ny = d->ny, nz = d->nz, nt = d->nt, n3 = nx * ny * nz;
    uint8_t* dil = nullptr;  // dilated mask, all frames (kept for the masked directories)
    struct DilGuard {
        uint8_t*& p;
        ~DilGuard() { if (p) cudaFree(p); }
    } dil_guard{dil};
    if (n_feat > 0) {
        uint8_t* stage = nullptr;
        int* boxes = nullptr;
        FH_CUDA(cudaMalloc(&stage, n3));
        cudaError_t e = cudaMalloc(&dil, (size_t)(n3 * nt));
        if (e != cudaSuccess) { dil = nullptr; cudaFree(stage); return cuda_error(e, "cudaMalloc(dilated mask)"); }
        e = cudaMalloc(&boxes, sizeof(int) * 6 * nt);
        if (e != cudaSuccess) { cudaFree(stage); return cuda_error(e, "cudaMalloc(boxes)"); }
        std::vector<int> hb(6 * nt);
        for (int64_t t = 0; t < nt; ++t) { hb[6 * t + 0] = hb[6 * t + 1] = hb[6 * t + 2] = INT32_MAX; hb[6 * t + 3] = hb[6 * t + 4] = hb[6 * t + 5] = -1; }
        cudaMemcpyAsync(boxes, hb.data(), sizeof(int) * 6 * nt, cudaMemcpyHostToDevice, st);
        for (int64_t t = 0; t < nt && e == cudaSuccess; ++t)
            for (int k = 0; k < n_feat && e == cudaSuccess; ++k) {  // each feature dilated, then OR-merged
                const uint8_t* src = d->n_masks > 0 ? d->masks[k] : d->mask;
                e = cudaMemcpyAsync(stage, src + t * n3, n3, cudaMemcpyHostToDevice, st);
                k_dilate<<<(unsigned)((n3 + 255) / 256), 256, 0, st>>>(stage, dil + t * n3, (int)nx, (int)ny, (int)nz,
                                                                      boxes + 6 * t, k > 0);
                if (e == cudaSuccess) e = cudaGetLastError();
            }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), boxes, sizeof(int) * 6 * nt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(stage);
        cudaFree(boxes);
        if (e != cudaSuccess) return cuda_error(e, "feature dilation");
        int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {-1, -1, -1};
        for (int64_t t = 0; t < nt; ++t) {
            if (hb[6 * t + 3] < 0) continue;  // empty frame
            for (int a = 0; a < 3; ++a) { lo[a] = std::min<int64_t>(lo[a], hb[6 * t + a]); hi[a] = std::max<int64_t>(hi[a], hb[6 * t + 3 + a]); }
        }
        if (hi[0] < 0) return set_error(FHASH_EINVAL, "feature mask is empty");
        for (int a = 0; a < 3; ++a) { m->fbb_lo[a] = lo[a]; m->fbb_size[a] = hi[a] - lo[a] + 1; }
    } else {
        m->fbb_lo[0] = m->fbb_lo[1] = m->fbb_lo[2] = 0;
        m->fbb_size[0] = nx; m->fbb_size[1] = ny; m->fbb_size[2] = nz;
    }

    // ---- occupancy bricks over the FBB, one set per time step
    const int64_t sx = m->fbb_size[0], sy = m->fbb_size[1], sz = m->fbb_size[2];
    m->nbx = (sx + 7) / 8; m->nby = (sy + 7) / 8; m->nbz = (sz + 7) / 8;
    const int64_t nbrick = m->nbx * m->nby * m->nbz;
    fhash_status s = dev_alloc(m, (void**)&m->occ, (size_t)(nbrick * 16 * 4 * nt));
    if (s == FHASH_OK) s = dev_alloc(m, (void**)&m->occ_any, (size_t)(nbrick * nt));
    if (s != FHASH_OK) return s;
    if (dil) {
        for (int64_t t = 0; t < nt; ++t)
            k_occupancy<<<(unsigned)nbrick, 512, 0, st>>>(dil + t * n3, (int)nx, (int)ny, (int)m->fbb_lo[0], (int)m->fbb_lo[1],
                                                          (int)m->fbb_lo[2], (int)sx, (int)sy, (int)sz, (int)m->nbx, (int)m->nby,
                                                          m->occ + t * nbrick * 16, m->occ_any + t * nbrick);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_error(e, "occupancy");
        if (!masked) { cudaFree(dil); dil = nullptr; }
    } else {
        // every voxel occupied; unused bits of partial bricks are never read
        FH_CUDA(cudaMemsetAsync(m->occ, 0xff, (size_t)(nbrick * 16 * 4 * nt), st));
        FH_CUDA(cudaMemsetAsync(m->occ_any, 1, (size_t)(nbrick * nt), st));
    }

    // ---- schedule and table sizing (Section 3.2.1-3.2.3)
    std::vector<std::array<int64_t, 4>> res;
    FH_TRY(make_schedule(d->sched, m->fbb_size, nt, res));
    const int L = (int)res.size();
    if (L * d->F > 64) return set_error(FHASH_EINVAL, "L*F = %d exceeds 64 (MLP input width)", L * d->F);
    m->lv.L = L;
    m->lv.F = d->F;
    uint64_t acc = 0;
    for (int l = 0; l < L; ++l) {
        Level& v = m->lv.lv[l];
        for (int a = 0; a < 4; ++a) { v.R[a] = (int32_t)res[l][a]; v.Rm1[a] = (float)(res[l][a] - 1); }
        uint64_t sxy = (uint64_t)res[l][0] * res[l][1];
        if (sxy >= (1ull << 32)) return set_error(FHASH_EINVAL, "level %d: Rx*Ry too large", l);
        v.sy = (uint32_t)res[l][0];
        v.sz = (uint32_t)sxy;
        uint64_t sxyz = sxy * res[l][2];
        if (sxyz >= (1ull << 32)) return set_error(FHASH_EINVAL, "level %d: Rx*Ry*Rz too large", l);
        v.st = sxyz;
        v.base = acc;
        v.nrows = sxyz * (uint64_t)res[l][3];
        v.dir = nullptr;
        v.layout = d->layout;
        acc += v.nrows;
    }
    m->total_rows = acc;
    if (masked) {
        FH_TRY(build_masked(m, dil, st));  // compact bases, row counts and directories
        if (dil) { cudaFree(dil); dil = nullptr; }
    }
    m->n_table = m->total_rows * (uint64_t)d->F;

    MlpShape& sh = m->mlp;
    sh.in = L * d->F;
    sh.width = d->mlp_width;
    sh.nh = d->mlp_hidden_layers;
    int off = 0;
    for (int k = 0; k <= sh.nh; ++k) {
        int fi = (k == 0) ? sh.in : sh.width, fo = (k == sh.nh) ? 1 : sh.width;
        sh.w_off[k] = off; off += fi * fo;
        sh.b_off[k] = off; off += fo;
    }
    sh.n_params = off;
    m->n_params = m->n_table + (uint64_t)off;

    // ---- state: param, grad, Adam m and v (+ bf16 shadow)
    const size_t bytes = (size_t)m->n_params * 4;
    FH_TRY(dev_alloc(m, (void**)&m->param, bytes));
    FH_TRY(dev_alloc(m, (void**)&m->grad, bytes));
    FH_TRY(dev_alloc(m, (void**)&m->adam_m, bytes));
    FH_TRY(dev_alloc(m, (void**)&m->adam_v, bytes));
    if (d->dtype == FHASH_BF16) FH_TRY(dev_alloc(m, (void**)&m->shadow, (size_t)m->n_params * 2));
    FH_CUDA(cudaMemsetAsync(m->grad, 0, bytes, st));
    FH_CUDA(cudaMemsetAsync(m->adam_m, 0, bytes, st));
    FH_CUDA(cudaMemsetAsync(m->adam_v, 0, bytes, st));

    // tables U(-r, r) from stream 200; MLP with nn.Linear bounds, streams 300+2k (W) / 301+2k (b)
    double r = d->init_range;
    k_init_uniform<<<num_sms() * 8, 256, 0, st>>>(m->param, m->n_table, sm_at(d->seed, 200), -r, r);
    FH_CUDA(cudaGetLastError());
    std::vector<float> hm(sh.n_params);
    for (int k = 0; k <= sh.nh; ++k) {
        int fi = (k == 0) ? sh.in : sh.width, fo = (k == sh.nh) ? 1 : sh.width;
        double bnd = 1.0 / sqrt((double)fi);
        uint64_t kw = sm_at(d->seed, 300 + 2 * k), kb = sm_at(d->seed, 301 + 2 * k);
        for (int i = 0; i < fi * fo; ++i) hm[sh.w_off[k] + i] = sm_uniform(kw, i, -bnd, bnd);
        for (int i = 0; i < fo; ++i) hm[sh.b_off[k] + i] = sm_uniform(kb, i, -bnd, bnd);
    }
    FH_CUDA(cudaMemcpyAsync(m->param + m->n_table, hm.data(), sizeof(float) * hm.size(), cudaMemcpyHostToDevice, st));
    FH_TRY(refresh_shadow(m, 0, m->n_params, st));
    FH_CUDA(cudaStreamSynchronize(st));

    *out = m;
    m = nullptr;  // release guard
    return FHASH_OK;
}

fhash_status fhash_active_range(int64_t v, int64_t S, int64_t R, int32_t is_time, int64_t* lo, int64_t* hi) {
    if (!lo || !hi) return set_error(FHASH_EINVAL, "fhash_active_range: null argument");
    if (S < 1 || S > (1 << 24) || R < 1 || R > (1 << 24) || v < 0 || v >= S)
        return set_error(FHASH_EINVAL, "fhash_active_range: need 0 <= v < S <= 2^24 and 1 <= R <= 2^24");
    active_range(v, S, R, is_time != 0, *lo, *hi);
    return FHASH_OK;
}

fhash_status fhash_plan(const fhash_schedule* sched, const int64_t fbb[3], int64_t nt, int32_t F, int32_t dtype,
                        int32_t nh, int32_t width, int32_t* n_levels, int32_t (*res)[4], uint64_t* table_rows,
                        uint64_t* n_params, uint64_t* state_bytes) {
    if (!sched || !fbb) return set_error(FHASH_EINVAL, "fhash_plan: null argument");
    for (int a = 0; a < 3; ++a)
        if (fbb[a] < 1 || fbb[a] > (1 << 20)) return set_error(FHASH_EINVAL, "fhash_plan: FBB size out of range");
    if (nt < 1) return set_error(FHASH_EINVAL, "fhash_plan: nt must be >= 1");
    if (F != 1 && F != 2 && F != 4 && F != 8) return set_error(FHASH_EINVAL, "F must be 1, 2, 4 or 8");
    if (dtype != FHASH_FP32 && dtype != FHASH_BF16) return set_error(FHASH_EINVAL, "dtype");
    if (nh < 1 || nh > FHASH_MAX_HIDDEN) return set_error(FHASH_EINVAL, "mlp_hidden_layers must be in 1..%d", FHASH_MAX_HIDDEN);
    if (width != 16 && width != 32 && width != 64) return set_error(FHASH_EINVAL, "mlp_width must be 16, 32 or 64");
    std::vector<std::array<int64_t, 4>> lv;
    FH_TRY(make_schedule(*sched, fbb, nt, lv));
    const int L = (int)lv.size();
    if (L * F > 64) return set_error(FHASH_EINVAL, "L*F = %d exceeds 64 (MLP input width)", L * F);
    uint64_t rows = 0;
    for (int l = 0; l < L; ++l) {
        const uint64_t sxy = (uint64_t)lv[l][0] * lv[l][1];
        if (sxy >= (1ull << 32)) return set_error(FHASH_EINVAL, "level %d: Rx*Ry too large", l);
        const uint64_t sxyz = sxy * lv[l][2];
        if (sxyz >= (1ull << 32)) return set_error(FHASH_EINVAL, "level %d: Rx*Ry*Rz too large", l);
        rows += sxyz * (uint64_t)lv[l][3];
        if (res)
            for (int a = 0; a < 4; ++a) res[l][a] = (int32_t)lv[l][a];
    }
    uint64_t mlp = 0;
    for (int k = 0; k <= nh; ++k) {
        const uint64_t fi = (k == 0) ? (uint64_t)(L * F) : (uint64_t)width, fo = (k == nh) ? 1 : (uint64_t)width;
        mlp += fi * fo + fo;
    }
    const uint64_t np = rows * (uint64_t)F + mlp;
    if (n_levels) *n_levels = L;
    if (table_rows) *table_rows = rows;
    if (n_params) *n_params = np;
    if (state_bytes) *state_bytes = np * 16 + (dtype == FHASH_BF16 ? np * 2 : 0);
    return FHASH_OK;
}

fhash_status fhash_get_info(const fhash_model* m, fhash_info* o) {
    if (!m || !o) return set_error(FHASH_EINVAL, "fhash_get_info: null argument");
    memset(o, 0, sizeof *o);
    o->n_levels = m->lv.L;
    o->F = m->lv.F;
    o->dtype = m->desc.dtype;
    o->n_mlp_layers = m->mlp.nh + 1;
    o->mlp_dims[0] = m->mlp.in;
    for (int k = 1; k <= m->mlp.nh; ++k) o->mlp_dims[k] = m->mlp.width;
    o->mlp_dims[m->mlp.nh + 1] = 1;
    for (int l = 0; l < m->lv.L; ++l) {
        for (int a = 0; a < 4; ++a) o->res[l][a] = m->lv.lv[l].R[a];
        o->base[l] = m->lv.lv[l].base;
    }
    o->total_rows = m->total_rows;
    o->n_table_params = m->n_table;
    o->n_mlp_params = (uint64_t)m->mlp.n_params;
    for (int a = 0; a < 3; ++a) { o->fbb_lo[a] = m->fbb_lo[a]; o->fbb_size[a] = m->fbb_size[a]; }
    o->nt = m->nt;
    o->step = m->step;
    o->device_bytes = m->device_bytes;
    return FHASH_OK;
}

static float* state_ptr(fhash_model* m, int which) {
    switch (which) {
        case FHASH_STATE_PARAM: return m->param;
        case FHASH_STATE_GRAD: return m->grad;
        case FHASH_STATE_ADAM_M: return m->adam_m;
        case FHASH_STATE_ADAM_V: return m->adam_v;
        default: return nullptr;
    }
}

fhash_status fhash_read_state(fhash_model* m, int32_t which, uint64_t off, uint64_t n, float* buf, fhash_stream stream) {
    if (!m || (!buf && n)) return set_error(FHASH_EINVAL, "fhash_read_state: null argument");
    float* p = state_ptr(m, which);
    if (!p) return set_error(FHASH_EINVAL, "fhash_read_state: unknown state %d", which);
    if (off > m->n_params || n > m->n_params - off) return set_error(FHASH_EINVAL, "fhash_read_state: range out of bounds");
    FH_TRY(settle_deferred(m, (cudaStream_t)stream));
    if (n) FH_CUDA(cudaMemcpyAsync(buf, p + off, n * 4, cudaMemcpyDefault, (cudaStream_t)stream));
    return FHASH_OK;
}

fhash_status fhash_write_state(fhash_model* m, int32_t which, uint64_t off, uint64_t n, const float* buf, fhash_stream stream) {
    if (!m || (!buf && n)) return set_error(FHASH_EINVAL, "fhash_write_state: null argument");
    float* p = state_ptr(m, which);
    if (!p) return set_error(FHASH_EINVAL, "fhash_write_state: unknown state %d", which);
    if (off > m->n_params || n > m->n_params - off) return set_error(FHASH_EINVAL, "fhash_write_state: range out of bounds");
    FH_TRY(settle_deferred(m, (cudaStream_t)stream));
    if (n) FH_CUDA(cudaMemcpyAsync(p + off, buf, n * 4, cudaMemcpyDefault, (cudaStream_t)stream));
    if (which == FHASH_STATE_PARAM) FH_TRY(refresh_shadow(m, off, n, (cudaStream_t)stream));
    return FHASH_OK;
}

fhash_status fhash_get_params(fhash_model* m, float* tables, float* mlp, fhash_stream stream) {
    if (!m) return set_error(FHASH_EINVAL, "fhash_get_params: null model");
    if (tables) FH_TRY(fhash_read_state(m, FHASH_STATE_PARAM, 0, m->n_table, tables, stream));
    if (mlp) FH_TRY(fhash_read_state(m, FHASH_STATE_PARAM, m->n_table, m->n_params - m->n_table, mlp, stream));
    if ((tables && !is_device_ptr(tables)) || (mlp && !is_device_ptr(mlp)))
        FH_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return FHASH_OK;
}

fhash_status fhash_set_params(fhash_model* m, const float* tables, const float* mlp, fhash_stream stream) {
    if (!m) return set_error(FHASH_EINVAL, "fhash_set_params: null model");
    if (tables) FH_TRY(fhash_write_state(m, FHASH_STATE_PARAM, 0, m->n_table, tables, stream));
    if (mlp) FH_TRY(fhash_write_state(m, FHASH_STATE_PARAM, m->n_table, m->n_params - m->n_table, mlp, stream));
    if ((tables && !is_device_ptr(tables)) || (mlp && !is_device_ptr(mlp)))
        FH_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return FHASH_OK;
}

fhash_status fhash_level_info(const fhash_model* m, int32_t* L, int32_t (*res)[4], uint64_t* base, int64_t fbb[6]) {
    if (!m) return set_error(FHASH_EINVAL, "fhash_level_info: null model");
    if (L) *L = m->lv.L;
    for (int l = 0; l < m->lv.L; ++l) {
        if (res)
            for (int d = 0; d < 4; ++d) res[l][d] = m->lv.lv[l].R[d];
        if (base) base[l] = m->lv.lv[l].base;
    }
    if (fbb)
        for (int d = 0; d < 3; ++d) {
            fbb[d] = m->fbb_lo[d];
            fbb[3 + d] = m->fbb_size[d];
        }
    return FHASH_OK;
}

fhash_status fhash_read_occupancy(fhash_model* m, int64_t t, uint8_t* out, fhash_stream stream) {
    if (!m || !out) return set_error(FHASH_EINVAL, "fhash_read_occupancy: null argument");
    if (t < 0 || t >= m->nt) return set_error(FHASH_EINVAL, "fhash_read_occupancy: t out of range");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = m->fbb_size[0] * m->fbb_size[1] * m->fbb_size[2];
    const int64_t nbrick = m->nbx * m->nby * m->nbz;
    uint8_t* dst = out;
    bool host = !is_device_ptr(out);
    if (host) { FH_TRY(grow(m, m->s_misc, n)); dst = (uint8_t*)m->s_misc.p; }
    k_occ_read<<<num_sms() * 8, 256, 0, st>>>(m->occ + t * nbrick * 16, (int)m->fbb_size[0], (int)m->fbb_size[1],
                                               (int)m->fbb_size[2], (int)m->nbx, (int)m->nby, dst);
    FH_CUDA(cudaGetLastError());
    if (host) {
        FH_CUDA(cudaMemcpyAsync(out, dst, n, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
    }
    return FHASH_OK;
}

fhash_status fhash_read_active(fhash_model* m, int32_t level, uint64_t word0, uint64_t n_words, uint64_t* bits,
                               fhash_stream stream) {
    if (!m || (!bits && n_words)) return set_error(FHASH_EINVAL, "fhash_read_active: null argument");
    if (m->desc.layout != FHASH_LAYOUT_MASKED || !m->dir)
        return set_error(FHASH_EINVAL, "fhash_read_active: the model does not use FHASH_LAYOUT_MASKED");
    if (level < 0 || level >= m->lv.L) return set_error(FHASH_EINVAL, "fhash_read_active: level out of range");
    const Level& v = m->lv.lv[level];
    const uint64_t nw = (level_dense_rows(v) + 63) / 64;
    if (word0 > nw || n_words > nw - word0) return set_error(FHASH_EINVAL, "fhash_read_active: words out of range");
    if (!n_words) return FHASH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // the low 8 bytes of each 16-byte record are the bits
    FH_CUDA(cudaMemcpy2DAsync(bits, 8, v.dir + word0, sizeof(uint4), 8, (size_t)n_words, cudaMemcpyDefault, st));
    if (!is_device_ptr(bits)) FH_CUDA(cudaStreamSynchronize(st));
    return FHASH_OK;
}

fhash_status fhash_check(fhash_model* m, fhash_stream stream) {
    if (!m) return set_error(FHASH_EINVAL, "fhash_check: null model");
    FH_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int w = 0;
    FH_CUDA(cudaMemcpy(&w, m->err_word, sizeof w, cudaMemcpyDeviceToHost));
    if (w) {
        FH_CUDA(cudaMemset(m->err_word, 0, sizeof(int)));
        return set_error(FHASH_EDEVICE, "device error word %d", w);
    }
    return FHASH_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ checkpoints
namespace fh {

struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    fhash_build_desc desc;
    Levels lv;
    MlpShape mlp;
    uint64_t total_rows, n_table, n_params;
    int64_t fbb_lo[3], fbb_size[3], nt, step, nbx, nby, nbz;
    uint64_t dir_words;  // masked layout: directory records after the occupancy grid
};
static const char kMagic[8] = {'F', 'H', 'A', 'S', 'H', 'C', 'K', '1'};

// Streams `bytes` between a device buffer and a file through a pinned host buffer.
static fhash_status stream_file(FILE* f, void* dev, uint64_t bytes, bool write, void* pin, size_t pin_bytes) {
    char* d = (char*)dev;
    for (uint64_t o = 0; o < bytes; o += pin_bytes) {
        const size_t k = (size_t)std::min<uint64_t>(pin_bytes, bytes - o);
        if (write) {
            FH_CUDA(cudaMemcpy(pin, d + o, k, cudaMemcpyDeviceToHost));
            if (fwrite(pin, 1, k, f) != k) return set_error(FHASH_EIO, "checkpoint write failed");
        } else {
            if (fread(pin, 1, k, f) != k) return set_error(FHASH_EIO, "checkpoint truncated");
            FH_CUDA(cudaMemcpy(d + o, pin, k, cudaMemcpyHostToDevice));
        }
    }
    return FHASH_OK;
}

}  // namespace fh

extern "C" {

fhash_status fhash_save(const fhash_model* mc, const char* path) {
    FH_RANGE("fhash_save");
    fhash_model* m = const_cast<fhash_model*>(mc);
    if (!m || !path) return set_error(FHASH_EINVAL, "fhash_save: null argument");
    FH_TRY(settle_deferred(m, 0));
    FH_CUDA(cudaDeviceSynchronize());
    FILE* f = fopen(path, "wb");
    if (!f) return set_error(FHASH_EIO, "fhash_save: cannot open %s", path);
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kMagic, 8);
    h.version = 3;  // 2: levels carry their row layout; 3: masked directories
    h.header_bytes = sizeof h;
    h.desc = m->desc;
    h.desc.mask = nullptr;
    h.lv = m->lv;
    h.mlp = m->mlp;
    h.total_rows = m->total_rows; h.n_table = m->n_table; h.n_params = m->n_params;
    for (int a = 0; a < 3; ++a) { h.fbb_lo[a] = m->fbb_lo[a]; h.fbb_size[a] = m->fbb_size[a]; }
    h.nt = m->nt; h.step = m->step; h.nbx = m->nbx; h.nby = m->nby; h.nbz = m->nbz;
    h.dir_words = m->dir ? m->dir_words : 0;
    for (int l = 0; l < h.lv.L; ++l) h.lv.lv[l].dir = nullptr;  // device addresses are not saved
    fhash_status rc = FHASH_OK;
    if (fwrite(&h, sizeof h, 1, f) != 1) rc = set_error(FHASH_EIO, "fhash_save: write failed");
    const size_t pin_bytes = 64u << 20;
    void* pin = nullptr;
    if (rc == FHASH_OK && cudaMallocHost(&pin, pin_bytes) != cudaSuccess) rc = set_error(FHASH_ENOMEM, "fhash_save: pinned buffer");
    const uint64_t nb = (uint64_t)(m->nbx * m->nby * m->nbz * m->nt);
    void* arrays[] = {m->param, m->grad, m->adam_m, m->adam_v, m->occ, m->occ_any, m->dir};
    const uint64_t sizes[] = {m->n_params * 4, m->n_params * 4, m->n_params * 4, m->n_params * 4, nb * 64, nb,
                              h.dir_words * sizeof(uint4)};
    for (int i = 0; i < 7 && rc == FHASH_OK; ++i)
        if (sizes[i]) rc = stream_file(f, arrays[i], sizes[i], true, pin, pin_bytes);
    if (pin) cudaFreeHost(pin);
    if (fclose(f) != 0 && rc == FHASH_OK) rc = set_error(FHASH_EIO, "fhash_save: close failed");
    return rc;
}

fhash_status fhash_load(const char* path, fhash_stream stream, fhash_model** out) {
    FH_RANGE("fhash_load");
    if (!path || !out) return set_error(FHASH_EINVAL, "fhash_load: null argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return set_error(FHASH_EIO, "fhash_load: cannot open %s", path);
    CkptHeader h;
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != 3 ||
        h.header_bytes != sizeof h || h.lv.L < 1 || h.lv.L > FHASH_MAX_LEVELS || h.n_params < h.n_table) {
        fclose(f);
        return set_error(FHASH_EIO, "fhash_load: %s is not an F-Hash checkpoint of this version", path);
    }
    fhash_model* m = new fhash_model();
    struct Guard {
        fhash_model*& m;
        FILE* f;
        ~Guard() { if (m) destroy_model(m); if (f) fclose(f); }
    } guard{m, f};
    cudaGetDevice(&m->device);
    m->desc = h.desc;
    m->lv = h.lv;
    m->mlp = h.mlp;
    m->total_rows = h.total_rows; m->n_table = h.n_table; m->n_params = h.n_params;
    for (int a = 0; a < 3; ++a) { m->fbb_lo[a] = h.fbb_lo[a]; m->fbb_size[a] = h.fbb_size[a]; }
    m->nt = h.nt; m->step = h.step; m->clean_step = h.step; m->nbx = h.nbx; m->nby = h.nby; m->nbz = h.nbz;
    const uint64_t nb = (uint64_t)(m->nbx * m->nby * m->nbz * m->nt);
    const size_t bytes = (size_t)m->n_params * 4;
    FH_TRY(dev_alloc(m, (void**)&m->err_word, sizeof(int)));
    FH_CUDA(cudaMemset(m->err_word, 0, sizeof(int)));
    FH_TRY(dev_alloc(m, (void**)&m->param, bytes));
    FH_TRY(dev_alloc(m, (void**)&m->grad, bytes));
    FH_TRY(dev_alloc(m, (void**)&m->adam_m, bytes));
    FH_TRY(dev_alloc(m, (void**)&m->adam_v, bytes));
    if (m->desc.dtype == FHASH_BF16) FH_TRY(dev_alloc(m, (void**)&m->shadow, (size_t)m->n_params * 2));
    FH_TRY(dev_alloc(m, (void**)&m->occ, (size_t)nb * 64));
    FH_TRY(dev_alloc(m, (void**)&m->occ_any, (size_t)nb));
    if (h.dir_words) {
        m->dir_words = h.dir_words;
        FH_TRY(dev_alloc(m, (void**)&m->dir, (size_t)h.dir_words * sizeof(uint4)));
    }
    link_dirs(m);
    const size_t pin_bytes = 64u << 20;
    void* pin = nullptr;
    if (cudaMallocHost(&pin, pin_bytes) != cudaSuccess) return set_error(FHASH_ENOMEM, "fhash_load: pinned buffer");
    void* arrays[] = {m->param, m->grad, m->adam_m, m->adam_v, m->occ, m->occ_any, m->dir};
    const uint64_t sizes[] = {bytes, bytes, bytes, bytes, nb * 64, nb, h.dir_words * sizeof(uint4)};
    fhash_status rc = FHASH_OK;
    for (int i = 0; i < 7 && rc == FHASH_OK; ++i)
        if (sizes[i]) rc = stream_file(f, arrays[i], sizes[i], false, pin, pin_bytes);
    cudaFreeHost(pin);
    if (rc != FHASH_OK) return rc;
    FH_TRY(refresh_shadow(m, 0, m->n_params, (cudaStream_t)stream));
    FH_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    *out = m;
    m = nullptr;
    return FHASH_OK;
}

}  // extern "C"
