// Feature-based coreset training (Section 3.1).
//
// The coreset is the union over key frames t_k of the dilated feature d_k: every vertex of d_k at t_k
// becomes a 4D sample (x, y, z, t_k) labelled with the volume value there.  The model's occupancy grid
// already holds d_k over the Feature Bounding Box (one bit per voxel, 8^3 Morton bricks), so building
// the coreset is a deterministic stream compaction of those bits over (key frame, z, y, x):
//   k_cs_count  per block of 256 voxels, the number of set bits;
//   (host)      exclusive scan of the block counts;
//   k_cs_write  per block, warp ballots give each set voxel its rank, which places it at
//               offset[block] + rank: samples keep key-frame, then (z, y, x) order.
// A sample is 12 bytes on the device: (x, y, z, t) packed as four 16-bit fields, and its float32 label.
//
// Epoch e visits every sample once, in the order of a keyed permutation of [0, N): a balanced 4-round
// Feistel network on k-bit integers (Luby and Rackoff) with SplitMix64 round functions, walked onto
// [0, N) by repeated application (cycle walking, Black and Rogaway 2002).  Batch b takes positions
// b*B .. b*B + B - 1; k_cs_batch writes their FBB-normalised coordinates and labels.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fh {

__device__ __forceinline__ int occ_bit(const uint32_t* __restrict__ words, int x, int y, int z, int nbx, int nby) {
    const int64_t b = ((int64_t)(z >> 3) * nby + (y >> 3)) * nbx + (x >> 3);
    const int lx = x & 7, ly = y & 7, lz = z & 7;
    int mi = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        mi |= (((lx >> k) & 1) << (3 * k)) | (((ly >> k) & 1) << (3 * k + 1)) | (((lz >> k) & 1) << (3 * k + 2));
    return (int)((words[b * 16 + (mi >> 5)] >> (mi & 31)) & 1u);
}

struct CsGrid {
    const uint32_t* occ;
    int64_t words_per_t;  // occupancy words of one time step
    const int32_t* keys;  // key frames (device)
    int sx, sy, sz, nbx, nby;
    int64_t total;        // key frames x FBB voxels
};

__device__ __forceinline__ int cs_voxel(const CsGrid& g, int64_t i, int& k, int& x, int& y, int& z) {
    if (i >= g.total) return 0;
    const int64_t per = (int64_t)g.sx * g.sy * g.sz;
    k = (int)(i / per);
    int64_t r = i - (int64_t)k * per;
    x = (int)(r % g.sx);
    r /= g.sx;
    y = (int)(r % g.sy);
    z = (int)(r / g.sy);
    return occ_bit(g.occ + (int64_t)g.keys[k] * g.words_per_t, x, y, z, g.nbx, g.nby);
}

__global__ void __launch_bounds__(256) k_cs_count(const CsGrid g, int* __restrict__ counts) {
    int k = 0, x = 0, y = 0, z = 0;
    const int bit = cs_voxel(g, blockIdx.x * 256LL + threadIdx.x, k, x, y, z);
    const int c = __syncthreads_count(bit);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void __launch_bounds__(256) k_cs_write(const CsGrid g, const int64_t* __restrict__ offsets,
                                                  const float* __restrict__ vol, int64_t nx, int64_t ny, int64_t nz,
                                                  int lox, int loy, int loz, uint64_t* __restrict__ ent,
                                                  float* __restrict__ val) {
    __shared__ int wsum[8];
    int k = 0, x = 0, y = 0, z = 0;
    const int bit = cs_voxel(g, blockIdx.x * 256LL + threadIdx.x, k, x, y, z);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, bit);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w) base += wsum[w];
    if (!bit) return;
    const int64_t pos = offsets[blockIdx.x] + base + __popc(bal & ((1u << lane) - 1u));
    const int64_t X = x + lox, Y = y + loy, Z = z + loz, T = g.keys[k];
    ent[pos] = (uint64_t)X | ((uint64_t)Y << 16) | ((uint64_t)Z << 32) | ((uint64_t)T << 48);
    val[pos] = vol[((T * nz + Z) * ny + Y) * nx + X];
}

struct Shuffle {
    uint64_t K[4];
    uint64_t N;
    int h;  // half width: the network permutes [0, 2^(2h))
};

__device__ __forceinline__ uint64_t feistel(const Shuffle& S, uint64_t v) {
    const uint64_t mask = (1ull << S.h) - 1ull;
    uint64_t L = v >> S.h, R = v & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint64_t nr = L ^ (sm_mix(R ^ S.K[r]) & mask);
        L = R;
        R = nr;
    }
    return (L << S.h) | R;
}

__global__ void __launch_bounds__(256) k_cs_batch(const uint64_t* __restrict__ ent, const float* __restrict__ val,
                                                  const Shuffle S, int64_t pos0, int64_t nb, int lox, int loy, int loz,
                                                  int sx, int sy, int sz, int nt, float* __restrict__ coords,
                                                  float* __restrict__ target, int* __restrict__ err) {
    const int64_t i = blockIdx.x * 256LL + threadIdx.x;
    if (i >= nb) return;
    // Cycle walking ends on the first value below N: the orbit of pos0 + i under the network returns to
    // it.  The iteration cap only guards against a broken network and reports through the error word.
    uint64_t j = feistel(S, (uint64_t)(pos0 + i));
    for (int it = 0; j >= S.N; ++it) {
        if (it >= (1 << 22)) {
            raise_error(err, 0x7C09);
            j = (uint64_t)(pos0 + i) % S.N;
            break;
        }
        j = feistel(S, j);
    }
    const uint64_t e = ent[j];
    const int X = (int)(e & 0xffff), Y = (int)((e >> 16) & 0xffff), Z = (int)((e >> 32) & 0xffff), T = (int)(e >> 48);
    float4 u;
    u.x = sx > 1 ? __fdiv_rn((float)(X - lox), (float)(sx - 1)) : 0.0f;
    u.y = sy > 1 ? __fdiv_rn((float)(Y - loy), (float)(sy - 1)) : 0.0f;
    u.z = sz > 1 ? __fdiv_rn((float)(Z - loz), (float)(sz - 1)) : 0.0f;
    u.w = nt > 1 ? __fdiv_rn((float)T, (float)(nt - 1)) : 0.0f;
    reinterpret_cast<float4*>(coords)[i] = u;
    target[i] = val[j];
}

static Shuffle make_shuffle(uint64_t seed, int64_t epoch, int64_t N) {
    Shuffle S{};
    int k = 2;
    while (k < 62 && (1ll << k) < N) ++k;
    k += k & 1;
    S.h = k / 2;
    S.N = (uint64_t)N;
    const uint64_t key = sm_at(sm_at(seed, 400), (uint64_t)epoch);
    for (int r = 0; r < 4; ++r) S.K[r] = sm_at(key, (uint64_t)r);
    return S;
}

fhash_status coreset_build(fhash_model* m, const float* volume, const int32_t* keys, int n_key, int64_t* count,
                           cudaStream_t st) {
    if (!volume || !keys || n_key <= 0) return set_error(FHASH_EINVAL, "fhash_coreset_build: need a volume and key frames");
    for (int i = 0; i < n_key; ++i)
        if (keys[i] < 0 || keys[i] >= m->nt || (i > 0 && keys[i] <= keys[i - 1]))
            return set_error(FHASH_EINVAL, "fhash_coreset_build: key frames must increase strictly within [0, %lld)",
                             (long long)m->nt);
    const int64_t nx = m->desc.nx, ny = m->desc.ny, nz = m->desc.nz;
    if (nx > 65535 || ny > 65535 || nz > 65535 || m->nt > 65535)
        return set_error(FHASH_EINVAL, "fhash_coreset_build: volume dimensions above 65535");
    const int64_t nvox = nx * ny * nz * m->nt;
    // the volume on the device for the duration of the call
    const float* dvol = volume;
    float* tmp_vol = nullptr;
    if (!is_device_ptr(volume)) {
        if (cudaMalloc((void**)&tmp_vol, (size_t)nvox * 4) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FHASH_ENOMEM, "fhash_coreset_build: no device memory for the volume");
        }
        cudaError_t e = cudaMemcpyAsync(tmp_vol, volume, (size_t)nvox * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cudaFree(tmp_vol);
            return set_error(FHASH_ECUDA, "fhash_coreset_build: %s", cudaGetErrorString(e));
        }
        dvol = tmp_vol;
    }
    fhash_status status = FHASH_OK;
    int32_t* dkeys = nullptr;
    int* counts = nullptr;
    int64_t* offsets = nullptr;
    CsGrid g{};
    g.occ = m->occ;
    g.words_per_t = m->nbx * m->nby * m->nbz * 16;
    g.sx = (int)m->fbb_size[0];
    g.sy = (int)m->fbb_size[1];
    g.sz = (int)m->fbb_size[2];
    g.nbx = (int)m->nbx;
    g.nby = (int)m->nby;
    g.total = (int64_t)n_key * g.sx * g.sy * g.sz;
    const int64_t blocks = (g.total + 255) / 256;
    std::vector<int> hc((size_t)blocks);
    std::vector<int64_t> ho((size_t)blocks);
    int64_t n = 0;
    auto fail = [&](fhash_status s) { status = s; };
    do {
        if (cudaMalloc((void**)&dkeys, (size_t)n_key * 4) != cudaSuccess || cudaMalloc((void**)&counts, (size_t)blocks * 4) != cudaSuccess ||
            cudaMalloc((void**)&offsets, (size_t)blocks * 8) != cudaSuccess) {
            cudaGetLastError();
            fail(set_error(FHASH_ENOMEM, "fhash_coreset_build: no device memory for the compaction"));
            break;
        }
        g.keys = dkeys;
        if (cudaMemcpyAsync(dkeys, keys, (size_t)n_key * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            fail(set_error(FHASH_ECUDA, "fhash_coreset_build: copy failed"));
            break;
        }
        k_cs_count<<<(unsigned)blocks, 256, 0, st>>>(g, counts);
        if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(hc.data(), counts, (size_t)blocks * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            fail(set_error(FHASH_ECUDA, "fhash_coreset_build: count failed"));
            break;
        }
        for (int64_t b = 0; b < blocks; ++b) {
            ho[(size_t)b] = n;
            n += hc[(size_t)b];
        }
        if ((status = grow(m, m->s_cs_ent, (size_t)std::max<int64_t>(n, 1) * 8)) != FHASH_OK) break;
        if ((status = grow(m, m->s_cs_val, (size_t)std::max<int64_t>(n, 1) * 4)) != FHASH_OK) break;
        if (cudaMemcpyAsync(offsets, ho.data(), (size_t)blocks * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            fail(set_error(FHASH_ECUDA, "fhash_coreset_build: copy failed"));
            break;
        }
        k_cs_write<<<(unsigned)blocks, 256, 0, st>>>(g, offsets, dvol, nx, ny, nz, (int)m->fbb_lo[0],
                                                     (int)m->fbb_lo[1], (int)m->fbb_lo[2], (uint64_t*)m->s_cs_ent.p,
                                                     (float*)m->s_cs_val.p);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
            fail(set_error(FHASH_ECUDA, "fhash_coreset_build: write failed"));
            break;
        }
    } while (false);
    cudaFree(dkeys);
    cudaFree(counts);
    cudaFree(offsets);
    if (tmp_vol) cudaFree(tmp_vol);
    if (status != FHASH_OK) {
        m->cs_n = 0;
        return status;
    }
    m->cs_n = n;
    if (count) *count = n;
    return FHASH_OK;
}

fhash_status coreset_batch(fhash_model* m, uint64_t seed, int64_t epoch, int64_t batch, int64_t B, float* coords,
                           float* target, int64_t* n_out, cudaStream_t st) {
    if (m->cs_n <= 0) return set_error(FHASH_EINVAL, "coreset: none built (fhash_coreset_build)");
    if (B <= 0 || batch < 0 || epoch < 0 || batch * B >= m->cs_n)
        return set_error(FHASH_EINVAL, "coreset: batch %lld of size %lld is past the %lld samples", (long long)batch,
                         (long long)B, (long long)m->cs_n);
    const int64_t pos0 = batch * B, nb = std::min(B, m->cs_n - pos0);
    const Shuffle S = make_shuffle(seed, epoch, m->cs_n);
    k_cs_batch<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
        (const uint64_t*)m->s_cs_ent.p, (const float*)m->s_cs_val.p, S, pos0, nb, (int)m->fbb_lo[0], (int)m->fbb_lo[1],
        (int)m->fbb_lo[2], (int)m->fbb_size[0], (int)m->fbb_size[1], (int)m->fbb_size[2], (int)m->nt, coords, target,
        m->err_word);
    FH_CUDA(cudaGetLastError());
    if (n_out) *n_out = nb;
    return FHASH_OK;
}

}  // namespace fh

using namespace fh;

extern "C" {

fhash_status fhash_coreset_build(fhash_model* m, const float* volume, const int32_t* key_frames, int32_t n_key,
                                 int64_t* count, fhash_stream stream) {
    FH_RANGE("fhash_coreset_build");
    if (!m) return set_error(FHASH_EINVAL, "fhash_coreset_build: null model");
    return coreset_build(m, volume, key_frames, n_key, count, (cudaStream_t)stream);
}

fhash_status fhash_coreset_batch(fhash_model* m, uint64_t seed, int64_t epoch, int64_t batch, int64_t batch_size,
                                 float* coords, float* target, int64_t* n_out, fhash_stream stream) {
    FH_RANGE("fhash_coreset_batch");
    if (!m || !coords || !target) return set_error(FHASH_EINVAL, "fhash_coreset_batch: null argument");
    if (!is_device_ptr(coords) || !is_device_ptr(target))
        return set_error(FHASH_EINVAL, "fhash_coreset_batch: buffers must be device memory");
    return coreset_batch(m, seed, epoch, batch, batch_size, coords, target, n_out, (cudaStream_t)stream);
}

fhash_status fhash_coreset_train_step(fhash_model* m, uint64_t seed, int64_t epoch, int64_t batch, int64_t batch_size,
                                      const fhash_adam* adam, double* loss, fhash_stream stream) {
    FH_RANGE("fhash_coreset_train_step");
    if (!m || !adam) return set_error(FHASH_EINVAL, "fhash_coreset_train_step: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t want = std::max<int64_t>(1, std::min(batch_size, m->cs_n));
    FH_TRY(grow(m, m->s_coords, (size_t)want * 16));
    FH_TRY(grow(m, m->s_target, (size_t)want * 4));
    int64_t n = 0;
    FH_TRY(coreset_batch(m, seed, epoch, batch, batch_size, (float*)m->s_coords.p, (float*)m->s_target.p, &n, st));
    return fhash_train_step(m, (const float*)m->s_coords.p, (const float*)m->s_target.p, n, adam, loss, stream);
}

}  // extern "C"
