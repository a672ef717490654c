// Diagnostics with no counterpart in the paper: the bounded-wait failure path of the tensor-core
// kernels (fhash_diag_wait_timeout) and the random-gather ceiling of the encoding's access pattern
// (fhash_diag_random_gather).
#include "kernels.cuh"
#include "tc.cuh"

namespace fh {
// One CTA waits on an mbarrier that nothing arrives on, with the same bounded wait the tensor-core
// kernels use; when the limit runs out it reports through the model's error word and returns.
__global__ void k_diag_wait(uint64_t limit_ns, int* __restrict__ err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit_ns)) raise_error(err, 0x7C07);
}
}  // namespace fh

extern "C" fhash_status fhash_diag_wait_timeout(fhash_model* m, uint64_t limit_ns, fhash_stream stream) {
    if (!m || limit_ns == 0 || limit_ns > 10000000000ull)
        return fh::set_error(FHASH_EINVAL, "fhash_diag_wait_timeout: limit must be in (0, 10 s]");
    fh::k_diag_wait<<<1, 32, 0, (cudaStream_t)stream>>>(limit_ns, m->err_word);
    FH_CUDA(cudaGetLastError());
    return FHASH_OK;
}

namespace fh {
// Random gathers of `width` bytes (4, 8 or 16) at uniformly drawn aligned positions of a device table,
// 8 independent loads in flight per thread; the per-block float sum goes to *sum so the loads cannot
// be removed.  Positions are SplitMix64 outputs modulo the slot count.
template <int W>
__global__ void __launch_bounds__(256) k_diag_gather(const uint8_t* __restrict__ table, uint64_t slots, int64_t n,
                                                     uint64_t seed, float* __restrict__ sum) {
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 8;
    for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 8; i0 < n; i0 += stride) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            v[u] = 0.0f;
            if (i0 + u < n) {
                const uint8_t* p = table + (sm_at(seed, (uint64_t)(i0 + u)) % slots) * W;
                if constexpr (W == 4) v[u] = __ldg(reinterpret_cast<const float*>(p));
                else if constexpr (W == 8) { const float2 q = __ldg(reinterpret_cast<const float2*>(p)); v[u] = q.x + q.y; }
                else { const float4 q = __ldg(reinterpret_cast<const float4*>(p)); v[u] = q.x + q.y + q.z + q.w; }
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    const double s = block_sum((double)acc);
    if (threadIdx.x == 0) atomicAdd(sum, (float)s);
}
}  // namespace fh

extern "C" fhash_status fhash_diag_random_gather(const void* table, uint64_t bytes, int32_t width, int64_t n,
                                                 uint64_t seed, float* sum, fhash_stream stream) {
    FH_RANGE("fhash_diag_random_gather");
    if (!table || !sum || n < 0 || (width != 4 && width != 8 && width != 16) || bytes < (uint64_t)width ||
        (reinterpret_cast<uintptr_t>(table) % 16) != 0 || !fh::is_device_ptr(table) || !fh::is_device_ptr(sum))
        return fh::set_error(FHASH_EINVAL, "fhash_diag_random_gather: bad arguments");
    if (n == 0) return FHASH_OK;
    const uint64_t slots = bytes / (uint64_t)width;
    const int grid = fh::num_sms() * 8;
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t* t = static_cast<const uint8_t*>(table);
    if (width == 4) fh::k_diag_gather<4><<<grid, 256, 0, st>>>(t, slots, n, seed, sum);
    else if (width == 8) fh::k_diag_gather<8><<<grid, 256, 0, st>>>(t, slots, n, seed, sum);
    else fh::k_diag_gather<16><<<grid, 256, 0, st>>>(t, slots, n, seed, sum);
    FH_CUDA(cudaGetLastError());
    return FHASH_OK;
}
