// fhash_compute_grads_noalloc: the gradient pass with its working memory in a fixed file-scope device
// array instead of buffers grown with cudaMalloc (for callers that cannot allocate device memory).
#include <mutex>

#include "kernels.cuh"

namespace fh {

cudaError_t run_fused_any(int F, int which, const FusedArgs& a);
__global__ void k_dw_partial(const float* __restrict__ a, const float* __restrict__ d, int fi, int fo, int64_t n,
                             int64_t chunk, float* __restrict__ partial);
__global__ void k_dw_reduce(const float* __restrict__ partial, int nchunk, int ne, float* __restrict__ grad);
__global__ void k_loss(const double* __restrict__ partial, int nb, int64_t n, double* __restrict__ loss);

// Held by every GPU that loads the library, until exit.  In host code this name is only a host-side
// stand-in: kernels must be given the device address obtained from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FHASH_NOALLOC_SCRATCH_BYTES];

static constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kMaxDevices];

// Device address of the scratch array on the current device, looked up once per device.
static fhash_status noalloc_scratch(void** out) {
    int dev = 0;
    FH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(FHASH_EINVAL, "fhash_compute_grads_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return FHASH_OK;
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace fh

using namespace fh;

extern "C" fhash_status fhash_compute_grads_noalloc(fhash_model* m, const float* coords, const float* target, int64_t n,
                                                    double* loss, fhash_stream stream) {
    FH_RANGE("fhash_compute_grads_noalloc");
    if (!m) return set_error(FHASH_EINVAL, "fhash_compute_grads_noalloc: null model");
    if (m->desc.layout == FHASH_LAYOUT_MASKED)
        return set_error(FHASH_EINVAL, "fhash_compute_grads_noalloc: FHASH_LAYOUT_MASKED models take fhash_compute_grads");
    if (n < 1 || n > FHASH_NOALLOC_MAX_SAMPLES || !coords || !target)
        return set_error(FHASH_EINVAL, "fhash_compute_grads_noalloc: need 1 <= n <= %d, coords and target",
                         FHASH_NOALLOC_MAX_SAMPLES);
    if (!is_device_ptr(coords) || !is_device_ptr(target))
        return set_error(FHASH_EINVAL, "fhash_compute_grads_noalloc: coords and target must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    FH_TRY(settle_deferred(m, st));  // a kernel launch over the model's own buffers: no allocation
    const MlpShape& sh = m->mlp;
    const int W = sh.width;
    const int64_t A = sh.in + (int64_t)sh.nh * W, D = (int64_t)sh.nh * W + 1;
    const int nb_loss = (int)std::max<int64_t>(1, std::min<int64_t>((n + TB - 1) / TB, (int64_t)num_sms() * 16));
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 2));
    const int64_t chunk = ((n + nchunk - 1) / nchunk + 31) / 32 * 32;
    int ne_max = 0;
    for (int j = 0; j <= sh.nh; ++j) {
        int fi = j == 0 ? sh.in : W, fo = j == sh.nh ? 1 : W;
        ne_max = std::max(ne_max, fo * fi + fo);
    }
    // carve the fixed array: activations, deltas, loss partials, loss, weight-gradient partials
    const size_t o_acts = 0;
    const size_t o_gacts = align256(o_acts + (size_t)(A * n) * 4);
    const size_t o_lpart = align256(o_gacts + (size_t)((D + 1) * n) * 4);
    const size_t o_loss = align256(o_lpart + (size_t)nb_loss * 8);
    const size_t o_wpart = align256(o_loss + 8);
    const size_t need = o_wpart + (size_t)nchunk * ne_max * 4;
    if (need > FHASH_NOALLOC_SCRATCH_BYTES)
        return set_error(FHASH_EINVAL, "fhash_compute_grads_noalloc: needs %zu scratch bytes for n=%lld, have %u", need,
                         (long long)n, (unsigned)FHASH_NOALLOC_SCRATCH_BYTES);
    void* base = nullptr;
    FH_TRY(noalloc_scratch(&base));
    char* b = (char*)base;
    float* acts = (float*)(b + o_acts);
    float* gy = (float*)(b + o_gacts);
    float* dl = gy + n;
    double* lpart = (double*)(b + o_lpart);
    double* lossd = (double*)(b + o_loss);
    float* wpart = (float*)(b + o_wpart);
    const bool dev_loss = loss && is_device_ptr(loss);

    FusedArgs a{};
    a.lv = &m->lv;
    a.sh = &m->mlp;
    a.T = m->param;
    a.G = m->grad;
    a.Pm = m->param + m->n_table;
    a.coords = coords;
    a.target = target;
    a.n = n;
    a.acts = acts;
    a.gy = gy;
    a.dl = dl;
    a.partial = lpart;
    a.grid = nb_loss;
    a.st = st;
    FH_CUDA(run_fused_any(m->lv.F, 1, a));
    k_loss<<<1, 256, 0, st>>>(lpart, nb_loss, n, dev_loss ? loss : lossd);
    FH_CUDA(cudaGetLastError());
    FH_CUDA(run_fused_any(m->lv.F, 2, a));
    float* gm = m->grad + m->n_table;
    for (int j = 0; j <= sh.nh; ++j) {
        int fi = j == 0 ? sh.in : W, fo = j == sh.nh ? 1 : W;
        const float* aj = (j == 0) ? acts : acts + (int64_t)(sh.in + (j - 1) * W) * n;
        const float* dj = dl + (int64_t)j * W * n;
        k_dw_partial<<<nchunk, 256, 0, st>>>(aj, dj, fi, fo, n, chunk, wpart);
        int ne = fo * fi + fo;
        k_dw_reduce<<<(ne + 255) / 256, 256, 0, st>>>(wpart, nchunk, ne, gm + sh.w_off[j]);
    }
    FH_CUDA(cudaGetLastError());
    if (loss && !dev_loss) {
        FH_CUDA(cudaMemcpyAsync(loss, lossd, 8, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
    }
    return FHASH_OK;
}
