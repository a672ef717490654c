// Host glue and small kernels of the float32 path: encode / lookup launches, MLP weight gradients,
// loss reduction, and the C-ABI entry points for encode, forward and training (Adam: csrc/adam.cu).
#include <math.h>

#include <algorithm>

#include "kernels.cuh"

namespace fh {

// Encoding steps 1-3 (Section 3.2.4) for inspection: 16 corner rows (Eq. 9) and weights per sample-level.
__global__ void k_lookup(const __grid_constant__ Levels lv, const float* __restrict__ coords, int64_t n,
                         uint64_t* __restrict__ rows, float* __restrict__ w) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * lv.L) return;
    int64_t s = idx / lv.L;
    int l = (int)(idx % lv.L);
    Corners k = corners(lv.lv[l], load_coord(coords, s));
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        rows[idx * 16 + c] = corner_row(k, c);
        if (w) w[idx * 16 + c] = corner_weight(k, c);
    }
}
// Weight gradient of one layer over a chunk of samples: partial[chunk][e], e < fo*fi -> dW[o][i],
// e >= fo*fi -> db[o].  a: [fi][n] column-major activations, d: [fo][n] deltas.
__global__ void k_dw_partial(const float* __restrict__ a, const float* __restrict__ d, int fi, int fo, int64_t n,
                             int64_t chunk, float* __restrict__ partial) {
    constexpr int TS = 32;
    __shared__ float sa[64][TS + 1];
    __shared__ float sd[64][TS + 1];
    const int ne = fo * fi + fo;
    const int64_t n0 = blockIdx.x * chunk, n1 = min(n, n0 + chunk);
    float acc[17];
#pragma unroll
    for (int j = 0; j < 17; ++j) acc[j] = 0.0f;
    for (int64_t t0 = n0; t0 < n1; t0 += TS) {
        __syncthreads();
        for (int q = threadIdx.x; q < (fi + fo) * TS; q += blockDim.x) {
            int r = q / TS, c = q % TS;
            int64_t s = t0 + c;
            float v = 0.0f;
            if (s < n1) v = (r < fi) ? a[(int64_t)r * n + s] : d[(int64_t)(r - fi) * n + s];
            if (r < fi) sa[r][c] = v; else sd[r - fi][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 17; ++j) {
            int e = threadIdx.x + j * blockDim.x;
            if (e < ne) {
                float x = acc[j];
                if (e < fo * fi) {
                    int o = e / fi, i = e % fi;
#pragma unroll 8
                    for (int c = 0; c < TS; ++c) x = fmaf(sd[o][c], sa[i][c], x);
                } else {
                    int o = e - fo * fi;
#pragma unroll 8
                    for (int c = 0; c < TS; ++c) x += sd[o][c];
                }
                acc[j] = x;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 17; ++j) {
        int e = threadIdx.x + j * blockDim.x;
        if (e < ne) partial[(int64_t)blockIdx.x * ne + e] = acc[j];
    }
}

// grad[e] += sum over chunks of partial[c][e] (fixed order: deterministic).
__global__ void k_dw_reduce(const float* __restrict__ partial, int nchunk, int ne, float* __restrict__ grad) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    float s = 0.0f;
    for (int c = 0; c < nchunk; ++c) s += partial[(int64_t)c * ne + e];
    grad[e] += s;
}

// loss = (sum of per-block partial sums of squared residuals) / n, float64, fixed order.
__global__ void k_loss(const double* __restrict__ partial, int nb, int64_t n, double* __restrict__ loss) {
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

cudaError_t run_fused_any(int F, int which, const FusedArgs& a);
cudaError_t run_tc_any(fhash_model* m, bool train, FusedArgs& a);

static cudaError_t dispatch_fused(fhash_model* m, int which, FusedArgs& a) {
    a.lv = &m->lv;
    a.sh = &m->mlp;
    a.T = m->param;
    a.G = m->grad;
    a.Pm = m->param + m->n_table;
    int64_t blocks = (a.n + TB - 1) / TB;
    a.grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms() * 16));
    return run_fused_any(m->lv.F, which, a);
}

fhash_status launch_lookup(fhash_model* m, const float* coords, int64_t n, uint64_t* rows, float* w, cudaStream_t st) {
    int64_t tot = n * m->lv.L;
    k_lookup<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m->lv, coords, n, rows, w);
    FH_CUDA(cudaGetLastError());
    return FHASH_OK;
}

fhash_status launch_encode(fhash_model* m, const float* coords, int64_t n, float* enc, cudaStream_t st) {
    int64_t tot = n * m->lv.L;
    unsigned g = (unsigned)((tot + 255) / 256);
    switch (m->lv.F) {
        case 1: k_encode<1><<<g, 256, 0, st>>>(m->lv, m->param, coords, n, enc); break;
        case 2: k_encode<2><<<g, 256, 0, st>>>(m->lv, m->param, coords, n, enc); break;
        case 4: k_encode<4><<<g, 256, 0, st>>>(m->lv, m->param, coords, n, enc); break;
        case 8: k_encode<8><<<g, 256, 0, st>>>(m->lv, m->param, coords, n, enc); break;
        default: return set_error(FHASH_EINVAL, "F=%d has no kernel (supported: 1, 2, 4, 8)", m->lv.F);
    }
    FH_CUDA(cudaGetLastError());
    return FHASH_OK;
}

// FHASH_FORWARD_AUTO takes the fused kernel: measured on GB300 (4M uniform points), the fused kernel
// serves 1.53 G samples/s on advect-128^3x32 and 0.99 G on advect-256^3x64, the split pair 1.46 G and
// 0.84 G.  The gathers dominate both, and the split pair adds the encoding round trip.

fhash_status launch_forward(fhash_model* m, const float* coords, int64_t n, float* out, cudaStream_t st) {
    if (n <= 0) return FHASH_OK;
    FusedArgs a{};
    a.coords = coords;
    a.n = n;
    a.out = out;
    a.st = st;
    if (m->shadow) {  // precision form: bf16 tables, MLP on the tensor cores
        if (m->forward_path == FHASH_FORWARD_SPLIT) return launch_forward_split(m, coords, n, out, st);
        FH_CUDA(run_tc_any(m, false, a));
    } else {
        FH_CUDA(dispatch_fused(m, 0, a));
    }
    return FHASH_OK;
}

// Persistent forward over the segment {offset, count} held in device memory at `seg`: the grid does
// not depend on the count, so the launch can be captured once and replayed with new segments.
fhash_status launch_forward_seg(fhash_model* m, const float* coords, float* out, const int64_t* seg, int64_t max_n,
                                cudaStream_t st) {
    FusedArgs a{};
    a.coords = coords;
    a.n = 0;
    a.out = out;
    a.st = st;
    a.seg = seg;
    if (m->shadow) {
        a.n = max_n;  // sizes the persistent grid; the kernel reads its count from `seg`
        FH_CUDA(run_tc_any(m, false, a));
    } else {
        a.n = max_n;  // sizes the persistent grid only
        FH_CUDA(dispatch_fused(m, 0, a));
    }
    return FHASH_OK;
}

}  // namespace fh

using namespace fh;

static fhash_status check_model(fhash_model* m, const char* fn) {
    if (!m) return set_error(FHASH_EINVAL, "%s: null model", fn);
    return FHASH_OK;
}

extern "C" {

fhash_status fhash_lookup(fhash_model* m, const float* coords, int64_t n, uint64_t* rows, float* w, fhash_stream stream) {
    FH_RANGE("fhash_lookup");
    FH_TRY(check_model(m, "fhash_lookup"));
    if (n < 0 || (n && (!coords || !rows))) return set_error(FHASH_EINVAL, "fhash_lookup: bad arguments");
    if (n == 0) return FHASH_OK;
    if (!is_device_ptr(coords) || !is_device_ptr(rows) || (w && !is_device_ptr(w)))
        return set_error(FHASH_EINVAL, "fhash_lookup: buffers must be device memory");
    return launch_lookup(m, coords, n, rows, w, (cudaStream_t)stream);
}

fhash_status fhash_encode(fhash_model* m, const float* coords, int64_t n, float* enc, fhash_stream stream) {
    FH_RANGE("fhash_encode");
    FH_TRY(check_model(m, "fhash_encode"));
    if (n < 0 || (n && (!coords || !enc))) return set_error(FHASH_EINVAL, "fhash_encode: bad arguments");
    if (n == 0) return FHASH_OK;
    if (!is_device_ptr(coords) || !is_device_ptr(enc)) return set_error(FHASH_EINVAL, "fhash_encode: buffers must be device memory");
    FH_TRY(settle_deferred(m, (cudaStream_t)stream));
    return launch_encode(m, coords, n, enc, (cudaStream_t)stream);
}

fhash_status fhash_encode_backward(fhash_model* m, const float* coords, const float* d_enc, int64_t n,
                                   fhash_stream stream) {
    FH_RANGE("fhash_encode_backward");
    FH_TRY(check_model(m, "fhash_encode_backward"));
    if (n < 0 || (n && (!coords || !d_enc))) return set_error(FHASH_EINVAL, "fhash_encode_backward: bad arguments");
    if (n == 0) return FHASH_OK;
    if (!is_device_ptr(coords) || !is_device_ptr(d_enc))
        return set_error(FHASH_EINVAL, "fhash_encode_backward: buffers must be device memory");
    FH_TRY(settle_deferred(m, (cudaStream_t)stream));
    return launch_encode_backward(m, coords, n, d_enc, (cudaStream_t)stream);
}

fhash_status fhash_set_forward_path(fhash_model* m, int32_t path) {
    FH_TRY(check_model(m, "fhash_set_forward_path"));
    if (path != FHASH_FORWARD_AUTO && path != FHASH_FORWARD_FUSED && path != FHASH_FORWARD_SPLIT)
        return set_error(FHASH_EINVAL, "fhash_set_forward_path: unknown path %d", path);
    m->forward_path = path;
    return FHASH_OK;
}

fhash_status fhash_forward(fhash_model* m, const float* coords, int64_t n, float* out, fhash_stream stream) {
    FH_RANGE("fhash_forward");
    FH_TRY(check_model(m, "fhash_forward"));
    if (n < 0 || (n && (!coords || !out))) return set_error(FHASH_EINVAL, "fhash_forward: bad arguments");
    if (n == 0) return FHASH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    FH_TRY(settle_deferred(m, st));
    const void* dc;
    FH_TRY(stage_in(m, m->s_coords, coords, (size_t)n * 16, st, &dc));
    bool host_out = !is_device_ptr(out);
    float* dout = out;
    if (host_out) { FH_TRY(grow(m, m->s_out, (size_t)n * 4)); dout = (float*)m->s_out.p; }
    FH_TRY(launch_forward(m, (const float*)dc, n, dout, st));
    if (host_out) {
        FH_CUDA(cudaMemcpyAsync(out, dout, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
    }
    return FHASH_OK;
}

fhash_status fhash_compute_grads(fhash_model* m, const float* coords, const float* target, int64_t n, double* loss,
                                 fhash_stream stream) {
    FH_RANGE("fhash_compute_grads");
    FH_TRY(check_model(m, "fhash_compute_grads"));
    if (n <= 0 || !coords || !target) return set_error(FHASH_EINVAL, "fhash_compute_grads: need n > 0, coords and target");
    cudaStream_t st = (cudaStream_t)stream;
    FH_TRY(settle_deferred(m, st));
    const void *dc, *dt;
    FH_TRY(stage_in(m, m->s_coords, coords, (size_t)n * 16, st, &dc));
    FH_TRY(stage_in(m, m->s_target, target, (size_t)n * 4, st, &dt));
    FH_TRY(grow(m, m->s_loss, 64));
    bool dev_loss = loss && is_device_ptr(loss);
    FH_TRY(launch_grads2(m, (const float*)dc, (const float*)dt, n, dev_loss ? loss : (double*)m->s_loss.p, st));
    if (loss && !dev_loss) {
        FH_CUDA(cudaMemcpyAsync(loss, m->s_loss.p, 8, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
    }
    return FHASH_OK;
}

fhash_status fhash_apply_adam(fhash_model* m, const fhash_adam* a, fhash_stream stream) {
    FH_RANGE("fhash_apply_adam");
    FH_TRY(check_model(m, "fhash_apply_adam"));
    if (!a || !(a->lr >= 0.0f) || !(a->beta1 >= 0.0f && a->beta1 < 1.0f) || !(a->beta2 >= 0.0f && a->beta2 < 1.0f) ||
        !(a->eps > 0.0f))
        return set_error(FHASH_EINVAL, "fhash_apply_adam: bad hyper-parameters");
    return launch_adam(m, a, (cudaStream_t)stream);
}

fhash_status fhash_train_step(fhash_model* m, const float* coords, const float* target, int64_t n, const fhash_adam* a,
                              double* loss, fhash_stream stream) {
    FH_RANGE("fhash_train_step");
    FH_TRY(check_model(m, "fhash_train_step"));
    if (!a) return set_error(FHASH_EINVAL, "fhash_train_step: null adam");
    if (n <= 0 || !coords || !target) return set_error(FHASH_EINVAL, "fhash_train_step: need n > 0, coords and target");
    cudaStream_t st = (cudaStream_t)stream;
    const void *dc, *dt;
    FH_TRY(stage_in(m, m->s_coords, coords, (size_t)n * 16, st, &dc));
    FH_TRY(stage_in(m, m->s_target, target, (size_t)n * 4, st, &dt));
    FH_TRY(grow(m, m->s_loss, 64));
    bool dev_loss = loss && is_device_ptr(loss);
    if (!(a->lr >= 0.0f) || !(a->beta1 >= 0.0f && a->beta1 < 1.0f) || !(a->beta2 >= 0.0f && a->beta2 < 1.0f) ||
        !(a->eps > 0.0f))
        return set_error(FHASH_EINVAL, "fhash_train_step: bad hyper-parameters");
    FH_TRY(launch_train_step(m, (const float*)dc, (const float*)dt, n, a, dev_loss ? loss : (double*)m->s_loss.p, st));
    if (loss && !dev_loss) {
        FH_CUDA(cudaMemcpyAsync(loss, m->s_loss.p, 8, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
    }
    return FHASH_OK;
}

}  // extern "C"
