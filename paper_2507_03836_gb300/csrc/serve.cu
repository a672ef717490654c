// Continuous-batching serving loop (see include/fhash_serve.h): admission by memory budget into a
// request-scratch pool, one packed sample buffer per tick, one sample-generation launch over all live
// requests, per-model CUDA-graph replays of the persistent encode+MLP launch, one compositing / decode
// scatter launch over all live requests, one readback per tick.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "fhash_serve.h"
#include "pool.h"
#include "render.cuh"

namespace fh {

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t id = 0;
    fhash_request r{};
    int state = FHASH_REQ_QUEUED;
    bool cancel = false;
    double t_submit = 0, t_done = 0;
    uint64_t need = 0, pool_off = 0;
    bool holds_pool = false;
    int slot = -1;
    // render
    RenderGeo g{};
    int64_t NR = 0;
    RayState* rs = nullptr;
    int* al[2] = {nullptr, nullptr};
    int* cnt = nullptr;
    int cur = 0, na = 0;
    bool fresh = false;
    // decode
    int64_t dims[3] = {0, 0, 0}, total = 0, next = 0;
    // this tick
    int64_t off = 0, take = 0;
    int ns = 0;
};

// One request's share of a packed per-tick launch: threads [w0, w0 + n) of the launch work on it.
struct TickWork {
    int64_t w0, n;
    int64_t off;        // first packed sample slot of the request in this tick
    int64_t next;       // decode: first grid point of this tick's chunk
    RayState* rs;
    int* alive;         // render: this round's alive list (its ray list at initialisation)
    int* next_alive;    // render: the next round's alive list
    int* cnt;           // render: samples emitted per alive ray
    int* n_next;        // render: counter of the list being appended to
    float4* rgba;
    int32_t* counts;
    const float4* tf;
    float* out;         // decode output
    int32_t kind, slot, ns, pad;
    int32_t dims[3];
    float t_norm;
};

// Entry holding thread i (entries sorted by w0, w0[0] = 0).
__device__ __forceinline__ int find_work(const TickWork* __restrict__ wk, int nw, int64_t i) {
    int lo = 0, hi = nw - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (wk[mid].w0 <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Rays of every render admitted in this tick (Algorithm 1's initialisation), one launch.
__global__ void k_tick_init(const TickWork* __restrict__ wk, int nw, int64_t total, const RenderGeo* __restrict__ geo) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const TickWork& w = wk[find_work(wk, nw, i)];
    ray_init_px(geo[w.slot], (int)(i - w.w0), w.rs, w.alive, w.n_next, w.rgba, w.counts);
}

// Sample generation of every live request, one launch: each render's alive rays march one ARM round, each
// decode writes the coordinates of its next chunk of grid points.
__global__ void k_tick_generate(const TickWork* __restrict__ wk, int nw, int64_t total, const RenderGeo* __restrict__ geo,
                                float4* __restrict__ coords) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const TickWork& w = wk[find_work(wk, nw, i)];
    const int64_t j = i - w.w0;
    if (w.kind == FHASH_REQ_RENDER) {
        if (j == 0) *w.n_next = 0;  // the composite launch appends the surviving rays to it
        arm_generate_ray(geo[w.slot], w.rs, w.alive[j], (int)j, w.ns, coords + w.off, w.cnt, nullptr);
    } else {
        const int64_t p = w.next + j;
        const int nx = w.dims[0], ny = w.dims[1], nz = w.dims[2];
        const int x = (int)(p % nx), y = (int)((p / nx) % ny), z = (int)(p / ((int64_t)nx * ny));
        coords[w.off + j] = make_float4(__fdiv_rn((float)x, (float)(nx - 1)), __fdiv_rn((float)y, (float)(ny - 1)),
                                        __fdiv_rn((float)z, (float)(nz - 1)), w.t_norm);
    }
}

// Compositing of every render's samples and the decode values into their outputs, one launch.
__global__ void k_tick_composite(const TickWork* __restrict__ wk, int nw, int64_t total, const RenderGeo* __restrict__ geo,
                                 const float* __restrict__ vals) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const TickWork& w = wk[find_work(wk, nw, i)];
    const int64_t j = i - w.w0;
    if (w.kind == FHASH_REQ_RENDER)
        arm_composite_ray(geo[w.slot], w.rs, w.alive[j], (int)j, w.ns, w.cnt, vals + w.off, w.tf, w.next_alive,
                          w.n_next, w.rgba, w.counts, nullptr);
    else
        w.out[w.next + j] = vals[w.off + j];
}

static uint64_t render_scratch(int64_t NR) {
    auto up = [](uint64_t x) { return (x + 255) / 256 * 256; };
    return up(NR * sizeof(RayState)) + 3 * up(NR * 4);
}

static uint64_t serving_bytes(const fhash_model* m) {
    const int64_t nbrick = m->nbx * m->nby * m->nbz;
    return m->n_params * 4 + (m->shadow ? m->n_params * 2 : 0) + (uint64_t)(nbrick * 17 * m->nt) + m->dir_words * 16;
}

}  // namespace fh

using namespace fh;

struct fhash_server {
    std::mutex mu;
    std::vector<fhash_model*> models;
    uint64_t budget = 0;
    int max_live = 0;
    int64_t cap = 0;
    float4* coords = nullptr;
    float* vals = nullptr;
    int64_t* segs = nullptr;    // device [n_models][2]
    int64_t* h_segs = nullptr;  // pinned
    int* ctr = nullptr;         // device [max_live]
    int* h_ctr = nullptr;       // pinned
    RenderGeo* geo = nullptr;   // device [max_live]: geometry of the render in each slot
    RenderGeo* h_geo = nullptr; // pinned mirror
    TickWork* work = nullptr;   // device [2 * max_live]: admission entries, then the tick's entries
    TickWork* h_work = nullptr; // pinned mirror
    char* pool_mem = nullptr;
    Pool pool;
    std::vector<cudaGraphExec_t> graphs;
    std::vector<cudaGraph_t> graph_defs;
    std::deque<Req*> queue;
    std::vector<Req*> live;
    std::map<uint64_t, Req*> all;
    std::vector<int> free_slots;
    uint64_t next_id = 1;
    int64_t ticks = 0, samples = 0, launches = 0, launches_aux = 0;
};

static void server_free(fhash_server* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    for (auto g : s->graphs) if (g) cudaGraphExecDestroy(g);
    for (auto g : s->graph_defs) if (g) cudaGraphDestroy(g);
    if (s->coords) cudaFree(s->coords);
    if (s->vals) cudaFree(s->vals);
    if (s->segs) cudaFree(s->segs);
    if (s->ctr) cudaFree(s->ctr);
    if (s->pool_mem) cudaFree(s->pool_mem);
    if (s->h_segs) cudaFreeHost(s->h_segs);
    if (s->h_ctr) cudaFreeHost(s->h_ctr);
    if (s->geo) cudaFree(s->geo);
    if (s->work) cudaFree(s->work);
    if (s->h_geo) cudaFreeHost(s->h_geo);
    if (s->h_work) cudaFreeHost(s->h_work);
    for (auto& kv : s->all) delete kv.second;
    delete s;
}

extern "C" {

fhash_status fhash_server_create(fhash_model* const* models, int32_t n_models, uint64_t budget, int32_t max_live,
                                 int64_t tick_samples, fhash_stream stream, fhash_server** out) {
    if (!models || n_models < 1 || n_models > 64 || max_live < 1 || max_live > 4096 || tick_samples < 128 ||
        tick_samples > (1ll << 30) || !out)
        return set_error(FHASH_EINVAL, "fhash_server_create: bad arguments");
    *out = nullptr;
    uint64_t fixed = (uint64_t)tick_samples * 20 + 4096;
    for (int i = 0; i < n_models; ++i) {
        if (!models[i]) return set_error(FHASH_EINVAL, "fhash_server_create: null model %d", i);
        FH_TRY(settle_deferred(models[i], (cudaStream_t)stream));
        fixed += serving_bytes(models[i]);
    }
    if (fixed >= budget)
        return set_error(FHASH_EINVAL, "fhash_server_create: models and packed buffers need %llu bytes, budget %llu",
                         (unsigned long long)fixed, (unsigned long long)budget);
    fhash_server* s = new fhash_server();
    s->models.assign(models, models + n_models);
    s->budget = budget;
    s->max_live = max_live;
    s->cap = tick_samples;
    struct Guard {
        fhash_server*& s;
        ~Guard() { if (s) server_free(s); }
    } guard{s};
    cudaStream_t st = (cudaStream_t)stream;
    FH_CUDA(cudaMalloc(&s->coords, (size_t)tick_samples * 16));
    FH_CUDA(cudaMalloc(&s->vals, (size_t)tick_samples * 4));
    FH_CUDA(cudaMalloc(&s->segs, (size_t)n_models * 16));
    FH_CUDA(cudaMalloc(&s->ctr, (size_t)max_live * 4));
    FH_CUDA(cudaMallocHost(&s->h_segs, (size_t)n_models * 16));
    FH_CUDA(cudaMallocHost(&s->h_ctr, (size_t)max_live * 4));
    FH_CUDA(cudaMalloc(&s->geo, (size_t)max_live * sizeof(RenderGeo)));
    FH_CUDA(cudaMallocHost(&s->h_geo, (size_t)max_live * sizeof(RenderGeo)));
    FH_CUDA(cudaMalloc(&s->work, (size_t)2 * max_live * sizeof(TickWork)));
    FH_CUDA(cudaMallocHost(&s->h_work, (size_t)2 * max_live * sizeof(TickWork)));
    const uint64_t pool = budget - fixed;
    FH_CUDA(cudaMalloc(&s->pool_mem, pool));
    s->pool.init(s->pool_mem, pool);
    for (int i = max_live - 1; i >= 0; --i) s->free_slots.push_back(i);
    // one packed encode+MLP launch per model, captured once (its segment lives in device memory)
    FH_CUDA(cudaStreamSynchronize(st));
    cudaStream_t cs;
    FH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    FH_CUDA(cudaMemsetAsync(s->segs, 0, (size_t)n_models * 16, cs));  // same stream as the first launches
    fhash_status rc = FHASH_OK;
    for (int i = 0; i < n_models && rc == FHASH_OK; ++i) {
        // a first launch (count 0) sets the kernels' attributes outside the capture
        rc = launch_forward_seg(models[i], (const float*)s->coords, s->vals, s->segs + 2 * i, tick_samples, cs);
        if (rc != FHASH_OK) break;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = launch_forward_seg(models[i], (const float*)s->coords, s->vals, s->segs + 2 * i, tick_samples, cs);
            e = cudaStreamEndCapture(cs, &g);
        }
        if (e == cudaSuccess && rc == FHASH_OK) e = cudaGraphInstantiate(&ge, g, 0);
        if (e != cudaSuccess) rc = cuda_error(e, "serving graph capture");
        s->graph_defs.push_back(g);
        s->graphs.push_back(ge);
    }
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
    if (rc != FHASH_OK) return rc;
    *out = s;
    s = nullptr;
    return FHASH_OK;
}

void fhash_server_destroy(fhash_server* s) { server_free(s); }

fhash_status fhash_server_submit(fhash_server* s, const fhash_request* r, uint64_t* id) {
    if (!s || !r || !id) return set_error(FHASH_EINVAL, "fhash_server_submit: null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    if (r->model < 0 || r->model >= (int)s->models.size()) return set_error(FHASH_EINVAL, "request: bad model index");
    if (!(r->t_norm >= 0.0f && r->t_norm <= 1.0f) || !r->out) return set_error(FHASH_EINVAL, "request: bad t_norm or out");
    fhash_model* m = s->models[r->model];
    Req* q = new Req();
    q->r = *r;
    if (r->kind == FHASH_REQ_RENDER) {
        if (r->w < 1 || r->h < 1 || (int64_t)r->w * r->h > (1 << 26) || r->max_pace < 1 || r->max_pace > 64 || !r->tf) {
            delete q;
            return set_error(FHASH_EINVAL, "render request: bad size, pace or tf");
        }
        q->NR = (int64_t)r->w * r->h;
        if (q->NR > s->cap) {  // one ARM round of every alive ray must fit in a tick
            delete q;
            return set_error(FHASH_EINVAL, "render request: %lld pixels exceed the %lld samples of a tick",
                             (long long)(int64_t)r->w * r->h, (long long)s->cap);
        }
        q->need = render_scratch(q->NR);
        q->g = make_geo(m, &r->cam, r->t_norm, r->w, r->h);
    } else if (r->kind == FHASH_REQ_DECODE) {
        if (r->upsample < 1 || r->upsample > 8) { delete q; return set_error(FHASH_EINVAL, "decode request: upsample 1..8"); }
        for (int a = 0; a < 3; ++a) q->dims[a] = decode_points(m->fbb_size[a], r->upsample);
        q->total = q->dims[0] * q->dims[1] * q->dims[2];
        q->need = 0;
    } else {
        delete q;
        return set_error(FHASH_EINVAL, "request: unknown kind %d", r->kind);
    }
    if (q->need > s->pool.bytes) {
        delete q;
        return set_error(FHASH_EINVAL, "request needs %llu scratch bytes, pool has %llu", (unsigned long long)q->need,
                         (unsigned long long)s->pool.bytes);
    }
    q->id = s->next_id++;
    q->t_submit = now_ms();
    s->queue.push_back(q);
    s->all[q->id] = q;
    *id = q->id;
    return FHASH_OK;
}

static void finish(fhash_server* s, Req* q, int state) {
    q->state = state;
    q->t_done = now_ms();
    if (q->holds_pool) s->pool.release(q->pool_off, q->need);
    q->holds_pool = false;
    if (q->slot >= 0) s->free_slots.push_back(q->slot);
    q->slot = -1;
}

fhash_status fhash_server_tick(fhash_server* s, fhash_stream stream, int32_t* n_completed) {
    FH_RANGE("fhash_server_tick");
    if (!s) return set_error(FHASH_EINVAL, "fhash_server_tick: null server");
    std::lock_guard<std::mutex> lock(s->mu);
    cudaStream_t st = (cudaStream_t)stream;
    for (fhash_model* m : s->models) FH_TRY(settle_deferred(m, st));  // a model trained since the last tick
    int done = 0;
    // drop cancelled live requests (their last tick has completed: every tick ends synchronised)
    for (size_t i = 0; i < s->live.size();) {
        if (s->live[i]->cancel) { finish(s, s->live[i], FHASH_REQ_CANCELLED); s->live.erase(s->live.begin() + i); }
        else ++i;
    }
    // 1. admission in arrival order
    bool admitted_render = false;
    while (!s->queue.empty() && (int)s->live.size() < s->max_live && !s->free_slots.empty()) {
        Req* q = s->queue.front();
        if (q->cancel) { s->queue.pop_front(); finish(s, q, FHASH_REQ_CANCELLED); continue; }
        uint64_t off = 0;
        if (q->need && !s->pool.alloc(q->need, &off)) break;  // head of line waits for memory
        s->queue.pop_front();
        q->pool_off = off;
        q->holds_pool = q->need != 0;
        q->slot = s->free_slots.back();
        s->free_slots.pop_back();
        q->state = FHASH_REQ_LIVE;
        if (q->r.kind == FHASH_REQ_RENDER) {
            char* b = s->pool.base + off;
            auto up = [](uint64_t x) { return (x + 255) / 256 * 256; };
            q->rs = (RayState*)b;
            q->al[0] = (int*)(b + up(q->NR * sizeof(RayState)));
            q->al[1] = (int*)((char*)q->al[0] + up(q->NR * 4));
            q->cnt = (int*)((char*)q->al[1] + up(q->NR * 4));
            s->h_geo[q->slot] = q->g;
            q->fresh = true;
            admitted_render = true;
        }
        s->live.push_back(q);
    }
    if (admitted_render) {
        // every admitted render's rays in one launch (the counters of the other slots were read already)
        int nw = 0;
        int64_t total = 0;
        for (Req* q : s->live) {
            if (!q->fresh) continue;
            TickWork& w = s->h_work[nw++];
            memset(&w, 0, sizeof w);
            w.w0 = total;
            w.n = q->NR;
            w.rs = q->rs;
            w.alive = q->al[0];
            w.n_next = s->ctr + q->slot;
            w.rgba = (float4*)q->r.out;
            w.counts = q->r.counts;
            w.slot = q->slot;
            total += q->NR;
        }
        FH_CUDA(cudaMemsetAsync(s->ctr, 0, (size_t)s->max_live * 4, st));
        FH_CUDA(cudaMemcpyAsync(s->geo, s->h_geo, (size_t)s->max_live * sizeof(RenderGeo), cudaMemcpyHostToDevice, st));
        FH_CUDA(cudaMemcpyAsync(s->work, s->h_work, (size_t)nw * sizeof(TickWork), cudaMemcpyHostToDevice, st));
        k_tick_init<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(s->work, nw, total, s->geo);
        FH_CUDA(cudaGetLastError());
        s->launches_aux += 1;
        FH_CUDA(cudaMemcpyAsync(s->h_ctr, s->ctr, (size_t)s->max_live * 4, cudaMemcpyDeviceToHost, st));
        FH_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i < s->live.size();) {
            Req* q = s->live[i];
            if (q->fresh) {
                q->fresh = false;
                q->na = s->h_ctr[q->slot];
                q->cur = 0;
                if (q->na == 0) { finish(s, q, FHASH_REQ_DONE); s->live.erase(s->live.begin() + i); ++done; continue; }
            }
            ++i;
        }
    }
    // 2. pack: each model's requests form one contiguous segment
    const int nm = (int)s->models.size();
    int64_t off = 0;
    for (Req* q : s->live) q->take = 0;
    for (int mi = 0; mi < nm; ++mi) {
        const int64_t base = off;
        for (Req* q : s->live) {
            if (q->r.model != mi) continue;
            if (q->r.kind == FHASH_REQ_RENDER) {
                const int64_t room = (s->cap - off) / std::max(q->na, 1);
                if (room < 1) continue;
                int ns = (int)std::max<int64_t>(1, std::min<int64_t>(q->NR / q->na, q->r.max_pace));
                ns = (int)std::min<int64_t>(ns, room);
                q->ns = ns;
                q->off = off;
                q->take = (int64_t)q->na * ns;
            } else {
                const int64_t take = std::min(q->total - q->next, s->cap - off);
                if (take < 1) continue;
                q->off = off;
                q->take = take;
            }
            off += q->take;
        }
        s->h_segs[2 * mi] = base;
        s->h_segs[2 * mi + 1] = off - base;
    }
    // 3. sample generation of every live request in one launch (a work table of their shares)
    TickWork* hw = s->h_work + s->max_live;
    int nw = 0;
    int64_t total = 0;
    for (Req* q : s->live) {
        if (!q->take) continue;
        TickWork& w = hw[nw++];
        memset(&w, 0, sizeof w);
        w.w0 = total;
        w.off = q->off;
        w.kind = q->r.kind;
        w.slot = q->slot;
        if (q->r.kind == FHASH_REQ_RENDER) {
            w.n = q->na;
            w.ns = q->ns;
            w.rs = q->rs;
            w.alive = q->al[q->cur];
            w.next_alive = q->al[1 - q->cur];
            w.cnt = q->cnt;
            w.n_next = s->ctr + q->slot;
            w.rgba = (float4*)q->r.out;
            w.counts = q->r.counts;
            w.tf = (const float4*)q->r.tf;
        } else {
            w.n = q->take;
            w.next = q->next;
            for (int a = 0; a < 3; ++a) w.dims[a] = (int32_t)q->dims[a];
            w.t_norm = q->r.t_norm;
            w.out = q->r.out;
        }
        total += w.n;
    }
    TickWork* dw = s->work + s->max_live;
    if (nw) {
        FH_CUDA(cudaMemcpyAsync(dw, hw, (size_t)nw * sizeof(TickWork), cudaMemcpyHostToDevice, st));
        k_tick_generate<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(dw, nw, total, s->geo, s->coords);
        FH_CUDA(cudaGetLastError());
        s->launches_aux += 1;
    }
    // 4. one packed encode+MLP launch per model with samples (graph replay)
    FH_CUDA(cudaMemcpyAsync(s->segs, s->h_segs, (size_t)nm * 16, cudaMemcpyHostToDevice, st));
    for (int mi = 0; mi < nm; ++mi) {
        if (s->h_segs[2 * mi + 1] == 0) continue;
        FH_CUDA(cudaGraphLaunch(s->graphs[mi], st));
        ++s->launches;
    }
    // 5. compositing and decode values of every live request in one launch
    if (nw) {
        k_tick_composite<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(dw, nw, total, s->geo, s->vals);
        FH_CUDA(cudaGetLastError());
        s->launches_aux += 1;
    }
    // 6. progress readback (one copy, one sync)
    FH_CUDA(cudaMemcpyAsync(s->h_ctr, s->ctr, (size_t)s->max_live * 4, cudaMemcpyDeviceToHost, st));
    FH_CUDA(cudaStreamSynchronize(st));
    s->samples += off;
    s->ticks += 1;
    for (size_t i = 0; i < s->live.size();) {
        Req* q = s->live[i];
        bool fin = false;
        if (q->take) {
            if (q->r.kind == FHASH_REQ_RENDER) {
                q->na = s->h_ctr[q->slot];
                q->cur = 1 - q->cur;
                fin = q->na == 0;
            } else {
                q->next += q->take;
                fin = q->next == q->total;
            }
        }
        if (fin) {
            finish(s, q, FHASH_REQ_DONE);
            s->live.erase(s->live.begin() + i);
            ++done;
        } else {
            ++i;
        }
    }
    if (n_completed) *n_completed = done;
    return FHASH_OK;
}

fhash_status fhash_server_poll(fhash_server* s, uint64_t id, int32_t* state, double* latency_ms) {
    if (!s || !state) return set_error(FHASH_EINVAL, "fhash_server_poll: null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return set_error(FHASH_EINVAL, "fhash_server_poll: unknown id");
    *state = it->second->state;
    if (latency_ms) *latency_ms = it->second->state == FHASH_REQ_DONE ? it->second->t_done - it->second->t_submit : -1.0;
    return FHASH_OK;
}

fhash_status fhash_server_cancel(fhash_server* s, uint64_t id) {
    if (!s) return set_error(FHASH_EINVAL, "fhash_server_cancel: null server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return set_error(FHASH_EINVAL, "fhash_server_cancel: unknown id");
    if (it->second->state == FHASH_REQ_QUEUED || it->second->state == FHASH_REQ_LIVE) it->second->cancel = true;
    return FHASH_OK;
}

fhash_status fhash_server_get_stats(fhash_server* s, fhash_server_stats* o) {
    if (!s || !o) return set_error(FHASH_EINVAL, "fhash_server_get_stats: null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    o->ticks = s->ticks;
    o->samples = s->samples;
    o->model_launches = s->launches;
    o->live = (int64_t)s->live.size();
    int64_t q = 0;
    for (Req* r : s->queue) q += r->cancel ? 0 : 1;
    o->queued = q;
    o->pool_bytes = s->pool.bytes;
    o->pool_used = s->pool.used;
    o->packed_launches = s->launches_aux;
    return FHASH_OK;
}

}  // extern "C"
