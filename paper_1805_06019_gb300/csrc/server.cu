// Serving runtime: resident light fields, continuous batching of view
// requests over several CUDA streams, admission by device memory.
//
// Threads: callers submit and poll under one mutex; a worker thread admits
// and launches; CUDA host callbacks (cudaLaunchHostFunc, run by the CUDA driver in
// stream order after a call's copies to the host) stamp completion, return
// the call's memory and pinned parameter slot, and wake the worker.  Host
// callbacks make no CUDA calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "rlfc_internal.h"

namespace rlfc {
namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t ticket;
    uint32_t lf;
    float u, v, d;
    uint32_t w, h;
    uint32_t u8;          // 1: 8-bit RGB output, 0: float RGB
    void *host_out;
    double t_submit;
};

// device bytes of one request: its view and its camera parameters
size_t view_bytes(uint32_t w, uint32_t h, uint32_t u8) { return (size_t)w * h * (u8 ? 3 : 12) + 12; }

constexpr uint32_t kParamSlots = 512;

}  // namespace
}  // namespace rlfc

struct rlfc_server;

namespace rlfc {
namespace {
struct Step {
    rlfc_server *srv;
    std::vector<Req> reqs;
    size_t bytes;
    uint32_t slot;
    uint32_t stream;
    int status;
    double t_start;
};
}  // namespace
}  // namespace rlfc

struct rlfc_server {
    rlfc_server_config cfg{};
    int device = 0;
    std::vector<const rlfc_stream *> lfs;
    std::vector<cudaStream_t> streams;
    std::vector<uint32_t> inflight;          // calls queued per stream
    float *pinned = nullptr;                 // kParamSlots slots of max_batch * 3 floats
    std::vector<uint32_t> free_slots;
    std::mutex mu;
    std::condition_variable cv;              // worker: work or capacity arrived
    std::condition_variable cv_done;         // pollers: completions arrived
    std::deque<rlfc::Req> queue;
    std::deque<rlfc_completion> done;
    size_t in_use = 0;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0;
    bool stop = false;
    std::thread worker;
};

namespace rlfc {
namespace {

void CUDART_CB on_step_done(void *p)
{
    Step *s = static_cast<Step *>(p);
    rlfc_server *srv = s->srv;
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (const Req &r : s->reqs) {
            rlfc_completion c{};
            c.ticket = r.ticket;
            c.status = s->status;
            c.lf = r.lf;
            c.batch = (uint32_t)s->reqs.size();
            c.t_submit = r.t_submit;
            c.t_start = s->t_start;
            c.t_done = t;
            srv->done.push_back(c);
        }
        srv->completed += s->reqs.size();
        srv->in_use -= s->bytes;
        srv->free_slots.push_back(s->slot);
        srv->inflight[s->stream]--;
    }
    srv->cv.notify_all();
    srv->cv_done.notify_all();
    delete s;
}

// Issue one render call for `reqs` (same light field, size and output
// format) on stream `si`; completion arrives through on_step_done.
void launch_step(rlfc_server *srv, std::vector<Req> &&reqs, size_t bytes, uint32_t slot, uint32_t si)
{
    Step *step = new Step{srv, std::move(reqs), bytes, slot, si, RLFC_OK, now_s()};
    const Req &r0 = step->reqs[0];
    const uint32_t n = (uint32_t)step->reqs.size(), w = r0.w, h = r0.h;
    cudaStream_t st = srv->streams[si];
    float *par = srv->pinned + (size_t)slot * srv->cfg.max_batch * 3;
    for (uint32_t i = 0; i < n; i++) {
        par[2 * i] = step->reqs[i].u;
        par[2 * i + 1] = step->reqs[i].v;
        par[2 * n + i] = step->reqs[i].d;
    }
    // one stream-ordered allocation: the parameters, then the views
    const size_t view = (size_t)w * h * 3 * (r0.u8 ? 1 : sizeof(float));
    const size_t par_bytes = (3 * (size_t)n * sizeof(float) + 255) / 256 * 256;
    uint8_t *d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d), par_bytes + view * n, st);
    int rc = RLFC_OK;
    if (e == cudaSuccess) {
        float *d_par = reinterpret_cast<float *>(d);
        uint8_t *d_view = d + par_bytes;
        e = cudaMemcpyAsync(d_par, par, 3 * (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            rc = r0.u8 ? launch_render(srv->lfs[r0.lf], d_par, d_par + 2 * n, w, h, n, nullptr, st, d_view)
                       : launch_render(srv->lfs[r0.lf], d_par, d_par + 2 * n, w, h, n,
                                       reinterpret_cast<float *>(d_view), st);
            for (uint32_t i = 0; i < n && rc == RLFC_OK && e == cudaSuccess; i++)
                e = cudaMemcpyAsync(step->reqs[i].host_out, d_view + view * i, view, cudaMemcpyDeviceToHost, st);
        }
        cudaFreeAsync(d, st);
    }
    if (e != cudaSuccess) {
        cuda_fail(e, "server step");
        rc = RLFC_E_CUDA;
    }
    step->status = rc;
    if (cudaLaunchHostFunc(st, on_step_done, step) != cudaSuccess) {
        // the stream cannot take the callback: complete the step here
        cudaGetLastError();
        cudaStreamSynchronize(st);
        step->status = step->status == RLFC_OK ? RLFC_E_CUDA : step->status;
        on_step_done(step);
    }
}

// The stream with the fewest queued calls, or -1 when all are full.
int pick_stream(const rlfc_server *srv)
{
    int best = -1;
    for (size_t i = 0; i < srv->inflight.size(); i++)
        if (srv->inflight[i] < srv->cfg.max_inflight && (best < 0 || srv->inflight[i] < srv->inflight[best]))
            best = (int)i;
    return best;
}

void worker_main(rlfc_server *srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        srv->cv.wait(lk, [&] {
            if (srv->queue.empty())
                return srv->stop;
            const Req &r = srv->queue.front();
            return srv->in_use + view_bytes(r.w, r.h, r.u8) <= srv->cfg.memory_budget && !srv->free_slots.empty() &&
                   pick_stream(srv) >= 0;
        });
        if (srv->queue.empty() && srv->stop)
            break;
        // admit in arrival order while the outputs fit; group by (light
        // field, size, format), keeping the order inside each group
        using Key = std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>;
        std::map<Key, std::vector<Req>> groups;
        std::vector<Key> order;
        size_t admitted = 0;
        while (!srv->queue.empty()) {
            const Req &r = srv->queue.front();
            const size_t b = view_bytes(r.w, r.h, r.u8);
            if (srv->in_use + admitted + b > srv->cfg.memory_budget)
                break;
            const Key key = std::make_tuple(r.lf, r.w, r.h, r.u8);
            auto it = groups.find(key);
            if (it == groups.end()) {
                order.push_back(key);
                it = groups.emplace(key, std::vector<Req>()).first;
            }
            it->second.push_back(r);
            admitted += b;
            srv->queue.pop_front();
        }
        // one call per max_batch views of a group, each with a pinned slot
        // and room on a stream; the rest go back to the head of the queue
        std::vector<std::tuple<std::vector<Req>, size_t, uint32_t, uint32_t>> calls;
        std::vector<Req> back;
        for (const auto &key : order) {
            std::vector<Req> &g = groups[key];
            for (size_t i = 0; i < g.size(); i += srv->cfg.max_batch) {
                const size_t j = std::min(g.size(), i + srv->cfg.max_batch);
                std::vector<Req> part(g.begin() + i, g.begin() + j);
                const int si = pick_stream(srv);
                if (srv->free_slots.empty() || si < 0) {
                    back.insert(back.end(), part.begin(), part.end());
                    continue;
                }
                size_t b = 0;
                for (const Req &r : part)
                    b += view_bytes(r.w, r.h, r.u8);
                const uint32_t slot = srv->free_slots.back();
                srv->free_slots.pop_back();
                srv->in_use += b;
                srv->inflight[si]++;
                calls.emplace_back(std::move(part), b, slot, (uint32_t)si);
            }
        }
        if (!back.empty()) {
            std::sort(back.begin(), back.end(), [](const Req &a, const Req &b) { return a.ticket < b.ticket; });
            srv->queue.insert(srv->queue.begin(), back.begin(), back.end());
        }
        lk.unlock();
        for (auto &c : calls)
            launch_step(srv, std::move(std::get<0>(c)), std::get<1>(c), std::get<2>(c), std::get<3>(c));
        lk.lock();
    }
}

}  // namespace
}  // namespace rlfc

extern "C" {

RLFC_API double rlfc_server_now(void) { return rlfc::now_s(); }

RLFC_API int rlfc_server_create(const rlfc_server_config *cfg, rlfc_server **out)
{
    using namespace rlfc;
    if (!cfg || !out || cfg->n_streams < 1 || cfg->n_streams > 64 || cfg->max_batch < 1 ||
        cfg->max_batch > 4096 || cfg->memory_budget == 0 || cfg->max_inflight < 1 || cfg->max_inflight > 64) {
        set_error("rlfc_server_create: invalid configuration");
        return RLFC_E_INVALID_ARG;
    }
    *out = nullptr;
    rlfc_server *srv = new (std::nothrow) rlfc_server;
    if (!srv) {
        set_error("rlfc_server_create: out of host memory");
        return RLFC_E_OOM;
    }
    srv->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&srv->device);
    for (uint32_t i = 0; i < cfg->n_streams && e == cudaSuccess; i++) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            srv->streams.push_back(st);
            srv->inflight.push_back(0);
        }
    }
    if (e == cudaSuccess)
        e = cudaMallocHost(&srv->pinned, (size_t)kParamSlots * cfg->max_batch * 3 * sizeof(float));
    if (e != cudaSuccess) {
        const int rc = e == cudaErrorMemoryAllocation ? RLFC_E_OOM : RLFC_E_CUDA;
        cuda_fail(e, "rlfc_server_create");
        for (cudaStream_t st : srv->streams)
            cudaStreamDestroy(st);
        delete srv;
        return rc;
    }
    for (uint32_t i = 0; i < kParamSlots; i++)
        srv->free_slots.push_back(kParamSlots - 1 - i);
    srv->worker = std::thread(worker_main, srv);
    *out = srv;
    return RLFC_OK;
}

RLFC_API int rlfc_server_add(rlfc_server *srv, const rlfc_stream *s, uint32_t *lf_id)
{
    if (!srv || !s || !lf_id || s->device != srv->device) {
        rlfc::set_error("rlfc_server_add: null argument or stream on another device");
        return RLFC_E_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    *lf_id = (uint32_t)srv->lfs.size();
    srv->lfs.push_back(s);
    return RLFC_OK;
}

static int server_submit(rlfc_server *srv, uint32_t lf_id, float u, float v, float disp, uint32_t out_w,
                         uint32_t out_h, void *host_out, uint32_t u8, uint64_t *ticket)
{
    using namespace rlfc;
    if (!srv || !host_out || out_w == 0 || out_h == 0) {
        set_error("rlfc_server_submit: null argument or empty size");
        return RLFC_E_INVALID_ARG;
    }
    if (out_w > 32768 || out_h > 32768 || view_bytes(out_w, out_h, u8) > srv->cfg.memory_budget) {
        set_error("rlfc_server_submit: view larger than the memory budget or the renderer's limit");
        return RLFC_E_RANGE;
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (lf_id >= srv->lfs.size() || srv->stop) {
            set_error("rlfc_server_submit: unknown light field");
            return RLFC_E_INVALID_ARG;
        }
        Req r{srv->next_ticket++, lf_id, u, v, disp, out_w, out_h, u8, host_out, now_s()};
        srv->queue.push_back(r);
        srv->submitted++;
        if (ticket)
            *ticket = r.ticket;
    }
    srv->cv.notify_all();
    return RLFC_OK;
}

RLFC_API int rlfc_server_submit(rlfc_server *srv, uint32_t lf_id, float u, float v, float disp,
                                uint32_t out_w, uint32_t out_h, float *host_out, uint64_t *ticket)
{
    return server_submit(srv, lf_id, u, v, disp, out_w, out_h, host_out, 0, ticket);
}

RLFC_API int rlfc_server_submit_u8(rlfc_server *srv, uint32_t lf_id, float u, float v, float disp,
                                   uint32_t out_w, uint32_t out_h, uint8_t *host_out, uint64_t *ticket)
{
    return server_submit(srv, lf_id, u, v, disp, out_w, out_h, host_out, 1, ticket);
}

RLFC_API int rlfc_server_poll(rlfc_server *srv, rlfc_completion *out, size_t cap, size_t *n, int wait)
{
    if (!srv || !n || (cap && !out)) {
        rlfc::set_error("rlfc_server_poll: null argument");
        return RLFC_E_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(srv->mu);
    if (wait)
        srv->cv_done.wait(lk, [&] { return srv->completed == srv->submitted; });
    size_t k = 0;
    while (k < cap && !srv->done.empty()) {
        out[k++] = srv->done.front();
        srv->done.pop_front();
    }
    *n = k;
    return RLFC_OK;
}

RLFC_API void rlfc_server_free(rlfc_server *srv)
{
    if (!srv)
        return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->worker.joinable())
        srv->worker.join();
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        srv->cv_done.wait(lk, [&] { return srv->completed == srv->submitted; });
    }
    rlfc::DeviceGuard g(srv->device);
    for (cudaStream_t st : srv->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    cudaFreeHost(srv->pinned);
    delete srv;
}

}  // extern "C"
