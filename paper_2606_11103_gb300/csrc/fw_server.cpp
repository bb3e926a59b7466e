// Serving runtime: continuous batching of simulation requests on one GPU.
//
// Threads:
//  * the caller's threads submit, poll and cancel (never touch the GPU);
//  * a builder thread turns admitted requests into device-resident media
//    (maps uploaded, classes tabulated, sources and receivers set);
//  * a scheduler thread admits queued requests by footprint, advances every
//    resident medium in chunks through its cached CUDA graphs on a pool of
//    non-blocking streams (two chunks in flight per request), and retires
//    finished requests (traces out, medium released).
// Work queue: every chunk launch enqueues the request's tiles (the CTAs of
// its sweeps) on its stream; the GPU's block scheduler hands free SM slots
// to the pending tiles of the highest-priority stream first.  The size-class
// policy (the default) uses three stream priorities: short requests (little
// work) at the top, so they never wait behind long ones; the oldest running
// long request in the middle, so the head of the long queue advances at
// nearly the speed it would have alone; the other long requests at the
// bottom, filling the slots the others leave idle.
// All device memory of the media comes from one arena allocated when the
// server is created, so admission is exact bookkeeping and releasing a
// medium never calls cudaFree (which would wait for the whole device).
#include "fw_internal.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace fwgb {
void set_thread_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *ctx);
}  // namespace fwgb

namespace {

// First-fit arena over one device allocation, 256-byte granules, free
// blocks coalesced on release.
class Arena {
public:
    int init(size_t bytes)
    {
        size_ = (bytes + 255) / 256 * 256;
        if (cudaMalloc(&base_, size_) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return FW_ERR_NOMEM;
        }
        free_[0] = size_;
        return FW_OK;
    }
    ~Arena()
    {
        if (base_) cudaFree(base_);
    }
    void *alloc(size_t n)
    {
        n = (n + 255) / 256 * 256;
        std::lock_guard<std::mutex> lk(mu_);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            used_[off] = n;
            return static_cast<char *>(base_) + off;
        }
        return nullptr;
    }
    void release(void *p)
    {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        const size_t off = (size_t)(static_cast<char *>(p) - static_cast<char *>(base_));
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t start = off, len = u->second;
        used_.erase(u);
        auto nx = free_.lower_bound(start);
        if (nx != free_.end() && nx->first == start + len) {
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == start) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = len;
    }
    size_t largest_free()
    {
        std::lock_guard<std::mutex> lk(mu_);
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    size_t size() const { return size_; }
    static void *alloc_cb(size_t n, void *ctx) { return static_cast<Arena *>(ctx)->alloc(n); }
    static void release_cb(void *p, void *ctx) { static_cast<Arena *>(ctx)->release(p); }

private:
    void *base_ = nullptr;
    size_t size_ = 0;
    std::mutex mu_;
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> used_;
};

struct Job {
    long long id = 0;
    fw_request r{};
    std::vector<fw_relax_params> classes;
    size_t footprint = 0;
    long long voxels = 0;
    double t_submit = 0, t_admit = -1;
    fw_medium *m = nullptr;
    int stream = 0;
    int level = -1;                // stream priority level of the chunks in flight
    bool short_job = false;        // voxels x steps <= the server's short_work
    int issued = 0;
    std::deque<cudaEvent_t> inflight;
    bool cancel = false;
    int skips = 0;
};

long long count_mask(const uint8_t *mask, size_t n)
{
    long long k = 0;
    for (size_t i = 0; i < n; ++i) k += mask[i] != 0;
    return k;
}

}  // namespace

struct fw_server {
    fw_server_opts o{};
    int device = 0;
    Arena arena;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_done, cv_work, cv_build;
    std::deque<Job *> queue;       // submitted, waiting for admission
    std::deque<Job *> to_build;    // admitted, waiting for the builder
    std::vector<Job *> ready;      // built, waiting for the scheduler
    std::map<long long, Job *> live;
    std::deque<fw_completion> done;
    size_t reserved = 0;
    int building = 0, n_active = 0, n_done = 0;
    bool stop = false;
    bool debug = false;            // FWGB_SERVER_DEBUG: log builds and failed chunks to stderr
    long long next_id = 1;
    std::vector<cudaStream_t> streams;        // kLevels x n_streams, level-major
    static constexpr int kLevels = 3;         // 0: short requests, 1: oldest long one, 2: other long ones
    std::thread sched, builder;
    cudaStream_t stream_of(int level, int k) const { return streams[(size_t)level * o.n_streams + k]; }

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    // caller holds mu
    void complete(Job *j, int status, float pmax)
    {
        fw_completion c{};
        c.id = j->id;
        c.tag = j->r.tag;
        c.status = status;
        c.t_submit = j->t_submit;
        c.t_admit = j->t_admit;
        c.t_done = now();
        c.voxel_steps = status == FW_OK || status == FW_ERR_UNSTABLE ? j->voxels * (long long)j->issued : 0;
        c.max_abs_p = pmax;
        done.push_back(c);
        ++n_done;
        live.erase(j->id);
        delete j;
        cv_done.notify_all();
        cv_work.notify_all();
    }

    void run_builder();
    void run_scheduler();
};

void fw_server::run_builder()
{
    cudaSetDevice(device);
    fwgb::set_thread_allocator(Arena::alloc_cb, Arena::release_cb, &arena);
    cudaStream_t bs = nullptr;
    cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    for (;;) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_build.wait(lk, [&] { return stop || !to_build.empty(); });
            if (to_build.empty()) break;
            j = to_build.front();
            to_build.pop_front();
            if (j->cancel || stop) {
                reserved -= j->footprint;
                complete(j, FW_CANCELLED, 0.f);
                continue;
            }
            ++building;
        }
        const fw_request &r = j->r;
        fw_medium *m = nullptr;
        int rc = fw_create_medium_classes(&r.grid, r.c, r.rho, r.beta, r.class_idx, j->classes.data(),
                                          (int)j->classes.size(), r.storage, bs, &m);
        if (!rc && r.src_mask) rc = fw_set_sources(m, r.src_mask, r.waveforms, r.n_wave, r.n_steps, r.wave_of);
        if (!rc && r.rcv_mask) rc = fw_set_receivers(m, r.rcv_mask, r.decim, r.n_steps);
        if (rc && m) {
            fw_destroy_medium(m);
            m = nullptr;
        }
        if (debug)
            std::fprintf(stderr, "[fw_server] built id=%lld tag=%lld grid %dx%dx%d rc=%d slab=%p bytes=%zu\n", j->id,
                         r.tag, r.grid.nx, r.grid.ny, r.grid.nz, rc, m ? m->slab : nullptr,
                         m ? m->slab_bytes : (size_t)0);
        std::lock_guard<std::mutex> lk(mu);
        --building;
        if (rc == FW_ERR_NOMEM && !stop && reserved > j->footprint) {
            // the arena is fragmented while others hold memory: retry when it frees up
            reserved -= j->footprint;
            j->t_admit = -1;
            j->skips = FW_SERVER_MAX_SKIPS + 1;
            queue.push_front(j);
        } else if (rc) {
            reserved -= j->footprint;
            complete(j, rc, 0.f);
        } else {
            j->m = m;
            ready.push_back(j);
        }
        cv_work.notify_all();
    }
    if (bs) cudaStreamDestroy(bs);
    fwgb::set_thread_allocator(nullptr, nullptr, nullptr);
}

void fw_server::run_scheduler()
{
    cudaSetDevice(device);
    fwgb::set_thread_allocator(Arena::alloc_cb, Arena::release_cb, &arena);
    std::vector<Job *> active;
    std::vector<cudaEvent_t> pool;
    int rr = 0;
    auto get_event = [&]() {
        cudaEvent_t e = nullptr;
        if (!pool.empty()) {
            e = pool.back();
            pool.pop_back();
        } else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
        }
        return e;
    };
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop && active.empty() && ready.empty() && to_build.empty() && building == 0) break;
            // admission: first fit in arrival order (short requests first
            // under the size-class policy); a request skipped too often
            // blocks the ones of its class behind it; long requests leave
            // two slots to short ones when there are four or more slots
            if (!stop) {
                const bool classes = o.policy == 0;
                int long_used = 0;
                for (Job *x : active) long_used += !x->short_job;
                for (Job *x : ready) long_used += !x->short_job;
                for (Job *x : to_build) long_used += !x->short_job;
                long_used += building;       // conservatively: builds in progress count as long
                const int long_cap = classes && o.max_active >= 4 ? o.max_active - 2 : o.max_active;
                for (int pass = classes ? 0 : 1; pass < 2; ++pass) {
                    for (auto it = queue.begin(); it != queue.end();) {
                        Job *j = *it;
                        if (j->cancel) {
                            it = queue.erase(it);
                            complete(j, FW_CANCELLED, 0.f);
                            continue;
                        }
                        if (classes && j->short_job != (pass == 0)) {
                            ++it;
                            continue;
                        }
                        const int slots = (int)(active.size() + ready.size() + to_build.size()) + building;
                        if (slots >= o.max_active) break;
                        if (classes && !j->short_job && long_used >= long_cap) break;
                        if (j->footprint <= o.hbm_budget - reserved) {
                            reserved += j->footprint;
                            j->t_admit = now();
                            long_used += !j->short_job;
                            to_build.push_back(j);
                            it = queue.erase(it);
                            cv_build.notify_one();
                            continue;
                        }
                        if (++j->skips > FW_SERVER_MAX_SKIPS) break;
                        ++it;
                    }
                }
            }
            for (Job *j : ready) {
                j->stream = rr++ % o.n_streams;
                active.push_back(j);
            }
            ready.clear();
            if (stop)
                for (Job *j : active) j->cancel = true;
            n_active = (int)active.size();
        }
        bool progress = false;
        // the oldest long request (lowest id) runs at the middle priority
        long long oldest_long = -1;
        for (Job *x : active)
            if (!x->short_job && (oldest_long < 0 || x->id < oldest_long)) oldest_long = x->id;
        for (size_t k = 0; k < active.size();) {
            Job *j = active[k];
            int status = FW_OK;
            bool finished = false;
            while (!j->inflight.empty()) {
                const cudaError_t q = cudaEventQuery(j->inflight.front());
                if (q == cudaErrorNotReady) break;
                pool.push_back(j->inflight.front());
                j->inflight.pop_front();
                progress = true;
                if (q != cudaSuccess) {
                    // a failed chunk: the request ends with the error once its
                    // other chunks are out of the way
                    if (debug) {
                        std::fprintf(stderr, "[fw_server] chunk of id=%lld tag=%lld failed (%s); in flight:\n", j->id,
                                     j->r.tag, cudaGetErrorString(q));
                        for (Job *x : active)
                            std::fprintf(stderr, "[fw_server]   id=%lld tag=%lld grid %dx%dx%d issued %d/%d stream %d\n",
                                         x->id, x->r.tag, x->r.grid.nx, x->r.grid.ny, x->r.grid.nz, x->issued,
                                         x->r.n_steps, x->stream);
                    }
                    cudaGetLastError();
                    cudaStreamSynchronize(stream_of(j->level < 0 ? 1 : j->level, j->stream));
                    if (!j->inflight.empty()) cudaEventSynchronize(j->inflight.back());
                    for (cudaEvent_t x : j->inflight) pool.push_back(x);
                    j->inflight.clear();
                    finished = true;
                    status = FW_ERR_CUDA;
                }
            }
            if (!finished && j->inflight.empty() && (j->cancel || j->issued >= j->r.n_steps)) {
                finished = true;
                status = j->cancel ? FW_CANCELLED : FW_OK;
            }
            while (!finished && !j->cancel && j->issued < j->r.n_steps && j->inflight.size() < 2) {
                const int n = std::min(o.chunk_steps, j->r.n_steps - j->issued);
                const int level = o.policy != 0 ? 1 : (j->short_job ? 0 : (j->id == oldest_long ? 1 : 2));
                cudaStream_t st = stream_of(level, j->stream);
                int rc = FW_OK;
                // a request that changes level: its next chunk waits for the last one queued
                if (j->level >= 0 && level != j->level && !j->inflight.empty() &&
                    cudaStreamWaitEvent(st, j->inflight.back(), 0) != cudaSuccess)
                    rc = FW_ERR_CUDA;
                j->level = level;
                if (!rc) rc = fw_run(j->m, n, st);
                cudaEvent_t e = rc ? nullptr : get_event();
                if (!rc && (!e || cudaEventRecord(e, st) != cudaSuccess)) rc = FW_ERR_CUDA;
                if (rc) {
                    if (e) pool.push_back(e);
                    // the chunks already queued must end before the medium goes
                    cudaGetLastError();
                    cudaStreamSynchronize(st);
                    if (!j->inflight.empty()) cudaEventSynchronize(j->inflight.back());
                    for (cudaEvent_t x : j->inflight) pool.push_back(x);
                    j->inflight.clear();
                    finished = true;
                    status = rc;
                    break;
                }
                j->inflight.push_back(e);
                j->issued += n;
                progress = true;
            }
            if (!finished) {
                ++k;
                continue;
            }
            float pmax = 0.f;
            if (status == FW_OK) {
                status = fw_status(j->m, &pmax);
                if ((status == FW_OK || status == FW_ERR_UNSTABLE) && j->r.traces_out && j->m->n_rcv > 0) {
                    int rc = fw_read_receivers(j->m, j->r.traces_out, 0, stream_of(j->level < 0 ? 1 : j->level,
                                                                                 j->stream));
                    if (rc) status = rc;
                }
            }
            fw_destroy_medium(j->m);
            j->m = nullptr;
            {
                std::lock_guard<std::mutex> lk(mu);
                reserved -= j->footprint;
                complete(j, status, pmax);
            }
            active.erase(active.begin() + k);
            progress = true;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    fwgb::set_thread_allocator(nullptr, nullptr, nullptr);
}

extern "C" {

int fw_server_create(const fw_server_opts *opts, fw_server **out)
{
    if (!opts || !out || opts->hbm_budget == 0 || opts->max_active < 1 || opts->chunk_steps < 1 ||
        opts->n_streams < 1 || (opts->policy != 0 && opts->policy != 1) || !(opts->short_work >= 0.0))
        return FW_ERR_ARG;
    *out = nullptr;
    fw_server *s = new (std::nothrow) fw_server();
    if (!s) return FW_ERR_NOMEM;
    s->o = *opts;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return FW_ERR_CUDA;
    }
    int rc = s->arena.init(opts->hbm_budget);
    if (rc) {
        delete s;
        return rc;
    }
    s->o.hbm_budget = s->arena.size();
    if (s->o.short_work <= 0.0) s->o.short_work = 5e9;
    const char *dbg = std::getenv("FWGB_SERVER_DEBUG");
    s->debug = dbg && *dbg && *dbg != '0';
    // stream priorities of the three levels: greatest, middle, least of the
    // device's range (all equal where the device has one level)
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    const int prio[fw_server::kLevels] = {greatest, (least + greatest) / 2, least};
    for (int lv = 0; lv < fw_server::kLevels; ++lv)
        for (int k = 0; k < opts->n_streams; ++k) {
            cudaStream_t st = nullptr;
            if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio[lv]) != cudaSuccess) {
                cudaGetLastError();
                for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
                delete s;
                return FW_ERR_CUDA;
            }
            s->streams.push_back(st);
        }
    s->t0 = std::chrono::steady_clock::now();
    s->builder = std::thread([s] { s->run_builder(); });
    s->sched = std::thread([s] { s->run_scheduler(); });
    *out = s;
    return FW_OK;
}

int fw_server_submit(fw_server *s, const fw_request *req, long long *id)
{
    if (!s || !req) return FW_ERR_ARG;
    const fw_request &r = *req;
    if (!r.c || !r.rho || !r.class_idx || !r.classes || r.n_classes < 1 || r.n_steps < 1 || r.decim < 1 ||
        (r.storage != FW_STORE_F32 && r.storage != FW_STORE_BF16 && r.storage != FW_STORE_F16))
        return FW_ERR_ARG;
    size_t bytes = 0;
    int rc = fw_medium_bytes(&r.grid, r.classes[0].n_mech, r.storage, r.beta != nullptr, &bytes);
    if (rc) return rc;
    Job *j = new (std::nothrow) Job();
    if (!j) return FW_ERR_NOMEM;
    j->r = r;
    j->classes.assign(r.classes, r.classes + r.n_classes);
    const size_t n = (size_t)r.grid.nx * r.grid.ny * r.grid.nz;
    j->voxels = (long long)n;
    j->short_job = (double)n * (double)r.n_steps <= s->o.short_work;
    const long long n_src = r.src_mask ? count_mask(r.src_mask, n) : 0;
    const long long n_rcv = r.rcv_mask ? count_mask(r.rcv_mask, n) : 0;
    const long long n_rec = (r.n_steps + r.decim - 1) / r.decim;
    // medium + upload staging (one dense map and the beta map at most) +
    // source and receiver buffers, each rounded to the arena's granule
    const size_t padded = (size_t)((r.grid.nx + 31) / 32 * 32) * r.grid.ny * r.grid.nz;
    j->footprint = bytes + padded * 8 + (size_t)n_src * 16 + (size_t)r.n_wave * r.n_steps * 8 +
                   (size_t)n_rcv * (8 + 4 * n_rec) + (16u << 20);
    std::lock_guard<std::mutex> lk(s->mu);
    j->id = s->next_id++;
    j->t_submit = s->now();
    if (id) *id = j->id;
    s->live[j->id] = j;
    if (j->footprint > s->o.hbm_budget) {
        s->complete(j, FW_ERR_NOMEM, 0.f);
        return FW_OK;
    }
    s->queue.push_back(j);
    s->cv_work.notify_all();
    return FW_OK;
}

int fw_server_poll(fw_server *s, fw_completion *out, int max, int *n, double timeout_s)
{
    if (!s || (max > 0 && !out) || !n) return FW_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_s > 0)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    return FW_OK;
}

int fw_server_cancel(fw_server *s, long long id)
{
    if (!s) return FW_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->live.find(id);
    if (it == s->live.end()) return FW_ERR_ARG;
    Job *j = it->second;
    auto q = std::find(s->queue.begin(), s->queue.end(), j);
    if (q != s->queue.end()) {
        s->queue.erase(q);
        s->complete(j, FW_CANCELLED, 0.f);
    } else {
        j->cancel = true;
        s->cv_work.notify_all();
    }
    return FW_OK;
}

int fw_server_stats_get(fw_server *s, fw_server_stats *st)
{
    if (!s || !st) return FW_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    st->queued = (int)s->queue.size();
    st->building = (int)s->to_build.size() + s->building;
    st->active = s->n_active + (int)s->ready.size();
    st->done = s->n_done;
    st->bytes_reserved = s->reserved;
    st->bytes_budget = s->o.hbm_budget;
    st->bytes_largest_free = s->arena.largest_free();
    return FW_OK;
}

double fw_server_now(fw_server *s) { return s ? s->now() : 0.0; }

void fw_server_destroy(fw_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        while (!s->queue.empty()) {
            Job *j = s->queue.front();
            s->queue.pop_front();
            s->complete(j, FW_CANCELLED, 0.f);
        }
        s->cv_build.notify_all();
        s->cv_work.notify_all();
    }
    if (s->builder.joinable()) s->builder.join();
    if (s->sched.joinable()) s->sched.join();
    for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
    delete s;
}

}  // extern "C"
