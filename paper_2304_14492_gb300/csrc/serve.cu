// Serving: continuous batching of moment requests on one GPU.
//
// Requests (host images) arrive at any time.  A scheduler thread admits
// waiting requests, in arrival order, while their device bytes fit a fixed
// arena (the HBM budget, allocated once), groups the admitted ones by polar
// grid, and launches each group on the stream bound to that grid: host->device
// copy, resampling, ring FFT, projection, device->host copy.  Where the GPU
// reads pageable host memory through the host page tables (GB300: NVLink-C2C
// with ATS), a kernel gathers each host image straight into the arena and
// scatters each result straight into the caller's `out`; elsewhere the copies
// go through a pinned mirror of the arena.  Groups of different grids run
// concurrently; requests
// that arrive meanwhile are admitted as soon as earlier ones complete and free
// their bytes.  Plans stay resident; a grid's plan is rebuilt only when a
// request needs a larger order than any seen before for it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "zm_internal.cuh"

namespace zm {

using Clock = std::chrono::steady_clock;

// host image rows (any pitch, pageable memory the GPU reads through the host
// page tables) -> packed rows in the device arena
__global__ void k_host_rows_in(const float* __restrict__ src, long long pitch, int h, int w, float* __restrict__ dst) {
    const long long n = (long long)h * w;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long y = e / w, x = e - y * w;
        dst[e] = src[y * pitch + x];
    }
}

// device result -> the caller's host buffer (pageable, through the host page tables)
__global__ void k_host_out(const float* __restrict__ src, int n, float* __restrict__ dst) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) dst[e] = src[e];
}

struct SrvRequest {
    unsigned long long ticket = 0;
    const float* image = nullptr;
    int h = 0, w = 0;
    long long pitch = 0;
    int n_max = 0, n_rho = 0, n_theta = 0;
    float* out = nullptr;
    unsigned flags = 0;
    Clock::time_point t_submit;
    // arena block once admitted: the image, then the request's own result slot
    // (used in the pinned mirror only)
    size_t off = 0, img_bytes = 0, out_bytes = 0;
};

// First-fit allocator over [0, size) in 256-byte units (host bookkeeping only).
struct Arena {
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;      // offset -> length
    void init(size_t n) {
        size = n;
        free_.clear();
        free_[0] = n;
    }
    static size_t round(size_t n) { return (n + 255) & ~(size_t)255; }
    bool alloc(size_t n, size_t* off) {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used += n;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round(n);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// A plan for one polar grid with its group moment buffer ([max_group][P][2],
// device); in-flight groups keep it alive.  Groups of one grid run in order
// on one stream, so they share the plan's workspaces and this buffer safely.
struct GridPlan {
    zm_plan_t plan = nullptr;
    int n_max = -1;
    float* out = nullptr;
    ~GridPlan() {
        if (out) cudaFree(out);
        if (plan) zm_plan_destroy(plan);
    }
};

struct SrvGroup {
    std::vector<SrvRequest> reqs;
    std::shared_ptr<GridPlan> gp;
    int stream = 0;
    cudaEvent_t done = nullptr;
};

// Groups one stream may have in flight: the next group's copies overlap the
// current one's kernels; anything beyond waits and joins a later, larger group.
constexpr int SRV_INFLIGHT_PER_STREAM = 2;

}  // namespace zm

struct zm_server_s {
    int device = 0;
    zm_server_config_t cfg{};
    uint8_t* dev = nullptr;              // device arena
    uint8_t* pinned = nullptr;           // pinned host mirror of the arena
    zm::Arena arena;
    std::vector<cudaStream_t> streams;
    std::map<std::pair<int, int>, std::shared_ptr<zm::GridPlan>> plans;   // (n_rho, n_theta)
    std::map<std::pair<int, int>, int> stream_of;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<zm::SrvRequest> incoming, waiting;
    std::vector<zm::SrvRequest> admitted;
    std::deque<zm::SrvGroup> inflight;
    std::vector<char> done;              // by ticket
    bool host_direct = false;            // kernels read / write the callers' host buffers
    unsigned long long next_ticket = 1;
    zm_server_stats_t st{};
    std::vector<double> lat_ms;
    zm::Clock::time_point t_first{}, t_last{};
    bool have_first = false, stop = false;
    int error = ZM_OK;
    std::thread worker;
};

namespace zm {

static int launch_group(zm_server_t s, SrvGroup& g, cudaStream_t st) {
    const int gb = (int)g.reqs.size();
    std::vector<zm_image_t> imgs(gb);
    for (int j = 0; j < gb; ++j) {
        const SrvRequest& r = g.reqs[j];
        float* d = reinterpret_cast<float*>(s->dev + r.off);
        if (s->host_direct) {
            // the GPU gathers the host rows itself (no CPU copy)
            const long long n = (long long)r.h * r.w;
            const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
            k_host_rows_in<<<blocks, 256, 0, st>>>(r.image, r.pitch, r.h, r.w, d);
            ZM_LAUNCH_CHECK("k_host_rows_in");
        } else {
            // host image -> pinned mirror -> device arena (rows packed, pitch = width)
            float* ph = reinterpret_cast<float*>(s->pinned + r.off);
            for (int y = 0; y < r.h; ++y)
                memcpy(ph + (size_t)y * r.w, r.image + (size_t)y * r.pitch, sizeof(float) * r.w);
            ZM_CUDA_TRY(cudaMemcpyAsync(d, ph, r.img_bytes, cudaMemcpyHostToDevice, st));
        }
        imgs[j] = zm_image_t{d, r.h, r.w, r.w, 0.f, 0.f, -1.f};
    }
    zm_plan_t p = g.gp->plan;
    const int P = num_moments(g.gp->n_max);
    const int rc = launch_moments(p, imgs.data(), nullptr, gb, g.gp->out, nullptr, g.reqs[0].flags, st);
    if (rc != ZM_OK) return rc;
    for (int j = 0; j < gb; ++j) {
        const SrvRequest& r = g.reqs[j];
        const float* src = g.gp->out + (size_t)j * P * 2;
        if (s->host_direct) {
            const int n = (int)(r.out_bytes / sizeof(float));
            k_host_out<<<(n + 255) / 256, 256, 0, st>>>(src, n, r.out);
            ZM_LAUNCH_CHECK("k_host_out");
        } else {
            ZM_CUDA_TRY(cudaMemcpyAsync(s->pinned + r.off + r.img_bytes, src, r.out_bytes, cudaMemcpyDeviceToHost, st));
        }
    }
    ZM_CUDA_TRY(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
    ZM_CUDA_TRY(cudaEventRecord(g.done, st));
    return ZM_OK;
}

// Plan for a grid that covers order n_max (rebuilt only when n_max grows).
// A build (table, weights, workspace; it ends in a device synchronisation)
// runs with the server lock released, so submitters are not held up by it;
// only this scheduler thread reads or changes the plan map.
static int grid_plan(zm_server_t s, int n_rho, int n_theta, int n_max, std::shared_ptr<GridPlan>* out,
                     std::unique_lock<std::mutex>& lk) {
    auto key = std::make_pair(n_rho, n_theta);
    auto it = s->plans.find(key);
    if (it != s->plans.end() && it->second->n_max >= n_max) {
        *out = it->second;
        return ZM_OK;
    }
    lk.unlock();
    struct Relock {
        std::unique_lock<std::mutex>& l;
        ~Relock() { l.lock(); }
    } relock{lk};
    auto gp = std::make_shared<GridPlan>();
    int rc = zm_plan(&gp->plan, n_max, n_rho, n_theta, s->cfg.plan_flags);
    if (rc == ZM_OK) rc = zm_plan_reserve(gp->plan, s->cfg.max_group);
    if (rc == ZM_OK) {
        const cudaError_t e =
            cudaMalloc(&gp->out, sizeof(float) * 2 * (size_t)num_moments(n_max) * s->cfg.max_group);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMalloc(server group buffer)");
    }
    if (rc != ZM_OK) return rc;
    gp->n_max = n_max;
    s->plans[key] = gp;
    *out = gp;
    return ZM_OK;
}

// One scheduler pass (called with s->mu held through lk, which a plan build
// releases for its duration): retire finished groups, admit waiting requests
// in arrival order while they fit, launch admitted requests grouped by grid
// and flags.  Returns true if anything happened.
static bool schedule_once(zm_server_t s, std::unique_lock<std::mutex>& lk) {
    bool acted = false;
    // 1. completions (groups retire in any order)
    for (auto it = s->inflight.begin(); it != s->inflight.end();) {
        const cudaError_t q = cudaEventQuery(it->done);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        if (q != cudaSuccess) s->error = cuda_error(q, "server group");
        const auto now = Clock::now();
        for (const SrvRequest& r : it->reqs) {
            if (!s->host_direct) memcpy(r.out, s->pinned + r.off + r.img_bytes, r.out_bytes);
            s->arena.release(r.off, r.img_bytes + r.out_bytes);
            s->done[r.ticket] = 1;
            s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
            ++s->st.completed;
        }
        s->t_last = now;
        cudaEventDestroy(it->done);
        it = s->inflight.erase(it);
        acted = true;
    }
    if (acted) s->cv_done.notify_all();
    // 2. admission by budget, first come first served
    while (!s->waiting.empty()) {
        SrvRequest& r = s->waiting.front();
        size_t off;
        if (!s->arena.alloc(r.img_bytes + r.out_bytes, &off)) break;
        r.off = off;
        s->admitted.push_back(r);
        s->waiting.pop_front();
        acted = true;
    }
    // 3. launch admitted requests, grouped by (grid, flags), in order of first
    //    arrival, on the stream bound to the grid while it has room
    std::vector<int> busy(s->streams.size(), 0);
    for (auto& g : s->inflight) ++busy[g.stream];
    std::vector<SrvRequest> keep;
    std::vector<char> taken(s->admitted.size(), 0);
    for (size_t h = 0; h < s->admitted.size(); ++h) {
        if (taken[h]) continue;
        const SrvRequest head = s->admitted[h];
        const auto key = std::make_pair(head.n_rho, head.n_theta);
        auto so = s->stream_of.find(key);
        if (so == s->stream_of.end())
            so = s->stream_of.emplace(key, (int)s->stream_of.size() % (int)s->streams.size()).first;
        const int sidx = so->second;
        if (busy[sidx] >= SRV_INFLIGHT_PER_STREAM) continue;
        std::vector<size_t> members;
        for (size_t j = h; j < s->admitted.size() && (int)members.size() < s->cfg.max_group; ++j) {
            const SrvRequest& r = s->admitted[j];
            if (!taken[j] && r.n_rho == head.n_rho && r.n_theta == head.n_theta && r.flags == head.flags)
                members.push_back(j);
        }
        // batching window: hold a partial group while its oldest request is
        // younger than max_wait_us and more requests can still be admitted
        if (s->cfg.max_wait_us > 0 && (int)members.size() < s->cfg.max_group && s->waiting.empty() && !s->stop) {
            const double age_us = std::chrono::duration<double, std::micro>(Clock::now() - head.t_submit).count();
            if (age_us < s->cfg.max_wait_us) continue;
        }
        SrvGroup g;
        g.stream = sidx;
        int n_max = 0;
        for (size_t j : members) {
            taken[j] = 1;
            g.reqs.push_back(s->admitted[j]);
            n_max = std::max(n_max, s->admitted[j].n_max);
        }
        int rc = grid_plan(s, head.n_rho, head.n_theta, n_max, &g.gp, lk);
        if (rc == ZM_OK) rc = launch_group(s, g, s->streams[sidx]);
        if (rc != ZM_OK) {
            s->error = rc;
            return true;
        }
        ++busy[sidx];
        ++s->st.groups_launched;
        s->inflight.push_back(std::move(g));
        acted = true;
    }
    for (size_t j = 0; j < s->admitted.size(); ++j)
        if (!taken[j]) keep.push_back(s->admitted[j]);
    s->admitted.swap(keep);
    return acted;
}

static void scheduler(zm_server_t s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        while (!s->incoming.empty()) {
            s->waiting.push_back(s->incoming.front());
            s->incoming.pop_front();
        }
        if (s->error != ZM_OK) {
            // after an error nothing new is launched; waiters see the status
            s->waiting.clear();
            s->admitted.clear();
        }
        const bool acted = schedule_once(s, lk);
        const bool idle = s->incoming.empty() && s->waiting.empty() && s->admitted.empty() && s->inflight.empty();
        if (s->stop && idle) break;
        if (!acted) {
            // nothing to launch or retire: sleep until a submission, or poll the
            // in-flight groups again shortly
            const bool poll = !s->inflight.empty() || !s->admitted.empty();
            s->cv_work.wait_for(lk, std::chrono::microseconds(poll ? 20 : 2000));
        }
    }
}

}  // namespace zm

using namespace zm;

extern "C" int zm_server_create(zm_server_t* server, const zm_server_config_t* config) {
    if (!server) return set_error(ZM_EINVAL, "server pointer is NULL");
    *server = nullptr;
    auto* s = new zm_server_s();
    if (config) s->cfg = *config;
    if (s->cfg.hbm_budget == 0) s->cfg.hbm_budget = 1ull << 30;
    if (s->cfg.streams <= 0) s->cfg.streams = 4;
    if (s->cfg.max_group <= 0) s->cfg.max_group = 64;
    int rc = ZM_OK;
    if (cudaGetDevice(&s->device) != cudaSuccess) rc = set_error(ZM_ECUDA, "no CUDA device");
    if (rc == ZM_OK) {
        // direct host access needs pageable memory reached through the host page
        // tables; ZM_SERVER_STAGING=1 keeps the pinned-mirror copies anyway
        int pageable = 0, host_tables = 0;
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, s->device);
        cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, s->device);
        const char* force = getenv("ZM_SERVER_STAGING");
        s->host_direct = pageable && host_tables && !(force && force[0] == '1');
    }
    const size_t n = Arena::round(s->cfg.hbm_budget);
    if (rc == ZM_OK) {
        cudaError_t e = cudaMalloc(&s->dev, n);
        if (e == cudaSuccess && !s->host_direct) e = cudaHostAlloc(&s->pinned, n, cudaHostAllocDefault);
        for (int k = 0; k < s->cfg.streams && e == cudaSuccess; ++k) {
            cudaStream_t st;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e == cudaSuccess) s->streams.push_back(st);
        }
        if (e != cudaSuccess) rc = cuda_error(e, "server set-up");
    }
    if (rc != ZM_OK) {
        for (auto st : s->streams) cudaStreamDestroy(st);
        if (s->pinned) cudaFreeHost(s->pinned);
        if (s->dev) cudaFree(s->dev);
        delete s;
        return rc;
    }
    s->arena.init(n);
    s->done.assign(1, 0);
    s->worker = std::thread(scheduler, s);
    *server = s;
    return ZM_OK;
}

extern "C" int zm_server_submit(zm_server_t s, const float* image, int height, int width, long long pitch,
                                int n_max, int n_rho, int n_theta, float* out, unsigned flags,
                                unsigned long long* ticket) {
    if (!s || !image || !out || !ticket) return set_error(ZM_EINVAL, "NULL argument");
    if (height < 1 || width < 1 || pitch < width) return set_error(ZM_EINVAL, "bad image size / pitch");
    if (n_max < 0 || n_rho < 1 || n_theta < 8 || (n_theta & (n_theta - 1)) || n_theta > 2048 ||
        n_theta < 2 * n_max + 1)
        return set_error(ZM_EINVAL, "bad order / grid (n_max %d, n_rho %d, n_theta %d)", n_max, n_rho, n_theta);
    if (flags & ~ZM_NEUMANN) return set_error(ZM_EINVAL, "unknown flags 0x%x", flags);
    SrvRequest r;
    r.image = image;
    r.h = height;
    r.w = width;
    r.pitch = pitch;
    r.n_max = n_max;
    r.n_rho = n_rho;
    r.n_theta = n_theta;
    r.out = out;
    r.flags = flags;
    r.img_bytes = Arena::round(sizeof(float) * (size_t)height * width);
    r.out_bytes = sizeof(float) * 2 * (size_t)num_moments(n_max);
    r.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error != ZM_OK) return set_error(s->error, "the server stopped after an error");
    if (Arena::round(r.img_bytes + r.out_bytes) > s->arena.size) {
        ++s->st.rejected;
        return set_error(ZM_ENOMEM, "request of %zu bytes exceeds the budget", r.img_bytes + r.out_bytes);
    }
    r.ticket = s->next_ticket++;
    s->done.push_back(0);
    if (!s->have_first) {
        s->t_first = r.t_submit;
        s->have_first = true;
    }
    ++s->st.submitted;
    s->incoming.push_back(r);
    *ticket = r.ticket;
    s->cv_work.notify_one();
    return ZM_OK;
}

extern "C" int zm_server_poll(zm_server_t s, unsigned long long ticket, int* done) {
    if (!s || !done) return set_error(ZM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) return set_error(ZM_EINVAL, "unknown ticket");
    *done = s->done[ticket] ? 1 : 0;
    return s->error;
}

extern "C" int zm_server_wait(zm_server_t s, unsigned long long ticket, double timeout_s) {
    if (!s) return set_error(ZM_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) return set_error(ZM_EINVAL, "unknown ticket");
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] { return s->done[ticket] || s->error != ZM_OK; });
    if (s->error != ZM_OK) return set_error(s->error, "the server stopped after an error");
    return ok ? ZM_OK : set_error(ZM_ETIMEOUT, "ticket %llu not done after %.3f s", ticket, timeout_s);
}

extern "C" int zm_server_drain(zm_server_t s, double timeout_s) {
    if (!s) return set_error(ZM_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        return s->st.completed == s->st.submitted || s->error != ZM_OK;
    });
    if (s->error != ZM_OK) return set_error(s->error, "the server stopped after an error");
    return ok ? ZM_OK : set_error(ZM_ETIMEOUT, "not drained after %.3f s", timeout_s);
}

extern "C" int zm_server_stats(zm_server_t s, zm_server_stats_t* out) {
    if (!s || !out) return set_error(ZM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    std::vector<double> l = s->lat_ms;
    std::sort(l.begin(), l.end());
    auto q = [&](double f) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(f * l.size()))]; };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    out->max_ms = l.empty() ? 0.0 : l.back();
    const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
    out->images_per_s = (span > 0 && s->st.completed) ? s->st.completed / span : 0.0;
    out->peak_bytes = s->arena.peak;
    out->host_direct = s->host_direct ? 1 : 0;
    return ZM_OK;
}

extern "C" int zm_server_reset_stats(zm_server_t s) {
    if (!s) return set_error(ZM_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->st.completed != s->st.submitted || !s->incoming.empty())
        return set_error(ZM_EINVAL, "requests are in flight: drain the server before resetting its statistics");
    s->st = zm_server_stats_t{};
    s->lat_ms.clear();
    s->have_first = false;
    s->arena.peak = s->arena.used;
    return ZM_OK;
}

extern "C" int zm_server_destroy(zm_server_t s, double timeout_s) {
    if (!s) return ZM_OK;
    int rc = zm_server_drain(s, timeout_s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        if (rc != ZM_OK) {
            // undrained work is dropped: the scheduler retires what is on the GPU
            s->incoming.clear();
            s->waiting.clear();
            s->admitted.clear();
        }
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    DeviceGuard dg(s->device);
    cudaDeviceSynchronize();
    for (auto& g : s->inflight) cudaEventDestroy(g.done);
    s->inflight.clear();
    s->plans.clear();
    for (auto st : s->streams) cudaStreamDestroy(st);
    cudaFreeHost(s->pinned);
    cudaFree(s->dev);
    delete s;
    return rc;
}
