// Uneven batches: images of different sizes, orders and polar grids in one
// CUDA-graph launch.
//
// Requests are grouped by polar grid (N_rho, N_theta).  Each group has one plan
// whose order is the group's largest: the moments of a request of order n are
// the first P(n) moments of its group's (Z_nm depends on n, m and the grid, not
// on the plan's n_max).  A group runs the ordinary path (resampling, ring FFT,
// projection into a group buffer); one small kernel then copies every
// request's prefix into its own output.  The whole sequence is captured once
// into a CUDA graph and replayed while the request pointers stay the same;
// the groups fork onto BATCH_BRANCHES side streams (balanced by pixel count),
// so they become parallel branches of the graph and small groups overlap.
// Launch choices per group come from a small autotuner (timed candidates,
// cached in a JSON file).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "zm_internal.cuh"

namespace zm {

struct CopyDesc {
    const float* src;    // group buffer row of this request
    float* dst;          // request output
    int n;               // floats to copy (2 P(n_max))
};

struct BatchGroup {
    int n_rho = 0, n_theta = 0, n_max = 0;
    zm_plan_t plan = nullptr;
    std::vector<int> members;          // request indices, sorted by geometry
    float* out_buf = nullptr;          // [members][P(n_max)][2]
};

constexpr int BATCH_BRANCHES = 4;      // side streams the groups fork onto

}  // namespace zm

struct zm_batch_s {
    int device = 0;
    cudaStream_t side[zm::BATCH_BRANCHES] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[zm::BATCH_BRANCHES] = {};
    std::vector<int> branch;           // side stream of each group
    unsigned plan_flags = 0;
    std::vector<zm_request_t> reqs;    // shapes (and pointers) at creation
    std::vector<zm::BatchGroup> groups;
    zm::CopyDesc* d_copy = nullptr;    // [count]
    cudaStream_t cap = nullptr;        // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<zm_request_t> captured;
    unsigned captured_flags = 0;
    int captures = 0;
};

namespace zm {

// copy each request's prefix out of its group buffer (one CTA per request)
__global__ void k_batch_copy(const CopyDesc* __restrict__ d) {
    const CopyDesc c = d[blockIdx.x];
    for (int e = threadIdx.x; e < c.n; e += blockDim.x) c.dst[e] = c.src[e];
}

static bool same_shape(const zm_request_t& a, const zm_request_t& b) {
    return a.n_max == b.n_max && a.n_rho == b.n_rho && a.n_theta == b.n_theta && same_geometry(a.image, b.image);
}

static bool same_pointers(const zm_request_t& a, const zm_request_t& b) {
    return a.image.data == b.image.data && a.image.pitch == b.image.pitch && a.out == b.out;
}

static int check_requests(const zm_request_t* reqs, int count) {
    if (count < 1 || !reqs) return set_error(ZM_EINVAL, "empty request list");
    for (int r = 0; r < count; ++r) {
        const zm_request_t& q = reqs[r];
        int s = check_images(&q.image, 1);
        if (s != ZM_OK) return set_error(s, "request %d: %s", r, zm_last_error());
        if (!q.out) return set_error(ZM_EINVAL, "request %d: out is NULL", r);
        if (q.n_max < 0 || q.n_rho < 1 || q.n_theta < 8 || (q.n_theta & (q.n_theta - 1)) || q.n_theta > 2048 ||
            q.n_theta < 2 * q.n_max + 1)
            return set_error(ZM_EINVAL, "request %d: bad order / grid (n_max %d, n_rho %d, n_theta %d)", r, q.n_max,
                             q.n_rho, q.n_theta);
    }
    return ZM_OK;
}

static void free_batch(zm_batch_t b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int k = 0; k < BATCH_BRANCHES; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->d_copy) cudaFree(b->d_copy);
    for (auto& g : b->groups) {
        if (g.out_buf) cudaFree(g.out_buf);
        if (g.plan) zm_plan_destroy(g.plan);
    }
    delete b;
}

}  // namespace zm

namespace zm {

// The whole batch from stream st: the groups fork onto the side streams (per
// group resampling + ring FFT + projection into its buffer), join back on st,
// then the prefix copies.
static int enqueue_batch(zm_batch_t b, const zm_request_t* reqs, unsigned flags, cudaStream_t st) {
    std::vector<zm_image_t> imgs;
    ZM_CUDA_TRY(cudaEventRecord(b->ev_fork, st));
    for (int k = 0; k < BATCH_BRANCHES; ++k) ZM_CUDA_TRY(cudaStreamWaitEvent(b->side[k], b->ev_fork, 0));
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        auto& g = b->groups[gi];
        imgs.clear();
        for (int r : g.members) imgs.push_back(reqs[r].image);
        const int gb = (int)g.members.size();
        const int s = launch_moments(g.plan, imgs.data(), nullptr, gb, g.out_buf, nullptr, flags,
                                     b->side[b->branch[gi]]);
        if (s != ZM_OK) return s;
    }
    for (int k = 0; k < BATCH_BRANCHES; ++k) {
        ZM_CUDA_TRY(cudaEventRecord(b->ev_join[k], b->side[k]));
        ZM_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_join[k], 0));
    }
    k_batch_copy<<<(unsigned)b->reqs.size(), 256, 0, st>>>(b->d_copy);
    ZM_LAUNCH_CHECK("k_batch_copy");
    return ZM_OK;
}

static int upload_copies(zm_batch_t b, const zm_request_t* reqs) {
    std::vector<CopyDesc> h(b->reqs.size());
    for (auto& g : b->groups) {
        const int P = num_moments(g.n_max);
        for (size_t j = 0; j < g.members.size(); ++j) {
            const int r = g.members[j];
            h[r] = CopyDesc{g.out_buf + (size_t)j * P * 2, reqs[r].out, 2 * num_moments(reqs[r].n_max)};
        }
    }
    ZM_CUDA_TRY(cudaMemcpy(b->d_copy, h.data(), sizeof(CopyDesc) * h.size(), cudaMemcpyHostToDevice));
    return ZM_OK;
}

// ------------------------------------------------------------------ autotuner
// Choices for one group: resampling path, rings per CTA of the ring FFT, and
// the projection's CTAs-per-SM target for its radial split.  Results are kept
// in a flat JSON object, one entry per line:
//   "key": {"gather": g, "rings": r, "split": s, "us": t},
struct TuneChoice {
    int gather = 0, rings = 0, split = 0;
    double us = 0;
};

static std::mutex g_tune_mu;

static std::string tune_key(zm_plan_t p, int batch, const GeoImage& g) {
    cudaDeviceProp prop;
    int major = 0, minor = 0;
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) {
        major = prop.major;
        minor = prop.minor;
    }
    int bb = 1;
    while (bb < batch) bb <<= 1;
    char buf[256];
    snprintf(buf, sizeof buf, "sm%d%d|nrho=%d|ntheta=%d|nmax=%d|batch=%d|prec=%d|grid=%d|img=%dx%d", major, minor,
             p->n_rho, p->n_theta, p->n_max, bb, p->prec, p->grid, g.h, g.w);
    return buf;
}

static std::map<std::string, TuneChoice> read_tune_cache(const char* path) {
    std::map<std::string, TuneChoice> out;
    FILE* f = path ? fopen(path, "r") : nullptr;
    if (!f) return out;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        char key[512];
        TuneChoice c;
        if (sscanf(line, " \"%511[^\"]\": {\"gather\": %d, \"rings\": %d, \"split\": %d, \"us\": %lf", key, &c.gather,
                   &c.rings, &c.split, &c.us) == 5)
            out[key] = c;
    }
    fclose(f);
    return out;
}

static void write_tune_cache(const char* path, const std::map<std::string, TuneChoice>& m) {
    if (!path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t k = 0;
    for (auto& e : m) {
        fprintf(f, "  \"%s\": {\"gather\": %d, \"rings\": %d, \"split\": %d, \"us\": %.3f}%s\n", e.first.c_str(),
                e.second.gather, e.second.rings, e.second.split, e.second.us, ++k < m.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

// Time one group's resampling + ring FFT + projection under the current plan
// choices (mean of three runs after one warm-up), in microseconds.
static int time_group(zm_batch_t b, BatchGroup& g, const zm_request_t* reqs, double* us) {
    std::vector<zm_image_t> imgs;
    for (int r : g.members) imgs.push_back(reqs[r].image);
    const int gb = (int)g.members.size();
    cudaEvent_t e0, e1;
    ZM_CUDA_TRY(cudaEventCreate(&e0));
    ZM_CUDA_TRY(cudaEventCreate(&e1));
    int s = ZM_OK;
    for (int it = 0; it < 4 && s == ZM_OK; ++it) {
        if (it == 1) cudaEventRecord(e0, b->cap);
        s = launch_moments(g.plan, imgs.data(), nullptr, gb, g.out_buf, nullptr, 0, b->cap);
    }
    cudaEventRecord(e1, b->cap);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != ZM_OK) return s;
    if (e != cudaSuccess) return cuda_error(e, "autotune timing");
    *us = 1000.0 * ms / 3.0;
    return ZM_OK;
}

static int tune_group(zm_batch_t b, BatchGroup& g, const zm_request_t* reqs,
                      std::map<std::string, TuneChoice>& cache, bool* changed) {
    const GeoImage geo = resolve(reqs[g.members[0]].image);
    const std::string key = tune_key(g.plan, (int)g.members.size(), geo);
    auto it = cache.find(key);
    if (it != cache.end()) {
        g.plan->tune_gather = it->second.gather;
        g.plan->tune_rings = it->second.rings;
        g.plan->tune_split = it->second.split;
        return ZM_OK;
    }
    bool tma = true;
    for (int r : g.members) tma = tma && tma_eligible(reqs[r].image);
    TuneChoice best;
    best.us = 1e30;
    for (int gather = 0; gather <= (tma ? 1 : 0); ++gather)
        for (int rings : {2, 4, 8})
            for (int split : {4, 8}) {
                g.plan->tune_gather = gather;
                g.plan->tune_rings = rings;
                g.plan->tune_split = split;
                double us = 0;
                const int s = time_group(b, g, reqs, &us);
                if (s != ZM_OK) return s;
                if (us < best.us) best = TuneChoice{gather, rings, split, us};
            }
    g.plan->tune_gather = best.gather;
    g.plan->tune_rings = best.rings;
    g.plan->tune_split = best.split;
    cache[key] = best;
    *changed = true;
    return ZM_OK;
}

}  // namespace zm

using namespace zm;

extern "C" int zm_batch_create(zm_batch_t* batch, const zm_request_t* reqs, int count, unsigned plan_flags) {
    if (!batch) return set_error(ZM_EINVAL, "batch pointer is NULL");
    *batch = nullptr;
    int s = check_requests(reqs, count);
    if (s != ZM_OK) return s;
    auto* b = new zm_batch_s();
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return set_error(ZM_ECUDA, "no CUDA device");
    }
    b->plan_flags = plan_flags;
    b->reqs.assign(reqs, reqs + count);
    // group by polar grid; inside a group, equal geometries next to each other
    std::map<std::pair<int, int>, int> gid;
    for (int r = 0; r < count; ++r) {
        const auto key = std::make_pair(reqs[r].n_rho, reqs[r].n_theta);
        auto it = gid.find(key);
        if (it == gid.end()) {
            it = gid.emplace(key, (int)b->groups.size()).first;
            b->groups.emplace_back();
            b->groups.back().n_rho = key.first;
            b->groups.back().n_theta = key.second;
        }
        BatchGroup& g = b->groups[it->second];
        g.members.push_back(r);
        g.n_max = std::max(g.n_max, reqs[r].n_max);
    }
    for (auto& g : b->groups) {
        std::stable_sort(g.members.begin(), g.members.end(), [&](int x, int y) {
            const GeoImage a = resolve(reqs[x].image), c = resolve(reqs[y].image);
            if (a.h != c.h) return a.h < c.h;
            if (a.w != c.w) return a.w < c.w;
            if (a.cx != c.cx) return a.cx < c.cx;
            if (a.cy != c.cy) return a.cy < c.cy;
            return a.r < c.r;
        });
        s = zm_plan(&g.plan, g.n_max, g.n_rho, g.n_theta, plan_flags);
        if (s == ZM_OK) s = zm_plan_reserve(g.plan, (int)g.members.size());
        if (s == ZM_OK) {
            const cudaError_t e =
                cudaMalloc(&g.out_buf, sizeof(float) * 2 * (size_t)num_moments(g.n_max) * g.members.size());
            if (e != cudaSuccess) s = cuda_error(e, "cudaMalloc(batch group buffer)");
        }
        if (s != ZM_OK) {
            free_batch(b);
            return s;
        }
    }
    cudaError_t e = cudaMalloc(&b->d_copy, sizeof(CopyDesc) * count);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int k = 0; k < BATCH_BRANCHES && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    // branches: largest groups first onto the least-loaded side stream (load =
    // pixels resampled + polar nodes transformed)
    {
        std::vector<std::pair<double, int>> cost;
        for (size_t gi = 0; gi < b->groups.size(); ++gi) {
            double c = 0;
            for (int r : b->groups[gi].members)
                c += (double)reqs[r].image.height * reqs[r].image.width + (double)reqs[r].n_rho * reqs[r].n_theta;
            cost.push_back({c, (int)gi});
        }
        std::stable_sort(cost.begin(), cost.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
        double load[BATCH_BRANCHES] = {0};
        b->branch.assign(b->groups.size(), 0);
        for (auto& cg : cost) {
            int k = 0;
            for (int j = 1; j < BATCH_BRANCHES; ++j)
                if (load[j] < load[k]) k = j;
            b->branch[cg.second] = k;
            load[k] += cg.first;
        }
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_error(e, "batch set-up");
    }
    // launch choices per group (timed on these images, or from the cache file)
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        const char* path = getenv("ZM_TUNE_CACHE");
        auto cache = read_tune_cache(path);
        bool changed = false;
        for (auto& g : b->groups) {
            s = tune_group(b, g, reqs, cache, &changed);
            if (s != ZM_OK) {
                free_batch(b);
                return s;
            }
        }
        if (changed) write_tune_cache(path, cache);
    }
    // one eager run grows every workspace and builds every tile plan, so that
    // graph capture later allocates nothing
    s = upload_copies(b, reqs);
    if (s == ZM_OK) s = enqueue_batch(b, reqs, 0, b->cap);
    if (s == ZM_OK) {
        e = cudaStreamSynchronize(b->cap);
        if (e != cudaSuccess) s = cuda_error(e, "batch warm-up");
    }
    if (s != ZM_OK) {
        free_batch(b);
        return s;
    }
    *batch = b;
    return ZM_OK;
}

extern "C" int zm_batch_run(zm_batch_t b, const zm_request_t* reqs, unsigned flags, void* stream) {
    if (!b) return set_error(ZM_EINVAL, "batch is NULL");
    if (flags & ~ZM_NEUMANN) return set_error(ZM_EINVAL, "unknown flags 0x%x", flags);
    const int count = (int)b->reqs.size();
    int s = check_requests(reqs, count);
    if (s != ZM_OK) return s;
    for (int r = 0; r < count; ++r)
        if (!same_shape(reqs[r], b->reqs[r]))
            return set_error(ZM_EINVAL, "request %d differs in shape from the batch it was created with", r);
    DeviceGuard dg(b->device);
    bool replay = b->exec && b->captured_flags == flags;
    for (int r = 0; r < count && replay; ++r) replay = same_pointers(reqs[r], b->captured[r]);
    if (!replay) {
        // new pointers or flags: capture the sequence again
        ZM_CUDA_TRY(cudaDeviceSynchronize());
        s = upload_copies(b, reqs);
        if (s != ZM_OK) return s;
        ZM_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        s = enqueue_batch(b, reqs, flags, b->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        if (s != ZM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture(batch)");
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_error(ei, "cudaGraphInstantiate(batch)");
        }
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->graph = graph;
        b->exec = exec;
        b->captured.assign(reqs, reqs + count);
        b->captured_flags = flags;
        ++b->captures;
    }
    ZM_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return ZM_OK;
}

extern "C" int zm_batch_info(zm_batch_t b, int* groups, int* captures) {
    if (!b) return set_error(ZM_EINVAL, "batch is NULL");
    if (groups) *groups = (int)b->groups.size();
    if (captures) *captures = b->captures;
    return ZM_OK;
}

extern "C" int zm_batch_destroy(zm_batch_t b) {
    if (!b) return ZM_OK;
    DeviceGuard dg(b->device);
    cudaDeviceSynchronize();
    free_batch(b);
    return ZM_OK;
}
