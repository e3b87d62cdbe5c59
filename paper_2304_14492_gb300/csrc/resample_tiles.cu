// Bilinear polar resampling (Sec. 2.5) driven by Cartesian image tiles.
//
// Every polar sample (rho_i, theta_k) interpolates the 2x2 pixels whose top-left
// corner ("anchor") is (floor X, floor Y).  The anchor plane is cut into 64x64
// tiles; a work item is one tile plus the ring and angle ranges whose samples
// can anchor in it (computed on the host from the geometry, with margins).
// Which samples a tile owns depends only on the geometry, so k_tile_plan
// decides it once per geometry (from the candidates' anchors, computed with the
// same float arithmetic as every later pass, so the tiles partition the samples
// exactly) and k_tile_records turns each into a 16-byte record: the stencil's
// offset in the tile box, the output offset and the two bilinear fractions.
// Per frame, a CTA starts one TMA copy of its tile and a one-pixel halo (a
// 68x65 box, zero outside the image), loads its records while the box is in
// flight, and interpolates exactly its own samples from shared memory into
// f_hat[b][i][k].  Each image pixel is read from HBM about once, every gather
// is a shared-memory access, and a CTA's critical path holds two dependent
// global loads (its item, then its records) besides the box.
//
// The ZM_TILE_* macros fix the tile shape and the launch shape; the defaults
// are the fastest of a sweep on GB300 at 4K (64x64 tiles in row-major order,
// four samples per thread in flight, eight CTAs per SM, two images per CTA: one
// read of a tile's records serves both boxes; 3 % faster per batch of 16 than
// one image per CTA once the polar samples stay in L2, three no faster, four
// slower).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "zm_internal.cuh"

namespace zm {

#ifndef ZM_TILE_W
#define ZM_TILE_W 64
#endif
#ifndef ZM_TILE_H
#define ZM_TILE_H 64
#endif
constexpr int TILE_W = ZM_TILE_W;        // anchors per tile row (a multiple of 4)
constexpr int TILE_H = ZM_TILE_H;        // anchor rows per tile
constexpr int BOX_W = TILE_W + 4;        // 16-byte multiple, covers x_t .. x_t + TILE_W
constexpr int BOX_H = TILE_H + 1;        // covers y_t .. y_t + TILE_H
constexpr int TILE_X0 = -4;              // x_t = -4 + 64 tx (multiple of 4, as TMA needs)
constexpr int TILE_Y0 = -1;              // y_t = -1 + 64 ty
constexpr int TILE_MAXC = 8192;          // candidates per work item
constexpr int TILE_MAXR = 1024;          // rings per work item
constexpr int TILE_MAX_IMG = 64;         // tensor maps per launch
constexpr int TILE_THREADS = 256;
#ifndef ZM_TILE_G
#define ZM_TILE_G 4
#endif
#ifndef ZM_TILE_MINB
#define ZM_TILE_MINB 8
#endif
#ifndef ZM_TILE_IPC
#define ZM_TILE_IPC 2
#endif
constexpr int TILE_IPC = ZM_TILE_IPC;    // images per CTA (boxes in flight per CTA)
constexpr int TILE_BOX_FLOATS = ((BOX_H * BOX_W + 31) / 32) * 32;   // 128-byte aligned boxes
constexpr int TILE_G = ZM_TILE_G;        // samples per thread handled together
constexpr int TILE_MINB = ZM_TILE_MINB;  // resident CTAs per SM the registers allow
constexpr unsigned long long TILE_WAIT_NS = 2000000000ull;

struct __align__(16) TileItem {
    int x_t, y_t;        // anchor origin of the tile
    int i_lo, i_hi;      // rings [i_lo, i_hi)
    int k_lo, k_n;       // angles (k_lo + j) mod N, j < k_n; k_lo in [0, N)
    int s0, cnt;         // the item's samples: [s0, s0 + cnt) of the plan's list
};

// Packed sample of a work item: (ring offset << 11) | angle offset in the
// item's staged angle window (ring offset < 1024, angle offset < 2048).
constexpr int SAMPLE_KBITS = 11;

// A planned sample, ready to interpolate: shared-memory offset of its 2x2
// stencil in the box, output offset in the item's ring block, and the bilinear
// fractions (as float bits).
struct TileRecord {
    int so, oo, fx, fy;
};

struct TileParams {
    const TileItem* items;
    const int4* recs;            // TileRecord of every planned sample, item after item
    float* fhat;
    int* status;
    int n_rho, N, b_off;
    int keep_l2;                 // fhat is scratch the next kernel reads: stores marked evict_last
    int nb;                      // images in this launch
    CUtensorMap maps[TILE_MAX_IMG];
};

__device__ __forceinline__ unsigned long long tile_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Sample coordinates: the single definition every pass uses.
__device__ __forceinline__ void sample_xy(float rad, float2 cv, float cx, float cy, float* X, float* Y) {
    *X = fmaf(rad, cv.x, cx);
    *Y = fmaf(-rad, cv.y, cy);
}

// Planning pass over the candidate (ring, angle) pairs of each item: keeps
// those whose anchor lies in the item's tile.  count_only: counts[item];
// otherwise writes the packed samples in candidate order from items[item].s0.
struct PlanParams {
    const TileItem* items;
    const float* rho32;
    const float2* cs;
    int* counts;
    uint32_t* samples;
    int4* recs;
    int N;
    float cx, cy, r;
    int count_only;
};

__global__ void __launch_bounds__(TILE_THREADS) k_tile_plan(const __grid_constant__ PlanParams p) {
    __shared__ int warp_tot[TILE_THREADS / 32];
    __shared__ int base_s;
    const TileItem it = p.items[blockIdx.x];
    const int N = p.N;
    const int nr = it.i_hi - it.i_lo, kn = it.k_n;
    const int total = nr * kn;
    const float xt = (float)it.x_t, yt = (float)it.y_t;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int mine = 0;
    if (threadIdx.x == 0) base_s = p.count_only ? 0 : it.s0;
    __syncthreads();
    for (int c0 = 0; c0 < total; c0 += TILE_THREADS) {
        const int c = c0 + threadIdx.x;
        bool valid = false;
        int ii = 0, j = 0;
        if (c < total) {
            ii = c / kn;
            j = c - ii * kn;
            const float rad = p.r * __ldg(&p.rho32[it.i_lo + ii]);
            const float2 cv = __ldg(&p.cs[(it.k_lo + j) & (N - 1)]);
            float X, Y;
            sample_xy(rad, cv, p.cx, p.cy, &X, &Y);
            const int lx = (int)(floorf(X) - xt), ly = (int)(floorf(Y) - yt);
            valid = (unsigned)lx < (unsigned)TILE_W && (unsigned)ly < (unsigned)TILE_H;
        }
        if (p.count_only) {
            mine += valid ? 1 : 0;
            continue;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < TILE_THREADS / 32; ++w) {
            before += (w < warp) ? warp_tot[w] : 0;
            all += warp_tot[w];
        }
        if (valid) {
            const int pos = base_s + before + __popc(bal & ((1u << lane) - 1u));
            p.samples[pos] = ((uint32_t)ii << SAMPLE_KBITS) | (uint32_t)j;
        }
        __syncthreads();
        if (threadIdx.x == 0) base_s += all;
        __syncthreads();
    }
    if (p.count_only) {
        for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if (lane == 0) warp_tot[warp] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < TILE_THREADS / 32; ++w) t += warp_tot[w];
            p.counts[blockIdx.x] = t;
        }
    }
}

// The record of one planned sample (same float arithmetic as the planning
// pass, so the anchor is the one that placed the sample in this tile).
__global__ void __launch_bounds__(TILE_THREADS) k_tile_records(const __grid_constant__ PlanParams p) {
    const TileItem it = p.items[blockIdx.x];
    const int N = p.N;
    for (int c = threadIdx.x; c < it.cnt; c += TILE_THREADS) {
        const uint32_t code = p.samples[it.s0 + c];
        const int ii = (int)(code >> SAMPLE_KBITS);
        const int j = (int)(code & ((1u << SAMPLE_KBITS) - 1u));
        float X, Y;
        sample_xy(p.r * __ldg(&p.rho32[it.i_lo + ii]), __ldg(&p.cs[(it.k_lo + j) & (N - 1)]), p.cx, p.cy, &X, &Y);
        const float xf = floorf(X), yf = floorf(Y);
        // the clamp only keeps later shared-memory reads in the box should the
        // anchor ever differ from the planning pass's
        const int lx = min(max((int)(xf - (float)it.x_t), 0), TILE_W - 1);
        const int ly = min(max((int)(yf - (float)it.y_t), 0), TILE_H - 1);
        p.recs[it.s0 + c] = make_int4(ly * BOX_W + lx, ii * N + ((it.k_lo + j) & (N - 1)), __float_as_int(X - xf),
                                      __float_as_int(Y - yf));
    }
}

// Records [c0, c0 + TILE_G * TILE_THREADS) of the item: this thread's TILE_G
// of them, all loads issued before any use.
__device__ __forceinline__ void tile_group(const int4* rec, int cnt, int c0, int4 (&ts)[TILE_G], bool (&on)[TILE_G]) {
#pragma unroll
    for (int k = 0; k < TILE_G; ++k) {
        const int c = c0 + threadIdx.x + k * TILE_THREADS;
        on[k] = c < cnt;
        ts[k] = on[k] ? __ldg(&rec[c]) : make_int4(0, 0, 0, 0);
    }
}

__device__ __forceinline__ void tile_interp(const float* tile, float* out, const int4 (&ts)[TILE_G],
                                            const bool (&on)[TILE_G], uint64_t pol) {
    float val[TILE_G];
#pragma unroll
    for (int k = 0; k < TILE_G; ++k) {
        const float* t0p = tile + ts[k].x;
        const float fx = __int_as_float(ts[k].z), fy = __int_as_float(ts[k].w);
        const float p00 = t0p[0], p01 = t0p[1], p10 = t0p[BOX_W], p11 = t0p[BOX_W + 1];
        const float top = fmaf(fx, p01 - p00, p00);
        const float bot = fmaf(fx, p11 - p10, p10);
        val[k] = fmaf(fy, bot - top, top);
    }
#pragma unroll
    for (int k = 0; k < TILE_G; ++k)
        if (on[k]) asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(out + ts[k].y), "f"(val[k]), "l"(pol)
                                : "memory");
}

__device__ __forceinline__ bool tile_try_wait(uint32_t bar) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(ok) : "r"(bar) : "memory");
    return ok != 0;
}

// Bounded wait for a box (phase 0 of its barrier).
__device__ __forceinline__ bool tile_wait(uint32_t bar) {
    if (tile_try_wait(bar)) return true;
    const unsigned long long t0 = tile_ns();
    while (!tile_try_wait(bar))
        if (tile_ns() - t0 > TILE_WAIT_NS) return false;
    return true;
}

// One CTA per (item, TILE_IPC images): the boxes of its images arrive by TMA
// while the threads load the records of their first samples, which then serve
// every image; the rest of a heavy item follows in groups.  Launched as a
// programmatic dependent: the record loads start before the previous kernel
// has finished, the boxes (and every store) after.
__global__ void __launch_bounds__(TILE_THREADS, TILE_MINB) k_resample_tiles(const __grid_constant__ TileParams p) {
    extern __shared__ __align__(128) float tile_sm[];          // [TILE_IPC][TILE_BOX_FLOATS]
    __shared__ __align__(8) uint64_t bar[TILE_IPC];
    __shared__ int s_ok;
    const TileItem it = p.items[blockIdx.x];
    const int b0 = blockIdx.y * TILE_IPC;
    const int nimg = min(TILE_IPC, p.nb - b0);
    const uint32_t bar_a = static_cast<uint32_t>(__cvta_generic_to_shared(&bar[0]));
    const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(tile_sm));
    // this thread's first samples: the records belong to the plan (written
    // before any launch), so their loads go out before the wait below and
    // overlap the previous kernel's end
    const int cnt = it.cnt;
    const int4* rec = p.recs + it.s0;
    int4 ts[TILE_G];
    bool on[TILE_G];
    tile_group(rec, cnt, 0, ts, on);
    if (threadIdx.x == 0) {
        for (int k = 0; k < nimg; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a + 8u * k));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // the images may come from the previous kernel, and it may still read
    // f_hat.  (No early launch of the dependents: the ring FFT's CTAs would
    // take SM room from this kernel's later waves.)
    griddep_wait();
    if (threadIdx.x == 0) {
        uint64_t pol;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
        for (int k = 0; k < nimg; ++k) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a + 8u * k),
                         "r"((uint32_t)(BOX_H * BOX_W * 4)) : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst + 4u * TILE_BOX_FLOATS * k), "l"(&p.maps[b0 + k]),
                "r"(it.x_t), "r"(it.y_t), "r"(bar_a + 8u * k), "l"(pol)
                : "memory");
        }
    }
    // one thread waits for the boxes (bounded); the others wait at the barrier
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int k = 0; k < nimg && ok; ++k) ok = tile_wait(bar_a + 8u * k);
        if (!ok) {
            // a copy did not arrive in time: report it and let them drain (bounded)
            atomicExch(p.status, ZM_ETIMEOUT);
            for (int k = 0; k < nimg; ++k) tile_wait(bar_a + 8u * k);
        }
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) return;

    const size_t img_stride = (size_t)p.n_rho * p.N;
    float* out = p.fhat + ((size_t)(p.b_off + b0) * p.n_rho + it.i_lo) * p.N;
    uint64_t spol;
    if (p.keep_l2) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(spol));
    else asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(spol));
#pragma unroll
    for (int k = 0; k < TILE_IPC; ++k)
        if (k < nimg) tile_interp(tile_sm + k * TILE_BOX_FLOATS, out + k * img_stride, ts, on, spol);
    for (int c0 = TILE_G * TILE_THREADS; c0 < cnt; c0 += TILE_G * TILE_THREADS) {
        tile_group(rec, cnt, c0, ts, on);
#pragma unroll
        for (int k = 0; k < TILE_IPC; ++k)
            if (k < nimg) tile_interp(tile_sm + k * TILE_BOX_FLOATS, out + k * img_stride, ts, on, spol);
    }
}

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// An image can be staged by TMA when its base and row pitch are 16-byte
// multiples and its extents fit the tensor-map limits.
bool tma_eligible(const zm_image_t& im) {
    return ((uintptr_t)im.data & 15u) == 0 && ((im.pitch * 4) & 15) == 0 && im.width <= (1 << 30) &&
           im.height <= (1 << 30) && encode_fn() != nullptr;
}

static int encode_map(const zm_image_t& im, CUtensorMap* map) {
    cuuint64_t dims[2] = {(cuuint64_t)im.width, (cuuint64_t)im.height};
    cuuint64_t strides[1] = {(cuuint64_t)im.pitch * 4};
    cuuint32_t box[2] = {BOX_W, BOX_H};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(im.data), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(ZM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ZM_OK;
}

struct TileList {
    TileItem* items = nullptr;
    int4* recs = nullptr;      // TileRecord of every planned sample, item after item
    int n = 0;
    long long n_samples = 0;
    bool need_zero = false;   // some samples anchor outside every tile (they are 0)
    ~TileList() {
        if (items) cudaFree(items);
        if (recs) cudaFree(recs);
    }
};

// Work items for one geometry.  Ring range from the distance range of the
// tile's anchor rectangle to the centre (2 px margin); angle range from its
// corners' polar angles (1.5 steps margin), the full circle when the centre is
// within 2 px of the rectangle.
static int build_tiles(zm_plan_t p, const GeoImage& g, TileList* tl) {
    const int N = p->n_theta, n_rho = p->n_rho;
    std::vector<double> rho(n_rho);
    {
        std::vector<float> r32(n_rho);
        ZM_CUDA_TRY(cudaMemcpy(r32.data(), p->rho32, sizeof(float) * n_rho, cudaMemcpyDeviceToHost));
        for (int i = 0; i < n_rho; ++i) rho[i] = (double)r32[i];
    }
    const double cx = g.cx, cy = g.cy, R = g.r;
    const double rmax = R * rho[n_rho - 1];
    const int ntx = (g.w + 3 - TILE_X0 + TILE_W - 1) / TILE_W;   // covers anchors up to w - 1
    const int nty = (g.h + 0 - TILE_Y0 + TILE_H - 1) / TILE_H;   // covers anchors up to h - 1
    const double gx0 = TILE_X0, gy0 = TILE_Y0, gx1 = TILE_X0 + (double)ntx * TILE_W,
                 gy1 = TILE_Y0 + (double)nty * TILE_H;
    // samples anchor within +-(rmax + float error) of the centre; those outside
    // the tile grid see only zero pixels and are written by a memset
    const double e = 0.5;
    tl->need_zero = (cx - rmax - e < gx0) || (cx + rmax + e >= gx1) || (cy - rmax - e < gy0) || (cy + rmax + e >= gy1);
    std::vector<std::pair<long, TileItem>> items;
    const double kPi = 3.14159265358979323846, two_pi = 2.0 * kPi;
    for (int ty = 0; ty < nty; ++ty) {
        for (int tx = 0; tx < ntx; ++tx) {
            const int x_t = TILE_X0 + tx * TILE_W, y_t = TILE_Y0 + ty * TILE_H;
            // rectangle in centred coordinates, y up
            const double u0 = x_t - cx, u1 = x_t + TILE_W - cx;
            const double v0 = cy - (y_t + TILE_H), v1 = cy - y_t;
            const double du = (u0 > 0) ? u0 : (u1 < 0 ? -u1 : 0.0);
            const double dv = (v0 > 0) ? v0 : (v1 < 0 ? -v1 : 0.0);
            const double dmin = std::sqrt(du * du + dv * dv);
            const double mu = std::max(std::fabs(u0), std::fabs(u1)), mv = std::max(std::fabs(v0), std::fabs(v1));
            const double dmax = std::sqrt(mu * mu + mv * mv);
            if (dmin - 2.0 > rmax) continue;
            const double lo = (dmin - 2.0) / R, hi = (dmax + 2.0) / R;
            const int i_lo = (int)(std::lower_bound(rho.begin(), rho.end(), lo) - rho.begin());
            const int i_hi = (int)(std::upper_bound(rho.begin(), rho.end(), hi) - rho.begin());
            if (i_lo >= i_hi) continue;
            int k_lo = 0, k_n = N;
            if (dmin > 2.0) {
                const double ac = std::atan2(0.5 * (v0 + v1), 0.5 * (u0 + u1));
                double dlo = 0, dhi = 0;
                const double us[2] = {u0, u1}, vs[2] = {v0, v1};
                for (double uu : us)
                    for (double vv : vs) {
                        double d = std::atan2(vv, uu) - ac;
                        while (d > kPi) d -= two_pi;
                        while (d <= -kPi) d += two_pi;
                        dlo = std::min(dlo, d);
                        dhi = std::max(dhi, d);
                    }
                const double ka = (ac + dlo) * N / two_pi - 1.5, kb = (ac + dhi) * N / two_pi + 1.5;
                const long kl = (long)std::floor(ka), kh = (long)std::ceil(kb);
                if (kh - kl + 1 < N) {
                    k_lo = (int)(((kl % N) + N) % N);
                    k_n = (int)(kh - kl + 1);
                }
            }
            // split heavy tiles by ring ranges
            const int per = std::min(TILE_MAXR, std::max(1, TILE_MAXC / k_n));
            for (int a = i_lo; a < i_hi; a += per) {
                TileItem t{x_t, y_t, a, std::min(i_hi, a + per), k_lo, k_n};
                items.push_back({(long)(t.i_hi - t.i_lo) * k_n, t});
            }
        }
    }
    // items stay in row-major tile order: CTAs that run together then read
    // horizontally adjacent boxes, which share DRAM pages (measured faster than
    // ordering by weight); ZM_TILE_SORT=1 orders them heaviest first instead
#ifndef ZM_TILE_SORT
#define ZM_TILE_SORT 0
#endif
    if (ZM_TILE_SORT)
        std::stable_sort(items.begin(), items.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<TileItem> h(items.size());
    for (size_t j = 0; j < items.size(); ++j) h[j] = items[j].second;
    tl->n = (int)h.size();
    if (!tl->n) return ZM_OK;
    ZM_CUDA_TRY(cudaMalloc(&tl->items, sizeof(TileItem) * h.size()));
    ZM_CUDA_TRY(cudaMemcpy(tl->items, h.data(), sizeof(TileItem) * h.size(), cudaMemcpyHostToDevice));
    // plan: count the samples each tile owns, store them packed, then turn
    // them into records
    PlanParams pp;
    pp.items = tl->items;
    pp.rho32 = p->rho32;
    pp.cs = p->cs;
    pp.N = N;
    pp.cx = g.cx;
    pp.cy = g.cy;
    pp.r = g.r;
    pp.samples = nullptr;
    pp.recs = nullptr;
    ZM_CUDA_TRY(cudaMalloc(&pp.counts, sizeof(int) * tl->n));
    pp.count_only = 1;
    k_tile_plan<<<tl->n, TILE_THREADS>>>(pp);
    cudaError_t ce = cudaGetLastError();
    std::vector<int> cnt(tl->n);
    if (ce == cudaSuccess) ce = cudaMemcpy(cnt.data(), pp.counts, sizeof(int) * tl->n, cudaMemcpyDeviceToHost);
    cudaFree(pp.counts);
    if (ce != cudaSuccess) return cuda_error(ce, "k_tile_plan (count)");
    count_launch();
    long long total = 0;
    for (int j = 0; j < tl->n; ++j) {
        h[j].s0 = (int)total;
        h[j].cnt = cnt[j];
        total += cnt[j];
    }
    if (total >= (1ll << 31)) return set_error(ZM_EINVAL, "too many polar samples for one geometry (%lld)", total);
    tl->n_samples = total;
    ZM_CUDA_TRY(cudaMemcpy(tl->items, h.data(), sizeof(TileItem) * h.size(), cudaMemcpyHostToDevice));
    ZM_CUDA_TRY(cudaMalloc(&pp.samples, sizeof(uint32_t) * std::max<long long>(1, total)));
    ce = cudaMalloc(&tl->recs, sizeof(int4) * std::max<long long>(1, total));
    if (ce == cudaSuccess) {
        pp.recs = tl->recs;
        pp.count_only = 0;
        k_tile_plan<<<tl->n, TILE_THREADS>>>(pp);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) {
            count_launch();
            k_tile_records<<<tl->n, TILE_THREADS>>>(pp);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) {
            count_launch();
            ce = cudaDeviceSynchronize();
        }
    }
    cudaFree(pp.samples);
    if (ce != cudaSuccess) return cuda_error(ce, "tile plan");
    return ZM_OK;
}

// Work lists cached per (plan, geometry); released with the plan.
struct TileCache {
    std::mutex mu;
    std::map<std::tuple<zm_plan_t, int, int, float, float, float>, std::unique_ptr<TileList>> lists;
};
static TileCache g_tiles;

void release_tiles(zm_plan_t p) {
    std::lock_guard<std::mutex> lk(g_tiles.mu);
    for (auto it = g_tiles.lists.begin(); it != g_tiles.lists.end();) {
        if (std::get<0>(it->first) == p) it = g_tiles.lists.erase(it);
        else ++it;
    }
}

static int get_tiles(zm_plan_t p, const GeoImage& g, TileList** out) {
    std::lock_guard<std::mutex> lk(g_tiles.mu);
    auto key = std::make_tuple(p, g.h, g.w, g.cx, g.cy, g.r);
    auto it = g_tiles.lists.find(key);
    if (it == g_tiles.lists.end()) {
        auto tl = std::make_unique<TileList>();
        const int s = build_tiles(p, g, tl.get());
        if (s != ZM_OK) return s;
        it = g_tiles.lists.emplace(key, std::move(tl)).first;
    }
    *out = it->second.get();
    return ZM_OK;
}

// Resample images [b0, b0 + nb) (all TMA-eligible, one geometry) into
// fhat[b][i][k] (fhat points at image 0 of the whole batch).
int launch_resample_tiles(zm_plan_t p, const zm_image_t* imgs, int b0, int nb, float* fhat, cudaStream_t st,
                          bool keep_l2) {
    const GeoImage g = resolve(imgs[b0]);
    TileList* tl = nullptr;
    int s = get_tiles(p, g, &tl);
    if (s != ZM_OK) return s;
    const size_t per_img = (size_t)p->n_rho * p->n_theta;
    if (tl->need_zero) ZM_CUDA_TRY(cudaMemsetAsync(fhat + (size_t)b0 * per_img, 0, sizeof(float) * per_img * nb, st));
    if (tl->n == 0) return ZM_OK;
    static thread_local TileParams tp;
    tp.items = tl->items;
    tp.recs = tl->recs;
    tp.fhat = fhat;
    tp.status = p->status;
    tp.keep_l2 = keep_l2 ? 1 : 0;
    tp.n_rho = p->n_rho;
    tp.N = p->n_theta;
    for (int c0 = 0; c0 < nb; c0 += TILE_MAX_IMG) {
        const int nc = std::min(TILE_MAX_IMG, nb - c0);
        tp.b_off = b0 + c0;
        for (int j = 0; j < nc; ++j) {
            s = encode_map(imgs[b0 + c0 + j], &tp.maps[j]);
            if (s != ZM_OK) return s;
        }
        tp.nb = nc;
        const size_t smem = sizeof(float) * TILE_BOX_FLOATS * TILE_IPC;
        if (smem > 48 * 1024) {
            static bool configured[64] = {false};
            const int dev = p->device;
            if (dev < 0 || dev >= 64 || !configured[dev]) {
                ZM_CUDA_TRY(
                    cudaFuncSetAttribute(k_resample_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                if (dev >= 0 && dev < 64) configured[dev] = true;
            }
        }
        ZM_LAUNCH_PDL("k_resample_tiles", k_resample_tiles, dim3(tl->n, (nc + TILE_IPC - 1) / TILE_IPC),
                      dim3(TILE_THREADS), smem, st, tp);
    }
    return ZM_OK;
}

bool same_geometry(const zm_image_t& a, const zm_image_t& b) {
    const GeoImage ga = resolve(a), gb = resolve(b);
    return ga.h == gb.h && ga.w == gb.w && ga.cx == gb.cx && ga.cy == gb.cy && ga.r == gb.r;
}

}  // namespace zm
