// Polar resampling (Sec. 2.5) fused with the ring FFT of Eq. 1: image pixels in,
// ring spectra F_m(rho_i), m <= n_max, out.  The polar samples exist only in
// registers.
//
// A CTA takes one image and a band of FU_R = 16 consecutive rings; warp w owns
// ring i0 + w and holds it the way the warp FFT of ring_fft.cuh wants its
// input: lane t, register s = the samples at angles 64 s + 2 t and 64 s + 2 t + 1.
// The circle is cut into slots of 32 angles (half a register) and consecutive
// slots into stages.  For each stage a host-built plan lists the image rows its
// samples' bilinear stencils touch and, per row, the exact span of 16-byte
// units that holds those pixels.  Groups of 8 lanes copy the spans with
// 16-byte cp.async into shared-memory stage buffers (units outside the image
// are written as zeros); the next stage's pixels are in flight while the warps
// sample the current one, and the row entries of a stage are copied into
// shared memory a stage before its pixels, so nothing between a barrier and
// the copies it releases waits on a global load.  (One bulk copy per row span
// through the TMA engine was measured twice as slow: the engine spends tens of
// cycles per copy, and a 4K frame has about 150 thousand spans.)  A per-row pair of base
// offsets turns a stencil's pixel coordinates into its two shared-memory rows.
// A warp samples 32 consecutive angles of its ring at a time and shuffles them
// into the FFT's register layout.  After the last stage the stage buffers
// become the FFT's work rows: each warp transforms its ring, splits the packed
// spectrum into F_m (the e^{-j m theta} symmetry of Sec. 2), and the CTA writes
// F as FP32 rows or as the bf16 hi / lo operand blocks of the tensor-core
// projection.
//
// The plan computes every sample's stencil anchor with the same float
// operations as the kernel (r * rho_i, then fmaf with cos / sin theta_k), so
// the staged spans cover the stencils exactly; every shared-memory index is
// clamped into its buffer all the same.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ring_fft.cuh"
#include "tc_common.cuh"
#include "zm_internal.cuh"

namespace zm {

constexpr int FU_R = 16;                  // rings per band = warps per CTA
constexpr int FU_THREADS = FU_R * 32;
constexpr int FU_SLOT = 32;               // angles per slot (half a warp-FFT register)
#ifndef ZM_FU_NBUF
#define ZM_FU_NBUF 2
#endif
#if ZM_FU_NBUF == 2
constexpr int FU_STAGE_FLOATS = 8192;     // floats per stage buffer
constexpr int FU_MAX_ROWS = 512;          // staged rows per stage
#else
constexpr int FU_STAGE_FLOATS = 4608;
constexpr int FU_MAX_ROWS = 384;
#endif
constexpr int FU_NBUF = ZM_FU_NBUF;       // stage buffers
constexpr int FU_LOOK = FU_NBUF - 1;      // stages whose pixels are in flight while one is sampled
constexpr int FU_NENT = 2 * FU_LOOK + 1;  // row-entry buffers: fetched 2 LOOK stages ahead, read until the stage ends
constexpr int FU_MAX_IMG = 128;           // images per launch
constexpr double FU_MERGE_SLACK = 1.25;   // a merged stage may cost this much more than its parts
// stage buffers and row entries (16 bytes each), in floats
constexpr int FU_STAGING = FU_NBUF * FU_STAGE_FLOATS + FU_NENT * 4 * FU_MAX_ROWS;

struct __align__(16) FuStage {
    int y_lo, nrows, row0, h_lo;          // first image row, rows, first row entry, first half-register
    int h_hi, bytes, pad0, pad1;          // end half-register, image bytes the stage copies
};

struct FuParams {
    const int* order;        // bands by decreasing weight
    const int2* band_st;     // per band: stages [x, y)
    const FuStage* stages;
    const int4* rows;        // per staged row, see FusedPlan
    const float* rho32;
    const float2* cs;        // (cos, sin) theta_k
    const float2* tw;
    uint8_t* Fblk;           // bf16 hi / lo operand blocks, or NULL
    size_t fblk_half;
    float* F;                // [n_max+1][batch_total][2][n_rho] when Fblk is NULL
    float* fhat_out;         // [batch_total][n_rho][N] or NULL
    int* status;
    int n_rho, n_max, batch_total, b_off, nb, n_chunks;
    int h, w;
    float cx, cy, r;
    const float* data[FU_MAX_IMG];
    long long pitch[FU_MAX_IMG];
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared memory of one CTA (floats): the staging area (stage buffers, row-base
// pairs, row entries), which the FFT rows reuse after the last stage; the
// band's stage records; the split spectra; the twiddles.
template <int LOGN>
struct FuSmem {
    static constexpr int ROW = RingFFT<LOGN>::ROW_FLOATS;
    static constexpr int REGION = FU_STAGING > FU_R * ROW ? FU_STAGING : FU_R * ROW;
    static constexpr int MAX_STAGES = (1 << LOGN) / FU_SLOT;   // a band has at most one stage per slot
    static size_t bytes(int n_max) {
        const size_t fs = ((size_t)FU_R * 2 * (n_max + 1) + 3) & ~(size_t)3;
        return sizeof(float) * ((size_t)REGION + 8 * MAX_STAGES + fs) +
               sizeof(float2) * ((size_t)RingFFT<LOGN>::TW_FLOAT2 + n_max + 1);
    }
};

template <int LOGN>
__global__ void __launch_bounds__(FU_THREADS, LOGN >= 11 ? 1 : 2) k_ring_fused(const __grid_constant__ FuParams p) {
    using FFT = RingFFT<LOGN>;
    using SM = FuSmem<LOGN>;
    constexpr int N = FFT::N;
    constexpr int Q = FFT::Q;
    static_assert(FFT::L == 32, "the fused path needs N_theta >= 64");
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_max = p.n_max, nm1 = n_max + 1;
    float* bufs = smem;                                                              // [NBUF][STAGE]
    int4* ents = reinterpret_cast<int4*>(smem + FU_NBUF * FU_STAGE_FLOATS);         // [NENT][MAX_ROWS]
    FuStage* srec = reinterpret_cast<FuStage*>(smem + SM::REGION);                  // [MAX_STAGES]
    float* Fs = reinterpret_cast<float*>(srec + SM::MAX_STAGES);                    // [ring][re/im][m]
    float2* twt = reinterpret_cast<float2*>(Fs + ((FU_R * 2 * nm1 + 3) & ~3));
    float2* twm = twt + FFT::TW_FLOAT2;                                              // e^{-2 pi i m / N}
    FFT::load_twiddles(twt, p.tw);
    for (int m = threadIdx.x; m < nm1; m += blockDim.x) twm[m] = __ldg(&p.tw[m]);

    const int bi = blockIdx.x % p.nb;
    const int band = __ldg(&p.order[blockIdx.x / p.nb]);
    const int b = p.b_off + bi;
    const int i0 = band * FU_R;
    const int ring = i0 + warp;
    const bool live = ring < p.n_rho;
    const float rad = live ? p.r * __ldg(&p.rho32[ring]) : 0.f;
    const int2 sr = __ldg(&p.band_st[band]);
    const int ns = sr.y - sr.x;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) srec[j] = p.stages[sr.x + j];
    const float* img = p.data[bi];
    const long long pitch = p.pitch[bi];
    __syncthreads();                         // stage records
    griddep_wait();                          // the images may come from the previous kernel

    // row entries of stage j: one 16-byte cp.async per row
    auto fetch_entries = [&](int j) {
        if (j < ns && (int)threadIdx.x < srec[j].nrows)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(ents + (j % FU_NENT) * FU_MAX_ROWS +
                                                                                    threadIdx.x)),
                         "l"(p.rows + srec[j].row0 + threadIdx.x)
                         : "memory");
    };
    // pixels of stage j: groups of 8 lanes per staged row, one 16-byte
    // cp.async per lane and unit; rows the plan marks as reaching outside the
    // image take the checked path (units outside written as zeros)
    const int grp = warp * 4 + (lane >> 3), l8 = lane & 7;
    auto fetch_pixels = [&](int j) {
        if (j >= ns) return;
        const int bb = j % FU_NBUF;
        const int nrows = srec[j].nrows, y_lo = srec[j].y_lo;
        const uint32_t buf = smem_u32(bufs + bb * FU_STAGE_FLOATS);
        const int4* ent = ents + (j % FU_NENT) * FU_MAX_ROWS;
#pragma unroll 1
        for (int rr = grp; rr < nrows; rr += FU_THREADS / 8) {
            const int2 e = *reinterpret_cast<const int2*>(&ent[rr].z);
            const int soff = e.x & 0xffff, nu = (e.x >> 16) & 0xfff, xu = e.y;
            const int y = y_lo + rr;
            if (e.x >= 0) {                                  // inside the image
                const float* src = img + (long long)y * pitch + 4 * xu;
#pragma unroll 1
                for (int u = l8; u < nu; u += 8)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(buf + 16u * (soff / 4 + u)),
                                 "l"(src + 4 * u)
                                 : "memory");
            } else {
                const bool yin = (unsigned)y < (unsigned)p.h;
                const float* src = img + (long long)(yin ? y : 0) * pitch;
                for (int u = l8; u < nu; u += 8) {
                    const int xq = xu + u;
                    if (yin && (unsigned)xq < (unsigned)(p.w >> 2))
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(buf + 16u * (soff / 4 + u)),
                                     "l"(src + 4 * xq)
                                     : "memory");
                    else
                        *reinterpret_cast<float4*>(bufs + bb * FU_STAGE_FLOATS + soff + 4 * u) =
                            make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
    };

    float2 v[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) v[s] = make_float2(0.f, 0.f);

    if (ns > 0) {
#pragma unroll
        for (int j = 0; j < FU_LOOK; ++j) fetch_entries(j);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();                     // entries of the first stages
#pragma unroll
        for (int j = 0; j < FU_LOOK; ++j) {
            fetch_pixels(j);
            fetch_entries(j + FU_LOOK);
            cp_async_commit();
        }
        // The half-registers h = 0 .. 2Q - 1 in order, unrolled so that the
        // register each one fills is known at compile time; the stages cover
        // consecutive runs of them, and the pipeline advances (one barrier)
        // where a stage ends.  Two half-registers of one stage are sampled
        // together (independent chains the scheduler can interleave).
        int g = 0, h_end = 0, y_lo = 0;
        unsigned nr2 = 0;
        const float* buf = bufs;
        const int4* ent = ents;
        auto advance = [&]() {
            cp_async_wait<FU_LOOK - 1>();    // this thread's pixels of stage g and entries of stage g + LOOK
            __syncthreads();                 // everybody's; stage g - 1 is no longer read
            fetch_pixels(g + FU_LOOK);
            fetch_entries(g + 2 * FU_LOOK);
            cp_async_commit();               // possibly empty: the group count stays uniform
            buf = bufs + (g % FU_NBUF) * FU_STAGE_FLOATS;
            ent = ents + (g % FU_NENT) * FU_MAX_ROWS;
            y_lo = srec[g].y_lo;
            nr2 = (unsigned)(srec[g].nrows - 2);
            h_end = srec[g].h_hi;
            ++g;
        };
        // lane l's sample at angle 32 h + l
        auto sample = [&](int h) -> float {
            const float2 c = __ldg(&p.cs[32 * h + lane]);
            const float X = fmaf(rad, c.x, p.cx), Y = fmaf(-rad, c.y, p.cy);
            const float xf = floorf(X), yf = floorf(Y);
            const float fx = X - xf, fy = Y - yf;
            const unsigned ry = min((unsigned)((int)yf - y_lo), nr2);
            const int x0 = (int)xf;
            const int2 rb = *reinterpret_cast<const int2*>(&ent[ry]);
            const unsigned a0 = min((unsigned)(rb.x + x0), (unsigned)(FU_STAGE_FLOATS - 2));
            const unsigned a1 = min((unsigned)(rb.y + x0), (unsigned)(FU_STAGE_FLOATS - 2));
            const float p00 = buf[a0], p01 = buf[a0 + 1], p10 = buf[a1], p11 = buf[a1 + 1];
            const float top = fmaf(fx, p01 - p00, p00);
            const float bot = fmaf(fx, p11 - p10, p10);
            return fmaf(fy, bot - top, top);
        };
        // lanes 16 (h & 1) .. + 15 of register h / 2 take the pairs (2 t', 2 t' + 1)
        auto place = [&](int h, float val) {
            const int tq = 2 * (lane & 15);
            const float x0v = __shfl_sync(0xffffffffu, val, tq);
            const float x1v = __shfl_sync(0xffffffffu, val, tq + 1);
            if ((lane >> 4) == (h & 1)) v[h >> 1] = make_float2(x0v, x1v);
        };
#pragma unroll
        for (int h = 0; h < 2 * Q; h += 2) {
            if (h == h_end) advance();
            if (h + 1 == h_end) {
                if (live) place(h, sample(h));
                advance();
                if (live) place(h + 1, sample(h + 1));
            } else if (live) {
                const float va = sample(h), vb = sample(h + 1);
                place(h, va);
                place(h + 1, vb);
            }
        }
    }
    cp_async_wait<0>();                      // nothing may land in the buffers the FFT reuses
    __syncthreads();                         // staging area -> FFT rows
    griddep_launch();

    // ---- polar samples out, when asked for
    if (p.fhat_out && live) {
        float2* dst = reinterpret_cast<float2*>(p.fhat_out + ((size_t)b * p.n_rho + ring) * N);
#pragma unroll
        for (int s = 0; s < Q; ++s) dst[32 * s + lane] = v[s];
    }

    // ---- ring FFT and split: F_m = (Z_m + conj Z_{M-m})/2 + e^{-2 pi i m/N} (Z_m - conj Z_{M-m})/(2i)
    float* fre = Fs + (warp * 2 + 0) * nm1;
    float* fim = Fs + (warp * 2 + 1) * nm1;
    if (live) {
        float2* X = reinterpret_cast<float2*>(bufs + warp * FFT::ROW_FLOATS);
        FFT::fwd(v, lane, twt, X);
#pragma unroll
        for (int r = 0; r < Q; ++r) X[FFT::pad(FFT::fwd_index(r, lane))] = v[r];
        __syncwarp();
        for (int m = lane; m <= n_max; m += 32) {
            const float2 A = X[FFT::pad(m)];
            const float2 Bc = cconj(X[FFT::pad((FFT::M - m) & (FFT::M - 1))]);
            const float2 E = cscale(cadd(A, Bc), 0.5f);
            const float2 D = csub(A, Bc);
            const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
            const float2 Fm = cadd(E, cmul(twm[m], O));
            fre[m] = Fm.x;
            fim[m] = Fm.y;
        }
    } else {
        for (int m = lane; m <= n_max; m += 32) {
            fre[m] = 0.f;
            fim[m] = 0.f;
        }
    }
    __syncthreads();

    // ---- spectra out
    if (p.Fblk) {
        // per (ring group q, m, re/im): one 16-byte row of 8 rings per half;
        // re and im of an image are adjacent rows (one 32-byte sector)
        const int ncol = 2 * p.batch_total;
        for (int e = threadIdx.x; e < 4 * nm1; e += blockDim.x) {
            const int c = e & 1, t = e >> 1;
            const int q = t / nm1, m = t - q * nm1;
            uint32_t hv[4], lv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float x0 = Fs[((8 * q + 2 * k) * 2 + c) * nm1 + m];
                const float x1 = Fs[((8 * q + 2 * k + 1) * 2 + c) * nm1 + m];
                const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
                hv[k] = __bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                lv[k] = __bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            const size_t o = fblk_row(m, i0 + 8 * q, 2 * b + c, p.n_chunks, ncol);
            *reinterpret_cast<uint4*>(p.Fblk + o) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
            *reinterpret_cast<uint4*>(p.Fblk + p.fblk_half + o) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
        }
    } else {
        for (int e = threadIdx.x; e < 32 * nm1; e += blockDim.x) {
            const int rr = e & 15, c = (e >> 4) & 1, m = e >> 5;
            const int i = i0 + rr;
            if (i < p.n_rho)
                p.F[(((size_t)m * p.batch_total + b) * 2 + c) * p.n_rho + i] = Fs[(rr * 2 + c) * nm1 + m];
        }
    }
}

// ------------------------------------------------------------------ host plan
struct FusedPlan {
    bool ok = false;            // every slot fits one stage buffer
    int n_live = 0;             // bands holding rings < n_rho
    int n_all = 0;              // bands up to the last 64-ring chunk (operand blocks)
    int* order = nullptr;       // [n_all] bands by decreasing weight (bands past n_rho last)
    int* order_live = nullptr;  // [n_live] the live bands by decreasing weight
    int2* band_st = nullptr;    // [n_all]
    FuStage* stages = nullptr;
    // per staged row: (x) buffer offset minus 4 x first unit, i.e. the
    // shared-memory index of pixel 0 of the row, (y) the same for the next
    // row, (z) buffer offset | units << 16 | 1 << 31 when the span reaches
    // outside the image, (w) first 16-byte unit
    int4* rows = nullptr;
    long long staged_floats = 0;  // floats staged per image, all bands
    ~FusedPlan() {
        cudaFree(order);
        cudaFree(order_live);
        cudaFree(band_st);
        cudaFree(stages);
        cudaFree(rows);
    }
};

static inline int floordiv4(int x) { return x >= 0 ? x / 4 : -((-x + 3) / 4); }

// Row footprint of a set of samples: per image row, the pixel range
// [lo, hi] that their 2x2 stencils touch (lo > hi: none).
struct Footprint {
    int y0 = 0;
    std::vector<int> lo, hi;
    bool empty() const { return lo.empty(); }
    int rows() const { return (int)lo.size(); }
    void add(int y, int xa, int xb) {
        if (lo.empty()) {
            y0 = y;
            lo.assign(1, xa);
            hi.assign(1, xb);
            return;
        }
        if (y < y0) {
            lo.insert(lo.begin(), y0 - y, INT32_MAX);
            hi.insert(hi.begin(), y0 - y, INT32_MIN);
            y0 = y;
        } else if (y >= y0 + rows()) {
            lo.resize(y - y0 + 1, INT32_MAX);
            hi.resize(y - y0 + 1, INT32_MIN);
        }
        lo[y - y0] = std::min(lo[y - y0], xa);
        hi[y - y0] = std::max(hi[y - y0], xb);
    }
    void merge(const Footprint& o) {
        for (int r = 0; r < o.rows(); ++r)
            if (o.lo[r] <= o.hi[r]) add(o.y0 + r, o.lo[r], o.hi[r]);
    }
    long long floats() const {
        long long f = 0;
        for (int r = 0; r < rows(); ++r)
            if (lo[r] <= hi[r]) f += 4ll * (floordiv4(hi[r]) - floordiv4(lo[r]) + 1);
        return f;
    }
};

static int build_fused(zm_plan_t p, const GeoImage& g, FusedPlan* fp) {
    const int N = p->n_theta, n_rho = p->n_rho;
    const int nslot = N / FU_SLOT;
    std::vector<float> rho(n_rho);
    std::vector<float2> cs(N);
    ZM_CUDA_TRY(cudaMemcpy(rho.data(), p->rho32, sizeof(float) * n_rho, cudaMemcpyDeviceToHost));
    ZM_CUDA_TRY(cudaMemcpy(cs.data(), p->cs, sizeof(float2) * N, cudaMemcpyDeviceToHost));
    fp->n_live = (n_rho + FU_R - 1) / FU_R;
    fp->n_all = std::max(fp->n_live, p->n_chunks * (64 / FU_R));
    std::vector<int2> band_st(fp->n_all, make_int2(0, 0));
    std::vector<FuStage> stages;
    std::vector<int4> rows;
    std::vector<long long> weight(fp->n_all, -1);
    long long staged = 0;
    for (int band = 0; band < fp->n_live; ++band) {
        const int ia = band * FU_R, ib = std::min(n_rho, ia + FU_R);
        band_st[band].x = (int)stages.size();
        long long wsum = 0;
        Footprint cur;
        int cur_lo = 0;
        long long cur_f = 0;
        auto close = [&](int end_slot) {
            FuStage st = {};
            st.y_lo = cur.y0;
            st.nrows = cur.rows();
            st.row0 = (int)rows.size();
            st.h_lo = cur_lo;                  // slots are half-registers
            st.h_hi = end_slot;
            int soff = 0, bytes = 0;
            const size_t first = rows.size();
            for (int r = 0; r < cur.rows(); ++r) {
                const int y = cur.y0 + r;
                if (cur.lo[r] <= cur.hi[r]) {
                    const int xu = floordiv4(cur.lo[r]);
                    const int nu = floordiv4(cur.hi[r]) - xu + 1;
                    const bool inside = y >= 0 && y < g.h && xu >= 0 && xu + nu <= g.w / 4;
                    rows.push_back(make_int4(soff - 4 * xu, 0, soff | (nu << 16) | (inside ? 0 : (int)0x80000000u), xu));
                    soff += 4 * nu;
                    if (y >= 0 && y < g.h) {
                        const int xa = std::max(xu, 0), xb = std::min(xu + nu, g.w / 4);
                        if (xb > xa) bytes += 16 * (xb - xa);
                    }
                } else {
                    rows.push_back(make_int4(soff, 0, soff, 0));
                }
            }
            for (size_t k = first; k + 1 < rows.size(); ++k) rows[k].y = rows[k + 1].x;
            st.bytes = bytes;
            stages.push_back(st);
            wsum += soff + 256;   // a fixed cost per stage (its two barriers)
            staged += soff;
        };
        for (int sl = 0; sl < nslot; ++sl) {
            Footprint f;
            for (int i = ia; i < ib; ++i) {
                const float rad = g.r * rho[i];
                for (int k = sl * FU_SLOT; k < (sl + 1) * FU_SLOT; ++k) {
                    const float X = std::fmaf(rad, cs[k].x, g.cx);
                    const float Y = std::fmaf(-rad, cs[k].y, g.cy);
                    const float xf = std::floor(X), yf = std::floor(Y);
                    if (!(std::fabs(xf) < 1e9f && std::fabs(yf) < 1e9f)) return ZM_OK;   // not planned
                    const int x0 = (int)xf, y0 = (int)yf;
                    f.add(y0, x0, x0 + 1);
                    f.add(y0 + 1, x0, x0 + 1);
                }
            }
            const long long ff = f.floats();
            if (ff > FU_STAGE_FLOATS || f.rows() > FU_MAX_ROWS) return ZM_OK;   // a slot too large: not fused
            if (!cur.empty()) {
                Footprint u = cur;
                u.merge(f);
                const long long uf = u.floats();
                if (uf <= FU_STAGE_FLOATS && u.rows() <= FU_MAX_ROWS && uf <= FU_MERGE_SLACK * (cur_f + ff)) {
                    cur = std::move(u);
                    cur_f = uf;
                    continue;
                }
                close(sl);
            }
            cur = std::move(f);
            cur_lo = sl;
            cur_f = ff;
        }
        close(nslot);
        band_st[band].y = (int)stages.size();
        if (band_st[band].y - band_st[band].x > nslot) return ZM_OK;   // cannot happen: one stage per slot at most
        weight[band] = wsum;
    }
    std::vector<int> order(fp->n_all);
    for (int j = 0; j < fp->n_all; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return weight[a] > weight[c]; });
    std::vector<int> order_live;
    for (int j : order)
        if (j < fp->n_live) order_live.push_back(j);
    ZM_CUDA_TRY(cudaMalloc(&fp->order, sizeof(int) * order.size()));
    ZM_CUDA_TRY(cudaMalloc(&fp->order_live, sizeof(int) * order_live.size()));
    ZM_CUDA_TRY(cudaMalloc(&fp->band_st, sizeof(int2) * band_st.size()));
    ZM_CUDA_TRY(cudaMalloc(&fp->stages, sizeof(FuStage) * std::max<size_t>(1, stages.size())));
    ZM_CUDA_TRY(cudaMalloc(&fp->rows, sizeof(int4) * std::max<size_t>(1, rows.size())));
    ZM_CUDA_TRY(cudaMemcpy(fp->order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    ZM_CUDA_TRY(cudaMemcpy(fp->order_live, order_live.data(), sizeof(int) * order_live.size(), cudaMemcpyHostToDevice));
    ZM_CUDA_TRY(cudaMemcpy(fp->band_st, band_st.data(), sizeof(int2) * band_st.size(), cudaMemcpyHostToDevice));
    if (!stages.empty())
        ZM_CUDA_TRY(cudaMemcpy(fp->stages, stages.data(), sizeof(FuStage) * stages.size(), cudaMemcpyHostToDevice));
    if (!rows.empty())
        ZM_CUDA_TRY(cudaMemcpy(fp->rows, rows.data(), sizeof(int4) * rows.size(), cudaMemcpyHostToDevice));
    fp->staged_floats = staged;
    fp->ok = true;
    return ZM_OK;
}

struct FusedCache {
    std::mutex mu;
    std::map<std::tuple<zm_plan_t, int, int, float, float, float>, std::unique_ptr<FusedPlan>> plans;
};
static FusedCache g_fused;

void release_fused(zm_plan_t p) {
    std::lock_guard<std::mutex> lk(g_fused.mu);
    for (auto it = g_fused.plans.begin(); it != g_fused.plans.end();) {
        if (std::get<0>(it->first) == p) it = g_fused.plans.erase(it);
        else ++it;
    }
}

static int get_fused(zm_plan_t p, const GeoImage& g, FusedPlan** out) {
    std::lock_guard<std::mutex> lk(g_fused.mu);
    auto key = std::make_tuple(p, g.h, g.w, g.cx, g.cy, g.r);
    auto it = g_fused.plans.find(key);
    if (it == g_fused.plans.end()) {
        auto fp = std::make_unique<FusedPlan>();
        const int s = build_fused(p, g, fp.get());
        if (s != ZM_OK) return s;
        it = g_fused.plans.emplace(key, std::move(fp)).first;
    }
    *out = it->second.get();
    return ZM_OK;
}

// An image the fused kernel can stage: 16-byte aligned base, a row pitch and
// a width that are multiples of 4 floats, and a plan whose angle count the
// warp FFT takes with 32 lanes.
bool fused_eligible(zm_plan_t p, const zm_image_t& im) {
    return p->n_theta >= 64 && p->n_theta <= 2048 && ((uintptr_t)im.data & 15u) == 0 && (im.pitch & 3) == 0 &&
           (im.width & 3) == 0 && im.width < (1 << 28) && im.height < (1 << 28);
}

static size_t fused_smem(int logn, int n_max) {
    switch (logn) {
        case 6: return FuSmem<6>::bytes(n_max);
        case 7: return FuSmem<7>::bytes(n_max);
        case 8: return FuSmem<8>::bytes(n_max);
        case 9: return FuSmem<9>::bytes(n_max);
        case 10: return FuSmem<10>::bytes(n_max);
        case 11: return FuSmem<11>::bytes(n_max);
        default: return ~(size_t)0;
    }
}

template <int LOGN>
static int launch_fused_t(zm_plan_t p, FuParams& fp_, int grid, cudaStream_t st) {
    const size_t smem = FuSmem<LOGN>::bytes(p->n_max);
    int dev = p->device;
    static size_t configured[64] = {0};
    if (smem > 48 * 1024 && (dev < 0 || dev >= 64 || smem > configured[dev])) {
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_ring_fused<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev >= 0 && dev < 64) configured[dev] = smem;
    }
    ZM_LAUNCH_PDL("k_ring_fused", k_ring_fused<LOGN>, dim3(grid), dim3(FU_THREADS), smem, st, fp_);
    return ZM_OK;
}

// Ring spectra of images [b0, b0 + nb) of a batch of `batch` (one geometry,
// all fused-eligible) into F (FP32) or Fblk (operand blocks); fhat_out, when
// set, also receives the polar samples.  Returns ZM_EUNSUPPORTED, having
// launched nothing, when the geometry does not fit the stage buffers.
int launch_ring_fused(zm_plan_t p, const zm_image_t* imgs, int b0, int nb, int batch, float* F, uint8_t* Fblk,
                      float* fhat_out, cudaStream_t st) {
    const GeoImage g = resolve(imgs[b0]);
    FusedPlan* fp = nullptr;
    int s = get_fused(p, g, &fp);
    if (s != ZM_OK) return s;
    if (!fp->ok) return ZM_EUNSUPPORTED;
    if (fused_smem(p->log_theta, p->n_max) > 227 * 1024) return ZM_EUNSUPPORTED;
    static thread_local FuParams kp;
    kp.order = Fblk ? fp->order : fp->order_live;
    kp.band_st = fp->band_st;
    kp.stages = fp->stages;
    kp.rows = fp->rows;
    kp.rho32 = p->rho32;
    kp.cs = p->cs;
    kp.tw = p->tw;
    kp.Fblk = Fblk;
    kp.fblk_half = fblk_half_bytes(p->n_max, p->n_chunks, 2 * batch);
    kp.F = F;
    kp.fhat_out = fhat_out;
    kp.status = p->status;
    kp.n_rho = p->n_rho;
    kp.n_max = p->n_max;
    kp.batch_total = batch;
    kp.n_chunks = p->n_chunks;
    kp.h = g.h;
    kp.w = g.w;
    kp.cx = g.cx;
    kp.cy = g.cy;
    kp.r = g.r;
    const int nbands = Fblk ? fp->n_all : fp->n_live;
    for (int c0 = b0; c0 < b0 + nb; c0 += FU_MAX_IMG) {
        const int nc = std::min(FU_MAX_IMG, b0 + nb - c0);
        kp.b_off = c0;
        kp.nb = nc;
        for (int j = 0; j < nc; ++j) {
            kp.data[j] = imgs[c0 + j].data;
            kp.pitch[j] = imgs[c0 + j].pitch;
        }
        const int grid = nbands * nc;
        switch (p->log_theta) {
            case 6: s = launch_fused_t<6>(p, kp, grid, st); break;
            case 7: s = launch_fused_t<7>(p, kp, grid, st); break;
            case 8: s = launch_fused_t<8>(p, kp, grid, st); break;
            case 9: s = launch_fused_t<9>(p, kp, grid, st); break;
            case 10: s = launch_fused_t<10>(p, kp, grid, st); break;
            case 11: s = launch_fused_t<11>(p, kp, grid, st); break;
            default: return ZM_EUNSUPPORTED;
        }
        if (s != ZM_OK) return s;
    }
    return ZM_OK;
}

// Bytes the fused kernel stages per image for this plan and geometry (the
// spans of 16-byte units), for the roofline; 0 when the geometry is not fused.
long long fused_staged_bytes(zm_plan_t p, const zm_image_t& im) {
    FusedPlan* fp = nullptr;
    if (get_fused(p, resolve(im), &fp) != ZM_OK || !fp->ok) return 0;
    return 4 * fp->staged_floats;
}

}  // namespace zm
