// Moments (Eq. 1): bilinear polar resampling (Sec. 2.5) fused with a real FFT of
// every ring (the e^{-j m theta} factor), then the radial projection with the
// (n+1)/pi weight, and the Neumann factor of Eq. 14-15.
#include <cuda_bf16.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "ring_fft.cuh"
#include "zm_internal.cuh"

namespace zm {

int launch_projection_tc(zm_plan_t p, const float* F, int batch, float* out, unsigned flags, cudaStream_t st);

// ============================================================== K-b
constexpr int KB_MAX_IMG = 128;

struct KbParams {
    int n_rho, n_max, batch_total, b_off;
    int nb;                // images in this launch
    uint8_t* Fblk;         // bf16 hi / lo operand blocks of F (R = 8), or NULL
    size_t fblk_half;      // bytes of one half
    int n_chunks;          // 64-node chunks of the radial index
    const float* rho32;    // [n_rho]
    const float2* cs;      // [N] (cos theta_k, sin theta_k)
    const float2* tw;      // [N] e^{-2 pi i j / N}
    float* F;              // [n_max+1][batch_total][2][n_rho]
    float* fhat_out;       // [batch_total][n_rho][N] or NULL
    const float* fhat_in;  // [batch_total][n_rho][N] (polar input mode)
    int discard_in;        // fhat_in is the plan's scratch: its L2 lines are dropped once read
    GeoImage img[KB_MAX_IMG];
};

enum { KB_GATHER = 0, KB_POLAR = 1, KB_RESAMPLE = 2 };

// Bilinear value at pixel coordinates (X, Y); neighbours outside the image are 0.
__device__ __forceinline__ float bilinear(const GeoImage& im, float X, float Y) {
    const float xf = floorf(X), yf = floorf(Y);
    const float fx = X - xf, fy = Y - yf;
    const int x0 = (int)fminf(fmaxf(xf, -2.f), (float)im.w + 1.f);
    const int y0 = (int)fminf(fmaxf(yf, -2.f), (float)im.h + 1.f);
    const float* d = im.data;
    const bool xa = (unsigned)x0 < (unsigned)im.w, xb = (unsigned)(x0 + 1) < (unsigned)im.w;
    const bool ya = (unsigned)y0 < (unsigned)im.h, yb = (unsigned)(y0 + 1) < (unsigned)im.h;
    const float* r0 = d + (long long)y0 * im.pitch;
    const float* r1 = r0 + im.pitch;
    const float p00 = (xa && ya) ? __ldg(r0 + x0) : 0.f;
    const float p01 = (xb && ya) ? __ldg(r0 + x0 + 1) : 0.f;
    const float p10 = (xa && yb) ? __ldg(r1 + x0) : 0.f;
    const float p11 = (xb && yb) ? __ldg(r1 + x0 + 1) : 0.f;
    const float top = fmaf(fx, p01 - p00, p00);
    const float bot = fmaf(fx, p11 - p10, p10);
    return fmaf(fy, bot - top, top);
}

// One CTA = R consecutive rings of one image at a time, one warp per ring
// (R = blockDim/32); the grid is persistent and each CTA walks ring blocks
// (image, block) after loading the FFT twiddles once.
// Phase 1: the R x N samples into shared memory (bilinear gather; polar input
// goes straight from global memory into the FFT registers).  Phase 2: per
// warp, the N-point real FFT of its ring as an N/2-point complex FFT plus the
// split
//   F_m = (Z_m + conj Z_{M-m})/2 + e^{-2 pi i m/N} (Z_m - conj Z_{M-m})/(2i),
// for m = 0..n_max.  Phase 3: F[m][b][re/im][i0..i0+R) written as segments.
template <int LOGN, int MODE>
__global__ void __launch_bounds__(256, (LOGN >= 11 ? 2 : 4)) k_ring_spectra(const __grid_constant__ KbParams p) {
    using FFT = RingFFT<LOGN>;
    constexpr int N = FFT::N;
    constexpr int ROW = FFT::ROW_FLOATS;
    extern __shared__ __align__(16) float smem[];
    const int R = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_rho = p.n_rho;
    const int n_max = p.n_max;
    float* rings = smem;
    float* Fs = smem + R * ROW;                  // [2][n_max+1][R]
    float2* twt = reinterpret_cast<float2*>(smem + ((R * ROW + 2 * (n_max + 1) * R + 1) & ~1));
    float2* twm = twt + FFT::TW_FLOAT2;            // e^{-2 pi i m / N}, m <= n_max
    if (MODE != KB_RESAMPLE) {
        FFT::load_twiddles(twt, p.tw);
        for (int m = threadIdx.x; m <= n_max; m += blockDim.x) twm[m] = __ldg(&p.tw[m]);
    }
    // with operand blocks, ring blocks run up to the last 64-node chunk (rings
    // past n_rho are zero), so that every block of the chunk is written
    const int n_rb = p.Fblk ? p.n_chunks * (64 / R) : (n_rho + R - 1) / R;
    const int n_items = n_rb * p.nb;
    // polar input: this warp's ring of a ring block straight into the FFT
    // registers (lane t holds z[t + L s]); the next block's ring is loaded as
    // soon as the current FFT has left the registers
    float2 v[FFT::Q];
    auto load_ring = [&](int item) {
        const int bl = item / n_rb;
        const int i = (item - bl * n_rb) * R + warp;
        const bool live = lane < FFT::L && i < n_rho;
        const float* src = p.fhat_in + ((size_t)(p.b_off + bl) * n_rho + (live ? i : 0)) * N;
        if ((reinterpret_cast<uintptr_t>(p.fhat_in) & 7) == 0) {
            const float2* z = reinterpret_cast<const float2*>(src);
#pragma unroll
            for (int s = 0; s < FFT::Q; ++s) v[s] = live ? __ldg(&z[lane + FFT::L * s]) : make_float2(0.f, 0.f);
        } else {
#pragma unroll
            for (int s = 0; s < FFT::Q; ++s) {
                const int j = lane + FFT::L * s;
                v[s] = live ? make_float2(__ldg(src + 2 * j), __ldg(src + 2 * j + 1)) : make_float2(0.f, 0.f);
            }
        }
    };
    if (MODE == KB_POLAR && (int)blockIdx.x < n_items) load_ring(blockIdx.x);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int bl = item / n_rb;
        const int i0 = (item - bl * n_rb) * R;
        const int b = p.b_off + bl;
        if (MODE != KB_POLAR) {
            const GeoImage im = p.img[bl];
#pragma unroll 4
            for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
                const int r = idx >> LOGN, k = idx & (N - 1);
                const int i = i0 + r;
                float vv = 0.f;
                if (i < n_rho) {
                    const float rad = im.r * __ldg(&p.rho32[i]);
                    const float2 c = __ldg(&p.cs[k]);
                    vv = bilinear(im, fmaf(rad, c.x, im.cx), fmaf(-rad, c.y, im.cy));
                    if (p.fhat_out) p.fhat_out[((size_t)b * n_rho + i) * N + k] = vv;
                }
                if (MODE != KB_RESAMPLE) rings[r * ROW + k] = vv;
            }
        }
        if (MODE == KB_RESAMPLE) continue;
        __syncthreads();   // the twiddles (first block) and the gathered rings

        {
            float* row = rings + warp * ROW;
            if (MODE != KB_POLAR) {
                const float2* z = reinterpret_cast<const float2*>(row);
#pragma unroll
                for (int s = 0; s < FFT::Q; ++s)
                    v[s] = (lane < FFT::L) ? z[lane + FFT::L * s] : make_float2(0.f, 0.f);
                __syncwarp();
            }
            float2* X = reinterpret_cast<float2*>(row);
            FFT::fwd(v, lane, twt, X);                 // the row doubles as the transpose buffer
            if (lane < FFT::L) {
#pragma unroll
                for (int r = 0; r < FFT::Q; ++r) X[FFT::pad(FFT::fwd_index(r, lane))] = v[r];
            }
            __syncwarp();
            if (MODE == KB_POLAR && item + (int)gridDim.x < n_items) load_ring(item + gridDim.x);
            for (int m = lane; m <= n_max; m += 32) {
                const float2 A = X[FFT::pad(m)];
                const float2 B = cconj(X[FFT::pad((FFT::M - m) & (FFT::M - 1))]);
                const float2 E = cscale(cadd(A, B), 0.5f);
                const float2 D = csub(A, B);
                const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
                const float2 Fm = cadd(E, cmul(twm[m], O));
                Fs[m * R + warp] = Fm.x;
                Fs[((n_max + 1) + m) * R + warp] = Fm.y;
            }
        }
        __syncthreads();
        const int nm1 = n_max + 1;
        if (p.Fblk) {
            // R = 8 rings = one 16-byte row per (m, re/im): bf16 hi and lo halves
            const int ncol = 2 * p.batch_total;
            for (int e = threadIdx.x; e < 2 * nm1; e += blockDim.x) {
                const int c = e >= nm1 ? 1 : 0;
                const int m = e - c * nm1;
                const float* src = Fs + (size_t)e * 8;
                uint32_t h[4], l[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(src[2 * q]), h1 = __float2bfloat16_rn(src[2 * q + 1]);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(src[2 * q] - __bfloat162float(h0));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(src[2 * q + 1] - __bfloat162float(h1));
                    h[q] = __bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    l[q] = __bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
                const size_t o = fblk_row(m, i0, 2 * b + c, p.n_chunks, ncol);
                *reinterpret_cast<uint4*>(p.Fblk + o) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(p.Fblk + p.fblk_half + o) = make_uint4(l[0], l[1], l[2], l[3]);
            }
        } else {
            const int lgR = __ffs(R) - 1;                 // R is a power of two
            const int tot = 2 * nm1 * R;
            for (int e = threadIdx.x; e < tot; e += blockDim.x) {
                const int r = e & (R - 1);
                const int cm = e >> lgR;
                const int c = cm >= nm1 ? 1 : 0;
                const int m = cm - c * nm1;
                const int i = i0 + r;
                if (i < n_rho) p.F[(((size_t)m * p.batch_total + b) * 2 + c) * n_rho + i] = Fs[e];
            }
        }
        __syncthreads();   // rings and Fs are refilled for the next block
    }
}

// Polar samples -> ring spectra as bf16 operand blocks (the blocked
// projection's F), one item = a block of 8 rings of a group of 4 images (one
// 8-column group of the blocks).  Warp w transforms ring i0 + w of the 4
// images in turn (the next ring's samples are loaded as soon as the current
// FFT has left the registers), splits each into F_m, m <= n_max, and stages
// them as Fs[image][re/im][ring][m]; then 8 consecutive threads write one
// full 128-byte line (8 columns x 8 rings) per order and half.
// Occupancy: three CTAs per SM at N = 1024 (shared memory, 69 KB each), so the
// register bound is set for three (77 registers; at 64 for four the kernel was
// 0.7 us per batch of 16 4K frames slower).
template <int LOGN>
__global__ void __launch_bounds__(256, (LOGN >= 11 ? 2 : (LOGN == 10 ? 3 : 4)))
    k_ring_blk(const __grid_constant__ KbParams p) {
    using FFT = RingFFT<LOGN>;
    constexpr int N = FFT::N;
    constexpr int ROW = FFT::ROW_FLOATS;
    constexpr int R = 8;                           // rings per block = warps
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_rho = p.n_rho, n_max = p.n_max, nm1 = n_max + 1;
    float* rows = smem;                                       // [R][ROW]
    float* Fs = smem + R * ROW;                               // [4][2][R][nm1]
    float2* twt = reinterpret_cast<float2*>(smem + ((R * ROW + 64 * nm1 + 3) & ~3));
    float2* twm = twt + FFT::TW_FLOAT2;                       // e^{-2 pi i m / N}, m <= n_max
    FFT::load_twiddles(twt, p.tw);
    for (int m = threadIdx.x; m <= n_max; m += blockDim.x) twm[m] = __ldg(&p.tw[m]);
    const int n_rb = p.n_chunks * (64 / R);
    const int g0 = p.b_off >> 2, g1 = (p.b_off + p.nb - 1) >> 2;
    const int ng = g1 - g0 + 1;
    const int n_items = n_rb * ng;
    const int ncol = 2 * p.batch_total;
    auto in_run = [&](int b) { return b >= p.b_off && b < p.b_off + p.nb; };
    float2 v[FFT::Q];
    // the ring of (item, q) for this warp
    auto load_ring = [&](int item, int q) {
        const int gi = item / n_rb;
        const int i = (item - gi * n_rb) * R + warp;
        const int b = (g0 + gi) * 4 + q;
        const bool live = lane < FFT::L && i < n_rho && in_run(b);
        const float* src = p.fhat_in + ((size_t)(live ? b : 0) * n_rho + (live ? i : 0)) * N;
        if ((reinterpret_cast<uintptr_t>(p.fhat_in) & 7) == 0) {
            const float2* z = reinterpret_cast<const float2*>(src);
#pragma unroll
            for (int s2 = 0; s2 < FFT::Q; ++s2) v[s2] = live ? __ldg(&z[lane + FFT::L * s2]) : make_float2(0.f, 0.f);
        } else {
#pragma unroll
            for (int s2 = 0; s2 < FFT::Q; ++s2) {
                const int j = lane + FFT::L * s2;
                v[s2] = live ? make_float2(__ldg(src + 2 * j), __ldg(src + 2 * j + 1)) : make_float2(0.f, 0.f);
            }
        }
    };
    griddep_wait();                                           // the polar samples are written
    griddep_launch();
    if ((int)blockIdx.x < n_items) load_ring(blockIdx.x, 0);
    __syncthreads();                                          // twiddles
    float* row = rows + warp * ROW;
    float2* X = reinterpret_cast<float2*>(row);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int gi = item / n_rb;
        const int rb = item - gi * n_rb;
        const int i0 = rb * R;
        for (int q = 0; q < 4; ++q) {
            FFT::fwd(v, lane, twt, X);
            if constexpr (N >= 32) {
                // the ring's samples are in the registers now: when they are the
                // plan's scratch, their L2 lines are invalidated without a write
                // back (every line of a ring row belongs to that ring alone)
                const int b = (g0 + gi) * 4 + q;
                if (p.discard_in && i0 + warp < n_rho && in_run(b)) {
                    const char* base = reinterpret_cast<const char*>(p.fhat_in + ((size_t)b * n_rho + i0 + warp) * N);
                    for (int l = lane; l < N / 32; l += 32)
                        asm volatile("discard.global.L2 [%0], 128;" ::"l"(base + 128 * l) : "memory");
                }
            }
            if (lane < FFT::L) {
#pragma unroll
                for (int r = 0; r < FFT::Q; ++r) X[FFT::pad(FFT::fwd_index(r, lane))] = v[r];
            }
            __syncwarp();
            // the next ring into the registers while this one is split
            if (q < 3) load_ring(item, q + 1);
            else if (item + (int)gridDim.x < n_items) load_ring(item + gridDim.x, 0);
            float* fre = Fs + ((q * 2 + 0) * R + warp) * nm1;
            float* fim = Fs + ((q * 2 + 1) * R + warp) * nm1;
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
            __syncwarp();                                     // X is rewritten by the next FFT
        }
        __syncthreads();
        // (m, column) -> one 16-byte row of 8 rings; columns of images outside
        // this run (or past the batch) are left to their own launch
        for (int e = threadIdx.x; e < 8 * nm1; e += blockDim.x) {
            const int col8 = e & 7, m = e >> 3;
            const int q = col8 >> 1, c = col8 & 1;
            const int b = (g0 + gi) * 4 + q;
            if (!in_run(b)) continue;
            const float* src = Fs + ((q * 2 + c) * R) * nm1 + m;
            uint32_t h[4], l[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float x0 = src[(2 * k) * nm1], x1 = src[(2 * k + 1) * nm1];
                const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
                h[k] = __bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                l[k] = __bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            const size_t o = fblk_row(m, i0, 2 * b + c, p.n_chunks, ncol);
            *reinterpret_cast<uint4*>(p.Fblk + o) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(p.Fblk + p.fblk_half + o) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        __syncthreads();                                      // Fs is refilled for the next item
    }
}

template <int LOGN>
static int launch_blk_t(const KbParams& kp, int nb, cudaStream_t st) {
    using FFT = RingFFT<LOGN>;
    const size_t smem = sizeof(float) * (((size_t)8 * FFT::ROW_FLOATS + 64 * (kp.n_max + 1) + 3) & ~(size_t)3) +
                        sizeof(float2) * ((size_t)FFT::TW_FLOAT2 + kp.n_max + 1);
    int dev = 0;
    cudaGetDevice(&dev);
    static size_t configured[64] = {0};
    if (smem > 48 * 1024 && (dev >= 64 || smem > configured[dev])) {
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_ring_blk<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev < 64) configured[dev] = smem;
    }
    static std::mutex mu;
    static std::map<size_t, int> resident;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = resident.find(smem);
        if (it != resident.end()) {
            per_sm = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ring_blk<LOGN>, 256, smem) != cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            resident[smem] = per_sm;
        }
    }
    KbParams& k = const_cast<KbParams&>(kp);
    k.nb = nb;
    const int ng = ((kp.b_off + nb - 1) >> 2) - (kp.b_off >> 2) + 1;
    const long long items = (long long)kp.n_chunks * 8 * ng;
    const int grid = (int)std::min<long long>(items, (long long)per_sm * num_sms(dev));
    ZM_LAUNCH_PDL("k_ring_blk", k_ring_blk<LOGN>, dim3(grid), dim3(256), smem, st, kp);
    return ZM_OK;
}

static int launch_blk(int logn, const KbParams& kp, int nb, cudaStream_t st) {
    switch (logn) {
        case 3: return launch_blk_t<3>(kp, nb, st);
        case 4: return launch_blk_t<4>(kp, nb, st);
        case 5: return launch_blk_t<5>(kp, nb, st);
        case 6: return launch_blk_t<6>(kp, nb, st);
        case 7: return launch_blk_t<7>(kp, nb, st);
        case 8: return launch_blk_t<8>(kp, nb, st);
        case 9: return launch_blk_t<9>(kp, nb, st);
        case 10: return launch_blk_t<10>(kp, nb, st);
        case 11: return launch_blk_t<11>(kp, nb, st);
        default: return set_error(ZM_EUNSUPPORTED, "n_theta 2^%d", logn);
    }
}

template <int LOGN, int MODE>
static int launch_kb_t(const KbParams& kp, int R, int nb, cudaStream_t st) {
    using FFT = RingFFT<LOGN>;
    const size_t smem = sizeof(float) * ((size_t)R * FFT::ROW_FLOATS +
                                         (MODE == KB_RESAMPLE ? 0 : (size_t)2 * (kp.n_max + 1) * R + 2)) +
                        (MODE == KB_RESAMPLE ? 0 : sizeof(float2) * ((size_t)FFT::TW_FLOAT2 + kp.n_max + 1));
    int dev = 0;
    cudaGetDevice(&dev);
    static size_t configured[64] = {0};
    if (smem > 48 * 1024 && (dev >= 64 || smem > configured[dev])) {
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_ring_spectra<LOGN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        if (dev < 64) configured[dev] = smem;
    }
    static std::mutex mu;
    static std::map<std::pair<int, size_t>, int> resident;   // (R, smem) -> CTAs per SM
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = resident.find({R, smem});
        if (it != resident.end()) {
            per_sm = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ring_spectra<LOGN, MODE>, R * 32, smem) !=
                    cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            resident[{R, smem}] = per_sm;
        }
    }
    KbParams& k = const_cast<KbParams&>(kp);
    k.nb = nb;
    const long long items = (long long)(kp.Fblk ? kp.n_chunks * (64 / R) : (kp.n_rho + R - 1) / R) * nb;
    const int grid = (int)std::min<long long>(items, (long long)per_sm * num_sms(dev));
    k_ring_spectra<LOGN, MODE><<<grid, R * 32, smem, st>>>(kp);
    ZM_LAUNCH_CHECK("k_ring_spectra");
    return ZM_OK;
}

template <int MODE>
static int launch_kb_mode(int logn, const KbParams& kp, int R, int nb, cudaStream_t st) {
    switch (logn) {
        case 3: return launch_kb_t<3, MODE>(kp, R, nb, st);
        case 4: return launch_kb_t<4, MODE>(kp, R, nb, st);
        case 5: return launch_kb_t<5, MODE>(kp, R, nb, st);
        case 6: return launch_kb_t<6, MODE>(kp, R, nb, st);
        case 7: return launch_kb_t<7, MODE>(kp, R, nb, st);
        case 8: return launch_kb_t<8, MODE>(kp, R, nb, st);
        case 9: return launch_kb_t<9, MODE>(kp, R, nb, st);
        case 10: return launch_kb_t<10, MODE>(kp, R, nb, st);
        case 11: return launch_kb_t<11, MODE>(kp, R, nb, st);
        default: return set_error(ZM_EUNSUPPORTED, "n_theta 2^%d", logn);
    }
}

// ============================================================== K-c (FP32)
// For each m: the (K_m x N_rho) x (N_rho x 2B) product
//   D[n][col] = sum_i A[row(m,n)][i] F[m][col][i],   col = 2b + re/im,
// split over i into S partial sums (part[s][row][col]); k_project_reduce adds
// them in a fixed order and applies the Neumann factor.
constexpr int KC_ROWS = 64, KC_COLS = 32, KC_K = 32;

__global__ void __launch_bounds__(256)
k_project_fp32(const float* __restrict__ A32, const float* __restrict__ F, const int* __restrict__ mrow,
               int n_max, int n_rho, int ncol, int chunk, int P, float* __restrict__ part) {
    __shared__ float As[KC_K][KC_ROWS + 1];
    __shared__ float Fs[KC_K][KC_COLS + 1];
    const int m = blockIdx.x;
    const int col0 = blockIdx.y * KC_COLS;
    const int s = blockIdx.z;
    const int Km = (n_max - m) / 2 + 1;
    const int rowbase = mrow[m];
    const int ib = s * chunk, ie = min(n_rho, ib + chunk);
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    const float* Fm = F + ((size_t)m * ncol + col0) * n_rho;
    for (int rt = 0; rt < Km; rt += KC_ROWS) {
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        for (int kk = ib; kk < ie; kk += KC_K) {
            for (int e = tid; e < KC_ROWS * KC_K; e += 256) {
                const int row = e >> 5, k = e & 31;
                const int gr = rt + row, gk = kk + k;
                As[k][row] = (gr < Km && gk < ie) ? __ldg(&A32[(size_t)(rowbase + gr) * n_rho + gk]) : 0.f;
            }
            for (int e = tid; e < KC_COLS * KC_K; e += 256) {
                const int col = e >> 5, k = e & 31;
                const int gk = kk + k;
                Fs[k][col] = (col0 + col < ncol && gk < ie) ? __ldg(&Fm[(size_t)col * n_rho + gk]) : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < KC_K; ++k) {
                const float a0 = As[k][2 * ty], a1 = As[k][2 * ty + 1];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float f = Fs[k][4 * tx + j];
                    acc[0][j] = fmaf(a0, f, acc[0][j]);
                    acc[1][j] = fmaf(a1, f, acc[1][j]);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int gr = rt + 2 * ty + a;
            if (gr >= Km) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = col0 + 4 * tx + j;
                if (col < ncol) part[((size_t)s * P + rowbase + gr) * ncol + col] = acc[a][j];
            }
        }
    }
}

__global__ void k_project_reduce(const float* __restrict__ part, int S, int P, int ncol,
                                 const int2* __restrict__ pair_nm, const int* __restrict__ mrow,
                                 int batch, int neumann, float* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch * P) return;
    const int b = idx / P, q = idx - b * P;
    const int2 nm = pair_nm[q];
    const int row = mrow[nm.y] + (nm.x - nm.y) / 2;
    float re = 0.f, im = 0.f;
    for (int s = 0; s < S; ++s) {
        const float* ps = part + ((size_t)s * P + row) * ncol + 2 * b;
        re += ps[0];
        im += ps[1];
    }
    const float f = (neumann && nm.y == 0) ? 0.5f : 1.f;
    out[(size_t)idx * 2] = re * f;
    out[(size_t)idx * 2 + 1] = im * f;
}

// Radial split of the FP32 projection: S slices of `chunk` nodes (a multiple
// of KC_K) aiming at the tuned number of CTAs per SM, at most max_slices of
// them (re-deriving S from the chunk never raises it).
static void fp32_split(zm_plan_t p, int batch, long long max_slices, int* S_out, int* chunk_out) {
    const int ctiles = (2 * batch + KC_COLS - 1) / KC_COLS;
    const int base = (p->n_max + 1) * ctiles;
    const int target = (p->tune_split > 0 ? p->tune_split : 4) * num_sms(p->device);
    const int kchunks = (p->n_rho + KC_K - 1) / KC_K;
    long long S = std::max(1, std::min(kchunks, (target + base - 1) / base));
    S = std::max(1ll, std::min(S, max_slices));
    const int chunk = (int)((kchunks + S - 1) / S) * KC_K;
    *S_out = (p->n_rho + chunk - 1) / chunk;
    *chunk_out = chunk;
}

static int launch_projection_fp32(zm_plan_t p, const float* F, int batch, float* out, unsigned flags,
                                  cudaStream_t st) {
    int S, chunk;
    fp32_split(p, batch, 1ll << 40, &S, &chunk);
    const int st_ = p->ws_part.grow(sizeof(float) * (size_t)S * p->P * 2 * batch);
    if (st_ != ZM_OK) return st_;
    return launch_projection_fp32_parts(p, F, batch, out, flags, (float*)p->ws_part.ptr,
                                        p->ws_part.bytes / sizeof(float), st);
}

int launch_projection_fp32_parts(zm_plan_t p, const float* F, int batch, float* out, unsigned flags, float* part,
                                 size_t part_floats, cudaStream_t st) {
    const int ncol = 2 * batch;
    const size_t one_slice = (size_t)p->P * ncol;
    if (one_slice > part_floats)
        return set_error(ZM_EINVAL, "projection partial sums: %zu floats per slice, %zu available", one_slice,
                         part_floats);
    int S, chunk;
    fp32_split(p, batch, (long long)(part_floats / one_slice), &S, &chunk);
    const int ctiles = (ncol + KC_COLS - 1) / KC_COLS;
    dim3 grid(p->n_max + 1, ctiles, S);
    k_project_fp32<<<grid, 256, 0, st>>>(p->A32, F, p->mrow, p->n_max, p->n_rho, ncol,
                                          chunk, p->P, part);
    ZM_LAUNCH_CHECK("k_project_fp32");
    const int tot = batch * p->P;
    k_project_reduce<<<(tot + 255) / 256, 256, 0, st>>>(part, S, p->P, ncol, p->pair_nm, p->mrow, batch,
                                                         (flags & ZM_NEUMANN) ? 1 : 0, out);
    ZM_LAUNCH_CHECK("k_project_reduce");
    return ZM_OK;
}

// ============================================================== driver
static int pick_rings(zm_plan_t p, int batch) {
    if (p->tune_rings == 2 || p->tune_rings == 4 || p->tune_rings == 8) return p->tune_rings;
    int R = 8;
    const int want = 2 * num_sms(p->device);
    while (R > 2 && ((p->n_rho + R - 1) / R) * batch < want) R >>= 1;
    return R;
}

// Fused gather kernel on images [b0, b0 + nb) (any alignment): writes F and,
// when fhat_out is set, the polar samples.
static int launch_gather(zm_plan_t p, const zm_image_t* imgs, int b0, int nb, int batch, float* F, float* fhat_out,
                         bool resample_only, uint8_t* Fblk, cudaStream_t st) {
    const int R = Fblk ? 8 : pick_rings(p, batch);
    static thread_local KbParams kp;
    kp.Fblk = resample_only ? nullptr : Fblk;
    kp.fblk_half = fblk_half_bytes(p->n_max, p->n_chunks, 2 * batch);
    kp.n_chunks = p->n_chunks;
    kp.n_rho = p->n_rho;
    kp.n_max = p->n_max;
    kp.batch_total = batch;
    kp.rho32 = p->rho32;
    kp.cs = p->cs;
    kp.tw = p->tw;
    kp.F = F;
    kp.fhat_out = fhat_out;
    kp.fhat_in = nullptr;
    kp.discard_in = 0;
    for (int c0 = b0; c0 < b0 + nb; c0 += KB_MAX_IMG) {
        const int nc = std::min(KB_MAX_IMG, b0 + nb - c0);
        kp.b_off = c0;
        for (int j = 0; j < nc; ++j) kp.img[j] = resolve(imgs[c0 + j]);
        const int s = resample_only ? launch_kb_mode<KB_RESAMPLE>(p->log_theta, kp, R, nc, st)
                                    : launch_kb_mode<KB_GATHER>(p->log_theta, kp, R, nc, st);
        if (s != ZM_OK) return s;
    }
    return ZM_OK;
}

// Angular transform of given polar samples fhat[b][i][k] -> F (or the
// operand blocks Fblk) for images [b0, b0 + nb) of a batch of `batch`: the
// tensor-core DFT where the plan allows it, else the ring FFT.
static int launch_polar_fft(zm_plan_t p, const float* fhat, int b0, int nb, int batch, float* F, uint8_t* Fblk,
                            cudaStream_t st, bool scratch = false) {
    if (Fblk && polar_dft_eligible(p, fhat)) return launch_polar_dft(p, fhat, b0, nb, batch, Fblk, st);
    const int R = Fblk ? 8 : pick_rings(p, batch);
    static thread_local KbParams kp;
    kp.Fblk = Fblk;
    kp.fblk_half = fblk_half_bytes(p->n_max, p->n_chunks, 2 * batch);
    kp.n_chunks = p->n_chunks;
    kp.n_rho = p->n_rho;
    kp.n_max = p->n_max;
    kp.batch_total = batch;
    kp.rho32 = p->rho32;
    kp.cs = p->cs;
    kp.tw = p->tw;
    kp.F = F;
    kp.fhat_out = nullptr;
    kp.fhat_in = fhat;
    kp.discard_in = scratch && Fblk && ((uintptr_t)fhat & 127u) == 0 ? 1 : 0;
    for (int c0 = b0; c0 < b0 + nb; c0 += 65535) {
        const int nc = std::min(65535, b0 + nb - c0);
        kp.b_off = c0;
        const int s = Fblk ? launch_blk(p->log_theta, kp, nc, st) : launch_kb_mode<KB_POLAR>(p->log_theta, kp, R, nc, st);
        if (s != ZM_OK) return s;
    }
    return ZM_OK;
}

// Ring spectra of a batch.  Polar input: FFT only.  Images: runs of one
// geometry go through the tensor-core DFT kernel when the plan asks for it
// (dft_mode, off by default) and the spectra are wanted as operand blocks
// only (no polar samples out), else through the fused kernel when its fused_mode allows (resampling
// and ring FFT in one pass, polar samples written only to the caller's
// fhat_out);
// other runs of TMA-eligible images go through the tile resampler into the
// polar buffer (the caller's fhat_out, else the plan workspace) and then the
// ring FFT; the rest take the gather kernel.
int launch_spectra(zm_plan_t p, const zm_image_t* imgs, const float* fhat_in, int batch, float* F,
                   float* fhat_out, bool resample_only, cudaStream_t st, uint8_t* Fblk) {
    if (fhat_in) return launch_polar_fft(p, fhat_in, 0, batch, batch, F, Fblk, st);
    const bool fuse = p->fused_mode > 0 ||
                      (p->fused_mode == 0 && (long long)p->n_rho * p->n_theta <= FUSED_AUTO_SAMPLES);
    const bool dft = Fblk && !fhat_out && !resample_only && !p->tune_gather && p->dft_mode > 0;
    auto use_dft = [&](int b) { return dft && dft_eligible(p, imgs[b]); };
    auto use_fused = [&](int b) { return fuse && !resample_only && !p->tune_gather && fused_eligible(p, imgs[b]); };
    auto use_tma = [&](int b) { return !p->tune_gather && tma_eligible(imgs[b]); };
    float* fh = fhat_out;
    int b = 0;
    while (b < batch) {
        int e = b + 1;
        int s;
        if (use_dft(b)) {
            while (e < batch && use_dft(e) && same_geometry(imgs[b], imgs[e])) ++e;
            s = launch_ring_dft(p, imgs, b, e - b, batch, Fblk, st);
            if (s == ZM_OK) {
                b = e;
                continue;
            }
            if (s != ZM_EUNSUPPORTED) return s;
            e = b + 1;                       // a geometry whose stages the buffers cannot hold
        }
        if (use_fused(b)) {
            while (e < batch && use_fused(e) && same_geometry(imgs[b], imgs[e])) ++e;
            s = launch_ring_fused(p, imgs, b, e - b, batch, F, Fblk, fhat_out, st);
            if (s == ZM_OK) {
                b = e;
                continue;
            }
            if (s != ZM_EUNSUPPORTED) return s;
            e = b + 1;                       // a geometry the stage buffers cannot hold
        }
        if (use_tma(b)) {
            while (e < batch && use_tma(e) && same_geometry(imgs[b], imgs[e])) ++e;
            if (!fh) {
                s = p->ws_fhat.grow(sizeof(float) * (size_t)batch * p->n_rho * p->n_theta);
                if (s != ZM_OK) return s;
                fh = (float*)p->ws_fhat.ptr;
            }
            // the plan's scratch (no caller buffer): the samples are kept in L2
            // for the ring FFT, which drops them once read (not for the opt-in
            // tensor-core DFT, which does not)
            const bool scratch = fh != fhat_out && !resample_only;
            const bool keep = scratch && !(Fblk && polar_dft_eligible(p, fh));
            s = launch_resample_tiles(p, imgs, b, e - b, fh, st, keep);
            if (s == ZM_OK && !resample_only) s = launch_polar_fft(p, fh, b, e - b, batch, F, Fblk, st, scratch);
        } else {
            while (e < batch && !use_tma(e)) ++e;
            s = launch_gather(p, imgs, b, e - b, batch, F, fhat_out, resample_only, Fblk, st);
        }
        if (s != ZM_OK) return s;
        b = e;
    }
    return ZM_OK;
}

int launch_projection(zm_plan_t p, const float* F, int batch, float* out, unsigned flags, cudaStream_t st) {
    if (p->prec == PREC_FP32) return launch_projection_fp32(p, F, batch, out, flags, st);
    return launch_projection_tc(p, F, batch, out, flags, st);
}

// Stage 1 of the moments: ring spectra of a batch (images, or polar samples
// when fhat_in is set) into the plan's workspace, in the form its projection
// reads (bf16 operand blocks for the blocked tensor-core projection, FP32
// rows otherwise).
int launch_stage_spectra(zm_plan_t p, const zm_image_t* imgs, const float* fhat_in, int batch, float* fhat_out,
                         cudaStream_t st) {
    if (blocked_projection(p)) {
        const size_t half = fblk_half_bytes(p->n_max, p->n_chunks, 2 * batch);
        const int s = p->ws_Fblk.grow(2 * half);
        if (s != ZM_OK) return s;
        return launch_spectra(p, imgs, fhat_in, batch, nullptr, fhat_out, false, st, (uint8_t*)p->ws_Fblk.ptr);
    }
    const int s = p->ws_F.grow(sizeof(float) * (size_t)(p->n_max + 1) * batch * 2 * p->n_rho);
    if (s != ZM_OK) return s;
    return launch_spectra(p, imgs, fhat_in, batch, (float*)p->ws_F.ptr, fhat_out, false, st);
}

// Stage 2: the radial projection of the spectra stage 1 left in the workspace
// (consume: no later call reads them, so the blocked form drops them from L2).
int launch_stage_project(zm_plan_t p, int batch, float* out, unsigned flags, cudaStream_t st, bool consume = false) {
    if (blocked_projection(p))
        return launch_projection_blocked(p, (const uint8_t*)p->ws_Fblk.ptr, batch, out, flags, st, consume);
    return launch_projection(p, (const float*)p->ws_F.ptr, batch, out, flags, st);
}

int launch_moments(zm_plan_t p, const zm_image_t* imgs, const float* fhat_in, int batch, float* out,
                   float* fhat_out, unsigned flags, cudaStream_t st) {
    const int s = launch_stage_spectra(p, imgs, fhat_in, batch, fhat_out, st);
    return s != ZM_OK ? s : launch_stage_project(p, batch, out, flags, st, true);
}

}  // namespace zm

using namespace zm;

static int moments_common(zm_plan_t plan, const zm_image_t* imgs, const float* fhat_in, int batch, float* out,
                          float* fhat_out, unsigned flags, void* stream) {
    if (!plan) return set_error(ZM_EINVAL, "plan is NULL");
    if (batch < 1) return set_error(ZM_EINVAL, "batch must be >= 1 (got %d)", batch);
    if (!out) return set_error(ZM_EINVAL, "output pointer is NULL");
    if (flags & ~ZM_NEUMANN) return set_error(ZM_EINVAL, "unknown flags 0x%x", flags);
    if (!fhat_in) {
        const int s = check_images(imgs, batch);
        if (s != ZM_OK) return s;
    }
    DeviceGuard g(plan->device);
    if (!g.ok) return set_error(ZM_ECUDA, "cannot select device %d", plan->device);
    return launch_moments(plan, imgs, fhat_in, batch, out, fhat_out, flags, (cudaStream_t)stream);
}

extern "C" int zm_moments(zm_plan_t plan, const zm_image_t* imgs, int batch, float* out, unsigned flags,
                          void* stream) {
    return moments_common(plan, imgs, nullptr, batch, out, nullptr, flags, stream);
}

extern "C" int zm_moments_ex(zm_plan_t plan, const zm_image_t* imgs, int batch, float* out, float* fhat,
                             unsigned flags, void* stream) {
    return moments_common(plan, imgs, nullptr, batch, out, fhat, flags, stream);
}

extern "C" int zm_moments_polar(zm_plan_t plan, const float* fhat, int batch, float* out, unsigned flags,
                                void* stream) {
    if (!fhat) return set_error(ZM_EINVAL, "fhat is NULL");
    return moments_common(plan, nullptr, fhat, batch, out, nullptr, flags, stream);
}

extern "C" int zm_resample(zm_plan_t plan, const zm_image_t* imgs, int batch, float* fhat, void* stream) {
    if (!plan) return set_error(ZM_EINVAL, "plan is NULL");
    if (!fhat) return set_error(ZM_EINVAL, "fhat is NULL");
    const int s = check_images(imgs, batch);
    if (s != ZM_OK) return s;
    DeviceGuard g(plan->device);
    return launch_spectra(plan, imgs, nullptr, batch, nullptr, fhat, true, (cudaStream_t)stream);
}

extern "C" int zm_ring_spectra(zm_plan_t plan, const zm_image_t* imgs, int batch, float* spectra, float* fhat,
                               void* stream) {
    if (!plan) return set_error(ZM_EINVAL, "plan is NULL");
    if (!spectra) return set_error(ZM_EINVAL, "spectra is NULL");
    const int s = check_images(imgs, batch);
    if (s != ZM_OK) return s;
    DeviceGuard g(plan->device);
    return launch_spectra(plan, imgs, nullptr, batch, spectra, fhat, false, (cudaStream_t)stream);
}

extern "C" int zm_project(zm_plan_t plan, const float* spectra, int batch, float* out, unsigned flags,
                          void* stream) {
    if (!plan || !spectra || !out) return set_error(ZM_EINVAL, "NULL argument");
    if (batch < 1) return set_error(ZM_EINVAL, "batch must be >= 1 (got %d)", batch);
    if (flags & ~ZM_NEUMANN) return set_error(ZM_EINVAL, "unknown flags 0x%x", flags);
    DeviceGuard g(plan->device);
    return launch_projection(plan, spectra, batch, out, flags, (cudaStream_t)stream);
}

extern "C" int zm_stage_spectra(zm_plan_t plan, const zm_image_t* imgs, int batch, void* stream) {
    if (!plan) return set_error(ZM_EINVAL, "plan is NULL");
    const int s = check_images(imgs, batch);
    if (s != ZM_OK) return s;
    DeviceGuard g(plan->device);
    if (!g.ok) return set_error(ZM_ECUDA, "cannot select device %d", plan->device);
    const int r = launch_stage_spectra(plan, imgs, nullptr, batch, nullptr, (cudaStream_t)stream);
    plan->staged_batch = (r == ZM_OK) ? batch : 0;
    return r;
}

extern "C" int zm_stage_project(zm_plan_t plan, int batch, float* out, unsigned flags, void* stream) {
    if (!plan || !out) return set_error(ZM_EINVAL, "NULL argument");
    if (flags & ~ZM_NEUMANN) return set_error(ZM_EINVAL, "unknown flags 0x%x", flags);
    if (batch < 1 || batch != plan->staged_batch)
        return set_error(ZM_EINVAL, "zm_stage_project: batch %d, but the plan holds spectra of %d images", batch,
                         plan->staged_batch);
    DeviceGuard g(plan->device);
    if (!g.ok) return set_error(ZM_ECUDA, "cannot select device %d", plan->device);
    return launch_stage_project(plan, batch, out, flags, (cudaStream_t)stream);
}

extern "C" int zm_plan_reserve(zm_plan_t plan, int batch) {
    if (!plan) return set_error(ZM_EINVAL, "plan is NULL");
    if (batch < 1) return set_error(ZM_EINVAL, "batch must be >= 1");
    DeviceGuard g(plan->device);
    const size_t nb = (size_t)batch;
    int s = plan->ws_F.grow(sizeof(float) * (size_t)(plan->n_max + 1) * nb * 2 * plan->n_rho);
    // polar samples of the tile resampler
    if (s == ZM_OK) s = plan->ws_fhat.grow(sizeof(float) * nb * plan->n_rho * plan->n_theta);
    // projection partials: the radial split never exceeds one slice per 32 nodes
    const size_t S = (size_t)(plan->n_rho + KC_K - 1) / KC_K;
    if (s == ZM_OK) s = plan->ws_part.grow(sizeof(float) * S * plan->P * 2 * nb);
    if (s == ZM_OK) s = plan->ws_colmax.grow(sizeof(unsigned) * 2 * nb);
    if (s == ZM_OK) s = plan->ws_G.grow(sizeof(float) * g_floats(batch, plan->n_rho, plan->n_max));
    // reductions: 64 records per image (pixel errors) or one per ring (fused errors)
    const size_t rec = std::max<size_t>(64, (size_t)plan->n_rho);
    if (s == ZM_OK) s = plan->ws_red.grow(sizeof(double) * nb * rec * 4);
    if (s == ZM_OK) s = plan->ws_scale.grow(sizeof(float) * 2 * nb);
    if (s == ZM_OK && blocked_projection(plan))
        s = plan->ws_Fblk.grow(2 * fblk_half_bytes(plan->n_max, plan->n_chunks, 2 * batch));
    return s;
}
