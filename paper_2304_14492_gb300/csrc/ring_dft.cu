// Polar resampling (Sec. 2.5) and the angular transform of Eq. 1 on the tensor
// cores, for bf16 plans on large grids: image pixels in, the projection's bf16
// operand blocks of F_m(rho_i), m <= n_max, out; the polar samples exist only
// in registers and as a 16-bit operand tile in shared memory.
//
// F_m(rho_i) = sum_k f(rho_i, theta_k) e^{-j m theta_k} is a product of the
// samples (rings x angles) with the DFT matrix (angles x (re, im) of m), so a
// CTA computes it for 128 rings at once as D[ring][col] = sum_k A[ring][k] B[col][k]
// with tcgen05.mma (kind::f16, M = 128, N = 2 * ncols <= 256, K = 16 per
// instruction), the accumulator in TMEM.  Both operands are split into a bf16
// hi and lo part and D accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32
// (the projection's split).  Only the needed m are computed, where the radix
// FFT of the other kernels transforms all N/2 + 1 bins.
//
// Rows: a pair of 64-ring bands, band j and band nb - 1 - j (inner with outer,
// so that every CTA of an image covers the same area); one CTA per (image,
// pair).  The circle is cut into stages of 16 angles, one MMA K-step each.
// Per stage a host-built plan (the kernel's own float operations) lists, per
// band, the image rows the stage's bilinear stencils touch and each row's exact
// span of 16-byte units; 8-lane groups copy the spans with cp.async into one of
// three stage buffers (row entries one stage earlier, as in ring_fused.cu).
// Each thread samples 4 consecutive angles of one ring, splits the values and
// stores them into the stage's A tile (canonical K-major, no swizzle); one
// thread issues the stage's three MMAs a stage later, against the DFT tile of
// the stage that a bulk copy brought in (the plan's table, 13 KB per stage at
// n_max 100).  After the last stage the accumulator goes through shared memory
// into the operand blocks.  Every wait is bounded (2 s); one that runs out sets
// the plan's status word to ZM_ETIMEOUT, lets the issued copies and MMAs drain
// (bounded again) and frees TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "dft_tiles.cuh"
#include "tc_common.cuh"
#include "zm_internal.cuh"

namespace zm {

constexpr int DF_ROWS = 128;              // rings per CTA = MMA M
constexpr int DF_BAND = 64;               // rings per band (two bands per CTA)
constexpr int DF_THREADS = 512;
constexpr int DF_K = 16;                  // angles per stage = MMA K
constexpr int DF_STAGE_FLOATS = 9216;     // floats per stage buffer
constexpr int DF_MAX_ROWS = 384;          // staged rows per stage (both bands)
constexpr int DF_NBUF = 3;                // stage buffers
constexpr int DF_LOOK = DF_NBUF - 1;
constexpr int DF_NENT = 2 * DF_LOOK + 1;  // row-entry buffers
constexpr int DF_NB = 3;                  // DFT tile buffers
constexpr int DF_MAX_IMG = 128;
constexpr int DF_ATILE = DF_ROWS * DF_K * 2;   // bytes of one 16-bit A tile (4 KB)

struct __align__(16) DfStage {
    int ya, na, yb, nb;       // band a / b: first image row and row count (nb = 0: no band b)
    int row0, pad0, pad1, pad2;   // first row entry (band a's rows, then band b's)
};

struct DfParams {
    const DfStage* stages;    // [pair][chunk]
    const int4* rows;         // row entries (as ring_fused.cu)
    const uint8_t* dft;       // DFT tiles: [chunk][hi / lo][ncol2 rows x 16 k], canonical K-major
    const float* rho32;
    const float2* cs;
    uint8_t* Fblk;
    size_t fblk_half;
    int* status;
    int n_rho, n_max, batch_total, b_off, nb, n_chunks, n_theta;
    int nband, npair, nstage;  // 64-ring bands, pairs, stages per pair
    int ncol2;                 // MMA N: 2 * ncols, ncols = 8 * ceil((n_max + 1) / 8)
    int h, w;
    float cx, cy, r;
    const float* data[DF_MAX_IMG];
    long long pitch[DF_MAX_IMG];
};

__device__ __forceinline__ void df_cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

struct DfSmem {
    static constexpr size_t BUFS = (size_t)DF_NBUF * DF_STAGE_FLOATS * 4;           // 110,592 (later D)
    static constexpr size_t ENTS = (size_t)DF_NENT * DF_MAX_ROWS * 16;              // 30,720
    static constexpr size_t ATILES = 2 * 2 * (size_t)DF_ATILE;                      // 16,384
    __host__ __device__ static size_t btile(int ncol2) { return (size_t)ncol2 * DF_K * 2; }   // one half
    static size_t bytes(int ncol2, int nstage) {
        return BUFS + ENTS + ATILES + (size_t)DF_NB * 2 * btile(ncol2) + sizeof(DfStage) * (size_t)nstage + 128;
    }
};
// the accumulator, staged as FP32 [256 columns][128 rows], reuses the stage
// buffers and row entries
static_assert(DfSmem::BUFS + DfSmem::ENTS >= 256u * DF_ROWS * 4u, "accumulator staging does not fit");

__global__ void __launch_bounds__(DF_THREADS, 1) k_ring_dft(const __grid_constant__ DfParams p) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* bufs = reinterpret_cast<float*>(dsm);
    int4* ents = reinterpret_cast<int4*>(dsm + DfSmem::BUFS);
    uint8_t* atiles = dsm + DfSmem::BUFS + DfSmem::ENTS;                           // [2][hi, lo][4 KB]
    const size_t bt = DfSmem::btile(p.ncol2);
    uint8_t* btiles = atiles + DfSmem::ATILES;                                        // [NB][hi, lo][bt]
    DfStage* srec = reinterpret_cast<DfStage*>(btiles + DF_NB * 2 * bt);
    uint64_t* bar_b = reinterpret_cast<uint64_t*>(srec + p.nstage);                  // [NB] DFT tile arrived
    uint64_t* bar_m = bar_b + DF_NB;                                                  // [2] MMAs of a stage done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_m + 2);
    volatile int* okflag = reinterpret_cast<volatile int*>(tslot + 1);

    const int bi = blockIdx.x % p.nb;
    const int pair = blockIdx.x / p.nb;
    const int b = p.b_off + bi;
    const int band_a = pair, band_b = p.nband - 1 - pair;
    const bool has_b = band_b != band_a;
    const int ns = p.nstage;
    const DfStage* stg = p.stages + (size_t)pair * ns;
    for (int j = tid; j < ns; j += blockDim.x) srec[j] = stg[j];
    const uint32_t bb0 = smem_u32(bar_b), bm0 = smem_u32(bar_m);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(256u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k < DF_NB; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bb0 + 8 * k));
        for (int k = 0; k < 2; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bm0 + 8 * k));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *okflag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // this thread's ring and angles: row = tid / 4 (rows 0-63 band a, 64-127
    // band b), angles 16 g + 4 (tid & 3) .. + 3 of stage g
    const int row = tid >> 2, kq = tid & 3;
    const bool in_b = row >= DF_BAND;
    const int ring = in_b ? band_b * DF_BAND + (row - DF_BAND) : band_a * DF_BAND + row;
    const bool live = ring < p.n_rho && (!in_b || has_b);
    const float rad = live ? p.r * __ldg(&p.rho32[ring]) : 0.f;
    const float* img = p.data[bi];
    const long long pitch = p.pitch[bi];
    griddep_wait();                          // the images may come from the previous kernel

    auto fetch_entries = [&](int j) {
        if (j < ns && tid < srec[j].na + srec[j].nb)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(ents + (j % DF_NENT) * DF_MAX_ROWS +
                                                                                   tid)),
                         "l"(p.rows + srec[j].row0 + tid)
                         : "memory");
    };
    const int grp = warp * 4 + (lane >> 3), l8 = lane & 7;
    auto fetch_pixels = [&](int j) {
        if (j >= ns) return;
        const int bb = j % DF_NBUF;
        const DfStage S = srec[j];
        const int nrows = S.na + S.nb;
        const uint32_t buf = smem_u32(bufs + bb * DF_STAGE_FLOATS);
        const int4* ent = ents + (j % DF_NENT) * DF_MAX_ROWS;
#pragma unroll 1
        for (int rr = grp; rr < nrows; rr += DF_THREADS / 8) {
            const int2 e = *reinterpret_cast<const int2*>(&ent[rr].z);
            const int soff = e.x & 0xffff, nu = (e.x >> 16) & 0xfff, xu = e.y;
            const int y = rr < S.na ? S.ya + rr : S.yb + (rr - S.na);
            if (e.x >= 0) {
                const float* src = img + (long long)y * pitch + 4 * xu;
#pragma unroll 1
                for (int u = l8; u < nu; u += 8) df_cp_async16(buf + 16u * (soff / 4 + u), src + 4 * u);
            } else {
                const bool yin = (unsigned)y < (unsigned)p.h;
                const float* src = img + (long long)(yin ? y : 0) * pitch;
                for (int u = l8; u < nu; u += 8) {
                    const int xq = xu + u;
                    if (yin && (unsigned)xq < (unsigned)(p.w >> 2))
                        df_cp_async16(buf + 16u * (soff / 4 + u), src + 4 * xq);
                    else
                        *reinterpret_cast<float4*>(bufs + bb * DF_STAGE_FLOATS + soff + 4 * u) =
                            make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
    };
    // the DFT tile of stage c into buffer c % NB (thread 0)
    int n_issued = 0, n_fetched = 0;        // thread 0: stages whose MMAs / DFT tiles were issued, in order
    auto fetch_dft = [&](int c) {
        ++n_fetched;
        const uint32_t bar = bb0 + 8 * (c % DF_NB);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)(2 * bt))
                     : "memory");
        bulk_copy(smem_u32(btiles + (c % DF_NB) * 2 * bt), p.dft + (size_t)c * 2 * bt, (uint32_t)(2 * bt), bar);
    };
    const unsigned long long t0 = global_ns();
    const uint32_t idesc = instr_desc(p.ncol2, 0);
    // the MMAs of stage s (thread 0): A tile s % 2, DFT tile s % NB
    auto issue_mma = [&](int s) -> bool {
        if (!mbar_wait(bb0 + 8 * (s % DF_NB), (uint32_t)(s / DF_NB) & 1u, t0)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(atiles + (s & 1) * 2 * DF_ATILE), al = ah + DF_ATILE;
        const uint32_t bh = smem_u32(btiles + (s % DF_NB) * 2 * bt), bl = bh + (uint32_t)bt;
        const uint64_t dah = smem_desc(ah, 256), dal = smem_desc(al, 256);
        const uint64_t dbh = smem_desc(bh, 256), dbl = smem_desc(bl, 256);
        const uint32_t acc0 = s > 0 ? 1u : 0u;
        asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n"
                     ::"r"(tmem), "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
        asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n"
                     ::"r"(tmem), "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
        asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n"
                     ::"r"(tmem), "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bm0 + 8 * (s & 1))
                     : "memory");
        ++n_issued;
        return true;
    };

    // prologue
#pragma unroll
    for (int j = 0; j < DF_LOOK; ++j) fetch_entries(j);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (tid == 0) {
        fetch_dft(0);
        if (ns > 1) fetch_dft(1);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < DF_LOOK; ++j) {
        fetch_pixels(j);
        fetch_entries(j + DF_LOOK);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    bool ok = true;
    for (int g = 0; g <= ns; ++g) {
        if (g < ns) asm volatile("cp.async.wait_group %0;" ::"n"(DF_LOOK - 1) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // A tile of stage g - 1 -> tensor core
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0 && *okflag) {
            bool good = true;
            if (g >= 1) good = issue_mma(g - 1);
            // DFT tile g + 1 replaces that of stage g - 2, whose MMAs must be done
            if (good && g + 1 < ns && g + 1 >= DF_NB) {
                good = mbar_wait(bm0 + 8 * ((g - 2) & 1), (uint32_t)((g - 2) >> 1) & 1u, t0);
                if (good) fetch_dft(g + 1);
            } else if (good && g + 1 < ns && g + 1 >= 2) {
                fetch_dft(g + 1);
            }
            if (!good) {
                *okflag = 0;
                atomicExch(p.status, ZM_ETIMEOUT);
            }
        }
        if (g == ns) break;
        fetch_pixels(g + DF_LOOK);
        fetch_entries(g + 2 * DF_LOOK);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // A tile g % 2 was read by the MMAs of stage g - 2
        if (g >= 2 && ok && !mbar_wait(bm0 + 8 * (g & 1), (uint32_t)((g - 2) >> 1) & 1u, t0)) {
            ok = false;
            *okflag = 0;
            atomicExch(p.status, ZM_ETIMEOUT);
        }
        if (!ok) continue;
        const DfStage S = srec[g];
        const float* buf = bufs + (g % DF_NBUF) * DF_STAGE_FLOATS;
        const int4* ent = ents + (g % DF_NENT) * DF_MAX_ROWS + (in_b ? S.na : 0);
        const int y_lo = in_b ? S.yb : S.ya;
        const unsigned nr2 = (unsigned)((in_b ? S.nb : S.na) - 2);
        float val[4] = {0.f, 0.f, 0.f, 0.f};
        if (live) {
            const float4 c01 = __ldg(reinterpret_cast<const float4*>(p.cs + DF_K * g + 4 * kq));
            const float4 c23 = __ldg(reinterpret_cast<const float4*>(p.cs + DF_K * g + 4 * kq + 2));
            const float cc[4] = {c01.x, c01.z, c23.x, c23.z}, ss[4] = {c01.y, c01.w, c23.y, c23.w};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const float X = fmaf(rad, cc[s], p.cx), Y = fmaf(-rad, ss[s], p.cy);
                const float xf = floorf(X), yf = floorf(Y);
                const float fx = X - xf, fy = Y - yf;
                const unsigned ry = min((unsigned)((int)yf - y_lo), nr2);
                const int x0 = (int)xf;
                const int2 rb = *reinterpret_cast<const int2*>(&ent[ry]);
                const unsigned a0 = min((unsigned)(rb.x + x0), (unsigned)(DF_STAGE_FLOATS - 2));
                const unsigned a1 = min((unsigned)(rb.y + x0), (unsigned)(DF_STAGE_FLOATS - 2));
                const float p00 = buf[a0], p01 = buf[a0 + 1], p10 = buf[a1], p11 = buf[a1 + 1];
                const float top = fmaf(fx, p01 - p00, p00);
                const float bot = fmaf(fx, p11 - p10, p10);
                val[s] = fmaf(fy, bot - top, top);
            }
        }
        uint32_t hv[2], lv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(val[2 * q]), h1 = __float2bfloat16_rn(val[2 * q + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(val[2 * q] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(val[2 * q + 1] - __bfloat162float(h1));
            hv[q] = __bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lv[q] = __bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        uint8_t* at = atiles + (g & 1) * 2 * DF_ATILE;
        const uint32_t o = dft_tile_off<DF_K>(row, 4 * kq);
        *reinterpret_cast<uint2*>(at + o) = make_uint2(hv[0], hv[1]);
        *reinterpret_cast<uint2*>(at + DF_ATILE + o) = make_uint2(lv[0], lv[1]);
    }
    // the last stage's MMAs (committed in the final pass above) finish
    bool fine = *okflag != 0 && ok;
    if (tid == 0 && fine && ns > 0 && !mbar_wait(bm0 + 8 * ((ns - 1) & 1), (uint32_t)((ns - 1) >> 1) & 1u, t0)) {
        *okflag = 0;
        atomicExch(p.status, ZM_ETIMEOUT);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    fine = *okflag != 0;
    griddep_launch();
    const int nm1 = p.n_max + 1, ncols = p.ncol2 / 2;
    float* D = bufs;                                   // [re/im][ncols][128], rows fastest
    if (fine) {
        // TMEM lanes 32 w .. 32 w + 31 are rows of D: warps 0-3 read them
        if (warp < 4) {
            for (int c0 = 0; c0 < p.ncol2; c0 += 16) {
                uint32_t rr[16];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                      "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                      "=r"(rr[14]), "=r"(rr[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) D[(c0 + j) * DF_ROWS + warp * 32 + lane] = __uint_as_float(rr[j]);
            }
        }
    } else {
        // a wait ran out: let what was issued drain (bounded) before TMEM is freed
        // (each barrier has at most one phase outstanding: a stage's MMAs are
        // issued after those two stages earlier finished, a DFT tile is
        // fetched after the MMAs that read its buffer finished)
        if (tid == 0) {
            const unsigned long long t1 = global_ns();
            for (int k = 0; k < 2; ++k) {
                const int cnt = (n_issued + 1 - k) / 2;
                if (cnt > 0) mbar_wait(bm0 + 8 * k, (uint32_t)(cnt - 1) & 1u, t1);
            }
            for (int k = 0; k < DF_NB; ++k) {
                const int cnt = (n_fetched + DF_NB - 1 - k) / DF_NB;
                if (cnt > 0) mbar_wait(bb0 + 8 * k, (uint32_t)(cnt - 1) & 1u, t1);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u));
    }
    if (!fine) return;
    // D -> bf16 hi / lo operand blocks: per (m, re/im, group of 8 rings) one
    // 16-byte row per half; ring groups vary fastest over the threads (distinct
    // shared-memory banks; consecutive 128-byte rows of a block)
    const int ncol = 2 * p.batch_total;
    const int ngroups = has_b ? 16 : 8;
    for (int e = tid; e < 2 * nm1 * ngroups; e += blockDim.x) {
        const int q = e % ngroups, c = (e / ngroups) & 1, m = e / (2 * ngroups);
        const float* src = D + (c * ncols + m) * DF_ROWS + 8 * q;
        const float4 x0 = *reinterpret_cast<const float4*>(src), x1 = *reinterpret_cast<const float4*>(src + 4);
        const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(xs[2 * k]), h1 = __float2bfloat16_rn(xs[2 * k + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(xs[2 * k] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(xs[2 * k + 1] - __bfloat162float(h1));
            hv[k] = __bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lv[k] = __bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        const int ring0 = q < 8 ? band_a * DF_BAND + 8 * q : band_b * DF_BAND + 8 * (q - 8);
        const size_t off = fblk_row(m, ring0, 2 * b + c, p.n_chunks, ncol);
        *reinterpret_cast<uint4*>(p.Fblk + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(p.Fblk + p.fblk_half + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
}

// ------------------------------------------------------------------ host plan
struct DftPlan {
    bool ok = false;
    int nband = 0, npair = 0, nstage = 0;
    DfStage* stages = nullptr;
    int4* rows = nullptr;
    long long staged_floats = 0;
    ~DftPlan() {
        cudaFree(stages);
        cudaFree(rows);
    }
};

static inline int floordiv4d(int x) { return x >= 0 ? x / 4 : -((-x + 3) / 4); }

// Rows [y0, y0 + n) and per row the pixel range [lo, hi] the stencils touch.
struct DfFoot {
    int y0 = 0;
    std::vector<int> lo, hi;
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
        } else if (y >= y0 + (int)lo.size()) {
            lo.resize(y - y0 + 1, INT32_MAX);
            hi.resize(y - y0 + 1, INT32_MIN);
        }
        lo[y - y0] = std::min(lo[y - y0], xa);
        hi[y - y0] = std::max(hi[y - y0], xb);
    }
};

static int build_dft(zm_plan_t p, const GeoImage& g, DftPlan* dp) {
    const int N = p->n_theta, n_rho = p->n_rho;
    std::vector<float> rho(n_rho);
    std::vector<float2> cs(N);
    ZM_CUDA_TRY(cudaMemcpy(rho.data(), p->rho32, sizeof(float) * n_rho, cudaMemcpyDeviceToHost));
    ZM_CUDA_TRY(cudaMemcpy(cs.data(), p->cs, sizeof(float2) * N, cudaMemcpyDeviceToHost));
    dp->nband = (n_rho + DF_BAND - 1) / DF_BAND;
    dp->npair = (dp->nband + 1) / 2;
    dp->nstage = N / DF_K;
    std::vector<DfStage> stages;
    std::vector<int4> rows;
    long long staged = 0;
    for (int pr = 0; pr < dp->npair; ++pr) {
        const int bands[2] = {pr, dp->nband - 1 - pr};
        for (int c = 0; c < dp->nstage; ++c) {
            DfStage st = {};
            st.row0 = (int)rows.size();
            int soff = 0;
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && bands[1] == bands[0]) break;
                const int ia = bands[h] * DF_BAND, ib = std::min(n_rho, ia + DF_BAND);
                DfFoot f;
                for (int i = ia; i < ib; ++i) {
                    const float rad = g.r * rho[i];
                    for (int k = DF_K * c; k < DF_K * (c + 1); ++k) {
                        const float X = std::fmaf(rad, cs[k].x, g.cx), Y = std::fmaf(-rad, cs[k].y, g.cy);
                        const float xf = std::floor(X), yf = std::floor(Y);
                        if (!(std::fabs(xf) < 1e9f && std::fabs(yf) < 1e9f)) return ZM_OK;
                        f.add((int)yf, (int)xf, (int)xf + 1);
                        f.add((int)yf + 1, (int)xf, (int)xf + 1);
                    }
                }
                if (f.lo.empty()) continue;
                const size_t first = rows.size();
                for (int r = 0; r < (int)f.lo.size(); ++r) {
                    const int y = f.y0 + r;
                    if (f.lo[r] <= f.hi[r]) {
                        const int xu = floordiv4d(f.lo[r]);
                        const int nu = floordiv4d(f.hi[r]) - xu + 1;
                        const bool inside = y >= 0 && y < g.h && xu >= 0 && xu + nu <= g.w / 4;
                        rows.push_back(make_int4(soff - 4 * xu, 0, soff | (nu << 16) | (inside ? 0 : (int)0x80000000u), xu));
                        soff += 4 * nu;
                    } else {
                        rows.push_back(make_int4(soff, 0, soff, 0));
                    }
                }
                for (size_t k = first; k + 1 < rows.size(); ++k) rows[k].y = rows[k + 1].x;
                if (h == 0) {
                    st.ya = f.y0;
                    st.na = (int)f.lo.size();
                } else {
                    st.yb = f.y0;
                    st.nb = (int)f.lo.size();
                }
            }
            if (soff > DF_STAGE_FLOATS || st.na + st.nb > DF_MAX_ROWS || (st.na > 0 && st.na < 2) ||
                (st.nb > 0 && st.nb < 2) || soff >= 0xffff)
                return ZM_OK;                                  // a stage too large: not this kernel
            staged += soff;
            stages.push_back(st);
        }
    }
    ZM_CUDA_TRY(cudaMalloc(&dp->stages, sizeof(DfStage) * stages.size()));
    ZM_CUDA_TRY(cudaMalloc(&dp->rows, sizeof(int4) * std::max<size_t>(1, rows.size())));
    ZM_CUDA_TRY(cudaMemcpy(dp->stages, stages.data(), sizeof(DfStage) * stages.size(), cudaMemcpyHostToDevice));
    if (!rows.empty())
        ZM_CUDA_TRY(cudaMemcpy(dp->rows, rows.data(), sizeof(int4) * rows.size(), cudaMemcpyHostToDevice));
    dp->staged_floats = staged;
    dp->ok = true;
    return ZM_OK;
}

struct DftCache {
    std::mutex mu;
    std::map<std::tuple<zm_plan_t, int, int, float, float, float>, std::unique_ptr<DftPlan>> plans;
};
static DftCache g_dft;

void release_dft(zm_plan_t p) {
    std::lock_guard<std::mutex> lk(g_dft.mu);
    for (auto it = g_dft.plans.begin(); it != g_dft.plans.end();) {
        if (std::get<0>(it->first) == p) it = g_dft.plans.erase(it);
        else ++it;
    }
}

// The plan's 16-deep DFT tiles (built on first use; freed with the plan).
static int dft_table(zm_plan_t p) {
    if (p->dft) return ZM_OK;
    ZM_CUDA_TRY(cudaMalloc(&p->dft, dft_table_bytes<DF_K>(p->n_theta, p->n_max)));
    k_build_dft_tiles<DF_K><<<p->n_theta / DF_K, 256>>>(p->n_theta, p->n_max, dft_ncols(p->n_max), p->dft);
    ZM_LAUNCH_CHECK("k_build_dft_tiles");
    ZM_CUDA_TRY(cudaDeviceSynchronize());
    return ZM_OK;
}

bool dft_eligible(zm_plan_t p, const zm_image_t& im) {
    return p->prec == PREC_BF16X3 && blocked_projection(p) && p->n_max <= 127 && p->n_theta >= DF_K &&
           p->n_theta % DF_K == 0 && p->n_theta <= 4096 &&
           ((uintptr_t)im.data & 15u) == 0 && (im.pitch & 3) == 0 && (im.width & 3) == 0 &&
           im.width < (1 << 28) && im.height < (1 << 28);
}

// Operand blocks of the spectra of images [b0, b0 + nb) of a batch of `batch`
// (one geometry, all dft-eligible) into Fblk.  Returns ZM_EUNSUPPORTED,
// having launched nothing, when the geometry's stages do not fit the buffers.
int launch_ring_dft(zm_plan_t p, const zm_image_t* imgs, int b0, int nb, int batch, uint8_t* Fblk, cudaStream_t st) {
    const GeoImage g = resolve(imgs[b0]);
    DftPlan* dp = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_dft.mu);
        auto key = std::make_tuple(p, g.h, g.w, g.cx, g.cy, g.r);
        auto it = g_dft.plans.find(key);
        if (it == g_dft.plans.end()) {
            auto np = std::make_unique<DftPlan>();
            const int s = build_dft(p, g, np.get());
            if (s != ZM_OK) return s;
            it = g_dft.plans.emplace(key, std::move(np)).first;
        }
        dp = it->second.get();
    }
    if (!dp->ok) return ZM_EUNSUPPORTED;
    int s = dft_table(p);
    if (s != ZM_OK) return s;
    const int ncols = dft_ncols(p->n_max);
    const size_t smem = DfSmem::bytes(2 * ncols, dp->nstage);
    if (smem > 227 * 1024) return ZM_EUNSUPPORTED;
    static size_t configured[64] = {0};
    const int dev = p->device;
    if (dev < 0 || dev >= 64 || smem > configured[dev]) {
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_ring_dft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev >= 0 && dev < 64) configured[dev] = smem;
    }
    static thread_local DfParams kp;
    kp.stages = dp->stages;
    kp.rows = dp->rows;
    kp.dft = p->dft;
    kp.rho32 = p->rho32;
    kp.cs = p->cs;
    kp.Fblk = Fblk;
    kp.fblk_half = fblk_half_bytes(p->n_max, p->n_chunks, 2 * batch);
    kp.status = p->status;
    kp.n_rho = p->n_rho;
    kp.n_max = p->n_max;
    kp.batch_total = batch;
    kp.n_chunks = p->n_chunks;
    kp.n_theta = p->n_theta;
    kp.nband = dp->nband;
    kp.npair = dp->npair;
    kp.nstage = dp->nstage;
    kp.ncol2 = 2 * ncols;
    kp.h = g.h;
    kp.w = g.w;
    kp.cx = g.cx;
    kp.cy = g.cy;
    kp.r = g.r;
    for (int c0 = b0; c0 < b0 + nb; c0 += DF_MAX_IMG) {
        const int nc = std::min(DF_MAX_IMG, b0 + nb - c0);
        kp.b_off = c0;
        kp.nb = nc;
        for (int j = 0; j < nc; ++j) {
            kp.data[j] = imgs[c0 + j].data;
            kp.pitch[j] = imgs[c0 + j].pitch;
        }
        ZM_LAUNCH_PDL("k_ring_dft", k_ring_dft, dim3(dp->npair * nc), dim3(DF_THREADS), smem, st, kp);
    }
    return ZM_OK;
}

}  // namespace zm
