// The angular sums of Eq. 1 on the tensor cores, from polar samples: for bf16
// plans with the blocked projection, F_m(rho_i) = sum_k f(rho_i, theta_k)
// e^{-j m theta_k}, m <= n_max <= 127, as the product of the samples (rings x
// angles) with the DFT matrix (dft_tiles.cuh), written straight into the
// projection's bf16 hi / lo operand blocks.  Where the radix FFT transforms
// all N/2 + 1 bins of each ring, this computes only the 2 * ceil((n_max+1)/8)*8
// real columns the projection reads.
//
// One CTA = one image and 128 consecutive rings (the MMA's M); the angles run
// in stages of 32 (two K = 16 steps of tcgen05.mma, kind::f16, N = 2 * ncols,
// FP32 accumulator in TMEM).  Both operands are split into bf16 hi + lo and
// the accumulator takes A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// Warp roles.  Warps 0-15 (512 threads) produce the A tiles: thread (row r,
// quarter q) loads angles 8q .. 8q + 7 of ring r with two coalesced 16-byte
// loads, four stages ahead in registers, splits them and stores one 16-byte
// core-matrix row of the hi tile and one of the lo tile; stages go in pairs
// (one slot wait, one proxy fence per pair), after which a warp's lane 0
// arrives on both stages' "full" barriers.  Warp 17 (lane 0) bulk-copies each
// stage's DFT tiles into its B slot once the slot's previous MMAs are done;
// the copy arrives on the same "full" barrier (17 arrivals and the copy's
// bytes complete it).  Warp 16 (lane 0) issues the six MMAs of a stage once
// that barrier completes and commits them to the "done" barriers of the
// stage's A slot and B slot; an MMA issue blocks while the tensor pipe is
// busy, so this thread does nothing else.  Eight A slots and three B slots: a slot's round trip
// (written, fenced, read by the MMAs, seen done) spans several stages, and
// with fewer slots the producers and the tensor core took turns.  Every wait is
// bounded (2 s from the kernel's start); one that runs out sets the plan's
// status word to ZM_ETIMEOUT, the producers stop, the issued copies and MMAs
// drain (bounded again) and TMEM is freed.
//
// After the last stage the producer warps read the accumulator (rows = TMEM
// lanes, four warps per lane quarter) into shared memory, and all threads
// write the operand blocks (rings past n_rho hold zeros: their A rows were
// zero).
#include <cuda_bf16.h>

#include <algorithm>

#include "dft_tiles.cuh"
#include "tc_common.cuh"
#include "zm_internal.cuh"

namespace zm {

constexpr int PD_M = 128;                 // rings per CTA = MMA M
constexpr int PD_K = 32;                  // angles per stage (two MMA K-steps)
constexpr int PD_NA = 8;                  // A-tile slots (the producers run up to 8 stages ahead)
constexpr int PD_NB = 3;                  // DFT-tile slots
constexpr int PD_PROD = 512;              // producer threads (warps 0-15)
constexpr int PD_THREADS = PD_PROD + 64;  // + the MMA warp and the DFT-tile warp
constexpr int PD_AHALF = PD_M * PD_K * 2;           // bytes of one 16-bit A tile half (8 KB)
constexpr int PD_ASLOT = 2 * PD_AHALF;              // hi + lo
constexpr int PD_AREGION = PD_NA * PD_ASLOT;        // 128 KB
constexpr int PD_DEPTH = 4;               // stages of samples a producer holds in registers (two pairs)

struct PdParams {
    const float* fhat;        // polar samples [batch_total][n_rho][n_theta], 16-byte aligned
    const uint8_t* dft;       // 32-deep DFT tiles (dft_tiles.cuh)
    uint8_t* Fblk;            // operand blocks (fblk_row)
    size_t fblk_half;
    int* status;
    int n_rho, n_max, batch_total, b_off, nb, n_chunks, n_theta;
    int ntile;                // ceil(n_rho / 128)
    int ncol2;                // MMA N
    int nstage;               // n_theta / 32
};

__host__ __device__ inline size_t pd_btile(int ncol2) { return (size_t)ncol2 * PD_K * 2; }   // one half
inline size_t pd_smem_bytes(int ncol2) {
    return (size_t)PD_AREGION + (size_t)PD_NB * 2 * pd_btile(ncol2) + 8 * (2 * PD_NA + PD_NB) + 16;
}

__device__ __forceinline__ void pd_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n"
                 ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void pd_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// x split into bf16 hi + lo, two values at a time: (hi pair, lo pair), lower k
// in the low half
__device__ __forceinline__ void pd_split2(float a, float b, uint32_t* hi, uint32_t* lo) {
    const __nv_bfloat162 h = __float22bfloat162_rn(make_float2(a, b));
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __float22bfloat162_rn(make_float2(a - hf.x, b - hf.y));
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
}

__global__ void __launch_bounds__(PD_THREADS, 1) k_polar_dft(const __grid_constant__ PdParams p) {
    extern __shared__ __align__(1024) unsigned char psm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t bt = pd_btile(p.ncol2);
    uint8_t* areg = psm;                                          // [slot][hi, lo][8 KB]
    uint8_t* breg = psm + PD_AREGION;                             // [slot][hi, lo][bt]
    uint64_t* bars = reinterpret_cast<uint64_t*>(breg + PD_NB * 2 * bt);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * PD_NA + PD_NB);
    volatile int* okflag = reinterpret_cast<volatile int*>(tslot + 1);
    const uint32_t bar0 = smem_u32(bars);
    // per A slot: "full" (the stage's A tile and DFT tiles are in: 16 producer
    // warps and the tile copier arrive, the copy's bytes complete it) and
    // "done" (MMA commit); per B slot: "done" (MMA commit).  One barrier for
    // both tiles: the MMA thread's waits are on its critical path.
    auto bar_full = [&](int slot) { return bar0 + 8u * (uint32_t)slot; };
    auto bar_adone = [&](int slot) { return bar0 + 8u * (uint32_t)(PD_NA + slot); };
    auto bar_bdone = [&](int slot) { return bar0 + 8u * (uint32_t)(2 * PD_NA + slot); };

    const int tile = blockIdx.x % p.ntile;
    const int b = p.b_off + blockIdx.x / p.ntile;
    const int ns = p.nstage;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(256u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k < PD_NA; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_full(k)), "r"(PD_PROD / 32 + 1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_adone(k)));
        }
        for (int k = 0; k < PD_NB; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_bdone(k)));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *okflag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    griddep_wait();                          // the polar samples come from the previous kernel
    const unsigned long long t0 = global_ns();

    if (warp < PD_PROD / 32) {
        // ---- producers: thread (row, kq) takes angles 8 kq .. 8 kq + 7 of every stage
        const int row = tid >> 2, kq = tid & 3;
        const int ring = tile * PD_M + row;
        const bool live = ring < p.n_rho;
        const float* src = p.fhat + ((size_t)b * p.n_rho + (live ? ring : 0)) * p.n_theta + 8 * kq;
        const uint32_t aoff = dft_tile_off<PD_K>(row, 8 * kq);
        float4 q[PD_DEPTH][2];
        auto load = [&](int s, float4 (&d)[2]) {
            if (live && s < ns) {
                d[0] = __ldg(reinterpret_cast<const float4*>(src + PD_K * s));
                d[1] = __ldg(reinterpret_cast<const float4*>(src + PD_K * s + 4));
            } else {
                d[0] = d[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
#pragma unroll
        for (int j = 0; j < PD_DEPTH; ++j) load(j, q[j]);
        // stages go in pairs: one wait, one proxy fence and one arrival per
        // barrier for two stages (the fence and the wait are the long steps)
        bool ok = true;
        for (int s0 = 0; s0 < ns && ok; s0 += PD_DEPTH) {
#pragma unroll
            for (int h = 0; h < PD_DEPTH / 2; ++h) {
                const int s = s0 + 2 * h;
                if (s >= ns || !ok) break;                    // warp-uniform
                // the pair's slots were read by the MMAs of stages s - NA and
                // s + 1 - NA.  Lane 0 waits (512 threads polling one barrier
                // word serialise), the warp's barrier orders the other lanes'
                // stores after it, and the warp decides together.
                int w = 1;
                if (lane == 0)
                    for (int st = min(s + 1, ns - 1); st >= s && w; --st)
                        if (st >= PD_NA) w = mbar_wait(bar_adone(st % PD_NA), (uint32_t)((st / PD_NA) - 1) & 1u, t0);
                __syncwarp();
                if (!__shfl_sync(0xffffffffu, w, 0)) {
                    ok = false;
                    if (lane == 0) {
                        *okflag = 0;
                        atomicExch(p.status, ZM_ETIMEOUT);
                    }
                    break;
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int st = s + u;
                    if (st < ns) {
                        float4 (&d)[2] = q[2 * h + u];
                        uint32_t hv[4], lv[4];
                        pd_split2(d[0].x, d[0].y, &hv[0], &lv[0]);
                        pd_split2(d[0].z, d[0].w, &hv[1], &lv[1]);
                        pd_split2(d[1].x, d[1].y, &hv[2], &lv[2]);
                        pd_split2(d[1].z, d[1].w, &hv[3], &lv[3]);
                        uint8_t* a = areg + (st % PD_NA) * PD_ASLOT;
                        *reinterpret_cast<uint4*>(a + aoff) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<uint4*>(a + PD_AHALF + aoff) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                        load(st + PD_DEPTH, d);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // A tiles -> tensor core
                __syncwarp();
                if (lane == 0) {
                    pd_arrive(bar_full(s % PD_NA));
                    if (s + 1 < ns) pd_arrive(bar_full((s + 1) % PD_NA));
                }
            }
        }
    } else if (warp == PD_PROD / 32 && lane == 0) {
        // ---- warp 16, lane 0: MMAs only (an issue blocks while the tensor
        // pipe is busy, so this thread does nothing else between stages)
        const uint32_t idesc = instr_desc(p.ncol2, 0);
        int n_issued = 0;
        auto ready = [&](int s) {
            return mbar_wait(bar_full(s % PD_NA), (uint32_t)(s / PD_NA) & 1u, t0);
        };
        bool ok = ns == 0 || ready(0);
        for (int s = 0; s < ns && ok; ++s) {
            const int sa = s % PD_NA, sb = s % PD_NB;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(areg + sa * PD_ASLOT), al = ah + PD_AHALF;
            const uint32_t bh = smem_u32(breg + sb * 2 * bt), bl = bh + (uint32_t)bt;
#pragma unroll
            for (int j = 0; j < PD_K / 16; ++j) {
                const uint64_t dah = smem_desc(ah + 256u * j, 512), dal = smem_desc(al + 256u * j, 512);
                const uint64_t dbh = smem_desc(bh + 256u * j, 512), dbl = smem_desc(bl + 256u * j, 512);
                pd_mma(tmem, dah, dbh, idesc, (s > 0 || j > 0) ? 1u : 0u);
                pd_mma(tmem, dah, dbl, idesc, 1u);
                pd_mma(tmem, dal, dbh, idesc, 1u);
                // wait for the next stage's tiles while this stage's MMAs are queued
                if (j == 0 && s + 1 < ns) ok = ready(s + 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_adone(sa))
                         : "memory");
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_bdone(sb))
                         : "memory");
            ++n_issued;
        }
        // the MMAs complete in order: the last commit covers them all
        if (ok && ns > 0) ok = mbar_wait(bar_adone((ns - 1) % PD_NA), (uint32_t)((ns - 1) / PD_NA) & 1u, t0);
        if (!ok) {
            *okflag = 0;
            atomicExch(p.status, ZM_ETIMEOUT);
            // let the issued MMAs drain before TMEM is freed (each "done"
            // barrier has at most one phase outstanding: a stage is issued only
            // after the producers saw the slot's previous MMAs complete)
            const unsigned long long t1 = global_ns();
            for (int k = 0; k < PD_NA; ++k) {
                const int cm = (n_issued + PD_NA - 1 - k) / PD_NA;
                if (cm > 0) mbar_wait(bar_adone(k), (uint32_t)(cm - 1) & 1u, t1);
            }
        }
    } else if (warp == PD_PROD / 32 + 1 && lane == 0) {
        // ---- warp 17, lane 0: the DFT tiles of stage s into B slot s % NB once
        // the MMAs of stage s - NB (the slot's last reader) have completed
        int n_fetched = 0;
        bool ok = true;
        for (int s = 0; s < ns; ++s) {
            const int slot = s % PD_NB;
            if (s >= PD_NB && !mbar_wait(bar_bdone(slot), (uint32_t)((s / PD_NB) - 1) & 1u, t0)) {
                ok = false;
                break;
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_full(s % PD_NA)),
                         "r"((uint32_t)(2 * bt))
                         : "memory");
            bulk_copy(smem_u32(breg + slot * 2 * bt), p.dft + (size_t)s * 2 * bt, (uint32_t)(2 * bt), bar_full(s % PD_NA));
            ++n_fetched;
        }
        if (!ok) {
            *okflag = 0;
            atomicExch(p.status, ZM_ETIMEOUT);
            // the copies in flight land before the kernel ends: wait (bounded)
            // for the "full" phase of the last stage fetched into each A slot
            // (one phase at most outstanding: a stage is fetched after the
            // MMAs of the slot's previous stage completed)
            const unsigned long long t1 = global_ns();
            for (int k = 0; k < PD_NA; ++k) {
                const int cb = (n_fetched + PD_NA - 1 - k) / PD_NA;
                if (cb > 0) mbar_wait(bar_full(k), (uint32_t)(cb - 1) & 1u, t1);
            }
        }
    }

    // ---- epilogue: accumulator -> shared memory -> operand blocks
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool fine = *okflag != 0;
    griddep_launch();
    const int nm1 = p.n_max + 1, ncols = p.ncol2 / 2;
    // D[col][row], rows fastest: every MMA has completed and every bulk copy
    // landed, so the tile slots are free (ncol2 * 512 bytes <= the A and B regions)
    float* D = reinterpret_cast<float*>(psm);
    if (fine && warp < PD_PROD / 32) {
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of D), 16-column
        // chunks w / 4, w / 4 + 4, ...
        const int qd = warp & 3;
        for (int c0 = 16 * (warp >> 2); c0 < p.ncol2; c0 += 64) {
            uint32_t rr[16];
            const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                  "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                  "=r"(rr[14]), "=r"(rr[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) D[(c0 + j) * PD_M + qd * 32 + lane] = __uint_as_float(rr[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u));
    }
    if (!fine) return;
    // per (m, re/im, group of 8 rings) one 16-byte row per half; ring groups
    // vary fastest over the threads (distinct banks, consecutive 128-byte rows)
    const int ncol = 2 * p.batch_total;
    const int last_ring = p.n_chunks * 64;       // the blocks end with the last 64-ring chunk
    for (int e = tid; e < 2 * nm1 * 16; e += blockDim.x) {
        const int qg = e & 15, c = (e >> 4) & 1, m = e >> 5;
        const int ring0 = tile * PD_M + 8 * qg;
        if (ring0 >= last_ring) continue;
        const float* src = D + (c * ncols + m) * PD_M + 8 * qg;
        const float4 x0 = *reinterpret_cast<const float4*>(src), x1 = *reinterpret_cast<const float4*>(src + 4);
        const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) pd_split2(xs[2 * k], xs[2 * k + 1], &hv[k], &lv[k]);
        const size_t off = fblk_row(m, ring0, 2 * b + c, p.n_chunks, ncol);
        *reinterpret_cast<uint4*>(p.Fblk + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(p.Fblk + p.fblk_half + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
}

// ------------------------------------------------------------------ host
bool polar_dft_eligible(zm_plan_t p, const float* fhat) {
    return p->pdft_mode > 0 && p->prec == PREC_BF16X3 && blocked_projection(p) && p->n_max <= 127 &&
           p->n_theta >= PD_K && p->n_theta % PD_K == 0 && ((uintptr_t)fhat & 15u) == 0;
}

// The plan's 32-deep DFT tiles (built on first use; freed with the plan).
static int pdft_table(zm_plan_t p) {
    if (p->dft32) return ZM_OK;
    ZM_CUDA_TRY(cudaMalloc(&p->dft32, dft_table_bytes<PD_K>(p->n_theta, p->n_max)));
    k_build_dft_tiles<PD_K><<<p->n_theta / PD_K, 256>>>(p->n_theta, p->n_max, dft_ncols(p->n_max), p->dft32);
    ZM_LAUNCH_CHECK("k_build_dft_tiles");
    ZM_CUDA_TRY(cudaDeviceSynchronize());
    return ZM_OK;
}

// Operand blocks of the spectra of images [b0, b0 + nb) of a batch of `batch`
// from their polar samples fhat[b][i][k] (b the index in the batch).
int launch_polar_dft(zm_plan_t p, const float* fhat, int b0, int nb, int batch, uint8_t* Fblk, cudaStream_t st) {
    int s = pdft_table(p);
    if (s != ZM_OK) return s;
    const int ncols = dft_ncols(p->n_max);
    const size_t smem = pd_smem_bytes(2 * ncols);
    static size_t configured[64] = {0};
    const int dev = p->device;
    if (dev < 0 || dev >= 64 || smem > configured[dev]) {
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_polar_dft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev >= 0 && dev < 64) configured[dev] = smem;
    }
    PdParams kp;
    kp.fhat = fhat;
    kp.dft = p->dft32;
    kp.Fblk = Fblk;
    kp.fblk_half = fblk_half_bytes(p->n_max, p->n_chunks, 2 * batch);
    kp.status = p->status;
    kp.n_rho = p->n_rho;
    kp.n_max = p->n_max;
    kp.batch_total = batch;
    kp.n_chunks = p->n_chunks;
    kp.n_theta = p->n_theta;
    kp.ntile = (p->n_rho + PD_M - 1) / PD_M;
    kp.ncol2 = 2 * ncols;
    kp.nstage = p->n_theta / PD_K;
    const int per_launch = std::max(1, (1 << 30) / kp.ntile);
    for (int c0 = b0; c0 < b0 + nb; c0 += per_launch) {
        kp.b_off = c0;
        kp.nb = std::min(per_launch, b0 + nb - c0);
        ZM_LAUNCH_PDL("k_polar_dft", k_polar_dft, dim3(kp.nb * kp.ntile), dim3(PD_THREADS), smem, st, kp);
    }
    return ZM_OK;
}

}  // namespace zm
