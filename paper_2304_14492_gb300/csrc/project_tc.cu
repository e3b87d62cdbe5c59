// Radial projection of Eq. 1 on the 5th-generation tensor cores.
//
// For each repetition m the projection is the contraction
//   D[col][n] = sum_i F_m[col][i] A_m[n][i],   col = 2b + re/im,
// with A_m[n][i] = (n+1)/pi * wr_i * 2pi/N_theta * R_nm(rho_i).  Both operands
// are split into a high and a low 16-bit part (bf16 or fp16): x = x_hi + x_lo,
// and the product is accumulated in FP32 as F_hi A_hi + F_hi A_lo + F_lo A_hi
// (the dropped F_lo A_lo term is below the FP32 rounding of the sum).
//
// One CTA = one m, 128 image columns (the MMA's M), all K_m orders (the MMA's
// N, padded to a multiple of 16) and one slice of the radial index i (the
// reduction, split over CTAs and summed by k_project_reduce).  Per 64-wide
// chunk of i: the 128 threads load F (fp32), split it and store both halves in
// the K-major, no-swizzle canonical layout (8-row x 16-byte core matrices;
// core matrices adjacent in K are LBO = 128 B apart, 8-row groups SBO = 1024 B
// apart); the precomputed A halves are copied in the same layout; one thread
// issues 4 k-steps x 3 tcgen05.mma (kind::f16, cta_group::1) into a TMEM
// accumulator and commits them to an mbarrier.  The epilogue reads TMEM with
// tcgen05.ld (warp w owns lanes 32w..32w+31 = columns of D's M dimension).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "tc_common.cuh"
#include "zm_internal.cuh"

namespace zm {

constexpr int TC_M = 128;            // image columns per CTA (MMA M)
constexpr int TC_KC = 64;            // radial nodes per chunk
constexpr int TC_THREADS = 128;
constexpr int TC_NMAX = 256;         // orders per CTA (MMA N upper bound)
constexpr int TC_FTILE = TC_M * TC_KC * 2;          // bytes of one 16-bit F tile

struct TcParams {
    const float* F;          // [n_max+1][ncol][n_rho]
    const uint16_t* Ahi;     // [P][n_rho] m-major rows
    const uint16_t* Alo;
    const int* mrow;
    float* part;             // [S][P][ncol]
    int* status;             // device status word (ZM_ETIMEOUT on a timed-out wait)
    int n_max, n_rho, ncol, P, chunk;
    int ntmax;               // A tile rows reserved in shared memory (widest N of the launch)
    int fp16;                // 0: bf16 halves, 1: fp16 halves (scaled)
    float a_scale;           // A halves hold A * a_scale
    const unsigned* colmax;  // fp16: per column max |F| (float bits); NULL = no scaling
};

// Power-of-two scale putting a column's largest |F| just below 2^14, so the
// fp16 halves neither overflow nor lose the low part to subnormals.
__device__ __forceinline__ float column_scale(const unsigned* colmax, int col) {
    if (!colmax) return 1.f;
    const float mx = __uint_as_float(colmax[col]);
    if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
    int e;
    frexpf(mx, &e);
    return ldexpf(1.f, 14 - e);
}

// max |F[m][col][i]| over m and i, per column, as ordered float bits.
__global__ void k_colmax(const float* __restrict__ F, int nm1, int ncol, int n_rho, unsigned* __restrict__ out) {
    const int col = blockIdx.x;
    float mx = 0.f;
    for (int e = threadIdx.x + blockIdx.y * blockDim.x; e < nm1 * n_rho; e += blockDim.x * gridDim.y) {
        const int m = e / n_rho, i = e - m * n_rho;
        mx = fmaxf(mx, fabsf(__ldg(&F[((size_t)m * ncol + col) * n_rho + i])));
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + col, __float_as_uint(mx));
}

__global__ void __launch_bounds__(TC_THREADS) k_project_tc(const __grid_constant__ TcParams p) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint8_t* fhi = sm;
    uint8_t* flo = sm + TC_FTILE;
    uint8_t* ahi = sm + 2 * TC_FTILE;
    uint8_t* alo = ahi + p.ntmax * TC_KC * 2;
    uint64_t* bar = reinterpret_cast<uint64_t*>(alo + p.ntmax * TC_KC * 2);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    volatile int* okflag = reinterpret_cast<volatile int*>(tslot + 1);

    const int m = blockIdx.x;
    const int col0 = blockIdx.y * TC_M;
    const int s = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Km = (p.n_max - m) / 2 + 1;
    const int rowbase = p.mrow[m];
    const int ib = s * p.chunk;
    const int ie = min(p.n_rho, ib + p.chunk);
    const int vrows = min(TC_M, p.ncol - col0);             // real columns in this tile
    const int n_tiles = (Km + TC_NMAX - 1) / TC_NMAX;
    const int nt_max = min(Km, TC_NMAX);
    const int NTa = ((nt_max + 15) / 16) * 16;             // MMA N of the widest tile
    uint32_t ncols = 32;
    while (ncols < (uint32_t)NTa) ncols <<= 1;

    const uint32_t bar_a = smem_u32(bar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_a), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const float* Fm = p.F + (size_t)m * p.ncol * p.n_rho;
    const bool fvec = (p.n_rho & 3) == 0;
    const bool avec = (p.n_rho & 7) == 0;
    const unsigned long long t0 = global_ns();
    uint32_t phase = 0;
    bool ok = true;

    for (int nt = 0; nt < n_tiles && ok; ++nt) {
        const int n0 = nt * TC_NMAX;
        const int nrow = min(TC_NMAX, Km - n0);
        const int NT = ((nrow + 15) / 16) * 16;
        const uint32_t idesc = instr_desc(NT, p.fp16);
        int first = 1;
        for (int k0 = ib; k0 < ie && ok; k0 += TC_KC) {
            // F chunk -> hi / lo tiles: only the rows of real columns.  Rows past
            // the batch keep stale values; D rows are independent, so they only
            // produce D rows that are never read.
            for (int task = tid; task < vrows * 8; task += TC_THREADS) {
                const int row = task >> 3, g = task & 7;
                const int col = col0 + row;
                const int kk = k0 + g * 8;
                float x[8];
                {
                    const float* src = Fm + (size_t)col * p.n_rho + kk;
                    if (fvec && kk + 8 <= ie) {
                        const float4 a = __ldg(reinterpret_cast<const float4*>(src));
                        const float4 b = __ldg(reinterpret_cast<const float4*>(src) + 1);
                        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
                        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[e] = (kk + e < ie) ? __ldg(src + e) : 0.f;
                    }
                }
                const float fs = column_scale(p.colmax, col);
                uint16_t h[8], l[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) split2(x[e] * fs, p.fp16, &h[e], &l[e]);
                uint4 vh, vl;
                vh.x = h[0] | ((uint32_t)h[1] << 16); vh.y = h[2] | ((uint32_t)h[3] << 16);
                vh.z = h[4] | ((uint32_t)h[5] << 16); vh.w = h[6] | ((uint32_t)h[7] << 16);
                vl.x = l[0] | ((uint32_t)l[1] << 16); vl.y = l[2] | ((uint32_t)l[3] << 16);
                vl.z = l[4] | ((uint32_t)l[5] << 16); vl.w = l[6] | ((uint32_t)l[7] << 16);
                const uint32_t o = tile_off(row, g);
                *reinterpret_cast<uint4*>(fhi + o) = vh;
                *reinterpret_cast<uint4*>(flo + o) = vl;
            }
            // A chunk (hi / lo): rows past K_m likewise only feed unread D columns
            for (int task = tid; task < nrow * 8 * 2; task += TC_THREADS) {
                const int half = task >= nrow * 8;
                const int t2 = half ? task - nrow * 8 : task;
                const int row = t2 >> 3, g = t2 & 7;
                const int kk = k0 + g * 8;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                {
                    const uint16_t* src = (half ? p.Alo : p.Ahi) + (size_t)(rowbase + n0 + row) * p.n_rho + kk;
                    if (avec && kk + 8 <= ie) {
                        v = __ldg(reinterpret_cast<const uint4*>(src));
                    } else {
                        uint16_t e8[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) e8[e] = (kk + e < ie) ? __ldg(src + e) : (uint16_t)0;
                        v.x = e8[0] | ((uint32_t)e8[1] << 16); v.y = e8[2] | ((uint32_t)e8[3] << 16);
                        v.z = e8[4] | ((uint32_t)e8[5] << 16); v.w = e8[6] | ((uint32_t)e8[7] << 16);
                    }
                }
                *reinterpret_cast<uint4*>((half ? alo : ahi) + tile_off(row, g)) = v;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t fh = smem_u32(fhi), fl = smem_u32(flo), ah = smem_u32(ahi), al = smem_u32(alo);
#pragma unroll
                for (int ks = 0; ks < TC_KC / 16; ++ks) {
                    const uint32_t off = ks * 256;      // 16 k = two core matrices along K
                    const uint64_t dfh = smem_desc(fh + off), dfl = smem_desc(fl + off);
                    const uint64_t dah = smem_desc(ah + off), dal = smem_desc(al + off);
                    const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(dfh), "l"(dah), "r"(idesc), "r"(acc0));
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(dfh), "l"(dal), "r"(idesc), "r"(1u));
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(dfl), "l"(dah), "r"(idesc), "r"(1u));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                             : "memory");
            }
            first = 0;
            // the tiles are rewritten next chunk: one thread waits for the MMAs to
            // finish reading them, the others wait at the barrier
            if (tid == 0) {
                const bool done = mbar_wait(bar_a, phase, t0);
                *okflag = done ? 1 : 0;
                if (!done) atomicExch(p.status, ZM_ETIMEOUT);
            }
            phase ^= 1u;
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            ok = *okflag != 0;
        }
        if (!ok) break;
        // epilogue: lanes 32w..32w+31 of TMEM = D rows (image columns)
        const int col = col0 + warp * 32 + lane;
        const float inv = (col < p.ncol) ? 1.0f / (p.a_scale * column_scale(p.colmax, col)) : 0.f;
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (col < p.ncol) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = c0 + j;
                    if (n < nrow)
                        p.part[((size_t)s * p.P + rowbase + n0 + n) * p.ncol + col] = __uint_as_float(r[j]) * inv;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok) {
        // a wait ran out: give in-flight MMAs a bounded time to drain before TMEM is freed
        const unsigned long long t1 = global_ns();
        mbar_wait(bar_a, phase ^ 1u, t1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

__global__ void k_project_reduce_tc(const float* __restrict__ part, int S, int P, int ncol,
                                    const int2* __restrict__ pair_nm, const int* __restrict__ mrow, int batch,
                                    int neumann, float* __restrict__ out) {
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

int launch_projection_tc(zm_plan_t p, const float* F, int batch, float* out, unsigned flags, cudaStream_t st) {
    if (!p->Ahi || !p->Alo) return set_error(ZM_EINVAL, "plan has no tensor-core operands");
    const int ncol = 2 * batch;
    int s = ZM_OK;
    const unsigned* colmax = nullptr;
    if (p->prec == PREC_FP16X3) {
        s = p->ws_colmax.grow(sizeof(unsigned) * (size_t)ncol);
        if (s != ZM_OK) return s;
        ZM_CUDA_TRY(cudaMemsetAsync(p->ws_colmax.ptr, 0, sizeof(unsigned) * (size_t)ncol, st));
        k_colmax<<<dim3(ncol, 4), 256, 0, st>>>(F, p->n_max + 1, ncol, p->n_rho, (unsigned*)p->ws_colmax.ptr);
        ZM_LAUNCH_CHECK("k_colmax");
        colmax = (const unsigned*)p->ws_colmax.ptr;
    }
    const int ctiles = (ncol + TC_M - 1) / TC_M;
    const int base = (p->n_max + 1) * ctiles;
    // enough CTAs to cover the load -> MMA latency: up to one 64-wide chunk of
    // the radial index per CTA, at most 32 slices
    const int target = (p->tune_split > 0 ? p->tune_split : 8) * num_sms(p->device);
    const int kchunks = (p->n_rho + TC_KC - 1) / TC_KC;
    int S = std::max(1, std::min(std::min(kchunks, 32), (target + base - 1) / base));
    const int chunk = ((kchunks + S - 1) / S) * TC_KC;
    S = (p->n_rho + chunk - 1) / chunk;
    s = p->ws_part.grow(sizeof(float) * (size_t)S * p->P * ncol);
    if (s != ZM_OK) return s;
    TcParams tp;
    tp.F = F;
    tp.Ahi = p->Ahi;
    tp.Alo = p->Alo;
    tp.mrow = p->mrow;
    tp.part = (float*)p->ws_part.ptr;
    tp.status = p->status;
    tp.n_max = p->n_max;
    tp.n_rho = p->n_rho;
    tp.ncol = ncol;
    tp.P = p->P;
    tp.chunk = chunk;
    tp.fp16 = p->prec == PREC_FP16X3 ? 1 : 0;
    tp.a_scale = p->a_scale;
    tp.colmax = colmax;
    // Shared memory also caps the resident CTAs so that their TMEM columns
    // (<= 256 each) never exceed the SM's 512.
    const int Km0 = p->n_max / 2 + 1;
    const int NTa = ((std::min(Km0, TC_NMAX) + 15) / 16) * 16;
    tp.ntmax = NTa;
    int ncols = 32;
    while (ncols < NTa) ncols <<= 1;
    const size_t need = 2 * TC_FTILE + 2 * (size_t)NTa * TC_KC * 2 + 64;
    const size_t cap = 227 * 1024;
    const size_t by_tmem = cap / (512 / ncols) + 1024;
    const size_t smem = std::max(need, std::min(cap, by_tmem));
    static size_t configured[64] = {0};
    int dev = p->device;
    if (dev >= 64 || smem > configured[dev]) {
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev < 64) configured[dev] = smem;
    }
    dim3 grid(p->n_max + 1, ctiles, S);
    k_project_tc<<<grid, TC_THREADS, smem, st>>>(tp);
    ZM_LAUNCH_CHECK("k_project_tc");
    const int tot = batch * p->P;
    k_project_reduce_tc<<<(tot + 255) / 256, 256, 0, st>>>(tp.part, S, p->P, ncol, p->pair_nm, p->mrow, batch,
                                                            (flags & ZM_NEUMANN) ? 1 : 0, out);
    ZM_LAUNCH_CHECK("k_project_reduce_tc");
    return ZM_OK;
}

// ============================================================== blocked form
// The same contraction with the roles of the operands swapped and no
// register work in the main loop: one CTA per (m, column tile) computes
//   D[n][col] = sum_i A_m[n][i] F_m[col][i]
// over the whole radial range (no split, no partial sums).  A (the MMA's M
// side, K_m <= 128 rows) comes from the plan's operand blocks, F (the N side,
// up to 256 columns) from blocks the ring-FFT kernel wrote, both already in
// the canonical layout, so each 64-node chunk is four bulk copies into a ring
// of shared-memory stages.  The A copies of the first stages are issued before
// the grid-dependency wait (A is the plan's, F the previous kernel's output).
// One thread waits for a stage, issues its MMAs and commits them to the
// stage's "empty" barrier; a second thread refills each stage as soon as its
// MMAs have read it.  At this size an MMA costs about the same whatever its N,
// so the split products share MMAs: F lo lies right after F hi in a stage, so
// B = [F hi | F lo] (N = 2 x columns) gives A_hi F_hi and A_hi F_lo at once,
// and when every order has at most 64 rows A = [A hi; A lo] on M (rows 0..63,
// 64..127) adds A_lo F_hi (and A_lo F_lo) in the same MMA: one MMA per
// 16-node step instead of three.  The epilogue adds the column halves and the
// lo rows (passed through the consumed stages) and writes the moments
// (Neumann factor applied) straight into out[b][idx(n, m)].
// With ksplit = 2 the radial range is split between the two CTAs of a
// cluster (blockIdx.z = 0, 1): rank 1 stores its partial D into a buffer in
// rank 0's shared memory, and rank 0 adds it to its own after a cluster
// barrier, in a fixed order (deterministic).  Halving the chunks per CTA
// halves the longest copy stream and spreads the orders over twice the SMs.
constexpr int BLK_A_BYTES = 16 * 1024;        // what the M = 128 MMA reads of an A half: 128 rows x 64 k x 2 B
constexpr int BLK_CPC_MAX = 4;                // 64-ring chunks per stage, at most

struct BlkParams {
    const uint8_t* Ablk;
    const long long* ablk_off;
    long long ablk_half;
    const uint8_t* Fblk;
    long long fblk_half;
    float* out;
    int* status;
    int n_max, n_chunks, ncol, P;
    int stages;              // stage ring
    int cpc;                 // 64-ring chunks per stage
    int ksplit;              // 1, or 2: the radial range split over a cluster of two CTAs
    int buf_off;             // byte offset of rank 0's receive buffer (ksplit = 2)
    int neumann;
    float inv_scale;
    int discard_f;           // the F blocks are the call's scratch: their L2 lines are dropped once copied
    int stack;               // K_m <= 64 and 2 NT <= 256: one MMA per k step, A hi and lo stacked on M
};

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__global__ void __launch_bounds__(TC_THREADS) k_project_blk(const __grid_constant__ BlkParams p) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[8];
    __shared__ __align__(8) uint64_t empty[8];
    __shared__ uint32_t tslot;
    __shared__ int okflag;
    __shared__ int mma_done, mma_ok, prod_loaded, prod_ok;
    const int m = blockIdx.x, t = blockIdx.y, z = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Km = (p.n_max - m) / 2 + 1;
    const int rg = (Km + 7) / 8;
    const int cg = (p.ncol + 7) / 8;
    const int cg0 = t * 32, cgt = min(32, cg - cg0);
    const int cols_t = min(256, p.ncol - t * 256);
    const int NT = ((cols_t + 15) / 16) * 16;
    // F lo follows F hi in a stage, so one N = 2 NT MMA reads [F hi | F lo]
    // and A hi once for both products (D columns NT.. hold A_hi F_lo)
    const bool comb = 2 * NT <= 256;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(comb ? 2 * NT : NT)) ncols <<= 1;
    // this CTA's chunks of the radial range
    const int per = (p.n_chunks + p.ksplit - 1) / p.ksplit;
    const int c_begin = z * per;
    const int S = p.stages, nch = min(per, p.n_chunks - c_begin);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[k])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        okflag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (p.ksplit > 1) cluster_sync_all();     // both CTAs of the pair run before any shared memory crosses
    const uint32_t tmem = tslot;
    const uint32_t sm0 = smem_u32(sm);

    // a stage holds p.cpc consecutive 64-ring chunks, each as
    // [A hi: rg KB][A lo: rg KB][F hi: bg KB][F lo: bg KB], or, stacked,
    // [A hi: rg KB, padded to 8 KB][A lo: rg KB][F hi][F lo]; the M = 128 MMA
    // reads 16 KB from an A base, past rg KB into whatever follows (a 16 KB
    // pad after the last stage keeps that inside the allocation): those rows
    // only feed D rows >= K_m (of each half, stacked), which are never read
    const int bg = NT / 8;
    const uint32_t a_bytes = (uint32_t)rg * 1024u, b_bytes = (uint32_t)bg * 1024u;
    const uint32_t a_lo_off = p.stack ? 8192u : a_bytes;
    const uint32_t sub_bytes = a_lo_off + a_bytes + 2u * b_bytes;
    const int cpc = p.cpc;
    const uint32_t stage_bytes = cpc * sub_bytes;
    const size_t a_chunk = (size_t)rg * 1024;
    const uint8_t* a_src = p.Ablk + p.ablk_off[m] + (size_t)c_begin * a_chunk;
    const size_t f_chunk = (size_t)cg * 1024;
    const uint8_t* f_src = p.Fblk + (((size_t)m * p.n_chunks + c_begin) * cg + cg0) * 1024;
    const int nst = (nch + cpc - 1) / cpc;            // stage loads (groups of chunks)
    const int npre = min(nst, S);                     // stages loaded before the first MMA
    auto subs = [&](int c) { return min(cpc, nch - c * cpc); };
    // stage load, in two parts: the barrier's byte count and the A copies
    // (plan constants), then the F copies (the previous kernel's output)
    auto load_a = [&](int c) {
        const int st = c % S;
        const uint32_t base = sm0 + (uint32_t)st * stage_bytes;
        const uint32_t bar = smem_u32(&full[st]);
        const int ns = subs(c);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)ns * 2u * (a_bytes + (uint32_t)cgt * 1024u))
                     : "memory");
        for (int j = 0; j < ns; ++j) {
            const size_t ch = (size_t)c * cpc + j;
            const uint32_t d = base + j * sub_bytes;
            bulk_copy(d, a_src + ch * a_chunk, a_bytes, bar);
            bulk_copy(d + a_lo_off, a_src + p.ablk_half + ch * a_chunk, a_bytes, bar);
        }
    };
    auto load_f = [&](int c) {
        const int st = c % S;
        const uint32_t base = sm0 + (uint32_t)st * stage_bytes;
        const uint32_t bar = smem_u32(&full[st]);
        const int ns = subs(c);
        for (int j = 0; j < ns; ++j) {
            const size_t ch = (size_t)c * cpc + j;
            const uint32_t d = base + j * sub_bytes;
            bulk_copy(d + a_lo_off + a_bytes, f_src + ch * f_chunk, (uint32_t)cgt * 1024, bar);
            bulk_copy(d + a_lo_off + a_bytes + b_bytes, f_src + p.fblk_half + ch * f_chunk, (uint32_t)cgt * 1024, bar);
        }
    };
    // the first stages' A blocks are in flight while the previous kernel finishes
    if (tid == 0)
        for (int c = 0; c < npre; ++c) load_a(c);
    griddep_wait();                    // the spectra blocks are written, `out` is free
    griddep_launch();

    if (tid == 0) {
        const uint32_t idesc = instr_desc(NT, 0), idesc2 = instr_desc(2 * NT, 0);
        const unsigned long long t0 = global_ns();
        int done = 0;
        bool ok = true;
        for (int c = 0; c < npre; ++c) load_f(c);
        for (int c = 0; c < nst && ok; ++c) {
            const int st = c % S;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((c / S) & 1), t0)) {
                ok = false;
                break;
            }
            const int ns = subs(c);
            for (int j = 0; j < ns; ++j) {
                const uint32_t base = sm0 + (uint32_t)st * stage_bytes + j * sub_bytes;
                const uint32_t ah = base, al = base + a_lo_off;
                const uint32_t fh = al + a_bytes, fl = fh + b_bytes;
#pragma unroll
                for (int ks = 0; ks < TC_KC / 16; ++ks) {
                    const uint32_t off = ks * 256;      // 16 k = two core matrices along K
                    const uint64_t dah = smem_desc(ah + off), dal = smem_desc(al + off);
                    const uint64_t dfh = smem_desc(fh + off), dfl = smem_desc(fl + off);
                    const uint32_t acc0 = (c == 0 && j == 0 && ks == 0) ? 0u : 1u;
                    if (p.stack) {
                        // [A hi; A lo] x [F hi | F lo]: all four products in one MMA
                        asm volatile(
                            "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                            "l"(dah), "l"(dfh), "r"(idesc2), "r"(acc0));
                        continue;
                    }
                    asm volatile(
                        "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                        "l"(dah), "l"(dfh), "r"(comb ? idesc2 : idesc), "r"(acc0));
                    if (!comb)
                        asm volatile(
                            "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                            "l"(dah), "l"(dfl), "r"(idesc), "r"(1u));
                    asm volatile(
                        "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                        "l"(dal), "l"(dfh), "r"(idesc), "r"(1u));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[st]))
                         : "memory");
            done = c + 1;
        }
        if (ok) ok = mbar_wait(smem_u32(&empty[(nst - 1) % S]), (uint32_t)(((nst - 1) / S) & 1), t0);
        mma_done = done;
        mma_ok = ok ? 1 : 0;
    } else if (tid == 32) {
        // the refills: stage k is loaded as soon as the MMAs of stage k - S
        // have read its buffer
        const unsigned long long t0 = global_ns();
        int k = npre;
        bool ok = true;
        for (; k < nst; ++k) {
            if (!mbar_wait(smem_u32(&empty[k % S]), (uint32_t)(((k - S) / S) & 1), t0)) {
                ok = false;
                break;
            }
            load_a(k);
            load_f(k);
        }
        prod_loaded = k;
        prod_ok = ok ? 1 : 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && !(mma_ok && prod_ok)) {
        // a wait ran out: report it, then give the copies and MMAs in flight a
        // bounded time to land before the shared memory and TMEM are released
        atomicExch(p.status, ZM_ETIMEOUT);
        const unsigned long long t1 = global_ns();
        for (int c = mma_done; c < prod_loaded; ++c) mbar_wait(smem_u32(&full[c % S]), (uint32_t)((c / S) & 1), t1);
        if (mma_done > 0)
            mbar_wait(smem_u32(&empty[(mma_done - 1) % S]), (uint32_t)(((mma_done - 1) / S) & 1), t1);
        okflag = 0;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // every F block of this CTA is in shared memory and read by its MMAs: a
    // scratch copy is dead, so its L2 lines are dropped without a write-back
    // (each (m, chunk, column group) block is read by this CTA alone).  The
    // drops take a while; stacked, they wait until after the pair's exchange
    // and go to the warps with nothing left to do
    auto discard_f = [&](int t0, int nt) {
        const int lines = cgt * 8;                     // 128-byte lines per chunk and half
        for (int e = t0; e < nch * 2 * lines; e += nt) {
            const int ch = e / (2 * lines), r = e - ch * 2 * lines;
            const uint8_t* a =
                f_src + (size_t)ch * f_chunk + (r >= lines ? p.fblk_half : 0) + (size_t)(r % lines) * 128;
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
        }
    };
    if (p.discard_f && okflag && !p.stack) discard_f(tid, TC_THREADS);

    // epilogue: TMEM lane = row n_local of D (warp w owns lanes 32w..32w+31)
    // TMEM loads of this warp's 32 lanes, 16 columns each; the values are
    // usable after tmem_wait (whose operands tie them to the wait)
    auto tmem_ld16 = [&](int c0, uint32_t (&r)[16]) {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    };
    auto tmem_wait = [&](uint32_t (&r)[16]) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                       "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                       "+r"(r[14]), "+r"(r[15])
                     :
                     : "memory");
    };
    auto tmem_hold = [&](uint32_t (&r)[16]) {     // orders r after the preceding wait
        asm volatile(""
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                       "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                       "+r"(r[14]), "+r"(r[15])
                     :
                     : "memory");
    };
    // columns c0.. of D, plus (two-column-block form) the A_hi F_lo columns
    // NT + c0.., both loads under one wait
    auto ld_pair16 = [&](int c0, uint32_t (&r)[16]) {
        tmem_ld16(c0, r);
        if (comb) {
            uint32_t q[16];
            tmem_ld16(NT + c0, q);
            tmem_wait(r);
            tmem_hold(q);
#pragma unroll
            for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(q[j]));
        } else {
            tmem_wait(r);
        }
    };
    const int nl = warp * 32 + lane;
    const int bstride = NT + 4;                       // floats per buffer row (16-byte rows, conflict-free)
    const uint32_t buf = sm0 + (uint32_t)p.buf_off;   // rank 0's receive buffer [row][bstride]
    // stacked: D rows 64 + n hold the A_lo products of row n; the warps that
    // hold them pass their sums on through the consumed stages, [row][bstride]
    float* xb = reinterpret_cast<float*>(sm);
    if (p.stack) {
        if (okflag && warp >= 2 && (warp - 2) * 32 < Km) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // after the MMAs' operand reads
            float* row = xb + (nl - 64) * bstride;
            for (int c0 = 0; c0 < NT; c0 += 16) {
                uint32_t r[16];
                ld_pair16(c0, r);
                if (nl - 64 < Km) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(row + c0 + j) =
                            make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                        __uint_as_float(r[j + 3]));
                }
            }
        }
        __syncthreads();
    }
    // the value of D row nl (nl < K_m): its column halves, and stacked, the A_lo row
    auto row16 = [&](int c0, uint32_t (&r)[16]) {
        ld_pair16(c0, r);
        if (p.stack) {
            const float* q = xb + nl * bstride + c0;
#pragma unroll
            for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + q[j]);
        }
    };
    if (p.ksplit > 1) {
        // tcgen05.ld is warp-wide: the condition is uniform per warp, the
        // stores are per row
        if (z == 1 && okflag && warp * 32 < Km) {
            // the partial D rows go to the same place in rank 0's shared memory
            const uint32_t dst = cluster_map(buf + (uint32_t)(nl * bstride) * 4u, 0);
            for (int c0 = 0; c0 < NT; c0 += 16) {
                uint32_t r[16];
                row16(c0, r);
                if (nl < Km) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                                         dst + (uint32_t)(c0 + j) * 4u),
                                     "r"(r[j]), "r"(r[j + 1]), "r"(r[j + 2]), "r"(r[j + 3])
                                     : "memory");
                }
            }
        } else if (z == 0 && okflag && p.stack && warp * 32 < Km) {
            // meanwhile rank 0 puts its own rows, complete, in place of its A_lo rows
            for (int c0 = 0; c0 < NT; c0 += 16) {
                uint32_t r[16];
                row16(c0, r);
                if (nl < Km) {
                    float* q = xb + nl * bstride + c0;
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(q + j) = make_float4(
                            __uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                            __uint_as_float(r[j + 3]));
                }
            }
        }
        __syncwarp();
        cluster_sync_all();                           // rank 1's rows are in rank 0's buffer
    }
    const bool own_in_xb = p.ksplit > 1 && p.stack;   // rank 0's rows are in xb already
    if (p.stack && p.discard_f && okflag && (z == 1 || warp >= 2))
        discard_f(z == 1 ? tid : tid - 64, z == 1 ? TC_THREADS : TC_THREADS - 64);
    if (okflag && z == 0 && warp * 32 < Km) {
        const bool live = nl < Km;
        const int idx = live ? moment_index(m + 2 * nl, m) : 0;
        const float f = p.inv_scale * ((p.neumann && m == 0) ? 0.5f : 1.f);
        const float* bufp = reinterpret_cast<const float*>(sm + p.buf_off) + nl * bstride;
        const bool v2 = ((uintptr_t)p.out & 7u) == 0;   // (re, im) pairs as one 8-byte store
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            if (own_in_xb) {
#pragma unroll
                for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(xb[nl * bstride + c0 + j]);
            } else {
                row16(c0, r);
            }
            if (live) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
                if (p.ksplit > 1) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        const float4 q = *reinterpret_cast<const float4*>(bufp + c0 + j);
                        v[j] += q.x;
                        v[j + 1] += q.y;
                        v[j + 2] += q.z;
                        v[j + 3] += q.w;
                    }
                }
                if (v2) {
                    // columns come in (re, im) pairs of one image: col even, cols_t even
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const int col = t * 256 + c0 + j;
                        if (c0 + j < cols_t)
                            *reinterpret_cast<float2*>(p.out + ((size_t)(col >> 1) * p.P + idx) * 2) =
                                make_float2(v[j] * f, v[j + 1] * f);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = t * 256 + c0 + j;
                        if (c0 + j < cols_t) p.out[((size_t)(col >> 1) * p.P + idx) * 2 + (col & 1)] = v[j] * f;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

// A halves -> operand blocks: row r < ceil(K_m/8)*8 of order m, chunk c;
// rows past K_m and nodes past n_rho are zero.
__global__ void k_build_ablk(const uint16_t* __restrict__ Ahi, const uint16_t* __restrict__ Alo,
                             const int* __restrict__ mrow, const long long* __restrict__ ablk_off, long long half,
                             int n_max, int n_rho, uint8_t* __restrict__ Ablk) {
    const int m = blockIdx.x, c = blockIdx.y;
    const int Km = (n_max - m) / 2 + 1, rg = (Km + 7) / 8;
    for (int task = threadIdx.x; task < rg * 8 * 8; task += blockDim.x) {
        const int row = task >> 3, kg = task & 7;
        uint16_t h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int i = c * TC_KC + kg * 8 + e;
            const bool on = row < Km && i < n_rho;
            const size_t src = (size_t)(mrow[m] + row) * n_rho + i;
            h[e] = on ? Ahi[src] : (uint16_t)0;
            l[e] = on ? Alo[src] : (uint16_t)0;
        }
        const size_t o = ablk_off[m] + (size_t)c * rg * 1024 + (size_t)(row >> 3) * 1024 + kg * 128 + (row & 7) * 16;
        uint4 vh, vl;
        vh.x = h[0] | ((uint32_t)h[1] << 16); vh.y = h[2] | ((uint32_t)h[3] << 16);
        vh.z = h[4] | ((uint32_t)h[5] << 16); vh.w = h[6] | ((uint32_t)h[7] << 16);
        vl.x = l[0] | ((uint32_t)l[1] << 16); vl.y = l[2] | ((uint32_t)l[3] << 16);
        vl.z = l[4] | ((uint32_t)l[5] << 16); vl.w = l[6] | ((uint32_t)l[7] << 16);
        *reinterpret_cast<uint4*>(Ablk + o) = vh;
        *reinterpret_cast<uint4*>(Ablk + half + o) = vl;
    }
}

int build_tc_blocks(zm_plan_t p) {
    p->n_chunks = (p->n_rho + TC_KC - 1) / TC_KC;
    if (p->prec != PREC_BF16X3 || p->n_max / 2 + 1 > TC_M) return ZM_OK;   // blocked form not used
    p->ablk_off_h.assign(p->n_max + 2, 0);
    for (int m = 0; m <= p->n_max; ++m) {
        const int rg = ((p->n_max - m) / 2 + 1 + 7) / 8;
        p->ablk_off_h[m + 1] = p->ablk_off_h[m] + (long long)p->n_chunks * rg * 1024;
    }
    p->ablk_half = p->ablk_off_h[p->n_max + 1];
    ZM_CUDA_TRY(cudaMalloc(&p->Ablk, 2 * (size_t)p->ablk_half));
    ZM_CUDA_TRY(cudaMalloc(&p->ablk_off, sizeof(long long) * (p->n_max + 2)));
    ZM_CUDA_TRY(cudaMemcpy(p->ablk_off, p->ablk_off_h.data(), sizeof(long long) * (p->n_max + 2),
                           cudaMemcpyHostToDevice));
    k_build_ablk<<<dim3(p->n_max + 1, p->n_chunks), 256>>>(p->Ahi, p->Alo, p->mrow, p->ablk_off, p->ablk_half,
                                                           p->n_max, p->n_rho, p->Ablk);
    ZM_LAUNCH_CHECK("k_build_ablk");
    ZM_CUDA_TRY(cudaDeviceSynchronize());
    return ZM_OK;
}

bool blocked_projection(zm_plan_t p) { return p->Ablk != nullptr; }

int launch_projection_blocked(zm_plan_t p, const uint8_t* Fblk, int batch, float* out, unsigned flags,
                              cudaStream_t st, bool consume) {
    const int ncol = 2 * batch;
    const int tiles = (ncol + 255) / 256;
    const int nt_max = ((std::min(ncol, 256) + 15) / 16) * 16;
    BlkParams bp;
    bp.Ablk = p->Ablk;
    bp.ablk_off = p->ablk_off;
    bp.ablk_half = p->ablk_half;
    bp.Fblk = Fblk;
    bp.fblk_half = (long long)fblk_half_bytes(p->n_max, p->n_chunks, ncol);
    bp.out = out;
    bp.status = p->status;
    bp.n_max = p->n_max;
    bp.n_chunks = p->n_chunks;
    bp.ncol = ncol;
    bp.P = p->P;
    // chunks per stage: the most (measured: fewer, larger copies pay; one
    // chunk in each of four stages was slower than two in each of two) that
    // still leave room for two stages within `cap` bytes after `tail`
    const int rg_max = (p->n_max / 2 + 1 + 7) / 8;
    // A hi and lo stacked on the MMA's M (rows 0..63 and 64..127) when every
    // order has at most 64 rows and [F hi | F lo] fits one MMA's N
    const bool stack = rg_max <= 8 && 2 * nt_max <= 256;
    auto stage_bytes = [&](int c) { return c * ((stack ? 8 + rg_max : 2 * rg_max) + 2 * (nt_max / 8)) * 1024; };
    auto fit = [&](int cap, int tail, int* cpc, int* stages) {
        const int budget = cap - tail;
        int c = BLK_CPC_MAX;
        while (c > 1 && 2 * stage_bytes(c) > budget) c >>= 1;
        *cpc = c;
        *stages = std::min(8, budget / stage_bytes(c));
        return *stages >= 2;
    };
    // split the radial range over a cluster of two CTAs when every order's
    // pair fits on the SMs in one wave at two CTAs per SM; rank 0's receive
    // buffer (rows of nt_max + 4 floats) doubles as the pad after the stages
    const int rows = ((p->n_max / 2 + 1 + 31) / 32) * 32;
    const int buf_bytes = rows * (nt_max + 4) * 4;
    const int tail2 = std::max(BLK_A_BYTES, buf_bytes);
    const int cap2 = 114 * 1024;                                 // half an SM's shared memory, less reserves
    int cpc = 0, stages = 0;
    bool split = p->n_chunks >= 2 && 2 * (p->n_max + 1) * tiles <= 2 * num_sms(p->device) &&
                 fit(cap2, tail2, &cpc, &stages);
    if (!split && !fit(225 * 1024, BLK_A_BYTES, &cpc, &stages))
        return set_error(ZM_EUNSUPPORTED, "blocked projection: stages of %d B do not fit", stage_bytes(1));
    bp.cpc = cpc;
    bp.stages = stages;
    bp.ksplit = split ? 2 : 1;
    bp.buf_off = stages * stage_bytes(cpc);
    bp.neumann = (flags & ZM_NEUMANN) ? 1 : 0;
    bp.inv_scale = 1.0f / p->a_scale;
    bp.discard_f = consume && ((uintptr_t)Fblk & 127u) == 0 && bp.fblk_half % 128 == 0 ? 1 : 0;
    // the epilogue's rows (64 x (nt_max + 4) floats: the A_lo rows, then rank
    // 0's own rows) go through the stages of the smallest order (rg = 1),
    // which always hold them
    bp.stack = stack && (size_t)bp.stages * bp.cpc * (9 + 2 * (nt_max / 8)) * 1024 >= (size_t)64 * (nt_max + 4) * 4
                   ? 1 : 0;
    const size_t smem = (size_t)bp.buf_off + (split ? tail2 : BLK_A_BYTES);
    static size_t configured[64] = {0};
    const int dev = p->device;
    if (dev >= 64 || smem > configured[dev]) {
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_project_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev < 64) configured[dev] = smem;
    }
    if (split) {
        cudaError_t e = launch_pdl_cluster(k_project_blk, dim3(p->n_max + 1, tiles, 2), dim3(TC_THREADS),
                                           dim3(1, 1, 2), smem, st, bp);
        if (e == cudaSuccess) {
            count_launch();
            return ZM_OK;
        }
        // a device or partition that cannot place the pairs: the same stages,
        // one CTA per order over the whole radial range
        cudaGetLastError();
        bp.ksplit = 1;
    }
    ZM_LAUNCH_PDL("k_project_blk", k_project_blk, dim3(p->n_max + 1, tiles), dim3(TC_THREADS), smem, st, bp);
    return ZM_OK;
}

}  // namespace zm
