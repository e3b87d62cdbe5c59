// Radial part of the reconstruction (Eq. 9) on the tensor cores:
//   G(b, i, m, re/im) = c_m sum_{n = m, m+2, ..} R_nm(rho_i) Z_nm (layout g_index),
// per m the contraction (rings i) x (orders n) x (image columns), i.e. an MMA
// with the rings on M (128 per CTA), the columns 2b + re/im on N and the K_m
// orders on K.  R is split into bf16 hi + lo once per plan and kept as
// operand blocks in the canonical K-major core-matrix layout (8-row x 16-byte
// core matrices; a row group holds the chunk's k-groups, so SBO = k-groups x
// 128 B), one block per (m, 128-ring tile, 64-order chunk); the moments are
// split the same way into the B tile by the CTA itself.  The product is
// accumulated in FP32 in TMEM as R_hi Z_hi + R_hi Z_lo + R_lo Z_hi.
#include <algorithm>

#include "tc_common.cuh"
#include "zm_internal.cuh"

namespace zm {

constexpr int RT_ROWS = 128;      // rings per CTA (MMA M)
constexpr int RT_KC = 64;         // orders per chunk
constexpr int RT_THREADS = 128;
constexpr int RT_NMAX = 256;      // image columns per CTA (MMA N)

// k-groups (8 orders each, rounded to whole 16-order MMA steps) of chunk kc
__host__ __device__ inline int rt_kgroups(int Km, int kc) {
    const int k = (Km - kc * RT_KC < RT_KC) ? Km - kc * RT_KC : RT_KC;
    return 2 * ((k + 15) / 16);
}
__host__ __device__ inline int rt_chunks(int Km) { return (Km + RT_KC - 1) / RT_KC; }
// bytes of one half of the blocks of one 128-ring tile of order m
__host__ __device__ inline long long rt_tile_bytes(int Km) {
    long long t = 0;
    for (int kc = 0; kc < rt_chunks(Km); ++kc) t += 16LL * rt_kgroups(Km, kc) * 128;
    return t;
}

// R32m -> blocks: block (m, tile, kc) holds R[n = m + 2k][i], k = kc*64 + k',
// i = tile*128 + row; orders past K_m and rings past n_rho are zero.
__global__ void k_build_rblk(const float* __restrict__ R32m, const int* __restrict__ mrow,
                             const long long* __restrict__ rblk_off, long long half, int n_max, int n_rho,
                             uint8_t* __restrict__ Rblk) {
    const int m = blockIdx.x, tile = blockIdx.y;
    const int Km = (n_max - m) / 2 + 1;
    long long o = rblk_off[m] + (long long)tile * rt_tile_bytes(Km);
    for (int kc = 0; kc < rt_chunks(Km); ++kc) {
        const int nkg = rt_kgroups(Km, kc);
        for (int task = threadIdx.x; task < RT_ROWS * nkg; task += blockDim.x) {
            const int row = task / nkg, kg = task - row * nkg;
            const int i = tile * RT_ROWS + row;
            uint16_t h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = kc * RT_KC + kg * 8 + e;
                const float x = (k < Km && i < n_rho) ? R32m[(size_t)(mrow[m] + k) * n_rho + i] : 0.f;
                split2(x, 0, &h[e], &l[e]);
            }
            const long long d = o + (long long)(row >> 3) * nkg * 128 + kg * 128 + (row & 7) * 16;
            uint4 vh, vl;
            vh.x = h[0] | ((uint32_t)h[1] << 16); vh.y = h[2] | ((uint32_t)h[3] << 16);
            vh.z = h[4] | ((uint32_t)h[5] << 16); vh.w = h[6] | ((uint32_t)h[7] << 16);
            vl.x = l[0] | ((uint32_t)l[1] << 16); vl.y = l[2] | ((uint32_t)l[3] << 16);
            vl.z = l[4] | ((uint32_t)l[5] << 16); vl.w = l[6] | ((uint32_t)l[7] << 16);
            *reinterpret_cast<uint4*>(Rblk + d) = vh;
            *reinterpret_cast<uint4*>(Rblk + half + d) = vl;
        }
        o += 16LL * nkg * 128;
    }
}

struct RtParams {
    const uint8_t* Rblk;
    const long long* rblk_off;
    long long rblk_half;
    const float* Z;          // [batch][P][2]
    float* G;                // layout g_index
    int* status;
    int n_max, n_rho, P, ncol;
    int neumann;
};

// One CTA = (m, 128-ring tile, 256-column tile).  Shared memory, per chunk:
// [R hi][R lo] (16 row groups) then [Z hi][Z lo] (NT / 8 row groups).
__global__ void __launch_bounds__(RT_THREADS) k_recon_tc(const __grid_constant__ RtParams p) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar[2];      // 0: copies of R, 1: MMA commit
    __shared__ uint32_t tslot;
    __shared__ int okflag;
    const int m = blockIdx.x, tile = blockIdx.y, ct = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nm1 = p.n_max + 1;
    const int Km = (p.n_max - m) / 2 + 1;
    const int nkc = rt_chunks(Km);
    const int cols_t = min(RT_NMAX, p.ncol - ct * RT_NMAX);
    const int NT = ((cols_t + 15) / 16) * 16;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)NT) ncols <<= 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        okflag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tslot;
    const uint32_t sm0 = smem_u32(sm);

    // R blocks of this (m, tile): one bulk copy per chunk and half
    if (tid == 0) {
        const uint8_t* src = p.Rblk + p.rblk_off[m] + (long long)tile * rt_tile_bytes(Km);
        uint32_t total = 0;
        for (int kc = 0; kc < nkc; ++kc) total += 2u * 16u * rt_kgroups(Km, kc) * 128u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar[0])), "r"(total)
                     : "memory");
        uint32_t dst = sm0;
        for (int kc = 0; kc < nkc; ++kc) {
            const int nkg = rt_kgroups(Km, kc);
            const uint32_t a = 16u * nkg * 128u;
            const uint32_t b = (uint32_t)(NT / 8) * nkg * 128u;
            bulk_copy(dst, src, a, smem_u32(&bar[0]));
            bulk_copy(dst + a, src + p.rblk_half, a, smem_u32(&bar[0]));
            src += a;
            dst += 2 * a + 2 * b;
        }
    }
    griddep_wait();                    // the moments are written, G is free
    griddep_launch();
    // the moments of the column tile as Z hi / lo blocks (orders past K_m and
    // columns past the batch are zero)
    {
        uint32_t off = 0;
        for (int kc = 0; kc < nkc; ++kc) {
            const int nkg = rt_kgroups(Km, kc);
            const uint32_t a = 16u * nkg * 128u;
            const uint32_t b = (uint32_t)(NT / 8) * nkg * 128u;
            unsigned char* zh = sm + off + 2 * a;
            unsigned char* zl = zh + b;
            for (int task = tid; task < NT * nkg; task += RT_THREADS) {
                const int col = task / nkg, kg = task - col * nkg;
                const int gcol = ct * RT_NMAX + col;
                uint16_t h[8], l[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int k = kc * RT_KC + kg * 8 + e;
                    float x = 0.f;
                    if (k < Km && gcol < p.ncol)
                        x = __ldg(&p.Z[((size_t)(gcol >> 1) * p.P + moment_index(m + 2 * k, m)) * 2 + (gcol & 1)]);
                    split2(x, 0, &h[e], &l[e]);
                }
                const uint32_t d = (uint32_t)(col >> 3) * nkg * 128 + kg * 128 + (col & 7) * 16;
                uint4 vh, vl;
                vh.x = h[0] | ((uint32_t)h[1] << 16); vh.y = h[2] | ((uint32_t)h[3] << 16);
                vh.z = h[4] | ((uint32_t)h[5] << 16); vh.w = h[6] | ((uint32_t)h[7] << 16);
                vl.x = l[0] | ((uint32_t)l[1] << 16); vl.y = l[2] | ((uint32_t)l[3] << 16);
                vl.z = l[4] | ((uint32_t)l[5] << 16); vl.w = l[6] | ((uint32_t)l[7] << 16);
                *reinterpret_cast<uint4*>(zh + d) = vh;
                *reinterpret_cast<uint4*>(zl + d) = vl;
            }
            off += 2 * a + 2 * b;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        const unsigned long long t0 = global_ns();
        bool ok = mbar_wait(smem_u32(&bar[0]), 0, t0);
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = instr_desc(NT, 0);
            uint32_t off = 0;
            bool first = true;
            for (int kc = 0; kc < nkc; ++kc) {
                const int nkg = rt_kgroups(Km, kc);
                const uint32_t a = 16u * nkg * 128u;
                const uint32_t b = (uint32_t)(NT / 8) * nkg * 128u;
                const uint32_t rh = sm0 + off, rl = rh + a, zh = rh + 2 * a, zl = zh + b;
                const uint32_t sbo = (uint32_t)nkg * 128u;
                for (int ks = 0; ks < nkg / 2; ++ks) {
                    const uint32_t o = ks * 256;
                    const uint64_t drh = smem_desc(rh + o, sbo), drl = smem_desc(rl + o, sbo);
                    const uint64_t dzh = smem_desc(zh + o, sbo), dzl = smem_desc(zl + o, sbo);
                    const uint32_t acc0 = first ? 0u : 1u;
                    first = false;
                    asm volatile(
                        "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                        "l"(drh), "l"(dzh), "r"(idesc), "r"(acc0));
                    asm volatile(
                        "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                        "l"(drh), "l"(dzl), "r"(idesc), "r"(1u));
                    asm volatile(
                        "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
                        "l"(drl), "l"(dzh), "r"(idesc), "r"(1u));
                }
                off += 2 * a + 2 * b;
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[1]))
                         : "memory");
            ok = mbar_wait(smem_u32(&bar[1]), 0, t0);
            if (!ok) mbar_wait(smem_u32(&bar[1]), 0, global_ns());    // let the MMAs drain (bounded)
        } else {
            mbar_wait(smem_u32(&bar[0]), 0, global_ns());             // let the copies land (bounded)
        }
        if (!ok) {
            atomicExch(p.status, ZM_ETIMEOUT);
            okflag = 0;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: TMEM lane = ring (warp w owns lanes 32w..32w+31)
    if (okflag) {
        const int i = tile * RT_ROWS + warp * 32 + lane;
        const float cm = (p.neumann && m > 0) ? 2.f : 1.f;
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
            if (i < p.n_rho) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int gcol = ct * RT_NMAX + c0 + j;
                    if (c0 + j < cols_t)
                        p.G[g_index(gcol >> 1, i, m, gcol & 1, (p.n_rho + 7) / 8, nm1)] = cm * __uint_as_float(r[j]);
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

int build_recon_blocks(zm_plan_t p) {
    if (p->prec != PREC_BF16X3) return ZM_OK;
    p->n_rtiles = (p->n_rho + RT_ROWS - 1) / RT_ROWS;
    p->rblk_off_h.assign(p->n_max + 2, 0);
    for (int m = 0; m <= p->n_max; ++m)
        p->rblk_off_h[m + 1] = p->rblk_off_h[m] + p->n_rtiles * rt_tile_bytes((p->n_max - m) / 2 + 1);
    p->rblk_half = p->rblk_off_h[p->n_max + 1];
    ZM_CUDA_TRY(cudaMalloc(&p->Rblk, 2 * (size_t)p->rblk_half));
    ZM_CUDA_TRY(cudaMalloc(&p->rblk_off, sizeof(long long) * (p->n_max + 2)));
    ZM_CUDA_TRY(cudaMemcpy(p->rblk_off, p->rblk_off_h.data(), sizeof(long long) * (p->n_max + 2),
                           cudaMemcpyHostToDevice));
    k_build_rblk<<<dim3(p->n_max + 1, p->n_rtiles), 256>>>(p->R32m, p->mrow, p->rblk_off, p->rblk_half, p->n_max,
                                                            p->n_rho, p->Rblk);
    ZM_LAUNCH_CHECK("k_build_rblk");
    ZM_CUDA_TRY(cudaDeviceSynchronize());
    return ZM_OK;
}

int launch_radial_tc(zm_plan_t p, const float* moments, int batch, unsigned flags, float* G, cudaStream_t st) {
    const int ncol = 2 * batch;
    const int ctiles = (ncol + RT_NMAX - 1) / RT_NMAX;
    const int NT = ((std::min(ncol, RT_NMAX) + 15) / 16) * 16;
    int ncols = 32;
    while (ncols < NT) ncols <<= 1;
    // shared memory of the widest order (m = 0)
    const int Km0 = p->n_max / 2 + 1;
    size_t need = 0;
    for (int kc = 0; kc < rt_chunks(Km0); ++kc) {
        const int nkg = rt_kgroups(Km0, kc);
        need += 2 * (size_t)16 * nkg * 128 + 2 * (size_t)(NT / 8) * nkg * 128;
    }
    // resident CTAs must not ask for more than the SM's 512 TMEM columns
    const size_t cap = 227 * 1024;
    const size_t by_tmem = cap / (512 / ncols) + 1024;
    const size_t smem = std::max(need, std::min(cap, by_tmem));
    if (need > cap) return set_error(ZM_EUNSUPPORTED, "reconstruction blocks need %zu B of shared memory", need);
    static size_t configured[64] = {0};
    const int dev = p->device;
    if (dev >= 64 || smem > configured[dev]) {
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_recon_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev < 64) configured[dev] = smem;
    }
    RtParams rp;
    rp.Rblk = p->Rblk;
    rp.rblk_off = p->rblk_off;
    rp.rblk_half = p->rblk_half;
    rp.Z = moments;
    rp.G = G;
    rp.status = p->status;
    rp.n_max = p->n_max;
    rp.n_rho = p->n_rho;
    rp.P = p->P;
    rp.ncol = ncol;
    rp.neumann = (flags & ZM_NEUMANN) ? 1 : 0;
    ZM_LAUNCH_PDL("k_recon_tc", k_recon_tc, dim3(p->n_max + 1, p->n_rtiles, ctiles), dim3(RT_THREADS), smem, st, rp);
    return ZM_OK;
}

}  // namespace zm
