// Zernike moments by Cartesian summation (Eq. 3-6): the moment integral as a
// sum over the pixels whose centres lie in the unit disk, each weighted by
// its area Delta^2 = 1/r^2 (disk radius r in pixels; Eq. 5's first-order
// approximation, with the prefactor of Eq. 3-5: Eq. 6 prints 1/(pi N^2) where
// Delta = 2/N of Eq. 5 gives 4/N^2 for an N x N image):
//
//   Z_nm = (n + 1) / (pi r^2) sum_{x^2 + y^2 <= 1} f(x, y) R_nm(rho) e^{-j m theta}.
//
// 8-point symmetry (the paper's Fig. 5 timings use it): when the disk centre
// sits at the same offset (0 or 1/2) from the pixel grid in x and y, the
// pixel centres come in orbits of (+-u, +-v), (+-v, +-u) that share rho.  One
// thread takes one representative u >= v >= 0, reads the eight pixels, folds
// them with the factors (-1)^m, (+-j)^m their angles give relative to
// theta_0 = atan2(v, u), and evaluates R_nm(rho) and e^{-j m theta_0} once.
// Other geometries take one thread per pixel.
//
// R_nm(rho) e^{-j m theta} = P_s^{(0,m)}(2 rho^2 - 1) (x - j y)^m, s = (n - m)/2:
// the Jacobi three-term recurrence for P (coefficients per block in shared
// memory; the per-pixel radii are not on any grid, so the Eq. 7 table of the
// polar path does not apply, and the recurrence is stable on [0, 1]) and the
// complex power by repeated squaring (m is the same in every thread).
//
// Sums: FP32 per thread and per block (shuffle tree), FP64 over the blocks in
// a fixed order (deterministic).
#include <algorithm>
#include <cmath>

#include "zm_internal.cuh"

namespace zm {

constexpr int CS_MAXP = 4;              // (n, m) pairs per pass
constexpr int CS_MAXS = 512;            // recurrence steps: (n - m) / 2 < 512
constexpr int CS_MAXI = 8;              // images per pass
constexpr int CS_TX = 32, CS_TY = 8;    // tile of representatives (or pixels) per block
constexpr int CS_THREADS = CS_TX * CS_TY;

struct CsImage {
    const float* data;
    long long pitch;
    int h, w;
    float cx, cy, r;
    int fold;               // 8-point symmetry: cx, cy on the same offset (0 or 1/2) from the grid
    int amax;               // fold: largest representative index a (a + half <= r)
    int inside;             // fold: every pixel of the orbits lies in the image (no bounds checks)
    int half;               // fold: 1 if that offset is 1/2
    int ox, oy;             // fold: column of offset +u is ox + a, row of offset +v is oy - c
    int tx, tiles;          // tiles per row, tiles in all
};

struct CsParams {
    int np;
    int n[CS_MAXP], m[CS_MAXP];
    CsImage im[CS_MAXI];
    double* part;           // [image][gridDim.x][np][2]
};

template <bool CHECK>
__device__ __forceinline__ float pix(const CsImage& g, int col, int row) {
    if (!CHECK) return __ldg(g.data + (long long)row * g.pitch + col);
    return ((unsigned)col < (unsigned)g.w && (unsigned)row < (unsigned)g.h)
               ? __ldg(g.data + (long long)row * g.pitch + col)
               : 0.f;
}

// (x - j y)^m by repeated squaring
__device__ __forceinline__ float2 cpow_conj(float x, float y, int m) {
    float wr = 1.f, wi = 0.f, br = x, bi = -y;
    for (int e = m; e; e >>= 1) {
        if (e & 1) {
            const float t = wr * br - wi * bi;
            wi = wr * bi + wi * br;
            wr = t;
        }
        if (e > 1) {
            const float t = br * br - bi * bi;
            bi = 2.f * br * bi;
            br = t;
        }
    }
    return make_float2(wr, wi);
}

// (A_s, B_s, C_s) of P_{s+1} = (A_s x + B_s) P_s - C_s P_{s-1}, the Jacobi
// polynomials P^{(0, beta)} with beta = m (P_0 = 1, P_{-1} = 0)
__device__ __forceinline__ float3 jacobi_coef(int s, int m) {
    const float b = (float)m, sf = (float)s;
    if (s == 0) return make_float3(0.5f * (b + 2.f), -0.5f * b, 0.f);
    const float a = 2.f * sf + b;
    const float d = 2.f * (sf + 1.f) * (sf + b + 1.f);
    return make_float3((a + 1.f) * (a + 2.f) / d, -(a + 1.f) * b * b / (d * a),
                       2.f * sf * (sf + b) * (a + 2.f) / (d * a));
}

// blockIdx.y = image; the block walks that image's tiles with stride gridDim.x.
// NP = pairs carried per thread (p.np <= NP): fewer accumulators, fewer
// registers, more resident blocks for single moments.
template <int NP>
__global__ void __launch_bounds__(CS_THREADS, (NP <= 2 ? 6 : 4)) k_cartesian(const __grid_constant__ CsParams p) {
    __shared__ float3 coef[NP][CS_MAXS];
    __shared__ float red[CS_THREADS / 32][NP][2];
    __shared__ float tq[4][CS_TX][CS_TY + 1];      // transposed orbit points of a tile, [point][a][c]
    const int tid = threadIdx.y * CS_TX + threadIdx.x;
    for (int k = 0; k < p.np; ++k) {
        const int S = (p.n[k] - p.m[k]) / 2;
        for (int s = tid; s < S; s += CS_THREADS) coef[k][s] = jacobi_coef(s, p.m[k]);
    }
    __syncthreads();
    const CsImage& g = p.im[blockIdx.y];
    float acc[NP][2];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k][0] = acc[k][1] = 0.f;
    const float inv_r = 1.f / g.r;

    for (int t = blockIdx.x; t < g.tiles; t += gridDim.x) {
        const int tyi = t / g.tx, txi = t - tyi * g.tx;
        const int a0 = txi * CS_TX, c0 = tyi * CS_TY;
        const int a = a0 + threadIdx.x, c = c0 + threadIdx.y;
        float f8[8];
        float x, y, wgt;
        if (g.fold) {
            // tiles wholly below the diagonal or outside the disk (block-uniform)
            const float h = g.half ? 0.5f : 0.f;
            if (a0 + CS_TX - 1 < c0 || a0 > g.amax) continue;
            if (((float)a0 + h) * ((float)a0 + h) + ((float)c0 + h) * ((float)c0 + h) > g.r * g.r) continue;
            // the points (+-v, +-u) of the tile lie in 32 rows (one per a) x 8
            // columns (one per c): stage them through shared memory, eight
            // lanes per row, so that the loads read whole 32-byte segments
            // this thread's representative (u, v) = (a + h, c + h), u >= v >= 0
            x = (float)a + h;
            y = (float)c + h;
            const bool live = a >= c && a <= g.amax && x * x + y * y <= g.r * g.r;
            // its points (+-u, +-v): columns of +-u, rows of +-v (offset -w lies
            // at column ox - w - half, row oy + w + half); issued with the
            // tile's staging loads below, so that one memory latency covers both
            const int cpu = g.ox + a, cmu = g.ox - a - g.half;
            const int rpv = g.oy - c, rmv = g.oy + c + g.half;
            if (live && g.inside) {
                f8[0] = pix<false>(g, cpu, rpv);
                f8[1] = pix<false>(g, cmu, rpv);
                f8[2] = pix<false>(g, cmu, rmv);
                f8[3] = pix<false>(g, cpu, rmv);
            } else if (live) {
                f8[0] = pix<true>(g, cpu, rpv);      // ( u,  v)  angle theta_0
                f8[1] = pix<true>(g, cmu, rpv);      // (-u,  v)  pi - theta_0
                f8[2] = pix<true>(g, cmu, rmv);      // (-u, -v)  pi + theta_0
                f8[3] = pix<true>(g, cpu, rmv);      // ( u, -v)  -theta_0
            }
            // the points (+-v, +-u) of the tile lie in 32 rows (one per a) x 8
            // columns (one per c): stage them through shared memory, eight
            // lanes per row, so that the loads read whole 32-byte segments
            __syncthreads();                       // tq of the previous tile is read
            {
                const int rr = tid >> 3, cc = tid & 7;  // a = a0 + rr, c = c0 + cc
                const int ra = a0 + rr, cb = c0 + cc;
                const int cpv_ = g.ox + cb, cmv_ = g.ox - cb - g.half;
                const int rpu_ = g.oy - ra, rmu_ = g.oy + ra + g.half;
                tq[0][rr][cc] = pix<true>(g, cpv_, rpu_);   // ( v,  u)
                tq[1][rr][cc] = pix<true>(g, cmv_, rpu_);   // (-v,  u)
                tq[2][rr][cc] = pix<true>(g, cmv_, rmu_);   // (-v, -u)
                tq[3][rr][cc] = pix<true>(g, cpv_, rmu_);   // ( v, -u)
            }
            __syncthreads();
            if (!live) continue;
            f8[4] = tq[0][threadIdx.x][threadIdx.y];  // ( v,  u)  pi/2 - theta_0
            f8[5] = tq[1][threadIdx.x][threadIdx.y];  // (-v,  u)  pi/2 + theta_0
            f8[6] = tq[2][threadIdx.x][threadIdx.y];  // (-v, -u)  -pi/2 - theta_0
            f8[7] = tq[3][threadIdx.x][threadIdx.y];  // ( v, -u)  -pi/2 + theta_0
            // orbits with repeated points: each distinct pixel appears twice
            // (v = 0 or u = v) or eight times (the centre)
            wgt = (x == 0.f) ? 0.125f : ((y == 0.f || x == y) ? 0.5f : 1.f);
        } else {
            if (a >= g.w || c >= g.h) continue;
            x = (float)a - g.cx;
            y = g.cy - (float)c;
            if (x * x + y * y > g.r * g.r) continue;
            f8[0] = __ldg(g.data + (long long)c * g.pitch + a);
            wgt = 1.f;
        }
        const float xr = x * inv_r, yr = y * inv_r;
        const float rho2 = xr * xr + yr * yr;
        const float xx = 2.f * rho2 - 1.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if (k >= p.np) break;
            const int m = p.m[k], S = (p.n[k] - m) / 2;
            float P0 = 1.f, P1 = 0.f;
            for (int s = 0; s < S; ++s) {
                const float3 q = coef[k][s];
                const float P2 = fmaf(fmaf(q.x, xx, q.y), P0, -q.z * P1);
                P1 = P0;
                P0 = P2;
            }
            // rho^m e^{-j m theta_0} = (x - j y)^m: cs - j sn
            const float2 W = cpow_conj(xr, yr, m);
            const float cs = W.x, sn = -W.y;
            const float R = P0 * wgt;
            float re, im;
            if (g.fold) {
                // sum_8 f e^{-j m theta} = E A + conj(E) B with E = e^{-j m theta_0},
                //   A = f(u,v) + (-1)^m f(-u,-v) + (-j)^m f(-v,u) + j^m f(v,-u)
                //   B = f(u,-v) + (-1)^m f(-u,v) + (-j)^m f(v,u) + j^m f(-v,-u)
                float Ar, Ai, Br, Bi;
                switch (m & 3) {
                    case 0:
                        Ar = f8[0] + f8[2] + f8[5] + f8[7];
                        Br = f8[3] + f8[1] + f8[4] + f8[6];
                        Ai = Bi = 0.f;
                        break;
                    case 2:
                        Ar = f8[0] + f8[2] - f8[5] - f8[7];
                        Br = f8[3] + f8[1] - f8[4] - f8[6];
                        Ai = Bi = 0.f;
                        break;
                    case 1:
                        Ar = f8[0] - f8[2];
                        Ai = f8[7] - f8[5];
                        Br = f8[3] - f8[1];
                        Bi = f8[6] - f8[4];
                        break;
                    default:
                        Ar = f8[0] - f8[2];
                        Ai = f8[5] - f8[7];
                        Br = f8[3] - f8[1];
                        Bi = f8[4] - f8[6];
                        break;
                }
                re = cs * (Ar + Br) + sn * (Ai - Bi);
                im = cs * (Ai + Bi) + sn * (Br - Ar);
            } else {
                re = f8[0] * cs;
                im = -f8[0] * sn;
            }
            acc[k][0] = fmaf(R, re, acc[k][0]);
            acc[k][1] = fmaf(R, im, acc[k][1]);
        }
    }
    // block sums (shuffle tree, then the warps in order)
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        float v0 = acc[k][0], v1 = acc[k][1];
        for (int o = 16; o; o >>= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        }
        if (lane == 0) {
            red[warp][k][0] = v0;
            red[warp][k][1] = v1;
        }
    }
    __syncthreads();
    if (tid < 2 * p.np) {
        const int k = tid >> 1, c = tid & 1;
        float s = 0.f;
        for (int w = 0; w < CS_THREADS / 32; ++w) s += red[w][k][c];
        p.part[(((size_t)blockIdx.y * gridDim.x + blockIdx.x) * p.np + k) * 2 + c] = (double)s;
    }
}

struct CsFinal {
    int blocks, nimg, np;
    float scale[CS_MAXI][CS_MAXP];
    float* out;             // image b, pair k at out[b * stride + (k0 + k) * 2]
    int stride, k0;
};

// out = (n + 1) / (pi r^2) (/ eps_m with Neumann) x the FP64 sum of the block
// partials: one warp per output value, lanes over the blocks with stride 32,
// then the shuffle tree (fixed order)
__global__ void k_cartesian_final(const double* __restrict__ part, const __grid_constant__ CsFinal f) {
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= f.nimg * f.np * 2) return;
    const int c = e & 1, bk = e >> 1;
    const int b = bk / f.np, k = bk - b * f.np;
    double s = 0.0;
    for (int j = lane; j < f.blocks; j += 32) s += part[(((size_t)b * f.blocks + j) * f.np + k) * 2 + c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) f.out[(size_t)b * f.stride + (size_t)(f.k0 + k) * 2 + c] = (float)(s * (double)f.scale[b][k]);
}

// blocks of k_cartesian<NP> that are resident at once on the device (cached)
template <int NP>
static int cs_blocks_t(int dev) {
    static int cached[64] = {0};
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cartesian<NP>, CS_THREADS, 0) != cudaSuccess || per < 1)
        per = 1;
    const int n = per * num_sms(dev);
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}
static int cs_blocks(int dev, int np) {
    return np == 1 ? cs_blocks_t<1>(dev) : (np == 2 ? cs_blocks_t<2>(dev) : cs_blocks_t<CS_MAXP>(dev));
}
static int cs_blocks_max(int dev) {
    return std::max(cs_blocks(dev, 1), std::max(cs_blocks(dev, 2), cs_blocks(dev, CS_MAXP)));
}

}  // namespace zm

using namespace zm;

extern "C" int zm_cartesian_work_bytes(int batch, int count, unsigned long long* bytes) {
    if (!bytes || batch < 1 || count < 1) return set_error(ZM_EINVAL, "bad arguments");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    // the block partials of one pass: CS_MAXI images x blocks x CS_MAXP pairs
    *bytes = (unsigned long long)CS_MAXI * cs_blocks_max(dev) * CS_MAXP * 2 * sizeof(double);
    return ZM_OK;
}

extern "C" int zm_cartesian_moments(const zm_image_t* imgs, int batch, const int* nm, int count, float* out,
                                    void* work, unsigned long long work_bytes, unsigned flags, void* stream) {
    if (!nm || !out || !work || count < 1) return set_error(ZM_EINVAL, "NULL argument or count < 1");
    int s = check_images(imgs, batch);
    if (s != ZM_OK) return s;
    for (int k = 0; k < count; ++k) {
        const int n = nm[2 * k], m = nm[2 * k + 1];
        if (n < 0 || m < 0 || m > n || ((n - m) & 1) || (n - m) / 2 >= CS_MAXS)
            return set_error(ZM_EINVAL, "pair %d: (n, m) = (%d, %d) is not a stored moment of order < %d", k, n, m,
                             2 * CS_MAXS);
    }
    unsigned long long need = 0;
    s = zm_cartesian_work_bytes(batch, count, &need);
    if (s != ZM_OK) return s;
    if (work_bytes < need) return set_error(ZM_EINVAL, "work holds %llu bytes, %llu needed", work_bytes, need);
    if ((reinterpret_cast<uintptr_t>(work) & 7u) != 0) return set_error(ZM_EINVAL, "work must be 8-byte aligned");
    int dev = 0;
    ZM_CUDA_TRY(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)stream;
    double* part = (double*)work;
    for (int b0 = 0; b0 < batch; b0 += CS_MAXI) {
        const int nb = std::min(CS_MAXI, batch - b0);
        CsParams p;
        int max_tiles = 1;
        for (int j = 0; j < nb; ++j) {
            const GeoImage g = resolve(imgs[b0 + j]);
            CsImage& ci = p.im[j];
            ci.data = g.data;
            ci.pitch = g.pitch;
            ci.h = g.h;
            ci.w = g.w;
            ci.cx = g.cx;
            ci.cy = g.cy;
            ci.r = g.r;
            const float fx = g.cx - std::floor(g.cx), fy = g.cy - std::floor(g.cy);
            ci.fold = (fx == fy && (fx == 0.f || fx == 0.5f)) ? 1 : 0;
            ci.half = (fx == 0.5f) ? 1 : 0;
            // offset +u = a + half sits at column floor(cx) + half + a, offset
            // +v = c + half at row floor(cy) - c
            ci.ox = (int)std::floor(g.cx) + ci.half;
            ci.oy = (int)std::floor(g.cy);
            // orbit offsets a + half <= r: a <= amax (exact, in double)
            ci.amax = (int)std::floor((double)g.r - 0.5 * ci.half);
            const int am = ci.amax;
            ci.inside = (ci.fold && ci.ox - am - ci.half >= 0 && ci.ox + am < g.w && ci.oy - am >= 0 &&
                         ci.oy + am + ci.half < g.h) ? 1 : 0;
            int tx, ty;
            if (ci.fold) {
                const int reps = (int)std::ceil(g.r) + 1;
                tx = (reps + CS_TX - 1) / CS_TX;
                ty = (reps + CS_TY - 1) / CS_TY;
            } else {
                tx = (g.w + CS_TX - 1) / CS_TX;
                ty = (g.h + CS_TY - 1) / CS_TY;
            }
            ci.tx = tx;
            ci.tiles = tx * ty;
            max_tiles = std::max(max_tiles, ci.tiles);
        }
        for (int k0 = 0; k0 < count; k0 += CS_MAXP) {
            const int np = std::min(CS_MAXP, count - k0);
            const int NP = np == 1 ? 1 : (np == 2 ? 2 : CS_MAXP);
            // as many blocks as fit on the device at once, shared by the images
            const int grid = std::min(max_tiles, std::max(1, cs_blocks(dev, NP) / nb));
            p.np = np;
            CsFinal f;
            for (int k = 0; k < np; ++k) {
                p.n[k] = nm[2 * (k0 + k)];
                p.m[k] = nm[2 * (k0 + k) + 1];
                for (int j = 0; j < nb; ++j) {
                    const double eps = ((flags & ZM_NEUMANN) && p.m[k] == 0) ? 2.0 : 1.0;
                    const double r = p.im[j].r;
                    f.scale[j][k] = (float)((p.n[k] + 1) / (3.14159265358979323846 * r * r) / eps);
                }
            }
            p.part = part;
            if (NP == 1)
                k_cartesian<1><<<dim3(grid, nb), dim3(CS_TX, CS_TY), 0, st>>>(p);
            else if (NP == 2)
                k_cartesian<2><<<dim3(grid, nb), dim3(CS_TX, CS_TY), 0, st>>>(p);
            else
                k_cartesian<CS_MAXP><<<dim3(grid, nb), dim3(CS_TX, CS_TY), 0, st>>>(p);
            ZM_LAUNCH_CHECK("k_cartesian");
            f.blocks = grid;
            f.nimg = nb;
            f.np = np;
            f.out = out + (size_t)b0 * count * 2;
            f.stride = count * 2;
            f.k0 = k0;
            const int tot = nb * np * 2;                         // one warp each
            k_cartesian_final<<<(tot + 3) / 4, 128, 0, st>>>(part, f);
            ZM_LAUNCH_CHECK("k_cartesian_final");
        }
    }
    return ZM_OK;
}
