// Plans: the FP64 Zernike radial polynomial table by the Chebyshev-U / DFT
// identity of Sec. 2.1 (Eq. 7-8), the radial grid, and the operands derived
// from them.  Also the library's error state and index helpers.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdlib>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "zm_internal.cuh"

namespace zm {

// ============================================================== error state
static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

int set_error(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int cuda_error(cudaError_t e, const char* what) {
    const int st = (e == cudaErrorMemoryAllocation) ? ZM_ENOMEM : ZM_ECUDA;
    return set_error(st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int check_images(const zm_image_t* imgs, int batch) {
    if (batch < 1) return set_error(ZM_EINVAL, "batch must be >= 1 (got %d)", batch);
    if (!imgs) return set_error(ZM_EINVAL, "image descriptor array is NULL");
    for (int b = 0; b < batch; ++b) {
        const zm_image_t& im = imgs[b];
        if (!im.data) return set_error(ZM_EINVAL, "image %d: data is NULL", b);
        if (im.height < 1 || im.width < 1)
            return set_error(ZM_EINVAL, "image %d: size %dx%d", b, im.height, im.width);
        if (im.pitch < im.width)
            return set_error(ZM_EINVAL, "image %d: pitch %lld < width %d", b, im.pitch, im.width);
        if (im.radius > 0.f && !(std::isfinite(im.cx) && std::isfinite(im.cy) && std::isfinite(im.radius)))
            return set_error(ZM_EINVAL, "image %d: non-finite geometry", b);
    }
    return ZM_OK;
}

Workspace::~Workspace() {
    if (ptr) cudaFree(ptr);
}

int Workspace::grow(size_t need) {
    if (need <= bytes) return ZM_OK;
    if (ptr) {
        cudaError_t e = cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        if (e != cudaSuccess) return cuda_error(e, "cudaFree(workspace)");
    }
    cudaError_t e = cudaMalloc(&ptr, need);
    if (e != cudaSuccess) {
        ptr = nullptr;
        return cuda_error(e, "cudaMalloc(workspace)");
    }
    bytes = need;
    return ZM_OK;
}

// ============================================================== radial grid
// Midpoint rule: rho_i = (i + 1/2) / N, wr_i = rho_i / N (the Jacobian rho of
// Eq. 1 folded into the weight).
__global__ void k_grid_midpoint(int n, double* rho, double* wr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = (i + 0.5) / n;
    rho[i] = r;
    wr[i] = r / n;
}

// Gauss-Legendre rule on [0, 1]: node x_j of P_N on [-1, 1] by Newton's method
// from the asymptotic guess cos(pi (j + 3/4) / (N + 1/2)), weight
// 2 / ((1 - x^2) P_N'(x)^2); mapped to rho = (1 + x)/2, wr = w/2 * rho, in
// ascending rho.  The Newton loop is bounded.
__global__ void k_grid_gauss(int n, double* rho, double* wr) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double x = cospi((j + 0.75) / (n + 0.5));
    double dp = 1.0;
    int extra = 2;                              // polishing steps after convergence
    for (int it = 0; it < 100 && extra > 0; ++it) {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        const double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-13) --extra;
    }
    {   // derivative at the final node
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
    }
    const double w = 2.0 / ((1.0 - x * x) * dp * dp);
    const int i = n - 1 - j;
    const double r = 0.5 * (1.0 + x);
    rho[i] = r;
    wr[i] = 0.5 * w * r;
}

// ============================================================== Eq. 7 table
// One CTA per radial node rho_i.  With N = n_z (a multiple of 4) and
// x_k = rho cos(2 pi k / N), Eq. 7 reads
//   R_nm(rho) = (1/N) sum_{k=0}^{N-1} U_n(x_k) cos(2 pi m k / N).
// The summand is even in k -> N - k, and for n - m even also symmetric under
// k -> N/2 - k (x changes sign, U_n gets (-1)^n, the cosine (-1)^m), so
//   R_nm = (2/N) sum_{k=0}^{N/4} c_k U_n(x_k) cos(2 pi m k / N),
// c_0 = c_{N/4} = 1, c_k = 2 otherwise.  U_n comes from the three-term
// recurrence U_{n+1} = 2x U_n - U_{n-1} (exact at x = +-1 where the sine ratio
// of Eq. 8 is 0/0).  FP64 throughout; n_z > n + m removes every alias.
constexpr int KA_THREADS = 256;
constexpr int KA_NB = 8;        // orders per shared-memory block
constexpr int KA_KPT = 4;       // k values per thread (N/4 + 1 <= 1024)

__global__ void __launch_bounds__(KA_THREADS)
k_zrp_eq7(const double* __restrict__ rho, int n_rho, int n_max, int n_z, double* __restrict__ R) {
    extern __shared__ double sm[];
    const int Qk = n_z >> 2;                  // k = 0..Qk
    double* cosz = sm;                        // [n_z]
    double* U = sm + n_z;                     // [KA_NB][Qk + 1]
    const int i = blockIdx.x;
    const int tid = threadIdx.x;
    for (int j = tid; j < n_z; j += KA_THREADS) cosz[j] = cospi(2.0 * j / n_z);
    __syncthreads();

    const double r = rho[i];
    double x[KA_KPT], ua[KA_KPT], ub[KA_KPT];   // U_{n-1}, U_n
#pragma unroll
    for (int c = 0; c < KA_KPT; ++c) {
        const int k = tid + c * KA_THREADS;
        x[c] = (k <= Qk) ? r * cosz[k] : 0.0;
        ua[c] = 0.0;                           // U_{-1}
        ub[c] = 1.0;                           // U_0
    }
    const double scale = 2.0 / n_z;
    for (int n0 = 0; n0 <= n_max; n0 += KA_NB) {
        const int nb = min(KA_NB, n_max + 1 - n0);
        for (int t = 0; t < nb; ++t) {
            const int n = n0 + t;
#pragma unroll
            for (int c = 0; c < KA_KPT; ++c) {
                const int k = tid + c * KA_THREADS;
                if (n > 0) {
                    const double un = 2.0 * x[c] * ub[c] - ua[c];
                    ua[c] = ub[c];
                    ub[c] = un;
                }
                if (k <= Qk) U[t * (Qk + 1) + k] = ((k == 0 || k == Qk) ? 1.0 : 2.0) * ub[c];
            }
        }
        __syncthreads();
        int total = 0;
        for (int t = 0; t < nb; ++t) total += (n0 + t) / 2 + 1;
        for (int p = tid; p < total; p += KA_THREADS) {
            int t = 0, pp = p;
            while (pp >= (n0 + t) / 2 + 1) { pp -= (n0 + t) / 2 + 1; ++t; }
            const int n = n0 + t;
            const int m = (n & 1) + 2 * pp;
            const double* u = U + t * (Qk + 1);
            double acc = 0.0;
            int idx = 0;
            for (int k = 0; k <= Qk; ++k) {
                acc = fma(u[k], cosz[idx], acc);
                idx = (idx + m) & (n_z - 1);
            }
            R[(size_t)moment_index(n, m) * n_rho + i] = acc * scale;
        }
        __syncthreads();
    }
}

// ============================================================== table cache
ZrpTable::~ZrpTable() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (device >= 0 && cur != device) cudaSetDevice(device);
    if (rho) cudaFree(rho);
    if (wr) cudaFree(wr);
    if (R) cudaFree(R);
    if (cur >= 0 && cur != device) cudaSetDevice(cur);
}

static std::mutex g_cache_mu;
static std::map<std::tuple<int, int, int>, std::shared_ptr<ZrpTable>> g_cache;

static int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

static int build_table(int device, int grid, int n_rho, int n_max, std::shared_ptr<ZrpTable>* out) {
    auto t = std::make_shared<ZrpTable>();
    t->device = device;
    t->grid = grid;
    t->n_rho = n_rho;
    t->n_max = n_max;
    t->n_z = std::max(8, next_pow2(2 * n_max + 2));
    const int P = num_moments(n_max);
    ZM_CUDA_TRY(cudaMalloc(&t->rho, sizeof(double) * n_rho));
    ZM_CUDA_TRY(cudaMalloc(&t->wr, sizeof(double) * n_rho));
    ZM_CUDA_TRY(cudaMalloc(&t->R, sizeof(double) * (size_t)P * n_rho));
    cudaEvent_t e0, e1;
    ZM_CUDA_TRY(cudaEventCreate(&e0));
    ZM_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, 0);
    const int gb = (n_rho + 127) / 128;
    if (grid == ZM_GRID_GAUSS) k_grid_gauss<<<gb, 128>>>(n_rho, t->rho, t->wr);
    else k_grid_midpoint<<<gb, 128>>>(n_rho, t->rho, t->wr);
    ZM_LAUNCH_CHECK("grid kernel");
    const int Qk = t->n_z >> 2;
    if (Qk + 1 > KA_THREADS * KA_KPT) return set_error(ZM_EUNSUPPORTED, "n_max %d too large for the table kernel", n_max);
    const size_t smem = sizeof(double) * (t->n_z + (size_t)KA_NB * (Qk + 1));
    if (smem > 48 * 1024)
        ZM_CUDA_TRY(cudaFuncSetAttribute(k_zrp_eq7, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_zrp_eq7<<<n_rho, KA_THREADS, smem>>>(t->rho, n_rho, n_max, t->n_z, t->R);
    ZM_LAUNCH_CHECK("k_zrp_eq7");
    cudaEventRecord(e1, 0);
    ZM_CUDA_TRY(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&t->plan_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = t;
    return ZM_OK;
}

int acquire_table(int device, int grid, int n_rho, int n_max, std::shared_ptr<ZrpTable>* out) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto key = std::make_tuple(device, grid, n_rho);
    auto it = g_cache.find(key);
    if (it != g_cache.end() && it->second->n_max >= n_max) {
        *out = it->second;
        return ZM_OK;
    }
    std::shared_ptr<ZrpTable> t;
    const int st = build_table(device, grid, n_rho, n_max, &t);
    if (st != ZM_OK) return st;
    g_cache[key] = t;
    *out = t;
    return ZM_OK;
}

// ============================================================== derived operands
// For each stored (n, m) (blockIdx.x = moment index) and node i:
//   A[row][i]    = 2(n+1)/N_theta * wr_i * R_nm(rho_i)   ((n+1)/pi * wr * 2 pi/N_theta)
//   R32m[row][i] = R_nm(rho_i)
// with row = mrow[m] + (n - m)/2 (m-major), and the hi/lo split of A for the
// tensor-core projection: hi = round(A s), lo = round(A s - hi).
__global__ void k_derive(const double* __restrict__ R, const double* __restrict__ wr, int n_rho,
                         int n_theta, const int2* __restrict__ pair_nm, const int* __restrict__ mrow,
                         float* __restrict__ A32, float* __restrict__ R32m, uint16_t* __restrict__ Ahi,
                         uint16_t* __restrict__ Alo, int prec, double a_scale) {
    const int p = blockIdx.x;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= n_rho) return;
    const int2 nm = pair_nm[p];
    const int row = mrow[nm.y] + (nm.x - nm.y) / 2;
    const double r = R[(size_t)p * n_rho + i];
    const double a = 2.0 * (nm.x + 1) / n_theta * wr[i] * r;
    const size_t o = (size_t)row * n_rho + i;
    A32[o] = (float)a;
    R32m[o] = (float)r;
    if (prec == PREC_BF16X3) {
        const __nv_bfloat16 hi = __double2bfloat16(a);
        const __nv_bfloat16 lo = __double2bfloat16(a - (double)__bfloat162float(hi));
        Ahi[o] = __bfloat16_as_ushort(hi);
        Alo[o] = __bfloat16_as_ushort(lo);
    } else if (prec == PREC_FP16X3) {
        const double as = a * a_scale;
        const __half hi = __double2half(as);
        const __half lo = __double2half(as - (double)__half2float(hi));
        Ahi[o] = __half_as_ushort(hi);
        Alo[o] = __half_as_ushort(lo);
    }
}

// Angular tables: tw[j] = e^{-2 pi i j / N}, cs[k] = (cos theta_k, sin theta_k).
__global__ void k_angles(int n_theta, float2* tw, float2* cs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_theta) return;
    double s, c;
    sincospi(2.0 * j / n_theta, &s, &c);
    tw[j] = make_float2((float)c, (float)-s);
    cs[j] = make_float2((float)c, (float)s);
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_absmax(const double* __restrict__ R, const double* __restrict__ wr, int n_rho,
                         int n_theta, const int2* __restrict__ pair_nm, int P, unsigned long long* out) {
    // max |A| over the table (as ordered bits of a non-negative double)
    double m = 0.0;
    const size_t total = (size_t)P * n_rho;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(e / n_rho);
        const int i = (int)(e % n_rho);
        const double a = fabs(2.0 * (pair_nm[p].x + 1) / n_theta * wr[i] * R[e]);
        m = fmax(m, a);
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

int build_plan_tables(zm_plan_t p) {
    const int P = p->P, n_rho = p->n_rho;
    // m-major row starts
    p->mrow_h.assign(p->n_max + 2, 0);
    for (int m = 0; m <= p->n_max; ++m) p->mrow_h[m + 1] = p->mrow_h[m] + (p->n_max - m) / 2 + 1;
    std::vector<int2> pairs(P);
    for (int n = 0; n <= p->n_max; ++n)
        for (int m = n & 1; m <= n; m += 2) pairs[moment_index(n, m)] = make_int2(n, m);
    const size_t tab = (size_t)P * n_rho;
    ZM_CUDA_TRY(cudaMalloc(&p->rho32, sizeof(float) * n_rho));
    ZM_CUDA_TRY(cudaMalloc(&p->A32, sizeof(float) * tab));
    ZM_CUDA_TRY(cudaMalloc(&p->R32m, sizeof(float) * tab));
    if (p->prec != PREC_FP32) {
        ZM_CUDA_TRY(cudaMalloc(&p->Ahi, sizeof(uint16_t) * tab));
        ZM_CUDA_TRY(cudaMalloc(&p->Alo, sizeof(uint16_t) * tab));
    }
    ZM_CUDA_TRY(cudaMalloc(&p->tw, sizeof(float2) * p->n_theta));
    ZM_CUDA_TRY(cudaMalloc(&p->cs, sizeof(float2) * p->n_theta));
    ZM_CUDA_TRY(cudaMalloc(&p->mrow, sizeof(int) * (p->n_max + 2)));
    ZM_CUDA_TRY(cudaMalloc(&p->status, sizeof(int)));
    ZM_CUDA_TRY(cudaMemset(p->status, 0, sizeof(int)));
    ZM_CUDA_TRY(cudaMalloc(&p->work, 2 * sizeof(int)));
    ZM_CUDA_TRY(cudaMemset(p->work, 0, 2 * sizeof(int)));
    ZM_CUDA_TRY(cudaMalloc(&p->pair_nm, sizeof(int2) * P));
    ZM_CUDA_TRY(cudaMemcpy(p->mrow, p->mrow_h.data(), sizeof(int) * (p->n_max + 2), cudaMemcpyHostToDevice));
    ZM_CUDA_TRY(cudaMemcpy(p->pair_nm, pairs.data(), sizeof(int2) * P, cudaMemcpyHostToDevice));

    k_angles<<<(p->n_theta + 127) / 128, 128>>>(p->n_theta, p->tw, p->cs);
    ZM_LAUNCH_CHECK("k_angles");
    k_to_float<<<(n_rho + 255) / 256, 256>>>(p->table->rho, p->rho32, n_rho);
    ZM_LAUNCH_CHECK("k_to_float");
    double a_scale = 1.0;
    if (p->prec == PREC_FP16X3) {
        // power-of-two scale putting max |A| near 2^14, inside fp16's range,
        // so that the lo parts of the significant entries stay normal
        unsigned long long* d = nullptr;
        ZM_CUDA_TRY(cudaMalloc(&d, sizeof(unsigned long long)));
        ZM_CUDA_TRY(cudaMemset(d, 0, sizeof(unsigned long long)));
        k_absmax<<<256, 256>>>(p->table->R, p->table->wr, n_rho, p->n_theta, p->pair_nm, P, d);
        unsigned long long bits = 0;
        cudaError_t e = cudaMemcpy(&bits, d, sizeof bits, cudaMemcpyDeviceToHost);
        cudaFree(d);
        ZM_CUDA_TRY(e);
        double amax;
        memcpy(&amax, &bits, sizeof amax);
        if (amax > 0) a_scale = std::ldexp(1.0, 14 - (int)std::ceil(std::log2(amax)));
    }
    p->a_scale = (float)a_scale;
    dim3 g(P, (n_rho + 127) / 128);
    k_derive<<<g, 128>>>(p->table->R, p->table->wr, n_rho, p->n_theta, p->pair_nm, p->mrow, p->A32,
                         p->R32m, p->Ahi, p->Alo, p->prec, a_scale);
    ZM_LAUNCH_CHECK("k_derive");
    ZM_CUDA_TRY(cudaDeviceSynchronize());
    const int s = build_tc_blocks(p);
    return s != ZM_OK ? s : build_recon_blocks(p);
}

static void free_plan(zm_plan_t p) {
    if (!p) return;
    release_tiles(p);
    release_fused(p);
    release_dft(p);
    cudaFree(p->dft);
    cudaFree(p->dft32);
    cudaFree(p->rho32);
    cudaFree(p->A32);
    cudaFree(p->R32m);
    cudaFree(p->Ahi);
    cudaFree(p->Alo);
    cudaFree(p->Ablk);
    cudaFree(p->ablk_off);
    cudaFree(p->Rblk);
    cudaFree(p->rblk_off);
    cudaFree(p->tw);
    cudaFree(p->cs);
    cudaFree(p->mrow);
    cudaFree(p->pair_nm);
    cudaFree(p->status);
    cudaFree(p->work);
    delete p;
}

}  // namespace zm

using namespace zm;

// ============================================================== C ABI
extern "C" int zm_num_moments(int n_max) { return num_moments(n_max); }

extern "C" int zm_index(int n, int m) {
    if (n < 0 || m < 0 || m > n || ((n - m) & 1)) return -1;
    return moment_index(n, m);
}

extern "C" const char* zm_strerror(int status) {
    switch (status) {
        case ZM_OK: return "ok";
        case ZM_EINVAL: return "invalid argument";
        case ZM_ENOMEM: return "out of device memory";
        case ZM_ECUDA: return "CUDA error";
        case ZM_ETIMEOUT: return "timed out";
        case ZM_EUNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

extern "C" const char* zm_last_error(void) { return g_last_error.c_str(); }

extern "C" unsigned long long zm_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" int zm_plan(zm_plan_t* plan, int n_max, int n_rho, int n_theta, unsigned flags) {
    g_last_error.clear();
    if (!plan) return set_error(ZM_EINVAL, "plan pointer is NULL");
    *plan = nullptr;
    if (n_max < 0) return set_error(ZM_EINVAL, "n_max must be >= 0 (got %d)", n_max);
    if (n_rho < 1 || n_rho > 65536) return set_error(ZM_EINVAL, "n_rho must be in [1, 65536] (got %d)", n_rho);
    if (n_theta < 8 || (n_theta & (n_theta - 1)))
        return set_error(ZM_EINVAL, "n_theta must be a power of two >= 8 (got %d)", n_theta);
    if (n_theta > 2048) return set_error(ZM_EUNSUPPORTED, "n_theta > 2048 is not supported (got %d)", n_theta);
    if (n_theta < 2 * n_max + 1)
        return set_error(ZM_EINVAL, "n_theta (%d) must be >= 2 n_max + 1 (%d)", n_theta, 2 * n_max + 1);
    const unsigned grid = flags & 0xFu;
    const unsigned prec = flags & 0xF0u;
    if (grid != ZM_GRID_MIDPOINT && grid != ZM_GRID_GAUSS) return set_error(ZM_EINVAL, "unknown grid flag 0x%x", grid);
    if (prec != ZM_PREC_FP32 && prec != ZM_PREC_BF16X3 && prec != ZM_PREC_FP16X3)
        return set_error(ZM_EINVAL, "unknown precision flag 0x%x", prec);
    if (flags & ~0xFFu) return set_error(ZM_EINVAL, "unknown plan flags 0x%x", flags);

    auto* p = new zm_plan_s();
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return set_error(ZM_ECUDA, "no CUDA device");
    }
    p->n_max = n_max;
    p->n_rho = n_rho;
    p->n_theta = n_theta;
    p->log_theta = 0;
    while ((1 << p->log_theta) < n_theta) ++p->log_theta;
    p->P = num_moments(n_max);
    p->flags = flags;
    p->grid = (int)grid;
    p->prec = prec == ZM_PREC_BF16X3 ? PREC_BF16X3 : prec == ZM_PREC_FP16X3 ? PREC_FP16X3 : PREC_FP32;
    if (const char* f = std::getenv("ZM_FUSED")) p->fused_mode = (f[0] == '1') ? 1 : (f[0] == '0') ? -1 : 0;
    if (const char* f = std::getenv("ZM_RING_DFT")) p->dft_mode = (f[0] == '1') ? 1 : 0;
    if (const char* f = std::getenv("ZM_POLAR_DFT")) p->pdft_mode = (f[0] == '1') ? 1 : 0;
    int st = acquire_table(p->device, (int)grid, n_rho, n_max, &p->table);
    if (st == ZM_OK) st = build_plan_tables(p);
    if (st != ZM_OK) {
        free_plan(p);
        return st;
    }
    *plan = p;
    return ZM_OK;
}

extern "C" int zm_plan_destroy(zm_plan_t plan) {
    if (!plan) return ZM_OK;
    DeviceGuard g(plan->device);
    cudaDeviceSynchronize();
    free_plan(plan);
    return ZM_OK;
}

extern "C" int zm_plan_status(zm_plan_t plan) {
    if (!plan) return set_error(ZM_EINVAL, "plan is NULL");
    DeviceGuard g(plan->device);
    ZM_CUDA_TRY(cudaDeviceSynchronize());
    int st = 0;
    ZM_CUDA_TRY(cudaMemcpy(&st, plan->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        ZM_CUDA_TRY(cudaMemset(plan->status, 0, sizeof(int)));
        return set_error(st, "a kernel of this plan gave up a bounded wait");
    }
    return ZM_OK;
}

extern "C" int zm_plan_info(zm_plan_t plan, int* n_max, int* n_rho, int* n_theta, int* num, unsigned* flags) {
    if (!plan) return set_error(ZM_EINVAL, "plan is NULL");
    if (n_max) *n_max = plan->n_max;
    if (n_rho) *n_rho = plan->n_rho;
    if (n_theta) *n_theta = plan->n_theta;
    if (num) *num = plan->P;
    if (flags) *flags = plan->flags;
    return ZM_OK;
}

extern "C" int zm_plan_table(zm_plan_t plan, double* dst, void* stream) {
    if (!plan || !dst) return set_error(ZM_EINVAL, "NULL argument");
    DeviceGuard g(plan->device);
    ZM_CUDA_TRY(cudaMemcpyAsync(dst, plan->table->R, sizeof(double) * (size_t)plan->P * plan->n_rho,
                                cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return ZM_OK;
}

extern "C" int zm_plan_nodes(zm_plan_t plan, double* rho, double* wr, void* stream) {
    if (!plan) return set_error(ZM_EINVAL, "plan is NULL");
    DeviceGuard g(plan->device);
    if (rho)
        ZM_CUDA_TRY(cudaMemcpyAsync(rho, plan->table->rho, sizeof(double) * plan->n_rho,
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    if (wr)
        ZM_CUDA_TRY(cudaMemcpyAsync(wr, plan->table->wr, sizeof(double) * plan->n_rho,
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return ZM_OK;
}
