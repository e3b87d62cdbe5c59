// Radial projection for callers that cannot allocate device memory.
//
// zm_project keeps its split-K partial sums in a workspace that the plan grows
// with cudaMalloc when a larger batch arrives.  Some callers cannot let the
// library allocate at call time: their device memory is already handed out by
// another allocator (a framework's caching pool that reserved the GPU up
// front), or they run in a loop where cudaMalloc's implicit device-wide
// synchronisation and unbounded latency are not acceptable.  zm_project_noalloc
// computes the same projection (the FP32 form) with the partial sums in a fixed
// array in device memory that belongs to this file; it allocates nothing.
// There is no counterpart in the paper: this is an interface matter only.
#include <algorithm>
#include <mutex>

#include "zm_internal.cuh"

namespace zm {

// Fixed scratch: 2^21 floats (8 MiB).  Every GPU that loads this library's
// module holds it until the process exits.
constexpr size_t NOALLOC_FLOATS = (size_t)1 << 21;
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];

constexpr int NA_ROWS = 64, NA_COLS = 32, NA_K = 32;

// Split-K FP32 projection: part[s][row(m,n)][col] = sum over the s-th slice of
// i of A[row(m,n)][i] F[m][col][i] (the same contraction as k_project_fp32).
__global__ void __launch_bounds__(256)
k_project_noalloc(const float* __restrict__ A32, const float* __restrict__ F, const int* __restrict__ mrow,
                  int n_max, int n_rho, int ncol, int chunk, int P, float* __restrict__ part) {
    __shared__ float As[NA_K][NA_ROWS + 1];
    __shared__ float Fs[NA_K][NA_COLS + 1];
    const int m = blockIdx.x;
    const int col0 = blockIdx.y * NA_COLS;
    const int s = blockIdx.z;
    const int Km = (n_max - m) / 2 + 1;
    const int rowbase = mrow[m];
    const int ib = s * chunk, ie = min(n_rho, ib + chunk);
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    const float* Fm = F + ((size_t)m * ncol + col0) * n_rho;
    for (int rt = 0; rt < Km; rt += NA_ROWS) {
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        for (int kk = ib; kk < ie; kk += NA_K) {
            for (int e = tid; e < NA_ROWS * NA_K; e += 256) {
                const int row = e >> 5, k = e & 31;
                const int gr = rt + row, gk = kk + k;
                As[k][row] = (gr < Km && gk < ie) ? __ldg(&A32[(size_t)(rowbase + gr) * n_rho + gk]) : 0.f;
            }
            for (int e = tid; e < NA_COLS * NA_K; e += 256) {
                const int col = e >> 5, k = e & 31;
                const int gk = kk + k;
                Fs[k][col] = (col0 + col < ncol && gk < ie) ? __ldg(&Fm[(size_t)col * n_rho + gk]) : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < NA_K; ++k) {
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

// Sum of the S partial slices in a fixed order, Neumann factor, moment layout.
__global__ void k_project_noalloc_reduce(const float* __restrict__ part, int S, int P, int ncol,
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

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (in host code the symbol itself is only a stand-in).
static int noalloc_scratch(int dev, float** out) {
    static std::mutex mu;
    static float* addr[64] = {nullptr};
    if (dev < 0 || dev >= 64) return set_error(ZM_EUNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* a = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
        addr[dev] = static_cast<float*>(a);
    }
    *out = addr[dev];
    return ZM_OK;
}

}  // namespace zm

using namespace zm;

extern "C" int zm_project_noalloc(zm_plan_t plan, const float* spectra, int batch, float* out, unsigned flags,
                                  void* stream) {
    if (!plan || !spectra || !out) return set_error(ZM_EINVAL, "NULL argument");
    if (batch < 1) return set_error(ZM_EINVAL, "batch must be >= 1 (got %d)", batch);
    if (flags & ~ZM_NEUMANN) return set_error(ZM_EINVAL, "unknown flags 0x%x", flags);
    const int ncol = 2 * batch;
    const size_t one_slice = (size_t)plan->P * ncol;
    if (one_slice > NOALLOC_FLOATS)
        return set_error(ZM_EINVAL,
                         "zm_project_noalloc: P(n_max) * 2 * batch = %zu floats exceeds its fixed scratch of %zu "
                         "floats; use a smaller batch or zm_project",
                         one_slice, NOALLOC_FLOATS);
    DeviceGuard g(plan->device);
    if (!g.ok) return set_error(ZM_ECUDA, "cannot select device %d", plan->device);
    float* part = nullptr;
    int s = noalloc_scratch(plan->device, &part);
    if (s != ZM_OK) return s;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device) != cudaSuccess || sms <= 0)
        sms = 148;
    const int ctiles = (ncol + NA_COLS - 1) / NA_COLS;
    const int base = (plan->n_max + 1) * ctiles;
    const int kchunks = (plan->n_rho + NA_K - 1) / NA_K;
    int S = std::max(1, std::min(kchunks, (4 * sms + base - 1) / base));
    while (S > 1 && (size_t)S * one_slice > NOALLOC_FLOATS) --S;
    const int chunk = ((kchunks + S - 1) / S) * NA_K;
    S = (plan->n_rho + chunk - 1) / chunk;
    const cudaStream_t st = (cudaStream_t)stream;
    dim3 grid(plan->n_max + 1, ctiles, S);
    k_project_noalloc<<<grid, 256, 0, st>>>(plan->A32, spectra, plan->mrow, plan->n_max, plan->n_rho, ncol, chunk,
                                            plan->P, part);
    ZM_LAUNCH_CHECK("k_project_noalloc");
    const int tot = batch * plan->P;
    k_project_noalloc_reduce<<<(tot + 255) / 256, 256, 0, st>>>(part, S, plan->P, ncol, plan->pair_nm, plan->mrow,
                                                                 batch, (flags & ZM_NEUMANN) ? 1 : 0, out);
    ZM_LAUNCH_CHECK("k_project_noalloc_reduce");
    return ZM_OK;
}
