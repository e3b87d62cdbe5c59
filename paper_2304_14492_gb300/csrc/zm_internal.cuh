// Internal declarations of the Zernike moment library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "../../include/zm.h"

namespace zm {

// ---------------------------------------------------------------- errors
int set_error(int status, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

#define ZM_CUDA_TRY(expr)                                        \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return ::zm::cuda_error(_e, #expr); \
    } while (0)

#define ZM_LAUNCH_CHECK(what)                                    \
    do {                                                         \
        cudaError_t _e = cudaGetLastError();                     \
        if (_e != cudaSuccess) return ::zm::cuda_error(_e, what); \
        ::zm::count_launch();                                    \
    } while (0)

// Programmatic dependent launch: a kernel launched this way may start while
// the previous kernel of the stream is finishing.  It runs its prologue (shared
// memory, TMEM, barriers, reads of plan constants) and then griddep_wait(),
// which returns once the previous kernel has completed and its writes are
// visible; nothing before that wait may read or write memory the previous
// kernels use.  griddep_launch() lets the next kernel start early.  Both are
// no-ops when the launch carries no programmatic dependency.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Streaming multiprocessors of device `dev` (cached).
inline int num_sms(int dev) {
    static int cached[64] = {0};
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}

// launch_pdl() with thread-block clusters of `cluster` CTAs.
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl_cluster(void (*kernel)(Params...), dim3 grid, dim3 block, dim3 cluster, size_t smem,
                                      cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = cluster.x;
    attr[1].val.clusterDim.y = cluster.y;
    attr[1].val.clusterDim.z = cluster.z;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

#define ZM_LAUNCH_PDL(what, kernel, grid, block, smem, st, ...)                         \
    do {                                                                              \
        cudaError_t _e = ::zm::launch_pdl(kernel, grid, block, smem, st, __VA_ARGS__);  \
        if (_e != cudaSuccess) return ::zm::cuda_error(_e, what);                     \
        ::zm::count_launch();                                                         \
    } while (0)

// Makes `dev` current for the lifetime of the guard and restores the caller's
// device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------- index set
// Stored pairs (n, m): m >= 0, n - m even, ordered by n then m (Sec. 2).
inline int num_moments(int n_max) {
    if (n_max < 0) return -1;
    const int n = n_max + 1;               // off(n) of the next order
    const int q = n / 2;
    return (n % 2 == 0) ? q * (q + 1) : (q + 1) * (q + 1);
}
__host__ __device__ inline int moment_index(int n, int m) {
    const int q = n / 2;
    const int off = (n % 2 == 0) ? q * (q + 1) : (q + 1) * (q + 1);
    return off + (m - (n & 1)) / 2;
}

// ---------------------------------------------------------------- FP64 table cache
// One Eq. 7 table per (device, grid, N_rho), grown in n_max; plans hold a
// reference, so a table outlives its cache slot while plans use it.
struct ZrpTable {
    int device = -1, grid = 0, n_rho = 0, n_max = -1, n_z = 0;
    double* rho = nullptr;   // [n_rho] radial nodes
    double* wr = nullptr;    // [n_rho] radial weights (Jacobian rho included)
    double* R = nullptr;     // [P(n_max)][n_rho], moment order
    float plan_ms = 0.f;     // time of the table build
    ~ZrpTable();
};
int acquire_table(int device, int grid, int n_rho, int n_max, std::shared_ptr<ZrpTable>* out);

// ---------------------------------------------------------------- plan
enum Prec { PREC_FP32 = 0, PREC_BF16X3 = 1, PREC_FP16X3 = 2 };

struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
    int grow(size_t need);   // cudaMalloc on growth only (synchronous)
    ~Workspace();
};

}  // namespace zm

struct zm_plan_s {
    int device = 0;
    int n_max = 0, n_rho = 0, n_theta = 0, log_theta = 0, P = 0;
    unsigned flags = 0;
    int grid = 0, prec = 0;
    std::shared_ptr<zm::ZrpTable> table;
    // device constants of the plan
    float* rho32 = nullptr;     // [n_rho]
    float* A32 = nullptr;       // [P][n_rho], m-major rows: 2(n+1)/N_theta * wr_i * R_nm(rho_i)
    float* R32m = nullptr;      // [P][n_rho], m-major rows: R_nm(rho_i) (reconstruction)
    uint16_t* Ahi = nullptr;    // [P][n_rho], m-major: hi part of A (bf16 or fp16 bits)
    uint16_t* Alo = nullptr;    // [P][n_rho], m-major: lo part of A
    float a_scale = 1.f;        // Ahi/Alo hold A * a_scale (fp16 range); 1 for bf16
    float2* tw = nullptr;       // [n_theta] e^{-2 pi i j / N_theta}
    float2* cs = nullptr;       // [n_theta] (cos theta_k, sin theta_k)
    int* mrow = nullptr;        // [n_max + 2] first m-major row of each m
    int2* pair_nm = nullptr;    // [P] (n, m) of each moment index
    std::vector<int> mrow_h;
    // bf16 plans with K_m <= 128: the A halves as tensor-core operand blocks,
    // chunk by chunk of 64 radial nodes, each chunk in the canonical K-major
    // core-matrix layout (8 rows x 16 B; 8-row groups 1 KB apart), so that one
    // bulk copy moves a chunk into shared memory.  Half h, order m, chunk c:
    // Ablk + h * ablk_half + ablk_off_h[m] + c * ceil(K_m / 8) KB.
    uint8_t* Ablk = nullptr;
    std::vector<long long> ablk_off_h;
    long long* ablk_off = nullptr;   // device copy of ablk_off_h
    long long ablk_half = 0;
    int n_chunks = 0;                // ceil(n_rho / 64)
    // bf16 plans: R (reconstruction) split into hi / lo operand blocks, one per
    // (m, 128-ring tile, 64-order chunk); half h of order m starts at
    // Rblk + h * rblk_half + rblk_off_h[m]
    uint8_t* Rblk = nullptr;
    std::vector<long long> rblk_off_h;
    long long* rblk_off = nullptr;
    long long rblk_half = 0;
    int n_rtiles = 0;
    // workspace (grown on demand)
    zm::Workspace ws_F;         // ring spectra F[m][b][2][n_rho] (fp32)
    zm::Workspace ws_fhat;      // polar samples f[b][i][k] (fp32)
    zm::Workspace ws_part;      // split-K partial sums of the projection
    zm::Workspace ws_G;         // reconstruction radial spectra G[b][m][2][n_rho]
    zm::Workspace ws_red;       // reduction partials
    zm::Workspace ws_scale;     // per-image min / max (normalisation)
    zm::Workspace ws_colmax;    // per-column max |F| (fp16 split scaling)
    zm::Workspace ws_Fblk;      // ring spectra as bf16 hi / lo operand blocks (blocked projection)
    int* status = nullptr;      // device status word: ZM_ETIMEOUT after a timed-out wait
    int* work = nullptr;        // device {next item, CTAs done} of the inverse ring FFT, 0 between launches
    // launch choices
    int kb_rings = 8;           // rings per CTA in the resample + FFT kernel
    // set by the batch autotuner (0 = built-in heuristic)
    int tune_gather = 0;        // 1: resample with the fused gather kernel even where TMA could stage
    int tune_rings = 0;         // rings per CTA of the ring-FFT kernels (2, 4 or 8)
    int tune_split = 0;         // CTAs per SM aimed at by the projection's radial split
    // resampling fused with the ring FFT (ring_fused.cu): 0 = for images of at
    // most FUSED_AUTO_SAMPLES polar samples (where it measured faster than
    // the tile resampler + ring FFT), 1 = wherever it applies, -1 = never;
    // set from the environment variable ZM_FUSED ("1" / "0") at plan creation
    int fused_mode = 0;
    int staged_batch = 0;       // images whose spectra zm_stage_spectra left in the workspace
    // resampling with the angular transform on the tensor cores (ring_dft.cu),
    // bf16 plans with the blocked projection: 1 = wherever it applies, else
    // never (the default: the tile path measured faster on the 4K frame); set
    // from the environment variable ZM_RING_DFT ("1") at plan creation
    int dft_mode = 0;
    uint8_t* dft = nullptr;     // its DFT tiles (bf16 hi / lo), built on first use
    // the angular sums from polar samples on the tensor cores (polar_dft.cu),
    // bf16 plans with the blocked projection and n_max <= 127: 1 = wherever it
    // applies, else never (the default: the radix ring FFT measured as fast on
    // the 4K frame, and the zm_moments step faster with it); set from the
    // environment variable ZM_POLAR_DFT ("1") at plan creation
    int pdft_mode = 0;
    uint8_t* dft32 = nullptr;   // its 32-deep DFT tiles, built on first use
};

namespace zm {

// ---------------------------------------------------------------- launchers
// Fblk: write the spectra as bf16 operand blocks instead of F (see fblk_row).
int launch_spectra(zm_plan_t p, const zm_image_t* imgs, const float* fhat_in, int batch,
                   float* F, float* fhat_out, bool resample_only, cudaStream_t st, uint8_t* Fblk = nullptr);
int launch_projection(zm_plan_t p, const float* F, int batch, float* out, unsigned flags,
                      cudaStream_t st);
// FP32 split-K projection with its partial sums in `part` (part_floats floats);
// the radial split is lowered until its slices fit (ZM_EINVAL if one does not).
int launch_projection_fp32_parts(zm_plan_t p, const float* F, int batch, float* out, unsigned flags, float* part,
                                 size_t part_floats, cudaStream_t st);
// Moments of a batch (images, or polar samples when fhat_in is set): ring
// spectra, then the projection; bf16 plans take the blocked tensor-core path.
int launch_moments(zm_plan_t p, const zm_image_t* imgs, const float* fhat_in, int batch, float* out,
                   float* fhat_out, unsigned flags, cudaStream_t st);
// Blocked tensor-core projection (project_tc.cu).
int build_tc_blocks(zm_plan_t p);
bool blocked_projection(zm_plan_t p);
// consume: the blocks are scratch of this call (zm_moments), dropped from L2 once read
int launch_projection_blocked(zm_plan_t p, const uint8_t* Fblk, int batch, float* out, unsigned flags,
                              cudaStream_t st, bool consume = false);
// Tensor-core radial reconstruction (recon_tc.cu), bf16 plans.
int build_recon_blocks(zm_plan_t p);
int launch_radial_tc(zm_plan_t p, const float* moments, int batch, unsigned flags, float* G, cudaStream_t st);

// Radial reconstruction spectra G (Eq. 9), ring-block-major so that the 8 rings
// an inverse-FFT block transforms are one contiguous run: image b, ring i,
// order m, re/im c at ((b * nrb + i / 8) * (n_max + 1) + m) * 16 + c * 8 + i % 8,
// nrb = ceil(n_rho / 8).
__host__ __device__ inline size_t g_index(int b, int i, int m, int c, int nrb, int nm1) {
    return ((((size_t)b * nrb + (i >> 3)) * nm1 + m) << 4) + (c << 3) + (i & 7);
}
__host__ __device__ inline size_t g_floats(int batch, int n_rho, int n_max) {
    return (size_t)batch * ((n_rho + 7) / 8) * (n_max + 1) * 16;
}

// Layout of the spectra blocks: half-size in bytes, and the byte offset of the
// 16-byte row holding F[m][col][i .. i+7] (i a multiple of 8) within a half.
__host__ __device__ inline size_t fblk_half_bytes(int n_max, int n_chunks, int ncol) {
    return (size_t)(n_max + 1) * n_chunks * ((ncol + 7) / 8) * 1024;
}
__host__ __device__ inline size_t fblk_row(int m, int i, int col, int n_chunks, int ncol) {
    const int cg = (ncol + 7) / 8;
    return ((((size_t)m * n_chunks + (i >> 6)) * cg + (col >> 3)) << 10) + (((i & 63) >> 3) << 7) + ((col & 7) << 4);
}
void count_launch(int n = 1);
int launch_reconstruct(zm_plan_t p, const float* moments, int batch, float* out,
                       unsigned flags, cudaStream_t st);
int launch_polar_to_cart(zm_plan_t p, const float* polar, int batch, const zm_canvas_t* cv,
                         cudaStream_t st);
int launch_errors(zm_plan_t p, const zm_image_t* ref, const zm_image_t* test,
                  const float* fhat, const float* frec, int batch, double* out,
                  cudaStream_t st);
int launch_disk_minmax(zm_plan_t p, const zm_image_t* imgs, int batch, float* out,
                       cudaStream_t st);
int launch_minmax_normalize(zm_plan_t p, const zm_canvas_t* cv, int batch,
                            const float* target, cudaStream_t st);
int build_plan_tables(zm_plan_t p);

// ---------------------------------------------------------------- shared device code
struct GeoImage {          // device-side image descriptor (geometry resolved)
    const float* data;
    long long pitch;
    int h, w;
    float cx, cy, r;
};

inline GeoImage resolve(const zm_image_t& im) {
    GeoImage g;
    g.data = im.data;
    g.pitch = im.pitch;
    g.h = im.height;
    g.w = im.width;
    if (im.radius > 0.f) {
        g.cx = im.cx; g.cy = im.cy; g.r = im.radius;
    } else {
        g.cx = 0.5f * (float)(im.width - 1);
        g.cy = 0.5f * (float)(im.height - 1);
        g.r = 0.5f * (float)(im.width < im.height ? im.width : im.height);
    }
    return g;
}

int check_images(const zm_image_t* imgs, int batch);

// Cartesian-tile resampling (resample_tiles.cu)
bool tma_eligible(const zm_image_t& im);
bool same_geometry(const zm_image_t& a, const zm_image_t& b);
// keep_l2: fhat is scratch that the next kernel reads (stored with an L2
// evict_last policy)
int launch_resample_tiles(zm_plan_t p, const zm_image_t* imgs, int b0, int nb, float* fhat, cudaStream_t st,
                          bool keep_l2 = false);
void release_tiles(zm_plan_t p);

// Resampling fused with the ring FFT (ring_fused.cu): polar samples stay on chip
constexpr long long FUSED_AUTO_SAMPLES = 1ll << 17;
bool fused_eligible(zm_plan_t p, const zm_image_t& im);
int launch_ring_fused(zm_plan_t p, const zm_image_t* imgs, int b0, int nb, int batch, float* F, uint8_t* Fblk,
                      float* fhat_out, cudaStream_t st);
long long fused_staged_bytes(zm_plan_t p, const zm_image_t& im);
void release_fused(zm_plan_t p);

// Resampling fused with the angular transform as a tensor-core DFT
// (ring_dft.cu): writes the blocked projection's operand blocks only
bool dft_eligible(zm_plan_t p, const zm_image_t& im);
int launch_ring_dft(zm_plan_t p, const zm_image_t* imgs, int b0, int nb, int batch, uint8_t* Fblk, cudaStream_t st);
void release_dft(zm_plan_t p);

// The angular sums from polar samples as a tensor-core DFT (polar_dft.cu):
// writes the blocked projection's operand blocks
bool polar_dft_eligible(zm_plan_t p, const float* fhat);
int launch_polar_dft(zm_plan_t p, const float* fhat, int b0, int nb, int batch, uint8_t* Fblk, cudaStream_t st);

}  // namespace zm
