/*
 * zm.h - C ABI of the GB300 (sm_103a) FFT-based Zernike moment library.
 *
 * Method: M. Al-Rawi, "Ultra-Fast Zernike Moments using FFT and GPU"
 * (arXiv 2304.14492).  Moments follow Eq. 1 on a polar grid; the radial
 * polynomials come from the Chebyshev-U / DFT identity of Sec. 2.1 (Eq. 7-8);
 * reconstruction follows Eq. 9; the Neumann factor is Eq. 14-15; the errors are
 * Eq. 10 and Eq. 13 (Sec. 2.4); min-max normalisation is the step of Sec. 3 /
 * Table I.
 *
 * Conventions shared by every entry point:
 *  - Every function returns a status code (ZM_OK = 0 on success) and never
 *    aborts.  On failure zm_last_error() gives a per-thread detail string.
 *  - Image, moment and output buffers are DEVICE pointers owned by the caller
 *    (e.g. the data_ptr() of a CUDA tensor).  The descriptor arrays
 *    (zm_image_t / zm_canvas_t) are HOST arrays read during the call.
 *  - Moment buffers and polar reconstruction outputs must be 8-byte aligned
 *    (they are accessed as float pairs); ZM_EINVAL otherwise.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously on it; results are valid once the stream
 *    has been synchronised.  A plan may be used from one stream at a time.
 *  - Geometry: pixel (x = column, y = row) has its centre at integer
 *    coordinates; the unit disk maps to the circle of centre (cx, cy) and
 *    radius `radius` pixels; theta runs counter-clockwise with y pointing up,
 *    so the polar point (rho, theta) sits at X = cx + radius rho cos(theta),
 *    Y = cy - radius rho sin(theta).  radius <= 0 selects the inscribed,
 *    centred disk: cx = (W-1)/2, cy = (H-1)/2, radius = min(H, W)/2.
 *  - Polar grid: theta_k = 2 pi k / N_theta; rho_i = (i + 1/2) / N_rho
 *    (midpoint rule, default) or the Gauss-Legendre nodes on [0, 1].  Image
 *    values are sampled bilinearly, neighbours outside the image count as 0.
 *  - Moment layout: for each image, P(n_max) complex values as interleaved
 *    float pairs (re, im), in the order n = 0..n_max, then m = n mod 2, ..., n
 *    step 2 (only m >= 0 is stored; Z_{n,-m} = conj(Z_nm), Sec. 2).  The index
 *    of (n, m) is zm_index(n, m); P(n_max) = zm_num_moments(n_max).
 */
#ifndef ZM_H
#define ZM_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define ZM_OK            0
#define ZM_EINVAL        1  /* bad argument: sizes, flags, null pointer      */
#define ZM_ENOMEM        2  /* device allocation failed or budget exceeded   */
#define ZM_ECUDA         3  /* CUDA launch / API error (detail kept)         */
#define ZM_ETIMEOUT      4  /* a bounded wait ran out                        */
#define ZM_EUNSUPPORTED  5  /* valid request the library does not implement  */

/* ---- plan flags (zm_plan) ---------------------------------------------- */
#define ZM_GRID_MIDPOINT 0x0u   /* rho_i = (i + 1/2)/N_rho, weight rho_i/N_rho */
#define ZM_GRID_GAUSS    0x1u   /* Gauss-Legendre nodes and weights on [0, 1]  */
#define ZM_PREC_FP32     0x00u  /* radial projection in FP32 (CUDA cores)      */
#define ZM_PREC_BF16X3   0x10u  /* projection on tensor cores, bf16 hi+lo split */
#define ZM_PREC_FP16X3   0x20u  /* projection on tensor cores, fp16 hi+lo split */

/* ---- call flags --------------------------------------------------------- */
#define ZM_NEUMANN       0x1u   /* see zm_moments / zm_reconstruct            */

typedef struct zm_plan_s* zm_plan_t;

/* A read-only device image.  Row y starts at data + y * pitch (elements). */
typedef struct {
    const float* data;
    int height, width;
    long long pitch;
    float cx, cy, radius;
} zm_image_t;

/* A writable device image of the same layout (reconstruction target). */
typedef struct {
    float* data;
    int height, width;
    long long pitch;
    float cx, cy, radius;
} zm_canvas_t;

/* ---- index set (D5 layout; Sec. 2, Eq. 1 conditions) -------------------- */

/* P(n_max): number of stored moments with n <= n_max; -1 if n_max < 0. */
int zm_num_moments(int n_max);

/* Position of (n, m) in a moment vector; -1 unless 0 <= m <= n, n-m even. */
int zm_index(int n, int m);

/* Static text for a status code. */
const char* zm_strerror(int status);

/* Detail of the last failure on the calling thread ("" if none). */
const char* zm_last_error(void);

/* ---- plans (Sec. 2.1, Eq. 7-8) ------------------------------------------- */

/*
 * Create a plan for moments up to order n_max on an N_rho x N_theta polar grid.
 * Builds, on the current CUDA device, the FP64 table R_nm(rho_i) with Eq. 7
 * (the DFT over k of U_n(rho cos(2 pi k / N_z)) with N_z the next power of two
 * >= max(8, 2 n_max + 2), so N_z > n + m always), the projection operands
 * derived from it, and the angular tables.  Synchronous; allocates device
 * memory.  FP64 tables are cached per (device, grid, N_rho) and shared by plans
 * of any n_max up to the largest built so far.
 *  n_max   >= 0
 *  n_rho   in [1, 65536]
 *  n_theta a power of two in [8, 2048] with n_theta >= 2 n_max + 1
 *  flags   one ZM_GRID_* | one ZM_PREC_*
 * The calls on one plan share its workspace and counters: order them (one
 * stream, or streams joined by events); concurrent pipelines take one plan
 * each.
 * Errors: ZM_EINVAL, ZM_ENOMEM, ZM_ECUDA, ZM_EUNSUPPORTED.
 */
int zm_plan(zm_plan_t* plan, int n_max, int n_rho, int n_theta, unsigned flags);

/* Release the plan and its workspace (waits for the device). NULL is ok. */
int zm_plan_destroy(zm_plan_t plan);

/* Grow the plan's workspace so that later calls with batch <= `batch`
 * allocate nothing (e.g. before CUDA graph capture).  Synchronous. */
int zm_plan_reserve(zm_plan_t plan, int batch);

/* Synchronise the device, then report ZM_ETIMEOUT if any kernel of this plan
 * gave up a bounded wait since the previous call (and clear that flag);
 * ZM_OK otherwise. */
int zm_plan_status(zm_plan_t plan);

/* Plan parameters; any output pointer may be NULL. */
int zm_plan_info(zm_plan_t plan, int* n_max, int* n_rho, int* n_theta,
                 int* num_moments, unsigned* flags);

/* Copy the FP64 table R_nm(rho_i), shape [P(n_max)][N_rho] in moment order,
 * to device buffer `dst` (Eq. 7 output).  Asynchronous on `stream`. */
int zm_plan_table(zm_plan_t plan, double* dst, void* stream);

/* Copy the radial nodes rho_i and radial weights wr_i (the Jacobian rho
 * included: sum_i wr_i g(rho_i) approximates the integral of g(rho) rho over
 * [0, 1]) to device buffers of N_rho doubles.  Either may be NULL. */
int zm_plan_nodes(zm_plan_t plan, double* rho, double* wr, void* stream);

/* ---- moments (Eq. 1, Eq. 14-15) ------------------------------------------ */

/*
 * Zernike moments of `batch` images: bilinear polar resampling, a real FFT of
 * every ring, and the radial projection
 *     Z_nm = (n+1)/pi * sum_i wr_i (2 pi / N_theta) R_nm(rho_i) F_m(rho_i),
 * F_m(rho_i) = sum_k f(rho_i, theta_k) e^{-j m theta_k}.
 *  imgs  host array of `batch` device image descriptors (any sizes)
 *  out   device float[batch][P][2]
 *  flags ZM_NEUMANN divides each moment by eps_m (2 for m = 0, else 1; Eq. 14)
 * Path: images with a 16-byte aligned base and a pitch and width that are
 * multiples of 4 floats are resampled and ring-transformed in one kernel (the
 * polar samples stay on chip) when a plan has at most 2^17 polar samples per
 * image, where that kernel measured faster; larger grids resample by image
 * tiles into a workspace first.  Both paths give the same moments, bit for
 * bit.  The environment variable ZM_FUSED, read when a plan is created,
 * overrides the choice: "1" fuses wherever the geometry fits the kernel's
 * stage buffers, "0" never fuses.  ZM_RING_DFT=1, read likewise, sends bf16x3
 * plans with n_max <= 127 to a third kernel that resamples and computes the
 * angular sums of Eq. 1 as a product with the DFT matrix on the tensor cores
 * (split operands, FP32 accumulation; moments within the split bar of the
 * FFT paths, not bit-equal to them); it is off by default, being slower than
 * the tile path on the 4K frame.  ZM_POLAR_DFT=1 likewise sends the angular
 * transform of polar samples (the tile path's resampled samples, and
 * zm_moments_polar) of such plans to a tensor-core DFT instead of the radix
 * ring FFT; also off by default (no faster on the 4K frame).
 * Errors: ZM_EINVAL (batch < 1, null pointers, image < 1x1, bad pitch),
 * ZM_ENOMEM (workspace growth), ZM_ECUDA.
 */
int zm_moments(zm_plan_t plan, const zm_image_t* imgs, int batch, float* out,
               unsigned flags, void* stream);

/* As zm_moments, and also writes the polar samples f(rho_i, theta_k) to
 * `fhat` (device float[batch][N_rho][N_theta]) when it is not NULL. */
int zm_moments_ex(zm_plan_t plan, const zm_image_t* imgs, int batch, float* out,
                  float* fhat, unsigned flags, void* stream);

/* Moments of functions already sampled on the plan's polar grid:
 * `fhat` is device float[batch][N_rho][N_theta]. */
int zm_moments_polar(zm_plan_t plan, const float* fhat, int batch, float* out,
                     unsigned flags, void* stream);

/*
 * Host frames -> device disk boxes (no counterpart in the paper; the data
 * movement in front of Eq. 1).  Only the pixels a polar sample's bilinear
 * stencil can touch are needed.  For each image the device buffer holds the
 * bounding box of its disk, columns floor(cx - r) - 1 (rounded down to a
 * multiple of 4) .. floor(cx + r) + 2 and rows floor(cy - r) - 1 ..
 * floor(cy + r) + 2, clipped to the image, boxes packed one after another with
 * a 16-byte multiple as pitch.  Of box row y only the span the disk covers is
 * copied: columns floor(cx - hw) - 3 (rounded down to a multiple of 4) ..
 * floor(cx + hw) + 3 with hw = sqrt(r^2 - d^2), d = max(0, |y - cy| - 1),
 * clipped to the box (rows with d >= r: none); the other pixels of the box
 * are left as they were, and no entry point reads them.  A kernel copies the
 * spans from `host_imgs[b].data` (host memory the device can read: pinned or
 * registered, or pageable where the device reaches pageable memory through
 * the host page tables) into `dev` and fills `dev_imgs[b]` with the device
 * descriptor of the box and the shifted geometry (explicit cx, cy, radius), so
 * that zm_moments* on dev_imgs gives the moments of the host images.  `dev`
 * (device, 16-byte aligned) must hold zm_upload_disk_bytes(...) bytes;
 * zm_upload_disk_traffic(...) gives the bytes a call reads from the host.
 * Asynchronous on `stream`: the host images must stay valid until it has run.
 * ZM_EUNSUPPORTED if a host buffer cannot be read by the device; ZM_EINVAL for
 * bad sizes or a short `dev`.
 */
int zm_upload_disk_bytes(const zm_image_t* host_imgs, int batch, unsigned long long* bytes);
int zm_upload_disk_traffic(const zm_image_t* host_imgs, int batch, unsigned long long* bytes);
int zm_upload_disk(const zm_image_t* host_imgs, int batch, float* dev, unsigned long long dev_bytes,
                   zm_image_t* dev_imgs, void* stream);

/*
 * Zernike moments by Cartesian summation (Sec. 2, Eq. 3-6; the route of the
 * paper's Fig. 5 timings): for each image b and each requested pair
 * (n, m) = (nm[2k], nm[2k+1]) (host int[count][2], m >= 0, n - m even,
 * (n - m)/2 < 512),
 *   out[b][k] = (n + 1)/(pi r^2) sum f(x, y) R_nm(rho) e^{-j m theta}
 * over the pixel centres with x^2 + y^2 <= 1, x = (col - cx)/r,
 * y = (cy - row)/r (the polar path's geometry; the pixel area 1/r^2 is
 * Delta^2 of Eq. 5, i.e. 4/N^2 for an N x N image), divided by eps_m with
 * ZM_NEUMANN.  No interpolation.  When cx and cy sit at the same offset, 0 or
 * 1/2, from the pixel grid (the centred default always does), the pixels are
 * taken in orbits of the 8-point symmetry.  `imgs`: device images (host array
 * of descriptors); `out`: device float[batch][count][2]; `work`: device
 * scratch of zm_cartesian_work_bytes() bytes, 8-byte aligned; asynchronous on
 * `stream`.  ZM_EINVAL for a bad pair, NULL pointers or a short `work`.
 */
int zm_cartesian_work_bytes(int batch, int count, unsigned long long* bytes);
int zm_cartesian_moments(const zm_image_t* imgs, int batch, const int* nm, int count,
                         float* out, void* work, unsigned long long work_bytes,
                         unsigned flags, void* stream);

/* Only the bilinear polar resampling (Sec. 2.5): fhat = device
 * float[batch][N_rho][N_theta]. */
int zm_resample(zm_plan_t plan, const zm_image_t* imgs, int batch, float* fhat,
                void* stream);

/* The two halves of zm_moments, for callers that keep the ring spectra.
 * Spectra layout: device float[n_max+1][batch][2][N_rho] with
 *   spectra[m][b][0][i] + j spectra[m][b][1][i] = F_m(rho_i)
 *                       = sum_k f(rho_i, theta_k) e^{-j m theta_k}
 * for image b (the angular transform of Eq. 1, before any weighting).
 * zm_ring_spectra also writes the polar samples to `fhat` unless it is NULL. */
int zm_ring_spectra(zm_plan_t plan, const zm_image_t* imgs, int batch, float* spectra,
                    float* fhat, void* stream);

/* Radial projection of given spectra (layout above, `batch` images) into
 * moments out = device float[batch][P][2]; flags as zm_moments. */
int zm_project(zm_plan_t plan, const float* spectra, int batch, float* out,
               unsigned flags, void* stream);

/* The projection of zm_project for callers that cannot allocate device memory
 * at call time: their device memory is already handed out by another
 * allocator (e.g. a framework's caching pool that reserved the GPU up front),
 * or they run in a loop where cudaMalloc's device-wide synchronisation and
 * unbounded latency are not acceptable.  It allocates nothing: the split-K
 * partial sums live in a fixed 8 MiB array in device memory that belongs to
 * the library (held by every GPU that loads it, until the process exits).
 * The paper has no counterpart; this is an interface matter only.
 *  - Computes in FP32 whatever the plan's precision flag; the plan itself is
 *    made beforehand with zm_plan (which does allocate).
 *  - Requires P(n_max) * 2 * batch <= 2^21 floats; larger requests return
 *    ZM_EINVAL without touching the device.
 *  - The first call on a device looks up the array's device address (set-up,
 *    with that device current); make that first call before any stream
 *    capture.  The address is kept for the process's lifetime: resetting the
 *    device (cudaDeviceReset) between calls is not supported.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents; each call overwrites the part it reads, so nothing needs
 *    clearing, but calls that overlap on the GPU (other streams, other
 *    threads) race: serialise them.
 * Arguments, layouts and flags as zm_project. */
int zm_project_noalloc(zm_plan_t plan, const float* spectra, int batch, float* out,
                       unsigned flags, void* stream);

/* The two stages of zm_moments as separate calls (Eq. 1): zm_stage_spectra
 * computes the ring spectra F_m(rho_i), m <= n_max, of `batch` images (the
 * resampling and angular FFT of zm_moments) into the plan's workspace, in the
 * form the plan's projection reads; zm_stage_project then applies the radial
 * projection (and ZM_NEUMANN) to them and writes out = device
 * float[batch][P][2].  zm_moments gives the same moments as the two calls in
 * turn.  Use them to time or overlap the stages; the spectra stay in the plan
 * until the next call that computes spectra with this plan, so calls on one
 * plan must not overlap on the GPU.  Such a call in between (zm_moments and
 * its variants use the same workspace, and zm_moments drops its spectra from
 * L2 once projected) leaves zm_stage_project with undefined values until the
 * next zm_stage_spectra.  zm_stage_project returns ZM_EINVAL if `batch`
 * differs from the last zm_stage_spectra's.  Asynchronous on `stream`;
 * zm_stage_spectra may grow the workspace (cudaMalloc). */
int zm_stage_spectra(zm_plan_t plan, const zm_image_t* imgs, int batch, void* stream);
int zm_stage_project(zm_plan_t plan, int batch, float* out, unsigned flags, void* stream);

/* ---- uneven batches ------------------------------------------------------ */

/* One request of an uneven batch: an image with its own order and polar grid.
 * out: device float[P(n_max)][2] (moment layout as zm_moments). */
typedef struct {
    zm_image_t image;
    int n_max;
    int n_rho, n_theta;      /* n_theta a power of two >= 2 n_max + 1 */
    float* out;
} zm_request_t;

typedef struct zm_batch_s* zm_batch_t;

/*
 * Prepare an uneven batch: requests are grouped by (n_rho, n_theta); each group
 * gets one plan whose n_max is the group's largest (a request's moments are the
 * prefix P(n_max) of the group's, since Z_nm does not depend on the plan's
 * order).  Workspaces are reserved, and for every group the launch choices
 * (resampling by TMA tiles or by the fused gather kernel, rings per CTA of the
 * ring FFT, radial split of the projection) are picked by timing candidates on
 * the given images, or read from the JSON cache named by the environment
 * variable ZM_TUNE_CACHE (which is then updated).  Synchronous; allocates.
 *  plan_flags: one ZM_GRID_* | one ZM_PREC_*, for every group.
 */
int zm_batch_create(zm_batch_t* batch, const zm_request_t* reqs, int count, unsigned plan_flags);

/*
 * Moments of every request of the batch, enqueued on `stream` as one CUDA graph
 * launch.  `reqs` must match the batch's requests in count, sizes, geometry,
 * orders and grids; its image and output pointers may change, in which case
 * the graph is captured again (synchronously) before it is launched.
 *  flags: ZM_NEUMANN as zm_moments.
 */
int zm_batch_run(zm_batch_t batch, const zm_request_t* reqs, unsigned flags, void* stream);

/* Number of groups (plans) of the batch and number of graph captures so far;
 * either pointer may be NULL. */
int zm_batch_info(zm_batch_t batch, int* groups, int* captures);

/* Release the batch, its plans and graph (waits for the device). */
int zm_batch_destroy(zm_batch_t batch);

/* ---- serving (continuous batching) ---------------------------------------- */

typedef struct zm_server_s* zm_server_t;

typedef struct {
    unsigned long long hbm_budget;  /* bytes of device memory for requests in flight
                                       (images and moments); 0 = 1 GiB */
    int streams;                    /* CUDA streams work overlaps on; 0 = 4 */
    int max_group;                  /* most requests launched together per grid; 0 = 64 */
    unsigned plan_flags;            /* ZM_GRID_* | ZM_PREC_* of every plan */
    int max_wait_us;                /* batching window: an admitted request waits at
                                       most this long for others of its grid before
                                       its group launches, unless the group is full
                                       or the budget is exhausted; 0 = launch as soon
                                       as the grid's stream has room */
} zm_server_config_t;

typedef struct {
    unsigned long long submitted, completed, rejected;
    unsigned long long groups_launched;
    double p50_ms, p99_ms, max_ms;  /* latency: submit -> result on the host */
    double images_per_s;            /* completed / (last completion - first submit) */
    unsigned long long peak_bytes;  /* largest device footprint of requests in flight */
    int host_direct;                /* 1: kernels read the host images and write the results
                                       in place (the GPU reaches pageable host memory through
                                       the host page tables); 0: copies through a pinned mirror
                                       of the arena (also forced by ZM_SERVER_STAGING=1) */
} zm_server_stats_t;

/*
 * A server that computes moments of host images as requests arrive.  A
 * scheduler thread admits waiting requests while their device bytes fit the
 * budget (the arena is allocated once, here), groups the admitted ones by
 * polar grid (one plan per (n_rho, n_theta), order = the largest seen), and
 * launches each group on the stream bound to its grid: copy in, resampling,
 * ring FFT, projection, copy out (by kernels reading and writing the callers'
 * host buffers where the GPU reaches pageable host memory through the host
 * page tables, else through a pinned mirror of the arena).  Groups of different grids overlap on the
 * device; requests arriving meanwhile are admitted as memory frees up.
 * Plans (tables on the device) stay resident for the server's lifetime.
 */
int zm_server_create(zm_server_t* server, const zm_server_config_t* config);

/*
 * Queue one request.  `image` (host, row pitch in elements) and `out` (host
 * float[P(n_max)][2]) must stay valid until the request completes.  Returns a
 * ticket in *ticket.  ZM_EINVAL for bad arguments; ZM_ENOMEM if the request
 * alone exceeds the budget.  Geometry: the inscribed, centred disk.
 */
int zm_server_submit(zm_server_t server, const float* image, int height, int width, long long pitch,
                     int n_max, int n_rho, int n_theta, float* out, unsigned flags,
                     unsigned long long* ticket);

/* 1 in *done if the ticket's result is in its `out`, else 0. */
int zm_server_poll(zm_server_t server, unsigned long long ticket, int* done);

/* Wait for a ticket at most timeout_s seconds: ZM_OK or ZM_ETIMEOUT. */
int zm_server_wait(zm_server_t server, unsigned long long ticket, double timeout_s);

/* Wait (at most timeout_s) until every submitted request has completed. */
int zm_server_drain(zm_server_t server, double timeout_s);

int zm_server_stats(zm_server_t server, zm_server_stats_t* stats);

/* Zero every counter and latency sample (e.g. after warm-up requests that
 * built the plans).  Only on a drained server: ZM_EINVAL while requests are
 * in flight. */
int zm_server_reset_stats(zm_server_t server);

/* Stop the scheduler (after draining at most timeout_s) and free everything. */
int zm_server_destroy(zm_server_t server, double timeout_s);

/*
 * Diagnostic (no counterpart in the paper): one kernel waits, through the
 * bounded mbarrier wait every tensor-core and copy pipeline here uses, on a
 * barrier whose phase never completes; the wait gives up after its limit
 * (2 s) and the kernel writes ZM_ETIMEOUT to the device int *status and
 * returns, leaving the context usable.  Shows that a stalled pipeline ends in
 * a status, not a hang.  Asynchronous on `stream`.
 */
int zm_probe_bounded_wait(int* status, void* stream);

/* Number of kernels this library has launched in this process so far
 * (a diagnostic counter; never reset). */
unsigned long long zm_launch_count(void);

/* ---- reconstruction (Eq. 9) ------------------------------------------------ */

/*
 * Reconstruction on the polar nodes:
 *     f~(rho_i, theta_k) = Re sum_n sum_{m >= 0} c_m Z_nm R_nm(rho_i) e^{j m theta_k}
 * with c_m = 2/eps_m (c_0 = 1, c_m = 2), the literal Eq. 9 over m = -n..n,
 * when ZM_NEUMANN is set, and c_m = 1 (the sum over the stored m >= 0 only,
 * which over-weights m = 0) otherwise.  `moments` is device float[batch][P][2]
 * as written by zm_moments without ZM_NEUMANN; `out` is device
 * float[batch][N_rho][N_theta].
 */
int zm_reconstruct(zm_plan_t plan, const float* moments, int batch, float* out,
                   unsigned flags, void* stream);

/*
 * zm_reconstruct fused with zm_errors_polar: the polar reconstruction is
 * compared, inside the same kernel, with the polar samples `fhat` (device
 * float[batch][N_rho][N_theta], e.g. kept by zm_moments_ex) and err (device
 * double[batch][4]) receives eps_1 (Eq. 10), eps (Eq. 13), f_max and the node
 * count.  `out` receives the reconstruction, or may be NULL.
 */
int zm_reconstruct_errors(zm_plan_t plan, const float* moments, int batch, float* out,
                          const float* fhat, double* err, unsigned flags, void* stream);

/*
 * Reconstruction onto pixels: the polar reconstruction above, then bilinear
 * interpolation in (ring, angle) at every pixel centre of each canvas inside
 * its disk (ring bracket rho_i <= rho < rho_{i+1}, clamped to the first / last
 * ring; angle periodic); pixels outside the disk are set to 0.  `polar_tmp`
 * is a device float[batch][N_rho][N_theta] scratch the caller provides (it
 * holds the polar reconstruction afterwards).
 */
int zm_reconstruct_cartesian(zm_plan_t plan, const float* moments, int batch,
                             const zm_canvas_t* canvases, float* polar_tmp,
                             unsigned flags, void* stream);

/* ---- errors and normalisation (Eq. 10, Eq. 13, Table I) ------------------- */

/*
 * Per image, over the pixel centres inside the disk of `ref[b]`:
 *   out[b][0] = eps_1 = sum (f - f~)^2 / sum f^2                  (Eq. 10)
 *   out[b][1] = eps   = sum (f - f~)^2 / (f_max^2 * count)        (Eq. 13)
 *   out[b][2] = f_max over the disk, out[b][3] = count
 * `ref` and `test` are host arrays of device images of equal size; `out` is
 * device double[batch][4].
 */
int zm_errors(zm_plan_t plan, const zm_image_t* ref, const zm_image_t* test,
              int batch, double* out, void* stream);

/* As zm_errors over all polar nodes (plain sums over i, k): `fhat` and
 * `frec` are device float[batch][N_rho][N_theta]; count = N_rho N_theta. */
int zm_errors_polar(zm_plan_t plan, const float* fhat, const float* frec,
                    int batch, double* out, void* stream);

/* min and max of each image over the pixels inside its disk: `out` is device
 * float[batch][2] (min, max) - the per-band values Sec. 2.3 stores. */
int zm_disk_minmax(zm_plan_t plan, const zm_image_t* imgs, int batch,
                   float* out, void* stream);

/* Min-max normalisation in place (Sec. 3, Table I): every disk pixel of
 * canvas b is mapped linearly so that the canvas' own min / max over the disk
 * become target[b][0] / target[b][1] (device float[batch][2]); pixels outside
 * the disk are left unchanged. */
int zm_minmax_normalize(zm_plan_t plan, const zm_canvas_t* canvases, int batch,
                        const float* target, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ZM_H */
