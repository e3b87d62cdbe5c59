// Host frames -> device disk boxes (zm_upload_disk).
//
// Only the pixels a polar sample's bilinear stencil can touch are needed.  The
// device buffer holds the bounding box of the disk (X in [cx - r, cx + r], Y in
// [cy - r, cy + r], plus the stencil's right / lower neighbour and a pixel of
// margin), and of each box row only the span the disk covers is copied: a
// sample at height Y uses rows floor(Y) and floor(Y) + 1, so row y serves
// samples with Y in [y - 1, y + 1), whose |X - cx| is at most
// hw = sqrt(r^2 - d^2), d = max(0, |y - cy| - 1); the span is
// floor(cx - hw) - 3 .. floor(cx + hw) + 3 (three pixels of margin for the
// stencil's neighbour and float rounding of the sample positions).  Pixels of
// the box outside the spans are not written and no kernel reads them.  A
// kernel reads the spans from host memory the GPU can reach (pinned, or
// pageable where the device walks the host page tables).  At 4K (3840x2160,
// disk of diameter 2160) that is 14.8 MB of the frame's 33.2 MB (the box:
// 18.7 MB).
#include <algorithm>
#include <cmath>

#include "zm_internal.cuh"

namespace zm {

constexpr int UP_MAX_IMG = 64;

struct UpBox {
    const float* src;     // host row 0, column 0 of the box (device-usable address)
    long long spitch;     // host pitch (elements)
    int w, h;             // box size
    long long dst;        // offset of the box in the device buffer (floats)
    int dpitch;           // device pitch (elements, multiple of 4)
    int x0, y0;           // box origin in the image
    float cx, cy, r;      // disk in image coordinates
};

// Columns [*xs, *xe] (image coordinates, before clipping) that row y needs;
// false if none.  Double arithmetic with every operation correctly rounded
// and none contracted, on the host and the device alike, so that the host's
// byte count (zm_upload_disk_traffic) is what the kernel copies.
__host__ __device__ inline bool disk_row_span(int y, float cx, float cy, float r, int* xs, int* xe) {
    double d = (double)y - (double)cy;           // exact: both fit in 53 bits
    d = (d < 0 ? -d : d) - 1.0;                  // exact
    if (d < 0) d = 0;
#ifdef __CUDA_ARCH__
    const double h2 = __dsub_rn(__dmul_rn((double)r, (double)r), __dmul_rn(d, d));
    if (!(h2 > 0)) return false;
    const double hw = __dsqrt_rn(h2);
    *xs = (int)floor(__dsub_rn((double)cx, hw)) - 3;
    *xe = (int)floor(__dadd_rn((double)cx, hw)) + 3;
#else
    volatile double rr = (double)r * (double)r;
    volatile double dd = d * d;
    volatile double h2 = rr - dd;
    if (!(h2 > 0)) return false;
    volatile double hw = std::sqrt((double)h2);
    volatile double lo = (double)cx - hw, hi = (double)cx + hw;
    *xs = (int)std::floor((double)lo) - 3;
    *xe = (int)std::floor((double)hi) + 3;
#endif
    return true;
}

// The box-relative columns [*s, *e] copied of box row yb (*s a multiple of 4);
// false if none.
__host__ __device__ inline bool box_row_copy(int yb, int x0, int y0, int w, float cx, float cy, float r, int* s,
                                             int* e) {
    int xs, xe;
    if (!disk_row_span(y0 + yb, cx, cy, r, &xs, &xe)) return false;
    xs = xs - x0 < 0 ? 0 : xs - x0;
    xe = xe - x0 > w - 1 ? w - 1 : xe - x0;
    if (xs > xe) return false;
    *s = xs & ~3;
    *e = xe;
    return true;
}

struct UpParams {
    float* dev;
    int n;
    UpBox box[UP_MAX_IMG];
};

// blockIdx.y = box; each warp copies whole rows (row = warp index over the
// grid's warps, strided): lane 0 finds the row's span (the FP64 arithmetic of
// disk_row_span) and broadcasts it, and the warp copies it.  Eight rows per
// block are in flight at once, with no block barrier between rows; rows whose
// host start is 16-byte aligned (and pitch a multiple of 4) move as float4
// with four loads in flight per lane: the host link has a long latency, so
// many bytes must be in flight.  The rest of a row takes the scalar loop.
__global__ void __launch_bounds__(256) k_upload_boxes(const __grid_constant__ UpParams p) {
    const UpBox bx = p.box[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const bool vec = ((reinterpret_cast<uintptr_t>(bx.src) & 15u) == 0) && (bx.spitch & 3) == 0;
    for (int y = blockIdx.x * wpb + (threadIdx.x >> 5); y < bx.h; y += gridDim.x * wpb) {
        int x_s = 0, x_e = -1;
        if (lane == 0 && !box_row_copy(y, bx.x0, bx.y0, bx.w, bx.cx, bx.cy, bx.r, &x_s, &x_e)) x_e = -1;
        x_s = __shfl_sync(0xffffffffu, x_s, 0);
        x_e = __shfl_sync(0xffffffffu, x_e, 0);
        if (x_e < x_s) continue;
        const float* s = bx.src + (long long)y * bx.spitch + x_s;
        float* d = p.dev + bx.dst + (long long)y * bx.dpitch + x_s;
        const int n = x_e - x_s + 1;
        int done = 0;
        if (vec) {
            const int n4 = n >> 2;
            const float4* s4 = reinterpret_cast<const float4*>(s);
            float4* d4 = reinterpret_cast<float4*>(d);
            for (int x0 = lane; x0 < n4; x0 += 4 * 32) {
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int x = x0 + u * 32;
                    if (x < n4) v[u] = s4[x];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int x = x0 + u * 32;
                    if (x < n4) d4[x] = v[u];
                }
            }
            done = n4 << 2;
        }
        for (int x = done + lane; x < n; x += 32) d[x] = s[x];
    }
}

struct Box {
    int x0, y0, w, h, pitch;
};

// the box of image im (geometry resolved), clipped to the image
static Box disk_box(const zm_image_t& im) {
    const GeoImage g = resolve(im);
    // left edge rounded down to a multiple of 4 columns: box rows of a 16-byte
    // aligned frame then start 16-byte aligned (vector loads)
    const int x0 = std::max(0, (int)std::floor(g.cx - g.r) - 1) & ~3;
    const int y0 = std::max(0, (int)std::floor(g.cy - g.r) - 1);
    const int x1 = std::min(g.w - 1, (int)std::floor(g.cx + g.r) + 2);
    const int y1 = std::min(g.h - 1, (int)std::floor(g.cy + g.r) + 2);
    Box b;
    b.x0 = std::min(x0, g.w - 1);
    b.y0 = std::min(y0, g.h - 1);
    b.w = std::max(1, x1 - b.x0 + 1);
    b.h = std::max(1, y1 - b.y0 + 1);
    b.pitch = (b.w + 3) & ~3;
    return b;
}

// device-usable address of a host buffer, or NULL if the device cannot read it
static const float* device_view(const float* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer ? static_cast<const float*>(a.devicePointer) : p;
    int pageable = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
    return pageable ? p : nullptr;
}

}  // namespace zm

using namespace zm;

extern "C" int zm_upload_disk_traffic(const zm_image_t* host_imgs, int batch, unsigned long long* bytes) {
    if (!bytes) return set_error(ZM_EINVAL, "bytes is NULL");
    int s = check_images(host_imgs, batch);
    if (s != ZM_OK) return s;
    unsigned long long t = 0;
    for (int b = 0; b < batch; ++b) {
        const Box bx = disk_box(host_imgs[b]);
        const GeoImage g = resolve(host_imgs[b]);
        for (int y = 0; y < bx.h; ++y) {
            int s0, e0;
            if (box_row_copy(y, bx.x0, bx.y0, bx.w, g.cx, g.cy, g.r, &s0, &e0))
                t += sizeof(float) * (unsigned long long)(e0 - s0 + 1);
        }
    }
    *bytes = t;
    return ZM_OK;
}

extern "C" int zm_upload_disk_bytes(const zm_image_t* host_imgs, int batch, unsigned long long* bytes) {
    if (!bytes) return set_error(ZM_EINVAL, "bytes is NULL");
    int s = check_images(host_imgs, batch);
    if (s != ZM_OK) return s;
    unsigned long long t = 0;
    for (int b = 0; b < batch; ++b) {
        const Box bx = disk_box(host_imgs[b]);
        t += sizeof(float) * (unsigned long long)bx.pitch * bx.h;
    }
    *bytes = t;
    return ZM_OK;
}

extern "C" int zm_upload_disk(const zm_image_t* host_imgs, int batch, float* dev, unsigned long long dev_bytes,
                              zm_image_t* dev_imgs, void* stream) {
    if (!dev || !dev_imgs) return set_error(ZM_EINVAL, "NULL argument");
    if ((reinterpret_cast<uintptr_t>(dev) & 15u) != 0) return set_error(ZM_EINVAL, "dev must be 16-byte aligned");
    int s = check_images(host_imgs, batch);
    if (s != ZM_OK) return s;
    int device = 0;
    ZM_CUDA_TRY(cudaGetDevice(&device));
    static thread_local UpParams up;
    up.dev = dev;
    long long off = 0;
    for (int c0 = 0; c0 < batch; c0 += UP_MAX_IMG) {
        const int nc = std::min(UP_MAX_IMG, batch - c0);
        int max_h = 1;
        for (int j = 0; j < nc; ++j) {
            const zm_image_t& im = host_imgs[c0 + j];
            const float* view = device_view(im.data, device);
            if (!view)
                return set_error(ZM_EUNSUPPORTED, "image %d: host memory the device cannot read (pin it or register it)",
                                 c0 + j);
            const Box bx = disk_box(im);
            if ((unsigned long long)(off + (long long)bx.pitch * bx.h) * sizeof(float) > dev_bytes)
                return set_error(ZM_EINVAL, "dev holds %llu bytes; the boxes need more (zm_upload_disk_bytes)",
                                 dev_bytes);
            UpBox& u = up.box[j];
            u.src = view + (long long)bx.y0 * im.pitch + bx.x0;
            u.spitch = im.pitch;
            u.w = bx.w;
            u.h = bx.h;
            u.dst = off;
            u.dpitch = bx.pitch;
            const GeoImage g = resolve(im);
            u.x0 = bx.x0;
            u.y0 = bx.y0;
            u.cx = g.cx;
            u.cy = g.cy;
            u.r = g.r;
            dev_imgs[c0 + j] = zm_image_t{dev + off, bx.h, bx.w, bx.pitch, g.cx - (float)bx.x0, g.cy - (float)bx.y0, g.r};
            off += (long long)bx.pitch * bx.h;
            max_h = std::max(max_h, bx.h);
        }
        up.n = nc;
        // about two blocks (16 rows in flight) per SM in all: many more bytes in
        // flight than the host link's latency needs, while SMs stay free for
        // kernels that run beside the upload on other streams
        const int per = std::max(4, 2 * num_sms(device) / nc);
        k_upload_boxes<<<dim3(std::min((max_h + 7) / 8, per), nc), 256, 0, (cudaStream_t)stream>>>(up);
        ZM_LAUNCH_CHECK("k_upload_boxes");
    }
    return ZM_OK;
}
