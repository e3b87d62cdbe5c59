"""ctypes binding of libzm.so (include/zm.h): the same entry points under the
same names, doing argument marshalling only.

Device buffers are passed as CUDA tensors (their data_ptr) or raw integer
addresses; streams as torch.cuda.Stream, raw cudaStream_t integers or None
(torch's current stream).  A failing call raises ZmError with the library's
status and detail text.  Importing this module does not load the library;
``lib()`` does and raises if ``libzm.so`` has not been built.
"""

import ctypes
import os

from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_longlong, c_uint, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libzm.so")

ZM_OK, ZM_EINVAL, ZM_ENOMEM, ZM_ECUDA, ZM_ETIMEOUT, ZM_EUNSUPPORTED = range(6)
ZM_GRID_MIDPOINT = 0x0
ZM_GRID_GAUSS = 0x1
ZM_PREC_FP32 = 0x00
ZM_PREC_BF16X3 = 0x10
ZM_PREC_FP16X3 = 0x20
ZM_NEUMANN = 0x1


class ZmError(RuntimeError):
    def __init__(self, status, detail):
        super().__init__("zm status %d (%s): %s" % (status, _STATUS.get(status, "?"), detail))
        self.status = status


_STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "timed out",
           5: "unsupported"}


class zm_image_t(ctypes.Structure):
    _fields_ = [("data", c_void_p), ("height", c_int), ("width", c_int), ("pitch", c_longlong),
                ("cx", c_float), ("cy", c_float), ("radius", c_float)]


class zm_canvas_t(ctypes.Structure):
    _fields_ = [("data", c_void_p), ("height", c_int), ("width", c_int), ("pitch", c_longlong),
                ("cx", c_float), ("cy", c_float), ("radius", c_float)]


class zm_request_t(ctypes.Structure):
    _fields_ = [("image", zm_image_t), ("n_max", c_int), ("n_rho", c_int), ("n_theta", c_int), ("out", c_void_p)]


class zm_server_config_t(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_ulonglong), ("streams", c_int), ("max_group", c_int), ("plan_flags", c_uint),
                ("max_wait_us", c_int)]


class zm_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("completed", ctypes.c_ulonglong),
                ("rejected", ctypes.c_ulonglong), ("groups_launched", ctypes.c_ulonglong),
                ("p50_ms", c_double), ("p99_ms", c_double), ("max_ms", c_double),
                ("images_per_s", c_double), ("peak_bytes", ctypes.c_ulonglong), ("host_direct", c_int)]


# name -> (restype, argtypes); mirrors include/zm.h
SIGNATURES = {
    "zm_num_moments": (c_int, [c_int]),
    "zm_index": (c_int, [c_int, c_int]),
    "zm_strerror": (c_char_p, [c_int]),
    "zm_last_error": (c_char_p, []),
    "zm_plan": (c_int, [POINTER(c_void_p), c_int, c_int, c_int, c_uint]),
    "zm_plan_destroy": (c_int, [c_void_p]),
    "zm_plan_reserve": (c_int, [c_void_p, c_int]),
    "zm_plan_status": (c_int, [c_void_p]),
    "zm_plan_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                             POINTER(c_uint)]),
    "zm_plan_table": (c_int, [c_void_p, c_void_p, c_void_p]),
    "zm_plan_nodes": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "zm_moments": (c_int, [c_void_p, POINTER(zm_image_t), c_int, c_void_p, c_uint, c_void_p]),
    "zm_moments_ex": (c_int, [c_void_p, POINTER(zm_image_t), c_int, c_void_p, c_void_p, c_uint, c_void_p]),
    "zm_moments_polar": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_uint, c_void_p]),
    "zm_upload_disk_bytes": (c_int, [c_void_p, c_int, POINTER(ctypes.c_ulonglong)]),
    "zm_upload_disk_traffic": (c_int, [c_void_p, c_int, POINTER(ctypes.c_ulonglong)]),
    "zm_cartesian_work_bytes": (c_int, [c_int, c_int, POINTER(ctypes.c_ulonglong)]),
    "zm_cartesian_moments": (c_int, [POINTER(zm_image_t), c_int, POINTER(c_int), c_int, c_void_p, c_void_p,
                                     ctypes.c_ulonglong, c_uint, c_void_p]),
    "zm_upload_disk": (c_int, [c_void_p, c_int, c_void_p, ctypes.c_ulonglong, c_void_p, c_void_p]),
    "zm_resample": (c_int, [c_void_p, POINTER(zm_image_t), c_int, c_void_p, c_void_p]),
    "zm_ring_spectra": (c_int, [c_void_p, POINTER(zm_image_t), c_int, c_void_p, c_void_p, c_void_p]),
    "zm_project": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_uint, c_void_p]),
    "zm_project_noalloc": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_uint, c_void_p]),
    "zm_stage_spectra": (c_int, [c_void_p, POINTER(zm_image_t), c_int, c_void_p]),
    "zm_stage_project": (c_int, [c_void_p, c_int, c_void_p, c_uint, c_void_p]),
    "zm_batch_create": (c_int, [POINTER(c_void_p), POINTER(zm_request_t), c_int, c_uint]),
    "zm_batch_run": (c_int, [c_void_p, POINTER(zm_request_t), c_uint, c_void_p]),
    "zm_batch_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int)]),
    "zm_batch_destroy": (c_int, [c_void_p]),
    "zm_server_create": (c_int, [POINTER(c_void_p), POINTER(zm_server_config_t)]),
    "zm_server_submit": (c_int, [c_void_p, c_void_p, c_int, c_int, c_longlong, c_int, c_int, c_int, c_void_p, c_uint,
                                 POINTER(ctypes.c_ulonglong)]),
    "zm_server_poll": (c_int, [c_void_p, ctypes.c_ulonglong, POINTER(c_int)]),
    "zm_server_wait": (c_int, [c_void_p, ctypes.c_ulonglong, c_double]),
    "zm_server_drain": (c_int, [c_void_p, c_double]),
    "zm_server_stats": (c_int, [c_void_p, POINTER(zm_server_stats_t)]),
    "zm_server_reset_stats": (c_int, [c_void_p]),
    "zm_server_destroy": (c_int, [c_void_p, c_double]),
    "zm_probe_bounded_wait": (c_int, [c_void_p, c_void_p]),
    "zm_launch_count": (ctypes.c_ulonglong, []),
    "zm_reconstruct": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_uint, c_void_p]),
    "zm_reconstruct_errors": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_uint, c_void_p]),
    "zm_reconstruct_cartesian": (c_int, [c_void_p, c_void_p, c_int, POINTER(zm_canvas_t), c_void_p, c_uint,
                                         c_void_p]),
    "zm_errors": (c_int, [c_void_p, POINTER(zm_image_t), POINTER(zm_image_t), c_int, c_void_p, c_void_p]),
    "zm_errors_polar": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "zm_disk_minmax": (c_int, [c_void_p, POINTER(zm_image_t), c_int, c_void_p, c_void_p]),
    "zm_minmax_normalize": (c_int, [c_void_p, POINTER(zm_canvas_t), c_int, c_void_p, c_void_p]),
}

_lib = None


def lib():
    """Load libzm.so once; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libzm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != ZM_OK:
        raise ZmError(status, lib().zm_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError("cannot take a device pointer of %r" % type(x))


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _geometry(g):
    if g is None:
        return 0.0, 0.0, -1.0
    return float(g[0]), float(g[1]), float(g[2])


def image_desc(t, geometry=None):
    """zm_image_t for a 2-D float32 CUDA tensor (rows may be strided)."""
    if t.dim() != 2 or t.dtype.__str__() != "torch.float32" or not t.is_cuda or t.stride(1) != 1:
        raise ValueError("images must be 2-D float32 CUDA tensors with unit column stride")
    cx, cy, r = _geometry(geometry)
    return zm_image_t(t.data_ptr(), t.shape[0], t.shape[1], t.stride(0), cx, cy, r)


def host_image_desc(t, geometry=None):
    """zm_image_t for a 2-D float32 host image: a CPU tensor (pinned or not) or a
    numpy array, rows may be strided, unit column stride."""
    cx, cy, r = _geometry(geometry)
    if hasattr(t, "data_ptr"):
        if t.dim() != 2 or str(t.dtype) != "torch.float32" or t.is_cuda or t.stride(1) != 1:
            raise ValueError("host images must be 2-D float32 CPU tensors with unit column stride")
        return zm_image_t(t.data_ptr(), t.shape[0], t.shape[1], t.stride(0), cx, cy, r)
    if t.ndim != 2 or t.dtype.name != "float32" or t.strides[1] != 4:
        raise ValueError("host images must be 2-D float32 arrays with unit column stride")
    return zm_image_t(t.ctypes.data, t.shape[0], t.shape[1], t.strides[0] // 4, cx, cy, r)


def canvas_desc(t, geometry=None):
    d = image_desc(t, geometry)
    return zm_canvas_t(d.data, d.height, d.width, d.pitch, d.cx, d.cy, d.radius)


def image_array(images, geometries=None):
    """The zm_image_t array of a list of 2-D float32 CUDA tensors, to be built
    once and passed to the image entry points in place of the list."""
    return _images(images, geometries)[0]


def _images(imgs, geometries=None):
    if isinstance(imgs, ctypes.Array):                 # descriptors built already (e.g. zm_upload_disk)
        return imgs, len(imgs)
    imgs = list(imgs)
    geos = list(geometries) if geometries is not None else [None] * len(imgs)
    arr = (zm_image_t * len(imgs))(*[image_desc(t, g) for t, g in zip(imgs, geos)])
    return arr, len(imgs)


def canvas_array(canvases, geometries=None):
    """The zm_canvas_t array of a list of 2-D float32 CUDA tensors, to be built
    once and passed to the canvas entry points in place of the list."""
    return _canvases(canvases, geometries)[0]


def _canvases(cvs, geometries=None):
    if isinstance(cvs, ctypes.Array):
        return cvs, len(cvs)
    cvs = list(cvs)
    geos = list(geometries) if geometries is not None else [None] * len(cvs)
    arr = (zm_canvas_t * len(cvs))(*[canvas_desc(t, g) for t, g in zip(cvs, geos)])
    return arr, len(cvs)


# ------------------------------------------------------------------ entry points
def zm_num_moments(n_max):
    return lib().zm_num_moments(n_max)


def zm_index(n, m):
    return lib().zm_index(n, m)


def zm_strerror(status):
    return lib().zm_strerror(status).decode()


def zm_last_error():
    return lib().zm_last_error().decode()


def zm_plan(n_max, n_rho, n_theta, flags=0):
    h = c_void_p()
    _check(lib().zm_plan(ctypes.byref(h), n_max, n_rho, n_theta, flags))
    return h.value


def zm_plan_destroy(plan):
    _check(lib().zm_plan_destroy(plan))


def zm_plan_reserve(plan, batch):
    _check(lib().zm_plan_reserve(plan, batch))


def zm_plan_status(plan):
    _check(lib().zm_plan_status(plan))


def zm_plan_info(plan):
    a, b, c, d, f = c_int(), c_int(), c_int(), c_int(), c_uint()
    _check(lib().zm_plan_info(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                              ctypes.byref(f)))
    return {"n_max": a.value, "n_rho": b.value, "n_theta": c.value, "num_moments": d.value, "flags": f.value}


def zm_plan_table(plan, dst, stream=None):
    _check(lib().zm_plan_table(plan, _ptr(dst), _stream(stream)))


def zm_plan_nodes(plan, rho=None, wr=None, stream=None):
    _check(lib().zm_plan_nodes(plan, _ptr(rho), _ptr(wr), _stream(stream)))


def zm_moments(plan, images, out, flags=0, stream=None, geometries=None):
    arr, n = _images(images, geometries)
    _check(lib().zm_moments(plan, arr, n, _ptr(out), flags, _stream(stream)))


def zm_moments_ex(plan, images, out, fhat=None, flags=0, stream=None, geometries=None):
    arr, n = _images(images, geometries)
    _check(lib().zm_moments_ex(plan, arr, n, _ptr(out), _ptr(fhat), flags, _stream(stream)))


def zm_moments_polar(plan, fhat, batch, out, flags=0, stream=None):
    _check(lib().zm_moments_polar(plan, _ptr(fhat), batch, _ptr(out), flags, _stream(stream)))


def _host_images(imgs, geometries=None):
    imgs = list(imgs)
    geos = list(geometries) if geometries is not None else [None] * len(imgs)
    return (zm_image_t * len(imgs))(*[host_image_desc(t, g) for t, g in zip(imgs, geos)]), len(imgs)


def zm_upload_disk_bytes(host_images, geometries=None):
    arr, n = _host_images(host_images, geometries)
    b = ctypes.c_ulonglong()
    _check(lib().zm_upload_disk_bytes(arr, n, ctypes.byref(b)))
    return b.value


def zm_cartesian_work_bytes(batch, count):
    b = ctypes.c_ulonglong()
    _check(lib().zm_cartesian_work_bytes(batch, count, ctypes.byref(b)))
    return b.value


def zm_cartesian_moments(images, pairs, out, work, flags=0, stream=None, geometries=None):
    """Moments (n, m) in `pairs` by Cartesian summation (Eq. 6) into the device
    tensor out[batch][len(pairs)][2]; `work` a device tensor of at least
    zm_cartesian_work_bytes(batch, len(pairs)) bytes."""
    arr, n = _images(images, geometries)
    pairs = list(pairs)
    nm = (c_int * (2 * len(pairs)))(*[v for pr in pairs for v in pr])
    nbytes = work.numel() * work.element_size()
    _check(lib().zm_cartesian_moments(arr, n, nm, len(pairs), _ptr(out), _ptr(work), nbytes, flags,
                                      _stream(stream)))


def zm_upload_disk_traffic(host_images, geometries=None):
    """Bytes zm_upload_disk reads from the host for these images."""
    arr, n = _host_images(host_images, geometries)
    b = ctypes.c_ulonglong()
    _check(lib().zm_upload_disk_traffic(arr, n, ctypes.byref(b)))
    return b.value


def zm_upload_disk(host_images, dev, stream=None, geometries=None):
    """Copy the disk boxes of host images (pinned tensors / arrays the device can
    read) into the device tensor `dev`; returns the zm_image_t array of the boxes,
    to pass as `images` to zm_moments* (reuse it while the buffers stay put)."""
    arr, n = _host_images(host_images, geometries)
    out = (zm_image_t * n)()
    _check(lib().zm_upload_disk(arr, n, _ptr(dev), dev.numel() * dev.element_size(), out, _stream(stream)))
    return out


def zm_probe_bounded_wait(status, stream=None):
    _check(lib().zm_probe_bounded_wait(_ptr(status), _stream(stream)))


def zm_resample(plan, images, fhat, stream=None, geometries=None):
    arr, n = _images(images, geometries)
    _check(lib().zm_resample(plan, arr, n, _ptr(fhat), _stream(stream)))


def zm_ring_spectra(plan, images, spectra, fhat=None, stream=None, geometries=None):
    arr, n = _images(images, geometries)
    _check(lib().zm_ring_spectra(plan, arr, n, _ptr(spectra), _ptr(fhat), _stream(stream)))


def zm_project(plan, spectra, batch, out, flags=0, stream=None):
    _check(lib().zm_project(plan, _ptr(spectra), batch, _ptr(out), flags, _stream(stream)))


def zm_stage_spectra(plan, images, stream=None, geometries=None):
    arr, n = _images(images, geometries)
    _check(lib().zm_stage_spectra(plan, arr, n, _stream(stream)))


def zm_stage_project(plan, batch, out, flags=0, stream=None):
    _check(lib().zm_stage_project(plan, batch, _ptr(out), flags, _stream(stream)))


def zm_project_noalloc(plan, spectra, batch, out, flags=0, stream=None):
    _check(lib().zm_project_noalloc(plan, _ptr(spectra), batch, _ptr(out), flags, _stream(stream)))


def requests(items):
    """zm_request_t array from (image tensor, n_max, n_rho, n_theta, out tensor[, geometry]) tuples."""
    items = list(items)
    arr = (zm_request_t * len(items))()
    for j, it in enumerate(items):
        img, n_max, n_rho, n_theta, out = it[:5]
        geo = it[5] if len(it) > 5 else None
        arr[j] = zm_request_t(image_desc(img, geo), n_max, n_rho, n_theta, _ptr(out))
    return arr


def zm_batch_create(reqs, plan_flags=0):
    arr = reqs if isinstance(reqs, ctypes.Array) else requests(reqs)
    h = c_void_p()
    _check(lib().zm_batch_create(ctypes.byref(h), arr, len(arr), plan_flags))
    return h.value


def zm_batch_run(batch, reqs, flags=0, stream=None):
    arr = reqs if isinstance(reqs, ctypes.Array) else requests(reqs)
    _check(lib().zm_batch_run(batch, arr, flags, _stream(stream)))


def zm_batch_info(batch):
    g, c = c_int(), c_int()
    _check(lib().zm_batch_info(batch, ctypes.byref(g), ctypes.byref(c)))
    return {"groups": g.value, "captures": c.value}


def zm_batch_destroy(batch):
    _check(lib().zm_batch_destroy(batch))


def zm_server_create(hbm_budget=0, streams=0, max_group=0, plan_flags=0, max_wait_us=0):
    cfg = zm_server_config_t(hbm_budget, streams, max_group, plan_flags, max_wait_us)
    h = c_void_p()
    _check(lib().zm_server_create(ctypes.byref(h), ctypes.byref(cfg)))
    return h.value


def zm_server_submit(server, image, n_max, n_rho, n_theta, out, flags=0):
    """image: C-contiguous float32 numpy array (host); out: float32 numpy array of
    shape [P(n_max), 2].  Both must stay alive until the ticket completes."""
    import numpy as np
    if image.dtype != np.float32 or image.ndim != 2 or not image.flags.c_contiguous:
        raise ValueError("image must be a C-contiguous 2-D float32 array")
    if out.dtype != np.float32 or not out.flags.c_contiguous or out.size < 2 * zm_num_moments(n_max):
        raise ValueError("out must be a C-contiguous float32 array of P(n_max) x 2")
    t = ctypes.c_ulonglong()
    _check(lib().zm_server_submit(server, image.ctypes.data, image.shape[0], image.shape[1], image.shape[1],
                                  n_max, n_rho, n_theta, out.ctypes.data, flags, ctypes.byref(t)))
    return t.value


def zm_server_poll(server, ticket):
    d = c_int()
    _check(lib().zm_server_poll(server, ticket, ctypes.byref(d)))
    return bool(d.value)


def zm_server_wait(server, ticket, timeout_s=10.0):
    _check(lib().zm_server_wait(server, ticket, timeout_s))


def zm_server_drain(server, timeout_s=60.0):
    _check(lib().zm_server_drain(server, timeout_s))


def zm_server_stats(server):
    st = zm_server_stats_t()
    _check(lib().zm_server_stats(server, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in zm_server_stats_t._fields_}


def zm_server_reset_stats(server):
    _check(lib().zm_server_reset_stats(server))


def zm_server_destroy(server, timeout_s=60.0):
    _check(lib().zm_server_destroy(server, timeout_s))


def zm_launch_count():
    return int(lib().zm_launch_count())


def zm_reconstruct(plan, moments, batch, out, flags=0, stream=None):
    _check(lib().zm_reconstruct(plan, _ptr(moments), batch, _ptr(out), flags, _stream(stream)))


def zm_reconstruct_errors(plan, moments, batch, out, fhat, err, flags=0, stream=None):
    _check(lib().zm_reconstruct_errors(plan, _ptr(moments), batch, _ptr(out), _ptr(fhat), _ptr(err), flags,
                                       _stream(stream)))


def zm_reconstruct_cartesian(plan, moments, canvases, polar_tmp, flags=0, stream=None, geometries=None):
    arr, n = _canvases(canvases, geometries)
    _check(lib().zm_reconstruct_cartesian(plan, _ptr(moments), n, arr, _ptr(polar_tmp), flags, _stream(stream)))


def zm_errors(plan, ref, test, out, stream=None, geometries=None):
    ra, n = _images(ref, geometries)
    ta, n2 = _images(test, geometries)
    if n != n2:
        raise ValueError("reference and test batches differ")
    _check(lib().zm_errors(plan, ra, ta, n, _ptr(out), _stream(stream)))


def zm_errors_polar(plan, fhat, frec, batch, out, stream=None):
    _check(lib().zm_errors_polar(plan, _ptr(fhat), _ptr(frec), batch, _ptr(out), _stream(stream)))


def zm_disk_minmax(plan, images, out, stream=None, geometries=None):
    arr, n = _images(images, geometries)
    _check(lib().zm_disk_minmax(plan, arr, n, _ptr(out), _stream(stream)))


def zm_minmax_normalize(plan, canvases, target, stream=None, geometries=None):
    arr, n = _canvases(canvases, geometries)
    _check(lib().zm_minmax_normalize(plan, arr, n, _ptr(target), _stream(stream)))
