"""GB300-native branchless generalized Joseph projector (GJP).

Thin PyTorch-facing layer over the C ABI of ``libgjp.so`` (``include/gjp.h``):
torch supplies device memory and the current CUDA stream; every step of the
projection runs in the library's CUDA kernels.  There is no CPU fallback --
calls raise if the library is missing or a tensor is not on a CUDA device.

    geom = Geometry(src, det_origin, det_u, det_v, nu, nv)   # float64 (n_views, 3)
    proj = forward(volume, geom, voxel_size=(1, 1, 1))         # (n_views, nv, nu) float32
    back = adjoint(proj, geom, volume.shape, voxel_size=(1, 1, 1))
"""
from __future__ import annotations

import numpy as np

from . import _capi, tuning_cache
from ._capi import GjpError

__all__ = ["Geometry", "Batch", "forward", "adjoint", "footprint_voxels", "stream_status", "trim_workspace", "GjpError",
           "library_path"]


def library_path() -> str:
    return _capi.LIB_PATH


class Geometry:
    """Owns a ``gjp_geometry`` handle (host copy of the per-view source and
    detector frames; device tables are built on first use per device)."""

    def __init__(self, src, det_origin, det_u, det_v, nu: int, nv: int, weight: str = "lin"):
        src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
        self.n_views = int(src.shape[0])
        self.nu, self.nv = int(nu), int(nv)
        st, h = _capi.gjp_geometry_create(self.n_views, self.nu, self.nv, src, det_origin, det_u, det_v)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_geometry_create")
        self.handle = h
        self.digest = tuning_cache.geometry_digest(src, det_origin, det_u, det_v, self.nu, self.nv)
        self.weight = "lin"
        self.fov = 0.0
        if weight != "lin":
            self.set_weight(weight)

    @classmethod
    def from_cone(cls, cg, weight: str = "lin") -> "Geometry":
        """From any object with ``src, det_origin, det_u, det_v, nu, nv``."""
        return cls(cg.src, cg.det_origin, cg.det_u, cg.det_v, cg.nu, cg.nv, weight=weight)

    def set_weight(self, weight: str):
        """Interpolation weight: "lin" (w_lin, Eq. 13) or "spl" (w_spl, Eq. 14)."""
        code = {"lin": _capi.GJP_WEIGHT_LIN, "spl": _capi.GJP_WEIGHT_SPL}[weight]
        st = _capi.gjp_geometry_set_weight(self.handle, code)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_geometry_set_weight")
        self.weight = weight

    def set_launch(self, tile_u: int = 4, view_group: int = 16):
        """Launch shape of the one-thread-per-ray kernels: ``tile_u`` detector
        columns per block (1, 2, 4 or 8) and ``view_group`` views issued tile
        by tile together.  Changes speed only, never a result."""
        st = _capi.gjp_geometry_set_launch(self.handle, tile_u, view_group)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_geometry_set_launch")

    def set_fov(self, radius: float):
        """Clip every ray to the cylinder of world ``radius`` around the axis
        through the volume centre parallel to z (0 turns it off)."""
        st = _capi.gjp_geometry_set_fov(self.handle, radius)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_geometry_set_fov")
        self.fov = float(radius)

    @property
    def launch(self):
        st, tu, vg = _capi.gjp_geometry_get_launch(self.handle)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_geometry_get_launch")
        return tu, vg

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            _capi.gjp_geometry_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def proj_shape(self):
        return (self.n_views, self.nv, self.nu)


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    m = {torch.float32: _capi.GJP_F32, torch.bfloat16: _capi.GJP_BF16, torch.float16: _capi.GJP_F16}
    if t.dtype not in m:
        raise TypeError(f"volume dtype {t.dtype} is not float32/bfloat16/float16")
    return m[t.dtype]


def _check_cuda(t, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the projector has no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be C-contiguous")


def _stream(t, stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(t.device)
    return int(stream.cuda_stream)


_PATHS = {"auto": 0, "gather": 1, "slab": 2, "prefetch": 3, "combine": 4, "texture": 5, "hwlin": 6,
          "pairs": 7}


def forward(volume, geometry: Geometry, voxel_size=(1.0, 1.0, 1.0), origin=None, out=None, stream=None,
            path: str = "auto"):
    """GJP forward projection (Algorithm 1) of a ``(nx, ny, nz)`` CUDA
    volume (float32, bfloat16 or float16 storage) into ``(n_views, nv, nu)``
    float32 projections.  ``path`` selects the kernel family ("auto",
    "gather", "pairs", "slab", "prefetch", "texture" or "hwlin"; see
    ``gjp_forward_ex``)."""
    torch = _torch()
    _check_cuda(volume, "volume")
    if volume.dim() != 3:
        raise ValueError("volume must be 3-D (nx, ny, nz)")
    if out is None:
        out = torch.empty(geometry.proj_shape, dtype=torch.float32, device=volume.device)
    _check_cuda(out, "out")
    if out.dtype != torch.float32 or tuple(out.shape) != geometry.proj_shape or out.device != volume.device:
        raise ValueError("out must be float32 (n_views, nv, nu) on the volume's device")
    with torch.cuda.device(volume.device):
        st = _capi.gjp_forward_ex(volume.data_ptr(), _dtype_code(volume), *volume.shape, voxel_size, origin,
                                  geometry.handle, out.data_ptr(), _PATHS[path], _stream(volume, stream))
    if st != _capi.GJP_OK:
        raise GjpError(st, "gjp_forward")
    return out


def adjoint(proj, geometry: Geometry, shape, voxel_size=(1.0, 1.0, 1.0), origin=None, out=None,
            accumulate: bool = False, stream=None, path: str = "auto"):
    """Matched transpose of :func:`forward`: ``A^T proj`` as a float32
    ``shape`` volume (added into ``out`` when ``accumulate``).  ``path`` is
    "auto", "gather" (global atomics) or "slab" (shared-memory boxes with
    TMA bulk reduction)."""
    torch = _torch()
    _check_cuda(proj, "proj")
    if proj.dtype != torch.float32 or tuple(proj.shape) != geometry.proj_shape:
        raise ValueError("proj must be float32 (n_views, nv, nu)")
    shape = tuple(int(s) for s in shape)
    if out is None:
        out = (torch.zeros if accumulate else torch.empty)(shape, dtype=torch.float32, device=proj.device)
    _check_cuda(out, "out")
    if out.dtype != torch.float32 or tuple(out.shape) != shape or out.device != proj.device:
        raise ValueError("out must be a float32 volume of the given shape on proj's device")
    with torch.cuda.device(proj.device):
        st = _capi.gjp_adjoint_ex(proj.data_ptr(), geometry.handle, *shape, voxel_size, origin, out.data_ptr(),
                                  1 if accumulate else 0, _PATHS[path], _stream(proj, stream))
    if st != _capi.GJP_OK:
        raise GjpError(st, "gjp_adjoint")
    return out


def footprint_voxels(geometry: Geometry, shape, voxel_size=(1.0, 1.0, 1.0), origin=None, views=None,
                     device=None):
    """Per view, the number of distinct voxels that receive a non-zero
    interpolation weight (the view's compulsory volume traffic in voxels).
    Measurement helper for roofline accounting."""
    torch = _torch()
    device = torch.device("cuda") if device is None else torch.device(device)
    shape = tuple(int(s) for s in shape)
    marks = torch.empty(shape, dtype=torch.uint8, device=device)
    views = range(geometry.n_views) if views is None else views
    counts = []
    with torch.cuda.device(device):
        for v in views:
            marks.zero_()
            st = _capi.gjp_footprint(geometry.handle, int(v), *shape, voxel_size, origin, marks.data_ptr(),
                                     _stream(marks, None))
            if st != _capi.GJP_OK:
                raise GjpError(st, "gjp_footprint")
            counts.append(torch.count_nonzero(marks))
    return [int(c.item()) for c in counts]


def trim_workspace():
    """Returns to the device the memory the library keeps between calls for
    the z-paired copies of the "pairs" forward (``gjp_trim_workspace``)."""
    st = _capi.gjp_trim_workspace()
    if st != _capi.GJP_OK:
        raise GjpError(st, "gjp_trim_workspace")


def stream_status(stream=None):
    """Synchronise the stream and raise if a kernel of the library gave up a
    bounded wait since the last check (its output is then invalid)."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    st = _capi.gjp_stream_status(int(stream.cuda_stream))
    if st != _capi.GJP_OK:
        raise GjpError(st, "gjp_stream_status")


class Batch:
    """Many independent forward projections in one persistent launch
    (``gjp_batch_*``).  ``problems`` is a sequence of
    ``(volume, geometry, voxel_size, origin, out)`` with CUDA tensors on one
    device; the tensors and geometries are kept alive by the batch and must
    not be reallocated while it is used (their contents may change between
    launches).  ``forward()`` launches on the current stream and can be
    captured into a CUDA graph."""

    def __init__(self, problems):
        torch = _torch()
        self._keep = []
        self._sigs = []
        recs = []
        self.device = None
        for vol, geom, h, origin, out in problems:
            _check_cuda(vol, "volume")
            _check_cuda(out, "out")
            if vol.dim() != 3:
                raise ValueError("volume must be 3-D (nx, ny, nz)")
            if out.dtype != torch.float32 or tuple(out.shape) != geom.proj_shape or out.device != vol.device:
                raise ValueError("out must be float32 (n_views, nv, nu) on the volume's device")
            if self.device is None:
                self.device = vol.device
            elif vol.device != self.device:
                raise ValueError("all problems of a batch live on one device")
            r = _capi.GjpProblem()
            r.d_volume = vol.data_ptr()
            r.dtype = _dtype_code(vol)
            r.nx, r.ny, r.nz = (int(v) for v in vol.shape)
            r.voxel_size[:] = [float(v) for v in h]
            if origin is not None:
                r.volume_origin[:] = [float(v) for v in origin]
                r.has_origin = 1
            r.geometry = geom.handle
            r.d_proj = out.data_ptr()
            recs.append(r)
            self._keep.append((vol, geom, out))
            self._sigs.append(tuning_cache.problem_signature(str(vol.dtype).replace("torch.", ""), vol.shape, h,
                                                             origin, geom.digest, geom.weight,
                                                             getattr(geom, "fov", 0.0)))
        self.handle = None
        with torch.cuda.device(self.device):
            st, h = _capi.gjp_batch_create(recs)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_batch_create")
        self.handle = h
        self.outputs = [k[2] for k in self._keep]

    def forward(self, stream=None):
        torch = _torch()
        with torch.cuda.device(self.device):
            s = torch.cuda.current_stream(self.device) if stream is None else stream
            st = _capi.gjp_batch_forward(self.handle, int(s.cuda_stream))
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_batch_forward")
        return self.outputs

    def autotune(self, reps: int = 2, stream=None, cache: str | None = None):
        """Launch-shape search (``gjp_batch_autotune``).  With ``cache`` (a
        JSON file path), shapes found before for the same GPU model and the
        same problems are read from it instead of timed again, and new ones
        are added to it.  Returns the ``(tile_u, view_group)`` per problem."""
        torch = _torch()
        gpu = torch.cuda.get_device_name(self.device)
        key = tuning_cache.batch_key(gpu, self._sigs) if cache else None
        if cache:
            hit = tuning_cache.lookup(cache, key, len(self._keep))
            if hit is not None:
                for i, (t, v) in enumerate(hit):
                    self.set_tuning(i, t, v)
                return hit
        with torch.cuda.device(self.device):
            s = torch.cuda.current_stream(self.device) if stream is None else stream
            st = _capi.gjp_batch_autotune(self.handle, int(s.cuda_stream), reps)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_batch_autotune")
        tunings = [self.tuning(i) for i in range(len(self._keep))]
        if cache:
            tuning_cache.store(cache, key, gpu, tunings)
        return tunings

    @property
    def launches(self) -> int:
        """Kernel launches per ``forward()`` (``gjp_batch_launch_count``)."""
        st, n = _capi.gjp_batch_launch_count(self.handle)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_batch_launch_count")
        return n

    def tuning(self, i: int):
        st, tu, vg = _capi.gjp_batch_get_tuning(self.handle, i)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_batch_get_tuning")
        return tu, vg

    def set_tuning(self, i: int, tile_u: int, view_group: int):
        torch = _torch()
        with torch.cuda.device(self.device):
            st = _capi.gjp_batch_set_tuning(self.handle, i, tile_u, view_group)
        if st != _capi.GJP_OK:
            raise GjpError(st, "gjp_batch_set_tuning")

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            _capi.gjp_batch_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
