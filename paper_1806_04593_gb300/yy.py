"""Thin ctypes binding of libyy (include/yy.h), same names as the C ABI.

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Arrays are passed as torch tensors (device memory, float64,
C-contiguous) or as raw integer addresses; streams as torch.cuda.Stream or
raw cudaStream_t integers.  Loading fails loudly when libyy.so is missing:
there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libyy.so")

YY_OK = 0
YY_ERR_INVALID_ARG = 1
YY_ERR_OOM = 2
YY_ERR_CUDA = 3
YY_ERR_NOT_SUPPORTED = 4
YY_ERR_TIMEOUT = 5
YY_ERR_DEVICE_CHECK = 6

YY_FP64 = 0
YY_FP32 = 1
YY_TF32 = 2
YY_BF16X3 = 3
YY_FP16X2 = 4
YY_FP64_OZAKI = 5
PRECISIONS = {"fp64": YY_FP64, "fp32": YY_FP32, "tf32": YY_TF32, "bf16x3": YY_BF16X3, "fp16x2": YY_FP16X2,
              "fp64_ozaki": YY_FP64_OZAKI}

YY_TABLE_WEIGHTS = 0
YY_TABLE_TBAR = 1
YY_TABLE_ANALYSIS = 2
YY_TABLE_SYNTH = 3
YY_TABLE_SYNTH_T = 4
YY_TABLE_SYNTH_P = 5
YY_TABLE_MOMENTS = 6
YY_TABLE_COEFF = 7
YY_ANALYSIS_AUTO = 0
YY_ANALYSIS_SEPARABLE = 1
YY_ANALYSIS_DENSE = 2
ANALYSES = {"auto": YY_ANALYSIS_AUTO, "separable": YY_ANALYSIS_SEPARABLE, "dense": YY_ANALYSIS_DENSE}
YY_TABLE_ROTATION = 8
YY_TABLE_MOMENTS_TOTAL = 9

_lib = None


class YYError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {yy_status_string(status)} (status {status})")


def load():
    """Load libyy.so (build it first with paper_1806_04593_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libyy.so not found at {LIB_PATH}; run paper_1806_04593_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    lib.yy_grid_create.argtypes = [P, I, I, I, D, D, I, D, ctypes.POINTER(P)]
    lib.yy_grid_create.restype = I
    lib.yy_polar_grid_create.argtypes = [P, I, I, I, I, D, ctypes.POINTER(P)]
    lib.yy_polar_grid_create.restype = I
    lib.yy_grid_prepare.argtypes = [P, I]
    lib.yy_grid_prepare.restype = I
    lib.yy_grid_set_analysis.argtypes = [P, I]
    lib.yy_grid_set_analysis.restype = I
    lib.yy_grid_analysis_splits.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.yy_grid_analysis_splits.restype = I
    lib.yy_grid_set_analysis_splits.argtypes = [P, I, I]
    lib.yy_grid_set_analysis_splits.restype = I
    lib.yy_potential.argtypes = [P, P, P, P, P, P, P, I, P]
    lib.yy_potential.restype = I
    lib.yy_potential_host.argtypes = [P, P, P, P, P, P, P, I, P]
    lib.yy_potential_host.restype = I
    lib.yy_potential_host_async.argtypes = [P, P, P, P, P, P, P, I, P]
    lib.yy_potential_host_async.restype = I
    lib.yy_potential_host_wait.argtypes = [P]
    lib.yy_potential_host_wait.restype = I
    lib.yy_grid_copy_table.argtypes = [P, I, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.yy_grid_copy_table.restype = I
    lib.yy_last_device_status.argtypes = [P]
    lib.yy_last_device_status.restype = I
    lib.yy_destroy.argtypes = [P]
    lib.yy_destroy.restype = None
    lib.yy_status_string.argtypes = [I]
    lib.yy_status_string.restype = ctypes.c_char_p
    lib.yy_solve_flops.argtypes = [P, I]
    lib.yy_solve_flops.restype = D
    lib.yy_radial_scan_static.argtypes = [P, I, I, D, P, P, P]
    lib.yy_radial_scan_static.restype = I
    lib.yy_last_launch_count.argtypes = [P]
    lib.yy_last_launch_count.restype = I
    lib.yy_grid_set_profiling.argtypes = [P, I]
    lib.yy_grid_set_profiling.restype = I
    lib.yy_grid_stage_ms.argtypes = [P, ctypes.POINTER(D)]
    lib.yy_grid_stage_ms.restype = I
    lib.yy_grid_kernel_ms.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_char_p)]
    lib.yy_grid_kernel_ms.restype = I
    lib.yy_debug_fail_alloc_after.argtypes = [I]
    lib.yy_debug_fail_alloc_after.restype = None
    lib.yy_batch_create.argtypes = [P, I, ctypes.POINTER(P)]
    lib.yy_batch_create.restype = I
    lib.yy_batch_prepare.argtypes = [P, I]
    lib.yy_batch_prepare.restype = I
    lib.yy_batch_tune.argtypes = [P, I, I, I, P]
    lib.yy_batch_tune.restype = I
    lib.yy_batch_set_analysis.argtypes = [P, I, I]
    lib.yy_batch_set_analysis.restype = I
    lib.yy_batch_potential.argtypes = [P, P, P, P, P, P, P, I, P]
    lib.yy_batch_potential.restype = I
    lib.yy_batch_grid.argtypes = [P, I]
    lib.yy_batch_grid.restype = P
    lib.yy_batch_last_launch_count.argtypes = [P]
    lib.yy_batch_last_launch_count.restype = I
    lib.yy_batch_branches.argtypes = [P]
    lib.yy_batch_branches.restype = I
    lib.yy_batch_analysis_splits.argtypes = [P, I, I]
    lib.yy_batch_analysis_splits.restype = I
    lib.yy_batch_set_grouping.argtypes = [P, I]
    lib.yy_batch_set_grouping.restype = I
    lib.yy_batch_groups.argtypes = [P]
    lib.yy_batch_groups.restype = I
    lib.yy_batch_last_device_status.argtypes = [P]
    lib.yy_batch_last_device_status.restype = I
    lib.yy_batch_destroy.argtypes = [P]
    lib.yy_batch_destroy.restype = None
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def yy_status_string(status):
    return load().yy_status_string(int(status)).decode()


def yy_grid_create(r_edges, n_theta, n_phi, delta_theta, delta_phi, l_max, G=1.0):
    """Returns (status, handle)."""
    r = np.ascontiguousarray(r_edges, dtype=np.float64)
    h = ctypes.c_void_p()
    st = load().yy_grid_create(r.ctypes.data, int(r.size - 1), int(n_theta), int(n_phi),
                               float(delta_theta), float(delta_phi), int(l_max), float(G),
                               ctypes.byref(h))
    return st, h.value


def yy_polar_grid_create(r_edges, n_theta, n_phi, l_max, G=1.0):
    """Returns (status, handle) of a full spherical polar grid."""
    r = np.ascontiguousarray(r_edges, dtype=np.float64)
    h = ctypes.c_void_p()
    st = load().yy_polar_grid_create(r.ctypes.data, int(r.size - 1), int(n_theta), int(n_phi), int(l_max),
                                     float(G), ctypes.byref(h))
    return st, h.value


def yy_grid_prepare(handle, prec):
    return load().yy_grid_prepare(handle, int(prec))


def yy_grid_set_analysis(handle, method):
    return load().yy_grid_set_analysis(handle, int(method))


def yy_grid_analysis_splits(handle, prec):
    """(current split, the sizes' default, the largest accepted split)."""
    rule, cap = ctypes.c_int(0), ctypes.c_int(0)
    cur = load().yy_grid_analysis_splits(handle, int(prec), ctypes.byref(rule), ctypes.byref(cap))
    return cur, rule.value, cap.value


def yy_grid_set_analysis_splits(handle, prec, splits):
    return load().yy_grid_set_analysis_splits(handle, int(prec), int(splits))


def yy_potential(handle, rho_yin, rho_yang, phi_yin, phi_yang, grad_yin=None, grad_yang=None,
                 prec=YY_FP64, stream=None):
    return load().yy_potential(handle, _ptr(rho_yin), _ptr(rho_yang), _ptr(phi_yin), _ptr(phi_yang),
                               _ptr(grad_yin), _ptr(grad_yang), int(prec), _stream(stream))


def yy_potential_host(handle, rho_yin, rho_yang, phi_yin, phi_yang, grad_yin=None, grad_yang=None,
                      prec=YY_FP64, stream=None):
    return load().yy_potential_host(handle, _ptr(rho_yin), _ptr(rho_yang), _ptr(phi_yin),
                                    _ptr(phi_yang), _ptr(grad_yin), _ptr(grad_yang), int(prec),
                                    _stream(stream))


def yy_potential_host_async(handle, rho_yin, rho_yang, phi_yin, phi_yang, grad_yin=None, grad_yang=None,
                            prec=YY_FP64, stream=None):
    return load().yy_potential_host_async(handle, _ptr(rho_yin), _ptr(rho_yang), _ptr(phi_yin),
                                          _ptr(phi_yang), _ptr(grad_yin), _ptr(grad_yang), int(prec),
                                          _stream(stream))


def yy_potential_host_wait(handle):
    return load().yy_potential_host_wait(handle)


def yy_grid_copy_table(handle, which):
    """Returns (status, numpy float64 array)."""
    lib = load()
    n = ctypes.c_size_t(0)
    st = lib.yy_grid_copy_table(handle, int(which), None, ctypes.byref(n))
    if st != YY_OK:
        return st, None
    out = np.empty(n.value, dtype=np.float64)
    st = lib.yy_grid_copy_table(handle, int(which), out.ctypes.data, ctypes.byref(n))
    return st, out


def yy_last_device_status(handle):
    return load().yy_last_device_status(handle)


def yy_destroy(handle):
    load().yy_destroy(handle)


def yy_solve_flops(handle, with_gradient):
    return load().yy_solve_flops(handle, int(bool(with_gradient)))


def yy_radial_scan_static(r_edges, n_r, l_max, G, moments, coeff, stream=None):
    """Allocation-free radial scan (device pointers / tensors)."""
    return load().yy_radial_scan_static(_ptr(r_edges), int(n_r), int(l_max), float(G), _ptr(moments),
                                        _ptr(coeff), _stream(stream))


def yy_last_launch_count(handle):
    return load().yy_last_launch_count(handle)


YY_STAGE_COUNT = 3
STAGES = ("analysis", "scan", "synthesis")


def yy_grid_set_profiling(handle, enable):
    return load().yy_grid_set_profiling(handle, int(bool(enable)))


def yy_grid_stage_ms(handle):
    """Returns (status, dict stage -> ms of the last solve)."""
    buf = (ctypes.c_double * YY_STAGE_COUNT)()
    st = load().yy_grid_stage_ms(handle, buf)
    return st, dict(zip(STAGES, list(buf)))


def yy_grid_kernel_ms(handle, index):
    """Returns (status, ms, name) of kernel `index` of the last profiled solve."""
    ms = ctypes.c_double(0.0)
    name = ctypes.c_char_p()
    st = load().yy_grid_kernel_ms(handle, int(index), ctypes.byref(ms), ctypes.byref(name))
    return st, ms.value, (name.value.decode() if name.value else None)


def yy_grid_kernels_ms(handle):
    """List of (name, ms) for every kernel of the last profiled solve."""
    out = []
    for i in range(min(yy_last_launch_count(handle), 32)):
        st, ms, name = yy_grid_kernel_ms(handle, i)
        if st != YY_OK:
            raise YYError(st, "yy_grid_kernel_ms")
        out.append((name, ms))
    return out


def yy_debug_fail_alloc_after(n):
    load().yy_debug_fail_alloc_after(int(n))


class FieldDesc(ctypes.Structure):
    """yy_field_desc (include/yy.h)."""
    _fields_ = [("r_edges", ctypes.c_void_p), ("n_r", ctypes.c_int), ("n_theta", ctypes.c_int),
                ("n_phi", ctypes.c_int), ("delta_theta", ctypes.c_double), ("delta_phi", ctypes.c_double),
                ("l_max", ctypes.c_int), ("G", ctypes.c_double)]


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, x in enumerate(items):
        arr[i] = _ptr(x)
    return arr


class Batch:
    """Owning wrapper of a yy_batch handle (many fields, one CUDA graph)."""

    def __init__(self, specs):
        self.specs = list(specs)
        self._r = [np.ascontiguousarray(sp.r_edges, dtype=np.float64) for sp in self.specs]
        descs = (FieldDesc * len(self.specs))()
        for d, sp, r in zip(descs, self.specs, self._r):
            d.r_edges = r.ctypes.data
            d.n_r, d.n_theta, d.n_phi = int(r.size - 1), int(sp.n_theta), int(sp.n_phi)
            d.delta_theta, d.delta_phi = float(sp.delta_theta), float(sp.delta_phi)
            d.l_max, d.G = int(sp.lmax), float(sp.G)
        h = ctypes.c_void_p()
        st = load().yy_batch_create(ctypes.cast(descs, ctypes.c_void_p), len(self.specs), ctypes.byref(h))
        if st != YY_OK:
            raise YYError(st, "yy_batch_create")
        self.handle = h.value

    def prepare(self, prec):
        st = load().yy_batch_prepare(self.handle, PRECISIONS.get(prec, prec))
        if st != YY_OK:
            raise YYError(st, "yy_batch_prepare")

    def tune(self, prec, gradient=True, reps=2):
        chosen = (ctypes.c_int * len(self.specs))()
        st = load().yy_batch_tune(self.handle, PRECISIONS.get(prec, prec), int(bool(gradient)), int(reps),
                                  ctypes.cast(chosen, ctypes.c_void_p))
        if st != YY_OK:
            raise YYError(st, "yy_batch_tune")
        return list(chosen)

    def set_analysis(self, field, method):
        st = load().yy_batch_set_analysis(self.handle, int(field), ANALYSES.get(method, method))
        if st != YY_OK:
            raise YYError(st, "yy_batch_set_analysis")

    def potential(self, rho_yin, rho_yang, phi_yin, phi_yang, grad_yin=None, grad_yang=None,
                  prec=YY_FP64, stream=None):
        gy = _ptr_array(grad_yin) if grad_yin is not None else None
        gg = _ptr_array(grad_yang) if grad_yang is not None else None
        vp = lambda a: ctypes.cast(a, ctypes.c_void_p) if a is not None else None
        st = load().yy_batch_potential(self.handle, vp(_ptr_array(rho_yin)), vp(_ptr_array(rho_yang)),
                                       vp(_ptr_array(phi_yin)), vp(_ptr_array(phi_yang)), vp(gy), vp(gg),
                                       PRECISIONS.get(prec, prec), _stream(stream))
        if st != YY_OK:
            raise YYError(st, "yy_batch_potential")

    def launch_count(self):
        return load().yy_batch_last_launch_count(self.handle)

    def branches(self):
        return load().yy_batch_branches(self.handle)

    def groups(self):
        return load().yy_batch_groups(self.handle)

    def grid_handle(self, field):
        return load().yy_batch_grid(self.handle, int(field))

    def analysis_splits(self, field, prec):
        return load().yy_batch_analysis_splits(self.handle, int(field), PRECISIONS.get(prec, prec))

    def set_grouping(self, groups):
        """Grouped solves in `groups` concurrent groups of fields (one launch per
        stage each; tensor-core forms, dense fields), or 0 for per-field graphs."""
        st = load().yy_batch_set_grouping(self.handle, int(groups))
        if st != YY_OK:
            raise YYError(st, "yy_batch_set_grouping")

    def device_status(self):
        return load().yy_batch_last_device_status(self.handle)

    def close(self):
        if self.handle:
            load().yy_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """Owning wrapper of a yy_grid handle with torch-tensor conveniences."""

    def __init__(self, r_edges, n_theta, n_phi, delta_theta, delta_phi, l_max, G=1.0):
        st, h = yy_grid_create(r_edges, n_theta, n_phi, delta_theta, delta_phi, l_max, G)
        if st != YY_OK:
            raise YYError(st, "yy_grid_create")
        self.handle = h
        self.n_r = int(np.asarray(r_edges).size - 1)
        self.n_theta, self.n_phi, self.l_max = int(n_theta), int(n_phi), int(l_max)
        self.n_lm = (self.l_max + 1) ** 2

    @classmethod
    def from_spec(cls, spec):
        if getattr(spec, "polar", False):
            return PolarGrid(spec.r_edges, spec.n_theta, spec.n_phi, spec.lmax, spec.G)
        return cls(spec.r_edges, spec.n_theta, spec.n_phi, spec.delta_theta, spec.delta_phi,
                   spec.lmax, spec.G)

    @property
    def field_shape(self):
        return (self.n_r, self.n_theta, self.n_phi)

    def set_analysis(self, method):
        st = yy_grid_set_analysis(self.handle, ANALYSES.get(method, method))
        if st != YY_OK:
            raise YYError(st, "yy_grid_set_analysis")

    def analysis_splits(self, prec):
        """(current, default, largest) K split of the dense analysis of a form."""
        return yy_grid_analysis_splits(self.handle, PRECISIONS.get(prec, prec))

    def set_analysis_splits(self, prec, splits):
        st = yy_grid_set_analysis_splits(self.handle, PRECISIONS.get(prec, prec), splits)
        if st != YY_OK:
            raise YYError(st, "yy_grid_set_analysis_splits")

    def prepare(self, prec):
        st = yy_grid_prepare(self.handle, PRECISIONS.get(prec, prec))
        if st != YY_OK:
            raise YYError(st, "yy_grid_prepare")

    def potential(self, rho_yin, rho_yang, phi_yin, phi_yang, grad_yin=None, grad_yang=None,
                  prec=YY_FP64, stream=None):
        st = yy_potential(self.handle, rho_yin, rho_yang, phi_yin, phi_yang, grad_yin, grad_yang,
                          PRECISIONS.get(prec, prec), stream)
        if st != YY_OK:
            raise YYError(st, "yy_potential")

    def solve(self, rho_yin, rho_yang, gradient=False, prec=YY_FP64, stream=None):
        """Allocate outputs (torch, same device) and solve; returns a dict."""
        import torch
        phi_yin = torch.empty_like(rho_yin)
        phi_yang = torch.empty_like(rho_yang)
        g_yin = g_yang = None
        if gradient:
            g_yin = torch.empty((3,) + tuple(rho_yin.shape), dtype=torch.float64, device=rho_yin.device)
            g_yang = torch.empty_like(g_yin)
        self.potential(rho_yin, rho_yang, phi_yin, phi_yang, g_yin, g_yang, prec, stream)
        out = {"phi_yin": phi_yin, "phi_yang": phi_yang}
        if gradient:
            out["grad_yin"], out["grad_yang"] = g_yin, g_yang
        return out

    def table(self, which):
        st, arr = yy_grid_copy_table(self.handle, which)
        if st != YY_OK:
            raise YYError(st, "yy_grid_copy_table")
        return arr

    def flops(self, gradient):
        return yy_solve_flops(self.handle, gradient)

    def close(self):
        if self.handle:
            yy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PolarGrid(Grid):
    """Owning wrapper of a full spherical polar grid handle (one patch)."""

    def __init__(self, r_edges, n_theta, n_phi, l_max, G=1.0):
        st, h = yy_polar_grid_create(r_edges, n_theta, n_phi, l_max, G)
        if st != YY_OK:
            raise YYError(st, "yy_polar_grid_create")
        self.handle = h
        self.n_r = int(np.asarray(r_edges).size - 1)
        self.n_theta, self.n_phi, self.l_max = int(n_theta), int(n_phi), int(l_max)
        self.n_lm = (self.l_max + 1) ** 2

    def solve(self, rho, rho_yang=None, gradient=False, prec=YY_FP64, stream=None):
        """Allocate outputs and solve; returns {'phi': ..., 'grad': ...}."""
        import torch
        if rho_yang is not None:
            raise ValueError("a polar grid has one patch")
        phi = torch.empty_like(rho)
        grad = torch.empty((3,) + tuple(rho.shape), dtype=torch.float64, device=rho.device) if gradient else None
        self.potential(rho, None, phi, None, grad, None, prec, stream)
        out = {"phi": phi}
        if gradient:
            out["grad"] = grad
        return out

