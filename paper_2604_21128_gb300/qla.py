"""Thin Python binding of libqla (the C ABI declared in include/qla.h).

The module-level functions carry the C names and only marshal arguments:
every step of the computation runs in the CUDA library.  ``Grid`` wraps one
context and takes its device workspace and stream from PyTorch.

Loading fails loudly: if ``libqla.so`` has not been built, or no CUDA device
is present when a context is created, an exception is raised.  There is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqla.so")

QLA_FP64, QLA_FP32 = 0, 1
QLA_TE_ONLY = 1
QLA_POTENTIAL_LITERAL = 2
QLA_POTENTIAL_NONE = 4
QLA_ANISOTROPIC = 8
QLA_POTENTIAL_LCU = 16
QLA_DOUBLE_SINGLE = 32
QLA_KERNEL_AUTO, QLA_KERNEL_TILE, QLA_KERNEL_MARCH, QLA_KERNEL_MARCH_PLAIN = 0, 1, 2, 3
QLA_KERNEL_MARCH_STEP, QLA_KERNEL_MARCH_FLOW = 4, 5

STATUS = {0: "QLA_OK", 1: "QLA_EINVAL", 2: "QLA_ESTATE", 3: "QLA_ENOMEM",
          4: "QLA_ECUDA", 5: "QLA_ETIMEOUT", 6: "QLA_ENONFINITE"}


class QLAError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s%s" % (STATUS.get(status, str(status)), (": " + msg) if msg else ""))


class qla_packet(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("x0", "y0", "angle", "k0", "width", "transverse_width", "amplitude")]


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)


def load():
    """Load libqla.so (raises OSError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libqla.so not built: run __graft_entry__.build() "
                          "(or python paper_2604_21128_gb300/build.py)")
        lib = ctypes.CDLL(LIB_PATH)
        c_int, c_ll, c_sz, c_vp, c_u = (ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t,
                                        ctypes.c_void_p, ctypes.c_uint)
        lib.qla_workspace_bytes.argtypes = [c_int, c_int, c_int, c_u]
        lib.qla_workspace_bytes.restype = c_sz
        lib.qla_init_grid.argtypes = [ctypes.POINTER(c_vp), c_int, c_int, ctypes.c_double,
                                      c_int, c_u, c_vp, c_vp, c_sz]
        for name, args in (("qla_set_medium", [c_vp, c_vp]),
                           ("qla_set_medium_tensor", [c_vp, c_vp, c_vp, c_vp]),
                           ("qla_set_packet", [c_vp, ctypes.POINTER(qla_packet)]),
                           ("qla_set_state", [c_vp, c_vp]),
                           ("qla_get_state", [c_vp, c_vp]),
                           ("qla_step", [c_vp, c_ll]),
                           ("qla_energy", [c_vp, _DP]),
                           ("qla_divergence", [c_vp, c_vp]),
                           ("qla_fields", [c_vp] + [c_vp] * 6),
                           ("qla_probe", [c_vp, c_int, c_vp, c_vp, c_vp]),
                           ("qla_set_step_kernel", [c_vp, c_int]),
                           ("qla_set_march_tuning", [c_vp, c_int, c_int]),
                           ("qla_march_plan", [c_vp, c_vp, c_vp, c_vp]),
                           ("qla_flow_plan", [c_vp, c_vp]),
                           ("qla_debug_flow", [c_vp, c_ll, c_ll]),
                           ("qla_flow_item_deps", [c_int, c_int, c_int, c_int, c_vp, c_int,
                                                   c_vp]),
                           ("qla_set_packet_window", [c_vp, ctypes.POINTER(qla_packet), c_int,
                                                      c_int, c_int, c_int]),
                           ("qla_pack_box", [c_vp, c_int, c_int, c_int, c_int, c_vp]),
                           ("qla_unpack_box", [c_vp, c_int, c_int, c_int, c_int, c_vp]),
                           ("qla_energy_box", [c_vp, c_int, c_int, c_int, c_int, _DP])):
            getattr(lib, name).argtypes = args
            getattr(lib, name).restype = c_int
        lib.qla_init_grid.restype = c_int
        lib.qla_box_bytes.argtypes = [c_vp, c_int, c_int]
        lib.qla_box_bytes.restype = c_sz
        lib.qla3_workspace_bytes.argtypes = [c_int, c_int, c_int, c_int, c_u]
        lib.qla3_workspace_bytes.restype = c_sz
        lib.qla3_init.argtypes = [ctypes.POINTER(c_vp), c_int, c_int, c_int, ctypes.c_double,
                                  c_int, c_u, c_vp, c_vp, c_sz]
        lib.qla3_init.restype = c_int
        for name, args in (("qla3_set_medium", [c_vp, c_vp]), ("qla3_set_state", [c_vp, c_vp]),
                           ("qla3_get_state", [c_vp, c_vp]), ("qla3_step", [c_vp, c_ll]),
                           ("qla3_energy", [c_vp, _DP]), ("qla3_set_step_kernel", [c_vp, c_int]),
                           ("qla3_divergence", [c_vp, c_vp]),
                           ("qla3_set_packet", [c_vp, ctypes.POINTER(qla_packet)])):
            getattr(lib, name).argtypes = args
            getattr(lib, name).restype = c_int
        lib.qla3_launch_count.argtypes = [c_vp]
        lib.qla3_launch_count.restype = c_ll
        lib.qla3_last_error.argtypes = [c_vp]
        lib.qla3_last_error.restype = ctypes.c_char_p
        lib.qla3_destroy.argtypes = [c_vp]
        lib.qla3_destroy.restype = None
        lib.qla_batch_workspace_bytes.argtypes = [c_int, c_vp, c_vp, c_int, c_u]
        lib.qla_batch_workspace_bytes.restype = c_sz
        lib.qla_batch_create.argtypes = [ctypes.POINTER(c_vp), c_int, c_vp, c_vp,
                                         ctypes.c_double, c_int, c_u, c_vp, c_vp, c_sz]
        lib.qla_batch_create.restype = c_int
        lib.qla_batch_instance.argtypes = [c_vp, c_int]
        lib.qla_batch_instance.restype = c_vp
        for name, args in (("qla_batch_step", [c_vp, c_ll]),
                           ("qla_batch_run", [c_vp, c_ll, c_ll, c_vp]),
                           ("qla_batch_energy", [c_vp, c_vp]),
                           ("qla_batch_autotune", [c_vp, c_int, c_vp, c_vp]),
                           ("qla_batch_set_tuning", [c_vp, c_int, c_int]),
                           ("qla_batch_debug_barrier", [c_vp, c_ll, c_int])):
            getattr(lib, name).argtypes = args
            getattr(lib, name).restype = c_int
        lib.qla_batch_launch_count.argtypes = [c_vp]
        lib.qla_batch_launch_count.restype = c_ll
        lib.qla_batch_last_error.argtypes = [c_vp]
        lib.qla_batch_last_error.restype = ctypes.c_char_p
        lib.qla_batch_destroy.argtypes = [c_vp]
        lib.qla_batch_destroy.restype = None
        lib.surr_workspace_bytes.argtypes = [c_int, c_int, c_int]
        lib.surr_workspace_bytes.restype = c_sz
        lib.surr_create.argtypes = [ctypes.POINTER(c_vp), c_int, c_int, c_int, ctypes.c_ulonglong,
                                    c_vp, c_vp, c_sz]
        lib.surr_create.restype = c_int
        lib.surr_param_count.argtypes = [c_vp]
        lib.surr_param_count.restype = c_ll
        for name, args in (("surr_get_params", [c_vp, c_vp]),
                           ("surr_set_params", [c_vp, c_vp]),
                           ("surr_forward", [c_vp, c_vp, c_int, c_vp]),
                           ("surr_loss_grad", [c_vp, c_vp, c_vp, c_int, c_vp, c_vp]),
                           ("surr_train_step", [c_vp, c_vp, c_vp, c_int, ctypes.c_float, c_vp]),
                           ("surr_features", [c_vp, c_vp]),
                           ("surr_advance", [c_vp, c_vp, c_int, c_int, ctypes.c_double,
                                             ctypes.c_double, c_vp, c_vp, c_vp]),
                           ("surr_conv3x3_raw", [c_vp, c_int, c_int, c_int, c_int, c_vp, c_int,
                                                 c_vp, c_vp]),
                           ("surr_weight_grad_raw", [c_vp, c_vp, c_int, c_int, c_int, c_int, c_int,
                                                     c_int, c_vp, c_vp, c_vp])):
            getattr(lib, name).argtypes = args
            getattr(lib, name).restype = c_int
        lib.surr_last_error.argtypes = [c_vp]
        lib.surr_last_error.restype = ctypes.c_char_p
        lib.surr_destroy.argtypes = [c_vp]
        lib.surr_destroy.restype = None
        lib.qla_launch_count.argtypes = [c_vp]
        lib.qla_launch_count.restype = c_ll
        lib.qla_last_error.argtypes = [c_vp]
        lib.qla_last_error.restype = ctypes.c_char_p
        lib.qla_status_string.argtypes = [c_int]
        lib.qla_status_string.restype = ctypes.c_char_p
        lib.qla_destroy.argtypes = [c_vp]
        lib.qla_destroy.restype = None
        _lib = lib
    return _lib


def _check(ctx, status):
    if status != 0:
        msg = load().qla_last_error(ctx).decode() if ctx else ""
        raise QLAError(status, msg)


def _host_ptr(a, n_expected, writable=False):
    """Pointer to a contiguous FP64 host buffer (numpy array or CPU tensor)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous float64")
        if writable and not a.flags.writeable:
            raise TypeError("output array is read-only")
        if a.size != n_expected:
            raise ValueError("expected %d values, got %d" % (n_expected, a.size))
        return ctypes.c_void_p(a.ctypes.data)
    import torch
    if not isinstance(a, torch.Tensor) or a.device.type != "cpu" or a.dtype != torch.float64 \
            or not a.is_contiguous() or a.numel() != n_expected:
        raise TypeError("host buffers must be contiguous float64 CPU tensors or numpy arrays")
    return ctypes.c_void_p(a.data_ptr())


# ---------------------------------------------------------------------------
# C-named functions
# ---------------------------------------------------------------------------

def qla_workspace_bytes(nx, ny, precision, flags):
    return int(load().qla_workspace_bytes(nx, ny, precision, flags))


def qla_init_grid(nx, ny, delta, precision, flags, cuda_stream, workspace, workspace_bytes):
    ctx = ctypes.c_void_p()
    st = load().qla_init_grid(ctypes.byref(ctx), int(nx), int(ny), float(delta), int(precision),
                              int(flags), ctypes.c_void_p(cuda_stream or 0),
                              ctypes.c_void_p(workspace or 0), int(workspace_bytes))
    _check(None, st)
    return ctx


def qla_set_medium(ctx, n, nx, ny):
    _check(ctx, load().qla_set_medium(ctx, _host_ptr(n, nx * ny)))


def qla_set_medium_tensor(ctx, n_x, n_y, n_z, nx, ny):
    _check(ctx, load().qla_set_medium_tensor(ctx, _host_ptr(n_x, nx * ny), _host_ptr(n_y, nx * ny),
                                             _host_ptr(n_z, nx * ny)))


def qla_set_packet(ctx, x0, y0, angle, k0, width, transverse_width=0.0, amplitude=1.0):
    p = qla_packet(float(x0), float(y0), float(angle), float(k0), float(width),
                   float(transverse_width), float(amplitude))
    _check(ctx, load().qla_set_packet(ctx, ctypes.byref(p)))


def qla_set_state(ctx, q, nx, ny):
    _check(ctx, load().qla_set_state(ctx, _host_ptr(q, 6 * nx * ny)))


def qla_get_state(ctx, out, nx, ny):
    _check(ctx, load().qla_get_state(ctx, _host_ptr(out, 6 * nx * ny, writable=True)))


def qla_step(ctx, n_steps):
    _check(ctx, load().qla_step(ctx, int(n_steps)))


def qla_energy(ctx):
    v = ctypes.c_double()
    _check(ctx, load().qla_energy(ctx, ctypes.byref(v)))
    return v.value


DIV_KEYS = ("div_b_sq", "grad_b_sq", "div_d_sq", "grad_d_sq", "div_b_max", "div_d_max")


def qla_divergence(ctx):
    out = np.empty(6)
    _check(ctx, load().qla_divergence(ctx, ctypes.c_void_p(out.ctypes.data)))
    return dict(zip(DIV_KEYS, (float(v) for v in out)))


def qla_fields(ctx, nx, ny, Ex=None, Ey=None, Ez=None, Bx=None, By=None, Bz=None):
    ptrs = [_host_ptr(a, nx * ny, writable=True) if a is not None else ctypes.c_void_p(0)
            for a in (Ex, Ey, Ez, Bx, By, Bz)]
    _check(ctx, load().qla_fields(ctx, *ptrs))


def qla_probe(ctx, i, j):
    """Amplitudes q0..q5 at sites (i[k], j[k]); returns an array (count, 6)."""
    i = np.ascontiguousarray(i, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    if i.shape != j.shape or i.ndim != 1:
        raise ValueError("i and j must be 1-D of equal length")
    out = np.empty((i.size, 6))
    _check(ctx, load().qla_probe(ctx, int(i.size), ctypes.c_void_p(i.ctypes.data),
                                 ctypes.c_void_p(j.ctypes.data), ctypes.c_void_p(out.ctypes.data)))
    return out




def qla_set_packet_window(ctx, i0, j0, gnx, gny, x0, y0, angle, k0, width,
                          transverse_width=0.0, amplitude=1.0):
    p = qla_packet(float(x0), float(y0), float(angle), float(k0), float(width),
                   float(transverse_width), float(amplitude))
    _check(ctx, load().qla_set_packet_window(ctx, ctypes.byref(p), int(i0), int(j0), int(gnx),
                                             int(gny)))


def qla_box_bytes(ctx, w, h):
    return int(load().qla_box_bytes(ctx, int(w), int(h)))


def qla_pack_box(ctx, i0, j0, w, h, dst_dev_ptr):
    _check(ctx, load().qla_pack_box(ctx, int(i0), int(j0), int(w), int(h),
                                    ctypes.c_void_p(dst_dev_ptr)))


def qla_unpack_box(ctx, i0, j0, w, h, src_dev_ptr):
    _check(ctx, load().qla_unpack_box(ctx, int(i0), int(j0), int(w), int(h),
                                      ctypes.c_void_p(src_dev_ptr)))


def qla_energy_box(ctx, i0, j0, w, h):
    v = ctypes.c_double()
    _check(ctx, load().qla_energy_box(ctx, int(i0), int(j0), int(w), int(h), ctypes.byref(v)))
    return v.value


def qla_set_step_kernel(ctx, kernel):
    _check(ctx, load().qla_set_step_kernel(ctx, int(kernel)))


def qla_set_march_tuning(ctx, lane_cols=0, rows=0):
    _check(ctx, load().qla_set_march_tuning(ctx, int(lane_cols), int(rows)))


def qla_launch_count(ctx):
    return int(load().qla_launch_count(ctx))


def qla_march_plan(ctx):
    """(work items, plateau items, plateau records) of the marching plan."""
    a, b, n = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(ctx, load().qla_march_plan(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
    return a.value, b.value, n.value


def qla_flow_plan(ctx):
    """Segment rows of the current dataflow plan (0: one launch per step)."""
    v = ctypes.c_int(0)
    _check(ctx, load().qla_flow_plan(ctx, ctypes.byref(v)))
    return v.value


def qla_flow_item_deps(nx, ny, segment_rows, item):
    """Items that a unit of `item` waits for in a dataflow plan (see
    qla_flow_item_deps); host only."""
    buf = (ctypes.c_int * 64)()
    n = ctypes.c_int(0)
    st = load().qla_flow_item_deps(int(nx), int(ny), int(segment_rows), int(item), buf, 64,
                                   ctypes.byref(n))
    if st != 0:
        raise QLAError(st, "qla_flow_item_deps(%d, %d, %d, %d)" % (nx, ny, segment_rows, item))
    return [buf[k] for k in range(min(n.value, 64))]


def qla_debug_flow(ctx, budget_cycles=0, withhold_unit=-1):
    _check(ctx, load().qla_debug_flow(ctx, int(budget_cycles), int(withhold_unit)))


def qla_last_error(ctx):
    return load().qla_last_error(ctx).decode()


def qla_destroy(ctx):
    load().qla_destroy(ctx)


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class Grid:
    """One QLA lattice on a CUDA device.

    precision: "fp64" or "fp32"; te_only: evolve only q2, q3, q4;
    potential: "rotation" (default reading), "literal", "none" or "lcu";
    tensor: a diagonal index tensor (set_medium with a (3, ny, nx) array);
    double_single: FP64 contexts step in double-single arithmetic on the FP32
    pipes (QLA_DOUBLE_SINGLE).
    The device workspace is a torch uint8 tensor; work is enqueued on
    ``stream`` (default: torch's current stream on the device)."""

    def __init__(self, nx, ny, delta=1.0, precision="fp64", te_only=False,
                 potential="rotation", device=None, stream=None, tensor=False,
                 double_single=False):
        import torch
        load()
        if not torch.cuda.is_available():
            raise RuntimeError("libqla needs a CUDA device; none is available")
        self.nx, self.ny, self.delta = int(nx), int(ny), float(delta)
        self.precision = {"fp64": QLA_FP64, "fp32": QLA_FP32}[precision]
        flags = (QLA_TE_ONLY if te_only else 0) | (QLA_ANISOTROPIC if tensor else 0) | \
            (QLA_DOUBLE_SINGLE if double_single else 0) | {
            "rotation": 0, "literal": QLA_POTENTIAL_LITERAL, "none": QLA_POTENTIAL_NONE,
            "lcu": QLA_POTENTIAL_LCU}[potential]
        self.flags = flags
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else (device if isinstance(device, int) else device.index or 0))
        nbytes = qla_workspace_bytes(self.nx, self.ny, self.precision, flags)
        if nbytes == 0:
            raise QLAError(1, "invalid lattice")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self._ctx = qla_init_grid(self.nx, self.ny, self.delta, self.precision, flags,
                                      self.stream.cuda_stream, self.workspace.data_ptr(), nbytes)

    # context-managed device selection for every call
    def _dev(self):
        import torch
        return torch.cuda.device(self.device)

    def set_medium(self, n):
        """n: (ny, nx) scalar index, or (3, ny, nx) = (n_x, n_y, n_z) for a
        context made with tensor=True."""
        with self._dev():
            if getattr(n, "ndim", 2) == 3:
                a = [np.ascontiguousarray(n[c], dtype=np.float64) for c in range(3)]
                qla_set_medium_tensor(self._ctx, a[0], a[1], a[2], self.nx, self.ny)
            else:
                qla_set_medium(self._ctx, n, self.nx, self.ny)

    def set_packet(self, x0, y0, angle, k0, width, transverse_width=0.0, amplitude=1.0):
        with self._dev():
            qla_set_packet(self._ctx, x0, y0, angle, k0, width, transverse_width, amplitude)

    def set_state(self, q):
        with self._dev():
            qla_set_state(self._ctx, q, self.nx, self.ny)

    def get_state(self, out=None):
        if out is None:
            out = np.empty((6, self.ny, self.nx))
        with self._dev():
            qla_get_state(self._ctx, out, self.nx, self.ny)
        return out

    def step(self, n_steps):
        with self._dev():
            qla_step(self._ctx, n_steps)

    def energy(self):
        with self._dev():
            return qla_energy(self._ctx)

    def divergence(self):
        """Gauss-law monitors, a dict with the keys of DIV_KEYS."""
        with self._dev():
            return qla_divergence(self._ctx)

    def fields(self):
        out = {k: np.empty((self.ny, self.nx)) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
        with self._dev():
            qla_fields(self._ctx, self.nx, self.ny, **out)
        return out

    def probe(self, i, j):
        with self._dev():
            return qla_probe(self._ctx, i, j)

    def set_step_kernel(self, kernel):
        """"auto", "tile", "march", "march_plain", "march_step" or "march_flow"
        (see qla_set_step_kernel)."""
        k = {"auto": QLA_KERNEL_AUTO, "tile": QLA_KERNEL_TILE, "march": QLA_KERNEL_MARCH,
             "march_plain": QLA_KERNEL_MARCH_PLAIN, "march_step": QLA_KERNEL_MARCH_STEP,
             "march_flow": QLA_KERNEL_MARCH_FLOW}
        qla_set_step_kernel(self._ctx, k.get(kernel, kernel))

    def set_march_tuning(self, lane_cols=0, rows=0):
        qla_set_march_tuning(self._ctx, lane_cols, rows)

    # domain decomposition (qla_set_packet_window, qla_*_box)
    def set_packet_window(self, i0, j0, gnx, gny, x0, y0, angle, k0, width,
                          transverse_width=0.0, amplitude=1.0):
        with self._dev():
            qla_set_packet_window(self._ctx, i0, j0, gnx, gny, x0, y0, angle, k0, width,
                                  transverse_width, amplitude)

    def box_dtype(self):
        import torch
        return torch.float64 if self.precision == QLA_FP64 else torch.float32

    def pack_box(self, i0, j0, w, h, out=None):
        """The stored values of a rectangle as a device tensor (planes, h, w)."""
        import torch
        planes = 3 if self.flags & QLA_TE_ONLY else 6
        if out is None:
            out = torch.empty((planes, h, w), dtype=self.box_dtype(), device=self.device)
        if not out.is_contiguous() or out.device != self.device or out.numel() != planes * h * w \
                or out.dtype != self.box_dtype():
            raise ValueError("pack_box: out must be a contiguous (%d, %d, %d) %s tensor on %s"
                             % (planes, h, w, self.box_dtype(), self.device))
        with self._dev():
            qla_pack_box(self._ctx, i0, j0, w, h, out.data_ptr())
        return out

    def unpack_box(self, i0, j0, w, h, src):
        planes = 3 if self.flags & QLA_TE_ONLY else 6
        if not src.is_contiguous() or src.device != self.device or src.numel() != planes * h * w \
                or src.dtype != self.box_dtype():
            raise ValueError("unpack_box: src must be a contiguous (%d, %d, %d) %s tensor on %s"
                             % (planes, h, w, self.box_dtype(), self.device))
        with self._dev():
            qla_unpack_box(self._ctx, i0, j0, w, h, src.data_ptr())

    def energy_box(self, i0, j0, w, h):
        with self._dev():
            return qla_energy_box(self._ctx, i0, j0, w, h)


    @property
    def launches(self):
        return qla_launch_count(self._ctx)

    @property
    def march_plan(self):
        """(work items, plateau items, plateau records) of the last marching step."""
        return qla_march_plan(self._ctx)

    @property
    def flow_plan(self):
        """Segment rows of the dataflow plan (0: one launch per step)."""
        return qla_flow_plan(self._ctx)

    def debug_flow(self, budget_cycles=0, withhold_unit=-1):
        """Test hook for the dataflow waits (see qla_debug_flow)."""
        qla_debug_flow(self._ctx, budget_cycles, withhold_unit)

    def close(self):
        if getattr(self, "_borrowed", False):
            self._ctx = None
            return
        if getattr(self, "_ctx", None):
            with self._dev():
                qla_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# Batched lattices
# ---------------------------------------------------------------------------

def _bcheck(b, status):
    if status != 0:
        raise QLAError(status, load().qla_batch_last_error(b).decode() if b else "")


class Batch:
    """Many independent lattices advanced together by one persistent launch
    per chunk of steps (qla_batch_* in the C ABI).  ``instance(k)`` is a
    ``Grid``-like view of lattice k (medium, packet, state, energy, fields).
    """

    def __init__(self, sizes, delta=1.0, precision="fp32", te_only=False,
                 potential="rotation", device=None, stream=None):
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("libqla needs a CUDA device; none is available")
        self.count = len(sizes)
        nx = np.ascontiguousarray([int(a) for a, _ in sizes], dtype=np.int32)
        ny = np.ascontiguousarray([int(b) for _, b in sizes], dtype=np.int32)
        self.sizes = list(zip(nx.tolist(), ny.tolist()))
        prec = {"fp64": QLA_FP64, "fp32": QLA_FP32}[precision]
        flags = (QLA_TE_ONLY if te_only else 0) | {
            "rotation": 0, "literal": QLA_POTENTIAL_LITERAL, "none": QLA_POTENTIAL_NONE}[potential]
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else device)
        nbytes = int(lib.qla_batch_workspace_bytes(self.count, ctypes.c_void_p(nx.ctypes.data),
                                                   ctypes.c_void_p(ny.ctypes.data), prec, flags))
        if nbytes == 0:
            raise QLAError(1, "invalid batch (each nx a multiple of 4 and >= 128, ny >= 8)")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            b = ctypes.c_void_p()
            st = lib.qla_batch_create(ctypes.byref(b), self.count, ctypes.c_void_p(nx.ctypes.data),
                                      ctypes.c_void_p(ny.ctypes.data), float(delta), prec, flags,
                                      ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.c_void_p(self.workspace.data_ptr()), nbytes)
            _bcheck(None, st)
            self._b = b

    def _dev(self):
        import torch
        return torch.cuda.device(self.device)

    def instance(self, k):
        """A Grid bound to lattice k (owned by the batch)."""
        ctx = load().qla_batch_instance(self._b, int(k))
        if not ctx:
            raise IndexError(k)
        g = Grid.__new__(Grid)
        g.nx, g.ny = self.sizes[k]
        g.device, g.stream = self.device, self.stream
        g._ctx = ctypes.c_void_p(ctx)
        g._borrowed = True
        return g

    def step(self, n_steps):
        with self._dev():
            _bcheck(self._b, load().qla_batch_step(self._b, int(n_steps)))

    def run(self, n_steps, every):
        """Graph-captured run; returns energies of shape (n_steps // every, count)."""
        out = np.empty((int(n_steps) // int(every), self.count))
        with self._dev():
            _bcheck(self._b, load().qla_batch_run(self._b, int(n_steps), int(every),
                                                  ctypes.c_void_p(out.ctypes.data)))
        return out

    def energy(self):
        out = np.empty(self.count)
        with self._dev():
            _bcheck(self._b, load().qla_batch_energy(self._b, ctypes.c_void_p(out.ctypes.data)))
        return out

    def autotune(self, trial_steps=2):
        lx, rows = ctypes.c_int(), ctypes.c_int()
        with self._dev():
            _bcheck(self._b, load().qla_batch_autotune(self._b, int(trial_steps), ctypes.byref(lx),
                                                       ctypes.byref(rows)))
        return lx.value, rows.value

    def set_tuning(self, lane_cols=0, rows=0):
        _bcheck(self._b, load().qla_batch_set_tuning(self._b, int(lane_cols), int(rows)))

    def debug_barrier(self, budget_cycles=0, skip_block=-1):
        _bcheck(self._b, load().qla_batch_debug_barrier(self._b, int(budget_cycles),
                                                        int(skip_block)))

    @property
    def launches(self):
        return int(load().qla_batch_launch_count(self._b))

    def close(self):
        if getattr(self, "_b", None):
            with self._dev():
                load().qla_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Grid3:
    """A three-dimensional context (qla3_* in the C ABI): nx x ny x nz
    periodic lattice, six planes, precision "fp64" or "fp32", potential
    "rotation" or "none".  Arrays are (6, nz, ny, nx) states and (nz, ny, nx)
    media; the workspace is a torch uint8 tensor, work runs on ``stream``.
    double_single: FP64 contexts step in double-single arithmetic
    (QLA_DOUBLE_SINGLE; the slices and column kernels)."""

    def __init__(self, nx, ny, nz, delta=1.0, precision="fp64", potential="rotation",
                 stream=None, double_single=False):
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("libqla needs a CUDA device; none is available")
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        prec = {"fp64": QLA_FP64, "fp32": QLA_FP32}[precision]
        flags = {"rotation": 0, "none": QLA_POTENTIAL_NONE}[potential] | \
            (QLA_DOUBLE_SINGLE if double_single else 0)
        nbytes = int(lib.qla3_workspace_bytes(self.nx, self.ny, self.nz, prec, flags))
        if nbytes == 0:
            raise QLAError(1, "invalid 3D lattice or flags")
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        ctx = ctypes.c_void_p()
        st = lib.qla3_init(ctypes.byref(ctx), self.nx, self.ny, self.nz, float(delta), prec, flags,
                           ctypes.c_void_p(self.stream.cuda_stream),
                           ctypes.c_void_p(self.workspace.data_ptr()), nbytes)
        if st != 0:
            raise QLAError(st, "qla3_init")
        self._ctx = ctx

    def _check(self, st):
        if st != 0:
            raise QLAError(st, load().qla3_last_error(self._ctx).decode())

    @property
    def sites(self):
        return self.nx * self.ny * self.nz

    def set_medium(self, n):
        a = np.ascontiguousarray(n, dtype=np.float64)
        assert a.size == self.sites
        self._check(load().qla3_set_medium(self._ctx, ctypes.c_void_p(a.ctypes.data)))

    def set_packet(self, x0, y0, angle, k0, width, transverse_width=0.0, amplitude=1.0):
        """The E_z packet of Grid.set_packet, uniform along z."""
        p = qla_packet(x0, y0, angle, k0, width, transverse_width, amplitude)
        self._check(load().qla3_set_packet(self._ctx, ctypes.byref(p)))

    def set_state(self, q):
        a = np.ascontiguousarray(q, dtype=np.float64)
        assert a.size == 6 * self.sites
        self._check(load().qla3_set_state(self._ctx, ctypes.c_void_p(a.ctypes.data)))

    def get_state(self):
        out = np.empty((6, self.nz, self.ny, self.nx))
        self._check(load().qla3_get_state(self._ctx, ctypes.c_void_p(out.ctypes.data)))
        return out

    def step(self, n=1):
        self._check(load().qla3_step(self._ctx, int(n)))

    def set_step_kernel(self, kernel):
        """"auto" (default), "passes" (one launch per axis), "march" (fused
        along z) or "slices" (2D march per slice + column pipeline along z)."""
        k = {"auto": 0, "march": 1, "slices": 2, "passes": 3}[kernel]
        self._check(load().qla3_set_step_kernel(self._ctx, k))

    def energy(self):
        v = ctypes.c_double()
        self._check(load().qla3_energy(self._ctx, ctypes.byref(v)))
        return v.value

    def divergence(self):
        """3D Gauss-law monitors, a dict with the keys of DIV_KEYS."""
        out = np.empty(6)
        self._check(load().qla3_divergence(self._ctx, ctypes.c_void_p(out.ctypes.data)))
        return dict(zip(DIV_KEYS, (float(v) for v in out)))

    @property
    def launches(self):
        return int(load().qla3_launch_count(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None):
            load().qla3_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
