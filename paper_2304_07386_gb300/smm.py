"""Thin ctypes binding of the SMM C ABI (include/smm.h).

Argument marshalling only: every step of the hot path runs in libsmm.so.
Host inputs are NumPy arrays; device buffers are CUDA torch tensors (FP64,
contiguous) whose data pointers are passed through; the stream is torch's
current stream unless one is given.  The binding raises if the library is
missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsmm.so")

SMM_OK = 0
STATUS = {0: "SMM_OK", 1: "SMM_ERR_INVALID_ARG", 2: "SMM_ERR_CUDA", 3: "SMM_ERR_OOM", 4: "SMM_ERR_MESH",
          5: "SMM_ERR_CYCLE", 6: "SMM_ERR_NONFINITE", 7: "SMM_ERR_NOT_CONVERGED", 8: "SMM_ERR_DEVICE_TIMEOUT"}
SMM_SOURCE_ISOTROPIC, SMM_SOURCE_ANGULAR = 0, 1
SMM_INFLOW_VACUUM, SMM_INFLOW_NODAL = 0, 1
SMM_SWEEP_FP64, SMM_SWEEP_FP32_REFINED = 0, 1
SMM_PRECOND_BLOCK_JACOBI, SMM_PRECOND_MULTIGRID = 0, 1
SMM_SOLVER_LU, SMM_SOLVER_CACHED_INVERSE = 0, 1
SMM_MOMENT_IP, SMM_MOMENT_CG = 0, 1
SMM_SMOOTHER_JACOBI, SMM_SMOOTHER_CHEBYSHEV = 0, 1


class smm_mesh(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("geom_order", C.c_int32), ("n_nodes", C.c_int32),
                ("nodes", C.POINTER(C.c_double)), ("elem_nodes", C.POINTER(C.c_int32))]


class smm_options(C.Structure):
    _fields_ = [("sweep_precision", C.c_int32), ("tol_cg", C.c_double), ("max_cg", C.c_int32),
                ("kappa_scale", C.c_double), ("spin_timeout_s", C.c_double), ("precond", C.c_int32),
                ("sweep_solver", C.c_int32), ("anderson_depth", C.c_int32), ("guess_check", C.c_int32),
                ("mg_smooth_steps", C.c_int32), ("moment_discretization", C.c_int32),
                ("negative_flux_fixup", C.c_int32), ("sweep_tiles", C.c_int32), ("mg_smoother", C.c_int32),
                ("cg_device_loop", C.c_int32), ("resume_history", C.c_int32), ("cycle_lagging", C.c_int32),
                ("cg_tol_adaptive", C.c_double), ("cg_guess_extrapolate", C.c_int32)]


class smm_info(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("p", C.c_int32), ("m", C.c_int32), ("n_dof_elem", C.c_int32),
                ("n_ord", C.c_int32), ("n_bface", C.c_int32), ("n_fq", C.c_int32), ("n_levels", C.c_int32),
                ("n_angular", C.c_int64), ("n_lagged", C.c_int64)]


class smm_stats(C.Structure):
    _fields_ = [("outer_iterations", C.c_int32), ("cg_total", C.c_int32), ("cg_min", C.c_int32),
                ("cg_max", C.c_int32), ("last_diff", C.c_double), ("last_rel_diff", C.c_double),
                ("ms_residual", C.c_double), ("ms_sweep", C.c_double), ("ms_moments", C.c_double),
                ("ms_rhs", C.c_double), ("ms_solve", C.c_double), ("n_launches", C.c_int64),
                ("guess_rejected", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SMMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str | None = None):
    """Load libsmm.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libsmm.so not found at {p}: run __graft_entry__.build() first")
    lib = C.CDLL(p)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    lib.smm_default_options.argtypes = [C.POINTER(smm_options)]
    lib.smm_default_options.restype = None
    lib.smm_last_error.restype = C.c_char_p
    lib.smm_quadrature.argtypes = [C.c_int32, dp, dp, ip]
    lib.smm_create.argtypes = [C.POINTER(smm_mesh), C.c_int32, C.c_int32, dp, dp, C.c_int32, dp, C.c_int32, dp,
                               C.POINTER(smm_options), vp, C.POINTER(vp)]
    lib.smm_get_info.argtypes = [vp, C.POINTER(smm_info)]
    lib.smm_sweep.argtypes = [vp, vp, vp]
    lib.smm_moments.argtypes = [vp, vp, vp]
    lib.smm_set_moments.argtypes = [vp, vp, vp]
    lib.smm_get_psi.argtypes = [vp, vp]
    lib.smm_moment_solve.argtypes = [vp, vp, ip]
    lib.smm_iterate.argtypes = [vp, C.c_double, C.c_int32, C.c_int32, vp, C.POINTER(smm_stats)]
    lib.smm_destroy.argtypes = [vp]
    lib.smm_set_spin_timeout.argtypes = [vp, C.c_double]
    lib.smm_state_size.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.smm_get_state.argtypes = [vp, vp, C.c_int64]
    lib.smm_set_state.argtypes = [vp, vp, C.c_int64]
    lib.smm_batch_create.argtypes = [C.c_int32, C.POINTER(vp), C.POINTER(vp)]
    lib.smm_batch_schedule.argtypes = [vp, ip, ip, dp, C.POINTER(C.c_int64)]
    lib.smm_batch_sweep.argtypes = [vp, C.POINTER(vp)]
    lib.smm_batch_iterate.argtypes = [vp, C.c_double, C.c_int32, C.c_int32, C.POINTER(vp), C.POINTER(smm_stats)]
    lib.smm_batch_destroy.argtypes = [vp]
    for name in ("smm_batch_create", "smm_batch_schedule", "smm_batch_sweep", "smm_batch_iterate", "smm_batch_destroy"):
        getattr(lib, name).restype = C.c_int
    fp = C.POINTER(C.c_float)
    lib.smm_guess_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, vp,
                                     C.POINTER(vp)]
    lib.smm_guess_num_params.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.smm_guess_forward.argtypes = [vp, C.c_int32, vp, vp]
    lib.smm_guess_train_step.argtypes = [vp, C.c_int32, vp, vp, C.c_float, fp]
    lib.smm_guess_gradients.argtypes = [vp, C.c_int32, vp, vp, fp, fp]
    lib.smm_guess_get_params.argtypes = [vp, fp]
    lib.smm_guess_set_params.argtypes = [vp, fp]
    lib.smm_guess_destroy.argtypes = [vp]
    for name in ("smm_guess_create", "smm_guess_num_params", "smm_guess_forward", "smm_guess_train_step",
                 "smm_guess_gradients", "smm_guess_get_params", "smm_guess_set_params", "smm_guess_destroy"):
        getattr(lib, name).restype = C.c_int
    lib.smm_block_pcg_noalloc.argtypes = [C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp, C.c_double, C.c_int32, vp, ip]
    lib.smm_block_pcg_noalloc.restype = C.c_int
    for name in ("smm_quadrature", "smm_create", "smm_get_info", "smm_sweep", "smm_moments", "smm_set_moments",
                 "smm_get_psi", "smm_moment_solve", "smm_iterate", "smm_destroy", "smm_state_size", "smm_get_state",
                 "smm_set_state", "smm_set_spin_timeout"):
        getattr(lib, name).restype = C.c_int
    if path is None:
        _lib = lib
    return lib


def _check(status):
    if status != SMM_OK:
        raise SMMError(status, load_library().smm_last_error().decode())
    return status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _devptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
        raise ValueError("device buffers must be contiguous CUDA float64 tensors")
    return C.c_void_p(t.data_ptr())


def _anybuf(t, count, what):
    """Pointer to a float64 buffer of exactly count elements in host memory (a
    C-contiguous NumPy array) or device memory (a CUDA tensor)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if t.dtype != np.float64 or not t.flags["C_CONTIGUOUS"] or not t.flags["WRITEABLE"]:
            raise ValueError(f"{what}: host buffers must be writeable C-contiguous float64 arrays")
        if t.size != count:
            raise ValueError(f"{what}: expected {count} elements, got {t.size}")
        return C.c_void_p(t.ctypes.data)
    return _devbuf(t, count, what)


def _rawbuf(buf):
    """(pointer, size in bytes) of a contiguous NumPy array or CUDA tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("state buffer must be contiguous")
        return C.c_void_p(buf.ctypes.data), buf.nbytes
    if not (buf.is_cuda and buf.is_contiguous()):
        raise ValueError("state buffer must be a contiguous CUDA tensor or a NumPy array")
    return C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size()


def _devbuf(t, count, what):
    """_devptr of a buffer that must hold exactly count elements: the C calls
    take plain pointers, so a short buffer would be read or written past its
    end on the device."""
    if t is None:
        return None
    ptr = _devptr(t)
    if t.numel() != count:
        raise ValueError(f"{what}: expected {count} elements, got {t.numel()}")
    return ptr


def smm_default_options() -> smm_options:
    o = smm_options()
    load_library().smm_default_options(C.byref(o))
    return o


def smm_quadrature(sn_order: int):
    """(omega [nd][2], weights [nd]) of the library's LQ_N set."""
    lib = load_library()
    nd = C.c_int32(0)
    _check(lib.smm_quadrature(sn_order, None, None, C.byref(nd)))
    om = np.zeros((nd.value, 2))
    w = np.zeros(nd.value)
    _check(lib.smm_quadrature(sn_order, _dptr(om), _dptr(w), C.byref(nd)))
    return om, w


class Handle:
    """Owns one smm_handle; methods mirror the C calls."""

    def __init__(self, ptr, stream_keepalive=None):
        self.ptr = ptr
        self._keep = stream_keepalive
        self._info = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.ptr:
            load_library().smm_destroy(self.ptr)
            self.ptr = None

    def info(self) -> smm_info:
        i = smm_info()
        _check(load_library().smm_get_info(self.ptr, C.byref(i)))
        return i

    def sizes(self) -> smm_info:
        """info(), fetched once (the sizes of a handle never change)."""
        if self._info is None:
            self._info = self.info()
        return self._info

    def n_phi(self) -> int:
        i = self.sizes()
        return i.n_elem * i.n_dof_elem


def smm_create(nodes, elem_nodes, geom_order, p, sn_order, sigma_t, sigma_s, q, source_kind=None,
               inflow=None, options: smm_options | None = None, stream=None) -> Handle:
    """Build a solver.  nodes [n_nodes][2], elem_nodes [n_elem][(m+1)^2],
    sigma_t/sigma_s [n_elem], q [n_elem][n] (isotropic) or [n_ord][n_elem][n],
    inflow None or [n_ord][n_bface][p+1]; stream: a torch.cuda.Stream or None
    (torch's current stream)."""
    import torch

    lib = load_library()
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    en = np.ascontiguousarray(elem_nodes, dtype=np.int32)
    st = np.ascontiguousarray(sigma_t, dtype=np.float64)
    ss = np.ascontiguousarray(sigma_s, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if source_kind is None:
        source_kind = SMM_SOURCE_ANGULAR if q.ndim == 3 else SMM_SOURCE_ISOTROPIC
    mesh = smm_mesh(len(en), geom_order, len(nodes), _dptr(nodes), en.ctypes.data_as(C.POINTER(C.c_int32)))
    ik = SMM_INFLOW_VACUUM
    inf_ptr = None
    if inflow is not None:
        inflow = np.ascontiguousarray(inflow, dtype=np.float64)
        ik = SMM_INFLOW_NODAL
        inf_ptr = _dptr(inflow)
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_void_p()
    _check(lib.smm_create(C.byref(mesh), p, sn_order, _dptr(st), _dptr(ss), source_kind, _dptr(q), ik, inf_ptr,
                          C.byref(options) if options is not None else None, C.c_void_p(s.cuda_stream),
                          C.byref(out)))
    return Handle(out, s)


def smm_sweep(h: Handle, phi=None, phi_t=None):
    """One sweep from varphi = phi (None: zero); phi_t (None, a CUDA float64
    tensor or a float64 NumPy array of n_elem * n values) receives phi_T."""
    _check(load_library().smm_sweep(h.ptr, _devbuf(phi, h.n_phi(), "phi"), _anybuf(phi_t, h.n_phi(), "phi_t")))


def _moment_bufs(h: Handle, moments, beta):
    i = h.sizes()
    return (_devbuf(moments, 6 * i.n_elem * i.n_dof_elem, "moments"),
            _devbuf(beta, i.n_bface * i.n_fq, "beta"))


def smm_moments(h: Handle, moments=None, beta=None):
    _check(load_library().smm_moments(h.ptr, *_moment_bufs(h, moments, beta)))


def smm_set_moments(h: Handle, moments, beta=None):
    _check(load_library().smm_set_moments(h.ptr, *_moment_bufs(h, moments, beta)))


def smm_get_psi(h: Handle, psi):
    _check(load_library().smm_get_psi(h.ptr, _devbuf(psi, h.sizes().n_angular, "psi")))


def smm_moment_solve(h: Handle, phi) -> int:
    it = C.c_int32(0)
    _check(load_library().smm_moment_solve(h.ptr, _devbuf(phi, h.n_phi(), "phi"), C.byref(it)))
    return it.value


def smm_iterate(h: Handle, phi, tol: float, max_outer: int = 200, relative: bool = False, raise_on_error=True):
    """phi: CUDA float64 tensor or float64 NumPy array (guess in, last iterate
    out).  Returns (status, stats dict)."""
    st = smm_stats()
    rc = load_library().smm_iterate(h.ptr, tol, int(relative), max_outer, _anybuf(phi, h.n_phi(), "phi"),
                                    C.byref(st))
    if raise_on_error:
        _check(rc)
    return rc, st.as_dict()


def smm_destroy(h: Handle):
    h.destroy()


def smm_set_spin_timeout(h: Handle, seconds: float):
    _check(load_library().smm_set_spin_timeout(h.ptr, seconds))


def smm_state_size(h: Handle) -> int:
    n = C.c_int64(0)
    _check(load_library().smm_state_size(h.ptr, C.byref(n)))
    return n.value


def smm_get_state(h: Handle, buf=None):
    """Save the handle's state into buf (a uint8 NumPy array or CUDA tensor of
    at least smm_state_size bytes); with buf None a new NumPy array is
    returned."""
    n = smm_state_size(h)
    if buf is None:
        buf = np.zeros(n, dtype=np.uint8)
    ptr, size = _rawbuf(buf)
    _check(load_library().smm_get_state(h.ptr, ptr, size))
    return buf


def smm_set_state(h: Handle, buf):
    ptr, size = _rawbuf(buf)
    _check(load_library().smm_set_state(h.ptr, ptr, size))


def smm_block_pcg_noalloc(diag_blocks, off_blocks, nbr, pinv_blocks, b, x, tol=1e-12, max_iters=20000,
                          stream=None) -> int:
    """Allocation-free block-Jacobi PCG (see include/smm.h).  Blocks are CUDA
    float64 tensors [n_elem][n][n] / [n_elem][4][n][n], column-major per block;
    nbr a CUDA int32 tensor [n_elem][4]; b, x CUDA float64 [n_elem*n]."""
    import torch

    n_elem, n = int(diag_blocks.shape[0]), int(diag_blocks.shape[1])
    if not (nbr.is_cuda and nbr.is_contiguous() and nbr.dtype == torch.int32):
        raise ValueError("nbr must be a contiguous CUDA int32 tensor")
    if nbr.numel() != 4 * n_elem:
        raise ValueError(f"nbr: expected {4 * n_elem} elements, got {nbr.numel()}")
    ptrs = (_devbuf(diag_blocks, n_elem * n * n, "diag_blocks"), _devbuf(off_blocks, 4 * n_elem * n * n, "off_blocks"),
            C.c_void_p(nbr.data_ptr()), _devbuf(pinv_blocks, n_elem * n * n, "pinv_blocks"),
            _devbuf(b, n_elem * n, "b"), _devbuf(x, n_elem * n, "x"))
    s = stream if stream is not None else torch.cuda.current_stream()
    it = C.c_int32(0)
    _check(load_library().smm_block_pcg_noalloc(n_elem, n, *ptrs, tol, max_iters, C.c_void_p(s.cuda_stream),
                                                C.byref(it)))
    return it.value


class Batch:
    """Owns an smm_batch; keeps its problems' handles alive."""

    def __init__(self, ptr, handles):
        self.ptr = ptr
        self.handles = list(handles)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.ptr:
            load_library().smm_batch_destroy(self.ptr)
            self.ptr = None

    def schedule(self):
        g, b, n = C.c_int32(0), C.c_int32(0), C.c_int64(0)
        ms = C.c_double(0.0)
        _check(load_library().smm_batch_schedule(self.ptr, C.byref(g), C.byref(b), C.byref(ms), C.byref(n)))
        return dict(grid=g.value, block=b.value, tuned_ms=ms.value, n_tasks=n.value)


def _ptr_array(handles, tensors):
    if len(tensors) != len(handles):
        raise ValueError(f"expected {len(handles)} buffers, got {len(tensors)}")
    arr = (C.c_void_p * len(tensors))()
    for i, (h, t) in enumerate(zip(handles, tensors)):
        arr[i] = None if t is None else _devbuf(t, h.n_phi(), "phi[%d]" % i).value
    return arr


def smm_batch_create(handles) -> Batch:
    arr = (C.c_void_p * len(handles))(*[h.ptr.value if isinstance(h.ptr, C.c_void_p) else h.ptr for h in handles])
    out = C.c_void_p()
    _check(load_library().smm_batch_create(len(handles), arr, C.byref(out)))
    return Batch(out, handles)


def smm_batch_sweep(b: Batch, phis=None):
    arr = _ptr_array(b.handles, phis if phis is not None else [None] * len(b.handles))
    _check(load_library().smm_batch_sweep(b.ptr, arr))


def smm_batch_iterate(b: Batch, phis, tol: float, max_outer: int = 200, relative: bool = False):
    arr = _ptr_array(b.handles, phis)
    st = (smm_stats * len(phis))()
    rc = load_library().smm_batch_iterate(b.ptr, tol, int(relative), max_outer, arr, st)
    _check(rc)
    return [s.as_dict() for s in st]


def _fdev(t, count=None, what="buffer"):
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"):
        raise ValueError("network buffers must be contiguous CUDA float32 tensors")
    if count is not None and t.numel() != count:
        raise ValueError(f"{what}: expected {count} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Guess:
    """Owns an smm_guess network; methods mirror the C calls."""

    def __init__(self, height, width, n_out, max_batch, seed=0, stream=None, c1=24, c2=32):
        import torch

        self.shape = (height, width, n_out)
        self.widths = (c1, c2)
        self.max_batch = max_batch
        s = stream if stream is not None else torch.cuda.current_stream()
        self._stream = s
        self.ptr = C.c_void_p()
        _check(load_library().smm_guess_create(height, width, n_out, c1, c2, max_batch, seed,
                                               C.c_void_p(s.cuda_stream), C.byref(self.ptr)))
        n = C.c_int64(0)
        _check(load_library().smm_guess_num_params(self.ptr, C.byref(n)))
        self.n_params = n.value

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.ptr:
            load_library().smm_guess_destroy(self.ptr)
            self.ptr = None

    def _io(self, x, y, what):
        """(batch, input pointer, output/target pointer): inputs [batch][3][H][W],
        outputs and targets [batch][n_out][H][W], batch <= max_batch."""
        h, w, n_out = self.shape
        batch = int(x.shape[0])
        if not 0 < batch <= self.max_batch:
            raise ValueError(f"batch {batch} outside 1..{self.max_batch}")
        return batch, _fdev(x, batch * 3 * h * w, "inputs"), _fdev(y, batch * n_out * h * w, what)

    def forward(self, x, out):
        _check(load_library().smm_guess_forward(self.ptr, *self._io(x, out, "outputs")))

    def train_step(self, x, target, lr):
        loss = C.c_float(0.0)
        _check(load_library().smm_guess_train_step(self.ptr, *self._io(x, target, "targets"), lr, C.byref(loss)))
        return loss.value

    def gradients(self, x, target):
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_float(0.0)
        _check(load_library().smm_guess_gradients(self.ptr, *self._io(x, target, "targets"),
                                                  g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
        return loss.value, g

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(load_library().smm_guess_get_params(self.ptr, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"params: expected {self.n_params} values, got {p.size}")
        _check(load_library().smm_guess_set_params(self.ptr, p.ctypes.data_as(C.POINTER(C.c_float))))
