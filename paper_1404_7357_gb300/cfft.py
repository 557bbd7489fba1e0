"""ctypes binding of libcfft.so (include/cfft.h), argument marshalling only.

Every method maps to one C entry point of the same name.  Device buffers are
torch CUDA tensors (PyTorch supplies device memory and streams); host buffers
are numpy arrays.  No part of the method runs here: a missing or unloadable
library raises ``CfftLibraryError`` at import time.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcfft.so")

CFFT_FP64 = 0
CFFT_FP32_MIXED = 1
(OPT_N_ALPHA, OPT_SIGMA, OPT_BP_TAPS, OPT_FILL_TAPS, OPT_ALPHA_MARGIN, OPT_CHECK_FINITE,
 OPT_DERIVATIVES, OPT_BP_GATHER, OPT_FILL_BLOCK, OPT_SPECTRA_SIMT, OPT_BP_SIMT, OPT_FILL_SIMT,
 OPT_FILL_REFINE, OPT_CONTOUR_SERIES, OPT_BP_KERNEL, OPT_SOLVE_SIMT,
 OPT_FFT_SUB_LEN, OPT_SOLVE_GRID_PANEL) = range(18)
STATUS = {0: "CFFT_OK", 1: "CFFT_ERR_ARG", 2: "CFFT_ERR_STATE", 3: "CFFT_ERR_OOM",
          4: "CFFT_ERR_CUDA", 5: "CFFT_ERR_NUMERIC", 6: "CFFT_ERR_TIMEOUT"}

# every symbol include/cfft.h declares
EXPORTS = ["cfft_create", "cfft_destroy", "cfft_last_error", "cfft_set_substrate",
           "cfft_set_mbf_spectra_strip", "cfft_set_mbf_spectra", "cfft_build_contour",
           "cfft_set_option", "cfft_contour_series_order", "cfft_tabulate_reactions", "cfft_get_table",
           "cfft_copy_table",
           "cfft_fill_reduced_matrix", "cfft_fill_reduced_matrix_host", "cfft_get_info",
           "cfft_debug_buffer", "cfft_synchronize", "cfft_backproject_static",
           "cfft_get_derivative_table", "cfft_fill_backward", "cfft_tabulate_batch",
           "cfft_get_batch_info", "cfft_mbf_spectra", "cfft_selftest_bounded_wait", "cfft_load_table",
           "cfft_fill_backward_residual", "cfft_test_fail_allocation", "cfft_measure_peak",
           "cfft_reduced_excitation", "cfft_port_excitation", "cfft_port_currents", "cfft_solve_reduced",
           "cfft_get_solve_info", "cfft_tabulate_cartesian", "cfft_get_cartesian_table", "cfft_fill_cartesian",
           "cfft_set_green_extraction"]


class CfftLibraryError(ImportError):
    pass


class CfftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class BatchItem(ctypes.Structure):
    _fields_ = [("eps_r", ctypes.c_double), ("h", ctypes.c_double), ("k0", ctypes.c_double),
                ("n", ctypes.c_int), ("beta_max", ctypes.c_double), ("beta_p", ctypes.c_double),
                ("height", ctypes.c_double), ("taylor_order", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("ms_integrand", "ms_fft", "ms_backproject", "ms_graph",
                                                "work_subffts", "work_bp_nodes")] + \
               [(n, ctypes.c_int) for n in ("sub_len", "rchunk", "waves", "launches", "bp_tc", "captures")]


class Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("taylor_order", "n_alpha", "sigma", "fft_len", "sub_len", "grid_half", "bp_taps",
                 "fill_taps", "series", "classes", "n_pairs", "n_harm")] + \
               [(n, ctypes.c_double) for n in
                ("delta_s", "ms_contour", "ms_integrand", "ms_fft", "ms_backproject")] + \
               [(n, ctypes.c_int) for n in ("launches", "n_basis")] + \
               [(n, ctypes.c_double) for n in ("work_points", "work_subffts", "work_bp_nodes")] + \
               [(n, ctypes.c_int) for n in ("spectra_tc", "bp_form")] + \
               [(n, ctypes.c_double) for n in ("work_bp_macs", "work_bp_stencils")] + \
               [("fill_form", ctypes.c_int), ("fill_err_est", ctypes.c_double)] + \
               [(n, ctypes.c_int) for n in ("fill_refine", "fill_n_rho")] + \
               [(n, ctypes.c_double) for n in ("tc_flops_integrand", "tc_flops_backproject")] + \
               [("contour_series", ctypes.c_int), ("bp_kernel", ctypes.c_int)]


class CartesianInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("n_grid", "n_table", "taylor_order", "monomials", "complex128")] + \
               [(n, ctypes.c_double) for n in ("x0", "step", "rho_max", "ms")]


class SolveInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("ms_factor", "ms_solve", "residual")] + \
               [(n, ctypes.c_int) for n in ("n", "mode", "refinements", "panel_width", "update_tc",
                                          "cluster_panels", "panel_cluster")]


def _load():
    if not os.path.exists(LIB_PATH):
        raise CfftLibraryError("libcfft.so not built (run __graft_entry__.build()): %s" % LIB_PATH)
    try:
        lib = ctypes.CDLL(LIB_PATH)
    except OSError as e:
        raise CfftLibraryError("cannot load %s: %s" % (LIB_PATH, e))
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "cfft_create": ([ctypes.POINTER(P), I, P], I),
        "cfft_destroy": ([P], None),
        "cfft_last_error": ([P], ctypes.c_char_p),
        "cfft_set_substrate": ([P, D, D, D], I),
        "cfft_set_mbf_spectra_strip": ([P, D, D], I),
        "cfft_set_mbf_spectra": ([P, I, P, P, P, P, I, P], I),
        "cfft_build_contour": ([P, I, D, D, D, I], I),
        "cfft_set_option": ([P, I, D], I),
        "cfft_contour_series_order": ([D, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "cfft_tabulate_reactions": ([P, I, D, I, I, I], I),
        "cfft_get_table": ([P, ctypes.POINTER(P), ctypes.POINTER(L), ctypes.POINTER(I)], I),
        "cfft_copy_table": ([P, P, L, I], I),
        "cfft_fill_reduced_matrix": ([P, I, P, P, P, L, I], I),
        "cfft_fill_reduced_matrix_host": ([P, I, P, P, P, L, I], I),
        "cfft_get_info": ([P, ctypes.POINTER(Info)], I),
        "cfft_debug_buffer": ([P, ctypes.c_char_p, ctypes.POINTER(P), ctypes.POINTER(L)], I),
        "cfft_synchronize": ([P], I),
        "cfft_backproject_static": ([I, P, P, P, I, I, I, D, I, D, I, I, D, D, I], I),
        "cfft_get_derivative_table": ([P, I, ctypes.POINTER(P), ctypes.POINTER(L)], I),
        "cfft_fill_backward": ([P, I, P, P, P, L, I, P, P], I),
        "cfft_fill_backward_residual": ([P, I, P, P, P, P, I, P, P], I),
        "cfft_test_fail_allocation": ([I], None),
        "cfft_tabulate_batch": ([P, I, ctypes.POINTER(BatchItem), I, D, I, I, P, I], I),
        "cfft_get_batch_info": ([P, ctypes.POINTER(BatchInfo)], I),
        "cfft_mbf_spectra": ([P, I, P, P], I),
        "cfft_selftest_bounded_wait": ([P, ctypes.c_uint], I),
        "cfft_load_table": ([P, I, I, D, I, I, I, I, P, I], I),
        "cfft_measure_peak": ([I, I, I, ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "cfft_reduced_excitation": ([P, I, P, P, I], I),
        "cfft_port_excitation": ([P, I, I, P, P, I], I),
        "cfft_port_currents": ([P, I, I, P, P, I], I),
        "cfft_solve_reduced": ([P, I, P, L, P, P, I, I], I),
        "cfft_get_solve_info": ([P, ctypes.POINTER(SolveInfo)], I),
        "cfft_tabulate_cartesian": ([P, I, D, I, I], I),
        "cfft_get_cartesian_table": ([P, ctypes.POINTER(P), ctypes.POINTER(CartesianInfo)], I),
        "cfft_fill_cartesian": ([P, I, P, P, L, I], I),
        "cfft_set_green_extraction": ([P, I, D], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def lib():
    return _lib


def contour_series_order(x, precision, series_opt=0):
    """(series, order, transforms) of the contour factor that the automatic choice of
    cfft_tabulate_reactions takes for x = height * rho_max: series 0 Taylor, 1 Chebyshev
    (cfft_contour_series_order; host only, no device needed)."""
    s, o, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    st = _lib.cfft_contour_series_order(float(x), int(precision), int(series_opt), ctypes.byref(s),
                                        ctypes.byref(o), ctypes.byref(f))
    if st != 0:
        raise CfftError(st, "contour_series_order: x must be finite and >= 0, the precision valid, "
                            "and some order up to 64 must reach the bound")
    return s.value, o.value, f.value


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class _DeviceArray:
    """Zero-copy view of a borrowed device buffer for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


class Context:
    """One cfft_ctx on a CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device=0, stream=None):
        import torch
        self._torch = torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.device = device
        self._h = ctypes.c_void_p()
        st = _lib.cfft_create(ctypes.byref(self._h), int(device), ctypes.c_void_p(handle))
        if st != 0:
            raise CfftError(st, "cfft_create failed")

    def close(self):
        if self._h:
            _lib.cfft_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise CfftError(st, _lib.cfft_last_error(self._h).decode())

    # ---- problem description
    def set_substrate(self, eps_r, h, k0):
        self._check(_lib.cfft_set_substrate(self._h, eps_r, h, k0))

    def set_green_extraction(self, extract=True, eps_eff=0.0):
        """Tabulate Z^l: the slab's Green's function minus an effective homogeneous medium
        (eps_eff, default (eps_r + 1) / 2) and its image through the ground plane."""
        self._check(_lib.cfft_set_green_extraction(self._h, int(bool(extract)), float(eps_eff)))

    def set_mbf_spectra_strip(self, length, width):
        self._check(_lib.cfft_set_mbf_spectra_strip(self._h, length, width))
        self.n_mbf = 1

    def set_mbf_spectra(self, centers, direction, half_len, width, q):
        centers = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 2)
        direction = np.ascontiguousarray(direction, dtype=np.int32)
        half_len = np.ascontiguousarray(half_len, dtype=np.float64)
        width = np.ascontiguousarray(width, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.complex128)
        b, m = q.shape
        self._check(_lib.cfft_set_mbf_spectra(self._h, b, _ptr(centers), _ptr(direction),
                                              _ptr(half_len), _ptr(width), m, _ptr(q)))
        self.n_mbf = m

    def build_contour(self, n, beta_max, beta_p, height, taylor_order=-1):
        self._check(_lib.cfft_build_contour(self._h, n, beta_max, beta_p, height, taylor_order))

    def set_option(self, key, value):
        self._check(_lib.cfft_set_option(self._h, key, float(value)))

    def tabulate_reactions(self, q_max, rho_max, n_rho, precision, rotation_classes=1):
        self._table_desc = {"q_max": int(q_max), "rho_max": float(rho_max), "n_rho": int(n_rho),
                            "precision": int(precision), "rotation_classes": int(rotation_classes)}
        self._check(_lib.cfft_tabulate_reactions(self._h, q_max, rho_max, n_rho, precision,
                                                 rotation_classes))

    # ---- results
    def table_shape(self):
        ptr = ctypes.c_void_p()
        shape = (ctypes.c_int64 * 4)()
        is128 = ctypes.c_int()
        self._check(_lib.cfft_get_table(self._h, ctypes.byref(ptr), shape, ctypes.byref(is128)))
        return tuple(shape), bool(is128.value), ptr.value

    def get_table(self):
        """Borrowed zero-copy torch view of the context-owned table."""
        shape, is128, ptr = self.table_shape()
        return self._torch.as_tensor(_DeviceArray(ptr, shape, "<c16" if is128 else "<c8"),
                                     device="cuda:%d" % self.device)

    def copy_table(self, out=None, host=False):
        shape, is128, _ = self.table_shape()
        torch = self._torch
        dt = torch.complex128 if is128 else torch.complex64
        if out is None:
            out = (torch.empty(shape, dtype=dt, pin_memory=True) if host
                   else torch.empty(shape, dtype=dt, device="cuda:%d" % self.device))
        self._check(_lib.cfft_copy_table(self._h, ctypes.c_void_p(out.data_ptr()),
                                         out.numel() * out.element_size(), int(not out.is_cuda)))
        return out

    def _check_layout(self, pos, rot, z, device):
        """The fill's buffers as the C entry points read them: pos (A, 2) float64,
        rot (A,) int32 or None, z a complex64/complex128 matrix of at least A*M x A*M
        with unit column stride (rows ld = z's row stride apart)."""
        torch = self._torch

        def bad(msg):
            raise ValueError("fill arguments: " + msg)
        if pos.dtype not in (torch.float64, np.float64) or tuple(pos.shape)[1:] != (2,):
            bad("pos must be float64 of shape (A, 2)")
        a = int(pos.shape[0])
        n = a * int(getattr(self, "n_mbf", 0))      # no element yet: the library reports the state
        if rot is not None and (rot.dtype not in (torch.int32, np.int32) or tuple(rot.shape) != (a,)):
            bad("rot must be int32 of shape (A,)")
        if z.dtype not in (torch.complex64, torch.complex128, np.complex64, np.complex128):
            bad("the matrix must be complex64 or complex128")
        if len(z.shape) != 2 or z.shape[0] < n or z.shape[1] < n:
            bad("the matrix must be at least (A*M, A*M) = (%d, %d), got %s" % (n, n, tuple(z.shape)))
        for t in (pos, rot, z):
            if t is None:
                continue
            on_dev = bool(getattr(t, "is_cuda", False))
            if on_dev != device:
                bad("expected %s buffers" % ("CUDA" if device else "host"))
        if device:
            if not pos.is_contiguous() or (rot is not None and not rot.is_contiguous()) or z.stride(-1) != 1:
                bad("pos and rot must be contiguous and the matrix rows unit-stride")
        return a

    def fill_reduced_matrix(self, pos, rot, out):
        """pos: cuda float64 (A, 2); rot: cuda int32 (A,) or None; out: cuda complex (A*M, ld)."""
        torch = self._torch
        a = self._check_layout(pos, rot, out, device=True)
        self._check(_lib.cfft_fill_reduced_matrix(
            self._h, a, ctypes.c_void_p(pos.data_ptr()),
            ctypes.c_void_p(rot.data_ptr() if rot is not None else 0),
            ctypes.c_void_p(out.data_ptr()), out.stride(0), int(out.dtype == torch.complex128)))
        return out

    def fill_reduced_matrix_host(self, pos, rot, out):
        """Host variant: C-contiguous numpy arrays in and out (out rows may be padded)."""
        pos = np.ascontiguousarray(pos)
        rot = None if rot is None else np.ascontiguousarray(rot)
        a = self._check_layout(pos, rot, out, device=False)
        if not isinstance(out, np.ndarray) or out.strides[1] != out.itemsize or not out.flags.writeable:
            raise ValueError("fill arguments: out must be a writeable numpy matrix with unit-stride rows")
        self._check(_lib.cfft_fill_reduced_matrix_host(
            self._h, a, _ptr(pos), ctypes.c_void_p(rot.ctypes.data if rot is not None else 0),
            _ptr(out), out.strides[0] // out.itemsize, int(out.dtype == np.complex128)))
        return out

    def derivative_table(self, which):
        """Borrowed device view of the table (0) or its d/d eps_r (1), d/d h (2) companion."""
        ptr = ctypes.c_void_p()
        shape = (ctypes.c_int64 * 4)()
        self._check(_lib.cfft_get_derivative_table(self._h, which, ctypes.byref(ptr), shape))
        _, is128, _ = self.table_shape()
        return self._torch.as_tensor(_DeviceArray(ptr.value, tuple(shape), "<c16" if is128 else "<c8"),
                                     device="cuda:%d" % self.device)

    def fill_backward(self, pos, rot, grad_z, substrate=True):
        """Adjoint of the fill: (grad_pos (A, 2) float64, grad_eps_h (2,) float64 or None)."""
        torch = self._torch
        self._check_layout(pos, rot, grad_z, device=True)
        grad_pos = torch.empty_like(pos)
        g_th = torch.empty(2, dtype=torch.float64, device=pos.device) if substrate else None
        self._check(_lib.cfft_fill_backward(
            self._h, pos.shape[0], ctypes.c_void_p(pos.data_ptr()),
            ctypes.c_void_p(rot.data_ptr() if rot is not None else 0),
            ctypes.c_void_p(grad_z.data_ptr()), grad_z.stride(0),
            int(grad_z.dtype == torch.complex128), ctypes.c_void_p(grad_pos.data_ptr()),
            ctypes.c_void_p(g_th.data_ptr() if g_th is not None else 0)))
        return grad_pos, g_th

    def tabulate_batch(self, items, q_max, rho_max, n_rho, precision, out=None, graph=True,
                       autotune=False):
        """cfft_tabulate_batch over dict-like items (eps_r, h, k0, n, beta_max, beta_p, height,
        taylor_order); returns the (n_items, M*M, 2*q_max+1, n_rho) device tensor."""
        torch = self._torch
        arr = (BatchItem * len(items))()
        for i, it in enumerate(items):
            arr[i] = BatchItem(it["eps_r"], it["h"], it["k0"], int(it["n"]), it["beta_max"],
                               it["beta_p"], it["height"], int(it.get("taylor_order", -1)))
        m2 = self.n_mbf ** 2
        dt = torch.complex128 if precision == CFFT_FP64 else torch.complex64
        shape = (len(items), m2, 2 * q_max + 1, n_rho)
        if out is None:
            out = torch.empty(shape, dtype=dt, device="cuda:%d" % self.device)
        assert tuple(out.shape) == shape and out.dtype == dt and out.is_contiguous()
        self._check(_lib.cfft_tabulate_batch(self._h, len(items), arr, q_max, float(rho_max), n_rho,
                                             precision, ctypes.c_void_p(out.data_ptr()),
                                             int(graph) | (2 if autotune else 0)))
        return out

    def fill_backward_residual(self, pos, rot, v, resid, substrate=True):
        """Adjoint for L = sum |Z' v - t|^2 from v and r = Z' v - t (cuda complex vectors of
        A*M entries): (grad_pos (A, 2) float64, grad_eps_h (2,) float64 or None)."""
        torch = self._torch
        n = pos.shape[0] * int(getattr(self, "n_mbf", 0))
        for x in (v, resid):
            if not (x.is_cuda and x.dtype == resid.dtype and x.dtype in (torch.complex64, torch.complex128)
                    and x.is_contiguous() and x.numel() == n):
                raise ValueError("v and resid: contiguous CUDA complex vectors of A*M = %d entries, "
                                 "one dtype" % n)
        if not (pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous() and
                tuple(pos.shape[1:]) == (2,)):
            raise ValueError("pos must be a contiguous CUDA float64 tensor of shape (A, 2)")
        if rot is not None and not (rot.is_cuda and rot.dtype == torch.int32 and rot.is_contiguous() and
                                    tuple(rot.shape) == (pos.shape[0],)):
            raise ValueError("rot must be a contiguous CUDA int32 tensor of shape (A,)")
        grad_pos = torch.empty_like(pos)
        g_th = torch.empty(2, dtype=torch.float64, device=pos.device) if substrate else None
        self._check(_lib.cfft_fill_backward_residual(
            self._h, pos.shape[0], ctypes.c_void_p(pos.data_ptr()),
            ctypes.c_void_p(rot.data_ptr() if rot is not None else 0),
            ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(resid.data_ptr()),
            int(resid.dtype == torch.complex128), ctypes.c_void_p(grad_pos.data_ptr()),
            ctypes.c_void_p(g_th.data_ptr() if g_th is not None else 0)))
        return grad_pos, g_th

    def save_table(self, path):
        """Checkpoint: the current table as `path`.npy and its description as `path`.json."""
        import json
        import numpy as np
        desc = dict(self._table_desc)
        desc["n_mbf"] = int(self.n_mbf)
        desc["fill_taps"] = int(self.info()["fill_taps"])
        np.save(path + ".npy", self.copy_table(host=True).numpy())
        with open(path + ".json", "w") as f:
            json.dump(desc, f, indent=1)
        return desc

    def load_table(self, path):
        """Resume from save_table: the table is installed (cfft_load_table) and the fill
        runs without a tabulation."""
        import json
        import numpy as np
        with open(path + ".json") as f:
            d = json.load(f)
        t = np.ascontiguousarray(np.load(path + ".npy"))
        want = np.complex128 if d["precision"] == CFFT_FP64 else np.complex64
        assert t.dtype == want and t.shape == (d["rotation_classes"], d["n_mbf"] ** 2, 2 * d["q_max"] + 1,
                                               d["n_rho"])
        self._check(_lib.cfft_load_table(self._h, d["n_mbf"], d["q_max"], d["rho_max"], d["n_rho"],
                                         d["precision"], d["rotation_classes"], d["fill_taps"],
                                         ctypes.c_void_p(t.ctypes.data), 1))
        self.n_mbf = d["n_mbf"]
        self._table_desc = {k: d[k] for k in ("q_max", "rho_max", "n_rho", "precision", "rotation_classes")}
        return d

    def selftest_bounded_wait(self, polls=4096):
        """cfft_selftest_bounded_wait: a device-side wait that nothing ends runs out after
        `polls` tries; raises CfftError with status CFFT_ERR_TIMEOUT (the designed outcome)."""
        self._check(_lib.cfft_selftest_bounded_wait(self._h, ctypes.c_uint(polls)))

    def mbf_spectra(self, k, out=None):
        """cfft_mbf_spectra: k cuda complex64 (n, 2) wavevectors -> (n, 2 sides, M, 2 comps)
        complex64 MBF spectra (side 0: Eq. 11; side 1: the conjugated continuation)."""
        torch = self._torch
        if not (k.is_cuda and k.dtype == torch.complex64 and k.is_contiguous() and k.dim() == 2 and
                k.shape[1] == 2):
            raise ValueError("k must be a contiguous CUDA complex64 tensor of shape (n, 2)")
        n = k.shape[0]
        shape = (n, 2, int(getattr(self, "n_mbf", 1)), 2)   # no element yet: the library refuses
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device=k.device)
        if not (out.is_cuda and tuple(out.shape) == shape and out.dtype == torch.complex64 and
                out.is_contiguous()):
            raise ValueError("out must be a contiguous CUDA complex64 tensor of shape %s" % (shape,))
        self._check(_lib.cfft_mbf_spectra(self._h, n, ctypes.c_void_p(k.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr())))
        return out

    def batch_info(self):
        inf = BatchInfo()
        self._check(_lib.cfft_get_batch_info(self._h, ctypes.byref(inf)))
        return {n: getattr(inf, n) for n, _ in BatchInfo._fields_}

    def info(self):
        inf = Info()
        self._check(_lib.cfft_get_info(self._h, ctypes.byref(inf)))
        return {n: getattr(inf, n) for n, _ in Info._fields_}

    def debug_buffer(self, name):
        """Copy of an intermediate device buffer ("harmonics", "grid", "contour")."""
        ptr = ctypes.c_void_p()
        shape = (ctypes.c_int64 * 4)()
        self._check(_lib.cfft_debug_buffer(self._h, name.encode(), ctypes.byref(ptr), shape))
        _, is128, _ = self.table_shape()
        ts = "<c16" if (is128 or name == "contour") else "<c8"
        view = self._torch.as_tensor(_DeviceArray(ptr.value, tuple(shape), ts),
                                     device="cuda:%d" % self.device)
        return view.clone()

    def synchronize(self):
        self._check(_lib.cfft_synchronize(self._h))

    # ---- reduced system (Section II): excitation, direct solution, port currents

    def _vec(self, t, name, n=None):
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype in (torch.complex64, torch.complex128)
                and t.is_contiguous()):
            raise ValueError("%s: a contiguous complex CUDA tensor" % name)
        if n is not None and t.numel() != n:
            raise ValueError("%s: %d entries expected, got %d" % (name, n, t.numel()))
        return int(t.dtype == torch.complex128)

    def reduced_excitation(self, v):
        """V' = Q^H V_m per element (Eq. 4): v (A, n_basis) complex CUDA -> (A * M,)."""
        if v.dim() != 2:
            raise ValueError("v: (n_elements, n_basis)")
        c128 = self._vec(v, "v")
        out = self._torch.empty(v.shape[0] * self.n_mbf, dtype=v.dtype, device=v.device)
        self._check(_lib.cfft_reduced_excitation(self._h, v.shape[0], ctypes.c_void_p(v.data_ptr()),
                                                 ctypes.c_void_p(out.data_ptr()), c128))
        return out

    def port_excitation(self, port, amplitudes):
        """V' of delta-gap ports across basis function `port`: amplitudes (A,) -> (A * M,)."""
        c128 = self._vec(amplitudes, "amplitudes")
        a = amplitudes.numel()
        out = self._torch.empty(a * self.n_mbf, dtype=amplitudes.dtype, device=amplitudes.device)
        self._check(_lib.cfft_port_excitation(self._h, a, int(port), ctypes.c_void_p(amplitudes.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()), c128))
        return out

    def port_currents(self, port, i_red):
        """(Q I'_m)[port] for every element: i_red (A * M,) -> (A,)."""
        c128 = self._vec(i_red, "i_red")
        if i_red.numel() % self.n_mbf:
            raise ValueError("i_red: a multiple of M entries")
        a = i_red.numel() // self.n_mbf
        out = self._torch.empty(a, dtype=i_red.dtype, device=i_red.device)
        self._check(_lib.cfft_port_currents(self._h, a, int(port), ctypes.c_void_p(i_red.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), c128))
        return out

    def solve_reduced(self, z, v, refine=False):
        """I' with Z' I' = V' (dense LU with partial pivoting on the GPU): z (n, ld >= n) complex
        CUDA with unit-stride rows (not modified), v (n,).  refine: complex128 z factored in
        complex64 and refined in float64."""
        torch = self._torch
        if not (isinstance(z, torch.Tensor) and z.is_cuda and z.dim() == 2 and z.stride(1) == 1 and
                z.shape[1] >= z.shape[0] and z.dtype in (torch.complex64, torch.complex128)):
            raise ValueError("z: complex CUDA matrix (n, >= n) with unit-stride rows")
        n = z.shape[0]
        c128 = self._vec(v, "v", n)
        if v.dtype != z.dtype:
            raise ValueError("z and v: the same dtype")
        out = torch.empty(n, dtype=z.dtype, device=z.device)
        self._check(_lib.cfft_solve_reduced(self._h, n, ctypes.c_void_p(z.data_ptr()), z.stride(0),
                                            ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            c128, 1 if refine else 0))
        return out

    # ---- the paper's 2-D Cartesian C-FFT (Eq. 21-24, Appendix I)

    def tabulate_cartesian(self, n_grid, rho_max, precision, taylor_order=-1):
        self._check(_lib.cfft_tabulate_cartesian(self._h, int(n_grid), float(rho_max), int(taylor_order),
                                                 precision))
        return self.cartesian_info()

    def cartesian_info(self):
        ptr = ctypes.c_void_p()
        inf = CartesianInfo()
        self._check(_lib.cfft_get_cartesian_table(self._h, ctypes.byref(ptr), ctypes.byref(inf)))
        return {n: getattr(inf, n) for n, _ in CartesianInfo._fields_}

    def cartesian_table(self):
        """Copy of the Cartesian table: (M*M, 2 n_grid, 2 n_grid) complex CUDA tensor, axis 1 = dx."""
        ptr = ctypes.c_void_p()
        inf = CartesianInfo()
        self._check(_lib.cfft_get_cartesian_table(self._h, ctypes.byref(ptr), ctypes.byref(inf)))
        shape = (self.n_mbf * self.n_mbf, inf.n_table, inf.n_table)
        view = _DeviceArray(ptr.value, shape, "<c16" if inf.complex128 else "<c8")
        return self._torch.as_tensor(view, device="cuda:%d" % self.device).clone()

    def fill_cartesian(self, pos, out):
        """Reduced matrix of unrotated elements from the Cartesian table (second-order
        interpolation): pos cuda float64 (A, 2), out cuda complex (A*M, ld)."""
        torch = self._torch
        a = self._check_layout(pos, None, out, device=True)
        self._check(_lib.cfft_fill_cartesian(self._h, a, ctypes.c_void_p(pos.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                             int(out.dtype == torch.complex128)))
        return out

    def solve_info(self):
        inf = SolveInfo()
        self._check(_lib.cfft_get_solve_info(self._h, ctypes.byref(inf)))
        return {n: getattr(inf, n) for n, _ in SolveInfo._fields_}


def test_fail_allocation(after):
    """cfft_test_fail_allocation: after `after` successful device allocations the next one
    fails as out of memory (host-side injection; after < 0 disarms)."""
    _lib.cfft_test_fail_allocation(int(after))


PEAK_FP32, PEAK_FP64, PEAK_TF32, PEAK_BF16 = range(4)


def measure_peak(device, which, reps=5):
    """cfft_measure_peak: (TFLOP/s, ms) of the best of ``reps`` timed launches of the
    microbenchmark ``which`` (PEAK_FP32, PEAK_FP64 FMA pipes; PEAK_TF32, PEAK_BF16 tensor
    cores) on CUDA device ``device``."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    st = _lib.cfft_measure_peak(int(device), int(which), int(reps), ctypes.byref(tf), ctypes.byref(ms))
    if st != 0:
        raise CfftError(st, "cfft_measure_peak failed")
    return tf.value, ms.value


def backproject_static(grid, table, series_per_q, q_max, rho_max, grid_half, delta_s, sigma, taps,
                       beta_abs_max, alpha_margin=24.0, stream=None):
    """cfft_backproject_static: back-project a transform grid (torch CUDA tensor, layout of
    Context.debug_buffer("grid")) into ``table`` (torch CUDA tensor [series, n_rho]) without
    any device allocation by the library.  Queued on ``stream`` (default: torch's current)."""
    import torch
    dev = grid.device.index or 0
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if not (grid.is_cuda and table.is_cuda and grid.dtype == table.dtype and
            grid.dtype in (torch.complex64, torch.complex128)):
        raise ValueError("grid and table: CUDA tensors of one complex dtype")
    if not (grid.is_contiguous() and table.is_contiguous()):
        raise ValueError("grid and table must be contiguous")
    series = series_per_q * (2 * q_max + 1)
    n_rho = table.shape[-1]
    if grid.numel() != series * (2 * grid_half + 1) or table.numel() != series * n_rho:
        raise ValueError("grid must hold [series][2*grid_half+1] and table [series][n_rho], "
                         "series = series_per_q * (2*q_max+1) = %d" % series)
    st = _lib.cfft_backproject_static(dev, ctypes.c_void_p(handle), ctypes.c_void_p(grid.data_ptr()),
                                      ctypes.c_void_p(table.data_ptr()), series_per_q, q_max, n_rho,
                                      float(rho_max), grid_half, float(delta_s), sigma, taps,
                                      float(beta_abs_max), float(alpha_margin),
                                      int(grid.dtype == torch.complex128))
    if st != 0:
        raise CfftError(st, "cfft_backproject_static rejected the request or failed")
    return table
