"""Thin ctypes binding of the C ABI in include/tbs.h.

Functions carry the C names (``tbs_plan``, ``tbs_set_medium``, ...) and take
plain integers for device pointers and the stream, exactly as the C calls do;
``Plan`` adds torch-tensor marshalling on top (data_ptr, current stream).
Every step of the Born series runs in libtbs.so: this module only marshals
arguments and raises on error codes.  There is no CPU fallback: if the
library is not built, importing the binding fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libtbs.so")

TBS_OK = 0
STATUS_NAMES = {0: "CONVERGED", 1: "MAX_TERMS", 2: "DIVERGED", 3: "NONFINITE", 4: "WAIT_TIMEOUT",
                5: "COPY_CHECK_FAILED"}
TBS_STOP_L2, TBS_STOP_L1_ROW = 0, 1
TBS_FLAG_KEEP_TERMS, TBS_FLAG_NO_GRAPH = 1, 2
TBS_FLAG_CHECKPOINT_TERMS = 1 << 2
TBS_FLAG_PERIODIC = 1 << 3
TBS_FLAG_KSPACE_ABSORPTION = 1 << 4
TBS_FLAG_CBS = 1 << 5
TBS_MAX_N = 2048

# every symbol include/tbs.h declares
EXPORTED = [
    "tbs_plan_desc_init", "tbs_plan", "tbs_plan_with_workspace", "tbs_plan_device_bytes", "tbs_plan_padded_size",
    "tbs_set_medium", "tbs_set_potential", "tbs_set_sources", "tbs_set_source_field",
    "tbs_set_harmonic2_source", "tbs_set_harmonic_source", "tbs_solve", "tbs_solve_adjoint", "tbs_apply_green",
    "tbs_get_ghat", "tbs_set_timing", "tbs_get_timing", "tbs_destroy", "tbs_status_string",
    "tbs_last_error", "tbs_apply_green_noalloc", "tbs_batch_create", "tbs_batch_solve",
    "tbs_batch_destroy", "tbs_debug_set", "tbs_col_variants", "tbs_set_col_variant", "tbs_autotune",
    "tbs_synthesize", "tbs_potential_max_abs", "tbs_plan_eps", "tbs_device_error", "tbs_col_variant_name",
    "tbs_row_variants", "tbs_row_variant_name", "tbs_set_row_variant", "tbs_autotune_rows",
]
TBS_DEBUG_WAIT_LIMIT_NS, TBS_DEBUG_EXTRA_TX = 1, 2
TBS_WAIT_TIMEOUT, TBS_COPY_CHECK_FAILED = 4, 5
TBS_NOALLOC_MAX_N = 256


class TbsError(RuntimeError):
    def __init__(self, call, code, msg):
        super().__init__("%s -> %s: %s" % (call, _status_name(code), msg))
        self.code = code


class tbs_plan_desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_rhs", C.c_int32), ("dx", C.c_double),
                ("freq_hz", C.c_double), ("c0", C.c_double), ("max_terms", C.c_int32),
                ("tol", C.c_double), ("stop_mode", C.c_int32), ("l1_row", C.c_int32),
                ("div_grace", C.c_int32), ("div_window", C.c_int32),
                ("div_factor", C.c_double), ("flags", C.c_uint32),
                ("eps_factor", C.c_double), ("abl_width", C.c_int32), ("abl_zeta", C.c_double),
                ("kspace_alpha0", C.c_double), ("kspace_nu", C.c_double),
                ("kspace_absorption_only", C.c_int32)]


class tbs_synth_freq(C.Structure):
    _fields_ = [("field", C.c_void_p), ("n", C.c_int32), ("dx", C.c_double), ("freq_hz", C.c_double),
                ("weight", C.c_double)]


class tbs_solve_info(C.Structure):
    _fields_ = [("terms", C.c_int32), ("status", C.c_int32), ("residual", C.c_double),
                ("term_norm_max", C.c_double), ("psi_norm", C.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtbs.so (built by ``paper_2507_13754_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libtbs.so not found at %s: build it with "
                           "paper_2507_13754_gb300.build.build() (needs nvcc)" % path)
    lib = C.CDLL(path)
    P, I32, D, U32 = C.c_void_p, C.c_int32, C.c_double, C.c_uint32
    st = C.c_int
    sig = {
        "tbs_plan_desc_init": (None, [C.POINTER(tbs_plan_desc)]),
        "tbs_plan": (st, [C.POINTER(tbs_plan_desc), P, C.POINTER(P)]),
        "tbs_plan_with_workspace": (st, [C.POINTER(tbs_plan_desc), P, C.c_size_t, P, C.POINTER(P)]),
        "tbs_plan_device_bytes": (st, [C.POINTER(tbs_plan_desc), C.POINTER(C.c_size_t)]),
        "tbs_plan_padded_size": (I32, [P]),
        "tbs_set_medium": (st, [P, P, P, D, D, P]),
        "tbs_set_potential": (st, [P, P, P]),
        "tbs_set_sources": (st, [P, I32, P, P, P, P]),
        "tbs_set_source_field": (st, [P, P, P]),
        "tbs_set_harmonic2_source": (st, [P, P, P, P, P, D, P]),
        "tbs_set_harmonic_source": (st, [P, I32, C.POINTER(P), C.POINTER(D), P, P, P, D, D, P]),
        "tbs_solve": (st, [P, P, P, P]),
        "tbs_solve_adjoint": (st, [P, P, P, P, P]),
        "tbs_apply_green": (st, [P, P, P, I32, P]),
        "tbs_get_ghat": (st, [P, P]),
        "tbs_set_timing": (st, [P, I32]),
        "tbs_get_timing": (st, [P, C.POINTER(D), C.POINTER(I32), C.POINTER(D), C.POINTER(I32)]),
        "tbs_destroy": (st, [P]),
        "tbs_status_string": (C.c_char_p, [st]),
        "tbs_last_error": (C.c_char_p, []),
        "tbs_apply_green_noalloc": (st, [I32, P, P, P, I32, P]),
        "tbs_batch_create": (st, [C.POINTER(P), I32, C.POINTER(P), C.POINTER(P), C.POINTER(P)]),
        "tbs_batch_solve": (st, [P, P]),
        "tbs_batch_destroy": (st, [P]),
        "tbs_debug_set": (st, [P, I32, C.c_int64]),
        "tbs_col_variants": (I32, [P]),
        "tbs_set_col_variant": (st, [P, I32]),
        "tbs_autotune": (st, [P, I32, C.POINTER(D), C.POINTER(I32), P]),
        "tbs_synthesize": (st, [C.POINTER(tbs_synth_freq), I32, I32, D, D, D, D, I32, I32, D, D, I32, P, P]),
        "tbs_potential_max_abs": (st, [P, C.POINTER(D), P]),
        "tbs_plan_eps": (D, [P]),
        "tbs_device_error": (st, [P, C.POINTER(I32), P]),
        "tbs_col_variant_name": (C.c_char_p, [P, I32]),
        "tbs_row_variants": (I32, [P]),
        "tbs_row_variant_name": (C.c_char_p, [P, I32]),
        "tbs_set_row_variant": (st, [P, I32]),
        "tbs_autotune_rows": (st, [P, I32, C.POINTER(D), C.POINTER(I32), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _status_name(code):
    try:
        return load_library().tbs_status_string(code).decode()
    except Exception:
        return str(code)


def _check(call, code):
    if code != TBS_OK:
        raise TbsError(call, code, load_library().tbs_last_error().decode())


# ---- C-named wrappers (pointer/int arguments) ------------------------------

def tbs_plan_desc_init() -> tbs_plan_desc:
    d = tbs_plan_desc()
    load_library().tbs_plan_desc_init(C.byref(d))
    return d


def tbs_plan(desc: tbs_plan_desc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check("tbs_plan", load_library().tbs_plan(C.byref(desc), stream, C.byref(h)))
    return h.value


def tbs_plan_with_workspace(desc: tbs_plan_desc, workspace: int, workspace_bytes: int, stream: int = 0) -> int:
    h = C.c_void_p()
    _check("tbs_plan_with_workspace",
           load_library().tbs_plan_with_workspace(C.byref(desc), workspace, workspace_bytes, stream, C.byref(h)))
    return h.value


def tbs_plan_device_bytes(desc: tbs_plan_desc) -> int:
    b = C.c_size_t()
    _check("tbs_plan_device_bytes", load_library().tbs_plan_device_bytes(C.byref(desc), C.byref(b)))
    return b.value


def tbs_plan_padded_size(plan: int) -> int:
    return int(load_library().tbs_plan_padded_size(plan))


def tbs_set_medium(plan, c_ptr, alpha_ptr, y_pow, f_ref_hz, stream=0):
    _check("tbs_set_medium", load_library().tbs_set_medium(plan, c_ptr, alpha_ptr or None,
                                                            y_pow, f_ref_hz, stream))


def tbs_set_potential(plan, v_ptr, stream=0):
    _check("tbs_set_potential", load_library().tbs_set_potential(plan, v_ptr, stream))


def tbs_set_sources(plan, n_pts, ix_host, iy_host, amp_host, stream=0):
    _check("tbs_set_sources", load_library().tbs_set_sources(plan, n_pts, ix_host, iy_host,
                                                              amp_host, stream))


def tbs_set_source_field(plan, s_ptr, stream=0):
    _check("tbs_set_source_field", load_library().tbs_set_source_field(plan, s_ptr, stream))


def tbs_set_harmonic_source(plan, order, psi_ptrs, beta_ptr, rho_ptr, c_ptr, omega, stream=0, psi_scale=None,
                            source_scale=1.0):
    arr = (C.c_void_p * len(psi_ptrs))(*psi_ptrs)
    sc = None if psi_scale is None else (C.c_double * len(psi_ptrs))(*psi_scale)
    _check("tbs_set_harmonic_source", load_library().tbs_set_harmonic_source(
        plan, order, arr, sc, beta_ptr, rho_ptr, c_ptr, omega, source_scale, stream))


def tbs_set_harmonic2_source(plan, psi1_ptr, beta_ptr, rho_ptr, c_ptr, omega, stream=0):
    _check("tbs_set_harmonic2_source", load_library().tbs_set_harmonic2_source(
        plan, psi1_ptr, beta_ptr, rho_ptr, c_ptr, omega, stream))


def tbs_solve(plan, psi_ptr, info_ptr, stream=0):
    _check("tbs_solve", load_library().tbs_solve(plan, psi_ptr, info_ptr, stream))


def tbs_solve_adjoint(plan, grad_psi_ptr, grad_c_ptr, grad_alpha_ptr, stream=0):
    _check("tbs_solve_adjoint", load_library().tbs_solve_adjoint(
        plan, grad_psi_ptr, grad_c_ptr or None, grad_alpha_ptr or None, stream))


def tbs_apply_green(plan, f_ptr, out_ptr, conj_kernel=0, stream=0):
    _check("tbs_apply_green", load_library().tbs_apply_green(plan, f_ptr, out_ptr,
                                                              int(conj_kernel), stream))


def tbs_apply_green_noalloc(n, ghat_ptr, f_ptr, out_ptr, conj_kernel=0, stream=0):
    """out = G f (or G^H f) for one n x n field with no device allocation:
    the library's fixed scratch array replaces plan buffers (n <= 256)."""
    _check("tbs_apply_green_noalloc", load_library().tbs_apply_green_noalloc(
        n, ghat_ptr, f_ptr, out_ptr, int(conj_kernel), stream))


def tbs_synthesize(entries, n_rhs, x0, y0, sx, sy, nx, ny, t0, dt, n_t, out_ptr, stream=0):
    """entries: [(field_ptr, n, dx, freq_hz, weight)]; out [n_rhs][ny][nx][n_t] complex64."""
    arr = (tbs_synth_freq * len(entries))(*[tbs_synth_freq(*e) for e in entries])
    _check("tbs_synthesize", load_library().tbs_synthesize(arr, len(entries), n_rhs, x0, y0, sx, sy, nx, ny,
                                                            t0, dt, n_t, out_ptr, stream))


def synthesize(fields, dxs, freqs_hz, weights, origin, step, counts, t0, dt, n_t, out=None, stream=None):
    """Time signal s(X, t) = sum_k w_k psi_k(X) exp(-2 pi i f_k t) at the
    receivers X = origin + (ix, iy) * step, 0 <= ix, iy < counts, for
    t_j = t0 + j dt (tbs_synthesize).  fields[k]: CUDA complex64 [n_rhs, n_k,
    n_k].  Returns complex64 [n_rhs, ny, nx, n_t] (Re = pressure)."""
    torch = _torch()
    if not (len(fields) == len(dxs) == len(freqs_hz) == len(weights)) or not fields:
        raise ValueError("one dx, frequency and weight per field")
    n_rhs = fields[0].shape[0]
    entries = []
    for k, f in enumerate(fields):
        n = f.shape[-1]
        entries.append((_dev_ptr(f, torch.complex64, (n_rhs, n, n), "fields[%d]" % k), n, float(dxs[k]),
                        float(freqs_hz[k]), float(weights[k])))
    nx, ny = counts
    if out is None:
        out = torch.empty((n_rhs, ny, nx, n_t), dtype=torch.complex64, device="cuda")
    ptr = _dev_ptr(out, torch.complex64, (n_rhs, ny, nx, n_t), "out")
    tbs_synthesize(entries, n_rhs, float(origin[0]), float(origin[1]), float(step[0]), float(step[1]), nx, ny,
                   float(t0), float(dt), n_t, ptr, _stream(stream))
    return out


def tbs_batch_create(plans, psi_ptrs, info_ptrs) -> int:
    n = len(plans)
    arr = lambda xs: (C.c_void_p * n)(*xs)
    h = C.c_void_p()
    _check("tbs_batch_create", load_library().tbs_batch_create(arr(plans), n, arr(psi_ptrs),
                                                                arr(info_ptrs), C.byref(h)))
    return h.value


def tbs_batch_solve(batch, stream=0):
    _check("tbs_batch_solve", load_library().tbs_batch_solve(batch, stream))


def tbs_batch_destroy(batch):
    _check("tbs_batch_destroy", load_library().tbs_batch_destroy(batch))


class Batch:
    """Several plans solved by one graph launch (tbs_batch_*).  Outputs land in
    torch tensors: psi[i] [n_rhs_i, N_i, N_i] complex64 and a device info
    buffer per plan (``infos()`` copies them to the host)."""

    def __init__(self, plans):
        import torch
        self.plans = list(plans)
        self.psi = [torch.empty((p.n_rhs, p.n, p.n), dtype=torch.complex64, device="cuda")
                    for p in self.plans]
        isz = C.sizeof(tbs_solve_info)
        self.info = [torch.empty((p.n_rhs * isz,), dtype=torch.uint8, device="cuda") for p in self.plans]
        self.handle = tbs_batch_create([p.handle for p in self.plans], [t.data_ptr() for t in self.psi],
                                       [t.data_ptr() for t in self.info])

    def solve(self, stream=None):
        tbs_batch_solve(self.handle, _stream(stream))

    def infos(self):
        out = []
        for p, t in zip(self.plans, self.info):
            raw = t.cpu().numpy().tobytes()
            recs = (tbs_solve_info * p.n_rhs).from_buffer_copy(raw)
            out.append(Plan.info_dicts(recs))
        return out

    def close(self):
        if getattr(self, "handle", None):
            tbs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tbs_get_ghat(plan, out_host_ptr):
    _check("tbs_get_ghat", load_library().tbs_get_ghat(plan, out_host_ptr))


def tbs_set_timing(plan, enable):
    _check("tbs_set_timing", load_library().tbs_set_timing(plan, int(enable)))


def tbs_get_timing(plan):
    rm, rn, cm, cn = C.c_double(), C.c_int32(), C.c_double(), C.c_int32()
    _check("tbs_get_timing", load_library().tbs_get_timing(plan, C.byref(rm), C.byref(rn),
                                                            C.byref(cm), C.byref(cn)))
    return rm.value, rn.value, cm.value, cn.value


def tbs_col_variants(plan):
    return int(load_library().tbs_col_variants(plan))


def tbs_set_col_variant(plan, variant):
    _check("tbs_set_col_variant", load_library().tbs_set_col_variant(plan, int(variant)))


def tbs_autotune(plan, reps=5, stream=0):
    """(best variant, [ms per launch of each variant])"""
    nv = tbs_col_variants(plan)
    times = (C.c_double * max(1, nv))()
    best = C.c_int32()
    _check("tbs_autotune", load_library().tbs_autotune(plan, int(reps), times, C.byref(best), stream))
    return best.value, list(times)[:nv]


def tbs_col_variant_name(plan, variant=-1):
    """Description of column-pass variant `variant` (-1: the active one)."""
    r = load_library().tbs_col_variant_name(plan, int(variant))
    return r.decode() if r else None


def tbs_row_variants(plan):
    return int(load_library().tbs_row_variants(plan))


def tbs_row_variant_name(plan, variant=-1):
    """Description of steady-state row-pass variant `variant` (-1: the active one)."""
    r = load_library().tbs_row_variant_name(plan, int(variant))
    return r.decode() if r else None


def tbs_set_row_variant(plan, variant):
    _check("tbs_set_row_variant", load_library().tbs_set_row_variant(plan, int(variant)))


def tbs_autotune_rows(plan, reps=5, stream=0):
    """(best row-pass variant, [ms per launch of each variant])"""
    nv = tbs_row_variants(plan)
    times = (C.c_double * max(1, nv))()
    best = C.c_int32()
    _check("tbs_autotune_rows", load_library().tbs_autotune_rows(plan, int(reps), times, C.byref(best), stream))
    return best.value, list(times)[:nv]


def tbs_potential_max_abs(plan, stream=0):
    """max |U| over the plan's potential (U = V + i eps), FP64 on the device"""
    out = C.c_double()
    _check("tbs_potential_max_abs", load_library().tbs_potential_max_abs(plan, C.byref(out), stream))
    return out.value


def tbs_plan_eps(plan):
    return float(load_library().tbs_plan_eps(plan))


def tbs_device_error(plan, stream=0):
    """0, TBS_WAIT_TIMEOUT or TBS_COPY_CHECK_FAILED for the plan's last call"""
    code = C.c_int32()
    _check("tbs_device_error", load_library().tbs_device_error(plan, C.byref(code), stream))
    return code.value


def tbs_debug_set(plan, key, value):
    _check("tbs_debug_set", load_library().tbs_debug_set(plan, int(key), int(value)))


def tbs_destroy(plan):
    _check("tbs_destroy", load_library().tbs_destroy(plan))


# ---- torch marshalling -------------------------------------------------------

def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev_ptr(t, dtype, shape, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor of shape %s (got %s %s)"
                         % (name, dtype, tuple(shape), t.dtype, tuple(t.shape)))
    return t.data_ptr()


class Plan:
    """One (N, k0, n_rhs) problem family on the current CUDA device."""

    def __init__(self, n, dx, freq_hz, c0, n_rhs=1, max_terms=64, tol=1e-6,
                 stop_mode=TBS_STOP_L2, l1_row=-1, div_grace=8, div_window=4,
                 div_factor=1e6, keep_terms=False, use_graph=True, stream=None, workspace=None,
                 checkpoint=False, periodic=False, eps_factor=0.8, abl_width=0, abl_zeta=0.0,
                 kspace_alpha0=None, kspace_nu=1.5, kspace_dispersion=True, cbs=False):
        """Arguments mirror tbs_plan_desc (include/tbs.h).  The flags:
        keep_terms / checkpoint (adjoint term storage), use_graph=False
        (host-launched kernels), periodic (the paper's periodic grid with
        eps = eps_factor k0^2 and the abl_width / abl_zeta layer),
        kspace_alpha0 (periodic: the k-space absorbing(-dispersive)
        potential with kspace_nu; kspace_dispersion=False drops eta) and cbs
        (periodic: the convergent Born series preconditioner; eps_factor=0
        lets the library choose eps = 1.01 max|U| from each medium).
        workspace: None (the plan allocates its buffers), True (a uint8
        tensor from torch's caching allocator holds them, kept as
        self.workspace) or such a CUDA tensor of >= tbs_plan_device_bytes."""
        d = tbs_plan_desc_init()
        d.n, d.n_rhs, d.dx, d.freq_hz, d.c0 = n, n_rhs, dx, freq_hz, c0
        d.max_terms, d.tol, d.stop_mode, d.l1_row = max_terms, tol, stop_mode, l1_row
        d.div_grace, d.div_window, d.div_factor = div_grace, div_window, div_factor
        d.flags = (TBS_FLAG_KEEP_TERMS if keep_terms else 0) | (0 if use_graph else TBS_FLAG_NO_GRAPH) | \
            (TBS_FLAG_CHECKPOINT_TERMS if checkpoint else 0) | (TBS_FLAG_PERIODIC if periodic else 0)
        d.eps_factor, d.abl_width, d.abl_zeta = eps_factor, abl_width, abl_zeta
        if kspace_alpha0 is not None:  # the paper's absorbing-dispersive case II (periodic only)
            d.flags |= TBS_FLAG_KSPACE_ABSORPTION
            d.kspace_alpha0, d.kspace_nu = kspace_alpha0, kspace_nu
            d.kspace_absorption_only = 0 if kspace_dispersion else 1
        if cbs:  # the convergent Born series preconditioner (periodic; eps_factor >= max|U| / k0^2)
            d.flags |= TBS_FLAG_CBS
        self.desc = d
        self.n, self.n_rhs, self.freq_hz = n, n_rhs, freq_hz
        self.periodic = bool(periodic)
        self.workspace = None
        if workspace is None:
            self.handle = tbs_plan(d, _stream(stream))
        else:
            torch = _torch()
            if workspace is True:
                workspace = torch.empty(tbs_plan_device_bytes(d), dtype=torch.uint8, device="cuda")
            if not (isinstance(workspace, torch.Tensor) and workspace.is_cuda and workspace.is_contiguous()):
                raise TypeError("workspace must be a contiguous CUDA tensor")
            self.workspace = workspace  # must outlive the plan
            self.handle = tbs_plan_with_workspace(d, workspace.data_ptr(),
                                                  workspace.numel() * workspace.element_size(), _stream(stream))
        self.m = tbs_plan_padded_size(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            tbs_destroy(self.handle)
            self.handle = None
        if getattr(self, "workspace", None) is not None:
            _torch().cuda.synchronize()  # no launch of the plan may still use the memory
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- inputs
    def set_medium(self, c, alpha=None, y_pow=1.0, f_ref_hz=None, stream=None):
        torch = _torch()
        n = self.n
        cp = _dev_ptr(c, torch.float32, (n, n), "c")
        ap = _dev_ptr(alpha, torch.float32, (n, n), "alpha") if alpha is not None else None
        tbs_set_medium(self.handle, cp, ap, y_pow,
                       self.freq_hz if f_ref_hz is None else f_ref_hz, _stream(stream))

    def set_potential(self, V, stream=None):
        torch = _torch()
        tbs_set_potential(self.handle, _dev_ptr(V, torch.complex64, (self.n, self.n), "V"),
                          _stream(stream))

    def set_sources(self, ix, iy, amp, stream=None):
        import numpy as np
        ix = np.ascontiguousarray(ix, np.int32)
        iy = np.ascontiguousarray(iy, np.int32)
        amp = np.ascontiguousarray(amp, np.complex64).reshape(self.n_rhs, ix.size)
        tbs_set_sources(self.handle, ix.size, ix.ctypes.data, iy.ctypes.data, amp.ctypes.data,
                        _stream(stream))

    def set_source_field(self, S, stream=None):
        torch = _torch()
        n = self.n
        tbs_set_source_field(self.handle, _dev_ptr(S, torch.complex64, (self.n_rhs, n, n), "S"),
                             _stream(stream))

    def set_harmonic2_source(self, psi1, beta, rho, c, omega_fundamental, stream=None):
        torch = _torch()
        n = self.n
        tbs_set_harmonic2_source(
            self.handle, _dev_ptr(psi1, torch.complex64, (self.n_rhs, n, n), "psi1"),
            _dev_ptr(beta, torch.float32, (n, n), "beta"), _dev_ptr(rho, torch.float32, (n, n), "rho"),
            _dev_ptr(c, torch.float32, (n, n), "c"), omega_fundamental, _stream(stream))

    def set_harmonic_source(self, order, lower, beta, rho, c, omega_fundamental, stream=None, psi_scale=None,
                            source_scale=1.0):
        """Sum-term source of harmonic `order` from lower = [psi_1, ..., psi_{order-1}]
        (each stored divided by its psi_scale entry), written times source_scale."""
        torch = _torch()
        n = self.n
        ptrs = [_dev_ptr(p, torch.complex64, (self.n_rhs, n, n), "psi_%d" % (k + 1)) for k, p in enumerate(lower)]
        tbs_set_harmonic_source(self.handle, order, ptrs, _dev_ptr(beta, torch.float32, (n, n), "beta"),
                                _dev_ptr(rho, torch.float32, (n, n), "rho"), _dev_ptr(c, torch.float32, (n, n), "c"),
                                omega_fundamental, _stream(stream), psi_scale, source_scale)

    # -- compute
    def solve(self, psi=None, stream=None, sync=True, info=None):
        """Returns (psi [n_rhs, N, N] complex64, the solve records).

        The records go to host memory (ctypes array; the call then waits for
        the solve) unless ``info`` is a CUDA uint8 tensor of at least
        n_rhs * sizeof(tbs_solve_info) bytes, which is filled asynchronously
        and returned (read it with ``Plan.device_info_dicts``)."""
        torch = _torch()
        n = self.n
        if psi is None:
            psi = torch.empty((self.n_rhs, n, n), dtype=torch.complex64, device="cuda")
        if info is None:
            infos = (tbs_solve_info * self.n_rhs)()
            iptr = C.addressof(infos)
        else:
            need = self.n_rhs * C.sizeof(tbs_solve_info)
            if not (info.is_cuda and info.dtype == torch.uint8 and info.is_contiguous() and info.numel() >= need):
                raise TbsError(1, "info must be a contiguous CUDA uint8 tensor of >= %d bytes" % need)
            infos, iptr = info, info.data_ptr()
        tbs_solve(self.handle, _dev_ptr(psi, torch.complex64, (self.n_rhs, n, n), "psi"), iptr, _stream(stream))
        if sync:
            torch.cuda.synchronize()
        return psi, infos

    def device_info_dicts(self, info):
        """Info dicts from a device record buffer filled by solve(info=...)."""
        raw = info[: self.n_rhs * C.sizeof(tbs_solve_info)].cpu().numpy().tobytes()
        return Plan.info_dicts((tbs_solve_info * self.n_rhs).from_buffer_copy(raw))

    @staticmethod
    def info_dicts(infos):
        return [dict(terms=i.terms, status=i.status, status_name=STATUS_NAMES.get(i.status, "?"),
                     residual=i.residual, term_norm_max=i.term_norm_max, psi_norm=i.psi_norm)
                for i in infos]

    def solve_adjoint(self, grad_psi, grad_c=None, grad_alpha=None, stream=None):
        torch = _torch()
        n = self.n
        gp = _dev_ptr(grad_psi, torch.complex64, (self.n_rhs, n, n), "grad_psi")
        gc = _dev_ptr(grad_c, torch.float32, (n, n), "grad_c") if grad_c is not None else None
        ga = _dev_ptr(grad_alpha, torch.float32, (n, n), "grad_alpha") if grad_alpha is not None else None
        tbs_solve_adjoint(self.handle, gp, gc, ga, _stream(stream))

    def apply_green(self, f, out=None, conj_kernel=False, stream=None):
        torch = _torch()
        n = self.n
        if out is None:
            out = torch.empty((self.n_rhs, n, n), dtype=torch.complex64, device="cuda")
        tbs_apply_green(self.handle, _dev_ptr(f, torch.complex64, (self.n_rhs, n, n), "f"),
                        _dev_ptr(out, torch.complex64, (self.n_rhs, n, n), "out"),
                        int(conj_kernel), _stream(stream))
        return out

    def ghat_quadrant(self):
        import numpy as np
        q = self.m // 2 + 1
        out = np.zeros((q, q), np.complex64)
        tbs_get_ghat(self.handle, out.ctypes.data)
        return out

    def set_timing(self, enable=True):
        tbs_set_timing(self.handle, enable)

    def timing(self):
        return tbs_get_timing(self.handle)
