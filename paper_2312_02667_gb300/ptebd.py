"""Python binding of libptebd (C ABI in include/ptebd.h).

Argument marshalling only: every step of the pTEBD layer runs in the CUDA
library.  PyTorch provides the device buffers (caching allocator) and the
stream.  The module-level functions carry the C names; ``State`` is a thin
owner of one handle and its two device buffers.

Importing this module loads ``_build/libptebd.so`` and fails loudly if it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libptebd.so")

PTEBD_OK = 0
ERRORS = {
    -1: "PTEBD_ERR_INVALID", -2: "PTEBD_ERR_UNSUPPORTED", -3: "PTEBD_ERR_MEMORY", -4: "PTEBD_ERR_CUDA",
    -5: "PTEBD_ERR_OVERLAP", -6: "PTEBD_ERR_NUMERIC", -7: "PTEBD_ERR_NOT_CONVERGED", -8: "PTEBD_ERR_SHAPE",
    -9: "PTEBD_ERR_TIMEOUT",
}
PTEBD_FP64, PTEBD_MIXED = 0, 1
PTEBD_EPS_SCHMIDT, PTEBD_EPS_ABSOLUTE, PTEBD_EPS_RELATIVE = 0, 1, 2
PTEBD_CHI_LIMIT = 256

# every symbol include/ptebd.h declares
EXPORTS = (
    "ptebd_required_bytes", "ptebd_create", "ptebd_destroy", "ptebd_set_stream", "ptebd_reset",
    "ptebd_last_error", "ptebd_get_config", "ptebd_apply_layer", "ptebd_apply_bonds", "ptebd_regauge",
    "ptebd_sync", "ptebd_norm", "ptebd_overlap", "ptebd_expect", "ptebd_expect2", "ptebd_get_chi",
    "ptebd_get_lambda", "ptebd_get_site", "ptebd_set_lambda", "ptebd_set_site", "ptebd_trunc_error",
    "ptebd_bond_stats", "ptebd_svd_sweeps", "ptebd_timing", "ptebd_timing_read",
    "ptebd_work_counters", "ptebd_svd_workspace_bytes", "ptebd_svd_batched",
    "ptebd_batch_create", "ptebd_batch_destroy", "ptebd_batch_last_error", "ptebd_batch_apply_layer",
    "ptebd_svd_batched_noalloc", "ptebd_canonicalize", "ptebd_sample", "ptebd_sample_workspace_bytes",
    "ptebd_set_chunk_streams", "ptebd_test_wait_timeout", "ptebd_alu_peak", "ptebd_set_regauge_precision",
    "ptebd_set_jacobi_width", "ptebd_set_jacobi_pairs", "ptebd_set_ptsu_shortcut", "ptebd_autotune", "ptebd_set_tensor_cores",
    "ptebd_set_svd_polish",
)
KERNEL_KINDS = ("theta", "svd", "truncate", "gamma", "reduce", "factor", "resolve")


class ptebd_config(ctypes.Structure):
    _fields_ = [
        ("n_sites", ctypes.c_int32), ("d", ctypes.c_int32), ("chi_max", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("g", ctypes.c_int32), ("eps_mode", ctypes.c_int32),
        ("cutoff", ctypes.c_double), ("resolve", ctypes.c_double),
    ]


class PtebdError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)
_SZ = ctypes.POINTER(ctypes.c_size_t)
_CFG = ctypes.POINTER(ptebd_config)

_SIGS = {
    "ptebd_required_bytes": (_CFG, _SZ, _SZ, _SZ),
    "ptebd_create": (_CFG, _P, ctypes.c_size_t, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)),
    "ptebd_destroy": (_P,),
    "ptebd_set_stream": (_P, _P),
    "ptebd_reset": (_P,),
    "ptebd_get_config": (_P, _CFG),
    "ptebd_apply_layer": (_P, _D, ctypes.c_int32, ctypes.c_int32),
    "ptebd_apply_bonds": (_P, _I, ctypes.c_int32, _D, ctypes.c_int32),
    "ptebd_regauge": (_P, ctypes.c_int32),
    "ptebd_sync": (_P,),
    "ptebd_norm": (_P, _D),
    "ptebd_overlap": (_P, _P, _D),
    "ptebd_expect": (_P, ctypes.c_int32, _D, _D),
    "ptebd_expect2": (_P, ctypes.c_int32, _D, _D),
    "ptebd_get_chi": (_P, _I),
    "ptebd_get_lambda": (_P, ctypes.c_int32, _D, _I),
    "ptebd_get_site": (_P, ctypes.c_int32, _I, _I, _D),
    "ptebd_set_lambda": (_P, ctypes.c_int32, ctypes.c_int32, _D),
    "ptebd_set_site": (_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _D),
    "ptebd_trunc_error": (_P, _D, _D),
    "ptebd_bond_stats": (_P, _D, _D, _I),
    "ptebd_svd_sweeps": (_P, _I, _I),
    "ptebd_timing": (_P, ctypes.c_int32),
    "ptebd_timing_read": (_P, _D, _I, ctypes.c_int32),
    "ptebd_work_counters": (_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32),
    "ptebd_svd_workspace_bytes": (ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _SZ),
    "ptebd_svd_batched": (ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                          _P, _P, ctypes.c_int32, _P, ctypes.c_size_t, _P, ctypes.c_int32),
    "ptebd_batch_create": (ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(_P)),
    "ptebd_batch_destroy": (_P,),
    "ptebd_batch_apply_layer": (_P, ctypes.POINTER(_D), _I, _I),
    "ptebd_svd_batched_noalloc": (ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                                  ctypes.c_int32, _P, _P, ctypes.c_int32, _P, ctypes.c_int32),
    "ptebd_canonicalize": (_P,),
    "ptebd_sample": (_P, ctypes.c_int32, _D, _I, _P, ctypes.c_size_t),
    "ptebd_sample_workspace_bytes": (_P, ctypes.c_int32, _SZ),
    "ptebd_set_chunk_streams": (_P, ctypes.c_int32),
    "ptebd_test_wait_timeout": (_P, ctypes.c_int32),
    "ptebd_alu_peak": (ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t, _P, _D, _D),
    "ptebd_set_regauge_precision": (_P, ctypes.c_int32),
    "ptebd_set_jacobi_width": (_P, ctypes.c_int32),
    "ptebd_set_jacobi_pairs": (_P, ctypes.c_int32),
    "ptebd_set_ptsu_shortcut": (_P, ctypes.c_int32),
    "ptebd_set_tensor_cores": (_P, ctypes.c_int32),
    "ptebd_set_svd_polish": (_P, ctypes.c_int32),
    "ptebd_autotune": (_P, _D, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t, _D),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libptebd not built ({path} missing): run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = list(args)
        fn.restype = ctypes.c_int
    lib.ptebd_last_error.argtypes = [_P]
    lib.ptebd_last_error.restype = ctypes.c_char_p
    lib.ptebd_batch_last_error.argtypes = [_P]
    lib.ptebd_batch_last_error.restype = ctypes.c_char_p
    return lib


lib = load_library()


def _check(rc, handle=None):
    if rc != PTEBD_OK:
        msg = lib.ptebd_last_error(handle).decode() if handle else ""
        raise PtebdError(rc, msg)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_I)


# ---------------------------------------------------------------- C names --

def make_config(n_sites, chi_max, precision="mixed", cutoff=1e-12, g=0, eps_mode="schmidt", resolve=-1.0):
    prec = {"fp64": PTEBD_FP64, "mixed": PTEBD_MIXED}[precision] if isinstance(precision, str) else int(precision)
    mode = {"schmidt": PTEBD_EPS_SCHMIDT, "relative": PTEBD_EPS_RELATIVE, "absolute": PTEBD_EPS_ABSOLUTE}[eps_mode] \
        if isinstance(eps_mode, str) else int(eps_mode)
    return ptebd_config(int(n_sites), 2, int(chi_max), prec, int(g), mode, float(cutoff), float(resolve))


def ptebd_required_bytes(cfg: ptebd_config):
    s, w, wmin = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib.ptebd_required_bytes(ctypes.byref(cfg), ctypes.byref(s), ctypes.byref(w), ctypes.byref(wmin)))
    return s.value, w.value, wmin.value


def ptebd_create(cfg, state_ptr, state_bytes, ws_ptr, ws_bytes, stream):
    h = _P()
    _check(lib.ptebd_create(ctypes.byref(cfg), _P(state_ptr), state_bytes, _P(ws_ptr), ws_bytes, _P(stream),
                            ctypes.byref(h)))
    return h


def ptebd_destroy(h):
    _check(lib.ptebd_destroy(h))


def ptebd_set_stream(h, stream):
    _check(lib.ptebd_set_stream(h, _P(stream)), h)


def ptebd_reset(h):
    _check(lib.ptebd_reset(h), h)


def ptebd_get_config(h) -> ptebd_config:
    c = ptebd_config()
    _check(lib.ptebd_get_config(h, ctypes.byref(c)), h)
    return c


def _gates_arg(gates):
    """(host array, on_device flag, keepalive) for a gate batch."""
    try:
        import torch
        if isinstance(gates, torch.Tensor) and gates.is_cuda:
            t = gates
            if t.dtype == torch.complex128:
                t = torch.view_as_real(t.contiguous())
            if t.dtype != torch.float64:
                raise TypeError("device gates must be complex128 or float64")
            t = t.contiguous()
            return ctypes.cast(_P(t.data_ptr()), _D), 1, t
    except ImportError:  # pragma: no cover
        pass
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.complex128)).view(np.float64).reshape(-1)
    g = np.ascontiguousarray(g)
    return _dptr(g), 0, g


def ptebd_apply_layer(h, gates, parity):
    p, dev, keep = _gates_arg(gates)
    _check(lib.ptebd_apply_layer(h, p, int(parity), dev), h)
    return keep


def ptebd_apply_bonds(h, bonds, gates):
    b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32))
    p, dev, keep = _gates_arg(gates)
    _check(lib.ptebd_apply_bonds(h, _iptr(b), len(b), p, dev), h)
    return keep


def ptebd_regauge(h, g):
    _check(lib.ptebd_regauge(h, int(g)), h)


def ptebd_sync(h):
    _check(lib.ptebd_sync(h), h)


def ptebd_norm(h) -> float:
    out = ctypes.c_double()
    _check(lib.ptebd_norm(h, ctypes.byref(out)), h)
    return out.value


def ptebd_overlap(a, b) -> complex:
    out = np.zeros(2)
    _check(lib.ptebd_overlap(a, b, _dptr(out)), a)
    return complex(out[0], out[1])


def ptebd_expect(h, site, op) -> complex:
    o = np.ascontiguousarray(np.asarray(op, dtype=np.complex128)).view(np.float64).reshape(-1).copy()
    out = np.zeros(2)
    _check(lib.ptebd_expect(h, int(site), _dptr(o), _dptr(out)), h)
    return complex(out[0], out[1])


def ptebd_expect2(h, site, op) -> complex:
    o = np.ascontiguousarray(np.asarray(op, dtype=np.complex128)).view(np.float64).reshape(-1).copy()
    out = np.zeros(2)
    _check(lib.ptebd_expect2(h, int(site), _dptr(o), _dptr(out)), h)
    return complex(out[0], out[1])


def ptebd_get_chi(h, n_sites) -> np.ndarray:
    out = np.zeros(n_sites - 1, dtype=np.int32)
    _check(lib.ptebd_get_chi(h, _iptr(out)), h)
    return out


def ptebd_get_lambda(h, bond, chi_max) -> np.ndarray:
    out = np.zeros(chi_max)
    k = ctypes.c_int32()
    _check(lib.ptebd_get_lambda(h, int(bond), _dptr(out), ctypes.byref(k)), h)
    return out[: k.value].copy()


def ptebd_get_site(h, site) -> np.ndarray:
    cl, cr = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.ptebd_get_site(h, int(site), ctypes.byref(cl), ctypes.byref(cr), None), h)
    out = np.zeros(2 * cl.value * cr.value * 2)
    _check(lib.ptebd_get_site(h, int(site), ctypes.byref(cl), ctypes.byref(cr), _dptr(out)), h)
    return out.view(np.complex128).reshape(2, cl.value, cr.value)


def ptebd_set_lambda(h, bond, values):
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
    _check(lib.ptebd_set_lambda(h, int(bond), len(v), _dptr(v)), h)


def ptebd_set_site(h, site, gamma):
    g = np.ascontiguousarray(np.asarray(gamma, dtype=np.complex128))
    flat = np.ascontiguousarray(g.view(np.float64).reshape(-1))
    _check(lib.ptebd_set_site(h, int(site), g.shape[1], g.shape[2], _dptr(flat)), h)


def ptebd_trunc_error(h):
    e, l = ctypes.c_double(), ctypes.c_double()
    _check(lib.ptebd_trunc_error(h, ctypes.byref(e), ctypes.byref(l)), h)
    return e.value, l.value


def ptebd_bond_stats(h, n_sites):
    eps = np.zeros(n_sites - 1)
    nu = np.zeros(n_sites - 1)
    rk = np.zeros(n_sites - 1, dtype=np.int32)
    _check(lib.ptebd_bond_stats(h, _dptr(eps), _dptr(nu), _iptr(rk)), h)
    return eps, nu, rk


def ptebd_svd_sweeps(h, n_sites):
    sw = np.zeros(n_sites - 1, dtype=np.int32)
    layers = ctypes.c_int32()
    _check(lib.ptebd_svd_sweeps(h, _iptr(sw), ctypes.byref(layers)), h)
    return sw, layers.value


def ptebd_canonicalize(h):
    _check(lib.ptebd_canonicalize(h), h)


def ptebd_sample_workspace_bytes(h, n_samples) -> int:
    out = ctypes.c_size_t()
    _check(lib.ptebd_sample_workspace_bytes(h, int(n_samples), ctypes.byref(out)), h)
    return out.value


def ptebd_sample(h, uniforms, workspace=None) -> np.ndarray:
    """Bit strings (n_samples, N) drawn with the given uniforms (n_samples, N);
    workspace: a CUDA uint8 tensor used as scratch, or None for the state's own."""
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    bits = np.zeros(u.shape, dtype=np.int32)
    wp, wb = (workspace.data_ptr(), workspace.numel()) if workspace is not None else (None, 0)
    _check(lib.ptebd_sample(h, u.shape[0], _dptr(u), _iptr(bits), wp, wb), h)
    return bits


def ptebd_set_chunk_streams(h, n):
    _check(lib.ptebd_set_chunk_streams(h, int(n)), h)


def ptebd_set_regauge_precision(h, precision):
    _check(lib.ptebd_set_regauge_precision(h, PTEBD_FP64 if precision == "fp64" else PTEBD_MIXED), h)


def ptebd_set_svd_polish(h, mode):
    _check(lib.ptebd_set_svd_polish(h, int(mode)), h)


def ptebd_set_tensor_cores(h, enable):
    """enable: False/0 off, True/1 gated stages (default), 2 the tSU steps as well."""
    _check(lib.ptebd_set_tensor_cores(h, 2 if (enable == 2 and enable is not True) else (1 if enable else 0)), h)


def ptebd_set_jacobi_width(h, nw):
    _check(lib.ptebd_set_jacobi_width(h, int(nw)), h)


def ptebd_set_jacobi_pairs(h, pairs):
    _check(lib.ptebd_set_jacobi_pairs(h, int(pairs)), h)


def ptebd_set_ptsu_shortcut(h, enable):
    _check(lib.ptebd_set_ptsu_shortcut(h, 1 if enable else 0), h)


def ptebd_autotune(h, gates, parity, scratch_ptr, scratch_bytes):
    """(block width, chunks, best ms, ms of the previous configuration, columns per warp)."""
    ptr, on_dev, keep = _gates_arg(gates)
    best = np.zeros(5)
    _check(lib.ptebd_autotune(h, ptr, int(parity), on_dev, _P(scratch_ptr), int(scratch_bytes), _dptr(best)), h)
    return int(best[0]), int(best[1]), float(best[2]), float(best[3]), int(best[4])


def ptebd_test_wait_timeout(h, enable):
    _check(lib.ptebd_test_wait_timeout(h, int(bool(enable))), h)


def ptebd_timing(h, enable):
    _check(lib.ptebd_timing(h, int(bool(enable))), h)


def ptebd_timing_read(h):
    """{kind: (ms, launches)} of the kernels launched while timing was on."""
    n = len(KERNEL_KINDS)
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int32)
    _check(lib.ptebd_timing_read(h, _dptr(ms), _iptr(cnt), n), h)
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)}


def ptebd_work_counters(h):
    """(Jacobi pair-row visits, theta flops, rotations applied, sweeps summed,
    SVDs, tSU visits, tSU sweeps, tSU SVDs, bonds recomputed in FP64 by the
    resolution of a mixed state, their Jacobi visits) since create/reset."""
    out = np.zeros(16, dtype=np.uint64)
    _check(lib.ptebd_work_counters(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), 16), h)
    return tuple(int(x) for x in out[:10])


def ptebd_svd_workspace_bytes(precision, batch, rows, cols) -> int:
    out = ctypes.c_size_t()
    _check(lib.ptebd_svd_workspace_bytes(int(precision), int(batch), int(rows), int(cols), ctypes.byref(out)))
    return out.value


def ptebd_svd_batched(precision, batch, rows, cols, a_ptr, lda, sigma_ptr, u_ptr, ldu, ws_ptr, ws_bytes, stream,
                      check=1):
    _check(lib.ptebd_svd_batched(int(precision), int(batch), int(rows), int(cols), _P(a_ptr), int(lda),
                                 _P(sigma_ptr), _P(u_ptr) if u_ptr else None, int(ldu), _P(ws_ptr), int(ws_bytes),
                                 _P(stream), int(check)))


def ptebd_svd_batched_noalloc(precision, batch, rows, cols, a_ptr, lda, sigma_ptr, u_ptr, ldu, stream, check=1):
    """The allocation-free batched SVD (scratch in the library's fixed device array)."""
    _check(lib.ptebd_svd_batched_noalloc(int(precision), int(batch), int(rows), int(cols), _P(a_ptr), int(lda),
                                         _P(sigma_ptr), _P(u_ptr) if u_ptr else None, int(ldu), _P(stream),
                                         int(check)))


def ptebd_alu_peak(kind, iters, scratch_ptr, scratch_bytes, stream):
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.ptebd_alu_peak(int(kind), int(iters), _P(scratch_ptr), int(scratch_bytes), _P(stream),
                              ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


ALU_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def alu_peak(kind, target_ms=150.0):
    """Measured FMA throughput of the current GPU for `kind` in ALU_KINDS:
    one short launch sizes a second one of about target_ms, whose rate is
    returned as (TFLOP/s, ms, iterations)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    scratch = torch.empty(8 * sms * 256, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    k = ALU_KINDS[kind]
    iters = 16
    _, ms = ptebd_alu_peak(k, iters, scratch.data_ptr(), scratch.numel() * 8, stream)
    iters = max(16, int(iters * target_ms / max(ms, 1e-3)))
    tf, ms = ptebd_alu_peak(k, iters, scratch.data_ptr(), scratch.numel() * 8, stream)
    return tf, ms, iters


def svd_batched(a, want_u=False, check=True):
    """Singular values (descending) and optionally left singular vectors of a
    batch of complex matrices: a torch tensor (batch, rows, cols) of
    complex64 or complex128 on the GPU.  Returns (sigma, u) tensors."""
    import torch
    if a.dtype not in (torch.complex64, torch.complex128) or not a.is_cuda or a.dim() != 3:
        raise TypeError("a must be a (batch, rows, cols) complex CUDA tensor")
    prec = PTEBD_FP64 if a.dtype == torch.complex128 else PTEBD_MIXED
    batch, rows, cols = a.shape
    am = a.transpose(1, 2).contiguous()  # column-major per matrix
    sigma = torch.empty((batch, cols), dtype=torch.float64, device=a.device)
    u = torch.empty((batch, cols, rows), dtype=a.dtype, device=a.device) if want_u else None
    wb = ptebd_svd_workspace_bytes(prec, batch, rows, cols)
    ws = torch.empty(wb, dtype=torch.uint8, device=a.device)
    ptebd_svd_batched(prec, batch, rows, cols, am.data_ptr(), rows, sigma.data_ptr(),
                      u.data_ptr() if u is not None else 0, rows, ws.data_ptr(), wb,
                      torch.cuda.current_stream(a.device).cuda_stream, 1 if check else 0)
    return sigma, (u.transpose(1, 2) if u is not None else None)


def ptebd_batch_create(handles):
    arr = (_P * len(handles))(*[h.value if isinstance(h, _P) else h for h in handles])
    out = _P()
    _check(lib.ptebd_batch_create(arr, len(handles), ctypes.byref(out)))
    return out


def ptebd_batch_destroy(b):
    _check(lib.ptebd_batch_destroy(b))


def ptebd_batch_last_error(b) -> str:
    return lib.ptebd_batch_last_error(b).decode()


def ptebd_batch_apply_layer(b, gates_list, parities):
    """gates_list[i]: (n_i, 4, 4) complex host array or CUDA tensor for state i."""
    n = len(parities)
    keep = []
    ptrs = (_D * n)()
    dev = np.zeros(n, dtype=np.int32)
    for i, g in enumerate(gates_list):
        p, d, k = _gates_arg(g)
        ptrs[i] = p
        dev[i] = d
        keep.append(k)
    par = np.ascontiguousarray(np.asarray(parities, dtype=np.int32))
    rc = lib.ptebd_batch_apply_layer(b, ptrs, _iptr(par), _iptr(dev))
    if rc != PTEBD_OK:
        raise PtebdError(rc, lib.ptebd_batch_last_error(b).decode())
    return keep


class Batch:
    """Independent states advanced together (one CUDA graph per parity pattern)."""

    def __init__(self, states):
        self.states = list(states)
        self.handle = ptebd_batch_create([s.handle for s in self.states])

    def apply_layer(self, gates_list, parities):
        self._keep = ptebd_batch_apply_layer(self.handle, gates_list, parities)

    def close(self):
        if getattr(self, "handle", None):
            ptebd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ owner --

class State:
    """One MPS on the current CUDA device, its buffers allocated by torch."""

    def __init__(self, n_sites, chi_max, precision="mixed", cutoff=1e-12, g=0, eps_mode="schmidt",
                 resolve=-1.0, workspace_bytes=None, stream=None, device=None):
        import torch
        self.cfg = make_config(n_sites, chi_max, precision, cutoff, g, eps_mode, resolve)
        self.n_sites, self.chi_max = int(n_sites), int(chi_max)
        sb, wb, wmin = ptebd_required_bytes(self.cfg)
        if workspace_bytes is not None:
            wb = max(int(workspace_bytes), wmin)
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self._state_buf = torch.empty(sb, dtype=torch.uint8, device=dev)
        self._ws_buf = torch.empty(wb, dtype=torch.uint8, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        self.handle = ptebd_create(self.cfg, self._state_buf.data_ptr(), sb, self._ws_buf.data_ptr(), wb,
                                   stream.cuda_stream)
        self.state_bytes, self.workspace_bytes = sb, wb
        self._keep = None

    def close(self):
        if getattr(self, "handle", None):
            ptebd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # thin forwards
    def apply_layer(self, gates, parity):
        self._keep = ptebd_apply_layer(self.handle, gates, parity)

    def apply_bonds(self, bonds, gates):
        self._keep = ptebd_apply_bonds(self.handle, bonds, gates)

    def regauge(self, g):
        ptebd_regauge(self.handle, g)

    def sync(self):
        ptebd_sync(self.handle)

    def reset(self):
        ptebd_reset(self.handle)

    def norm(self):
        return ptebd_norm(self.handle)

    def overlap(self, other: "State"):
        return ptebd_overlap(self.handle, other.handle)

    def expect(self, site, op):
        return ptebd_expect(self.handle, site, op)

    def expect2(self, site, op):
        return ptebd_expect2(self.handle, site, op)

    def chi(self):
        return ptebd_get_chi(self.handle, self.n_sites)

    def lam(self, bond):
        return ptebd_get_lambda(self.handle, bond, self.chi_max)

    def site(self, s):
        return ptebd_get_site(self.handle, s)

    def trunc_error(self):
        return ptebd_trunc_error(self.handle)

    def bond_stats(self):
        return ptebd_bond_stats(self.handle, self.n_sites)

    def svd_sweeps(self):
        return ptebd_svd_sweeps(self.handle, self.n_sites)

    def canonicalize(self):
        ptebd_canonicalize(self.handle)

    def sample(self, uniforms):
        """Bit strings drawn with the given uniforms; scratch beyond the
        state's workspace is allocated for the call."""
        n = int(np.shape(uniforms)[0])
        need = ptebd_sample_workspace_bytes(self.handle, n)
        ws = None
        if need > self.workspace_bytes:
            import torch
            ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return ptebd_sample(self.handle, uniforms, ws)

    def timing(self, enable):
        ptebd_timing(self.handle, enable)

    def set_chunk_streams(self, n):
        """Bond chunks a layer may run concurrently (0: automatic, 1: one stream)."""
        ptebd_set_chunk_streams(self.handle, n)

    def timing_read(self):
        return ptebd_timing_read(self.handle)

    def work_counters(self):
        return ptebd_work_counters(self.handle)

    def set_regauge_precision(self, precision):
        ptebd_set_regauge_precision(self.handle, precision)

    def set_jacobi_width(self, nw):
        ptebd_set_jacobi_width(self.handle, nw)

    def set_jacobi_pairs(self, pairs):
        ptebd_set_jacobi_pairs(self.handle, pairs)

    def set_ptsu_shortcut(self, enable):
        ptebd_set_ptsu_shortcut(self.handle, enable)

    def set_tensor_cores(self, enable):
        ptebd_set_tensor_cores(self.handle, enable)

    def set_svd_polish(self, mode):
        ptebd_set_svd_polish(self.handle, mode)

    def autotune(self, gates, parity):
        """Tune the launch configuration on this state's next layer (the state is
        left unchanged); scratch of state_bytes from the caching allocator."""
        import torch
        scratch = torch.empty(self._state_buf.numel(), dtype=torch.uint8, device=self.device)
        return ptebd_autotune(self.handle, gates, parity, scratch.data_ptr(), scratch.numel())

    def export(self):
        """(gammas, lambdas) as complex128 / float64 numpy arrays."""
        return ([self.site(s) for s in range(self.n_sites)],
                [self.lam(b) for b in range(self.n_sites - 1)])

    def load(self, gammas, lambdas):
        """Import a Vidal MPS: bond vectors first (they fix the dimensions)."""
        for b, l in enumerate(lambdas):
            ptebd_set_lambda(self.handle, b, l)
        for s, g in enumerate(gammas):
            ptebd_set_site(self.handle, s, g)
