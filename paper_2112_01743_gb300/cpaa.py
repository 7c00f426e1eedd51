"""ctypes binding of libcpaa.so with the names of include/cpaa.h.

Arguments may be torch tensors (host or CUDA), numpy arrays, or raw integer
addresses.  The functions only marshal arguments and check the returned
status; the computation happens in the library.  A non-OK status raises
``CpaaError`` (``CPAA_ENOTCONV`` only when ``raise_notconv`` is set).
"""
import ctypes
import os

import numpy as np

__all__ = [
    "CpaaError", "CpaaOptions", "CpaaInfo", "lib", "library_path",
    "CPAA_OK", "CPAA_EINVAL", "CPAA_ENOMEM", "CPAA_ENOTCONV", "CPAA_ECUDA", "CPAA_ETIMEOUT",
    "CPAA_EBUSY", "CPAA_ECANCELLED", "CPAA_ENOTFOUND",
    "CPAA_F64", "CPAA_F32", "CPAA_BF16", "CPAA_DF64", "CPAA_GRAPH_DEVICE_INPUT", "CPAA_GRAPH_VALIDATE",
    "CPAA_GRAPH_TRUSTED", "CPAA_GRAPH_AUTOTUNE", "CpaaLayoutParams", "cpaa_graph_create_ex",
    "CPAA_DEVICE_IO", "CPAA_TIME_ROUNDS", "CPAA_SERVER_FUSED", "CPAA_SPARSE_FRONTIER", "CPAA_INTERVAL",
    "CPAA_CERTIFY_INTERVAL", "cpaa_rounds_needed_interval", "cpaa_l1_bound_interval", "cpaa_graph_spectrum_bound",
    "CPAA_STOP_RIGOROUS",
    "CPAA_STOP_POSTERIORI",
    "cpaa_options_init", "cpaa_graph_create", "cpaa_graph_destroy", "cpaa_graph_info", "cpaa_graph_layout",
    "CpaaLayout", "cpaa_solve", "cpaa_solve_batch", "cpaa_rounds_needed", "cpaa_l1_bound",
    "cpaa_status_string", "cpaa_last_error", "cpaa_solve_fixed_noalloc", "cpaa_power_solve", "Graph",
    "EXPORTED_SYMBOLS", "CPAA_NOALLOC_MAX_N", "CPAA_SERVER_MAX_SEEDS", "CpaaServerStats",
    "cpaa_server_create", "cpaa_server_add_graph", "cpaa_server_submit", "cpaa_server_wait",
    "cpaa_server_cancel", "cpaa_server_get_stats", "cpaa_server_destroy", "Server",
]

CPAA_OK, CPAA_EINVAL, CPAA_ENOMEM, CPAA_ENOTCONV, CPAA_ECUDA = 0, 1, 2, 3, 4
CPAA_ETIMEOUT, CPAA_EBUSY, CPAA_ECANCELLED, CPAA_ENOTFOUND = 5, 6, 7, 8
CPAA_F64, CPAA_F32, CPAA_BF16, CPAA_DF64 = 0, 1, 2, 3
CPAA_GRAPH_DEVICE_INPUT, CPAA_GRAPH_VALIDATE, CPAA_GRAPH_TRUSTED, CPAA_GRAPH_AUTOTUNE = 1, 2, 4, 8
CPAA_DEVICE_IO = 1
CPAA_NOALLOC_MAX_N = 1300000
CPAA_SERVER_MAX_SEEDS = 64
CPAA_TIME_ROUNDS = 2
CPAA_SERVER_FUSED = 4
CPAA_SPARSE_FRONTIER = 8
CPAA_INTERVAL = 16
CPAA_CERTIFY_INTERVAL = 32
CPAA_STOP_RIGOROUS, CPAA_STOP_POSTERIORI = 0, 1

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "_build", "libcpaa.so")

# Every function include/cpaa.h declares (the CPU test checks the exports).
EXPORTED_SYMBOLS = [
    "cpaa_options_init", "cpaa_graph_create", "cpaa_graph_create_ex", "cpaa_graph_destroy", "cpaa_graph_info",
    "cpaa_graph_layout", "cpaa_solve", "cpaa_solve_batch", "cpaa_rounds_needed", "cpaa_l1_bound",
    "cpaa_status_string", "cpaa_last_error", "cpaa_solve_fixed_noalloc", "cpaa_power_solve",
    "cpaa_server_create", "cpaa_server_add_graph", "cpaa_server_submit", "cpaa_server_wait",
    "cpaa_server_cancel", "cpaa_server_get_stats", "cpaa_server_destroy",
    "cpaa_rounds_needed_interval", "cpaa_l1_bound_interval", "cpaa_graph_spectrum_bound",
]


class CpaaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_status_name(status), message))
        self.status = status


class CpaaLayout(ctypes.Structure):
    _fields_ = [("hub_rows", ctypes.c_int64), ("hub_entries", ctypes.c_int64), ("hub_tiles", ctypes.c_int64),
                ("chunks", ctypes.c_int64), ("long_chunks", ctypes.c_int64), ("sell_entries", ctypes.c_int64),
                ("hub_degree", ctypes.c_int), ("hub_tile", ctypes.c_int),
                ("long_chunk", ctypes.c_int), ("sort_window", ctypes.c_int),
                ("tuned", ctypes.c_int), ("tune_candidates", ctypes.c_int)]


class CpaaLayoutParams(ctypes.Structure):
    _fields_ = [("hub_degree", ctypes.c_int), ("hub_tile", ctypes.c_int), ("long_chunk", ctypes.c_int),
                ("sort_window", ctypes.c_int), ("tune_precision", ctypes.c_int)]


class CpaaOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("normalize", ctypes.c_int),
                ("fixed_rounds", ctypes.c_int), ("max_rounds", ctypes.c_int),
                ("flags", ctypes.c_uint), ("stream", ctypes.c_void_p),
                ("history", ctypes.POINTER(ctypes.c_double)), ("batch_width", ctypes.c_int),
                ("stop_rule", ctypes.c_int), ("lambda_lo", ctypes.c_double)]


class CpaaInfo(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("bound", ctypes.c_double), ("kappa", ctypes.c_double),
                ("mass", ctypes.c_double), ("l1", ctypes.c_double), ("sum_pibar", ctypes.c_double),
                ("rounds_ms", ctypes.c_double), ("lambda_lo", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class CpaaServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("pending", ctypes.c_int64), ("running", ctypes.c_int64), ("slots", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("admit_p50_us", ctypes.c_double), ("rounds", ctypes.c_uint64),
                ("round_columns", ctypes.c_uint64), ("relayouts", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libcpaa.so; raise if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(library_path):
        raise ImportError("libcpaa.so is not built (%s); run __graft_entry__.build()" % library_path)
    L = ctypes.CDLL(library_path)
    vp, i64, dbl, cint, cuint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_uint
    L.cpaa_options_init.restype = None
    L.cpaa_options_init.argtypes = [ctypes.POINTER(CpaaOptions)]
    L.cpaa_graph_create.restype = cint
    L.cpaa_graph_create.argtypes = [i64, i64, vp, vp, cuint, ctypes.POINTER(vp)]
    L.cpaa_graph_create_ex.restype = cint
    L.cpaa_graph_create_ex.argtypes = [i64, i64, vp, vp, cuint, ctypes.POINTER(CpaaLayoutParams),
                                       ctypes.POINTER(vp)]
    L.cpaa_graph_destroy.restype = cint
    L.cpaa_graph_destroy.argtypes = [vp]
    L.cpaa_graph_info.restype = cint
    L.cpaa_graph_info.argtypes = [vp] + [ctypes.POINTER(i64)] * 4
    L.cpaa_graph_layout.restype = cint
    L.cpaa_graph_layout.argtypes = [vp, ctypes.POINTER(CpaaLayout)]
    L.cpaa_solve.restype = cint
    L.cpaa_solve.argtypes = [vp, vp, dbl, dbl, vp, ctypes.POINTER(CpaaOptions), ctypes.POINTER(CpaaInfo)]
    L.cpaa_power_solve.restype = cint
    L.cpaa_power_solve.argtypes = [vp, vp, dbl, dbl, vp, ctypes.POINTER(CpaaOptions), ctypes.POINTER(CpaaInfo)]
    L.cpaa_solve_batch.restype = cint
    L.cpaa_solve_batch.argtypes = [vp, cint, vp, vp, dbl, vp, ctypes.POINTER(CpaaOptions),
                                   ctypes.POINTER(CpaaInfo)]
    L.cpaa_rounds_needed.restype = cint
    L.cpaa_rounds_needed.argtypes = [dbl, dbl, dbl, cint, cint]
    L.cpaa_l1_bound.restype = dbl
    L.cpaa_l1_bound.argtypes = [dbl, cint, dbl, cint]
    L.cpaa_solve_fixed_noalloc.restype = cint
    L.cpaa_solve_fixed_noalloc.argtypes = [i64, i64, vp, vp, vp, dbl, cint, cint, vp, vp]
    L.cpaa_server_create.restype = cint
    L.cpaa_server_create.argtypes = [ctypes.c_size_t, ctypes.POINTER(CpaaOptions), ctypes.POINTER(vp)]
    L.cpaa_server_add_graph.restype = cint
    L.cpaa_server_add_graph.argtypes = [vp, vp, cint, ctypes.POINTER(cint)]
    L.cpaa_server_submit.restype = cint
    L.cpaa_server_submit.argtypes = [vp, cint, cint, vp, vp, dbl, dbl, ctypes.POINTER(ctypes.c_uint64)]
    L.cpaa_server_wait.restype = cint
    L.cpaa_server_wait.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(CpaaInfo), i64]
    L.cpaa_server_cancel.restype = cint
    L.cpaa_server_cancel.argtypes = [vp, ctypes.c_uint64]
    L.cpaa_server_get_stats.restype = cint
    L.cpaa_server_get_stats.argtypes = [vp, ctypes.POINTER(CpaaServerStats)]
    L.cpaa_server_destroy.restype = cint
    L.cpaa_server_destroy.argtypes = [vp]
    L.cpaa_rounds_needed_interval.restype = cint
    L.cpaa_rounds_needed_interval.argtypes = [dbl, dbl, dbl, dbl, cint, cint]
    L.cpaa_l1_bound_interval.restype = dbl
    L.cpaa_l1_bound_interval.argtypes = [dbl, dbl, cint, dbl, cint]
    L.cpaa_graph_spectrum_bound.restype = cint
    L.cpaa_graph_spectrum_bound.argtypes = [vp, ctypes.POINTER(dbl)]
    L.cpaa_status_string.restype = ctypes.c_char_p
    L.cpaa_status_string.argtypes = [cint]
    L.cpaa_last_error.restype = ctypes.c_char_p
    L.cpaa_last_error.argtypes = []
    _lib = L
    return L


def _status_name(s):
    try:
        return lib().cpaa_status_string(int(s)).decode()
    except Exception:
        return "status %d" % s


def _check(status, raise_notconv=True):
    if status == CPAA_OK or (status == CPAA_ENOTCONV and not raise_notconv):
        return status
    raise CpaaError(status, lib().cpaa_last_error().decode())


def _addr(x):
    """Address of a tensor / ndarray / int (no copy, no conversion)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError("unsupported argument type %r" % type(x))


def _is_device(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def cpaa_options_init():
    o = CpaaOptions()
    lib().cpaa_options_init(ctypes.byref(o))
    return o


def cpaa_graph_create(n, nnz, row_ptr, col_idx, flags=0):
    """Upload a symmetric CSR graph; returns the opaque handle (int)."""
    h = ctypes.c_void_p()
    if _is_device(row_ptr):
        flags |= CPAA_GRAPH_DEVICE_INPUT
    _check(lib().cpaa_graph_create(int(n), int(nnz), _addr(row_ptr), _addr(col_idx), int(flags),
                                   ctypes.byref(h)))
    return h.value


def cpaa_graph_create_ex(n, nnz, row_ptr, col_idx, flags=0, params=None):
    """cpaa_graph_create with layout parameters: a dict of CpaaLayoutParams
    fields (missing ones 0, i.e. default) or None."""
    h = ctypes.c_void_p()
    if _is_device(row_ptr):
        flags |= CPAA_GRAPH_DEVICE_INPUT
    lp = None
    if params is not None:
        lp = CpaaLayoutParams(**{k: int(v) for k, v in params.items()})
    _check(lib().cpaa_graph_create_ex(int(n), int(nnz), _addr(row_ptr), _addr(col_idx), int(flags),
                                      ctypes.byref(lp) if lp is not None else None, ctypes.byref(h)))
    return h.value


def cpaa_graph_destroy(g):
    return _check(lib().cpaa_graph_destroy(g))


def cpaa_graph_layout(g):
    o = CpaaLayout()
    _check(lib().cpaa_graph_layout(g, ctypes.byref(o)))
    return {f: getattr(o, f) for f, _ in o._fields_}


def cpaa_graph_info(g):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().cpaa_graph_info(g, *[ctypes.byref(x) for x in v]))
    return {"n": v[0].value, "nnz": v[1].value, "device_bytes": v[2].value, "num_tiles": v[3].value}


def _options(precision, normalize, fixed_rounds, max_rounds, device_io, stream, history,
             time_rounds=False, stop_rule=CPAA_STOP_RIGOROUS, frontier=False, lambda_lo=None,
             certify_interval=False):
    o = cpaa_options_init()
    if lambda_lo is not None:
        o.lambda_lo = float(lambda_lo)
    o.stop_rule = int(stop_rule)
    o.precision = int(precision)
    o.normalize = int(normalize)
    o.fixed_rounds = int(fixed_rounds)
    if max_rounds:
        o.max_rounds = int(max_rounds)
    o.flags = (CPAA_DEVICE_IO if device_io else 0) | (CPAA_TIME_ROUNDS if time_rounds else 0) | \
        (CPAA_SPARSE_FRONTIER if frontier else 0) | (CPAA_INTERVAL if lambda_lo is not None else 0) | \
        (CPAA_CERTIFY_INTERVAL if certify_interval else 0)
    o.stream = stream
    if history is not None:
        o.history = history.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return o


def _stream_of(x, stream):
    if stream is not None:
        return int(stream)
    if _is_device(x):
        import torch
        return torch.cuda.current_stream(x.device).cuda_stream
    return None


def cpaa_solve(g, p, c, tol, pi, precision=CPAA_F64, normalize=0, fixed_rounds=0, max_rounds=0,
               stream=None, history=None, raise_notconv=True, time_rounds=False,
               stop_rule=CPAA_STOP_RIGOROUS, frontier=False, lambda_lo=None, certify_interval=False):
    """pi <- CPAA(p); p, pi FP64 length n (both host or both device).
    lambda_lo (a certified lower bound on P's spectrum) sets CPAA_INTERVAL;
    certify_interval sets CPAA_CERTIFY_INTERVAL."""
    dev = _is_device(p)
    if dev != _is_device(pi):
        raise ValueError("p and pi must both be host or both be device buffers")
    o = _options(precision, normalize, fixed_rounds, max_rounds, dev, _stream_of(p, stream), history,
                 time_rounds, stop_rule, frontier, lambda_lo, certify_interval)
    info = CpaaInfo()
    st = lib().cpaa_solve(g, _addr(p), float(c), float(tol), _addr(pi), ctypes.byref(o), ctypes.byref(info))
    _check(st, raise_notconv)
    return info


def cpaa_power_solve(g, p, c, tol, pi, precision=CPAA_F64, normalize=0, fixed_rounds=0, max_rounds=0,
                     stream=None, history=None, raise_notconv=True, time_rounds=False,
                     stop_rule=CPAA_STOP_RIGOROUS):
    """Power-method baseline (same layout and kernels): pi <- x_T."""
    dev = _is_device(p)
    if dev != _is_device(pi):
        raise ValueError("p and pi must both be host or both be device buffers")
    o = _options(precision, normalize, fixed_rounds, max_rounds, dev, _stream_of(p, stream), history,
                 time_rounds, stop_rule)
    info = CpaaInfo()
    st = lib().cpaa_power_solve(g, _addr(p), float(c), float(tol), _addr(pi), ctypes.byref(o),
                                ctypes.byref(info))
    _check(st, raise_notconv)
    return info


def cpaa_solve_batch(g, B, P, c, tol, PI, precision=CPAA_F32, normalize=0, fixed_rounds=0,
                     max_rounds=0, stream=None, raise_notconv=True, batch_width=0,
                     stop_rule=CPAA_STOP_RIGOROUS, frontier=False, lambda_lo=None, certify_interval=False):
    """Column b of P (n x B column-major, i.e. B vectors back to back) with
    damping c[b] -> column b of PI.  Returns a list of B info records."""
    dev = _is_device(P)
    cvec = np.ascontiguousarray(np.broadcast_to(np.asarray(c, dtype=np.float64), (int(B),)))
    o = _options(precision, normalize, fixed_rounds, max_rounds, dev, _stream_of(P, stream), None,
                 False, stop_rule, frontier, lambda_lo, certify_interval)
    o.batch_width = int(batch_width)
    infos = (CpaaInfo * int(B))()
    st = lib().cpaa_solve_batch(g, int(B), _addr(P), cvec.ctypes.data, float(tol), _addr(PI),
                                ctypes.byref(o), infos)
    _check(st, raise_notconv)
    return list(infos)


def cpaa_solve_fixed_noalloc(n, nnz, row_ptr, col_idx, p, c, rounds, pi, normalize=0,
                             stream=None):
    """Fixed-round FP64 solve that allocates nothing (all arguments in device
    memory; intermediates in the library's fixed per-device scratch array)."""
    st = lib().cpaa_solve_fixed_noalloc(int(n), int(nnz), _addr(row_ptr), _addr(col_idx), _addr(p),
                                        float(c), int(rounds), int(normalize), _addr(pi),
                                        _stream_of(p, stream))
    return _check(st)


def cpaa_server_create(budget_bytes, precision=CPAA_F32, normalize=0, max_rounds=0,
                       stop_rule=CPAA_STOP_RIGOROUS, fused=False, frontier=False):
    o = cpaa_options_init()
    o.precision = int(precision)
    o.normalize = int(normalize)
    o.stop_rule = int(stop_rule)
    if fused:
        o.flags |= CPAA_SERVER_FUSED
    if frontier:
        o.flags |= CPAA_SPARSE_FRONTIER
    if max_rounds:
        o.max_rounds = int(max_rounds)
    h = ctypes.c_void_p()
    _check(lib().cpaa_server_create(int(budget_bytes), ctypes.byref(o), ctypes.byref(h)))
    return h.value


def cpaa_server_add_graph(s, g, max_slots=0):
    gid = ctypes.c_int()
    _check(lib().cpaa_server_add_graph(s, g, int(max_slots), ctypes.byref(gid)))
    return gid.value


def cpaa_server_submit(s, graph_id, seeds, weights, c, tol):
    sd = np.ascontiguousarray(seeds, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    t = ctypes.c_uint64()
    _check(lib().cpaa_server_submit(s, int(graph_id), int(sd.size), sd.ctypes.data,
                                    None if w is None else w.ctypes.data, float(c), float(tol),
                                    ctypes.byref(t)))
    return t.value


def cpaa_server_wait(s, ticket, pi=None, timeout_us=-1, raise_errors=True):
    """Wait for a query; returns (status, info).  pi: host float64 array or None."""
    info = CpaaInfo()
    st = lib().cpaa_server_wait(s, ctypes.c_uint64(ticket), _addr(pi), ctypes.byref(info),
                                int(timeout_us))
    if raise_errors and st not in (CPAA_OK, CPAA_ETIMEOUT, CPAA_ECANCELLED):
        _check(st)
    return st, info


def cpaa_server_cancel(s, ticket):
    return lib().cpaa_server_cancel(s, ctypes.c_uint64(ticket))


def cpaa_server_get_stats(s):
    o = CpaaServerStats()
    _check(lib().cpaa_server_get_stats(s, ctypes.byref(o)))
    return o.as_dict()


def cpaa_server_destroy(s):
    return _check(lib().cpaa_server_destroy(s))


class Server:
    """Owning wrapper of a cpaa_server handle."""

    def __init__(self, budget_bytes, precision=CPAA_F32, normalize=0, max_rounds=0,
                 stop_rule=CPAA_STOP_RIGOROUS, fused=False, frontier=False):
        self.handle = cpaa_server_create(budget_bytes, precision, normalize, max_rounds, stop_rule, fused,
                                         frontier)

    def add_graph(self, graph, max_slots=0):
        return cpaa_server_add_graph(self.handle, graph.handle, max_slots)

    def submit(self, graph_id, seeds, weights, c, tol):
        return cpaa_server_submit(self.handle, graph_id, seeds, weights, c, tol)

    def wait(self, ticket, pi=None, timeout_us=-1):
        return cpaa_server_wait(self.handle, ticket, pi, timeout_us)

    def cancel(self, ticket):
        return cpaa_server_cancel(self.handle, ticket)

    def stats(self):
        return cpaa_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            cpaa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cpaa_rounds_needed(c, tol, kappa, normalize=0, max_rounds=2000):
    return lib().cpaa_rounds_needed(float(c), float(tol), float(kappa), int(normalize), int(max_rounds))


def cpaa_l1_bound(c, M, kappa, normalize=0):
    return lib().cpaa_l1_bound(float(c), int(M), float(kappa), int(normalize))


def cpaa_rounds_needed_interval(c, lambda_lo, tol, kappa, normalize=0, max_rounds=2000):
    return lib().cpaa_rounds_needed_interval(float(c), float(lambda_lo), float(tol), float(kappa),
                                             int(normalize), int(max_rounds))


def cpaa_l1_bound_interval(c, lambda_lo, M, kappa, normalize=0):
    return lib().cpaa_l1_bound_interval(float(c), float(lambda_lo), int(M), float(kappa), int(normalize))


def cpaa_graph_spectrum_bound(g):
    v = ctypes.c_double()
    _check(lib().cpaa_graph_spectrum_bound(g, ctypes.byref(v)))
    return v.value


def cpaa_status_string(s):
    return lib().cpaa_status_string(int(s)).decode()


def cpaa_last_error():
    return lib().cpaa_last_error().decode()


class Graph:
    """Owning wrapper of a cpaa_graph handle."""

    def __init__(self, row_ptr, col_idx, n=None, validate=True, layout=None, autotune=False):
        """validate=False passes CPAA_GRAPH_TRUSTED (no row-order or symmetry
        check; the column range is checked either way); layout is a dict of
        cpaa_layout_params fields; autotune passes CPAA_GRAPH_AUTOTUNE."""
        n = int(n if n is not None else len(row_ptr) - 1)
        nnz = int(col_idx.numel() if hasattr(col_idx, "numel") else len(col_idx))
        self.n, self.nnz = n, nnz
        flags = (0 if validate else CPAA_GRAPH_TRUSTED) | (CPAA_GRAPH_AUTOTUNE if autotune else 0)
        if layout is None and not autotune:
            self.handle = cpaa_graph_create(n, nnz, row_ptr, col_idx, flags)
        else:
            self.handle = cpaa_graph_create_ex(n, nnz, row_ptr, col_idx, flags, layout)

    def info(self):
        return cpaa_graph_info(self.handle)

    def layout(self):
        return cpaa_graph_layout(self.handle)

    def spectrum_bound(self):
        return cpaa_graph_spectrum_bound(self.handle)

    def solve(self, p, c, tol, pi, **kw):
        return cpaa_solve(self.handle, p, c, tol, pi, **kw)

    def power_solve(self, p, c, tol, pi, **kw):
        return cpaa_power_solve(self.handle, p, c, tol, pi, **kw)

    def solve_batch(self, B, P, c, tol, PI, **kw):
        return cpaa_solve_batch(self.handle, B, P, c, tol, PI, **kw)

    def close(self):
        if self.handle:
            cpaa_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
