"""Python binding of libcbdfs.so, the batched CB-DFS heuristic library for sm_103a.

Argument marshalling only: every function forwards to the C entry point of the same name
declared in include/cbdfs.h, and raises CbdfsError when it returns a non-zero status.
Arrays may be numpy arrays (host) or torch tensors (host or, for heur_eval_device, CUDA).
There is no fallback: if libcbdfs.so is missing, importing this package fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcbdfs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python paper_2507_11916_b300/build.py`")

_lib = ctypes.CDLL(LIB_PATH)


def load_builder():
    """The build module, loaded by path (see build.py)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("_cbdfs_build", os.path.join(HERE, "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod

# ---- constants (cbdfs.h) ----
CBDFS_OK, CBDFS_EINVAL, CBDFS_ENOMEM, CBDFS_ETIMEDOUT = 0, -1, -2, -3
CBDFS_EDEVICE, CBDFS_ECANCELED, CBDFS_ENOTFOUND = -4, -5, -6
DOM_STP3, DOM_STP4, DOM_RC3 = 0, 1, 2
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
HEAD_REGRESSION, HEAD_CLASSIFIER, HEAD_REAL, HEAD_QUANTILE = 0, 1, 2, 3
LOSS_CE, LOSS_MSE = 0, 1
ALGO_IDA, ALGO_BTS = 0, 1
HEUR_ZERO, HEUR_MD, HEUR_NONE = -1, -2, -100
MAX_ITERS = 256

_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ETIMEDOUT", -4: "EDEVICE", -5: "ECANCELED",
           -6: "ENOTFOUND"}


class CbdfsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget", ctypes.c_size_t),
                ("max_batch", ctypes.c_uint32), ("n_slots", ctypes.c_int),
                ("device_wait_ns", ctypes.c_uint64)]


class NetDesc(ctypes.Structure):
    _fields_ = [("domain", ctypes.c_int), ("n_layers", ctypes.c_int),
                ("dims", ctypes.POINTER(ctypes.c_int)),
                ("weights", ctypes.POINTER(ctypes.POINTER(ctypes.c_float))),
                ("biases", ctypes.POINTER(ctypes.POINTER(ctypes.c_float))),
                ("prec", ctypes.c_int), ("head", ctypes.c_int), ("max_with_md", ctypes.c_int),
                ("act_scales", ctypes.POINTER(ctypes.c_float)), ("h_offset", ctypes.c_float),
                ("quantile", ctypes.c_float)]


class ComboDesc(ctypes.Structure):
    _fields_ = [("domain", ctypes.c_int), ("n_groups", ctypes.c_int),
                ("group_size", ctypes.POINTER(ctypes.c_int)), ("members", ctypes.POINTER(ctypes.c_int)),
                ("add_md", ctypes.c_int)]


class PdbDesc(ctypes.Structure):
    _fields_ = [("domain", ctypes.c_int), ("n_patterns", ctypes.c_int),
                ("k", ctypes.POINTER(ctypes.c_int)), ("tiles", ctypes.POINTER(ctypes.c_int)),
                ("tables", ctypes.POINTER(ctypes.c_void_p)), ("div", ctypes.c_int)]


class SearchCfg(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("work_num", ctypes.c_int), ("d_init", ctypes.c_int),
                ("batch", ctypes.c_uint32), ("timeout_us", ctypes.c_uint32),
                ("complete_final", ctypes.c_int), ("fixed_tree_heur", ctypes.c_int),
                ("bts_n0", ctypes.c_uint64), ("bts_c1", ctypes.c_int), ("bts_c2", ctypes.c_int),
                ("node_limit", ctypes.c_uint64), ("time_limit_s", ctypes.c_double)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("batch", ctypes.c_uint32), ("epochs", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("loss", ctypes.c_int), ("max_steps", ctypes.c_int64)]


class TrainReport(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("samples", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("first_loss", ctypes.c_float), ("last_loss", ctypes.c_float)]


class DriveRequest(ctypes.Structure):
    _fields_ = [("heur_id", ctypes.c_int), ("domain", ctypes.c_int), ("states", ctypes.c_void_p),
                ("g", ctypes.c_void_p), ("bound", ctypes.c_uint32), ("n", ctypes.c_uint32),
                ("h_out", ctypes.c_void_p), ("mask_out", ctypes.c_void_p), ("minf_out", ctypes.c_void_p)]


class Ticket(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int), ("bucket_min", ctypes.c_uint32),
                ("bucket_max", ctypes.c_uint32), ("mem_budget", ctypes.c_size_t),
                ("coalesce", ctypes.c_int), ("direct", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("states", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("states_per_s", ctypes.c_double), ("stage_us_per_launch", ctypes.c_double),
                ("flight_us_per_launch", ctypes.c_double), ("finish_us_per_launch", ctypes.c_double),
                ("replay_us_per_launch", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_int), ("path_len", ctypes.c_int), ("path", ctypes.c_int * 256),
                ("n_iters", ctypes.c_int),
                ("iter_bound", ctypes.c_int64 * MAX_ITERS),
                ("iter_expanded", ctypes.c_int64 * MAX_ITERS),
                ("iter_generated", ctypes.c_int64 * MAX_ITERS),
                ("iter_limit", ctypes.c_int64 * MAX_ITERS),
                ("iter_cut", ctypes.c_int * MAX_ITERS),
                ("expanded", ctypes.c_int64), ("generated", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("evaluated", ctypes.c_int64),
                ("seconds", ctypes.c_double), ("d_init", ctypes.c_int),
                ("work_items", ctypes.c_int64), ("batch_fill_us", ctypes.c_double),
                ("batch_flight_us", ctypes.c_double), ("submit_us", ctypes.c_double),
                ("real_valued", ctypes.c_int), ("iter_bound_real", ctypes.c_double * MAX_ITERS),
                ("batch_hist", ctypes.c_int64 * 16), ("gpu_busy_s", ctypes.c_double)]


_vp, _u64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)
_lib.cbdfs_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(_vp)]
_lib.cbdfs_destroy.argtypes = [_vp]
_lib.cbdfs_server_drive.argtypes = [_vp, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double)]
_lib.cbdfs_debug_withhold_publish.argtypes = [_vp, ctypes.c_int]
_lib.cbdfs_destroy.restype = None
_lib.cbdfs_last_error.restype = ctypes.c_char_p
_lib.cbdfs_mem_used.argtypes = [_vp]
_lib.cbdfs_mem_used.restype = ctypes.c_size_t
_lib.cbdfs_net_load.argtypes = [_vp, ctypes.POINTER(NetDesc), ctypes.POINTER(ctypes.c_int)]
_lib.cbdfs_pdb_load.argtypes = [_vp, ctypes.POINTER(PdbDesc), ctypes.POINTER(ctypes.c_int)]
_lib.cbdfs_combo_load.argtypes = [_vp, ctypes.POINTER(ComboDesc), ctypes.POINTER(ctypes.c_int)]
_lib.pdb_build.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _vp,
                           ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
_lib.heur_submit_batch.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint32,
                                   ctypes.c_uint32, _vp, _vp, _vp, _vp]
_lib.heur_eval_device.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint32,
                                  ctypes.c_uint32, _vp, _vp, _vp, _vp, _vp]
_lib.heur_submit_batch_async.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint32,
                                         ctypes.c_uint32, _vp, _vp, _vp, ctypes.POINTER(Ticket)]
_lib.heur_wait.argtypes = [_vp, Ticket, ctypes.c_uint64]
_lib.heur_submit_batch_real.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_float,
                                        ctypes.c_uint32, _vp, _vp, _vp]
_lib.heur_eval_device_real.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_float,
                                       ctypes.c_uint32, _vp, _vp, _vp, _vp]
_lib.cbdfs_device_status.argtypes = [_vp]
_lib.cbdfs_eval_trace.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint32,
                                  ctypes.c_uint32, _vp, _vp, _vp, _vp, _vp, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int)]
_lib.heur_eval_device_static.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint32,
                                         ctypes.c_uint32, _vp, _vp, _vp, _vp]
_lib.cbdfs_eval_profile.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint32,
                                    ctypes.c_uint32, _vp, _vp, _vp, _vp,
                                    ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]
_FPP = ctypes.POINTER(ctypes.POINTER(ctypes.c_float))
_lib.net_train.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_uint64, ctypes.POINTER(TrainCfg),
                           ctypes.POINTER(TrainReport)]
_lib.cbdfs_train_grad.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_uint32, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_float), _FPP, _FPP]
_lib.cbdfs_net_read.argtypes = [_vp, ctypes.c_int, _FPP, _FPP]
_lib.cbdfs_train_save.argtypes = [_vp, ctypes.c_int, ctypes.c_char_p]
_lib.cbdfs_train_load.argtypes = [_vp, ctypes.c_int, ctypes.c_char_p]
_IP = ctypes.POINTER(ctypes.c_int)
_lib.cbdfs_pdb_file_write.argtypes = [ctypes.c_char_p, ctypes.c_int, _IP, ctypes.c_int, ctypes.c_uint32, _vp,
                                      ctypes.c_uint64]
_lib.cbdfs_pdb_file_read.argtypes = [ctypes.c_char_p, _IP, _IP, _IP, ctypes.POINTER(ctypes.c_uint32), _vp,
                                     ctypes.c_uint64, _u64p]
_lib.cbdfs_gen_walk_states.argtypes = [_vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_int, _vp]
_lib.cbdfs_server_start.argtypes = [_vp, ctypes.POINTER(ServerCfg)]
_lib.cbdfs_server_stop.argtypes = [_vp]
_lib.heur_request_submit.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint32,
                                     ctypes.c_uint32, _vp, _vp, _vp, ctypes.POINTER(Ticket)]
_lib.heur_request_wait.argtypes = [_vp, Ticket, ctypes.c_uint64]
_lib.cbdfs_server_get_stats.argtypes = [_vp, ctypes.POINTER(ServerStats)]
_lib.cbdfs_apply_moves.argtypes = [ctypes.c_int, _u64p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                   _u64p]
_lib.cbdfs_manhattan.argtypes = [ctypes.c_int, ctypes.c_uint64]
_lib.cbdfs_solve.argtypes = [_vp, ctypes.c_int, _u64p, ctypes.c_int, ctypes.c_int,
                             ctypes.POINTER(SearchCfg), ctypes.POINTER(Result)]
_lib.cbdfs_search_defaults.argtypes = [ctypes.POINTER(SearchCfg)]
_lib.cbdfs_search_defaults.restype = None
_lib.cbdfs_cancel.argtypes = [_vp]
_lib.cbdfs_cancel.restype = None

# every symbol include/cbdfs.h declares
EXPORTED = ["cbdfs_create", "cbdfs_destroy", "cbdfs_last_error", "cbdfs_mem_used", "cbdfs_net_load",
            "cbdfs_pdb_load", "cbdfs_combo_load", "pdb_build", "heur_submit_batch", "heur_eval_device",
            "heur_submit_batch_real", "heur_eval_device_real", "heur_eval_device_static",
            "heur_submit_batch_async", "heur_wait",
            "cbdfs_device_status", "cbdfs_debug_withhold_publish", "cbdfs_eval_profile", "cbdfs_eval_trace", "net_train",
            "cbdfs_train_grad", "cbdfs_net_read", "cbdfs_train_save", "cbdfs_train_load",
            "cbdfs_pdb_file_write", "cbdfs_pdb_file_read", "cbdfs_gen_walk_states", "cbdfs_server_start",
            "cbdfs_server_stop", "cbdfs_server_drive", "cbdfs_server_prepare", "cbdfs_server_reset_stats", "heur_request_submit", "heur_request_wait", "cbdfs_server_get_stats", "cbdfs_apply_moves", "cbdfs_manhattan", "cbdfs_solve",
            "cbdfs_search_defaults", "cbdfs_cancel"]


def _check(status):
    if status != CBDFS_OK:
        raise CbdfsError(status, cbdfs_last_error())
    return status


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def cbdfs_last_error() -> str:
    return _lib.cbdfs_last_error().decode()


def cbdfs_create(device=0, mem_budget=0, max_batch=0, n_slots=0, device_wait_ns=0):
    cfg = Config(device, mem_budget, max_batch, n_slots, device_wait_ns)
    h = _vp()
    _check(_lib.cbdfs_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def cbdfs_destroy(ctx):
    _lib.cbdfs_destroy(ctx)


def cbdfs_mem_used(ctx) -> int:
    return _lib.cbdfs_mem_used(ctx)


def cbdfs_net_load(ctx, domain, weights, biases, prec=PREC_BF16, head=HEAD_REGRESSION,
                   max_with_md=0, act_scales=None, h_offset=0.0, quantile=0.0) -> int:
    Ws = [np.ascontiguousarray(w, dtype=np.float32) for w in weights]
    bs = [np.ascontiguousarray(b, dtype=np.float32) for b in biases]
    dims = [Ws[0].shape[1]] + [w.shape[0] for w in Ws]
    FP = ctypes.POINTER(ctypes.c_float)
    wp = (FP * len(Ws))(*(w.ctypes.data_as(FP) for w in Ws))
    bp = (FP * len(bs))(*(b.ctypes.data_as(FP) for b in bs))
    sc = None
    if act_scales is not None:
        sc_arr = np.ascontiguousarray(act_scales, dtype=np.float32)
        sc = sc_arr.ctypes.data_as(FP)
    d = NetDesc(domain, len(Ws), (ctypes.c_int * len(dims))(*dims), wp, bp, prec, head,
                max_with_md, sc, h_offset, quantile)
    out = ctypes.c_int()
    _check(_lib.cbdfs_net_load(ctx, ctypes.byref(d), ctypes.byref(out)))
    return out.value


def cbdfs_pdb_load(ctx, domain, patterns, tables=None, div=1) -> int:
    ks = [len(p) for p in patterns]
    tiles = [t for p in patterns for t in p]
    tabs = None
    if tables is not None:
        tables = [np.ascontiguousarray(t, dtype=np.uint8) for t in tables]
        tabs = (ctypes.c_void_p * len(tables))(*(t.ctypes.data for t in tables))
    d = PdbDesc(domain, len(patterns), (ctypes.c_int * len(ks))(*ks),
                (ctypes.c_int * len(tiles))(*tiles), tabs, int(div))
    out = ctypes.c_int()
    _check(_lib.cbdfs_pdb_load(ctx, ctypes.byref(d), ctypes.byref(out)))
    return out.value


def cbdfs_combo_load(ctx, domain, groups, add_md=False) -> int:
    """A composite heuristic: [MD] + sum over groups of the minimum over each group's member
    heuristic ids (groups: a list of lists of ids)."""
    sizes = [len(g) for g in groups]
    members = [m for g in groups for m in g]
    d = ComboDesc(domain, len(groups), (ctypes.c_int * len(sizes))(*sizes),
                  (ctypes.c_int * max(1, len(members)))(*members), int(bool(add_md)))
    out = ctypes.c_int()
    _check(_lib.cbdfs_combo_load(ctx, ctypes.byref(d), ctypes.byref(out)))
    return out.value


def pdb_build(ctx, domain, tiles) -> np.ndarray:
    """One pattern's table built on the GPU (the cube: tiles 0..7, the 8-corner table)."""
    if domain == DOM_RC3:
        P = 40320 * 2187
    else:
        n = 9 if domain == DOM_STP3 else 16
        P = 1
        for i in range(len(tiles)):
            P *= n - i
    table = np.empty(P, dtype=np.uint8)
    entries = ctypes.c_size_t()
    _check(_lib.pdb_build(ctx, domain, (ctypes.c_int * len(tiles))(*tiles), len(tiles),
                          table.ctypes.data, table.nbytes, ctypes.byref(entries)))
    return table[:entries.value]


def heur_submit_batch(ctx, heur_id, domain, states, g, bound, want_y=False, n_out=1, out=None):
    """Host arrays in, host arrays out: (h uint8[n], mask uint32[ceil(n/32)], minf[, y]).
    out=(h, mask): caller-owned output arrays (contiguous uint8[n], uint32[ceil(n/32)]); with
    page-locked states, g, h and mask the kernels read and write them in place."""
    states = np.ascontiguousarray(states, dtype=np.uint64)
    g = np.ascontiguousarray(g, dtype=np.uint8)
    n = len(g)
    if out is not None:
        h, mask = out
        if h.dtype != np.uint8 or mask.dtype != np.uint32 or len(h) < n or len(mask) < (n + 31) // 32 \
                or not (h.flags.c_contiguous and mask.flags.c_contiguous):
            raise ValueError("out: contiguous uint8[n] and uint32[ceil(n/32)] arrays")
    else:
        h = np.empty(n, dtype=np.uint8)
        mask = np.empty((n + 31) // 32, dtype=np.uint32)
    minf = np.empty(1, dtype=np.uint32)
    y = np.empty((n, n_out), dtype=np.float32) if want_y else None
    _check(_lib.heur_submit_batch(ctx, heur_id, domain, _ptr(states), _ptr(g), bound, n,
                                  _ptr(h), _ptr(mask), _ptr(minf), _ptr(y)))
    return (h, mask, int(minf[0]), y) if want_y else (h, mask, int(minf[0]))


class AsyncBatch:
    """An asynchronous batch: wait() returns (h, mask, minf) once the results are in."""

    def __init__(self, ctx, ticket, keep, h, mask, minf):
        self.ctx, self.ticket, self._keep = ctx, ticket, keep
        self.h, self.mask, self._minf = h, mask, minf

    def wait(self, timeout_us=0):
        _check(_lib.heur_wait(self.ctx, self.ticket, timeout_us))
        return self.h, self.mask, int(self._minf[0])


def heur_submit_batch_async(ctx, heur_id, domain, states, g, bound, out=None) -> AsyncBatch:
    """heur_submit_batch without waiting: the arrays (and out=(h, mask), caller-owned) are kept
    alive by the returned object until its wait()."""
    states = np.ascontiguousarray(states, dtype=np.uint64)
    g = np.ascontiguousarray(g, dtype=np.uint8)
    n = len(g)
    if out is not None:
        h, mask = out
    else:
        h = np.empty(n, dtype=np.uint8)
        mask = np.empty((n + 31) // 32, dtype=np.uint32)
    minf = np.empty(1, dtype=np.uint32)
    t = Ticket()
    _check(_lib.heur_submit_batch_async(ctx, heur_id, domain, _ptr(states), _ptr(g), bound, n, _ptr(h),
                                        _ptr(mask), _ptr(minf), ctypes.byref(t)))
    return AsyncBatch(ctx, t, (states, g), h, mask, minf)


def heur_submit_batch_real(ctx, heur_id, domain, states, g, bound):
    """A real-valued network: (h float32[n], mask uint32[ceil(n/32)], minf float)."""
    states = np.ascontiguousarray(states, dtype=np.uint64)
    g = np.ascontiguousarray(g, dtype=np.uint8)
    n = len(g)
    h = np.empty(n, dtype=np.float32)
    mask = np.empty((n + 31) // 32, dtype=np.uint32)
    minf = np.empty(1, dtype=np.float32)
    _check(_lib.heur_submit_batch_real(ctx, heur_id, domain, _ptr(states), _ptr(g), float(bound), n,
                                       _ptr(h), _ptr(mask), _ptr(minf)))
    return h, mask, float(minf[0])


def heur_eval_device_real(ctx, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf,
                          stream=None):
    """Device tensors: d_h float32[n], d_mask int32[ceil(n/32)], d_minf float32[1]."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(_lib.heur_eval_device_real(ctx, heur_id, domain, _ptr(d_states), _ptr(d_g), float(bound), n,
                                      _ptr(d_h), _ptr(d_mask), _ptr(d_minf), s))


def heur_eval_device(ctx, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf, d_y=None,
                     stream=None):
    """Device tensors in and out; enqueued on `stream` (a torch.cuda.Stream or raw handle)."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(_lib.heur_eval_device(ctx, heur_id, domain, _ptr(d_states), _ptr(d_g), bound, n,
                                 _ptr(d_h), _ptr(d_mask), _ptr(d_minf), _ptr(d_y), s))


def heur_eval_device_static(ctx, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf,
                            stream=None):
    """heur_eval_device without any device allocation in the call: the activation scratch is
    the library's file-scope device array (see include/cbdfs.h for its limit)."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(_lib.heur_eval_device_static(ctx, heur_id, domain, _ptr(d_states), _ptr(d_g), bound, n,
                                        _ptr(d_h), _ptr(d_mask), _ptr(d_minf), s))


def cbdfs_eval_profile(ctx, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf,
                       stream=None):
    """Runs the pipeline once and returns the device milliseconds of each of its kernels."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    ms = (ctypes.c_float * 16)()
    k = ctypes.c_int()
    _check(_lib.cbdfs_eval_profile(ctx, heur_id, domain, _ptr(d_states), _ptr(d_g), bound, n,
                                   _ptr(d_h), _ptr(d_mask), _ptr(d_minf), s, ms, 16, ctypes.byref(k)))
    return list(ms[:k.value])


def cbdfs_eval_trace(ctx, heur_id, domain, d_states, d_g, bound, n, d_h, d_mask, d_minf,
                     d_trace, tiles_per_cta, stream=None) -> int:
    """Runs the pipeline once recording the fused kernel's tile timeline into d_trace (a CUDA
    uint64/int64 tensor of at least SMs x tiles_per_cta x 8); returns the CTA count."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    k = ctypes.c_int()
    _check(_lib.cbdfs_eval_trace(ctx, heur_id, domain, _ptr(d_states), _ptr(d_g), bound, n,
                                 _ptr(d_h), _ptr(d_mask), _ptr(d_minf), s, _ptr(d_trace),
                                 tiles_per_cta, ctypes.byref(k)))
    return k.value


def cbdfs_debug_withhold_publish(ctx, row_block: int) -> None:
    _check(_lib.cbdfs_debug_withhold_publish(ctx, row_block))


def cbdfs_device_status(ctx) -> int:
    r = _lib.cbdfs_device_status(ctx)
    if r < 0:
        _check(r)
    return r


def _float_ptrs(arrays):
    FP = ctypes.POINTER(ctypes.c_float)
    return (FP * len(arrays))(*(a.ctypes.data_as(FP) for a in arrays))


def _net_shapes(ctx_dims):
    return [(ctx_dims[l + 1], ctx_dims[l]) for l in range(len(ctx_dims) - 1)]


def net_train(ctx, heur_id, states, labels, batch=8192, epochs=1, lr=1e-3, beta1=0.9, beta2=0.999,
              eps=1e-8, seed=0, loss=LOSS_CE, max_steps=0) -> dict:
    states = np.ascontiguousarray(states, dtype=np.uint64)
    labels = np.ascontiguousarray(labels, dtype=np.uint8)
    cfg = TrainCfg(lr, beta1, beta2, eps, batch, epochs, seed, loss, max_steps)
    rep = TrainReport()
    _check(_lib.net_train(ctx, heur_id, _ptr(states), _ptr(labels), len(labels), ctypes.byref(cfg),
                          ctypes.byref(rep)))
    return {name: getattr(rep, name) for name, _ in TrainReport._fields_}


def cbdfs_train_grad(ctx, heur_id, states, labels, dims, loss=LOSS_CE):
    """(loss, [dW_l], [db_l]) of the mean loss over the batch at the current weights."""
    states = np.ascontiguousarray(states, dtype=np.uint64)
    labels = np.ascontiguousarray(labels, dtype=np.uint8)
    gw = [np.zeros((o, i), np.float32) for o, i in _net_shapes(dims)]
    gb = [np.zeros(o, np.float32) for o, _ in _net_shapes(dims)]
    out = ctypes.c_float()
    _check(_lib.cbdfs_train_grad(ctx, heur_id, _ptr(states), _ptr(labels), len(labels), loss,
                                 ctypes.byref(out), _float_ptrs(gw), _float_ptrs(gb)))
    return out.value, gw, gb


def cbdfs_train_save(ctx, heur_id, path):
    """The network's training state (masters, Adam moments, step) to a checkpoint file."""
    _check(_lib.cbdfs_train_save(ctx, heur_id, os.fsencode(path)))


def cbdfs_train_load(ctx, heur_id, path):
    """A checkpoint back into the network: net_train continues from it."""
    _check(_lib.cbdfs_train_load(ctx, heur_id, os.fsencode(path)))


def cbdfs_pdb_file_write(path, domain, tiles, table, div=1):
    """One pattern's table (uint8) to a PDB file with its pattern and hash."""
    tiles = [int(t) for t in tiles]
    table = np.ascontiguousarray(table, dtype=np.uint8)
    _check(_lib.cbdfs_pdb_file_write(os.fsencode(path), domain, (ctypes.c_int * len(tiles))(*tiles), len(tiles),
                                     div, _ptr(table), len(table)))


def cbdfs_pdb_file_read(path):
    """(domain, tiles, div, table) of a PDB file; the table's hash is checked."""
    dom, k, div = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint32()
    tiles = (ctypes.c_int * 16)()
    entries = ctypes.c_uint64()
    p = os.fsencode(path)
    _check(_lib.cbdfs_pdb_file_read(p, ctypes.byref(dom), tiles, ctypes.byref(k), ctypes.byref(div), None, 0,
                                    ctypes.byref(entries)))
    table = np.empty(entries.value, dtype=np.uint8)
    _check(_lib.cbdfs_pdb_file_read(p, ctypes.byref(dom), tiles, ctypes.byref(k), ctypes.byref(div), _ptr(table),
                                    len(table), ctypes.byref(entries)))
    return dom.value, list(tiles[:k.value]), div.value, table


def cbdfs_net_read(ctx, heur_id, dims):
    Ws = [np.zeros((o, i), np.float32) for o, i in _net_shapes(dims)]
    bs = [np.zeros(o, np.float32) for o, _ in _net_shapes(dims)]
    _check(_lib.cbdfs_net_read(ctx, heur_id, _float_ptrs(Ws), _float_ptrs(bs)))
    return Ws, bs


def cbdfs_gen_walk_states(ctx, domain, tag, first, n, max_len) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _check(_lib.cbdfs_gen_walk_states(ctx, domain, tag, first, n, max_len, _ptr(out)))
    return out


def cbdfs_server_start(ctx, max_inflight=0, bucket_min=32, bucket_max=4096, mem_budget=0, coalesce=1, direct=0):
    _check(_lib.cbdfs_server_start(ctx, ctypes.byref(ServerCfg(max_inflight, bucket_min, bucket_max,
                                                               mem_budget, coalesce, direct))))


def cbdfs_server_stop(ctx):
    _check(_lib.cbdfs_server_stop(ctx))


def cbdfs_server_prepare(ctx, heur_id, domain):
    _check(_lib.cbdfs_server_prepare(ctx, heur_id, domain))


def cbdfs_server_reset_stats(ctx):
    _check(_lib.cbdfs_server_reset_stats(ctx))


def cbdfs_server_drive(ctx, reqs, threads=64, depth=1):
    """reqs: (heur_id, domain, states, g, bound) tuples, driven through the running server by
    native client threads.  Returns (seconds, [(h, mask, minf), ...]) in request order."""
    keep, outs = [], []
    arr = (DriveRequest * max(1, len(reqs)))()
    for k, (heur, dom, s, g, bound) in enumerate(reqs):
        s = np.ascontiguousarray(s, dtype=np.uint64)
        g = np.ascontiguousarray(g, dtype=np.uint8)
        n = len(g)
        # result buffers written once here, so that the drive does not time first-touch faults
        h = np.full(n, 0xFF, np.uint8)
        m = np.full((n + 31) // 32, 0xFFFFFFFF, np.uint32)
        f = np.full(1, 0xFFFFFFFF, np.uint32)
        keep.append((s, g))
        outs.append((h, m, f))
        arr[k] = DriveRequest(heur, dom, _ptr(s), _ptr(g), bound, n, _ptr(h), _ptr(m), _ptr(f))
    sec = ctypes.c_double()
    _check(_lib.cbdfs_server_drive(ctx, arr, len(reqs), threads, depth, ctypes.byref(sec)))
    return sec.value, [(h, m, int(f[0])) for h, m, f in outs]


class Request:
    """A queued request; its result arrays are owned here until wait() returns."""

    def __init__(self, ctx, heur_id, domain, states, g, bound):
        self.ctx = ctx
        self.states = np.ascontiguousarray(states, dtype=np.uint64)
        self.g = np.ascontiguousarray(g, dtype=np.uint8)
        n = len(self.g)
        self.h = np.empty(n, dtype=np.uint8)
        self.mask = np.empty((n + 31) // 32, dtype=np.uint32)
        self.minf = np.empty(1, dtype=np.uint32)
        self.ticket = Ticket()
        _check(_lib.heur_request_submit(ctx, heur_id, domain, _ptr(self.states), _ptr(self.g), bound, n,
                                        _ptr(self.h), _ptr(self.mask), _ptr(self.minf),
                                        ctypes.byref(self.ticket)))

    def wait(self, timeout_us=60_000_000):
        _check(_lib.heur_request_wait(self.ctx, self.ticket, timeout_us))
        return self.h, self.mask, int(self.minf[0])


def heur_request_submit(ctx, heur_id, domain, states, g, bound) -> Request:
    return Request(ctx, heur_id, domain, states, g, bound)


def heur_request_wait(ctx, req: Request, timeout_us=60_000_000):
    return req.wait(timeout_us)


def cbdfs_server_get_stats(ctx) -> dict:
    st = ServerStats()
    _check(_lib.cbdfs_server_get_stats(ctx, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


def cbdfs_apply_moves(domain, start, moves):
    """start: an int (STP) or a pair of ints (RC); returns the same shape."""
    words = list(start) if isinstance(start, (tuple, list)) else [int(start)]
    inp = (ctypes.c_uint64 * 2)(*(words + [0] * (2 - len(words))))
    out = (ctypes.c_uint64 * 2)()
    mv = (ctypes.c_int * max(1, len(moves)))(*moves)
    _check(_lib.cbdfs_apply_moves(domain, inp, mv, len(moves), out))
    return (out[0], out[1]) if domain == DOM_RC3 else out[0]


def cbdfs_manhattan(domain, state) -> int:
    r = _lib.cbdfs_manhattan(domain, ctypes.c_uint64(int(state)))
    return _check(r) if r < 0 else r


def cbdfs_search_defaults() -> dict:
    c = SearchCfg()
    _lib.cbdfs_search_defaults(ctypes.byref(c))
    return {name: getattr(c, name) for name, _ in SearchCfg._fields_}


def cbdfs_solve(ctx, domain, start, algo=ALGO_IDA, heur_id=HEUR_MD, partial_ok=False, **cfg) -> dict:
    """Returns the result as a dict.  With partial_ok, a search stopped by its node or time
    limit returns its partial counts with "status" set instead of raising."""
    c = SearchCfg()
    _lib.cbdfs_search_defaults(ctypes.byref(c))
    for k, v in cfg.items():
        if not hasattr(c, k):
            raise TypeError(f"unknown search option {k}")
        setattr(c, k, v)
    words = list(start) if isinstance(start, (tuple, list)) else [int(start)]
    st = (ctypes.c_uint64 * 2)(*(words + [0] * (2 - len(words))))
    r = Result()
    status = _lib.cbdfs_solve(ctx, domain, st, algo, heur_id, ctypes.byref(c), ctypes.byref(r))
    if not (partial_ok and status in (CBDFS_ETIMEDOUT, CBDFS_ECANCELED)):
        _check(status)
    k = min(r.n_iters, MAX_ITERS)
    return dict(status=status, cost=r.cost, path=list(r.path[:r.path_len]),
                iters=[(r.iter_bound_real[i] if r.real_valued else r.iter_bound[i], r.iter_expanded[i],
                        r.iter_generated[i]) for i in range(k)],
                real_valued=bool(r.real_valued),
                iter_limit=list(r.iter_limit[:k]), iter_cut=list(r.iter_cut[:k]),
                n_iters=r.n_iters, expanded=r.expanded, generated=r.generated,
                batches=r.batches, evaluated=r.evaluated, seconds=r.seconds, d_init=r.d_init,
                work_items=r.work_items, batch_fill_us=r.batch_fill_us,
                batch_flight_us=r.batch_flight_us, submit_us=r.submit_us, batch_hist=list(r.batch_hist),
                gpu_busy_s=r.gpu_busy_s)


def cbdfs_cancel(ctx):
    _lib.cbdfs_cancel(ctx)
