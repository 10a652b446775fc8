"""Python binding of liblr.so, the GB300 list-ranking library.

Thin ctypes marshalling over the C ABI in include/lr.h: torch tensors supply
device memory and streams, every step of the ranking runs in the library's
CUDA kernels.  There is no CPU fallback: if the shared library is missing or
cannot load, importing the ranking functions raises.

    import paper_2606_09318_gb300 as lr
    rank = lr.rank(succ)                      # succ: cuda uint32/int32 tensor
    rank = lr.rank(succ, weight)              # int64 weights -> int64 ranks
    rank = lr.rank_batch(offsets, succ, w)    # many lists, one launch sequence
"""
import ctypes
import os
import threading

__all__ = [
    "LRError", "Tuning", "load", "lib_path", "rank", "rank_ex", "rank_batch", "rank_host",
    "rank_batch_ptrs", "device_status", "workspace_size", "status_string", "version", "profile_enable",
    "profile_read", "kernel_launch_count", "probe_memory", "Server", "STATUS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
# LR_DEBUG_LIB=1: the debug build (build.py, debug=True), whose kernels check
# the indices they derive and report a failed check instead of faulting
_LIB_PATH = (os.path.join(_HERE, "_build_debug", "liblr_debug.so") if os.environ.get("LR_DEBUG_LIB") == "1"
             else os.path.join(_HERE, "_build", "liblr.so"))

STATUS = {
    0: "LR_OK", 1: "LR_ERR_INVALID_ARGUMENT", 2: "LR_ERR_OUT_OF_RANGE", 3: "LR_ERR_CYCLE",
    4: "LR_ERR_NOT_A_LIST", 5: "LR_ERR_OUT_OF_MEMORY", 6: "LR_ERR_BUDGET", 7: "LR_ERR_TIMEOUT",
    8: "LR_ERR_CUDA", 9: "LR_ERR_CAPACITY", 10: "LR_ERR_NOT_FOUND", 11: "LR_ERR_CANCELLED",
    12: "LR_ERR_CAPTURE",
    13: "LR_ERR_INTERNAL",
}
LR_NONE, LR_I32, LR_I64 = 0, 1, 2


class LRError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = int(code)
        self.name = STATUS.get(self.code, "LR_ERR_%d" % self.code)
        super().__init__("%s%s" % (self.name, (": " + what) if what else ""))


class Tuning(ctypes.Structure):
    _fields_ = [("f0_inv", ctypes.c_uint32), ("f_inv", ctypes.c_uint32), ("cutoff", ctypes.c_uint32),
                ("chase_block", ctypes.c_uint32), ("chase_ctas", ctypes.c_uint32),
                ("algorithm", ctypes.c_uint32), ("contract", ctypes.c_uint32),
                ("spawn", ctypes.c_uint32), ("chase0", ctypes.c_uint32)]


ALGO_SRS, ALGO_WYLLIE = 0, 1
CONTRACT_AUTO, CONTRACT_OFF, CONTRACT_ON = 0, 1, 2
CHASE0_AUTO, CHASE0_EXCHANGE, CHASE0_LOG = 0, 1, 2


class _Opts(ctypes.Structure):
    _fields_ = [("wtype", ctypes.c_int), ("rtype", ctypes.c_int), ("tuning", ctypes.POINTER(Tuning)),
                ("workspace", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t),
                ("validate", ctypes.c_int32), ("sync", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("max_lists", ctypes.c_int64), ("n_total", ctypes.c_int64)]


class _Outputs(ctypes.Structure):
    _fields_ = [("term", ctypes.c_void_p), ("prefix", ctypes.c_void_p),
                ("inclusive_tail", ctypes.c_int32)]


class _TuneEntry(ctypes.Structure):
    _fields_ = [("log2n", ctypes.c_int32), ("weighted", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("tuning", Tuning), ("ms", ctypes.c_float)]


class _Profile(ctypes.Structure):
    _fields_ = [("ms_prep", ctypes.c_double), ("ms_select", ctypes.c_double),
                ("ms_chase0", ctypes.c_double), ("ms_chase_rest", ctypes.c_double),
                ("ms_base", ctypes.c_double), ("ms_finalize", ctypes.c_double),
                ("calls", ctypes.c_int64), ("chase0_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("elements", ctypes.c_int64),
                ("chase0_log_launches", ctypes.c_int64)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("n_streams", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_batch_elems", ctypes.c_int64),
                ("device", ctypes.c_int32), ("plain", ctypes.c_int32), ("alone_min_n", ctypes.c_int64)]


class _Request(ctypes.Structure):
    _fields_ = [("succ", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("rank", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("wtype", ctypes.c_int), ("rtype", ctypes.c_int),
                ("on_device", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("t_submit_ms", ctypes.c_double),
                ("t_admit_ms", ctypes.c_double), ("t_launch_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("elements", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("elements_per_s", ctypes.c_double), ("peak_resident_bytes", ctypes.c_size_t),
                ("ranked_alone", ctypes.c_int64)]


class _ProbeResult(ctypes.Structure):
    _fields_ = [("copy_gbs", ctypes.c_double), ("gather_gsteps", ctypes.c_double),
                ("gather_xchg_gsteps", ctypes.c_double), ("footprint_bytes", ctypes.c_size_t),
                ("indep_gather_gsteps", ctypes.c_double), ("region_gather_gsteps", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
_V, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_SIGS = {
    "lr_opts_default": (None, [ctypes.POINTER(_Opts)]),
    "lr_rank": (ctypes.c_int, [_V, _V, _I64, _V, _V]),
    "lr_rank_ex": (ctypes.c_int, [_V, _V, _I64, _V, ctypes.POINTER(_Opts), _V]),
    "lr_rank_batch": (ctypes.c_int, [_V, _V, _V, _V, _I32, _V]),
    "lr_rank_batch_ex": (ctypes.c_int, [_V, _V, _V, _V, _I32, ctypes.POINTER(_Opts), _V]),
    "lr_rank_batch_ptrs": (ctypes.c_int, [_V, _V, _V, _V, _I32, ctypes.POINTER(_Opts), _V]),
    "lr_rank_host": (ctypes.c_int, [_V, _V, _I64, _V, ctypes.POINTER(_Opts), _V]),
    "lr_rank_host_async": (ctypes.c_int, [_V, _V, _I64, _V, ctypes.POINTER(_Opts), _V]),
    "lr_workspace_size": (_SZ, [_I64, _I32, ctypes.POINTER(_Opts)]),
    "lr_workspace_size_outputs": (_SZ, [_I64, _I32, ctypes.POINTER(_Outputs), ctypes.POINTER(_Opts)]),
    "lr_rank_outputs": (ctypes.c_int, [_V, _V, _I64, _V, ctypes.POINTER(_Outputs),
                                       ctypes.POINTER(_Opts), _V]),
    "lr_rank_batch_outputs": (ctypes.c_int, [_V, _V, _V, _V, _I32, ctypes.POINTER(_Outputs),
                                             ctypes.POINTER(_Opts), _V]),
    "lr_get_device_status": (ctypes.c_int, [_V]),
    "lr_level_sizes": (_I32, [_V, ctypes.POINTER(_I64), _I32]),
    "lr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lr_version": (ctypes.c_char_p, []),
    "lr_profile_enable": (ctypes.c_int, [_I32]),
    "lr_profile_read": (ctypes.c_int, [ctypes.POINTER(_Profile), _I32]),
    "lr_kernel_launch_count": (_I64, []),
    "lr_probe_memory": (ctypes.c_int, [_V, _SZ, ctypes.POINTER(_ProbeResult), _V]),
    "lr_server_config_default": (None, [ctypes.POINTER(_ServerConfig)]),
    "lr_server_create": (ctypes.c_int, [ctypes.POINTER(_ServerConfig), ctypes.POINTER(_V)]),
    "lr_server_submit": (ctypes.c_int, [_V, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]),
    "lr_server_wait": (ctypes.c_int, [_V, ctypes.c_uint64, _I64, ctypes.POINTER(_Result)]),
    "lr_server_stats_get": (ctypes.c_int, [_V, ctypes.POINTER(_ServerStats)]),
    "lr_server_destroy": (None, [_V]),
    "lr_autotune": (ctypes.c_int, [_V, _V, _V, _I64, _I32, ctypes.POINTER(_Opts), _V,
                                   ctypes.POINTER(Tuning)]),
    "lr_autotune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "lr_autotune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "lr_autotune_entries": (_I32, [ctypes.POINTER(_TuneEntry), _I32]),
    "lr_autotune_clear": (None, []),
    "lr_pipeline_create": (ctypes.c_int, [_I64, ctypes.POINTER(_Opts), _I32, ctypes.POINTER(_V)]),
    "lr_pipeline_submit": (ctypes.c_int, [_V, _V, _V, _I64, _V]),
    "lr_pipeline_wait": (ctypes.c_int, [_V, ctypes.POINTER(_I64)]),
    "lr_pipeline_destroy": (None, [_V]),
}


def lib_path():
    return _LIB_PATH


def load():
    """Load liblr.so (built by build.py / __graft_entry__.build()); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise ImportError("liblr.so is not built (%s); run paper_2606_09318_gb300/build.py"
                                  % _LIB_PATH)
            lib = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def status_string(code):
    return load().lr_status_string(int(code)).decode()


def version():
    return load().lr_version().decode()


def _check(code, what=""):
    if code != 0:
        raise LRError(code, what)


# ---------------------------------------------------------------- torch glue
def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name, dtypes):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype not in dtypes:
        raise TypeError("%s has dtype %s, expected one of %s" % (name, t.dtype, dtypes))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _succ_dtypes():
    torch = _torch()
    return tuple(d for d in (getattr(torch, "uint32", None), torch.int32) if d is not None)


def _wcode(weight):
    torch = _torch()
    if weight is None:
        return LR_NONE
    return {torch.int32: LR_I32, torch.int64: LR_I64}[weight.dtype]


def _opts(wtype, rtype, validate=False, seed=0x5EED, max_lists=0, tuning=None, sync=False,
          n_total=0, workspace=None):
    o = _Opts()
    load().lr_opts_default(ctypes.byref(o))
    o.wtype, o.rtype = wtype, rtype
    o.validate = 1 if validate else 0
    o.sync = 1 if sync else 0
    o.seed = int(seed) & (2**64 - 1)
    o.max_lists = int(max_lists)
    o.n_total = int(n_total)
    if tuning is not None:
        o.tuning = ctypes.pointer(tuning)
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.ws_bytes = workspace.numel() * workspace.element_size()
    return o


def _rank_dtype(weight, rank_dtype):
    torch = _torch()
    if rank_dtype is None:
        return torch.int32 if weight is None else torch.int64
    return rank_dtype


def rank_ex(succ, weight=None, out=None, rank_dtype=None, validate=False, seed=0x5EED,
            max_lists=0, tuning=None, sync=True, stream=None, workspace=None):
    """Rank a successor array held in a CUDA tensor.

    Returns the rank tensor (int32 when unweighted, int64 when weighted,
    unless rank_dtype says otherwise).  With sync=True the device status is
    checked and errors raise LRError; with sync=False the call only queues
    work on the stream (use device_status() later).
    """
    torch = _torch()
    lib = load()
    rdt = _rank_dtype(weight, rank_dtype)
    sp = _dev_ptr(succ, "succ", _succ_dtypes())
    n = succ.numel()
    wp = None if weight is None else _dev_ptr(weight, "weight", (torch.int32, torch.int64))
    if weight is not None and weight.numel() != n:
        raise ValueError("weight and succ differ in length")
    if out is None:
        out = torch.empty(n, dtype=rdt, device=succ.device)
    rp = _dev_ptr(out, "out", (torch.int32, torch.int64))
    if out.numel() != n:
        raise ValueError("out has the wrong length")
    o = _opts(_wcode(weight), LR_I32 if out.dtype == torch.int32 else LR_I64, validate, seed,
              max_lists, tuning, sync, workspace=workspace)
    code = lib.lr_rank_ex(sp, wp, n, rp, ctypes.byref(o), _stream_handle(stream))
    _check(code, "lr_rank_ex")
    return out


def rank(succ, weight=None, out=None, stream=None, **kw):
    """The lr_rank entry point (waits for the device and checks the status)."""
    return rank_ex(succ, weight, out=out, stream=stream, **kw)


def rank_batch(offsets, succ, weight=None, out=None, rank_dtype=None, validate=False,
               seed=0x5EED, max_lists=0, n_total=0, tuning=None, sync=True, stream=None,
               workspace=None):
    """Rank k instances back to back (offsets: CUDA int64[k+1], local ids)."""
    torch = _torch()
    lib = load()
    op = _dev_ptr(offsets, "offsets", (torch.int64,))
    k = offsets.numel() - 1
    rdt = _rank_dtype(weight, rank_dtype)
    sp = _dev_ptr(succ, "succ", _succ_dtypes())
    wp = None if weight is None else _dev_ptr(weight, "weight", (torch.int32, torch.int64))
    if out is None:
        out = torch.empty(succ.numel(), dtype=rdt, device=succ.device)
    rp = _dev_ptr(out, "out", (torch.int32, torch.int64))
    o = _opts(_wcode(weight), LR_I32 if out.dtype == torch.int32 else LR_I64, validate, seed,
              max_lists, tuning, sync, n_total=n_total or succ.numel(), workspace=workspace)
    code = lib.lr_rank_batch_ex(op, sp, wp, rp, k, ctypes.byref(o), _stream_handle(stream))
    _check(code, "lr_rank_batch_ex")
    return out


def rank_batch_ptrs(succs, weights=None, outs=None, rank_dtype=None, validate=False,
                    seed=0x5EED, max_lists=0, tuning=None, sync=True, stream=None):
    """Rank k lists held in separate CUDA tensors as one forest in one launch
    sequence (the lr_rank_batch_ptrs entry point).

    succs: CUDA int32/uint32 tensors of local successors, one per instance;
    weights: None or one int32/int64 tensor per instance (one dtype);
    outs: None or one rank tensor per instance.  Returns the rank tensors.
    """
    torch = _torch()
    lib = load()
    succs = list(succs)
    k = len(succs)
    if weights is not None:
        weights = list(weights)
        if len(weights) != k:
            raise ValueError("weights and succs differ in count")
    if outs is not None:
        outs = list(outs)
        if len(outs) != k:
            raise ValueError("outs and succs differ in count")
    if k == 0:
        return []
    device = succs[0].device
    wdt = None if weights is None else weights[0].dtype
    rdt = _rank_dtype(None if weights is None else weights[0], rank_dtype)
    sizes, sp, wp, rp = [], [], [], []
    if outs is None:
        outs = [torch.empty(t.numel(), dtype=rdt, device=device) for t in succs]
    for j, t in enumerate(succs):
        if t.device != device:
            raise ValueError("every tensor must be on the same device")
        sp.append(_dev_ptr(t, "succs[%d]" % j, _succ_dtypes()).value or 0)
        sizes.append(t.numel())
        if weights is not None:
            w = weights[j]
            if w.dtype != wdt or w.numel() != t.numel():
                raise ValueError("weights[%d] has another dtype or length" % j)
            wp.append(_dev_ptr(w, "weights[%d]" % j, (torch.int32, torch.int64)).value or 0)
        o = outs[j]
        if o.dtype != outs[0].dtype or o.numel() != t.numel():
            raise ValueError("outs[%d] has another dtype or length" % j)
        rp.append(_dev_ptr(o, "outs[%d]" % j, (torch.int32, torch.int64)).value or 0)
    offsets = torch.zeros(k + 1, dtype=torch.int64)
    offsets[1:] = torch.cumsum(torch.tensor(sizes, dtype=torch.int64), 0)
    if stream is None:
        stream = torch.cuda.current_stream(device)
    with torch.cuda.stream(stream):          # the tables are copied on the stream that reads them
        d_off = offsets.to(device)
        d_sp = torch.tensor(sp, dtype=torch.int64).to(device)
        d_rp = torch.tensor(rp, dtype=torch.int64).to(device)
        d_wp = None if weights is None else torch.tensor(wp, dtype=torch.int64).to(device)
    wcode = LR_NONE if weights is None else {torch.int32: LR_I32, torch.int64: LR_I64}[wdt]
    o = _opts(wcode, LR_I32 if outs[0].dtype == torch.int32 else LR_I64, validate, seed,
              max_lists, tuning, sync, n_total=int(offsets[-1]))
    code = lib.lr_rank_batch_ptrs(ctypes.c_void_p(d_off.data_ptr()), ctypes.c_void_p(d_sp.data_ptr()),
                                  None if d_wp is None else ctypes.c_void_p(d_wp.data_ptr()),
                                  ctypes.c_void_p(d_rp.data_ptr()), k, ctypes.byref(o), _stream_handle(stream))
    _check(code, "lr_rank_batch_ptrs")
    return outs


def _outputs(succ, rdt, term, prefix, inclusive_tail):
    """Allocate (or check) the extra output tensors; returns (struct, term, prefix)."""
    torch = _torch()
    o = _Outputs()
    t = p = None
    if term is not None and term is not False:
        t = torch.empty(succ.numel(), dtype=torch.int32, device=succ.device) if term is True else term
        o.term = _dev_ptr(t, "term", (torch.int32,) + tuple(d for d in (getattr(torch, "uint32", None),) if d))
    if prefix is not None and prefix is not False:
        p = torch.empty(succ.numel(), dtype=rdt, device=succ.device) if prefix is True else prefix
        o.prefix = _dev_ptr(p, "prefix", (rdt,))
    o.inclusive_tail = 1 if inclusive_tail else 0
    for a in (t, p):
        if a is not None and a.numel() != succ.numel():
            raise ValueError("extra output has the wrong length")
    return o, t, p


def rank_outputs(succ, weight=None, term=True, prefix=False, inclusive_tail=False, out=None,
                 rank_dtype=None, validate=False, seed=0x5EED, max_lists=0, tuning=None, sync=True,
                 stream=None, workspace=None):
    """Rank plus the other outputs of Section 1.1 (lr_rank_outputs): term /
    prefix may be True (allocate), a CUDA tensor to fill, or False/None.
    Returns (rank, term, prefix); term holds int32 views of the uint32 ids."""
    torch = _torch()
    lib = load()
    rdt = out.dtype if out is not None else _rank_dtype(weight, rank_dtype)
    sp = _dev_ptr(succ, "succ", _succ_dtypes())
    n = succ.numel()
    wp = None if weight is None else _dev_ptr(weight, "weight", (torch.int32, torch.int64))
    if out is None:
        out = torch.empty(n, dtype=rdt, device=succ.device)
    rp = _dev_ptr(out, "out", (torch.int32, torch.int64))
    outs, t, p = _outputs(succ, rdt, term, prefix, inclusive_tail)
    o = _opts(_wcode(weight), LR_I32 if rdt == torch.int32 else LR_I64, validate, seed,
              max_lists, tuning, sync, workspace=workspace)
    code = lib.lr_rank_outputs(sp, wp, n, rp, ctypes.byref(outs), ctypes.byref(o), _stream_handle(stream))
    _check(code, "lr_rank_outputs")
    return out, t, p


def rank_batch_outputs(offsets, succ, weight=None, term=True, prefix=False, inclusive_tail=False,
                       out=None, rank_dtype=None, validate=False, seed=0x5EED, max_lists=0,
                       n_total=0, tuning=None, sync=True, stream=None, workspace=None):
    """Batched rank_outputs (lr_rank_batch_outputs); terminal ids are local."""
    torch = _torch()
    lib = load()
    op = _dev_ptr(offsets, "offsets", (torch.int64,))
    k = offsets.numel() - 1
    rdt = out.dtype if out is not None else _rank_dtype(weight, rank_dtype)
    sp = _dev_ptr(succ, "succ", _succ_dtypes())
    wp = None if weight is None else _dev_ptr(weight, "weight", (torch.int32, torch.int64))
    if out is None:
        out = torch.empty(succ.numel(), dtype=rdt, device=succ.device)
    rp = _dev_ptr(out, "out", (torch.int32, torch.int64))
    outs, t, p = _outputs(succ, rdt, term, prefix, inclusive_tail)
    o = _opts(_wcode(weight), LR_I32 if rdt == torch.int32 else LR_I64, validate, seed,
              max_lists, tuning, sync, n_total=n_total or succ.numel(), workspace=workspace)
    code = lib.lr_rank_batch_outputs(op, sp, wp, rp, k, ctypes.byref(outs), ctypes.byref(o),
                                     _stream_handle(stream))
    _check(code, "lr_rank_batch_outputs")
    return out, t, p


def rank_host(succ, weight=None, out=None, rank_dtype=None, validate=False, seed=0x5EED,
              max_lists=0, stream=None, wait=True):
    """End-to-end form on host tensors / numpy arrays: copy in, rank, copy out.

    wait=False enqueues everything on `stream` and returns at once (the
    lr_rank_host_async entry point); `out` is valid after the stream is
    synchronised, and device_status(stream) gives the status."""
    import numpy as np
    torch = _torch()
    lib = load()

    def host_ptr(a):
        if isinstance(a, torch.Tensor):
            assert not a.is_cuda and a.is_contiguous()
            return ctypes.c_void_p(a.data_ptr()), a.numel()
        a = np.ascontiguousarray(a)
        return a.ctypes.data_as(ctypes.c_void_p), a.size

    sp, n = host_ptr(succ)
    wp = None if weight is None else host_ptr(weight)[0]
    if weight is None:
        wt = LR_NONE
    else:
        wdt = weight.dtype
        wt = LR_I32 if wdt in (torch.int32, np.int32, np.dtype(np.int32)) else LR_I64
    if out is None:
        rdt = rank_dtype or (np.int32 if weight is None else np.int64)
        out = np.empty(n, dtype=rdt)
    rp = host_ptr(out)[0]
    o = _opts(wt, LR_I32 if out.dtype in (np.int32, torch.int32) else LR_I64, validate, seed, max_lists)
    fn = lib.lr_rank_host if wait else lib.lr_rank_host_async
    code = fn(sp, wp, n, rp, ctypes.byref(o), _stream_handle(stream))
    _check(code, "lr_rank_host" if wait else "lr_rank_host_async")
    return out


def level_sizes(stream=None):
    """Sizes of the recursion levels of the last ruling-set call on `stream`
    (waits for it): [n, rulers at level 1, ...]."""
    arr = (_I64 * 16)()
    cnt = load().lr_level_sizes(_stream_handle(stream), arr, 16)
    if cnt < 0:
        raise LRError(8, "lr_level_sizes")
    return [int(x) for x in arr[:cnt]]


def device_status(stream=None):
    """Wait for the stream; return the status code of its last call (0 = OK)."""
    return load().lr_get_device_status(_stream_handle(stream))


def workspace_size(n_total, k=0, weighted=False, rank64=None, max_lists=0, tuning=None,
                   term=False, prefix=False, inclusive_tail=False):
    """lr_workspace_size (or lr_workspace_size_outputs when extra outputs
    are named: only whether each is asked for matters)."""
    if rank64 is None:
        rank64 = weighted
    o = _Opts()
    load().lr_opts_default(ctypes.byref(o))
    o.wtype = LR_I64 if weighted else LR_NONE
    o.rtype = LR_I64 if rank64 else LR_I32
    o.max_lists = int(max_lists)
    if tuning is not None:
        o.tuning = ctypes.pointer(tuning)
    if term or prefix or inclusive_tail:
        outs = _Outputs()
        outs.term = 1 if term else None        # only non-NULL-ness is read
        outs.prefix = 1 if prefix else None
        outs.inclusive_tail = 1 if inclusive_tail else 0
        return int(load().lr_workspace_size_outputs(int(n_total), int(k), ctypes.byref(outs),
                                                    ctypes.byref(o)))
    return int(load().lr_workspace_size(int(n_total), int(k), ctypes.byref(o)))


def profile_enable(on=True):
    _check(load().lr_profile_enable(1 if on else 0))


def profile_read(reset=True):
    p = _Profile()
    _check(load().lr_profile_read(ctypes.byref(p), 1 if reset else 0))
    return {f: getattr(p, f) for f, _ in _Profile._fields_}


def kernel_launch_count():
    return int(load().lr_kernel_launch_count())


def probe_memory(buf, stream=None):
    """Random-access and streaming ceilings measured on a CUDA byte buffer
    (contents destroyed); see lr_probe_memory in include/lr.h."""
    r = _ProbeResult()
    _check(load().lr_probe_memory(ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(),
                                  ctypes.byref(r), _stream_handle(stream)), "lr_probe_memory")
    return {f: getattr(r, f) for f, _ in _ProbeResult._fields_}


def autotune(n_total=None, k=0, succ=None, weight=None, offsets=None, wtype=None, rank_dtype=None,
             max_lists=0, validate=False, stream=None):
    """Autotune the recursion for one input shape (lr_autotune).  With succ
    (a CUDA tensor; offsets for a batch) the caller's data is used, else a
    synthetic random list (k == 0) or k equal random instances of n_total
    elements with weights of wtype ("int32" / "int64" / None).  Returns the
    winning Tuning; later calls of the same (log2 n, weighted, batched) shape
    that pass no tuning use it."""
    torch = _torch()
    lib = load()
    if succ is not None:
        n_total = succ.numel()
        sp = _dev_ptr(succ, "succ", _succ_dtypes())
        wt = _wcode(weight)
        wp = None if weight is None else _dev_ptr(weight, "weight", (torch.int32, torch.int64))
        op = None if offsets is None else _dev_ptr(offsets, "offsets", (torch.int64,))
        if offsets is not None:
            k = offsets.numel() - 1
    else:
        sp = wp = op = None
        wt = {None: LR_NONE, "int32": LR_I32, "int64": LR_I64, torch.int32: LR_I32,
              torch.int64: LR_I64}[wtype]
    if rank_dtype is None:
        rank_dtype = torch.int32 if wt == LR_NONE else torch.int64
    o = _opts(wt, LR_I32 if rank_dtype == torch.int32 else LR_I64, validate, 0x5EED, max_lists)
    t = Tuning()
    _check(lib.lr_autotune(sp, wp, op, int(n_total), int(k), ctypes.byref(o), _stream_handle(stream),
                           ctypes.byref(t)), "lr_autotune")
    return t


def autotune_entries():
    """The autotuned table as a list of dicts."""
    lib = load()
    cnt = lib.lr_autotune_entries(None, 0)
    arr = (_TuneEntry * max(1, cnt))()
    cnt = lib.lr_autotune_entries(arr, cnt)
    out = []
    for e in arr[:cnt]:
        d = {"log2n": e.log2n, "weighted": e.weighted, "batch": e.batch, "ms": e.ms}
        d.update({f: getattr(e.tuning, f) for f, _ in Tuning._fields_ if f != "reserved"})
        out.append(d)
    return out


def autotune_save(path):
    _check(load().lr_autotune_save(os.fsencode(path)), "lr_autotune_save")


def autotune_load(path):
    _check(load().lr_autotune_load(os.fsencode(path)), "lr_autotune_load")


def autotune_clear():
    load().lr_autotune_clear()


class Pipeline:
    """Host-buffer pipeline (lr_pipeline_* of the C ABI): submissions of
    host-resident lists whose copies overlap the neighbouring rankings.

    Submitted arrays (and outputs) are kept referenced until wait(); pass
    pinned tensors for the copies to overlap."""

    def __init__(self, max_n, wtype=None, rank_dtype=None, depth=2, max_lists=0,
                 validate=False, seed=0x5EED, tuning=None):
        import numpy as np
        torch = _torch()
        self._wt = {None: LR_NONE, "int32": LR_I32, "int64": LR_I64, np.int32: LR_I32,
                    np.int64: LR_I64, torch.int32: LR_I32, torch.int64: LR_I64}[wtype]
        rdt = rank_dtype or (torch.int32 if self._wt == LR_NONE else torch.int64)
        self._rdt = {torch.int32: torch.int32, np.int32: torch.int32, "int32": torch.int32,
                     torch.int64: torch.int64, np.int64: torch.int64, "int64": torch.int64}[rdt]
        o = _opts(self._wt, LR_I32 if self._rdt == torch.int32 else LR_I64, validate, seed,
                  max_lists, tuning)
        h = ctypes.c_void_p()
        _check(load().lr_pipeline_create(int(max_n), ctypes.byref(o), int(depth), ctypes.byref(h)),
               "lr_pipeline_create")
        self._h = h
        self._keep = []

    def submit(self, succ, weight=None, out=None):
        """Enqueue one host list; returns the output (valid after wait())."""
        import numpy as np
        torch = _torch()

        def host(a):
            if isinstance(a, torch.Tensor):
                assert not a.is_cuda and a.is_contiguous()
                return a
            return torch.from_numpy(np.ascontiguousarray(a))

        succ = host(succ)
        weight = None if weight is None else host(weight)
        n = succ.numel()
        if out is None:
            out = torch.empty(n, dtype=self._rdt)
        out = host(out)
        _check(load().lr_pipeline_submit(self._h, ctypes.c_void_p(succ.data_ptr()),
                                         None if weight is None else ctypes.c_void_p(weight.data_ptr()),
                                         n, ctypes.c_void_p(out.data_ptr())), "lr_pipeline_submit")
        self._keep.append((succ, weight, out))
        return out

    def wait(self):
        """Wait for every submission; raises LRError naming the first failed one."""
        idx = ctypes.c_int64(-1)
        code = load().lr_pipeline_wait(self._h, ctypes.byref(idx))
        self._keep = []
        if code != 0:
            err = LRError(code, "lr_pipeline_wait (submission %d)" % idx.value)
            err.index = idx.value
            raise err

    def close(self):
        if self._h:
            load().lr_pipeline_destroy(self._h)
            self._h = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching ranking server (lr_server_* of the C ABI).

    Requests of at least alone_min_n elements (0: the library's default,
    2^23; negative: never) are ranked on their own through the single-list
    path; smaller ones that wait together are ranked as one forest.  With
    plain=True every request is ranked on its own (the baseline mode)."""

    def __init__(self, budget_bytes=40_000_000_000, n_streams=4, max_batch=256,
                 max_batch_elems=1 << 28, device=0, plain=False, alone_min_n=0):
        lib = load()
        c = _ServerConfig()
        lib.lr_server_config_default(ctypes.byref(c))
        c.budget_bytes, c.n_streams, c.max_batch = int(budget_bytes), int(n_streams), int(max_batch)
        c.max_batch_elems, c.device, c.plain = int(max_batch_elems), int(device), 1 if plain else 0
        c.alone_min_n = int(alone_min_n)
        h = ctypes.c_void_p()
        _check(lib.lr_server_create(ctypes.byref(c), ctypes.byref(h)), "lr_server_create")
        self._h = h
        self._keep = {}

    def submit(self, succ, weight=None, out=None, rank_dtype=None):
        """Submit a request (CUDA tensors are ranked in place; host tensors are
        copied by the server).  Returns a ticket."""
        import numpy as np
        torch = _torch()
        on_dev = isinstance(succ, torch.Tensor) and succ.is_cuda
        n = succ.numel() if isinstance(succ, torch.Tensor) else np.asarray(succ).size
        if out is None:
            rdt = rank_dtype or (torch.int32 if weight is None else torch.int64)
            out = torch.empty(n, dtype=rdt, device=succ.device if on_dev else "cpu",
                              pin_memory=False)
        r = _Request()
        r.succ = succ.data_ptr()
        r.weight = None if weight is None else weight.data_ptr()
        r.rank = out.data_ptr()
        r.n = n
        r.wtype = _wcode(weight)
        r.rtype = LR_I32 if out.dtype == torch.int32 else LR_I64
        r.on_device = 1 if on_dev else 0
        t = ctypes.c_uint64()
        _check(load().lr_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "lr_server_submit")
        self._keep[t.value] = (succ, weight, out)
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """Wait for a request; returns (rank tensor, result dict); raises on error."""
        res = _Result()
        code = load().lr_server_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(res))
        keep = self._keep.pop(ticket, (None, None, None)) if code != 7 else self._keep.get(ticket)
        info = {f: getattr(res, f) for f, _ in _Result._fields_}
        if code != 0:
            raise LRError(code, "request %d" % ticket)
        return keep[2], info

    def stats(self):
        s = _ServerStats()
        _check(load().lr_server_stats_get(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _ServerStats._fields_}

    def close(self):
        if self._h:
            load().lr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
