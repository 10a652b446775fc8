"""Sequential CPU oracle for list ranking -- TEST INFRASTRUCTURE ONLY.

The oracle is the plain definition of the list ranking problem (Section 1.1 of
"Engineering Scalable Distributed List Ranking") written out as a one-thread C
program (``lr_oracle.c``).  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the GPU library never does, and the
two share no code.

Status codes returned by the oracle (its own numbering; the tests map them):
``OK=0, INVALID=1, OUT_OF_RANGE=2, CYCLE=3, NOT_A_LIST=4, NO_MEMORY=5``.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liblr_oracle.so")

OK, INVALID, OUT_OF_RANGE, CYCLE, NOT_A_LIST, NO_MEMORY = range(6)
STATUS_NAMES = {OK: "OK", INVALID: "INVALID", OUT_OF_RANGE: "OUT_OF_RANGE",
                CYCLE: "CYCLE", NOT_A_LIST: "NOT_A_LIST", NO_MEMORY: "NO_MEMORY"}

_W_CODES = {None: 0, np.dtype(np.int32): 1, np.dtype(np.int64): 2}
_R_CODES = {np.dtype(np.int32): 1, np.dtype(np.int64): 2}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler (plain -O2, no tuning)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.lro_rank.restype = ctypes.c_int
            lib.lro_rank.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
            lib.lro_rank_batch.restype = ctypes.c_int
            lib.lro_rank_batch.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_int]
            lib.lro_rank_ext.restype = ctypes.c_int
            lib.lro_rank_ext.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.lro_rank_ext_batch.restype = ctypes.c_int
            lib.lro_rank_ext_batch.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check_inputs(succ, weight, rank_dtype):
    succ = np.ascontiguousarray(succ)
    if succ.dtype != np.uint32:
        succ = succ.astype(np.uint32)
    if weight is not None:
        weight = np.ascontiguousarray(weight)
        if weight.dtype not in (np.int32, np.int64):
            raise TypeError("weights must be int32 or int64")
        if weight.shape != succ.shape:
            raise ValueError("weight and succ differ in length")
    rdt = np.dtype(rank_dtype)
    if rdt not in _R_CODES:
        raise TypeError("rank dtype must be int32 or int64")
    return succ, weight, rdt


def rank_status(succ, weight=None, rank_dtype=np.int32):
    """Rank one successor array; returns (status, rank array)."""
    succ, weight, rdt = _check_inputs(succ, weight, rank_dtype)
    n = succ.shape[0]
    out = np.zeros(n, dtype=rdt)
    wcode = _W_CODES[None if weight is None else weight.dtype]
    st = _load().lro_rank(_ptr(succ), _ptr(weight), wcode, n, _ptr(out), _R_CODES[rdt])
    return st, out


def rank(succ, weight=None, rank_dtype=np.int32):
    """Rank one successor array; raises ValueError on invalid input."""
    st, out = rank_status(succ, weight, rank_dtype)
    if st != OK:
        raise ValueError("oracle: " + STATUS_NAMES.get(st, str(st)))
    return out


def rank_batch_status(offsets, succ, weight=None, rank_dtype=np.int64):
    """Rank k instances stored back to back (local successor ids)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    succ, weight, rdt = _check_inputs(succ, weight, rank_dtype)
    k = offsets.shape[0] - 1
    out = np.zeros(succ.shape[0], dtype=rdt)
    wcode = _W_CODES[None if weight is None else weight.dtype]
    st = _load().lro_rank_batch(_ptr(offsets), k, _ptr(succ), _ptr(weight), wcode,
                                _ptr(out), _R_CODES[rdt])
    return st, out


def rank_batch(offsets, succ, weight=None, rank_dtype=np.int64):
    st, out = rank_batch_status(offsets, succ, weight, rank_dtype)
    if st != OK:
        raise ValueError("oracle: " + STATUS_NAMES.get(st, str(st)))
    return out


def rank_ext(succ, weight=None, rank_dtype=np.int32, inclusive=False):
    """Rank plus the other outputs Section 1.1 defines: returns
    (rank, term, prefix) -- the terminal of every element's list and the
    head-relative rank; inclusive=True adds the terminal's own weight to rank
    (the paper's in-place form).  Raises ValueError on invalid input."""
    succ, weight, rdt = _check_inputs(succ, weight, rank_dtype)
    n = succ.shape[0]
    out = np.zeros(n, dtype=rdt)
    term = np.zeros(n, dtype=np.uint32)
    prefix = np.zeros(n, dtype=rdt)
    wcode = _W_CODES[None if weight is None else weight.dtype]
    st = _load().lro_rank_ext(_ptr(succ), _ptr(weight), wcode, n, _ptr(out), _R_CODES[rdt],
                              _ptr(term), _ptr(prefix), 1 if inclusive else 0)
    if st != OK:
        raise ValueError("oracle: " + STATUS_NAMES.get(st, str(st)))
    return out, term, prefix


def rank_ext_batch(offsets, succ, weight=None, rank_dtype=np.int64, inclusive=False):
    """Batched rank_ext; terminal ids are local to their instance."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    succ, weight, rdt = _check_inputs(succ, weight, rank_dtype)
    k = offsets.shape[0] - 1
    n = succ.shape[0]
    out = np.zeros(n, dtype=rdt)
    term = np.zeros(n, dtype=np.uint32)
    prefix = np.zeros(n, dtype=rdt)
    wcode = _W_CODES[None if weight is None else weight.dtype]
    st = _load().lro_rank_ext_batch(_ptr(offsets), k, _ptr(succ), _ptr(weight), wcode, _ptr(out),
                                    _R_CODES[rdt], _ptr(term), _ptr(prefix), 1 if inclusive else 0)
    if st != OK:
        raise ValueError("oracle: " + STATUS_NAMES.get(st, str(st)))
    return out, term, prefix
