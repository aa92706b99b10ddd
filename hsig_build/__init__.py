"""Host HSIG builder (input producer) and a numpy reader of the index file.

The builder is C++ (hsig_build.cpp, compiled in place by ``compile()``); it
turns seeded vectors and attributes into the serialised HSIG that both the CPU
oracle and the CUDA search read as input data. It shares no code with either.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsig_build.cpp")
_LIB = os.path.join(_HERE, "libhsig_build.so")
_lock = threading.Lock()
_lib = None

DTYPES = {1: np.int8, 2: np.uint8, 3: np.int32, 4: np.uint32, 5: np.int64, 6: np.float32}
META_FIELDS = ["n", "d", "S", "M", "max_level", "entry_global", "n_upper", "efc", "seed", "W"]


def source_digest() -> str:
    """Short digest of the builder source (names cached index files)."""
    import hashlib
    with open(_SRC, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:10]


def cached_index_path(cache_dir: str, name: str, n: int, seed: int) -> str:
    """File name under cache_dir for the index of a seeded workload (shared by the
    benchmark and the full-size tests so one build serves both)."""
    return os.path.join(cache_dir, f"{name}_n{n}_s{seed}_{source_digest()}.idx")


def compile(force: bool = False) -> str:
    """Compile the builder into hsig_build/libhsig_build.so (skipped when current)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["g++", "-O3", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", _LIB + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            compile()
            lib = ctypes.CDLL(_LIB)
            lib.hsig_build_index.restype = ctypes.c_int
            lib.hsig_build_index.argtypes = [
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_char_p,
                ctypes.c_char_p, ctypes.c_int]
            lib.hsig_build_index_ex.restype = ctypes.c_int
            lib.hsig_build_index_ex.argtypes = lib.hsig_build_index.argtypes + [ctypes.c_void_p] * 4
            _lib = lib
    return _lib


def build_index(vectors: np.ndarray, attrs: np.ndarray, path: str, S: int, M: int, efc: int,
                seed: int = 0, threads: int = 0, assist=None) -> str:
    """Build the HSIG for (vectors, attrs) and write it to ``path``.

    ``assist``: optional (propose, apply, fetch, context) addresses of C callbacks
    with the signatures of ``unify_propose_fn``, ``unify_apply_fn`` and
    ``unify_fetch_fn`` (apply and fetch may both be None). propose takes over the
    searches of every batch of at least 64 nodes; apply and fetch take over edge
    application from the first proposal on."""
    x = np.ascontiguousarray(vectors, dtype=np.float32)
    a = np.ascontiguousarray(attrs, dtype=np.int64)
    if x.ndim != 2 or a.shape != (x.shape[0],):
        raise ValueError("vectors must be (n, d) and attrs (n,)")
    lib = _load()
    err = ctypes.create_string_buffer(512)
    tmp = path + ".tmp"
    if assist is None:
        rc = lib.hsig_build_index(x.ctypes.data, a.ctypes.data, x.shape[0], x.shape[1], S, M, efc,
                                  seed, threads, tmp.encode(), err, 512)
    else:
        rc = lib.hsig_build_index_ex(x.ctypes.data, a.ctypes.data, x.shape[0], x.shape[1], S, M, efc,
                                     seed, threads, tmp.encode(), err, 512, *assist)
    if rc != 0:
        raise RuntimeError(f"hsig_build_index failed ({rc}): {err.value.decode()}")
    os.replace(tmp, path)
    return path


def _fnv1a_words(buf: np.ndarray) -> int:
    b = buf.view(np.uint8).reshape(-1)
    pad = (-len(b)) % 8
    if pad:
        b = np.concatenate([b, np.zeros(pad, np.uint8)])
    w = b.view("<u8")
    h = 0xCBF29CE484222325
    p = 0x100000001B3
    mask = (1 << 64) - 1
    for x in w.tolist():
        h = ((h ^ x) * p) & mask
    return h


def read_index(path: str, verify: bool = False) -> dict:
    """Map the index file into a dict of numpy arrays (plus 'meta' scalars)."""
    raw = np.memmap(path, dtype=np.uint8, mode="r")
    if bytes(raw[:8]) != b"UNIFYHSG":
        raise ValueError("bad magic")
    version, nsec = np.frombuffer(raw[8:16], dtype="<u4")
    if version != 1:
        raise ValueError(f"unsupported version {version}")
    out = {}
    for s in range(int(nsec)):
        e = raw[16 + 96 * s: 16 + 96 * (s + 1)]
        name = bytes(e[:24]).split(b"\0")[0].decode()
        dtype, ndim = np.frombuffer(e[24:32], dtype="<u4")
        shape = tuple(int(v) for v in np.frombuffer(e[32:64], dtype="<u8")[:ndim])
        off, nbytes, ck = (int(v) for v in np.frombuffer(e[64:88], dtype="<u8"))
        arr = np.frombuffer(raw, dtype=DTYPES[int(dtype)], count=nbytes // np.dtype(DTYPES[int(dtype)]).itemsize,
                            offset=off).reshape(shape)
        if verify and _fnv1a_words(np.ascontiguousarray(arr)) != ck:
            raise ValueError(f"checksum mismatch in section {name}")
        out[name] = arr
    meta = out["meta"]
    for i, f in enumerate(META_FIELDS):
        out[f] = int(meta[i])
    return out
