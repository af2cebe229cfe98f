"""Thin Python binding of the C ABI in include/jk.h (argument marshalling only).

Every step of the JK build runs in the CUDA library ``_build/libjk.so``;
this module converts numpy basis arrays and torch CUDA tensors to the plain
pointers and sizes the C functions take, and turns error codes into
exceptions. There is no CPU fallback: if the library is missing, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libjk.so")

JK_OK, JK_ERR_ARG, JK_ERR_UNSUPPORTED, JK_ERR_CUDA, JK_ERR_OOM, JK_ERR_TIMEOUT, JK_ERR_NAN, JK_ERR_COMPILE = range(8)
JK_PREC_FP64, JK_PREC_MIXED, JK_PREC_MIXED_ROUTED, JK_PREC_FP32 = range(4)
PRECISION = {"fp64": JK_PREC_FP64, "mixed": JK_PREC_MIXED, "routed": JK_PREC_MIXED_ROUTED,
             "fp32": JK_PREC_FP32}

# every function include/jk.h declares
EXPORTED = ["jk_init", "jk_init_batch", "jk_build", "jk_build_batch", "jk_set_option",
            "jk_get_option", "jk_info", "jk_schwarz", "jk_check", "jk_destroy", "jk_router_collect", "jk_router_train",
            "jk_router_forward", "jk_router_gradient", "jk_router_gradient_noalloc", "jk_router_load",
            "jk_profile", "jk_measure_peak",
            "jk_compile_class", "jk_compile_basis", "jk_autotune", "jk_fragment_candidates",
            "jk_last_error"]

ROUTER_NIN = 12
ROUTER_NPARAM = 5313
ROUTER_MAGIC = 0x4a4b5254


class JKError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"JK error {code}: {msg}")
        self.code = code


class JkShell(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("atom", "l", "nprim", "prim_off", "ao_off", "spherical")]


class JkStats(ctypes.Structure):
    _fields_ = [("quartets_fp64", ctypes.c_int64), ("quartets_fp32", ctypes.c_int64),
                ("quartets_routed", ctypes.c_int64), ("prim_quartets", ctypes.c_int64),
                ("flops_model", ctypes.c_double), ("ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class JkLaunchProf(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("la", "lb", "lc", "ld", "na", "nb", "nc", "nd", "tier",
                                             "threads_per_quartet", "regs", "local_bytes")] + \
               [("quartets", ctypes.c_int64), ("prim_quartets", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops_model", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class JkRouterBlob(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint32),
                ("mu", ctypes.c_float * 16), ("isd", ctypes.c_float * 16),
                ("theta", ctypes.c_float * ROUTER_NPARAM), ("margin", ctypes.c_float),
                ("quantile", ctypes.c_float)]

    def to_bytes(self) -> bytes:
        return ctypes.string_at(ctypes.addressof(self), ctypes.sizeof(self))

    @classmethod
    def from_bytes(cls, b: bytes):
        blob = cls()
        ctypes.memmove(ctypes.addressof(blob), b, ctypes.sizeof(cls))
        return blob


class JkTrainOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("quantile", ctypes.c_float), ("seed", ctypes.c_uint64)]


class JkTrainStats(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


class JkTuneReport(ctypes.Structure):
    _fields_ = [("launches_tuned", ctypes.c_int32), ("candidates_timed", ctypes.c_int32),
                ("changed", ctypes.c_int32), ("pad", ctypes.c_int32), ("ms_before", ctypes.c_double),
                ("ms_after", ctypes.c_double), ("tune_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


def load_library() -> ctypes.CDLL:
    """Load libjk.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build() or python -m paper_2507_09772_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    dp = P(ctypes.c_double)
    i32 = ctypes.c_int32
    lib.jk_init.argtypes = [P(JkShell), i32, dp, i32, dp, dp, i32, P(vp)]
    lib.jk_init_batch.argtypes = [i32, P(i32), P(JkShell), i32, dp, i32, dp, dp, i32, P(vp)]
    lib.jk_build.argtypes = [vp, vp, i32, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                             vp, vp, vp, P(JkStats)]
    lib.jk_build_batch.argtypes = [vp, P(vp), i32, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, P(vp), P(vp), vp, P(JkStats)]
    lib.jk_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_double]
    lib.jk_get_option.argtypes = [vp, ctypes.c_char_p, dp]
    lib.jk_info.argtypes = [vp, i32, P(i32), P(i32), P(i32)]
    lib.jk_schwarz.argtypes = [vp, dp]
    lib.jk_destroy.argtypes = [vp]
    lib.jk_check.argtypes = [vp, vp]
    lib.jk_compile_class.argtypes = [i32] * 14 + [P(i32), dp]
    lib.jk_profile.argtypes = [vp, P(JkLaunchProf), i32, P(i32)]
    lib.jk_compile_basis.argtypes = [P(JkShell), i32, i32, i32, i32, i32, i32, dp, P(i32)]
    lib.jk_router_collect.argtypes = [vp, P(vp), i32, ctypes.c_double, P(vp), P(vp), vp, vp, ctypes.c_int64,
                                      P(ctypes.c_int64), vp]
    lib.jk_router_train.argtypes = [vp, vp, ctypes.c_int64, P(JkTrainOpts), P(JkRouterBlob), P(JkTrainStats)]
    lib.jk_router_forward.argtypes = [P(JkRouterBlob), vp, ctypes.c_int64, vp]
    lib.jk_router_gradient.argtypes = [P(JkRouterBlob), vp, vp, ctypes.c_int64, ctypes.c_float,
                                       P(ctypes.c_float), P(ctypes.c_double)]
    lib.jk_router_load.argtypes = [vp, P(JkRouterBlob)]
    lib.jk_router_gradient_noalloc.argtypes = [P(JkRouterBlob), vp, vp, ctypes.c_int64, ctypes.c_float,
                                               P(ctypes.c_float), P(ctypes.c_double), vp]
    lib.jk_measure_peak.argtypes = [i32, ctypes.c_double, dp]
    lib.jk_autotune.argtypes = [vp, P(vp), i32, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                P(vp), P(vp), vp, i32, ctypes.c_double, P(JkTuneReport)]
    lib.jk_fragment_candidates.argtypes = [i32, i32, i32, i32, i32, i32, P(i32), P(i32)]
    lib.jk_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "jk_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def jk_last_error() -> str:
    return load_library().jk_last_error().decode(errors="replace")


def _check(rc: int):
    if rc != JK_OK:
        raise JKError(rc, jk_last_error())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _shell_array(shells) -> ctypes.Array:
    sh = np.ascontiguousarray(shells, dtype=np.int32).reshape(-1, 6)
    arr = (JkShell * len(sh))()
    ctypes.memmove(arr, sh.ctypes.data, sh.nbytes)
    return arr


def jk_init(shells, coords, exps, coeffs) -> ctypes.c_void_p:
    lib = load_library()
    sh = _shell_array(shells)
    c = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 3)
    e = np.ascontiguousarray(exps, dtype=np.float64)
    k = np.ascontiguousarray(coeffs, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib.jk_init(sh, len(sh), _dptr(c), c.shape[0], _dptr(e), _dptr(k), len(e), ctypes.byref(h)))
    return h


def jk_init_batch(mol_shell_off, shells, coords, exps, coeffs) -> ctypes.c_void_p:
    lib = load_library()
    off = np.ascontiguousarray(mol_shell_off, dtype=np.int32)
    sh = _shell_array(shells)
    c = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 3)
    e = np.ascontiguousarray(exps, dtype=np.float64)
    k = np.ascontiguousarray(coeffs, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib.jk_init_batch(len(off) - 1, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), sh, len(sh),
                             _dptr(c), c.shape[0], _dptr(e), _dptr(k), len(e), ctypes.byref(h)))
    return h


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return int(getattr(stream, "cuda_stream", stream))


def jk_build(h, D, n_dm, with_j, with_k, cutoff, precision_mode, J, K, stream=None, stats=False):
    """D, J, K: torch float64 CUDA tensors (n_dm, nao, nao). Returns a stats dict if asked."""
    lib = load_library()
    st = JkStats() if stats else None
    _check(lib.jk_build(h, _ptr(D), int(n_dm), int(bool(with_j)), int(bool(with_k)), float(cutoff),
                        int(precision_mode), _ptr(J), _ptr(K), _stream_ptr(stream),
                        ctypes.byref(st) if st is not None else None))
    return st.as_dict() if st is not None else None


def jk_build_batch(h, Ds: Sequence, n_dm, with_j, with_k, cutoff, precision_mode, Js, Ks, stream=None,
                   stats=False):
    lib = load_library()
    n = len(Ds)
    arr = ctypes.c_void_p * n
    d = arr(*[_ptr(x) for x in Ds])
    j = arr(*[_ptr(x) for x in Js]) if Js is not None else None
    k = arr(*[_ptr(x) for x in Ks]) if Ks is not None else None
    st = JkStats() if stats else None
    _check(lib.jk_build_batch(h, d, int(n_dm), int(bool(with_j)), int(bool(with_k)), float(cutoff),
                              int(precision_mode), j, k, _stream_ptr(stream),
                              ctypes.byref(st) if st is not None else None))
    return st.as_dict() if st is not None else None


def jk_set_option(h, key: str, value: float):
    _check(load_library().jk_set_option(h, key.encode(), float(value)))


def jk_get_option(h, key: str) -> float:
    v = ctypes.c_double()
    _check(load_library().jk_get_option(h, key.encode(), ctypes.byref(v)))
    return v.value


def jk_info(h, mol: int = 0):
    nao, nsh, nmol = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().jk_info(h, int(mol), ctypes.byref(nao), ctypes.byref(nsh), ctypes.byref(nmol)))
    return nao.value, nsh.value, nmol.value


def jk_schwarz(h) -> np.ndarray:
    _, nsh, _ = jk_info(h, 0)
    q = np.zeros((nsh, nsh))
    _check(load_library().jk_schwarz(h, _dptr(q)))
    return q


def jk_check(h, stream=None):
    """Synchronise the stream and raise if a build on the handle saw a
    non-finite density (the device error word)."""
    _check(load_library().jk_check(h, _stream_ptr(stream)))


def jk_destroy(h):
    _check(load_library().jk_destroy(h))


def jk_router_collect(h, Ds, n_dm, cutoff, Js, Ks, X, y, stream=None) -> int:
    """FP64 build that also writes band-quartet features X (cap x 12) and
    labels y (cap) (torch float32 CUDA tensors); returns the number seen."""
    n = len(Ds)
    arr = ctypes.c_void_p * n
    cnt = ctypes.c_int64()
    _check(load_library().jk_router_collect(h, arr(*[_ptr(d) for d in Ds]), int(n_dm), float(cutoff),
                                            arr(*[_ptr(j) for j in Js]), arr(*[_ptr(k) for k in Ks]),
                                            _ptr(X), _ptr(y), int(y.shape[0]), ctypes.byref(cnt),
                                            _stream_ptr(stream)))
    return cnt.value


def jk_router_train(X, y, steps=2000, batch=4096, lr=2e-3, quantile=0.9, seed=1):
    """Train on the device (X: n x 12, y: n, torch float32 CUDA). Returns (blob, stats)."""
    opts = JkTrainOpts(int(steps), int(batch), float(lr), float(quantile), int(seed))
    blob = JkRouterBlob()
    st = JkTrainStats()
    _check(load_library().jk_router_train(_ptr(X), _ptr(y), int(y.shape[0]), ctypes.byref(opts),
                                          ctypes.byref(blob), ctypes.byref(st)))
    return blob, st.as_dict()


def jk_router_forward(blob, X, y_out):
    _check(load_library().jk_router_forward(ctypes.byref(blob), _ptr(X), int(X.shape[0]), _ptr(y_out)))


def jk_router_gradient(blob, X, y, quantile):
    g = (ctypes.c_float * ROUTER_NPARAM)()
    loss = ctypes.c_double()
    _check(load_library().jk_router_gradient(ctypes.byref(blob), _ptr(X), _ptr(y), int(y.shape[0]),
                                             float(quantile), g, ctypes.byref(loss)))
    return np.frombuffer(g, dtype=np.float32).copy(), loss.value


def jk_router_gradient_noalloc(blob, X, y, quantile, stream=None):
    """Same result as jk_router_gradient from the variant that allocates no
    device memory (fixed library scratch; see include/jk.h)."""
    g = (ctypes.c_float * ROUTER_NPARAM)()
    loss = ctypes.c_double()
    _check(load_library().jk_router_gradient_noalloc(ctypes.byref(blob), _ptr(X), _ptr(y), int(y.shape[0]),
                                                     float(quantile), g, ctypes.byref(loss),
                                                     _stream_ptr(stream)))
    return np.frombuffer(g, dtype=np.float32).copy(), loss.value


def jk_router_load(h, blob):
    _check(load_library().jk_router_load(h, ctypes.byref(blob)))


def jk_profile(h):
    """Per-launch records of the last profiled build (option "profile" = 1)."""
    n = ctypes.c_int32()
    _check(load_library().jk_profile(h, None, 0, ctypes.byref(n)))
    arr = (JkLaunchProf * max(1, n.value))()
    _check(load_library().jk_profile(h, arr, n.value, ctypes.byref(n)))
    return [arr[i].as_dict() for i in range(n.value)]


def jk_measure_peak(which: str = "fp64", ms: float = 200.0) -> float:
    """FMA-chain FLOP/s of the current device (which = "fp64" or "fp32")."""
    v = ctypes.c_double()
    _check(load_library().jk_measure_peak(0 if which == "fp64" else 1, float(ms), ctypes.byref(v)))
    return v.value


def jk_compile_basis(shells, n_dm=1, with_j=1, with_k=1, fp32=0, mode=0):
    """Compile every kernel a basis of these shell types needs (no GPU needed)."""
    sh = _shell_array(shells)
    ms = ctypes.c_double()
    nk = ctypes.c_int32()
    _check(load_library().jk_compile_basis(sh, len(sh), n_dm, with_j, with_k, fp32, mode, ctypes.byref(ms),
                                           ctypes.byref(nk)))
    return nk.value, ms.value


def jk_compile_class(la, lb, lc, ld, na, nb, nc, nd, n_dm=1, with_j=1, with_k=1, fp32=0, mode=0, op=0):
    g = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(load_library().jk_compile_class(la, lb, lc, ld, na, nb, nc, nd, n_dm, with_j, with_k, fp32, mode, op,
                                           ctypes.byref(g), ctypes.byref(ms)))
    return g.value, ms.value


# ------------------------------------------------------------ convenience
def jk_autotune(h, Ds: Sequence, n_dm, with_j, with_k, cutoff, precision_mode, Js, Ks, stream=None,
                max_candidates=4, min_share=0.005) -> dict:
    """Fragment-shape autotuning on the given densities (J/K are scratch)."""
    lib = load_library()
    n = len(Ds)
    arr = ctypes.c_void_p * n
    d = arr(*[_ptr(x) for x in Ds])
    j = arr(*[_ptr(x) for x in Js]) if Js is not None else None
    k = arr(*[_ptr(x) for x in Ks]) if Ks is not None else None
    rep = JkTuneReport()
    _check(lib.jk_autotune(h, d, int(n_dm), int(bool(with_j)), int(bool(with_k)), float(cutoff),
                           int(precision_mode), j, k, _stream_ptr(stream), int(max_candidates),
                           float(min_share), ctypes.byref(rep)))
    return rep.as_dict()


def jk_fragment_candidates(la, lb, lc, ld, fp32=0, max_candidates=8):
    """Candidate fragment shapes [(ga, gb, gc, gd), ...] for a class (no GPU needed)."""
    lib = load_library()
    buf = (ctypes.c_int32 * (4 * max_candidates))()
    n = ctypes.c_int32()
    _check(lib.jk_fragment_candidates(la, lb, lc, ld, fp32, max_candidates, buf, ctypes.byref(n)))
    return [tuple(buf[4 * i:4 * i + 4]) for i in range(n.value)]


class JK:
    """Owns a handle for one molecule or a batch of molecules.

    ``molecules``: objects with ``shells``, ``coords``, ``exps``, ``coeffs``
    and ``nao`` (e.g. ``synth.Molecule``). Batches concatenate the arrays
    with global atom and primitive offsets and molecule-local AO offsets.
    """

    def __init__(self, molecules):
        if not isinstance(molecules, (list, tuple)):
            molecules = [molecules]
        self.nmol = len(molecules)
        self.nao = [int(m.nao) for m in molecules]
        shells, coords, exps, coeffs, off = [], [], [], [], [0]
        natm = nprim = 0
        for m in molecules:
            sh = np.array(m.shells, dtype=np.int32).copy()
            sh[:, 0] += natm
            sh[:, 3] += nprim
            shells.append(sh)
            coords.append(np.asarray(m.coords, dtype=np.float64))
            exps.append(np.asarray(m.exps, dtype=np.float64))
            coeffs.append(np.asarray(m.coeffs, dtype=np.float64))
            natm += len(m.coords)
            nprim += len(m.exps)
            off.append(off[-1] + len(sh))
        if self.nmol == 1:
            self.h = jk_init(shells[0], coords[0], exps[0], coeffs[0])
        else:
            self.h = jk_init_batch(np.array(off, dtype=np.int32), np.concatenate(shells),
                                   np.concatenate(coords), np.concatenate(exps), np.concatenate(coeffs))

    def set_option(self, key, value):
        jk_set_option(self.h, key, value)

    def get_option(self, key):
        return jk_get_option(self.h, key)

    def load_router(self, blob):
        jk_router_load(self.h, blob)

    def build(self, D, with_j=True, with_k=True, cutoff=1e-13, precision="fp64", J=None, K=None,
              stream=None, stats=False, check=True):
        """D: torch float64 CUDA tensor (n_dm, nao, nao), or a list for batches.
        Returns (J, K, stats-or-None); J/K allocated with torch if not given.
        With check (the default) a build without stats synchronises the
        stream and raises on a non-finite density (jk_check); check=False
        leaves the build asynchronous (the next call on the handle reports)."""
        import torch
        mode = PRECISION[precision] if isinstance(precision, str) else int(precision)
        Dl = list(D) if isinstance(D, (list, tuple)) else [D]
        Dl = [d if d.dim() == 3 else d.unsqueeze(0) for d in Dl]
        ndm = Dl[0].shape[0]
        if J is None and with_j:
            J = [torch.empty_like(d) for d in Dl]
        if K is None and with_k:
            K = [torch.empty_like(d) for d in Dl]
        if self.nmol == 1:
            listed = isinstance(D, (list, tuple))
            Jl = J if isinstance(J, list) else [J]
            Kl = K if isinstance(K, list) else [K]
            st = jk_build(self.h, Dl[0], ndm, with_j, with_k, cutoff, mode,
                          Jl[0] if with_j else None, Kl[0] if with_k else None, stream, stats)
            if check and not stats:
                jk_check(self.h, stream)
            if listed:
                return (Jl if with_j else None), (Kl if with_k else None), st
            return (Jl[0] if with_j else None), (Kl[0] if with_k else None), st
        st = jk_build_batch(self.h, Dl, ndm, with_j, with_k, cutoff, mode,
                            J if with_j else None, K if with_k else None, stream, stats)
        if check and not stats:
            jk_check(self.h, stream)
        return J, K, st

    def autotune(self, D, with_j=True, with_k=True, cutoff=1e-13, precision="fp64", max_candidates=4,
                 min_share=0.005, stream=None):
        """Autotune the fragment shapes on these densities (jk_autotune)."""
        import torch
        mode = PRECISION[precision] if isinstance(precision, str) else int(precision)
        Dl = list(D) if isinstance(D, (list, tuple)) else [D]
        Dl = [d if d.dim() == 3 else d.unsqueeze(0) for d in Dl]
        Js = [torch.empty_like(d) for d in Dl] if with_j else None
        Ks = [torch.empty_like(d) for d in Dl] if with_k else None
        return jk_autotune(self.h, Dl, Dl[0].shape[0], with_j, with_k, cutoff, mode, Js, Ks, stream,
                           max_candidates, min_share)

    def close(self):
        if getattr(self, "h", None) is not None:
            jk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
