"""ctypes binding of libmcmp2 (C ABI in include/mcmp2.h).

Argument marshalling only: every step of the Monte Carlo path runs in the
library's CUDA kernels.  PyTorch supplies the device workspace and the
stream.  There is no fallback: if the library is not built, or the device is
not an sm_103 GPU, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmcmp2.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mcmp2.h")

MCMP2_OK = 0
MCMP2_FP64 = 0
MCMP2_MIXED = 1
MCMP2_TF32 = 2
MCMP2_COULOMB = 0
MCMP2_GAUNT = 1
MCMP2_BREIT = 2
MCMP2_EUNSUPPORTED = -7
STATUS = {-1: "EINVAL", -2: "ENOTLOADED", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT", -6: "ENOSPACE",
          -7: "EUNSUPPORTED"}


class McMp2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Dims(ctypes.Structure):
    _fields_ = [("n_centres", ctypes.c_int), ("n_functions", ctypes.c_int), ("n_occ", ctypes.c_int),
                ("n_vir", ctypes.c_int), ("m", ctypes.c_int), ("n_tau", ctypes.c_int)]


class Basis(ctypes.Structure):
    _fields_ = [("n_centres", ctypes.c_int), ("centres", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("n_shells", ctypes.c_int), ("shell_centre", ctypes.c_void_p), ("shell_l", ctypes.c_void_p),
                ("shell_alpha", ctypes.c_void_p), ("shell_coef", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("variance", ctypes.c_double), ("error", ctypes.c_double),
                ("n_blocks", ctypes.c_int64), ("steps", ctypes.c_int64), ("mean_all", ctypes.c_double),
                ("last_step", ctypes.c_double), ("accept_rate", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProfileCounters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("pair_launches", ctypes.c_int64), ("pair_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64

SIGNATURES = {
    "mcmp2_create": (_I, [ctypes.POINTER(_P), _I, _P, _I]),
    "mcmp2_destroy": (None, [_P]),
    "mcmp2_last_error": (ctypes.c_char_p, [_P]),
    "mcmp2_workspace_bytes": (_I, [ctypes.POINTER(Dims), _I, ctypes.POINTER(_SZ)]),
    "mcmp2_bind_workspace": (_I, [_P, ctypes.POINTER(Dims), _P, _SZ]),
    "mcmp2_load_system": (_I, [_P, ctypes.POINTER(Basis), _I, _I, _P, _P]),
    "mcmp2_load_system_2c": (_I, [_P, ctypes.POINTER(Basis), _I, _I, _P, _P]),
    "mcmp2_set_walkers": (_I, [_P, _P, _U64, _I64]),
    "mcmp2_run_steps": (_I, [_P, _I64, _U64, ctypes.POINTER(Result)]),
    "mcmp2_eval_fixed": (_I, [_P, _I64, _P, _P, _P]),
    "mcmp2_get_walkers": (_I, [_P, _P, _P]),
    "mcmp2_backward": (_I, [_P, _I64, _P, _P, _P, _P, _P]),
    "mcmp2_debug_partials": (_I, [_P, _P, _SZ, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mcmp2_debug_elements": (_I, [_P, _P, _P, _I, _I, _P, _SZ, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(_I)]),
    "mcmp2_profile": (_I, [_P, _I, ctypes.POINTER(ProfileCounters)]),
    "mcmp2_test_stall_next": (_I, [_P, ctypes.c_double]),
    "mcmp2_set_interaction": (_I, [_P, _I]),
    "mcmp2_checkpoint_bytes": (_I, [_P, ctypes.POINTER(_SZ)]),
    "mcmp2_pair_sum_f64_noalloc": (_I, [_I, _I, _I, _I, _P, _P, _P, ctypes.c_double, _P, _P]),
    "mcmp2_checkpoint": (_I, [_P, _P, _SZ]),
    "mcmp2_restore": (_I, [_P, _P, _SZ]),
}

_lib = None


def header_symbols():
    """Entry points declared in include/mcmp2.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(mcmp2_[a-z0-9_]+)\s*\(", text)))


def load_library(path: str = LIB_PATH):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmcmp2 is not built ({path} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def workspace_bytes(dims: Dims, precision: int) -> int:
    n = _SZ(0)
    rc = load_library().mcmp2_workspace_bytes(ctypes.byref(dims), precision, ctypes.byref(n))
    if rc != MCMP2_OK:
        raise McMp2Error(rc, "invalid dims")
    return n.value


class Context:
    """One library context bound to a system, a torch-allocated workspace and a stream.

    system: any object with the fields of ``synthetic.System`` (centres, weight,
    shell_centre, shell_l, shell_alpha, shell_coef, n_occ, n_vir, C, eps).
    """

    def __init__(self, system, m: int, n_tau: int, precision: int = MCMP2_FP64, device: int = 0,
                 stream=None):
        import torch

        self.lib = load_library()
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.precision = precision
        self.system = system
        h = _P()
        rc = self.lib.mcmp2_create(ctypes.byref(h), device, _P(self.stream.cuda_stream), precision)
        if rc != MCMP2_OK:
            raise McMp2Error(rc, "mcmp2_create failed (needs an sm_103 GPU)")
        self.h = h
        n_l = int(sum({0: 1, 1: 3, 2: 6}[int(l)] for l in system.shell_l))
        self.dims = Dims(len(system.centres), n_l, int(system.n_occ), int(system.n_vir), int(m), int(n_tau))
        self.m, self.n_tau, self.n_l = int(m), int(n_tau), n_l
        nbytes = workspace_bytes(self.dims, precision)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self._check(self.lib.mcmp2_bind_workspace(self.h, ctypes.byref(self.dims), _P(self._ws_ptr), nbytes))
        self._keep = [
            _c(system.centres, np.float64), _c(system.weight, np.float64), _c(system.shell_centre, np.int32),
            _c(system.shell_l, np.int32), _c(system.shell_alpha, np.float64), _c(system.shell_coef, np.float64),
        ]
        k = self._keep
        self._basis = Basis(len(k[0]), _ptr(k[0]).value, _ptr(k[1]).value, len(k[3]), _ptr(k[2]).value,
                            _ptr(k[3]).value, _ptr(k[4]).value, _ptr(k[5]).value)
        self._load(system)

    # -- helpers ---------------------------------------------------------
    def _load(self, sysobj):
        """mcmp2_load_system, or mcmp2_load_system_2c (alpha and beta rows of C) for a
        two-component system (``n_comp == 2``, small-component rows of C zero)."""
        eps = _c(sysobj.eps, np.float64)
        if getattr(sysobj, "n_comp", 4) == 2:
            C = _c(sysobj.C[:2 * self.n_l], np.complex128)
            rc = self.lib.mcmp2_load_system_2c(self.h, ctypes.byref(self._basis), int(sysobj.n_occ),
                                               int(sysobj.n_vir), _ptr(C), _ptr(eps))
        else:
            C = _c(sysobj.C, np.complex128)
            rc = self.lib.mcmp2_load_system(self.h, ctypes.byref(self._basis), int(sysobj.n_occ),
                                            int(sysobj.n_vir), _ptr(C), _ptr(eps))
        self._check(rc)

    def _check(self, rc):
        if rc != MCMP2_OK:
            msg = self.lib.mcmp2_last_error(self.h).decode()
            raise McMp2Error(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mcmp2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API -------------------------------------------------------------
    def set_walkers(self, r, seed: int, burn_in: int):
        """Initial positions [m][2][3], or None to draw them from g(r1) g(r2) on the device."""
        if r is None:
            self._check(self.lib.mcmp2_set_walkers(self.h, None, int(seed), int(burn_in)))
            return
        r = _c(r, np.float64).reshape(self.m, 2, 3)
        self._check(self.lib.mcmp2_set_walkers(self.h, _ptr(r), int(seed), int(burn_in)))

    def run_steps(self, n: int, seed: int) -> dict:
        res = Result()
        self._check(self.lib.mcmp2_run_steps(self.h, int(n), int(seed), ctypes.byref(res)))
        return res.as_dict()

    def run_steps_async(self, n: int, seed: int):
        """Issue n steps without reading the statistics back (no host synchronisation)."""
        self._check(self.lib.mcmp2_run_steps(self.h, int(n), int(seed), None))

    def eval_fixed(self, r, tau, out=None) -> np.ndarray:
        r = _c(r, np.float64)
        tau = _c(tau, np.float64)
        n = r.shape[0]
        assert r.shape == (n, self.m, 2, 3) and tau.shape == (n, self.n_tau)
        if out is None:
            out = np.zeros(n)
        self._check(self.lib.mcmp2_eval_fixed(self.h, n, _P(r.ctypes.data), _P(tau.ctypes.data),
                                              _P(out.ctypes.data)))
        return out

    def eval_fixed_ptr(self, n: int, r_ptr: int, tau_ptr: int, out_ptr: int):
        """Replay from raw host pointers (e.g. pinned torch tensors)."""
        self._check(self.lib.mcmp2_eval_fixed(self.h, int(n), _P(r_ptr), _P(tau_ptr), _P(out_ptr)))

    def load(self, eps=None, C=None):
        """Reload the system with new orbital energies and/or coefficients (same basis)."""
        import dataclasses
        sysobj = self.system
        if eps is not None or C is not None:
            sysobj = dataclasses.replace(sysobj, eps=self.system.eps if eps is None else np.asarray(eps),
                                         C=self.system.C if C is None else np.asarray(C))
        self._load(sysobj)
        self.system = sysobj

    def backward(self, r, tau):
        """(E, dE/d eps, dE/dC) of the replay estimate for the given samples (FP64 contexts)."""
        r = _c(r, np.float64)
        tau = _c(tau, np.float64)
        n = r.shape[0]
        e = ctypes.c_double(0.0)
        d_eps = np.zeros(self.system.n_occ + self.system.n_vir)
        d_C = np.zeros((4 * self.n_l, self.system.n_occ + self.system.n_vir), dtype=np.complex128)
        self._check(self.lib.mcmp2_backward(self.h, n, _P(r.ctypes.data), _P(tau.ctypes.data), ctypes.byref(e),
                                            _ptr(d_eps), _ptr(d_C)))
        return e.value, d_eps, d_C

    def get_walkers(self):
        r = np.zeros((self.m, 2, 3))
        d = ctypes.c_double(0.0)
        self._check(self.lib.mcmp2_get_walkers(self.h, _ptr(r), ctypes.byref(d)))
        return r, d.value

    def debug_partials(self):
        nt, tp = _I(0), _I(0)
        self._check(self.lib.mcmp2_debug_partials(self.h, None, 0, ctypes.byref(nt), ctypes.byref(tp)))
        out = np.zeros((self.n_tau, nt.value))
        self._check(self.lib.mcmp2_debug_partials(self.h, _ptr(out), out.size, ctypes.byref(nt),
                                                  ctypes.byref(tp)))
        return out, tp.value

    def tile_pairs(self) -> int:
        """Walker pairs per side of the contraction's tiles (8 FP64, 16 tensor-core, 32 two-component there)."""
        nt, tp = _I(0), _I(0)
        self._check(self.lib.mcmp2_debug_partials(self.h, None, 0, ctypes.byref(nt), ctypes.byref(tp)))
        return tp.value

    def debug_elements(self, r_step, tau_step, bp: int, bq: int):
        """Every summand Re f/(w w w) of the tile (bp, bq) for one replay step:
        returns (elements [n_tau][T][T], I'_n of the step, T)."""
        r = _c(r_step, np.float64)
        tau = _c(tau_step, np.float64)
        assert r.shape == (self.m, 2, 3) and tau.shape == (self.n_tau,)
        tp = self.tile_pairs()
        out = np.zeros((self.n_tau, tp, tp))
        step = ctypes.c_double(0.0)
        got = _I(0)
        self._check(self.lib.mcmp2_debug_elements(self.h, _ptr(r), _ptr(tau), int(bp), int(bq), _ptr(out), out.size,
                                                  ctypes.byref(step), ctypes.byref(got)))
        assert got.value == tp
        return out, step.value, tp

    def profile(self, mode: int = 0):
        """mode 1: reset and time the contraction kernel; 2: reset, no timing; 0: read."""
        pc = ProfileCounters()
        self._check(self.lib.mcmp2_profile(self.h, int(mode), ctypes.byref(pc) if mode == 0 else None))
        return {k: getattr(pc, k) for k, _ in pc._fields_} if mode == 0 else None

    def set_interaction(self, interaction: int):
        """MCMP2_COULOMB (default), MCMP2_GAUNT or MCMP2_BREIT for the following steps (four-component systems)."""
        self._check(self.lib.mcmp2_set_interaction(self.h, int(interaction)))

    def test_stall_next(self, wait_limit_s: float):
        """Test hook: the next contraction launch withholds its first copy (bounded wait runs out)."""
        self._check(self.lib.mcmp2_test_stall_next(self.h, float(wait_limit_s)))

    def checkpoint(self) -> bytes:
        n = _SZ(0)
        self._check(self.lib.mcmp2_checkpoint_bytes(self.h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self.lib.mcmp2_checkpoint(self.h, buf, n.value))
        return buf.raw

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self.lib.mcmp2_restore(self.h, buf, len(blob)))


def tile_pairs_of(precision: int) -> int:
    return 8 if precision == MCMP2_FP64 else 16


def pair_sum_f64_noalloc(m, n_occ, n_vir, n_tau, phi, scale, a, lam, out, stream=None):
    """Allocation-free step estimate (mcmp2_pair_sum_f64_noalloc) on device tensors.

    For callers that cannot allocate device memory: the library's own fixed
    scratch array holds the intermediate sums.  phi, scale, a and out are
    CUDA tensors the caller already owns (layouts as in include/mcmp2.h)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = load_library().mcmp2_pair_sum_f64_noalloc(int(m), int(n_occ), int(n_vir), int(n_tau),
                                                   _P(phi.data_ptr()), _P(scale.data_ptr()), _P(a.data_ptr()),
                                                   float(lam), _P(out.data_ptr()), _P(st.cuda_stream))
    if rc != MCMP2_OK:
        raise McMp2Error(rc, "mcmp2_pair_sum_f64_noalloc failed")
