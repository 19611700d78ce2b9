"""The oracle -- TEST INFRASTRUCTURE ONLY, not the product.

A plain FP64 CPU restatement of the Monte Carlo four-component relativistic
MP2 method (arXiv 2203.05632, Sec. III) and of the deterministic MP2 energy
it estimates (Eq. FinalMP2), used to check the CUDA library.  Only the test
suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the library.

The C sources are compiled on first use (or by ``build()``) into
``oracle/_build/liboracle.so`` with gcc, OpenMP and no floating-point
contraction, so that every operation rounds as written.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
SOURCES = ["mcmp2_oracle.c", "mp2_reference.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library; returns its path."""
    srcs = [os.path.join(_HERE, s) for s in SOURCES]
    if not force and os.path.exists(_SO):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_SO) >= newest:
            return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


class OrSystem(ctypes.Structure):
    _fields_ = [
        ("n_centres", ctypes.c_int),
        ("centres", ctypes.c_void_p),
        ("weight", ctypes.c_void_p),
        ("n_shells", ctypes.c_int),
        ("shell_centre", ctypes.c_void_p),
        ("shell_l", ctypes.c_void_p),
        ("shell_alpha", ctypes.c_void_p),
        ("shell_coef", ctypes.c_void_p),
        ("n_occ", ctypes.c_int),
        ("n_vir", ctypes.c_int),
        ("C", ctypes.c_void_p),
        ("eps", ctypes.c_void_p),
        ("interaction", ctypes.c_int),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_long
_D = ctypes.c_double
_U64 = ctypes.c_uint64


def _declare(L):
    sig = {
        "or_n_functions": (_I, [_P]),
        "or_basis_at": (None, [_P, _P, _P, _P]),
        "or_spinors_at": (None, [_P, _P, _P]),
        "or_g": (_D, [_P, _P]),
        "or_Ng": (_D, [_P]),
        "or_lambda": (_D, [_P]),
        "or_green": (None, [_P, _P, _P, _D, _I, _P]),
        "or_pair_value": (None, [_P, _P, _P, _P, _P, _D, _P]),
        "or_eval_steps": (_I, [_P, _L, _I, _I, _P, _P, _P, _P, _I]),
        "or_eval_pairs": (_I, [_P, _I, _I, _P, _P, _I, _P, _P, _P, _I]),
        "or_philox4x32_10": (None, [_P, _P, _P]),
        "or_tau_draws": (None, [_U64, _U64, _I, _D, _P]),
        "or_metropolis": (_L, [_P, _I, _P, _U64, _U64, _L, _D]),
        "or_burn_in": (_D, [_P, _I, _P, _U64, _L, _D, _I]),
        "or_blocking": (None, [_P, _L, _I, _P]),
        "or_run": (_D, [_P, _I, _P, _U64, _L, _D, _I, _L, _I, _P, _P, _P, _I]),
        "or_max_threads": (_I, []),
        "mp2_prim_eri": (_D, [_P, _D, _P, _P, _D, _P, _P, _D, _P, _P, _D, _P]),
        "mp2_ao_eri": (_D, [_P, _P, _P]),
        "mp2_pair_eri_matrix": (_I, [_P, _I, _P, _P, _I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# Constants of the sampling scheme (also stated in the library's header).
DELTA0 = 0.6          # initial Metropolis displacement, bohr
ADAPT_WINDOW = 20     # burn-in adaptation window, steps
BLOCK_SIZE = 100      # Flyvbjerg-Petersen block size N_b (Sec. IV)


class Oracle:
    """The oracle bound to one system (a ``synthetic.System``)."""

    COULOMB, GAUNT, BREIT = 0, 1, 2

    def __init__(self, system, n_threads: int | None = None, interaction: int = 0):
        """interaction: 0 Coulomb (the paper's runs), 1 Coulomb + Gaunt, 2 Coulomb + Gaunt + gauge
        (the full Breit operator of Sec. II)."""
        if interaction not in (0, 1, 2):
            raise ValueError("interaction must be 0, 1 or 2")
        self.system = system
        self.interaction = interaction
        self._keep = dict(
            centres=_f64(system.centres), weight=_f64(system.weight),
            shell_centre=np.ascontiguousarray(system.shell_centre, dtype=np.int32),
            shell_l=np.ascontiguousarray(system.shell_l, dtype=np.int32),
            shell_alpha=_f64(system.shell_alpha), shell_coef=_f64(system.shell_coef),
            C=np.ascontiguousarray(system.C, dtype=np.complex128), eps=_f64(system.eps))
        k = self._keep
        self._sys = OrSystem(len(k["centres"]), _ptr(k["centres"]).value, _ptr(k["weight"]).value,
                             len(k["shell_l"]), _ptr(k["shell_centre"]).value, _ptr(k["shell_l"]).value,
                             _ptr(k["shell_alpha"]).value, _ptr(k["shell_coef"]).value,
                             int(system.n_occ), int(system.n_vir), _ptr(k["C"]).value, _ptr(k["eps"]).value,
                             int(interaction))
        self.L = lib()
        self.n_threads = n_threads or self.L.or_max_threads()

    @property
    def sp(self):
        return ctypes.byref(self._sys)

    @property
    def n_orb(self):
        return self.system.n_occ + self.system.n_vir

    def n_functions(self) -> int:
        return self.L.or_n_functions(self.sp)

    def basis_at(self, r):
        n = self.n_functions()
        v = np.zeros(n)
        g = np.zeros((n, 3))
        self.L.or_basis_at(self.sp, _ptr(_f64(r)), _ptr(v), _ptr(g))
        return v, g

    def spinors_at(self, r) -> np.ndarray:
        """phi[k, c] complex, c = L-alpha, L-beta, S-alpha, S-beta."""
        out = np.zeros((self.n_orb, 4), dtype=np.complex128)
        self.L.or_spinors_at(self.sp, _ptr(_f64(r)), _ptr(out))
        return out

    def g(self, r) -> float:
        return self.L.or_g(self.sp, _ptr(_f64(r)))

    def Ng(self) -> float:
        return self.L.or_Ng(self.sp)

    def lam(self) -> float:
        return self.L.or_lambda(self.sp)

    def green(self, phi_d, phi_o, tau, kind):
        G = np.zeros((4, 4), dtype=np.complex128)
        self.L.or_green(self.sp, _ptr(np.ascontiguousarray(phi_d, dtype=np.complex128)),
                        _ptr(np.ascontiguousarray(phi_o, dtype=np.complex128)), float(tau), int(kind), _ptr(G))
        return G

    def pair_value(self, r1, r2, r3, r4, tau) -> complex:
        out = np.zeros(2)
        self.L.or_pair_value(self.sp, _ptr(_f64(r1)), _ptr(_f64(r2)), _ptr(_f64(r3)), _ptr(_f64(r4)),
                             float(tau), _ptr(out))
        return complex(out[0], out[1])

    def eval_steps(self, r, tau, with_abs=False):
        r = _f64(r)
        tau = _f64(tau)
        n, m = r.shape[0], r.shape[1]
        n_tau = tau.shape[1]
        per = np.zeros(n)
        ab = np.zeros(n)
        rc = self.L.or_eval_steps(self.sp, n, m, n_tau, _ptr(r), _ptr(tau), _ptr(per), _ptr(ab),
                                  self.n_threads)
        if rc != 0:
            raise ValueError("or_eval_steps rejected its arguments")
        return (per, ab) if with_abs else per

    def eval_pairs(self, r_step, tau_step, p, q):
        r = _f64(r_step)
        tau = _f64(tau_step)
        p = np.ascontiguousarray(p, dtype=np.int32)
        q = np.ascontiguousarray(q, dtype=np.int32)
        out = np.zeros((len(p), len(tau)))
        rc = self.L.or_eval_pairs(self.sp, r.shape[0], len(tau), _ptr(r), _ptr(tau), len(p), _ptr(p),
                                  _ptr(q), _ptr(out), self.n_threads)
        if rc != 0:
            raise ValueError("or_eval_pairs rejected its arguments")
        return out

    def metropolis(self, r, seed, step0, n_steps, delta):
        r = _f64(r).copy()
        acc = self.L.or_metropolis(self.sp, r.shape[0], _ptr(r), seed, step0, n_steps, delta)
        return r, acc

    def burn_in(self, r, seed, n_burn, delta=DELTA0, window=ADAPT_WINDOW):
        r = _f64(r).copy()
        d = self.L.or_burn_in(self.sp, r.shape[0], _ptr(r), seed, n_burn, delta, window)
        return r, d

    def run(self, r, seed, n_burn, n_steps, n_tau, delta0=DELTA0, window=ADAPT_WINDOW):
        r = _f64(r).copy()
        per = np.zeros(n_steps)
        taus = np.zeros((n_steps, n_tau))
        acc = ctypes.c_long(0)
        d = self.L.or_run(self.sp, r.shape[0], _ptr(r), seed, n_burn, delta0, window, n_steps, n_tau,
                          _ptr(per), _ptr(taus), ctypes.byref(acc), self.n_threads)
        return dict(per_step=per, taus=taus, positions=r, delta=d, accepted=acc.value)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def tau_draws(seed, step, n_tau, lam) -> np.ndarray:
    out = np.zeros(n_tau)
    lib().or_tau_draws(seed, step, n_tau, lam, _ptr(out))
    return out


def blocking(per_step, nb=BLOCK_SIZE):
    """(I_N, sigma_N^2, sigma-bar_N, n_blocks) of Eq. uncertainty."""
    x = _f64(per_step)
    out = np.zeros(4)
    lib().or_blocking(_ptr(x), len(x), nb, _ptr(out))
    return float(out[0]), float(out[1]), float(out[2]), int(out[3])
