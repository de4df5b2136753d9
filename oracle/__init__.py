"""CPU FP64 oracle for the path action of path-accelerated MD (arXiv:1907.09529).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product library never calls it and shares no code with it.

The arithmetic lives in ``pamd_oracle.c`` (plain C, double precision, no FMA
contraction); this module compiles it with gcc and marshals numpy arrays to it.
Each wrapper names the part of the paper it follows:

* ``force`` / ``hvp`` / ``potential_energy`` -- the potentials of Sec. IV
  (harmonic oscillator; cut-and-force-shifted Lennard-Jones, Eq. (11)).
* ``residuals`` / ``action_grad`` -- Eq. (3) (short-time propagator) and
  Eq. (4) (path likelihood exp(-S)), with the gradient derived from them.
* ``euler`` -- the forward Euler-Maruyama step, Eq. (2).
* ``mala_step`` -- a Metropolis-Hastings path update with the tail slice
  fixed (Sec. III), proposing along the path gradient.
* ``philox`` / ``normals`` -- Philox4x32-10 (Salmon et al., SC'11) and
  Box-Muller normals, used where the method draws random numbers.
* ``pair_count_f32`` -- the cutoff decision in single precision, for
  bit-exact index parity with the GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pamd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

HARMONIC = 0
LJ = 1


def build(force: bool = False) -> str:
    """Compile ``pamd_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("k", ctypes.c_double), ("eps", ctypes.c_double),
                ("sigma", ctypes.c_double), ("rc", ctypes.c_double), ("box", ctypes.c_double)]


def harmonic(k: float = 1.0) -> Potential:
    return Potential(HARMONIC, k, 0.0, 0.0, 0.0, 0.0)


def lennard_jones(box: float, rc: float = 2.5, eps: float = 1.0, sigma: float = 1.0) -> Potential:
    return Potential(LJ, 0.0, eps, sigma, rc, box)


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_P = ctypes.POINTER(Potential)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c_int, c_double, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "or_lj_pair_energy": (c_double, [_P, c_double]),
            "or_lj_pair_dU": (c_double, [_P, c_double]),
            "or_lj_pair_d2U": (c_double, [_P, c_double]),
            "or_potential_energy": (c_double, [_P, c_int, c_int, _D]),
            "or_force": (None, [_P, c_int, c_int, _D, _D]),
            "or_hvp": (None, [_P, c_int, c_int, _D, _D, _D]),
            "or_residuals": (c_int, [_P, c_int, c_int, c_int, c_double, c_double, c_double, _D, _D]),
            "or_action_grad": (c_int, [_P, c_int, c_int, c_int, c_double, c_double, c_double, _D,
                                       _D, _D, c_int]),
            "or_step_actions": (c_int, [_P, c_int, c_int, c_int, c_double, c_double, c_double, _D,
                                        c_int, _I, _D]),
            "or_grad_slices": (c_int, [_P, c_int, c_int, c_int, c_double, c_double, c_double, _D,
                                       c_int, _I, _D]),
            "or_euler": (c_int, [_P, c_int, c_int, c_int, c_double, c_double, c_double, _D, c_int,
                                 _D]),
            "or_euler_batch": (c_int, [_P, c_int, c_int, c_int, c_int, c_double, c_double, c_double,
                                       _D, c_int, _D, c_int]),
            "or_mala_step": (c_int, [_P, c_int, c_int, c_int, c_double, c_double, c_double, c_double,
                                     _D, c_double, _D, _D, c_double, c_int, _D, _D, _D, _D, _I,
                                     c_int]),
            "or_fragment_step": (c_int, [_P, c_int, c_int, c_int, c_double, c_double, c_double,
                                         c_int, c_int, _D, _D, _D, _I, _I, c_int]),
            "or_shift_regenerate": (None, [c_int, c_int, c_int, c_double, c_double, c_int, _D, _D,
                                           _D, _D]),
            "or_philox4x32_10": (None, [_U32, _U32, _U32]),
            "or_normals": (None, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, _D]),
            "or_uniform": (c_double, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_uint32]),
            "or_pair_count_f32": (c_ll, [c_int, c_double, c_double, _F]),
            "or_hs_first_overlap": (c_int, [ctypes.POINTER(Potential), c_int, c_int, c_int, _D,
                                            _D]),
            "or_hs_overlap_f32": (c_int, [c_int, c_double, c_double, c_double, _F]),
            "or_num_threads_available": (c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(_load().or_num_threads_available())


# ---------------------------------------------------------------- pair functions (Eq. (11))
def lj_pair_energy(pot: Potential, r: float) -> float:
    return _load().or_lj_pair_energy(ctypes.byref(pot), float(r))


def lj_pair_dU(pot: Potential, r: float) -> float:
    return _load().or_lj_pair_dU(ctypes.byref(pot), float(r))


def lj_pair_d2U(pot: Potential, r: float) -> float:
    return _load().or_lj_pair_d2U(ctypes.byref(pot), float(r))


# ---------------------------------------------------------------- one slice x[d][N]
def potential_energy(pot: Potential, x: np.ndarray) -> float:
    x = _f64(x)
    d, N = x.shape
    return _load().or_potential_energy(ctypes.byref(pot), N, d, _d(x))


def force(pot: Potential, x: np.ndarray) -> np.ndarray:
    x = _f64(x)
    d, N = x.shape
    F = np.empty_like(x)
    _load().or_force(ctypes.byref(pot), N, d, _d(x), _d(F))
    return F


def hvp(pot: Potential, x: np.ndarray, v: np.ndarray) -> np.ndarray:
    x, v = _f64(x), _f64(v)
    d, N = x.shape
    out = np.empty_like(x)
    _load().or_hvp(ctypes.byref(pot), N, d, _d(x), _d(v), _d(out))
    return out


# ---------------------------------------------------------------- one path pos[T+1][d][N]
def residuals(pot: Potential, pos: np.ndarray, D: float, beta: float, dt: float) -> np.ndarray:
    pos = _f64(pos)
    T = pos.shape[0] - 1
    _, d, N = pos.shape
    r = np.empty((T, d, N))
    rc = _load().or_residuals(ctypes.byref(pot), N, d, T, D, beta, dt, _d(pos), _d(r))
    if rc:
        raise MemoryError("oracle residuals")
    return r


def action_grad(pot: Potential, pos: np.ndarray, D: float, beta: float, dt: float,
                grad: bool = True, nthreads: int = 1):
    """S (Eq. (4), unnormalised) and dS/dx for one chain; pos is [T+1][d][N]."""
    pos = _f64(pos)
    T = pos.shape[0] - 1
    _, d, N = pos.shape
    S = ctypes.c_double(0.0)
    g = np.empty_like(pos) if grad else None
    rc = _load().or_action_grad(ctypes.byref(pot), N, d, T, D, beta, dt, _d(pos),
                                ctypes.byref(S), _d(g) if grad else None, int(nthreads))
    if rc:
        raise MemoryError("oracle action_grad")
    return (S.value, g) if grad else S.value


def step_actions(pot: Potential, pos: np.ndarray, D: float, beta: float, dt: float, t_list):
    pos = _f64(pos)
    T = pos.shape[0] - 1
    _, d, N = pos.shape
    ts = np.ascontiguousarray(t_list, dtype=np.int32)
    out = np.empty(len(ts))
    _load().or_step_actions(ctypes.byref(pot), N, d, T, D, beta, dt, _d(pos), len(ts),
                            ts.ctypes.data_as(_I), _d(out))
    return out


def grad_slices(pot: Potential, pos: np.ndarray, D: float, beta: float, dt: float, t_list):
    pos = _f64(pos)
    T = pos.shape[0] - 1
    _, d, N = pos.shape
    ts = np.ascontiguousarray(t_list, dtype=np.int32)
    out = np.empty((len(ts), d, N))
    _load().or_grad_slices(ctypes.byref(pot), N, d, T, D, beta, dt, _d(pos), len(ts),
                           ts.ctypes.data_as(_I), _d(out))
    return out


def euler(pot: Potential, x0: np.ndarray, xi: np.ndarray, D: float, beta: float, dt: float,
          store_f32: bool = False) -> np.ndarray:
    """Euler-Maruyama path (Eq. (2)) from x0 [d][N] with noise xi [T][d][N]."""
    x0, xi = _f64(x0), _f64(xi)
    T = xi.shape[0]
    d, N = x0.shape
    pos = np.empty((T + 1, d, N))
    pos[0] = x0
    if _load().or_euler(ctypes.byref(pot), N, d, T, D, beta, dt, _d(xi), int(store_f32), _d(pos)):
        raise MemoryError("oracle euler")
    return pos


def euler_batch(pot: Potential, x0: np.ndarray, xi: np.ndarray, D: float, beta: float,
                dt: float, store_f32: bool = False, nthreads: int = 0) -> np.ndarray:
    """Independent chains: x0 [B][d][N], xi [B][T][d][N] -> pos [B][T+1][d][N]."""
    x0, xi = _f64(x0), _f64(xi)
    B, T = xi.shape[:2]
    _, d, N = x0.shape
    pos = np.empty((B, T + 1, d, N))
    pos[:, 0] = x0
    nth = nthreads if nthreads > 0 else max_threads()
    if _load().or_euler_batch(ctypes.byref(pot), B, N, d, T, D, beta, dt, _d(xi),
                              int(store_f32), _d(pos), nth):
        raise MemoryError("oracle euler_batch")
    return pos


def mala_step(pot: Potential, pos: np.ndarray, S: float, grad: np.ndarray, eta: np.ndarray,
              log_u: float, h: float, D: float, beta: float, dt: float,
              store_f32: bool = False, nthreads: int = 1):
    """One whole-path MALA proposal + Metropolis-Hastings test (tail x_0 fixed).

    Returns dict(prop, S_prop, grad_prop, log_alpha, accepted)."""
    pos, grad, eta = _f64(pos), _f64(grad), _f64(eta)
    T = pos.shape[0] - 1
    _, d, N = pos.shape
    prop = np.empty_like(pos)
    gp = np.empty_like(pos)
    Sp = ctypes.c_double(0.0)
    la = ctypes.c_double(0.0)
    acc = ctypes.c_int(0)
    rc = _load().or_mala_step(ctypes.byref(pot), N, d, T, D, beta, dt, h, _d(pos), float(S),
                              _d(grad), _d(eta), float(log_u), int(store_f32), _d(prop),
                              ctypes.byref(Sp), _d(gp), ctypes.byref(la), ctypes.byref(acc),
                              int(nthreads))
    if rc:
        raise MemoryError("oracle mala_step")
    return dict(prop=prop, S_prop=Sp.value, grad_prop=gp, log_alpha=la.value,
                accepted=bool(acc.value))


def fragment_step(pot: Potential, pos: np.ndarray, level: int, offset: int, z: np.ndarray,
                  log_u, D: float, beta: float, dt: float, exact_ho: bool = False):
    """One multilevel sliding-and-sampling MC step (Sec. III, Fig. 5) with
    free-particle trials; pos [T+1][d][N] is updated in place.  z has the layout
    of pos (slice-0 entries unused); log_u holds one log uniform per fragment.
    exact_ho: the oscillator's exact transition density in place of Eq. (3).
    Returns (n_fragments, n_accepted, n_proposed)."""
    assert pos.dtype == np.float64 and pos.flags.c_contiguous
    T = pos.shape[0] - 1
    _, d, N = pos.shape
    z = _f64(z)
    lu = _f64(log_u)
    acc, prop = ctypes.c_int(0), ctypes.c_int(0)
    nf = _load().or_fragment_step(ctypes.byref(pot), N, d, T, D, beta, dt, int(level), int(offset),
                                  _d(z), _d(lu), _d(pos), ctypes.byref(acc), ctypes.byref(prop),
                                  int(bool(exact_ho)))
    if nf == -2:
        raise ValueError("exact_ho needs the harmonic potential")
    if nf < 0:
        raise MemoryError("oracle fragment_step")
    return nf, acc.value, prop.value


def shift_regenerate(pos: np.ndarray, n_shift: int, z: np.ndarray, D: float, dt: float):
    """Shift by n_shift steps and regrow the nose with free-particle steps (Fig. 2).
    Returns (new path, trajectory points x_1..x_{n_shift})."""
    pos, z = _f64(pos), _f64(z)
    T = pos.shape[0] - 1
    _, d, N = pos.shape
    out = np.empty_like(pos)
    traj = np.empty((n_shift, d, N))
    _load().or_shift_regenerate(N, d, T, D, dt, int(n_shift), _d(pos), _d(z), _d(out), _d(traj))
    return out, traj


def n_fragments(T: int, level: int, offset: int) -> int:
    """Fragments of a path of T steps at this level and offset."""
    return 1 + sum(1 for e in range(offset, T, 1 << level) if e > 0)


# ---------------------------------------------------------------- random numbers
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    _load().or_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32),
                             out.ctypes.data_as(_U32))
    return out


def normals(seed: int, counter: int, stream: int, chain: int, n: int, e0: int = 0) -> np.ndarray:
    out = np.empty(int(n))
    _load().or_normals(seed, counter, stream, chain, e0, int(n), _d(out))
    return out


def uniform(seed: int, counter: int, stream: int, chain: int) -> float:
    return _load().or_uniform(seed, counter, stream, chain)


# ---------------------------------------------------------------- index parity
def pair_count_f32(box: float, rc: float, x: np.ndarray) -> int:
    """Ordered in-cutoff pairs of one slice x[3][N] (float32), decided in FP32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    d, N = x.shape
    assert d == 3
    return int(_load().or_pair_count_f32(N, float(box), float(rc), x.ctypes.data_as(_F)))


def hs_first_overlap(pot: Potential, pos: np.ndarray, sigma_hs) -> int:
    """First slice t of pos [T+1][d][N] with a pair at r <= sigma_hs[t] (within the
    cutoff), or -1: the slices where the hard-sphere bias of the paper's LJ runs
    (Sec. IV.B) is infinite."""
    pos = _f64(pos)
    T = pos.shape[0] - 1
    _, d, N = pos.shape
    sig = np.ascontiguousarray(sigma_hs, dtype=np.float64)
    assert sig.shape == (T + 1,)
    return int(_load().or_hs_first_overlap(ctypes.byref(pot), N, d, T, _d(pos), _d(sig)))


def action_grad_hs(pot: Potential, pos: np.ndarray, sigma_hs, D: float, beta: float, dt: float,
                   nthreads: int = 1):
    """Action and gradient with the hard-sphere path bias: the LJ action, or +inf
    if any slice t has a pair at r <= sigma_hs[t]; the gradient is the LJ one
    (the bias adds no force where it is finite)."""
    S, g = action_grad(pot, pos, D, beta, dt, nthreads=nthreads)
    if hs_first_overlap(pot, pos, sigma_hs) >= 0:
        S = float("inf")
    return S, g


def hs_overlap_f32(box: float, rc: float, sigma: float, x: np.ndarray) -> bool:
    """The hard-sphere overlap decision at one slice x[3][N] (float32) in single
    precision, by the GPU's documented rule."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    N = x.shape[-1]
    return bool(_load().or_hs_overlap_f32(N, float(box), float(rc), float(sigma),
                                          x.ctypes.data_as(_F)))
