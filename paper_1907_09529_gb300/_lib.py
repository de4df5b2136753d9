"""ctypes binding of libpamd's C ABI (``include/pamd.h``); argument marshalling only.

The shared library is built in-tree by ``paper_1907_09529_gb300.build``.  There is
no fallback: if the library is missing or cannot be loaded, every entry point
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# PAMD_LIBRARY=debug loads the bounds-checked build (libpamd_debug.so) instead
LIB_PATH = os.path.join(HERE, "libpamd_debug.so" if os.environ.get("PAMD_LIBRARY") == "debug"
                        else "libpamd.so")

PAMD_OK = 0
PAMD_ERR_ARG = -1
PAMD_ERR_UNSUPPORTED = -2
PAMD_ERR_CUDA = -3
PAMD_ERR_TIMEOUT = -4
PAMD_ERR_NONFINITE = -5
PAMD_ERR_ALLOC = -6

PAMD_HARMONIC = 0
PAMD_LJ = 1
PAMD_FP32 = 0
PAMD_FP64 = 1
PAMD_FLAG_ONE_CHAIN_PER_LAUNCH = 1
PAMD_FLAG_HO_EXACT_PROPAGATOR = 2
PAMD_FLAG_REGENERATE_FLAT = 4

#: Every entry point declared in include/pamd.h.
EXPORTS = (
    "pamd_action", "pamd_action_grad", "pamd_path_update", "pamd_euler_reference",
    "pamd_lj_pair_counts", "pamd_philox", "pamd_normals", "pamd_status_string",
    "pamd_release_cache", "pamd_version", "pamd_tune", "pamd_ho_action_grad_noalloc",
    "pamd_device_status", "pamd_fragment_mc", "pamd_shift_regenerate", "pamd_event",
    "pamd_cache_stats", "pamd_fp32_fma_probe", "pamd_fp64_fma_probe", "pamd_pipeline_timeline",
    "pamd_mala_propose", "pamd_mala_reverse", "pamd_mala_accept", "pamd_mala_commit",
    "pamd_debug_status", "pamd_action_grad_hs",
)

#: Scratch capacity of pamd_ho_action_grad_noalloc (block sums; one per 4096 elements).
PAMD_NOALLOC_MAX_BLOCKS = 65536


class pamd_potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("k", ctypes.c_double), ("eps", ctypes.c_double),
                ("sigma", ctypes.c_double), ("rc", ctypes.c_double), ("box", ctypes.c_double)]


class pamd_system(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int), ("n_steps", ctypes.c_int), ("dim", ctypes.c_int),
                ("n_chains", ctypes.c_int), ("pos_offset", ctypes.c_longlong),
                ("pot", pamd_potential), ("first_slice", ctypes.c_longlong),
                ("halo_lo", ctypes.c_int), ("halo_hi", ctypes.c_int)]


class pamd_problem(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("beta", ctypes.c_double), ("dt", ctypes.c_double),
                ("n_systems", ctypes.c_int), ("systems", ctypes.POINTER(pamd_system)),
                ("precision", ctypes.c_int), ("flags", ctypes.c_int)]


class PamdError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed: {msg} ({status})")
        self.status = status


_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_PP = ctypes.POINTER(pamd_problem)


def load(path: str = LIB_PATH):
    """Load libpamd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(
                f"libpamd.so not found at {path}; build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        u32, u64, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_longlong
        sig = {
            "pamd_action": (ctypes.c_int, [_PP, _VP, _VP, _VP]),
            "pamd_action_grad": (ctypes.c_int, [_PP, _VP, _VP, _VP, _VP]),
            "pamd_path_update": (ctypes.c_int, [_PP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                                u64, u64, _VP, _VP, _VP, _VP, _VP]),
            "pamd_euler_reference": (ctypes.c_int, [_PP, _VP, u64, u64, _VP, _VP]),
            "pamd_lj_pair_counts": (ctypes.c_int, [_PP, _VP, _VP, _VP]),
            "pamd_philox": (ctypes.c_int, [u32, u32, u32, u32, u32, u32, i64, _VP, _VP]),
            "pamd_normals": (ctypes.c_int, [u64, u64, u32, u32, i64, i64, _VP, _VP]),
            "pamd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "pamd_release_cache": (ctypes.c_int, []),
            "pamd_version": (ctypes.c_int, []),
            "pamd_tune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int]),
            "pamd_ho_action_grad_noalloc": (ctypes.c_int, [_PP, _VP, _VP, _VP, _VP]),
            "pamd_device_status": (ctypes.c_int, [_VP]),
            "pamd_cache_stats": (ctypes.c_int, [_VP, _VP]),
            "pamd_debug_status": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
            "pamd_action_grad_hs": (ctypes.c_int, [_PP, _VP, _VP, _VP, _VP, _VP]),
            "pamd_mala_propose": (ctypes.c_int, [_PP, _VP, _VP, _VP, ctypes.c_double, u64, u64,
                                                 _VP, _VP, _VP]),
            "pamd_mala_reverse": (ctypes.c_int, [_PP, _VP, _VP, _VP, ctypes.c_double, _VP, _VP]),
            "pamd_mala_accept": (ctypes.c_int, [_PP, _VP, _VP, _VP, _VP, ctypes.c_double, u64, u64,
                                                _VP, _VP, _VP, _VP, _VP]),
            "pamd_mala_commit": (ctypes.c_int, [_PP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
            "pamd_pipeline_timeline": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
            "pamd_fp32_fma_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, _VP, _VP, _VP]),
            "pamd_fp64_fma_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   _VP, _VP, _VP]),
            "pamd_fragment_mc": (ctypes.c_int, [_PP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                u64, u64, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
            "pamd_shift_regenerate": (ctypes.c_int, [_PP, _VP, _VP, ctypes.c_int, _VP, u64, u64,
                                                     _VP, _VP]),
            "pamd_event": (ctypes.c_int, [_PP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _VP, u64, u64, _VP, _VP, _VP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(fn: str, status: int) -> None:
    if status != PAMD_OK:
        msg = load().pamd_status_string(status).decode()
        raise PamdError(fn, status, msg)


def _call(name, *args):
    st = getattr(load(), name)(*args)
    check(name, st)
    return st


# Same names as the C ABI; arguments are ctypes values / raw addresses.
def pamd_action(prob, pos, S, stream):
    return _call("pamd_action", prob, pos, S, stream)


def pamd_action_grad(prob, pos, S, grad, stream):
    return _call("pamd_action_grad", prob, pos, S, grad, stream)


def pamd_action_grad_hs(prob, pos, sigma_hs, S, grad, stream):
    return _call("pamd_action_grad_hs", prob, pos, sigma_hs, S, grad, stream)


def pamd_path_update(prob, pos, grad, S, h, n_updates, seed, counter, noise, log_u, n_accepted,
                     log_alpha, stream):
    return _call("pamd_path_update", prob, pos, grad, S, h, n_updates, seed, counter, noise,
                 log_u, n_accepted, log_alpha, stream)


def pamd_mala_propose(prob, pos, grad, prop, h, seed, counter, noise, q_fwd, stream):
    return _call("pamd_mala_propose", prob, pos, grad, prop, h, seed, counter, noise, q_fwd, stream)


def pamd_mala_reverse(prob, pos, prop, grad_prop, h, q_rev, stream):
    return _call("pamd_mala_reverse", prob, pos, prop, grad_prop, h, q_rev, stream)


def pamd_mala_accept(prob, S, S_prop, q_fwd, q_rev, h, seed, counter, log_u, accept, n_accepted,
                     log_alpha, stream):
    return _call("pamd_mala_accept", prob, S, S_prop, q_fwd, q_rev, h, seed, counter, log_u,
                 accept, n_accepted, log_alpha, stream)


def pamd_mala_commit(prob, pos, grad, S, prop, grad_prop, S_prop, accept, stream):
    return _call("pamd_mala_commit", prob, pos, grad, S, prop, grad_prop, S_prop, accept, stream)


def pamd_euler_reference(prob, pos, seed, counter, noise, stream):
    return _call("pamd_euler_reference", prob, pos, seed, counter, noise, stream)


def pamd_lj_pair_counts(prob, pos, counts, stream):
    return _call("pamd_lj_pair_counts", prob, pos, counts, stream)


def pamd_philox(ctr0, ctr1, ctr2, ctr3, key0, key1, n, out, stream):
    return _call("pamd_philox", ctr0, ctr1, ctr2, ctr3, key0, key1, n, out, stream)


def pamd_normals(seed, counter, stream_id, chain, e0, n, out, stream):
    return _call("pamd_normals", seed, counter, stream_id, chain, e0, n, out, stream)


def pamd_tune(tile_steps, threads_per_particle, max_neighbours, skin, window_steps):
    return _call("pamd_tune", tile_steps, threads_per_particle, max_neighbours, skin, window_steps)


def pamd_fragment_mc(prob, pos, l_min, l_max, n_steps, seed, counter, levels, offsets, noise,
                     log_u, n_accepted, n_proposed, stream):
    return _call("pamd_fragment_mc", prob, pos, l_min, l_max, n_steps, seed, counter, levels,
                 offsets, noise, log_u, n_accepted, n_proposed, stream)


def pamd_shift_regenerate(prob, pos, pos_out, n_shift, traj, seed, counter, noise, stream):
    return _call("pamd_shift_regenerate", prob, pos, pos_out, n_shift, traj, seed, counter, noise,
                 stream)


def pamd_event(prob, pos, pos_out, n_sample, n_shift, l_min, l_max, traj, seed, event,
               n_accepted, n_proposed, stream):
    return _call("pamd_event", prob, pos, pos_out, n_sample, n_shift, l_min, l_max, traj, seed,
                 event, n_accepted, n_proposed, stream)


def pamd_device_status(stream):
    return _call("pamd_device_status", stream)


def pamd_release_cache():
    return _call("pamd_release_cache")


def pamd_pipeline_timeline():
    """(total ms, [(inputs on device, update done, results on host) ms per chunk]) of
    the last host-buffer update pipelined over chunks of chains."""
    n = ctypes.c_int(0)
    _call("pamd_pipeline_timeline", None, 0, ctypes.byref(n))
    buf = (ctypes.c_float * (1 + 3 * n.value))()
    _call("pamd_pipeline_timeline", buf, 1 + 3 * n.value, ctypes.byref(n))
    return buf[0], [tuple(buf[1 + 3 * k:4 + 3 * k]) for k in range(n.value)]


def pamd_debug_status():
    """(checks compiled, out-of-bounds accesses, first site, its index, its bound)
    of the kernels since the last call; see include/pamd.h."""
    v = [ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_longlong(0),
         ctypes.c_longlong(0)]
    _call("pamd_debug_status", *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def pamd_cache_stats():
    """(cached plans, captured update graphs) of the library's cache."""
    n_plans, n_graphs = ctypes.c_int(0), ctypes.c_int(0)
    _call("pamd_cache_stats", ctypes.byref(n_plans), ctypes.byref(n_graphs))
    return n_plans.value, n_graphs.value


def pamd_fp32_fma_probe(packed, blocks, threads, iters, out, stream):
    """Launch the FMA throughput probe; returns the flops it performs."""
    flops = ctypes.c_double(0.0)
    _call("pamd_fp32_fma_probe", int(packed), int(blocks), int(threads), int(iters), out,
          ctypes.byref(flops), stream)
    return flops.value


def pamd_fp64_fma_probe(blocks, threads, iters, out, stream):
    """Launch the FP64 FMA throughput probe; returns the flops it performs."""
    flops = ctypes.c_double(0.0)
    _call("pamd_fp64_fma_probe", int(blocks), int(threads), int(iters), out,
          ctypes.byref(flops), stream)
    return flops.value


def pamd_version():
    return load().pamd_version()


def pamd_ho_action_grad_noalloc(prob, pos, S, grad, stream):
    """Harmonic action + gradient using only the caller's buffers and the
    library's fixed scratch array (no device allocation); see include/pamd.h."""
    return _call("pamd_ho_action_grad_noalloc", prob, pos, S, grad, stream)
