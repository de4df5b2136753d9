"""The FMA throughput probes behind the roofline denominators (pamd_fp32_fma_probe,
pamd_fp64_fma_probe): each thread's chains follow a <- a b + c, so after n steps
a = b^n a0 + c (1 - b^n) / (1 - b); the probes must compute that, report the flops
they perform, and refuse host memory."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1907_09529_gb300 import _lib
    return _lib


def _expected(tid, n, b, c, chains, scale):
    a0 = tid * scale + np.arange(chains)[None, :]
    bn = b ** n
    return (bn * a0 + c * (1 - bn) / (1 - b)).sum(axis=1)


def test_fp64_probe_computes_its_chains(lib):
    blocks, threads, iters = 3, 64, 500
    out = torch.zeros(blocks * threads, dtype=torch.float64, device="cuda")
    fl = lib.pamd_fp64_fma_probe(blocks, threads, iters, ctypes.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert fl == 2.0 * 8 * iters * blocks * threads
    tid = np.arange(blocks * threads, dtype=np.float64)[:, None]
    want = _expected(tid, iters, 0.999999999, 1e-9, 8, 1e-9)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-12)


@pytest.mark.parametrize("packed", [0, 1])
def test_fp32_probe_computes_its_chains(lib, packed):
    blocks, threads, iters = 2, 96, 400
    out = torch.zeros(blocks * threads, dtype=torch.float32, device="cuda")
    fl = lib.pamd_fp32_fma_probe(packed, blocks, threads, iters, ctypes.c_void_p(out.data_ptr()),
                                 None)
    torch.cuda.synchronize()
    assert fl == 2.0 * (2 if packed else 1) * 8 * iters * blocks * threads
    tid = np.arange(blocks * threads, dtype=np.float64)[:, None]
    b, c = float(np.float32(0.999999)), float(np.float32(1e-6))
    want = _expected(tid, iters, b, c, 8, float(np.float32(1e-7)))
    if packed:  # second lane of each pair starts at q / 2
        a0 = 0.5 * np.arange(8)[None, :]
        bn = b ** iters
        want = want + (bn * a0 + c * (1 - bn) / (1 - b)).sum(axis=1)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-4)


def test_probes_refuse_host_memory(lib):
    h32 = torch.zeros(64, dtype=torch.float32)
    h64 = torch.zeros(64, dtype=torch.float64)
    with pytest.raises(lib.PamdError):
        lib.pamd_fp32_fma_probe(0, 1, 64, 10, ctypes.c_void_p(h32.data_ptr()), None)
    with pytest.raises(lib.PamdError):
        lib.pamd_fp64_fma_probe(1, 64, 10, ctypes.c_void_p(h64.data_ptr()), None)
