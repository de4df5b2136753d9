"""pamd_ho_action_grad_noalloc: the harmonic action and gradient for callers
that cannot allocate device memory at run time (their allocator already owns
the GPU's memory, or allocation is forbidden after start-up).  It must give the
same S and gradient as pamd_action_grad, call after call, through the C ABI.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import pamd_inputs as inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problem(pamd, precision):
    systems = [pamd.System("harmonic", 1, 3, 4133, 3, k=1.0),
               pamd.System("harmonic", 5, 2, 977, 2, k=0.7)]
    return pamd.Problem(systems, 1.0, 1.0, 0.005, precision=precision)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_noalloc_matches_planned_entry_point(precision, tol):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1907_09529_gb300 as pamd
    from paper_1907_09529_gb300 import _lib
    prob = _problem(pamd, precision)
    buf = prob.empty("cuda")
    for q, s in enumerate(prob.systems):
        x = inputs.gaussian_path(inputs.SEED_BASE + 40 + q, s.n_chains, s.T, s.d, s.N, 1.0)
        prob.view(buf, q).copy_(torch.from_numpy(x).to(prob.dtype))
    S_ref, g_ref = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        S = torch.full((prob.n_chains,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full_like(buf, float("nan"))
        st = _lib.load().pamd_ho_action_grad_noalloc(prob.ref, ctypes.c_void_p(buf.data_ptr()),
                                                     ctypes.c_void_p(S.data_ptr()),
                                                     ctypes.c_void_p(g.data_ptr()), stream)
        assert st == _lib.PAMD_OK, _lib.load().pamd_status_string(st)
        torch.cuda.synchronize()
        rs = ((S - S_ref).abs() / S_ref.abs()).max().item()
        assert rs <= tol, (call, rs)
        for q in range(len(prob.systems)):
            a, b = prob.view(g, q).double(), prob.view(g_ref, q).double()
            assert ((a - b).norm() / b.norm()).item() <= tol, (call, q)


def test_noalloc_matches_oracle():
    """One shape against the FP64 CPU oracle directly (plain FP64 path, 1e-12)."""
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1907_09529_gb300 as pamd
    from paper_1907_09529_gb300 import _lib
    D, beta, dt, k = 1.0, 1.0, 0.005, 0.7
    prob = pamd.Problem([pamd.System("harmonic", 5, 2, 977, 2, k=k)], D, beta, dt, precision="fp64")
    x = inputs.gaussian_path(inputs.SEED_BASE + 45, 2, 977, 2, 5, 1.0)
    buf = prob.empty("cuda")
    prob.view(buf, 0).copy_(torch.from_numpy(x))
    S = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full_like(buf, float("nan"))
    p = ctypes.c_void_p
    st = _lib.load().pamd_ho_action_grad_noalloc(prob.ref, p(buf.data_ptr()), p(S.data_ptr()),
                                                 p(g.data_ptr()), p(0))
    assert st == _lib.PAMD_OK, _lib.load().pamd_status_string(st)
    torch.cuda.synchronize()
    gk = prob.view(g, 0).cpu().numpy()
    for b in range(2):
        So, go = oracle.action_grad(oracle.harmonic(k), x[b], D, beta, dt, nthreads=4)
        assert abs(S[b].item() - So) <= 1e-12 * abs(So)
        assert np.linalg.norm(gk[b] - go) <= 1e-12 * np.linalg.norm(go)


def test_noalloc_rejects_oversize_and_non_harmonic():
    """Rejected before anything is enqueued.  The buffers are host memory, so a
    regression in the size checks is stopped by the pointer check (PAMD_ERR_ARG,
    failing the assertion) instead of launching over a too-small buffer."""
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1907_09529_gb300 as pamd
    from paper_1907_09529_gb300 import _lib
    lib = _lib.load()
    small = torch.zeros(64)      # host memory
    S = torch.zeros(4, dtype=torch.float64)
    p = ctypes.c_void_p
    # one chain needing one block more than the scratch array holds
    T = (_lib.PAMD_NOALLOC_MAX_BLOCKS * 4096) // 3
    big = pamd.Problem([pamd.System("harmonic", 1, 3, T, 1)], 1.0, 1.0, 0.01)
    st = lib.pamd_ho_action_grad_noalloc(big.ref, p(small.data_ptr()), p(S.data_ptr()),
                                         p(small.data_ptr()), p(0))
    assert st == _lib.PAMD_ERR_UNSUPPORTED
    # 65536 one-block chains: within the block budget, beyond the grid's 65535 rows
    wide = pamd.Problem([pamd.System("harmonic", 1, 1, 1, 65536)], 1.0, 1.0, 0.01)
    st = lib.pamd_ho_action_grad_noalloc(wide.ref, p(small.data_ptr()), p(S.data_ptr()),
                                         p(small.data_ptr()), p(0))
    assert st == _lib.PAMD_ERR_UNSUPPORTED
    lj = pamd.Problem([pamd.System("lj", 8, 3, 4, 1, box=6.0, rc=2.5)], 1.0, 1.0, 1e-4)
    st = lib.pamd_ho_action_grad_noalloc(lj.ref, p(small.data_ptr()), p(S.data_ptr()),
                                         p(small.data_ptr()), p(0))
    assert st == _lib.PAMD_ERR_ARG
    # a valid shape with host buffers: refused by the pointer check
    ok = pamd.Problem([pamd.System("harmonic", 1, 3, 4, 1)], 1.0, 1.0, 0.01)
    st = lib.pamd_ho_action_grad_noalloc(ok.ref, p(small.data_ptr()), p(S.data_ptr()),
                                         p(small.data_ptr()), p(0))
    assert st == _lib.PAMD_ERR_ARG
