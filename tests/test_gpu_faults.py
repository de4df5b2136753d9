"""Error paths, exercised by host-side fault injection (PAMD_FAULT_INJECT): the
documented status comes back, nothing half-built stays cached, and the library
works normally once the fault is gone.  Nothing faults on the device."""
import os

import pytest

import pamd_inputs as inputs
from _common import gpu_system, start_paths

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pamd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1907_09529_gb300 as pamd
    pamd.tune()
    return pamd


@pytest.fixture
def fault():
    def set_(what):
        if what:
            os.environ["PAMD_FAULT_INJECT"] = what
        else:
            os.environ.pop("PAMD_FAULT_INJECT", None)
    yield set_
    os.environ.pop("PAMD_FAULT_INJECT", None)


def _case(pamd):
    w = inputs.workload("lj108", "small")
    prob = pamd.Problem([gpu_system(s, pamd) for s in w.systems], w.D, w.beta, w.dt)
    buf = prob.empty("cuda")
    for q, p in enumerate(start_paths(w, "fp32")):
        prob.view(buf, q).copy_(torch.from_numpy(p).float())
    return prob, buf


def test_allocation_failure_leaves_no_plan(pamd, fault):
    prob, buf = _case(pamd)
    pamd.release_cache()
    fault("alloc")
    with pytest.raises(pamd.PamdError) as ei:
        pamd.action_grad(prob, buf)
    assert ei.value.status == -6  # PAMD_ERR_ALLOC
    assert pamd.cache_stats() == (0, 0)
    fault(None)
    S, g = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    assert pamd.cache_stats() == (1, 0) and bool(torch.isfinite(S).all())


def test_cuda_failure_is_reported_and_recovers(pamd, fault):
    prob, buf = _case(pamd)
    pamd.release_cache()
    S0, g0 = pamd.action_grad(prob, buf)  # plan built and cached
    torch.cuda.synchronize()
    fault("launch")
    with pytest.raises(pamd.PamdError) as ei:
        pamd.action_grad(prob, buf)
    assert ei.value.status == -3  # PAMD_ERR_CUDA
    nacc = torch.zeros(prob.n_chains, dtype=torch.int32, device="cuda")
    with pytest.raises(pamd.PamdError) as ei:  # a capture that fails caches no graph
        pamd.path_update(prob, buf, g0.clone(), S0.clone(), 1e-6, n_updates=3, n_accepted=nacc)
    assert ei.value.status == -3
    assert pamd.cache_stats() == (1, 0)
    fault(None)
    S1, g1 = pamd.action_grad(prob, buf)
    torch.cuda.synchronize()
    assert torch.equal(S1, S0) and torch.equal(g1, g0)
    pamd.path_update(prob, buf, g1, S1, 1e-6, n_updates=3, n_accepted=nacc)
    torch.cuda.synchronize()
    assert pamd.cache_stats() == (1, 1)


def test_nonfinite_flag_is_reported_once(pamd, fault):
    prob, buf = _case(pamd)
    pamd.device_status()  # clear anything earlier
    fault("nonfinite")
    pamd.action_grad(prob, buf)
    fault(None)
    with pytest.raises(pamd.PamdError) as ei:
        pamd.device_status()
    assert ei.value.status == -5  # PAMD_ERR_NONFINITE
    pamd.device_status()  # cleared
    pamd.action_grad(prob, buf)
    pamd.device_status()  # a clean call reports nothing
