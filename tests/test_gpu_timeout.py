"""Failure detection without a GPU fault: the bounded waits that every kernel
uses give up after their budget on a barrier phase that nothing completes
(a flag nothing sets), report VBH_ETIMEOUT, and leave the CUDA context
usable; a phase completed by a bulk copy is still observed."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2401_10068_gb300 import synth, vbh

pytestmark = pytest.mark.gpu

VBH_OK, VBH_ETIMEOUT = 0, -5


@pytest.fixture(scope="module")
def built():
    from paper_2401_10068_gb300 import _build
    _build.build_all()


@pytest.mark.parametrize("budget_ns", [1_000, 2_000_000])
def test_wait_on_a_phase_nothing_completes_runs_out(built, budget_ns):
    stream = torch.cuda.current_stream()
    status, waited = vbh.selftest_wait(budget_ns, 0, stream)
    assert status == [VBH_ETIMEOUT, VBH_ETIMEOUT, VBH_OK, VBH_OK]
    assert budget_ns <= waited < budget_ns + 50_000_000          # gave up after the budget, not much later
    # the context is still usable: a small fit matches the oracle
    S, V = 3, 4000
    r, d, _ = synth.generate(V, S, seed=11)
    h = vbh.Handle(0, stream)
    res = h.fit(torch.from_numpy(r).cuda(), torch.from_numpy(d).cuda(), S, None, tol=0.0, max_iter=5)
    h.close()
    want = O.fit(r, d, O.paper_prior(S), tol=0.0, max_iter=5)
    assert res["status"] == 0 and res["iters"] == 5
    assert np.allclose(res["kappa"], want["kappa"], rtol=1e-4, atol=1e-6)


def test_selftest_rejects_bad_budgets(built):
    for bad in (0, 2_000_000_000):
        with pytest.raises(vbh.VBHError):
            vbh.selftest_wait(bad)
