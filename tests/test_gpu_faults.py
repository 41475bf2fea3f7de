"""Failure handling with faults made on the host (no GPU fault, trap or
hang): with FK_TEST_FAIL_ALLOC=n the n-th device allocation after the
variable is set fails as if the device were out of memory.

* plan creation fails with FK_ERR_OOM at each of its allocations, frees
  what it had, and the next plan works;
* the adjoint fails with FK_ERR_OOM when its workspace cannot be had, and
  runs afterwards;
* the bounded device waits are covered in test_gpu_batched.py (a barrier
  whose phantom CTA never arrives ends with FK_ERR_TIMEOUT).
"""
import math

import pytest

import fk_inputs

pytestmark = pytest.mark.gpu

SPEC = dict(n=(81, 41), lo=(0.0, 0.0), hi=(2.0, 1.0), family="cellular_flow",
            params=(1.0, 0.2, 2 * math.pi, 0.02), q=4, dt=1e-3, n_steps=10)


@pytest.fixture(scope="module")
def fk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_14561_gb300 as fk
    fk.load()
    return fk


def _spec(fk, **kw):
    return fk.PlanSpec(**{**SPEC, **kw})


def test_plan_create_allocation_failures(fk, monkeypatch):
    import torch
    from paper_2104_14561_gb300 import _lib as L
    ref_plan = fk.Plan(_spec(fk))
    ref = ref_plan.solve()
    torch.cuda.synchronize()
    failed = 0
    for n in range(1, 9):
        monkeypatch.setenv("FK_TEST_FAIL_ALLOC", str(n))
        try:
            plan = fk.Plan(_spec(fk))
        except L.FkError as e:
            assert L.STATUS[e.status] == "FK_ERR_OOM"
            failed += 1
        else:
            plan.close()  # n is past the plan's allocations
        monkeypatch.delenv("FK_TEST_FAIL_ALLOC")
        plan = fk.Plan(_spec(fk))  # the library is still usable
        assert torch.equal(plan.solve(), ref)
        plan.close()
    assert failed >= 3  # error word, scratch field and both tables at least
    ref_plan.close()


def test_adjoint_allocation_failure(fk, monkeypatch):
    import torch
    from paper_2104_14561_gb300 import _lib as L
    plan = fk.Plan(_spec(fk))
    g = torch.ones(plan.shape, dtype=torch.float64, device="cuda")
    monkeypatch.setenv("FK_TEST_FAIL_ALLOC", "1")
    with pytest.raises(L.FkError) as e:
        plan.adjoint(g)
    assert L.STATUS[e.value.status] == "FK_ERR_OOM"
    monkeypatch.delenv("FK_TEST_FAIL_ALLOC")
    dth, du = plan.adjoint(g)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    assert torch.isfinite(dth).all() and torch.isfinite(du).all()
    plan.close()
