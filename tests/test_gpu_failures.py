"""Device-side failure handling, exercised without faulting or hanging the GPU.

A bounded mbarrier wait (the one every tensor-core kernel uses) that nothing satisfies gives
up after its limit and reports FM_ERR_TIMEOUT through a status word, after which the context
keeps working; a non-finite parameter vector surfaces as FM_ERR_NONFINITE at the next status
check and the handle keeps working once the status has been read."""
import numpy as np
import pytest

from gpu_cases import as_complex, bound, handle, make_case, quant, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_07090_gb300 import build
    build.build()


def test_bounded_wait_times_out_and_the_context_stays_usable():
    import torch
    from paper_2504_07090_gb300 import fm
    # about a millisecond of SM clock; nothing ever arrives at the barrier
    assert fm.diag_bounded_wait(2_000_000) == fm.FM_ERR_TIMEOUT
    assert fm.diag_bounded_wait(2_000_000) == fm.FM_ERR_TIMEOUT
    # the same context still computes correctly
    p, o, th, d, mu, lam = make_case("small")
    h = handle(p, "fp32")
    v = h.forward(torch.tensor(quant("fp32", th), dtype=torch.float32, device="cuda"))
    assert rel_l2(as_complex(v), o.model(quant("fp32", th))) < bound("direct", "V", "fp32")
    h.sync_status()


def test_nonfinite_parameters_report_and_clear():
    import torch
    from paper_2504_07090_gb300 import fm
    p, o, th, d, mu, lam = make_case("small")
    d, mu, lam = quant("fp32", d, mu, lam)
    h = handle(p, "fp32", d, mu, lam)
    bad = torch.tensor(th, dtype=torch.float32, device="cuda")
    bad[3] = float("nan")
    h.chi2_grad(bad)
    with pytest.raises(fm.FmError) as e:
        h.sync_status()
    assert e.value.status == fm.FM_ERR_NONFINITE
    # reading the status cleared it: a finite evaluation goes through
    good = torch.tensor(quant("fp32", th), dtype=torch.float32, device="cuda")
    scal, _ = h.chi2_grad(good)
    h.sync_status()
    assert np.isfinite(float(scal[0]))
