"""Host-side validation at the C ABI (no GPU fault is provoked: every case
is rejected before any kernel runs)."""
import ctypes as C

import pytest
import torch

import oracle
from helpers import make

pytestmark = pytest.mark.gpu


def _call_eval(gp, K=1, ws_bytes=None, ws_offset=0, prec=1):
    from paper_2404_11631_gb300 import saa
    cp = gp.c_struct()
    X = torch.zeros(max(K, 1), gp.d, dtype=torch.float64, device="cuda")
    f = torch.zeros(max(K, 1), dtype=torch.float64, device="cuda")
    ws = torch.empty(1 << 22, dtype=torch.uint8, device="cuda")
    n = ws.numel() - ws_offset if ws_bytes is None else ws_bytes
    return saa.lib().saa_eval(saa.context(), C.byref(cp), K, C.c_void_p(X.data_ptr()), prec,
                              C.c_void_p(f.data_ptr()), None, None, C.c_void_p(ws.data_ptr() + ws_offset), n,
                              None)


def test_invalid_arguments_are_rejected():
    from paper_2404_11631_gb300 import saa
    gp, _, _ = make(4, 100)
    assert _call_eval(gp) == saa.SAA_OK
    torch.cuda.synchronize()
    bad = make(4, 1)[0]
    assert _call_eval(bad) == saa.SAA_EINVAL
    assert _call_eval(gp, K=0) == saa.SAA_EINVAL
    assert _call_eval(gp, ws_bytes=16) == saa.SAA_ENOMEM
    assert _call_eval(gp, ws_offset=8) == saa.SAA_EINVAL
    assert _call_eval(gp, prec=3) == saa.SAA_EUNSUPPORTED
    t_odd = make(4, 100, law=oracle.LAW_STUDENT_T, nu=3)[0]
    assert _call_eval(t_odd) == saa.SAA_EINVAL
    assert b"nu" in saa.lib().saa_last_error()


def test_too_large_dimension_is_unsupported():
    from paper_2404_11631_gb300 import saa
    gp, _, _ = make(saa.max_dim("fp32") + 1, 100)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_eval(gp, torch.zeros(1, gp.d, dtype=torch.float64, device="cuda"), "fp32")
    assert e.value.status == saa.SAA_EINVAL or e.value.status == saa.SAA_EUNSUPPORTED


def test_ctx_sync_reports_clean_state():
    from paper_2404_11631_gb300 import saa
    saa.saa_ctx_sync()


def test_bounded_wait_times_out_and_context_survives():
    # a wait on an mbarrier that nothing completes gives up after ~1 ms and
    # reports through the error word; no fault, and the context keeps working
    from paper_2404_11631_gb300 import saa
    saa.saa_selftest_timeout(1000)
    with pytest.raises(saa.SAAError) as e:
        saa.saa_ctx_sync()
    assert e.value.status == saa.SAA_ETIMEOUT
    saa.saa_ctx_sync()    # cleared
    gp, _, _ = make(8, 1000)
    out = saa.saa_eval(gp, torch.zeros(2, 8, dtype=torch.float64, device="cuda"), "f16x3")
    saa.saa_ctx_sync()
    assert torch.isfinite(out["f"]).all()
