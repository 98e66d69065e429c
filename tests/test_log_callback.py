"""The optional log sink (pifepic_set_log_callback): every error message the
library records also reaches the callback.  Checked without a GPU, where
context creation fails at its first device call with ECUDA and a message."""
import pytest


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="context creation succeeds on a GPU machine")
def test_errors_reach_the_log_callback_and_stop_when_it_is_removed():
    from paper_2011_10214_gb300 import capi
    msgs = []
    capi.set_log_callback(msgs.append)
    try:
        with pytest.raises(capi.PifepicError) as err:
            capi.Simulation((4, 4, 4), 0.5, 0.05)
    finally:
        capi.set_log_callback(None)
    assert len(msgs) == 1 and msgs[0] and msgs[0] in str(err.value)
    with pytest.raises(capi.PifepicError):
        capi.Simulation((4, 4, 4), 0.5, 0.05)
    assert len(msgs) == 1
