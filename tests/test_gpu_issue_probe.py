"""The measured issue rate (pdv_measure_issue_rate) that the transport
kernels' roofline is read against: positive, at most the nominal rate of the
device (SMs x 4 schedulers x 32 lanes x 2.07 GHz, the maximum SM clock of
this part) and well above half of it; invalid arguments are refused."""
import pytest

from paper_2012_00963_gb300 import pdv

pytestmark = pytest.mark.gpu


def test_issue_rate_is_close_to_nominal():
    torch = pytest.importorskip("torch")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 4 * 32 * 2.07e9
    with pdv.Context(0) as ctx:
        r = pdv.pdv_measure_issue_rate(ctx.handle, 0.1)
        with pytest.raises(pdv.PdvError) as e:
            pdv.pdv_measure_issue_rate(ctx.handle, 0.0)
        assert e.value.status == pdv.PDV_EINVAL
    assert 0.5 * nominal < r <= 1.02 * nominal, (r, nominal)
