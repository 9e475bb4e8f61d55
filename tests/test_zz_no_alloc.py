"""The allocation-free polarization readout, spinrp_polarization_noalloc.

It is for callers that cannot allocate device memory: code running inside a
host application that owns every device allocation, or a loop in which an
allocation would synchronize the device.  The call reduces N_up / N_dn of a
device state the caller owns into a device buffer the caller passes in, using
only a fixed scratch array compiled into the library.

Here it is called through the C ABI on the amplitude buffer of a library
state, and its (P, norm) is compared with what the existing path records for
the same state (the series spinrp_evolve writes after every step), within the
tolerances of the parity tests, on two calls in a row (evolving in between).
This file is collected last so that a failure here leaves every other test
already run.
"""
import numpy as np
import pytest

from paper_0710_3747_gb300 import spinrp
from paper_0710_3747_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-4}  # |dP| bars of the parity tests


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_noalloc_matches_recorded_series(prec):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "needs a CUDA device"
    sysm = spinrp.System(W.star_dipolar(14, 3), spinrp.DIPOLAR)
    st = spinrp.State(sysm, prec, series_cap=32)
    st.init_random_phase(5)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        st.evolve(0.02, 7)
        spinrp.polarization_noalloc(st.device_ptr(), st.M, prec, 1, st.layout(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        P, N = out.tolist()
        assert abs(P - st.polarization()[-1]) <= TOL[prec], (call, P)
        assert abs(N - st.norm_series()[-1]) <= TOL[prec], (call, N)
        assert abs(P) < 1.0


def test_noalloc_rejects_oversized_requests():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "needs a CUDA device"
    psi = torch.zeros(2 << 10, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(spinrp.SpinrpError) as e:
        spinrp.polarization_noalloc(psi.data_ptr(), 10, "c64", 1, None, out.data_ptr(), blocks=1217)
    assert e.value.code == spinrp.EINVAL and "1216" in str(e.value)
    with pytest.raises(spinrp.SpinrpError) as e:
        spinrp.polarization_noalloc(psi.data_ptr(), 35, "c64", 1, None, out.data_ptr())
    assert e.value.code == spinrp.EINVAL
