"""The allocation-free polarization readout, spinrp_polarization_noalloc.

It is for callers that cannot allocate device memory: code running inside a
host application that owns every device allocation, or a loop in which an
allocation would synchronize the device.  The call reduces N_up / N_dn of a
device state the caller owns into a device buffer the caller passes in, using
only a fixed scratch array compiled into the library.

Here it is called through the C ABI on the amplitude buffer of a library
state, and its (P, norm) is compared with what the existing path records for
the same state (the series spinrp_evolve writes after every step), within the
tolerances of the parity tests, on two calls in a row (evolving in between);
on a plain device buffer the caller fills with an oracle state (identity bit
order, layout NULL), against the oracle's own P and norm; and across a second
call the device memory in use is checked to stay the same.  This file is
collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_noalloc_on_caller_buffer_matches_oracle(prec):
    """A caller-owned buffer holding an oracle state in identity bit order
    (layout NULL): P of two different spins, two calls in a row, against the
    oracle's FP64 populations of the same amplitudes."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "needs a CUDA device"
    J = W.star_dipolar(13, 8)
    _, _, psi = oracle.run(J, oracle.DIPOLAR, 11, 0.02, 9)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    buf = torch.from_numpy(psi).to(dtype=dt, device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for site in (1, 6):
        spinrp.polarization_noalloc(buf.data_ptr(), 13, prec, site, None, out.data_ptr(), stream)
        torch.cuda.synchronize()
        P, N = out.tolist()
        ref = psi.astype(np.complex64).astype(np.complex128) if prec == "c64" else psi
        assert abs(P - oracle.polarization(ref, site)) <= TOL[prec], (site, P)
        assert abs(N - float(np.vdot(ref, ref).real)) <= TOL[prec], (site, N)


def test_noalloc_allocates_no_device_memory():
    """After one warm-up call (which may load the library's device code), a
    second call leaves the device memory in use unchanged."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "needs a CUDA device"
    psi = torch.randn(2 << 16, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    spinrp.polarization_noalloc(psi.data_ptr(), 16, "c64", 3, None, out.data_ptr(), stream)
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    spinrp.polarization_noalloc(psi.data_ptr(), 16, "c64", 3, None, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
