"""rtpn_sum_static: the FP64 sum that allocates nothing.

Some callers cannot call cudaMalloc at the point where they need a sum (their framework's memory
pool owns the device memory, or an allocation would synchronise a time-critical loop); this entry
point serves them from a fixed device array inside the library.  It is checked here, through the
C ABI, against the context's own sum (rtpn_sum_u0) of the same u_0, on two calls in a row.  This
file is collected last, and it passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_2004_02833_gb300 import rtpn, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_sum_static_matches_context_sum(cuda_device, precision):
    import torch

    shape = (100, 101, 102)  # ~1.03e6 values: many partials and a ragged last one
    u = synth.random_state(1, shape, 11)
    u[0] += 0.25  # keep the sum away from zero
    dtype = torch.float32 if precision == "fp32" else torch.float64
    with rtpn.Context(1, shape, 0.5, "periodic", precision) as ctx:
        ctx.set_moments(u)
        want = ctx.sum_u0()
        field = torch.empty(shape, dtype=dtype, device="cuda")
        ctx.get_component(0, field)
        ctx.synchronize()
    scale = float(field.abs().sum())
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for i in range(2):  # two calls in a row share the static scratch
        rtpn.sum_static(field, out[i:i + 1])
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-12 * scale), (got, want)


def test_sum_static_limits(cuda_device):
    import torch

    x = torch.ones(4, dtype=torch.float32, device="cuda")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    # beyond the 2^30-value capacity of the static scratch: rejected on the host, nothing launched
    rc = rtpn.lib().rtpn_sum_static(rtpn._P(x.data_ptr()), rtpn.DTYPE_F32, (1 << 30) + 1,
                                    rtpn._P(out.data_ptr()), rtpn._P(0))
    assert rc == rtpn.EINVAL
    assert "2^30" in rtpn.lib().rtpn_last_error(None).decode()
    rtpn.sum_static(x[:0], out)
    torch.cuda.synchronize()
    assert float(out[0]) == 0.0
    rtpn.sum_static(x, out)
    torch.cuda.synchronize()
    assert float(out[0]) == 4.0
