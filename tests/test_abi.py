"""CPU checks of the C-ABI library: it loads, exports every symbol declared in include/*.h, and
its host-side coefficient generator and placement agree with the oracle's quadrature (no GPU)."""
import glob
import os
import re

import numpy as np
import pytest

from oracle import sh
from paper_2004_02833_gb300 import rtpn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(rtpn_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(rtpn_lib):
    names = declared_symbols()
    assert len(names) >= 20
    for name in sorted(names):
        assert hasattr(rtpn_lib, name), name
        assert name in rtpn.SIGNATURES, f"binding lacks {name}"


def test_strerror_and_version(rtpn_lib):
    assert rtpn_lib.rtpn_version() >= 100
    assert rtpn_lib.rtpn_strerror(rtpn.ECFL).decode().startswith("time step")


@pytest.mark.parametrize("N", [0, 1, 3, 7, 15, 39])
def test_closed_form_coupling_matches_quadrature(rtpn_lib, coupling_cache, N):
    # the library's ladder closed forms vs the oracle's spherical quadrature (Eq. 3)
    (mats, slots) = coupling_cache(N)
    for axis in range(3):
        got = rtpn.coupling_dense(N, axis)
        assert np.array_equal(got != 0, mats[axis] != 0), axis
        assert np.abs(got - mats[axis]).max() < 2e-13


@pytest.mark.parametrize("N", [1, 3, 7, 39])
def test_component_info_matches_placement(rtpn_lib, coupling_cache, N):
    (mats, slots) = coupling_cache(N)
    comps = sh.components(N)
    for c in range(len(comps)):
        l, m, sl, cls = rtpn.component_info(N, c)
        assert (l, m) == comps[c]
        assert sl == tuple(slots[c])
        assert cls == sh.parity_class(slots[c:c + 1])[0]


def test_bad_arguments_rejected(rtpn_lib):
    with pytest.raises(rtpn.RtpnError) as e:
        rtpn.component_info(3, 16)
    assert e.value.code == rtpn.EINVAL
    with pytest.raises(rtpn.RtpnError):
        rtpn.coupling_dense(-1, 0)


def test_create_validates_before_touching_the_device(rtpn_lib):
    # argument and CFL checks come first, so they hold on a machine without a GPU as well
    with pytest.raises(rtpn.RtpnError) as e:
        rtpn.Context(3, (4, 4, 4), 0.1, dt=0.04)
    assert e.value.code == rtpn.ECFL
    with pytest.raises(rtpn.RtpnError) as e:
        rtpn.Context(-1, (4, 4, 4), 0.1)
    assert e.value.code == rtpn.EINVAL
    with pytest.raises(rtpn.RtpnError) as e:
        rtpn.Context(3, (0, 4, 4), 0.1)
    assert e.value.code == rtpn.EINVAL


def test_new_entry_points_reject_a_null_context(rtpn_lib):
    # no GPU needed: argument checks come before any device call
    assert rtpn_lib.rtpn_set_spacing(None, 0.1, 0.1, 0.1) == rtpn.EINVAL
    assert rtpn_lib.rtpn_set_scattering(None, None, 0) == rtpn.EINVAL


def test_sum_static_refuses_other_dtypes_before_any_launch(rtpn_lib):
    # the kernel reads numel() values of 4 or 8 bytes: a bf16 / f16 / integer tensor, or an empty
    # output, is refused by the binding before the library is called (CPU tensors suffice here)
    import torch

    out = torch.zeros(1, dtype=torch.float64)
    for dt in (torch.bfloat16, torch.float16, torch.int32, torch.int64):
        with pytest.raises(TypeError):
            rtpn.sum_static(torch.zeros(8, dtype=dt), out)
    with pytest.raises(ValueError):
        rtpn.sum_static(torch.zeros(8, dtype=torch.float32), torch.zeros(0, dtype=torch.float64))
    with pytest.raises(ValueError):
        rtpn.sum_static(torch.zeros(8, dtype=torch.float32), torch.zeros(1, dtype=torch.float32))


def test_autograd_form_refuses_host_tensors():
    # the autograd wrapper hands device pointers to the library: host tensors are refused before
    # any call reaches it
    import torch

    from paper_2004_02833_gb300.autograd import detector_response

    t = torch.zeros((2, 2, 2), dtype=torch.float64, requires_grad=True)
    with pytest.raises(TypeError):
        detector_response(None, t, t, t, torch.zeros((4, 2, 2, 2), dtype=torch.float64), t.detach(), 1)
