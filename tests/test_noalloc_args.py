"""The Python binding of lb_fields_noalloc checks its tensors before calling
into the library: a tensor of the wrong shape, dtype, device or layout would
let the kernels read or write past a smaller buffer. These checks raise on
the CPU, before any launch."""

import pytest
import torch

from paper_1501_03857_gb300 import lb


CFG = lb.Config(Lx=8, Ly=6)


def _args(**over):
    a = {"fpost": torch.zeros(9, 6, 8), "theta": torch.zeros(6, 8)}
    a.update(over)
    return a


@pytest.mark.parametrize("over", [
    {"fpost": torch.zeros(9, 6, 7)},                      # too small
    {"theta": torch.zeros(6, 8, dtype=torch.float64)},    # wrong dtype
    {"theta": torch.zeros(8, 6).t()},                     # not contiguous
    {"rho": torch.zeros(5, 8)},                           # output too small
    {"fpost": None},                                      # missing input
])
def test_wrong_tensors_raise_before_the_call(over):
    a = _args(**over)
    with pytest.raises(ValueError):
        lb.fields_noalloc(CFG, 0.0, 3.0, a["fpost"], a["theta"], rho=a.get("rho"))


def test_host_tensors_raise_before_the_call():
    """Correct shapes on the host (not CUDA tensors) are refused too."""
    a = _args()
    with pytest.raises(ValueError, match="CUDA"):
        lb.fields_noalloc(CFG, 0.0, 3.0, a["fpost"], a["theta"])
