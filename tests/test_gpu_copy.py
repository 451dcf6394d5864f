"""crk_copy (the SM-driven staging copy) against torch's copies: device to
device, page-locked host to device and back, unaligned heads and tails,
pointers of different alignment, and refusals that launch nothing (pageable
host memory, overlapping ranges)."""
import pytest
import torch

from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300.solver import copy_

pytestmark = pytest.mark.gpu


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("nbytes", [1, 15, 63, 64, 1000, (1 << 20) + 3, (64 << 20) + 17])
@pytest.mark.parametrize("offs", [(0, 0), (3, 3), (5, 9)])
def test_copy_matches_torch(nbytes, offs):
    g = torch.Generator().manual_seed(nbytes)
    src_h = torch.randint(0, 256, (nbytes + 32,), dtype=torch.uint8, generator=g).pin_memory()
    dev = torch.zeros(nbytes + 32, dtype=torch.uint8, device="cuda")
    back = torch.zeros(nbytes + 32, dtype=torch.uint8).pin_memory()
    dev2 = torch.zeros(nbytes + 32, dtype=torch.uint8, device="cuda")
    a, b = offs
    L.crk_copy(_stream(), dev.data_ptr() + b, src_h.data_ptr() + a, nbytes)       # host -> device
    L.crk_copy(_stream(), dev2.data_ptr() + a, dev.data_ptr() + b, nbytes)        # device -> device
    L.crk_copy(_stream(), back.data_ptr() + b, dev2.data_ptr() + a, nbytes)       # device -> host
    torch.cuda.synchronize()
    want = src_h[a:a + nbytes]
    assert torch.equal(dev[b:b + nbytes].cpu(), want)
    assert torch.equal(back[b:b + nbytes], want)
    # nothing outside the ranges was written
    assert int(dev[:b].sum()) == 0 and int(dev[b + nbytes:].sum()) == 0
    assert int(back[:b].sum()) == 0 and int(back[b + nbytes:].sum()) == 0


def test_tensor_helper_and_refusals():
    x = torch.randn(3, 1000, dtype=torch.float64).pin_memory()
    d = torch.empty_like(x, device="cuda")
    copy_(d, x)
    torch.cuda.synchronize()
    assert torch.equal(d.cpu(), x)
    pageable = torch.zeros(4096, dtype=torch.uint8)
    dd = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.CRKError):
        L.crk_copy(_stream(), dd.data_ptr(), pageable.data_ptr(), 4096)
    with pytest.raises(L.CRKError):
        L.crk_copy(_stream(), dd.data_ptr() + 16, dd.data_ptr(), 64)  # overlap
    with pytest.raises(ValueError):
        copy_(d, x.float())
    torch.cuda.synchronize()
