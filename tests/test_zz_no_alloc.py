"""cl_scan_noalloc: the offset scan for callers that cannot allocate device
memory (a real-time loop that cannot take cudaMalloc's device
synchronisation, a plug-in whose host owns all device memory).  Its result
must equal cl_scan's, exactly (integer output), on two calls in a row --
the second call reuses the library's fixed scratch array left over from the
first.  Collected last so that a failure here cannot hide other tests."""
import numpy as np
import pytest
import torch

from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu


def test_noalloc_scan_equals_cl_scan_on_two_calls():
    P = lib()
    from paper_1406_1215_gb300.generator import Generator

    w = inputs.powerlaw_degrees(3_000_000, 2.3, 2, 5000, 31)  # ~1500 scan tiles, ragged last tile
    g = Generator(cuda(w), 17)
    g.count()
    g.scan(True)
    torch.cuda.synchronize()
    ref = g.offsets.clone()
    n = g.n_items
    out = torch.empty_like(ref)
    for _ in range(2):
        out.fill_(-1)
        P.cl_scan_noalloc(g.counts, n, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    # a shorter input afterwards still matches (no stale partials are read)
    k = 4097
    out2 = torch.full((k + 1,), -1, dtype=torch.int64, device="cuda")
    P.cl_scan_noalloc(g.counts[:k], k, out2)
    torch.cuda.synchronize()
    c = g.counts[:k].cpu().numpy().astype(np.int64)
    assert np.array_equal(out2.cpu().numpy(), np.concatenate([[0], np.cumsum(c)]))
    g.close()


def test_noalloc_scan_rejects_oversize_without_touching_output():
    P = lib()
    out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    counts = torch.zeros(3, dtype=torch.int32, device="cuda")
    # raw addresses go straight to the C entry point, which refuses the size
    with pytest.raises(P.ClError) as ei:
        P.cl_scan_noalloc(counts.data_ptr(), (1 << 28) + 1, out.data_ptr())
    assert ei.value.status == 4  # CL_ERR_RANGE
    # tensors are checked by the binding before the call: too short, wrong dtype
    with pytest.raises(ValueError):
        P.cl_scan_noalloc(counts, 3, out[:3])
    with pytest.raises(ValueError):
        P.cl_scan_noalloc(counts.to(torch.int64), 3, out)
    torch.cuda.synchronize()
    assert bool((out == -1).all())
