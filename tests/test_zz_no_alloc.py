"""The allocation-free correlation entry point against the regular one.

dl_correlate_noalloc serves callers that cannot call cudaMalloc (their device
memory is reserved by another allocator, or they cannot accept an allocation's
implicit synchronisation); its scratch is a fixed device array inside the
library.  This file is collected last so that a failure here comes after every
other test has run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1509_05054_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dl():
    from paper_1509_05054_gb300 import build as _b
    _b.build()
    from paper_1509_05054_gb300 import dl as _dl
    _dl.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return _dl


def _regular(dl, Y, D, m):
    p, n = D.shape[1], D.shape[0]
    ctx = dl.dl_init(p, n, m, 1, dl.DL_FP32, torch.cuda.current_stream())
    A = torch.zeros(m, n, device="cuda")
    dl.dl_correlate(ctx, Y, m, D, A)
    dl.dl_sync(ctx)
    dl.dl_destroy(ctx)
    return A


def test_noalloc_correlations_match_regular_entry_point_twice(dl):
    """Two calls in a row (different dictionaries, so the second call must not
    depend on what the first left in the shared scratch)."""
    stream = torch.cuda.current_stream()
    for k, (name, m) in enumerate([("patch_n512", 3001), ("patch_n256", 2000)]):
        Yn, Dn, _ = synth.workload_inputs(name, m=m)
        Y, D = torch.from_numpy(Yn).cuda(), torch.from_numpy(Dn).cuda()
        p, n = Dn.shape[1], Dn.shape[0]
        A = torch.full((m, n), float("nan"), device="cuda")
        dl.dl_correlate_noalloc(Y, m, D, p, n, A, stream)
        torch.cuda.synchronize()
        ref = _regular(dl, Y, D, m)
        scale = (np.linalg.norm(Yn.astype(np.float64), axis=1)[:, None] *
                 np.linalg.norm(Dn.astype(np.float64), axis=1)[None, :])
        err = np.max(np.abs(A.cpu().numpy() - ref.cpu().numpy()) / scale)
        assert err < 1e-5, (k, err)


def test_noalloc_rejects_sizes_beyond_its_scratch(dl):
    Y = torch.zeros(4, 64, device="cuda")
    D = torch.zeros(1024, 64, device="cuda")
    A = torch.zeros(4, 1024, device="cuda")
    with pytest.raises(dl.DLError) as e:
        dl.dl_correlate_noalloc(Y, 4, D, 64, 1024, A)
    assert e.value.status == dl.DL_EINVAL
