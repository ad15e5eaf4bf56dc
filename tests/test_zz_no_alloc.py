"""The allocation-free correlation entry point.

dl_correlate_noalloc serves callers that cannot call cudaMalloc (their device
memory is reserved by another allocator, or they cannot accept an allocation's
implicit synchronisation); its scratch is a fixed device array inside the
library.  The tests compare it with the FP64 product and with the regular
entry point, on both of its paths (tcgen05 split-TF32 and the CUDA-core GEMM),
check that a call leaves the device's free memory unchanged, and read the
device-side status with dl_correlate_noalloc_status.

This file is collected last so that a failure here comes after every other
test has run; it also passes on its own in a fresh process.
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


def _fp64_error(A, Yn, Dn):
    """max |A - Y D^T| / (||y_i|| ||d_j||), the product taken in FP64."""
    Y64, D64 = Yn.astype(np.float64), Dn.astype(np.float64)
    exact = Y64 @ D64.T
    scale = np.linalg.norm(Y64, axis=1)[:, None] * np.linalg.norm(D64, axis=1)[None, :]
    return float(np.max(np.abs(A.cpu().numpy().astype(np.float64) - exact) / scale))


def _random_inputs(m, p, n, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((m, p)).astype(np.float32)
    D = rng.standard_normal((n, p))
    D = (D / np.linalg.norm(D, axis=1, keepdims=True)).astype(np.float32)
    return Y, D


def test_noalloc_correlations_match_fp64_and_regular_entry_point_twice(dl):
    """Two calls in a row with different dictionaries (the second call must not
    depend on what the first left in the shared scratch): each within 1e-5 of
    the FP64 product and of dl_correlate, and a clean device-side status."""
    stream = torch.cuda.current_stream()
    for k, (name, m) in enumerate([("patch_n512", 3001), ("patch_n256", 2000)]):
        Yn, Dn, _ = synth.workload_inputs(name, m=m)
        Y, D = torch.from_numpy(Yn).cuda(), torch.from_numpy(Dn).cuda()
        p, n = Dn.shape[1], Dn.shape[0]
        A = torch.full((m, n), float("nan"), device="cuda")
        dl.dl_correlate_noalloc(Y, m, D, p, n, A, stream)
        assert dl.dl_correlate_noalloc_status(stream) == dl.DL_OK
        assert _fp64_error(A, Yn, Dn) < 1e-5, k
        ref = _regular(dl, Y, D, m)
        assert _fp64_error(ref, Yn, Dn) < 1e-5, k
        scale = (np.linalg.norm(Yn.astype(np.float64), axis=1)[:, None] *
                 np.linalg.norm(Dn.astype(np.float64), axis=1)[None, :])
        err = np.max(np.abs(A.cpu().numpy() - ref.cpu().numpy()) / scale)
        assert err < 1e-5, (k, err)


def test_noalloc_cuda_core_path_matches_fp64(dl):
    """Shapes and views the tensor-core kernel does not take (p not a multiple
    of 4, n not a multiple of 16, an output A off a 16-byte boundary) go to the
    CUDA-core GEMM, which needs no scratch: still within 1e-5 of FP64."""
    stream = torch.cuda.current_stream()
    for (m, p, n, offset, seed) in [(517, 36, 37, 0, 1), (300, 64, 50, 0, 2), (257, 64, 512, 1, 3)]:
        Yn, Dn = _random_inputs(m, p, n, seed)
        Y, D = torch.from_numpy(Yn).cuda(), torch.from_numpy(Dn).cuda()
        buf = torch.full((m * n + offset,), float("nan"), device="cuda")
        A = buf[offset:].view(m, n)  # offset 1: a view 4 bytes past a 16-byte boundary
        dl.dl_correlate_noalloc(Y, m, D, p, n, A.data_ptr(), stream)
        assert dl.dl_correlate_noalloc_status(stream) == dl.DL_OK
        assert _fp64_error(A, Yn, Dn) < 1e-5, (m, p, n, offset)


def test_noalloc_leaves_free_device_memory_unchanged(dl):
    """After one warm-up call per path (which loads the kernels' code), further
    calls take no device memory: cudaMemGetInfo's free bytes stay the same."""
    stream = torch.cuda.current_stream()
    cases = []
    for (m, p, n, seed) in [(4096, 64, 512, 4), (1000, 36, 37, 5)]:
        Yn, Dn = _random_inputs(m, p, n, seed)
        Y, D = torch.from_numpy(Yn).cuda(), torch.from_numpy(Dn).cuda()
        A = torch.empty(m, n, device="cuda")
        cases.append((Y, D, A, m, p, n))
    for (Y, D, A, m, p, n) in cases:  # warm-up
        dl.dl_correlate_noalloc(Y, m, D, p, n, A, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        for (Y, D, A, m, p, n) in cases:
            dl.dl_correlate_noalloc(Y, m, D, p, n, A, stream)
    assert dl.dl_correlate_noalloc_status(stream) == dl.DL_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch(dl):
    Y = torch.zeros(4, 64, device="cuda")
    D = torch.zeros(1024, 64, device="cuda")
    A = torch.zeros(4, 1024, device="cuda")
    with pytest.raises(dl.DLError) as e:
        dl.dl_correlate_noalloc(Y, 4, D, 64, 1024, A)
    assert e.value.status == dl.DL_EINVAL
