"""Failure detection on the GPU without a fault: the bounded mbarrier wait of
the tensor-core kernels is made to run out (a barrier nothing completes), the
kernel flags the timeout and returns, the host reads DL_ETIMEOUT, and the same
context then computes correct results again."""
import time

import numpy as np
import pytest

import oracle
from paper_1509_05054_gb300 import synth

from _common import assert_support_parity, csc_to_slots

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


def test_bounded_wait_times_out_and_context_stays_usable(dl):
    Y, D, spec = synth.workload_inputs("tiny")
    m, p, n, s = spec["m"], spec["p"], spec["n"], spec["s"]
    ctx = dl.dl_init(p, n, m, s, dl.DL_FP32, torch.cuda.current_stream())
    t0 = time.perf_counter()
    status = dl.dl_check_bounded_wait(ctx)
    waited = time.perf_counter() - t0
    assert status == dl.DL_ETIMEOUT, dl.dl_strerror(status)
    assert 1.5 < waited < 60.0, waited
    # the error word was read and cleared: the context codes correctly again
    cp = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
    ri = torch.zeros(m * s, dtype=torch.int32, device="cuda")
    v = torch.zeros(m * s, dtype=torch.float32, device="cuda")
    dl.omp_code(ctx, torch.from_numpy(Y).cuda(), m, torch.from_numpy(D.copy()).cuda(), s, cp, ri, v)
    dl.dl_sync(ctx)
    dl.dl_destroy(ctx)
    idx_g, _, cnt_g = csc_to_slots(cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), s)
    idx_o, _, cnt_o, gaps = oracle.omp(Y.astype(np.float64), D.astype(np.float64), s,
                                       return_gaps=True)
    assert_support_parity(idx_g, cnt_g, idx_o, cnt_o, gaps)
