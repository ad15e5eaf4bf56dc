"""Batched uneven problems (one CUDA graph launch for all problems and
iterations) against the FP64 oracle and against per-problem dl_iterate.

Shapes follow the batched workload (p in {36, 64, 100}, n in {128..1024},
s in 4..12) with m scaled by 0.1 so the oracle finishes in seconds; these
shapes exercise the CUDA-core correlation path (p = 100, n = 1024), the
shared-memory u-vector OMP kernel (large n*s) and the global-atomic error
accumulation (n*p*4 > 200 KB).
"""
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


def _device_problems(probs):
    out = []
    for q in probs:
        m, s = q["m"], q["s"]
        out.append(dict(p=q["p"], n=q["n"], s=s, m=m, Y=torch.from_numpy(q["Y"]).cuda(),
                        D=torch.from_numpy(q["D"].copy()).cuda(),
                        colptr=torch.zeros(m + 1, dtype=torch.int64, device="cuda"),
                        rowidx=torch.zeros(m * s, dtype=torch.int32, device="cuda"),
                        val=torch.zeros(m * s, dtype=torch.float32, device="cuda")))
    return out


@pytest.fixture(scope="module")
def problems():
    return synth.batched_problems(16, m_scale=0.1)


def test_batched_first_iteration_matches_oracle(dl, problems):
    dev = _device_problems(problems)
    st = torch.cuda.Stream()
    b = dl.dl_batch_create(dev, autotune=False, stream=st)
    rm = np.zeros(len(dev) * 2)
    dl.dl_batch_iterate(b, 1, rm)
    dl.dl_batch_destroy(b)
    rm = rm.reshape(len(dev), 2)
    for k, (q, d) in enumerate(zip(problems, dev)):
        Y64, D64 = q["Y"].astype(np.float64), q["D"].astype(np.float64)
        idx_o, val_o, cnt_o, gaps = oracle.omp(Y64, D64, q["s"], return_gaps=True)
        r_omp = oracle.rmse(Y64, D64, idx_o, val_o, cnt_o)
        D1, v1, _ = oracle.jau(Y64, D64, idx_o, val_o, cnt_o)
        r_jau = oracle.rmse(Y64, D1, idx_o, v1, cnt_o)
        assert abs(rm[k, 0] - r_omp) <= 1e-4, (k, q["p"], q["n"], q["s"], rm[k], r_omp)
        assert abs(rm[k, 1] - r_jau) <= 1e-4, (k, q["p"], q["n"], q["s"], rm[k], r_jau)
        idx_g, _, cnt_g = csc_to_slots(d["colptr"].cpu().numpy(), d["rowidx"].cpu().numpy(),
                                       d["val"].cpu().numpy(), q["s"])
        assert_support_parity(idx_g, cnt_g, idx_o, cnt_o, gaps)


def test_batched_equals_per_problem_iterations_and_autotune_keeps_results(dl, problems):
    iters = 5
    sub = problems[:6]
    st = torch.cuda.Stream()
    ref = []
    for q in sub:
        d = _device_problems([q])[0]
        ctx = dl.dl_init(q["p"], q["n"], q["m"], q["s"], dl.DL_FP32, st)
        r = np.zeros(2 * iters)
        dl.dl_iterate(ctx, d["Y"], q["m"], d["D"], q["s"], iters, d["colptr"], d["rowidx"], d["val"], r)
        dl.dl_destroy(ctx)
        ref.append(r)
    for tune in (False, True):
        dev = _device_problems(sub)
        b = dl.dl_batch_create(dev, autotune=tune, stream=st)
        rm = np.zeros(len(dev) * 2 * iters)
        dl.dl_batch_iterate(b, iters, rm)
        cfgs = [dl.dl_batch_config(b, k) for k in range(len(dev))]
        launches = dl.dl_batch_kernel_launches(b)
        dl.dl_batch_destroy(b)
        rm = rm.reshape(len(dev), 2 * iters)
        for k in range(len(dev)):
            np.testing.assert_allclose(rm[k], ref[k], rtol=0, atol=2e-5)
        for c in cfgs:
            assert c["omp_warps"] in (1, 2, 4) and c["rows_per_sm"] in (2, 4, 8)
        assert launches > 0
