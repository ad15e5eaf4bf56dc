"""Dictionary recovery (Section 4.1, Table 1) on the GPU.

Each row of the table is run as one batch per sparsity level: 4 SNR levels x
50 runs = 200 independent problems (p=20, n=50, m=1500), 9 s^2 iterations of
the full loop (OMP coding and the Jacobi atom update, ntilde = n) captured as
one CUDA graph per s^2 iterations.  The learned dictionaries are compared with
the generating ones by the recovery criterion of Section 4.1 and the means
against the paper's P-SGK and P-NSGK rows, with the tolerance of the oracle's
own Table 1 pin (4 percentage points, widened to 3 standard errors of the
50-run mean).  The seeds are the oracle pin's, so the two see the same
problems.
"""
import os

import numpy as np
import pytest

from paper_1509_05054_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SNRS = (10.0, 20.0, 30.0, None)
RUNS = 50
P, N, M = 20, 50, 1500


@pytest.fixture(scope="module")
def dl():
    from paper_1509_05054_gb300 import build as _b
    _b.build()
    from paper_1509_05054_gb300 import dl as _dl
    _dl.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return _dl


def _row(name, s):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            v = line.split()
            if v and not line.startswith("#") and int(v[0]) == s:
                return dict(zip(SNRS, map(float, v[1:])))
    raise KeyError(s)


def _recovered(D0, D):
    """Fraction of generating atoms d0 with some learned d at 1 - |d0^T d| < 0.01."""
    c = np.abs(D0 @ D.T)
    return float(np.mean((1.0 - c.max(axis=1)) < 0.01))


@pytest.mark.parametrize("s", [3, 4, 5])
def test_table1_recovery_on_the_gpu(dl, s):
    cells, dev = [], []
    for snr in SNRS:
        for r in range(RUNS):
            Y, D0, _, _ = synth.recovery_problem(P, N, M, s, snr, seed=10000 + 97 * r)
            Dinit = synth.dictionary_from_signals(Y, N, seed=20000 + r)
            cells.append((snr, D0, torch.from_numpy(Dinit.astype(np.float32))))
            dev.append(dict(p=P, n=N, s=s, m=M,
                            Y=torch.from_numpy(Y.astype(np.float32)).cuda(),
                            D=torch.from_numpy(Dinit.astype(np.float32)).cuda(),
                            colptr=torch.zeros(M + 1, dtype=torch.int64, device="cuda"),
                            rowidx=torch.zeros(M * s, dtype=torch.int32, device="cuda"),
                            val=torch.zeros(M * s, dtype=torch.float32, device="cuda")))
    st = torch.cuda.Stream()
    b = dl.dl_batch_create(dev, autotune=False, stream=st)
    try:
        for name, rule in (("table1_recovery_psgk.txt", dl.DL_RULE_SGK),
                           ("table1_recovery_pnsgk.txt", dl.DL_RULE_NSGK)):
            for (_, _, Dinit), d in zip(cells, dev):
                d["D"].copy_(Dinit)
            torch.cuda.synchronize()
            dl.dl_batch_set_update_rule(b, rule)
            rm = np.zeros(len(dev) * 2 * s * s)
            for _ in range(9):
                dl.dl_batch_iterate(b, s * s, rm)
            assert np.all(np.isfinite(rm))
            table = _row(name, s)
            for snr in SNRS:
                res = [_recovered(D0, d["D"].cpu().numpy().astype(np.float64))
                       for (c_snr, D0, _), d in zip(cells, dev) if c_snr == snr]
                assert len(res) == RUNS
                mean = 100.0 * np.mean(res)
                se = 100.0 * np.std(res) / np.sqrt(RUNS)
                tol = max(4.0, 3.0 * se)
                assert abs(mean - table[snr]) <= tol, (name, s, snr, mean, table[snr], tol)
                norms = [np.linalg.norm(d["D"].cpu().numpy(), axis=1)
                         for (c_snr, _, _), d in zip(cells, dev) if c_snr == snr]
                np.testing.assert_allclose(np.concatenate(norms), 1.0, atol=1e-4)
    finally:
        dl.dl_batch_destroy(b)


def test_batch_rule_and_group_setters_check_arguments(dl):
    Y, _, _, _ = synth.recovery_problem(P, N, 512, 3, 30.0, seed=5)
    Dinit = synth.dictionary_from_signals(Y, N, seed=6)
    q = dict(p=P, n=N, s=3, m=512, Y=torch.from_numpy(Y.astype(np.float32)).cuda(),
             D=torch.from_numpy(Dinit.astype(np.float32)).cuda(),
             colptr=torch.zeros(513, dtype=torch.int64, device="cuda"),
             rowidx=torch.zeros(512 * 3, dtype=torch.int32, device="cuda"),
             val=torch.zeros(512 * 3, dtype=torch.float32, device="cuda"))
    st = torch.cuda.Stream()
    b = dl.dl_batch_create([q], autotune=False, stream=st)
    try:
        with pytest.raises(dl.DLError):
            dl.dl_batch_set_update_rule(b, 7)
        with pytest.raises(dl.DLError):
            dl.dl_batch_set_group_size(b, N + 1)
        with pytest.raises(dl.DLError):
            dl.dl_batch_set_group_size(b, 0)
        dl.dl_batch_set_group_size(b, 16)
        dl.dl_batch_set_update_rule(b, dl.DL_RULE_NSGK)
        rm = np.zeros(2 * 2)
        dl.dl_batch_iterate(b, 2, rm)
        assert np.all(np.isfinite(rm))
        cnt = np.diff(q["colptr"].cpu().numpy())
        assert cnt.min() >= 1 and cnt.max() <= 3
    finally:
        dl.dl_batch_destroy(b)
