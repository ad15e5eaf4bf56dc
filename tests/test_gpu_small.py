"""Small problems in one launch (one CTA per problem runs every DL iteration)
against the FP64 oracle.

dl_batch takes this path when every problem has p <= 32, n <= 64, s <= 8 and
the group size is n (the dictionary-recovery experiment of Section 4.1 is
such a batch).  The shapes below span the limits: p from 1 to 32, n from 1 to
64 (n < 32 and 32 < n < 64 leave lanes of the second correlation register
empty), m from 1 to 2500 (the CSC scan runs in chunks of 1024 signals), s up
to 8, and a zero signal.  Per rule (AK-SVD, SGK, P-NSGK): the first
iteration's supports follow the oracle's OMP up to near-ties, its values and
atoms agree within FP32 accumulation error, and the RMSE trajectory over three
iterations follows the oracle's Algorithm 1.
"""
import numpy as np
import pytest

import oracle
from paper_1509_05054_gb300 import synth

from _common import assert_support_parity, csc_to_slots

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (p, n, m, s): recovery-shaped problems and the corners of the small path
SHAPES = [(20, 50, 1500, 3), (20, 50, 1500, 5), (32, 64, 2500, 8), (32, 64, 1024, 4),
          (16, 40, 777, 2), (24, 33, 1025, 6), (8, 16, 300, 3), (12, 31, 1, 2),
          (5, 7, 64, 1), (1, 1, 10, 1), (20, 64, 2049, 5), (32, 20, 500, 8)]


@pytest.fixture(scope="module")
def dl():
    from paper_1509_05054_gb300 import build as _b
    _b.build()
    from paper_1509_05054_gb300 import dl as _dl
    _dl.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return _dl


def _problems(seed0=0):
    out = []
    for k, (p, n, m, s) in enumerate(SHAPES):
        if p >= 4 and n >= 2 * s:
            Y, _, _, _ = synth.recovery_problem(p, n, m, s, 30.0, seed=seed0 + 31 * k)
        else:  # too small for a recovery instance: Gaussian signals
            Y = np.random.default_rng(seed0 + 31 * k).standard_normal((m, p))
        Y = Y.astype(np.float32)
        if m >= n:
            D = synth.dictionary_from_signals(Y.astype(np.float64), n, seed=seed0 + 31 * k + 1)
        else:  # fewer signals than atoms: random unit atoms
            D = np.random.default_rng(seed0 + 31 * k + 1).standard_normal((n, p))
            D /= np.linalg.norm(D, axis=1, keepdims=True)
        if m >= 8:
            Y[m // 2] = 0.0  # a zero signal: empty support
        out.append(dict(p=p, n=n, m=m, s=s, Y=Y, D=D.astype(np.float32)))
    return out


def _device(probs):
    return [dict(p=q["p"], n=q["n"], s=q["s"], m=q["m"], Y=torch.from_numpy(q["Y"]).cuda(),
                 D=torch.from_numpy(q["D"].copy()).cuda(),
                 colptr=torch.zeros(q["m"] + 1, dtype=torch.int64, device="cuda"),
                 rowidx=torch.zeros(q["m"] * q["s"], dtype=torch.int32, device="cuda"),
                 val=torch.zeros(q["m"] * q["s"], dtype=torch.float32, device="cuda"))
            for q in probs]


def _check_csc(d, q):
    colptr = d["colptr"].cpu().numpy()
    cnt = np.diff(colptr)
    assert colptr[0] == 0 and np.all(cnt >= 0) and np.all(cnt <= q["s"])
    idx, val, cnt = csc_to_slots(colptr, d["rowidx"].cpu().numpy(), d["val"].cpu().numpy(), q["s"])
    for i in range(q["m"]):
        row = idx[i, :cnt[i]]
        assert np.all(np.diff(row) > 0) and (len(row) == 0 or (row[0] >= 0 and row[-1] < q["n"]))
    return idx, val, cnt


@pytest.mark.parametrize("rule", ["AKSVD", "SGK", "NSGK"])
def test_small_batch_matches_oracle(dl, rule):
    rid = {"AKSVD": dl.DL_RULE_AKSVD, "SGK": dl.DL_RULE_SGK, "NSGK": dl.DL_RULE_NSGK}[rule]
    probs = _problems()
    dev = _device(probs)
    st = torch.cuda.Stream()
    b = dl.dl_batch_create(dev, autotune=False, stream=st)
    try:
        dl.dl_batch_set_update_rule(b, rid)
        for d, q in zip(dev, probs):
            d["D"].copy_(torch.from_numpy(q["D"]))
        torch.cuda.synchronize()
        l0 = dl.dl_batch_kernel_launches(b)
        rm1 = np.zeros(len(dev) * 2)
        dl.dl_batch_iterate(b, 1, rm1)
        assert dl.dl_batch_kernel_launches(b) - l0 == 1  # one launch for all problems
        rm1 = rm1.reshape(len(dev), 2)
        first = []
        for k, (q, d) in enumerate(zip(probs, dev)):
            Y64, D64 = q["Y"].astype(np.float64), q["D"].astype(np.float64)
            idx_o, val_o, cnt_o, gaps = oracle.omp(Y64, D64, q["s"], return_gaps=True)
            r_omp = oracle.rmse(Y64, D64, idx_o, val_o, cnt_o)
            orule = oracle.RULE_AKSVD if rule == "AKSVD" else oracle.RULE_SGK  # P-NSGK's first = SGK
            D1, v1, _ = oracle.atom_update(Y64, D64, idx_o, val_o, cnt_o, rule=orule)
            r_end = oracle.rmse(Y64, D1, idx_o, v1, cnt_o)
            assert abs(rm1[k, 0] - r_omp) <= 1e-4, (k, SHAPES[k], rm1[k], r_omp)
            assert abs(rm1[k, 1] - r_end) <= 1e-4, (k, SHAPES[k], rm1[k], r_end)
            idx_g, val_g, cnt_g = _check_csc(d, q)
            same = assert_support_parity(idx_g, cnt_g, idx_o, cnt_o, gaps)
            np.testing.assert_allclose(val_g[same], v1[same], rtol=1e-3, atol=1e-4)
            # atoms that no differing signal uses in either support
            touched = np.zeros(q["n"], bool)
            for i in np.nonzero(~same)[0]:
                touched[idx_g[i, :cnt_g[i]]] = True
                touched[idx_o[i, :cnt_o[i]]] = True
            Dg = d["D"].cpu().numpy().astype(np.float64)
            np.testing.assert_allclose(Dg[~touched], D1[~touched], atol=2e-4)
            np.testing.assert_allclose(np.linalg.norm(Dg, axis=1), 1.0, atol=1e-5)
            first.append(rm1[k])
        # two more iterations continue from D1 (and, for P-NSGK, X1 as X_prev)
        rm23 = np.zeros(len(dev) * 4)
        dl.dl_batch_iterate(b, 2, rm23)
        rm23 = rm23.reshape(len(dev), 2, 2)
        for k, q in enumerate(probs):
            *_, r_o = oracle.dl(q["Y"].astype(np.float64), q["D"].astype(np.float64), q["s"], 3,
                                rule=rid)
            np.testing.assert_allclose(first[k], r_o[0], atol=1e-4)
            np.testing.assert_allclose(rm23[k], r_o[1:], atol=1e-3, err_msg=str(SHAPES[k]))
    finally:
        dl.dl_batch_destroy(b)


def test_small_batch_group_size_below_n_takes_the_graph_path(dl):
    probs = _problems(seed0=500)[:2]
    dev = _device(probs)
    st = torch.cuda.Stream()
    b = dl.dl_batch_create(dev, autotune=False, stream=st)
    try:
        dl.dl_batch_set_group_size(b, 16)
        l0 = dl.dl_batch_kernel_launches(b)
        rm = np.zeros(len(dev) * 2)
        dl.dl_batch_iterate(b, 1, rm)
        assert dl.dl_batch_kernel_launches(b) - l0 > 1  # per-problem kernels
        assert np.all(np.isfinite(rm))
        dl.dl_batch_set_group_size(b, 50)  # n: the one-launch path again
        l1 = dl.dl_batch_kernel_launches(b)
        dl.dl_batch_iterate(b, 1, rm)
        assert dl.dl_batch_kernel_launches(b) - l1 == 1
        for d, q in zip(dev, probs):
            _check_csc(d, q)
    finally:
        dl.dl_batch_destroy(b)
