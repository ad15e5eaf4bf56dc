"""The atom update with group size ntilde < n (Algorithm 1 steps 2-5: groups of
ntilde consecutive atoms updated one after another, each from the error left by
the earlier groups) against the FP64 oracle's grouped update, through the C ABI.

Tolerances as in test_gpu_parity.py, widened for the sequential groups (each
group starts from FP32 atoms and coefficients the previous groups produced):
atoms within 2e-5, coefficients within 5e-4, RMSE within 1e-5.
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


def _csc(idx, val, cnt, s):
    m = len(cnt)
    colptr = np.zeros(m + 1, np.int64)
    colptr[1:] = np.cumsum(cnt)
    mask = idx >= 0
    r = torch.zeros(m * s, dtype=torch.int32, device="cuda")
    v = torch.zeros(m * s, dtype=torch.float32, device="cuda")
    r[: mask.sum()] = torch.from_numpy(idx[mask].astype(np.int32)).cuda()
    v[: mask.sum()] = torch.from_numpy(val[mask].astype(np.float32)).cuda()
    return torch.from_numpy(colptr).cuda(), r, v


@pytest.mark.parametrize("ntilde", [64, 37, 1])
def test_grouped_jau_update_matches_oracle(dl, ntilde):
    name, m, s = "patch_n256", 3001, 6
    Y, D, _ = synth.workload_inputs(name, m=m)
    Y64, D64 = Y.astype(np.float64), D.astype(np.float64)
    idx, val, cnt = oracle.omp(Y64, D64, s)
    val32 = val.astype(np.float32).astype(np.float64)
    D1_o, val1_o, _ = oracle.atom_update(Y64, D64, idx, val32, cnt, ntilde=ntilde)
    p, n = D.shape[1], D.shape[0]
    ctx = dl.dl_init(p, n, m, s, dl.DL_FP32, torch.cuda.current_stream())
    dl.dl_set_group_size(ctx, ntilde)
    Dd = torch.from_numpy(D.copy()).cuda()
    colptr, rowidx, v = _csc(idx, val, cnt, s)
    rm = np.zeros(2)
    dl.jau_update(ctx, torch.from_numpy(Y).cuda(), m, Dd, colptr, rowidx, v, rm)
    dl.dl_destroy(ctx)
    np.testing.assert_allclose(Dd.cpu().numpy(), D1_o, rtol=0, atol=2e-5)
    _, val1_g, _ = csc_to_slots(colptr.cpu().numpy(), rowidx.cpu().numpy(), v.cpu().numpy(), s)
    np.testing.assert_allclose(val1_g, val1_o, rtol=0, atol=5e-4)
    assert abs(rm[0] - oracle.rmse(Y64, D64, idx, val32, cnt)) <= 1e-5
    assert abs(rm[1] - oracle.rmse(Y64, D1_o, idx, val1_o, cnt)) <= 1e-5
    # grouping changes the result (Eq. 2 vs Eq. 5): not the Jacobi update
    D1_j, _, _ = oracle.jau(Y64, D64, idx, val32, cnt)
    assert np.max(np.abs(D1_o - D1_j)) > 1e-3


def test_grouped_dl_iterate_teacher_forced(dl):
    """Two iterations with ntilde = n/2, each against the oracle started from the
    GPU's own dictionary (graph-captured from the second iteration)."""
    name, m, s, nt = "patch_n256", 4003, 6, 128
    Y, D, _ = synth.workload_inputs(name, m=m)
    Y64 = Y.astype(np.float64)
    p, n = D.shape[1], D.shape[0]
    ctx = dl.dl_init(p, n, m, s, dl.DL_FP32, torch.cuda.current_stream())
    dl.dl_set_group_size(ctx, nt)
    Yd, Dd = torch.from_numpy(Y).cuda(), torch.from_numpy(D.copy()).cuda()
    cp, ri, v = (torch.zeros(m + 1, dtype=torch.int64, device="cuda"),
                 torch.zeros(m * s, dtype=torch.int32, device="cuda"),
                 torch.zeros(m * s, dtype=torch.float32, device="cuda"))
    for k in range(3):
        Dk = Dd.cpu().numpy().astype(np.float64)
        rm = np.zeros(2)
        dl.dl_iterate(ctx, Yd, m, Dd, s, 1, cp, ri, v, rm)
        idx_o, val_o, cnt_o, gaps = oracle.omp(Y64, Dk, s, return_gaps=True)
        D1_o, val1_o, _ = oracle.atom_update(Y64, Dk, idx_o, val_o, cnt_o, ntilde=nt)
        assert abs(rm[0] - oracle.rmse(Y64, Dk, idx_o, val_o, cnt_o)) <= 1e-4
        assert abs(rm[1] - oracle.rmse(Y64, D1_o, idx_o, val1_o, cnt_o)) <= 1e-4
        idx_g, val_g, cnt_g = csc_to_slots(cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), s)
        assert_support_parity(idx_g, cnt_g, idx_o, cnt_o, gaps)
    dl.dl_destroy(ctx)


def test_group_size_arguments(dl):
    Y, D, _ = synth.workload_inputs("patch_n256", m=600)
    ctx = dl.dl_init(64, 256, 600, 6, dl.DL_FP32, torch.cuda.current_stream())
    for bad in (0, -3, 257):
        with pytest.raises(dl.DLError) as e:
            dl.dl_set_group_size(ctx, bad)
        assert e.value.status == dl.DL_EINVAL
    dl.dl_set_group_size(ctx, 256)      # the Jacobi form
    dl.dl_destroy(ctx)
    # p % 4 != 0 (5x5 patches) has no grouped path
    Y25 = synth.image_patches(500, side=5, workload_id=77)
    D25 = synth.random_dictionary(25, 60, seed=9, dtype=np.float32)
    ctx = dl.dl_init(25, 60, 500, 4, dl.DL_FP32, torch.cuda.current_stream())
    dl.dl_set_group_size(ctx, 20)
    cp, ri, v = (torch.zeros(501, dtype=torch.int64, device="cuda"),
                 torch.zeros(2000, dtype=torch.int32, device="cuda"),
                 torch.zeros(2000, dtype=torch.float32, device="cuda"))
    with pytest.raises(dl.DLError) as e:
        dl.dl_iterate(ctx, torch.from_numpy(Y25).cuda(), 500, torch.from_numpy(D25).cuda(), 4, 1,
                      cp, ri, v, None)
    assert e.value.status == dl.DL_ENOTIMPL
    dl.dl_destroy(ctx)


@pytest.mark.parametrize("ntilde", [256, 64])
def test_sgk_rule_matches_oracle(dl, ntilde):
    """P-SGK (Eq. 6, Algorithm 2): atoms from F x^T / (x x^T), normalised, the
    coefficients left as the coding pass made them."""
    name, m, s = "patch_n256", 2501, 6
    Y, D, _ = synth.workload_inputs(name, m=m)
    Y64, D64 = Y.astype(np.float64), D.astype(np.float64)
    idx, val, cnt = oracle.omp(Y64, D64, s)
    val32 = val.astype(np.float32).astype(np.float64)
    D1_o, val1_o, _ = oracle.atom_update(Y64, D64, idx, val32, cnt, ntilde=ntilde,
                                         rule=oracle.RULE_SGK)
    np.testing.assert_array_equal(val1_o, val32)
    p, n = D.shape[1], D.shape[0]
    ctx = dl.dl_init(p, n, m, s, dl.DL_FP32, torch.cuda.current_stream())
    dl.dl_set_group_size(ctx, ntilde)
    dl.dl_set_update_rule(ctx, dl.DL_RULE_SGK)
    Dd = torch.from_numpy(D.copy()).cuda()
    colptr, rowidx, v = _csc(idx, val, cnt, s)
    rm = np.zeros(2)
    dl.jau_update(ctx, torch.from_numpy(Y).cuda(), m, Dd, colptr, rowidx, v, rm)
    with pytest.raises(dl.DLError):
        dl.dl_set_update_rule(ctx, 7)
    dl.dl_destroy(ctx)
    np.testing.assert_allclose(Dd.cpu().numpy(), D1_o, rtol=0, atol=2e-5)
    _, val1_g, _ = csc_to_slots(colptr.cpu().numpy(), rowidx.cpu().numpy(), v.cpu().numpy(), s)
    np.testing.assert_allclose(val1_g, val32, rtol=0, atol=1e-7)
    assert abs(rm[1] - oracle.rmse(Y64, D1_o, idx, val1_o, cnt)) <= 1e-5


@pytest.mark.parametrize("ntilde", [256, 64])
def test_nsgk_dl_iterate_matches_oracle(dl, ntilde):
    """P-NSGK (Eq. 7) over three iterations: each GPU atom update against the
    oracle's, given the GPU's own dictionary, representations X^(k) and the
    previous iteration's X^(k-1) (the first iteration uses its own X)."""
    name, m, s = "patch_n256", 3001, 6
    Y, D, _ = synth.workload_inputs(name, m=m)
    Y64 = Y.astype(np.float64)
    p, n = D.shape[1], D.shape[0]
    ctx = dl.dl_init(p, n, m, s, dl.DL_FP32, torch.cuda.current_stream())
    dl.dl_set_group_size(ctx, ntilde)
    dl.dl_set_update_rule(ctx, dl.DL_RULE_NSGK)
    Yd, Dd = torch.from_numpy(Y).cuda(), torch.from_numpy(D.copy()).cuda()
    cp, ri, v = (torch.zeros(m + 1, dtype=torch.int64, device="cuda"),
                 torch.zeros(m * s, dtype=torch.int32, device="cuda"),
                 torch.zeros(m * s, dtype=torch.float32, device="cuda"))
    prev = None
    for k in range(3):
        Dk = Dd.cpu().numpy().astype(np.float64)
        rm = np.zeros(2)
        dl.dl_iterate(ctx, Yd, m, Dd, s, 1, cp, ri, v, rm)
        idx_g, val_g, cnt_g = csc_to_slots(cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), s)
        idx_o, _, cnt_o, gaps = oracle.omp(Y64, Dk, s, return_gaps=True)
        assert_support_parity(idx_g, cnt_g, idx_o, cnt_o, gaps)
        val64 = val_g.astype(np.float64)
        pi, pv, pc = prev if prev is not None else (idx_g, val64, cnt_g)
        D1_o, _ = oracle.atom_update_nsgk(Y64, Dk, idx_g, val64, cnt_g, pi, pv, pc, ntilde=ntilde)
        np.testing.assert_allclose(Dd.cpu().numpy(), D1_o, rtol=0, atol=2e-5)
        assert abs(rm[1] - oracle.rmse(Y64, D1_o, idx_g, val64, cnt_g)) <= 1e-5
        if k == 1:   # from the second iteration on, P-NSGK is not P-SGK
            D1_s, _, _ = oracle.atom_update(Y64, Dk, idx_g, val64, cnt_g, ntilde=ntilde,
                                            rule=oracle.RULE_SGK)
            assert np.max(np.abs(D1_o - D1_s)) > 1e-4
        prev = (idx_g, val64, cnt_g)
    dl.dl_destroy(ctx)


@pytest.mark.parametrize("rule,ntilde", [(0, 50), (0, 16), (1, 50), (2, 50), (2, 16)])
def test_recovery_shape_iterations_match_oracle(dl, rule, ntilde):
    """The dictionary-recovery shape of Section 4.1 (p=20, n=50, m=1500, s=3):
    n p + n = 1050 is not a multiple of 4, so the float4 accumulation's copies
    of U sit at a padded stride, and n % 4 != 0 sends both products to the
    CUDA-core GEMM.  Three iterations of each rule, each atom update against
    the oracle's from the GPU's own dictionary and representations."""
    p, n, m, s = 20, 50, 1500, 3
    Y, _, _, _ = synth.recovery_problem(p, n, m, s, 20.0, seed=10000)
    D = synth.dictionary_from_signals(Y, n, seed=20000)
    Y, D = Y.astype(np.float32), D.astype(np.float32)
    Y64 = Y.astype(np.float64)
    ctx = dl.dl_init(p, n, m, s, dl.DL_FP32, torch.cuda.current_stream())
    dl.dl_set_group_size(ctx, ntilde)
    dl.dl_set_update_rule(ctx, rule)
    Yd, Dd = torch.from_numpy(Y).cuda(), torch.from_numpy(D.copy()).cuda()
    cp, ri, v = (torch.zeros(m + 1, dtype=torch.int64, device="cuda"),
                 torch.zeros(m * s, dtype=torch.int32, device="cuda"),
                 torch.zeros(m * s, dtype=torch.float32, device="cuda"))
    prev = None
    for k in range(3):
        Dk = Dd.cpu().numpy().astype(np.float64)
        rm = np.zeros(2)
        dl.dl_iterate(ctx, Yd, m, Dd, s, 1, cp, ri, v, rm)
        idx_g, val_g, cnt_g = csc_to_slots(cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), s)
        idx_o, val_o, cnt_o, gaps = oracle.omp(Y64, Dk, s, return_gaps=True)
        assert_support_parity(idx_g, cnt_g, idx_o, cnt_o, gaps)
        assert abs(rm[0] - oracle.rmse(Y64, Dk, idx_o, val_o, cnt_o)) <= 1e-4
        if rule == dl.DL_RULE_NSGK:
            # the coding pass's X (the GPU's slots hold it: P-NSGK leaves X)
            val64 = val_g.astype(np.float64)
            pi, pv, pc = prev if prev is not None else (idx_g, val64, cnt_g)
            D1_o, _ = oracle.atom_update_nsgk(Y64, Dk, idx_g, val64, cnt_g, pi, pv, pc,
                                              ntilde=ntilde)
            prev = (idx_g, val64, cnt_g)
        else:
            D1_o, _, _ = oracle.atom_update(Y64, Dk, idx_o, val_o, cnt_o, ntilde=ntilde,
                                            rule=rule)
        np.testing.assert_allclose(Dd.cpu().numpy(), D1_o, rtol=0, atol=5e-5)
    dl.dl_destroy(ctx)
