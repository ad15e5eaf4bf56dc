"""The residual-form OMP (Algorithm 1 step 1 with the correlations of every
step recomputed on the tensor cores) against the FP64 oracle at the limits of
the kernel that runs it.

The plain FP32 form codes with it when 256 < n <= 512, p <= 64, p % 4 == 0,
s <= 8 and the call fills most of one round of tiles; these tests take it for
every supported call (DL_OMP_RES=2).  The shapes below reach each edge of that
kernel: p from 4 to 64 (the FP16 residual rows padded with zeros to 64), n
from 40 and 256 (one accumulator unit per step, the units alternating) and 257
(one atom in the second unit) to 512, s from 1 to 8, m = 1, m = 129 (a second,
ragged tile), and m one full round of tiles plus five signals (all SMs and
both slots busy, then a last round with one tile).  The BF16 form of the
kernel (BF16 operands for the correlations, FP32 elsewhere) is checked for
FP32-accurate coefficients on its own supports and for the coding error.  Degenerate inputs: zero
signals (empty support), exactly 1- and 2-sparse signals (the residual stop
rule), and a pair of nearly parallel atoms (Cholesky pivots below 1e-6, the
hand-off to the FP64 re-solve).  Supports must match the oracle on >= 99.9%
of the signals with every mismatch a near-tie, values within 5e-4, and the
coding error no worse than the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_1509_05054_gb300 import synth

from _common import assert_support_parity, csc_to_slots

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROUND = 152 * 2 * 128  # signals of one round of tiles on a 152-SM GB300
SHAPES = [(64, 512, 3001, 8), (60, 300, 2049, 5), (4, 257, 130, 1), (32, 384, 129, 8),
          (64, 511, 1, 3), (44, 480, 1000, 6), (64, 512, ROUND + 5, 2), (64, 256, 2500, 6),
          (16, 40, 700, 4)]


@pytest.fixture(autouse=True)
def residual_form_for_every_call(monkeypatch):
    monkeypatch.setenv("DL_OMP_RES", "2")


@pytest.fixture(scope="module")
def dl():
    from paper_1509_05054_gb300 import build as _b
    _b.build()
    from paper_1509_05054_gb300 import dl as _dl
    _dl.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return _dl


def _code(dl, Y, D, s):
    """omp_code on the device; returns slots and the coding kernel that ran."""
    m, p = Y.shape
    n = D.shape[0]
    ctx = dl.dl_init(p, n, max(1, m), s, dl.DL_FP32, torch.cuda.current_stream())
    try:
        Yd = torch.from_numpy(np.ascontiguousarray(Y, np.float32)).cuda()
        Dd = torch.from_numpy(np.ascontiguousarray(D, np.float32)).cuda()
        colptr = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
        rowidx = torch.zeros(max(1, m * s), dtype=torch.int32, device="cuda")
        val = torch.zeros(max(1, m * s), dtype=torch.float32, device="cuda")
        dl.omp_code(ctx, Yd, m, Dd, s, colptr, rowidx, val)
        dl.dl_sync(ctx)
        kind = dl.dl_last_omp_kernel(ctx)
        resolved = dl.dl_last_resolved(ctx)
    finally:
        dl.dl_destroy(ctx)
    idx, v, cnt = csc_to_slots(colptr.cpu().numpy(), rowidx.cpu().numpy(), val.cpu().numpy(), s)
    return idx, v, cnt, kind, resolved


def _check_against_oracle(Y, D, s, idx_g, val_g, cnt_g):
    Y64, D64 = Y.astype(np.float64), D.astype(np.float64)
    idx_o, val_o, cnt_o, gaps = oracle.omp(Y64, D64, s, return_gaps=True)
    same = assert_support_parity(idx_g, cnt_g, idx_o, cnt_o, gaps)
    np.testing.assert_allclose(val_g[same], val_o[same], rtol=0, atol=5e-4)
    assert (oracle.rmse(Y64, D64, idx_g, val_g.astype(np.float64), cnt_g)
            <= oracle.rmse(Y64, D64, idx_o, val_o, cnt_o) + 1e-4)
    return idx_o, val_o, cnt_o


@pytest.mark.parametrize("p,n,m,s", SHAPES)
def test_residual_omp_limits_match_oracle(dl, p, n, m, s):
    Y, _, _, _ = synth.recovery_problem(p, n, m, s, 30.0, seed=700 + p + n + s)
    D = synth.random_dictionary(p, n, seed=800 + p + n, dtype=np.float32)
    Y = Y.astype(np.float32)
    idx_g, val_g, cnt_g, kind, _ = _code(dl, Y, D, s)
    assert kind == 2, kind  # the residual-form OMP ran
    _check_against_oracle(Y, D, s, idx_g, val_g, cnt_g)


def test_residual_omp_degenerate_signals(dl):
    p, n, m, s = 64, 512, 600, 8
    rng = np.random.default_rng(901)
    D = synth.random_dictionary(p, n, seed=902, dtype=np.float64)
    # atoms 0 and 1 nearly parallel: a pivot of about 1e-8 once both are chosen
    D[1] = D[0] + 1e-4 * rng.standard_normal(p)
    D[1] /= np.linalg.norm(D[1])
    D = D.astype(np.float32)
    Y = (rng.standard_normal((m, p)) * 0.2).astype(np.float32)
    Y[0:10] = 0.0                                                     # empty supports
    for k in range(10, 20):                                           # 1-sparse
        Y[k] = 3.0 * D[100 + k]
    for k in range(20, 30):                                           # 2-sparse
        Y[k] = D[200 + k] - 0.5 * D[300 + k]
    for k in range(30, 40):                                           # along atoms 0 and 1
        Y[k] = D[0] + (k - 34.5) * 0.1 * D[1] + 0.01 * rng.standard_normal(p).astype(np.float32)
    idx_g, val_g, cnt_g, kind, resolved = _code(dl, Y, D, s)
    assert kind == 2, kind
    assert np.all(cnt_g[0:10] == 0)
    for k in range(10, 20):
        assert cnt_g[k] == 1 and idx_g[k, 0] == 100 + k, (k, cnt_g[k], idx_g[k])
        assert abs(val_g[k, 0] - 3.0) < 1e-5
    for k in range(20, 30):
        assert cnt_g[k] == 2, (k, cnt_g[k])
        assert list(idx_g[k, :2]) == [200 + k, 300 + k]
        np.testing.assert_allclose(val_g[k, :2], [1.0, -0.5], atol=1e-5)
    _check_against_oracle(Y, D, s, idx_g, val_g, cnt_g)


def test_residual_omp_nonfinite_signal_is_reported(dl):
    p, n, m, s = 64, 512, 400, 8
    Y, _, _, _ = synth.recovery_problem(p, n, m, s, 30.0, seed=911)
    D = synth.random_dictionary(p, n, seed=912, dtype=np.float32)
    Yd = torch.from_numpy(Y.astype(np.float32)).cuda()
    Dd = torch.from_numpy(D).cuda()
    ctx = dl.dl_init(p, n, m, s, dl.DL_FP32, torch.cuda.current_stream())
    try:
        colptr = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
        rowidx = torch.zeros(m * s, dtype=torch.int32, device="cuda")
        val = torch.zeros(m * s, dtype=torch.float32, device="cuda")
        Ybad = Yd.clone()
        Ybad[77, 5] = float("inf")
        dl.omp_code(ctx, Ybad, m, Dd, s, colptr, rowidx, val)
        with pytest.raises(dl.DLError) as e:
            dl.dl_sync(ctx)
        assert e.value.status == dl.DL_ENUMERIC
        assert dl.dl_last_omp_kernel(ctx) == 2
        dl.omp_code(ctx, Yd, m, Dd, s, colptr, rowidx, val)  # the context stays usable
        dl.dl_sync(ctx)
        idx, v, cnt = csc_to_slots(colptr.cpu().numpy(), rowidx.cpu().numpy(),
                                   val.cpu().numpy(), s)
        _check_against_oracle(Y.astype(np.float32), D, s, idx, v, cnt)
    finally:
        dl.dl_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_host_buffer_iteration_splits_at_a_round_of_tiles(dl, prec):
    """dl_iterate with pinned host buffers (FP32 and BF16 forms) stages Y in
    two pieces (the first one full round of the OMP kernel's tiles) and gives
    the device path's result:
    the coding of each signal depends on nothing but its own data, so the
    supports are identical; the atom update sums in L2 in no fixed order."""
    name, s = "patch_n512", 8
    m = ROUND + 1000
    Y, D, _ = synth.workload_inputs(name, m=m)
    p, n = D.shape[1], D.shape[0]
    st = torch.cuda.Stream()
    outs = []
    for host in (False, True):
        ctx = dl.dl_init(p, n, m, s, prec, st)
        try:
            if host:
                args = [torch.from_numpy(Y).pin_memory(), torch.from_numpy(D.copy()).pin_memory(),
                        torch.zeros(m + 1, dtype=torch.int64).pin_memory(),
                        torch.zeros(m * s, dtype=torch.int32).pin_memory(),
                        torch.zeros(m * s, dtype=torch.float32).pin_memory()]
            else:
                args = [torch.from_numpy(Y).cuda(), torch.from_numpy(D.copy()).cuda(),
                        torch.zeros(m + 1, dtype=torch.int64, device="cuda"),
                        torch.zeros(m * s, dtype=torch.int32, device="cuda"),
                        torch.zeros(m * s, dtype=torch.float32, device="cuda")]
            rm = np.zeros(2)
            with torch.cuda.stream(st):
                dl.dl_iterate(ctx, args[0], m, args[1], s, 1, args[2], args[3], args[4], rm)
            st.synchronize()
            assert dl.dl_last_omp_kernel(ctx) == 2
            outs.append((args[1].cpu().numpy(),) +
                        csc_to_slots(args[2].cpu().numpy(), args[3].cpu().numpy(),
                                     args[4].cpu().numpy(), s) + (rm.copy(),))
        finally:
            dl.dl_destroy(ctx)
    (Dd, idx_d, val_d, cnt_d, rm_d), (Dh, idx_h, val_h, cnt_h, rm_h) = outs
    assert np.array_equal(cnt_d, cnt_h) and np.array_equal(idx_d, idx_h)
    np.testing.assert_allclose(val_h, val_d, rtol=0, atol=1e-5)
    np.testing.assert_allclose(Dh, Dd, rtol=0, atol=1e-5)
    np.testing.assert_allclose(rm_h, rm_d, rtol=0, atol=1e-6)


BF16_SHAPES = [("patch", 64, 512, 4000, 8), ("recovery", 36, 300, 1500, 5),
               ("recovery", 64, 256, 1200, 6), ("recovery", 16, 40, 600, 4)]


@pytest.mark.parametrize("kind,p,n,m,s", BF16_SHAPES)
def test_bf16_residual_form_keeps_fp32_coefficients(dl, kind, p, n, m, s):
    """The BF16 form of the residual OMP: correlations from BF16 operands (the
    argmax may differ from the FP64 oracle's on close calls), but alpha_sel, the
    Cholesky factor and the residual in FP32 from D put back together exactly:
    every signal's coefficients are the least-squares solution on its own
    support to FP32 accuracy, and the coding error is the oracle's to 1%.
    Shapes: the patch workload, and recovery problems with p < 64, n = 256 and
    n = 40 (one accumulator unit per step)."""
    if kind == "patch":
        Y, D, _ = synth.workload_inputs("patch_n512", m=m)
    else:
        Y, _, _, _ = synth.recovery_problem(p, n, m, s, 30.0, seed=1300 + p + n)
        D = synth.random_dictionary(p, n, seed=1400 + p + n, dtype=np.float32)
        Y = Y.astype(np.float32)
    ctx = dl.dl_init(p, n, m, s, dl.DL_BF16, torch.cuda.current_stream())
    try:
        colptr = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
        rowidx = torch.zeros(m * s, dtype=torch.int32, device="cuda")
        val = torch.zeros(m * s, dtype=torch.float32, device="cuda")
        dl.omp_code(ctx, torch.from_numpy(Y).cuda(), m, torch.from_numpy(D).cuda(), s, colptr,
                    rowidx, val)
        dl.dl_sync(ctx)
        assert dl.dl_last_omp_kernel(ctx) == 2
    finally:
        dl.dl_destroy(ctx)
    idx, v, cnt = csc_to_slots(colptr.cpu().numpy(), rowidx.cpu().numpy(), val.cpu().numpy(), s)
    Y64, D64 = Y.astype(np.float64), D.astype(np.float64)
    for i in range(m):
        I = idx[i, :cnt[i]]
        assert len(set(I.tolist())) == len(I) and np.all(np.diff(I) > 0)
        g, *_ = np.linalg.lstsq(D64[I].T, Y64[i], rcond=None)
        np.testing.assert_allclose(v[i, :cnt[i]], g, rtol=0, atol=1e-4)
    idx_o, val_o, cnt_o = oracle.omp(Y64, D64, s)
    same = np.mean(np.all(idx == idx_o, axis=1) & (cnt == cnt_o))
    r_g = oracle.rmse(Y64, D64, idx, v.astype(np.float64), cnt)
    r_o = oracle.rmse(Y64, D64, idx_o, val_o, cnt_o)
    print(f"bf16 residual form: identical supports {100 * same:.2f}%, rmse {100 * (r_g / r_o - 1):+.4f}%")
    assert same > 0.9
    if kind == "patch":
        assert same < 0.999  # BF16 correlations, not the FP32 path
    assert r_g <= 1.01 * r_o


def test_bf16_residual_form_reaches_plain_rmse(dl):
    """Ten Jacobi iterations of the BF16 residual form end within 1% of the
    FP32 form's relative RMSE from the same start."""
    Y, D, spec = synth.workload_inputs("patch_n512", m=20000)
    m, p, n, s, iters = 20000, D.shape[1], D.shape[0], spec["s"], 10
    out = {}
    for prec in (dl.DL_FP32, dl.DL_BF16):
        st = torch.cuda.Stream()
        ctx = dl.dl_init(p, n, m, s, prec, st)
        try:
            Dd = torch.from_numpy(D.copy()).cuda()
            cp = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
            ri = torch.zeros(m * s, dtype=torch.int32, device="cuda")
            v = torch.zeros(m * s, device="cuda")
            rm = np.zeros(2 * iters)
            dl.dl_iterate(ctx, torch.from_numpy(Y).cuda(), m, Dd, s, iters, cp, ri, v, rm)
            assert dl.dl_last_omp_kernel(ctx) == 2
        finally:
            dl.dl_destroy(ctx)
        out[prec] = rm.reshape(iters, 2)
    gap = out[dl.DL_BF16][-1, 1] / out[dl.DL_FP32][-1, 1] - 1
    print(f"bf16 residual form: final rmse {100 * gap:+.3f}% against the FP32 form")
    assert abs(gap) <= 0.01
