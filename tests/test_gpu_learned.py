"""The learned support proposer against the FP64 reference network
(oracle/mlp.py) and the learned DL iteration against plain OMP + JAU.

Tolerances: BF16 weights and activations (8-bit mantissa) give logits and
gradients within a few percent of the FP64 network evaluated on the same
BF16-rounded weights and inputs; the bounds below are relative Frobenius
norms.  The learned DL run must end within 1% of the plain run's RMSE.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1509_05054_gb300 import synth

from _common import csc_to_slots

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


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _shapes(p, n, h):
    return [(h, p), (h,), (h, h), (h,), (n, h), (n,)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_logits_match_reference_network(dl):
    p, n, h, B = 64, 256, 512, 640
    params = synth.proposer_init(p, n, h, seed=1)
    params[1] += 0.05
    params[5] -= 0.1
    Y, _, _ = synth.workload_inputs("patch_n256", m=B)
    prop = dl.dl_proposer_create(p, n, h, 256, torch.cuda.current_stream())
    dl.dl_proposer_set_weights(prop, params)
    logits = torch.zeros(B, n, device="cuda")
    cand = torch.zeros(B, 16, dtype=torch.int32, device="cuda")
    Yd = torch.from_numpy(Y).cuda()
    dl.dl_proposer_forward(prop, Yd, B, logits=logits, cand=cand, K=16)
    dl.dl_proposer_destroy(prop)
    pb = [_bf16(w) if w.ndim == 2 else w for w in params]
    z_ref, _ = mlp.forward(pb, _bf16(Y))
    z = logits.cpu().numpy()
    assert _rel(z, z_ref) < 2e-2, _rel(z, z_ref)
    c = cand.cpu().numpy()
    assert np.all(np.diff(c, axis=1) > 0)
    # the proposed atoms are the reference's top 16 up to BF16 near-ties
    top_ref = np.argsort(-z_ref, axis=1)[:, :16]
    overlap = np.mean([len(set(a) & set(b)) / 16 for a, b in zip(c, top_ref)])
    assert overlap > 0.9, overlap


def test_gradients_match_reference_network(dl):
    """One training step with lr = 0 (gradients only) against oracle/mlp.backward."""
    p, n, h, B = 64, 128, 256, 512
    params = synth.proposer_init(p, n, h, seed=2)
    g = np.random.default_rng(3)
    Y, _, _ = synth.workload_inputs("patch_n256", m=B)
    s = 6
    sup = np.sort(np.argsort(g.random((B, n)), axis=1)[:, :s], axis=1).astype(np.int32)
    prop = dl.dl_proposer_create(p, n, h, B, torch.cuda.current_stream())
    dl.dl_proposer_set_weights(prop, params)
    loss = dl.dl_proposer_train(prop, torch.from_numpy(Y).cuda(), B, torch.from_numpy(sup).cuda(), s,
                                None, B, 0.0)
    grads = dl.dl_proposer_get(prop, 1, _shapes(p, n, h))
    dl.dl_proposer_destroy(prop)
    pb = [_bf16(w) if w.ndim == 2 else w for w in params]
    T = mlp.multi_hot(sup, np.full(B, s), n)
    z, cache = mlp.forward(pb, _bf16(Y))
    ref = mlp.backward(pb, cache, z, T)
    assert abs(loss - mlp.loss(z, T)) < 1e-2 * mlp.loss(z, T)
    for k, (gk, rk) in enumerate(zip(grads, ref)):
        assert _rel(gk, rk) < 5e-2, (k, _rel(gk, rk))


def _labelled_set(dl, n=256, s=6, m_train=131072, warm=3):
    """Plain DL warm-up on patches, then OMP supports of disjoint training patches."""
    Ytr = synth.image_patches(m_train, side=8, workload_id=31, first_image=600)
    Ydl, D, _ = synth.workload_inputs("patch_n256", m=20000)
    st = torch.cuda.Stream()
    ctx = dl.dl_init(64, n, max(m_train, 20000), s, dl.DL_FP32, st)
    Dd = torch.from_numpy(D.copy()).cuda()
    cp = torch.zeros(m_train + 1, dtype=torch.int64, device="cuda")
    ri = torch.zeros(m_train * s, dtype=torch.int32, device="cuda")
    v = torch.zeros(m_train * s, device="cuda")
    dl.dl_iterate(ctx, torch.from_numpy(Ydl).cuda(), 20000, Dd, s, warm, cp, ri, v, np.zeros(2 * warm))
    dl.omp_code(ctx, torch.from_numpy(Ytr).cuda(), m_train, Dd, s, cp, ri, v)
    dl.dl_sync(ctx)
    dl.dl_destroy(ctx)
    idx, _, cnt = csc_to_slots(cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), s)
    return Ytr, idx, cnt, Ydl, Dd.cpu().numpy()


@pytest.fixture(scope="module")
def trained(dl):
    p, n, h, s = 64, 256, 512, 6
    Ytr, sup, cnt, Ydl, Dw = _labelled_set(dl, n=n, s=s)
    prop = dl.dl_proposer_create(p, n, h, 1024, torch.cuda.current_stream())
    dl.dl_proposer_set_weights(prop, synth.proposer_init(p, n, h, seed=7, positives=s))
    Yt, St = torch.from_numpy(Ytr).cuda(), torch.from_numpy(sup).cuda()
    losses = []
    for ep in range(8):
        perm = torch.randperm(len(Ytr), device="cuda")
        losses.append(dl.dl_proposer_train(prop, Yt, len(Ytr), St, s, perm, 1024, 1e-3))
    yield dict(prop=prop, losses=losses, Ytr=Ytr, sup=sup, cnt=cnt, Ydl=Ydl, Dw=Dw, n=n, s=s, h=h)
    dl.dl_proposer_destroy(prop)


def _recall(dl, prop, Y, sup, cnt, K=12):
    m = len(Y)
    cand = torch.zeros(m, K, dtype=torch.int32, device="cuda")
    dl.dl_proposer_forward(prop, torch.from_numpy(Y).cuda(), m, cand=cand, K=K)
    c = cand.cpu().numpy()
    hit = [len(set(c[i]) & set(sup[i, :cnt[i]])) / max(cnt[i], 1) for i in range(m)]
    return float(np.mean(hit))


def test_training_reduces_loss_and_learns_the_supports(dl, trained):
    L = trained["losses"]
    print("epoch losses", L)
    assert L[-1] < 0.8 * L[0]
    Yv = trained["Ytr"][-4096:]
    r_trained = _recall(dl, trained["prop"], Yv, trained["sup"][-4096:], trained["cnt"][-4096:])
    fresh = dl.dl_proposer_create(64, trained["n"], trained["h"], 1024, torch.cuda.current_stream())
    dl.dl_proposer_set_weights(fresh, synth.proposer_init(64, trained["n"], trained["h"], seed=7,
                                                      positives=trained["s"]))
    r_fresh = _recall(dl, fresh, Yv, trained["sup"][-4096:], trained["cnt"][-4096:])
    dl.dl_proposer_destroy(fresh)
    # top-2s of |D^T y| (the proposer without a network) for context
    print(f"support recall in the top 2s: trained {r_trained:.3f}, untrained {r_fresh:.3f}")
    assert r_trained > 0.3 and r_trained > r_fresh + 0.2


def test_learned_dl_restricted_omp_parity_and_equal_rmse(dl, trained):
    """Restricted OMP equals the oracle's OMP on the candidate sub-dictionary for
    the signals kept (no fallback); the run ends within 1% of plain's RMSE; the
    trained proposer needs far fewer fallbacks than an untrained one."""
    n, s, iters = trained["n"], trained["s"], 6
    Y, D = trained["Ydl"], trained["Dw"]
    m = len(Y)
    Yd = torch.from_numpy(Y).cuda()
    st = torch.cuda.Stream()

    def run(prop):
        ctx = dl.dl_init(64, n, m, s, dl.DL_FP32, st)
        if prop is not None:
            dl.dl_attach_proposer(ctx, prop, 2 * s, 3, 0.01)
        Dd = torch.from_numpy(D.copy()).cuda()
        cp = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
        ri = torch.zeros(m * s, dtype=torch.int32, device="cuda")
        v = torch.zeros(m * s, device="cuda")
        rm = np.zeros(2 * iters)
        fbs = []
        for k in range(iters):
            Dk = Dd.cpu().numpy()
            r2 = np.zeros(2)
            dl.dl_iterate(ctx, Yd, m, Dd, s, 1, cp, ri, v, r2)
            rm[2 * k: 2 * k + 2] = r2
            fbs.append(dl.dl_last_fallbacks(ctx) if prop is not None else 0)
            if prop is not None and k == 1:    # a learned iteration: check the restricted OMP
                cand = torch.zeros(m, 2 * s, dtype=torch.int32, device="cuda")
                dl.dl_proposer_forward(prop, Yd, m, cand=cand, K=2 * s)
                c = cand.cpu().numpy()
                idx_g, _, cnt_g = csc_to_slots(cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), s)
                agree = 0
                sample = range(0, m, 97)
                for i in sample:
                    y64 = Y[i:i + 1].astype(np.float64)
                    Dsub = Dk[c[i]].astype(np.float64)
                    ii, _, cc = oracle.omp(y64, Dsub, s)            # restricted to the candidates
                    jj, _, dd = oracle.omp(y64, Dk.astype(np.float64), s)   # full (fallback)
                    got = set(idx_g[i, :cnt_g[i]])
                    agree += got == set(c[i][ii[0, :cc[0]]]) or got == set(jj[0, :dd[0]])
                assert agree >= 0.98 * len(sample), (agree, len(sample))
        dl.dl_destroy(ctx)
        return rm.reshape(iters, 2), fbs

    r_plain, _ = run(None)
    r_learn, fb = run(trained["prop"])
    fresh = dl.dl_proposer_create(64, n, trained["h"], 1024, torch.cuda.current_stream())
    dl.dl_proposer_set_weights(fresh, synth.proposer_init(64, n, trained["h"], seed=7, positives=s))
    _, fb_fresh = run(fresh)
    dl.dl_proposer_destroy(fresh)
    gap = r_learn[-1, 1] / r_plain[-1, 1] - 1
    print(f"final rmse learned {r_learn[-1, 1]:.6f} vs plain {r_plain[-1, 1]:.6f} ({100 * gap:+.3f}%); "
          f"fallbacks trained {fb}, untrained {fb_fresh}")
    assert gap <= 0.01
    learned_iters = [k for k in range(iters) if k % 3 != 0]
    assert sum(fb[k] for k in learned_iters) <= sum(fb_fresh[k] for k in learned_iters)


def test_correlation_proposer_parity_and_comparison(dl, trained):
    """The network-free proposer (candidates = the 2s largest |D^T y|, the same
    restricted OMP and fallback rule): restricted OMP equals the oracle's OMP on
    that candidate sub-dictionary for the signals kept, the run ends within 1%
    of plain's RMSE, and the fallbacks of both proposers are reported side by
    side (what the trained network gains over the method without it)."""
    n, s, iters, K = trained["n"], trained["s"], 6, 2 * trained["s"]
    Y, D = trained["Ydl"], trained["Dw"]
    m = len(Y)
    Yd = torch.from_numpy(Y).cuda()
    st = torch.cuda.Stream()

    def run(mode):
        ctx = dl.dl_init(64, n, m, s, dl.DL_FP32, st)
        if mode == "learned":
            dl.dl_attach_proposer(ctx, trained["prop"], K, 3, 0.01)
        elif mode == "correlations":
            dl.dl_attach_correlation_proposer(ctx, K, 3, 0.01)
        Dd = torch.from_numpy(D.copy()).cuda()
        cp = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
        ri = torch.zeros(m * s, dtype=torch.int32, device="cuda")
        v = torch.zeros(m * s, device="cuda")
        rm = np.zeros(2 * iters)
        fbs = []
        for k in range(iters):
            Dk = Dd.cpu().numpy().astype(np.float64)
            r2 = np.zeros(2)
            dl.dl_iterate(ctx, Yd, m, Dd, s, 1, cp, ri, v, r2)
            rm[2 * k: 2 * k + 2] = r2
            fbs.append(dl.dl_last_fallbacks(ctx) if mode != "plain" else 0)
            if mode == "correlations" and k == 1:   # an iteration on the proposed candidates
                idx_g, _, cnt_g = csc_to_slots(cp.cpu().numpy(), ri.cpu().numpy(), v.cpu().numpy(), s)
                agree, sample = 0, range(0, m, 97)
                for i in sample:
                    y64 = Y[i:i + 1].astype(np.float64)
                    a = np.abs(Dk @ y64[0])
                    c = np.sort(np.argsort(-a, kind="stable")[:K])
                    ii, _, cc = oracle.omp(y64, Dk[c], s)       # restricted to the candidates
                    jj, _, dd = oracle.omp(y64, Dk, s)          # full (fallback)
                    got = set(idx_g[i, :cnt_g[i]])
                    agree += got == set(c[ii[0, :cc[0]]]) or got == set(jj[0, :dd[0]])
                assert agree >= 0.98 * len(sample), (agree, len(sample))
        dl.dl_destroy(ctx)
        return rm.reshape(iters, 2), fbs

    r_plain, _ = run("plain")
    r_corr, fb_corr = run("correlations")
    r_learn, fb_learn = run("learned")
    gap = r_corr[-1, 1] / r_plain[-1, 1] - 1
    learned_iters = [k for k in range(iters) if k % 3 != 0]
    print(f"fallbacks on proposed iterations: learned {[fb_learn[k] for k in learned_iters]}, "
          f"|D^T y| {[fb_corr[k] for k in learned_iters]} of {m}; final rmse learned "
          f"{r_learn[-1, 1]:.6f}, |D^T y| {r_corr[-1, 1]:.6f}, plain {r_plain[-1, 1]:.6f}")
    assert gap <= 0.01
