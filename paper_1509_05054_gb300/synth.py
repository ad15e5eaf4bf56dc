"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no dictionary-learning arithmetic: it only draws signals and
starting dictionaries.  The GPU library, the FP64 oracle, the tests and the
benchmark all read their inputs from here, so both sides see identical bytes.

Workloads (Section 4 of the paper):

* Dictionary recovery (Section 4.1): a random dictionary D0 with unit-norm
  N(0,1) atoms, signals that are combinations of exactly s distinct atoms with
  N(0,1) coefficients, white Gaussian noise at a global SNR, and a starting
  dictionary made of randomly selected (normalised) data vectors.
* Image-patch DL (Section 4.2): the paper trains on 8x8 blocks of USC-SIPI
  images, which are not available here.  The stand-in is a 1/f^2 Gaussian
  random field: white N(0,1) noise, 2-D FFT, amplitude scaled by 1/|f| (power
  ~ 1/f^2, DC removed), inverse FFT, real part; 512x512 images.  Patches are
  cut at uniformly random positions, mean-removed and scaled to unit
  population variance (||y||^2 = p).  The starting dictionary has i.i.d.
  N(0,1) atoms normalised to unit norm ("random atoms", Section 4.2).

Seeds: image k uses ``1000 + k``; patch positions ``2000 + workload_id``;
the initial dictionary ``3000 + workload_id``.  All generators are numpy
PCG64.

Array layout: signals are returned as ``(m, p)`` float arrays (row i is
signal i -- the column-major ``p x m`` matrix of the paper), dictionaries as
``(n, p)`` (row j is atom j).
"""
from __future__ import annotations

import numpy as np

IMAGE_SIZE = 512
PATCHES_PER_IMAGE = 4096


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian_field_image(k: int, size: int = IMAGE_SIZE) -> np.ndarray:
    """Image k of the 1/f^2 random-field family (float64, size x size)."""
    g = _rng(1000 + k)
    white = g.standard_normal((size, size))
    fy = np.fft.fftfreq(size)[:, None]
    fx = np.fft.fftfreq(size)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    amp = np.zeros_like(f)
    amp[f > 0] = 1.0 / f[f > 0]
    img = np.real(np.fft.ifft2(np.fft.fft2(white) * amp))
    return img


def image_patches(m: int, side: int = 8, workload_id: int = 1, first_image: int = 0,
                  dtype=np.float32) -> np.ndarray:
    """m mean-removed, unit-variance side x side patches as an (m, side*side) array.

    Patches are taken ``PATCHES_PER_IMAGE`` per image, from images
    ``first_image, first_image+1, ...``; patches whose variance is below 1e-12
    are skipped (redrawn).
    """
    p = side * side
    out = np.empty((m, p), dtype=np.float64)
    g = _rng(2000 + workload_id)
    filled = 0
    k = first_image
    while filled < m:
        img = gaussian_field_image(k)
        k += 1
        want = min(PATCHES_PER_IMAGE, m - filled)
        got = 0
        while got < want:
            r = g.integers(0, IMAGE_SIZE - side + 1, size=want - got)
            c = g.integers(0, IMAGE_SIZE - side + 1, size=want - got)
            rows = r[:, None, None] + np.arange(side)[None, :, None]
            cols = c[:, None, None] + np.arange(side)[None, None, :]
            P = img[rows, cols].reshape(-1, p)
            P = P - P.mean(axis=1, keepdims=True)
            var = (P * P).mean(axis=1)
            keep = var >= 1e-12
            P = P[keep] / np.sqrt(var[keep])[:, None]
            out[filled + got: filled + got + P.shape[0]] = P
            got += P.shape[0]
        filled += want
    return out.astype(dtype)


def random_dictionary(p: int, n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """n atoms of length p with i.i.d. N(0,1) entries, each scaled to unit norm."""
    g = _rng(seed)
    D = g.standard_normal((n, p))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    return D.astype(dtype)


def dictionary_from_signals(Y: np.ndarray, n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """n distinct randomly chosen signals (rows of Y), each scaled to unit norm."""
    g = _rng(seed)
    sel = g.choice(Y.shape[0], size=n, replace=False)
    D = np.asarray(Y[sel], dtype=np.float64).copy()
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    return D.astype(dtype)


def sparse_codes(n: int, m: int, s: int, seed: int):
    """Exactly s distinct random atoms per signal with N(0,1) weights.

    Returns (rows (m, s) int32 sorted ascending, vals (m, s) float64).
    """
    g = _rng(seed)
    rows = np.argsort(g.random((m, n)), axis=1)[:, :s]
    rows.sort(axis=1)
    vals = g.standard_normal((m, s))
    return rows.astype(np.int32), vals


def recovery_problem(p: int, n: int, m: int, s: int, snr_db: float | None, seed: int):
    """Synthetic dictionary-recovery problem of Section 4.1.

    Returns (Y (m, p), D0 (n, p), rows, vals) in float64.  ``snr_db=None`` is
    the noise-free case.  Noise variance is global:
    sigma^2 = ||D0 X0||_F^2 / (p m 10^(snr/10)).
    """
    D0 = random_dictionary(p, n, seed)
    rows, vals = sparse_codes(n, m, s, seed + 1)
    clean = np.einsum("ms,msp->mp", vals, D0[rows])
    if snr_db is None:
        return clean, D0, rows, vals
    g = _rng(seed + 2)
    sigma2 = float((clean * clean).sum()) / (p * m * 10.0 ** (snr_db / 10.0))
    Y = clean + np.sqrt(sigma2) * g.standard_normal(clean.shape)
    return Y, D0, rows, vals


# Named workloads (sizes of the paper's experiments, Sections 4.1-4.4).
WORKLOADS = {
    # tiny FP64-checkable recovery-style problem
    "tiny": dict(p=16, n=32, m=1000, s=3, iters=10, kind="recovery", snr_db=30.0, wid=0),
    # image-patch shaped, plain FP32
    "patch_n256": dict(p=64, n=256, m=20000, s=6, iters=50, kind="patch", wid=1),
    # the throughput shape: p=64, n=512, s=8, m=1e5
    "patch_n512": dict(p=64, n=512, m=100000, s=8, iters=50, kind="patch", wid=2),
    # learned-proposer shape
    "patch_n512_m2e5": dict(p=64, n=512, m=200000, s=8, iters=50, kind="patch", wid=4),
}


def batched_problems(count: int = 16, m_scale: float = 1.0, seed: int = 5000, dtype=np.float32):
    """Independent DL problems of uneven shapes (the batched workload): p in
    {36, 64, 100} (6x6, 8x8, 10x10 patches of the 1/f^2 images), n in
    {128, 256, 512, 1024}, m uniform in 5000..60000 (times m_scale), s uniform in
    4..12.  Returns a list of dicts with p, n, m, s, Y (m, p) and D (n, p)."""
    g = _rng(seed)
    out = []
    for k in range(count):
        side = int(g.choice([6, 8, 10]))
        n = int(g.choice([128, 256, 512, 1024]))
        m = max(64, int(round(int(g.integers(5000, 60001)) * m_scale)))
        s = int(g.integers(4, 13))
        p = side * side
        Y = image_patches(m, side=side, workload_id=100 + k, first_image=200 + 20 * k, dtype=dtype)
        D = random_dictionary(p, n, seed=6000 + k, dtype=dtype)
        out.append(dict(p=p, n=n, m=m, s=s, Y=np.ascontiguousarray(Y), D=np.ascontiguousarray(D)))
    return out


def proposer_init(p: int, n: int, hidden: int = 512, seed: int = 0, positives: int | None = None):
    """Seeded starting weights of the support proposer MLP p -> hidden -> hidden -> n:
    [W1 (hidden, p), b1, W2 (hidden, hidden), b2, W3 (n, hidden), b3], weights
    N(0, 2 / fan_in), zero biases; with `positives` (expected ones per target row)
    the output bias starts at the base-rate log-odds log(positives / (n - positives))."""
    g = _rng(seed)
    W1 = g.standard_normal((hidden, p)) * np.sqrt(2.0 / p)
    W2 = g.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden)
    W3 = g.standard_normal((n, hidden)) * np.sqrt(2.0 / hidden)
    b3 = np.zeros(n) if positives is None else np.full(n, np.log(positives / (n - positives)))
    return [W1, np.zeros(hidden), W2, np.zeros(hidden), W3, b3]


def workload_inputs(name: str, m: int | None = None, dtype=np.float32):
    """(Y, D_init, spec) for a named workload; m may be reduced for sampling."""
    spec = dict(WORKLOADS[name])
    if m is not None:
        spec["m"] = int(m)
    if spec["kind"] == "recovery":
        Y, _, _, _ = recovery_problem(spec["p"], spec["n"], spec["m"], spec["s"],
                                      spec["snr_db"], seed=4000 + spec["wid"])
        D = dictionary_from_signals(Y, spec["n"], seed=3000 + spec["wid"])
    else:
        side = int(round(np.sqrt(spec["p"])))
        Y = image_patches(spec["m"], side=side, workload_id=spec["wid"])
        D = random_dictionary(spec["p"], spec["n"], seed=3000 + spec["wid"])
    return np.ascontiguousarray(Y, dtype=dtype), np.ascontiguousarray(D, dtype=dtype), spec
