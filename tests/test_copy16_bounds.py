"""The error analysis behind the all-column search on 16-bit operands, checked
on emulated data (CPU; numpy's float16 rounds to nearest even like the GPU's
conversions).

The search multiplies a 16-bit copy y~ = fp16(s y) / s of each FP32 column y
(s a power of two, values clamped to the FP16 range) by the centroids' two-part
split mu~ = (fp16(s mu) + fp16(s mu - fp16(s mu))) / s.  Its decisions and
bounds rest on four facts, each checked here, including on columns whose
values outgrow the range the scale was chosen for (clamped) and on values
below FP16's normal range:

1. |mu . y - mu~ . y~| <= ||mu|| e + serr ||y~||, with e = ||y - y~|| and
   serr = ||mu - mu~|| computed from the stored values (so each score
   ||mu||^2 - 2 mu . y is within 2 ||mu|| e + 2 serr ||y~|| of the computed one);
2. ||y - mu|| <= sqrt(||y~||^2 - 2 mu~ . y~ + ||mu||^2 + 2 serr ||y~||) + e
   (the upper bound through y~);
3. ||y - mu|| >= sqrt(||y~||^2 - 2 mu~ . y~ + ||mu||^2 - 2 serr ||y~||) - e
   (the lower bound);
4. where the widened scores separate the best centroid from every other, the
   computed best is the exact argmin (checked on constructed near ties).
"""
import numpy as np

F16_MAX = 65504.0


def copy_scale(m):
    """The power of two s with s m in [2^10, 2^11) (1 when m is 0 or not finite)."""
    if not (m > 0.0) or not np.isfinite(m):
        return 1.0
    _, e = np.frexp(m)
    return float(np.ldexp(1.0, int(min(100, max(-100, 11 - e)))))


def copy16(y, s):
    """y~ = fp16(clamp(s y)) / s, in FP32 like the GPU."""
    h = np.clip(y.astype(np.float32) * np.float32(s), -F16_MAX, F16_MAX).astype(np.float16)
    return h.astype(np.float32) / np.float32(s)


def split16(mu, s):
    """mu~ = (p1 + p2) / s with p1 = fp16(clamp(s mu)), p2 = fp16(clamp(s mu - p1))."""
    w = mu.astype(np.float32) * np.float32(s)
    p1 = np.clip(w, -F16_MAX, F16_MAX).astype(np.float16)
    r = w - p1.astype(np.float32)
    p2 = np.clip(r, -F16_MAX, F16_MAX).astype(np.float16)
    return (p1.astype(np.float64) + p2.astype(np.float64)) / s


def cases(rng):
    d = 300
    base = rng.standard_normal((d, 40)).astype(np.float32)
    yield "ordinary", base, 1.0
    yield "wide range", (base * np.exp(rng.uniform(-8, 8, size=(d, 1)))).astype(np.float32), 1.0
    # the scale was chosen for a smaller max |L| than these columns have: clamped values
    yield "clamped", (base * 3e3).astype(np.float32), 1e-3
    # values below FP16's normal range after scaling
    yield "subnormal", (base * 1e-7).astype(np.float32), 1e4


def test_copy16_error_bounds_hold():
    rng = np.random.default_rng(7)
    for name, Y, shrink in cases(rng):
        d, n = Y.shape
        s = copy_scale(float(np.abs(Y).max()) * shrink)
        Yt = copy16(Y, s).astype(np.float64)
        Y64 = Y.astype(np.float64)
        mus = Y64[:, :6] + 0.3 * rng.standard_normal((d, 6))      # centroids near some columns
        mus = mus.astype(np.float32).astype(np.float64)
        clamped = np.abs(Y64 * s) > F16_MAX
        if name == "clamped":
            assert clamped.any()
        for j in range(n):
            y, yt = Y64[:, j], Yt[:, j]
            e = np.linalg.norm(y - yt)
            ny = np.linalg.norm(yt)
            for i in range(mus.shape[1]):
                mu = mus[:, i]
                mut = split16(mu, s)
                serr = np.linalg.norm(mu - mut)
                nm = np.linalg.norm(mu)
                # 1: the product error
                assert abs(mu @ y - mut @ yt) <= nm * e + serr * ny + 1e-12 * (nm * np.linalg.norm(y) + 1), name
                # 2, 3: the distance bounds through y~
                core = ny * ny - 2.0 * (mut @ yt) + nm * nm
                dist = np.linalg.norm(y - mu)
                ub = np.sqrt(max(core + 2.0 * serr * ny, 0.0)) + e
                lb = np.sqrt(max(core - 2.0 * serr * ny, 0.0)) - e
                tol = 1e-9 * (dist + ny + nm)
                assert dist <= ub + tol, name
                assert dist >= lb - tol, name


def near_ties(rng, d=256, per=400, scale=1.0):
    """Adversarial near ties: columns y whose copy y~ is a grid point near the
    bisector of two centroids and whose rounding error y - y~ (a quarter of the
    FP16 spacing per element, signed along +-(mu_a - mu_b)) is as parallel to
    mu_a - mu_b as rounding allows, so the copy shifts the score gap by about
    the full Cauchy-Schwarz bound; the push toward one centroid spans that
    scale.  Returns the columns, their exact argmins and the centroids."""
    mu_a = (rng.standard_normal(d) * scale).astype(np.float32).astype(np.float64)
    # nearly antipodal: ||mu_a - mu_b|| = ||mu_a|| + ||mu_b||, where the scores' separate
    # widenings add up to exactly the bound on the gap's shift
    mu_b = (-mu_a + 0.01 * scale * rng.standard_normal(d)).astype(np.float32).astype(np.float64)
    u = mu_a - mu_b
    m = 0.5 * (mu_a + mu_b)
    Y0 = []
    for _ in range(per):
        w = 0.1 * scale * rng.standard_normal(d)
        w -= (w @ u) / (u @ u) * u
        delta = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-6, -1)
        Y0.append(m + w + delta * u)
    Y0 = np.stack(Y0, axis=1).astype(np.float32)
    s = copy_scale(float(np.abs(Y0).max()))
    Yt = copy16(Y0, s).astype(np.float64)
    h = np.abs(Yt * s).astype(np.float16)
    spacing = np.spacing(h).astype(np.float64) / s             # FP16 spacing above |y~| (halved below a power of 2)
    sigma = rng.choice([-1.0, 1.0], size=(1, per))
    Y = (Yt + 0.24 * spacing * np.sign(u)[:, None] * sigma).astype(np.float32)
    assert np.array_equal(copy16(Y, s).astype(np.float64), Yt)   # same copy
    Y = Y.astype(np.float64)
    da = ((Y - mu_a[:, None]) ** 2).sum(axis=0)
    db = ((Y - mu_b[:, None]) ** 2).sum(axis=0)
    exact = np.where(db < da, 1, 0)                              # ties to the lower index
    return Y, exact, np.stack([mu_a, mu_b], axis=1), s


def decide(Y, mus, s, widen=1.0):
    """The search's rule on emulated operands: the computed best wins where the
    widened score intervals separate it from every other, else queued (-1)."""
    Yt = copy16(Y.astype(np.float32), s).astype(np.float64)
    muts = np.stack([split16(mus[:, i], s) for i in range(mus.shape[1])], axis=1)
    serr = np.linalg.norm(mus - muts, axis=0)
    nm2 = (mus * mus).sum(axis=0)
    out = []
    for j in range(Y.shape[1]):
        y, yt = Y[:, j], Yt[:, j]
        e = np.linalg.norm(y - yt)
        ny = np.linalg.norm(yt)
        sc = nm2 - 2.0 * (muts.T @ yt)
        er = widen * (2.0 * np.sqrt(nm2) * e + 2.0 * serr * ny)
        b = int(np.argmin(sc))
        ok = all(sc[i] - sc[b] > er[i] + er[b] for i in range(len(sc)) if i != b)
        out.append(b if ok else -1)
    return np.array(out)


def test_copy16_decisions_are_exact_argmins():
    """Where the widened scores separate the best centroid from the other, the
    computed best is the exact argmin; near ties are left to the exact
    re-decision.  The centroids are nearly antipodal, so the two scores'
    widenings add up to the bound on the gap's shift, and the rounding errors
    are aligned with mu_a - mu_b: a rule with the widening halved (a dropped
    factor 2) decides some of the same columns wrongly."""
    rng = np.random.default_rng(11)
    for scale in (1.0, 3e3, 1e-6):
        Y, exact, mus, s = near_ties(rng, scale=scale)
        got = decide(Y, mus, s)
        decided = got >= 0
        assert decided.sum() > 0 and (~decided).sum() > 0
        np.testing.assert_array_equal(got[decided], exact[decided])
        cut = decide(Y, mus, s, widen=0.5)
        assert np.any((cut >= 0) & (cut != exact)), scale


def test_copy_scale_rule():
    """The scale puts the reference magnitude in [2^10, 2^11), 32x inside FP16's
    range; it is a power of two, clamped to 2^-100 .. 2^100 (beyond that the
    copy's clamping and error norms still keep the search exact)."""
    for m in (1e-20, 3e-5, 0.7, 1.0, 2048.0, 65504.0, 1e30):
        s = copy_scale(m)
        assert 1024.0 <= m * s < 2048.0
        assert np.log2(s) == int(np.log2(s))
    assert copy_scale(1e-40) == 2.0 ** 100 and copy_scale(1e40) == 2.0 ** -100
    assert copy_scale(0.0) == 1.0 and copy_scale(float("inf")) == 1.0
