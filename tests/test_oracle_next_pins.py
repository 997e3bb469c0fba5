"""Pins of the sampler and reconstruction-loss oracles (CPU only).

Each pin checks the oracle against something other than itself: the
generator's published known-answer vectors, FP64 library functions, the
distribution the draws must follow, the stationary law of Langevin dynamics,
closed forms, a library convolution, finite differences, and structural
identities of the split and merge transitions."""
import json
import os
import types

import numpy as np
import pytest
from scipy import ndimage, stats

import oracle
from oracle import mcmc, ssim


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


# ----------------------------------------------------------------------------
# Philox4x32-10 and the normals
# ----------------------------------------------------------------------------

def test_philox_known_answers():
    """Known-answer vectors published with Philox4x32-10 (Salmon et al.,
    SC'11; the Random123 distribution's kat_vectors): counter, key -> output."""
    kat = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in kat:
        got = mcmc.philox4x32_10(np.array([ctr], dtype=np.uint64), np.array(key, dtype=np.uint64))[0]
        assert tuple(int(v) for v in got) == want


def test_log32_and_sincos32_against_fp64():
    rng = np.random.default_rng(0)
    u = (rng.integers(1, 2 ** 24 + 1, 100_000) * 2.0 ** -24).astype(np.float32)
    u = np.concatenate([u, np.float32([2.0 ** -24, 0.5, 1.0, 0.70710677, 1.4142135, 3.0, 1e-30, 7e30])])
    got = mcmc.log32(u).astype(np.float64)
    want = np.log(u.astype(np.float64))
    ulp = np.spacing(np.abs(want).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(got - want) <= 3 * ulp + 1e-45)
    assert mcmc.log32(np.float32([1.0]))[0] == 0.0
    v = (rng.integers(0, 2 ** 24, 100_000) * 2.0 ** -24).astype(np.float32)
    v = np.concatenate([v, np.float32([0.0, 0.125, 0.25, 0.375, 0.5, 0.75, 1 - 2 ** -24])])
    s, c = mcmc.sincos2pi32(v)
    t = 2.0 * np.pi * v.astype(np.float64)
    assert np.abs(s - np.sin(t)).max() < 2e-7 and np.abs(c - np.cos(t)).max() < 2e-7
    assert s[-7] == 0.0 and c[-7] == 1.0          # u = 0
    assert c[-5] == 0.0 and s[-5] == 1.0          # u = 1/4: quadrant boundary is exact


def test_normals_fp32_match_fp64_and_are_standard_normal():
    bits = mcmc.draws(np.arange(100_000), 0, 0, 3, 2024)
    z64 = mcmc.normals64(bits)
    z32 = mcmc.normals32(bits).astype(np.float64)
    assert np.all(np.abs(z32 - z64) <= 3e-7 * (1.0 + np.abs(z64)))
    z = z64.ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # pairs from one Box-Muller draw are uncorrelated, and so are streams and steps
    assert abs(np.corrcoef(z64[:, 0], z64[:, 1])[0, 1]) < 5 / np.sqrt(len(z64))
    other = mcmc.normals64(mcmc.draws(np.arange(100_000), 1, 0, 3, 2024)).ravel()
    later = mcmc.normals64(mcmc.draws(np.arange(100_000), 0, 0, 4, 2024)).ravel()
    assert abs(np.corrcoef(z, other)[0, 1]) < 5 / np.sqrt(z.size)
    assert abs(np.corrcoef(z, later)[0, 1]) < 5 / np.sqrt(z.size)


# ----------------------------------------------------------------------------
# parameter update (SGLD)
# ----------------------------------------------------------------------------

def _toy_scene(n, k_sr, k_sh, degree, rng):
    b = (degree + 1) ** 2
    return types.SimpleNamespace(
        n=n, k_sr=k_sr, k_sh=k_sh, sh_degree=degree,
        pos=rng.normal(size=(n, 3)).astype(np.float32),
        opacity_logit=rng.normal(size=n).astype(np.float32),
        sr_rows=rng.normal(size=(k_sr, 8)).astype(np.float32),
        sh_rows=rng.normal(size=(k_sh, b, 3)).astype(np.float32),
        g2sr=rng.integers(0, k_sr, n).astype(np.uint16), g2sh=rng.integers(0, k_sh, n).astype(np.uint16))


def test_sgld_zero_step_is_identity_and_pad_column_is_fixed():
    rng = np.random.default_rng(1)
    sc = _toy_scene(100, 16, 16, 1, rng)
    grads = {"dpos": rng.normal(size=(100, 3)), "dlogit": rng.normal(size=100),
             "d_sr": rng.normal(size=(16, 8)), "d_sh": rng.normal(size=(16, 4, 3))}
    out = mcmc.sgld_update(sc, grads, {"pos": 0.0, "logit": 0.0, "sr": 0.0, "sh": 0.0}, 5, 9)
    assert np.array_equal(out["pos"], sc.pos.astype(np.float64))
    assert np.array_equal(out["sh"], sc.sh_rows.astype(np.float64))
    out = mcmc.sgld_update(sc, grads, {"pos": 1e-2, "logit": 1e-2, "sr": 1e-2, "sh": 1e-2}, 5, 9)
    assert np.array_equal(out["sr"][:, 7], sc.sr_rows[:, 7].astype(np.float64))
    assert not np.array_equal(out["sr"][:, :7], sc.sr_rows[:, :7].astype(np.float64))


def test_sgld_samples_the_gaussian_posterior():
    """Langevin dynamics on L = |x|^2 / (2 s^2): x' = a x + sqrt(eps) z with
    a = 1 - eps / (2 s^2), so after T steps from 0 the variance is
    eps (1 - a^(2T)) / (1 - a^2) and the mean 0 (a dropped sqrt, a wrong sign
    of the gradient or eps in place of eps/2 all miss this)."""
    n, s2, eps, steps = 20_000, 0.25, 0.02, 60
    sc = types.SimpleNamespace(pos=np.zeros((n, 3), np.float32), opacity_logit=np.zeros(1, np.float32),
                               sr_rows=np.zeros((1, 8), np.float32), sh_rows=np.zeros((1, 1, 3), np.float32))
    x = np.zeros((n, 3))
    zero = {"dlogit": np.zeros(1), "d_sr": np.zeros((1, 8)), "d_sh": np.zeros((1, 1, 3))}
    for t in range(steps):
        sc.pos = x
        x = mcmc.sgld_update(sc, {"dpos": x / s2, **zero}, {"pos": eps, "logit": 0, "sr": 0, "sh": 0}, t, 77)["pos"]
    a = 1.0 - eps / (2.0 * s2)
    var = eps * (1.0 - a ** (2 * steps)) / (1.0 - a * a)
    assert abs(x.mean()) < 5 * np.sqrt(var / x.size)
    assert abs(x.var() / var - 1.0) < 5 * np.sqrt(2.0 / x.size)


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, -2.5, 0.0], dtype=np.float64)
    want = np.array([1.0, 1.0, 1.0 + 4 * 2 ** -8, 1.0 + 2 ** -7, -2.5, 0.0], dtype=np.float32)
    assert np.array_equal(mcmc.bf16_rne64(x), want)
    assert np.array_equal(mcmc.bf16_rne(x.astype(np.float32)), want)


# ----------------------------------------------------------------------------
# split and merge
# ----------------------------------------------------------------------------

def _codebook(k, k_cap, width, n, rng, zipf=True):
    rows = np.zeros((k_cap, width), dtype=np.float32)
    rows[:k] = rng.normal(size=(k, width)).astype(np.float32)
    parent = np.full(k_cap, -1, dtype=np.int32)
    g2x = (rng.zipf(1.5, n) - 1) % k if zipf else rng.integers(0, k, n)
    return rows, parent, g2x.astype(np.int64)


@pytest.mark.parametrize("codebook,degree", [(0, 3), (1, 3), (1, 1)])
def test_split_all_then_merge_all_is_identity(codebook, degree):
    rng = np.random.default_rng(3)
    dims, width = mcmc.row_dims(codebook, degree)
    k, n = 40, 500
    rows, parent, g2x = _codebook(k, 2000, width, n, rng)
    sp = mcmc.split(rows, parent, g2x, k, 2000, codebook, degree, lam=-1000.0, eps_split=0.1, eps_merge=0.05,
                    step=11, seed=5)
    members = np.bincount(g2x, minlength=k)
    assert sp["k"] == k + int((members - 1).clip(0).sum())       # every eligible Gaussian split
    moved = np.nonzero(sp["g2x"] != g2x)[0]
    assert np.array_equal(sp["g2x"][moved], k + np.arange(moved.size))
    assert np.array_equal(sp["parent"][k + np.arange(moved.size)], g2x[moved])
    # the new rows are c + eps_split z with the FP64 normals of the same draws
    z64 = np.concatenate([mcmc.normals64(mcmc.draws(np.arange(n), mcmc.STREAM_SPLIT_U + codebook, j, 11, 5))
                          for j in range((dims + 3) // 4)], axis=1)[:, :dims]
    u = sp["rows"][sp["g2x"][moved], :dims].astype(np.float64) - rows[g2x[moved], :dims]
    assert np.all(np.abs(u - 0.1 * z64[moved]) <= 1e-6 * (1 + np.abs(rows[g2x[moved], :dims])))
    assert np.array_equal(sp["rows"][:k], rows[:k])
    # merge everything back: wide merge kernel, strong row penalty
    mg = mcmc.merge(sp["rows"], sp["parent"], sp["g2x"], sp["k"], codebook, degree, lam=100.0, eps_split=0.1,
                    eps_merge=1e3, step=12, seed=5)
    assert mg["k"] == k
    assert np.array_equal(mg["g2x"], g2x)
    assert np.array_equal(mg["rows"][:k], rows[:k])
    assert np.all(mg["parent"][:k] == -1)


def test_split_respects_penalty_eligibility_and_capacity():
    rng = np.random.default_rng(4)
    k, n = 30, 400
    rows, parent, g2x = _codebook(k, 64, 8, n, rng)
    none = mcmc.split(rows, parent, g2x, k, 64, 0, 3, lam=100.0, eps_split=0.1, eps_merge=0.05, step=1, seed=2)
    assert none["k"] == k and np.array_equal(none["g2x"], g2x)
    capped = mcmc.split(rows, parent, g2x, k, k + 3, 0, 3, lam=-100.0, eps_split=0.1, eps_merge=0.05, step=1,
                        seed=2)
    assert capped["k"] == k + 3
    first_three = np.nonzero(capped["proposed_accept"])[0][:3]
    assert np.array_equal(np.nonzero(capped["g2x"] != g2x)[0], first_three)
    # a row keeps its first member; single-member rows never split
    members = np.bincount(g2x, minlength=k)
    first = np.array([np.nonzero(g2x == r)[0][0] if members[r] else -1 for r in range(k)])
    elig = capped["eligible"]
    assert not elig[first[members > 0]].any()
    assert not elig[members[g2x] == 1].any()


def test_split_acceptance_rate_matches_min_one_exp():
    """Fraction of eligible proposals accepted ~ mean of min(1, e^-lambda / q_sm(u))."""
    rng = np.random.default_rng(6)
    k, n = 8, 60_000
    rows, parent, g2x = _codebook(k, 2 * n, 8, n, rng, zipf=False)
    es, em, lam = 0.1, 0.3, 0.2
    sp = mcmc.split(rows, parent, g2x, k, 2 * n, 0, 3, lam=lam, eps_split=es, eps_merge=em, step=2, seed=8)
    z64 = np.concatenate([mcmc.normals64(mcmc.draws(np.arange(n), mcmc.STREAM_SPLIT_U, j, 2, 8))
                          for j in range(2)], axis=1)[:, :7]
    u2 = (es * z64) ** 2
    a = np.minimum(1.0, np.exp(-lam + 0.5 * u2.sum(1) * (1 / es ** 2 - 1 / em ** 2)))
    el = sp["eligible"]
    p = a[el].mean()
    assert abs(sp["accepted"][el].mean() - p) < 5 * np.sqrt(p * (1 - p) / el.sum())


def _paper():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_hyperparameters.json")) as f:
        return json.load(f)


def test_paper_hyperparameters_fixture():
    """The printed values (Sec. 5.1, Sec. 4.4): a probability mixture and the
    split / merge widths with eps_merge < eps_split, the regime in which the
    split kernel q_sm grows with |u| (kc < 0)."""
    hp = _paper()
    assert abs(hp["p_update"] + hp["p_split"] + hp["p_merge"] - 1.0) < 1e-12
    assert hp["eps_merge"] < hp["eps_split"]
    _, kc, km = mcmc._coefs(hp["eps_split"], hp["eps_merge"])
    assert float(kc) == pytest.approx(0.5 * (1 / 0.1 ** 2 - 1 / 0.05 ** 2), rel=1e-6)   # -150
    assert float(km) == pytest.approx(0.5 / 0.05 ** 2, rel=1e-6)                       # 200


def test_split_acceptance_closed_form_at_paper_hyperparameters():
    """With the paper's lambda_SR, eps_split and eps_merge, e^-lambda / q_sm(u)
    = exp(-lambda + kc |u|^2) < 1 for every u (kc < 0), and |u|^2 =
    eps_split^2 chi^2_D, so an eligible proposal is accepted with probability
    e^-lambda E[exp(kc eps_split^2 chi^2_D)] = e^-lambda (1 - 2 kc eps_split^2)^(-D/2)
    (the chi-square moment generating function): e^-3 4^-3.5 = e^-3 / 128 for
    the 7 moved values of an SR row.  The oracle's accepted count must match
    that binomial mean."""
    hp = _paper()
    rng = np.random.default_rng(11)
    k, n = 32, 600_000
    rows, parent, g2x = _codebook(k, k + n, 8, n, rng, zipf=False)
    sp = mcmc.split(rows, parent, g2x, k, k + n, 0, 3, lam=hp["lambda_sr"], eps_split=hp["eps_split"],
                    eps_merge=hp["eps_merge"], step=5, seed=13)
    es, em = hp["eps_split"], hp["eps_merge"]
    kc = 0.5 * (1 / es ** 2 - 1 / em ** 2)
    p = np.exp(-hp["lambda_sr"]) * (1 - 2 * kc * es ** 2) ** (-7 / 2)
    assert p == pytest.approx(np.exp(-3.0) / 128, rel=1e-12)
    el = int(sp["eligible"].sum())
    assert el > n - 2 * k
    got = int(sp["accepted"].sum())
    assert abs(got - el * p) < 5 * np.sqrt(el * p * (1 - p)), (got, el * p)
    # the SH rows' 48 moved values make a split practically impossible at these settings
    p_sh = np.exp(-hp["lambda_sh"]) * (1 - 2 * kc * es ** 2) ** (-48 / 2)
    assert p_sh < 1e-15


def test_merge_closed_form_at_paper_hyperparameters():
    """A row split off its parent by u ~ N(0, eps_split^2 I) (D = 7 moved values)
    is proposed for merging with exp(-km |u|^2) and, with lambda > 0 and
    kc < 0, always accepted (min(1, exp(lambda - kc |u|^2)) = 1); so it merges
    with probability E[exp(-km eps_split^2 chi^2_7)] = (1 + 2 km eps_split^2)^(-7/2)
    = 5^-3.5 at the paper's values (parents that are roots never merge)."""
    hp = _paper()
    rng = np.random.default_rng(12)
    k0, width = 200_000, 8
    rows = np.zeros((2 * k0, width), dtype=np.float32)
    rows[:k0] = rng.normal(size=(k0, width)).astype(np.float32)
    rows[k0:] = rows[:k0]
    rows[k0:, :7] += (hp["eps_split"] * rng.normal(size=(k0, 7))).astype(np.float32)
    parent = np.concatenate([np.full(k0, -1), np.arange(k0)]).astype(np.int32)
    g2x = np.arange(2 * k0)
    mg = mcmc.merge(rows, parent, g2x, 2 * k0, 0, 3, lam=hp["lambda_sr"], eps_split=hp["eps_split"],
                    eps_merge=hp["eps_merge"], step=6, seed=14)
    km = 0.5 / hp["eps_merge"] ** 2
    p = (1 + 2 * km * hp["eps_split"] ** 2) ** (-7 / 2)
    assert p == pytest.approx(5.0 ** -3.5, rel=1e-12)
    got = int(mg["merged"][k0:].sum())
    assert not mg["merged"][:k0].any()
    assert abs(got - k0 * p) < 5 * np.sqrt(k0 * p * (1 - p)), (got, k0 * p)


def test_merge_acceptance_rate_and_parent_rule():
    rng = np.random.default_rng(7)
    k0 = 20_000
    width = 8
    rows = np.zeros((2 * k0, width), dtype=np.float32)
    rows[:k0] = rng.normal(size=(k0, width)).astype(np.float32)
    rows[k0:] = rows[:k0] + rng.normal(0, 0.03, size=(k0, width)).astype(np.float32)
    parent = np.concatenate([np.full(k0, -1), np.arange(k0)]).astype(np.int32)
    g2x = np.arange(2 * k0)
    es, em, lam = 0.1, 0.05, -1.0
    mg = mcmc.merge(rows, parent, g2x, 2 * k0, 0, 3, lam=lam, eps_split=es, eps_merge=em, step=4, seed=1)
    d2 = ((rows[k0:, :7].astype(np.float64) - rows[:k0, :7]) ** 2).sum(1)
    p = np.exp(-d2 / (2 * em ** 2)) * np.minimum(1.0, np.exp(lam + 0.5 * d2 * (1 / em ** 2 - 1 / es ** 2)))
    rate = mg["merged"][k0:].mean()
    assert abs(rate - p.mean()) < 5 * np.sqrt(p.mean() / k0)
    merged = np.nonzero(mg["merged"])[0]
    assert np.array_equal(mg["g2x"][merged], mg["g2x"][parent[merged]])   # members join the parent's row
    assert mg["k"] == 2 * k0 - merged.size

    # chain 0 <- 1 <- 2 with equal rows: 1 merges into 0, 2 waits for its parent
    rows = np.zeros((3, 8), dtype=np.float32)
    mg = mcmc.merge(rows, np.array([-1, 0, 1], np.int32), np.array([0, 1, 2, 2]), 3, 0, 3, lam=50.0,
                    eps_split=0.1, eps_merge=1e3, step=0, seed=0)
    assert mg["k"] == 2
    assert list(mg["merged"]) == [False, True, False]
    assert list(mg["g2x"]) == [0, 0, 1, 1]
    assert list(mg["parent"][:2]) == [-1, 0]


# ----------------------------------------------------------------------------
# reconstruction loss (Eq. 4)
# ----------------------------------------------------------------------------

def test_window_and_moments_match_scipy():
    rng = np.random.default_rng(9)
    x = rng.random((37, 53))
    g = ssim.window1d()
    assert abs(g.sum() - 1.0) < 1e-15 and np.allclose(g, g[::-1], atol=0, rtol=0)
    ref = ndimage.gaussian_filter(x, sigma=1.5, mode="constant", cval=0.0, truncate=5 / 1.5)
    assert np.abs(ssim.windowed(x) - ref).max() < 1e-14
    ref2 = ndimage.correlate(x * x, ssim.window2d(), mode="constant", cval=0.0)
    assert np.abs(ssim.windowed(x * x) - ref2).max() < 1e-14


def test_ssim_identities_and_closed_form():
    rng = np.random.default_rng(10)
    x = rng.random((30, 40))
    y = rng.random((30, 40))
    m = ssim.ssim_maps(x, x)
    assert np.abs(m["s"] - 1.0).max() < 1e-12
    assert np.abs(ssim.ssim_maps(x, y)["s"] - ssim.ssim_maps(y, x)["s"]).max() < 1e-14
    a, b = 0.3, 0.7
    s = ssim.ssim_maps(np.full((30, 40), a), np.full((30, 40), b))["s"]
    interior = s[5:-5, 5:-5]
    assert np.abs(interior - (2 * a * b + ssim.C1) / (a * a + b * b + ssim.C1)).max() < 1e-12
    cam = types.SimpleNamespace(width=40, height=30)
    img = rng.random(3 * 30 * 40)
    r = ssim.recon_loss(img, img, [cam])
    assert abs(r["loss"]) < 1e-12 and np.abs(r["grad"]).max() < 1e-12


def test_recon_loss_gradient_by_finite_differences():
    rng = np.random.default_rng(11)
    cams = [types.SimpleNamespace(width=23, height=17), types.SimpleNamespace(width=9, height=12)]
    m = sum(3 * c.width * c.height for c in cams)
    x = rng.random(m)
    y = np.clip(x + rng.normal(0, 0.2, m), 0, 1)
    r = ssim.recon_loss(x, y, cams, lam=0.2)
    h = 1e-6
    for i in rng.choice(m, 40, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (ssim.recon_loss(xp, y, cams)["loss"] - ssim.recon_loss(xm, y, cams)["loss"]) / (2 * h)
        assert abs(fd - r["grad"][i]) <= 1e-6 * abs(fd) + 1e-9, (i, fd, r["grad"][i])
    assert abs(r["loss"] - (0.8 * np.abs(x - y).mean() + 0.2 * r["l_ssim"])) < 1e-15


# ----------------------------------------------------------------------------
# growth
# ----------------------------------------------------------------------------

def test_growth_copies_gaussians_in_proportion_to_opacity():
    rng = np.random.default_rng(12)
    n = 50
    logit = rng.normal(0, 2, n).astype(np.float32)
    pos = rng.normal(size=(n, 3)).astype(np.float32)
    g2sr = rng.integers(0, 9, n).astype(np.uint16)
    g2sh = rng.integers(0, 9, n).astype(np.uint16)
    out = mcmc.grow(pos, logit, g2sr, g2sh, 200_000, step=3, seed=4)
    src = out["src"]
    assert src.min() >= 0 and src.max() < n
    # copies are exact
    assert np.array_equal(out["pos"][n:], pos[src]) and np.array_equal(out["g2sh"][n:], g2sh[src])
    assert np.array_equal(out["pos"][:n], pos) and np.array_equal(out["logit"][n:], logit[src])
    # frequencies follow the opacities (chi-square against o / sum o)
    o = 1.0 / (1.0 + np.exp(-logit.astype(np.float64)))
    expected = o / o.sum() * src.size
    observed = np.bincount(src, minlength=n)
    assert stats.chisquare(observed, expected).pvalue > 1e-3
    # the FP32 opacity equals the FP64 sigmoid to a few ulp
    assert np.abs(mcmc.sigmoid32(logit) - o).max() < 1e-6
    # deterministic, and another step draws other copies
    again = mcmc.grow(pos, logit, g2sr, g2sh, 200_000, step=3, seed=4)["src"]
    other = mcmc.grow(pos, logit, g2sr, g2sh, 200_000, step=4, seed=4)["src"]
    assert np.array_equal(src, again) and not np.array_equal(src, other)
    # every weight 0: uniform choice
    flat = mcmc.grow(pos, np.full(n, -200.0, np.float32), g2sr, g2sh, 100_000, step=1, seed=1)["src"]
    assert stats.chisquare(np.bincount(flat, minlength=n)).pvalue > 1e-3
