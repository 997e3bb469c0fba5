"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, library routines, invariants, brute force and finite
differences.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_03775_gb300 import scenes

# ---------------------------------------------------------------------------
# exp of the FP32 decision arithmetic
# ---------------------------------------------------------------------------


def test_e32_accuracy_and_range():
    x = np.concatenate([np.linspace(-86.9, 87.9, 20001, dtype=np.float32),
                        np.float32([-5.5, -1e-3, 0.0, 1e-3, 0.5, 1.0])])
    got = oracle.e32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    rel = np.abs(got - ref) / ref
    # the Taylor truncation (< 1.3e-7) plus a few roundings
    assert rel.max() < 4e-7, rel.max()
    assert oracle.e32([0.0])[0] == 1.0
    assert oracle.e32([-87.0])[0] == 0.0 and oracle.e32([-1000.0])[0] == 0.0
    assert np.isinf(oracle.e32([88.0])[0]) and np.isinf(oracle.e32([1e9])[0])
    assert oracle.e32([np.nan])[0] == 0.0


# ---------------------------------------------------------------------------
# SH basis (colour of Sec. 2.1, SH codebook rows of Sec. 4.1)
# ---------------------------------------------------------------------------


def _real_sh_scipy(l, m, theta, phi):
    """Real SH from scipy's complex SH (Condon-Shortley phase included):
    sqrt(2) Re Y_l^m for m > 0, sqrt(2) Im Y_l^|m| for m < 0."""
    from scipy.special import sph_harm_y
    if m > 0:
        return math.sqrt(2) * sph_harm_y(l, m, theta, phi).real
    if m < 0:
        return math.sqrt(2) * sph_harm_y(l, -m, theta, phi).imag
    return sph_harm_y(l, 0, theta, phi).real


def test_sh_basis_matches_scipy():
    pytest.importorskip("scipy")
    rng = np.random.default_rng(0)
    for _ in range(50):
        theta, phi = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)
        d = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
        Y, _ = oracle.sh_basis(3, d)
        k = 0
        for l in range(4):
            for m in range(-l, l + 1):
                assert abs(Y[k] - _real_sh_scipy(l, m, theta, phi)) < 1e-12, (l, m)
                k += 1


def test_sh_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for degree <= 6 products
    nodes, weights = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for z, wz in zip(nodes, weights):
        s = math.sqrt(1 - z * z)
        for j in range(nphi):
            phi = 2 * math.pi * j / nphi
            Y, _ = oracle.sh_basis(3, [s * math.cos(phi), s * math.sin(phi), z])
            G += np.outer(Y, Y) * wz * (2 * math.pi / nphi)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_basis_derivative_fd():
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.normal(size=3)
        _, dY = oracle.sh_basis(3, d)
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1e-6
            fd = (oracle.sh_basis(3, d + e)[0] - oracle.sh_basis(3, d - e)[0]) / 2e-6
            assert np.abs(fd - dY[:, a]).max() < 1e-7


def test_sh_consts32_are_rounded_closed_forms():
    k = oracle.sh_consts32()
    pi = math.pi
    ref = [0.5 / math.sqrt(pi), -math.sqrt(3 / (4 * pi)), math.sqrt(3 / (4 * pi)), -math.sqrt(3 / (4 * pi)),
           math.sqrt(15 / (4 * pi)), -math.sqrt(15 / (4 * pi)), math.sqrt(5 / (16 * pi)),
           -math.sqrt(15 / (4 * pi)), math.sqrt(15 / (16 * pi)), -math.sqrt(35 / (32 * pi)),
           math.sqrt(105 / (4 * pi)), -math.sqrt(21 / (32 * pi)), math.sqrt(7 / (16 * pi)),
           -math.sqrt(21 / (32 * pi)), math.sqrt(105 / (16 * pi)), -math.sqrt(35 / (32 * pi))]
    assert np.array_equal(k, np.float32(ref))


# ---------------------------------------------------------------------------
# Eq. 2: Sigma = R(q) S S^T R(q)^T
# ---------------------------------------------------------------------------


def test_sigma_identity_quaternion_is_diagonal():
    ls = np.array([-1.0, 0.3, -2.5])
    s6 = oracle.sr_sigma([*ls, 1.0, 0.0, 0.0, 0.0])
    assert np.allclose(oracle.full3(s6), np.diag(np.exp(2 * ls)), rtol=1e-14, atol=0)


def test_sigma_equal_scales_is_rotation_invariant():
    rng = np.random.default_rng(2)
    for _ in range(20):
        q = rng.normal(size=4)
        s6 = oracle.sr_sigma([-0.7, -0.7, -0.7, *q])
        assert np.allclose(oracle.full3(s6), math.exp(-1.4) * np.eye(3), rtol=1e-13, atol=1e-15)


def test_sigma_matches_scipy_rotation_and_quaternion_scale():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.normal(size=4)
        ls = rng.normal(-2, 0.5, size=3)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy order x y z w
        ref = R @ np.diag(np.exp(2 * ls)) @ R.T
        s6 = oracle.sr_sigma([*ls, *q])
        assert np.allclose(oracle.full3(s6), ref, rtol=1e-12, atol=1e-16)
        s6b = oracle.sr_sigma([*ls, *(3.7 * q)])
        assert np.allclose(s6, s6b, rtol=1e-13, atol=1e-18)


def test_sigma32_close_to_fp64():
    rng = np.random.default_rng(4)
    for _ in range(200):
        row = np.float32([*rng.normal(-3, 0.5, 3), *rng.normal(size=4)])
        a = oracle.sr_sigma32(row).astype(np.float64)
        b = oracle.sr_sigma(row.astype(np.float64))
        scale = np.abs(b).max()
        assert np.abs(a - b).max() < 2e-6 * scale


def test_sigma_backward_fd():
    rng = np.random.default_rng(5)
    for _ in range(10):
        row = np.array([*rng.normal(-2, 0.5, 3), *rng.normal(size=4)])
        g = rng.normal(size=6)
        an = oracle.sr_sigma_backward(row, g)
        for e in range(7):
            d = np.zeros(7)
            d[e] = 1e-6
            fd = (g @ oracle.sr_sigma(row + d) - g @ oracle.sr_sigma(row - d)) / 2e-6
            assert abs(fd - an[e]) < 1e-6 * max(1.0, abs(an[e])), (e, fd, an[e])


# ---------------------------------------------------------------------------
# projection (EWA) and the closed-form isotropic image
# ---------------------------------------------------------------------------


def _single_scene(p, ls, logit, dc_rgb, degree=0):
    nb = (degree + 1) ** 2
    sh = np.zeros((1, nb, 3), dtype=np.float32)
    c0 = 0.5 / math.sqrt(math.pi)
    sh[0, 0, :] = (np.asarray(dc_rgb) - 0.5) / c0
    sr = np.zeros((1, 8), dtype=np.float32)
    sr[0, :3] = ls
    sr[0, 3] = 1.0
    return scenes.Scene(pos=np.float32([p]), opacity_logit=np.float32([logit]),
                        g2sr=np.zeros(1, np.uint16), g2sh=np.zeros(1, np.uint16),
                        sr_rows=sr, sh_rows=sh, sh_degree=degree)


def _axis_camera(width=64, height=64, z_eye=-3.0):
    return scenes.look_at([0.0, 0.0, z_eye], width, height)


def test_isotropic_on_axis_covariance_closed_form():
    cam = _axis_camera()
    s = math.exp(-2.5)
    sc = _single_scene([0.0, 0.0, 0.0], [math.log(s)] * 3, 0.0, [0.7, 0.2, 0.4])
    r = oracle.Render(sc, [cam])
    rec = r.rec64[0]
    z = 3.0
    f = cam.fx
    var = (f * s / z) ** 2 + 0.3
    assert np.allclose(rec["cov"], [var, 0.0, var], rtol=1e-6, atol=1e-9)
    assert np.allclose(rec["mean"], [cam.cx, cam.cy], atol=1e-5)
    assert abs(rec["t"][2] - z) < 1e-6


def test_isotropic_single_gaussian_image_closed_form():
    cam = _axis_camera(96, 80)
    s = math.exp(-3.0)
    logit = 1.2
    rgb = np.array([0.9, 0.3, 0.55])
    sc = _single_scene([0.0, 0.0, 0.0], [math.log(s)] * 3, logit, rgb)
    bg = np.array([0.1, 0.2, 0.3])
    r = oracle.Render(sc, [cam], bg=bg)
    q = r.rec32[0]
    rec = r.rec64[0]
    sig2 = rec["cov"][0]
    o = 1 / (1 + math.exp(-logit))
    img = r.view_image(0)
    H, W = cam.height, cam.width
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (rec["mean"][0] - (xs + 0.5)) ** 2 + (rec["mean"][1] - (ys + 0.5)) ** 2
    alpha = np.minimum(0.99, o * np.exp(-0.5 * d2 / sig2))
    tile = 16
    inside = ((xs // tile >= q["x0"]) & (xs // tile < q["x1"]) & (ys // tile >= q["y0"]) & (ys // tile < q["y1"]))
    alpha = np.where(inside & (alpha >= 1 / 255), alpha, 0.0)
    for c in range(3):
        ref = alpha * rgb[c] + (1 - alpha) * bg[c]
        assert np.abs(img[c] - ref).max() < 1e-5
    # the 3-sigma rectangle of an on-axis isotropic Gaussian is centred
    rad = math.ceil(3 * math.sqrt(sig2))
    assert q["x0"] == max(0, math.floor((rec["mean"][0] - rad) / tile))


def test_projection_jacobian_and_covariance_by_sampling():
    """Sigma_2D - 0.3 I must be the covariance of the exact pinhole image of
    a small 3D Gaussian (first-order), checked by sampling the pinhole map."""
    rng = np.random.default_rng(6)
    cam = scenes.look_at([1.0, -0.5, -3.0], 200, 160)
    p = np.array([0.3, -0.2, 0.1])
    row = np.array([-4.5, -5.0, -4.2, *rng.normal(size=4)])
    sc = scenes.Scene(pos=np.float32([p]), opacity_logit=np.float32([0.0]), g2sr=np.zeros(1, np.uint16),
                      g2sh=np.zeros(1, np.uint16), sr_rows=np.float32([row]),
                      sh_rows=np.zeros((1, 1, 3), np.float32), sh_degree=0)
    r = oracle.Render(sc, [cam])
    rec = r.rec64[0]
    Sigma = oracle.full3(oracle.sr_sigma(row.astype(np.float32).astype(np.float64)))
    x = rng.multivariate_normal(sc.pos[0].astype(np.float64), Sigma, size=400_000)
    W = cam.world_to_cam.astype(np.float64)
    t = x @ W[:, :3].T + W[:, 3]
    u = cam.fx * t[:, 0] / t[:, 2] + cam.cx
    v = cam.fy * t[:, 1] / t[:, 2] + cam.cy
    emp = np.cov(np.stack([u, v]))
    model = np.array([[rec["cov"][0] - 0.3, rec["cov"][1]], [rec["cov"][1], rec["cov"][2] - 0.3]])
    assert np.allclose(emp, model, rtol=0.02, atol=0.02 * np.abs(model).max())
    assert abs(u.mean() - rec["mean"][0]) < 0.05 and abs(v.mean() - rec["mean"][1]) < 0.05


# ---------------------------------------------------------------------------
# Eq. 3: compositing invariants and hand-computed sums
# ---------------------------------------------------------------------------


def _white_scene(base):
    sc = base.copy()
    nb = (sc.sh_degree + 1) ** 2
    sh = np.zeros((sc.k_sh, nb, 3), dtype=np.float32)
    sh[:, 0, :] = 0.5 / (0.5 / math.sqrt(math.pi))
    sc.sh_rows = sh
    return sc


@pytest.mark.parametrize("mode", [0, 1])
def test_transmittance_invariant(mode):
    sc, cams, _ = scenes.config_tiny()
    w = _white_scene(sc)
    r1 = oracle.Render(w, cams, bg=(1, 1, 1), mode=mode)
    # every colour is the same value white = 0.5 + C0 * fl32(0.5 / C0), 1 up to FP32 storage
    white = r1.rec64["rgb"][r1.rec32["visible"].astype(bool)][0]
    assert np.allclose(r1.rec64["rgb"][r1.rec32["visible"].astype(bool)], white, rtol=0, atol=0)
    assert np.abs(white - 1).max() < 1e-7
    img1 = r1.image.reshape(3, -1)
    for c in range(3):
        # sum_k alpha_k T_k + T_final telescopes to 1
        assert np.abs(img1[c] - (1.0 + (white[c] - 1.0) * (1.0 - r1.t_final))).max() < 1e-12
    r0 = oracle.Render(w, cams, bg=(0, 0, 0), mode=mode)
    for c in range(3):
        assert np.abs(r0.image.reshape(3, -1)[c] - white[c] * (1 - r0.t_final)).max() < 1e-12
    if mode == 0:
        assert r0.t_final.min() >= 1e-4 * (1 - 1e-6)


def test_three_gaussians_on_axis_by_hand():
    cam = _axis_camera(32, 32)
    pos = [[0.0, 0.0, -1.0], [0.0, 0.0, 0.0], [0.0, 0.0, 1.0]]   # depths 2, 3, 4
    ls = [-2.0, -2.3, -1.8]
    logits = [-0.5, 0.4, 1.5]
    cols = [[0.9, 0.1, 0.2], [0.2, 0.8, 0.3], [0.1, 0.3, 0.95]]
    c0 = 0.5 / math.sqrt(math.pi)
    sh = np.zeros((3, 1, 3), np.float32)
    sr = np.zeros((3, 8), np.float32)
    for i in range(3):
        sh[i, 0] = (np.asarray(cols[i]) - 0.5) / c0
        sr[i, :3] = ls[i]
        sr[i, 3] = 1.0
    order = [2, 0, 1]   # list order in the arrays is not depth order
    sc = scenes.Scene(pos=np.float32(pos)[order], opacity_logit=np.float32(logits)[order],
                      g2sr=np.uint16(order), g2sh=np.uint16(order), sr_rows=sr, sh_rows=sh, sh_degree=0)
    for mode in (0, 1):
        r = oracle.Render(sc, [cam], mode=mode)
        img = r.view_image(0)
        x = y = 16
        C = np.zeros(3)
        T = 1.0
        for i in range(3):     # front to back: depths 2, 3, 4
            z = 3.0 + pos[i][2]
            sig2 = (cam.fx * math.exp(ls[i]) / z) ** 2 + 0.3
            d2 = (cam.cx - (x + 0.5)) ** 2 + (cam.cy - (y + 0.5)) ** 2
            a = 1 / (1 + math.exp(-logits[i])) * math.exp(-0.5 * d2 / sig2)
            if mode == 0:
                a = min(a, 0.99)
            C += a * T * np.asarray(cols[i])
            T *= 1 - a
        assert np.abs(img[:, y, x] - C).max() < 1e-6


# ---------------------------------------------------------------------------
# tiles, lists and order vs a brute-force renderer without tiles
# ---------------------------------------------------------------------------


def _brute_force(r):
    """Eq. 3 per pixel over every visible record whose rectangle holds the
    pixel's tile, ordered by (FP32 depth bits, record index); FP64; mode 1."""
    out = np.zeros_like(r.image)
    q, rec = r.rec32, r.rec64
    for v, cam in enumerate(r.cams):
        ids = np.nonzero(q["visible"][v * r.n:(v + 1) * r.n])[0] + v * r.n
        order = ids[np.lexsort((ids, q["depth_bits"][ids]))]
        H, W = cam.height, cam.width
        ys, xs = np.mgrid[0:H, 0:W]
        tx, ty = xs // r.tile, ys // r.tile
        C = np.zeros((3, H, W))
        T = np.ones((H, W))
        for rid in order:
            inside = (tx >= q["x0"][rid]) & (tx < q["x1"][rid]) & (ty >= q["y0"][rid]) & (ty < q["y1"][rid])
            dx = rec["mean"][rid][0] - (xs + 0.5)
            dy = rec["mean"][rid][1] - (ys + 0.5)
            c = rec["conic"][rid]
            a = rec["opacity"][rid] * np.exp(-0.5 * (c[0] * dx * dx + c[2] * dy * dy) - c[1] * dx * dy)
            a = np.where(inside, a, 0.0)
            C += a * T * rec["rgb"][rid][:, None, None]
            T *= 1 - a
        b = 3 * r.pix_base[v]
        out[b:b + 3 * H * W] = (C + T * r.bg[:, None, None]).ravel()
    return out


def test_tiled_equals_brute_force():
    sc, cams, _ = scenes.config_tiny()
    cam2 = scenes.look_at([2.2, 1.0, 1.5], 72, 40)
    r = oracle.Render(sc, [cams[0], cam2], mode=1, bg=(0.2, 0.1, 0.05))
    assert np.abs(r.image - _brute_force(r)).max() < 1e-12


def test_lists_sorted_and_ranges_consistent():
    sc, cams, _ = scenes.config_tiny()
    r = oracle.Render(sc, cams)
    keys = r.keys
    assert np.all(keys[1:] >= keys[:-1])
    tiles = keys >> np.uint64(32)
    for gt in range(r.n_tiles):
        b, e = r.ranges[gt]
        assert np.all(tiles[b:e] == gt)
    assert int((r.ranges[:, 1] - r.ranges[:, 0]).sum()) == r.k_pairs
    # pairs of a tile are exactly the visible records whose rectangle holds it
    # and that pass the tile test
    q = r.rec32
    for gt in [0, 17, 35, 63]:
        ty, tx = divmod(gt, r.tiles_x[0])
        cand = np.nonzero(q["visible"].astype(bool) & (q["x0"] <= tx) & (q["x1"] > tx) &
                          (q["y0"] <= ty) & (q["y1"] > ty))[0]
        want = [int(i) for i in cand if oracle.tile_keep32(*[float(q[f][i]) for f in ("mx", "my", "h0", "h1", "h2", "o")],
                                                              tx, ty, 16)]
        assert sorted(r.tile_list(gt).tolist()) == want


def test_fp32_rects_agree_with_fp64_rects():
    """The FP32 decision rectangle equals the 3-sigma rectangle computed in
    FP64 except where FP64 sits within rounding of a ceil / floor edge."""
    sc, cams = scenes.config_single(n=20_000, k=512, width=320, height=240)
    r = oracle.Render(sc, cams)
    rec, q = r.rec64, r.rec32
    vis = q["visible"].astype(bool)
    a, b, c = rec["cov"][:, 0], rec["cov"][:, 1], rec["cov"][:, 2]
    mid = 0.5 * (a + c)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - (a * c - b * b)))
    rad = np.ceil(3 * np.sqrt(lam))
    x0 = np.clip(np.floor((rec["mean"][:, 0] - rad) / 16), 0, r.tiles_x[0])
    x1 = np.clip(np.floor((rec["mean"][:, 0] + rad + 15) / 16), 0, r.tiles_x[0])
    same = (x0 == q["x0"]) & (x1 == q["x1"])
    assert same[vis].mean() > 0.999
    assert vis.sum() > 10_000


# ---------------------------------------------------------------------------
# backward: central finite differences of the FP64 forward under fixed
# decisions (the render is piecewise smooth; its decisions are piecewise
# constant)
# ---------------------------------------------------------------------------


def _as64(s):
    s = s.copy()
    s.pos = s.pos.astype(np.float64)
    s.opacity_logit = s.opacity_logit.astype(np.float64)
    s.sr_rows = s.sr_rows.astype(np.float64)
    s.sh_rows = s.sh_rows.astype(np.float64)
    return s


def _fd_check(r, sc64, w, grads, params, h=1e-5, rtol=1e-5):
    def L(img):
        return float(w @ img)

    # rounding noise of the FP64 loss, divided by the step
    atol = 64 * np.finfo(np.float64).eps * float(np.abs(w) @ np.abs(r.image)) / (2 * h)

    for kind, idx in params:
        def run(sign):
            s = sc64.copy()
            arr = {"pos": s.pos, "logit": s.opacity_logit, "sr": s.sr_rows, "sh": s.sh_rows}[kind]
            arr[idx] += sign * h
            return L(r.replay(s))

        fd = (run(+1) - run(-1)) / (2 * h)
        an = {"pos": grads["dpos"], "logit": grads["dlogit"], "sr": grads["d_sr"], "sh": grads["d_sh"]}[kind][idx]
        assert abs(fd - an) <= rtol * abs(an) + atol, (kind, idx, fd, an)


@pytest.mark.parametrize("mode", [0, 1])
def test_backward_matches_finite_differences_tiny(mode):
    sc, cams, _ = scenes.config_tiny()
    r = oracle.Render(sc, cams, mode=mode, bg=(0.3, 0.2, 0.1))
    rng = np.random.default_rng(7)
    w = rng.normal(size=r.image.shape)
    grads = r.backward(w)
    vis = np.nonzero(r.rec32["visible"])[0]
    params = []
    for g in rng.choice(vis, 6, replace=False):
        params += [("pos", (g, a)) for a in range(3)] + [("logit", g)]
    for k in rng.choice(np.unique(sc.g2sr[vis]), 3, replace=False):
        params += [("sr", (k, e)) for e in range(7)]
    for k in rng.choice(np.unique(sc.g2sh[vis]), 2, replace=False):
        params += [("sh", (k, b, c)) for b in range(4) for c in range(3)]
    _fd_check(r, _as64(sc), w, grads, params)


def test_backward_matches_finite_differences_two_views_degree3():
    sc, _ = scenes.config_single(n=3000, k=64, width=96, height=80)
    cams = [scenes.look_at([0.5, -0.8, -2.8], 96, 80), scenes.look_at([-2.5, 0.4, 1.2], 64, 48)]
    r = oracle.Render(sc, cams, bg=(0.0, 0.5, 1.0))
    rng = np.random.default_rng(8)
    w = rng.normal(size=r.image.shape)
    grads = r.backward(w)
    vis = np.nonzero(r.rec32["visible"][:sc.n] & r.rec32["visible"][sc.n:])[0]
    params = []
    for g in rng.choice(vis, 4, replace=False):
        params += [("pos", (g, a)) for a in range(3)] + [("logit", g)]
    for k in rng.choice(np.unique(sc.g2sr), 2, replace=False):
        params += [("sr", (k, e)) for e in range(7)]
    for k in rng.choice(np.unique(sc.g2sh), 1, replace=False):
        params += [("sh", (k, b, c)) for b in range(16) for c in range(3)]
    _fd_check(r, _as64(sc), w, grads, params)


# ---------------------------------------------------------------------------
# codebook reduction: sums over the Gaussians that index a row
# ---------------------------------------------------------------------------


def test_codebook_reduce_identity_total_and_general():
    sc, cams, _ = scenes.config_tiny()
    rng = np.random.default_rng(9)
    r = oracle.Render(sc, cams)
    w = rng.normal(size=r.image.shape)
    g = r.backward(w)
    n, nb = sc.n, 4
    # general mapping: plain scatter-add of the per-Gaussian terms
    d_sr, d_sh = oracle.codebook_reduce(sc, r.rec64, g["dsigma"], g["drgb"], 1)
    Y = np.stack([oracle.sh_basis(1, d)[0] for d in r.rec64["dir"]])
    ref_sh = np.zeros((sc.k_sh, nb, 3))
    np.add.at(ref_sh, sc.g2sh.astype(np.int64), Y[:, :, None] * g["drgb"][:, None, :])
    assert np.allclose(d_sh, ref_sh, rtol=1e-12, atol=1e-14)
    sum_sig = np.zeros((sc.k_sr, 6))
    np.add.at(sum_sig, sc.g2sr.astype(np.int64), g["dsigma"])
    ref_sr = np.stack([oracle.sr_sigma_backward(sc.sr_rows[k].astype(np.float64), sum_sig[k])
                       for k in range(sc.k_sr)])
    assert np.allclose(d_sr, ref_sr, rtol=1e-12, atol=1e-14)
    # K = N identity mapping: each row's gradient is its own Gaussian's
    ident = sc.copy()
    ident.g2sr = np.arange(n, dtype=np.uint16)
    ident.g2sh = np.arange(n, dtype=np.uint16)
    ident.sr_rows = sc.sr_rows[sc.g2sr]
    ident.sh_rows = sc.sh_rows[sc.g2sh]
    ri = oracle.Render(ident, cams)
    gi = ri.backward(w)
    assert np.array_equal(ri.image, r.image)
    assert np.allclose(gi["d_sh"], Y[:, :, None] * g["drgb"][:, None, :], rtol=1e-12, atol=1e-14)
    own_sr = np.stack([oracle.sr_sigma_backward(ident.sr_rows[i].astype(np.float64), g["dsigma"][i])
                       for i in range(n)])
    assert np.allclose(gi["d_sr"], own_sr, rtol=1e-12, atol=1e-14)
    # K = 1: the row gradient is the total
    one = sc.copy()
    one.g2sh = np.zeros(n, dtype=np.uint16)
    one.sh_rows = sc.sh_rows[:1]
    _, d_sh_1 = oracle.codebook_reduce(one, r.rec64, g["dsigma"], g["drgb"], 1)
    assert np.allclose(d_sh_1[0], (Y[:, :, None] * g["drgb"][:, None, :]).sum(0), rtol=1e-12, atol=1e-14)


def test_tile_test_drops_only_pairs_every_pixel_skips():
    """Listing a Gaussian only in the tiles where alpha >= 1/255 is reachable
    leaves the image, the final transmittance and every gradient unchanged,
    bit for bit (each dropped pair was skipped by every pixel of its tile),
    while dropping a good share of the pairs."""
    sc, cams = scenes.config_single(n=20_000, k=512, width=240, height=160)
    a = oracle.Render(sc, cams, bg=(0.2, 0.3, 0.4), cull=True)
    b = oracle.Render(sc, cams, bg=(0.2, 0.3, 0.4), cull=False)
    assert a.k_pairs < 0.9 * b.k_pairs
    assert np.array_equal(a.image, b.image)
    assert np.array_equal(a.t_final, b.t_final)
    w = np.random.default_rng(12).normal(size=a.image.shape)
    ga, gb = a.backward(w), b.backward(w)
    for k in ("dpos", "dlogit", "d_sr", "d_sh"):
        assert np.allclose(ga[k], gb[k], rtol=1e-13, atol=1e-18), k


def test_stop_positions_bound_the_lists():
    """Where a pixel stops compositing (its transmittance would fall below
    the floor), nothing later in its tile's list can change it: rendering
    with every tile's list cut right after the last stop of its pixels, for
    the tiles whose pixels all stop, gives bit-identical image, final
    transmittance and contributor counts.  Stops follow the last
    contributor; pixels that never stop keep their full lists."""
    sc, cams = scenes.config_single(n=20_000, k=256, width=96, height=80)
    r = oracle.Render(sc, cams)
    stop = r.term_pos
    assert np.all((stop == -1) | (stop >= r.n_contrib))
    assert (stop >= 0).mean() > 0.2          # enough stopped pixels for the cut to bite
    cut = r.ranges.astype(np.int64).copy()
    cam = cams[0]
    tx = -(-cam.width // 16)
    st = stop.reshape(cam.height, cam.width)
    shortened = 0
    for gt in range(r.n_tiles):
        ty, txx = divmod(gt, tx)
        blk = st[16 * ty:16 * ty + 16, 16 * txx:16 * txx + 16]
        if np.all(blk >= 0):
            new_end = cut[gt, 0] + int(blk.max()) + 1
            shortened += int(cut[gt, 1] - new_end)
            cut[gt, 1] = new_end
    assert shortened > 0
    image = np.zeros(3 * r.P)
    t_final = np.zeros(r.P)
    n_contrib = np.zeros(r.P, dtype=np.int32)
    stop2 = np.zeros(r.P, dtype=np.int32)
    ranges = np.ascontiguousarray(cut.astype(np.uint32))
    _p = oracle._ptr
    oracle.lib().or_blend_forward(r._c, r.V, r.tile, _p(r.bg), r.mode, _p(r.rec32), _p(r.rec64), _p(r.list),
                                  _p(ranges), None, _p(image), _p(t_final), _p(n_contrib), _p(stop2))
    assert np.array_equal(image, r.image)
    assert np.array_equal(t_final, r.t_final)
    assert np.array_equal(n_contrib, r.n_contrib)
    assert np.array_equal(stop2, stop)
