"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names what it pins and why a plausible mistake would fail it.
No GPU, no CUDA library.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_03207_gb300 import synthetic as S

C0 = 0.5 / math.sqrt(math.pi)


def _scene(n, means, log_scales, quats=None, logits=None, sh=None):
    quats = np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None else quats
    logits = np.full(n, 2.0) if logits is None else logits
    if sh is None:
        sh = np.zeros((n, 16, 3))
        sh[:, 0, :] = 0.5 / C0  # colour exactly 1 in every channel
    return {"means": np.asarray(means, float).reshape(n, 3),
            "log_scales": np.asarray(log_scales, float).reshape(n, 3),
            "quats": np.asarray(quats, float).reshape(n, 4),
            "opacity_logits": np.asarray(logits, float).reshape(n), "sh": np.asarray(sh, float)}


def _cam(w=64, h=64, f=64.0, viewmat=None, bg=(0.0, 0.0, 0.0)):
    vm = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], float) if viewmat is None else viewmat
    return {"viewmat": vm, "fx": f, "fy": f, "cx": w / 2, "cy": h / 2, "width": w, "height": h,
            "znear": 0.2, "bg": bg}


# ------------------------------------------------------------------ SH (§2.1)

def _sphere_quadrature(nz=8, nphi=16):
    z, wz = np.polynomial.legendre.leggauss(nz)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    pts, wts = [], []
    for zi, wi in zip(z, wz):
        st = math.sqrt(1 - zi * zi)
        for p in phi:
            pts.append((st * math.cos(p), st * math.sin(p), zi))
            wts.append(wi * 2 * np.pi / nphi)
    return np.array(pts), np.array(wts)


def test_sh_orthonormal_exact_quadrature():
    """The 16 basis functions are orthonormal on the sphere. Gauss-Legendre in
    cos(theta) x uniform phi integrates their products exactly; a wrong
    normalisation constant, factorial or recurrence breaks this."""
    pts, wts = _sphere_quadrature()
    Y = np.array([oracle.sh_basis(p) for p in pts])
    gram = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_addition_theorem():
    """Addition theorem: sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every direction
    and band (so every band is complete and rotation invariant)."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y = oracle.sh_basis(d)
        for l in range(4):
            band = Y[l * l:(l + 1) * (l + 1)]
            assert abs(np.sum(band ** 2) - (2 * l + 1) / (4 * math.pi)) < 1e-12


def test_sh_pole_values_and_phase_convention():
    """At d = +z only m = 0 survives with value sqrt((2l+1)/4pi). The
    Condon-Shortley phase makes the l = 1 functions -y, z, -x (3DGS/PLY
    coefficient convention)."""
    Y = oracle.sh_basis([0, 0, 1])
    for l in range(4):
        for m in range(-l, l + 1):
            expect = math.sqrt((2 * l + 1) / (4 * math.pi)) if m == 0 else 0.0
            assert abs(Y[l * l + l + m] - expect) < 1e-14
    k1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(oracle.sh_basis([1, 0, 0])[1:4], [0, 0, -k1], atol=1e-14)
    np.testing.assert_allclose(oracle.sh_basis([0, 1, 0])[1:4], [-k1, 0, 0], atol=1e-14)


def test_sh_cartesian_form_matches_definition_and_gradient():
    """The Cartesian polynomials used by the backward equal the Legendre
    definition on the sphere, and their gradients match central differences."""
    rng = np.random.default_rng(12)
    for _ in range(40):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        y_def = oracle.sh_basis(d)
        y_cart, g = oracle.sh_basis_cart(d)
        np.testing.assert_allclose(y_cart, y_def, atol=1e-13)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (oracle.sh_basis_cart(d + e)[0] - oracle.sh_basis_cart(d - e)[0]) / (2 * h)
            np.testing.assert_allclose(g[:, a], fd, atol=1e-8)


def _odd_band_terms(d):
    """A few real SH functions with the Condon-Shortley phase, typed from the
    textbook Cartesian table (not from the oracle): l = 1, m = +1 and -1;
    l = 3, m = -3, 0, +3. Index l^2 + l + m."""
    x, y, z = d
    k1 = math.sqrt(3 / (4 * math.pi))
    k33 = math.sqrt(35 / (32 * math.pi))
    k30 = math.sqrt(7 / (16 * math.pi))
    return {3: -k1 * x, 1: -k1 * y,
            9: -k33 * y * (3 * x * x - y * y), 12: k30 * z * (2 * z * z - 3 * x * x - 3 * y * y),
            15: -k33 * x * (x * x - 3 * y * y)}


def test_sh_colour_uses_direction_from_camera_centre():
    """§2.1 colours a splat with SH(k, d), d the unit vector from the camera
    centre to the splat's mean. The eye position is taken from the test (not
    from the view matrix) and the colour is compared with 1/2 + sum k Y(d) for
    splats behind, in front of and beside the look-at target, with only odd-band
    coefficients set. A wrong camera centre (e.g. t instead of -R^T t) or a
    reversed d (which negates every odd band) moves each channel by far more
    than the tolerance; the test also checks that on its own expected values."""
    rng = np.random.default_rng(21)
    eyes = [(6.0, -4.0, 3.0), (-5.0, 7.0, -2.0), (0.5, -8.0, 6.0)]
    target = np.array([0.3, -0.2, 0.4])
    # channel 0: l=1 m=+1; channel 1: l=3 m=-3 and l=1 m=-1; channel 2: l=3 m=0 and m=+3
    chan_terms = {0: (3,), 1: (9, 1), 2: (12, 15)}
    for eye in eyes:
        eye = np.array(eye)
        cam = S.look_at_camera(eye, target, 96, 96, fov_x_deg=50.0)
        fwd = (target - eye) / np.linalg.norm(target - eye)
        right = np.cross(fwd, [0.0, 0.0, 1.0])
        right /= np.linalg.norm(right)
        means = np.stack([target + 0.6 * fwd, target - 0.6 * fwd, target + 0.6 * right,
                          target - 0.4 * right + 0.3 * fwd])
        n = means.shape[0]
        sh = np.zeros((n, 16, 3))
        for ch, idx in chan_terms.items():
            for k in idx:
                # |sum| < 1/2, so no channel reaches the clamp at 0
                sh[:, k, ch] = rng.uniform(0.2, 0.45, n) * rng.choice([-1.0, 1.0], n)
        p = oracle.preprocess(_scene(n, means, np.full((n, 3), -4.0), sh=sh), cam)
        assert list(p["reason"]) == [0] * n
        for i in range(n):
            d = means[i] - eye
            d /= np.linalg.norm(d)
            Y, Yrev = _odd_band_terms(d), _odd_band_terms(-d)
            wrong = means[i] - cam["viewmat"][:, 3].astype(float)  # t_v mistaken for the centre
            Ybad = _odd_band_terms(wrong / np.linalg.norm(wrong))
            for ch, idx in chan_terms.items():
                s = sum(sh[i, k, ch] * Y[k] for k in idx)
                expect = max(0.0, 0.5 + s)
                assert abs(p["rgb"][i, ch] - expect) < 1e-6, (eye, i, ch)
                # the pin is discriminating: the mistaken directions give other colours
                rev = max(0.0, 0.5 + sum(sh[i, k, ch] * Yrev[k] for k in idx))
                bad = max(0.0, 0.5 + sum(sh[i, k, ch] * Ybad[k] for k in idx))
                assert abs(rev - expect) > 1e-3 or abs(s) < 1e-3
                assert abs(bad - expect) > 1e-4 or abs(s) < 1e-3


# -------------------------------------------------------- preprocess (§3.2)

def test_isotropic_on_axis_closed_form():
    """Isotropic s at (0, 0, z), camera at the origin: Sigma' = ((f s / z)^2 +
    0.3) I, conic its inverse, centre at the principal point, and the extent
    where alpha = 1/255 is sqrt(2 ln(255 sigma) Sigma'_xx) (§3.4)."""
    z, s, f, logit = 4.0, 0.05, 64.0, 1.0
    sc = _scene(1, [0, 0, z], [math.log(s)] * 3, logits=[logit])
    p = oracle.preprocess(sc, _cam(f=f))
    v = (f * s / z) ** 2 + 0.3
    np.testing.assert_allclose(p["cov2d"][0], [v, 0, v], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(p["conic"][0], [1 / v, 0, 1 / v], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(p["mean2d"][0], [32, 32], atol=1e-13)
    sigma = 1 / (1 + math.exp(-logit))
    e = math.sqrt(2 * math.log(255 * sigma) * v)
    np.testing.assert_allclose(p["extent"][0], [e, e], rtol=1e-13)
    assert p["depth"][0] == np.float32(z)
    np.testing.assert_allclose(p["rgb"][0], [1, 1, 1], rtol=1e-14)
    assert p["reason"][0] == 0


def test_isotropic_off_axis_closed_form():
    """Isotropic s at (x, 0, z): J = [[f/z, 0, -f x/z^2], [0, f/z, 0]] gives
    Sigma'_xx = s^2 f^2/z^2 (1 + x^2/z^2) + 0.3, Sigma'_yy = s^2 f^2/z^2 + 0.3;
    past the guard band the ratio x/z is clamped inside J only."""
    f, s, z = 64.0, 0.05, 4.0
    for x in (1.0, -1.5):
        sc = _scene(1, [x, 0, z], [math.log(s)] * 3)
        p = oracle.preprocess(sc, _cam(f=f))
        k = (s * f / z) ** 2
        np.testing.assert_allclose(p["cov2d"][0], [k * (1 + x * x / z / z) + 0.3, 0, k + 0.3], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(p["mean2d"][0], [f * x / z + 32, 32], rtol=1e-14)
    # x/z = 2 > 1.3 * (W/2)/f = 0.65: the Jacobian uses 0.65
    sc = _scene(1, [8.0, 0, z], [math.log(s)] * 3)
    p = oracle.preprocess(sc, _cam(f=f))
    k = (s * f / z) ** 2
    np.testing.assert_allclose(p["cov2d"][0, 0], k * (1 + 0.65 ** 2) + 0.3, rtol=1e-12)


def test_dilation_and_guard_band_are_taken_from_the_configuration():
    """Reading 2: the low-pass dilation and the guard band are configuration
    values, not constants: on-axis Sigma' = ((f s / z)^2 + dilation) I for
    dilations 0 and 1; with a guard band of 2 the ratio x/z = 2 is clamped
    to 2 (W/2)/f = 1 inside J, and x/z = 0.75, which the default band of 1.3
    clamps to 0.65, is not clamped."""
    z, s, f = 4.0, 0.05, 64.0
    k = (f * s / z) ** 2
    for dil in (0.0, 1.0):
        p = oracle.preprocess(_scene(1, [0, 0, z], [math.log(s)] * 3), _cam(f=f), dilation=dil)
        np.testing.assert_allclose(p["cov2d"][0], [k + dil, 0, k + dil], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(p["conic"][0], [1 / (k + dil), 0, 1 / (k + dil)], rtol=1e-13)
    p = oracle.preprocess(_scene(1, [8.0, 0, z], [math.log(s)] * 3), _cam(f=f), guard=2.0)
    np.testing.assert_allclose(p["cov2d"][0, 0], k * (1 + 1.0 ** 2) + 0.3, rtol=1e-12)
    sc = _scene(1, [3.0, 0, z], [math.log(s)] * 3)
    p = oracle.preprocess(sc, _cam(f=f), guard=2.0)
    np.testing.assert_allclose(p["cov2d"][0, 0], k * (1 + 0.75 ** 2) + 0.3, rtol=1e-12)
    p = oracle.preprocess(sc, _cam(f=f))
    np.testing.assert_allclose(p["cov2d"][0, 0], k * (1 + 0.65 ** 2) + 0.3, rtol=1e-12)


def test_general_covariance_against_numerical_jacobian():
    """Sigma' = J W Sigma W^T J^T + 0.3 I for a rotated anisotropic Gaussian and
    a look-at camera, checked against an independent route: scipy's quaternion
    rotation and a central-difference Jacobian of the pinhole map."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(13)
    cam0 = S.look_at_camera((3.0, -2.0, 1.5), (0.1, 0.2, 0.0), 96, 80, fov_x_deg=50)
    # and a camera with fx != fy and an off-centre principal point
    cam1 = dict(cam0, fx=110.0, fy=80.0, cx=41.0, cy=46.5)
    for cam in (cam0, cam1):
        _check_covariance_against_numerical_jacobian(cam, rng, Rotation)


def _check_covariance_against_numerical_jacobian(cam, rng, Rotation):
    vm = np.asarray(cam["viewmat"], float)
    Rv, tv = vm[:, :3], vm[:, 3]

    def proj(X):
        t = Rv @ X + tv
        return np.array([cam["fx"] * t[0] / t[2] + cam["cx"], cam["fy"] * t[1] / t[2] + cam["cy"]])

    for _ in range(10):
        X = rng.uniform(-0.3, 0.3, 3)
        ls = rng.normal(-2.5, 0.5, 3)
        q = rng.standard_normal(4)
        sc = _scene(1, X, ls, quats=q * 1.7)  # unnormalised on purpose
        p = oracle.preprocess(sc, cam)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = R @ np.diag(np.exp(2 * ls)) @ R.T
        h = 1e-6
        Jn = np.stack([(proj(X + h * e) - proj(X - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        Sp = Jn @ Sig @ Jn.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(p["cov2d"][0], [Sp[0, 0], Sp[0, 1], Sp[1, 1]], rtol=1e-7)
        np.testing.assert_allclose(p["conic"][0].take([0, 1, 1, 2]).reshape(2, 2), np.linalg.inv(Sp), rtol=1e-7)
        np.testing.assert_allclose(p["mean2d"][0], proj(X), rtol=1e-13)


def test_look_at_target_projects_to_principal_point():
    cam = S.hd_camera(3)
    sc = _scene(1, [0, 0, 0], [-3] * 3)
    p = oracle.preprocess(sc, cam)
    np.testing.assert_allclose(p["mean2d"][0], [960, 540], atol=1e-9)


def test_opacity_cull_boundary():
    """§3.4: a splat with sigma < 1/255 is culled; sigma = 1/255 is kept.
    sigma < 1/255 <=> logit < -ln 254; the float32 logits on both sides of
    that value fall on the two sides of the decision."""
    tau = -math.log(254.0)
    t32 = np.float32(tau)
    below = np.nextafter(t32, np.float32(-np.inf)) if float(t32) >= tau else t32
    above = np.nextafter(t32, np.float32(np.inf)) if float(t32) < tau else t32
    assert float(below) < tau < float(above)
    logits = np.array([below, above, -8.0, 0.0], np.float32).astype(float)
    sc = _scene(4, np.tile([0, 0, 3.0], (4, 1)), np.full((4, 3), -3.0), logits=logits)
    p = oracle.preprocess(sc, _cam())
    assert list(p["reason"]) == [1, 0, 1, 0]
    # exactly at sigma = 1/255 the extent is zero and the centre pixel is kept
    assert p["extent"][1, 0] < 1e-3


def test_near_plane_zero_quaternion_and_offscreen():
    """Near-plane cull on the float32 depth, a zero quaternion is culled,
    and a splat whose box misses the viewport by ~1 px is culled while one
    touching it stays (§3.2 AABB culling)."""
    f, s = 64.0, 0.02
    v = (f * s / 2.0) ** 2 + 0.3
    e = math.sqrt(2 * math.log(255 / (1 + math.exp(-2.0))) * v)
    x_out = (-1.0 - e - 32) * 2.0 / f      # centre at -1 - e px: box ends 1 px left of 0
    x_in = (1.0 - e - 32) * 2.0 / f        # box reaches 1 px into the image
    means = [[0, 0, 0.1], [0, 0, 2.0], [x_out, 0, 2.0], [x_in, 0, 2.0]]
    quats = [[1, 0, 0, 0], [0, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0]]
    sc = _scene(4, means, np.full((4, 3), math.log(s)), quats=quats)
    p = oracle.preprocess(sc, _cam(f=f))
    assert list(p["reason"]) == [3, 2, 5, 0]
    assert p["touched"][3] == 2 and list(p["rect"][3]) == [0, 1, 0, 2]


def test_tile_corner_touches_four_tiles():
    """A small splat centred on the corner shared by four 16-px tiles touches
    exactly those four; one centred in a tile touches one."""
    sc = _scene(2, [[(16 - 32) / 32.0, (16 - 32) / 32.0, 2.0], [(8 - 32) / 32.0, (8 - 32) / 32.0, 2.0]],
                np.full((2, 3), math.log(0.02)))
    p = oracle.preprocess(sc, _cam())
    assert list(p["touched"]) == [4, 1]
    assert list(p["rect"][0]) == [0, 0, 1, 1] and list(p["rect"][1]) == [0, 0, 0, 0]


def test_depth32_is_float32_evaluation():
    """The float32 depth with R = I is exactly fl(z + t_z)."""
    rng = np.random.default_rng(14)
    vm = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3]], float)
    for _ in range(200):
        X = rng.uniform(-1, 1, 3).astype(np.float32).astype(float)
        assert oracle.depth32(X, vm) == np.float32(X[2]) + np.float32(3)


# ------------------------------------------------------------ blend (§2.1)

def test_single_gaussian_on_pixel_centre():
    """At the centre of a pixel the splat alpha is min(0.99, sigma):
    C = c alpha, T = 1 - alpha (E4 with one term)."""
    for logit in (0.3, 8.0):
        sc = _scene(1, [(10.5 - 32) / 32.0, (20.5 - 32) / 32.0, 2.0], [math.log(0.03)] * 3, logits=[logit])
        out = oracle.render(sc, _cam())
        a = min(0.99, 1 / (1 + math.exp(-logit)))
        np.testing.assert_allclose(out["image"][20, 10], [a, a, a], rtol=1e-14)
        np.testing.assert_allclose(out["t_final"][20, 10], 1 - a, rtol=1e-14)
        assert out["last_gid"][20, 10] == 0


def test_stacked_identical_gaussians():
    """K identical splats at increasing depth but the same projected footprint
    (scaled with depth): T = (1 - a)^K and C = c (1 - (1 - a)^K)."""
    K = 7
    zs = 2.0 + 0.25 * np.arange(K)
    means = np.stack([np.zeros(K), np.zeros(K), zs], 1) + 0.5 / 64.0 * np.array([1, 1, 0]) * zs[:, None]
    ls = np.log(0.01 * zs / 2.0)[:, None].repeat(3, 1)
    sh = np.zeros((K, 16, 3))
    sh[:, 0, :] = (0.8 - 0.5) / C0
    sc = _scene(K, means, ls, logits=np.full(K, 0.0), sh=sh)
    out = oracle.render(sc, _cam())
    a = 0.5
    np.testing.assert_allclose(out["t_final"][32, 32], (1 - a) ** K, rtol=1e-12)
    np.testing.assert_allclose(out["image"][32, 32], 0.8 * (1 - (1 - a) ** K), rtol=1e-12)


def test_white_scene_obeys_one_minus_transmittance():
    """With every colour 1 and a black background, E4 gives C = sum a_i T_i =
    1 - T_final at every pixel: a dropped term or a wrong transmittance
    update breaks this."""
    scene, cam = S.small_forward()
    sc = dict(scene)
    sh = np.zeros_like(scene["sh"])
    sh[:, 0, :] = 0.5 / C0
    sc["sh"] = sh.astype(np.float32)
    out = oracle.render(sc, cam)
    for ch in range(3):
        np.testing.assert_allclose(out["image"][..., ch], 1 - out["t_final"], atol=1e-12)


def test_tile_lists_equal_brute_force_back_to_front():
    """The per-tile front-to-back result equals a per-pixel back-to-front
    "over" composite of every visible splat with no tiles (§2.1's order):
    the opacity-aware extent (§3.4) is conservative, so tiles lose nothing."""
    scene = S.uniform_scene(400, seed=21)
    cam = {"viewmat": np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3]], np.float32),
           "fx": 40.0, "fy": 40.0, "cx": 24.0, "cy": 20.0, "width": 48, "height": 40,
           "znear": 0.2, "bg": (0.1, 0.2, 0.3)}
    for tile in (8, 16, 32):
        out = oracle.render(scene, cam, tile=tile)
        img, tf = oracle.blend_brute(cam, out["proj"])
        ok = out["n_amb"] == 0
        assert ok.mean() > 0.99
        np.testing.assert_allclose(out["image"][ok], img[ok], atol=1e-12)
        np.testing.assert_allclose(out["t_final"][ok], tf[ok], atol=1e-12)


# ------------------------------------------------------------- sort (§3.3)

@pytest.mark.parametrize("n", [0, 1, 31, 4097, 100_000])
@pytest.mark.parametrize("kind", ["random", "equal", "sorted", "reversed", "few"])
def test_sort_is_stable_sort(n, kind):
    """§3.3.2: equal keys keep their input order. Matches numpy's stable
    argsort (a library special case) on every input shape."""
    rng = np.random.default_rng(n + len(kind))
    if kind == "random":
        keys = rng.integers(0, 2 ** 45, n, dtype=np.uint64)
    elif kind == "equal":
        keys = np.full(n, 12345, np.uint64)
    elif kind == "sorted":
        keys = np.sort(rng.integers(0, 2 ** 40, n, dtype=np.uint64))
    elif kind == "reversed":
        keys = np.sort(rng.integers(0, 2 ** 40, n, dtype=np.uint64))[::-1].copy()
    else:
        keys = rng.integers(0, 3, n).astype(np.uint64) << np.uint64(33)
    vals = np.arange(n, dtype=np.uint32)
    k, v = oracle.sort_pairs(keys, vals)
    perm = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(k, keys[perm])
    np.testing.assert_array_equal(v, vals[perm])


def test_emission_and_ranges():
    """Key emission: Gaussian i emits touched_i keys in row-major tile order,
    offsets are their exclusive scan; tile ranges equal searchsorted bounds."""
    scene, cam = S.small_forward()
    out = oracle.render(scene, cam)
    p = out["proj"]
    np.testing.assert_array_equal(np.diff(out["offsets"]), p["touched"])
    keys, vals = out["keys"], out["vals"]
    np.testing.assert_array_equal(np.bincount(vals, minlength=p["touched"].size), p["touched"])
    assert np.all((keys & np.uint64(0x7FFFFFFF)) == p["depth"][vals].view(np.uint32))
    tx = (cam["width"] + 15) // 16
    tiles = (keys >> np.uint64(31)).astype(np.int64)
    i = 123
    r = p["rect"][i]
    got = tiles[out["offsets"][i]:out["offsets"][i + 1]]
    exp = [ty * tx + x for ty in range(r[1], r[3] + 1) for x in range(r[0], r[2] + 1)]
    assert list(got) == exp
    sk = out["sorted_keys"]
    st = (sk >> np.uint64(31)).astype(np.int64)
    rng_ = out["ranges"]
    for t in range(0, tx * tx, 7):
        lo, hi = np.searchsorted(st, t, "left"), np.searchsorted(st, t, "right")
        if hi > lo:
            assert (rng_[t] == [lo, hi]).all()


# ----------------------------------------------------------- gradient (§1)

@pytest.mark.parametrize("kind", ["small", "big", "needles", "background"])
def test_gradient_matches_central_differences(kind):
    """The oracle's analytic FP64 gradient of L = 1/2 ||C - target||^2 agrees
    with FP64 central differences on 64 Gaussians at 32x32 (entries whose
    step changes a discrete decision are skipped and counted). The second
    scene uses larger, overlapping splats so occlusion terms matter; the
    third, 24 needles (one long axis, the others e^-6) in random orientations,
    whose projected covariances have condition numbers up to ~200, so the
    anisotropic parts of the chain (the conic of a thin ellipse, the rotation
    gradient) carry weight. The fourth is the first with a non-black
    background, which enters every pair's alpha derivative through the colour
    behind it. Step h = 1e-5: the rounding noise of a central difference,
    about eps L / h for a loss L of a few hundred, then stays two orders of
    magnitude below the 1e-6 bar (at h = 1e-6 it reached ~1e-6 on the
    quaternion gradients), and the truncation error, O(h^2), further below."""
    scene, cam, target = S.gradcheck_scene()
    if kind == "background":
        cam = dict(cam, bg=(0.3, 0.6, 0.9))
    if kind == "big":
        scene = S.uniform_scene(64, seed=7, log_scale_mean=-2.3, log_scale_std=0.3)
    elif kind == "needles":
        scene = S.uniform_scene(24, seed=8)
        rng = np.random.default_rng(9)
        ls = np.full((24, 3), -6.0)
        ls[:, 0] = rng.uniform(-1.2, -0.4, 24)
        scene["log_scales"] = ls.astype(np.float32)
        scene["opacity_logits"] = rng.normal(0.5, 1.0, 24).astype(np.float32)
    sc = {k: v.astype(np.float64) for k, v in scene.items()}
    base = oracle.loss_grad(sc, cam, target)
    h = 1e-5
    skipped = checked = 0
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        flat = sc[name].reshape(-1)
        g = base["grads"][name].reshape(-1)
        fd = np.zeros_like(g)
        mask = np.zeros(g.size, bool)
        for j in range(flat.size):
            old = flat[j]
            flat[j] = old + h
            p = oracle.loss_grad(sc, cam, target, grads=False)
            flat[j] = old - h
            m = oracle.loss_grad(sc, cam, target, grads=False)
            flat[j] = old
            if p["fingerprint"] != base["fingerprint"] or m["fingerprint"] != base["fingerprint"]:
                skipped += 1
                continue
            fd[j] = (p["loss"] - m["loss"]) / (2 * h)
            mask[j] = True
        checked += mask.sum()
        err = np.linalg.norm(g[mask] - fd[mask]) / max(np.linalg.norm(fd[mask]), 1e-12)
        assert err < 1e-6, (name, err)
        # sanity: gradients are non-trivial
        assert np.linalg.norm(g[mask]) > 0, name
    assert skipped < 0.02 * (checked + skipped)


def test_ablations_leave_the_image_unchanged():
    """§4.4's ablations only add work: keeping sigma < 1/255 splats, keeping
    off-screen boxes (-CULL) and the opacity-independent box (-RADIUS) do not
    change the image, because every added pair has alpha < 1/255. They do
    add (tile, splat) pairs."""
    scene = S.uniform_scene(600, seed=51)
    scene["opacity_logits"][:60] = -7.0  # below 1/255
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 64, 48)
    base = oracle.render(scene, cam)
    for flags in (oracle.NO_OPACITY_CULL, oracle.NO_AABB_CULL, oracle.FIXED_RADIUS,
                  oracle.NO_OPACITY_CULL | oracle.NO_AABB_CULL | oracle.FIXED_RADIUS):
        out = oracle.render(scene, cam, flags=flags)
        ok = (base["n_amb"] == 0) & (out["n_amb"] == 0)
        np.testing.assert_allclose(out["image"][ok], base["image"][ok], atol=1e-14)
        assert out["keys"].size > base["keys"].size


def _fd_check(sc, cam, target, names, h=1e-6):
    """Analytic FP64 gradient against central differences on the named
    parameters (entries whose step changes a discrete decision skipped)."""
    base = oracle.loss_grad(sc, cam, target)
    for name in names:
        flat = sc[name].reshape(-1)
        g = base["grads"][name].reshape(-1)
        for j in range(flat.size):
            old = flat[j]
            flat[j] = old + h
            p = oracle.loss_grad(sc, cam, target, grads=False)
            flat[j] = old - h
            m = oracle.loss_grad(sc, cam, target, grads=False)
            flat[j] = old
            if p["fingerprint"] != base["fingerprint"] or m["fingerprint"] != base["fingerprint"]:
                continue
            fd = (p["loss"] - m["loss"]) / (2 * h)
            assert abs(g[j] - fd) <= 1e-6 * max(1.0, abs(fd)), (name, j, g[j], fd)
    return base


def test_no_gradient_through_the_clamps():
    """Reading 12: a colour channel clamped at 0 passes no gradient to its SH
    coefficients, and an alpha clamped at 0.99 none to the splat's opacity
    or shape from that pixel; the analytic values agree with central
    differences there (a gradient taken through either clamp would not)."""
    sh = np.zeros((2, 16, 3))
    sh[:, 0, :] = 0.3 / C0  # colour 0.8
    sh[0, 0, 0] = -2.0 / C0  # red of splat 0: 0.5 - 2 + small terms < 0, clamped
    sh[0, 1:4, 0] = [0.05, -0.03, 0.02]
    # splat 1 centred on the centre of pixel (16, 16) at sigma ~ 0.9997
    z1 = 5.0
    means = [[0.3, -0.2, 4.0], [0.5 * z1 / 32.0, 0.5 * z1 / 32.0, z1]]
    sc = _scene(2, means, [[-1.6] * 3, [-1.5] * 3], logits=[1.0, 8.0], sh=sh)
    cam = _cam(32, 32, 32.0)
    # the 0.99 clamp is active: splat 1 alone gives C = 0.8 * 0.99 at its centre
    one = {k: v[1:] for k, v in sc.items()}
    out = oracle.render(one, cam)
    np.testing.assert_allclose(out["image"][16, 16], [0.8 * 0.99] * 3, rtol=1e-12)
    target = np.random.default_rng(18).random((32, 32, 3))
    base = _fd_check(sc, cam, target, ("opacity_logits", "log_scales", "sh"))
    g = base["grads"]["sh"]
    assert not np.any(g[0, :, 0])  # the clamped channel
    assert np.all(g[0, 0, 1:] != 0) and np.all(g[1, 0, :] != 0)
    # splat 1 alone: its clamped centre pixel adds nothing to the opacity
    # gradient, so a target that matches the image everywhere else gives 0
    img = oracle.render(one, cam)["image"]
    tgt = img.copy()
    tgt[16, 16] += 0.25
    g1 = oracle.loss_grad(one, cam, tgt)["grads"]
    assert g1["opacity_logits"][0] == 0 and not np.any(g1["log_scales"]) and not np.any(g1["means"])
    assert np.any(g1["sh"])  # the colour still gets the residual of that pixel


def test_gradient_with_the_guard_band_clamp_active():
    """Reading 2 / 12: a splat whose centre lies beyond the 1.3x guard band
    (t_x / t_z = 0.8 against a limit of 0.65 here) has its Jacobian built
    from the clamped ratio, and the analytic gradient, which passes nothing
    through the clamped ratio, agrees with central differences; the splat
    still reaches into the image, so its gradient is not zero."""
    sh = np.zeros((2, 16, 3))
    sh[:, 0, :] = 0.3 / C0
    sh[0, 1:4, :] = 0.1  # view-dependent colour: the direction term as well
    means = [[0.8 * 4.0, 0.1, 4.0], [-0.2, 0.1, 5.0]]
    sc = _scene(2, means, [[0.0, -0.3, -0.6], [-1.8] * 3], logits=[1.5, 0.5], sh=sh,
                quats=[[0.9, 0.1, 0.3, -0.2], [1.0, 0.0, 0.0, 0.0]])
    cam = _cam(32, 32, 32.0)
    out = oracle.render(sc, cam)
    assert out["proj"]["touched"][0] > 0 and out["proj"]["mean2d"][0][0] > 32  # centre off-screen
    target = np.random.default_rng(19).random((32, 32, 3))
    base = _fd_check(sc, cam, target, ("means", "log_scales", "quats", "opacity_logits"))
    assert np.linalg.norm(base["grads"]["means"][0]) > 0


def test_gradient_does_not_depend_on_the_tile_size():
    """The tile decomposition is a schedule, not part of the method: the loss
    and the analytic gradient for 8-, 16- and 32-pixel tiles agree to FP64
    rounding (a tile-dependent pixel coordinate, list or sum in the backward
    would show here)."""
    scene = S.uniform_scene(400, seed=22)
    cam = S.look_at_camera((2.0, -1.2, 0.9), (0.3, 0.1, 0.0), 72, 56)
    target = np.random.default_rng(17).random((56, 72, 3))
    base = oracle.loss_grad(scene, cam, target, tile=16)
    assert np.linalg.norm(base["grads"]["means"]) > 0
    for tile in (8, 32):
        out = oracle.loss_grad(scene, cam, target, tile=tile)
        assert abs(out["loss"] - base["loss"]) <= 1e-12 * abs(base["loss"])
        for k, g in base["grads"].items():
            np.testing.assert_allclose(out["grads"][k], g, rtol=0, atol=1e-12 * max(1.0, np.abs(g).max()))


def test_ablations_leave_the_gradient_unchanged():
    """The same ablations leave the loss and its analytic gradient unchanged:
    an added pair's alpha is below 1/255 at every pixel, so it is never
    composited and its partials are zero (a mistake that let the flags reach
    the adjoint, e.g. a gradient through the fixed radius, would show here)."""
    scene = S.uniform_scene(600, seed=51)
    scene["opacity_logits"][:60] = -7.0
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 64, 48)
    target = np.random.default_rng(16).random((48, 64, 3))
    base = oracle.loss_grad(scene, cam, target)
    assert np.linalg.norm(base["grads"]["means"]) > 0
    for flags in (oracle.NO_OPACITY_CULL, oracle.NO_AABB_CULL, oracle.FIXED_RADIUS,
                  oracle.NO_OPACITY_CULL | oracle.NO_AABB_CULL | oracle.FIXED_RADIUS):
        out = oracle.loss_grad(scene, cam, target, flags=flags)
        assert abs(out["loss"] - base["loss"]) <= 1e-12 * abs(base["loss"])
        for k, g in base["grads"].items():
            np.testing.assert_allclose(out["grads"][k], g, rtol=0, atol=1e-12 * max(1.0, np.abs(g).max()))


# ------------------------------------------------------------ packed record

def test_f16_rounding_is_ieee_binary16():
    """§3.2 packs the ellipse axes as binary16: or_round_f16 is numpy's
    float64 -> float16 conversion (round to nearest, ties to even), across
    the normal and subnormal ranges, exact ties and overflow."""
    rng = np.random.default_rng(8)
    x = np.concatenate([
        rng.uniform(-3, 3, 2000), np.exp(rng.uniform(-20, 11, 2000)) * rng.choice([-1, 1], 2000),
        # exact ties: odd multiples of half an ulp
        (2 * rng.integers(1, 1000, 200) + 1) * 2.0 ** -11 + 1.0, 2049.0 + 2 * np.arange(50),
        (2 * rng.integers(0, 500, 50) + 1) * 2.0 ** -25,   # subnormal ties
        [0.0, -0.0, 65504.0, 65519.99, 65520.0, 1e6, 5.96e-8, 2.9e-8, 3.0e-8]])
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(oracle.round_f16(x), want)


def test_axes_reconstruct_the_covariance():
    """v1 v1^T + v2 v2^T = Sigma', v1 is along the larger eigenvalue and
    v2 is v1 turned by +90 degrees, with lengths sqrt(l1) >= sqrt(l2) (the
    eigenvalues numpy's eigh gives), for isotropic, axis-aligned, rotated
    and very elongated covariances."""
    rng = np.random.default_rng(9)
    cases = [(1.0, 0.0, 1.0), (4.0, 0.0, 1.0), (1.0, 0.0, 4.0), (2.0, 1.999, 2.0), (0.3, -0.0, 0.3)]
    for _ in range(300):
        l1, l2 = np.sort(np.exp(rng.uniform(-2, 9, 2)))[::-1]
        th = rng.uniform(0, np.pi)
        U = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        Sg = U @ np.diag([l1, l2]) @ U.T
        cases.append((Sg[0, 0], Sg[0, 1], Sg[1, 1]))
    for sxx, sxy, syy in cases:
        v1, v2 = oracle.axes(sxx, sxy, syy)
        Sg = np.array([[sxx, sxy], [sxy, syy]])
        rec = np.outer(v1, v1) + np.outer(v2, v2)
        np.testing.assert_allclose(rec, Sg, rtol=1e-12, atol=1e-12 * np.abs(Sg).max())
        ev = np.linalg.eigvalsh(Sg)
        np.testing.assert_allclose([v1 @ v1, v2 @ v2], ev[::-1], rtol=1e-10, atol=1e-12 * ev.max())
        assert abs(v1 @ v2) <= 1e-12 * (v1 @ v1)
        assert v1[0] * v2[1] - v1[1] * v2[0] >= 0  # v2 is v1 turned by +90 degrees


def test_packed_record_quantisation():
    """With PACKED the pre-processing stores opacity and clamped colour on
    8 bits (multiples of 1/255 within half a step of the float values), the
    centre in float32 and the conic of the binary16 axes."""
    scene = S.uniform_scene(800, seed=61)
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 96, 72)
    full = oracle.preprocess(scene, cam)
    pk = oracle.preprocess(scene, cam, flags=oracle.PACKED)
    vis = pk["touched"] > 0
    assert vis.sum() > 300
    for k in ("opacity", "rgb"):
        q = pk[k][vis] * 255.0
        np.testing.assert_allclose(q, np.round(q), atol=1e-9)
        ref = np.clip(full[k][vis], 0.0, 1.0)
        assert np.abs(pk[k][vis] - ref).max() <= 0.5 / 255 + 1e-12
    np.testing.assert_array_equal(pk["mean2d"][vis], full["mean2d"][vis].astype(np.float32).astype(np.float64))
    for i in np.nonzero(vis)[0][:200]:
        c = full["cov2d"][i]
        v1, v2 = oracle.axes(c[0], c[1], c[2])
        v1, v2 = oracle.round_f16(v1), oracle.round_f16(v2)
        Sg = np.outer(v1, v1) + np.outer(v2, v2)
        np.testing.assert_allclose(pk["cov2d"][i], [Sg[0, 0], Sg[0, 1], Sg[1, 1]], rtol=1e-15, atol=0)
        Q = np.linalg.inv(Sg)
        np.testing.assert_allclose(pk["conic"][i], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-12)
        # binary16 axes keep the covariance within ~1e-3 relative
        assert np.abs(Sg - np.array([[c[0], c[1]], [c[1], c[2]]])).max() <= 2e-3 * max(c[0], c[2])


def test_packed_image_close_to_the_float_image():
    """Where no colour exceeds 1 (nothing for the 8-bit clamp to cut), the
    packed record changes each pixel by well under 1/255: the quantisation
    steps are below 1/510 each and alpha-weighted."""
    scene = S.uniform_scene(1500, seed=62)
    scene["sh"][:, 0, :] = np.clip(scene["sh"][:, 0, :], -0.6, 0.6)
    scene["sh"][:, 1:, :] *= 0.2
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 96, 72)
    full = oracle.render(scene, cam)
    assert full["proj"]["rgb"][full["proj"]["touched"] > 0].max() < 1.0
    pk = oracle.render(scene, cam, flags=oracle.PACKED)
    ok = (full["n_amb"] == 0) & (pk["n_amb"] == 0)
    d = np.abs(pk["image"] - full["image"])[ok]
    assert d.max() <= 1.0 / 255, d.max()
    assert np.median(d) <= 1e-3
