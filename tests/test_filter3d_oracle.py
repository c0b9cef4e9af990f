"""Pins of the oracle's 3-D smoothing filter (Mip-Splatting's 3-D filter, the
"proper filtering" of Sec. 4.3): the filtered Gaussian against the filter's
definition (covariance Sigma + v I, opacity times sqrt(det Sigma / det(Sigma +
v I))) computed with numpy linear algebra and scipy rotations, the preserved
integral, the chain rule against FP64 central differences of the rendered loss,
and the sampling-rate rule by hand."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2506_05558_gb300 import synth

from test_oracle_pins import _fd_scene, _loss


def _cov(scene):
    """World covariances R diag(s^2) R^T, rotations by scipy (quaternion w, x, y, z)."""
    q = np.asarray(scene.quat, np.float64)
    R = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    s2 = np.exp(2 * np.asarray(scene.scale, np.float64)[:, :3])
    return np.einsum("nij,nj,nkj->nik", R, s2, R)


def _random_scene(n=200, seed=3):
    rng = np.random.default_rng(seed)
    sc = synth.gaussians(rng, n, [-1, -1, 2], [1, 1, 6], -3.0, 0.6, 0)
    return sc, rng.uniform(1e-5, 5e-3, n)


def test_filtered_covariance_and_opacity_match_the_definition():
    sc, v = _random_scene()
    f = O.filtered_scene(sc, v)
    cov, covf = _cov(sc), _cov(f)
    np.testing.assert_allclose(covf, cov + v[:, None, None] * np.eye(3), rtol=1e-12, atol=1e-15)
    o = 1 / (1 + np.exp(-np.asarray(sc.mean_opa, np.float64)[:, 3]))
    of = 1 / (1 + np.exp(-f.mean_opa[:, 3]))
    ratio = np.linalg.det(cov) / np.linalg.det(cov + v[:, None, None] * np.eye(3))
    np.testing.assert_allclose(of, o * np.sqrt(ratio), rtol=1e-10)
    # the opacity-weighted integral o (2 pi)^(3/2) sqrt(det Sigma) is unchanged
    np.testing.assert_allclose(of * np.sqrt(np.linalg.det(covf)), o * np.sqrt(np.linalg.det(cov)), rtol=1e-10)
    # v = 0 changes nothing
    f0 = O.filtered_scene(sc, np.zeros(sc.n))
    np.testing.assert_allclose(f0.scale[:, :3], sc.scale[:, :3], rtol=0, atol=1e-14)
    np.testing.assert_allclose(f0.mean_opa, sc.mean_opa, rtol=0, atol=1e-12)


@pytest.mark.parametrize("sh_degree", [0, 3])
def test_filter_chain_matches_central_differences(sh_degree):
    """d loss / d (log-scale, logit) of the filtered render: the oracle's adjoint
    of the filtered scene carried back by filter3d_chain, against central
    differences of the loss with the filter applied to perturbed parameters."""
    cfg = O.Config(sh_degree=sh_degree, bg=(0.1, 0.2, 0.3))
    for seed in range(11, 60):
        sc, cam, rng = _fd_scene(sh_degree, seed)
        v = rng.uniform(2e-3, 2e-2, sc.n)  # comparable to the scene's squared scales
        view = O.render_view(O.filtered_scene(sc, v), cam, cfg)
        if view["amb"].sum() == 0 and view["proj"]["amb"].sum() == 0:
            break
    assert view["amb"].sum() == 0 and view["proj"]["amb"].sum() == 0
    w = rng.standard_normal((3, cam["height"], cam["width"]))
    g = O.filter3d_chain(sc, v, O.backward_view(O.filtered_scene(sc, v), cam, cfg, view, w))
    lists = (view["start"], view["ids"])
    h = 1e-6

    def fd(field, i, c):
        arr = getattr(sc, field)
        old = arr[i, c]
        step = h * max(1.0, abs(old))
        vals = []
        for sgn in (1, -1):
            arr[i, c] = old + sgn * step
            vals.append(_loss(O.filtered_scene(sc, v), cam, cfg, w, lists)[0])
        arr[i, c] = old
        return (vals[0] - vals[1]) / (2 * step)

    vis = np.nonzero(view["proj"]["n_tiles"])[0]
    checks = []
    for i in vis[:8]:
        for c in range(3):
            checks.append((fd("scale", i, c), g["log_scale"][i, c]))
        checks.append((fd("mean_opa", i, 3), g["logit"][i]))
    num = np.array([a for a, _ in checks])
    an = np.array([b for _, b in checks])
    assert np.abs(num).max() > 0
    np.testing.assert_allclose(an, num, rtol=1e-5, atol=1e-6 * np.abs(num).max())


def test_sampling_rate_rule_by_hand():
    """Two cameras on the z axis looking down +z, fx = 100, 64x48 images:
    camera A at the origin, camera B 2 m further back. A Gaussian on the axis
    at z = 4 is sampled by A at 100 / 4 and by B at 100 / 6: v = 0.2 / 25^2. One
    at x = 3, z = 4 projects to u = 32 + 75 = 107 > 1.15 x 64 = 73.6 in A and to
    32 + 50 = 82 in B: outside both, so unsampled. One behind A (z = -1) and 1 m
    in front of B (z = 1 in B's frame) is sampled by B alone at 100 / 1. The
    unsampled Gaussian takes the largest variance of the sampled ones."""
    def cam(z0):
        return dict(R=np.eye(3), t=np.array([0.0, 0.0, -z0]), fx=100.0, fy=100.0, cx=32.0, cy=24.0,
                    width=64, height=48)
    cams = [cam(0.0), cam(-2.0)]
    mo = np.array([[0.0, 0.0, 4.0, 0.0], [3.0, 0.0, 4.0, 0.0], [0.0, 0.0, -1.0, 0.0]])
    sc = synth.Scene(mo, np.zeros((3, 4)), np.tile([1.0, 0, 0, 0], (3, 1)), np.zeros((3, 48)), 0)
    v, amb = O.filter3d_variance(sc, cams, near_z=0.2, s2=0.2)
    want_a = 0.2 / (100 / 4) ** 2
    want_c = 0.2 / (100 / 1) ** 2
    np.testing.assert_allclose(v, [want_a, max(want_a, want_c), want_c], rtol=1e-14)
    assert not amb.any()
