"""The seeded input generators shared by the oracle side and the CUDA side:
the same seed gives the same inputs bit for bit, another seed other inputs, and
the structural properties the workload recipes state hold (quaternion and SH
shapes, the bf16 rounding of feature maps, the planted outlier fractions)."""
import numpy as np

from paper_2506_05558_gb300 import synth


def _arrays(x, prefix=""):
    """Flattens the numeric contents of a generator's output to (name, array)."""
    if isinstance(x, synth.Scene):
        for k in ("mean_opa", "scale", "quat", "sh"):
            yield prefix + k, np.asarray(getattr(x, k))
    elif isinstance(x, dict):
        for k in sorted(x):
            yield from _arrays(x[k], f"{prefix}{k}.")
    elif isinstance(x, (list, tuple)):
        for i, v in enumerate(x):
            yield from _arrays(v, f"{prefix}{i}.")
    elif isinstance(x, np.ndarray) or np.isscalar(x):
        yield prefix, np.asarray(x)


def _same(a, b):
    la, lb = list(_arrays(a)), list(_arrays(b))
    assert [k for k, _ in la] == [k for k, _ in lb]
    return all(np.array_equal(x, y, equal_nan=True) for (_, x), (_, y) in zip(la, lb))


GENERATORS = {
    "tiny_scene": lambda s: synth.tiny_scene(seed=s)[:2],
    "multiview_scene": lambda s: synth.multiview_scene(seed=s, n=2000, n_views=3, sizes=[(64, 48)] * 3)[:2],
    "projected_items": lambda s: synth.projected_items(np.random.default_rng(s), 500, 8, 6, 16),
    "ba_problem": lambda s: synth.ba_problem(seed=s, n_frames=4, n_points=256),
    "ba_pose_problem": lambda s: synth.ba_pose_problem(seed=s, n_obs=256),
    "guided_scene": lambda s: synth.guided_scene(seed=s, width=48, height=32, f=40.0, n_nb=2, channels=8),
}


def test_generators_are_deterministic_per_seed():
    for name, gen in GENERATORS.items():
        assert _same(gen(11), gen(11)), name
        assert not _same(gen(11), gen(12)), name


def test_scene_recipe_shapes():
    sc, cam, _ = synth.tiny_scene()
    assert sc.mean_opa.shape == (sc.n, 4) and sc.scale.shape == (sc.n, 4) and sc.quat.shape == (sc.n, 4)
    assert sc.sh.shape == (sc.n, 48) and np.all(sc.sh[:, 3:] == 0)  # SH0 scene: higher bands zero
    assert (cam["width"], cam["height"]) == (64, 64)


def test_guided_features_are_bf16_values():
    sc = synth.guided_scene(seed=3, width=48, height=32, f=40.0, n_nb=2, channels=8)
    f = sc["feats"]
    assert f.dtype == np.uint16  # bf16 bit patterns
    as_f32 = (f.astype(np.uint32) << 16).view(np.float32)
    assert np.all(np.isfinite(as_f32))
    assert np.array_equal(synth.to_bf16(as_f32), f)  # already on the bf16 grid


def test_planted_outlier_fractions():
    """Gross outliers are offsets of 30-80 px; inlier noise is N(0, 0.5) px."""
    pb = synth.ba_pose_problem(seed=5, n_obs=4000, outlier_frac=0.1)
    r = np.linalg.norm(pb["noise"], axis=-1)
    assert abs(np.mean(r > 10) - 0.1) < 0.02
    assert np.all((r < 5) | ((r > 27) & (r < 83)))  # magnitude 30-80 plus the inlier noise
    b = synth.ba_problem(seed=5, n_frames=4, n_points=2000, outlier_frac=0.03)
    r = np.linalg.norm(b["noise"], axis=-1)
    assert abs(np.mean(r > 10) - 0.03) < 0.01
