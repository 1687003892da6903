"""The pattern recipe of the kernel fits (Sec. 5.1, Fig. 5) and the fitting
scene, checked on the CPU."""
import numpy as np

from paper_2411_12440_gb300 import fitting


def test_patterns_recipe():
    p = fitting.pattern("stripes", 4, 64)
    assert p.shape == (64, 64, 3) and set(np.unique(p)) == {np.float32(0.1), np.float32(0.9)}
    assert (p[:, :8] == np.float32(0.9)).all() and (p[:, 8:16] == np.float32(0.1)).all()  # 4 periods of 16 px
    c = fitting.pattern("checkerboard", 2, 32)
    assert c[0, 0, 0] != c[0, 8, 0] and c[0, 0, 0] != c[8, 0, 0] and c[0, 0, 0] == c[8, 8, 0]
    r = fitting.pattern("circles", 2, 64)
    assert r[32, 32, 0] == np.float32(0.9) and r[32, 32 + 9, 0] == np.float32(0.1)


def test_fitting_scene_covers_the_image():
    """Primitives on a jittered grid in the plane z = 4 whose projections
    cover the image, isotropic with half the grid spacing as deviation."""
    scene, cam = fitting.init_scene(16, 64, seed=1)
    assert scene.n == 256 and scene.sh_degree == 0
    px = scene.means[:, 0] * cam["fx"] / scene.means[:, 2] + cam["cx"]
    py = scene.means[:, 1] * cam["fy"] / scene.means[:, 2] + cam["cy"]
    assert px.min() > 0 and px.max() < 64 and py.min() > 0 and py.max() < 64
    assert np.allclose(scene.scales * cam["fx"] / 4.0, 2.0, rtol=1e-5)  # 0.5 x 4-pixel spacing
