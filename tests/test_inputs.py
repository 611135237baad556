"""The seeded input generators, on the host: the bubble-cloud quantities
keep the ranges and relations their recipe states (gas fraction in [0, 1],
density = alpha + 1000 (1 - alpha), pressure = 1e5 + pressure modes -
9e4 alpha), fields are a pure function of (recipe, shape, seed), the FP32
field is the FP64 one rounded once, and the thread count changes nothing
(every point depends only on its coordinates and the draws)."""
import numpy as np
import pytest

from paper_1903_07761_gb300 import inputs


def test_bubble_cloud_ranges_and_relations():
    shape, seed, nb = (48, 40, 64), 7, 30
    a = inputs.field(inputs.ALPHA, shape, np.float64, seed=seed, nbubbles=nb)
    rho = inputs.field(inputs.RHO, shape, np.float64, seed=seed, nbubbles=nb)
    p = inputs.field(inputs.P, shape, np.float64, seed=seed, nbubbles=nb)
    assert a.min() >= 0.0 and a.max() <= 1.0
    assert a.max() > 0.99 and a.min() < 1e-6  # bubbles and liquid both present
    np.testing.assert_allclose(rho, a * 1.0 + (1.0 - a) * 1000.0, rtol=0, atol=1e-9)
    # pressure: 1e5 plus a mean of eight unit sines times 1e4, minus 9e4 alpha
    modes = p - 1e5 + 9e4 * a
    assert np.abs(modes).max() <= 1e4 + 1e-6
    assert modes.std() > 100.0  # the modes are there
    # the Gaussian-bubble field is 1 plus non-negative bubbles plus tiny noise
    g = inputs.field(inputs.GAUSS, (32, 32, 32), np.float64, seed=seed)
    assert g.min() > 1.0 - 1e-3 and g.max() > 10.0


@pytest.mark.parametrize("recipe", [inputs.GAUSS, inputs.ALPHA, inputs.RHO, inputs.P])
def test_seeded_and_rounded_once(recipe):
    shape = (16, 24, 32)
    f64a = inputs.field(recipe, shape, np.float64, seed=11, nbubbles=12)
    f64b = inputs.field(recipe, shape, np.float64, seed=11, nbubbles=12)
    f32 = inputs.field(recipe, shape, np.float32, seed=11, nbubbles=12)
    other = inputs.field(recipe, shape, np.float64, seed=12, nbubbles=12)
    np.testing.assert_array_equal(f64a, f64b)
    np.testing.assert_array_equal(f32, f64a.astype(np.float32))
    assert not np.array_equal(f64a, other)


def test_fields_do_not_depend_on_the_thread_count(tmp_path):
    """Every point is a function of its coordinates and the seed only: one
    OpenMP thread gives the same bytes as all of them."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = tmp_path / "one_thread.npy"
    code = ("import numpy as np; from paper_1903_07761_gb300 import inputs; "
            f"np.save({str(out)!r}, inputs.field(inputs.GAUSS, (24, 16, 32), np.float64, seed=9)); "
            f"np.save({str(out)!r}.replace('one', 'p_one'), inputs.field(inputs.P, (24, 16, 32), np.float64, seed=9, nbubbles=9))")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    subprocess.run([sys.executable, "-c", code], cwd=root, env=env, check=True, timeout=300)
    np.testing.assert_array_equal(np.load(out), inputs.field(inputs.GAUSS, (24, 16, 32), np.float64, seed=9))
    np.testing.assert_array_equal(np.load(str(out).replace("one", "p_one")),
                                  inputs.field(inputs.P, (24, 16, 32), np.float64, seed=9, nbubbles=9))
