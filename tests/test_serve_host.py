"""Host-side logic of the serving loop (no GPU): the seeded request stream."""
import numpy as np

from paper_2311_15439_gb300 import synth  # noqa: F401  (package import without the CUDA library)


def test_poisson_load_statistics():
    from paper_2311_15439_gb300.serve import poisson_load
    t, ds, sizes = poisson_load(1000.0, 20000, (2, 3, 4, 5), 4096, 4 << 20, seed=3)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 1000.0) < 40.0                  # arrival rate
    assert sizes.min() >= 4096 and sizes.max() <= 4 << 20
    logs = np.log(sizes)
    # log-uniform: the log-sizes are uniform, so each quarter of the log range holds ~25%
    edges = np.linspace(np.log(4096), np.log(4 << 20), 5)
    frac = np.histogram(logs, edges)[0] / len(logs)
    assert np.all(np.abs(frac - 0.25) < 0.02)
    assert set(np.unique(ds)) == {2, 3, 4, 5}
    t2, ds2, s2 = poisson_load(1000.0, 20000, (2, 3, 4, 5), 4096, 4 << 20, seed=3)
    assert np.array_equal(t, t2) and np.array_equal(s2, sizes)
