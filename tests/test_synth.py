"""The seeded synthetic inputs: the same seed gives the same data (the oracle and
the CUDA path see identical inputs), and each recipe has the stated shape, label
balance and dtype."""
import numpy as np

from paper_2305_12019_gb300 import synth


def test_seeded_inputs_are_reproducible():
    a = synth.gaussian(seed=11, d=300, n=50, n_pos=20)
    b = synth.gaussian(seed=11, d=300, n=50, n_pos=20)
    c = synth.gaussian(seed=12, d=300, n=50, n_pos=20)
    assert np.array_equal(a.Z, b.Z) and np.array_equal(a.y, b.y)
    assert not np.array_equal(a.Z, c.Z)


def test_recipes_shapes_labels_and_dtypes():
    p = synth.plain_fp64()
    assert p.Z.shape == (500, 100) and p.Z.dtype == np.float64
    assert int((p.y == 1).sum()) == 50 and p.q == 1.0 and p.C == 1.0
    s = synth.spiked_fp32(d=2000, m_test=10)
    assert s.Z.shape == (2000, 1000) and s.Z.dtype == np.float32
    assert int((s.y == 1).sum()) == 500 and s.C == 10.0
    assert np.array_equal(s.Z, (s.X * s.y).astype(np.float32))       # Z = X diag(y), eq-r
    h = synth.heavy_tailed(seed=3, d=400, n=80, n_pos=20)
    assert h.Z.shape == (400, 80) and int((h.y == 1).sum()) == 20
    shapes = synth.uneven_batch(5, count=6)
    assert len(shapes) == 6
    assert all(5000 <= sh["d"] <= 50000 and 200 <= sh["n"] <= 2000 for sh in shapes)
