"""The seeded input generators: deterministic, shaped like the paper's workloads."""
import numpy as np

import workloads


def test_deterministic_and_shaped():
    a = workloads.config0()
    b = workloads.config0()
    assert np.array_equal(a["angles"], b["angles"])
    assert a["angles"].shape == (32, 3, 64) and a["angles"].dtype == np.float32
    assert np.all(a["angles"][:, 2] == np.float32(np.pi))
    c1 = workloads.config1()
    L = c1["lengths"]
    assert L.min() >= 128 and L.max() <= 350 and c1["seq"].max() < 20
    assert c1["angles"].shape[2] % 4 == 0


def test_loguniform_lengths_and_padding_zero():
    rng = workloads.rng_for(2)
    L = workloads.lengths_loguniform(2000, 50, 1000, rng)
    assert L.min() >= 50 and L.max() <= 1000
    assert abs(np.log(L).mean() - 0.5 * (np.log(50) + np.log(1000))) < 0.1
    a = workloads.backbone_angles(L[:5], rng)
    for b in range(5):
        assert np.all(a[b, :, L[b]:] == 0)


def test_lrmsd_clouds():
    rng = workloads.rng_for(3)
    x, y, n = workloads.lrmsd_clouds(8, 100, 500, rng)
    assert x.shape == y.shape and x.shape[0] == 8 and n.min() >= 100 and n.max() <= 500
    for p in range(8):
        assert np.all(x[p, n[p]:] == 0) and np.all(y[p, n[p]:] == 0)
