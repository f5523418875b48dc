"""The synthetic workloads follow their stated recipes (CPU): grid sizes,
domains, boundary conditions, schemes and horizons of the benchmark
configurations, the seeded draws of the batched workload, and determinism
(the same seed gives the same inputs on both sides of every comparison)."""
import numpy as np
import pytest

from paper_2411_03501_gb300 import workloads as W


def test_air3d_benchmark_configuration():
    spec, phi0, g = W.air3d(n=201)
    assert spec["n"] == [201, 201, 201] and spec["ndim"] == 3
    assert spec["lo"] == [-6, -10, 0] and spec["hi"][:2] == [20, 10]
    assert spec["hi"][2] == pytest.approx(2 * np.pi)
    assert spec["periodic"] == [False, False, True]
    assert (spec["scheme"], spec["rk"], spec["cfl"], spec["dtype"]) == ("weno5", 3, 0.75, "f32")
    assert spec["tube"] and spec["t_final"] == pytest.approx(2.8)
    assert spec["params"][:2] == [5.0, 5.0]
    # target: the cylinder of radius 5 in (x, y); phi0 = target
    assert np.array_equal(phi0, g)
    x = spec["lo"][0] + np.arange(201) * (26.0 / 200)
    y = spec["lo"][1] + np.arange(201) * (20.0 / 200)
    want = np.sqrt(x[:, None] ** 2 + y[None, :] ** 2) - 5.0
    np.testing.assert_allclose(g[:, :, 17], want, atol=1e-12)


def test_car4d_benchmark_configuration():
    spec, phi0, g = W.car4d(n=81)
    assert spec["n"] == [81] * 4
    assert spec["periodic"] == [False, False, True, False]
    assert (spec["scheme"], spec["rk"], spec["cfl"], spec["dtype"]) == ("eno3", 3, 0.75, "f32")
    assert spec["lo"][:2] == [-4, -4] and spec["hi"][:2] == [4, 4] and spec["hi"][3] == 2
    assert spec["t_final"] == pytest.approx(1.0) and spec["tube"]
    assert np.array_equal(phi0, g)
    assert g.nbytes // 2 == 43046721 * 4  # 172 MB per field in FP32


def test_normal_speed_2d_configuration():
    spec, phi0, _ = W.normal_speed_2d()
    assert spec["n"] == [101, 101] and spec["dtype"] == "f64"
    assert (spec["scheme"], spec["rk"], spec["cfl"]) == ("eno2", 2, 0.9)
    assert spec["t_final"] == pytest.approx(0.5)
    x = np.linspace(-1, 1, 101)
    np.testing.assert_allclose(phi0, np.sqrt(x[:, None] ** 2 + x[None, :] ** 2) - 0.3,
                               atol=1e-12)


def test_batched_draws_follow_the_recipe():
    probs = W.batched()
    assert len(probs) == 256
    two, three = probs[:128], probs[128:]
    assert all(p[0]["ndim"] == 2 and p[0]["dyn"] == "normal_speed" for p in two)
    assert all(p[0]["ndim"] == 3 and p[0]["dyn"] == "air3d" for p in three)
    sides2 = np.array([p[0]["n"][0] for p in two])
    sides3 = np.array([p[0]["n"][0] for p in three])
    assert sides2.min() >= 64 and sides2.max() <= 256
    assert sides3.min() >= 48 and sides3.max() <= 128
    speeds = np.array([p[0]["params"][0] for p in probs])
    assert speeds.min() >= 2.0 and speeds.max() <= 6.0
    for p in probs:
        spec = p[0]
        assert (spec["scheme"], spec["rk"], spec["dtype"]) == ("weno5", 3, "f32") and spec["tube"]
        if spec["ndim"] == 3:
            assert spec["params"][0] == spec["params"][1]  # v_e = v_p = speed
            assert spec["t_final"] == pytest.approx(2.8)
        else:  # t_final = (0.9 - r) / speed, r in [0.2, 0.6]
            r = 0.9 - spec["t_final"] * spec["params"][0]
            assert 0.2 - 1e-12 <= r <= 0.6 + 1e-12
    # total points: ~3.7 M in 2-D, ~105 M in 3-D (the recipe's expectation)
    pts = sum(int(np.prod(p[0]["n"])) for p in probs)
    assert 80e6 < pts < 140e6


def test_batched_draws_are_deterministic():
    a, b = W.batched(count=8), W.batched(count=8)
    for (sa, pa, ga), (sb, pb, gb) in zip(a, b):
        assert sa == sb and np.array_equal(pa, pb) and np.array_equal(ga, gb)
    c = W.batched(count=8, seed=1)
    assert any(sa["n"] != sc["n"] for (sa, _, _), (sc, _, _) in zip(a, c))
