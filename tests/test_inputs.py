"""The seeded synthetic inputs (paper_2210_05547_gb300/inputs.py) that stand in for the paper's
cases: reproducible by seed, and within the stated recipe. The serving stream holds grids of
128 x 32 to 1024 x 256 and boundary layers at Mach 5-20 with walls at 300-1500 K. Its shock
interactions take at least 128 rows and a time step of 5e-4, each request takes its configured
step range, and the eleven-species share follows its own stream. The sweep states span
300-15000 K and 1e-4-1 kg/m^3 with normalised mass fractions, and the state noise lies in [-1, 1].
"""
import numpy as np

from paper_2210_05547_gb300 import inputs as I


def test_serving_stream_recipe():
    reqs = I.serving_requests(200, seed=100, steps=(500, 2000), air11=0.25)
    assert len(reqs) == 200
    n11 = 0
    for cfg, steps, gap in reqs:
        assert 500 <= steps <= 2000 and gap >= 0.0
        assert cfg["nx"] in (128, 256, 512, 1024) and cfg["ny"] in (32, 64, 128, 256)
        if "_bl_" in cfg["name"]:
            assert 5.0 <= cfg["mach"] <= 20.0
            assert 300.0 <= cfg["T_wall"] <= 1500.0
        if "sbli" in cfg["name"]:
            assert cfg["ny"] >= 128 and cfg["dt"] == 5.0e-4
        n11 += len(cfg["Y_inf"]) == 11
    assert 30 <= n11 <= 70                 # a quarter of 200, drawn from its own stream


def test_serving_stream_is_reproducible_and_share_independent():
    a = I.serving_requests(40, seed=7, steps=(10, 20))
    b = I.serving_requests(40, seed=7, steps=(10, 20))
    c = I.serving_requests(40, seed=7, steps=(10, 20), air11=1.0)
    assert [(x["name"], s, g) for x, s, g in a] == [(x["name"], s, g) for x, s, g in b]
    # the eleven-species share changes the gas, not the grids, step counts or arrivals
    assert [(x["nx"], x["ny"], s, g) for x, s, g in a] == [(x["nx"], x["ny"], s, g) for x, s, g in c]
    assert all(len(x["Y_inf"]) == 11 for x, _, _ in c)


def test_thermo_states_recipe():
    T, rho, Y = I.thermo_states(5000, seed=3)
    assert T.min() >= 300.0 and T.max() <= 15000.0
    assert rho.min() >= 1e-4 and rho.max() <= 1.0
    assert Y.shape == (5, 5000) and (Y >= 0.0).all()
    assert np.allclose(Y.sum(axis=0), 1.0, rtol=0, atol=1e-14)
    T2, _, _ = I.thermo_states(5000, seed=3)
    assert np.array_equal(T, T2)


def test_state_noise_range_and_seed():
    a = I.state_noise(1000, 5)
    assert a.min() >= -1.0 and a.max() <= 1.0
    assert np.array_equal(a, I.state_noise(1000, 5))
    assert not np.array_equal(a, I.state_noise(1000, 6))
