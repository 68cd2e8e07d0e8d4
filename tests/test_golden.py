"""Golden fixtures: the oracle still reproduces its committed expected values,
and the paper's Table III parameter sets parse into valid runs."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_table3():
    rows = []
    with open(os.path.join(HERE, "table3_parameters.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            exp, term, dt, sigma, ts, sigma1 = line.split()
            rows.append(dict(experiment=exp, term=term, dt=float(dt),
                             sigma=float(sigma), ts=int(ts),
                             sigma1=None if sigma1 == "-" else float(sigma1)))
    return rows


def test_table3_rows_are_valid_runs():
    rows = load_table3()
    assert len(rows) == 14
    for r in rows:
        assert r["term"] in ("region", "edge")
        assert r["ts"] % 2 == 1 and 3 <= r["ts"] <= 31
        # Sec. IV-D: time steps above 25 may be unstable; the paper uses 15-18
        assert 0 < r["dt"] <= 25 and r["sigma"] > 0
        assert (r["sigma1"] is not None) == (r["term"] == "edge")


@pytest.mark.parametrize("name", ["region_step1", "region_step5",
                                  "edge_indicator", "edge_step3"])
def test_oracle_reproduces_golden(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    img, phi0 = mg.fixture_inputs()
    expected = np.loadtxt(os.path.join(HERE, f"oracle_{name}_12x16.txt"))
    g = oracle.edge_indicator(img, 1.0, 9, 255.0)
    got = {
        "region_step1": lambda: oracle.evolve(img, phi0, "region", iterations=1)[0],
        "region_step5": lambda: oracle.evolve(img, phi0, "region", iterations=5)[0],
        "edge_indicator": lambda: g,
        "edge_step3": lambda: oracle.evolve(img, -phi0, "edge", g=g, iterations=3)[0],
    }[name]()
    np.testing.assert_allclose(got, expected, rtol=1e-12, atol=1e-13)
