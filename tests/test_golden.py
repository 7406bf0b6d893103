"""Golden fixtures (tests/golden/): values printed in the paper, each line with
its citation, against the oracle's constants and worked examples, and the PPO
hyperparameters against the library's defaults (a host-only call)."""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def test_paper_parameters_are_the_oracles():
    P = O.default_params()
    lines = rows("paper_parameters.txt")
    assert len(lines) >= 35
    for r in lines:
        name, value = r[0], float(r[1])
        assert hasattr(P, name), name
        assert abs(float(getattr(P, name)) - value) <= 1e-12 * max(1.0, abs(value)), (name, getattr(P, name), value)


def test_wheel_inertia_from_the_printed_wheel():
    (m, s, r), = [[float(x) for x in row] for row in rows("wheel_inertia.txt")]
    assert abs(O.default_params().wheel_inertia - 0.5 * m * r * r * s) < 1e-12


def test_ttc_circle_geometry_worked_example():
    for L, W, WB, r, d in [[float(x) for x in row] for row in rows("ttc_circles.txt")]:
        rr, dd = O.ttc_circles(L, W, WB)
        assert abs(rr - r) <= 0.005 and abs(dd - d) <= 0.005


def test_ppo_defaults_are_the_papers():
    sf = pytest.importorskip("paper_2605_08528_b300.sf")
    from paper_2605_08528_b300 import build as B
    B.build()
    cfg = sf.sf_ppo_default_config()
    for name, value in rows("ppo_hparams.txt"):
        assert abs(float(getattr(cfg, name)) - float(value)) <= 1e-6 * max(1.0, abs(float(value))), name
