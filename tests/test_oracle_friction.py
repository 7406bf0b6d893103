"""Pins of the oracle's weather-to-friction builder (App. B, the modified ALL
model at 13.89 m/s, read as F5: the printed mu_static(h) points joined
linearly, down to the 1e-3 floor at the 0.85 mm aquaplaning threshold).

The model's calibration (sigma_0, mu_s, mu_c, alpha, L, Y_R(h), Y_F(h)) is not
given, so the builder is pinned only where the paper prints values: the 27
points of Fig. friction_mu_vs_film, Tab. friction_mu (a second, rounded
source), the floor, the presets, and Eq. app_stribeck_speed's closed form.
"""
import math

from oracle import oracle as O
from tests.test_golden import rows

SURF = {"AC": 0, "SMA": 1, "OGFC": 2}


def test_printed_curve_points_are_reproduced():
    pts = rows("all_mu_static.txt")
    assert len(pts) == 27
    for s, h, mu in pts:
        film = int(round(float(h) * 100))
        assert abs(O.all_mu_static(SURF[s], film) - float(mu)) < 1e-12, (s, h)


def test_the_rounded_table_agrees_with_the_curves():
    """Tab. friction_mu and the figure are two printed sources: the curve points
    round to the table's entries, and films of 1.0 and 2.0 mm give the floor."""
    for s, m0, m3, m5, m10, m20 in rows("all_mu_table.txt"):
        k = SURF[s]
        for film, m in ((0, m0), (30, m3), (50, m5)):
            assert abs(O.all_mu_static(k, film) - float(m)) <= 5e-4 + 1e-12, (s, film)
        assert m10 == m20 == "<=1e-3"
        for film in (100, 200, 255):
            assert O.all_mu_static(k, film) == 1e-3


def test_texture_coefficient_scaling():
    """With sigma_1 = sigma_2 = 0 (App. B) Eq. app_mu_all is
    mu = max(theta Y_R - Y_F, 0) * theta Y_R sigma_0 z*, and the steady state of
    Eq. app_bristle_ode makes theta Y_R sigma_0 z* = sigma_0 v_r g / (sigma_0 |v_r|
    + K |w_r| g), free of theta.  While the hydrodynamic force ratio Y_F is small
    (no lift yet), mu is therefore proportional to theta at every film: the SMA
    and OGFC curves are the AC curve times 1.09 and 1.21 (a transposed or
    misread entry breaks this).  The printed points hold it to 0.5 %."""
    th = {r[0]: float(r[1]) for r in rows("all_presets.txt") if r[0] in SURF}
    P = O.default_params()
    assert [P.all_theta[i] for i in range(3)] == [th["AC"], th["SMA"], th["OGFC"]]
    for film in range(0, 81, 10):
        ac = O.all_mu_static(0, film)
        for s in ("SMA", "OGFC"):
            ratio = O.all_mu_static(SURF[s], film) / ac
            assert abs(ratio / (th[s] / th["AC"]) - 1.0) < 5e-3, (s, film, ratio)


def test_interpolation_reading():
    """Between printed points the film is interpolated linearly; from 0.8 mm
    mu falls linearly to the floor at 0.85 mm; it never rises with the film."""
    for k in range(3):
        for film in range(0, 80):
            a, b = film // 10, film // 10 + 1
            lo, hi = O.all_mu_static(k, 10 * a), O.all_mu_static(k, 10 * b)
            t = (film - 10 * a) / 10.0
            assert abs(O.all_mu_static(k, film) - (lo + t * (hi - lo))) < 1e-12
        assert abs(O.all_mu_static(k, 82) - (O.all_mu_static(k, 80) * 0.6 + 1e-3 * 0.4)) < 1e-12
        seq = [O.all_mu_static(k, f) for f in range(0, 256)]
        assert all(x >= y for x, y in zip(seq, seq[1:]))
        assert min(seq) == 1e-3


def test_stribeck_speed_closed_form_properties():
    """Eq. app_stribeck_speed with b2 < 0: v_s decreases with the film toward
    the asymptote b4, and the excess v_s - b4 is exponential in the film: its
    ratio between films h + 0.1 mm and h is exp(1000 b2 * 1e-4 m), whatever h."""
    b = [float(x) for x in [r for r in rows("all_presets.txt") if r[0] == "stribeck"][0][1:]]
    P = O.default_params()
    assert [P.stribeck_b[i] for i in range(4)] == b
    vs = [O.stribeck_vs(h * 1e-4) for h in range(0, 30)]          # 0 ... 2.9 mm
    assert all(x > y for x, y in zip(vs, vs[1:]))
    assert abs(O.stribeck_vs(1.0) - b[3]) < 1e-12                  # a metre of water: the b4 asymptote
    for h in (0.0, 2e-4, 7e-4):
        r = (O.stribeck_vs(h + 1e-4) - b[3]) / (O.stribeck_vs(h) - b[3])
        assert abs(r - math.exp(1000.0 * b[1] * 1e-4)) < 1e-12
    # dry: b1 e^b3 + b4 (the film term at h = 0)
    assert abs((O.stribeck_vs(0.0) - b[3]) / b[0] - math.exp(b[2])) < 1e-12


def test_weather_model_sets_mu_and_the_token():
    """With the ALL model a placed agent gets mu_static of its surface and film
    and the ego group's weather token is Eq. weather_obs (h / h_norm, one-hot
    AC, SMA, OGFC)."""
    from paper_2605_08528_b300 import synth
    P = O.default_params()
    P.weather_model = O.WEATHER_ALL
    sc = synth.straight_road(num_agents=1)
    orc = O.Oracle(sc, P)
    F, I = orc.empty_state()
    orc.place(F, I, 0, 0.0, -1.8, 0.0, 10.0, 80.0, -1.8, precip=30, surface=2)   # OGFC, 0.30 mm
    assert F[0, O.F_MU] == O.all_mu_static(2, 30)
    o = orc.observe(F, I)["obs"][0]
    assert abs(o[7] - 0.30) < 1e-15 and list(o[8:11]) == [0, 0, 1]
    assert abs(o[13] - 1.1617) < 1e-12
