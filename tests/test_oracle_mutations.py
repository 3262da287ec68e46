"""The oracle's pins against planted mistakes.

Each case copies the C oracle, plants one plausible mistake (a dropped term,
a wrong sign, a wrong weight or index, a swapped set), builds it into a
separate library and runs a few of the pins on it: at least one must fail.
The mistakes are planted only in temporary copies of the oracle, on the
CPU; the regular oracle is restored afterwards.  CPU only.
"""
import math

import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_sides as side_pins

P = oracle

# (name, original line fragment, planted mistake, pins expected to catch it)
MUTATIONS = [
    ("source term dropped (Eq. 16)",
     "s[i] = -(1.0 - 1.0 / (2.0 * tau)) * 5.0 * a_w(i) * cq / (3.0 * tau_r);",
     "s[i] = 0.0 * cq;",
     [pins.test_collision_conserves_energy_and_normal_flux,
      pins.test_uniform_flux_decay_on_lattice]),
    ("tau_r in place of tau in (1 - 1/(2 tau)) (Eq. 16)",
     "s[i] = -(1.0 - 1.0 / (2.0 * tau)) * 5.0 * a_w(i) * cq / (3.0 * tau_r);",
     "s[i] = -(1.0 - 1.0 / (2.0 * tau_r)) * 5.0 * a_w(i) * cq / (3.0 * tau_r);",
     [pins.test_source_moments_eqs_26_to_28,
      pins.test_collision_conserves_energy_and_normal_flux]),
    ("kappa missing from the flux moment (Eq. 54)",
     "*qx = k * mx;", "*qx = mx;",
     [pins.test_uniform_flux_decay_on_lattice,
      lambda: pins.test_fourier_mode_exact(1, 0)]),
    ("5/3 dropped from the equilibrium (Eq. 15)",
     "eeq[i] = omega_w(i) * e + 5.0 * a_w(i) * cq / 3.0;",
     "eeq[i] = omega_w(i) * e + a_w(i) * cq;",
     [pins.test_equilibrium_moments_eqs_22_to_25]),
    ("diagonal weight 1/18 instead of 1/36 (Eq. 17)",
     "return i < 4 ? 2.0 / 9.0 : 1.0 / 36.0;", "return i < 4 ? 2.0 / 9.0 : 1.0 / 18.0;",
     [pins.test_equilibrium_moments_eqs_22_to_25, pins.test_weights_and_flux_factor]),
    ("tau = tau_C without the 1/2 (Eq. 49)",
     "out[0] = tau_C + 0.5;", "out[0] = tau_C + 0.25;",
     [pins.test_paper_relaxation_times]),
    ("relaxation by tau_r instead of tau (Eq. 13)",
     "post[i] = f[i] + (eeq[i] - f[i]) / tau + s[i];",
     "post[i] = f[i] + (eeq[i] - f[i]) / tau_r + s[i];",
     [lambda: pins.test_fourier_mode_exact(1, 1),
      lambda: pins.test_brute_force_matrix(5, 4, oracle.PERIODIC_GRADIENT, oracle.PERIODIC,
                                           -0.21)]),
    ("streaming against c_i (Eq. 13 left-hand side)",
     "int tx = x + CX[i];", "int tx = x - CX[i];",
     [lambda: pins.test_fourier_mode_exact(1, 0),
      lambda: pins.test_brute_force_matrix(4, 3, oracle.PERIODIC_GRADIENT, oracle.WALLS, 0.37)]),
    ("seam jump with the wrong sign (Eq. 59)",
     "v = omega_w(i) * delta_e + v;", "v = v - omega_w(i) * delta_e;",
     [pins.test_periodic_gradient_steady_state_is_affine,
      pins.test_energy_conserved_periodic_with_seam]),
    ("wall takes the leaving populations as incident (Eq. 58)",
     "if (CY[i] * ny_out > 0) incident += g[i];", "if (CY[i] * ny_out < 0) incident += g[i];",
     [pins.test_wall_nodes_have_zero_normal_flux,
      lambda: pins.test_brute_force_matrix(3, 5, oracle.PERIODIC, oracle.WALLS, 0.0)]),
    ("heat-flux side without 1/kappa (Eq. 57)",
     "double extra = q0 / flux_factor(tau_r);", "double extra = q0;",
     [side_pins.test_side_nodes_satisfy_eqs_55_to_58]),
    ("isothermal side with equal weights (Eq. 55)",
     "for (int i = 0; i < 8; ++i) g[i] = omega_w(i) * e_s;",
     "for (int i = 0; i < 8; ++i) g[i] = 0.125 * e_s;",
     [side_pins.test_side_nodes_satisfy_eqs_55_to_58,
      lambda: side_pins.test_brute_force_matrix_with_sides(*side_pins.SIDE_CASES[0])]),
]


@pytest.fixture
def planted(tmp_path):
    def build(old, new):
        src = open(oracle._SRC).read()
        assert src.count(old) == 1, old
        path = tmp_path / "oracle_mut.c"
        path.write_text(src.replace(old, new))
        lib = oracle.compile_library(str(path), str(tmp_path / "liboracle_mut.so"))
        oracle.use_library(lib)
        return lib
    yield build
    oracle.use_library(None)


@pytest.mark.parametrize("name,old,new,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(planted, name, old, new, checks):
    planted(old, new)
    caught = []
    for check in checks:
        try:
            check()
        except (AssertionError, ValueError, FloatingPointError):
            caught.append(check)
    assert caught, f"no pin caught: {name}"


def test_unmutated_copy_passes_the_same_pins(planted):
    """Control: the identical copy built the same way passes every pin used
    above, so a caught mutation is the planted mistake, not the build."""
    planted("out[0] = tau_C + 0.5;", "out[0] = tau_C + 0.5;")
    seen = set()
    for *_, checks in MUTATIONS:
        for check in checks:
            if id(check) not in seen:
                seen.add(id(check))
                check()


# --- the numpy oracles: D3Q14 / D1Q2 and the continuum solutions -----------------
def test_lattice_pins_catch_wrong_d3q14_weights(monkeypatch):
    """Corner flux weight 1/12 instead of 1/24: the moment conditions and the
    continuum dispersion must reject it."""
    import numpy as np
    from oracle import lattices as lt
    from tests import test_oracle_lattices as lat_pins
    bad = lt.Lattice("D3Q14", 3, lt.D3Q14.c, lt.D3Q14.w,
                     np.array([1 / 3] * 6 + [1 / 12] * 8), lt.D3Q14.speed)
    monkeypatch.setattr(lat_pins, "D3", bad)
    monkeypatch.setattr(lt, "D3Q14", bad)
    with pytest.raises(AssertionError):
        lat_pins.test_equilibrium_and_source_moments(bad)
    with pytest.raises(AssertionError):
        lat_pins.test_d3q14_longitudinal_modes_follow_eq52((1, 0, 0))


def test_closed_form_pins_catch_planted_mistakes(monkeypatch):
    import numpy as np
    from oracle import analytic
    from tests import test_oracle_sides as sp

    good_1d = analytic.fourier_transient_1d

    def film_without_third(X, t_star, kn_R, terms=4000):      # Kn^2 n^2 pi^2 t* (no /3)
        return good_1d(X, 3.0 * t_star, kn_R, terms)
    monkeypatch.setattr(analytic, "fourier_transient_1d", film_without_third)
    with pytest.raises(AssertionError):
        sp.test_fourier_transient_solves_heat_equation()
    monkeypatch.setattr(analytic, "fourier_transient_1d", good_1d)

    good_sq = analytic.square_steady

    def square_flipped_qy(X, Y, Q0=1.0, terms=400):
        th, qx, qy = good_sq(X, Y, Q0, terms)
        return th, qx, -qy
    monkeypatch.setattr(analytic, "square_steady", square_flipped_qy)
    with pytest.raises(AssertionError):
        sp.test_square_steady_solves_laplace_with_its_boundary_values()
    monkeypatch.setattr(analytic, "square_steady", good_sq)

    good_tr = analytic.heat_pulse_transforms

    def pulse_wrong_reflection(X, kn_N, kn_R, t_pulse=100.0):  # C1 with the wrong sign
        both = good_tr(X, kn_N, kn_R, t_pulse)
        Xc = np.asarray(X, dtype=np.float64)[:, None]
        kn_C = 1.0 / (1.0 / kn_N + 1.0 / kn_R)

        def wrong(s):
            Tb, Qb = both(s)
            s = np.asarray(s, dtype=np.complex128)[None, :]
            A = np.sqrt((kn_R / kn_N * s + 1.0) /
                        (kn_N * kn_R / (3.0 * s) + 4.0 / 15.0 * kn_C * kn_R))
            A = np.where(A.real < 0, -A, A)
            C2 = (1.0 / s) * (1.0 - np.exp(-t_pulse * s)) / (1.0 - np.exp(-2.0 * A))
            up = -C2 * np.exp(-A * (2.0 - Xc))
            return Tb + 2 * (kn_N / s) * A * up, Qb - 2 * up
        return wrong
    monkeypatch.setattr(analytic, "heat_pulse_transforms", pulse_wrong_reflection)
    with pytest.raises(AssertionError):
        sp.test_heat_pulse_energy_balance_and_boundary_flux()
