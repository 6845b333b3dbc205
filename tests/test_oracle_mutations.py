"""The oracle's pins catch plausible mistakes: each test plants one mistake in the oracle (on the
CPU, through monkeypatch) and checks that at least one pin of tests/test_oracle_pins.py or
tests/test_oracle_thermal.py then fails."""
import numpy as np
import pytest

from oracle import mrt_d2q8 as fl
from oracle import thermal_d2q5 as th
from tests import test_oracle_pins as pins
from tests import test_oracle_thermal as tpins

FLOW_PINS = [
    pins.test_equilibrium_moments_equal_eq22_distribution,
    pins.test_collision_conserves_mass_and_adds_force_to_momentum,
    pins.test_conserved_moment_rates_do_not_change_the_result,
    pins.test_explicit_velocity_solves_implicit_eq17,
    pins.test_single_rate_reduces_to_bgk_with_eq22,
    pins.test_Cx_Cy_match_printed_eqA4,
    lambda: pins.test_brute_force_8x8_matches_literal_eq6(
        "wall", "wall", {"bottom": (0.0, 0.01), "top": (0.1, 0.0), "left": (0.0, 0.02), "right": (0.0, -0.03)}),
    pins.test_free_fluid_poiseuille_is_exact_parabola_at_magic_rates,
    pins.test_porous_couette_sinh_profile_pins_moving_wall,
    pins.test_nee_walls_porous_couette_moving_node,
    pins.test_nee_wall_node_is_equilibrium_at_wall_velocity_for_equilibrium_neighbour,
]
THERMAL_PINS = [
    tpins.test_collision_keeps_T_and_relaxes_flux_to_uT,
    tpins.test_conduction_between_isothermal_walls_is_linear_and_nu_is_one,
    tpins.test_advected_sine_mode_decays_and_moves_as_eqB1,
    tpins.test_stably_stratified_rest_state_is_hydrostatic_with_upward_buoyancy,
    tpins.test_side_heated_cavity_rises_at_the_hot_wall,
]


def _caught(pin_list):
    for pin in pin_list:
        try:
            pin()
        except (AssertionError, FloatingPointError, ValueError):
            return True
    return False


def _mut_forcing_sign(monkeypatch):
    orig = fl.forcing_moments

    def wrong(ux, uy, Fx, Fy, phi, rho0):
        S = orig(ux, uy, Fx, Fy, phi, rho0)
        S[1] = -S[1]  # sign of S2
        return S

    monkeypatch.setattr(fl, "forcing_moments", wrong)


def _mut_l0(monkeypatch):
    orig = fl.velocity

    def wrong(f, phi, K, nu, rho0, forchheimer, ax, ay):
        ux, uy = orig(f, phi, K, nu, rho0, forchheimer, ax, ay)
        return 0.98 * ux, 0.98 * uy  # a stray factor in the Eq. 18 denominator

    monkeypatch.setattr(fl, "velocity", wrong)


def _mut_minv_transposed(monkeypatch):
    monkeypatch.setattr(fl, "M_INV", np.linalg.inv(fl.M).T.copy())


def _mut_bb_weights(monkeypatch):
    monkeypatch.setattr(fl, "W", np.full(8, 1.0 / 9.0))  # diagonal links with the axis weight


def _mut_pressure_s0(monkeypatch):
    def wrong(f, ux, uy, phi, rho0):
        s0 = fl.W0 * (+1.5 * (ux * ux + uy * uy) / phi)  # sign of s0 flipped
        return fl.C_S2 / (phi * (1.0 - fl.W0)) * (f.sum(axis=0) + rho0 * s0)

    monkeypatch.setattr(fl, "pressure", wrong)


def _mut_meq_gamma(monkeypatch):
    monkeypatch.setattr(fl, "GAMMA1", 1.0)  # p_xx equilibrium coefficient


def _mut_drag_phi(monkeypatch):
    orig = fl.body_force

    def wrong(ux, uy, phi, K, nu, forchheimer, ax, ay):
        Fx, Fy = orig(ux, uy, phi, K, nu, forchheimer, ax, ay)
        return Fx + 0.0 * (phi * ax) - 0.5 * phi * ax, Fy - 0.5 * phi * ay  # half the body force

    monkeypatch.setattr(fl, "body_force", wrong)


def _mut_opposite(monkeypatch):
    opp = fl.OPP.copy()
    opp[4], opp[5] = opp[5], opp[4]  # e5 bounced into e8 instead of e7
    monkeypatch.setattr(fl, "OPP", opp)


def _mut_nee_neighbour_velocity(monkeypatch):
    """Wall nodes that ignore the walls' velocities (a moving lid treated as fixed)."""
    orig_nodes = fl.wall_nodes

    def wrong_nodes(f, flow, phi=None, K=None):
        import dataclasses
        return orig_nodes(f, dataclasses.replace(flow, u_top=(0.0, 0.0), u_bottom=(0.0, 0.0)), phi, K)

    monkeypatch.setattr(fl, "wall_nodes", wrong_nodes)


@pytest.mark.parametrize(
    "mutation",
    [_mut_forcing_sign, _mut_l0, _mut_minv_transposed, _mut_bb_weights, _mut_pressure_s0, _mut_meq_gamma, _mut_drag_phi,
     _mut_opposite, _mut_nee_neighbour_velocity],
)
def test_flow_pins_catch_planted_mistake(monkeypatch, mutation):
    mutation(monkeypatch)
    with np.errstate(all="ignore"):
        assert _caught(FLOW_PINS), mutation.__name__


def _mut_thermal_flux(monkeypatch):
    orig = th.equilibrium_moments

    def wrong(T, ux, uy, p):
        n = orig(T, ux, uy, p)
        n[1] = 0.5 * n[1]  # u_x T / sigma halved
        return n

    monkeypatch.setattr(th, "equilibrium_moments", wrong)


def _mut_thermal_antibb(monkeypatch):
    orig = th.Thermal.rest_weights
    monkeypatch.setattr(th.Thermal, "rest_weights", lambda self: 1.1 * orig(self))


def _mut_thermal_rate(monkeypatch):
    orig = th.Thermal.rates
    monkeypatch.setattr(th.Thermal, "rates", lambda self: orig(self)[[0, 3, 3, 3, 4]])


def _mut_buoyancy_sign(monkeypatch):
    """a = -g beta (T - T0) j: gravity taken along +y."""
    from dataclasses import replace

    def wrong(flow, p, T):
        ax0, ay0 = fl._accel(flow, T)
        return replace(flow, accel=np.stack([ax0 + 0.0 * T, ay0 - p.g_beta * (T - p.T0)]))

    monkeypatch.setattr(th, "_buoyant", wrong)


@pytest.mark.parametrize("mutation", [_mut_thermal_flux, _mut_thermal_antibb, _mut_thermal_rate, _mut_buoyancy_sign])
def test_thermal_pins_catch_planted_mistake(monkeypatch, mutation):
    mutation(monkeypatch)
    with np.errstate(all="ignore"):
        assert _caught(THERMAL_PINS), mutation.__name__


def test_unmutated_oracle_passes_the_same_pins():
    assert not _caught(FLOW_PINS)
    assert not _caught(THERMAL_PINS)
