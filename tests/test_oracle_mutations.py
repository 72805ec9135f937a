"""Mistakes planted in the oracle's arithmetic (a mutated copy of one
function, on the CPU) must be caught by the pins that claim to catch them."""
import inspect

import pytest

import test_oracle_initial as init_pins
from oracle import coupled, project


def _mutant(module, name, old, new):
    """``module.name`` with the source text ``old`` replaced by ``new``."""
    src = inspect.getsource(getattr(module, name))
    assert src.count(old) == 1, old
    ns = dict(module.__dict__)
    exec(compile(src.replace(old, new), f"<mutant of {name}>", "exec"), ns)
    return ns[name]


def test_transposed_g_in_the_state_projection_is_caught(monkeypatch):
    init_pins.test_state_projection_inverts_the_reconstruction()
    bad = _mutant(project, "project_state", "G[j] @ Y[", "G[j].T @ Y[")
    monkeypatch.setattr(project, "project_state", bad)
    with pytest.raises(AssertionError):
        init_pins.test_state_projection_inverts_the_reconstruction()


def test_wrong_sign_of_the_half_step_start_is_caught(monkeypatch):
    fixture = init_pins.coupled_small.__wrapped__()
    init_pins.test_eigenmode_start_follows_the_discrete_cosine_and_sine(fixture)
    bad = _mutant(coupled, "step_structured", "dX -= 0.5 * dt * dt * accel(",
                  "dX += 0.5 * dt * dt * accel(")
    monkeypatch.setattr(coupled, "step_structured", bad)
    with pytest.raises(AssertionError):
        init_pins.test_eigenmode_start_follows_the_discrete_cosine_and_sine(fixture)


def test_dropped_lower_flux_in_the_interior_update_is_caught(monkeypatch):
    fixture = init_pins.coupled_small.__wrapped__()
    bad = _mutant(coupled, "step_structured", "phi[:, 1:] - phi[:, :-1] + src[:, 1:]",
                  "phi[:, 1:] + src[:, 1:]")
    monkeypatch.setattr(coupled, "step_structured", bad)
    with pytest.raises(AssertionError):
        init_pins.test_initial_value_stepping_equals_the_assembled_leapfrog(fixture)


def test_wrong_sign_in_the_gamma_recursion_is_caught(monkeypatch):
    """Eq. 13 with +Gamma_{j-1} instead of -Gamma_{j-1}: the block chain no
    longer returns its blocks."""
    import test_oracle_sfrac as sfrac_pins
    from oracle import sfrac
    sfrac_pins.test_block_chain_gives_back_its_blocks()
    bad = _mutant(sfrac, "gamma_transform", "Gi.T @ alpha[j] @ Gi - prev", "Gi.T @ alpha[j] @ Gi + prev")
    monkeypatch.setattr(sfrac, "gamma_transform", bad)
    with pytest.raises(Exception):
        sfrac_pins.test_block_chain_gives_back_its_blocks()


def test_wrong_edge_conductance_is_caught(monkeypatch):
    """h/2 instead of h/4 per cell edge: the interior rows are no longer the
    7-point Laplacian c^2 Delta_h."""
    import test_oracle_fine as fine_pins
    from oracle import fine
    fine_pins.test_uniform_interior_rows_are_7_point_laplacian()
    bad = _mutant(fine, "assemble", "np.full(ci.shape, h / 4.0)", "np.full(ci.shape, h / 2.0)")
    monkeypatch.setattr(fine, "assemble", bad)
    with pytest.raises(AssertionError):
        fine_pins.test_uniform_interior_rows_are_7_point_laplacian()


@pytest.mark.slow
def test_arithmetic_instead_of_harmonic_face_coupling_is_caught(monkeypatch):
    """H_f = (sum of the sides' blocks)^{-1} instead of (sum of their
    inverses)^{-1}: the ROM no longer converges to the slit fine grid."""
    import test_oracle_coupled as coupled_pins
    bad = _mutant(coupled, "face_H", "acc = acc + np.linalg.inv(rs.Gammahat[s][0][sl, sl])",
                  "acc = acc + rs.Gammahat[s][0][sl, sl]")
    monkeypatch.setattr(coupled, "face_H", bad)
    with pytest.raises(AssertionError):
        coupled_pins.test_rom_converges_to_the_slit_fine_grid()


def test_wrong_sign_of_the_fine_half_step_start_is_caught(monkeypatch):
    import test_oracle_fine as fine_pins
    from oracle import fine
    fine_pins.test_fine_initial_value_start_follows_the_discrete_cosine_and_sine()
    bad = _mutant(fine, "leapfrog", "v -= 0.5 * dt * dt * minv", "v += 0.5 * dt * dt * minv")
    monkeypatch.setattr(fine, "leapfrog", bad)
    with pytest.raises(AssertionError):
        fine_pins.test_fine_initial_value_start_follows_the_discrete_cosine_and_sine()


def test_one_shift_for_every_block_is_caught(monkeypatch):
    """Distinct shifts (Eq. 6) collapsed to the first one: the ROM no longer
    interpolates the NtD map at the other shifts."""
    import test_oracle_multishift as ms_pins
    from oracle import pipeline
    ms_pins.test_interpolates_the_ntd_map_and_its_derivative_at_every_shift(ms_pins.multi.__wrapped__())
    bad = _mutant(pipeline, "SubdomainROM", "solve = [cache[x] for x in shifts]",
                  "solve = [cache[shifts[0]] for x in shifts]")
    monkeypatch.setattr(pipeline, "SubdomainROM", bad)
    with pytest.raises(AssertionError):
        ms_pins.test_interpolates_the_ntd_map_and_its_derivative_at_every_shift(
            ms_pins.multi.__wrapped__())
