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
