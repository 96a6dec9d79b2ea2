"""The FP64 oracle against closed forms, invariants, textbook formulas and brute force
(no GPU).  The pins themselves live in pins.py so that the mutation test can run them
against deliberately broken copies of the oracle."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_FAST, ids=lambda f: f.__name__)
def test_pin(ref, pin):
    pin(ref)


def test_brute_force_mpmath(ref):
    pytest.importorskip("mpmath")
    pins.pin_brute_force(ref)


@pytest.mark.parametrize("pin", pins.ALL_MPMATH, ids=lambda f: f.__name__)
def test_pin_mpmath(ref, pin):
    pytest.importorskip("mpmath")
    pin(ref)
