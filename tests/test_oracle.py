"""CPU pins of the FP64 oracle (run without a GPU).

Each test runs one pin from ``oracle_pins``; see that module for what each
pin checks and which passage of the paper or which mathematical fact fixes it.
"""

import pytest

import oracle_pins


@pytest.mark.parametrize("name", sorted(oracle_pins.PINS))
def test_pin(name, oracle_mod):
    oracle_pins.PINS[name]()
