"""Pins of the oracle's unit conversions against published values.

The NVE and Maxwell-Boltzmann tests only see the product of the two
kinetic conversions and the oracle's own k_B; these literals come from the
CODATA 2018 constants and the published metal-unit conversion factors
(tests/golden/units.txt), not from the oracle's formulas, so a wrong atomic
mass unit, Boltzmann constant or pressure unit fails here."""
import pytest

from conftest import golden


@pytest.mark.parametrize("row", golden("units.txt"), ids=lambda r: r[0])
def test_unit_conversion_matches_published_value(oracle, row):
    name, value, tol = row[0], float(row[1]), float(row[2])
    got = oracle.constants()[name]
    assert got == pytest.approx(value, rel=tol)


def test_kinetic_conversions_are_inverse(oracle):
    c = oracle.constants()
    assert c["mv2_to_ev"] * c["force_to_acc"] == pytest.approx(1.0, rel=1e-14)


def test_thermal_energy_at_300K(oracle):
    # k_B T at 300 K = 25.852 meV (textbook room-temperature value)
    assert 300.0 * oracle.constants()["kb_ev"] == pytest.approx(0.025852, rel=2e-5)
