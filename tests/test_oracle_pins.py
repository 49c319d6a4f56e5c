"""The FP64 oracle against the lattice table, exact identities, conservation
laws, symmetries and closed-form flows (CPU only)."""
import os

import pytest

import oracle_pins as P


def test_lattice_table_matches_textbook(orc, golden_dir):
    P.check_lattice_table(orc, os.path.join(golden_dir, "d3q19_lattice.txt"))


def test_textbook_table_isotropy(golden_dir):
    P.check_rational_identities(os.path.join(golden_dir, "d3q19_lattice.txt"))


@pytest.mark.parametrize("check", P.ALL_ORACLE_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(orc, check):
    check(orc)
