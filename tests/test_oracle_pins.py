"""The CPU oracle against facts that do not come from the oracle itself."""
import pytest

import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(lib, pin):
    pin(lib)


def test_golden_fixture_shape():
    rules, h, expect = P.parse_golden()
    assert len(rules) == 7 and len(expect) == len(h["src"]) >= 20
    # the fixture exercises every rule and default deny
    got = {e[0] for e in expect}
    assert got >= set(range(7)) | {-1}
