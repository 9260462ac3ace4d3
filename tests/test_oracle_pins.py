"""The CPU oracle against what the paper and plain mathematics fix (no GPU)."""
import pytest

import oracle
import oracle_pins


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(oracle.default())


def test_paper_literal_bound_skips_bit_31():
    # The paper's loop stops before the sign bit (t-1 passes).  For uint32
    # keys that leaves bit 31 unexamined: 2^31 and 1 come out in input order.
    o = oracle.default()
    assert o.paper_sort_u32([0x80000000, 1], 31).tolist() == [0x80000000, 1]
    assert o.paper_sort_u32([0x80000000, 1], 32).tolist() == [1, 0x80000000]
    # below 2^31 the literal bound already sorts
    assert o.paper_sort_u32([5, 0x7FFFFFFF, 3], 31).tolist() == [3, 5, 0x7FFFFFFF]
