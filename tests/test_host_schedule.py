"""Host logic of the library (no GPU): the greedy Givens schedule that the
Givens panel uploads (ssv_givens_schedule) against the paper's worked example
and against the oracle's independent implementation of Algorithm 9."""
import pytest

from oracle.givens import greedy_schedule
from paper_1708_06290_gb300 import ssv
from tests.test_oracle_pins import _golden_schedule


def test_library_schedule_is_the_papers_figure():
    assert ssv.givens_schedule(8, 6) == [rots for _, rots in _golden_schedule()]


@pytest.mark.parametrize("rows,m", [(1, 1), (3, 1), (5, 2), (16, 16), (32, 16), (32, 32), (7, 12), (32, 8)])
def test_library_schedule_equals_the_oracle(rows, m):
    assert ssv.givens_schedule(rows, m) == greedy_schedule(rows, rows + m)


def test_bad_sizes_are_refused():
    with pytest.raises(ssv.SsvError):
        ssv.givens_schedule(0, 4)


def test_library_schedule_equals_the_oracle_on_every_small_shape():
    # the library's column-frontier formulation and the oracle's label-based
    # one are written independently; they must agree on every block shape
    for rows in range(1, 25):
        for m in range(1, 13):
            assert ssv.givens_schedule(rows, m) == greedy_schedule(rows, rows + m), (rows, m)
