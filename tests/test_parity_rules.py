"""The top-K comparison rule of the parity tests, checked on hand-made lists
(no GPU): planted mistakes must fail it and legitimate near-tie orders pass."""
import numpy as np
import pytest

from tests.parity import assert_scores, assert_topk, near_tie_groups, rank_order


def test_rank_order_ties_by_id():
    assert rank_order([5, 3, 9, 1], [1.0, 2.0, 1.0, 2.0]).tolist() == [1, 3, 5, 9]


def test_groups():
    s = [3.0, 3.0 * (1 - 1e-14), 2.0, 1.0, 1.0, 0.0]
    assert near_tie_groups(s).tolist() == [0, 0, 1, 2, 2, 3]


def test_exact_order_passes_and_reports_no_groups():
    ref = np.array([0.5, 0.9, 0.1, 0.7, 0.3])
    assert assert_topk([1, 3, 0], np.arange(5), ref, 3) == (0, 0)


def test_swap_outside_a_group_fails():
    ref = np.array([0.5, 0.9, 0.1, 0.7, 0.3])
    with pytest.raises(AssertionError):
        assert_topk([3, 1, 0], np.arange(5), ref, 3)


def test_wrong_member_fails():
    ref = np.array([0.5, 0.9, 0.1, 0.7, 0.3])
    with pytest.raises(AssertionError):
        assert_topk([1, 3, 4], np.arange(5), ref, 3)


def test_near_tie_swap_passes():
    ref = np.array([0.5, 0.9, 0.9 * (1 - 1e-14), 0.7, 0.3])
    assert assert_topk([2, 1, 3], np.arange(5), ref, 3) == (1, 2)


def test_boundary_group_may_hold_any_member():
    ref = np.array([0.9, 0.5, 0.5 * (1 + 1e-14), 0.5 * (1 - 1e-14), 0.1])
    assert assert_topk([0, 3], np.arange(5), ref, 2)[0] == 1
    with pytest.raises(AssertionError):
        assert_topk([0, 4], np.arange(5), ref, 2)


def test_gpu_id_without_oracle_score_fails():
    with pytest.raises(AssertionError):
        assert_topk([7, 1], np.arange(3), np.array([0.1, 0.5, 0.2]), 2)


def test_scores_rule():
    assert assert_scores([1.0, 0.0, 2.0], [1.0 + 1e-13, 0.0, 2.0]) < 1e-12
    with pytest.raises(AssertionError):
        assert_scores([1.0, 1e-300, 2.0], [1.0, 0.0, 2.0])
    with pytest.raises(AssertionError):
        assert_scores([1.0], [1.0 + 1e-11])
