"""Plan construction on the host (no kernel runs): bt_plan_workspace_size
measures a plan's device memory through the same layout the plans use, so the
planner's structure and its argument checks are testable without a GPU."""
import pytest


def _ws(kind, n, m, nr=1, prec="fp64", tuning=None):
    import paper_0912_3678_gb300 as bt
    return bt.bt_plan_workspace_size(kind, n, m, nr, prec, tuning)


def test_babd_cyclic_reduction_refuses_unsupported_blocks_and_precisions():
    import paper_0912_3678_gb300 as bt
    for m, prec in ((4, "fp64"), (2, "fp64"), (8, "fp32_ir"), (16, "bf16_ir"), (12, "fp64")):
        with pytest.raises(bt.BtError):
            _ws(1, 1000, m, 1, prec, {"reduced": 1})


def test_babd_cyclic_reduction_memory_is_linear_in_n():
    """Levels of N, N/2, N/4, ... rows: the factor storage is about twice the
    first level's, so doubling N doubles the plan."""
    a = _ws(1, 1 << 16, 8, 1, "fp64", {"reduced": 1})
    b = _ws(1, 1 << 17, 8, 1, "fp64", {"reduced": 1})
    assert 1.9 < b / a < 2.1
    # per block row: Rinv, T, S', R' (4 blocks for every pair, summed over the
    # halving levels) plus the boundary copies: between 2 and 6 blocks of m^2 doubles
    per_row = b / (1 << 17) / (8 * 8 * 8)
    assert 2.0 < per_row < 6.0


def test_workspace_grows_with_right_hand_sides():
    for kind, m in ((0, 16), (0, 4), (1, 8)):
        one = _ws(kind, 20000, m, 1)
        many = _ws(kind, 20000, m, 8)
        assert many > one


def test_pivoted_plans_reserve_the_enlarged_reduced_system():
    """A pivoted plan holds room for up to max(2 p0, N/16) + 15 separators,
    so it needs more memory than the plain plan of the same shape."""
    plain = _ws(0, 1 << 20, 1, 1, "fp64", {"p0": 4096})
    piv = _ws(0, 1 << 20, 1, 1, "fp64", {"p0": 4096, "pivot": 1})
    assert piv > plain
