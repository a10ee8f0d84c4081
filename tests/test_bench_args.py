"""bench.py's options (CPU): the chosen form's solver decides its default
lookahead and factorisation CTAs per SM, explicit values win, and the
warm-up floor of three steps is enforced."""
import pytest

import bench


def test_headline_defaults():
    a = bench.parse_args([])
    assert (a.solver, a.lookahead, a.factor_ctas_per_sm) == ("mixed_inv", 8, 2)
    assert a.gpus == 1 and a.impl == "ours" and a.warmup >= 3


@pytest.mark.parametrize("solver", ["mixed", "mixed_tc"])
def test_other_forms_defaults(solver):
    a = bench.parse_args(["--solver", solver])
    assert (a.lookahead, a.factor_ctas_per_sm) == (6, 1)


def test_explicit_values_win():
    a = bench.parse_args(["--lookahead", "0", "--factor-ctas-per-sm", "0"])
    assert (a.lookahead, a.factor_ctas_per_sm) == (0, 0)
    a = bench.parse_args(["--solver", "mixed", "--lookahead", "3", "--factor-ctas-per-sm", "2"])
    assert (a.lookahead, a.factor_ctas_per_sm) == (3, 2)


def test_warmup_floor():
    with pytest.raises(SystemExit):
        bench.parse_args(["--warmup", "2"])


def test_every_solver_has_a_form_description():
    assert set(bench.FORM_OF_SOLVER) == {"mixed", "mixed_tc", "mixed_inv"}
