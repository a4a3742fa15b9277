"""The alpha heuristic of Sec. 3.7 on the oracle: the selection rule on
hand-made tallies, and a sweep on a small beam, where the Newton count must
grow with alpha (a stiffer penalty, the paper's observation) and the choice
must follow the rule on the counts the sweep tallied."""
from emu_inputs import box_beam
from oracle import OracleParams
from oracle.alpha import alpha_sweep, pick_alpha


def test_rule_takes_the_value_before_the_first_sharp_increase():
    alphas = [1.0, 10.0, 100.0, 1000.0, 1e4]
    assert pick_alpha(alphas, [20, 25, 31, 95, 400], 3.0) == (100.0, 2)
    assert pick_alpha(alphas, [20, 61, 70], 3.0) == (1.0, 0)          # 61 > 3 x 20
    assert pick_alpha(alphas, [20, 60, 70], 3.0) == (100.0, 2)         # exactly 3 x is not above it
    assert pick_alpha(alphas, [20, 22, None], 3.0) == (10.0, 1)        # a failed solve is a jump
    assert pick_alpha(alphas, [20, 22, 25, 27, 30], 3.0) == (1e4, 4)  # no jump: the last value
    assert pick_alpha(alphas[:1], [20], 3.0) == (1.0, 0)


def test_sweep_on_a_beam_counts_more_iterations_at_higher_alpha():
    mesh = box_beam(2, 2, 4, activation=0.5)
    a, alphas, iters = alpha_sweep(mesh, 0.5, max_steps=4, jump=3.0, max_newton=1500,
                                   params=OracleParams(weight_mode=0, ls_sigma0=1.0))
    assert alphas[0] == 1.0 and all(b == 10.0 * x for x, b in zip(alphas, alphas[1:]))
    counted = [i for i in iters if i is not None]
    assert all(y > x for x, y in zip(counted, counted[1:]))  # stiffer penalty, more Newton iterations
    assert (a, alphas.index(a)) == pick_alpha(alphas, iters, 3.0)
