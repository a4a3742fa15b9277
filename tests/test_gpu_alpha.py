"""The alpha heuristic of Sec. 3.7 on the device solver (emu_alpha_sweep):
the Newton count grows with alpha, the chosen value follows the rule on the
counts the sweep tallied (the oracle's pick_alpha applied to them), and it
lies within one step of the value the oracle's own sweep picks (the two
searches differ in their line searches, so their counts differ)."""
import math

import numpy as np
import pytest

from emu_inputs import box_beam
from oracle import OracleParams
from oracle.alpha import alpha_sweep as oracle_sweep, pick_alpha

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def emu():
    import torch

    assert torch.cuda.is_available()
    from paper_2006_08821_gb300 import build as b

    b.build()
    import paper_2006_08821_gb300 as emu

    emu.load_library()
    return emu


@pytest.mark.parametrize("precision", [0, 1])
def test_sweep_follows_the_rule_and_agrees_with_the_oracle(emu, precision):
    mesh = box_beam(2, 2, 4, activation=0.5)
    p = emu.Params(tol_rel_residual=1e-6, precision=precision, max_newton=1500)
    a, alphas, iters = emu.alpha_sweep(mesh, 0.5, params=p, max_steps=4, jump=3.0)
    assert len(alphas) == len(iters) >= 2 and alphas[0] == 1.0
    counted = [i for i in iters if i >= 0]
    assert all(y > x for x, y in zip(counted, counted[1:]))
    ref = pick_alpha(alphas, [i if i >= 0 else None for i in iters], 3.0)
    assert (a, alphas.index(a)) == ref
    ao, _, _ = oracle_sweep(mesh, 0.5, max_steps=4, jump=3.0, max_newton=1500,
                            params=OracleParams(weight_mode=0, ls_sigma0=1.0))
    assert abs(math.log10(a) - math.log10(ao)) <= 1.0 + 1e-12, (a, iters, ao)


def test_sweep_rejects_bad_arguments(emu):
    mesh = box_beam(1, 1, 2)
    with pytest.raises(emu.EmuError) as e:
        emu.alpha_sweep(mesh, 0.5, factor=1.0)
    assert e.value.code == -1
