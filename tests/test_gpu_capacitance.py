"""The capacitance of the Woodbury direction (Eq. 12, Gram form) on the two
tensor-core kernels of the mixed path, against an FP64 evaluation of its
definition on the same seeded per-tet factors:

  C  = sum_i Yh_i^T Yh_i,  Yh_i[r][16 d + l] = sqrt(w_i) sum_b U_i[r][3 d + b] Gamma_i[b][l]
  By = sum_i w_i sum_b Gamma_i[b][l] y_i[3 d + b]   at entry 16 d + l.

Yh is rounded to TF32 (11-bit significand) before the products, so C is held
to 2e-3 of its largest entry; By runs in FP32 (2e-5). The tcgen05 kernel's C
must be exactly symmetric and positive semi-definite.
"""
import numpy as np
import pytest

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


def factors(m, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((54, m)).astype(np.float32)
    gamma = (rng.standard_normal((48, m)) * 40.0).astype(np.float32)
    y = rng.standard_normal((9, m)).astype(np.float32)
    w = np.exp(rng.uniform(np.log(1e-3), 0.0, m)).astype(np.float32)  # weights over three decades
    return U, gamma, y, w


def reference(U, gamma, y, w):
    m = w.shape[0]
    U6 = U.astype(np.float64).reshape(6, 3, 3, m)        # U_i[r][3 d + b]
    G = gamma.astype(np.float64).reshape(16, 3, m)       # Gamma_i[b][l] at row 3 l + b
    sw = np.sqrt(w.astype(np.float64))
    Yh = np.einsum("rdbi,lbi->irdl", U6, G).reshape(m, 6, 48) * sw[:, None, None]
    Cm = np.einsum("irc,ire->ce", Yh, Yh)
    By = np.einsum("lbi,dbi,i->dl", G, y.astype(np.float64).reshape(3, 3, m), w.astype(np.float64)).reshape(48)
    return Cm, By


@pytest.mark.parametrize("m", [4, 16, 20, 4096, 50000])
@pytest.mark.parametrize("kernel", [1, 2])
def test_capacitance_matches_its_definition(emu, m, kernel):
    U, gamma, y, w = factors(m, seed=m + kernel)
    Cr, Byr = reference(U, gamma, y, w)
    Cm, By = emu.eval_capacitance(U, gamma, y, w, kernel=kernel)
    scale = np.abs(Cr).max()
    err = np.abs(Cm - Cr).max() / scale
    assert err <= 2e-3, (m, kernel, err)
    assert np.abs(By - Byr).max() <= 2e-5 * np.abs(Byr).max(), (m, kernel)
    if kernel == 1:
        np.testing.assert_array_equal(Cm, Cm.T)
        assert np.linalg.eigvalsh(Cm).min() >= -1e-6 * scale


def test_both_kernels_agree_and_the_automatic_choice(emu):
    U, gamma, y, w = factors(12000, seed=7)
    C1, B1 = emu.eval_capacitance(U, gamma, y, w, kernel=1)
    C2, B2 = emu.eval_capacitance(U, gamma, y, w, kernel=2)
    C0, B0 = emu.eval_capacitance(U, gamma, y, w, kernel=0)
    scale = np.abs(C1).max()
    assert np.abs(C1 - C2).max() <= 2e-3 * scale
    np.testing.assert_array_equal(C0, C1)  # m % 4 == 0: the tcgen05 kernel
    np.testing.assert_array_equal(B0, B1)
    # a second call is bitwise the same (fixed reduction order)
    C1b, B1b = emu.eval_capacitance(U, gamma, y, w, kernel=1)
    np.testing.assert_array_equal(C1, C1b)
    np.testing.assert_array_equal(B1, B1b)


def test_ragged_count_takes_the_mma_sync_kernel(emu):
    U, gamma, y, w = factors(1002, seed=3)
    with pytest.raises(emu.EmuError) as e:
        emu.eval_capacitance(U, gamma, y, w, kernel=1)
    assert e.value.code == -1
    C0, _ = emu.eval_capacitance(U, gamma, y, w, kernel=0)
    C2, _ = emu.eval_capacitance(U, gamma, y, w, kernel=2)
    np.testing.assert_array_equal(C0, C2)
    Cr, _ = reference(U, gamma, y, w)
    assert np.abs(C0 - Cr).max() <= 2e-3 * np.abs(Cr).max()
