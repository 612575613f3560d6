"""Full-size check of the CUDA path against the paper's own simulation results
(cases too large for the oracle): drag and lift of a fixed sphere near the
resting wall of a shear flow (Sec. 2.5), at half the paper's resolution
(D = 10 instead of 20, 480 x 160 x 80 cells) so it runs in seconds. The paper
prints C_D = 34.44, C_L = 2.30 for L = 1 and Re = 1 (TRT+aB); the full
resolution run of paper_2003_01490_gb300/validation.py gives 34.47 and 2.302."""
import pytest

pytestmark = pytest.mark.gpu


def test_shear_drag_lift_at_half_resolution():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    from paper_2003_01490_gb300 import validation
    res = validation.shear_drag_lift(1.0, 1.0, D=10.0, storage='f32')
    print(res)
    assert res['converged']
    assert abs(res['C_D'] / 34.44 - 1) < 0.02
    assert abs(res['C_L'] / 2.30 - 1) < 0.03
