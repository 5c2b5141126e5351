"""The SH layout choice and conversion of the Python layer (host logic, no
GPU): layout 1 is picked exactly when the degree in use reads fewer
coefficients than are stored, and [N][K][3] <-> [K][N][3] round-trips."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_09277_gb300.rasterize import sh_layout_for, sh_to_layout


@pytest.mark.parametrize("deg,stride,want", [(0, 16, 1), (1, 16, 1), (2, 16, 1), (3, 16, 0),
                                             (0, 1, 0), (1, 4, 0), (2, 9, 0), (1, 9, 1)])
def test_layout_follows_the_coefficients_in_use(deg, stride, want):
    assert sh_layout_for(deg, stride) == want


def test_coefficient_major_conversion():
    rng = np.random.default_rng(0)
    sh = rng.standard_normal((7, 16, 3)).astype(np.float32)
    assert sh_to_layout(sh, 0) is sh
    cm = np.ascontiguousarray(sh_to_layout(sh, 1))
    assert cm.shape == (16, 7, 3)
    # value (g, k, c) sits at (k * N + g) * 3 + c of the flat array
    flat = cm.reshape(-1)
    for g, k, c in [(0, 0, 0), (6, 15, 2), (3, 7, 1)]:
        assert flat[(k * 7 + g) * 3 + c] == sh[g, k, c]
    t = torch.as_tensor(sh)
    assert torch.equal(sh_to_layout(t, 1).transpose(0, 1), t)
