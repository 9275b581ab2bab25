"""Host-side helpers of the learned part (no GPU): the bound-margin
calibration and the widening of predicted bounds."""

import torch

from paper_2401_13772_gb300 import learned as L


def test_calibrated_margin_covers_the_overshoot_quantile():
    g = torch.Generator().manual_seed(0)
    T = torch.rand(1000, 2, generator=g) * 0.2
    over = torch.linspace(0.0, 0.1, 1000)
    Y = T.clone()
    Y[:, 0] += over          # predictions above the target by 0 .. 0.1
    Y[:, 1] -= 0.05          # under-shooting is harmless
    m = L.calibrate_margin(Y, T, quantile=0.97, floor=0.0)
    assert abs(m - 0.097) < 1e-3
    covered = (Y[:, 0] - m <= T[:, 0] + 1e-12).double().mean().item()
    assert covered >= 0.97
    assert L.calibrate_margin(T, T, floor=0.02) == 0.02


def test_predicted_bounds_stay_inside_gershgorin():
    emin = torch.tensor([-2.0, -1.0], dtype=torch.float64)
    emax = torch.tensor([2.0, 3.0], dtype=torch.float64)
    Y = torch.tensor([[0.1, 0.2], [0.9, 0.9]])
    b = L.predicted_bounds(Y, emin, emax, 0.05)
    assert torch.allclose(b[0], torch.tensor([-2.0 + 4 * 0.05, 2.0 - 4 * 0.15],
                                             dtype=torch.float64))
    # crossing predictions fall back to the Gershgorin enclosure
    assert torch.equal(b[1], torch.tensor([-1.0, 3.0], dtype=torch.float64))
