"""The paper-style study's cost model and sum-rate evaluation (host logic, no GPU)."""
import math

import numpy as np
import torch

from paper_2512_16543_gb300 import experiment as ex


def test_op_count_reproduces_the_papers_cost_values():
    # Section V: normalised cost of the proposed method at K = 100 (Fig. 1 / Table IV)
    assert abs(ex.op_count(100, 50, False) / ex.op_count(100, 0, True) - 0.885) < 1e-12
    assert abs(ex.op_count(100, 100, False) / 100 ** 3 - 3.01) < 1e-12
    # K = 16, r = 4: 61 % savings, the scale of Table V at eta = 65 %
    assert abs(1 - ex.op_count(16, 4, False) / 16 ** 3 - 0.609375) < 1e-12


def test_true_sum_rate_single_user_closed_form():
    # K = 1: R = log2(1 + P_t |h f|^2 / sigma^2) whatever the digital precoder's phase
    h = torch.tensor([[[0.3 + 0.4j]]], dtype=torch.complex128)
    F = torch.ones(1, 1, 1, dtype=torch.complex128)
    W = torch.tensor([[[2.0 - 1.0j]]], dtype=torch.complex128)
    R = ex.true_sum_rate(h, F, W, p_t=2.0, sigma2=0.5)
    assert abs(float(R[0]) - math.log2(1 + 2.0 * 0.25 / 0.5)) < 1e-12


def test_true_sum_rate_zero_forcing_has_no_interference():
    rng = np.random.default_rng(3)
    H = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    W = np.linalg.inv(H)                               # H W = I: diagonal gains only
    Ht = torch.from_numpy(H[None])
    F = torch.eye(4, dtype=torch.complex128)[None]
    R = ex.true_sum_rate(Ht, F, torch.from_numpy(W[None]), p_t=1.0, sigma2=0.1)
    s = 1.0 / np.linalg.norm(W)
    assert abs(float(R[0]) - 4 * math.log2(1 + s * s / 0.1)) < 1e-9
