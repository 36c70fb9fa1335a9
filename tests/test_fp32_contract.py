"""Pins of the near-nodal classification used by the FP32 parity contract
(tests/fp32_contract.py): sigma is the first-order sensitivity of log|Psi_D| =
log|sum_p c_p prod_s det A_{p,s}| (Eq. 21) to relative perturbations of the
orbital entries, rho the cancellation ratio of the determinant sum."""
import numpy as np

from fp32_contract import sigma_rho


def _log_psi(mats, c):
    vals = [c[p] * np.prod([np.linalg.det(M) for M in blocks]) for p, blocks in enumerate(mats)]
    return np.log(abs(sum(vals)))


def test_diagonal_and_single_determinant():
    D = np.diag([2.0, -3.0, 0.5])
    sigma, rho = sigma_rho([[D]], [1.0])
    assert sigma == 3.0 and rho == 1.0  # sum_ij |A^-1_ji A_ij| = n for a diagonal matrix


def test_worst_case_perturbation_is_first_order_exact():
    rng = np.random.default_rng(0)
    for n in (2, 4, 7):
        A = rng.normal(size=(n, n))
        B = rng.normal(size=(n, n))
        sigma, _ = sigma_rho([[A, B]], [0.7])
        eps = 1e-7
        # the perturbation that moves every term tr(A^-1 dA) the same way
        pa = A * (1 + eps * np.sign(np.linalg.inv(A).T * A))
        pb = B * (1 + eps * np.sign(np.linalg.inv(B).T * B))
        d = _log_psi([[pa, pb]], [0.7]) - _log_psi([[A, B]], [0.7])
        assert abs(d / (eps * sigma) - 1) < 1e-4


def test_random_perturbations_bounded_by_sigma():
    rng = np.random.default_rng(1)
    mats = [[rng.normal(size=(3, 3)), rng.normal(size=(3, 3))] for _ in range(4)]
    c = rng.normal(size=4)
    sigma, rho = sigma_rho(mats, c)
    assert 0 < rho <= 1
    eps = 1e-8
    for _ in range(20):
        pert = [[M * (1 + eps * rng.uniform(-1, 1, size=M.shape)) for M in blocks] for blocks in mats]
        assert abs(_log_psi(pert, c) - _log_psi(mats, c)) <= eps * sigma * (1 + 1e-6)


def test_cancellation_ratio():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(3, 3))
    delta = 1e-7
    sigma, rho = sigma_rho([[A], [A]], [1.0, -1.0 + delta])
    assert abs(rho - delta / (2 - delta)) < 1e-12
    assert sigma > 1e6  # the weights |c_p det| / |Psi_D| are ~1/delta
    assert sigma_rho([[A], [A]], [1.0, -1.0]) == (np.inf, 0.0)
