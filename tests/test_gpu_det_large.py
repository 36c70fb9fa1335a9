"""Determinant jets of the FP32 modes for blocks of 9 to 28 electrons (Eq. 21 and, with
the full determinant, Eq. 22): the FP32 LU with a refined double-float inverse and the
double-float tangent products in the large-block layout, against the FP64 oracle.

Cases cover every column-group layout of that path: 10 x 10 (three column groups per
warp, H2O full determinant), 14 x 14 (two groups, N2 full determinant), 16 x 16 (two
groups of eight, C2H4 full determinant), 21 x 21 (one group in three column chunks,
benzene spin blocks) and 28 x 28 (four chunks, C4H4 full determinant).  Bounds: the
FP32 contract of tests/fp32_contract.py.  Matrices whose FP32 inverse refines to 1e-8
stay off the FP64 path (dq_fp64_matrix_count)."""
import dataclasses
import os

import numpy as np
import pytest
import torch

import oracle
from fp32_contract import check_fp32_oracle
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()
    oracle.build()
    oracle.Oracle.set_threads(os.cpu_count() or 1)


CASES = {  # molecule, full determinant, walkers
    "h2o_full_10": ("H2O", 1, 24),
    "n2_full_14": ("N2", 1, 16),
    "c2h4_full_16": ("C2H4", 1, 12),
    "c6h6_21": ("C6H6", 0, 6),
    "c4h4_full_28": ("C4H4", 1, 4),
}


@pytest.mark.parametrize("case", list(CASES))
def test_large_blocks_fp32_against_oracle(case):
    from paper_2307_14123_gb300 import Ansatz
    mol, full, B = CASES[case]
    system = fx.molecule(mol)
    cfg = dataclasses.replace(fx.AnsatzCfg(32, 2, 2), full_det=full)
    h = Ansatz(system, cfg, "fp32", device="cuda:0")
    theta = fx.init_params(system, cfg, 5).astype(np.float32).astype(np.float64)
    r = fx.init_walkers(system, B, 6).astype(np.float32).astype(np.float64)
    h.fp64_matrix_count()  # clear
    la, sg, el = h.local_energy(torch.tensor(theta, dtype=torch.float32, device="cuda:0"),
                                torch.tensor(r, dtype=torch.float32, device="cuda:0"))
    n64 = h.fp64_matrix_count()
    n_mat = B * cfg.n_det * (1 if full else 2)
    print(f"{case}: {n64} of {n_mat} matrices on the FP64 path")
    assert h.device_status() & 0x4 == 0
    o = oracle.Oracle(system, cfg)
    check_fp32_oracle(f"{case} FP32", la.cpu().numpy(), sg.cpu().numpy(), el.cpu().numpy(), o, theta, r,
                      max_exception_frac=0.25)
    # random-initialised blocks are often ill-conditioned (most 28 x 28 ones here), but the
    # FP32 path must carry at least a quarter of the matrices
    assert n64 <= (3 * n_mat) // 4


def test_large_blocks_deterministic_and_chunked():
    """Benzene spin blocks (21 x 21): bit-identical results from two calls and from walker
    chunks of 5 (ragged last chunk) against one chunk."""
    from paper_2307_14123_gb300 import Ansatz
    system = fx.molecule("C6H6")
    cfg = fx.AnsatzCfg(32, 2, 2)
    h = Ansatz(system, cfg, "fp32", device="cuda:0")
    th = torch.tensor(fx.init_params(system, cfg, 5), dtype=torch.float32, device="cuda:0")
    r = torch.tensor(fx.init_walkers(system, 13, 7), dtype=torch.float32, device="cuda:0")
    a = h.local_energy(th, r)
    b = h.local_energy(th, r)
    h.set_max_chunk(5)
    c = h.local_energy(th, r)
    for x, y, z in zip(a, b, c):
        assert torch.equal(x, y) and torch.equal(x, z)
