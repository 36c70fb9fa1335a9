"""Tile shapes and the autotuner (no counterpart in the paper): the determinant kernels' CTA
size changes no bit of the results (one matrix per warp either way); dq_autotune reports the
tile set it chose through dq_tile_set and caches it per configuration, so that a second handle
of the same molecule, ansatz shape, precision and walker count takes the cached set without
timing; the batch autotuner reports its set through dq_multi_tile_set."""
import pytest
import torch

from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()


def _inputs(system, cfg, B, seed=5):
    th = torch.tensor(fx.init_params(system, cfg, seed), dtype=torch.float32, device="cuda:0")
    r = torch.tensor(fx.init_walkers(system, B, seed + 1), dtype=torch.float32, device="cuda:0")
    return th, r


@pytest.mark.parametrize("mol,full", [("N2", 0), ("C2H4", 1), ("C6H6", 0)])
def test_det_warps_bit_identical(mol, full):
    """7 x 7 (small-block body), 16 x 16 (large body, two column groups), 21 x 21 (large body,
    column chunks): 2 and 4 warps per CTA give the same bits, also with a ragged last CTA."""
    import dataclasses

    from paper_2307_14123_gb300 import Ansatz
    system = fx.molecule(mol)
    cfg = dataclasses.replace(fx.AnsatzCfg(32, 2, 3), full_det=full)
    h = Ansatz(system, cfg, "fp32", device="cuda:0")
    th, r = _inputs(system, cfg, 7)
    a = h.local_energy(th, r)
    h.set_det_warps(2)
    assert h.tile_set()["det_warps"] == 2
    b = h.local_energy(th, r)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    from paper_2307_14123_gb300.binding import DQError
    with pytest.raises(DQError):
        h.set_det_warps(3)


def test_autotune_reports_and_caches():
    from paper_2307_14123_gb300 import Ansatz
    wl = fx.workload("n2_fp32")
    th, r = _inputs(wl.system, wl.cfg, 1024)
    h1 = Ansatz(wl.system, wl.cfg, "fp32", device="cuda:0")
    ms1, chunk1, ib1 = h1.autotune(th, r)
    ts1 = h1.tile_set()
    assert ms1 > 0 and ts1["max_chunk"] == chunk1 and ts1["msg_ib"] == ib1
    assert ts1["layer_kernel"] in (1, 2) and ts1["det_warps"] in (2, 4)
    h2 = Ansatz(wl.system, wl.cfg, "fp32", device="cuda:0")
    ms2, _, _ = h2.autotune(th, r)
    assert ms2 == ms1  # the cached time: no new timing
    assert h2.tile_set() == ts1
    # a different walker count is a different key: timed again
    ms3, _, _ = Ansatz(wl.system, wl.cfg, "fp32", device="cuda:0").autotune(th, r[:512])
    assert ms3 != ms1
    la1 = h1.local_energy(th, r)
    la2 = h2.local_energy(th, r)
    for x, y in zip(la1, la2):
        assert torch.equal(x, y)


def test_batch_tile_set():
    from paper_2307_14123_gb300 import AnsatzBatch
    wls = fx.batch_workload("mixed_fp32")[:3]
    batch = AnsatzBatch([w.system for w in wls], [w.cfg for w in wls], "fp32", device="cuda:0")
    th = [torch.tensor(fx.init_params(w.system, w.cfg, w.param_seed), dtype=torch.float32, device="cuda:0")
          for w in wls]
    r = [torch.tensor(fx.init_walkers(w.system, 256, w.walker_seed), dtype=torch.float32, device="cuda:0")
         for w in wls]
    before = [e.clone() for e in batch.local_energy(th, r)[2]]
    ms, rounds, ib = batch.autotune(th, r)
    ts = batch.tile_set()
    assert ts["rounds"] == rounds and ts["msg_ib"] == ib and ts["det_warps"] in (2, 4)
    assert ts["fused_layers"] == 3  # H2O, NH3, C2H4 all run the fused layer kernel
    after = batch.local_energy(th, r)[2]
    for x, y in zip(before, after):  # tile shapes change no bit (per-walker arithmetic in fixed orders)
        assert torch.equal(x, y)
