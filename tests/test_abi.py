"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol that include/dqmc.h declares; the binding refuses to run without a GPU
(there is no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dqmc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s+([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_14123_gb300 import _build
    _build.build()
    from paper_2307_14123_gb300 import binding
    return binding.load_library()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("ansatz_eval", "local_energy", "mcmc_step", "grad_logpsi", "vmc_loss_weights", "dq_create"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2307_14123_gb300 import binding
    names = declared_functions()
    assert sorted(binding.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_status_strings(lib):
    lib.dq_status_string.restype = ctypes.c_char_p
    assert lib.dq_status_string(0) == b"ok"
    assert b"workspace" in lib.dq_status_string(5)


def test_null_arguments_are_rejected_without_touching_the_device(lib):
    assert lib.dq_create(None, None, 1, None) == 1
    assert lib.dq_param_count(None, None) == 1
    assert lib.dq_destroy(None) == 1


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the behaviour without a GPU")
def test_no_cpu_fallback():
    from paper_2307_14123_gb300 import Ansatz, DQError
    from paper_2307_14123_gb300 import fixtures as fx
    wl = fx.workload("lih_fp64")
    with pytest.raises(DQError):
        Ansatz(wl.system, wl.cfg, "fp64")


def test_full_determinant_arguments_are_checked_on_the_host(lib):
    """full_det must be 0 or 1, and the full determinant needs N <= 32; both are refused before
    any device call (these run without a GPU)."""
    import numpy as np

    from paper_2307_14123_gb300 import binding
    from paper_2307_14123_gb300 import fixtures as fx
    for mol, full, want in (("C6H6", 1, 2), ("N2", 2, 1)):
        s = fx.molecule(mol)
        Z = np.ascontiguousarray(s.Z, dtype=np.float64)
        R = np.ascontiguousarray(s.R, dtype=np.float64)
        sysc = binding._System(len(Z), Z.ctypes.data, R.ctypes.data, s.n_up, s.n_down)
        cfgc = binding._Cfg(32, 1, 1, 16, 10.0, 1, 1, 1.0, full, 0, 0)
        h = ctypes.c_void_p()
        assert lib.dq_create(ctypes.byref(sysc), ctypes.byref(cfgc), 1, ctypes.byref(h)) == want
        assert not h.value


def test_electron_nucleus_embedding_flag_is_checked_on_the_host(lib):
    """el_init outside {0, 1} is an argument error, returned before any device call."""
    import numpy as np

    from paper_2307_14123_gb300 import binding
    from paper_2307_14123_gb300 import fixtures as fx
    s = fx.molecule("LiH")
    Z = np.ascontiguousarray(s.Z, dtype=np.float64)
    R = np.ascontiguousarray(s.R, dtype=np.float64)
    sysc = binding._System(len(Z), Z.ctypes.data, R.ctypes.data, s.n_up, s.n_down)
    cfgc = binding._Cfg(32, 2, 1, 16, 10.0, 1, 1, 1.0, 0, 0, 2)
    h = ctypes.c_void_p()
    assert lib.dq_create(ctypes.byref(sysc), ctypes.byref(cfgc), 1, ctypes.byref(h)) == 1 and not h.value


def test_bf16_mode_needs_width_multiple_of_64(lib):
    """The BF16 embedding GEMMs take K = D and 3D in 64-wide tiles: dq_create refuses other widths
    in that mode (DQ_ERR_SHAPE) before any device call."""
    import numpy as np

    from paper_2307_14123_gb300 import binding
    from paper_2307_14123_gb300 import fixtures as fx
    s = fx.molecule("LiH")
    Z = np.ascontiguousarray(s.Z, dtype=np.float64)
    R = np.ascontiguousarray(s.R, dtype=np.float64)
    sysc = binding._System(len(Z), Z.ctypes.data, R.ctypes.data, s.n_up, s.n_down)
    cfgc = binding._Cfg(96, 2, 1, 16, 10.0, 1, 1, 1.0, 0, 0, 0)
    h = ctypes.c_void_p()
    assert lib.dq_create(ctypes.byref(sysc), ctypes.byref(cfgc), 2, ctypes.byref(h)) == 2 and not h.value
