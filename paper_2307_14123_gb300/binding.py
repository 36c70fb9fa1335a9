"""Thin ctypes binding of libdqmc (include/dqmc.h).

Argument marshalling only: tensors are checked for device, dtype and
contiguity, their device pointers and the current CUDA stream are handed to
the C ABI, and every step of the computation runs in the library's kernels.
There is no CPU fallback: without the compiled library or a CUDA device every
call raises.

PyTorch provides device memory (outputs and the cached workspace) and
streams.  Host (CPU) tensors are accepted by the methods of :class:`Ansatz`
for an end-to-end call: they are copied to the device from pinned memory,
the library runs, and results are copied back.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdqmc.so")

DQ_FP64, DQ_FP32, DQ_BF16_MIXED = 0, 1, 2
(OP_EVAL, OP_LOCAL_ENERGY, OP_MCMC, OP_GRAD, OP_LOSS_WEIGHTS, OP_MALA, OP_AUTOTUNE, OP_NATGRAD,
 OP_UPDATE) = 0, 1, 2, 3, 4, 5, 6, 7, 8
FLAG_SINGULAR, FLAG_NONFINITE = 0x1, 0x2
CLIP_MODES = {"hard": 0, "log": 1}
PRECISIONS = {"fp64": DQ_FP64, "fp32": DQ_FP32, "bf16": DQ_BF16_MIXED}

# Every symbol declared in include/dqmc.h.
EXPORTS = ["dq_create", "dq_destroy", "dq_param_count", "dq_max_chunk", "dq_set_max_chunk", "dq_workspace_size",
           "ansatz_eval", "local_energy", "mcmc_step", "grad_logpsi", "vmc_loss_weights", "dq_last_device_status",
           "dq_status_string", "dq_profile_enable", "dq_profile_reset", "dq_profile_read", "dq_profile_kind_name",
           "dq_profile_kind_count", "vmc_loss_weights_noalloc", "vmc_loss_weights_clip", "dq_fp64_matrix_count", "dq_test_gemm_bf16",
           "dq_test_gemm_tf32x3", "mcmc_step_dev", "mala_step", "dq_create_multi", "dq_destroy_multi",
           "dq_multi_handle", "dq_multi_set_rounds", "dq_multi_rounds", "dq_multi_workspace_size",
           "ansatz_eval_multi", "local_energy_multi", "mcmc_step_multi", "grad_logpsi_multi",
           "vmc_loss_weights_multi", "dq_autotune_multi", "dq_multi_tuning", "dq_set_msg_tile", "dq_msg_tile", "dq_set_msg_kernel", "dq_msg_kernel", "dq_autotune", "natural_gradient", "param_update", "dq_pp_workspace_size",
           "pseudopotential_energy", "dq_fma_rate_probe", "dq_set_layer_kernel", "dq_layer_kernel",
           "dq_set_det_warps", "dq_tile_set", "dq_multi_tile_set", "mcmc_step_eloc"]


class DQError(RuntimeError):
    pass


class _PP(ctypes.Structure):
    _fields_ = [("nucleus", ctypes.c_int32), ("l_max", ctypes.c_int32), ("n_terms", ctypes.c_int32),
                ("coef", ctypes.c_void_p)]


class _System(ctypes.Structure):
    _fields_ = [("n_nuc", ctypes.c_int32), ("Z", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("n_up", ctypes.c_int32), ("n_down", ctypes.c_int32)]


class _Cfg(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("n_layers", ctypes.c_int32), ("n_det", ctypes.c_int32),
                ("n_rbf", ctypes.c_int32), ("rbf_cutoff", ctypes.c_double), ("use_jastrow", ctypes.c_int32),
                ("use_cusp", ctypes.c_int32), ("cusp_alpha", ctypes.c_double), ("full_det", ctypes.c_int32),
                ("edge_update", ctypes.c_int32), ("el_init", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load_library(path=None):
    """Loads libdqmc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or LIB_PATH
        if not os.path.exists(path):
            raise DQError(f"libdqmc.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, i32, i64, u64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_size_t)
        lib.dq_create.argtypes = [P, P, i32, P]
        lib.dq_destroy.argtypes = [P]
        lib.dq_param_count.argtypes = [P, P]
        lib.dq_max_chunk.argtypes = [P, P]
        lib.dq_set_max_chunk.argtypes = [P, i64]
        lib.dq_workspace_size.argtypes = [P, i64, i32, P]
        lib.ansatz_eval.argtypes = [P, P, P, i64, P, P, P, sz, P]
        lib.local_energy.argtypes = [P, P, P, i64, P, P, P, P, P, sz, P]
        lib.mcmc_step.argtypes = [P, P, P, P, i64, i32, f64, u64, u64, P, P, sz, P]
        lib.mcmc_step_dev.argtypes = [P, P, P, P, i64, i32, f64, u64, P, P, P, sz, P]
        lib.mala_step.argtypes = [P, P, P, P, P, P, i32, i64, i32, f64, u64, u64, P, P, P, sz, P]
        lib.mcmc_step_eloc.argtypes = [P, P, P, P, P, i64, i32, f64, u64, u64, P, P, P, sz, P]
        lib.grad_logpsi.argtypes = [P, P, P, i64, P, i32, P, P, sz, P]
        lib.vmc_loss_weights.argtypes = [P, P, i64, f64, P, P, P, sz, P]
        lib.vmc_loss_weights_noalloc.argtypes = [P, P, i64, f64, P, P, P]
        lib.vmc_loss_weights_clip.argtypes = [P, P, i64, f64, ctypes.c_int32, P, P, P, sz, P]
        lib.dq_last_device_status.argtypes = [P, P, P]
        lib.dq_fp64_matrix_count.argtypes = [P, P, P]
        lib.dq_test_gemm_bf16.argtypes = [P, i64, i32, i64, P, i32, P, i32, P, i64, P, P]
        lib.dq_test_gemm_tf32x3.argtypes = [P, i64, i32, i64, P, i32, P, i32, P, i64, P, P, P]
        lib.dq_status_string.argtypes = [ctypes.c_int]
        lib.dq_profile_enable.argtypes = [P, i32]
        lib.dq_profile_reset.argtypes = [P]
        lib.dq_profile_read.argtypes = [P, i32, P, P]
        lib.dq_profile_kind_name.argtypes = [i32]
        lib.dq_profile_kind_count.argtypes = []
        lib.dq_create_multi.argtypes = [i32, P, P, i32, P]
        lib.dq_destroy_multi.argtypes = [P]
        lib.dq_multi_handle.argtypes = [P, i32, P]
        lib.dq_multi_set_rounds.argtypes = [P, i32]
        lib.dq_multi_rounds.argtypes = [P, P]
        lib.dq_multi_workspace_size.argtypes = [P, P, i32, P]
        lib.ansatz_eval_multi.argtypes = [P, P, P, P, P, P, P, sz, P]
        lib.local_energy_multi.argtypes = [P, P, P, P, P, P, P, P, P, sz, P]
        lib.mcmc_step_multi.argtypes = [P, P, P, P, P, i32, f64, u64, u64, P, P, P, sz, P]
        lib.grad_logpsi_multi.argtypes = [P, P, P, P, P, P, P, sz, P]
        lib.vmc_loss_weights_multi.argtypes = [P, P, P, f64, P, P, P, sz, P]
        lib.dq_autotune_multi.argtypes = [P, P, P, P, P, sz, P, P]
        lib.dq_multi_tuning.argtypes = [P, P, P]
        lib.dq_set_msg_tile.argtypes = [P, i32]
        lib.dq_set_msg_kernel.argtypes = [P, i32]
        lib.dq_msg_kernel.argtypes = [P, ctypes.POINTER(i32)]
        lib.dq_msg_tile.argtypes = [P, P]
        lib.dq_autotune.argtypes = [P, P, P, i64, P, sz, P, P]
        lib.natural_gradient.argtypes = [P, P, P, i64, f64, i32, f64, P, P, P, sz, P]
        lib.param_update.argtypes = [P, P, P, f64, f64, P, P, sz, P]
        lib.dq_pp_workspace_size.argtypes = [P, i64, i32, P]
        lib.pseudopotential_energy.argtypes = [P, P, P, i64, i32, P, P, P, P, P, P, P, sz, P]
        lib.dq_fma_rate_probe.argtypes = [i32, i32, i32, P, P, P]
        lib.dq_set_layer_kernel.argtypes = [P, i32]
        lib.dq_layer_kernel.argtypes = [P, P]
        lib.dq_set_det_warps.argtypes = [P, i32]
        lib.dq_tile_set.argtypes = [P, P, P, P, P]
        lib.dq_multi_tile_set.argtypes = [P, P, P, P, P]
        for name in EXPORTS:
            getattr(lib, name).restype = ctypes.c_int
        lib.dq_status_string.restype = ctypes.c_char_p
        lib.dq_profile_kind_name.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(st):
    if st != 0:
        raise DQError(f"libdqmc: {_lib.dq_status_string(st).decode()} (status {st})")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Ansatz:
    """A handle of the library: one molecule, one ansatz, one precision, one device.

    ``system`` needs ``Z``, ``R`` (bohr), ``n_up``, ``n_down``; ``cfg`` needs
    ``width, n_layers, n_det, n_rbf, rbf_cutoff, use_jastrow, use_cusp,
    cusp_alpha`` and optionally ``full_det``, ``edge_update``, ``el_init`` (see :mod:`paper_2307_14123_gb300.fixtures`).
    """

    def __init__(self, system, cfg, precision="fp32", device=None):
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise DQError("no CUDA device: the library has no CPU path")
        device = torch.device("cuda") if device is None else torch.device(device)
        if device.type != "cuda":
            raise DQError("the library runs on CUDA devices only")
        self.device = torch.device("cuda", torch.cuda.current_device() if device.index is None else device.index)
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.N = int(system.n_up + system.n_down)
        self._Z = (ctypes.c_double * len(system.Z))(*[float(z) for z in system.Z])
        flatR = [float(x) for x in torch.as_tensor(system.R, dtype=torch.float64).reshape(-1).tolist()]
        self._R = (ctypes.c_double * len(flatR))(*flatR)
        sysc = _System(len(system.Z), ctypes.cast(self._Z, ctypes.c_void_p), ctypes.cast(self._R, ctypes.c_void_p),
                       int(system.n_up), int(system.n_down))
        cfgc = _Cfg(int(cfg.width), int(cfg.n_layers), int(cfg.n_det), int(cfg.n_rbf), float(cfg.rbf_cutoff),
                    int(cfg.use_jastrow), int(cfg.use_cusp), float(cfg.cusp_alpha),
                    int(getattr(cfg, "full_det", 0)), int(getattr(cfg, "edge_update", 0)),
                    int(getattr(cfg, "el_init", 0)))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.dq_create(ctypes.byref(sysc), ctypes.byref(cfgc), PRECISIONS[precision], ctypes.byref(h)))
        self.h = h
        P = ctypes.c_int64()
        _check(self.lib.dq_param_count(self.h, ctypes.byref(P)))
        self.P = P.value
        self._ws = None

    def __del__(self):
        if getattr(self, "h", None) and self.lib is not None:
            try:
                self.lib.dq_destroy(self.h)
            except Exception:
                pass
            self.h = None

    # -- plumbing -----------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def set_msg_tile(self, msg_ib):
        """Receivers per warp task of the jet message kernel (8 or 4; 0: default)."""
        _check(self.lib.dq_set_msg_tile(self.h, int(msg_ib)))

    def set_msg_kernel(self, mode):
        """Jet message kernel of the separate layer path: 1 general, 2 sender-tiled, 0 by size."""
        _check(self.lib.dq_set_msg_kernel(self.h, int(mode)))

    def msg_kernel(self):
        """The jet message kernel the separate layer path takes (1 general, 2 sender-tiled)."""
        v = ctypes.c_int32()
        _check(self.lib.dq_msg_kernel(self.h, ctypes.byref(v)))
        return v.value

    def autotune(self, params, r):
        """Times local_energy on these walkers for the candidate layer kernels (fused or separate),
        walker chunks and message register tiles, and keeps the fastest; returns (ms, chunk,
        msg_ib)."""
        params = self._dev(params, shape=(self.P,))
        r = self._dev(r)
        B = r.numel() // (3 * self.N)
        keep = self.max_chunk()
        keep_lk = self.layer_kernel_fused()
        self.set_max_chunk(4096)  # the largest candidate
        n = self.workspace_size(B, OP_LOCAL_ENERGY)
        if self.precision in ("fp32", "bf16"):  # both modes have the fused and the separate layer path
            _check(self.lib.dq_set_layer_kernel(self.h, 2))  # the separate kernels' message buffer
            n = max(n, self.workspace_size(B, OP_LOCAL_ENERGY))
            _check(self.lib.dq_set_layer_kernel(self.h, 1 if keep_lk else 2))
        n += 2 * ((B * 4 + 255) // 256 * 256) + (B + 255) // 256 * 256
        self.set_max_chunk(keep)
        ws = self._ws if self._ws is not None and self._ws.numel() >= n else torch.empty(n, dtype=torch.uint8,
                                                                                       device=self.device)
        self._ws = ws
        best = ctypes.c_double()
        _check(self.lib.dq_autotune(self.h, _ptr(params), _ptr(r), B, _ptr(ws), ws.numel(), self._stream(),
                                    ctypes.byref(best)))
        return best.value, self.max_chunk(), self._msg_ib()

    def set_layer_kernel(self, mode):
        """Jet layers: 1 fused kernel (messages as the tensor-core operand), 2 separate kernels, 0 the
        default (fused where supported)."""
        _check(self.lib.dq_set_layer_kernel(self.h, int(mode)))

    def set_det_warps(self, warps):
        """Warps (matrices) per CTA of the determinant kernels: 4 or 2."""
        _check(self.lib.dq_set_det_warps(self.h, int(warps)))

    def tile_set(self):
        """The current tile set: {max_chunk, msg_ib, layer_kernel (1 fused, 2 separate), det_warps}."""
        c, ib, lk, dw = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.dq_tile_set(self.h, ctypes.byref(c), ctypes.byref(ib), ctypes.byref(lk), ctypes.byref(dw)))
        return {"max_chunk": c.value, "msg_ib": ib.value, "layer_kernel": lk.value, "det_warps": dw.value}

    def layer_kernel_fused(self):
        v = ctypes.c_int32()
        _check(self.lib.dq_layer_kernel(self.h, ctypes.byref(v)))
        return bool(v.value)

    def _msg_ib(self):
        v = ctypes.c_int32()
        _check(self.lib.dq_msg_tile(self.h, ctypes.byref(v)))
        return v.value

    def set_max_chunk(self, chunk):
        _check(self.lib.dq_set_max_chunk(self.h, int(chunk)))

    def max_chunk(self):
        c = ctypes.c_int64()
        _check(self.lib.dq_max_chunk(self.h, ctypes.byref(c)))
        return c.value

    def workspace_size(self, B, op):
        n = ctypes.c_size_t()
        _check(self.lib.dq_workspace_size(self.h, int(B), int(op), ctypes.byref(n)))
        return n.value

    def workspace(self, B, op):
        n = max(self.workspace_size(B, op), 256)
        if self._ws is None or self._ws.numel() < n:
            self._ws = None
            self._ws = torch.empty(n, dtype=torch.uint8, device=self.device)
        return self._ws

    def _dev(self, t, dtype=None, shape=None):
        dtype = dtype or self.dtype
        if not isinstance(t, torch.Tensor):
            t = torch.as_tensor(t)
        if t.device != self.device:
            if t.device.type == "cpu" and not t.is_pinned():
                t = t.to(dtype).contiguous().pin_memory()
            t = t.to(self.device, dtype=dtype, non_blocking=True)
        if t.dtype != dtype:
            raise DQError(f"expected {dtype}, got {t.dtype}")
        t = t.contiguous()
        if shape is not None and tuple(t.shape) != tuple(shape):
            t = t.reshape(shape)
        return t

    # -- the four calls of the hot path ---------------------------------------
    def ansatz_eval(self, params, r):
        host = isinstance(r, torch.Tensor) and r.device.type == "cpu"
        params = self._dev(params, shape=(self.P,))
        r = self._dev(r)
        B = r.numel() // (3 * self.N)
        logabs = torch.empty(B, dtype=self.dtype, device=self.device)
        sign = torch.empty(B, dtype=torch.int8, device=self.device)
        ws = self.workspace(B, OP_EVAL)
        _check(self.lib.ansatz_eval(self.h, _ptr(params), _ptr(r), B, _ptr(logabs), _ptr(sign), _ptr(ws),
                                    ws.numel(), self._stream()))
        if host:
            return logabs.cpu(), sign.cpu()
        return logabs, sign

    def local_energy(self, params, r, sums=False):
        """Returns (logabs, sign, e_loc) and, with ``sums``, the FP64 [sum E, sum E^2]."""
        host = isinstance(r, torch.Tensor) and r.device.type == "cpu"
        params = self._dev(params, shape=(self.P,))
        r = self._dev(r)
        B = r.numel() // (3 * self.N)
        logabs = torch.empty(B, dtype=self.dtype, device=self.device)
        sign = torch.empty(B, dtype=torch.int8, device=self.device)
        e_loc = torch.empty(B, dtype=self.dtype, device=self.device)
        e2 = torch.empty(2, dtype=torch.float64, device=self.device) if sums else None
        ws = self.workspace(B, OP_LOCAL_ENERGY)
        _check(self.lib.local_energy(self.h, _ptr(params), _ptr(r), B, _ptr(logabs), _ptr(sign), _ptr(e_loc),
                                     _ptr(e2), _ptr(ws), ws.numel(), self._stream()))
        out = (logabs, sign, e_loc) + ((e2,) if sums else ())
        if host:
            out = tuple(t.cpu() for t in out)
        return out

    def mcmc_step(self, params, r, logabs, n_steps=1, step_size=0.2, seed=0, step_counter=0):
        """In-place Metropolis update of device tensors r and logabs; returns the accepted count (device int64).

        step_counter: an int, or a one-element int64 CUDA tensor holding the counter on the device
        (read by the kernels and advanced by n_steps: the form a captured CUDA graph can replay)."""
        params = self._dev(params, shape=(self.P,))
        for t in (r, logabs):
            if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
                raise DQError("mcmc_step updates r and logabs in place: pass contiguous device tensors")
        B = r.numel() // (3 * self.N)
        n_acc = torch.empty(1, dtype=torch.int64, device=self.device)
        ws = self.workspace(B, OP_MCMC)
        if isinstance(step_counter, torch.Tensor):
            if step_counter.device != self.device or step_counter.dtype != torch.int64 or step_counter.numel() != 1:
                raise DQError("a device step counter is a one-element int64 tensor on the handle's device")
            _check(self.lib.mcmc_step_dev(self.h, _ptr(params), _ptr(r), _ptr(logabs), B, int(n_steps),
                                          float(step_size), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(step_counter),
                                          _ptr(n_acc), _ptr(ws), ws.numel(), self._stream()))
        else:
            _check(self.lib.mcmc_step(self.h, _ptr(params), _ptr(r), _ptr(logabs), B, int(n_steps),
                                      float(step_size), int(seed) & 0xFFFFFFFFFFFFFFFF, int(step_counter), _ptr(n_acc),
                                      _ptr(ws), ws.numel(), self._stream()))
        return n_acc

    def mala_step(self, params, r, logabs, grad, n_steps=1, tau=0.05, seed=0, step_counter=0, grad_valid=True,
                  e_loc=None):
        """In-place Metropolis-adjusted Langevin update of device tensors r, logabs and grad
        (d log|psi| / d r at r) and, if given, e_loc (E_loc at r); grad_valid=False computes
        them first (n_steps=0 then only sets them up).  Returns the accepted count (device
        int64).  step_counter: an int, or a one-element int64 CUDA tensor (read on the
        device and advanced by n_steps)."""
        params = self._dev(params, shape=(self.P,))
        for t in (r, logabs, grad) + ((e_loc,) if e_loc is not None else ()):
            if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
                raise DQError("mala_step updates r, logabs, grad and e_loc in place: pass contiguous device tensors")
        B = r.numel() // (3 * self.N)
        if grad.numel() != r.numel() or logabs.numel() != B or (e_loc is not None and e_loc.numel() != B):
            raise DQError("grad has the shape of r; logabs and e_loc one value per walker")
        n_acc = torch.empty(1, dtype=torch.int64, device=self.device)
        ws = self.workspace(B, OP_MALA)
        dev_ctr = None
        if isinstance(step_counter, torch.Tensor):
            if step_counter.device != self.device or step_counter.dtype != torch.int64 or step_counter.numel() != 1:
                raise DQError("a device step counter is a one-element int64 tensor on the handle's device")
            dev_ctr, step_counter = step_counter, 0
        _check(self.lib.mala_step(self.h, _ptr(params), _ptr(r), _ptr(logabs), _ptr(grad), _ptr(e_loc),
                                  1 if grad_valid else 0, B, int(n_steps), float(tau), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                  int(step_counter), _ptr(dev_ctr), _ptr(n_acc), _ptr(ws), ws.numel(), self._stream()))
        return n_acc

    def mcmc_step_eloc(self, params, r, logabs, e_loc, n_steps=1, step_size=0.2, seed=0, step_counter=0):
        """In-place Metropolis update of device tensors r, logabs and e_loc whose proposals are
        evaluated with the jets forward (mcmc_step's proposals, uniforms and acceptance, E_loc
        carried with the positions).  logabs and e_loc must be local_energy's values at r.
        Returns the accepted count (device int64).  step_counter: an int, or a one-element int64
        CUDA tensor (read on the device and advanced by n_steps)."""
        params = self._dev(params, shape=(self.P,))
        for t in (r, logabs, e_loc):
            if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
                raise DQError("mcmc_step_eloc updates r, logabs and e_loc in place: pass contiguous device tensors")
        B = r.numel() // (3 * self.N)
        if logabs.numel() != B or e_loc.numel() != B:
            raise DQError("logabs and e_loc hold one value per walker")
        n_acc = torch.empty(1, dtype=torch.int64, device=self.device)
        ws = self.workspace(B, OP_MALA)
        dev_ctr = None
        if isinstance(step_counter, torch.Tensor):
            if step_counter.device != self.device or step_counter.dtype != torch.int64 or step_counter.numel() != 1:
                raise DQError("a device step counter is a one-element int64 tensor on the handle's device")
            dev_ctr, step_counter = step_counter, 0
        _check(self.lib.mcmc_step_eloc(self.h, _ptr(params), _ptr(r), _ptr(logabs), _ptr(e_loc), B, int(n_steps),
                                       float(step_size), int(seed) & 0xFFFFFFFFFFFFFFFF, int(step_counter),
                                       _ptr(dev_ctr), _ptr(n_acc), _ptr(ws), ws.numel(), self._stream()))
        return n_acc

    def grad_logpsi(self, params, r, weights=None, mode=0):
        """mode 0: sum_b w_b d log|psi_b|/d theta -> [P]; mode 1: per walker -> [B][P]."""
        params = self._dev(params, shape=(self.P,))
        r = self._dev(r)
        B = r.numel() // (3 * self.N)
        w = self._dev(weights, shape=(B,)) if weights is not None else None
        out = torch.empty((self.P,) if mode == 0 else (B, self.P), dtype=self.dtype, device=self.device)
        ws = self.workspace(B, OP_GRAD)
        _check(self.lib.grad_logpsi(self.h, _ptr(params), _ptr(r), B, _ptr(w), int(mode), _ptr(out), _ptr(ws),
                                    ws.numel(), self._stream()))
        return out

    def natural_gradient(self, G, w, lam, max_iter=200, tol=1e-8):
        """Natural-gradient direction (F + lam I)^-1 G^T w from per-walker gradients G [B][P]
        (grad_logpsi mode 1) and walker weights w; returns (delta [P], stats [iterations,
        relative residual, ||w||, lam])."""
        G = self._dev(G)
        B = G.numel() // self.P
        w = self._dev(w, shape=(B,))
        delta = torch.empty(self.P, dtype=self.dtype, device=self.device)
        stats = torch.empty(4, dtype=torch.float64, device=self.device)
        ws = self.workspace(B, OP_NATGRAD)
        _check(self.lib.natural_gradient(self.h, _ptr(G), _ptr(w), B, float(lam), int(max_iter), float(tol),
                                         _ptr(delta), _ptr(stats), _ptr(ws), ws.numel(), self._stream()))
        return delta, stats

    def pseudopotential_energy(self, params, r, pps, rot, logabs, sign):
        """Local and non-local pseudopotential energies per walker by the 12-point icosahedral
        quadrature.  pps: list of (nucleus index, coef [(l_max + 2)][n_terms][3] = (beta, n,
        alpha), V first then W_0 .. W_lmax); rot [B][3][3] rotations; logabs, sign of r.
        Returns (v_loc, v_nl)."""
        params = self._dev(params, shape=(self.P,))
        r = self._dev(r)
        B = r.numel() // (3 * self.N)
        rot = self._dev(rot, shape=(B, 3, 3))
        keep, arr = [], (_PP * len(pps))()
        for q, (nuc, coef) in enumerate(pps):
            c = torch.as_tensor(coef, dtype=torch.float64).contiguous()
            keep.append(c)
            arr[q] = _PP(int(nuc), int(c.shape[0] - 2), int(c.shape[1]), ctypes.c_void_p(c.data_ptr()))
        n = ctypes.c_size_t()
        _check(self.lib.dq_pp_workspace_size(self.h, B, len(pps), ctypes.byref(n)))
        ws = self._ws if self._ws is not None and self._ws.numel() >= n.value else torch.empty(
            max(n.value, 256), dtype=torch.uint8, device=self.device)
        self._ws = ws
        v_loc = torch.empty(B, dtype=self.dtype, device=self.device)
        v_nl = torch.empty(B, dtype=self.dtype, device=self.device)
        _check(self.lib.pseudopotential_energy(self.h, _ptr(params), _ptr(r), B, len(pps), arr, _ptr(rot),
                                               _ptr(logabs), _ptr(sign), _ptr(v_loc), _ptr(v_nl), _ptr(ws),
                                               ws.numel(), self._stream()))
        return v_loc, v_nl

    def param_update(self, params, delta, lr, max_norm=0.0):
        """In place: params -= lr * s * delta with s = min(1, max_norm / (lr ||delta||)) (max_norm <= 0:
        s = 1); returns stats [||delta||, s] (device float64)."""
        if params.device != self.device or params.dtype != self.dtype or not params.is_contiguous():
            raise DQError("param_update updates params in place: pass a contiguous device tensor")
        delta = self._dev(delta, shape=(self.P,))
        stats = torch.empty(2, dtype=torch.float64, device=self.device)
        ws = self.workspace(1, OP_UPDATE)
        _check(self.lib.param_update(self.h, _ptr(params), _ptr(delta), float(lr), float(max_norm), _ptr(stats),
                                     _ptr(ws), ws.numel(), self._stream()))
        return stats

    def vmc_loss_weights(self, e_loc, clip_k=5.0, clip="hard"):
        """Median/MAD-clipped gradient weights; returns (weights, stats[mu, half-width, mean E^, mean E]).
        clip: "hard" (clamp to the window) or "log" (logarithmic soft window)."""
        e_loc = self._dev(e_loc)
        B = e_loc.numel()
        w = torch.empty(B, dtype=self.dtype, device=self.device)
        stats = torch.empty(4, dtype=torch.float64, device=self.device)
        ws = self.workspace(B, OP_LOSS_WEIGHTS)
        if clip not in CLIP_MODES:
            raise DQError(f"clip must be one of {sorted(CLIP_MODES)}")
        _check(self.lib.vmc_loss_weights_clip(self.h, _ptr(e_loc), B, float(clip_k), CLIP_MODES[clip], _ptr(w),
                                              _ptr(stats), _ptr(ws), ws.numel(), self._stream()))
        return w, stats

    # -- measurement ---------------------------------------------------------
    def profile(self, on=True):
        """Enable or disable per-launch CUDA-event timing inside the library."""
        _check(self.lib.dq_profile_enable(self.h, 1 if on else 0))

    def profile_reset(self):
        _check(self.lib.dq_profile_reset(self.h))

    def profile_read(self):
        """{kernel kind: (total ms, launches)} since the last reset (kinds with launches only)."""
        out = {}
        for k in range(self.lib.dq_profile_kind_count()):
            ms, n = ctypes.c_double(), ctypes.c_int64()
            st = self.lib.dq_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n))
            if st not in (0, 5):
                _check(st)
            if n.value:
                out[self.lib.dq_profile_kind_name(k).decode()] = (ms.value, n.value)
        return out

    def fp64_matrix_count(self):
        """Determinant matrices that took the FP64 path since the last read (then cleared)."""
        c = ctypes.c_int64()
        _check(self.lib.dq_fp64_matrix_count(self.h, self._stream(), ctypes.byref(c)))
        return c.value

    def device_status(self):
        f = ctypes.c_uint32()
        _check(self.lib.dq_last_device_status(self.h, self._stream(), ctypes.byref(f)))
        return f.value


def _sys_cfg(system, cfg, keep):
    Z = (ctypes.c_double * len(system.Z))(*[float(z) for z in system.Z])
    flatR = [float(x) for x in torch.as_tensor(system.R, dtype=torch.float64).reshape(-1).tolist()]
    R = (ctypes.c_double * len(flatR))(*flatR)
    keep += [Z, R]
    sysc = _System(len(system.Z), ctypes.cast(Z, ctypes.c_void_p), ctypes.cast(R, ctypes.c_void_p),
                   int(system.n_up), int(system.n_down))
    cfgc = _Cfg(int(cfg.width), int(cfg.n_layers), int(cfg.n_det), int(cfg.n_rbf), float(cfg.rbf_cutoff),
                int(cfg.use_jastrow), int(cfg.use_cusp), float(cfg.cusp_alpha),
                    int(getattr(cfg, "full_det", 0)), int(getattr(cfg, "edge_update", 0)),
                    int(getattr(cfg, "el_init", 0)))
    return sysc, cfgc


def _ptrs(ts):
    """Host array of device pointers (None for a missing entry)."""
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])


class AnsatzBatch:
    """A batch of molecules (``dq_multi``): each its own system, ansatz sizes and
    parameters, all in one precision (fp32 or bf16).  Every step of the forward
    pass, the Metropolis sampler and the loss weights runs as one kernel launch
    over all molecules' walkers.  Methods take and return lists with one entry
    per molecule (device tensors, laid out as for :class:`Ansatz`)."""

    def __init__(self, systems, cfgs, precision="fp32", device=None):
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise DQError("no CUDA device: the library has no CPU path")
        device = torch.device("cuda") if device is None else torch.device(device)
        self.device = torch.device("cuda", torch.cuda.current_device() if device.index is None else device.index)
        self.precision = precision
        self.dtype = torch.float32
        self.n = len(systems)
        self._keep = []
        pairs = [_sys_cfg(sy, cf, self._keep) for sy, cf in zip(systems, cfgs)]
        sys_arr = (_System * self.n)(*[p[0] for p in pairs])
        cfg_arr = (_Cfg * self.n)(*[p[1] for p in pairs])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.dq_create_multi(self.n, sys_arr, cfg_arr, PRECISIONS[precision], ctypes.byref(h)))
        self.h = h
        self.handles, self.P = [], []
        for k in range(self.n):
            hk = ctypes.c_void_p()
            _check(self.lib.dq_multi_handle(self.h, k, ctypes.byref(hk)))
            P = ctypes.c_int64()
            _check(self.lib.dq_param_count(hk, ctypes.byref(P)))
            self.handles.append(hk)
            self.P.append(P.value)
        self.N = [int(sy.n_up + sy.n_down) for sy in systems]
        self._ws = None

    def __del__(self):
        if getattr(self, "h", None) and self.lib is not None:
            try:
                self.lib.dq_destroy_multi(self.h)
            except Exception:
                pass
            self.h = None

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _B(self, r):
        return (ctypes.c_int64 * self.n)(*[t.numel() // (3 * N) for t, N in zip(r, self.N)])

    def _check_in(self, ts, what):
        for t in ts:
            if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
                raise DQError(f"{what}: contiguous {self.dtype} tensors on {self.device} expected")

    def set_rounds(self, rounds):
        _check(self.lib.dq_multi_set_rounds(self.h, int(rounds)))

    def rounds(self):
        v = ctypes.c_int32()
        _check(self.lib.dq_multi_rounds(self.h, ctypes.byref(v)))
        return v.value

    def workspace(self, B, op):
        n = ctypes.c_size_t()
        _check(self.lib.dq_multi_workspace_size(self.h, B, int(op), ctypes.byref(n)))
        size = max(n.value, 256)
        if self._ws is None or self._ws.numel() < size:
            self._ws = None
            self._ws = torch.empty(size, dtype=torch.uint8, device=self.device)
        return self._ws

    def autotune(self, params, r):
        """Times local_energy on these walkers for every candidate tile shape (walkers per
        launch, message-kernel register tile), keeps the fastest; returns (ms, rounds, msg_ib)."""
        self._check_in(list(params) + list(r), "autotune")
        B = self._B(r)
        ws = self.workspace(B, OP_AUTOTUNE)
        best = ctypes.c_double()
        _check(self.lib.dq_autotune_multi(self.h, _ptrs(params), _ptrs(r), B, _ptr(ws), ws.numel(), self._stream(),
                                          ctypes.byref(best)))
        return (best.value,) + self.tuning()

    def tuning(self):
        rounds, ib = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.dq_multi_tuning(self.h, ctypes.byref(rounds), ctypes.byref(ib)))
        return rounds.value, ib.value

    def tile_set(self):
        """The batch's tile set: {rounds, msg_ib, fused_layers (molecules), det_warps}."""
        r, ib, f, dw = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.dq_multi_tile_set(self.h, ctypes.byref(r), ctypes.byref(ib), ctypes.byref(f), ctypes.byref(dw)))
        return {"rounds": r.value, "msg_ib": ib.value, "fused_layers": f.value, "det_warps": dw.value}

    def ansatz_eval(self, params, r):
        self._check_in(list(params) + list(r), "ansatz_eval")
        B = self._B(r)
        la = [torch.empty(B[k], dtype=self.dtype, device=self.device) for k in range(self.n)]
        sg = [torch.empty(B[k], dtype=torch.int8, device=self.device) for k in range(self.n)]
        ws = self.workspace(B, OP_EVAL)
        _check(self.lib.ansatz_eval_multi(self.h, _ptrs(params), _ptrs(r), B, _ptrs(la), _ptrs(sg), _ptr(ws),
                                          ws.numel(), self._stream()))
        return la, sg

    def local_energy(self, params, r, sums=False):
        """Lists (logabs, sign, e_loc) and, with ``sums``, an FP64 [n][2] tensor of [sum E, sum E^2]."""
        self._check_in(list(params) + list(r), "local_energy")
        B = self._B(r)
        la = [torch.empty(B[k], dtype=self.dtype, device=self.device) for k in range(self.n)]
        sg = [torch.empty(B[k], dtype=torch.int8, device=self.device) for k in range(self.n)]
        el = [torch.empty(B[k], dtype=self.dtype, device=self.device) for k in range(self.n)]
        e2 = torch.empty((self.n, 2), dtype=torch.float64, device=self.device) if sums else None
        ws = self.workspace(B, OP_LOCAL_ENERGY)
        _check(self.lib.local_energy_multi(self.h, _ptrs(params), _ptrs(r), B, _ptrs(la), _ptrs(sg), _ptrs(el),
                                           _ptrs(list(e2)) if sums else None, _ptr(ws), ws.numel(),
                                           self._stream()))
        return (la, sg, el) + ((e2,) if sums else ())

    def mcmc_step(self, params, r, logabs, n_steps=1, step_size=0.2, seed=0, step_counter=0):
        """In-place Metropolis update of every molecule's walkers; returns the accepted counts
        ([n] device int64).  step_counter: int, or a one-element int64 CUDA tensor."""
        self._check_in(list(params) + list(r) + list(logabs), "mcmc_step")
        B = self._B(r)
        n_acc = torch.zeros(self.n, dtype=torch.int64, device=self.device)
        ws = self.workspace(B, OP_MCMC)
        dev_ctr = None
        if isinstance(step_counter, torch.Tensor):
            dev_ctr, step_counter = step_counter, 0
        _check(self.lib.mcmc_step_multi(self.h, _ptrs(params), _ptrs(r), _ptrs(logabs), B, int(n_steps),
                                        float(step_size), int(seed) & 0xFFFFFFFFFFFFFFFF, int(step_counter),
                                        _ptr(dev_ctr), _ptrs(list(n_acc.view(self.n, 1))), _ptr(ws), ws.numel(),
                                        self._stream()))
        return n_acc

    def vmc_loss_weights(self, e_loc, clip_k=5.0):
        """Lists of weights and an FP64 [n][4] tensor of stats (see :meth:`Ansatz.vmc_loss_weights`)."""
        self._check_in(list(e_loc), "vmc_loss_weights")
        B = (ctypes.c_int64 * self.n)(*[t.numel() for t in e_loc])
        w = [torch.empty_like(t) for t in e_loc]
        stats = torch.empty((self.n, 4), dtype=torch.float64, device=self.device)
        ws = self.workspace(B, OP_LOSS_WEIGHTS)
        _check(self.lib.vmc_loss_weights_multi(self.h, _ptrs(e_loc), B, float(clip_k), _ptrs(w), _ptrs(list(stats)),
                                               _ptr(ws), ws.numel(), self._stream()))
        return w, stats

    def grad_logpsi(self, params, r, weights):
        """Weighted gradients sum_b w_b d log|psi_b| / d theta, one [P_m] tensor per molecule."""
        self._check_in(list(params) + list(r) + list(weights), "grad_logpsi")
        B = self._B(r)
        out = [torch.empty(P, dtype=self.dtype, device=self.device) for P in self.P]
        ws = self.workspace(B, OP_GRAD)
        _check(self.lib.grad_logpsi_multi(self.h, _ptrs(params), _ptrs(r), B, _ptrs(weights), _ptrs(out), _ptr(ws),
                                          ws.numel(), self._stream()))
        return out

    # -- measurement: launches of the batch are timed on molecule 0's handle ------------
    def profile(self, on=True):
        _check(self.lib.dq_profile_enable(self.handles[0], 1 if on else 0))

    def profile_reset(self):
        _check(self.lib.dq_profile_reset(self.handles[0]))

    def profile_read(self):
        out = {}
        for k in range(self.lib.dq_profile_kind_count()):
            ms, n = ctypes.c_double(), ctypes.c_int64()
            st = self.lib.dq_profile_read(self.handles[0], k, ctypes.byref(ms), ctypes.byref(n))
            if st not in (0, 5):
                _check(st)
            if n.value:
                out[self.lib.dq_profile_kind_name(k).decode()] = (ms.value, n.value)
        return out


def test_gemm_bf16(X, W, bias=None, bias_period=1):
    """Runs the BF16 tensor-core GEMM on its own (test support): X [rows][K],
    W [n][K] BF16 CUDA tensors; returns (Y FP32 [rows][n], status flags)."""
    lib = load_library()
    rows, K = X.shape
    n = W.shape[0]
    Y = torch.empty((rows, n), dtype=torch.float32, device=X.device)
    st = torch.zeros(1, dtype=torch.int32, device=X.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(X.device).cuda_stream)
    _check(lib.dq_test_gemm_bf16(_ptr(X), rows, K, X.stride(0), _ptr(W), n, _ptr(bias), bias_period, _ptr(Y), n,
                                 _ptr(st), stream))
    return Y, st


def test_gemm_tf32x3(X, W, bias=None, bias_period=1):
    """Runs the FP32-accurate (3 x TF32) tensor-core GEMM on its own (test
    support): X [rows][K], W [n][K] FP32 CUDA tensors; returns (Y FP32
    [rows][n], status flags)."""
    lib = load_library()
    rows, K = X.shape
    n = W.shape[0]
    Y = torch.empty((rows, n), dtype=torch.float32, device=X.device)
    st = torch.zeros(1, dtype=torch.int32, device=X.device)
    wsplit = torch.empty(2 * n * K, dtype=torch.float32, device=X.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(X.device).cuda_stream)
    _check(lib.dq_test_gemm_tf32x3(_ptr(X), rows, K, X.stride(0), _ptr(W.contiguous()), n, _ptr(bias), bias_period,
                                   _ptr(Y), n, _ptr(wsplit), _ptr(st), stream))
    return Y, st


def fma_rate(kind="fp32", device=None, blocks=152 * 8, iters=None, reps=5):
    """Measured FMA rate of the CUDA cores in TFLOP/s (kind "fp32" or "fp64"): the best of
    ``reps`` timed launches of dq_fma_rate_probe (CUDA events on the current stream)."""
    lib = load_library()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    k = {"fp32": 0, "fp64": 1}[kind]
    iters = iters or (4096 if k == 0 else 256)
    sink = torch.empty(blocks, dtype=torch.float64, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    flops = ctypes.c_double()
    _check(lib.dq_fma_rate_probe(k, blocks, max(1, iters // 64), _ptr(sink), stream, ctypes.byref(flops)))  # warm-up
    best = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _check(lib.dq_fma_rate_probe(k, blocks, iters, _ptr(sink), stream, ctypes.byref(flops)))
        b.record()
        torch.cuda.synchronize(dev)
        best = max(best, flops.value / (a.elapsed_time(b) / 1e3) / 1e12)
    return best


class LogAbsPsi(torch.autograd.Function):
    """log|psi| of every walker as a differentiable function of the parameters.

    Forward: ``ansatz_eval``.  Backward: ``grad_logpsi`` in weighted mode with
    the incoming gradient as the walker weights, i.e. sum_b g_b d log|psi_b| /
    d theta (the form the gradient estimator of Eq. (30) takes).  Positions
    get no gradient.
    """

    @staticmethod
    def forward(ctx, params, r, handle):
        logabs, _ = handle.ansatz_eval(params, r)
        ctx.save_for_backward(params, r)
        ctx.handle = handle
        return logabs

    @staticmethod
    def backward(ctx, grad_out):
        params, r = ctx.saved_tensors
        h = ctx.handle
        g = h.grad_logpsi(params, r, grad_out.to(h.dtype).contiguous(), mode=0)
        return g, None, None


def log_abs_psi(handle, params, r):
    """Differentiable log|psi| (see :class:`LogAbsPsi`)."""
    return LogAbsPsi.apply(params, r, handle)


# C-ABI names as free functions over a handle.
def ansatz_eval(h: Ansatz, params, r):
    return h.ansatz_eval(params, r)


def local_energy(h: Ansatz, params, r, sums=False):
    return h.local_energy(params, r, sums)


def mcmc_step(h: Ansatz, params, r, logabs, n_steps=1, step_size=0.2, seed=0, step_counter=0):
    return h.mcmc_step(params, r, logabs, n_steps, step_size, seed, step_counter)


def grad_logpsi(h: Ansatz, params, r, weights=None, mode=0):
    return h.grad_logpsi(params, r, weights, mode)


def vmc_loss_weights(h: Ansatz, e_loc, clip_k=5.0, clip="hard"):
    return h.vmc_loss_weights(e_loc, clip_k, clip)


def vmc_train_step(h: Ansatz, params, r, logabs, lr, damping=-0.1, max_norm=0.0, step_size=0.2, seed=0,
                   step_counter=0, clip_k=5.0, cg_iters=200, cg_tol=1e-8, clip="hard"):
    """One step of the VMC training loop with every computation in the library: a Metropolis sweep
    (positions and log|psi| updated in place), local energies, clipped-energy weights, per-walker
    gradients (clip: "hard" or "log", see :meth:`Ansatz.vmc_loss_weights`), the natural-gradient direction (damping < 0: relative to the Gram matrix's mean
    eigenvalue) and the parameter update (params in place).  Returns a dict of device tensors:
    e_sum2 ([sum E, sum E^2] of the unclipped energies before the update), loss-weight stats,
    natural-gradient stats and update stats."""
    h.mcmc_step(params, r, logabs, 1, step_size, seed, step_counter)
    _, _, e_loc, e2 = h.local_energy(params, r, sums=True)
    w, wstats = h.vmc_loss_weights(e_loc, clip_k, clip)
    G = h.grad_logpsi(params, r, mode=1)
    delta, ngstats = h.natural_gradient(G, w, damping, cg_iters, cg_tol)
    ustats = h.param_update(params, delta, lr, max_norm)
    return {"e_sum2": e2, "weights": wstats, "natural_gradient": ngstats, "update": ustats}

