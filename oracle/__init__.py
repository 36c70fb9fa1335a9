"""FP64 CPU oracle of the DeepQMC-style VMC hot path (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and the
two share no code: the oracle is ``oracle.cpp`` (plain C++ on doubles,
hyper-dual and dual numbers) plus the few numpy routines below.

Functions, each following the paper's definitions:

* :func:`evaluate` - log|psi| and sign psi (Sec. 3, Eqs. 13-28).
* :func:`local_energy` - E_loc of Eq. (31), second derivatives one coordinate
  at a time with hyper-dual numbers (the "serial" Laplacian of App. A.2).
* :func:`grad_jvp`, :func:`grad_index` - derivatives of log|psi| along
  parameter directions (dual numbers), the ingredient of Eq. (30).
* :func:`metropolis_step` - one random-walk Metropolis step (Sec. 5) on
  draws passed in.
* :func:`mala_step` - one Metropolis-adjusted Langevin step (Sec. 5, the
  Langevin sampler, with per-electron drift limiting) on draws passed in.
* :func:`clipped_loss_weights` - median/MAD clipping (hard or logarithmic) of Sec. 4.4 and the
  per-walker weights of the gradient estimator, Eq. (30).
* :func:`energy_estimate` - Eq. (33) and the batch-means error bar, Eq. (35).
* :func:`pseudopotential` - local and non-local pseudopotential energies of
  Eqs. 11 and 12: the angular integral by the
  12-point icosahedral quadrature over a rotated icosahedron, psi ratios from
  :meth:`Oracle.evaluate`.
* :func:`param_update` - the optimiser's parameter step with its step-length
  limit (Sec. 4, "Optimizer").
* :func:`natural_gradient` - the natural-gradient direction of the optimiser
  section (Sec. 4, "Optimizer"): the loss gradient preconditioned by the damped
  Fisher information of |psi|^2, estimated from walker-centred per-walker
  gradients of log|psi|; dense FP64 solve.

Parity status: all functions are pinned by the ``-m "not gpu"`` tests
(closed forms, invariants, finite differences and brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
# The oracle proper (FP64) and the same source compiled with FP32 scalars,
# which only serves to measure the rounding floor of an FP32 evaluation.
_LIBS = {"fp64": os.path.join(_HERE, "liboracle.so"), "fp32": os.path.join(_HERE, "liboracle_fp32.so")}
_DTYPES = {"fp64": np.float64, "fp32": np.float32}


def build(force=False, real="fp64"):
    """Compile the oracle library with g++ (OpenMP over walkers)."""
    path = _LIBS[real]
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
    if real == "fp32":
        cmd.insert(1, "-DORACLE_REAL=float")
    subprocess.check_call(cmd)
    os.replace(tmp, path)
    return path


def _spec_class(c_real):
    class _Spec(ctypes.Structure):
        _fields_ = [("n_nuc", ctypes.c_int32), ("Z", ctypes.c_void_p), ("R", ctypes.c_void_p),
                    ("n_up", ctypes.c_int32), ("n_dn", ctypes.c_int32),
                    ("D", ctypes.c_int32), ("L", ctypes.c_int32), ("K", ctypes.c_int32), ("Q", ctypes.c_int32),
                    ("rc", c_real), ("use_jastrow", ctypes.c_int32), ("use_cusp", ctypes.c_int32),
                    ("alpha", c_real), ("full_det", ctypes.c_int32), ("edge_update", ctypes.c_int32),
                    ("el_init", ctypes.c_int32)]
    return _Spec


_SPECS = {"fp64": _spec_class(ctypes.c_double), "fp32": _spec_class(ctypes.c_float)}
_libs = {}


def _load(real="fp64"):
    if real not in _libs:
        build(real=real)
        lib = ctypes.CDLL(_LIBS[real])
        P = ctypes.c_void_p
        lib.oracle_param_count.argtypes = [P, P]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_eval.argtypes = [P, P, P, ctypes.c_int64, P, P]
        lib.oracle_local_energy.argtypes = [P, P, P, ctypes.c_int64, P, P, P, P, P]
        lib.oracle_potential.argtypes = [P, P, ctypes.c_int64, P]
        lib.oracle_grad_jvp.argtypes = [P, P, P, ctypes.c_int64, P, ctypes.c_int32, P]
        lib.oracle_grad_index.argtypes = [P, P, P, ctypes.c_int64, P, ctypes.c_int32, P]
        lib.oracle_metropolis_step.argtypes = [P, P, P, P, ctypes.c_int64, P, P, ctypes.c_double, P]
        lib.oracle_mala_step.argtypes = [P, P, P, P, P, ctypes.c_int64, P, P, ctypes.c_double, P, P]
        lib.oracle_intermediates.argtypes = [P, P, P, P, P]
        _libs[real] = lib
    return _libs[real]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Oracle:
    """The oracle for one molecule and ansatz configuration."""

    def __init__(self, system, cfg, real="fp64"):
        self.lib = _load(real)
        self.real, self.dt = real, _DTYPES[real]
        self.system, self.cfg = system, cfg
        self._Z = np.ascontiguousarray(system.Z, dtype=self.dt)
        self._R = np.ascontiguousarray(system.R, dtype=self.dt)
        self.spec = _SPECS[real](len(self._Z), self._Z.ctypes.data, self._R.ctypes.data, system.n_up, system.n_down,
                          cfg.width, cfg.n_layers, cfg.n_det, cfg.n_rbf, cfg.rbf_cutoff,
                          int(cfg.use_jastrow), int(cfg.use_cusp), cfg.cusp_alpha, int(cfg.full_det),
                          int(cfg.edge_update), int(cfg.el_init))
        self.N = system.n_up + system.n_down
        P = ctypes.c_int64()
        self.lib.oracle_param_count(ctypes.byref(self.spec), ctypes.byref(P))
        self.P = P.value

    @staticmethod
    def set_threads(n):
        for real in _LIBS:
            if real in _libs or real == "fp64":
                _load(real).oracle_set_threads(int(n))

    @staticmethod
    def threads():
        return int(_load().oracle_threads())

    def _fp64_only(self):
        if self.real != "fp64":
            raise ValueError("the FP32 build of the oracle only serves evaluate() and local_energy()")

    def _prep(self, theta, r):
        theta = np.ascontiguousarray(theta, dtype=self.dt)
        assert theta.size == self.P, (theta.size, self.P)
        r = np.ascontiguousarray(r, dtype=self.dt).reshape(-1, self.N, 3)
        return theta, r

    def evaluate(self, theta, r):
        theta, r = self._prep(theta, r)
        B = r.shape[0]
        la = np.empty(B, dtype=self.dt)
        sg = np.empty(B, dtype=np.int8)
        self.lib.oracle_eval(ctypes.byref(self.spec), _ptr(theta), _ptr(r), B, _ptr(la), _ptr(sg))
        return la, sg

    def local_energy(self, theta, r, with_grad=False):
        theta, r = self._prep(theta, r)
        B = r.shape[0]
        la, el, lap = np.empty(B, self.dt), np.empty(B, self.dt), np.empty(B, self.dt)
        sg = np.empty(B, dtype=np.int8)
        grad = np.empty((B, 3 * self.N), self.dt) if with_grad else None
        self.lib.oracle_local_energy(ctypes.byref(self.spec), _ptr(theta), _ptr(r), B, _ptr(la), _ptr(sg),
                                     _ptr(el), _ptr(grad), _ptr(lap))
        out = {"logabs": la, "sign": sg, "e_loc": el, "lap": lap}
        if with_grad:
            out["grad"] = grad
        return out

    def potential(self, r):
        self._fp64_only()
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, self.N, 3)
        V = np.empty(r.shape[0])
        self.lib.oracle_potential(ctypes.byref(self.spec), _ptr(r), r.shape[0], _ptr(V))
        return V

    def grad_jvp(self, theta, r, dirs):
        self._fp64_only()
        theta, r = self._prep(theta, r)
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, self.P)
        out = np.empty((r.shape[0], dirs.shape[0]))
        self.lib.oracle_grad_jvp(ctypes.byref(self.spec), _ptr(theta), _ptr(r), r.shape[0], _ptr(dirs),
                                 dirs.shape[0], _ptr(out))
        return out

    def grad_index(self, theta, r, idx):
        self._fp64_only()
        theta, r = self._prep(theta, r)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.empty((r.shape[0], idx.size))
        self.lib.oracle_grad_index(ctypes.byref(self.spec), _ptr(theta), _ptr(r), r.shape[0], _ptr(idx),
                                   idx.size, _ptr(out))
        return out

    def metropolis_step(self, theta, r, logabs, xi, u, step):
        """Returns (r_new, logabs_new, accepted) without modifying inputs."""
        self._fp64_only()
        theta, r = self._prep(theta, r)
        r = r.copy()
        la = np.ascontiguousarray(logabs, dtype=np.float64).copy()
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(r.shape)
        u = np.ascontiguousarray(u, dtype=np.float64)
        acc = np.empty(r.shape[0], dtype=np.int8)
        self.lib.oracle_metropolis_step(ctypes.byref(self.spec), _ptr(theta), _ptr(r), _ptr(la), r.shape[0],
                                        _ptr(xi), _ptr(u), float(step), _ptr(acc))
        return r, la, acc

    def mala_step(self, theta, r, logabs, grad, xi, u, tau):
        """Metropolis-adjusted Langevin step (Sec. 5) on draws passed in; returns
        (r_new, logabs_new, grad_new, accepted, log_alpha) without modifying inputs.
        grad is d log|psi| / d r at r ([B][N][3])."""
        self._fp64_only()
        theta, r = self._prep(theta, r)
        r = r.copy()
        la = np.ascontiguousarray(logabs, dtype=np.float64).copy()
        g = np.ascontiguousarray(grad, dtype=np.float64).reshape(r.shape).copy()
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(r.shape)
        u = np.ascontiguousarray(u, dtype=np.float64)
        acc = np.empty(r.shape[0], dtype=np.int8)
        lal = np.empty(r.shape[0])
        self.lib.oracle_mala_step(ctypes.byref(self.spec), _ptr(theta), _ptr(r), _ptr(la), _ptr(g), r.shape[0],
                                  _ptr(xi), _ptr(u), float(tau), _ptr(acc), _ptr(lal))
        return r, la, g, acc, lal

    def intermediates(self, theta, r):
        """Final embeddings f[N][D] and orbital matrices A[blocks][K][nmax][nmax] of one walker: blocks
        = 2 (spin up, spin down; nmax = max(n_up, n_down)), or 1 (the full determinant; nmax = N)."""
        self._fp64_only()
        theta, r = self._prep(theta, r)
        full = bool(self.cfg.full_det)
        nmax = self.N if full else max(self.system.n_up, self.system.n_down)
        f = np.empty((self.N, self.cfg.width))
        A = np.zeros((1 if full else 2, self.cfg.n_det, nmax, nmax))
        self.lib.oracle_intermediates(ctypes.byref(self.spec), _ptr(theta), _ptr(r[0]), _ptr(f), _ptr(A))
        return f, A


# ----------------------------------------------------------------------------
# Clipping and loss weights (Sec. 4.4, Eq. 30)
# ----------------------------------------------------------------------------
def log_clip(e, mu, sigma):
    """Logarithmically scaling soft clipping (Sec. 4.4, the scheme of Hermann
    et al.): the identity inside |e - mu| <= sigma; outside, the excess
    distance is replaced by its logarithm,
        E^ = mu + sign(e - mu) * sigma * (1 + ln(|e - mu| / sigma)),
    which is continuous with a continuous first derivative at |e - mu| =
    sigma and grows without bound, but only logarithmically.  The paper
    names the scheme without a formula; this is the reading taken."""
    e = np.asarray(e, dtype=np.float64)
    u = e - mu
    a = np.abs(u)
    out = e.copy()
    far = a > sigma
    out[far] = mu + np.sign(u[far]) * sigma * (1.0 + np.log(a[far] / sigma))
    return out


def clipped_loss_weights(e_loc, k=5.0, soft=False):
    """Clip local energies to median +- k * MAD and form gradient weights.

    Centre = median (mean of the two middle values for even B); half-width
    = k times the mean absolute deviation from the median (von Glehn et al.,
    cited in Sec. 4.4).  soft=False clamps to the window; soft=True applies
    :func:`log_clip` (k must be > 0).  Weights w_b = (2/B) (E^_b - mean E^),
    so that sum_b w_b grad log|psi_b| is the estimator of Eq. (30) on clipped
    energies.  Returns (weights, clipped, centre, half_width).
    """
    e = np.asarray(e_loc, dtype=np.float64)
    B = e.size
    s = np.sort(e)
    med = s[B // 2] if B % 2 else 0.5 * (s[B // 2 - 1] + s[B // 2])
    mad = np.mean(np.abs(e - med))
    lo, hi = med - k * mad, med + k * mad
    if soft:
        if not k > 0:
            raise ValueError("soft clipping needs k > 0")
        clipped = log_clip(e, med, k * mad) if mad > 0 else e.copy()
    else:
        clipped = np.minimum(np.maximum(e, lo), hi)
    w = (2.0 / B) * (clipped - clipped.mean())
    return w, clipped, med, k * mad


def energy_estimate(e_loc_steps):
    """Energy estimate (Eq. 33) and batch-means error (Eq. 35).

    ``e_loc_steps``: array [n_b walkers][n_s steps].
    """
    e = np.asarray(e_loc_steps, dtype=np.float64)
    nb = e.shape[0]
    mean = e.mean()
    batch = e.mean(axis=1)
    err = np.sqrt(np.sum((batch - mean) ** 2) / (nb * (nb - 1)))
    return mean, err


def natural_gradient(G, w, lam, form="sample"):
    """Natural-gradient direction delta = (F + lam I)^-1 g (Sec. 4, "Optimizer"):
    F = Gc^T Gc / B, the Fisher information of the density |psi|^2 up to the
    constant factor 4 (which lam absorbs), estimated from the per-walker gradients
    G[b] = d log|psi_b| / d theta centred over the walkers (Gc = G - mean_b G), and
    g = G^T w the loss gradient of Eq. (30) for the walker weights w (sum_b w_b = 0
    for the clipped-energy weights, so G^T w = Gc^T w).

    form "sample": Gc^T (Gc Gc^T / B + lam I)^-1 w, a B x B solve; form "parameter":
    (Gc^T Gc / B + lam I)^-1 Gc^T w, a P x P solve (small P only).  The two are equal
    by the push-through identity (A^T A + c I)^-1 A^T = A^T (A A^T + c I)^-1."""
    G = np.asarray(G, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B, P = G.shape
    Gc = G - G.mean(axis=0, keepdims=True)
    if form == "sample":
        x = np.linalg.solve(Gc @ Gc.T / B + lam * np.eye(B), w)
        return Gc.T @ x
    return np.linalg.solve(Gc.T @ Gc / B + lam * np.eye(P), Gc.T @ w)


def param_update(theta, delta, lr, max_norm=0.0):
    """The optimiser's parameter step around a direction delta (Sec. 4, "Optimizer"; the paper
    takes the step from a third-party library, so its plain form is the reading):
    theta - lr s delta with the step-length limit s = min(1, max_norm / (lr ||delta||)), s = 1
    when max_norm <= 0.  Returns (new theta, ||delta||, s), all FP64."""
    theta = np.asarray(theta, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    nrm = float(np.sqrt(np.sum(delta * delta)))
    s = 1.0 if max_norm <= 0 or lr * nrm <= max_norm else max_norm / (lr * nrm)
    return theta - lr * s * delta, nrm, s


_GOLDEN = (1.0 + 5.0 ** 0.5) / 2.0


def icosahedron():
    """The 12 vertices of a regular icosahedron on the unit sphere."""
    v = []
    for a in (-1.0, 1.0):
        for b in (-_GOLDEN, _GOLDEN):
            v += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    v = np.array(v)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def pp_radial(coef, r):
    """sum_k beta_k r^(n_k - 2) exp(-alpha_k r^2) for coef [n_terms][3] = (beta, n, alpha)."""
    coef = np.asarray(coef, dtype=np.float64)
    return float(np.sum(coef[:, 0] * r ** (coef[:, 1] - 2.0) * np.exp(-coef[:, 2] * r * r)))


def legendre(l, x):
    """P_l(x), l <= 3."""
    return [1.0, x, 0.5 * (3 * x * x - 1), 0.5 * (5 * x ** 3 - 3 * x)][l]


def pseudopotential(orc, theta, r, pps, rot, with_abs=False):
    """Local and non-local pseudopotential energies of every walker (Eqs. 11 and 12).
    pps: list of (nucleus index, coef [(l_max + 2)][n_terms][3]) with the local
    function V first, then W_0 .. W_lmax; rot [B][3][3] rotations of the icosahedron (one per
    walker).  For electron i and nucleus I the angular integral of Y_lm^* psi-ratio, summed over
    m with Y_lm(Omega), is (2l + 1) / (4 pi) int P_l(cos) psi'/psi dOmega' by the addition
    theorem; the quadrature replaces int dOmega' by 4 pi / 12 times the sum over the 12 vertices.
    Returns (v_loc [B], v_nl [B]) and, with ``with_abs``, the sums of |w psi'/psi| (the size
    of the quadrature sums, for error bounds)."""
    theta = np.asarray(theta, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64).reshape(-1, orc.N, 3)
    B = r.shape[0]
    R = np.asarray(orc.system.R, dtype=np.float64).reshape(-1, 3)
    ico = icosahedron()
    la0, sg0 = orc.evaluate(theta, r)
    v_loc = np.zeros(B)
    v_nl = np.zeros(B)
    v_abs = np.zeros(B)
    for b in range(B):
        verts = ico @ np.asarray(rot[b], dtype=np.float64).T  # R u_k
        configs, weights = [], []
        for I, coef in pps:
            coef = np.asarray(coef, dtype=np.float64)
            lmax = coef.shape[0] - 2
            for i in range(orc.N):
                d = r[b, i] - R[I]
                rr = float(np.linalg.norm(d))
                v_loc[b] += pp_radial(coef[0], rr)
                u = d / rr
                for k in range(12):
                    c = r[b].copy()
                    c[i] = R[I] + rr * verts[k]
                    configs.append(c)
                    cos = float(verts[k] @ u)
                    weights.append(sum(pp_radial(coef[1 + l], rr) * (2 * l + 1) / 12.0 * legendre(l, cos)
                                       for l in range(lmax + 1)))
        la, sg = orc.evaluate(theta, np.array(configs))
        ratio = sg * sg0[b] * np.exp(la - la0[b])
        v_nl[b] = float(np.sum(np.array(weights) * ratio))
        v_abs[b] = float(np.sum(np.abs(np.array(weights) * ratio)))
    return (v_loc, v_nl, v_abs) if with_abs else (v_loc, v_nl)

