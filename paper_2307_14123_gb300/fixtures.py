"""Seeded synthetic inputs: molecules, walkers, parameter blobs and the
Metropolis random draws.

This module holds no part of the method's arithmetic.  It only produces
inputs, which the CUDA library and the FP64 oracle both consume:

* molecule geometries (nuclear charges and positions in bohr), built from the
  bond lengths and angles in angstrom stated for each workload;
* the flat parameter blob of the DeepQMC-style ansatz, drawn from a
  counter-based generator (Xavier-normal matrices, N(0,1) embeddings, zero
  biases, unit envelope weights, envelope exponents U(0.5, 2), unit
  determinant coefficients);
* initial walkers, placed "by charge" around the nuclei;
* the Gaussian proposals and acceptance uniforms of the random-walk
  Metropolis sampler (Sec. 5), which the CUDA library regenerates on the
  device from the same counters, and which the oracle receives as inputs.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), written here from that published
definition, with Box-Muller normals.  Counter words:
``ctr = [walker, step_lo, (tag << 24) | block, step_hi]``, ``key = [seed_lo,
seed_hi]``; tags INIT=0, PROPOSE=1, ACCEPT=2, PARAMS=3.  One Philox call
yields four 32-bit words x0..x3; uniforms are ``(x + 0.5) * 2**-32`` and the
pairs (x0, x1), (x2, x3) give normals ``sqrt(-2 ln u_a) * (cos, sin)(2 pi u_b)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Philox4x32-10
# ----------------------------------------------------------------------------
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

TAG_INIT, TAG_PROPOSE, TAG_ACCEPT, TAG_PARAMS = 0, 1, 2, 3
BOHR_PER_ANGSTROM = 1.0 / 0.529177210903  # CODATA 2018


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on arrays of counters.

    ``ctr``: uint array ``[..., 4]``; ``key``: uint array ``[..., 2]``
    (broadcastable).  Returns uint32 ``[..., 4]``.
    """
    c = np.asarray(ctr, dtype=np.uint64) & _MASK32
    k = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & _MASK32
            k1 = (k1 + PHILOX_W1) & _MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _uniform(x):
    return (np.asarray(x, dtype=np.float64) + 0.5) * 2.0 ** -32


def _box_muller(x):
    """uint32 [..., 4] -> four standard normals [..., 4] (FP64)."""
    u = _uniform(x)
    ra = np.sqrt(-2.0 * np.log(u[..., 0]))
    th_a = 2.0 * math.pi * u[..., 1]
    rb = np.sqrt(-2.0 * np.log(u[..., 2]))
    th_b = 2.0 * math.pi * u[..., 3]
    return np.stack([ra * np.cos(th_a), ra * np.sin(th_a),
                     rb * np.cos(th_b), rb * np.sin(th_b)], axis=-1)


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def walker_normals(seed, walkers, step, tag, n):
    """``n`` standard normals per walker for (step, tag): ``[len(walkers), n]``."""
    walkers = np.asarray(walkers, dtype=np.uint64)
    nblk = (n + 3) // 4
    step = int(step)
    ctr = np.zeros((walkers.size, nblk, 4), dtype=np.uint64)
    ctr[..., 0] = walkers[:, None]
    ctr[..., 1] = step & 0xFFFFFFFF
    ctr[..., 2] = (np.uint64(tag) << np.uint64(24)) | np.arange(nblk, dtype=np.uint64)[None, :]
    ctr[..., 3] = (step >> 32) & 0xFFFFFFFF
    z = _box_muller(philox4x32_10(ctr, _key(seed)))
    return z.reshape(walkers.size, nblk * 4)[:, :n]


def walker_uniform(seed, walkers, step, tag):
    """One uniform in (0, 1) per walker for (step, tag): word x0 of block 0."""
    walkers = np.asarray(walkers, dtype=np.uint64)
    step = int(step)
    ctr = np.zeros((walkers.size, 4), dtype=np.uint64)
    ctr[:, 0] = walkers
    ctr[:, 1] = step & 0xFFFFFFFF
    ctr[:, 2] = np.uint64(tag) << np.uint64(24)
    ctr[:, 3] = (step >> 32) & 0xFFFFFFFF
    return _uniform(philox4x32_10(ctr, _key(seed))[:, 0])


def _param_stream(seed, n, sub):
    """Per-parameter stream: normals (sub=0) or uniform words (sub=1)."""
    nblk = (n + 3) // 4
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64) & _MASK32
    ctr[:, 1] = np.arange(nblk, dtype=np.uint64) >> np.uint64(32)
    ctr[:, 2] = (np.uint64(TAG_PARAMS) << np.uint64(24)) | np.uint64(sub)
    x = philox4x32_10(ctr, _key(seed))
    if sub == 0:
        return _box_muller(x).reshape(-1)[:n]
    return _uniform(x).reshape(-1)[:n]


# ----------------------------------------------------------------------------
# Molecules
# ----------------------------------------------------------------------------
@dataclass
class System:
    """Nuclei (charges ``Z[M]``, positions ``R[M][3]`` in bohr) and spins."""
    Z: np.ndarray
    R: np.ndarray
    n_up: int
    n_down: int
    name: str = ""

    @property
    def n_elec(self):
        return self.n_up + self.n_down

    @property
    def n_nuc(self):
        return len(self.Z)


def _neutral(name, Z, R_bohr):
    Z = np.asarray(Z, dtype=np.float64)
    n = int(round(Z.sum()))
    return System(Z=Z, R=np.asarray(R_bohr, dtype=np.float64).reshape(-1, 3),
                  n_up=(n + 1) // 2, n_down=n // 2, name=name)


def molecule(name):
    """Geometries of the benchmark molecules, in bohr."""
    a = BOHR_PER_ANGSTROM
    if name == "LiH":
        return _neutral(name, [3, 1], [[0, 0, 0], [0, 0, 3.015]])
    if name == "N2":
        return _neutral(name, [7, 7], [[0, 0, 1.034], [0, 0, -1.034]])
    if name == "C4H4":
        # rectangle of C with C-C bonds 1.34 A (along x) and 1.57 A (along y);
        # C-H 1.08 A pointing outward along the rectangle's diagonals; z = 0.
        hx, hy = 1.34 / 2, 1.57 / 2
        dn = math.hypot(hx, hy)
        C, H = [], []
        for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
            C.append([sx * hx, sy * hy, 0.0])
            H.append([sx * (hx + 1.08 * hx / dn), sy * (hy + 1.08 * hy / dn), 0.0])
        return _neutral(name, [6] * 4 + [1] * 4, np.array(C + H) * a)
    if name == "H2O":
        d, th = 0.9572, math.radians(104.5) / 2
        return _neutral(name, [8, 1, 1], np.array([[0, 0, 0],
                        [d * math.sin(th), 0, d * math.cos(th)],
                        [-d * math.sin(th), 0, d * math.cos(th)]]) * a)
    if name == "NH3":
        d, th = 1.012, math.radians(106.7)
        rho = d * math.sqrt(2.0 * (1.0 - math.cos(th)) / 3.0)
        h = math.sqrt(d * d - rho * rho)
        R = [[0, 0, 0]] + [[rho * math.cos(2 * math.pi * k / 3),
                            rho * math.sin(2 * math.pi * k / 3), -h] for k in range(3)]
        return _neutral(name, [7, 1, 1, 1], np.array(R) * a)
    if name == "C2H4":
        cc, ch, hch = 1.339, 1.087, math.radians(117.4)
        phi = math.pi - hch / 2  # angle of C-H against the +x axis on the +x carbon
        R = [[cc / 2, 0, 0], [-cc / 2, 0, 0]]
        for sx in (1, -1):
            for sy in (1, -1):
                R.append([sx * (cc / 2 - ch * math.cos(phi)), sy * ch * math.sin(phi), 0])
        return _neutral(name, [6, 6, 1, 1, 1, 1], np.array(R) * a)
    if name == "C6H6":
        rc, rh = 1.39, 1.39 + 1.09
        R = [[rc * math.cos(math.pi * k / 3), rc * math.sin(math.pi * k / 3), 0] for k in range(6)]
        R += [[rh * math.cos(math.pi * k / 3), rh * math.sin(math.pi * k / 3), 0] for k in range(6)]
        return _neutral(name, [6] * 6 + [1] * 6, np.array(R) * a)
    if name == "H":
        return System(Z=np.array([1.0]), R=np.zeros((1, 3)), n_up=1, n_down=0, name="H")
    raise KeyError(name)


# ----------------------------------------------------------------------------
# Ansatz hyper-parameters and the flat parameter layout
# ----------------------------------------------------------------------------
@dataclass
class AnsatzCfg:
    width: int = 32          # D, embedding width
    n_layers: int = 2        # L, message-passing layers
    n_det: int = 1           # K, determinant pairs
    n_rbf: int = 16          # Gaussian distance features
    rbf_cutoff: float = 10.0
    use_jastrow: int = 1
    use_cusp: int = 1
    cusp_alpha: float = 1.0
    full_det: int = 0        # 1: one determinant of all N electrons per p (Eq. 22)
    edge_update: int = 0     # 1: edge embeddings iterated between layers (Eq. 16, second case)
    el_init: int = 0         # 1: initial embeddings from electron-nucleus differences (Eq. 13, second case)


def param_layout(system: System, cfg: AnsatzCfg):
    """Flat parameter layout: list of (name, shape, init-kind).

    Order: E_spin[2][D] (or, with cfg.el_init, the initial-embedding MLP
    W_e1[D][3M], b_e1[D], W_e2[D][D], b_e2[D]); per layer l: W_h[D][D], then for edge types
    (same-spin, opposite-spin, electron-nucleus) [U[n_rbf][n_rbf], c[n_rbf]
    when cfg.edge_update and l >= 1: the edge-embedding update], W1[D][n_rbf], b1[D],
    W2[D][D], b2[D]; Y[M][D]; W_g[D][3D], b_g[D]; then per spin (up, down)
    W_o[K*n_c][D], b_o[K*n_c], omega[K*n_c][M], zeta[K*n_c][M]; then c[K];
    W_J1[D][D], b_J1[D], w_J2[D].  Matrices are [out][in], row-major.  n_c, the
    orbitals per determinant, is n_s (that spin's electrons) for spin-factorised
    determinants and N for the full determinant (cfg.full_det).
    """
    D, L, K, Q, M = cfg.width, cfg.n_layers, cfg.n_det, cfg.n_rbf, system.n_nuc
    if getattr(cfg, "el_init", 0):
        out = [("W_e1", (D, 3 * M), "xavier"), ("b_e1", (D,), "zero"), ("W_e2", (D, D), "xavier"),
               ("b_e2", (D,), "zero")]
    else:
        out = [("E_spin", (2, D), "normal")]
    for l in range(L):
        out.append((f"W_h{l}", (D, D), "xavier"))
        for t in ("par", "anti", "nuc"):
            if getattr(cfg, "edge_update", 0) and l > 0:
                out += [(f"U_{t}{l}", (Q, Q), "xavier"), (f"c_{t}{l}", (Q,), "zero")]
            out += [(f"W1_{t}{l}", (D, Q), "xavier"), (f"b1_{t}{l}", (D,), "zero"),
                    (f"W2_{t}{l}", (D, D), "xavier"), (f"b2_{t}{l}", (D,), "zero")]
        out.append((f"Y{l}", (M, D), "normal"))
        out += [(f"W_g{l}", (D, 3 * D), "xavier"), (f"b_g{l}", (D,), "zero")]
    N = system.n_up + system.n_down
    full = bool(getattr(cfg, "full_det", 0))
    for s, ns in (("up", system.n_up), ("dn", system.n_down)):
        nc = N if full else ns
        out += [(f"W_o_{s}", (K * nc, D), "xavier"), (f"b_o_{s}", (K * nc,), "zero"),
                (f"omega_{s}", (K * nc, M), "one"), (f"zeta_{s}", (K * nc, M), "zeta")]
    out.append(("c", (K,), "one"))
    out += [("W_J1", (D, D), "xavier"), ("b_J1", (D,), "zero"), ("w_J2", (1, D), "xavier")]
    return out


def param_count(system, cfg):
    return int(sum(int(np.prod(s)) for _, s, _ in param_layout(system, cfg)))


def param_offsets(system, cfg):
    off, o = {}, 0
    for name, shape, _ in param_layout(system, cfg):
        n = int(np.prod(shape))
        off[name] = (o, shape)
        o += n
    return off


def init_params(system, cfg, seed):
    """Seeded random-init parameter blob (FP64, flat)."""
    P = param_count(system, cfg)
    z = _param_stream(seed, P, 0)
    u = _param_stream(seed, P, 1)
    theta = np.zeros(P, dtype=np.float64)
    o = 0
    for _, shape, kind in param_layout(system, cfg):
        n = int(np.prod(shape))
        sl = slice(o, o + n)
        if kind == "normal":
            theta[sl] = z[sl]
        elif kind == "xavier":
            fan_out, fan_in = shape
            theta[sl] = z[sl] * math.sqrt(2.0 / (fan_in + fan_out))
        elif kind == "one":
            theta[sl] = 1.0
        elif kind == "zeta":
            theta[sl] = 0.5 + 1.5 * u[sl]
        o += n
    return theta


def network_off_params(system, cfg, zeta):
    """Parameters that switch the network off: orbitals are the bare envelopes.

    W_o = 0, b_o = 1 (so phi = 1), all Jastrow weights 0, omega = 1, every
    envelope exponent set to ``zeta`` (scalar, or per nucleus), c = 1; all
    other weights random from seed 0 (they cannot reach psi).
    """
    theta = init_params(system, cfg, 0)
    off = param_offsets(system, cfg)

    def put(name, val):
        o, shape = off[name]
        n = int(np.prod(shape))
        theta[o:o + n] = np.broadcast_to(np.asarray(val, dtype=np.float64), shape).reshape(-1)

    for s in ("up", "dn"):
        put(f"W_o_{s}", 0.0)
        put(f"b_o_{s}", 1.0)
        put(f"omega_{s}", 1.0)
        o, shape = off[f"zeta_{s}"]
        if shape[0]:
            put(f"zeta_{s}", np.broadcast_to(np.asarray(zeta, dtype=np.float64), (shape[1],))[None, :])
    put("c", 1.0)
    put("W_J1", 0.0)
    put("b_J1", 0.0)
    put("w_J2", 0.0)
    return theta


def smooth_params(system, cfg, seed, orbital_scale=0.3):
    """Seeded parameters of a smooth state with small kinetic terms: the random-init blob of
    ``seed`` with the orbital head W_o scaled by ``orbital_scale`` and its bias b_o set to 1, so
    that every orbital is its envelope modulated by the network by about +-orbital_scale
    (the network, Jastrow and envelopes keep their random-init values)."""
    theta = init_params(system, cfg, seed)
    off = param_offsets(system, cfg)
    for s in ("up", "dn"):
        for name, f in ((f"W_o_{s}", lambda x: x * orbital_scale), (f"b_o_{s}", lambda x: np.ones_like(x))):
            o, shape = off[name]
            n = int(np.prod(shape))
            theta[o:o + n] = f(theta[o:o + n])
    return theta


# ----------------------------------------------------------------------------
# Walkers
# ----------------------------------------------------------------------------
def electron_slots(system):
    """Nucleus index of each electron for the "by charge" placement.

    Nuclei are listed in order, each repeated Z_I times; slots are handed out
    alternately to spin-up and spin-down (the other channel once one is full);
    within a channel electrons are filled in order.  Returns ``[N]`` nucleus
    index per electron (spin-sorted order: up electrons first).
    """
    slots = []
    for I, z in enumerate(system.Z):
        slots += [I] * int(round(z))
    N = system.n_elec
    if len(slots) < N:  # charged systems: wrap around
        slots += [slots[k % len(slots)] for k in range(N - len(slots))]
    slots = slots[:N]
    up, dn = [], []
    want_up = True
    for s in slots:
        if (want_up and len(up) < system.n_up) or len(dn) >= system.n_down:
            up.append(s)
        else:
            dn.append(s)
        want_up = not want_up
    return np.array(up + dn, dtype=np.int64)


def init_walkers(system, B, seed, sigma=1.0, walker_offset=0):
    """Initial walkers ``r[B][N][3]`` (FP64): N(R_slot, sigma^2) per electron."""
    N = system.n_elec
    slot = electron_slots(system)
    xi = walker_normals(seed, np.arange(walker_offset, walker_offset + B), 0, TAG_INIT, 3 * N)
    return system.R[slot][None, :, :] + sigma * xi.reshape(B, N, 3)


def metropolis_draws(seed, B, N, step, walker_offset=0):
    """Proposal normals ``xi[B][N][3]`` and acceptance uniforms ``u[B]`` of one
    Metropolis step with global index ``step``."""
    w = np.arange(walker_offset, walker_offset + B)
    xi = walker_normals(seed, w, step, TAG_PROPOSE, 3 * N).reshape(B, N, 3)
    u = walker_uniform(seed, w, step, TAG_ACCEPT)
    return xi, u


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    system: System
    cfg: AnsatzCfg
    B: int
    param_seed: int
    walker_seed: int
    precision: str
    extra: dict = field(default_factory=dict)


def workload(name):
    """The benchmark workloads by name (molecule, ansatz size, walkers)."""
    if name == "lih_fp64":  # LiH, D=32, L=2, K=1, 512 walkers, seed 0
        return Workload(name, molecule("LiH"), AnsatzCfg(32, 2, 1), 512, 0, 0, "fp64",
                        {"mcmc_steps": 10, "step_size": 0.2})
    if name == "n2_fp32":  # N2, D=128, L=3, K=16, 4096 walkers, seed 1
        return Workload(name, molecule("N2"), AnsatzCfg(128, 3, 16), 4096, 1, 1, "fp32",
                        {"mcmc_steps": 1, "step_size": 0.2})
    if name == "n2_bf16":  # the N2 workload with the BF16 embedding GEMMs
        return Workload(name, molecule("N2"), AnsatzCfg(128, 3, 16), 4096, 1, 1, "bf16",
                        {"mcmc_steps": 1, "step_size": 0.2})
    if name == "c4h4_bf16":  # C4H4, D=256, L=4, K=32, 8192 walkers
        return Workload(name, molecule("C4H4"), AnsatzCfg(256, 4, 32), 8192, 3, 3, "bf16")
    raise KeyError(name)


BATCH_MOLECULES = (("H2O", 8192), ("NH3", 8192), ("C2H4", 4096), ("C6H6", 2048))


def batch_workload(name="mixed_fp32"):
    """Molecules with uneven electron counts (10, 10, 16, 42) that run as one batch:
    each D=128, L=3, K=8, parameters and walkers from seed 4, its own walker count."""
    prec = {"mixed_fp32": "fp32", "mixed_bf16": "bf16"}[name]
    cfg = AnsatzCfg(128, 3, 8)
    return [Workload(f"{m.lower()}_{prec}", molecule(m), cfg, B, 4, 4, prec) for m, B in BATCH_MOLECULES]


def synthetic_pseudopotential(l_max=2, seed=0):
    """Stand-in coefficients of a pseudopotential (no ccECP / BFD tables here): for the local
    function V and the channels W_0 .. W_lmax, two Gaussian terms (beta, n, alpha) each, of the
    magnitudes such tables have (a few hartree, exponents 0.5 - 5 bohr^-2)."""
    rng = np.random.default_rng(seed)
    coef = np.zeros((l_max + 2, 2, 3))
    coef[0] = [(-rng.uniform(1, 3), 1, rng.uniform(0.5, 2)), (rng.uniform(0.5, 2), 2, rng.uniform(1, 5))]
    for l in range(l_max + 1):
        coef[1 + l] = [(rng.uniform(1, 6), 2, rng.uniform(0.5, 3)), (-rng.uniform(0.2, 1), 2, rng.uniform(2, 5))]
    return coef


def random_rotations(B, seed):
    """B orthogonal 3 x 3 matrices (QR of Gaussian matrices), the rotations of the quadrature."""
    rng = np.random.default_rng(seed)
    return np.array([np.linalg.qr(rng.standard_normal((3, 3)))[0] for _ in range(B)])
